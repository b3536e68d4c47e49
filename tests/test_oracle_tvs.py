"""Pins for the oracle's total-variation superiorization (Sec. 4.2): the TV
gradient against central differences, a constant image as the minimum, no
perturbation ever raising TV, and beta0 = 0 reducing to the plain solvers."""
import numpy as np

from paper_1707_05014_gb300 import synthetic as S


def test_tv_gradient_matches_central_differences(oracle):
    g = S.Grid(5, 4, 3, 1.0, 1.0, 1.0)
    rng = np.random.Generator(np.random.Philox(3))
    x = rng.random(g.m)
    gr = oracle.tv_grad(g, x, eps=1e-2)
    for v in range(g.m):
        e = np.zeros(g.m)
        e[v] = 1e-6
        fd = (oracle.tv_value(g, x + e, 1e-2) - oracle.tv_value(g, x - e, 1e-2)) / 2e-6
        assert abs(fd - gr[v]) < 1e-6


def test_constant_image_is_the_minimum(oracle):
    g = S.Grid(6, 5, 4, 1.0, 1.0, 1.0)
    x = np.full(g.m, 1.04)
    assert abs(oracle.tv_value(g, x, 1e-3) - g.m * 1e-3) < 1e-12
    assert np.abs(oracle.tv_grad(g, x, 1e-3)).max() == 0.0


def test_tvs_never_raises_tv_and_reduces_to_plain_solvers(oracle):
    wl = S.tiny_workload(6000, seed=91)
    g = wl.grid
    rec = S.make_histories(wl)
    for carp in (0, 3):
        plain = oracle.carp(g, rec, 3, 2) if carp else oracle.drop(g, rec, 3, 2)
        same = oracle.solve_tvs(g, rec, 3, 2, carp=carp, beta0=0.0)
        assert np.abs(same - plain).max() <= 1e-12 * max(1.0, np.abs(plain).max())
        sup = oracle.solve_tvs(g, rec, 3, 2, carp=carp, beta0=0.05)
        assert oracle.tv_value(g, sup) < oracle.tv_value(g, plain)  # smoother (Sec. 4.2)
