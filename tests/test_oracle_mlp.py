"""Pins for the oracle's MLP table (Sec. 2; MLP form of Schulte et al. 2008).

Each check uses something other than the oracle itself: the exact
relativistic value of 1/(beta^2 p^2), numpy's Gauss-Legendre rule, closed-form
polynomial integrals, the Gaussian-conditioning (Kalman / Woodbury) form of the
same estimator, exact invariances of any linear path estimator, and the cubic
Hermite interpolant that the MLP reduces to when scattering power is constant.
"""
import math

import numpy as np
import pytest

from paper_1707_05014_gb300 import synthetic as S

GRIDS = [S.Grid(32, 32, 32, 2.0, 2.0, 2.0), S.Grid(160, 160, 64, 1.25, 1.25, 1.25), S.Grid(200, 200, 48, 1.0, 1.0, 2.0)]

# Schulte et al. 2008 water polynomial (MeV^-2 cm^-i), restated for the
# independent closed-form route below.
POLY = np.array([7.457e-6, 4.548e-7, -5.777e-8, 1.301e-8, -9.228e-10, 2.687e-11])
E0, X0 = 13.6, 36.08


def test_entry_value_matches_relativistic_kinematics(oracle):
    # 1/(beta^2 p^2) at T = 200 MeV from E = T + m, p^2 = E^2 - m^2, beta = p/E.
    m, T = 938.272, 200.0
    E = T + m
    p2 = E * E - m * m
    exact = 1.0 / (p2 / (E * E) * p2)
    assert abs(oracle.inv_beta2p2(0.0) / exact - 1.0) < 0.01
    # the energy loss makes 1/(beta^2 p^2) grow monotonically with depth
    w = np.linspace(0, 20, 81)
    v = [oracle.inv_beta2p2(x) for x in w]
    assert np.all(np.diff(v) > 0)


def test_energy_polynomial_follows_bethe_stopping_in_water(oracle):
    # Independent physics: integrate the Bethe stopping power of a 200 MeV
    # proton in water (Z/A = 0.5551, I = 75 eV, no shell or density terms)
    # along the depth and form 1/(beta^2 p^2). The fitted polynomial the MLP
    # uses must follow it over the depths the slabs here span (<= 20 cm):
    # within 1 % to 15 cm and 2 % to 20 cm. A wrong order, sign or exponent in
    # any coefficient leaves this band.
    mp, me, K, ZA, I = 938.272, 0.51099895, 0.307075, 0.5551, 75e-6

    def dedx(T):
        g = 1.0 + T / mp
        b2 = 1.0 - 1.0 / (g * g)
        bg2 = b2 * g * g
        tmax = 2 * me * bg2 / (1 + 2 * g * me / mp + (me / mp) ** 2)
        return K * ZA / b2 * (0.5 * math.log(2 * me * bg2 * tmax / I**2) - b2)

    T, w, h = 200.0, 0.0, 0.01
    while w <= 20.0 + 1e-9:
        E = T + mp
        p2 = E * E - mp * mp
        ref = 1.0 / (p2 / (E * E) * p2)
        rel = abs(oracle.inv_beta2p2(w) / ref - 1.0)
        assert rel < (0.01 if w <= 15.0 else 0.02), (w, rel)
        k1 = -dedx(T)
        k2 = -dedx(T + 0.5 * h * k1)
        k3 = -dedx(T + 0.5 * h * k2)
        k4 = -dedx(T + h * k3)
        T += h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        w += h


def test_gauss_legendre_matches_numpy(oracle):
    for n in (8, 33, 64):
        x, w = oracle.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.abs(x - xr).max() < 1e-14
        assert np.abs(w - wr).max() < 1e-14


def _closed_moment(a, b, c, m, const=False):
    """integral over [a, b] of (c - w)^m f(w) with f the polynomial above,
    exactly, after the substitution s = c - w (no cancellation for c = b)."""
    f = np.polynomial.Polynomial(POLY[:1] if const else POLY)
    g = np.polynomial.Polynomial([0.0] * m + [1.0]) * f(np.polynomial.Polynomial([c, -1.0]))
    G = g.integ()
    return G(c - a) - G(c - b)


@pytest.mark.parametrize("m", [0, 1, 2])
def test_quadrature_equals_closed_form(oracle, m):
    W = 20.0
    for w1 in (0.05, 0.3, 5.0, 12.5, 19.9):
        for (a, b, c) in ((0.0, w1, w1), (w1, W, W)):
            ref = _closed_moment(a, b, c, m)
            got = oracle.moment(a, b, c, m)
            assert abs(got - ref) <= 1e-13 * abs(ref)


def _kalman_table(g):
    """MLP coefficients by Gaussian conditioning: y1 = R0 y0 + n1,
    y2 = R1 y1 + n2 gives E[y1 | y0, y2] = R0 y0 + S1 R1^T C^-1 (y2 - R1 R0 y0)
    with C = R1 S1 R1^T + S2 (closed-form moments)."""
    R = g.radius
    step = min(g.hx, g.hy, g.hz) / 2
    K = int(math.ceil(2 * R / step - 1e-9))
    du = 2 * R / K
    W = 2 * R / 10.0
    out = np.zeros((K + 1, 4))
    out[0] = (1, 0, 0, 0)
    out[K] = (0, 0, 1, 0)
    hl = lambda L: E0 * E0 * (1 + 0.038 * math.log(L / X0)) ** 2 / X0  # noqa: E731
    for k in range(1, K):
        w1 = k * du / 10.0
        S1 = hl(w1) * np.array([[_closed_moment(0, w1, w1, 2), _closed_moment(0, w1, w1, 1)],
                                [_closed_moment(0, w1, w1, 1), _closed_moment(0, w1, w1, 0)]])
        S2 = hl(W - w1) * np.array([[_closed_moment(w1, W, W, 2), _closed_moment(w1, W, W, 1)],
                                    [_closed_moment(w1, W, W, 1), _closed_moment(w1, W, W, 0)]])
        R0 = np.array([[1.0, w1], [0.0, 1.0]])
        R1 = np.array([[1.0, W - w1], [0.0, 1.0]])
        C = R1 @ S1 @ R1.T + S2
        G = S1 @ R1.T @ np.linalg.inv(C)
        A0 = (np.eye(2) - G @ R1) @ R0
        out[k] = (A0[0, 0], 10 * A0[0, 1], G[0, 0], 10 * G[0, 1])
    return out


@pytest.mark.parametrize("gi", [0, 1, 2])
def test_table_equals_conditioning_form(oracle, gi):
    g = GRIDS[gi]
    tab = oracle.mlp_table(g)
    ref = _kalman_table(g)
    scale = np.array([1.0, 2 * g.radius, 1.0, 2 * g.radius])
    assert np.abs((tab - ref) / scale).max() < 1e-12


@pytest.mark.parametrize("gi", [0, 1, 2])
def test_table_invariances(oracle, gi):
    # Translation invariance (shifting t0 and t2 by c shifts every node by c):
    # c1 + c3 = 1. Straight-line invariance (t = a + s (u - u0) reproduced
    # exactly): c2 + c3 (u2 - u0) + c4 = u_k - u0.
    g = GRIDS[gi]
    R, du, K, _ = oracle.geom_info(g)
    tab = oracle.mlp_table(g)
    uk = np.arange(K + 1) * du
    assert np.abs(tab[:, 0] + tab[:, 2] - 1.0).max() < 1e-12
    assert np.abs(tab[:, 1] + tab[:, 2] * 2 * R + tab[:, 3] - uk).max() < 1e-12 * 2 * R
    # endpoints take the measurements exactly
    assert tuple(tab[0]) == (1.0, 0.0, 0.0, 0.0)
    assert tuple(tab[K]) == (0.0, 0.0, 1.0, 0.0)


@pytest.mark.parametrize("gi", [0, 1])
def test_depth_reversal_with_constant_scattering(oracle, gi):
    # With scattering power independent of depth, running the slab backwards
    # maps the estimator onto itself: c1(u) = c3(L - u), c2(u) = -c4(L - u).
    g = GRIDS[gi]
    _, _, K, _ = oracle.geom_info(g)
    tab = oracle.mlp_table(g, flags=oracle.F_CONST_SCATTER)
    rev = tab[::-1]
    L = 2 * g.radius
    assert np.abs(tab[:, 0] - rev[:, 2]).max() < 1e-12
    assert np.abs(tab[:, 1] + rev[:, 3]).max() < 1e-12 * L
    # with the real (depth dependent) scattering the symmetry is broken
    real = oracle.mlp_table(g)
    assert np.abs(real[:, 0] - real[::-1, 2]).max() > 1e-3


@pytest.mark.parametrize("gi", [0, 1])
def test_constant_scattering_is_cubic_hermite(oracle, gi):
    # Constant scattering power and a fixed Highland factor make the slope a
    # Brownian motion; conditioned on both end states its mean path is the
    # cubic Hermite interpolant of (t0, st0) and (t2, st2).
    g = GRIDS[gi]
    _, _, K, _ = oracle.geom_info(g)
    tab = oracle.mlp_table(g, flags=oracle.F_CONST_SCATTER | oracle.F_NO_LOG)
    L = 2 * g.radius
    s = np.arange(K + 1) / K
    ref = np.stack([2 * s**3 - 3 * s**2 + 1, L * (s**3 - 2 * s**2 + s), -2 * s**3 + 3 * s**2, L * (s**3 - s**2)], 1)
    assert np.abs(tab - ref).max() < 1e-12 * L


def test_fp32_nodes_close_to_fp64(oracle):
    # The single-precision node order differs from the FP64 nodes by rounding
    # only: at most 1e-4 voxel (the stated precision budget of the nodes).
    wl = S.head_workload(2000)
    rec = S.make_histories(wl)
    n32 = oracle.nodes(wl.grid, rec, mode=oracle.MODE_FP32).astype(np.int64)
    n64 = oracle.nodes(wl.grid, rec, mode=oracle.MODE_FP64).astype(np.int64)
    err = np.abs(n32 - n64) / 2.0**20
    assert err.max() < 1e-4
    assert np.sqrt((err**2).mean()) < 2e-5


def test_straight_measurement_gives_straight_nodes(oracle):
    # A consistent straight record (exit = entry + 2R slope, equal slopes)
    # yields nodes on that line for any depth dependence of the scattering.
    g = GRIDS[1]
    R, du, K, _ = oracle.geom_info(g)
    rec = S.straight_records(g, [10.0, -33.0], [5.0, -12.0], [0.02, -0.01], [0.0, 0.015], [0.3, 2.0])
    q = oracle.nodes(g, rec, mode=oracle.MODE_FP64).astype(np.float64) / 2.0**20
    for i in range(2):
        c, s = float(rec["cphi"][i]), float(rec["sphi"][i])
        u = -R + np.arange(K + 1) * du
        t = float(rec["t0"][i]) + float(rec["st0"][i]) * (u + R)
        v = float(rec["v0"][i]) + float(rec["sv0"][i]) * (u + R)
        ref = np.stack([(u * c - t * s) / g.hx + g.nx / 2, (u * s + t * c) / g.hy + g.ny / 2, v / g.hz + g.nz / 2], 1)
        assert np.abs(q[i] - ref).max() < 5e-6


@pytest.mark.slow
@pytest.mark.parametrize("layer", ["slab", "hull_layer"])
def test_table_is_the_conditional_mean_of_a_simulated_scattering_walk(oracle, layer):
    # Independent of the estimator's formula: simulate lateral multiple
    # scattering as a random walk whose slope variance grows at a rate
    # proportional to 1/(beta^2 p^2)(depth) (the same energy polynomial, pinned
    # above), draw 200k walks across the 200 mm slab of the head grid, and
    # regress the position at interior nodes on (t0, s0, t2, s2). For this
    # Gaussian process the conditional mean is linear in the four measurements
    # and the regression recovers it, so the coefficients must match the
    # oracle's table without the Highland log term (the log term depends on
    # the whole sub-path length and is not a property of such a walk) within a
    # few standard errors; the table with scattering held at its entry value
    # must not (it is off by about a hundred standard errors).
    # The hull layer case: a water layer of 150 node intervals (93.75 mm) that
    # the proton enters at its first node, with depth counted from there.
    g = S.Grid(160, 160, 8, 1.25, 1.25, 1.25)
    R, du, K, _ = oracle.geom_info(g)
    if layer == "slab":
        tab = oracle.mlp_table(g, flags=oracle.F_NO_LOG)
        flat = oracle.mlp_table(g, flags=oracle.F_NO_LOG | oracle.F_CONST_SCATTER)
    else:
        K = 150
        R = K * du / 2
        tab = oracle.mlp_table_n(g, K, flags=oracle.F_NO_LOG)
        flat = oracle.mlp_table_n(g, K, flags=oracle.F_NO_LOG | oracle.F_CONST_SCATTER)
    rng = np.random.Generator(np.random.Philox(7))
    n = 200_000
    t0, s0 = rng.normal(0.0, 1.0, n), rng.normal(0.0, 0.01, n)
    t, s = t0.copy(), s0.copy()
    q0, f0 = 1e-4 / (2 * R), oracle.inv_beta2p2(0.0)
    probe = (K // 4, K // 2, 3 * K // 4)
    at = {}
    for k in range(K):
        # one exact step of ds = sqrt(q) dW, dt = s du over du, with q taken at
        # the step's mid-depth (it changes by < 1 % over a step)
        q = q0 * oracle.inv_beta2p2((k + 0.5) * du / 10.0) / f0
        z1, z2 = rng.standard_normal(n), rng.standard_normal(n)
        t += s * du + math.sqrt(q * du**3) * (0.5 * z1 + z2 / math.sqrt(12.0))
        s += math.sqrt(q * du) * z1
        if k + 1 in probe:
            at[k + 1] = t.copy()
    X = np.stack([t0, s0, t, s], axis=1)
    worst_flat = 0.0
    for k in probe:
        c = np.linalg.lstsq(X, at[k], rcond=None)[0]
        resid = at[k] - X @ c
        se = np.sqrt(np.diag(np.linalg.inv(X.T @ X)) * resid.var())
        assert np.all(np.abs(c - tab[k]) <= 5.0 * se), (k, c, tab[k], se)
        worst_flat = max(worst_flat, float(np.max(np.abs(c - flat[k]) / se)))
    assert worst_flat > 30.0


def test_scattering_covariance_follows_the_highland_width(oracle):
    """The slope variance the oracle gives a water slab is the published
    Highland width theta0 = 13.6 MeV / (beta c p) sqrt(L/X0) (1 + 0.038 ln(L/X0)),
    X0 = 36.08 cm: for thin slabs at the 200 MeV entry, with beta and p from the
    relativistic kinematics here (within 2 %: the energy polynomial's entry value
    and the loss across the slab), so the log term's sign and size are pinned;
    and wherever a slab sits, the factor on its 1/(beta p)^2 integral is that of
    its own thickness (the log's argument is the sub-path length, not the depth)."""
    mp, T, X0 = 938.272, 200.0, 36.08
    E = T + mp
    pc = math.sqrt(E * E - mp * mp)
    bcp = pc * pc / E
    for L in (0.05, 0.1, 0.2):
        theta0 = 13.6 / bcp * math.sqrt(L / X0) * (1.0 + 0.038 * math.log(L / X0))
        cov = oracle.scatter_cov(0.0, L)
        assert abs(cov[2] / theta0**2 - 1.0) < 0.02, (L, cov[2], theta0**2)
        # without the log term the variance moves by far more than that
        assert abs(oracle.scatter_cov(0.0, L, flags=oracle.F_NO_LOG)[2] / theta0**2 - 1.0) > 0.5
    for a, L in ((0.0, 1.0), (8.0, 1.0), (15.0, 1.0), (3.0, 5.0)):
        cov = oracle.scatter_cov(a, a + L)
        factor = cov[2] / oracle.moment(a, a + L, a + L, 0)
        want = 13.6**2 * (1.0 + 0.038 * math.log(L / X0)) ** 2 / X0
        assert abs(factor / want - 1.0) < 1e-12, (a, L)
        # the position terms are the first and second moments about the exit
        assert abs(cov[1] / cov[2] - oracle.moment(a, a + L, a + L, 1) / oracle.moment(a, a + L, a + L, 0)) < 1e-12
