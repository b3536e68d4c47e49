"""Pins for the oracle's DROP solver (Sec. 2.1, Fig. 1).

* B = 1: the fixed point of x <- x + lam S^-1 A^T W (b - A x) satisfies
  A^T W (b - A x) = 0, so DROP converges to the weighted least-squares
  solution, which a dense Cholesky/lstsq solve gives independently.
* One proton per block with lam = 1 is a Kaczmarz (ART) projection: right
  after its block a proton's residual is exactly zero.
* Consistent data (b = A x_true): the residual falls towards zero and the
  image approaches x_true.
"""
import numpy as np
import pytest

from paper_1707_05014_gb300 import synthetic as S


def _tiny():
    g = S.Grid(4, 4, 2, 2.0, 2.0, 2.0)
    wl = S.Workload("tiny442", g, 200, 21, 0, 4.0, 2.0, 1, 1, "water")
    rec = S.make_histories(wl)
    rec["wepl"] = (np.random.Generator(np.random.Philox(5)).random(200) * 8.0).astype(np.float32)
    return g, rec


def _dense(oracle, g, rec):
    rp, vox, ln = oracle.rows(g, rec)
    n = len(rp) - 1
    A = np.zeros((n, g.m))
    nn = np.zeros(n)
    for i in range(n):
        for j, l in zip(vox[rp[i]:rp[i + 1]], ln[rp[i]:rp[i + 1]]):
            A[i, j] += l
        nn[i] = (ln[rp[i]:rp[i + 1]] ** 2).sum()
    return A, nn


def test_single_block_converges_to_weighted_least_squares(oracle):
    g, rec = _tiny()
    A, nn = _dense(oracle, g, rec)
    keep = nn > 0
    assert np.linalg.matrix_rank(A[keep]) == g.m
    # rows without repeated voxels: |a_i|^2 (sum over runs) is the textbook norm
    assert np.allclose(nn, (A**2).sum(1))
    b = rec["wepl"].astype(np.float64)
    Wh = 1.0 / np.sqrt(nn[keep])
    xs = np.linalg.lstsq(A[keep] * Wh[:, None], b[keep] * Wh, rcond=None)[0]
    x = oracle.drop(g, rec, n_blocks=1, n_sweeps=4000, lam=1.5)
    assert np.abs(x - xs).max() <= 1e-9 * np.abs(xs).max()


def test_one_proton_block_is_an_exact_projection(oracle):
    g, rec = _tiny()
    for n in (1, 2, 7):
        r = S.subset(rec, slice(0, n))
        x = oracle.drop(g, r, n_blocks=n, n_sweeps=1, lam=1.0)
        y = oracle.project(g, r, x)
        assert abs(y[n - 1] - float(r["wepl"][n - 1])) < 1e-12 * max(1.0, float(r["wepl"][n - 1]))
    # lam scales the step: the residual of the last proton becomes (1 - lam) r
    r = S.subset(rec, slice(0, 1))
    x = oracle.drop(g, r, n_blocks=1, n_sweeps=1, lam=0.25)
    y = oracle.project(g, r, x)
    assert abs((float(r["wepl"][0]) - y[0]) - 0.75 * float(r["wepl"][0])) < 1e-12


def test_repeated_proton_block_divides_by_the_run_counts(oracle):
    # A block of m copies of one proton: every voxel of its row has s_j = m,
    # and the m equal contributions a_ij r divided by s_j make one exact
    # projection, so the residual is exactly zero after the block. Without the
    # division the step would be m times too long (residual -(m-1) r).
    g, rec = _tiny()
    for m in (2, 3):
        r = S.subset(rec, np.zeros(m, dtype=np.int64))
        assert np.all(oracle.block_counts(g, r, 1, 0)[oracle.rows(g, r)[1]] == m)
        x = oracle.drop(g, r, n_blocks=1, n_sweeps=1, lam=1.0)
        y = oracle.project(g, r, x)
        assert np.all(np.abs(y - float(r["wepl"][0])) < 1e-12 * max(1.0, float(r["wepl"][0])))


def test_block_counts_are_run_counts(oracle):
    g, rec = _tiny()
    rp, vox, _ = oracle.rows(g, rec)
    for B, b in ((1, 0), (4, 2)):
        lo, hi = b * 200 // B, (b + 1) * 200 // B
        ref = np.bincount(vox[rp[lo]:rp[hi]], minlength=g.m).astype(np.float64)
        assert np.array_equal(oracle.block_counts(g, rec, B, b), ref)


@pytest.mark.parametrize("B", [1, 5])
def test_consistent_data_residual_vanishes(oracle, B):
    wl = S.tiny_workload(4000, seed=3)
    g = wl.grid
    rec = S.make_histories(wl)
    xt = S.voxelize(wl.phantom(), g)
    rec["wepl"] = oracle.project(g, rec, xt).astype(np.float32)
    x, res = oracle.drop(g, rec, B, 30, lam=1.0, return_resid=True)
    assert np.all(np.diff(res[1:]) < 0)
    assert res[-1] < 2e-3 * res[0]


@pytest.mark.slow
def test_noise_free_tiny_workload_converges(oracle):
    # Noise-free consistent data on the 32^3 water cylinder: the mean RSP error
    # over partial-volume-free voxels falls below 1% within 10 sweeps of 100
    # blocks and keeps falling.
    wl = S.tiny_workload(100_000)
    g = wl.grid
    rec = S.make_histories(wl)
    xt = S.voxelize(wl.phantom(), g)
    rec["wepl"] = oracle.project(g, rec, xt).astype(np.float32)
    e5 = S.mean_rsp_error(oracle.drop(g, rec, 100, 5), xt, g)
    e10 = S.mean_rsp_error(oracle.drop(g, rec, 100, 10), xt, g)
    assert e10 < e5
    assert e10 < 0.01


@pytest.mark.slow
def test_noise_free_error_falls_below_a_tenth_of_a_percent(oracle):
    # The same noise-free data run longer: every interior voxel of the water
    # cylinder is crossed by >= 50 runs, and the mean RSP error there falls
    # below 0.1 % by 40 sweeps of 100 blocks (0.85 % at 10, 0.12 % at 30,
    # 0.03 % at 60). The threaded oracle differs from the single-thread one
    # only in the order of its sums.
    wl = S.tiny_workload(100_000)
    g = wl.grid
    rec = S.make_histories(wl)
    xt = S.voxelize(wl.phantom(), g)
    rec["wepl"] = oracle.project(g, rec, xt).astype(np.float32)
    rp, vox, _ = oracle.rows(g, rec)
    m = S.interior_mask(xt, g)
    assert np.all(np.bincount(vox, minlength=g.m)[m] >= 50)
    e20 = S.mean_rsp_error(oracle.drop_threads(g, rec, 100, 20), xt, g)
    e40 = S.mean_rsp_error(oracle.drop_threads(g, rec, 100, 40), xt, g)
    assert e40 < 0.5 * e20
    assert e40 < 1e-3


def test_carp_single_string_is_drop_single_block(oracle):
    g, rec = _tiny()
    a = oracle.drop(g, rec, n_blocks=1, n_sweeps=5, lam=0.7)
    b = oracle.carp(g, rec, n_strings=1, n_sweeps=5, lam=0.7)
    assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(a).max())


@pytest.mark.parametrize("per_string", [1, 3])
def test_carp_is_the_component_average_of_string_sweeps(oracle, per_string):
    # one sweep of CARP from x0 equals, voxel by voxel, the mean of the strings'
    # own DROP sweeps (over their blocks) across the strings that touch the voxel
    g, rec = _tiny()
    S_ = 4
    B = S_ * per_string
    x0 = np.linspace(0.1, 1.0, g.m)
    got = oracle.carp(g, rec, n_strings=S_, n_sweeps=1, x0=x0, n_blocks=B)
    rp, vox, _ = oracle.rows(g, rec)
    num = np.zeros(g.m)
    den = np.zeros(g.m)
    for s in range(S_):
        lo, hi = (s * per_string) * 200 // B, ((s + 1) * per_string) * 200 // B
        xs = oracle.drop(g, S.subset(rec, slice(lo, hi)), n_blocks=per_string, n_sweeps=1, x0=x0)
        touched = np.zeros(g.m, dtype=bool)
        touched[vox[rp[lo]:rp[hi]]] = True
        num[touched] += xs[touched]
        den[touched] += 1
    ref = np.where(den > 0, num / np.maximum(den, 1), x0)
    assert np.abs(got - ref).max() <= 1e-12


def test_carp_consistent_data_residual_decreases(oracle):
    wl = S.tiny_workload(4000, seed=4)
    g = wl.grid
    rec = S.make_histories(wl)
    xt = S.voxelize(wl.phantom(), g)
    rec["wepl"] = oracle.project(g, rec, xt).astype(np.float32)
    x, res = oracle.carp(g, rec, 5, 30, lam=1.0, return_resid=True)
    assert np.all(np.diff(res[1:]) < 0)
    assert res[-1] < 2e-2 * res[0]


def test_threaded_drop_equals_single_thread(oracle):
    # The all-core oracle (histories of a block split over threads, per-thread
    # updates summed in thread order) is the same DROP: only the order of the
    # sums differs. With and without an object hull.
    wl = S.tiny_workload(6000, seed=21)
    g = wl.grid
    rec = S.make_histories(wl)
    hull = (S.voxelize(wl.phantom(), g, ss=1) > 0.5).astype(np.uint8)
    for h in (None, hull):
        a = oracle.drop(g, rec, 4, 2, hull=h)
        b = oracle.drop_threads(g, rec, 4, 2, threads=3, hull=h)
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(a).max())


@pytest.mark.parametrize("n,B", [(200, 3), (157, 7)])
def test_blocks_are_consecutive_ranges_applied_in_sequence(oracle, n, B):
    # Sec. 2.1 / Fig. 1: the image each block produces seeds the next block,
    # and a sweep visits the blocks in order; block b holds histories
    # [b n / B, (b + 1) n / B). One B-block sweep must equal B one-block sweeps
    # over those ranges chained through x0, and two sweeps must chain the same
    # way (a ragged n checks the rounding of the block boundaries).
    g, rec = _tiny()
    rec = S.subset(rec, slice(0, n))
    x = np.zeros(g.m)
    for _ in range(2):
        for b in range(B):
            lo, hi = b * n // B, (b + 1) * n // B
            x = oracle.drop(g, S.subset(rec, slice(lo, hi)), 1, 1, lam=0.8, x0=x)
    ref = oracle.drop(g, rec, B, 2, lam=0.8)
    assert np.abs(ref - x).max() <= 1e-12 * max(1.0, np.abs(x).max())
    # a different split of the same histories gives a different image
    other = oracle.drop(g, rec, B + 1, 2, lam=0.8)
    assert np.abs(other - ref).max() > 1e-6
