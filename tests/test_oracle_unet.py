"""Pins for the FP64 reference of the warm-start network (oracle/unet.py):
convolution against scipy's correlate, exact adjoint (dot-product) identities
for every linear step, and the full gradient against central differences."""
import numpy as np
import pytest

from oracle import unet as U


def test_conv_matches_scipy_correlate():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.Generator(np.random.Philox(1))
    x = rng.standard_normal((6, 7, 5, 1))
    W = rng.standard_normal((27, 1, 1))
    y = U.conv(x, W, np.zeros(1), 1)[..., 0]
    k = W[:, 0, 0].reshape(3, 3, 3)
    ref = ndimage.correlate(x[..., 0], k, mode="constant", cval=0.0)
    assert np.abs(y - ref).max() < 1e-12


def test_stride2_is_subsampled_stride1_and_up_is_repeat():
    rng = np.random.Generator(np.random.Philox(2))
    x = rng.standard_normal((8, 6, 4, 3))
    W = rng.standard_normal((27, 3, 2))
    b = rng.standard_normal(2)
    assert np.abs(U.conv(x, W, b, 2) - U.conv(x, W, b, 1)[::2, ::2, ::2]).max() < 1e-12
    u = U.up2(x)
    assert u.shape == (16, 12, 8, 3) and np.array_equal(u[1::2, ::2, 1::2], x)


@pytest.mark.parametrize("stride", [1, 2])
def test_adjoints(stride):
    rng = np.random.Generator(np.random.Philox(3 + stride))
    x = rng.standard_normal((8, 6, 4, 3))
    W = rng.standard_normal((27, 3, 5))
    y = U.conv(x, W, np.zeros(5), stride)
    g = rng.standard_normal(y.shape)
    lhs = float((y * g).sum())
    assert abs(lhs - float((x * U.conv_adjoint(x.shape, g, W, stride)).sum())) < 1e-9 * abs(lhs)
    assert abs(lhs - float((W * U.conv_wgrad(x, g, stride)).sum())) < 1e-9 * abs(lhs)
    u = rng.standard_normal((4, 3, 2, 3))
    v = rng.standard_normal((8, 6, 4, 3))
    assert abs(float((U.up2(u) * v).sum()) - float((u * U.down2_sum(v)).sum())) < 1e-9


def test_gradient_matches_central_differences():
    rng = np.random.Generator(np.random.Philox(7))
    p = U.init_params(3)
    p += 0.01 * rng.standard_normal(p.size) * (p != 0)
    # non-zero biases so every layer's bias gradient is exercised
    off = 0
    for ci, co, _, _ in U.SPEC:
        off += 27 * ci * co
        p[off:off + co] = 0.05 * rng.standard_normal(co)
        off += co
    x1 = rng.random((8, 16, 8))
    target = x1 + 0.3 * rng.standard_normal(x1.shape)
    loss, g = U.loss_and_grads(p, x1, target)
    # probe parameters with a clear gradient in every layer
    offs, o = [], 0
    for ci, co, _, _ in U.SPEC:
        offs.append((o, 27 * ci * co + co))
        o += 27 * ci * co + co
    idx = []
    for lo, n in offs:
        seg = np.abs(g[lo:lo + n])
        idx.extend(lo + np.argsort(seg)[-2:])
    eps = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = eps
        fd = (U.loss_and_grads(p + e, x1, target)[0] - U.loss_and_grads(p - e, x1, target)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-4 * abs(g[i]) + 1e-9, (i, fd, g[i])


def test_bf16_rounding_is_round_half_even():
    v = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-9, -2.5, 3.0e38])
    r = U.to_bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0  # tie to even
    assert r[2] == 1.0 + 2**-7 and r[3] == -2.5


def test_gradient_bound_scales_bound_the_gradient():
    """The magnitude chains of loss_and_grads(scales=True): core <= relaxed
    everywhere, the two coincide when no position is ambiguous (margin 0 on
    FP64 data, where no pre-activation is exactly zero), and each gradient
    element is at most its relaxed chain (|sum of terms| <= sum of |terms|;
    BF16 storage may round a stored gradient up by 2^-9 of itself per layer)."""
    rng = np.random.Generator(np.random.Philox(12))
    p = U.init_params(5)
    off = 0
    for ci, co, _, _ in U.SPEC:
        off += 27 * ci * co
        p[off:off + co] = 0.05 * rng.standard_normal(co)
        off += co
    x1 = rng.random((8, 8, 16))
    target = x1 + 0.3 * rng.standard_normal(x1.shape)
    for bf16 in (False, True):
        loss, g, core, rel = U.loss_and_grads(p, x1, target, bf16=bf16, scales=True, relu_margin=2.0**-6)
        assert np.all(core >= 0) and np.all(core <= rel)
        slack = (1.0 + 2.0**-8) ** len(U.SPEC) if bf16 else 1.0 + 1e-12
        assert np.all(np.abs(g) <= rel * slack + 1e-300)
        assert (rel > core).any()  # some positions are ambiguous at this margin
        _, g0, core0, rel0 = U.loss_and_grads(p, x1, target, bf16=bf16, scales=True, relu_margin=0.0)
        assert np.array_equal(g0, g)
        assert np.allclose(core0, rel0, rtol=1e-12, atol=0)


def test_layer_functions_chain_to_the_network():
    """The per-layer functions (the GPU's per-layer check uses them) chained
    over the topology give the whole network's forward output and every
    parameter gradient exactly (BF16 storage on)."""
    rng = np.random.Generator(np.random.Philox(13))
    p = U.init_params(6)
    off = 0
    for ci, co, _, _ in U.SPEC:
        off += 27 * ci * co
        p[off:off + co] = 0.05 * rng.standard_normal(co)
        off += co
    x1 = rng.random((8, 8, 16))
    target = x1 + 0.3 * rng.standard_normal(x1.shape)
    x0, c = U.forward(p, x1, bf16=True)
    h = c["inp"]
    acts = []
    for li, (_, _, _, skip) in enumerate(U.SPEC[:-1]):
        h, mag = U.layer_forward(p, li, h, acts[skip] if skip >= 0 else None)
        assert np.array_equal(h, c["acts"][li]) and np.all(mag >= 0)
        acts.append(h)
    _, g = U.loss_and_grads(p, x1, target, bf16=True)
    nl = len(U.SPEC)
    df = np.zeros(x0.shape + (16,))
    df[..., 0] = np.sign(x0 - target) / x0.size
    gpre = [None] * nl
    gpre[nl - 1] = U.to_bf16(df)
    offs = np.cumsum([0] + [27 * ci * co + co for ci, co, _, _ in U.SPEC])
    for li in range(nl - 1, -1, -1):
        hin = c["inp"] if li == 0 else acts[li - 1]
        gw, mw = U.layer_weight_grad(li, hin, gpre[li])
        assert np.array_equal(gw, g[offs[li]:offs[li + 1]]) and np.all(np.abs(gw) <= mw + 1e-300)
        if li == 0:
            break
        adds = [gpre[u] for u, (_, _, _, skip) in enumerate(U.SPEC) if skip == li - 1]
        gpre[li - 1], md = U.layer_data_grad(p, li, gpre[li], acts[li - 1], adds[0] if adds else None)
        assert np.all(md >= 0)
