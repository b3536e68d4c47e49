"""Warm-start network kernels (tensor-core implicit GEMMs) against the FP64
reference oracle/unet.py: forward output, every parameter gradient, and a
training run that lowers the loss.

Element-wise bounds. The reference with bf16=True rounds weights and every
stored activation and gradient to BF16 where the kernels store them, so the two
sides differ by FP32 summation order, plus the rare stored value that lies
within that summation difference of a BF16 rounding boundary and so rounds to
the neighbouring BF16 value: a change of at most one BF16 ulp, 2^-7 of the
value. A sum of terms each of which changes by at most a relative e changes by
at most e times the sum of the terms' magnitudes. Every output element is held
to BF16_BOUND = 2^-6 (two ulps: both factors of a product may have moved)
times that magnitude sum (forward_scale), plus FP32 rounding.

Gradients. A ReLU decision on a pre-activation within rounding of zero may go
either way on the two sides (a float32 re-run of the reference itself flips a
few dozen per layer), and every gradient term that runs through such a position
is then present on one side only. loss_and_grads(scales=True) returns two
magnitude chains (|dLoss/df| carried back with |W| in place of W): `core`
through the clearly decided positions only, `relaxed` also through every
position whose pre-activation is within RELU_MARGIN = 2^-6 of its magnitude sum
of zero (the forward bound's own margin). A gradient element of layer L is
held to 2^-7 (nl - L + 1) times the relaxed chain (one ulp per stored gradient
on the way back, plus the stored activation it multiplies) plus relaxed - core
(the terms that a flipped decision may add or remove). Near the output the
chains coincide and the bound is tight; towards the input the flipped terms
fan out and the bound loosens accordingly. The loss gradient sign(x0 - target)/n
is itself a decision: the test's targets sit at least 0.05 from the reference's
x0, far outside the forward bound, so that both sides take the same sign."""
import numpy as np
import pytest

from oracle import unet as U

pytestmark = pytest.mark.gpu

SHAPE = (8, 16, 24)


@pytest.fixture(scope="module")
def P():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1707_05014_gb300 import build
    from paper_1707_05014_gb300 import pct

    build.build()
    return pct


def _data(seed=0):
    rng = np.random.Generator(np.random.Philox(seed))
    x1 = rng.random(SHAPE) * 1.5
    target = x1 + 0.2 * rng.standard_normal(SHAPE)
    p = U.init_params(seed + 1)
    off = 0
    for ci, co, _, _ in U.SPEC:  # small non-zero biases
        off += 27 * ci * co
        p[off:off + co] = 0.05 * rng.standard_normal(co)
        off += co
    return x1, target, p.astype(np.float32).astype(np.float64)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_param_layout_matches_reference(P):
    with P.Net(*SHAPE) as net:
        assert net.n_params == U.param_count()
        p = net.get_params()
        assert np.all(np.isfinite(p))


BF16_BOUND = 2.0**-6
FP32_FLOOR = 1e-6  # FP32 rounding of the sums, relative to their magnitude sum
RELU_MARGIN = 2.0**-6  # a pre-activation this close to zero (relative) may take either ReLU decision


@pytest.mark.parametrize("seed", [1, 3])
def test_forward_matches_reference(P, seed):
    import torch

    x1, _, p = _data(seed)
    x1 = x1.astype(np.float32).astype(np.float64)
    with P.Net(*SHAPE) as net:
        net.set_params(p)
        x0 = net.forward(torch.tensor(x1.ravel(), dtype=torch.float32, device="cuda")).cpu().numpy()
    ref16, _ = U.forward(p, x1, bf16=True)
    ref64, _ = U.forward(p, x1, bf16=False)
    f_gpu = x0.astype(np.float64) - x1.ravel().astype(np.float32)
    f16 = (ref16 - x1).ravel()
    scale = U.forward_scale(p, x1, bf16=True).ravel()
    # element by element against the BF16-emulating reference
    bound = (BF16_BOUND + FP32_FLOOR) * scale + 2.0**-23 * np.abs(x1.ravel())
    bad = np.abs(f_gpu - f16) > bound
    assert not bad.any(), (int(bad.sum()), float((np.abs(f_gpu - f16) / scale).max()))
    # and, as a whole, close to the FP64 network without BF16 storage
    assert _rel(f_gpu, (ref64 - x1).ravel()) < 5e-2


@pytest.mark.parametrize("seed", [2, 5])
def test_gradients_match_reference(P, seed):
    import torch

    x1, _, p = _data(seed)
    x1 = x1.astype(np.float32).astype(np.float64)
    # targets away from the reference output: the loss gradient's sign is the same on both sides
    rng = np.random.Generator(np.random.Philox(100 + seed))
    x0_ref, _ = U.forward(p, x1, bf16=True)
    sgn = np.where(rng.random(SHAPE) < 0.5, -1.0, 1.0)
    target = (x0_ref + sgn * (0.05 + 0.2 * rng.random(SHAPE))).astype(np.float32).astype(np.float64)
    with P.Net(*SHAPE) as net:
        net.set_params(p)
        loss, g = net.gradients(torch.tensor(x1.ravel(), dtype=torch.float32, device="cuda"),
                                torch.tensor(target.ravel(), dtype=torch.float32, device="cuda"))
    rloss, rg, core, rel = U.loss_and_grads(p, x1, target, bf16=True, scales=True, relu_margin=RELU_MARGIN)
    assert abs(loss - rloss) < 1e-3 * rloss
    off = 0
    nl = len(U.SPEC)
    worst = []
    for li, (ci, co, _, _) in enumerate(U.SPEC):
        n = 27 * ci * co + co
        a, b = g[off:off + n].astype(np.float64), rg[off:off + n]
        sc, sr = core[off:off + n], rel[off:off + n]
        # every weight and bias gradient of the layer, element by element
        bound = (2.0**-7 * (nl - li + 1) + FP32_FLOOR) * sr + (sr - sc) + 1e-30
        worst.append(float(np.max(np.abs(a - b) / bound)))
        off += n
    assert max(worst) <= 1.0, worst


def test_training_lowers_the_loss(P):
    import torch

    rng = np.random.Generator(np.random.Philox(9))
    x1 = rng.random(SHAPE).astype(np.float32)
    # target: a smoothed copy (what the warm start learns: denoise/deblur)
    t = x1.copy()
    for ax in range(3):
        t = (np.roll(t, 1, ax) + t + np.roll(t, -1, ax)) / 3.0
    dx1 = torch.tensor(x1.ravel(), device="cuda")
    dt = torch.tensor(t.ravel(), device="cuda")
    with P.Net(*SHAPE, seed=4) as net:
        l0 = net.train_step(dx1, dt, lr=2e-3)
        for _ in range(150):
            net.train_step(dx1, dt, lr=2e-3, want_loss=False)
        l1 = net.train_step(dx1, dt, lr=2e-3)
    assert l1 < 0.5 * l0


def _bf16_bits(a):
    """float64 values already on the BF16 grid -> int16 CUDA tensor of bits."""
    import torch

    u = (np.asarray(a, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)
    return torch.from_numpy(u.view(np.int16).ravel().copy()).cuda()


def _from_bf16_bits(t, shape):
    u = t.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    return u.view(np.float32).astype(np.float64).reshape(shape)


@pytest.mark.parametrize("seed", [4])
def test_every_layer_matches_reference_element_wise(P, seed):
    """Each layer's forward, data gradient and weight gradient on the same
    seeded BF16 inputs on both sides (oracle/unet.py layer_*): the stored
    results differ by the FP32 summation order (at most K 2^-24 of the
    magnitude sum for K summed terms) plus one BF16 ulp (2^-7) of the value
    where that difference crosses a rounding boundary; the FP32 weight
    gradients by the summation order alone. A wrong halo row, tap, stride or
    skip changes elements by O(1) of their magnitude."""
    rng = np.random.Generator(np.random.Philox(200 + seed))
    _, _, p = _data(seed)
    D, H, W = SHAPE
    nl = len(U.SPEC)
    worst = {}
    with P.Net(*SHAPE) as net:
        net.set_params(p)
        for li, (ci, co, kind, skip) in enumerate(U.SPEC):
            _, _, lin, lout = net.layer_shape(li)
            din = (D >> lin, H >> lin, W >> lin, ci)
            dout = (D >> lout, H >> lout, W >> lout, co)
            h = U.to_bf16(np.maximum(rng.standard_normal(din), 0.0))
            dy = U.to_bf16(1e-3 * rng.standard_normal(dout))
            taps = 27 * ci
            if li < nl - 1:
                sk = U.to_bf16(np.maximum(rng.standard_normal(dout), 0.0)) if skip >= 0 else None
                ref, mag = U.layer_forward(p, li, h, sk)
                got = _from_bf16_bits(net.layer(li, P.NET_FORWARD, inp=_bf16_bits(h),
                                                skip=None if sk is None else _bf16_bits(sk)), dout)
                bound = 2.0**-7 * np.abs(ref) * 1.01 + 2 * (taps + 2) * 2.0**-24 * mag + 1e-30
                worst[(li, "fwd")] = float((np.abs(got - ref) / bound).max())
            if li > 0:
                mask = U.to_bf16(np.maximum(rng.standard_normal(din), 0.0))
                adds = [u for u, s in enumerate(U.SPEC) if s[3] == li - 1]
                ad = U.to_bf16(1e-3 * rng.standard_normal(din)) if adds and kind != "up" else None
                ref, mag = U.layer_data_grad(p, li, dy, mask, ad)
                got = _from_bf16_bits(net.layer(li, P.NET_DATA_GRAD, dy=_bf16_bits(dy), mask=_bf16_bits(mask),
                                                add=None if ad is None else _bf16_bits(ad)), din)
                terms = 27 * co * (8 if kind == "up" else 1) + 2
                bound = 2.0**-7 * np.abs(ref) * 1.01 + 2 * terms * 2.0**-24 * mag + 1e-30
                worst[(li, "dgrad")] = float((np.abs(got - ref) / bound).max())
            ref, mag = U.layer_weight_grad(li, h, dy)
            got = net.layer(li, P.NET_WEIGHT_GRAD, inp=_bf16_bits(h), dy=_bf16_bits(dy)).cpu().numpy()
            vox = dout[0] * dout[1] * dout[2]
            bound = 2 * (vox + 32) * 2.0**-24 * mag + 1e-30
            worst[(li, "wgrad")] = float((np.abs(got.astype(np.float64) - ref) / bound).max())
    bad = {k: v for k, v in worst.items() if v > 1.0}
    assert not bad, bad
