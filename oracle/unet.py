"""FP64 numpy reference of the warm-start network (test infrastructure only).

Only the tests import this module. It computes, from the definition, the
network that the library's pct_net_* entry points implement:

  L0: a0 = relu(conv(x1)), a1 = relu(conv(a0))                      16 ch
  L1: b0 = relu(conv_s2(a1)), b1 = relu(conv(b0))                   32 ch
  L2: c0 = relu(conv_s2(b1)), c1 = relu(conv(c0))                   64 ch
  L3: d0 = relu(conv_s2(c1)), d1 = relu(conv(d0))                  128 ch
  u2 = relu(upconv(d1) + c1), e2 = relu(conv(u2))                    64 ch
  u1 = relu(upconv(e2) + b1), e1 = relu(conv(u1))                    32 ch
  u0 = relu(upconv(e1) + a1), e0 = relu(conv(u0))                    16 ch
  f = conv(e0) (channel 0), x0 = x1 + f;  loss = mean |x0 - target|

conv: 3x3x3 cross-correlation with zero padding 1 (stride 1 or 2); upconv:
nearest x2 upsampling then conv. Parameters are one flat vector, per layer
27*Cin*Cout weights [tap][ci][co] (tap = 9 tz + 3 ty + tx) then Cout biases,
channel counts padded to 16 (input channel 0 of layer 0 and output channel 0
of the last layer are the real ones). Gradients are the hand-written
adjoints of each step. ``bf16=True`` rounds weights and every stored
activation / gradient to bfloat16 (round half even) where the GPU kernels
store them, so that GPU and reference differ only by FP32 summation order.
"""
from __future__ import annotations

import numpy as np

# (Cin, Cout, kind, skip source layer or -1)
SPEC = [
    (16, 16, "s1", -1), (16, 16, "s1", -1), (16, 32, "s2", -1), (32, 32, "s1", -1),
    (32, 64, "s2", -1), (64, 64, "s1", -1), (64, 128, "s2", -1), (128, 128, "s1", -1),
    (128, 64, "up", 5), (64, 64, "s1", -1), (64, 32, "up", 3), (32, 32, "s1", -1),
    (32, 16, "up", 1), (16, 16, "s1", -1), (16, 16, "s1", -1),
]


def param_count() -> int:
    return sum(27 * ci * co + co for ci, co, _, _ in SPEC)


def unpack(p: np.ndarray):
    out, off = [], 0
    for ci, co, _, _ in SPEC:
        W = p[off:off + 27 * ci * co].reshape(27, ci, co)
        off += 27 * ci * co
        b = p[off:off + co]
        off += co
        out.append((W, b))
    return out


def to_bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _taps():
    for tz in range(3):
        for ty in range(3):
            for tx in range(3):
                yield tz * 9 + ty * 3 + tx, tz, ty, tx


def conv(x, W, b, stride=1):
    """y[o] = b + sum_t x[stride*o + t - 1] @ W[t] (zero padding 1)."""
    D, H, Wd, _ = x.shape
    Do, Ho, Wo = (D + 2 - 3) // stride + 1, (H + 2 - 3) // stride + 1, (Wd + 2 - 3) // stride + 1
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((Do, Ho, Wo, W.shape[2])) + b
    for t, tz, ty, tx in _taps():
        xs = xp[tz:tz + stride * Do:stride, ty:ty + stride * Ho:stride, tx:tx + stride * Wo:stride, :]
        y += xs @ W[t]
    return y


def conv_adjoint(x_shape, dy, W, stride=1):
    """dx of conv (the transpose of the linear map x -> conv(x, W, 0))."""
    D, H, Wd, C = x_shape
    Do, Ho, Wo, _ = dy.shape
    dxp = np.zeros((D + 2, H + 2, Wd + 2, C))
    for t, tz, ty, tx in _taps():
        dxp[tz:tz + stride * Do:stride, ty:ty + stride * Ho:stride, tx:tx + stride * Wo:stride, :] += dy @ W[t].T
    return dxp[1:-1, 1:-1, 1:-1, :]


def conv_wgrad(x, dy, stride=1):
    D, H, Wd, C = x.shape
    Do, Ho, Wo, Co = dy.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    dW = np.zeros((27, C, Co))
    g = dy.reshape(-1, Co)
    for t, tz, ty, tx in _taps():
        xs = xp[tz:tz + stride * Do:stride, ty:ty + stride * Ho:stride, tx:tx + stride * Wo:stride, :]
        dW[t] = xs.reshape(-1, C).T @ g
    return dW


def up2(x):
    return x.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2)


def down2_sum(x):
    D, H, W, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(1, 3, 5))


def forward(p: np.ndarray, x1: np.ndarray, bf16: bool = False):
    """x1: (D, H, W) -> (x0, cache)."""
    q = (lambda a: to_bf16(a)) if bf16 else (lambda a: a)
    layers = [(q(W), b) for W, b in unpack(p)]
    inp = np.zeros(x1.shape + (16,))
    inp[..., 0] = x1
    inp = q(inp)
    acts = []
    h = inp
    for li, ((ci, co, kind, skip), (W, b)) in enumerate(zip(SPEC, layers)):
        if kind == "s1":
            pre = conv(h, W, b, 1)
        elif kind == "s2":
            pre = conv(h, W, b, 2)
        else:
            pre = conv(up2(h), W, b, 1)
        if skip >= 0:
            pre = pre + acts[skip]
        if li == len(SPEC) - 1:
            f = pre[..., 0]
            x0 = x1 + f
            return x0, {"inp": inp, "acts": acts, "layers": layers, "x1": x1, "x0": x0}
        h = q(np.maximum(pre, 0.0))
        acts.append(h)
    raise AssertionError("unreachable")


def forward_scale(p: np.ndarray, x1: np.ndarray, bf16: bool = False) -> np.ndarray:
    """Per voxel, |b| + sum over taps and channels of |W| |h| of the last layer
    (h its input): the sum of the magnitudes of the terms that make up f. A
    change of every stored input activation by at most a relative e changes f
    by at most e times this scale."""
    _, c = forward(p, x1, bf16)
    W, b = c["layers"][-1]
    h = c["acts"][-1]
    return conv(np.abs(h), np.abs(W), np.abs(b), 1)[..., 0]


def loss_and_grads(p: np.ndarray, x1: np.ndarray, target: np.ndarray, bf16: bool = False, scales: bool = False):
    """L1 loss mean|x0 - target| and its gradient w.r.t. p (flat, like p).
    With scales=True also returns, per parameter, the scale of an element-wise
    bound on its gradient: sum |h| G for a weight and sum G for a bias, where G
    is the magnitude chain of the backward pass -- |dLoss/df| carried back
    through every layer with |W| in place of W and the same ReLU masks -- so
    that G bounds the sum of the magnitudes of all the terms that make up each
    stored gradient element."""
    q = (lambda a: to_bf16(a)) if bf16 else (lambda a: a)
    x0, c = forward(p, x1, bf16)
    n = x0.size
    loss = float(np.abs(x0 - target).mean())
    acts, layers, inp = c["acts"], c["layers"], c["inp"]
    nl = len(SPEC)
    gpre = [None] * nl  # gradient of each layer's pre-activation (after the ReLU mask)
    df = np.zeros(x0.shape + (16,))
    df[..., 0] = np.sign(x0 - target) / n
    gpre[nl - 1] = q(df)
    gabs = [None] * nl
    gabs[nl - 1] = np.abs(gpre[nl - 1])
    grads = []
    sgrads = []
    for li in range(nl - 1, -1, -1):
        ci, co, kind, _ = SPEC[li]
        W, _ = layers[li]
        h = inp if li == 0 else acts[li - 1]
        g = gpre[li]
        if kind == "s1":
            dW = conv_wgrad(h, g, 1)
        elif kind == "s2":
            dW = conv_wgrad(h, g, 2)
        else:
            dW = conv_wgrad(up2(h), g, 1)
        if scales:
            ah, ag = np.abs(h), gabs[li]
            if kind == "s1":
                sW = conv_wgrad(ah, ag, 1)
            elif kind == "s2":
                sW = conv_wgrad(ah, ag, 2)
            else:
                sW = conv_wgrad(up2(ah), ag, 1)
            sgrads.append((li, sW, ag.reshape(-1, co).sum(axis=0)))
        grads.append((li, dW, g.reshape(-1, co).sum(axis=0)))
        if li == 0:
            break
        if kind == "s1":
            dh = conv_adjoint(h.shape, g, W, 1)
        elif kind == "s2":
            dh = conv_adjoint(h.shape, g, W, 2)
        else:
            dh = down2_sum(conv_adjoint(up2(h).shape, g, W, 1))
        for u, (_, _, _, skip) in enumerate(SPEC):
            if skip == li - 1:
                dh = dh + gpre[u]
        gpre[li - 1] = q(dh * (acts[li - 1] > 0))
        if scales:
            aW = np.abs(W)
            if kind == "s1":
                da = conv_adjoint(h.shape, gabs[li], aW, 1)
            elif kind == "s2":
                da = conv_adjoint(h.shape, gabs[li], aW, 2)
            else:
                da = down2_sum(conv_adjoint(up2(h).shape, gabs[li], aW, 1))
            for u, (_, _, _, skip) in enumerate(SPEC):
                if skip == li - 1:
                    da = da + gabs[u]
            gabs[li - 1] = da * (acts[li - 1] > 0)
    off = []
    o = 0
    for ci, co, _, _ in SPEC:
        off.append(o)
        o += 27 * ci * co + co

    def pack(items):
        flat = np.zeros(param_count())
        for li, dW, db in items:
            ci, co, _, _ = SPEC[li]
            flat[off[li]:off[li] + 27 * ci * co] = dW.ravel()
            flat[off[li] + 27 * ci * co:off[li] + 27 * ci * co + co] = db
        return flat

    if scales:
        return loss, pack(grads), pack(sgrads)
    return loss, pack(grads)


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights on the real channels, zero biases (test inputs)."""
    rng = np.random.Generator(np.random.Philox(seed))
    p = np.zeros(param_count())
    off = 0
    for li, (ci, co, _, _) in enumerate(SPEC):
        cin = 1 if li == 0 else ci
        cout = 1 if li == len(SPEC) - 1 else co
        W = np.zeros((27, ci, co))
        W[:, :cin, :cout] = rng.standard_normal((27, cin, cout)) * np.sqrt(2.0 / (27 * cin))
        p[off:off + 27 * ci * co] = W.ravel()
        off += 27 * ci * co + co
    return p
