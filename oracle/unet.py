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
    acts, pres = [], []
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
            return x0, {"inp": inp, "acts": acts, "pres": pres, "layers": layers, "x1": x1, "x0": x0}
        pres.append(pre)
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


def _layer_pre_magnitudes(c) -> list:
    """Per hidden layer, the magnitude sum of its pre-activation: |b| + sum of
    |W| |h| over taps and channels (+ the skip input, which is >= 0)."""
    layers, acts, inp = c["layers"], c["acts"], c["inp"]
    mags = []
    for li in range(len(SPEC) - 1):
        _, _, kind, skip = SPEC[li]
        W, b = layers[li]
        h = inp if li == 0 else acts[li - 1]
        aW, ab = np.abs(W), np.abs(b)
        if kind == "s1":
            m = conv(np.abs(h), aW, ab, 1)
        elif kind == "s2":
            m = conv(np.abs(h), aW, ab, 2)
        else:
            m = conv(up2(np.abs(h)), aW, ab, 1)
        if skip >= 0:
            m = m + acts[skip]
        mags.append(m)
    return mags


def _magnitude_chain(c, g_last, masks, hmag):
    """Per parameter, sum |h| G (weights) and sum G (biases), where G is the
    backward pass run on magnitudes: |dLoss/df| carried back through every
    layer with |W| in place of W and the given 0/1 masks in place of the ReLU
    masks; hmag[li] is the activation magnitude used for layer li's input."""
    layers = c["layers"]
    nl = len(SPEC)
    G = [None] * nl
    G[nl - 1] = g_last
    out = []
    for li in range(nl - 1, -1, -1):
        ci, co, kind, _ = SPEC[li]
        W, _ = layers[li]
        h = hmag[li]
        if kind == "s1":
            sW = conv_wgrad(h, G[li], 1)
        elif kind == "s2":
            sW = conv_wgrad(h, G[li], 2)
        else:
            sW = conv_wgrad(up2(h), G[li], 1)
        out.append((li, sW, G[li].reshape(-1, co).sum(axis=0)))
        if li == 0:
            break
        aW = np.abs(W)
        if kind == "s1":
            da = conv_adjoint(h.shape, G[li], aW, 1)
        elif kind == "s2":
            da = conv_adjoint(h.shape, G[li], aW, 2)
        else:
            da = down2_sum(conv_adjoint(up2(h).shape, G[li], aW, 1))
        for u, (_, _, _, skip) in enumerate(SPEC):
            if skip == li - 1:
                da = da + G[u]
        G[li - 1] = da * masks[li - 1]
    return out


def loss_and_grads(p: np.ndarray, x1: np.ndarray, target: np.ndarray, bf16: bool = False, scales: bool = False,
                   relu_margin: float = 1e-3):
    """L1 loss mean|x0 - target| and its gradient w.r.t. p (flat, like p).

    With scales=True also returns two per-parameter scales for an element-wise
    bound on the gradient of an implementation that sums in another order.
    Each is sum |h| G for a weight and sum G for a bias, G being the backward
    pass run on magnitudes (|dLoss/df| carried back with |W| in place of W):

      core:    ReLU masks only where the pre-activation is clearly positive
               (pre > relu_margin times its magnitude sum), activations zero
               where it is not clearly decided;
      relaxed: masks also open where |pre| <= relu_margin times its magnitude
               sum, those activations counted at up to that margin.

    Where a pre-activation lies that close to zero, a different summation
    order may take the other ReLU decision; every term of the gradient that
    runs through such a position may then be present on one side and absent on
    the other, and those terms are exactly relaxed - core. The terms through
    clearly decided positions only differ by rounding, bounded relative to the
    relaxed scale. Returns (loss, grads, core, relaxed)."""
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
    grads = []
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

    if not scales:
        return loss, pack(grads)
    mags = _layer_pre_magnitudes(c)
    pres = c["pres"]
    amb = [np.abs(pres[li]) <= relu_margin * mags[li] for li in range(nl - 1)]
    sure = [(pres[li] > 0) & ~amb[li] for li in range(nl - 1)]
    g_last = np.abs(gpre[nl - 1])
    h_core = [np.abs(inp)] + [np.abs(acts[li]) * sure[li] for li in range(nl - 1)]
    h_rel = [np.abs(inp)] + [np.abs(acts[li]) + relu_margin * mags[li] * amb[li] for li in range(nl - 1)]
    core = _magnitude_chain(c, g_last, [m.astype(np.float64) for m in sure], h_core)
    rel = _magnitude_chain(c, g_last, [((acts[li] > 0) | amb[li]).astype(np.float64) for li in range(nl - 1)], h_rel)
    return loss, pack(grads), pack(core), pack(rel)


def _layer_conv(kind, h, W, b):
    if kind == "s1":
        return conv(h, W, b, 1)
    if kind == "s2":
        return conv(h, W, b, 2)
    return conv(up2(h), W, b, 1)


def layer_forward(p: np.ndarray, li: int, h: np.ndarray, skip=None):
    """Hidden layer li (0..13) on its stored input h (channels last): the
    stored output bf16(relu(conv(h) + b + skip)) with BF16 weights, and the
    magnitude sum |b| + sum |W| |h| (+ skip) of every pre-activation."""
    W, b = unpack(p)[li]
    W = to_bf16(W)
    kind = SPEC[li][2]
    pre = _layer_conv(kind, h, W, b)
    mag = _layer_conv(kind, np.abs(h), np.abs(W), np.abs(b))
    if skip is not None:
        pre = pre + skip
        mag = mag + np.abs(skip)
    return to_bf16(np.maximum(pre, 0.0)), mag


def layer_data_grad(p: np.ndarray, li: int, dy: np.ndarray, mask: np.ndarray, add=None):
    """Layer li's (1..14) gradient into layer li-1's output: bf16((conv^T(dy)
    + add) * [mask > 0]) with BF16 weights, dy the gradient of li's
    pre-activation and mask li-1's stored activation; and the magnitude sum
    of every element (before the mask)."""
    W, _ = unpack(p)[li]
    W = to_bf16(W)
    kind = SPEC[li][2]
    shape = mask.shape
    if kind == "s1":
        dh = conv_adjoint(shape, dy, W, 1)
        mag = conv_adjoint(shape, np.abs(dy), np.abs(W), 1)
    elif kind == "s2":
        dh = conv_adjoint(shape, dy, W, 2)
        mag = conv_adjoint(shape, np.abs(dy), np.abs(W), 2)
    else:
        up_shape = (2 * shape[0], 2 * shape[1], 2 * shape[2], shape[3])
        dh = down2_sum(conv_adjoint(up_shape, dy, W, 1))
        mag = down2_sum(conv_adjoint(up_shape, np.abs(dy), np.abs(W), 1))
    if add is not None:
        dh = dh + add
        mag = mag + np.abs(add)
    return to_bf16(dh * (mask > 0)), mag


def layer_weight_grad(li: int, h: np.ndarray, dy: np.ndarray):
    """Layer li's parameter gradient from its input h and the gradient dy of
    its pre-activation: flat [dW (tap, ci, co), db] and the magnitude sum of
    every element."""
    kind = SPEC[li][2]
    hh = up2(h) if kind == "up" else h
    stride = 2 if kind == "s2" else 1
    co = dy.shape[-1]
    g = np.concatenate([conv_wgrad(hh, dy, stride).ravel(), dy.reshape(-1, co).sum(axis=0)])
    m = np.concatenate([conv_wgrad(np.abs(hh), np.abs(dy), stride).ravel(), np.abs(dy).reshape(-1, co).sum(axis=0)])
    return g, m


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
