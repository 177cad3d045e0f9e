"""CPU oracle of the learned initial guess (test infrastructure only).

The paper has no network; this restates, in float64 numpy, the network the
library defines for its learned initial guess: an encoder-decoder of 3x3
convolutions with L levels and c_l = min(c0 * 2^l, cmax) channels,

* encoder level l: conv + ReLU, conv + ReLU (the result is skip_l); level 0
  reads the 3-channel image, level l > 0 the 2x2 average pool of skip_{l-1};
* decoder level l = L-2 .. 0: nearest 2x upsampling of the level below,
  conv (c_{l+1} -> c_l) + ReLU, add skip_l, conv + ReLU;
* output: conv (c_0 -> 2) without activation,

with the parameters in one flat array, layer by layer in that order, each
layer its weights [cout][cin][3][3] followed by its bias [cout].  A 3x3
convolution is the zero-padded cross-correlation
out[o](y, x) = bias[o] + sum_c sum_{ky,kx} w[o, c, ky, kx] in[c](y+ky-1, x+kx-1).

The backward pass is written out by hand, layer by layer (the chain rule in
reverse order), so that tests can check it against central finite
differences of the forward pass.  Also here: the mean-squared-error loss,
Adam (Kingma & Ba, 2015), the image normalisation that maps a problem
(eps, b, x) to network input and target, and the minimal-residual scaling of
a guess with its zero-guess fallback (after one sweep of the preconditioner
from the network field).

Parity status: forward and backward are pinned by central finite
differences, by an independent torch.nn.functional restatement with
autograd, and by scipy's correlate2d for the convolution; the scaling by the
closed-form least-squares solution.  The tensor-core mode's operand rounding
(conv3x3_tc, conv3x3_backward_tc) is pinned by a torch restatement whose
autograd functions round with torch's own bfloat16 conversion at the same
points (forward, input-gradient and weight-gradient operands).
"""
from __future__ import annotations

import numpy as np


def channels(L, c0, cmax):
    return [min(cmax, c0 << l) for l in range(L)]


def layer_shapes(L, c0, cmax):
    """(cin, cout) of every layer in parameter order."""
    ch = channels(L, c0, cmax)
    shapes = []
    for l in range(L):
        shapes.append((3 if l == 0 else ch[l - 1], ch[l]))
        shapes.append((ch[l], ch[l]))
    for l in range(L - 2, -1, -1):
        shapes.append((ch[l + 1], ch[l]))
        shapes.append((ch[l], ch[l]))
    shapes.append((ch[0], 2))
    return shapes


def num_params(L, c0, cmax):
    return sum(co * ci * 9 + co for ci, co in layer_shapes(L, c0, cmax))


def unpack(params, L, c0, cmax):
    """List of (W [cout, cin, 3, 3], b [cout]) views of the flat array."""
    out, off = [], 0
    for ci, co in layer_shapes(L, c0, cmax):
        W = params[off:off + co * ci * 9].reshape(co, ci, 3, 3)
        off += co * ci * 9
        b = params[off:off + co]
        off += co
        out.append((W, b))
    assert off == params.size
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


# ---------------------------------------------------------------- layers

def conv3x3(x, W, b):
    """x [N, C, H, W] -> [N, O, H, W]."""
    N, C, H, Wd = x.shape
    xp = np.zeros((N, C, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    out = np.broadcast_to(b[None, :, None, None], (N, W.shape[0], H, Wd)).copy()
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("oc,nchw->nohw", W[:, :, ky, kx], xp[:, :, ky:ky + H, kx:kx + Wd])
    return out


def conv3x3_backward(x, W, gout):
    """Gradients (gx, gW, gb) of sum(gout * conv3x3(x, W, b))."""
    N, C, H, Wd = x.shape
    xp = np.zeros((N, C, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    gW = np.zeros_like(W)
    gxp = np.zeros_like(xp)
    for ky in range(3):
        for kx in range(3):
            gW[:, :, ky, kx] = np.einsum("nohw,nchw->oc", gout, xp[:, :, ky:ky + H, kx:kx + Wd])
            gxp[:, :, ky:ky + H, kx:kx + Wd] += np.einsum("oc,nohw->nchw", W[:, :, ky, kx], gout)
    gb = gout.sum(axis=(0, 2, 3))
    return gxp[:, :, 1:-1, 1:-1], gW, gb


def relu(x):
    return np.maximum(x, 0.0)


def pool2(x):
    """2x2 average pooling (H, W even)."""
    return 0.25 * (x[:, :, 0::2, 0::2] + x[:, :, 1::2, 0::2] + x[:, :, 0::2, 1::2] + x[:, :, 1::2, 1::2])


def pool2_T(g):
    """Adjoint of pool2."""
    return 0.25 * np.repeat(np.repeat(g, 2, axis=2), 2, axis=3)


def up2(x):
    """Nearest-neighbour 2x upsampling."""
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up2_T(g):
    """Adjoint of up2."""
    return g[:, :, 0::2, 0::2] + g[:, :, 1::2, 0::2] + g[:, :, 0::2, 1::2] + g[:, :, 1::2, 1::2]


# ---------------------------------------------------------------- network

def _conv(x, W, b):
    return conv3x3(x, W, b)


def _conv_backward(x, W, gout):
    return conv3x3_backward(x, W, gout)


# Tensor-core mode (round_act).  The network's convolutions run as matrix
# products on BF16 operands with FP32 (here: exact) accumulation, so exactly
# the values that enter a product as an operand are rounded to BF16, and
# nothing else:
#   forward            out = conv(bf16(x), W) + b      operands: layer input, weights
#   input gradient     gx  = conv_T(bf16(g), W)        operands: output gradient, weights
#   weight gradient    gW  = corr(bf16(x), bf16(g))    operands: layer input, output gradient
#   bias gradient      gb  = sum(g)                    a plain sum, not a product: unrounded
# (the weights W are the BF16 copy of the master weights in this mode).
def conv3x3_tc(x, W, b):
    """Forward convolution of the tensor-core mode: the layer input rounded
    to BF16 before the product."""
    return _conv(bf16_round(x), W, b)


def conv3x3_backward_tc(x, W, gout):
    """Backward convolution of the tensor-core mode: (gx, gW, gb) with the
    output gradient rounded to BF16 in both gradient products, the layer
    input rounded to BF16 in the weight-gradient product, and the bias
    gradient summed from the unrounded output gradient."""
    gr = bf16_round(gout)
    gx, _, _ = _conv_backward(x, W, gr)
    _, gW, _ = _conv_backward(bf16_round(x), W, gr)
    return gx, gW, gout.sum(axis=(0, 2, 3))


def forward(params, x, L, c0, cmax, round_bf16=False, round_act=False):
    """Network output [N, 2, H, W] and the cache the backward pass needs.
    round_bf16 rounds the weights to BF16; round_act also rounds every
    convolution's input to BF16 (the operand rounding of the tensor-core
    mode; it makes the loss piecewise constant, so finite differences do not
    apply to it)."""
    p = bf16_round(params) if round_bf16 else params
    conv3x3 = conv3x3_tc if round_act else _conv
    layers = unpack(p, L, c0, cmax)
    enc = [(layers[2 * l], layers[2 * l + 1]) for l in range(L)]
    dec = {}
    k = 2 * L
    for l in range(L - 2, -1, -1):
        dec[l] = (layers[k], layers[k + 1])
        k += 2
    out_layer = layers[k]
    cache = dict(x=x, layers=layers, enc_in=[], encA=[], skip=[], up={}, decC={}, sum={}, d={})
    h = x
    for l in range(L):
        if l > 0:
            h = pool2(cache["skip"][l - 1])
        cache["enc_in"].append(h)
        a = relu(conv3x3(h, *enc[l][0]))
        cache["encA"].append(a)
        cache["skip"].append(relu(conv3x3(a, *enc[l][1])))
    d = cache["skip"][L - 1]
    for l in range(L - 2, -1, -1):
        u = up2(d)
        cache["up"][l] = u
        c = relu(conv3x3(u, *dec[l][0]))
        cache["decC"][l] = c
        s = c + cache["skip"][l]
        cache["sum"][l] = s
        d = relu(conv3x3(s, *dec[l][1]))
        cache["d"][l] = d
    cache["last"] = d
    cache["enc"], cache["dec"], cache["out_layer"] = enc, dec, out_layer
    cache["round_act"] = round_act
    return conv3x3(d, *out_layer), cache


def backward(cache, gout, L):
    """Flat parameter gradient and input gradient for output gradient gout
    (the chain rule through forward() in reverse order)."""
    enc, dec, out_layer = cache["enc"], cache["dec"], cache["out_layer"]
    conv3x3_backward = conv3x3_backward_tc if cache.get("round_act") else _conv_backward
    grads = {}
    gd, gW, gb = conv3x3_backward(cache["last"], out_layer[0], gout)
    grads["out"] = (gW, gb)
    gskip = [np.zeros_like(s) for s in cache["skip"]]
    if L == 1:
        gskip[0] += gd
    for l in range(0, L - 1):
        gd = gd * (cache["d"][l] > 0)
        gs, gW, gb = conv3x3_backward(cache["sum"][l], dec[l][1][0], gd)
        grads[("D", l)] = (gW, gb)
        gskip[l] += gs
        gc = gs * (cache["decC"][l] > 0)
        gu, gW, gb = conv3x3_backward(cache["up"][l], dec[l][0][0], gc)
        grads[("C", l)] = (gW, gb)
        gd = up2_T(gu)
        if l + 1 == L - 1:
            gskip[L - 1] += gd
    gx = None
    for l in range(L - 1, -1, -1):
        g = gskip[l] * (cache["skip"][l] > 0)
        ga, gW, gb = conv3x3_backward(cache["encA"][l], enc[l][1][0], g)
        grads[("B", l)] = (gW, gb)
        ga = ga * (cache["encA"][l] > 0)
        gi, gW, gb = conv3x3_backward(cache["enc_in"][l], enc[l][0][0], ga)
        grads[("A", l)] = (gW, gb)
        if l > 0:
            gskip[l - 1] += pool2_T(gi)
        else:
            gx = gi
    order = []
    for l in range(L):
        order += [grads[("A", l)], grads[("B", l)]]
    for l in range(L - 2, -1, -1):
        order += [grads[("C", l)], grads[("D", l)]]
    order.append(grads["out"])
    return pack(order), gx


def mse(pred, target):
    """Loss sum((pred - target)^2) / n and its gradient."""
    d = pred - target
    return float((d * d).sum() / d.size), 2.0 * d / d.size


def loss_and_grad(params, x, target, L, c0, cmax, round_bf16=False, round_act=False):
    out, cache = forward(params, x, L, c0, cmax, round_bf16, round_act)
    loss, g = mse(out, target)
    gp, gx = backward(cache, g, L)
    return loss, gp, gx


def adam_step(w, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected moments); returns (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(a):
    """Round float values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


# ---------------------------------------------------------------- solver glue

def images(eps, b, x=None, unit=1.0, H=None, W=None):
    """Network input [3, H, W] (and target [2, H, W] if x is given) of one
    problem: node (i, j) is pixel (row j, column i); channels (eps - 1) / 10,
    Re b / s, Im b / s with s = max(|Re b|, |Im b|); target x / (s * unit)."""
    nx, ny = eps.shape
    H = ny if H is None else H
    W = nx if W is None else W
    s = max(np.abs(b.real).max(), np.abs(b.imag).max())
    inv = 1.0 / s if s > 0 else 0.0
    inp = np.zeros((3, H, W))
    inp[0, :ny, :nx] = ((eps - 1.0) / 10.0).T
    inp[1, :ny, :nx] = (b.real * inv).T
    inp[2, :ny, :nx] = (b.imag * inv).T
    if x is None:
        return inp, s
    tgt = np.zeros((2, H, W))
    if s > 0:
        tgt[0, :ny, :nx] = (x.real / (s * unit)).T
        tgt[1, :ny, :nx] = (x.imag / (s * unit)).T
    return inp, tgt, s


def raw_guess(params, eps, b, dx, dy, L, c0, cmax, round_bf16=True):
    """Network field y (nx, ny) complex for one problem, the grid zero-padded
    to a multiple of 2^(L-1)."""
    nx, ny = eps.shape
    f = 1 << (L - 1)
    H, W = -(-ny // f) * f, -(-nx // f) * f
    inp, s = images(eps, b, H=H, W=W)
    out, _ = forward(params, inp[None], L, c0, cmax, round_bf16)
    y = (out[0, 0, :ny, :nx] + 1j * out[0, 1, :ny, :nx]).T
    return y * s * dx * dy


def learned_start(A, apply_minv, b, y):
    """The solver's learned start: one sweep of the method from the network
    field, x = y + M^-1 (b - A y), then scaled_guess.  Returns (x0, raw_rel
    of y, scaled_rel of x0, used)."""
    raw = np.linalg.norm(b - A @ y) / np.linalg.norm(b)
    x = y + apply_minv(b - A @ y)
    x0, _, scaled, used = scaled_guess(A, b, x)
    return x0, raw, scaled, used


def scaled_guess(A, b, y):
    """Minimal-residual multiple alpha*y of a guess, alpha = (Ay)^H b /
    ||Ay||^2, and the zero-guess fallback when it does not lower ||b - A x0||
    below ||b||.  Returns (x0, raw_rel, scaled_rel, used)."""
    Ay = A @ y
    nb = np.linalg.norm(b)
    raw = np.linalg.norm(b - Ay) / nb
    aa = np.vdot(Ay, Ay).real
    if aa == 0 or not np.isfinite(aa):
        return np.zeros_like(b), raw, 1.0, False
    alpha = np.vdot(Ay, b) / aa
    scaled = np.linalg.norm(b - alpha * Ay) / nb
    if not scaled < 1.0 - 1e-12:
        return np.zeros_like(b), raw, 1.0, False
    return alpha * y, raw, scaled, True
