"""Pins of the learned-guess oracle (oracle/nn.py) against things other than
itself: central finite differences, an independent torch.nn.functional
restatement with autograd, scipy's correlate2d, adjoint identities, the
closed-form first Adam step and the least-squares solution of the scaling."""
import numpy as np
import pytest
import scipy.signal

from oracle import nn as O

L, C0, CMAX = 2, 4, 4


def _case(seed=0, N=1, H=16, W=16, L=L, c0=C0, cmax=CMAX):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(O.num_params(L, c0, cmax)) * 0.3
    x = rng.standard_normal((N, 3, H, W))
    t = rng.standard_normal((N, 2, H, W))
    return p, x, t


def test_layer_shapes_and_count():
    sh = O.layer_shapes(3, 4, 8)
    # channels 4, 8, 8: encoder (3->4, 4->4), (4->8, 8->8), (8->8, 8->8); decoder
    # level 1 (8->8, 8->8), level 0 (8->4, 4->4); output 4->2
    assert sh == [(3, 4), (4, 4), (4, 8), (8, 8), (8, 8), (8, 8), (8, 8), (8, 8), (8, 4), (4, 4), (4, 2)]
    assert O.num_params(3, 4, 8) == sum(co * ci * 9 + co for ci, co in sh)


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 9, 7))
    Wt = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    got = O.conv3x3(x, Wt, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(scipy.signal.correlate2d(x[n, c], Wt[o, c], mode="same", boundary="fill")
                             for c in range(3))
            np.testing.assert_allclose(got[n, o], ref, rtol=1e-12, atol=1e-12)


def test_pool_up_adjoints_and_closed_forms():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 3, 8, 6))
    g = rng.standard_normal((2, 3, 4, 3))
    assert np.isclose(np.vdot(O.pool2(x), g), np.vdot(x, O.pool2_T(g)))
    assert np.isclose(np.vdot(O.up2(g), x), np.vdot(g, O.up2_T(x)))
    np.testing.assert_allclose(O.pool2(O.up2(g)), g)
    np.testing.assert_allclose(O.pool2(np.full((1, 1, 4, 4), 3.0)), np.full((1, 1, 2, 2), 3.0))


def _fd_check(p, x, t, L, c0, cmax, n_params=None, h=1e-6):
    loss, gp, gx = O.loss_and_grad(p, x, t, L, c0, cmax)
    idx = np.arange(p.size) if n_params is None else np.random.default_rng(3).choice(p.size, n_params, False)
    fd = np.empty(len(idx))
    for k, i in enumerate(idx):
        q = p.copy()
        q[i] += h
        lp = O.mse(O.forward(q, x, L, c0, cmax)[0], t)[0]
        q[i] -= 2 * h
        lm = O.mse(O.forward(q, x, L, c0, cmax)[0], t)[0]
        fd[k] = (lp - lm) / (2 * h)
    err_p = np.abs(fd - gp[idx]).max() / np.abs(gp).max()
    # input gradient on a few pixels
    rng = np.random.default_rng(4)
    err_x = 0.0
    for _ in range(8):
        c, yy, xx = rng.integers(3), rng.integers(x.shape[2]), rng.integers(x.shape[3])
        xp = x.copy()
        xp[0, c, yy, xx] += h
        lp = O.mse(O.forward(p, xp, L, c0, cmax)[0], t)[0]
        xp[0, c, yy, xx] -= 2 * h
        lm = O.mse(O.forward(p, xp, L, c0, cmax)[0], t)[0]
        err_x = max(err_x, abs((lp - lm) / (2 * h) - gx[0, c, yy, xx]) / np.abs(gx).max())
    return err_p, err_x


def test_gradient_central_differences_2level():
    p, x, t = _case()
    err_p, err_x = _fd_check(p, x, t, L, C0, CMAX)
    assert err_p < 1e-6 and err_x < 1e-6, (err_p, err_x)


def test_gradient_central_differences_3level_batch():
    p, x, t = _case(seed=5, N=2, H=8, W=16, L=3, c0=2, cmax=4)
    # the loss is a sum over the batch: check a subset of parameters
    loss, gp, _ = O.loss_and_grad(p, x, t, 3, 2, 4)
    idx = np.random.default_rng(6).choice(p.size, 60, False)
    h = 1e-6
    for i in idx:
        q = p.copy()
        q[i] += h
        lp = O.mse(O.forward(q, x, 3, 2, 4)[0], t)[0]
        q[i] -= 2 * h
        lm = O.mse(O.forward(q, x, 3, 2, 4)[0], t)[0]
        assert abs((lp - lm) / (2 * h) - gp[i]) <= 1e-6 * np.abs(gp).max()


def _torch_net(p, x, L, c0, cmax):
    """Independent restatement with torch.nn.functional (float64 CPU)."""
    import torch
    import torch.nn.functional as F
    ch = [min(cmax, c0 << l) for l in range(L)]
    P = torch.tensor(p, requires_grad=True)
    X = torch.tensor(x, requires_grad=True)
    off = [0]

    def take(ci, co):
        w = P[off[0]:off[0] + co * ci * 9].view(co, ci, 3, 3)
        off[0] += co * ci * 9
        b = P[off[0]:off[0] + co]
        off[0] += co
        return w, b

    encw = []
    for l in range(L):
        encw.append((take(3 if l == 0 else ch[l - 1], ch[l]), take(ch[l], ch[l])))
    decw = {}
    for l in range(L - 2, -1, -1):
        decw[l] = (take(ch[l + 1], ch[l]), take(ch[l], ch[l]))
    outw = take(ch[0], 2)
    skips = []
    h = X
    for l in range(L):
        if l > 0:
            h = F.avg_pool2d(skips[-1], 2)
        h = F.relu(F.conv2d(h, *encw[l][0], padding=1))
        skips.append(F.relu(F.conv2d(h, *encw[l][1], padding=1)))
    d = skips[-1]
    for l in range(L - 2, -1, -1):
        u = F.interpolate(d, scale_factor=2, mode="nearest")
        c = F.relu(F.conv2d(u, *decw[l][0], padding=1))
        d = F.relu(F.conv2d(c + skips[l], *decw[l][1], padding=1))
    return P, X, F.conv2d(d, *outw, padding=1)


@pytest.mark.parametrize("L_,c0,cmax,H,W", [(2, 4, 4, 16, 16), (3, 2, 6, 8, 16), (1, 3, 3, 6, 5)])
def test_matches_torch_autograd(L_, c0, cmax, H, W):
    import torch
    p, x, t = _case(seed=7, N=2, H=H, W=W, L=L_, c0=c0, cmax=cmax)
    out, cache = O.forward(p, x, L_, c0, cmax)
    P, X, Y = _torch_net(p, x, L_, c0, cmax)
    np.testing.assert_allclose(out, Y.detach().numpy(), rtol=1e-12, atol=1e-12)
    loss = ((Y - torch.tensor(t)) ** 2).mean()
    loss.backward()
    l2, gp, gx = O.loss_and_grad(p, x, t, L_, c0, cmax)
    assert np.isclose(l2, loss.item(), rtol=1e-12)
    np.testing.assert_allclose(gp, P.grad.numpy(), rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(gx, X.grad.numpy(), rtol=1e-10, atol=1e-13)


def test_mutation_is_caught_by_finite_differences(monkeypatch):
    """A wrong adjoint planted in the oracle (up2_T off by a factor) must
    fail the finite-difference pin."""
    p, x, t = _case()
    monkeypatch.setattr(O, "up2_T", lambda g: 0.5 * (g[:, :, 0::2, 0::2] + g[:, :, 1::2, 0::2]
                                                     + g[:, :, 0::2, 1::2] + g[:, :, 1::2, 1::2]))
    err_p, err_x = _fd_check(p, x, t, L, C0, CMAX, n_params=200)
    assert max(err_p, err_x) > 1e-3


def test_mutation_dropped_skip_is_caught_by_torch(monkeypatch):
    """An oracle whose decoder drops the skip addition must fail the
    independent restatement."""
    p, x, _ = _case(seed=8)
    _, _, Y = _torch_net(p, x, L, C0, CMAX)
    out, _ = O.forward(p, x, L, C0, CMAX)
    assert np.abs(out - Y.detach().numpy()).max() < 1e-12
    real_conv = O.conv3x3
    seen = {"n": 0}

    def conv_plant(xx, Wt, b):
        seen["n"] += 1
        if seen["n"] == 6:   # the decoder's second conv reads decC + skip: give it decC
            xx = xx - cache_skip[0]
        return real_conv(xx, Wt, b)
    layers = O.unpack(p, L, C0, CMAX)
    cache_skip = [O.relu(real_conv(O.relu(real_conv(x, *layers[0])), *layers[1]))]
    monkeypatch.setattr(O, "conv3x3", conv_plant)
    wrong, _ = O.forward(p, x, L, C0, CMAX)
    assert seen["n"] == 7
    assert np.abs(wrong - Y.detach().numpy()).max() > 1e-3


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(9)
    w = rng.standard_normal(50)
    g = rng.standard_normal(50)
    w1, m, v = O.adam_step(w, g, np.zeros(50), np.zeros(50), 1, lr=1e-2)
    # bias-corrected first step: m_hat = g, v_hat = g^2
    np.testing.assert_allclose(w1, w - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_bf16_round_matches_torch():
    import torch
    rng = np.random.default_rng(10)
    a = np.concatenate([rng.standard_normal(1000) * 10 ** rng.uniform(-6, 6, 1000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38]]).astype(np.float32)
    ref = torch.tensor(a).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.bf16_round(a), ref)


def test_scaled_guess_is_least_squares_and_falls_back():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((30, 30)) + 1j * rng.standard_normal((30, 30))
    b = rng.standard_normal(30) + 1j * rng.standard_normal(30)
    y = rng.standard_normal(30) + 1j * rng.standard_normal(30)
    x0, raw, scaled, used = O.scaled_guess(A, b, y)
    alpha = np.linalg.lstsq((A @ y)[:, None], b, rcond=None)[0][0]
    np.testing.assert_allclose(x0, alpha * y, rtol=1e-12)
    assert used and scaled < 1
    assert np.isclose(raw, np.linalg.norm(b - A @ y) / np.linalg.norm(b))
    # a guess whose image is orthogonal to b cannot help: zero guess
    Ay = A @ y
    b2 = b - np.vdot(Ay, b) / np.vdot(Ay, Ay) * Ay
    x0, _, scaled, used = O.scaled_guess(A, b2, y)
    assert not used and scaled == 1.0 and not x0.any()


def test_images_layout():
    eps = np.arange(12, dtype=float).reshape(4, 3) + 1.0        # nx=4, ny=3
    b = np.zeros((4, 3), complex)
    b[2, 1] = -4.0 + 2.0j
    x = np.zeros((4, 3), complex)
    x[3, 2] = 1.0 - 0.5j
    inp, tgt, s = O.images(eps, b, x, unit=0.5, H=4, W=8)
    assert s == 4.0
    assert inp.shape == (3, 4, 8) and tgt.shape == (2, 4, 8)
    assert inp[0, 1, 2] == (eps[2, 1] - 1) / 10 and inp[0, 3, :].sum() == 0 and inp[0, :, 4:].sum() == 0
    assert inp[1, 1, 2] == -1.0 and inp[2, 1, 2] == 0.5
    assert tgt[0, 2, 3] == 1.0 / 2.0 and tgt[1, 2, 3] == -0.25


# ------------------------------------------------ tensor-core operand rounding
def _torch_net_tc(p, x, L, c0, cmax):
    """Independent restatement of the tensor-core mode in torch float64: the
    weights are the BF16 copy of the master weights (gradient passed straight
    through to the masters), and every convolution is an autograd function
    whose products read BF16-rounded operands -- forward: the layer input;
    input gradient: the output gradient; weight gradient: the layer input and
    the output gradient -- while the bias gradient sums the unrounded output
    gradient.  Rounding is torch's own float64 -> bfloat16 conversion."""
    import torch
    import torch.nn.functional as F
    from torch.nn.grad import conv2d_input, conv2d_weight

    def bf(t):
        return t.to(torch.bfloat16).to(torch.float64)

    class RoundSTE(torch.autograd.Function):
        @staticmethod
        def forward(ctx, t):
            return bf(t)

        @staticmethod
        def backward(ctx, g):
            return g

    class ConvTC(torch.autograd.Function):
        @staticmethod
        def forward(ctx, inp, w, b):
            ctx.save_for_backward(inp, w)
            return F.conv2d(bf(inp), w, b, padding=1)

        @staticmethod
        def backward(ctx, g):
            inp, w = ctx.saved_tensors
            gr = bf(g)
            gx = conv2d_input(inp.shape, w, gr, padding=1)
            gw = conv2d_weight(bf(inp), w.shape, gr, padding=1)
            return gx, gw, g.sum(dim=(0, 2, 3))

    ch = [min(cmax, c0 << l) for l in range(L)]
    P = torch.tensor(p, requires_grad=True)
    X = torch.tensor(x, requires_grad=True)
    Pr = RoundSTE.apply(P)
    off = [0]

    def take(ci, co):
        w = Pr[off[0]:off[0] + co * ci * 9].view(co, ci, 3, 3)
        off[0] += co * ci * 9
        b = Pr[off[0]:off[0] + co]
        off[0] += co
        return w, b

    conv = ConvTC.apply
    encw = [(take(3 if l == 0 else ch[l - 1], ch[l]), take(ch[l], ch[l])) for l in range(L)]
    decw = {}
    for l in range(L - 2, -1, -1):
        decw[l] = (take(ch[l + 1], ch[l]), take(ch[l], ch[l]))
    outw = take(ch[0], 2)
    skips = []
    h = X
    for l in range(L):
        if l > 0:
            h = F.avg_pool2d(skips[-1], 2)
        h = F.relu(conv(h, *encw[l][0]))
        skips.append(F.relu(conv(h, *encw[l][1])))
    d = skips[-1]
    for l in range(L - 2, -1, -1):
        u = F.interpolate(d, scale_factor=2, mode="nearest")
        c = F.relu(conv(u, *decw[l][0]))
        d = F.relu(conv(c + skips[l], *decw[l][1]))
    return P, X, conv(d, *outw)


def _tc_compare(L_, c0, cmax, H, W, seed=12):
    import torch
    p, x, t = _case(seed=seed, N=2, H=H, W=W, L=L_, c0=c0, cmax=cmax)
    P, X, Y = _torch_net_tc(p, x, L_, c0, cmax)
    loss = ((Y - torch.tensor(t)) ** 2).mean()
    loss.backward()
    out, _ = O.forward(p, x, L_, c0, cmax, round_bf16=True, round_act=True)
    l2, gp, gx = O.loss_and_grad(p, x, t, L_, c0, cmax, round_bf16=True, round_act=True)
    return (np.abs(out - Y.detach().numpy()).max() / np.abs(out).max(), abs(l2 - loss.item()) / loss.item(),
            np.abs(gp - P.grad.numpy()).max() / np.abs(gp).max(),
            np.abs(gx - X.grad.numpy()).max() / np.abs(gx).max())


@pytest.mark.parametrize("L_,c0,cmax,H,W", [(2, 4, 4, 16, 16), (3, 2, 6, 8, 16), (1, 3, 3, 6, 5)])
def test_tensor_core_rounding_matches_torch_restatement(L_, c0, cmax, H, W):
    """The oracle's tensor-core mode (BF16 weights, BF16 operands of every
    convolution product) equals the torch restatement with autograd functions
    that round at the same operands: forward, loss, parameter and input
    gradients."""
    e_out, e_loss, e_gp, e_gx = _tc_compare(L_, c0, cmax, H, W)
    assert e_out < 1e-12 and e_loss < 1e-12
    assert e_gp < 1e-10 and e_gx < 1e-10


def test_tensor_core_rounding_differs_from_unrounded():
    """The rounding is visible: the unrounded network's gradients differ from
    the tensor-core mode's by far more than the restatement's tolerance."""
    p, x, t = _case(seed=12, N=2, H=16, W=16)
    _, g_tc, _ = O.loss_and_grad(p, x, t, L, C0, CMAX, round_bf16=True, round_act=True)
    _, g_w, _ = O.loss_and_grad(p, x, t, L, C0, CMAX, round_bf16=True)
    assert np.abs(g_tc - g_w).max() / np.abs(g_w).max() > 1e-4


@pytest.mark.parametrize("plant", ["bias_from_rounded", "input_grad_unrounded", "wgrad_input_unrounded",
                                   "forward_unrounded"])
def test_tensor_core_rounding_mutations_are_caught(monkeypatch, plant):
    """Each rounding point moved in the oracle (planted here, on the CPU)
    fails the torch restatement."""
    real_bwd, real_conv = O.conv3x3_backward_tc, O._conv_backward

    def bias_from_rounded(x, W, gout):
        gx, gW, _ = real_bwd(x, W, gout)
        return gx, gW, O.bf16_round(gout).sum(axis=(0, 2, 3))

    def input_grad_unrounded(x, W, gout):
        _, gW, gb = real_bwd(x, W, gout)
        gx, _, _ = real_conv(x, W, gout)
        return gx, gW, gb

    def wgrad_input_unrounded(x, W, gout):
        gx, _, gb = real_bwd(x, W, gout)
        _, gW, _ = real_conv(x, W, O.bf16_round(gout))
        return gx, gW, gb

    if plant == "forward_unrounded":
        monkeypatch.setattr(O, "conv3x3_tc", lambda x, W, b: O._conv(x, W, b))
    else:
        monkeypatch.setattr(O, "conv3x3_backward_tc", locals()[plant])
    e_out, e_loss, e_gp, e_gx = _tc_compare(2, 4, 4, 16, 16)
    assert max(e_out, e_loss, e_gp, e_gx) > 1e-6
