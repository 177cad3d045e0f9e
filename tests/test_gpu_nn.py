"""GPU parity of the learned initial guess: network forward, gradients and
Adam step against the CPU oracle (oracle/nn.py), the image preparation, the
guess inside the solver (scaling and fallback), and what a trained network
gains over the zero guess."""
import numpy as np
import pytest

import workloads as W
from oracle import nn as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _lib():
    from paper_2509_20801_gb300 import learned
    return learned


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch.device("cuda:0")


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def _net(L, c0, cmax, bf16, seed=0, params=None, mode=None):
    learned = _lib()
    net = learned.Network(L, c0, cmax, mode=mode or ("bf16" if bf16 else "fp32"), seed=seed)
    if params is not None:
        net.set_params(params)
    return net


CASES = [
    # L, c0, cmax, N, H, W: one tile, several tiles with ragged edges and
    # channel counts that are not multiples of the 16-channel blocks
    (2, 4, 4, 1, 16, 16),
    (3, 8, 24, 2, 40, 72),
    (1, 3, 3, 1, 7, 5),
]


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("case", CASES)
def test_forward_and_gradient_match_oracle(case, bf16):
    dev = _dev()
    L, c0, cmax, N, H, Wd = case
    rng = np.random.default_rng(1)
    p = (rng.standard_normal(O.num_params(L, c0, cmax)) * 0.3).astype(np.float32)
    x = rng.standard_normal((N, 3, H, Wd)).astype(np.float32)
    t = rng.standard_normal((N, 2, H, Wd)).astype(np.float32)
    net = _net(L, c0, cmax, bf16, params=p)
    assert net.num_params() == O.num_params(L, c0, cmax)
    np.testing.assert_array_equal(net.get_params(), p)
    xin = torch.from_numpy(x).to(dev)
    out = torch.empty((N, 2, H, Wd), dtype=torch.float32, device=dev)
    net.forward(xin, out)
    ref, _ = O.forward(p.astype(np.float64), x.astype(np.float64), L, c0, cmax, round_bf16=bf16)
    # FP32 activations and accumulation against FP64 with the same weights
    assert _rel(out.cpu().numpy(), ref) < 1e-5
    loss, g = net.gradient(xin, torch.from_numpy(t).to(dev))
    rl, rg, _ = O.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), L, c0, cmax,
                                round_bf16=bf16)
    assert abs(loss - rl) <= 1e-5 * rl
    assert _rel(g, rg) < 1e-5
    net.close()


TC_CASES = CASES + [
    # 8 input chunks, 256 output channels (the widest tile)
    (2, 128, 256, 1, 32, 48),
    # weight gradient: three 64-pixel column strips with a 5-pixel ragged
    # one, rows not 16-byte aligned (W odd), two images (the row walk
    # restarts per strip and image)
    (1, 32, 32, 2, 9, 133),
    # two levels with 136 and 68 pixel rows, 136 output channels (two
    # 128-channel tiles, the second ragged)
    (2, 40, 136, 3, 20, 136),
]


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("case", TC_CASES)
def test_tensor_core_mode_matches_oracle(case):
    """BF16 operands on the tensor cores: against the oracle with the same
    operand rounding (tight), and against the unrounded oracle (the BF16
    error itself)."""
    dev = _dev()
    L, c0, cmax, N, H, Wd = case
    rng = np.random.default_rng(12)
    p = (rng.standard_normal(O.num_params(L, c0, cmax)) * (0.3 if c0 < 64 else 0.05)).astype(np.float32)
    x = rng.standard_normal((N, 3, H, Wd)).astype(np.float32)
    t = rng.standard_normal((N, 2, H, Wd)).astype(np.float32)
    net = _net(L, c0, cmax, True, params=p, mode="tc")
    xin = torch.from_numpy(x).to(dev)
    out = torch.empty((N, 2, H, Wd), dtype=torch.float32, device=dev)
    net.forward(xin, out)
    got = out.cpu().numpy()
    p64, x64, t64 = p.astype(np.float64), x.astype(np.float64), t.astype(np.float64)
    ref_r, _ = O.forward(p64, x64, L, c0, cmax, round_bf16=True, round_act=True)
    ref, _ = O.forward(p64, x64, L, c0, cmax, round_bf16=True)
    e_r, e = _rel_l2(got, ref_r), _rel_l2(got, ref)
    loss, g = net.gradient(xin, torch.from_numpy(t).to(dev))
    _, rg_r, _ = O.loss_and_grad(p64, x64, t64, L, c0, cmax, round_bf16=True, round_act=True)
    rl, rg, _ = O.loss_and_grad(p64, x64, t64, L, c0, cmax, round_bf16=True)
    g_r, g_e = _rel_l2(g, rg_r), _rel_l2(g, rg)
    print(f"\ntc {case}: forward rel L2 {e_r:.2e} (rounded oracle) {e:.2e} (plain); "
          f"gradient {g_r:.2e} / {g_e:.2e}")
    # the same rounding on both sides: what is left are operands that land on
    # the other side of a BF16 rounding boundary after FP32 summation-order
    # differences, each one unit roundoff u = 2^-9; bound 2.5 u
    u = 2.0 ** -9
    assert e_r < 2.5 * u and g_r < 2.5 * u
    assert e < 2e-2 and g_e < 2e-2
    assert abs(loss - rl) <= 1e-2 * rl
    net.close()


def test_bf16_weights_change_the_result():
    """The BF16 mode really rounds (else the two parities above would be one)."""
    dev = _dev()
    L, c0, cmax, N, H, Wd = CASES[1]
    rng = np.random.default_rng(2)
    p = (rng.standard_normal(O.num_params(L, c0, cmax)) * 0.3).astype(np.float32)
    x = torch.from_numpy(rng.standard_normal((N, 3, H, Wd)).astype(np.float32)).to(dev)
    outs = []
    for bf16 in (False, True):
        net = _net(L, c0, cmax, bf16, params=p)
        o = torch.empty((N, 2, H, Wd), dtype=torch.float32, device=dev)
        net.forward(x, o)
        outs.append(o.cpu().numpy())
        net.close()
    assert 1e-4 < _rel(outs[1], outs[0]) < 5e-2


def test_adam_step_matches_oracle():
    dev = _dev()
    L, c0, cmax, N, H, Wd = CASES[1]
    rng = np.random.default_rng(3)
    p = (rng.standard_normal(O.num_params(L, c0, cmax)) * 0.3).astype(np.float32)
    x = rng.standard_normal((N, 3, H, Wd)).astype(np.float32)
    t = rng.standard_normal((N, 2, H, Wd)).astype(np.float32)
    net = _net(L, c0, cmax, False, params=p)
    xi, ti = torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev)
    lr = 1e-3
    w = p.astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    for step in (1, 2, 3):
        _, g, _ = O.loss_and_grad(w, x.astype(np.float64), t.astype(np.float64), L, c0, cmax)
        w, m, v = O.adam_step(w, g, m, v, step, lr)
        net.train_step(xi, ti, lr)
    got = net.get_params().astype(np.float64)
    # Adam's early steps are ~lr * sign(g): compare the step, where the
    # gradient is not so small that FP32 rounding can flip its sign
    _, g0, _ = O.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), L, c0, cmax)
    sel = np.abs(g0) > 1e-3 * np.abs(g0).max()
    d_got, d_ref = got - p, w - p
    assert np.abs(d_got[sel] - d_ref[sel]).max() < 1e-2 * lr
    net.close()


def test_training_reduces_loss():
    dev = _dev()
    rng = np.random.default_rng(4)
    x = torch.from_numpy(rng.standard_normal((4, 3, 32, 32)).astype(np.float32)).to(dev)
    # a target the network can represent: half the two source channels
    t = (0.5 * x[:, 1:3]).contiguous()
    net = _net(3, 8, 16, True, seed=1)
    losses = [net.train_step(x, t, 3e-3) for _ in range(150)]
    assert losses[-1] < 0.2 * losses[0]
    net.close()


def test_images_match_oracle():
    dev = _dev()
    w = W.ellipses(100, 60, seed=5, npml=10, nrhs=1, sources="point")
    net = _net(3, 4, 4, True)
    H, Wd = net.image_shape(w.nx, w.ny)
    assert (H, Wd) == (60, 100)
    H, Wd = 64, 104
    rng = np.random.default_rng(6)
    x = rng.standard_normal((w.nx, w.ny)) + 1j * rng.standard_normal((w.nx, w.ny))
    inp = torch.full((3, H, Wd), 7.0, dtype=torch.float32, device=dev)
    tgt = torch.full((2, H, Wd), 7.0, dtype=torch.float32, device=dev)
    unit = w.dx * w.dy
    net.images(unit, torch.from_numpy(w.eps_node).to(dev), torch.from_numpy(w.b[0]).to(dev),
               torch.from_numpy(x).to(dev), inp, tgt)
    ri, rt, _ = O.images(w.eps_node, w.b[0], x, unit=unit, H=H, W=Wd)
    np.testing.assert_allclose(inp.cpu().numpy(), ri, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(tgt.cpu().numpy(), rt, rtol=1e-6, atol=1e-6 * np.abs(rt).max())
    net.close()


def _solve(w, net, x0, maxit, precision=0):
    learned = _lib()
    return learned.solve_workload(w, precision=precision, rtol=1e-12, maxit=maxit, x0=x0, net=net)


def test_learned_guess_in_solver_matches_oracle():
    """maxit = 0 returns the start itself: the network field after one
    preconditioner sweep, scaled to the minimal residual."""
    _dev()
    from oracle.fdfd import Problem
    w = W.ellipses(120, 88, seed=7, npml=12, overlap=6, interface_pml=12, nsub=2, nrhs=2, sources="mixed")
    L, c0, cmax = 3, 8, 16
    rng = np.random.default_rng(8)
    p = (rng.standard_normal(O.num_params(L, c0, cmax)) * 0.2).astype(np.float32)
    net = _net(L, c0, cmax, True, params=p)
    x, info = _solve(w, net, "learned", 0)
    from oracle.stddm import DDM
    prob = Problem.from_workload(w)
    A = prob.A
    ddm = DDM.from_workload(w, prob)
    ddm.factor()
    for q in range(w.nrhs):
        y = O.raw_guess(p.astype(np.float64), w.eps_node, w.b[q], w.dx, w.dy, L, c0, cmax, round_bf16=True)
        x0, raw, scaled, used = O.learned_start(A, ddm.apply_Minv, w.b[q].ravel(), y.ravel())
        assert info["guess_used"][q] == used
        assert abs(info["guess_raw"][q] - raw) <= 1e-4 * raw
        assert abs(info["guess_scaled"][q] - scaled) <= 1e-4
        got = x[q].cpu().numpy().ravel()
        assert np.linalg.norm(got - x0) <= 1e-4 * max(np.linalg.norm(x0), 1e-30)
        assert abs(info["r0"][q] - scaled) <= 1e-4
    net.close()


def test_nonfinite_network_falls_back_to_zero_guess():
    _dev()
    w = W.ellipses(96, 64, seed=9, npml=10, overlap=6, interface_pml=10, nsub=2, nrhs=2)
    net = _net(2, 4, 4, True)
    p = np.zeros(net.num_params(), np.float32)
    p[-1] = np.nan                       # output bias: every pixel non-finite
    net.set_params(p)
    x, info = _solve(w, net, "learned", 0)
    assert info["guess_used"] == [False, False]
    assert not x.abs().max().item()
    assert info["r0"] == [1.0, 1.0]
    net.close()


def test_zero_network_start_is_one_sweep_from_zero():
    """With y = 0 the start is alpha M^-1 b, the first iterate of the method."""
    _dev()
    from oracle.fdfd import Problem
    from oracle.stddm import DDM
    w = W.ellipses(96, 64, seed=9, npml=10, overlap=6, interface_pml=10, nsub=2, nrhs=1)
    net = _net(2, 4, 4, True)
    net.set_params(np.zeros(net.num_params(), np.float32))
    x, info = _solve(w, net, "learned", 0)
    prob = Problem.from_workload(w)
    ddm = DDM.from_workload(w, prob)
    ddm.factor()
    x0, _, scaled, used = O.learned_start(prob.A, ddm.apply_Minv, w.b[0].ravel(), np.zeros(w.n, complex))
    assert used and info["guess_used"] == [True]
    assert abs(info["r0"][0] - scaled) <= 1e-9
    got = x[0].cpu().numpy().ravel()
    assert np.linalg.norm(got - x0) <= 1e-9 * np.linalg.norm(x0)
    net.close()


def test_learned_guess_without_network_is_a_state_error():
    _dev()
    from paper_2509_20801_gb300 import binding as B
    w = W.ellipses(96, 64, seed=9, npml=10, overlap=6, interface_pml=10, nsub=2, nrhs=1)
    with pytest.raises(B.StddError) as e:
        _solve(w, None, "learned", 5)
    assert e.value.status == B.STDD_ESTATE


def test_learned_start_reaches_the_same_solution():
    _dev()
    from oracle.fdfd import Problem
    w = W.ellipses(120, 88, seed=10, npml=12, overlap=6, interface_pml=12, nsub=2, nrhs=1, sources="point")
    L, c0, cmax = 3, 8, 16
    rng = np.random.default_rng(11)
    net = _net(L, c0, cmax, True, params=(rng.standard_normal(O.num_params(L, c0, cmax)) * 0.2).astype(np.float32))
    x, info = _solve(w, net, "learned", 300)
    assert info["converged"]
    ref = Problem.from_workload(w).solve(w.b[0].ravel())
    got = x[0].cpu().numpy().ravel()
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)
    net.close()


def test_trained_network_gains_over_zero_guess():
    """Train a small network on fields the DDM computes for seeded ellipse
    geometries, then solve held-out geometries from the zero start and from
    the learned start.  Training must lower the loss and the network's field
    error on the held-out problems; the learned start (which spends one
    preconditioner application of its own) must cost at most that one
    application on average, and both starts must reach the same field.  The
    measured counts are printed: the gain is small, because one sweep of the
    method already removes most of what a guess of this accuracy offers."""
    _dev()
    learned = _lib()
    kw = dict(npml=16, overlap=8, interface_pml=16, nsub=2, sources="mixed")
    train_w = [W.ellipses(128, 128, seed=1000 + s, nrhs=4, **kw) for s in range(32)]
    test_w = [W.ellipses(128, 128, seed=2000 + s, nrhs=2, **kw) for s in range(6)]
    net = learned.Network(4, 16, 64, mode="tc", seed=3)
    H, Wd = net.image_shape(128, 128)
    ref = [learned.solve_workload(w, precision=0, rtol=1e-10)[0] for w in test_w]
    e0 = learned.field_error(net, test_w, ref)
    inp, tgt, _ = learned.make_dataset(net, train_w, H, Wd)
    losses = learned.train(net, inp, tgt, epochs=60, batch=8, lr=2e-3, lr_final=2e-4, seed=0)
    e1 = learned.field_error(net, test_w, ref)
    rows = learned.compare(net, test_w, precision=1, rtol=1e-8)
    s1 = np.array([r["guess_scaled"] for r in rows])
    iz = np.array([r["minv_zero"] for r in rows])
    il = np.array([r["minv_learned"] for r in rows])
    print(f"\nloss {np.mean(losses[:16]):.3e} -> {np.mean(losses[-16:]):.3e}; held-out field error "
          f"{np.median(e0):.3f} -> {np.median(e1):.3f}; start residual {np.median(s1):.3f}; "
          f"preconditioner applications zero {iz.tolist()} learned {il.tolist()}")
    assert np.mean(losses[-16:]) < 0.5 * np.mean(losses[:16])
    assert np.median(e1) < 0.9 * np.median(e0)
    assert all(r["conv_zero"] and r["conv_learned"] for r in rows)
    assert il.mean() <= iz.mean() + 1
    for r in rows:
        a, b = r["x_learned"].cpu().numpy(), r["x_zero"].cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
    net.close()
