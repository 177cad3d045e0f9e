"""Learned initial guess: the network object, training-data generation with
the solver itself, training, and the comparison with the zero guess.

Every numerical step runs in libstdd.so (network forward/backward/Adam,
image preparation, the DDM solves); torch provides device memory only.
The network is described in include/stdd.h (stdd_nn_*)."""
from __future__ import annotations

import time

import numpy as np

from . import binding as _b


class Network:
    """Encoder-decoder guess network on one GPU (see stdd_nn_create)."""

    MODES = {"fp32": _b.STDD_NN_FP32, "bf16": _b.STDD_NN_BF16, "tc": _b.STDD_NN_TC}

    def __init__(self, levels=6, base_channels=32, max_channels=256, mode="tc", seed=0, device=0, stream=None):
        self.levels, self.base, self.cmax = int(levels), int(base_channels), int(max_channels)
        self.mode = mode
        self.device = int(device)
        self.h = _b.stdd_nn_create(device, stream, levels, base_channels, max_channels, self.MODES[mode], seed)

    @property
    def multiple(self):
        """Image sides must be multiples of this."""
        return 1 << (self.levels - 1)

    def num_params(self):
        return _b.stdd_nn_num_params(self.h)

    def get_params(self):
        return _b.stdd_nn_get_params(self.h)

    def set_params(self, p):
        _b.stdd_nn_set_params(self.h, p)

    def save(self, path):
        np.savez(path, params=self.get_params(), levels=self.levels, base=self.base, cmax=self.cmax,
                 mode=self.mode)

    @classmethod
    def load(cls, path, device=0, stream=None):
        z = np.load(path)
        net = cls(int(z["levels"]), int(z["base"]), int(z["cmax"]), str(z["mode"]), device=device, stream=stream)
        net.set_params(z["params"])
        return net

    def forward(self, inp, out):
        _b.stdd_nn_forward(self.h, inp, out)

    def gradient(self, inp, target):
        return _b.stdd_nn_gradient(self.h, inp, target)

    def train_step(self, inp, target, lr):
        return _b.stdd_nn_train_step(self.h, inp, target, lr)

    def images(self, unit, eps, b, x, inp, target=None):
        _b.stdd_nn_make_images(self.h, unit, eps, b, x, inp, target)

    def image_shape(self, nx, ny):
        f = self.multiple
        return -(-ny // f) * f, -(-nx // f) * f

    def close(self):
        if self.h is not None:
            _b.stdd_nn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _solver(w, precision, device):
    from . import Solver
    import torch
    dev = torch.device("cuda", device)
    eps = torch.from_numpy(w.eps_node).to(dev)
    s = Solver.from_workload(w, eps=eps, precision=precision, device=device)
    return s, eps


def solve_workload(w, precision=_b.STDD_PREC_FP64, rtol=None, restart=None, maxit=1000, device=0, x0=None,
                   net=None):
    """Factor and solve every right-hand side of workload w on the GPU.
    Returns (x [nrhs, nx, ny] complex128 device tensor, info dict)."""
    import torch
    dev = torch.device("cuda", device)
    s, eps = _solver(w, precision, device)
    try:
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        s.factor()
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        b = torch.from_numpy(w.b).to(dev)
        s.set_sources(b)
        if net is not None:
            _b.stdd_set_learned_guess(s.ctx, net.h)
        x = torch.empty_like(b)
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        st = s.solve(x, restart=restart or w.restart, rtol=rtol or w.rtol, maxit=maxit, x0=x0,
                     allow_noconv=True)
        torch.cuda.synchronize(dev)
        t3 = time.perf_counter()
        hist = [s.history(q) for q in range(w.nrhs)]
        info = dict(factor_s=t1 - t0, solve_s=t3 - t2, converged=st == _b.STDD_OK,
                    iterations=[len(h) - 1 for h in hist], r0=[float(h[0]) for h in hist],
                    final=[float(h[-1]) for h in hist])
        if x0 == "learned":
            g = [_b.stdd_learned_guess_info(s.ctx, q) for q in range(w.nrhs)]
            info["guess_raw"] = [a for a, _, _ in g]
            info["guess_scaled"] = [c for _, c, _ in g]
            info["guess_used"] = [u for _, _, u in g]
        return x, info
    finally:
        s.close()


def make_dataset(net, workloads, H, W, precision=_b.STDD_PREC_FP64, rtol=1e-8, device=0, log=None):
    """Solve each workload's right-hand sides with the DDM and turn every
    (eps, b, x) into a network image pair.  Returns (inputs [S, 3, H, W],
    targets [S, 2, H, W]) float32 device tensors and the solve infos."""
    import torch
    dev = torch.device("cuda", device)
    S = sum(w.nrhs for w in workloads)
    inputs = torch.zeros((S, 3, H, W), dtype=torch.float32, device=dev)
    targets = torch.zeros((S, 2, H, W), dtype=torch.float32, device=dev)
    infos, k = [], 0
    for wi, w in enumerate(workloads):
        if w.nx > W or w.ny > H:
            raise ValueError("workload larger than the image")
        x, info = solve_workload(w, precision=precision, rtol=rtol, device=device)
        infos.append(info)
        eps = torch.from_numpy(w.eps_node).to(dev)
        b = torch.from_numpy(w.b).to(dev)
        for q in range(w.nrhs):
            net.images(w.dx * w.dy, eps, b[q], x[q], inputs[k], targets[k])
            k += 1
        if log and (wi % 16 == 0 or wi + 1 == len(workloads)):
            log(f"dataset: {wi + 1}/{len(workloads)} geometries, {k} samples")
    return inputs, targets, infos


def train(net, inputs, targets, epochs=10, batch=8, lr=1e-3, lr_final=None, seed=0, log=None):
    """Adam on the mean squared error, shuffled mini-batches (samples are
    copied into one batch buffer).  lr decays geometrically to lr_final.
    Returns the per-step losses."""
    import torch
    S = inputs.shape[0]
    batch = min(batch, S)
    rng = np.random.default_rng(seed)
    bi = torch.empty((batch,) + tuple(inputs.shape[1:]), dtype=inputs.dtype, device=inputs.device)
    bt = torch.empty((batch,) + tuple(targets.shape[1:]), dtype=targets.dtype, device=targets.device)
    steps = epochs * (S // batch)
    lr_final = lr if lr_final is None else lr_final
    decay = (lr_final / lr) ** (1.0 / max(1, steps - 1))
    losses, step = [], 0
    for ep in range(epochs):
        perm = rng.permutation(S)
        for k0 in range(0, S - batch + 1, batch):
            for j, i in enumerate(perm[k0:k0 + batch]):
                bi[j].copy_(inputs[int(i)])
                bt[j].copy_(targets[int(i)])
            losses.append(net.train_step(bi, bt, lr * decay ** step))
            step += 1
        if log:
            log(f"epoch {ep + 1}/{epochs}: loss {np.mean(losses[-max(1, S // batch):]):.4e}")
    return losses


def field_error(net, workloads, fields, device=0):
    """Relative L2 error of the network's field against solved fields, per
    right-hand side, in the network's normalised units (image pixels outside
    the grid are zero on both sides)."""
    import torch
    dev = torch.device("cuda", device)
    errs = []
    for w, x in zip(workloads, fields):
        H, Wd = net.image_shape(w.nx, w.ny)
        inp = torch.empty((1, 3, H, Wd), dtype=torch.float32, device=dev)
        tgt = torch.empty((1, 2, H, Wd), dtype=torch.float32, device=dev)
        out = torch.empty((1, 2, H, Wd), dtype=torch.float32, device=dev)
        eps = torch.from_numpy(w.eps_node).to(dev)
        b = torch.from_numpy(w.b).to(dev)
        for q in range(w.nrhs):
            net.images(w.dx * w.dy, eps, b[q], x[q], inp[0], tgt[0])
            net.forward(inp, out)
            errs.append(float(torch.linalg.vector_norm(out - tgt) / torch.linalg.vector_norm(tgt)))
    return errs


def compare(net, workloads, precision=_b.STDD_PREC_C64, rtol=1e-8, restart=None, maxit=1000, device=0):
    """Solve each workload with the zero start and with the learned start on
    the same factorization (same precision and tolerance); per right-hand
    side: iterations, preconditioner applications, solve times (CUDA events)
    and the start's residuals."""
    import torch
    dev = torch.device("cuda", device)
    rows = []
    for w in workloads:
        s, _ = _solver(w, precision, device)
        try:
            s.factor()
            b = torch.from_numpy(w.b).to(dev)
            s.set_sources(b)
            _b.stdd_set_learned_guess(s.ctx, net.h)
            res = {}
            for mode in (None, "learned"):
                x = torch.empty_like(b)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize(dev)
                e0.record()
                st = s.solve(x, restart=restart or w.restart, rtol=rtol, maxit=maxit, x0=mode, allow_noconv=True)
                e1.record()
                torch.cuda.synchronize(dev)
                hist = [s.history(q) for q in range(w.nrhs)]
                info = dict(x=x, ms=e0.elapsed_time(e1), ok=st == _b.STDD_OK, its=[len(h) - 1 for h in hist])
                if mode:
                    info["g"] = [_b.stdd_learned_guess_info(s.ctx, q) for q in range(w.nrhs)]
                res[mode] = info
        finally:
            s.close()
        z, l = res[None], res["learned"]
        for q in range(w.nrhs):
            rows.append(dict(nx=w.nx, ny=w.ny, seed=w.meta.get("seed"), rhs=q,
                             its_zero=z["its"][q], its_learned=l["its"][q],
                             # preconditioner applications: the learned start spends one sweep
                             minv_zero=z["its"][q], minv_learned=l["its"][q] + 1,
                             solve_s_zero=z["ms"] / 1e3 / w.nrhs, solve_s_learned=l["ms"] / 1e3 / w.nrhs,
                             guess_raw=l["g"][q][0], guess_scaled=l["g"][q][1], guess_used=l["g"][q][2],
                             conv_zero=z["ok"], conv_learned=l["ok"], x_zero=z["x"][q], x_learned=l["x"][q]))
    return rows


def experiment(n_train=4000, train_side=512, n_eval=256, eval_shape=(1024, 512), levels=6, base=32, cmax=256,
               train_seconds=300.0, batch=8, lr=1e-3, lr_final=1e-4, rhs_per_geometry=8, train_seed=4,
               eval_seed=5, precision=_b.STDD_PREC_C64, rtol=1e-8, device=0, log=print):
    """Train a guess network on fields the FP64 DDM computes for seeded
    ellipse geometries (n_train fields, rhs_per_geometry random point or line
    sources per geometry, train_side^2 grids), then compare zero and learned
    starts on n_eval held-out instances of eval_shape (one source each) at
    the given precision and tolerance.  Geometry g of a set uses seed
    set_seed * 1_000_000 + g.  Returns a summary dict."""
    import torch
    import workloads as W
    t_all = time.perf_counter()
    net = Network(levels, base, cmax, mode="tc", seed=train_seed, device=device)
    n_geo = -(-n_train // rhs_per_geometry)
    train_w = [W.ellipses(train_side, train_side, seed=train_seed * 1_000_000 + g, nrhs=rhs_per_geometry)
               for g in range(n_geo)]
    H, Wd = net.image_shape(train_side, train_side)
    t0 = time.perf_counter()
    inp, tgt, infos = make_dataset(net, train_w, H, Wd, precision=_b.STDD_PREC_FP64, rtol=rtol, device=device,
                                   log=log)
    t_data = time.perf_counter() - t0
    inp, tgt = inp[:n_train], tgt[:n_train]
    # epochs from the time budget, measured on the first steps
    bi, bt = inp[:batch].contiguous(), tgt[:batch].contiguous()
    net.train_step(bi, bt, 1e-7)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        net.train_step(bi, bt, 1e-7)
    torch.cuda.synchronize()
    t_step = (time.perf_counter() - t0) / 3
    epochs = max(1, int(train_seconds / (t_step * (n_train // batch))))
    t0 = time.perf_counter()
    losses = train(net, inp, tgt, epochs=epochs, batch=batch, lr=lr, lr_final=lr_final, seed=train_seed, log=log)
    t_train = time.perf_counter() - t0
    del inp, tgt, bi, bt
    torch.cuda.empty_cache()
    nx, ny = eval_shape
    eval_w = [W.ellipses(nx, ny, seed=eval_seed * 1_000_000 + g, nrhs=1) for g in range(n_eval)]
    rows = compare(net, eval_w, precision=precision, rtol=rtol, device=device)
    ref = [r["x_zero"][None] for r in rows]
    ferr = field_error(net, eval_w, ref, device=device)
    iz = np.array([r["its_zero"] for r in rows])
    il = np.array([r["its_learned"] for r in rows])
    tz = np.array([r["solve_s_zero"] for r in rows])
    tl = np.array([r["solve_s_learned"] for r in rows])
    used = np.array([r["guess_used"] for r in rows])
    # forward time of the network at the evaluation size
    Hh, Ww = net.image_shape(nx, ny)
    xi = torch.zeros((1, 3, Hh, Ww), dtype=torch.float32, device=f"cuda:{device}")
    xo = torch.empty((1, 2, Hh, Ww), dtype=torch.float32, device=f"cuda:{device}")
    for _ in range(3):
        net.forward(xi, xo)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(10):
        net.forward(xi, xo)
    torch.cuda.synchronize()
    t_fwd = (time.perf_counter() - t0) / 10
    summary = dict(
        network=dict(levels=levels, base_channels=base, max_channels=cmax, params=net.num_params(), mode="tc"),
        train=dict(fields=int(n_train), side=train_side, geometries=n_geo, epochs=epochs, batch=batch,
                   step_ms=t_step * 1e3, data_s=t_data, train_s=t_train, loss_first=float(np.mean(losses[:50])),
                   loss_last=float(np.mean(losses[-50:])), ddm_iterations_mean=float(
                       np.mean([np.mean(i["iterations"]) for i in infos]))),
        eval=dict(instances=len(rows), shape=list(eval_shape), precision=int(precision), rtol=rtol,
                  field_error_median=float(np.median(ferr)), start_residual_median=float(
                      np.median([r["guess_scaled"] for r in rows])), used_fraction=float(used.mean()),
                  its_zero_mean=float(iz.mean()), its_learned_mean=float(il.mean()),
                  minv_zero_mean=float(iz.mean()), minv_learned_mean=float(il.mean() + 1),
                  solve_ms_zero_mean=float(tz.mean() * 1e3), solve_ms_learned_mean=float(tl.mean() * 1e3),
                  forward_ms=t_fwd * 1e3, fewer_iterations_fraction=float((il + 1 < iz).mean()),
                  all_converged=bool(all(r["conv_zero"] and r["conv_learned"] for r in rows))),
        wall_s=time.perf_counter() - t_all)
    net.close()
    return summary


if __name__ == "__main__":
    import argparse
    import json
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    ap = argparse.ArgumentParser(description="train the guess network and compare it with the zero guess")
    ap.add_argument("--train", type=int, default=4000)
    ap.add_argument("--train-side", type=int, default=512)
    ap.add_argument("--eval", type=int, default=256)
    ap.add_argument("--eval-shape", default="1024x512")
    ap.add_argument("--net", default="6,32,256", help="levels,base,max channels")
    ap.add_argument("--train-seconds", type=float, default=300.0)
    ap.add_argument("--out", default=None)
    ap.add_argument("--bench-forward", default=None, metavar="WxH",
                    help="only time the network forward at this image size (random weights) and exit")
    ap.add_argument("--bench-train", default=None, metavar="WxHxB",
                    help="only time training steps (forward, backward, Adam) on B images of W x H and exit")
    ap.add_argument("--mode", default="tc", choices=("tc", "bf16", "fp32"))
    a = ap.parse_args()
    if a.bench_forward or a.bench_train:
        import torch
        L, c0, cm = (int(v) for v in a.net.split(","))
        spec = [int(v) for v in (a.bench_forward or a.bench_train).split("x")]
        fw, fh, nb = spec[0], spec[1], (spec[2] if len(spec) > 2 else 1)
        net = Network(L, c0, cm, mode=a.mode)
        fh, fw = net.image_shape(fw, fh)
        xi = torch.randn((nb, 3, fh, fw), dtype=torch.float32, device="cuda:0")
        xo = torch.randn((nb, 2, fh, fw), dtype=torch.float32, device="cuda:0")
        if a.bench_forward:
            step = lambda: net.forward(xi, xo)  # noqa: E731
        else:
            xo.mul_(0.1)
            step = lambda: net.train_step(xi, xo, 1e-4)  # noqa: E731
        for _ in range(3):
            step()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(10):
            step()
        ev[1].record()
        torch.cuda.synchronize()
        flops = 0
        ch = [min(cm, c0 << lv) for lv in range(L)]
        for lv in range(L):
            px = (fh >> lv) * (fw >> lv)
            cin = 3 if lv == 0 else ch[lv - 1]
            flops += 2 * 9 * px * (cin * ch[lv] + ch[lv] * ch[lv])
            if lv < L - 1:
                flops += 2 * 9 * px * (ch[lv + 1] * ch[lv] + ch[lv] * ch[lv])
        flops += 2 * 9 * fh * fw * ch[0] * 2
        flops *= nb
        ms = ev[0].elapsed_time(ev[1]) / 10
        if a.bench_forward:
            print(json.dumps(dict(image=[fw, fh], mode=a.mode, forward_ms=ms, conv_gflop=flops / 1e9,
                                  tflops=flops / ms / 1e9)))
        else:
            # forward, input gradient and weight gradient: three times the
            # forward's convolution work
            print(json.dumps(dict(image=[fw, fh], batch=nb, mode=a.mode, train_step_ms=ms,
                                  conv_gflop=3 * flops / 1e9, tflops=3 * flops / ms / 1e9)))
        net.close()
        sys.exit(0)
    L, c0, cm = (int(v) for v in a.net.split(","))
    ex, ey = (int(v) for v in a.eval_shape.split("x"))
    res = experiment(a.train, a.train_side, a.eval, (ex, ey), L, c0, cm, a.train_seconds,
                     log=lambda m: print(m, file=sys.stderr, flush=True))
    line = json.dumps(res)
    print(line)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")
