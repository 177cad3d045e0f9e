#!/usr/bin/env python
"""Benchmark of the GB300 overlapping source-transfer DDM solver.

One step = the whole hot path on one synthetic problem whose inputs are
already in HBM: numeric multifrontal factorization of every strip, then
flexible GMRES(50) preconditioned by the batched source-transfer sweep until
the relative residual is <= 1e-8.  Default workload: the mixed-precision
single large instance, a waveguide network of 8192 x 2048 nodes (16.8 M
unknowns) at lambda/24 with 32-cell PML and 32 strips (overlap 16), excited
by its input guide's fundamental mode; the main line is the plain FP64 form
(complex128 factors, symmetric multiplicative strip order, the fastest FP64
order on this workload), and the mixed forms (complex64 factors, FP32 or
FP16 tensor-core front updates, FP64 Krylov) are measured beside it on the
same problem with their difference from the FP64 field.

Printed: one JSON line (rank 0).  value = MDoF/s = nx*ny*nrhs / (seconds per
step) / 1e6, summed over ranks (replicas, weak scaling).

The CPU baseline (and --impl reference) runs the CPU oracle -- SuperLU
factors of every strip and the oracle's textbook FGMRES to 1e-8 with the
additive (Algorithm 1) preconditioner -- on the host cores, one process per
group of strips (the paper's parallel axis), on a shrunk instance of the same
generator.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solve time to 1e-8 residual & MDoF/s: mixed/learned vs plain FP64, one GB300"
RTOL = 1e-8
RESTART = 50
FP64_NOMINAL_TFLOPS = 1.25     # GB300 FP64 (non-tensor and tensor), NVIDIA's figure

# DRAM bytes (read + write) of a kernel per unit of its work -- per executed
# flop for the elimination kernels, per algorithmic byte for the substitution
# sweeps, per BF16 tensor flop for the split update -- from ncu captures on
# the 2048 x 512 waveguide network (the traffic grows with the work, so it
# scales to the benchmark's launches); used only while the kernel's source
# text (between the two markers) still has the recorded SHA-256, else the
# roofline's traffic is null.
_MF = "paper_2509_20801_gb300/csrc/kernels_mf.cu"
_SWEEP = ("// ------------------------------------------------------- substitutions",
          "// ------------------------------------------- persistent one-strip sweep",
          "56a3ddad56c1f20446e6d2e928c83d1a8237b30558a874c4064731bfcb59327c")
NCU_TRAFFIC = {
    "mf_gj_update<double>": {
        "dram_per_unit": 1394.992640e6 / 11.533996032e9,   # 3 launches: DRAM bytes / executed flops
        "source": _MF,
        "begin": "// acc[4][4] += A(64 x K) B(K x 64)",
        "end": "// ------------------------------------------------------- substitutions",
        "sha256": "6decf2105b755b886e043790beeea94ba39fdd151acf1da500560430b40715db",
        "profile": "profiles/ncu_dram_mf_gj_update_fp64_waveguide_2048x512.md",
    },
    "mf_gj_update_sym<double>": {
        "dram_per_unit": 1036.804608e6 / 5.778714624e9,    # 3 launches: DRAM bytes / executed flops
        "source": _MF,
        "begin": "// Symmetric form: the update of step k",
        "end": "// acc[4][4] += A(64 x K) B(K x 64)",
        "sha256": "e5e1aff1ceb0885192828b398982ea8200ca281f09b33292924e2efb99982387",
        "profile": "profiles/ncu_dram_mf_gj_update_sym_fp64_waveguide_2048x512.md",
    },
    "mf_gj_update_oz": {
        "dram_per_unit": 349.049344e6 / 86.06711808e9,     # 1 launch: DRAM bytes / BF16 tensor flops
        "source": "paper_2509_20801_gb300/csrc/kernels_tc.cu",
        "begin": "// ===================================================== FP64 on BF16 units",
        "end": "// The column panel of step k on the tensor cores",
        "sha256": "4c31819e1882c3b1aa455134b4bf67896c3454260ddbcf587c3c4b87e728a8c4",
        "profile": "profiles/ncu_mf_gj_update_oz_fp64_waveguide_2048x512.md",
    },
    "mf_down<double>": {
        "dram_per_unit": 158.460e6 / 131.123e6,   # one strip solve's 14 launches: DRAM bytes / factor bytes
        "source": _MF, "begin": _SWEEP[0], "end": _SWEEP[1], "sha256": _SWEEP[2],
        "profile": "profiles/ncu_dram_mf_down_fp64_waveguide_2048x512.md",
    },
}


def ncu_traffic(kernel, units_per_launch):
    import hashlib
    rec = NCU_TRAFFIC.get(kernel)
    if not rec or not units_per_launch:
        return None
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), rec["source"])
    try:
        with open(path) as f:
            src = f.read()
        a, b = src.index(rec["begin"]), src.index(rec["end"])
        if hashlib.sha256(src[a:b].encode()).hexdigest() != rec["sha256"]:
            return None
    except (OSError, ValueError):
        return None
    return rec["dram_per_unit"] * units_per_launch


FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x FMA x max clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "c64", "bf16", "fp16"],
                    help="factor precision: complex128, complex64, or complex64 with tensor-core (tcgen05) "
                         "front updates from BF16 / FP16 inputs")
    ap.add_argument("--workload", default="waveguide",
                    choices=["waveguide", "waveguide-small", "metalens", "metalens-small", "cylinder"],
                    help="waveguide: 8192x2048 network, 32 strips (the benchmark); waveguide-small: 2048x512, "
                         "8 strips (profiling captures); metalens: 4096x1024, 16 strips; metalens-small: "
                         "1024x1024, 4 strips; cylinder: 200x200, 2 strips")
    ap.add_argument("--nrhs", type=int, default=1, help="right-hand sides per step (metalens: line sources)")
    ap.add_argument("--leaf", type=int, default=16, help="nested-dissection leaf size (nodes)")
    ap.add_argument("--band", type=int, default=None, choices=[0, 1],
                    help="1: band-space FGMRES (FP64 factors, additive order; same iterates, band-sized "
                         "vectors); default 1 where it applies")
    ap.add_argument("--order", default=None, choices=["additive", "multiplicative", "red-black", "forward"],
                    help="preconditioner order (default: multiplicative on the waveguide, additive -- "
                         "Algorithm 1 -- elsewhere)")
    ap.add_argument("--static-pivot", type=int, default=None,
                    help="static-pivot exponent of the tensor-core (FP16 / BF16) forms (default 2 on the "
                         "waveguide, else 0)")
    ap.add_argument("--pivoting", type=int, default=None, choices=[0, 1],
                    help="partial pivoting within the fronts for the complex64 forms (default 1 on the "
                         "waveguide, else 0)")
    ap.add_argument("--symmetric", type=int, default=1, choices=[0, 1, 2],
                    help="1: factor the symmetric form D A of each strip (lower-triangle front updates) for "
                         "complex128 factors without partial pivoting; 2: complex64 factors too")
    ap.add_argument("--fp64-tc", type=int, default=1, choices=[0, 1],
                    help="1: complex128 symmetric-form front updates and column panels on the BF16 tensor cores "
                         "by exact splitting (FP64 accuracy); 0: the FP64 pipe")
    ap.add_argument("--sweep-split", type=int, default=0, choices=[0, 1, 2, 4, 8, 16],
                    help="substitution products: 0 tuned per level, k warps of a block per item, 16 across the grid")
    ap.add_argument("--maxit", type=int, default=2000, help="FGMRES iteration limit per right-hand side")
    ap.add_argument("--graphs", type=int, default=1, choices=[0, 1],
                    help="1: replay captured CUDA graphs of the factorization and of M^-1")
    ap.add_argument("--persistent", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="k > 0: one persistent launch (k blocks per SM) per strip solve in the sequential orders; "
                         "0: per-level launches; -1: the library's choice by precision")
    ap.add_argument("--no-compare", action="store_true", help="skip the other-precision and other-order runs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3, help="timed steps of the end-to-end run")
    return ap.parse_args()


def make_workload(name, nrhs=1):
    import workloads as W
    if name == "waveguide":
        return W.waveguide_network()
    if name == "waveguide-small":
        return W.waveguide_network(2048, 512, nsub=8)
    if name == "metalens":
        return W.metalens(nrhs=nrhs)
    if name == "metalens-small":
        return W.metalens(nx=1024, ny=1024, nsub=4, nrhs=nrhs)
    return W.cylinder()


def cpu_sample_workload(name, small=False):
    """(workload, description) of the CPU oracle's sample: the same generator
    shrunk (strip widths kept, fewer strips and rows)."""
    import workloads as W
    if name.startswith("waveguide"):
        nx, ny, ns = (1024, 384, 4) if small else (2048, 512, 8)
        return W.waveguide_network(nx, ny, nsub=ns), f"waveguide network shrunk to {nx}x{ny}, {ns} strips"
    if name.startswith("metalens"):
        nx, ny, ns = (512, 256, 2) if small else (1024, 512, 4)
        return W.metalens(nx=nx, ny=ny, nsub=ns), f"metalens shrunk to {nx}x{ny}, {ns} strips"
    return W.cylinder(), "cylinder 200x200, 2 strips"


def workload_desc(w):
    return (f"{w.name} {w.nx}x{w.ny} grid ({w.n} DoF) at lambda/{round(w.wavelength / w.dx)}, "
            f"{w.npml[0]}-cell SC-PML m={w.pml_order} R={w.pml_R:g}, {w.nsub} strips, overlap "
            f"{w.overlap}, interface PML {w.interface_pml}, {w.nrhs} RHS")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ peaks
def measured_peaks():
    peaks = {"hbm_gbs": 6800.0, "source_hbm": "fallback", "bf16_tflops": 1900.0, "source_bf16": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        peaks["hbm_gbs"] = float(mp["hbm_gbs"])
        peaks["source_hbm"] = "measured (MEASURED_PEAKS.json, copy)"
        peaks["bf16_tflops"] = float(mp["bf16_tflops_sustained"])
        peaks["source_bf16"] = "measured (MEASURED_PEAKS.json, cuBLAS bf16 sustained; FP16 dense rate is the same)"
    except (OSError, KeyError, ValueError):
        pass
    return peaks


def gemm_peak(torch, dtype, n, reps=3):
    """Dense GEMM throughput through cuBLAS (TFLOP/s), best of reps."""
    a = torch.randn(n, n, dtype=dtype, device="cuda")
    b = torch.randn(n, n, dtype=dtype, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        torch.matmul(a, b)
        e.record()
        e.synchronize()
        best = max(best, 2.0 * n ** 3 / (s.elapsed_time(e) * 1e-3) / 1e12)
    del a, b
    return best


# ------------------------------------------------------------- CPU oracle
def _oracle_worker(conn, prob_kw, ddm_kw, strips, shm_in, shm_out, offs):
    """One host process of the CPU baseline: it holds the oracle's strip
    operators for `strips` and serves requests from the parent: "factor"
    (assemble and SuperLU-factor its strips from scratch) and "solve" (local
    solutions of the shared input vector into the shared output buffer)."""
    import numpy as np
    from multiprocessing import shared_memory

    from oracle.fdfd import Problem
    from oracle.stddm import DDM
    P = Problem(**prob_kw)
    D = DDM(P, **ddm_kw)
    si = shared_memory.SharedMemory(name=shm_in)
    so = shared_memory.SharedMemory(name=shm_out)
    vin = np.ndarray((P.n,), np.complex128, buffer=si.buf)
    vout = np.ndarray((offs[-1],), np.complex128, buffer=so.buf)
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg == "factor":
            for k in strips:
                D._lu[k] = None
                D._A_loc[k] = None
                D.factor(k)
            conn.send("done")
        elif msg == "solve":
            for k in strips:
                vout[offs[k]:offs[k + 1]] = D.local_solve(k, D.restrict_owned(k, vin))
            conn.send("done")
        else:
            break
    del vin, vout
    si.close()
    so.close()


class ParallelOracle:
    """The CPU oracle's strip method on the host cores: SuperLU factors of
    every strip (oracle.stddm.DDM) spread over worker processes (started with
    spawn, before or after CUDA is initialised), the additive
    preconditioner M^-1 v = sum_i E_i A_i^-1 R_i^I v with the strips' local
    solves run in parallel, the global operator and FGMRES of the oracle
    (oracle.krylov.gmres) in the parent."""

    def __init__(self, w, procs=None):
        import multiprocessing as mp
        from multiprocessing import shared_memory

        import numpy as np

        from oracle.fdfd import Problem
        from oracle.stddm import DDM
        self.w = w
        prob_kw = dict(nx=w.nx, ny=w.ny, dx=w.dx, dy=w.dy, wavelength=w.wavelength, eps_node=w.eps_node,
                       npml=w.npml, pml_order=w.pml_order, pml_R=w.pml_R)
        ddm_kw = dict(nsub=w.nsub, overlap=w.overlap, interface_pml=w.interface_pml)
        self.P = Problem(**prob_kw)
        self.D = DDM(self.P, **ddm_kw)
        self.A = self.P.A.tocsr()
        ny = w.ny
        self.offs = [0]
        for st in self.D.strips:
            self.offs.append(self.offs[-1] + st.width * ny)
        ncpu = os.cpu_count() or 1
        self.procs = max(1, min(w.nsub, ncpu if procs is None else procs))
        self.shm_in = shared_memory.SharedMemory(create=True, size=16 * w.n)
        self.shm_out = shared_memory.SharedMemory(create=True, size=16 * self.offs[-1])
        self.vin = np.ndarray((w.n,), np.complex128, buffer=self.shm_in.buf)
        self.vout = np.ndarray((self.offs[-1],), np.complex128, buffer=self.shm_out.buf)
        ctx = mp.get_context("spawn")
        self.conns, self.workers = [], []
        # one thread per worker: SuperLU's BLAS threads in several processes
        # at once oversubscribe the cores and stall (the spawned children
        # read these variables when they load numpy)
        saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
        os.environ.update({k: "1" for k in saved})
        try:
            self._start(ctx, prob_kw, ddm_kw)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        try:
            for c in self.conns:
                if self._recv(c, 600) != "ready":
                    raise RuntimeError("oracle worker failed to start")
        except Exception:
            self.close()
            raise

    def _start(self, ctx, prob_kw, ddm_kw):
        w = self.w
        for r in range(self.procs):
            ks = list(range(r, w.nsub, self.procs))
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, prob_kw, ddm_kw, ks, self.shm_in.name,
                                                         self.shm_out.name, self.offs), daemon=True)
            p.start()
            b.close()          # the child holds its end: a dead child then ends recv() with EOFError
            self.conns.append(a)
            self.workers.append(p)

    @staticmethod
    def _recv(c, timeout):
        if not c.poll(timeout):
            raise RuntimeError("oracle worker did not answer within %d s" % timeout)
        return c.recv()

    def _all(self, msg):
        for c in self.conns:
            c.send(msg)
        for c in self.conns:
            self._recv(c, 3600)

    def minv(self, v):
        import numpy as np
        self.vin[:] = v
        self._all("solve")
        out = np.zeros(self.w.n, np.complex128)
        ny = self.w.ny
        for k, st in enumerate(self.D.strips):
            out[st.x0 * ny:st.x1 * ny] += self.vout[self.offs[k]:self.offs[k + 1]]
        return out

    def step(self, rtol=RTOL, restart=RESTART, maxit=2000):
        """Factor every strip, then FGMRES to rtol; returns (seconds,
        factor seconds, iterations, final true relative residual)."""
        import numpy as np

        from oracle.krylov import gmres
        t0 = time.perf_counter()
        self._all("factor")
        t1 = time.perf_counter()
        b = self.w.b[0].ravel()
        x, hist, its = gmres(lambda z: self.A @ z, self.minv, b, restart=restart, rtol=rtol, maxit=maxit)
        t2 = time.perf_counter()
        res = float(np.linalg.norm(b - self.A @ x) / np.linalg.norm(b))
        return t2 - t0, t1 - t0, its, res

    def close(self):
        for c in self.conns:
            try:
                c.send("stop")
            except (OSError, BrokenPipeError):
                pass
        for p in self.workers:
            p.join(timeout=10)
            if p.is_alive():
                p.terminate()
        del self.vin, self.vout
        self.shm_in.close()
        self.shm_in.unlink()
        self.shm_out.close()
        self.shm_out.unlink()


def host_info():
    ram = None
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemTotal:"):
                    ram = round(int(ln.split()[1]) / 2 ** 20, 1)
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "host_ram_gib": ram}


def cpu_baseline(name, small=False, steps=1, warmup=0):
    """Time the CPU oracle (ParallelOracle) on the shrunk sample of workload
    `name`: `warmup` untimed steps, then the median of `steps` timed ones."""
    w, desc = cpu_sample_workload(name, small)
    po = ParallelOracle(w)
    try:
        for _ in range(warmup):
            po.step()
        rows = [po.step() for _ in range(steps)]
    finally:
        po.close()
    t = statistics.median(r[0] for r in rows)
    last = rows[-1]
    info = host_info()
    return dict(value=w.n * w.nrhs / t / 1e6, unit="MDoF/s", cores=po.procs, kind="oracle",
                sample=(f"{desc} ({w.n} DoF): SuperLU factors of every strip + the oracle's FGMRES("
                        f"{RESTART}) with the additive preconditioner to {RTOL:g}, whole solve timed, "
                        f"{po.procs} worker processes"),
                seconds=t, factor_s=last[1], iterations=last[2], final_residual=last[3], **info)


# ----------------------------------------------------------------- ours
def stencil_phase(ms_per_call, calls_per_step, nodes, hbm_gbs, fp64_tflops, **extra):
    """Roofline of the complex128 stencil: per node 40 bytes (x, y, eps) and
    five complex multiply-adds (40 flops), about 1 flop per byte, which on a
    GPU whose FP64 rate is far below its HBM rate (GB300: ~1.1 TFLOP/s
    against ~6.8 TB/s) makes it bound by the FP64 pipe."""
    t = ms_per_call * 1e-3
    gbs = 40 * nodes / t / 1e9
    tflops = 40 * nodes / t / 1e12
    d = dict(ms_per_call=ms_per_call, calls_per_step=calls_per_step, bytes_per_call=40 * nodes,
             flops_per_call=40 * nodes, gbs=gbs, tflops=tflops, hbm_frac=gbs / hbm_gbs,
             fp64_frac=tflops / fp64_tflops,
             bound="alu" if hbm_gbs > 1000.0 * fp64_tflops else "hbm")  # 1 flop per byte vs machine balance
    d.update(extra)
    return d


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest of the ranks' values, on every rank (the value itself
    without a process group): step times are taken as the slowest rank's."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds_max, world):
    """Aggregate rate of `world` replicas that each process units_per_rank
    units in at most seconds_max seconds (weak scaling)."""
    return units_per_rank * world / seconds_max


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2509_20801_gb300 as S
    from paper_2509_20801_gb300 import binding as B

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    w = make_workload(args.workload, args.nrhs)
    N = w.n * w.nrhs
    wave = w.name.startswith("waveguide")
    if args.order is None:
        args.order = "multiplicative" if wave else "additive"
    if args.static_pivot is None:
        args.static_pivot = 2 if wave else 0
    if args.pivoting is None:
        args.pivoting = 1 if wave else 0

    def pivots_for(p):
        """(partial pivoting, static-pivot exponent) of a factor precision:
        FP64 factors take neither; complex64 factors with FP32 updates take
        partial pivoting within the fronts (no floor needed with it); the
        tensor-core forms take the static-pivot floor, which suits their
        coarser updates better than the interchanges."""
        if p == S.STDD_PREC_FP64:
            return 0, 0
        if p == S.STDD_PREC_C64:
            return args.pivoting, 0 if args.pivoting else args.static_pivot
        return 0, args.static_pivot
    peaks = measured_peaks()
    fp64_tf = gemm_peak(torch, torch.float64, 4096)
    fp32_tf = gemm_peak(torch, torch.float32, 8192)
    stream = torch.cuda.Stream(device=dev)
    eps_d = torch.from_numpy(w.eps_node).to(dev)
    b_d = torch.from_numpy(w.b).to(dev)
    x_d = torch.empty_like(b_d)
    prec = {"fp64": S.STDD_PREC_FP64, "c64": S.STDD_PREC_C64, "bf16": S.STDD_PREC_C64_BF16,
            "fp16": S.STDD_PREC_C64_FP16}[args.precision]

    orders = {"additive": 0, "multiplicative": 1, "red-black": 2, "forward": 3}

    def band_for(p, order, band):
        if band is None:
            band = 1 if args.band is None else args.band
        return 1 if (band and p == S.STDD_PREC_FP64 and order == "additive") else 0

    def make_solver(p, order=None, band=None):
        sv = S.Solver.from_workload(w, eps=eps_d, precision=p, device=local_rank, stream=stream.cuda_stream)
        order = order or args.order
        S.stdd_set_option(sv.ctx, S.STDD_OPT_ORDER, orders[order])
        if args.leaf != 16:
            S.stdd_set_option(sv.ctx, S.STDD_OPT_LEAF, args.leaf)
        S.stdd_set_option(sv.ctx, S.STDD_OPT_BAND, band_for(p, order, band))
        piv, sp = pivots_for(p)
        S.stdd_set_option(sv.ctx, S.STDD_OPT_PERSISTENT, args.persistent)
        S.stdd_set_option(sv.ctx, S.STDD_OPT_GRAPHS, args.graphs)
        S.stdd_set_option(sv.ctx, S.STDD_OPT_PIVOTING, piv)
        S.stdd_set_option(sv.ctx, S.STDD_OPT_STATIC_PIVOT, sp)
        S.stdd_set_option(sv.ctx, S.STDD_OPT_SYMMETRIC, args.symmetric)
        S.stdd_set_option(sv.ctx, S.STDD_OPT_FP64_TC, args.fp64_tc)
        if args.sweep_split:
            S.stdd_set_option(sv.ctx, S.STDD_OPT_SWEEP_SPLIT, args.sweep_split)
        return sv

    def step(sv):
        sv.factor()
        return sv.solve(x_d, restart=RESTART, rtol=RTOL, maxit=args.maxit, allow_noconv=True) == B.STDD_OK

    def timed(p, warm, steps, profile, order=None, band=None):
        """warm-up, then `steps` timed steps, with phase spans if profile >= 1
        (the M^-1 graphs stay on); with profile = 2 one more step with
        per-launch kernel spans (level 2) for the kernel rooflines."""
        sv = make_solver(p, order, band)
        sv.set_sources(b_d)
        for _ in range(warm):
            step(sv)
        torch.cuda.synchronize()
        barrier()
        B.stdd_get_profile(sv.ctx, reset=True)
        B.stdd_set_profiling(sv.ctx, 1 if profile else 0)
        kernel_step = profile == 2
        l0 = B.stdd_get_profile(sv.ctx, reset=True)["launches"]
        clocks = ClockSampler(local_rank)
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        if kernel_step:   # the main line's timed steps, for profilers' NVTX filters
            torch.cuda.nvtx.range_push("timed")
        for _ in range(steps):
            step(sv)
        if kernel_step:
            torch.cuda.nvtx.range_pop()
        e1.record(stream)
        torch.cuda.synchronize()
        ck = clocks.stop()
        ms = e0.elapsed_time(e1) / steps
        prof = B.stdd_get_profile(sv.ctx, reset=True)
        launches = prof["launches"] - l0
        st = sv.stats()
        hist = sv.history(0)
        kprof = None
        if kernel_step:
            B.stdd_set_profiling(sv.ctx, 2)
            k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k0.record(stream)
            step(sv)
            k1.record(stream)
            torch.cuda.synchronize()
            kprof = B.stdd_get_profile(sv.ctx, reset=True)
            kprof["step_ms"] = k0.elapsed_time(k1)
            B.stdd_set_profiling(sv.ctx, 0)
        return sv, ms, prof, launches, st, hist, ck, kprof

    sv, ms, prof, launches, st, hist, ck, kprof = timed(prec, args.warmup, args.steps, 2)
    its = len(hist) - 1
    x_main = x_d.clone()
    r_rel = B.stdd_residual(sv.ctx, x_d[0].reshape(-1).contiguous(), b_d[0].reshape(-1).contiguous(),
                            torch.empty(w.n, dtype=torch.complex128, device=dev))
    ms_max = max_over_ranks(ms, dist, dev)

    # phase rooflines (algorithmic bytes / flops per phase call)
    steps = args.steps
    band_main = bool(band_for(prec, args.order, None))
    E = st["factor_entries"]
    elem = 16 if prec == S.STDD_PREC_FP64 else 8
    phases = {}
    if prof["minv_calls"]:
        t = prof["minv_ms"] / prof["minv_calls"] * 1e-3
        phases["substitution_sweep"] = dict(
            ms_per_call=t * 1e3, calls_per_step=prof["minv_calls"] / steps,
            bytes_per_call=E * elem, flops_per_call=st["solve_flops"],
            gbs=E * elem / t / 1e9, tflops=st["solve_flops"] / t / 1e12)
    if prof["factor_ms"]:
        t = prof["factor_ms"] / steps * 1e-3
        phases["factorization"] = dict(ms_per_call=t * 1e3, calls_per_step=1,
                                       flops_per_call=st["factor_flops"],
                                       tflops=st["factor_flops"] / t / 1e12)
    if prof["matvec_calls"] and not band_main:
        phases["stencil_matvec"] = stencil_phase(prof["matvec_ms"] / prof["matvec_calls"],
                                                 prof["matvec_calls"] / steps, w.n, peaks["hbm_gbs"], fp64_tf)
    elif prof["matvec_calls"]:
        # band space: this span is the band operator (I + T) s, i.e. a band
        # application of M^-1 plus the band stencil; the full stencil's rate
        # is taken from the full-space comparison step below
        t = prof["matvec_ms"] / prof["matvec_calls"] * 1e-3
        phases["band_operator"] = dict(ms_per_call=t * 1e3, calls_per_step=prof["matvec_calls"] / steps)
    if prof["ortho_calls"]:
        # one classical Gram-Schmidt pass at basis size m = j+1: a multi-dot
        # (m N complex multiply-adds, reading m+1 vectors) and a multi-axpy
        # (m N, reading m+1 vectors and writing one); the first pass also
        # forms ||w||^2.  Second passes (selective reorthogonalisation) are
        # counted from the solver's statistics, assumed at the mean basis size.
        calls = prof["ortho_calls"]
        js = [j % RESTART for j in range(its)]
        extra = st.get("reorth_passes", 0)
        mean_m = sum(j + 1 for j in js) / max(1, len(js))
        fl = (sum(16 * (j + 1) * w.n for j in js) + extra * 16 * mean_m * w.n) * steps
        by = (sum(16 * (2 * (j + 1) + 3) * w.n for j in js) + extra * 16 * (2 * mean_m + 3) * w.n) * steps
        t = prof["ortho_ms"] * 1e-3
        phases["gram_schmidt"] = dict(ms_per_call=t / calls * 1e3, calls_per_step=calls / steps,
                                      reorth_passes_per_step=extra, gbs=by / t / 1e9, tflops=fl / t / 1e12)
    # per-kernel rooflines from the launch-by-launch profile: the two
    # Gauss-Jordan elimination kernels (flops, ALU-bound) and the two
    # substitution sweeps (factor bytes; FP64 arithmetic is ALU-bound on this
    # part at 0.5 flop/byte, complex64 is HBM-bound)
    alu_pk = fp64_tf if prec == S.STDD_PREC_FP64 else fp32_tf
    alu_src = "measured cuBLAS DGEMM" if prec == S.STDD_PREC_FP64 else "measured cuBLAS SGEMM"
    tensor = prec in (S.STDD_PREC_C64_BF16, S.STDD_PREC_C64_FP16)
    kernels = {}

    def add_kernel(name, ms, calls, units, kind, executed=None):
        # measured over one extra profiled step (kprof: one launch span per
        # kernel launch), so per-step figures use steps = 1.  Elimination
        # kernels: units = the LU flops of their trailing-block updates
        # (algorithmic), executed = the Gauss-Jordan flops they run.
        if not calls:
            return
        t = ms * 1e-3 / calls
        u = units / calls
        if kind == "tensor":
            k = dict(bound="tensor", achieved=u / t / 1e12, peak=peaks["bf16_tflops"], unit="TFLOP/s",
                     peak_source=peaks["source_bf16"])
        elif kind == "flops":
            k = dict(bound="alu", achieved=u / t / 1e12, peak=alu_pk, unit="TFLOP/s", peak_source=alu_src)
        elif prec == S.STDD_PREC_FP64:   # sweep, complex128: 8 flops per 16-byte entry
            k = dict(bound="alu", achieved=u / 2 / t / 1e12, peak=fp64_tf, unit="TFLOP/s",
                     peak_source="measured cuBLAS DGEMM")
        else:
            k = dict(bound="hbm", achieved=u / t / 1e9, peak=peaks["hbm_gbs"], unit="GB/s",
                     peak_source=peaks["source_hbm"])
        k.update(frac=k["achieved"] / k["peak"], ms_per_step=ms, launches_per_step=calls,
                 units_per_launch=u, unit_kind=kind, ms_per_launch=t * 1e3)
        if executed is not None:
            lu = "LDL^T flops (one triangle of each trailing-block update)" if sym else "LU flops (trailing-block updates)"
            k.update(unit_kind=lu, executed_flops_per_launch=executed / calls,
                     executed_tflops=executed / calls / t / 1e12)
        kernels[name] = k

    tname = "double" if prec == S.STDD_PREC_FP64 else "float"
    sym = bool(args.symmetric and not pivots_for(prec)[0] and not tensor and (
        prec == S.STDD_PREC_FP64 or args.symmetric == 2))
    oz = sym and args.fp64_tc and prec == S.STDD_PREC_FP64
    if oz:
        # the split products on the BF16 tensor pipe: their own flops against
        # the measured BF16 peak; the FP64 (LDL^T) flops they stand for beside
        add_kernel("mf_gj_update_oz", kprof["update_ms"], kprof["update_calls"], kprof["update_flops_executed"],
                   "tensor")
        ko = kernels.get("mf_gj_update_oz")
        if ko:
            ko["unit_kind"] = ("BF16 tensor flops of the exact-splitting products (36 slice products of "
                               "128 x 32 x 64 real per 64 x 32 complex sub-tile)")
            ko["fp64_equivalent_flops_per_launch"] = kprof["update_flops"] / kprof["update_calls"]
            ko["fp64_equivalent_tflops"] = ko["fp64_equivalent_flops_per_launch"] / (ko["ms_per_launch"] * 1e-3) / 1e12
            ko["fp64_equivalent_vs_dgemm"] = ko["fp64_equivalent_tflops"] / fp64_tf
    elif tensor:
        add_kernel(f"mf_gj_update_tc<{args.precision}>", kprof["update_ms"], kprof["update_calls"],
                   kprof["update_flops"], "tensor", kprof["update_flops_executed"])
    else:
        add_kernel(f"mf_gj_update{'_sym' if sym else ''}<{tname}>", kprof["update_ms"], kprof["update_calls"],
                   kprof["update_flops"], "flops", kprof["update_flops_executed"])
    add_kernel(f"mf_gj_small<{tname}>", kprof["small_ms"], kprof["small_calls"], kprof["small_flops"], "flops",
               kprof["small_flops_executed"])
    add_kernel(f"mf_down<{tname}>", kprof["down_ms"], kprof["down_calls"], kprof["down_bytes"], "bytes")
    add_kernel(f"mf_up<{tname}>", kprof["up_ms"], kprof["up_calls"], kprof["up_bytes"], "bytes")
    add_kernel(f"mf_strip_sweep<{tname}>", kprof["sweep_ms"], kprof["sweep_calls"], kprof["sweep_bytes"], "bytes")
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    d = kernels[dom]
    roof = {k: d[k] for k in ("bound", "achieved", "peak", "unit", "frac", "peak_source")}
    roof["kernel"] = dom
    roof["units_per_launch"] = d["units_per_launch"]
    roof["unit_kind"] = d["unit_kind"]
    if "executed_flops_per_launch" in d:
        roof["executed_flops_per_launch"] = d["executed_flops_per_launch"]
        roof["executed_tflops"] = d["executed_tflops"]
    roof["measured_over"] = ("one extra step after the timed region with a CUDA-event span around every launch "
                             "(graphs bypassed); profiled step %.1f ms" % kprof["step_ms"])
    roof["traffic"] = ncu_traffic(dom, d.get("executed_flops_per_launch", d["units_per_launch"]))
    roof["traffic_source"] = NCU_TRAFFIC.get(dom, {}).get("profile") if roof["traffic"] is not None else None

    out = {
        "metric": METRIC,
        "value": whole_job_rate(N, ms_max * 1e-3, world) / 1e6,
        "unit": "MDoF/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {S.STDD_PREC_FP64: "c128", S.STDD_PREC_C64: "c64-factors+c128-krylov",
                  S.STDD_PREC_C64_BF16: "c64-factors(bf16 tensor-core updates)+c128-krylov",
                  S.STDD_PREC_C64_FP16: "c64-factors(fp16 tensor-core updates)+c128-krylov"}[prec],
        "data": "synthetic",
        "config": {"workload": workload_desc(w), "precision": args.precision, "order": args.order,
                   "pivoting": pivots_for(prec)[0], "static_pivot": pivots_for(prec)[1],
                   "symmetric_form": int(bool(args.symmetric and not pivots_for(prec)[0] and not tensor and (
                       prec == S.STDD_PREC_FP64 or args.symmetric == 2))),
                   "fp64_products": ("BF16 tensor cores, exact 8 x 7-bit splitting" if (
                       args.fp64_tc and args.symmetric and prec == S.STDD_PREC_FP64) else "FP64 pipe"),
                   "persistent_sweeps": (args.persistent if args.persistent >= 0 else
                                         (0 if prec == S.STDD_PREC_FP64 else 2)),
                   "krylov_space": "band" if band_main else "full", "leaf": args.leaf, "rtol": RTOL,
                   "restart": RESTART, "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "inputs larger than L2 (factors %.1f GB, Krylov basis %.1f GB)"
                         % (E * elem / 1e9, (2 * RESTART + 1) * w.n * 16 / 1e9)},
        "iterations": its,
        "converged": bool(st["final_residual"] <= RTOL),
        "final_residual": st["final_residual"],
        "true_residual_check": r_rel,
        "factor_flops_lu": st["factor_flops_lu"],
        "factor_flops_executed": st["factor_flops"],
        "t_factor_ms": prof["factor_ms"] / args.steps,
        "t_solve_ms": prof["solve_ms"] / args.steps,
        "phases": phases,
        "kernels": kernels,
        "roofline": roof,
        "gpu_launches": int(launches),
        "clocks": ck,
        "peaks": {"hbm_gbs": peaks["hbm_gbs"], "fp64_tflops_dgemm": fp64_tf, "fp32_tflops_sgemm": fp32_tf,
                  "fp64_nominal": FP64_NOMINAL_TFLOPS, "fp32_nominal": FP32_NOMINAL_TFLOPS},
    }
    sv.close()

    def summary(ms_, prof_, st_, hist_, **extra):
        diff = float(torch.linalg.vector_norm(x_d - x_main) / torch.linalg.vector_norm(x_main))
        d_ = {"ms_per_step": ms_, "value": N / (ms_ * 1e-3) / 1e6, "iterations": len(hist_) - 1,
              "final_residual": st_["final_residual"], "converged": bool(st_["final_residual"] <= RTOL),
              "t_factor_ms": prof_["factor_ms"], "t_solve_ms": prof_["solve_ms"], "rel_diff_vs_main": diff,
              "solve_phases_ms": {"minv": prof_["minv_ms"], "minv_calls": prof_["minv_calls"],
                                  "matvec": prof_["matvec_ms"], "gram_schmidt": prof_["ortho_ms"]}}
        d_.update(extra)
        return d_

    if not args.no_compare:
        # the mixed forms on the same problem (FP64 Krylov iteration in all of
        # them): complex64 factors with FP32 updates, and with FP16 tensor-core
        # updates; or plain FP64 when the main line is a mixed form
        others = ([S.STDD_PREC_C64, S.STDD_PREC_C64_FP16] if prec == S.STDD_PREC_FP64 else [S.STDD_PREC_FP64])
        names = {S.STDD_PREC_FP64: "fp64", S.STDD_PREC_C64: "c64", S.STDD_PREC_C64_FP16: "fp16"}
        out["compare_modes"] = {}
        for other in others:
            sv2, ms2, prof2, _, st2, hist2, _, _ = timed(other, 1, 1, 1)
            piv2, sp2 = pivots_for(other)
            out["compare_modes"][names[other]] = summary(
                ms2, prof2, st2, hist2, precision=names[other], pivoting=piv2, static_pivot=sp2,
                raised_pivots=st2["raised_pivots"], order=args.order)
            sv2.close()
        out["compare"] = out["compare_modes"][names[others[0]]]
        # the other strip orders of the same method (same precision as the
        # main line), one step each
        out["orders"] = {}
        for name in orders:
            if name == args.order:
                continue
            sv3, ms3, prof3, _, st3, hist3, _, _ = timed(prec, 1, 1, 1, order=name)
            out["orders"][name] = summary(ms3, prof3, st3, hist3,
                                          krylov_space="band" if band_for(prec, name, None) else "full")
            sv3.close()
        # the same iteration in band space (FP64 additive) or not
        if prec == S.STDD_PREC_FP64 and args.order == "additive":
            sv4, ms4, prof4, _, st4, hist4, _, _ = timed(prec, 1, 1, 1, band=0 if band_main else 1)
            out["band_space" if not band_main else "full_space"] = summary(ms4, prof4, st4, hist4)
            if band_main and prof4["matvec_calls"]:
                # the full-space step's matvec spans hold only the stencil
                # (inner steps) and the residual (restarts): 40 B per node
                out["phases"]["stencil_matvec"] = stencil_phase(
                    prof4["matvec_ms"] / prof4["matvec_calls"], prof4["matvec_calls"], w.n, peaks["hbm_gbs"],
                    fp64_tf, measured_over="the full-space comparison step")
            sv4.close()

    if not args.no_e2e:
        # through the public API with host buffers: permittivity and sources
        # copied in from pinned memory, the solution copied out, every step
        eps_h = torch.from_numpy(w.eps_node).pin_memory()
        b_h = torch.from_numpy(w.b).pin_memory()
        x_h = torch.empty(w.b.shape, dtype=torch.complex128).pin_memory()
        sv = make_solver(prec)
        sv.set_sources(b_h)
        S.stdd_set_permittivity(sv.ctx, eps_h)
        sv.factor()
        sv.solve(x_h, restart=RESTART, rtol=RTOL, maxit=args.maxit, allow_noconv=True)
        barrier()
        ne = max(1, min(args.steps, args.e2e_steps))
        t0 = time.perf_counter()
        for _ in range(ne):
            S.stdd_set_permittivity(sv.ctx, eps_h)
            sv.factor()
            S.stdd_set_sources(sv.ctx, w.nrhs, b_h)
            sv.solve(x_h, restart=RESTART, rtol=RTOL, maxit=args.maxit, allow_noconv=True)
        dt = (time.perf_counter() - t0) / ne
        dt = max_over_ranks(dt, dist, dev)
        out["e2e"] = {"value": whole_job_rate(N, dt, world) / 1e6, "unit": "MDoF/s", "ms_per_step": dt * 1e3,
                      "steps": ne,
                      "h2d_bytes_per_step": int(w.eps_node.nbytes + w.b.nbytes),
                      "d2h_bytes_per_step": int(w.b.nbytes)}
        sv.close()

    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(args.workload)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


# ------------------------------------------------------------- reference
def run_reference(args, rank):
    """The CPU oracle on the host cores (the reference arm): each step factors
    every strip of a shrunk instance of the benchmark's generator and runs the
    oracle's FGMRES to 1e-8 with the additive preconditioner, local solves in
    parallel worker processes; W untimed steps, then the median of K."""
    if rank != 0:
        return
    w, desc = cpu_sample_workload(args.workload, small=True)
    N = w.n * w.nrhs
    po = ParallelOracle(w)
    try:
        for _ in range(args.warmup):
            po.step()
        rows = [po.step() for _ in range(args.steps)]
    finally:
        po.close()
    t = statistics.median(r[0] for r in rows)
    v = N / t / 1e6
    info = host_info()
    cb = {"value": v, "unit": "MDoF/s", "cores": po.procs, "kind": "oracle",
          "sample": (f"{desc} ({w.n} DoF): SuperLU factors of every strip + the oracle's FGMRES({RESTART}) with "
                     f"the additive preconditioner to {RTOL:g} per step, {po.procs} worker processes"),
          "iterations": rows[-1][2], "final_residual": rows[-1][3], **info}
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MDoF/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
           "config": {"workload": f"{desc} ({w.n} DoF), a bounded sample of {args.workload}", "precision": "fp64",
                      "order": "additive", "rtol": RTOL, "restart": RESTART},
           "cpu_baseline": cb,
           "e2e": {"value": v, "unit": "MDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
