"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2):
the step time every rank reports is the slowest rank's, the whole-job rate
sums the replicas' units over that time, and the reference arm prints only
on rank 0."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(times[rank], dist)
        rate = bench.whole_job_rate(1000, got, world)
        buf = io.StringIO()
        with redirect_stdout(buf):
            bench.run_reference(None, rank) if rank != 0 else None
        out.put((rank, got, rate, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [0.25, 0.75]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate, printed in res:
        assert got == 0.75                  # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 1000 / 0.75)
        assert printed == ""                # the reference arm prints on rank 0 only


def test_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.whole_job_rate(4194304, 0.8, 1) == pytest.approx(4194304 / 0.8)


def test_stencil_phase_roofline():
    """The stencil's figures from one measured call time: 40 B and 40 flops
    per node; FP64-bound where the FP64 rate is below 1 flop per HBM byte."""
    sys.path.insert(0, ROOT)
    import bench
    d = bench.stencil_phase(0.2, 36, 4194304, 6794.1, 1.0985)
    assert d["bytes_per_call"] == d["flops_per_call"] == 40 * 4194304
    assert d["gbs"] == pytest.approx(838.86, rel=1e-4)
    assert d["tflops"] == pytest.approx(0.83886, rel=1e-4)
    assert d["fp64_frac"] == pytest.approx(0.83886 / 1.0985, rel=1e-4)
    assert d["bound"] == "alu"
    assert bench.stencil_phase(0.2, 1, 100, 1000.0, 10.0)["bound"] == "hbm"
    assert bench.stencil_phase(0.2, 1, 100, 1000.0, 1.0, measured_over="x")["measured_over"] == "x"


def test_traffic_records_follow_their_kernel_source(tmp_path, monkeypatch):
    """roofline.traffic scales a recorded DRAM capture only while the
    kernel's source text between the record's markers still hashes to the
    recorded SHA-256; an edited kernel reports null instead of a stale
    figure.  Every record's markers exist in its source file."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    for name, rec in bench.NCU_TRAFFIC.items():
        src = open(os.path.join(ROOT, rec["source"])).read()
        assert src.index(rec["begin"]) < src.index(rec["end"]), name
        assert os.path.exists(os.path.join(ROOT, rec["profile"])), name
    f = tmp_path / "k.cu"
    f.write_text("head\n// BEGIN\nkernel body v1\n// END\ntail\n")
    digest = hashlib.sha256("// BEGIN\nkernel body v1\n".encode()).hexdigest()
    rec = {"dram_per_unit": 2.5, "source": str(f), "begin": "// BEGIN", "end": "// END", "sha256": digest,
           "profile": "x"}
    monkeypatch.setitem(bench.NCU_TRAFFIC, "k<double>", rec)
    assert bench.ncu_traffic("k<double>", 4.0) == 10.0
    assert bench.ncu_traffic("k<double>", 0) is None
    assert bench.ncu_traffic("unknown", 4.0) is None
    f.write_text("head\n// BEGIN\nkernel body v2\n// END\ntail\n")
    assert bench.ncu_traffic("k<double>", 4.0) is None
