"""The strip method's exchange step on CPU ranks (gloo, world sizes 2 and 3):
each rank owns a contiguous group of strips and keeps vectors only on its
owned columns; the stencil swaps one boundary column per cut, the synthesis
swaps the ext = overlap + interface PML columns that local fields spill past
each cut, and FGMRES sums its inner products over the ranks.  Against the
single-process oracle: the same matrix-vector products and preconditioner
(to rounding), the same FGMRES iteration count and solution, and the
exchange volume the design predicts."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASE = dict(nx=203, ny=77, ppw=16, seed=21, npml=8, nsub=6, overlap=5, interface_pml=9, nsrc=1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import workloads as W
    from oracle.distributed import RankStrips
    from oracle.fdfd import Problem
    from oracle.krylov import gmres
    from oracle.stddm import DDM
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = W.random_medium(**CASE)
        P = Problem.from_workload(w)
        R = RankStrips(P, w.nsub, w.overlap, w.interface_pml, rank, world, dist)
        D = DDM(P, w.nsub, w.overlap, w.interface_pml)
        v = W.random_vector(P.n, seed=9)[0]
        mv = R.matvec(R.owned(v))
        mv_ref = R.owned(P.A @ v)
        sent0 = R.sent_values
        pc = R.precond(R.owned(v))
        sent_pc = R.sent_values - sent0
        pc_ref = R.owned(D.apply_Minv(v))
        b = w.b[0].ravel()
        x, hist, its = R.solve(R.owned(b), restart=30, rtol=1e-10, maxit=200)
        xr, hr, itr = gmres(P.matvec, D.apply_Minv, b, restart=30, rtol=1e-10, maxit=200)
        out.put(dict(rank=rank, C=(R.C0, R.C1),
                     mv=float(np.linalg.norm(mv - mv_ref) / np.linalg.norm(mv_ref)),
                     pc=float(np.linalg.norm(pc - pc_ref) / np.linalg.norm(pc_ref)),
                     sent_pc=sent_pc, its=its, its_ref=itr,
                     x=float(np.linalg.norm(x - R.owned(xr)) / np.linalg.norm(R.owned(xr))),
                     res=float(hist[-1])))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_strips_over_gloo_ranks_match_the_single_process_oracle(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda d: d["rank"])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ny, ext = CASE["ny"], CASE["overlap"] + CASE["interface_pml"]
    # the owned column ranges tile the grid
    assert res[0]["C"][0] == 0 and res[-1]["C"][1] == CASE["nx"]
    for a, b in zip(res, res[1:]):
        assert a["C"][1] == b["C"][0]
    for r in res:
        assert r["mv"] <= 1e-14
        assert r["pc"] <= 1e-13
        assert r["its"] == r["its_ref"] and r["res"] <= 1e-10
        assert r["x"] <= 1e-10
        # one preconditioner application: ext x ny values across each of the
        # rank's cuts (one cut for the end ranks, two for inner ones)
        cuts = (r["rank"] > 0) + (r["rank"] < world - 1)
        assert r["sent_pc"] == cuts * ext * ny


def test_rank_narrower_than_the_spill_is_rejected():
    """Every rank must own at least overlap + interface PML columns, else a
    neighbour's local field would spill past it to the next rank.  The
    partition already refuses strips narrower than that (each strip is some
    strip's neighbour), so every rank of at least one strip owns enough
    columns; the rank split checks it again, and a split that breaks it is
    refused before any exchange (no process group is needed)."""
    sys.path.insert(0, ROOT)
    import workloads as W
    from oracle.distributed import RankStrips
    from oracle.fdfd import Problem
    w = W.random_medium(60, 24, ppw=16, seed=3, npml=6, nsub=6, overlap=4, interface_pml=6)
    P = Problem.from_workload(w)
    # 6 strips of 10 columns over 6 ranks: 10 owned columns, ext = 10 -> allowed
    R = RankStrips(P, 6, 4, 6, 0, 6, comm=None)
    assert R.C1 - R.C0 == 10
    # ext = 12 > 10 owned columns per rank -> refused
    with pytest.raises(ValueError, match="fewer than overlap|wider than a neighbouring strip"):
        RankStrips(P, 6, 6, 6, 0, 6, comm=None)
