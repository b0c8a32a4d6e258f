"""The BDDC split over processes (oracle/distributed.py), on two gloo CPU
ranks: each rank works on its own block of subdomains and only the
interface sums, the operator product and the coarse all-gather combine
them; the result equals the one-process apply (Section 4, one subdomain per
process on an unassembled matrix; Section 7, redundant coarse solve)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, scaling, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle.assembly import FEProblem
        from oracle.bddc import BDDC
        from oracle.distributed import DistributedBDDC, owned
        from oracle.krylov import gmres
        from workloads import slab_problem

        prob = slab_problem(6, 4, 3, order=1, parts=(3, 2, 2), jitter=0.15, pressure=1.0e3, gamma=3.0e4)
        fe = FEProblem(prob)
        X = fe.coords[fe.free_nodes]
        d = (0.02 * X[:, 2:3] * np.sin(X + 1.0)).reshape(-1)
        K, (Ke, Kf) = fe.tangent(d, 0.7)
        pc = BDDC(fe, Ke, Kf, "VE", scaling=scaling)
        dpc = DistributedBDDC(pc, dist)
        rng = np.random.default_rng(5)
        r = rng.standard_normal(fe.n_free)
        z1 = pc.apply(r)
        z2 = dpc.apply(r)
        y2 = dpc.matvec(r)
        x1, its1, _ = gmres(lambda v: K @ v, r, pc.apply, tol=1e-10)
        x2, its2, _ = gmres(dpc.matvec, r, dpc.apply, tol=1e-10)
        lo, hi = owned(prob["n_parts"], rank, world)
        out[rank] = dict(apply=float(np.linalg.norm(z2 - z1) / np.linalg.norm(z1)),
                         apply_max=float(np.abs(z2 - z1).max() / np.abs(z1).max()),
                         matvec=float(np.linalg.norm(y2 - K @ r) / np.linalg.norm(K @ r)),
                         its=(its1, its2), x=float(np.linalg.norm(x2 - x1) / np.linalg.norm(x1)),
                         owned=(lo, hi), exchanged=dpc.exchanged, z_sum=float(z2.sum()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("scaling", ["counting", "deluxe"])
def test_two_rank_bddc_equals_one_rank(scaling):
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, scaling, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0]["owned"] == (0, 6) and res[1]["owned"] == (6, 12)
    for q in range(world):
        assert res[q]["apply"] <= 1e-12 and res[q]["apply_max"] <= 1e-12
        assert res[q]["matvec"] <= 1e-12
        its1, its2 = res[q]["its"]
        assert its1 == its2 and res[q]["x"] <= 1e-9
        assert res[q]["exchanged"] > 0
    # every rank holds the same result, to the bit (sums in rank order)
    assert res[0]["z_sum"] == res[1]["z_sum"]
