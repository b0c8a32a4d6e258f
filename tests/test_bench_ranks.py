"""The multi-process paths of bench.py on CPU (gloo, world size 2): the
timing is the maximum over ranks, and the oracle arm runs on rank 0 only.
GPU runs use one replica per GPU with the same helpers."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench._max_over_ranks(10.0 + rank, world)
    bench._barrier(world)
    dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert dict(out) == {0: 11.0, 1: 11.0}


def test_reference_arm_is_silent_off_rank_zero(capsys):
    import bench

    class Args:
        steps, warmup, gpus, oracle_budget_s, workload = 1, 0, 2, 1.0, bench.WORKLOAD
    bench.run_reference(Args(), 2, 1)
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_the_contract_line(capsys):
    # one oracle sample of the default workload: 16 clamped subdomains of
    # the P2 ventricle through assembly, BDDC setup and three GMRES
    # iterations (about 15 s), extrapolated to the whole workload
    import json

    import bench

    class Args:
        steps, warmup, gpus, oracle_budget_s, workload = 1, 3, 1, 300.0, bench.WORKLOAD
    bench.run_reference(Args(), 1, 0)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is False and d["steps"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert "16 clamped level-1 subdomains" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload_name"] == bench.WORKLOAD
