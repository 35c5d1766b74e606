"""Host logic of the multi-GPU path: one independent chain per rank.

The path does not shard, so N > 1 means N replicas; the only collectives
are the timing barrier and the maximum of the elapsed time over ranks.
These tests run that logic on CPU with the gloo backend, world size 2.
"""

import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = [1.5, 2.5][rank]              # rank 1 is the slowest
        m = bench.reduce_max(elapsed, world, "cpu")
        rate = bench.whole_job_rate(10, world, m)
        dist.barrier()
        q.put((rank, m, rate, bench.rank_seeds(rank)))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_sum_the_work():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, m, rate, seeds in out:
        assert m == 2.5
        assert rate == pytest.approx(2 * 10 / 2.5)
    # every rank runs its own chain
    assert out[0][3]["hot_start"] != out[1][3]["hot_start"]
    assert out[0][3]["device_rng"] != out[1][3]["device_rng"]


def test_single_rank_needs_no_process_group():
    assert bench.reduce_max(3.0, 1, "cpu") == 3.0
    assert bench.whole_job_rate(20, 1, 4.0) == 5.0


def test_reference_arm_only_runs_on_rank_zero(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, lattice, integrator, dt, gpus, link_reals, precision = 1, 0, 32, "fg", 0.25, 2, 18, "fp32"
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    """Rank 0 of the reference arm prints one JSON line with the keys the
    driver reads (the oracle's trajectory timing is stubbed: the line's
    structure is what is tested here)."""
    import json
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    import time

    class FakePool:
        """Stands in for the spawned process pool: each oracle trajectory
        'takes' 10 ms of wall time."""
        def __enter__(self):
            return self

        def __exit__(self, *a):
            return False

        def map(self, fn, jobs):
            jobs = list(jobs)
            time.sleep(0.01)
            return [0.01] * len(jobs)

    monkeypatch.setattr(bench, "oracle_pool", lambda n: FakePool())

    class A:
        steps, warmup, lattice, integrator, dt, gpus, link_reals, precision = 2, 1, 32, "fg", 0.25, 1, 18, "fp32"
    assert bench.run_reference(A()) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True
    # only timings that ran: ms_per_step x steps fits the run; the volume scaling is labelled apart
    assert d["ms_per_step"] * d["steps"] / 1000.0 <= d["run_s"]
    sf = d["scaled_from"]
    assert d["value"] == pytest.approx(sf["trajectories_per_s_measured"] * sf["factor"])
    assert sf["factor"] == pytest.approx((8 / 32) ** 4)
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"]
