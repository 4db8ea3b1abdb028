"""Multi-GPU form (independent replicas, one process per GPU) on CPU: sharding of the pairs,
the host-side maximum over ranks and the whole-job rate, with two gloo ranks."""
import argparse
import multiprocessing as mp
import os
import socket

import pytest

from paper_1603_03590_gb300 import replicas


def test_shard_is_disjoint_complete_and_balanced():
    for n in range(0, 40):
        for world in range(1, 9):
            spans = [replicas.shard(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    for bad in [(5, 2, 2), (5, -1, 2), (5, 0, 0), (-1, 0, 1)]:
        with pytest.raises(ValueError):
            replicas.shard(*bad)


def test_single_process_is_identity():
    assert replicas.max_over_ranks([3.0, 1.5]) == [3.0, 1.5]
    replicas.barrier()
    assert replicas.aggregate_rate(32 * 20, 1, 2.0) == 320.0
    with pytest.raises(ValueError):
        replicas.aggregate_rate(1, 1, 0.0)


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, local, w = replicas.env_rank_world()
        lo, hi = replicas.shard(11, r, w)
        # per-rank "times": the slowest rank decides each entry
        m = replicas.max_over_ranks([1.0 + r, 5.0 - r, float(hi - lo)])
        replicas.barrier()
        q.put((r, local, w, lo, hi, m, replicas.aggregate_rate(hi - lo, w, m[0])))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    (r0, l0, w0, lo0, hi0, m0, rate0), (r1, l1, w1, lo1, hi1, m1, rate1) = res
    assert (r0, l0, w0, r1, l1, w1) == (0, 0, 2, 1, 1, 2)
    assert (lo0, hi0, lo1, hi1) == (0, 6, 6, 11)
    assert m0 == m1 == [2.0, 5.0, 6.0]
    assert rate0 == 2 * 6 / 2.0 and rate1 == 2 * 5 / 2.0


def test_reference_arm_is_silent_on_other_ranks(capsys):
    import bench
    args = argparse.Namespace(steps=1, warmup=3, preset="dense", gpus=2)
    assert bench.run_reference(args, 1, 2) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_0(capsys, monkeypatch):
    """The reference arm's JSON line: the same metric, unit and config as the GPU arm, the rate of
    the timed steps only (warm-up steps discarded), no host-device copies, and the oracle sample
    described.  The oracle itself is replaced by a stand-in that reports a given rate per call."""
    import json
    import bench
    rates = iter([9.0, 9.0, 9.0, 0.5, 0.25])  # three warm-up calls, then two timed steps

    def fake_cpu_baseline(preset, workload="flow", norm="l2", fb=False, term_eps=0.0):
        return {"value": next(rates), "unit": bench.UNIT, "cores": 1, "kind": "oracle", "sample": "stand-in"}

    monkeypatch.setattr(bench, "cpu_baseline", fake_cpu_baseline)
    args = argparse.Namespace(steps=2, warmup=3, preset="dense", gpus=1, workload="flow", norm="l2", fb=False,
                              term_eps=0.0, batch=32)
    bench.run_reference(args, 0, 1)
    line = json.loads(capsys.readouterr().out.strip())
    metric, W, H = bench.WORKLOADS["flow"][:3]
    assert line["impl"] == "reference" and line["metric"] == metric and line["unit"] == bench.UNIT
    # each step is 1/4 of a pair's area at the sampled rate: 0.5 and 0.25 pairs/s take 0.5 s and 1 s
    assert abs(line["value"] - 2 * 0.25 / 1.5) < 1e-12
    assert line["steps"] == 2 and line["warmup"] == 3 and line["higher_is_better"] is True
    assert line["dtype"] == "f64" and line["vs_baseline"] is None
    assert line["config"] == bench.workload_config(args, 32, 1)
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    assert "%dx%d" % (W // 2, H // 2) in cb["sample"]


def test_bench_defaults_keep_the_timing_rules(monkeypatch):
    """No flags: one GPU, at least three warm-up steps, and a warm-up below three is raised to three."""
    import bench
    seen = {}
    monkeypatch.setattr(bench, "run_reference", lambda args, rank, world: seen.update(vars(args)))
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference"])
    bench.main()
    assert seen["gpus"] == 1 and seen["warmup"] >= 3 and seen["steps"] >= 1 and seen["batch"] == 32
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--warmup", "1"])
    bench.main()
    assert seen["warmup"] == 3

