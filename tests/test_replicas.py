"""Multi-GPU form (independent replicas, one process per GPU) on CPU: sharding of the pairs,
the host-side maximum over ranks and the whole-job rate, with two gloo ranks."""
import argparse
import multiprocessing as mp
import os
import socket

import numpy as np
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


class _FakePool:
    """Stand-in for bench.OraclePool: records the specs it is given and reports 0.5 s of oracle
    time per unit, one pair each, without running the oracle."""
    seen = []

    def __init__(self, procs):
        self.procs = procs

    def map(self, specs):
        _FakePool.seen.append(list(specs))
        return [(0.5, 1.0, None) for _ in specs]

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


def test_reference_arm_line_on_rank_0(capsys, monkeypatch):
    """The reference arm's JSON line: the same metric, unit and workload config as the GPU arm,
    one full-size pair per step, warm-up steps run first on other pairs, the rate of the timed
    steps over their wall time (ms_per_step x steps is that wall time), no host-device copies,
    and the oracle run described.  The pool of oracle processes is replaced by a stand-in."""
    import json
    import bench
    _FakePool.seen = []
    monkeypatch.setattr(bench, "OraclePool", _FakePool)
    args = argparse.Namespace(steps=2, warmup=3, preset="dense", gpus=1, workload="flow", norm="l2", fb=False,
                              term_eps=0.0, batch=32)
    bench.run_reference(args, 0, 1)
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["metric"] == bench.WORKLOADS["flow"]["metric"]
    assert line["unit"] == bench.UNIT and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 3
    assert line["dtype"] == "f64" and line["vs_baseline"] is None
    assert line["config"] == bench.workload_config(args, 32, 1)
    # warm-up units first (pairs 2, 3, 4), then the timed ones (pairs 0, 1), one pair per step
    assert [sp[2] for sp in _FakePool.seen[0]] == [[2], [3], [4]]
    assert [sp[2] for sp in _FakePool.seen[1]] == [[0], [1]]
    assert all(sp[0] == "flow" and sp[1] == "dense" and sp[3] is None for sp in _FakePool.seen[1])
    wall = line["ms_per_step"] * line["steps"] / 1000.0
    assert abs(line["value"] - 2 / wall) <= 1e-9 * line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == line["value"]
    assert "1024x436" in cb["sample"] and "0.50 s median" in cb["sample"]


def test_cpu_units_match_the_workloads():
    """The CPU legs' units: full pairs of the workload's generator (the GPU arm's pair k), or a
    stated sample at 1/16 (RGB 4K) and 1/4 (stereo) of the area."""
    import bench
    from paper_1603_03590_gb300 import synth
    I0, I1, gt, q, per, _ = bench.cpu_unit("flow", "dense", 1)
    r0, r1, _ = synth.workload_pair("layered1024x436", 1)
    assert np.array_equal(I0, r0) and np.array_equal(I1, r1) and per == 1.0
    assert q["patch_size"] == 12 and q["grad_iters"] == 128 and q["coarsest_scale"] == 4 and q["refine"] == 1
    q = bench.cpu_unit("flow", "fast", 0)[3]
    assert (q["patch_size"], q["grad_iters"], q["finest_scale"], q["refine"]) == (8, 16, 2, 0)
    I0, _, _, q, per, _ = bench.cpu_unit("rgb4k", "dense", 0)
    assert I0.shape == (3, 540, 960) and per == 1.0 / 16 and q["channels"] == 3 and q["coarsest_scale"] == 4
    I0, _, _, q, per, _ = bench.cpu_unit("stereo", "stereo_dense", 0)
    assert I0.shape == (480, 720) and per == 0.25 and q["dof"] == 1
    I0, _, _, q, per, _ = bench.cpu_unit("translate128x96", "cfg0", 0)
    assert I0.shape == (96, 128) and q["stride_override"] == 4


def test_bench_defaults_keep_the_timing_rules(monkeypatch):
    """No flags: one GPU, at least three warm-up steps, and a warm-up below three is raised to three."""
    import bench
    seen = {}
    monkeypatch.setattr(bench, "run_reference", lambda args, rank, world: seen.update(vars(args)))
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference"])
    bench.main()
    assert seen["gpus"] == 1 and seen["warmup"] >= 3 and seen["steps"] >= 1 and seen["batch"] == 32
    assert seen["unique"] == 32  # 32 distinct scenes per batch
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--warmup", "1"])
    bench.main()
    assert seen["warmup"] == 3



def test_bench_parity_block_uses_the_tests_determination():
    """The bench's parity block classifies pixels as the end-to-end parity tests do."""
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import test_gpu_parity
    assert (bench.PERTURB, bench.STABLE_TOL) == (test_gpu_parity.PERTURB, test_gpu_parity.STABLE_TOL)
    ref = np.zeros((4, 5, 2))
    got = ref + 1e-3
    spread = np.zeros((4, 5))
    spread[0, 0] = 1.0  # one pixel not determined
    st = bench.parity_stats(got, ref, spread, ref)
    assert st["stable_frac"] == 19 / 20 and abs(st["stable_mean_abs_du"] - 1e-3) < 1e-15
