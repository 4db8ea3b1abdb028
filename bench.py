#!/usr/bin/env python
"""Benchmark of the DIS hot path on synthetic scenes shaped like the paper's workloads.

Default (--workload flow): frame-pairs/s at 1024x436.  One step = the whole method (pyramid,
per-level patch search, densification, variational refinement, up-scaling) over one batch of
32 distinct layered 1024x436 pairs, run by the batched entry point (one CUDA-graph replay of
persistent kernels over all pairs); --preset dense (default: patch 12, 75 % overlap, 128
iterations, refinement) or fast (patch 8, 30 % overlap, 16 iterations, finest two levels
skipped, no refinement).  The same pairs through sequential single-pair calls (the plain form)
are timed beside it.  Inputs are resident in HBM for `value`; `e2e` adds the host->device copy
of the frames from pinned memory and the device->host copy of the flows to every step.  L2 is
flushed (a 256 MB write) between timed steps, outside the timed events.

Other workloads, each with its own metric:
  --workload mixed    64 pairs of mixed resolution (320x240 ... 1920x1080, displacements 4 % of
                      the width), medium preset, autotuned, one graph replay per step;
  --workload rgb4k    4 RGB pairs at 3840x2160 (2 degree rotation, displacements up to 200 px),
                      dense preset, 7 levels;
  --workload stereo   rectified 1440x960 pairs (horizontal layered scenes, disparities up to
                      96 px), batches of 8, dense preset with one degree of freedom;
  --workload diff     the differentiable form: 8 pairs of 512x256, 4 levels, patch 8, 50 %
                      overlap, 10 unrolled sweeps per level; a step is the forward map and the
                      backward pass of the mean Charbonnier photometric loss to both frames
                      and the initial flow.
--norm l1 / huber, --fb and --term-eps E select the robust error norms, forward-backward
consistency and early termination (supplementary Secs. B, C).

CPU legs (the FP64 oracle, the correctness reference of this repository; the paper's own CPU
code is not available): `cpu_baseline` times it on one host core on one full-size pair of the
workload (a bounded sample where a full pair would take minutes, stated in `sample`) and, for
the 1024x436 workload, compares the GPU flow of that pair with it (the `parity` block).
--impl reference times the same oracle on the host cores, one pair of the workload per step,
the pairs spread over a pool of single-threaded processes.  --cpu-report times the oracle's
single-core cases (128x96 translation; 1024x436 fast and dense, median of three) and a
pair-parallel all-cores pass over the 64 mixed pairs.

Multi-GPU (torchrun): frame pairs are independent, so each rank runs its own batch
(replicas, weak scaling, no collective on the data path); value = all ranks' pairs / max time.
"""
import argparse
import json
import multiprocessing as mp
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

UNIT = "frame-pairs/s"

# Parameter values of the named presets (the same values as the library's dis_default_params,
# checked by the CPU tests), so that the CPU legs build the oracle's parameters without loading
# the CUDA library.
PRESETS = {
    "fast": dict(patch_size=8, overlap=0.30, grad_iters=16, finest_scale=2, refine=0),
    "medium": dict(patch_size=8, overlap=0.50, grad_iters=32, finest_scale=0, refine=1),
    "dense": dict(patch_size=12, overlap=0.75, grad_iters=128, finest_scale=0, refine=1),
    "stereo_dense": dict(patch_size=12, overlap=0.75, grad_iters=64, finest_scale=0, refine=1, dof=1),
}
# the differentiable workload's parameters (4 levels, patch 8, 50 % overlap, 10 unrolled sweeps)
DIFF_PARAMS = dict(patch_size=8, overlap=0.5, grad_iters=16, coarsest_scale=3, finest_scale=0, refine=1,
                   var_outer=1, var_inner=10)
NORM_CODES = {"l2": 0, "l1": 1, "huber": 2}
# library kernels one pair of the differentiable workload launches per step (FP32 search with its
# graph, FP64 replay, loss, FP64 backward), from the ncu launch list of that step
DIFF_KERNELS_PER_PAIR = 667

# name -> metric, synthetic workload, default preset, default batch, theta_ss (-1: automatic),
# channels, description
WORKLOADS = {
    "flow": dict(metric="DIS flow frame-pairs/s at 1024x436 (batched)", synth="layered1024x436", preset="dense",
                 batch=32, coarsest=4, channels=1, text="layered 1024x436 (20 textured ellipses, piecewise "
                                                         "affine motion up to 40 px)"),
    "mixed": dict(metric="DIS flow frame-pairs/s over 64 mixed-resolution pairs (batched)", synth="mixed",
                  preset="medium", batch=64, coarsest=-1, channels=1,
                  text="64 layered pairs of mixed resolution (320x240, 640x480, 1024x436, 1280x720, 1920x1080; "
                       "displacements 4 % of the width)"),
    "rgb4k": dict(metric="DIS flow frame-pairs/s at 3840x2160 RGB (batched)", synth="rgb3840x2160", preset="dense",
                  batch=4, coarsest=6, channels=3,
                  text="layered RGB 3840x2160 (2 degree rotation, displacements up to 200 px)"),
    "stereo": dict(metric="DIS stereo frame-pairs/s at 1440x960 (batched)", synth="stereo1440x960",
                   preset="stereo_dense", batch=8, coarsest=5, channels=1,
                   text="rectified stereo 1440x960 (horizontal layered scenes, disparities up to 96 px)"),
    "diff": dict(metric="differentiable DIS frame-pairs/s at 512x256 (forward + backward)", synth="layered512x256",
                 preset="diff", batch=8, coarsest=3, channels=1,
                 text="layered 512x256, 4 levels, patch 8, 50 % overlap, 10 unrolled sweeps per level, gradients "
                      "of the mean Charbonnier photometric loss to both frames and the initial flow"),
}

# DRAM bytes per pair of the dominant kernel's launch (ncu dram__bytes_read.sum +
# dram__bytes_write.sum of a small-case capture, divided by the pairs of that launch; every input
# of the launch is read once, so it grows with the pairs), by (workload, preset, search variant),
# with the summary that holds the capture.
TRAFFIC = {
    ("flow", "dense", 16): (17.83e6 / 4, "profiles/search_kernel_dense1024x436_ncu.md (4-pair launch)"),
}


# ------------------------------------------------------------------------------ inputs
def _gen(args):
    name, k = args
    from paper_1603_03590_gb300 import synth
    return synth.workload_pair(name, k)


def gen_pairs(name, n):
    """Pairs 0..n-1 of a seeded workload, generated in spawned processes (pure numpy / scipy)."""
    if n == 1:
        return [_gen((name, 0))]
    procs = max(1, min(n, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_gen, [(name, k) for k in range(n)], chunksize=1)


def oracle_params(preset, workload, norm="l2", fb=False, term_eps=0.0):
    """Keyword parameters of the oracle for a workload and preset (plain values, no library)."""
    if workload == "diff":
        q = dict(DIFF_PARAMS)
    else:
        q = dict(PRESETS[preset])
        q["coarsest_scale"] = WORKLOADS[workload]["coarsest"]
        q["channels"] = WORKLOADS[workload]["channels"]
    q.update(norm=NORM_CODES[norm], fb=1 if fb else 0, term_eps=float(term_eps))
    return q


def cpu_unit(workload, preset, k, norm="l2", fb=False, term_eps=0.0):
    """Unit k of the CPU legs: (I0, I1, gt, oracle keyword parameters, pairs of the workload one
    run stands for, description).  A unit is one full-size pair of the workload, except at
    3840x2160 RGB and 1440x960 stereo, where a full pair would take minutes on one core: there it
    is one pair of the same generator at a quarter (stereo) or a sixteenth (RGB) of the area with
    as many levels fewer (the method's cost is linear in area, supplementary Sec. C)."""
    from paper_1603_03590_gb300 import synth
    if workload == "translate128x96":  # 3 levels, patch 8, stride 4, 16 iterations, 5 sweeps of one pass
        I0, I1, gt = synth.translation_pair(k)
        q = dict(patch_size=8, stride_override=4, grad_iters=16, coarsest_scale=2, finest_scale=0, var_outer=1,
                 var_inner=5)
        return I0, I1, gt, q, 1.0, "128x96 translation pairs"
    q = oracle_params(preset, workload, norm, fb, term_eps)
    if workload == "rgb4k":
        I0, I1, gt = synth.layered_pair(4000 + k, width=960, height=540, max_disp=25.0, channels=3, rotation_deg=2.0)
        q["coarsest_scale"] = 4
        return I0, I1, gt, q, 1.0 / 16, "960x540 RGB pairs (1/16 of the 3840x2160 area, two levels fewer)"
    if workload == "stereo":
        I0, I1, gt = synth.layered_pair(6000 + k, width=720, height=480, max_disp=48.0, horizontal=True)
        q["coarsest_scale"] = 4
        return I0, I1, gt, q, 0.25, "720x480 stereo pairs (1/4 of the 1440x960 area, one level fewer)"
    name = WORKLOADS[workload]["synth"]
    I0, I1, gt = synth.workload_pair(name, k % 64 if workload == "mixed" else k)
    what = {"flow": "full 1024x436 pairs", "mixed": "full pairs of the 64-pair mixed set",
            "diff": "full 512x256 pairs, forward map only (the oracle has no adjoint)"}[workload]
    return I0, I1, gt, q, 1.0, what


def _oracle_job(spec):
    """Worker of the CPU legs (runs in a spawned process): generates the units `ks` of the
    workload and times the FP64 oracle on each; with `perturb` (a seed) I1 is first perturbed by
    PERTURB on the 0..255 scale.  Returns (seconds of oracle time, pairs, flow of the first unit or
    None)."""
    import oracle
    workload, preset, ks, perturb, want_flow, mode = spec
    total, pairs, first = 0.0, 0.0, None
    for k in ks:
        I0, I1, _, q, per, _ = cpu_unit(workload, preset, k, *mode)
        if perturb is not None:
            I1 = I1.astype(np.float64) + np.random.default_rng(perturb).standard_normal(I1.shape) * (PERTURB / 255.0)
        prm = oracle.params(**q)
        t = time.perf_counter()
        f = oracle.dis_flow(I0, I1, prm)
        total += time.perf_counter() - t
        pairs += per
        if want_flow and first is None:
            first = f
    return total, pairs, first


class OraclePool:
    """A pool of spawned single-threaded processes running _oracle_job (spawned, so that no
    worker inherits a CUDA context)."""

    def __init__(self, procs):
        self.procs = procs
        self.pool = mp.get_context("spawn").Pool(procs)

    def map(self, specs):
        return self.pool.map(_oracle_job, specs, chunksize=1)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.pool.terminate()
        self.pool.join()


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


# The end-to-end determination of the parity tests: I1 perturbed by PERTURB grey levels (0..255
# scale, the size whose effect on the search matches the FP32 path's rounding error); pixels whose
# FP64 flow moves by more than STABLE_TOL px are not determined at FP32 resolution.
PERTURB, STABLE_TOL = 1e-3, 0.03


def parity_stats(got, ref, spread, gt):
    """The end-to-end comparison of the parity tests: pixels whose FP64 flow moves by more than
    STABLE_TOL under two PERTURB perturbations of I1 are counted apart; mean and 99.9th
    percentile of |du| on the others and on all pixels."""
    stable = spread <= STABLE_TOL
    d_all = np.abs(got - ref)
    d = d_all[stable]
    return {"pixels": int(stable.size), "stable_frac": float(stable.mean()),
            "stable_mean_abs_du": float(d.mean()), "stable_p999_abs_du": float(np.quantile(d, 0.999)),
            "all_mean_abs_du": float(d_all.mean()), "all_p999_abs_du": float(np.quantile(d_all, 0.999)),
            "oracle_self_spread_p999": float(np.quantile(spread, 0.999)),
            "bar": {"mean": 0.01, "p999": 0.05},
            "determination": "FP64 flow moves by <= %g px under two perturbations of I1 by %g grey levels"
                             % (STABLE_TOL, PERTURB),
            "epe_gpu": float(np.linalg.norm(got - gt, axis=-1).mean()),
            "epe_oracle": float(np.linalg.norm(ref - gt, axis=-1).mean())}


def cpu_baseline(args, gpu_flow0=None):
    """The FP64 oracle on one host core on the workload's pair 0 (a full pair; a series of pairs
    when one takes under a second; a bounded sample at 3840x2160 and 1440x960, see cpu_unit).
    With gpu_flow0 (the GPU's flow of pair 0) the oracle is also run twice more, on I1 perturbed
    by PERTURB, in parallel processes, and the returned `parity` block compares the two flows as the
    parity tests do.  Returns (cpu_baseline dict, parity dict or None)."""
    import oracle
    oracle.build()
    mode = (args.norm, args.fb, args.term_eps)
    wl, preset = args.workload, args.preset
    jobs = [(wl, preset, [0], None, gpu_flow0 is not None, mode)]
    if gpu_flow0 is not None:
        jobs += [(wl, preset, [0], seed, True, mode) for seed in (1, 2)]
    with OraclePool(len(jobs)) as pool:
        res = pool.map(jobs)
        dt, pairs, ref = res[0]
        if dt < 1.0:  # fast presets: time a series of pairs for a steadier figure
            dt, pairs, _ = pool.map([(wl, preset, list(range(min(args.batch, 32))), None, False, mode)])[0]
    _, _, _, _, _, what = cpu_unit(wl, preset, 0, *mode)
    cb = {"value": pairs / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
          "sample": "%s: %g pair(s) of the workload in %.2f s on one core (%s, %d cores on the host)"
                    % (what, pairs, dt, cpu_model(), _cores())}
    parity = None
    if gpu_flow0 is not None:
        spread = np.maximum(np.abs(res[1][2] - ref).max(-1), np.abs(res[2][2] - ref).max(-1))
        gt = cpu_unit(wl, preset, 0, *mode)[2]
        parity = {"pair": 0, **parity_stats(gpu_flow0, ref, spread, gt)}
    return cb, parity


def run_reference(args, rank, world):
    """The oracle arm: rank 0 alone runs the FP64 oracle on one unit of the workload per step
    (see cpu_unit), the steps spread over a pool of single-threaded processes (one per host
    core, at most one per step); warm-up steps run first, untimed.  value = pairs of the timed
    steps / their wall time."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    wl, preset = args.workload, args.preset
    mode = (args.norm, args.fb, args.term_eps)
    procs = max(1, min(args.steps, _cores()))
    with OraclePool(procs) as pool:
        pool.map([(wl, preset, [args.steps + k], None, False, mode) for k in range(args.warmup)])
        t0 = time.perf_counter()
        res = pool.map([(wl, preset, [k], None, False, mode) for k in range(args.steps)])
        wall = time.perf_counter() - t0
    pairs = sum(r[1] for r in res)
    per_run = [r[0] for r in res]
    value = pairs / wall
    what = cpu_unit(wl, preset, 0, *mode)[5]
    line = {"impl": "reference", "metric": WORKLOADS[wl]["metric"], "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, args.batch, world),
            "step": "one unit of the workload (%s) per step, %d oracle processes in parallel" % (what, procs),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": "%d steps of %s on %d of %d cores (%s); one unit took %.2f s median on "
                                       "one core" % (args.steps, what, procs, _cores(), cpu_model(),
                                                     statistics.median(per_run))},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def cpu_report(args):
    """Single-core oracle times (median of three runs, run side by side on separate cores) of the
    128x96 translation, the 1024x436 fast and dense presets, and one pair-parallel pass over the
    64 mixed pairs on every core."""
    import oracle
    oracle.build()
    out = {"kind": "oracle", "cpu_model": cpu_model(), "nproc": _cores(), "single_core_s": {}}
    l2 = ("l2", False, 0.0)
    with OraclePool(min(3, _cores())) as pool:
        for wl, preset in [("translate128x96", "cfg0"), ("flow", "fast"), ("flow", "dense")]:
            ts = [r[0] for r in pool.map([(wl, preset, [0], None, False, l2)] * 3)]
            out["single_core_s"]["%s_%s" % (wl, preset)] = {"median": statistics.median(ts), "runs": ts}
    procs = _cores()
    with OraclePool(procs) as pool:
        t0 = time.perf_counter()
        res = pool.map([("mixed", "medium", [k], None, False, l2) for k in range(64)])
        wall = time.perf_counter() - t0
    out["mixed64_all_cores"] = {"pairs": 64, "wall_s": wall, "pairs_per_s": 64 / wall, "processes": procs,
                                "sum_single_core_s": sum(r[0] for r in res)}
    print(json.dumps(out))


# ------------------------------------------------------------------------------ GPU arm
class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows if len(r) >= 9 for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_params(dis, args):
    if args.workload == "diff":
        return dis.dis_default_params("default", channels=1, **DIFF_PARAMS)
    wl = WORKLOADS[args.workload]
    return dis.dis_default_params(args.preset, coarsest_scale=wl["coarsest"], channels=wl["channels"],
                                  norm=NORM_CODES[args.norm], fb=1 if args.fb else 0, term_eps=args.term_eps)


def level_dims(w, h, s):
    for _ in range(s):
        w, h = (w + 1) // 2, (h + 1) // 2
    return w, h


def algorithmic_bytes(dis, p, width, height):
    """Bytes each array of the method moves once per stage (float32), per pair."""
    ss, sf, tot = dis.dis_levels(width, height, p)
    N = [level_dims(width, height, s)[0] * level_dims(width, height, s)[1] for s in range(ss + 1)]
    C = p.channels
    b = 8 * C * N[0] + 8 * sum(N[1:ss + 1])                      # read frames, write pyramid
    for s in range(ss, sf - 1, -1):
        b += 8 * N[s] + 8 * (N[s + 1] if s < ss else 0) + 16 * tot // max(1, ss - sf + 1)  # search
        b += 8 * N[s] + 8 * N[s]                                  # densify: frames, U write
        if p.refine:
            outer = s + 1 if p.var_outer < 0 else p.var_outer
            b += outer * (8 * C + 8 + 8 + 8) * N[s]               # refine per outer pass
    if sf > 0:
        b += 8 * N[0]
    return b


def search_flops(dis, p, width, height):
    """Algorithmic FP32 operations of the inverse search of level theta_sf: 12 per bilinear
    sample (3 lerps as sub+FMA, mean accumulation, residual, two FMA accumulations), 11 with one
    degree of freedom (one accumulation); the robust norms' error transform (a square root) is
    not counted.  Returns (flops, patches)."""
    ss, sf, _ = dis.dis_levels(width, height, p)
    w, h = level_dims(width, height, sf)
    ps = p.patch_size
    stride = p.stride_override or max(1, ps - int(np.floor(p.overlap * ps + 1e-4)))
    n = ((w - ps + stride - 1) // stride + 1) * ((h - ps + stride - 1) // stride + 1)
    return n * p.grad_iters * ps * ps * (12 if p.dof == 2 else 11), n


def search_form(p, lanes):
    if p.dof == 1 or p.norm != 0 or p.term_eps > 0:
        return "grouped search, %s%s" % ("one degree of freedom" if p.dof == 1 else "flow",
                                         "" if p.norm == 0 else ", %s norm" % ["l2", "l1", "huber"][p.norm])
    return "search variant %d" % lanes


def workload_config(args, batch, world):
    wl = WORKLOADS[args.workload]
    levels = "4 levels" if args.workload == "diff" else (
        "%d levels" % (wl["coarsest"] + 1) if wl["coarsest"] >= 0 else "automatic levels")
    text = "%s, %s preset, %s, batch %d per GPU" % (wl["text"], args.preset, levels, batch)
    if args.norm != "l2":
        text += ", %s search norm" % args.norm
    if args.fb:
        text += ", forward-backward consistency"
    if args.term_eps > 0:
        text += ", search ends at a step <= %g px" % args.term_eps
    c = {"workload": text, "batch_per_gpu": batch, "preset": args.preset,
         "parallelism": "replicas" if world > 1 else "single"}
    if args.norm != "l2":
        c["norm"] = args.norm
    if args.fb:
        c["fb"] = True
    if args.term_eps > 0:
        c["term_eps"] = args.term_eps
    return c


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def run_ours(args, rank, local, world):
    import torch
    import torch.distributed as tdist
    from paper_1603_03590_gb300 import build, dis, replicas
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=dev)
    barrier = replicas.barrier
    wl = WORKLOADS[args.workload]
    B = args.batch
    uniq = gen_pairs(wl["synth"], min(args.unique, B))
    pairs = [uniq[k % len(uniq)] for k in range(B)]
    p = gpu_params(dis, args)
    C = p.channels
    sizes = [(a.shape[-1], a.shape[-2]) for a, _, _ in pairs]
    Wm, Hm = max(w for w, _ in sizes), max(h for _, h in sizes)
    h = dis.dis_create(Wm, Hm, 2 * B if args.fb else B, C)
    I0d = [torch.from_numpy(a).to(dev) for a, _, _ in pairs]
    I1d = [torch.from_numpy(b).to(dev) for _, b, _ in pairs]
    flows = [torch.empty((hh, ww, 2), device=dev) for ww, hh in sizes]
    arr = dis.make_pairs([(a, b, w, hh, w, f) for a, b, (w, hh), f in zip(I0d, I1d, sizes, flows)])
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    if args.variant is None:
        lanes = dis.dis_autotune(h, arr, B, p, stream)  # before any timing
    else:
        dis.dis_set_search_variant(h, p.patch_size, args.variant)
        lanes = args.variant
    refine_form = dis.dis_get_tuning(h, p.patch_size)[1]

    def step_batched():
        dis.dis_compute_flow_batched(h, arr, B, p, stream)

    def step_plain():
        for k in range(B):
            w, hh = sizes[k]
            dis.dis_compute_flow(h, I0d[k], I1d[k], w, hh, w, p, flows[k], stream)

    def timed(fn, steps, warmup, sample_clocks=False, probe=None):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        barrier()
        clk = Clocks(local) if sample_clocks else None
        evs = []
        t0 = time.perf_counter()
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
            if probe is not None:
                probe.append(dis.dis_probe_ms(h))  # waits for the probed launch of this step only
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - t0
        ms = sum(a.elapsed_time(b) for a, b in evs)
        return ms, wall, (clk.stop() if clk else None)

    # the dominant kernel (the inverse search of the finest level, over the whole batch) is timed
    # inside every timed step by events the library records around that launch in its graph
    sf = p.finest_scale
    dis.dis_set_probe(h, "search", sf)
    probe = []
    ms_b, wall_b, clocks = timed(step_batched, args.steps, args.warmup, sample_clocks=True, probe=probe)
    kernels_per_call = dis.dis_last_call_kernels(h)
    dis.dis_set_probe(h, -1)
    flow0 = flows[0].detach().cpu().numpy().astype(np.float64)  # the timed graph's flow of pair 0
    plain_steps = max(3, args.steps // 4)
    ms_p, _, _ = timed(step_plain, plain_steps, 3)

    # end to end through the public API: pinned host inputs -> device, compute, flows -> host
    hin0 = [torch.from_numpy(a).pin_memory() for a, _, _ in pairs]
    hin1 = [torch.from_numpy(b).pin_memory() for _, b, _ in pairs]
    hout = [torch.empty((hh, w, 2), pin_memory=True) for w, hh in sizes]
    harr = dis.make_pairs([(a, b, w, hh, w, f) for a, b, (w, hh), f in zip(hin0, hin1, sizes, hout)])

    def step_e2e():
        # host frames in, host flows out, through the library's host-buffer call (its copies
        # overlap the computation of the previous step)
        dis.dis_compute_flow_batched_host(h, harr, B, p, stream)

    def timed_e2e(steps, warmup):
        """The whole run of `steps` calls between two events, the last flows in host memory
        before the closing event (the copies of one step overlap the next, so per-step event
        pairs would miss them); L2 flushes between steps run inside."""
        for _ in range(warmup):
            step_e2e()
        dis.dis_host_flows_ready(h, stream)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            flush.fill_(1.0)
            step_e2e()
        dis.dis_host_flows_ready(h, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return e0.elapsed_time(e1)

    e2e_steps = args.steps
    ms_e = timed_e2e(e2e_steps, 3)
    # the flows really arrived: the last step's host flows equal the device-resident result
    step_batched()
    torch.cuda.synchronize()
    assert all(torch.equal(hout[k], flows[k].cpu()) for k in range(B)), "host-buffer flows differ"
    h2d = sum(2 * C * w * hh * 4 for w, hh in sizes)
    d2h = sum(w * hh * 2 * 4 for w, hh in sizes)

    k_ms = statistics.mean(probe)
    fl = [search_flops(dis, p, w, hh) for w, hh in sizes]
    flops, npatch = sum(f for f, _ in fl), sum(n for _, n in fl)
    # one traced call: device time per launch group (stage shares of the batched step)
    stages = {}
    for kind, lev, ms in dis.dis_trace_batched(h, arr, B, p, stream):
        stages[kind] = stages.get(kind, 0.0) + ms

    ms_b, ms_p, ms_e, k_ms = replicas.max_over_ranks([ms_b, ms_p, ms_e, k_ms], device=dev)
    dis.dis_destroy(h)
    if rank != 0:
        return

    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    sm_max = pk.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s: 152 SMs x 128 FP32 lanes x FMA
    value = replicas.aggregate_rate(B * args.steps, world, ms_b / 1000.0)
    plain = replicas.aggregate_rate(B * plain_steps, world, ms_p / 1000.0)
    e2e = replicas.aggregate_rate(B * e2e_steps, world, ms_e / 1000.0)
    abytes = sum(algorithmic_bytes(dis, p, w, hh) for w, hh in sizes)  # per step (the batch)
    achieved = flops / (k_ms / 1000.0) / 1e12
    tr = TRAFFIC.get((args.workload, args.preset, lanes)) if p.norm == 0 and not args.fb and p.term_eps == 0 else None
    line = {
        "metric": wl["metric"], "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_b / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(args, B, world),
                       l2="flushed between timed steps (256 MB write, outside the timed events)"),
        "tuning": {"search_variant": lanes, "refine_launch_form": refine_form,
                   "how": "pinned search variant" if args.variant is not None else "autotuned"},
        "plain": {"value": plain, "unit": UNIT, "ms_per_pair": ms_p / (B * plain_steps)},
        "hbm_roofline": {"algorithmic_bytes_per_pair": abytes / B,
                         "achieved_gbs": abytes / (ms_b / args.steps / 1000.0) / 1e9, "peak_gbs": hbm,
                         "frac": abytes / (ms_b / args.steps / 1000.0) / 1e9 / hbm, "peak_source": "measured"},
        "roofline": {"kernel": "inverse search of level %d over the batch (%d pairs, %d patches, %d iterations, "
                               "%s), timed inside the timed steps"
                               % (sf, B, npatch, p.grad_iters, search_form(p, lanes)),
                     "ms_per_launch": k_ms, "launches_timed": len(probe),
                     "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak,
                     "traffic": tr[0] * B if tr else None,
                     "traffic_source": ("ncu DRAM bytes per pair, scaled by the pairs of the launch: " + tr[1])
                     if tr else "no capture of this configuration's launch",
                     "algorithmic_flops_per_launch": flops,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % sm_max},
        "stages_ms_per_step": {k: round(v, 4) for k, v in stages.items()},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": kernels_per_call * args.steps if kernels_per_call > 0 else None,
        "gpu_launches_source": "kernel nodes of the replayed CUDA graph (dis_last_call_kernels) x timed steps",
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        cb, parity = cpu_baseline(args, flow0 if args.workload == "flow" else None)
        line["cpu_baseline"] = cb
        if parity is not None:
            line["parity"] = parity
    print(json.dumps(line))


def run_diff(args, rank, local, world):
    """The differentiable form: per step, each pair's forward map (FP32 search recording its
    increments, FP64 replay of the frozen map), the photometric loss and the backward pass to
    both frames and the initial flow.  Batched: the pairs side by side, one handle and stream per
    pair (BatchedDifferentiableDIS), one backward over the sum of their losses; plain: the same
    pairs one after another on one handle."""
    import torch
    from paper_1603_03590_gb300 import autograd, build, replicas
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=dev)
    B = args.batch
    uniq = gen_pairs(WORKLOADS["diff"]["synth"], min(args.unique, B))
    pairs = [uniq[k % len(uniq)] for k in range(B)]
    H, W = pairs[0][0].shape
    single = autograd.DifferentiableDIS(W, H, "default", **DIFF_PARAMS)
    batched = autograd.BatchedDifferentiableDIS(W, H, B, "default", **DIFF_PARAMS)
    hs, ws = single.coarsest_shape(W, H)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    I0d = [torch.from_numpy(a).to(dev) for a, _, _ in pairs]
    I1d = [torch.from_numpy(b).to(dev) for _, b, _ in pairs]
    init = [torch.zeros((hs, ws, 2), device=dev) for _ in pairs]

    def leaves(ts):
        return [t.detach().requires_grad_(True) for t in ts]

    def step_batched(a0=None, a1=None, u0=None):
        a, b, u = leaves(a0 or I0d), leaves(a1 or I1d), leaves(u0 or init)
        flows = batched(a, b, u)
        losses = [autograd.photometric_loss(x, y, f) for x, y, f in zip(a, b, flows)]
        torch.stack(losses).sum().backward()
        return [(l.detach(), x.grad, y.grad, z.grad) for l, x, y, z in zip(losses, a, b, u)]

    def step_plain():
        out = []
        for a0, b0, u0 in zip(I0d, I1d, init):
            a, b, u = leaves([a0, b0, u0])
            loss = autograd.photometric_loss(a, b, single(a, b, u))
            loss.backward()
            out.append((loss.detach(), a.grad, b.grad, u.grad))
        return out

    def timed(fn, steps, warmup, clocks=False):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        replicas.barrier()
        clk = Clocks(local) if clocks else None
        evs = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs), (clk.stop() if clk else None)

    ms, clocks = timed(step_batched, args.steps, args.warmup, clocks=True)
    ms_p, _ = timed(step_plain, max(3, args.steps // 2), 3)
    # the batched gradients are those of single-pair calls, bit for bit
    gb, gp = step_batched(), step_plain()
    torch.cuda.synchronize()
    assert all(torch.equal(x, y) for rb, rp in zip(gb, gp) for x, y in zip(rb, rp)), "batched gradients differ"
    # end to end: frames and initial flows from pinned host memory, loss and the three gradients
    # back to host memory, every step
    hin = [(torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory(), torch.zeros((hs, ws, 2)).pin_memory())
           for a, b, _ in pairs]
    hout = [(torch.empty(1, dtype=torch.float32, pin_memory=True), torch.empty((H, W), pin_memory=True),
             torch.empty((H, W), pin_memory=True), torch.empty((hs, ws, 2), pin_memory=True)) for _ in pairs]

    def step_e2e():
        a = [x.to(dev, non_blocking=True) for x, _, _ in hin]
        b = [y.to(dev, non_blocking=True) for _, y, _ in hin]
        u = [z.to(dev, non_blocking=True) for _, _, z in hin]
        for outs, r in zip(hout, step_batched(a, b, u)):
            for dst, src in zip(outs, r):
                dst.copy_(src.reshape(dst.shape), non_blocking=True)

    for _ in range(3):
        step_e2e()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        flush.fill_(1.0)
        step_e2e()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e = e0.elapsed_time(e1)
    ms, ms_p, ms_e = replicas.max_over_ranks([ms, ms_p, ms_e], device=dev)
    single.close()
    batched.close()
    if rank != 0:
        return
    plain_steps = max(3, args.steps // 2)
    value = replicas.aggregate_rate(B * args.steps, world, ms / 1000.0)
    plain = replicas.aggregate_rate(B * plain_steps, world, ms_p / 1000.0)
    e2e = replicas.aggregate_rate(B * args.steps, world, ms_e / 1000.0)
    line = {"metric": WORKLOADS["diff"]["metric"], "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 search, f64 replay and adjoint", "data": "synthetic",
            "config": dict(workload_config(args, B, world), l2="flushed between timed steps (256 MB write)"),
            "plain": {"value": plain, "unit": UNIT, "ms_per_pair": ms_p / (B * plain_steps),
                      "note": "the same pairs one after another on one handle"},
            "roofline": None,
            "roofline_note": "no per-kernel work model of the FP64 replay and adjoint: a chain of small "
                             "latency-bound launches (profiles/launches_diff512x256_batch8.md)",
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": B * (2 * H * W * 4 + hs * ws * 8),
                    "d2h_bytes_per_step": B * (4 + 2 * H * W * 4 + hs * ws * 8)},
            "gpu_launches": DIFF_KERNELS_PER_PAIR * B * args.steps,
            "gpu_launches_source": "library kernels per pair and step in the ncu launch list of this step "
                                   "(profiles/launches_diff512x256_batch8.md) x pairs x timed steps",
            "clocks": clocks}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)[0]
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # 60 steps of 32 pairs take about 0.9 s: long enough for several clock samples at 200 ms
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="flow", choices=sorted(WORKLOADS))
    ap.add_argument("--norm", default="l2", choices=sorted(NORM_CODES))
    ap.add_argument("--fb", action="store_true", help="forward-backward consistency")
    ap.add_argument("--term-eps", type=float, default=0.0, help="early termination of the patch search (px)")
    ap.add_argument("--preset", default=None, help="default: the workload's (dense, medium, stereo_dense)")
    ap.add_argument("--batch", type=int, default=None, help="default: the workload's batch")
    ap.add_argument("--unique", type=int, default=None,
                    help="distinct synthetic pairs cycled through the batch (default: the batch size)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-report", action="store_true", help="time the oracle's CPU cases only (no GPU)")
    ap.add_argument("--variant", type=int, default=None,
                    help="search variant to pin (dis_search_variants); default: the autotuner's choice")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    wl = WORKLOADS[args.workload]
    args.preset = args.preset or wl["preset"]
    args.batch = args.batch or wl["batch"]
    args.unique = args.unique or args.batch
    if args.cpu_report:
        return cpu_report(args)

    from paper_1603_03590_gb300 import replicas
    rank, local, world = replicas.env_rank_world()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "diff":
        return run_diff(args, rank, local, world)
    return run_ours(args, rank, local, world)


if __name__ == "__main__":
    main()
