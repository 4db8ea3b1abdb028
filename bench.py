#!/usr/bin/env python
"""Benchmark of the DIS hot path: frame-pairs/s at 1024x436 on synthetic layered scenes.

One step = the whole method (pyramid, per-level patch search, densification, variational
refinement, up-scaling) over one batch of `--batch` frame pairs of 1024x436, run by the
batched entry point (one CUDA-graph replay of persistent kernels over all pairs).  The same
batch through sequential single-pair calls (the plain form) is timed beside it.  Inputs are
resident in HBM for `value`; `e2e` adds the host->device copy of the inputs from pinned
memory and the device->host read of the flows to every step.  L2 is flushed (a 256 MB
write) between timed steps, outside the timed events.

--impl reference times the FP64 CPU oracle (the correctness reference of this repository)
on the host cores instead, on a bounded sample of the same workload.

--workload stereo measures depth from stereo instead (supplementary, depth from stereo):
rectified synthetic pairs of 1440x960 (half-resolution Middlebury size, disparities up to
96 px), the dense preset with one degree of freedom and theta_it halved, batches of 8.
--norm l1 / huber runs the patch search with that robust error norm (supplementary, robust
error norms).  --fb adds forward-backward consistency (supplementary Sec. B (ii)): both
directions per pair, merged in the densification; the forward flows are the output.
--term-eps E stops each patch's search after its first step of at most E px (early termination
for small residuals, supplementary Sec. C).

Multi-GPU (torchrun): frame pairs are independent, so each rank runs its own batch
(replicas, weak scaling, no collective on the data path); value = all ranks' pairs / max time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

UNIT = "frame-pairs/s"
# name -> (metric, width, height, default preset, default batch, theta_ss, workload text)
WORKLOADS = {
    "flow": ("DIS flow frame-pairs/s at 1024x436 (batched)", 1024, 436, "dense", 32, 4, "layered 1024x436"),
    "stereo": ("DIS stereo frame-pairs/s at 1440x960 (batched)", 1440, 960, "stereo_dense", 8, 5,
               "rectified stereo 1440x960 (horizontal layered scenes, disparities up to 96 px)"),
}
NORM_CODES = {"l2": 0, "l1": 1, "huber": 2}


def workload_pair(workload, k):
    from paper_1603_03590_gb300 import synth
    if workload == "stereo":
        return synth.workload_pair("stereo1440x960", k)
    return synth.layered_pair(1000 + k)


def preset_params(dis, name, workload="flow", norm="l2", fb=False, term_eps=0.0):
    # theta_ss fixed per workload (five levels at 1024x436, six at 1440x960: the automatic value)
    return dis.dis_default_params(name, coarsest_scale=WORKLOADS[workload][5], norm=NORM_CODES[norm],
                                  fb=1 if fb else 0, term_eps=term_eps)


def search_form(p, lanes):
    if p.dof == 1 or p.norm != 0 or p.term_eps > 0:
        return "grouped search, %s%s" % ("one degree of freedom" if p.dof == 1 else "flow",
                                         "" if p.norm == 0 else ", %s norm" % ["l2", "l1", "huber"][p.norm])
    return "search variant %d" % lanes


def launches_per_call(dis, p, width, height, lanes, batch, refine_form=1):
    # (forward-backward consistency: the densification of each level is five launches)
    """Kernels one batched call launches (mirrors the host plan: prep, pyramid, per level search
    planes (lane-per-patch search variant only) + search + densify (+ refinement: 3 setup, then
    per outer pass one fused launch, two when the level has more than 128 Ki pixels over the batch,
    or weights + 2 x inner per-sweep launches, then apply), final up-scaling)."""
    ss, sf, _ = dis.dis_levels(width, height, p)
    w, h = width, height
    dims = [(w, h)]
    for _ in range(ss):
        w, h = (w + 1) // 2, (h + 1) // 2
        dims.append((w, h))
    n = 1 + ss
    dirs = 2 if p.fb else 1
    for s in range(ss, sf - 1, -1):
        n += 2 + (1 if lanes == 1 else 0) + (4 if p.fb else 0)
        if p.refine:
            outer = s + 1 if p.var_outer < 0 else p.var_outer
            npx = dirs * batch * dims[s][0] * dims[s][1]
            fused = 0 < p.var_inner <= 5 and refine_form != 0
            chunks = 2 if refine_form == 3 or (refine_form == 1 and npx > (1 << 17)) else 1
            n += 3 + (outer * chunks if fused else outer * (1 + 2 * p.var_inner)) + 1
    return n + (1 if sf > 0 else 0)


def algorithmic_bytes(dis, p, width, height):
    """Bytes each array of the method moves once per stage (float32), per pair."""
    ss, sf, tot = dis.dis_levels(width, height, p)
    dims = [(width, height)]
    for _ in range(ss):
        dims.append(((dims[-1][0] + 1) // 2, (dims[-1][1] + 1) // 2))
    N = [w * h for w, h in dims]
    b = 8 * N[0] + 8 * sum(N[1:ss + 1])                          # read frames, write pyramid
    for s in range(ss, sf - 1, -1):
        b += 8 * N[s] + 8 * (N[s + 1] if s < ss else 0) + 16 * tot // max(1, ss - sf + 1)  # search
        b += 8 * N[s] + 8 * N[s]                                  # densify: frames, U write
        if p.refine:
            outer = s + 1 if p.var_outer < 0 else p.var_outer
            b += outer * (16 + 8 + 8) * N[s]                      # refine per outer pass
    if sf > 0:
        b += 8 * N[0]
    return b


def search_flops(dis, p, width, height):
    """Algorithmic FP32 operations of the inverse search of level theta_sf: 12 per bilinear
    sample (3 lerps as sub+FMA, mean accumulation, residual, two FMA accumulations), 11 with one
    degree of freedom (one accumulation); the robust norms' error transform (a square root) is
    not counted."""
    ss, sf, _ = dis.dis_levels(width, height, p)
    w, h = width, height
    for _ in range(sf):
        w, h = (w + 1) // 2, (h + 1) // 2
    ps = p.patch_size
    stride = p.stride_override or max(1, ps - int(np.floor(p.overlap * ps + 1e-4)))
    n = ((w - ps + stride - 1) // stride + 1) * ((h - ps + stride - 1) // stride + 1)
    return n * p.grad_iters * ps * ps * (12 if p.dof == 2 else 11), (w, h), n


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


def cpu_baseline(preset, workload="flow", norm="l2", fb=False, term_eps=0.0):
    """FP64 oracle on one pair of the workload at half width and height (a quarter of the area,
    one level fewer; the method's cost is linear in area), scaled to pairs/s at full size."""
    import oracle
    from paper_1603_03590_gb300 import synth
    _, W, H, _, _, ss, _ = WORKLOADS[workload]
    w, h = W // 2, H // 2
    I0, I1, _ = synth.layered_pair(1000, width=w, height=h, max_disp=20.0 if workload == "flow" else 48.0,
                                   horizontal=workload == "stereo")
    from paper_1603_03590_gb300 import dis
    p = preset_params(dis, preset, workload, norm, fb, term_eps)
    q = oracle.params(patch_size=p.patch_size, overlap=round(float(p.overlap), 6), grad_iters=p.grad_iters,
                      coarsest_scale=ss - 1, finest_scale=p.finest_scale, refine=p.refine, dof=p.dof, norm=p.norm,
                      huber_b=round(float(p.huber_b), 6), fb=p.fb, term_eps=float(p.term_eps))
    oracle.build()
    t = time.perf_counter()
    oracle.dis_flow(I0, I1, q)
    dt = time.perf_counter() - t
    return {"value": 0.25 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "one %dx%d pair (1/4 of the %dx%d area, one level fewer), %s preset, %.1f s; "
                      "scaled by area to pairs/s at %dx%d" % (w, h, W, H, preset, dt, W, H)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    steps, warmup = args.steps, args.warmup
    metric, W, H, _, _, ss, wtext = WORKLOADS[args.workload]
    times = []
    for k in range(warmup + steps):
        r = cpu_baseline(args.preset, args.workload, args.norm, args.fb, args.term_eps)
        if k >= warmup:
            times.append(0.25 / r["value"])
    dt = sum(times)
    value = steps * 0.25 / dt
    line = {"impl": "reference", "metric": metric, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warmup, "ms_per_step": 1000.0 * args.batch / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, args.batch, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "per step one %dx%d pair of the workload (1/4 of the area, one level "
                                       "fewer), scaled by area to pairs/s at %dx%d; the batch's other pairs "
                                       "would cost the same each" % (W // 2, H // 2, W, H)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def workload_config(args, batch, world):
    _, W, H, _, _, ss, wtext = WORKLOADS[args.workload]
    text = "%s, %s preset, %d levels, batch %d per GPU" % (wtext, args.preset, ss + 1, batch)
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
    ap.add_argument("--preset", default=None, help="default: dense (flow), stereo_dense (stereo)")
    ap.add_argument("--batch", type=int, default=None, help="default: 32 (flow), 8 (stereo)")
    ap.add_argument("--unique", type=int, default=4, help="distinct synthetic pairs cycled through the batch")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variant", type=int, default=None,
                    help="search variant to pin (dis_search_variants); default: the autotuner's choice")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    metric, W, H, dpreset, dbatch, _, _ = WORKLOADS[args.workload]
    args.preset = args.preset or dpreset
    args.batch = args.batch or dbatch

    from paper_1603_03590_gb300 import replicas
    rank, local, world = replicas.env_rank_world()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as tdist
    from paper_1603_03590_gb300 import build, dis, synth
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=dev)
    barrier = replicas.barrier

    B = args.batch
    uniq = [workload_pair(args.workload, k) for k in range(args.unique)]
    p = preset_params(dis, args.preset, args.workload, args.norm, args.fb, args.term_eps)
    h = dis.dis_create(W, H, 2 * B if args.fb else B, 1)
    I0d = [torch.from_numpy(uniq[k % len(uniq)][0]).to(dev) for k in range(B)]
    I1d = [torch.from_numpy(uniq[k % len(uniq)][1]).to(dev) for k in range(B)]
    flows = [torch.empty((H, W, 2), device=dev) for _ in range(B)]
    arr = dis.make_pairs([(a, b, W, H, W, f) for a, b, f in zip(I0d, I1d, flows)])
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
            dis.dis_compute_flow(h, I0d[k], I1d[k], W, H, W, p, flows[k], stream)

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
    ss, sf, _ = dis.dis_levels(W, H, p)
    dis.dis_set_probe(h, "search", sf)
    probe = []
    ms_b, wall_b, clocks = timed(step_batched, args.steps, args.warmup, sample_clocks=True, probe=probe)
    dis.dis_set_probe(h, -1)
    plain_steps = max(3, args.steps // 4)
    ms_p, _, _ = timed(step_plain, plain_steps, 3)

    # end to end through the public API: pinned host inputs -> device, compute, flows -> host
    hin0 = [torch.from_numpy(uniq[k % len(uniq)][0]).pin_memory() for k in range(B)]
    hin1 = [torch.from_numpy(uniq[k % len(uniq)][1]).pin_memory() for k in range(B)]
    hout = [torch.empty((H, W, 2), pin_memory=True) for _ in range(B)]

    harr = dis.make_pairs([(a, b, W, H, W, f) for a, b, f in zip(hin0, hin1, hout)])

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
    h2d = B * 2 * W * H * 4
    d2h = B * W * H * 2 * 4

    k_ms = statistics.mean(probe)
    flops, (lw, lh), npatch = search_flops(dis, p, W, H)
    # one traced call: device time per launch group (stage shares of the batched step)
    stages = {}
    for kind, lev, ms in dis.dis_trace_batched(h, arr, B, p, stream):
        stages[kind] = stages.get(kind, 0.0) + ms

    # max over ranks
    ms_b, ms_p, ms_e, k_ms = replicas.max_over_ranks([ms_b, ms_p, ms_e, k_ms], device=dev)
    dis.dis_destroy(h)
    if rank != 0:
        return

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s: 152 SMs x 128 FP32 lanes x FMA
    value = replicas.aggregate_rate(B * args.steps, world, ms_b / 1000.0)
    plain = replicas.aggregate_rate(B * plain_steps, world, ms_p / 1000.0)
    e2e = replicas.aggregate_rate(B * e2e_steps, world, ms_e / 1000.0)
    abytes = algorithmic_bytes(dis, p, W, H)
    achieved = flops * B / (k_ms / 1000.0) / 1e12
    config = workload_config(args, B, world)
    config.update({"l2": "flushed between timed steps (256 MB write, outside the timed events)",
                   "search_variant": lanes, "refine_launch_form": refine_form,
                   "tuning": "pinned search variant" if args.variant is not None else "autotuned"})
    line = {
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_b / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config,
        "plain": {"value": plain, "unit": UNIT, "ms_per_pair": ms_p / (B * plain_steps)},
        "hbm_roofline": {"algorithmic_bytes_per_pair": abytes,
                         "achieved_gbs": abytes * value / world / 1e9, "peak_gbs": hbm,
                         "frac": abytes * value / world / 1e9 / hbm},
        "roofline": {"kernel": "inverse search of level %d over the batch (%d pairs x %d patches x %d iterations, "
                               "%s), timed inside the timed steps"
                               % (sf, B, npatch, p.grad_iters, search_form(p, lanes)),
                     "ms_per_launch": k_ms, "launches_timed": len(probe),
                     "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak,
                     # DRAM bytes of the same launch at 4 pairs (ncu dram__bytes_read.sum +
                     # dram__bytes_write.sum, 17.82 MB: the level images and the coarser flow,
                     # each read once), scaled by the pairs a launch processes
                     "traffic": (17.82e6 * B / 4 if args.workload == "flow" and args.preset == "dense" and lanes == 16
                                 and p.norm == 0 else None),
                     "traffic_source": "ncu capture of the 4-pair launch, scaled by pairs (profiles/)",
                     "algorithmic_flops_per_launch": flops * B,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % sm_max},
        "stages_ms_per_step": {k: round(v, 4) for k, v in stages.items()},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_call(dis, p, W, H, lanes if p.dof == 2 and p.norm == 0 and p.term_eps == 0 else 0, B,
                                          refine_form) * args.steps,
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.preset, args.workload, args.norm, args.fb, args.term_eps)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
