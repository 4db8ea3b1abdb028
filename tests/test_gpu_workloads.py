"""The batched workloads at their full sizes, through the C ABI.

- 64 pairs of mixed resolution (320x240 ... 1920x1080, displacements 4 % of the width), medium
  preset, one batched call with the autotuned search form: every flow equals the single-pair
  call bit for bit, and the first pair of every resolution (up to three of 320x240) matches the
  FP64 oracle end to end; the end-point error against the generated ground truth is reported
  for all.
- 4 RGB pairs at 3840x2160 (2 degree rotation, displacements up to 200 px), dense preset with 7
  levels: batched equals single-pair calls bit for bit and repeats bit for bit, the flow is
  informative (end-point error under half that of a zero flow), and pair 0 matches the FP64
  oracle end to end (channel-mean search and densification, per-channel data terms in the
  refinement: supplementary Sec. B (i)); the finest level's refinement, run alone on the full
  frame, also matches the oracle on crops (the refinement at level 0 reaches no further than one
  outer pass of 10 half-sweeps plus the 2-pixel derivative stencils, so a crop with a 16-pixel
  margin reproduces the full-frame result in its interior exactly).

The oracle runs of an end-to-end comparison (the flow and its two perturbed replicas, which
mark the pixels the FP64 result does not determine at FP32 resolution) run side by side in
spawned processes.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle
from paper_1603_03590_gb300 import synth
from test_gpu_parity import STAGE_TOL, check_e2e, host, ndimage_smooth, oracle_e2e_many, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_03590_gb300 import build
    build.build()
    from paper_1603_03590_gb300 import dis
    return torch, dis, torch.device("cuda:0")


def epe(f, gt):
    return float(np.linalg.norm(f - gt, axis=-1).mean())


def _gen(args):
    name, i = args
    return synth.workload_pair(name, i)


def oracle_e2e_parallel(cases):
    """(flow, spread) of test_gpu_parity.oracle_e2e for every (I0, I1, oracle params) case."""
    return oracle_e2e_many([(I0, I1, q, {}) for I0, I1, q in cases])


def generate(name, n):
    """The workload's pairs, generated in a pool of spawned processes (the seeded generator is
    pure numpy / scipy and slow at 1080p and 4K)."""
    with mp.get_context("spawn").Pool(min(n, os.cpu_count() or 1)) as pool:
        return pool.map(_gen, [(name, i) for i in range(n)], chunksize=1)


def test_mixed_batch_of_64_pairs(env):
    torch, dis, dev = env
    pairs = generate("mixed", 64)
    p = dis.dis_default_params("medium")
    Wm = max(a.shape[1] for a, _, _ in pairs)
    Hm = max(a.shape[0] for a, _, _ in pairs)
    h = dis.dis_create(Wm, Hm, len(pairs), 1)
    try:
        dev_pairs = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)) for a, b, _ in pairs]
        flows = [torch.full((a.shape[0], a.shape[1], 2), float("nan"), device=dev) for a, _, _ in pairs]
        items = [(da, db, a.shape[1], a.shape[0], a.shape[1], f) for (da, db), (a, _, _), f in zip(dev_pairs, pairs, flows)]
        arr = dis.make_pairs(items)
        variant = dis.dis_autotune(h, arr, len(items), p)
        dis.dis_compute_flow_batched(h, arr, len(items), p)
        torch.cuda.synchronize()
        batched = [host(f) for f in flows]
        for k, ((da, db), (a, _, _)) in enumerate(zip(dev_pairs, pairs)):
            f = torch.full((a.shape[0], a.shape[1], 2), float("nan"), device=dev)
            dis.dis_compute_flow(h, da, db, a.shape[1], a.shape[0], a.shape[1], p, f)
            torch.cuda.synchronize()
            assert np.array_equal(host(f), batched[k]), (k, a.shape)
    finally:
        dis.dis_destroy(h)
    sizes = sorted({a.shape for a, _, _ in pairs})
    for shp in sizes:
        e = [epe(batched[k], gt) for k, (a, _, gt) in enumerate(pairs) if a.shape == shp]
        print("mixed batch, search variant %d: %d pairs of %dx%d, mean EPE %.3f px" % (variant, len(e), shp[1], shp[0],
                                                                                      np.mean(e)))
    # the first pair of every resolution (three of the smallest) against the oracle end to end
    picked = []
    for shp in sizes:
        ks = [k for k, (a, _, _) in enumerate(pairs) if a.shape == shp]
        picked += ks[:3] if shp == (240, 320) else ks[:1]
    assert {pairs[k][0].shape for k in picked} == set(synth_shapes()), "the seeded draw holds every resolution"
    refs = oracle_e2e_parallel([(pairs[k][0], pairs[k][1], oracle_params(p)) for k in picked])
    for k, rs in zip(picked, refs):
        I0, I1, gt = pairs[k]
        check_e2e("mixed pair %d (%dx%d, medium)" % (k, I0.shape[1], I0.shape[0]), batched[k], rs, gt)


def synth_shapes():
    return [(h, w) for w, h in synth.MIXED_SIZES]


@pytest.mark.slow
def test_rgb_4k_batch_of_4(env):
    torch, dis, dev = env
    pairs = generate("rgb3840x2160", 4)
    W, H, C = 3840, 2160, 3
    p = dis.dis_default_params("dense", channels=C, coarsest_scale=6)
    assert dis.dis_levels(W, H, p)[0] == 6  # 7 levels
    h = dis.dis_create(W, H, len(pairs), C)
    try:
        dev_pairs = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)) for a, b, _ in pairs]
        runs = []
        for _ in range(2):
            flows = [torch.full((H, W, 2), float("nan"), device=dev) for _ in pairs]
            arr = dis.make_pairs([(da, db, W, H, W, f) for (da, db), f in zip(dev_pairs, flows)])
            dis.dis_compute_flow_batched(h, arr, len(pairs), p)
            torch.cuda.synchronize()
            runs.append([host(f) for f in flows])
        f = torch.full((H, W, 2), float("nan"), device=dev)
        dis.dis_compute_flow(h, dev_pairs[0][0], dev_pairs[0][1], W, H, W, p, f)
        torch.cuda.synchronize()
        plain0 = host(f)
    finally:
        dis.dis_destroy(h)
    for k, (_, _, gt) in enumerate(pairs):
        assert np.isfinite(runs[0][k]).all()
        assert np.array_equal(runs[0][k], runs[1][k]), k
        e = epe(runs[0][k], gt)
        zero = float(np.linalg.norm(gt, axis=-1).mean())  # the end-point error of a zero flow
        print("rgb 3840x2160 pair %d: EPE %.3f px (zero flow: %.3f px; displacements up to %.1f px)"
              % (k, e, zero, float(np.abs(gt).max())))
        assert e < 0.5 * zero
    assert np.array_equal(plain0, runs[0][0])
    # pair 0 end to end against the oracle
    I0, I1, gt = pairs[0]
    (ref,) = oracle_e2e_parallel([(I0, I1, oracle_params(p))])
    check_e2e("rgb 3840x2160 pair 0 (dense, 7 levels)", runs[0][0], ref, gt)

    # the finest level's refinement alone, on the full frame, against the oracle on crops
    I0, I1, _ = pairs[0]
    P0 = (I0 * 255.0).astype(np.float32)
    P1 = (I1 * 255.0).astype(np.float32)
    g = np.random.default_rng(11)
    U0 = (ndimage_smooth(g.normal(0, 2.0, (H // 8, W // 8, 2))).repeat(8, 0).repeat(8, 1) * 3.0).astype(np.float32)
    a = torch.from_numpy(P0).to(dev)
    b = torch.from_numpy(P1).to(dev)
    U = torch.from_numpy(U0).to(dev)
    U2 = U.clone()
    h = dis.dis_create(W, H, 1, C)
    try:
        dis.dis_refine_level(h, a, b, W, H, W, C, U, 1, 5)
        dis.dis_set_refine_fusion(h, 2)  # one fused launch on all 8.3 M pixels too
        dis.dis_refine_level(h, a, b, W, H, W, C, U2, 1, 5)
        U3 = torch.from_numpy(U0).to(dev)
        dis.dis_set_refine_fusion(h, 0)  # and one launch per half-sweep
        dis.dis_refine_level(h, a, b, W, H, W, C, U3, 1, 5)
        torch.cuda.synchronize()
    finally:
        dis.dis_destroy(h)
    assert torch.equal(U, U2) and torch.equal(U, U3)
    Ug = host(U)
    M = 16
    for (y0, x0, hh, ww) in [(0, 0, 96, 128), (1000, 1800, 96, 96), (H - 80, W - 112, 80, 112)]:
        ya, xa = max(0, y0 - M), max(0, x0 - M)
        yb, xb = min(H, y0 + hh + M), min(W, x0 + ww + M)
        Uo = oracle.refine_level(P0[:, ya:yb, xa:xb].astype(np.float64), P1[:, ya:yb, xa:xb].astype(np.float64),
                                 U0[ya:yb, xa:xb].astype(np.float64), 1, 5)
        got = Ug[y0:y0 + hh, x0:x0 + ww]
        ref = Uo[y0 - ya:y0 - ya + hh, x0 - xa:x0 - xa + ww]
        err = float(np.abs(got - ref).max())
        print("rgb 3840x2160 level-0 refinement, crop at (%d, %d): max |dU| %.2e" % (x0, y0, err))
        assert err <= STAGE_TOL
