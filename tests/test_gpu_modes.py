"""Stereo (one degree of freedom) and robust error norms on the GPU, against the FP64 oracle,
through the C ABI.

- Search stage: every mode (dof 1 with L2, L1, Huber; dof 2 with L1, Huber) on the level
  inputs of the flow parity cases plus a scene whose right half has no horizontal texture
  (flat patches of the scalar search), max |du| <= 1e-3 px on the patches whose FP64 result is
  determined at FP32 resolution; in dof 1 the v component equals u_init exactly.
- Refinement stage with dof 1: the oracle within 1e-3 px, v untouched bit for bit, every launch
  form of the refinement equal bit for bit.
- End to end: stereo presets on horizontal pairs and robust norms on flow pairs, the oracle
  within the end-to-end bar (mean 0.01 px, 99.9th percentile 0.05 px); batched calls equal
  single-pair calls; in stereo the flow's v is exactly 0.
"""
import numpy as np
import pytest

import oracle
from paper_1603_03590_gb300 import synth
from test_gpu_parity import (STAGE_TOL, check_e2e, gpu_level_images, host, ndimage_smooth, oracle_e2e,
                             oracle_params, run_gpu, to_dev)
from test_gpu_parity import compare_search

pytestmark = pytest.mark.gpu

MODES = [(1, 0, 5.0), (2, 1, 5.0), (2, 2, 5.0), (2, 2, 1.0), (1, 1, 5.0), (1, 2, 5.0)]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_03590_gb300 import build
    build.build()
    from paper_1603_03590_gb300 import dis
    return torch, dis, torch.device("cuda:0")


def stripes_pair(seed=31, W=96, H=64):
    """Random texture on the left half; on the right half a texture that varies along y only
    (no horizontal gradient: flat for the scalar search, and for the 2x2 one).  Frame 1 is
    frame 0 shifted by 1.3 px along x (cubic spline) plus noise of 0.2 grey levels: an exact
    integer shift would leave residuals at zero, where the L1 transform sqrt|e| amplifies FP32
    rounding ~100-fold (the FP64 search moves by 1e-2 px under a 1e-4 change of I1) and no
    FP32 search is determined to 1e-3 px."""
    from scipy import ndimage
    g = np.random.default_rng(seed)
    I0 = ndimage.gaussian_filter(g.standard_normal((H, W)), 1.5)
    col = ndimage.gaussian_filter(g.standard_normal(H), 1.5)
    I0[:, W // 2:] = col[:, None]
    I0 = 0.5 + 0.15 * I0 / np.abs(I0).max()
    I1 = ndimage.shift(I0, (0.0, 1.3), order=3, mode="nearest") + g.normal(0, 0.2 / 255, I0.shape)
    return I0.astype(np.float32), I1.astype(np.float32)


def search_case(case):
    if case == "translate":
        I0, I1, _ = synth.translation_pair(0)
        return I0, I1, 0, 8, 4, 16
    if case == "ragged":
        I0, I1, _ = synth.layered_pair(11, width=173, height=91, max_disp=6.0)
        return I0, I1, 0, 9, 4, 40
    if case == "stereo":
        I0, I1, _ = synth.workload_pair("stereo320x240", 0)
        return I0, I1, 0, 8, 4, 32
    if case == "stripes":
        I0, I1 = stripes_pair()
        return I0, I1, 0, 5, 3, 20
    I0, I1, _ = synth.layered_pair(1000)
    return I0, I1, 2, 12, 3, 128


@pytest.mark.parametrize("case", ["translate", "ragged", "layered-dense", "stereo", "stripes"])
def test_search_modes_stage(env, case):
    torch, dis, dev = env
    I0, I1, lv, ps, stride, iters = search_case(case)
    a, b, W, H, pitch = gpu_level_images(torch, dis, dev, I0, I1, lv)[lv]
    g = np.random.default_rng(5)
    wc, hc = (W + 1) // 2, (H + 1) // 2
    Uc_h = ndimage_smooth(g.normal(0, 1.5, (hc, wc, 2))).astype(np.float32)
    Uc = torch.from_numpy(Uc_h).to(dev)
    nx, ny = oracle.grid_n(W, ps, stride), oracle.grid_n(H, ps, stride)
    A, B = host(a, W), host(b, W)
    widths = dis.dis_search_mode_variants(ps)
    assert widths
    for dof, norm, hb in MODES:
        refs = None
        outs = {}
        # variant 0 is the first width; every width is compared with the oracle
        for variant in [0] + widths:
            u = torch.zeros((ny * nx, 2), device=dev)
            ui = torch.zeros((ny * nx, 2), device=dev)
            st = torch.zeros(ny * nx, dtype=torch.int32, device=dev)
            dis.dis_search_level_ex2(a, b, W, H, pitch, Uc, wc, hc, 2.0, ps, stride, iters, variant, dof, norm, hb,
                                     u, ui, st)
            torch.cuda.synchronize()
            outs[variant] = (host(u), host(ui), st.cpu().numpy())
        assert all(np.array_equal(x, y) for x, y in zip(outs[0], outs[widths[0]]))
        for variant in widths:
            u_g, ui_g, st_g = outs[variant]
            if dof == 1:
                assert np.array_equal(u_g[:, 1], ui_g[:, 1])
            mode = dict(dof=dof, norm=norm, huber_b=hb)
            e, ndiff, refs = compare_search(A, B, Uc_h.astype(np.float64), 2.0, ps, stride, iters, u_g, ui_g, st_g,
                                            refs, mode=mode)
            nflat = int((st_g == 2).sum())
            print("search %s dof %d norm %d b %.1f width %d: %d patches (%d flat), max |du| %.2e, %s"
                  % (case, dof, norm, hb, variant, nx * ny, nflat, e, ndiff))
            assert e <= STAGE_TOL
            if case == "stripes":
                assert nflat > 0  # the right half is flat
    u = torch.zeros((ny * nx, 2), device=dev)
    for bad in [(3, 0, 5.0), (0, 0, 5.0), (2, 3, 5.0), (2, 2, 0.0), (2, 2, float("nan"))]:
        with pytest.raises(dis.DisError):
            dis.dis_search_level_ex2(a, b, W, H, pitch, Uc, wc, hc, 2.0, ps, stride, iters, 0, *bad, u)
    not_mode = [v for v in dis.dis_search_variants(ps) if v not in widths]
    if not_mode:  # a flow-only form (lane per patch, cooperative) is not a variant of these searches
        with pytest.raises(dis.DisError):
            dis.dis_search_level_ex2(a, b, W, H, pitch, Uc, wc, hc, 2.0, ps, stride, iters, not_mode[0], 1, 0, 5.0, u)


@pytest.mark.parametrize("case", ["stereo", "ragged", "tiny"])
def test_refine_stereo_stage(env, case):
    torch, dis, dev = env
    outer, inner = 2, 5
    if case == "stereo":
        I0, I1, _ = synth.workload_pair("stereo320x240", 1)
    elif case == "ragged":
        I0, I1, _ = synth.layered_pair(12, width=173, height=91, max_disp=6.0, horizontal=True)
        outer, inner = 3, 7
    else:
        I0, I1, _ = synth.layered_pair(15, width=13, height=9, max_disp=1.0, n_ellipses=1, horizontal=True)
    H, W = I0.shape
    P0 = (I0 * 255.0).astype(np.float32)[None]
    P1 = (I1 * 255.0).astype(np.float32)[None]
    pitch = W + 9
    a, b = to_dev(torch, P0, dev, pitch), to_dev(torch, P1, dev, pitch)
    g = np.random.default_rng(3)
    U0 = ndimage_smooth(g.normal(0, 2.0, (H, W, 2))).astype(np.float32) * 3.0
    results = []
    h = dis.dis_create(pitch, H, 1, 1)
    try:
        for mode in (1, 0, 2, 3):
            dis.dis_set_refine_fusion(h, mode)
            U = torch.from_numpy(U0).to(dev)
            dis.dis_refine_level_ex(h, a, b, W, H, pitch, 1, U, outer, inner, dof=1)
            torch.cuda.synchronize()
            results.append(host(U))
        with pytest.raises(dis.DisError):
            dis.dis_refine_level_ex(h, a, b, W, H, pitch, 1, U, outer, inner, dof=3)
    finally:
        dis.dis_destroy(h)
    for r in results[1:]:
        assert np.array_equal(r, results[0])
    got = results[0]
    assert np.array_equal(got[..., 1], U0[..., 1].astype(np.float64))
    ref = oracle.refine_level(P0.astype(np.float64), P1.astype(np.float64), U0.astype(np.float64), outer, inner, dof=1)
    err = float(np.abs(got - ref).max())
    print("refine stereo %s: %dx%d, max |dU| %.2e (moved by %.2e)" % (case, W, H, err, np.abs(ref - U0).max()))
    assert err <= STAGE_TOL


def run_batched(torch, dis, dev, pairs, p):
    """One autotuned batched call over `pairs` ((I0, I1) host arrays), then single-pair calls of
    the same pairs on the same handle (the same tuned forms); returns both lists of host flows
    and the tuned search variant."""
    W = max(a.shape[-1] for a, _ in pairs)
    H = max(a.shape[-2] for a, _ in pairs)
    C = 1 if pairs[0][0].ndim == 2 else 3
    h = dis.dis_create(W, H, len(pairs), C)
    try:
        dp = [(to_dev(torch, a, dev), to_dev(torch, b, dev)) for a, b in pairs]
        flows = [torch.full((a.shape[-2], a.shape[-1], 2), float("nan"), device=dev) for a, _ in pairs]
        items = [(x, y, a.shape[-1], a.shape[-2], a.shape[-1], f) for (x, y), (a, _), f in zip(dp, pairs, flows)]
        arr = dis.make_pairs(items)
        variant = dis.dis_autotune(h, arr, len(items), p)
        assert variant in dis.dis_search_mode_variants(p.patch_size)
        dis.dis_compute_flow_batched(h, arr, len(items), p)
        torch.cuda.synchronize()
        batched = [host(f) for f in flows]
        single = []
        for (x, y), (a, _) in zip(dp, pairs):
            f = torch.full((a.shape[-2], a.shape[-1], 2), float("nan"), device=dev)
            dis.dis_compute_flow(h, x, y, a.shape[-1], a.shape[-2], a.shape[-1], p, f)
            torch.cuda.synchronize()
            single.append(host(f))
        return batched, single, variant
    finally:
        dis.dis_destroy(h)


@pytest.mark.parametrize("preset", ["stereo_op3", "stereo_dense", "stereo_op1"])
def test_e2e_stereo(env, preset):
    torch, dis, dev = env
    p = dis.dis_default_params(preset)
    base = dis.dis_default_params(preset.replace("stereo_", ""))
    assert p.dof == 1 and p.grad_iters == base.grad_iters // 2
    pairs = [synth.workload_pair("stereo320x240", i) for i in range(3)]
    batched, single, variant = run_batched(torch, dis, dev, [(a, b) for a, b, _ in pairs], p)
    for k, (I0, I1, gt) in enumerate(pairs):
        got = batched[k]
        assert np.array_equal(got, single[k])
        assert (got[..., 1] == 0.0).all()
        if k == 0:
            check_e2e("stereo320x240-%s (width %d)" % (preset, variant), got,
                      oracle_e2e(I0, I1, oracle_params(p)), gt)


def test_differentiable_form_replays_stereo(env):
    """The differentiable form takes the stereo mode: its FP64 replay of the recorded increments
    reproduces the FP32 stereo flow to the end-to-end bar and keeps v at 0."""
    torch, dis, dev = env
    p = dis.dis_default_params("stereo_dense")
    I0, I1, _ = synth.workload_pair("stereo320x240", 0)
    n = dis.dis_levels(320, 240, p)[2]
    ws_bytes = dis.dis_backward_workspace_bytes(320, 240, p)
    h = dis.dis_create(320, 240, 1, 1)
    try:
        a, b = to_dev(torch, I0, dev), to_dev(torch, I1, dev)
        ws = torch.zeros(ws_bytes // 4 + 1, device=dev)
        rec = torch.zeros((n, 2), device=dev)
        f32 = torch.zeros((240, 320, 2), device=dev)
        dis.dis_compute_flow_ex(h, a, b, 320, 240, 320, p, None, None, rec, None, f32)
        flow = torch.zeros((240, 320, 2), device=dev)
        dis.dis_replay_flow(h, a, b, 320, 240, 320, p, None, rec, flow, ws, ws.numel() * 4)
        torch.cuda.synchronize()
    finally:
        dis.dis_destroy(h)
    d = (flow - f32).abs()
    assert float(d.mean()) <= 0.01 and float(torch.quantile(d.flatten(), 0.999)) <= 0.05
    assert float(flow[..., 1].abs().max()) == 0.0


@pytest.mark.parametrize("norm,hb", [("l1", 5.0), ("huber", 5.0), ("huber", 20.0)])
def test_e2e_robust_norms(env, norm, hb):
    torch, dis, dev = env
    p = dis.dis_default_params("medium", norm=norm, huber_b=hb)
    pairs = [synth.layered_pair(2100 + i, width=320, height=240, max_disp=12.8) for i in range(2)]
    batched, single, variant = run_batched(torch, dis, dev, [(a, b) for a, b, _ in pairs], p)
    for k in range(len(pairs)):
        assert np.array_equal(single[k], batched[k])
    I0, I1, gt = pairs[0]
    check_e2e("layered320x240-medium-%s-b%g (width %d)" % (norm, hb, variant), batched[0],
              oracle_e2e(I0, I1, oracle_params(p)), gt)
    # the L2 flow differs: the norm reached the search
    l2, _ = run_gpu(torch, dis, dev, I0, I1, dis.dis_default_params("medium"))
    assert not np.array_equal(l2, batched[0])


def test_e2e_stereo_robust_dense(env):
    """Stereo with the Huber norm on the dense stereo preset (every mode combined), RGB input."""
    torch, dis, dev = env
    I0, I1, gt = synth.layered_pair(5100, width=320, height=240, n_ellipses=8, max_disp=12.0, channels=3,
                                    horizontal=True)
    p = dis.dis_default_params("stereo_dense", channels=3, norm="huber")
    got, _ = run_gpu(torch, dis, dev, I0, I1, p)
    assert (got[..., 1] == 0.0).all()
    check_e2e("stereo-rgb320x240-dense-huber", got, oracle_e2e(I0, I1, oracle_params(p)), gt)


@pytest.mark.parametrize("W,H,kw", [
    (12, 12, dict(patch_size=12, coarsest_scale=0, dof=1)),
    (13, 9, dict(patch_size=8, stride_override=3, norm="l1")),
    (37, 29, dict(patch_size=5, overlap=0.6, grad_iters=0, norm="huber", huber_b=2.0, dof=1)),
    (67, 45, dict(patch_size=16, overlap=0.5, finest_scale=1, fb=1)),
    (100, 64, dict(patch_size=7, overlap=0.9, grad_iters=24, refine=0, fb=1, dof=1, term_eps=0.02)),
])
def test_e2e_edge_sizes_of_the_extensions(env, W, H, kw):
    """The extensions on degenerate and ragged sizes: a frame of one patch, a 13x9 frame, no
    iterations, a 16x16 patch with the final up-scaling and consistency, stride 1 without
    refinement with every extension at once."""
    torch, dis, dev = env
    I0, I1, gt = synth.layered_pair(18, width=W, height=H, n_ellipses=2, max_disp=2.0,
                                    horizontal=kw.get("dof", 2) == 1)
    p = dis.dis_default_params(**kw)
    a, b = to_dev(torch, I0, dev, W + 1), to_dev(torch, I1, dev, W + 1)
    f = torch.full((H, W, 2), float("nan"), device=dev)
    h = dis.dis_create(W, H, 2, 1)
    try:
        dis.dis_compute_flow(h, a, b, W, H, W + 1, p, f)
        torch.cuda.synchronize()
    finally:
        dis.dis_destroy(h)
    got = host(f)
    if p.dof == 1:
        assert (got[..., 1] == 0.0).all()
    q = oracle_params(p)
    ref, spread = oracle_e2e(I0, I1, q)
    if q.term_eps > 0:
        eps = q.term_eps
        for fct in (1.0 - 2e-3, 1.0 + 2e-3):
            q.term_eps = eps * fct
            spread = np.maximum(spread, np.abs(oracle.dis_flow(I0, I1, q) - ref).max(-1))
        q.term_eps = eps
    check_e2e("extensions edge %dx%d %s" % (W, H, kw), got, (ref, spread), max_unstable=0.05)
