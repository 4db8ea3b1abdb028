"""GPU-vs-oracle parity through the C ABI.

Per stage, each stage's input is produced on the GPU, widened to FP64 and fed to the oracle's
stage; the bar is max |du| <= 1e-3 px.  End to end the bar is mean |du| <= 0.01 px and
99.9th percentile <= 0.05 px.  Discrete decisions (outlier reset, flat patch) taken on
either side of the threshold by FP32 and FP64 are counted, checked to be borderline in FP64,
and excluded from the element-wise comparison.
"""
import numpy as np
import pytest

import oracle
from paper_1603_03590_gb300 import synth

pytestmark = pytest.mark.gpu

STAGE_TOL = 1e-3        # px, per stage on identical inputs
E2E_MEAN, E2E_P999 = 0.01, 0.05  # px, end to end
# End-to-end determination: the FP64 result is recomputed with I1 perturbed by PERTURB grey levels
# (0..255 scale); pixels that move by more than STABLE_TOL px are not determined at FP32
# resolution.  PERTURB is calibrated to the FP32 path's own error: on the search of a dense-preset
# level, a 1e-3 perturbation moves the FP64 patches by 2.9e-4 px at the 99th percentile, the size
# of the FP32 search's largest per-stage deviation (3e-4 px), while 1e-4 moves them ten times
# less.  STABLE_TOL stays below the 99.9th-percentile bar.
PERTURB, STABLE_TOL = 1e-3, 0.03


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_03590_gb300 import build
    build.build()
    from paper_1603_03590_gb300 import dis
    return torch, dis, torch.device("cuda:0")


def to_dev(torch, a, dev, pitch=None):
    """(H, W) or (C, H, W) float array -> device tensor view with row pitch `pitch`."""
    a = np.asarray(a, dtype=np.float32)
    H, W = a.shape[-2:]
    pitch = W if pitch is None else pitch
    buf = torch.zeros(a.shape[:-1] + (pitch,), dtype=torch.float32, device=dev)
    buf[..., :W] = torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return buf


def host(t, W=None):
    a = t.detach().cpu().numpy().astype(np.float64)
    return a if W is None else a[..., :W]


def gpu_level_images(torch, dis, dev, I0, I1, levels, scale=255.0):
    """Scaled level-0 images and `levels` GPU pyramid steps (pitched), as device tensors."""
    out = []
    a, b = to_dev(torch, I0 * scale, dev, pitch=I0.shape[1] + 7), to_dev(torch, I1 * scale, dev, pitch=I0.shape[1] + 7)
    H, W = I0.shape
    out.append((a, b, W, H, a.shape[-1]))
    for _ in range(levels):
        w2, h2 = (W + 1) // 2, (H + 1) // 2
        pa = torch.zeros((h2, w2 + 3), device=dev)
        pb = torch.zeros((h2, w2 + 3), device=dev)
        dis.dis_pyr_down(a, W, H, a.shape[-1], pa, pa.shape[-1])
        dis.dis_pyr_down(b, W, H, b.shape[-1], pb, pb.shape[-1])
        a, b, W, H = pa, pb, w2, h2
        out.append((a, b, W, H, a.shape[-1]))
    return out


# ------------------------------------------------------------------------------ stages
@pytest.mark.parametrize("H,W", [(96, 128), (91, 173), (436, 1024), (5, 3)])
def test_pyr_down_and_sobel(env, H, W):
    torch, dis, dev = env
    g = np.random.default_rng(H * 1000 + W)
    img = g.uniform(0, 255, (H, W))
    a = to_dev(torch, img, dev, pitch=W + 5)
    w2, h2 = (W + 1) // 2, (H + 1) // 2
    out = torch.full((h2, w2 + 2), -1.0, device=dev)
    dis.dis_pyr_down(a, W, H, W + 5, out, w2 + 2)
    gx = torch.full((H, W + 1), -1.0, device=dev)
    gy = torch.full((H, W + 1), -1.0, device=dev)
    dis.dis_sobel(a, W, H, W + 5, gx, gy, W + 1)
    torch.cuda.synchronize()
    img32 = host(a, W)
    np.testing.assert_allclose(host(out, w2), oracle.pyr_down(img32), rtol=0, atol=2e-4)
    assert (host(out)[:, w2:] == -1.0).all()  # padding untouched
    ox, oy = oracle.sobel(img32)
    np.testing.assert_allclose(host(gx, W), ox, rtol=0, atol=2e-4)
    np.testing.assert_allclose(host(gy, W), oy, rtol=0, atol=2e-4)


def _flat_borderline(I0, ps, stride, idx, dof=2):
    """FP64 det / (tr/2)^2 of the Hessian of patch idx (dof 1: h00 / (tr/2)), for flat-decision
    checks."""
    gx, gy = oracle.sobel(I0)
    h, w = I0.shape
    nx = oracle.grid_n(w, ps, stride)
    j, i = divmod(idx, nx)
    px, py = oracle.grid_pos(i, w, ps, stride), oracle.grid_pos(j, h, ps, stride)
    X, Y = gx[py:py + ps, px:px + ps], gy[py:py + ps, px:px + ps]
    h00, h01, h11 = (X * X).sum(), (X * Y).sum(), (Y * Y).sum()
    if dof == 1:
        return h00 / (0.5 * (h00 + h11))
    return (h00 * h11 - h01 * h01) / (0.5 * (h00 + h11)) ** 2


def compare_search(I0, I1, Uc, cscale, ps, stride, iters, u_g, ui_g, st_g, ref=None, mode=None, max_unstable=0.02):
    """Element-wise comparison of GPU and FP64 patch flows.

    A patch whose FP64 result moves by more than 1e-4 px when I1 is perturbed by 1e-5 (the
    size of FP32 rounding on the 0..255 scale) is not determined by its inputs at FP32
    resolution (a search that cycles instead of converging); such patches are counted,
    checked for validity and excluded.  Among the others a differing reset / flat decision
    must be borderline in FP64.  `ref`: the oracle results of an earlier call on the same
    inputs (returned as the third value).  `mode`: dict of the oracle's dof / norm / huber_b."""
    mode = mode or {}
    if ref is None:
        gx, gy = oracle.sobel(I0)
        u_o, ui_o, st_o = oracle.search_level(I0, gx, gy, I1, ps, stride, iters, Uc=Uc, cscale=cscale, **mode)
        u_o, ui_o, st_o = u_o.reshape(-1, 2), ui_o.reshape(-1, 2), st_o.reshape(-1)
        unstable = np.zeros(len(st_o), bool)
        for seed in (1, 2):
            I1p = I1 + 1e-5 * np.random.default_rng(seed).standard_normal(I1.shape)
            u_p, _, st_p = oracle.search_level(I0, gx, gy, I1p, ps, stride, iters, Uc=Uc, cscale=cscale, **mode)
            unstable |= (np.abs(u_p.reshape(-1, 2) - u_o).max(1) > 1e-4) | (st_p.reshape(-1) != st_o)
        if mode.get("term_eps", 0.0) > 0.0:
            # early termination is a threshold decision on a step length: patches whose result
            # changes when the threshold moves by 0.2 % (far more than FP32 moves a step) stop at
            # an iteration that FP32 does not determine
            for f in (1.0 - 2e-3, 1.0 + 2e-3):
                m2 = dict(mode, term_eps=mode["term_eps"] * f)
                u_p, _, st_p = oracle.search_level(I0, gx, gy, I1, ps, stride, iters, Uc=Uc, cscale=cscale, **m2)
                unstable |= (np.abs(u_p.reshape(-1, 2) - u_o).max(1) > 1e-4) | (st_p.reshape(-1) != st_o)
        ref = (u_o, ui_o, st_o, unstable)
    u_o, ui_o, st_o, unstable = ref
    assert np.abs(ui_g - ui_o).max() <= 1e-4
    assert unstable.mean() < max_unstable, unstable.mean()
    assert np.isfinite(u_g).all()
    # a result of an unstable patch is still a valid outcome: within theta_ps of u_init
    assert (np.hypot(*(u_g - ui_g)[unstable].T) <= ps + 1e-3).all()
    differ = np.nonzero((st_g != st_o) & ~unstable)[0]
    for k in differ:
        if 2 in (st_g[k], st_o[k]):
            r = _flat_borderline(I0, ps, stride, k, mode.get("dof", 2))
            assert abs(r - 1e-6) < 1e-7, ("flat decision not borderline", k, r)
        else:
            # one side reset, the other did not: the non-resetting side's distance from
            # u_init must sit at theta_ps
            uu, base = (u_g[k], ui_g[k]) if st_g[k] == 0 else (u_o[k], ui_o[k])
            dist = float(np.hypot(*(uu - base)))
            assert abs(dist - ps) < 1e-2, ("reset decision not borderline", k, dist)
    same = (st_g == st_o) & ~unstable
    err = np.abs(u_g - u_o)[same]
    return err.max() if err.size else 0.0, "%d decisions differ, %d unstable" % (len(differ), unstable.sum()), ref


@pytest.mark.parametrize("case", ["translate", "layered-dense", "layered-fast", "ragged"])
def test_search_stage(env, case):
    """Per-stage search of every variant against the FP64 oracle on the same level inputs."""
    torch, dis, dev = env
    if case == "translate":
        I0, I1, _ = synth.translation_pair(0)
        lv, ps, stride, iters = 0, 8, 4, 16
    elif case == "ragged":
        I0, I1, _ = synth.layered_pair(11, width=173, height=91, max_disp=6.0)
        lv, ps, stride, iters = 0, 9, 4, 40
    else:
        I0, I1, _ = synth.layered_pair(1000)
        lv, ps, stride, iters = (2, 12, 3, 128) if case == "layered-dense" else (2, 8, 6, 16)
    a, b, W, H, pitch = gpu_level_images(torch, dis, dev, I0, I1, lv)[lv]
    g = np.random.default_rng(5)
    wc, hc = (W + 1) // 2, (H + 1) // 2
    Uc_h = (ndimage_smooth(g.normal(0, 1.5, (hc, wc, 2))) * 1.0).astype(np.float32)
    Uc = torch.from_numpy(Uc_h).to(dev)
    nx, ny = oracle.grid_n(W, ps, stride), oracle.grid_n(H, ps, stride)
    ref = None
    for variant in [0] + dis.dis_search_variants(ps):
        u = torch.zeros((ny * nx, 2), device=dev)
        ui = torch.zeros((ny * nx, 2), device=dev)
        st = torch.zeros(ny * nx, dtype=torch.int32, device=dev)
        dis.dis_search_level_ex(a, b, W, H, pitch, Uc, wc, hc, 2.0, ps, stride, iters, variant, u, ui, st)
        torch.cuda.synchronize()
        e, ndiff, ref = compare_search(host(a, W), host(b, W), Uc_h.astype(np.float64), 2.0, ps, stride, iters,
                                       host(u), host(ui), st.cpu().numpy(), ref)
        print("search %s variant %d: %d patches, max |du| %.2e, %s" % (case, variant, nx * ny, e, ndiff))
        assert e <= STAGE_TOL
    with pytest.raises(dis.DisError):
        dis.dis_search_level_ex(a, b, W, H, pitch, Uc, wc, hc, 2.0, ps, stride, iters, 3, u, ui, st)


def ndimage_smooth(a):
    from scipy import ndimage
    return np.stack([ndimage.gaussian_filter(a[..., k], 3.0) for k in range(a.shape[-1])], -1)


@pytest.mark.parametrize("case", ["translate", "layered-dense"])
def test_densify_stage(env, case):
    torch, dis, dev = env
    if case == "translate":
        I0, I1, _ = synth.translation_pair(1)
        lv, ps, stride, iters = 0, 8, 4, 16
    else:
        I0, I1, _ = synth.layered_pair(1001)
        lv, ps, stride, iters = 1, 12, 3, 64
    a, b, W, H, pitch = gpu_level_images(torch, dis, dev, I0, I1, lv)[lv]
    nx, ny = oracle.grid_n(W, ps, stride), oracle.grid_n(H, ps, stride)
    u = torch.zeros((ny * nx, 2), device=dev)
    dis.dis_search_level(a, b, W, H, pitch, None, 0, 0, 2.0, ps, stride, iters, u)
    U = torch.zeros((H, W, 2), device=dev)
    dis.dis_densify_level(a, b, W, H, pitch, u, ps, stride, None, 0, 0, 2.0, U)
    torch.cuda.synchronize()
    Uo = oracle.densify_level(host(a, W), host(b, W), host(u), ps, stride)
    e = np.abs(host(U) - Uo).max()
    print("densify %s: max |dU| %.2e" % (case, e))
    assert e <= STAGE_TOL


@pytest.mark.parametrize("case", ["translate", "layered", "rgb", "ragged", "ragged-fused", "tiny"])
def test_refine_stage(env, case):
    """Refinement of one level against the FP64 oracle; the fused form (one launch per outer
    pass, up to 5 inner sweeps) and the per-sweep form agree bit for bit."""
    torch, dis, dev = env
    outer, inner = 2, 5
    if case == "translate":
        I0, I1, _ = synth.translation_pair(2)
        lv = 0
    elif case == "ragged":
        I0, I1, _ = synth.layered_pair(12, width=173, height=91, max_disp=6.0)
        lv, outer, inner = 0, 3, 7
    elif case == "ragged-fused":
        I0, I1, _ = synth.layered_pair(14, width=173, height=91, max_disp=6.0)
        lv, outer, inner = 0, 3, 4
    elif case == "tiny":
        I0, I1, _ = synth.layered_pair(15, width=13, height=9, max_disp=1.0, n_ellipses=1)
        lv, outer, inner = 0, 2, 5
    elif case == "rgb":
        I0, I1, _ = synth.layered_pair(13, width=160, height=120, max_disp=8.0, channels=3)
        lv = 0
    else:
        I0, I1, _ = synth.layered_pair(1002)
        lv, outer = 1, 2
    C = 1 if I0.ndim == 2 else 3
    H, W = I0.shape[-2:]
    Hl, Wl = H, W
    for _ in range(lv):
        Wl, Hl = (Wl + 1) // 2, (Hl + 1) // 2
    # level images built by the oracle's pyramid (inputs only; FP32 on both sides)
    P0, P1 = [], []
    for c in range(C):
        x0 = (I0 if C == 1 else I0[c]) * 255.0
        x1 = (I1 if C == 1 else I1[c]) * 255.0
        for _ in range(lv):
            x0, x1 = oracle.pyr_down(x0), oracle.pyr_down(x1)
        P0.append(x0)
        P1.append(x1)
    P0 = np.stack(P0).astype(np.float32)
    P1 = np.stack(P1).astype(np.float32)
    pitch = Wl + 9
    a, b = to_dev(torch, P0, dev, pitch), to_dev(torch, P1, dev, pitch)
    g = np.random.default_rng(3)
    U0 = ndimage_smooth(g.normal(0, 2.0, (Hl, Wl, 2))).astype(np.float32) * 3.0
    U = torch.from_numpy(U0).to(dev)
    U2 = U.clone()
    h = dis.dis_create(pitch, Hl, 1, C)
    try:
        dis.dis_refine_level(h, a, b, Wl, Hl, pitch, C, U, outer, inner)
        others = []
        for mode in (0, 3):
            dis.dis_set_refine_fusion(h, mode)
            Uk = U2.clone()
            dis.dis_refine_level(h, a, b, Wl, Hl, pitch, C, Uk, outer, inner)
            others.append(Uk)
        torch.cuda.synchronize()
    finally:
        dis.dis_destroy(h)
    for Uk in others:
        assert torch.equal(U, Uk), float((U - Uk).abs().max())
    Uo = oracle.refine_level(P0.astype(np.float64), P1.astype(np.float64), U0.astype(np.float64), outer, inner)
    e = np.abs(host(U) - Uo).max()
    print("refine %s: max |dU| %.2e (update magnitude %.2e)" % (case, e, np.abs(Uo - U0).max()))
    assert e <= STAGE_TOL


@pytest.mark.parametrize("factor,src,dst", [(2.0, (55, 128), (109, 256)), (4.0, (28, 64), (109, 256)),
                                            (1.0, (17, 13), (17, 13))])
def test_upsample_stage(env, factor, src, dst):
    torch, dis, dev = env
    g = np.random.default_rng(9)
    Uin = g.normal(0, 3, src + (2,)).astype(np.float32)
    out = torch.zeros(dst + (2,), device=dev)
    dis.dis_upsample_flow(torch.from_numpy(Uin).to(dev), src[1], src[0], factor, out, dst[1], dst[0])
    torch.cuda.synchronize()
    ref = oracle.upsample_flow(Uin.astype(np.float64), factor, dst)
    assert np.abs(host(out) - ref).max() <= 1e-4


# ------------------------------------------------------------------------------ end to end
def run_gpu(torch, dis, dev, I0, I1, params, pitch_pad=0, init=None, frozen=None, record=False):
    C = 1 if I0.ndim == 2 else 3
    H, W = I0.shape[-2:]
    pitch = W + pitch_pad
    a, b = to_dev(torch, I0, dev, pitch), to_dev(torch, I1, dev, pitch)
    flow = torch.full((H, W, 2), float("nan"), device=dev)
    h = dis.dis_create(W, H, 1, C)
    try:
        rec = None
        if init is None and frozen is None and not record:
            dis.dis_compute_flow(h, a, b, W, H, pitch, params, flow)
        else:
            n = dis.dis_levels(W, H, params)[2]
            rec = torch.zeros((n, 2), device=dev) if record else None
            it = None if init is None else torch.from_numpy(np.asarray(init, np.float32)).to(dev)
            fz = None if frozen is None else torch.from_numpy(np.asarray(frozen, np.float32)).to(dev)
            dis.dis_compute_flow_ex(h, a, b, W, H, pitch, params, it, fz, rec, None, flow)
        torch.cuda.synchronize()
    finally:
        dis.dis_destroy(h)
    return host(flow), (None if rec is None else host(rec))


def oracle_params(p):
    return oracle.params(patch_size=p.patch_size, overlap=round(float(p.overlap), 6), stride_override=p.stride_override,
                         grad_iters=p.grad_iters, coarsest_scale=p.coarsest_scale, finest_scale=p.finest_scale,
                         refine=p.refine, var_outer=p.var_outer, var_inner=p.var_inner, delta=p.delta,
                         gamma=p.gamma, alpha=p.alpha, sor_omega=round(float(p.sor_omega), 6),
                         intensity_scale=p.intensity_scale, channels=p.channels, dof=p.dof, norm=p.norm,
                         huber_b=round(float(p.huber_b), 6), fb=p.fb, term_eps=float(p.term_eps))


def _oracle_run(args):
    """One FP64 oracle run (in a spawned process); I1 perturbed by PERTURB on the 0..255 scale
    with the given seed (None: unperturbed)."""
    I0, I1, fields, seed, kw = args
    if seed is not None:
        I1 = I1.astype(np.float64) + np.random.default_rng(seed).standard_normal(I1.shape) * (PERTURB / 255.0)
    return oracle.dis_flow(I0, I1, oracle.params(**fields), **kw)


def oracle_fields(q):
    """The oracle's parameter structure as plain keyword values (picklable)."""
    return {name: getattr(q, name) for name, _ in q._fields_}


def oracle_e2e_many(cases, replicas=2):
    """(flow, spread) of oracle_e2e for every (I0, I1, oracle params, keyword arguments) case; all
    oracle runs side by side in spawned processes."""
    import multiprocessing as mp
    import os
    tasks = [(I0, I1, oracle_fields(q), seed, kw) for I0, I1, q, kw in cases
             for seed in [None] + list(range(1, replicas + 1))]
    with mp.get_context("spawn").Pool(min(len(tasks), os.cpu_count() or 1)) as pool:
        res = pool.map(_oracle_run, tasks, chunksize=1)
    out = []
    for c in range(len(cases)):
        ref = res[(replicas + 1) * c]
        reps = res[(replicas + 1) * c + 1:(replicas + 1) * (c + 1)]
        out.append((ref, np.max([np.abs(f - ref).max(-1) for f in reps], axis=0)))
    return out


def oracle_e2e(I0, I1, q, replicas=2, **kw):
    """FP64 flow and its own spread: the largest change of the FP64 result under `replicas`
    perturbations of I1 by PERTURB on the 0..255 scale (a perturbation whose effect on the
    search matches the FP32 path's own rounding error).  Pixels whose FP64 result moves by more
    than STABLE_TOL under such a perturbation are not determined by the inputs at FP32
    resolution (patch searches that cycle instead of converging, outlier resets at their
    threshold, ill-conditioned refinement); no FP32 implementation can be held to them."""
    return oracle_e2e_many([(I0, I1, q, kw)], replicas)[0]


def check_e2e(name, got, ref_spread, gt=None, max_unstable=0.03):
    ref, spread = ref_spread
    stable = spread <= STABLE_TOL
    d_all = np.abs(got - ref)
    d = d_all[stable]
    mean, p999 = d.mean(), np.quantile(d, 0.999)
    msg = ("%s: stable pixels %.2f%%  mean |du| %.2e  p99.9 %.2e | all pixels: mean %.2e p99.9 %.2e "
           "(FP64 self-spread p99.9 %.2e)" % (name, 100 * stable.mean(), mean, p999, d_all.mean(),
                                             np.quantile(d_all, 0.999), np.quantile(spread, 0.999)))
    if gt is not None:
        msg += "  EPE gpu %.3f oracle %.3f" % (np.linalg.norm(got - gt, axis=-1).mean(),
                                              np.linalg.norm(ref - gt, axis=-1).mean())
    print(msg)
    assert np.isfinite(got).all()
    assert 1.0 - stable.mean() <= max_unstable, msg
    assert mean <= E2E_MEAN and p999 <= E2E_P999, msg


def test_e2e_translation_128x96(env):
    torch, dis, dev = env
    I0, I1, gt = synth.translation_pair(0)
    p = dis.dis_default_params(patch_size=8, stride_override=4, grad_iters=16, coarsest_scale=2, var_outer=1)
    got, _ = run_gpu(torch, dis, dev, I0, I1, p, pitch_pad=3)
    check_e2e("translate128x96", got, oracle_e2e(I0, I1, oracle_params(p)), gt)


@pytest.mark.parametrize("preset", ["fast", "dense", "op2", "medium"])
def test_e2e_layered_1024x436(env, preset):
    torch, dis, dev = env
    I0, I1, gt = synth.layered_pair(1000)
    p = dis.dis_default_params(preset, coarsest_scale=4 if preset in ("fast", "dense") else -1)
    got, _ = run_gpu(torch, dis, dev, I0, I1, p)
    check_e2e("layered1024x436-" + preset, got, oracle_e2e(I0, I1, oracle_params(p)), gt)


@pytest.mark.parametrize("W,H,kw", [(12, 12, dict(patch_size=12, coarsest_scale=0)),
                                    (13, 9, dict(patch_size=8, stride_override=3)),
                                    (37, 29, dict(patch_size=5, overlap=0.6, grad_iters=0)),
                                    (67, 45, dict(patch_size=16, overlap=0.5, finest_scale=1)),
                                    (100, 64, dict(patch_size=7, overlap=0.9, grad_iters=24, refine=0))])
def test_e2e_edge_sizes(env, W, H, kw):
    torch, dis, dev = env
    I0, I1, gt = synth.layered_pair(17, width=W, height=H, n_ellipses=2, max_disp=2.0)
    p = dis.dis_default_params(**kw)
    got, _ = run_gpu(torch, dis, dev, I0, I1, p, pitch_pad=1)
    check_e2e("edge %dx%d" % (W, H), got, oracle_e2e(I0, I1, oracle_params(p)))


@pytest.mark.parametrize("preset,C", [("medium", 1), ("dense", 3)])
def test_e2e_fused_refinement_equals_per_sweep_bit_exact(env, preset, C):
    """Whole pipeline, batched over uneven sizes: fused and per-sweep refinement give the same
    flows bit for bit, and so does form 1 with a split threshold between the level sizes."""
    torch, dis, dev = env
    sizes = [(173, 91), (320, 240), (64, 48)]
    pairs = [synth.layered_pair(80 + k, width=w, height=h, n_ellipses=4, max_disp=0.04 * w, channels=C)
             for k, (w, h) in enumerate(sizes)]
    p = dis.dis_default_params(preset, channels=C, grad_iters=16)
    h = dis.dis_create(320, 240, len(pairs), C)
    try:
        dev_pairs = [(to_dev(torch, a, dev, a.shape[-1] + 5), to_dev(torch, b, dev, b.shape[-1] + 5)) for a, b, _ in pairs]
        out = []
        for fused, split in ((1, -1), (0, -1), (2, -1), (3, -1), (1, 20000)):
            dis.dis_set_refine_fusion(h, fused)
            dis.dis_set_refine_split(h, split)  # (1, 20000): the levels above 20000 pixels split
            assert dis.dis_get_refine_split(h) == split
            flows = [torch.full((a.shape[-2], a.shape[-1], 2), float("nan"), device=dev) for a, _, _ in pairs]
            items = [(da, db, a.shape[-1], a.shape[-2], da.shape[-1], f)
                     for (da, db), (a, _, _), f in zip(dev_pairs, pairs, flows)]
            dis.dis_compute_flow_batched(h, dis.make_pairs(items), len(items), p)
            torch.cuda.synchronize()
            out.append([host(f) for f in flows])
        with pytest.raises(dis.DisError):
            dis.dis_set_refine_fusion(h, 4)
    finally:
        dis.dis_destroy(h)
    for k in range(len(pairs)):
        assert np.isfinite(out[0][k]).all()
        assert all(np.array_equal(out[0][k], o[k]) for o in out[1:]), (preset, sizes[k])


def test_search_work_queue_equals_grid_stride_bit_exact(env):
    """Patch scheduling: the work queue (default) and the fixed grid stride give the same flows
    bit for bit, over a batch of uneven sizes, in repeated calls (graph replays) and after calls
    with a different number of patches (another grid size): the queue starts every launch from
    zero."""
    torch, dis, dev = env
    sizes = [(173, 91), (320, 240), (64, 48)]
    pairs = [synth.layered_pair(90 + k, width=w, height=h, n_ellipses=4, max_disp=0.04 * w) for k, (w, h) in enumerate(sizes)]
    p = dis.dis_default_params("dense", grad_iters=32)
    h = dis.dis_create(320, 240, len(pairs), 1)
    try:
        dev_pairs = [(to_dev(torch, a, dev), to_dev(torch, b, dev)) for a, b, _ in pairs]

        def run(subset):
            flows = [torch.full((pairs[k][0].shape[-2], pairs[k][0].shape[-1], 2), float("nan"), device=dev) for k in subset]
            items = [(dev_pairs[k][0], dev_pairs[k][1], pairs[k][0].shape[-1], pairs[k][0].shape[-2],
                      pairs[k][0].shape[-1], f) for k, f in zip(subset, flows)]
            dis.dis_compute_flow_batched(h, dis.make_pairs(items), len(items), p)
            torch.cuda.synchronize()
            return [host(f) for f in flows]

        every = list(range(len(pairs)))
        ref = run(every)                     # queue, first call (graph captured)
        again = run(every)                   # queue, graph replay
        small = run([2])                     # another grid in between
        after = run(every)
        dis.dis_set_work_queue(h, False)
        stride = run(every)                  # fixed grid stride
        small_stride = run([2])
        dis.dis_set_work_queue(h, True)
        back = run(every)
        assert dis._lib.dis_set_work_queue(h, 2) == dis.DIS_ERR_INVALID_ARG
    finally:
        dis.dis_destroy(h)
    for k in range(len(pairs)):
        assert np.isfinite(ref[k]).all()
        for o in (again, after, stride, back):
            assert np.array_equal(ref[k], o[k]), sizes[k]
    assert np.array_equal(small[0], ref[2]) and np.array_equal(small_stride[0], ref[2])


def test_e2e_rgb(env):
    torch, dis, dev = env
    I0, I1, gt = synth.layered_pair(4000, width=256, height=144, max_disp=10.0, channels=3, rotation_deg=2.0)
    p = dis.dis_default_params("dense", channels=3, grad_iters=32)
    got, _ = run_gpu(torch, dis, dev, I0, I1, p, pitch_pad=4)
    check_e2e("rgb256x144", got, oracle_e2e(I0, I1, oracle_params(p)), gt)


def test_too_small_is_refused(env):
    torch, dis, dev = env
    I0 = np.zeros((6, 6), np.float32)
    with pytest.raises(dis.DisError) as e:
        run_gpu(torch, dis, dev, I0, I0, dis.dis_default_params(patch_size=8))
    assert e.value.status == dis.DIS_ERR_TOO_SMALL


def test_record_replay_and_init_flow(env):
    torch, dis, dev = env
    I0, I1, gt = synth.layered_pair(3000, width=512, height=256, max_disp=20.0)
    p = dis.dis_default_params(patch_size=8, overlap=0.5, grad_iters=16, coarsest_scale=3, var_outer=1, var_inner=10)
    flow, rec = run_gpu(torch, dis, dev, I0, I1, p, record=True)
    again, _ = run_gpu(torch, dis, dev, I0, I1, p, frozen=rec)
    # replay adds the recorded increment back onto u_init in FP32: equal up to the rounding of
    # that sum, which the lagged refinement weights (Psi' peaks at the eps of Sec. 2.3) can
    # amplify at a few pixels; held to the end-to-end bar
    d = np.abs(flow - again)
    assert d.mean() <= E2E_MEAN and np.quantile(d, 0.999) <= E2E_P999, (d.mean(), np.quantile(d, 0.999))
    q = oracle_params(p)
    ref_frozen = oracle.dis_flow(I0, I1, q, frozen=rec)
    check_e2e("frozen replay", again, (ref_frozen, np.zeros(ref_frozen.shape[:2])))
    # an initial flow at the coarsest level's resolution (64 x 32 at theta_ss = 3)
    g = np.random.default_rng(1)
    init = ndimage_smooth(g.normal(0, 1.0, (32, 64, 2)))
    got, _ = run_gpu(torch, dis, dev, I0, I1, p, init=init)
    check_e2e("init flow", got, oracle_e2e(I0, I1, q, init_flow=init.astype(np.float32)))


def test_batched_matches_plain_bit_exact(env):
    torch, dis, dev = env
    sizes = [(128, 96), (173, 91), (320, 240), (64, 48), (256, 109)]
    pairs = [synth.layered_pair(50 + k, width=w, height=h, n_ellipses=4, max_disp=0.04 * w) for k, (w, h) in
             enumerate(sizes)]
    for preset in ["medium", "fast"]:
        p = dis.dis_default_params(preset)
        plain = [run_gpu(torch, dis, dev, a, b, p)[0] for a, b, _ in pairs]
        h = dis.dis_create(320, 240, len(pairs), 1)
        try:
            dev_pairs = [(to_dev(torch, a, dev), to_dev(torch, b, dev)) for a, b, _ in pairs]
            flows = [torch.full((a.shape[0], a.shape[1], 2), float("nan"), device=dev) for a, _, _ in pairs]
            items = [(da, db, da.shape[1], da.shape[0], da.shape[1], f) for (da, db), f in zip(dev_pairs, flows)]
            arr = dis.make_pairs(items)
            for _ in range(2):  # second call replays the cached graph
                dis.dis_compute_flow_batched(h, arr, len(items), p)
            torch.cuda.synchronize()
        finally:
            dis.dis_destroy(h)
        for k, f in enumerate(flows):
            assert np.array_equal(host(f), plain[k]), (preset, sizes[k])


def test_host_buffer_calls_match_device_calls(env):
    """dis_compute_flow_batched_host on host frames (pinned and pageable) gives the flows of the
    device call bit for bit, over consecutive calls that alternate the staging halves."""
    torch, dis, dev = env
    sizes = [(173, 91), (320, 240), (64, 48)]
    sets = [[synth.layered_pair(90 + 10 * r + k, width=w, height=h, n_ellipses=4, max_disp=0.04 * w)
             for k, (w, h) in enumerate(sizes)] for r in range(3)]
    p = dis.dis_default_params("medium")
    h = dis.dis_create(320, 240, len(sizes), 1)
    try:
        want = []
        for pairs in sets:
            flows = [torch.zeros((a.shape[0], a.shape[1], 2), device=dev) for a, _, _ in pairs]
            items = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev), a.shape[1], a.shape[0], a.shape[1], f)
                     for (a, b, _), f in zip(pairs, flows)]
            dis.dis_compute_flow_batched(h, dis.make_pairs(items), len(items), p)
            torch.cuda.synchronize()
            want.append([host(f) for f in flows])
        keep, outs = [], []
        for r, pairs in enumerate(sets):
            pin = r != 1  # the middle call uses pageable memory
            fr = [(torch.from_numpy(a), torch.from_numpy(b)) for a, b, _ in pairs]
            if pin:
                fr = [(a.pin_memory(), b.pin_memory()) for a, b in fr]
            out = [torch.full((a.shape[0], a.shape[1], 2), float("nan"), pin_memory=pin) for a, _, _ in pairs]
            arr = dis.make_pairs([(a, b, a.shape[1], a.shape[0], a.shape[1], f) for (a, b), f in zip(fr, out)])
            dis.dis_compute_flow_batched_host(h, arr, len(pairs), p)
            keep.append((fr, arr))
            outs.append(out)
        dis.dis_host_flows_ready(h)
        torch.cuda.synchronize()
        for r in range(len(sets)):
            for k in range(len(sizes)):
                assert np.array_equal(outs[r][k].numpy().astype(np.float64), want[r][k]), (r, k)
    finally:
        dis.dis_destroy(h)


def test_trace_and_probe(env):
    """dis_trace_batched lists the plan's launch groups with device times and gives the same
    flows as a normal call; the probe times one group inside the replayed graph."""
    torch, dis, dev = env
    pairs = [synth.layered_pair(70 + k, width=320, height=240, n_ellipses=4, max_disp=10.0) for k in range(2)]
    p = dis.dis_default_params("medium")
    h = dis.dis_create(320, 240, len(pairs), 1)
    try:
        dev_pairs = [(to_dev(torch, a, dev), to_dev(torch, b, dev)) for a, b, _ in pairs]
        flows = [torch.zeros((240, 320, 2), device=dev) for _ in pairs]
        arr = dis.make_pairs([(a, b, 320, 240, 320, f) for (a, b), f in zip(dev_pairs, flows)])
        recs = dis.dis_trace_batched(h, arr, len(pairs), p)
        traced = [host(f) for f in flows]
        ss, sf, _ = dis.dis_levels(320, 240, p)
        kinds = [r[0] for r in recs]
        print("trace:", ["%s%d %.3f" % r for r in recs])
        assert kinds[0] == "prep" and kinds.count("pyramid") == ss
        assert kinds.count("search") == kinds.count("densify") == kinds.count("refine") == ss - sf + 1
        assert all(ms > 0 for _, _, ms in recs)
        dis.dis_set_probe(h, "search", sf)
        with pytest.raises(dis.DisError):
            dis.dis_probe_ms(h)
        for _ in range(2):  # the second call replays the cached graph, with the probe's events
            dis.dis_compute_flow_batched(h, arr, len(pairs), p)
        ms = dis.dis_probe_ms(h)
        torch.cuda.synchronize()
        assert ms > 0
        for k, f in enumerate(flows):
            assert np.array_equal(host(f), traced[k])
        dis.dis_set_probe(h, -1)
        with pytest.raises(dis.DisError):
            dis.dis_probe_ms(h)
    finally:
        dis.dis_destroy(h)


@pytest.mark.parametrize("preset", ["fast", "dense"])
def test_pipeline_search_equals_per_stage_search_bit_exact(env, preset):
    """For every search variant, the pipeline's search (batched job tables; the lane-per-patch
    variant reading the per-pixel search planes) and the per-stage entry point (one job; that
    variant reading the images) give the same patch increments bit for bit at every level.
    Refinement is off so that the checkpoint of level s+1 is the flow the search of level s
    starts from."""
    torch, dis, dev = env
    I0, I1, _ = synth.layered_pair(1001)
    W, H = 1024, 436
    p = dis.dis_default_params(preset, coarsest_scale=4, refine=0)
    ss, sf, ntot = dis.dis_levels(W, H, p)
    ps = p.patch_size
    stride = p.stride_override or max(1, ps - int(np.floor(p.overlap * ps + 1e-4)))
    dims = [(W, H)]
    for _ in range(ss):
        dims.append(((dims[-1][0] + 1) // 2, (dims[-1][1] + 1) // 2))
    a, b = to_dev(torch, I0, dev), to_dev(torch, I1, dev)
    lv = gpu_level_images(torch, dis, dev, I0, I1, ss, scale=p.intensity_scale)
    h = dis.dis_create(W, H, 1, 1)
    try:
        for variant in dis.dis_search_variants(ps):
            dis.dis_set_search_variant(h, ps, variant)
            ck = torch.zeros(sum(dims[s][0] * dims[s][1] for s in range(sf, ss + 1)) * 2, device=dev)
            rec = torch.zeros((ntot, 2), device=dev)
            flow = torch.zeros((H, W, 2), device=dev)
            dis.dis_compute_flow_ex(h, a, b, W, H, W, p, None, None, rec, ck, flow)
            off_r = off_c = 0
            prev = None
            for s in range(ss, sf - 1, -1):
                A, B, w, hh, pitch = lv[s]
                n = oracle.grid_n(w, ps, stride) * oracle.grid_n(hh, ps, stride)
                u = torch.zeros((n, 2), device=dev)
                ui = torch.zeros((n, 2), device=dev)
                Uc, wc, hc, cs = (None, w, hh, 1.0) if prev is None else prev + (2.0,)
                dis.dis_search_level_ex(A, B, w, hh, pitch, Uc, wc, hc, cs, ps, stride, p.grad_iters, variant, u, ui)
                torch.cuda.synchronize()
                nd = int((u - ui != rec[off_r:off_r + n]).any(1).sum())
                print("variant %d level %d (%dx%d): %d patches, %d differ" % (variant, s, w, hh, n, nd))
                assert nd == 0
                off_r += n
                prev = (ck[off_c:off_c + w * hh * 2], w, hh)
                off_c += w * hh * 2
    finally:
        dis.dis_destroy(h)


@pytest.mark.parametrize("preset", ["fast", "dense"])
def test_every_search_variant_and_the_autotuner_keep_parity(env, preset):
    """Each search variant (one lane per patch, and the grouped forms) end to end against the
    FP64 oracle on the same pairs, then the variant the autotuner keeps."""
    torch, dis, dev = env
    pairs = [synth.layered_pair(60 + k, width=320, height=240, n_ellipses=6, max_disp=12.0) for k in range(2)]
    p = dis.dis_default_params(preset)
    refs = [oracle_e2e(a, b, oracle_params(p)) for a, b, _ in pairs]
    variants = dis.dis_search_variants(p.patch_size)
    assert 1 in variants and len(set(variants)) == len(variants) >= 2
    h = dis.dis_create(320, 240, len(pairs), 1)
    try:
        dev_pairs = [(to_dev(torch, a, dev), to_dev(torch, b, dev)) for a, b, _ in pairs]
        flows = [torch.zeros((240, 320, 2), device=dev) for _ in pairs]
        arr = dis.make_pairs([(a, b, 320, 240, 320, f) for (a, b), f in zip(dev_pairs, flows)])
        with pytest.raises(dis.DisError):
            dis.dis_set_search_variant(h, p.patch_size, 3)
        for lanes in variants:
            dis.dis_set_search_variant(h, p.patch_size, lanes)
            dis.dis_compute_flow_batched(h, arr, len(pairs), p)
            torch.cuda.synchronize()
            for k, f in enumerate(flows):
                check_e2e("%s lanes=%d pair %d" % (preset, lanes, k), host(f), refs[k])
        lanes = dis.dis_autotune(h, arr, len(pairs), p)
        assert lanes in variants
        tv, tr = dis.dis_get_tuning(h, p.patch_size)
        assert tv == lanes and tr in ((0, 1, 2, 3) if p.refine else (1,))
        print("%s: autotuned search variant %d, refinement launch form %d" % (preset, tv, tr))
        dis.dis_compute_flow_batched(h, arr, len(pairs), p)
        torch.cuda.synchronize()
        for k, f in enumerate(flows):
            check_e2e("%s autotuned lanes=%d pair %d" % (preset, lanes, k), host(f), refs[k])
    finally:
        dis.dis_destroy(h)
