"""Forward-backward consistency (supplementary Sec. B (ii)) on the GPU, against the FP64
oracle, through the C ABI.

- Densification stage (`dis_densify_level_fb`): both directions' merged fields from the GPU's
  own patch flows of both directions, and from random patch flows (integer and fractional
  moves, boxes leaving the frame, every backward patch piled onto one spot so that a tile
  lists more patches than one shared-memory chunk holds), max |dU| <= 1e-3 px against
  `oracle.densify_level_fb`; repeated calls agree bit for bit.
- End to end (`dis_compute_flow_fb`): forward and backward flows against the oracle within the
  end-to-end bar; a batch of uneven pairs with fb on equals the single-pair calls bit for bit.
- Refusals: too few pair slots, initial flows, the differentiable form.
"""
import numpy as np
import pytest

import oracle
from paper_1603_03590_gb300 import synth
from test_gpu_parity import (STAGE_TOL, check_e2e, gpu_level_images, host, oracle_e2e, oracle_e2e_many, oracle_params,
                             to_dev)

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


def run_densify_fb(torch, dis, dev, a, b, W, H, pitch, u, ub, ps, stride):
    h = dis.dis_create(pitch, H, 2, 1)
    try:
        U = torch.full((H, W, 2), float("nan"), device=dev)
        Ub = torch.full((H, W, 2), float("nan"), device=dev)
        out = []
        for _ in range(2):
            dis.dis_densify_level_fb(h, a, b, W, H, pitch, u, ub, ps, stride, U, Ub)
            torch.cuda.synchronize()
            out.append((host(U), host(Ub)))
    finally:
        dis.dis_destroy(h)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    return out[0]


def check_densify(name, A, B, u_h, ub_h, ps, stride, got_f, got_b):
    ref_f = oracle.densify_level_fb(A, B, u_h, ub_h, ps, stride)
    ref_b = oracle.densify_level_fb(B, A, ub_h, u_h, ps, stride)
    ef, eb = float(np.abs(got_f - ref_f).max()), float(np.abs(got_b - ref_b).max())
    print("densify fb %s: max |dU| forward %.2e backward %.2e" % (name, ef, eb))
    assert np.isfinite(got_f).all() and np.isfinite(got_b).all()
    assert ef <= STAGE_TOL and eb <= STAGE_TOL


@pytest.mark.parametrize("case", ["translate", "layered", "ragged"])
def test_densify_fb_stage_on_searched_patches(env, case):
    torch, dis, dev = env
    if case == "translate":
        I0, I1, _ = synth.translation_pair(3)
        lv, ps, stride, iters = 0, 8, 4, 16
    elif case == "ragged":
        I0, I1, _ = synth.layered_pair(16, width=173, height=91, max_disp=6.0)
        lv, ps, stride, iters = 0, 9, 4, 40
    else:
        I0, I1, _ = synth.layered_pair(1003)
        lv, ps, stride, iters = 1, 12, 3, 64
    a, b, W, H, pitch = gpu_level_images(torch, dis, dev, I0, I1, lv)[lv]
    nx, ny = oracle.grid_n(W, ps, stride), oracle.grid_n(H, ps, stride)
    u = torch.zeros((ny * nx, 2), device=dev)
    ub = torch.zeros((ny * nx, 2), device=dev)
    dis.dis_search_level(a, b, W, H, pitch, None, 0, 0, 2.0, ps, stride, iters, u)
    dis.dis_search_level(b, a, W, H, pitch, None, 0, 0, 2.0, ps, stride, iters, ub)
    torch.cuda.synchronize()
    got_f, got_b = run_densify_fb(torch, dis, dev, a, b, W, H, pitch, u, ub, ps, stride)
    check_densify(case, host(a, W), host(b, W), host(u), host(ub), ps, stride, got_f, got_b)


@pytest.mark.parametrize("case", ["random", "integer", "piled"])
def test_densify_fb_stage_on_random_patches(env, case):
    torch, dis, dev = env
    g = np.random.default_rng({"random": 51, "integer": 52, "piled": 53}[case])
    W, H, ps, stride = 97, 70, 8, 3
    A = (g.uniform(0, 1, (H, W)) * 255).astype(np.float32)
    B = (np.roll(A, 3, axis=1) + g.normal(0, 3, (H, W))).astype(np.float32)
    n = oracle.grid_n(W, ps, stride) * oracle.grid_n(H, ps, stride)
    u_h = g.uniform(-12, 12, (n, 2)).astype(np.float32)
    ub_h = g.uniform(-12, 12, (n, 2)).astype(np.float32)
    if case == "integer":
        ub_h = np.round(ub_h)
        u_h[::2] = np.round(u_h[::2])
    if case == "piled":
        # every backward patch lands on the same 8 x 8 box near (40, 30): one tile lists all
        # of them (more than one chunk of 256)
        nx = oracle.grid_n(W, ps, stride)
        k = np.arange(n)
        px = np.minimum((k % nx) * stride, W - ps)
        py = np.minimum((k // nx) * stride, H - ps)
        ub_h = np.stack([40.25 - px, 30.5 - py], -1).astype(np.float32)
        assert n > 256
    pitch = W + 3
    a, b = to_dev(torch, A, dev, pitch), to_dev(torch, B, dev, pitch)
    u = torch.from_numpy(u_h).to(dev)
    ub = torch.from_numpy(ub_h).to(dev)
    got_f, got_b = run_densify_fb(torch, dis, dev, a, b, W, H, pitch, u, ub, ps, stride)
    check_densify(case, A.astype(np.float64), B.astype(np.float64), u_h.astype(np.float64), ub_h.astype(np.float64),
                  ps, stride, got_f, got_b)


def fb_params(dis, preset, **kw):
    p = dis.dis_default_params(preset, **kw)
    p.fb = 1
    return p


@pytest.mark.parametrize("name,preset,kw", [
    ("translate128x96", "default", dict(patch_size=8, stride_override=4, grad_iters=16, coarsest_scale=2, var_outer=1)),
    ("layered320x240-medium", "medium", {}),
    ("layered320x240-dense", "dense", {}),
    ("layered192x144-dense-rgb", "dense", dict(channels=3, finest_scale=1)),
])
def test_e2e_fb(env, name, preset, kw):
    torch, dis, dev = env
    if name.startswith("translate"):
        I0, I1, gt = synth.translation_pair(0)
    elif name.startswith("layered192"):
        I0, I1, gt = synth.layered_pair(2201, width=192, height=144, n_ellipses=8, max_disp=8.0, channels=3)
    else:
        I0, I1, gt = synth.layered_pair(2200, width=320, height=240, max_disp=12.8)
    p = fb_params(dis, preset, **kw)
    C = 1 if I0.ndim == 2 else 3
    H, W = I0.shape[-2:]
    a, b = to_dev(torch, I0, dev, W + 5), to_dev(torch, I1, dev, W + 5)
    f = torch.full((H, W, 2), float("nan"), device=dev)
    fb_ = torch.full((H, W, 2), float("nan"), device=dev)
    h = dis.dis_create(W, H, 2, C)
    try:
        dis.dis_compute_flow_fb(h, a, b, W, H, W + 5, p, f, fb_)
        f2 = torch.full((H, W, 2), float("nan"), device=dev)
        dis.dis_compute_flow(h, a, b, W, H, W + 5, p, f2)  # p.fb = 1: the forward flow alone
        torch.cuda.synchronize()
    finally:
        dis.dis_destroy(h)
    got_f, got_b = host(f), host(fb_)
    assert np.array_equal(got_f, host(f2))
    q = oracle_params(p)
    q.fb = 1
    # The medium preset at 320x240 is ill-conditioned: under the perturbations of I1 of
    # test_gpu_parity.oracle_e2e the FP64 oracle's own flow moves by more than the stability
    # tolerance at several per cent of this pair's pixels, more with the consistency than
    # without it (the merged fields take in the other direction's outlier patches too); those
    # pixels are not determined at FP32 resolution, and four perturbations instead of two find
    # them.  The determined ones are held to the usual bar.
    cap, reps = (0.06, 4) if preset == "medium" else (0.03, 2)
    fwd, bwd = oracle_e2e_many([(I0, I1, q, {}), (I1, I0, q, {})], reps)
    check_e2e(name + " forward", got_f, fwd, gt, max_unstable=cap)
    check_e2e(name + " backward", got_b, bwd, max_unstable=cap)
    plain_q = oracle_params(p)
    plain_q.fb = 0
    assert np.abs(oracle.dis_flow(I0, I1, plain_q) - oracle.dis_flow(I0, I1, q)).max() > 1e-3


def test_batched_fb_equals_single_pair_calls(env):
    torch, dis, dev = env
    sizes = [(160, 120), (203, 97), (96, 64)]
    pairs = [synth.layered_pair(2300 + k, width=w, height=h, max_disp=0.04 * w) for k, (w, h) in enumerate(sizes)]
    p = fb_params(dis, "medium")
    Wm, Hm = max(s[0] for s in sizes), max(s[1] for s in sizes)
    h = dis.dis_create(Wm, Hm, 2 * len(pairs), 1)
    try:
        dp = [(to_dev(torch, a, dev), to_dev(torch, b, dev)) for a, b, _ in pairs]
        flows = [torch.full((hh, ww, 2), float("nan"), device=dev) for ww, hh in sizes]
        items = [(x, y, ww, hh, ww, f) for (x, y), (ww, hh), f in zip(dp, sizes, flows)]
        arr = dis.make_pairs(items)
        dis.dis_autotune(h, arr, len(items), p)
        runs = []
        for _ in range(2):
            dis.dis_compute_flow_batched(h, arr, len(items), p)
            torch.cuda.synchronize()
            runs.append([host(f) for f in flows])
        for k, ((x, y), (ww, hh)) in enumerate(zip(dp, sizes)):
            f = torch.full((hh, ww, 2), float("nan"), device=dev)
            dis.dis_compute_flow_fb(h, x, y, ww, hh, ww, p, f)
            torch.cuda.synchronize()
            assert np.array_equal(host(f), runs[0][k]), k
            assert np.array_equal(runs[0][k], runs[1][k]), k
        # one slot too few
        with pytest.raises(dis.DisError) as ei:
            dis.dis_compute_flow_batched(h, dis.make_pairs(items + items[:1]), len(items) + 1, p)
        assert ei.value.status == dis.DIS_ERR_INVALID_ARG
    finally:
        dis.dis_destroy(h)


def test_fb_refusals(env):
    torch, dis, dev = env
    I0, I1, _ = synth.translation_pair(0)
    H, W = I0.shape
    a, b = to_dev(torch, I0, dev), to_dev(torch, I1, dev)
    p = fb_params(dis, "default", patch_size=8, stride_override=4, coarsest_scale=2)
    flow = torch.zeros((H, W, 2), device=dev)
    h1 = dis.dis_create(W, H, 1, 1)
    try:
        with pytest.raises(dis.DisError):
            dis.dis_compute_flow_fb(h1, a, b, W, H, W, p, flow)  # one slot: needs two
    finally:
        dis.dis_destroy(h1)
    h = dis.dis_create(W, H, 2, 1)
    try:
        ss = dis.dis_levels(W, H, p)[0]
        init = torch.zeros(((H + (1 << ss) - 1) >> ss, (W + (1 << ss) - 1) >> ss, 2), device=dev)
        with pytest.raises(dis.DisError) as ei:
            dis.dis_compute_flow_ex(h, a, b, W, H, W, p, init, None, None, None, flow)
        assert ei.value.status == dis.DIS_ERR_NOT_SUPPORTED
        n = dis.dis_levels(W, H, p)[2]
        ws_bytes = dis.dis_backward_workspace_bytes(W, H, p)
        ws = torch.zeros(ws_bytes // 4 + 1, device=dev)
        fz = torch.zeros((n, 2), device=dev)
        with pytest.raises(dis.DisError) as ei:
            dis.dis_replay_flow(h, a, b, W, H, W, p, None, fz, flow, ws, ws.numel() * 4)
        assert ei.value.status == dis.DIS_ERR_NOT_SUPPORTED
        p.fb = 2
        with pytest.raises(dis.DisError):
            dis.dis_compute_flow(h, a, b, W, H, W, p, flow)
    finally:
        dis.dis_destroy(h)


def test_e2e_fb_combined_with_stereo_huber_and_early_termination(env):
    """The extensions together: forward-backward consistency on a rectified pair with the stereo
    preset, the Huber search norm and early termination (the flow's v stays 0 both ways)."""
    torch, dis, dev = env
    I0, I1, gt = synth.workload_pair("stereo320x240", 2)
    p = dis.dis_default_params("stereo_dense", norm="huber", term_eps=0.01)
    p.fb = 1
    H, W = I0.shape
    a, b = to_dev(torch, I0, dev), to_dev(torch, I1, dev)
    f = torch.full((H, W, 2), float("nan"), device=dev)
    fb_ = torch.full((H, W, 2), float("nan"), device=dev)
    h = dis.dis_create(W, H, 2, 1)
    try:
        dis.dis_compute_flow_fb(h, a, b, W, H, W, p, f, fb_)
        torch.cuda.synchronize()
    finally:
        dis.dis_destroy(h)
    got_f, got_b = host(f), host(fb_)
    assert (got_f[..., 1] == 0.0).all() and (got_b[..., 1] == 0.0).all()
    q = oracle_params(p)
    q.fb = 1

    def ref_spread(A, B):
        ref, spread = oracle_e2e(A, B, q)
        eps = q.term_eps
        for fct in (1.0 - 2e-3, 1.0 + 2e-3):  # the termination threshold's decisions too
            q.term_eps = eps * fct
            spread = np.maximum(spread, np.abs(oracle.dis_flow(A, B, q) - ref).max(-1))
        q.term_eps = eps
        return ref, spread

    check_e2e("stereo320x240 fb+huber+term forward", got_f, ref_spread(I0, I1), gt, max_unstable=0.05)
    check_e2e("stereo320x240 fb+huber+term backward", got_b, ref_spread(I1, I0), max_unstable=0.05)
