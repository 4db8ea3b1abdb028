"""Early termination of the patch search on a small step (supplementary Sec. C; reading: a
patch stops after the first update whose step is at most term_eps px) on the GPU, against the
FP64 oracle, through the C ABI.

- Search stage (`dis_search_level_ex2` with term_eps): the flow search and the stereo / Huber
  modes, every group width, max |du| <= 1e-3 px on the patches whose stopping iteration is
  determined (the oracle's result does not move when the threshold moves by 0.2 %, nor under
  1e-5 perturbations of I1).
- End to end: the medium and dense presets with term_eps against the oracle with the same
  threshold, within the end-to-end bar on the determined pixels; term_eps = 0 reproduces the
  default result bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_1603_03590_gb300 import synth
from test_gpu_parity import (STAGE_TOL, check_e2e, compare_search, gpu_level_images, host, ndimage_smooth,
                             oracle_params, run_gpu)

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


@pytest.mark.parametrize("case", ["translate", "layered-dense", "ragged"])
def test_search_stage_with_early_termination(env, case):
    torch, dis, dev = env
    if case == "translate":
        I0, I1, _ = synth.translation_pair(0)
        lv, ps, stride, iters = 0, 8, 4, 64
    elif case == "ragged":
        I0, I1, _ = synth.layered_pair(11, width=173, height=91, max_disp=6.0)
        lv, ps, stride, iters = 0, 9, 4, 64
    else:
        I0, I1, _ = synth.layered_pair(1000)
        lv, ps, stride, iters = 2, 12, 3, 128
    a, b, W, H, pitch = gpu_level_images(torch, dis, dev, I0, I1, lv)[lv]
    g = np.random.default_rng(5)
    wc, hc = (W + 1) // 2, (H + 1) // 2
    Uc_h = ndimage_smooth(g.normal(0, 1.5, (hc, wc, 2))).astype(np.float32)
    Uc = torch.from_numpy(Uc_h).to(dev)
    nx, ny = oracle.grid_n(W, ps, stride), oracle.grid_n(H, ps, stride)
    A, B = host(a, W), host(b, W)
    for dof, norm, eps in [(2, 0, 0.05), (2, 0, 0.005), (1, 0, 0.02), (2, 2, 0.02)]:
        refs = None
        for variant in dis.dis_search_mode_variants(ps):
            u = torch.zeros((ny * nx, 2), device=dev)
            ui = torch.zeros((ny * nx, 2), device=dev)
            st = torch.zeros(ny * nx, dtype=torch.int32, device=dev)
            dis.dis_search_level_ex2(a, b, W, H, pitch, Uc, wc, hc, 2.0, ps, stride, iters, variant, dof, norm, 5.0,
                                     u, ui, st, term_eps=eps)
            torch.cuda.synchronize()
            mode = dict(dof=dof, norm=norm, huber_b=5.0, term_eps=eps)
            e, ndiff, refs = compare_search(A, B, Uc_h.astype(np.float64), 2.0, ps, stride, iters, host(u), host(ui),
                                            st.cpu().numpy(), refs, mode=mode, max_unstable=0.05)
            print("search %s dof %d norm %d term %.3f width %d: max |du| %.2e, %s"
                  % (case, dof, norm, eps, variant, e, ndiff))
            assert e <= STAGE_TOL
    u = torch.zeros((ny * nx, 2), device=dev)
    with pytest.raises(dis.DisError):
        dis.dis_search_level_ex2(a, b, W, H, pitch, Uc, wc, hc, 2.0, ps, stride, iters, 0, 2, 0, 5.0, u,
                                 term_eps=-1.0)


def oracle_e2e_term(I0, I1, q):
    """FP64 flow and its spread over two 1e-4 perturbations of I1 and two 0.2 % moves of the
    termination threshold."""
    ref = oracle.dis_flow(I0, I1, q)
    spread = np.zeros(ref.shape[:2])
    for seed in (1, 2):
        n = np.random.default_rng(seed).standard_normal(I1.shape) * (1e-4 / 255.0)
        spread = np.maximum(spread, np.abs(oracle.dis_flow(I0, I1.astype(np.float64) + n, q) - ref).max(-1))
    eps = q.term_eps
    for f in (1.0 - 2e-3, 1.0 + 2e-3):
        q.term_eps = eps * f
        spread = np.maximum(spread, np.abs(oracle.dis_flow(I0, I1, q) - ref).max(-1))
    q.term_eps = eps
    return ref, spread


@pytest.mark.parametrize("preset,eps", [("medium", 0.01), ("dense", 0.02)])
def test_e2e_with_early_termination(env, preset, eps):
    torch, dis, dev = env
    I0, I1, gt = synth.layered_pair(2400, width=320, height=240, max_disp=12.8)
    p = dis.dis_default_params(preset, term_eps=eps)
    got, _ = run_gpu(torch, dis, dev, I0, I1, p)
    q = oracle_params(p)
    check_e2e("layered320x240-%s term %.3f" % (preset, eps), got, oracle_e2e_term(I0, I1, q), gt, max_unstable=0.05)
    p0 = dis.dis_default_params(preset)
    p0z = dis.dis_default_params(preset, term_eps=0.0)
    a, _ = run_gpu(torch, dis, dev, I0, I1, p0)
    b, _ = run_gpu(torch, dis, dev, I0, I1, p0z)
    assert np.array_equal(a, b)
    print("term %.3f vs none: mean |du| %.2e px" % (eps, float(np.abs(got - a).mean())))
