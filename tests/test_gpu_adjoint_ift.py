"""Implicit-function gradient through the patch search (dis_params.search_grad = 1) against
FP64 central finite differences of the oracle's converged-search map.

The map: per level, every patch with a nonzero recorded increment is the solution of its
search's stationarity condition g(u) = sum S'(w~ - T) = 0 reached from u_init + increment (the
oracle solves it by Newton steps, `polish`); zero increments stay at u_init; densification,
refinement and the pyramid as in the frozen map.  The increments the GPU replays are the
oracle's converged ones (so the replay point is the solution to FP32 resolution), and the
GPU's analytic gradient of the mean Charbonnier loss (FP64 replay, the search adjoint
lambda = -J^-T g_u scattered into both frames, the rest of the adjoint unchanged) is compared
with central differences at seeded coordinates of I0, I1 and the initial flow, with the
coordinate filters of the frozen-map test (decision flips within h/2, unconverged differences).
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle
from paper_1603_03590_gb300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-3
H_STEP = 1e-4
PARAMS = dict(patch_size=8, overlap=0.5, grad_iters=64, coarsest_scale=2, var_outer=1, var_inner=5)
POLISH = 60


def library_values(kw):
    """The oracle's keyword parameters with the values the library evaluates: its dis_params
    fields are FP32, so the SOR relaxation factor is 1.6f = 1.600000024, not 1.6.  A finite
    difference of the FP64 oracle must differentiate the same map as the FP64 adjoint; with the
    double 1.6 the two maps differ by 2.4e-8 in omega, which the levels and sweeps compound
    into relative gradient differences up to 2e-3 at four levels."""
    q = dict(kw)
    q.setdefault("sor_omega", 1.6)
    for k in ("sor_omega", "delta", "gamma", "alpha"):
        if k in q:
            q[k] = float(np.float32(q[k]))
    return q

_W = {}


def _init_worker(I0, I1, rec, init, kw):
    _W.update(I0=I0, I1=I1, rec=rec, init=init, q=oracle.params(polish=POLISH, **library_values(kw)))


def _init_worker_kw(I0, I1, rec, init, kw):
    _W.update(I0=I0, I1=I1, rec=rec, init=init, q=oracle.params(**library_values(kw)))


def _fd_task(task):
    kind, idx, step = task
    I0, I1, init = _W["I0"].copy(), _W["I1"].copy(), _W["init"].copy()
    arr = {"I0": I0, "I1": I1, "init": init}[kind]
    arr.reshape(-1)[idx] += step
    flow, hv = oracle.dis_flow(I0, I1, _W["q"], init_flow=init, frozen=_W["rec"], want_hash=True)
    loss, hv2 = oracle.charbonnier_loss(I0, I1, flow, 1e-3, hash_seed=hv)
    return loss, hv2


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_03590_gb300 import build
    build.build()
    from paper_1603_03590_gb300 import autograd, dis
    return torch, dis, autograd, torch.device("cuda:0")


def test_implicit_search_gradient_matches_fp64_finite_differences(env):
    torch, dis, ag, dev = env
    W, H = 192, 128
    I0, I1, _ = synth.layered_pair(3100, width=W, height=H, n_ellipses=6, max_disp=6.0)
    dd = ag.DifferentiableDIS(W, H, search_grad=1, **PARAMS)
    try:
        hs, ws = dd.coarsest_shape(W, H)
        from scipy import ndimage
        g = np.random.default_rng(8)
        init = np.stack([ndimage.gaussian_filter(g.normal(0, 0.5, (hs, ws)), 2.0) for _ in range(2)], -1)
        init = init.astype(np.float32)
        a = torch.tensor(I0, device=dev, requires_grad=True)
        b = torch.tensor(I1, device=dev, requires_grad=True)
        it = torch.tensor(init, device=dev, requires_grad=True)
        # increments of the FP32 search, then converged by the oracle (FP64 Newton on g = 0)
        n = dis.dis_levels(W, H, dd.params)[2]
        rec0 = torch.empty((n, 2), device=dev)
        tmp = torch.empty((H, W, 2), device=dev)
        dis.dis_compute_flow_ex(dd.handle, a.detach(), b.detach(), W, H, W, dd.params, it.detach(), None, rec0, None,
                                tmp)
        torch.cuda.synchronize()
        q = oracle.params(polish=POLISH, **library_values(PARAMS))
        _, rec_star = oracle.dis_flow(I0.astype(np.float64), I1.astype(np.float64), q,
                                      init_flow=init.astype(np.float64),
                                      frozen=rec0.cpu().numpy().astype(np.float64), record=True)
        rec_star = rec_star.astype(np.float32)
        moved = np.abs(rec_star).max(1) > 0
        assert moved.mean() > 0.8
        frozen = torch.from_numpy(rec_star).to(dev)
        flow = dd(a, b, it, frozen=frozen)
        loss = ag.photometric_loss(a, b, flow)
        loss.backward()
        grads = {"I0": a.grad.cpu().numpy().astype(np.float64), "I1": b.grad.cpu().numpy().astype(np.float64),
                 "init": it.grad.cpu().numpy().astype(np.float64)}
        # deterministic: a second backward is bit-identical
        a2 = a.detach().clone().requires_grad_(True)
        b2 = b.detach().clone().requires_grad_(True)
        it2 = it.detach().clone().requires_grad_(True)
        ag.photometric_loss(a2, b2, dd(a2, b2, it2, frozen=frozen)).backward()
        assert torch.equal(a2.grad, a.grad) and torch.equal(b2.grad, b.grad) and torch.equal(it2.grad, it.grad)
        # the frozen-increment gradient differs: the search's dependence on the frames entered
        dd.params.search_grad = 0
        a3 = a.detach().clone().requires_grad_(True)
        ag.photometric_loss(a3, b.detach(), dd(a3, b.detach(), it.detach(), frozen=frozen)).backward()
        assert not torch.equal(a3.grad, a.grad)
    finally:
        dd.close()
    rng = np.random.default_rng(4321)
    coords = ([("I0", int(i)) for i in rng.integers(0, I0.size, 80)] +
              [("I1", int(i)) for i in rng.integers(0, I1.size, 80)] +
              [("init", int(i)) for i in rng.integers(0, init.size, 30)])
    steps = (H_STEP, -H_STEP, 0.5 * H_STEP, -0.5 * H_STEP)
    tasks = [(k, i, st) for k, i in coords for st in steps] + [("I0", 0, 0.0)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, os.cpu_count() or 1), initializer=_init_worker,
                  initargs=(I0.astype(np.float64), I1.astype(np.float64), rec_star.astype(np.float64),
                            init.astype(np.float64), PARAMS)) as pool:
        res = pool.map(_fd_task, tasks, chunksize=4)
    h0 = res[-1][1]
    flips, unconverged, errs = 0, 0, []
    for c, (k, i) in enumerate(coords):
        (lp, hp), (lm, hm), (lp2, hp2), (lm2, hm2) = res[4 * c:4 * c + 4]
        if hp2 != h0 or hm2 != h0:
            flips += 1
            continue
        fd = (lp - lm) / (2 * H_STEP)
        fd2 = (lp2 - lm2) / H_STEP
        an = grads[k].reshape(-1)[i]
        if abs(fd - fd2) > 0.3 * REL_TOL * max(abs(fd), 1e-12):
            unconverged += 1
            continue
        errs.append((abs(an - fd) / max(abs(fd), 1e-12), k, i, an, fd))
    errs.sort(reverse=True)
    print("implicit search gradient vs FD (step %g): %d coordinates compared; excluded: %d with a decision flip "
          "within h/2, %d whose FD has not converged at that step; worst: %s"
          % (H_STEP, len(errs), flips, unconverged, errs[:5]))
    assert len(errs) >= 60
    mags = np.array([abs(e[4]) for e in errs])
    floor = 1e-3 * np.median(mags)
    bad = [e for e in errs if abs(e[3] - e[4]) > REL_TOL * max(abs(e[4]), floor)]
    assert not bad, bad[:10]


@pytest.mark.parametrize("search_grad", [0, 1])
def test_stereo_gradient_matches_fp64_finite_differences(env, search_grad):
    """The differentiable form in the stereo mode (one degree of freedom: the scalar SOR update in
    the replay and its adjoint), with the search frozen or differentiated implicitly (the scalar
    stationarity condition in u)."""
    torch, dis, ag, dev = env
    W, H = 192, 128
    kw = dict(PARAMS, dof=1)
    I0, I1, _ = synth.layered_pair(3101, width=W, height=H, n_ellipses=6, max_disp=6.0, horizontal=True)
    dd = ag.DifferentiableDIS(W, H, search_grad=search_grad, **kw)
    try:
        hs, ws = dd.coarsest_shape(W, H)
        from scipy import ndimage
        g = np.random.default_rng(10)
        init = np.stack([ndimage.gaussian_filter(g.normal(0, 0.5, (hs, ws)), 2.0), np.zeros((hs, ws))], -1)
        init = init.astype(np.float32)
        a = torch.tensor(I0, device=dev, requires_grad=True)
        b = torch.tensor(I1, device=dev, requires_grad=True)
        it = torch.tensor(init, device=dev, requires_grad=True)
        n = dis.dis_levels(W, H, dd.params)[2]
        rec0 = torch.empty((n, 2), device=dev)
        tmp = torch.empty((H, W, 2), device=dev)
        dis.dis_compute_flow_ex(dd.handle, a.detach(), b.detach(), W, H, W, dd.params, it.detach(), None, rec0, None,
                                tmp)
        torch.cuda.synchronize()
        rec = rec0.cpu().numpy().astype(np.float64)
        if search_grad:
            q = oracle.params(polish=POLISH, **library_values(kw))
            _, rec = oracle.dis_flow(I0.astype(np.float64), I1.astype(np.float64), q,
                                     init_flow=init.astype(np.float64), frozen=rec, record=True)
        rec = rec.astype(np.float32)
        assert (rec[:, 1] == 0.0).all()
        flow = dd(a, b, it, frozen=torch.from_numpy(rec).to(dev))
        loss = ag.photometric_loss(a, b, flow)
        loss.backward()
        grads = {"I0": a.grad.cpu().numpy().astype(np.float64), "I1": b.grad.cpu().numpy().astype(np.float64),
                 "init": it.grad.cpu().numpy().astype(np.float64)}
    finally:
        dd.close()
    rng = np.random.default_rng(4400 + search_grad)
    coords = ([("I0", int(i)) for i in rng.integers(0, I0.size, 50)] +
              [("I1", int(i)) for i in rng.integers(0, I1.size, 50)] +
              [("init", int(i)) for i in rng.integers(0, init.size, 20)])
    steps = (H_STEP, -H_STEP, 0.5 * H_STEP, -0.5 * H_STEP)
    tasks = [(k, i, st) for k, i in coords for st in steps] + [("I0", 0, 0.0)]
    ctx = mp.get_context("spawn")
    kw_fd = dict(kw, polish=POLISH if search_grad else 0)
    with ctx.Pool(min(16, os.cpu_count() or 1), initializer=_init_worker_kw,
                  initargs=(I0.astype(np.float64), I1.astype(np.float64), rec.astype(np.float64),
                            init.astype(np.float64), kw_fd)) as pool:
        res = pool.map(_fd_task, tasks, chunksize=4)
    h0 = res[-1][1]
    flips, unconverged, errs = 0, 0, []
    for c, (k, i) in enumerate(coords):
        (lp, hp), (lm, hm), (lp2, hp2), (lm2, hm2) = res[4 * c:4 * c + 4]
        if hp2 != h0 or hm2 != h0:
            flips += 1
            continue
        fd = (lp - lm) / (2 * H_STEP)
        fd2 = (lp2 - lm2) / H_STEP
        an = grads[k].reshape(-1)[i]
        if abs(fd - fd2) > 0.3 * REL_TOL * max(abs(fd), 1e-12):
            unconverged += 1
            continue
        errs.append((abs(an - fd) / max(abs(fd), 1e-12), k, i, an, fd))
    errs.sort(reverse=True)
    print("stereo gradient (search_grad %d) vs FD: %d compared, %d flips, %d unconverged; worst: %s"
          % (search_grad, len(errs), flips, unconverged, errs[:4]))
    assert len(errs) >= 40
    mags = np.array([abs(e[4]) for e in errs])
    floor = 1e-3 * np.median(mags)
    bad = [e for e in errs if abs(e[3] - e[4]) > REL_TOL * max(abs(e[4]), floor)]
    assert not bad, bad[:10]
