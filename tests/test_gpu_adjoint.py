"""Adjoint of the differentiable DIS map against FP64 central finite differences.

The map replays every patch's recorded search increment (u_i = u_init,i + Delta_i, Delta_i
frozen) and differentiates through the initial-displacement sampling, densification (Eq. 3),
ten unrolled red-black SOR sweeps per level (Sec. 2.3) and the pyramid, into the mean
Charbonnier photometric loss.  The GPU's analytic gradient (the FP64 replay and adjoint of
dis_backward, through torch.autograd) is compared with central differences (step 1e-4) of the FP64 oracle run with
the same frozen increments, at seeded coordinates of I0, I1 and the initial flow, drawn until
200 of them are comparable (the number drawn is printed).  The
map is not smooth at the scale of that step everywhere: the robust weights Psi'(a^2) =
1 / (2 sqrt(a^2 + eps^2)), eps = 0.001, bend sharply where residuals are near eps, and bilinear
cells and the max(1, |d|) branch give kinks.  A coordinate is therefore compared only when its
central difference has converged at step h (halving the step changes it by less than 0.3 of
the tolerance) and no discrete decision (the oracle's decision trace) flips within h of the
point; the others are counted and reported.
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
PARAMS = dict(patch_size=8, overlap=0.5, grad_iters=16, coarsest_scale=3, var_outer=1, var_inner=10)


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
    _W.update(I0=I0, I1=I1, rec=rec, init=init, q=oracle.params(**library_values(kw)))


def _fd_task(task):
    kind, idx, step = task
    I0, I1, init = _W["I0"].copy(), _W["I1"].copy(), _W["init"].copy()
    arr = {"I0": I0, "I1": I1, "init": init}[kind]
    arr.reshape(-1)[idx] += step
    flow, hv = oracle.dis_flow(I0, I1, _W["q"], init_flow=init, frozen=_W["rec"], want_hash=True)
    loss, hv2 = oracle.charbonnier_loss(I0, I1, flow, 1e-3, hash_seed=hv)
    return loss, hv2


def fd_compare(I0, I1, rec, init, kw, grads, seed, want, max_draw, split=(0.4, 0.4, 0.2), label="adjoint"):
    """Compares the analytic gradients `grads` (dict I0 / I1 / init of arrays) with FP64 central
    differences of the oracle's frozen map at seeded coordinates of I0, I1 and the initial flow
    (in the proportions `split`), drawn in rounds until `want` of them are comparable (at most
    `max_draw` drawn).  A coordinate is comparable when no decision of the oracle's trace flips
    within h of it (all four stencil points take the centre's decisions: a boundary between h/2
    and h would bend the step-h difference alone) and its central difference has converged at
    step h (halving the step changes it by less than 0.3 of the tolerance).  Returns (errors,
    drawn, flips, unconverged); errors are (relative error, kind, index, analytic, FD at h, FD at
    h/2)."""
    rng = np.random.default_rng(seed)
    steps = (H_STEP, -H_STEP, 0.5 * H_STEP, -0.5 * H_STEP)
    sizes = {"I0": I0.size, "I1": I1.size, "init": init.size}
    errs, drawn, flips, unconverged = [], 0, 0, 0
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, os.cpu_count() or 1), initializer=_init_worker,
                  initargs=(I0.astype(np.float64), I1.astype(np.float64), rec, init.astype(np.float64), kw)) as pool:
        h0 = pool.map(_fd_task, [("I0", 0, 0.0)])[0][1]
        while len(errs) < want and drawn < max_draw:
            n = min(max_draw - drawn, max(40, int(1.5 * (want - len(errs)) * max(1.0, drawn / max(1, len(errs))))))
            counts = [int(round(f * n)) for f in split]
            coords = [(k, int(i)) for k, c in zip(("I0", "I1", "init"), counts)
                      for i in rng.integers(0, sizes[k], c)]
            drawn += len(coords)
            res = pool.map(_fd_task, [(k, i, st) for k, i in coords for st in steps], chunksize=4)
            for c, (k, i) in enumerate(coords):
                (lp, hp), (lm, hm), (lp2, hp2), (lm2, hm2) = res[4 * c:4 * c + 4]
                # a decision boundary within h of the point bends the central differences
                # towards the mean of the two one-sided slopes: not comparable
                if hp != h0 or hm != h0 or hp2 != h0 or hm2 != h0:
                    flips += 1
                    continue
                fd = (lp - lm) / (2 * H_STEP)
                fd2 = (lp2 - lm2) / H_STEP
                # converged at step h: halving the step changes it by less than 0.3 tol (its own
                # error is then 4/3 of that), so the map is smooth at scale h
                if abs(fd - fd2) > 0.3 * REL_TOL * max(abs(fd), 1e-12):
                    unconverged += 1
                    continue
                an = grads[k].reshape(-1)[i]
                errs.append((abs(an - fd) / max(abs(fd), 1e-12), k, i, an, fd, fd2))
    errs.sort(reverse=True)
    print("%s vs FD (step %g): %d coordinates compared of %d drawn; excluded: %d with a decision flip within h, "
          "%d whose FD has not converged at that step; worst: %s"
          % (label, H_STEP, len(errs), drawn, flips, unconverged, errs[:5]))
    return errs, drawn, flips, unconverged


def assert_within_tolerance(errs):
    mags = np.array([abs(e[4]) for e in errs])
    floor = 1e-3 * np.median(mags)  # gradients below this are compared absolutely
    bad = [e for e in errs if abs(e[3] - e[4]) > REL_TOL * max(abs(e[4]), floor)]
    assert not bad, bad[:10]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_03590_gb300 import build
    build.build()
    from paper_1603_03590_gb300 import autograd, dis
    return torch, dis, autograd, torch.device("cuda:0")


def _pair(seed):
    I0, I1, _ = synth.layered_pair(seed, width=512, height=256, max_disp=20.0)
    return I0, I1


def test_photometric_loss_gradient_matches_fd(env):
    torch, dis, ag, dev = env
    g = np.random.default_rng(0)
    I0, I1 = _pair(3001)
    flow = (g.normal(0, 1.0, (256, 512, 2)) + np.array([3.3, -1.2])).astype(np.float32)
    a = torch.tensor(I0, device=dev, requires_grad=True)
    b = torch.tensor(I1, device=dev, requires_grad=True)
    f = torch.tensor(flow, device=dev, requires_grad=True)
    loss = ag.photometric_loss(a, b, f)
    loss.backward()
    ref = oracle.charbonnier_loss(I0, I1, flow)
    assert abs(float(loss.detach()) - ref) <= 1e-6 * max(1.0, abs(ref))
    ga, gb, gf = a.grad.cpu().numpy(), b.grad.cpu().numpy(), f.grad.cpu().numpy()
    for _ in range(30):
        k = int(g.integers(0, 3))
        arr, grad = [(I0, ga), (I1, gb), (flow, gf)][k]
        idx = int(g.integers(0, arr.size))
        vals, hs = [], []
        for sgn in (1, -1):
            c = [x.astype(np.float64).copy() for x in (I0, I1, flow)]
            c[k].reshape(-1)[idx] += sgn * H_STEP
            v, hv = oracle.charbonnier_loss(c[0], c[1], c[2], 1e-3, hash_seed=0)
            vals.append(v)
            hs.append(hv)
        if hs[0] != hs[1]:
            continue
        fd = (vals[0] - vals[1]) / (2 * H_STEP)
        an = float(grad.reshape(-1)[idx])
        assert abs(an - fd) <= REL_TOL * max(abs(fd), 1e-7) + 1e-9, (k, idx, an, fd)


def test_adjoint_matches_fp64_finite_differences(env):
    torch, dis, ag, dev = env
    W, H = 512, 256
    I0, I1 = _pair(3000)
    dd = ag.DifferentiableDIS(W, H, **PARAMS)
    try:
        hs, ws = dd.coarsest_shape(W, H)
        from scipy import ndimage
        g = np.random.default_rng(7)
        init = np.stack([ndimage.gaussian_filter(g.normal(0, 1.0, (hs, ws)), 2.0) for _ in range(2)], -1)
        init = init.astype(np.float32)
        a = torch.tensor(I0, device=dev, requires_grad=True)
        b = torch.tensor(I1, device=dev, requires_grad=True)
        it = torch.tensor(init, device=dev, requires_grad=True)
        flow = dd(a, b, it)
        loss = ag.photometric_loss(a, b, flow)
        loss.backward()
        grads = {"I0": a.grad.cpu().numpy().astype(np.float64), "I1": b.grad.cpu().numpy().astype(np.float64),
                 "init": it.grad.cpu().numpy().astype(np.float64)}
        # the increments the forward recorded (the FP32 search is deterministic: record them
        # again) reproduce the forward's FP64 replay exactly
        n = dis.dis_levels(W, H, dd.params)[2]
        rec = torch.empty((n, 2), device=dev)
        tmp = torch.empty((H, W, 2), device=dev)
        dis.dis_compute_flow_ex(dd.handle, a.detach(), b.detach(), W, H, W, dd.params, it.detach(), None, rec, None,
                                tmp)
        nb = dis.dis_backward_workspace_bytes(W, H, dd.params)
        ws = torch.empty(nb, device=dev, dtype=torch.uint8)
        fl2 = torch.empty((H, W, 2), device=dev)
        dis.dis_replay_flow(dd.handle, a.detach(), b.detach(), W, H, W, dd.params, it.detach(), rec, fl2, ws, nb)
        torch.cuda.synchronize()
        assert torch.equal(fl2, flow.detach())
        # the FP64 replay agrees with the FP32 flow to the end-to-end bar
        dflow = (tmp - flow.detach()).abs()
        assert float(dflow.mean()) <= 0.01 and float(torch.quantile(dflow.flatten(), 0.999)) <= 0.05
        rec = rec.cpu().numpy().astype(np.float64)
        # a second backward is bit-identical (fixed-point scatters)
        a2 = a.detach().clone().requires_grad_(True)
        b2 = b.detach().clone().requires_grad_(True)
        it2 = it.detach().clone().requires_grad_(True)
        ag.photometric_loss(a2, b2, dd(a2, b2, it2)).backward()
        assert torch.equal(a2.grad, a.grad) and torch.equal(b2.grad, b.grad) and torch.equal(it2.grad, it.grad)
    finally:
        dd.close()
    errs, drawn, _, _ = fd_compare(I0, I1, rec, init, PARAMS, grads, 1234, 200, 1600)
    assert len(errs) >= 200, (len(errs), drawn)
    assert_within_tolerance(errs)


def test_repeated_calls_replay_a_graph_bit_exact(env):
    """A differentiable-form call seen before (same buffers, sizes and parameters) is replayed as
    one CUDA graph: the first call launches directly, the second captures, the third replays; all
    three give the same flow and gradients bit for bit."""
    torch, dis, ag, dev = env
    W, H = 512, 256
    I0, I1 = _pair(3100)
    dd = ag.DifferentiableDIS(W, H, **PARAMS)
    try:
        hs, ws_ = dd.coarsest_shape(W, H)
        p = dd.params
        a, b = torch.tensor(I0, device=dev), torch.tensor(I1, device=dev)
        it = torch.full((hs, ws_, 2), 0.25, device=dev)
        n = dis.dis_levels(W, H, p)[2]
        rec = torch.empty((n, 2), device=dev)
        tmp = torch.empty((H, W, 2), device=dev)
        dis.dis_compute_flow_ex(dd.handle, a, b, W, H, W, p, it, None, rec, None, tmp)
        nb = dis.dis_backward_workspace_bytes(W, H, p)
        ws = torch.empty(nb, device=dev, dtype=torch.uint8)
        flow = torch.empty((H, W, 2), device=dev)
        g = torch.from_numpy(np.random.default_rng(5).normal(0, 1e-3, (H, W, 2)).astype(np.float32)).to(dev)
        outs = [torch.empty((H, W), device=dev), torch.empty((H, W), device=dev), torch.empty_like(it)]
        flows, grads, kernels = [], [], []
        for _ in range(3):
            flow.fill_(float("nan"))
            dis.dis_replay_flow(dd.handle, a, b, W, H, W, p, it, rec, flow, ws, nb)
            kf = dis.dis_last_call_kernels(dd.handle)
            for o in outs:
                o.fill_(float("nan"))
            dis.dis_backward(dd.handle, a, b, W, H, W, p, it, rec, g, outs[0], outs[1], W, outs[2], ws, nb)
            kernels.append((kf, dis.dis_last_call_kernels(dd.handle)))
            torch.cuda.synchronize()
            flows.append(flow.clone())
            grads.append([o.clone() for o in outs])
        assert kernels[0] == (-1, -1), kernels
        assert kernels[1] == kernels[2] and min(kernels[1]) > 100, kernels
        assert bool(torch.isfinite(flows[0]).all()) and all(bool(torch.isfinite(o).all()) for o in grads[0])
        for k in (1, 2):
            assert torch.equal(flows[k], flows[0])
            assert all(torch.equal(x, y) for x, y in zip(grads[k], grads[0]))
    finally:
        dd.close()


def test_batch_of_eight_pairs(env):
    """The eight 512x256 pairs of the differentiable workload: every pair's gradient (to I0, I1
    and a smooth initial flow) through single-pair calls on one handle against FP64 central
    differences of the oracle's frozen map at 12 comparable coordinates per pair; the batched
    form (BatchedDifferentiableDIS: the pairs side by side, a handle and stream each, one backward
    over the sum of the losses) reproduces every loss and gradient bit for bit, twice in a row."""
    torch, dis, ag, dev = env
    W, H = 512, 256
    dd = ag.DifferentiableDIS(W, H, **PARAMS)
    bd = ag.BatchedDifferentiableDIS(W, H, 8, **PARAMS)
    from scipy import ndimage
    cases, inputs, single = [], [], []
    try:
        hs, ws = dd.coarsest_shape(W, H)
        for k in range(8):
            I0, I1 = _pair(3000 + k)
            g = np.random.default_rng(100 + k)
            init = np.stack([ndimage.gaussian_filter(g.normal(0, 1.0, (hs, ws)), 2.0) for _ in range(2)], -1)
            init = init.astype(np.float32)
            inputs.append((I0, I1, init))
            a = torch.tensor(I0, device=dev, requires_grad=True)
            b = torch.tensor(I1, device=dev, requires_grad=True)
            it = torch.tensor(init, device=dev, requires_grad=True)
            loss = ag.photometric_loss(a, b, dd(a, b, it))
            loss.backward()
            grads = (a.grad.clone(), b.grad.clone(), it.grad.clone())
            assert all(torch.isfinite(x).all() for x in grads)
            single.append((loss.detach().clone(),) + grads)
            n = dis.dis_levels(W, H, dd.params)[2]
            rec = torch.empty((n, 2), device=dev)
            tmp = torch.empty((H, W, 2), device=dev)
            dis.dis_compute_flow_ex(dd.handle, a.detach(), b.detach(), W, H, W, dd.params, it.detach(), None, rec,
                                    None, tmp)
            torch.cuda.synchronize()
            cases.append((I0, I1, rec.cpu().numpy().astype(np.float64), init,
                          {"I0": grads[0].cpu().numpy().astype(np.float64),
                           "I1": grads[1].cpu().numpy().astype(np.float64),
                           "init": grads[2].cpu().numpy().astype(np.float64)}))
        for _ in range(2):
            a = [torch.tensor(I0, device=dev, requires_grad=True) for I0, _, _ in inputs]
            b = [torch.tensor(I1, device=dev, requires_grad=True) for _, I1, _ in inputs]
            it = [torch.tensor(init, device=dev, requires_grad=True) for _, _, init in inputs]
            flows = bd(a, b, it)
            losses = [ag.photometric_loss(x, y, f) for x, y, f in zip(a, b, flows)]
            torch.stack(losses).sum().backward()
            torch.cuda.synchronize()
            for k in range(8):
                got = (losses[k].detach(), a[k].grad, b[k].grad, it[k].grad)
                assert all(torch.equal(x, y) for x, y in zip(got, single[k])), k
    finally:
        dd.close()
        bd.close()
    for k, (I0, I1, rec, init, grads) in enumerate(cases):
        errs, drawn, _, _ = fd_compare(I0, I1, rec, init, PARAMS, grads, 500 + k, 12, 200,
                                       label="batch pair %d" % k)
        assert len(errs) >= 12, (k, len(errs), drawn)
        assert_within_tolerance(errs)


def test_adjoint_with_final_upscaling_matches_fd(env):
    """theta_sf = 1: the map ends with the bilinear up-scaling of level 1 to full resolution, and
    the backward starts with its transpose."""
    torch, dis, ag, dev = env
    W, H = 256, 128
    kw = dict(PARAMS, coarsest_scale=3, finest_scale=1)
    I0, I1, _ = synth.layered_pair(3002, width=W, height=H, max_disp=10.0)
    dd = ag.DifferentiableDIS(W, H, **kw)
    try:
        hs, ws = dd.coarsest_shape(W, H)
        from scipy import ndimage
        g = np.random.default_rng(9)
        init = np.stack([ndimage.gaussian_filter(g.normal(0, 1.0, (hs, ws)), 2.0) for _ in range(2)], -1)
        init = init.astype(np.float32)
        a = torch.tensor(I0, device=dev, requires_grad=True)
        b = torch.tensor(I1, device=dev, requires_grad=True)
        it = torch.tensor(init, device=dev, requires_grad=True)
        flow = dd(a, b, it)
        loss = ag.photometric_loss(a, b, flow)
        loss.backward()
        grads = {"I0": a.grad.cpu().numpy().astype(np.float64), "I1": b.grad.cpu().numpy().astype(np.float64),
                 "init": it.grad.cpu().numpy().astype(np.float64)}
        n = dis.dis_levels(W, H, dd.params)[2]
        rec = torch.empty((n, 2), device=dev)
        tmp = torch.empty((H, W, 2), device=dev)
        dis.dis_compute_flow_ex(dd.handle, a.detach(), b.detach(), W, H, W, dd.params, it.detach(), None, rec, None,
                                tmp)
        torch.cuda.synchronize()
        dflow = (tmp - flow.detach()).abs()
        assert float(dflow.mean()) <= 0.01 and float(torch.quantile(dflow.flatten(), 0.999)) <= 0.05
        rec = rec.cpu().numpy().astype(np.float64)
    finally:
        dd.close()
    errs, drawn, _, _ = fd_compare(I0, I1, rec, init, kw, grads, 77, 100, 800, label="adjoint with theta_sf = 1")
    assert len(errs) >= 100, (len(errs), drawn)
    assert_within_tolerance(errs)
