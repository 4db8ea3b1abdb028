"""The allocation-free refinement entry point against the handle-based one.

dis_refine_level_noalloc exists for callers that cannot allocate device memory (a plugin
inside an application that owns the device-memory budget, a loop where cudaMalloc is not
allowed because it can synchronise the device): its scratch is a fixed array inside the
library instead of a handle's arena.  Both calls must give the same refined flow; two calls
in a row check that leftovers of the previous call in the shared array do not leak into the
next one.  Both run the same kernels with the same arguments and launch form, so the flows
must agree bit for bit (stricter than the 1e-3 px per-stage tolerance of the oracle parity
tests; bit equality would also expose leftovers of the previous call, such as stale padding
columns, that a tolerance could hide).  This file is collected last so that a failure here stops a `-x` run only after
every other test has run; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_1603_03590_gb300 import synth

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


def _level(seed, w, h, channels):
    from scipy import ndimage
    I0, I1, _ = synth.layered_pair(seed, width=w, height=h, max_disp=6.0, channels=channels)
    g = np.random.default_rng(seed)
    U = np.stack([ndimage.gaussian_filter(g.normal(0, 2.0, (h, w)), 3.0) for _ in range(2)], -1) * 3.0
    return (I0 * 255.0).astype(np.float32), (I1 * 255.0).astype(np.float32), U.astype(np.float32)


def test_noalloc_matches_handle_entry_point_twice(env):
    torch, dis, dev = env
    cases = [(1, 320, 240, 1, 2, 5), (2, 173, 91, 3, 1, 7)]  # second call: other size, colour
    for seed, w, h, C, outer, inner in cases:
        I0, I1, U0 = _level(seed, w, h, C)
        pitch = w + 3
        a = torch.zeros(I0.shape[:-1] + (pitch,), device=dev)
        b = torch.zeros(I1.shape[:-1] + (pitch,), device=dev)
        a[..., :w] = torch.from_numpy(I0).to(dev)
        b[..., :w] = torch.from_numpy(I1).to(dev)
        U_ref = torch.from_numpy(U0).to(dev)
        U_new = torch.from_numpy(U0).to(dev)
        hd = dis.dis_create(pitch, h, 1, C)
        try:
            dis.dis_refine_level(hd, a, b, w, h, pitch, C, U_ref, outer, inner)
        finally:
            torch.cuda.synchronize()
            dis.dis_destroy(hd)
        dis.dis_refine_level_noalloc(a, b, w, h, pitch, C, U_new, outer, inner)
        torch.cuda.synchronize()
        ref, new = U_ref.cpu().numpy(), U_new.cpu().numpy()
        assert np.isfinite(new).all()
        assert np.array_equal(new, ref), (w, h, C, np.abs(new - ref).max())
        assert np.abs(new - U0).max() > 1e-3  # the refinement did change the flow


def test_noalloc_rejects_levels_above_its_fixed_scratch(env):
    torch, dis, dev = env
    w, h = 1024, 436  # (15 + 8) * 1024 * 436 floats > DIS_NOALLOC_SCRATCH_FLOATS
    a = torch.zeros((h, w), device=dev)
    U = torch.zeros((h, w, 2), device=dev)
    with pytest.raises(dis.DisError) as e:
        dis.dis_refine_level_noalloc(a, a, w, h, w, 1, U, 1, 1)
    assert e.value.status == dis.DIS_ERR_INVALID_ARG
    assert "scratch" in dis.dis_last_error_string(None)
