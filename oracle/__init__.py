"""FP64 CPU oracle for Dense Inverse Search (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg import
this package.  It wraps ``dis_oracle.c`` (plain C, double precision, single thread) with
ctypes and numpy; it shares nothing with the CUDA path of ``paper_1603_03590_gb300``.

Layouts: images are (H, W) or (C, H, W) float64 arrays; flows are (H, W, 2) with
(u, v) = (displacement along x / columns, along y / rows).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dis_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile dis_oracle.c into liboracle.so next to it (gcc -O2, no SIMD intrinsics)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class OrParams(ctypes.Structure):
    _fields_ = [
        ("patch_size", ctypes.c_int),
        ("overlap", ctypes.c_double),
        ("stride_override", ctypes.c_int),
        ("grad_iters", ctypes.c_int),
        ("coarsest_scale", ctypes.c_int),
        ("finest_scale", ctypes.c_int),
        ("refine", ctypes.c_int),
        ("var_outer", ctypes.c_int),
        ("var_inner", ctypes.c_int),
        ("delta", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("sor_omega", ctypes.c_double),
        ("intensity_scale", ctypes.c_double),
        ("channels", ctypes.c_int),
        ("dof", ctypes.c_int),
        ("norm", ctypes.c_int),
        ("huber_b", ctypes.c_double),
        ("fb", ctypes.c_int),
        ("term_eps", ctypes.c_double),
        ("polish", ctypes.c_int),
    ]


def params(**kw):
    """Parameter set with the paper's defaults (Sec. 3.1) overridden by keyword."""
    d = dict(patch_size=8, overlap=0.3, stride_override=0, grad_iters=16, coarsest_scale=-1,
             finest_scale=0, refine=1, var_outer=-1, var_inner=5, delta=5.0, gamma=10.0,
             alpha=10.0, sor_omega=1.6, intensity_scale=255.0, channels=1, dof=2, norm=0, huber_b=5.0,
             fb=0, term_eps=0.0, polish=0)
    d.update(kw)
    return OrParams(**d)


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i, d, u64p = ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)
        P = ctypes.POINTER(OrParams)
        sig = {
            "or_bilinear": (d, [_D, i, i, d, d]),
            "or_robust_error": (d, [d, i, d]),
            "or_pyr_down": (None, [_D, i, i, _D]),
            "or_sobel": (None, [_D, i, i, _D, _D]),
            "or_stride": (i, [i, d, i]),
            "or_grid_n": (i, [i, i, i]),
            "or_grid_pos": (i, [i, i, i, i]),
            "or_levels": (i, [i, i, P, _I, _I]),
            "or_search_level": (None, [_D, _D, _D, _D, i, i, _D, i, i, d, i, i, i, _D, _D, _D, _I, i, i, d, d, i]),
            "or_densify_level": (None, [_D, _D, i, i, _D, i, i, _D, i, i, d, _D]),
            "or_refine_level": (None, [_D, _D, i, i, i, _D, i, i, d, d, d, d, i]),
            "or_upsample_flow": (None, [_D, i, i, d, _D, i, i]),
            "or_total_patches": (i, [i, i, P]),
            "or_dis_flow": (i, [_D, _D, i, i, P, _D, _D, _D, _D, u64p]),
            "or_dis_flow_fb": (i, [_D, _D, i, i, P, _D, _D, _D, _D, _D, u64p]),
            "or_densify_level_fb": (None, [_D, _D, i, i, _D, _D, i, i, _D, i, i, d, _D]),
            "or_charbonnier_loss": (d, [_D, _D, i, i, i, _D, d, u64p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return None if a is None else a.ctypes.data_as(_D)


def bilinear(img, x, y):
    img = _f64(img)
    h, w = img.shape
    return _load().or_bilinear(_p(img), w, h, float(x), float(y))


def pyr_down(img):
    img = _f64(img)
    h, w = img.shape
    out = np.empty(((h + 1) // 2, (w + 1) // 2))
    _load().or_pyr_down(_p(img), w, h, _p(out))
    return out


def sobel(img):
    img = _f64(img)
    h, w = img.shape
    gx, gy = np.empty_like(img), np.empty_like(img)
    _load().or_sobel(_p(img), w, h, _p(gx), _p(gy))
    return gx, gy


def stride(ps, overlap, stride_override=0):
    return _load().or_stride(ps, float(overlap), stride_override)


def grid_n(length, ps, stride_):
    return _load().or_grid_n(length, ps, stride_)


def grid_pos(i, length, ps, stride_):
    return _load().or_grid_pos(i, length, ps, stride_)


def levels(W, H, prm):
    ss, sf = ctypes.c_int(), ctypes.c_int()
    rc = _load().or_levels(W, H, ctypes.byref(prm), ctypes.byref(ss), ctypes.byref(sf))
    return rc, ss.value, sf.value


def robust_error(e, norm, huber_b=5.0):
    """Per-pixel error transform of the robust norms (0 L2, 1 L1, 2 Huber)."""
    return _load().or_robust_error(float(e), int(norm), float(huber_b))


def search_level(I0, Ix, Iy, I1, ps, stride_, iters, Uc=None, cscale=2.0, frozen=None, dof=2, norm=0, huber_b=5.0,
                 term_eps=0.0, polish=0):
    """Inverse search of one level.  Returns (u, u_init, status) with u, u_init of shape
    (ny, nx, 2) and status (ny, nx) in {0 ok, 1 reset, 2 flat}.  dof = 1: horizontal only;
    norm: 0 L2, 1 L1, 2 Huber with threshold huber_b; term_eps > 0: a patch stops after the
    first step of length <= term_eps."""
    I0, Ix, Iy, I1 = _f64(I0), _f64(Ix), _f64(Iy), _f64(I1)
    h, w = I0.shape
    nx, ny = grid_n(w, ps, stride_), grid_n(h, ps, stride_)
    u = np.zeros((ny, nx, 2))
    ui = np.zeros((ny, nx, 2))
    st = np.zeros((ny, nx), dtype=np.int32)
    wc = hc = 0
    if Uc is not None:
        Uc = _f64(Uc)
        hc, wc = Uc.shape[:2]
    fz = None if frozen is None else _f64(frozen)
    _load().or_search_level(_p(I0), _p(Ix), _p(Iy), _p(I1), w, h, _p(Uc), wc, hc, float(cscale), ps, stride_,
                            iters, _p(fz), _p(u), _p(ui), st.ctypes.data_as(_I), int(dof), int(norm),
                            float(huber_b), float(term_eps), int(polish))
    return u, ui, st


def densify_level_fb(I0, I1, u, ub, ps, stride_, Uc=None, cscale=2.0):
    """Densification with forward-backward consistency: this direction's patch flows u (grid on
    I0) merged with the other direction's ub (grid on I1, displacements into I0).  Returns the
    dense field on I0's grid; the other direction's is densify_level_fb(I1, I0, ub, u, ...)."""
    I0, I1, u, ub = _f64(I0), _f64(I1), _f64(u), _f64(ub)
    h, w = I0.shape
    U = np.zeros((h, w, 2))
    wc = hc = 0
    if Uc is not None:
        Uc = _f64(Uc)
        hc, wc = Uc.shape[:2]
    _load().or_densify_level_fb(_p(I0), _p(I1), w, h, _p(u), _p(ub), ps, stride_, _p(Uc), wc, hc, float(cscale),
                                _p(U))
    return U


def dis_flow_fb(I0, I1, prm):
    """Whole method with forward-backward consistency (prm.fb is set here): returns the forward
    and the backward flow, both (H, W, 2)."""
    I0, I1 = _f64(I0), _f64(I1)
    H, W = I0.shape[-2:]
    prm.fb = 1
    flow = np.zeros((H, W, 2))
    flow_b = np.zeros((H, W, 2))
    rc = _load().or_dis_flow_fb(_p(I0), _p(I1), W, H, ctypes.byref(prm), None, None, None, _p(flow), _p(flow_b), None)
    if rc != 0:
        raise ValueError("oracle error %d" % rc)
    return flow, flow_b


def densify_level(I0, I1, u, ps, stride_, Uc=None, cscale=2.0):
    I0, I1, u = _f64(I0), _f64(I1), _f64(u)
    h, w = I0.shape
    U = np.zeros((h, w, 2))
    wc = hc = 0
    if Uc is not None:
        Uc = _f64(Uc)
        hc, wc = Uc.shape[:2]
    _load().or_densify_level(_p(I0), _p(I1), w, h, _p(u), ps, stride_, _p(Uc), wc, hc, float(cscale), _p(U))
    return U


def refine_level(I0, I1, U, outer, inner, delta=5.0, gamma=10.0, alpha=10.0, omega=1.6, dof=2):
    """Variational refinement of one level; I0, I1 are (H, W) or (C, H, W).  Returns U + dU.
    dof = 1: the increment is horizontal only."""
    I0, I1 = _f64(I0), _f64(I1)
    if I0.ndim == 2:
        I0, I1 = I0[None], I1[None]
    C, h, w = I0.shape
    U = _f64(U).copy()
    _load().or_refine_level(_p(I0), _p(I1), w, h, C, _p(U), outer, inner, float(delta), float(gamma),
                            float(alpha), float(omega), int(dof))
    return U


def upsample_flow(U, factor, out_hw):
    U = _f64(U)
    hi, wi = U.shape[:2]
    ho, wo = out_hw
    out = np.zeros((ho, wo, 2))
    _load().or_upsample_flow(_p(U), wi, hi, float(factor), _p(out), wo, ho)
    return out


def total_patches(W, H, prm):
    return _load().or_total_patches(W, H, ctypes.byref(prm))


def dis_flow(I0, I1, prm, init_flow=None, frozen=None, record=False, want_hash=False):
    """Whole method (Alg. 1).  I0, I1: (H, W) or (C, H, W) in [0,1].
    Returns flow (H, W, 2), plus the recorded per-patch increments and/or the decision
    hash when asked.  Raises ValueError on an oracle error code."""
    I0, I1 = _f64(I0), _f64(I1)
    H, W = I0.shape[-2:]
    rec = None
    if record:
        n = total_patches(W, H, prm)
        if n < 0:
            raise ValueError("invalid level configuration")
        rec = np.zeros((n, 2))
    fz = None if frozen is None else _f64(frozen)
    init = None if init_flow is None else _f64(init_flow)
    flow = np.zeros((H, W, 2))
    hv = ctypes.c_uint64(1469598103934665603)
    rc = _load().or_dis_flow(_p(I0), _p(I1), W, H, ctypes.byref(prm), _p(init), _p(fz), _p(rec), _p(flow),
                             ctypes.byref(hv) if want_hash else None)
    if rc != 0:
        raise ValueError("oracle error %d" % rc)
    out = [flow]
    if record:
        out.append(rec)
    if want_hash:
        out.append(hv.value)
    return out[0] if len(out) == 1 else tuple(out)


def charbonnier_loss(I0, I1, flow, eps_c=1e-3, hash_seed=None):
    """Mean Charbonnier photometric loss; with hash_seed (an int) also returns the decision
    trace of the loss's samples continued from that seed."""
    I0, I1, flow = _f64(I0), _f64(I1), _f64(flow)
    if I0.ndim == 2:
        I0, I1 = I0[None], I1[None]
    C, H, W = I0.shape
    hv = ctypes.c_uint64(0 if hash_seed is None else hash_seed)
    v = _load().or_charbonnier_loss(_p(I0), _p(I1), W, H, C, _p(flow), float(eps_c),
                                    None if hash_seed is None else ctypes.byref(hv))
    return v if hash_seed is None else (v, hv.value)
