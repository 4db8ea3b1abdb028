"""Python binding of libdis.so (include/dis.h): argument marshalling only.

Every function has the C name and argument order; tensors are passed as device pointers
(``tensor.data_ptr()``) and the stream as ``torch.cuda.current_stream().cuda_stream`` unless
given.  All compute runs in the library's CUDA kernels; there is no fallback: importing this
module raises when libdis.so is missing, and every non-zero status raises DisError with the
library's message.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdis.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libdis.so is not built (%s); run __graft_entry__.build() or "
                      "python paper_1603_03590_gb300/build.py" % LIB_PATH)
_lib = ctypes.CDLL(LIB_PATH)

DIS_OK, DIS_ERR_INVALID_ARG, DIS_ERR_OUT_OF_MEMORY, DIS_ERR_CUDA = 0, 1, 2, 3
DIS_ERR_TOO_SMALL, DIS_ERR_TIMEOUT, DIS_ERR_NOT_SUPPORTED = 4, 5, 6
PRESETS = {"default": 0, "op1": 1, "op2": 2, "op3": 3, "op4": 4, "fast": 5, "medium": 6, "dense": 7,
           "stereo_op1": 8, "stereo_op2": 9, "stereo_op3": 10, "stereo_op4": 11, "stereo_dense": 12}
NORMS = {"l2": 0, "l1": 1, "huber": 2}


class DisError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("dis status %d: %s" % (status, msg))
        self.status = status


class dis_params(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("patch_size", ctypes.c_int32),
        ("overlap", ctypes.c_float),
        ("stride_override", ctypes.c_int32),
        ("grad_iters", ctypes.c_int32),
        ("coarsest_scale", ctypes.c_int32),
        ("finest_scale", ctypes.c_int32),
        ("refine", ctypes.c_int32),
        ("var_outer", ctypes.c_int32),
        ("var_inner", ctypes.c_int32),
        ("delta", ctypes.c_float),
        ("gamma", ctypes.c_float),
        ("alpha", ctypes.c_float),
        ("sor_omega", ctypes.c_float),
        ("intensity_scale", ctypes.c_float),
        ("channels", ctypes.c_int32),
        ("dof", ctypes.c_int32),
        ("norm", ctypes.c_int32),
        ("huber_b", ctypes.c_float),
        ("term_eps", ctypes.c_float),
        ("fb", ctypes.c_int32),
        ("search_grad", ctypes.c_int32),
    ]


class dis_pair(ctypes.Structure):
    _fields_ = [
        ("I0", ctypes.c_void_p),
        ("I1", ctypes.c_void_p),
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("pitch", ctypes.c_int64),
        ("flow_out", ctypes.c_void_p),
    ]


_vp, _i, _f, _i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_int64
_P = ctypes.POINTER(dis_params)
_SIGS = {
    "dis_default_params": (None, [_P, _i]),
    "dis_levels": (_i, [_i, _i, _P, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i64)]),
    "dis_create": (_i, [ctypes.POINTER(_vp), _i, _i, _i, _i]),
    "dis_destroy": (None, [_vp]),
    "dis_last_error_string": (ctypes.c_char_p, [_vp]),
    "dis_arena_bytes": (_i64, [_vp]),
    "dis_compute_flow": (_i, [_vp, _vp, _vp, _i, _i, _i64, _P, _vp, _vp]),
    "dis_compute_flow_ex": (_i, [_vp, _vp, _vp, _i, _i, _i64, _P, _vp, _vp, _vp, _vp, _vp, _vp]),
    "dis_compute_flow_batched": (_i, [_vp, ctypes.POINTER(dis_pair), _i, _P, _vp]),
    "dis_compute_flow_batched_host": (_i, [_vp, ctypes.POINTER(dis_pair), _i, _P, _vp]),
    "dis_host_flows_ready": (_i, [_vp, _vp]),
    "dis_autotune": (_i, [_vp, ctypes.POINTER(dis_pair), _i, _P, _vp, ctypes.POINTER(_i)]),
    "dis_search_variants": (_i, [_i, ctypes.POINTER(_i), _i]),
    "dis_get_tuning": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "dis_last_call_kernels": (_i, [_vp, ctypes.POINTER(_i)]),
    "dis_set_refine_split": (_i, [_vp, _i64]),
    "dis_get_refine_split": (_i, [_vp, ctypes.POINTER(_i64)]),
    "dis_set_probe": (_i, [_vp, _i, _i]),
    "dis_set_refine_fusion": (_i, [_vp, _i]),
    "dis_set_work_queue": (_i, [_vp, _i]),
    "dis_probe_ms": (_i, [_vp, ctypes.POINTER(_f)]),
    "dis_trace_batched": (_i, [_vp, ctypes.POINTER(dis_pair), _i, _P, _vp, _vp, _i, ctypes.POINTER(_i)]),
    "dis_set_search_variant": (_i, [_vp, _i, _i]),
    "dis_pyr_down": (_i, [_vp, _i, _i, _i64, _vp, _i64, _vp]),
    "dis_sobel": (_i, [_vp, _i, _i, _i64, _vp, _vp, _i64, _vp]),
    "dis_search_level": (_i, [_vp, _vp, _i, _i, _i64, _vp, _i, _i, _f, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "dis_search_level_ex": (_i, [_vp, _vp, _i, _i, _i64, _vp, _i, _i, _f, _i, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "dis_search_mode_variants": (_i, [_i, _vp, _i]),
    "dis_compute_flow_fb": (_i, [_vp, _vp, _vp, _i, _i, _i64, _P, _vp, _vp, _vp]),
    "dis_densify_level_fb": (_i, [_vp, _vp, _vp, _i, _i, _i64, _vp, _vp, _i, _i, _vp, _vp, _vp]),
    "dis_search_level_ex2": (_i, [_vp, _vp, _i, _i, _i64, _vp, _i, _i, _f, _i, _i, _i, _i, _i, _i, _f, _f, _vp, _vp,
                                  _vp, _vp]),
    "dis_refine_level_ex": (_i, [_vp, _vp, _vp, _i, _i, _i64, _i, _vp, _i, _i, _f, _f, _f, _f, _i, _vp]),
    "dis_densify_level": (_i, [_vp, _vp, _i, _i, _i64, _vp, _i, _i, _vp, _i, _i, _f, _vp, _vp]),
    "dis_refine_level": (_i, [_vp, _vp, _vp, _i, _i, _i64, _i, _vp, _i, _i, _f, _f, _f, _f, _vp]),
    "dis_upsample_flow": (_i, [_vp, _i, _i, _f, _vp, _i, _i, _vp]),
    "dis_refine_level_noalloc": (_i, [_vp, _vp, _i, _i, _i64, _i, _vp, _i, _i, _f, _f, _f, _f, _vp]),
    "dis_photometric_loss_scratch_bytes": (_i64, [_i, _i, _i64, _i]),
    "dis_photometric_loss": (_i, [_vp, _vp, _i, _i, _i64, _i, _vp, _f, _vp, _vp, _vp, _vp, _vp, _i64, _vp]),
    "dis_backward_workspace_bytes": (_i64, [_i, _i, _P]),
    "dis_replay_flow": (_i, [_vp, _vp, _vp, _i, _i, _i64, _P, _vp, _vp, _vp, _vp, _i64, _vp]),
    "dis_backward": (_i, [_vp, _vp, _vp, _i, _i, _i64, _P, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _i64, _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def _ptr(t):
    """Device pointer of a tensor (or None / int passthrough)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status, handle=None):
    if status != DIS_OK:
        msg = _lib.dis_last_error_string(handle)
        raise DisError(status, msg.decode() if msg else "")


def dis_default_params(preset="default", **overrides):
    """dis_params of a preset (name or number) with keyword overrides."""
    p = dis_params()
    _lib.dis_default_params(ctypes.byref(p), PRESETS[preset] if isinstance(preset, str) else int(preset))
    for k, v in overrides.items():
        setattr(p, k, NORMS[v] if k == "norm" and isinstance(v, str) else v)
    return p


def dis_levels(width, height, params):
    ss, sf, tot = _i(), _i(), _i64()
    _check(_lib.dis_levels(width, height, ctypes.byref(params), ctypes.byref(ss), ctypes.byref(sf), ctypes.byref(tot)))
    return ss.value, sf.value, tot.value


def dis_create(max_w, max_h, max_batch=1, channels=1):
    h = _vp()
    _check(_lib.dis_create(ctypes.byref(h), max_w, max_h, max_batch, channels))
    return h.value


def dis_destroy(handle):
    _lib.dis_destroy(handle)


def dis_last_error_string(handle=None):
    return _lib.dis_last_error_string(handle).decode()


def dis_arena_bytes(handle):
    return _lib.dis_arena_bytes(handle)


def dis_compute_flow(handle, I0, I1, w, h, pitch, params, flow_out, stream=None):
    _check(_lib.dis_compute_flow(handle, _ptr(I0), _ptr(I1), w, h, pitch, ctypes.byref(params), _ptr(flow_out),
                                 _stream(stream)), handle)


def dis_compute_flow_fb(handle, I0, I1, w, h, pitch, params, flow_out, flow_b_out=None, stream=None):
    """Forward-backward consistency: forward flow into flow_out, backward flow into flow_b_out."""
    _check(_lib.dis_compute_flow_fb(handle, _ptr(I0), _ptr(I1), w, h, pitch, ctypes.byref(params), _ptr(flow_out),
                                    _ptr(flow_b_out), _stream(stream)), handle)


def dis_compute_flow_ex(handle, I0, I1, w, h, pitch, params, init_flow, frozen_in, record_out, checkpoints,
                        flow_out, stream=None):
    _check(_lib.dis_compute_flow_ex(handle, _ptr(I0), _ptr(I1), w, h, pitch, ctypes.byref(params), _ptr(init_flow),
                                    _ptr(frozen_in), _ptr(record_out), _ptr(checkpoints), _ptr(flow_out),
                                    _stream(stream)), handle)


def make_pairs(items):
    """dis_pair array from (I0, I1, width, height, pitch, flow_out) tuples."""
    arr = (dis_pair * len(items))()
    for k, (a, b, w, h, pitch, f) in enumerate(items):
        arr[k].I0, arr[k].I1, arr[k].width, arr[k].height = _ptr(a), _ptr(b), w, h
        arr[k].pitch, arr[k].flow_out = pitch, _ptr(f)
    return arr


def dis_compute_flow_batched(handle, pairs, n, params, stream=None):
    _check(_lib.dis_compute_flow_batched(handle, pairs, n, ctypes.byref(params), _stream(stream)), handle)


def dis_compute_flow_batched_host(handle, pairs, n, params, stream=None):
    """Batched call on host frames and flows (make_pairs of CPU tensors / arrays); asynchronous."""
    _check(_lib.dis_compute_flow_batched_host(handle, pairs, n, ctypes.byref(params), _stream(stream)), handle)


def dis_host_flows_ready(handle, stream=None):
    """Order `stream` after the host copies of all earlier host-buffer calls."""
    _check(_lib.dis_host_flows_ready(handle, _stream(stream)), handle)


def dis_autotune(handle, pairs, n, params, stream=None):
    """Time the search-kernel variants on these pairs, keep the fastest; returns its lanes."""
    lanes = _i()
    _check(_lib.dis_autotune(handle, pairs, n, ctypes.byref(params), _stream(stream), ctypes.byref(lanes)), handle)
    return lanes.value


class dis_launch_record(ctypes.Structure):
    _fields_ = [("kind", _i), ("level", _i), ("ms", _f)]


LAUNCH_KINDS = ("prep", "pyramid", "search_planes", "search", "densify", "refine", "upsample")


def dis_trace_batched(handle, pairs, n, params, stream=None, cap=256):
    """Run the batched call once with events around every launch group; returns a list of
    (kind name, level, milliseconds)."""
    out = (dis_launch_record * cap)()
    cnt = _i()
    _check(_lib.dis_trace_batched(handle, pairs, n, ctypes.byref(params), _stream(stream), out, cap,
                                  ctypes.byref(cnt)), handle)
    return [(LAUNCH_KINDS[out[k].kind], out[k].level, out[k].ms) for k in range(min(cnt.value, cap))]


def dis_set_refine_fusion(handle, mode):
    """Refinement launch form: 0 per-half-sweep launches, 1 fused as measured fastest (default),
    2 one fused launch per pass, 3 two per pass (True / False map to 1 / 0)."""
    _check(_lib.dis_set_refine_fusion(handle, int(mode)), handle)


def dis_set_work_queue(handle, on):
    """Work scheduling: True hands search patches and forward-backward densification tiles out
    from the handle's work queue (default), False uses a fixed grid stride; both give the same
    flow bit for bit."""
    _check(_lib.dis_set_work_queue(handle, int(bool(on))), handle)


def dis_set_probe(handle, kind, level=0):
    """Record events around launch group (kind name or number, level) in every later call."""
    k = LAUNCH_KINDS.index(kind) if isinstance(kind, str) else kind
    _check(_lib.dis_set_probe(handle, k, level), handle)


def dis_probe_ms(handle):
    """Device time (ms) of the probed launch group in the most recent call."""
    ms = _f()
    _check(_lib.dis_probe_ms(handle, ctypes.byref(ms)), handle)
    return ms.value


def dis_get_tuning(handle, patch_size):
    """(search variant, refinement launch form) the handle uses for this patch size."""
    v, r = _i(), _i()
    _check(_lib.dis_get_tuning(handle, patch_size, ctypes.byref(v), ctypes.byref(r)), handle)
    return v.value, r.value


def dis_set_refine_split(handle, pixels):
    """Refinement form 1 splits passes of launches above `pixels` (< 0: never)."""
    _check(_lib.dis_set_refine_split(handle, pixels), handle)


def dis_get_refine_split(handle):
    """Split threshold of refinement form 1 (-1: never split)."""
    v = _i64()
    _check(_lib.dis_get_refine_split(handle, ctypes.byref(v)), handle)
    return v.value


def dis_last_call_kernels(handle):
    """Kernels the most recent call on the handle launched (its graph's kernel nodes; -1 when it
    ran without a graph)."""
    c = _i()
    _check(_lib.dis_last_call_kernels(handle, ctypes.byref(c)), handle)
    return c.value


def dis_search_variants(patch_size):
    """Lanes-per-patch variants of the search for this patch size (the default first)."""
    out = (_i * 8)()
    n = _lib.dis_search_variants(patch_size, out, 8)
    return [out[k] for k in range(n)]


def dis_search_mode_variants(patch_size):
    """Group widths of the stereo and robust-norm searches for this patch size (default first)."""
    out = (_i * 8)()
    n = _lib.dis_search_mode_variants(patch_size, out, 8)
    return [out[k] for k in range(n)]


def dis_set_search_variant(handle, patch_size, lanes):
    """Pin the search variant of the handle for this patch size."""
    _check(_lib.dis_set_search_variant(handle, patch_size, lanes), handle)


def dis_pyr_down(inp, w, h, in_pitch, out, out_pitch, stream=None):
    _check(_lib.dis_pyr_down(_ptr(inp), w, h, in_pitch, _ptr(out), out_pitch, _stream(stream)))


def dis_sobel(inp, w, h, pitch, gx, gy, out_pitch, stream=None):
    _check(_lib.dis_sobel(_ptr(inp), w, h, pitch, _ptr(gx), _ptr(gy), out_pitch, _stream(stream)))


def dis_search_level(I0, I1, w, h, pitch, Uc, wc, hc, cscale, ps, stride, iters, u_out, uinit_out=None,
                     status_out=None, stream=None):
    _check(_lib.dis_search_level(_ptr(I0), _ptr(I1), w, h, pitch, _ptr(Uc), wc, hc, cscale, ps, stride, iters,
                                 _ptr(u_out), _ptr(uinit_out), _ptr(status_out), _stream(stream)))


def dis_search_level_ex(I0, I1, w, h, pitch, Uc, wc, hc, cscale, ps, stride, iters, variant, u_out, uinit_out=None,
                        status_out=None, stream=None):
    _check(_lib.dis_search_level_ex(_ptr(I0), _ptr(I1), w, h, pitch, _ptr(Uc), wc, hc, cscale, ps, stride, iters,
                                    variant, _ptr(u_out), _ptr(uinit_out), _ptr(status_out), _stream(stream)))


def dis_densify_level(I0, I1, w, h, pitch, u, ps, stride, Uc, wc, hc, cscale, U_out, stream=None):
    _check(_lib.dis_densify_level(_ptr(I0), _ptr(I1), w, h, pitch, _ptr(u), ps, stride, _ptr(Uc), wc, hc, cscale,
                                  _ptr(U_out), _stream(stream)))


def dis_densify_level_fb(handle, I0, I1, w, h, pitch, u, ub, ps, stride, U_out, Ub_out, stream=None):
    """Both directions' dense fields with forward-backward consistency (handle scratch)."""
    _check(_lib.dis_densify_level_fb(handle, _ptr(I0), _ptr(I1), w, h, pitch, _ptr(u), _ptr(ub), ps, stride,
                                     _ptr(U_out), _ptr(Ub_out), _stream(stream)), handle)


def dis_search_level_ex2(I0, I1, w, h, pitch, Uc, wc, hc, cscale, ps, stride, iters, variant, dof, norm, huber_b,
                         u_out, uinit_out=None, status_out=None, stream=None, term_eps=0.0):
    """dis_search_level_ex with the degrees of freedom (1 stereo, 2 flow), the error norm (0 L2,
    1 L1, 2 Huber with threshold huber_b) and early termination (term_eps > 0)."""
    _check(_lib.dis_search_level_ex2(_ptr(I0), _ptr(I1), w, h, pitch, _ptr(Uc), wc, hc, cscale, ps, stride, iters,
                                     variant, dof, NORMS.get(norm, norm), huber_b, term_eps, _ptr(u_out),
                                     _ptr(uinit_out), _ptr(status_out), _stream(stream)))


def dis_refine_level_ex(handle, I0, I1, w, h, pitch, channels, U, outer, inner, delta=5.0, gamma=10.0, alpha=10.0,
                        omega=1.6, dof=2, stream=None):
    """dis_refine_level with the degrees of freedom (1: stereo, v kept)."""
    _check(_lib.dis_refine_level_ex(handle, _ptr(I0), _ptr(I1), w, h, pitch, channels, _ptr(U), outer, inner, delta,
                                    gamma, alpha, omega, dof, _stream(stream)), handle)


def dis_refine_level(handle, I0, I1, w, h, pitch, channels, U, outer, inner, delta=5.0, gamma=10.0, alpha=10.0,
                     omega=1.6, stream=None):
    _check(_lib.dis_refine_level(handle, _ptr(I0), _ptr(I1), w, h, pitch, channels, _ptr(U), outer, inner, delta,
                                 gamma, alpha, omega, _stream(stream)), handle)


def dis_upsample_flow(Uin, wi, hi, factor, Uout, wo, ho, stream=None):
    _check(_lib.dis_upsample_flow(_ptr(Uin), wi, hi, factor, _ptr(Uout), wo, ho, _stream(stream)))


DIS_NOALLOC_SCRATCH_FLOATS = 1 << 22


def dis_refine_level_noalloc(I0, I1, w, h, pitch, channels, U, outer, inner, delta=5.0, gamma=10.0, alpha=10.0,
                             omega=1.6, stream=None):
    """dis_refine_level without a handle: scratch is the library's fixed device array
    (for callers that cannot allocate device memory; see include/dis.h)."""
    _check(_lib.dis_refine_level_noalloc(_ptr(I0), _ptr(I1), w, h, pitch, channels, _ptr(U), outer, inner, delta,
                                         gamma, alpha, omega, _stream(stream)))


def dis_photometric_loss_scratch_bytes(w, h, pitch, channels=1):
    return _lib.dis_photometric_loss_scratch_bytes(w, h, pitch, channels)


def dis_photometric_loss(I0, I1, w, h, pitch, channels, flow, eps, loss_out, grad_flow, grad_I0, grad_I1, scratch,
                         scratch_bytes, stream=None):
    _check(_lib.dis_photometric_loss(_ptr(I0), _ptr(I1), w, h, pitch, channels, _ptr(flow), eps, _ptr(loss_out),
                                     _ptr(grad_flow), _ptr(grad_I0), _ptr(grad_I1), _ptr(scratch), scratch_bytes,
                                     _stream(stream)))


def dis_backward_workspace_bytes(w, h, params):
    return _lib.dis_backward_workspace_bytes(w, h, ctypes.byref(params))


def dis_replay_flow(handle, I0, I1, w, h, pitch, params, init_flow, frozen, flow_out, workspace, workspace_bytes,
                    stream=None):
    _check(_lib.dis_replay_flow(handle, _ptr(I0), _ptr(I1), w, h, pitch, ctypes.byref(params), _ptr(init_flow),
                                _ptr(frozen), _ptr(flow_out), _ptr(workspace), workspace_bytes, _stream(stream)), handle)


def dis_backward(handle, I0, I1, w, h, pitch, params, init_flow, frozen, grad_flow, grad_I0, grad_I1, grad_pitch,
                 grad_init_flow, workspace, workspace_bytes, stream=None):
    _check(_lib.dis_backward(handle, _ptr(I0), _ptr(I1), w, h, pitch, ctypes.byref(params), _ptr(init_flow),
                             _ptr(frozen), _ptr(grad_flow), _ptr(grad_I0), _ptr(grad_I1), grad_pitch,
                             _ptr(grad_init_flow), _ptr(workspace), workspace_bytes, _stream(stream)), handle)
