"""CPU tests of the C-ABI library: it loads, exports every entry point include/dis.h declares,
and its host logic (presets, stride and level arithmetic, argument checks) agrees with the
oracle's readings.  No call here reaches the GPU."""
import ctypes
import os
import re

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dis():
    from paper_1603_03590_gb300 import build
    build.build()
    from paper_1603_03590_gb300 import dis as d
    return d


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dis.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dis_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(dis):
    names = declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(dis.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_header_compiles_as_plain_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "dis.h"\nint main(void){dis_params p; dis_default_params(&p, 0); return p.patch_size != 8;}\n')
    import subprocess
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-c", str(src), "-I", os.path.join(ROOT, "include"),
                        "-o", str(tmp_path / "t.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_presets_match_paper_operating_points(dis):
    import json
    gv = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_values.json")))
    for k, (sf, it, ps, ov) in enumerate(gv["operating_points"]["points"], start=1):
        p = dis.dis_default_params(k)
        assert (p.finest_scale, p.grad_iters, p.patch_size) == (sf, it, ps)
        assert abs(p.overlap - ov) < 1e-6
        assert p.refine == (0 if k == 1 else 1)
    p = dis.dis_default_params()
    assert (p.delta, p.gamma, p.alpha, p.var_inner, p.var_outer) == (5.0, 10.0, 10.0, 5, -1)
    assert p.struct_size == ctypes.sizeof(dis.dis_params)


@pytest.mark.parametrize("W,H", [(1024, 436), (640, 480), (128, 96), (3840, 2160), (320, 240), (1920, 1080),
                                 (13, 9), (8, 8), (1242, 375), (173, 91)])
@pytest.mark.parametrize("preset", ["op1", "op2", "op3", "op4", "fast", "medium", "dense"])
def test_levels_and_patch_counts_match_oracle(dis, W, H, preset):
    p = dis.dis_default_params(preset)
    q = oracle.params(patch_size=p.patch_size, overlap=round(p.overlap, 6), grad_iters=p.grad_iters,
                      finest_scale=p.finest_scale, refine=p.refine)
    rc, ss, sf = oracle.levels(W, H, q)
    if rc != 0:
        with pytest.raises(dis.DisError) as e:
            dis.dis_levels(W, H, p)
        assert e.value.status == dis.DIS_ERR_TOO_SMALL
        return
    gss, gsf, tot = dis.dis_levels(W, H, p)
    assert (gss, gsf) == (ss, sf)
    assert tot == oracle.total_patches(W, H, q)


def test_host_side_errors_need_no_gpu(dis):
    p = dis.dis_default_params()
    lib = dis._lib
    assert lib.dis_compute_flow(None, None, None, 8, 8, 8, ctypes.byref(p), None, None) == dis.DIS_ERR_INVALID_ARG
    assert lib.dis_search_level(None, None, 8, 8, 8, None, 0, 0, 2.0, 8, 4, 4, None, None, None, None) == \
        dis.DIS_ERR_INVALID_ARG
    assert "dis_search_level" in dis.dis_last_error_string(None)
    h = ctypes.c_void_p()
    assert lib.dis_create(ctypes.byref(h), 0, 10, 1, 1) == dis.DIS_ERR_INVALID_ARG and not h.value
    assert lib.dis_create(ctypes.byref(h), 10, 10, 1, 2) == dis.DIS_ERR_INVALID_ARG
    bad = dis.dis_default_params()
    bad.struct_size = 4
    with pytest.raises(dis.DisError):
        dis.dis_levels(100, 100, bad)
    for field, val in [("patch_size", 1), ("patch_size", 17), ("overlap", 1.0), ("overlap", -0.1), ("sor_omega", 2.0),
                       ("channels", 2), ("grad_iters", -1), ("alpha", float("nan"))]:
        q = dis.dis_default_params()
        setattr(q, field, val)
        with pytest.raises(dis.DisError) as e:
            dis.dis_levels(100, 100, q)
        assert e.value.status == dis.DIS_ERR_INVALID_ARG, field
    with pytest.raises(dis.DisError) as e:
        dis.dis_levels(7, 7, dis.dis_default_params(coarsest_scale=0))
    assert e.value.status == dis.DIS_ERR_TOO_SMALL
    lib.dis_destroy(None)


def test_stride_reading_matches_oracle_for_decimal_overlaps(dis):
    for ps in range(2, 17):
        for k in range(0, 100):
            ov = k / 100.0
            p = dis.dis_default_params(patch_size=ps, overlap=ov, coarsest_scale=0, finest_scale=0)
            q = oracle.params(patch_size=ps, overlap=ov, coarsest_scale=0, finest_scale=0)
            W = H = 64
            assert dis.dis_levels(W, H, p)[2] == oracle.total_patches(W, H, q), (ps, ov)


def test_search_variants_are_listed_without_a_gpu(dis):
    assert dis.dis_search_variants(8) == [8, 4, 1, 102, 104, 108]
    assert dis.dis_search_variants(12) == [16, 8, 1, 102, 104]
    for ps in range(2, 17):
        v = dis.dis_search_variants(ps)
        assert v[0] == (8 if ps <= 8 else 16) and 1 in v and len(set(v)) == len(v), ps
    assert dis.dis_search_variants(1) == [] and dis.dis_search_variants(17) == []
    lib = ctypes.CDLL(dis.LIB_PATH)
    assert lib.dis_search_variants(12, None, 0) == 5
    assert lib.dis_set_search_variant(None, 12, 1) == dis.DIS_ERR_INVALID_ARG


def test_trace_and_probe_argument_checks_need_no_gpu(dis):
    lib = ctypes.CDLL(dis.LIB_PATH)
    assert lib.dis_set_probe(None, 3, 0) == dis.DIS_ERR_INVALID_ARG
    assert lib.dis_set_refine_fusion(None, 1) == dis.DIS_ERR_INVALID_ARG
    assert lib.dis_set_work_queue(None, 1) == dis.DIS_ERR_INVALID_ARG
    assert lib.dis_set_refine_split(None, ctypes.c_int64(1)) == dis.DIS_ERR_INVALID_ARG
    assert lib.dis_get_refine_split(None, None) == dis.DIS_ERR_INVALID_ARG
    assert lib.dis_last_call_kernels(None, None) == dis.DIS_ERR_INVALID_ARG
    assert lib.dis_get_tuning(None, 8, None, None) == dis.DIS_ERR_INVALID_ARG
    assert lib.dis_probe_ms(None, None) == dis.DIS_ERR_INVALID_ARG
    assert lib.dis_trace_batched(None, None, 1, None, None, None, 0, None) == dis.DIS_ERR_INVALID_ARG
    assert dis.LAUNCH_KINDS.index("search") == 3 and len(dis.LAUNCH_KINDS) == 7


def test_host_buffer_call_argument_checks_need_no_gpu(dis):
    lib = ctypes.CDLL(dis.LIB_PATH)
    assert lib.dis_compute_flow_batched_host(None, None, 1, None, None) == dis.DIS_ERR_INVALID_ARG
    assert lib.dis_host_flows_ready(None, None) == dis.DIS_ERR_INVALID_ARG


def test_frames_beyond_32_bit_pixel_indexing_are_refused(dis):
    lib = ctypes.CDLL(dis.LIB_PATH)
    h = ctypes.c_void_p()
    assert lib.dis_create(ctypes.byref(h), 65536, 32768, 1, 1) == dis.DIS_ERR_INVALID_ARG and not h.value
    assert lib.dis_pyr_down(ctypes.c_void_p(16), 65536, 32768, ctypes.c_int64(65536), ctypes.c_void_p(16),
                            ctypes.c_int64(32768), None) == dis.DIS_ERR_INVALID_ARG


def test_refinement_size_checks_cannot_wrap(dis):
    """A pitch so large that (15 C + 8) * pitch * h wraps 64 bits must still be refused before
    any work is enqueued (the pointers are never dereferenced)."""
    lib = ctypes.CDLL(dis.LIB_PATH)
    fake = ctypes.c_void_p(256)
    for pitch, h in [(1 << 62, 4), (1 << 40, 1 << 24), ((1 << 31) + 5, 2), ((1 << 22) + 1, 1)]:
        st = lib.dis_refine_level_noalloc(fake, fake, 8, h, ctypes.c_int64(pitch), 1, fake, 1, 1, ctypes.c_float(5.0),
                                          ctypes.c_float(10.0), ctypes.c_float(10.0), ctypes.c_float(1.6), None)
        assert st == dis.DIS_ERR_INVALID_ARG, (pitch, h)
        assert "scratch" in dis.dis_last_error_string(None)


def test_bench_preset_table_matches_the_library(dis):
    """bench.py builds the oracle's parameters of its CPU legs from a plain table (so that those
    legs load no product code); the table must hold the library's preset values."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    for name, vals in bench.PRESETS.items():
        p = dis.dis_default_params(name)
        for k, v in vals.items():
            assert abs(getattr(p, k) - v) < 1e-6, (name, k, getattr(p, k), v)
    p = dis.dis_default_params("default", **bench.DIFF_PARAMS)
    assert (p.patch_size, p.var_outer, p.var_inner, p.coarsest_scale) == (8, 1, 10, 3)
