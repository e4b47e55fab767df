"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every symbol declared in include/eagpt.h; argument checks that need no
device memory reject bad input.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "eagpt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eagpt_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_23065_gb300 import build, capi
    build.build()
    return capi.lib()


def test_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert len(syms) >= 10
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_signatures_cover_header(lib):
    from paper_2601_23065_gb300 import capi
    assert set(declared_symbols()) <= set(capi.SIGNATURES), set(declared_symbols()) - set(capi.SIGNATURES)


def test_defaults_and_sizes(lib):
    from paper_2601_23065_gb300 import capi
    p = capi.default_params()
    assert abs(p.tau_E - 0.1) < 1e-7 and p.support_sigma == 3.0 and p.flags == 0
    assert lib.eagpt_bvh_bytes(0) > 0
    assert lib.eagpt_bvh_bytes(1000) > 1000 * 64
    assert lib.eagpt_bvh_bytes(-1) == 0
    cam = capi.Camera(64, 64, 32.0, 32.0, 32.0, 32.0)
    a = lib.eagpt_render_workspace_bytes(ctypes.byref(cam), 4, 1)
    b = lib.eagpt_render_workspace_min_bytes(ctypes.byref(cam), 4, 1)
    assert a >= b > 64 * 64 * 48


def test_host_argument_checks(lib):
    from paper_2601_23065_gb300 import capi
    p = capi.default_params()
    out = capi.Bvh()
    assert lib.eagpt_build_bvh(None, ctypes.byref(p), None, 0, ctypes.byref(out), None) == 1
    sc = capi.Scene()
    sc.n = 5  # pointers NULL
    assert lib.eagpt_build_bvh(ctypes.byref(sc), ctypes.byref(p), None, 0, ctypes.byref(out), None) == 1
    assert b"pos" in lib.eagpt_last_error()
    sc.n = -3
    assert lib.eagpt_build_bvh(ctypes.byref(sc), ctypes.byref(p), None, 0, ctypes.byref(out), None) == 1
    bad = capi.default_params()
    bad.T_min = 0.0
    sc.n = 0
    assert lib.eagpt_build_bvh(ctypes.byref(sc), ctypes.byref(bad), None, 0, ctypes.byref(out), None) == 1
    bad = capi.default_params()
    bad.flags = 2
    assert lib.eagpt_build_bvh(ctypes.byref(sc), ctypes.byref(bad), None, 0, ctypes.byref(out), None) == 1
    # stale BVH: version mismatch is refused before anything is launched
    cam = capi.Camera(8, 8, 4.0, 4.0, 4.0, 4.0)
    bvh = capi.Bvh()
    bvh.n, bvh.scene_version, bvh.support_sigma = 0, 3, 3.0
    sc.version = 4
    rgb = ctypes.c_void_p(16)
    st = lib.eagpt_render_path_traced(ctypes.byref(sc), ctypes.byref(bvh), ctypes.byref(cam), ctypes.byref(p), 4, 2,
                                      2, 0, rgb, None, None, None, ctypes.c_void_p(256), 1 << 20, None)
    assert st == 4
    sc.version = 3
    st = lib.eagpt_render_path_traced(ctypes.byref(sc), ctypes.byref(bvh), ctypes.byref(cam), ctypes.byref(p), 0, 2,
                                      2, 0, rgb, None, None, None, ctypes.c_void_p(256), 1 << 20, None)
    assert st == 1 and b"spp" in lib.eagpt_last_error()
    st = lib.eagpt_render_path_traced(ctypes.byref(sc), ctypes.byref(bvh), ctypes.byref(cam), ctypes.byref(p), 4, 99,
                                      2, 0, rgb, None, None, None, ctypes.c_void_p(256), 1 << 20, None)
    assert st == 1
    st = lib.eagpt_render_path_traced(ctypes.byref(sc), ctypes.byref(bvh), ctypes.byref(cam), ctypes.byref(p), 4, 2,
                                      2, 0, rgb, None, None, None, ctypes.c_void_p(256), 16, None)
    assert st == 2  # workspace too small


def test_sample_cache_argument_checks(lib):
    """The forward-to-adjoint cache: its size, and the checks made before
    any launch (missing or misaligned cache, stale BVH)."""
    from paper_2601_23065_gb300 import capi
    cam = capi.Camera(8, 6, 4.0, 4.0, 4.0, 3.0)
    assert lib.eagpt_single_bounce_cache_bytes(ctypes.byref(cam), 5) == 8 * 6 * 5 * 16
    assert lib.eagpt_single_bounce_cache_bytes(ctypes.byref(cam), 0) == 0
    assert lib.eagpt_single_bounce_cache_bytes(None, 4) == 0
    p = capi.default_params()
    sc = capi.Scene()
    sc.n, sc.version = 0, 3
    bvh = capi.Bvh()
    bvh.n, bvh.scene_version, bvh.support_sigma = 0, 3, 3.0
    rgb, ws = ctypes.c_void_p(256), ctypes.c_void_p(512)
    fwd = lib.eagpt_render_single_bounce_cached
    assert fwd(ctypes.byref(sc), ctypes.byref(bvh), ctypes.byref(cam), ctypes.byref(p), 4, 0, rgb, None, ws, 1 << 20,
               None) == 1
    assert b"sample_cache" in lib.eagpt_last_error()
    assert fwd(ctypes.byref(sc), ctypes.byref(bvh), ctypes.byref(cam), ctypes.byref(p), 4, 0, rgb, ctypes.c_void_p(8),
               ws, 1 << 20, None) == 1
    sc.version = 4  # the BVH was built for version 3
    assert fwd(ctypes.byref(sc), ctypes.byref(bvh), ctypes.byref(cam), ctypes.byref(p), 4, 0, rgb,
               ctypes.c_void_p(1024), ws, 1 << 20, None) == 4
    g = capi.SceneGrad()
    bwd = lib.eagpt_render_single_bounce_backward_cached
    assert bwd(ctypes.byref(sc), ctypes.byref(bvh), ctypes.byref(cam), ctypes.byref(p), 4, 0, rgb, None,
               ctypes.byref(g), ws, 1 << 20, None) == 1
    assert b"sample_cache" in lib.eagpt_last_error()


def test_level_of_detail_argument_checks(lib):
    """The level-of-detail entry points: workspace size, the checks made
    before any launch (grid, capacity, emitter sampling, lod_from, stale
    merged BVH), and an empty scene, which merges to nothing without a
    launch."""
    from paper_2601_23065_gb300 import capi
    assert lib.eagpt_lod_workspace_bytes(1000) >= 1000 * 4 * 7
    assert lib.eagpt_lod_workspace_bytes(-1) == 0
    p = capi.default_params()
    sc = capi.Scene()
    out = capi.Scene()
    org = (ctypes.c_float * 3)(0.0, 0.0, 0.0)
    cnt = ctypes.c_int64(-1)
    ws = ctypes.c_void_p(256)
    build = lib.eagpt_build_lod
    for h in (0.0, -1.0, float("inf"), float("nan"), 1e-45):
        assert build(ctypes.byref(sc), ctypes.byref(p), org, h, ctypes.byref(out), None, ctypes.byref(cnt), ws,
                     1 << 20, None) == 1
        assert b"cell_size" in lib.eagpt_last_error()
    bad = (ctypes.c_float * 3)(0.0, float("inf"), 0.0)
    assert build(ctypes.byref(sc), ctypes.byref(p), bad, 0.1, ctypes.byref(out), None, ctypes.byref(cnt), ws,
                 1 << 20, None) == 1
    assert build(ctypes.byref(sc), ctypes.byref(p), org, 0.1, ctypes.byref(out), None, None, ws, 1 << 20, None) == 1
    assert build(ctypes.byref(sc), ctypes.byref(p), org, 0.1, ctypes.byref(out), None, ctypes.byref(cnt), ws,
                 1 << 20, None) == 0
    assert cnt.value == 0
    buf = (ctypes.c_float * 64)()
    addr = ctypes.addressof(buf)
    for k in ("pos", "quat", "scale", "opacity", "albedo", "radiance", "emissive"):
        setattr(sc, k, addr)
    sc.n, out.n = 5, 4
    assert build(ctypes.byref(sc), ctypes.byref(p), org, 0.1, ctypes.byref(out), None, ctypes.byref(cnt), ws,
                 1 << 20, None) == 2
    assert b"capacity" in lib.eagpt_last_error()
    # render
    sc.n = 0
    sc.version = 3
    lsc = capi.Scene()
    lsc.version = 7
    bvh, lbvh = capi.Bvh(), capi.Bvh()
    bvh.n, bvh.scene_version, bvh.support_sigma = 0, 3, 3.0
    lbvh.n, lbvh.scene_version, lbvh.support_sigma = 0, 6, 3.0
    cam = capi.Camera(8, 8, 4.0, 4.0, 4.0, 4.0)
    rgb = ctypes.c_void_p(256)
    render = lib.eagpt_render_path_traced_lod

    def call(prm, lod_from):
        return render(ctypes.byref(sc), ctypes.byref(bvh), ctypes.byref(lsc), ctypes.byref(lbvh), lod_from,
                      ctypes.byref(cam), ctypes.byref(prm), 0, 4, 3, 2, 0, rgb, None, None, None, ws, 1 << 20, None)

    mis = capi.default_params()
    mis.flags = capi.FLAG_EMITTER_SAMPLING
    assert call(mis, 2) == 6
    assert call(p, 0) == 1 and b"lod_from" in lib.eagpt_last_error()
    assert call(p, 2) == 4  # the merged BVH was built for another version of the merged scene
