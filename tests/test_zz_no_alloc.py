"""The allocation-free path-traced render.

Callers that may not allocate device memory (a plugin whose host application
owns the device heap, a latency-critical loop that must not call cudaMalloc)
use eagpt_render_path_traced_noalloc(), which takes its workspace from a
scratch array compiled into the library.  Results do not depend on how many
samples a render pass holds, so each call must equal the regular entry point
(caller-allocated workspace) bit for bit.  Here it is called through the C ABI
twice in a row, with a render of another seed in between so that the second
call starts from a scratch full of that render's data, for a camera that
renders several samples per pass, one that fits only one sample per pass, and
one with emitter sampling; a render too large for the scratch (the emitter-
sampling layout at the limit included) is refused.  The file is named to be
collected last so a run that stops at the first failure has run every other
test already; it also passes on its own in a fresh process.
"""
import ctypes

import pytest

from paper_2601_23065_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _setup():
    from paper_2601_23065_gb300 import api, build, capi
    build.build()
    L = capi.lib()
    scene = S.tiny_room(4096)
    ds = api.DeviceScene.from_host(scene)
    bvh = api.BVH(ds)
    return api, capi, L, ds, bvh


def _regular(api, capi, L, ds, bvh, cam, prm, spp, B, rr, seed, stream):
    import torch
    c = api.camera(cam)
    kind = 2 if prm.flags & capi.FLAG_EMITTER_SAMPLING else 1
    ws_bytes = L.eagpt_render_workspace_bytes(ctypes.byref(c), spp, kind)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    ref = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    capi.check(L.eagpt_render_path_traced(ctypes.byref(ds.c()), ctypes.byref(bvh.c()), ctypes.byref(c),
                                          ctypes.byref(prm), spp, B, rr, ctypes.c_uint64(seed),
                                          ctypes.c_void_p(ref.data_ptr()), None, None, None,
                                          ctypes.c_void_p(ws.data_ptr()), ws_bytes, stream))
    capi.check(L.eagpt_sync_status(stream))
    return ref


def _noalloc(api, capi, L, ds, bvh, cam, prm, spp, B, rr, seed, stream):
    import torch
    out = torch.full((cam.height, cam.width, 3), -1.0, dtype=torch.float32, device="cuda")
    capi.check(L.eagpt_render_path_traced_noalloc(ctypes.byref(ds.c()), ctypes.byref(bvh.c()),
                                                  ctypes.byref(api.camera(cam)), ctypes.byref(prm), spp, B, rr,
                                                  ctypes.c_uint64(seed), ctypes.c_void_p(out.data_ptr()), stream))
    capi.check(L.eagpt_sync_status(stream))
    return out


@pytest.mark.parametrize("case", ["several_per_pass", "one_per_pass", "emitter_sampling"])
def test_noalloc_equals_regular_render_twice(case):
    import torch
    api, capi, L, ds, bvh = _setup()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if case == "several_per_pass":
        cam, prm, spp = S.horizontal_camera(320, 240, hfov=100.0), api.params(), 8
    elif case == "one_per_pass":
        cam, prm, spp = S.horizontal_camera(400, 300, hfov=100.0), api.params(), 3
    else:
        cam, prm, spp = S.horizontal_camera(160, 120, hfov=100.0), api.params(flags=capi.FLAG_EMITTER_SAMPLING), 4
    B, rr, seed = 3, 2, 11
    c = api.camera(cam)
    kind = 2 if case == "emitter_sampling" else 1
    scratch = L.eagpt_render_path_traced_noalloc_max_bytes()
    assert L.eagpt_render_workspace_min_bytes(ctypes.byref(c), spp, kind) <= scratch
    if case == "one_per_pass":  # a pass of two samples does not fit
        assert L.eagpt_render_workspace_bytes(ctypes.byref(c), 2, kind) > scratch
    elif case == "several_per_pass":
        assert L.eagpt_render_workspace_bytes(ctypes.byref(c), spp, kind) > scratch
    ref = _regular(api, capi, L, ds, bvh, cam, prm, spp, B, rr, seed, stream)
    assert float(ref.max()) > 0
    first = _noalloc(api, capi, L, ds, bvh, cam, prm, spp, B, rr, seed, stream)
    assert torch.equal(first, ref)
    # another render leaves its own data in the shared scratch
    other = _noalloc(api, capi, L, ds, bvh, cam, prm, spp, B, rr, seed + 1, stream)
    assert not torch.equal(other, ref)
    second = _noalloc(api, capi, L, ds, bvh, cam, prm, spp, B, rr, seed, stream)
    assert torch.equal(second, ref)


def test_noalloc_refuses_renders_larger_than_its_scratch():
    import torch
    api, capi, L, ds, bvh = _setup()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = torch.empty((4, 4, 3), dtype=torch.float32, device="cuda")
    scratch = L.eagpt_render_path_traced_noalloc_max_bytes()
    # far too large
    big = api.camera(S.horizontal_camera(4096, 4096))
    st = L.eagpt_render_path_traced_noalloc(ctypes.byref(ds.c()), ctypes.byref(bvh.c()), ctypes.byref(big),
                                            ctypes.byref(api.params()), 4, 3, 2, ctypes.c_uint64(1),
                                            ctypes.c_void_p(out.data_ptr()), stream)
    assert st == 1 and b"scratch" in L.eagpt_last_error()
    # fits the plain layout but not the emitter-sampling one (two more queues)
    cam = api.camera(S.horizontal_camera(480, 320))
    assert L.eagpt_render_workspace_min_bytes(ctypes.byref(cam), 4, 1) <= scratch
    assert L.eagpt_render_workspace_min_bytes(ctypes.byref(cam), 4, 2) > scratch
    prm = api.params(flags=capi.FLAG_EMITTER_SAMPLING)
    st = L.eagpt_render_path_traced_noalloc(ctypes.byref(ds.c()), ctypes.byref(bvh.c()), ctypes.byref(cam),
                                            ctypes.byref(prm), 4, 3, 2, ctypes.c_uint64(1),
                                            ctypes.c_void_p(out.data_ptr()), stream)
    assert st == 1 and b"scratch" in L.eagpt_last_error()
    capi.check(L.eagpt_sync_status(stream))
