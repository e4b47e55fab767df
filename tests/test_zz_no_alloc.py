"""The allocation-free path-traced render.

Callers that may not allocate device memory (a plugin whose host application
owns the device heap, a latency-critical loop that must not call cudaMalloc)
use eagpt_render_path_traced_noalloc(), which takes its workspace from a
scratch array compiled into the library.  Here it is called through the C ABI
twice in a row and each result is compared with the regular entry point's,
which renders into a caller-allocated workspace, within the radiance
tolerance the parity tests use.  The file is named to be collected last so a
run that stops at the first failure has run every other test already; it
also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2601_23065_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_render_twice():
    import torch

    from paper_2601_23065_gb300 import api, build, capi
    build.build()
    L = capi.lib()
    scene = S.tiny_room(4096)
    cam = S.horizontal_camera(64, 48, hfov=100.0)
    ds = api.DeviceScene.from_host(scene)
    bvh = api.BVH(ds)
    prm = api.params()
    c = api.camera(cam)
    sc = ds.c()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    spp, B, rr, seed = 8, 3, 2, 11

    # regular entry point, caller-allocated workspace
    ws_bytes = L.eagpt_render_workspace_bytes(ctypes.byref(c), spp, 1)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    ref = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    capi.check(L.eagpt_render_path_traced(ctypes.byref(sc), ctypes.byref(bvh.c()), ctypes.byref(c),
                                          ctypes.byref(prm), spp, B, rr, ctypes.c_uint64(seed),
                                          ctypes.c_void_p(ref.data_ptr()), None, None, None,
                                          ctypes.c_void_p(ws.data_ptr()), ws_bytes, stream))
    ref_np = ref.cpu().numpy().astype(np.float64)
    assert ref_np.max() > 0

    assert L.eagpt_render_path_traced_noalloc_max_bytes() >= L.eagpt_render_workspace_min_bytes(
        ctypes.byref(c), spp, 1)
    for _ in range(2):
        out = torch.full((cam.height, cam.width, 3), -1.0, dtype=torch.float32, device="cuda")
        capi.check(L.eagpt_render_path_traced_noalloc(ctypes.byref(sc), ctypes.byref(bvh.c()), ctypes.byref(c),
                                                      ctypes.byref(prm), spp, B, rr, ctypes.c_uint64(seed),
                                                      ctypes.c_void_p(out.data_ptr()), stream))
        capi.check(L.eagpt_sync_status(stream))
        got = out.cpu().numpy().astype(np.float64)
        bound = 1e-4 * np.maximum(np.abs(ref_np), 1e-3 * np.abs(ref_np).mean())
        assert np.all(np.abs(got - ref_np) <= bound)

    # a render too large for the scratch is refused with a clear message
    big = api.camera(S.horizontal_camera(4096, 4096))
    st = L.eagpt_render_path_traced_noalloc(ctypes.byref(sc), ctypes.byref(bvh.c()), ctypes.byref(big),
                                            ctypes.byref(prm), spp, B, rr, ctypes.c_uint64(seed),
                                            ctypes.c_void_p(out.data_ptr()), stream)
    assert st == 1 and b"scratch" in L.eagpt_last_error()
