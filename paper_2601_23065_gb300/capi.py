"""ctypes declarations of the C ABI in ``include/eagpt.h``.

Argument marshalling only: every step of the render runs in the CUDA
library.  Loading fails loudly when the library has not been built; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libeagpt.so")

_lock = threading.Lock()
_lib = None

P = ctypes.POINTER
c_f = ctypes.c_float
c_i32 = ctypes.c_int32
c_i64 = ctypes.c_int64
c_u64 = ctypes.c_uint64
c_sz = ctypes.c_size_t
c_vp = ctypes.c_void_p

STATUS = {0: "EAGPT_OK", 1: "EAGPT_ERR_INVALID_ARGUMENT", 2: "EAGPT_ERR_OUT_OF_MEMORY", 3: "EAGPT_ERR_CUDA",
          4: "EAGPT_ERR_STALE_BVH", 5: "EAGPT_ERR_TIMEOUT", 6: "EAGPT_ERR_NOT_SUPPORTED",
          7: "EAGPT_ERR_DEVICE_CHECK"}


class EagptError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Scene(ctypes.Structure):
    _fields_ = [("n", c_i64), ("pos", c_vp), ("quat", c_vp), ("scale", c_vp), ("opacity", c_vp),
                ("albedo", c_vp), ("radiance", c_vp), ("emissive", c_vp), ("version", c_u64)]


SceneMut = Scene  # same memory layout (non-const pointers)


class SceneGrad(ctypes.Structure):
    _fields_ = [("n", c_i64), ("pos", c_vp), ("quat", c_vp), ("scale", c_vp), ("opacity", c_vp),
                ("albedo", c_vp), ("radiance", c_vp)]


class Camera(ctypes.Structure):
    _fields_ = [("width", c_i32), ("height", c_i32), ("fx", c_f), ("fy", c_f), ("cx", c_f), ("cy", c_f),
                ("c2w", c_f * 12)]


class Params(ctypes.Structure):
    _fields_ = [("tau_E", c_f), ("T_min", c_f), ("alpha_min", c_f), ("alpha_max", c_f),
                ("support_sigma", c_f), ("bounce_offset", c_f), ("flags", c_i32)]


class Bvh(ctypes.Structure):
    _fields_ = [("storage", c_vp), ("bytes", c_sz), ("n", c_i64), ("scene_version", c_u64),
                ("support_sigma", c_f), ("build_area", c_f)]


class Edit(ctypes.Structure):
    _fields_ = [("op", c_i32), ("reserved", c_i32), ("count", c_i64), ("idx", c_vp), ("per_index", c_vp),
                ("value", c_f * 16)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("arena", c_vp), ("arena_bytes", c_sz), ("queue_paths", c_i64), ("max_active", c_i32),
                ("rebuild_ratio", c_f)]


class RenderRequest(ctypes.Structure):
    _fields_ = [("cam", Camera), ("spp", c_i32), ("max_bounces", c_i32), ("rr_start_bounce", c_i32),
                ("seed", c_u64), ("out_rgb", c_vp), ("timeout_s", ctypes.c_double)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("state", c_i32), ("rebuilt", c_i32), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("scene_version", c_u64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", c_i64), ("admitted", c_i64), ("completed", c_i64), ("failed", c_i64),
                ("edits", c_i64), ("rebuilds", c_i64), ("waves", c_i64), ("segments", c_i64), ("paths", c_i64),
                ("busy_s", ctypes.c_double), ("arena_free_bytes", c_i64)]


class Adam(ctypes.Structure):
    _fields_ = [("lr", c_f), ("beta1", c_f), ("beta2", c_f), ("eps", c_f), ("lo", c_f), ("hi", c_f)]


class FitConfig(ctypes.Structure):
    _fields_ = [("field", c_i32), ("spp", c_i32), ("seed", c_u64), ("peak", c_f), ("lambda_c", c_f),
                ("adam", Adam)]


FLAG_EMITTER_SAMPLING = 1

REQ_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "cancelled", 5: "timed_out"}

# symbol -> (restype, argtypes)
SIGNATURES = {
    "eagpt_default_params": (None, [P(Params)]),
    "eagpt_last_error": (ctypes.c_char_p, []),
    "eagpt_version": (ctypes.c_char_p, []),
    "eagpt_bvh_bytes": (c_sz, [c_i64]),
    "eagpt_build_bvh": (c_i32, [P(Scene), P(Params), c_vp, c_sz, P(Bvh), c_vp]),
    "eagpt_render_workspace_bytes": (c_sz, [P(Camera), c_i32, c_i32]),
    "eagpt_render_workspace_min_bytes": (c_sz, [P(Camera), c_i32, c_i32]),
    "eagpt_render_single_bounce": (c_i32, [P(Scene), P(Bvh), P(Camera), P(Params), c_i32, c_u64, c_vp, c_vp,
                                           c_vp, c_vp, c_sz, c_vp]),
    "eagpt_render_path_traced": (c_i32, [P(Scene), P(Bvh), P(Camera), P(Params), c_i32, c_i32, c_i32, c_u64,
                                         c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "eagpt_render_segments": (c_i32, [c_vp, c_vp, c_vp]),
    "eagpt_render_path_traced_range": (c_i32, [P(Scene), P(Bvh), P(Camera), P(Params), c_i32, c_i32, c_i32, c_i32,
                                               c_u64, c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "eagpt_lod_workspace_bytes": (c_sz, [c_i64]),
    "eagpt_build_lod": (c_i32, [P(Scene), P(Params), P(c_f), c_f, P(Scene), c_vp, P(c_i64), c_vp, c_sz, c_vp]),
    "eagpt_render_path_traced_lod": (c_i32, [P(Scene), P(Bvh), P(Scene), P(Bvh), c_i32, P(Camera), P(Params), c_i32,
                                             c_i32, c_i32, c_i32, c_u64, c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "eagpt_trace_rays": (c_i32, [P(Scene), P(Bvh), P(Params), c_i32, c_vp, c_i64, c_vp, c_vp, c_i32, c_vp, c_vp]),
    "eagpt_select_scratch_bytes": (c_sz, [c_i64]),
    "eagpt_select": (c_i32, [P(Scene), c_i32, P(c_f), c_vp, c_i64, c_vp, c_vp, c_sz, c_vp]),
    "eagpt_apply_edit": (c_i32, [P(Scene), P(Bvh), P(Params), P(Edit), c_f, P(c_i32), c_vp]),
    "eagpt_server_arena_bytes": (c_sz, [c_i64, c_i64]),
    "eagpt_server_create": (c_i32, [P(Scene), P(Bvh), P(Params), P(ServerConfig), P(c_vp)]),
    "eagpt_server_submit_render": (c_i32, [c_vp, P(RenderRequest), P(c_u64)]),
    "eagpt_server_submit_edit": (c_i32, [c_vp, P(Edit), P(c_u64)]),
    "eagpt_server_poll": (c_i32, [c_vp, c_u64, P(RequestInfo)]),
    "eagpt_server_wait": (c_i32, [c_vp, c_u64, ctypes.c_double, P(RequestInfo)]),
    "eagpt_server_cancel": (c_i32, [c_vp, c_u64]),
    "eagpt_server_get_stats": (c_i32, [c_vp, P(ServerStats)]),
    "eagpt_server_scene": (c_i32, [c_vp, P(Scene), P(Bvh)]),
    "eagpt_server_destroy": (c_i32, [c_vp]),
    "eagpt_render_path_traced_noalloc_max_bytes": (c_sz, []),
    "eagpt_render_path_traced_noalloc": (c_i32, [P(Scene), P(Bvh), P(Camera), P(Params), c_i32, c_i32, c_i32, c_u64,
                                                 c_vp, c_vp]),
    "eagpt_render_backward_workspace_bytes": (c_sz, [P(Camera), c_i32]),
    "eagpt_render_backward_workspace_min_bytes": (c_sz, [P(Camera), c_i32]),
    "eagpt_render_single_bounce_backward": (c_i32, [P(Scene), P(Bvh), P(Camera), P(Params), c_i32, c_u64, c_vp,
                                                    P(SceneGrad), c_vp, c_sz, c_vp]),
    "eagpt_single_bounce_cache_bytes": (c_sz, [P(Camera), c_i32]),
    "eagpt_render_single_bounce_cached": (c_i32, [P(Scene), P(Bvh), P(Camera), P(Params), c_i32, c_u64, c_vp, c_vp,
                                                  c_vp, c_sz, c_vp]),
    "eagpt_render_single_bounce_backward_cached": (c_i32, [P(Scene), P(Bvh), P(Camera), P(Params), c_i32, c_u64,
                                                           c_vp, c_vp, P(SceneGrad), c_vp, c_sz, c_vp]),
    "eagpt_render_radiance": (c_i32, [P(Scene), P(Bvh), P(Camera), P(Params), c_vp, c_vp, c_vp]),
    "eagpt_render_radiance_backward": (c_i32, [P(Scene), P(Bvh), P(Camera), P(Params), c_vp, P(SceneGrad), c_vp]),
    "eagpt_render_single_bounce_incident": (c_i32, [P(Scene), P(Bvh), P(Camera), P(Params), c_i32, c_u64, c_vp,
                                                    c_vp, c_vp, c_sz, c_vp]),
    "eagpt_render_shading_backward": (c_i32, [P(Scene), P(Bvh), P(Camera), P(Params), c_i32, c_vp, c_vp, c_vp,
                                              c_vp]),
    "eagpt_pq_l1_scratch_bytes": (c_sz, [c_i64]),
    "eagpt_pq_l1_loss": (c_i32, [c_vp, c_vp, c_i64, c_f, c_f, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "eagpt_adam_step": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64, P(Adam), c_i64, c_i32, c_vp]),
    "eagpt_fit_workspace_bytes": (c_sz, [P(FitConfig), c_vp, c_i32, c_i64]),
    "eagpt_fit": (c_i32, [P(FitConfig), P(Scene), P(Bvh), P(Params), c_vp, c_vp, c_i32, c_vp, c_i64, c_i32,
                          c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "eagpt_delete_scratch_bytes": (c_sz, [c_i64]),
    "eagpt_delete_surfels": (c_i32, [P(Scene), P(Bvh), P(Params), c_vp, c_i64, c_vp, c_sz, c_vp]),
    "eagpt_insert_surfels": (c_i32, [P(Scene), c_i64, P(Scene), P(Bvh), P(Params), c_vp]),
    "eagpt_sync_status": (c_i32, [c_vp]),
    "eagpt_launch_count": (c_i64, []),
    "eagpt_profile_begin": (c_i32, []),
    "eagpt_profile_end": (c_i32, [c_vp, c_i32, P(c_i32)]),
}


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", c_i64), ("total_ms", ctypes.c_double)]


def profile_end(capacity: int = 64) -> dict:
    """Stops the launch profiler; returns {kernel: (launches, total_ms)}."""
    arr = (KernelTime * capacity)()
    n = c_i32(0)
    check(lib().eagpt_profile_end(ctypes.cast(arr, c_vp), capacity, ctypes.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(min(n.value, capacity))}


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                                   "(run __graft_entry__.build() or python -m paper_2601_23065_gb300.build)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name, None)
                if f is None:
                    continue
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(status: int) -> None:
    if status != 0:
        raise EagptError(status, lib().eagpt_last_error().decode(errors="replace"))


def default_params() -> Params:
    p = Params()
    lib().eagpt_default_params(ctypes.byref(p))
    return p
