"""FP64 brute-force oracle (ctypes binding of ``eagpt_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  It shares no code with the CUDA
path (``paper_2601_23065_gb300``), and neither imports the other; both take
their inputs from ``paper_2601_23065_gb300.scenes``, which holds no rendering
arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eagpt_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

FLAGS = {
    "support": 1 << 0, "tlo": 1 << 1, "amin": 1 << 2, "amax": 1 << 3, "order": 1 << 4,
    "tstop": 1 << 5, "emit": 1 << 6, "rr": 1 << 7, "onb": 1 << 8, "graze": 1 << 9, "cond": 1 << 10,
    "hemi": 1 << 11,
}
FP32_EPS = 2.0 ** -24


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11 + pthreads)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "eagpt_oracle.h"))):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class _Scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64)] + [(k, ctypes.POINTER(ctypes.c_double)) for k in
                                          ("pos", "quat", "scale", "opacity", "albedo", "radiance", "emissive")]


class _Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_double),
                ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("c2w", ctypes.c_double * 12)]


class _Params(ctypes.Structure):
    _fields_ = [("tau_E", ctypes.c_double), ("T_min", ctypes.c_double), ("alpha_min", ctypes.c_double),
                ("alpha_max", ctypes.c_double), ("support_sigma", ctypes.c_double),
                ("bounce_offset", ctypes.c_double), ("emitters_reflect", ctypes.c_int32),
                ("fp32_eps", ctypes.c_double), ("cond_tol", ctypes.c_double), ("mis", ctypes.c_int32)]


class _Segment(ctypes.Structure):
    _fields_ = [("N", ctypes.c_double * 3), ("D", ctypes.c_double), ("R", ctypes.c_double * 3),
                ("E", ctypes.c_double), ("P", ctypes.c_double * 3), ("A", ctypes.c_double),
                ("Nn", ctypes.c_double * 3), ("Dn", ctypes.c_double), ("n_hits", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("eR", ctypes.c_double), ("eP", ctypes.c_double),
                ("eE", ctypes.c_double), ("eN", ctypes.c_double), ("eD", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i32, i64, u32, u64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
            lib.ora_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
            lib.ora_cosine_direction.argtypes = [P(d), d, d, P(d)]
            lib.ora_trace_segment.argtypes = [P(_Scene), P(_Params), P(d), P(d), d, i32, P(_Segment), P(i32), i32]
            lib.ora_trace_rays.argtypes = [P(_Scene), P(_Params), P(d), i64, i32, P(d), P(i32), P(u32), P(i32),
                                           i32, P(d), i32]
            lib.ora_primary.argtypes = [P(_Scene), P(_Camera), P(_Params), i32, P(i32), i64, P(d), P(u32), i32]
            lib.ora_render.argtypes = [P(_Scene), P(_Camera), P(_Params), i32, i32, i32, i32, u64, P(i32), i64,
                                       P(d), P(d), P(u32), P(i64), P(d), i32]
            lib.ora_render_lod.argtypes = [P(_Scene), P(_Scene), i32, P(_Camera), P(_Params), i32, i32, i32, u64,
                                           P(i32), i64, P(d), P(d), P(u32), P(i64), P(d), i32]
            lib.ora_single_bounce_grad.argtypes = [P(_Scene), P(_Camera), P(_Params), i32, u64, P(i32), i64,
                                                   P(d), P(d), P(u32), i32, i32]
            lib.ora_light_pdf.argtypes = [P(_Scene), P(_Params), P(d), P(d), P(d)]
            lib.ora_light_pdf.restype = i32
            lib.ora_radiance_grad.argtypes = [P(_Scene), P(_Camera), P(_Params), P(i32), i64, P(d), P(d), P(u32),
                                              i32, i32]
            for f in ("ora_trace_segment", "ora_trace_rays", "ora_primary", "ora_render", "ora_render_lod",
                      "ora_single_bounce_grad", "ora_radiance_grad"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return os.cpu_count() or 1


class Params:
    """Method constants.  Defaults: tau_E = 0.1 (Eq. 4); the others are the
    stated readings of constants the paper does not give."""

    def __init__(self, tau_E=0.1, T_min=1e-3, alpha_min=1.0 / 255.0, alpha_max=0.99, support_sigma=3.0,
                 bounce_offset=1e-3, emitters_reflect=False, fp32_eps=FP32_EPS, cond_tol=2.5e-5, mis=False):
        self.tau_E, self.T_min, self.alpha_min, self.alpha_max = tau_E, T_min, alpha_min, alpha_max
        self.support_sigma, self.bounce_offset = support_sigma, bounce_offset
        self.emitters_reflect, self.fp32_eps, self.cond_tol = emitters_reflect, fp32_eps, cond_tol
        self.mis = mis

    def _c(self):
        return _Params(self.tau_E, self.T_min, self.alpha_min, self.alpha_max, self.support_sigma,
                       self.bounce_offset, 1 if self.emitters_reflect else 0, self.fp32_eps,
                       self.cond_tol if self.fp32_eps > 0 else 0.0, 1 if self.mis else 0)


class OracleScene:
    """The FP32 scene widened exactly to FP64 (and kept alive for ctypes)."""

    def __init__(self, scene, overrides=None):
        arrs = {}
        for name in ("pos", "quat", "scale", "opacity", "albedo", "radiance", "emissive"):
            a = getattr(scene, name) if overrides is None or name not in overrides else overrides[name]
            arrs[name] = np.ascontiguousarray(a, dtype=np.float64)
        self.arrays = arrs
        self.n = arrs["pos"].shape[0]
        self._c = _Scene(self.n, *[_ptr(arrs[k], ctypes.c_double) for k in
                                   ("pos", "quat", "scale", "opacity", "albedo", "radiance", "emissive")])


def _cam(camera):
    c2w = np.asarray(camera.c2w, np.float64).reshape(12)
    return _Camera(int(camera.width), int(camera.height), float(camera.fx), float(camera.fy),
                   float(camera.cx), float(camera.cy), (ctypes.c_double * 12)(*c2w))


def _oscene(scene):
    return scene if isinstance(scene, OracleScene) else OracleScene(scene)


def philox4x32_10(ctr, key):
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.ora_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def cosine_direction(n, u0, u1):
    lib = _load()
    nn = (ctypes.c_double * 3)(*[float(x) for x in n])
    o = (ctypes.c_double * 3)()
    lib.ora_cosine_direction(nn, float(u0), float(u1), o)
    return np.array(list(o))


def trace_segment(scene, O, w, t_lo=0.0, mode=0, params=None, max_hits=64):
    """One segment; returns (dict of composites, hit index list)."""
    lib = _load()
    sc = _oscene(scene)
    prm = (params or Params())._c()
    seg = _Segment()
    hits = np.full(max_hits, -1, np.int32)
    Oc = (ctypes.c_double * 3)(*[float(x) for x in O])
    wc = (ctypes.c_double * 3)(*[float(x) for x in w])
    rc = lib.ora_trace_segment(ctypes.byref(sc._c), ctypes.byref(prm), Oc, wc, float(t_lo), int(mode),
                               ctypes.byref(seg), _ptr(hits, ctypes.c_int32), max_hits)
    if rc:
        raise RuntimeError("oracle trace_segment failed")
    out = {"N": np.array(seg.N[:]), "D": seg.D, "R": np.array(seg.R[:]), "E": seg.E, "P": np.array(seg.P[:]),
           "A": seg.A, "Nn": np.array(seg.Nn[:]), "Dn": seg.Dn, "n_hits": seg.n_hits, "flags": seg.flags}
    return out, hits[:min(seg.n_hits, max_hits)]


def trace_rays(scene, rays, mode=0, params=None, max_hits=64, n_threads=None, want_dev=False):
    """rays (m, 6) origin+direction -> (rec (m,12), n_hits, flags, hit_idx
    (m,max_hits)) and, with want_dev, dev (m,12): per record column the
    largest change over the conditioning re-traces (+inf where a re-trace
    changes the blended surfel list)."""
    lib = _load()
    sc = _oscene(scene)
    rays = np.ascontiguousarray(rays, np.float64).reshape(-1, 6)
    m = rays.shape[0]
    rec = np.zeros((m, 12))
    nh = np.zeros(m, np.int32)
    fl = np.zeros(m, np.uint32)
    hi = np.full((m, max_hits), -1, np.int32)
    dev = np.zeros((m, 12)) if want_dev else None
    prm = (params or Params())._c()
    rc = lib.ora_trace_rays(ctypes.byref(sc._c), ctypes.byref(prm), _ptr(rays, ctypes.c_double), m, int(mode),
                            _ptr(rec, ctypes.c_double), _ptr(nh, ctypes.c_int32), _ptr(fl, ctypes.c_uint32),
                            _ptr(hi, ctypes.c_int32), max_hits, _ptr(dev, ctypes.c_double),
                            n_threads or default_threads())
    if rc:
        raise RuntimeError("oracle trace_rays failed")
    if want_dev:
        return rec, nh, fl, hi, dev
    return rec, nh, fl, hi


def primary(scene, camera, pixels, mode=0, params=None, n_threads=None):
    lib = _load()
    sc = _oscene(scene)
    pixels = np.ascontiguousarray(pixels, np.int32)
    rec = np.zeros((pixels.size, 12))
    fl = np.zeros(pixels.size, np.uint32)
    prm = (params or Params())._c()
    cam = _cam(camera)
    rc = lib.ora_primary(ctypes.byref(sc._c), ctypes.byref(cam), ctypes.byref(prm), int(mode),
                         _ptr(pixels, ctypes.c_int32), pixels.size, _ptr(rec, ctypes.c_double),
                         _ptr(fl, ctypes.c_uint32), n_threads or default_threads())
    if rc:
        raise RuntimeError("oracle primary failed")
    return rec, fl


def render(scene, camera, pixels, kind, spp, max_bounces=1, rr_start=2, seed=0, params=None,
           want_samples=False, n_threads=None, want_dev=False):
    """kind 'single' (Eq. 6) or 'pt' (Eq. 8).  Returns dict with rgb (m,3),
    samples (m,spp,3), sample_flags (m,spp), segments (m,) and, with
    want_dev, sample_dev (m,spp,3): per sample and channel the largest change
    over the conditioning runs (+inf where a run changes a discrete outcome
    along the path)."""
    lib = _load()
    sc = _oscene(scene)
    pixels = np.ascontiguousarray(pixels, np.int32)
    m = pixels.size
    rgb = np.zeros((m, 3))
    samples = np.zeros((m, spp, 3)) if want_samples else None
    dev = np.zeros((m, spp, 3)) if want_dev else None
    sflags = np.zeros((m, spp), np.uint32)
    segs = np.zeros(m, np.int64)
    prm = (params or Params())._c()
    cam = _cam(camera)
    k = {"single": 0, "pt": 1}[kind]
    rc = lib.ora_render(ctypes.byref(sc._c), ctypes.byref(cam), ctypes.byref(prm), k, int(spp), int(max_bounces),
                        int(rr_start), ctypes.c_uint64(int(seed)), _ptr(pixels, ctypes.c_int32), m,
                        _ptr(rgb, ctypes.c_double), _ptr(samples, ctypes.c_double), _ptr(sflags, ctypes.c_uint32),
                        _ptr(segs, ctypes.c_int64), _ptr(dev, ctypes.c_double), n_threads or default_threads())
    if rc:
        raise RuntimeError("oracle render failed")
    out = {"rgb": rgb, "samples": samples, "sample_flags": sflags, "segments": segs}
    if want_dev:
        out["sample_dev"] = dev
    return out


def render_lod(scene, lod_scene, lod_from, camera, pixels, spp, max_bounces=1, rr_start=2, seed=0, params=None,
               want_samples=False, n_threads=None, want_dev=False):
    """Path tracing (Eq. 8) whose bounce segments k >= lod_from trace
    ``lod_scene`` (the primary and earlier bounces trace ``scene``).  Returns
    the dict of ``render``."""
    lib = _load()
    sc = _oscene(scene)
    lsc = _oscene(lod_scene)
    pixels = np.ascontiguousarray(pixels, np.int32)
    m = pixels.size
    rgb = np.zeros((m, 3))
    samples = np.zeros((m, spp, 3)) if want_samples else None
    dev = np.zeros((m, spp, 3)) if want_dev else None
    sflags = np.zeros((m, spp), np.uint32)
    segs = np.zeros(m, np.int64)
    prm = (params or Params())._c()
    cam = _cam(camera)
    rc = lib.ora_render_lod(ctypes.byref(sc._c), ctypes.byref(lsc._c), int(lod_from), ctypes.byref(cam),
                            ctypes.byref(prm), int(spp), int(max_bounces), int(rr_start), ctypes.c_uint64(int(seed)),
                            _ptr(pixels, ctypes.c_int32), m, _ptr(rgb, ctypes.c_double),
                            _ptr(samples, ctypes.c_double), _ptr(sflags, ctypes.c_uint32),
                            _ptr(segs, ctypes.c_int64), _ptr(dev, ctypes.c_double), n_threads or default_threads())
    if rc:
        raise RuntimeError("oracle level-of-detail render failed")
    out = {"rgb": rgb, "samples": samples, "sample_flags": sflags, "segments": segs}
    if want_dev:
        out["sample_dev"] = dev
    return out


def single_bounce_grad(scene, camera, pixels, dL_drgb, spp, seed=0, params=None, n_threads=None, run=0):
    """Returns (grad (n,16), pixel flags).  run > 0: conditioning run r (rays
    and sigma g perturbed at FP32 scale)."""
    lib = _load()
    sc = _oscene(scene)
    pixels = np.ascontiguousarray(pixels, np.int32)
    dL = np.ascontiguousarray(dL_drgb, np.float64).reshape(pixels.size, 3)
    grad = np.zeros((sc.n, 16))
    fl = np.zeros(pixels.size, np.uint32)
    prm = (params or Params())._c()
    cam = _cam(camera)
    rc = lib.ora_single_bounce_grad(ctypes.byref(sc._c), ctypes.byref(cam), ctypes.byref(prm), int(spp),
                                    ctypes.c_uint64(int(seed)), _ptr(pixels, ctypes.c_int32), pixels.size,
                                    _ptr(dL, ctypes.c_double), _ptr(grad, ctypes.c_double),
                                    _ptr(fl, ctypes.c_uint32), n_threads or default_threads(), int(run))
    if rc:
        raise RuntimeError("oracle grad failed")
    return grad, fl


def radiance_grad(scene, camera, pixels, dL_drgb, params=None, n_threads=None, run=0):
    """Gradient of sum(dL_drgb * R_primary) (0-bounce render); returns (grad (n,16), flags).
    run > 0: conditioning run r (rays and sigma g perturbed at FP32 scale)."""
    lib = _load()
    sc = _oscene(scene)
    pixels = np.ascontiguousarray(pixels, np.int32)
    dL = np.ascontiguousarray(dL_drgb, np.float64).reshape(pixels.size, 3)
    grad = np.zeros((sc.n, 16))
    fl = np.zeros(pixels.size, np.uint32)
    prm = (params or Params())._c()
    cam = _cam(camera)
    rc = lib.ora_radiance_grad(ctypes.byref(sc._c), ctypes.byref(cam), ctypes.byref(prm),
                               _ptr(pixels, ctypes.c_int32), pixels.size, _ptr(dL, ctypes.c_double),
                               _ptr(grad, ctypes.c_double), _ptr(fl, ctypes.c_uint32), n_threads or default_threads(),
                               int(run))
    if rc:
        raise RuntimeError("oracle radiance grad failed")
    return grad, fl


def light_pdf(scene, origin, direction, params=None):
    """Solid-angle density of the emitter-sampling strategy (mis) at origin
    for a unit direction, summed over every emitter crossed (no occlusion);
    returns (pdf, number of emitters crossed)."""
    lib = _load()
    sc = _oscene(scene)
    prm = (params or Params(mis=True))._c()
    O = np.ascontiguousarray(origin, np.float64)
    w = np.ascontiguousarray(direction, np.float64)
    out = np.zeros(1)
    n = lib.ora_light_pdf(ctypes.byref(sc._c), ctypes.byref(prm), _ptr(O, ctypes.c_double),
                          _ptr(w, ctypes.c_double), _ptr(out, ctypes.c_double))
    if n < 0:
        raise RuntimeError("oracle light_pdf failed")
    return float(out[0]), int(n)


def grad_split(grad):
    """(n,16) -> dict of per-parameter gradients in the scene's layout."""
    return {"pos": grad[:, 0:3], "quat": grad[:, 3:7], "scale": grad[:, 7:9], "opacity": grad[:, 9],
            "albedo": grad[:, 10:13], "radiance": grad[:, 13:16]}
