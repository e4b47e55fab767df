"""Python front end of the C ABI.

PyTorch supplies device memory and streams; every computation runs in the
CUDA library (``libeagpt.so``).  Names follow the paper: a scene of surfels
with centre p, rotation q, scales s, opacity sigma, albedo rho, radiance r and
emissive term e (Sec. 3.1); renders by the single-bounce estimator (Eq. 6) and
by path tracing (Eq. 8).
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import capi
from .scenes import Camera as HostCamera
from .scenes import SurfelScene

FIELDS = ("pos", "quat", "scale", "opacity", "albedo", "radiance", "emissive")
GRAD_FIELDS = ("pos", "quat", "scale", "opacity", "albedo", "radiance")
SHAPES = {"pos": 3, "quat": 4, "scale": 2, "opacity": 1, "albedo": 3, "radiance": 3, "emissive": 1}


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def params(**overrides) -> capi.Params:
    """Method constants (defaults: tau_E = 0.1 from Eq. 4; the rest are the
    stated readings of unstated constants)."""
    p = capi.default_params()
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def camera(cam: HostCamera) -> capi.Camera:
    c = capi.Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c2w = np.asarray(cam.c2w, np.float32).reshape(12)
    for i in range(12):
        c.c2w[i] = float(c2w[i])
    return c


class DeviceScene:
    """Surfel parameters resident on the device (structure of arrays)."""

    def __init__(self, tensors: dict, version: int = 0):
        n = tensors["pos"].shape[0]
        for k in FIELDS:
            t = tensors[k]
            want = (n, SHAPES[k]) if SHAPES[k] > 1 else (n,)
            if tuple(t.shape) != want or t.dtype != torch.float32 or not t.is_contiguous() or not t.is_cuda:
                raise ValueError(f"{k}: want contiguous CUDA float32 {want}, got {t.dtype} {tuple(t.shape)}")
        self.t = dict(tensors)
        self.n = n
        self.version = int(version)

    @classmethod
    def from_host(cls, scene: SurfelScene, device="cuda", non_blocking=False):
        return cls({k: torch.as_tensor(getattr(scene, k)).to(device, non_blocking=non_blocking).contiguous()
                    for k in FIELDS})

    def to_host(self) -> SurfelScene:
        return SurfelScene(*[self.t[k].cpu().numpy() for k in FIELDS])

    def c(self) -> capi.Scene:
        s = capi.Scene()
        s.n = self.n
        for k in FIELDS:
            setattr(s, k, self.t[k].data_ptr() if self.n else None)
        s.version = self.version
        return s


class BVH:
    """Software LBVH over the surfels' support bounds; storage is a torch
    uint8 buffer owned by this object."""

    def __init__(self, scene: DeviceScene, prm: Optional[capi.Params] = None, stream=None):
        self.params = prm or params()
        nbytes = capi.lib().eagpt_bvh_bytes(scene.n)
        self.storage = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=scene.t["pos"].device)
        self.handle = capi.Bvh()
        sc = scene.c()
        capi.check(capi.lib().eagpt_build_bvh(ctypes.byref(sc), ctypes.byref(self.params),
                                               _ptr(self.storage), self.storage.numel(),
                                               ctypes.byref(self.handle), _stream(stream)))

    def c(self) -> capi.Bvh:
        return self.handle


class Renderer:
    """Holds a reusable device workspace and calls the render entry points."""

    def __init__(self, device="cuda", max_workspace_bytes: Optional[int] = None):
        self.device = torch.device(device)
        self.ws = None
        self.max_ws = max_workspace_bytes

    def _workspace(self, cam: capi.Camera, spp: int, kind: int) -> torch.Tensor:
        want = capi.lib().eagpt_render_workspace_bytes(ctypes.byref(cam), spp, kind)
        if self.max_ws is not None:
            want = max(min(want, self.max_ws), capi.lib().eagpt_render_workspace_min_bytes(ctypes.byref(cam), spp, kind))
        if self.ws is None or self.ws.numel() < want:
            self.ws = None
            self.ws = torch.empty(want, dtype=torch.uint8, device=self.device)
        return self.ws

    def path_traced(self, scene: DeviceScene, bvh: BVH, cam: HostCamera, spp: int, max_bounces: int,
                    rr_start: int = 2, seed: int = 0, prm: Optional[capi.Params] = None, want_aux=False,
                    want_samples=False, want_stats=False, out: Optional[torch.Tensor] = None, stream=None,
                    first_sample: int = 0):
        """Eq. 8 render; returns dict(rgb (H,W,3)[, aux (H,W,12)][, samples (H,W,spp,3)][, stats]).
        With ``prm.flags`` containing capi.FLAG_EMITTER_SAMPLING the path
        tracer samples emitters at every reflection (MIS).  ``first_sample``
        > 0 renders samples first_sample .. first_sample + spp - 1 of each
        pixel (a slice of a longer frame, same paths as in the full render)."""
        c = camera(cam)
        prm = prm or bvh.params
        ws = self._workspace(c, spp, 2 if prm.flags & capi.FLAG_EMITTER_SAMPLING else 1)
        H, W = cam.height, cam.width
        rgb = out if out is not None else torch.empty((H, W, 3), dtype=torch.float32, device=self.device)
        aux = torch.empty((H, W, 12), dtype=torch.float32, device=self.device) if want_aux else None
        smp = torch.empty((H, W, spp, 3), dtype=torch.float32, device=self.device) if want_samples else None
        st = torch.zeros(16, dtype=torch.int64, device=self.device) if want_stats else None
        sc = scene.c()
        if first_sample:
            capi.check(capi.lib().eagpt_render_path_traced_range(
                ctypes.byref(sc), ctypes.byref(bvh.c()), ctypes.byref(c), ctypes.byref(prm), int(first_sample),
                int(spp), int(max_bounces), int(rr_start), ctypes.c_uint64(int(seed)), _ptr(rgb), _ptr(aux),
                _ptr(smp), _ptr(st), _ptr(ws), ws.numel(), _stream(stream)))
        else:
            capi.check(capi.lib().eagpt_render_path_traced(
                ctypes.byref(sc), ctypes.byref(bvh.c()), ctypes.byref(c), ctypes.byref(prm), int(spp),
                int(max_bounces), int(rr_start), ctypes.c_uint64(int(seed)), _ptr(rgb), _ptr(aux), _ptr(smp),
                _ptr(st), _ptr(ws), ws.numel(), _stream(stream)))
        r = {"rgb": rgb}
        if want_aux:
            r["aux"] = aux
        if want_samples:
            r["samples"] = smp
        if want_stats:
            r["stats"] = st
        return r

    def path_traced_lod(self, scene: DeviceScene, bvh: BVH, lod: "LevelOfDetail", lod_from: int, cam: HostCamera,
                        spp: int, max_bounces: int, rr_start: int = 2, seed: int = 0,
                        prm: Optional[capi.Params] = None, want_samples=False, want_stats=False,
                        out: Optional[torch.Tensor] = None, stream=None, first_sample: int = 0):
        """Eq. 8 render whose bounce segments k >= lod_from trace the merged
        surfels of ``lod``; returns dict(rgb[, samples][, stats])."""
        c = camera(cam)
        prm = prm or bvh.params
        ws = self._workspace(c, spp, 1)
        H, W = cam.height, cam.width
        rgb = out if out is not None else torch.empty((H, W, 3), dtype=torch.float32, device=self.device)
        smp = torch.empty((H, W, spp, 3), dtype=torch.float32, device=self.device) if want_samples else None
        st = torch.zeros(16, dtype=torch.int64, device=self.device) if want_stats else None
        capi.check(capi.lib().eagpt_render_path_traced_lod(
            ctypes.byref(scene.c()), ctypes.byref(bvh.c()), ctypes.byref(lod.scene.c()), ctypes.byref(lod.bvh.c()),
            int(lod_from), ctypes.byref(c), ctypes.byref(prm), int(first_sample), int(spp), int(max_bounces),
            int(rr_start), ctypes.c_uint64(int(seed)), _ptr(rgb), None, _ptr(smp), _ptr(st), _ptr(ws), ws.numel(),
            _stream(stream)))
        r = {"rgb": rgb}
        if want_samples:
            r["samples"] = smp
        if want_stats:
            r["stats"] = st
        return r

    def segments(self, stream=None):
        """(primary, secondary) segments traced by this renderer's last render
        (synchronises the stream)."""
        out = (ctypes.c_int64 * 2)()
        capi.check(capi.lib().eagpt_render_segments(_ptr(self.ws), ctypes.cast(out, ctypes.c_void_p), _stream(stream)))
        return int(out[0]), int(out[1])

    def single_bounce(self, scene: DeviceScene, bvh: BVH, cam: HostCamera, spp: int, seed: int = 0,
                      prm: Optional[capi.Params] = None, want_aux=False, want_samples=False, want_cache=False,
                      stream=None):
        """Eq. 6 render; returns dict(rgb[, aux][, samples][, cache]).  With
        ``want_cache`` the render also keeps each sample's secondary R and T
        (16 bytes per sample) for single_bounce_backward(cache=...), which
        then skips one traversal per secondary segment."""
        c = camera(cam)
        prm = prm or bvh.params
        ws = self._workspace(c, spp, 0)
        H, W = cam.height, cam.width
        rgb = torch.empty((H, W, 3), dtype=torch.float32, device=self.device)
        if want_cache:
            if want_aux or want_samples:
                raise ValueError("the cached render writes no aux or sample output")
            L = capi.lib()
            cache = torch.empty(L.eagpt_single_bounce_cache_bytes(ctypes.byref(c), spp) // 4, dtype=torch.float32,
                                device=self.device)
            sc = scene.c()
            capi.check(L.eagpt_render_single_bounce_cached(
                ctypes.byref(sc), ctypes.byref(bvh.c()), ctypes.byref(c), ctypes.byref(prm), int(spp),
                ctypes.c_uint64(int(seed)), _ptr(rgb), _ptr(cache), _ptr(ws), ws.numel(), _stream(stream)))
            return {"rgb": rgb, "cache": cache}
        aux = torch.empty((H, W, 12), dtype=torch.float32, device=self.device) if want_aux else None
        smp = torch.empty((H, W, spp, 3), dtype=torch.float32, device=self.device) if want_samples else None
        sc = scene.c()
        capi.check(capi.lib().eagpt_render_single_bounce(
            ctypes.byref(sc), ctypes.byref(bvh.c()), ctypes.byref(c), ctypes.byref(prm), int(spp),
            ctypes.c_uint64(int(seed)), _ptr(rgb), _ptr(aux), _ptr(smp), _ptr(ws), ws.numel(), _stream(stream)))
        r = {"rgb": rgb}
        if want_aux:
            r["aux"] = aux
        if want_samples:
            r["samples"] = smp
        return r


def build_lod(scene: DeviceScene, origin, cell_size: float, prm: Optional[capi.Params] = None, stream=None,
              want_keys=False):
    """Merged surfels of the level of detail (eagpt_build_lod): returns
    (DeviceScene of the merged surfels[, keys int64 tensor]).  Synchronises
    the stream once (the group count is read back)."""
    prm = prm or params()
    dev = scene.t["pos"].device
    n = scene.n
    out = {k: torch.empty((n, SHAPES[k]) if SHAPES[k] > 1 else (n,), dtype=torch.float32, device=dev)
           for k in FIELDS}
    keys = torch.empty(n, dtype=torch.int64, device=dev) if want_keys else None
    ws = torch.empty(max(capi.lib().eagpt_lod_workspace_bytes(n), 256), dtype=torch.uint8, device=dev)
    o = DeviceScene(out).c()
    org = (capi.c_f * 3)(*[float(v) for v in origin])
    count = capi.c_i64(0)
    capi.check(capi.lib().eagpt_build_lod(ctypes.byref(scene.c()), ctypes.byref(prm), org, float(cell_size),
                                          ctypes.byref(o), _ptr(keys), ctypes.byref(count), _ptr(ws), ws.numel(),
                                          _stream(stream)))
    m = int(count.value)
    merged = DeviceScene({k: v[:m].contiguous() for k, v in out.items()})
    return (merged, keys[:m]) if want_keys else merged


class LevelOfDetail:
    """Merged surfels (build_lod) and their BVH, for path_traced_lod."""

    def __init__(self, scene: DeviceScene, origin, cell_size: float, prm: Optional[capi.Params] = None,
                 stream=None):
        self.origin, self.cell_size = tuple(float(v) for v in origin), float(cell_size)
        self.scene = build_lod(scene, origin, cell_size, prm, stream)
        self.bvh = BVH(self.scene, prm, stream)

    @classmethod
    def of(cls, scene: DeviceScene, bvh: BVH) -> "LevelOfDetail":
        """A level of detail made of a given scene and its BVH."""
        lod = cls.__new__(cls)
        lod.origin, lod.cell_size, lod.scene, lod.bvh = None, None, scene, bvh
        return lod


def trace_rays(scene: DeviceScene, bvh: BVH, rays: torch.Tensor, mode: int = 0, max_hits: int = 0,
               prm: Optional[capi.Params] = None, stream=None):
    """Traces caller rays (n, 6) -> dict(rec (n,12)[, hits (n,max_hits), nhits (n,)])."""
    rays = rays.contiguous()
    n = rays.shape[0]
    dev = rays.device
    rec = torch.empty((n, 12), dtype=torch.float32, device=dev)
    hits = torch.empty((n, max_hits), dtype=torch.int32, device=dev) if max_hits > 0 else None
    nh = torch.empty((n,), dtype=torch.int32, device=dev)
    prm = prm or bvh.params
    sc = scene.c()
    capi.check(capi.lib().eagpt_trace_rays(ctypes.byref(sc), ctypes.byref(bvh.c()), ctypes.byref(prm), int(mode),
                                           _ptr(rays), n, _ptr(rec), _ptr(hits), int(max_hits), _ptr(nh),
                                           _stream(stream)))
    out = {"rec": rec, "nhits": nh}
    if hits is not None:
        out["hits"] = hits
    return out


def sync_status(stream=None) -> None:
    """Synchronise and raise if a kernel recorded a device-side error."""
    capi.check(capi.lib().eagpt_sync_status(_stream(stream)))


def single_bounce_backward(scene: DeviceScene, bvh: BVH, cam: HostCamera, spp: int, seed: int, dL_drgb: torch.Tensor,
                           grads: Optional[dict] = None, prm: Optional[capi.Params] = None, stream=None,
                           workspace: Optional[torch.Tensor] = None, cache: Optional[torch.Tensor] = None) -> dict:
    """Adjoint of the single-bounce render: accumulates dL/dtheta for
    L = sum(dL_drgb * image) into ``grads`` (created zeroed if None).
    ``cache``: the per-sample cache of a single_bounce(want_cache=True) render
    with the same scene, BVH, camera, spp, seed and params."""
    dev = scene.t["pos"].device
    if grads is None:
        grads = {k: torch.zeros_like(scene.t[k]) for k in GRAD_FIELDS}
    g = capi.SceneGrad()
    g.n = scene.n
    for k in GRAD_FIELDS:
        setattr(g, k, grads[k].data_ptr() if scene.n else None)
    c = camera(cam)
    prm = prm or bvh.params
    L = capi.lib()
    need = L.eagpt_render_backward_workspace_bytes(ctypes.byref(c), spp)
    ws = workspace if workspace is not None and workspace.numel() >= need else torch.empty(
        need, dtype=torch.uint8, device=dev)
    dL = dL_drgb.contiguous().to(torch.float32)
    sc = scene.c()
    if cache is not None:
        capi.check(L.eagpt_render_single_bounce_backward_cached(
            ctypes.byref(sc), ctypes.byref(bvh.c()), ctypes.byref(c), ctypes.byref(prm), int(spp),
            ctypes.c_uint64(int(seed)), _ptr(dL), _ptr(cache), ctypes.byref(g), _ptr(ws), ws.numel(),
            _stream(stream)))
        return grads
    capi.check(L.eagpt_render_single_bounce_backward(ctypes.byref(sc), ctypes.byref(bvh.c()), ctypes.byref(c),
                                                     ctypes.byref(prm), int(spp), ctypes.c_uint64(int(seed)),
                                                     _ptr(dL), ctypes.byref(g), _ptr(ws), ws.numel(),
                                                     _stream(stream)))
    return grads


class _SingleBounceFn(torch.autograd.Function):
    """Differentiable single-bounce render (Eq. 6): forward and hand-written
    adjoint both run in the CUDA library; PyTorch only carries the tensors."""

    @staticmethod
    def forward(ctx, pos, quat, scale, opacity, albedo, radiance, emissive, cam, spp, seed, renderer, prm):
        ds = DeviceScene({"pos": pos.detach().contiguous(), "quat": quat.detach().contiguous(),
                          "scale": scale.detach().contiguous(), "opacity": opacity.detach().contiguous(),
                          "albedo": albedo.detach().contiguous(), "radiance": radiance.detach().contiguous(),
                          "emissive": emissive.detach().contiguous()})
        bvh = BVH(ds, prm)
        out = renderer.single_bounce(ds, bvh, cam, spp, seed=seed, prm=prm, want_cache=True)
        ctx.state = (ds, bvh, cam, spp, seed, prm, out["cache"])
        return out["rgb"]

    @staticmethod
    def backward(ctx, grad_rgb):
        ds, bvh, cam, spp, seed, prm, cache = ctx.state
        g = single_bounce_backward(ds, bvh, cam, spp, seed, grad_rgb, prm=prm, cache=cache)
        return (g["pos"], g["quat"], g["scale"], g["opacity"], g["albedo"], g["radiance"], None, None, None, None,
                None, None)


def render_single_bounce(tensors: dict, cam: HostCamera, spp: int, seed: int = 0,
                         renderer: Optional[Renderer] = None, prm: Optional[capi.Params] = None) -> torch.Tensor:
    """Autograd entry point: ``tensors`` maps the scene fields to CUDA float32
    tensors (any of them may require grad); returns the (H, W, 3) image.  The
    emissive term gets no gradient (it enters only through threshold tests)."""
    renderer = renderer or Renderer(device=tensors["pos"].device)
    prm = prm or params()
    return _SingleBounceFn.apply(tensors["pos"], tensors["quat"], tensors["scale"], tensors["opacity"],
                                 tensors["albedo"], tensors["radiance"], tensors["emissive"], cam, spp, seed,
                                 renderer, prm)


def radiance(scene: DeviceScene, bvh: BVH, cam: HostCamera, prm: Optional[capi.Params] = None, want_aux=False,
             stream=None) -> dict:
    """0-bounce render of the radiant scene: per pixel the blended radiance R
    of its primary segment; returns dict(rgb[, aux])."""
    dev = scene.t["pos"].device
    c = camera(cam)
    prm = prm or bvh.params
    H, W = cam.height, cam.width
    rgb = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    aux = torch.empty((H, W, 12), dtype=torch.float32, device=dev) if want_aux else None
    sc = scene.c()
    capi.check(capi.lib().eagpt_render_radiance(ctypes.byref(sc), ctypes.byref(bvh.c()), ctypes.byref(c),
                                                ctypes.byref(prm), _ptr(rgb), _ptr(aux), _stream(stream)))
    r = {"rgb": rgb}
    if want_aux:
        r["aux"] = aux
    return r


def radiance_backward(scene: DeviceScene, bvh: BVH, cam: HostCamera, dL_drgb: torch.Tensor,
                      grads: Optional[dict] = None, prm: Optional[capi.Params] = None, stream=None) -> dict:
    """Adjoint of :func:`radiance`: accumulates dL/dtheta for
    L = sum(dL_drgb * R) into ``grads`` (created zeroed if None)."""
    if grads is None:
        grads = {k: torch.zeros_like(scene.t[k]) for k in GRAD_FIELDS}
    g = capi.SceneGrad()
    g.n = scene.n
    for k in GRAD_FIELDS:
        setattr(g, k, grads[k].data_ptr() if scene.n else None)
    c = camera(cam)
    prm = prm or bvh.params
    dL = dL_drgb.contiguous().to(torch.float32)
    sc = scene.c()
    capi.check(capi.lib().eagpt_render_radiance_backward(ctypes.byref(sc), ctypes.byref(bvh.c()), ctypes.byref(c),
                                                         ctypes.byref(prm), _ptr(dL), ctypes.byref(g),
                                                         _stream(stream)))
    return grads


class _RadianceFn(torch.autograd.Function):
    """Differentiable 0-bounce render; forward and adjoint run in the CUDA
    library."""

    @staticmethod
    def forward(ctx, pos, quat, scale, opacity, albedo, radiance_, emissive, cam, prm):
        ds = DeviceScene({"pos": pos.detach().contiguous(), "quat": quat.detach().contiguous(),
                          "scale": scale.detach().contiguous(), "opacity": opacity.detach().contiguous(),
                          "albedo": albedo.detach().contiguous(), "radiance": radiance_.detach().contiguous(),
                          "emissive": emissive.detach().contiguous()})
        bvh = BVH(ds, prm)
        out = radiance(ds, bvh, cam, prm=prm)
        ctx.state = (ds, bvh, cam, prm)
        return out["rgb"]

    @staticmethod
    def backward(ctx, grad_rgb):
        ds, bvh, cam, prm = ctx.state
        g = radiance_backward(ds, bvh, cam, grad_rgb, prm=prm)
        return (g["pos"], g["quat"], g["scale"], g["opacity"], g["albedo"], g["radiance"], None, None, None)


def render_radiance(tensors: dict, cam: HostCamera, prm: Optional[capi.Params] = None) -> torch.Tensor:
    """Autograd entry point of the 0-bounce render (radiant scene, Sec. 3.2)."""
    prm = prm or params()
    return _RadianceFn.apply(tensors["pos"], tensors["quat"], tensors["scale"], tensors["opacity"],
                             tensors["albedo"], tensors["radiance"], tensors["emissive"], cam, prm)


# ---------------------------------------------------------------------------
# optimisation of the shading parameters (Stage 1, Eq. 7; light baking, Eq. 10)
# ---------------------------------------------------------------------------
FIELDS_OPT = {"albedo": 0, "radiance": 1}


def single_bounce_incident(scene: DeviceScene, bvh: BVH, cam: HostCamera, spp: int, seed: int = 0,
                           renderer: Optional[Renderer] = None, prm: Optional[capi.Params] = None,
                           stream=None) -> dict:
    """Single-bounce render plus the per-pixel incident radiance estimate
    L_i = mean_s R(w_s); returns dict(rgb, li)."""
    renderer = renderer or Renderer(device=scene.t["pos"].device)
    c = camera(cam)
    prm = prm or bvh.params
    ws = renderer._workspace(c, spp, 0)
    H, W = cam.height, cam.width
    rgb = torch.empty((H, W, 3), dtype=torch.float32, device=renderer.device)
    li = torch.empty((H, W, 3), dtype=torch.float32, device=renderer.device)
    sc = scene.c()
    capi.check(capi.lib().eagpt_render_single_bounce_incident(
        ctypes.byref(sc), ctypes.byref(bvh.c()), ctypes.byref(c), ctypes.byref(prm), int(spp),
        ctypes.c_uint64(int(seed)), _ptr(rgb), _ptr(li), _ptr(ws), ws.numel(), _stream(stream)))
    return {"rgb": rgb, "li": li}


def shading_backward(scene: DeviceScene, bvh: BVH, cam: HostCamera, field: str, dL_drgb: torch.Tensor,
                     li: Optional[torch.Tensor] = None, grad: Optional[torch.Tensor] = None,
                     prm: Optional[capi.Params] = None, stream=None) -> torch.Tensor:
    """Gradient (n, 3), accumulated into ``grad``, of sum(dL_drgb * image) with
    respect to the albedo (single-bounce image; needs ``li``) or the radiance
    (0-bounce image)."""
    if grad is None:
        grad = torch.zeros((scene.n, 3), dtype=torch.float32, device=scene.t["pos"].device)
    c = camera(cam)
    prm = prm or bvh.params
    dL = dL_drgb.contiguous().to(torch.float32)
    lic = li.contiguous() if li is not None else None
    sc = scene.c()
    capi.check(capi.lib().eagpt_render_shading_backward(ctypes.byref(sc), ctypes.byref(bvh.c()), ctypes.byref(c),
                                                        ctypes.byref(prm), FIELDS_OPT[field], _ptr(dL), _ptr(lic),
                                                        _ptr(grad), _stream(stream)))
    return grad


def pq_l1_loss(pred: torch.Tensor, target: torch.Tensor, peak: float = 100.0, lambda_c: float = 1.0,
               want_grad: bool = True, stream=None):
    """(loss (device float64 scalar tensor), dL/dpred or None) of
    lambda_c * mean |PQ(pred / peak) - PQ(target / peak)|."""
    pred = pred.contiguous()
    target = target.contiguous()
    n = pred.numel()
    dev = pred.device
    L = capi.lib()
    scratch = torch.empty(max(L.eagpt_pq_l1_scratch_bytes(n) // 8, 1), dtype=torch.float64, device=dev)
    loss = torch.empty((), dtype=torch.float64, device=dev)
    grad = torch.empty_like(pred) if want_grad else None
    capi.check(L.eagpt_pq_l1_loss(_ptr(pred), _ptr(target), n, float(peak), float(lambda_c), _ptr(grad), _ptr(loss),
                                  _ptr(scratch), scratch.numel() * 8, _stream(stream)))
    return loss, grad


def adam_config(lr=0.01, beta1=0.9, beta2=0.999, eps=1e-8, lo=-float("inf"), hi=float("inf")) -> capi.Adam:
    a = capi.Adam()
    a.lr, a.beta1, a.beta2, a.eps, a.lo, a.hi = lr, beta1, beta2, eps, lo, hi
    return a


def adam_step(param: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, step: int,
              cfg: Optional[capi.Adam] = None, zero_grad: bool = False, stream=None) -> None:
    """One Adam step t = step, in place on contiguous float32 tensors."""
    cfg = cfg or adam_config()
    capi.check(capi.lib().eagpt_adam_step(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(),
                                          ctypes.byref(cfg), int(step), int(zero_grad), _stream(stream)))


class ShadingFit:
    """The native optimisation loop (eagpt_fit) over one field: 'albedo'
    (Stage 1, Eq. 7, single-bounce render at ``spp``) or 'radiance' (light
    baking, Eq. 10, 0-bounce render).  Keeps the Adam moments, the step count
    and the workspace between calls."""

    def __init__(self, scene: DeviceScene, bvh: BVH, cams, targets, field: str, spp: int = 1, seed: int = 0,
                 peak: float = 100.0, lambda_c: float = 1.0, adam: Optional[capi.Adam] = None):
        self.scene, self.bvh = scene, bvh
        self.cfg = capi.FitConfig()
        self.cfg.field = FIELDS_OPT[field]
        self.cfg.spp = int(spp)
        self.cfg.seed = int(seed)
        self.cfg.peak = float(peak)
        self.cfg.lambda_c = float(lambda_c)
        if adam is None:
            adam = adam_config(lr=0.01, lo=0.0, hi=1.0) if field == "albedo" else adam_config(lr=0.01, lo=0.0)
        self.cfg.adam = adam
        self.cams = (capi.Camera * len(cams))(*[camera(c) for c in cams])
        self.targets = [t.contiguous().to(torch.float32) for t in targets]
        self.tptrs = (ctypes.c_void_p * len(cams))(*[t.data_ptr() for t in self.targets])
        dev = scene.t["pos"].device
        self.m = torch.zeros((scene.n, 3), dtype=torch.float32, device=dev)
        self.v = torch.zeros((scene.n, 3), dtype=torch.float32, device=dev)
        self.step = 0
        need = capi.lib().eagpt_fit_workspace_bytes(ctypes.byref(self.cfg), self.cams, len(cams), scene.n)
        self.ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)

    def run(self, iters: int, view_order=None, stream=None) -> torch.Tensor:
        """Runs ``iters`` steps; returns the per-step losses (device float64)."""
        dev = self.scene.t["pos"].device
        losses = torch.empty(max(iters, 1), dtype=torch.float64, device=dev)
        order = None
        if view_order is not None:
            order = (ctypes.c_int32 * iters)(*[int(x) for x in view_order])
        sm = self.scene.c()
        capi.check(capi.lib().eagpt_fit(ctypes.byref(self.cfg), ctypes.byref(sm), ctypes.byref(self.bvh.handle),
                                        ctypes.byref(self.bvh.params), self.cams, self.tptrs, len(self.targets),
                                        order, int(self.step), int(iters), _ptr(self.m), _ptr(self.v),
                                        _ptr(losses), _ptr(self.ws), self.ws.numel(), _stream(stream)))
        self.scene.version = int(sm.version)
        self.step += iters
        return losses[:iters]


EDIT_OPS = {"set_emission": 0, "toggle_emission": 1, "scale_albedo": 2, "translate": 3, "rigid": 4}


def select(scene: DeviceScene, shape: str, values, stream=None) -> torch.Tensor:
    """Indices (int32, increasing) of the surfels whose centre lies in a box
    (values = lo3 + hi3) or a sphere (values = centre3 + (radius,))."""
    dev = scene.t["pos"].device
    sh = {"box": 0, "sphere": 1}[shape]
    v = (ctypes.c_float * 6)(*[float(x) for x in list(values) + [0.0] * (6 - len(values))])
    L = capi.lib()
    scratch = torch.empty(max(L.eagpt_select_scratch_bytes(scene.n), 4), dtype=torch.uint8, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    cap = scene.n
    out = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    sc = scene.c()
    capi.check(L.eagpt_select(ctypes.byref(sc), sh, v, _ptr(out), cap, _ptr(count), _ptr(scratch), scratch.numel(),
                              _stream(stream)))
    return out[:int(count.item())]


def apply_edit(scene: DeviceScene, bvh: BVH, op: str, idx: torch.Tensor, value=(), per_index=None,
               rebuild_ratio: float = 1.5, stream=None) -> bool:
    """Applies an edit in place (see eagpt_apply_edit); returns True when the
    BVH was rebuilt instead of refit.  Bumps scene.version."""
    L = capi.lib()
    idx = idx.to(torch.int32).contiguous()
    e = capi.Edit()
    e.op = EDIT_OPS[op]
    e.reserved = 0
    e.count = idx.numel()
    e.idx = idx.data_ptr() if idx.numel() else None
    pi = per_index.to(torch.float32).contiguous() if per_index is not None else None
    e.per_index = pi.data_ptr() if pi is not None else None
    vals = list(value) + [0.0] * (16 - len(value))
    for k in range(16):
        e.value[k] = float(vals[k])
    sm = scene.c()
    rebuilt = ctypes.c_int32(0)
    capi.check(L.eagpt_apply_edit(ctypes.byref(sm), ctypes.byref(bvh.handle), ctypes.byref(bvh.params),
                                  ctypes.byref(e), float(rebuild_ratio), ctypes.byref(rebuilt), _stream(stream)))
    scene.version = int(sm.version)
    return bool(rebuilt.value)


def delete_surfels(scene: DeviceScene, bvh: BVH, idx: torch.Tensor, stream=None) -> int:
    """Removes the listed surfels, keeping the others in order
    (eagpt_delete_surfels); the scene's tensors become views of their first n
    rows and the BVH is rebuilt.  Returns the new surfel count."""
    L = capi.lib()
    dev = scene.t["pos"].device
    idx = idx.to(device=dev, dtype=torch.int32).contiguous()
    scratch = torch.empty(max(L.eagpt_delete_scratch_bytes(scene.n), 256), dtype=torch.uint8, device=dev)
    sm = scene.c()
    capi.check(L.eagpt_delete_surfels(ctypes.byref(sm), ctypes.byref(bvh.handle), ctypes.byref(bvh.params),
                                      _ptr(idx), idx.numel(), _ptr(scratch), scratch.numel(), _stream(stream)))
    scene.n, scene.version = int(sm.n), int(sm.version)
    scene.t = {k: v[:scene.n] for k, v in scene.t.items()}
    return scene.n


def insert_surfels(scene: DeviceScene, bvh: BVH, src: DeviceScene, stream=None) -> int:
    """Appends the surfels of ``src`` (eagpt_insert_surfels) and rebuilds the
    BVH; the scene's tensors and the BVH storage are reallocated first when
    they are too small.  Returns the new surfel count."""
    L = capi.lib()
    n, m = scene.n, src.n
    cap = n + m
    for k in FIELDS:
        t = scene.t[k]
        if t.untyped_storage().nbytes() // 4 < cap * SHAPES[k] or t.storage_offset() != 0:
            grown = torch.empty((cap,) + tuple(t.shape[1:]), dtype=torch.float32, device=t.device)
            grown[:n].copy_(t[:n])
            scene.t[k] = grown
        else:
            scene.t[k] = t.as_strided((cap,) + tuple(t.shape[1:]), t.stride())
    need = L.eagpt_bvh_bytes(cap)
    if bvh.storage.numel() < need:
        bvh.storage = torch.empty(need, dtype=torch.uint8, device=bvh.storage.device)
        bvh.handle.storage = bvh.storage.data_ptr()
        bvh.handle.bytes = bvh.storage.numel()
    sm = scene.c()
    srcc = src.c()
    capi.check(L.eagpt_insert_surfels(ctypes.byref(sm), cap, ctypes.byref(srcc), ctypes.byref(bvh.handle),
                                      ctypes.byref(bvh.params), _stream(stream)))
    scene.n, scene.version = int(sm.n), int(sm.version)
    return scene.n


class Server:
    """Continuous-batching request loop (eagpt_server_*): renders and edits
    are submitted from any thread; the library's own thread batches them."""

    def __init__(self, scene: DeviceScene, bvh: BVH, queue_paths: int = 1 << 24, max_active: int = 16,
                 arena_bytes: Optional[int] = None, rebuild_ratio: float = 1.5):
        L = capi.lib()
        need = L.eagpt_server_arena_bytes(scene.n, queue_paths)
        self.arena = torch.empty(arena_bytes or need, dtype=torch.uint8, device=scene.t["pos"].device)
        cfg = capi.ServerConfig()
        cfg.arena = self.arena.data_ptr()
        cfg.arena_bytes = self.arena.numel()
        cfg.queue_paths = int(queue_paths)
        cfg.max_active = int(max_active)
        cfg.rebuild_ratio = float(rebuild_ratio)
        self.scene, self.bvh = scene, bvh
        self.h = ctypes.c_void_p()
        sm = scene.c()
        capi.check(L.eagpt_server_create(ctypes.byref(sm), ctypes.byref(bvh.handle), ctypes.byref(bvh.params),
                                         ctypes.byref(cfg), ctypes.byref(self.h)))
        self._keep = {}
        self.device = scene.t["pos"].device

    def submit_render(self, cam: HostCamera, spp: int, max_bounces: int, rr_start: int = 2, seed: int = 0,
                      out: Optional[torch.Tensor] = None, timeout_s: float = 0.0):
        """Returns (request id, output tensor written when the request is done)."""
        out = out if out is not None else torch.empty((cam.height, cam.width, 3), dtype=torch.float32,
                                                       device=self.device)
        r = capi.RenderRequest()
        r.cam = camera(cam)
        r.spp, r.max_bounces, r.rr_start_bounce = int(spp), int(max_bounces), int(rr_start)
        r.seed = int(seed)
        r.out_rgb = out.data_ptr()
        r.timeout_s = float(timeout_s)
        rid = ctypes.c_uint64()
        capi.check(capi.lib().eagpt_server_submit_render(self.h, ctypes.byref(r), ctypes.byref(rid)))
        self._keep[rid.value] = (out,)
        return rid.value, out

    def submit_edit(self, op: str, idx: torch.Tensor, value=(), per_index: Optional[torch.Tensor] = None) -> int:
        idx = idx.to(torch.int32).contiguous()
        pi = per_index.to(torch.float32).contiguous() if per_index is not None else None
        e = capi.Edit()
        e.op = EDIT_OPS[op]
        e.reserved = 0
        e.count = idx.numel()
        e.idx = idx.data_ptr() if idx.numel() else None
        e.per_index = pi.data_ptr() if pi is not None else None
        vals = list(value) + [0.0] * (16 - len(value))
        for k in range(16):
            e.value[k] = float(vals[k])
        torch.cuda.current_stream(self.device).synchronize()  # the edit's inputs are ready before the server reads them
        rid = ctypes.c_uint64()
        capi.check(capi.lib().eagpt_server_submit_edit(self.h, ctypes.byref(e), ctypes.byref(rid)))
        self._keep[rid.value] = (idx, pi)
        return rid.value

    @staticmethod
    def _info(i: "capi.RequestInfo") -> dict:
        return {"state": capi.REQ_STATES.get(i.state, i.state), "rebuilt": bool(i.rebuilt), "t_submit": i.t_submit,
                "t_admit": i.t_admit, "t_done": i.t_done, "scene_version": i.scene_version}

    def poll(self, rid: int) -> dict:
        i = capi.RequestInfo()
        capi.check(capi.lib().eagpt_server_poll(self.h, ctypes.c_uint64(rid), ctypes.byref(i)))
        return self._info(i)

    def wait(self, rid: int, timeout_s: float = 0.0) -> dict:
        i = capi.RequestInfo()
        capi.check(capi.lib().eagpt_server_wait(self.h, ctypes.c_uint64(rid), float(timeout_s), ctypes.byref(i)))
        self._keep.pop(rid, None)
        return self._info(i)

    def cancel(self, rid: int) -> None:
        capi.check(capi.lib().eagpt_server_cancel(self.h, ctypes.c_uint64(rid)))

    def stats(self) -> dict:
        s = capi.ServerStats()
        capi.check(capi.lib().eagpt_server_get_stats(self.h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in capi.ServerStats._fields_}

    def close(self) -> None:
        if self.h:
            capi.check(capi.lib().eagpt_server_destroy(self.h))
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
