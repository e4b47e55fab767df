"""Seeded synthetic inputs: surfel scenes and pinhole cameras.

This module only *draws* inputs. It contains none of the rendering arithmetic
(no quaternion-to-frame conversion, no ray generation, no intersection, no
compositing, no sampling), so the CUDA path and the FP64 oracle can both
consume its output without sharing any of the method's code.

Scene law (stands in for the paper's reconstructed indoor scenes, whose
datasets are not available: Blender b- scenes with 200k Gaussians, FIPT f-
scenes with 500k, Eyeful e- scenes with 1M, Sec. 4.1-4.2):

* wall surfels: uniform on each face of an axis-aligned box, count proportional
  to face area, normal = face normal, random in-plane rotation, offset along
  the normal U[-5 mm, 5 mm] (the non-zero thickness of reconstructed surfaces
  the paper notes in its appendix discussion);
* interior surfels: uniform in the box shrunk by 5 %, uniformly random
  orientation (Shoemake's uniform quaternion);
* scales log-uniform in [0.005, 0.05] m, opacity U[0.5, 1], albedo RGB
  U[0.1, 0.8]; in rooms whose wall surfels are denser than the medium room's
  (200k surfels in 5x4x3 m: 1,558 per m^2), every scale is multiplied by
  sqrt(medium density / density), so that a point of a wall is covered by as
  many surfels as in the medium room and the interior stays as transparent: a
  finer reconstruction of the same surfaces, not a denser fog (with the fixed
  scale law, the 6M-surfel layout's primary rays stop 0.14 m from the camera
  and no path reaches an emitter);
* emitters e = 1 with radiance RGB U[1, 10]; non-emitters e = 0 with a
  radiance cache RGB U[0, 0.5].

Every array is float32 and C-contiguous; quaternions are (w, x, y, z) and are
not required to be unit length by the renderer (it normalises them).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

WALL_FRACTION = 3000.0 / 4096.0  # wall : interior = 3000 : 1096 in every room
# wall surfels per m^2 of the medium room (200k surfels, 5 x 4 x 3 m box)
REF_WALL_DENSITY = round(200_000 * WALL_FRACTION) / 94.0


def scale_factor(n_wall: int, wall_area: float) -> float:
    """Factor on the scale law for a room with n_wall wall surfels over
    wall_area m^2: sqrt(REF_WALL_DENSITY / density), never above 1."""
    density = n_wall / wall_area
    return 1.0 if density <= REF_WALL_DENSITY else math.sqrt(REF_WALL_DENSITY / density)


@dataclasses.dataclass
class SurfelScene:
    """Structure-of-arrays 2D Gaussian surfel scene (Eq. 1 parameters plus the
    traced quantities r, e, rho of Eq. 3)."""

    pos: np.ndarray       # (n, 3) centre p
    quat: np.ndarray      # (n, 4) rotation q (w, x, y, z)
    scale: np.ndarray     # (n, 2) in-plane scales (s_u, s_v)
    opacity: np.ndarray   # (n,)   sigma
    albedo: np.ndarray    # (n, 3) diffuse albedo rho
    radiance: np.ndarray  # (n, 3) linear radiance r
    emissive: np.ndarray  # (n,)   emissive term e in [0, 1]

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def arrays(self):
        return (self.pos, self.quat, self.scale, self.opacity, self.albedo,
                self.radiance, self.emissive)

    def copy(self) -> "SurfelScene":
        return SurfelScene(*[a.copy() for a in self.arrays()])

    def validate(self) -> None:
        n = self.n
        shapes = {"pos": (n, 3), "quat": (n, 4), "scale": (n, 2), "opacity": (n,),
                  "albedo": (n, 3), "radiance": (n, 3), "emissive": (n,)}
        for name, shp in shapes.items():
            a = getattr(self, name)
            if a.shape != shp or a.dtype != np.float32 or not a.flags.c_contiguous:
                raise ValueError(f"{name}: want float32 C-contiguous {shp}, got {a.dtype} {a.shape}")


@dataclasses.dataclass
class Camera:
    """OpenCV pinhole camera: +x right, +y down, +z forward in camera space;
    ``c2w`` is the row-major 3x4 camera-to-world matrix [R | centre]."""

    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    c2w: np.ndarray  # (3, 4) float32

    def scaled_crop(self, x0: int, y0: int, w: int, h: int) -> "Camera":
        """Camera whose image is the (x0, y0, w, h) window of this one."""
        return Camera(w, h, self.fx, self.fy, self.cx - x0, self.cy - y0, self.c2w.copy())


def look_at_camera(width: int, height: int, hfov_deg: float, centre, forward, up) -> Camera:
    """Pinhole camera at ``centre`` looking along ``forward`` with ``up`` the
    world up vector; square pixels, principal point at the image centre."""
    f = np.asarray(forward, np.float64)
    f = f / np.linalg.norm(f)
    u = np.asarray(up, np.float64)
    down = -(u - f * np.dot(u, f))
    down /= np.linalg.norm(down)
    right = np.cross(down, f)
    c2w = np.zeros((3, 4), np.float64)
    c2w[:, 0] = right
    c2w[:, 1] = down
    c2w[:, 2] = f
    c2w[:, 3] = centre
    fx = (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    return Camera(int(width), int(height), float(fx), float(fx), width / 2.0, height / 2.0,
                  c2w.astype(np.float32))


# ----------------------------------------------------------------------------
# quaternion construction (input drawing only)
# ----------------------------------------------------------------------------

def _qmul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Hamilton product of (..., 4) quaternions (w, x, y, z)."""
    aw, ax, ay, az = np.moveaxis(a, -1, 0)
    bw, bx, by, bz = np.moveaxis(b, -1, 0)
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], axis=-1)


def _quat_z_to(normal) -> np.ndarray:
    """Quaternion of the shortest rotation taking +z onto the unit ``normal``."""
    n = np.asarray(normal, np.float64)
    z = np.array([0.0, 0.0, 1.0])
    c = float(np.dot(z, n))
    if c > 1.0 - 1e-12:
        return np.array([1.0, 0.0, 0.0, 0.0])
    if c < -1.0 + 1e-12:
        return np.array([0.0, 1.0, 0.0, 0.0])  # pi about x
    axis = np.cross(z, n)
    axis /= np.linalg.norm(axis)
    half = math.acos(c) / 2.0
    return np.concatenate([[math.cos(half)], math.sin(half) * axis])


def _uniform_quats(rng: np.random.Generator, m: int) -> np.ndarray:
    """Shoemake's uniformly distributed unit quaternions."""
    u1, u2, u3 = rng.random(m), rng.random(m), rng.random(m)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    t2, t3 = 2 * np.pi * u2, 2 * np.pi * u3
    return np.stack([b * np.cos(t3), a * np.sin(t2), a * np.cos(t2), b * np.sin(t3)], axis=1)


# ----------------------------------------------------------------------------
# room generators
# ----------------------------------------------------------------------------

# faces of an axis-aligned box: (axis, side) with side -1 = min face, +1 = max face
_FACES = [(0, -1), (0, 1), (1, -1), (1, 1), (2, -1), (2, 1)]


def _face_area(lo, hi, axis):
    ext = np.asarray(hi) - np.asarray(lo)
    o = [a for a in range(3) if a != axis]
    return float(ext[o[0]] * ext[o[1]])


def _rect_samples(rng, m, lo, hi, axis, coord, holes=()):
    """m points uniform on the axis-aligned rectangle of box face ``axis`` at
    ``coord``, rejecting points inside any (lo2, hi2) hole of the 2 free axes."""
    o = [a for a in range(3) if a != axis]
    out = np.empty((0, 3))
    while out.shape[0] < m:
        k = int((m - out.shape[0]) * 1.3) + 16
        pts = np.empty((k, 3))
        pts[:, axis] = coord
        pts[:, o[0]] = rng.uniform(lo[o[0]], hi[o[0]], k)
        pts[:, o[1]] = rng.uniform(lo[o[1]], hi[o[1]], k)
        keep = np.ones(k, bool)
        for (h0, h1) in holes:
            inside = ((pts[:, o[0]] >= h0[0]) & (pts[:, o[0]] <= h1[0]) &
                      (pts[:, o[1]] >= h0[1]) & (pts[:, o[1]] <= h1[1]))
            keep &= ~inside
        out = np.concatenate([out, pts[keep]])
    return out[:m]


def _wall_surfels(rng, m, lo, hi, faces=_FACES, holes=None):
    """Wall surfels on the listed faces of box [lo, hi]; returns pos, quat,
    face id per surfel.  ``holes[f]`` lists door openings on face f."""
    holes = holes or {}
    areas = np.array([_face_area(lo, hi, ax) for (ax, _s) in faces])
    counts = np.floor(m * areas / areas.sum()).astype(int)
    counts[np.argmax(areas)] += m - counts.sum()
    pos, quat, face = [], [], []
    for fi, ((ax, side), c) in enumerate(zip(faces, counts)):
        coord = lo[ax] if side < 0 else hi[ax]
        p = _rect_samples(rng, int(c), lo, hi, ax, coord, holes.get(fi, ()))
        p[:, ax] += rng.uniform(-5e-3, 5e-3, int(c))
        nrm = np.zeros(3)
        nrm[ax] = -side  # faces point into the room
        qf = _quat_z_to(nrm)
        th = rng.uniform(0.0, 2 * np.pi, int(c))
        qz = np.stack([np.cos(th / 2), np.zeros_like(th), np.zeros_like(th), np.sin(th / 2)], 1)
        pos.append(p)
        quat.append(_qmul(np.broadcast_to(qf, qz.shape), qz))
        face.append(np.full(int(c), fi))
    return np.concatenate(pos), np.concatenate(quat), np.concatenate(face)


def _common_attributes(rng, n, scale_f=1.0):
    scale = np.exp(rng.uniform(math.log(0.005), math.log(0.05), (n, 2))) * scale_f
    opacity = rng.uniform(0.5, 1.0, n)
    albedo = rng.uniform(0.1, 0.8, (n, 3))
    radiance = rng.uniform(0.0, 0.5, (n, 3))   # radiance cache of non-emitters
    emissive = np.zeros(n)
    return scale, opacity, albedo, radiance, emissive


def _make_emitters(rng, radiance, emissive, idx):
    emissive[idx] = 1.0
    radiance[idx] = rng.uniform(1.0, 10.0, (len(idx), 3))


def _pack(pos, quat, scale, opacity, albedo, radiance, emissive) -> SurfelScene:
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    s = SurfelScene(f(pos), f(quat), f(scale), f(opacity), f(albedo), f(radiance), f(emissive))
    s.validate()
    return s


def box_room(n: int, lo, hi, seed: int, emitter_mode: str, emitter_frac: float,
             n_patches: int = 4, shrink: float = 0.05) -> SurfelScene:
    """One closed box room with n surfels (wall:interior = 3000:1096).

    ``emitter_mode`` "uniform": a fraction of all surfels chosen uniformly;
    "ceiling": the ceiling surfels nearest the centres of ``n_patches`` square
    patches (z-max face), equally many per patch."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    n_wall = int(round(n * WALL_FRACTION))
    n_int = n - n_wall
    wpos, wquat, wface = _wall_surfels(rng, n_wall, lo, hi)
    c = (lo + hi) / 2
    h = (hi - lo) / 2 * (1 - shrink)
    ipos = rng.uniform(c - h, c + h, (n_int, 3))
    iquat = _uniform_quats(rng, n_int)
    pos = np.concatenate([wpos, ipos])
    quat = np.concatenate([wquat, iquat])
    area = sum(_face_area(lo, hi, ax) for ax, _s in _FACES)
    scale, opacity, albedo, radiance, emissive = _common_attributes(rng, n, scale_factor(n_wall, area))
    n_emit = int(round(n * emitter_frac))
    if emitter_mode == "uniform":
        idx = rng.choice(n, n_emit, replace=False)
    elif emitter_mode == "ceiling":
        ceil = np.nonzero(wface == 5)[0]
        idx = _ceiling_patch_emitters(pos, ceil, lo, hi, n_emit, n_patches)
    else:
        raise ValueError(emitter_mode)
    _make_emitters(rng, radiance, emissive, idx)
    return _pack(pos, quat, scale, opacity, albedo, radiance, emissive)


def _ceiling_patch_emitters(pos, ceil_idx, lo, hi, n_emit, n_patches):
    """Indices of the ceiling surfels nearest to ``n_patches`` patch centres laid
    out on a regular grid over the ceiling (equally many per patch)."""
    gx = int(math.ceil(math.sqrt(n_patches)))
    gy = int(math.ceil(n_patches / gx))
    centres = []
    for i in range(n_patches):
        ix, iy = i % gx, i // gx
        centres.append([lo[0] + (ix + 0.5) * (hi[0] - lo[0]) / gx,
                        lo[1] + (iy + 0.5) * (hi[1] - lo[1]) / gy])
    per = [n_emit // n_patches + (1 if i < n_emit % n_patches else 0) for i in range(n_patches)]
    chosen = set()
    xy = pos[ceil_idx, :2]
    for cxy, k in zip(centres, per):
        d = np.sum((xy - np.asarray(cxy)) ** 2, axis=1)
        order = np.argsort(d, kind="stable")
        got = 0
        for j in order:
            if ceil_idx[j] not in chosen:
                chosen.add(int(ceil_idx[j]))
                got += 1
                if got == k:
                    break
    return np.array(sorted(chosen), dtype=np.int64)


def three_room_layout(n: int, seed: int, emitter_frac: float = 0.005) -> SurfelScene:
    """Three 5x4x3 m rooms along x (x in [-7.5, 7.5]) whose two shared walls have
    1.0 x 2.0 m door openings; ceiling emitter patches in every room."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rooms = [(np.array([-7.5, -2.0, -1.5]), np.array([-2.5, 2.0, 1.5])),
             (np.array([-2.5, -2.0, -1.5]), np.array([2.5, 2.0, 1.5])),
             (np.array([2.5, -2.0, -1.5]), np.array([7.5, 2.0, 1.5]))]
    door = ((np.array([-0.5, -1.5])), np.array([0.5, 0.5]))   # (y, z) window on x-faces
    # walls: 3 rooms' x-faces are shared (interior x = -2.5, 2.5 once each) ...
    faces_per_room = [
        [(0, -1), (1, -1), (1, 1), (2, -1), (2, 1), (0, 1)],
        [(1, -1), (1, 1), (2, -1), (2, 1)],
        [(0, 1), (1, -1), (1, 1), (2, -1), (2, 1), (0, -1)],
    ]
    # ... so the middle room lists none of its x-faces; the left room owns x=-2.5
    # and the right room owns x=2.5, each with a door.
    total_area = 0.0
    for (lo, hi), faces in zip(rooms, faces_per_room):
        total_area += sum(_face_area(lo, hi, ax) for ax, _s in faces)
    door_area = 2 * (1.0 * 2.0)
    total_area -= door_area
    n_wall = int(round(n * WALL_FRACTION))
    n_int = n - n_wall
    pos, quat, face_room, face_kind = [], [], [], []
    done = 0
    for ri, ((lo, hi), faces) in enumerate(zip(rooms, faces_per_room)):
        holes = {}
        area = 0.0
        for fi, (ax, s) in enumerate(faces):
            a = _face_area(lo, hi, ax)
            if (ri == 0 and (ax, s) == (0, 1)) or (ri == 2 and (ax, s) == (0, -1)):
                holes[fi] = [door]
                a -= 2.0
            area += a
        m = n_wall - done if ri == 2 else int(round(n_wall * area / total_area))
        done += m
        # distribute m over faces by (open) area
        areas = np.array([_face_area(lo, hi, ax) - (2.0 if fi in holes else 0.0)
                          for fi, (ax, _s) in enumerate(faces)])
        counts = np.floor(m * areas / areas.sum()).astype(int)
        counts[np.argmax(areas)] += m - counts.sum()
        for fi, ((ax, side), c) in enumerate(zip(faces, counts)):
            p, q, _ = _wall_surfels(rng, int(c), lo, hi, faces=[(ax, side)],
                                    holes={0: holes.get(fi, ())})
            pos.append(p)
            quat.append(q)
            face_room.append(np.full(int(c), ri))
            face_kind.append(np.full(int(c), 1 if (ax, side) == (2, 1) else 0))
    wpos = np.concatenate(pos)
    wquat = np.concatenate(quat)
    room_of = np.concatenate(face_room)
    is_ceil = np.concatenate(face_kind) == 1
    # interior surfels: split over rooms by volume (all equal)
    ipos, iquat = [], []
    for ri, (lo, hi) in enumerate(rooms):
        k = n_int // 3 + (1 if ri < n_int % 3 else 0)
        c = (lo + hi) / 2
        h = (hi - lo) / 2 * 0.95
        ipos.append(rng.uniform(c - h, c + h, (k, 3)))
        iquat.append(_uniform_quats(rng, k))
    all_pos = np.concatenate([wpos] + ipos)
    all_quat = np.concatenate([wquat] + iquat)
    scale, opacity, albedo, radiance, emissive = _common_attributes(rng, n, scale_factor(n_wall, total_area))
    n_emit = int(round(n * emitter_frac))
    idx = []
    for ri, (lo, hi) in enumerate(rooms):
        k = n_emit // 3 + (1 if ri < n_emit % 3 else 0)
        ceil = np.nonzero(is_ceil & (room_of == ri))[0]
        idx.append(_ceiling_patch_emitters(all_pos, ceil, lo, hi, k, 4))
    _make_emitters(rng, radiance, emissive, np.concatenate(idx))
    return _pack(all_pos, all_quat, scale, opacity, albedo, radiance, emissive)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    scene_fn: object
    camera: Camera
    spp: int
    max_bounces: int
    rr_start: int
    seed: int = 0
    # factor the generator applied to the scale law log-U[0.005, 0.05] m
    # (rooms with denser walls than the medium room get smaller surfels)
    scale_factor: float = 1.0


def _box_wall_area(lo, hi) -> float:
    return sum(_face_area(np.asarray(lo, np.float64), np.asarray(hi, np.float64), ax) for ax, _s in _FACES)


def _layout_wall_area() -> float:
    """Open wall area of the three-room layout: 94 + 70 + 94 m^2 minus two
    1 x 2 m doors."""
    full = _box_wall_area([-2.5, -2.0, -1.5], [2.5, 2.0, 1.5])
    middle = full - 2 * 12.0  # its x-faces belong to its neighbours
    return 2 * full + middle - 2 * 2.0


def workload_scale_factor(n: int, wall_area: float) -> float:
    return scale_factor(int(round(n * WALL_FRACTION)), wall_area)


def tiny_room(n: int = 4096) -> SurfelScene:
    """4,096 surfels in the unit box, 2 % uniformly chosen emitters."""
    return box_room(n, [-0.5] * 3, [0.5] * 3, seed=1001, emitter_mode="uniform", emitter_frac=0.02)


def medium_room(n: int = 200_000, seed: int = 1002) -> SurfelScene:
    """200k surfels in a 5x4x3 m box, 1 % ceiling-patch emitters."""
    return box_room(n, [-2.5, -2.0, -1.5], [2.5, 2.0, 1.5], seed=seed, emitter_mode="ceiling",
                    emitter_frac=0.01)


def diff_room(n: int = 1_000_000) -> SurfelScene:
    """1M surfels, same law as the medium room (differentiable workload)."""
    return medium_room(n, seed=1003)


def serving_room(n: int = 3_000_000) -> SurfelScene:
    """3M surfels in a 10x8x3 m box, 1 % ceiling-patch emitters."""
    return box_room(n, [-5.0, -4.0, -1.5], [5.0, 4.0, 1.5], seed=1004, emitter_mode="ceiling",
                    emitter_frac=0.01, n_patches=8)


def large_layout(n: int = 6_000_000) -> SurfelScene:
    """6M surfels, three connected rooms, 0.5 % ceiling emitters."""
    return three_room_layout(n, seed=1005)


def horizontal_camera(width, height, centre=(0.0, 0.0, 0.0), forward=(1.0, 0.0, 0.0), hfov=90.0):
    return look_at_camera(width, height, hfov, centre, forward, (0.0, 0.0, 1.0))


def workload(name: str) -> Workload:
    """The named workload: tiny | medium | diff | serving | large."""
    if name == "tiny":
        return Workload("tiny room 4096 surfels 64x64 4spp 1 bounce", tiny_room,
                        Camera(64, 64, 32.0, 32.0, 32.0, 32.0, horizontal_camera(64, 64).c2w),
                        spp=4, max_bounces=1, rr_start=2)
    if name == "medium":
        return Workload("medium room 200k surfels 512x512 64spp 4 bounces RR>=2", medium_room,
                        horizontal_camera(512, 512), spp=64, max_bounces=4, rr_start=2)
    if name == "diff":
        f = workload_scale_factor(1_000_000, _box_wall_area([-2.5, -2.0, -1.5], [2.5, 2.0, 1.5]))
        return Workload("single bounce fwd+bwd 1M surfels 800x800 16spp", diff_room,
                        horizontal_camera(800, 800), spp=16, max_bounces=1, rr_start=2, scale_factor=f)
    if name == "serving":
        f = workload_scale_factor(3_000_000, _box_wall_area([-5.0, -4.0, -1.5], [5.0, 4.0, 1.5]))
        return Workload("serving room 3M surfels", serving_room,
                        horizontal_camera(512, 512), spp=16, max_bounces=3, rr_start=2, scale_factor=f)
    if name == "large":
        f = workload_scale_factor(6_000_000, _layout_wall_area())
        return Workload("large three-room 6M surfels 1920x1080 1024spp 5 bounces RR>=2",
                        large_layout, horizontal_camera(1920, 1080), spp=1024, max_bounces=5,
                        rr_start=2, scale_factor=f)
    raise KeyError(name)


# ----------------------------------------------------------------------------
# closed-form test scenes
# ----------------------------------------------------------------------------

def giant_box(half=(1.0, 1.0, 1.0), gap=1e-3, giant=1e4, rho=0.5, r=1.0, e=1.0,
              emissive_faces=None, floor_rho=None, floor_cache=0.0) -> SurfelScene:
    """Closed box of 12 giant surfels: every face carries two surfels (layers
    ``gap`` apart, the second outside the first), opacity 1, scale ``giant``
    so the Gaussian response is 1 to ~1e-9 anywhere in the box.

    ``emissive_faces``: face ids (order -x,+x,-y,+y,-z,+z) with e = ``e`` and
    radiance ``r``; other faces get e = 0 and radiance ``floor_cache``.  None
    makes every face emissive.  ``floor_rho`` overrides the albedo of face 4
    (the floor, -z)."""
    half = np.asarray(half, np.float64)
    pos, quat, alb, rad, emi = [], [], [], [], []
    for fi, (ax, side) in enumerate(_FACES):
        nrm = np.zeros(3)
        nrm[ax] = -side
        q = _quat_z_to(nrm)
        for layer in range(2):
            p = np.zeros(3)
            p[ax] = side * (half[ax] + layer * gap)
            pos.append(p)
            quat.append(q)
            is_e = emissive_faces is None or fi in emissive_faces
            a = rho if not (fi == 4 and floor_rho is not None) else floor_rho
            alb.append([a] * 3)
            rad.append([r] * 3 if is_e else [floor_cache] * 3)
            emi.append(e if is_e else 0.0)
    m = len(pos)
    return _pack(np.array(pos), np.array(quat), np.full((m, 2), giant), np.ones(m),
                 np.array(alb), np.array(rad), np.array(emi))


def random_small_scene(n: int, seed: int, spread=0.3, emit_frac=0.3) -> SurfelScene:
    """A few randomly placed and oriented surfels in front of the origin
    (around (1, 0, 0)), for brute-force and finite-difference checks."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = np.array([1.0, 0.0, 0.0]) + rng.uniform(-spread, spread, (n, 3))
    quat = _uniform_quats(rng, n) * rng.uniform(0.5, 2.0, (n, 1))  # not unit on purpose
    scale = np.exp(rng.uniform(math.log(0.05), math.log(0.3), (n, 2)))
    opacity = rng.uniform(0.5, 1.0, n)
    albedo = rng.uniform(0.1, 0.8, (n, 3))
    radiance = rng.uniform(0.0, 0.5, (n, 3))
    emissive = np.zeros(n)
    k = max(1, int(round(emit_frac * n)))
    idx = rng.choice(n, k, replace=False)
    emissive[idx] = 1.0
    radiance[idx] = rng.uniform(1.0, 10.0, (k, 3))
    return _pack(pos, quat, scale, opacity, albedo, radiance, emissive)


# ----------------------------------------------------------------------------
# serving request stream (serving room, 10 x 8 x 3 m)
# ----------------------------------------------------------------------------

SERVING_RESOLUTIONS = [(256, 256), (512, 512), (1280, 720), (1920, 1080)]
SERVING_SPP = [16, 64, 256]


def serving_requests(scene: SurfelScene, n: int, seed: int = 13, edit_frac: float = 0.1,
                     lo=(-5.0, -4.0, -1.5), hi=(5.0, 4.0, 1.5), spp_choices=None, res_choices=None):
    """Seeded request list: renders with a random horizontal camera pose inside
    the room, resolution and spp uniform over the serving sets, bounces
    uniform in 1..5; a fraction ``edit_frac`` are edits, uniform over:
    toggle emission on 5 % of the surfels (new emitters get radiance
    U[1, 10]); albedo scale U[0.5, 1.5] for the surfels within 0.5 m of a
    random centre; move the surfels within 0.25 m of a random surfel centre
    (about a thousand on a wall of this room) by a random vector of length
    <= 0.2 m.  Returns a list of dicts (no rendering arithmetic here)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.asarray(lo)
    hi = np.asarray(hi)
    spp_choices = spp_choices or SERVING_SPP
    res_choices = res_choices or SERVING_RESOLUTIONS
    out = []
    for k in range(n):
        if rng.random() < edit_frac:
            kind = int(rng.integers(0, 3))
            if kind == 0:
                idx = np.sort(rng.choice(scene.n, max(1, scene.n // 20), replace=False)).astype(np.int32)
                rad = rng.uniform(1.0, 10.0, (len(idx), 3)).astype(np.float32)
                out.append({"type": "edit", "op": "toggle_emission", "idx": idx, "per_index": rad})
            elif kind == 1:
                c = rng.uniform(lo * 0.9, hi * 0.9)
                out.append({"type": "edit", "op": "scale_albedo", "sphere": list(c) + [0.5],
                            "value": [float(rng.uniform(0.5, 1.5))] * 3})
            else:
                c = scene.pos[int(rng.integers(0, scene.n))].astype(np.float64)
                v = rng.normal(size=3)
                v *= rng.uniform(0.0, 0.2) / np.linalg.norm(v)
                out.append({"type": "edit", "op": "translate", "sphere": list(c) + [0.25], "value": list(v)})
        else:
            w, h = res_choices[int(rng.integers(0, len(res_choices)))]
            centre = rng.uniform(lo * 0.8, hi * 0.8)
            yaw = rng.uniform(0, 2 * np.pi)
            fwd = (np.cos(yaw), np.sin(yaw), 0.0)
            out.append({"type": "render", "camera": look_at_camera(w, h, 90.0, centre, fwd, (0.0, 0.0, 1.0)),
                        "spp": int(spp_choices[int(rng.integers(0, len(spp_choices)))]),
                        "max_bounces": int(rng.integers(1, 6)), "seed": int(rng.integers(0, 2 ** 31))})
    return out
