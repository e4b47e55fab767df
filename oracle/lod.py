"""Level-of-detail surfel merge: the oracle's plain FP64 definition.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` alone.  It shares no code
with the CUDA path.

The paper names a level-of-detail hierarchy over the reconstruction as the
way to cut the ray-Gaussian intersections per ray (Sec. 5, conclusion, and
Appendix D, path tracing: fewer Gaussians gave fewer intersections and a faster
render), and
gives no algorithm.  The reading this library implements, written out here:

* Groups.  A surfel belongs to the group (cell, axis, emitter) where cell is
  the cell of a uniform grid (origin o, edge h) holding its centre p, axis is
  the coordinate axis its normal n is closest to (largest |n_j|, the lower
  axis on a tie) and emitter is e > tau_E (Eq. 4).  Cell coordinates are
  clamped to [0, 2^20 - 1].  These three integer decisions are taken in FP32,
  in the operation order stated in ``group_keys``, on both sides.
* Merge (moment matching of the group's Gaussians, in FP64 here).  Weights
  w_i = sigma_i s_u,i s_v,i (opacity x footprint, the integral of sigma g over
  the surfel plane up to 2 pi).  W = sum w_i.
    p = sum w_i p_i / W
    n = normalise(sum w_i n_i'), n_i' = n_i flipped to n_i[axis] > 0
    M = sum w_i (d_i d_i^T + s_u,i^2 t_u,i t_u,i^T + s_v,i^2 t_v,i t_v,i^T) / W,
        d_i = p_i - p
    the merged in-plane covariance is P M P with P = I - n n^T: t_u is its
    principal direction, s_u^2 its largest eigenvalue, t_v = n x t_u and
    s_v^2 = t_v^T M t_v
    sigma = W / (s_u s_v)   (the group's footprint is kept; sigma may exceed
                             1, alpha = min(sigma g, alpha_max) stays <= alpha_max)
    rho, r, e = the w-weighted means.
  A group with W = 0 takes unit weights and sigma = 0.
* Order.  Merged surfels are written in ascending group key, the key packing
  (cell x, cell y, cell z, axis, emitter) into 63 bits as in ``group_keys``.
"""
from __future__ import annotations

import numpy as np

CELL_BITS = 20
CELL_MAX = (1 << CELL_BITS) - 1


def group_keys(pos, quat, emissive, origin, cell_size, tau_E=0.1):
    """(n,) uint64 group keys; FP32 decisions.

    cell_j = clamp(floor((p_j - o_j) * (1 / h)), 0, 2^20 - 1), each operation
    rounded to FP32 (1 / h too).  Normal direction from the raw quaternion
    (w, x, y, z) without normalisation (the argmax does not depend on the
    scale): n' = (2 (x z + w y), 2 (y z - w x), (w w + z z) - (x x + y y)),
    each product and sum rounded to FP32 in that order.  key = cx << 43 |
    cy << 23 | cz << 3 | axis << 1 | emitter."""
    f32 = np.float32
    p = np.asarray(pos, f32)
    q = np.asarray(quat, f32)
    o = np.asarray(origin, f32).reshape(1, 3)
    inv_h = f32(1.0) / f32(cell_size)
    c = np.floor((p - o) * inv_h)
    c = np.clip(c, f32(0.0), f32(CELL_MAX)).astype(np.int64)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    two = f32(2.0)
    nx = two * (x * z + w * y)
    ny = two * (y * z - w * x)
    nz = (w * w + z * z) - (x * x + y * y)
    ax_, ay_, az_ = np.abs(nx), np.abs(ny), np.abs(nz)
    axis = np.where((ax_ >= ay_) & (ax_ >= az_), 0, np.where(ay_ >= az_, 1, 2)).astype(np.int64)
    em = (np.asarray(emissive, f32) > f32(tau_E)).astype(np.int64)
    key = (c[:, 0] << 43) | (c[:, 1] << 23) | (c[:, 2] << 3) | (axis << 1) | em
    return key.astype(np.uint64), axis


def frames(quat):
    """(t_u, t_v, n) of each surfel from its normalised quaternion (Eq. 1's
    rotation: t_u, t_v are its first two columns, n = t_u x t_v)."""
    q = np.asarray(quat, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    tu = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)], 1)
    tv = np.stack([2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)], 1)
    return tu, tv, np.cross(tu, tv)


def quat_from_frame(tu, tv, n):
    """Unit quaternion (w, x, y, z) of the rotation with columns (t_u, t_v, n)
    (Shepperd's method: the largest of the four squared components first)."""
    R = np.stack([tu, tv, n], 1)  # R[:, j] = column j
    tr = R[0, 0] + R[1, 1] + R[2, 2]
    cands = [tr, R[0, 0], R[1, 1], R[2, 2]]
    k = int(np.argmax(cands))
    if k == 0:
        s = 2.0 * np.sqrt(1.0 + tr)
        q = [0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s]
    elif k == 1:
        s = 2.0 * np.sqrt(1.0 + R[0, 0] - R[1, 1] - R[2, 2])
        q = [(R[2, 1] - R[1, 2]) / s, 0.25 * s, (R[0, 1] + R[1, 0]) / s, (R[0, 2] + R[2, 0]) / s]
    elif k == 2:
        s = 2.0 * np.sqrt(1.0 + R[1, 1] - R[0, 0] - R[2, 2])
        q = [(R[0, 2] - R[2, 0]) / s, (R[0, 1] + R[1, 0]) / s, 0.25 * s, (R[1, 2] + R[2, 1]) / s]
    else:
        s = 2.0 * np.sqrt(1.0 + R[2, 2] - R[0, 0] - R[1, 1])
        q = [(R[1, 0] - R[0, 1]) / s, (R[0, 2] + R[2, 0]) / s, (R[1, 2] + R[2, 1]) / s, 0.25 * s]
    return np.array(q)


def merge_group(p, tu, tv, n, scale, sigma, rho, r, e, axis):
    """One group's merged surfel (FP64), following the module docstring.
    Returns dict(pos, quat, scale, opacity, albedo, radiance, emissive,
    cov) with cov = s_u^2 t_u t_u^T + s_v^2 t_v t_v^T."""
    w = sigma * scale[:, 0] * scale[:, 1]
    W = float(w.sum())
    zero = not W > 0.0
    if zero:
        w = np.ones_like(w)
        W = float(w.sum())
    pc = (w[:, None] * p).sum(0) / W
    flip = np.where(n[:, axis] < 0.0, -1.0, 1.0)
    nsum = (w[:, None] * flip[:, None] * n).sum(0)
    nc = nsum / np.linalg.norm(nsum)
    d = p - pc
    M = np.zeros((3, 3))
    for i in range(len(w)):
        M += w[i] * (np.outer(d[i], d[i]) + scale[i, 0] ** 2 * np.outer(tu[i], tu[i])
                     + scale[i, 1] ** 2 * np.outer(tv[i], tv[i]))
    M /= W
    P = np.eye(3) - np.outer(nc, nc)
    S = P @ M @ P
    lam, vec = np.linalg.eigh(S)
    tuc = vec[:, 2] - nc * float(vec[:, 2] @ nc)
    tuc /= np.linalg.norm(tuc)
    tvc = np.cross(nc, tuc)
    su = np.sqrt(max(float(lam[2]), 0.0))
    sv = np.sqrt(max(float(tvc @ M @ tvc), 0.0))
    sig = 0.0 if zero else W / (su * sv)
    return {
        "pos": pc, "quat": quat_from_frame(tuc, tvc, nc), "scale": np.array([su, sv]), "opacity": sig,
        "albedo": (w[:, None] * rho).sum(0) / W, "radiance": (w[:, None] * r).sum(0) / W,
        "emissive": float((w * e).sum() / W),
        "cov": su * su * np.outer(tuc, tuc) + sv * sv * np.outer(tvc, tvc), "normal": nc, "weight": W,
    }


def quat_from_frames(tu, tv, n):
    """quat_from_frame for every row of (m, 3) frames (the same branch rule,
    row by row)."""
    R = np.stack([tu, tv, n], 2)  # R[g, :, j] = column j
    r = lambda i, j: R[:, i, j]
    tr = r(0, 0) + r(1, 1) + r(2, 2)
    k = np.argmax(np.stack([tr, r(0, 0), r(1, 1), r(2, 2)], 1), 1)
    q = np.zeros((len(tr), 4))
    with np.errstate(invalid="ignore", divide="ignore"):
        cand = []
        s = 2.0 * np.sqrt(1.0 + tr)
        cand.append([0.25 * s, (r(2, 1) - r(1, 2)) / s, (r(0, 2) - r(2, 0)) / s, (r(1, 0) - r(0, 1)) / s])
        s = 2.0 * np.sqrt(1.0 + r(0, 0) - r(1, 1) - r(2, 2))
        cand.append([(r(2, 1) - r(1, 2)) / s, 0.25 * s, (r(0, 1) + r(1, 0)) / s, (r(0, 2) + r(2, 0)) / s])
        s = 2.0 * np.sqrt(1.0 + r(1, 1) - r(0, 0) - r(2, 2))
        cand.append([(r(0, 2) - r(2, 0)) / s, (r(0, 1) + r(1, 0)) / s, 0.25 * s, (r(1, 2) + r(2, 1)) / s])
        s = 2.0 * np.sqrt(1.0 + r(2, 2) - r(0, 0) - r(1, 1))
        cand.append([(r(1, 0) - r(0, 1)) / s, (r(0, 2) + r(2, 0)) / s, (r(1, 2) + r(2, 1)) / s, 0.25 * s])
    for b in range(4):
        sel = k == b
        q[sel] = np.stack(cand[b], 1)[sel]
    return q


def merge(scene, origin, cell_size, tau_E=0.1, with_members=True):
    """The merged scene of ``scene`` (a SurfelScene): dict of FP64 arrays in
    ascending key order, plus 'keys' (uint64), 'cov' (m, 3, 3), 'normal'
    (m, 3), 'weight' (m,) and, with_members, 'members' (list of index
    arrays, ascending).  Every group at once: the sums of merge_group taken
    per group with np.add.reduceat over the key-sorted surfels, the
    projected moments decomposed by a batched np.linalg.eigh; the same
    definition, step for step, as merge_group (a test holds the two equal)."""
    keys, axis = group_keys(scene.pos, scene.quat, scene.emissive, origin, cell_size, tau_E)
    order = np.argsort(keys, kind="stable")
    ks = keys[order]
    N = len(ks)
    if N == 0:
        res = {k: np.zeros((0, 3)) for k in ("pos", "albedo", "radiance", "normal")}
        res.update(quat=np.zeros((0, 4)), scale=np.zeros((0, 2)), opacity=np.zeros(0), emissive=np.zeros(0),
                   cov=np.zeros((0, 3, 3)), weight=np.zeros(0), keys=ks)
        if with_members:
            res["members"] = []
        return res
    starts = np.flatnonzero(np.concatenate([[True], ks[1:] != ks[:-1]]))
    ends = np.append(starts[1:], N)
    gid = np.repeat(np.arange(len(starts)), ends - starts)
    f64 = lambda a: np.asarray(a, np.float64)[order]
    p, sc, sg = f64(scene.pos), f64(scene.scale), f64(scene.opacity)
    rho, r, e = f64(scene.albedo), f64(scene.radiance), f64(scene.emissive)
    tu, tv, n = frames(np.asarray(scene.quat)[order])
    ax = axis[order]
    seg = lambda x: np.add.reduceat(x, starts, axis=0)
    w = sg * sc[:, 0] * sc[:, 1]
    W = seg(w)
    zero = ~(W > 0.0)
    w = np.where(zero[gid], 1.0, w)
    W = seg(w)
    pc = seg(w[:, None] * p) / W[:, None]
    flip = np.where(n[np.arange(N), ax] < 0.0, -1.0, 1.0)
    nsum = seg((w * flip)[:, None] * n)
    nc = nsum / np.linalg.norm(nsum, axis=1, keepdims=True)
    d = p - pc[gid]
    outer = lambda a: a[:, :, None] * a[:, None, :]
    M = seg(w[:, None, None] * (outer(d) + sc[:, 0, None, None] ** 2 * outer(tu) + sc[:, 1, None, None] ** 2 * outer(tv)))
    M /= W[:, None, None]
    P = np.eye(3)[None] - outer(nc)
    S = P @ M @ P
    lam, vec = np.linalg.eigh(S)
    v = vec[:, :, 2]
    tuc = v - nc * (v * nc).sum(1, keepdims=True)
    tuc /= np.linalg.norm(tuc, axis=1, keepdims=True)
    tvc = np.cross(nc, tuc)
    su = np.sqrt(np.maximum(lam[:, 2], 0.0))
    sv = np.sqrt(np.maximum(np.einsum("gi,gij,gj->g", tvc, M, tvc), 0.0))
    sig = np.where(zero, 0.0, W / (su * sv))
    res = {"pos": pc, "quat": quat_from_frames(tuc, tvc, nc), "scale": np.stack([su, sv], 1), "opacity": sig,
           "albedo": seg(w[:, None] * rho) / W[:, None], "radiance": seg(w[:, None] * r) / W[:, None],
           "emissive": seg(w * e) / W, "cov": su[:, None, None] ** 2 * outer(tuc) + sv[:, None, None] ** 2 * outer(tvc),
           "normal": nc, "weight": W, "keys": ks[starts]}
    if with_members:
        res["members"] = [order[a:b] for a, b in zip(starts, ends)]
    return res


def merge_by_group(scene, origin, cell_size, tau_E=0.1):
    """merge() computed one group at a time with merge_group (the plain
    form; slow on large scenes)."""
    keys, axis = group_keys(scene.pos, scene.quat, scene.emissive, origin, cell_size, tau_E)
    order = np.argsort(keys, kind="stable")
    ks = keys[order]
    starts = np.flatnonzero(np.concatenate([[True], ks[1:] != ks[:-1]]))
    ends = np.append(starts[1:], len(ks))
    p = np.asarray(scene.pos, np.float64)
    tu, tv, n = frames(scene.quat)
    sc = np.asarray(scene.scale, np.float64)
    sg = np.asarray(scene.opacity, np.float64)
    rho = np.asarray(scene.albedo, np.float64)
    r = np.asarray(scene.radiance, np.float64)
    e = np.asarray(scene.emissive, np.float64)
    out = {k: [] for k in ("pos", "quat", "scale", "opacity", "albedo", "radiance", "emissive", "cov", "normal",
                           "weight")}
    members = []
    for a, b in zip(starts, ends):
        idx = order[a:b]
        g = merge_group(p[idx], tu[idx], tv[idx], n[idx], sc[idx], sg[idx], rho[idx], r[idx], e[idx],
                        int(axis[idx[0]]))
        for k in out:
            out[k].append(g[k])
        members.append(idx)
    res = {k: np.array(v) for k, v in out.items()}
    res["keys"] = ks[starts]
    res["members"] = members
    return res


def to_scene(merged, scene_cls):
    """The merged surfels as a FP32 scene of class ``scene_cls`` (SurfelScene)."""
    f = lambda k: np.ascontiguousarray(merged[k], np.float32)
    return scene_cls(f("pos"), f("quat"), f("scale"), f("opacity"), f("albedo"), f("radiance"), f("emissive"))
