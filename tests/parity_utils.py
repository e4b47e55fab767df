"""Comparison helpers shared by the parity tests (no GPU needed).

Everything here is test-side: it compares GPU output with the oracle, and it
chooses inputs (pixels, rays) from the oracle's own records and from seeded
NumPy draws, never from GPU output."""
import numpy as np

import oracle as O

REL_TOL = 1e-4     # per-pixel relative radiance tolerance
FLOOR_FRAC = 1e-3  # relative floor: fraction of the image's mean radiance


def radiance_close(gpu, ref, rel=REL_TOL, floor_frac=FLOOR_FRAC, mean_ref=None):
    """Boolean mask of |gpu - ref| <= rel * max(|ref|, floor_frac * mean(ref))
    per channel (all channels must pass)."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    m = float(np.mean(np.abs(ref))) if mean_ref is None else mean_ref
    bound = rel * np.maximum(np.abs(ref), floor_frac * m)
    ok = np.abs(gpu - ref) <= bound
    return ok.all(axis=-1)


COND_DEV_K = 8.0  # ill-conditioned samples, entries and segments: bound + 8 x the conditioning spread


def compare_samples(gpu_samples, ref_samples, sample_flags, rel=REL_TOL, primary_emitter=None, sample_dev=None):
    """Sample by sample, on every sample the oracle did not flag as near a
    discrete decision or ill-conditioned in FP32:
    |L_gpu - L_ref| <= rel * max(|L_ref|, 1e-3 * mean |L_ref|) per channel.
    With sample_dev (per sample and channel, how far the oracle's
    conditioning runs move the sample; +inf where they change a discrete
    outcome), a sample flagged only as ill-conditioned whose spread is finite
    is compared too, held to |L_gpu - L_ref| <= bound + 8 dev per channel.
    Returns (ok (pixels, spp): True where compared and within the bound or
    not compared, stats).  stats counts the samples compared at the bound and
    the ill-conditioned ones compared at bound + 8 dev, the lit ones (radiance
    > 0) of each and, with primary_emitter (per pixel: the pixel sees an
    emitter directly), the lit ones whose light came through a bounce."""
    g = np.asarray(gpu_samples, np.float64)
    r = np.asarray(ref_samples, np.float64)
    flags = np.asarray(sample_flags)
    keep = flags == 0
    mean_ref = float(np.mean(np.abs(r)))
    floor = FLOOR_FRAC * mean_ref
    bound = rel * np.maximum(np.abs(r), floor)
    within = (np.abs(g - r) <= bound).all(axis=-1)
    cond = np.zeros(keep.shape, bool)
    within_c = np.zeros(keep.shape, bool)
    if sample_dev is not None:
        d = np.asarray(sample_dev, np.float64)
        cond = (flags == O.FLAGS["cond"]) & np.isfinite(d).all(axis=-1)
        within_c = (np.abs(g - r) <= bound + COND_DEV_K * np.where(np.isfinite(d), d, 0.0)).all(axis=-1)
    ok = np.where(keep, within, np.where(cond, within_c, True))
    err = np.abs(g - r) / np.maximum(np.abs(r), floor + 1e-30)
    err_k = err[keep].max(axis=-1) if keep.any() else np.zeros(0)
    lit = np.abs(r).max(axis=-1) > 0
    stats = {"samples": int(keep.size), "compared": int(keep.sum()), "fail": int((~ok).sum()),
             "flagged_samples": float(1 - keep.mean()) if keep.size else 0.0,
             "lit_compared": int((lit & keep).sum()), "lit_samples": int(lit.sum()),
             "max_rel": float(err_k.max()) if err_k.size else 0.0,
             "p999_rel": float(np.quantile(err_k, 0.999)) if err_k.size else 0.0,
             "mean_rel": float(err_k.mean()) if err_k.size else 0.0}
    if sample_dev is not None:
        stats["cond_compared"] = int(cond.sum())
        stats["lit_cond_compared"] = int((lit & cond).sum())
    if primary_emitter is not None:
        bounced = lit & ~np.asarray(primary_emitter, bool)[:, None]
        stats["lit_bounced_compared"] = int((bounced & keep).sum())
        if sample_dev is not None:
            stats["lit_bounced_cond_compared"] = int((bounced & cond).sum())
    if stats["fail"]:
        bad = np.argwhere(~ok)[:4]
        stats["worst"] = [{"pixel_row": int(i), "sample": int(j), "gpu": g[i, j].tolist(), "ref": r[i, j].tolist(),
                           "rel": float(err[i, j].max()), "flags": int(flags[i, j])} for i, j in bad]
    return ok, stats


GRAD_TOL = 1e-3  # gradient tolerance (per group and per entry)


def oracle_grad_with_conditioning(fn, *args, **kw):
    """The oracle's gradient (fn = O.single_bounce_grad or O.radiance_grad)
    and, per entry, how far its four conditioning runs (rays and sigma g
    perturbed at FP32 rounding scale, as the render's) move it:
    (grad, pixel flags, dev)."""
    g, fl = fn(*args, **kw)
    dev = np.zeros_like(g)
    for run in (1, 2, 3, 4):
        gj, _ = fn(*args, run=run, **kw)
        dev = np.maximum(dev, np.abs(gj - g))
    return g, fl, dev


def grad_errors(g_gpu, g_ref, tol=GRAD_TOL, dev=None):
    """Gradient of one parameter group, GPU vs reference: the group's relative
    error ||g - r|| / ||r|| and the per-entry criterion
    |g - r| <= tol * max(|r|, 1e-3 * rms(r)) on every entry.  With dev (per
    entry, how far the oracle's conditioning runs move it) an entry that
    FP32-scale perturbations move by more than a quarter of its bound is
    ill-conditioned in FP32, as samples are: it is counted and held only to
    |g - r| <= bound + 8 dev.  Returns (group error, ok mask of the entries,
    worst well-conditioned entry's ratio to its bound, number of
    ill-conditioned entries)."""
    g = np.asarray(g_gpu, np.float64)
    r = np.asarray(g_ref, np.float64)
    nrm = np.linalg.norm(r)
    group = float(np.linalg.norm(g - r) / nrm) if nrm > 0 else float(np.linalg.norm(g))
    rms = float(np.sqrt(np.mean(r * r))) if r.size else 0.0
    if rms == 0.0:
        ok = g == 0.0
        return group, ok, float(np.abs(g).max()) if g.size else 0.0, 0
    bound = tol * np.maximum(np.abs(r), 1e-3 * rms)
    err = np.abs(g - r)
    ill = np.zeros(r.shape, bool)
    if dev is not None:
        d = np.asarray(dev, np.float64)
        ill = d > 0.25 * bound
        ok = np.where(ill, err <= bound + COND_DEV_K * d, err <= bound)
    else:
        ok = err <= bound
    well = ~ill
    worst = float((err[well] / bound[well]).max()) if well.any() else 0.0
    return group, ok, worst, int(ill.sum())


def flag_names(bits):
    return [k for k, v in O.FLAGS.items() if bits & v]


# --------------------------------------------------------------------------
# inputs chosen from the oracle's records
# --------------------------------------------------------------------------
def camera_rays(cam, pixels):
    """Pinhole rays through the pixel centres (FP64; the same camera model as
    both renderers)."""
    pixels = np.asarray(pixels, np.int64)
    c2w = np.asarray(cam.c2w, np.float64).reshape(3, 4)
    x = (pixels % cam.width).astype(np.float64)
    y = (pixels // cam.width).astype(np.float64)
    d = np.stack([(x + 0.5 - cam.cx) / cam.fx, (y + 0.5 - cam.cy) / cam.fy, np.ones_like(x)], 1) @ c2w[:, :3].T
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return np.broadcast_to(c2w[:, 3], d.shape).copy(), d


def _field(scene, name):
    """A scene array of a SurfelScene or an oracle.OracleScene, as FP64."""
    a = scene.arrays[name] if hasattr(scene, "arrays") and isinstance(scene.arrays, dict) else getattr(scene, name)
    return np.asarray(a, np.float64)


def emitter_frames(scene, tau_E=0.1):
    """Centres, unit normals and Gaussian areas 2 pi sigma s_u s_v of the
    emitter surfels (e > tau_E)."""
    em = np.nonzero(_field(scene, "emissive") > tau_E)[0]
    q = _field(scene, "quat")[em]
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    tu = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)], 1)
    tv = np.stack([2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)], 1)
    s = _field(scene, "scale")[em]
    area = 2 * np.pi * s[:, 0] * s[:, 1] * _field(scene, "opacity")[em]
    return em, _field(scene, "pos")[em], np.cross(tu, tv), area


def primary_vertices(scene, cam, pixels, n_threads=None):
    """Oracle primary records of the pixels (path-tracing mode): returns
    (hit X, normal N~, emitter?, hit?) per pixel."""
    rec, _fl = O.primary(scene, cam, np.asarray(pixels, np.int32), mode=1, params=O.Params(fp32_eps=0.0),
                         n_threads=n_threads)
    o, d = camera_rays(cam, pixels)
    X = o + rec[:, 3:4] * d
    return X, rec[:, 0:3], rec[:, 7] > 0.1, rec[:, 11] > 0


def lit_pixels(scene, cam, n_pick, n_cand, seed=7, n_threads=None):
    """n_pick pixels, from n_cand random candidates (seeded), whose primary
    vertex (a non-emitter hit in the oracle's primary records) has the
    largest unoccluded form factor to the emitters, sum_i A_i cos_x cos_i /
    (pi r^2): the pixels whose paths reach an emitter most often.  Pixels
    whose primary segment the oracle flags (a decision every sample of the
    pixel shares) come last.  The choice uses the oracle's records only."""
    rng = np.random.default_rng(seed)
    npix = cam.width * cam.height
    cand = rng.choice(npix, min(n_cand, npix), replace=False).astype(np.int32)
    X, N, emit, hit = primary_vertices(scene, cam, cand, n_threads)
    _rec, pfl = O.primary(scene, cam, cand, mode=1, n_threads=n_threads)
    _em, P, nE, area = emitter_frames(scene)
    F = np.full(cand.size, -1.0)
    ok = hit & ~emit
    idx = np.nonzero(ok)[0]
    for a in range(0, idx.size, 128):
        b = idx[a:a + 128]
        d = P[None, :, :] - X[b, None, :]
        r2 = (d * d).sum(-1)
        dn = d / np.sqrt(r2)[..., None]
        cx = np.clip((dn * N[b, None, :]).sum(-1), 0.0, None)
        ce = np.abs((dn * nE[None]).sum(-1))
        F[b] = (area[None] * cx * ce / (np.pi * r2)).sum(-1)
    order = np.lexsort((-F, pfl != 0))
    return np.sort(cand[order[:n_pick]])


def secondary_rays(scene, cam, n_pixels, seed=5, offset=1e-3, aim_frac=0.75, n_threads=None):
    """Rays shaped like the path tracer's bounces, for segment-level checks at
    full scene size: from the oracle's primary vertices of n_pixels random
    pixels (seeded), origin X + offset N~; a fraction aim_frac aimed at the
    centre of an emitter surfel drawn from the eighth nearest to the origin
    (so that many segments blend an emitter), the rest cosine-distributed
    about N~.  Returns float32 (m, 6) origin + direction."""
    rng = np.random.default_rng(seed)
    npix = cam.width * cam.height
    pix = rng.choice(npix, min(n_pixels, npix), replace=False).astype(np.int32)
    X, N, emit, hit = primary_vertices(scene, cam, pix, n_threads)
    keep = hit & ~emit
    X, N = X[keep], N[keep]
    O0 = X + offset * N
    m = X.shape[0]
    # cosine-weighted directions about N (any orthonormal basis will do here)
    a = np.where(np.abs(N[:, 0:1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    b1 = np.cross(N, a)
    b1 /= np.linalg.norm(b1, axis=1, keepdims=True)
    b2 = np.cross(N, b1)
    u0, u1 = rng.random(m), rng.random(m)
    r, phi = np.sqrt(u0), 2 * np.pi * u1
    cosd = (r * np.cos(phi))[:, None] * b1 + (r * np.sin(phi))[:, None] * b2 + np.sqrt(1 - u0)[:, None] * N
    _em, P, _nE, _area = emitter_frames(scene)
    near = max(1, P.shape[0] // 8)
    pick = rng.integers(0, near, m)
    tgt = np.empty((m, 3))
    for a in range(0, m, 256):
        d2 = ((O0[a:a + 256, None, :] - P[None, :, :]) ** 2).sum(-1)
        order = np.argpartition(d2, near - 1, axis=1)[:, :near]
        tgt[a:a + 256] = P[order[np.arange(order.shape[0]), pick[a:a + 256]]]
    to_em = tgt - O0
    to_em /= np.linalg.norm(to_em, axis=1, keepdims=True)
    aim = rng.random(m) < aim_frac
    w = np.where(aim[:, None], to_em, cosd)
    rays = np.concatenate([O0, w], 1).astype(np.float32)
    # the direction is renormalised after rounding so both sides trace the same unit vector
    d = rays[:, 3:].astype(np.float64)
    rays[:, 3:] = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    return rays
