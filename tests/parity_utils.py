"""Comparison helpers shared by the parity tests (no GPU needed)."""
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


def compare_samples(gpu_samples, ref_samples, sample_flags, rel=REL_TOL):
    """Per pixel, the mean over the samples the oracle did not flag as
    near-boundary, GPU vs oracle.  Returns (ok mask per pixel, stats)."""
    g = np.asarray(gpu_samples, np.float64)
    r = np.asarray(ref_samples, np.float64)
    keep = (np.asarray(sample_flags) == 0)
    cnt = keep.sum(axis=1)
    gm = (g * keep[..., None]).sum(axis=1) / np.maximum(cnt, 1)[:, None]
    rm = (r * keep[..., None]).sum(axis=1) / np.maximum(cnt, 1)[:, None]
    ok = radiance_close(gm, rm, rel, mean_ref=float(np.mean(np.abs(r))))
    ok |= cnt == 0
    err = np.abs(gm - rm) / np.maximum(np.abs(rm), FLOOR_FRAC * float(np.mean(np.abs(r))) + 1e-30)
    stats = {"pixels": int(ok.size), "fail": int((~ok).sum()), "flagged_samples": float(1 - keep.mean()),
             "max_rel": float(err.max()) if err.size else 0.0, "p999_rel": float(np.quantile(err, 0.999)) if err.size else 0.0,
             "mean_rel": float(err.mean()) if err.size else 0.0}
    return ok, stats


def flag_names(bits):
    return [k for k, v in O.FLAGS.items() if bits & v]
