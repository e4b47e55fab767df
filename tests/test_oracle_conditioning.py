"""The oracle's conditioning outputs (test infrastructure, no GPU).

The parity tests compare a sample, or a traced segment, that the oracle marks
as ill-conditioned in FP32 within the 1e-4 bound plus a multiple of how far
the oracle's conditioning runs move it.  These checks tie that spread to the
flag it comes from and show that asking for it changes nothing else.
"""
import numpy as np

import oracle as O
from paper_2601_23065_gb300 import scenes as S

COND = O.FLAGS["cond"]


def _pixels(cam, n, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(cam.width * cam.height, n, replace=False)).astype(np.int32)


def test_sample_spread_matches_the_flag():
    sc = S.tiny_room(4096)
    cam = S.horizontal_camera(48, 40)
    pix = _pixels(cam, 160, 3)
    prm = O.Params()
    a = O.render(sc, cam, pix, "pt", 4, max_bounces=3, rr_start=2, seed=5, want_samples=True, want_dev=True)
    b = O.render(sc, cam, pix, "pt", 4, max_bounces=3, rr_start=2, seed=5, want_samples=True)
    # asking for the spread changes neither the samples nor the flags
    assert np.array_equal(a["samples"], b["samples"]) and np.array_equal(a["sample_flags"], b["sample_flags"])
    dev, L, fl = a["sample_dev"], a["samples"], a["sample_flags"]
    assert (dev >= 0).all()
    # a discrete change is reported on every channel
    inf = np.isinf(dev)
    assert np.array_equal(inf.any(-1), inf.all(-1))
    flagged = (fl & COND) != 0
    rule = inf.any(-1) | (dev > prm.cond_tol * np.abs(L)).any(-1)
    assert np.array_equal(flagged, rule)
    assert flagged.any() and (~flagged).any()
    # without FP32 perturbations there is no spread
    c = O.render(sc, cam, pix, "pt", 4, max_bounces=3, rr_start=2, seed=5, want_samples=True, want_dev=True,
                 params=O.Params(fp32_eps=0.0))
    assert (c["sample_dev"] == 0).all()


def test_segment_spread_matches_the_flag():
    sc = S.tiny_room(4096)
    rng = np.random.default_rng(9)
    o = rng.uniform(-0.4, 0.4, (400, 3))
    d = rng.normal(size=(400, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.concatenate([o, d], 1).astype(np.float32).astype(np.float64)
    rec, nh, fl, hi, dev = O.trace_rays(sc, rays, mode=1, max_hits=64, want_dev=True)
    rec2, nh2, fl2, hi2 = O.trace_rays(sc, rays, mode=1, max_hits=64)
    assert np.array_equal(rec, rec2) and np.array_equal(nh, nh2) and np.array_equal(hi, hi2)
    # with the spread both re-traces run, so the flag can only be the same
    assert np.array_equal(fl, fl2)
    assert (dev >= 0).all()
    assert (dev[nh == 0] == 0).all()
    inf = np.isinf(dev)
    assert np.array_equal(inf.any(-1), inf.all(-1))
    tol = O.Params().cond_tol
    # the segment rule: R, E, P, A and D~ relative to the value, N~ absolute
    rel_cols = [3, 4, 5, 6, 7, 8, 9, 10, 11]
    rule = inf.any(-1) | (dev[:, rel_cols] > tol * np.abs(rec[:, rel_cols])).any(-1) | \
        (dev[:, 0:3] > tol / 5.0).any(-1)
    flagged = (fl & COND) != 0
    assert np.array_equal(flagged[nh > 0], rule[nh > 0])
    assert flagged.any() and (~flagged[nh > 0]).any()
