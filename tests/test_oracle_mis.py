"""Pins of the oracle's emitter sampling with multiple importance sampling:
the light strategy's solid-angle density integrates to one over the sphere,
and the MIS estimator has the plain estimator's expectation (Eq. 8) with a
smaller variance when the emitters are small."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2601_23065_gb300 import scenes as S


def _fib_sphere(n):
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    r = np.sqrt(1.0 - z * z)
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def _one_emitter(scale=(0.4, 0.25), tilt=0.3):
    q = np.array([[math.cos(tilt / 2), math.sin(tilt / 2), 0.0, 0.0]], np.float32)
    return S.SurfelScene(np.array([[0.0, 0.0, 1.0]], np.float32), q, np.array([scale], np.float32),
                         np.array([0.9], np.float32), np.array([[0.5, 0.5, 0.5]], np.float32),
                         np.array([[4.0, 2.0, 1.0]], np.float32), np.array([1.0], np.float32))


def test_light_density_integrates_to_one():
    sc = _one_emitter()
    dirs = _fib_sphere(60000)
    vals = np.array([O.light_pdf(sc, (0.1, -0.2, 0.0), w)[0] for w in dirs])
    integral = vals.mean() * 4.0 * math.pi
    assert integral == pytest.approx(1.0, rel=0.02)
    # two emitters: each carries its selection probability, the sum is one
    two = S.SurfelScene(*[np.concatenate([getattr(sc, k), getattr(_one_emitter((0.2, 0.2), -0.5), k)])
                          for k in ("pos", "quat", "scale", "opacity", "albedo", "radiance", "emissive")])
    two.pos[1] = [0.6, 0.3, 0.8]
    vals = np.array([O.light_pdf(two, (0.1, -0.2, 0.0), w)[0] for w in dirs])
    assert vals.mean() * 4.0 * math.pi == pytest.approx(1.0, rel=0.02)
    # a direction that misses every emitter has density zero
    assert O.light_pdf(sc, (0.1, -0.2, 0.0), (0.0, 0.0, -1.0)) == (0.0, 0)


def _lamp_box(n_lamps=6, seed=3):
    """Closed giant-surfel box (no emissive face, caches 0) with small
    emissive surfels under the ceiling facing down."""
    box = S.giant_box(rho=0.6, r=0.0, e=0.0, emissive_faces=[], floor_cache=0.0)
    rng = np.random.default_rng(seed)
    pos = np.column_stack([rng.uniform(-0.6, 0.6, n_lamps), rng.uniform(-0.6, 0.6, n_lamps),
                           np.full(n_lamps, 0.9)]).astype(np.float32)
    quat = np.tile(np.array([[0.0, 1.0, 0.0, 0.0]], np.float32), (n_lamps, 1))  # normal -z
    lamps = S.SurfelScene(pos, quat, np.full((n_lamps, 2), 0.03, np.float32), np.full(n_lamps, 0.95, np.float32),
                          np.full((n_lamps, 3), 0.5, np.float32),
                          rng.uniform(20.0, 60.0, (n_lamps, 3)).astype(np.float32), np.ones(n_lamps, np.float32))
    return S.SurfelScene(*[np.concatenate([getattr(box, k), getattr(lamps, k)])
                           for k in ("pos", "quat", "scale", "opacity", "albedo", "radiance", "emissive")])


@pytest.mark.parametrize("B,rr", [(1, 2), (3, 2)])
def test_mis_has_the_plain_expectation(B, rr):
    sc = _lamp_box()
    cam = S.look_at_camera(8, 6, 90.0, (0.0, 0.0, -0.3), (0.3, 0.2, -1.0), (0, 0, 1))
    pix = np.arange(48, dtype=np.int32)
    spp = 1024
    plain = O.render(sc, cam, pix, "pt", spp, max_bounces=B, rr_start=rr, seed=1, want_samples=True,
                     params=O.Params(fp32_eps=0.0))
    mis = O.render(sc, cam, pix, "pt", spp, max_bounces=B, rr_start=rr, seed=2, want_samples=True,
                   params=O.Params(fp32_eps=0.0, mis=True))
    a = plain["samples"].mean(axis=(0, 2))   # per-sample-index average over pixels and channels
    b = mis["samples"].mean(axis=(0, 2))
    ma, mb = a.mean(), b.mean()
    se = math.sqrt(a.var() / a.size + b.var() / b.size)
    assert abs(ma - mb) <= 4.0 * se, (ma, mb, se)
    assert ma > 0
    # the lamps are tiny: emitter sampling cuts the variance by a large factor
    assert b.var() < 0.25 * a.var()


def test_mis_without_emitters_is_plain():
    sc = S.giant_box(rho=0.6, r=0.0, e=0.0, emissive_faces=[], floor_cache=0.0)
    cam = S.look_at_camera(4, 3, 90.0, (0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0, 0, 1))
    pix = np.arange(12, dtype=np.int32)
    a = O.render(sc, cam, pix, "pt", 8, max_bounces=3, seed=4, want_samples=True, params=O.Params(fp32_eps=0.0))
    b = O.render(sc, cam, pix, "pt", 8, max_bounces=3, seed=4, want_samples=True,
                 params=O.Params(fp32_eps=0.0, mis=True))
    np.testing.assert_array_equal(a["samples"], b["samples"])
