"""GPU path vs the FP64 oracle, through the C ABI.

Inputs are seeded and identical on both sides.  Radiance must agree within
1e-4 relative per channel (floor 1e-3 of the mean radiance), sample by
sample, on every sample the oracle does not flag as near a discrete decision
boundary or ill-conditioned in FP32; hit index sets of caller rays must be
identical away from flagged decisions.  Each test prints how many samples
(and how many lit ones) it compared.
"""
import numpy as np
import pytest

import oracle as O
from parity_utils import (COND_DEV_K, compare_samples, lit_pixels, primary_vertices, radiance_close,
                          secondary_rays)
from paper_2601_23065_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eg():
    import torch
    from paper_2601_23065_gb300 import api, build
    build.build()
    torch.cuda.init()
    return api


def _setup(eg, scene):
    ds = eg.DeviceScene.from_host(scene)
    bvh = eg.BVH(ds)
    return ds, bvh


def _random_rays(rng, m, lo, hi):
    o = rng.uniform(lo, hi, (m, 3))
    d = rng.normal(size=(m, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return np.concatenate([o, d], 1).astype(np.float32)


@pytest.mark.parametrize("n", [1, 3, 4, 5, 17, 4096])
def test_trace_rays_hit_sets(eg, n):
    """Caller rays: blended records within tolerance and hit lists identical
    to the brute-force oracle on every ray without a flagged decision."""
    import torch
    scene = S.tiny_room(4096) if n == 4096 else S.random_small_scene(n, 40 + n, spread=0.4)
    ds, bvh = _setup(eg, scene)
    rng = np.random.default_rng(n)
    rays = _random_rays(rng, 3000, -0.45, 0.45) if n == 4096 else _random_rays(rng, 3000, -0.2, 0.2)
    if n != 4096:
        rays[:, 3:] = np.abs(rays[:, 3:]) * np.array([1, 0.3, 0.3]) + np.array([0.5, 0, 0])
        rays[:, 3:] /= np.linalg.norm(rays[:, 3:], axis=1, keepdims=True)
    rays_d = torch.from_numpy(rays).cuda()
    for mode in (0, 1):
        out = eg.trace_rays(ds, bvh, rays_d, mode=mode, max_hits=64)
        rec_g = out["rec"].cpu().numpy()
        hits_g = out["hits"].cpu().numpy()
        nh_g = out["nhits"].cpu().numpy()
        rec_o, nh_o, fl_o, hits_o = O.trace_rays(scene, rays.astype(np.float64), mode=mode, max_hits=64)
        clean = fl_o == 0
        assert clean.mean() > 0.9
        assert np.array_equal(nh_g[clean], nh_o[clean])
        assert np.array_equal(hits_g[clean], hits_o[clean])
        hit = clean & (nh_o > 0)
        for cols in (slice(4, 7), slice(8, 11), slice(11, 12), slice(7, 8)):
            ok = radiance_close(rec_g[hit, cols], rec_o[hit, cols], rel=1e-4, floor_frac=1e-3)
            assert ok.all(), (cols, np.argwhere(~ok)[:5])
        np.testing.assert_allclose(rec_g[hit, 0:3], rec_o[hit, 0:3], atol=2e-5)
        np.testing.assert_allclose(rec_g[hit, 3], rec_o[hit, 3], rtol=1e-4, atol=1e-6)
        assert np.all(rec_g[~(nh_o > 0) & clean, 11] == 0)
    eg.sync_status()


def test_primary_records_tiny_room(eg):
    wl = S.workload("tiny")
    scene = wl.scene_fn()
    ds, bvh = _setup(eg, scene)
    r = eg.Renderer()
    for kind, mode in (("pt", 1), ("single", 0)):
        if kind == "pt":
            out = r.path_traced(ds, bvh, wl.camera, 1, 1, want_aux=True)
        else:
            out = r.single_bounce(ds, bvh, wl.camera, 1, want_aux=True)
        aux = out["aux"].cpu().numpy().reshape(-1, 12)
        pix = np.arange(64 * 64, dtype=np.int32)
        rec, fl = O.primary(scene, wl.camera, pix, mode=mode)
        clean = fl == 0
        assert clean.mean() > 0.97
        for cols in (slice(4, 7), slice(7, 8), slice(8, 11), slice(11, 12)):
            assert radiance_close(aux[clean, cols], rec[clean, cols]).all()
        np.testing.assert_allclose(aux[clean, 0:3], rec[clean, 0:3], atol=2e-5)
        np.testing.assert_allclose(aux[clean, 3], rec[clean, 3], rtol=1e-4)


def _parity(eg, scene, cam, kind, spp, B, rr, seed, pixels=None, ws_cap=None):
    ds, bvh = _setup(eg, scene)
    r = eg.Renderer(max_workspace_bytes=ws_cap)
    if kind == "pt":
        out = r.path_traced(ds, bvh, cam, spp, B, rr_start=rr, seed=seed, want_samples=True)
    else:
        out = r.single_bounce(ds, bvh, cam, spp, seed=seed, want_samples=True)
    eg.sync_status()
    npix = cam.width * cam.height
    pix = np.arange(npix, dtype=np.int32) if pixels is None else np.asarray(pixels, np.int32)
    g_s = out["samples"].cpu().numpy().reshape(npix, spp, 3)[pix]
    g_rgb = out["rgb"].cpu().numpy().reshape(npix, 3)[pix]
    osc = O.OracleScene(scene)
    ref = O.render(osc, cam, pix, kind, spp, max_bounces=B, rr_start=rr, seed=seed, want_samples=True,
                   want_dev=True)
    _X, _N, emit, _hit = primary_vertices(osc, cam, pix)
    ok, st = compare_samples(g_s, ref["samples"], ref["sample_flags"], primary_emitter=emit,
                             sample_dev=ref["sample_dev"])
    # the image is the sample mean
    np.testing.assert_allclose(g_rgb, g_s.mean(1), rtol=2e-6, atol=1e-7)
    return ok, st, out, ref


@pytest.mark.parametrize("kind", ["pt", "single"])
def test_tiny_room_full_image(eg, kind):
    """Tiny room (4,096 surfels), 64x64, 4 spp, 1 bounce: every pixel."""
    wl = S.workload("tiny")
    ok, st, out, ref = _parity(eg, wl.scene_fn(), wl.camera, kind, 4, 1, 2, 0)
    print(kind, st)
    # single bounce reads every surfel's radiance cache, so more samples are
    # FP32-sensitive than in path tracing (which reads emitters only)
    assert st["flagged_samples"] < (0.1 if kind == "pt" else 0.25)
    assert st["lit_bounced_compared"] >= (400 if kind == "pt" else 10000), st
    assert ok.all(), st


def test_tiny_room_multibounce_ragged(eg):
    """Ragged 37x23 image, 3 bounces with roulette from bounce 2, 6 spp."""
    cam = S.horizontal_camera(37, 23, hfov=100.0)
    ok, st, _, _ = _parity(eg, S.tiny_room(4096), cam, "pt", 6, 3, 2, 7)
    print(st)
    assert st["lit_bounced_compared"] >= 200, st
    assert ok.all(), st


def test_batch_size_and_determinism(eg):
    """One pass over all samples or one sample per pass: bitwise equal; two
    runs: bitwise equal."""
    import torch
    wl = S.workload("tiny")
    ds, bvh = _setup(eg, wl.scene_fn())
    big = eg.Renderer()
    cam = S.horizontal_camera(48, 40)
    a = big.path_traced(ds, bvh, cam, 8, 3, rr_start=2, seed=5)["rgb"].clone()
    b = big.path_traced(ds, bvh, cam, 8, 3, rr_start=2, seed=5)["rgb"].clone()
    small = eg.Renderer(max_workspace_bytes=1)
    c = small.path_traced(ds, bvh, cam, 8, 3, rr_start=2, seed=5)["rgb"].clone()
    assert torch.equal(a, b) and torch.equal(a, c)
    d = big.path_traced(ds, bvh, cam, 8, 3, rr_start=2, seed=6)["rgb"]
    assert not torch.equal(a, d)


def test_floor_reflector_room_gpu(eg):
    """Closed-form room (see the oracle pins): wall pixels L_e A, floor pixels
    rho_f A L_e A for any bounce limit >= 1."""
    sc = S.giant_box(rho=0.5, r=2.0, emissive_faces=[0, 1, 2, 3, 5], floor_rho=0.3, floor_cache=0.7, gap=1e-6)
    cam = S.look_at_camera(16, 16, 100.0, (0, 0, 0), (1, 0, -1), (0, 0, 1))
    ds, bvh = _setup(eg, sc)
    r = eg.Renderer()
    ref = O.render(sc, cam, np.arange(256, dtype=np.int32), "pt", 4, max_bounces=3)["rgb"]
    vals = set(np.round(ref[:, 0], 6))
    assert len(vals) == 2
    for B in (1, 3):
        g = r.path_traced(ds, bvh, cam, 4, B, rr_start=100)["rgb"].cpu().numpy().reshape(-1, 3)
        np.testing.assert_allclose(g, ref, rtol=2e-6)


def test_edge_cases(eg):
    import torch
    cam = S.horizontal_camera(5, 3)
    empty = S.SurfelScene(*[np.zeros((0,) + s, np.float32) for s in [(3,), (4,), (2,), (), (3,), (3,), ()]])
    ds, bvh = _setup(eg, empty)
    r = eg.Renderer()
    out = r.path_traced(ds, bvh, cam, 2, 3)["rgb"]
    assert torch.count_nonzero(out) == 0
    # one pixel, one sample, no bounce: emitters only
    one = S.horizontal_camera(1, 1)
    sc = S.tiny_room(4096)
    ds, bvh = _setup(eg, sc)
    g = r.path_traced(ds, bvh, one, 1, 0)["rgb"].cpu().numpy().reshape(1, 3)
    ref = O.render(sc, one, np.zeros(1, np.int32), "pt", 1, max_bounces=0)["rgb"]
    assert radiance_close(g, ref).all()
    eg.sync_status()


@pytest.mark.slow
def test_medium_room_full_size_lit_pixels(eg):
    """Medium room at full size (200k surfels, 512x512, 64 spp, 4 bounces,
    roulette from bounce 2) in the benchmark's launch configuration.  The
    room is dark (small ceiling emitters: about 1 % of random samples carry
    light), so the oracle picks, from 16,000 random pixels, the 2,560 whose
    primary vertex has the largest form factor to the emitters (unflagged
    primary segments first), and computes them one by one.  Every unflagged
    sample must match, every sample flagged only as ill-conditioned must
    match within the bound + 8 x its conditioning spread, the GPU and the
    oracle must agree on which unflagged samples are lit, and at least 1,000
    lit samples whose light came through a bounce are compared."""
    wl = S.workload("medium")
    scene = wl.scene_fn()
    pix = lit_pixels(O.OracleScene(scene), wl.camera, 2560, 16000)
    ok, st, out, ref = _parity(eg, scene, wl.camera, "pt", wl.spp, wl.max_bounces, wl.rr_start, 0, pixels=pix)
    print(st)
    clean = ref["sample_flags"] == 0
    lit_ref = np.abs(ref["samples"]).max(-1) > 0
    g_s = out["samples"].cpu().numpy().reshape(512 * 512, wl.spp, 3)[pix]
    lit_gpu = np.abs(g_s).max(-1) > 0
    assert np.array_equal(lit_ref[clean], lit_gpu[clean])
    assert st["lit_bounced_compared"] >= 15, st
    assert st["lit_bounced_compared"] + st["lit_bounced_cond_compared"] >= 1000, st
    assert ok.all(), st


@pytest.mark.slow
def test_large_layout_lit_pixels(eg):
    """Three-room layout at full size (6M surfels, surfel scales x0.30 of the
    medium room's law, 1920x1080, 5 bounces, roulette from bounce 2) at
    4 spp: the Philox counters make these the first 4 samples of the full
    1024-spp frame.  The oracle picks 96 of 1,500 random pixels by form
    factor to the emitters and computes them one by one; the GPU image must
    carry light, every unflagged sample must match, and the two sides must
    agree on which unflagged samples are lit."""
    wl = S.workload("large")
    scene = wl.scene_fn()
    npix = wl.camera.width * wl.camera.height
    pix = lit_pixels(O.OracleScene(scene), wl.camera, 96, 1500)
    ok, st, out, ref = _parity(eg, scene, wl.camera, "pt", 4, wl.max_bounces, wl.rr_start, 0, pixels=pix)
    print(st)
    g_all = out["samples"].cpu().numpy().reshape(npix, 4, 3)
    assert (np.abs(g_all).max(-1) > 0).mean() > 1e-3
    clean = ref["sample_flags"] == 0
    lit_ref = np.abs(ref["samples"]).max(-1) > 0
    lit_gpu = np.abs(g_all[pix]).max(-1) > 0
    assert np.array_equal(lit_ref[clean], lit_gpu[clean])
    assert ok.all(), st


@pytest.mark.slow
def test_serving_room_full_size_lit_pixels(eg):
    """Path tracing in the serving room at full size (3M surfels, scales
    x0.436, 10x8x3 m), a 512x512 view from the room centre, 16 spp,
    3 bounces; the oracle picks 48 of 800 random pixels by form factor to
    the emitters."""
    wl = S.workload("serving")
    scene = wl.scene_fn()
    pix = lit_pixels(O.OracleScene(scene), wl.camera, 48, 800)
    ok, st, out, ref = _parity(eg, scene, wl.camera, "pt", wl.spp, wl.max_bounces, wl.rr_start, 0, pixels=pix)
    print(st)
    clean = ref["sample_flags"] == 0
    lit_ref = np.abs(ref["samples"]).max(-1) > 0
    g_s = out["samples"].cpu().numpy().reshape(-1, wl.spp, 3)[pix]
    assert np.array_equal(lit_ref[clean], np.abs(g_s).max(-1)[clean] > 0)
    assert ok.all(), st


@pytest.mark.slow
@pytest.mark.parametrize("name,n_rays", [("medium", 3000), ("serving", 3000), ("large", 3000)])
def test_full_size_bounce_segments(eg, name, n_rays):
    """Segments shaped like the path tracer's bounces, traced through the full
    scenes of the medium room (200k surfels), the serving room (3M, scales
    x0.436) and the large layout (6M, scales x0.30): from the oracle's primary
    vertices of random pixels, origin X + 1e-3 N~, three quarters aimed at a
    nearby emitter surfel and the rest cosine-distributed about N~.  Path
    tracing's blend (non-emitter radiance dropped): per ray without a
    flagged decision, the blended surfel list must equal the oracle's
    brute-force list; per ray that is also well conditioned in FP32 the
    blended record (N~, D~, R, E, P, A) must match within 1e-4, and per ray
    flagged only as ill-conditioned (its record moves under FP32-scale
    perturbations, its surfel list does not) within the same bound + 8 x
    the oracle's spread of that column.  At least 1,000 lit segments are
    compared per scene."""
    import torch
    wl = S.workload(name)
    scene = wl.scene_fn()
    osc = O.OracleScene(scene)
    rays = secondary_rays(osc, wl.camera, n_rays)
    ds, bvh = _setup(eg, scene)
    out = eg.trace_rays(ds, bvh, torch.from_numpy(rays).cuda(), mode=1, max_hits=96)
    eg.sync_status()
    rec_g, hits_g, nh_g = out["rec"].cpu().numpy(), out["hits"].cpu().numpy(), out["nhits"].cpu().numpy()
    rec_o, nh_o, fl_o, hits_o, dev_o = O.trace_rays(osc, rays.astype(np.float64), mode=1, max_hits=96,
                                                     want_dev=True)
    decided = (fl_o & ~np.uint32(O.FLAGS["cond"])) == 0
    clean = fl_o == 0
    cond = (fl_o == O.FLAGS["cond"]) & np.isfinite(dev_o).all(1)
    lit_o = rec_o[:, 4:7].max(1) > 0
    print(name, "rays", len(rays), "hit lists compared", int(decided.sum()), "records compared", int(clean.sum()),
          "lit", int((clean & lit_o).sum()), "ill-conditioned records compared", int(cond.sum()),
          "lit", int((cond & lit_o).sum()), "lit (any flags)", int(lit_o.sum()),
          "mean hits", float(nh_o[decided].mean()))
    assert (clean & lit_o).sum() + (cond & lit_o).sum() >= 1000
    assert np.array_equal(nh_g[decided], nh_o[decided])
    assert np.array_equal(hits_g[decided], hits_o[decided])
    hit = clean & (nh_o > 0)
    hc = cond & (nh_o > 0)
    K = COND_DEV_K
    for cols in (slice(4, 7), slice(8, 11), slice(11, 12), slice(7, 8)):
        ok = radiance_close(rec_g[hit, cols], rec_o[hit, cols], rel=1e-4, floor_frac=1e-3)
        assert ok.all(), (cols, np.argwhere(~ok)[:5])
        m = float(np.mean(np.abs(rec_o[hit, cols])))
        r, g, d = rec_o[hc, cols], rec_g[hc, cols].astype(np.float64), dev_o[hc, cols]
        okc = (np.abs(g - r) <= 1e-4 * np.maximum(np.abs(r), 1e-3 * m) + K * d).all(1)
        assert okc.all(), (cols, np.argwhere(~okc)[:5])
    np.testing.assert_allclose(rec_g[hit, 0:3], rec_o[hit, 0:3], atol=2e-5)
    np.testing.assert_allclose(rec_g[hit, 3], rec_o[hit, 3], rtol=1e-4, atol=1e-6)
    r, g, d = rec_o[hc, 0:4], rec_g[hc, 0:4].astype(np.float64), dev_o[hc, 0:4]
    tol = np.concatenate([np.full((len(r), 3), 2e-5), 1e-4 * np.abs(r[:, 3:4]) + 1e-6], 1)
    okc = (np.abs(g - r) <= tol + K * d).all(1)
    assert okc.all(), np.argwhere(~okc)[:5]


@pytest.mark.slow
def test_diff_room_forward_crop(eg):
    """Single-bounce forward (Eq. 6) of the differentiable workload at full
    size (1M surfels, scales x0.447, 800x800, 16 spp) on the 16x16 crop of
    the image centre the gradient tests use: every sample the oracle does not
    flag must match.  Both segments of a sample blend dozens of thin surfels
    and every blended cache contributes, so almost all samples are
    ill-conditioned in FP32 (about 98 %): the few dozen left are compared at
    the bound, and the ill-conditioned ones whose conditioning runs change no
    discrete outcome (about half) at the bound + 8 x their spread."""
    wl = S.workload("diff")
    cam = wl.camera
    crop = np.array([(y * cam.width + x) for y in range(392, 408) for x in range(392, 408)], np.int32)
    ok, st, _out, _ref = _parity(eg, wl.scene_fn(), cam, "single", wl.spp, 1, 2, 0, pixels=crop)
    print(st)
    assert st["compared"] >= 40, st
    assert st["compared"] + st["cond_compared"] >= 1000, st
    assert ok.all(), st
