"""Level of detail on the GPU against the oracle, through the C ABI.

* The merge (eagpt_build_lod): group keys bit for bit (FP32 decisions on both
  sides), and every merged surfel (centre, Gaussian covariance, normal,
  opacity, albedo, radiance, emissive term) within FP32 accuracy of the
  oracle's FP64 merge, on the tiny (5 and 2 cm cells) and medium (5 cm)
  rooms in full and on 2,000
  sampled groups of the 6M-surfel layout (scales x0.300, keys of all 6M).
* The render (eagpt_render_path_traced_lod): sample by sample against the
  oracle's level-of-detail render on the same two scenes (the merged scene is
  the oracle's, cast to FP32, on both sides), with the parity rule of the
  other path-tracing tests; bit for bit the plain render when the level of
  detail starts after the last bounce or is the scene itself.
* On the medium room the merged bounces blend fewer surfels per segment.
"""
import numpy as np
import pytest

import oracle as O
from oracle import lod as L
from parity_utils import compare_samples, primary_vertices
from paper_2601_23065_gb300 import scenes as S

pytestmark = pytest.mark.gpu

# grid corners that put the room walls in mid-cell for 5 cm cells
TINY_ORIGIN = (-0.6125, -0.6125, -0.6125)
MEDIUM_ORIGIN = (-2.6125, -2.1125, -1.6125)
LARGE_ORIGIN = (-7.6125, -2.1125, -1.6125)


@pytest.fixture(scope="module")
def eg():
    import torch
    from paper_2601_23065_gb300 import api, build
    build.build()
    torch.cuda.init()
    return api


def _check_groups(gpu, ref):
    """Merged surfels of the GPU (dict of numpy arrays) against the oracle's
    merge (dict from oracle.lod.merge or merge_group), row by row."""
    n = len(ref["pos"])
    p_ref = np.asarray(ref["pos"])
    assert np.all(np.abs(gpu["pos"] - p_ref) <= 2e-6 * np.maximum(1.0, np.abs(p_ref).max(1, keepdims=True)))
    tu, tv, nn = L.frames(gpu["quat"].astype(np.float64))
    s = gpu["scale"].astype(np.float64)
    cov = s[:, 0, None, None] ** 2 * tu[:, :, None] * tu[:, None, :] + s[:, 1, None, None] ** 2 * tv[:, :, None] * tv[:, None, :]
    cref = np.asarray(ref["cov"])
    big = np.abs(cref).max((1, 2))
    err = np.abs(cov - cref).max((1, 2)) / big
    assert err.max() <= 1e-4, ("covariance", float(err.max()), int(err.argmax()))
    assert np.abs(nn - np.asarray(ref["normal"])).max() <= 1e-5
    for k, rel in (("opacity", 1e-4), ("albedo", 1e-5), ("radiance", 1e-5), ("emissive", 1e-5)):
        g = gpu[k].astype(np.float64)
        r = np.asarray(ref[k], np.float64).reshape(g.shape)
        assert np.all(np.abs(g - r) <= rel * np.abs(r) + 1e-7), (k, float(np.abs(g - r).max()))
    return n


def _gpu_merge(eg, scene, origin, h):
    ds = eg.DeviceScene.from_host(scene)
    merged, keys = eg.build_lod(ds, origin, h, want_keys=True)
    eg.sync_status()
    return {k: v.cpu().numpy() for k, v in merged.t.items()}, keys.cpu().numpy().astype(np.uint64)


@pytest.mark.parametrize("name", ["tiny", "medium"])
def test_merge_matches_oracle(eg, name):
    scene, origin = (S.tiny_room(4096), TINY_ORIGIN) if name == "tiny" else (S.medium_room(), MEDIUM_ORIGIN)
    for h in ((0.05, 0.02) if name == "tiny" else (0.05,)):
        gpu, keys = _gpu_merge(eg, scene, origin, h)
        ref = L.merge(scene, origin, h)
        assert np.array_equal(keys, ref["keys"])
        n = _check_groups(gpu, ref)
        print(name, h, "groups", n, "of", scene.n)
        assert n < scene.n


def test_merge_large_layout_sampled(eg):
    """6M surfels: every group key, and 2,000 sampled groups merged by the
    oracle one by one."""
    scene = S.large_layout()
    h = 0.05
    gpu, keys = _gpu_merge(eg, scene, LARGE_ORIGIN, h)
    kref, axis = L.group_keys(scene.pos, scene.quat, scene.emissive, LARGE_ORIGIN, h)
    order = np.argsort(kref, kind="stable")
    ks = kref[order]
    starts = np.flatnonzero(np.concatenate([[True], ks[1:] != ks[:-1]]))
    ends = np.append(starts[1:], len(ks))
    assert np.array_equal(keys, ks[starts])
    rng = np.random.default_rng(17)
    pick = np.sort(rng.choice(len(starts), 2000, replace=False))
    tu, tv, n = L.frames(scene.quat)
    cols = {k: [] for k in ("pos", "cov", "normal", "opacity", "albedo", "radiance", "emissive")}
    f64 = lambda a: np.asarray(a, np.float64)
    for g in pick:
        idx = order[starts[g]:ends[g]]
        r = L.merge_group(f64(scene.pos[idx]), tu[idx], tv[idx], n[idx], f64(scene.scale[idx]),
                          f64(scene.opacity[idx]), f64(scene.albedo[idx]), f64(scene.radiance[idx]),
                          f64(scene.emissive[idx]), int(axis[idx[0]]))
        for k in cols:
            cols[k].append(r[k])
    _check_groups({k: v[pick] for k, v in gpu.items()}, {k: np.array(v) for k, v in cols.items()})
    print("large layout groups", len(starts), "of", scene.n)


def _lod_parity(eg, scene, origin, h, cam, spp, B, rr, lod_from, seed):
    """GPU level-of-detail render vs the oracle's, both on the oracle's merged
    scene cast to FP32."""
    coarse = L.to_scene(L.merge(scene, origin, h), S.SurfelScene)
    ds = eg.DeviceScene.from_host(scene)
    bvh = eg.BVH(ds)
    cds = eg.DeviceScene.from_host(coarse)
    lod = eg.LevelOfDetail.of(cds, eg.BVH(cds))
    out = eg.Renderer().path_traced_lod(ds, bvh, lod, lod_from, cam, spp, B, rr_start=rr, seed=seed,
                                        want_samples=True)
    eg.sync_status()
    npix = cam.width * cam.height
    pix = np.arange(npix, dtype=np.int32)
    g_s = out["samples"].cpu().numpy().reshape(npix, spp, 3)
    osc = O.OracleScene(scene)
    ref = O.render_lod(osc, O.OracleScene(coarse), lod_from, cam, pix, spp, max_bounces=B, rr_start=rr, seed=seed,
                       want_samples=True, want_dev=True)
    _X, _N, emit, _hit = primary_vertices(osc, cam, pix)
    ok, st = compare_samples(g_s, ref["samples"], ref["sample_flags"], primary_emitter=emit,
                             sample_dev=ref["sample_dev"])
    np.testing.assert_allclose(out["rgb"].cpu().numpy().reshape(npix, 3), g_s.mean(1), rtol=2e-6, atol=1e-7)
    return ok, st


@pytest.mark.parametrize("lod_from", [1, 2])
def test_render_matches_oracle_tiny_room(eg, lod_from):
    """Tiny room, 48x40, 6 spp, 3 bounces with roulette from bounce 2."""
    cam = S.horizontal_camera(48, 40, hfov=100.0)
    ok, st = _lod_parity(eg, S.tiny_room(4096), TINY_ORIGIN, 0.05, cam, 6, 3, 2, lod_from, 3)
    print(lod_from, st)
    assert st["lit_bounced_compared"] >= 200, st
    assert ok.all(), st


def test_render_reduces_to_the_plain_render(eg):
    """Bit for bit the plain render when the level of detail starts after the
    last bounce, or is the scene itself."""
    import torch
    scene = S.tiny_room(4096)
    ds = eg.DeviceScene.from_host(scene)
    bvh = eg.BVH(ds)
    cam = S.horizontal_camera(64, 48, hfov=100.0)
    r = eg.Renderer()
    ref = r.path_traced(ds, bvh, cam, 8, 3, rr_start=2, seed=9)["rgb"].clone()
    lod = eg.LevelOfDetail(ds, TINY_ORIGIN, 0.05)
    late = r.path_traced_lod(ds, bvh, lod, 4, cam, 8, 3, rr_start=2, seed=9)["rgb"].clone()
    same = eg.LevelOfDetail.of(ds, bvh)
    itself = r.path_traced_lod(ds, bvh, same, 1, cam, 8, 3, rr_start=2, seed=9)["rgb"].clone()
    merged = r.path_traced_lod(ds, bvh, lod, 2, cam, 8, 3, rr_start=2, seed=9)["rgb"].clone()
    eg.sync_status()
    assert torch.equal(late, ref) and torch.equal(itself, ref)
    assert not torch.equal(merged, ref)


def test_fewer_blended_surfels_per_merged_segment(eg):
    """Medium room, 5 cm cells: the bounce segments that trace the merged
    surfels blend fewer of them than the full scene's segments do, and the
    image stays close to the full-detail one."""
    scene = S.medium_room()
    ds = eg.DeviceScene.from_host(scene)
    bvh = eg.BVH(ds)
    lod = eg.LevelOfDetail(ds, MEDIUM_ORIGIN, 0.05)
    cam = S.horizontal_camera(256, 256, hfov=90.0)
    r = eg.Renderer()
    full = r.path_traced(ds, bvh, cam, 16, 4, rr_start=2, seed=1, want_stats=True)
    fs = full["stats"].cpu().numpy().copy()
    frgb = full["rgb"].cpu().numpy().copy()
    coarse = r.path_traced_lod(ds, bvh, lod, 1, cam, 16, 4, rr_start=2, seed=1, want_stats=True)
    cs = coarse["stats"].cpu().numpy().copy()
    crgb = coarse["rgb"].cpu().numpy().copy()
    eg.sync_status()
    assert lod.scene.n < scene.n
    # stats: [1] secondary segments, [3] their blended hits, [5] their surfel tests
    per = lambda st, k: st[k] / max(st[1], 1)
    print("secondary segments full", fs[1], "lod", cs[1], "| blended per segment", per(fs, 3), per(cs, 3),
          "| surfel tests per segment", per(fs, 5), per(cs, 5))
    assert per(cs, 3) < per(fs, 3)
    assert np.isfinite(crgb).all() and crgb.mean() > 0
    rel = abs(crgb.mean() - frgb.mean()) / frgb.mean()
    print("mean image full", frgb.mean(), "lod", crgb.mean(), "relative difference", rel)
    assert rel < 0.25
