"""Path tracing with emitter sampling and MIS on the GPU against the oracle's
same estimator (same Philox draws, sample by sample): per pixel, the mean
over the samples the oracle does not flag agrees within 1e-4."""
import numpy as np
import pytest

import oracle as O
from paper_2601_23065_gb300 import scenes as S
from parity_utils import compare_samples

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    from paper_2601_23065_gb300 import api, build
    build.build()
    torch.cuda.init()
    return api


def _mis_params(api):
    return api.params(flags=api.capi.FLAG_EMITTER_SAMPLING)


def _render(api, scene, cam, spp, B, rr, seed, mis=True, ws_cap=None):
    ds = api.DeviceScene.from_host(scene)
    bvh = api.BVH(ds)
    r = api.Renderer(max_workspace_bytes=ws_cap)
    prm = _mis_params(api) if mis else None
    out = r.path_traced(ds, bvh, cam, spp, B, rr_start=rr, seed=seed, prm=prm, want_samples=True)
    api.sync_status()
    return out


def _parity(api, scene, cam, spp, B, rr, seed, pixels=None, max_flagged=0.1):
    out = _render(api, scene, cam, spp, B, rr, seed)
    npix = cam.width * cam.height
    pix = np.arange(npix, dtype=np.int32) if pixels is None else np.asarray(pixels, np.int32)
    g = out["samples"].cpu().numpy().reshape(npix, spp, 3)[pix]
    ref = O.render(scene, cam, pix, "pt", spp, max_bounces=B, rr_start=rr, seed=seed, want_samples=True,
                   params=O.Params(mis=True))
    ok, st = compare_samples(g, ref["samples"], ref["sample_flags"])
    print(st)
    assert st["flagged_samples"] < max_flagged
    assert ok.all(), st
    np.testing.assert_allclose(out["rgb"].cpu().numpy().reshape(npix, 3)[pix], g.mean(1), rtol=2e-6, atol=1e-7)
    return out, ref


def _lamp_box(n_lamps=6, seed=3):
    box = S.giant_box(rho=0.6, r=0.0, e=0.0, emissive_faces=[], floor_cache=0.0)
    rng = np.random.default_rng(seed)
    pos = np.column_stack([rng.uniform(-0.6, 0.6, n_lamps), rng.uniform(-0.6, 0.6, n_lamps),
                           np.full(n_lamps, 0.9)]).astype(np.float32)
    quat = np.tile(np.array([[0.0, 1.0, 0.0, 0.0]], np.float32), (n_lamps, 1))
    lamps = S.SurfelScene(pos, quat, np.full((n_lamps, 2), 0.03, np.float32), np.full(n_lamps, 0.95, np.float32),
                          np.full((n_lamps, 3), 0.5, np.float32),
                          rng.uniform(20.0, 60.0, (n_lamps, 3)).astype(np.float32), np.ones(n_lamps, np.float32))
    return S.SurfelScene(*[np.concatenate([getattr(box, k), getattr(lamps, k)])
                           for k in ("pos", "quat", "scale", "opacity", "albedo", "radiance", "emissive")])


@pytest.mark.parametrize("B", [1, 3])
def test_mis_tiny_room(api, B):
    # every reflection adds an emitter-sample segment, and the MIS pdfs
    # depend on the blended normal directly: more samples are FP32-sensitive
    # than in plain path tracing
    wl = S.workload("tiny")
    _parity(api, wl.scene_fn(), wl.camera, 4, B, 2, 0, max_flagged=0.35)


def test_mis_lamp_box(api):
    # the box's axis-aligned walls put the basis-branch decision (normal z = 0)
    # on a third of the samples, with or without emitter sampling
    cam = S.look_at_camera(16, 12, 90.0, (0.0, 0.0, -0.3), (0.3, 0.2, -1.0), (0, 0, 1))
    _parity(api, _lamp_box(), cam, 8, 2, 2, 5, max_flagged=0.7)


def test_mis_ragged_multibounce(api):
    cam = S.horizontal_camera(37, 23, hfov=100.0)
    _parity(api, S.tiny_room(4096), cam, 6, 3, 2, 7, max_flagged=0.35)


def test_mis_without_emitters_equals_plain(api):
    import torch
    sc = S.giant_box(rho=0.6, r=0.0, e=0.0, emissive_faces=[], floor_cache=0.3)
    cam = S.horizontal_camera(20, 14)
    a = _render(api, sc, cam, 4, 3, 2, 1, mis=True)["rgb"]
    b = _render(api, sc, cam, 4, 3, 2, 1, mis=False)["rgb"]
    assert torch.equal(a, b)


def test_mis_deterministic_and_pass_independent(api):
    import torch
    wl = S.workload("tiny")
    cam = S.horizontal_camera(24, 16)
    sc = wl.scene_fn()
    a = _render(api, sc, cam, 8, 3, 2, 11)
    b = _render(api, sc, cam, 8, 3, 2, 11)
    assert torch.equal(a["rgb"], b["rgb"])
    ws_min = api.capi.lib().eagpt_render_workspace_min_bytes(api.camera(cam), 8, 2)
    c = _render(api, sc, cam, 8, 3, 2, 11, ws_cap=ws_min)   # one sample per pass
    assert torch.equal(a["rgb"], c["rgb"])


def test_mis_follows_emission_edits(api):
    """Toggling emitters rebuilds the emitter table: the edited scene's MIS
    render matches the oracle on the edited scene."""
    import torch
    wl = S.workload("tiny")
    host = wl.scene_fn()
    cam = S.horizontal_camera(24, 16)
    ds = api.DeviceScene.from_host(host)
    bvh = api.BVH(ds)
    rng = np.random.default_rng(2)
    idx = rng.choice(host.n, 60, replace=False).astype(np.int32)
    rad = rng.uniform(1.0, 10.0, (60, 3)).astype(np.float32)
    api.apply_edit(ds, bvh, "toggle_emission", torch.from_numpy(idx).cuda(), per_index=torch.from_numpy(rad).cuda())
    out = api.Renderer().path_traced(ds, bvh, cam, 4, 2, rr_start=2, seed=3, prm=_mis_params(api),
                                     want_samples=True)
    api.sync_status()
    edited = ds.to_host()
    pix = np.arange(cam.width * cam.height, dtype=np.int32)
    ref = O.render(edited, cam, pix, "pt", 4, max_bounces=2, rr_start=2, seed=3, want_samples=True,
                   params=O.Params(mis=True))
    g = out["samples"].cpu().numpy().reshape(-1, 4, 3)
    ok, st = compare_samples(g, ref["samples"], ref["sample_flags"])
    print(st)
    assert ok.all(), st
