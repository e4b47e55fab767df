"""Inserting and deleting surfels (the surfel count changes; the BVH is
rebuilt).  The edited scene must equal the host-edited list of surfels field
by field, render bit for bit like a fresh upload of that list, and match the
oracle on it."""
import numpy as np
import pytest

import oracle as O
from paper_2601_23065_gb300 import scenes as S
from parity_utils import compare_samples

pytestmark = pytest.mark.gpu

FIELDS = ("pos", "quat", "scale", "opacity", "albedo", "radiance", "emissive")


@pytest.fixture(scope="module")
def api():
    import torch
    from paper_2601_23065_gb300 import api, build
    build.build()
    torch.cuda.init()
    return api


def _check_against(api, ds, bvh, ref, cam, spp=4, B=3, seed=2):
    import torch
    for k in FIELDS:
        np.testing.assert_array_equal(ds.t[k].cpu().numpy(), getattr(ref, k).astype(np.float32))
    r = api.Renderer()
    a = r.path_traced(ds, bvh, cam, spp, B, rr_start=2, seed=seed, want_samples=True)
    fresh = api.DeviceScene.from_host(ref)
    b = r.path_traced(fresh, api.BVH(fresh), cam, spp, B, rr_start=2, seed=seed)["rgb"]
    api.sync_status()
    assert torch.equal(a["rgb"], b)
    pix = np.arange(0, cam.width * cam.height, 5, dtype=np.int32)
    g = a["samples"].cpu().numpy().reshape(-1, spp, 3)[pix]
    o = O.render(ref, cam, pix, "pt", spp, max_bounces=B, rr_start=2, seed=seed, want_samples=True)
    ok, st = compare_samples(g, o["samples"], o["sample_flags"])
    print(st)
    assert ok.all(), st


def test_delete_keeps_the_rest_in_order(api):
    import torch
    host = S.workload("tiny").scene_fn()
    cam = S.horizontal_camera(40, 30)
    rng = np.random.default_rng(5)
    idx = rng.choice(host.n, host.n // 10, replace=False)
    listed = np.concatenate([idx, idx[:7]])  # duplicates are allowed
    ds = api.DeviceScene.from_host(host)
    bvh = api.BVH(ds)
    v0 = ds.version
    n = api.delete_surfels(ds, bvh, torch.from_numpy(listed.astype(np.int32)))
    keep = np.setdiff1d(np.arange(host.n), idx)
    ref = S.SurfelScene(*[getattr(host, k)[keep] for k in FIELDS])
    assert n == keep.size and ds.version == v0 + 1 and bvh.handle.scene_version == ds.version
    _check_against(api, ds, bvh, ref, cam)


def test_delete_everything_and_out_of_range(api):
    import torch
    host = S.random_small_scene(12, 3)
    ds = api.DeviceScene.from_host(host)
    bvh = api.BVH(ds)
    assert api.delete_surfels(ds, bvh, torch.arange(12, dtype=torch.int32)) == 0
    out = api.Renderer().path_traced(ds, bvh, S.horizontal_camera(8, 6), 2, 2)["rgb"]
    api.sync_status()
    assert torch.count_nonzero(out).item() == 0
    # an index outside [0, n) is skipped and reported; the listed valid one goes
    ds = api.DeviceScene.from_host(host)
    bvh = api.BVH(ds)
    n = api.delete_surfels(ds, bvh, torch.tensor([3, 12, -1], dtype=torch.int32))
    with pytest.raises(api.capi.EagptError):
        api.sync_status()
    assert n == 11
    np.testing.assert_array_equal(ds.t["pos"].cpu().numpy(), np.delete(host.pos, 3, axis=0))


def test_insert_an_object(api):
    """Insert a cluster of 600 surfels (an 'imported object': a ball of
    emitters and reflectors) into the room, then delete part of it again."""
    import torch
    host = S.workload("tiny").scene_fn()
    rng = np.random.default_rng(9)
    m = 600
    obj = S.random_small_scene(m, 21, spread=0.12, emit_frac=0.1)
    obj.pos[:] = obj.pos - np.array([1.0, 0.0, 0.0], np.float32) + np.array([0.25, 0.1, -0.1], np.float32)
    obj.scale[:] = rng.uniform(0.005, 0.02, (m, 2)).astype(np.float32)
    cam = S.horizontal_camera(40, 30)
    ds = api.DeviceScene.from_host(host)
    bvh = api.BVH(ds)
    n = api.insert_surfels(ds, bvh, api.DeviceScene.from_host(obj))
    ref = S.SurfelScene(*[np.concatenate([getattr(host, k), getattr(obj, k)]) for k in FIELDS])
    assert n == host.n + m
    _check_against(api, ds, bvh, ref, cam)
    # delete the first half of the object again: back to a list the host can state
    idx = np.arange(host.n, host.n + m // 2)
    api.delete_surfels(ds, bvh, torch.from_numpy(idx.astype(np.int32)))
    keep = np.setdiff1d(np.arange(host.n + m), idx)
    ref2 = S.SurfelScene(*[getattr(ref, k)[keep] for k in FIELDS])
    _check_against(api, ds, bvh, ref2, cam)


def test_insert_capacity_and_storage_checks(api):
    import ctypes
    import torch
    host = S.random_small_scene(10, 4)
    ds = api.DeviceScene.from_host(host)
    bvh = api.BVH(ds)
    src = api.DeviceScene.from_host(S.random_small_scene(5, 6))
    L = api.capi.lib()
    sm, sc = ds.c(), src.c()
    # capacity smaller than n + m: refused, nothing changes
    st = L.eagpt_insert_surfels(ctypes.byref(sm), 12, ctypes.byref(sc), ctypes.byref(bvh.handle),
                                ctypes.byref(bvh.params), None)
    assert st == 2 and sm.n == 10 and sm.version == 0
    torch.cuda.synchronize()
