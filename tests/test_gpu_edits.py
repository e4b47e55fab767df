"""Scene edits on the GPU: selection and every edit op against their plain
definitions, BVH refit / rebuild correctness (hit sets and renders against
the brute-force oracle on the edited scene), and scene versioning."""
import ctypes
import math

import numpy as np
import pytest

import oracle as O
from parity_utils import compare_samples
from paper_2601_23065_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    from paper_2601_23065_gb300 import api, build
    build.build()
    torch.cuda.init()
    return api


def test_select_box_and_sphere(api):
    sc = S.tiny_room(4096)
    ds = api.DeviceScene.from_host(sc)
    box = [-0.2, -0.3, -0.5, 0.25, 0.1, 0.0]
    got = api.select(ds, "box", box).cpu().numpy()
    p = sc.pos
    want = np.nonzero(np.all((p >= np.array(box[:3], np.float32)) & (p <= np.array(box[3:], np.float32)), 1))[0]
    assert np.array_equal(got, want)
    c, r = np.array([0.1, 0.0, -0.2], np.float32), np.float32(0.3)
    got = api.select(ds, "sphere", list(c) + [float(r)]).cpu().numpy()
    d = p - c
    want = np.nonzero((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]) <= r * r)[0]
    assert np.array_equal(got, want)
    assert api.select(ds, "box", [5, 5, 5, 6, 6, 6]).numel() == 0


def _quat_mul(a, b):
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz, aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx, aw * bz + ax * by - ay * bx + az * bw])


def test_edit_ops_match_definitions(api):
    import torch
    sc = S.tiny_room(4096)
    ds = api.DeviceScene.from_host(sc)
    bvh = api.BVH(ds)
    rng = np.random.default_rng(3)
    idx = np.sort(rng.choice(sc.n, 200, replace=False)).astype(np.int32)
    it = torch.from_numpy(idx).cuda()
    v0 = ds.version
    # toggle emission with new radiance for new emitters
    rad = rng.uniform(1, 10, (200, 3)).astype(np.float32)
    api.apply_edit(ds, bvh, "toggle_emission", it, per_index=torch.from_numpy(rad).cuda())
    e = sc.emissive.copy()
    r = sc.radiance.copy()
    e[idx] = 1 - e[idx]
    became = idx[e[idx] > 0.5]
    r[became] = rad[e[idx] > 0.5]
    np.testing.assert_array_equal(ds.t["emissive"].cpu().numpy(), e)
    np.testing.assert_array_equal(ds.t["radiance"].cpu().numpy(), r)
    assert ds.version == v0 + 1 and bvh.handle.scene_version == ds.version
    # albedo scaling, clamped to [0, 1]
    api.apply_edit(ds, bvh, "scale_albedo", it, value=(1.7, 0.5, 1.2))
    a = sc.albedo.copy()
    a[idx] = np.clip(a[idx] * np.array([1.7, 0.5, 1.2], np.float32), 0, 1)
    np.testing.assert_allclose(ds.t["albedo"].cpu().numpy(), a, rtol=1e-6)
    # translation
    api.apply_edit(ds, bvh, "translate", it, value=(0.01, -0.02, 0.005))
    p = sc.pos.copy()
    p[idx] += np.array([0.01, -0.02, 0.005], np.float32)
    np.testing.assert_allclose(ds.t["pos"].cpu().numpy(), p, atol=1e-7)
    # rigid motion: 30 degrees about z around c, then t
    th = math.radians(30)
    qr = np.array([math.cos(th / 2), 0, 0, math.sin(th / 2)])
    c = np.array([0.1, 0.1, 0.0])
    t = np.array([0.0, 0.02, 0.01])
    api.apply_edit(ds, bvh, "rigid", it, value=tuple(qr) + tuple(c) + tuple(t))
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    p2 = p.astype(np.float64)
    p2[idx] = (p2[idx] - c) @ Rz.T + c + t
    np.testing.assert_allclose(ds.t["pos"].cpu().numpy(), p2, atol=2e-6)
    q = sc.quat.astype(np.float64).copy()
    for k in idx:
        q[k] = _quat_mul(qr, q[k])
    np.testing.assert_allclose(ds.t["quat"].cpu().numpy(), q, atol=2e-6)
    api.sync_status()


def test_refit_and_rebuild_match_oracle(api):
    """After moving surfels (refit) and after a large move (rebuild), the
    BVH returns the brute-force hit sets and the render matches the oracle."""
    import torch
    sc = S.tiny_room(4096)
    ds = api.DeviceScene.from_host(sc)
    bvh = api.BVH(ds)
    sel = api.select(ds, "sphere", [0.1, 0.0, 0.0, 0.25])
    assert sel.numel() > 50
    rebuilt = api.apply_edit(ds, bvh, "translate", sel, value=(0.0, 0.05, -0.03))
    assert not rebuilt
    rng = np.random.default_rng(9)
    for step in range(2):
        host = ds.to_host()
        rays = np.concatenate([rng.uniform(-0.4, 0.4, (2000, 3)), rng.normal(size=(2000, 3))], 1)
        rays[:, 3:] /= np.linalg.norm(rays[:, 3:], axis=1, keepdims=True)
        rays = rays.astype(np.float32)
        out = api.trace_rays(ds, bvh, torch.from_numpy(rays).cuda(), max_hits=64)
        rec_o, nh_o, fl_o, hits_o = O.trace_rays(host, rays.astype(np.float64), max_hits=64)
        clean = fl_o == 0
        assert np.array_equal(out["hits"].cpu().numpy()[clean], hits_o[clean])
        cam = S.horizontal_camera(24, 16, hfov=100.0)
        r = api.Renderer()
        g = r.path_traced(ds, bvh, cam, 4, 2, rr_start=2, seed=1, want_samples=True)["samples"]
        ref = O.render(host, cam, np.arange(24 * 16, dtype=np.int32), "pt", 4, max_bounces=2, rr_start=2, seed=1,
                       want_samples=True)
        ok, st = compare_samples(g.cpu().numpy().reshape(-1, 4, 3), ref["samples"], ref["sample_flags"])
        print(st)
        assert st["lit_compared"] >= 20, st
        assert ok.all(), st
        if step == 0:
            # scattering a random tenth of the surfels breaks the spatial order
            # the tree was built for; the refit's surface-area sum grows past
            # the ratio and the BVH is rebuilt (moving a spatially coherent
            # block would only shift its subtree)
            pick = np.sort(rng.choice(sc.n, sc.n // 10, replace=False)).astype(np.int32)
            rebuilt = api.apply_edit(ds, bvh, "translate", torch.from_numpy(pick).cuda(), value=(0.3, 0.0, 0.0),
                                     rebuild_ratio=1.05)
            assert rebuilt
    api.sync_status()


def test_stale_bvh_is_refused(api):
    import torch
    from paper_2601_23065_gb300 import capi
    sc = S.tiny_room(1024)
    ds = api.DeviceScene.from_host(sc)
    bvh = api.BVH(ds)
    old = capi.Bvh()
    ctypes.memmove(ctypes.byref(old), ctypes.byref(bvh.handle), ctypes.sizeof(capi.Bvh))
    api.apply_edit(ds, bvh, "scale_albedo", torch.arange(10, dtype=torch.int32, device="cuda"), value=(0.5, 0.5, 0.5))
    class Stale:
        params = bvh.params
        handle = old

        def c(self):
            return old
    with pytest.raises(capi.EagptError) as ei:
        api.Renderer().path_traced(ds, Stale(), S.horizontal_camera(8, 8), 1, 1)
    assert ei.value.status == 4
