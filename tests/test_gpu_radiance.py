"""0-bounce render of the radiant scene (Sec. 3.2: each pixel shows the blended
radiance R of its primary segment) and its hand-written adjoint, GPU vs the
FP64 oracle.  The oracle's radiance gradient is pinned to central finite
differences in the CPU tests.  Forward: per pixel within 1e-4 relative on the
pixels the oracle does not flag; backward: relative error per parameter group
<= 1e-3 with flagged pixels weighted 0 on both sides."""
import numpy as np
import pytest

import oracle as O
from parity_utils import grad_errors, oracle_grad_with_conditioning
from paper_2601_23065_gb300 import scenes as S
from parity_utils import radiance_close

pytestmark = pytest.mark.gpu

GROUPS = {"pos": (0, 3), "quat": (3, 7), "scale": (7, 9), "opacity": (9, 10), "radiance": (13, 16)}


@pytest.fixture(scope="module")
def api():
    import torch
    from paper_2601_23065_gb300 import api, build
    build.build()
    torch.cuda.init()
    return api


def _forward(api, scene, cam):
    ds = api.DeviceScene.from_host(scene)
    bvh = api.BVH(ds)
    out = api.radiance(ds, bvh, cam, want_aux=True)
    api.sync_status()
    return out["rgb"].cpu().numpy().reshape(-1, 3), out["aux"].cpu().numpy().reshape(-1, 12)


@pytest.mark.parametrize("size", [(64, 64), (37, 23)])
def test_radiance_matches_oracle_tiny_room(api, size):
    wl = S.workload("tiny")
    scene = wl.scene_fn()
    cam = wl.camera if size == (64, 64) else S.horizontal_camera(*size)
    rgb, aux = _forward(api, scene, cam)
    pix = np.arange(cam.width * cam.height, dtype=np.int32)
    rec, fl = O.primary(scene, cam, pix, mode=0)
    clean = fl == 0
    assert clean.mean() > 0.97
    ok = radiance_close(rgb[clean], rec[clean, 4:7])
    assert ok.all(), np.flatnonzero(~ok)[:10]
    # the image is the R column of the primary record
    np.testing.assert_array_equal(rgb, aux[:, 4:7])
    # misses are exactly zero
    miss = rec[:, 11] <= 0
    assert (rgb[miss & clean] == 0).all()


def test_radiance_empty_scene_is_black(api):
    import torch
    sc = S.SurfelScene(*[np.zeros((0,) + s, np.float32) for s in [(3,), (4,), (2,), (), (3,), (3,), ()]])
    cam = S.horizontal_camera(9, 7)
    ds = api.DeviceScene.from_host(sc)
    bvh = api.BVH(ds)
    out = api.radiance(ds, bvh, cam)
    api.sync_status()
    assert torch.count_nonzero(out["rgb"]).item() == 0
    g = api.radiance_backward(ds, bvh, cam, torch.ones((7, 9, 3), device="cuda"))
    assert all(v.numel() == 0 for v in g.values())


def _compare_grad(api, scene, cam, pixels, wseed, tol=1e-3):
    import torch
    rng = np.random.default_rng(wseed)
    npix = cam.width * cam.height
    w = np.zeros((npix, 3))
    w[pixels] = rng.uniform(-1, 1, (len(pixels), 3))
    _, fl = O.primary(scene, cam, np.asarray(pixels, np.int32), mode=0)
    decision = np.uint32(~O.FLAGS["cond"] & 0xFFFFFFFF)
    bad = (fl & decision) != 0
    w[np.asarray(pixels)[bad]] = 0.0
    ds = api.DeviceScene.from_host(scene)
    bvh = api.BVH(ds)
    dL = torch.from_numpy(w.reshape(cam.height, cam.width, 3).astype(np.float32)).cuda()
    g = api.radiance_backward(ds, bvh, cam, dL)
    api.sync_status()
    ref, _, ref_dev = oracle_grad_with_conditioning(O.radiance_grad, scene, cam, np.asarray(pixels, np.int32),
                                                    w[pixels])
    errs, worst, ill = {}, {}, {}
    for k, (a, b) in GROUPS.items():
        gg = g[k].cpu().numpy().astype(np.float64).reshape(scene.n, -1)
        rr = ref[:, a:b]
        errs[k], ok, worst[k], ill[k] = grad_errors(gg, rr, tol, ref_dev[:, a:b])
        assert ok.all(), (k, "entries over the per-entry bound:", int((~ok).sum()), "worst ratio", worst[k],
                          np.argwhere(~ok)[:5])
    print("relative gradient error per group:", errs, "worst entry / its bound:", worst,
          "ill-conditioned entries:", ill, "pixels zeroed:", int(bad.sum()))
    for k, e in errs.items():
        assert e <= tol, (k, errs)
    # the 0-bounce image does not depend on the albedo
    assert float(g["albedo"].abs().max()) == 0.0
    assert np.abs(ref[:, 10:13]).max() == 0.0


def test_radiance_gradients_small_scene(api):
    sc = S.random_small_scene(8, 31, spread=0.25, emit_frac=0.25)
    cam = S.look_at_camera(12, 10, 50.0, (0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0, 0, 1))
    _compare_grad(api, sc, cam, np.arange(120), 5)


def test_radiance_gradients_tiny_room(api):
    wl = S.workload("tiny")
    cam = wl.camera
    _compare_grad(api, wl.scene_fn(), cam, np.arange(cam.width * cam.height), 7)


def test_radiance_autograd_function(api):
    import torch
    sc = S.tiny_room(4096)
    cam = S.horizontal_camera(24, 16)
    t = {k: torch.from_numpy(getattr(sc, k)).cuda().requires_grad_(k != "emissive") for k in api.FIELDS}
    img = api.render_radiance(t, cam)
    w = torch.rand_like(img)
    (img * w).sum().backward()
    ds = api.DeviceScene({k: v.detach() for k, v in t.items()})
    bvh = api.BVH(ds)
    g = api.radiance_backward(ds, bvh, cam, w)
    for k in api.GRAD_FIELDS:
        a, b = t[k].grad, g[k]
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-6 * float(b.abs().max()) + 1e-12), k
