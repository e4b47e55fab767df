"""The continuous-batching serving loop: every request's image equals the
plain single-request render bit for bit, whatever else is in the mix; edits
apply in submission order (earlier renders see the old scene, later ones the
new); timeouts and cancellation end requests without touching the GPU."""
import numpy as np
import pytest

from paper_2601_23065_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    from paper_2601_23065_gb300 import api, build
    build.build()
    torch.cuda.init()
    return api


REQS = [  # (width, height, spp, bounces, seed, camera centre, forward)
    (64, 48, 8, 3, 1, (0.0, 0.0, 0.0), (1, 0, 0)),
    (32, 32, 16, 1, 2, (0.1, 0.1, 0.0), (0, 1, 0)),
    (96, 64, 4, 5, 3, (-0.2, 0.0, 0.1), (1, 1, 0)),
    (17, 13, 32, 2, 4, (0.0, -0.2, -0.1), (-1, 0, 0)),
    (128, 72, 2, 4, 5, (0.2, 0.2, 0.2), (0, -1, 0)),
    (48, 48, 12, 3, 6, (0.0, 0.0, 0.2), (1, -1, 0)),
]


def _plain(api, ds, bvh, w, h, spp, B, seed, c, f):
    cam = S.look_at_camera(w, h, 90.0, c, f, (0, 0, 1))
    return api.Renderer().path_traced(ds, bvh, cam, spp, B, rr_start=2, seed=seed)["rgb"].clone()


def test_results_equal_alone_and_in_mix(api):
    import torch
    sc = S.tiny_room(4096)
    ds = api.DeviceScene.from_host(sc)
    bvh = api.BVH(ds)
    alone = [_plain(api, ds, bvh, *r) for r in REQS]
    torch.cuda.synchronize()
    # small queue and few slots: requests wait, join mid-stream and share waves
    srv = api.Server(ds, bvh, queue_paths=40000, max_active=3)
    ids = []
    for (w, h, spp, B, seed, c, f) in REQS:
        cam = S.look_at_camera(w, h, 90.0, c, f, (0, 0, 1))
        ids.append(srv.submit_render(cam, spp, B, rr_start=2, seed=seed))
    for (rid, out), ref in zip(ids, alone):
        info = srv.wait(rid, timeout_s=120.0)
        assert info["state"] == "done", info
        assert info["t_submit"] <= info["t_admit"] <= info["t_done"]
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    st = srv.stats()
    assert st["completed"] == len(REQS) and st["waves"] >= 2 and st["segments"] > 0
    srv.close()
    api.sync_status()


def test_edits_apply_in_submission_order(api):
    import torch
    sc = S.tiny_room(4096)
    # reference renders: original scene, and the scene after the same edit
    ds_ref = api.DeviceScene.from_host(sc)
    bvh_ref = api.BVH(ds_ref)
    r0 = REQS[0]
    before = _plain(api, ds_ref, bvh_ref, *r0)
    sel = api.select(ds_ref, "sphere", [0.3, 0.0, 0.0, 0.3])
    api.apply_edit(ds_ref, bvh_ref, "toggle_emission", sel)
    after = _plain(api, ds_ref, bvh_ref, *r0)
    assert not torch.equal(before, after)
    # the same through the server: render, edit, render
    ds = api.DeviceScene.from_host(sc)
    bvh = api.BVH(ds)
    srv = api.Server(ds, bvh, queue_paths=1 << 16, max_active=4)
    w, h, spp, B, seed, c, f = r0
    cam = S.look_at_camera(w, h, 90.0, c, f, (0, 0, 1))
    a, out_a = srv.submit_render(cam, spp, B, rr_start=2, seed=seed)
    e = srv.submit_edit("toggle_emission", sel)
    b, out_b = srv.submit_render(cam, spp, B, rr_start=2, seed=seed)
    ia, ie, ib = srv.wait(a, 120.0), srv.wait(e, 120.0), srv.wait(b, 120.0)
    assert ia["state"] == ie["state"] == ib["state"] == "done"
    assert ib["scene_version"] == ia["scene_version"] + 1
    torch.cuda.synchronize()
    assert torch.equal(out_a, before) and torch.equal(out_b, after)
    srv.close()


def test_timeout_and_cancel(api):
    from paper_2601_23065_gb300 import capi
    sc = S.tiny_room(4096)
    ds = api.DeviceScene.from_host(sc)
    bvh = api.BVH(ds)
    srv = api.Server(ds, bvh, queue_paths=1 << 14, max_active=1)
    big = S.horizontal_camera(128, 128)
    first, _ = srv.submit_render(big, 256, 5, seed=1)       # occupies the only slot for a while
    doomed, _ = srv.submit_render(big, 4, 1, seed=2, timeout_s=1e-3)
    queued, _ = srv.submit_render(big, 4, 1, seed=3)
    srv.cancel(queued)
    with pytest.raises(capi.EagptError) as ei:
        srv.wait(first, timeout_s=1e-3)
    assert ei.value.status == 5
    assert srv.wait(doomed, 120.0)["state"] == "timed_out"
    assert srv.wait(queued, 120.0)["state"] == "cancelled"
    assert srv.wait(first, 300.0)["state"] == "done"
    srv.close()
    api.sync_status()


def test_small_requests_do_not_wait_on_a_large_one(api):
    """Each wave's queue is filled shortest remaining work first, with one
    sample per request first: renders submitted just after a large one finish
    long before it, and the large one still progresses every wave and ends."""
    import torch
    sc = S.tiny_room(4096)
    ds = api.DeviceScene.from_host(sc)
    bvh = api.BVH(ds)
    srv = api.Server(ds, bvh, queue_paths=200_000, max_active=8)
    big_cam = S.look_at_camera(256, 256, 90.0, (0.0, 0.0, 0.0), (1, 0, 0), (0, 0, 1))
    big = srv.submit_render(big_cam, 64, 5, rr_start=2, seed=9)  # 4.2 M paths: 21 full waves at least
    small = []
    for k in range(4):
        cam = S.look_at_camera(32, 32, 90.0, (0.05 * k, 0.0, 0.0), (0, 1, 0), (0, 0, 1))
        small.append((srv.submit_render(cam, 8, 2, rr_start=2, seed=20 + k), cam, 20 + k))
    done_small = []
    for (rid, out), cam, seed in small:
        info = srv.wait(rid, timeout_s=120.0)
        assert info["state"] == "done", info
        done_small.append(info["t_done"])
        torch.cuda.synchronize()
        ref = api.Renderer().path_traced(ds, bvh, cam, 8, 2, rr_start=2, seed=seed)["rgb"]
        assert torch.equal(out, ref)
    info = srv.wait(big[0], timeout_s=300.0)
    assert info["state"] == "done", info
    assert max(done_small) < info["t_done"]
    assert srv.stats()["waves"] >= 21
    srv.close()
    api.sync_status()


def test_cancel_a_running_request(api):
    """A render cancelled while its waves are in flight ends as cancelled; its
    memory is released only after those waves, so renders admitted after it
    (which may reuse that memory on the other wave stream) stay exact."""
    import time

    import torch
    sc = S.tiny_room(4096)
    ds = api.DeviceScene.from_host(sc)
    bvh = api.BVH(ds)
    srv = api.Server(ds, bvh, queue_paths=100_000, max_active=2)
    big_cam = S.look_at_camera(256, 256, 90.0, (0.0, 0.0, 0.0), (1, 0, 0), (0, 0, 1))
    big, _ = srv.submit_render(big_cam, 128, 5, rr_start=2, seed=5)
    t0 = time.time()
    while srv.poll(big)["state"] != "running" and time.time() - t0 < 60:
        time.sleep(1e-3)
    srv.cancel(big)
    after = []
    for k in range(3):
        cam = S.look_at_camera(48, 40, 90.0, (0.0, 0.05 * k, 0.0), (0, 1, 0), (0, 0, 1))
        after.append((srv.submit_render(cam, 6, 3, rr_start=2, seed=30 + k), cam, 30 + k))
    assert srv.wait(big, 120.0)["state"] == "cancelled"
    for (rid, out), cam, seed in after:
        assert srv.wait(rid, 120.0)["state"] == "done"
        torch.cuda.synchronize()
        ref = api.Renderer().path_traced(ds, bvh, cam, 6, 3, rr_start=2, seed=seed)["rgb"]
        assert torch.equal(out, ref)
    st = srv.stats()
    assert st["completed"] == 3 and st["failed"] >= 1
    srv.close()
    api.sync_status()
