"""Pins of the oracle's level-of-detail merge and render (CPU only).

The merge is a definition (moment matching of a group's Gaussians); these
tests check it against what geometry fixes without re-typing it: a group of
one surfel must come back unchanged, two surfels whose union has a known
second moment must give that moment, and the merged footprint, weight and
weighted albedo must be conserved.  Group keys are checked against hand-worked
cells.  The render is pinned by a furnace pair (a full box and a merged box
with other radiance and albedo) whose radiance is a known two-part geometric
series, so the bounce index at which the merged surfels take over is fixed.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import lod as L
from paper_2601_23065_gb300 import scenes as S

f32 = lambda a: np.ascontiguousarray(a, np.float32)


def scene_of(pos, quat, scale, sigma, rho=None, r=None, e=None):
    m = len(pos)
    rho = np.full((m, 3), 0.5) if rho is None else rho
    r = np.zeros((m, 3)) if r is None else r
    e = np.zeros(m) if e is None else e
    return S.SurfelScene(f32(pos), f32(quat), f32(scale), f32(sigma), f32(rho), f32(r), f32(e))


def qz(theta):
    """rotation by theta about z: t_u = (cos, sin, 0), t_v = (-sin, cos, 0), n = +z"""
    return [math.cos(theta / 2), 0.0, 0.0, math.sin(theta / 2)]


def cov_of(quat, scale):
    tu, tv, _ = L.frames(np.asarray(quat, np.float64).reshape(-1, 4))
    s = np.asarray(scale, np.float64).reshape(-1, 2)
    return (s[:, 0, None, None] ** 2 * tu[:, :, None] * tu[:, None, :]
            + s[:, 1, None, None] ** 2 * tv[:, :, None] * tv[:, None, :])


# ------------------------------------------------------------- frames ----

def test_frames_textbook_rotations():
    """Columns of textbook rotations: about z by theta, about x by 90 deg."""
    th = 0.7
    tu, tv, n = L.frames(np.array([qz(th)]))
    np.testing.assert_allclose(tu[0], [math.cos(th), math.sin(th), 0], atol=1e-15)
    np.testing.assert_allclose(tv[0], [-math.sin(th), math.cos(th), 0], atol=1e-15)
    np.testing.assert_allclose(n[0], [0, 0, 1], atol=1e-15)
    c = math.cos(math.pi / 4)
    tu, tv, n = L.frames(np.array([[c, c, 0.0, 0.0]]) * 3.0)  # not unit on purpose
    np.testing.assert_allclose(tu[0], [1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(tv[0], [0, 0, 1], atol=1e-15)
    np.testing.assert_allclose(n[0], [0, -1, 0], atol=1e-15)


def test_frames_and_quaternion_round_trip_against_scipy():
    """frames() equals scipy's rotation matrix (scalar-last convention), and
    quat_from_frame() inverts it up to the quaternion's sign."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(5)
    q = rng.normal(size=(64, 4))
    tu, tv, n = L.frames(q)
    M = Rot.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()
    np.testing.assert_allclose(tu, M[:, :, 0], atol=1e-13)
    np.testing.assert_allclose(tv, M[:, :, 1], atol=1e-13)
    np.testing.assert_allclose(n, M[:, :, 2], atol=1e-13)
    for i in range(64):
        qb = L.quat_from_frame(tu[i], tv[i], n[i])
        qa = q[i] / np.linalg.norm(q[i])
        assert min(np.abs(qb - qa).max(), np.abs(qb + qa).max()) < 1e-13


# --------------------------------------------------------------- keys ----

def test_group_keys_hand_worked_cells():
    """Cells, axis and emitter bit of surfels placed by hand (every value
    exact in FP32)."""
    c = math.cos(math.pi / 4)
    quats = [qz(0.3),                    # n = +z -> axis 2
             [c, c, 0.0, 0.0],           # n = -y -> axis 1
             [c, 0.0, c, 0.0],           # n = +x -> axis 0
             [0.5, -0.5, 0.5, 0.0],      # n' = (0.5, 0.5, -0.25): tie -> axis 0
             qz(0.0), qz(0.0)]
    pos = [[0.1, 0.6, 1.3], [0.0, 0.25, 0.49], [0.74, 0.76, 0.0], [0.3, 0.3, 0.3],
           [-5.0, 0.1, 0.1], [1e9, 0.1, 0.1]]
    e = [1.0, 0.0, 0.05, 0.2, 0.0, 0.0]
    keys, axis = L.group_keys(f32(pos), f32(quats), f32(e), (0.0, 0.0, 0.0), 0.25, tau_E=0.1)
    want = [(0, 2, 5, 2, 1), (0, 1, 1, 1, 0), (2, 3, 0, 0, 0), (1, 1, 1, 0, 1),
            (0, 0, 0, 2, 0), (L.CELL_MAX, 0, 0, 2, 0)]
    for k, (cx, cy, cz, ax, em) in zip(keys, want):
        assert int(k) == (cx << 43) | (cy << 23) | (cz << 3) | (ax << 1) | em
    assert list(axis) == [w[3] for w in want]


def test_group_keys_agree_with_fp64_away_from_boundaries():
    """On the tiny room the FP32 cell and axis decisions equal the FP64 ones
    for every surfel not within 1e-5 of a cell boundary or an axis tie."""
    sc = S.tiny_room(4096)
    o, h = (-0.6, -0.6, -0.6), 0.05
    keys, axis = L.group_keys(sc.pos, sc.quat, sc.emissive, o, h)
    x = (sc.pos.astype(np.float64) - np.array(o)) / h
    far = (np.abs(x - np.round(x)) > 1e-5).all(1)
    cell64 = np.floor(x).astype(np.int64)
    cells = np.stack([(keys.astype(np.int64) >> s) & L.CELL_MAX for s in (43, 23, 3)], 1)
    assert far.mean() > 0.99
    assert (cells[far] == cell64[far]).all()
    _, _, n = L.frames(sc.quat)
    a = np.sort(np.abs(n), 1)
    clear = a[:, 2] - a[:, 1] > 1e-5
    assert (axis[clear] == np.argmax(np.abs(n), 1)[clear]).all()


# -------------------------------------------------------------- merge ----

def test_single_surfel_groups_reproduce_their_surfel():
    """With cells far smaller than the surfel spacing every group holds one
    surfel, and the merge returns it: the same centre, Gaussian (covariance
    s_u^2 t_u t_u^T + s_v^2 t_v t_v^T), normal up to sign, opacity, albedo,
    radiance and emissive term."""
    sc = S.tiny_room(4096)
    m = L.merge(sc, (-0.6, -0.6, -0.6), 1e-5)
    assert len(m["keys"]) == sc.n and all(len(g) == 1 for g in m["members"])
    src = np.array([g[0] for g in m["members"]])
    assert sorted(src) == list(range(sc.n))
    np.testing.assert_allclose(m["pos"], sc.pos[src].astype(np.float64), rtol=0, atol=1e-15)
    cin = cov_of(sc.quat[src], sc.scale[src])
    cout = cov_of(m["quat"], m["scale"])
    s2 = (sc.scale[src].astype(np.float64) ** 2).max(1)
    assert (np.abs(cout - cin).max((1, 2)) <= 1e-12 * s2).all()
    np.testing.assert_allclose(m["cov"], cout, rtol=0, atol=1e-14)
    _, _, n = L.frames(sc.quat[src])
    np.testing.assert_allclose(np.abs((m["normal"] * n).sum(1)), 1.0, atol=1e-12)
    np.testing.assert_allclose(m["opacity"], sc.opacity[src], rtol=1e-12)
    np.testing.assert_allclose(m["albedo"], sc.albedo[src], rtol=1e-15)
    np.testing.assert_allclose(m["radiance"], sc.radiance[src], rtol=1e-15)
    np.testing.assert_allclose(m["emissive"], sc.emissive[src], rtol=1e-15)


@pytest.mark.parametrize("sig", [(1.0, 1.0), (0.9, 0.3)])
def test_two_coplanar_isotropic_surfels(sig):
    """Two isotropic surfels (scale s) at (+-a, 0, 0) in the plane z = 0:
    with weights w_k = sigma_k s^2 the union's second moment along x is
    s^2 + w1 w2 (2a)^2 / W^2 and along y s^2."""
    a, s = 0.01, 0.004
    sc = scene_of([[-a, 0, 0], [a, 0, 0]], [qz(0.2), qz(1.1)], [[s, s], [s, s]], list(sig),
                  rho=[[0.2, 0.4, 0.6], [0.8, 0.6, 0.4]])
    m = L.merge(sc, (-1.5, -1.5, -1.5), 1.0)
    assert len(m["keys"]) == 1
    x = sc.pos[:, 0].astype(np.float64)
    ss = float(np.float32(s)) ** 2
    w = np.array(sig, np.float32).astype(np.float64) * ss
    W = w.sum()
    su2 = ss + w[0] * w[1] * (x[1] - x[0]) ** 2 / W ** 2
    np.testing.assert_allclose(m["pos"][0], [(w @ x) / W, 0, 0], atol=1e-17)
    np.testing.assert_allclose(m["cov"][0], np.diag([su2, ss, 0.0]), atol=1e-18)
    np.testing.assert_allclose(m["scale"][0], [math.sqrt(su2), math.sqrt(ss)], rtol=1e-12)
    np.testing.assert_allclose(np.abs(m["normal"][0]), [0, 0, 1], atol=1e-15)
    np.testing.assert_allclose(m["opacity"][0], W / math.sqrt(su2 * ss), rtol=1e-12)
    np.testing.assert_allclose(m["albedo"][0], (w[:, None] * sc.albedo.astype(np.float64)).sum(0) / W,
                               rtol=1e-12)


def test_crossed_anisotropic_surfels_merge_isotropic():
    """Two surfels at one centre with scales (s1, s2), rotated 0 and 90 deg
    in-plane: the union's covariance is (s1^2 + s2^2)/2 I in the plane."""
    s1, s2 = 0.02, 0.005
    sc = scene_of([[0.3, 0.3, 0.3]] * 2, [qz(0.0), qz(math.pi / 2)], [[s1, s2]] * 2, [0.8, 0.8])
    m = L.merge(sc, (0, 0, 0), 1.0)
    a, b = (float(np.float32(v)) for v in (s1, s2))
    v = (a * a + b * b) / 2
    np.testing.assert_allclose(m["cov"][0], np.diag([v, v, 0.0]), atol=1e-15 * v)
    np.testing.assert_allclose(m["opacity"][0], 2 * float(np.float32(0.8)) * a * b / v, rtol=1e-7)


def test_layers_offset_along_the_normal_and_flipped_normals():
    """Two parallel layers 2 mm apart along the normal, one of them facing
    the other way: the offset lies along the merged normal and is projected
    out (scale unchanged), the flipped normal is aligned before averaging,
    and the footprint doubles into the opacity."""
    s = 0.01
    c = math.cos(math.pi / 2)
    flipped = [c, 1.0, 0.0, 0.0]  # 180 deg about x: n = -z
    sc = scene_of([[0.5, 0.5, 0.5], [0.5, 0.5, 0.502]], [qz(0.4), flipped], [[s, s]] * 2, [1.0, 1.0])
    m = L.merge(sc, (0, 0, 0), 1.0)
    assert len(m["keys"]) == 1
    np.testing.assert_allclose(m["normal"][0], [0, 0, 1], atol=1e-15)
    ss = float(np.float32(s)) ** 2
    np.testing.assert_allclose(m["cov"][0], np.diag([ss, ss, 0.0]), atol=1e-16)
    np.testing.assert_allclose(m["opacity"][0], 2.0, rtol=1e-12)


def test_groups_partition_and_conserve_weight_footprint_albedo():
    """Medium cells on the tiny room: members partition the surfels and share
    their group's key, keys ascend, and the total weight, footprint
    sum sigma s_u s_v and weighted albedo are conserved."""
    sc = S.tiny_room(4096)
    o, h = (-0.6, -0.6, -0.6), 0.05
    m = L.merge(sc, o, h)
    keys, _ = L.group_keys(sc.pos, sc.quat, sc.emissive, o, h)
    allm = np.concatenate(m["members"])
    assert sorted(allm) == list(range(sc.n))
    for k, g in zip(m["keys"], m["members"]):
        assert (keys[g] == k).all() and (np.diff(g) > 0).all()
    assert (np.diff(m["keys"].astype(np.float64)) > 0).all()
    assert len(m["keys"]) < 0.9 * sc.n
    w = sc.opacity.astype(np.float64) * sc.scale[:, 0].astype(np.float64) * sc.scale[:, 1]
    np.testing.assert_allclose(m["weight"].sum(), w.sum(), rtol=1e-12)
    np.testing.assert_allclose((m["opacity"] * m["scale"][:, 0] * m["scale"][:, 1]).sum(), w.sum(), rtol=1e-12)
    np.testing.assert_allclose((m["weight"][:, None] * m["albedo"]).sum(0),
                               (w[:, None] * sc.albedo.astype(np.float64)).sum(0), rtol=1e-12)
    # emitters never share a group with non-emitters
    assert set(np.unique(m["emissive"])) <= {0.0, 1.0}


def test_zero_weight_group():
    """A group whose opacities are all 0 takes unit weights and opacity 0."""
    sc = scene_of([[0.1, 0.1, 0.1], [0.2, 0.1, 0.1]], [qz(0.0)] * 2, [[0.01, 0.01]] * 2, [0.0, 0.0])
    m = L.merge(sc, (0, 0, 0), 1.0)
    np.testing.assert_allclose(m["pos"][0], [0.15, 0.1, 0.1], rtol=1e-7)
    assert m["opacity"][0] == 0.0


# ------------------------------------------------------------- render ----

A2 = 1.0 - 1e-4  # coverage of a two-layer opaque wall


@pytest.mark.parametrize("lod_from", [1, 2, 3])
def test_furnace_pair_switches_at_lod_from(lod_from):
    """Furnace box (every face emissive L_e, albedo rho, emitters reflecting)
    for the segments before lod_from and a second furnace box (radiance r',
    albedo rho') for the segments from lod_from on: every sample is
    sum_{k<m} (rho A)^k A L_e + sum_{k=m..B} (rho A)^m (rho' A)^(k-m) A r'."""
    full = S.giant_box(rho=0.3, r=1.7, gap=1e-6)
    coarse = S.giant_box(rho=0.6, r=2.9, gap=1e-6)
    Le, rho = float(full.radiance[0, 0]), float(full.albedo[0, 0])
    r2, rho2 = float(coarse.radiance[0, 0]), float(coarse.albedo[0, 0])
    cam = S.horizontal_camera(10, 10, hfov=120.0)
    pix = np.arange(100, dtype=np.int32)
    prm = O.Params(emitters_reflect=True)
    for B in [0, 1, 2, 4]:
        out = O.render_lod(full, coarse, lod_from, cam, pix, 2, max_bounces=B, rr_start=1000, params=prm,
                           want_samples=True)
        m = min(lod_from, B + 1)
        exp = sum((rho * A2) ** k * A2 * Le for k in range(m))
        exp += sum((rho * A2) ** m * (rho2 * A2) ** (k - m) * A2 * r2 for k in range(m, B + 1))
        np.testing.assert_allclose(out["samples"], exp, rtol=1e-11)


def test_lod_render_reduces_to_the_plain_render():
    """A level of detail that is the scene itself, or that starts after the
    last bounce, gives the plain render bit for bit (samples, flags,
    segments)."""
    sc = S.tiny_room(4096)
    cam = S.horizontal_camera(24, 24, hfov=90.0)
    pix = np.arange(0, 576, 7, dtype=np.int32)
    prm = O.Params()
    ref = O.render(sc, cam, pix, "pt", 2, max_bounces=3, rr_start=2, seed=5, params=prm, want_samples=True)
    coarse = L.to_scene(L.merge(sc, (-0.6, -0.6, -0.6), 0.05), S.SurfelScene)
    for lsc, lf in [(sc, 1), (coarse, 4)]:
        out = O.render_lod(sc, lsc, lf, cam, pix, 2, max_bounces=3, rr_start=2, seed=5, params=prm,
                           want_samples=True)
        for k in ("samples", "sample_flags", "segments"):
            assert np.array_equal(out[k], ref[k]), k
    out = O.render_lod(sc, coarse, 2, cam, pix, 2, max_bounces=3, rr_start=2, seed=5, params=prm,
                       want_samples=True)
    assert not np.array_equal(out["samples"], ref["samples"])


def test_lod_render_rejects_emitter_sampling():
    sc = S.tiny_room(4096)
    cam = S.horizontal_camera(4, 4)
    with pytest.raises(RuntimeError):
        O.render_lod(sc, sc, 1, cam, np.arange(4, dtype=np.int32), 1, max_bounces=2, params=O.Params(mis=True))


def test_vectorised_merge_equals_group_by_group():
    """merge() (all groups at once) equals merge_by_group() (merge_group one
    group at a time) on the tiny room: keys, members and every merged value,
    the Gaussian through its covariance (also as rebuilt from the merged
    quaternion and scales; the in-plane axis of a round group is arbitrary)."""
    sc = S.tiny_room(4096)
    for h in (0.05, 0.2):
        a = L.merge(sc, (-0.6125,) * 3, h)
        b = L.merge_by_group(sc, (-0.6125,) * 3, h)
        assert np.array_equal(a["keys"], b["keys"])
        assert all(np.array_equal(x, y) for x, y in zip(a["members"], b["members"]))
        for k in ("pos", "scale", "opacity", "albedo", "radiance", "emissive", "normal", "weight"):
            np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-15, err_msg=k)
        big = np.abs(b["cov"]).max((1, 2), keepdims=True)
        assert (np.abs(a["cov"] - b["cov"]) <= 1e-12 * big).all()
        assert (np.abs(cov_of(a["quat"], a["scale"]) - b["cov"]) <= 1e-12 * big).all()


def test_quaternions_of_many_frames_row_by_row():
    """quat_from_frames() equals quat_from_frame() row by row, on random
    frames that take every one of its four branches."""
    rng = np.random.default_rng(8)
    q = rng.normal(size=(400, 4))
    q[:100, 0] *= 20
    q[100:200, 1] *= 20
    q[200:300, 2] *= 20
    q[300:, 3] *= 20
    tu, tv, n = L.frames(q)
    many = L.quat_from_frames(tu, tv, n)
    one = np.array([L.quat_from_frame(a, b, c) for a, b, c in zip(tu, tv, n)])
    assert np.array_equal(many, one)


def test_merged_gaussian_matches_sampled_union():
    """Moment matching checked by sampling: points drawn from every member's
    Gaussian (in its own plane, N(0, s_u^2) along t_u and N(0, s_v^2) along
    t_v about p), the member chosen with probability w_i / W, have a mean and
    an in-plane second moment that the merged surfel's centre and covariance
    must match within the sampling error (5 coplanar surfels of random
    rotation, scale and opacity, 2e6 points)."""
    rng = np.random.default_rng(21)
    m = 5
    th = rng.uniform(0, math.pi, m)
    pos = np.column_stack([rng.uniform(0.40, 0.46, m), rng.uniform(0.40, 0.46, m), np.full(m, 0.45)])
    scale = np.exp(rng.uniform(math.log(0.003), math.log(0.02), (m, 2)))
    sigma = rng.uniform(0.5, 1.0, m)
    sc = scene_of(pos, [qz(t) for t in th], scale, sigma)
    g = L.merge(sc, (0, 0, 0), 0.5)
    assert len(g["keys"]) == 1
    p = sc.pos.astype(np.float64)
    s = sc.scale.astype(np.float64)
    w = sc.opacity.astype(np.float64) * s[:, 0] * s[:, 1]
    tu, tv, _ = L.frames(sc.quat)
    N = 2_000_000
    who = rng.choice(m, N, p=w / w.sum())
    a = rng.standard_normal(N) * s[who, 0]
    b = rng.standard_normal(N) * s[who, 1]
    x = p[who] + a[:, None] * tu[who] + b[:, None] * tv[who]
    mean = x.mean(0)
    d = x - mean
    C = d.T @ d / N
    spread = math.sqrt(np.trace(C))
    assert np.abs(g["pos"][0] - mean).max() < 5 * spread / math.sqrt(N)
    np.testing.assert_allclose(g["cov"][0][:2, :2], C[:2, :2], atol=6 * np.abs(C).max() * math.sqrt(2 / N))
    assert np.abs(g["cov"][0][2]).max() < 1e-15 and np.abs(C[2]).max() < 1e-15
