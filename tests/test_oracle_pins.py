"""Pins of the FP64 oracle against closed forms, invariants and brute force.

None of these tests re-types the oracle's formulas: each expected value comes
from geometry set up so the answer is known (an axis-aligned surfel hit at a
chosen local coordinate, a furnace box whose radiance is a geometric series,
a room whose light paths are forced), from a statistical property of the
sampler, or from an independent finite difference.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2601_23065_gb300 import scenes as S

HERE = os.path.dirname(os.path.abspath(__file__))
A2 = 1.0 - 1e-4  # coverage of a two-layer opaque wall: T = 0.01 * 0.01


def one_surfel(p, theta, su, sv, sigma, rho=(0.2, 0.4, 0.6), r=(1.0, 2.0, 3.0), e=0.0, qscale=1.0):
    """A single surfel in the plane z = p_z, rotated by theta about z."""
    q = np.array([[math.cos(theta / 2), 0.0, 0.0, math.sin(theta / 2)]]) * qscale
    f = lambda a: np.ascontiguousarray(a, np.float32)
    return S.SurfelScene(f([p]), f(q), f([[su, sv]]), f([sigma]), f([rho]), f([r]), f([e]))


def stack(scenes):
    return S.SurfelScene(*[np.ascontiguousarray(np.concatenate([getattr(s, k) for s in scenes]))
                           for k in ("pos", "quat", "scale", "opacity", "albedo", "radiance", "emissive")])


# ---------------------------------------------------------------- Eq. 1 ----

@pytest.mark.parametrize("theta", [0.0, 0.7, 2.5])
@pytest.mark.parametrize("uv", [(0.0, 0.0), (0.5, -0.3), (1.7, 2.0), (-2.0, 0.4)])
@pytest.mark.parametrize("qscale", [1.0, 2.5])
def test_single_surfel_analytic_hit(theta, uv, qscale):
    """Ray straight down onto a surfel rotated by theta about z: the hit sits
    at local (u, v) by construction, so alpha = sigma exp(-(u^2+v^2)/2)."""
    su, sv, sigma = 0.05, 0.02, 0.8
    p = np.array([0.25, -0.5, 0.125])
    sc = one_surfel(p.astype(np.float32), theta, su, sv, sigma, qscale=qscale)
    # the stored FP32 values, widened: a quaternion (c, 0, 0, s) is a rotation
    # by 2 atan2(s, c) about z
    p = sc.pos[0].astype(np.float64)
    su, sv = map(float, sc.scale[0])
    sigma = float(sc.opacity[0])
    theta = 2.0 * math.atan2(float(sc.quat[0, 3]), float(sc.quat[0, 0]))
    tu = np.array([math.cos(theta), math.sin(theta), 0.0])
    tv = np.array([-math.sin(theta), math.cos(theta), 0.0])
    u, v = uv
    x = p + u * su * tu + v * sv * tv
    O_ = x + np.array([0.0, 0.0, 1.5])
    seg, hits = O.trace_segment(sc, O_, [0.0, 0.0, -1.0])
    alpha = sigma * math.exp(-0.5 * (u * u + v * v))
    if alpha < 1 / 255:
        assert seg["n_hits"] == 0 and seg["A"] == 0.0
        return
    assert list(hits) == [0]
    assert seg["A"] == pytest.approx(alpha, rel=1e-12)
    np.testing.assert_allclose(seg["R"], alpha * sc.radiance[0].astype(np.float64), rtol=1e-12)
    np.testing.assert_allclose(seg["P"], alpha * sc.albedo[0].astype(np.float64), rtol=1e-12)
    assert seg["Dn"] == pytest.approx(1.5, rel=1e-12)
    np.testing.assert_allclose(seg["Nn"], [0, 0, 1], atol=1e-12)  # faces the origin above
    # from below the facing normal flips
    seg2, _ = O.trace_segment(sc, x - np.array([0.0, 0.0, 0.75]), [0.0, 0.0, 1.0])
    np.testing.assert_allclose(seg2["Nn"], [0, 0, -1], atol=1e-12)
    assert seg2["Dn"] == pytest.approx(0.75, rel=1e-12)


def test_support_alpha_limits():
    """Outside 3 sigma there is no hit even when alpha would exceed alpha_min
    (sigma = 1: alpha(3 sigma) = exp(-4.5) = 0.011 > 1/255); the clamp caps
    alpha at 0.99 at the centre of an opaque surfel."""
    sc = one_surfel(np.zeros(3, np.float32), 0.0, 0.1, 0.1, 1.0)
    for u, hit in [(2.99, True), (3.01, False)]:
        seg, _ = O.trace_segment(sc, [u * 0.1, 0.0, 1.0], [0.0, 0.0, -1.0])
        assert (seg["n_hits"] == 1) == hit
    seg, _ = O.trace_segment(sc, [0.0, 0.0, 1.0], [0.0, 0.0, -1.0])
    assert seg["A"] == 0.99
    # below alpha_min: sigma 0.5 at u = 2.5: 0.5 e^-3.125 = 0.022 (hit), at u = 2.9: 0.0149 (hit),
    # sigma = 0.01 at the centre: 0.01 > 1/255 (hit), sigma = 0.003 < 1/255 (miss)
    for sig, hit in [(0.01, True), (0.003, False)]:
        s2 = one_surfel(np.zeros(3, np.float32), 0.0, 0.1, 0.1, sig)
        seg, _ = O.trace_segment(s2, [0.0, 0.0, 1.0], [0.0, 0.0, -1.0])
        assert (seg["n_hits"] == 1) == hit


# ---------------------------------------------------------------- Eq. 2 ----

def test_two_parallel_surfels_compositing():
    """V = alpha1 v1 + (1 - alpha1) alpha2 v2, nearer surfel first, in both
    directions (the order reverses with the ray)."""
    a = one_surfel(np.array([0, 0, 0.0], np.float32), 0.3, 0.2, 0.2, 0.6, rho=(0.1, 0.2, 0.3), r=(1, 0, 0))
    b = one_surfel(np.array([0, 0, -0.5], np.float32), 1.1, 0.2, 0.2, 0.7, rho=(0.5, 0.5, 0.5), r=(0, 1, 0))
    sc = stack([a, b])
    for origin, direction, first, t1, t2 in [([0, 0, 1.0], [0, 0, -1.0], 0, 1.0, 1.5),
                                             ([0, 0, -2.0], [0, 0, 1.0], 1, 1.5, 2.0)]:
        seg, hits = O.trace_segment(sc, origin, direction)
        assert list(hits) == [first, 1 - first]
        a1 = float(sc.opacity[first])
        a2 = float(sc.opacity[1 - first])
        v = lambda arr: arr.astype(np.float64)
        for key, arr in (("P", sc.albedo), ("R", sc.radiance)):
            exp = a1 * v(arr[first]) + (1 - a1) * a2 * v(arr[1 - first])
            np.testing.assert_allclose(seg[key], exp, rtol=1e-12)
        A = 1 - (1 - a1) * (1 - a2)
        assert seg["A"] == pytest.approx(A, rel=1e-12)
        assert seg["Dn"] == pytest.approx((a1 * t1 + (1 - a1) * a2 * t2) / A, rel=1e-12)


def test_transmittance_stop_after_crossing():
    """12 parallel surfels of alpha 0.5: T = 2^-k drops below 1e-3 at k = 10,
    and that 10th hit is the last one blended."""
    layers = [one_surfel(np.array([0, 0, -0.1 * k], np.float32), 0.0, 1.0, 1.0, 0.5) for k in range(12)]
    seg, hits = O.trace_segment(stack(layers), [0, 0, 1.0], [0, 0, -1.0])
    assert seg["n_hits"] == 10 and list(hits) == list(range(10))
    assert seg["A"] == pytest.approx(1 - 2.0 ** -10, rel=1e-14)


def test_compositing_invariants_random_scenes():
    """On random scenes: weights are non-negative and sum to A <= 1,
    composites lie in the hull of the blended values, the normal is unit and
    D~ lies between the nearest and farthest blended hit."""
    rng = np.random.default_rng(5)
    for seed in range(6):
        sc = S.random_small_scene(40, seed, spread=0.4)
        for _ in range(25):
            d = rng.normal(size=3)
            d[0] = abs(d[0]) + 1.0
            d /= np.linalg.norm(d)
            seg, hits = O.trace_segment(sc, [0.0, 0.0, 0.0], d, max_hits=64)
            A = seg["A"]
            assert 0.0 <= A <= 1.0
            if seg["n_hits"] == 0:
                assert A == 0.0
                continue
            rho = sc.albedo[hits].astype(np.float64)
            assert np.all(seg["P"] >= A * rho.min(0) - 1e-12) and np.all(seg["P"] <= A * rho.max(0) + 1e-12)
            assert abs(np.linalg.norm(seg["Nn"]) - 1) < 1e-12
            ts = []
            for h in hits:
                s1, _ = O.trace_segment(S.SurfelScene(*[a[h:h + 1] for a in sc.arrays()]), [0, 0, 0], d)
                ts.append(s1["Dn"])
            assert min(ts) - 1e-9 <= seg["Dn"] <= max(ts) + 1e-9
            assert ts == sorted(ts)  # blended in depth order


# -------------------------------------------------- furnace (loop, weights) --

@pytest.mark.parametrize("rho", [0.3, 0.8])
def test_furnace_geometric_series(rho):
    """Closed box, every face emissive L_e and Lambertian rho, emitters
    reflecting (general rendering equation): every sample of every pixel is
    L_e * A * sum_{k=0..B} (rho A)^k exactly; as B grows it approaches
    L_e A / (1 - rho A) (the L = E / (1 - rho) furnace identity)."""
    sc = S.giant_box(rho=rho, r=1.7, gap=1e-6)
    Le, rho = float(sc.radiance[0, 0]), float(sc.albedo[0, 0])  # FP32 values, widened
    cam = S.horizontal_camera(12, 12, hfov=120.0)
    pix = np.arange(144, dtype=np.int32)
    prm = O.Params(emitters_reflect=True)
    for B in [0, 1, 2, 3, 7]:
        out = O.render(sc, cam, pix, "pt", 3, max_bounces=B, rr_start=1000, params=prm, want_samples=True)
        exp = Le * A2 * sum((rho * A2) ** k for k in range(B + 1))
        np.testing.assert_allclose(out["samples"], exp, rtol=1e-11)
    out = O.render(sc, cam, pix[:8], "pt", 2, max_bounces=120, rr_start=1000, params=prm)
    limit = Le * A2 / (1 - rho * A2)
    assert np.all(np.abs(out["rgb"] - limit) <= limit * (rho * A2) ** 121 / (1 - rho * A2) + 1e-10)
    assert abs(limit - Le / (1 - rho)) < 1e-3 * Le / (1 - rho)


# -------------------------------------------- Eq. 4 / Eq. 8 emitter semantics --

def _floor_room(floor_rho=0.3, Le=2.0, cache=0.7):
    return S.giant_box(rho=0.5, r=Le, emissive_faces=[0, 1, 2, 3, 5], floor_rho=floor_rho,
                       floor_cache=cache, gap=1e-6)


def _floor_pixels(cam):
    """Pixels whose primary ray hits the floor z = -1 inside the box (ray-box
    geometry, independent of the renderer)."""
    out = []
    R = cam.c2w[:, :3].astype(np.float64)
    c = cam.c2w[:, 3].astype(np.float64)
    for y in range(cam.height):
        for x in range(cam.width):
            d = R @ np.array([(x + 0.5 - cam.cx) / cam.fx, (y + 0.5 - cam.cy) / cam.fy, 1.0])
            d /= np.linalg.norm(d)
            ts = []
            for ax in range(3):
                if abs(d[ax]) > 1e-12:
                    ts.append(((np.sign(d[ax]) - c[ax]) / d[ax], ax, np.sign(d[ax])))
            t, ax, sg = min(ts)
            out.append(ax == 2 and sg < 0)
    return np.array(out)


def test_floor_reflector_room():
    """Floor non-emissive (albedo rho_f), other faces emissive L_e, emitters do
    not reflect (Eq. 4).  Wall pixels show L_e A; floor pixels receive exactly
    rho_f A * L_e A for any bounce limit >= 1 (a floor cannot see itself, so
    every first bounce lands on an emitter), 0 with no bounce; the floor's
    radiance cache is ignored by path tracing and unused by single bounce."""
    sc = _floor_room(0.3, 2.0)
    Le, rf = float(sc.radiance[0, 0]), float(sc.albedo[8, 0])
    cam = S.look_at_camera(16, 16, 100.0, (0, 0, 0), (1, 0, -1), (0, 0, 1))
    is_floor = _floor_pixels(cam)
    assert 20 < is_floor.sum() < 250
    pix = np.arange(256, dtype=np.int32)
    wall = Le * A2
    floor = rf * A2 * Le * A2
    for kind, B in [("pt", 1), ("pt", 2), ("pt", 5), ("single", 1)]:
        out = O.render(sc, cam, pix, kind, 4, max_bounces=B, rr_start=1000)
        got = out["rgb"][:, 0]
        np.testing.assert_allclose(got[~is_floor], wall, rtol=1e-12)
        np.testing.assert_allclose(got[is_floor], floor, rtol=1e-12)
    out = O.render(sc, cam, pix, "pt", 4, max_bounces=0, rr_start=1000)
    np.testing.assert_allclose(out["rgb"][is_floor, 0], 0.0, atol=0)
    np.testing.assert_allclose(out["rgb"][~is_floor, 0], wall, rtol=1e-12)


def test_first_bounce_geometry_coloured_box():
    """Each wall emits its own colour; the camera sees the non-emissive floor.
    The single-bounce sample of pixel p is rho_f A * A * L(face hit by the
    secondary ray), where the secondary ray starts at X + eps N (X = the
    blended floor point, N = +z) along the cosine direction of the sample's
    Philox draws.  The face is found here by ray-box geometry."""
    colours = {0: (1, 0, 0), 1: (0, 1, 0), 2: (0, 0, 1), 3: (1, 1, 0), 5: (0, 1, 1)}
    sc = S.giant_box(rho=0.5, r=1.0, emissive_faces=list(colours), floor_rho=0.4, gap=1e-6)
    for f, col in colours.items():
        sc.radiance[2 * f:2 * f + 2] = np.array(col, np.float32) * 3.0
    cam = S.look_at_camera(8, 8, 40.0, (0.1, -0.2, 0.3), (0.1, 0.05, -1), (1, 0, 0))
    assert _floor_pixels(cam).all()
    pix = np.arange(64, dtype=np.int32)
    spp, seed, eps = 16, 1234, 1e-3
    out = O.render(sc, cam, pix, "single", spp, seed=seed, want_samples=True)
    R = cam.c2w[:, :3].astype(np.float64)
    c = cam.c2w[:, 3].astype(np.float64)
    checked = 0
    for p in pix:
        x, y = p % 8, p // 8
        d = R @ np.array([(x + 0.5 - cam.cx) / cam.fx, (y + 0.5 - cam.cy) / cam.fy, 1.0])
        d /= np.linalg.norm(d)
        t1 = (-1.0 - c[2]) / d[2]
        t2 = (-1.0 - 1e-6 - c[2]) / d[2]
        Dn = (0.99 * t1 + 0.01 * 0.99 * t2) / A2
        X = c + Dn * d + np.array([0, 0, eps])
        for s in range(spp):
            o = O.philox4x32_10([p, s, 1, 0], [seed, 0])
            u0, u1 = (o[0] >> 8) / 2.0 ** 24, (o[1] >> 8) / 2.0 ** 24
            w = np.array([math.sqrt(u0) * math.cos(2 * math.pi * u1), math.sqrt(u0) * math.sin(2 * math.pi * u1),
                          math.sqrt(1 - u0)])  # basis of n = +z is the identity
            ts = [((np.sign(w[a]) * 1.0 - X[a]) / w[a], a, np.sign(w[a])) for a in range(3) if abs(w[a]) > 1e-12]
            ts.sort()
            if len(ts) > 1 and ts[1][0] - ts[0][0] < 1e-4:
                continue  # lands within a hair of a box edge
            t, a, sg = ts[0]
            face = 2 * a + (1 if sg > 0 else 0)
            exp = float(sc.albedo[8, 0]) * A2 * A2 * sc.radiance[2 * face].astype(np.float64)
            np.testing.assert_allclose(out["samples"][p, s], exp, rtol=1e-9, atol=1e-12)
            checked += 1
    assert checked > 900


def test_single_bounce_equals_pt1_without_caches():
    """With every non-emitter's radiance cache zero and tau_E = 0 (so that any
    vertex carrying emitted radiance counts as an emitter), the single-bounce
    estimator (Eq. 6) and path tracing with one bounce (Eq. 8) agree sample
    for sample.  With tau_E = 0.1 they differ exactly on the secondaries whose
    emitter coverage E lies in (0, 0.1]."""
    sc = S.tiny_room(1024)
    sc.radiance[sc.emissive == 0] = 0.0
    cam = S.Camera(24, 24, 12.0, 12.0, 12.0, 12.0, S.horizontal_camera(24, 24).c2w)
    pix = np.arange(576, dtype=np.int32)
    prm = O.Params(tau_E=0.0)
    a = O.render(sc, cam, pix, "single", 4, seed=3, want_samples=True, params=prm)
    b = O.render(sc, cam, pix, "pt", 4, max_bounces=1, seed=3, want_samples=True, params=prm)
    np.testing.assert_array_equal(a["samples"], b["samples"])
    assert a["rgb"].max() > 0
    # with caches on they differ (single bounce reads the cache at vertex 2)
    sc2 = S.tiny_room(1024)
    c = O.render(sc2, cam, pix, "single", 4, seed=3)
    d = O.render(sc2, cam, pix, "pt", 4, max_bounces=1, seed=3)
    assert np.abs(c["rgb"] - d["rgb"]).max() > 1e-3


def test_russian_roulette_unbiased_closed_form():
    """Floor room with roulette from the first bounce: a floor path survives
    with probability q = rho_f A and is re-weighted to 1, so the mean equals
    the deterministic value rho_f A * L_e A (binomial error bound)."""
    sc = _floor_room(0.3, 2.0)
    Le, rf = float(sc.radiance[0, 0]), float(sc.albedo[8, 0])
    cam = S.look_at_camera(4, 4, 30.0, (0, 0, 0), (0, 0, -1), (1, 0, 0))
    pix = np.arange(16, dtype=np.int32)
    spp = 4096
    out = O.render(sc, cam, pix, "pt", spp, max_bounces=3, rr_start=1, seed=9, want_samples=True)
    q = rf * A2
    vals = out["samples"][:, :, 0]
    np.testing.assert_allclose(np.unique(np.round(vals, 12)), sorted({0.0, round(Le * A2, 12)}))
    mean = vals.mean()
    exp = rf * A2 * Le * A2
    se = Le * A2 * math.sqrt(q * (1 - q) / vals.size)
    assert abs(mean - exp) < 4 * se


# ------------------------------------------------------------- sampler ----

@pytest.mark.parametrize("n", [(0, 0, 1), (0, 0, -1), (1, 0, 0), (0.3, -0.5, 0.81), (0.6, 0.8, -1e-9)])
def test_cosine_sampling_distribution(n):
    """cos(theta) of the sampled directions has density 2c on [0, 1] (so c^2
    is uniform and E[c] = 2/3), directions are unit and in the hemisphere of n,
    and the azimuth about n is uniform."""
    n = np.asarray(n, np.float64)
    n /= np.linalg.norm(n)
    m = 40000
    rng = np.random.default_rng(1)
    u = rng.random((m, 2))
    ws = np.array([O.cosine_direction(n, a, b) for a, b in u])
    assert np.allclose(np.linalg.norm(ws, axis=1), 1.0, atol=1e-12)
    c = ws @ n
    assert c.min() >= -1e-12
    assert abs(c.mean() - 2.0 / 3.0) < 4 * math.sqrt(1 / 18.0 / m)
    counts, _ = np.histogram(c ** 2, bins=20, range=(0, 1))
    chi2 = ((counts - m / 20) ** 2 / (m / 20)).sum()
    assert chi2 < 45  # 19 dof, p ~ 1e-3
    # azimuth: project onto any plane basis orthogonal to n
    a = np.cross(n, [1.0, 0, 0] if abs(n[0]) < 0.9 else [0, 1.0, 0])
    a /= np.linalg.norm(a)
    b = np.cross(n, a)
    phi = np.arctan2(ws @ b, ws @ a)
    counts, _ = np.histogram(phi, bins=16, range=(-math.pi, math.pi))
    assert ((counts - m / 16) ** 2 / (m / 16)).sum() < 40


def test_philox_statistics():
    """The counter-based generator: uniform top bytes, streams differ per key
    and per counter word, and one flipped counter bit flips about half the
    output bits (the paper does not fix an RNG; these are the properties the
    estimator relies on)."""
    m = 20000
    outs = np.array([O.philox4x32_10([i, 7, 3, 0], [11, 0]) for i in range(m)], np.uint64)
    top = (outs >> np.uint64(24)).ravel()
    counts = np.bincount(top.astype(np.int64), minlength=256)
    chi2 = ((counts - top.size / 256) ** 2 / (top.size / 256)).sum()
    assert chi2 < 340  # 255 dof
    assert len({tuple(o) for o in outs.tolist()}) == m
    flips = []
    for i in range(500):
        a = O.philox4x32_10([i, 1, 2, 0], [5, 6])
        for bit in (0, 17, 31):
            b = O.philox4x32_10([i ^ (1 << bit), 1, 2, 0], [5, 6])
            flips.append(sum(bin(x ^ y).count("1") for x, y in zip(a, b)))
    assert abs(np.mean(flips) - 64) < 1.0
    assert O.philox4x32_10([1, 2, 3, 4], [5, 6]) != O.philox4x32_10([1, 2, 3, 4], [5, 7])
    assert O.philox4x32_10([1, 2, 3, 4], [5, 6]) != O.philox4x32_10([1, 2, 3, 5], [5, 6])


# ------------------------------------------------------------ gradients ----

def _fd_check(sc, cam, spp, seed, wts, params_to_check, h_rel=1e-6, tol=1e-6):
    pix = np.arange(cam.width * cam.height, dtype=np.int32)
    prm = O.Params(fp32_eps=0.0)
    grad, _ = O.single_bounce_grad(sc, cam, pix, wts, spp, seed=seed, params=prm)
    base = {k: getattr(sc, k).astype(np.float64) for k in ("pos", "quat", "scale", "opacity", "albedo", "radiance")}
    cols = {"pos": (0, 3), "quat": (3, 7), "scale": (7, 9), "opacity": (9, 10), "albedo": (10, 13),
            "radiance": (13, 16)}

    def loss(over):
        out = O.render(O.OracleScene(sc, over), cam, pix, "single", spp, seed=seed, params=prm)
        return float((out["rgb"] * wts).sum())

    n_ok = 0
    for (name, i, j) in params_to_check:
        arr = base[name].reshape(sc.n, -1)
        x0 = arr[i, j]
        h = h_rel * max(abs(x0), 1.0)
        vals = []
        for s in (-1, 0, 1):
            a2 = arr.copy()
            a2[i, j] = x0 + s * h
            vals.append(loss({name: a2.reshape(base[name].shape)}))
        fd = (vals[2] - vals[0]) / (2 * h)
        left, right = (vals[1] - vals[0]) / h, (vals[2] - vals[1]) / h
        if abs(left - right) > 1e-3 * (abs(fd) + 1e-6):
            continue  # a discrete decision flipped inside [x - h, x + h]
        c0 = cols[name][0]
        g = grad[i, c0 + j]
        assert abs(g - fd) <= tol * (abs(fd) + 1e-3) + 1e-7, (name, i, j, g, fd)
        n_ok += 1
    return grad, n_ok


def test_adjoint_matches_central_differences_small_scene():
    """FP64 adjoint of the single-bounce render vs central differences on
    every parameter of a few-surfel scene (including geometry, through the
    bounce origin X(D~) and direction w'(N~))."""
    sc = S.random_small_scene(6, 21, spread=0.25, emit_frac=0.34)
    # a floor-like big surfel behind, so secondary rays find the others
    cam = S.look_at_camera(8, 8, 50.0, (0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0, 0, 1))
    wts = np.random.default_rng(2).uniform(-1, 1, (64, 3))
    todo = []
    for i in range(sc.n):
        for name, m in (("pos", 3), ("quat", 4), ("scale", 2), ("opacity", 1), ("albedo", 3), ("radiance", 3)):
            for j in range(m):
                todo.append((name, i, j))
    grad, n_ok = _fd_check(sc, cam, 4, 5, wts, todo)
    assert n_ok > 0.9 * len(todo)
    assert np.abs(grad[:, 0:10]).max() > 0  # geometry gradients are non-trivial
    # conditioning runs: the same gradient at rays perturbed at FP32 scale,
    # close to it (the scene is well conditioned) but not identical
    pix = np.arange(cam.width * cam.height, dtype=np.int32)
    g1, _ = O.single_bounce_grad(sc, cam, pix, wts, 4, seed=5, params=O.Params(fp32_eps=0.0))
    assert np.array_equal(g1, grad)
    gj, _ = O.single_bounce_grad(sc, cam, pix, wts, 4, seed=5, run=1)
    assert not np.array_equal(gj, grad)
    assert np.abs(gj - grad).max() <= 1e-4 * np.abs(grad).max()


def test_adjoint_bounce_dependence():
    """A non-emissive plate facing emitters: the plate's own geometry changes
    the bounce origin and direction, so its position gradient has a term the
    primary alone would not give; central differences see the same value."""
    plate = one_surfel(np.array([1.0, 0, 0], np.float32), 0.0, 0.4, 0.4, 0.9)
    plate.quat[:] = np.array([math.cos(math.pi / 4), 0, -math.sin(math.pi / 4), 0], np.float32)  # normal -x
    # lamps off the camera's view cone (3 sigma = 0.36 < their 0.63+ offset)
    lamps = [one_surfel(np.array([0.3, y, z], np.float32), 0.2 * k, 0.12, 0.12, 0.8, r=(5, 4, 3), e=1.0)
             for k, (y, z) in enumerate([(0.6, 0.2), (-0.5, -0.4), (0.1, 0.7)])]
    for l in lamps:
        l.quat[:] = np.array([0.9, 0.2, 0.3, 0.1], np.float32)
    sc = stack([plate] + lamps)
    cam = S.look_at_camera(6, 6, 20.0, (0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0, 0, 1))
    prim, _ = O.primary(sc, cam, np.arange(36, dtype=np.int32))
    assert np.all(prim[:, 7] == 0.0) and np.all(prim[:, 11] > 0.5)  # every pixel sees only the plate
    img = O.render(sc, cam, np.arange(36, dtype=np.int32), "single", 8, seed=3)["rgb"]
    assert img.max() > 0.05  # light arrives through the bounce
    wts = np.ones((36, 3))
    todo = [("pos", 0, j) for j in range(3)] + [("quat", 0, j) for j in range(4)] + \
           [("scale", 0, j) for j in range(2)] + [("opacity", 0, 0), ("albedo", 0, 1)] + \
           [("pos", k, j) for k in (1, 2, 3) for j in range(3)] + [("radiance", 1, 0)]
    grad, n_ok = _fd_check(sc, cam, 8, 3, wts, todo)
    assert n_ok >= len(todo) - 4  # the rest straddle a support edge within +-h


# ------------------------------------------------------------ edge cases ----

def test_empty_scene_and_misses():
    sc = S.SurfelScene(*[np.zeros((0,) + s, np.float32) for s in [(3,), (4,), (2,), (), (3,), (3,), ()]])
    cam = S.horizontal_camera(4, 4)
    out = O.render(sc, cam, np.arange(16, dtype=np.int32), "pt", 2, max_bounces=3)
    assert np.all(out["rgb"] == 0) and np.all(out["segments"] == 1)
    seg, hits = O.trace_segment(S.tiny_room(64), [0, 0, 0], [1, 0, 0], t_lo=1e9)
    assert seg["n_hits"] == 0 and seg["A"] == 0 and len(hits) == 0


def test_paper_constants_golden():
    """The oracle's defaults carry the constants the paper prints."""
    g = json.load(open(os.path.join(HERE, "golden", "paper_constants.json")))
    assert O.Params().tau_E == g["tau_E"]["value"]


def test_radiance_render_adjoint_matches_central_differences():
    """0-bounce (radiance) render, the radiant scene's image R of the primary
    segment (Sec. 3.2; what light baking, Eq. 10, optimises): FP64 adjoint vs
    central differences on every parameter of a few-surfel scene."""
    sc = S.random_small_scene(7, 44, spread=0.25, emit_frac=0.3)
    cam = S.look_at_camera(9, 7, 50.0, (0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0, 0, 1))
    pix = np.arange(63, dtype=np.int32)
    wts = np.random.default_rng(8).uniform(-1, 1, (63, 3))
    prm = O.Params(fp32_eps=0.0)
    grad, _ = O.radiance_grad(sc, cam, pix, wts, params=prm)
    cols = {"pos": (0, 3), "quat": (3, 7), "scale": (7, 9), "opacity": (9, 10), "albedo": (10, 13),
            "radiance": (13, 16)}

    def loss(over):
        rec, _ = O.primary(O.OracleScene(sc, over), cam, pix, mode=0, params=prm)
        return float((rec[:, 4:7] * wts).sum())

    n_ok = n_all = 0
    for name, (c0, c1) in cols.items():
        base = getattr(sc, name).astype(np.float64).reshape(sc.n, -1)
        for i in range(sc.n):
            for j in range(c1 - c0):
                n_all += 1
                h = 1e-6 * max(abs(base[i, j]), 1.0)
                vals = []
                for s in (-1, 0, 1):
                    a = base.copy()
                    a[i, j] += s * h
                    vals.append(loss({name: a.reshape(getattr(sc, name).shape)}))
                fd = (vals[2] - vals[0]) / (2 * h)
                if abs((vals[1] - vals[0]) - (vals[2] - vals[1])) > 1e-3 * (abs(fd) * h + 1e-12):
                    continue
                assert abs(grad[i, c0 + j] - fd) <= 1e-6 * (abs(fd) + 1e-3) + 1e-7, (name, i, j)
                n_ok += 1
    assert n_ok > 0.9 * n_all
    assert np.all(grad[:, 10:13] == 0)  # albedo does not enter the radiance render
