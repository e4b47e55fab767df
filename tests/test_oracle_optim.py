"""Pins of the optimisation oracle (PQ curve, L1 colour loss, Adam, the fit
loop) against closed forms, the standard's own inverse, finite differences
and textbook behaviour."""
import numpy as np
import pytest

import oracle as O
from oracle import optim as OP
from paper_2601_23065_gb300 import scenes as S


def test_pq_end_points_closed_form():
    # c1 + c2 = 1 + c3 in ST 2084, so the curve reaches exactly 1 at Y = 1
    assert OP.C1 + OP.C2 == 1.0 + OP.C3
    assert OP.pq_curve(1.0) == 1.0
    assert OP.pq_curve(0.0) == pytest.approx(OP.C1 ** OP.M2, rel=1e-15)


def test_pq_inverts_the_standard_eotf():
    Y = np.logspace(-9, 0, 200)
    np.testing.assert_allclose(OP.pq_eotf(OP.pq_curve(Y)), Y, rtol=1e-9)
    E = np.linspace(0.05, 1.0, 50)
    np.testing.assert_allclose(OP.pq_curve(OP.pq_eotf(E)), E, rtol=1e-12)


def test_pq_reference_white():
    # 100 cd/m^2 (1 % of the 10000 cd/m^2 peak) encodes to about 0.508
    assert OP.pq_curve(0.01) == pytest.approx(0.5081, abs=5e-4)
    # monotone increasing over the whole range
    v = OP.pq_curve(np.linspace(0, 1, 10001))
    assert (np.diff(v) > 0).all()


def test_pq_derivative_matches_central_differences():
    peak = 100.0
    x = np.array([1e-6, 1e-3, 0.05, 0.7, 3.0, 40.0, 99.0])
    _, d = OP.pq(x, peak)
    h = 1e-6 * x
    fd = (OP.pq(x + h, peak)[0] - OP.pq(x - h, peak)[0]) / (2 * h)
    np.testing.assert_allclose(d, fd, rtol=1e-6)
    # at or above the peak: value 1, slope 0; at or below 0: value PQ(0) and
    # the slope at the 1e-10 floor (finite, positive)
    v, d = OP.pq(np.array([-1.0, 0.0, 1e-12, 100.0, 150.0]), peak)
    assert v[3] == v[4] == 1.0 and d[3] == d[4] == 0.0
    assert v[0] == v[1] == OP.C1 ** OP.M2
    assert d[0] == d[1] == d[2] == OP.pq(np.array([1e-10 * peak]), peak)[1][0] > 0


def test_pq_l1_loss_and_gradient():
    rng = np.random.default_rng(4)
    pred = rng.uniform(0, 20, 300)
    target = rng.uniform(0, 20, 300)
    loss, g = OP.pq_l1(pred, target, 100.0, 0.5)
    a, _ = OP.pq(pred, 100.0)
    b, _ = OP.pq(target, 100.0)
    assert loss == pytest.approx(0.5 * np.mean(np.abs(a - b)), rel=1e-14)
    # gradient against central differences of the loss, one element at a time
    for k in (0, 17, 123, 299):
        h = 1e-6 * pred[k]
        p1, p2 = pred.copy(), pred.copy()
        p1[k] += h
        p2[k] -= h
        fd = (OP.pq_l1(p1, target, 100.0, 0.5)[0] - OP.pq_l1(p2, target, 100.0, 0.5)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5)
    # zero at the optimum, symmetric, and sign(0) = 0 in the gradient
    l0, g0 = OP.pq_l1(pred, pred, 100.0)
    assert l0 == 0.0 and (g0 == 0).all()
    assert OP.pq_l1(target, pred, 100.0, 0.5)[0] == pytest.approx(loss, rel=1e-14)
    assert OP.pq_l1(np.zeros(0), np.zeros(0), 100.0) == (0.0, pytest.approx(np.zeros(0)))


def test_adam_first_step_and_constant_gradient():
    rng = np.random.default_rng(5)
    g = rng.normal(size=50)
    p0 = rng.normal(size=50)
    lr, eps = 0.01, 1e-8
    # bias correction makes m_hat = g and v_hat = g^2 at every step of a
    # constant gradient: each step is -lr g / (|g| + eps)
    p, m, v = p0, np.zeros(50), np.zeros(50)
    for t in range(1, 6):
        p_prev = p
        p, m, v = OP.adam_step(p, g, m, v, t, lr, eps=eps)
        np.testing.assert_allclose(p - p_prev, -lr * g / (np.abs(g) + eps), rtol=1e-9, atol=1e-15)
    # beta1 = beta2 = 0: the same normalised step from any history
    p, m, v = OP.adam_step(p0, g, rng.normal(size=50), rng.uniform(0, 1, 50), 7, lr, beta1=0.0, beta2=0.0, eps=eps)
    np.testing.assert_allclose(p - p0, -lr * g / (np.abs(g) + eps), rtol=1e-9, atol=1e-15)
    # projection
    p, _, _ = OP.adam_step(np.array([0.001, 0.999]), np.array([1.0, -1.0]), np.zeros(2), np.zeros(2), 1, 0.01,
                           lo=0.0, hi=1.0)
    assert p.tolist() == [0.0, 1.0]


def test_adam_minimises_a_quadratic():
    x, m, v = np.array([-2.0, 5.0]), np.zeros(2), np.zeros(2)
    for t in range(1, 3001):
        x, m, v = OP.adam_step(x, 2 * (x - np.array([3.0, -1.0])), m, v, t, 0.05)
    np.testing.assert_allclose(x, [3.0, -1.0], atol=1e-2)


def test_radiance_fit_recovers_a_single_surfel():
    """0-bounce fit (Eq. 10) of one surfel's radiance to a target rendered
    with known radiance: the blend is linear in r with a positive weight, so
    the unique minimiser is the known radiance."""
    sc = S.random_small_scene(1, 3, spread=0.0, emit_frac=0.0)
    sc.scale[:] = 0.3
    cam = S.look_at_camera(6, 6, 20.0, (0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0, 0, 1))
    pix = np.arange(36, dtype=np.int32)
    r_gt = np.array([[2.0, 0.5, 7.0]], np.float32)
    gt = S.SurfelScene(sc.pos, sc.quat, sc.scale, sc.opacity, sc.albedo, r_gt, sc.emissive)
    target = O.primary(gt, cam, pix, mode=0)[0][:, 4:7]
    assert (target.max(axis=1) > 0).sum() > 10
    # start from grey (baking starts from the existing radiance; from black the
    # unbounded PQ slope at 0 gives one huge first gradient that stalls Adam)
    start = S.SurfelScene(sc.pos, sc.quat, sc.scale, sc.opacity, sc.albedo, np.ones((1, 3), np.float32),
                          sc.emissive)
    adam = dict(lr=0.1, beta1=0.9, beta2=0.999, eps=1e-8, lo=0.0, hi=np.inf)
    _, r, _, _, losses, _ = OP.fit(start, [cam], [target], 1, 400, adam=adam)
    # a constant-step Adam ends oscillating within about lr of the minimiser
    assert losses[-1] < 5e-2 * losses[0]
    np.testing.assert_allclose(r[0], r_gt[0], atol=0.1)


def test_stage1_fit_recovers_face_albedo():
    """Stage 1 (Eq. 7) of the oracle in a closed box of giant surfels lit by
    an emissive ceiling: single-bounce targets rendered with a known albedo
    per face; from 0.5 everywhere the loop recovers each visible
    non-emissive face's albedo (a sign or index slip in the loss, the
    albedo gradient or Adam would not)."""
    sc = S.giant_box(rho=0.5, r=4.0, e=1.0, emissive_faces=[5], floor_cache=0.4)
    face_rho = np.random.default_rng(3).uniform(0.2, 0.8, 6)
    alb = np.repeat(face_rho, 2)[:, None].repeat(3, 1).astype(np.float32)
    gt = S.SurfelScene(sc.pos, sc.quat, sc.scale, sc.opacity, alb, sc.radiance, sc.emissive)
    cams = [S.horizontal_camera(16, 12, forward=f)
            for f in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0.0), (0.3, 0.2, -1.0))]
    targets = [O.render(gt, c, np.arange(c.width * c.height, dtype=np.int32), "single", 64, seed=77)["rgb"]
               for c in cams]
    start = S.SurfelScene(sc.pos, sc.quat, sc.scale, sc.opacity, np.full_like(alb, 0.5), sc.radiance,
                          sc.emissive)
    adam = dict(lr=0.02, beta1=0.9, beta2=0.999, eps=1e-8, lo=0.0, hi=1.0)
    _, x, _, _, losses, _ = OP.fit(start, cams, targets, 0, 200, spp=16, seed=1, peak=100.0, adam=adam)
    err = np.abs(x[0::2, 0] - face_rho)[:5]
    assert err.max() < 0.06 and err.mean() < 0.03
    assert x[10, 0] == 0.5  # the emitting ceiling's albedo never enters an image
