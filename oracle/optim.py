"""FP64 oracle of the shading-parameter optimisation: the PQ colour loss of
Eq. 7 and Eq. 10, Adam, and the two loops (Stage 1, Eq. 7: albedo through the
single-bounce render with r fixed; light baking, Eq. 10: radiance through the
0-bounce render).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: imported by ``tests/``
and the CPU-baseline leg of ``bench.py``; it shares no code with the CUDA
path.  Plain numpy in float64, written from the definitions:

* PQ: the inverse EOTF of SMPTE ST 2084 (the curve Sec. 3.2 applies to linear
  radiance before the colour loss), on Y = x / peak clamped to [0, 1]; its
  slope, unbounded at Y = 0, is taken at max(Y, 1e-10), and is 0 at or above
  the peak (the reading both sides use).
* L_c: mean absolute difference of the PQ values (the L1 colour loss of the
  3DGS family the paper cites for L_c; the D-SSIM term is not named and is
  left out), weighted by lambda_c; sign(0) = 0 in the gradient.
* Adam: Kingma and Ba (2015), Algorithm 1, with bias-corrected moments,
  followed by a projection onto [lo, hi].
"""
from __future__ import annotations

import numpy as np

from . import primary, radiance_grad, render, single_bounce_grad

# SMPTE ST 2084 constants (exact binary fractions given by the standard)
M1 = 2610.0 / 16384.0
M2 = 2523.0 / 4096.0 * 128.0
C1 = 3424.0 / 4096.0
C2 = 2413.0 / 4096.0 * 32.0
C3 = 2392.0 / 4096.0 * 32.0
Y_LO = 1e-10


def pq_curve(Y):
    """Inverse EOTF of ST 2084 on normalised luminance Y in [0, 1]."""
    Y = np.asarray(Y, np.float64)
    y = Y ** M1
    return ((C1 + C2 * y) / (1.0 + C3 * y)) ** M2


def pq_eotf(E):
    """EOTF of ST 2084 (PQ value -> normalised luminance), the standard's
    inverse formula; used only to pin ``pq_curve``."""
    E = np.asarray(E, np.float64)
    e = E ** (1.0 / M2)
    return (np.maximum(e - C1, 0.0) / (C2 - C3 * e)) ** (1.0 / M1)


def pq(x, peak):
    """(PQ(clamp(x / peak, 0, 1)), slope).  The slope is dPQ/dx at
    max(x / peak, 1e-10) below the peak (the curve's slope is unbounded at 0)
    and 0 at or above it."""
    x = np.asarray(x, np.float64)
    Yr = x / peak
    v = pq_curve(np.clip(Yr, 0.0, 1.0))
    Y = np.clip(Yr, Y_LO, 1.0)
    y = Y ** M1
    f = (C1 + C2 * y) / (1.0 + C3 * y)
    df_dy = (C2 - C1 * C3) / (1.0 + C3 * y) ** 2
    dy_dY = M1 * Y ** (M1 - 1.0)
    d = M2 * f ** (M2 - 1.0) * df_dy * dy_dY / peak
    return v, np.where(Yr < 1.0, d, 0.0)


def pq_l1(pred, target, peak, lambda_c=1.0):
    """(loss, dloss/dpred) of lambda_c * mean |PQ(pred) - PQ(target)|."""
    pred = np.asarray(pred, np.float64).ravel()
    target = np.asarray(target, np.float64).ravel()
    n = pred.size
    if n == 0:
        return 0.0, np.zeros(0)
    a, da = pq(pred, peak)
    b, _ = pq(target, peak)
    diff = a - b
    loss = lambda_c * np.abs(diff).sum() / n
    grad = lambda_c / n * np.sign(diff) * da
    return float(loss), grad


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, lo=-np.inf, hi=np.inf):
    """One step t = step of Adam; returns new (p, m, v)."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    p = np.clip(p - lr * mhat / (np.sqrt(vhat) + eps), lo, hi)
    return p, m, v


def fit(scene, cams, targets, field, iters, spp=1, seed=0, peak=100.0, lambda_c=1.0, adam=None,
        first_step=0, m=None, v=None, params=None):
    """The optimisation loop, step t = first_step + k + 1 on view
    (first_step + k) mod len(cams): render, PQ-L1 loss, gradient of the field
    (albedo for field 0, radiance for field 1), Adam.  Returns
    (scene with the updated field, m, v, losses, gradients of each step)."""
    import copy
    adam = dict(lr=0.01, beta1=0.9, beta2=0.999, eps=1e-8, lo=0.0, hi=1.0) if adam is None else adam
    sc = copy.deepcopy(scene)
    name = "albedo" if field == 0 else "radiance"
    cols = slice(10, 13) if field == 0 else slice(13, 16)
    x = getattr(sc, name).astype(np.float64).reshape(-1)
    m = np.zeros_like(x) if m is None else np.asarray(m, np.float64).reshape(-1)
    v = np.zeros_like(x) if v is None else np.asarray(v, np.float64).reshape(-1)
    losses, grads = [], []
    for k in range(iters):
        t = first_step + k + 1
        vi = (first_step + k) % len(cams)
        cam = cams[vi]
        pix = np.arange(cam.width * cam.height, dtype=np.int32)
        setattr(sc, name, x.reshape(-1, 3).astype(np.float32))
        if field == 0:
            img = render(sc, cam, pix, "single", spp, seed=seed + t, params=params)["rgb"]
        else:
            img = primary(sc, cam, pix, mode=0, params=params)[0][:, 4:7]
        loss, dL = pq_l1(img, targets[vi], peak, lambda_c)
        dL = dL.reshape(-1, 3)
        if field == 0:
            g = single_bounce_grad(sc, cam, pix, dL, spp, seed=seed + t, params=params)[0][:, cols]
        else:
            g = radiance_grad(sc, cam, pix, dL, params=params)[0][:, cols]
        g = g.reshape(-1)
        x, m, v = adam_step(x, g, m, v, t, **adam)
        losses.append(loss)
        grads.append(g)
    # the parameters are FP32 on the render side: the oracle keeps its own
    # FP64 copy but hands the scene FP32 values
    setattr(sc, name, x.reshape(-1, 3).astype(np.float32))
    return sc, x.reshape(-1, 3), m, v, losses, grads
