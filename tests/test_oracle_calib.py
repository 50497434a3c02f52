"""Pins of the oracle's calibration objective and gradient (Sec. V-B): central finite
differences of Eq. CalibrationProb, and the (c u, d / c) invariance of P = u d^T."""

import numpy as np
import pytest

from oracle import fdl_oracle as O
from scenes import jittered_grid, occluding_planes


def _problem(seed=0, H=16, W=16, g=1, N=5):
    rng = np.random.default_rng(seed)
    u_true = jittered_grid(g, 0.15, rng)
    views, _ = occluding_planes(seed, H, W, 1, u_true, n_planes=3, drange=2.0)
    b = O.half_spectrum(views.astype(np.float64))  # [K][C][H][Wh]
    K, C = b.shape[:2]
    wy, wx = O.half_grid(H, W)
    sel = rng.choice(len(wy), 40, replace=False)
    bq = np.moveaxis(b.reshape(K, C, -1), -1, 0)[sel]
    u0 = np.asarray(jittered_grid(g, 0.05, rng), np.float64)
    d0 = np.linspace(-2, 2, N) + rng.uniform(-0.1, 0.1, N)
    return bq, wy[sel], wx[sel], u0, d0


@pytest.mark.parametrize("reg", [O.REG_LAYER2, O.REG_L2])
def test_gradient_matches_central_differences(reg):
    bq, wy, wx, u, d = _problem()
    lam = 1e-1
    loss, gu, gd = O.calib_loss_grad(bq, wy, wx, u, d, lam, reg)
    # fourth-order central differences, so that truncation stays below 1e-9
    h = 1e-3

    def central(f):
        return (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h)

    num_u = np.zeros_like(u)
    for j in range(u.shape[0]):
        for a in range(2):
            def fu(t, j=j, a=a):
                v = u.copy()
                v[j, a] += t
                return O.calib_loss(bq, wy, wx, v, d, lam, reg)
            num_u[j, a] = central(fu)
    num_d = np.zeros_like(d)
    for k in range(len(d)):
        def fd(t, k=k):
            v = d.copy()
            v[k] += t
            return O.calib_loss(bq, wy, wx, u, v, lam, reg)
        num_d[k] = central(fd)
    assert np.linalg.norm(gu - num_u) <= 1e-6 * np.linalg.norm(num_u)
    assert np.linalg.norm(gd - num_d) <= 1e-6 * np.linalg.norm(num_d)


def test_loss_invariant_under_rescaling_of_u_and_d():
    bq, wy, wx, u, d = _problem(1)
    l0 = O.calib_loss(bq, wy, wx, u, d, 1e-1)
    l1 = O.calib_loss(bq, wy, wx, 2.5 * u, d / 2.5, 1e-1)
    assert np.isclose(l0, l1, rtol=1e-10)


def test_view_regulariser_rejected_for_calibration():
    bq, wy, wx, u, d = _problem(2)
    with pytest.raises(ValueError):
        O.calib_loss_grad(bq, wy, wx, u, d, 1e-1, O.REG_VIEW2)
