"""GPU calibration objective and gradient (Sec. V-B) against the FP64 oracle.

Tolerance: gradients within relative L2 1e-4 of the FP64 reference gradient (itself pinned by
finite differences in the CPU tests); the loss within 1e-5 relative.
"""

import numpy as np
import pytest
import torch

from oracle import fdl_oracle as O
from scenes import jittered_grid, occluding_planes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def calib_problem():
    rng = np.random.default_rng(3)
    u_true = jittered_grid(2, 0.15, rng)
    H = W = 32
    views, _ = occluding_planes(5, H, W, 1, u_true, n_planes=4, drange=2.0)
    spec = np.ascontiguousarray(O.half_spectrum(views.astype(np.float64)).astype(np.complex64))
    u0 = np.asarray(jittered_grid(2, 0.0, rng), np.float32)
    d0 = np.linspace(-2, 2, 12).astype(np.float32)
    return spec, u0, d0


def _oracle(spec, u, d, lam, reg, bins):
    K, C, H, Wh = spec.shape
    W = 2 * (Wh - 1)
    wy, wx = O.half_grid(H, W)
    bq = np.moveaxis(spec.astype(np.complex128).reshape(K, C, -1), -1, 0)
    return O.calib_loss_grad(bq[bins], wy[bins], wx[bins], u.astype(np.float64), d.astype(np.float64), lam, reg)


@pytest.mark.parametrize("reg,precision", [("layer2", "df"), ("l2", "df"), ("layer2", "f64")])
def test_gradient_matches_fp64_reference(fdl, calib_problem, reg, precision):
    spec, u, d = calib_problem
    lam = 1e-1
    r = {"layer2": O.REG_LAYER2, "l2": O.REG_L2}[reg]
    nb = spec.shape[2] * spec.shape[3]
    for bins in (np.arange(nb), np.random.default_rng(1).choice(nb, 96, replace=False)):
        loss, gu, gd = fdl.calib_grad(torch.from_numpy(spec).cuda(), torch.from_numpy(u).cuda(),
                                      torch.from_numpy(d).cuda(), lam, reg=reg,
                                      bins=torch.from_numpy(bins.astype(np.int32)).cuda(), precision=precision)
        L_ref, gu_ref, gd_ref = _oracle(spec, u, d, lam, r, bins)
        assert abs(loss.item() - L_ref) <= 1e-5 * abs(L_ref)
        gu = gu.cpu().numpy()
        gd = gd.cpu().numpy()
        assert np.linalg.norm(gu - gu_ref) <= 1e-4 * np.linalg.norm(gu_ref)
        assert np.linalg.norm(gd - gd_ref) <= 1e-4 * np.linalg.norm(gd_ref)


def test_all_bins_default_and_determinism(fdl, calib_problem):
    spec, u, d = calib_problem
    S, U, D = (torch.from_numpy(a).cuda() for a in (spec, u, d))
    a = fdl.calib_grad(S, U, D, 1e-1)
    b = fdl.calib_grad(S, U, D, 1e-1)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    nb = spec.shape[2] * spec.shape[3]
    c = fdl.calib_grad(S, U, D, 1e-1, bins=torch.arange(nb, dtype=torch.int32, device="cuda"))
    for x, y in zip(a, c):
        assert torch.equal(x, y)
