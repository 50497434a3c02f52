"""Pins of the oracle's general system (Eq. AMatGeneral): free shifts (the relaxed model) and
per-view apertures (focal stacks), by consistency with the rank-1 sub-aperture case, the chain
rule, finite differences and model synthesis."""

import numpy as np

from oracle import fdl_oracle as O
from scenes import layered_scene, random_layer_spectra, view_grid


def _bins(H, W, n, seed):
    rng = np.random.default_rng(seed)
    wy, wx = O.half_grid(H, W)
    q = rng.choice(wy.size, n, replace=False)
    return wy[q], wx[q]


def test_rank_one_shifts_reproduce_the_sub_aperture_system():
    u = view_grid(1).astype(np.float64)
    d = np.linspace(-2, 2, 5)
    wy, wx = _bins(16, 16, 40, 0)
    assert np.allclose(O.system_matrix_general(wy, wx, O.shifts_of(u, d)), O.system_matrix(u, d, wy, wx), atol=1e-12)
    views, _ = layered_scene(1, 16, 24, 2, u, d, sigma=1e-3)
    a = O.fit(views, u, d, lam=1e-2)
    b = O.fit_spectra_general(O.half_spectrum(views.astype(np.float64)), O.shifts_of(u, d), 1e-2, d=d, W=24)
    assert np.allclose(a, b, atol=1e-10 * np.abs(a).max())


def test_shift_gradient_chains_to_the_u_and_d_gradients():
    """With P = u d^T, Eq. gradD is the chain rule of dL/dP (Eq. gradP)."""
    rng = np.random.default_rng(1)
    u = view_grid(1).astype(np.float64) + rng.uniform(-0.1, 0.1, (9, 2))
    d = np.linspace(-1.5, 1.5, 4)
    wy, wx = _bins(32, 32, 60, 1)
    b = rng.standard_normal((60, 9, 2)) + 1j * rng.standard_normal((60, 9, 2))
    L0, gu, gd = O.calib_loss_grad(b, wy, wx, u, d, 1e-2, O.REG_LAYER2)
    L1, gP = O.calib_loss_grad_shifts(b, wy, wx, O.shifts_of(u, d), 1e-2, O.REG_LAYER2)
    assert np.isclose(L0, L1, rtol=1e-12)
    assert np.allclose(np.einsum("jka,k->ja", gP, d), gu, rtol=1e-9, atol=1e-9 * np.abs(gu).max())
    assert np.allclose(np.einsum("jka,ja->k", gP, u), gd, rtol=1e-9, atol=1e-9 * np.abs(gd).max())


def test_shift_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    P = rng.uniform(-2, 2, (5, 3, 2))
    wy, wx = _bins(16, 16, 30, 2)
    b = rng.standard_normal((30, 5, 1)) + 1j * rng.standard_normal((30, 5, 1))
    _, g = O.calib_loss_grad_shifts(b, wy, wx, P, 1e-2, O.REG_L2)
    h = 1e-3
    for (j, k, a) in [(0, 0, 0), (2, 1, 1), (4, 2, 0), (3, 0, 1)]:
        def L(t):
            Q = P.copy()
            Q[j, k, a] += t
            return O.calib_loss_grad_shifts(b, wy, wx, Q, 1e-2, O.REG_L2)[0]
        fd = (-L(2 * h) + 8 * L(h) - 8 * L(-h) + L(-2 * h)) / (12 * h)
        assert np.isclose(g[j, k, a], fd, rtol=1e-6, atol=1e-8 * np.abs(g).max())


def test_render_with_shifts_of_a_view_is_the_view():
    X = random_layer_spectra(3, 4, 2, 16, 20).astype(np.complex128)
    d = np.array([-1.0, -0.3, 0.4, 1.2])
    u0 = np.array([0.7, -0.4])
    assert np.allclose(O.render_shifts(X, u0[None] * d[:, None], W=20), O.render(X, d, u0, W=20), atol=1e-13)


def test_focal_stack_from_its_own_model_gives_the_layers_back():
    """Images rendered with a disc aperture at several focus values (Eq. BsFourier) are fitted with
    the same per-image apertures: the layers come back as lambda -> 0 where A is well conditioned."""
    H = W = 16
    N = 3
    X = random_layer_spectra(4, N, 1, H, W).astype(np.complex128)
    d = np.array([-1.5, 0.0, 1.5])
    svals = np.linspace(-2.5, 2.5, 7)
    views = [(O.AP_DISC, 1.0, s, None) for s in svals]
    B = np.stack([O.render_spectrum(X, d, (0.0, 0.0), s, O.AP_DISC, 1.0) for s in svals])  # [K][C][H][Wh]
    P = O.shifts_of(np.zeros((len(svals), 2)), d)
    x = O.fit_spectra_general(B, P, 1e-12, reg=O.REG_L2, d=d, views=views)
    wy, wx = O.half_grid(H, W)
    A = O.system_matrix_general(wy, wx, P, d, views)
    sv = np.linalg.svd(A, compute_uv=False)
    good = (sv[:, 0] / sv[:, -1] < 1e3).reshape(H, W // 2 + 1)
    assert good.sum() > 20
    assert np.allclose(x[:, 0][:, good], X[:, 0][:, good], atol=1e-6 * np.abs(X).max())
    # pinhole views through the general path are the sub-aperture fit
    u = view_grid(1).astype(np.float64)
    pv = [(O.AP_PINHOLE, 0.0, 0.0, None)] * len(u)
    Bv = np.stack([O.render_spectrum(X, d, tuple(uj), 0.0) for uj in u])
    a = O.fit_spectra(Bv, u, d, 1e-2, reg=O.REG_L2)
    b = O.fit_spectra_general(Bv, O.shifts_of(u, d), 1e-2, reg=O.REG_L2, d=d, views=pv)
    assert np.allclose(a, b, atol=1e-12 * np.abs(a).max())
