"""Pins of the oracle's per-frequency solve (Sec. V-A, V-C) against library routines,
closed forms, layer recovery on synthetic scenes, and symmetry."""

import os

import numpy as np
import pytest

from oracle import fdl_oracle as O
from scenes import layered_scene, view_grid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gauss_solve_matches_library_and_pivots():
    rng = np.random.default_rng(0)
    G = rng.standard_normal((5, 7, 7)) + 1j * rng.standard_normal((5, 7, 7))
    Y = rng.standard_normal((5, 7, 3)) + 1j * rng.standard_normal((5, 7, 3))
    X = O.gauss_solve(G, Y)
    assert np.allclose(X, np.linalg.solve(G, Y), atol=1e-10)
    # a zero leading pivot needs a row exchange
    G2 = np.array([[0, 1, 2], [1, 0, 3], [4, -3, 8]], complex)
    y2 = np.array([[1], [2], [3]], complex)
    assert np.allclose(G2 @ O.gauss_solve(G2, y2), y2, atol=1e-13)


def test_system_matrix_hand_values():
    # u = (1, 0), d = 2, w = (w_y, w_x) = (0, 1/8): phase 2 * 1/8 cycles = pi/2 -> i
    A = O.system_matrix([[1.0, 0.0]], [2.0], [0.0], [1 / 8])
    assert np.allclose(A[0, 0, 0], 1j, atol=1e-15)
    # u = (-1, 3), d = 0.5, w = (1/4, 1/8): theta = -1/8 + 3/4 = 5/8, phase 5/16 cycles
    A = O.system_matrix([[-1.0, 3.0]], [0.5], [0.25], [0.125])
    assert np.allclose(A[0, 0, 0], np.exp(2j * np.pi * 5 / 16), atol=1e-15)


def test_layer2_gtg_matches_hand_expansion():
    ref = np.loadtxt(os.path.join(GOLDEN, "layer2_gtg_n5.txt"))
    assert np.array_equal(O.layer2_gtg(5), ref)


@pytest.mark.parametrize("reg", [O.REG_VIEW2, O.REG_LAYER2, O.REG_L2])
def test_solution_is_the_tikhonov_minimiser(reg):
    """Closed form == least squares on the stacked system [A; sqrt(lam) Gamma] (library lstsq)."""
    rng = np.random.default_rng(1)
    K, N, C = 9, 6, 2
    u = view_grid(1)
    d = np.linspace(-2, 2, N)
    lam, eps = 3e-2, 1e-3
    wy = np.array([0.1, -0.3, 0.0])
    wx = np.array([0.2, 0.05, 0.5])
    b = rng.standard_normal((3, K, C)) + 1j * rng.standard_normal((3, K, C))
    x = O.solve_bins(b, u, d, wy, wx, lam, eps, reg)
    A = O.system_matrix(u, d, wy, wx)
    for q in range(3):
        if reg == O.REG_VIEW2:
            w2 = wx[q] ** 2 + wy[q] ** 2
            Gam = np.diag(np.sqrt(w2 ** 2 * d ** 4 + eps))
        elif reg == O.REG_LAYER2:
            Gam = -2 * np.eye(N) + np.eye(N, k=1) + np.eye(N, k=-1)
        else:
            Gam = np.eye(N)
        M = np.vstack([A[q], np.sqrt(lam) * Gam])
        rhs = np.vstack([b[q], np.zeros((N, C))])
        ref = np.linalg.lstsq(M, rhs, rcond=None)[0]
        assert np.allclose(x[q], ref, atol=1e-10 * np.abs(ref).max())
        # normal-equation residual
        G = A[q].conj().T @ A[q] + lam * Gam.T @ Gam
        y = A[q].conj().T @ b[q]
        assert np.linalg.norm(G @ x[q] - y) <= 1e-13 * np.linalg.norm(y) * np.linalg.cond(G)


def test_dc_bin_closed_form():
    """At w = 0, A = 1 1^T: x_k = sum_j b_j / (K N + lambda eps) for every layer."""
    K, N = 9, 8
    u = view_grid(1)
    d = np.linspace(-2, 2, N)
    lam, eps = 1e-2, 1e-4
    rng = np.random.default_rng(2)
    b = rng.standard_normal((1, K, 1)) + 1j * rng.standard_normal((1, K, 1))
    x = O.solve_bins(b, u, d, [0.0], [0.0], lam, eps)
    assert np.allclose(x[0, :, 0], b.sum() / (K * N + lam * eps), rtol=1e-12)


def test_eigendecomposition_cross_check():
    rng = np.random.default_rng(3)
    u = view_grid(2)
    d = np.linspace(-3, 3, 11)
    wy = rng.uniform(-0.5, 0.5, 16)
    wx = rng.uniform(0, 0.5, 16)
    b = rng.standard_normal((16, len(u), 3)) + 1j * rng.standard_normal((16, len(u), 3))
    lam, eps = 1e-1, 1e-2
    x = O.solve_bins(b, u, d, wy, wx, lam, eps)
    A = O.system_matrix(u, d, wy, wx)
    AH = np.conj(np.swapaxes(A, 1, 2))
    G = AH @ A + lam * O.regulariser(O.REG_VIEW2, d, wy, wx, eps)
    ev, V = np.linalg.eigh(G)
    ref = V @ ((np.conj(np.swapaxes(V, 1, 2)) @ (AH @ b)) / ev[:, :, None])
    assert np.allclose(x, ref, atol=1e-9 * np.abs(ref).max())


def test_hermitian_symmetry_of_full_spectrum_solve():
    """Real inputs: b(-w) = conj b(w) and A(-w) = conj A(w), so x(-w) = conj x(w) (Sec. VII)."""
    rng = np.random.default_rng(4)
    u = view_grid(1)
    d = np.linspace(-2, 2, 5)
    wy = rng.uniform(-0.5, 0.5, 8)
    wx = rng.uniform(-0.5, 0.5, 8)
    b = rng.standard_normal((8, 9, 2)) + 1j * rng.standard_normal((8, 9, 2))
    x_pos = O.solve_bins(b, u, d, wy, wx, 1e-2, 1e-4)
    x_neg = O.solve_bins(np.conj(b), u, d, -wy, -wx, 1e-2, 1e-4)
    assert np.allclose(x_neg, np.conj(x_pos), atol=1e-13 * np.abs(x_pos).max())


@pytest.mark.parametrize("H,W", [(32, 32), (27, 45), (30, 42)])
def test_layer_recovery_from_model_views(H, W):
    """Views synthesised from N layers (K >= N, no noise) give the layers back as lambda -> 0
    on every bin where A is well conditioned (Sec. V-A; scene model of Sec. IV-A), for
    power-of-two and other sizes."""
    u = view_grid(1)
    d = np.linspace(-2, 2, 8)
    views, layers = layered_scene(7, H, W, 1, u, d, sigma=0.0)
    truth = np.fft.rfft2(layers)  # [N][C][H][W/2+1]
    x = O.fit(views, u, d, lam=1e-14, eps=1e-4)
    wy, wx = O.half_grid(H, W)
    A = O.system_matrix(u, d, wy, wx)
    sv = np.linalg.svd(A, compute_uv=False)
    good = (sv[:, 0] / sv[:, -1] <= 1e2).reshape(H, W // 2 + 1)
    assert good.sum() > 50
    xt = truth[:, 0][:, good]
    xr = x[:, 0][:, good]
    # the views are float32, so the recovered layers carry float32 input rounding
    rel = np.linalg.norm(xr - xt) / np.linalg.norm(xt)
    assert rel < 1e-5
    # with float64 views the recovery is exact to 1e-10
    views64 = np.zeros((len(u), 1, H, W))
    F = np.fft.fft2(layers)
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.fftfreq(W)[None, :]
    for j in range(len(u)):
        for k in range(len(d)):
            views64[j] += np.real(np.fft.ifft2(F[k] * np.exp(2j * np.pi * d[k] * (u[j, 0] * fx + u[j, 1] * fy))))
    x64 = O.fit(views64, u, d, lam=1e-14, eps=1e-4)
    rel = np.linalg.norm(x64[:, 0][:, good] - xt) / np.linalg.norm(xt)
    assert rel < 1e-10


def test_residual_shrinks_with_lambda():
    """The data term |A x - b| of the Tikhonov solution never grows as lambda decreases;
    measured through renders at every input view (Eq. FourierView)."""
    H = W = 16
    u = view_grid(1)
    d = np.linspace(-2, 2, 8)
    views, _ = layered_scene(3, H, W, 1, u, d, sigma=1e-2)
    errs = []
    for lam in [1e0, 1e-1, 1e-2, 1e-3, 1e-4]:
        x = O.fit(views, u, d, lam=lam, eps=1e-4)
        errs.append(sum(np.sum((O.render(x, d, u[j]) - views[j]) ** 2) for j in range(len(u))))
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-12) for i in range(len(errs) - 1))
    assert errs[-1] < 0.9 * errs[0]
