"""Pins of the oracle's rendering (Sec. III, Sec. IV-B Eq. BsFourier, Sec. VI-A):
brute-force spatial shift-and-sum, aperture closed forms against quadrature,
special cases psi = delta and d_k = s, and the direction of the shift (Appendix A)."""

import numpy as np
import pytest

from oracle import fdl_oracle as O
from scenes import noise_1f


def _layers(seed, N, C, H, W):
    rng = np.random.default_rng(seed)
    sp = np.stack([np.stack([noise_1f(rng, H, W) for _ in range(C)]) for _ in range(N)])
    return sp, np.fft.rfft2(sp)


@pytest.mark.parametrize("u0,s", [((0, 0), 0), ((1, -2), 1), ((-3, 2), -2), ((2, 1), 3)])
def test_fourier_render_equals_spatial_shift_and_sum(u0, s):
    """Integer d_k, s, u0 and a lattice aperture: Eq. BsFourier == Eq. refocus brute force."""
    H = W = 16
    d = [-2, -1, 0, 1, 3]
    sp, X = _layers(11, len(d), 2, H, W)
    pts = [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)]
    img = O.render(X, d, u0, s, O.AP_POINTS, 0.0, pts)
    ref = O.shift_and_sum(sp, d, u0, s, pts)
    assert np.max(np.abs(img - ref)) < 1e-13
    # pinhole: a single aperture point at the origin
    img = O.render(X, d, u0, s)
    ref = O.shift_and_sum(sp, d, u0, s, [(0, 0)])
    assert np.max(np.abs(img - ref)) < 1e-13


def test_shift_direction():
    """A bright pixel at x0 in layer k is seen at x0 - d_k u from view u (Eq. Prior2)."""
    H = W = 16
    layer = np.zeros((1, 1, H, W))
    layer[0, 0, 5, 7] = 1.0
    X = np.fft.rfft2(layer)
    img = O.render(X, [2.0], (1.0, -1.0))
    y, x = np.unravel_index(np.argmax(img[0]), img[0].shape)
    assert (y, x) == (5 - 2 * (-1), 7 - 2 * 1)


def test_disc_and_square_transforms_match_quadrature():
    """psi_hat of the normalised disc and square, against a midpoint-rule integral."""
    n = 801
    r = 1.3
    g = (np.arange(n) + 0.5) / n * 2 * r - r
    uy, ux = np.meshgrid(g, g, indexing="ij")
    da = (2 * r / n) ** 2
    disc = (ux ** 2 + uy ** 2 <= r * r).astype(float)
    disc /= disc.sum() * da
    sq = np.ones_like(ux) / (4 * r * r)
    for nu in [(0.0, 0.0), (0.1, 0.2), (-0.3, 0.05), (0.4, -0.4)]:
        kern = np.exp(-2j * np.pi * (ux * nu[1] + uy * nu[0])) * da
        got_d = O.aperture_ft(O.AP_DISC, r, nu[0], nu[1])
        got_s = O.aperture_ft(O.AP_SQUARE, r, nu[0], nu[1])
        assert abs(got_d - np.sum(disc * kern)) < 2e-3
        assert abs(got_s - np.sum(sq * kern)) < 1e-5


def test_pinhole_special_cases():
    """psi = delta gives psi_hat = 1: radius 0 of any shape is the pinhole render (Sec. IV-B)."""
    sp, X = _layers(5, 4, 1, 16, 16)
    d = [-1.5, -0.2, 0.7, 2.1]
    ref = O.render(X, d, (0.3, -0.8), 0.0)
    for kind in (O.AP_DISC, O.AP_SQUARE):
        assert np.array_equal(O.render(X, d, (0.3, -0.8), 1.7, kind, 0.0), ref)


def test_layer_in_focus_is_not_blurred():
    """A single layer with d_k = s renders identically for every aperture: psi_hat(0) = 1."""
    sp, X = _layers(6, 1, 1, 16, 16)
    d = [0.8]
    ref = O.render(X, d, (1.2, 0.4), 0.8)
    for kind in (O.AP_DISC, O.AP_SQUARE):
        for r in (0.5, 2.0):
            assert np.allclose(O.render(X, d, (1.2, 0.4), 0.8, kind, r), ref, atol=1e-14)


def test_refocus_blurs_out_of_focus_layer():
    """An out-of-focus layer loses contrast under a wide aperture; the mean is kept."""
    sp, X = _layers(8, 1, 1, 32, 32)
    sharp = O.render(X, [2.0], (0, 0), 0.0)
    blur = O.render(X, [2.0], (0, 0), 0.0, O.AP_DISC, 2.0)
    assert np.std(blur) < 0.7 * np.std(sharp)
    assert np.isclose(np.mean(blur), np.mean(sharp), rtol=1e-12)


def test_render_at_input_view_equals_model_prediction():
    """Render at u_j equals row j of A x (the model of Eq. FourierView), any lambda."""
    from scenes import layered_scene, view_grid
    u = view_grid(1)
    d = np.linspace(-2, 2, 6)
    views, _ = layered_scene(9, 16, 16, 1, u, d, sigma=1e-2)
    x = O.fit(views, u, d, lam=1e-1)
    wy, wx = O.half_grid(16, 16)
    A = O.system_matrix(u, d, wy, wx)  # [q, K, N]
    for j in (0, 4, 8):
        pred = np.einsum("qk,kq->q", A[:, j, :], x[:, 0].reshape(len(d), -1)).reshape(16, 9)
        spec = O.render_spectrum(x, d, u[j], 0.0)[0]
        assert np.allclose(spec, pred, atol=1e-10 * np.abs(pred).max())


@pytest.mark.parametrize("u0,s", [((1, 0), 2), ((-2, 1), -1)])
def test_asymmetric_aperture_points(u0, s):
    """An aperture that is not point-symmetric fixes the sign of psi_hat's argument."""
    H = W = 16
    d = [-1, 0, 2]
    sp, X = _layers(12, len(d), 1, H, W)
    pts = [(0, 0), (1, 0), (0, 1), (1, 1), (2, -1)]
    img = O.render(X, d, u0, s, O.AP_POINTS, 0.0, pts)
    assert np.max(np.abs(img - O.shift_and_sum(sp, d, u0, s, pts))) < 1e-13


def test_view_regulariser_is_mean_squared_angular_laplacian():
    """Eq. 2ndDer / Eq. GTG: Gamma*Gamma / r over a large region of the camera plane is the
    mean of |Laplacian_u L_u(w)|^2 / (4 pi^2)^2, and tends to diag(|w|^4 d^4) (Eq. 2ndOrderView).
    The Laplacian is taken by finite differences of the oracle's own render."""
    H = W = 8
    rng = np.random.default_rng(13)
    d = np.array([-1.7, -0.4, 0.9, 2.3])
    X = np.zeros((len(d), 1, H, W // 2 + 1), complex)
    ky, kx = 3, 1
    X[:, 0, ky, kx] = rng.standard_normal(len(d)) + 1j * rng.standard_normal(len(d))
    wy, wx = O.freq_y(H)[ky], O.freq_x_half(W)[kx]
    h = 1e-3
    acc = 0.0
    n = 4000
    for uu in rng.uniform(-400, 400, size=(n, 2)):
        def L(du):
            return O.render_spectrum(X, d, (uu[0] + du[0], uu[1] + du[1]), 0.0)[0, ky, kx]
        lap = (L((h, 0)) + L((-h, 0)) + L((0, h)) + L((0, -h)) - 4 * L((0, 0))) / h ** 2
        acc += abs(lap) ** 2
    mean = acc / n / (4 * np.pi ** 2) ** 2
    R = O.regulariser(O.REG_VIEW2, d, [wy], [wx], 0.0)[0]
    x = X[:, 0, ky, kx]
    ref = np.real(np.conj(x) @ R @ x)
    assert abs(mean - ref) < 0.05 * ref


# ---- drawn apertures (Sec. VI-A: rasterise, zero-pad, DFT, linear interpolation)

def test_aperture_table_of_one_pixel_is_a_pinhole():
    T = O.aperture_table(np.ones((1, 1)), 32)
    assert np.allclose(T, 1.0, atol=1e-14)
    rng = np.random.default_rng(0)
    nu = rng.uniform(-3, 3, (2, 50))
    assert np.allclose(O.aperture_lookup(T, 0.25, nu[0], nu[1]), 1.0, atol=1e-14)


def test_aperture_table_nodes_are_the_point_set_transform():
    """At table nodes the drawn aperture is exactly the discrete aperture of its pixels
    (weights as point multiplicities), including an asymmetric raster."""
    rng = np.random.default_rng(1)
    R = rng.integers(0, 3, (5, 5)).astype(float)
    R[2, 2] = 1.0
    h, Z = 0.3, 64
    T = O.aperture_table(R, Z)
    pts = [((ix - 2) * h, (iy - 2) * h) for iy in range(5) for ix in range(5) for _ in range(int(R[iy, ix]))]
    g = rng.integers(-40, 40, (2, 30))
    nu_y, nu_x = g[0] / (Z * h), g[1] / (Z * h)
    ref = O.aperture_ft(O.AP_POINTS, 0.0, nu_y, nu_x, np.array(pts))
    got = O.aperture_lookup(T, h, nu_y, nu_x)
    assert np.allclose(got, ref, atol=1e-12)
    assert np.allclose(O.aperture_lookup(T, h, -nu_y, -nu_x), np.conj(got), atol=1e-12)


def test_aperture_table_interpolation_error_shrinks_with_padding():
    """Between nodes the bilinear value approaches the transform with the error of linear
    interpolation, O((grid spacing)^2)."""
    R = np.ones((3, 3))
    h = 0.5
    pts = np.array([((ix - 1) * h, (iy - 1) * h) for iy in range(3) for ix in range(3)])
    rng = np.random.default_rng(2)
    nu = rng.uniform(-1.5, 1.5, (2, 200))
    ref = O.aperture_ft(O.AP_POINTS, 0.0, nu[0], nu[1], pts)
    errs = [np.max(np.abs(O.aperture_lookup(O.aperture_table(R, Z), h, nu[0], nu[1]) - ref)) for Z in (32, 64, 128)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-3 and errs[1] / errs[2] > 3.0


def test_render_with_a_one_pixel_table_is_the_pinhole_render():
    rng = np.random.default_rng(3)
    X = (rng.standard_normal((3, 1, 16, 9)) + 1j * rng.standard_normal((3, 1, 16, 9)))
    d = np.array([-1.0, 0.0, 1.5])
    T = O.aperture_table(np.ones((1, 1)), 16)
    a = O.render(X, d, (0.3, -0.2), 0.7, O.AP_TABLE, 0.4, T)
    b = O.render(X, d, (0.3, -0.2), 0.7, O.AP_PINHOLE, 0.0)
    assert np.allclose(a, b, atol=1e-13)


@pytest.mark.parametrize("H,W", [(15, 21), (16, 24)])
@pytest.mark.parametrize("kind,radius", [(O.AP_PINHOLE, 0.0), (O.AP_DISC, 1.3), (O.AP_SQUARE, 0.8),
                                         (O.AP_POINTS, 0.0)])
def test_rendered_spectrum_of_real_layers_is_hermitian(H, W, kind, radius):
    """Real layers and a real aperture give a real image, so the stored kx = 0 column of the
    rendered spectrum obeys B(-w_y, 0) = conj B(w_y, 0) (Sec. VII) for any non-integer u0, s and
    d_k; the even-H Nyquist row, whose partner is itself, is left out.  A frequency mapped
    without its sign (k / H instead of (k - H) / H past the middle) breaks it."""
    _, X = _layers(11, 5, 2, H, W)
    d = np.array([-2.3, -0.7, 0.4, 1.1, 2.6])
    pts = np.array([[0.0, 0.0], [1.3, -0.4], [-0.6, 2.1]])  # not symmetric: psi_hat is complex
    B = O.render_spectrum(X, d, (0.37, -1.41), 0.55, kind, radius, pts if kind == O.AP_POINTS else None, W)
    rows = [ky for ky in range(1, H) if 2 * ky != H]
    mirror = [(H - ky) % H for ky in rows]
    scale = np.abs(B[:, :, 0]).max()
    assert np.max(np.abs(B[:, mirror, 0] - np.conj(B[:, rows, 0]))) < 1e-12 * scale
    assert np.max(np.abs(B[:, 0, 0].imag)) < 1e-12 * scale  # the DC bin is real
