"""Plain FP64 CPU oracle of the Fourier Disparity Layer hot path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA path.

Everything is float64 / complex128 numpy, written for a reader to check
against the paper by eye; it is slow on purpose.  Sections and equations named
below are those of Le Pendu, Guillemot, Smolic, "A Fourier Disparity Layer
representation for Light Fields" (arXiv 1901.06919).

Conventions (the readings adopted where the paper is silent):

* forward DFT ``b(w) = sum_x B(x) exp(-2 pi i w.x)``, unnormalised (Sec. V-A:
  "the discrete Fourier Transform of each image"; sign of Eq. FourierLF);
* frequencies in cycles/pixel: ``w_y = fftfreq(H)[ky]`` (so ``ky = H/2`` is
  -1/2) and ``w_x = kx / W`` for the stored half ``kx = 0 .. W/2`` (Sec. VII:
  only half of the spectrum is computed);
* 2D phase ``A_jk = exp(+2 pi i d_k (u_j . w))`` (Eq. AMatGeneral with
  ``psi_j = delta``; the 2D form the paper calls straightforward, Sec. III);
* view regulariser ``Gamma*Gamma = diag(|w|^4 d_k^4 + eps)`` (Eq. 2ndOrderView
  plus the epsilon of Sec. V-C1), scaled by lambda;
* layer regulariser ``Gamma = tridiag(1, -2, 1)`` (Eq. 2ndOrderLayer); l2 is
  ``Gamma = I`` (Sec. V-C);
* an image is the real part of the inverse DFT of the spectrum completed by
  ``X(-w) := conj X(w)`` outside the stored half, divided by ``H*W``.

Parity pins for every function live in ``tests/test_oracle_*.py``.
"""

from __future__ import annotations

import numpy as np
from scipy.special import j1 as _bessel_j1

REG_VIEW2, REG_LAYER2, REG_L2 = 0, 1, 2
AP_PINHOLE, AP_DISC, AP_SQUARE, AP_POINTS, AP_TABLE = 0, 1, 2, 3, 4


# ----------------------------------------------------------------------------
# Discrete Fourier transforms (Sec. V-A, Sec. VI-A: "inverse Fourier transform")
# ----------------------------------------------------------------------------

def fft_radix2(x, axis: int = -1, inverse: bool = False) -> np.ndarray:
    """Textbook iterative radix-2 decimation-in-time DFT along ``axis``.

    Forward: ``X[k] = sum_n x[n] exp(-2 pi i k n / n_len)``; ``inverse=True``
    uses ``exp(+...)``.  No normalisation.  The length must be a power of two.
    """
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n = x.shape[-1]
    if n & (n - 1):
        raise ValueError("length must be a power of two")
    bits = n.bit_length() - 1
    idx = np.arange(n)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    x = x[..., rev]
    sign = 1.0 if inverse else -1.0
    lead = x.shape[:-1]
    m = 1
    while m < n:
        w = np.exp(sign * 1j * np.pi * np.arange(m) / m)  # exp(-/+ 2 pi i k / (2m))
        blocks = x.reshape(lead + (n // (2 * m), 2, m))
        even = blocks[..., 0, :]
        odd = blocks[..., 1, :] * w
        x = np.concatenate([even + odd, even - odd], axis=-1).reshape(lead + (n,))
        m *= 2
    return np.moveaxis(x, -1, axis)


def dft_direct(x, axis: int = -1, inverse: bool = False) -> np.ndarray:
    """DFT along ``axis`` by its definition, for any length: the product with the matrix
    ``F[k, n] = exp(-/+ 2 pi i (k n mod len) / len)`` (``inverse=True`` takes ``+``).  No
    normalisation.  ``k n`` is reduced modulo the length in integers before the exponential."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n = x.shape[-1]
    kn = np.outer(np.arange(n), np.arange(n)) % n
    sign = 1.0 if inverse else -1.0
    F = np.exp(sign * 2j * np.pi * kn / n)
    return np.moveaxis(x @ F.T, -1, axis)


def dft_1d(x, axis: int = -1, inverse: bool = False) -> np.ndarray:
    """The radix-2 DFT for power-of-two lengths, the definition otherwise."""
    n = np.shape(x)[axis]
    if n & (n - 1) == 0:
        return fft_radix2(x, axis=axis, inverse=inverse)
    return dft_direct(x, axis=axis, inverse=inverse)


def dft2(img) -> np.ndarray:
    """Full 2D forward DFT over the last two axes."""
    return dft_1d(dft_1d(img, axis=-1), axis=-2)


def half_spectrum(img) -> np.ndarray:
    """Stored half ``kx = 0 .. W/2`` of the 2D DFT of real images (Sec. VII)."""
    W = np.shape(img)[-1]
    return dft2(img)[..., : W // 2 + 1]


def dft_at_bins(img, ky, kx) -> np.ndarray:
    """DFT of images ``[..., H, W]`` at listed bins by the definition (no FFT):
    ``b = sum_{y,x} B(y, x) exp(-2 pi i (ky y / H + kx x / W))``; returns ``[..., nbins]``."""
    img = np.asarray(img, np.float64)
    H, W = img.shape[-2:]
    ky = np.asarray(ky)
    kx = np.asarray(kx)
    ex = np.exp(-2j * np.pi * np.outer(np.arange(W), kx) / W)  # [W, nb]
    ey = np.exp(-2j * np.pi * np.outer(np.arange(H), ky) / H)  # [H, nb]
    rows = img @ ex  # [..., H, nb]
    return np.einsum("...yb,yb->...b", rows, ey)


def complete_half(S: np.ndarray, W: int) -> np.ndarray:
    """Full spectrum from a stored half: ``X(-w) := conj X(w)`` for ``kx > W/2``."""
    H = S.shape[-2]
    full = np.zeros(S.shape[:-1] + (W,), dtype=np.complex128)
    full[..., : W // 2 + 1] = S
    for kx in range(W // 2 + 1, W):
        mirror_rows = (-np.arange(H)) % H
        full[..., :, kx] = np.conj(S[..., mirror_rows, W - kx])
    return full


def image_from_half(S: np.ndarray, W: int) -> np.ndarray:
    """Real image: Re(inverse DFT of the completed spectrum) / (H W)."""
    H = S.shape[-2]
    full = complete_half(S, W)
    z = dft_1d(dft_1d(full, axis=-1, inverse=True), axis=-2, inverse=True)
    return np.real(z) / (H * W)


# ----------------------------------------------------------------------------
# Frequencies and the per-frequency system (Sec. V-A, Eq. AMatGeneral)
# ----------------------------------------------------------------------------

def freq_y(H: int) -> np.ndarray:
    ky = np.arange(H)
    return np.where(ky < (H + 1) // 2, ky, ky - H) / H


def freq_x_half(W: int) -> np.ndarray:
    return np.arange(W // 2 + 1) / W


def half_grid(H: int, W: int):
    """``(w_y, w_x)`` of every stored bin, flattened row-major over ``[H][W/2+1]``."""
    wy, wx = np.meshgrid(freq_y(H), freq_x_half(W), indexing="ij")
    return wy.ravel(), wx.ravel()


def system_matrix(u, d, wy, wx) -> np.ndarray:
    """``A[q, j, k] = exp(+2 pi i d_k (u_j . w_q))`` (Eq. AMatGeneral, sub-aperture views)."""
    u = np.asarray(u, np.float64)
    d = np.asarray(d, np.float64)
    wy = np.atleast_1d(np.asarray(wy, np.float64))
    wx = np.atleast_1d(np.asarray(wx, np.float64))
    theta = wx[:, None] * u[None, :, 0] + wy[:, None] * u[None, :, 1]  # [q, j] cycles per unit d
    return np.exp(2j * np.pi * theta[:, :, None] * d[None, None, :])


def layer2_gtg(N: int) -> np.ndarray:
    """``Gamma^T Gamma`` for ``Gamma = tridiag(1, -2, 1)`` (Eq. 2ndOrderLayer)."""
    Gam = -2.0 * np.eye(N) + np.eye(N, k=1) + np.eye(N, k=-1)
    return Gam.T @ Gam


def regulariser(reg: int, d, wy, wx, eps: float) -> np.ndarray:
    """``Gamma*Gamma`` per bin, shape ``[q, N, N]`` (Sec. V-C).

    view2: ``diag(|w|^4 d_k^4 + eps)`` (Eq. 2ndOrderView, epsilon of Sec. V-C1);
    layer2: Eq. 2ndOrderLayer (no epsilon); l2: identity.
    """
    d = np.asarray(d, np.float64)
    N = len(d)
    q = np.atleast_1d(wy).shape[0]
    if reg == REG_VIEW2:
        w2 = np.atleast_1d(wx) ** 2 + np.atleast_1d(wy) ** 2
        diag = w2[:, None] ** 2 * d[None, :] ** 4 + eps
        out = np.zeros((q, N, N))
        out[:, np.arange(N), np.arange(N)] = diag
        return out
    if reg == REG_LAYER2:
        return np.broadcast_to(layer2_gtg(N), (q, N, N)).copy()
    if reg == REG_L2:
        return np.broadcast_to(np.eye(N), (q, N, N)).copy()
    raise ValueError("unknown regulariser")


def gauss_solve(G: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Solve ``G X = Y`` per batch entry by Gaussian elimination with partial pivoting.

    ``G``: ``[..., n, n]``, ``Y``: ``[..., n, m]``.  Plain row operations,
    vectorised only across the independent batch entries.
    """
    G = np.asarray(G, np.complex128)
    Y = np.asarray(Y, np.complex128)
    lead = G.shape[:-2]
    n = G.shape[-1]
    m = Y.shape[-1]
    M = np.concatenate([G, Y], axis=-1).reshape((-1, n, n + m)).copy()
    rows = np.arange(M.shape[0])
    for k in range(n):
        p = k + np.argmax(np.abs(M[:, k:, k]), axis=1)
        tmp = M[rows, k].copy()
        M[rows, k] = M[rows, p]
        M[rows, p] = tmp
        f = M[:, k + 1:, k] / M[:, k, k][:, None]
        M[:, k + 1:, k:] -= f[:, :, None] * M[:, k, None, k:]
    X = np.zeros((M.shape[0], n, m), np.complex128)
    for k in range(n - 1, -1, -1):
        acc = M[:, k, n:].copy()
        if k + 1 < n:
            acc -= np.einsum("bj,bjm->bm", M[:, k, k + 1:n], X[:, k + 1:])
        X[:, k] = acc / M[:, k, k][:, None]
    return X.reshape(lead + (n, m))


def solve_bins(b, u, d, wy, wx, lam: float, eps: float, reg: int = REG_VIEW2):
    """Tikhonov least squares at every listed bin (Eq. LayerConstructProb).

    ``b``: ``[q, K, C]`` input coefficients.  Returns ``x`` of shape
    ``[q, N, C]`` from the closed form ``(A*A + lambda Gamma*Gamma) x = A* b``
    (Eq. LayerConstructionClosedForm), solved by :func:`gauss_solve`.
    """
    A = system_matrix(u, d, wy, wx)
    AH = np.conj(np.swapaxes(A, -1, -2))
    G = AH @ A + lam * regulariser(reg, d, wy, wx, eps)
    y = AH @ np.asarray(b, np.complex128)
    return gauss_solve(G, y)


def full_width(Wh: int, W=None) -> int:
    """Image width of a stored half of ``Wh = W//2 + 1`` columns: ``W`` when given (an odd
    width cannot be told from ``Wh``), else the even width ``2 (Wh - 1)``."""
    if W is None:
        return 2 * (Wh - 1)
    if W // 2 + 1 != Wh:
        raise ValueError("W does not match the stored half")
    return int(W)


def fit_spectra(b_half, u, d, lam: float, eps: float = 1e-4, reg: int = REG_VIEW2,
                chunk: int = 2048, W=None) -> np.ndarray:
    """Layer spectra ``[N][C][H][W/2+1]`` from input half spectra ``[K][C][H][W/2+1]``."""
    K, C, H, Wh = b_half.shape
    W = full_width(Wh, W)
    wy, wx = half_grid(H, W)
    bq = np.moveaxis(b_half.reshape(K, C, H * Wh), -1, 0)  # [q, K, C]
    N = len(d)
    xq = np.empty((H * Wh, N, C), np.complex128)
    for s in range(0, H * Wh, chunk):
        sl = slice(s, s + chunk)
        xq[sl] = solve_bins(bq[sl], u, d, wy[sl], wx[sl], lam, eps, reg)
    return np.moveaxis(xq, 0, -1).reshape(N, C, H, Wh)


def fit(views, u, d, lam: float, eps: float = 1e-4, reg: int = REG_VIEW2) -> np.ndarray:
    """Layer construction of Sec. V-A: DFT of every view, then one solve per bin."""
    views = np.asarray(views, np.float64)
    return fit_spectra(half_spectrum(views), u, d, lam, eps, reg, W=views.shape[-1])


# ----------------------------------------------------------------------------
# Rendering (Sec. VI-A, Eq. BsFourier)
# ----------------------------------------------------------------------------

def aperture_table(raster, Z: int) -> np.ndarray:
    """Transform of a drawn aperture (Sec. VI-A: rasterise, zero-pad, DFT), half spectrum
    ``[Z][Z//2+1]`` normalised to ``psi_hat(0) = 1``.

    ``raster`` is ``[P][P]`` with P odd; pixel ``(iy, ix)`` sits at ``u = ((ix - c) h, (iy - c) h)``,
    ``c = (P - 1) / 2``.  It is placed in a ``Z x Z`` array with its centre pixel at index 0
    (wrap-around), so that table entry ``(gy, gx)`` is ``psi_hat`` at ``nu = (gy, gx) / (Z h)``.
    """
    R = np.asarray(raster, np.float64)
    P = R.shape[0]
    if R.shape != (P, P) or P % 2 == 0 or P > Z:
        raise ValueError("the raster must be square with an odd side no larger than Z")
    c = (P - 1) // 2
    pad = np.zeros((Z, Z))
    for iy in range(P):
        for ix in range(P):
            pad[(iy - c) % Z, (ix - c) % Z] += R[iy, ix]
    return half_spectrum(pad) / R.sum()


def aperture_lookup(T, h: float, nu_y, nu_x) -> np.ndarray:
    """``psi_hat(nu)`` from a table of :func:`aperture_table` by bilinear interpolation
    (Sec. VI-A: linear interpolation) on the grid ``nu = g / (Z h)``, periodic in ``g`` with
    period Z, the columns not stored taken from ``psi_hat(-nu) = conj psi_hat(nu)``."""
    T = np.asarray(T, np.complex128)
    Z = T.shape[0]
    gy = np.asarray(nu_y, np.float64) * Z * h
    gx = np.asarray(nu_x, np.float64) * Z * h
    y0 = np.floor(gy)
    x0 = np.floor(gx)
    fy = gy - y0
    fx = gx - x0
    y0 = y0.astype(np.int64)
    x0 = x0.astype(np.int64)

    def fetch(iy, ix):
        iy = iy % Z
        ix = ix % Z
        stored = ix <= Z // 2
        direct = T[iy, np.where(stored, ix, 0)]
        mirror = np.conj(T[(-iy) % Z, np.where(stored, 0, Z - ix)])
        return np.where(stored, direct, mirror)

    return ((1 - fy) * (1 - fx) * fetch(y0, x0) + (1 - fy) * fx * fetch(y0, x0 + 1)
            + fy * (1 - fx) * fetch(y0 + 1, x0) + fy * fx * fetch(y0 + 1, x0 + 1))


def aperture_ft(kind: int, radius: float, nu_y, nu_x, points=None) -> np.ndarray:
    """``psi_hat(nu) = int psi(u) exp(-2 pi i u . nu) du`` with ``int psi = 1``.

    DISC of radius r: ``2 J1(2 pi r |nu|) / (2 pi r |nu|)``; SQUARE of half
    side r: ``sinc(2 r nu_x) sinc(2 r nu_y)`` (normalised sinc, as in
    Eq. GTG); POINTS: ``(1/M) sum_m exp(-2 pi i u_m . nu)`` for offsets
    ``u_m`` given as they are; TABLE: :func:`aperture_lookup` of the table passed as
    ``points`` with raster pitch ``h = radius``; PINHOLE (or r = 0): 1 (Sec. III, psi = delta).
    """
    nu_y = np.asarray(nu_y, np.float64)
    nu_x = np.asarray(nu_x, np.float64)
    if kind == AP_TABLE:
        return aperture_lookup(points, radius, nu_y, nu_x)
    if kind == AP_POINTS:
        pts = np.asarray(points, np.float64)
        ph = pts[:, 0].reshape((-1,) + (1,) * nu_x.ndim) * nu_x + \
            pts[:, 1].reshape((-1,) + (1,) * nu_x.ndim) * nu_y
        return np.mean(np.exp(-2j * np.pi * ph), axis=0)
    if kind == AP_PINHOLE or radius == 0.0:
        return np.ones(np.broadcast(nu_y, nu_x).shape, np.complex128)
    if kind == AP_DISC:
        z = 2 * np.pi * radius * np.sqrt(nu_x ** 2 + nu_y ** 2)
        safe = np.where(z == 0, 1.0, z)
        return np.where(z == 0, 1.0, 2 * _bessel_j1(safe) / safe).astype(np.complex128)
    if kind == AP_SQUARE:
        return (np.sinc(2 * radius * nu_x) * np.sinc(2 * radius * nu_y)).astype(np.complex128)
    raise ValueError("unknown aperture")


def render_spectrum(layers, d, u0, s: float, kind: int = AP_PINHOLE, radius: float = 0.0,
                    points=None, W=None) -> np.ndarray:
    """Half spectrum of the image ``B^s_{u0}``:

    ``sum_k exp(+2 pi i d_k (u0 . w)) psi_hat((s - d_k) w) L^k(w)`` (Eq. BsFourier).
    """
    N, C, H, Wh = layers.shape
    W = full_width(Wh, W)
    wy, wx = half_grid(H, W)
    wy = wy.reshape(H, Wh)
    wx = wx.reshape(H, Wh)
    d = np.asarray(d, np.float64)
    out = np.zeros((C, H, Wh), np.complex128)
    for k in range(N):
        shift = np.exp(2j * np.pi * d[k] * (u0[0] * wx + u0[1] * wy))
        filt = aperture_ft(kind, radius, (s - d[k]) * wy, (s - d[k]) * wx, points)
        out += (shift * filt)[None] * layers[k]
    return out


def render(layers, d, u0, s: float = 0.0, kind: int = AP_PINHOLE, radius: float = 0.0,
           points=None, W=None) -> np.ndarray:
    """Rendered image ``[C][H][W]`` (Sec. VI-A: Eq. BsFourier, then the inverse DFT)."""
    W = full_width(layers.shape[-1], W)
    return image_from_half(render_spectrum(layers, d, u0, s, kind, radius, points, W), W)


def shift_and_sum(layers_spatial, d, u0, s, points) -> np.ndarray:
    """Spatial-domain image for integer shifts: Eq. refocus with a discrete aperture.

    ``B(x) = (1/M) sum_m sum_k layer_k(x + (u0 + u_m) d_k - u_m s)``, periodic;
    every shift must be an integer number of pixels.
    """
    out = np.zeros(layers_spatial.shape[1:])
    for (px, py) in points:
        for k, dk in enumerate(d):
            sx = (u0[0] + px) * dk - px * s
            sy = (u0[1] + py) * dk - py * s
            if sx != int(sx) or sy != int(sy):
                raise ValueError("shift_and_sum needs integer shifts")
            out += np.roll(layers_spatial[k], (-int(sy), -int(sx)), axis=(-2, -1))
    return out / len(points)


# ----------------------------------------------------------------------------
# Calibration (Sec. V-B, Eqs. CalibrationProb, gradD, gradP)
# ----------------------------------------------------------------------------

def calib_loss_grad(b, wy, wx, u, d, lam: float, reg: int = REG_LAYER2):
    """Objective of Eq. CalibrationProb over the listed bins, and its gradient.

    ``b``: ``[q, K, C]``.  The layers are first solved at the current ``u, d``
    with the closed form; the loss is ``sum_{q,c} |A x - b|^2 + lambda |Gamma x|^2``
    (every listed bin weighted 1).  With ``P^a = u_a d^T`` for ``a in {x, y}``,
    Eq. gradP gives ``dL/dP^a_jk = 4 pi sum_{q,c} w_a Im(r_j conj(A_jk) conj(x_k))``
    and Eq. gradD ``grad_u[j, a] = sum_k d_k dL/dP^a_jk``,
    ``grad_d[k] = sum_{j, a} u_{j,a} dL/dP^a_jk``.
    ``reg`` must not depend on ``d`` (layer2 or l2, Sec. V-C2).
    Returns ``(loss, grad_u [K][2], grad_d [N])``.
    """
    if reg == REG_VIEW2:
        raise ValueError("the calibration gradient needs a regulariser independent of d")
    u = np.asarray(u, np.float64)
    d = np.asarray(d, np.float64)
    wy = np.atleast_1d(np.asarray(wy, np.float64))
    wx = np.atleast_1d(np.asarray(wx, np.float64))
    x = solve_bins(b, u, d, wy, wx, lam, 0.0, reg)  # [q, N, C]
    A = system_matrix(u, d, wy, wx)  # [q, K, N]
    r = A @ x - b  # [q, K, C]
    R = regulariser(reg, d, wy, wx, 0.0)
    loss = np.sum(np.abs(r) ** 2) + lam * np.real(np.einsum("qkc,qkl,qlc->", np.conj(x), R, x))
    # core[q, j, k] = sum_c Im(r_jc conj(A_jk) conj(x_kc))
    core = np.imag(np.einsum("qjc,qjk,qkc->qjk", r, np.conj(A), np.conj(x)))
    gPx = 4 * np.pi * np.einsum("q,qjk->jk", wx, core)
    gPy = 4 * np.pi * np.einsum("q,qjk->jk", wy, core)
    grad_u = np.stack([gPx @ d, gPy @ d], axis=1)
    grad_d = u[:, 0] @ gPx + u[:, 1] @ gPy
    return float(loss), grad_u, grad_d


def calib_loss(b, wy, wx, u, d, lam: float, reg: int = REG_LAYER2) -> float:
    """Eq. CalibrationProb at its minimum over x, for fixed ``u, d``."""
    return calib_loss_grad(b, wy, wx, u, d, lam, reg)[0]


# ----------------------------------------------------------------------------
# The general system of Eq. AMatGeneral: free shifts (the relaxed model of the
# denoising section, P without the rank-1 constraint P = u d^T) and per-view
# apertures and focus (focal stacks and hybrid inputs, Sec. V)
# ----------------------------------------------------------------------------

def shifts_of(u, d) -> np.ndarray:
    """``P[j, k] = u_j d_k`` as ``[K][N][2]`` (x, y): the rank-1 shifts of Sec. V-B."""
    u = np.asarray(u, np.float64)
    d = np.asarray(d, np.float64)
    return u[:, None, :] * d[None, :, None]


def system_matrix_general(wy, wx, P, d=None, views=None) -> np.ndarray:
    """``A[q, j, k] = exp(+2 pi i P_jk . w_q) psi_hat_j((s_j - d_k) w_q)`` (Eq. AMatGeneral with
    the shift ``u_j d_k`` replaced by ``P_jk``).  ``views[j] = (kind, radius, s, points)`` is the
    aperture and focus of image j (None: every image a sub-aperture view, psi = delta); the
    aperture argument needs ``d``."""
    P = np.asarray(P, np.float64)
    wy = np.atleast_1d(np.asarray(wy, np.float64))
    wx = np.atleast_1d(np.asarray(wx, np.float64))
    phase = wx[:, None, None] * P[None, :, :, 0] + wy[:, None, None] * P[None, :, :, 1]
    A = np.exp(2j * np.pi * phase)
    if views is not None:
        d = np.asarray(d, np.float64)
        for j, (kind, radius, s, pts) in enumerate(views):
            nu_y = (s - d)[None, :] * wy[:, None]
            nu_x = (s - d)[None, :] * wx[:, None]
            A[:, j, :] = A[:, j, :] * aperture_ft(kind, radius, nu_y, nu_x, pts)
    return A


def solve_system(b, A, lam: float, R) -> np.ndarray:
    """Closed form of Eq. LayerConstructionClosedForm for given ``A [q, K, N]``, ``R [q, N, N]``."""
    AH = np.conj(np.swapaxes(A, -1, -2))
    return gauss_solve(AH @ A + lam * R, AH @ np.asarray(b, np.complex128))


def fit_spectra_general(b_half, P, lam: float, eps: float = 1e-4, reg: int = REG_VIEW2, d=None, views=None,
                        W=None, chunk: int = 2048) -> np.ndarray:
    """Layer spectra ``[N][C][H][W/2+1]`` for the general system (the view regulariser needs d)."""
    K, C, H, Wh = b_half.shape
    W = full_width(Wh, W)
    N = np.asarray(P).shape[1]
    wy, wx = half_grid(H, W)
    bq = np.moveaxis(b_half.reshape(K, C, H * Wh), -1, 0)
    dd = np.zeros(N) if d is None else np.asarray(d, np.float64)
    if reg == REG_VIEW2 and d is None:
        raise ValueError("the view regulariser needs the layer disparities")
    xq = np.empty((H * Wh, N, C), np.complex128)
    for s0 in range(0, H * Wh, chunk):
        sl = slice(s0, s0 + chunk)
        A = system_matrix_general(wy[sl], wx[sl], P, dd, views)
        xq[sl] = solve_system(bq[sl], A, lam, regulariser(reg, dd, wy[sl], wx[sl], eps))
    return np.moveaxis(xq, 0, -1).reshape(N, C, H, Wh)


def render_shifts(layers, Pb, W=None) -> np.ndarray:
    """Image ``sum_k layer_k`` shifted by ``Pb[k]`` (``[N][2]``), i.e. the view rendered with the
    relaxed model's shifts (Eq. FourierView with ``u0 d_k`` replaced by ``P_k``)."""
    N, C, H, Wh = layers.shape
    W = full_width(Wh, W)
    wy, wx = half_grid(H, W)
    Pb = np.asarray(Pb, np.float64)
    S = np.zeros((C, H * Wh), np.complex128)
    for k in range(N):
        S += np.exp(2j * np.pi * (Pb[k, 0] * wx + Pb[k, 1] * wy))[None] * layers[k].reshape(C, -1)
    return image_from_half(S.reshape(C, H, Wh), W)


def calib_loss_grad_shifts(b, wy, wx, P, lam: float, reg: int = REG_LAYER2):
    """Eq. CalibrationProb over the listed bins with free shifts ``P [K][N][2]`` and its gradient
    ``dL/dP [K][N][2]`` by Eq. gradP: ``4 pi sum_{q,c} w_a Im(r_j conj(A_jk) conj(x_k))``
    (the relaxed model calibrates P directly).  ``reg`` must not depend on d."""
    if reg == REG_VIEW2:
        raise ValueError("the calibration gradient needs a regulariser independent of d")
    P = np.asarray(P, np.float64)
    wy = np.atleast_1d(np.asarray(wy, np.float64))
    wx = np.atleast_1d(np.asarray(wx, np.float64))
    N = P.shape[1]
    A = system_matrix_general(wy, wx, P)
    R = regulariser(reg, np.zeros(N), wy, wx, 0.0)
    x = solve_system(b, A, lam, R)
    r = A @ x - b
    loss = np.sum(np.abs(r) ** 2) + lam * np.real(np.einsum("qkc,qkl,qlc->", np.conj(x), R, x))
    core = np.imag(np.einsum("qjc,qjk,qkc->qjk", r, np.conj(A), np.conj(x)))
    g = np.stack([4 * np.pi * np.einsum("q,qjk->jk", wx, core), 4 * np.pi * np.einsum("q,qjk->jk", wy, core)], -1)
    return float(loss), g
