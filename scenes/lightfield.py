"""Seeded synthetic light fields with the shapes of the paper's workloads.

Conventions shared by everything in this repository (Sec. III notation):

* a view position is ``u = (u_x, u_y)`` in view-grid units; views are stored
  ``[K][C][H][W]`` float32, row-major, ``y`` the row index;
* a layer of disparity ``d`` seen from ``u`` is the central-view layer
  translated so that ``view(x) = layer(x + u * d)`` (Appendix A, Eq. Prior2:
  ``L(x, u) = L(x + u d_k, 0)``), with periodic wrap-around.

Nothing here computes a layer construction or a render; inputs only.
"""

from __future__ import annotations

import numpy as np


def view_grid(g: int) -> np.ndarray:
    """Integer view positions of a (2g+1)x(2g+1) grid, float32 ``[K][2]``.

    View ``j = iy * (2g+1) + ix`` sits at ``(ix - g, iy - g)``.
    """
    r = np.arange(-g, g + 1, dtype=np.float32)
    uy, ux = np.meshgrid(r, r, indexing="ij")
    return np.stack([ux.ravel(), uy.ravel()], axis=1).astype(np.float32)


def jittered_grid(g: int, jitter: float, rng: np.random.Generator) -> np.ndarray:
    """A view grid with every position moved by U(-jitter, jitter) per axis."""
    u = view_grid(g).astype(np.float64)
    u += rng.uniform(-jitter, jitter, size=u.shape)
    return u.astype(np.float32)


def _freq_grid(H: int, W: int):
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.fftfreq(W)[None, :]
    return fy, fx


def noise_1f(rng: np.random.Generator, H: int, W: int, power: float = 1.0,
             zero_nyquist: bool = False) -> np.ndarray:
    """Real noise image with a 1/f^power amplitude spectrum, min-max scaled to [0, 1].

    The DC term is zero before scaling.  With ``zero_nyquist`` the row
    ``ky = H/2`` and the column ``kx = W/2`` of the spectrum are also zero, so
    that any sub-pixel translation of the image stays exactly band-limited.
    """
    white = rng.standard_normal((H, W))
    F = np.fft.fft2(white)
    fy, fx = _freq_grid(H, W)
    r = np.sqrt(fx * fx + fy * fy)
    r[0, 0] = 1.0
    F = F / r**power
    F[0, 0] = 0.0
    if zero_nyquist:
        if H % 2 == 0:
            F[H // 2, :] = 0.0
        if W % 2 == 0:
            F[:, W // 2] = 0.0
    img = np.real(np.fft.ifft2(F))
    img -= img.min()
    m = img.max()
    if m > 0:
        img /= m
    return img


def _translate_fourier(img_stack: np.ndarray, sy: float, sx: float) -> np.ndarray:
    """Exact periodic translation ``out(y, x) = img(y + sy, x + sx)`` of band-limited images."""
    H, W = img_stack.shape[-2:]
    fy, fx = _freq_grid(H, W)
    F = np.fft.fft2(img_stack, axes=(-2, -1))
    F = F * np.exp(2j * np.pi * (fy * sy + fx * sx))
    return np.real(np.fft.ifft2(F, axes=(-2, -1)))


def layered_scene(seed: int, H: int, W: int, C: int, u: np.ndarray, d: np.ndarray,
                  sigma: float = 0.0, zero_nyquist: bool = True):
    """Views synthesised exactly from N layers (the non-occluded scene model of Sec. IV-A).

    Each of the ``N = len(d)`` layers is 1/f noise scaled to ``[0, 1/N]`` (so a
    view, the sum of N translated layers, stays near ``[0, 1]``); view ``j`` is
    ``sum_k layer_k(x + u_j d_k)`` plus i.i.d. Gaussian noise of std ``sigma``.

    Returns ``(views, layers)``: views float32 ``[K][C][H][W]`` and the
    central-view layers float64 ``[N][C][H][W]`` (the ground truth).
    """
    rng = np.random.default_rng(seed)
    N = len(d)
    K = len(u)
    layers = np.empty((N, C, H, W))
    for k in range(N):
        for c in range(C):
            layers[k, c] = noise_1f(rng, H, W, zero_nyquist=zero_nyquist) / N
    views = np.zeros((K, C, H, W))
    for j in range(K):
        for k in range(N):
            views[j] += _translate_fourier(layers[k], float(u[j, 1]) * float(d[k]),
                                           float(u[j, 0]) * float(d[k]))
    if sigma > 0:
        views += rng.normal(0.0, sigma, size=views.shape)
    return views.astype(np.float32), layers


def _bilinear_translate(stack: np.ndarray, sy: float, sx: float) -> np.ndarray:
    """``out(y, x) = img(y + sy, x + sx)`` by bilinear interpolation with wrap-around."""
    y0 = int(np.floor(sy))
    x0 = int(np.floor(sx))
    fy = sy - y0
    fx = sx - x0
    a = np.roll(stack, (-y0, -x0), axis=(-2, -1))
    b = np.roll(a, -1, axis=-1)
    c = np.roll(a, -1, axis=-2)
    e = np.roll(c, -1, axis=-1)
    return (1 - fy) * ((1 - fx) * a + fx * b) + fy * ((1 - fx) * c + fx * e)


def occluding_planes(seed: int, H: int, W: int, C: int, u: np.ndarray, n_planes: int = 5,
                     drange: float = 2.5):
    """Fronto-parallel occluding planes, composited back to front in every view.

    Plane ``p`` has a 1/f texture per channel, a disparity drawn from
    ``U(-drange, drange)`` and a binary alpha mask (thresholded smooth 1/f^2
    noise); the farthest plane (smallest disparity: ``d = (z0 - z) / z``,
    Sec. III) is opaque.  In view ``j`` each plane is moved by bilinear
    sub-pixel translation, ``plane(x + u_j d_p)``, then alpha-composited in
    ascending ``d``.

    Returns ``(views, plane_disparities)``; views float32 ``[K][C][H][W]``.
    """
    rng = np.random.default_rng(seed)
    dp = np.sort(rng.uniform(-drange, drange, n_planes))
    planes = []
    for p in range(n_planes):
        st = np.empty((C + 1, H, W))
        for c in range(C):
            st[c] = noise_1f(rng, H, W)
        if p == 0:
            st[C] = 1.0
        else:
            st[C] = (noise_1f(rng, H, W, power=2.0) > 0.5).astype(np.float64)
        planes.append(st)
    K = len(u)
    views = np.empty((K, C, H, W), np.float32)
    for j in range(K):
        acc = np.zeros((C, H, W))
        for p in range(n_planes):
            sh = _bilinear_translate(planes[p], float(u[j, 1]) * dp[p], float(u[j, 0]) * dp[p])
            a = sh[C]
            acc = a * sh[:C] + (1.0 - a) * acc
        views[j] = acc.astype(np.float32)
    return views, dp


def random_layer_spectra(seed: int, N: int, C: int, H: int, W: int) -> np.ndarray:
    """Half spectra (``[N][C][H][W//2+1]`` complex64) of 1/f-noise layers scaled to ``[0, 1/N]``.

    Used as render inputs; computed with numpy's real FFT (input generation only).
    """
    rng = np.random.default_rng(seed)
    out = np.empty((N, C, H, W // 2 + 1), np.complex64)
    for k in range(N):
        for c in range(C):
            out[k, c] = np.fft.rfft2(noise_1f(rng, H, W) / N).astype(np.complex64)
    return out
