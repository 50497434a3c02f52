"""Image sizes that are not powers of two (the paper's 625 x 434, 379 x 379, 1920 x 1080 light
fields, Sec. VII): DFTs, layer construction and rendering against the FP64 oracle.

Lengths whose prime factors are at most 31 use mixed-radix passes, other lengths (379, 2 x 223,
odd primes) Bluestein's convolution; both in double-float, so the bounds are those of the
power-of-two tests.
"""

import numpy as np
import pytest
import torch

from oracle import fdl_oracle as O
from scenes import layered_scene, occluding_planes, random_layer_spectra, view_grid

pytestmark = pytest.mark.gpu

# (H, W): odd and even widths, a prime (Bluestein), products of 2, 3, 5, 7, 31
SIZES = [(434, 625), (379, 379), (48, 80), (27, 45), (33, 21), (446, 96), (1080, 1920), (17, 4096)]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("H,W", SIZES)
def test_rfft2_matches_oracle(fdl, H, W):
    rng = np.random.default_rng(H * 7 + W)
    n = 1 if H * W > 1_000_000 else 3
    img = rng.random((n, H, W)).astype(np.float32)
    got = fdl.rfft2(_dev(img)).cpu().numpy()
    ref = np.fft.rfft2(img.astype(np.float64)) if H * W > 200_000 else O.half_spectrum(img.astype(np.float64))
    assert got.shape == ref.shape
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel < 6e-8, rel
    assert np.max(np.abs(got - ref)) < 1e-7 * np.linalg.norm(ref[0])


def test_rfft2_large_sizes_against_the_definition_at_sampled_bins(fdl):
    """The DFT by its definition (no FFT) at listed bins, for the two largest paper shapes."""
    rng = np.random.default_rng(3)
    for H, W in ((434, 625), (1080, 1920)):
        img = rng.random((1, H, W)).astype(np.float32)
        got = fdl.rfft2(_dev(img)).cpu().numpy()
        ky = np.concatenate([[0, 1, H // 2, H - 1], rng.integers(0, H, 12)])
        kx = np.concatenate([[0, W // 2, 1, W // 2 - 1], rng.integers(0, W // 2 + 1, 12)])
        ref = O.dft_at_bins(img.astype(np.float64), ky, kx)
        scale = np.linalg.norm(np.fft.rfft2(img[0].astype(np.float64)))
        assert np.max(np.abs(got[:, ky, kx] - ref)) < 1e-7 * scale


@pytest.mark.parametrize("H,W", SIZES)
def test_irfft2_matches_oracle(fdl, H, W):
    rng = np.random.default_rng(H * 11 + W)
    Wh = W // 2 + 1
    # not Hermitian-consistent on the self-conjugate columns on purpose
    S = (rng.standard_normal((1, H, Wh)) + 1j * rng.standard_normal((1, H, Wh))).astype(np.complex64)
    got = fdl.irfft2(_dev(S), W).cpu().numpy()
    ref = np.fft.irfft2(S.astype(np.complex128), s=(H, W)) if H * W > 200_000 else O.image_from_half(
        S.astype(np.complex128), W)
    scale = np.sqrt(np.mean(ref ** 2))
    assert np.max(np.abs(got - ref)) < 1e-5 * scale


@pytest.mark.parametrize("H,W", [(27, 45), (30, 42)])
def test_fit_odd_and_even_widths(fdl, H, W):
    u = view_grid(1)
    d = np.linspace(-2, 2, 8).astype(np.float32)
    views, _ = layered_scene(0, H, W, 2, u, d, sigma=1e-3)
    ref = O.fit(views, u, d.astype(np.float64), lam=1e-2, eps=1e-4)
    for precision in ("mixed", "df", "f64"):
        x, ws = fdl.fit(_dev(views), _dev(u), _dev(d), 1e-2, precision=precision)
        got = x.cpu().numpy()
        assert got.shape == ref.shape
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < 1e-5, (precision, err)
        t = ws.tier_counts()
        assert t["fp32"] + t["df"] + t["fp64"] == H * (W // 2 + 1)


def test_fit_paper_shape_sampled_bins(fdl):
    """9x9 views of 625 x 434 RGB, 30 layers (the Lytro light fields of Sec. VII): the layers at
    sampled frequencies against the oracle's solve of the definition-level DFT at those bins."""
    H, W = 434, 625
    u = view_grid(4)
    d = np.linspace(-3, 3, 30).astype(np.float32)
    views, _ = occluding_planes(5, H, W, 3, u)
    x, ws = fdl.fit(_dev(views), _dev(u), _dev(d), 1e-2)
    got = x.cpu().numpy()
    rng = np.random.default_rng(9)
    ky = np.concatenate([[0, 1, 0, 2, H - 1], rng.integers(0, H, 19)])
    kx = np.concatenate([[0, 0, 1, 3, W // 2], rng.integers(0, W // 2 + 1, 19)])
    b = O.dft_at_bins(views.astype(np.float64), ky, kx)  # [K][C][nb]
    wy = O.freq_y(H)[ky]
    wx = kx / W
    ref = O.solve_bins(np.moveaxis(b, -1, 0), u, d.astype(np.float64), wy, wx, 1e-2, 1e-4)  # [nb][N][C]
    g = np.moveaxis(got[:, :, ky, kx], -1, 0)
    err = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert err < 1e-5, err


@pytest.mark.parametrize("H,W", [(45, 27), (38, 50), (379, 379)])
def test_render_and_refocus(fdl, H, W):
    X = random_layer_spectra(1, 6, 3, H, W)
    d = np.linspace(-1.5, 1.5, 6).astype(np.float32)
    u0 = np.array([[0.5, -0.25], [-1.0, 2.0]], np.float32)
    imgs = fdl.render(_dev(X), _dev(d), _dev(u0), W=W).cpu().numpy()
    for b in range(2):
        ref = O.render(X.astype(np.complex128), d, u0[b], W=W)
        assert np.max(np.abs(imgs[b] - ref)) < 1e-4
    specs = [fdl.RenderSpec(_dev(X), _dev(d), (0.25, 0.5), 0.7, "disc", 1.2, W=W),
             fdl.RenderSpec(_dev(X), _dev(d), (-0.5, 0.0), -0.4, "square", 0.8, W=W)]
    outs = fdl.refocus_specs(specs)
    for sp, o in zip(specs, outs):
        kind = {"disc": O.AP_DISC, "square": O.AP_SQUARE}[sp.aperture]
        ref = O.render(X.astype(np.complex128), d, sp.u0, sp.s, kind, sp.radius, W=W)
        assert np.max(np.abs(o.cpu().numpy() - ref)) < 1e-4
