"""Pins of the oracle's DFTs against brute force, closed forms and invariants (Sec. V-A, VII)."""

import numpy as np
import pytest

from oracle import fdl_oracle as O


def naive_dft(x, inverse=False):
    n = len(x)
    k = np.arange(n)
    sgn = 1 if inverse else -1
    M = np.exp(sgn * 2j * np.pi * np.outer(k, k) / n)
    return M @ x


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64])
def test_radix2_matches_bruteforce_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for inv in (False, True):
        got = O.fft_radix2(x, inverse=inv)
        ref = naive_dft(x, inverse=inv)
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_radix2_matches_library_fft_large():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 1024)) + 1j * rng.standard_normal((3, 1024))
    assert np.allclose(O.fft_radix2(x), np.fft.fft(x), rtol=0, atol=1e-9)
    y = rng.standard_normal((256, 8))
    assert np.allclose(O.fft_radix2(y, axis=0), np.fft.fft(y, axis=0), rtol=0, atol=1e-10)


def test_radix2_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        O.fft_radix2(np.ones(12))


def test_dft_of_delta_and_cosine_closed_forms():
    H, W = 16, 32
    img = np.zeros((H, W))
    y0, x0 = 3, 5
    img[y0, x0] = 1.0
    X = O.dft2(img)
    ky = np.arange(H)[:, None]
    kx = np.arange(W)[None, :]
    assert np.allclose(X, np.exp(-2j * np.pi * (ky * y0 / H + kx * x0 / W)), atol=1e-13)
    # cos(2 pi (2y/H + 3x/W)) -> two spikes of height HW/2 at (2,3) and (-2,-3)
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    X = O.dft2(np.cos(2 * np.pi * (2 * yy / H + 3 * xx / W)))
    ref = np.zeros((H, W), complex)
    ref[2, 3] = H * W / 2
    ref[H - 2, W - 3] = H * W / 2
    assert np.allclose(X, ref, atol=1e-10)


def test_parseval_and_hermitian_symmetry():
    rng = np.random.default_rng(2)
    img = rng.random((32, 64))
    X = O.dft2(img)
    assert np.isclose(np.sum(img ** 2), np.sum(np.abs(X) ** 2) / img.size, rtol=1e-12)
    mir = X[(-np.arange(32)) % 32][:, (-np.arange(64)) % 64]
    assert np.allclose(X, np.conj(mir), atol=1e-10)


def test_half_spectrum_round_trip():
    rng = np.random.default_rng(3)
    img = rng.random((2, 16, 32))
    S = O.half_spectrum(img)
    assert S.shape == (2, 16, 17)
    assert np.allclose(S, np.fft.rfft2(img), atol=1e-11)
    assert np.allclose(O.image_from_half(S, 32), img, atol=1e-13)


def test_image_from_half_takes_real_part_of_completed_spectrum():
    # A spectrum that is not Hermitian-consistent on the kx = 0 and kx = W/2
    # columns: the image is Re(full inverse DFT) of the completion.
    rng = np.random.default_rng(4)
    H, W = 8, 16
    S = rng.standard_normal((H, W // 2 + 1)) + 1j * rng.standard_normal((H, W // 2 + 1))
    full = np.zeros((H, W), complex)
    for ky in range(H):
        for kx in range(W):
            if kx <= W // 2:
                full[ky, kx] = S[ky, kx]
            else:
                full[ky, kx] = np.conj(S[(-ky) % H, W - kx])
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    ref = np.zeros((H, W))
    for ky in range(H):
        for kx in range(W):
            ref += np.real(full[ky, kx] * np.exp(2j * np.pi * (ky * yy / H + kx * xx / W)))
    ref /= H * W
    assert np.allclose(O.image_from_half(S, W), ref, atol=1e-13)
    # the same image as numpy's C2R, which drops the imaginary parts it cannot use
    assert np.allclose(O.image_from_half(S, W), np.fft.irfft2(S, s=(H, W)), atol=1e-13)


def test_frequency_convention():
    assert np.allclose(O.freq_y(8), [0, 1 / 8, 2 / 8, 3 / 8, -4 / 8, -3 / 8, -2 / 8, -1 / 8])
    assert np.allclose(O.freq_x_half(8), [0, 1 / 8, 2 / 8, 3 / 8, 4 / 8])


def test_dft_at_bins_is_the_definition():
    rng = np.random.default_rng(5)
    img = rng.random((2, 16, 32))
    ky = np.array([0, 3, 8, 15])
    kx = np.array([0, 7, 16, 5])
    ref = np.fft.fft2(img)[:, ky, kx]
    assert np.allclose(O.dft_at_bins(img, ky, kx), ref, atol=1e-11)
    assert np.allclose(O.dft_at_bins(img, ky, kx), O.dft2(img)[:, ky, kx], atol=1e-11)


# ---- lengths that are not powers of two (the paper's 625 x 434, 379 x 379, 1920 x 1080)

@pytest.mark.parametrize("n", [3, 5, 6, 7, 12, 31, 60])
def test_direct_dft_matches_bruteforce(n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for inv in (False, True):
        got = O.dft_direct(x, inverse=inv)
        ref = naive_dft(x, inverse=inv)
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_direct_dft_matches_library_fft_on_paper_lengths():
    rng = np.random.default_rng(7)
    for n in (379, 434, 625):
        x = rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))
        assert np.allclose(O.dft_1d(x), np.fft.fft(x), rtol=0, atol=1e-9)
        assert np.allclose(O.dft_1d(x, inverse=True), np.fft.ifft(x) * n, rtol=0, atol=1e-9)


@pytest.mark.parametrize("shape", [(15, 21), (12, 20), (7, 16), (16, 9)])
def test_half_spectrum_and_image_for_any_size(shape):
    H, W = shape
    rng = np.random.default_rng(H * 100 + W)
    img = rng.random((2, H, W))
    S = O.half_spectrum(img)
    assert S.shape == (2, H, W // 2 + 1)
    assert np.allclose(S, np.fft.rfft2(img), atol=1e-11)
    assert np.allclose(O.image_from_half(S, W), img, atol=1e-12)
    # a spectrum that is not Hermitian-consistent: numpy's C2R, which keeps the real
    # part of the completed inverse, gives the same image
    T = rng.standard_normal((H, W // 2 + 1)) + 1j * rng.standard_normal((H, W // 2 + 1))
    assert np.allclose(O.image_from_half(T, W), np.fft.irfft2(T, s=(H, W)), atol=1e-12)


def test_frequency_convention_odd_sizes():
    assert np.allclose(O.freq_y(5), [0, 1 / 5, 2 / 5, -2 / 5, -1 / 5])
    assert np.allclose(O.freq_x_half(5), [0, 1 / 5, 2 / 5])
    assert np.allclose(O.freq_y(6), np.fft.fftfreq(6))
