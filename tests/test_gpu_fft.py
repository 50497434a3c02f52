"""GPU 2D real DFTs against the oracle's textbook DFT (Sec. V-A, VI-A, VII)."""

import numpy as np
import pytest
import torch

from oracle import fdl_oracle as O

pytestmark = pytest.mark.gpu

SIZES = [(16, 16), (32, 64), (64, 16), (128, 256), (512, 512), (256, 1024), (2048, 64), (16, 4096), (1024, 1024)]


@pytest.mark.parametrize("H,W", SIZES)
def test_rfft2_matches_oracle(fdl, H, W):
    rng = np.random.default_rng(H * 7 + W)
    img = rng.random((3, H, W)).astype(np.float32)
    got = fdl.rfft2(torch.from_numpy(img).cuda()).cpu().numpy()
    ref = O.half_spectrum(img.astype(np.float64))
    assert got.shape == ref.shape
    # double-float passes: within about two roundings to complex64 of the exact DFT
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel < 6e-8, rel
    # every bin, against the scale of the whole spectrum
    assert np.max(np.abs(got - ref)) < 1e-7 * np.linalg.norm(ref[0])


@pytest.mark.parametrize("H,W", SIZES)
def test_irfft2_matches_oracle(fdl, H, W):
    rng = np.random.default_rng(H * 11 + W)
    # not Hermitian-consistent on the kx = 0 and kx = W/2 columns on purpose
    S = (rng.standard_normal((2, H, W // 2 + 1)) + 1j * rng.standard_normal((2, H, W // 2 + 1))).astype(np.complex64)
    got = fdl.irfft2(torch.from_numpy(S).cuda(), W).cpu().numpy()
    ref = O.image_from_half(S.astype(np.complex128), W)
    scale = np.sqrt(np.mean(ref ** 2))
    assert np.max(np.abs(got - ref)) < 1e-5 * scale


def test_round_trip_of_many_images(fdl):
    rng = np.random.default_rng(0)
    img = torch.from_numpy(rng.random((40, 64, 128)).astype(np.float32)).cuda()
    back = fdl.irfft2(fdl.rfft2(img), 128)
    assert torch.max(torch.abs(back - img)).item() < 1e-6
