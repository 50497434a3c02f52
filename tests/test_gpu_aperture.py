"""Drawn apertures (Sec. VI-A): the GPU table of a rasterised aperture and refocusing with it,
against the FP64 oracle's own table built from the same raster."""

import numpy as np
import pytest
import torch

from oracle import fdl_oracle as O
from scenes import random_layer_spectra

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _disc_raster(P, frac=0.8):
    c = (P - 1) / 2
    yy, xx = np.mgrid[0:P, 0:P]
    return ((xx - c) ** 2 + (yy - c) ** 2 <= (frac * c + 0.5) ** 2).astype(np.float32)


@pytest.mark.parametrize("P,Z", [(1, 32), (3, 64), (7, 48), (9, 250), (31, 256)])
def test_table_matches_oracle(fdl, P, Z):
    rng = np.random.default_rng(P * 100 + Z)
    R = rng.random((P, P)).astype(np.float32)  # asymmetric weights
    got = fdl.aperture_table(_dev(R), Z).cpu().numpy()
    ref = O.aperture_table(R.astype(np.float64), Z)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) < 1e-6
    assert abs(got[0, 0] - 1.0) < 1e-6


@pytest.mark.parametrize("H,W", [(64, 64), (45, 27)])
def test_refocus_with_a_drawn_aperture(fdl, H, W):
    X = random_layer_spectra(4, 6, 3, H, W)
    d = np.linspace(-1.5, 1.5, 6).astype(np.float32)
    R = _disc_raster(9)
    R[1, 4] = 0.0  # not symmetric: the table is complex
    h, Z = 0.25, 64
    T = fdl.aperture_table(_dev(R), Z)
    Tref = O.aperture_table(R.astype(np.float64), Z)
    specs = [fdl.RenderSpec(_dev(X), _dev(d), (0.3, -0.2), s, "table", h, T, W=W) for s in (-1.0, 0.4, 1.3)]
    specs.append(fdl.RenderSpec(_dev(X), _dev(d), (0.0, 0.5), 0.2, "disc", 0.8, W=W))  # mixed kinds in one call
    outs = fdl.refocus_specs(specs)
    for sp, o in zip(specs[:3], outs[:3]):
        ref = O.render(X.astype(np.complex128), d, sp.u0, sp.s, O.AP_TABLE, h, Tref, W=W)
        assert np.max(np.abs(o.cpu().numpy() - ref)) < 1e-4
    ref = O.render(X.astype(np.complex128), d, (0.0, 0.5), 0.2, O.AP_DISC, 0.8, W=W)
    assert np.max(np.abs(outs[3].cpu().numpy() - ref)) < 1e-4


def test_one_pixel_table_renders_as_the_pinhole(fdl):
    X = random_layer_spectra(5, 4, 1, 32, 32)
    d = np.linspace(-1, 1, 4).astype(np.float32)
    T = fdl.aperture_table(_dev(np.ones((1, 1), np.float32)), 32)
    a = fdl.refocus_specs([fdl.RenderSpec(_dev(X), _dev(d), (0.5, 0.25), 0.7, "table", 0.3, T)])[0]
    b = fdl.refocus_specs([fdl.RenderSpec(_dev(X), _dev(d), (0.5, 0.25), 0.7, "pinhole", 0.0)])[0]
    assert torch.max(torch.abs(a - b)).item() < 1e-6
