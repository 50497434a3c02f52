"""GPU layer construction (Sec. V-A) against the FP64 oracle on seeded synthetic light fields.

Tolerance (stated by the workload definition): layer spectra within relative L2 1e-5 of the
FP64 oracle, per lambda, on the same float32 views.
"""

import numpy as np
import pytest
import torch

from oracle import fdl_oracle as O
from scenes import layered_scene, occluding_planes, view_grid

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _gpu_fit(fdl, views, u, d, lam, eps=1e-4, reg="view2", precision="mixed"):
    V = torch.from_numpy(views).cuda()
    U = torch.from_numpy(np.asarray(u, np.float32)).cuda()
    D = torch.from_numpy(np.asarray(d, np.float32)).cuda()
    x, ws = fdl.fit(V, U, D, lam, eps, reg=reg, precision=precision)
    torch.cuda.synchronize()
    return x.cpu().numpy(), ws.tier_counts()


@pytest.fixture(scope="module")
def small_model_scene():
    """3x3 views, 64x64 gray, 8 layers on linspace(-2, 2): the small model-consistent workload."""
    u = view_grid(1)
    d = np.linspace(-2, 2, 8).astype(np.float32)
    views, _ = layered_scene(0, 64, 64, 1, u, d, sigma=1e-3)
    return views, u, d


@pytest.mark.parametrize("precision", ["mixed", "df", "f64"])
def test_small_scene_all_precisions(fdl, small_model_scene, precision):
    views, u, d = small_model_scene
    ref = O.fit(views, u, d.astype(np.float64), lam=1e-2, eps=1e-4)
    got, counts = _gpu_fit(fdl, views, u, d, 1e-2, precision=precision)
    err = rel_l2(got, ref)
    assert err < TOL, err
    nb = 64 * 33
    assert counts["fp32"] + counts["df"] + counts["fp64"] == nb
    assert counts["breakdown"] == 0 and counts["nonfinite"] == 0
    if precision == "df":
        # double-float everywhere, a few frequencies possibly re-solved in FP64 by its budget
        assert counts["fp32"] == 0 and counts["df"] + counts["fp64"] == nb
    if precision == "f64":
        assert counts["fp64"] == nb


@pytest.mark.parametrize("reg", ["layer2", "l2"])
def test_small_scene_other_regularisers(fdl, small_model_scene, reg):
    views, u, d = small_model_scene
    r = {"layer2": O.REG_LAYER2, "l2": O.REG_L2}[reg]
    ref = O.fit(views, u, d.astype(np.float64), lam=1e-1, eps=1e-4, reg=r)
    got, _ = _gpu_fit(fdl, views, u, d, 1e-1, reg=reg)
    err = rel_l2(got, ref)
    assert err < TOL, err


@pytest.fixture(scope="module")
def dense_grid_scene():
    """9x9 views at u in [-4, 4]^2, 64x64 RGB occluding planes, 30 layers on linspace(-3, 3)."""
    u = view_grid(4)
    d = np.linspace(-3, 3, 30).astype(np.float32)
    views, _ = occluding_planes(1, 64, 64, 3, u)
    return views, u, d


@pytest.mark.parametrize("precision", ["mixed", "df"])
def test_dense_grid_thirty_layers(fdl, dense_grid_scene, precision):
    views, u, d = dense_grid_scene
    ref = O.fit(views, u, d.astype(np.float64), lam=1e-2, eps=1e-4)
    got, counts = _gpu_fit(fdl, views, u, d, 1e-2, precision=precision)
    err = rel_l2(got, ref)
    assert err < TOL, err
    if precision == "mixed":
        # most frequencies of this geometry are ill conditioned: both tiers must be in use
        assert counts["fp32"] > 0 and counts["high_precision"] > 0


@pytest.mark.parametrize("lam", [1e-3, 1e-2, 1e-1])
def test_forty_layers_seven_by_seven(fdl, lam):
    """N = 40 > 32 (the wide-row path), 7x7 views, the lambda sweep of the precision workload."""
    u = view_grid(3)
    d = np.linspace(-4, 4, 40).astype(np.float32)
    views, _ = occluding_planes(2, 32, 32, 3, u)
    ref = O.fit(views, u, d.astype(np.float64), lam=lam, eps=1e-4)
    got, counts = _gpu_fit(fdl, views, u, d, lam)
    err = rel_l2(got, ref)
    assert err < TOL, err
    assert counts["breakdown"] == 0


def test_ragged_shapes_and_single_layer(fdl):
    """Non-square images, one view, one layer, one channel: the degenerate sizes."""
    rng = np.random.default_rng(5)
    views = rng.random((1, 1, 16, 64)).astype(np.float32)
    u = np.array([[0.3, -0.2]], np.float32)
    d = np.array([1.5], np.float32)
    ref = O.fit(views, u, d.astype(np.float64), lam=1e-2)
    got, _ = _gpu_fit(fdl, views, u, d, 1e-2)
    err = rel_l2(got, ref)
    assert err < TOL, err
    views = rng.random((4, 2, 128, 32)).astype(np.float32)
    u = rng.uniform(-1, 1, (4, 2)).astype(np.float32)
    d = np.linspace(-1, 1, 3).astype(np.float32)
    ref = O.fit(views, u, d.astype(np.float64), lam=1e-2)
    got, _ = _gpu_fit(fdl, views, u, d, 1e-2)
    err = rel_l2(got, ref)
    assert err < TOL, err


def test_fp32_only_mode_runs_everywhere(fdl, small_model_scene):
    views, u, d = small_model_scene
    got, counts = _gpu_fit(fdl, views, u, d, 1e-2, precision="f32")
    assert np.all(np.isfinite(got))
    # frequencies whose FP32 factorisation breaks down are left as zeros and counted
    assert counts["fp32"] + counts["breakdown"] == 64 * 33 and counts["high_precision"] == 0
    broken = np.all(got == 0, axis=(0, 1))
    assert broken.sum() == counts["breakdown"]


def test_fit_from_spectra_equals_fit_from_views(fdl, dense_grid_scene):
    views, u, d = dense_grid_scene
    V = torch.from_numpy(views).cuda()
    U = torch.from_numpy(u).cuda()
    D = torch.from_numpy(d).cuda()
    x1, _ = fdl.fit(V, U, D, 1e-2)
    x2, _ = fdl.fit_spectra(fdl.rfft2(V), U, D, 1e-2)
    torch.cuda.synchronize()
    a, b = x1.cpu().numpy(), x2.cpu().numpy()
    assert rel_l2(a, b) < 1e-6


def test_full_size_dense_grid_sampled_bins(fdl):
    """The 9x9, 512x512 RGB, 30-layer workload, fitted whole on the GPU; the oracle solves a
    sample of bins (low frequencies, where conditioning is worst, and random ones) from its own
    direct DFT of the same views."""
    u = view_grid(4)
    d = np.linspace(-3, 3, 30).astype(np.float32)
    views, _ = occluding_planes(3, 512, 512, 3, u)
    got, counts = _gpu_fit(fdl, views, u, d, 1e-2)
    rng = np.random.default_rng(9)
    ky = np.concatenate([[0, 0, 1, 2, 511, 3], rng.integers(0, 512, 26)])
    kx = np.concatenate([[0, 1, 0, 2, 1, 256], rng.integers(0, 257, 26)])
    b = O.dft_at_bins(views.astype(np.float64), ky, kx)  # [K][C][nb]
    wy = O.freq_y(512)[ky]
    wx = kx / 512.0
    x = O.solve_bins(np.moveaxis(b, -1, 0), u, d.astype(np.float64), wy, wx, 1e-2, 1e-4)  # [nb][N][C]
    ref = np.moveaxis(x, 0, -1)  # [N][C][nb]
    g = got[:, :, ky, kx]
    err = rel_l2(g, ref)
    assert err < TOL, err
    assert counts["fp32"] + counts["df"] + counts["fp64"] == 512 * 257
    assert counts["breakdown"] == 0


@pytest.mark.parametrize("precision", ["mixed", "df"])
def test_more_than_48_layers(fdl, precision):
    """N = 56: the double-float solve with the matrix in shared memory."""
    u = view_grid(2)
    d = np.linspace(-3, 3, 56).astype(np.float32)
    views, _ = occluding_planes(4, 32, 32, 2, u)
    ref = O.fit(views, u, d.astype(np.float64), lam=1e-1, eps=1e-4)
    got, counts = _gpu_fit(fdl, views, u, d, 1e-1, precision=precision)
    err = rel_l2(got, ref)
    assert err < TOL, err
    assert counts["breakdown"] == 0 and counts["high_precision"] == 32 * 17


@pytest.mark.parametrize("precision", ["mixed", "df", "f64"])
def test_many_views_wide_baseline(fdl, precision):
    """19x19 views spanning u in [-9, 9]: large phases d (u . w) and long sums over views.

    The sums over views of A*A and A*b at the low, worst-conditioned frequencies are where
    the double-float solve loses accuracy first (double-float alone, without its FP64 budget,
    lands near 3e-5 here); the error budgets of the mixed and double-float paths must hold
    against the FP64 oracle.
    """
    u = view_grid(9)
    d = np.linspace(-3, 3, 30).astype(np.float32)
    views, _ = occluding_planes(7, 64, 64, 1, u)
    ref = O.fit(views, u, d.astype(np.float64), lam=1e-2, eps=1e-4)
    got, counts = _gpu_fit(fdl, views, u, d, 1e-2, precision=precision)
    err = rel_l2(got, ref)
    assert err < TOL, err
    assert counts["fp32"] + counts["df"] + counts["fp64"] == 64 * 33


@pytest.mark.parametrize("precision", ["mixed", "df"])
def test_irregular_disparities_take_the_direct_gram(fdl, precision):
    """Disparities far from any grid (seeded, sorted uniform draws): the double-float solve
    must take its direct Gram form instead of the moment form and still meet the tolerance."""
    u = view_grid(3)
    d = np.sort(np.random.default_rng(4).uniform(-2.5, 2.5, 20)).astype(np.float32)
    views, _ = occluding_planes(2, 64, 64, 3, u)
    ref = O.fit(views, u, d.astype(np.float64), lam=1e-2, eps=1e-4)
    got, counts = _gpu_fit(fdl, views, u, d, 1e-2, precision=precision)
    err = rel_l2(got, ref)
    assert err < TOL, err
    assert counts["fp32"] + counts["df"] + counts["fp64"] == 64 * 33
