"""Requests of different image sizes in one render launch, and the device status word.

* fdl_refocus takes requests of any power-of-two sizes (and channel counts) within its
  (C, H, W) bounds in one launch (the mixed path: grouped render, per-request inverse DFT); each image
  must match the FP64 oracle's render of its own FDL within the pixel tolerance 1e-4 and the
  same request rendered alone.
* Requests the kernels reject (they cannot be checked on the host: the descriptors live in
  device memory) are skipped, leave their output untouched and set FDL_ST_BAD_REQUEST.
* A fit with a non-finite input sets FDL_ST_NONFINITE; a fit whose last factorisation breaks
  down (lambda = 0 at the DC frequency, where A*A = K 1 1^T is singular) sets
  FDL_ST_BREAKDOWN and leaves zeros there.
"""

import numpy as np
import pytest
import torch

from oracle import fdl_oracle as O
from scenes import layered_scene, random_layer_spectra, view_grid

pytestmark = pytest.mark.gpu

TOL = 1e-4
KINDS = {"pinhole": O.AP_PINHOLE, "disc": O.AP_DISC, "square": O.AP_SQUARE}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _oracle(X, d, sp, W=None):
    return O.render(X.astype(np.complex128), d.astype(np.float64), sp.u0, sp.s, KINDS[sp.aperture], sp.radius, W=W)


def test_mixed_image_sizes_in_one_launch(fdl):
    from paper_1901_06919_gb300 import _lib as L

    # (seed, N, C, H, W): square and non-square power-of-two images, one and three channels
    fdls = [(5, 8, 3, 64, 64), (6, 12, 3, 128, 128), (7, 5, 1, 32, 64), (8, 3, 2, 16, 16), (9, 6, 3, 128, 32)]
    data = []
    for seed, N, C, H, W in fdls:
        X = random_layer_spectra(seed, N, C, H, W)
        d = np.linspace(-2, 2.5, N).astype(np.float32)
        data.append((X, d, _dev(X), _dev(d)))
    rng = np.random.default_rng(3)
    specs = []
    for i in range(14):
        f = i % len(fdls)
        kind = ["pinhole", "disc", "square"][i % 3]
        X, d, Xd, dd = data[f]
        sp = fdl.RenderSpec(Xd, dd, tuple(rng.uniform(-3, 3, 2)), float(rng.uniform(-2, 2)), kind,
                            0.0 if kind == "pinhole" else float(rng.uniform(0.2, 2.5)))
        sp.out = torch.full(X.shape[1:3] + ((X.shape[3] - 1) * 2,), -7.0, device="cuda")
        specs.append((f, sp))
    # a request whose N exceeds the launch's Nmax: rejected on the device
    bad = fdl.RenderSpec(data[1][2], data[1][3], (0.0, 0.0))
    bad.out = torch.full((3, 128, 128), -7.0, device="cuda")
    all_specs = [sp for _, sp in specs] + [bad]
    req = fdl.pack_requests(all_specs, "cuda")
    ws = fdl.refocus(req, len(all_specs), 3, 128, 128, 11)  # Nmax 11 < 12: FDL 1's requests are bad too
    status = fdl.sync_status(ws)
    assert status & L.ST_BAD_REQUEST
    for f, sp in specs:
        X, d = data[f][0], data[f][1]
        if X.shape[0] > 11:
            assert torch.all(sp.out == -7.0)  # skipped, untouched
            continue
        got = sp.out.cpu().numpy()
        assert np.max(np.abs(got - _oracle(X, d, sp))) < TOL
        alone = fdl.refocus_specs([fdl.RenderSpec(sp.layers, sp.d, sp.u0, sp.s, sp.aperture, sp.radius)])[0]
        assert torch.max(torch.abs(alone - sp.out)).item() <= TOL
    assert torch.all(bad.out == -7.0)
    # the same launch with every request valid reports nothing
    good = [sp for f, sp in specs if data[f][0].shape[0] <= 11]
    ws = fdl.refocus(fdl.pack_requests(good, "cuda"), len(good), 3, 128, 128, 11)
    assert fdl.sync_status(ws) == 0


@pytest.mark.parametrize("H,W", [(2048, 32), (16, 4096), (16, 16)])
def test_extreme_aspect_ratios(fdl, H, W):
    """The mixed path at its edges: one column per strip (H = 2048), a 128-column strip and a
    single strip per image, next to a small request in the same launch."""
    X = random_layer_spectra(11, 4, 1, H, W)
    d = np.linspace(-1, 1, 4).astype(np.float32)
    Xs = random_layer_spectra(12, 3, 1, 16, 32)
    ds = np.linspace(-1, 2, 3).astype(np.float32)
    specs = [fdl.RenderSpec(_dev(X), _dev(d), (0.7, -1.3), 0.4, "disc", 1.2),
             fdl.RenderSpec(_dev(Xs), _dev(ds), (-0.5, 0.25), 0.0, "square", 0.8),
             fdl.RenderSpec(_dev(X), _dev(d), (2.0, 1.0))]
    imgs = [t.cpu().numpy() for t in fdl.refocus_specs(specs)]
    assert np.max(np.abs(imgs[0] - _oracle(X, d, specs[0]))) < TOL
    assert np.max(np.abs(imgs[1] - _oracle(Xs, ds, specs[1]))) < TOL
    assert np.max(np.abs(imgs[2] - _oracle(X, d, specs[2]))) < TOL


def test_status_of_a_clean_fit_and_render_is_zero(fdl):
    u = view_grid(1)
    d = np.linspace(-2, 2, 8).astype(np.float32)
    views, _ = layered_scene(0, 32, 32, 1, u, d, sigma=1e-3)
    x, ws = fdl.fit(_dev(views), _dev(u), _dev(d), 1e-2)
    assert ws.status() == 0
    from paper_1901_06919_gb300 import _lib as L

    need = L.load().fdl_render_workspace_size(2, 1, 32, 32)
    rws = fdl.workspace(need, "cuda")
    fdl.render(x, _dev(d), _dev(np.zeros((2, 2), np.float32)), ws=rws)
    assert fdl.sync_status(rws) == 0


@pytest.mark.parametrize("precision", ["mixed", "df", "f64"])
def test_status_reports_nonfinite_input(fdl, precision):
    from paper_1901_06919_gb300 import _lib as L

    u = view_grid(1)
    d = np.linspace(-2, 2, 8).astype(np.float32)
    views, _ = layered_scene(1, 32, 32, 1, u, d, sigma=1e-3)
    views[4, 0, 5, 7] = np.nan
    x, ws = fdl.fit(_dev(views), _dev(u), _dev(d), 1e-2, precision=precision)
    st = ws.status()
    assert st & L.ST_NONFINITE
    assert ws.tier_counts()["nonfinite"] == 32 * 17  # one NaN pixel reaches every frequency


def test_status_reports_breakdown(fdl):
    """lambda = 0 and 2 x 2 views: at DC, A*A = 4 1 1^T, whose Cholesky meets an exactly zero
    pivot in every arithmetic (4 - 2 * 2 = 0); the frequency is left as zeros."""
    from paper_1901_06919_gb300 import _lib as L

    u = np.array([[0, 0], [1, 0], [0, 1], [1, 1]], np.float32)
    d = np.linspace(-1, 1, 6).astype(np.float32)
    views, _ = layered_scene(2, 16, 16, 1, u, d, sigma=1e-3)
    x, ws = fdl.fit(_dev(views), _dev(u), _dev(d), 0.0, reg="l2")
    assert ws.status() & L.ST_BREAKDOWN
    assert ws.tier_counts()["breakdown"] >= 1
    assert torch.all(x[:, :, 0, 0] == 0)
