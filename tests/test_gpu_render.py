"""GPU rendering (Sec. VI-A, Eq. BsFourier + inverse DFT) against the FP64 oracle.

Tolerance (stated by the workload definition): rendered pixels within 1e-4 max abs on a [0, 1]
range.  Layer spectra come from the seeded scene generator, never from the GPU path.
"""

import numpy as np
import pytest
import torch

from oracle import fdl_oracle as O
from scenes import random_layer_spectra

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def fdl8():
    X = random_layer_spectra(0, 8, 3, 64, 64)
    d = np.linspace(-2, 2, 8).astype(np.float32)
    return X, d


def test_pinhole_views(fdl, fdl8):
    X, d = fdl8
    u0 = np.array([[0, 0], [1, -1], [-1, 1], [0.37, 0.81], [-4, 3.5], [2.2, -0.1]], np.float32)
    got = fdl.render(_dev(X), _dev(d), _dev(u0)).cpu().numpy()
    for b in range(len(u0)):
        ref = O.render(X.astype(np.complex128), d.astype(np.float64), u0[b].astype(np.float64))
        assert np.max(np.abs(got[b] - ref)) < TOL


@pytest.mark.parametrize("aperture,radius,s", [("disc", 1.0, -1.0), ("disc", 1.0, 0.0), ("disc", 1.0, 1.0),
                                               ("disc", 1.0, 2.0), ("square", 2.5, 0.7), ("disc", 3.0, -2.2),
                                               ("square", 0.4, 1.9)])
def test_refocus_apertures(fdl, fdl8, aperture, radius, s):
    X, d = fdl8
    u0 = (0.5, -0.25)
    spec = fdl.RenderSpec(_dev(X), _dev(d), u0, s, aperture, radius)
    img = fdl.refocus_specs([spec])[0].cpu().numpy()
    kind = {"disc": O.AP_DISC, "square": O.AP_SQUARE}[aperture]
    ref = O.render(X.astype(np.complex128), d.astype(np.float64), u0, s, kind, radius)
    assert np.max(np.abs(img - ref)) < TOL


def test_points_aperture_and_pinhole_radius_zero(fdl, fdl8):
    X, d = fdl8
    pts = np.array([[0, 0], [1, 0], [0, 1], [1, 1], [2, -1]], np.float32)
    sp = fdl.RenderSpec(_dev(X), _dev(d), (1.0, 0.0), 0.6, "points", 0.0, _dev(pts))
    img = fdl.refocus_specs([sp])[0].cpu().numpy()
    ref = O.render(X.astype(np.complex128), d.astype(np.float64), (1.0, 0.0), 0.6, O.AP_POINTS, 0.0, pts)
    assert np.max(np.abs(img - ref)) < TOL
    # psi = delta: any aperture of radius 0 is exactly the pinhole render
    specs = [fdl.RenderSpec(_dev(X), _dev(d), (0.3, 0.2), 1.1, a, 0.0) for a in ("pinhole", "disc", "square")]
    imgs = [t.cpu().numpy() for t in fdl.refocus_specs(specs)]
    assert np.array_equal(imgs[0], imgs[1]) and np.array_equal(imgs[0], imgs[2])


def test_mixed_fdls_in_one_call_and_batch_count(fdl):
    """Requests reading different FDLs (different N) in one launch; a device count limits the batch."""
    XA = random_layer_spectra(1, 5, 2, 32, 64)
    XB = random_layer_spectra(2, 12, 2, 32, 64)
    dA = np.linspace(-1, 1, 5).astype(np.float32)
    dB = np.linspace(-3, 2, 12).astype(np.float32)
    specs = [fdl.RenderSpec(_dev(XA), _dev(dA), (0.2, 0.1), 0.0, "pinhole", 0.0),
             fdl.RenderSpec(_dev(XB), _dev(dB), (-1.0, 0.5), 1.0, "disc", 1.5),
             fdl.RenderSpec(_dev(XA), _dev(dA), (0.0, 0.0), -0.5, "square", 1.0),
             fdl.RenderSpec(_dev(XB), _dev(dB), (2.0, 2.0), 0.0, "pinhole", 0.0)]
    for sp in specs:
        sp.out = torch.full((2, 32, 64), -7.0, device="cuda")
    req = fdl.pack_requests(specs, "cuda")
    count = torch.tensor([3], dtype=torch.int32, device="cuda")
    fdl.refocus(req, 4, 2, 32, 64, 12, count=count)
    torch.cuda.synchronize()
    kinds = {"pinhole": O.AP_PINHOLE, "disc": O.AP_DISC, "square": O.AP_SQUARE}
    for i, sp in enumerate(specs[:3]):
        X = XA if i % 2 == 0 else XB
        d = dA if i % 2 == 0 else dB
        ref = O.render(X.astype(np.complex128), d.astype(np.float64), sp.u0, sp.s, kinds[sp.aperture], sp.radius)
        assert np.max(np.abs(sp.out.cpu().numpy() - ref)) < TOL
    assert torch.all(specs[3].out == -7.0)  # beyond the count: untouched


def test_device_count_below_eight_on_one_fdl(fdl):
    """A launch for 8 requests of one FDL with 1, 2, 5 and 7 of them active (a device count, as
    in a captured serving batch): the tiled render stages the layer values for the active
    requests and leaves the rest untouched; pairs of views, of discs and lone squares."""
    X = random_layer_spectra(6, 10, 3, 32, 64)
    d = np.linspace(-2.5, 2, 10).astype(np.float32)
    Xd, dd = _dev(X), _dev(d)
    rng = np.random.default_rng(3)
    kinds = ["pinhole", "pinhole", "disc", "disc", "square", "pinhole", "disc", "square"]
    specs = [fdl.RenderSpec(Xd, dd, tuple(rng.uniform(-3, 3, 2)), float(rng.uniform(-2, 2)), k,
                            0.0 if k == "pinhole" else float(rng.uniform(0.3, 2.0))) for k in kinds]
    ap = {"pinhole": O.AP_PINHOLE, "disc": O.AP_DISC, "square": O.AP_SQUARE}
    refs = [O.render(X.astype(np.complex128), d.astype(np.float64), sp.u0, sp.s, ap[sp.aperture], sp.radius)
            for sp in specs]
    for n in (1, 2, 5, 7):
        for sp in specs:
            sp.out = torch.full((3, 32, 64), -7.0, device="cuda")
        req = fdl.pack_requests(specs, "cuda")
        count = torch.tensor([n], dtype=torch.int32, device="cuda")
        ws = fdl.refocus(req, 8, 3, 32, 64, 10, count=count)
        assert fdl.sync_status(ws) == 0
        for i, sp in enumerate(specs):
            if i < n:
                assert np.max(np.abs(sp.out.cpu().numpy() - refs[i])) < TOL
            else:
                assert torch.all(sp.out == -7.0)


def test_full_size_render(fdl):
    """512x512 RGB, 30 layers (the rendering side of the 9x9 workload), four views + four refocus."""
    X = random_layer_spectra(4, 30, 3, 512, 512)
    d = np.linspace(-3, 3, 30).astype(np.float32)
    Xd, dd = _dev(X), _dev(d)
    u0 = np.array([[0, 0], [4, -4], [-2.5, 1.25], [3.3, 0.1]], np.float32)
    views = fdl.render(Xd, dd, _dev(u0)).cpu().numpy()
    specs = [fdl.RenderSpec(Xd, dd, (0.0, 0.0), s, "disc", 1.0) for s in (-1.0, 0.0, 1.0, 2.0)]
    foc = [t.cpu().numpy() for t in fdl.refocus_specs(specs)]
    X64 = X.astype(np.complex128)
    d64 = d.astype(np.float64)
    for b in (0, 1, 3):
        ref = O.render(X64, d64, u0[b].astype(np.float64))
        assert np.max(np.abs(views[b] - ref)) < TOL
    for i, s in enumerate((-1.0, 2.0)):
        ref = O.render(X64, d64, (0.0, 0.0), s, O.AP_DISC, 1.0)
        assert np.max(np.abs(foc[0 if i == 0 else 3] - ref)) < TOL
