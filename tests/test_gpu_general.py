"""The general system of Eq. AMatGeneral on the GPU against the FP64 oracle: free shifts (the
relaxed model: fit, render and the gradient dL/dP of Eq. gradP) and per-image apertures and
focus (focal stacks).

Tolerances: layers within relative L2 1e-5 (double-float) or 1e-7 (FP64; complex64 output) of the oracle;
pixels within 1e-4; the loss within 1e-5 and dL/dP within relative L2 1e-4 (as for the rank-1
calibration gradient).
"""

import numpy as np
import pytest
import torch

from oracle import fdl_oracle as O
from scenes import jittered_grid, layered_scene, occluding_planes, random_layer_spectra, view_grid

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def views_problem():
    u = view_grid(1)
    d = np.linspace(-2, 2, 6).astype(np.float32)
    views, _ = layered_scene(2, 24, 30, 2, u, d, sigma=1e-3)
    spec = np.fft.rfft2(views.astype(np.float64)).astype(np.complex64)
    return spec, u, d


@pytest.mark.parametrize("precision,tol", [("df", 1e-5), ("f64", 1e-7)])
def test_rank_one_shifts_match_the_sub_aperture_fit(fdl, views_problem, precision, tol):
    spec, u, d = views_problem
    P = (u[:, None, :] * d[None, :, None]).astype(np.float32)
    got = fdl.fit_general(_dev(spec), len(d), 1e-2, precision=precision, P=_dev(P), d=_dev(d)).cpu().numpy()
    ref = O.fit_spectra(spec.astype(np.complex128), u, d.astype(np.float64), 1e-2)
    assert _rel(got, ref) < tol
    got2 = fdl.fit_general(_dev(spec), len(d), 1e-2, precision=precision, u=_dev(u), d=_dev(d)).cpu().numpy()
    assert _rel(got2, ref) < tol


@pytest.mark.parametrize("precision,tol", [("df", 1e-5), ("f64", 1e-7)])
def test_free_shifts_fit(fdl, views_problem, precision, tol):
    spec, u, d = views_problem
    rng = np.random.default_rng(7)
    P = (u[:, None, :] * d[None, :, None] + rng.uniform(-0.3, 0.3, (len(u), len(d), 2))).astype(np.float32)
    got = fdl.fit_general(_dev(spec), len(d), 1e-2, precision=precision, reg="layer2", P=_dev(P)).cpu().numpy()
    ref = O.fit_spectra_general(spec.astype(np.complex128), P.astype(np.float64), 1e-2, reg=O.REG_LAYER2, W=30)
    assert _rel(got, ref) < tol


def test_focal_stack_fit(fdl):
    """Seven images focused at s in [-2.5, 2.5] through a disc of radius 1, plus two square-aperture
    images off-centre (a hybrid capture)."""
    H, W, N = 32, 32, 4
    X = random_layer_spectra(4, N, 1, H, W).astype(np.complex128)
    d = np.linspace(-1.5, 1.5, N).astype(np.float32)
    svals = np.linspace(-2.5, 2.5, 7)
    views = [("disc", 1.0, s) for s in svals] + [("square", 0.5, 0.3), ("square", 0.5, -0.8)]
    u = np.zeros((len(views), 2), np.float32)
    u[-2:] = [[1.0, 0.0], [0.0, -1.0]]
    kinds = {"disc": O.AP_DISC, "square": O.AP_SQUARE}
    B = np.stack([O.render_spectrum(X, d.astype(np.float64), tuple(u[j]), s, kinds[k], r)
                  for j, (k, r, s) in enumerate(views)]).astype(np.complex64)
    ov = [(kinds[k], r, s, None) for (k, r, s) in views]
    ref = O.fit_spectra_general(B.astype(np.complex128), O.shifts_of(u, d), 1e-3, reg=O.REG_L2,
                                d=d.astype(np.float64), views=ov)
    got = fdl.fit_general(_dev(B), N, 1e-3, reg="l2", precision="f64", u=_dev(u), d=_dev(d),
                          views=fdl.pack_views(views, "cuda")).cpu().numpy()
    assert _rel(got, ref) < 1e-7
    got_df = fdl.fit_general(_dev(B), N, 1e-3, reg="l2", precision="df", u=_dev(u), d=_dev(d),
                             views=fdl.pack_views(views, "cuda")).cpu().numpy()
    assert _rel(got_df, ref) < 1e-5


@pytest.mark.parametrize("H,W", [(32, 32), (27, 45)])
def test_render_with_shifts(fdl, H, W):
    X = random_layer_spectra(6, 5, 3, H, W)
    d = np.linspace(-1.5, 1.5, 5).astype(np.float32)
    rng = np.random.default_rng(8)
    P = rng.uniform(-2.0, 2.0, (3, 5, 2)).astype(np.float32)
    imgs = fdl.render_shifts(_dev(X), _dev(P), W=W).cpu().numpy()
    for b in range(3):
        ref = O.render_shifts(X.astype(np.complex128), P[b].astype(np.float64), W=W)
        assert np.max(np.abs(imgs[b] - ref)) < 1e-4
    # shifts u0 d^T render the view
    u0 = np.array([[0.4, -0.7]], np.float32)
    a = fdl.render_shifts(_dev(X), _dev((u0[:, None, :] * d[None, :, None]).astype(np.float32)), W=W)
    b_ = fdl.render(_dev(X), _dev(d), _dev(u0), W=W)
    assert torch.max(torch.abs(a - b_)).item() < 1e-5


def test_render_with_shifts_many_requests(fdl):
    """Nine requests on one FDL: the CTA stages the layers in shared memory once (the batched
    path) while every request brings its own per-layer shifts."""
    H, W = 32, 40
    X = random_layer_spectra(12, 6, 3, H, W)
    rng = np.random.default_rng(12)
    P = rng.uniform(-2.5, 2.5, (9, 6, 2)).astype(np.float32)
    imgs = fdl.render_shifts(_dev(X), _dev(P), W=W).cpu().numpy()
    for b in range(9):
        ref = O.render_shifts(X.astype(np.complex128), P[b].astype(np.float64), W=W)
        assert np.max(np.abs(imgs[b] - ref)) < 1e-4


@pytest.mark.parametrize("reg,precision", [("layer2", "df"), ("l2", "f64")])
def test_shift_gradient_matches_oracle(fdl, reg, precision):
    rng = np.random.default_rng(3)
    u_true = jittered_grid(1, 0.15, rng)
    H = W = 32
    views, _ = occluding_planes(5, H, W, 1, u_true, n_planes=3, drange=2.0)
    spec = np.ascontiguousarray(O.half_spectrum(views.astype(np.float64)).astype(np.complex64))
    d0 = np.linspace(-2, 2, 6)
    P = (np.asarray(view_grid(1), np.float64)[:, None, :] * d0[None, :, None]
         + rng.uniform(-0.2, 0.2, (9, 6, 2))).astype(np.float32)
    lam = 1e-1
    r = {"layer2": O.REG_LAYER2, "l2": O.REG_L2}[reg]
    nb = H * (W // 2 + 1)
    wy, wx = O.half_grid(H, W)
    bq = np.moveaxis(spec.astype(np.complex128).reshape(9, 1, -1), -1, 0)
    for bins in (np.arange(nb), rng.choice(nb, 80, replace=False)):
        loss, gP = fdl.calib_grad_shifts(_dev(spec), _dev(P), lam, reg=reg, precision=precision,
                                         bins=_dev(bins.astype(np.int32)))
        L_ref, g_ref = O.calib_loss_grad_shifts(bq[bins], wy[bins], wx[bins], P.astype(np.float64), lam, r)
        assert abs(loss.item() - L_ref) <= 1e-5 * abs(L_ref)
        assert np.linalg.norm(gP.cpu().numpy() - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def test_relaxed_calibration_lowers_the_loss_below_the_rank_one_model(fdl):
    """Views synthesised with shifts that are not rank one (u d^T plus a perturbation, a stand-in
    for non-Lambertian content): starting from the rank-1 shifts, the relaxed calibration of P
    (Adam on dL/dP, seeded 1024-frequency subsets) must reduce the loss well below its start."""
    from paper_1901_06919_gb300.calib import calibrate_shifts

    H = W = 32
    u = view_grid(1).astype(np.float64)
    d = np.linspace(-1.5, 1.5, 4)
    rng = np.random.default_rng(11)
    P_true = u[:, None, :] * d[None, :, None] + rng.uniform(-0.4, 0.4, (9, 4, 2))
    X = random_layer_spectra(9, 4, 1, H, W).astype(np.complex128)
    views = np.stack([O.render_shifts(X, P_true[j], W=W) for j in range(9)]).astype(np.float32)
    spec = np.ascontiguousarray(O.half_spectrum(views.astype(np.float64)).astype(np.complex64))
    P0 = (u[:, None, :] * d[None, :, None]).astype(np.float32)
    res = calibrate_shifts(_dev(spec), _dev(P0), lam=1e-3, steps=150, lr=2e-2, subset=256, seed=1, reg="l2")
    S = _dev(spec)
    full0 = fdl.calib_grad_shifts(S, _dev(P0), 1e-3, reg="l2")[0].item()
    full1 = fdl.calib_grad_shifts(S, res.P.contiguous(), 1e-3, reg="l2")[0].item()
    assert full1 < 0.2 * full0, (full0, full1)
