"""Calibration loop (Sec. V-B) on the GPU: autograd wiring, finite differences of the GPU
loss, and recovery of jittered view positions from a model-consistent light field."""

import numpy as np
import pytest
import torch

from oracle import fdl_oracle as O
from scenes import layered_scene, view_grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jittered_scene():
    rng = np.random.default_rng(0)
    u_true = view_grid(2).astype(np.float64) + rng.uniform(-0.15, 0.15, (25, 2))
    d_true = np.sort(rng.uniform(-2, 2, 12))
    views, _ = layered_scene(1, 32, 32, 1, u_true.astype(np.float32), d_true.astype(np.float32), sigma=0.0)
    spec = np.ascontiguousarray(O.half_spectrum(views.astype(np.float64)).astype(np.complex64))
    return spec, u_true, d_true


def gauge_error(u, u_true):
    """RMS position error after removing the translation and the scale u -> c u
    (P = u d^T and the loss do not change under either)."""
    a = u - u.mean(0)
    t = u_true - u_true.mean(0)
    c = (a * t).sum() / (a * a).sum()
    return float(np.sqrt(((c * a - t) ** 2).mean()))


def test_autograd_function_returns_kernel_gradient(fdl, jittered_scene):
    from paper_1901_06919_gb300.calib import calib_loss

    spec, _, _ = jittered_scene
    S = torch.from_numpy(spec).cuda()
    u = torch.from_numpy(view_grid(2)).cuda().requires_grad_(True)
    d = torch.linspace(-2, 2, 12, device="cuda").requires_grad_(True)
    loss = calib_loss(u, d, S, 1e-2)
    loss.backward()
    ref_loss, gu, gd = fdl.calib_grad(S, u.detach(), d.detach(), 1e-2)
    assert torch.equal(loss.detach(), ref_loss[0])
    assert torch.equal(u.grad, gu) and torch.equal(d.grad, gd)


def test_gradient_against_central_differences_of_gpu_loss(fdl, jittered_scene):
    """Step 1e-4 central differences of the GPU loss (float32 output) match the kernel gradient."""
    spec, _, _ = jittered_scene
    S = torch.from_numpy(spec).cuda()
    u = torch.from_numpy(view_grid(2)).cuda()
    d = torch.linspace(-2, 2, 12, device="cuda")
    _, gu, gd = fdl.calib_grad(S, u, d, 1e-2)
    h = 1e-4
    fd_d = []
    for k in range(12):
        dp = d.clone(); dp[k] += h
        dm = d.clone(); dm[k] -= h
        fd_d.append((fdl.calib_grad(S, u, dp, 1e-2)[0] - fdl.calib_grad(S, u, dm, 1e-2)[0]).item() / (2 * h))
    fd_u = []
    for j in (0, 7, 12, 24):
        for a in range(2):
            up = u.clone(); up[j, a] += h
            um = u.clone(); um[j, a] -= h
            fd_u.append((fdl.calib_grad(S, up, d, 1e-2)[0] - fdl.calib_grad(S, um, d, 1e-2)[0]).item() / (2 * h))
    g_u = gu.cpu().numpy()[[0, 7, 12, 24]].ravel()
    assert np.linalg.norm(np.array(fd_d) - gd.cpu().numpy()) < 2e-2 * np.linalg.norm(gd.cpu().numpy())
    assert np.linalg.norm(np.array(fd_u) - g_u) < 2e-2 * np.linalg.norm(g_u)


def test_adam_calibration_recovers_view_positions(fdl, jittered_scene):
    from paper_1901_06919_gb300.calib import calibrate

    spec, u_true, _ = jittered_scene
    S = torch.from_numpy(spec).cuda()
    u0 = torch.from_numpy(view_grid(2)).cuda()
    d0 = torch.linspace(-2, 2, 12, device="cuda")
    res = calibrate(S, u0, d0, lam=1e-2, steps=200, lr=1e-2, subset=None)
    e0 = gauge_error(view_grid(2).astype(np.float64), u_true)
    e1 = gauge_error(res.u.cpu().numpy().astype(np.float64), u_true)
    assert e1 < 0.05 * e0, (e0, e1)
    assert res.losses[-1] < 0.1 * res.losses[0]


def test_stochastic_subsets_and_paper_rule_run(fdl, jittered_scene):
    from paper_1901_06919_gb300.calib import calibrate

    spec, u_true, _ = jittered_scene
    S = torch.from_numpy(spec).cuda()
    u0 = torch.from_numpy(view_grid(2)).cuda()
    d0 = torch.linspace(-2, 2, 12, device="cuda")
    res = calibrate(S, u0, d0, steps=60, subset=256, seed=3)
    before = fdl.calib_grad(S, u0, d0, 1e-2)[0].item()
    after = fdl.calib_grad(S, res.u, res.d, 1e-2)[0].item()
    assert after < 0.5 * before
    res = calibrate(S, u0, d0, steps=10, rule="paper", alpha=0.2, subset=None)
    assert np.isfinite(res.losses[-1])
