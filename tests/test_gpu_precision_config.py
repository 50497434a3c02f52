"""The precision workload at full size: 7 x 7 views, 1024 x 1024 RGB, N = 40 layers on
linspace(-4, 4), lambda in {1e-3, 1e-2, 1e-1} (occluding-plane scene).

Layers of the certified mixed path (FP32 / double-float / FP64 tiers) against the FP64 oracle,
element by element at 64 frequencies the oracle computes one by one: DC, the lowest rings
(where the systems are worst conditioned), the Nyquist row and column, and seeded random
bins; the oracle's inputs come from its own DFT of the same float32 views.  Tolerance: layer
relative L2 <= 1e-5 per lambda.  Views and refocused images rendered by the library from those
layers are compared with the oracle's render of the same layers: max abs <= 1e-4.
"""

import numpy as np
import pytest
import torch

from oracle import fdl_oracle as O
from scenes import occluding_planes, view_grid

pytestmark = pytest.mark.gpu

N_SIZE = 1024
TOL_LAYERS = 1e-5
TOL_PIX = 1e-4


def _bins(n, nrand=45, seed=5):
    low = [(0, 0), (0, 1), (1, 0), (1, 1), (n - 1, 1), (0, 2), (2, 0), (2, 1), (1, 2), (n - 1, 2), (n - 2, 1)]
    h = n // 2
    nyq = [(h, 0), (h, 1), (h, 100), (h, h), (0, h), (1, h), (300, h), (n - 1, h)]
    rng = np.random.default_rng(seed)
    rand = list(zip(rng.integers(0, n, nrand).tolist(), rng.integers(0, h + 1, nrand).tolist()))
    b = low + nyq + rand
    assert len(b) == 64
    return np.array([p[0] for p in b]), np.array([p[1] for p in b])


@pytest.fixture(scope="module")
def workload():
    u = view_grid(3)
    d = np.linspace(-4, 4, 40).astype(np.float32)
    views, _ = occluding_planes(7, N_SIZE, N_SIZE, 3, u)
    ky, kx = _bins(N_SIZE)
    # the oracle's DFT at the sampled bins, one view at a time
    b = np.stack([O.dft_at_bins(views[j].astype(np.float64), ky, kx) for j in range(views.shape[0])])  # [K][C][nb]
    return views, u, d, ky, kx, b


@pytest.mark.parametrize("lam", [1e-3, 1e-2, 1e-1])
def test_layers_and_renders_at_full_size(fdl, workload, lam):
    views, u, d, ky, kx, b = workload
    V = torch.from_numpy(views).cuda()
    x, ws = fdl.fit(V, torch.from_numpy(u).cuda(), torch.from_numpy(d).cuda(), lam)
    torch.cuda.synchronize()
    assert ws.status() == 0
    counts = ws.tier_counts()
    assert counts["fp32"] + counts["df"] + counts["fp64"] == N_SIZE * (N_SIZE // 2 + 1)
    ref = O.solve_bins(np.moveaxis(b, -1, 0), u, d.astype(np.float64), O.freq_y(N_SIZE)[ky], kx / N_SIZE, lam,
                       1e-4)  # [nb][N][C]
    got = np.moveaxis(x[:, :, torch.from_numpy(ky).cuda(), torch.from_numpy(kx).cuda()].cpu().numpy(), -1, 0)
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert err < TOL_LAYERS, err
    # renders from these layers: the library against the oracle's render of the same layers
    X64 = x.cpu().numpy().astype(np.complex128)
    d64 = d.astype(np.float64)
    Dd = torch.from_numpy(d).cuda()
    u0 = np.array([[0.0, 0.0], [2.5, -1.5]], np.float32)
    imgs = fdl.render(x, Dd, torch.from_numpy(u0).cuda()).cpu().numpy()
    for i in range(len(u0)):
        assert np.max(np.abs(imgs[i] - O.render(X64, d64, u0[i].astype(np.float64)))) < TOL_PIX
    specs = [fdl.RenderSpec(x, Dd, (0.5, 0.5), -1.0, "disc", 1.0), fdl.RenderSpec(x, Dd, (0.0, 0.0), 2.0, "square", 2.0)]
    foc = [t.cpu().numpy() for t in fdl.refocus_specs(specs)]
    assert np.max(np.abs(foc[0] - O.render(X64, d64, (0.5, 0.5), -1.0, O.AP_DISC, 1.0))) < TOL_PIX
    assert np.max(np.abs(foc[1] - O.render(X64, d64, (0.0, 0.0), 2.0, O.AP_SQUARE, 2.0))) < TOL_PIX
