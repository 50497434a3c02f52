"""The double-float per-frequency solve (Sec. V-A, Eq. LayerConstructionClosedForm) at layer
and channel counts that do not fill its register slots: N below the compiled size (unused
slots of the factorisation), N across the one- and two-rows-per-lane boundary (N > 32), and
1, 2 or 4 channels (partly used right-hand-side slots), in the moment form (disparities on a
grid) and the direct form (irregular disparities); and more inputs per frequency than the
kernel stages.  Layers against the FP64 oracle within relative L2 1e-5.
"""

import numpy as np
import pytest
import torch

from oracle import fdl_oracle as O
from scenes import occluding_planes, view_grid

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("N,C", [(5, 2), (13, 4), (25, 1), (29, 3), (33, 2), (47, 4)])
@pytest.mark.parametrize("grid", [True, False])
def test_df_layer_and_channel_counts(fdl, N, C, grid):
    u = view_grid(2)
    rng = np.random.default_rng(N * 10 + C)
    if grid:
        d = np.linspace(-2.5, 2.5, N).astype(np.float32)
    else:
        d = np.sort(rng.uniform(-2.5, 2.5, N)).astype(np.float32)
    views, _ = occluding_planes(N + C, 24, 24, C, u)
    ref = O.fit(views, u, d.astype(np.float64), lam=1e-1, eps=1e-4)
    x, ws = fdl.fit(torch.from_numpy(views).cuda(), torch.from_numpy(u).cuda(), torch.from_numpy(d).cuda(),
                    1e-1, precision="df")
    got = x.cpu().numpy()
    assert got.shape == ref.shape
    assert _rel(got, ref) < TOL
    t = ws.tier_counts()
    assert t["df"] + t["fp64"] == 24 * 13 and t["breakdown"] == 0


@pytest.mark.parametrize("g,N,C", [(2, 6, 4), (3, 7, 3)])
def test_df_inputs_read_per_view(fdl, g, N, C):
    """More spectrum values per frequency (K x C) than the kernel's staging area holds for
    this layer count (N <= 8: 72 values): the view loop reads them from global memory."""
    u = view_grid(g)
    assert len(u) * C > 72
    d = np.linspace(-2.0, 2.0, N).astype(np.float32)
    views, _ = occluding_planes(N + 5 * C, 24, 24, C, u)
    ref = O.fit(views, u, d.astype(np.float64), lam=1e-1, eps=1e-4)
    x, _ = fdl.fit(torch.from_numpy(views).cuda(), torch.from_numpy(u).cuda(), torch.from_numpy(d).cuda(), 1e-1,
                   precision="df")
    assert _rel(x.cpu().numpy(), ref) < TOL
