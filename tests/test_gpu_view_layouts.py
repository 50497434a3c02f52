"""Layer construction (Sec. V-A, Eq. LayerConstructionClosedForm) for the view layouts that
pick different ways of forming A in the solvers, against the FP64 oracle.

* Views on the integer lattice |u_x|, |u_y| <= 4 (full grids and scattered subsets, with
  negative coordinates): A_jk comes from per-frequency powers P_k^{u_x} Q_k^{u_y}.
* Jittered grids (the calibration workload's positions) and lattices reaching past 4: A_jk
  from the phase d_k (u_j . w) of every view, with the moment-form Gram.
* N = 8 (the smallest FP32 instance, which keeps the phase path) next to N = 16 and N = 30.

Tolerance: layer relative L2 <= 1e-5 of the oracle for the certified paths.
"""

import numpy as np
import pytest
import torch

from oracle import fdl_oracle as O
from scenes import jittered_grid, occluding_planes, view_grid

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _fit(fdl, views, u, d, lam, precision):
    x, ws = fdl.fit(torch.from_numpy(views).cuda(), torch.from_numpy(np.asarray(u, np.float32)).cuda(),
                    torch.from_numpy(np.asarray(d, np.float32)).cuda(), lam, 1e-4, precision=precision)
    torch.cuda.synchronize()
    assert ws.status() == 0
    return x.cpu().numpy(), ws.tier_counts()


def _check(fdl, u, N, lam=1e-2, size=(48, 64), C=1, seed=3):
    d = np.linspace(-3, 3, N).astype(np.float32)
    views, _ = occluding_planes(seed, size[0], size[1], C, u)
    ref = O.fit(views, u, d.astype(np.float64), lam=lam, eps=1e-4)
    out = {}
    for precision in ("mixed", "df"):
        got, counts = _fit(fdl, views, u, d, lam, precision)
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        assert err < TOL, (precision, err)
        assert counts["fp32"] + counts["df"] + counts["fp64"] == size[0] * (size[1] // 2 + 1)
        out[precision] = counts
    return out


def _lattice_subset(n, seed):
    rng = np.random.default_rng(seed)
    pts = view_grid(4)
    return pts[np.sort(rng.choice(len(pts), n, replace=False))]


@pytest.mark.parametrize("N", [8, 16, 30])
def test_lattice_subsets(fdl, N):
    u = _lattice_subset(40, N)
    assert np.all(u == np.rint(u)) and np.abs(u).max() == 4
    counts = _check(fdl, u, N)
    assert counts["mixed"]["fp32"] > 0


@pytest.mark.parametrize("g", [1, 4])
def test_full_lattice_grids_rgb(fdl, g):
    _check(fdl, view_grid(g), 30, C=3, size=(32, 32))


@pytest.mark.parametrize("N", [8, 30])
def test_jittered_grid_takes_the_phase_path(fdl, N):
    u = jittered_grid(4, 0.15, np.random.default_rng(7)).astype(np.float32)
    _check(fdl, u, N)


def test_lattice_past_four_takes_the_phase_path(fdl):
    u = np.concatenate([view_grid(2), np.array([[5.0, 0.0], [-5.0, 3.0]], np.float32)])
    _check(fdl, u, 24)


def test_lattice_and_phase_paths_agree(fdl):
    """The same scene with the views on the lattice and moved by 2^-20 (off the lattice): the
    two ways of forming A give layers that differ by no more than the moved views do in the
    FP64 oracle."""
    u = view_grid(3)
    d = np.linspace(-3, 3, 30).astype(np.float32)
    views, _ = occluding_planes(9, 48, 48, 1, u)
    u2 = (u + np.float32(2.0 ** -20)).astype(np.float32)
    a, _ = _fit(fdl, views, u, d, 1e-2, "mixed")
    b, _ = _fit(fdl, views, u2, d, 1e-2, "mixed")
    ra = O.fit(views, u, d.astype(np.float64), lam=1e-2, eps=1e-4)
    rb = O.fit(views, u2.astype(np.float64), d.astype(np.float64), lam=1e-2, eps=1e-4)
    shift = np.linalg.norm(ra - rb) / np.linalg.norm(ra)
    assert np.linalg.norm(a - b) / np.linalg.norm(ra) < shift + 2 * TOL
