"""The mixed render path's request groups (runs of consecutive requests that read one FDL).

One fdl_refocus launch over FDLs of different sizes, channel counts and layer counts, with
runs of 1, 2, 3, 8, 9 and 17 requests (groups under 8 give a warp 32 frequencies of a
256-frequency tile for all their requests; from 8 on the layer values are staged in shared
memory and the warps take the requests, two at a time for pinholes and discs), the same FDL
again after a run of another one, a rejected request in the middle of a run (it splits the
run), and apertures of every kind in one run.  Every image is compared with the FP64
oracle's render of its own FDL (max abs 1e-4, the pixel tolerance of the render tests).
"""

import numpy as np
import pytest
import torch

from oracle import fdl_oracle as O
from scenes import random_layer_spectra

pytestmark = pytest.mark.gpu

TOL = 1e-4
KINDS = {"pinhole": O.AP_PINHOLE, "disc": O.AP_DISC, "square": O.AP_SQUARE}


def _oracle(X, d, sp):
    return O.render(X.astype(np.complex128), d.astype(np.float64), sp.u0, sp.s, KINDS[sp.aperture], sp.radius)


def test_runs_of_every_length_in_one_launch(fdl):
    from paper_1901_06919_gb300 import _lib as L

    # (seed, N, C, H, W)
    fdls = [(21, 6, 3, 32, 32), (22, 9, 1, 64, 32), (23, 4, 2, 16, 64), (24, 12, 3, 64, 64)]
    data = []
    for seed, N, C, H, W in fdls:
        X = random_layer_spectra(seed, N, C, H, W)
        d = np.linspace(-2, 2, N).astype(np.float32)
        data.append((X, d, torch.from_numpy(X).cuda(), torch.from_numpy(d).cuda()))
    runs = [(0, 1), (1, 2), (2, 3), (3, 8), (0, 9), (1, 17), (3, 1), (2, 2)]
    rng = np.random.default_rng(11)
    specs, owner = [], []
    for f, n in runs:
        X, d, Xd, dd = data[f]
        for i in range(n):
            kind = ["pinhole", "disc", "square", "disc", "pinhole"][(i * 7 + f) % 5]
            sp = fdl.RenderSpec(Xd, dd, tuple(rng.uniform(-3, 3, 2)), float(rng.uniform(-2, 2)), kind,
                                0.0 if kind == "pinhole" else float(rng.uniform(0.3, 2.0)))
            sp.out = torch.full(X.shape[1:3] + ((X.shape[3] - 1) * 2,), -5.0, device="cuda")
            specs.append(sp)
            owner.append(f)
    # a request with N beyond the launch's Nmax in the middle of the 9-request run of FDL 0
    bad = fdl.RenderSpec(data[3][2], data[3][3], (0.5, 0.5))
    bad.out = torch.full((3, 64, 64), -5.0, device="cuda")
    mid = sum(n for _, n in runs[:4]) + 4
    specs.insert(mid, bad)
    owner.insert(mid, -1)
    req = fdl.pack_requests(specs, "cuda")
    ws = fdl.refocus(req, len(specs), 3, 64, 64, 11)  # Nmax 11 < 12: FDL 3's requests are rejected
    assert fdl.sync_status(ws) & L.ST_BAD_REQUEST
    for sp, f in zip(specs, owner):
        if f < 0 or data[f][0].shape[0] > 11:
            assert torch.all(sp.out == -5.0)  # skipped, untouched
            continue
        got = sp.out.cpu().numpy()
        assert np.max(np.abs(got - _oracle(data[f][0], data[f][1], sp))) < TOL


def test_interleaved_and_sorted_orders_agree(fdl):
    """The same requests with the FDLs interleaved (every request its own group) and sorted
    (one group per FDL) give the same images up to FP32 summation order."""
    fdls = [random_layer_spectra(31 + i, n, 3, 16 << i, 16 << i) for i, n in enumerate((5, 8, 3))]
    dev = [(torch.from_numpy(X).cuda(), torch.linspace(-1.5, 1.5, X.shape[0], device="cuda")) for X in fdls]
    rng = np.random.default_rng(5)
    base = []
    for i in range(18):
        Xd, dd = dev[i % 3]
        kind = ["pinhole", "disc", "square"][(i // 3) % 3]
        base.append((i % 3, tuple(rng.uniform(-2, 2, 2)), float(rng.uniform(-1, 1)), kind,
                     0.0 if kind == "pinhole" else float(rng.uniform(0.3, 1.5))))

    def render(order):
        specs = [fdl.RenderSpec(dev[b[0]][0], dev[b[0]][1], b[1], b[2], b[3], b[4]) for b in order]
        return [t.cpu().numpy() for t in fdl.refocus_specs(specs)]

    a = render(base)
    order = sorted(range(len(base)), key=lambda i: base[i][0])
    b = render([base[i] for i in order])
    for j, i in enumerate(order):
        assert np.max(np.abs(a[i] - b[j])) < 1e-5
