"""Continuous batching on the GPU: every result rendered in the mix (mixed FDLs, image sizes,
viewpoints, apertures, arrivals while other batches run) equals the same request rendered
alone, within the render tolerance 1e-4."""

import numpy as np
import pytest
import torch

from oracle import fdl_oracle as O
from scenes import occluding_planes, view_grid

pytestmark = pytest.mark.gpu


def test_results_are_the_same_alone_and_in_the_mix(fdl):
    from paper_1901_06919_gb300.serve import FdlStore, Request, Server

    dev = torch.device("cuda")
    store = FdlStore(budget_bytes=1 << 30, device=dev)
    specs = [(0, 64, 8), (1, 64, 12), (2, 128, 16)]  # (fid, size, N)
    u = view_grid(1)
    for fid, n, N in specs:
        views, _ = occluding_planes(10 + fid, n, n, 3, u)
        d = torch.linspace(-2, 2, N, device=dev)
        store.admit(fid, torch.from_numpy(views).to(dev), torch.from_numpy(u).to(dev), d, lam=1e-2)
    torch.cuda.synchronize()
    srv = Server(store, sizes=[(64, 64, 3), (128, 128, 3)], Nmax=16, capacity=8, pool=64)
    rng = np.random.default_rng(0)
    trace = []
    for i in range(60):
        fid = int(rng.integers(0, 3))
        kind = ["pinhole", "disc", "square"][i % 3]
        trace.append(Request(i, fid, tuple(rng.uniform(-4, 4, 2)), float(rng.uniform(-3, 3)), kind,
                             0.0 if kind == "pinhole" else float(rng.uniform(0, 3)),
                             t_arrival=float(i // 10) * 1e-3))  # bursts of ten every millisecond
    stats = srv.run_trace(trace, keep_outputs=True)
    assert stats["requests"] == 60 and all(r.t_done is not None for r in trace)
    assert stats["mean_batch"] > 1.0  # requests really were batched together
    # one graph serves every size: some launch rendered 64 x 64 and 128 x 128 images together
    sizes_of = {}
    for r in trace:
        sizes_of.setdefault(r.batch_id, set()).add(store.entries[r.fid].H)
    assert any(len(v) > 1 for v in sizes_of.values())
    assert fdl.sync_status(srv.batches[0].ws) == 0
    for r in trace:
        e = store.entries[r.fid]
        alone = fdl.refocus_specs([fdl.RenderSpec(e.layers, e.d, r.u0, r.s, r.aperture, r.radius)])[0]
        assert torch.max(torch.abs(alone - r.out)).item() <= 1e-4
    # and a few against the oracle
    kinds = {"pinhole": O.AP_PINHOLE, "disc": O.AP_DISC, "square": O.AP_SQUARE}
    for r in trace[:6]:
        e = store.entries[r.fid]
        ref = O.render(e.layers.cpu().numpy().astype(np.complex128), e.d.cpu().numpy().astype(np.float64),
                       r.u0, r.s, kinds[r.aperture], r.radius)
        assert np.max(np.abs(r.out.cpu().numpy() - ref)) < 1e-4
