"""The host pipeline (fdl_fit_render_host on two streams and two device slots) returns, for
every submission, what the step-by-step calls return for the same light field."""

import numpy as np
import pytest
import torch

from scenes import occluding_planes, view_grid

pytestmark = pytest.mark.gpu


def test_pipeline_matches_sequential_calls(fdl):
    from paper_1901_06919_gb300.pipeline import FitRenderPipeline

    K, C, H, W, N = 9, 3, 32, 48, 8
    u = torch.from_numpy(view_grid(1))
    d = torch.linspace(-2, 2, N)
    u0 = torch.tensor([[0.5, -0.25], [-1.0, 1.0], [0.0, 0.0]])
    refocus = [((0.25, 0.0), 0.7, "disc", 1.2), ((-0.5, 0.5), -0.4, "square", 0.8)]
    pipe = FitRenderPipeline(K, C, H, W, u, d, 1e-2, u0=u0, refocus=refocus)
    scenes = [occluding_planes(s, H, W, C, view_grid(1))[0] for s in range(5)]
    ins = [torch.from_numpy(v).pin_memory() for v in scenes]
    outs = [torch.empty((3 + 2, C, H, W)).pin_memory() for _ in scenes]
    tickets = [pipe.submit(i, o) for i, o in zip(ins, outs)]
    pipe.wait(tickets[1])
    pipe.wait()
    for v, o in zip(scenes, outs):
        x, _ = fdl.fit(torch.from_numpy(v).cuda(), u.cuda(), d.cuda(), 1e-2)
        ref = [fdl.render(x, d.cuda(), u0.cuda())]
        specs = [fdl.RenderSpec(x, d.cuda(), r[0], r[1], r[2], r[3]) for r in refocus]
        ref.append(torch.stack(fdl.refocus_specs(specs)))
        ref = torch.cat(ref).cpu()
        # one refocus launch over all the images sums the layers in its own order
        assert torch.max(torch.abs(o - ref)).item() < 1e-5


def test_pipeline_rejects_wrong_shapes(fdl):
    from paper_1901_06919_gb300.pipeline import FitRenderPipeline

    pipe = FitRenderPipeline(9, 1, 16, 16, torch.from_numpy(view_grid(1)), torch.linspace(-1, 1, 4), 1e-2,
                             u0=torch.zeros((1, 2)))
    with pytest.raises(ValueError):
        pipe.submit(torch.zeros((9, 1, 16, 17)), torch.zeros((1, 1, 16, 16)))
    with pytest.raises(ValueError):
        pipe.submit(torch.zeros((9, 1, 16, 16)), torch.zeros((2, 1, 16, 16)))
