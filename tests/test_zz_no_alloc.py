"""The fixed-scratch fit entry point, for callers that may not allocate device memory.

fdl_fit_spectra_noalloc keeps its scratch in an array inside the library instead of a
caller workspace.  This test calls it through the C ABI twice in a row, on two different
light fields, and checks each result against fdl_fit_spectra (which uses a workspace)
within the layer tolerance of the other fit tests.  The file is named so that pytest
collects it last.
"""

import ctypes as ct

import numpy as np
import pytest
import torch

from scenes import occluding_planes, view_grid

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _ptr(t):
    return ct.c_void_p(t.data_ptr())


def test_noalloc_fit_matches_workspace_fit_twice(fdl):
    from paper_1901_06919_gb300 import _lib as L

    lib = L.load()
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    # (views, disparities, image size, channels, seed): FP32 + double-float tiers (N <= 32), the
    # double-float-first path of N > 32, and an image at the size limit of the fixed scratch
    # (1024 x 1024: 525,312 stored frequencies)
    cases = [(view_grid(4), np.linspace(-3, 3, 30), 64, 3, 11), (view_grid(2), np.linspace(-2, 2, 12), 128, 1, 12),
             (view_grid(2), np.linspace(-3, 3, 40), 64, 3, 13), (view_grid(1), np.linspace(-2, 2, 8), 1024, 1, 14)]
    for i, (u, d, size, C, seed) in enumerate(cases):
        views, _ = occluding_planes(seed, size, size, C, u)
        V = torch.from_numpy(views).cuda()
        U = torch.from_numpy(u).cuda()
        D = torch.from_numpy(d.astype(np.float32)).cuda()
        S = fdl.rfft2(V)
        K, N = u.shape[0], d.size
        opts = L.FitOpts(1e-2, 1e-4, L.REG["view2"], L.PREC["mixed"], 0.0, 0.0)
        ref, _ = fdl.fit_spectra(S, U, D, 1e-2, 1e-4)
        out = torch.full_like(ref, float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = lib.fdl_fit_spectra_noalloc(_ptr(S), K, C, size, size, _ptr(U), _ptr(D), N, ct.byref(opts), _ptr(out),
                                         stream)
        assert st == L.FDL_OK, L.status_name(st)
        torch.cuda.synchronize()
        if i > 0:  # after the first call (which finds the array's address): no device memory taken
            assert torch.cuda.mem_get_info()[0] == free_before
        err = (torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref)).item()
        assert err < TOL, (size, d.size, err)


def test_noalloc_rejects_frequencies_beyond_its_scratch(fdl):
    from paper_1901_06919_gb300 import _lib as L

    lib = L.load()
    p = ct.c_void_p(0x1000)  # never used: the size check fails first
    opts = L.FitOpts(1e-2, 1e-4, 0, 0, 0.0, 0.0)
    st = lib.fdl_fit_spectra_noalloc(p, 9, 1, 2048, 1024, p, p, 8, ct.byref(opts), p, None)
    assert st == L.FDL_ENOMEM
