"""The C-ABI library builds, loads and exports every symbol include/fdl.h declares; host-side
argument checks and workspace queries (no GPU needed: nothing here launches a kernel)."""

import ctypes as ct
import os
import re
import subprocess

import pytest

from paper_1901_06919_gb300 import _lib as L
from paper_1901_06919_gb300 import build as B

HEADER = os.path.join(B.ROOT, "include", "fdl.h")


def declared_symbols():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"FDL_API\s+[\w\s\*]+?\b(fdl_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for core in ("fdl_fit", "fdl_render", "fdl_refocus", "fdl_calib_grad"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fdl_\w+)", out))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    # and nothing beyond the header leaks out with C linkage
    assert exported == set(declared_symbols())
    # the binding covers the whole header
    assert set(L.exported_symbols()) == set(declared_symbols())


def test_status_strings(lib):
    assert lib.fdl_strerror(0) == b"ok"
    assert lib.fdl_strerror(2) == b"workspace too small"
    assert lib.fdl_version() >= 1


def test_workspace_queries(lib):
    assert lib.fdl_fit_workspace_size(81, 3, 512, 512, 30) > 81 * 3 * 512 * 256 * 8
    # the paper's sizes that are not powers of two: 625 x 434 (prime factors <= 31),
    # 379 x 379 (prime: Bluestein), 1920 x 1080
    assert lib.fdl_fit_workspace_size(81, 3, 434, 625, 30) >= 81 * 3 * 434 * 313 * 8
    assert lib.fdl_fit_workspace_size(49, 3, 379, 379, 30) > 0
    assert lib.fdl_rfft2_workspace_size(1, 1080, 1920) > 0
    assert lib.fdl_render_workspace_size(4, 3, 434, 625) >= 4 * 3 * 434 * 313 * 8
    # a prime above 2048 has no Bluestein length within 4096; sizes below 16 are refused
    assert lib.fdl_fit_workspace_size(9, 1, 64, 2053, 8) == 0
    assert lib.fdl_rfft2_workspace_size(4, 8, 64) == 0  # H below 16
    assert lib.fdl_irfft2_workspace_size(4, 64, 15) == 0  # W below 16
    assert lib.fdl_render_workspace_size(113, 3, 512, 512) >= 113 * 3 * 512 * 257 * 8
    assert lib.fdl_refocus_workspace_size(0, 3, 512, 512) == 0
    assert lib.fdl_calib_grad_workspace_size(25, 1, 256, 256, 12, 4096) > 0


def _opts(**kw):
    o = dict(lam=1e-2, eps=1e-4, reg=0, precision=0, kappa_max=0.0, df_error_budget=0.0, f32_error_budget=0.0)
    o.update(kw)
    return L.FitOpts(o["lam"], o["eps"], o["reg"], o["precision"], o["kappa_max"], o["df_error_budget"],
                     o["f32_error_budget"])


def test_fit_rejects_bad_arguments_before_any_launch(lib):
    p = ct.c_void_p(0x1000)  # never dereferenced: every call below fails validation first
    o = _opts()
    call = lambda K=9, C=1, H=64, W=64, N=8, opts=o, ws=1 << 30, views=p: lib.fdl_fit(
        views, K, C, H, W, p, p, N, ct.byref(opts) if opts is not None else None, p, p, ws, None)
    assert call(K=0) == L.FDL_EINVAL
    assert call(C=5) == L.FDL_EINVAL
    assert call(N=65) == L.FDL_EINVAL
    assert call(H=2053) == L.FDL_EINVAL  # prime above 2048: no supported DFT length
    assert call(W=8192) == L.FDL_EINVAL
    assert call(opts=None) == L.FDL_EINVAL
    assert call(opts=_opts(lam=-1.0)) == L.FDL_EINVAL
    assert call(opts=_opts(lam=float("nan"))) == L.FDL_EINVAL
    assert call(opts=_opts(reg=7)) == L.FDL_EINVAL
    assert call(opts=_opts(precision=9)) == L.FDL_EINVAL
    assert call(opts=_opts(precision=3), N=40) == L.FDL_ENOTSUP
    assert call(opts=_opts(df_error_budget=float("nan"))) == L.FDL_EINVAL
    assert call(opts=_opts(f32_error_budget=float("nan"))) == L.FDL_EINVAL
    assert call(views=ct.c_void_p(0)) == L.FDL_EINVAL
    assert call(ws=1024) == L.FDL_ENOMEM


def test_other_entry_points_reject_bad_arguments(lib):
    p = ct.c_void_p(0x1000)
    assert lib.fdl_rfft2(p, 1, 12, 64, p, p, 1 << 30, None) == L.FDL_EINVAL
    assert lib.fdl_rfft2(p, 1, 64, 64, p, p, 16, None) == L.FDL_ENOMEM
    assert lib.fdl_irfft2(p, 0, 64, 64, p, p, 1 << 30, None) == L.FDL_EINVAL
    assert lib.fdl_render(p, p, 8, 3, 64, 64, p, 0, p, p, 1 << 30, None) == L.FDL_EINVAL
    assert lib.fdl_render(p, p, 8, 3, 64, 64, p, 4, p, p, 64, None) == L.FDL_ENOMEM
    assert lib.fdl_refocus(p, 4, None, 3, 64, 64, 80, p, 1 << 30, None) == L.FDL_EINVAL
    o = _opts(reg=0)
    assert lib.fdl_calib_grad(p, 9, 1, 64, 64, p, p, 8, ct.byref(o), None, 0, p, p, p, p, 1 << 30,
                              None) == L.FDL_EINVAL  # view regulariser depends on d
    o = _opts(reg=1)
    assert lib.fdl_calib_grad(p, 9, 1, 64, 64, p, p, 8, ct.byref(o), p, 0, p, p, p, p, 1 << 30,
                              None) == L.FDL_EINVAL  # empty bin list


def test_request_struct_layout_matches_header(lib):
    # fdl_request: 4 pointers, 3 ints, 4 floats, the image size (3 ints), 2 ints of padding
    assert ct.sizeof(L.Request) == 80
    assert L.Request.u0x.offset == 44
    assert L.Request.H.offset == 60 and L.Request.C.offset == 68
    assert ct.sizeof(L.FitOpts) == 48


def test_host_buffer_step_rejects_bad_arguments(lib):
    p = ct.c_void_p(0x1000)
    o = _opts()
    assert lib.fdl_fit_render_host_workspace_size(9, 1, 64, 64, 8, 4) > 9 * 64 * 64 * 4
    call = lambda B=4, views=p, ws=1 << 40: lib.fdl_fit_render_host(views, 9, 1, 64, 64, p, p, 8, ct.byref(o), p, p, B,
                                                                   p, 10, p, p, ws, None)
    assert call(B=0) == L.FDL_EINVAL
    assert call(views=ct.c_void_p(0)) == L.FDL_EINVAL
    assert call(ws=64) == L.FDL_ENOMEM


def test_status_word_call_rejects_null(lib):
    v = ct.c_int(0)
    assert lib.fdl_sync_status(None, ct.byref(v), None) == L.FDL_EINVAL
    assert lib.fdl_sync_status(ct.c_void_p(0x1000), None, None) == L.FDL_EINVAL
