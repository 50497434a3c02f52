"""PyTorch binding of libfdl: tensors in, tensors out, every step in the CUDA library.

The functions only check dtypes/devices, allocate outputs and workspaces with
torch, and pass raw pointers and the current CUDA stream to the C ABI of
``include/fdl.h``.
"""

from __future__ import annotations

import ctypes as ct
from dataclasses import dataclass

import torch

from . import _lib as L


def _lib():
    return L.load()


def _stream(stream=None) -> ct.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ct.c_void_p(s.cuda_stream)


def _p(t: torch.Tensor | None) -> ct.c_void_p:
    return ct.c_void_p(t.data_ptr() if t is not None else None)


def _need(t: torch.Tensor, dtype, name: str, ndim: int | None = None) -> None:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dimensions")


def workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _opts(lam, eps, reg, precision, kappa_max, df_error_budget=0.0, f32_error_budget=0.0) -> L.FitOpts:
    return L.FitOpts(float(lam), float(eps), L.REG[reg], L.PREC[precision], float(kappa_max), float(df_error_budget),
                     float(f32_error_budget))


def _width(Wh: int, W: int | None) -> int:
    """Image width of a stored half of ``Wh`` columns: ``W`` if given (an odd width cannot be
    told from ``Wh``), else the even width ``2 (Wh - 1)``."""
    if W is None:
        return 2 * (Wh - 1)
    if W // 2 + 1 != Wh:
        raise ValueError(f"width {W} does not match a stored half of {Wh} columns")
    return int(W)


# ---------------------------------------------------------------- DFTs
def rfft2(images: torch.Tensor, stream=None) -> torch.Tensor:
    """Half spectra (complex64 ``[..., H, W//2+1]``) of float32 images ``[..., H, W]``."""
    _need(images, torch.float32, "images")
    H, W = images.shape[-2:]
    nimg = images.numel() // (H * W)
    out = torch.empty(images.shape[:-1] + (W // 2 + 1,), dtype=torch.complex64, device=images.device)
    lib = _lib()
    ws = workspace(lib.fdl_rfft2_workspace_size(nimg, H, W), images.device)
    L.check(lib.fdl_rfft2(_p(images), nimg, H, W, _p(out), _p(ws), ws.numel(), _stream(stream)), "fdl_rfft2")
    return out


def irfft2(spectra: torch.Tensor, W: int, stream=None) -> torch.Tensor:
    """Images ``[..., H, W]`` from half spectra ``[..., H, W//2+1]`` (Re of the completed inverse DFT)."""
    _need(spectra, torch.complex64, "spectra")
    H = spectra.shape[-2]
    if spectra.shape[-1] != W // 2 + 1:
        raise ValueError("spectra last dimension must be W//2+1")
    nimg = spectra.numel() // (H * (W // 2 + 1))
    out = torch.empty(spectra.shape[:-1] + (W,), dtype=torch.float32, device=spectra.device)
    lib = _lib()
    ws = workspace(lib.fdl_irfft2_workspace_size(nimg, H, W), spectra.device)
    L.check(lib.fdl_irfft2(_p(spectra), nimg, H, W, _p(out), _p(ws), ws.numel(), _stream(stream)), "fdl_irfft2")
    return out


# ---------------------------------------------------------------- fit
@dataclass
class FitWorkspace:
    buf: torch.Tensor

    def tier_counts(self, stream=None) -> dict:
        c = (ct.c_int * 5)()
        L.check(_lib().fdl_fit_tier_counts(_p(self.buf), c, _stream(stream)), "fdl_fit_tier_counts")
        return {"fp32": c[0], "df": c[1], "fp64": c[2], "high_precision": c[1] + c[2], "breakdown": c[3],
                "nonfinite": c[4]}

    def status(self, stream=None) -> int:
        """Device status word of the last fit (``L.ST_*`` bits); synchronises the stream."""
        return sync_status(self, stream)


def fit(views: torch.Tensor, u: torch.Tensor, d: torch.Tensor, lam: float, eps: float = 1e-4,
        reg: str = "view2", precision: str = "mixed", kappa_max: float = 0.0,
        out: torch.Tensor | None = None, ws: FitWorkspace | None = None, stream=None, df_error_budget: float = 0.0,
        f32_error_budget: float = 0.0):
    """Layer construction (Sec. V-A) of ``views [K][C][H][W]``; returns ``(layers, workspace)``."""
    _need(views, torch.float32, "views", 4)
    _need(u, torch.float32, "u", 2)
    _need(d, torch.float32, "d", 1)
    K, C, H, W = views.shape
    N = d.numel()
    lib = _lib()
    if out is None:
        out = torch.empty((N, C, H, W // 2 + 1), dtype=torch.complex64, device=views.device)
    need = lib.fdl_fit_workspace_size(K, C, H, W, N)
    if ws is None or ws.buf.numel() < need:
        ws = FitWorkspace(workspace(need, views.device))
    o = _opts(lam, eps, reg, precision, kappa_max, df_error_budget, f32_error_budget)
    L.check(lib.fdl_fit(_p(views), K, C, H, W, _p(u), _p(d), N, ct.byref(o), _p(out), _p(ws.buf),
                        ws.buf.numel(), _stream(stream)), "fdl_fit")
    return out, ws


def fit_spectra(spectra: torch.Tensor, u: torch.Tensor, d: torch.Tensor, lam: float, eps: float = 1e-4,
                reg: str = "view2", precision: str = "mixed", kappa_max: float = 0.0,
                out: torch.Tensor | None = None, ws: FitWorkspace | None = None, stream=None,
                df_error_budget: float = 0.0, f32_error_budget: float = 0.0, W: int | None = None):
    """Per-frequency solve from half spectra ``[K][C][H][W//2+1]``; returns ``(layers, workspace)``.
    ``W``: image width, needed when it is odd."""
    _need(spectra, torch.complex64, "spectra", 4)
    _need(u, torch.float32, "u", 2)
    _need(d, torch.float32, "d", 1)
    K, C, H, Wh = spectra.shape
    W = _width(Wh, W)
    N = d.numel()
    lib = _lib()
    if out is None:
        out = torch.empty((N, C, H, Wh), dtype=torch.complex64, device=spectra.device)
    need = lib.fdl_fit_spectra_workspace_size(K, C, H, W, N)
    if ws is None or ws.buf.numel() < need:
        ws = FitWorkspace(workspace(need, spectra.device))
    o = _opts(lam, eps, reg, precision, kappa_max, df_error_budget, f32_error_budget)
    L.check(lib.fdl_fit_spectra(_p(spectra), K, C, H, W, _p(u), _p(d), N, ct.byref(o), _p(out), _p(ws.buf),
                                ws.buf.numel(), _stream(stream)), "fdl_fit_spectra")
    return out, ws


# ---------------------------------------------------------------- render
def render(layers: torch.Tensor, d: torch.Tensor, u0: torch.Tensor, out: torch.Tensor | None = None,
           ws: torch.Tensor | None = None, stream=None, W: int | None = None) -> torch.Tensor:
    """Sub-aperture views (Eq. FourierView) at ``u0 [B][2]``: float32 ``[B][C][H][W]``
    (``W``: image width, needed when it is odd)."""
    _need(layers, torch.complex64, "layers", 4)
    _need(d, torch.float32, "d", 1)
    _need(u0, torch.float32, "u0", 2)
    N, C, H, Wh = layers.shape
    W = _width(Wh, W)
    B = u0.shape[0]
    lib = _lib()
    if out is None:
        out = torch.empty((B, C, H, W), dtype=torch.float32, device=layers.device)
    need = lib.fdl_render_workspace_size(B, C, H, W)
    if ws is None or ws.numel() < need:
        ws = workspace(need, layers.device)
    L.check(lib.fdl_render(_p(layers), _p(d), N, C, H, W, _p(u0), B, _p(out), _p(ws), ws.numel(),
                           _stream(stream)), "fdl_render")
    return out


@dataclass
class RenderSpec:
    """One image of Eq. BsFourier: FDL (layers, d), viewpoint, focus and aperture."""
    layers: torch.Tensor
    d: torch.Tensor
    u0: tuple
    s: float = 0.0
    aperture: str = "pinhole"
    radius: float = 0.0
    pts: torch.Tensor | None = None
    out: torch.Tensor | None = None
    W: int | None = None  # image width, needed when it is odd


def pack_requests(specs: list[RenderSpec], device) -> torch.Tensor:
    """Device array of ``fdl_request`` for :func:`refocus` (outputs allocated if missing)."""
    arr = (L.Request * len(specs))()
    for i, sp in enumerate(specs):
        N, C, H, Wh = sp.layers.shape
        if sp.out is None:
            sp.out = torch.empty((C, H, _width(Wh, sp.W)), dtype=torch.float32, device=device)
        arr[i] = L.Request(sp.layers.data_ptr(), sp.d.data_ptr(), sp.out.data_ptr(),
                           sp.pts.data_ptr() if sp.pts is not None else None, N,
                           0 if sp.pts is None else sp.pts.shape[0], L.APERTURE[sp.aperture],
                           float(sp.u0[0]), float(sp.u0[1]), float(sp.s), float(sp.radius), H,
                           _width(Wh, sp.W), C)
    host = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8)
    return host.to(device)


def refocus(req_dev: torch.Tensor, B: int, C: int, H: int, W: int, Nmax: int, count: torch.Tensor | None = None,
            ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Render B requests (device array from :func:`pack_requests`) into their outputs.  C, H, W:
    the largest channel count and image size of any request (power-of-two sizes may differ
    between requests); returns the workspace, whose status :func:`sync_status` reads."""
    lib = _lib()
    need = lib.fdl_refocus_workspace_size(B, C, H, W)
    if ws is None or ws.numel() < need:
        ws = workspace(need, req_dev.device)
    L.check(lib.fdl_refocus(_p(req_dev), B, _p(count), C, H, W, Nmax, _p(ws), ws.numel(), _stream(stream)),
            "fdl_refocus")
    return ws


def sync_status(ws, stream=None) -> int:
    """Device status word (``L.ST_*`` bits) of the last call that used workspace ``ws`` (a
    tensor or a :class:`FitWorkspace`); synchronises the stream."""
    buf = ws.buf if isinstance(ws, FitWorkspace) else ws
    v = ct.c_int(0)
    L.check(_lib().fdl_sync_status(_p(buf), ct.byref(v), _stream(stream)), "fdl_sync_status")
    return v.value


def aperture_table(raster: torch.Tensor, Z: int, stream=None) -> torch.Tensor:
    """Table of a drawn aperture (Sec. VI-A): complex64 ``[Z][Z//2+1]`` from an odd-sided float32
    raster ``[P][P]`` centred on its middle pixel.  Render it with ``RenderSpec(...,
    aperture="table", radius=h, pts=table)``, h being the raster pitch in units of u."""
    _need(raster, torch.float32, "raster", 2)
    P = raster.shape[0]
    lib = _lib()
    out = torch.empty((Z, Z // 2 + 1), dtype=torch.complex64, device=raster.device)
    ws = workspace(lib.fdl_aperture_table_workspace_size(P, Z), raster.device)
    L.check(lib.fdl_aperture_table(_p(raster), P, Z, _p(out), _p(ws), ws.numel(), _stream(stream)),
            "fdl_aperture_table")
    return out


def refocus_specs(specs: list[RenderSpec], stream=None) -> list[torch.Tensor]:
    """Convenience: pack, render and return the output images of ``specs`` in one launch
    (image sizes may differ when they are powers of two)."""
    dev = specs[0].layers.device
    req = pack_requests(specs, dev)
    C = max(s.layers.shape[1] for s in specs)
    H = max(s.layers.shape[2] for s in specs)
    W = max(_width(s.layers.shape[3], s.W) for s in specs)
    Nmax = max(s.layers.shape[0] for s in specs)
    refocus(req, len(specs), C, H, W, Nmax, stream=stream)
    return [s.out for s in specs]


# ---------------------------------------------------------------- general system
def pack_views(views: list, device) -> torch.Tensor:
    """Device ``fdl_request`` array describing each input image's aperture and focus for
    :func:`fit_general`: entries ``(aperture, radius, s)`` or ``(aperture, radius, s, pts)``."""
    arr = (L.Request * len(views))()
    keep = []
    for i, v in enumerate(views):
        kind, radius, s = v[0], v[1], v[2]
        pts = v[3] if len(v) > 3 else None
        if pts is not None:
            keep.append(pts)
        npts = 0 if pts is None else pts.shape[0]
        arr[i] = L.Request(None, None, None, pts.data_ptr() if pts is not None else None, 0, npts, L.APERTURE[kind],
                           0.0, 0.0, float(s), float(radius))
    return torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).to(device)


def fit_general(spectra: torch.Tensor, N: int, lam: float, eps: float = 1e-4, reg: str = "view2",
                precision: str = "df", u: torch.Tensor | None = None, d: torch.Tensor | None = None,
                P: torch.Tensor | None = None, views: torch.Tensor | None = None, W: int | None = None,
                stream=None) -> torch.Tensor:
    """Layer construction for the general system of Eq. AMatGeneral: shifts ``u_j d_k`` or free
    ``P [K][N][2]`` (the relaxed model), per-image apertures from :func:`pack_views` (focal
    stacks, hybrid inputs).  ``precision``: "f64" or double-float."""
    _need(spectra, torch.complex64, "spectra", 4)
    for t, name in ((u, "u"), (d, "d"), (P, "P")):
        if t is not None:
            _need(t, torch.float32, name)
    K, C, H, Wh = spectra.shape
    W = _width(Wh, W)
    lib = _lib()
    out = torch.empty((N, C, H, Wh), dtype=torch.complex64, device=spectra.device)
    ws = workspace(lib.fdl_fit_general_workspace_size(K, C, H, W, N), spectra.device)
    sysd = L.System(_p(u).value, _p(d).value, _p(P).value, _p(views).value)
    o = _opts(lam, eps, reg, precision, 0.0)
    L.check(lib.fdl_fit_general(_p(spectra), K, C, H, W, N, ct.byref(sysd), ct.byref(o), _p(out), _p(ws),
                                ws.numel(), _stream(stream)), "fdl_fit_general")
    return out


def render_shifts(layers: torch.Tensor, P: torch.Tensor, W: int | None = None, stream=None) -> torch.Tensor:
    """Images ``[B][C][H][W]`` rendered with per-layer shifts ``P [B][N][2]`` (the relaxed model)."""
    _need(layers, torch.complex64, "layers", 4)
    _need(P, torch.float32, "P", 3)
    N, C, H, Wh = layers.shape
    W = _width(Wh, W)
    B = P.shape[0]
    lib = _lib()
    out = torch.empty((B, C, H, W), dtype=torch.float32, device=layers.device)
    ws = workspace(lib.fdl_render_shifts_workspace_size(B, C, H, W), layers.device)
    L.check(lib.fdl_render_shifts(_p(layers), _p(P), N, C, H, W, B, _p(out), _p(ws), ws.numel(), _stream(stream)),
            "fdl_render_shifts")
    return out


def calib_grad_shifts(spectra: torch.Tensor, P: torch.Tensor, lam: float, reg: str = "layer2",
                      bins: torch.Tensor | None = None, precision: str = "df", W: int | None = None, stream=None):
    """Loss of Eq. CalibrationProb with free shifts ``P [K][N][2]`` and ``dL/dP`` (Eq. gradP)."""
    _need(spectra, torch.complex64, "spectra", 4)
    _need(P, torch.float32, "P", 3)
    K, C, H, Wh = spectra.shape
    W = _width(Wh, W)
    N = P.shape[1]
    nb = 0
    if bins is not None:
        _need(bins, torch.int32, "bins", 1)
        nb = bins.numel()
    lib = _lib()
    loss = torch.empty(1, dtype=torch.float32, device=spectra.device)
    gP = torch.empty((K, N, 2), dtype=torch.float32, device=spectra.device)
    ws = workspace(lib.fdl_calib_grad_shifts_workspace_size(K, C, H, W, N, nb), spectra.device)
    o = _opts(lam, 0.0, reg, precision, 0.0)
    L.check(lib.fdl_calib_grad_shifts(_p(spectra), K, C, H, W, _p(P), N, ct.byref(o), _p(bins), nb, _p(loss),
                                      _p(gP), _p(ws), ws.numel(), _stream(stream)), "fdl_calib_grad_shifts")
    return loss, gP


# ---------------------------------------------------------------- calibration
def calib_grad(spectra: torch.Tensor, u: torch.Tensor, d: torch.Tensor, lam: float, reg: str = "layer2",
               bins: torch.Tensor | None = None, precision: str = "df", stream=None, W: int | None = None):
    """Loss of Eq. CalibrationProb and its gradient w.r.t. u [K][2] and d [N] (Eqs. gradP, gradD)."""
    _need(spectra, torch.complex64, "spectra", 4)
    _need(u, torch.float32, "u", 2)
    _need(d, torch.float32, "d", 1)
    K, C, H, Wh = spectra.shape
    W = _width(Wh, W)
    N = d.numel()
    nb = 0
    if bins is not None:
        _need(bins, torch.int32, "bins", 1)
        nb = bins.numel()
    lib = _lib()
    loss = torch.empty(1, dtype=torch.float32, device=spectra.device)
    gu = torch.empty((K, 2), dtype=torch.float32, device=spectra.device)
    gd = torch.empty(N, dtype=torch.float32, device=spectra.device)
    ws = workspace(lib.fdl_calib_grad_workspace_size(K, C, H, W, N, nb), spectra.device)
    o = _opts(lam, 0.0, reg, precision, 100.0)
    L.check(lib.fdl_calib_grad(_p(spectra), K, C, H, W, _p(u), _p(d), N, ct.byref(o), _p(bins), nb, _p(loss),
                               _p(gu), _p(gd), _p(ws), ws.numel(), _stream(stream)), "fdl_calib_grad")
    return loss, gu, gd
