"""Host-to-host pipeline over a sequence of light fields: views in pinned host memory ->
layers (Sec. V-A) -> rendered views and refocused images (Sec. VI-A) back in pinned host
memory, through the C ABI's ``fdl_fit_render_host`` (the library enqueues the copies, the
fit and the render).

A few slots (three by default), each with its own stream, layers, device images, request
descriptors and workspace; submission i goes to slot i % slots, so that the copies of one
light field overlap the computation of its neighbours on the other streams (9x9 views, 512^2
RGB on a GB300: 13.9 ms per light field with two slots, 13.3 ms with three, 12.8 ms for the
computation alone).  The host waits only in
:meth:`FitRenderPipeline.wait`.  The caller keeps each submission's host buffers alive and
unmodified until it has been waited for.
"""

from __future__ import annotations

import ctypes as ct
import time

import torch

from . import _lib as L
from . import fdl


class FitRenderPipeline:
    """Fit + render + refocus of same-shaped light fields, ``slots`` submissions in flight.

    ``u [K][2]``, ``d [N]``: view positions and disparities (shared by all submissions);
    ``u0 [B][2]``: viewpoints rendered with a pinhole; ``refocus``: ``(u0, s, aperture, radius)``
    per refocused image.  Output row ``b < B`` is view ``u0[b]``, row ``B + r`` refocused image r.
    """

    def __init__(self, K: int, C: int, H: int, W: int, u: torch.Tensor, d: torch.Tensor, lam: float,
                 eps: float = 1e-4, u0: torch.Tensor | None = None, refocus: list | tuple = (),
                 precision: str = "mixed", reg: str = "view2", device="cuda", slots: int = 3):
        self.K, self.C, self.H, self.W = K, C, H, W
        self.dev = torch.device(device)
        self.u = u.to(self.dev, torch.float32).contiguous()
        self.d = d.to(self.dev, torch.float32).contiguous()
        self.u0 = (u0 if u0 is not None else torch.zeros((0, 2))).to(self.dev, torch.float32).contiguous()
        self.B, self.R = self.u0.shape[0], len(refocus)
        self.N = self.d.numel()
        self.lam, self.eps, self.precision, self.reg = float(lam), float(eps), precision, reg
        lib = L.load()
        self.slots = []
        if slots < 1:
            raise ValueError("slots must be at least 1")
        for _ in range(slots):
            sl = {"layers": torch.empty((self.N, C, H, W // 2 + 1), dtype=torch.complex64, device=self.dev),
                  "out": torch.empty((self.B + self.R, C, H, W), dtype=torch.float32, device=self.dev),
                  "ws": fdl.workspace(lib.fdl_fit_render_host_workspace_size(K, C, H, W, self.N, self.B + self.R),
                                      self.dev),
                  "stream": torch.cuda.Stream(self.dev)}
            specs = [fdl.RenderSpec(sl["layers"], self.d, tuple(map(float, self.u0[b].tolist())), out=sl["out"][b])
                     for b in range(self.B)]
            specs += [fdl.RenderSpec(sl["layers"], self.d, tuple(map(float, r[0])), float(r[1]), r[2], float(r[3]),
                                     out=sl["out"][self.B + i]) for i, r in enumerate(refocus)]
            if not specs:
                raise ValueError("nothing to render: give u0 or refocus")
            sl["req"] = fdl.pack_requests(specs, self.dev)
            self.slots.append(sl)
        self.opts = fdl._opts(self.lam, self.eps, reg, precision, 0.0)
        torch.cuda.synchronize(self.dev)  # descriptors in place before the slot streams read them
        self.n = 0
        self.pending: dict[int, torch.cuda.Event] = {}

    def submit(self, views_host: torch.Tensor, out_host: torch.Tensor) -> int:
        """Queue one light field: ``views_host [K][C][H][W]`` float32 (pinned) in, ``out_host
        [B + R][C][H][W]`` float32 (pinned) out.  Returns a ticket for :meth:`wait`."""
        if tuple(views_host.shape) != (self.K, self.C, self.H, self.W) or views_host.dtype != torch.float32:
            raise ValueError("views_host must be float32 [K][C][H][W]")
        if tuple(out_host.shape) != (self.B + self.R, self.C, self.H, self.W) or out_host.dtype != torch.float32:
            raise ValueError("out_host must be float32 [B + R][C][H][W]")
        if views_host.is_cuda or out_host.is_cuda or not views_host.is_contiguous() or not out_host.is_contiguous():
            raise ValueError("views_host and out_host must be contiguous host tensors")
        sl = self.slots[self.n % len(self.slots)]
        st = sl["stream"]
        L.check(L.load().fdl_fit_render_host(
            views_host.data_ptr(), self.K, self.C, self.H, self.W, self.u.data_ptr(), self.d.data_ptr(), self.N,
            ct.byref(self.opts), sl["layers"].data_ptr(), sl["req"].data_ptr(), self.B + self.R,
            sl["out"].data_ptr(), sl["out"].numel(), out_host.data_ptr(), sl["ws"].data_ptr(), sl["ws"].numel(),
            ct.c_void_p(st.cuda_stream)), "fdl_fit_render_host")
        done = torch.cuda.Event()
        done.record(st)
        ticket = self.n
        self.pending[ticket] = done
        self.n += 1
        return ticket

    def wait(self, ticket: int | None = None, timeout: float = 600.0) -> None:
        """Block until the submission ``ticket`` (default: every submission) has landed in its
        host buffer; ``TimeoutError`` after ``timeout`` seconds of polling."""
        tickets = [ticket] if ticket is not None else sorted(self.pending)
        deadline = time.monotonic() + timeout
        for t in tickets:
            ev = self.pending.get(t)
            if ev is None:
                continue
            while not ev.query():
                if time.monotonic() > deadline:
                    raise TimeoutError(f"pipeline submission {t} not complete after {timeout} s")
                time.sleep(50e-6)
            del self.pending[t]
