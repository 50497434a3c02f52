"""Host-to-host pipeline over a sequence of light fields: views in pinned host memory ->
layers (Sec. V-A) -> rendered views and refocused images (Sec. VI-A) back in pinned host
memory, with the copies of one light field overlapping the computation of its neighbours.

Two device slots and three streams:

* copy-in: the views of submission i into slot i % 2, once the fit of submission i - 2 has
  finished reading that slot;
* compute: ``fdl_fit``, ``fdl_render`` and ``fdl_refocus`` of the slot, once its views are in
  and the copy-out of submission i - 2 has finished reading the slot's images;
* copy-out: the slot's images, one contiguous ``[B + R][C][H][W]`` block, to the caller's
  pinned buffer.

All ordering is by CUDA events; the host waits only in :meth:`FitRenderPipeline.wait`.  The
caller keeps each submission's host buffers alive and unmodified until it has been waited for.
"""

from __future__ import annotations

import time

import torch

from . import _lib as L
from . import fdl


class FitRenderPipeline:
    """Fit + render + refocus of same-shaped light fields, two submissions in flight.

    ``u [K][2]``, ``d [N]``: view positions and disparities (shared by all submissions);
    ``u0 [B][2]``: viewpoints rendered with a pinhole; ``refocus``: ``(u0, s, aperture, radius)``
    per refocused image.  Output row ``b < B`` is view ``u0[b]``, row ``B + r`` refocused image r.
    """

    def __init__(self, K: int, C: int, H: int, W: int, u: torch.Tensor, d: torch.Tensor, lam: float,
                 eps: float = 1e-4, u0: torch.Tensor | None = None, refocus: list | tuple = (),
                 precision: str = "mixed", reg: str = "view2", device="cuda"):
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
        for _ in range(2):
            s = {"views": torch.empty((K, C, H, W), dtype=torch.float32, device=self.dev),
                 "layers": torch.empty((self.N, C, H, W // 2 + 1), dtype=torch.complex64, device=self.dev),
                 "out": torch.empty((self.B + self.R, C, H, W), dtype=torch.float32, device=self.dev),
                 "ws_fit": fdl.FitWorkspace(fdl.workspace(lib.fdl_fit_workspace_size(K, C, H, W, self.N), self.dev)),
                 "ws_render": fdl.workspace(lib.fdl_render_workspace_size(max(self.B, 1), C, H, W), self.dev),
                 "ws_refocus": fdl.workspace(lib.fdl_refocus_workspace_size(max(self.R, 1), C, H, W), self.dev),
                 "views_read": None, "out_read": None, "done": None}
            if self.R:
                specs = [fdl.RenderSpec(s["layers"], self.d, tuple(map(float, r[0])), float(r[1]), r[2], float(r[3]),
                                        out=s["out"][self.B + i]) for i, r in enumerate(refocus)]
                s["req"] = fdl.pack_requests(specs, self.dev)
            self.slots.append(s)
        self.s_in = torch.cuda.Stream(self.dev)
        self.s_comp = torch.cuda.Stream(self.dev)
        self.s_out = torch.cuda.Stream(self.dev)
        self.n = 0
        self.pending: dict[int, torch.cuda.Event] = {}

    def submit(self, views_host: torch.Tensor, out_host: torch.Tensor) -> int:
        """Queue one light field: ``views_host [K][C][H][W]`` float32 (pinned) in, ``out_host
        [B + R][C][H][W]`` float32 (pinned) out.  Returns a ticket for :meth:`wait`."""
        if tuple(views_host.shape) != (self.K, self.C, self.H, self.W) or views_host.dtype != torch.float32:
            raise ValueError("views_host must be float32 [K][C][H][W]")
        if tuple(out_host.shape) != (self.B + self.R, self.C, self.H, self.W) or out_host.dtype != torch.float32:
            raise ValueError("out_host must be float32 [B + R][C][H][W]")
        s = self.slots[self.n % 2]
        ev_in = torch.cuda.Event()
        with torch.cuda.stream(self.s_in):
            if s["views_read"] is not None:
                self.s_in.wait_event(s["views_read"])
            s["views"].copy_(views_host, non_blocking=True)
            ev_in.record(self.s_in)
        with torch.cuda.stream(self.s_comp):
            self.s_comp.wait_event(ev_in)
            fdl.fit(s["views"], self.u, self.d, self.lam, self.eps, reg=self.reg, precision=self.precision,
                    out=s["layers"], ws=s["ws_fit"], stream=self.s_comp)
            s["views_read"] = torch.cuda.Event()
            s["views_read"].record(self.s_comp)
            if s["out_read"] is not None:
                self.s_comp.wait_event(s["out_read"])
            if self.B:
                fdl.render(s["layers"], self.d, self.u0, out=s["out"][:self.B], ws=s["ws_render"], stream=self.s_comp)
            if self.R:
                fdl.refocus(s["req"], self.R, self.C, self.H, self.W, self.N, ws=s["ws_refocus"], stream=self.s_comp)
            ev_comp = torch.cuda.Event()
            ev_comp.record(self.s_comp)
        with torch.cuda.stream(self.s_out):
            self.s_out.wait_event(ev_comp)
            out_host.copy_(s["out"], non_blocking=True)
            s["out_read"] = torch.cuda.Event()
            s["out_read"].record(self.s_out)
        # every stream that touched caller memory has to finish before the ticket completes
        done = torch.cuda.Event()
        self.s_out.wait_event(ev_in)
        done.record(self.s_out)
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
