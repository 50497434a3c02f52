"""Serving: resident FDLs and continuous batching of render / refocus requests.

* ``FdlStore`` keeps fitted FDLs (layer spectra + disparities) on the device under
  a byte budget; admitting a new light field fits it on a side stream, evicts the
  least recently used FDLs that no in-flight request reads, and rolls back
  cleanly if it cannot make room or the allocation fails.  Each entry carries a
  CUDA event recorded after its fit: no batch reads its layers before it.
* ``Server`` runs a few batch buffers, each with its own stream, device
  descriptor array (``fdl_request``), batch-count word and workspace, and a CUDA
  graph that copies the descriptors in and runs ``fdl_refocus`` over them.  One
  graph serves every image size: requests of different FDLs, power-of-two sizes,
  viewpoints and apertures share a launch.  A tick fills whichever buffer is
  free with the queued requests (up to its capacity) and replays its graph, so
  requests that arrive while a batch is on the GPU go into the next batch and
  the batches overlap on the device.  Completion is polled with bounded waits
  (``TimeoutError`` past the deadline).
"""

from __future__ import annotations

import collections
import ctypes as ct
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as L
from . import fdl


class AdmissionError(RuntimeError):
    pass


@dataclass
class FdlEntry:
    fid: int
    layers: torch.Tensor
    d: torch.Tensor
    H: int
    W: int
    C: int
    N: int
    nbytes: int
    refs: int = 0
    last_used: float = 0.0
    ready: object = None  # CUDA event recorded after the fit (None on the CPU)


class FdlStore:
    """Resident FDLs under a device-memory budget (bytes of layer spectra + disparities)."""

    def __init__(self, budget_bytes: int, device, allocate=None):
        self.budget = int(budget_bytes)
        self.device = torch.device(device)
        self.entries: collections.OrderedDict[int, FdlEntry] = collections.OrderedDict()
        self._allocate = allocate or (lambda shape, dtype: torch.empty(shape, dtype=dtype, device=self.device))

    @property
    def bytes_used(self) -> int:
        return sum(e.nbytes for e in self.entries.values())

    @staticmethod
    def fdl_bytes(N, C, H, W) -> int:
        return N * C * H * (W // 2 + 1) * 8 + N * 4

    def _make_room(self, need: int) -> list[int]:
        """FDLs to evict (least recently used, not in use) so that `need` more bytes fit."""
        free = self.budget - self.bytes_used
        victims = []
        for fid, e in sorted(self.entries.items(), key=lambda kv: kv[1].last_used):
            if free >= need:
                break
            if e.refs == 0:
                victims.append(fid)
                free += e.nbytes
        if free < need:
            raise AdmissionError(f"cannot fit {need} bytes within the {self.budget}-byte budget")
        return victims

    def admit(self, fid: int, views: torch.Tensor, u: torch.Tensor, d: torch.Tensor, lam: float = 1e-2,
              eps: float = 1e-4, stream=None) -> FdlEntry:
        """Fit and keep an FDL; on any failure nothing changes (already resident FDLs stay)."""
        if fid in self.entries:
            raise AdmissionError(f"FDL {fid} is already resident")
        K, C, H, W = views.shape
        N = d.numel()
        need = self.fdl_bytes(N, C, H, W)
        victims = self._make_room(need)
        try:
            layers = self._allocate((N, C, H, W // 2 + 1), torch.complex64)
            dd = self._allocate((N,), torch.float32)
        except (RuntimeError, MemoryError) as e:
            raise AdmissionError(f"allocation failed: {e}") from e
        dd.copy_(d)
        ready = None
        if layers.is_cuda:
            st = stream if stream is not None else torch.cuda.current_stream(layers.device)
            # the fit (and its workspace) runs on `st`; layers and d, allocated on the current
            # stream, are marked as used there so that the allocator keeps them until it is done
            dd_ready = torch.cuda.Event()
            dd_ready.record()
            st.wait_event(dd_ready)
            with torch.cuda.stream(st):
                fdl.fit(views, u, dd, lam, eps, out=layers, stream=st)
                ready = torch.cuda.Event()
                ready.record(st)
            layers.record_stream(st)
            dd.record_stream(st)
        for v in victims:
            self.entries.pop(v)
        e = FdlEntry(fid, layers, dd, H, W, C, N, need, last_used=time.perf_counter(), ready=ready)
        self.entries[fid] = e
        return e

    def get(self, fid: int) -> FdlEntry:
        e = self.entries[fid]
        e.last_used = time.perf_counter()
        return e

    def is_ready(self, fid: int) -> bool:
        """True once the FDL's fit has finished on the device (its event is then dropped, so
        later calls cost nothing and batches no longer wait on it)."""
        e = self.entries[fid]
        if e.ready is not None and e.ready.query():
            e.ready = None
        return e.ready is None


@dataclass
class Request:
    rid: int
    fid: int
    u0: tuple
    s: float = 0.0
    aperture: str = "pinhole"
    radius: float = 0.0
    t_arrival: float = 0.0
    t_done: float | None = None
    out: torch.Tensor | None = None
    batch_size: int = 0
    batch_id: int = -1  # the launch that rendered it


class _Batch:
    """One batch buffer: stream, descriptors, count, workspace and the captured graph of
    ``fdl_refocus`` over images up to (C, H, W)."""

    def __init__(self, H, W, C, cap, Nmax, device):
        self.H, self.W, self.C, self.cap, self.Nmax = H, W, C, cap, Nmax
        # the highest stream priority: admission fits run on default-priority streams, and
        # their short CTAs let batches of requests be scheduled in between
        self.stream = torch.cuda.Stream(device=device, priority=torch.cuda.Stream.priority_range()[1])
        self.host_desc = torch.zeros(cap * ct.sizeof(L.Request), dtype=torch.uint8).pin_memory()
        self.host_count = torch.zeros(1, dtype=torch.int32).pin_memory()
        self.dev_desc = torch.zeros(cap * ct.sizeof(L.Request), dtype=torch.uint8, device=device)
        self.dev_count = torch.zeros(1, dtype=torch.int32, device=device)
        lib = L.load()
        self.ws = fdl.workspace(lib.fdl_refocus_workspace_size(cap, C, H, W), device)
        self.graph = None
        self.done = torch.cuda.Event()
        self.requests: list[Request] = []
        self.busy = False

    def _body(self):
        self.dev_desc.copy_(self.host_desc, non_blocking=True)
        self.dev_count.copy_(self.host_count, non_blocking=True)
        fdl.refocus(self.dev_desc, self.cap, self.C, self.H, self.W, self.Nmax, count=self.dev_count, ws=self.ws)

    def capture(self):
        # warm up (loads modules, sets kernel attributes) with an empty batch, then capture
        with torch.cuda.stream(self.stream):
            self.host_count.zero_()
            self._body()
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self._body()
        self.stream.synchronize()

    def launch(self, reqs: list[Request], store: FdlStore, pts: dict, batch_id: int = -1, timeline=None):
        # requests of one FDL side by side: the mixed render stages each FDL's layer values
        # once per run of consecutive requests that read it
        reqs = sorted(reqs, key=lambda r: r.fid)
        arr = (L.Request * self.cap).from_buffer(self.host_desc.numpy())
        waits = {}
        for i, r in enumerate(reqs):
            e = store.get(r.fid)
            p = pts.get(r.aperture)
            arr[i] = L.Request(e.layers.data_ptr(), e.d.data_ptr(), r.out.data_ptr(),
                               p.data_ptr() if p is not None else None, e.N, 0 if p is None else p.shape[0],
                               L.APERTURE[r.aperture], float(r.u0[0]), float(r.u0[1]), float(r.s), float(r.radius),
                               e.H, e.W, e.C)
            r.batch_size = len(reqs)
            r.batch_id = batch_id
            if e.ready is not None:
                waits[e.fid] = e.ready
        self.host_count[0] = len(reqs)
        # algorithmic bytes of the batch: each FDL's layers read once, each image written once
        self.alg_bytes = sum(store.entries[f].nbytes for f in {r.fid for r in reqs}) + sum(
            4 * r.out.numel() for r in reqs)
        # a light field admitted moments ago may still be fitting on its side stream
        for ev in waits.values():
            self.stream.wait_event(ev)
        with torch.cuda.stream(self.stream):
            if timeline is not None:
                t0 = torch.cuda.Event(enable_timing=True)
                t1 = torch.cuda.Event(enable_timing=True)
                t0.record(self.stream)
            self.graph.replay()
            self.done.record(self.stream)
            if timeline is not None:
                t1.record(self.stream)
                timeline.append((t0, t1, self.alg_bytes, len(reqs)))
        self.requests = list(reqs)
        self.busy = True


class Server:
    """Continuous batching of render / refocus requests over resident FDLs.

    ``sizes``: the (H, W, C) image sizes served (powers of two); one graph per batch buffer
    covers all of them, each buffer holding up to ``capacity`` requests of any mix of sizes.
    """

    def __init__(self, store: FdlStore, sizes, Nmax: int = 64, capacity: int = 32, pool: int = 128,
                 buffers: int = 2):
        self.store = store
        self.dev = store.device
        self.sizes = [tuple(s) for s in sizes]
        H = max(s[0] for s in self.sizes)
        W = max(s[1] for s in self.sizes)
        C = max(s[2] for s in self.sizes)
        self.batches = [_Batch(H, W, C, capacity, Nmax, self.dev) for _ in range(buffers)]
        self.pool = {(h, w, c): [torch.empty((c, h, w), dtype=torch.float32, device=self.dev) for _ in range(pool)]
                     for (h, w, c) in self.sizes}
        for b in self.batches:
            b.capture()
        self.queue: collections.deque = collections.deque()
        self.completed: list[Request] = []
        self._fresh: list[Request] = []
        self.pts = {}
        self.alg_bytes = 0  # algorithmic bytes of every launched batch (layers once per FDL, images)
        self.launches = 0
        # with a list here, every launch appends (start event, end event, algorithmic bytes,
        # requests) recorded on its stream: device time of the batches (busy_ms)
        self.timeline: list | None = None

    def submit(self, r: Request):
        # a queued request holds its FDL: admissions do not evict it before it has rendered
        self.store.entries[r.fid].refs += 1
        self.queue.append(r)

    def release(self, r: Request):
        """Return a completed request's output buffer to its pool."""
        c, h, w = r.out.shape
        self.pool[(h, w, c)].append(r.out)
        r.out = None

    def _poll(self):
        now = None
        for b in self.batches:
            if b.busy and b.done.query():
                now = now or time.perf_counter()
                for r in b.requests:
                    r.t_done = now
                    self.store.entries[r.fid].refs -= 1
                    self.completed.append(r)
                    self._fresh.append(r)
                b.requests = []
                b.busy = False

    def _busy(self) -> bool:
        return any(b.busy for b in self.batches)

    def tick(self) -> int:
        """Poll finished batches, then launch queued requests into free buffers; returns launches."""
        self._poll()
        launched = 0
        for b in self.batches:
            if not self.queue:
                break
            if b.busy:
                continue
            reqs = []
            # FIFO; a request waits while the output pool of its size is empty
            while self.queue and len(reqs) < b.cap:
                r = self.queue[0]
                e = self.store.entries[r.fid]
                pool = self.pool[(e.H, e.W, e.C)]
                if not pool:
                    break
                r.out = pool.pop()
                reqs.append(self.queue.popleft())
            if not reqs:
                break
            b.launch(reqs, self.store, self.pts, self.launches, self.timeline)
            self.alg_bytes += b.alg_bytes
            self.launches += 1
            launched += 1
        return launched

    def busy_ms(self) -> float:
        """Device time during which at least one recorded batch ran (the union of the
        batches' [start, end] intervals; the batch streams overlap).  Synchronises."""
        if not self.timeline:
            return 0.0
        for _, t1, _, _ in self.timeline:
            t1.synchronize()
        ref = self.timeline[0][0]
        iv = sorted((ref.elapsed_time(t0), ref.elapsed_time(t1)) for t0, t1, _, _ in self.timeline)
        total, cur0, cur1 = 0.0, iv[0][0], iv[0][1]
        for a, b in iv[1:]:
            if a > cur1:
                total += cur1 - cur0
                cur0, cur1 = a, b
            else:
                cur1 = max(cur1, b)
        return total + cur1 - cur0

    def drain(self, timeout_s: float = 30.0):
        """Run ticks until every queued request has completed (bounded wait)."""
        t0 = time.perf_counter()
        while self.queue or self._busy():
            self.tick()
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("requests did not complete within the deadline")

    def run_trace(self, trace: list[Request], timeout_s: float = 120.0, keep_outputs: bool = False):
        """Replay requests at their arrival times (seconds from the start) in real time."""
        t0 = time.perf_counter()
        i = 0
        trace = sorted(trace, key=lambda r: r.t_arrival)
        for r in trace:
            r.t_arrival += t0
        while i < len(trace) or self.queue or self._busy():
            now = time.perf_counter()
            while i < len(trace) and trace[i].t_arrival <= now:
                self.submit(trace[i])
                i += 1
            self.tick()
            if not keep_outputs:
                for r in self._fresh:
                    self.release(r)
            self._fresh.clear()
            if now - t0 > timeout_s:
                raise TimeoutError("trace did not complete within the deadline")
        lat = np.array([(r.t_done - r.t_arrival) * 1e3 for r in trace])
        return {"requests": len(trace), "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                "wall_s": time.perf_counter() - t0,
                "mean_batch": float(np.mean([r.batch_size for r in trace]))}
