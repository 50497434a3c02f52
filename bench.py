"""Benchmark of the FDL hot path on GB300: layer construction + rendering.

One step = fit the 9x9-view, 512x512 RGB, 30-layer light field (DFT of the
243 view images, per-frequency solve at all 131,584 stored frequencies), then
render the 81 input viewpoints and 32 refocused images (disc aperture of
radius 1 at focus disparities linspace(-3, 3, 32)).  The reported value is
frequencies taken through the whole step per second (Mfreq/s); the fit-only
rate, the render rate in MPix/s and single-request render latencies are
reported beside it, together with the plain FP64 one-request-at-a-time GPU
path (torch complex128: rfft2, batched Cholesky, irfft2) and the FP64 oracle
on the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fdl|reference]
"""

from __future__ import annotations

import argparse
import json
import os
import signal
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H = W = 512
C = 3
GRID = 4  # 9x9 views
N = 30
LAM, EPS = 1e-2, 1e-4
N_REFOCUS = 32
SEED = 3
METRIC = "FDL-fit Mfreq/s and render MPix/s vs plain FP64 GPU path; render p50/p99 latency"
WORKLOAD = "9x9 views (u in [-4,4]^2), 512x512 RGB, N=30 d=linspace(-3,3,30), lambda=1e-2; fit + render 81 views + 32 refocus"


def workload_inputs():
    from scenes import occluding_planes, view_grid

    u = view_grid(GRID)
    d = np.linspace(-3, 3, N).astype(np.float32)
    views, _ = occluding_planes(SEED, H, W, C, u)
    s_list = np.linspace(-3, 3, N_REFOCUS).astype(np.float32)
    return views, u, d, s_list


def q_half():
    return H * (W // 2 + 1)


def pix_per_step(n_images):
    return n_images * H * W


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples taken during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ our path
class FdlPath:
    def __init__(self, device, views, u, d, s_list):
        import torch

        import paper_1901_06919_gb300 as F

        self.F = F
        self.torch = torch
        self.dev = device
        self.views = torch.from_numpy(views).to(device)
        self.u = torch.from_numpy(u).to(device)
        self.d = torch.from_numpy(d).to(device)
        self.u0 = torch.from_numpy(u).to(device)  # the 81 input viewpoints
        self.layers = torch.empty((N, C, H, W // 2 + 1), dtype=torch.complex64, device=device)
        self.views_out = torch.empty((len(u), C, H, W), dtype=torch.float32, device=device)
        self.ws_fit = None
        self.ws_render = F.workspace(F._lib.load().fdl_render_workspace_size(len(u), C, H, W), device)
        self.ws_refocus = F.workspace(F._lib.load().fdl_refocus_workspace_size(N_REFOCUS, C, H, W), device)
        self.s_list = list(s_list)
        self.specs = [F.RenderSpec(self.layers, self.d, (0.0, 0.0), float(s), "disc", 1.0) for s in s_list]
        self.req = F.pack_requests(self.specs, device)
        _, self.ws_fit = F.fit(self.views, self.u, self.d, LAM, EPS, out=self.layers)

    def fit(self):
        self.F.fit(self.views, self.u, self.d, LAM, EPS, out=self.layers, ws=self.ws_fit)

    def render(self):
        self.F.render(self.layers, self.d, self.u0, out=self.views_out, ws=self.ws_render)

    def refocus(self):
        self.F.refocus(self.req, N_REFOCUS, C, H, W, N, ws=self.ws_refocus)

    def step(self, ev=None):
        self.fit()
        if ev is not None:
            ev[0].record()
        self.render()
        if ev is not None:
            ev[1].record()
        self.refocus()


def time_device_steps(path, steps, warmup):
    torch = path.torch
    for _ in range(warmup):
        path.step()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    marks = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
    begins = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    start.record()
    for i in range(steps):
        begins[i].record()
        path.step(marks[i])
        ends[i].record()
    stop.record()
    torch.cuda.synchronize()
    total = start.elapsed_time(stop)
    fit_ms = sum(begins[i].elapsed_time(marks[i][0]) for i in range(steps)) / steps
    render_ms = sum(marks[i][0].elapsed_time(marks[i][1]) for i in range(steps)) / steps
    refocus_ms = sum(marks[i][1].elapsed_time(ends[i]) for i in range(steps)) / steps
    return total, {"fit_ms": fit_ms, "render81_ms": render_ms, "refocus32_ms": refocus_ms}


def time_e2e(path, views_host, steps, warmup, rounds=3):
    """Views from pinned host memory -> fit -> 81 + 32 images back to pinned host memory, each
    step one call of the C ABI's fdl_fit_render_host (copies, fit and render enqueued by the
    library) on one of three streams, so that the copies of one step overlap the computation of
    its neighbours.  Device span from the first copy-in to the last copy-out, CUDA events, per
    step; the median of `rounds` such spans of `steps` steps."""
    torch = path.torch
    from paper_1901_06919_gb300.pipeline import FitRenderPipeline

    refocus = [((0.0, 0.0), float(s), "disc", 1.0) for s in path.s_list]
    pipe = FitRenderPipeline(len(path.u), C, H, W, path.u, path.d, LAM, EPS, u0=path.u0, refocus=refocus,
                             device=path.dev)
    ns = len(pipe.slots)
    out_host = [torch.empty((len(path.u0) + len(refocus), C, H, W), dtype=torch.float32).pin_memory()
                for _ in range(ns)]
    for i in range(warmup):
        pipe.submit(views_host, out_host[i % ns])
    pipe.wait()
    torch.cuda.synchronize()
    streams = [sl["stream"] for sl in pipe.slots]
    spans = []
    for _ in range(rounds):
        a = torch.cuda.Event(enable_timing=True)
        a.record(streams[0])
        for s in streams[1:]:
            s.wait_event(a)
        n0 = pipe.n
        for i in range(steps):
            pipe.submit(views_host, out_host[(n0 + i) % ns])
        ends = []
        for s in streams:
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(s)
            ends.append(ev)
        pipe.wait()
        torch.cuda.synchronize()
        spans.append(max(a.elapsed_time(ev) for ev in ends) / steps)
    # the median of the rounds: the copies share the host's memory and NVLink-C2C with whatever
    # else the machine runs, and one disturbed round does not move it
    return float(np.median(spans)), views_host.numel() * 4, out_host[0].numel() * 4


def time_kernel_legs(path, reps=10):
    """Each stage of the step alone, for the per-kernel roofline and the stage table."""
    torch = path.torch
    F = path.F
    out = {}
    spectra = F.rfft2(path.views)
    ws_s = None

    def timed(fn, n=reps):
        # median of per-call device times (events around each call on the current stream):
        # one call disturbed by other work on a shared GPU does not move it
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        evs = []
        for _ in range(n):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            evs.append((a, b))
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in evs]))

    out["rfft2_ms"] = timed(lambda: F.rfft2(path.views))
    _, ws_s = F.fit_spectra(spectra, path.u, path.d, LAM, EPS, out=path.layers)
    out["solve_mixed_ms"] = timed(lambda: F.fit_spectra(spectra, path.u, path.d, LAM, EPS, out=path.layers, ws=ws_s))
    out["tiers"] = ws_s.tier_counts()
    out["solve_f32_all_ms"] = timed(lambda: F.fit_spectra(spectra, path.u, path.d, LAM, EPS, precision="f32",
                                                          out=path.layers, ws=ws_s))
    out["solve_df_all_ms"] = timed(lambda: F.fit_spectra(spectra, path.u, path.d, LAM, EPS, precision="df",
                                                         out=path.layers, ws=ws_s), n=5)
    out["solve_df_all_tiers"] = ws_s.tier_counts()
    # the library's own native FP64 solve at every frequency (a second FP64 reference)
    out["solve_f64_all_ms"] = timed(lambda: F.fit_spectra(spectra, path.u, path.d, LAM, EPS, precision="f64",
                                                          out=path.layers, ws=ws_s), n=2)
    # restore the accurate layers for anything that follows
    F.fit_spectra(spectra, path.u, path.d, LAM, EPS, out=path.layers, ws=ws_s)
    out["render81_ms"] = timed(path.render)
    out["refocus32_ms"] = timed(path.refocus)
    torch.cuda.synchronize()
    return out


def time_latency(path, n=64):
    """Single-image requests, one at a time (view or refocus), device time of each."""
    torch = path.torch
    F = path.F
    rng = np.random.default_rng(1)
    specs = []
    for i in range(n):
        u0 = tuple(rng.uniform(-4, 4, 2))
        if i % 2 == 0:
            specs.append(F.RenderSpec(path.layers, path.d, u0))
        else:
            specs.append(F.RenderSpec(path.layers, path.d, u0, float(rng.uniform(-3, 3)), "disc",
                                      float(rng.uniform(0, 3))))
    reqs = [F.pack_requests([s], path.dev) for s in specs]
    ws = F.workspace(F._lib.load().fdl_refocus_workspace_size(1, C, H, W), path.dev)
    for r in reqs[:4]:
        F.refocus(r, 1, C, H, W, N, ws=ws)
    torch.cuda.synchronize()
    lat = []
    for r in reqs:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        F.refocus(r, 1, C, H, W, N, ws=ws)
        b.record()
        b.synchronize()
        lat.append(a.elapsed_time(b))
    return float(np.percentile(lat, 50)), float(np.percentile(lat, 99))


# ------------------------------------------------------------------ plain FP64 GPU path
class Fp64TorchPath:
    """The plain FP64 one-request-at-a-time comparator: torch complex128 ops on the GPU
    (cuFFT, cuBLAS batched ZGEMM, cuSOLVER batched Cholesky, batched triangular solves)."""

    def __init__(self, device, views, u, d, H_=H, W_=W):
        import torch

        self.torch = torch
        self.dev = device
        self.H, self.W = H_, W_
        self.views = torch.from_numpy(views).to(device).double()
        self.u = torch.from_numpy(u).to(device).double()
        self.d = torch.from_numpy(d).to(device).double()
        ky = torch.fft.fftfreq(H_, device=device, dtype=torch.float64)
        kx = torch.arange(W_ // 2 + 1, device=device, dtype=torch.float64) / W_
        self.wy, self.wx = torch.meshgrid(ky, kx, indexing="ij")

    def fit(self, lam=LAM, eps=EPS, chunk=16384, split=None):
        """Layers [N][C][H][W/2+1] complex128.  split (dict): CUDA-event milliseconds per op."""
        torch = self.torch
        K, Cc = self.views.shape[:2]
        Nl = self.d.numel()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)] if split is not None else None

        def mark(i):
            if ev is not None:
                ev[i].record()

        def acc(name, i, j):
            if ev is not None:
                torch.cuda.synchronize()
                split[name] = split.get(name, 0.0) + ev[i].elapsed_time(ev[j])

        mark(0)
        b = torch.fft.rfft2(self.views).reshape(K, Cc, -1).permute(2, 0, 1)  # [q, K, C]
        mark(1)
        acc("rfft2", 0, 1)
        wy = self.wy.reshape(-1)
        wx = self.wx.reshape(-1)
        x = torch.empty((b.shape[0], Nl, Cc), dtype=torch.complex128, device=self.dev)
        one = torch.ones((), dtype=torch.float64, device=self.dev)
        nfail = 0
        for s in range(0, b.shape[0], chunk):
            sl = slice(s, s + chunk)
            mark(0)
            th = wx[sl, None] * self.u[None, :, 0] + wy[sl, None] * self.u[None, :, 1]
            A = torch.polar(one, 2 * torch.pi * th[:, :, None] * self.d[None, None, :])
            AH = A.conj().transpose(1, 2)
            mark(1)
            w2 = wx[sl] ** 2 + wy[sl] ** 2
            G = AH @ A + torch.diag_embed((lam * (w2[:, None] ** 2 * self.d[None, :] ** 4 + eps)).to(torch.complex128))
            mark(2)
            L, info = torch.linalg.cholesky_ex(G)
            mark(3)
            y = AH @ b[sl]
            mark(4)
            z = torch.linalg.solve_triangular(L, y, upper=False)
            xs = torch.linalg.solve_triangular(L.mH, z, upper=True)
            mark(5)
            bad = info != 0
            if bool(bad.any()):  # not positive definite in FP64: LU with pivoting there
                nfail += int(bad.sum())
                xs[bad] = torch.linalg.solve(G[bad], y[bad])
            x[sl] = xs
            mark(6)
            acc("phase_A", 0, 1)
            acc("gram", 1, 2)
            acc("cholesky", 2, 3)
            acc("rhs", 3, 4)
            acc("triangular_solves", 4, 5)
            acc("fallback", 5, 6)
        if split is not None:
            split["cholesky_failures"] = nfail
        torch.cuda.synchronize()
        return x.permute(1, 2, 0).reshape(Nl, Cc, self.H, self.W // 2 + 1)


def time_fp64_path(device, views, u, d, legs, steps=2):
    import torch

    p = Fp64TorchPath(device, views, u, d)
    X = p.fit()
    t = time.perf_counter()
    for _ in range(steps):
        X = p.fit()
    fit_ms = (time.perf_counter() - t) / steps * 1e3
    split = {}
    p.fit(split=split)
    rng = np.random.default_rng(1)
    lat = []
    r = Fp64Render(device, X.to(torch.complex64), p.d.float())
    for i in range(34):
        u0 = rng.uniform(-4, 4, 2)
        t = time.perf_counter()
        if i % 2 == 0:
            r.render(tuple(u0))
        else:
            r.render(tuple(u0), float(rng.uniform(-3, 3)), float(rng.uniform(0, 3)))
        if i >= 2:
            lat.append((time.perf_counter() - t) * 1e3)
    del p, r
    torch.cuda.empty_cache()
    return {"fit_ms": fit_ms, "fit_mfreq_s": q_half() / fit_ms / 1e3, "fit_split_ms": split,
            "library_f64_solve_ms": legs.get("solve_f64_all_ms"),
            "library_f64_note": "fdl_fit_spectra with FDL_PREC_F64: the library's native FP64 solve of every "
                                "frequency (shared-memory matrix, one warp per frequency), spectra given",
            "render_p50_ms": float(np.percentile(lat, 50)), "render_p99_ms": float(np.percentile(lat, 99)),
            "render_mpix_s": H * W / float(np.mean(lat)) / 1e3}


# ------------------------------------------------------------------ serving form
def serving_leg(device, n_requests=2000, rates=(2000.0, 20000.0), budget=2.5e9, seed=0, fp64_live=300,
                hbm_gbs=None):
    """16 resident FDLs (256^2 / 512^2 / 1024^2 RGB, N in {16, 30, 40}, fitted from 7x7-view
    occluding-plane scenes), Poisson arrivals at each rate, half view renders (u in [-4,4]^2)
    and half refocus (disc or square, radius U(0,3), focus U(-3,3)); a new light field is
    admitted every 500 requests under a byte budget smaller than the 16 FDLs, so admissions
    evict.  Also the same requests all at once (saturation, with the algorithmic-bytes rate
    of the batches against HBM), and the plain FP64 path serving the first `fp64_live`
    requests of the 2k req/s trace one at a time, live, on the same arrival times."""
    import torch

    from paper_1901_06919_gb300.serve import FdlStore, Request, Server
    from scenes import occluding_planes, view_grid

    rng = np.random.default_rng(seed)
    sizes = [256, 512, 1024]
    Ns = [16, 30, 40]
    u7 = view_grid(3)
    U = torch.from_numpy(u7).to(device)
    scenes = {n: torch.from_numpy(occluding_planes(20 + n, n, n, 3, u7)[0]).to(device) for n in sizes}
    store = FdlStore(int(budget), device)
    fit_stream = torch.cuda.Stream(device=device)
    size_of = {}
    evicted = [0]

    def admit(fid):
        n = sizes[fid % 3]
        Nl = Ns[(fid // 3) % 3]
        d = torch.linspace(-3, 3, Nl, device=device)
        before = set(store.entries)
        store.admit(fid, scenes[n], U, d, lam=1e-2, stream=fit_stream)
        evicted[0] += len(before - set(store.entries))
        size_of[fid] = n

    t0 = time.perf_counter()
    for fid in range(16):
        admit(fid)
    fit_stream.synchronize()
    admit_s = time.perf_counter() - t0
    srv = Server(store, sizes=[(n, n, 3) for n in sizes], Nmax=40, capacity=32, pool=96)

    def make_trace(t_gap, n=n_requests):
        tr = []
        t = 0.0
        for i in range(n):
            t += t_gap(i)
            view = i % 2 == 0
            tr.append(Request(i, -1, tuple(rng.uniform(-4, 4, 2)), 0.0 if view else float(rng.uniform(-3, 3)),
                              "pinhole" if view else ("disc" if rng.random() < 0.5 else "square"),
                              0.0 if view else float(rng.uniform(0, 3)), t_arrival=t))
        return tr

    def run(trace, admissions=True):
        next_fid = [max(store.entries) + 1]
        picks = rng.integers(0, 1 << 30, len(trace))
        orig_submit = srv.submit

        def submit(r):
            if admissions and r.rid > 0 and r.rid % 500 == 0:
                try:
                    admit(next_fid[0])
                except Exception:  # every resident FDL in use: no room this time
                    pass
                next_fid[0] += 1
            # requests go to light fields whose fit has finished (a new one is still fitting)
            live = [f for f in store.entries if store.is_ready(f)]
            r.fid = live[int(picks[r.rid]) % len(live)]
            orig_submit(r)

        srv.submit = submit
        b0, l0 = srv.alg_bytes, srv.launches
        try:
            st = srv.run_trace(trace)
        finally:
            srv.submit = orig_submit
        st["batches"] = srv.launches - l0
        st["alg_bytes"] = srv.alg_bytes - b0
        st["mpix_s"] = sum(size_of[r.fid] ** 2 for r in trace) / st["wall_s"] / 1e6
        return st

    run(make_trace(lambda i: 0.0, 64))  # warm-up
    out = {"fdls_admitted": 16, "budget_bytes": int(budget), "admit16_s": admit_s}
    traces = {}
    for rate in rates:
        tr = make_trace(lambda i, r=rate: float(rng.exponential(1.0 / r)))
        traces[rate] = [(r.t_arrival, r.u0, r.s, r.aperture, r.radius) for r in tr]
        st = run(tr)
        traces[rate] = [(a[0], r.fid) + a[1:] for a, r in zip(traces[rate], tr)]
        first = [(r.t_done - r.t_arrival) * 1e3 for r in tr[:fp64_live]]
        st["first_p50_ms"], st["first_p99_ms"] = float(np.percentile(first, 50)), float(np.percentile(first, 99))
        out[f"poisson_{int(rate)}"] = st
    sat = run(make_trace(lambda i: 0.0))
    sat["alg_gbs"] = sat["alg_bytes"] / sat["wall_s"] / 1e9
    if hbm_gbs:
        sat["hbm_frac"] = sat["alg_gbs"] / hbm_gbs
    out["saturation"] = sat
    # the same burst without admissions, each batch's device time recorded: the render's own
    # rate (device time during which a batch ran, the two batch streams overlapping)
    srv.timeline = []
    ren = run(make_trace(lambda i: 0.0), admissions=False)
    ren["busy_ms"] = srv.busy_ms()
    ren["alg_gbs_device"] = ren["alg_bytes"] / (ren["busy_ms"] / 1e3) / 1e9
    ren["requests_per_fdl_per_batch"] = float(np.mean([t[3] for t in srv.timeline])) / len(store.entries)
    srv.timeline = None
    if hbm_gbs:
        ren["hbm_frac_device"] = ren["alg_gbs_device"] / hbm_gbs
    out["saturation_render_only"] = ren
    out["fdls_resident"] = len(store.entries)
    out["fdl_bytes"] = store.bytes_used
    out["evictions"] = evicted[0]
    # the plain FP64 path, one request at a time, live on the same arrivals (first requests of
    # the lowest rate): each request waits for the previous one to finish
    first = traces[rates[0]][:fp64_live]
    renders = {}
    t_start = time.perf_counter()
    lat = []
    pix = 0
    for (ta, fid, u0, s_, ap, rad) in first:
        ta0 = ta - first[0][0]
        while time.perf_counter() - t_start < ta0:
            pass
        if fid not in store.entries:
            continue
        e = store.entries[fid]
        if fid not in renders:
            renders[fid] = Fp64Render(device, e.layers, e.d)
        renders[fid].render(u0, s_, rad if ap != "pinhole" else 0.0, square=(ap == "square"))
        lat.append((time.perf_counter() - t_start - ta0) * 1e3)
        pix += e.H * e.W
    wall = time.perf_counter() - t_start
    del renders
    torch.cuda.empty_cache()
    out["fp64_one_at_a_time_live"] = {"requests": len(lat), "p50_ms": float(np.percentile(lat, 50)),
                                      "p99_ms": float(np.percentile(lat, 99)), "mpix_s": pix / wall / 1e6,
                                      "arrivals": f"first {len(lat)} requests of the {int(rates[0])} req/s trace "
                                                  "(compare poisson_*.first_p50_ms / first_p99_ms)"}
    return out


class Fp64Render:
    """One image of Eq. BsFourier with torch complex128 ops (the plain FP64 path)."""

    def __init__(self, device, layers, d):
        import torch

        self.torch = torch
        self.X = layers.to(torch.complex128)
        self.d = d.double()
        Nl, Cl, Hh, Wh = layers.shape
        self.H, self.W = Hh, 2 * (Wh - 1)
        ky = torch.fft.fftfreq(Hh, device=device, dtype=torch.float64)
        kx = torch.arange(Wh, device=device, dtype=torch.float64) / self.W
        self.wy, self.wx = torch.meshgrid(ky, kx, indexing="ij")

    def render(self, u0, s=0.0, radius=0.0, square=False):
        torch = self.torch
        ph = 2 * torch.pi * self.d[:, None, None] * (u0[0] * self.wx + u0[1] * self.wy)[None]
        coef = torch.polar(torch.ones((), dtype=torch.float64, device=self.X.device), ph)
        if radius > 0 and square:
            sd = (s - self.d)[:, None, None]
            coef = coef * torch.sinc(2 * radius * sd * self.wx[None]) * torch.sinc(2 * radius * sd * self.wy[None])
        elif radius > 0:
            z = 2 * torch.pi * radius * ((s - self.d)[:, None, None] * torch.sqrt(self.wx ** 2 + self.wy ** 2)[None]).abs()
            safe = torch.where(z == 0, torch.ones_like(z), z)
            coef = coef * torch.where(z == 0, torch.ones_like(z), 2 * torch.special.bessel_j1(safe) / safe)
        img = torch.fft.irfft2((coef[:, None] * self.X).sum(0), s=(self.H, self.W))
        torch.cuda.synchronize()
        return img


# ------------------------------------------------------------------ precision form
# The paper's own light-field shapes (Sec. VII timing table; Matlab on a GTX 1080, context only):
# name, (H, W), view grid half-width, layer construction s, render ms
PAPER_SHAPES = [("Fruits 625x434x9x9", (434, 625), 4, 0.9, 12.0),
                ("Totoro WaterFall 379x379x7x7", (379, 379), 3, 0.4, 7.0),
                ("Chess Pieces 1920x1080x5x5", (1080, 1920), 2, 4.3, 53.0)]


def shapes_leg(device, reps=3):
    """Fit (DFT + tiers) and single-view render at the paper's sizes that are not powers of
    two, RGB, N = 30 layers on linspace(-3, 3), lambda = 1e-2, synthetic occluding planes."""
    import torch

    import paper_1901_06919_gb300 as F
    from scenes import occluding_planes, view_grid

    out = {}
    for name, (H, W), g, paper_fit_s, paper_render_ms in PAPER_SHAPES:
        u = view_grid(g)
        d = np.linspace(-3, 3, N).astype(np.float32)
        views, _ = occluding_planes(11, H, W, C, u)
        V, U, D = (torch.from_numpy(a).to(device) for a in (views, u, d))
        x, ws = F.fit(V, U, D, LAM, EPS)
        u0 = torch.tensor([[0.3, -0.2]], dtype=torch.float32, device=device)
        img = F.render(x, D, u0, W=W)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            F.fit(V, U, D, LAM, EPS, out=x, ws=ws)
        b.record()
        torch.cuda.synchronize()
        fit_ms = a.elapsed_time(b) / reps
        a.record()
        for _ in range(10):
            F.render(x, D, u0, out=img, W=W)
        b.record()
        torch.cuda.synchronize()
        render_ms = a.elapsed_time(b) / 10
        q = H * (W // 2 + 1)
        out[name] = {"fit_ms": fit_ms, "fit_mfreq_s": q / fit_ms / 1e3, "render_ms": render_ms,
                     "tiers": ws.tier_counts(), "paper_gtx1080_fit_ms": paper_fit_s * 1e3,
                     "paper_gtx1080_render_ms": paper_render_ms}
        del V, x, ws, img
        torch.cuda.empty_cache()
    return out


def precision_bins(n, nrand=45, seed=5):
    """64 sampled bins of an n x n spectrum: DC, the lowest rings (worst conditioned), the
    Nyquist row and column, seeded random bins."""
    low = [(0, 0), (0, 1), (1, 0), (1, 1), (n - 1, 1), (0, 2), (2, 0), (2, 1), (1, 2), (n - 1, 2), (n - 2, 1)]
    h = n // 2
    nyq = [(h, 0), (h, 1), (h, 100), (h, h), (0, h), (1, h), (300, h), (n - 1, h)]
    rng = np.random.default_rng(seed)
    rand = list(zip(rng.integers(0, n, nrand).tolist(), rng.integers(0, h + 1, nrand).tolist()))
    b = low + nyq + rand
    return np.array([q[0] for q in b]), np.array([q[1] for q in b])


def precision_leg(device, lams=(1e-3, 1e-2, 1e-1)):
    """7x7 views, 1024x1024 RGB, N=40 on linspace(-4, 4), per lambda: the certified mixed fit's
    time and tiers; its layers against the plain FP64 GPU path (torch complex128) and the
    library's native FP64 solve at every frequency, and against the FP64 oracle at 64 sampled
    frequencies (the oracle's inputs from its own direct DFT of the views); and the rendered
    max abs error of two views and two refocused images against the FP64 path's render of its
    FP64 layers."""
    import torch

    import paper_1901_06919_gb300 as F
    from oracle import fdl_oracle as O
    from scenes import occluding_planes, view_grid

    u = view_grid(3)
    d = np.linspace(-4, 4, 40).astype(np.float32)
    n = 1024
    views, _ = occluding_planes(7, n, n, 3, u)
    V, U, D = (torch.from_numpy(a).to(device) for a in (views, u, d))
    ky, kx = precision_bins(n)
    b = np.stack([O.dft_at_bins(views[j].astype(np.float64), ky, kx) for j in range(views.shape[0])])
    kyt, kxt = torch.from_numpy(ky).to(device), torch.from_numpy(kx).to(device)
    p64 = Fp64TorchPath(device, views, u, d, n, n)
    renders = [((0.0, 0.0), 0.0, "pinhole", 0.0), ((2.5, -1.5), 0.0, "pinhole", 0.0),
               ((0.5, 0.5), -1.0, "disc", 1.0), ((0.0, 0.0), 2.0, "square", 2.0)]
    out = {}
    for lam in lams:
        x, ws = F.fit(V, U, D, lam)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record()
        F.fit(V, U, D, lam, out=x, ws=ws)
        e.record()
        torch.cuda.synchronize()
        fit_ms = a.elapsed_time(e)
        tiers = ws.tier_counts()
        t = time.perf_counter()
        X64 = p64.fit(lam)
        fp64_ms = (time.perf_counter() - t) * 1e3
        x64lib, _ = F.fit(V, U, D, lam, precision="f64")
        nrm = torch.linalg.vector_norm(X64).item()
        rel_fp64 = torch.linalg.vector_norm(x.to(torch.complex128) - X64).item() / nrm
        rel_lib64 = torch.linalg.vector_norm(x64lib.to(torch.complex128) - X64).item() / nrm
        ref = O.solve_bins(np.moveaxis(b, -1, 0), u, d.astype(np.float64), O.freq_y(n)[ky], kx / n, lam, 1e-4)
        got = np.moveaxis(x[:, :, kyt, kxt].cpu().numpy(), -1, 0)
        got64 = np.moveaxis(X64[:, :, kyt, kxt].cpu().numpy(), -1, 0)
        r64 = Fp64Render(device, X64, D)
        pix = 0.0
        for (u0, s_, ap, rad) in renders:
            if ap == "pinhole":
                ours = F.render(x, D, torch.tensor([u0], dtype=torch.float32, device=device))[0]
            else:
                ours = F.refocus_specs([F.RenderSpec(x, D, u0, s_, ap, rad)])[0]
            ref_img = r64.render(u0, s_, rad, square=(ap == "square"))
            pix = max(pix, torch.max(torch.abs(ours.double() - ref_img)).item())
        del r64, X64, x64lib
        torch.cuda.empty_cache()
        out[str(lam)] = {"fit_ms": fit_ms, "fit_mfreq_s": n * (n // 2 + 1) / fit_ms / 1e3, "tiers": tiers,
                         "layer_rel_l2_vs_fp64_gpu_path": rel_fp64,
                         "library_f64_layer_rel_l2_vs_fp64_gpu_path": rel_lib64,
                         "layer_rel_l2_vs_oracle_64_bins": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                         "fp64_gpu_path_vs_oracle_64_bins": float(np.linalg.norm(got64 - ref) / np.linalg.norm(ref)),
                         "render_max_abs_vs_fp64_gpu_path": pix, "fp64_gpu_path_fit_ms": fp64_ms}
    del p64
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ differentiation form
def calib_leg(device, steps=200):
    """5x5 views jittered by U(+-0.15), 256x256 gray, 12 true disparities U(-2, 2); 200 Adam
    steps from the grid and linspace(-2, 2, 12) on 4096-frequency subsets."""
    import torch

    import paper_1901_06919_gb300 as F
    from paper_1901_06919_gb300.calib import calibrate
    from scenes import layered_scene, view_grid

    rng = np.random.default_rng(0)
    u_true = view_grid(2).astype(np.float64) + rng.uniform(-0.15, 0.15, (25, 2))
    d_true = np.sort(rng.uniform(-2, 2, 12))
    views, _ = layered_scene(1, 256, 256, 1, u_true.astype(np.float32), d_true.astype(np.float32), sigma=0.0)
    S = F.rfft2(torch.from_numpy(views).to(device))
    u0 = torch.from_numpy(view_grid(2)).to(device)
    d0 = torch.linspace(-2, 2, 12, device=device)
    calibrate(S, u0, d0, steps=3)
    torch.cuda.synchronize()
    t = time.perf_counter()
    res = calibrate(S, u0, d0, steps=steps, lr=1e-2, subset=4096)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    a = res.u.cpu().numpy().astype(np.float64)
    a -= a.mean(0)
    tt = u_true - u_true.mean(0)
    c = (a * tt).sum() / (a * a).sum()
    g = view_grid(2).astype(np.float64)
    g -= g.mean(0)
    c0 = (g * tt).sum() / (g * g).sum()
    return {"steps": steps, "steps_per_s": steps / dt, "loss_first": res.losses[0], "loss_last": res.losses[-1],
            "u_rms_err_init": float(np.sqrt(((c0 * g - tt) ** 2).mean())),
            "u_rms_err_final": float(np.sqrt(((c * a - tt) ** 2).mean()))}

# ------------------------------------------------------------------ oracle on the host
# The FP64 oracle timed on the host cores on a bounded sample of the step, in processes
# started with `spawn` (one BLAS thread each): every worker runs the same share of each stage
# (the DFT of some view images, the solve at some frequencies, some renders); the stage's wall
# time over the pool, scaled by (units of the full step / units of the sample), estimates
# the full step.
_ORACLE = {}


def _oracle_init(seed):
    from scenes import random_layer_spectra

    # render inputs: generated in the worker (not timed); the oracle's time does not depend on values
    _ORACLE["X"] = random_layer_spectra(seed, N, C, H, W).astype(np.complex128)


def _oracle_task(task):
    from oracle import fdl_oracle as O

    kind = task[0]
    t = time.perf_counter()
    if kind == "dft":
        O.half_spectrum(task[1])
    elif kind == "solve":
        _, b, u, d, wy, wx = task
        O.solve_bins(b, u, d, wy, wx, LAM, EPS)
    else:
        _, renders, d = task
        for (u0, s_, ap, rad) in renders:
            O.render(_ORACLE["X"], d, u0, s_, ap, rad)
    return time.perf_counter() - t


class OracleSample:
    """A pool of `workers` spawned processes, each taking img images, bins frequencies and
    renders renders of the step per sample."""

    def __init__(self, views, u, d, s_list, workers, img, bins, renders):
        import multiprocessing as mp

        from oracle import fdl_oracle as O

        self.workers, self.img, self.bins, self.renders = workers, img, bins, renders
        K = views.shape[0]
        flat = views.reshape(K * C, H, W)
        rng = np.random.default_rng(0)
        self.dft_tasks = [("dft", flat[(np.arange(img) + w * img) % (K * C)].astype(np.float64)) for w in range(workers)]
        wy, wx = O.half_grid(H, W)
        sel = rng.choice(len(wy), min(workers * bins, len(wy)), replace=False)
        # solve inputs: the views' spectra at the sampled bins (numpy's FFT; values do not change the time)
        spec = np.fft.rfft2(views.astype(np.float64)).reshape(K, C, -1)[:, :, sel]  # [K][C][nb]
        b = np.moveaxis(spec, -1, 0)
        d64 = d.astype(np.float64)
        self.solve_tasks = [("solve", b[w * bins:(w + 1) * bins], u, d64, wy[sel][w * bins:(w + 1) * bins],
                             wx[sel][w * bins:(w + 1) * bins]) for w in range(workers)]
        kinds = []
        for r in range(workers * renders):
            if r % 2 == 0:
                kinds.append((tuple(map(float, u[r % K])), 0.0, O.AP_PINHOLE, 0.0))
            else:
                kinds.append(((0.0, 0.0), float(s_list[r % len(s_list)]), O.AP_DISC, 1.0))
        self.render_tasks = [("render", kinds[w * renders:(w + 1) * renders], d64) for w in range(workers)]
        env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in env:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(workers, initializer=_oracle_init, initargs=(5,))
        finally:
            for k, v in env.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def run(self):
        out = {}
        for name, tasks in (("dft", self.dft_tasks), ("solve", self.solve_tasks), ("render", self.render_tasks)):
            t = time.perf_counter()
            self.pool.map(_oracle_task, tasks, chunksize=1)
            out[name + "_s"] = time.perf_counter() - t
        units = {"dft": self.workers * self.img, "solve": self.workers * self.bins, "render": self.workers * self.renders}
        full = {"dft": (2 * GRID + 1) ** 2 * C, "solve": q_half(), "render": (2 * GRID + 1) ** 2 + N_REFOCUS}
        out["sample_s"] = out["dft_s"] + out["solve_s"] + out["render_s"]
        out["estimated_step_s"] = sum(out[k + "_s"] * full[k] / units[k] for k in units)
        out["units"] = units
        return out

    def close(self):
        self.pool.close()
        self.pool.join()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(views, u, d, s_list):
    """The oracle at 1 core and at every host core, each on a bounded sample."""
    res = {}
    P = host_cores()
    for label, workers, img, bins, ren in (("cores_1", 1, 8, 4096, 4), ("cores_all", P, 8, 4096, 2)):
        smp = OracleSample(views, u, d, s_list, workers, img, bins, ren)
        try:
            r = smp.run()
        finally:
            smp.close()
        r["cores"] = workers
        r["mfreq_s"] = q_half() / r["estimated_step_s"] / 1e6
        res[label] = r
    a = res["cores_all"]
    return {"value": a["mfreq_s"], "unit": "Mfreq/s", "cores": P, "kind": "oracle",
            "sample": f"FP64 oracle (numpy, one BLAS thread per process) on {P} spawned processes, each taking "
                      "8 of the 243 view images (DFT), 4096 of the 131584 frequencies (solve) and 2 of the 113 "
                      "images (render); each stage's wall time scaled to the full step (an estimate: "
                      f"{a['sample_s']:.1f} s sampled of an estimated {a['estimated_step_s']:.0f} s step); "
                      "cores_1: the same with 4 renders on one process",
            "cores_1": res["cores_1"], "cores_all": a}


# ------------------------------------------------------------------ main
def max_over_ranks(value: float, device=None) -> float:
    """The slowest rank's time: every rank contributes its own, all receive the maximum."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Units processed by all ranks per second, in millions, over the slowest rank's time."""
    return world * units_per_rank / (ms / 1e3) / 1e6


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def run_reference(args, world, rank):
    """The oracle as the reference arm: each step a bounded sample (every host core, one
    spawned process per core), value = frequencies / estimated full-step time."""
    if rank != 0:
        return
    views, u, d, s_list = workload_inputs()
    P = host_cores()
    smp = OracleSample(views, u, d, s_list, P, 2, 1024, 1)
    try:
        for _ in range(args.warmup):
            smp.run()
        runs = [smp.run() for _ in range(args.steps)]
    finally:
        smp.close()
    est_ms = float(np.mean([r["estimated_step_s"] for r in runs])) * 1e3
    sample_ms = float(np.mean([r["sample_s"] for r in runs])) * 1e3
    val = q_half() / (est_ms / 1e3) / 1e6
    sample = (f"per step: FP64 oracle on {P} spawned processes (one per host core), each taking 2 of the 243 "
              "view images (DFT), 1024 of the 131584 frequencies (solve) and 1 of the 113 images (render); "
              f"ms_per_step is the sample's wall time, value uses the estimated full step ({est_ms:.0f} ms)")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mfreq/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sample_ms,
            "estimated_full_step_ms": est_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": val, "unit": "Mfreq/s", "cores": P, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "Mfreq/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fdl", choices=["fdl", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline leg")
    ap.add_argument("--no-fp64", action="store_true", help="skip the torch FP64 comparator leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-precision", action="store_true", help="skip the 1024x1024 precision leg")
    ap.add_argument("--no-shapes", action="store_true", help="skip the leg at the paper's non-power-of-two sizes")
    ap.add_argument("--no-calib", action="store_true", help="skip the calibration leg")
    ap.add_argument("--case", default=None, choices=sorted(CASES),
                    help="run one bounded case twice and exit (for profiler captures)")
    args = ap.parse_args()
    if args.case:
        CASES[args.case]()
        return
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch

    from paper_1901_06919_gb300 import build as B

    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    views, u, d, s_list = workload_inputs()
    path = FdlPath(device, views, u, d, s_list)

    clocks = ClockSampler(local)
    for _ in range(args.warmup):
        path.step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks.start()
    total_ms, stages = time_device_steps(path, args.steps, 0)
    clk = clocks.stop()
    total_ms = max_over_ranks(total_ms, device)
    ms = total_ms / args.steps
    value = whole_job_rate(q_half(), world, ms)

    views_host = torch.from_numpy(views).pin_memory()
    e2e_ms, h2d, d2h = time_e2e(path, views_host, max(4, args.steps), 2)
    e2e_ms = max_over_ranks(e2e_ms, device)
    legs = time_kernel_legs(path)
    p50, p99 = time_latency(path)
    # kernels per step (the ncu launch list of --case step): fit = 2 twiddle tables + rows +
    # cols + exp table + moment check + FP32 view sums + FP32 solve + 3 selection + 2
    # double-float solves (one exits at once) + 3 selection + FP64 solve + status = 17;
    # fdl_render = requests + render +
    # column and row passes = 4; fdl_refocus = plan + 4 launches of the mixed path (return at
    # once) + render + column and row passes = 8
    launches = 17 + 4 + 8

    fit_ms = stages["fit_ms"]
    render_ms = stages["render81_ms"] + stages["refocus32_ms"]
    # roofline: the high-precision solve (dominant kernel) on the method's flops; the DFT and
    # render stages against HBM
    rl = roofline_entry(legs, clk, moment_form_applies(u, d))
    stage_rl = stage_rooflines(legs, clk)
    line = {
        "metric": METRIC, "value": value, "unit": "Mfreq/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+df", "data": "synthetic",
        "config": {"workload": WORKLOAD, "frequencies_per_step": q_half(), "images_per_step": 113,
                   "l2": "inputs larger than L2 (views 255 MB per step)", "parallelism": f"replicas x{world}"},
        "stages": {"fit_ms": fit_ms, "fit_mfreq_s": q_half() / fit_ms / 1e3,
                   "render81_ms": stages["render81_ms"], "refocus32_ms": stages["refocus32_ms"],
                   "render_mpix_s": pix_per_step(113) / render_ms / 1e3},
        "legs": legs,
        "latency": {"render_p50_ms": p50, "render_p99_ms": p99, "requests": 64, "mode": "one at a time"},
        "e2e": {"value": world * q_half() / (e2e_ms / 1e3) / 1e6, "unit": "Mfreq/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "api": "fdl_fit_render_host (C ABI: views from pinned host memory, fit, 113 renders, images back to "
                       "pinned host memory), rotating over three streams and three device slots"},
        "gpu_launches": launches * args.steps,
        "clocks": clk,
        "roofline": rl,
        "roofline_stages": stage_rl,
    }
    if rank == 0 and not args.no_fp64:
        try:
            line["fp64_gpu_path"] = time_fp64_path(device, views, u, d, legs)
        except Exception as e:  # reported, not hidden
            line["fp64_gpu_path"] = {"error": repr(e)[:200]}
    def leg(name, fn):
        try:
            line[name] = fn()
        except Exception as e:  # reported, not hidden
            line[name] = {"error": repr(e)[:300]}
        torch.cuda.empty_cache()

    if rank == 0 and not args.no_serve:
        del path
        torch.cuda.empty_cache()
        hbm, src = measured_hbm()
        leg("serving", lambda: serving_leg(device, hbm_gbs=hbm))
    if rank == 0 and not args.no_serve and "error" not in line["serving"]:
        sat = line["serving"]["saturation_render_only"]
        line["roofline_stages"].append({"stage": "serving render at saturation (2,000 mixed-size requests at once, "
                                                 "batches of up to 32)",
                                        "kernel": "k_render_plan + k_render_grp + k_cols_req (x2) + "
                                                  "k_irfft_rows_req (+ the tiled passes, gated off)", "bound": "hbm",
                                        "achieved": sat["alg_gbs_device"], "peak": hbm, "unit": "GB/s",
                                        "frac": sat["alg_gbs_device"] / hbm, "algorithmic_bytes": sat["alg_bytes"],
                                        "traffic": None, "peak_source": src, "ms": sat["busy_ms"],
                                        "note": "device time of the batches (union of their intervals); "
                                                "algorithmic bytes: each FDL of a batch read once, each image "
                                                "written once"})
        line["latency"]["serving_p50_ms"] = line["serving"]["poisson_2000"]["p50_ms"]
        line["latency"]["serving_p99_ms"] = line["serving"]["poisson_2000"]["p99_ms"]
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_precision:
        leg("precision", lambda: precision_leg(device))
    if rank == 0 and not args.no_shapes:
        leg("paper_shapes", lambda: shapes_leg(device))
    if rank == 0 and not args.no_calib:
        leg("calibration", lambda: calib_leg(device))
    if rank == 0 and not args.no_cpu:
        leg("cpu_baseline", lambda: cpu_baseline(views, u, d, s_list))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def moment_form_applies(u, d):
    """The device-side test of the solve: 2 pi (spread of d about its grid) max|u| / sqrt(2) <= 1e-4."""
    d = np.asarray(d, np.float64)
    n = len(d)
    delta = float(np.float32((np.float32(d[-1]) - np.float32(d[0])) / np.float32(n - 1))) if n > 1 else 0.0
    e = d - d[0] - np.arange(n) * delta
    umax = float(np.max(np.hypot(u[:, 0], u[:, 1])))
    return 2 * np.pi * (e.max() - e.min()) * umax / np.sqrt(2) <= 1e-4


# Algorithmic flops per frequency of an FP32 solve with a Toeplitz Gram (9x9 views, N = 30, RGB):
# Gram 14.6k, A 14.6k, right-hand side 58.3k, Cholesky 36k, solves 21.6k.
FP32_METHOD_FLOPS_PER_FREQUENCY = 145_000

# From an ncu capture of the all-frequency k_solve_df<30, 15, moment form> launch (bench.py
# --case df512): DRAM bytes (read + write) and warp instructions per frequency.  The algorithmic
# bytes are the K x C spectrum values read and the N x C layer values written, 8 bytes each:
# 2,664 per frequency.
DF_DRAM_BYTES_PER_FREQUENCY = (270.752e6 + 79.548672e6) / 131_584
DF_WARP_INSTRUCTIONS_PER_FREQUENCY = 9_554_976_035 / 131_584
# The FP32 solve (k_f32_sums + k_solve_f32<32>, the pass with estimates, bench.py --case step):
# DRAM bytes per pass over all 131,584 frequencies (the view sums go through workspace scratch).
F32_DRAM_BYTES = (256.081408e6 + 163.084544e6) + (203.742464e6 + 64.532992e6)


# ------------------------------------------------------------------ bounded cases for profilers
def _case_device():
    import torch

    from paper_1901_06919_gb300 import build as B

    B.build()
    return torch, torch.device("cuda", 0)


def case_df512():
    """The double-float solve of every frequency of the 9x9-view 512x512 RGB workload, twice."""
    torch, dev = _case_device()
    import paper_1901_06919_gb300 as F

    views, u, d, _ = workload_inputs()
    S = F.rfft2(torch.from_numpy(views).to(dev))
    U, D = torch.from_numpy(u).to(dev), torch.from_numpy(d).to(dev)
    for _ in range(2):
        x, ws = F.fit_spectra(S, U, D, LAM, EPS, precision="df")
    torch.cuda.synchronize()
    print(json.dumps({"case": "df512", "tiers": ws.tier_counts()}))


def case_render81():
    """fdl_render of the 81 input views from the layers of the 9x9-view workload, twice."""
    torch, dev = _case_device()
    import paper_1901_06919_gb300 as F

    views, u, d, _ = workload_inputs()
    U, D = torch.from_numpy(u).to(dev), torch.from_numpy(d).to(dev)
    x, _ = F.fit(torch.from_numpy(views).to(dev), U, D, LAM, EPS)
    for _ in range(2):
        img = F.render(x, D, U)
    torch.cuda.synchronize()
    print(json.dumps({"case": "render81", "shape": list(img.shape)}))


def case_mixed_batch():
    """fdl_refocus over 24 requests of three FDLs of 256^2, 512^2 and 1024^2 RGB (N = 16, 30, 40;
    views, discs and squares): twice with the FDLs interleaved (every request its own group of
    the mixed render), then twice sorted by FDL (groups of 8)."""
    torch, dev = _case_device()
    import paper_1901_06919_gb300 as F
    from scenes import random_layer_spectra

    rng = np.random.default_rng(0)
    fdls = []
    for i, (n, Nl) in enumerate(((256, 16), (512, 30), (1024, 40))):
        X = torch.from_numpy(random_layer_spectra(i, Nl, 3, n, n)).to(dev)
        fdls.append((X, torch.linspace(-3, 3, Nl, device=dev)))
    specs = []
    for i in range(24):
        X, dd = fdls[i % 3]
        kind = ("pinhole", "disc", "square")[i % 3]
        specs.append(F.RenderSpec(X, dd, tuple(rng.uniform(-4, 4, 2)), float(rng.uniform(-3, 3)), kind,
                                  0.0 if kind == "pinhole" else float(rng.uniform(0.5, 3))))
    ordered = [specs[i] for k in range(3) for i in range(k, 24, 3)]
    for batch in (specs, specs, ordered, ordered):
        F.refocus_specs(batch)
    torch.cuda.synchronize()
    print(json.dumps({"case": "mixed_batch", "requests": len(specs)}))


def case_step():
    """Three warm-up steps and two steps of the benchmark (fit + 81 views + 32 refocused images)."""
    torch, dev = _case_device()
    views, u, d, s_list = workload_inputs()
    path = FdlPath(dev, views, u, d, s_list)
    for _ in range(5):
        path.step()
    torch.cuda.synchronize()
    print(json.dumps({"case": "step", "tiers": path.F.FitWorkspace.tier_counts(path.ws_fit)}))


def case_refocus32():
    """The 32 disc-aperture refocused images of the benchmark step, twice, after the fit."""
    torch, dev = _case_device()
    views, u, d, s_list = workload_inputs()
    path = FdlPath(dev, views, u, d, s_list)
    for _ in range(2):
        path.refocus()
    torch.cuda.synchronize()
    print(json.dumps({"case": "refocus32"}))


def case_latency():
    """Sixteen single-image requests (views and discs), one at a time, after the fit: the
    latency leg's launches."""
    torch, dev = _case_device()
    views, u, d, s_list = workload_inputs()
    path = FdlPath(dev, views, u, d, s_list)
    p50, p99 = time_latency(path, n=16)
    print(json.dumps({"case": "latency", "p50_ms": p50, "p99_ms": p99}))


CASES = {"df512": case_df512, "render81": case_render81, "mixed_batch": case_mixed_batch, "refocus32": case_refocus32,
         "latency": case_latency, "step": case_step}


def measured_hbm():
    """HBM copy bandwidth of the GB300s (driver-measured), else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"


def roofline_entry(legs, clk, moment):
    """The dominant kernel is the double-float solve (launch list), bound by the FP32 pipe.
    achieved = the method's own flops (an FP32 solve with a Toeplitz Gram: 145 kflop per
    frequency on this workload) per second of the all-frequency double-float launch; peak =
    152 SMs x 128 FP32 lanes x 2 flop per FMA x the median SM clock sampled in the run.
    issue_frac: the warp instructions the kernel issues (ncu count per frequency) per second of
    the same launch against the 4 issue slots of each SM per cycle: the double-float
    arithmetic's own bound."""
    ms = legs["solve_df_all_ms"]
    mhz = clk.get("sm_mhz") or 2070.0
    peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
    achieved = FP32_METHOD_FLOPS_PER_FREQUENCY * q_half() / (ms / 1e3) / 1e12
    wi = DF_WARP_INSTRUCTIONS_PER_FREQUENCY if moment else None
    form = "moment-form Gram" if moment else "direct Gram"
    return {"kernel": f"k_solve_df (double-float per-frequency solve, {form}, all 131,584 frequencies)",
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": DF_DRAM_BYTES_PER_FREQUENCY * q_half() if (moment and DF_DRAM_BYTES_PER_FREQUENCY) else None,
            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "algorithmic_bytes": ((2 * GRID + 1) ** 2 + N) * C * 8 * q_half(),
            "peak_source": f"152 SMs x 128 FP32 lanes x 2 flop (FMA) x {mhz:.0f} MHz (median SM clock in the run)",
            "method_flops_per_frequency": FP32_METHOD_FLOPS_PER_FREQUENCY,
            "warp_instructions_per_frequency": wi,
            "issue_frac": wi * q_half() / (ms / 1e3) / (152 * 4 * mhz * 1e6) if wi else None}


def roofline_hbm(stage, kernel, alg_bytes, ms, traffic=None):
    hbm, src = measured_hbm()
    ach = alg_bytes / (ms / 1e3) / 1e9
    return {"stage": stage, "kernel": kernel, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": ach / hbm, "algorithmic_bytes": alg_bytes, "traffic": traffic, "ms": ms, "peak_source": src}


def stage_rooflines(legs, clk):
    """The FP32 solve against the FP32 pipe (method flops as in roofline_entry), and the HBM
    roofline of the forward DFT and of the renders (algorithmic bytes: every input read once,
    every output written once).  The 81 views and the 32 refocused images each read one FDL,
    so the device gate sends them to the tiled path (render, inverse column pass, row pass)."""
    K = (2 * GRID + 1) ** 2
    img = C * H * W * 4
    layers = N * C * q_half() * 8
    mhz = clk.get("sm_mhz") or 2070.0
    peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
    f32 = FP32_METHOD_FLOPS_PER_FREQUENCY * q_half() / (legs["solve_f32_all_ms"] / 1e3) / 1e12
    tiled = "k_render + k_fft_cols<inverse> + k_irfft_rows"
    return [{"stage": "FP32 solve of every frequency (no estimate)", "kernel": "k_f32_sums + k_solve_f32<32>",
             "bound": "alu",
             "achieved": f32, "peak": peak, "unit": "TFLOP/s", "frac": f32 / peak,
             "ms": legs["solve_f32_all_ms"], "traffic": F32_DRAM_BYTES,
             "algorithmic_bytes": (K + N) * C * 8 * q_half(),
             "peak_source": f"152 SMs x 128 FP32 lanes x 2 flop (FMA) x {mhz:.0f} MHz"},
            roofline_hbm("forward DFT of the 243 view images", "k_rfft_rows_df + k_fft_cols_df",
                         K * img + K * C * q_half() * 8, legs["rfft2_ms"], DFT_DRAM_BYTES),
            roofline_hbm("render of the 81 input views", tiled, layers + K * img, legs["render81_ms"],
                         RENDER81_DRAM_BYTES),
            roofline_hbm("32 refocused images (disc)", tiled, layers + N_REFOCUS * img, legs["refocus32_ms"],
                         REFOCUS32_DRAM_BYTES)]


# DRAM bytes (read + write) per launch from ncu captures of the current kernels (None: not
# captured), all from bench.py --case render81: the forward DFT's two passes, and the tiled
# render of the 81 views (k_render, the inverse column pass, the row pass).
DFT_DRAM_BYTES = (254.848e6 + 209.98144e6) + (254.979328e6 + 197.8944e6)
RENDER81_DRAM_BYTES = (99.271936e6 + 198.1056e6) + (255.84896e6 + 190.7136e6) + (254.875136e6 + 206.172672e6)
# the 32 refocused images (the same three kernels, bench.py --case refocus32)
REFOCUS32_DRAM_BYTES = (98.184704e6 + 55.065088e6) + (101.079296e6 + 42.461952e6) + (100.725248e6 + 52.825088e6)


if __name__ == "__main__":
    main()
