// C ABI of libfdl: argument checks, workspace carving and kernel order.
// Every function returns an FDL_* status and never throws or aborts.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "kernels.h"

using namespace fdl;

namespace {

constexpr size_t kAlign = 256;
// Error of the double-float solve per unit of (condition estimate x solution norm),
// per square root of the number of views.  The Gram matrix and the right-hand side
// are sums over the K views whose terms are nearly equal at the low, worst-conditioned
// frequencies, so the rounding of the running sum grows like sqrt(K) in relative
// terms.  Measured against extended-precision solutions at the frequencies with the
// largest errors (kappa ~ 1e10): error / (kappa |x|) ~ 1.9e-15 at K = 49, 2.5e-15 at
// K = 81 and 8e-15 at K = 361; 1.0e-16 sqrt(K) keeps the estimate at or above the
// error of the layers over 49 to 361 views.
constexpr double kDfUnitPerSqrtView = 1.0e-16;
// Error of the FP32 solve per unit of (condition estimate x solution norm), about
// 4 times the FP32 unit roundoff: the high quantiles of measured error / (kappa |x|).
constexpr double kF32Unit = 4.5e-7;

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

bool pow2_shape(int H, int W) { return pow2_in(H, 16, 4096) && pow2_in(W, 16, 4096); }

// Powers of two use the radix-4/2 DFT kernels and the split spectrum layout; other sizes
// (16..4096, see gen_supported) the general-length kernels and the dense layout.
bool shape_ok(int H, int W) {
  if (pow2_shape(H, W)) return true;
  return H >= 16 && W >= 16 && H <= 4096 && W <= 4096 && gen_supported(H) && gen_supported(W);
}

// Plans of the general-length DFTs, their tables one after the other (H first).
struct GenPlans {
  GenPlan ph, pw;
  size_t elems;
};
GenPlans gen_plans(int H, int W) {
  GenPlans g;
  gen_plan(H, 0, &g.ph);
  gen_plan(W, g.ph.elems, &g.pw);
  g.elems = (size_t)g.ph.elems + g.pw.elems;
  return g;
}
// float4 entries of DFT tables a forward transform of an H x W image needs
size_t dft_table_elems(int H, int W) { return pow2_shape(H, W) ? (size_t)H + W : gen_plans(H, W).elems; }
// ... and an inverse one (the power-of-two inverse kernels need none)
size_t inv_table_elems(int H, int W) { return pow2_shape(H, W) ? 0 : gen_plans(H, W).elems; }

cudaError_t launch_gen_tables2(const GenPlans& g, float4* tables, cudaStream_t st) {
  cudaError_t e = launch_gen_tables(g.ph, tables, st);
  if (e == cudaSuccess) e = launch_gen_tables(g.pw, tables, st);
  return e;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? FDL_OK : FDL_ECUDA; }

struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* p) : base(static_cast<char*>(p)) {}
  template <class T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += align_up(count * sizeof(T));
    return p;
  }
};

// Fit workspace: counters first (fdl_fit_tier_counts finds them there).
struct FitWs {
  int* counters;
  float4* exp_table;
  float4* fft_tables;
  float2* mom;  // kMomSlots: disparity grid deviations for the moment-form Gram
  int* flagged;
  int* flagged64;
  float* err;
  float* xn2;
  void* select;
  float2* spec_main;
  float2* spec_nyq;
  float4* f32sums = nullptr;  // scratch of the FP32 solve's moment-form view sums (N <= 32)
  int f32sums_tiles = 0;
  size_t bytes;
};

FitWs carve_fit(void* ws, int K, int C, int H, int W, int N, bool with_spectra, bool sums = true) {
  Carver cv(ws);
  FitWs f;
  f.counters = cv.take<int>(kHeaderInts);
  f.exp_table = cv.take<float4>(1024);
  f.fft_tables = cv.take<float4>(dft_table_elems(H, W));
  f.mom = cv.take<float2>(kMomSlots);
  f.flagged = cv.take<int>((size_t)H * (W / 2 + 1));
  f.flagged64 = cv.take<int>((size_t)H * (W / 2 + 1));
  f.err = cv.take<float>((size_t)H * (W / 2 + 1));
  f.xn2 = cv.take<float>((size_t)H * (W / 2 + 1));
  f.select = cv.take<char>(select_scratch_bytes());
  if (sums && N <= 32) {
    // the view sums of up to kF32SumsTiles tiles of 8 frequencies at a time
    const int tiles = (int)std::min<long long>(((long long)H * (W / 2 + 1) + 7) / 8, kF32SumsTiles);
    f.f32sums_tiles = tiles;
    f.f32sums = cv.take<float4>((size_t)tiles * 8 * 32 * 3);  // float4 (W_0, W_1) + 4 float2 per lane
  }
  if (with_spectra) {
    f.spec_main = cv.take<float2>((size_t)K * C * H * (W / 2));
    f.spec_nyq = cv.take<float2>((size_t)K * C * H);
  } else {
    f.spec_main = f.spec_nyq = nullptr;
  }
  f.bytes = cv.off;
  return f;
}

int check_fit_args(int K, int C, int H, int W, int N, const fdl_fit_opts* o) {
  if (K < 1 || K > 1024 || C < 1 || C > 4 || N < 1 || N > 64 || !shape_ok(H, W)) return FDL_EINVAL;
  if (!o) return FDL_EINVAL;
  if (!(o->lambda >= 0.0) || !std::isfinite(o->lambda) || !(o->eps >= 0.0) || !std::isfinite(o->eps))
    return FDL_EINVAL;
  if (o->reg < FDL_REG_VIEW2 || o->reg > FDL_REG_L2) return FDL_EINVAL;
  if (o->precision < FDL_PREC_MIXED || o->precision > FDL_PREC_F32) return FDL_EINVAL;
  if (o->precision == FDL_PREC_F32 && N > 32) return FDL_ENOTSUP;
  if (std::isnan(o->kappa_max) || std::isnan(o->df_error_budget) || std::isnan(o->f32_error_budget))
    return FDL_EINVAL;
  return FDL_OK;
}

int run_solve(SpecView b, int K, int C, int H, int W, const float* u, const float* d, int N,
              const fdl_fit_opts* o, float* layers, const FitWs& f, cudaStream_t st) {
  SolveParams p;
  p.b = b;
  p.x = reinterpret_cast<float2*>(layers);
  p.u = u;
  p.d = d;
  p.K = K;
  p.C = C;
  p.N = N;
  p.H = H;
  p.W = W;
  p.reg = o->reg;
  p.lam = (float)o->lambda;
  p.lam_eps = (float)(o->lambda * (o->reg == FDL_REG_VIEW2 ? o->eps : 0.0));
  p.lam_d = o->lambda;
  p.lam_eps_d = o->lambda * (o->reg == FDL_REG_VIEW2 ? o->eps : 0.0);
  p.kappa_max = (float)(o->kappa_max > 0.0 ? o->kappa_max : 1e6);
  p.flagged = f.flagged;
  p.flagged64 = f.flagged64;
  p.err = nullptr;
  p.xn2 = nullptr;
  const double budget = o->df_error_budget > 0.0 ? o->df_error_budget : 4e-6;
  const double budget32 = o->f32_error_budget > 0.0 ? o->f32_error_budget : 2e-6;
  p.counters = f.counters;
  p.exp_table = f.exp_table;
  p.mom = f.mom;
  p.f32sums = f.f32sums;
  p.f32sums_tiles = f.f32sums_tiles;
  cudaError_t e = cudaMemsetAsync(f.counters, 0, kHeaderInts * sizeof(int), st);
  if (e != cudaSuccess) return FDL_ECUDA;
  e = launch_exp_table(f.exp_table, st);
  if (e == cudaSuccess && p.mom != nullptr) e = launch_mom_check(p, st);
  if (e != cudaSuccess) return FDL_ECUDA;
  // Each tier records an error scale per frequency (condition estimate x solution
  // norm); the frequencies with the largest estimated errors are re-solved in the next
  // tier until the estimated error of the rest is within that tier's budget (relative
  // L2 of the layers): FP32 -> double-float (registers for N <= 48, shared memory
  // beyond) -> native FP64.
  const int Qs = H * (W / 2 + 1);
  auto solve_df = [&](bool all_bins, bool fp64_tier) {
    if (!solve_df_supported(N)) return launch_solve_hp(p, all_bins, false, 0, st);
    cudaError_t r = cudaSuccess;
    if (fp64_tier) {
      p.err = f.err;
      p.xn2 = f.xn2;
      r = cudaMemsetAsync(f.err, 0, (size_t)Qs * sizeof(float), st);
      // after the FP32 pass xn2 already holds |x|^2 of every frequency (the
      // double-float pass overwrites its own), so the budget is relative to all of X
      if (r == cudaSuccess && all_bins) r = cudaMemsetAsync(f.xn2, 0, (size_t)Qs * sizeof(float), st);
    }
    if (r == cudaSuccess) r = launch_solve_df(p, all_bins, st);
    if (r == cudaSuccess && fp64_tier)
      r = launch_select_budget(f.err, f.xn2, Qs, kDfUnitPerSqrtView * std::sqrt((double)K), budget, f.select,
                               f.flagged64, f.counters + 5, st);
    if (r == cudaSuccess && fp64_tier) r = launch_solve_hp(p, false, true, 1, st);
    return r;
  };
  switch (o->precision) {
    case FDL_PREC_F32:
      e = launch_solve_f32(p, false, st);
      break;
    case FDL_PREC_DF:
      // double-float at every frequency, certified by the same FP64 budget as the mixed path
      e = solve_df(true, true);
      break;
    case FDL_PREC_F64:
      e = launch_solve_hp(p, true, true, 0, st);
      break;
    default:
      if (N > 32) {
        e = solve_df(true, true);
      } else {
        p.err = f.err;
        p.xn2 = f.xn2;
        e = launch_solve_f32(p, true, st);
        if (e == cudaSuccess)
          e = launch_select_budget(f.err, f.xn2, Qs, kF32Unit, budget32, f.select, f.flagged, f.counters + 4, st);
        if (e == cudaSuccess) e = solve_df(false, true);
      }
  }
  if (e == cudaSuccess) e = launch_fit_status(f.counters, st);
  return cuda_status(e);
}

size_t spec_tmp_bytes(int nimg, int H, int W) { return align_up((size_t)nimg * H * (W / 2) * sizeof(float2)); }

// header (counters and status word), [requests], spectra (split main part; the slots of the
// mixed path), the Nyquist plane, the DFT tables of the other paths and the mixed path's plan
size_t render_ws_bytes(int B, int C, int H, int W, bool with_reqs) {
  size_t s = align_up(kHeaderInts * sizeof(int));
  if (with_reqs) s += align_up((size_t)B * sizeof(fdl_request));
  s += align_up((size_t)B * C * H * (W / 2) * sizeof(float2));
  s += align_up((size_t)B * C * H * sizeof(float2));
  s += align_up(inv_table_elems(H, W) * sizeof(float4));
  s += align_up(render_plan_ints(B) * sizeof(int));
  return s;
}

// Spectra of a render, then the inverse DFT into images: `main`/`nyq` carved in that
// order (the dense layout of other sizes starts at `main` and fits in both), `tables`
// after them.
cudaError_t render_inverse(float2* main, float2* nyq, float4* tables, int B, int C, int H, int W, float* out,
                           const fdl_request* req, const int* count, cudaStream_t st, int nmax = 64,
                           const int* gate = nullptr) {
  const float scale = 1.f / ((float)H * (float)W);
  if (pow2_shape(H, W)) {
    cudaError_t e = launch_fft_cols_inv(spec_split(main, nyq, H, W), main, B * C, H, W, count, C, st, gate);
    if (e == cudaSuccess)
      e = launch_irfft_rows(main, out, (long long)B * C * H, H, W, scale, req, count, C, st, nmax, gate);
    return e;
  }
  const GenPlans g = gen_plans(H, W);
  const SpecView sp = spec_dense(main, H, W);
  cudaError_t e = launch_gen_tables2(g, tables, st);
  if (e == cudaSuccess) e = launch_gen_cols(sp, sp, B * C, H, W, true, g.ph, tables, count, C, st);
  if (e == cudaSuccess)
    e = launch_gen_rows_inv(sp, out, (long long)B * C * H, H, W, scale, req, count, C, g.pw, tables, st, nmax);
  return e;
}
SpecView render_spec_view(float2* main, float2* nyq, int H, int W) {
  return pow2_shape(H, W) ? spec_split(main, nyq, H, W) : spec_dense(main, H, W);
}

// Workspace of a render: header, [requests], then the spectra, Nyquist plane and tables.
struct RenderWs {
  int* header;
  fdl_request* req;
  float2* main;
  float2* nyq;
  float4* tables;
  int* plan;  // the mixed path's request groups (launch_render_plan)
};
RenderWs carve_render(void* ws, int B, int C, int H, int W, bool with_reqs) {
  Carver cv(ws);
  RenderWs r;
  r.header = cv.take<int>(kHeaderInts);
  r.req = with_reqs ? cv.take<fdl_request>(B) : nullptr;
  r.main = cv.take<float2>((size_t)B * C * H * (W / 2));
  r.nyq = cv.take<float2>((size_t)B * C * H);
  r.tables = cv.take<float4>(inv_table_elems(H, W));
  r.plan = cv.take<int>(render_plan_ints(B));
  return r;
}

// Renders B requests (validated on the device against C, H, W and Nmax).
//  * tiled: spectra of exactly H x W x C with the layer values of each tile of frequencies
//    staged once and reused by every request of one FDL, then the separate inverse DFT
//    passes; the only path for sizes that are not powers of two, H = 4096 and per-layer shifts;
//  * mixed: requests of any power-of-two sizes within (C, H, W) and of different FDLs in one
//    launch, the layer values staged once per run of consecutive requests of one FDL, each
//    request's spectrum in its own slot, then per-request inverse DFT passes.
// mixed = true (fdl_refocus): a one-CTA kernel on the device sets the gate word to 1 when the
// active requests all read one FDL of exactly H x W x C (the tiled path), else 0, and plans the
// request groups of the mixed path; both paths are enqueued and the one the gate rules out
// returns at once.
cudaError_t render_requests(const fdl_request* req, int B, const int* count, int C, int H, int W, int Nmax,
                            const RenderWs& w, cudaStream_t st, bool mixed, const float* shifts = nullptr) {
  int* status = w.header + kStatusWord;
  const int* gate = nullptr;
  if (mixed && shifts == nullptr && render_mixed_supported(H, W)) {
    int* g = w.header + kGateWord;
    cudaError_t e = launch_render_plan(req, B, count, C, H, W, Nmax, g, w.plan, st);
    if (e == cudaSuccess) e = launch_render_mixed(req, B, count, C, H, W, Nmax, w.main, w.nyq, w.plan, status, st, g);
    if (e != cudaSuccess) return e;
    gate = g;
  }
  cudaError_t e = launch_render_spectra(req, B, count, C, H, W, Nmax, render_spec_view(w.main, w.nyq, H, W), status,
                                        st, shifts, gate);
  if (e == cudaSuccess) e = render_inverse(w.main, w.nyq, w.tables, B, C, H, W, nullptr, req, count, st, Nmax, gate);
  return e;
}

}  // namespace

extern "C" {

FDL_API const char* fdl_strerror(int status) {
  switch (status) {
    case FDL_OK:
      return "ok";
    case FDL_EINVAL:
      return "invalid argument";
    case FDL_ENOMEM:
      return "workspace too small";
    case FDL_ECUDA:
      return "CUDA launch or runtime error";
    case FDL_ETIMEOUT:
      return "bounded wait timed out";
    case FDL_ENOTSUP:
      return "not supported by the library";
    default:
      return "unknown status";
  }
}

FDL_API int fdl_version(void) { return 1; }

// ------------------------------------------------------------------ DFTs
FDL_API size_t fdl_rfft2_workspace_size(int nimg, int H, int W) {
  if (nimg < 1 || !shape_ok(H, W)) return 0;
  return spec_tmp_bytes(nimg, H, W) + align_up(dft_table_elems(H, W) * sizeof(float4));
}

FDL_API int fdl_rfft2(const float* images, int nimg, int H, int W, float* spectra, void* workspace,
                      size_t workspace_bytes, void* stream) {
  if (nimg < 1 || !shape_ok(H, W) || !images || !spectra || !workspace) return FDL_EINVAL;
  if (workspace_bytes < fdl_rfft2_workspace_size(nimg, H, W)) return FDL_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float2* tmp = static_cast<float2*>(workspace);
  float4* tables = reinterpret_cast<float4*>(static_cast<char*>(workspace) + spec_tmp_bytes(nimg, H, W));
  if (!pow2_shape(H, W)) {
    const GenPlans g = gen_plans(H, W);
    const SpecView out = spec_dense(reinterpret_cast<float2*>(spectra), H, W);
    cudaError_t e = launch_gen_tables2(g, tables, st);
    if (e == cudaSuccess) e = launch_gen_rows_fwd(images, out, (long long)nimg * H, H, W, g.pw, tables, st);
    if (e == cudaSuccess) e = launch_gen_cols(out, out, nimg, H, W, false, g.ph, tables, nullptr, 1, st);
    return cuda_status(e);
  }
  cudaError_t e = launch_twiddle_tables(tables, H, W, st);
  if (e == cudaSuccess) e = launch_rfft_rows_df(images, tmp, (long long)nimg * H, W, tables, st);
  if (e == cudaSuccess)
    e = launch_fft_cols_fwd_df(spec_split(tmp, nullptr, H, W), spec_dense(reinterpret_cast<float2*>(spectra), H, W),
                               nimg, H, W, tables, st);
  return cuda_status(e);
}

FDL_API size_t fdl_irfft2_workspace_size(int nimg, int H, int W) {
  if (nimg < 1 || !shape_ok(H, W)) return 0;
  if (!pow2_shape(H, W))  // dense copy of the spectra, then the tables
    return align_up((size_t)nimg * H * (W / 2 + 1) * sizeof(float2)) + align_up(inv_table_elems(H, W) * sizeof(float4));
  return spec_tmp_bytes(nimg, H, W);
}

FDL_API int fdl_irfft2(const float* spectra, int nimg, int H, int W, float* images, void* workspace,
                       size_t workspace_bytes, void* stream) {
  if (nimg < 1 || !shape_ok(H, W) || !images || !spectra || !workspace) return FDL_EINVAL;
  if (workspace_bytes < fdl_irfft2_workspace_size(nimg, H, W)) return FDL_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float2* tmp = static_cast<float2*>(workspace);
  if (!pow2_shape(H, W)) {
    const GenPlans g = gen_plans(H, W);
    float4* tables =
        reinterpret_cast<float4*>(static_cast<char*>(workspace) + align_up((size_t)nimg * H * (W / 2 + 1) * sizeof(float2)));
    const SpecView in = spec_dense(const_cast<float2*>(reinterpret_cast<const float2*>(spectra)), H, W);
    const SpecView t = spec_dense(tmp, H, W);
    cudaError_t e = launch_gen_tables2(g, tables, st);
    if (e == cudaSuccess) e = launch_gen_cols(in, t, nimg, H, W, true, g.ph, tables, nullptr, 1, st);
    if (e == cudaSuccess)
      e = launch_gen_rows_inv(t, images, (long long)nimg * H, H, W, 1.f / ((float)H * (float)W), nullptr, nullptr, 1,
                              g.pw, tables, st);
    return cuda_status(e);
  }
  cudaError_t e = launch_fft_cols_inv(spec_dense(const_cast<float2*>(reinterpret_cast<const float2*>(spectra)), H, W),
                                      tmp, nimg, H, W, nullptr, 1, st);
  if (e == cudaSuccess)
    e = launch_irfft_rows(tmp, images, (long long)nimg * H, H, W, 1.f / ((float)H * (float)W), nullptr, nullptr, 1,
                          st);
  return cuda_status(e);
}

// ------------------------------------------------------------------ fit
FDL_API size_t fdl_fit_workspace_size(int K, int C, int H, int W, int N) {
  if (K < 1 || C < 1 || N < 1 || !shape_ok(H, W)) return 0;
  return carve_fit(nullptr, K, C, H, W, N, true).bytes;
}

FDL_API int fdl_fit(const float* views, int K, int C, int H, int W, const float* u, const float* d, int N,
                    const fdl_fit_opts* opts, float* layers, void* workspace, size_t workspace_bytes, void* stream) {
  int s = check_fit_args(K, C, H, W, N, opts);
  if (s != FDL_OK) return s;
  if (!views || !u || !d || !layers || !workspace) return FDL_EINVAL;
  if (workspace_bytes < fdl_fit_workspace_size(K, C, H, W, N)) return FDL_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FitWs f = carve_fit(workspace, K, C, H, W, N, true);
  const int nimg = K * C;
  if (!pow2_shape(H, W)) {
    // dense half spectra from spec_main (spec_main and spec_nyq are carved back to back)
    const GenPlans g = gen_plans(H, W);
    const SpecView b = spec_dense(f.spec_main, H, W);
    cudaError_t e = launch_gen_tables2(g, f.fft_tables, st);
    if (e == cudaSuccess) e = launch_gen_rows_fwd(views, b, (long long)nimg * H, H, W, g.pw, f.fft_tables, st);
    if (e == cudaSuccess) e = launch_gen_cols(b, b, nimg, H, W, false, g.ph, f.fft_tables, nullptr, 1, st);
    if (e != cudaSuccess) return FDL_ECUDA;
    return run_solve(b, K, C, H, W, u, d, N, opts, layers, f, st);
  }
  cudaError_t e = launch_twiddle_tables(f.fft_tables, H, W, st);
  if (e == cudaSuccess) e = launch_rfft_rows_df(views, f.spec_main, (long long)nimg * H, W, f.fft_tables, st);
  SpecView b = spec_split(f.spec_main, f.spec_nyq, H, W);
  if (e == cudaSuccess) e = launch_fft_cols_fwd_df(b, b, nimg, H, W, f.fft_tables, st);
  if (e != cudaSuccess) return FDL_ECUDA;
  return run_solve(b, K, C, H, W, u, d, N, opts, layers, f, st);
}

FDL_API size_t fdl_fit_spectra_workspace_size(int K, int C, int H, int W, int N) {
  if (K < 1 || C < 1 || N < 1 || !shape_ok(H, W)) return 0;
  return carve_fit(nullptr, K, C, H, W, N, false).bytes;
}

FDL_API int fdl_fit_spectra(const float* spectra, int K, int C, int H, int W, const float* u, const float* d, int N,
                            const fdl_fit_opts* opts, float* layers, void* workspace, size_t workspace_bytes,
                            void* stream) {
  int s = check_fit_args(K, C, H, W, N, opts);
  if (s != FDL_OK) return s;
  if (!spectra || !u || !d || !layers || !workspace) return FDL_EINVAL;
  if (workspace_bytes < fdl_fit_spectra_workspace_size(K, C, H, W, N)) return FDL_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FitWs f = carve_fit(workspace, K, C, H, W, N, false);
  SpecView b = spec_dense(const_cast<float2*>(reinterpret_cast<const float2*>(spectra)), H, W);
  return run_solve(b, K, C, H, W, u, d, N, opts, layers, f, st);
}

FDL_API int fdl_fit_tier_counts(const void* workspace, int* counts, void* stream) {
  if (!workspace || !counts) return FDL_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int tmp[7];
  cudaError_t e = cudaMemcpyAsync(tmp, workspace, sizeof(tmp), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return FDL_ECUDA;
  counts[0] = tmp[0];  // FP32
  counts[1] = tmp[1];  // double-float
  counts[2] = tmp[6];  // native FP64
  counts[3] = tmp[2];  // breakdowns
  counts[4] = tmp[3];  // non-finite inputs
  return FDL_OK;
}

// ------------------------------------------------------------------ render
FDL_API size_t fdl_render_workspace_size(int B, int C, int H, int W) {
  if (B < 1 || C < 1 || C > 4 || !shape_ok(H, W)) return 0;
  return render_ws_bytes(B, C, H, W, true);
}

FDL_API int fdl_render(const float* layers, const float* d, int N, int C, int H, int W, const float* u0, int B,
                       float* out, void* workspace, size_t workspace_bytes, void* stream) {
  if (B < 1 || C < 1 || C > 4 || N < 1 || N > 64 || !shape_ok(H, W)) return FDL_EINVAL;
  if (!layers || !d || !u0 || !out || !workspace) return FDL_EINVAL;
  if (workspace_bytes < fdl_render_workspace_size(B, C, H, W)) return FDL_ENOMEM;
  if (B > 65535) return FDL_ENOTSUP;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const RenderWs w = carve_render(workspace, B, C, H, W, true);
  cudaError_t e = cudaMemsetAsync(w.header, 0, kHeaderInts * sizeof(int), st);
  if (e == cudaSuccess) e = launch_pinhole_requests(w.req, layers, d, N, C, H, W, u0, B, out, st);
  if (e == cudaSuccess) e = render_requests(w.req, B, nullptr, C, H, W, N, w, st, false);
  return cuda_status(e);
}

// ------------------------------------------------------------------ drawn aperture
FDL_API size_t fdl_aperture_table_workspace_size(int P, int Z) {
  if (P < 1 || (P & 1) == 0 || P > Z || !shape_ok(Z, Z)) return 0;
  return align_up((size_t)Z * Z * sizeof(float)) + align_up(sizeof(double)) + fdl_rfft2_workspace_size(1, Z, Z);
}

FDL_API int fdl_aperture_table(const float* raster, int P, int Z, float* table, void* workspace,
                               size_t workspace_bytes, void* stream) {
  if (P < 1 || (P & 1) == 0 || P > Z || !shape_ok(Z, Z) || !raster || !table || !workspace) return FDL_EINVAL;
  if (workspace_bytes < fdl_aperture_table_workspace_size(P, Z)) return FDL_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carver cv(workspace);
  float* pad = cv.take<float>((size_t)Z * Z);
  double* sum = cv.take<double>(1);
  void* ws2 = static_cast<char*>(workspace) + cv.off;
  cudaError_t e = launch_aperture_table_prep(raster, P, Z, pad, sum, st);
  if (e != cudaSuccess) return FDL_ECUDA;
  const int s = fdl_rfft2(pad, 1, Z, Z, table, ws2, fdl_rfft2_workspace_size(1, Z, Z), stream);
  if (s != FDL_OK) return s;
  return cuda_status(launch_aperture_table_scale(reinterpret_cast<float2*>(table), Z, sum, st));
}

FDL_API size_t fdl_refocus_workspace_size(int B, int C, int H, int W) {
  if (B < 1 || C < 1 || C > 4 || !shape_ok(H, W)) return 0;
  return render_ws_bytes(B, C, H, W, false);
}

FDL_API int fdl_refocus(const fdl_request* req, int B, const int* count, int C, int H, int W, int Nmax,
                        void* workspace, size_t workspace_bytes, void* stream) {
  if (B < 1 || C < 1 || C > 4 || Nmax < 1 || Nmax > 64 || !shape_ok(H, W)) return FDL_EINVAL;
  if (!req || !workspace) return FDL_EINVAL;
  if (workspace_bytes < fdl_refocus_workspace_size(B, C, H, W)) return FDL_ENOMEM;
  if (B > 65535) return FDL_ENOTSUP;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const RenderWs w = carve_render(workspace, B, C, H, W, false);
  cudaError_t e = cudaMemsetAsync(w.header, 0, kHeaderInts * sizeof(int), st);
  // one request reads one FDL: the tiled path, without the device check (if its size is not
  // exactly (C, H, W) the kernels reject it)
  if (e == cudaSuccess) e = render_requests(req, B, count, C, H, W, Nmax, w, st, B > 1);
  return cuda_status(e);
}

// ------------------------------------------------------------------ host buffers
FDL_API size_t fdl_fit_render_host_workspace_size(int K, int C, int H, int W, int N, int B) {
  const size_t fit = fdl_fit_workspace_size(K, C, H, W, N);
  const size_t ren = fdl_refocus_workspace_size(B, C, H, W);
  if (fit == 0 || ren == 0) return 0;
  return align_up((size_t)K * C * H * W * sizeof(float)) + align_up(fit) + ren;
}

FDL_API int fdl_fit_render_host(const float* views_host, int K, int C, int H, int W, const float* u, const float* d,
                                int N, const fdl_fit_opts* opts, float* layers, const fdl_request* req, int B,
                                float* images, size_t image_floats, float* images_host, void* workspace,
                                size_t workspace_bytes, void* stream) {
  int s = check_fit_args(K, C, H, W, N, opts);
  if (s != FDL_OK) return s;
  if (B < 1 || !views_host || !u || !d || !layers || !req || !images || !images_host || !workspace) return FDL_EINVAL;
  if (workspace_bytes < fdl_fit_render_host_workspace_size(K, C, H, W, N, B)) return FDL_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(workspace);
  float* staging = reinterpret_cast<float*>(base);
  void* ws_fit = base + align_up((size_t)K * C * H * W * sizeof(float));
  const size_t fit_bytes = align_up(fdl_fit_workspace_size(K, C, H, W, N));
  void* ws_ren = static_cast<char*>(ws_fit) + fit_bytes;
  // The views are copied into the workspace by the copy engine, not read in place through the
  // host mapping by the forward DFT: with two light fields in flight on two streams the copy
  // overlaps the other's computation (9x9 views, 512^2 RGB on GB300: 14.6 ms per light field
  // from host to host against 15.2 ms read in place); the images go back the same way.
  if (cudaMemcpyAsync(staging, views_host, (size_t)K * C * H * W * sizeof(float), cudaMemcpyDefault, st) !=
      cudaSuccess)
    return FDL_ECUDA;
  const float* views = staging;
  s = fdl_fit(views, K, C, H, W, u, d, N, opts, layers, ws_fit, fit_bytes, stream);
  if (s != FDL_OK) return s;
  s = fdl_refocus(req, B, nullptr, C, H, W, N, ws_ren, fdl_refocus_workspace_size(B, C, H, W), stream);
  if (s != FDL_OK) return s;
  if (cudaMemcpyAsync(images_host, images, image_floats * sizeof(float), cudaMemcpyDefault, st) != cudaSuccess)
    return FDL_ECUDA;
  return FDL_OK;
}

// ------------------------------------------------------------------ device status
FDL_API int fdl_sync_status(const void* workspace, int* status, void* stream) {
  if (!workspace || !status) return FDL_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, static_cast<const int*>(workspace) + kStatusWord, sizeof(int),
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return FDL_ECUDA;
  *status = v;
  return FDL_OK;
}

// ------------------------------------------------------------------ calibration
FDL_API size_t fdl_calib_grad_workspace_size(int K, int C, int H, int W, int N, int nbins) {
  (void)C;
  (void)H;
  (void)W;
  (void)nbins;
  if (K < 1 || N < 1) return 0;
  return align_up(1024 * sizeof(float4)) + align_up((size_t)kCalibGrid * (1 + 2 * K + N) * sizeof(double));
}

FDL_API int fdl_calib_grad(const float* spectra, int K, int C, int H, int W, const float* u, const float* d, int N,
                           const fdl_fit_opts* opts, const int* bins, int nbins, float* loss, float* grad_u,
                           float* grad_d, void* workspace, size_t workspace_bytes, void* stream) {
  int s = check_fit_args(K, C, H, W, N, opts);
  if (s != FDL_OK && s != FDL_ENOTSUP) return s;
  if (opts->reg == FDL_REG_VIEW2) return FDL_EINVAL;
  if (!spectra || !u || !d || !loss || !grad_u || !grad_d || !workspace) return FDL_EINVAL;
  if (bins && nbins < 1) return FDL_EINVAL;
  if (workspace_bytes < fdl_calib_grad_workspace_size(K, C, H, W, N, nbins)) return FDL_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carver cv(workspace);
  CalibParams p;
  p.exp_table = cv.take<float4>(1024);
  p.partials = cv.take<double>((size_t)kCalibGrid * (1 + 2 * K + N));
  p.b = spec_dense(const_cast<float2*>(reinterpret_cast<const float2*>(spectra)), H, W);
  p.u = u;
  p.d = d;
  p.K = K;
  p.C = C;
  p.N = N;
  p.H = H;
  p.W = W;
  p.reg = opts->reg;
  p.lam = (float)opts->lambda;
  p.lam_d = opts->lambda;
  p.bins = bins;
  p.nbins = bins ? nbins : 0;
  p.loss = loss;
  p.grad_u = grad_u;
  p.grad_d = grad_d;
  p.counters = nullptr;
  p.f64 = opts->precision == FDL_PREC_F64;
  cudaError_t e = launch_exp_table(const_cast<float4*>(p.exp_table), st);
  if (e == cudaSuccess) e = launch_calib_grad(p, st);
  return cuda_status(e);
}

// ------------------------------------------------------------------ general system
FDL_API size_t fdl_fit_general_workspace_size(int K, int C, int H, int W, int N) {
  if (K < 1 || C < 1 || N < 1 || !shape_ok(H, W)) return 0;
  return carve_fit(nullptr, K, C, H, W, N, false, false).bytes;
}

FDL_API int fdl_fit_general(const float* spectra, int K, int C, int H, int W, int N, const fdl_system* sys,
                            const fdl_fit_opts* opts, float* layers, void* workspace, size_t workspace_bytes,
                            void* stream) {
  int s = check_fit_args(K, C, H, W, N, opts);
  if (s != FDL_OK && s != FDL_ENOTSUP) return s;
  if (!spectra || !sys || !layers || !workspace) return FDL_EINVAL;
  if (!sys->P && !(sys->u && sys->d)) return FDL_EINVAL;
  if ((sys->views || opts->reg == FDL_REG_VIEW2) && !sys->d) return FDL_EINVAL;
  if (workspace_bytes < fdl_fit_general_workspace_size(K, C, H, W, N)) return FDL_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FitWs f = carve_fit(workspace, K, C, H, W, N, false, false);
  SolveParams p{};
  p.b = spec_dense(const_cast<float2*>(reinterpret_cast<const float2*>(spectra)), H, W);
  p.x = reinterpret_cast<float2*>(layers);
  p.u = sys->u;
  p.d = sys->d;
  p.P = sys->P;
  p.views = sys->views;
  p.K = K;
  p.C = C;
  p.N = N;
  p.H = H;
  p.W = W;
  p.reg = opts->reg;
  p.lam = (float)opts->lambda;
  p.lam_eps = (float)(opts->lambda * (opts->reg == FDL_REG_VIEW2 ? opts->eps : 0.0));
  p.lam_d = opts->lambda;
  p.lam_eps_d = opts->lambda * (opts->reg == FDL_REG_VIEW2 ? opts->eps : 0.0);
  p.flagged = f.flagged;
  p.flagged64 = f.flagged64;
  p.counters = f.counters;
  p.exp_table = f.exp_table;
  p.mom = nullptr;
  cudaError_t e = cudaMemsetAsync(f.counters, 0, kHeaderInts * sizeof(int), st);
  if (e == cudaSuccess) e = launch_exp_table(f.exp_table, st);
  if (e == cudaSuccess) e = launch_solve_hp(p, true, opts->precision == FDL_PREC_F64, 0, st);
  if (e == cudaSuccess) e = launch_fit_status(f.counters, st);
  return cuda_status(e);
}

FDL_API size_t fdl_render_shifts_workspace_size(int B, int C, int H, int W) {
  if (B < 1 || C < 1 || C > 4 || !shape_ok(H, W)) return 0;
  return render_ws_bytes(B, C, H, W, true);
}

FDL_API int fdl_render_shifts(const float* layers, const float* P, int N, int C, int H, int W, int B, float* out,
                              void* workspace, size_t workspace_bytes, void* stream) {
  if (B < 1 || C < 1 || C > 4 || N < 1 || N > 64 || !shape_ok(H, W)) return FDL_EINVAL;
  if (!layers || !P || !out || !workspace) return FDL_EINVAL;
  if (workspace_bytes < fdl_render_shifts_workspace_size(B, C, H, W)) return FDL_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const RenderWs w = carve_render(workspace, B, C, H, W, true);
  cudaError_t e = cudaMemsetAsync(w.header, 0, kHeaderInts * sizeof(int), st);
  // pinhole requests on the FDL (d unused: the shifts replace u0 d_k)
  if (e == cudaSuccess) e = launch_pinhole_requests(w.req, layers, P, N, C, H, W, nullptr, B, out, st);
  if (e == cudaSuccess) e = render_requests(w.req, B, nullptr, C, H, W, N, w, st, false, P);
  return cuda_status(e);
}

FDL_API size_t fdl_calib_grad_shifts_workspace_size(int K, int C, int H, int W, int N, int nbins) {
  (void)C;
  (void)H;
  (void)W;
  (void)nbins;
  if (K < 1 || N < 1) return 0;
  return align_up(1024 * sizeof(float4)) + align_up((size_t)kCalibGrid * (1 + 2 * (size_t)K * N) * sizeof(double));
}

FDL_API int fdl_calib_grad_shifts(const float* spectra, int K, int C, int H, int W, const float* P, int N,
                                  const fdl_fit_opts* opts, const int* bins, int nbins, float* loss, float* grad_P,
                                  void* workspace, size_t workspace_bytes, void* stream) {
  int s = check_fit_args(K, C, H, W, N, opts);
  if (s != FDL_OK && s != FDL_ENOTSUP) return s;
  if (opts->reg == FDL_REG_VIEW2) return FDL_EINVAL;
  if (!spectra || !P || !loss || !grad_P || !workspace) return FDL_EINVAL;
  if (bins && nbins < 1) return FDL_EINVAL;
  // one block holds the FP64 solver's matrices and the 1 + 2 K N accumulators
  const size_t smem = (size_t)(N * (N + 1) + N + N * C + 4) * 16 + calib_shifts_acc_bytes(K, N);
  if (smem > 200 * 1024) return FDL_ENOTSUP;
  if (workspace_bytes < fdl_calib_grad_shifts_workspace_size(K, C, H, W, N, nbins)) return FDL_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carver cv(workspace);
  CalibParams p;
  p.exp_table = cv.take<float4>(1024);
  p.partials = cv.take<double>((size_t)kCalibGrid * (1 + 2 * (size_t)K * N));
  p.b = spec_dense(const_cast<float2*>(reinterpret_cast<const float2*>(spectra)), H, W);
  p.u = nullptr;
  p.d = nullptr;
  p.P = P;
  p.K = K;
  p.C = C;
  p.N = N;
  p.H = H;
  p.W = W;
  p.reg = opts->reg;
  p.lam = (float)opts->lambda;
  p.lam_d = opts->lambda;
  p.bins = bins;
  p.nbins = bins ? nbins : 0;
  p.loss = loss;
  p.grad_u = nullptr;
  p.grad_d = nullptr;
  p.grad_P = grad_P;
  p.counters = nullptr;
  p.f64 = opts->precision == FDL_PREC_F64;
  cudaError_t e = launch_exp_table(const_cast<float4*>(p.exp_table), st);
  if (e == cudaSuccess) e = launch_calib_grad(p, st);
  return cuda_status(e);
}

}  // extern "C"

// ------------------------------------------------------------------ fixed-scratch fit
// Scratch of fdl_fit_spectra_noalloc: a file-scope device array, so that the
// entry point never allocates.  Every GPU that loads the library holds it
// (8,455,168 bytes) until the process exits; all calls on a device share it.
namespace {

constexpr size_t kNoAllocMaxBins = 1024 * 513;  // H * (W/2 + 1) of a 1024 x 1024 image
constexpr size_t kNoAllocCounters = 1024;  // counters (64 B), then the kMomSlots float2 at 256
constexpr size_t kNoAllocTable = 1024 * sizeof(float4);
constexpr size_t kNoAllocSelect = 32768;  // >= select_scratch_bytes()
constexpr size_t kNoAllocBytes =
    kNoAllocCounters + kNoAllocTable + kNoAllocSelect + 4 * kNoAllocMaxBins * sizeof(int);

static_assert(256 + kMomSlots * sizeof(float2) <= kNoAllocCounters, "moment slots overlap the exp table");
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the array on the current device, looked up once per device.
// Host code must not hand the symbol itself to a kernel: on the host it only
// names a stand-in object.
int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return FDL_ECUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FDL_ECUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return FDL_OK;
}

}  // namespace

extern "C" FDL_API int fdl_fit_spectra_noalloc(const float* spectra, int K, int C, int H, int W, const float* u,
                                               const float* d, int N, const fdl_fit_opts* opts, float* layers,
                                               void* stream) {
  int s = check_fit_args(K, C, H, W, N, opts);
  if (s != FDL_OK) return s;
  if (!spectra || !u || !d || !layers) return FDL_EINVAL;
  if ((size_t)H * (W / 2 + 1) > kNoAllocMaxBins) return FDL_ENOMEM;
  if (select_scratch_bytes() > kNoAllocSelect) return FDL_ENOTSUP;
  void* base = nullptr;
  s = noalloc_scratch(&base);
  if (s != FDL_OK) return s;
  char* b = static_cast<char*>(base);
  FitWs f;
  f.counters = reinterpret_cast<int*>(b);
  f.mom = reinterpret_cast<float2*>(b + 256);
  f.exp_table = reinterpret_cast<float4*>(b + kNoAllocCounters);
  f.select = b + kNoAllocCounters + kNoAllocTable;
  f.flagged = reinterpret_cast<int*>(b + kNoAllocCounters + kNoAllocTable + kNoAllocSelect);
  f.flagged64 = f.flagged + kNoAllocMaxBins;
  f.err = reinterpret_cast<float*>(f.flagged64 + kNoAllocMaxBins);
  f.xn2 = f.err + kNoAllocMaxBins;
  f.fft_tables = nullptr;
  f.spec_main = f.spec_nyq = nullptr;
  f.bytes = kNoAllocBytes;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SpecView bv = spec_dense(const_cast<float2*>(reinterpret_cast<const float2*>(spectra)), H, W);
  return run_solve(bv, K, C, H, W, u, d, N, opts, layers, f, st);
}
