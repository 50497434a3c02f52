// Host-side launchers of the FDL kernels (internal to libfdl).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "fdl.h"

namespace fdl {

// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device; the attribute is set once per (kernel, device, size).
cudaError_t set_smem(const void* kernel, size_t bytes);
// SM count of the current device (queried once per process)
int num_sms();

// ---- FFT (fft.cu) ----------------------------------------------------------
// Inverse column pass: half spectra `in` (any layout) -> split layout `out`
// with pitch W/2 and the kx = 0 / kx = W/2 columns packed after taking
// their Hermitian parts.
// count (nullable, device): only images [0, *count * C) are transformed.
// gate (nullable, device): the inverse passes return at once unless *gate != 0.
cudaError_t launch_fft_cols_inv(SpecView in, float2* out, int nimg, int H, int W, const int* count, int C,
                                cudaStream_t st, const int* gate = nullptr);
// Forward passes, with double-float arithmetic inside each pass (fft_df.cu).
// Row pass: nrows rows of W floats -> W/2 complex each (element 0 packs
// X[0] + i X[W/2]), rows written with stride W/2.  Column pass: forward DFT
// along H of a row-transformed stack held in the split layout `in` (kx = 0
// column packed), written unpacked to `out` (may alias `in`).  `tables` =
// double-float twiddles of lengths W then H, built by launch_twiddle_tables
// into fft_df_table_bytes(H, W) of workspace.
size_t fft_df_table_bytes(int H, int W);
cudaError_t launch_twiddle_tables(float4* tables, int H, int W, cudaStream_t st);
cudaError_t launch_rfft_rows_df(const float* in, float2* out, long long nrows, int W, const float4* tables,
                                cudaStream_t st);
cudaError_t launch_fft_cols_fwd_df(SpecView in, SpecView out, int nimg, int H, int W, const float4* tables,
                                   cudaStream_t st);
// Row pass of the inverse real DFT: packed rows (pitch W/2) -> W floats, times scale.
// req (nullable, device): image b*C + c goes to req[b].out + c*H*W instead of
// the contiguous `out`; count (nullable, device) limits the images to *count * C.
// nmax: with req, rows of requests that request_ok(.., nmax, exact) rejects are not written.
cudaError_t launch_irfft_rows(const float2* in, float* out, long long nrows, int H, int W, float scale,
                              const fdl_request* req, const int* count, int C, cudaStream_t st, int nmax = 64,
                              const int* gate = nullptr);

// ---- per-frequency solve (solve.cu) -----------------------------------------
struct SolveParams {
  SpecView b;          // input spectra, images ordered [K][C]
  float2* x;           // output layers, dense [N][C][H][W/2+1]
  const float* u;      // [K][2]
  const float* d;      // [N]
  int K, C, N, H, W;
  int reg;
  float lam, lam_eps;  // lambda and lambda*eps
  double lam_d, lam_eps_d;
  float kappa_max;     // largest estimated condition number kept in FP32
  int* flagged;        // bins for the double-float pass (chosen from the FP32 err / xn2)
  int* flagged64;      // bins for the native FP64 pass (chosen from err / xn2)
  float* err;          // per bin: condition estimate x |x| of the last pass (nullable)
  float* xn2;          // per bin: |x|^2 of the last pass that solved it
  int* counters;       // [0] FP32 bins, [1] double-float bins, [2] breakdowns, [3] non-finite,
                       // [4] double-float list length, [5] FP64 list length, [6] FP64 bins,
                       // [8] moment form applies, [10] views on the integer lattice
  const float4* exp_table;  // df table of exp(2 pi i n / 1024), n in [0, 1024)
  const float* P = nullptr;               // free shifts [K][N][2] (k_solve_hp only)
  const fdl_request* views = nullptr;     // per-image apertures [K] (k_solve_hp only)
  // Moment form of the double-float Gram (nullable): kMomSlots float2, entries [0, N)
  // e_k = d_k - d_0 - k Delta as double-floats, written by the check kernel, which also
  // sets counters[8] to 1 when the moment form applies.
  float2* mom;
  // Scratch of the FP32 solve's moment-form view sums (nullable: the solve kernel forms them
  // itself), for f32sums_tiles tiles of 8 frequencies at a time: (W_0, W_1) float4
  // [tiles x 8][32], then the right-hand sides float2 [tiles x 8][4][32].
  float4* f32sums = nullptr;
  int f32sums_tiles = 0;
};
constexpr int kMomSlots = 65;
// the most tiles of 8 frequencies whose FP32 view sums one k_f32_sums launch writes
constexpr int kF32SumsTiles = 16448;
// FP32 solve of every stored bin; with estimate, also err / xn2 per bin (err = +inf
// where the result is not trusted) and every bin counted in counters[0].
cudaError_t launch_solve_f32(const SolveParams& p, bool estimate, cudaStream_t st);
// Solves the bins of list `list` (0: p.flagged / counters[4], 1: p.flagged64 /
// counters[5]) or, when all_bins, every stored bin; T = native FP64 when f64
// else double-float (shared-memory matrix, any N <= 64).
cudaError_t launch_solve_hp(const SolveParams& p, bool all_bins, bool f64, int list, cudaStream_t st);
cudaError_t launch_exp_table(float4* table, cudaStream_t st);
// Double-float solve with the matrix in registers (N <= 48); same contract as
// launch_solve_hp with f64 = false.
bool solve_df_supported(int N);
// Decides whether the disparities are close enough to a grid for the moment form of the
// Gram matrix (counters[8]) and writes their deviations e_k to p.mom; must precede the
// FP32 and double-float launches of a solve that sets p.mom.
cudaError_t launch_mom_check(const SolveParams& p, cudaStream_t st);
cudaError_t launch_solve_df(const SolveParams& p, bool all_bins, cudaStream_t st);

// ---- DFTs of lengths that are not powers of two (fft_gen.cu) -----------------
constexpr int kGenMaxRadix = 32;        // largest prime factor transformed directly
constexpr int kGenMaxPasses = 16;
constexpr int kGenMaxLength = 4096;
constexpr int kGenMaxBluestein = 4096;  // largest power-of-two length of a Bluestein convolution
struct GenPlan {
  int L;                        // transform length
  int np;                       // radix passes of L (0 with Bluestein)
  int radix[kGenMaxPasses];
  int M;                        // Bluestein convolution length (0: direct)
  int mp;                       // radix passes of M
  int mradix[kGenMaxPasses];
  int tw, chirp, twm, bhat;     // float4 offsets of the tables in the table area
  int elems;                    // float4 elements of tables this plan uses
};
struct GenPlanM {
  int np;
  int radix[kGenMaxPasses];
};
// lengths up to kGenMaxLength whose prime factors are <= kGenMaxRadix, or whose
// Bluestein length fits kGenMaxBluestein (L <= 2048)
bool gen_supported(int L);
// plan of length L with its tables starting at float4 offset `base`
bool gen_plan(int L, int base, GenPlan* p);
cudaError_t launch_gen_tables(const GenPlan& p, float4* tables, cudaStream_t st);
// real rows (nrows = images * H, length W) -> half spectra (kx <= W/2) in `out`
cudaError_t launch_gen_rows_fwd(const float* x, SpecView out, long long nrows, int H, int W, const GenPlan& pw,
                                const float4* tables, cudaStream_t st);
// columns of nimg half spectra from s to so (may alias; forward or inverse; images >= count*C skipped)
cudaError_t launch_gen_cols(SpecView s, SpecView so, int nimg, int H, int W, bool inverse, const GenPlan& ph,
                            const float4* tables, const int* count, int C, cudaStream_t st);
// Hermitian-completed inverse of the rows, real part x scale, to `out` or the requests' outputs
cudaError_t launch_gen_rows_inv(SpecView in, float* out, long long nrows, int H, int W, float scale,
                                const fdl_request* req, const int* count, int C, const GenPlan& pw,
                                const float4* tables, cudaStream_t st, int nmax = 64);

// A render request the kernels can serve: non-null, aligned FDL and output, 1 <= N <= Nmax <= 64,
// a known aperture, finite parameters, and an image size within (C, H, W): equal to it
// (exact: the general-length and fixed-size DFT paths) or any power-of-two size of at
// least 16 within it (the mixed power-of-two path).  Requests that fail are skipped
// and set FDL_ST_BAD_REQUEST.
__device__ __forceinline__ bool request_ok(const fdl_request& r, int C, int H, int W, int Nmax, bool exact) {
  if (r.layers == nullptr || r.d == nullptr || r.out == nullptr) return false;
  // complex64 layers and tables, float32 d; output rows whose width is a multiple of 4 are
  // written as float4
  const uintptr_t out_align = (r.W & 3) == 0 ? 15 : 3;
  if (((uintptr_t)r.layers & 7) != 0 || ((uintptr_t)r.d & 3) != 0 || ((uintptr_t)r.out & out_align) != 0 ||
      ((uintptr_t)r.pts & 7) != 0)
    return false;
  if (r.N < 1 || r.N > Nmax || r.N > 64) return false;
  if (r.aperture < FDL_AP_PINHOLE || r.aperture > FDL_AP_TABLE) return false;
  if ((r.aperture == FDL_AP_POINTS || r.aperture == FDL_AP_TABLE) && r.npts > 0 && r.pts == nullptr) return false;
  if (r.npts < 0 || !(r.radius >= 0.f) || !isfinite(r.radius) || !isfinite(r.u0x) || !isfinite(r.u0y) ||
      !isfinite(r.s))
    return false;
  if (exact) return r.H == H && r.W == W && r.C == C;
  const bool p2 = r.H >= 16 && r.W >= 16 && (r.H & (r.H - 1)) == 0 && (r.W & (r.W - 1)) == 0;
  return p2 && r.H <= H && r.W <= W && r.C >= 1 && r.C <= C;
}

// Every workspace starts with kHeaderInts ints: the counters of a fit and, at index
// kStatusWord, the device status word (FDL_ST_* bits) that fdl_sync_status reads.
constexpr int kHeaderInts = 16;
// Views on an integer lattice |u_x|, |u_y| <= kLatMax (counters[10], set by k_mom_check) let the
// solves form A_jk = P_k^{u_x} Q_k^{u_y} from per-frequency powers.
constexpr int kLatMax = 4;
constexpr int kStatusWord = 15;
constexpr int kGateWord = 14;  // renders: 1 = the tiled path serves the batch, 0 = the mixed path

// ---- tier selection (select.cu) ---------------------------------------------
// sets the status word of a fit from its breakdown and non-finite counters
cudaError_t launch_fit_status(int* counters, cudaStream_t st);
// Appends to `list` the frequencies with the largest err so that the rest keep
// u * sqrt(sum err^2) <= budget * sqrt(sum xn2); scratch of select_scratch_bytes().
size_t select_scratch_bytes();
cudaError_t launch_select_budget(const float* err, const float* xn2, int n, double u, double budget, void* scratch,
                                 int* list, int* count, cudaStream_t st);

// ---- render (render.cu) -----------------------------------------------------
// Nmax: largest N of any request; sizes the shared layer tile used when all
// requests read one FDL.
// shifts: optional [B][N][2] per-layer shifts of each request (the relaxed model's P_jk
// instead of u0 d_k; pinhole requests)
// gate (nullable, device): returns at once unless *gate != 0 (see launch_render_gate).
cudaError_t launch_render_spectra(const fdl_request* req, int B, const int* count, int C, int H, int W, int Nmax,
                                  SpecView out, int* status, cudaStream_t st, const float* shifts = nullptr,
                                  const int* gate = nullptr);
// One CTA: *gate = 1 when every active request is valid, reads the same FDL (layers, d, N)
// and has exactly the size (C, H, W): the tiled path (layer values staged once per tile of
// frequencies and reused by every request) serves it; otherwise 0 and the mixed path does,
// from `plan` (render_plan_ints(B) ints): the runs of consecutive valid requests of one FDL
// and their work items (tiles of 32 frequencies).
size_t render_plan_ints(int B);
cudaError_t launch_render_plan(const fdl_request* req, int B, const int* count, int C, int H, int W, int Nmax,
                               int* gate, int* plan, cudaStream_t st);
// drawn aperture: centred zero-padded raster and its sum (double), then the table scaling
cudaError_t launch_aperture_table_prep(const float* R, int P, int Z, float* pad, double* sum, cudaStream_t st);
cudaError_t launch_aperture_table_scale(float2* T, int Z, const double* sum, cudaStream_t st);
cudaError_t launch_pinhole_requests(fdl_request* req, const float* layers, const float* d, int N, int C, int H,
                                    int W, const float* u0, int B, float* out, cudaStream_t st);
// Mixed render of power-of-two sizes up to 2048 x 4096 (requests of different FDLs and
// sizes within (C, H, W) in one launch): each plan group's layer values staged per tile of
// frequencies and rendered for every request of the group into its slot of `slots` (split
// layout of the request's size, pitch W_b/2, slot_elems complex per request; kx = W_b/2 to
// nyq[(b C + c) H + ky]), then the inverse column DFT of each request in place and the row
// DFT into the requests' outputs.
bool render_mixed_supported(int H, int W);
size_t render_mixed_slot_elems(int C, int H, int W);
// gate (nullable, device): returns at once when *gate != 0.
cudaError_t launch_render_mixed(const fdl_request* req, int B, const int* count, int C, int H, int W, int Nmax,
                                float2* slots, float2* nyq, const int* plan, int* status, cudaStream_t st,
                                const int* gate = nullptr);

// ---- calibration (calib.cu) -------------------------------------------------
struct CalibParams {
  SpecView b;
  const float* u;
  const float* d;
  int K, C, N, H, W;
  int reg;
  float lam;
  const int* bins;     // nullable
  int nbins;
  double* partials;    // [kCalibGrid][1 + 2K + N] per-CTA sums (loss, grad_u, grad_d)
  float* loss;
  float* grad_u;
  float* grad_d;
  int* counters;
  const float4* exp_table;
  bool f64;
  double lam_d;
  const float* P = nullptr;  // free shifts [K][N][2]: dL/dP into grad_P instead of grad_u, grad_d
  float* grad_P = nullptr;   // [K][N][2]
};
constexpr int kCalibGrid = 512;
cudaError_t launch_calib_grad(const CalibParams& p, cudaStream_t st);
// shared-memory accumulators of the free-shift gradient (one CTA): 1 + 2 K N doubles
size_t calib_shifts_acc_bytes(int K, int N);

}  // namespace fdl
