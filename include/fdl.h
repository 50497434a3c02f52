/*
 * fdl.h -- C ABI of the GB300 (sm_103a) Fourier Disparity Layer library.
 *
 * The operations follow Le Pendu, Guillemot, Smolic, "A Fourier Disparity
 * Layer representation for Light Fields" (arXiv 1901.06919):
 *   - layer construction (Sec. V-A): a 2D DFT of every input view, then at
 *     every spatial frequency w the Tikhonov least-squares solve
 *     (A*A + lambda Gamma*Gamma) x = A* b, A_jk = exp(+2 pi i d_k (u_j . w))
 *     (Eqs. AMatGeneral, LayerConstructProb, LayerConstructionClosedForm);
 *   - rendering (Sec. VI-A): the layer spectra phase-shifted, aperture
 *     filtered and summed (Eq. BsFourier), then an inverse DFT;
 *   - calibration (Sec. V-B): the objective of Eq. CalibrationProb and its
 *     gradient with respect to view positions and disparities (Eqs. gradP,
 *     gradD).
 *
 * Conventions used by every entry point.
 *   Memory: every array argument is a DEVICE pointer unless it says "host".
 *     All memory is owned by the caller; the library allocates nothing and
 *     keeps no state between calls.  Scratch memory is a caller workspace
 *     whose size comes from the matching *_workspace_size() query; the
 *     workspace must be 256-byte aligned.
 *   Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 *     only enqueue work; they do not synchronise, except where stated.
 *   Complex numbers: interleaved float pairs (re, im), i.e. complex64.
 *   Images: float32 [C][H][W] row-major (y = row); 16 <= H, W <= 4096, each
 *     a power of two, or a length whose prime factors are all <= 31 (625,
 *     434 = 2 x 7 x 31, 1080, 1920, ...), or any length <= 2048 (379, a
 *     prime; transformed through Bluestein's convolution).  Other sizes are
 *     rejected with FDL_EINVAL.
 *   Spectra: the non-negative-kx half of the 2D DFT, complex64
 *     [..][H][W/2+1] (the layout of torch.fft.rfft2; W/2 rounds down).
 *     Frequencies are in cycles per pixel: w_y = ky/H for ky < (H+1)/2,
 *     (ky-H)/H otherwise; w_x = kx/W for kx = 0..W/2.  The forward DFT is
 *     unnormalised with sign -: b(w) = sum_x B(x) exp(-2 pi i w.x).
 *   Views: u is float32 [K][2] = (u_x, u_y) per view in view-grid units;
 *     a layer of disparity d is seen from u as layer(x + u d) (Appendix A,
 *     Eq. Prior2).  Disparities d are float32 [N], pixels per unit of u.
 *   Errors: every call returns FDL_OK or a positive FDL_E* code and never
 *     aborts; fdl_strerror() names a code.  Invalid arguments are rejected
 *     before anything is enqueued.
 */
#ifndef FDL_H
#define FDL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FDL_API __attribute__((visibility("default")))
#else
#define FDL_API
#endif

/* ---- status codes ------------------------------------------------------ */
#define FDL_OK 0
#define FDL_EINVAL 1   /* bad shape, count, pointer or option              */
#define FDL_ENOMEM 2   /* workspace smaller than the *_workspace_size()    */
#define FDL_ECUDA 3    /* a kernel launch or CUDA runtime call failed       */
#define FDL_ETIMEOUT 4 /* a bounded wait ran out                            */
#define FDL_ENOTSUP 5  /* valid request the library does not support        */

/* ---- device status word ------------------------------------------------
 * Conditions found on the device cannot be returned by the enqueuing call:
 * the kernels OR these bits into a status word at the start of the call's
 * workspace (cleared by each call), read by fdl_sync_status. */
#define FDL_ST_NONFINITE 1   /* fit: a frequency had non-finite input; its layer
                                values are not finite                            */
#define FDL_ST_BREAKDOWN 2   /* fit: the last factorisation of a frequency broke
                                down (a pivot not positive); its layers are zero */
#define FDL_ST_BAD_REQUEST 4 /* render: a request failed the device-side checks
                                (sizes, N, pointers, aperture, parameters) and
                                was skipped; its output is left untouched        */

/* ---- regularisers, Sec. V-C -------------------------------------------- */
#define FDL_REG_VIEW2 0  /* Gamma*Gamma = diag(|w|^4 d_k^4 + eps), Eq. 2ndOrderView */
#define FDL_REG_LAYER2 1 /* Gamma = tridiag(1,-2,1), Eq. 2ndOrderLayer              */
#define FDL_REG_L2 2     /* Gamma = I (Sec. V-C)                                     */

/* ---- arithmetic of the per-frequency solve ----------------------------- */
#define FDL_PREC_MIXED 0 /* FP32 everywhere the estimated FP32 error fits in
                            f32_error_budget; double-float (FP32 pairs,
                            ~2^-48) elsewhere, except the frequencies that
                            native FP64 must take to meet df_error_budget     */
#define FDL_PREC_DF 1    /* double-float at every frequency, certified like the
                            mixed path: the frequencies that native FP64 must
                            take to meet df_error_budget are re-solved in FP64
                            (N <= 48; beyond, double-float only)              */
#define FDL_PREC_F64 2   /* native FP64 at every frequency                    */
#define FDL_PREC_F32 3   /* FP32 at every frequency, no certification         */

/* ---- apertures psi of Eq. refocus, normalised to integrate to 1 ------- */
#define FDL_AP_PINHOLE 0 /* psi = delta: psi_hat = 1 (sub-aperture image)    */
#define FDL_AP_DISC 1    /* disc of radius r: 2 J1(2 pi r|v|) / (2 pi r|v|)    */
#define FDL_AP_SQUARE 2  /* square of half side r: sinc(2 r v_x) sinc(2 r v_y) */
#define FDL_AP_POINTS 3  /* (1/M) sum_m delta(u - u_m): discrete aperture     */
#define FDL_AP_TABLE 4   /* drawn aperture: psi_hat interpolated bilinearly in a
                            table of fdl_aperture_table (Sec. VI-A)            */

typedef struct fdl_fit_opts {
  double lambda;    /* Tikhonov weight lambda of Eq. LayerConstructProb, >= 0      */
  double eps;       /* epsilon added to the view regulariser's diagonal (Sec. V-C1;
                       the diagonal is lambda (|w|^4 d^4 + eps)); unused otherwise */
  int reg;          /* FDL_REG_*                                                   */
  int precision;    /* FDL_PREC_*                                                  */
  double kappa_max; /* FDL_PREC_MIXED: largest estimated condition number of
                       A*A + lambda Gamma*Gamma whose FP32 solution may be kept at
                       all; above it the estimate itself is not trusted
                       (<= 0 selects the default, 1e6)                             */
  double df_error_budget; /* FDL_PREC_MIXED, FDL_PREC_DF: estimated relative L2 error that the
                             double-float frequencies may leave in the layers; the
                             frequencies with the largest estimated errors (condition
                             estimate x solution norm), and any whose double-float
                             factorisation breaks down, are re-solved in native FP64
                             until the estimate of the rest is within it
                             (<= 0 selects the default, 4e-6; N <= 48 only)        */
  double f32_error_budget; /* FDL_PREC_MIXED, N <= 32: the same for the FP32 pass:
                              the frequencies with the largest estimated FP32
                              errors (and those above kappa_max, with a
                              factorisation that broke down or non-finite input)
                              are re-solved in double-float until the estimate of
                              the rest is within it (<= 0 selects the default, 2e-6) */
} fdl_fit_opts;

/* One image to render (Eq. BsFourier): the FDL it reads, the viewpoint u0,
 * the focus disparity s, the aperture and the image size.  The descriptors
 * live in device memory, so the host cannot check them: the kernels do
 * (request_ok in the library) and skip a request that fails, setting
 * FDL_ST_BAD_REQUEST. */
typedef struct fdl_request {
  const float* layers; /* device complex64 [N][C][H][W/2+1]                     */
  const float* d;      /* device float32 [N]                                    */
  float* out;          /* device float32 [C][H][W]                              */
  const float* pts;    /* FDL_AP_POINTS: device float32 [npts][2] offsets u_m;
                          FDL_AP_TABLE: device complex64 [npts][npts/2+1], a
                          table of fdl_aperture_table with Z = npts            */
  int N, npts;
  int aperture;        /* FDL_AP_*                                              */
  float u0x, u0y;      /* viewpoint on the camera plane                         */
  float s;             /* refocus parameter (disparity in focus), Sec. III      */
  float radius;        /* disc radius / square half side, in units of u (the
                          aperture-size factor f of Sec. VI-A); FDL_AP_TABLE:
                          the raster pitch h, in units of u                     */
  int H, W, C;         /* image size of the FDL and of `out`                    */
  int pad_[2];         /* keeps the struct 80 bytes; set to 0                   */
} fdl_request;

FDL_API const char* fdl_strerror(int status);
FDL_API int fdl_version(void);

/* ---- 2D real DFTs (Sec. V-A: "discrete Fourier Transform of each image";
 *      Sec. VI-A: inverse transform; Sec. VII: half spectrum) ------------ */

/* spectra[i] = half spectrum of image i, for nimg images [nimg][H][W]. */
FDL_API size_t fdl_rfft2_workspace_size(int nimg, int H, int W);
FDL_API int fdl_rfft2(const float* images, int nimg, int H, int W, float* spectra,
                      void* workspace, size_t workspace_bytes, void* stream);

/* images[i] = Re(inverse DFT of spectrum i completed by X(-w) = conj X(w)) / (H W),
 * i.e. the kx = 0 and kx = W/2 columns count through their Hermitian part. */
FDL_API size_t fdl_irfft2_workspace_size(int nimg, int H, int W);
FDL_API int fdl_irfft2(const float* spectra, int nimg, int H, int W, float* images,
                       void* workspace, size_t workspace_bytes, void* stream);

/* ---- layer construction (Sec. V-A) ------------------------------------ */

/* views [K][C][H][W] float32, u [K][2], d [N]  ->  layers [N][C][H][W/2+1]
 * complex64.  1 <= N <= 64, 1 <= K <= 1024, 1 <= C <= 4.  The channels share A and Gamma: one factorisation per
 * frequency serves all C right-hand sides.  The spectra of the views are
 * kept in the workspace. */
FDL_API size_t fdl_fit_workspace_size(int K, int C, int H, int W, int N);
FDL_API int fdl_fit(const float* views, int K, int C, int H, int W, const float* u,
                    const float* d, int N, const fdl_fit_opts* opts, float* layers,
                    void* workspace, size_t workspace_bytes, void* stream);

/* Same solve from precomputed half spectra [K][C][H][W/2+1] complex64. */
FDL_API size_t fdl_fit_spectra_workspace_size(int K, int C, int H, int W, int N);
FDL_API int fdl_fit_spectra(const float* spectra, int K, int C, int H, int W,
                            const float* u, const float* d, int N, const fdl_fit_opts* opts,
                            float* layers, void* workspace, size_t workspace_bytes,
                            void* stream);

/* fdl_fit_spectra without a workspace, for callers that may not allocate device
 * memory: real-time loops that cannot afford cudaMalloc's implicit
 * synchronisation, and hosts (plugins, renderers, frameworks with their own
 * caching allocator) that own the whole device-memory budget and forbid
 * allocations by libraries.
 * The paper has no counterpart: this is an integration variant only.
 * Its scratch is a fixed array inside the library (8,455,168 bytes on every
 * GPU that loads it, held until the process exits); H * (W/2 + 1) must not
 * exceed 525,312 (a 1024 x 1024 image), otherwise FDL_ENOMEM.  The first call
 * on each device looks up the array's device address, so make it before any
 * stream capture.  All calls on a device share the array: calls that may run
 * at the same time on the GPU (different streams, or different host threads)
 * race and must be serialised by the caller.  The counters of
 * fdl_fit_tier_counts are not available for this variant. */
FDL_API int fdl_fit_spectra_noalloc(const float* spectra, int K, int C, int H, int W, const float* u,
                                    const float* d, int N, const fdl_fit_opts* opts, float* layers,
                                    void* stream);

/* The device status word (FDL_ST_* bits, 0 if nothing was found) of the last
 * call that used `workspace`: fdl_fit, fdl_fit_spectra, fdl_fit_general,
 * fdl_render, fdl_refocus or fdl_render_shifts.  status is a HOST int; this
 * call synchronises `stream` (the call's stream).  The error convention of the
 * boundary: FDL_E* codes for what the host can check before enqueuing,
 * FDL_ST_* bits for what only the kernels see. */
FDL_API int fdl_sync_status(const void* workspace, int* status, void* stream);

/* After fdl_fit / fdl_fit_spectra on `stream`: counts[0] = frequencies solved
 * in FP32, counts[1] = in double-float, counts[2] = in native FP64,
 * counts[3] = frequencies whose last factorisation broke down (left as
 * zeros), counts[4] = frequencies with non-finite input.  counts is a HOST
 * int[5]; this call synchronises `stream`. */
FDL_API int fdl_fit_tier_counts(const void* workspace, int* counts, void* stream);

/* ---- rendering (Sec. VI-A, Eq. FourierView / Eq. BsFourier) ----------- */

/* B sub-aperture views of one FDL at viewpoints u0 [B][2] (psi = delta):
 * out [B][C][H][W].  The layer values of each tile of frequencies are read
 * once and shared by the B views.  B <= 65535. */
FDL_API size_t fdl_render_workspace_size(int B, int C, int H, int W);
FDL_API int fdl_render(const float* layers, const float* d, int N, int C, int H, int W,
                       const float* u0, int B, float* out, void* workspace,
                       size_t workspace_bytes, void* stream);

/* B general images, each described by a request (req: DEVICE array [B]).
 * C, H, W, Nmax bound every request: when H and W are powers of two and
 * H <= 2048, requests of ANY power-of-two sizes H_b <= H, W_b <= W (>= 16)
 * and C_b <= C share the launch (mixed FDLs and image sizes); each is
 * rendered by Eq. BsFourier straight into the inverse column DFT (the
 * rendered spectrum is never written to memory), then the inverse row DFT
 * writes its output.  Otherwise (sizes that are not powers of two, or
 * H = 4096), and for a single request (B = 1), every request must have
 * exactly H x W x C.  If count is not NULL
 * it is a DEVICE int: only requests [0, *count) are rendered, so that a
 * captured CUDA graph can be replayed with a varying batch.  Nmax <= 64. */
FDL_API size_t fdl_refocus_workspace_size(int B, int C, int H, int W);
FDL_API int fdl_refocus(const fdl_request* req, int B, const int* count, int C, int H,
                        int W, int Nmax, void* workspace, size_t workspace_bytes,
                        void* stream);

/* One light field from host memory to host memory: the views (HOST
 * float32 [K][C][H][W], pinned for an asynchronous copy) are copied into the
 * workspace, fitted into `layers` (DEVICE
 * [N][C][H][W/2+1]) as by
 * fdl_fit, the B requests (DEVICE array, as for fdl_refocus with bounds C, H,
 * W and Nmax = N; they read `layers` and write inside `images`) are rendered,
 * and `images` (DEVICE, image_floats floats) is copied to images_host (HOST,
 * pinned).  Everything is enqueued on `stream`; callers overlap the copies of
 * one light field with the computation of another by alternating two streams
 * and two sets of buffers.  Workspace: fdl_fit_render_host_workspace_size. */
FDL_API size_t fdl_fit_render_host_workspace_size(int K, int C, int H, int W, int N, int B);
FDL_API int fdl_fit_render_host(const float* views_host, int K, int C, int H, int W, const float* u,
                                const float* d, int N, const fdl_fit_opts* opts, float* layers,
                                const fdl_request* req, int B, float* images, size_t image_floats,
                                float* images_host, void* workspace, size_t workspace_bytes,
                                void* stream);

/* Table of a drawn aperture (Sec. VI-A: the aperture is drawn, zero-padded
 * and transformed, and psi_hat is linearly interpolated).  raster: DEVICE
 * float32 [P][P], P odd, 1 <= P <= Z; pixel (iy, ix) sits at u = ((ix - c) h,
 * (iy - c) h), c = (P-1)/2, for the pitch h that the requests give in
 * `radius`.  table: DEVICE complex64 [Z][Z/2+1] = psi_hat at nu = (gy, gx) /
 * (Z h) for the stored half, normalised so that psi_hat(0) = 1 (the raster's
 * sum must be positive).  Z is an image size the DFTs accept.  A request with
 * FDL_AP_TABLE interpolates it bilinearly, periodic in Z, with psi_hat(-nu) =
 * conj psi_hat(nu) for the columns not stored. */
FDL_API size_t fdl_aperture_table_workspace_size(int P, int Z);
FDL_API int fdl_aperture_table(const float* raster, int P, int Z, float* table, void* workspace,
                               size_t workspace_bytes, void* stream);

/* ---- the general system (Eq. AMatGeneral) ------------------------------ */
/* Images j of any kind (Sec. V: "the model of Eq. refocus"): a sub-aperture
 * view, an image with its own aperture psi_j and focus s_j (focal stacks,
 * hybrid captures), and shifts either u_j d_k or free P_jk (the relaxed FDL
 * model of the denoising application, which drops the rank-1 constraint
 * P = u d^T):  A_jk = exp(+2 pi i P_jk . w) psi_hat_j((s_j - d_k) w). */
typedef struct fdl_system {
  const float* u;           /* DEVICE float32 [K][2] view positions (with d), or NULL with P */
  const float* d;           /* DEVICE float32 [N] layer disparities: the shifts u_j d_k (without P),
                               the view regulariser and the aperture argument (s_j - d_k) w */
  const float* P;           /* DEVICE float32 [K][N][2] free shifts (x, y) in pixels, or NULL */
  const fdl_request* views; /* DEVICE [K]: aperture, radius, s, pts, npts of each image, or NULL
                               (every image a sub-aperture view); other fields ignored       */
} fdl_system;

/* Layer construction (Eq. LayerConstructionClosedForm) for the general system from
 * half spectra [K][C][H][W/2+1], with the shared-memory solver at every
 * frequency: native FP64 for FDL_PREC_F64, double-float otherwise (no tiers).
 * Needs P or both u and d; views and FDL_REG_VIEW2 need d.  N <= 64. */
FDL_API size_t fdl_fit_general_workspace_size(int K, int C, int H, int W, int N);
FDL_API int fdl_fit_general(const float* spectra, int K, int C, int H, int W, int N,
                            const fdl_system* sys, const fdl_fit_opts* opts, float* layers,
                            void* workspace, size_t workspace_bytes, void* stream);

/* Images rendered with per-layer shifts (the relaxed model: an input view j is
 * rendered with P_jk instead of u_j d_k; pinhole).  P: DEVICE float32 [B][N][2]
 * (the shifts of output image b); out: DEVICE float32 [B][C][H][W]. */
FDL_API size_t fdl_render_shifts_workspace_size(int B, int C, int H, int W);
FDL_API int fdl_render_shifts(const float* layers, const float* P, int N, int C, int H, int W, int B,
                              float* out, void* workspace, size_t workspace_bytes, void* stream);

/* The calibration objective over bins (as fdl_calib_grad) with free shifts P
 * [K][N][2] and its gradient grad_P = dloss/dP [K][N][2] by Eq. gradP (the
 * relaxed model searches P directly).  reg must be FDL_REG_LAYER2 or FDL_REG_L2;
 * FDL_ENOTSUP when (1 + 2 K N) doubles plus the solver's matrices exceed the
 * shared memory of one block (about K N <= 10,000). */
FDL_API size_t fdl_calib_grad_shifts_workspace_size(int K, int C, int H, int W, int N, int nbins);
FDL_API int fdl_calib_grad_shifts(const float* spectra, int K, int C, int H, int W, const float* P, int N,
                                  const fdl_fit_opts* opts, const int* bins, int nbins, float* loss,
                                  float* grad_P, void* workspace, size_t workspace_bytes, void* stream);

/* ---- calibration (Sec. V-B) ------------------------------------------- */

/* Over the frequencies listed in bins (DEVICE int [nbins], flattened index
 * ky*(W/2+1)+kx of the stored half; NULL = every stored frequency), with the
 * layers x re-solved at the current u, d by the closed form:
 *   loss   = sum_{bins, c} |A x - b|^2 + lambda |Gamma x|^2 (Eq. CalibrationProb)
 *   grad_u = dloss/du [K][2], grad_d = dloss/dd [N]      (Eqs. gradP, gradD)
 * loss is a DEVICE float [1]; reg must be FDL_REG_LAYER2 or FDL_REG_L2
 * (a regulariser that does not depend on d).  Arithmetic follows
 * opts->precision as in fdl_fit. */
FDL_API size_t fdl_calib_grad_workspace_size(int K, int C, int H, int W, int N, int nbins);
FDL_API int fdl_calib_grad(const float* spectra, int K, int C, int H, int W, const float* u,
                           const float* d, int N, const fdl_fit_opts* opts, const int* bins,
                           int nbins, float* loss, float* grad_u, float* grad_d,
                           void* workspace, size_t workspace_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FDL_H */
