// Inverse 2D real DFT of the FDL path in FP32 (Sec. VI-A: the inverse DFT of a
// rendered spectrum; Sec. VII: only the non-negative-kx half is kept); the
// forward DFT of the views is in fft_df.cu.
//
// Layout of a row-transformed image (the "split" layout): W/2 complex per row
// (pitch W/2, so every row starts on a 16-byte boundary), element 0 packing
// the two real values X[0] + i X[W/2]; after the column pass the kx = W/2
// column lives in a separate [img][H] plane.
//
// Every FFT here is a Stockham autosort FFT (radix 4, one radix-2 pass when
// log2 L is odd) run by a whole CTA on data staged in shared memory.
#include <cstdio>
#include <map>
#include <mutex>
#include <utility>

#include "kernels.h"
#include "stockham.cuh"

namespace fdl {

namespace {

// ---------------------------------------------------------------- row C2R
constexpr int kMaxRowsPerCta = 128;  // R = MAXB T / (M/4), T = max(256, M/4)
template <int MAXB>
__global__ void __launch_bounds__(512) k_irfft_rows(const float2* __restrict__ in, float* __restrict__ out,
                                                    long long nrows, int H, int W, int logM, float scale,
                                                    const fdl_request* __restrict__ req,
                                                    const int* __restrict__ count, int C, int nmax,
                                                    const int* __restrict__ gate) {
  extern __shared__ float2 sm[];
  __shared__ int rowok[kMaxRowsPerCta];
  if (gate != nullptr && *gate == 0) return;
  const int M = W >> 1;
  float2* tw = sm;
  float2* data = sm + M;
  const int q = M >> 2;
  const int R = MAXB * blockDim.x / q;
  const long long row0 = (long long)blockIdx.x * R;
  if (count) nrows = min(nrows, (long long)(*count) * C * H);
  if (row0 >= nrows) return;
  make_twiddles(tw, M);
  float2 h;  // exp(i pi / M)
  sincospif(1.f / (float)M, &h.y, &h.x);
  // rows of requests the render skipped are not written
  for (int rr = threadIdx.x; rr < R; rr += blockDim.x)
    rowok[rr] = req == nullptr || row0 + rr >= nrows || request_ok(req[(row0 + rr) / H / C], C, H, W, nmax, true);
  for (int e = threadIdx.x; e < R * M; e += blockDim.x) {
    const int r = e >> logM;
    float2 v = make_float2(0.f, 0.f);
    if (row0 + r < nrows) v = in[(row0 + r) * M + (e & (M - 1))];
    data[e] = v;
  }
  __syncthreads();
  // Z[k] = E[k] + i O[k], E[k] = X[k] + conj X[M-k],
  // O[k] = (X[k] - conj X[M-k]) exp(+2 pi i k / W); X[0], X[M] are packed in element 0.
  float2 zk[4 * MAXB];  // R * M = 4 * MAXB * blockDim.x elements, 4 * MAXB per thread
#pragma unroll
  for (int i = 0; i < 4 * MAXB; ++i) {
    const int e = threadIdx.x + i * blockDim.x;
    const int r = e >> logM, k = e & (M - 1);
    const float2* X = data + r * M;
    float2 Z;
    if (k == 0) {
      const float x0 = X[0].x, xm = X[0].y;
      Z = make_float2(x0 + xm, x0 - xm);
    } else {
      const float2 a = X[k], bm = X[M - k];
      const float2 E = make_float2(a.x + bm.x, a.y - bm.y);
      float2 O = make_float2(a.x - bm.x, a.y + bm.y);
      O = cmul(O, half_twiddle_conj(tw, k, h));
      Z = make_float2(E.x - O.y, E.y + O.x);
    }
    zk[i] = Z;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4 * MAXB; ++i) data[threadIdx.x + i * blockDim.x] = zk[i];
  __syncthreads();
  int lognfft = 0;
  while ((1 << lognfft) < R) ++lognfft;
  stockham<true, MAXB>(data, tw, M, logM, R, lognfft, M, 1);
  const long long rows_here = min((long long)R, nrows - row0);
  const int valid = (int)rows_here * (W >> 2);
  const int logW4 = logM - 1;
  for (int e = threadIdx.x; e < valid; e += blockDim.x) {
    float4 v = reinterpret_cast<const float4*>(data)[e];
    v.x *= scale;
    v.y *= scale;
    v.z *= scale;
    v.w *= scale;
    const long long row = row0 + (e >> logW4);
    if (!rowok[e >> logW4]) continue;
    float* rowp;
    if (req) {
      const long long img = row / H;
      const int y = (int)(row - img * H);
      const long long b = img / C;
      const int c = (int)(img - b * C);
      rowp = req[b].out + ((long long)c * H + y) * W;
    } else {
      rowp = out + row * W;
    }
    reinterpret_cast<float4*>(rowp)[e & ((W >> 2) - 1)] = v;
  }
}

// ---------------------------------------------------------------- columns
// CTA = one strip of SW columns of one image, all H rows, in shared memory.
template <bool INV, int MAXB>
__global__ void __launch_bounds__(512) k_fft_cols(SpecView in, SpecView out, int H, int logH, int W, int SW,
                                                  int logSW, const int* __restrict__ count, int C,
                                                  const int* __restrict__ gate) {
  extern __shared__ float2 sm[];
  if (gate != nullptr && *gate == 0) return;
  float2* tw = sm;
  float2* data = sm + H;
  const int c0 = blockIdx.x * SW;
  const long long img = blockIdx.y;
  if (count && img >= (long long)(*count) * C) return;
  make_twiddles(tw, H);
  const int n = H * SW;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int y = e >> logSW, c = e & (SW - 1);
    data[e] = in.main[img * in.img_stride + (long long)y * in.pitch + c0 + c];
  }
  __syncthreads();
  if (INV && c0 == 0) {
    // column 0 <- Herm(F0) + i Herm(FN), Herm(F)[ky] = (F[ky] + conj F[-ky]) / 2
    float2 pk[8];
    int cnt = 0;
    const float2* nyq = in.nyq + img * in.nyq_img_stride;
    for (int ky = threadIdx.x; ky < H; ky += blockDim.x, ++cnt) {
      const int km = (H - ky) & (H - 1);
      const float2 f0 = data[ky * SW], f0m = data[km * SW];
      const float2 fn = nyq[(long long)ky * in.nyq_stride], fnm = nyq[(long long)km * in.nyq_stride];
      const float2 h0 = make_float2(0.5f * (f0.x + f0m.x), 0.5f * (f0.y - f0m.y));
      const float2 hn = make_float2(0.5f * (fn.x + fnm.x), 0.5f * (fn.y - fnm.y));
      if (cnt < 8) pk[cnt] = make_float2(h0.x - hn.y, h0.y + hn.x);
    }
    __syncthreads();
    cnt = 0;
    for (int ky = threadIdx.x; ky < H; ky += blockDim.x, ++cnt)
      if (cnt < 8) data[ky * SW] = pk[cnt];
    __syncthreads();
  }
  stockham<INV, MAXB>(data, tw, H, logH, SW, logSW, 1, SW);
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int y = e >> logSW, c = e & (SW - 1);
    out.main[img * out.img_stride + (long long)y * out.pitch + c0 + c] = data[e];
  }
}

// columns per CTA of the inverse column pass: 4096 / H (8 at H = 512, 64-byte row segments;
// measured on 81 views of 512^2 RGB: 16 columns 0.94 ms, 8 columns 0.90 ms, 4 columns 0.91 ms
// for the whole render), within [4, 16]; halved (not below 4) while the launch of nimg images
// would leave SMs without a strip (a single image: its latency is the whole point)
int strip_width(int H, int W, long long nimg) {
  int sw = 4096 / H;
  if (sw > 16) sw = 16;
  if (sw < 4) sw = 4;
  while (sw > 4 && (long long)(W / 2 / sw) * nimg < num_sms()) sw >>= 1;
  if (sw > W / 2) sw = W / 2;
  return sw;
}

template <bool INV>
cudaError_t launch_cols(SpecView in, SpecView out, int nimg, int H, int W, const int* count, int C,
                        cudaStream_t st, const int* gate = nullptr) {
  const int SW = strip_width(H, W, nimg);
  const int T = 512;
  const int bpt = (SW * H / 4 + T - 1) / T;  // butterflies per thread per pass
  const size_t smem = (size_t)(H + SW * H) * sizeof(float2);
  dim3 grid((W / 2) / SW, nimg);
  const int logH = ilog2(H), logSW = ilog2(SW);
  cudaError_t e = cudaSuccess;
#define FDL_COLS(MB)                                                                              \
  {                                                                                               \
    e = set_smem((const void*)k_fft_cols<INV, MB>, smem);                                         \
    if (e != cudaSuccess) return e;                                                               \
    k_fft_cols<INV, MB><<<grid, T, smem, st>>>(in, out, H, logH, W, SW, logSW, count, C, gate);   \
  }
  if (bpt <= 1) FDL_COLS(1)
  else if (bpt <= 2) FDL_COLS(2)
  else if (bpt <= 4) FDL_COLS(4)
  else FDL_COLS(8)
#undef FDL_COLS
  return cudaGetLastError();
}

}  // namespace

cudaError_t set_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = done[{kernel, dev}];
  if (have >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

cudaError_t launch_irfft_rows(const float2* in, float* out, long long nrows, int H, int W, float scale,
                              const fdl_request* req, const int* count, int C, cudaStream_t st, int nmax,
                              const int* gate) {
  // two radix-4 butterflies per thread and pass (R = 2T / (M/4) rows per CTA), one for M < 16
  // where that would exceed kMaxRowsPerCta rows
  const int M = W / 2;
  const int T = (M / 4 > 256) ? M / 4 : 256;
  // one butterfly per thread and pass where two would leave SMs without a CTA (a single image)
  int mb = M >= 16 ? 2 : 1;
  if (mb == 2 && (nrows + 2 * T / (M / 4) - 1) / (2 * T / (M / 4)) < 2 * num_sms()) mb = 1;
  const int R = mb * T / (M / 4);
  const size_t smem = (size_t)(M + R * M) * sizeof(float2);
  const long long grid = (nrows + R - 1) / R;
  cudaError_t e = cudaSuccess;
#define FDL_ROWS(MB)                                                                                  \
  {                                                                                                   \
    e = set_smem((const void*)k_irfft_rows<MB>, smem);                                                \
    if (e != cudaSuccess) return e;                                                                   \
    k_irfft_rows<MB><<<(unsigned)grid, T, smem, st>>>(in, out, nrows, H, W, ilog2(M), scale, req, count, C, \
                                                      nmax, gate);                                    \
  }
  if (mb == 2) FDL_ROWS(2)
  else FDL_ROWS(1)
#undef FDL_ROWS
  return cudaGetLastError();
}

cudaError_t launch_fft_cols_inv(SpecView in, float2* out, int nimg, int H, int W, const int* count, int C,
                                cudaStream_t st, const int* gate) {
  SpecView o = spec_split(out, nullptr, H, W);
  return launch_cols<true>(in, o, nimg, H, W, count, C, st, gate);
}

}  // namespace fdl
