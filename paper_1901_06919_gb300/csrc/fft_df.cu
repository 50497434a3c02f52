// Forward 2D real DFT (Sec. V-A) with double-float arithmetic inside each pass.
//
// The layer solve amplifies errors of the input spectra (most at the
// ill-conditioned frequencies), so the forward transform of the views runs
// its butterflies and twiddle products in double-float (pairs of floats) and
// rounds to complex64 once at the end of each pass: the row pass and the
// column pass together stay within about two roundings of the exact DFT.
// Same data layout and Stockham structure as fft.cu (radix 4, one radix-2
// pass when log2 L is odd); twiddles come from a double-float table built by
// k_twiddle_table with FP64 sincospi.
#include "kernels.h"

namespace fdl {

namespace {

struct dcx {
  df re, im;
};

// Butterfly sums use the "sloppy" double-word addition of Joldes, Muller and
// Popescu (ACM TOMS 2017): its error is bounded by about 2^-46 (|a| + |b|)
// instead of 2^-46 |a + b|.  A DFT's error bound is normwise (relative to the
// norm of the input), so that weaker bound costs nothing here and saves about
// half the operations of the accurate addition.
__device__ __forceinline__ df sadd(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  const float w = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, w);
}
__device__ __forceinline__ df ssub(df a, df b) { return sadd(a, df_neg(b)); }
__device__ __forceinline__ dcx dadd(const dcx& a, const dcx& b) { return {sadd(a.re, b.re), sadd(a.im, b.im)}; }
__device__ __forceinline__ dcx dsub(const dcx& a, const dcx& b) { return {ssub(a.re, b.re), ssub(a.im, b.im)}; }
__device__ __forceinline__ dcx dmul(const dcx& a, const dcx& b) {
  return {ssub(df_mul(a.re, b.re), df_mul(a.im, b.im)), sadd(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ dcx dscale(const dcx& a, float s) { return {df_mul_f(a.re, s), df_mul_f(a.im, s)}; }
// stored as float4 (re.hi, im.hi, re.lo, im.lo)
__device__ __forceinline__ float4 dpack(const dcx& a) { return make_float4(a.re.hi, a.im.hi, a.re.lo, a.im.lo); }
__device__ __forceinline__ dcx dunpack(float4 v) { return {{v.x, v.z}, {v.y, v.w}}; }
__device__ __forceinline__ float2 dround(const dcx& a) { return make_float2(a.re.hi + a.re.lo, a.im.hi + a.im.lo); }

// twiddle exp(-2 pi i t / L) = table[t * (T / L)] for a table of length T
__device__ __forceinline__ dcx tw_at(const float4* tab, int i) { return dunpack(tab[i]); }

__device__ __forceinline__ void radix4_df(dcx& a0, dcx& a1, dcx& a2, dcx& a3) {
  const dcx t0 = dadd(a0, a2), t1 = dsub(a0, a2), t2 = dadd(a1, a3);
  dcx t3 = dsub(a1, a3);
  t3 = {t3.im, {-t3.re.hi, -t3.re.lo}};  // times -i
  a0 = dadd(t0, t2);
  a2 = dsub(t0, t2);
  a1 = dadd(t1, t3);
  a3 = dsub(t1, t3);
}

// In-place forward DFTs of nfft sequences of length L in shared memory
// (element (f, n) at s[f * fstride + n * estride]); tab holds exp(-2 pi i t / T)
// for t < T with T a multiple of L.
template <int MAXB>
__device__ __forceinline__ void stockham_df(float4* s, const float4* tab, int tscale, int L, int logL, int nfft,
                                            int lognfft, int fstride, int estride) {
  const int q = L >> 2;
  const int logq = logL - 2;
  const int total = nfft * q;
  const bool fmajor = (fstride == 1);
  int Ns = 1, logNs = 0;
  for (int pass = 0; pass < (logL >> 1); ++pass) {
    dcx v[MAXB][4];
    int ob[MAXB];
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
      const int task = threadIdx.x + b * blockDim.x;
      if (task < total) {
        int f, j;
        if (fmajor) {
          f = task & (nfft - 1);
          j = task >> lognfft;
        } else {
          f = task >> logq;
          j = task & (q - 1);
        }
        float4* p = s + f * fstride;
        const int k = j & (Ns - 1);
        dcx a0 = dunpack(p[j * estride]), a1 = dunpack(p[(j + q) * estride]);
        dcx a2 = dunpack(p[(j + 2 * q) * estride]), a3 = dunpack(p[(j + 3 * q) * estride]);
        if (pass > 0) {
          const int step = k << (logq - logNs);
          a1 = dmul(a1, tw_at(tab, step * tscale));
          a2 = dmul(a2, tw_at(tab, 2 * step * tscale));
          a3 = dmul(a3, tw_at(tab, 3 * step * tscale));
        }
        radix4_df(a0, a1, a2, a3);
        v[b][0] = a0;
        v[b][1] = a1;
        v[b][2] = a2;
        v[b][3] = a3;
        ob[b] = f * fstride + (((j - k) << 2) + k) * estride;
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
      const int task = threadIdx.x + b * blockDim.x;
      if (task < total) {
        const int e = Ns * estride;
        s[ob[b]] = dpack(v[b][0]);
        s[ob[b] + e] = dpack(v[b][1]);
        s[ob[b] + 2 * e] = dpack(v[b][2]);
        s[ob[b] + 3 * e] = dpack(v[b][3]);
      }
    }
    __syncthreads();
    Ns <<= 2;
    logNs += 2;
  }
  if (logL & 1) {
    const int h = L >> 1;
    const int logh = logL - 1;
    const int total2 = nfft * h;
#pragma unroll
    for (int b = 0; b < 2 * MAXB; ++b) {
      const int task = threadIdx.x + b * blockDim.x;
      if (task < total2) {
        int f, j;
        if (fmajor) {
          f = task & (nfft - 1);
          j = task >> lognfft;
        } else {
          f = task >> logh;
          j = task & (h - 1);
        }
        float4* p = s + f * fstride;
        const dcx a0 = dunpack(p[j * estride]);
        const dcx a1 = dmul(dunpack(p[(j + h) * estride]), tw_at(tab, j * tscale));
        p[j * estride] = dpack(dadd(a0, a1));
        p[(j + h) * estride] = dpack(dsub(a0, a1));
      }
    }
    __syncthreads();
  }
}

// table[t] = exp(-2 pi i t / T), t < T, double-float
__global__ void k_twiddle_table(float4* table, int T) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < T) {
    double s, c;
    sincospi(-2.0 * (double)t / (double)T, &s, &c);
    const float ch = (float)c, sh = (float)s;
    table[t] = make_float4(ch, sh, (float)(c - (double)ch), (float)(s - (double)sh));
  }
}

// Row pass: R rows per CTA, each W reals -> W/2 complex (element 0 packs X[0] + i X[W/2]).
__global__ void __launch_bounds__(512) k_rfft_rows_df(const float* __restrict__ in, float2* __restrict__ out,
                                                      long long nrows, int W, int logM, const float4* __restrict__ tabW) {
  extern __shared__ float4 sm4[];
  const int M = W >> 1;
  float4* tab = sm4;          // [W]: exp(-2 pi i t / W)
  float4* data = sm4 + W;     // [R][M]
  const int q = M >> 2;
  const int R = blockDim.x / q;
  const long long row0 = (long long)blockIdx.x * R;
  for (int t = threadIdx.x; t < W; t += blockDim.x) tab[t] = tabW[t];
  const long long rows_here = min((long long)R, nrows - row0);
  for (int e = threadIdx.x; e < R * M; e += blockDim.x) {
    const int r = e >> logM;
    float2 z = make_float2(0.f, 0.f);
    if (r < rows_here) z = __ldg(reinterpret_cast<const float2*>(in + (row0 + r) * W) + (e & (M - 1)));
    data[e] = make_float4(z.x, z.y, 0.f, 0.f);  // z[n] = x[2n] + i x[2n+1], exact
  }
  __syncthreads();
  int lognfft = 0;
  while ((1 << lognfft) < R) ++lognfft;
  stockham_df<1>(data, tab, 2, M, logM, R, lognfft, M, 1);
  for (int e = threadIdx.x; e < R * M; e += blockDim.x) {
    const int r = e >> logM, k = e & (M - 1);
    const long long row = row0 + r;
    if (row >= nrows) continue;
    const float4* z = data + r * M;
    const dcx Zk = dunpack(z[k]);
    dcx o;
    if (k == 0) {
      o = {sadd(Zk.re, Zk.im), ssub(Zk.re, Zk.im)};
    } else {
      const dcx Zm = dunpack(z[M - k]);
      // E = (Zk + conj Zm)/2, O = (Zk - conj Zm)/(2i), X = E + exp(-2 pi i k / W) O
      const dcx E = dscale({sadd(Zk.re, Zm.re), ssub(Zk.im, Zm.im)}, 0.5f);
      const dcx O = dscale({sadd(Zk.im, Zm.im), ssub(Zm.re, Zk.re)}, 0.5f);
      o = dadd(E, dmul(tw_at(tab, k), O));
    }
    out[row * M + k] = dround(o);
  }
}

// Column pass (forward): strip of SW columns of one image, all H rows.
template <int MAXB>
__global__ void __launch_bounds__(512) k_fft_cols_df(SpecView in, SpecView out, int H, int logH, int SW, int logSW,
                                                     const float4* __restrict__ tabH) {
  extern __shared__ float4 sm4[];
  float4* tab = sm4;
  float4* data = sm4 + H;
  const int c0 = blockIdx.x * SW;
  const long long img = blockIdx.y;
  for (int t = threadIdx.x; t < H; t += blockDim.x) tab[t] = tabH[t];
  const int n = H * SW;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int y = e >> logSW, c = e & (SW - 1);
    const float2 v = in.main[img * in.img_stride + (long long)y * in.pitch + c0 + c];
    data[e] = make_float4(v.x, v.y, 0.f, 0.f);
  }
  __syncthreads();
  stockham_df<MAXB>(data, tab, 1, H, logH, SW, logSW, 1, SW);
  if (c0 == 0) {
    // unpack column 0: Z = F0 + i FN with F0, FN the DFTs of the real columns X[0], X[W/2]
    float2 f0v[8];
    int cnt = 0;
    float2* nyq = out.nyq + img * out.nyq_img_stride;
    for (int ky = threadIdx.x; ky < H; ky += blockDim.x, ++cnt) {
      const int km = (H - ky) & (H - 1);
      const dcx z = dunpack(data[ky * SW]), zm = dunpack(data[km * SW]);
      const dcx f0 = dscale({sadd(z.re, zm.re), ssub(z.im, zm.im)}, 0.5f);
      const dcx fn = dscale({sadd(z.im, zm.im), ssub(zm.re, z.re)}, 0.5f);
      nyq[(long long)ky * out.nyq_stride] = dround(fn);
      if (cnt < 8) f0v[cnt] = dround(f0);
    }
    __syncthreads();
    cnt = 0;
    for (int ky = threadIdx.x; ky < H; ky += blockDim.x, ++cnt)
      if (cnt < 8) data[ky * SW] = make_float4(f0v[cnt].x, f0v[cnt].y, 0.f, 0.f);
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int y = e >> logSW, c = e & (SW - 1);
    const float4 v = data[e];
    out.main[img * out.img_stride + (long long)y * out.pitch + c0 + c] = make_float2(v.x + v.z, v.y + v.w);
  }
}

// columns per CTA of the forward column pass: 2048 / H (4 at H = 512; the 243 images of 512^2
// RGB took 1.31 / 1.13 / 1.11 ms with 16 / 8 / 4 columns), within [2, 16]
int strip_width_df(int H, int W) {
  int sw = 2048 / H;
  if (sw > 16) sw = 16;
  if (sw < 2) sw = 2;
  if (sw > W / 2) sw = W / 2;
  return sw;
}

}  // namespace

size_t fft_df_table_bytes(int H, int W) { return (size_t)(H + W) * sizeof(float4); }

cudaError_t launch_twiddle_tables(float4* tables, int H, int W, cudaStream_t st) {
  k_twiddle_table<<<(W + 255) / 256, 256, 0, st>>>(tables, W);
  k_twiddle_table<<<(H + 255) / 256, 256, 0, st>>>(tables + W, H);
  return cudaGetLastError();
}

cudaError_t launch_rfft_rows_df(const float* in, float2* out, long long nrows, int W, const float4* tables,
                                cudaStream_t st) {
  const int M = W / 2;
  const int T = (M / 4 > 256) ? M / 4 : 256;
  const int R = T / (M / 4);
  const size_t smem = (size_t)(W + R * M) * sizeof(float4);
  cudaError_t e = set_smem((const void*)k_rfft_rows_df, smem);
  if (e != cudaSuccess) return e;
  const long long grid = (nrows + R - 1) / R;
  k_rfft_rows_df<<<(unsigned)grid, T, smem, st>>>(in, out, nrows, W, ilog2(M), tables);
  return cudaGetLastError();
}

cudaError_t launch_fft_cols_fwd_df(SpecView in, SpecView out, int nimg, int H, int W, const float4* tables,
                                   cudaStream_t st) {
  const int SW = strip_width_df(H, W);
  const int T = 512;
  const int bpt = (SW * H / 4 + T - 1) / T;
  const size_t smem = (size_t)(H + SW * H) * sizeof(float4);
  dim3 grid((W / 2) / SW, nimg);
  const int logH = ilog2(H), logSW = ilog2(SW);
  const float4* tabH = tables + W;
  cudaError_t e = cudaSuccess;
#define FDL_COLS_DF(MB)                                                              \
  {                                                                                  \
    e = set_smem((const void*)k_fft_cols_df<MB>, smem);                              \
    if (e != cudaSuccess) return e;                                                  \
    k_fft_cols_df<MB><<<grid, T, smem, st>>>(in, out, H, logH, SW, logSW, tabH);     \
  }
  if (bpt <= 1) FDL_COLS_DF(1)
  else if (bpt <= 2) FDL_COLS_DF(2)
  else FDL_COLS_DF(4)
#undef FDL_COLS_DF
  return cudaGetLastError();
}

}  // namespace fdl
