// Discrete Fourier transforms of lengths that are not powers of two, for the
// DFT of every view (Sec. V-A) and the inverse DFT of a render (Sec. VI-A) on
// the paper's light fields of 625 x 434, 379 x 379 or 1920 x 1080 pixels.
//
// A length L whose prime factors are all <= kGenMaxRadix is transformed by
// Stockham passes of those radices in shared memory: pass r turns sequences of
// Ns-point transforms into (Ns r)-point ones,
//   out[jhi Ns r + u Ns + k] = sum_t in[j + t L/r] exp(-2 pi i t (k + u Ns) / (Ns r)),
// j = jhi Ns + k, one table lookup exp(-2 pi i n / L) per term.  Any other
// length (L <= 2048) goes through Bluestein's identity
//   X[k] = c_k sum_n (x_n c_n) conj(c_{k-n}),  c_n = exp(-i pi n^2 / L),
// a cyclic convolution of power-of-two length M >= 2L - 1 done with two such
// transforms and the precomputed transform of conj(c).  All arithmetic is
// double-float (complex values stored as float4 re.hi, im.hi, re.lo, im.lo);
// the tables come from FP64 sincospi with the angle reduced in integers.
// The inverse transform is conj(DFT(conj(X))).
#include "kernels.h"

namespace fdl {

namespace {

struct dcx {
  df re, im;
};
__device__ __forceinline__ dcx dadd(const dcx& a, const dcx& b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ dcx dmul(const dcx& a, const dcx& b) {
  return {df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ float4 dpack(const dcx& a) { return make_float4(a.re.hi, a.im.hi, a.re.lo, a.im.lo); }
__device__ __forceinline__ dcx dunpack(float4 v) { return {{v.x, v.z}, {v.y, v.w}}; }
__device__ __forceinline__ float4 conj4(float4 v) { return make_float4(v.x, -v.y, v.z, -v.w); }
__device__ __forceinline__ float4 df_from_double2(double re, double im) {
  const float rh = (float)re, ih = (float)im;
  return make_float4(rh, ih, (float)(re - (double)rh), (float)(im - (double)ih));
}

constexpr int kGenThreads = 256;
constexpr size_t kGenSmemBudget = 96 * 1024;  // per CTA, both ping-pong buffers

// Stockham passes over nseq sequences of length L at a[f * L + n]; ping-pong with b.
// Returns the buffer that holds the result.
__device__ float4* gen_passes(float4* a, float4* b, int nseq, int L, const int* radix, int np,
                              const float4* __restrict__ tw) {
  int Ns = 1;
  for (int i = 0; i < np; ++i) {
    const int r = radix[i];
    const int Lr = L / r, NsR = Ns * r, stepT = L / NsR;
    for (int task = threadIdx.x; task < nseq * L; task += blockDim.x) {
      const int f = task / L, o = task - f * L;
      const int jhi = o / NsR, rem = o - jhi * NsR;
      const int u = rem / Ns, k = rem - u * Ns;
      const int j = jhi * Ns + k;
      const float4* in = a + f * L;
      dcx acc = dunpack(in[j]);
      const int tstep = (k + u * Ns) * stepT;  // < L
      int ti = 0;
      for (int t = 1; t < r; ++t) {
        ti += tstep;
        if (ti >= L) ti -= L;
        acc = dadd(acc, dmul(dunpack(in[j + t * Lr]), dunpack(__ldg(tw + ti))));
      }
      b[f * L + o] = dpack(acc);
    }
    __syncthreads();
    float4* t = a;
    a = b;
    b = t;
    Ns = NsR;
  }
  return a;
}

// Transform of nseq sequences held at a[f * Leff + n] (Leff = L, or M with Bluestein, the
// entries n >= L zero); the result X[k], k < L, ends at ret[f * Leff + k].
__device__ float4* gen_transform(float4* a, float4* b, int nseq, const GenPlan& P, const float4* __restrict__ tab,
                                 bool inverse) {
  if (P.M == 0) {
    if (inverse) {
      for (int e = threadIdx.x; e < nseq * P.L; e += blockDim.x) a[e] = conj4(a[e]);
      __syncthreads();
    }
    float4* r = gen_passes(a, b, nseq, P.L, P.radix, P.np, tab + P.tw);
    if (inverse) {
      for (int e = threadIdx.x; e < nseq * P.L; e += blockDim.x) r[e] = conj4(r[e]);
      __syncthreads();
    }
    return r;
  }
  const int M = P.M, L = P.L;
  const float4* chirp = tab + P.chirp;
  for (int e = threadIdx.x; e < nseq * M; e += blockDim.x) {
    const int n = e % M;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (n < L) {
      const float4 x = inverse ? conj4(a[e]) : a[e];
      v = dpack(dmul(dunpack(x), dunpack(__ldg(chirp + n))));
    }
    a[e] = v;
  }
  __syncthreads();
  float4* r = gen_passes(a, b, nseq, M, P.mradix, P.mp, tab + P.twm);
  float4* o = r == a ? b : a;
  const float4* bhat = tab + P.bhat;
  for (int e = threadIdx.x; e < nseq * M; e += blockDim.x)
    r[e] = conj4(dpack(dmul(dunpack(r[e]), dunpack(__ldg(bhat + e % M)))));
  __syncthreads();
  r = gen_passes(r, o, nseq, M, P.mradix, P.mp, tab + P.twm);
  const float invM = 1.f / (float)M;  // M is a power of two: exact
  for (int e = threadIdx.x; e < nseq * M; e += blockDim.x) {
    const int k = e % M;
    if (k < L) {
      float4 c = conj4(r[e]);
      c = make_float4(c.x * invM, c.y * invM, c.z * invM, c.w * invM);
      float4 x = dpack(dmul(dunpack(c), dunpack(__ldg(chirp + k))));
      r[e] = inverse ? conj4(x) : x;
    }
  }
  __syncthreads();
  return r;
}

// ---- tables ---------------------------------------------------------------

__global__ void k_gen_twiddles(float4* tw, int L) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < L; n += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)n / (double)L, &s, &c);
    tw[n] = df_from_double2(c, s);
  }
}

// c_n = exp(-i pi n^2 / L) with n^2 reduced modulo 2L in integers; b = conj(c) wrapped
// into length M (b_m at m and M - m), to be transformed in place by k_gen_bhat
__global__ void k_gen_chirp(float4* chirp, float4* bhat, int L, int M) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < M; n += gridDim.x * blockDim.x) {
    if (n < L) {
      const long long m2 = ((long long)n * n) % (2LL * L);
      double s, c;
      sincospi(-(double)m2 / (double)L, &s, &c);
      chirp[n] = df_from_double2(c, s);
    }
    // b_n for n < L, b_{M - n} = b_n for 0 < n < L, zero between
    int src = -1;
    if (n < L) src = n;
    else if (n > M - L) src = M - n;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (src >= 0) {
      const long long m2 = ((long long)src * src) % (2LL * L);
      double s, c;
      sincospi((double)m2 / (double)L, &s, &c);
      v = df_from_double2(c, s);
    }
    bhat[n] = v;
  }
}

// bhat <- DFT_M(bhat), one CTA
__global__ void __launch_bounds__(kGenThreads) k_gen_bhat(float4* bhat, int M, GenPlanM pm, const float4* twm) {
  extern __shared__ float4 sm[];
  float4* a = sm;
  float4* b = sm + M;
  for (int e = threadIdx.x; e < M; e += blockDim.x) a[e] = bhat[e];
  __syncthreads();
  float4* r = gen_passes(a, b, 1, M, pm.radix, pm.np, twm);
  for (int e = threadIdx.x; e < M; e += blockDim.x) bhat[e] = r[e];
}

// ---- transforms -----------------------------------------------------------

// Real rows x[row][n], n < W -> half spectra out(img, ky, kx), kx <= W/2; row = img * H + ky.
__global__ void __launch_bounds__(kGenThreads) k_gen_rows_fwd(const float* __restrict__ x, SpecView out,
                                                              long long nrows, int H, int W, int rpc, GenPlan P,
                                                              const float4* __restrict__ tab) {
  extern __shared__ float4 sm[];
  const int Leff = P.M ? P.M : P.L;
  float4* a = sm;
  float4* b = sm + (size_t)rpc * Leff;
  const long long row0 = (long long)blockIdx.x * rpc;
  const int nr = (int)min((long long)rpc, nrows - row0);
  for (int e = threadIdx.x; e < nr * Leff; e += blockDim.x) {
    const int f = e / Leff, n = e - f * Leff;
    a[e] = n < W ? make_float4(x[(row0 + f) * W + n], 0.f, 0.f, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  const float4* r = gen_transform(a, b, nr, P, tab, false);
  const int Wh = W / 2 + 1;
  for (int e = threadIdx.x; e < nr * Wh; e += blockDim.x) {
    const int f = e / Wh, k = e - f * Wh;
    const long long row = row0 + f;
    const long long img = row / H;
    const int ky = (int)(row - img * H);
    const float4 v = r[f * Leff + k];
    *out.at(img, ky, k, W / 2) = make_float2(v.x + v.z, v.y + v.w);
  }
}

// Columns of the half spectra from s to so (may be the same): cw columns of one image per
// CTA, read completely before any is written.  Images at or beyond count * C (when count
// is given) are skipped.
__global__ void __launch_bounds__(kGenThreads) k_gen_cols(SpecView s, SpecView so, int H, int W, int cw, GenPlan P,
                                                          const float4* __restrict__ tab, int inverse,
                                                          const int* __restrict__ count, int C) {
  extern __shared__ float4 sm[];
  const int img = blockIdx.y;
  if (count && img >= *count * C) return;
  const int Leff = P.M ? P.M : P.L;
  const int Wh = W / 2 + 1;
  const int kx0 = blockIdx.x * cw;
  const int nc = min(cw, Wh - kx0);
  float4* a = sm;
  float4* b = sm + (size_t)cw * Leff;
  for (int e = threadIdx.x; e < nc * Leff; e += blockDim.x) {
    const int n = e / nc, f = e - n * nc;  // consecutive threads: consecutive columns
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (n < H) {
      const float2 z = *s.at(img, n, kx0 + f, W / 2);
      v = make_float4(z.x, z.y, 0.f, 0.f);
    }
    a[f * Leff + n] = v;
  }
  __syncthreads();
  const float4* r = gen_transform(a, b, nc, P, tab, inverse != 0);
  for (int e = threadIdx.x; e < nc * H; e += blockDim.x) {
    const int n = e / nc, f = e - n * nc;
    const float4 v = r[f * Leff + n];
    *so.at(img, n, kx0 + f, W / 2) = make_float2(v.x + v.z, v.y + v.w);
  }
}

// Half rows in(img, ky, kx) -> real rows: the row completed by X[W - k] = conj X[k],
// inverse-transformed, real part times scale.  Output row img * H + ky of `out`, or, with
// requests, row (c H + ky) of req[img / C].out for channel c = img % C.
__global__ void __launch_bounds__(kGenThreads) k_gen_rows_inv(SpecView in, float* __restrict__ out,
                                                              long long nrows, int H, int W, int rpc, float scale,
                                                              const fdl_request* __restrict__ req,
                                                              const int* __restrict__ count, int C, GenPlan P,
                                                              const float4* __restrict__ tab, int nmax) {
  extern __shared__ float4 sm[];
  const int Leff = P.M ? P.M : P.L;
  float4* a = sm;
  float4* b = sm + (size_t)rpc * Leff;
  const long long row0 = (long long)blockIdx.x * rpc;
  long long lim = nrows;
  if (count) lim = min(lim, (long long)(*count) * C * H);
  if (row0 >= lim) return;
  const int nr = (int)min((long long)rpc, lim - row0);
  const int half = W / 2;
  for (int e = threadIdx.x; e < nr * Leff; e += blockDim.x) {
    const int f = e / Leff, n = e - f * Leff;
    const long long row = row0 + f;
    const long long img = row / H;
    const int ky = (int)(row - img * H);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (n < W) {
      const bool mirror = n > half;
      const float2 z = *in.at(img, ky, mirror ? W - n : n, half);
      v = make_float4(z.x, mirror ? -z.y : z.y, 0.f, 0.f);
    }
    a[e] = v;
  }
  __syncthreads();
  const float4* r = gen_transform(a, b, nr, P, tab, true);
  for (int e = threadIdx.x; e < nr * W; e += blockDim.x) {
    const int f = e / W, n = e - f * W;
    const long long row = row0 + f;
    const float4 v = r[f * Leff + n];
    const float val = (v.x + v.z) * scale;
    if (req) {
      const long long img = row / H;
      const int ky = (int)(row - img * H);
      const int bq = (int)(img / C), c = (int)(img - (long long)bq * C);
      // requests the render skipped are not written
      if (request_ok(req[bq], C, H, W, nmax, true)) req[bq].out[((long long)c * H + ky) * W + n] = val;
    } else {
      out[row * W + n] = val;
    }
  }
}

int largest_prime_factor(int L) {
  int p = 1;
  for (int f = 2; f * f <= L; ++f)
    while (L % f == 0) {
      p = f;
      L /= f;
    }
  return L > 1 ? (L > p ? L : p) : p;
}

// radices of L (every prime factor <= kGenMaxRadix): 4s from pairs of 2s, then the rest
int factor_radices(int L, int* radix) {
  int n = 0;
  while (L % 4 == 0 && n < kGenMaxPasses) {
    radix[n++] = 4;
    L /= 4;
  }
  for (int f = 2; f <= L && n < kGenMaxPasses; ++f)
    while (L % f == 0 && n < kGenMaxPasses) {
      radix[n++] = f;
      L /= f;
    }
  return L == 1 ? n : -1;
}

size_t rows_smem(int Leff, int rpc) { return (size_t)2 * rpc * Leff * sizeof(float4); }
int seqs_per_cta(int Leff) {
  const int k = (int)(kGenSmemBudget / ((size_t)2 * Leff * sizeof(float4)));
  return k < 1 ? 1 : (k > 8 ? 8 : k);
}

}  // namespace

bool gen_supported(int L) {
  if (L < 1 || L > kGenMaxLength) return false;
  if (largest_prime_factor(L) <= kGenMaxRadix) return true;
  int M = 1;
  while (M < 2 * L - 1) M <<= 1;
  return M <= kGenMaxBluestein;
}

bool gen_plan(int L, int base, GenPlan* p) {
  if (!gen_supported(L)) return false;
  p->L = L;
  p->tw = base;
  if (largest_prime_factor(L) <= kGenMaxRadix) {
    p->np = factor_radices(L, p->radix);
    p->M = p->mp = 0;
    p->chirp = p->twm = p->bhat = base;
    p->elems = L;
    return p->np >= 0;
  }
  int M = 1;
  while (M < 2 * L - 1) M <<= 1;
  p->np = 0;
  p->M = M;
  p->mp = factor_radices(M, p->mradix);
  p->chirp = base + L;
  p->twm = p->chirp + L;
  p->bhat = p->twm + M;
  p->elems = 2 * L + 2 * M;
  return p->mp >= 0;
}

cudaError_t launch_gen_tables(const GenPlan& p, float4* tab, cudaStream_t st) {
  k_gen_twiddles<<<(p.L + 255) / 256, 256, 0, st>>>(tab + p.tw, p.L);
  if (p.M == 0) return cudaGetLastError();
  k_gen_twiddles<<<(p.M + 255) / 256, 256, 0, st>>>(tab + p.twm, p.M);
  k_gen_chirp<<<(p.M + 255) / 256, 256, 0, st>>>(tab + p.chirp, tab + p.bhat, p.L, p.M);
  GenPlanM pm;
  pm.np = p.mp;
  for (int i = 0; i < kGenMaxPasses; ++i) pm.radix[i] = p.mradix[i];
  const size_t smem = (size_t)2 * p.M * sizeof(float4);
  cudaError_t e = set_smem((const void*)k_gen_bhat, smem);
  if (e != cudaSuccess) return e;
  k_gen_bhat<<<1, kGenThreads, smem, st>>>(tab + p.bhat, p.M, pm, tab + p.twm);
  return cudaGetLastError();
}

cudaError_t launch_gen_rows_fwd(const float* x, SpecView out, long long nrows, int H, int W, const GenPlan& p,
                                const float4* tab, cudaStream_t st) {
  const int Leff = p.M ? p.M : p.L;
  const int rpc = seqs_per_cta(Leff);
  const size_t smem = rows_smem(Leff, rpc);
  cudaError_t e = set_smem((const void*)k_gen_rows_fwd, smem);
  if (e != cudaSuccess) return e;
  const long long grid = (nrows + rpc - 1) / rpc;
  k_gen_rows_fwd<<<(unsigned)grid, kGenThreads, smem, st>>>(x, out, nrows, H, W, rpc, p, tab);
  return cudaGetLastError();
}

cudaError_t launch_gen_cols(SpecView s, SpecView so, int nimg, int H, int W, bool inverse, const GenPlan& p,
                            const float4* tab, const int* count, int C, cudaStream_t st) {
  const int Leff = p.M ? p.M : p.L;
  const int cw = seqs_per_cta(Leff);
  const size_t smem = rows_smem(Leff, cw);
  cudaError_t e = set_smem((const void*)k_gen_cols, smem);
  if (e != cudaSuccess) return e;
  const int Wh = W / 2 + 1;
  dim3 grid((Wh + cw - 1) / cw, nimg);
  k_gen_cols<<<grid, kGenThreads, smem, st>>>(s, so, H, W, cw, p, tab, inverse ? 1 : 0, count, C);
  return cudaGetLastError();
}

cudaError_t launch_gen_rows_inv(SpecView in, float* out, long long nrows, int H, int W, float scale,
                                const fdl_request* req, const int* count, int C, const GenPlan& p, const float4* tab,
                                cudaStream_t st, int nmax) {
  const int Leff = p.M ? p.M : p.L;
  const int rpc = seqs_per_cta(Leff);
  const size_t smem = rows_smem(Leff, rpc);
  cudaError_t e = set_smem((const void*)k_gen_rows_inv, smem);
  if (e != cudaSuccess) return e;
  const long long grid = (nrows + rpc - 1) / rpc;
  k_gen_rows_inv<<<(unsigned)grid, kGenThreads, smem, st>>>(in, out, nrows, H, W, rpc, scale, req, count, C, p,
                                                            tab, nmax);
  return cudaGetLastError();
}

}  // namespace fdl
