// Double-float per-frequency solve with the matrix in registers.
//
// Same problem as k_solve_hp<Rdf> (Sec. V-A, Eqs. AMatGeneral and
// LayerConstructionClosedForm with the Sec. V-C regularisers), organised for
// the FP32 pipe of sm_103a:
//  * one warp per frequency; the N(N+1)/2 entries of the lower triangle of
//    A*A + lambda Gamma*Gamma are numbered column by column and entry e lives
//    in lane e % 32, register slot e / 32, so every lane holds about the same
//    number of entries;
//  * A_jk = hi + lo (double-float); the Gram sum over views takes the hi*hi
//    products exactly (TwoProd), adds them with TwoSum and collects every
//    rounding error, plus the hi*lo cross terms, in the low word;
//  * Cholesky runs on the register slots with the pivot column broadcast
//    through shared memory.  The right-hand sides ride along as N*C extra slots
//    (row-major (k, c) numbering), so the factorisation also performs the forward
//    substitution L z = A*b.  Both numberings put the entries still to be
//    updated at pivot k in the trailing slots, so the update loop runs from the
//    last slot down and stops at the first slot that holds nothing beyond
//    column (row) k; the entries left behind are final and no longer read from
//    registers.  The back substitution L* x = z runs on the same right-hand-side
//    slots, where the rows still open at step k are a prefix.
//
// Moment form of the Gram matrix (MOM = true).  G_rl = sum_j exp(2 pi i (d_l - d_r)
// theta_j) depends on the pair only through d_l - d_r.  Writing d_k = d_0 + k Delta + e_k
// (Delta = (d_{N-1} - d_0)/(N-1), e_k the deviation from an exact grid, e_0 = 0),
// w_jm = A_jm conj(A_j0) = exp(2 pi i (m Delta + e_m) theta_j) and m = r - l,
//   conj(A_jr) A_jl = conj(w_jm) exp(2 pi i eta theta_j),  eta = e_l - e_r + e_m,
//   G_rl = sum_s (2 pi i eta)^s / s! conj(W_s(m)),  W_s(m) = sum_j theta_j^s w_jm,
// an exact identity with the exponential of the small phase expanded to s <= 3.  Per
// view that is N moment sets (lane m) instead of N(N+1)/2 products.  It applies when
// x = 2 pi max|e_l - e_r| max|theta| <= kMomXLim (then |2 pi eta theta| <= 2x and the
// first omitted term, (2x)^4/24, is below 1e-17; float32 linspace disparities give
// x ~ 5e-6 for |u| <= 4); k_mom_check decides that on the device and exactly one of the
// two kernels does the work.  Precision: W_0 in double-float as K + sum (w - 1), W_1 in
// double-float (its term is ~2x of G), W_2, W_3 in FP32 (terms below 2x^2 and 2x^3 of G).
#include <algorithm>

#include "hp_solve.cuh"

namespace fdl {

namespace {

constexpr int kDfWarps = 4;
// CTAs per SM the register allocation must allow, by NMAX: measured on the 512x512
// light fields, all frequencies in double-float (N = 16: 7.8 / 6.2 / 5.7 ms with 2 / 3 / 4;
// N = 30: 23.6 / 19.7 / 23.6 ms; N = 40: 41.5 / 66.3 / 69.5 ms, where spills dominate).
constexpr int df_min_blocks(int nmax) { return nmax <= 16 ? 4 : (nmax <= 32 ? 3 : 2); }

// Views on an integer lattice u_j = (a_j, b_j), |a_j|, |b_j| <= kLatMax: A_jr = P_r^a Q_r^b with
// P_r^k = exp(2 pi i k d_r w_x), Q_r^k = exp(2 pi i k d_r w_y), formed once per frequency.
__host__ __device__ constexpr int df_lat_f4(int nmax) { return nmax <= 40 ? 2 * kLatMax * 32 * ((nmax + 31) / 32) : 0; }

// float4 words of shared memory per warp: A_j / next pivot column and the current column
// (NMAX + 1 each), the packed factor, [NMAX][4] right-hand sides, 2 x 4 pivot-row values,
// NMAX double-float reciprocals, 3 x 32 view-only values of a chunk of views (moment form),
// the lattice powers [2 kLatMax][32 R] (N <= 40)
__host__ __device__ constexpr int df_warp_f4(int nmax) {
  return 2 * (nmax + 1) + nmax * (nmax + 1) / 2 + 4 * nmax + 8 + (nmax + 1) / 2 + 96 + df_lat_f4(nmax);
}

// entry (r, l), l <= r, numbered column-major: column l starts at l*N - l(l-1)/2
__device__ __forceinline__ int col_start(int l, int N) { return l * N - (l * (l - 1)) / 2; }

struct dfc {
  df re, im;
};

__device__ __forceinline__ float4 pack(const dfc& a) { return make_float4(a.re.hi, a.im.hi, a.re.lo, a.im.lo); }
__device__ __forceinline__ dfc unpack(float4 v) { return {{v.x, v.z}, {v.y, v.w}}; }

// acc += conj(a) * b for a, b double-float complex stored as (re.hi, im.hi, re.lo, im.lo);
// acc's low words collect the rounding errors (renormalised by the caller).
__device__ __forceinline__ void gram_acc(dfc& g, float4 a, float4 b) {
  // real part: a.hx b.hx + a.hy b.hy (+ cross terms)
  {
    const float p1 = __fmul_rn(a.x, b.x), e1 = fmaf(a.x, b.x, -p1);
    const float p2 = __fmul_rn(a.y, b.y), e2 = fmaf(a.y, b.y, -p2);
    const df s1 = two_sum(g.re.hi, p1);
    const df s2 = two_sum(s1.hi, p2);
    float lo = g.re.lo + (s1.lo + s2.lo) + (e1 + e2);
    lo = fmaf(a.x, b.z, lo);
    lo = fmaf(a.y, b.w, lo);
    lo = fmaf(a.z, b.x, lo);
    lo = fmaf(a.w, b.y, lo);
    g.re = {s2.hi, lo};
  }
  // imaginary part: a.hx b.hy - a.hy b.hx (+ cross terms)
  {
    const float q1 = __fmul_rn(a.x, b.y), f1 = fmaf(a.x, b.y, -q1);
    const float q2 = __fmul_rn(a.y, b.x), f2 = fmaf(a.y, b.x, -q2);
    const df s1 = two_sum(g.im.hi, q1);
    const df s2 = two_sum(s1.hi, -q2);
    float lo = g.im.lo + (s1.lo + s2.lo) + (f1 - f2);
    lo = fmaf(a.x, b.w, lo);
    lo = fmaf(-a.y, b.z, lo);
    lo = fmaf(a.z, b.y, lo);
    lo = fmaf(-a.w, b.x, lo);
    g.im = {s2.hi, lo};
  }
}

// the low word may exceed a high word that cancelled, so TwoSum, not Fast2Sum
__device__ __forceinline__ void renorm(dfc& g) {
  g.re = two_sum(g.re.hi, g.re.lo);
  g.im = two_sum(g.im.hi, g.im.lo);
}

// hi*hi product of two double-float reals, exact (p + e), plus the hi*lo cross terms in x
struct prod3 {
  float p, e, x;
};
__device__ __forceinline__ prod3 mul3(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = fmaf(a.hi, b.hi, -p);
  const float x = fmaf(a.hi, b.lo, a.lo * b.hi);
  return {p, e, x};
}
// g + s1 * u + s2 * v (s1, s2 = +-1 folded into the products), compensated and renormalised
__device__ __forceinline__ df acc2(df g, prod3 u, prod3 v) {
  const df t1 = two_sum(g.hi, u.p);
  const df t2 = two_sum(t1.hi, v.p);
  const float lo = g.lo + (t1.lo + t2.lo) + ((u.e + v.e) + (u.x + v.x));
  return fast_two_sum(t2.hi, lo);
}
__device__ __forceinline__ prod3 neg3(prod3 a) { return {-a.p, -a.e, -a.x}; }

// g -= a * conj(b): re -= a.re b.re + a.im b.im, im -= a.im b.re - a.re b.im
__device__ __forceinline__ void sub_mul_conj(dfc& g, const dfc& a, const dfc& b) {
  g.re = acc2(g.re, neg3(mul3(a.re, b.re)), neg3(mul3(a.im, b.im)));
  g.im = acc2(g.im, neg3(mul3(a.im, b.re)), mul3(a.re, b.im));
}

// g -= a * b: re -= a.re b.re - a.im b.im, im -= a.re b.im + a.im b.re
__device__ __forceinline__ void sub_mul(dfc& g, const dfc& a, const dfc& b) {
  g.re = acc2(g.re, neg3(mul3(a.re, b.re)), mul3(a.im, b.im));
  g.im = acc2(g.im, neg3(mul3(a.re, b.im)), neg3(mul3(a.im, b.re)));
}

// g -= conj(a) * b: re -= a.re b.re + a.im b.im, im -= a.re b.im - a.im b.re
__device__ __forceinline__ void sub_conj_mul(dfc& g, const dfc& a, const dfc& b) {
  g.re = acc2(g.re, neg3(mul3(a.re, b.re)), neg3(mul3(a.im, b.im)));
  g.im = acc2(g.im, neg3(mul3(a.re, b.im)), mul3(a.im, b.re));
}

__device__ __forceinline__ dfc scale(const dfc& a, df s) { return {df_mul(a.re, s), df_mul(a.im, s)}; }

// y += conj(a) * b for a double-float (re.hi, im.hi, re.lo, im.lo), b single precision:
// the products of the high words exact (TwoProd), their sums by TwoSum, every rounding
// error and the low-word products collected in the low word, which is left
// unnormalised (renormalised once after the view loop)
__device__ __forceinline__ void rhs_acc(dfc& y, float4 a, float2 b) {
  {  // re += a.re b.x + a.im b.y
    const float p1 = __fmul_rn(a.x, b.x), e1 = fmaf(a.x, b.x, -p1);
    const float p2 = __fmul_rn(a.y, b.y), e2 = fmaf(a.y, b.y, -p2);
    const df s1 = two_sum(y.re.hi, p1);
    const df s2 = two_sum(s1.hi, p2);
    float lo = y.re.lo + (s1.lo + s2.lo) + (e1 + e2);
    lo = fmaf(a.z, b.x, lo);
    lo = fmaf(a.w, b.y, lo);
    y.re = {s2.hi, lo};
  }
  {  // im += a.re b.y - a.im b.x
    const float p1 = __fmul_rn(a.x, b.y), e1 = fmaf(a.x, b.y, -p1);
    const float p2 = __fmul_rn(a.y, b.x), e2 = fmaf(a.y, b.x, -p2);
    const df s1 = two_sum(y.im.hi, p1);
    const df s2 = two_sum(s1.hi, -p2);
    float lo = y.im.lo + (s1.lo + s2.lo) + (e1 - e2);
    lo = fmaf(a.z, b.y, lo);
    lo = fmaf(-a.w, b.x, lo);
    y.im = {s2.hi, lo};
  }
}

__device__ __forceinline__ float4 shfl4(float4 v, int src) {
  return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                     __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}

constexpr float kMomXLim = 5e-5f;

// One warp: Delta, e_k for k < N (double-float, exact), and the flag counters[8] = 1
// when 2 pi (max e - min e) (max_j |u_j| / sqrt(2)) <= kMomXLim (|w| <= 1/sqrt(2)).
__global__ void k_mom_check(const float* __restrict__ d, int N, const float* __restrict__ u, int K, float2* mom,
                            int* counters) {
  const int lane = threadIdx.x;
  const float d0 = d[0];
  const float delta = N > 1 ? (d[N - 1] - d0) / (float)(N - 1) : 0.f;
  float emin = INFINITY, emax = -INFINITY;
  bool finite = true;
  for (int k = lane; k < N; k += 32) {
    const float dk = d[k];
    finite = finite && isfinite(dk);
    const df e = df_sub(two_sum(dk, -d0), two_prod((float)k, delta));
    mom[k] = make_float2(e.hi, e.lo);
    emin = fminf(emin, e.hi);
    emax = fmaxf(emax, e.hi);
  }
  float umax = 0.f;
  bool lattice = true;
  for (int j = lane; j < K; j += 32) {
    const float ux = u[2 * j], uy = u[2 * j + 1];
    finite = finite && isfinite(ux) && isfinite(uy);
    umax = fmaxf(umax, sqrtf(ux * ux + uy * uy));
    lattice = lattice && ux == rintf(ux) && uy == rintf(uy) && fabsf(ux) <= (float)kLatMax && fabsf(uy) <= (float)kLatMax;
  }
  lattice = __all_sync(0xffffffffu, lattice);
  // the views fill the rectangle [a0, a1] x [b0, b1] of the lattice, each point once
  constexpr int kSide = 2 * kLatMax + 1;
  __shared__ int cell[kSide * kSide];
  for (int i = lane; i < kSide * kSide; i += 32) cell[i] = 0;
  int a0 = kLatMax, a1 = -kLatMax, b0 = kLatMax, b1 = -kLatMax;
  __syncwarp();
  if (lattice) {
    for (int j = lane; j < K; j += 32) {
      const int ux = (int)u[2 * j], uy = (int)u[2 * j + 1];
      atomicAdd(&cell[(uy + kLatMax) * kSide + ux + kLatMax], 1);
      a0 = min(a0, ux);
      a1 = max(a1, ux);
      b0 = min(b0, uy);
      b1 = max(b1, uy);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 = min(a0, __shfl_xor_sync(0xffffffffu, a0, o));
    a1 = max(a1, __shfl_xor_sync(0xffffffffu, a1, o));
    b0 = min(b0, __shfl_xor_sync(0xffffffffu, b0, o));
    b1 = max(b1, __shfl_xor_sync(0xffffffffu, b1, o));
  }
  __syncwarp();
  bool grid = lattice && K > 0 && K == (a1 - a0 + 1) * (b1 - b0 + 1);
  if (grid)
    for (int i = lane; i < K; i += 32) {
      const int na = a1 - a0 + 1;
      grid = grid && cell[(b0 + i / na + kLatMax) * kSide + a0 + i % na + kLatMax] == 1;
    }
  grid = __all_sync(0xffffffffu, grid);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    emin = fminf(emin, __shfl_xor_sync(0xffffffffu, emin, o));
    emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
  }
  const bool all_finite = __all_sync(0xffffffffu, finite);
  if (lane == 0) {
    // relative slack for the low words of e, which max/min of the high words ignore
    const float x = 6.2831853f * (emax - emin) * 1.0001f * umax * 0.70710678f + 1e-30f;
    counters[8] = (all_finite && N <= 64 && x <= kMomXLim) ? 1 : 0;
    counters[10] = (all_finite && lattice) ? 1 : 0;
    counters[11] = (all_finite && grid) ? 1 : 0;
    counters[12] = (a0 + kLatMax) | ((a1 + kLatMax) << 8) | ((b0 + kLatMax) << 16) | ((b1 + kLatMax) << 24);
  }
}

// a + b with the "sloppy" double-word addition (error ~2^-46 (|a| + |b|)): used where
// the absolute error is what matters (terms of magnitude <= 2)
__device__ __forceinline__ df sadd_df(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

// acc += v for double-float accumulators whose terms stay small (TwoSum on the high
// words, low words added)
__device__ __forceinline__ void acc_df(df& acc, df v) {
  const df s = two_sum(acc.hi, v.hi);
  acc = two_sum(s.hi, __fadd_rn(__fadd_rn(acc.lo, s.lo), v.lo));
}

template <int NMAX, int S, bool MOM>
__global__ void __launch_bounds__(kDfWarps * 32, df_min_blocks(NMAX)) k_solve_df(SolveParams p, int all_bins) {
  constexpr int R = (NMAX + 31) / 32;  // rows per lane in the solves
  if (p.mom != nullptr) {
    // exactly one of the moment and the general kernel runs (k_mom_check decided)
    const bool mom_on = *((volatile int*)(p.counters + 8)) == 1;
    if (mom_on != MOM) return;
  }
  extern __shared__ float4 sm4[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int N = p.N, C = p.C, K = p.K, M = p.W >> 1;
  const int E = N * (N + 1) / 2;
  constexpr int SY = (4 * NMAX + 31) / 32;  // right-hand-side slots per lane (C <= 4)
  float4* Arow = sm4 + warp * df_warp_f4(NMAX);  // A_j of one view; the next pivot column in the factorisation
  float4* col = Arow + NMAX + 1;                 // the current column of L
  float4* Ls = col + NMAX + 1;                   // packed lower triangle, column-major
  float4* zbuf = Ls + NMAX * (NMAX + 1) / 2;     // [N][C] right-hand sides, then z = L^-1 A*b
  float4* ynext = zbuf + 4 * NMAX;               // [C] right-hand sides of the next pivot row
  float4* zc = ynext + 4;                        // [C] z of the current pivot row
  float2* invd = reinterpret_cast<float2*>(zc + 4);  // 1 / L_kk as df
  float4* thb = reinterpret_cast<float4*>(invd) + (NMAX + 1) / 2;  // [32][3] view-only values
  float4* pq = thb + 96;  // lattice powers: [k - 1][32 R] P_r^k, then [kLatMax + k - 1][32 R] Q_r^k
  // the views lie on an integer lattice (k_mom_check): A from the lattice powers
  const bool lat = MOM && df_lat_f4(NMAX) > 0 && *((volatile int*)(p.counters + 10)) == 1;
  // ... and fill a rectangle [ga0, ga1] x [gb0, gb1] of it: the moments of w factor over the axes
  const bool grid = lat && *((volatile int*)(p.counters + 11)) == 1;
  const int gbox = *((volatile int*)(p.counters + 12));
  const int ga0 = (gbox & 255) - kLatMax, ga1 = ((gbox >> 8) & 255) - kLatMax;
  const int gb0 = ((gbox >> 16) & 255) - kLatMax, gb1 = ((gbox >> 24) & 255) - kLatMax;

  // coordinates (r, l) of this lane's slots, packed as r * 256 + l.  An unused slot
  // (entry number >= E) gets (N, N): it reads Arow[N] / col[N], which lie inside this
  // warp's shared region and are zeroed below, so the Gram loop needs no branch; it
  // never matches a pivot column k < N and is never stored.
  int rl[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int e = lane + 32 * s;
    rl[s] = (N << 8) | N;
    if (e < E) {
      int l = 0;
      while (col_start(l + 1, N) <= e) ++l;
      rl[s] = ((l + (e - col_start(l, N))) << 8) | l;
    }
  }
  // right-hand-side slots: entry i = k * C + c (layer k, channel c) in lane i % 32,
  // slot i / 32, packed as k * 256 + c; unused ones get layer N (col[N] stays zero)
  int yk[SY];
#pragma unroll
  for (int t = 0; t < SY; ++t) {
    const int i = lane + 32 * t;
    yk[t] = (i < N * C) ? (((i / C) << 8) | (i % C)) : (N << 8);
  }
#define SR(s) (rl[s] >> 8)
#define SL(s) (rl[s] & 255)
  for (int i = lane; i < 2 * (NMAX + 1); i += 32) Arow[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncwarp();
  float2 em[R];  // e_m of this lane's moments (moment form)
#pragma unroll
  for (int h = 0; h < R; ++h) em[h] = (MOM && lane + 32 * h < N) ? p.mom[lane + 32 * h] : make_float2(0.f, 0.f);
  const float4* tab = p.exp_table;
  const int total = all_bins ? p.H * (M + 1) : *((volatile int*)(p.counters + 4));
  int nhp = 0, nbad = 0, nnf = 0;
  for (int li = blockIdx.x * kDfWarps + warp; li < total; li += gridDim.x * kDfWarps) {
    const int q = all_bins ? li : p.flagged[li];
    int ky, kx;
    bin_coords(q, p.H, M, ky, kx);
    const Freq fq = bin_freq(ky, kx, p.H, p.W);

    dfc G[S];
#pragma unroll
    for (int s = 0; s < S; ++s) G[s] = {{0.f, 0.f}, {0.f, 0.f}};
    dfc y[R][4];
#pragma unroll
    for (int h = 0; h < R; ++h)
#pragma unroll
      for (int c = 0; c < 4; ++c) y[h][c] = {{0.f, 0.f}, {0.f, 0.f}};

    float dr[R];
#pragma unroll
    for (int h = 0; h < R; ++h) dr[h] = (lane + 32 * h < N) ? __ldg(p.d + lane + 32 * h) : 0.f;
    dfc Ssum[R];  // S_r = sum_j (A_jr - 1)
#pragma unroll
    for (int h = 0; h < R; ++h) Ssum[h] = {{0.f, 0.f}, {0.f, 0.f}};
    // moment form: M0 = sum (w - 1), M1 = sum theta (w - 1) (double-float), M2, M3 = sum
    // theta^2,3 (w - 1) (FP32), and the plain sums of theta^p (identical in every lane)
    dfc M0[R], M1[R];
    float2 M2[R], M3[R];
#pragma unroll
    for (int h = 0; h < R; ++h) {
      M0[h] = {{0.f, 0.f}, {0.f, 0.f}};
      M1[h] = {{0.f, 0.f}, {0.f, 0.f}};
      M2[h] = make_float2(0.f, 0.f);
      M3[h] = make_float2(0.f, 0.f);
    }
    df T1 = {0.f, 0.f};
    float T2 = 0.f, T3 = 0.f;

    // this frequency's K*C inputs staged in the (still unused) factor region, all lanes
    // loading at once, when they fit: one memory latency per frequency instead of per view
    const bool stage = K * C <= NMAX * (NMAX + 1);
    float2* bst = reinterpret_cast<float2*>(Ls);
    if (stage) {
      for (int e = lane; e < K * C; e += 32) bst[e] = *p.b.at(e, ky, kx, M);
      __syncwarp();
    }

    if (lat) {
      // P_r^k and Q_r^k from the exact-piece phases k d_r w_x, k d_r w_y; each lane reads
      // only its own entries back, so no barrier is needed
#pragma unroll
      for (int h = 0; h < R; ++h) {
        if (lane + 32 * h < N) {
#pragma unroll 1
          for (int k = 1; k <= kLatMax; ++k) {
            const cx<Rdf> pk = cexp2pi(phase_r(theta_r((float)k, 0.f, fq, Rdf{}), dr[h]), tab);
            const cx<Rdf> qk = cexp2pi(phase_r(theta_r(0.f, (float)k, fq, Rdf{}), dr[h]), tab);
            pq[(k - 1) * 32 * R + 32 * h + lane] = pack(dfc{pk.re.v, pk.im.v});
            pq[(kLatMax + k - 1) * 32 * R + 32 * h + lane] = pack(dfc{qk.re.v, qk.im.v});
          }
        }
      }
    }
    for (int j0 = 0; j0 < K; j0 += 32) {
      if constexpr (MOM) {
        // what depends on the view only (theta = u_j . w in exact pieces and as a double-float,
        // theta^2, theta^3 and their sums), once per view: one view per lane for a chunk of 32
        const int jl = j0 + lane;
        if (jl < K) {
          const float2 ul = __ldg(reinterpret_cast<const float2*>(p.u) + jl);
          const ThetaX t = theta_r(ul.x, ul.y, fq, Rdf{});
          const df theta = df_add(two_sum(t.p1, t.p2), df_from(__fadd_rn(__fadd_rn(t.e1, t.e2), t.g)));
          const float th2 = theta.hi * theta.hi, th3 = th2 * theta.hi;
          thb[3 * lane] = make_float4(t.p1, t.e1, t.p2, t.e2);
          thb[3 * lane + 1] = make_float4(t.g, theta.hi, theta.lo, th2);
          thb[3 * lane + 2] = make_float4(th3, ul.x, ul.y, 0.f);  // with the lattice coordinates
          acc_df(T1, theta);
          T2 += th2;
          T3 += th3;
        }
        __syncwarp();
      }
      const int jn = min(32, K - j0);
      for (int jj = 0; jj < jn; ++jj) {
        const int j = j0 + jj;
        ThetaX th;
        df theta = {0.f, 0.f};
        float th2 = 0.f, th3 = 0.f;
        int ax = 0, by = 0;  // lattice coordinates of the view
        if constexpr (MOM) {
          const float4 q0 = thb[3 * jj], q1 = thb[3 * jj + 1];
          th = {q0.x, q0.y, q0.z, q0.w, q1.x};
          theta = {q1.y, q1.z};
          th2 = q1.w;
          const float4 q2 = thb[3 * jj + 2];
          th3 = q2.x;
          ax = (int)q2.y;
          by = (int)q2.z;
        } else {
          const float2 uj = __ldg(reinterpret_cast<const float2*>(p.u) + j);
          th = theta_r(uj.x, uj.y, fq, Rdf{});
        }
        float2 bj[4];
#pragma unroll
        for (int c = 0; c < 4; ++c)
          bj[c] = c < C ? (stage ? bst[j * C + c] : *p.b.at((long long)j * C + c, ky, kx, M)) : make_float2(0.f, 0.f);
        dfc aR[R];  // A_jr of this lane's rows (moment form)
#pragma unroll
        for (int h = 0; h < R; ++h) {
          const int r = lane + 32 * h;
          aR[h] = {{0.f, 0.f}, {0.f, 0.f}};
          if (r < N) {
            cx<Rdf> a;
            if (lat) {
              // A_jr = P_r^a Q_r^b (conjugates for negative powers), one double-float product;
              // terms of magnitude <= 1, summed with the sloppy double-word addition
              dfc pa = {{1.f, 0.f}, {0.f, 0.f}}, qb = {{1.f, 0.f}, {0.f, 0.f}};
              if (ax != 0) pa = unpack(pq[(abs(ax) - 1) * 32 * R + 32 * h + lane]);
              if (by != 0) qb = unpack(pq[(kLatMax + abs(by) - 1) * 32 * R + 32 * h + lane]);
              if (ax < 0) pa.im = df_neg(pa.im);
              if (by < 0) qb.im = df_neg(qb.im);
              const df p1 = df_mul(pa.re, qb.re), p2 = df_neg(df_mul(pa.im, qb.im));
              const df q1 = df_mul(pa.re, qb.im), q2 = df_mul(pa.im, qb.re);
              const df r1 = two_sum(p1.hi, p2.hi), r2 = two_sum(q1.hi, q2.hi);
              a = {{fast_two_sum(r1.hi, __fadd_rn(r1.lo, __fadd_rn(p1.lo, p2.lo)))},
                   {fast_two_sum(r2.hi, __fadd_rn(r2.lo, __fadd_rn(q1.lo, q2.lo)))}};
            } else {
              a = cexp2pi(phase_r(th, dr[h]), tab);
            }
            aR[h] = {a.re.v, a.im.v};
            // A - 1: the subtraction of the high word is exact (TwoSum)
            const df t = two_sum(a.re.v.hi, -1.f);
            const df am = two_sum(t.hi, __fadd_rn(t.lo, a.re.v.lo));
            const float4 av = make_float4(am.hi, a.im.v.hi, am.lo, a.im.v.lo);
            if constexpr (!MOM) {
              Arow[r] = av;
              const df s1 = two_sum(Ssum[h].re.hi, am.hi);
              Ssum[h].re = two_sum(s1.hi, __fadd_rn(__fadd_rn(Ssum[h].re.lo, s1.lo), am.lo));
              const df s2 = two_sum(Ssum[h].im.hi, a.im.v.hi);
              Ssum[h].im = two_sum(s2.hi, __fadd_rn(__fadd_rn(Ssum[h].im.lo, s2.lo), a.im.v.lo));
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
              if (c < C) rhs_acc(y[h][c], av, bj[c]);
          }
        }
        if constexpr (MOM) {
          if (grid) continue;  // the moments come from the axis sums after the view loop
          // w_jm = A_jm conj(A_j0) for this lane's m (A_j0 from lane 0) and the moments of w - 1
          const dfc a0 = unpack(shfl4(pack(aR[0]), 0));
#pragma unroll
          for (int h = 0; h < R; ++h) {
            if (lane + 32 * h < N) {
              const dfc& am = aR[h];
              const df wr = sadd_df(df_mul(am.re, a0.re), df_mul(am.im, a0.im));
              const df wi = sadd_df(df_mul(am.im, a0.re), df_neg(df_mul(am.re, a0.im)));
              // w - 1 (exact subtraction of the high word)
              const df t = two_sum(wr.hi, -1.f);
              const df wm1r = two_sum(t.hi, __fadd_rn(t.lo, wr.lo));
              acc_df(M0[h].re, wm1r);
              acc_df(M0[h].im, wi);
              acc_df(M1[h].re, df_mul(theta, wm1r));
              acc_df(M1[h].im, df_mul(theta, wi));
              M2[h].x = fmaf(th2, wm1r.hi, M2[h].x);
              M2[h].y = fmaf(th2, wi.hi, M2[h].y);
              M3[h].x = fmaf(th3, wm1r.hi, M3[h].x);
              M3[h].y = fmaf(th3, wi.hi, M3[h].y);
            }
          }
          continue;
        }
        __syncwarp();
        // every slot, without a branch, so that the independent slot updates interleave;
        // diagonal slots are overwritten below (the sum of |A_jk|^2 is exactly K)
#pragma unroll
        for (int s = 0; s < S; ++s) {
          gram_acc(G[s], Arow[SR(s)], Arow[SL(s)]);
          // keep |lo| within an ulp of |hi| so that the low word's own rounding stays at 2^-48
          G[s].re = fast_two_sum(G[s].re.hi, G[s].re.lo);
          G[s].im = fast_two_sum(G[s].im.hi, G[s].im.lo);
        }
        __syncwarp();
      }
      if constexpr (MOM) __syncwarp();  // the next chunk rewrites thb
    }
    if (MOM && grid) {
      // Views filling the rectangle: w_jm = p_m^a q_m^b with p_m^a = P_m^a conj(P_0^a),
      // q_m^b = Q_m^b conj(Q_0^b), and theta_j = a w_x + b w_y, so with p~ = p - 1, q~ = q - 1
      //   sum_j a^s b^t (w_jm - 1) = X_st = SP_s sb_t + sa_s SQ_t + SP_s SQ_t,
      //   SP_s = sum_a a^s p~^a, sa_s = sum_a a^s (SQ_t, sb_t over b),
      // and M0 = X_00, M1 = w_x X_10 + w_y X_01, M2, M3 by the binomial expansion of theta^2,3
      // (double-float to first order, FP32 beyond, as in the view loop).
      __syncwarp();  // every lane reads row 0's powers
      const df wxd = {fq.wx, fq.wx_lo}, wyd = {fq.wy, fq.wy_lo};
#pragma unroll
      for (int h = 0; h < R; ++h) {
        if (lane + 32 * h >= N) continue;
        dfc SP[2][2];     // [axis][s] for s = 0, 1 (double-float)
        float2 SPf[2][4]; // [axis][s] high words, s = 0..3 (FP32)
        float sg[2][4];   // sa_s, sb_s
#pragma unroll
        for (int ax = 0; ax < 2; ++ax) {
          SP[ax][0] = SP[ax][1] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            SPf[ax][t] = make_float2(0.f, 0.f);
            sg[ax][t] = 0.f;
          }
          const int lo = ax == 0 ? ga0 : gb0, hi = ax == 0 ? ga1 : gb1;
#pragma unroll 1
          for (int a = lo; a <= hi; ++a) {
            const float fa = (float)a;
            sg[ax][0] += 1.f;
            sg[ax][1] += fa;
            sg[ax][2] += fa * fa;
            sg[ax][3] += fa * fa * fa;
            if (a == 0) continue;
            const int row = (ax * kLatMax + abs(a) - 1) * 32 * R;
            dfc pm = unpack(pq[row + 32 * h + lane]), p0 = unpack(pq[row]);
            if (a < 0) {
              pm.im = df_neg(pm.im);
              p0.im = df_neg(p0.im);
            }
            const df wr = sadd_df(df_mul(pm.re, p0.re), df_mul(pm.im, p0.im));
            const df wi = sadd_df(df_mul(pm.im, p0.re), df_neg(df_mul(pm.re, p0.im)));
            const df t = two_sum(wr.hi, -1.f);
            const df wm1r = two_sum(t.hi, __fadd_rn(t.lo, wr.lo));
            acc_df(SP[ax][0].re, wm1r);
            acc_df(SP[ax][0].im, wi);
            acc_df(SP[ax][1].re, df_mul_f(wm1r, fa));
            acc_df(SP[ax][1].im, df_mul_f(wi, fa));
            float pw = 1.f;
#pragma unroll
            for (int s2 = 0; s2 < 4; ++s2) {
              SPf[ax][s2].x = fmaf(pw, wm1r.hi, SPf[ax][s2].x);
              SPf[ax][s2].y = fmaf(pw, wi.hi, SPf[ax][s2].y);
              pw *= fa;
            }
          }
        }
        // double-float X_00, X_10, X_01
        auto xd = [&](int s1, int t1) -> dfc {
          const dfc& P = SP[0][s1];
          const dfc& Q = SP[1][t1];
          const df pr = df_mul(P.re, Q.re), pi = df_mul(P.im, Q.im);
          const df qr = df_mul(P.re, Q.im), qi = df_mul(P.im, Q.re);
          dfc x;
          x.re = df_add(df_add(df_mul_f(P.re, sg[1][t1]), df_mul_f(Q.re, sg[0][s1])), df_sub(pr, pi));
          x.im = df_add(df_add(df_mul_f(P.im, sg[1][t1]), df_mul_f(Q.im, sg[0][s1])), df_add(qr, qi));
          return x;
        };
        auto xf = [&](int s1, int t1) -> float2 {
          const float2 P = SPf[0][s1], Q = SPf[1][t1];
          return make_float2(fmaf(P.x, sg[1][t1], fmaf(Q.x, sg[0][s1], fmaf(P.x, Q.x, -P.y * Q.y))),
                             fmaf(P.y, sg[1][t1], fmaf(Q.y, sg[0][s1], fmaf(P.x, Q.y, P.y * Q.x))));
        };
        M0[h] = xd(0, 0);
        const dfc x10 = xd(1, 0), x01 = xd(0, 1);
        M1[h].re = df_add(df_mul(wxd, x10.re), df_mul(wyd, x01.re));
        M1[h].im = df_add(df_mul(wxd, x10.im), df_mul(wyd, x01.im));
        const float wx = fq.wx, wy = fq.wy;
        const float2 x20 = xf(2, 0), x11 = xf(1, 1), x02 = xf(0, 2);
        M2[h] = make_float2(wx * wx * x20.x + 2.f * wx * wy * x11.x + wy * wy * x02.x,
                            wx * wx * x20.y + 2.f * wx * wy * x11.y + wy * wy * x02.y);
        const float2 x30 = xf(3, 0), x21 = xf(2, 1), x12 = xf(1, 2), x03 = xf(0, 3);
        const float c30 = wx * wx * wx, c21 = 3.f * wx * wx * wy, c12 = 3.f * wx * wy * wy, c03 = wy * wy * wy;
        M3[h] = make_float2(c30 * x30.x + c21 * x21.x + c12 * x12.x + c03 * x03.x,
                            c30 * x30.y + c21 * x21.y + c12 * x12.y + c03 * x03.y);
      }
    }
    if constexpr (MOM) {
      // the sums of theta^p over the views, from the lanes' partial sums
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const df t = {__shfl_xor_sync(0xffffffffu, T1.hi, o), __shfl_xor_sync(0xffffffffu, T1.lo, o)};
        T1 = df_add(T1, t);
        T2 += __shfl_xor_sync(0xffffffffu, T2, o);
        T3 += __shfl_xor_sync(0xffffffffu, T3, o);
      }
    }
    // Assemble A*A and A*b from the sums over (A - 1).  With a = 1 + a~,
    //   conj(a_r) a_l = 1 + conj(a~_r) + a~_l + conj(a~_r) a~_l,
    // so G_rl = K + conj(S_r) + S_l + sum_j conj(a~_jr) a~_jl and
    // y_r = sum_j b_j + sum_j conj(a~_jr) b_j.  At the low, worst-conditioned
    // frequencies every A_jk is close to 1 and the sums over a~ stay small, so
    // their rounding does not grow with the number of views the way the
    // running sums of nearly equal terms of A*A and A*b would.
    const df Kdf = {(float)K, 0.f};
    if constexpr (MOM) {
      // moments to shared memory (the Ls region is free until after the factorisation):
      // per m, [M0 | M1 (with sum theta added) | M2, M3 (with sums of theta^2,3 added)]
      float4* Mm = Ls;
#pragma unroll
      for (int h = 0; h < R; ++h) {
        const int m = lane + 32 * h;
        if (m < N) {
          Mm[3 * m] = pack(M0[h]);
          const dfc m1 = {df_add(M1[h].re, T1), M1[h].im};
          Mm[3 * m + 1] = pack(m1);
          Mm[3 * m + 2] = make_float4(M2[h].x + T2, M2[h].y, M3[h].x + T3, M3[h].y);
        }
      }
      __syncwarp();
      const df twopi = {6.28318548202514648f, -1.74845553146951720e-07f};
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int r = SR(s), l = SL(s);
        if (r == l) {
          G[s] = {Kdf, {0.f, 0.f}};  // sum_j |A_jk|^2 = K exactly (also unused slots)
        } else {
          const int m = r - l;
          const float2 er = p.mom[r], el = p.mom[l], emm = p.mom[m];
          const df eta = df_add(df_sub({el.x, el.y}, {er.x, er.y}), {emm.x, emm.y});
          const df te = df_mul(eta, twopi);  // 2 pi eta
          const dfc m0 = unpack(Mm[3 * m]), m1 = unpack(Mm[3 * m + 1]);
          const float4 m23 = Mm[3 * m + 2];
          // s = 0: K + conj(W0); s = 1: (2 pi i eta) conj(W1) = 2 pi eta (W1.im + i W1.re)
          dfc g = {df_add(Kdf, m0.re), df_neg(m0.im)};
          g.re = df_add(g.re, df_mul(te, m1.im));
          g.im = df_add(g.im, df_mul(te, m1.re));
          // s = 2: -(2 pi eta)^2 / 2 conj(W2); s = 3: -(2 pi eta)^3 / 6 (W3.im + i W3.re)
          const float t = te.hi, c2 = -0.5f * t * t, c3 = -t * t * t * (1.f / 6.f);
          const float gr = fmaf(c2, m23.x, c3 * m23.w);
          const float gi = fmaf(-c2, m23.y, c3 * m23.z);
          g.re = df_add_f(g.re, gr);
          g.im = df_add_f(g.im, gi);
          G[s] = g;
        }
      }
      __syncwarp();
    } else {
#pragma unroll
      for (int h = 0; h < R; ++h)
        if (lane + 32 * h < N) col[lane + 32 * h] = pack(Ssum[h]);
      __syncwarp();
#pragma unroll
      for (int s = 0; s < S; ++s) {
        renorm(G[s]);
        if (SR(s) == SL(s)) {
          G[s] = {Kdf, {0.f, 0.f}};  // sum_j |A_jk|^2 = K exactly
        } else {
          const dfc sr = unpack(col[SR(s)]), sl = unpack(col[SL(s)]);
          G[s].re = df_add(G[s].re, df_add(Kdf, df_add(sr.re, sl.re)));
          G[s].im = df_add(G[s].im, df_sub(sl.im, sr.im));
        }
      }
    }
    // the right-hand sides were accumulated with unnormalised low words
#pragma unroll
    for (int h = 0; h < R; ++h)
#pragma unroll
      for (int c = 0; c < 4; ++c) renorm(y[h][c]);
    // sum_j b_j per channel: lanes over views, then a butterfly of double-float adds
    {
      dfc bs[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) bs[c] = {{0.f, 0.f}, {0.f, 0.f}};
      for (int j = lane; j < K; j += 32) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (c < C) {
            const float2 bv = *p.b.at((long long)j * C + c, ky, kx, M);
            bs[c].re = df_add_f(bs[c].re, bv.x);
            bs[c].im = df_add_f(bs[c].im, bv.y);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c < C) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float4 v = shfl4(pack(bs[c]), lane ^ o);
            const dfc w = unpack(v);
            bs[c].re = df_add(bs[c].re, w.re);
            bs[c].im = df_add(bs[c].im, w.im);
          }
#pragma unroll
          for (int h = 0; h < R; ++h) {
            y[h][c].re = df_add(y[h][c].re, bs[c].re);
            y[h][c].im = df_add(y[h][c].im, bs[c].im);
          }
        }
      }
    }

    // lambda Gamma*Gamma
    {
      const df wxd = {fq.wx, fq.wx_lo}, wyd = {fq.wy, fq.wy_lo};
      const df w2 = df_add(df_mul(wxd, wxd), df_mul(wyd, wyd));
      const df w4 = df_mul(w2, w2);
      const df lam = df_from_double(p.lam_d);
      const df lame = df_from_double(p.lam_eps_d);
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int r = SR(s), l = SL(s);
        if (r >= N) continue;
        if (p.reg == 0) {
          if (r == l) {
            const float dv = __ldg(p.d + r);
            const df d2 = two_prod(dv, dv);
            G[s].re = df_add(G[s].re, df_add(df_mul(lam, df_mul(w4, df_mul(d2, d2))), lame));
          }
        } else if (p.reg == 1) {
          if (r - l <= 2) G[s].re = df_add(G[s].re, df_mul_f(lam, layer2_gtg(r, l, N)));
        } else if (r == l) {
          G[s].re = df_add(G[s].re, lam);
        }
      }
    }

    // trace(G) >= largest eigenvalue, for the condition estimate
    float tr = 0.f;
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (SR(s) < N && SR(s) == SL(s)) tr += G[s].re.hi;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);

    // Cholesky with the right-hand sides as extra rows: the (N + c, k) entries of the
    // factor of [[G, y], [y*, .]] are conj(z_kc), z = L^-1 y.  The right-hand sides
    // move to their slots through shared memory.
#pragma unroll
    for (int h = 0; h < R; ++h) {
      const int r = lane + 32 * h;
      if (r < N)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (c < C) zbuf[r * C + c] = pack(y[h][c]);
    }
    __syncwarp();
    dfc Y[SY];
#pragma unroll
    for (int t = 0; t < SY; ++t) {
      const int i = lane + 32 * t;
      Y[t] = i < N * C ? unpack(zbuf[i]) : dfc{{0.f, 0.f}, {0.f, 0.f}};
    }
    // column 0 and the right-hand sides of row 0 start the pivot sequence
    if (lane < C) ynext[lane] = zbuf[lane];
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (SL(s) == 0 && SR(s) < N) Arow[SR(s)] = pack(G[s]);
    __syncwarp();
    bool ok = true;
    for (int k = 0; k < N; ++k) {
      // every lane takes the pivot, scales its rows of column k and publishes them
      const float4 pv = Arow[k];
      const df piv = {pv.x, pv.z};
      ok = ok && (piv.hi > 0.f);
      const df lkk = df_sqrt(piv.hi > 0.f ? piv : df_from(1.f));
      const df inv = df_div(df_from(1.f), lkk);
      const int ck = col_start(k, N);
#pragma unroll
      for (int h = 0; h < R; ++h) {
        const int r = lane + 32 * h;
        if (r >= k && r < N) {
          const float4 v = r == k ? make_float4(lkk.hi, 0.f, lkk.lo, 0.f) : pack(scale(unpack(Arow[r]), inv));
          col[r] = v;
          Ls[ck + (r - k)] = v;
        }
      }
      if (lane < C) {
        const float4 z = pack(scale(unpack(ynext[lane]), inv));
        zc[lane] = z;
        zbuf[k * C + lane] = z;
      }
      if (lane == 0) invd[k] = make_float2(inv.hi, inv.lo);
      __syncwarp();
      if (k + 1 < N) {
        // trailing update G_rl -= L_rk conj(L_lk) for l > k: the slots from the first one
        // holding an entry of column k + 1 on; the entries of column k + 1 go to Arow
        // for the next pivot
        const int s0 = col_start(k + 1, N) >> 5;
#pragma unroll
        for (int s = S - 1; s >= 0; --s) {
          if (s < s0) break;
          if (32 * s >= E) continue;  // unused slots (N < NMAX)
          sub_mul_conj(G[s], unpack(col[SR(s)]), unpack(col[SL(s)]));
          if (SL(s) == k + 1) Arow[SR(s)] = pack(G[s]);
        }
        // forward substitution y_rc -= L_rk z_kc for r > k
        const int t0 = ((k + 1) * C) >> 5;
#pragma unroll
        for (int t = SY - 1; t >= 0; --t) {
          if (t < t0) break;
          if (32 * t >= N * C) continue;  // unused slots (C < 4)
          const int r = yk[t] >> 8, c = yk[t] & 255;
          sub_mul(Y[t], unpack(col[r]), unpack(zc[c]));
          if (r == k + 1) ynext[c] = pack(Y[t]);
        }
      }
      __syncwarp();
    }

    // Condition estimate kappa ~ trace(G) |G^-1 v| after three steps of inverse iteration
    // with the factor (FP32 is enough for an error estimate).
    float kappa = 0.f;
    if (p.err != nullptr) {
      float2 v[R];
#pragma unroll
      for (int h = 0; h < R; ++h) {
        const int r = lane + 32 * h;
        v[h] = make_float2(0.f, 0.f);
        if (r < N) {
          float sn, cs;
          sincospif(2.f * 0.6180339887f * (float)(r * r), &sn, &cs);
          v[h] = make_float2(cs * rsqrtf((float)N), sn * rsqrtf((float)N));
        }
      }
      float vnorm = 0.f;
      for (int it = 0; it < 3; ++it) {
        for (int k = 0; k < N; ++k) {
          const float ikk = invd[k].x;
          const int owner = k & 31, hk = k >> 5;
          float2 mine = make_float2(0.f, 0.f);
#pragma unroll
          for (int h = 0; h < R; ++h)
            if (h == hk) mine = v[h];
          const float2 vk = make_float2(__shfl_sync(0xffffffffu, mine.x, owner) * ikk,
                                        __shfl_sync(0xffffffffu, mine.y, owner) * ikk);
#pragma unroll
          for (int h = 0; h < R; ++h) {
            const int r = lane + 32 * h;
            if (r > k && r < N) {
              const float4 l = Ls[col_start(k, N) + (r - k)];
              cfms_c(v[h], make_float2(l.x, l.y), cconj(vk));
            } else if (r == k) {
              v[h] = vk;
            }
          }
        }
        for (int k = N - 1; k >= 0; --k) {
          const float ikk = invd[k].x;
          const int owner = k & 31, hk = k >> 5;
          float2 mine = make_float2(0.f, 0.f);
#pragma unroll
          for (int h = 0; h < R; ++h)
            if (h == hk) mine = v[h];
          const float2 xk = make_float2(__shfl_sync(0xffffffffu, mine.x, owner) * ikk,
                                        __shfl_sync(0xffffffffu, mine.y, owner) * ikk);
#pragma unroll
          for (int h = 0; h < R; ++h) {
            const int r = lane + 32 * h;
            if (r < k) {
              const float4 l = Ls[col_start(r, N) + (k - r)];
              cfms_c(v[h], make_float2(l.x, -l.y), cconj(xk));
            } else if (r == k) {
              v[h] = xk;
            }
          }
        }
        float n2 = 0.f;
#pragma unroll
        for (int h = 0; h < R; ++h)
          if (lane + 32 * h < N) n2 += v[h].x * v[h].x + v[h].y * v[h].y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
        vnorm = sqrtf(n2);
        const float inv = vnorm > 0.f ? 1.f / vnorm : 0.f;
#pragma unroll
        for (int h = 0; h < R; ++h) v[h] = cscale(v[h], inv);
      }
      kappa = tr * vnorm;
    }

    // back substitution L* x = z on the right-hand-side slots: at step k the entries of
    // the rows r < k (a prefix of the row-major numbering) take x_k; the entries of row
    // k - 1 are then final and go to ynext for the next step; x_k goes to zbuf
#pragma unroll
    for (int t = 0; t < SY; ++t) {
      const int i = lane + 32 * t;
      Y[t] = i < N * C ? unpack(zbuf[i]) : dfc{{0.f, 0.f}, {0.f, 0.f}};
    }
    if (lane < C) ynext[lane] = zbuf[(N - 1) * C + lane];
    __syncwarp();
    for (int k = N - 1; k >= 0; --k) {
      if (lane < C) {
        const float2 iv = invd[k];
        const float4 x = pack(scale(unpack(ynext[lane]), df{iv.x, iv.y}));
        zc[lane] = x;
        zbuf[k * C + lane] = x;
      }
      __syncwarp();
      if (k > 0) {
        const int t1 = (k * C - 1) >> 5;  // the last slot holding an entry of a row r < k
#pragma unroll
        for (int t = 0; t < SY; ++t) {
          if (t > t1) break;
          const int r = yk[t] >> 8, c = yk[t] & 255;
          // x_r -= conj(L_kr) x_k, L_kr = entry (k, r) of column r; the entries of rows
          // r >= k are final (in zbuf) and their registers are no longer read
          const int li = r < k ? col_start(r, N) + (k - r) : 0;
          sub_conj_mul(Y[t], unpack(Ls[li]), unpack(zc[c]));
          if (r == k - 1) ynext[c] = pack(Y[t]);
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int h = 0; h < R; ++h) {
      const int r = lane + 32 * h;
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c < C && r < N) y[h][c] = unpack(zbuf[r * C + c]);
    }
    const long long plane = (long long)p.H * (M + 1);
    const long long off = (long long)ky * (M + 1) + kx;
    float n2 = 0.f;
    bool fin = true;
#pragma unroll
    for (int h = 0; h < R; ++h) {
      const int r = lane + 32 * h;
      if (r < N) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (c < C) {
            const float2 xv =
                ok ? make_float2(y[h][c].re.hi + y[h][c].re.lo, y[h][c].im.hi + y[h][c].im.lo) : make_float2(0.f, 0.f);
            p.x[((long long)r * C + c) * plane + off] = xv;
            n2 += xv.x * xv.x + xv.y * xv.y;
            fin = fin && isfinite(xv.x) && isfinite(xv.y);
          }
      }
    }
    // a non-finite input reaches the solution (A and Gamma are finite): counted by the
    // first pass over all frequencies (a listed frequency was counted by the FP32 pass)
    fin = __all_sync(0xffffffffu, fin);
    if (!fin && all_bins && lane == 0) ++nnf;
    if (p.err != nullptr) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
      if (lane == 0) {
        p.err[q] = ok ? kappa * sqrtf(n2) : INFINITY;
        p.xn2[q] = n2;
      }
    }
    if (lane == 0) {
      ++nhp;
      if (!ok) ++nbad;
    }
    __syncwarp();
  }
#undef SR
#undef SL
  if (lane == 0) {
    if (nhp) atomicAdd(p.counters + 1, nhp);
    // a listed frequency was first solved (and counted) by the FP32 pass
    if (nhp && !all_bins) atomicSub(p.counters + 0, nhp);
    if (nbad) atomicAdd(p.counters + 2, nbad);
    if (nnf) atomicAdd(p.counters + 3, nnf);
  }
}

template <int NMAX, int S, bool MOM>
cudaError_t launch_df_v(const SolveParams& p, bool all_bins, cudaStream_t st) {
  const size_t per_warp = (size_t)df_warp_f4(NMAX) * sizeof(float4);
  const size_t smem = per_warp * kDfWarps;
  cudaError_t e = set_smem((const void*)k_solve_df<NMAX, S, MOM>, smem);
  if (e != cudaSuccess) return e;
  // one frequency per warp for the largest possible list: short CTAs let
  // higher-priority streams interleave (CTAs past the list length exit at once).  The general
  // kernel launched beside the moment-form one (one of them returns at once, decided on the
  // device) strides with at most 8 CTAs per SM, so that returning costs a few microseconds.
  const int bins = p.H * (p.W / 2 + 1);
  int grid = (bins + kDfWarps - 1) / kDfWarps;
  if (!MOM && p.mom != nullptr) grid = std::min(grid, 8 * num_sms());
  k_solve_df<NMAX, S, MOM><<<grid, kDfWarps * 32, smem, st>>>(p, all_bins ? 1 : 0);
  return cudaGetLastError();
}

// With p.mom set (launch_mom_check has run): the moment-form kernel and the general
// kernel, of which exactly one does the work (the other exits at once).
template <int NMAX, int S>
cudaError_t launch_df_n(const SolveParams& p, bool all_bins, cudaStream_t st) {
  if (p.mom == nullptr) return launch_df_v<NMAX, S, false>(p, all_bins, st);
  cudaError_t e = launch_df_v<NMAX, S, true>(p, all_bins, st);
  if (e == cudaSuccess) e = launch_df_v<NMAX, S, false>(p, all_bins, st);
  return e;
}

}  // namespace

bool solve_df_supported(int N) { return N <= 48; }

cudaError_t launch_mom_check(const SolveParams& p, cudaStream_t st) {
  k_mom_check<<<1, 32, 0, st>>>(p.d, p.N, p.u, p.K, p.mom, p.counters);
  return cudaGetLastError();
}

cudaError_t launch_solve_df(const SolveParams& p, bool all_bins, cudaStream_t st) {
  // register slots per lane: ceil(NMAX (NMAX + 1) / 64)
  if (p.N <= 8) return launch_df_n<8, 2>(p, all_bins, st);
  if (p.N <= 12) return launch_df_n<12, 3>(p, all_bins, st);
  if (p.N <= 16) return launch_df_n<16, 5>(p, all_bins, st);
  if (p.N <= 20) return launch_df_n<20, 7>(p, all_bins, st);
  if (p.N <= 24) return launch_df_n<24, 10>(p, all_bins, st);
  if (p.N <= 28) return launch_df_n<28, 13>(p, all_bins, st);
  if (p.N <= 30) return launch_df_n<30, 15>(p, all_bins, st);
  if (p.N <= 32) return launch_df_n<32, 17>(p, all_bins, st);
  if (p.N <= 36) return launch_df_n<36, 21>(p, all_bins, st);
  if (p.N <= 40) return launch_df_n<40, 26>(p, all_bins, st);
  if (p.N <= 44) return launch_df_n<44, 31>(p, all_bins, st);
  return launch_df_n<48, 37>(p, all_bins, st);
}

}  // namespace fdl
