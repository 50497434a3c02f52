// Per-frequency Tikhonov solve of the layer construction (Sec. V-A):
//   (A*A + lambda Gamma*Gamma) x = A* b,  A_jk = exp(+2 pi i d_k (u_j . w))
// (Eqs. AMatGeneral, LayerConstructionClosedForm), Gamma*Gamma from Sec. V-C:
// the view regulariser diag(|w|^4 d^4 + eps) (Eq. 2ndOrderView, plus the
// epsilon of Sec. V-C1), the layer regulariser tridiag(1,-2,1)^T tridiag(1,-2,1)
// (Eq. 2ndOrderLayer) or the identity.  The C colour channels share A and
// Gamma, so one Cholesky factor serves C right-hand sides.
//
// Two kernels:
//  * k_solve_f32: FP32, one warp per frequency, lane i owns row i of the
//    Hermitian matrix in registers.  Where the moment form applies (the
//    disparities lie on a grid d_k = d_0 + k Delta + e_k with small e_k; the flag
//    k_mom_check sets) the Gram matrix is assembled from N sums per view instead of
//    N^2: G_rl = sum_j conj(A_jr) A_jl = W_0(m) + 2 pi i eta W_1(m) for l >= r,
//    m = l - r, eta = e_l - e_r - e_m, W_s(m) = sum_j theta_j^s conj(A_j0) A_jm,
//    theta_j = u_j . w (the exponential of the small phase 2 pi eta theta_j to
//    first order; the flag bounds it by 1e-4, whose square is below FP32
//    rounding), and G_rl = conj(G_lr) below the diagonal.  On an integer view
//    lattice A_jr = P_r^a Q_r^b from per-frequency powers P_r^k = exp(2 pi i k d_r w_x),
//    Q_r^k = exp(2 pi i k d_r w_y).  With estimate set it also records, per
//    frequency, an error scale kappa |x| (kappa from three steps of power
//    iteration for the largest eigenvalue and three steps of inverse
//    iteration with the factor for the smallest; +inf where the factorisation
//    broke down, the input was not finite or kappa exceeds kappa_max) and |x|^2,
//    from which the caller picks the frequencies to re-solve more precisely.
//  * k_solve_hp<T>: the same solve in double-float (T = Rdf) or native FP64
//    (T = R64) for the listed frequencies (or for all of them).
#include <algorithm>

#include "hp_solve.cuh"

namespace fdl {

// SM count of the current device (queried once)
static int g_num_sms = 0;
int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  return g_num_sms;
}

namespace {

constexpr int kTileBins = 8;    // bins per CTA tile = warps per CTA
constexpr int kViewChunk = 128;  // views staged per pass (one pass for K <= 128)

// ------------------------------------------------------------------ FP32
// Per-lane lattice powers P_r^k, Q_r^k (k = 1..kLatMax) of this lane's row r at frequency fq;
// only this lane reads them back.
__device__ __forceinline__ void f32_lattice_powers(float2* ptab, int lane, int N, const Freq& fq, float dl) {
  if (lane < N) {
#pragma unroll 1
    for (int k = 1; k <= kLatMax; ++k) {
      float2 t;
      sincospif(2.f * phase_cycles((float)k, 0.f, fq, dl), &t.y, &t.x);
      ptab[(k - 1) * 32 + lane] = t;
      sincospif(2.f * phase_cycles(0.f, (float)k, fq, dl), &t.y, &t.x);
      ptab[(kLatMax + k - 1) * 32 + lane] = t;
    }
  }
}

// Stages views [j0, j0 + nv) of the tile's kTileBins frequencies: b[j][c][bin] (consecutive
// threads read consecutive bins; a thread's bin is fixed, threadIdx.x % kTileBins) and u_j.
// CTA-wide; the caller puts barriers around it.
__device__ __forceinline__ void f32_stage(const SolveParams& p, int tile, int j0, int nv, int Qs, int M,
                                          float2* bstage, float2* ustage) {
  const int C = p.C;
  const int bi = threadIdx.x & (kTileBins - 1);
  int qy, qx;
  bin_coords(min(tile * kTileBins + bi, Qs - 1), p.H, M, qy, qx);
  for (int img = threadIdx.x / kTileBins; img < nv * C; img += blockDim.x / kTileBins)
    bstage[img * kTileBins + bi] = *p.b.at((long long)j0 * C + img, qy, qx, M);
  for (int j = threadIdx.x; j < nv; j += blockDim.x) ustage[j] = __ldg(reinterpret_cast<const float2*>(p.u) + j0 + j);
}

// Moment form, per warp (frequency fq, lane m / row r): W_0(m) = sum_j w_jm, W_1(m) = sum_j
// theta_j w_jm with w_jm = conj(A_j0) A_jm, and y_c(r) = sum_j conj(A_jr) b_jc over every view;
// A from the lattice powers in ptab when lat, else from the phase.  CTA-wide (stages views).
__device__ __forceinline__ void f32_mom_sums(const SolveParams& p, int tile, int Qs, int M, const Freq& fq, float dl,
                                             bool lat, float2* bstage, float2* ustage, const float2* ptab,
                                             float2& W0, float2& W1, float2 y[4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int C = p.C, N = p.N, K = p.K;
  const float wx = fq.wx, wy = fq.wy;
  for (int j0 = 0; j0 < K; j0 += kViewChunk) {
    const int nv = min(kViewChunk, K - j0);
    __syncthreads();
    f32_stage(p, tile, j0, nv, Qs, M, bstage, ustage);
    __syncthreads();
    // no loop-carried dependence but the sums, so the unrolled views overlap their latencies
#pragma unroll 4
    for (int jj = 0; jj < nv; ++jj) {
      const float2 uj = ustage[jj];
      float2 a = make_float2(0.f, 0.f);
      if (lane < N) {
        if (lat) {
          // A_jr = P_r^a Q_r^b, conjugates for negative powers
          const int ax = (int)uj.x, by = (int)uj.y;
          float2 pa = make_float2(1.f, 0.f), qb = make_float2(1.f, 0.f);
          if (ax != 0) pa = ptab[(abs(ax) - 1) * 32 + lane];
          if (by != 0) qb = ptab[(kLatMax + abs(by) - 1) * 32 + lane];
          if (ax < 0) pa.y = -pa.y;
          if (by < 0) qb.y = -qb.y;
          a = cmul(pa, qb);
        } else {
          const float f = phase_cycles(uj.x, uj.y, fq, dl);
          sincospif(2.f * f, &a.y, &a.x);
        }
      }
      const float2 a0 = make_float2(__shfl_sync(0xffffffffu, a.x, 0), __shfl_sync(0xffffffffu, a.y, 0));
      const float2 w = cmulc(a0, a);
      const float th = fmaf(uj.x, wx, uj.y * wy);
      W0.x += w.x;
      W0.y += w.y;
      W1.x = fmaf(th, w.x, W1.x);
      W1.y = fmaf(th, w.y, W1.y);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c < C) {
          cfmac(y[c], a, bstage[(jj * C + c) * kTileBins + warp]);
        }
      }
    }
  }
}

// The moment-form sums of the FP32 solve for tiles [t0, t1) (kTileBins frequencies each), when
// the moment form applies: wsum[i * 32 + lane] = (W_0, W_1) of lane m, ysum[(i * 4 + c) * 32 +
// lane] = y_c of row r, i = (tile - t0) kTileBins + warp.  Few registers and 49 KB of shared
// memory per CTA, so that four CTAs per SM hide the latencies of the view loop that the
// register- and shared-memory-heavy solve kernel (two CTAs per SM) cannot; k_solve_f32 reads them.
__global__ void __launch_bounds__(kTileBins * 32) k_f32_sums(SolveParams p, int t0, int t1, float4* __restrict__ wsum,
                                                             float2* __restrict__ ysum) {
  extern __shared__ float4 smem4[];
  __shared__ float2 ustage[kViewChunk];
  float2* bstage = reinterpret_cast<float2*>(smem4);             // [kViewChunk * 4][kTileBins]
  float2* ptabs = bstage + kViewChunk * 4 * kTileBins;           // [kTileBins][2 kLatMax][32]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int M = p.W >> 1, N = p.N;
  const bool mom = p.mom != nullptr && *((volatile int*)(p.counters + 8)) == 1;
  if (!mom) return;
  const bool lat = *((volatile int*)(p.counters + 10)) == 1;
  float2* ptab = ptabs + warp * 2 * kLatMax * 32;
  const int Qs = p.H * (M + 1);
  const float dl = lane < N ? __ldg(p.d + lane) : 0.f;
  for (int tile = t0 + blockIdx.x; tile < t1; tile += gridDim.x) {
    const int q = min(tile * kTileBins + warp, Qs - 1);
    int ky, kx;
    bin_coords(q, p.H, M, ky, kx);
    const Freq fq = bin_freq(ky, kx, p.H, p.W);
    float2 y[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) y[c] = make_float2(0.f, 0.f);
    float2 W0 = make_float2(0.f, 0.f), W1 = make_float2(0.f, 0.f);
    if (lat) {
      __syncwarp();  // the previous tile's reads of this lane's powers are done
      f32_lattice_powers(ptab, lane, N, fq, dl);
    }
    f32_mom_sums(p, tile, Qs, M, fq, dl, lat, bstage, ustage, ptab, W0, W1, y);
    const long long i = (long long)(tile - t0) * kTileBins + warp;
    wsum[i * 32 + lane] = make_float4(W0.x, W0.y, W1.x, W1.y);
#pragma unroll
    for (int c = 0; c < 4; ++c) ysum[(i * 4 + c) * 32 + lane] = y[c];
  }
}

template <int NMAX>
// two CTAs per SM: the register allocation must stay within 128 per thread
__global__ void __launch_bounds__(kTileBins * 32, 2) k_solve_f32(SolveParams p, int estimate, int t0, int t1,
                                                                  const float4* __restrict__ wsum,
                                                                  const float2* __restrict__ ysum) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int M = p.W >> 1;
  const int C = p.C, N = p.N, K = p.K;
  // shared memory carve-up
  float2* bstage = reinterpret_cast<float2*>(smem4);                  // [kViewChunk*C][kTileBins]
  float2* arow = bstage + kViewChunk * 4 * kTileBins;                   // [kTileBins][NMAX]
  float2* Ls = arow + kTileBins * NMAX;                                 // [kTileBins][NMAX][NMAX+1]
  float2* myA = arow + warp * NMAX;
  float2* myL = Ls + warp * NMAX * (NMAX + 1);
  __shared__ int cnt_local[4];
  __shared__ float2 ustage[kViewChunk];  // u_j of the staged views
  if (threadIdx.x < 4) cnt_local[threadIdx.x] = 0;

  const int Qs = p.H * (M + 1);
  const int ntiles = (Qs + kTileBins - 1) / kTileBins;  // the last tile may be partial
  const float dl = lane < N ? __ldg(p.d + lane) : 0.f;
  // moment form and view lattice (k_mom_check's flags; warp-uniform)
  const bool mom = p.mom != nullptr && NMAX <= 32 && *((volatile int*)(p.counters + 8)) == 1;
  // (the powers take 2 kLatMax x 32 words of the warp's factor storage)
  const bool lat = mom && NMAX * (NMAX + 1) >= 2 * kLatMax * 32 && *((volatile int*)(p.counters + 10)) == 1;
  const float el = (mom && lane < N) ? p.mom[lane].x : 0.f;  // e_lane
  float2* ptab = myL;  // lattice powers [2 kLatMax][32] while the Gram matrix is built

  for (int tile = t0 + blockIdx.x; tile < min(t1, ntiles); tile += gridDim.x) {
    // warps past the last bin of a partial tile solve the last bin again (every warp
    // takes part in the CTA's barriers) and write nothing
    const int q = min(tile * kTileBins + warp, Qs - 1);
    const bool qown = tile * kTileBins + warp < Qs;
    int ky, kx;
    bin_coords(q, p.H, M, ky, kx);
    const Freq fq = bin_freq(ky, kx, p.H, p.W);
    const float wy = fq.wy, wx = fq.wx;

    float2 G[NMAX];
#pragma unroll
    for (int l = 0; l < NMAX; ++l) G[l] = make_float2(0.f, 0.f);
    float2 y[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) y[c] = make_float2(0.f, 0.f);
    float2 W0 = make_float2(0.f, 0.f), W1 = make_float2(0.f, 0.f);  // moment sums, m = lane
    if (mom && wsum != nullptr) {
      // the sums of k_f32_sums
      const long long i = (long long)(tile - t0) * kTileBins + warp;
      const float4 w = wsum[i * 32 + lane];
      W0 = make_float2(w.x, w.y);
      W1 = make_float2(w.z, w.w);
#pragma unroll
      for (int c = 0; c < 4; ++c) y[c] = ysum[(i * 4 + c) * 32 + lane];
    } else if (mom) {
      if (lat) {
        // P^k, Q^k of this lane's row in the words of its factor (the barrier orders the
        // writes after the previous frequency's reads of the factor)
        __syncwarp();
        f32_lattice_powers(ptab, lane, N, fq, dl);
      }
      f32_mom_sums(p, tile, Qs, M, fq, dl, lat, bstage, ustage, ptab, W0, W1, y);
    } else {
      for (int j0 = 0; j0 < K; j0 += kViewChunk) {
        const int nv = min(kViewChunk, K - j0);
        __syncthreads();
        f32_stage(p, tile, j0, nv, Qs, M, bstage, ustage);
        __syncthreads();
        for (int jj = 0; jj < nv; ++jj) {
          const float2 uj = ustage[jj];
          float2 a = make_float2(0.f, 0.f);
          if (lane < N) {
            const float f = phase_cycles(uj.x, uj.y, fq, dl);
            sincospif(2.f * f, &a.y, &a.x);
          }
          if (lane < NMAX) myA[lane] = a;
          __syncwarp();
          const float4* A4 = reinterpret_cast<const float4*>(myA);
#pragma unroll
          for (int l2 = 0; l2 < NMAX / 2; ++l2) {
            const float4 v = A4[l2];
            cfmac(G[2 * l2], a, make_float2(v.x, v.y));
            cfmac(G[2 * l2 + 1], a, make_float2(v.z, v.w));
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (c < C) {
              cfmac(y[c], a, bstage[(jj * C + c) * kTileBins + warp]);
            }
          }
          __syncwarp();
        }
      }
    }

    if (mom) {
      // G_rl from the moment sums of lane m = |l - r|
#pragma unroll
      for (int l = 0; l < NMAX; ++l) {
        const bool up = l >= lane;
        const int m = up ? l - lane : lane - l;
        const float2 w0 = make_float2(__shfl_sync(0xffffffffu, W0.x, m), __shfl_sync(0xffffffffu, W0.y, m));
        const float2 w1 = make_float2(__shfl_sync(0xffffffffu, W1.x, m), __shfl_sync(0xffffffffu, W1.y, m));
        const float em = __shfl_sync(0xffffffffu, el, m), ell = __shfl_sync(0xffffffffu, el, l);
        const float t = 6.2831853f * ((up ? ell - el : el - ell) - em);
        float2 g = make_float2(fmaf(-t, w1.y, w0.x), fmaf(t, w1.x, w0.y));
        if (!up) g.y = -g.y;
        G[l] = (l < N && lane < N) ? g : make_float2(0.f, 0.f);
      }
    }
    // an input that is not finite reaches every right-hand side (|A_jk| = 1): lane 0's
    // row is checked
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c < C) finite = finite && isfinite(y[c].x) && isfinite(y[c].y);
    // regulariser lambda Gamma*Gamma
    {
      const float w2 = wx * wx + wy * wy;
      const float d2 = dl * dl;
#pragma unroll
      for (int l = 0; l < NMAX; ++l) {
        if (p.reg == 0) {
          if (l == lane) G[l].x += p.lam * (w2 * w2) * (d2 * d2) + p.lam_eps;
        } else if (p.reg == 1) {
          if (lane < N && l < N) G[l].x += p.lam * layer2_gtg(lane, l, N);
        } else {
          if (l == lane) G[l].x += p.lam;
        }
      }
    }
    // largest eigenvalue: power iteration from a vector with a component along
    // every eigenvector in practice (all-ones plus golden-angle phases)
    float lmax = 0.f;
    if (estimate) {
      float2 v = make_float2(0.f, 0.f);
      if (lane < N) {
        float sn, cs;
        sincospif(2.f * 0.6180339887f * (float)(lane * lane), &sn, &cs);
        v = make_float2(1.f + cs, sn);
      }
      for (int it = 0; it < 3; ++it) {
        float2 w = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < NMAX; ++l) {
          const float2 vl = make_float2(__shfl_sync(0xffffffffu, v.x, l), __shfl_sync(0xffffffffu, v.y, l));
          if (l < N) cfma(w, G[l], vl);
        }
        float n2 = lane < N ? w.x * w.x + w.y * w.y : 0.f;
        float v2 = lane < N ? v.x * v.x + v.y * v.y : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          n2 += __shfl_xor_sync(0xffffffffu, n2, o);
          v2 += __shfl_xor_sync(0xffffffffu, v2, o);
        }
        lmax = v2 > 0.f ? sqrtf(n2 / v2) : 0.f;  // |G v| / |v|
        const float inv = n2 > 0.f ? rsqrtf(n2) : 0.f;
        v = lane < N ? cscale(w, inv) : make_float2(0.f, 0.f);
      }
    }

    // Cholesky G = L L*, row i in lane i; lane k keeps 1 / L_kk
    bool ok = true;
    float dinv = 1.f;
#pragma unroll
    for (int k = 0; k < NMAX; ++k) {
      if (k < N) {
        const float piv = __shfl_sync(0xffffffffu, G[k].x, k);
        ok = ok && (piv > 1e-30f) && isfinite(piv);
        const float lkk = sqrtf(fmaxf(piv, 1e-30f));
        const float inv = 1.f / lkk;
        if (lane > k) G[k] = cscale(G[k], inv);
        else if (lane == k) {
          G[k] = make_float2(lkk, 0.f);
          dinv = inv;
        }
        if (lane < NMAX) myA[lane] = G[k];  // column k: L_lk in lane l
        __syncwarp();
#pragma unroll
        for (int l = k + 1; l < NMAX; ++l) {
          if (l < N && l <= lane) cfms_c(G[l], G[k], myA[l]);
        }
        __syncwarp();
      }
    }
    // L to shared memory (row i, pitch NMAX+1)
#pragma unroll
    for (int l = 0; l < NMAX; ++l)
      if (lane < NMAX) myL[lane * (NMAX + 1) + l] = (l <= lane) ? G[l] : make_float2(0.f, 0.f);
    __syncwarp();

    // solves: C right-hand sides plus the inverse-iteration vector v
    float2 v = make_float2(0.f, 0.f);
    if (lane < N) {
      float s, c;
      sincospif(2.f * 0.6180339887f * (float)(lane * lane), &s, &c);
      v = make_float2(c * rsqrtf((float)N), s * rsqrtf((float)N));
    }
    // a factorisation that broke down is not solved (the frequency is re-solved or zeroed);
    // without the estimate only the right-hand sides are
    float vnorm = 0.f;
    const int iters = ok ? (estimate ? 3 : 1) : 0;
    for (int it = 0; it < iters; ++it) {
      // forward: L z = rhs
      for (int k = 0; k < N; ++k) {
        const float ikk = __shfl_sync(0xffffffffu, dinv, k);
        const float2 lik = myL[(lane < NMAX ? lane : 0) * (NMAX + 1) + k];
        const float2 vk = cscale(make_float2(__shfl_sync(0xffffffffu, v.x, k), __shfl_sync(0xffffffffu, v.y, k)), ikk);
        if (lane > k) cfms_c(v, lik, cconj(vk));
        else if (lane == k) v = vk;
        if (it == 0) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (c < C) {
              const float2 yk = cscale(make_float2(__shfl_sync(0xffffffffu, y[c].x, k),
                                                   __shfl_sync(0xffffffffu, y[c].y, k)), ikk);
              if (lane > k) cfms_c(y[c], lik, cconj(yk));
              else if (lane == k) y[c] = yk;
            }
          }
        }
      }
      // backward: L* x = z
      for (int k = N - 1; k >= 0; --k) {
        const float ikk = __shfl_sync(0xffffffffu, dinv, k);
        const float2 lki = myL[k * (NMAX + 1) + (lane < NMAX ? lane : 0)];  // L_ki
        const float2 vk = cscale(make_float2(__shfl_sync(0xffffffffu, v.x, k), __shfl_sync(0xffffffffu, v.y, k)), ikk);
        if (lane < k) cfms_c(v, cconj(lki), cconj(vk));  // v_i -= conj(L_ki) x_k
        else if (lane == k) v = vk;
        if (it == 0) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (c < C) {
              const float2 yk = cscale(make_float2(__shfl_sync(0xffffffffu, y[c].x, k),
                                                   __shfl_sync(0xffffffffu, y[c].y, k)), ikk);
              if (lane < k) cfms_c(y[c], cconj(lki), cconj(yk));
              else if (lane == k) y[c] = yk;
            }
          }
        }
      }
      float n2 = lane < N ? v.x * v.x + v.y * v.y : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
      vnorm = sqrtf(n2);
      const float inv = vnorm > 0.f ? 1.f / vnorm : 0.f;
      v = cscale(v, inv);
    }
    const long long plane = (long long)p.H * (M + 1);
    const long long off = (long long)ky * (M + 1) + kx;
    // without the estimate a factorisation that broke down leaves zeros
    const bool broke = !ok;
    if (lane < N && qown) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c < C) p.x[((long long)lane * C + c) * plane + off] = broke ? make_float2(0.f, 0.f) : y[c];
    }
    if (estimate) {
      float n2 = 0.f;
      if (lane < N) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (c < C) n2 += y[c].x * y[c].x + y[c].y * y[c].y;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
      const float kappa = lmax * vnorm;
      const bool trusted = ok && finite && isfinite(kappa) && kappa <= p.kappa_max && isfinite(n2);
      if (lane == 0 && qown) {
        p.err[q] = trusted ? kappa * sqrtf(n2) : INFINITY;
        // |x|^2 for the budget's |X|: 0 where the factorisation broke down (no solution)
        p.xn2[q] = (ok && isfinite(n2)) ? n2 : 0.f;
      }
    }
    if (lane == 0 && qown) {
      if (estimate || !broke) atomicAdd(&cnt_local[0], 1);
      if (!estimate && broke) atomicAdd(&cnt_local[2], 1);
      if (!finite) atomicAdd(&cnt_local[3], 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (cnt_local[0]) atomicAdd(p.counters + 0, cnt_local[0]);
    if (cnt_local[2]) atomicAdd(p.counters + 2, cnt_local[2]);
    if (cnt_local[3]) atomicAdd(p.counters + 3, cnt_local[3]);
  }
}

// --------------------------------------------------------- high precision
__device__ __forceinline__ bool r_is_native(R64) { return true; }
__device__ __forceinline__ bool r_is_native(Rdf) { return false; }

template <class T>
__global__ void __launch_bounds__(128) k_solve_hp(SolveParams sp, int all_bins, int warps, int list) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int M = sp.W >> 1;
  HpProblem p;
  p.b = sp.b;
  p.u = sp.u;
  p.d = sp.d;
  p.exp_table = sp.exp_table;
  p.K = sp.K;
  p.C = sp.C;
  p.N = sp.N;
  p.H = sp.H;
  p.W = sp.W;
  p.reg = sp.reg;
  p.lam = sp.lam_d;
  p.lam_eps = sp.lam_eps_d;
  p.P = sp.P;
  p.views = sp.views;
  const int N = p.N, C = p.C;
  cx<T>* G = reinterpret_cast<cx<T>*>(smem4) + warp * hp_warp_elems<T>(N, C);
  cx<T>* Arow = G + N * (N + 1);
  cx<T>* Y = Arow + N;
  const int* lst = list == 0 ? sp.flagged : sp.flagged64;
  const int total = all_bins ? p.H * (M + 1) : *((volatile int*)(sp.counters + (list == 0 ? 4 : 5)));
  int nhp = 0, nbad = 0, nfixed = 0, nnf = 0;
  for (int li = blockIdx.x * warps + warp; li < total; li += gridDim.x * warps) {
    const int q = all_bins ? li : lst[li];
    int ky, kx;
    bin_coords(q, p.H, M, ky, kx);
    const bool ok = hp_solve_bin<T>(p, ky, kx, G, Arow, Y);
    const long long plane = (long long)p.H * (M + 1);
    const long long off = (long long)ky * (M + 1) + kx;
    bool fin = true;
    for (int e = lane; e < N * C; e += 32) {
      const int r = e / C, c = e - r * C;
      const cx<T> v = Y[e];
      const float2 xv = ok ? make_float2(r_to_float(v.re), r_to_float(v.im)) : make_float2(0.f, 0.f);
      fin = fin && isfinite(xv.x) && isfinite(xv.y);
      sp.x[((long long)r * C + c) * plane + off] = xv;
    }
    fin = __all_sync(0xffffffffu, fin);
    if (lane == 0) {
      ++nhp;
      if (!ok) ++nbad;
      // the double-float pass marked its breakdowns with err = +inf and counted them
      if (list == 1 && sp.err != nullptr && isinf(sp.err[q])) ++nfixed;
      if (!fin && all_bins) ++nnf;
    }
    __syncwarp();
  }
  if (lane == 0) {
    if (nhp) atomicAdd(sp.counters + (r_is_native(T{}) ? 6 : 1), nhp);
    // a frequency re-solved from the FP64 list was counted by the double-float pass
    if (nhp && list == 1) atomicSub(sp.counters + 1, nhp);
    if (nbad) atomicAdd(sp.counters + 2, nbad);
    if (nfixed) atomicSub(sp.counters + 2, nfixed);
    if (nnf) atomicAdd(sp.counters + 3, nnf);
  }
}

__global__ void k_exp_table(float4* tab) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < 1024) {
    double s, c;
    sincospi(2.0 * (double)n / 1024.0, &s, &c);
    const float ch = (float)c, sh = (float)s;
    tab[n] = make_float4(ch, (float)(c - (double)ch), sh, (float)(s - (double)sh));
  }
}


template <int NMAX>
cudaError_t launch_f32_n(const SolveParams& p, bool estimate, cudaStream_t st) {
  const size_t smem = (size_t)(kViewChunk * 4 * kTileBins + kTileBins * NMAX +
                               kTileBins * NMAX * (NMAX + 1)) * sizeof(float2);
  const size_t smem_sums = (size_t)(kViewChunk * 4 * kTileBins + kTileBins * 2 * kLatMax * 32) * sizeof(float2);
  cudaError_t e = set_smem((const void*)k_solve_f32<NMAX>, smem);
  if (e == cudaSuccess) e = set_smem((const void*)k_f32_sums, smem_sums);
  if (e != cudaSuccess) return e;
  // one tile per CTA: short CTAs let higher-priority work interleave; with p.f32sums the view
  // sums of each chunk of tiles go first to their own kernel
  const int ntiles = (p.H * (p.W / 2 + 1) + kTileBins - 1) / kTileBins;
  const int chunk = p.f32sums != nullptr ? p.f32sums_tiles : ntiles;
  for (int t0 = 0; t0 < ntiles; t0 += chunk) {
    const int t1 = std::min(ntiles, t0 + chunk);
    float4* wsum = nullptr;
    float2* ysum = nullptr;
    if (p.f32sums != nullptr) {
      wsum = p.f32sums;
      ysum = reinterpret_cast<float2*>(p.f32sums + (size_t)p.f32sums_tiles * kTileBins * 32);
      k_f32_sums<<<t1 - t0, kTileBins * 32, smem_sums, st>>>(p, t0, t1, wsum, ysum);
    }
    k_solve_f32<NMAX><<<t1 - t0, kTileBins * 32, smem, st>>>(p, estimate ? 1 : 0, t0, t1, wsum, ysum);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_hp_t(const SolveParams& p, bool all_bins, int list, cudaStream_t st) {
  const size_t per_warp = hp_warp_elems<T>(p.N, p.C) * sizeof(cx<T>);
  int warps = (int)(96 * 1024 / per_warp);
  if (warps > 4) warps = 4;
  if (warps < 1) warps = 1;
  const size_t smem = per_warp * warps;
  cudaError_t e = set_smem((const void*)k_solve_hp<T>, smem);
  if (e != cudaSuccess) return e;
  // every frequency: one per warp; a list (its length known on the device only, usually
  // short or empty): at most 8 CTAs per SM that stride over it, so that an empty list costs a
  // few microseconds instead of one CTA launch per possible entry
  const int bins = p.H * (p.W / 2 + 1);
  int grid = (bins + warps - 1) / warps;
  if (!all_bins) grid = std::min(grid, 8 * num_sms());
  k_solve_hp<T><<<grid, warps * 32, smem, st>>>(p, all_bins ? 1 : 0, warps, list);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_solve_f32(const SolveParams& p, bool estimate, cudaStream_t st) {
  if (p.N <= 8) return launch_f32_n<8>(p, estimate, st);
  if (p.N <= 16) return launch_f32_n<16>(p, estimate, st);
  return launch_f32_n<32>(p, estimate, st);
}

cudaError_t launch_solve_hp(const SolveParams& p, bool all_bins, bool f64, int list, cudaStream_t st) {
  return f64 ? launch_hp_t<R64>(p, all_bins, list, st) : launch_hp_t<Rdf>(p, all_bins, list, st);
}

cudaError_t launch_exp_table(float4* table, cudaStream_t st) {
  k_exp_table<<<4, 256, 0, st>>>(table);
  return cudaGetLastError();
}

}  // namespace fdl
