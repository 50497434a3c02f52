// High-precision per-frequency solve shared by the layer construction
// (Sec. V-A) and the calibration gradient (Sec. V-B).  One warp solves one
// frequency; the matrix lives in shared memory as cx<T>, T = Rdf
// (double-float) or R64 (native FP64).
#pragma once

#include "kernels.h"

namespace fdl {

__device__ __forceinline__ void bin_coords(int q, int H, int M, int& ky, int& kx) {
  const int main_bins = H * M;
  if (q < main_bins) {
    ky = q / M;
    kx = q - ky * M;
  } else {
    ky = q - main_bins;
    kx = M;
  }
}

// Gamma^T Gamma of Gamma = tridiag(1, -2, 1), N x N (Eq. 2ndOrderLayer).
__device__ __forceinline__ float layer2_gtg(int i, int l, int N) {
  const int dlt = i > l ? i - l : l - i;
  if (dlt == 0) return 4.f + (i > 0 ? 1.f : 0.f) + (i < N - 1 ? 1.f : 0.f);
  if (dlt == 1) return -4.f;
  if (dlt == 2) return 1.f;
  return 0.f;
}

// theta = u . w in cycles per unit of disparity, and the phase d theta of
// A_jk = exp(2 pi i d_k theta_j) (Eq. AMatGeneral).
//
// FP64: theta and d theta rounded once each (absolute phase error about
// 2^-53 |d theta|).  Double-float: theta is kept unevaluated as the exact sum
// p1 + e1 + p2 + e2 of two TwoProducts, each piece is multiplied by d exactly
// (TwoProduct again), the two large products are reduced mod 1 exactly
// (x - rint(x) is exact in floating point) and only then is everything
// summed.  The phase then carries an absolute error of about 2^-48 however
// large |d theta| is; rounding theta and d theta as double-floats instead
// would leave 2^-47 |d theta|, which at |d theta| ~ 20 cycles (views at
// |u| ~ 9) dominated the error of ill-conditioned frequencies.
// The frequency as each arithmetic wants it, formed once per bin: FP64 divides the
// integers; double-float keeps the float quotients and remainders.
struct FreqD {
  double wx, wy;
};
__device__ __forceinline__ FreqD freq_prep(const Freq& f, R64) {
  return {(double)f.kx / (double)f.W, (double)f.kyp / (double)f.H};
}
__device__ __forceinline__ const Freq& freq_prep(const Freq& f, Rdf) { return f; }

__device__ __forceinline__ R64 theta_r(float ux, float uy, const FreqD& f, R64) {
  return {(double)ux * f.wx + (double)uy * f.wy};
}
__device__ __forceinline__ R64 phase_r(R64 th, float d) { return {th.v * (double)d}; }

struct ThetaX {
  float p1, e1, p2, e2;
  float g;  // u . (remainders of w): 0 for power-of-two sizes
};
__device__ __forceinline__ ThetaX theta_r(float ux, float uy, const Freq& f, Rdf) {
  const df a = two_prod(ux, f.wx), b = two_prod(uy, f.wy);
  return {a.hi, a.lo, b.hi, b.lo, fmaf(ux, f.wx_lo, uy * f.wy_lo)};
}
__device__ __forceinline__ Rdf phase_r(const ThetaX& t, float d) {
  const df a = two_prod(d, t.p1), b = two_prod(d, t.p2);  // exact
  const df c = two_prod(d, t.e1), e = two_prod(d, t.e2);  // exact, |c|, |e| <= 2^-24 |a|, |b|
  const df s = two_sum(__fsub_rn(a.hi, rintf(a.hi)), __fsub_rn(b.hi, rintf(b.hi)));  // exact, |s| <= 1
  const df m1 = two_sum(a.lo, b.lo);
  const df m2 = two_sum(c.hi, e.hi);
  df m = two_sum(m1.hi, m2.hi);
  // d g: rounding 2^-24 |d g| ~ 2^-48 |d theta| (only for sizes that are not powers of two)
  const df m3 = two_sum(m.hi, d * t.g);
  m = {m3.hi, __fadd_rn(__fadd_rn(m.lo, m3.lo), __fadd_rn(__fadd_rn(m1.lo, m2.lo), __fadd_rn(c.lo, e.lo)))};
  // |s| <= 1 and |m| ~ 2^-24 |d theta|: the sloppy double-word addition (error ~2^-46
  // (|s| + |m|)) keeps the absolute error of the phase at that level
  const df v = two_sum(s.hi, m.hi);
  return {fast_two_sum(v.hi, __fadd_rn(v.lo, __fadd_rn(s.lo, m.lo)))};
}

// w in the solve's arithmetic: FP64 from the integers, double-float from the quotient and
// its remainder
__device__ __forceinline__ R64 freq_x_r(const FreqD& f, R64) { return {f.wx}; }
__device__ __forceinline__ R64 freq_y_r(const FreqD& f, R64) { return {f.wy}; }
__device__ __forceinline__ Rdf freq_x_r(const Freq& f, Rdf) { return {{f.wx, f.wx_lo}}; }
__device__ __forceinline__ Rdf freq_y_r(const Freq& f, Rdf) { return {{f.wy, f.wy_lo}}; }

// exp(2 pi i t), FP64: CUDA's sincospi after reduction to [-1/2, 1/2].
__device__ __forceinline__ cx<R64> cexp2pi(R64 t, const float4*) {
  const double f = t.v - rint(t.v);
  double s, c;
  sincospi(2.0 * f, &s, &c);
  return {{c}, {s}};
}

// exp(2 pi i t), double-float: t reduced to f in [-1/2, 1/2] and split as
// f = n/1024 + r (table-driven reduction); exp(2 pi i n/1024) comes from a
// double-float table, exp(2 pi i r) with |2 pi r| <= pi/1024 from its Taylor
// series (cos: 1 - x^2/2 + x^4/24, sin: x (1 - x^2/6 + x^4/120); the first
// omitted terms are below 2^-59).
__device__ __forceinline__ cx<Rdf> cexp2pi(Rdf t, const float4* tab) {
  const float nI = rintf(t.v.hi);
  const df f = two_sum(__fsub_rn(t.v.hi, nI), t.v.lo);
  const float nf = rintf(f.hi * 1024.f);
  const int n = (int)nf;
  const df r = two_sum(__fsub_rn(f.hi, nf * (1.f / 1024.f)), f.lo);
  const df twopi = {6.28318548202514648f, -1.74845553146951720e-07f};
  const df x = df_mul(r, twopi);
  const df x2 = df_mul(x, x);
  const float x2f = x2.hi;
  df cs = df_add_f(df_mul_f(x2, -0.5f), x2f * x2f * (1.f / 24.f));
  cs = df_add_f(cs, 1.f);
  const df sixth = {0.16666667163372040f, -4.96705387931228900e-09f};
  df sp = df_add_f(df_neg(df_mul(x2, sixth)), x2f * x2f * (1.f / 120.f));
  sp = df_add_f(sp, 1.f);
  const df sn = df_mul(x, sp);
  const float4 e = __ldg(tab + (n & 1023));
  const df ec = {e.x, e.y}, es = {e.z, e.w};
  // terms of magnitude <= 1: the sloppy double-word addition keeps the absolute error
  // at ~2^-46 (what A's entries need) for half the operations of the accurate one
  const df p1 = df_mul(ec, cs), p2 = df_neg(df_mul(es, sn));
  const df q1 = df_mul(ec, sn), q2 = df_mul(es, cs);
  const df r1 = two_sum(p1.hi, p2.hi), r2 = two_sum(q1.hi, q2.hi);
  const df re = fast_two_sum(r1.hi, __fadd_rn(r1.lo, __fadd_rn(p1.lo, p2.lo)));
  const df im = fast_two_sum(r2.hi, __fadd_rn(r2.lo, __fadd_rn(q1.lo, q2.lo)));
  return {{re}, {im}};
}

struct HpProblem {
  SpecView b;
  const float* u;
  const float* d;
  const float4* exp_table;
  int K, C, N, H, W, reg;
  double lam, lam_eps;
  const float* P = nullptr;             // free shifts [K][N][2] (the relaxed model) or null: u_j d_k
  const fdl_request* views = nullptr;   // per-image aperture and focus [K] or null: psi = delta
};

// psi_hat_j((s_j - d_k) w) of an image's aperture (Eq. AMatGeneral) in double: the closed
// forms of the disc (J1), the square (sinc) and a point set; a drawn-aperture table by
// bilinear interpolation of its FP32 entries.  wx, wy: the frequency in double.
__device__ __forceinline__ void view_aperture(const fdl_request& v, float dk, double wy, double wx, double& re,
                                              double& im) {
  re = 1.0;
  im = 0.0;
  const double sd = (double)v.s - (double)dk;
  const double nuy = sd * wy, nux = sd * wx;
  if (v.aperture == FDL_AP_POINTS) {
    double ar = 0.0, ai = 0.0;
    for (int m = 0; m < v.npts; ++m) {
      const double px = (double)__ldg(v.pts + 2 * m), py = (double)__ldg(v.pts + 2 * m + 1);
      double sn, cs;
      sincospi(-2.0 * (px * nux + py * nuy), &sn, &cs);
      ar += cs;
      ai += sn;
    }
    re = v.npts > 0 ? ar / v.npts : 0.0;
    im = v.npts > 0 ? ai / v.npts : 0.0;
    return;
  }
  if (v.aperture == FDL_AP_TABLE) {
    const int Z = v.npts;
    if (Z < 1) return;
    const float2* T = reinterpret_cast<const float2*>(v.pts);
    double gy = nuy * Z * (double)v.radius, gx = nux * Z * (double)v.radius;
    if (!(fabs(gy) < 1e30) || !(fabs(gx) < 1e30)) {
      re = 0.0;
      return;
    }
    gy -= Z * floor(gy / Z);
    gx -= Z * floor(gx / Z);
    const double y0f = fmin(floor(gy), (double)(Z - 1)), x0f = fmin(floor(gx), (double)(Z - 1));
    const double fy = gy - y0f, fx = gx - x0f;
    const int y0 = (int)y0f, x0 = (int)x0f;
    const int Zh = Z / 2 + 1;
    double acc_r = 0.0, acc_i = 0.0;
    for (int t = 0; t < 4; ++t) {
      int iy = y0 + (t >> 1), ix = x0 + (t & 1);
      iy = iy >= Z ? iy - Z : iy;
      ix = ix >= Z ? ix - Z : ix;
      float2 e;
      if (ix <= Z / 2) {
        e = __ldg(T + (long long)iy * Zh + ix);
      } else {
        e = __ldg(T + (long long)(iy ? Z - iy : 0) * Zh + (Z - ix));
        e.y = -e.y;
      }
      const double wgt = ((t >> 1) ? fy : 1.0 - fy) * ((t & 1) ? fx : 1.0 - fx);
      acc_r += wgt * e.x;
      acc_i += wgt * e.y;
    }
    re = acc_r;
    im = acc_i;
    return;
  }
  if (v.aperture == FDL_AP_PINHOLE || v.radius == 0.f) return;
  if (v.aperture == FDL_AP_DISC) {
    const double z = 6.283185307179586 * (double)v.radius * sqrt(nux * nux + nuy * nuy);
    re = z < 1e-8 ? 1.0 - 0.125 * z * z : 2.0 * j1(z) / z;
    return;
  }
  // square of half side r
  const double sx = 2.0 * (double)v.radius * nux, sy = 2.0 * (double)v.radius * nuy;
  const double fx = sx == 0.0 ? 1.0 : sinpi(sx) / (3.141592653589793 * sx);
  const double fy = sy == 0.0 ? 1.0 : sinpi(sy) / (3.141592653589793 * sy);
  re = fx * fy;
}
__device__ __forceinline__ double freq_x_double(const FreqD& f) { return f.wx; }
__device__ __forceinline__ double freq_y_double(const FreqD& f) { return f.wy; }
__device__ __forceinline__ double freq_x_double(const Freq& f) { return (double)f.wx + (double)f.wx_lo; }
__device__ __forceinline__ double freq_y_double(const Freq& f) { return (double)f.wy + (double)f.wy_lo; }

// Shared memory of one warp: G [N][N+1], Arow [N], Y [N][C] (cx<T>).
template <class T>
__host__ __device__ __forceinline__ size_t hp_warp_elems(int N, int C) {
  return (size_t)N * (N + 1) + N + (size_t)N * C;
}

// Builds G = A*A + lambda Gamma*Gamma and Y = A* b at bin (ky, kx), factors
// G = L L* in place and overwrites Y with x.  Returns false if a pivot was
// not positive.  All lanes of the warp must call.
template <class T>
__device__ bool hp_solve_bin(const HpProblem& p, int ky, int kx, cx<T>* G, cx<T>* Arow, cx<T>* Y) {
  const int lane = threadIdx.x & 31;
  const int N = p.N, C = p.C, M = p.W >> 1;
  const int ld = N + 1;
  const T zero = r_from(0.f, T{});
  const Freq fq0 = bin_freq(ky, kx, p.H, p.W);
  const auto fq = freq_prep(fq0, T{});
  for (int e = lane; e < N * ld; e += 32) G[e] = {zero, zero};
  for (int e = lane; e < N * C; e += 32) Y[e] = {zero, zero};
  __syncwarp();
  for (int j = 0; j < p.K; ++j) {
    if (p.P == nullptr) {
      const float2 uj = __ldg(reinterpret_cast<const float2*>(p.u) + j);
      const auto th = theta_r(uj.x, uj.y, fq, T{});
      for (int r = lane; r < N; r += 32) Arow[r] = cexp2pi(phase_r(th, __ldg(p.d + r)), p.exp_table);
    } else {
      for (int r = lane; r < N; r += 32) {
        const float2 pr = __ldg(reinterpret_cast<const float2*>(p.P) + (long long)j * N + r);
        Arow[r] = cexp2pi(phase_r(theta_r(pr.x, pr.y, fq, T{}), 1.f), p.exp_table);
      }
    }
    if (p.views != nullptr) {
      const fdl_request v = p.views[j];
      for (int r = lane; r < N; r += 32) {
        double ar, ai;
        view_aperture(v, __ldg(p.d + r), freq_y_double(fq), freq_x_double(fq), ar, ai);
        Arow[r] = cx_mul(Arow[r], cx<T>{r_from_double(ar, T{}), r_from_double(ai, T{})});
      }
    }
    __syncwarp();
    float2 bj[4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
      bj[c] = c < C ? *p.b.at((long long)j * C + c, ky, kx, M) : make_float2(0.f, 0.f);
    for (int r = lane; r < N; r += 32) {
      const cx<T> ar = Arow[r];
      for (int l = 0; l <= r; ++l) G[r * ld + l] = cx_add(G[r * ld + l], cx_mulc(ar, Arow[l]));
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c < C) Y[r * C + c] = cx_add(Y[r * C + c], cx_mulc_f(ar, bj[c]));
    }
    __syncwarp();
  }
  {
    const T wxr = freq_x_r(fq, T{}), wyr = freq_y_r(fq, T{});
    const T w2 = wxr * wxr + wyr * wyr;
    const T w4 = w2 * w2;
    const T lam = r_from_double(p.lam, T{});
    const T lame = r_from_double(p.lam_eps, T{});
    for (int r = lane; r < N; r += 32) {
      if (p.reg == 0) {
        const T dr = r_from(__ldg(p.d + r), T{});
        const T d2 = dr * dr;
        G[r * ld + r].re = G[r * ld + r].re + (lam * (w4 * (d2 * d2)) + lame);
      } else if (p.reg == 1) {
        for (int l = (r >= 2 ? r - 2 : 0); l <= r; ++l)
          G[r * ld + l].re = G[r * ld + l].re + mulf(lam, layer2_gtg(r, l, N));
      } else {
        G[r * ld + r].re = G[r * ld + r].re + lam;
      }
    }
  }
  __syncwarp();
  bool ok = true;
  const T one = r_from(1.f, T{});
  for (int k = 0; k < N; ++k) {
    const T piv = G[k * ld + k].re;
    const bool pos = r_to_double(piv) > 0.0;
    ok = ok && pos;
    const T lkk = r_sqrt(pos ? piv : one);
    const T inv = one / lkk;
    __syncwarp();
    for (int r = lane; r < N; r += 32) {
      if (r > k) G[r * ld + k] = cx_scale(G[r * ld + k], inv);
      else if (r == k) G[k * ld + k] = {lkk, zero};
    }
    __syncwarp();
    for (int r = lane; r < N; r += 32) {
      if (r > k) {
        const cx<T> lrk = G[r * ld + k];
        for (int l = k + 1; l <= r; ++l) G[r * ld + l] = cx_sub(G[r * ld + l], cx_mul_conj(lrk, G[l * ld + k]));
      }
    }
    __syncwarp();
  }
  if (lane < C) {
    const int c = lane;
    for (int k = 0; k < N; ++k) {
      cx<T> acc = Y[k * C + c];
      for (int l = 0; l < k; ++l) acc = cx_sub(acc, cx_mul(G[k * ld + l], Y[l * C + c]));
      Y[k * C + c] = cx_scale(acc, one / G[k * ld + k].re);
    }
    for (int k = N - 1; k >= 0; --k) {
      cx<T> acc = Y[k * C + c];
      for (int l = k + 1; l < N; ++l) acc = cx_sub(acc, cx_mulc(G[l * ld + k], Y[l * C + c]));
      Y[k * C + c] = cx_scale(acc, one / G[k * ld + k].re);
    }
  }
  __syncwarp();
  return ok;
}

}  // namespace fdl
