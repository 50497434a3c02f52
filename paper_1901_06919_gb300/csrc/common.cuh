// Shared device helpers of the FDL kernels: complex float arithmetic, the
// double-float ("df": an unevaluated sum hi + lo of two floats) arithmetic
// used for the high-precision solve, and the accessor of half spectra.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fdl {

constexpr int kWarp = 32;

// ---------------------------------------------------------------- complex f32
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
// acc += a * b
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}
// acc -= a * conj(b)
__device__ __forceinline__ void cfms_c(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(-a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// ------------------------------------------------------------- double-float
// Error-free transformations: TwoSum (Knuth), Fast2Sum (Dekker, needs
// |a| >= |b|), and the FMA-based TwoProd.  The arithmetic below follows the
// "accurate" double-word algorithms analysed by Joldes, Muller and Popescu
// (ACM TOMS 2017): relative error of a sum or product about 2^-47 or better.
struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = fmaf(a, b, -p);
  return {p, e};
}
__device__ __forceinline__ df df_from(float a) { return {a, 0.f}; }
__device__ __forceinline__ df df_from_double(double a) {
  float h = (float)a;
  return {h, (float)(a - (double)h)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  df t = two_sum(a.lo, b.lo);
  float c = __fadd_rn(s.lo, t.hi);
  df v = fast_two_sum(s.hi, c);
  float w = __fadd_rn(t.lo, v.lo);
  return fast_two_sum(v.hi, w);
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = two_sum(a.hi, b);
  float v = __fadd_rn(a.lo, s.lo);
  return fast_two_sum(s.hi, v);
}
__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  float t = __fmul_rn(a.hi, b.lo);
  t = fmaf(a.lo, b.hi, t);
  float c = __fadd_rn(p.lo, t);
  return fast_two_sum(p.hi, c);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  float c = fmaf(a.lo, b, p.lo);
  return fast_two_sum(p.hi, c);
}
// a / b: one quotient digit, two corrections.
__device__ __forceinline__ df df_div(df a, df b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  df r = df_sub(a, df_mul_f(b, q1));
  float q2 = __fdiv_rn(r.hi, b.hi);
  r = df_sub(r, df_mul_f(b, q2));
  float q3 = __fdiv_rn(r.hi, b.hi);
  df q = fast_two_sum(q1, q2);
  return df_add_f(q, q3);
}
// sqrt(a) for a > 0: float root refined by one Newton step in df.
__device__ __forceinline__ df df_sqrt(df a) {
  float s = __fsqrt_rn(a.hi);
  df r = df_sub(a, two_prod(s, s));
  float e = __fdiv_rn(r.hi, 2.f * s);
  return fast_two_sum(s, e);
}

// A real type for the high-precision solve: native double or df, used
// through the same names so one kernel template serves both.
struct R64 {
  double v;
};
struct Rdf {
  df v;
};

__device__ __forceinline__ R64 operator+(R64 a, R64 b) { return {a.v + b.v}; }
__device__ __forceinline__ R64 operator-(R64 a, R64 b) { return {a.v - b.v}; }
__device__ __forceinline__ R64 operator*(R64 a, R64 b) { return {a.v * b.v}; }
__device__ __forceinline__ R64 operator/(R64 a, R64 b) { return {a.v / b.v}; }
__device__ __forceinline__ R64 operator-(R64 a) { return {-a.v}; }
__device__ __forceinline__ R64 r_sqrt(R64 a) { return {sqrt(a.v)}; }  // sqrt
__device__ __forceinline__ R64 mulf(R64 a, float b) { return {a.v * (double)b}; }
__device__ __forceinline__ R64 r_from(float a, R64) { return {(double)a}; }
__device__ __forceinline__ R64 r_from_double(double a, R64) { return {a}; }
__device__ __forceinline__ float r_to_float(R64 a) { return (float)a.v; }
__device__ __forceinline__ double r_to_double(R64 a) { return a.v; }

__device__ __forceinline__ Rdf operator+(Rdf a, Rdf b) { return {df_add(a.v, b.v)}; }
__device__ __forceinline__ Rdf operator-(Rdf a, Rdf b) { return {df_sub(a.v, b.v)}; }
__device__ __forceinline__ Rdf operator*(Rdf a, Rdf b) { return {df_mul(a.v, b.v)}; }
__device__ __forceinline__ Rdf operator/(Rdf a, Rdf b) { return {df_div(a.v, b.v)}; }
__device__ __forceinline__ Rdf operator-(Rdf a) { return {df_neg(a.v)}; }
__device__ __forceinline__ Rdf r_sqrt(Rdf a) { return {df_sqrt(a.v)}; }
__device__ __forceinline__ Rdf mulf(Rdf a, float b) { return {df_mul_f(a.v, b)}; }
__device__ __forceinline__ Rdf r_from(float a, Rdf) { return {df_from(a)}; }
__device__ __forceinline__ Rdf r_from_double(double a, Rdf) { return {df_from_double(a)}; }
__device__ __forceinline__ float r_to_float(Rdf a) { return a.v.hi + a.v.lo; }
__device__ __forceinline__ double r_to_double(Rdf a) { return df_to_double(a.v); }

template <class T>
struct cx {
  T re, im;
};
template <class T>
__device__ __forceinline__ cx<T> cx_add(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T>
__device__ __forceinline__ cx<T> cx_sub(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <class T>
__device__ __forceinline__ cx<T> cx_mul(cx<T> a, cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <class T>
__device__ __forceinline__ cx<T> cx_mulc(cx<T> a, cx<T> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// a * conj(b)
template <class T>
__device__ __forceinline__ cx<T> cx_mul_conj(cx<T> a, cx<T> b) {
  return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
// conj(a) * b with b single precision
template <class T>
__device__ __forceinline__ cx<T> cx_mulc_f(cx<T> a, float2 b) {
  return {mulf(a.re, b.x) + mulf(a.im, b.y), mulf(a.re, b.y) - mulf(a.im, b.x)};
}
template <class T>
__device__ __forceinline__ cx<T> cx_scale(cx<T> a, T s) { return {a.re * s, a.im * s}; }

// --------------------------------------------------------------- spectra
// A stack of half spectra [img][H][W/2+1], stored either densely (pitch
// W/2+1, the public layout) or split (the kx < W/2 part with pitch W/2 and
// the kx = W/2 column in a separate [img][H] plane, the internal layout that
// keeps every row 16-byte aligned).
struct SpecView {
  float2* main;
  float2* nyq;
  long long img_stride;  // elements between images in `main`
  long long nyq_img_stride;
  int pitch;             // elements between rows in `main`
  int nyq_stride;        // elements between rows in `nyq`
  __device__ __forceinline__ float2* at(long long img, int ky, int kx, int half) const {
    return kx < half ? main + img * img_stride + (long long)ky * pitch + kx
                     : nyq + img * nyq_img_stride + (long long)ky * nyq_stride;
  }
};

inline SpecView spec_dense(float2* p, int H, int W) {
  SpecView s;
  s.main = p;
  s.nyq = p + W / 2;
  s.img_stride = (long long)H * (W / 2 + 1);
  s.nyq_img_stride = s.img_stride;
  s.pitch = W / 2 + 1;
  s.nyq_stride = W / 2 + 1;
  return s;
}
inline SpecView spec_split(float2* main, float2* nyq, int H, int W) {
  SpecView s;
  s.main = main;
  s.nyq = nyq;
  s.img_stride = (long long)H * (W / 2);
  s.nyq_img_stride = H;
  s.pitch = W / 2;
  s.nyq_stride = 1;
  return s;
}

// Frequency of stored bin (ky, kx) in cycles per pixel.
__device__ __forceinline__ float freq_y(int ky, int H) {
  return (ky < (H + 1) / 2 ? (float)ky : (float)(ky - H)) / (float)H;
}

// Frequency of stored bin (ky, kx), w = (ky', kx) / (H, W) with ky' = ky or ky - H: the
// correctly rounded quotient plus the float remainder of the division (wy + wy_lo,
// wx + wx_lo equal w to ~2^-48 relative; the remainders are 0 when H and W are powers of
// two, where the quotients are exact binary fractions).
struct Freq {
  float wy, wx, wy_lo, wx_lo;
  int kyp, kx, H, W;
};
__device__ __forceinline__ Freq bin_freq(int ky, int kx, int H, int W) {
  Freq f;
  f.kyp = ky < (H + 1) / 2 ? ky : ky - H;
  f.kx = kx;
  f.H = H;
  f.W = W;
  f.wy = __fdiv_rn((float)f.kyp, (float)H);
  f.wx = __fdiv_rn((float)kx, (float)W);
  // k - w n is exact (the remainder of a correctly rounded quotient)
  f.wy_lo = __fdiv_rn(fmaf(-f.wy, (float)H, (float)f.kyp), (float)H);
  f.wx_lo = __fdiv_rn(fmaf(-f.wx, (float)W, (float)kx), (float)W);
  return f;
}

// Phase in cycles reduced to [-1/2, 1/2]:  t = d (u_x w_x + u_y w_y) with w_x, w_y exact
// binary fractions; the products are kept exact (TwoProd).
__device__ __forceinline__ float phase_cycles_f(float ux, float uy, float wx, float wy, float d) {
  df px = two_prod(ux, wx);
  df py = two_prod(uy, wy);
  df th = df_add(px, py);
  df t = df_mul_f(th, d);
  const float n = rintf(t.hi);
  return __fadd_rn(__fsub_rn(t.hi, n), t.lo);
}

// Phase of A_jk in cycles, reduced to [-1/2, 1/2]:  t = d (u . w), accurate to a few ulp
// of 1/2 (the remainders of w enter the low word).
__device__ __forceinline__ float phase_cycles(float ux, float uy, const Freq& f, float d) {
  df px = two_prod(ux, f.wx);
  df py = two_prod(uy, f.wy);
  df th = df_add(px, py);
  th = df_add_f(th, fmaf(ux, f.wx_lo, uy * f.wy_lo));
  df t = df_mul_f(th, d);
  const float n = rintf(t.hi);
  return __fadd_rn(__fsub_rn(t.hi, n), t.lo);
}

int ilog2(int v);

}  // namespace fdl
