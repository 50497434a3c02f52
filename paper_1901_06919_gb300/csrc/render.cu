// Rendering of Sec. VI-A: the spectrum of the image seen from u0 with
// aperture psi focused at disparity s (Eq. BsFourier),
//   B_hat(w) = sum_k exp(+2 pi i d_k (u0 . w)) psi_hat((s - d_k) w) L_hat^k(w),
// written per request into the split half-spectrum layout, ready for the
// inverse column and row DFT passes.  psi is normalised to integrate to 1,
// so psi_hat(0) = 1 and a pinhole (psi = delta) gives psi_hat = 1 (Sec. IV-B).
#include <algorithm>

#include "hp_solve.cuh"
#include "stockham.cuh"

namespace fdl {

namespace {

// sin(pi x) / (pi x): the Taylor series in (pi x)^2 to the (pi x)^8 term for |x| < 1/4 (first
// omitted term below 3e-9), else the SFU sine of pi (x - 2 rint(x / 2)) in [-pi, pi] (absolute
// error about 2^-21 there) over pi x >= pi / 4.
__device__ __forceinline__ float sinc_pi(float x) {
  const float px = 3.14159265f * x;
  if (fabsf(x) < 0.25f) {
    const float t = px * px;
    return 1.f + t * (-1.f / 6.f + t * (1.f / 120.f + t * (-1.f / 5040.f + t * (1.f / 362880.f))));
  }
  const float xr = fmaf(-2.f, rintf(0.5f * x), x);
  return __fdividef(__sinf(3.14159265f * xr), px);
}

// Fourier transform of the aperture at nu = (s - d_k) w (cycles per unit of u).
__device__ __forceinline__ float2 aperture_hat(int kind, float radius, const float* pts, int npts, float nuy,
                                               float nux) {
  if (kind == FDL_AP_POINTS) {
    // (1/M) sum_m exp(-2 pi i u_m . nu)
    float2 acc = make_float2(0.f, 0.f);
    for (int m = 0; m < npts; ++m) {
      const float2 pm = __ldg(reinterpret_cast<const float2*>(pts) + m);
      const float f = phase_cycles_f(pm.x, pm.y, nux, nuy, -1.f);
      float sn, cs;
      sincospif(2.f * f, &sn, &cs);
      acc.x += cs;
      acc.y += sn;
    }
    const float inv = npts > 0 ? 1.f / (float)npts : 0.f;
    return make_float2(acc.x * inv, acc.y * inv);
  }
  if (kind == FDL_AP_PINHOLE || radius == 0.f) return make_float2(1.f, 0.f);
  if (kind == FDL_AP_DISC) {
    // 2 J1(z) / z with z = 2 pi r |nu|
    const float z = 6.283185307f * radius * sqrtf(nux * nux + nuy * nuy);
    if (z < 1e-3f) return make_float2(1.f - 0.125f * z * z, 0.f);
    return make_float2(2.f * j1f(z) / z, 0.f);
  }
  // square of half side r: sinc(2 r nu_x) sinc(2 r nu_y), sinc(x) = sin(pi x) / (pi x)
  return make_float2(sinc_pi(2.f * radius * nux) * sinc_pi(2.f * radius * nuy), 0.f);
}

// psi_hat(nu) of a drawn aperture: bilinear interpolation of the table T (half spectrum
// [Z][Z/2+1] of fdl_aperture_table) at grid coordinates g = nu Z h, periodic in Z, with
// T(-g) = conj T(g) for the columns not stored (Sec. VI-A).
__device__ __forceinline__ float2 table_fetch(const float2* __restrict__ T, int Z, int iy, int ix) {
  iy = iy >= Z ? iy - Z : iy;  // iy, ix in [0, 2Z)
  ix = ix >= Z ? ix - Z : ix;
  const int Zh = Z / 2 + 1;
  if (ix <= Z / 2) return __ldg(T + (long long)iy * Zh + ix);
  const float2 v = __ldg(T + (long long)(iy ? Z - iy : 0) * Zh + (Z - ix));
  return make_float2(v.x, -v.y);
}
__device__ __forceinline__ float2 aperture_table_hat(const float2* __restrict__ T, int Z, float h, float nuy,
                                                     float nux) {
  if (Z < 1) return make_float2(1.f, 0.f);
  float gy = nuy * (float)Z * h, gx = nux * (float)Z * h;
  if (!(fabsf(gy) < 1e30f) || !(fabsf(gx) < 1e30f)) return make_float2(0.f, 0.f);
  gy -= (float)Z * floorf(gy / (float)Z);  // [0, Z]
  gx -= (float)Z * floorf(gx / (float)Z);
  const float y0f = fminf(floorf(gy), (float)(Z - 1)), x0f = fminf(floorf(gx), (float)(Z - 1));
  const float fy = gy - y0f, fx = gx - x0f;
  const int y0 = max((int)y0f, 0), x0 = max((int)x0f, 0);
  const float2 a = table_fetch(T, Z, y0, x0), b = table_fetch(T, Z, y0, x0 + 1);
  const float2 c = table_fetch(T, Z, y0 + 1, x0), e = table_fetch(T, Z, y0 + 1, x0 + 1);
  const float w00 = (1.f - fy) * (1.f - fx), w01 = (1.f - fy) * fx, w10 = fy * (1.f - fx), w11 = fy * fx;
  return make_float2(w00 * a.x + w01 * b.x + w10 * c.x + w11 * e.x, w00 * a.y + w01 * b.y + w10 * c.y + w11 * e.y);
}

// psi_hat of a disc, 2 J1(z) / z for z >= 0, from the rational approximations of Abramowitz
// and Stegun, Handbook of Mathematical Functions, 9.4.4 (z <= 3: J1(z) / z as a polynomial in
// (z/3)^2, error below 1.3e-8) and 9.4.6 (z > 3: J1 = z^-1/2 f1 cos(theta1), f1 and theta1
// polynomials in 3/z, errors below 4e-8 and 9e-8); theta1 is reduced to [-pi, pi] with a
// two-part 2 pi before the SFU cosine.
__device__ __forceinline__ float disc_hat(float z) {
  if (z <= 3.f) {
    const float t = z * z * (1.f / 9.f);
    return 2.f * (0.5f +
                  t * (-0.56249985f +
                       t * (0.21093573f + t * (-0.03954289f + t * (0.00443319f + t * (-0.00031761f + t * 0.00001109f))))));
  }
  const float y = __fdividef(3.f, z);
  const float f1 =
      0.79788456f +
      y * (0.00000156f + y * (0.01659667f + y * (0.00017105f + y * (-0.00249511f + y * (0.00113653f + y * -0.00020033f)))));
  float th = z - 2.35619449f +
             y * (0.12499612f + y * (0.00005650f + y * (-0.00637879f + y * (0.00074348f + y * (0.00079824f + y * -0.00029166f)))));
  const float n = rintf(th * 0.15915494f);
  th = fmaf(-n, 6.28125f, th);
  th = fmaf(-n, 1.9353071795864769e-3f, th);
  return 2.f * f1 * __cosf(th) * rsqrtf(z) * (y * (1.f / 3.f));  // 2 J1(z) / z = 2 f1 cos(theta1) z^-3/2
}

// Phase of exp(+2 pi i d (u0 . w)) in cycles, reduced to [-1/2, 1/2], from
// theta = u0 . w kept as a double-float (computed once per request and bin).
__device__ __forceinline__ float phase_from_theta(df theta, float d) {
  const df t = df_mul_f(theta, d);
  const float n = rintf(t.hi);
  return __fadd_rn(__fsub_rn(t.hi, n), t.lo);
}

constexpr int kRenderWarps = 8;
constexpr int kTileMaxLC = 256;  // N * C of an FDL staged in shared memory

// Staging of a tile of layer values, tile[e] = x0[(e / 32) * plane + off] for e < nlc * 32 (this
// thread's frequency at element offset off; zeros where !valid), by asynchronous global-to-shared
// copies of 8 bytes: every thread's copies are in flight at once and hold no registers.  The
// block is a multiple of 32 threads, so e % 32 is the lane.  Completion: cp_async_wait<n>
// (all but the n most recently committed groups of this thread), then a barrier.
__device__ __forceinline__ void stage_async(float2* tile, const float2* __restrict__ x0, int nlc, long long plane,
                                            long long off, bool valid) {
  const int n = nlc * 32;
  const unsigned base = (unsigned)__cvta_generic_to_shared(tile);
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const float2* src = valid ? x0 + (long long)(e >> 5) * plane + off : x0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(base + 8u * (unsigned)e), "l"(src),
                 "r"(valid ? 8 : 0)
                 : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

// sum over layers k = k0, k0 + kstep, ... < r.N of the Eq. BsFourier terms of request r at
// this lane's frequency; layer values from the shared tile (TILE) or from global memory;
// SHIFTS: the request's per-layer shifts P_k in shb (the relaxed model), else u0 d_k.
// AP: 0 no aperture factor (pinhole, or a disc of radius 0), 1 disc, 2 drawn (table),
// 3 square or points.  UNR: layers unrolled (their global loads in flight together).
template <int CC, bool TILE, bool SHIFTS, int AP, int UNR>
__device__ __forceinline__ void render_terms_t(const fdl_request& r, int k0, int kstep, int C, df theta, float wy,
                                               float wx, float wabs, long long plane, long long off, bool valid,
                                               const float2* tile, const float* dsh, int lane, float2 acc[4],
                                               const float2* __restrict__ shb, const Freq& fq) {
  const float2* x = reinterpret_cast<const float2*>(r.layers);
  const float zscale = 6.283185307f * r.radius * wabs;  // 2 pi r |w|
#pragma unroll(UNR)
  for (int k = k0; k < r.N; k += kstep) {
    const float dk = TILE ? dsh[k] : __ldg(r.d + k);
    float ph;
    if constexpr (SHIFTS) {
      const float2 pk = __ldg(shb + k);
      ph = phase_cycles(pk.x, pk.y, fq, 1.f);
    } else {
      ph = phase_from_theta(theta, dk);
    }
    // |2 pi ph| <= pi: the hardware sine and cosine (absolute error about 2^-21 there)
    // keep |coef| within 1e-6 of exact, far below the FP32 sum over layers it enters
    float2 coef;
    __sincosf(6.28318531f * ph, &coef.y, &coef.x);
    if constexpr (AP != 0) {
      const float sd = r.s - dk;
      if constexpr (AP == 1) {
        coef = cscale(coef, disc_hat(zscale * fabsf(sd)));
      } else if constexpr (AP == 2) {
        coef = cmul(coef, aperture_table_hat(reinterpret_cast<const float2*>(r.pts), r.npts, r.radius, sd * wy, sd * wx));
      } else {
        coef = cmul(coef, aperture_hat(r.aperture, r.radius, r.pts, r.npts, sd * wy, sd * wx));
      }
    }
    if (valid) {
#pragma unroll
      for (int c = 0; c < CC; ++c)
        if (CC < 4 || c < C)
          cfma(acc[c], coef, TILE ? tile[(k * C + c) * 32 + lane] : __ldg(x + ((long long)k * C + c) * plane + off));
    }
  }
}

template <int CC, bool TILE, bool SHIFTS, int UNR>
__device__ __forceinline__ void render_terms_ap(const fdl_request& r, int k0, int kstep, int C, df theta, float wy,
                                                float wx, float wabs, long long plane, long long off, bool valid,
                                                const float2* tile, const float* dsh, int lane, float2 acc[4],
                                                const float2* __restrict__ shb, const Freq& fq) {
  const int ap = (r.aperture == FDL_AP_PINHOLE || (r.aperture == FDL_AP_DISC && r.radius == 0.f)) ? 0
                 : r.aperture == FDL_AP_DISC                                                  ? 1
                 : r.aperture == FDL_AP_TABLE                                                 ? 2
                                                                                              : 3;
#define FDL_TERMS(A) \
  render_terms_t<CC, TILE, SHIFTS, A, UNR>(r, k0, kstep, C, theta, wy, wx, wabs, plane, off, valid, tile, dsh, lane, acc, shb, fq)
  if (ap == 0) FDL_TERMS(0);
  else if (ap == 1) FDL_TERMS(1);
  else if (ap == 2) FDL_TERMS(2);
  else FDL_TERMS(3);
#undef FDL_TERMS
}

// the request's terms with the loop specialised for where the layers live, the shift model
// and the aperture kind (all uniform over the request).  The phase factor is evaluated
// directly at every layer here: a recurrence across layers measured slower in this kernel
// (a dependent chain per warp and request, and its set-up for the few layers each warp
// takes when the layers of one request are split across warps).  UNR applies to the layers
// read from global memory.
template <int CC, int UNR = 1>
__device__ __forceinline__ void render_terms(const fdl_request& r, int k0, int kstep, int C, df theta, float wy,
                                             float wx, float wabs, long long plane, long long off, bool valid,
                                             const float2* tile, const float* dsh, int lane, float2 acc[4],
                                             const float2* __restrict__ shb, const Freq& fq) {
#define FDL_AP(T, S) render_terms_ap<CC, T, S, T ? 1 : UNR>(r, k0, kstep, C, theta, wy, wx, wabs, plane, off, valid, tile, dsh, lane, acc, \
                                          shb, fq)
  if (tile != nullptr) {
    if (shb != nullptr) FDL_AP(true, true);
    else FDL_AP(true, false);
  } else {
    if (shb != nullptr) FDL_AP(false, true);
    else FDL_AP(false, false);
  }
#undef FDL_AP
}

// Two requests of one FDL, pinhole (AP 0) or disc (AP 1), no shift model: one pass over the
// layers loads each layer value once for both (from the shared tile when TILE, else from
// global memory at plane stride, UNR layers unrolled) and keeps two independent chains of
// phase, aperture and sums in flight.
template <int CC, int AP, bool TILE = true, int UNR = 1>
__device__ __forceinline__ void render_pair(const fdl_request& r1, const fdl_request& r2, int C, df th1, df th2,
                                            float wabs, bool valid, const float2* tile, const float* dsh, int lane,
                                            float2 acc1[4], float2 acc2[4], long long plane = 0,
                                            long long off = 0) {
  const float z1 = 6.283185307f * r1.radius * wabs, z2 = 6.283185307f * r2.radius * wabs;
  const float2* x = reinterpret_cast<const float2*>(r1.layers);
#pragma unroll(UNR)
  for (int k = 0; k < r1.N; ++k) {
    const float dk = TILE ? dsh[k] : __ldg(r1.d + k);
    float2 c1, c2;
    __sincosf(6.28318531f * phase_from_theta(th1, dk), &c1.y, &c1.x);
    __sincosf(6.28318531f * phase_from_theta(th2, dk), &c2.y, &c2.x);
    if constexpr (AP == 1) {
      c1 = cscale(c1, disc_hat(z1 * fabsf(r1.s - dk)));
      c2 = cscale(c2, disc_hat(z2 * fabsf(r2.s - dk)));
    }
    if (valid) {
#pragma unroll
      for (int c = 0; c < CC; ++c) {
        if (CC < 4 || c < C) {
          const float2 v = TILE ? tile[(k * C + c) * 32 + lane] : __ldg(x + ((long long)k * C + c) * plane + off);
          cfma(acc1[c], c1, v);
          cfma(acc2[c], c2, v);
        }
      }
    }
  }
}

// the aperture class of a request for render_pair: 0 pinhole (or a disc of radius 0), 1 disc,
// -1 anything else
__device__ __forceinline__ int pair_class(const fdl_request& r) {
  if (r.aperture == FDL_AP_PINHOLE || (r.aperture == FDL_AP_DISC && r.radius == 0.f)) return 0;
  return r.aperture == FDL_AP_DISC ? 1 : -1;
}

// CTA: 32 consecutive stored bins (lane = bin) x 8 warps; launched for B >= 8 requests
// (k_render_few takes smaller launches).
//  * 8 or more active requests: warp w renders requests w, w + 8, ...; when every request
//    reads the same FDL (and N*C <= tile_lc) the CTA first stages that FDL's layer values for
//    its 32 bins in shared memory and all requests read them there.
//  * fewer than 8 active (a device-side count below B, as in a captured serving batch): the
//    8 / count warps given to a request split its layers and their partial sums are added
//    through shared memory, so that one request still occupies the whole CTA.
template <int CC>
__global__ void __launch_bounds__(kRenderWarps * 32) k_render(const fdl_request* __restrict__ req, int B,
                                                              const int* __restrict__ count, int C, int H, int W,
                                                              int tile_lc, int nmax, SpecView out,
                                                              const float* __restrict__ shifts, int* __restrict__ status,
                                                              const int* __restrict__ gate) {
  extern __shared__ float2 tile[];  // [tile_lc][32]
  __shared__ float dsh[64];
  __shared__ float2 part[kRenderWarps][4][32];
  __shared__ int uniform;
  if (gate != nullptr && *gate == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int M = W >> 1;
  const int Qs = H * (M + 1);
  const int q = blockIdx.x * 32 + lane;
  const bool valid = q < Qs;
  int ky, kx;
  bin_coords(valid ? q : 0, H, M, ky, kx);
  const Freq fq = bin_freq(ky, kx, H, W);
  const float wy = fq.wy, wx = fq.wx;
  const float wylo = fq.wy_lo, wxlo = fq.wx_lo;
  const float wabs = sqrtf(wx * wx + wy * wy);
  const long long plane = (long long)H * (M + 1);
  const long long off = (long long)ky * (M + 1) + kx;
  const int Bact = count ? min(*count, B) : B;
  if (Bact <= 0) return;

  if (Bact < kRenderWarps) {
    const int G = kRenderWarps / Bact;  // warps per request
    const int b = warp / G, sl = warp - b * G;
    float2 acc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = make_float2(0.f, 0.f);
    const bool rok = b < Bact && request_ok(req[b], C, H, W, nmax, true);
    if (b < Bact && !rok && blockIdx.x == 0 && sl == 0 && lane == 0) atomicOr(status, FDL_ST_BAD_REQUEST);
    if (rok) {
      const fdl_request r = req[b];
      const df theta = df_add_f(df_add(two_prod(r.u0x, wx), two_prod(r.u0y, wy)), fmaf(r.u0x, wxlo, r.u0y * wylo));
      const float2* shb = shifts ? reinterpret_cast<const float2*>(shifts) + (long long)b * r.N : nullptr;
      render_terms<CC>(r, sl, G, C, theta, wy, wx, wabs, plane, off, valid, nullptr, nullptr, lane, acc, shb, fq);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) part[warp][c][lane] = acc[c];
    __syncthreads();
    if (rok && sl == 0 && valid) {
      for (int w = 1; w < G; ++w) {
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] = cadd(acc[c], part[warp + w][c][lane]);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c < C) *out.at((long long)b * C + c, ky, kx, M) = acc[c];
    }
    return;
  }

  if (threadIdx.x == 0) uniform = 1;
  __syncthreads();
  const float* L0 = req[0].layers;
  const int N0 = req[0].N;
  for (int b = threadIdx.x; b < Bact; b += blockDim.x)
    if (req[b].layers != L0 || req[b].d != req[0].d || req[b].N != N0 || !request_ok(req[b], C, H, W, nmax, true))
      uniform = 0;
  __syncthreads();
  const bool shared = uniform && N0 * C <= tile_lc && N0 <= 64;
  if (shared) {
    stage_async(tile, reinterpret_cast<const float2*>(L0), N0 * C, plane, off, valid);
    cp_async_commit();
    for (int k = threadIdx.x; k < N0; k += blockDim.x) dsh[k] = __ldg(req[0].d + k);
    cp_async_wait<0>();
    __syncthreads();
  }
  for (int b = warp; b < Bact; b += kRenderWarps) {
    if (!request_ok(req[b], C, H, W, nmax, true)) {
      if (blockIdx.x == 0 && lane == 0) atomicOr(status, FDL_ST_BAD_REQUEST);
      continue;
    }
    const fdl_request r = req[b];
    const df theta = df_add_f(df_add(two_prod(r.u0x, wx), two_prod(r.u0y, wy)), fmaf(r.u0x, wxlo, r.u0y * wylo));
    // this warp's next request along with this one when both read the staged layers with an
    // aperture render_pair takes (the uniform test above checked it too)
    const int b2 = b + kRenderWarps;
    if (shared && shifts == nullptr && b2 < Bact) {
      const fdl_request r2 = req[b2];
      const int k1 = pair_class(r), k2 = pair_class(r2);
      if (k1 >= 0 && k1 == k2) {
        const df th2 =
            df_add_f(df_add(two_prod(r2.u0x, wx), two_prod(r2.u0y, wy)), fmaf(r2.u0x, wxlo, r2.u0y * wylo));
        float2 a1[4], a2[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) a1[c] = a2[c] = make_float2(0.f, 0.f);
        if (k1 == 0) render_pair<CC, 0>(r, r2, C, theta, th2, wabs, valid, tile, dsh, lane, a1, a2);
        else render_pair<CC, 1>(r, r2, C, theta, th2, wabs, valid, tile, dsh, lane, a1, a2);
        if (valid) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (c < C) {
              *out.at((long long)b * C + c, ky, kx, M) = a1[c];
              *out.at((long long)b2 * C + c, ky, kx, M) = a2[c];
            }
          }
        }
        b = b2;  // the loop's increment moves on past b2
        continue;
      }
    }
    float2 acc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = make_float2(0.f, 0.f);
    const float2* shb = shifts ? reinterpret_cast<const float2*>(shifts) + (long long)b * r.N : nullptr;
    render_terms<CC>(r, 0, 1, C, theta, wy, wx, wabs, plane, off, valid, shared ? tile : nullptr, dsh, lane, acc, shb,
                     fq);
    if (valid) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c < C) *out.at((long long)b * C + c, ky, kx, M) = acc[c];
    }
  }
}

// two requests read one FDL (the same layer values, disparities and sizes)
__device__ __forceinline__ bool same_fdl(const fdl_request& a, const fdl_request& b) {
  return a.layers == b.layers && a.d == b.d && a.N == b.N && a.H == b.H && a.W == b.W && a.C == b.C;
}

// Fewer than 8 requests (single renders, small batches): each warp takes its own 32 consecutive
// stored bins (lane = bin) and renders every request there, reading the layer values from
// global memory (a layer value is used by at most B < 8 requests: staging it in shared memory
// costs more instructions than it saves), two requests at a time where render_pair applies.
// Setting up a frequency (its coordinates, w as a double-float, u0 . w) is done once per
// request, not once per warp of a layer split.
constexpr int kFewWarps = 4;  // CTAs of 128 threads: a single 512^2 render (1028 CTAs) fits one wave
template <int CC>
__global__ void __launch_bounds__(kFewWarps * 32) k_render_few(const fdl_request* __restrict__ req, int B,
                                                                  const int* __restrict__ count, int C, int H, int W,
                                                                  int nmax, SpecView out,
                                                                  const float* __restrict__ shifts,
                                                                  int* __restrict__ status,
                                                                  const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int M = W >> 1;
  const int Qs = H * (M + 1);
  const long long plane = (long long)H * (M + 1);
  const int Bact = count ? min(*count, B) : B;
  const int q = (blockIdx.x * kFewWarps + warp) * 32 + lane;
  if (Bact <= 0 || q - lane >= Qs) return;  // this warp's 32 bins lie past the image
  const bool valid = q < Qs;
  int ky, kx;
  bin_coords(valid ? q : 0, H, M, ky, kx);
  const Freq fq = bin_freq(ky, kx, H, W);
  const float wabs = sqrtf(fq.wx * fq.wx + fq.wy * fq.wy);
  const long long off = (long long)ky * (M + 1) + kx;
  auto theta_of = [&](const fdl_request& r) {
    return df_add_f(df_add(two_prod(r.u0x, fq.wx), two_prod(r.u0y, fq.wy)), fmaf(r.u0x, fq.wx_lo, r.u0y * fq.wy_lo));
  };
  auto put = [&](int b, const float2* a) {
    if (valid) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c < C) *out.at((long long)b * C + c, ky, kx, M) = a[c];
    }
  };
  for (int b = 0; b < Bact; ++b) {
    if (!request_ok(req[b], C, H, W, nmax, true)) {
      if (blockIdx.x == 0 && warp == 0 && lane == 0) atomicOr(status, FDL_ST_BAD_REQUEST);
      continue;
    }
    const fdl_request r = req[b];
    const df theta = theta_of(r);
    if (shifts == nullptr && b + 1 < Bact) {
      const fdl_request r2 = req[b + 1];
      const int k1 = pair_class(r), k2 = pair_class(r2);
      if (k1 >= 0 && k1 == k2 && same_fdl(r, r2) && request_ok(r2, C, H, W, nmax, true)) {
        float2 a1[4], a2[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) a1[c] = a2[c] = make_float2(0.f, 0.f);
        const df th2 = theta_of(r2);
        if (k1 == 0)
          render_pair<CC, 0, false, 2>(r, r2, C, theta, th2, wabs, valid, nullptr, nullptr, lane, a1, a2, plane, off);
        else
          render_pair<CC, 1, false, 2>(r, r2, C, theta, th2, wabs, valid, nullptr, nullptr, lane, a1, a2, plane, off);
        put(b, a1);
        put(b + 1, a2);
        ++b;
        continue;
      }
    }
    float2 acc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = make_float2(0.f, 0.f);
    const float2* shb = shifts ? reinterpret_cast<const float2*>(shifts) + (long long)b * r.N : nullptr;
    render_terms<CC, 4>(r, 0, 1, C, theta, fq.wy, fq.wx, wabs, plane, off, valid, nullptr, nullptr, lane, acc, shb, fq);
    put(b, acc);
  }
}

// Work-item span (frequencies) of a group of nb requests in the mixed render: 32 (one per lane,
// the layer values staged once for the 8 warps) from 8 requests on, else 256 (one tile of 32
// per warp, the layer values read once per warp for its nb requests).
__host__ __device__ __forceinline__ int grp_span(int nb) { return nb >= kRenderWarps ? 32 : 32 * kRenderWarps; }

// Mixed path, render: work item w of the plan is tile t of group g.  Groups of 8 requests or
// more: the CTA stages the group's layer values of 32 frequencies in shared memory once and the
// warps take the requests (two at a time where render_pair applies).  Smaller groups: each warp
// takes 32 frequencies of a 256-frequency tile and renders every request of the group there,
// reading each layer value once from global memory for all of them.  Request b's spectrum goes
// to its slot in the split layout of its own size (pitch M_b = W_b/2; kx = W_b/2 to
// nyq[(b Cmax + c) Hmax + ky]).  A persistent grid strides over the work items.
template <int CC>
__global__ void __launch_bounds__(kRenderWarps * 32) k_render_grp(const fdl_request* __restrict__ req, int B,
                                                                  int Cmax, int Hmax, const int* __restrict__ plan,
                                                                  float2* __restrict__ slots, long long slot_elems,
                                                                  float2* __restrict__ nyq,
                                                                  const int* __restrict__ gate) {
  extern __shared__ float2 tile[];  // [N C][32]
  __shared__ float dsh[64];
  if (gate != nullptr && *gate != 0) return;
  const int ng = plan[0], total = plan[1];
  const int* gstart = plan + 2;
  const int* gcount = gstart + B;
  const int* gprefix = gcount + B;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    int lo = 0, hi = ng - 1;  // the last group starting at or before w
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (gprefix[mid] <= w) lo = mid;
      else hi = mid - 1;
    }
    const int b0 = gstart[lo], nb = gcount[lo];
    const int t = w - gprefix[lo];
    const bool staged = nb >= kRenderWarps;
    const fdl_request r0 = req[b0];
    const int H = r0.H, W = r0.W, C = r0.C, N = r0.N, M = W >> 1;
    const int Qs = H * (M + 1);
    const int q = t * grp_span(nb) + (staged ? 0 : 32 * warp) + lane;
    const bool valid = q < Qs;
    int ky, kx;
    bin_coords(valid ? q : 0, H, M, ky, kx);
    const Freq fq = bin_freq(ky, kx, H, W);
    const float wy = fq.wy, wx = fq.wx;
    const float wabs = sqrtf(wx * wx + wy * wy);
    const long long plane = (long long)H * (M + 1);
    const long long off = (long long)ky * (M + 1) + kx;
    auto put = [&](int b, const float2* a) {
      float2* sl = slots + (long long)b * slot_elems;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c < C) {
          if (kx < M) sl[((long long)c * H + ky) * M + kx] = a[c];
          else nyq[((long long)b * Cmax + c) * Hmax + ky] = a[c];
        }
      }
    };
    auto theta_of = [&](const fdl_request& r) {
      return df_add_f(df_add(two_prod(r.u0x, wx), two_prod(r.u0y, wy)), fmaf(r.u0x, fq.wx_lo, r.u0y * fq.wy_lo));
    };
    if (staged) {
      __syncthreads();  // the previous staged work item's reads of tile and dsh are done
      stage_async(tile, reinterpret_cast<const float2*>(r0.layers), N * C, plane, off, valid);
      cp_async_commit();
      for (int k = threadIdx.x; k < N; k += blockDim.x) dsh[k] = __ldg(r0.d + k);
      cp_async_wait<0>();
      __syncthreads();
    } else if (q - lane >= Qs) {
      continue;  // this warp's 32 frequencies lie past the image
    }
    // requests bi = first, first + step, ...: the warps over the requests (staged), or every
    // request in each warp
    const int first = staged ? warp : 0, step = staged ? kRenderWarps : 1;
    for (int bi = first; bi < nb; bi += step) {
      const fdl_request r = req[b0 + bi];
      const df theta = theta_of(r);
      const int bi2 = bi + step;
      if (bi2 < nb) {
        const fdl_request r2 = req[b0 + bi2];
        const int k1 = pair_class(r), k2 = pair_class(r2);
        if (k1 >= 0 && k1 == k2) {
          float2 a1[4], a2[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) a1[c] = a2[c] = make_float2(0.f, 0.f);
          const df th2 = theta_of(r2);
          if (staged) {
            if (k1 == 0) render_pair<CC, 0, true>(r, r2, C, theta, th2, wabs, valid, tile, dsh, lane, a1, a2);
            else render_pair<CC, 1, true>(r, r2, C, theta, th2, wabs, valid, tile, dsh, lane, a1, a2);
          } else {
            if (k1 == 0)
              render_pair<CC, 0, false>(r, r2, C, theta, th2, wabs, valid, nullptr, nullptr, lane, a1, a2, plane, off);
            else
              render_pair<CC, 1, false>(r, r2, C, theta, th2, wabs, valid, nullptr, nullptr, lane, a1, a2, plane, off);
          }
          if (valid) {
            put(b0 + bi, a1);
            put(b0 + bi2, a2);
          }
          bi = bi2;
          continue;
        }
      }
      float2 acc[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c] = make_float2(0.f, 0.f);
      render_terms<CC>(r, 0, 1, C, theta, wy, wx, wabs, plane, off, valid, staged ? tile : nullptr, dsh, lane, acc,
                       nullptr, fq);
      if (valid) put(b0 + bi, acc);
    }
  }
}


// *gate = 1 when every active request passes request_ok with exactly (C, H, W) and reads the
// same FDL (layers, d, N) as request 0 (the tiled path), else 0.  plan = [ngroups, tiles,
// gstart[B], gcount[B], gprefix[B + 1]]: the groups of the mixed path, runs of consecutive
// valid requests of one FDL (same layers, d, N and size), group g covering work items
// [gprefix[g], gprefix[g + 1]), one per tile of grp_span(gcount[g]) of its H (W/2 + 1)
// frequencies.
__global__ void __launch_bounds__(256) k_render_plan(const fdl_request* __restrict__ req, int B,
                                                     const int* __restrict__ count, int C, int H, int W, int Nmax,
                                                     int* __restrict__ gate, int* __restrict__ plan) {
  __shared__ int ok;
  int* gstart = plan + 2;
  int* gcount = gstart + B;
  int* gprefix = gcount + B;
  if (threadIdx.x == 0) ok = 1;
  for (int i = threadIdx.x; i < B; i += blockDim.x) gcount[i] = 0;
  __syncthreads();
  const int Bact = count ? min(*count, B) : B;
  for (int b = threadIdx.x; b < Bact; b += blockDim.x) {
    const fdl_request& r = req[b];
    if (!request_ok(r, C, H, W, Nmax, true) || r.layers != req[0].layers || r.d != req[0].d || r.N != req[0].N)
      ok = 0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    // group ids by a ballot over chunks of 32 requests: a valid request starts a group unless
    // the request before it is valid and reads the same FDL
    int ng = 0;
    for (int i0 = 0; i0 < Bact; i0 += 32) {
      const int i = i0 + lane;
      bool v = false, st = false;
      if (i < Bact) {
        v = request_ok(req[i], C, H, W, Nmax, false);
        st = v && !(i > 0 && request_ok(req[i - 1], C, H, W, Nmax, false) && same_fdl(req[i - 1], req[i]));
      }
      const unsigned starts = __ballot_sync(0xffffffffu, st);
      const int gid = ng + __popc(starts & (0xffffffffu >> (31 - lane))) - 1;
      if (st) gstart[gid] = i;
      if (v) atomicAdd(gcount + gid, 1);
      ng += __popc(starts);
    }
    __syncwarp();
    // work items: an exclusive scan of the groups' tile counts
    int acc = 0;
    for (int g0 = 0; g0 < ng; g0 += 32) {
      const int g = g0 + lane;
      int t = 0;
      if (g < ng) {
        const fdl_request& r = req[gstart[g]];
        const int span = grp_span(gcount[g]);
        t = (r.H * (r.W / 2 + 1) + span - 1) / span;
      }
      int x = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (g < ng) gprefix[g] = acc + x - t;
      acc += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) {
      gprefix[ng] = acc;
      plan[0] = ng;
      plan[1] = acc;
    }
  }
  if (threadIdx.x == 0) *gate = ok;
}

__global__ void k_pinhole_requests(fdl_request* req, const float* layers, const float* d, int N, int C, int H,
                                   int W, const float* u0, int B, float* out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  fdl_request r;
  r.layers = layers;
  r.d = d;
  r.out = out + (long long)b * C * H * W;
  r.H = H;
  r.W = W;
  r.C = C;
  r.pad_[0] = r.pad_[1] = 0;
  r.pts = nullptr;
  r.N = N;
  r.npts = 0;
  r.aperture = FDL_AP_PINHOLE;
  r.u0x = u0 ? u0[2 * b] : 0.f;  // null: shifts given per layer instead
  r.u0y = u0 ? u0[2 * b + 1] : 0.f;
  r.s = 0.f;
  r.radius = 0.f;
  req[b] = r;
}

// centred zero-padded raster: pad[iy'][ix'] = R[(iy' + c) mod Z][(ix' + c) mod Z] when that
// pixel exists (P <= Z, so each padded entry has at most one source)
__global__ void k_place_raster(const float* __restrict__ R, int P, int Z, float* __restrict__ pad) {
  const long long n = (long long)Z * Z;
  const int c = (P - 1) / 2;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int iyp = (int)(e / Z), ixp = (int)(e - (long long)iyp * Z);
    int iy = iyp + c, ix = ixp + c;
    iy = iy >= Z ? iy - Z : iy;
    ix = ix >= Z ? ix - Z : ix;
    pad[e] = (iy < P && ix < P) ? R[iy * P + ix] : 0.f;
  }
}

// sum of the raster in double, one CTA, fixed order: deterministic
__global__ void k_raster_sum(const float* __restrict__ R, int n, double* __restrict__ out) {
  __shared__ double part[256];
  double s = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) s += (double)R[e];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = part[0];
}

__global__ void k_scale_table(float2* __restrict__ T, long long n, const double* __restrict__ sum) {
  const double s = sum[0];
  const float inv = s > 0.0 ? (float)(1.0 / s) : 0.f;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    T[e] = make_float2(T[e].x * inv, T[e].y * inv);
}

// ------------------------------------------------------------ mixed power-of-two path
// Requests of different FDLs and power-of-two sizes in one launch: k_render_grp writes each
// request's rendered half spectrum into its slot (split layout of its own size); a CTA of
// k_cols_req then takes a strip of SW columns of one request (all H rows) into shared memory,
// runs the inverse DFT along y there and writes the strip back in place; k_irfft_rows_req
// finishes the rows.  Every CTA reads its request's sizes from the descriptor (grids sized
// for the largest).
constexpr int kRcThreads = 256;
constexpr int kRcFreqs = 2048;  // H * SW of a CTA's strip (the strip of one column when H > 2048 is not used)
constexpr int kRcMaxH = 2048;

// columns per strip for an image of H rows and M = W/2 stored columns below the Nyquist one
__host__ __device__ __forceinline__ int rc_strip(int H, int M) {
  int sw = kRcFreqs / H;
  if (sw < 1) sw = 1;
  if (sw > M) sw = M;
  return sw;
}

__device__ __forceinline__ int log2_pow2(int v) { return 31 - __clz(v); }

// FIRST: column 0 and the Nyquist column kx = W/2 of every request (from nyq), packed as
// Herm(F0) + i Herm(FN) before the inverse DFT (the split layout's element 0 of each row);
// otherwise strip blockIdx.y of SW columns (column 0 of strip 0 is left to the FIRST launch,
// which runs after this one).  Request b = blockIdx.x.
template <bool FIRST>
__global__ void __launch_bounds__(kRcThreads) k_cols_req(const fdl_request* __restrict__ req,
                                                         const int* __restrict__ count, int Cmax, int Hmax, int Wmax,
                                                         int Nmax, float2* __restrict__ slots, long long slot_elems,
                                                         const float2* __restrict__ nyqp, int* __restrict__ status,
                                                         const int* __restrict__ gate) {
  extern __shared__ float2 sm[];
  const int b = blockIdx.x;
  if (gate != nullptr && *gate != 0) return;
  if (count != nullptr && b >= *count) return;
  const fdl_request r = req[b];
  if (!request_ok(r, Cmax, Hmax, Wmax, Nmax, false)) {
    if (FIRST && threadIdx.x == 0) atomicOr(status, FDL_ST_BAD_REQUEST);
    return;
  }
  const int H = r.H, W = r.W, C = r.C, M = W >> 1;
  const int SW = FIRST ? 1 : rc_strip(H, M);
  const int c0 = FIRST ? 0 : (int)blockIdx.y * SW;
  if (c0 >= M) return;
  const int logH = log2_pow2(H), logSW = log2_pow2(SW);
  const int HS = H * SW;
  float2* tw = sm;           // [H]
  float2* data = sm + Hmax;  // [C][H][SW]
  float2* nyq = data + (long long)Cmax * Hmax;  // FIRST: [C][H], the Nyquist column
  make_twiddles(tw, H);
  float2* slot = slots + (long long)b * slot_elems;
  const int nf = FIRST ? 2 * H : HS;
  for (int f = threadIdx.x; f < nf; f += blockDim.x) {
    if (FIRST) {
      const int ky = f < H ? f : f - H;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c < C) {
          if (f < H) data[c * H + ky] = slot[((long long)c * H + ky) * M];
          else nyq[c * H + ky] = nyqp[((long long)b * Cmax + c) * Hmax + ky];
        }
      }
    } else {
      const int ky = f >> logSW, kx = c0 + (f & (SW - 1));
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c < C) data[c * HS + f] = slot[((long long)c * H + ky) * M + kx];
    }
  }
  __syncthreads();
  if (FIRST) {
    // column 0 <- Herm(F0) + i Herm(FN), Herm(F)[ky] = (F[ky] + conj F[-ky]) / 2
    for (int c = 0; c < C; ++c) {
      constexpr int kRows = kRcMaxH / kRcThreads;
      float2 pk[kRows];
#pragma unroll
      for (int i = 0; i < kRows; ++i) {
        const int ky = threadIdx.x + i * kRcThreads;
        if (ky < H) {
          const int km = (H - ky) & (H - 1);
          const float2 f0 = data[c * H + ky], f0m = data[c * H + km];
          const float2 fn = nyq[c * H + ky], fnm = nyq[c * H + km];
          const float2 h0 = make_float2(0.5f * (f0.x + f0m.x), 0.5f * (f0.y - f0m.y));
          const float2 hn = make_float2(0.5f * (fn.x + fnm.x), 0.5f * (fn.y - fnm.y));
          pk[i] = make_float2(h0.x - hn.y, h0.y + hn.x);
        }
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < kRows; ++i) {
        const int ky = threadIdx.x + i * kRcThreads;
        if (ky < H) data[c * H + ky] = pk[i];
      }
      __syncthreads();
    }
  }
  for (int c = 0; c < C; ++c) stockham<true, 2>(data + c * HS, tw, H, logH, SW, logSW, 1, SW);
  for (int f = threadIdx.x; f < HS; f += blockDim.x) {
    const int ky = f >> logSW, kx = c0 + (f & (SW - 1));
    if (!FIRST && kx == 0) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c < C) slot[((long long)c * H + ky) * M + kx] = data[c * HS + f];
  }
}

// Inverse row DFT of the mixed path: rows of request b's slot (pitch M = W_b/2, element 0
// packing X[0] + i X[W/2]) -> the request's output, times 1 / (H W).  A CTA takes
// kRcFreqs / M consecutive rows of one request.
__global__ void __launch_bounds__(kRcThreads) k_irfft_rows_req(const fdl_request* __restrict__ req,
                                                               const int* __restrict__ count, int Cmax, int Hmax,
                                                               int Wmax, int Nmax, const float2* __restrict__ slots,
                                                               long long slot_elems, const int* __restrict__ gate) {
  extern __shared__ float2 sm[];
  const int b = blockIdx.y;
  if (gate != nullptr && *gate != 0) return;
  if (count != nullptr && b >= *count) return;
  const fdl_request r = req[b];
  if (!request_ok(r, Cmax, Hmax, Wmax, Nmax, false)) return;
  const int H = r.H, W = r.W, C = r.C, M = W >> 1, logM = log2_pow2(M);
  const int R = kRcFreqs / M;  // M <= 2048
  const long long nrows = (long long)C * H;
  const long long row0 = (long long)blockIdx.x * R;
  if (row0 >= nrows) return;
  float2* tw = sm;
  float2* data = sm + (Wmax >> 1);
  make_twiddles(tw, M);
  float2 h;  // exp(i pi / M)
  sincospif(1.f / (float)M, &h.y, &h.x);
  const float2* in = slots + (long long)b * slot_elems;
  for (int e = threadIdx.x; e < R * M; e += blockDim.x) {
    const int rr = e >> logM;
    data[e] = row0 + rr < nrows ? in[(row0 + rr) * M + (e & (M - 1))] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  // Z[k] = E[k] + i O[k], E[k] = X[k] + conj X[M-k],
  // O[k] = (X[k] - conj X[M-k]) exp(+2 pi i k / W); X[0], X[M] are packed in element 0.
  constexpr int kPer = kRcFreqs / kRcThreads;  // R * M = kRcFreqs elements, kPer per thread
  float2 zk[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int e = threadIdx.x + i * kRcThreads;
    const int rr = e >> logM, k = e & (M - 1);
    const float2* X = data + rr * M;
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
  for (int i = 0; i < kPer; ++i) data[threadIdx.x + i * kRcThreads] = zk[i];
  __syncthreads();
  stockham<true, 2>(data, tw, M, logM, R, log2_pow2(R), M, 1);
  const float scale = 1.f / ((float)H * (float)W);
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
    reinterpret_cast<float4*>(r.out + row * W)[e & ((W >> 2) - 1)] = v;
  }
}

}  // namespace

cudaError_t launch_aperture_table_prep(const float* R, int P, int Z, float* pad, double* sum, cudaStream_t st) {
  const long long n = (long long)Z * Z;
  k_place_raster<<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, st>>>(R, P, Z, pad);
  k_raster_sum<<<1, 256, 0, st>>>(R, P * P, sum);
  return cudaGetLastError();
}

cudaError_t launch_aperture_table_scale(float2* T, int Z, const double* sum, cudaStream_t st) {
  const long long n = (long long)Z * (Z / 2 + 1);
  k_scale_table<<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, st>>>(T, n, sum);
  return cudaGetLastError();
}

size_t render_plan_ints(int B) { return 3 * (size_t)B + 3; }

cudaError_t launch_render_plan(const fdl_request* req, int B, const int* count, int C, int H, int W, int Nmax,
                               int* gate, int* plan, cudaStream_t st) {
  k_render_plan<<<1, 256, 0, st>>>(req, B, count, C, H, W, Nmax, gate, plan);
  return cudaGetLastError();
}

cudaError_t launch_render_spectra(const fdl_request* req, int B, const int* count, int C, int H, int W, int Nmax,
                                  SpecView out, int* status, cudaStream_t st, const float* shifts, const int* gate) {
  const int Qs = H * (W / 2 + 1);
  const int tile_lc = min(Nmax * C, kTileMaxLC);
  const size_t smem = (size_t)tile_lc * 32 * sizeof(float2);
  const int ntiles = (Qs + 31) / 32;
  cudaError_t e = cudaSuccess;
  // the channel loop unrolled for one and three channels, predicated up to four otherwise;
  // fewer than 8 requests: k_render_few, a warp per 32 bins
#define FDL_RENDER(CC)                                                                                         \
  if (B < kRenderWarps) {                                                                                      \
    k_render_few<CC><<<(ntiles + kFewWarps - 1) / kFewWarps, kFewWarps * 32, 0, st>>>(req, B, count, C, H, W,  \
                                                                                      Nmax, out, shifts,       \
                                                                                      status, gate);           \
  } else {                                                                                                     \
    e = set_smem((const void*)k_render<CC>, (size_t)kTileMaxLC * 32 * sizeof(float2));                        \
    if (e != cudaSuccess) return e;                                                                            \
    k_render<CC><<<ntiles, kRenderWarps * 32, smem, st>>>(req, B, count, C, H, W, tile_lc, Nmax, out, shifts,  \
                                                          status, gate);                                       \
  }
  if (C == 1) FDL_RENDER(1)
  else if (C == 3) FDL_RENDER(3)
  else FDL_RENDER(4)
#undef FDL_RENDER
  return cudaGetLastError();
}

cudaError_t launch_pinhole_requests(fdl_request* req, const float* layers, const float* d, int N, int C, int H,
                                    int W, const float* u0, int B, float* out, cudaStream_t st) {
  k_pinhole_requests<<<(B + 127) / 128, 128, 0, st>>>(req, layers, d, N, C, H, W, u0, B, out);
  return cudaGetLastError();
}

bool render_mixed_supported(int H, int W) {
  auto p2 = [](int v) { return v >= 16 && (v & (v - 1)) == 0; };
  return p2(H) && p2(W) && H <= kRcMaxH && W <= 4096;
}

size_t render_mixed_slot_elems(int C, int H, int W) { return (size_t)C * H * (W / 2); }

cudaError_t launch_render_mixed(const fdl_request* req, int B, const int* count, int C, int H, int W, int Nmax,
                                float2* slots, float2* nyq, const int* plan, int* status, cudaStream_t st,
                                const int* gate) {
  if (!render_mixed_supported(H, W) || B < 1 || B > 65535 || Nmax < 1 || Nmax > 64 || C < 1 || C > 4)
    return cudaErrorInvalidValue;
  const long long se = (long long)render_mixed_slot_elems(C, H, W);
  const int M = W / 2;
  // render: a persistent grid over the plan's work items (at most B tiles of the largest size)
  const long long items = (long long)B * (((long long)H * (M + 1) + 31) / 32);
  const int grid_r = (int)std::min<long long>(items, (long long)num_sms() * 12);
  const size_t smem_r = (size_t)Nmax * C * 32 * sizeof(float2);
  // inverse column pass: a request within (C, H, W) has at most as many strips and row blocks
  // as one of that size
  const int strips = M / rc_strip(H, M);
  const long long row_blocks = ((long long)C * H * M + kRcFreqs - 1) / kRcFreqs;
  const size_t smem_main = (size_t)(H + (size_t)C * (H > kRcFreqs ? H : kRcFreqs)) * sizeof(float2);
  const size_t smem_first = (size_t)(H + 2 * (size_t)C * H) * sizeof(float2);
  const size_t smem_rows = (size_t)(M + kRcFreqs) * sizeof(float2);
  cudaError_t e = set_smem((const void*)k_render_grp<4>, smem_r);
  if (e == cudaSuccess) e = set_smem((const void*)k_cols_req<false>, smem_main);
  if (e == cudaSuccess) e = set_smem((const void*)k_cols_req<true>, smem_first);
  if (e == cudaSuccess) e = set_smem((const void*)k_irfft_rows_req, smem_rows);
  if (e != cudaSuccess) return e;
  k_render_grp<4><<<grid_r, kRenderWarps * 32, smem_r, st>>>(req, B, C, H, plan, slots, se, nyq, gate);
  k_cols_req<false><<<dim3(B, strips), kRcThreads, smem_main, st>>>(req, count, C, H, W, Nmax, slots, se, nyq, status,
                                                                    gate);
  k_cols_req<true><<<dim3(B, 1), kRcThreads, smem_first, st>>>(req, count, C, H, W, Nmax, slots, se, nyq, status, gate);
  k_irfft_rows_req<<<dim3((unsigned)row_blocks, B), kRcThreads, smem_rows, st>>>(req, count, C, H, W, Nmax, slots,
                                                                                 se, gate);
  return cudaGetLastError();
}

}  // namespace fdl
