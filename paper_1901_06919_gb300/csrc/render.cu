// Rendering of Sec. VI-A: the spectrum of the image seen from u0 with
// aperture psi focused at disparity s (Eq. BsFourier),
//   B_hat(w) = sum_k exp(+2 pi i d_k (u0 . w)) psi_hat((s - d_k) w) L_hat^k(w),
// written per request into the split half-spectrum layout, ready for the
// inverse column and row DFT passes.  psi is normalised to integrate to 1,
// so psi_hat(0) = 1 and a pinhole (psi = delta) gives psi_hat = 1 (Sec. IV-B).
#include "hp_solve.cuh"

namespace fdl {

namespace {

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
  const float sx = 2.f * radius * nux, sy = 2.f * radius * nuy;
  const float fx = sx == 0.f ? 1.f : sinpif(sx) / (3.14159265358979f * sx);
  const float fy = sy == 0.f ? 1.f : sinpif(sy) / (3.14159265358979f * sy);
  return make_float2(fx * fy, 0.f);
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

// sum over layers k = k0, k0 + kstep, ... < r.N of the Eq. BsFourier terms of request r at
// this lane's frequency; layer values from the shared tile (TILE) or from global memory;
// SHIFTS: the request's per-layer shifts P_k in shb (the relaxed model), else u0 d_k.
// AP: 0 no aperture factor (pinhole, or a disc of radius 0), 1 disc, 2 drawn (table),
// 3 square or points.
template <bool TILE, bool SHIFTS, int AP>
__device__ __forceinline__ void render_terms_t(const fdl_request& r, int k0, int kstep, int C, df theta, float wy,
                                               float wx, float wabs, long long plane, long long off, bool valid,
                                               const float2* tile, const float* dsh, int lane, float2 acc[4],
                                               const float2* __restrict__ shb, const Freq& fq) {
  const float2* x = reinterpret_cast<const float2*>(r.layers);
  const float zscale = 6.283185307f * r.radius * wabs;  // 2 pi r |w|
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
      for (int c = 0; c < 4; ++c)
        if (c < C) cfma(acc[c], coef, TILE ? tile[(k * C + c) * 32 + lane] : __ldg(x + ((long long)k * C + c) * plane + off));
    }
  }
}

template <bool TILE, bool SHIFTS>
__device__ __forceinline__ void render_terms_ap(const fdl_request& r, int k0, int kstep, int C, df theta, float wy,
                                                float wx, float wabs, long long plane, long long off, bool valid,
                                                const float2* tile, const float* dsh, int lane, float2 acc[4],
                                                const float2* __restrict__ shb, const Freq& fq) {
  const int ap = (r.aperture == FDL_AP_PINHOLE || (r.aperture == FDL_AP_DISC && r.radius == 0.f)) ? 0
                 : r.aperture == FDL_AP_DISC                                                  ? 1
                 : r.aperture == FDL_AP_TABLE                                                 ? 2
                                                                                              : 3;
#define FDL_TERMS(A) \
  render_terms_t<TILE, SHIFTS, A>(r, k0, kstep, C, theta, wy, wx, wabs, plane, off, valid, tile, dsh, lane, acc, shb, fq)
  if (ap == 0) FDL_TERMS(0);
  else if (ap == 1) FDL_TERMS(1);
  else if (ap == 2) FDL_TERMS(2);
  else FDL_TERMS(3);
#undef FDL_TERMS
}

// the request's terms with the loop specialised for where the layers live, the shift model
// and the aperture kind (all uniform over the request)
__device__ __forceinline__ void render_terms(const fdl_request& r, int k0, int kstep, int C, df theta, float wy,
                                             float wx, float wabs, long long plane, long long off, bool valid,
                                             const float2* tile, const float* dsh, int lane, float2 acc[4],
                                             const float2* __restrict__ shb, const Freq& fq) {
  if (tile != nullptr) {
    if (shb != nullptr)
      render_terms_ap<true, true>(r, k0, kstep, C, theta, wy, wx, wabs, plane, off, valid, tile, dsh, lane, acc, shb, fq);
    else
      render_terms_ap<true, false>(r, k0, kstep, C, theta, wy, wx, wabs, plane, off, valid, tile, dsh, lane, acc, shb, fq);
  } else {
    if (shb != nullptr)
      render_terms_ap<false, true>(r, k0, kstep, C, theta, wy, wx, wabs, plane, off, valid, tile, dsh, lane, acc, shb, fq);
    else
      render_terms_ap<false, false>(r, k0, kstep, C, theta, wy, wx, wabs, plane, off, valid, tile, dsh, lane, acc, shb, fq);
  }
}

// CTA: 32 consecutive stored bins (lane = bin) x 8 warps.
//  * B >= 8 requests: warp w renders requests w, w + 8, ...; when every request reads
//    the same FDL (and N*C <= tile_lc) the CTA first stages that FDL's layer values for
//    its 32 bins in shared memory and all requests read them there.
//  * B < 8 (single renders, small batches): the 8 / B warps given to a request split its
//    layers and their partial sums are added through shared memory, so that one request
//    still occupies the whole CTA.
__global__ void __launch_bounds__(kRenderWarps * 32) k_render(const fdl_request* __restrict__ req, int B,
                                                              const int* __restrict__ count, int C, int H, int W,
                                                              int tile_lc, SpecView out, const float* __restrict__ shifts) {
  extern __shared__ float2 tile[];  // [tile_lc][32]
  __shared__ float dsh[64];
  __shared__ float2 part[kRenderWarps][4][32];
  __shared__ int uniform;
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
    if (b < Bact) {
      const fdl_request r = req[b];
      const df theta = df_add_f(df_add(two_prod(r.u0x, wx), two_prod(r.u0y, wy)), fmaf(r.u0x, wxlo, r.u0y * wylo));
      const float2* shb = shifts ? reinterpret_cast<const float2*>(shifts) + (long long)b * r.N : nullptr;
      render_terms(r, sl, G, C, theta, wy, wx, wabs, plane, off, valid, nullptr, nullptr, lane, acc, shb, fq);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) part[warp][c][lane] = acc[c];
    __syncthreads();
    if (b < Bact && sl == 0 && valid) {
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
    if (req[b].layers != L0 || req[b].d != req[0].d) uniform = 0;
  __syncthreads();
  const bool shared = uniform && N0 * C <= tile_lc && N0 <= 64;
  if (shared) {
    const float2* x0 = reinterpret_cast<const float2*>(L0);
    for (int e = threadIdx.x; e < N0 * C * 32; e += blockDim.x) {
      const int lc = e >> 5, l2 = e & 31;
      const int qq = blockIdx.x * 32 + l2;
      float2 v = make_float2(0.f, 0.f);
      if (qq < Qs) {
        int yy, xx;
        bin_coords(qq, H, M, yy, xx);
        v = __ldg(x0 + (long long)lc * plane + (long long)yy * (M + 1) + xx);
      }
      tile[e] = v;
    }
    for (int k = threadIdx.x; k < N0; k += blockDim.x) dsh[k] = __ldg(req[0].d + k);
    __syncthreads();
  }
  for (int b = warp; b < Bact; b += kRenderWarps) {
    const fdl_request r = req[b];
    const df theta = df_add_f(df_add(two_prod(r.u0x, wx), two_prod(r.u0y, wy)), fmaf(r.u0x, wxlo, r.u0y * wylo));
    float2 acc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = make_float2(0.f, 0.f);
    const float2* shb = shifts ? reinterpret_cast<const float2*>(shifts) + (long long)b * r.N : nullptr;
    render_terms(r, 0, 1, C, theta, wy, wx, wabs, plane, off, valid, shared ? tile : nullptr, dsh, lane, acc, shb,
                 fq);
    if (valid) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c < C) *out.at((long long)b * C + c, ky, kx, M) = acc[c];
    }
  }
}

__global__ void k_pinhole_requests(fdl_request* req, const float* layers, const float* d, int N,
                                   const float* u0, int B, float* out, long long img_elems) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  fdl_request r;
  r.layers = layers;
  r.d = d;
  r.out = out + (long long)b * img_elems;
  r.pts = nullptr;
  r.N = N;
  r.npts = 0;
  r.aperture = FDL_AP_PINHOLE;
  r.u0x = u0 ? u0[2 * b] : 0.f;  // null: shifts given per layer instead
  r.u0y = u0 ? u0[2 * b + 1] : 0.f;
  r.s = 0.f;
  r.radius = 0.f;
  r.pad_ = 0;
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

cudaError_t launch_render_spectra(const fdl_request* req, int B, const int* count, int C, int H, int W, int Nmax,
                                  SpecView out, cudaStream_t st, const float* shifts) {
  const int Qs = H * (W / 2 + 1);
  const int tile_lc = min(Nmax * C, kTileMaxLC);
  const size_t smem = (size_t)tile_lc * 32 * sizeof(float2);
  cudaError_t e = set_smem((const void*)k_render, (size_t)kTileMaxLC * 32 * sizeof(float2));
  if (e != cudaSuccess) return e;
  k_render<<<(Qs + 31) / 32, kRenderWarps * 32, smem, st>>>(req, B, count, C, H, W, tile_lc, out, shifts);
  return cudaGetLastError();
}

cudaError_t launch_pinhole_requests(fdl_request* req, const float* layers, const float* d, int N,
                                    const float* u0, int B, float* out, long long img_elems, cudaStream_t st) {
  k_pinhole_requests<<<(B + 127) / 128, 128, 0, st>>>(req, layers, d, N, u0, B, out, img_elems);
  return cudaGetLastError();
}

}  // namespace fdl
