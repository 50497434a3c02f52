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
      const float f = phase_cycles(pm.x, pm.y, nux, nuy, -1.f);
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

// CTA: 32 consecutive stored bins (lane = bin) x 8 warps; warp w renders
// requests w, w + 8 gridDim.y, ...
__global__ void __launch_bounds__(256) k_render(const fdl_request* __restrict__ req, int B,
                                                const int* __restrict__ count, int C, int H, int W,
                                                SpecView out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int M = W >> 1;
  const int Qs = H * (M + 1);
  const int q = blockIdx.x * 32 + lane;
  const bool valid = q < Qs;
  int ky, kx;
  bin_coords(valid ? q : 0, H, M, ky, kx);
  const float wy = freq_y(ky, H);
  const float wx = (float)kx / (float)W;
  const long long plane = (long long)H * (M + 1);
  const long long off = (long long)ky * (M + 1) + kx;
  const int Bact = count ? min(*count, B) : B;
  for (int b = blockIdx.y * 8 + warp; b < Bact; b += gridDim.y * 8) {
    const fdl_request r = req[b];
    const float2* x = reinterpret_cast<const float2*>(r.layers);
    float2 acc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = make_float2(0.f, 0.f);
    for (int k = 0; k < r.N; ++k) {
      const float dk = __ldg(r.d + k);
      const float f = phase_cycles(r.u0x, r.u0y, wx, wy, dk);
      float2 sh;
      sincospif(2.f * f, &sh.y, &sh.x);
      const float sd = r.s - dk;
      const float2 coef = cmul(sh, aperture_hat(r.aperture, r.radius, r.pts, r.npts, sd * wy, sd * wx));
      if (valid) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (c < C) cfma(acc[c], coef, __ldg(x + ((long long)k * C + c) * plane + off));
      }
    }
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
  r.u0x = u0[2 * b];
  r.u0y = u0[2 * b + 1];
  r.s = 0.f;
  r.radius = 0.f;
  r.pad_ = 0;
  req[b] = r;
}

}  // namespace

cudaError_t launch_render_spectra(const fdl_request* req, int B, const int* count, int C, int H, int W,
                                  SpecView out, cudaStream_t st) {
  const int Qs = H * (W / 2 + 1);
  dim3 grid((Qs + 31) / 32, (B + 7) / 8);
  if (grid.y > 65535) grid.y = 65535;
  k_render<<<grid, 256, 0, st>>>(req, B, count, C, H, W, out);
  return cudaGetLastError();
}

cudaError_t launch_pinhole_requests(fdl_request* req, const float* layers, const float* d, int N,
                                    const float* u0, int B, float* out, long long img_elems, cudaStream_t st) {
  k_pinhole_requests<<<(B + 127) / 128, 128, 0, st>>>(req, layers, d, N, u0, B, out, img_elems);
  return cudaGetLastError();
}

}  // namespace fdl
