// Radix-4/2 Stockham FFTs of power-of-two lengths run by a whole CTA on data
// staged in shared memory (shared by the DFT kernels of fft.cu and the fused
// render + inverse column pass of render.cu).
#pragma once

#include "common.cuh"

namespace fdl {

// tw[t] = exp(-2 pi i t / L)
__device__ __forceinline__ void make_twiddles(float2* tw, int L) {
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    float s, c;
    sincospif(-2.0f * (float)t / (float)L, &s, &c);
    tw[t] = make_float2(c, s);
  }
}

// exp(+i pi k / M), 0 <= k < M, from tw[t] = exp(-2 pi i t / M): conj(tw[k / 2]), times
// h = exp(i pi / M) for odd k (the twiddle of the real-to-complex split of a length-2M DFT)
__device__ __forceinline__ float2 half_twiddle_conj(const float2* tw, int k, float2 h) {
  const float2 t = tw[k >> 1];
  const float2 c = make_float2(t.x, -t.y);
  return (k & 1) ? make_float2(c.x * h.x - c.y * h.y, c.x * h.y + c.y * h.x) : c;
}

template <bool INV>
__device__ __forceinline__ float2 twid(const float2* tw, int i) {
  float2 w = tw[i];
  if (INV) w.y = -w.y;
  return w;
}

template <bool INV>
__device__ __forceinline__ void radix4(float2& a0, float2& a1, float2& a2, float2& a3) {
  float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = csub(a1, a3);
  t3 = INV ? make_float2(-t3.y, t3.x) : make_float2(t3.y, -t3.x);  // times +i / -i
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

// In-place DFTs of `nfft` sequences of length L = 2^logL held in shared
// memory at s[f * fstride + n * estride].  All threads of the CTA must call
// it; each handles at most MAXB radix-4 butterflies per pass.
template <bool INV, int MAXB>
__device__ __forceinline__ void stockham(float2* s, const float2* tw, int L, int logL, int nfft,
                                         int lognfft, int fstride, int estride) {
  const int q = L >> 2;
  const int logq = logL - 2;
  const int total = nfft * q;
  const bool fmajor = (fstride == 1);
  int Ns = 1, logNs = 0;
  for (int pass = 0; pass < (logL >> 1); ++pass) {
    float2 v[MAXB][4];
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
        float2* p = s + f * fstride;
        const int k = j & (Ns - 1);
        float2 a0 = p[j * estride], a1 = p[(j + q) * estride];
        float2 a2 = p[(j + 2 * q) * estride], a3 = p[(j + 3 * q) * estride];
        if (pass > 0) {
          const int step = k << (logq - logNs);  // k * L / (4 Ns)
          a1 = cmul(a1, twid<INV>(tw, step));
          a2 = cmul(a2, twid<INV>(tw, 2 * step));
          a3 = cmul(a3, twid<INV>(tw, 3 * step));
        }
        radix4<INV>(a0, a1, a2, a3);
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
        s[ob[b]] = v[b][0];
        s[ob[b] + e] = v[b][1];
        s[ob[b] + 2 * e] = v[b][2];
        s[ob[b] + 3 * e] = v[b][3];
      }
    }
    __syncthreads();
    Ns <<= 2;
    logNs += 2;
  }
  if (logL & 1) {
    // last pass, radix 2 with Ns = L/2: reads and writes the same two slots.
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
        float2* p = s + f * fstride;
        float2 a0 = p[j * estride];
        float2 a1 = cmul(p[(j + h) * estride], twid<INV>(tw, j));
        p[j * estride] = cadd(a0, a1);
        p[(j + h) * estride] = csub(a0, a1);
      }
    }
    __syncthreads();
  }
}

}  // namespace fdl
