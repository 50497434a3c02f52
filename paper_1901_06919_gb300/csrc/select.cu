// Choice of the frequencies re-solved in the next precision tier
// (FP32 -> double-float, double-float -> native FP64).
//
// A solve pass records, per frequency q, an error scale e_q = kappa_q |x_q|
// (condition estimate times solution norm; 0 for frequencies solved
// elsewhere, +inf where its result is not trusted) and |x_q|^2.  With u the
// error of that pass per unit of e_q, the estimated error of the layers is
// sqrt(sum (u e_q)^2).  These kernels pick the smallest set of largest e_q
// whose removal brings the estimate of the rest under budget * |X|:
//   k_err_hist     histogram of log2 e_q: count and sum of e_q^2 per bucket;
//   k_err_thresh   a prefix sum over the buckets gives the cut;
//   k_err_compact  appends every frequency at or above the threshold.
#include "kernels.h"

namespace fdl {

namespace {

// eight buckets per octave: bucket b holds e in [2^((b-1024)/8), 2^((b-1023)/8));
// the last bucket also holds +inf (factorisations that broke down)
constexpr int kBuckets = 2048;
constexpr int kPerOctave = 8;

__device__ __forceinline__ int bucket_of(float e) {
  if (!(e > 0.f)) return -1;
  if (isinf(e) || isnan(e)) return kBuckets - 1;
  const int b = (int)floorf(log2f(e) * kPerOctave) + kBuckets / 2;
  return b < 0 ? 0 : (b >= kBuckets ? kBuckets - 1 : b);
}

__global__ void __launch_bounds__(512) k_err_hist(const float* __restrict__ err, const float* __restrict__ xn2, int n,
                           double* __restrict__ hist_sq, unsigned int* __restrict__ hist_n, double* __restrict__ xnorm2) {
  __shared__ double sq[kBuckets];
  __shared__ unsigned int cnt[kBuckets];
  __shared__ double xs;
  for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) {
    sq[i] = 0.0;
    cnt[i] = 0;
  }
  if (threadIdx.x == 0) xs = 0.0;
  __syncthreads();
  double xl = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const float e = err[q];
    const int b = bucket_of(e);
    if (b >= 0) {
      atomicAdd(&cnt[b], 1u);
      if (isfinite(e)) atomicAdd(&sq[b], (double)e * (double)e);
    }
    const float x2 = xn2[q];
    if (isfinite(x2)) xl += (double)x2;
  }
  for (int o = 16; o > 0; o >>= 1) xl += __shfl_xor_sync(0xffffffffu, xl, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&xs, xl);
  __syncthreads();
  for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) {
    if (cnt[i]) {
      atomicAdd(&hist_n[i], cnt[i]);
      atomicAdd(&hist_sq[i], sq[i]);
    }
  }
  if (threadIdx.x == 0) atomicAdd(xnorm2, xs);
}

// threshold: smallest e such that frequencies with e_q >= threshold go to FP64 and
// u^2 * sum_{e_q < threshold} e_q^2 <= (budget^2) * sum |x|^2.
// With P(c) = sum_{b < c} hist_sq[b] (nondecreasing in c), the cut bucket is the
// largest c <= kBuckets - 1 with P(c) <= allowed; the last bucket (+inf, the
// breakdowns) always goes to FP64.  One CTA of kThreshThreads threads scans the
// buckets, kBuckets / kThreshThreads consecutive buckets per thread.
constexpr int kThreshThreads = 512;
constexpr int kPerThread = kBuckets / kThreshThreads;

__global__ void __launch_bounds__(kThreshThreads) k_err_thresh(const double* __restrict__ hist_sq,
                                                               const double* __restrict__ xnorm2, double u,
                                                               double budget, float* __restrict__ thresh) {
  __shared__ double warp_sum[kThreshThreads / 32];
  __shared__ int cut;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double v[kPerThread];
  double own = 0.0;
#pragma unroll
  for (int i = 0; i < kPerThread; ++i) {
    v[i] = hist_sq[t * kPerThread + i];
    own += v[i];
  }
  // inclusive scan of the per-thread sums: within the warp, then across warps
  double inc = own;
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_sum[warp] = inc;
  if (t == 0) cut = 0;
  __syncthreads();
  double before = 0.0;
  for (int w = 0; w < warp; ++w) before += warp_sum[w];
  double p = before + inc - own;  // P(t * kPerThread)
  const double allow = budget * budget * xnorm2[0] / (u * u);
  int best = -1;
#pragma unroll
  for (int i = 0; i < kPerThread; ++i) {
    const int c = t * kPerThread + i;
    if (c <= kBuckets - 1 && p <= allow) best = c;
    p += v[i];
  }
  if (best >= 0) atomicMax(&cut, best);
  __syncthreads();
  if (t == 0) {
    const int c = cut;
    thresh[0] = c == kBuckets - 1 ? INFINITY : exp2f((float)(c - kBuckets / 2) / kPerOctave);
  }
}

__global__ void k_err_compact(const float* __restrict__ err, int n, const float* __restrict__ thresh,
                              int* __restrict__ list, int* __restrict__ count) {
  const float t = thresh[0];
  const int tb = isinf(t) ? kBuckets - 1 : (int)floorf(log2f(t) * kPerOctave) + kBuckets / 2;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int b = bucket_of(err[q]);
    if (b >= 0 && b >= tb) list[atomicAdd(count, 1)] = q;
  }
}

// status word of a fit: the bits of the counters the solve passes left behind
__global__ void k_fit_status(int* counters) {
  int st = counters[kStatusWord];
  if (counters[2] > 0) st |= FDL_ST_BREAKDOWN;
  if (counters[3] > 0) st |= FDL_ST_NONFINITE;
  counters[kStatusWord] = st;
}

}  // namespace

cudaError_t launch_fit_status(int* counters, cudaStream_t st) {
  k_fit_status<<<1, 1, 0, st>>>(counters);
  return cudaGetLastError();
}

size_t select_scratch_bytes() { return kBuckets * (sizeof(double) + sizeof(unsigned int)) + 64; }

cudaError_t launch_select_budget(const float* err, const float* xn2, int n, double u, double budget, void* scratch,
                                 int* list, int* count, cudaStream_t st) {
  double* hist_sq = static_cast<double*>(scratch);
  unsigned int* hist_n = reinterpret_cast<unsigned int*>(hist_sq + kBuckets);
  double* xnorm2 = reinterpret_cast<double*>(hist_n + kBuckets);
  float* thresh = reinterpret_cast<float*>(xnorm2 + 1);
  cudaError_t e = cudaMemsetAsync(scratch, 0, select_scratch_bytes(), st);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = sms * 2;
  k_err_hist<<<grid, 512, 0, st>>>(err, xn2, n, hist_sq, hist_n, xnorm2);
  k_err_thresh<<<1, kThreshThreads, 0, st>>>(hist_sq, xnorm2, u, budget, thresh);
  k_err_compact<<<grid, 512, 0, st>>>(err, n, thresh, list, count);
  return cudaGetLastError();
}

}  // namespace fdl
