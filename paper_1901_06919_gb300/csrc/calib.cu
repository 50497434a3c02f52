// Calibration objective and gradient of Sec. V-B.
// At every listed frequency w the layers x are re-solved at the current
// (u, d) by the closed form (recomputed, not stored); then with r = A x - b
//   loss   += sum_c |r_c|^2 + lambda x_c* Gamma*Gamma x_c        (Eq. CalibrationProb)
//   core_jk = sum_c Im(r_jc conj(A_jk) conj(x_kc))
//   dL/dP^a_jk = 4 pi sum_w w_a core_jk, P^a = u_a d^T             (Eq. gradP, 2D)
//   grad_u[j][a] = sum_k d_k dL/dP^a_jk,  grad_d[k] = sum_{j,a} u_ja dL/dP^a_jk  (Eq. gradD)
// Sums run in a fixed order (fixed warp-to-frequency assignment, per-CTA
// partials, a final ordered reduction), so results are reproducible.
#include "hp_solve.cuh"

namespace fdl {

namespace {

constexpr int kCalibWarps = 4;

template <class T>
__global__ void __launch_bounds__(kCalibWarps * 32) k_calib(CalibParams cp) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int M = cp.W >> 1;
  const int N = cp.N, C = cp.C, K = cp.K;
  const int nacc = 1 + 2 * K + N;
  HpProblem p;
  p.b = cp.b;
  p.u = cp.u;
  p.d = cp.d;
  p.exp_table = cp.exp_table;
  p.K = K;
  p.C = C;
  p.N = N;
  p.H = cp.H;
  p.W = cp.W;
  p.reg = cp.reg;
  p.lam = cp.lam_d;
  p.lam_eps = 0.0;
  const size_t pw = hp_warp_elems<T>(N, C) + 4;  // + r_j for C channels
  cx<T>* G = reinterpret_cast<cx<T>*>(smem4) + warp * pw;
  cx<T>* Arow = G + N * (N + 1);
  cx<T>* Y = Arow + N;
  cx<T>* Rj = Y + N * C;
  double* acc = reinterpret_cast<double*>(reinterpret_cast<cx<T>*>(smem4) + kCalibWarps * pw) + warp * nacc;
  for (int e = lane; e < nacc; e += 32) acc[e] = 0.0;
  double gd_lane[2] = {0.0, 0.0};  // grad_d for rows lane, lane + 32 (before the 4 pi factor)
  double loss_lane = 0.0;
  __syncwarp();
  const int total = cp.bins ? cp.nbins : cp.H * (M + 1);
  for (int li = blockIdx.x * kCalibWarps + warp; li < total; li += gridDim.x * kCalibWarps) {
    const int qd = cp.bins ? cp.bins[li] : li;  // dense index ky * (M+1) + kx
    if (qd < 0 || qd >= cp.H * (M + 1)) continue;  // out-of-range entries of a caller's list are skipped
    const int ky = qd / (M + 1), kx = qd - ky * (M + 1);
    hp_solve_bin<T>(p, ky, kx, G, Arow, Y);
    const Freq fq0 = bin_freq(ky, kx, cp.H, cp.W);
    const auto fq = freq_prep(fq0, T{});
    // w in double for the gradient factors of Eq. gradP
    const double wx = (double)kx / (double)cp.W, wy = (double)fq0.kyp / (double)cp.H;
    // lambda x* Gamma*Gamma x (Gamma independent of d)
    if (lane < C) {
      const int c = lane;
      double rq = 0.0;
      for (int i = 0; i < N; ++i) {
        const int l0 = cp.reg == 1 ? (i >= 2 ? i - 2 : 0) : i;
        const int l1 = cp.reg == 1 ? (i + 2 < N ? i + 2 : N - 1) : i;
        for (int l = l0; l <= l1; ++l) {
          const double g = cp.reg == 1 ? (double)layer2_gtg(i, l, N) : 1.0;
          const cx<T> xi = Y[i * C + c], xl = Y[l * C + c];
          rq += g * (r_to_double(xi.re) * r_to_double(xl.re) + r_to_double(xi.im) * r_to_double(xl.im));
        }
      }
      loss_lane += cp.lam_d * rq;
    }
    for (int j = 0; j < K; ++j) {
      const float2 uj = __ldg(reinterpret_cast<const float2*>(cp.u) + j);
      const auto th = theta_r(uj.x, uj.y, fq, T{});
      for (int r = lane; r < N; r += 32) Arow[r] = cexp2pi(phase_r(th, __ldg(cp.d + r)), cp.exp_table);
      __syncwarp();
      if (lane < C) {
        const int c = lane;
        const float2 bj = *cp.b.at((long long)j * C + c, ky, kx, M);
        cx<T> r = {r_from(-bj.x, T{}), r_from(-bj.y, T{})};
        for (int k = 0; k < N; ++k) r = cx_add(r, cx_mul(Arow[k], Y[k * C + c]));
        Rj[c] = r;
        const double rr = r_to_double(r.re), ri = r_to_double(r.im);
        loss_lane += rr * rr + ri * ri;
      }
      __syncwarp();
      const double thd = (double)uj.x * wx + (double)uj.y * wy;
      double sj = 0.0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = lane + 32 * h;
        if (k < N) {
          double core = 0.0;
          for (int c = 0; c < C; ++c) {
            const cx<T> z = cx_mul_conj(cx_mul_conj(Rj[c], Arow[k]), Y[k * C + c]);
            core += r_to_double(z.im);
          }
          sj += (double)__ldg(cp.d + k) * core;
          gd_lane[h] += thd * core;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sj += __shfl_xor_sync(0xffffffffu, sj, o);
      if (lane == 0) {
        acc[1 + 2 * j] += wx * sj;
        acc[1 + 2 * j + 1] += wy * sj;
      }
      __syncwarp();
    }
  }
  // per-warp totals -> shared accumulators
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) loss_lane += __shfl_xor_sync(0xffffffffu, loss_lane, o);
  if (lane == 0) acc[0] = loss_lane;
  for (int h = 0; h < 2; ++h)
    if (lane + 32 * h < N) acc[1 + 2 * K + lane + 32 * h] = gd_lane[h];
  __syncthreads();
  double* base = reinterpret_cast<double*>(reinterpret_cast<cx<T>*>(smem4) + kCalibWarps * pw);
  for (int e = threadIdx.x; e < nacc; e += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < kCalibWarps; ++w) s += base[w * nacc + e];
    cp.partials[(long long)blockIdx.x * nacc + e] = s;
  }
}

// Relaxed model (free shifts P): one warp per CTA, per-CTA accumulators
// [loss | dL/dP^x_jk, dL/dP^y_jk for (j, k) row-major] in shared memory, lane k adding
// w_a core_jk for its own layers (no two lanes touch one entry); fixed order, reproducible.
template <class T>
__global__ void __launch_bounds__(32) k_calib_shifts(CalibParams cp) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x;
  const int M = cp.W >> 1;
  const int N = cp.N, C = cp.C, K = cp.K;
  const int nacc = 1 + 2 * K * N;
  HpProblem p;
  p.b = cp.b;
  p.u = nullptr;
  p.d = cp.d;
  p.exp_table = cp.exp_table;
  p.K = K;
  p.C = C;
  p.N = N;
  p.H = cp.H;
  p.W = cp.W;
  p.reg = cp.reg;
  p.lam = cp.lam_d;
  p.lam_eps = 0.0;
  p.P = cp.P;
  const size_t pw = hp_warp_elems<T>(N, C) + 4;
  cx<T>* G = reinterpret_cast<cx<T>*>(smem4);
  cx<T>* Arow = G + N * (N + 1);
  cx<T>* Y = Arow + N;
  cx<T>* Rj = Y + N * C;
  double* acc = reinterpret_cast<double*>(reinterpret_cast<cx<T>*>(smem4) + pw);
  for (int e = lane; e < nacc; e += 32) acc[e] = 0.0;
  double loss_lane = 0.0;
  __syncwarp();
  const float2* P2 = reinterpret_cast<const float2*>(cp.P);
  const int total = cp.bins ? cp.nbins : cp.H * (M + 1);
  for (int li = blockIdx.x; li < total; li += gridDim.x) {
    const int qd = cp.bins ? cp.bins[li] : li;
    if (qd < 0 || qd >= cp.H * (M + 1)) continue;
    const int ky = qd / (M + 1), kx = qd - ky * (M + 1);
    hp_solve_bin<T>(p, ky, kx, G, Arow, Y);
    const Freq fq0 = bin_freq(ky, kx, cp.H, cp.W);
    const auto fq = freq_prep(fq0, T{});
    const double wx = (double)kx / (double)cp.W, wy = (double)fq0.kyp / (double)cp.H;
    if (lane < C) {
      const int c = lane;
      double rq = 0.0;
      for (int i = 0; i < N; ++i) {
        const int l0 = cp.reg == 1 ? (i >= 2 ? i - 2 : 0) : i;
        const int l1 = cp.reg == 1 ? (i + 2 < N ? i + 2 : N - 1) : i;
        for (int l = l0; l <= l1; ++l) {
          const double g = cp.reg == 1 ? (double)layer2_gtg(i, l, N) : 1.0;
          const cx<T> xi = Y[i * C + c], xl = Y[l * C + c];
          rq += g * (r_to_double(xi.re) * r_to_double(xl.re) + r_to_double(xi.im) * r_to_double(xl.im));
        }
      }
      loss_lane += cp.lam_d * rq;
    }
    for (int j = 0; j < K; ++j) {
      for (int r = lane; r < N; r += 32) {
        const float2 pr = __ldg(P2 + (long long)j * N + r);
        Arow[r] = cexp2pi(phase_r(theta_r(pr.x, pr.y, fq, T{}), 1.f), cp.exp_table);
      }
      __syncwarp();
      if (lane < C) {
        const int c = lane;
        const float2 bj = *cp.b.at((long long)j * C + c, ky, kx, M);
        cx<T> r = {r_from(-bj.x, T{}), r_from(-bj.y, T{})};
        for (int k = 0; k < N; ++k) r = cx_add(r, cx_mul(Arow[k], Y[k * C + c]));
        Rj[c] = r;
        const double rr = r_to_double(r.re), ri = r_to_double(r.im);
        loss_lane += rr * rr + ri * ri;
      }
      __syncwarp();
      for (int k = lane; k < N; k += 32) {
        double core = 0.0;
        for (int c = 0; c < C; ++c) {
          const cx<T> z = cx_mul_conj(cx_mul_conj(Rj[c], Arow[k]), Y[k * C + c]);
          core += r_to_double(z.im);
        }
        acc[1 + 2 * (j * N + k)] += wx * core;
        acc[2 + 2 * (j * N + k)] += wy * core;
      }
      __syncwarp();
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) loss_lane += __shfl_xor_sync(0xffffffffu, loss_lane, o);
  if (lane == 0) acc[0] = loss_lane;
  __syncwarp();
  for (int e = lane; e < nacc; e += 32) cp.partials[(long long)blockIdx.x * nacc + e] = acc[e];
}

__global__ void k_calib_shifts_reduce(const double* partials, int nblocks, int nacc, float* loss, float* grad_P) {
  const double fourpi = 12.566370614359172;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nacc; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[(long long)b * nacc + e];
    if (e == 0) loss[0] = (float)s;
    else grad_P[e - 1] = (float)(fourpi * s);
  }
}

__global__ void k_calib_reduce(const double* partials, int nblocks, int K, int N, float* loss, float* grad_u,
                               float* grad_d) {
  const int nacc = 1 + 2 * K + N;
  const double fourpi = 12.566370614359172;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nacc; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[(long long)b * nacc + e];
    if (e == 0) loss[0] = (float)s;
    else if (e < 1 + 2 * K) grad_u[e - 1] = (float)(fourpi * s);
    else grad_d[e - 1 - 2 * K] = (float)(fourpi * s);
  }
}

template <class T>
cudaError_t launch_t(const CalibParams& p, cudaStream_t st) {
  const size_t pw = hp_warp_elems<T>(p.N, p.C) + 4;
  const size_t smem = kCalibWarps * pw * sizeof(cx<T>) + (size_t)kCalibWarps * (1 + 2 * p.K + p.N) * sizeof(double);
  cudaError_t e = set_smem((const void*)k_calib<T>, smem);
  if (e != cudaSuccess) return e;
  k_calib<T><<<kCalibGrid, kCalibWarps * 32, smem, st>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_calib_reduce<<<4, 256, 0, st>>>(p.partials, kCalibGrid, p.K, p.N, p.loss, p.grad_u, p.grad_d);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_shifts_t(const CalibParams& p, cudaStream_t st) {
  const size_t pw = hp_warp_elems<T>(p.N, p.C) + 4;
  const size_t smem = pw * sizeof(cx<T>) + calib_shifts_acc_bytes(p.K, p.N);
  cudaError_t e = set_smem((const void*)k_calib_shifts<T>, smem);
  if (e != cudaSuccess) return e;
  k_calib_shifts<T><<<kCalibGrid, 32, smem, st>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nacc = 1 + 2 * p.K * p.N;
  k_calib_shifts_reduce<<<(nacc + 255) / 256, 256, 0, st>>>(p.partials, kCalibGrid, nacc, p.loss, p.grad_P);
  return cudaGetLastError();
}

}  // namespace

size_t calib_shifts_acc_bytes(int K, int N) { return (size_t)(1 + 2 * K * N) * sizeof(double); }

cudaError_t launch_calib_grad(const CalibParams& p, cudaStream_t st) {
  if (p.P != nullptr) return p.f64 ? launch_shifts_t<R64>(p, st) : launch_shifts_t<Rdf>(p, st);
  return p.f64 ? launch_t<R64>(p, st) : launch_t<Rdf>(p, st);
}

}  // namespace fdl
