// Smoothed best response with the dilated entropy DGF (Sec. 5) and the plain
// FP64 best response (the mu -> 0 limit used by the saddle-point residual).
//
// Sec. 5: argmin_q <q, g> + mu sum_j beta_j q_{p_j} d_j(q^j / q_{p_j}) is solved
// bottom-up: at simplex j every branch i gets g_hat_i = g_i + (values of the
// child simplexes D_j^i); the simplex problem has q_bar_i proportional to
// exp(-g_hat_i / (mu beta_j)) and value  g_hat_i* + t log q_bar_i* + t log n_j
// (t = mu beta_j) taken at i* = argmax q_bar (= argmin g_hat), which is
// m - t log(sum_i exp(-(g_hat_i - m) / t)) + t log n_j with m = min g_hat.
// The kernel evaluates that value as m - t log1p(sum_i expm1(-(g_hat_i - m)/t) / n_j),
// the same quantity without the cancellation of the two logarithms in FP32.
// Top-down: q_i = q_{p_j} q_bar_i.
//
// Sec. 6: the per-hand treeplexes form a Cartesian product at the root, so
// hands are independent.  One CTA owns 32 hands (one per lane, so loads of a
// sequence row are 128-byte coalesced) and all simplexes; within a level its
// warps split the simplexes; levels are separated by __syncthreads.  Child
// values V[j][lane] and the conditional q_bar (then q) live in shared memory.
// The value summed over hands and root simplexes is reduced in FP64: per-CTA
// partials, the last CTA to finish adds them in index order (deterministic).
#include <math.h>

#include "egt_internal.cuh"

namespace egt {
namespace {

// Sum of per-CTA values in a fixed order by the last CTA to arrive.
// cta_value is read from thread 0.
__device__ void finish_value(double cta_value, double scale, double* partials,
                             unsigned int* counter, double* value_dev, int* status) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = cta_value;
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last && threadIdx.x < 32) {
    __threadfence();
    double v = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) v += __ldcg(partials + i);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if (threadIdx.x == 0) {
      v *= scale;
      *value_dev = v;
      if (!isfinite(v) && status) atomicExch(status, 1);
      *counter = 0u;
    }
  }
}

__global__ void __launch_bounds__(kSbrHands* kSbrWarps)
    sbr_kernel(DevGame g, int player, SbrArgs a) {
  extern __shared__ __align__(16) float sm[];
  const DevTpx tp = g.tpx[player];
  float* V = sm;                                   // [J][32] simplex values
  float* U = V + (size_t)tp.J * kSbrHands;         // [S][32] g_hat -> q_bar -> q
  float* tj = U + (size_t)tp.S * kSbrHands;        // [J] t_j = mu beta_j
  float* itj = tj + tp.J;                          // [J] 1 / t_j
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int h = blockIdx.x * kSbrHands + lane;
  const bool live = h < g.H;
  const int ld = g.ld;

  for (int j = threadIdx.x; j < tp.J; j += blockDim.x) {
    const double t = a.mu * tp.beta[j];
    tj[j] = (float)t;
    itj[j] = (float)(1.0 / t);
  }
  __syncthreads();

  // bottom-up: deepest level first
  for (int l = tp.L - 1; l >= 0; --l) {
    for (int j = tp.level_ptr[l] + warp; j < tp.level_ptr[l + 1]; j += kSbrWarps) {
      const int s0 = tp.inf_first[j], n = tp.inf_n[j];
      float m = INFINITY;
      for (int i = 0; i < n; ++i) {
        const int s = s0 + i;
        float gh = (a.g != nullptr && live) ? a.sign * a.g[(size_t)s * ld + h] : 0.f;
        for (int c = tp.child_ptr[s]; c < tp.child_ptr[s + 1]; ++c)
          gh += V[tp.child_idx[c] * kSbrHands + lane];
        U[s * kSbrHands + lane] = gh;
        m = fminf(m, gh);
      }
      // e_i = exp(-(g_hat_i - m)/t) keeps tiny q_bar accurate; X = sum_i (e_i - 1) from
      // expm1 keeps the value accurate when t >> spread of g_hat (there log(sum e) and
      // log n nearly cancel): t log q_bar_i* + t log n = -t log1p(X / n)
      const float it = itj[j];
      float sum = 0.f, X = 0.f;
      for (int i = 0; i < n; ++i) {
        float* u = U + (s0 + i) * kSbrHands + lane;
        const float d = -(*u - m) * it;
        const float e = expf(d);
        X += expm1f(d);
        *u = e;
        sum += e;
      }
      const float inv = 1.f / sum;
      for (int i = 0; i < n; ++i) U[(s0 + i) * kSbrHands + lane] *= inv;
      V[j * kSbrHands + lane] = m - tj[j] * log1pf(X / (float)n);
    }
    __syncthreads();
  }

  if (a.value_dev != nullptr) {
    __shared__ double cta_val;
    if (warp == 0) {
      double v = 0.0;
      if (live)
        for (int j = tp.level_ptr[0]; j < tp.level_ptr[1]; ++j) v += (double)V[j * kSbrHands + lane];
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
      if (lane == 0) cta_val = v;
    }
    __syncthreads();
    finish_value(cta_val, 1.0, a.partials, a.counter, a.value_dev, a.status);
  }

  if (a.out == nullptr) return;
  // top-down: q_i = q_{p_j} q_bar_i, written (or mixed into old) as it is produced
  const float tau = a.tau, omt = 1.f - a.tau;
  for (int l = 0; l < tp.L; ++l) {
    for (int j = tp.level_ptr[l] + warp; j < tp.level_ptr[l + 1]; j += kSbrWarps) {
      const int p = tp.inf_parent[j];
      const float qp = p < 0 ? 1.f : U[p * kSbrHands + lane];
      const int s0 = tp.inf_first[j], n = tp.inf_n[j];
      for (int i = 0; i < n; ++i) {
        const int s = s0 + i;
        const float q = qp * U[s * kSbrHands + lane];
        U[s * kSbrHands + lane] = q;
        const size_t idx = (size_t)s * ld + h;
        float o = q;
        if (a.old != nullptr) o = omt * a.old[idx] + tau * q;
        a.out[idx] = live ? o : 0.f;
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSbrHands* kSbrWarps)
    br64_kernel(DevGame g, int player, const double* __restrict__ gv, double sign,
                double* value_dev, double* partials, unsigned int* counter) {
  extern __shared__ __align__(16) double smd[];
  const DevTpx tp = g.tpx[player];
  double* V = smd;                                 // [J][32]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int h = blockIdx.x * kSbrHands + lane;
  const bool live = h < g.H;
  const int ld = g.ld;
  for (int l = tp.L - 1; l >= 0; --l) {
    for (int j = tp.level_ptr[l] + warp; j < tp.level_ptr[l + 1]; j += kSbrWarps) {
      const int s0 = tp.inf_first[j], n = tp.inf_n[j];
      double m = INFINITY;
      for (int i = 0; i < n; ++i) {
        const int s = s0 + i;
        double gh = live ? sign * gv[(size_t)s * ld + h] : 0.0;
        for (int c = tp.child_ptr[s]; c < tp.child_ptr[s + 1]; ++c)
          gh += V[tp.child_idx[c] * kSbrHands + lane];
        m = fmin(m, gh);
      }
      V[j * kSbrHands + lane] = m;
    }
    __syncthreads();
  }
  __shared__ double cta_val;
  if (warp == 0) {
    double v = 0.0;
    if (live)
      for (int j = tp.level_ptr[0]; j < tp.level_ptr[1]; ++j) v += V[j * kSbrHands + lane];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if (lane == 0) cta_val = v;
  }
  __syncthreads();
  finish_value(cta_val, sign, partials, counter, value_dev, nullptr);
}

}  // namespace

size_t sbr_smem_bytes(const DevGame& g, int player) {
  const DevTpx& tp = g.tpx[player];
  return ((size_t)tp.J * kSbrHands + (size_t)tp.S * kSbrHands + 2 * (size_t)tp.J) * sizeof(float);
}

size_t br_smem_bytes(const DevGame& g, int player) {
  return (size_t)g.tpx[player].J * kSbrHands * sizeof(double);
}

int opt_in_dynamic_smem(const void* kernel) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa{};
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, kernel) != cudaSuccess)
    return -1;
  const int limit = optin - (int)fa.sharedSizeBytes;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, limit) != cudaSuccess)
    return -1;
  return limit;
}

void launch_sbr(const DevGame& g, int player, const SbrArgs& a, cudaStream_t st) {
  static int limit = 0;
  if (limit == 0) limit = opt_in_dynamic_smem((const void*)sbr_kernel);
  const int grid = g.ld / kSbrHands;
  sbr_kernel<<<grid, kSbrHands * kSbrWarps, sbr_smem_bytes(g, player), st>>>(g, player, a);
}

void launch_br64(const DevGame& g, int player, const double* gv, double sign, double* value_dev,
                 double* partials, unsigned int* counter, cudaStream_t st) {
  static int limit = 0;
  if (limit == 0) limit = opt_in_dynamic_smem((const void*)br64_kernel);
  const int grid = g.ld / kSbrHands;
  br64_kernel<<<grid, kSbrHands * kSbrWarps, br_smem_bytes(g, player), st>>>(
      g, player, gv, sign, value_dev, partials, counter);
}

}  // namespace egt
