// Standalone smoothed-best-response and FP64 best-response kernels: one CTA per
// 16 hands running the shared bodies of sbr_impl.cuh (Sec. 5 recursion).  The
// value summed over hands and root simplexes is reduced in FP64: per-CTA
// partials, the last CTA to finish adds them in a fixed order (deterministic).
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "egt_internal.cuh"
#include "sbr_impl.cuh"

namespace egt {
namespace {

// The last CTA to arrive sums the per-CTA partials (fixed order) into *value_dev.
__device__ void finish_value(double* partials, unsigned int* counter, double* value_dev,
                             int* status) {
  __shared__ bool is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last && threadIdx.x < 32) {
    __threadfence();
    const double v = reduce_partials(partials, gridDim.x, threadIdx.x);
    if (threadIdx.x == 0) {
      *value_dev = v;
      if (!isfinite(v) && status) atomicExch(status, 1);
      *counter = 0u;
    }
  }
}

// finish_value over the n CTAs [first, first + n) of the grid that share partials and
// counter (the same fixed-order sum of n partials).
__device__ void finish_value_n(double* partials, int n, unsigned int* counter, double* value_dev) {
  __shared__ bool is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    is_last = (prev == (unsigned int)n - 1u);
  }
  __syncthreads();
  if (is_last && threadIdx.x < 32) {
    __threadfence();
    const double v = reduce_partials(partials, n, threadIdx.x);
    if (threadIdx.x == 0) {
      *value_dev = v;
      *counter = 0u;
    }
  }
}

__global__ void __launch_bounds__(kItemThreads) sbr_kernel(DevGame g, int player, SbrArgs a) {
  extern __shared__ __align__(16) float sm[];
  SbrItemArgs ia;
  ia.g = a.g;
  ia.contrib = a.contrib;
  ia.grz = player ? g.rz[1] : g.rz[0];
  ia.sign = a.sign;
  ia.mu = a.mu;
  ia.old = a.old;
  ia.tau = a.tau;
  ia.out = a.out;
  ia.value_partial = a.value_dev != nullptr ? a.partials + blockIdx.x : nullptr;
  unsigned char* raw = reinterpret_cast<unsigned char*>(sm);
  const TpxTab tt = stage_tpx_tab(g, player, raw);
  __syncthreads();
  sbr_item(g, tt, blockIdx.x, ia, reinterpret_cast<float*>(raw + tpx_tab_bytes(g, player)));
  if (a.value_dev != nullptr) finish_value(a.partials, a.counter, a.value_dev, a.status);
}

__global__ void __launch_bounds__(kItemThreads)
    br64_kernel(DevGame g, int player, const double* __restrict__ gv, bool contrib, double sign,
                double* value_dev, double* partials, unsigned int* counter) {
  extern __shared__ __align__(16) double smd[];
  unsigned char* raw = reinterpret_cast<unsigned char*>(smd);
  const TpxTab tt = stage_tpx_tab(g, player, raw);
  __syncthreads();
  const double* grz = player ? g.rz64[1] : g.rz64[0];
  br64_item(g, tt, blockIdx.x, gv, contrib, grz, sign, partials + blockIdx.x,
            reinterpret_cast<double*>(raw + tpx_tab_bytes(g, player)));
  finish_value(partials, counter, value_dev, nullptr);
}

// CTAs [0, NB): player 0 (sign +1, gv0); [NB, 2 NB): player 1 (sign -1, gv1).
__global__ void __launch_bounds__(kItemThreads)
    br64_pair_kernel(DevGame g, const double* __restrict__ gv0, const double* __restrict__ gv1, double* value0,
                     double* value1, double* partials, unsigned int* counter) {
  extern __shared__ __align__(16) double smd[];
  const int NB = g.ld / kSbrHands;
  const int p = (int)blockIdx.x >= NB ? 1 : 0;
  const int blk = (int)blockIdx.x - p * NB;
  unsigned char* raw = reinterpret_cast<unsigned char*>(smd);
  const TpxTab tt = stage_tpx_tab(g, p, raw);
  __syncthreads();
  const double* grz = p ? g.rz64[1] : g.rz64[0];
  double* part = partials + p * NB;
  br64_item(g, tt, blk, p ? gv1 : gv0, true, grz, p ? -1.0 : 1.0, part + blk,
            reinterpret_cast<double*>(raw + tpx_tab_bytes(g, p)));
  finish_value_n(part, NB, counter + p, p ? value1 : value0);
}

}  // namespace

size_t sbr_smem_bytes(const DevGame& g, int player) {
  return tpx_tab_bytes(g, player) + sbr_item_smem(g, player);
}

size_t br_smem_bytes(const DevGame& g, int player) {
  return tpx_tab_bytes(g, player) + br_item_smem(g, player);
}

// The opt-in is a property of (kernel, device): cudaFuncSetAttribute acts on the
// device current at the call.  Successful opt-ins are remembered per pair under a
// lock (host threads may launch concurrently); a failed one is retried next time.
int opt_in_dynamic_smem(const void* kernel) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(kernel, dev);
  const auto it = done.find(key);
  if (it != done.end()) return it->second;
  int optin = 0;
  cudaFuncAttributes fa{};
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, kernel) != cudaSuccess)
    return -1;
  const int limit = optin - (int)fa.sharedSizeBytes;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, limit) != cudaSuccess)
    return -1;
  done[key] = limit;
  return limit;
}

void launch_sbr(const DevGame& g, int player, const SbrArgs& a, cudaStream_t st) {
  opt_in_dynamic_smem((const void*)sbr_kernel);
  const int grid = g.ld / kSbrHands;
  sbr_kernel<<<grid, kItemThreads, sbr_smem_bytes(g, player), st>>>(g, player, a);
}

void launch_br64_pair(const DevGame& g, const double* gv0, const double* gv1, double* value0, double* value1,
                      double* partials, unsigned int* counter, cudaStream_t st) {
  opt_in_dynamic_smem((const void*)br64_pair_kernel);
  const int NB = g.ld / kSbrHands;
  const size_t smem = std::max(br_smem_bytes(g, 0), br_smem_bytes(g, 1));
  br64_pair_kernel<<<2 * NB, kItemThreads, smem, st>>>(g, gv0, gv1, value0, value1, partials, counter);
}

void launch_br64(const DevGame& g, int player, const double* gv, bool contrib, double sign, double* value_dev,
                 double* partials, unsigned int* counter, cudaStream_t st) {
  opt_in_dynamic_smem((const void*)br64_kernel);
  const int grid = g.ld / kSbrHands;
  br64_kernel<<<grid, kItemThreads, br_smem_bytes(g, player), st>>>(g, player, gv, contrib, sign,
                                                                     value_dev, partials, counter);
}

}  // namespace egt
