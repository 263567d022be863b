// Standalone gradient-product kernels.  The terminal kernel runs one CTA per
// terminal of the output player's grouping on the shared body term_item
// (grad_impl.cuh: Sec. 3 products over the poker river payoff structure, exact
// fixed-point sums), after staging the per-game tables in shared memory.  The
// combine kernel turns those contributions into dense product rows (the public
// egt_grad / egt_grad_f64); the solver's own kernels read the contributions
// directly.
#include "egt_internal.cuh"
#include "grad_impl.cuh"

namespace egt {
namespace {

template <typename TIn>
__global__ void __launch_bounds__(kItemThreads)
    term_kernel(DevGame g, int player, const TIn* __restrict__ in, float* __restrict__ c32,
                double* __restrict__ c64) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GradTab tb = stage_grad_tab(g, smem_raw);
  __syncthreads();
  term_item<TIn>(g, tb, player, blockIdx.x, in, c32, c64, smem_raw + grad_tab_bytes(g));
}

// CTAs [0, T0): player 0's terminals (A y from y); [T0, T0 + T1): player 1's (A^T x from x).
__global__ void __launch_bounds__(kItemThreads)
    term_pair64_kernel(DevGame g, const float* __restrict__ y, const float* __restrict__ x,
                       double* __restrict__ c64_0, double* __restrict__ c64_1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GradTab tb = stage_grad_tab(g, smem_raw);
  __syncthreads();
  const int T0 = g.terms[0].n;
  const int p = (int)blockIdx.x >= T0 ? 1 : 0;
  term_item<float>(g, tb, p, (int)blockIdx.x - p * T0, p ? x : y, nullptr, p ? c64_1 : c64_0,
                   smem_raw + grad_tab_bytes(g));
}

__device__ __forceinline__ float combine_one(const float* c, const int* ptr, int s, int ld, int h,
                                             const DevGame& g, int player) {
  return product32(c, ptr, s, ld, h, (player ? g.rz[1] : g.rz[0])[h]);
}

__device__ __forceinline__ double combine_one(const double* c, const int* ptr, int s, int ld, int h,
                                              const DevGame& g, int player) {
  return product64(c, ptr, s, ld, h, (player ? g.rz64[1] : g.rz64[0])[h]);
}

template <typename T>
__global__ void __launch_bounds__(256) combine_kernel(DevGame g, int player, const T* __restrict__ c,
                                                      T* __restrict__ out) {
  const int S = player ? g.tpx[1].S : g.tpx[0].S;
  const int* ptr = player ? g.terms[1].ptr : g.terms[0].ptr;
  const size_t n = (size_t)S * g.ld;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(i / g.ld), h = (int)(i % g.ld);
    out[i] = h < g.H ? combine_one(c, ptr, s, g.ld, h, g, player) : T(0);
  }
}

template <typename TIn>
void launch_t(const DevGame& g, int player, const TIn* in, float* c32, double* c64, cudaStream_t st) {
  opt_in_dynamic_smem((const void*)term_kernel<TIn>);   // once per device
  const int T = player ? g.terms[1].n : g.terms[0].n;
  if (T == 0) return;
  term_kernel<TIn><<<T, kItemThreads, grad_smem_bytes(g), st>>>(g, player, in, c32, c64);
}

}  // namespace

size_t grad_smem_bytes(const DevGame& g) { return grad_tab_bytes(g) + grad_item_smem(g); }

template <>
void launch_terms<float>(const DevGame& g, int player, const float* in, float* c32, double* c64,
                         cudaStream_t st) {
  launch_t<float>(g, player, in, c32, c64, st);
}

template <>
void launch_terms<double>(const DevGame& g, int player, const double* in, float* c32, double* c64,
                          cudaStream_t st) {
  launch_t<double>(g, player, in, c32, c64, st);
}

void launch_terms_pair64(const DevGame& g, const float* y, const float* x, double* c64_0, double* c64_1,
                         cudaStream_t st) {
  opt_in_dynamic_smem((const void*)term_pair64_kernel);
  const int T = g.terms[0].n + g.terms[1].n;
  if (T == 0) return;
  term_pair64_kernel<<<T, kItemThreads, grad_smem_bytes(g), st>>>(g, y, x, c64_0, c64_1);
}

template <typename T>
void launch_combine(const DevGame& g, int player, const T* c, T* out, cudaStream_t st) {
  const int S = player ? g.tpx[1].S : g.tpx[0].S;
  const size_t n = (size_t)S * g.ld;
  const int grid = (int)std::min<size_t>((n + 255) / 256, 148 * 8);
  if (grid > 0) combine_kernel<T><<<grid, 256, 0, st>>>(g, player, c, out);
}

template void launch_combine<float>(const DevGame&, int, const float*, float*, cudaStream_t);
template void launch_combine<double>(const DevGame&, int, const double*, double*, cudaStream_t);

}  // namespace egt
