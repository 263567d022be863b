// Standalone gradient-product kernel: one CTA per output sequence running the
// shared body grad_item (grad_impl.cuh: Sec. 3 products over the poker river
// payoff structure, exact fixed-point prefix sums).  The per-game tables are
// staged in shared memory first.
#include "egt_internal.cuh"
#include "grad_impl.cuh"

namespace egt {
namespace {

template <typename TIn, typename T>
__global__ void __launch_bounds__(kItemThreads)
    grad_kernel(DevGame g, int player, const TIn* __restrict__ in, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GradTab tb = stage_grad_tab(g, smem_raw);
  __syncthreads();
  grad_item<TIn, T>(g, tb, player, blockIdx.x, in, out, smem_raw + grad_tab_bytes(g));
}

}  // namespace

size_t grad_smem_bytes(const DevGame& g, bool f64) {
  return grad_tab_bytes(g) + grad_item_smem(g, f64);
}

template <typename TIn, typename T>
void launch_grad(const DevGame& g, int player, const TIn* in, T* out, cudaStream_t st) {
  static int limit = 0;   // one process-wide opt-in per instantiation
  if (limit == 0) limit = opt_in_dynamic_smem((const void*)grad_kernel<TIn, T>);
  grad_kernel<TIn, T><<<g.tpx[player].S, kItemThreads, grad_smem_bytes(g, sizeof(T) == 8), st>>>(
      g, player, in, out);
}

template void launch_grad<float, float>(const DevGame&, int, const float*, float*, cudaStream_t);
template void launch_grad<double, double>(const DevGame&, int, const double*, double*,
                                          cudaStream_t);
template void launch_grad<float, double>(const DevGame&, int, const float*, double*,
                                         cudaStream_t);

}  // namespace egt
