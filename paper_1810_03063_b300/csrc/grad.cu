// Standalone gradient-product kernel: one CTA per output sequence running the
// shared body grad_item (grad_impl.cuh: Sec. 3 products over the poker river
// payoff structure, exact fixed-point sums).  The per-game tables are staged
// in shared memory first.
#include "egt_internal.cuh"
#include "grad_impl.cuh"

namespace egt {
namespace {

template <typename TIn>
__global__ void __launch_bounds__(kItemThreads)
    grad_kernel(DevGame g, int player, const TIn* __restrict__ in, float* __restrict__ out32,
                double* __restrict__ out64) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GradTab tb = stage_grad_tab(g, smem_raw);
  __syncthreads();
  grad_item<TIn>(g, tb, player, blockIdx.x, in, out32, out64, smem_raw + grad_tab_bytes(g));
}

template <typename TIn>
void launch(const DevGame& g, int player, const TIn* in, float* out32, double* out64, cudaStream_t st) {
  static int limit = 0;   // one process-wide opt-in per instantiation
  if (limit == 0) limit = opt_in_dynamic_smem((const void*)grad_kernel<TIn>);
  grad_kernel<TIn><<<g.tpx[player].S, kItemThreads, grad_smem_bytes(g, true), st>>>(g, player, in,
                                                                                    out32, out64);
}

}  // namespace

size_t grad_smem_bytes(const DevGame& g, bool) { return grad_tab_bytes(g) + grad_item_smem(g); }

template <>
void launch_grad<float, float>(const DevGame& g, int player, const float* in, float* out, cudaStream_t st) {
  launch<float>(g, player, in, out, nullptr, st);
}

template <>
void launch_grad<double, double>(const DevGame& g, int player, const double* in, double* out,
                                 cudaStream_t st) {
  launch<double>(g, player, in, nullptr, out, st);
}

template <>
void launch_grad<float, double>(const DevGame& g, int player, const float* in, double* out,
                                cudaStream_t st) {
  launch<float>(g, player, in, nullptr, out, st);
}

void launch_grad_dual(const DevGame& g, int player, const float* in, float* out32, double* out64,
                      cudaStream_t st) {
  launch<float>(g, player, in, out32, out64, st);
}

}  // namespace egt
