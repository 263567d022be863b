// Gradient products A y and A^T x over the poker river payoff structure.
//
// Sec. 3: every EGT step needs grad f = A y and grad phi = A^T x.  Sec. 6 notes
// that for poker the product can use the per-terminal hand-vs-hand structure
// instead of a sparse matrix.  For a terminal b and an output hand h:
//
//   fold:     r_me(h)/Z * u_b * sum_{h' disjoint from h} w(h')
//   showdown: r_me(h)/Z * c_b * (sum_{disjoint, stronger} w - sum_{disjoint, weaker} w)
//
// with w = r_opp (.) in[sigma_opp(b)].  Disjoint sums use card-removal
// inclusion-exclusion: total - per-card totals of h's cards + w(h) (the only
// hand holding both cards is h itself).  Weaker / stronger sums use exclusive
// prefix sums over the hands in ascending strength (up to h's tie group start /
// from its end) minus the same prefix over each of h's cards' hand lists.
//
// One CTA per output sequence s: it loops over the terminals whose own
// sequence is s, stages w in shared memory, scans it (raking scan + warp
// shuffles) and the per-card lists (one warp per card), and accumulates the
// output column in registers.  Each output column is written exactly once, in
// a fixed order: no atomics, deterministic.
//
// FP32 path: all sums and the per-hand combination in float-float (TwoSum /
// TwoProd, each float carried with its rounding error), rounded once at the
// end.  FP64 path: plain doubles (the stopping gap).
#include <algorithm>

#include "egt_internal.cuh"

namespace egt {
namespace {

struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  // TwoSum of the high parts, low parts folded into the error, renormalised
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  err = __fadd_rn(err, __fadd_rn(a.lo, b.lo));
  const float hi = __fadd_rn(s, err);
  const float lo = __fsub_rn(err, __fsub_rn(hi, s));
  return {hi, lo};
}

template <typename T>
struct Arith;

template <>
struct Arith<float> {
  using Acc = FF;
  static __device__ __forceinline__ Acc zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ Acc from(float x) { return {x, 0.f}; }
  static __device__ __forceinline__ Acc add(Acc a, Acc b) { return ff_add(a, b); }
  static __device__ __forceinline__ Acc sub(Acc a, Acc b) { return ff_add(a, {-b.hi, -b.lo}); }
  // c * a with the product's rounding error kept (TwoProd by fma)
  static __device__ __forceinline__ Acc scale(float c, Acc a) {
    const float p = __fmul_rn(c, a.hi);
    const float e = __fmaf_rn(c, a.hi, -p);
    return ff_add({p, 0.f}, {e, __fmul_rn(c, a.lo)});
  }
  static __device__ __forceinline__ float round(Acc a) { return __fadd_rn(a.hi, a.lo); }
  static __device__ __forceinline__ Acc shfl_up(Acc a, int d) {
    return {__shfl_up_sync(0xffffffffu, a.hi, d), __shfl_up_sync(0xffffffffu, a.lo, d)};
  }
  static __device__ __forceinline__ Acc shfl(Acc a, int src) {
    return {__shfl_sync(0xffffffffu, a.hi, src), __shfl_sync(0xffffffffu, a.lo, src)};
  }
};

template <>
struct Arith<double> {
  using Acc = double;
  static __device__ __forceinline__ Acc zero() { return 0.0; }
  static __device__ __forceinline__ Acc from(double x) { return x; }
  static __device__ __forceinline__ Acc add(Acc a, Acc b) { return a + b; }
  static __device__ __forceinline__ Acc sub(Acc a, Acc b) { return a - b; }
  static __device__ __forceinline__ Acc scale(double c, Acc a) { return c * a; }
  static __device__ __forceinline__ double round(Acc a) { return a; }
  static __device__ __forceinline__ Acc shfl_up(Acc a, int d) {
    return __shfl_up_sync(0xffffffffu, a, d);
  }
  static __device__ __forceinline__ Acc shfl(Acc a, int src) {
    return __shfl_sync(0xffffffffu, a, src);
  }
};

template <typename T>
__device__ __forceinline__ typename Arith<T>::Acc warp_incl_scan(typename Arith<T>::Acc v,
                                                                 int lane) {
  using A = Arith<T>;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    auto o = A::shfl_up(v, d);
    if (lane >= d) v = A::add(v, o);
  }
  return v;
}

constexpr int kMaxHandsPerThread = 8;   // ld <= 2048 with 256 threads

template <typename T>
__device__ __forceinline__ const T* ranges(const DevGame& g, int p);
template <>
__device__ __forceinline__ const float* ranges<float>(const DevGame& g, int p) { return g.r[p]; }
template <>
__device__ __forceinline__ const double* ranges<double>(const DevGame& g, int p) { return g.r64[p]; }
template <typename T>
__device__ __forceinline__ const T* ranges_z(const DevGame& g, int p);
template <>
__device__ __forceinline__ const float* ranges_z<float>(const DevGame& g, int p) { return g.rz[p]; }
template <>
__device__ __forceinline__ const double* ranges_z<double>(const DevGame& g, int p) {
  return g.rz64[p];
}
template <typename T>
__device__ __forceinline__ T term_coef(const DevTerms& t, int e);
template <>
__device__ __forceinline__ float term_coef<float>(const DevTerms& t, int e) { return t.coef[e]; }
template <>
__device__ __forceinline__ double term_coef<double>(const DevTerms& t, int e) {
  return t.coef64[e];
}

template <typename TIn, typename T>
__global__ void __launch_bounds__(kGradThreads)
    grad_kernel(DevGame g, int player, const TIn* __restrict__ in, T* __restrict__ out) {
  using A = Arith<T>;
  using Acc = typename A::Acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Acc warp_tot[kGradThreads / 32];

  const int ld = g.ld, H = g.H, opp = 1 - player;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kGradThreads / 32;
  T* w = reinterpret_cast<T*>(smem_raw);              // [ld]
  Acc* P = reinterpret_cast<Acc*>(w + ld);            // [ld + 1] exclusive prefix in strength order
  const int lstride = g.lmax + 1;
  Acc* PC = P + (ld + 1);                             // [n_slots][lmax + 1] per-card exclusive prefix

  const int s = blockIdx.x;
  const DevTerms tm = g.terms[player];
  const int e0 = tm.ptr[s], e1 = tm.ptr[s + 1];
  const T* __restrict__ r_opp = ranges<T>(g, opp);

  Acc acc[kMaxHandsPerThread];
#pragma unroll
  for (int k = 0; k < kMaxHandsPerThread; ++k) acc[k] = A::zero();

  const int K = (ld + kGradThreads - 1) / kGradThreads;   // raking chunk
  const int k0 = min(tid * K, ld), k1 = min(k0 + K, ld);

  for (int e = e0; e < e1; ++e) {
    const int os = tm.opp_seq[e];
    const int kind = tm.kind[e];
    const T coef = term_coef<T>(tm, e);
    const TIn* __restrict__ col = in + (size_t)os * ld;
    for (int h = tid; h < ld; h += kGradThreads)
      w[h] = h < H ? r_opp[h] * (T)col[h] : T(0);
    __syncthreads();

    // exclusive prefix over ascending strength: P[i] = sum_{k < i} w[k], P[ld] = total
    Acc loc = A::zero();
    for (int i = k0; i < k1; ++i) loc = A::add(loc, A::from(w[i]));
    Acc inc = warp_incl_scan<T>(loc, lane);
    if (lane == 31) warp_tot[warp] = inc;
    Acc lane_excl = A::shfl_up(inc, 1);
    if (lane == 0) lane_excl = A::zero();
    __syncthreads();
    Acc base = A::zero();
    for (int q = 0; q < warp; ++q) base = A::add(base, warp_tot[q]);
    Acc run = A::add(base, lane_excl);
    for (int i = k0; i < k1; ++i) {
      P[i] = run;
      run = A::add(run, A::from(w[i]));
    }
    if (k0 < ld && k1 == ld) P[ld] = run;

    // per-card exclusive prefixes, one warp per card slot
    for (int c = warp; c < g.n_slots; c += kWarps) {
      const int len = g.card_len[c];
      const uint16_t* lst = g.card_hands + (size_t)c * g.lmax;
      const T v0 = lane < len ? w[lst[lane]] : T(0);
      const T v1 = lane + 32 < len ? w[lst[lane + 32]] : T(0);
      const Acc a0 = warp_incl_scan<T>(A::from(v0), lane);
      const Acc t0 = A::shfl(a0, 31);
      const Acc a1 = A::add(warp_incl_scan<T>(A::from(v1), lane), t0);
      Acc* pc = PC + (size_t)c * lstride;
      if (lane == 0) pc[0] = A::zero();
      if (lane < len) pc[lane + 1] = a0;
      if (lane + 32 < len) pc[lane + 33] = a1;
    }
    __syncthreads();

    const Acc W = P[ld];
#pragma unroll
    for (int k = 0; k < kMaxHandsPerThread; ++k) {
      const int h = tid + k * kGradThreads;
      if (h >= ld) break;
      const uchar2 cc = g.hcard[h];
      const Acc* pc0 = PC + (size_t)cc.x * lstride;
      const Acc* pc1 = PC + (size_t)cc.y * lstride;
      const Acc C0 = pc0[g.card_len[cc.x]];
      const Acc C1 = pc1[g.card_len[cc.y]];
      Acc val;
      if (kind == 0) {
        val = A::sub(A::sub(W, C0), C1);
        if (g.hand_size == 2) val = A::add(val, A::from(w[h]));
      } else {
        const ushort2 gr = g.grp[h];
        const uchar4 cp = g.cpos[h];
        const Acc lt = A::sub(A::sub(P[gr.x], pc0[cp.x]), pc1[cp.z]);
        const Acc gt = A::sub(A::sub(A::sub(W, P[gr.y]), A::sub(C0, pc0[cp.y])),
                              A::sub(C1, pc1[cp.w]));
        val = A::sub(gt, lt);
      }
      acc[k] = A::add(acc[k], A::scale(coef, val));
    }
    __syncthreads();   // w / P / PC are rewritten by the next terminal
  }

  const T* __restrict__ rz = ranges_z<T>(g, player);
  T* o = out + (size_t)s * ld;
#pragma unroll
  for (int k = 0; k < kMaxHandsPerThread; ++k) {
    const int h = tid + k * kGradThreads;
    if (h >= ld) break;
    o[h] = h < H ? rz[h] * A::round(acc[k]) : T(0);
  }
}

template <typename T>
size_t smem_for(const DevGame& g) {
  using Acc = typename Arith<T>::Acc;
  return (size_t)g.ld * sizeof(T) + (size_t)(g.ld + 1) * sizeof(Acc) +
         (size_t)g.n_slots * (g.lmax + 1) * sizeof(Acc);
}

}  // namespace

size_t grad_smem_bytes(const DevGame& g, bool f64) {
  return f64 ? smem_for<double>(g) : smem_for<float>(g);
}

template <typename TIn, typename T>
void launch_grad(const DevGame& g, int player, const TIn* in, T* out, cudaStream_t st) {
  const size_t smem = smem_for<T>(g);
  static int limit = 0;   // one process-wide opt-in per instantiation
  if (limit == 0) limit = opt_in_dynamic_smem((const void*)grad_kernel<TIn, T>);
  grad_kernel<TIn, T><<<g.tpx[player].S, kGradThreads, smem, st>>>(g, player, in, out);
}

template void launch_grad<float, float>(const DevGame&, int, const float*, float*, cudaStream_t);
template void launch_grad<double, double>(const DevGame&, int, const double*, double*,
                                          cudaStream_t);
template void launch_grad<float, double>(const DevGame&, int, const float*, double*,
                                         cudaStream_t);

}  // namespace egt
