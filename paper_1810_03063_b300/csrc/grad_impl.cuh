// Gradient product body shared by the standalone kernels and the solver engine.
//
// Sec. 3: every EGT step needs grad f = A y and grad phi = A^T x.  For a
// terminal b and an output hand h (Sec. 7 payoffs, chance r1 r2 / Z):
//
//   fold:     r_me(h)/Z * u_b * sum_{h' disjoint from h} w(h')
//   showdown: r_me(h)/Z * c_b * (sum_{disjoint, stronger} w - sum_{disjoint, weaker} w)
//
// with w = r_opp (.) in[sigma_opp(b)].  Disjoint sums use card-removal
// inclusion-exclusion (total - per-card totals of h's cards + w(h), the only
// hand holding both cards being h itself); weaker / stronger sums use exclusive
// prefix sums over the hands in ascending strength, up to h's tie group start /
// from its end, minus the same prefix over each of h's cards' hand lists.
//
// One CTA (512 threads) per terminal writes that terminal's contribution column
// coef_b x (sum) for every hand; the consumer of the product (the smoothed best
// response, the FP64 best response, or the combine kernel of egt_grad) adds the
// one or two contributions of a sequence in terminal order and multiplies by
// r_me / Z while it loads them.
//
// Arithmetic: each w is put in 63-bit fixed point, an int64 at a per-column
// power-of-two scale 2^ex that maps the column's largest |w| below 2^52 (so a
// sum of up to 2048 terms stays below 2^63), and every prefix sum, per-card
// correction and tie-aware difference is an exact integer operation:
// deterministic in any order, on the full-rate integer pipes, and the same bits
// whichever items or threads form it.  For FP32 inputs w 2^ex is formed from
// the range split in two FP32 parts, r = r_hi + r_lo: p = r_hi a exactly as an
// FMA product and its error, plus r_lo a, with a = y 2^ex (exact), each part
// rounded to an integer; so the fixed-point w is within 2^-47 |w 2^ex| + 1.5 of
// the exact one (ranges below 2^-60, where a could overflow, take the same
// product in FP64).  FP64 inputs (the public FP64 product) use w = r y in
// FP64.  From the same sums the CTA can emit an FP32 contribution (the path of
// every EGT step) and an FP64 one (the stopping residual): the int64 sum
// rounded once to each format; asking for the FP64 one does not change the
// FP32 one.
#pragma once
#include <climits>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "egt_internal.cuh"

namespace egt {

constexpr int kItemThreads = 512;     // threads of a CTA of the engine and of the kernels

namespace gradimpl {

// Bit-level helpers that also compile for the host: the arithmetic functions below
// (w 2^ex in fixed point, rounding back to FP32 / FP64) are checked on the CPU
// against rational arithmetic.
__host__ __device__ __forceinline__ int clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}
__host__ __device__ __forceinline__ int clz32(unsigned x) {
#ifdef __CUDA_ARCH__
  return __clz((int)x);
#else
  return x ? __builtin_clz(x) : 32;
#endif
}
__host__ __device__ __forceinline__ unsigned long long f64_bits(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}
__host__ __device__ __forceinline__ double bits_f64(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, 8);
  return x;
#endif
}
__host__ __device__ __forceinline__ unsigned f32_bits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  unsigned b;
  std::memcpy(&b, &x, 4);
  return b;
#endif
}
__host__ __device__ __forceinline__ float bits_f32(unsigned b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float x;
  std::memcpy(&x, &b, 4);
  return x;
#endif
}

// fixed point: one signed int64 (w 2^ex rounded to an integer)
struct Fx {
  long long v0;
};

__host__ __device__ __forceinline__ Fx fx_zero() { return {0}; }
__host__ __device__ __forceinline__ Fx fx_add(Fx a, Fx b) { return {a.v0 + b.v0}; }
__host__ __device__ __forceinline__ Fx fx_sub(Fx a, Fx b) { return {a.v0 - b.v0}; }
__device__ __forceinline__ Fx fx_shfl_up(Fx a, int d) { return {__shfl_up_sync(0xffffffffu, a.v0, d)}; }
__device__ __forceinline__ Fx fx_shfl(Fx a, int src) { return {__shfl_sync(0xffffffffu, a.v0, src)}; }
__device__ __forceinline__ Fx fx_scan(Fx v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    Fx o = fx_shfl_up(v, d);
    if (lane >= d) v = fx_add(v, o);
  }
  return v;
}
// inclusive scan within each 16-lane half of the warp (sl = lane & 15)
__device__ __forceinline__ Fx fx_scan16(Fx v, int sl) {
#pragma unroll
  for (int d = 1; d < 16; d <<= 1) {
    const Fx o = {__shfl_up_sync(0xffffffffu, v.v0, d, 16)};
    if (sl >= d) v = fx_add(v, o);
  }
  return v;
}

// 2^e as float (e in [-126, 127]) / double (e in [-1022, 1023]), from the exponent field
__host__ __device__ __forceinline__ float pow2f(int e) { return bits_f32((unsigned)(e + 127) << 23); }
__host__ __device__ __forceinline__ double pow2d(int e) {
  return bits_f64((unsigned long long)(e + 1023) << 52);
}

// round to the nearest integer, ties to even (the default rounding mode on the host)
__host__ __device__ __forceinline__ long long rint_ll(float x) {
#ifdef __CUDA_ARCH__
  return __float2ll_rn(x);
#else
  return std::llrint(x);
#endif
}
__host__ __device__ __forceinline__ long long rint_ll(double x) {
#ifdef __CUDA_ARCH__
  return __double2ll_rn(x);
#else
  return std::llrint(x);
#endif
}
__host__ __device__ __forceinline__ float fma32(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}

// An upper bound on floor(log2 |r y|) for FP32 y from the two exponents alone (the
// significand product is below 4, so the bound is the true value or one more);
// INT_MIN when r y = 0.  Enough to choose a column's fixed-point scale (scale_of)
// without forming the products twice.
__host__ __device__ __forceinline__ int lg_bound(double r, float y) {
  const unsigned long long rb = f64_bits(r);
  const unsigned yb = f32_bits(y);
  const int er = (int)((rb >> 52) & 0x7ffull), ey = (int)((yb >> 23) & 0xffu);
  const unsigned long long mr = rb & ((1ull << 52) - 1);
  const unsigned my = yb & 0x7fffffu;
  if ((er == 0 && mr == 0) || (ey == 0 && my == 0)) return INT_MIN;
  const int lr = er ? er - 1023 : (63 - clz64(mr)) - 1074;   // floor(log2 |r|), subnormals too
  const int ly = ey ? ey - 127 : (31 - clz32(my)) - 149;
  return lr + ly + 1;
}

// floor(log2 |w|) of an FP64 value (INT_MIN when 0), subnormals included
__host__ __device__ __forceinline__ int lg64(double w) {
  const unsigned long long b = f64_bits(w);
  const int e = (int)((b >> 52) & 0x7ffull);
  const unsigned long long m = b & ((1ull << 52) - 1);
  if (e == 0 && m == 0) return INT_MIN;
  return e ? e - 1023 : (63 - clz64(m)) - 1074;
}

// The scale exponent of a column whose largest |w| has floor(log2) <= maxlg: |w| 2^ex <
// 2^52.  Clamped to [-252, 252] (a column below 2^-201 or above 2^303 keeps a coarser
// scale; its sums stay exact at that scale), where 2^ex and 2^-ex are each a product of
// two normal FP32 powers of two.
__host__ __device__ __forceinline__ int scale_of(int maxlg) {
  if (maxlg == INT_MIN) return 0;
  const int ex = 51 - maxlg;
  return ex < -252 ? -252 : (ex > 252 ? 252 : ex);
}

// 2^ex as two float factors, each a normal power of two (|ex| <= 252)
struct Pow2f {
  float a, b;
};
__host__ __device__ __forceinline__ Pow2f pow2f_split(int ex) {
  const int e1 = ex < -126 ? -126 : (ex > 127 ? 127 : ex);
  return {pow2f(e1), pow2f(ex - e1)};
}

// r y 2^ex as an integer, FP32 y, r = r64 = r_hi + r_lo with r_hi = RN32(r64) and r_lo =
// RN32(r64 - r_hi); s = pow2f_split(ex).  With a = y 2^ex (exact unless it underflows,
// where the term is below 2^-126 and rounds to 0 anyway): r_hi a = p + e exactly (FMA),
// r_lo a is rounded once (relative 2^-24 of a term at most 2^-24 |r a|), and each part
// is rounded to an integer; with |r - r_hi - r_lo| <= 2^-48 |r|, |result - r y 2^ex| <=
// 2^-47 |r y 2^ex| + 1.5.  A range below
// 2^-60 (a could overflow there) takes w = r64 y in FP64 instead.
__host__ __device__ __forceinline__ long long fx_of(double r64, float r_hi, float r_lo, float y, Pow2f s,
                                                   int ex) {
  if (!(r_hi >= 1.0f / 1152921504606846976.0f)) {            // r_hi < 2^-60 (0 included)
    if (r64 == 0.0) return 0;
    return rint_ll(r64 * (double)y * pow2d(ex));
  }
  const float a = (y * s.a) * s.b;
  const float p = r_hi * a;
  const float e = fma32(r_hi, a, -p);
  const float q = r_lo * a;
  return rint_ll(p) + rint_ll(e) + rint_ll(q);
}

// r y 2^ex as an integer, FP64 y: w = r y rounded once in FP64 (relative 2^-53)
__host__ __device__ __forceinline__ long long fx_of64(double r64, double y, int ex) {
  return rint_ll(r64 * y * pow2d(ex));
}

// FP32 and FP64 values of a fixed-point sum S 2^-ex: S rounded once to each format (to
// nearest, ties to even), then scaled by the power of two.  Two forms with the same
// results.  fx_to_f32_f64_conv: the conversion instructions and a power-of-two scale
// (exact for a normal result; a subnormal result is rounded a second time).
// fx_to_f32_f64: where both results are normal (every sum of a product in practice)
// the roundings are integer operations on the magnitude shifted to bit 63 and the scale
// goes into the exponent fields, with no FP64 pipe (a narrow one on this part) and no
// conversion unit; otherwise the first form.  Measured: the integer form is faster in
// items that run back to back on a CTA (batches, merged items), the conversion form
// where each item has a CTA of its own (the one-game driver's full-deck products).
__host__ __device__ __forceinline__ void fx_to_f32_f64_conv(Fx a, int ex, float& r32, double& r64) {
#ifdef __CUDA_ARCH__
  const float f = __ll2float_rn(a.v0);
  const double d = __ll2double_rn(a.v0);
#else
  const float f = (float)a.v0;
  const double d = (double)a.v0;
#endif
  const Pow2f s = pow2f_split(-ex);
  r32 = (f * s.a) * s.b;
  r64 = d * pow2d(-ex);
}

__host__ __device__ __forceinline__ void fx_to_f32_f64(Fx a, int ex, float& r32, double& r64) {
  const long long S = a.v0;
  if (S == 0) {
    r32 = 0.f;
    r64 = 0.0;
    return;
  }
  const bool neg = S < 0;
  const unsigned long long u = neg ? 0ull - (unsigned long long)S : (unsigned long long)S;
  const int lz = clz64(u);
  const unsigned long long T = u << lz;                      // leading bit at bit 63
  const int e = 63 - lz - ex;                                // exponent of the leading bit
  unsigned long long q = T >> 11;                            // FP64: 53 bits, round on bit 10
  q += ((T >> 10) & 1ull) & (unsigned long long)(((T & 0x3ffull) != 0) | (q & 1ull));
  int e64 = e;
  if (q >> 53) {
    q >>= 1;
    ++e64;
  }
  unsigned long long p = T >> 40;                            // FP32: 24 bits, round on bit 39
  p += ((T >> 39) & 1ull) & (unsigned long long)(((T & ((1ull << 39) - 1ull)) != 0) | (p & 1ull));
  int e32 = e;
  if (p >> 24) {
    p >>= 1;
    ++e32;
  }
  if (e64 + 1023 < 1 || e64 + 1023 > 2046 || e32 + 127 < 1 || e32 + 127 > 254) {
    fx_to_f32_f64_conv(a, ex, r32, r64);
    return;
  }
  r64 = bits_f64(((unsigned long long)neg << 63) | ((unsigned long long)(e64 + 1023) << 52) |
                 (q & ((1ull << 52) - 1ull)));
  r32 = bits_f32(((unsigned)neg << 31) | ((unsigned)(e32 + 127) << 23) | (unsigned)(p & 0x7fffffull));
}

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

constexpr int kMaxLd = 1536;

}  // namespace gradimpl

// CTA barrier of an item run by kThreads threads: the whole CTA, or a warp half with
// its own named barrier `bar` (two items side by side).
template <int kThreads>
__device__ __forceinline__ void item_sync(int bar) {
  if (kThreads == kItemThreads) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(kThreads) : "memory");
}

// Shared memory of one terminal item: F (w in fixed point), P, PC, warp maxima,
// warp totals (without the staged tables).
__host__ __device__ inline size_t grad_item_smem(const DevGame& g) {
  using gradimpl::align16;
  const size_t fx = sizeof(gradimpl::Fx);
  size_t b = align16((size_t)g.ld * fx);
  b += align16((size_t)(g.ld + 1) * fx);
  b += align16((size_t)g.n_slots * pc_stride(g.lmax) * fx);
  b += 16 * sizeof(int) + 16 * fx + 16;
  return align16(b);
}

// Per-game tables the product reads for every terminal, staged once in shared memory.
struct GradTab {
  const uint4* hinfo;          // [ld] per-hand flat indices (see DevGame::hinfo)
  const int* card_len;         // [n_slots]
  const uint16_t* card_hands;  // [n_slots][lmax]
  const double* r64[2];        // [ld] normalised ranges of both players
  const float* rhi[2];         // [ld] their FP32 split r = r_hi + r_lo (DevGame::r, DevGame::rlo)
  const float* rlo[2];
};

__host__ __device__ inline size_t grad_tab_bytes(const DevGame& g) {
  using gradimpl::align16;
  return align16((size_t)g.ld * sizeof(uint4)) + align16((size_t)g.n_slots * sizeof(int)) +
         align16((size_t)g.n_slots * g.lmax * sizeof(uint16_t)) + 2 * align16((size_t)g.ld * sizeof(double)) +
         4 * align16((size_t)g.ld * sizeof(float));
}

// Copy the tables into dst (all threads of the CTA; the caller synchronises before use).
__device__ inline GradTab stage_grad_tab(const DevGame& g, unsigned char* dst) {
  using gradimpl::align16;
  uint4* hi = reinterpret_cast<uint4*>(dst);
  unsigned char* p = dst + align16((size_t)g.ld * sizeof(uint4));
  int* cl = reinterpret_cast<int*>(p);
  p += align16((size_t)g.n_slots * sizeof(int));
  uint16_t* ch = reinterpret_cast<uint16_t*>(p);
  p += align16((size_t)g.n_slots * g.lmax * sizeof(uint16_t));
  double* r0 = reinterpret_cast<double*>(p);
  double* r1 = r0 + align16((size_t)g.ld * sizeof(double)) / sizeof(double);
  p += 2 * align16((size_t)g.ld * sizeof(double));
  const size_t fs = align16((size_t)g.ld * sizeof(float)) / sizeof(float);
  float* h0 = reinterpret_cast<float*>(p);
  float* h1 = h0 + fs;
  float* l0 = h1 + fs;
  float* l1 = l0 + fs;
  for (int i = threadIdx.x; i < g.ld; i += blockDim.x) {
    hi[i] = g.hinfo[i];
    r0[i] = g.r64[0][i];
    r1[i] = g.r64[1][i];
    h0[i] = g.r[0][i];
    h1[i] = g.r[1][i];
    l0[i] = g.rlo[0][i];
    l1[i] = g.rlo[1][i];
  }
  for (int i = threadIdx.x; i < g.n_slots; i += blockDim.x) cl[i] = g.card_len[i];
  for (int i = threadIdx.x; i < g.n_slots * g.lmax; i += blockDim.x) ch[i] = g.card_hands[i];
  GradTab t;
  t.hinfo = hi;
  t.card_len = cl;
  t.card_hands = ch;
  t.r64[0] = r0;
  t.r64[1] = r1;
  t.rhi[0] = h0;
  t.rhi[1] = h1;
  t.rlo[0] = l0;
  t.rlo[1] = l1;
  return t;
}

// Product item `item` of player `player`'s grouping (DevTerms): terminal `item` alone,
// or with `merged` the showdown and / or fold terminal of the item-th opponent column
// (DevTerms::col).  For each terminal e of the item, c32[e][h] and / or c64[e][h]
// (either may be NULL) = coef_e x the
// card-removal / strength sum of w = r_opp (.) in[sigma_opp], without the r_me / Z factor.
// The exact sums are formed once for both terminals: the fold needs only the column
// total and the per-card totals, the showdown the strength prefix and the per-card
// prefixes as well (whose last entries are the per-card totals), so a fold that has no
// showdown beside it skips the prefixes.  The sums are exact integers, so the results
// do not depend on which terminals share an item, nor on kThreads: the whole CTA, or
// the warp half starting at warp first_warp with named barrier `bar`.  `in` is read
// through L2 (it may have been written earlier in the same launch by other CTAs).
template <typename TIn, int kThreads = kItemThreads>
__device__ inline void prod_item(const DevGame& g, const GradTab& tb, int player, int item, bool merged,
                                 const TIn* __restrict__ in, float* __restrict__ c32,
                                 double* __restrict__ c64, unsigned char* smem, int first_warp = 0,
                                 int bar = 0) {
  using namespace gradimpl;
  constexpr int kMaxHandsPerThread = (kMaxLd + kThreads - 1) / kThreads;
  constexpr int kWarps = kThreads / 32;
  const int ld = g.ld, H = g.H, opp = 1 - player;
  const int tid = threadIdx.x - first_warp * 32, lane = threadIdx.x & 31, warp = tid >> 5;
  const int lstride = pc_stride(g.lmax);

  Fx* F = reinterpret_cast<Fx*>(smem);
  Fx* P = F + ld;                                                          // [ld + 1]
  Fx* PC = reinterpret_cast<Fx*>(reinterpret_cast<unsigned char*>(P) + align16((size_t)(ld + 1) * sizeof(Fx)));
  int* wmax = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(PC) +
                                     align16((size_t)g.n_slots * lstride * sizeof(Fx)));
  Fx* wtot = reinterpret_cast<Fx*>(wmax + 16);

  // (selects instead of runtime indices into struct arrays, which would go to local memory)
  const DevTerms tm = player ? g.terms[1] : g.terms[0];
  const double* __restrict__ r_opp = opp ? tb.r64[1] : tb.r64[0];
  const float* __restrict__ rhi_opp = opp ? tb.rhi[1] : tb.rhi[0];
  const float* __restrict__ rlo_opp = opp ? tb.rlo[1] : tb.rlo[0];
  // the item's terminals and opponent column (loads independent of each other: the column
  // is not kept waiting for the terminals' kinds)
  int os, e_sd, e_fold;
  if (merged) {
    const int4 c = tm.col[item];
    e_sd = c.x;
    e_fold = c.y;
    os = c.z;
  } else {
    os = tm.opp_seq[item];
    const bool showdown = tm.kind[item] != 0;
    e_sd = showdown ? item : -1;
    e_fold = showdown ? -1 : item;
  }
  const bool sd = e_sd >= 0;
  const TIn* col = in + (size_t)os * ld;
  // the coefficients are first read after the sums: fetch their lines into L1 now
  if (tid == 0) {
    if (sd) {
      asm volatile("prefetch.global.L1 [%0];" ::"l"(tm.coef + e_sd));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(tm.coef64 + e_sd));
    }
    if (e_fold >= 0) {
      asm volatile("prefetch.global.L1 [%0];" ::"l"(tm.coef + e_fold));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(tm.coef64 + e_fold));
    }
  }

  // pass 1: all of this thread's inputs loaded at once, the column's largest exponent of
  // |w| (for FP32 inputs an upper bound from the exponents, at most one too large)
  TIn y[kMaxHandsPerThread];
#pragma unroll
  for (int k = 0; k < kMaxHandsPerThread; ++k) {
    const int h = tid + k * kThreads;
    y[k] = h < H ? __ldcg(col + h) : TIn(0);
  }
  int mlg = INT_MIN;
#pragma unroll
  for (int k = 0; k < kMaxHandsPerThread; ++k) {
    const int h = tid + k * kThreads;
    if (h < ld) {
      if constexpr (std::is_same<TIn, float>::value) mlg = max(mlg, lg_bound(r_opp[h], y[k]));
      else mlg = max(mlg, lg64(r_opp[h] * y[k]));   // (FP64 y: the rounded product's exact lg)
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) mlg = max(mlg, __shfl_xor_sync(0xffffffffu, mlg, d));
  if (lane == 0) wmax[warp] = mlg;
  item_sync<kThreads>(bar);
  int M = INT_MIN;
#pragma unroll
  for (int q = 0; q < kWarps; ++q) M = max(M, wmax[q]);
  const int ex = scale_of(M);
  const Pow2f s2 = pow2f_split(ex);
  // pass 2: fixed point
#pragma unroll
  for (int k = 0; k < kMaxHandsPerThread; ++k) {
    const int h = tid + k * kThreads;
    if (h < ld) {
      if constexpr (std::is_same<TIn, float>::value) F[h] = {fx_of(r_opp[h], rhi_opp[h], rlo_opp[h], y[k], s2, ex)};
      else F[h] = {fx_of64(r_opp[h], y[k], ex)};
    }
  }
  item_sync<kThreads>(bar);

  // the column total W; with a showdown the exclusive prefix over ascending strength:
  // P[i] = sum_{k < i} w[k], P[ld] = W
  const int K = (ld + kThreads - 1) / kThreads;   // raking chunk
  const int k0 = min(tid * K, ld), k1 = min(k0 + K, ld);
  Fx loc = fx_zero();
  for (int i = k0; i < k1; ++i) loc = fx_add(loc, F[i]);
  const Fx inc = fx_scan(loc, lane);
  if (lane == 31) wtot[warp] = inc;
  item_sync<kThreads>(bar);
  if (sd) {
    Fx run = fx_shfl_up(inc, 1);
    if (lane == 0) run = fx_zero();
#pragma unroll
    for (int q = 0; q < kWarps; ++q)   // (unrolled: the loads issue together)
      if (q < warp) run = fx_add(run, wtot[q]);
    for (int i = k0; i < k1; ++i) {
      P[i] = run;
      run = fx_add(run, F[i]);
    }
    if (k0 < ld && k1 == ld) P[ld] = run;
  }

  // per-card sums: a card slot per 16-lane half warp, four consecutive list entries (at
  // most 64) per lane, summed serially; with a showdown one half-warp scan gives the
  // exclusive prefixes (the last one is the card's total), else a half-warp sum gives
  // the total alone, stored where the prefixes would end
  {
    const int sub = lane >> 4, sl = lane & 15, i0 = 4 * sl;
    for (int c0 = 2 * warp; c0 < g.n_slots; c0 += 2 * kWarps) {   // (warp-uniform trip count)
      const int c = c0 + sub;
      const bool ok = c < g.n_slots;
      const int len = ok ? tb.card_len[c] : 0;
      const uint16_t* lst = tb.card_hands + (size_t)(ok ? c : 0) * g.lmax;
      Fx a[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) a[j] = i0 + j < len ? F[lst[i0 + j]] : fx_zero();
#pragma unroll
      for (int j = 1; j < 4; ++j) a[j] = fx_add(a[j - 1], a[j]);
      Fx* pc = PC + (size_t)(ok ? c : 0) * lstride;
      const Fx inc4 = fx_scan16(a[3], sl);
      if (sd) {
        const Fx before = fx_sub(inc4, a[3]);
        if (ok && sl == 0) pc[0] = fx_zero();
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (ok && i0 + j < len) pc[pc_pad(i0 + j + 1)] = fx_add(before, a[j]);
      } else if (ok && sl == 15) {
        pc[pc_pad(len)] = inc4;   // the card's total (lane 15 holds the sum of the list)
      }
    }
  }
  item_sync<kThreads>(bar);
  Fx W;
  if (sd) {
    W = P[ld];
  } else {
    W = fx_zero();
#pragma unroll
    for (int q = 0; q < kWarps; ++q) W = fx_add(W, wtot[q]);
  }

  // the showdown terminal's contributions, then the fold's (one copy of the conversion)
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    const int e = pass == 0 ? e_sd : e_fold;
    if (e < 0) continue;
    const float coef32 = tm.coef[e];
    const double coef64 = tm.coef64[e];
#pragma unroll
    for (int k = 0; k < kMaxHandsPerThread; ++k) {
      const int h = tid + k * kThreads;
      if (h >= ld) break;
      const uint4 hi = tb.hinfo[h];
      const Fx C0 = PC[hi.z & 0xffffu];
      const Fx C1 = PC[hi.w >> 16];
      Fx val;
      if (pass == 1) {
        val = fx_sub(fx_sub(W, C0), C1);
        if (g.hand_size == 2) val = fx_add(val, F[h]);
      } else {
        const Fx lt = fx_sub(fx_sub(P[hi.x & 0xffffu], PC[hi.y & 0xffffu]), PC[hi.z >> 16]);
        const Fx gt = fx_sub(fx_sub(fx_sub(W, P[hi.x >> 16]), fx_sub(C0, PC[hi.y >> 16])),
                             fx_sub(C1, PC[hi.w & 0xffffu]));
        val = fx_sub(gt, lt);
      }
      const bool live = h < H;
      float v32;
      double v64;
      fx_to_f32_f64(val, ex, v32, v64);
      if (c32 != nullptr) c32[(size_t)e * ld + h] = live ? coef32 * v32 : 0.f;
      if (c64 != nullptr) c64[(size_t)e * ld + h] = live ? coef64 * v64 : 0.0;
    }
  }
  item_sync<kThreads>(bar);   // shared memory is reused by the caller's next item
}

// Contribution of terminal e alone (the standalone product kernels, one CTA per terminal).
template <typename TIn, int kThreads = kItemThreads>
__device__ inline void term_item(const DevGame& g, const GradTab& tb, int player, int e,
                                 const TIn* __restrict__ in, float* __restrict__ c32,
                                 double* __restrict__ c64, unsigned char* smem, int first_warp = 0,
                                 int bar = 0) {
  prod_item<TIn, kThreads>(g, tb, player, e, false, in, c32, c64, smem, first_warp, bar);
}

// One terminal per item with the strength and per-card prefixes formed for every
// terminal kind (the one-game driver's product items: a fold item is never the longest
// of its phase there, and this body keeps that driver's code smaller).  Same results
// as prod_item.
template <typename TIn, int kThreads = kItemThreads>
__device__ inline void term_item_whole(const DevGame& g, const GradTab& tb, int player, int e,
                                 const TIn* __restrict__ in, float* __restrict__ c32,
                                 double* __restrict__ c64, unsigned char* smem, int first_warp = 0,
                                 int bar = 0) {
  using namespace gradimpl;
  constexpr int kMaxHandsPerThread = (kMaxLd + kThreads - 1) / kThreads;
  constexpr int kWarps = kThreads / 32;
  const int ld = g.ld, H = g.H, opp = 1 - player;
  const int tid = threadIdx.x - first_warp * 32, lane = threadIdx.x & 31, warp = tid >> 5;
  const int lstride = pc_stride(g.lmax);

  Fx* F = reinterpret_cast<Fx*>(smem);
  Fx* P = F + ld;                                                          // [ld + 1]
  Fx* PC = reinterpret_cast<Fx*>(reinterpret_cast<unsigned char*>(P) + align16((size_t)(ld + 1) * sizeof(Fx)));
  int* wmax = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(PC) +
                                     align16((size_t)g.n_slots * lstride * sizeof(Fx)));
  Fx* wtot = reinterpret_cast<Fx*>(wmax + 16);

  // (selects instead of runtime indices into struct arrays, which would go to local memory)
  const DevTerms tm = player ? g.terms[1] : g.terms[0];
  const double* __restrict__ r_opp = opp ? tb.r64[1] : tb.r64[0];
  const float* __restrict__ rhi_opp = opp ? tb.rhi[1] : tb.rhi[0];
  const float* __restrict__ rlo_opp = opp ? tb.rlo[1] : tb.rlo[0];
  const int os = tm.opp_seq[e];
  const int kind = tm.kind[e];
  const float coef32 = tm.coef[e];
  const double coef64 = tm.coef64[e];
  const TIn* col = in + (size_t)os * ld;

  // pass 1: all of this thread's inputs loaded at once, the column's largest exponent of
  // |w| (for FP32 inputs an upper bound from the exponents, at most one too large)
  TIn y[kMaxHandsPerThread];
#pragma unroll
  for (int k = 0; k < kMaxHandsPerThread; ++k) {
    const int h = tid + k * kThreads;
    y[k] = h < H ? __ldcg(col + h) : TIn(0);
  }
  int mlg = INT_MIN;
#pragma unroll
  for (int k = 0; k < kMaxHandsPerThread; ++k) {
    const int h = tid + k * kThreads;
    if (h < ld) {
      if constexpr (std::is_same<TIn, float>::value) mlg = max(mlg, lg_bound(r_opp[h], y[k]));
      else mlg = max(mlg, lg64(r_opp[h] * y[k]));   // (FP64 y: the rounded product's exact lg)
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) mlg = max(mlg, __shfl_xor_sync(0xffffffffu, mlg, d));
  if (lane == 0) wmax[warp] = mlg;
  item_sync<kThreads>(bar);
  int M = INT_MIN;
#pragma unroll
  for (int q = 0; q < kWarps; ++q) M = max(M, wmax[q]);
  const int ex = scale_of(M);
  const Pow2f s2 = pow2f_split(ex);
  // pass 2: fixed point
#pragma unroll
  for (int k = 0; k < kMaxHandsPerThread; ++k) {
    const int h = tid + k * kThreads;
    if (h < ld) {
      if constexpr (std::is_same<TIn, float>::value) F[h] = {fx_of(r_opp[h], rhi_opp[h], rlo_opp[h], y[k], s2, ex)};
      else F[h] = {fx_of64(r_opp[h], y[k], ex)};
    }
  }
  item_sync<kThreads>(bar);

  // exclusive prefix over ascending strength: P[i] = sum_{k < i} w[k], P[ld] = total
  const int K = (ld + kThreads - 1) / kThreads;   // raking chunk
  const int k0 = min(tid * K, ld), k1 = min(k0 + K, ld);
  Fx loc = fx_zero();
  for (int i = k0; i < k1; ++i) loc = fx_add(loc, F[i]);
  const Fx inc = fx_scan(loc, lane);
  if (lane == 31) wtot[warp] = inc;
  Fx run = fx_shfl_up(inc, 1);
  if (lane == 0) run = fx_zero();
  item_sync<kThreads>(bar);
#pragma unroll
  for (int q = 0; q < kWarps; ++q)   // (unrolled: the loads issue together)
    if (q < warp) run = fx_add(run, wtot[q]);
  for (int i = k0; i < k1; ++i) {
    P[i] = run;
    run = fx_add(run, F[i]);
  }
  if (k0 < ld && k1 == ld) P[ld] = run;

  // per-card exclusive prefixes: a card slot per 16-lane half warp, four consecutive
  // list entries (at most 64) per lane, summed serially, then one half-warp scan
  {
    const int sub = lane >> 4, sl = lane & 15, i0 = 4 * sl;
    for (int c0 = 2 * warp; c0 < g.n_slots; c0 += 2 * kWarps) {   // (warp-uniform trip count)
      const int c = c0 + sub;
      const bool ok = c < g.n_slots;
      const int len = ok ? tb.card_len[c] : 0;
      const uint16_t* lst = tb.card_hands + (size_t)(ok ? c : 0) * g.lmax;
      Fx a[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) a[j] = i0 + j < len ? F[lst[i0 + j]] : fx_zero();
#pragma unroll
      for (int j = 1; j < 4; ++j) a[j] = fx_add(a[j - 1], a[j]);
      const Fx inc = fx_scan16(a[3], sl);
      const Fx before = fx_sub(inc, a[3]);
      Fx* pc = PC + (size_t)(ok ? c : 0) * lstride;
      if (ok && sl == 0) pc[0] = fx_zero();
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (ok && i0 + j < len) pc[pc_pad(i0 + j + 1)] = fx_add(before, a[j]);
    }
  }
  item_sync<kThreads>(bar);

  const Fx W = P[ld];
#pragma unroll
  for (int k = 0; k < kMaxHandsPerThread; ++k) {
    const int h = tid + k * kThreads;
    if (h >= ld) break;
    const uint4 hi = tb.hinfo[h];
    const Fx C0 = PC[hi.z & 0xffffu];
    const Fx C1 = PC[hi.w >> 16];
    Fx val;
    if (kind == 0) {
      val = fx_sub(fx_sub(W, C0), C1);
      if (g.hand_size == 2) val = fx_add(val, F[h]);
    } else {
      const Fx lt = fx_sub(fx_sub(P[hi.x & 0xffffu], PC[hi.y & 0xffffu]), PC[hi.z >> 16]);
      const Fx gt = fx_sub(fx_sub(fx_sub(W, P[hi.x >> 16]), fx_sub(C0, PC[hi.y >> 16])),
                           fx_sub(C1, PC[hi.w & 0xffffu]));
      val = fx_sub(gt, lt);
    }
    const bool live = h < H;
    float v32;
    double v64;
    fx_to_f32_f64_conv(val, ex, v32, v64);
    if (c32 != nullptr) c32[(size_t)e * ld + h] = live ? coef32 * v32 : 0.f;
    if (c64 != nullptr) c64[(size_t)e * ld + h] = live ? coef64 * v64 : 0.0;
  }
  item_sync<kThreads>(bar);   // shared memory is reused by the caller's next item
}

// Product row s of a player at hand h from the terminal contributions: the
// contributions of its terminals [ptr[s], ptr[s+1]) added in order, times r / Z.
__device__ __forceinline__ float product32(const float* c, const int* ptr, int s, int ld, int h, float rz) {
  float acc = 0.f;
  for (int e = ptr[s]; e < ptr[s + 1]; ++e) acc += __ldcg(c + (size_t)e * ld + h);
  return rz * acc;
}

__device__ __forceinline__ double product64(const double* c, const int* ptr, int s, int ld, int h,
                                            double rz) {
  double acc = 0.0;
  for (int e = ptr[s]; e < ptr[s + 1]; ++e) acc += __ldcg(c + (size_t)e * ld + h);
  return rz * acc;
}

// -product64 (the negation folds into the multiply)
__device__ __forceinline__ double neg_product64(const double* c, const int* ptr, int s, int ld, int h,
                                                double rz) {
  double acc = 0.0;
  for (int e = ptr[s]; e < ptr[s + 1]; ++e) acc += __ldcg(c + (size_t)e * ld + h);
  return (-rz) * acc;
}

}  // namespace egt
