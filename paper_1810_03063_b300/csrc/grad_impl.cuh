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
// r_me / Z while it loads them.  All sums are exact: each w is put in fixed point with two int64 limbs
// (integer part at a per-terminal power-of-two scale leaving 2^59 headroom,
// then 40 more fraction bits), so prefix sums, per-card corrections and the
// tie-aware differences are integer operations, deterministic in any order and
// on the full-rate integer pipes.  For FP32 inputs w = r (FP64 range) x y is
// formed exactly as the 77-bit product of the two mantissas, with integer
// operations only (B300's FP64 pipe is a small fraction of the integer rate).
// From the same exact sums the CTA can emit an FP32 contribution (the path of
// every EGT step) and an FP64 one (the stopping residual); asking for the FP64
// one does not change the FP32 one.
#pragma once
#include <climits>
#include <cstring>
#include <type_traits>

#include "egt_internal.cuh"

namespace egt {

constexpr int kItemThreads = 512;     // threads of a CTA of the engine and of the kernels

namespace gradimpl {

// Bit-level helpers that also compile for the host: the exact-arithmetic functions
// below (w = r y, fixed point, rounding back to FP32 / FP64) are checked on the CPU
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
__host__ __device__ __forceinline__ unsigned long long umul64hi(unsigned long long a, unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
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

// fixed point: v0 = integer part, v1 = the next 40 fraction bits (both carry the sign)
struct Fx {
  long long v0, v1;
};

__host__ __device__ __forceinline__ Fx fx_zero() { return {0, 0}; }
__host__ __device__ __forceinline__ Fx fx_add(Fx a, Fx b) { return {a.v0 + b.v0, a.v1 + b.v1}; }
__host__ __device__ __forceinline__ Fx fx_sub(Fx a, Fx b) { return {a.v0 - b.v0, a.v1 - b.v1}; }
__device__ __forceinline__ Fx fx_shfl_up(Fx a, int d) {
  return {__shfl_up_sync(0xffffffffu, a.v0, d), __shfl_up_sync(0xffffffffu, a.v1, d)};
}
__device__ __forceinline__ Fx fx_shfl(Fx a, int src) {
  return {__shfl_sync(0xffffffffu, a.v0, src), __shfl_sync(0xffffffffu, a.v1, src)};
}
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
    const Fx o = {__shfl_up_sync(0xffffffffu, v.v0, d, 16), __shfl_up_sync(0xffffffffu, v.v1, d, 16)};
    if (sl >= d) v = fx_add(v, o);
  }
  return v;
}

// 2^e as float / double for the exponent ranges used here (split in two factors)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }
__device__ __forceinline__ double pow2d(int e) {
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// floor(P / 2^k) of the 128-bit P = hi:lo, low 64 bits
__host__ __device__ __forceinline__ unsigned long long shr128(unsigned long long hi, unsigned long long lo, int k) {
  if (k <= 0) return lo;
  if (k >= 128) return 0;
  if (k >= 64) return hi >> (k - 64);
  return (lo >> k) | (hi << (64 - k));
}

// |w| = P 2^E with P = hi:lo an exact integer, sign neg, lg = floor(log2 |w|)
// (INT_MIN when w = 0).
struct WBits {
  unsigned long long hi, lo;
  int E, lg, neg;
};

// w = r * y exactly: 53-bit x 24-bit mantissa product
__host__ __device__ __forceinline__ WBits wprod(double r, float y) {
  const unsigned long long rb = f64_bits(r);
  const unsigned yb = f32_bits(y);
  int er = (int)((rb >> 52) & 0x7ffull), ey = (int)((yb >> 23) & 0xffu);
  unsigned long long mr = rb & ((1ull << 52) - 1), my = yb & 0x7fffffu;
  WBits w;
  w.neg = (int)((rb >> 63) ^ (yb >> 31));
  if ((er == 0 && mr == 0) || (ey == 0 && my == 0)) {
    w.hi = w.lo = 0;
    w.E = 0;
    w.lg = INT_MIN;
    return w;
  }
  if (er == 0) er = 1;
  else mr |= 1ull << 52;
  if (ey == 0) ey = 1;
  else my |= 1ull << 23;
  w.lo = mr * my;
  w.hi = umul64hi(mr, my);
  w.E = (er - 1075) + (ey - 150);
  const int nb = w.hi ? 128 - clz64(w.hi) : 64 - clz64(w.lo);
  w.lg = w.E + nb - 1;
  return w;
}

// w = r * y for an FP64 y: rounded once in FP64, then exact from there
__host__ __device__ __forceinline__ WBits wprod(double r, double y) {
  const double w = r * y;
  const unsigned long long b = f64_bits(w);
  int e = (int)((b >> 52) & 0x7ffull);
  unsigned long long m = b & ((1ull << 52) - 1);
  WBits x;
  x.neg = (int)(b >> 63);
  if (e == 0 && m == 0) {
    x.hi = x.lo = 0;
    x.E = 0;
    x.lg = INT_MIN;
    return x;
  }
  if (e == 0) e = 1;
  else m |= 1ull << 52;
  x.hi = 0;
  x.lo = m;
  x.E = e - 1075;
  x.lg = x.E + (64 - clz64(m)) - 1;
  return x;
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

// |w| 2^ex as integer part + 40 truncated fraction bits, signed
__host__ __device__ __forceinline__ Fx to_fx(const WBits& w, int ex) {
  if (w.lg == INT_MIN) return fx_zero();
  const int s = w.E + ex;
  unsigned long long a, b;
  if (s >= 0) {
    a = w.lo << s;          // |w| 2^ex < 2^48 keeps this in range
    b = 0;
  } else {
    // Q = P 2^(s + 40) truncated, holding a (integer part) and b (40 fraction bits),
    // from one right shift of P 2^39 (P < 2^77) by u = -s - 1: no branch on the
    // magnitude while u < 64 (hands within 35 binades of the column's largest |w|)
    const unsigned long long Lhi = (w.hi << 39) | (w.lo >> 25), Llo = w.lo << 39;
    const int u = -s - 1;
    unsigned long long qhi = 0, qlo = 0;
    if (u < 64) {
      qlo = u ? (Llo >> u) | (Lhi << (64 - u)) : Llo;
      qhi = Lhi >> u;
    } else if (u < 128) {
      qlo = Lhi >> (u - 64);
    }
    a = (qhi << 24) | (qlo >> 40);
    b = qlo & ((1ull << 40) - 1);
  }
  const long long sa = (long long)a, sb = (long long)b;
  return w.neg ? Fx{-sa, -sb} : Fx{sa, sb};
}

// scale so that |w| 2^ex < 2^48 for the largest |w| (sums of 2048 terms < 2^59)
__host__ __device__ __forceinline__ int scale_of(int maxlg) { return maxlg == INT_MIN ? 0 : 47 - maxlg; }

// |N| of a fixed-point sum, N = v0 2^40 + v1 as a signed 128-bit integer
// (uh:ul), its sign and bit length (0 when N = 0).
struct Wide {
  unsigned long long uh, ul;
  int nb, neg;
};

__host__ __device__ __forceinline__ Wide fx_wide(Fx a) {
  unsigned long long lo = (unsigned long long)a.v0 << 40;
  long long hi = a.v0 >> 24;
  const unsigned long long lo2 = lo + (unsigned long long)a.v1;
  hi += (a.v1 < 0 ? -1 : 0) + (lo2 < lo ? 1 : 0);
  lo = lo2;
  Wide w;
  w.neg = hi < 0;
  w.uh = (unsigned long long)hi;
  w.ul = lo;
  if (w.neg) {
    w.ul = ~w.ul + 1ull;
    w.uh = ~w.uh + (w.ul == 0 ? 1ull : 0ull);
  }
  w.nb = w.uh ? 128 - clz64(w.uh) : (w.ul ? 64 - clz64(w.ul) : 0);
  return w;
}

// The leading P bits of |N| (nb >= 1, 1 <= P <= 53) rounded to nearest even:
// the mantissa in [2^(P-1), 2^P]; a carry to 2^P is left to the caller.
__host__ __device__ __forceinline__ unsigned long long round_top(const Wide& w, int P) {
  if (w.nb <= P) return w.ul << (P - w.nb);
  const int sh = w.nb - P;
  const unsigned long long mant = shr128(w.uh, w.ul, sh);
  const int rb = sh - 1;                                     // position of the rounding bit
  const unsigned long long round = rb < 64 ? (w.ul >> rb) & 1ull : (w.uh >> (rb - 64)) & 1ull;
  bool sticky;
  if (rb == 0) sticky = false;
  else if (rb < 64) sticky = (w.ul & ((1ull << rb) - 1ull)) != 0;
  else if (rb == 64) sticky = w.ul != 0;
  else sticky = w.ul != 0 || (w.uh & ((1ull << (rb - 64)) - 1ull)) != 0;
  return mant + ((round && (sticky || (mant & 1ull))) ? 1ull : 0ull);
}

// |N| 2^s (N from fx_wide) correctly rounded to a binary format with P-bit
// significands, minimum normal exponent emin and bias `bias`: the magnitude's
// bit pattern (exponent field << (P - 1) | fraction), or the all-ones exponent
// field (infinity) on overflow.
__host__ __device__ __forceinline__ unsigned long long fx_round(const Wide& w, int s, int P, int emin, int emax) {
  const int e0 = w.nb - 1 + s;                                // exponent of the leading bit
  if (e0 > emax) return (unsigned long long)(emax - emin + 2) << (P - 1);
  if (e0 >= emin) {
    unsigned long long mant = round_top(w, P);
    int e = e0;
    if (mant >> P) {
      mant >>= 1;
      ++e;
    }
    if (e > emax) return (unsigned long long)(emax - emin + 2) << (P - 1);
    return ((unsigned long long)(e - emin + 1) << (P - 1)) | (mant & ((1ull << (P - 1)) - 1ull));
  }
  // subnormal: P - (emin - e0) significant bits remain
  const int q = P - (emin - e0);
  if (q < 0) return 0;
  if (q == 0) {   // |value| in [min subnormal / 2, min subnormal): rounds up unless exactly half
    const bool above = w.nb >= 2 && (w.nb - 1 >= 64 ? (w.ul != 0 || (w.uh & ((1ull << (w.nb - 65)) - 1ull)) != 0)
                                                    : (w.ul & ((1ull << (w.nb - 1)) - 1ull)) != 0);
    return above ? 1ull : 0ull;
  }
  return round_top(w, q);   // a carry to 2^q lands on the smallest normal, as it should
}

// FP32 and FP64 values of a fixed-point sum, a x 2^-ex, both correctly rounded
// (every bit of the sum counts), with integer operations and one normalisation:
// the magnitude, a 104-bit integer hi:lo, is shifted so that its leading bit is
// bit 63 of T, and each significand is rounded to nearest even from the top of T,
// the bits below it (in T, and past T: `rest`) acting as the sticky bit.  Only
// subnormal and overflowing results branch off, to the general path.
__host__ __device__ __forceinline__ void fx_to_f32_f64(Fx a, int ex, float& r32, double& r64) {
  const long long v0 = a.v0 + (a.v1 >> 40);
  const unsigned long long f = (unsigned long long)a.v1 & ((1ull << 40) - 1ull);
  const bool neg = v0 < 0;
  const unsigned long long m0 = neg ? (unsigned long long)(-(v0 + (f ? 1 : 0))) : (unsigned long long)v0;
  const unsigned long long m1 = neg ? (f ? (1ull << 40) - f : 0ull) : f;
  const unsigned long long hi = m0 >> 24, lo = (m0 << 40) | m1;   // |sum| = hi 2^64 + lo
  if ((hi | lo) == 0) {
    r32 = 0.f;
    r64 = 0.0;
    return;
  }
  // hi < 2^40, so lz is in [24, 127] and every shift below is in [1, 63]
  const int lz = hi ? clz64(hi) : 64 + clz64(lo);
  const unsigned long long T = lz < 64 ? (hi << lz) | (lo >> (64 - lz)) : lo << (lz - 64);
  const bool rest = lz < 64 && (lo << lz) != 0;
  const int e = 127 - lz - 40 - ex;                               // exponent of the leading bit
  unsigned long long q = T >> 11;
  q += ((T >> 10) & 1ull) & (unsigned long long)(((T & 0x3ffull) != 0) | rest | (q & 1ull));
  int e64 = e;
  if (q >> 53) {
    q >>= 1;
    ++e64;
  }
  unsigned long long p = T >> 40;
  p += ((T >> 39) & 1ull) & (unsigned long long)(((T & ((1ull << 39) - 1ull)) != 0) | rest | (p & 1ull));
  int e32 = e;
  if (p >> 24) {
    p >>= 1;
    ++e32;
  }
  if (e64 + 1023 < 1 || e64 + 1023 > 2046 || e32 + 127 < 1 || e32 + 127 > 254) {
    const Wide w = fx_wide(a);
    r64 = bits_f64(((unsigned long long)w.neg << 63) | fx_round(w, -40 - ex, 53, -1022, 1023));
    r32 = bits_f32(((unsigned)w.neg << 31) | (unsigned)fx_round(w, -40 - ex, 24, -126, 127));
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
};

__host__ __device__ inline size_t grad_tab_bytes(const DevGame& g) {
  using gradimpl::align16;
  return align16((size_t)g.ld * sizeof(uint4)) + align16((size_t)g.n_slots * sizeof(int)) +
         align16((size_t)g.n_slots * g.lmax * sizeof(uint16_t)) + 2 * align16((size_t)g.ld * sizeof(double));
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
  for (int i = threadIdx.x; i < g.ld; i += blockDim.x) {
    hi[i] = g.hinfo[i];
    r0[i] = g.r64[0][i];
    r1[i] = g.r64[1][i];
  }
  for (int i = threadIdx.x; i < g.n_slots; i += blockDim.x) cl[i] = g.card_len[i];
  for (int i = threadIdx.x; i < g.n_slots * g.lmax; i += blockDim.x) ch[i] = g.card_hands[i];
  GradTab t;
  t.hinfo = hi;
  t.card_len = cl;
  t.card_hands = ch;
  t.r64[0] = r0;
  t.r64[1] = r1;
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
      else mlg = max(mlg, wprod(r_opp[h], y[k]).lg);   // (FP64 y: rounded product, exact lg)
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
  // pass 2: exact fixed point
#pragma unroll
  for (int k = 0; k < kMaxHandsPerThread; ++k) {
    const int h = tid + k * kThreads;
    if (h < ld) F[h] = to_fx(wprod(r_opp[h], y[k]), ex);
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
      else mlg = max(mlg, wprod(r_opp[h], y[k]).lg);   // (FP64 y: rounded product, exact lg)
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
  // pass 2: exact fixed point
#pragma unroll
  for (int k = 0; k < kMaxHandsPerThread; ++k) {
    const int h = tid + k * kThreads;
    if (h < ld) F[h] = to_fx(wprod(r_opp[h], y[k]), ex);
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
    fx_to_f32_f64(val, ex, v32, v64);
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
