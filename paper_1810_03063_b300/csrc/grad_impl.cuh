// Gradient product body shared by the standalone kernel and the solver engine.
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
// One CTA (512 threads) per output sequence; its two halves take the
// sequence's terminals in pairs (every sequence of the river games has one or
// two).  Sums are exact: each w is converted once to fixed point (int64 limbs,
// a per-terminal power-of-two scale from max |w| leaving 2^59 headroom), so
// prefix sums, per-card corrections and the tie-aware differences are integer
// operations in any order -- deterministic, and on the full-rate integer pipes.
// FP32 path: one limb (resolution max|w| 2^-48); FP64 path: two limbs (the
// second holds the next 40 bits of the first's fraction).  The per-hand result
// is rounded once to T, scaled by the terminal's coefficient and accumulated
// over terminals in float-float (FP32) or double (FP64).
#pragma once
#include "egt_internal.cuh"

namespace egt {

constexpr int kItemThreads = 512;     // threads of a CTA of the engine and of the kernels
constexpr int kHalfThreads = 256;     // one terminal per half CTA

namespace gradimpl {

struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  err = __fadd_rn(err, __fadd_rn(a.lo, b.lo));
  const float hi = __fadd_rn(s, err);
  return {hi, __fsub_rn(err, __fsub_rn(hi, s))};
}

// c * v with the product's rounding error kept (TwoProd by fma)
__device__ __forceinline__ FF ff_prod(float c, float v) {
  const float p = __fmul_rn(c, v);
  return {p, __fmaf_rn(c, v, -p)};
}

template <int NL>
struct Fx {
  long long v[NL];
};

template <int NL>
__device__ __forceinline__ Fx<NL> fx_zero() {
  Fx<NL> r;
#pragma unroll
  for (int i = 0; i < NL; ++i) r.v[i] = 0;
  return r;
}
template <int NL>
__device__ __forceinline__ Fx<NL> fx_add(Fx<NL> a, Fx<NL> b) {
#pragma unroll
  for (int i = 0; i < NL; ++i) a.v[i] += b.v[i];
  return a;
}
template <int NL>
__device__ __forceinline__ Fx<NL> fx_sub(Fx<NL> a, Fx<NL> b) {
#pragma unroll
  for (int i = 0; i < NL; ++i) a.v[i] -= b.v[i];
  return a;
}
template <int NL>
__device__ __forceinline__ Fx<NL> fx_shfl_up(Fx<NL> a, int d) {
#pragma unroll
  for (int i = 0; i < NL; ++i) a.v[i] = __shfl_up_sync(0xffffffffu, a.v[i], d);
  return a;
}
template <int NL>
__device__ __forceinline__ Fx<NL> fx_shfl(Fx<NL> a, int src) {
#pragma unroll
  for (int i = 0; i < NL; ++i) a.v[i] = __shfl_sync(0xffffffffu, a.v[i], src);
  return a;
}
template <int NL>
__device__ __forceinline__ Fx<NL> fx_scan(Fx<NL> v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    Fx<NL> o = fx_shfl_up(v, d);
    if (lane >= d) v = fx_add(v, o);
  }
  return v;
}

// 2^e as float / double for the exponent ranges used here (split in two factors)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }
__device__ __forceinline__ double pow2d(int e) {
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// Conversions to and from fixed point work on the IEEE bit fields with integer
// operations: B300's FP64 pipe (and 64-bit conversions routed through it) runs
// at a small fraction of the integer rate.

// round(m 2^sh) for an integer mantissa m (sh < 0: right shift, half rounds up)
__device__ __forceinline__ long long shift_round(unsigned long long m, int sh) {
  if (sh >= 0) return (long long)(m << sh);
  const int r = -sh;
  if (r > 63) return 0;
  return (long long)((m >> r) + ((m >> (r - 1)) & 1ull));
}

// int64 -> float rounded to nearest even (leading-zero count and shifts)
__device__ __forceinline__ float i64_to_f32(long long v) {
  if (v == 0) return 0.f;
  const unsigned long long u = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int nb = 64 - __clzll(u);
  float f;
  if (nb <= 24) {
    f = __uint2float_rn((unsigned)u);
  } else {
    int sh = nb - 24;
    unsigned long long mant = u >> sh;
    const unsigned long long rem = u & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ull))) ++mant;
    if (mant == (1ull << 24)) {
      mant >>= 1;
      ++sh;
    }
    f = __int_as_float(((127 + 23 + sh) << 23) | (int)(mant & 0x7fffffull));
  }
  return v < 0 ? -f : f;
}

template <typename T>
struct Conv;

template <>
struct Conv<float> {
  static constexpr int NL = 1;
  // round(w 2^e): w = m 2^(E - 150) with a 24-bit integer mantissa m
  static __device__ __forceinline__ Fx<1> to_fx(float w, int e) {
    const unsigned bits = __float_as_uint(w);
    int E = (bits >> 23) & 0xff;
    unsigned m = bits & 0x7fffffu;
    Fx<1> r;
    r.v[0] = 0;
    if (E == 0 && m == 0) return r;
    if (E == 0) E = 1;
    else m |= 0x800000u;
    const long long a = shift_round(m, E - 150 + e);
    r.v[0] = (bits >> 31) ? -a : a;
    return r;
  }
  static __device__ __forceinline__ float from_fx(Fx<1> a, int e) {
    const int e1 = e >> 1;
    return i64_to_f32(a.v[0]) * pow2f(-e1) * pow2f(e1 - e);
  }
  static __device__ __forceinline__ float absmax(float a, float b) { return fmaxf(a, fabsf(b)); }
  // scale exponent so that |sum| of up to 2048 terms stays below 2^59
  static __device__ __forceinline__ int scale(float M) {
    return M > 0.f ? 48 - (ilogbf(M) + 1) : 0;
  }
};

template <>
struct Conv<double> {
  static constexpr int NL = 2;
  // |w| 2^e split as a + b 2^-40 (a the integer part, b the next 40 bits of the
  // fraction, both truncated), w = m 2^(E - 1075) with a 53-bit integer mantissa m
  static __device__ __forceinline__ Fx<2> to_fx(double w, int e) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(w);
    int E = (int)((bits >> 52) & 0x7ffull);
    unsigned long long m = bits & ((1ull << 52) - 1);
    Fx<2> r;
    r.v[0] = r.v[1] = 0;
    if (E == 0 && m == 0) return r;
    if (E == 0) E = 1;
    else m |= (1ull << 52);
    const int sh = E - 1075 + e;
    long long a = 0, b = 0;
    if (sh >= 0) {
      a = (long long)(m << sh);
    } else {
      const int k = -sh;                       // fractional bits of m 2^sh
      if (k < 64) {
        a = (long long)(m >> k);
        const unsigned long long frac = m & ((1ull << k) - 1);
        b = k <= 40 ? (long long)(frac << (40 - k)) : (k - 40 < 64 ? (long long)(frac >> (k - 40)) : 0);
      } else if (k - 40 < 64) {
        b = (long long)(m >> (k - 40));
      }
    }
    if (bits >> 63) {
      a = -a;
      b = -b;
    }
    r.v[0] = a;
    r.v[1] = b;
    return r;
  }
  static __device__ __forceinline__ double from_fx(Fx<2> a, int e) {
    const double s = (double)a.v[0] + (double)a.v[1] * (1.0 / 1099511627776.0);
    const int e1 = e >> 1;
    return s * pow2d(-e1) * pow2d(e1 - e);
  }
  static __device__ __forceinline__ double absmax(double a, double b) { return fmax(a, fabs(b)); }
  static __device__ __forceinline__ int scale(double M) { return M > 0.0 ? 48 - (ilogb(M) + 1) : 0; }
};

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
__device__ __forceinline__ const double* ranges_z<double>(const DevGame& g, int p) { return g.rz64[p]; }
template <typename T>
__device__ __forceinline__ T term_coef(const DevTerms& t, int e);
template <>
__device__ __forceinline__ float term_coef<float>(const DevTerms& t, int e) { return t.coef[e]; }
template <>
__device__ __forceinline__ double term_coef<double>(const DevTerms& t, int e) { return t.coef64[e]; }

// accumulator of one hand over terminals
template <typename T>
struct Acc;
template <>
struct Acc<float> {
  FF a;
  __device__ __forceinline__ void zero() { a = {0.f, 0.f}; }
  __device__ __forceinline__ void add(float c, float v) { a = ff_add(a, ff_prod(c, v)); }
  __device__ __forceinline__ float value() const { return __fadd_rn(a.hi, a.lo); }
};
template <>
struct Acc<double> {
  double a;
  __device__ __forceinline__ void zero() { a = 0.0; }
  __device__ __forceinline__ void add(double c, double v) { a += c * v; }
  __device__ __forceinline__ double value() const { return a; }
};

__device__ __forceinline__ void half_sync(int half) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + half), "r"(kHalfThreads) : "memory");
}

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// shared memory of one half: w, F (w in fixed point), P, PC, warp maxima, warp totals
template <typename T>
__host__ __device__ inline size_t half_bytes(int ld, int n_slots, int lmax) {
  constexpr int NL = sizeof(T) == 4 ? 1 : 2;
  const size_t fx = sizeof(long long) * NL;
  size_t b = align16((size_t)ld * sizeof(T));
  b += align16((size_t)ld * fx);
  b += align16((size_t)(ld + 1) * fx);
  b += align16((size_t)n_slots * (lmax + 1) * fx);
  b += 8 * sizeof(T) + 8 * fx + 16;
  return align16(b);
}

constexpr int kMaxHandsPerThread = 8;   // ld <= 2048 with 256 threads per half

}  // namespace gradimpl

// Shared memory of one gradient CTA (without the staged tables).
inline size_t grad_item_smem(const DevGame& g, bool f64) {
  return 2 * (f64 ? gradimpl::half_bytes<double>(g.ld, g.n_slots, g.lmax)
                  : gradimpl::half_bytes<float>(g.ld, g.n_slots, g.lmax));
}

// Per-game tables the product reads for every terminal, staged once in shared memory.
struct GradTab {
  const uint4* hinfo;          // [ld] per-hand flat indices (see DevGame::hinfo)
  const int* card_len;         // [n_slots]
  const uint16_t* card_hands;  // [n_slots][lmax]
};

__host__ __device__ inline size_t grad_tab_bytes(const DevGame& g) {
  using gradimpl::align16;
  return align16((size_t)g.ld * sizeof(uint4)) + align16((size_t)g.n_slots * sizeof(int)) +
         align16((size_t)g.n_slots * g.lmax * sizeof(uint16_t));
}

// Copy the tables into dst (all threads of the CTA; the caller synchronises before use).
__device__ inline GradTab stage_grad_tab(const DevGame& g, unsigned char* dst) {
  using gradimpl::align16;
  uint4* hi = reinterpret_cast<uint4*>(dst);
  int* cl = reinterpret_cast<int*>(dst + align16((size_t)g.ld * sizeof(uint4)));
  uint16_t* ch = reinterpret_cast<uint16_t*>(reinterpret_cast<unsigned char*>(cl) +
                                             align16((size_t)g.n_slots * sizeof(int)));
  for (int i = threadIdx.x; i < g.ld; i += blockDim.x) hi[i] = g.hinfo[i];
  for (int i = threadIdx.x; i < g.n_slots; i += blockDim.x) cl[i] = g.card_len[i];
  for (int i = threadIdx.x; i < g.n_slots * g.lmax; i += blockDim.x) ch[i] = g.card_hands[i];
  return {hi, cl, ch};
}

// Output column s of player `player` (out[s][*] = (A in)[s] for player 0, (A^T in)[s]
// for player 1), computed by one CTA of kItemThreads threads.  `in` is read through L2
// (it may have been written earlier in the same launch by other CTAs).
template <typename TIn, typename T>
__device__ inline void grad_item(const DevGame& g, const GradTab& tb, int player, int s,
                                 const TIn* __restrict__ in, T* __restrict__ out,
                                 unsigned char* smem) {
  using namespace gradimpl;
  using C = Conv<T>;
  constexpr int NL = C::NL;
  const int ld = g.ld, H = g.H, opp = 1 - player;
  const int tid = threadIdx.x, half = tid / kHalfThreads, th = tid % kHalfThreads;
  const int lane = tid & 31, hw = th >> 5;
  constexpr int kHalfWarps = kHalfThreads / 32;
  const int lstride = g.lmax + 1;

  unsigned char* hs = smem + half * half_bytes<T>(ld, g.n_slots, g.lmax);
  T* w = reinterpret_cast<T*>(hs);
  Fx<NL>* F = reinterpret_cast<Fx<NL>*>(hs + align16((size_t)ld * sizeof(T)));
  Fx<NL>* P = reinterpret_cast<Fx<NL>*>(reinterpret_cast<unsigned char*>(F) +
                                        align16((size_t)ld * sizeof(Fx<NL>)));
  Fx<NL>* PC = reinterpret_cast<Fx<NL>*>(reinterpret_cast<unsigned char*>(P) +
                                         align16((size_t)(ld + 1) * sizeof(Fx<NL>)));
  T* wmax = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(PC) +
                                 align16((size_t)g.n_slots * lstride * sizeof(Fx<NL>)));
  Fx<NL>* wtot = reinterpret_cast<Fx<NL>*>(reinterpret_cast<unsigned char*>(wmax) + 8 * sizeof(T));

  const DevTerms tm = g.terms[player];
  const int e0 = tm.ptr[s], e1 = tm.ptr[s + 1];
  const T* __restrict__ r_opp = ranges<T>(g, opp);

  Acc<T> acc[kMaxHandsPerThread];
#pragma unroll
  for (int k = 0; k < kMaxHandsPerThread; ++k) acc[k].zero();

  const int K = (ld + kHalfThreads - 1) / kHalfThreads;   // raking chunk
  const int k0 = min(th * K, ld), k1 = min(k0 + K, ld);

  for (int base = e0; base < e1; base += 2) {
    const int e = base + half;
    if (e >= e1) continue;                                   // uniform within a half
    const int os = tm.opp_seq[e];
    const int kind = tm.kind[e];
    const T coef = term_coef<T>(tm, e);
    const TIn* col = in + (size_t)os * ld;

    T m = T(0);
    for (int h = th; h < ld; h += kHalfThreads) {
      const T wv = h < H ? r_opp[h] * (T)__ldcg(col + h) : T(0);
      w[h] = wv;
      m = C::absmax(m, wv);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) m = C::absmax(m, __shfl_xor_sync(0xffffffffu, m, d));
    if (lane == 0) wmax[hw] = m;
    half_sync(half);
    T M = T(0);
#pragma unroll
    for (int q = 0; q < kHalfWarps; ++q) M = C::absmax(M, wmax[q]);
    const int ex = C::scale(M);
    for (int h = th; h < ld; h += kHalfThreads) F[h] = C::to_fx(w[h], ex);
    half_sync(half);

    // exclusive prefix over ascending strength: P[i] = sum_{k < i} w[k], P[ld] = total
    Fx<NL> loc = fx_zero<NL>();
    for (int i = k0; i < k1; ++i) loc = fx_add(loc, F[i]);
    const Fx<NL> inc = fx_scan(loc, lane);
    if (lane == 31) wtot[hw] = inc;
    Fx<NL> run = fx_shfl_up(inc, 1);
    if (lane == 0) run = fx_zero<NL>();
    half_sync(half);
    for (int q = 0; q < hw; ++q) run = fx_add(run, wtot[q]);
    for (int i = k0; i < k1; ++i) {
      P[i] = run;
      run = fx_add(run, F[i]);
    }
    if (k0 < ld && k1 == ld) P[ld] = run;

    // per-card exclusive prefixes, one warp per card slot
    for (int c = hw; c < g.n_slots; c += kHalfWarps) {
      const int len = tb.card_len[c];
      const uint16_t* lst = tb.card_hands + (size_t)c * g.lmax;
      const Fx<NL> v0 = lane < len ? F[lst[lane]] : fx_zero<NL>();
      const Fx<NL> v1 = lane + 32 < len ? F[lst[lane + 32]] : fx_zero<NL>();
      const Fx<NL> a0 = fx_scan(v0, lane);
      const Fx<NL> t0 = fx_shfl(a0, 31);
      const Fx<NL> a1 = fx_add(fx_scan(v1, lane), t0);
      Fx<NL>* pc = PC + (size_t)c * lstride;
      if (lane == 0) pc[0] = fx_zero<NL>();
      if (lane < len) pc[lane + 1] = a0;
      if (lane + 32 < len) pc[lane + 33] = a1;
    }
    half_sync(half);

    const Fx<NL> W = P[ld];
#pragma unroll
    for (int k = 0; k < kMaxHandsPerThread; ++k) {
      const int h = th + k * kHalfThreads;
      if (h >= ld) break;
      const uint4 hi = tb.hinfo[h];
      const Fx<NL> C0 = PC[hi.z & 0xffffu];
      const Fx<NL> C1 = PC[hi.w >> 16];
      Fx<NL> val;
      if (kind == 0) {
        val = fx_sub(fx_sub(W, C0), C1);
        if (g.hand_size == 2) val = fx_add(val, F[h]);
      } else {
        const Fx<NL> lt = fx_sub(fx_sub(P[hi.x & 0xffffu], PC[hi.y & 0xffffu]), PC[hi.z >> 16]);
        const Fx<NL> gt = fx_sub(fx_sub(fx_sub(W, P[hi.x >> 16]), fx_sub(C0, PC[hi.y >> 16])),
                                 fx_sub(C1, PC[hi.w & 0xffffu]));
        val = fx_sub(gt, lt);
      }
      acc[k].add(coef, C::from_fx(val, ex));
    }
    half_sync(half);   // w / F / P / PC are rewritten by the next terminal of this half
  }

  // combine the halves: half 1 leaves its per-hand sums in its w area
  __syncthreads();
  T* other = reinterpret_cast<T*>(smem + half_bytes<T>(ld, g.n_slots, g.lmax));
  if (half == 1) {
#pragma unroll
    for (int k = 0; k < kMaxHandsPerThread; ++k) {
      const int h = th + k * kHalfThreads;
      if (h >= ld) break;
      other[h] = acc[k].value();
    }
  }
  __syncthreads();
  if (half == 0) {
    const T* __restrict__ rz = ranges_z<T>(g, player);
    T* o = out + (size_t)s * ld;
#pragma unroll
    for (int k = 0; k < kMaxHandsPerThread; ++k) {
      const int h = th + k * kHalfThreads;
      if (h >= ld) break;
      o[h] = h < H ? rz[h] * (acc[k].value() + other[h]) : T(0);
    }
  }
  __syncthreads();   // shared memory is reused by the caller's next item
}

}  // namespace egt
