// Smoothed best response (Sec. 5) and FP64 best response bodies, shared by the
// standalone kernels and the solver engine.
//
// Sec. 5: argmin_q <q, g> + mu sum_j beta_j q_{p_j} d_j(q^j / q_{p_j}) is solved
// bottom-up: at simplex j every branch i gets g_hat_i = g_i + (values of the
// child simplexes D_j^i); the simplex problem has q_bar_i proportional to
// exp(-g_hat_i / (mu beta_j)) and value  g_hat_i* + t log q_bar_i* + t log n_j
// (t = mu beta_j) taken at i* = argmax q_bar (= argmin g_hat), which is
// m - t log(sum_i exp(-(g_hat_i - m) / t)) + t log n_j with m = min g_hat.
// The value is evaluated as m - t log1p(sum_i expm1(-(g_hat_i - m)/t) / n_j),
// the same quantity without the cancellation of the two logarithms in FP32.
// Top-down: q_i = q_{p_j} q_bar_i, i.e. q_bar_i times the q_bar of every ancestor
// sequence, which needs no ordering between simplexes once all q_bar are known.
//
// Sec. 6: the per-hand treeplexes form a Cartesian product at the root, so
// hands are independent.  One item = 16 hands; a warp holds each hand twice
// (lane = hand + 16 x sub-lane) and the two sub-lanes take a simplex's branches
// alternately, halving the dependent chain of every simplex; the minimum and
// the sums over branches combine the sub-lanes with one shuffle.  (The SBR item
// also comes in an 8-hand form, each hand four times and two simplexes per
// warp, with the same bits: see sbr_item.)  The whole
// [S][16] tile of g (and of the previous iterate the output is mixed with) is
// fetched into shared memory before the recursion (two 64-byte row pieces per
// warp load), which then runs on shared memory: the warps split the simplexes
// of a level, levels are separated by CTA barriers; the top-down products then
// run on all warps at once, one (sequence, hand) per lane.
#pragma once
#include <math.h>

#include "grad_impl.cuh"

namespace egt {

struct SbrItemArgs {
  const float* g;          // gradient of the player's own loss up to `sign`; NULL = 0
  bool contrib;            // false: g is dense [S][ld]; true: g holds the player's terminal
  const float* grz;        //   contributions [T][ld] and row s is grz[h] x (sum over the
                           //   terminals [tptr[s], tptr[s+1]) of g[e][h], in order)
  float sign;              // +1 player 0 (g = A y), -1 player 1 (g = A^T x)
  double mu;
  const float* old;        // if non-NULL the output is (1 - tau) old + tau q
  float tau;
  float* out;              // [S][ld] or NULL (value only)
  double* value_partial;   // if non-NULL: this item's sum over live hands and root simplexes
};

// (the shared memory below excludes the staged tables)
template <int kH = kSbrHands>
__host__ __device__ inline size_t sbr_item_smem(const DevGame& g, int player) {
  const DevTpx& tp = g.tpx[player];
  return ((size_t)2 * tp.S * kH + (size_t)tp.J * kH + 2 * (size_t)tp.J) * sizeof(float);
}

__host__ __device__ inline size_t br_item_smem(const DevGame& g, int player) {
  const DevTpx& tp = g.tpx[player];
  return ((size_t)tp.S * kSbrHands + (size_t)tp.J * kSbrHands) * sizeof(double);
}

// One player's treeplex tables (Sec. 4 notation), staged once in shared memory.
struct TpxTab {
  int S, J, L;
  const int* tptr;         // [S+1] the player's terminals grouped by sequence (DevTerms::ptr)
  const double* beta;      // [J]
  const int* level_ptr;    // [L+1]
  const int* inf_first;    // [J]
  const int* inf_n;        // [J]
  const int* child_ptr;    // [S+1]
  const int* child_idx;    // [<= J]
  const int* seq_par;      // [S] (DevTpx::seq_par)
};

__host__ __device__ inline size_t tpx_tab_bytes(const DevGame& g, int player) {
  const DevTpx& tp = g.tpx[player];
  return gradimpl::align16((size_t)tp.J * sizeof(double)) +
         gradimpl::align16((size_t)(tp.L + 1 + 3 * tp.J + 2 * (tp.S + 1) + tp.S) * sizeof(int));
}

// Copy player's tables into dst (all threads; the caller synchronises before use).
__device__ inline TpxTab stage_tpx_tab(const DevGame& g, int player, unsigned char* dst) {
  const DevTpx& tp = g.tpx[player];
  TpxTab t;
  t.S = tp.S;
  t.J = tp.J;
  t.L = tp.L;
  double* beta = reinterpret_cast<double*>(dst);
  int* ip = reinterpret_cast<int*>(dst + gradimpl::align16((size_t)tp.J * sizeof(double)));
  int* lp = ip;
  int* fi = lp + tp.L + 1;
  int* nn = fi + tp.J;
  int* cp = nn + tp.J;
  int* ci = cp + tp.S + 1;
  const int nchild = tp.child_ptr[tp.S];
  int* tq = ci + nchild;
  int* sp = tq + tp.S + 1;
  const int* tsrc = player ? g.terms[1].ptr : g.terms[0].ptr;
  for (int i = threadIdx.x; i <= tp.S; i += blockDim.x) tq[i] = tsrc[i];
  for (int i = threadIdx.x; i < tp.S; i += blockDim.x) sp[i] = tp.seq_par[i];
  for (int i = threadIdx.x; i < tp.J; i += blockDim.x) {
    beta[i] = tp.beta[i];
    fi[i] = tp.inf_first[i];
    nn[i] = tp.inf_n[i];
  }
  for (int i = threadIdx.x; i <= tp.L; i += blockDim.x) lp[i] = tp.level_ptr[i];
  for (int i = threadIdx.x; i <= tp.S; i += blockDim.x) cp[i] = tp.child_ptr[i];
  for (int i = threadIdx.x; i < nchild; i += blockDim.x) ci[i] = tp.child_idx[i];
  t.beta = beta;
  t.level_ptr = lp;
  t.inf_first = fi;
  t.inf_n = nn;
  t.child_ptr = cp;
  t.child_idx = ci;
  t.tptr = tq;
  t.seq_par = sp;
  return t;
}

// Sum of n partial values in a fixed order (lane-strided, then a shuffle tree);
// called by one full warp, result valid in lane 0.
__device__ __forceinline__ double reduce_partials(const double* p, int n, int lane) {
  double v = 0.0;
  for (int i = lane; i < n; i += 32) v += __ldcg(p + i);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  return v;
}

// Lane layout of an item: hand hl = lane % 16, branch sub-lane bl = lane / 16.
constexpr int kSubLanes = 32 / kSbrHands;
static_assert(kSbrHands * kSubLanes == 32, "an item's hands times sub-lanes fill a warp");

// A level with more simplexes than this runs one simplex per half warp (each lane one
// hand, all branches in turn) instead of one per warp with the branches split over the
// two sub-lanes: the warps then hold twice as many independent simplexes, where one warp
// would otherwise take several in a row.  A fixed count, so that an item run by the
// whole CTA and one run by a warp half take the same form on every level.
constexpr int kSplitLevel = 16;

// The simplex problem of simplex j (Sec. 5) for hand lane hl, all branches by one lane:
// g_hat_i = g_i + child values into G, then q_bar into G and the value into V.  The sums
// over branches are kept per branch parity and added at the end: the order in which the
// two sub-lanes of the one-simplex-per-warp form add them, so both forms give the same
// bits.
template <int kH>
__device__ __forceinline__ void sbr_simplex_serial(const TpxTab& tp, int j, float* G, float* V, const float* tj,
                                                   const float* itj, int hl) {
  const int s0 = tp.inf_first[j], n = tp.inf_n[j];
  float m = INFINITY;
  for (int i = 0; i < n; ++i) {
    const int s = s0 + i;
    float gh = G[s * kH + hl];
    for (int c = tp.child_ptr[s]; c < tp.child_ptr[s + 1]; ++c) gh += V[tp.child_idx[c] * kH + hl];
    G[s * kH + hl] = gh;
    m = fminf(m, gh);
  }
  const float it = itj[j];
  float sum0 = 0.f, sum1 = 0.f, X0 = 0.f, X1 = 0.f;
  for (int i = 0; i < n; ++i) {
    float* u = G + (s0 + i) * kH + hl;
    const float d = -(*u - m) * it;
    const float e = expf(d);
    if (i & 1) {
      X1 += expm1f(d);
      sum1 += e;
    } else {
      X0 += expm1f(d);
      sum0 += e;
    }
    *u = e;
  }
  const float sum = sum0 + sum1, X = X0 + X1;
  const float inv = 1.f / sum;
  for (int i = 0; i < n; ++i) G[(s0 + i) * kH + hl] *= inv;
  V[j * kH + hl] = m - tj[j] * log1pf(X / (float)n);
}

// The warps that run an item: all of the CTA (bar = 0: __syncthreads), or half of it
// with its own named barrier (bar = 1 or 2) so that two items run side by side.
struct WarpGroup {
  int first_warp, n_warps, bar;
};
constexpr WarpGroup kWholeCta = {0, kItemThreads / 32, 0};

__device__ __forceinline__ void group_sync(const WarpGroup& wg) {
  if (wg.bar == 0) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"r"(wg.bar), "r"(wg.n_warps * 32) : "memory");
}

// One item (kH hands starting at blk * kH) of player `player`'s smoothed best response.
// kH = 16: a warp holds each hand twice (two branch sub-lanes).  kH = 8: four times, and
// its two halves take a simplex each where kH = 16 takes one per warp (four where it
// takes two); every (sequence, hand) result is formed by the same operations in the
// same order either way, so both give the same bits.  The value partial sums the
// item's hands, so it depends on kH.
template <int kH = kSbrHands>
__device__ inline void sbr_item(const DevGame& g, const TpxTab& tp, int blk, const SbrItemArgs& a,
                                float* sm, WarpGroup wg = kWholeCta) {
  static_assert(kH == 8 || kH == 16, "8 or 16 hands per item");
  constexpr int kSL = 32 / kH;                     // lanes per hand
  constexpr int kGroups = kSL / 2;                 // simplexes per warp, one per two sub-lanes
  const int S = tp.S, J = tp.J, ld = g.ld;
  const int kWarps = wg.n_warps;
  float* G = sm;                                   // [S][kH] sign*g -> g_hat -> q_bar -> q
  float* O = G + (size_t)S * kH;                   // [S][kH] previous iterate
  float* V = O + (size_t)S * kH;                   // [J][kH] simplex values
  float* tj = V + (size_t)J * kH;                  // [J] t_j = mu beta_j
  float* itj = tj + J;                             // [J] 1 / t_j
  const int tid = threadIdx.x - wg.first_warp * 32, lane = threadIdx.x & 31, warp = tid >> 5;
  const int hl = lane % kH, sq = lane / kH;        // hand, copy of the hand (0 .. kSL - 1)
  const int bl = sq & 1, grp = sq >> 1;            // branch sub-lane, simplex group
  const unsigned gmask = kGroups == 1 ? 0xffffffffu : 0xffffu << (16 * grp);
  const int h0 = blk * kH, h = h0 + hl;
  const bool live = h < g.H;

  // the [S][kH] tile of sign * g (and of the previous iterate): each warp takes rows
  // kSL warp + sq, then kSL warps further on, ...; the loads of kU rows are issued before
  // any is used
  {
    constexpr int kU = 4;
    const int kRowStep = kWarps * kSL;
    const float rz = (a.g != nullptr && a.contrib && live) ? a.grz[h] : 0.f;
    for (int s0 = kSL * warp + sq; s0 < S; s0 += kRowStep * kU) {
      float c0[kU], c1[kU], o[kU];
      int e0[kU], e1[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int s = s0 + u * kRowStep;
        c0[u] = c1[u] = o[u] = 0.f;
        e0[u] = e1[u] = 0;
        if (s < S) {
          if (a.g != nullptr && live) {
            if (a.contrib) {
              e0[u] = tp.tptr[s];
              e1[u] = tp.tptr[s + 1];
              if (e0[u] < e1[u]) c0[u] = __ldcg(a.g + (size_t)e0[u] * ld + h);
              if (e0[u] + 1 < e1[u]) c1[u] = __ldcg(a.g + (size_t)(e0[u] + 1) * ld + h);
            } else {
              c0[u] = __ldcg(a.g + (size_t)s * ld + h);
            }
          }
          if (a.old != nullptr) o[u] = __ldcg(a.old + (size_t)s * ld + h);
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int s = s0 + u * kRowStep;
        if (s < S) {
          float v = c0[u];
          if (a.contrib) {
            // rz x (sum of the sequence's contributions in terminal order)
            float acc = 0.f;
            if (e0[u] < e1[u]) acc += c0[u];
            if (e0[u] + 1 < e1[u]) acc += c1[u];
            for (int e = e0[u] + 2; e < e1[u]; ++e) acc += __ldcg(a.g + (size_t)e * ld + h);
            v = rz * acc;
          }
          G[s * kH + hl] = a.sign * v;
          if (a.old != nullptr) O[s * kH + hl] = o[u];
        }
      }
    }
  }
  for (int j = tid; j < J; j += kWarps * 32) {
    const float t = (float)(a.mu * tp.beta[j]);
    tj[j] = t;
    itj[j] = 1.f / t;
  }
  group_sync(wg);

  for (int l = tp.L - 1; l >= 0; --l) {
    if (tp.level_ptr[l + 1] - tp.level_ptr[l] > kSplitLevel) {
      for (int j = tp.level_ptr[l] + kSL * warp + sq; j < tp.level_ptr[l + 1]; j += kSL * kWarps)
        sbr_simplex_serial<kH>(tp, j, G, V, tj, itj, hl);
      group_sync(wg);
      continue;
    }
    for (int j = tp.level_ptr[l] + kGroups * warp + grp; j < tp.level_ptr[l + 1]; j += kGroups * kWarps) {
      const int s0 = tp.inf_first[j], n = tp.inf_n[j];
      float m = INFINITY;
      for (int i = bl; i < n; i += 2) {
        const int s = s0 + i;
        float gh = G[s * kH + hl];
        for (int c = tp.child_ptr[s]; c < tp.child_ptr[s + 1]; ++c) gh += V[tp.child_idx[c] * kH + hl];
        G[s * kH + hl] = gh;
        m = fminf(m, gh);
      }
      m = fminf(m, __shfl_xor_sync(gmask, m, kH));
      // e_i = exp(-(g_hat_i - m)/t) keeps tiny q_bar accurate; X = sum_i (e_i - 1) via expm1
      // keeps the value accurate: t log q_bar_i* + t log n = -t log1p(X / n)
      const float it = itj[j];
      float sum = 0.f, X = 0.f;
      for (int i = bl; i < n; i += 2) {
        float* u = G + (s0 + i) * kH + hl;
        const float d = -(*u - m) * it;
        const float e = expf(d);
        X += expm1f(d);
        *u = e;
        sum += e;
      }
      // both sub-lanes get partial(0) + partial(1) (addition commutes: the same bits)
      sum += __shfl_xor_sync(gmask, sum, kH);
      X += __shfl_xor_sync(gmask, X, kH);
      const float inv = 1.f / sum;
      for (int i = bl; i < n; i += 2) G[(s0 + i) * kH + hl] *= inv;
      if (bl == 0) V[j * kH + hl] = m - tj[j] * log1pf(X / (float)n);
    }
    group_sync(wg);
  }

  if (a.value_partial != nullptr && warp == 0) {
    double v = 0.0;
    if (live && sq == 0)
      for (int j = tp.level_ptr[0]; j < tp.level_ptr[1]; ++j) v += (double)V[j * kH + hl];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if (lane == 0) *a.value_partial = v;
  }

  if (a.out != nullptr) {
    // top-down: q(s) = q_bar(s) times q_bar of each ancestor sequence (the parent sequence
    // of s's simplex, and so on up to a root simplex).  Once the bottom-up pass has
    // normalised q_bar every (sequence, hand) is independent: no level barriers, and
    // every warp takes rows
    const float tau = a.tau, omt = 1.f - a.tau;
    for (int s = kSL * warp + sq; s < S; s += kWarps * kSL) {
      float q = G[s * kH + hl];
      for (int p = tp.seq_par[s]; p >= 0; p = tp.seq_par[p]) q *= G[p * kH + hl];
      float o = q;
      if (a.old != nullptr) o = omt * O[s * kH + hl] + tau * q;
      a.out[(size_t)s * ld + h] = live ? o : 0.f;
    }
  }
  group_sync(wg);   // shared memory is reused by the caller's next item
}

// Order-preserving integer key of an FP64 value (not NaN): the bits of x >= 0 as they
// are, the magnitude bits of x < 0 inverted, compared as signed int64 (-0 below +0).
// Applying it twice gives x back.  The FP64 compare-and-select is a long dependent
// step on this part's narrow FP64 pipe; the integer minimum is not.
__device__ __forceinline__ long long ord_key(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
__device__ __forceinline__ double ord_key(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffll));
}

// One item of the FP64 best-response value: sign * min over the treeplex of
// <q, sign * g> summed over the item's live hands, written to *value_partial.
// gv as in SbrItemArgs: dense [S][ld] or (contrib) terminal contributions.  Same
// lane layout as sbr_item.
__device__ inline void br64_item(const DevGame& g, const TpxTab& tp, int blk, const double* gv,
                                 bool contrib, const double* grz, double sign,
                                 double* value_partial, double* sm, WarpGroup wg = kWholeCta) {
  constexpr int kH = kSbrHands;
  const int S = tp.S, ld = g.ld;
  const int kWarps = wg.n_warps;
  double* G = sm;                                  // [S][kH]
  double* V = G + (size_t)S * kH;                  // [J][kH]
  const int tid = threadIdx.x - wg.first_warp * 32, lane = threadIdx.x & 31, warp = tid >> 5;
  const int hl = lane % kH, bl = lane / kH;
  const int h0 = blk * kH, h = h0 + hl;
  const bool live = h < g.H;
  const double rz = (contrib && live) ? grz[h] : 0.0;
  {
    constexpr int kU = 4;
    const int kRowStep = kWarps * kSubLanes;
    const bool neg = sign < 0;
    for (int s0 = kSubLanes * warp + bl; s0 < S; s0 += kRowStep * kU) {
      double c0[kU], c1[kU];
      int e0[kU], e1[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int s = s0 + u * kRowStep;
        c0[u] = c1[u] = 0.0;
        e0[u] = e1[u] = 0;
        if (s < S && live) {
          if (contrib) {
            e0[u] = tp.tptr[s];
            e1[u] = tp.tptr[s + 1];
            if (e0[u] < e1[u]) c0[u] = __ldcg(gv + (size_t)e0[u] * ld + h);
            if (e0[u] + 1 < e1[u]) c1[u] = __ldcg(gv + (size_t)(e0[u] + 1) * ld + h);
          } else {
            c0[u] = __ldcg(gv + (size_t)s * ld + h);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int s = s0 + u * kRowStep;
        if (s < S) {
          double v = c0[u];
          if (contrib) {
            double acc = 0.0;
            if (e0[u] < e1[u]) acc += c0[u];
            if (e0[u] + 1 < e1[u]) acc += c1[u];
            for (int e = e0[u] + 2; e < e1[u]; ++e) acc += __ldcg(gv + (size_t)e * ld + h);
            v = neg ? -acc : acc;              // (r / Z of the hand scales the value at the end)
          } else if (neg) {
            v = -v;
          }
          G[s * kH + hl] = v;
        }
      }
    }
  }
  group_sync(wg);
  for (int l = tp.L - 1; l >= 0; --l) {
    if (tp.level_ptr[l + 1] - tp.level_ptr[l] > kSplitLevel) {
      // one simplex per half warp (the minimum is exact: the same value in either form)
      for (int j = tp.level_ptr[l] + kSubLanes * warp + bl; j < tp.level_ptr[l + 1]; j += kSubLanes * kWarps) {
        const int s0 = tp.inf_first[j], n = tp.inf_n[j];
        long long m = ord_key(INFINITY);
        for (int i = 0; i < n; ++i) {
          const int s = s0 + i;
          double gh = G[s * kH + hl];
          for (int c = tp.child_ptr[s]; c < tp.child_ptr[s + 1]; ++c) gh += V[tp.child_idx[c] * kH + hl];
          m = min(m, ord_key(gh));
        }
        V[j * kH + hl] = ord_key(m);
      }
      group_sync(wg);
      continue;
    }
    for (int j = tp.level_ptr[l] + warp; j < tp.level_ptr[l + 1]; j += kWarps) {
      const int s0 = tp.inf_first[j], n = tp.inf_n[j];
      long long m = ord_key(INFINITY);      // the minimum on integer keys (integer pipes)
      for (int i = bl; i < n; i += kSubLanes) {
        const int s = s0 + i;
        double gh = G[s * kH + hl];
        for (int c = tp.child_ptr[s]; c < tp.child_ptr[s + 1]; ++c) gh += V[tp.child_idx[c] * kH + hl];
        m = min(m, ord_key(gh));
      }
      m = min(m, __shfl_xor_sync(0xffffffffu, m, kH));
      if (bl == 0) V[j * kH + hl] = ord_key(m);   // (the key map is its own inverse)
    }
    group_sync(wg);
  }
  if (warp == 0) {
    double v = 0.0;
    if (live && bl == 0) {
      for (int j = tp.level_ptr[0]; j < tp.level_ptr[1]; ++j) v += V[j * kH + hl];
      // a hand's gradient rows all carry its factor r / Z > 0, so its min over the
      // treeplex is r / Z times the min of the unscaled rows: one FP64 product per hand
      // instead of one per (sequence, hand)
      if (contrib) v *= rz;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if (lane == 0) *value_partial = sign * v;
  }
  group_sync(wg);
}

}  // namespace egt
