// Device-resident EGT driver: one cooperative launch runs whole iterations of
// Alg. 1 (theory schedule), practical EGT or Alg. 3 / 4 (EGT/as) -- every phase
// of Alg. 2's Step, the excessive-gap check with its tau back-off, the mu / tau
// bookkeeping and the FP64 stopping residual -- with no host round trip.
//
// The CTAs of a launch are split into groups; each group runs the jobs (games)
// assigned to it one after the other.  Phases are separated by a group barrier;
// the work of a phase (SBR and best-response items of 16 hands, or 8; product items
// of one terminal, or of one opponent column) is spread over the group's CTAs.
// Products stay in terminal-contribution form; the SBR items add a sequence's
// contributions while they load their tile.
// One CTA of the group (the last rank, which holds the fewest items of a phase)
// keeps the solver state (t, mu, tau, buffer index) and takes every decision
// (EGV sign, tau back-off, gap target) from the per-item FP64 partials, summed in
// the same fixed order as the standalone kernels; it publishes each verdict and
// the next schedule in the control block, and the others read them at the next
// attempt's first product barrier.  The group starts each attempt before the
// verdict on the previous one is known (see engine_job), so the sums and the FP64
// decisions are off the other CTAs' critical path.  A run here reproduces the
// host-driven loop of api.cu bit for bit, and a game's iterates do not depend on
// the group size or on the other games of the launch.
//
// The group barrier is a monotone 64-bit arrival counter in the job's control
// block: barrier k completes when it reaches k x (CTAs of the group).  Waits are bounded in time: if one runs
// out (a CTA that never arrives), the kernel records EGT_ERR_TIMEOUT and every
// CTA returns; the host reads the status and the context stays usable.
#include <algorithm>

#include "../../include/egt.h"
#include "egt_internal.cuh"
#include "engine.cuh"
#include "grad_impl.cuh"
#include "sbr_impl.cuh"

namespace egt {
namespace {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

struct GridBar {
  unsigned long long* arrive;   // monotone arrival counter (zeroed by the host per launch)
  int* status;
  unsigned long long expected;  // arrivals per barrier (the grid, unless a test adds phantoms)
  unsigned long long limit_ns;
};

// Phase clock of CTA 0 (thread 0), kept in shared memory and written to the
// control block at exit: per phase, the time from the previous barrier exit to
// this CTA's arrival at the next barrier (its own work) and to the exit.
struct PhaseClock {
  unsigned long long last, arrive;
  unsigned long long ns[kEnginePhases];
  unsigned long long work[kEnginePhases];
  unsigned int n[kEnginePhases];
};

// All CTAs meet here; k counts this CTA's barriers.  Returns false (in every
// thread) if the wait ran out or an error status was recorded.
__device__ bool grid_sync(const GridBar& b, unsigned long long& k, PhaseClock* clk, bool clock_cta) {
  __shared__ int ok_s;
  __syncthreads();
  ++k;
  if (b.expected == 1) {   // a one-CTA group: the CTA barrier is the group barrier
    if (clock_cta && threadIdx.x == 0) clk->arrive = global_ns();
    return true;
  }
  if (threadIdx.x == 0) {
    if (clock_cta) clk->arrive = global_ns();
    int ok = 1;
    // arrival with release semantics at GPU scope: the CTA barrier above ordered every
    // thread's writes of the phase before it (cumulativity), no separate fence needed
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(b.arrive) : "memory");
    const unsigned long long target = k * b.expected;
    unsigned int polls = 0;
    unsigned long long t0 = 0;
    while (ld_acquire(b.arrive) < target) {
      if ((++polls & 1023u) == 0) {
        const unsigned long long now = global_ns();
        if (t0 == 0) {
          t0 = now;
        } else if (now - t0 > b.limit_ns) {
          atomicCAS(b.status, 0, (int)EGT_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        if (ld_volatile(b.status) != 0) {
          ok = 0;
          break;
        }
      }
    }
    // no status read on the way out: a CTA that timed out never arrives again, and
    // the others see its status in the loop above at their next barrier
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Verdicts the deciding CTA publishes on the previous attempt.
constexpr int kGo = 0;      // accepted (or none pending): the running attempt stands
constexpr int kRedo = 1;    // rejected: the running attempt is void, run EngineCtl::redo
constexpr int kStop = 2;    // leave the iteration loop

// grid_sync that also waits for the verdict word of epoch `tag` (published by the
// deciding CTA before its arrival, so the barrier completes with it in sight: the
// word is polled beside the arrival counter) and returns its verdict in *code.
__device__ __forceinline__ bool grid_sync_verdict(const GridBar& b, unsigned long long& k, PhaseClock* clk, bool clock_cta,
                                  const unsigned long long* word, unsigned long long tag, int* code) {
  __shared__ int ok_s, code_s;
  __syncthreads();
  ++k;
  if (threadIdx.x == 0) {
    if (clock_cta) clk->arrive = global_ns();
    const bool group = b.expected != 1;
    int ok = 1;
    if (group) asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(b.arrive) : "memory");
    const unsigned long long target = k * b.expected;
    unsigned long long w = 0;
    unsigned int polls = 0;
    unsigned long long t0 = 0;
    // the deciding CTA publishes the word before it arrives, so once every arrival
    // is in (acquire) the word is read once; it is polled only while still stale
    bool all = !group;
    for (;;) {
      if (!all) all = ld_acquire(b.arrive) >= target;
      if (all) {
        w = ld_acquire(word);
        if ((w >> 8) == tag) break;
      }
      if ((++polls & 1023u) == 0) {
        const unsigned long long now = global_ns();
        if (t0 == 0) {
          t0 = now;
        } else if (now - t0 > b.limit_ns) {
          atomicCAS(b.status, 0, (int)EGT_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        if (ld_volatile(b.status) != 0) {
          ok = 0;
          break;
        }
      }
    }
    ok_s = ok;
    code_s = (int)(w & 0xffu);
  }
  __syncthreads();
  *code = code_s;
  return ok_s != 0;
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Copy a schedule published in the control block (read at L2: another CTA wrote it).
__device__ __forceinline__ void load_sched(EngineSched& dst, const EngineSched* src) {
  const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(&dst);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(EngineSched) / 8); ++i) d[i] = __ldcg(s + i);
}

// CTA 0 books the time since the last mark to `phase` (work done without a barrier).
__device__ __forceinline__ void phase_cut(PhaseClock* c, int phase, bool clock_cta) {
  if (clock_cta && threadIdx.x == 0) {
    const unsigned long long now = global_ns();
    c->ns[phase] += now - c->last;
    c->work[phase] += now - c->last;
    c->n[phase] += 1;
    c->last = now;
  }
}

// End of a phase: grid barrier, then CTA 0 books the phase's time.
__device__ __forceinline__ bool phase_end(const GridBar& b, unsigned long long& k, PhaseClock* c, int phase,
                                          bool clock_cta) {
  if (!grid_sync(b, k, c, clock_cta)) return false;
  if (clock_cta && threadIdx.x == 0) {
    const unsigned long long now = global_ns();
    c->ns[phase] += now - c->last;
    c->work[phase] += c->arrive - c->last;
    c->n[phase] += 1;
    c->last = now;
  }
  return true;
}

// A group of CTAs running one job: this CTA's rank in it and its size.
struct Grp {
  int rank, size;
};

// Tables staged once per job at the start of shared memory.
struct Tabs {
  GradTab grad;
  TpxTab tpx[2];
};

__host__ __device__ inline size_t tabs_bytes(const DevGame& g) {
  return grad_tab_bytes(g) + tpx_tab_bytes(g, 0) + tpx_tab_bytes(g, 1);
}

// Field-by-field selection (a runtime index into a struct array would force a
// local-memory copy of the array)
__device__ __forceinline__ TpxTab pick(const Tabs& tb, int p) {
  const TpxTab& a = tb.tpx[0];
  const TpxTab& c = tb.tpx[1];
  TpxTab t;
  t.S = p ? c.S : a.S;
  t.J = p ? c.J : a.J;
  t.L = p ? c.L : a.L;
  t.beta = p ? c.beta : a.beta;
  t.level_ptr = p ? c.level_ptr : a.level_ptr;
  t.inf_first = p ? c.inf_first : a.inf_first;
  t.inf_n = p ? c.inf_n : a.inf_n;
  t.seq_par = p ? c.seq_par : a.seq_par;
  t.child_ptr = p ? c.child_ptr : a.child_ptr;
  t.child_idx = p ? c.child_idx : a.child_idx;
  t.tptr = p ? c.tptr : a.tptr;
  return t;
}

// Shared memory of one SBR / best-response item of either player (a warp half's share
// when items run in pairs).
__device__ __forceinline__ size_t pair_half_bytes(const DevGame& g) {
  size_t m = 0;
  for (int p = 0; p < 2; ++p) m = max(m, max(sbr_item_smem(g, p), br_item_smem(g, p)));
  return gradimpl::align16(m);
}

// The items of an SBR / best-response phase this CTA takes: one at a time on the whole
// CTA, or (pairs) two at a time, one per warp half with its own named barrier, when the
// job allows it and the group has at least two items per CTA.  Calls f(item, wg, smem).
template <typename F>
__device__ __forceinline__ void for_items(const DevGame& g, Grp gr, int n_items, bool pair_ok, unsigned char* sm,
                                          F f) {
  const bool pair = pair_ok && 2 * gr.size <= n_items;
  if (!pair) {
    for (int item = gr.rank; item < n_items; item += gr.size) f(item, WarpGroup{0, kItemThreads / 32, 0}, sm);
    return;
  }
  constexpr int kHalf = kItemThreads / 64;
  const int half = (int)(threadIdx.x >> 5) >= kHalf ? 1 : 0;
  const WarpGroup wg{half * kHalf, kHalf, 1 + half};
  unsigned char* hs = sm + half * pair_half_bytes(g);
  for (int base = 2 * gr.rank; base < n_items; base += 2 * gr.size)
    if (base + half < n_items) f(base + half, wg, hs);
}

// One SBR phase: all kH-hand items of `player`, spread over the CTAs; gv holds the
// player's terminal contributions (or is NULL).
template <int kH = kSbrHands>
__device__ __forceinline__ void run_sbr(const DevGame& g, const Tabs& tb, Grp gr, bool pair_ok, int player,
                                        const float* gv, double mu, const float* old, float tau, float* out,
                                        double* partials, unsigned char* sm) {
  const int NB = g.ld / kH;
  const TpxTab tp = pick(tb, player);
  for_items(g, gr, NB, pair_ok, sm, [&](int item, const WarpGroup& wg, unsigned char* ism) {
    SbrItemArgs a;
    a.g = gv;
    a.contrib = true;
    a.grz = player ? g.rz[1] : g.rz[0];
    a.sign = player == 0 ? 1.f : -1.f;
    a.mu = mu;
    a.old = old;
    a.tau = tau;
    a.out = out;
    a.value_partial = partials ? partials + item : nullptr;
    sbr_item<kH>(g, tp, item, a, reinterpret_cast<float*>(ism), wg);
  });
}

// An SBR phase without value partials: in the one-game merged kernel, 8-hand items where
// one round of them fits the group (twice the items, each half the work: the large
// game's 136 items on 148 CTAs instead of 68), else 16-hand items.  The same bits.
template <int kProd>
__device__ __forceinline__ void run_sbr_plain(const DevGame& g, const Tabs& tb, Grp gr, bool pair_ok, int player,
                                              const float* gv, double mu, const float* old, float tau, float* out,
                                              unsigned char* sm) {
  if constexpr (kProd == 3) {
    if (!pair_ok && g.ld / 8 <= gr.size) {
      run_sbr<8>(g, tb, gr, pair_ok, player, gv, mu, old, tau, out, nullptr, sm);
      return;
    }
  }
  run_sbr<kSbrHands>(g, tb, gr, pair_ok, player, gv, mu, old, tau, out, nullptr, sm);
}

// Product items of a phase of `player`: one per terminal when the group has a CTA for
// every terminal, else one per opponent column, whose showdown and fold terminals share
// the column's sums (less work per phase; in batches, where a group runs many items per
// phase, this measured faster even where it saves no round of items).  The one-game
// driver picks its kernel by merge_items instead.  The results are the same bits either
// way (the sums are exact).
__device__ __forceinline__ int prod_items(const DevTerms& tm, Grp gr, bool& merged) {
  merged = gr.size < tm.n;
  return merged ? tm.n_col : tm.n;
}

// One product phase: every terminal of `player`'s grouping; c64 (FP64 contributions
// for the residual) may be NULL.  With pairs (the job allows them and the group has at
// least two items per CTA) each warp half takes its own items.
// kProd selects the product items: 0, one terminal per item (term_item_whole), the
// one-game kernel's items when every terminal of a phase has its own CTA; 2,
// prod_item, merged per opponent column when the group has fewer CTAs than
// terminals, the CTAs taking the items round-robin (batches); 3, the same items in
// rounds of alternating direction (round_unit: the one-game kernel when its CTAs are
// fewer than its terminals).  The results are the same bits in every form.
template <int kProd>
__device__ __forceinline__ void one_prod_item(const DevGame& g, const GradTab& tb, int player, int item,
                                              bool merged, const float* in, float* c32, double* c64,
                                              unsigned char* sm) {
  if constexpr (kProd == 0) term_item_whole<float>(g, tb, player, item, in, c32, c64, sm);
  else prod_item<float>(g, tb, player, item, merged, in, c32, c64, sm);
}

// The unit (item, or pair of items) this CTA takes in round r of `rounds` rounds of
// gr.size units: the rounds alternate direction and the last one, which may be partial,
// runs from rank 0 up, so the group's last rank (the deciding CTA) holds the fewest
// units, and units in descending order of work (merged product items are: a showdown
// and a fold, a showdown alone, a fold alone: DevTerms::col_order) give every CTA
// about the same total, where taking them round-robin gives rank 0 the largest of
// every round.
__device__ __forceinline__ int round_unit(int r, int rounds, Grp gr) {
  return r * gr.size + (((rounds - 1 - r) & 1) ? gr.size - 1 - gr.rank : gr.rank);
}

template <int kProd>
__device__ __forceinline__ void run_grad(const DevGame& g, const Tabs& tb, Grp gr, bool pair_ok, int player,
                                         const float* in, float* c32, double* c64, unsigned char* sm) {
  const DevTerms tm = player ? g.terms[1] : g.terms[0];
  bool merged;
  int n = prod_items(tm, gr, merged);
  if (kProd == 0 && merged) {
    merged = false;
    n = tm.n;
  }
  if (!(pair_ok && 2 * gr.size <= n)) {
    if constexpr (kProd == 3) {
      const int rounds = (n + gr.size - 1) / gr.size;
      for (int r = 0; r < rounds; ++r) {
        const int u = round_unit(r, rounds, gr);
        if (u < n) one_prod_item<kProd>(g, tb.grad, player, merged ? tm.col_order[u] : u, merged, in, c32, c64, sm);
      }
    } else {
      for (int item = gr.rank; item < n; item += gr.size)
        one_prod_item<kProd>(g, tb.grad, player, item, merged, in, c32, c64, sm);
    }
    return;
  }
  constexpr int kHalf = kItemThreads / 64;
  const int half = (int)(threadIdx.x >> 5) >= kHalf ? 1 : 0;
  unsigned char* hs = sm + half * gradimpl::align16(grad_item_smem(g));
  auto pair_item = [&](int base) {
    if (base + half < n) {
      if constexpr (kProd == 0) {
        term_item_whole<float, kItemThreads / 2>(g, tb.grad, player, base + half, in, c32, c64, hs,
                                                 half * kHalf, 1 + half);
      } else {
        const int item = kProd == 3 && merged ? tm.col_order[base + half] : base + half;
        prod_item<float, kItemThreads / 2>(g, tb.grad, player, item, merged, in, c32, c64, hs,
                                           half * kHalf, 1 + half);
      }
    }
  };
  if constexpr (kProd == 3) {
    const int n_pairs = (n + 1) / 2;
    const int rounds = (n_pairs + gr.size - 1) / gr.size;
    for (int r = 0; r < rounds; ++r) pair_item(2 * round_unit(r, rounds, gr));
  } else {
    for (int base = 2 * gr.rank; base < n; base += 2 * gr.size) pair_item(base);
  }
}

// Item `item` of player p's FP64 best response of the residual (player 0: min over x of
// <x, A y>, player 1: max over y of <y, A^T x>), its partial to partBR0 / partBR1.
__device__ __forceinline__ void run_br_item(const DevGame& g, const Tabs& tb, int p, int item,
                                            const EngineBufs& b, double* partBR0, double* partBR1,
                                            unsigned char* sm, const WarpGroup& wg) {
  if (p == 0)
    br64_item(g, tb.tpx[0], item, b.g64[0], true, g.rz64[0], 1.0, partBR0 + item,
              reinterpret_cast<double*>(sm), wg);
  else
    br64_item(g, tb.tpx[1], item, b.g64[1], true, g.rz64[1], -1.0, partBR1 + item,
              reinterpret_cast<double*>(sm), wg);
}

// Fixed-order sums of the per-item partial arrays [first, last) (each of n
// values, consecutive in p): warp k of every CTA sums array first + k, the CTA
// shares the results in red[first .. last).
__device__ __forceinline__ void reduce_arrays(const double* p, int n, int first, int last, double* red) {
  __shared__ double s[4];
  const int w = threadIdx.x >> 5;
  if (w < last - first) {
    const double v = reduce_partials(p + (size_t)(first + w) * n, n, threadIdx.x & 31);
    if ((threadIdx.x & 31) == 0) s[first + w] = v;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (k >= first && k < last) red[k] = s[k];
  __syncthreads();
}

// Player to step and tau of iteration t (Alg. 1: alternate by parity, tau_t = 2/(t+3);
// practical EGT: the player with the larger mu, same tau; EGT/as: that player, the
// carried tau).
__device__ __forceinline__ void choose(int variant, int t, double mu0, double mu1, double tau_as, int& me,
                                       double& tau) {
  if (variant == EGT_AS) {   // (no division on the EGT/as path: FP64 is a narrow pipe here)
    me = mu0 > mu1 ? 0 : 1;
    tau = tau_as;
  } else if (variant == EGT_THEORY) {
    me = t % 2 == 0 ? 0 : 1;
    tau = 2.0 / (t + 3);
  } else {
    me = mu0 > mu1 ? 0 : 1;
    tau = 2.0 / (t + 3);
  }
}

using Sched = EngineSched;

// The solver's scalar state (t, mu, tau, buffer index, counters, the attempt in
// flight), kept in shared memory by thread 0 of the group's deciding CTA.  Every CTA
// starts from the control block and plans the first attempt itself; after that only
// the decider advances the state and publishes each verdict and schedule (FP64 is a
// narrow pipe on this part: one thread of one CTA takes the decisions, off the
// critical path of the other CTAs).
struct Solver {
  double mu0, mu1, tau_as, gap, eps_mbb, mbb_scale;
  double tau, egv, mu_next, last_tau, last_egv;
  int t, cur, it, done, backoffs_total, products, gap_checks, reached, status;
  int last_player, last_backoffs, me, backoffs, spec, gap_due, pre, new_iter;
};

struct LoopCfg {
  int variant, n_iters, gap_every, max_t;
  bool check;   // EGT/as: the excessive-gap check decides acceptance
};

// Start an attempt from the state: the loop's stop test, the player and tau of a new
// iteration, and the attempt's schedule.  The next iteration's choice if this attempt
// is accepted decides where its v_hat is computed ahead: with the last product when
// the same player steps again (its gradient and iterate are final there), else in the
// last phase, from the same smoothed best response as the other's EGV part (same
// gradient, same mu).
__device__ __forceinline__ Sched plan_attempt(Solver& s, const LoopCfg& k) {
  Sched sc;
  sc.stop = !(s.it < k.n_iters && s.status == 0) || (s.it > 0 && s.new_iter && (s.reached || s.t >= k.max_t));
  sc.cur = sc.me = sc.gap_due = sc.spec = sc.pre = 0;
  sc.tau = sc.tau2 = 0.f;
  sc.mu_me = sc.mu_ot = sc.mu_tilde = 0.0;
  if (sc.stop) return sc;
  if (s.new_iter) {
    choose(k.variant, s.t, s.mu0, s.mu1, s.tau_as, s.me, s.tau);
    s.backoffs = 0;
    s.egv = 0.0 / 0.0;
  }
  const bool xs = s.me == 0;
  s.gap_due = (s.t + 1) % k.gap_every == 0 || s.t + 1 >= k.max_t;
  s.mu_next = (1 - s.tau) * (xs ? s.mu0 : s.mu1);   // mu of the stepping player if accepted
  int me2;
  double tau2;
  choose(k.variant, s.t + 1, xs ? s.mu_next : s.mu0, xs ? s.mu1 : s.mu_next, s.tau, me2, tau2);
  s.spec = me2 == s.me ? 1 : (k.check || s.gap_due ? 2 : 0);
  sc.cur = s.cur;
  sc.me = s.me;
  sc.gap_due = s.gap_due;
  sc.spec = s.spec;
  sc.pre = s.pre;
  sc.tau = (float)s.tau;
  sc.tau2 = (float)tau2;
  sc.mu_me = xs ? s.mu0 : s.mu1;
  sc.mu_ot = xs ? s.mu1 : s.mu0;
  sc.mu_tilde = s.mu_next;
  return sc;
}

// Alg. 2's last lines for an accepted attempt: mu_me^+ = (1 - tau) mu_me (computed with
// the attempt), swap the iterate buffers, count.
__device__ __forceinline__ void accept_attempt(Solver& s, int variant) {
  if (s.me == 0) s.mu0 = s.mu_next;
  else s.mu1 = s.mu_next;
  if (variant == EGT_AS) s.tau_as = s.tau;
  s.cur = 1 - s.cur;
  s.t += 1;
  s.backoffs_total += s.backoffs;
  s.done += 1;
  s.last_player = s.me;
  s.last_backoffs = s.backoffs;
  s.last_tau = s.tau;
  s.last_egv = s.egv;
  s.pre = s.spec != 0;
  s.it += 1;
  s.new_iter = 1;
}

// The verdict on the attempt in flight from its sums red (EGV parts, residual values):
// accept (Alg. 2, then the residual of the new point when it was due), or halve tau and
// retry (Alg. 4's Decr).  Returns true if accepted.
__device__ __forceinline__ bool decide(Solver& s, const LoopCfg& k, const double* red, const EngineBufs& b) {
  s.products += 3;
  bool accept = true;
  if (k.check) {
    const double phi = s.me == 0 ? red[0] : red[1], negf = s.me == 0 ? red[1] : red[0];
    s.egv = phi + negf;
    if (!isfinite(s.egv)) {
      s.status = EGT_ERR_NUMERIC;
      accept = false;
    } else if (s.egv < 0) {
      accept = false;
      s.tau *= 0.5;
      if (s.tau < 1.0 / (1u << 30)) s.status = EGT_ERR_TAU_UNDERFLOW;
      else ++s.backoffs;
    }
  }
  if (!accept) {
    s.pre = 0;
    s.new_iter = 0;
    return false;
  }
  if (b.log != nullptr && s.it < b.log_cap) {
    egt_iter_log& L = b.log[s.it];
    L.t = s.t;
    L.player = s.me;
    L.backoffs = s.backoffs;
    L.tau = s.tau;
    L.mu[0] = s.me == 0 ? s.mu_next : s.mu0;
    L.mu[1] = s.me == 0 ? s.mu1 : s.mu_next;
    L.egv = k.check ? s.egv : 0.0 / 0.0;
    L.gap_mbb = s.gap;
    L.time_ns = global_ns();
  }
  const int gap_due = s.gap_due;
  accept_attempt(s, k.variant);
  if (gap_due) {
    // eps_sad of the new iterates from the FP64 products of the Step:
    // max_y <y, A^T x> - min_x <x, A y>
    s.gap = (red[3] - red[2]) * s.mbb_scale;
    s.gap_checks += 1;
    if (!isfinite(s.gap)) s.status = EGT_ERR_NUMERIC;
    else s.reached = s.eps_mbb > 0 && s.gap <= s.eps_mbb ? 1 : 0;
  }
  return true;
}

// The deciding CTA's thread 0: the verdict on the pending attempt (if any) from its
// sums red, then, unless that voids or ends the running attempt, the schedule of the
// attempt after the running one (as if the running one is accepted); published with
// the verdict word of epoch ep.
__device__ __forceinline__ void settle(Solver& S, Solver& S2, EngineCtl* ctl, const EngineBufs& b, const double* red,
                                    bool pending, bool stop_now, unsigned int ep) {
  const LoopCfg kc{ctl->variant, ctl->n_iters, ctl->gap_every, ctl->max_t, ctl->variant == EGT_AS};
  int code = kGo;
  if (pending) {
    const bool acc = decide(S, kc, red, b);
    const Sched x = plan_attempt(S, kc);
    if (x.stop) {
      code = kStop;
    } else if (!acc) {
      code = kRedo;
      ctl->redo = x;
    }
  }
  if (code == kGo && !stop_now) {
    S2 = S;
    accept_attempt(S2, kc.variant);
    ctl->next = plan_attempt(S2, kc);
  }
  st_release(&ctl->verdict, ((unsigned long long)ep << 8) | (unsigned long long)code);
}

// One job (game) run by the group `gr`: its tables staged in smem_all, then up to
// ctl->n_iters iterations.  Returns when the job stops or fails (status recorded).
//
// The verdict on an attempt (its EGV sign, the residual against the target) needs the
// sums of the attempt's last phase.  The group does not wait for it: right after that
// phase every CTA starts the next attempt as if the verdict were "accepted, continue"
// (its schedule was published one attempt ahead), while the deciding CTA (the last
// rank, which holds the fewest items of a phase) sums the partials, takes the
// verdict and publishes it before it arrives at the new attempt's first product
// barrier.  Everything the new attempt writes before that barrier is scratch (the
// v_hat buffer and the other player's gradient at v_hat), so a rejected attempt is
// retried from unchanged iterates, and a stop discards only scratch.
template <int kProd>
__device__ __forceinline__ void engine_job(const DevGame& g, const EngineBufs& b, EngineCtl* ctl, Grp gr,
                                           int pair_bits, unsigned long long expected,
                                           unsigned long long limit_ns, unsigned char* smem_all) {
  const bool pair_ok = (pair_bits & kPairSbr) != 0, pair_terms = (pair_bits & kPairTerms) != 0;
  Tabs tb;
  tb.grad = stage_grad_tab(g, smem_all);
  tb.tpx[0] = stage_tpx_tab(g, 0, smem_all + grad_tab_bytes(g));
  tb.tpx[1] = stage_tpx_tab(g, 1, smem_all + grad_tab_bytes(g) + tpx_tab_bytes(g, 0));
  // (the tables are first read after the CTA barrier at the top of the iteration loop)
  unsigned char* sm = smem_all + tabs_bytes(g);   // per-phase working area
  const GridBar bar{&ctl->bar_arrive, &ctl->status, expected, limit_ns};
  unsigned long long bk = 0;                      // barriers passed by this CTA
  __shared__ PhaseClock clk_s;
  __shared__ Sched sc, sc_next;                   // the running attempt; the one after it
  __shared__ Solver S, S2;                        // thread 0 (advanced by the decider only)
  PhaseClock* clk = &clk_s;
  const bool lead = threadIdx.x == 0;
  const bool clock_cta = gr.rank == 0 && ctl->trace != 0;
  const bool decider = gr.rank == gr.size - 1;
  const int NB = g.ld / kSbrHands;
  double* partA = b.partials;
  double* partB = b.partials + NB;
  double* partBR0 = b.partials + 2 * NB;
  double* partBR1 = b.partials + 3 * NB;
  const bool check = ctl->variant == EGT_AS;

  if (lead) {
    clk->last = global_ns();
    clk->arrive = clk->last;
    for (int k = 0; k < kEnginePhases; ++k) {
      clk->ns[k] = 0;
      clk->work[k] = 0;
      clk->n[k] = 0;
    }
    S.t = ctl->t;
    S.cur = ctl->cur;
    S.mu0 = ctl->mu[0];
    S.mu1 = ctl->mu[1];
    S.tau_as = ctl->tau;
    S.gap = ctl->gap_mbb;
    S.eps_mbb = ctl->eps_mbb;
    S.mbb_scale = ctl->mbb_scale;
    S.tau = 0;
    S.egv = S.last_tau = S.last_egv = 0.0 / 0.0;
    S.mu_next = 0;
    S.it = S.done = S.backoffs_total = S.products = S.gap_checks = S.reached = S.status = 0;
    S.last_player = -1;
    S.last_backoffs = S.me = S.backoffs = S.spec = S.gap_due = S.pre = 0;
    S.new_iter = 1;
    const LoopCfg kc{ctl->variant, ctl->n_iters, ctl->gap_every, ctl->max_t, check};
    sc = plan_attempt(S, kc);   // the same in every CTA
  }

  bool pending = false;      // the previous attempt awaits its verdict
  bool pend_sums = false;    // ... and its verdict needs the sums of its last phase
  int pend_gap = 0;          // ... which include the residual's best responses
  unsigned int ep = 0;       // verdict epochs (one per attempt)
  for (;;) {
    __syncthreads();
    const bool stop_now = sc.stop != 0;
    if (stop_now && !pending) break;
    ++ep;
    const int c = sc.cur, m = sc.me, gap_due = sc.gap_due, sp = sc.spec;
    const bool have_hat = sc.pre != 0;
    const bool tail = check || gap_due;              // a phase after the Step's last product

    // the decider: the verdict on the previous attempt, then (unless it voids or ends
    // the running one) the schedule of the attempt after the running one
    if (decider) {
      double red[4] = {0.0, 0.0, 0.0, 0.0};
      // the EGV parts (partA, partB) and the residual's values (partBR0, partBR1) in one pass
      if (pending && pend_sums) reduce_arrays(b.partials, NB, check ? 0 : 2, pend_gap ? 4 : 2, red);
      if (lead) settle(S, S2, ctl, b, red, pending, stop_now, ep);
    }
    phase_cut(clk, 7, clock_cta);
    if (stop_now) {
      // the schedule said stop if the previous attempt is accepted: its verdict decides
      // between stopping and retrying it
      int code = kStop;
      if (!grid_sync_verdict(bar, bk, clk, clock_cta, &ctl->verdict, ep, &code)) return;
      if (code != kRedo) break;
      if (lead) load_sched(sc, &ctl->redo);
      pending = false;
      continue;
    }

    // Alg. 2 Step focused on m (the y-focused step swaps roles, A -> -A^T)
    const int ot = 1 - m;
    const bool xs = m == 0;
    float* xc = c ? b.x[1] : b.x[0];
    float* xn = c ? b.x[0] : b.x[1];
    float* yc = c ? b.y[1] : b.y[0];
    float* yn = c ? b.y[0] : b.y[1];
    float* gxc = c ? b.gx[1] : b.gx[0];
    float* gxn = c ? b.gx[0] : b.gx[1];
    float* gyc = c ? b.gy[1] : b.gy[0];
    float* gyn = c ? b.gy[0] : b.gy[1];
    float* v_me = xs ? xc : yc;                      // my iterate
    float* v_ot = xs ? yc : xc;                      // the other's iterate
    float* v_me_n = xs ? xn : yn;
    float* v_ot_n = xs ? yn : xn;
    float* g_me = xs ? gxc : gyc;                    // my loss gradient at v_ot
    float* g_me_n = xs ? gxn : gyn;
    float* g_ot_n = xs ? gyn : gxn;
    float* t_me = xs ? b.tx : b.ty;
    float* t_ot = xs ? b.ty : b.tx;
    // the residual of the new point is due: the Step's products of y_+ and x_+ also
    // write their FP64 copies, and the best responses run in the last phase
    double* g64_me = gap_due ? (xs ? b.g64[0] : b.g64[1]) : nullptr;
    double* g64_ot = gap_due ? (xs ? b.g64[1] : b.g64[0]) : nullptr;

    // v_hat = (1 - tau) v + tau v_mu(other)
    if (!have_hat) {
      run_sbr_plain<kProd>(g, tb, gr, pair_ok, m, g_me, sc.mu_me, v_me, sc.tau, t_me, sm);
      if (!phase_end(bar, bk, clk, 0, clock_cta)) return;
    }
    phase_cut(clk, 8, clock_cta);
    run_grad<kProd>(g, tb, gr, pair_terms, ot, t_me, t_ot, nullptr, sm);   // the other's loss gradient at v_hat
    {
      int code = kGo;
      if (!grid_sync_verdict(bar, bk, clk, clock_cta, &ctl->verdict, ep, &code)) return;
      if (clock_cta && lead) {
        const unsigned long long now = global_ns();
        clk->ns[1] += now - clk->last;
        clk->work[1] += clk->arrive - clk->last;
        clk->n[1] += 1;
        clk->last = now;
      }
      if (code == kStop) break;
      if (code == kRedo) {
        // the previous attempt was rejected: this one is void (it wrote scratch only)
        if (lead) load_sched(sc, &ctl->redo);
        pending = false;
        continue;
      }
      if (lead) load_sched(sc_next, &ctl->next);   // (first read at the end of the attempt)
    }
    // other_+ = (1 - tau) other + tau other_mu(v_hat)
    run_sbr_plain<kProd>(g, tb, gr, pair_ok, ot, t_ot, sc.mu_ot, v_ot, sc.tau, v_ot_n, sm);
    if (!phase_end(bar, bk, clk, 2, clock_cta)) return;
    run_grad<kProd>(g, tb, gr, pair_terms, m, v_ot_n, g_me_n, g64_me, sm);   // my loss gradient at other_+
    if (!phase_end(bar, bk, clk, 3, clock_cta)) return;
    // v_tilde = v_{(1-tau) mu}(other_+), v_+ = (1 - tau) v + tau v_tilde; value: my EGV part.
    // When the residual is due, my FP64 best response (on the FP64 product of the last
    // phase) runs beside it as items [NB, 2 NB).
    {
      const int n_items = gap_due ? 2 * NB : NB;
      const TpxTab tp = pick(tb, m);
      for_items(g, gr, n_items, pair_ok, sm, [&](int item, const WarpGroup& wg, unsigned char* ism) {
        if (item < NB) {
          SbrItemArgs a;
          a.g = g_me_n;
          a.contrib = true;
          a.grz = m ? g.rz[1] : g.rz[0];
          a.sign = m == 0 ? 1.f : -1.f;
          a.mu = sc.mu_tilde;
          a.old = v_me;
          a.tau = sc.tau;
          a.out = v_me_n;
          a.value_partial = partA + item;
          sbr_item(g, tp, item, a, reinterpret_cast<float*>(ism), wg);
        } else {
          run_br_item(g, tb, m, item - NB, b, partBR0, partBR1, ism, wg);
        }
      });
    }
    if (!phase_end(bar, bk, clk, 4, clock_cta)) return;
    if (sp != 1) {
      run_grad<kProd>(g, tb, gr, pair_terms, ot, v_me_n, g_ot_n, g64_ot, sm);   // the other's at v_+
    } else {
      // the other's loss gradient at v_+, and the next v_hat (the same player steps again)
      const DevTerms tmo = ot ? g.terms[1] : g.terms[0];
      bool merged;
      int T = prod_items(tmo, gr, merged);
      if (kProd == 0 && merged) {
        merged = false;
        T = tmo.n;
      }
      const int n_items = T + NB;
      for (int item = gr.rank; item < n_items; item += gr.size) {
        if (item < T) {
          one_prod_item<kProd>(g, tb.grad, ot, item, merged, v_me_n, g_ot_n, g64_ot, sm);
        } else {
          SbrItemArgs a;
          a.g = g_me_n;
          a.contrib = true;
          a.grz = m ? g.rz[1] : g.rz[0];
          a.sign = m == 0 ? 1.f : -1.f;
          a.mu = sc.mu_tilde;
          a.old = v_me_n;
          a.tau = sc.tau2;
          a.out = t_me;
          a.value_partial = nullptr;
          sbr_item(g, pick(tb, m), item - T, a, reinterpret_cast<float*>(sm));
        }
      }
    }
    if (!phase_end(bar, bk, clk, 5, clock_cta)) return;
    if (tail) {
      // the other's EGV part and / or the next v_hat (items [0, NB)), the other's FP64
      // best response when the residual is due (the following NB items)
      const int n_sbr = check || sp == 2 ? NB : 0;
      const int n_items = n_sbr + (gap_due ? NB : 0);
      const TpxTab tp = pick(tb, ot);
      for_items(g, gr, n_items, pair_ok, sm, [&](int item, const WarpGroup& wg, unsigned char* ism) {
        if (item < n_sbr) {
          SbrItemArgs a;
          a.g = g_ot_n;
          a.contrib = true;
          a.grz = ot ? g.rz[1] : g.rz[0];
          a.sign = ot == 0 ? 1.f : -1.f;
          a.mu = sc.mu_ot;
          a.old = sp == 2 ? v_ot_n : nullptr;
          a.tau = sp == 2 ? sc.tau2 : 0.f;
          a.out = sp == 2 ? t_ot : nullptr;
          a.value_partial = check ? partB + item : nullptr;
          sbr_item(g, tp, item, a, reinterpret_cast<float*>(ism), wg);
        } else {
          run_br_item(g, tb, ot, item - n_sbr, b, partBR0, partBR1, ism, wg);
        }
      });
      if (!phase_end(bar, bk, clk, 6, clock_cta)) return;
    }
    // the next attempt starts at once, on the schedule published for "accepted"
    pending = true;
    pend_sums = tail;
    pend_gap = gap_due;
    if (lead) sc = sc_next;
  }

  if (decider && lead) {
    ctl->t = S.t;
    ctl->cur = S.cur;
    ctl->mu[0] = S.mu0;
    ctl->mu[1] = S.mu1;
    ctl->tau = S.tau_as;
    ctl->gap_mbb = S.gap;
    ctl->reached = S.reached;
    ctl->done_iters = S.done;
    ctl->backoffs = S.backoffs_total;
    ctl->products = S.products;
    ctl->gap_checks = S.gap_checks;
    ctl->last_player = S.last_player;
    ctl->last_tau = S.last_tau;
    ctl->last_backoffs = S.last_backoffs;
    ctl->last_egv = S.last_egv;
    if (S.status != 0) atomicCAS(&ctl->status, 0, S.status);
  }
  if (clock_cta && lead) {
#pragma unroll
    for (int k = 0; k < kEnginePhases; ++k) {
      ctl->phase_ns[k] = clk->ns[k];
      ctl->phase_work_ns[k] = clk->work[k];
      ctl->phase_n[k] = clk->n[k];
    }
  }
}

// One job on the whole grid, its description in the kernel parameters: a CTA for every
// terminal of a product phase (one terminal per item) ...
__global__ void __launch_bounds__(kItemThreads, 1)
    engine_kernel_one(EngineJob job, unsigned int extra, unsigned long long limit_ns) {
  extern __shared__ __align__(16) unsigned char smem_all[];
  engine_job<0>(job.g, job.b, job.ctl, Grp{(int)blockIdx.x, (int)gridDim.x}, job.pair,
                (unsigned long long)gridDim.x + extra, limit_ns, smem_all);
}

// ... or fewer CTAs than terminals (items merged per opponent column).  Two kernels
// rather than one with both item bodies: the second body in the first kernel cost
// its games 1.4 % of their iteration rate.
__global__ void __launch_bounds__(kItemThreads, 1)
    engine_kernel_one_merged(EngineJob job, unsigned int extra, unsigned long long limit_ns) {
  extern __shared__ __align__(16) unsigned char smem_all[];
  engine_job<3>(job.g, job.b, job.ctl, Grp{(int)blockIdx.x, (int)gridDim.x}, job.pair,
                (unsigned long long)gridDim.x + extra, limit_ns, smem_all);
}

// CTA groups of a launch as the plan gives them (group q: CTAs [first, first +
// size), jobs [job0, job1) in turn).  Each job's game description and buffers
// are copied to shared memory first.
__global__ void __launch_bounds__(kItemThreads, 1)
    engine_kernel(const EngineJob* __restrict__ jobs, const EngineGroup* __restrict__ plan, int n_groups,
                  unsigned int extra, unsigned long long limit_ns) {
  extern __shared__ __align__(16) unsigned char smem_all[];
  __shared__ __align__(16) EngineJob job_s;
  int q = 0;
  while (q < n_groups && !(plan[q].first <= (int)blockIdx.x && (int)blockIdx.x < plan[q].first + plan[q].size))
    ++q;
  if (q == n_groups) return;
  const EngineGroup pg = plan[q];
  const Grp gr{(int)blockIdx.x - pg.first, pg.size};
  for (int j = pg.job0; j < pg.job1; ++j) {
    __syncthreads();   // the previous job's readers of job_s are done
    {
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(jobs + j);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&job_s);
      for (int i = threadIdx.x; i < (int)(sizeof(EngineJob) / 8); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    engine_job<2>(job_s.g, job_s.b, job_s.ctl, gr, job_s.pair, (unsigned long long)pg.size + extra, limit_ns,
               smem_all);
  }
}

}  // namespace

size_t engine_smem_bytes(const DevGame& g, int pair_bits) {
  size_t m = 0;
  for (int p = 0; p < 2; ++p) {
    m = std::max(m, sbr_item_smem(g, p));
    m = std::max(m, br_item_smem(g, p));
  }
  size_t need = std::max(m, grad_item_smem(g));
  if (pair_bits & kPairSbr) need = std::max(need, 2 * gradimpl::align16(m));
  if (pair_bits & kPairTerms) need = std::max(need, 2 * gradimpl::align16(grad_item_smem(g)));
  return tabs_bytes(g) + need;
}

cudaError_t engine_launch_one(const EngineJob& job, int grid, size_t smem, unsigned int extra,
                              unsigned long long limit_ns, cudaStream_t st) {
  EngineJob j = job;
  unsigned int ex = extra;
  unsigned long long lim = limit_ns;
  void* args[] = {&j, &ex, &lim};
  const bool merged = merge_items(job.g.terms[0].n, job.g.terms[0].n_col, grid) ||
                      merge_items(job.g.terms[1].n, job.g.terms[1].n_col, grid);
  return cudaLaunchCooperativeKernel(merged ? (const void*)engine_kernel_one_merged : (const void*)engine_kernel_one,
                                     dim3(grid), dim3(kItemThreads), args, smem, st);
}

cudaError_t engine_launch(const EngineJob* jobs_dev, const EngineGroup* plan_dev, int n_groups, int grid,
                          size_t smem, unsigned int extra, unsigned long long limit_ns, cudaStream_t st) {
  int ng = n_groups;
  unsigned int ex = extra;
  unsigned long long lim = limit_ns;
  void* args[] = {(void*)&jobs_dev, (void*)&plan_dev, &ng, &ex, &lim};
  return cudaLaunchCooperativeKernel((const void*)engine_kernel, dim3(grid), dim3(kItemThreads), args,
                                     smem, st);
}

int engine_smem_limit(bool batch) {
  if (batch) return opt_in_dynamic_smem((const void*)engine_kernel);
  return std::min(opt_in_dynamic_smem((const void*)engine_kernel_one),
                  opt_in_dynamic_smem((const void*)engine_kernel_one_merged));
}

int engine_max_grid(size_t smem, bool batch) {
  const int limit = engine_smem_limit(batch);
  if (limit < 0) return -1;
  if (smem > (size_t)limit) return 0;
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess)
    return -1;
  cudaError_t e;
  if (batch) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, engine_kernel, kItemThreads, smem);
  } else {
    int per_sm2 = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, engine_kernel_one, kItemThreads, smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, engine_kernel_one_merged, kItemThreads, smem);
    per_sm = std::min(per_sm, per_sm2);
  }
  if (e != cudaSuccess) return -1;
  if (!coop) return 0;
  return sms * per_sm;
}

int engine_items(const DevGame& g) {
  const int NB = g.ld / kSbrHands;
  // widest phase: the last product with the next v_hat, or an SBR phase with one of
  // the residual's best responses
  return std::max(2 * NB, std::max(g.terms[0].n, g.terms[1].n) + NB);
}

}  // namespace egt
