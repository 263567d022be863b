// Device-resident EGT driver: one cooperative launch runs whole iterations of
// Alg. 1 (theory schedule), practical EGT or Alg. 3 / 4 (EGT/as) -- every phase
// of Alg. 2's Step, the excessive-gap check with its tau back-off, the mu / tau
// bookkeeping and the FP64 stopping residual -- with no host round trip.
//
// The CTAs of a launch are split into groups; each group runs the jobs (games)
// assigned to it one after the other.  Phases are separated by a group barrier;
// the work of a phase (32-hand SBR items, one terminal per product item) is
// spread over the group's CTAs.  Products stay
// in terminal-contribution form; the SBR items add a sequence's contributions
// while they load their tile.
// Every CTA keeps its own copy of the solver state (t, mu, tau, buffer index)
// and takes every decision (EGV sign, tau back-off, gap target) itself from
// the same per-item FP64 partials, summed in the same fixed order as the
// standalone kernels: all CTAs of a group agree without a broadcast, a run here
// reproduces the host-driven loop of api.cu bit for bit, and a game's iterates
// do not depend on the group size or on the other games of the launch.
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
    if (ld_volatile(b.status) != 0) ok = 0;
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
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

// One SBR phase: all 32-hand items of `player`, spread over the CTAs; gv holds the
// player's terminal contributions (or is NULL).
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

__device__ __forceinline__ void run_sbr(const DevGame& g, const Tabs& tb, Grp gr, bool pair_ok, int player,
                                        const float* gv, double mu, const float* old, float tau, float* out,
                                        double* partials, unsigned char* sm) {
  const int NB = g.ld / kSbrHands;
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
    sbr_item(g, tp, item, a, reinterpret_cast<float*>(ism), wg);
  });
}

// One product phase: every terminal of `player`'s grouping; c64 (FP64 contributions
// for the residual) may be NULL.  With pairs (the job allows them and the group has at
// least two terminals per CTA) each warp half takes its own terminals.
__device__ __forceinline__ void run_grad(const DevGame& g, const Tabs& tb, Grp gr, bool pair_ok, int player,
                                         const float* in, float* c32, double* c64, unsigned char* sm) {
  const int T = player ? g.terms[1].n : g.terms[0].n;
  if (!(pair_ok && 2 * gr.size <= T)) {
    for (int item = gr.rank; item < T; item += gr.size)
      term_item<float>(g, tb.grad, player, item, in, c32, c64, sm);
    return;
  }
  constexpr int kHalf = kItemThreads / 64;
  const int half = (int)(threadIdx.x >> 5) >= kHalf ? 1 : 0;
  unsigned char* hs = sm + half * gradimpl::align16(grad_item_smem(g));
  for (int base = 2 * gr.rank; base < T; base += 2 * gr.size)
    if (base + half < T)
      term_item<float, kItemThreads / 2>(g, tb.grad, player, base + half, in, c32, c64, hs, half * kHalf,
                                         1 + half);
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

// Decisions of the current attempt, written by thread 0 of the CTA (the only
// thread that runs the solver's FP64 bookkeeping: FP64 is a narrow pipe on this
// part, and 512 redundant copies of it cost microseconds per iteration) and read
// by all threads after a CTA barrier.
struct Sched {
  int stop;             // leave the iteration loop
  int cur, me, gap_due, spec, pre;
  float tau, tau2;      // this attempt's tau, the next iteration's (FP32, for the mixing)
  double mu_me, mu_ot;  // mu of the stepping player and of the other
  double mu_tilde;      // (1 - tau) mu_me
};

// One job (game) run by the group `gr`: its tables staged in smem_all, then up to
// ctl->n_iters iterations.  Returns when the job stops or fails (status recorded).
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
  __shared__ Sched sc;
  PhaseClock* clk = &clk_s;
  const bool lead = threadIdx.x == 0;
  if (lead) {
    clk->last = global_ns();
    clk->arrive = clk->last;
    for (int k = 0; k < kEnginePhases; ++k) {
      clk->ns[k] = 0;
      clk->work[k] = 0;
      clk->n[k] = 0;
    }
  }
  const bool clock_cta = gr.rank == 0;
  const bool writer = clock_cta && lead;
  const int NB = g.ld / kSbrHands;
  double* partA = b.partials;
  double* partB = b.partials + NB;
  double* partBR0 = b.partials + 2 * NB;
  double* partBR1 = b.partials + 3 * NB;
  const int variant = ctl->variant, n_iters = ctl->n_iters, gap_every = ctl->gap_every;
  const int max_t = ctl->max_t;
  const bool check = variant == EGT_AS;

  // solver state: meaningful in thread 0 only (identical in every CTA)
  int t = 0, cur = 0, done = 0, backoffs_total = 0, products = 0, gap_checks = 0, reached = 0;
  int status = 0, last_player = -1, last_backoffs = 0, it = 0, me = 0, backoffs = 0, spec = 0;
  double mu0 = 0, mu1 = 0, tau_as = 0, gap = 0, tau = 0, eps_mbb = 0, mbb_scale = 1;
  double last_tau = 0.0 / 0.0, last_egv = 0.0 / 0.0, egv = 0.0 / 0.0, mu_next = 0;
  bool pre = false;        // v_hat of this iteration already computed (ahead, by the previous one)
  bool new_iter = true;    // the next attempt starts an iteration (else it retries with tau / 2)
  if (lead) {
    t = ctl->t;
    cur = ctl->cur;
    mu0 = ctl->mu[0];
    mu1 = ctl->mu[1];
    tau_as = ctl->tau;
    gap = ctl->gap_mbb;
    eps_mbb = ctl->eps_mbb;
    mbb_scale = ctl->mbb_scale;
  }

  for (;;) {
    if (lead) {
      int stop = !(it < n_iters && status == 0) || (it > 0 && new_iter && (reached || t >= max_t));
      if (!stop) {
        if (new_iter) {
          choose(variant, t, mu0, mu1, tau_as, me, tau);
          backoffs = 0;
          egv = 0.0 / 0.0;
        }
        const bool xs = me == 0;
        const int gap_due = (t + 1) % gap_every == 0 || t + 1 >= max_t;
        // The next iteration's choice if this attempt is accepted, and its v_hat computed
        // ahead: with the last product when the same player steps again (its gradient and
        // iterate are final there), else in the last phase, from the same smoothed best
        // response as the other's EGV part (same gradient, same mu).
        int me2;
        double tau2;
        mu_next = (1 - tau) * (xs ? mu0 : mu1);   // mu of the stepping player if accepted
        choose(variant, t + 1, xs ? mu_next : mu0, xs ? mu1 : mu_next, tau, me2, tau2);
        spec = me2 == me ? 1 : (check || gap_due ? 2 : 0);
        sc.cur = cur;
        sc.me = me;
        sc.gap_due = gap_due;
        sc.spec = spec;
        sc.pre = pre;
        sc.tau = (float)tau;
        sc.tau2 = (float)tau2;
        sc.mu_me = xs ? mu0 : mu1;
        sc.mu_ot = xs ? mu1 : mu0;
        sc.mu_tilde = mu_next;
      }
      sc.stop = stop;
    }
    __syncthreads();
    if (sc.stop) break;
    const int c = sc.cur, m = sc.me, gap_due = sc.gap_due, sp = sc.spec;
    const bool have_hat = sc.pre != 0;
    const float tau_f = sc.tau, tau2_f = sc.tau2;
    const double mu_me = sc.mu_me, mu_ot = sc.mu_ot, mu_tilde = sc.mu_tilde;
    const bool tail = check || gap_due;              // a phase after the Step's last product

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
      run_sbr(g, tb, gr, pair_ok, m, g_me, mu_me, v_me, tau_f, t_me, nullptr, sm);
      if (!phase_end(bar, bk, clk, 0, clock_cta)) return;
    }
    phase_cut(clk, 8, clock_cta);
    run_grad(g, tb, gr, pair_terms, ot, t_me, t_ot, nullptr, sm);   // the other's loss gradient at v_hat
    if (!phase_end(bar, bk, clk, 1, clock_cta)) return;
    // other_+ = (1 - tau) other + tau other_mu(v_hat)
    run_sbr(g, tb, gr, pair_ok, ot, t_ot, mu_ot, v_ot, tau_f, v_ot_n, nullptr, sm);
    if (!phase_end(bar, bk, clk, 2, clock_cta)) return;
    run_grad(g, tb, gr, pair_terms, m, v_ot_n, g_me_n, g64_me, sm);   // my loss gradient at other_+
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
          a.mu = mu_tilde;
          a.old = v_me;
          a.tau = tau_f;
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
      run_grad(g, tb, gr, pair_terms, ot, v_me_n, g_ot_n, g64_ot, sm);   // the other's at v_+
    } else {
      // the other's loss gradient at v_+, and the next v_hat (the same player steps again)
      const int T = ot ? g.terms[1].n : g.terms[0].n;
      const int n_items = T + NB;
      for (int item = gr.rank; item < n_items; item += gr.size) {
        if (item < T) {
          term_item<float>(g, tb.grad, ot, item, v_me_n, g_ot_n, g64_ot, sm);
        } else {
          SbrItemArgs a;
          a.g = g_me_n;
          a.contrib = true;
          a.grz = m ? g.rz[1] : g.rz[0];
          a.sign = m == 0 ? 1.f : -1.f;
          a.mu = mu_tilde;
          a.old = v_me_n;
          a.tau = tau2_f;
          a.out = t_me;
          a.value_partial = nullptr;
          sbr_item(g, pick(tb, m), item - T, a, reinterpret_cast<float*>(sm));
        }
      }
    }
    if (!phase_end(bar, bk, clk, 5, clock_cta)) return;
    double red[4] = {0.0, 0.0, 0.0, 0.0};
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
          a.mu = mu_ot;
          a.old = sp == 2 ? v_ot_n : nullptr;
          a.tau = sp == 2 ? tau2_f : 0.f;
          a.out = sp == 2 ? t_ot : nullptr;
          a.value_partial = check ? partB + item : nullptr;
          sbr_item(g, tp, item, a, reinterpret_cast<float*>(ism), wg);
        } else {
          run_br_item(g, tb, ot, item - n_sbr, b, partBR0, partBR1, ism, wg);
        }
      });
      if (!phase_end(bar, bk, clk, 6, clock_cta)) return;
      // the EGV parts (partA, partB) and the residual's values (partBR0, partBR1) in one pass
      reduce_arrays(b.partials, NB, check ? 0 : 2, gap_due ? 4 : 2, red);
      phase_cut(clk, 7, clock_cta);
    }

    if (lead) {
      products += 3;
      bool accept = true;
      if (check) {
        const double phi = xs ? red[0] : red[1], negf = xs ? red[1] : red[0];
        egv = phi + negf;
        if (!isfinite(egv)) {
          status = EGT_ERR_NUMERIC;
          accept = false;
        } else if (egv < 0) {
          accept = false;
          tau *= 0.5;
          if (tau < 1.0 / (1u << 30)) status = EGT_ERR_TAU_UNDERFLOW;
          else ++backoffs;
        }
      }
      if (accept) {
        // accept (Alg. 2 last lines): mu_me^+ = (1 - tau) mu_me, swap the iterate buffers
        if (xs) mu0 = mu_next;   // (1 - tau) mu_x, computed with the attempt
        else mu1 = mu_next;
        if (variant == EGT_AS) tau_as = tau;
        if (writer && b.log != nullptr && it < b.log_cap) {
          egt_iter_log& L = b.log[it];
          L.t = t;
          L.player = me;
          L.backoffs = backoffs;
          L.tau = tau;
          L.mu[0] = mu0;
          L.mu[1] = mu1;
          L.egv = check ? egv : 0.0 / 0.0;
          L.gap_mbb = gap;
          L.time_ns = global_ns();
        }
        cur = 1 - cur;
        t += 1;
        backoffs_total += backoffs;
        done += 1;
        last_player = me;
        last_backoffs = backoffs;
        last_tau = tau;
        last_egv = egv;
        pre = spec != 0;
        if (gap_due) {
          // eps_sad of the new iterates from the FP64 products of the Step:
          // max_y <y, A^T x> - min_x <x, A y>
          gap = (red[3] - red[2]) * mbb_scale;
          gap_checks += 1;
          if (!isfinite(gap)) status = EGT_ERR_NUMERIC;
          else reached = eps_mbb > 0 && gap <= eps_mbb ? 1 : 0;
        }
        it += 1;
        new_iter = true;
      } else {
        pre = false;
        new_iter = false;
      }
    }
  }

  if (writer) {
    ctl->t = t;
    ctl->cur = cur;
    ctl->mu[0] = mu0;
    ctl->mu[1] = mu1;
    ctl->tau = tau_as;
    ctl->gap_mbb = gap;
    ctl->reached = reached;
    ctl->done_iters = done;
    ctl->backoffs = backoffs_total;
    ctl->products = products;
    ctl->gap_checks = gap_checks;
    ctl->last_player = last_player;
    ctl->last_backoffs = last_backoffs;
    ctl->last_tau = last_tau;
    ctl->last_egv = last_egv;
    if (status != 0) atomicCAS(&ctl->status, 0, status);
#pragma unroll
    for (int k = 0; k < kEnginePhases; ++k) {
      ctl->phase_ns[k] = clk->ns[k];
      ctl->phase_work_ns[k] = clk->work[k];
      ctl->phase_n[k] = clk->n[k];
    }
  }
}

// One job on the whole grid, its description in the kernel parameters.
__global__ void __launch_bounds__(kItemThreads, 1)
    engine_kernel_one(EngineJob job, unsigned int extra, unsigned long long limit_ns) {
  extern __shared__ __align__(16) unsigned char smem_all[];
  engine_job(job.g, job.b, job.ctl, Grp{(int)blockIdx.x, (int)gridDim.x}, job.pair,
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
    engine_job(job_s.g, job_s.b, job_s.ctl, gr, job_s.pair, (unsigned long long)pg.size + extra, limit_ns,
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
  return cudaLaunchCooperativeKernel((const void*)engine_kernel_one, dim3(grid), dim3(kItemThreads), args,
                                     smem, st);
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
  static int limit_one = 0, limit_batch = 0;
  if (limit_one == 0) limit_one = opt_in_dynamic_smem((const void*)engine_kernel_one);
  if (limit_batch == 0) limit_batch = opt_in_dynamic_smem((const void*)engine_kernel);
  return batch ? limit_batch : limit_one;
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
  const cudaError_t e = batch ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, engine_kernel,
                                                                              kItemThreads, smem)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, engine_kernel_one,
                                                                              kItemThreads, smem);
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
