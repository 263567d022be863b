// Device-resident EGT driver (engine.cu): control block, buffers, launch helpers.
#pragma once
#include <cuda_runtime.h>

#include "../../include/egt.h"
#include "egt_internal.cuh"

namespace egt {

// Phases of an iteration timed by the engine (egt_engine_trace): the Step's
// three SBR and three product phases (the last one may carry the next v_hat), and
// the last phase (the other's EGV part, the residual's FP64 best responses, the
// next v_hat when the other player steps next), then CTA 0's time from the top of
// the iteration loop to its first phase (the sums behind the EGV and residual
// decisions and the decisions themselves when CTA 0 is the deciding CTA), then to
// its first product phase (no barrier).
constexpr int kEnginePhases = 9;

// Schedule of one attempt of Alg. 2's Step (with Alg. 4's back-off): what every CTA
// of the group needs to run its phases.
struct EngineSched {
  int stop;             // leave the iteration loop
  int cur, me, gap_due, spec, pre;
  float tau, tau2;      // this attempt's tau, the next iteration's (FP32, for the mixing)
  double mu_me, mu_ot;  // mu of the stepping player and of the other
  double mu_tilde;      // (1 - tau) mu_me
};
static_assert(sizeof(EngineSched) % 8 == 0, "EngineSched is copied in 8-byte words");

// Control block in device memory, one per game.  The host writes the
// configuration and the solver state before a launch and reads everything back
// after it.
struct EngineCtl {
  // configuration
  int variant, n_iters, gap_every, max_t;
  int trace;                   // CTA 0 times the phases (phase_ns ...): costs ~2 % of the rate
  int pad0;
  double eps_mbb, mbb_scale;   // gap target; 1000 / bb (mbb per unit of payoff)
  // solver state (persists between launches)
  double mu[2];
  double tau;
  int cur, t;
  // results of the launch
  int status, reached, retry, done_iters, backoffs, products, gap_checks;
  int last_player, last_backoffs;
  double gap_mbb, egv, last_tau, last_egv;
  // grid barrier: monotone arrival counter
  unsigned long long bar_arrive;
  // published by the group's deciding CTA before it arrives at an attempt's first
  // product barrier: (epoch << 8) | verdict on the previous attempt, the schedule of
  // the attempt after the running one (if the running one is accepted) and the
  // schedule of a retry
  unsigned long long verdict;
  EngineSched next, redo;
  // device time per phase (CTA 0, between consecutive barrier exits), ns
  unsigned long long phase_ns[kEnginePhases];
  unsigned long long phase_work_ns[kEnginePhases];   // CTA 0's own work (to its barrier arrival)
  unsigned long long phase_n[kEnginePhases];
};

struct EngineBufs {
  float* x[2];
  float* y[2];
  float* gx[2];     // A y of the matching y buffer (terminal contributions, [T][ld])
  float* gy[2];     // A^T x of the matching x buffer (terminal contributions)
  float* tx;        // [max(S0, T)][ld] scratch
  float* ty;        // [max(S1, T)][ld] scratch
  double* g64[2];   // FP64 products of the residual (terminal contributions)
  double* partials; // 4 x (ld / 32) per-item values
  egt_iter_log* log;
  int log_cap;
};

// One game of a launch: its device tables, buffers and control block.
struct EngineJob {
  DevGame g;
  EngineBufs b;
  EngineCtl* ctl;
  int pair;       // kPair* bits: items that may run two at a time on the CTA's warp halves
  int pad;
};
static_assert(sizeof(EngineJob) % 8 == 0, "EngineJob is copied in 8-byte words");

// Items a batch job may pair on the CTA's two warp halves.
constexpr int kPairSbr = 1;     // smoothed / FP64 best-response items
constexpr int kPairTerms = 2;   // product (terminal) items

// Dynamic shared memory the driver needs for game g (tables + the largest item, or two
// items side by side for the kPair* bits set).
size_t engine_smem_bytes(const DevGame& g, int pair_bits = 0);

// Items of the widest phase of game g (more CTAs per game than this idle).
int engine_items(const DevGame& g);

// Largest dynamic shared memory per CTA of the driver's kernels on the current device
// (-1: CUDA error).
int engine_smem_limit(bool batch);

// Largest co-resident grid of the driver (batch: the multi-job kernel, else the
// one-job kernel) with `smem` bytes of dynamic shared memory per CTA on the
// current device (0: cannot run, -1: CUDA error).
int engine_max_grid(size_t smem, bool batch);

// Cooperative launch of one job on `grid` CTAs (its description passed by value).
cudaError_t engine_launch_one(const EngineJob& job, int grid, size_t smem, unsigned int extra,
                              unsigned long long limit_ns, cudaStream_t st);

// A group of a multi-job launch: CTAs [first, first + size) run jobs [job0, job1)
// one after the other.
struct EngineGroup {
  int first, size, job0, job1;
};

// Cooperative launch of `grid` CTAs over the jobs in device memory, split into
// the n_groups groups of plan_dev (disjoint CTA ranges inside the grid).
// `extra` phantom arrivals per group barrier (a timeout test: every wait then
// runs out after limit_ns instead of completing).
cudaError_t engine_launch(const EngineJob* jobs_dev, const EngineGroup* plan_dev, int n_groups, int grid,
                          size_t smem, unsigned int extra, unsigned long long limit_ns, cudaStream_t st);

}  // namespace egt
