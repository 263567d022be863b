// C-ABI of libegt, batches (include/egt.h): many games advanced by one
// device-resident cooperative launch per step, the CTAs split into groups over
// the members by a launch shape, and the launch-shape autotuner.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "api_internal.hpp"

using namespace egt;
using namespace egtapi;

struct egt_batch {
  int device = 0;
  struct Member {
    egt_game* G = nullptr;     // NULL: free slot
    int variant = EGT_AS, gap_every = 1, max_iters = 0;
    double eps_mbb = 0.0;
    int active = 0, status = EGT_OK, iters = 0, products = 0, backoffs = 0, gap_checks = 0;
    double seconds = 0.0;
  };
  std::vector<Member> members;
  EngineCtl* ctl_dev = nullptr;
  EngineCtl* ctl_host = nullptr;
  EngineJob* jobs_dev = nullptr;
  EngineJob* jobs_host = nullptr;
  EngineGroup* plan_dev = nullptr;
  EngineGroup* plan_host = nullptr;
  int cap = 0;
  int last_group = 0, last_grid = 0;
  egt_launch_shape shape{3, 1, 100, 0, 128, 16};
  cudaEvent_t ev[2] = {nullptr, nullptr};   // timing of tuning trials (created on first use)
};

namespace {

bool shape_ok(const egt_launch_shape& x) {
  return x.share >= 0 && x.share <= 4 && (x.pairs == 0 || x.pairs == 1) && x.grid_pct >= 1 && x.grid_pct <= 100 &&
         (x.pack == 0 || x.pack == 1) && x.wave_mb >= 0 && x.wave_min >= 1;
}

void batch_free_arrays(egt_batch* B) {
  cudaFree(B->ctl_dev);
  cudaFree(B->jobs_dev);
  cudaFree(B->plan_dev);
  if (B->ctl_host) cudaFreeHost(B->ctl_host);
  if (B->jobs_host) cudaFreeHost(B->jobs_host);
  if (B->plan_host) cudaFreeHost(B->plan_host);
  B->ctl_dev = nullptr;
  B->jobs_dev = nullptr;
  B->plan_dev = nullptr;
  B->ctl_host = nullptr;
  B->jobs_host = nullptr;
  B->plan_host = nullptr;
  B->cap = 0;
}

egt_status batch_reserve(egt_batch* B, int n) {
  if (n <= B->cap) return EGT_OK;
  const int cap = std::max(n, 2 * B->cap);
  batch_free_arrays(B);
  CUDA_TRY(cudaMalloc(&B->ctl_dev, (size_t)cap * sizeof(EngineCtl)));
  CUDA_TRY(cudaMalloc(&B->jobs_dev, (size_t)cap * sizeof(EngineJob)));
  CUDA_TRY(cudaHostAlloc(&B->ctl_host, (size_t)cap * sizeof(EngineCtl), cudaHostAllocDefault));
  CUDA_TRY(cudaHostAlloc(&B->jobs_host, (size_t)cap * sizeof(EngineJob), cudaHostAllocDefault));
  CUDA_TRY(cudaMalloc(&B->plan_dev, (size_t)cap * sizeof(EngineGroup)));
  CUDA_TRY(cudaHostAlloc(&B->plan_host, (size_t)cap * sizeof(EngineGroup), cudaHostAllocDefault));
  B->cap = cap;
  return EGT_OK;
}

// Relative cost of one iteration of a game (three product phases of T terminal
// items of ld hands, about seven SBR / best-response passes over S x ld).
double iteration_work(const egt_game* G) {
  const double S = 0.5 * (G->comp.tpx[0].S + G->comp.tpx[1].S);
  return (double)G->ld * (3.0 * (double)G->comp.term.size() + 7.0 * S);
}

// Split maxg co-resident CTAs over n jobs (work w, useful CTAs at most cap each).
// group > 0: groups of that size, jobs dealt round-robin.  Else one group per job
// with CTAs in proportion to its work when the jobs fit, or one-CTA groups each
// running a least-loaded share of the jobs when they do not.  Fills plan (groups
// with contiguous job ranges) and order (job position -> input index); returns
// the number of groups and sets *grid.
int plan_groups(const std::vector<double>& w, const std::vector<int>& cap, int maxg, int group,
                std::vector<EngineGroup>& plan, std::vector<int>& order, int* grid) {
  const int n = (int)w.size();
  plan.clear();
  order.clear();
  if (group > 0 || n > maxg) {
    const int gsize = group > 0 ? std::min(group, maxg) : 1;
    const int ng = std::min(n, maxg / gsize);
    std::vector<std::vector<int>> lists(ng);
    if (group > 0) {
      for (int j = 0; j < n; ++j) lists[j % ng].push_back(j);
    } else {
      std::vector<int> idx(n);
      std::iota(idx.begin(), idx.end(), 0);
      std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return w[a] > w[b]; });
      std::vector<double> load(ng, 0.0);
      for (int j : idx) {
        const int q = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lists[q].push_back(j);
        load[q] += w[j];
      }
    }
    for (int q = 0; q < ng; ++q) {
      EngineGroup e{q * gsize, gsize, (int)order.size(), 0};
      for (int j : lists[q]) order.push_back(j);
      e.job1 = (int)order.size();
      plan.push_back(e);
    }
    *grid = ng * gsize;
    return ng;
  }
  double W = 0.0;
  for (double x : w) W += x;
  std::vector<int> c(n);
  int used = 0;
  for (int j = 0; j < n; ++j) {
    c[j] = std::max(1, std::min(cap[j], (int)std::floor(maxg * w[j] / W)));
    used += c[j];
  }
  while (used > maxg) {   // rounding up to one CTA each overshot: take from the largest
    const int j = (int)(std::max_element(c.begin(), c.end()) - c.begin());
    --c[j];
    --used;
  }
  while (used < maxg) {   // leftovers to the job with the most work per CTA that can use one
    int best = -1;
    for (int j = 0; j < n; ++j)
      if (c[j] < cap[j] && (best < 0 || w[j] / c[j] > w[best] / c[best])) best = j;
    if (best < 0) break;
    ++c[best];
    ++used;
  }
  int first = 0;
  for (int j = 0; j < n; ++j) {
    plan.push_back(EngineGroup{first, c[j], j, j + 1});
    order.push_back(j);
    first += c[j];
  }
  *grid = first;
  return n;
}

// Makespan-balanced plan over maxg CTAs (launch shape pack = 1): with a member's
// time modelled as its work over its CTAs, find (bisection) the least makespan M
// for which every member heavier than M gets ceil(w / M) CTAs of its own (at most
// its widest phase) and the lighter ones, packed first-fit by decreasing work,
// share one-CTA groups that run them in turn, all within maxg CTAs; CTAs left
// over go to the heavy members with the most work per CTA.  Same outputs as
// plan_groups.
int plan_groups_packed(const std::vector<double>& w, const std::vector<int>& cap, int maxg,
                       std::vector<EngineGroup>& plan, std::vector<int>& order, int* grid) {
  const int n = (int)w.size();
  std::vector<int> by_w(n);
  std::iota(by_w.begin(), by_w.end(), 0);
  std::stable_sort(by_w.begin(), by_w.end(), [&](int a, int b) { return w[a] > w[b]; });
  std::vector<int> c;
  std::vector<std::vector<int>> bins;
  auto fit = [&](double M) {   // CTAs the plan for makespan M needs (maxg + 1: infeasible)
    c.assign(n, 0);
    bins.clear();
    std::vector<double> load;
    int total = 0;
    for (int j : by_w) {
      if (w[j] > M) {
        c[j] = (int)std::ceil(w[j] / M);
        if (c[j] > cap[j]) return maxg + 1;
        total += c[j];
      } else {
        size_t b = 0;
        while (b < load.size() && load[b] + w[j] > M) ++b;
        if (b == load.size()) {
          load.push_back(0.0);
          bins.emplace_back();
        }
        load[b] += w[j];
        bins[b].push_back(j);
      }
      if (total + (int)bins.size() > maxg) return maxg + 1;
    }
    return total + (int)bins.size();
  };
  double lo = 0.0, hi = 0.0;
  for (int j = 0; j < n; ++j) {
    lo = std::max(lo, w[j] / std::max(1, cap[j]));
    hi += w[j];
  }
  hi = std::max(hi, lo);
  for (int it = 0; it < 60 && hi - lo > 1e-9 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    (fit(mid) <= maxg ? hi : lo) = mid;
  }
  fit(hi);
  int used = 0;
  for (int j = 0; j < n; ++j) used += c[j];
  used += (int)bins.size();
  while (used < maxg) {   // leftovers to the heavy member with the most work per CTA that can use one
    int best = -1;
    for (int j = 0; j < n; ++j)
      if (c[j] > 0 && c[j] < cap[j] && (best < 0 || w[j] / c[j] > w[best] / c[best])) best = j;
    if (best < 0) break;
    ++c[best];
    ++used;
  }
  plan.clear();
  order.clear();
  int first = 0;
  for (int j : by_w)
    if (c[j] > 0) {
      plan.push_back(EngineGroup{first, c[j], (int)order.size(), (int)order.size() + 1});
      order.push_back(j);
      first += c[j];
    }
  for (const auto& b : bins) {
    EngineGroup e{first, 1, (int)order.size(), 0};
    for (int j : b) order.push_back(j);
    e.job1 = (int)order.size();
    plan.push_back(e);
    first += 1;
  }
  *grid = first;
  return (int)plan.size();
}

egt_status check_slot(const egt_batch* B, int32_t slot) {
  if (!B) return fail(EGT_ERR_INVALID_ARG, "batch is NULL");
  if (slot < 0 || slot >= (int)B->members.size() || !B->members[slot].G)
    return fail(EGT_ERR_INVALID_ARG, "no such batch member");
  return EGT_OK;
}

// One batch launch under launch shape `sh` (group > 0 overrides its split); with
// ms != NULL the engine launch is timed with CUDA events and *done gets the
// member-iterations it ran.
egt_status launch_members(egt_batch* B, const std::vector<int>& act, int32_t n_iters, int32_t group,
                          const egt_launch_shape& sh, int32_t* n_active, cudaStream_t st, float* ms,
                          long long* done) {
  if (done) *done = 0;
  if (ms) *ms = 0.f;
  const int n = (int)act.size();
  if (n_active) *n_active = n;
  if (n == 0) return EGT_OK;
  EGT_TRY(batch_reserve(B, n));
  size_t smem = 0;
  std::vector<double> w(n), wraw(n);
  std::vector<int> cap(n), pair(n);
  const int limit = engine_smem_limit(true);
  for (int i = 0; i < n; ++i) {
    const egt_game* G = B->members[act[i]].G;
    // two items per CTA at a time where shared memory allows
    pair[i] = 0;
    if (sh.pairs)
      for (int bit : {kPairTerms, kPairSbr})
        if (limit > 0 && engine_smem_bytes(G->dg, pair[i] | bit) <= (size_t)limit) pair[i] |= bit;
    smem = std::max(smem, engine_smem_bytes(G->dg, pair[i]));
    const double work = iteration_work(G);
    wraw[i] = work;
    w[i] = sh.share == 4 ? work : std::pow(work, 0.25 * sh.share);
    cap[i] = engine_items(G->dg);
  }
  const int maxg_all = engine_max_grid(smem, true);
  if (maxg_all <= 0) return fail(EGT_ERR_CUDA, "the device-resident driver cannot run on this device");
  const int maxg = std::max(1, maxg_all * sh.grid_pct / 100);
  std::vector<EngineGroup> plan;
  std::vector<int> order;
  int grid = 0;
  const int n_groups = group == 0 && sh.pack ? plan_groups_packed(wraw, cap, maxg, plan, order, &grid)
                                             : plan_groups(w, cap, maxg, group, plan, order, &grid);
  int widest = 0;
  for (const auto& e : plan) widest = std::max(widest, e.size);
  B->last_group = widest;
  B->last_grid = grid;
  std::vector<int> slot_of(n);
  for (int i = 0; i < n; ++i) {
    slot_of[i] = act[order[i]];
    egt_batch::Member& m = B->members[slot_of[i]];
    const int left = m.max_iters - m.iters;
    engine_ctl_init(m.G, B->ctl_host[i], m.variant, m.eps_mbb, m.gap_every, std::min(n_iters, left));
    // the residual at the member's last iteration, as egt_solve does
    B->ctl_host[i].max_t = m.G->t + left;
    EngineJob& j = B->jobs_host[i];
    std::memset(&j, 0, sizeof(j));
    j.g = m.G->dg;
    j.b = engine_bufs(m.G, nullptr, 0);
    j.ctl = B->ctl_dev + i;
    j.pair = pair[order[i]];
  }
  std::copy(plan.begin(), plan.end(), B->plan_host);
  const unsigned extra = (unsigned)std::max(0, env_int("EGT_TEST_BARRIER_EXTRA", 0));
  const unsigned long long limit_ns =
      1000000ull * (unsigned long long)std::max(1, env_int("EGT_BARRIER_TIMEOUT_MS", 2000));
  const auto t0 = std::chrono::steady_clock::now();
  CUDA_TRY(cudaMemcpyAsync(B->ctl_dev, B->ctl_host, (size_t)n * sizeof(EngineCtl), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(B->jobs_dev, B->jobs_host, (size_t)n * sizeof(EngineJob), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(B->plan_dev, B->plan_host, (size_t)n_groups * sizeof(EngineGroup),
                           cudaMemcpyHostToDevice, st));
  if (ms) {
    for (auto& e : B->ev)
      if (!e) CUDA_TRY(cudaEventCreate(&e));
    CUDA_TRY(cudaEventRecord(B->ev[0], st));
  }
  const cudaError_t le = engine_launch(B->jobs_dev, B->plan_dev, n_groups, grid, smem, extra, limit_ns, st);
  if (le != cudaSuccess) return fail(EGT_ERR_CUDA, std::string("engine launch: ") + cudaGetErrorString(le));
  if (ms) CUDA_TRY(cudaEventRecord(B->ev[1], st));
  CUDA_TRY(cudaMemcpyAsync(B->ctl_host, B->ctl_dev, (size_t)n * sizeof(EngineCtl), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (ms) CUDA_TRY(cudaEventElapsedTime(ms, B->ev[0], B->ev[1]));
  int still = 0;
  for (int i = 0; i < n; ++i) {
    egt_batch::Member& m = B->members[slot_of[i]];
    const EngineCtl& c = B->ctl_host[i];
    engine_ctl_apply(m.G, c, nullptr);
    m.iters += c.done_iters;
    if (done) *done += c.done_iters;
    m.products += c.products;
    m.backoffs += c.backoffs;
    m.gap_checks += c.gap_checks;
    m.seconds += sec;
    if (c.status != 0) {
      m.active = 0;
      m.status = c.status;
    } else if (c.reached) {
      m.active = 0;
      m.status = EGT_OK;
    } else if (m.iters >= m.max_iters) {
      m.active = 0;
      m.status = m.eps_mbb > 0 ? EGT_ERR_NOT_CONVERGED : EGT_OK;
    }
    still += m.active;
  }
  if (n_active) *n_active = still;
  return EGT_OK;
}

// One batch step under launch shape `sh`: the active members in one launch, or
// (sh.wave_mb > 0) in k = ceil(total device bytes / wave_mb MB) consecutive waves of
// about equal bytes, one launch each, so that a wave's state can stay in L2, but no
// more waves than (active members / sh.wave_min).  ms / done add up over the waves.
egt_status batch_launch(egt_batch* B, int32_t n_iters, int32_t group, const egt_launch_shape& sh,
                        int32_t* n_active, cudaStream_t st, float* ms, long long* done) {
  if (n_iters <= 0) return fail(EGT_ERR_INVALID_ARG, "n_iters must be > 0");
  if (group < 0) return fail(EGT_ERR_INVALID_ARG, "group must be >= 0");
  DeviceGuard guard(B->device);
  std::vector<int> act;
  for (int k = 0; k < (int)B->members.size(); ++k)
    if (B->members[k].G && B->members[k].active) act.push_back(k);
  if (sh.wave_mb <= 0) return launch_members(B, act, n_iters, group, sh, n_active, st, ms, done);
  const double budget = (double)((size_t)sh.wave_mb << 20);
  double total = 0.0;
  for (int k : act) total += (double)B->members[k].G->device_bytes;
  const int waves = std::max(1, std::min((int)std::ceil(total / budget), (int)act.size() / sh.wave_min));
  const double target = total / waves;
  if (done) *done = 0;
  if (ms) *ms = 0.f;
  int still = 0;
  double before = 0.0;   // bytes of the members in earlier waves
  for (size_t i = 0; i < act.size();) {
    std::vector<int> wave;
    const int q = std::min(waves - 1, (int)(before / target));
    while (i < act.size() && (wave.empty() || std::min(waves - 1, (int)(before / target)) == q)) {
      before += (double)B->members[act[i]].G->device_bytes;
      wave.push_back(act[i++]);
    }
    float w_ms = 0.f;
    long long w_done = 0;
    int32_t w_active = 0;
    EGT_TRY(launch_members(B, wave, n_iters, group, sh, &w_active, st, ms ? &w_ms : nullptr, &w_done));
    if (ms) *ms += w_ms;
    if (done) *done += w_done;
    still += w_active;
  }
  if (n_active) *n_active = still;
  return EGT_OK;
}

}  // namespace

extern "C" {

egt_status egt_batch_create(int32_t device, egt_batch** out) {
  if (!out) return fail(EGT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(EGT_ERR_INVALID_ARG, "no such device");
  egt_batch* B = new (std::nothrow) egt_batch();
  if (!B) return fail(EGT_ERR_OOM, "host allocation failed");
  B->device = device;
  *out = B;
  return EGT_OK;
}

egt_status egt_batch_destroy(egt_batch* B) {
  if (!B) return EGT_OK;
  DeviceGuard guard(B->device);
  cudaDeviceSynchronize();
  batch_free_arrays(B);
  for (auto& e : B->ev)
    if (e) cudaEventDestroy(e);
  delete B;
  return EGT_OK;
}

egt_status egt_batch_add(egt_batch* B, egt_game* G, const egt_solve_opts* o, int32_t* slot) {
  if (!B || !G || !o || !slot) return fail(EGT_ERR_INVALID_ARG, "NULL argument");
  if (G->host_only || G->device != B->device)
    return fail(EGT_ERR_INVALID_ARG, "the game is not on the batch's device");
  if (!G->initialised) return fail(EGT_ERR_INVALID_ARG, "egt_solver_init has not been called");
  if (o->variant < EGT_THEORY || o->variant > EGT_AS) return fail(EGT_ERR_INVALID_ARG, "unknown variant");
  if (o->max_iters <= 0) return fail(EGT_ERR_INVALID_ARG, "max_iters must be > 0");
  if (o->replay_n > 0 || o->log) return fail(EGT_ERR_INVALID_ARG, "replay and log are not accepted in a batch");
  for (const auto& m : B->members)
    if (m.G == G) return fail(EGT_ERR_INVALID_ARG, "the game is already a member");
  egt_batch::Member m;
  m.G = G;
  m.variant = o->variant;
  m.gap_every = std::max(1, o->gap_every);
  m.max_iters = o->max_iters;
  m.eps_mbb = o->eps_mbb;
  m.active = 1;
  int k = 0;
  while (k < (int)B->members.size() && B->members[k].G) ++k;
  // the launch arrays for every member, allocated here rather than in a step
  {
    DeviceGuard guard(B->device);
    EGT_TRY(batch_reserve(B, std::max(k + 1, (int)B->members.size())));
  }
  if (k == (int)B->members.size()) B->members.push_back(m);
  else B->members[k] = m;
  *slot = k;
  return EGT_OK;
}

egt_status egt_batch_remove(egt_batch* B, int32_t slot) {
  EGT_TRY(check_slot(B, slot));
  B->members[slot] = egt_batch::Member();
  return EGT_OK;
}

egt_status egt_batch_step(egt_batch* B, int32_t n_iters, int32_t group, int32_t* n_active, void* stream) {
  Range nvtx_range("egt_batch_step");
  if (!B) return fail(EGT_ERR_INVALID_ARG, "batch is NULL");
  return batch_launch(B, n_iters, group, B->shape, n_active, S(stream), nullptr, nullptr);
}

egt_status egt_batch_set_shape(egt_batch* B, const egt_launch_shape* shape) {
  if (!B || !shape) return fail(EGT_ERR_INVALID_ARG, "NULL argument");
  if (!shape_ok(*shape)) return fail(EGT_ERR_INVALID_ARG, "launch shape out of range (share 0-4, pairs 0/1, grid_pct 1-100)");
  B->shape = *shape;
  return EGT_OK;
}

egt_status egt_batch_get_shape(const egt_batch* B, egt_launch_shape* shape) {
  if (!B || !shape) return fail(EGT_ERR_INVALID_ARG, "NULL argument");
  *shape = B->shape;
  return EGT_OK;
}

egt_status egt_batch_tune(egt_batch* B, int32_t n_iters, int32_t reps, egt_tune_report* rep, void* stream) {
  Range nvtx_range("egt_batch_tune");
  if (!B) return fail(EGT_ERR_INVALID_ARG, "batch is NULL");
  if (n_iters <= 0 || reps <= 0) return fail(EGT_ERR_INVALID_ARG, "n_iters and reps must be > 0");
  DeviceGuard guard(B->device);
  egt_tune_report r;
  std::memset(&r, 0, sizeof(r));
  r.best = -1;
  for (int share : {4, 3, 2, 1, 0}) r.shape[r.n++] = egt_launch_shape{share, 1, 100, 0, 0, 16};
  for (int share : {4, 3, 2}) r.shape[r.n++] = egt_launch_shape{share, 0, 100, 0, 0, 16};
  r.shape[r.n++] = egt_launch_shape{3, 1, 75, 0, 0, 16};
  r.shape[r.n++] = egt_launch_shape{4, 1, 100, 1, 0, 16};
  for (int mb : {64, 96, 128}) r.shape[r.n++] = egt_launch_shape{3, 1, 100, 0, mb, 16};   // L2: 126 MB
  static_assert(5 + 3 + 1 + 1 + 3 <= EGT_TUNE_MAX, "tuning candidates");
  double best = 0.0;
  for (int k = 0; k < r.n; ++k) {
    double us_best = 0.0;
    int it_best = 0;
    for (int q = 0; q < reps; ++q) {
      float ms = 0.f;
      long long done = 0;
      int active = 0;
      EGT_TRY(batch_launch(B, n_iters, 0, r.shape[k], &active, S(stream), &ms, &done));
      if (done <= 0) continue;
      const double us = 1000.0 * (double)ms / (double)done;
      if (it_best == 0 || us < us_best) {
        us_best = us;
        it_best = (int)done;
      }
    }
    r.us_per_iter[k] = us_best;
    r.iters[k] = it_best;
    if (it_best > 0 && (r.best < 0 || us_best < best)) {
      best = us_best;
      r.best = k;
    }
  }
  if (r.best >= 0) B->shape = r.shape[r.best];
  if (rep) *rep = r;
  return EGT_OK;
}

egt_status egt_batch_member(const egt_batch* B, int32_t slot, egt_batch_member_info* out) {
  EGT_TRY(check_slot(B, slot));
  if (!out) return fail(EGT_ERR_INVALID_ARG, "out is NULL");
  const egt_batch::Member& m = B->members[slot];
  out->active = m.active;
  out->status = m.status;
  out->rep.iters = m.iters;
  out->rep.products = m.products;
  out->rep.backoffs = m.backoffs;
  out->rep.gap_checks = m.gap_checks;
  out->rep.gap_mbb = m.G->last_gap;
  out->rep.mu[0] = m.G->mu[0];
  out->rep.mu[1] = m.G->mu[1];
  out->rep.tau = m.G->tau;
  out->rep.seconds = m.seconds;
  return EGT_OK;
}

egt_status egt_batch_launch_shape(const egt_batch* B, int32_t* group, int32_t* grid) {
  if (!B) return fail(EGT_ERR_INVALID_ARG, "batch is NULL");
  if (group) *group = B->last_group;
  if (grid) *grid = B->last_grid;
  return EGT_OK;
}

}  // extern "C"
