// egt_server_*: continuous batching of endgame-solving requests on one device,
// built on the public C-ABI only (egt_create_game, egt_solver_init, egt_batch_*,
// egt_state_get).
//
// Requests wait in a FIFO queue.  Every egt_server_step admits queued requests
// in order while their device memory (egt_dims.device_bytes, known before
// upload) fits under the budget, then runs one egt_batch_step over every
// running request, then retires the requests that stopped: their iterates are
// copied to host memory, their games destroyed, their memory returned to the
// budget.  A request therefore joins and leaves the device between launches
// while the others keep their device-resident x / y / mu state; its result is
// bit for bit the one egt_solve gives the same request alone, since a batch
// member's iterates do not depend on the other members.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/egt.h"

namespace egt {
void set_last_error(const std::string& msg);   // the library's thread-local message (egt_last_error)
}

namespace {

const char* kStateNames[] = {"queued", "running", "done"};

egt_status fail(egt_status st, const std::string& msg) {
  egt::set_last_error(msg);
  return st;
}

enum { kQueued = 0, kRunning = 1, kDone = 2 };

struct Request {
  // owned copy of the description
  std::vector<int32_t> cards;
  std::vector<int32_t> strength;
  std::vector<double> r0, r1, bets;
  std::vector<egt_menu> menus;
  std::vector<std::vector<double>> menu_fracs;
  egt_game_desc desc{};
  egt_solve_opts opts{};
  int64_t bytes = 0;
  int state = kQueued;
  egt_status status = EGT_OK;
  double t_submit = 0, t_admit = -1, t_done = -1;
  egt_game* game = nullptr;
  int32_t slot = -1;
  int32_t S[2] = {0, 0}, ld = 0;
  egt_solve_report rep{};
  std::vector<float> x, y;
};

}  // namespace

struct egt_server {
  int device = 0;
  egt_server_opts opts{};
  egt_batch* batch = nullptr;
  std::unordered_map<int64_t, Request> reqs;
  std::deque<int64_t> queue;
  std::vector<int64_t> running;
  int64_t next_id = 1;
  int64_t budget = 0, used = 0;
  float* stage = nullptr;   // device staging for retiring iterates
  size_t stage_elems = 0;
  std::chrono::steady_clock::time_point t0;
  int64_t steps = 0, launches = 0, completed = 0;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(dev);
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Copy the finished request's iterates to host memory, then release its device state.
egt_status retire(egt_server* V, Request& r, cudaStream_t st) {
  egt_batch_member_info m{};
  egt_status s = egt_batch_member(V->batch, r.slot, &m);
  if (s != EGT_OK) return s;
  r.rep = m.rep;
  r.status = (egt_status)m.status;
  const size_t n0 = (size_t)r.S[0] * r.ld, n1 = (size_t)r.S[1] * r.ld;
  if (n0 + n1 > V->stage_elems) {
    cudaFree(V->stage);
    V->stage = nullptr;
    V->stage_elems = 0;
    if (cudaMalloc(&V->stage, (n0 + n1) * sizeof(float)) != cudaSuccess)
      return fail(EGT_ERR_OOM, "egt_server_step: staging allocation failed");
    V->stage_elems = n0 + n1;
  }
  double mu[2];
  s = egt_state_get(r.game, V->stage, V->stage + n0, mu, st);
  if (s != EGT_OK) return s;
  r.x.resize(n0);
  r.y.resize(n1);
  if (cudaMemcpyAsync(r.x.data(), V->stage, n0 * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(r.y.data(), V->stage + n0, n1 * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(EGT_ERR_CUDA, "egt_server_step: copying a result to the host failed");
  egt_batch_remove(V->batch, r.slot);
  egt_destroy_game(r.game);
  r.game = nullptr;
  r.slot = -1;
  V->used -= r.bytes;
  r.state = kDone;
  r.t_done = V->now();
  V->completed += 1;
  return EGT_OK;
}

// Create, initialise and add the request's game; a failure finishes the request with
// that status.  Returns true if the request now runs.
bool admit(egt_server* V, Request& r, cudaStream_t st) {
  r.t_admit = V->now();
  egt_status s = egt_create_game(&r.desc, V->device, st, &r.game);
  if (s == EGT_OK) s = egt_solver_init(r.game, &r.opts, st);
  if (s == EGT_OK) s = egt_batch_add(V->batch, r.game, &r.opts, &r.slot);
  if (s != EGT_OK) {
    if (r.game) egt_destroy_game(r.game);
    r.game = nullptr;
    r.state = kDone;
    r.status = s;
    r.t_done = V->now();
    V->completed += 1;
    return false;
  }
  r.state = kRunning;
  V->used += r.bytes;
  return true;
}

}  // namespace

extern "C" {

egt_status egt_server_create(int32_t device, const egt_server_opts* opts, egt_server** out) {
  if (!out) return fail(EGT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return fail(EGT_ERR_INVALID_ARG, "no such device");
  egt_server* V = new (std::nothrow) egt_server();
  if (!V) return fail(EGT_ERR_OOM, "host allocation failed");
  V->device = device;
  if (opts) V->opts = *opts;
  if (V->opts.iters_per_step <= 0) V->opts.iters_per_step = 200;
  DeviceScope scope(device);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    delete V;
    return fail(EGT_ERR_CUDA, "cudaMemGetInfo failed");
  }
  const int64_t cap = (int64_t)(0.9 * (double)free_b);
  V->budget = V->opts.mem_budget_bytes > 0 ? std::min<int64_t>(V->opts.mem_budget_bytes, cap) : cap;
  egt_status s = egt_batch_create(device, &V->batch);
  if (s != EGT_OK) {
    delete V;
    return s;
  }
  V->t0 = std::chrono::steady_clock::now();
  *out = V;
  return EGT_OK;
}

egt_status egt_server_destroy(egt_server* V) {
  if (!V) return EGT_OK;
  DeviceScope scope(V->device);
  for (auto& kv : V->reqs)
    if (kv.second.game) egt_destroy_game(kv.second.game);
  egt_batch_destroy(V->batch);
  cudaFree(V->stage);
  delete V;
  return EGT_OK;
}

double egt_server_clock(const egt_server* V) { return V ? V->now() : 0.0; }

egt_status egt_server_submit(egt_server* V, const egt_game_desc* d, const egt_solve_opts* o, double arrival,
                             int64_t* id) {
  if (!V || !d || !o || !id) return fail(EGT_ERR_INVALID_ARG, "NULL argument");
  if (o->max_iters <= 0) return fail(EGT_ERR_INVALID_ARG, "max_iters must be > 0");
  if (o->replay_n > 0 || o->log) return fail(EGT_ERR_INVALID_ARG, "replay and log are not accepted");
  if (!d->hand_cards || !d->strength || !d->range[0] || !d->range[1] || (d->n_bets > 0 && !d->bet_fracs) ||
      d->n_hands <= 0 || d->hand_size <= 0 || d->n_bets < 0)
    return fail(EGT_ERR_INVALID_ARG, "incomplete game description");
  const int64_t k = V->next_id++;
  Request& r = V->reqs[k];
  const size_t H = (size_t)d->n_hands;
  r.cards.assign(d->hand_cards, d->hand_cards + H * d->hand_size);
  r.strength.assign(d->strength, d->strength + H);
  r.r0.assign(d->range[0], d->range[0] + H);
  r.r1.assign(d->range[1], d->range[1] + H);
  r.bets.assign(d->bet_fracs, d->bet_fracs + d->n_bets);
  r.desc = *d;
  r.desc.hand_cards = r.cards.data();
  r.desc.strength = r.strength.data();
  r.desc.range[0] = r.r0.data();
  r.desc.range[1] = r.r1.data();
  r.desc.bet_fracs = r.bets.empty() ? nullptr : r.bets.data();
  if (d->menus) {
    r.menus.assign(d->menus, d->menus + 8);
    r.menu_fracs.resize(8);
    for (int m = 0; m < 8; ++m) {
      if (r.menus[m].n > 0 && r.menus[m].fracs)
        r.menu_fracs[m].assign(r.menus[m].fracs, r.menus[m].fracs + r.menus[m].n);
      r.menus[m].fracs = r.menu_fracs[m].empty() ? nullptr : r.menu_fracs[m].data();
    }
    r.desc.menus = r.menus.data();
  }
  r.opts = *o;
  r.opts.log = nullptr;
  r.opts.log_cap = 0;
  // sizes from a host-only compile (validates the description too)
  egt_game* h = nullptr;
  egt_status s = egt_create_game(&r.desc, -1, nullptr, &h);
  if (s != EGT_OK) {
    const std::string msg = egt_last_error();
    V->reqs.erase(k);
    return fail(s, "egt_server_submit: " + msg);
  }
  egt_dims dims{};
  egt_dims_query(h, &dims);
  egt_destroy_game(h);
  if (dims.device_bytes > V->budget) {
    V->reqs.erase(k);
    return fail(EGT_ERR_OOM, "egt_server_submit: the game needs more device memory than the server's budget");
  }
  r.bytes = dims.device_bytes;
  r.S[0] = dims.S[0];
  r.S[1] = dims.S[1];
  r.ld = dims.ld;
  r.t_submit = arrival >= 0 ? arrival : V->now();
  V->queue.push_back(k);
  *id = k;
  return EGT_OK;
}

egt_status egt_server_step(egt_server* V, egt_server_stats* stats, void* stream) {
  if (!V) return fail(EGT_ERR_INVALID_ARG, "server is NULL");
  DeviceScope scope(V->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  V->steps += 1;
  // admission: FIFO while the head fits the memory budget and the member cap
  while (!V->queue.empty()) {
    if (V->opts.max_running > 0 && (int)V->running.size() >= V->opts.max_running) break;
    Request& r = V->reqs.at(V->queue.front());
    if (V->used + r.bytes > V->budget) break;
    const int64_t k = V->queue.front();
    V->queue.pop_front();
    if (admit(V, r, st)) V->running.push_back(k);
  }
  if (!V->running.empty()) {
    int32_t n_active = 0;
    egt_status s = egt_batch_step(V->batch, V->opts.iters_per_step, V->opts.group, &n_active, st);
    if (s != EGT_OK) {
      const std::string msg = egt_last_error();
      return fail(s, "egt_server_step: " + msg);
    }
    V->launches += 1;
    std::vector<int64_t> keep;
    for (int64_t k : V->running) {
      Request& r = V->reqs.at(k);
      egt_batch_member_info m{};
      s = egt_batch_member(V->batch, r.slot, &m);
      if (s != EGT_OK) return s;
      if (m.active) {
        keep.push_back(k);
        continue;
      }
      s = retire(V, r, st);
      if (s != EGT_OK) return s;
    }
    V->running.swap(keep);
  }
  if (stats) {
    stats->queued = (int32_t)V->queue.size();
    stats->running = (int32_t)V->running.size();
    stats->completed = V->completed;
    stats->launches = V->launches;
    stats->used_bytes = V->used;
    stats->budget_bytes = V->budget;
    stats->clock = V->now();
  }
  return EGT_OK;
}

egt_status egt_server_result(egt_server* V, int64_t id, egt_server_request_info* info, float* x, float* y,
                             int32_t release) {
  if (!V || !info) return fail(EGT_ERR_INVALID_ARG, "NULL argument");
  auto it = V->reqs.find(id);
  if (it == V->reqs.end()) return fail(EGT_ERR_INVALID_ARG, "no such request");
  Request& r = it->second;
  info->state = r.state;
  info->status = r.status;
  info->t_submit = r.t_submit;
  info->t_admit = r.t_admit;
  info->t_done = r.t_done;
  info->rep = r.rep;
  info->S[0] = r.S[0];
  info->S[1] = r.S[1];
  info->ld = r.ld;
  if (r.state == kDone) {
    if (x && !r.x.empty()) std::memcpy(x, r.x.data(), r.x.size() * sizeof(float));
    if (y && !r.y.empty()) std::memcpy(y, r.y.data(), r.y.size() * sizeof(float));
    if (release) V->reqs.erase(it);
  }
  return EGT_OK;
}

const char* egt_server_state_name(int32_t state) {
  return state >= 0 && state <= 2 ? kStateNames[state] : "?";
}

}  // extern "C"
