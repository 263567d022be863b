// Internals of libegt shared by the C-ABI translation units (api.cu: games, hot-path
// entry points and solver drivers; batch.cu: batches): the game object, error
// reporting, and the device-resident driver's control-block helpers.
#pragma once
#include <cmath>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/egt.h"
#include "egt_internal.cuh"
#include "engine.cuh"
#include "tree.hpp"

namespace egtapi {

// Record msg as the calling thread's egt_last_error text and return st.
egt_status fail(egt_status st, const std::string& msg);

#define CUDA_TRY(expr)                                                                 \
  do {                                                                                 \
    cudaError_t e__ = (expr);                                                          \
    if (e__ != cudaSuccess)                                                            \
      return fail(e__ == cudaErrorMemoryAllocation ? EGT_ERR_OOM : EGT_ERR_CUDA,       \
                  std::string(#expr) + ": " + cudaGetErrorString(e__));                \
  } while (0)

#define EGT_TRY(expr)                  \
  do {                                 \
    egt_status s__ = (expr);           \
    if (s__ != EGT_OK) return s__;     \
  } while (0)

// Restores the caller's current device when it goes out of scope.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (dev < 0) return;   // host-only game: no CUDA calls
    if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// An NVTX range over a public call (shown by Nsight tools; a no-op without one).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Integer value of environment variable `name`, or dflt when unset or empty.
int env_int(const char* name, int dflt);

}  // namespace egtapi

struct egt_game {
  int device = 0;
  egt::Compiled comp;
  // host copies
  int H = 0, ld = 0, hand_size = 2, n_slots = 0, lmax = 0;
  double Z = 0, normA = 0, M[2] = {0, 0}, Omega[2] = {0, 0}, bb = 1, pot = 1;
  std::vector<int32_t> order;
  // device arena of tables
  void* arena = nullptr;
  egt::DevGame dg{};
  // solver state and scratch (device)
  float* vec = nullptr;          // all float vectors
  // iterates x, y [S_p][ld]; products gx, gy in terminal-contribution form [T][ld];
  // scratch tx [max(S0, T)][ld], ty [max(S1, T)][ld]
  float *x[2], *y[2], *gx[2], *gy[2], *tx, *ty;
  int cur = 0;                   // index of the current iterate / cached products
  // player whose Step intermediate point (x_hat in tx / y_hat in ty) the last egt_step left in
  // the scratch; -1 once another call reused it (the device-resident driver writes it too)
  mutable int vhat_player = -1;
  double* g64[2] = {nullptr, nullptr};   // FP64 products for the gap (contributions)
  double* pub = nullptr;         // [T][ld] contributions of the public egt_grad / egt_grad_f64
  double* partials = nullptr;    // per-CTA value partials
  unsigned int* counter = nullptr;
  double* vals = nullptr;        // device value slots
  int* status = nullptr;         // device NaN flag
  double* pinned = nullptr;      // host readback of value slots
  double mu[2] = {0, 0};
  int t = 0;                     // iterations since egt_solver_init
  double tau = 0.5;              // EGT/as step size carried between iterations
  double last_gap = NAN;         // last residual computed by the solver (mbb)
  bool initialised = false;
  // device-resident driver (engine.cu)
  egt::EngineCtl* ctl_dev = nullptr;
  egt::EngineCtl* ctl_host = nullptr;
  double* eng_partials = nullptr;
  int eng_grid = -2;             // -2: not queried yet, <= 0: engine unavailable
  double eng_phase_ns[egt::kEnginePhases] = {0};
  double eng_phase_work_ns[egt::kEnginePhases] = {0};
  long long eng_phase_n[egt::kEnginePhases] = {0};
  bool host_only = false;        // compiled tables only (device = -1): queries work, kernels do not
  long long products = 0;
  // per-kernel device time accounting (egt_profile): CUDA events around each launch
  struct ProfRec {
    int kind;
    cudaEvent_t a, b;
  };
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<ProfRec> prof_pending;
  double prof_ms[EGT_KERNEL_KINDS] = {0};
  long long prof_n[EGT_KERNEL_KINDS] = {0};
  long long launches[EGT_KERNEL_KINDS] = {0};   // always counted, reset by egt_profile
  size_t table_bytes = 0;
  size_t device_bytes = 0;       // tables + solver state on the device (known before upload)
};

namespace egtapi {

// The game's buffers as the device-resident driver sees them.
egt::EngineBufs engine_bufs(const egt_game* G, egt_iter_log* log_dev, int log_cap);
// Control block of a launch of up to n iterations from the game's solver state.
void engine_ctl_init(const egt_game* G, egt::EngineCtl& c, int variant, double eps_mbb, int gap_every, int n);
// Take back the solver state a launch left in its control block (rep: host, may be NULL).
void engine_ctl_apply(egt_game* G, const egt::EngineCtl& c, egt_solve_report* rep);

}  // namespace egtapi
