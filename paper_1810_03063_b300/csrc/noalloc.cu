// egt_gap_noalloc: the saddle-point residual with its scratch memory in a
// file-scope device array instead of memory the library allocates.
//
// egt_gap keeps its FP64 product vectors and reduction partials in buffers
// that egt_create_game allocates for each game.  Some callers must not
// allocate device memory on their path: a serving process whose device memory
// is all reserved up front by another allocator, or a latency-critical loop
// that cannot afford the device-wide synchronisation cudaMalloc / cudaFree
// imply.  This entry point serves them: it allocates nothing; its scratch is
// g_noalloc_scratch below, a fixed kNoAllocScratchBytes array that every GPU
// which loads the library holds until the process exits.
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address with cudaGetSymbolAddress (in host code the array's
// name is only a host-side stand-in, never a device address) and caches it.
// That first call on each device should therefore come before any stream
// capture.  Every call ends by copying the residual to the host and waiting
// for its stream.  Every call shares the one array and it keeps the last call's
// contents: each call clears the parts that must start at zero (the value
// slots and the arrival counter of the reductions), and calls whose work
// overlaps on the GPU (different streams, no ordering) race on it.
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/egt.h"
#include "egt_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(2) << 20;   // 2 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// byte offsets inside the scratch array (256-byte aligned)
constexpr size_t kValsOff = 0;                 // 2 doubles: min_x <x, Ay>, max_y <y, A^T x>
constexpr size_t kCounterOff = 256;            // arrival counter of the value reductions
constexpr size_t kZeroBytes = 512;             // values + counter: cleared by every call
constexpr size_t kPartialsOff = 512;           // per-CTA partial values, <= 1024 CTAs
constexpr size_t kProdOff = kPartialsOff + 1024 * sizeof(double);   // FP64 A y, then A^T x
                                                                    // (terminal contributions [T][ld])

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
unsigned char* g_addr[kMaxDevices] = {};

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

egt_status fail(egt_status st, const std::string& msg) {
  egt::set_last_error("egt_gap_noalloc: " + msg);
  return st;
}

// Device address of the scratch array on the current device (looked up once per device).
egt_status scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return fail(EGT_ERR_INVALID_ARG, "device index above 63");
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return fail(EGT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[device] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[device];
  return EGT_OK;
}

}  // namespace

extern "C" egt_status egt_gap_noalloc(const egt_game* game, const float* x, const float* y,
                                      double* gap_mbb, void* stream) {
  egt::GameView v{};
  if (!egt::game_view(game, &v)) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (v.host_only) return fail(EGT_ERR_INVALID_ARG, "host-only game (device -1) has no device tables");
  if (!x || !y || !gap_mbb) return fail(EGT_ERR_INVALID_ARG, "NULL argument");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15)
    return fail(EGT_ERR_INVALID_ARG, "x and y must be 16-byte aligned");
  const egt::DevGame& dg = *v.dg;
  const size_t n0 = (size_t)dg.terms[0].n * dg.ld, n1 = (size_t)dg.terms[1].n * dg.ld;
  const size_t need = kProdOff + round256(n0 * sizeof(double)) + n1 * sizeof(double);
  if (need > kNoAllocScratchBytes)
    return fail(EGT_ERR_INVALID_ARG, "the game needs " + std::to_string(need) +
                                         " bytes of scratch; the static scratch holds " +
                                         std::to_string(kNoAllocScratchBytes));
  if (dg.ld / egt::kSbrHands > 1024) return fail(EGT_ERR_INVALID_ARG, "too many hands");

  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(v.device) != cudaSuccess)
    return fail(EGT_ERR_CUDA, "cannot make the game's device current");
  struct Restore {
    int d;
    ~Restore() {
      if (d >= 0) cudaSetDevice(d);
    }
  } restore{prev};

  unsigned char* base = nullptr;
  egt_status s = scratch_address(v.device, &base);
  if (s != EGT_OK) return s;
  double* vals = reinterpret_cast<double*>(base + kValsOff);
  unsigned int* counter = reinterpret_cast<unsigned int*>(base + kCounterOff);
  double* partials = reinterpret_cast<double*>(base + kPartialsOff);
  double* ay = reinterpret_cast<double*>(base + kProdOff);
  double* atx = reinterpret_cast<double*>(base + kProdOff + round256(n0 * sizeof(double)));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  cudaError_t e = cudaMemsetAsync(base, 0, kZeroBytes, st);
  if (e != cudaSuccess) return fail(EGT_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  egt::launch_terms<float>(dg, 0, y, nullptr, ay, st);                            // A y
  egt::launch_terms<float>(dg, 1, x, nullptr, atx, st);                           // A^T x
  egt::launch_br64(dg, 0, ay, true, 1.0, vals + 0, partials, counter, st);        // min_x <x, Ay>
  egt::launch_br64(dg, 1, atx, true, -1.0, vals + 1, partials, counter, st);      // max_y <y, A^T x>
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(EGT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  double host_vals[2] = {0.0, 0.0};
  e = cudaMemcpyAsync(host_vals, vals, sizeof(host_vals), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(EGT_ERR_CUDA, std::string("readback: ") + cudaGetErrorString(e));
  const double eps = host_vals[1] - host_vals[0];
  if (!std::isfinite(eps)) return fail(EGT_ERR_NUMERIC, "non-finite saddle-point residual");
  *gap_mbb = eps * (1000.0 / v.bb);
  return EGT_OK;
}
