// Device-side game tables and kernel entry points (internal to libegt).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace egt {

constexpr int kSbrHands = 16;       // hands per SBR / best-response item (two lanes each)
constexpr int kMaxListLen = 64;     // max hands holding one card (four per lane in a half-warp scan)

// Per-card prefix arrays of a product item in shared memory: card slot c's prefix
// before its k-th hand (k = 0 .. list length) sits at pc_index(c, k, lmax).  One
// 16-byte entry of padding after every four keeps the card scan's stores (four
// consecutive entries per lane) free of bank conflicts.
__host__ __device__ inline int pc_pad(int k) { return k + (k >> 2); }
__host__ __device__ inline int pc_stride(int lmax) { return pc_pad(lmax) + 1; }
__host__ __device__ inline int pc_index(int c, int k, int lmax) { return c * pc_stride(lmax) + pc_pad(k); }

// One player's per-hand treeplex on the device (Sec. 4 notation).
struct DevTpx {
  int S, J, L;
  const int* inf_parent;   // [J] p_j, -1 for a root simplex
  const int* inf_first;    // [J] first sequence of I_j
  const int* inf_n;        // [J] n_j
  const int* level_ptr;    // [L+1]
  const int* child_ptr;    // [S+1] CSR of D_j^i
  const int* child_idx;
  const int* seq_par;      // [S] parent sequence of the sequence's simplex, -1 at a root simplex
  const double* beta;      // [J]
  const float* log_n;      // [J] log n_j
};

// Terminals grouped by the sequence of the output player (CSR over that player's sequences).
struct DevTerms {
  int n;                   // terminals
  const int* ptr;          // [S_p + 1]
  const int* opp_seq;      // [n] opponent sequence of the terminal
  const int* kind;         // [n] 0 fold, 1 showdown
  const float* coef;       // [n] signed: fold payoff to player 2, showdown +-stake
  const double* coef64;
  // Product items with merged terminals: one per opponent column the terminals read,
  // (showdown terminal, fold terminal, the column, 0), -1 where the column has no
  // terminal of a kind (every column has at most one of each)
  int n_col;
  const int4* col;         // [n_col]
  const int* col_order;    // [n_col] the items in descending order of work (showdown and
                           // fold, showdown, fold; column order within each)
};

// Whether a group of `ctas` CTAs takes a product phase of T terminals over n_col opponent
// columns in merged items (one per column): when that needs fewer rounds of items per
// CTA than one item per terminal (each round lasts about one item).
__host__ __device__ inline bool merge_items(int T, int n_col, int ctas) {
  return ctas > 0 && (n_col + ctas - 1) / ctas < (T + ctas - 1) / ctas;
}

struct DevGame {
  int H, ld;               // hands, leading dimension (multiple of 32)
  int hand_size;           // 1 or 2
  int n_slots;             // card slots (live cards + 1 empty slot used by padding / 1-card hands)
  int lmax;                // longest card list
  const uchar2* hcard;     // [ld] card slots of each (sorted) hand
  const ushort2* grp;      // [ld] tie group [lo, hi) in sorted order
  const uchar4* cpos;      // [ld] hands of card k before lo / hi: (lo0, hi0, lo1, hi1)
  // [ld] per hand, eight uint16: tie group lo, hi; then for each of its two card slots the
  // flat index (pc_index) of the per-card prefix before lo, before hi, and of the card's
  // total
  const uint4* hinfo;
  const uint16_t* card_hands;  // [n_slots][lmax] sorted hand indices holding the card
  const int* card_len;     // [n_slots]
  const float* r[2];       // [ld] normalised ranges rounded to FP32 (0 on padding): r_hi
  const float* rlo[2];     // [ld] RN32(r64 - r_hi): r64 = r_hi + r_lo to within 2^-48 r64
  const float* rz[2];      // [ld] r / Z
  const double* r64[2];
  const double* rz64[2];
  DevTpx tpx[2];
  DevTerms terms[2];       // terms[p]: grouped by player p's sequences (output of player p)
};

// Read-only view of a game's device tables, for entry points outside api.cu.
struct GameView {
  const DevGame* dg;
  int device;
  double bb;
  bool host_only;
};
bool game_view(const struct egt_game* G, GameView* out);

// Set the thread-local message returned by egt_last_error().
void set_last_error(const std::string& msg);

// Opt a kernel into the largest dynamic shared memory the device allows next to
// its static shared memory; returns the limit (bytes) or -1 on failure.
int opt_in_dynamic_smem(const void* kernel);

// ---- kernels ----
// Terminal contributions of player `player`'s product (A y for player 0, A^T x for
// player 1): c32 / c64 (either may be NULL) [terms[player].n][ld], row e = coef_e x the
// exact payoff sum of terminal e, without the r / Z factor (grad_impl.cuh).
template <typename TIn>
void launch_terms(const DevGame& g, int player, const TIn* in, float* c32, double* c64, cudaStream_t st);

// Both players' FP64 contributions in one launch (the saddle-point residual): player 0's
// from y into c64_0, player 1's from x into c64_1; every CTA runs the body of
// launch_terms, so the results are the same bits as two launches.
void launch_terms_pair64(const DevGame& g, const float* y, const float* x, double* c64_0, double* c64_1,
                         cudaStream_t st);

// Product rows from contributions: out[s][h] = rz[h] x (sum of the contributions of the
// terminals of sequence s, in terminal order); 0 on padding hands.
template <typename T>
void launch_combine(const DevGame& g, int player, const T* c, T* out, cudaStream_t st);

size_t grad_smem_bytes(const DevGame& g);

// SBR of player p on g (sign: +1 player 0, -1 player 1), temperature mu * beta_j.
// g may be NULL (treated as 0: the uniform behavioural strategy); with contrib it
// holds player p's terminal contributions (launch_terms), else a dense [S][ld] row set.  If out is
// non-NULL writes q, or (1 - tau) old + tau q when old is non-NULL.  If
// value_dev is non-NULL writes sum over hands and root simplexes of the value
// (FP64) to *value_dev, reducing per-CTA partials (partials[grid], counter).
struct SbrArgs {
  const float* g;
  bool contrib;
  float sign;
  double mu;
  const float* old;
  float tau;
  float* out;
  double* value_dev;
  double* partials;
  unsigned int* counter;
  int* status;             // set to 1 if a value turns NaN / Inf
};
void launch_sbr(const DevGame& g, int player, const SbrArgs& a, cudaStream_t st);
size_t sbr_smem_bytes(const DevGame& g, int player);

// Plain best response value in FP64: sign * (min over the treeplex of <q, sign * g>);
// g as in SbrArgs (contributions or dense rows).
void launch_br64(const DevGame& g, int player, const double* gv, bool contrib, double sign, double* value_dev,
                 double* partials, unsigned int* counter, cudaStream_t st);
size_t br_smem_bytes(const DevGame& g, int player);

// Both players' best-response values of the residual in one launch, from their
// terminal contributions: *value0 = min over x of <x, A y> (gv0), *value1 = max over y
// of <y, A^T x> (gv1).  Each player's CTAs reduce their own partials (partials[0 .. NB)
// and [NB .. 2 NB), counter[0] and counter[1]) in the order launch_br64 uses: the same
// bits as two launches.
void launch_br64_pair(const DevGame& g, const double* gv0, const double* gv1, double* value0, double* value1,
                      double* partials, unsigned int* counter, cudaStream_t st);

}  // namespace egt
