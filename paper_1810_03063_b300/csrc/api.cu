// C-ABI of libegt (include/egt.h): game compilation and upload, the gradient /
// smoothed-best-response / gap entry points, and the EGT drivers (Alg. 1-4).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "api_internal.hpp"

using namespace egt;
using namespace egtapi;

namespace {

thread_local std::string g_last_error;

constexpr int kMaxLd = 1536;   // 3 hands per thread of a 512-thread CTA in the product kernels
constexpr double kTauMin = 1.0 / (1u << 30);

}  // namespace

namespace egtapi {

egt_status fail(egt_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return v && *v ? std::atoi(v) : dflt;
}

}  // namespace egtapi


namespace {

size_t vec_elems(const egt_game* G, int p) { return (size_t)G->comp.tpx[p].S * G->ld; }
size_t contrib_elems(const egt_game* G) { return std::max<size_t>(G->comp.term.size(), 1) * G->ld; }

// Device bytes alloc_state takes (the sizes of alloc_state below).
size_t state_bytes(const egt_game* G) {
  const size_t n0 = vec_elems(G, 0), n1 = vec_elems(G, 1), nc = contrib_elems(G);
  const size_t t0 = std::max(n0, nc), t1 = std::max(n1, nc);
  const size_t floats = 2 * n0 + 2 * n1 + 4 * nc + t0 + t1 + 10 * 64;
  return floats * sizeof(float) + 3 * nc * sizeof(double) + 1024 * sizeof(double) + 16 * 4 + 16 * 8 + 4 +
         sizeof(EngineCtl) + 4 * (size_t)(G->ld / kSbrHands) * sizeof(double);
}


egt_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(EGT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return EGT_OK;
}

egt_status validate(const egt_game_desc* d) {
  if (!d) return fail(EGT_ERR_INVALID_ARG, "desc is NULL");
  if (d->hand_size != 1 && d->hand_size != 2) return fail(EGT_ERR_INVALID_ARG, "hand_size must be 1 or 2");
  if (d->n_cards < 1 || d->n_cards > 254) return fail(EGT_ERR_INVALID_ARG, "n_cards out of range [1, 254]");
  if (d->n_hands < 1) return fail(EGT_ERR_INVALID_ARG, "n_hands < 1");
  if (!d->hand_cards || !d->strength || !d->range[0] || !d->range[1])
    return fail(EGT_ERR_INVALID_ARG, "NULL hand_cards / strength / range");
  if (!(d->pot > 0) || !(d->stack >= 0) || !(d->bb > 0) || !std::isfinite(d->pot) ||
      !std::isfinite(d->stack) || !std::isfinite(d->bb))
    return fail(EGT_ERR_INVALID_ARG, "pot, bb must be > 0 and stack >= 0, finite");
  if (d->n_bets < 0 || (d->n_bets > 0 && !d->bet_fracs)) return fail(EGT_ERR_INVALID_ARG, "bad bet menu");
  for (int i = 0; i < d->n_bets; ++i)
    if (!(d->bet_fracs[i] > 0) || !std::isfinite(d->bet_fracs[i]))
      return fail(EGT_ERR_INVALID_ARG, "bet fractions must be > 0 and finite");
  if (d->raise_cap < 0) return fail(EGT_ERR_INVALID_ARG, "raise_cap < 0");
  if (d->menus)
    for (int m = 0; m < 8; ++m) {
      const egt_menu& mu = d->menus[m];
      if (mu.n < 0 || (mu.n > 0 && !mu.fracs)) return fail(EGT_ERR_INVALID_ARG, "bad bet menu");
      for (int i = 0; i < mu.n; ++i)
        if (!(mu.fracs[i] > 0) || !std::isfinite(mu.fracs[i]))
          return fail(EGT_ERR_INVALID_ARG, "menu pot fractions must be finite and > 0");
    }
  const int H = d->n_hands, k = d->hand_size;
  std::vector<std::pair<int, int>> seen;
  seen.reserve(H);
  for (int h = 0; h < H; ++h) {
    int a = d->hand_cards[h * k], b = k == 2 ? d->hand_cards[h * k + 1] : -1;
    if (a < 0 || a >= d->n_cards || (k == 2 && (b < 0 || b >= d->n_cards)))
      return fail(EGT_ERR_INVALID_ARG, "card id out of range at hand " + std::to_string(h));
    if (k == 2 && a == b) return fail(EGT_ERR_INVALID_ARG, "repeated card in hand " + std::to_string(h));
    if (k == 2 && a > b) std::swap(a, b);
    seen.push_back({a, b});
  }
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
    return fail(EGT_ERR_INVALID_ARG, "two hands hold the same cards");
  for (int p = 0; p < 2; ++p) {
    double tot = 0;
    for (int h = 0; h < H; ++h) {
      double r = d->range[p][h];
      if (!(r >= 0) || !std::isfinite(r)) return fail(EGT_ERR_INVALID_ARG, "range entries must be finite and >= 0");
      tot += r;
    }
    if (!(tot > 0)) return fail(EGT_ERR_INVALID_ARG, "a range is all zero");
  }
  return EGT_OK;
}

template <typename T>
T* carve(char*& p, size_t n) {
  p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p) + 255) & ~uintptr_t(255));
  T* out = reinterpret_cast<T*>(p);
  p += n * sizeof(T);
  return out;
}

// Host tables (card slots, tie groups, ranges, Z, ||A||, M, Omega, terminal CSR); with
// to_device, uploaded as one device arena that G->dg points into.
egt_status upload(egt_game* G, const egt_game_desc* d, bool to_device, cudaStream_t st) {
  const int H = G->H, ld = G->ld, k = d->hand_size;
  Compiled& C = G->comp;

  // card slots: live cards in ascending id, plus an empty slot (padding, 1-card hands)
  std::vector<int> slot_of(d->n_cards, -1);
  for (int h = 0; h < H; ++h)
    for (int c = 0; c < k; ++c) slot_of[d->hand_cards[h * k + c]] = 1;
  int ns = 0;
  for (int c = 0; c < d->n_cards; ++c)
    if (slot_of[c] > 0) slot_of[c] = ns++;
  const int empty = ns;
  G->n_slots = ns + 1;
  if (G->n_slots > 255) return fail(EGT_ERR_INVALID_ARG, "more than 254 live cards");

  std::vector<uchar2> hcard(ld);
  std::vector<std::vector<int>> lists(G->n_slots);
  for (int s = 0; s < ld; ++s) {
    if (s < H) {
      const int h = G->order[s];
      const int a = slot_of[d->hand_cards[h * k]];
      const int b = k == 2 ? slot_of[d->hand_cards[h * k + 1]] : empty;
      hcard[s] = make_uchar2((unsigned char)a, (unsigned char)b);
      lists[a].push_back(s);
      if (k == 2) lists[b].push_back(s);
    } else {
      hcard[s] = make_uchar2((unsigned char)empty, (unsigned char)empty);
    }
  }
  G->lmax = 1;
  for (auto& l : lists) G->lmax = std::max<int>(G->lmax, (int)l.size());
  if (G->lmax > kMaxListLen) return fail(EGT_ERR_INVALID_ARG, "a card is held by more than 64 hands");

  // tie groups in sorted order; padding forms one group at the end
  std::vector<ushort2> grp(ld);
  for (int s = 0; s < H;) {
    int e = s;
    const int str = d->strength[G->order[s]];
    while (e < H && d->strength[G->order[e]] == str) ++e;
    for (int i = s; i < e; ++i) grp[i] = make_ushort2((unsigned short)s, (unsigned short)e);
    s = e;
  }
  for (int s = H; s < ld; ++s) grp[s] = make_ushort2((unsigned short)H, (unsigned short)ld);

  std::vector<uchar4> cpos(ld, make_uchar4(0, 0, 0, 0));
  auto count_below = [&](int slot, int bound) {
    const auto& l = lists[slot];
    return (unsigned char)(std::lower_bound(l.begin(), l.end(), bound) - l.begin());
  };
  for (int s = 0; s < H; ++s) {
    cpos[s] = make_uchar4(count_below(hcard[s].x, grp[s].x), count_below(hcard[s].x, grp[s].y),
                          count_below(hcard[s].y, grp[s].x), count_below(hcard[s].y, grp[s].y));
  }
  std::vector<uint16_t> card_hands((size_t)G->n_slots * G->lmax, 0);
  // per-hand record of flat shared-memory indices used by the product kernels
  std::vector<uint4> hinfo(ld);
  {
    auto at = [&](unsigned slot, unsigned k) { return (unsigned)pc_index((int)slot, (int)k, G->lmax); };
    for (int s = 0; s < ld; ++s) {
      const unsigned a = hcard[s].x, b = hcard[s].y;
      const unsigned la = (unsigned)lists[a].size(), lb = (unsigned)lists[b].size();
      hinfo[s] = make_uint4(grp[s].x | ((unsigned)grp[s].y << 16),
                            at(a, cpos[s].x) | (at(a, cpos[s].y) << 16),
                            at(a, la) | (at(b, cpos[s].z) << 16),
                            at(b, cpos[s].w) | (at(b, lb) << 16));
    }
  }
  std::vector<int> card_len(G->n_slots);
  for (int c = 0; c < G->n_slots; ++c) {
    card_len[c] = (int)lists[c].size();
    for (size_t i = 0; i < lists[c].size(); ++i) card_hands[(size_t)c * G->lmax + i] = (uint16_t)lists[c][i];
  }

  // ranges: normalised, Z by inclusion-exclusion over shared cards
  std::vector<double> r[2];
  std::vector<double> per_card[2];
  double R[2];
  for (int p = 0; p < 2; ++p) {
    r[p].assign(ld, 0.0);
    double tot = 0;
    for (int h = 0; h < H; ++h) tot += d->range[p][h];
    for (int s = 0; s < H; ++s) r[p][s] = d->range[p][G->order[s]] / tot;
    R[p] = 0;
    for (int s = 0; s < H; ++s) R[p] += r[p][s];
    per_card[p].assign(G->n_slots, 0.0);
    for (int s = 0; s < H; ++s) {
      per_card[p][hcard[s].x] += r[p][s];
      if (k == 2) per_card[p][hcard[s].y] += r[p][s];
    }
  }
  double Z = R[0] * R[1];
  for (int c = 0; c < ns; ++c) Z -= per_card[0][c] * per_card[1][c];
  if (k == 2)
    for (int s = 0; s < H; ++s) Z += r[0][s] * r[1][s];
  if (!(Z > 0)) return fail(EGT_ERR_INVALID_ARG, "no compatible hand pair has positive probability (Z = 0)");
  G->Z = Z;

  // ||A|| = max_ij |A_ij|: largest |coef| of each terminal kind times the largest chance
  // weight r1(a) r2(b) over compatible pairs (any pair for folds, pairs of unequal
  // strength for showdowns).  For each a the largest r2(b) over the b it may meet gives
  // its largest product (a product with r1(a) >= 0 is monotone in r2(b)), so each a scans
  // the hands in descending r2 only past those that share a card with it (at most two
  // card lists) and, for showdowns, its tie group as well.
  double max_any = 0, max_diff = 0;
  {
    std::vector<int> by_r1(H);
    std::iota(by_r1.begin(), by_r1.end(), 0);
    std::stable_sort(by_r1.begin(), by_r1.end(), [&](int u, int v) { return r[1][u] > r[1][v]; });
    for (int a = 0; a < H; ++a) {
      bool got_any = false;
      for (int b : by_r1) {
        const bool share = hcard[a].x == hcard[b].x || (k == 2 && (hcard[a].x == hcard[b].y ||
                                                                   hcard[a].y == hcard[b].x ||
                                                                   hcard[a].y == hcard[b].y));
        if (share) continue;
        const double w = r[0][a] * r[1][b];
        if (!got_any) {
          max_any = std::max(max_any, w);
          got_any = true;
        }
        if (d->strength[G->order[a]] != d->strength[G->order[b]]) {
          max_diff = std::max(max_diff, w);
          break;
        }
      }
    }
  }
  double na = 0;
  for (auto& t : C.term) na = std::max(na, std::fabs(t.coef) * (t.kind == 0 ? max_any : max_diff));
  G->normA = na / Z;
  for (int p = 0; p < 2; ++p) {
    G->M[p] = H * C.tpx[p].m_root;
    G->Omega[p] = H * C.tpx[p].omega_root;
  }

  // terminals grouped by each player's own sequence
  std::vector<int> tptr[2], topp[2], tkind[2];
  std::vector<float> tcoef[2];
  std::vector<double> tcoef64[2];
  for (int p = 0; p < 2; ++p) {
    const int S = C.tpx[p].S;
    tptr[p].assign(S + 1, 0);
    for (auto& t : C.term) tptr[p][t.seq[p] + 1]++;
    for (int s = 0; s < S; ++s) tptr[p][s + 1] += tptr[p][s];
    std::vector<int> fill(tptr[p].begin(), tptr[p].end() - 1);
    const int n = (int)C.term.size();
    topp[p].resize(n);
    tkind[p].resize(n);
    tcoef[p].resize(n);
    tcoef64[p].resize(n);
    for (auto& t : C.term) {
      const int e = fill[t.seq[p]]++;
      topp[p][e] = t.seq[1 - p];
      tkind[p][e] = t.kind;
      // showdown: payoff to player 2 is +stake when player 2 is stronger; the kernel forms
      // (stronger - weaker) from the output hand's view, so player 2's rows flip the sign
      const double c = t.kind == 0 ? t.coef : (p == 0 ? t.coef : -t.coef);
      tcoef64[p][e] = c;
      tcoef[p][e] = (float)c;
    }
  }
  // merged product items: the showdown and fold terminals of each opponent column
  std::vector<int> tcol[2], tord[2];
  for (int p = 0; p < 2; ++p) {
    const int S_opp = C.tpx[1 - p].S;
    std::vector<int> at(S_opp, -1);
    const int n = (int)C.term.size();
    for (int e = 0; e < n; ++e) {
      const int o = topp[p][e];
      if (at[o] < 0) {
        at[o] = (int)tcol[p].size() / 4;
        tcol[p].insert(tcol[p].end(), {-1, -1, o, 0});
      }
      int& slot = tcol[p][4 * at[o] + (tkind[p][e] ? 0 : 1)];
      if (slot >= 0) return fail(EGT_ERR_INVALID_ARG, "internal: two terminals of one kind read one column");
      slot = e;
    }
    // the items in descending order of work (a showdown and a fold, a showdown alone, a
    // fold alone, which skips the prefixes): the order in which the one-game driver
    // deals them out in rounds of alternating direction, which gives every CTA about the
    // same work.  Each item writes only its own terminals' rows, so no order changes a
    // result.  (Batches keep the column order: there the sorted order measured slower.)
    const int nc = (int)tcol[p].size() / 4;
    tord[p].resize(nc);
    for (int i = 0; i < nc; ++i) tord[p][i] = i;
    auto cls = [&](int i) {
      const bool sd = tcol[p][4 * i] >= 0, fo = tcol[p][4 * i + 1] >= 0;
      return sd && fo ? 0 : (sd ? 1 : 2);
    };
    std::stable_sort(tord[p].begin(), tord[p].end(), [&](int a, int b) { return cls(a) < cls(b); });
  }

  // sizes of the arena
  std::vector<float> rf[2], rlof[2], rzf[2];
  std::vector<double> rz64[2];
  for (int p = 0; p < 2; ++p) {
    rf[p].resize(ld);
    rlof[p].resize(ld);
    rzf[p].resize(ld);
    rz64[p].resize(ld);
    for (int s = 0; s < ld; ++s) {
      rf[p][s] = (float)r[p][s];
      rlof[p][s] = (float)(r[p][s] - (double)rf[p][s]);
      rz64[p][s] = r[p][s] / Z;
      rzf[p][s] = (float)rz64[p][s];
    }
  }
  struct TpxHost {
    std::vector<float> log_n;
  } th[2];
  for (int p = 0; p < 2; ++p) {
    th[p].log_n.resize(C.tpx[p].J);
    for (int j = 0; j < C.tpx[p].J; ++j) th[p].log_n[j] = (float)std::log((double)C.tpx[p].inf_n[j]);
  }

  size_t bytes = 1 << 16;
  bytes += ld * (sizeof(uchar2) + sizeof(ushort2) + sizeof(uchar4) + sizeof(uint4)) + card_hands.size() * 2 +
           card_len.size() * 4;
  for (int p = 0; p < 2; ++p) {
    bytes += ld * (3 * sizeof(float) + 2 * sizeof(double));
    const Treeplex& T = C.tpx[p];
    bytes += (4 * T.J + T.L + 1 + 2 * T.S + 1 + T.child_idx.size()) * sizeof(int) + T.J * (sizeof(double) + sizeof(float));
    bytes += (tptr[p].size() + 2 * topp[p].size() + tcol[p].size() + tord[p].size()) * sizeof(int) +
             tcoef[p].size() * (sizeof(float) + sizeof(double));
  }
  bytes += 64 * 256;   // alignment slack
  G->device_bytes = bytes + state_bytes(G);
  if (!to_device) return EGT_OK;
  std::vector<char> host(bytes, 0);
  CUDA_TRY(cudaMalloc(&G->arena, bytes));
  char* hp = host.data();
  const uintptr_t base_h = reinterpret_cast<uintptr_t>(host.data());
  const uintptr_t base_d = reinterpret_cast<uintptr_t>(G->arena);
  bool overflow = false;
  auto put = [&](const void* src, size_t nbytes) -> const void* {
    hp = reinterpret_cast<char*>(base_h + ((reinterpret_cast<uintptr_t>(hp) - base_h + 255) & ~uintptr_t(255)));
    if ((size_t)(reinterpret_cast<uintptr_t>(hp) - base_h) + nbytes > bytes) {
      overflow = true;
      return nullptr;
    }
    if (nbytes) std::memcpy(hp, src, nbytes);
    const void* dev = reinterpret_cast<const void*>(base_d + (reinterpret_cast<uintptr_t>(hp) - base_h));
    hp += nbytes;
    return dev;
  };
  DevGame& g = G->dg;
  g.H = H;
  g.ld = ld;
  g.hand_size = k;
  g.n_slots = G->n_slots;
  g.lmax = G->lmax;
  g.hcard = (const uchar2*)put(hcard.data(), ld * sizeof(uchar2));
  g.grp = (const ushort2*)put(grp.data(), ld * sizeof(ushort2));
  g.cpos = (const uchar4*)put(cpos.data(), ld * sizeof(uchar4));
  g.hinfo = (const uint4*)put(hinfo.data(), ld * sizeof(uint4));
  g.card_hands = (const uint16_t*)put(card_hands.data(), card_hands.size() * 2);
  g.card_len = (const int*)put(card_len.data(), card_len.size() * 4);
  for (int p = 0; p < 2; ++p) {
    g.r[p] = (const float*)put(rf[p].data(), ld * 4);
    g.rlo[p] = (const float*)put(rlof[p].data(), ld * 4);
    g.rz[p] = (const float*)put(rzf[p].data(), ld * 4);
    g.r64[p] = (const double*)put(r[p].data(), ld * 8);
    g.rz64[p] = (const double*)put(rz64[p].data(), ld * 8);
    const Treeplex& T = C.tpx[p];
    DevTpx& dt = g.tpx[p];
    dt.S = T.S;
    dt.J = T.J;
    dt.L = T.L;
    dt.inf_parent = (const int*)put(T.inf_parent.data(), T.J * 4);
    dt.inf_first = (const int*)put(T.inf_first.data(), T.J * 4);
    dt.inf_n = (const int*)put(T.inf_n.data(), T.J * 4);
    dt.level_ptr = (const int*)put(T.level_ptr.data(), (T.L + 1) * 4);
    dt.child_ptr = (const int*)put(T.child_ptr.data(), (T.S + 1) * 4);
    dt.child_idx = (const int*)put(T.child_idx.data(), T.child_idx.size() * 4);
    std::vector<int> seq_par(T.S, -1);
    for (int j = 0; j < T.J; ++j)
      for (int i = 0; i < T.inf_n[j]; ++i) seq_par[T.inf_first[j] + i] = T.inf_parent[j];
    dt.seq_par = (const int*)put(seq_par.data(), T.S * 4);
    dt.beta = (const double*)put(T.beta.data(), T.J * 8);
    dt.log_n = (const float*)put(th[p].log_n.data(), T.J * 4);
    DevTerms& tm = g.terms[p];
    tm.n = (int)C.term.size();
    tm.ptr = (const int*)put(tptr[p].data(), tptr[p].size() * 4);
    tm.opp_seq = (const int*)put(topp[p].data(), topp[p].size() * 4);
    tm.kind = (const int*)put(tkind[p].data(), tkind[p].size() * 4);
    tm.coef = (const float*)put(tcoef[p].data(), tcoef[p].size() * 4);
    tm.coef64 = (const double*)put(tcoef64[p].data(), tcoef64[p].size() * 8);
    tm.n_col = (int)tcol[p].size() / 4;
    tm.col = (const int4*)put(tcol[p].data(), tcol[p].size() * 4);
    tm.col_order = (const int*)put(tord[p].data(), tord[p].size() * 4);
  }
  const size_t used = reinterpret_cast<uintptr_t>(hp) - base_h;
  if (overflow || used > bytes) return fail(EGT_ERR_INVALID_ARG, "internal: table arena overflow");
  G->table_bytes = used;
  CUDA_TRY(cudaMemcpyAsync(G->arena, host.data(), used, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return EGT_OK;
}

egt_status alloc_state(egt_game* G) {
  const size_t n0 = vec_elems(G, 0), n1 = vec_elems(G, 1), nc = contrib_elems(G);
  const size_t t0 = std::max(n0, nc), t1 = std::max(n1, nc);
  const size_t total = 2 * n0 + 2 * n1 + 4 * nc + t0 + t1 + 10 * 64;   // each rounded up to 64 floats
  CUDA_TRY(cudaMalloc(&G->vec, total * sizeof(float)));
  CUDA_TRY(cudaMemset(G->vec, 0, total * sizeof(float)));
  float* p = G->vec;
  auto take = [&](size_t n) {
    float* q = p;
    p += (n + 63) / 64 * 64;
    return q;
  };
  for (int i = 0; i < 2; ++i) {
    G->x[i] = take(n0);
    G->gx[i] = take(nc);
    G->y[i] = take(n1);
    G->gy[i] = take(nc);
  }
  G->tx = take(t0);
  G->ty = take(t1);
  CUDA_TRY(cudaMalloc(&G->g64[0], nc * sizeof(double)));
  CUDA_TRY(cudaMalloc(&G->g64[1], nc * sizeof(double)));
  CUDA_TRY(cudaMalloc(&G->pub, nc * sizeof(double)));
  CUDA_TRY(cudaMalloc(&G->partials, 1024 * sizeof(double)));
  CUDA_TRY(cudaMalloc(&G->counter, 16 * sizeof(unsigned int)));
  CUDA_TRY(cudaMemset(G->counter, 0, 16 * sizeof(unsigned int)));
  CUDA_TRY(cudaMalloc(&G->vals, 16 * sizeof(double)));
  CUDA_TRY(cudaMemset(G->vals, 0, 16 * sizeof(double)));
  CUDA_TRY(cudaMalloc(&G->status, sizeof(int)));
  CUDA_TRY(cudaMemset(G->status, 0, sizeof(int)));
  CUDA_TRY(cudaHostAlloc(&G->pinned, 16 * sizeof(double), cudaHostAllocDefault));
  CUDA_TRY(cudaMalloc(&G->ctl_dev, sizeof(EngineCtl)));
  CUDA_TRY(cudaHostAlloc(&G->ctl_host, sizeof(EngineCtl), cudaHostAllocDefault));
  CUDA_TRY(cudaMalloc(&G->eng_partials, 4 * (size_t)(G->ld / kSbrHands) * sizeof(double)));
  return EGT_OK;
}

void free_game(egt_game* G) {
  if (!G) return;
  if (G->host_only) {
    delete G;
    return;
  }
  cudaFree(G->arena);
  cudaFree(G->vec);
  cudaFree(G->g64[0]);
  cudaFree(G->g64[1]);
  cudaFree(G->pub);
  cudaFree(G->partials);
  cudaFree(G->counter);
  cudaFree(G->vals);
  cudaFree(G->status);
  if (G->pinned) cudaFreeHost(G->pinned);
  cudaFree(G->ctl_dev);
  if (G->ctl_host) cudaFreeHost(G->ctl_host);
  cudaFree(G->eng_partials);
  for (auto& r : G->prof_pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : G->ev_pool) cudaEventDestroy(e);
  delete G;
}


egt_status check_player(int p) {
  if (p != 0 && p != 1) return fail(EGT_ERR_INVALID_ARG, "player must be 0 or 1");
  return EGT_OK;
}

egt_status check_ptr(const void* p, const char* name) {
  if (!p) return fail(EGT_ERR_INVALID_ARG, std::string(name) + " is NULL");
  if (reinterpret_cast<uintptr_t>(p) & 15) return fail(EGT_ERR_INVALID_ARG, std::string(name) + " is not 16-byte aligned");
  return EGT_OK;
}

// ---- per-kernel timing ----

cudaEvent_t prof_event(egt_game* G) {
  if (!G->ev_pool.empty()) {
    cudaEvent_t e = G->ev_pool.back();
    G->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Fold finished timing records into the totals (waits for each record's end event).
egt_status prof_drain(egt_game* G) {
  for (auto& r : G->prof_pending) {
    float ms = 0.f;
    CUDA_TRY(cudaEventSynchronize(r.b));
    CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
    G->prof_ms[r.kind] += ms;
    G->prof_n[r.kind] += 1;
    G->ev_pool.push_back(r.a);
    G->ev_pool.push_back(r.b);
  }
  G->prof_pending.clear();
  return EGT_OK;
}

// Run one kernel launch, bracketed by events when accounting is on.
template <typename F>
egt_status timed(egt_game* G, int kind, cudaStream_t st, const char* what, F&& launch, int count = 1) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (G->prof_on) {
    if (G->prof_pending.size() > 4096) EGT_TRY(prof_drain(G));
    a = prof_event(G);
    b = prof_event(G);
    cudaEventRecord(a, st);
  }
  launch();
  G->launches[kind] += count;
  egt_status s = check_launch(what);
  if (G->prof_on) {
    cudaEventRecord(b, st);
    G->prof_pending.push_back({kind, a, b});
  }
  return s;
}

// ---- internal launches (no argument checks) ----

// Player's product of `in` in terminal-contribution form (out [T][ld]).
egt_status grad32(egt_game* G, int player, const float* in, float* out, cudaStream_t st) {
  G->products++;
  return timed(G, EGT_KERNEL_GRAD_F32, st, "grad kernel",
               [&] { launch_terms<float>(G->dg, player, in, out, nullptr, st); });
}

// SBR of player p with loss gradient sign * g (player 1 receives A^T x and negates);
// g holds contributions (grad32) unless dense.
egt_status sbr(egt_game* G, int p, const float* g, double mu, const float* old, double tau,
               float* out, int value_slot, cudaStream_t st, bool dense = false) {
  SbrArgs a{};
  a.g = g;
  a.contrib = !dense;
  a.sign = p == 0 ? 1.f : -1.f;
  a.mu = mu;
  a.old = old;
  a.tau = (float)tau;
  a.out = out;
  a.value_dev = value_slot >= 0 ? G->vals + value_slot : nullptr;
  a.partials = G->partials;
  a.counter = G->counter;
  a.status = G->status;
  return timed(G, EGT_KERNEL_SBR, st, "sbr kernel", [&] { launch_sbr(G->dg, p, a, st); });
}

// Copy value slots [first, first + n) to the pinned host buffer and check them.
egt_status read_vals(egt_game* G, int first, int n, cudaStream_t st) {
  CUDA_TRY(cudaMemcpyAsync(G->pinned + first, G->vals + first, n * sizeof(double),
                           cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = first; i < first + n; ++i)
    if (!std::isfinite(G->pinned[i])) return fail(EGT_ERR_NUMERIC, "non-finite value in a best response");
  return EGT_OK;
}

// The two products and the two best responses each run as one launch over both
// players (the same bits as one launch per player); each counts as one launch per player.
egt_status gap_internal(egt_game* G, const float* x, const float* y, double* gap_mbb, cudaStream_t st) {
  EGT_TRY(timed(G, EGT_KERNEL_GRAD_F64, st, "grad f64 kernel",               // A y, A^T x
                [&] { launch_terms_pair64(G->dg, y, x, G->g64[0], G->g64[1], st); }, 2));
  EGT_TRY(timed(G, EGT_KERNEL_BR_F64, st, "br kernel", [&] {                // min_x <x, Ay>, max_y <y, A^T x>
    launch_br64_pair(G->dg, G->g64[0], G->g64[1], G->vals + 8, G->vals + 9, G->partials, G->counter, st);
  }, 2));
  CUDA_TRY(cudaMemcpyAsync(G->pinned + 8, G->vals + 8, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  const double eps = G->pinned[9] - G->pinned[8];
  if (!std::isfinite(eps)) return fail(EGT_ERR_NUMERIC, "non-finite saddle-point residual");
  *gap_mbb = eps * (1000.0 / G->bb);   // mbb per hand (the engine uses the same scale)
  return EGT_OK;
}

// Initial point (Alg. 1 / 3 first lines) at the given mu; leaves x, y, Ay, A^T x in slot cur.
egt_status init_point(egt_game* G, cudaStream_t st) {
  G->vhat_player = -1;
  const int c = G->cur;
  EGT_TRY(sbr(G, 0, nullptr, 1.0, nullptr, 0, G->tx, -1, st));          // x_omega (uniform)
  EGT_TRY(grad32(G, 1, G->tx, G->gy[c], st));                            // A^T x_omega
  EGT_TRY(sbr(G, 1, G->gy[c], G->mu[1], nullptr, 0, G->y[c], -1, st));    // y0 = y_mu_y(x_omega)
  EGT_TRY(grad32(G, 0, G->y[c], G->gx[c], st));                          // A y0
  EGT_TRY(sbr(G, 0, G->gx[c], G->mu[0], nullptr, 0, G->x[c], 0, st));     // x0 = x_mu_x(y0), phi
  EGT_TRY(grad32(G, 1, G->x[c], G->gy[c], st));                          // A^T x0
  return EGT_OK;
}

// EGV(x, y) of the current state = phi_mu_x(y) - f_mu_y(x); slot 0 must hold phi already.
egt_status current_egv(egt_game* G, double* egv, cudaStream_t st) {
  const int c = G->cur;
  EGT_TRY(sbr(G, 1, G->gy[c], G->mu[1], nullptr, 0, nullptr, 1, st));   // value of SBR_Y(-A^T x) = -f
  EGT_TRY(read_vals(G, 0, 2, st));
  *egv = G->pinned[0] + G->pinned[1];
  return EGT_OK;
}

// One Step (Alg. 2) focused on `me` at tau, from state slot cur into slot 1 - cur.
// Products are taken of the new iterates directly, so the cached A y / A^T x of the
// state are always products of its own iterates.  With want_egv, the EGV of the
// new point is left in value slots 2 (phi) and 3 (-f).
egt_status step_once(egt_game* G, int me, double tau, bool want_egv, cudaStream_t st) {
  const int c = G->cur, n = 1 - c;
  const double mx = G->mu[0], my = G->mu[1];
  if (me == 0) {
    // x_hat = (1-tau) x + tau x_mu_x(y)
    EGT_TRY(sbr(G, 0, G->gx[c], mx, G->x[c], tau, G->tx, -1, st));
    EGT_TRY(grad32(G, 1, G->tx, G->ty, st));                               // A^T x_hat
    // y_+ = (1-tau) y + tau y_mu_y(x_hat)
    EGT_TRY(sbr(G, 1, G->ty, my, G->y[c], tau, G->y[n], -1, st));
    EGT_TRY(grad32(G, 0, G->y[n], G->gx[n], st));                          // A y_+
    // x_tilde = x_{(1-tau) mu_x}(y_+); x_+ = (1-tau) x + tau x_tilde; value = phi_{mu_x+}(y_+)
    EGT_TRY(sbr(G, 0, G->gx[n], (1 - tau) * mx, G->x[c], tau, G->x[n], 2, st));
    EGT_TRY(grad32(G, 1, G->x[n], G->gy[n], st));                          // A^T x_+
    if (want_egv) EGT_TRY(sbr(G, 1, G->gy[n], my, nullptr, 0, nullptr, 3, st));   // -f_mu_y(x_+)
  } else {
    EGT_TRY(sbr(G, 1, G->gy[c], my, G->y[c], tau, G->ty, -1, st));        // y_hat
    EGT_TRY(grad32(G, 0, G->ty, G->tx, st));                               // A y_hat
    EGT_TRY(sbr(G, 0, G->tx, mx, G->x[c], tau, G->x[n], -1, st));          // x_+
    EGT_TRY(grad32(G, 1, G->x[n], G->gy[n], st));                          // A^T x_+
    // y_tilde = y_{(1-tau) mu_y}(x_+), y_+; value = -f_{mu_y+}(x_+)
    EGT_TRY(sbr(G, 1, G->gy[n], (1 - tau) * my, G->y[c], tau, G->y[n], 3, st));
    EGT_TRY(grad32(G, 0, G->y[n], G->gx[n], st));                          // A y_+
    if (want_egv) EGT_TRY(sbr(G, 0, G->gx[n], mx, nullptr, 0, nullptr, 2, st));   // phi_mu_x(y_+)
  }
  return EGT_OK;
}

egt_status do_step(egt_game* G, int player, double* tau_io, int mode, egt_step_info* info,
                   cudaStream_t st) {
  if (!G->initialised) return fail(EGT_ERR_INVALID_ARG, "egt_solver_init has not been called");
  if (!tau_io || !(*tau_io > 0) || !(*tau_io < 1)) return fail(EGT_ERR_INVALID_ARG, "tau must be in (0, 1)");
  if (mode < 0 || mode > 2) return fail(EGT_ERR_INVALID_ARG, "unknown step mode");
  const int me = player < 0 ? (G->mu[0] > G->mu[1] ? 0 : 1) : player;
  if (me != 0 && me != 1) return fail(EGT_ERR_INVALID_ARG, "player must be -1, 0 or 1");
  const long long p0 = G->products;
  double tau = *tau_io, egv = NAN;
  int backoffs = 0;
  bool accepted = true;
  for (;;) {
    EGT_TRY(step_once(G, me, tau, mode != EGT_STEP_PLAIN, st));
    if (mode == EGT_STEP_PLAIN) break;
    EGT_TRY(read_vals(G, 2, 2, st));
    egv = G->pinned[2] + G->pinned[3];
    if (egv >= 0) break;
    if (mode == EGT_STEP_CHECK) {
      accepted = false;
      break;
    }
    tau *= 0.5;
    ++backoffs;
    if (tau < kTauMin) return fail(EGT_ERR_TAU_UNDERFLOW, "Decr halved tau below 2^-30");
  }
  G->vhat_player = me;
  if (accepted) {
    G->mu[me] *= (1.0 - tau);
    G->cur = 1 - G->cur;
    G->t += 1;
    if (mode == EGT_STEP_DECR) G->tau = tau;
  }
  *tau_io = tau;
  if (info) {
    info->player = me;
    info->accepted = accepted ? 1 : 0;
    info->backoffs = backoffs;
    info->products = (int32_t)(G->products - p0);
    info->tau = tau;
    info->egv = egv;
    info->mu[0] = G->mu[0];
    info->mu[1] = G->mu[1];
  }
  return EGT_OK;
}

egt_status solver_init(egt_game* G, const egt_solve_opts* o, cudaStream_t st) {
  if (!o) return fail(EGT_ERR_INVALID_ARG, "opts is NULL");
  if (o->variant < 0 || o->variant > 2) return fail(EGT_ERR_INVALID_ARG, "unknown variant");
  const double theory = G->normA * std::sqrt(G->M[0] * G->M[1]);
  const bool given = o->mu0[0] > 0 && o->mu0[1] > 0;
  if (given) {
    G->mu[0] = o->mu0[0];
    G->mu[1] = o->mu0[1];
  } else if (o->variant == EGT_THEORY) {
    G->mu[0] = G->mu[1] = theory;
  } else {
    if (!(o->alpha > 0)) return fail(EGT_ERR_INVALID_ARG, "alpha must be > 0");
    G->mu[0] = G->mu[1] = o->alpha * theory;
  }
  if (!(G->mu[0] > 0) || !(G->mu[1] > 0) || !std::isfinite(G->mu[0]) || !std::isfinite(G->mu[1]))
    return fail(EGT_ERR_INVALID_ARG, "initial mu must be finite and > 0");
  G->cur = 0;
  EGT_TRY(init_point(G, st));
  if (!given && o->variant != EGT_THEORY) {
    for (int k = 0;; ++k) {
      double egv;
      EGT_TRY(current_egv(G, &egv, st));
      if (egv >= 0) break;
      if (k > 200) return fail(EGT_ERR_NUMERIC, "initial mu guard did not reach EGV >= 0");
      G->mu[0] *= 2;
      G->mu[1] *= 2;
      EGT_TRY(init_point(G, st));
    }
  }
  G->t = 0;
  G->tau = 0.5;
  G->last_gap = NAN;
  G->initialised = true;
  return EGT_OK;
}

// Grid of the device-resident driver for this game (0: not available here).
int engine_grid(egt_game* G) {
  if (G->eng_grid == -2) {
    const int maxg = engine_max_grid(engine_smem_bytes(G->dg), false);
    G->eng_grid = maxg <= 0 ? 0 : std::min(maxg, engine_items(G->dg));
  }
  return G->eng_grid;
}

}  // namespace

namespace egtapi {

// The game's buffers as the device-resident driver sees them.
EngineBufs engine_bufs(const egt_game* G, egt_iter_log* log_dev, int log_cap) {
  EngineBufs b{};
  G->vhat_player = -1;           // the driver reuses the Step scratch
  for (int i = 0; i < 2; ++i) {
    b.x[i] = G->x[i];
    b.y[i] = G->y[i];
    b.gx[i] = G->gx[i];
    b.gy[i] = G->gy[i];
    b.g64[i] = G->g64[i];
  }
  b.tx = G->tx;
  b.ty = G->ty;
  b.partials = G->eng_partials;
  b.log = log_dev;
  b.log_cap = log_cap;
  return b;
}

// Control block of a launch of n iterations from the game's solver state.
void engine_ctl_init(const egt_game* G, EngineCtl& c, int variant, double eps_mbb, int gap_every, int n) {
  std::memset(&c, 0, sizeof(c));
  c.variant = variant;
  c.n_iters = n;
  c.gap_every = std::max(1, gap_every);
  c.max_t = G->t + n;
  c.trace = G->prof_on ? 1 : 0;
  c.eps_mbb = eps_mbb;
  c.mbb_scale = 1000.0 / G->bb;
  c.mu[0] = G->mu[0];
  c.mu[1] = G->mu[1];
  c.tau = G->tau;
  c.cur = G->cur;
  c.t = G->t;
  c.gap_mbb = G->last_gap;
  c.egv = c.last_tau = c.last_egv = NAN;
}

// The game's solver state after a launch (from its control block).
void engine_ctl_apply(egt_game* G, const EngineCtl& c, egt_solve_report* rep) {
  G->mu[0] = c.mu[0];
  G->mu[1] = c.mu[1];
  G->cur = c.cur;
  G->t = c.t;
  G->tau = c.tau;
  G->last_gap = c.gap_mbb;
  G->products += c.products;
  for (int k = 0; k < kEnginePhases; ++k) {
    G->eng_phase_ns[k] += (double)c.phase_ns[k];
    G->eng_phase_work_ns[k] += (double)c.phase_work_ns[k];
    G->eng_phase_n[k] += (long long)c.phase_n[k];
  }
  if (rep) {
    rep->iters = c.done_iters;
    rep->products = c.products;
    rep->backoffs = c.backoffs;
    rep->gap_checks = c.gap_checks;
    rep->gap_mbb = c.gap_mbb;
    rep->mu[0] = c.mu[0];
    rep->mu[1] = c.mu[1];
    rep->tau = c.tau;
  }
}

}  // namespace egtapi

namespace {

egt_status engine_status(const EngineCtl& c) {
  if (c.status == EGT_ERR_TIMEOUT)
    return fail(EGT_ERR_TIMEOUT, "a group barrier of the device-resident driver ran out of time; "
                                 "the solver state is undefined until egt_solver_init");
  if (c.status == EGT_ERR_TAU_UNDERFLOW) return fail(EGT_ERR_TAU_UNDERFLOW, "Decr halved tau below 2^-30");
  if (c.status != 0) return fail((egt_status)c.status, "non-finite value in the device-resident driver");
  return EGT_OK;
}

// Items the one-game launch runs two at a time on its CTAs' warp halves: the product
// (terminal) items, when a phase has at least two terminals per CTA and shared memory
// allows two items side by side (results are the same either way: exact sums).
int engine_pair_bits(const egt_game* G, int grid) {
  const int limit = engine_smem_limit(false);
  if (limit <= 0 || 2 * grid > (int)G->comp.term.size()) return 0;
  const size_t smem = engine_smem_bytes(G->dg, kPairTerms);
  if (smem > (size_t)limit || engine_max_grid(smem, false) < grid) return 0;
  return kPairTerms;
}

// Run up to n iterations of `variant` from the solver state on the device (one
// cooperative launch), as the host loop of egt_solve would: Step (with the
// EGT/as back-off), then the residual every gap_every iterations and at the end.
egt_status engine_run(egt_game* G, int variant, double eps_mbb, int gap_every, int n,
                      egt_iter_log* log_dev, int log_cap, egt_solve_report* rep, cudaStream_t st) {
  const int grid = engine_grid(G);
  if (grid <= 0) return fail(EGT_ERR_CUDA, "the device-resident driver cannot run on this device");
  EngineCtl& c = *G->ctl_host;
  engine_ctl_init(G, c, variant, eps_mbb, gap_every, n);
  EngineJob job{};
  job.g = G->dg;
  job.b = engine_bufs(G, log_dev, log_cap);
  job.ctl = G->ctl_dev;
  job.pair = engine_pair_bits(G, grid);
  // fault-injection hooks for tests: phantom arrivals make every group barrier wait run
  // out after the time limit instead of completing
  const unsigned extra = (unsigned)std::max(0, env_int("EGT_TEST_BARRIER_EXTRA", 0));
  const unsigned long long limit_ns =
      1000000ull * (unsigned long long)std::max(1, env_int("EGT_BARRIER_TIMEOUT_MS", 2000));
  CUDA_TRY(cudaMemcpyAsync(G->ctl_dev, &c, sizeof(c), cudaMemcpyHostToDevice, st));
  cudaError_t le = cudaSuccess;
  EGT_TRY(timed(G, EGT_KERNEL_ENGINE, st, "engine kernel", [&] {
    le = engine_launch_one(job, grid, engine_smem_bytes(G->dg, job.pair), extra, limit_ns, st);
  }));
  if (le != cudaSuccess) return fail(EGT_ERR_CUDA, std::string("engine launch: ") + cudaGetErrorString(le));
  CUDA_TRY(cudaMemcpyAsync(&c, G->ctl_dev, sizeof(c), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  engine_ctl_apply(G, c, rep);
  return engine_status(c);
}

}  // namespace

namespace egt {
void set_last_error(const std::string& msg) { g_last_error = msg; }

bool game_view(const egt_game* G, GameView* out) {
  if (!G || !out) return false;
  out->dg = &G->dg;
  out->device = G->device;
  out->bb = G->bb;
  out->host_only = G->host_only;
  return true;
}
}  // namespace egt

extern "C" {

const char* egt_last_error(void) { return g_last_error.c_str(); }

egt_status egt_create_game(const egt_game_desc* desc, int32_t device, void* stream, egt_game** out) {
  Range nvtx_range("egt_create_game");
  if (!out) return fail(EGT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  EGT_TRY(validate(desc));
  const bool host_only = device == -1;
  if (!host_only) {
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(EGT_ERR_INVALID_ARG, "no such device");
  }
  DeviceGuard guard(host_only ? -1 : device);
  if (!host_only && !guard.ok) return fail(EGT_ERR_CUDA, "cudaSetDevice failed");
  egt_game* G = new (std::nothrow) egt_game();
  if (!G) return fail(EGT_ERR_OOM, "host allocation failed");
  G->device = device;
  G->host_only = host_only;
  G->H = desc->n_hands;
  G->ld = (desc->n_hands + 31) / 32 * 32;
  G->hand_size = desc->hand_size;
  G->bb = desc->bb;
  G->pot = desc->pot;
  if (G->ld > kMaxLd) {
    delete G;
    return fail(EGT_ERR_INVALID_ARG, "n_hands above 1536");
  }
  Menus menus = uniform_menus(desc->bet_fracs, desc->n_bets, desc->allin != 0);
  if (desc->menus)
    for (int p = 0; p < 2; ++p)
      for (int k = 0; k < 4; ++k) {
        const egt_menu& mu = desc->menus[4 * p + k];
        menus.m[p][k].fracs.assign(mu.fracs, mu.fracs + mu.n);
        menus.m[p][k].allin = mu.allin != 0;
        menus.m[p][k].fold = mu.fold != 0;
      }
  std::string err = compile_betting(desc->pot, desc->stack, menus, desc->raise_cap, G->comp);
  if (!err.empty()) {
    delete G;
    return fail(EGT_ERR_INVALID_ARG, err);
  }
  G->order.resize(G->H);
  std::iota(G->order.begin(), G->order.end(), 0);
  std::stable_sort(G->order.begin(), G->order.end(),
                   [&](int a, int b) { return desc->strength[a] < desc->strength[b]; });
  egt_status st = upload(G, desc, !host_only, S(stream));
  if (st == EGT_OK && !host_only) st = alloc_state(G);
  if (st == EGT_OK && !host_only) {
    int dev_smem = 0;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    const size_t room = (size_t)std::max(0, dev_smem - 1024);   // static shared memory of the kernels
    for (int p = 0; p < 2 && st == EGT_OK; ++p)
      if (sbr_smem_bytes(G->dg, p) > room || br_smem_bytes(G->dg, p) > room)
        st = fail(EGT_ERR_INVALID_ARG, "betting tree too large for the shared-memory SBR tile");
    if (st == EGT_OK && grad_smem_bytes(G->dg) > room)
      st = fail(EGT_ERR_INVALID_ARG, "hand count too large for the shared-memory gradient tile");
  }
  if (st != EGT_OK) {
    std::string keep = g_last_error;
    free_game(G);
    g_last_error = keep;
    return st;
  }
  *out = G;
  return EGT_OK;
}

egt_status egt_destroy_game(egt_game* game) {
  if (!game) return EGT_OK;
  if (!game->host_only) {
    DeviceGuard guard(game->device);
    cudaDeviceSynchronize();
    free_game(game);
  } else {
    free_game(game);
  }
  return EGT_OK;
}

egt_status egt_dims_query(const egt_game* G, egt_dims* o) {
  if (!G || !o) return fail(EGT_ERR_INVALID_ARG, "NULL argument");
  o->H = G->H;
  o->ld = G->ld;
  for (int p = 0; p < 2; ++p) {
    o->S[p] = G->comp.tpx[p].S;
    o->J[p] = G->comp.tpx[p].J;
    o->L[p] = G->comp.tpx[p].L;
    o->M[p] = G->M[p];
    o->Omega[p] = G->Omega[p];
  }
  o->T = (int32_t)G->comp.term.size();
  o->n_fold = 0;
  for (auto& t : G->comp.term) o->n_fold += t.kind == 0;
  o->Z = G->Z;
  o->normA = G->normA;
  o->table_bytes = (int64_t)G->table_bytes;
  o->device_bytes = (int64_t)G->device_bytes;
  return EGT_OK;
}

egt_status egt_hand_order(const egt_game* G, int32_t* order) {
  if (!G || !order) return fail(EGT_ERR_INVALID_ARG, "NULL argument");
  std::copy(G->order.begin(), G->order.end(), order);
  return EGT_OK;
}

egt_status egt_treeplex_query(const egt_game* G, int32_t player, int32_t* parent, int32_t* first,
                              int32_t* n_actions, int32_t* level, double* beta) {
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  EGT_TRY(check_player(player));
  const Treeplex& T = G->comp.tpx[player];
  for (int j = 0; j < T.J; ++j) {
    if (parent) parent[j] = T.inf_parent[j];
    if (first) first[j] = T.inf_first[j];
    if (n_actions) n_actions[j] = T.inf_n[j];
    if (level) level[j] = T.inf_level[j];
    if (beta) beta[j] = T.beta[j];
  }
  return EGT_OK;
}

egt_status egt_terminal_query(const egt_game* G, int32_t* seq1, int32_t* seq2, int32_t* kind, double* coef) {
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  for (size_t b = 0; b < G->comp.term.size(); ++b) {
    const Terminal& t = G->comp.term[b];
    if (seq1) seq1[b] = t.seq[0];
    if (seq2) seq2[b] = t.seq[1];
    if (kind) kind[b] = t.kind;
    if (coef) coef[b] = t.coef;
  }
  return EGT_OK;
}

egt_status egt_grad(egt_game* G, int32_t player, const float* in, float* out, void* stream) {
  Range nvtx_range("egt_grad");
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (G->host_only) return fail(EGT_ERR_INVALID_ARG, "host-only game (device -1) has no device state");
  EGT_TRY(check_player(player));
  EGT_TRY(check_ptr(in, "in"));
  EGT_TRY(check_ptr(out, "out"));
  if (in == out) return fail(EGT_ERR_INVALID_ARG, "in and out must differ");
  DeviceGuard guard(G->device);
  cudaStream_t st = S(stream);
  float* c = reinterpret_cast<float*>(G->pub);
  EGT_TRY(grad32(G, player, in, c, st));
  return timed(G, EGT_KERNEL_GRAD_F32, st, "combine kernel",
               [&] { launch_combine<float>(G->dg, player, c, out, st); });
}

egt_status egt_grad_f64(egt_game* G, int32_t player, const double* in, double* out, void* stream) {
  Range nvtx_range("egt_grad_f64");
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (G->host_only) return fail(EGT_ERR_INVALID_ARG, "host-only game (device -1) has no device state");
  EGT_TRY(check_player(player));
  EGT_TRY(check_ptr(in, "in"));
  EGT_TRY(check_ptr(out, "out"));
  if ((const void*)in == (const void*)out) return fail(EGT_ERR_INVALID_ARG, "in and out must differ");
  DeviceGuard guard(G->device);
  cudaStream_t st = S(stream);
  EGT_TRY(timed(G, EGT_KERNEL_GRAD_F64, st, "grad f64 kernel",
                [&] { launch_terms<double>(G->dg, player, in, nullptr, G->pub, st); }));
  return timed(G, EGT_KERNEL_GRAD_F64, st, "combine kernel",
               [&] { launch_combine<double>(G->dg, player, G->pub, out, st); });
}

egt_status egt_smoothed_br(egt_game* G, int32_t player, const float* g, double mu, float* q_out,
                           double* value_out, void* stream) {
  Range nvtx_range("egt_smoothed_br");
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (G->host_only) return fail(EGT_ERR_INVALID_ARG, "host-only game (device -1) has no device state");
  EGT_TRY(check_player(player));
  EGT_TRY(check_ptr(g, "g"));
  if (q_out) EGT_TRY(check_ptr(q_out, "q_out"));
  if (!(mu > 0) || !std::isfinite(mu)) return fail(EGT_ERR_INVALID_ARG, "mu must be finite and > 0");
  DeviceGuard guard(G->device);
  EGT_TRY(sbr(G, player, g, mu, nullptr, 0, q_out, value_out ? 4 : -1, S(stream), true));
  if (value_out) {
    EGT_TRY(read_vals(G, 4, 1, S(stream)));
    // player 1's kernel solved min <y, -g> + mu d(y); its own maximum is the negation
    *value_out = player == 0 ? G->pinned[4] : -G->pinned[4];
  }
  return EGT_OK;
}

egt_status egt_best_response_f64(egt_game* G, int32_t player, const double* g, double* value_out,
                                 void* stream) {
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (G->host_only) return fail(EGT_ERR_INVALID_ARG, "host-only game (device -1) has no device state");
  EGT_TRY(check_player(player));
  EGT_TRY(check_ptr(g, "g"));
  if (!value_out) return fail(EGT_ERR_INVALID_ARG, "value_out is NULL");
  DeviceGuard guard(G->device);
  cudaStream_t st = S(stream);
  EGT_TRY(timed(G, EGT_KERNEL_BR_F64, st, "br kernel", [&] {
    launch_br64(G->dg, player, g, false, player == 0 ? 1.0 : -1.0, G->vals + 10, G->partials, G->counter, st);
  }));
  CUDA_TRY(cudaMemcpyAsync(G->pinned + 10, G->vals + 10, sizeof(double), cudaMemcpyDeviceToHost, S(stream)));
  CUDA_TRY(cudaStreamSynchronize(S(stream)));
  *value_out = G->pinned[10];
  return EGT_OK;
}

egt_status egt_gap(egt_game* G, const float* x, const float* y, double* gap_mbb, void* stream) {
  Range nvtx_range("egt_gap");
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (G->host_only) return fail(EGT_ERR_INVALID_ARG, "host-only game (device -1) has no device state");
  EGT_TRY(check_ptr(x, "x"));
  EGT_TRY(check_ptr(y, "y"));
  if (!gap_mbb) return fail(EGT_ERR_INVALID_ARG, "gap_mbb is NULL");
  DeviceGuard guard(G->device);
  return gap_internal(G, x, y, gap_mbb, S(stream));
}

egt_status egt_solver_init(egt_game* G, const egt_solve_opts* opts, void* stream) {
  Range nvtx_range("egt_solver_init");
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (G->host_only) return fail(EGT_ERR_INVALID_ARG, "host-only game (device -1) has no device state");
  DeviceGuard guard(G->device);
  return solver_init(G, opts, S(stream));
}

egt_status egt_step(egt_game* G, int32_t player, double* tau_inout, int32_t mode, egt_step_info* info,
                    void* stream) {
  Range nvtx_range("egt_step");
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (G->host_only) return fail(EGT_ERR_INVALID_ARG, "host-only game (device -1) has no device state");
  DeviceGuard guard(G->device);
  return do_step(G, player, tau_inout, mode, info, S(stream));
}

egt_status egt_step_point(egt_game* G, float* v_hat, int32_t* player, void* stream) {
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (G->host_only) return fail(EGT_ERR_INVALID_ARG, "host-only game (device -1) has no device state");
  if (!player) return fail(EGT_ERR_INVALID_ARG, "player is NULL");
  EGT_TRY(check_ptr(v_hat, "v_hat"));
  const int me = G->vhat_player;
  if (me != 0 && me != 1) return fail(EGT_ERR_INVALID_ARG, "no egt_step since the scratch was last reused");
  DeviceGuard guard(G->device);
  CUDA_TRY(cudaMemcpyAsync(v_hat, me == 0 ? G->tx : G->ty, vec_elems(G, me) * 4, cudaMemcpyDeviceToDevice,
                           S(stream)));
  *player = me;
  return EGT_OK;
}

egt_status egt_state_get(egt_game* G, float* x, float* y, double* mu, void* stream) {
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (G->host_only) return fail(EGT_ERR_INVALID_ARG, "host-only game (device -1) has no device state");
  if (!G->initialised) return fail(EGT_ERR_INVALID_ARG, "egt_solver_init has not been called");
  DeviceGuard guard(G->device);
  const int c = G->cur;
  if (x) CUDA_TRY(cudaMemcpyAsync(x, G->x[c], vec_elems(G, 0) * 4, cudaMemcpyDeviceToDevice, S(stream)));
  if (y) CUDA_TRY(cudaMemcpyAsync(y, G->y[c], vec_elems(G, 1) * 4, cudaMemcpyDeviceToDevice, S(stream)));
  if (mu) {
    mu[0] = G->mu[0];
    mu[1] = G->mu[1];
  }
  return EGT_OK;
}

egt_status egt_state_set(egt_game* G, const float* x, const float* y, const double* mu, void* stream) {
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (G->host_only) return fail(EGT_ERR_INVALID_ARG, "host-only game (device -1) has no device state");
  EGT_TRY(check_ptr(x, "x"));
  EGT_TRY(check_ptr(y, "y"));
  if (!mu || !(mu[0] > 0) || !(mu[1] > 0)) return fail(EGT_ERR_INVALID_ARG, "mu must be > 0");
  DeviceGuard guard(G->device);
  const int c = G->cur;
  cudaStream_t st = S(stream);
  CUDA_TRY(cudaMemcpyAsync(G->x[c], x, vec_elems(G, 0) * 4, cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(G->y[c], y, vec_elems(G, 1) * 4, cudaMemcpyDeviceToDevice, st));
  G->mu[0] = mu[0];
  G->mu[1] = mu[1];
  G->vhat_player = -1;
  EGT_TRY(grad32(G, 0, G->y[c], G->gx[c], st));
  EGT_TRY(grad32(G, 1, G->x[c], G->gy[c], st));
  G->initialised = true;
  return EGT_OK;
}

egt_status egt_checkpoint_get(egt_game* G, float* x, float* y, egt_checkpoint* ck, void* stream) {
  if (!ck) return fail(EGT_ERR_INVALID_ARG, "ck is NULL");
  EGT_TRY(egt_state_get(G, x, y, ck->mu, stream));
  ck->t = G->t;
  ck->tau = G->tau;
  ck->gap_mbb = G->last_gap;
  return EGT_OK;
}

egt_status egt_checkpoint_set(egt_game* G, const float* x, const float* y, const egt_checkpoint* ck,
                              void* stream) {
  if (!ck) return fail(EGT_ERR_INVALID_ARG, "ck is NULL");
  if (ck->t < 0) return fail(EGT_ERR_INVALID_ARG, "t must be >= 0");
  if (!(ck->tau > 0 && ck->tau <= 1)) return fail(EGT_ERR_INVALID_ARG, "tau must be in (0, 1]");
  EGT_TRY(egt_state_set(G, x, y, ck->mu, stream));
  G->t = ck->t;
  G->tau = ck->tau;
  G->last_gap = ck->gap_mbb;
  return EGT_OK;
}

egt_status egt_state_gap(egt_game* G, double* gap_mbb, void* stream) {
  Range nvtx_range("egt_state_gap");
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (G->host_only) return fail(EGT_ERR_INVALID_ARG, "host-only game (device -1) has no device state");
  if (!G->initialised) return fail(EGT_ERR_INVALID_ARG, "egt_solver_init has not been called");
  if (!gap_mbb) return fail(EGT_ERR_INVALID_ARG, "gap_mbb is NULL");
  DeviceGuard guard(G->device);
  return gap_internal(G, G->x[G->cur], G->y[G->cur], gap_mbb, S(stream));
}

egt_status egt_iterate(egt_game* G, const egt_solve_opts* o, int32_t n_iters, egt_solve_report* rep,
                       void* stream) {
  Range nvtx_range("egt_iterate");
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (G->host_only) return fail(EGT_ERR_INVALID_ARG, "host-only game (device -1) has no device state");
  if (!G->initialised) return fail(EGT_ERR_INVALID_ARG, "egt_solver_init has not been called");
  if (!o) return fail(EGT_ERR_INVALID_ARG, "opts is NULL");
  if (o->variant < 0 || o->variant > 2) return fail(EGT_ERR_INVALID_ARG, "unknown variant");
  if (o->replay_n > 0) return fail(EGT_ERR_INVALID_ARG, "replay schedules run on the host-driven loop (egt_solve)");
  if (n_iters < 0) return fail(EGT_ERR_INVALID_ARG, "n_iters < 0");
  DeviceGuard guard(G->device);
  const auto t0 = std::chrono::steady_clock::now();
  egt_solve_report r{};
  r.gap_mbb = G->last_gap;
  r.mu[0] = G->mu[0];
  r.mu[1] = G->mu[1];
  r.tau = G->tau;
  if (n_iters > 0) EGT_TRY(engine_run(G, o->variant, o->eps_mbb, o->gap_every, n_iters, nullptr, 0, &r, S(stream)));
  if (rep) {
    *rep = r;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return EGT_OK;
}

egt_status egt_solve(egt_game* G, const egt_solve_opts* o, float* x_out, float* y_out,
                     egt_solve_report* rep, void* stream) {
  Range nvtx_range("egt_solve");
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (G->host_only) return fail(EGT_ERR_INVALID_ARG, "host-only game (device -1) has no device state");
  if (!o) return fail(EGT_ERR_INVALID_ARG, "opts is NULL");
  if (o->max_iters < 0) return fail(EGT_ERR_INVALID_ARG, "max_iters < 0");
  if (o->replay_n > 0 && (!o->replay_player || !o->replay_tau))
    return fail(EGT_ERR_INVALID_ARG, "replay arrays are NULL");
  if (x_out) EGT_TRY(check_ptr(x_out, "x_out"));
  if (y_out) EGT_TRY(check_ptr(y_out, "y_out"));
  DeviceGuard guard(G->device);
  cudaStream_t st = S(stream);
  const auto t0 = std::chrono::steady_clock::now();
  G->products = 0;
  EGT_TRY(solver_init(G, o, st));
  const int gap_every = std::max(1, o->gap_every);
  if (o->engine == EGT_ENGINE_DEVICE && o->replay_n <= 0 && engine_grid(G) > 0) {
    // residual at t = 0 (the loop test of Alg. 1 / 3), then the iterations on the device
    double gap = INFINITY;
    EGT_TRY(gap_internal(G, G->x[G->cur], G->y[G->cur], &gap, st));
    G->last_gap = gap;
    egt_solve_report r{};
    r.gap_mbb = gap;
    r.mu[0] = G->mu[0];
    r.mu[1] = G->mu[1];
    r.tau = G->tau;
    const bool done = (o->eps_mbb > 0 && gap <= o->eps_mbb) || o->max_iters == 0;
    egt_iter_log* dlog = nullptr;
    const int log_n = (o->log && o->log_cap > 0) ? std::min(o->log_cap, o->max_iters) : 0;
    if (log_n > 0) CUDA_TRY(cudaMalloc(&dlog, (size_t)log_n * sizeof(egt_iter_log)));
    egt_status es = EGT_OK;
    if (!done) es = engine_run(G, o->variant, o->eps_mbb, gap_every, o->max_iters, dlog, log_n, &r, st);
    if (dlog) {
      if (es == EGT_OK) {
        const int n = std::min(log_n, r.iters);
        cudaMemcpyAsync(o->log, dlog, (size_t)n * sizeof(egt_iter_log), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
      }
      cudaFree(dlog);
    }
    if (es != EGT_OK) return es;
    if (x_out) CUDA_TRY(cudaMemcpyAsync(x_out, G->x[G->cur], vec_elems(G, 0) * 4, cudaMemcpyDeviceToDevice, st));
    if (y_out) CUDA_TRY(cudaMemcpyAsync(y_out, G->y[G->cur], vec_elems(G, 1) * 4, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (rep) {
      *rep = r;
      rep->products = (int32_t)G->products;
      rep->gap_checks = r.gap_checks + 1;
      rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (o->eps_mbb > 0 && !(r.gap_mbb <= o->eps_mbb))
      return fail(EGT_ERR_NOT_CONVERGED, "gap target not reached within max_iters");
    return EGT_OK;
  }
  int t = 0, backoffs = 0, gap_checks = 0;
  double tau = 0.5, gap = INFINITY;
  for (;;) {
    if (t % gap_every == 0 || t >= o->max_iters) {
      EGT_TRY(gap_internal(G, G->x[G->cur], G->y[G->cur], &gap, st));
      ++gap_checks;
    }
    if ((o->eps_mbb > 0 && gap <= o->eps_mbb) || t >= o->max_iters || (o->replay_n > 0 && t >= o->replay_n))
      break;
    egt_step_info info{};
    if (o->replay_n > 0) {
      double tt = o->replay_tau[t];
      EGT_TRY(do_step(G, o->replay_player[t], &tt, EGT_STEP_PLAIN, &info, st));
    } else if (o->variant == EGT_THEORY) {
      double tt = 2.0 / (t + 3);
      EGT_TRY(do_step(G, t % 2 == 0 ? 0 : 1, &tt, EGT_STEP_PLAIN, &info, st));
    } else if (o->variant == EGT_PRACTICAL) {
      double tt = 2.0 / (t + 3);
      EGT_TRY(do_step(G, -1, &tt, EGT_STEP_PLAIN, &info, st));
    } else {
      EGT_TRY(do_step(G, -1, &tau, EGT_STEP_DECR, &info, st));
      backoffs += info.backoffs;
    }
    if (o->log && t < o->log_cap) {
      egt_iter_log& L = o->log[t];
      L.t = t;
      L.player = info.player;
      L.backoffs = info.backoffs;
      L.tau = info.tau;
      L.mu[0] = G->mu[0];
      L.mu[1] = G->mu[1];
      L.egv = info.egv;
      L.gap_mbb = gap;
      L.time_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                      std::chrono::steady_clock::now().time_since_epoch()).count();
    }
    ++t;
  }
  if (x_out) CUDA_TRY(cudaMemcpyAsync(x_out, G->x[G->cur], vec_elems(G, 0) * 4, cudaMemcpyDeviceToDevice, st));
  if (y_out) CUDA_TRY(cudaMemcpyAsync(y_out, G->y[G->cur], vec_elems(G, 1) * 4, cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (rep) {
    rep->iters = t;
    rep->products = (int32_t)G->products;
    rep->backoffs = backoffs;
    rep->gap_checks = gap_checks;
    rep->gap_mbb = gap;
    rep->mu[0] = G->mu[0];
    rep->mu[1] = G->mu[1];
    rep->tau = tau;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (o->eps_mbb > 0 && !(gap <= o->eps_mbb))
    return fail(EGT_ERR_NOT_CONVERGED, "gap target not reached within max_iters");
  return EGT_OK;
}

egt_status egt_profile(egt_game* G, int32_t enable) {
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (G->host_only) return fail(EGT_ERR_INVALID_ARG, "host-only game (device -1) has no device state");
  DeviceGuard guard(G->device);
  EGT_TRY(prof_drain(G));
  for (int k = 0; k < EGT_KERNEL_KINDS; ++k) {
    if (enable) {
      G->prof_ms[k] = 0;
      G->prof_n[k] = 0;
    }
    G->launches[k] = 0;
  }
  G->prof_on = enable != 0;
  return EGT_OK;
}

egt_status egt_engine_trace(egt_game* G, int32_t reset, double* phase_us, double* work_us,
                            int64_t* phase_count) {
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  for (int k = 0; k < kEnginePhases; ++k) {
    if (phase_us) phase_us[k] = G->eng_phase_ns[k] * 1e-3;
    if (work_us) work_us[k] = G->eng_phase_work_ns[k] * 1e-3;
    if (phase_count) phase_count[k] = G->eng_phase_n[k];
    if (reset) {
      G->eng_phase_ns[k] = 0;
      G->eng_phase_work_ns[k] = 0;
      G->eng_phase_n[k] = 0;
    }
  }
  return EGT_OK;
}

egt_status egt_profile_read(egt_game* G, double* ms, int64_t* launches) {
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (G->host_only) return fail(EGT_ERR_INVALID_ARG, "host-only game (device -1) has no device state");
  DeviceGuard guard(G->device);
  EGT_TRY(prof_drain(G));
  for (int k = 0; k < EGT_KERNEL_KINDS; ++k) {
    if (ms) ms[k] = G->prof_ms[k];
    if (launches) launches[k] = G->launches[k];
  }
  return EGT_OK;
}
}  // extern "C"
