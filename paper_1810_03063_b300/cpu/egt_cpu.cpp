// libegt_cpu: FP64 multi-core CPU EGT/as on the structured products (include/egt_cpu.h).
//
// Layout: vectors [seq][hand] with hands in ascending strength (ties by input
// index), H columns, no padding.  Per terminal e of player p's grouping (its
// own sequence sigma_p(e)) the product adds to row sigma_p(e):
//
//   r_p(h) / Z * coef_e * S_e(h),   S_e(h) over the opponent column v = in[sigma_opp(e)],
//   w = r_opp (.) v:
//   fold:     S = W - W_card[a] - W_card[b] + w(h)          (cards a, b of h; hand-vs-hand
//                                                           disjointness by inclusion-exclusion)
//   showdown: S = sum_{disjoint, stronger} w - sum_{disjoint, weaker} w
//           = (W - P[hi] - (Wc_a - Pc_a[hi]) - (Wc_b - Pc_b[hi]))
//             - (P[lo] - Pc_a[lo] - Pc_b[lo])
//
// with P the exclusive prefix over the strength order, [lo, hi) h's tie group
// and Pc_c the exclusive prefix over the hands holding card c (Sec. 7 payoffs:
// the stronger hand wins the stake, ties pay nothing).  Sums are plain FP64.
#include "../../include/egt_cpu.h"

#include <omp.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <limits>
#include <numeric>
#include <string>
#include <vector>

#include "../csrc/tree.hpp"

namespace {

thread_local std::string g_err;

egt_status fail(egt_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

using Vec = std::vector<double>;

}  // namespace

struct egt_cpu_game {
  int H = 0, k = 2, n_slots = 0;
  double Z = 0, normA = 0, bb = 1, M[2] = {0, 0};
  egt::Compiled C;
  std::vector<int> order;                 // sorted position -> input index
  std::vector<int> card[2];               // [H] card slot of each hand (second: empty slot for 1-card hands)
  std::vector<int> lo, hi;                // [H] tie group [lo, hi)
  std::vector<int> cnt_lo[2], cnt_hi[2];  // [H] hands of card[i] sorted before lo / hi
  std::vector<std::vector<int>> lists;    // per card slot: sorted positions of the hands holding it
  Vec r[2], rz[2];                        // [H] normalised ranges, r / Z
  // terminals grouped by each player's own sequence
  std::vector<int> tptr[2], topp[2], tkind[2];
  Vec tcoef[2];
  // per player: simplexes in bottom-up order
  std::vector<int> up[2];
};

namespace {

// exclusive prefix sums of w over the strength order and over each card's hands
struct Sums {
  Vec P;                       // [H + 1]
  std::vector<Vec> Pc;         // per card slot [len + 1]
};

void column_sums(const egt_cpu_game& G, const double* w, Sums& s) {
  s.P.resize(G.H + 1);
  double run = 0;
  for (int h = 0; h < G.H; ++h) {
    s.P[h] = run;
    run += w[h];
  }
  s.P[G.H] = run;
  s.Pc.resize(G.n_slots);
  for (int c = 0; c < G.n_slots; ++c) {
    const auto& l = G.lists[c];
    s.Pc[c].resize(l.size() + 1);
    double rc = 0;
    for (size_t i = 0; i < l.size(); ++i) {
      s.Pc[c][i] = rc;
      rc += w[l[i]];
    }
    s.Pc[c][l.size()] = rc;
  }
}

// out[s][h] for player p (0: A y with in = y, 1: A^T x with in = x), rows [S_p][H]
void product(const egt_cpu_game& G, int p, const Vec& in, Vec& out, std::vector<Vec>& contrib) {
  const int H = G.H, T = (int)G.topp[p].size(), opp = 1 - p;
  const int S = G.C.tpx[p].S;
  contrib.resize(T);
#pragma omp parallel
  {
    Vec w(H);
    Sums s;
#pragma omp for schedule(dynamic, 1)
    for (int e = 0; e < T; ++e) {
      const double* v = in.data() + (size_t)G.topp[p][e] * H;
      for (int h = 0; h < H; ++h) w[h] = G.r[opp][h] * v[h];
      column_sums(G, w.data(), s);
      Vec& c = contrib[e];
      c.resize(H);
      const double W = s.P[H];
      for (int h = 0; h < H; ++h) {
        const int ca = G.card[0][h], cb = G.card[1][h];
        const Vec& Pa = s.Pc[ca];
        const Vec& Pb = s.Pc[cb];
        const double Wa = Pa.back(), Wb = Pb.back();
        double val;
        if (G.tkind[p][e] == 0) {
          val = W - Wa - Wb + (G.k == 2 ? w[h] : 0.0);
        } else {
          const double lt = s.P[G.lo[h]] - Pa[G.cnt_lo[0][h]] - Pb[G.cnt_lo[1][h]];
          const double gt = (W - s.P[G.hi[h]]) - (Wa - Pa[G.cnt_hi[0][h]]) - (Wb - Pb[G.cnt_hi[1][h]]);
          val = gt - lt;
        }
        c[h] = G.tcoef[p][e] * val;
      }
    }
    // rows: the sequence's terminals in order, times r / Z
#pragma omp for schedule(static)
    for (int q = 0; q < S; ++q) {
      double* o = out.data() + (size_t)q * H;
      for (int h = 0; h < H; ++h) o[h] = 0;
      for (int e = G.tptr[p][q]; e < G.tptr[p][q + 1]; ++e)
        for (int h = 0; h < H; ++h) o[h] += contrib[e][h];
      for (int h = 0; h < H; ++h) o[h] *= G.rz[p][h];
    }
  }
}

// Smoothed best response of player p: argmin <q, loss> + mu d(q) over the treeplex of
// every hand (Sec. 5 recursion, the value propagated from the largest q_bar), q into
// q_out (may be NULL), the value summed over hands returned.  mu = 0: plain best
// response (min instead of the soft min).
double sbr(const egt_cpu_game& G, int p, const Vec& loss, double mu, Vec* q_out) {
  const egt::Treeplex& T = G.C.tpx[p];
  const int H = G.H, J = T.J, S = T.S;
  std::vector<double> per_hand(H);
  if (q_out) q_out->assign((size_t)S * H, 0.0);
#pragma omp parallel
  {
    std::vector<double> V(J), qbar(S), gh(64), q(S);
#pragma omp for schedule(static)
    for (int h = 0; h < H; ++h) {
      for (int j : G.up[p]) {
        const int f = T.inf_first[j], n = T.inf_n[j];
        if ((int)gh.size() < n) gh.resize(n);
        double m = std::numeric_limits<double>::infinity();
        int im = 0;
        for (int i = 0; i < n; ++i) {
          const int sq = f + i;
          double v = loss[(size_t)sq * H + h];
          for (int c = T.child_ptr[sq]; c < T.child_ptr[sq + 1]; ++c) v += V[T.child_idx[c]];
          gh[i] = v;
          if (v < m) {
            m = v;
            im = i;
          }
        }
        if (mu == 0) {
          V[j] = m;
          for (int i = 0; i < n; ++i) qbar[f + i] = i == im ? 1.0 : 0.0;
          continue;
        }
        const double t = mu * T.beta[j];
        double z = 0;
        for (int i = 0; i < n; ++i) {
          const double e = std::exp(-(gh[i] - m) / t);
          qbar[f + i] = e;
          z += e;
        }
        for (int i = 0; i < n; ++i) qbar[f + i] /= z;
        V[j] = m - t * std::log(z) + t * std::log((double)n);
      }
      double vh = 0;
      for (int j = 0; j < J; ++j)
        if (T.inf_parent[j] < 0) vh += V[j];
      per_hand[h] = vh;
      if (q_out) {
        // top-down: simplexes in reverse bottom-up order
        for (auto it = G.up[p].rbegin(); it != G.up[p].rend(); ++it) {
          const int j = *it, f = T.inf_first[j], n = T.inf_n[j];
          const double qp = T.inf_parent[j] < 0 ? 1.0 : q[T.inf_parent[j]];
          for (int i = 0; i < n; ++i) q[f + i] = qp * qbar[f + i];
        }
        for (int sq = 0; sq < S; ++sq) (*q_out)[(size_t)sq * H + h] = q[sq];
      }
    }
  }
  double total = 0;   // summed in hand order: the same bits for any thread count
  for (int h = 0; h < H; ++h) total += per_hand[h];
  return total;
}

void mix(Vec& out, const Vec& a, const Vec& b, double tau) {
  out.resize(a.size());
  for (size_t i = 0; i < a.size(); ++i) out[i] = (1.0 - tau) * a[i] + tau * b[i];
}

void negate(Vec& v) {
  for (auto& x : v) x = -x;
}

}  // namespace

extern "C" {

const char* egt_cpu_last_error(void) { return g_err.c_str(); }

egt_status egt_cpu_create(const egt_game_desc* d, egt_cpu_game** out) {
  if (!out) return fail(EGT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!d) return fail(EGT_ERR_INVALID_ARG, "desc is NULL");
  if (d->hand_size != 1 && d->hand_size != 2) return fail(EGT_ERR_INVALID_ARG, "hand_size must be 1 or 2");
  if (d->n_hands < 1 || d->n_cards < 1 || !d->hand_cards || !d->strength || !d->range[0] || !d->range[1])
    return fail(EGT_ERR_INVALID_ARG, "bad hands / cards / strength / ranges");
  if (!(d->pot > 0) || !(d->stack >= 0) || !(d->bb > 0)) return fail(EGT_ERR_INVALID_ARG, "bad pot / stack / bb");
  auto* G = new egt_cpu_game();
  const int H = d->n_hands, k = d->hand_size;
  G->H = H;
  G->k = k;
  G->bb = d->bb;
  for (int h = 0; h < H; ++h)
    for (int c = 0; c < k; ++c)
      if (d->hand_cards[h * k + c] < 0 || d->hand_cards[h * k + c] >= d->n_cards) {
        delete G;
        return fail(EGT_ERR_INVALID_ARG, "card id out of range");
      }
  egt::Menus menus = egt::uniform_menus(d->bet_fracs, d->n_bets, d->allin != 0);
  if (d->menus)
    for (int p = 0; p < 2; ++p)
      for (int q = 0; q < 4; ++q) {
        const egt_menu& mu = d->menus[4 * p + q];
        menus.m[p][q].fracs.assign(mu.fracs, mu.fracs + mu.n);
        menus.m[p][q].allin = mu.allin != 0;
        menus.m[p][q].fold = mu.fold != 0;
      }
  const std::string err = egt::compile_betting(d->pot, d->stack, menus, d->raise_cap, G->C);
  if (!err.empty()) {
    delete G;
    return fail(EGT_ERR_INVALID_ARG, err);
  }
  // hands in ascending strength, ties by input index
  G->order.resize(H);
  std::iota(G->order.begin(), G->order.end(), 0);
  std::stable_sort(G->order.begin(), G->order.end(), [&](int a, int b) { return d->strength[a] < d->strength[b]; });
  // card slots: live cards, plus one empty slot for 1-card hands
  std::vector<int> slot(d->n_cards, -1);
  for (int h = 0; h < H; ++h)
    for (int c = 0; c < k; ++c) slot[d->hand_cards[h * k + c]] = 0;
  int ns = 0;
  for (int c = 0; c < d->n_cards; ++c)
    if (slot[c] == 0) slot[c] = ns++;
  G->n_slots = ns + 1;
  G->lists.assign(G->n_slots, {});
  for (int i = 0; i < 2; ++i) G->card[i].resize(H);
  for (int s = 0; s < H; ++s) {
    const int h = G->order[s];
    G->card[0][s] = slot[d->hand_cards[h * k]];
    G->card[1][s] = k == 2 ? slot[d->hand_cards[h * k + 1]] : ns;
    G->lists[G->card[0][s]].push_back(s);
    if (k == 2) G->lists[G->card[1][s]].push_back(s);
  }
  G->lo.resize(H);
  G->hi.resize(H);
  for (int s = 0; s < H;) {
    int e = s;
    while (e < H && d->strength[G->order[e]] == d->strength[G->order[s]]) ++e;
    for (int i = s; i < e; ++i) {
      G->lo[i] = s;
      G->hi[i] = e;
    }
    s = e;
  }
  for (int i = 0; i < 2; ++i) {
    G->cnt_lo[i].resize(H);
    G->cnt_hi[i].resize(H);
    for (int s = 0; s < H; ++s) {
      const auto& l = G->lists[G->card[i][s]];
      G->cnt_lo[i][s] = (int)(std::lower_bound(l.begin(), l.end(), G->lo[s]) - l.begin());
      G->cnt_hi[i][s] = (int)(std::lower_bound(l.begin(), l.end(), G->hi[s]) - l.begin());
    }
  }
  // ranges, Z = sum over disjoint pairs of r1 r2 (brute force over pairs: O(H^2) once)
  for (int p = 0; p < 2; ++p) {
    double tot = 0;
    for (int h = 0; h < H; ++h) {
      if (!(d->range[p][h] >= 0) || !std::isfinite(d->range[p][h])) {
        delete G;
        return fail(EGT_ERR_INVALID_ARG, "range entries must be finite and >= 0");
      }
      tot += d->range[p][h];
    }
    if (!(tot > 0)) {
      delete G;
      return fail(EGT_ERR_INVALID_ARG, "a range is all zero");
    }
    G->r[p].resize(H);
    for (int s = 0; s < H; ++s) G->r[p][s] = d->range[p][G->order[s]] / tot;
  }
  double Z = 0, max_any = 0, max_diff = 0;
  for (int a = 0; a < H; ++a)
    for (int b = 0; b < H; ++b) {
      const bool share = G->card[0][a] == G->card[0][b] ||
                         (k == 2 && (G->card[0][a] == G->card[1][b] || G->card[1][a] == G->card[0][b] ||
                                     G->card[1][a] == G->card[1][b]));
      if (share) continue;
      const double w = G->r[0][a] * G->r[1][b];
      Z += w;
      max_any = std::max(max_any, w);
      if (G->lo[a] != G->lo[b]) max_diff = std::max(max_diff, w);
    }
  if (!(Z > 0)) {
    delete G;
    return fail(EGT_ERR_INVALID_ARG, "no compatible hand pair has positive probability (Z = 0)");
  }
  G->Z = Z;
  double na = 0;
  for (auto& t : G->C.term) na = std::max(na, std::fabs(t.coef) * (t.kind == 0 ? max_any : max_diff));
  G->normA = na / Z;
  for (int p = 0; p < 2; ++p) {
    G->rz[p].resize(H);
    for (int s = 0; s < H; ++s) G->rz[p][s] = G->r[p][s] / Z;
    G->M[p] = H * G->C.tpx[p].m_root;
  }
  // terminals grouped by each player's sequence; showdown sign from the output hand's view
  for (int p = 0; p < 2; ++p) {
    const int S = G->C.tpx[p].S, n = (int)G->C.term.size();
    G->tptr[p].assign(S + 1, 0);
    for (auto& t : G->C.term) G->tptr[p][t.seq[p] + 1]++;
    for (int s = 0; s < S; ++s) G->tptr[p][s + 1] += G->tptr[p][s];
    std::vector<int> fill(G->tptr[p].begin(), G->tptr[p].end() - 1);
    G->topp[p].resize(n);
    G->tkind[p].resize(n);
    G->tcoef[p].resize(n);
    for (auto& t : G->C.term) {
      const int e = fill[t.seq[p]]++;
      G->topp[p][e] = t.seq[1 - p];
      G->tkind[p][e] = t.kind;
      G->tcoef[p][e] = t.kind == 0 ? t.coef : (p == 0 ? t.coef : -t.coef);
    }
    const egt::Treeplex& T = G->C.tpx[p];
    G->up[p].resize(T.J);
    std::iota(G->up[p].begin(), G->up[p].end(), 0);
    std::stable_sort(G->up[p].begin(), G->up[p].end(),
                     [&](int a, int b) { return T.inf_level[a] > T.inf_level[b]; });
  }
  *out = G;
  return EGT_OK;
}

egt_status egt_cpu_destroy(egt_cpu_game* G) {
  delete G;
  return EGT_OK;
}

egt_status egt_cpu_dims(const egt_cpu_game* G, int32_t* S, int32_t* H) {
  if (!G) return fail(EGT_ERR_INVALID_ARG, "game is NULL");
  if (S) {
    S[0] = G->C.tpx[0].S;
    S[1] = G->C.tpx[1].S;
  }
  if (H) *H = G->H;
  return EGT_OK;
}

egt_status egt_cpu_solve(egt_cpu_game* G, const egt_cpu_opts* o, double* x_out, double* y_out,
                         egt_cpu_report* rep) {
  if (!G || !o) return fail(EGT_ERR_INVALID_ARG, "game or opts is NULL");
  if (!(o->alpha > 0) || o->max_iters < 0 || o->gap_every < 1 || o->threads < 0)
    return fail(EGT_ERR_INVALID_ARG, "alpha > 0, max_iters >= 0, gap_every >= 1, threads >= 0");
  // threads = 0: every processor (the runtime's setting may have been lowered by an
  // earlier call, or by OMP_NUM_THREADS in the environment)
  omp_set_num_threads(o->threads > 0 ? o->threads : omp_get_num_procs());
  const auto t0 = std::chrono::steady_clock::now();
  const int H = G->H;
  const int S0 = G->C.tpx[0].S, S1 = G->C.tpx[1].S;
  std::vector<Vec> contrib;
  int products = 0;
  // loss gradients: x minimises <x, A y>, y minimises <y, -A^T x>
  auto loss = [&](int p, const Vec& other, Vec& g) {
    g.assign((size_t)(p ? S1 : S0) * H, 0.0);
    product(*G, p, other, g, contrib);
    if (p == 1) negate(g);
    ++products;
  };
  const double scale = 1000.0 / G->bb;
  // eps_sad = max_y <y, A^T x> - min_x <x, A y> from the two loss gradients
  auto gap = [&](const Vec& gx, const Vec& gy) { return (-sbr(*G, 1, gy, 0, nullptr) - sbr(*G, 0, gx, 0, nullptr)) * scale; };

  // initial point (Alg. 3 first lines, the minus sign restored): y0 = y_mu_y(x_omega),
  // x0 = x_mu_x(y0); mu doubled while EGV < 0 there
  Vec zero_x((size_t)S0 * H, 0.0), x_omega, x, y, gx, gy;
  sbr(*G, 0, zero_x, 1.0, &x_omega);
  double mu0 = o->alpha * G->normA * std::sqrt(G->M[0] * G->M[1]), mu1 = mu0;
  Vec g_omega;
  loss(1, x_omega, g_omega);
  for (int k = 0;; ++k) {
    sbr(*G, 1, g_omega, mu1, &y);
    loss(0, y, gx);
    const double phi = sbr(*G, 0, gx, mu0, &x);
    loss(1, x, gy);
    const double negf = sbr(*G, 1, gy, mu1, nullptr);
    if (phi + negf >= 0) break;
    if (k > 200) return fail(EGT_ERR_NUMERIC, "initial mu guard did not reach EGV >= 0");
    mu0 *= 2;
    mu1 *= 2;
  }
  // gx = A y, gy = -A^T x: the products of the current iterates
  double tau = 0.5, g_mbb = std::numeric_limits<double>::quiet_NaN();
  int t = 0, backoffs = 0;
  egt_status status = EGT_OK;
  Vec s, vhat, go, o_q, other_p, g3, tilde, me_p, g4;
  while (t < o->max_iters) {
    const int me = mu0 > mu1 ? 0 : 1, ot = 1 - me;
    const double mu_me = me ? mu1 : mu0, mu_ot = me ? mu0 : mu1;
    Vec& v_me = me ? y : x;
    Vec& v_ot = me ? x : y;
    const Vec& g_me = me ? gy : gx;
    for (;;) {
      // Alg. 2 Step focused on me (A -> -A^T for y)
      sbr(*G, me, g_me, mu_me, &s);
      mix(vhat, v_me, s, tau);
      loss(ot, vhat, go);
      sbr(*G, ot, go, mu_ot, &o_q);
      mix(other_p, v_ot, o_q, tau);
      loss(me, other_p, g3);
      const double val_me = sbr(*G, me, g3, (1.0 - tau) * mu_me, &tilde);
      mix(me_p, v_me, tilde, tau);
      loss(ot, me_p, g4);
      const double val_ot = sbr(*G, ot, g4, mu_ot, nullptr);
      // Alg. 4: accept when the excessive gap holds at the new point, else halve tau
      if (val_me + val_ot >= 0) break;
      tau *= 0.5;
      ++backoffs;
      if (tau < 1.0 / (1u << 30)) return fail(EGT_ERR_TAU_UNDERFLOW, "Decr halved tau below 2^-30");
    }
    if (me == 0) {
      mu0 *= (1.0 - tau);
      x.swap(me_p);
      y.swap(other_p);
      gx.swap(g3);
      gy.swap(g4);
    } else {
      mu1 *= (1.0 - tau);
      y.swap(me_p);
      x.swap(other_p);
      gy.swap(g3);
      gx.swap(g4);
    }
    ++t;
    if (t % o->gap_every == 0 || t == o->max_iters) {
      g_mbb = gap(gx, gy);
      if (!std::isfinite(g_mbb)) return fail(EGT_ERR_NUMERIC, "residual is not finite");
      if (o->eps_mbb > 0 && g_mbb <= o->eps_mbb) break;
    }
  }
  if (o->eps_mbb > 0 && !(g_mbb <= o->eps_mbb)) status = EGT_ERR_NOT_CONVERGED;
  const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  auto unsort = [&](const Vec& v, int S, double* dst) {
    for (int q = 0; q < S; ++q)
      for (int s2 = 0; s2 < H; ++s2) dst[(size_t)q * H + G->order[s2]] = v[(size_t)q * H + s2];
  };
  if (x_out) unsort(x, S0, x_out);
  if (y_out) unsort(y, S1, y_out);
  if (rep) {
    rep->iters = t;
    rep->backoffs = backoffs;
    rep->products = products;
    rep->threads = omp_get_max_threads();
    rep->gap_mbb = g_mbb;
    rep->mu[0] = mu0;
    rep->mu[1] = mu1;
    rep->tau = tau;
    rep->seconds = sec;
  }
  if (status != EGT_OK) return fail(status, "eps_mbb not reached within max_iters");
  return EGT_OK;
}

}  // extern "C"
