// Betting tree enumeration and treeplex tables (see tree.hpp).
#include "tree.hpp"

#include <algorithm>
#include <cmath>
#include <functional>

namespace egt {

namespace {
enum : int { A_FOLD = 0, A_CHECK = 1, A_CALL = 2, A_ALLIN = 3, A_PASS = 4, A_BET0 = 16 };
constexpr double kEps = 1e-12;
constexpr size_t kMaxNodes = 1u << 22;
}  // namespace

Menus uniform_menus(const double* fracs, int n_fracs, bool allin) {
  Menus m;
  for (int p = 0; p < 2; ++p)
    for (int k = 0; k < 4; ++k) {
      m.m[p][k].fracs.assign(fracs, fracs + n_fracs);
      m.m[p][k].allin = allin;
      m.m[p][k].fold = false;
    }
  return m;
}

std::string compile_betting(double pot, double stack, const Menus& menus, int cap, Compiled& out) {
  auto& nodes = out.nodes;
  nodes.clear();
  std::string err;

  // depth-first enumeration; a node's index is assigned when it is created,
  // terminal children are created in action order between subtree visits (preorder)
  std::function<int(int, double, double, int, int)> visit =
      [&](int player, double c0, double c1, int n_bets, int parent) -> int {
    if (nodes.size() >= kMaxNodes) {
      err = "betting tree too large";
      return -1;
    }
    int me_idx = (int)nodes.size();
    nodes.emplace_back();
    nodes[me_idx].player = player;
    nodes[me_idx].c[0] = c0;
    nodes[me_idx].c[1] = c1;
    nodes[me_idx].n_bets = n_bets;
    nodes[me_idx].parent = parent;
    double c[2] = {c0, c1};
    const int me = player, opp = 1 - player;
    const double to_call = c[opp] - c[me];
    const double remaining = stack - c[me];
    const Menu& menu = menus.m[me][std::min(n_bets, 3)];
    std::vector<std::pair<int, double>> acts;
    if (to_call > 0) {
      acts.push_back({A_FOLD, 0.0});
      acts.push_back({A_CALL, to_call});
    } else {
      if (menu.fold) acts.push_back({A_FOLD, 0.0});
      acts.push_back({A_CHECK, 0.0});
    }
    if (n_bets < cap) {
      const double pot_total = pot + c[0] + c[1];
      for (size_t i = 0; i < menu.fracs.size(); ++i) {
        const double add = to_call + menu.fracs[i] * (pot_total + to_call);
        if (add < remaining - kEps) acts.push_back({A_BET0 + (int)i, add});
      }
      if (menu.allin && remaining > to_call + kEps) acts.push_back({A_ALLIN, remaining});
    }
    for (auto& [code, add] : acts) {
      if (!err.empty()) return -1;
      if (code == A_FOLD && me == 0 && parent < 0) {
        // player 1 folds before player 2 has acted (a menu with fold when not facing a
        // bet): player 2 gets a one-action decision before the terminal, so that every
        // terminal has a sequence of both players (no affine term in the objective)
        int q = (int)nodes.size();
        nodes.emplace_back();
        nodes[q].player = 1;
        nodes[q].c[0] = c0;
        nodes[q].c[1] = c1;
        nodes[q].n_bets = n_bets;
        nodes[q].parent = me_idx;
        nodes[me_idx].actions.push_back({code, q});
        int t = (int)nodes.size();
        nodes.emplace_back();
        nodes[t].c[0] = c0;
        nodes[t].c[1] = c1;
        nodes[t].n_bets = n_bets;
        nodes[t].parent = q;
        nodes[t].kind = 0;
        nodes[t].folder = 0;
        nodes[q].actions.push_back({A_PASS, t});
      } else if (code == A_FOLD) {
        int t = (int)nodes.size();
        nodes.emplace_back();
        nodes[t].c[0] = c0;
        nodes[t].c[1] = c1;
        nodes[t].n_bets = n_bets;
        nodes[t].parent = me_idx;
        nodes[t].kind = 0;
        nodes[t].folder = me;
        nodes[me_idx].actions.push_back({code, t});
      } else if (code == A_CALL || (code == A_CHECK && player == 1)) {
        int t = (int)nodes.size();
        nodes.emplace_back();
        double nc[2] = {c0, c1};
        nc[me] += add;
        nodes[t].c[0] = nc[0];
        nodes[t].c[1] = nc[1];
        nodes[t].n_bets = n_bets;
        nodes[t].parent = me_idx;
        nodes[t].kind = 1;
        nodes[me_idx].actions.push_back({code, t});
      } else if (code == A_CHECK) {
        int ch = visit(1, c0, c1, n_bets, me_idx);
        nodes[me_idx].actions.push_back({code, ch});
      } else {
        double nc[2] = {c0, c1};
        nc[me] += add;
        int ch = visit(opp, nc[0], nc[1], n_bets + 1, me_idx);
        nodes[me_idx].actions.push_back({code, ch});
      }
    }
    return me_idx;
  };
  visit(0, 0.0, 0.0, 0, -1);
  if (!err.empty()) return err;

  const int N = (int)nodes.size();
  // for every node and player: (last own decision node, action slot) on the path, and level
  std::vector<int> own_node[2], own_slot[2], level[2];
  for (int p = 0; p < 2; ++p) {
    own_node[p].assign(N, -1);
    own_slot[p].assign(N, -1);
    level[p].assign(N, 0);
  }
  for (int n = 0; n < N; ++n) {       // parents precede children in preorder
    int par = nodes[n].parent;
    if (par < 0) continue;
    int slot = -1;
    for (int a = 0; a < (int)nodes[par].actions.size(); ++a)
      if (nodes[par].actions[a].second == n) slot = a;
    for (int p = 0; p < 2; ++p) {
      if (nodes[par].player == p) {
        own_node[p][n] = par;
        own_slot[p][n] = slot;
        level[p][n] = level[p][par] + 1;
      } else {
        own_node[p][n] = own_node[p][par];
        own_slot[p][n] = own_slot[p][par];
        level[p][n] = level[p][par];
      }
    }
  }

  std::vector<int> seq_of_node_first[2];  // first sequence index of decision node n (for player p)
  for (int p = 0; p < 2; ++p) {
    Treeplex& T = out.tpx[p];
    seq_of_node_first[p].assign(N, -1);
    std::vector<int> info;
    for (int n = 0; n < N; ++n)
      if (nodes[n].player == p) info.push_back(n);
    std::stable_sort(info.begin(), info.end(), [&](int a, int b) {
      if (level[p][a] != level[p][b]) return level[p][a] < level[p][b];
      return a < b;
    });
    T.J = (int)info.size();
    T.S = 0;
    T.inf_parent.resize(T.J);
    T.inf_first.resize(T.J);
    T.inf_n.resize(T.J);
    T.inf_level.resize(T.J);
    T.inf_node = info;
    for (int j = 0; j < T.J; ++j) {
      int n = info[j];
      T.inf_first[j] = T.S;
      T.inf_n[j] = (int)nodes[n].actions.size();
      T.inf_level[j] = level[p][n];
      seq_of_node_first[p][n] = T.S;
      T.S += T.inf_n[j];
    }
    for (int j = 0; j < T.J; ++j) {
      int n = info[j];
      int on = own_node[p][n];
      T.inf_parent[j] = on < 0 ? -1 : seq_of_node_first[p][on] + own_slot[p][n];
    }
    T.L = T.J ? T.inf_level[T.J - 1] + 1 : 0;
    T.level_ptr.assign(T.L + 1, 0);
    for (int j = 0; j < T.J; ++j) T.level_ptr[T.inf_level[j] + 1]++;
    for (int l = 0; l < T.L; ++l) T.level_ptr[l + 1] += T.level_ptr[l];
    T.seq_infoset.resize(T.S);
    for (int j = 0; j < T.J; ++j)
      for (int a = 0; a < T.inf_n[j]; ++a) T.seq_infoset[T.inf_first[j] + a] = j;
    T.child_ptr.assign(T.S + 1, 0);
    for (int j = 0; j < T.J; ++j)
      if (T.inf_parent[j] >= 0) T.child_ptr[T.inf_parent[j] + 1]++;
    for (int s = 0; s < T.S; ++s) T.child_ptr[s + 1] += T.child_ptr[s];
    T.child_idx.assign(T.child_ptr[T.S], 0);
    std::vector<int> fill(T.child_ptr.begin(), T.child_ptr.end() - 1);
    for (int j = 0; j < T.J; ++j)
      if (T.inf_parent[j] >= 0) T.child_idx[fill[T.inf_parent[j]]++] = j;

    // beta_j = 2 + sum over all child simplexes 2 beta_k; M and Omega by backward induction
    T.beta.assign(T.J, 0.0);
    std::vector<double> m(T.J, 0.0), w(T.J, 0.0);
    for (int j = T.J - 1; j >= 0; --j) {   // deeper levels come later in the order
      double b = 2.0, best_m = 0.0, best_w = 0.0;
      for (int a = 0; a < T.inf_n[j]; ++a) {
        int s = T.inf_first[j] + a;
        double sm = 1.0, sw = 0.0;
        for (int k = T.child_ptr[s]; k < T.child_ptr[s + 1]; ++k) {
          int ch = T.child_idx[k];
          b += 2.0 * T.beta[ch];
          sm += m[ch];
          sw += w[ch];
        }
        best_m = std::max(best_m, sm);
        best_w = a == 0 ? sw : std::max(best_w, sw);
      }
      T.beta[j] = b;
      m[j] = best_m;
      w[j] = b * std::log((double)T.inf_n[j]) + best_w;
    }
    T.m_root = 0.0;
    T.omega_root = 0.0;
    for (int j = 0; j < T.J; ++j)
      if (T.inf_parent[j] < 0) {
        T.m_root += m[j];
        T.omega_root += w[j];
      }
  }

  out.term.clear();
  for (int n = 0; n < N; ++n) {
    if (nodes[n].player >= 0) continue;
    Terminal t;
    for (int p = 0; p < 2; ++p) {
      int on = own_node[p][n];
      if (on < 0) return "a terminal without an action of both players is not supported";
      t.seq[p] = seq_of_node_first[p][on] + own_slot[p][n];
    }
    t.kind = nodes[n].kind;
    if (t.kind == 0)
      t.coef = nodes[n].folder == 0 ? pot / 2 + nodes[n].c[0] : -(pot / 2 + nodes[n].c[1]);
    else
      t.coef = pot / 2 + nodes[n].c[0];
    out.term.push_back(t);
  }
  return "";
}

}  // namespace egt
