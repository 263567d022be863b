// Host-side game compiler: public betting tree -> per-player treeplex tables,
// terminal tables, hand/card tables for the structured gradient.
//
// Game (Sec. 7 "Experiments", subgame description): chance deals private
// hands from each player's range, player 1 acts first, fold ends the game,
// call or check-check goes to showdown (better hand wins, tie splits).
// Betting rules applied to the menus (equal stacks, bet = f * pot_total,
// raise = call + f * (pot_total + call), sizes reaching the stack dropped,
// all-in while under the cap and chips remain, cap counts the opening bet and
// raises, fold when not facing a bet only where the menu offers it) are the
// reading of Sec. 7's Libratus menus; the menu of a decision depends on the
// player and on the bets / raises made so far (0, 1, 2, 3 or more).
//
// Canonical numbering (stated in include/egt.h): public tree depth first with
// actions fold, check/call, menu sizes, all-in; information sets of a player
// sorted by (level, preorder index); sequences infoset by infoset in action
// order; terminals in preorder; hands in ascending strength, ties by input
// index.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace egt {

struct PubNode {
  int player = -1;          // 0/1 acting, -1 terminal
  double c[2] = {0, 0};     // river chips in
  int n_bets = 0;
  int parent = -1;
  int kind = 0;             // terminal: 0 fold, 1 showdown
  int folder = -1;
  std::vector<std::pair<int, int>> actions;  // (action code, child index)
};

// per-player treeplex of one hand
struct Treeplex {
  int S = 0, J = 0, L = 0;               // sequences, simplexes (infosets), levels
  std::vector<int> inf_parent;           // [J] parent sequence, -1 = root (q_{p_j} = 1)
  std::vector<int> inf_first;            // [J] first sequence of simplex j
  std::vector<int> inf_n;                // [J] number of actions n_j
  std::vector<int> inf_level;            // [J] b_Q^j
  std::vector<int> inf_node;             // [J] public node
  std::vector<int> level_ptr;            // [L+1] simplexes of level l: [level_ptr[l], level_ptr[l+1])
  std::vector<int> child_ptr;            // [S+1] CSR: child simplexes D_j^i of sequence i
  std::vector<int> child_idx;
  std::vector<int> seq_infoset;          // [S]
  std::vector<double> beta;              // [J] beta_j = 2 + sum over children 2 beta_k
  double m_root = 0;                     // max l1 norm of one hand's treeplex
  double omega_root = 0;                 // max d over one hand's treeplex (min is 0)
};

struct Terminal {
  int seq[2];        // sigma_1(b), sigma_2(b)
  int kind;          // 0 fold, 1 showdown
  double coef;       // fold: payoff to player 2; showdown: stake (pot/2 + chips)
};

// The menu of one decision situation.
struct Menu {
  std::vector<double> fracs;
  bool allin = true;
  bool fold = false;     // fold offered when not facing a bet
};

// menus[p][k]: player p after k bets / raises (k = 3: three or more)
struct Menus {
  Menu m[2][4];
};

struct Compiled {
  std::vector<PubNode> nodes;
  Treeplex tpx[2];
  std::vector<Terminal> term;
};

// Build the public tree and both treeplexes. Returns "" on success, else a message.
std::string compile_betting(double pot, double stack, const Menus& menus, int cap, Compiled& out);

// The same menu everywhere (no fold unless facing a bet).
Menus uniform_menus(const double* fracs, int n_fracs, bool allin);

}  // namespace egt
