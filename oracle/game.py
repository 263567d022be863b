"""O1: river endgame -> extensive-form game -> sequence form (oracle, FP64).

Game (Sec. 7, "Experiments", the subgame description): chance deals each
player a private hand from that player's range; the pot and the board are
fixed; player 1 moves first; the game ends on a fold (the other player wins),
on a call or on two opening checks (showdown: better hand wins, tie splits).

Betting rules (the paper lists Libratus' menus only; the synthetic games use
this reading, applied identically by the CUDA library):

* equal effective stacks; each player already has ``pot / 2`` in the pot;
* not facing a bet: check, or bet ``f * pot_total`` for each f of the menu;
* facing a bet: fold, call, or raise to ``call + f * (pot_total + call)``;
* a size that reaches the remaining stack is dropped; all-in is offered
  while bets remain under the cap and chips remain after calling;
* ``raise_cap`` counts the opening bet plus the raises;
* no fold when not facing a bet; check-check and call go to showdown.

Sec. 7 describes Libratus' abstraction with a different menu per player and
per betting situation (its opening, facing the first bet, facing a raise,
facing later raises) and with fold offered even when not facing a bet.  With
``menus`` given, the menu of a decision is ``menus[player][min(k, 3)]`` with
k the bets and raises made so far: (pot fractions, all-in offered, fold
offered when not facing a bet); every other rule above is unchanged.  When
player 1 folds before player 2 has acted, player 2 gets a decision with the one
action "pass" before that terminal: the game (and its value) is unchanged, and
every terminal keeps a sequence of both players, so the objective stays
bilinear with no affine term (y's pass coordinate is always 1).

Payoffs are to player 2 (the maximiser y of min_x max_y <x, Ay>): the loser of
a fold or showdown pays ``pot / 2`` plus their river chips, a tie pays 0.

Sequence form (Sec. 4 treeplex notation): for player p, an information set
is (public node where p acts, p's private hand).  A sequence is an
(information set, action) pair.  Vectors are laid out ``[seq][hand]``: the
public sequence index ``s`` (shared by all hands) and the hand index.  The
empty sequence is not stored (its value is 1).

Canonical numbering (the CUDA library follows the same definition, so indices
agree without any shared code):

* public tree visited depth first, actions in the order fold, check/call,
  bet or raise sizes in menu order, all-in;
* information sets of a player sorted by (level, preorder index of their
  public node), level = number of the player's own earlier actions (b_Q^j);
* sequences numbered information set by information set, actions in order;
* terminals in preorder.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

FOLD, CHECK, CALL, BET, ALLIN, PASS = "f", "k", "c", "b", "a", "p"


@dataclass
class PublicNode:
    pre: int                 # preorder index
    player: int              # 0 / 1 to act, -1 for a terminal
    contrib: tuple           # river chips (c0, c1) put in so far
    n_bets: int
    history: tuple           # ((player, label), ...)
    parent: int = -1
    actions: list = field(default_factory=list)   # [(label, child pre index)]
    kind: str = ""           # terminal kind: "fold" / "showdown"
    folder: int = -1


def build_public_tree(pot, stack, bet_fracs, allin, raise_cap, menus=None):
    """Enumerate the public betting tree under the rules in the module docstring."""
    nodes: list[PublicNode] = []
    eps = 1e-12

    def menu_of(player, n_bets):
        if menus is None:
            return tuple(bet_fracs), bool(allin), False
        fr, al, fo = menus[player][min(n_bets, 3)]
        return tuple(fr), bool(al), bool(fo)

    def visit(player, contrib, n_bets, history, parent):
        node = PublicNode(pre=len(nodes), player=player, contrib=contrib, n_bets=n_bets,
                          history=history, parent=parent)
        nodes.append(node)
        me, opp = player, 1 - player
        to_call = contrib[opp] - contrib[me]
        remaining = stack - contrib[me]
        fracs, can_allin, fold_unfacing = menu_of(player, n_bets)
        acts = []
        if to_call > 0:
            acts.append((FOLD, 0.0))
            acts.append((CALL, to_call))
        else:
            if fold_unfacing:
                acts.append((FOLD, 0.0))
            acts.append((CHECK, 0.0))
        if n_bets < raise_cap:
            pot_total = pot + contrib[0] + contrib[1]
            for i, f in enumerate(fracs):
                add = to_call + f * (pot_total + to_call)
                if add < remaining - eps:
                    acts.append((f"{BET}{i}", add))
            if can_allin and remaining > to_call + eps:
                acts.append((ALLIN, remaining))
        for label, add in acts:
            h = history + ((player, label),)
            if label == FOLD and player == 0 and parent < 0:
                q = PublicNode(pre=len(nodes), player=1, contrib=contrib, n_bets=n_bets, history=h,
                               parent=node.pre)
                nodes.append(q)
                node.actions.append((label, q.pre))
                t = PublicNode(pre=len(nodes), player=-1, contrib=contrib, n_bets=n_bets,
                               history=h + ((1, PASS),), parent=q.pre, kind="fold", folder=0)
                nodes.append(t)
                q.actions.append((PASS, t.pre))
            elif label == FOLD:
                t = PublicNode(pre=len(nodes), player=-1, contrib=contrib, n_bets=n_bets,
                               history=h, parent=node.pre, kind="fold", folder=me)
                nodes.append(t)
                node.actions.append((label, t.pre))
            elif label == CALL or (label == CHECK and player == 1):
                c = list(contrib)
                c[me] += add
                t = PublicNode(pre=len(nodes), player=-1, contrib=tuple(c), n_bets=n_bets,
                               history=h, parent=node.pre, kind="showdown")
                nodes.append(t)
                node.actions.append((label, t.pre))
            elif label == CHECK:
                child = visit(1, contrib, n_bets, h, node.pre)
                node.actions.append((label, child))
            else:
                c = list(contrib)
                c[me] += add
                child = visit(opp, tuple(c), n_bets + 1, h, node.pre)
                node.actions.append((label, child))
        return node.pre

    visit(0, (0.0, 0.0), 0, (), -1)
    return nodes


@dataclass
class Treeplex:
    """Sequence-form strategy polytope of one player for ONE private hand.

    The full strategy space is the Cartesian product of this treeplex over
    the hands (the root Cartesian product, Sec. 6).

    infoset_parent[j]  parent sequence p_j of simplex j (-1: none, q_{p_j}=1)
    infoset_seqs[j]    list of sequence indices I_j of simplex j
    infoset_level[j]   b_Q^j (number of branching operations above j)
    """

    infoset_parent: list
    infoset_seqs: list
    infoset_level: list
    infoset_node: list = field(default_factory=list)

    @property
    def n_seq(self):
        return sum(len(s) for s in self.infoset_seqs)

    @property
    def n_infosets(self):
        return len(self.infoset_parent)

    def seq_infoset(self):
        out = np.empty(self.n_seq, dtype=np.int64)
        for j, seqs in enumerate(self.infoset_seqs):
            out[seqs] = j
        return out

    def children(self):
        """D_j^i: for each sequence i, the simplexes whose parent is i."""
        ch = [[] for _ in range(self.n_seq)]
        for j, p in enumerate(self.infoset_parent):
            if p >= 0:
                ch[p].append(j)
        return ch

    def roots(self):
        return [j for j, p in enumerate(self.infoset_parent) if p < 0]


@dataclass
class Terminal:
    pre: int
    kind: str          # "fold" / "showdown"
    seq: tuple         # (sigma_1(b), sigma_2(b)); -1 would be the empty sequence
    folder: int
    contrib: tuple


@dataclass
class SequenceForm:
    nodes: list
    tpx: tuple          # (Treeplex of player 1, Treeplex of player 2)
    terminals: list
    seq_labels: tuple   # per player: list of public histories ending with that sequence's action


def sequence_form(pot, stack, bet_fracs, allin, raise_cap, menus=None) -> SequenceForm:
    nodes = build_public_tree(pot, stack, bet_fracs, allin, raise_cap, menus)

    # information sets of each player with their parent (public) sequence
    info = [[], []]
    # parent sequence of node n for player p = last (node, action) of p on the path
    def last_own_action(n, p):
        child = n
        node = nodes[n].parent
        while node >= 0:
            if nodes[node].player == p:
                label = next(lbl for lbl, c in nodes[node].actions if c == child)
                return (node, label)
            child = node
            node = nodes[node].parent
        return None

    def level(n, p):
        cnt, node = 0, nodes[n].parent
        while node >= 0:
            if nodes[node].player == p:
                cnt += 1
            node = nodes[node].parent
        return cnt

    for n in nodes:
        if n.player >= 0:
            info[n.player].append(n.pre)

    tpx, labels, seq_of = [], [], [{}, {}]
    for p in range(2):
        order = sorted(info[p], key=lambda n: (level(n, p), n))
        seqs, lvls, lab = [], [], []
        s = 0
        for n in order:
            ids = []
            for label, _ in nodes[n].actions:
                seq_of[p][(n, label)] = s
                lab.append(nodes[n].history + ((p, label),))
                ids.append(s)
                s += 1
            seqs.append(ids)
            lvls.append(level(n, p))
        parents = []
        for n in order:
            pa = last_own_action(n, p)
            parents.append(-1 if pa is None else seq_of[p][pa])
        tpx.append(Treeplex(parents, seqs, lvls, list(order)))
        labels.append(lab)

    terminals = []
    for n in nodes:
        if n.player < 0:
            sig = []
            for p in range(2):
                pa = last_own_action(n.pre, p)
                sig.append(-1 if pa is None else seq_of[p][pa])
            terminals.append(Terminal(n.pre, n.kind, tuple(sig), n.folder, n.contrib))
    return SequenceForm(nodes, tuple(tpx), terminals, tuple(labels))


def terminal_payoff_to_p2(term: Terminal, pot: float, s1: float, s2: float) -> float:
    """Payoff to player 2 at a terminal for hands of strength s1 (P1) and s2 (P2)."""
    if term.kind == "fold":
        if term.folder == 0:
            return pot / 2 + term.contrib[0]
        return -(pot / 2 + term.contrib[1])
    stake = pot / 2 + term.contrib[0]
    return float(np.sign(s2 - s1)) * stake


def compatible(hand_a, hand_b) -> bool:
    """Two private hands can be dealt together iff they share no card."""
    return not (set(int(c) for c in hand_a) & set(int(c) for c in hand_b))


def chance(spec):
    """Chance probabilities p(h1, h2) = r1(h1) r2(h2) [compatible] / Z, by brute force."""
    hands = np.asarray(spec.hands)
    H, k = hands.shape
    # C[a, b] = 1 iff no card of hand a equals a card of hand b (all k x k card pairs compared)
    share = np.zeros((H, H), dtype=bool)
    for i in range(k):
        for j in range(k):
            share |= hands[:, i][:, None] == hands[:, j][None, :]
    C = (~share).astype(np.float64)
    W = spec.ranges[0][:, None] * spec.ranges[1][None, :] * C
    Z = W.sum()
    return W / Z, C, Z


def uniform_behavioural(tpx: Treeplex, n_hands: int) -> np.ndarray:
    """DGF centre x_omega: each simplex plays uniformly (d = 0 there)."""
    q = np.zeros((tpx.n_seq, n_hands))
    for j in sorted(range(tpx.n_infosets), key=lambda j: tpx.infoset_level[j]):
        par = 1.0 if tpx.infoset_parent[j] < 0 else q[tpx.infoset_parent[j]]
        for i in tpx.infoset_seqs[j]:
            q[i] = par / len(tpx.infoset_seqs[j])
    return q
