"""Pins of the oracle's game model and payoff products (O1, O2).

Each test ties the oracle to something outside itself: Kuhn poker's known
value, an LP solve, the closed-form showdown equity of a check-only game,
betting-tree counts, and a second (structured) formula for the products.
"""
import json
import os
from itertools import combinations

import numpy as np
import pytest

from oracle import game as G
from oracle import lp, payoff
from paper_1810_03063_b300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def counts(spec):
    sf = G.sequence_form(spec.pot, spec.stack, spec.bet_fracs, spec.allin, spec.raise_cap)
    n_fold = sum(t.kind == "fold" for t in sf.terminals)
    return ([t.n_seq for t in sf.tpx], [t.n_infosets for t in sf.tpx],
            (n_fold, len(sf.terminals) - n_fold))


@pytest.mark.parametrize("make,S,J,T", [
    (lambda: synth.tiny(), 10, 4, (6, 7)),
    (lambda: synth.full_deck(), 61, 21, (40, 41)),
    (lambda: synth.full_deck(stack=2.0), 22, 8, (14, 15)),
    (lambda: synth.large(), 508, 170, (338, 339)),
])
def test_betting_tree_counts(make, S, J, T):
    spec = make()
    s, j, t = counts(spec)
    assert s == [S, S] and j == [J, J] and t == T


def test_hand_counts():
    assert synth.tiny().n_hands == 105          # C(15, 2)
    assert synth.full_deck().n_hands == 1081    # C(47, 2)


def test_kuhn_structure_and_value():
    gold = json.load(open(os.path.join(GOLD, "kuhn_value.json")))
    spec = synth.kuhn()
    g = payoff.make_game(spec)
    assert g.S[0] * g.H == gold["sequences_per_player_without_empty"]
    assert g.S[1] * g.H == gold["sequences_per_player_without_empty"]
    assert g.tpx[0].n_infosets * g.H == gold["infosets_per_player"]
    v, _ = lp.game_value(g)
    assert abs(v - gold["value_to_player2"]) < 1e-9


def test_check_only_game_is_showdown_equity():
    """cap 0: both players only check; value = sum_{h1,h2} p(h1,h2) sign(s2 - s1) pot/2."""
    base = synth.tiny(seed=5)
    spec = synth.GameSpec(**{**base.__dict__, "raise_cap": 0})
    g = payoff.make_game(spec)
    assert g.S == (1, 1)
    x = np.ones((1, g.H))
    y = np.ones((1, g.H))
    # brute force over dealt pairs, straight from the game description
    num = 0.0
    Z = 0.0
    for a in range(spec.n_hands):
        for b in range(spec.n_hands):
            if set(spec.hands[a]) & set(spec.hands[b]):
                continue
            w = spec.ranges[0][a] * spec.ranges[1][b]
            Z += w
            num += w * np.sign(spec.strength[b] - spec.strength[a]) * spec.pot / 2
    assert abs(g.value(x, y) - num / Z) < 1e-13


def test_products_agree_and_zero_sum():
    spec = synth.tiny(seed=11)
    d = payoff.DenseGame(spec)
    f = payoff.FactoredGame(spec)
    b = payoff.BatchedFactoredGame(spec)
    rng = np.random.default_rng(0)
    y = rng.random((d.S[1], d.H))
    x = rng.random((d.S[0], d.H))
    for other in (f, b):
        assert np.allclose(other.Ay(y), d.Ay(y), rtol=1e-13, atol=1e-16)
        assert np.allclose(other.Atx(x), d.Atx(x), rtol=1e-13, atol=1e-16)
    # <x, Ay> = <A^T x, y>: catches a transposed block or a swapped sigma
    for gm in (d, f, b):
        assert abs(np.sum(x * gm.Ay(y)) - np.sum(gm.Atx(x) * y)) < 1e-12 * np.abs(x).sum()


def test_norm_A_is_max_entry():
    spec = synth.tiny(seed=3)
    d = payoff.DenseGame(spec)
    assert d.norm_A() == np.abs(d.A).max()


def test_lp_value_within_gap_of_egt():
    from oracle import egt
    spec = synth.tiny()
    g = payoff.make_game(spec)
    v, _ = lp.game_value(g)
    P = egt.Problem(g)
    r = egt.solve(P, variant="egt_as", eps_mbb=50.0, max_iters=300, gap_every=25)
    eps = P.eps_sad(r.x, r.y)
    val = g.value(r.x, r.y)
    assert abs(val - v) <= eps + 1e-9


# ---- the structured products the CUDA path uses, written out independently ----

def structured_products(spec, sf, vec, out_player):
    """Card-removal inclusion-exclusion + strength-sorted sums, per terminal (pure numpy)."""
    H = spec.n_hands
    hands = spec.hands
    r = spec.ranges
    # Z = sum over compatible pairs of r1 r2 by inclusion-exclusion over shared cards
    R = [r[0].sum(), r[1].sum()]
    per_card = np.zeros((2, spec.n_cards))
    for p in range(2):
        for c in range(hands.shape[1]):
            np.add.at(per_card[p], hands[:, c], r[p])
    Z = R[0] * R[1] - per_card[0] @ per_card[1] + (r[0] * r[1]).sum()
    opp = 1 - out_player
    S_out = sf.tpx[out_player].n_seq
    out = np.zeros((S_out, H))
    s = spec.strength
    for t in sf.terminals:
        w = r[opp] * vec[t.seq[opp]]
        W = w.sum()
        card_tot = np.zeros(spec.n_cards)
        for c in range(2):
            np.add.at(card_tot, hands[:, c], w)
        if t.kind == "fold":
            u = G.terminal_payoff_to_p2(t, spec.pot, 0, 0)
            compat = W - card_tot[hands[:, 0]] - card_tot[hands[:, 1]] + w
            contrib = u * compat
        else:
            stake = spec.pot / 2 + t.contrib[0]
            # prefix sums in ascending strength; ties are neither weaker nor stronger
            order = np.argsort(s, kind="stable")
            s_sorted = s[order]
            pref = np.concatenate([[0.0], np.cumsum(w[order])])
            lo = np.searchsorted(s_sorted, s, "left")
            hi = np.searchsorted(s_sorted, s, "right")
            lt = pref[lo]
            gt = W - pref[hi]
            # card removal: subtract, for each own card, the same sums over hands holding it
            for c in range(spec.n_cards):
                holders = np.where((hands == c).any(1))[0]
                if len(holders) == 0:
                    continue
                ho = holders[np.argsort(s[holders], kind="stable")]
                hs = s[ho]
                cp = np.concatenate([[0.0], np.cumsum(w[ho])])
                mine = np.where((hands == c).any(1))[0]
                lt[mine] -= cp[np.searchsorted(hs, s[mine], "left")]
                gt[mine] -= cp[-1] - cp[np.searchsorted(hs, s[mine], "right")]
            # payoff to P2 is +stake when P2's hand is stronger
            contrib = stake * ((gt - lt) if out_player == 0 else (lt - gt))
        out[t.seq[out_player]] += r[out_player] / Z * contrib
    return out


def test_structured_products_match_brute_force():
    spec = synth.tiny(seed=21)
    g = payoff.DenseGame(spec)
    rng = np.random.default_rng(1)
    y = rng.random((g.S[1], g.H))
    x = rng.random((g.S[0], g.H))
    assert np.allclose(structured_products(spec, g.sf, y, 0), g.Ay(y), rtol=1e-12, atol=1e-15)
    assert np.allclose(structured_products(spec, g.sf, x, 1), g.Atx(x), rtol=1e-12, atol=1e-15)


def test_libratus_menus_match_the_hand_derived_tree():
    """Sec. 7's asymmetric menus at stack = pot, derived by hand in the golden file."""
    import json
    import pathlib
    gold = json.loads((pathlib.Path(__file__).parent / "golden" / "libratus_stack1.json").read_text())
    sf = G.sequence_form(gold["game"]["pot"], gold["game"]["stack"], (), True, 64, synth.LIBRATUS_MENUS)
    assert len(sf.terminals) == gold["terminals"]
    assert [sf.tpx[0].n_seq, sf.tpx[1].n_seq] == gold["sequences"]
    for p, key in enumerate(("player1", "player2")):
        sizes = sorted(len(s) for s in sf.tpx[p].infoset_seqs)
        assert sizes == sorted(gold["infoset_sizes"][key])


def test_uniform_menus_reproduce_the_single_menu_tree():
    spec = synth.large()
    same = tuple(tuple((spec.bet_fracs, spec.allin, False) for _ in range(4)) for _ in range(2))
    a = G.sequence_form(spec.pot, spec.stack, spec.bet_fracs, spec.allin, spec.raise_cap)
    b = G.sequence_form(spec.pot, spec.stack, (), False, spec.raise_cap, same)
    assert [t.seq for t in a.terminals] == [t.seq for t in b.terminals]
    for p in range(2):
        assert a.tpx[p].infoset_seqs == b.tpx[p].infoset_seqs
        assert a.tpx[p].infoset_parent == b.tpx[p].infoset_parent


def test_fold_before_the_opponent_acts_keeps_the_game_bilinear():
    """Player 1's opening fold gets a one-action pass decision of player 2: every terminal
    has a sequence of both players, and the pass sequence is the only action of its simplex."""
    sf = G.sequence_form(1.0, 2.0, (), True, 64, synth.LIBRATUS_MENUS)
    assert all(t.seq[0] >= 0 and t.seq[1] >= 0 for t in sf.terminals)
    folds_at_root = [t for t in sf.terminals if t.kind == "fold" and t.folder == 0 and t.contrib == (0.0, 0.0)]
    assert len(folds_at_root) == 1
    s2 = folds_at_root[0].seq[1]
    j = [k for k, seqs in enumerate(sf.tpx[1].infoset_seqs) if s2 in seqs]
    assert len(j) == 1 and len(sf.tpx[1].infoset_seqs[j[0]]) == 1
