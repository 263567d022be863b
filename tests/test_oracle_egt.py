"""Pins of the oracle's EGT drivers (O7, O8).

* eps_sad from the best-response recursion == eps_sad from two LPs;
* the excessive gap condition after every accepted step and the bound
  eps_sad <= mu_x Omega_X + mu_y Omega_Y it implies (Sec. 3);
* the O(1/T) bound of Sec. 3 in the theory mode;
* the closed-form prox (used by the CUDA path) == the literal Alg. 2 prox;
* Kuhn poker converges to its known value;
* planted mistakes (in the oracle, on the CPU) break these pins.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import egt, lp, payoff
from oracle import treeplex as T
from paper_1810_03063_b300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tiny():
    g = payoff.make_game(synth.tiny())
    return g, egt.Problem(g)


def test_gap_equals_lp_duality_gap(tiny):
    g, P = tiny
    r = egt.solve(P, variant="egt_as", eps_mbb=0.0, max_iters=15)
    x_init, _ = egt.initial_point(P, 1e-3, 1e-3)
    for x, y in [(r.x, r.y), (x_init, r.y)]:
        eps = P.eps_sad(x, y)
        lp_eps = lp.best_response_lp(g, 1, x) - lp.best_response_lp(g, 0, y)
        assert eps >= 0
        assert abs(eps - lp_eps) < 1e-6 * max(1.0, abs(lp_eps))


def test_excessive_gap_invariants_egt_as(tiny):
    g, P = tiny
    r = egt.solve(P, variant="egt_as", eps_mbb=0.0, max_iters=40, log_egv=True)
    x, y = r.x, r.y
    for e in r.log:
        assert e["egv"] >= 0
    assert P.eps_sad(x, y) <= r.mux * P.Omega[0] + r.muy * P.Omega[1] + 1e-12
    assert T.is_in_treeplex(P.tpx[0], x, 1e-12) and T.is_in_treeplex(P.tpx[1], y, 1e-12)


def test_theory_mode_rate_bound():
    g = payoff.make_game(synth.kuhn())
    P = egt.Problem(g)
    K = 4 * P.normA * math.sqrt(P.Omega[0] * P.Omega[1] * P.M[0] * P.M[1])
    for Tn in (1, 5, 20, 80):
        r = egt.solve(P, variant="theory", eps_mbb=0.0, max_iters=Tn, log_egv=True)
        assert all(e["egv"] >= -1e-14 for e in r.log)
        assert P.eps_sad(r.x, r.y) <= K / (Tn + 1)


def test_closed_prox_equals_literal_prox(tiny):
    g, P = tiny
    mux = muy = 0.01 * P.theory_mu()
    x, y = egt.initial_point(P, mux, muy)
    for t in range(12):
        me = t % 2
        mu_me, mu_o = (mux, muy) if me == 0 else (muy, mux)
        vm, vo = (x, y) if me == 0 else (y, x)
        a = egt.step(P, me, mu_me, mu_o, vm, vo, 0.3, prox="literal")
        b = egt.step(P, me, mu_me, mu_o, vm, vo, 0.3, prox="closed")
        assert abs(a[0] - b[0]) == 0
        assert np.abs(a[1] - b[1]).max() < 1e-10
        assert np.abs(a[2] - b[2]).max() == 0
        if me == 0:
            mux, x, y = b
        else:
            muy, y, x = b


def test_initial_point_reading(tiny):
    """x^0 = grad d*(-grad f / mu_x) is the smoothed best response to y^0 at mu_x."""
    g, P = tiny
    mux, muy = 0.02, 0.03
    x0, y0 = egt.initial_point(P, mux, muy)
    ref, _ = P.sbr(0, y0, mux)
    assert np.abs(x0 - ref).max() < 1e-12


def test_products_per_step(tiny):
    g, P = tiny
    P.products = 0
    egt.solve(P, variant="egt", eps_mbb=0.0, max_iters=0)
    base = P.products
    P.products = 0
    egt.solve(P, variant="egt", eps_mbb=0.0, max_iters=10, gap_every=1000)
    # init, guard and the first gap check are common; the run adds 3 per Step
    # plus the 2 products of its final gap check
    assert P.products - base == 3 * 10 + 2


def test_kuhn_converges_to_value():
    gold = json.load(open(os.path.join(GOLD, "kuhn_value.json")))
    g = payoff.make_game(synth.kuhn())
    P = egt.Problem(g)
    r = egt.solve(P, variant="egt_as", eps_mbb=0.5, max_iters=5000)
    assert r.gap_mbb <= 0.5
    assert abs(g.value(r.x, r.y) - gold["value_to_player2"]) <= P.eps_sad(r.x, r.y) + 1e-12


def test_planted_sign_mistake_is_caught(monkeypatch):
    """A y-player that maximises the wrong sign (+A^T x) must break the pins above."""
    g = payoff.make_game(synth.kuhn())
    P = egt.Problem(g)
    orig = P.loss_grad

    def wrong(player, other):
        v = orig(player, other)
        return -v if player == 1 else v

    monkeypatch.setattr(P, "loss_grad", wrong)
    r = egt.solve(P, variant="egt", eps_mbb=0.0, max_iters=300, mu0=(0.05, 0.05))
    monkeypatch.setattr(P, "loss_grad", orig)
    gold = json.load(open(os.path.join(GOLD, "kuhn_value.json")))
    assert P.to_mbb(P.eps_sad(r.x, r.y)) > 10.0 or abs(g.value(r.x, r.y) - gold["value_to_player2"]) > 1e-3


def test_planted_beta_mistake_is_caught():
    """beta_j without the factor 2 on children changes Omega away from the vertex maximum."""
    from tests.test_oracle_treeplex import pure_strategies, small_treeplexes
    tpx = small_treeplexes()[0]
    wrong_beta = np.array([1.0 + sum(T.weights(tpx)[k] for i in tpx.infoset_seqs[j]
                                     for k in tpx.children()[i]) for j in range(tpx.n_infosets)])
    V = pure_strategies(tpx)
    true_max = max(T.dgf(tpx, v[:, None]) for v in V)
    assert not np.isclose(T.omega(tpx, wrong_beta), true_max)
