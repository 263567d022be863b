"""Pins of the oracle's treeplex routines (O3-O6): beta, depth, M, Omega, SBR, BR, grad d.

Checks come from outside the code under test: the text of the Fig. 1
example, closed-form softmax / log-sum-exp on one simplex (scipy), a generic
constrained optimiser (scipy SLSQP), enumeration of pure strategies (the
vertices of the treeplex), finite differences and the Appendix-A identity.
"""
import itertools
import json
import os

import numpy as np
import pytest
from scipy.optimize import minimize
from scipy.special import logsumexp, softmax

from oracle import treeplex as T
from oracle.game import Treeplex, sequence_form, uniform_behavioural
from paper_1810_03063_b300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def fig1_treeplex():
    gold = json.load(open(os.path.join(GOLD, "fig1_treeplex.json")))
    dims, parvar = gold["simplex_dims"], gold["parent_var_1based"]
    seqs, start = [], 0
    for n in dims:
        seqs.append(list(range(start, start + n)))
        start += n
    parents = [p - 1 for p in parvar]          # 0-based sequence, -1 = none
    # level = number of branchings above
    level = []
    for j, p in enumerate(parents):
        lv, pp = 0, p
        while pp >= 0:
            lv += 1
            owner = next(k for k, s in enumerate(seqs) if pp in s)
            pp = parents[owner]
        level.append(lv)
    return Treeplex(parents, seqs, level), gold["expected"]


def test_fig1_text_facts():
    tpx, exp = fig1_treeplex()
    assert [i + 1 for i in tpx.infoset_seqs[0]] == exp["I_1"]
    assert [i + 1 for i in tpx.infoset_seqs[1]] == exp["I_2"]
    d = T.depths(tpx)
    for k, v in exp["d"].items():
        assert d[int(k) - 1] == v
    for k, v in exp["b"].items():
        assert tpx.infoset_level[int(k) - 1] == v
    assert tpx.infoset_parent[2] + 1 == exp["p_3"]
    beta = T.weights(tpx)
    for k, v in exp["beta_by_hand"].items():
        if k != "note":
            assert beta[int(k) - 1] == v


def pure_strategies(tpx):
    """All vertices of one hand's treeplex: choose one branch in every simplex, zero unreached."""
    choices = itertools.product(*[range(len(s)) for s in tpx.infoset_seqs])
    out = []
    for ch in choices:
        q = np.zeros(tpx.n_seq)
        for j in sorted(range(tpx.n_infosets), key=lambda j: tpx.infoset_level[j]):
            par = 1.0 if tpx.infoset_parent[j] < 0 else q[tpx.infoset_parent[j]]
            q[tpx.infoset_seqs[j][ch[j]]] = par
        out.append(q)
    return np.unique(np.array(out), axis=0)


def small_treeplexes():
    tpx_fig1, _ = fig1_treeplex()
    sf = sequence_form(1.0, 2.0, (1.0,), True, 2)           # tiny game, per-hand trees
    kuhn = sequence_form(2.0, 1.0, (0.5,), True, 1)
    return [tpx_fig1, sf.tpx[0], sf.tpx[1], kuhn.tpx[0], kuhn.tpx[1]]


@pytest.mark.parametrize("k", range(5))
def test_M_and_Omega_by_vertex_enumeration(k):
    tpx = small_treeplexes()[k]
    V = pure_strategies(tpx)
    assert np.isclose(T.max_l1(tpx), V.sum(1).max())
    d_vals = [T.dgf(tpx, v[:, None]) for v in V]
    centre = uniform_behavioural(tpx, 1)
    assert abs(T.dgf(tpx, centre)) < 1e-12                 # min d = 0 at the centre
    assert np.isclose(T.omega(tpx), max(d_vals))


@pytest.mark.parametrize("k", range(5))
def test_best_response_by_vertex_enumeration(k):
    tpx = small_treeplexes()[k]
    V = pure_strategies(tpx)
    rng = np.random.default_rng(k)
    g = rng.normal(size=(tpx.n_seq, 3))
    q, val, per = T.best_response(tpx, g)
    for h in range(3):
        assert np.isclose(per[h], (V @ g[:, h]).min())
    assert np.isclose(val, np.sum(q * g))
    assert T.is_in_treeplex(tpx, q)


@pytest.mark.parametrize("mu", [1.0, 0.3, 0.01])
def test_single_simplex_closed_form(mu):
    tpx = Treeplex([-1], [[0, 1, 2, 3, 4]], [0])
    rng = np.random.default_rng(7)
    g = rng.normal(size=(5, 4)) * 3
    q, val, per = T.smoothed_br(tpx, g, mu)
    beta = 2.0
    assert np.allclose(q, softmax(-g / (mu * beta), axis=0), rtol=1e-13)
    ref = -mu * beta * logsumexp(-g / (mu * beta), axis=0) + mu * beta * np.log(5)
    assert np.allclose(per, ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("k", range(5))
@pytest.mark.parametrize("mu", [2.0, 0.2])
def test_sbr_value_is_objective_and_invariants(k, mu):
    tpx = small_treeplexes()[k]
    rng = np.random.default_rng(10 + k)
    g = rng.normal(size=(tpx.n_seq, 2))
    q, val, per = T.smoothed_br(tpx, g, mu)
    assert T.is_in_treeplex(tpx, q, tol=1e-13)
    assert (q > 0).all()
    # value from the recursion == objective evaluated directly with d(q)
    assert np.isclose(val, np.sum(q * g) + mu * T.dgf(tpx, q), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("k", [0, 1, 3])
def test_sbr_against_generic_solver(k):
    tpx = small_treeplexes()[k]
    rng = np.random.default_rng(3 + k)
    g = rng.normal(size=(tpx.n_seq, 1))
    mu = 0.7
    q, val, _ = T.smoothed_br(tpx, g, mu)
    S = tpx.n_seq
    cons = []
    for j in range(tpx.n_infosets):
        seqs, p = tpx.infoset_seqs[j], tpx.infoset_parent[j]
        cons.append({"type": "eq", "fun": (lambda z, seqs=seqs, p=p:
                                           z[seqs].sum() - (1.0 if p < 0 else z[p]))})

    def obj(z):
        return float(z @ g[:, 0] + mu * T.dgf(tpx, np.maximum(z, 1e-300)[:, None]))

    x0 = uniform_behavioural(tpx, 1)[:, 0]
    res = minimize(obj, x0, constraints=cons, bounds=[(1e-12, 1)] * S, method="SLSQP",
                   options=dict(ftol=1e-14, maxiter=1000))
    assert res.fun >= val - 1e-9                    # nothing feasible beats the SBR
    assert abs(res.fun - val) < 1e-6
    assert np.abs(res.x - q[:, 0]).max() < 1e-3


@pytest.mark.parametrize("k", range(5))
def test_grad_d_finite_differences_and_appendix_identity(k):
    tpx = small_treeplexes()[k]
    rng = np.random.default_rng(20 + k)
    q, _, _ = T.smoothed_br(tpx, rng.normal(size=(tpx.n_seq, 1)), 1.0)
    gd = T.grad_dgf(tpx, q)
    # directional derivative along feasible directions (difference of two interior points)
    q2, _, _ = T.smoothed_br(tpx, rng.normal(size=(tpx.n_seq, 1)), 1.0)
    v = q2 - q
    h = 1e-6
    fd = (T.dgf(tpx, q + h * v) - T.dgf(tpx, q - h * v)) / (2 * h)
    assert np.isclose(fd, float(np.sum(gd * v)), rtol=1e-6, atol=1e-8)
    # Appendix A: -d(q) + <grad d(q), q> = -sum_roots beta_j (log n_j - 1)
    lhs = -T.dgf(tpx, q) + float(np.sum(gd * q))
    assert np.isclose(lhs, T.prox_shift_constant(tpx, 1), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("k", range(5))
def test_conjugate_gradient_inverts_grad_d(k):
    """grad d*(grad d(q)) = q for interior q (d strictly convex, grad d* its inverse map)."""
    tpx = small_treeplexes()[k]
    rng = np.random.default_rng(30 + k)
    q, _, _ = T.smoothed_br(tpx, rng.normal(size=(tpx.n_seq, 2)), 0.5)
    back = T.conj_grad(tpx, T.grad_dgf(tpx, q))
    assert np.allclose(back, q, rtol=1e-10, atol=1e-13)
