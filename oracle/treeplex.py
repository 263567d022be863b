"""O3-O6: dilated entropy DGF on a treeplex, smoothed / plain best responses (oracle, FP64).

Notation of Sec. 4-5: simplex j has variables I_j (``infoset_seqs[j]``),
parent variable p_j (``infoset_parent[j]``, -1 meaning q_{p_j} = 1), and for
a branch i the child simplexes D_j^i (``children()[i]``).  Vectors are
``[seq][hand]``; every hand carries its own copy of the per-hand treeplex
(Cartesian product at the root, Sec. 6), so every routine below works on all
hands at once with numpy rows and loops over simplexes only.

* beta_j = 2 + sum_{k in D^j} 2 beta_k with D^j = all children of j    (Sec. 5)
* d_j(u) = sum_i u_i log u_i + log n_j,   d(q) = sum_j beta_j q_{p_j} d_j(q^j / q_{p_j})
* modulus 1/M, M = max l1 norm over Q                                   (Sec. 5)
* Omega = max d - min d over Q                                           (Sec. 3)
* SBR: argmin <q, g> + mu d(q) by the bottom-up / top-down recursion of Sec. 5
* grad d and the prox-shift identity of Appendix A.
"""
from __future__ import annotations

import numpy as np

from .game import Treeplex


def _bottom_up(tpx: Treeplex):
    """Simplexes deepest first (children before parents)."""
    return sorted(range(tpx.n_infosets), key=lambda j: -tpx.infoset_level[j])


def _top_down(tpx: Treeplex):
    return sorted(range(tpx.n_infosets), key=lambda j: tpx.infoset_level[j])


def weights(tpx: Treeplex) -> np.ndarray:
    """beta_j = 2 + sum over all child simplexes k of 2 beta_k (leaf: beta = 2)."""
    ch = tpx.children()
    beta = np.zeros(tpx.n_infosets)
    for j in _bottom_up(tpx):
        beta[j] = 2.0 + sum(2.0 * beta[k] for i in tpx.infoset_seqs[j] for k in ch[i])
    return beta


def depths(tpx: Treeplex) -> np.ndarray:
    """d_j: largest number of simplexes met in a chain of branchings below j (leaf: 0)."""
    ch = tpx.children()
    d = np.zeros(tpx.n_infosets, dtype=np.int64)
    for j in _bottom_up(tpx):
        below = [d[k] + 1 for i in tpx.infoset_seqs[j] for k in ch[i]]
        d[j] = max(below) if below else 0
    return d


def max_l1(tpx: Treeplex) -> float:
    """M for one hand: max over Q of sum_i q_i (q >= 0), by backward induction."""
    ch = tpx.children()
    m = np.zeros(tpx.n_infosets)
    for j in _bottom_up(tpx):
        m[j] = max(1.0 + sum(m[k] for k in ch[i]) for i in tpx.infoset_seqs[j])
    return float(sum(m[j] for j in tpx.roots()))


def omega(tpx: Treeplex, beta=None) -> float:
    """Omega for one hand = max_Q d (min_Q d = 0 at the uniform point).

    d is convex, so its maximum over each simplex sits at a vertex, where
    d_j = log n_j; backward induction: w_j = beta_j log n_j + max_i sum_{k in D_j^i} w_k.
    """
    beta = weights(tpx) if beta is None else beta
    ch = tpx.children()
    w = np.zeros(tpx.n_infosets)
    for j in _bottom_up(tpx):
        n = len(tpx.infoset_seqs[j])
        w[j] = beta[j] * np.log(n) + max(sum(w[k] for k in ch[i]) for i in tpx.infoset_seqs[j])
    return float(sum(w[j] for j in tpx.roots()))


def _parent_mass(tpx, q, j):
    p = tpx.infoset_parent[j]
    return np.ones(q.shape[1]) if p < 0 else q[p]


def _xlogy(x, y):
    """x * log(y) with the convention 0 * log 0 = 0."""
    out = np.zeros_like(x)
    nz = x > 0
    out[nz] = x[nz] * np.log(y[nz])
    return out


def dgf(tpx: Treeplex, q: np.ndarray, beta=None) -> float:
    """d(q) = sum_j beta_j q_{p_j} d_j(q^j / q_{p_j}), summed over hands."""
    beta = weights(tpx) if beta is None else beta
    total = np.zeros(q.shape[1])
    for j in range(tpx.n_infosets):
        qp = _parent_mass(tpx, q, j)
        seqs = tpx.infoset_seqs[j]
        n = len(seqs)
        inner = np.zeros(q.shape[1])
        for i in seqs:
            safe_qp = np.where(qp > 0, qp, 1.0)
            inner += _xlogy(q[i], q[i] / safe_qp)   # q_pj * u_i log u_i with u_i = q_i / q_pj
        total += beta[j] * (inner + qp * np.log(n))
    return float(total.sum())


def grad_dgf(tpx: Treeplex, q: np.ndarray, beta=None) -> np.ndarray:
    """Appendix A: grad_{ji} d(q) = beta_j (log(q_i / q_{p_j}) + 1) + sum_{k in D_j^i} beta_k (log n_k - 1).

    Valid on the relative interior of Q (q > 0); a zero entry gives -inf.
    """
    beta = weights(tpx) if beta is None else beta
    ch = tpx.children()
    out = np.zeros_like(q)
    with np.errstate(divide="ignore"):
        for j in range(tpx.n_infosets):
            qp = _parent_mass(tpx, q, j)
            for i in tpx.infoset_seqs[j]:
                out[i] = beta[j] * (np.log(q[i] / qp) + 1.0)
                for k in ch[i]:
                    out[i] += beta[k] * (np.log(len(tpx.infoset_seqs[k])) - 1.0)
    return out


def smoothed_br(tpx: Treeplex, g: np.ndarray, mu: float, beta=None):
    """argmin_{q in Q} <q, g> + mu d(q) and its value (Sec. 5).

    Bottom-up: at simplex j the child simplex values are added to the branch
    that scales them, giving g_hat; the leaf problem over the simplex has
    q_bar_i proportional to exp(-g_hat_i / (mu beta_j)); the value sent to the
    parent is g_hat_i + mu beta_j log q_bar_i + mu beta_j log n_j at the
    index with the largest q_bar_i.  Top-down: q_i = q_{p_j} q_bar_i.

    Returns (q [S, H], total value summed over hands, per-hand value [H]).
    """
    beta = weights(tpx) if beta is None else beta
    S, H = g.shape
    ch = tpx.children()
    V = np.zeros((tpx.n_infosets, H))
    qbar = np.zeros((S, H))
    for j in _bottom_up(tpx):
        seqs = tpx.infoset_seqs[j]
        n = len(seqs)
        t = mu * beta[j]
        ghat = np.stack([g[i] + sum((V[k] for k in ch[i]), np.zeros(H)) for i in seqs])
        istar = np.argmin(ghat, axis=0)                       # largest q_bar
        gstar = ghat[istar, np.arange(H)]
        e = np.exp(-(ghat - gstar[None, :]) / t)
        ub = e / e.sum(axis=0)
        qbar[seqs] = ub
        V[j] = gstar + t * np.log(ub[istar, np.arange(H)]) + t * np.log(n)
    q = np.zeros((S, H))
    for j in _top_down(tpx):
        qp = _parent_mass(tpx, q, j)
        for i in tpx.infoset_seqs[j]:
            q[i] = qp * qbar[i]
    per_hand = sum(V[j] for j in tpx.roots())
    return q, float(per_hand.sum()), per_hand


def best_response(tpx: Treeplex, g: np.ndarray):
    """min_{q in Q} <q, g> (the mu -> 0 limit): min instead of the smoothed value.

    Returns (pure minimiser q with first-index tie break, total value, per-hand value).
    """
    S, H = g.shape
    ch = tpx.children()
    V = np.zeros((tpx.n_infosets, H))
    choice = np.zeros((tpx.n_infosets, H), dtype=np.int64)
    for j in _bottom_up(tpx):
        seqs = tpx.infoset_seqs[j]
        ghat = np.stack([g[i] + sum((V[k] for k in ch[i]), np.zeros(H)) for i in seqs])
        choice[j] = np.argmin(ghat, axis=0)
        V[j] = ghat.min(axis=0)
    q = np.zeros((S, H))
    for j in _top_down(tpx):
        qp = _parent_mass(tpx, q, j)
        seqs = tpx.infoset_seqs[j]
        for a, i in enumerate(seqs):
            q[i] = qp * (choice[j] == a)
    per_hand = sum(V[j] for j in tpx.roots())
    return q, float(per_hand.sum()), per_hand


def conj_grad(tpx: Treeplex, s: np.ndarray, beta=None) -> np.ndarray:
    """grad d*(s) = argmax_q <s, q> - d(q) = argmin <-s, q> + d(q) (Sec. 3)."""
    q, _, _ = smoothed_br(tpx, -s, 1.0, beta)
    return q


def prox_shift_constant(tpx: Treeplex, n_hands: int, beta=None) -> float:
    """Appendix A: -d(q) + <grad d(q), q> = -sum over root simplexes of beta_j (log n_j - 1)."""
    beta = weights(tpx) if beta is None else beta
    return -n_hands * sum(beta[j] * (np.log(len(tpx.infoset_seqs[j])) - 1.0) for j in tpx.roots())


def is_in_treeplex(tpx: Treeplex, q: np.ndarray, tol=1e-12) -> bool:
    """Sequence-form constraints: q >= 0, each simplex sums to its parent variable (root: 1)."""
    if (q < -tol).any():
        return False
    for j in range(tpx.n_infosets):
        qp = _parent_mass(tpx, q, j)
        if np.abs(q[tpx.infoset_seqs[j]].sum(axis=0) - qp).max() > tol:
            return False
    return True
