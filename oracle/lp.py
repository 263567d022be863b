"""Sequence-form linear programs (Sec. 1, the von Stengel LP) -- an independent pin.

Used only to check the oracle: it never calls the best-response or SBR code.

Treeplex constraints per hand: for every simplex j, sum_{i in I_j} q_i - q_{p_j} = [j is a root].
``game_value``: min_x max_y <x, Ay>; the inner max over Y is replaced by its LP
dual min f^T v s.t. F^T v >= A^T x, giving one LP in (x, v).
``best_response_lp``: max_y <x, Ay> or min_x <x, Ay> as a plain LP.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.optimize import linprog


def constraints(tpx, H):
    """(E, e) with E q = e the sequence-form constraints of the H-fold product, q = [seq][hand]."""
    S, J = tpx.n_seq, tpx.n_infosets
    rows, cols, vals = [], [], []
    e = np.zeros(J * H)
    for j in range(J):
        for h in range(H):
            r = j * H + h
            for i in tpx.infoset_seqs[j]:
                rows.append(r); cols.append(i * H + h); vals.append(1.0)
            p = tpx.infoset_parent[j]
            if p >= 0:
                rows.append(r); cols.append(p * H + h); vals.append(-1.0)
            else:
                e[r] = 1.0
    E = sp.csr_matrix((vals, (rows, cols)), shape=(J * H, S * H))
    return E, e


def _A(game):
    if hasattr(game, "A"):
        return sp.csr_matrix(game.A)
    H = game.H
    blocks = sp.lil_matrix((game.S[0] * H, game.S[1] * H))
    for b, t in enumerate(game.sf.terminals):
        s1, s2 = t.seq
        blocks[s1 * H:(s1 + 1) * H, s2 * H:(s2 + 1) * H] += game.block(b)
    return blocks.tocsr()


def game_value(game):
    """Value of min_x max_y <x, Ay> and an optimal x (reshaped [S1][H])."""
    A = _A(game)
    H = game.H
    E, e = constraints(game.tpx[0], H)
    F, f = constraints(game.tpx[1], H)
    nx, nv = A.shape[0], F.shape[0]
    c = np.concatenate([np.zeros(nx), f])
    # A^T x - F^T v <= 0
    A_ub = sp.hstack([A.T, -F.T]).tocsr()
    b_ub = np.zeros(A.shape[1])
    A_eq = sp.hstack([E, sp.csr_matrix((E.shape[0], nv))]).tocsr()
    bounds = [(0, None)] * nx + [(None, None)] * nv
    res = linprog(c, A_ub=A_ub, b_ub=b_ub, A_eq=A_eq, b_eq=e, bounds=bounds, method="highs")
    if res.status != 0:
        raise RuntimeError(res.message)
    return float(res.fun), res.x[:nx].reshape(game.S[0], H)


def best_response_lp(game, player, other):
    """player 1 (index 1): max_y <x, Ay> for x = other; player 0: min_x <x, Ay> for y = other."""
    A = _A(game)
    H = game.H
    if player == 1:
        c = -(A.T @ other.reshape(-1))
        E, e = constraints(game.tpx[1], H)
        res = linprog(c, A_eq=E, b_eq=e, bounds=(0, None), method="highs")
        return -float(res.fun)
    c = A @ other.reshape(-1)
    E, e = constraints(game.tpx[0], H)
    res = linprog(c, A_eq=E, b_eq=e, bounds=(0, None), method="highs")
    return float(res.fun)
