"""O2: sequence-form payoff matrix A and the products A y, A^T x (oracle, FP64).

Eq. 1 / Eq. 2 of the paper: Nash equilibrium = min_x max_y <x, A y> with A
the sequence-form payoff matrix.  Here x is player 1 (the minimiser) and A
holds the expected payoff *to player 2*:

    A[(s1, h1), (s2, h2)] = sum over terminals b with sigma_1(b) = s1 and
                            sigma_2(b) = s2 of p(h1, h2) * u_b(h1, h2)

with p(h1, h2) = r1(h1) r2(h2) [h1, h2 share no card] / Z the chance
probability and u_b the payoff to player 2 at b.  Every entry comes from a
brute-force loop over terminals and hand pairs; no prefix sums, no card
removal algebra.

``DenseGame`` materialises A (small games).  ``FactoredGame`` keeps, for
every terminal b, the H x H block M_b = [p(h1, h2) u_b(h1, h2)] in the
Kronecker form A = sum_b e_{sigma1(b)} e_{sigma2(b)}^T (x) M_b, where only two
H x H matrices exist: P (chance) and P o sign(s2 - s1); fold blocks are
u_b P and showdown blocks are stake_b (P o sign).  Products are plain GEMMs.
"""
from __future__ import annotations

import numpy as np

from . import game as G


class _Base:
    def __init__(self, spec):
        self.spec = spec
        self.sf = G.sequence_form(spec.pot, spec.stack, spec.bet_fracs, spec.allin, spec.raise_cap,
                                  getattr(spec, "menus", None))
        self.tpx = self.sf.tpx
        self.H = spec.n_hands
        self.S = (self.tpx[0].n_seq, self.tpx[1].n_seq)
        self.P, self.C, self.Z = G.chance(spec)
        s = np.asarray(spec.strength, dtype=np.float64)
        self.sign = np.sign(s[None, :] - s[:, None])          # sign(s2 - s1), rows h1, cols h2
        self.coef = np.array([self._coef(t) for t in self.sf.terminals])

    def _coef(self, t):
        """Payoff magnitude: u_b for a fold, the stake for a showdown."""
        if t.kind == "fold":
            return G.terminal_payoff_to_p2(t, self.spec.pot, 0.0, 0.0)
        return self.spec.pot / 2 + t.contrib[0]

    def block(self, b):
        """M_b = [p(h1, h2) u_b(h1, h2)]_{h1, h2}."""
        t = self.sf.terminals[b]
        if t.kind == "fold":
            return self.coef[b] * self.P
        return self.coef[b] * (self.P * self.sign)

    def norm_A(self):
        """l1 -> l_inf operator norm of A = max_ij |A_ij| (each entry is one (b, h1, h2))."""
        return max(np.abs(self.block(b)).max() for b in range(len(self.sf.terminals)))

    def value(self, x, y):
        return float(np.sum(x * self.Ay(y)))


class DenseGame(_Base):
    """A materialised as an (S1*H) x (S2*H) matrix, row (s1, h1) = s1 * H + h1."""

    def __init__(self, spec):
        super().__init__(spec)
        H = self.H
        A = np.zeros((self.S[0] * H, self.S[1] * H))
        for b, t in enumerate(self.sf.terminals):
            s1, s2 = t.seq
            for h1 in range(H):
                for h2 in range(H):
                    p = self.P[h1, h2]
                    if p == 0.0:
                        continue
                    u = G.terminal_payoff_to_p2(t, self.spec.pot, float(self.spec.strength[h1]),
                                                float(self.spec.strength[h2]))
                    A[s1 * H + h1, s2 * H + h2] += p * u
        self.A = A

    def Ay(self, y):
        return (self.A @ y.reshape(-1)).reshape(self.S[0], self.H)

    def Atx(self, x):
        return (self.A.T @ x.reshape(-1)).reshape(self.S[1], self.H)


class FactoredGame(_Base):
    """A kept as per-terminal H x H blocks (see module docstring)."""

    def Ay(self, y):
        out = np.zeros((self.S[0], self.H))
        for b, t in enumerate(self.sf.terminals):
            s1, s2 = t.seq
            out[s1] += self.block(b) @ y[s2]
        return out

    def Atx(self, x):
        out = np.zeros((self.S[1], self.H))
        for b, t in enumerate(self.sf.terminals):
            s1, s2 = t.seq
            out[s2] += self.block(b).T @ x[s1]
        return out


class BatchedFactoredGame(FactoredGame):
    """Same products as FactoredGame, grouped into two GEMMs (fold / showdown blocks).

    sum over b of u_b P y[sigma2(b)] = P @ Y_fold @ diag(u) scattered by sigma1;
    used for the large games where a loop over 677 terminals of H x H
    matrix-vector products is slow.  Identical arithmetic definition.
    """

    def __init__(self, spec):
        super().__init__(spec)
        term = self.sf.terminals
        self.fold = np.array([b for b, t in enumerate(term) if t.kind == "fold"], dtype=np.int64)
        self.sd = np.array([b for b, t in enumerate(term) if t.kind != "fold"], dtype=np.int64)
        self.sig = np.array([t.seq for t in term], dtype=np.int64)
        self.PS = self.P * self.sign

    def _prod(self, M, vec, idx, src, dst, n_out):
        if len(idx) == 0:
            return np.zeros((n_out, self.H))
        cols = vec[self.sig[idx, src]].T                   # H x nb
        res = (M @ cols) * self.coef[idx][None, :]         # H x nb
        out = np.zeros((n_out, self.H))
        np.add.at(out, self.sig[idx, dst], res.T)
        return out

    def Ay(self, y):
        return (self._prod(self.P, y, self.fold, 1, 0, self.S[0])
                + self._prod(self.PS, y, self.sd, 1, 0, self.S[0]))

    def Atx(self, x):
        return (self._prod(self.P.T, x, self.fold, 0, 1, self.S[1])
                + self._prod(self.PS.T, x, self.sd, 0, 1, self.S[1]))


def make_game(spec, kind="auto"):
    if kind == "dense" or (kind == "auto" and spec.n_hands <= 128):
        return DenseGame(spec)
    if kind == "factored":
        return FactoredGame(spec)
    return BatchedFactoredGame(spec)
