"""O7-O8: EGT drivers (Algorithms 1-4), excessive gap and saddle-point residual (oracle, FP64).

Sec. 3 notation.  x (player 1) minimises <x, Ay>, y (player 2) maximises it.

  f_{mu_y}(x)   = max_y <x, Ay> - mu_y d_Y(y)     attained at y_{mu_y}(x)
  phi_{mu_x}(y) = min_x <x, Ay> + mu_x d_X(x)     attained at x_{mu_x}(y)
  EGV(x, y)     = phi_{mu_x}(y) - f_{mu_y}(x)
  eps_sad(x, y) = max_y' x^T A y' - min_x' x'^T A y

Smoothed best responses: x_{mu}(y) = SBR_X(A y, mu) and
y_{mu}(x) = argmin_y <y, -A^T x> + mu d_Y(y) = SBR_Y(-A^T x, mu), so that
phi = value(SBR_X) and f = -value(SBR_Y).

Every product is recomputed from the current iterates (no caching) and
counted in ``products``.

Readings where the paper is silent or garbled (each one a test below):

* Alg. 1 / 3 first line: x^0 = grad d*(-mu_x^{-1} grad f_{mu_y}(x_omega)), the
  minus sign restored (grad d* is an argmax, the minimiser needs -grad f).
* x_omega = uniform behavioural strategy (d = 0 there, the DGF centre).
* Theory mu: mu_x = mu_y = ||A|| sqrt(M_X M_Y) = ||A|| / sqrt(phi_X phi_Y).
* "Practically tuned" mu: alpha times the theory value, doubled while EGV < 0
  at the initial point.
* Alg. 4 checks EGV at the new point (mu_x^+, mu_y, x^+, y^+); retries restart
  from the same (x, y); tau never increases; tau < 2^-30 is an error.
* Practical EGT: tau_t = 2 / (t + 3) with mu balancing; a tie mu_x = mu_y
  steps y (the else branch of Alg. 3).
* y-focused Step = Alg. 2 with the roles swapped and A replaced by -A^T.
* 1 mbb = bb / 1000 (bb is a game input); chance is normalised by Z so the
  residual is per hand dealt.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import treeplex as T
from .game import uniform_behavioural

TAU_MIN = 2.0 ** -30


class Problem:
    """A game from ``oracle.payoff`` plus the DGF quantities of both treeplexes."""

    def __init__(self, game):
        self.game = game
        self.H = game.H
        self.tpx = game.tpx
        self.beta = tuple(T.weights(t) for t in self.tpx)
        self.M = tuple(self.H * T.max_l1(t) for t in self.tpx)        # l1 bound of the full space
        self.Omega = tuple(self.H * T.omega(t, b) for t, b in zip(self.tpx, self.beta))
        self.normA = game.norm_A()
        self.products = 0

    # gradients of each player's loss (x: A y, y: -A^T x)
    def loss_grad(self, player, other):
        self.products += 1
        return self.game.Ay(other) if player == 0 else -self.game.Atx(other)

    def sbr(self, player, other, mu):
        """Smoothed best response of ``player`` to the other player's ``other``; (q, value)."""
        q, val, _ = T.smoothed_br(self.tpx[player], self.loss_grad(player, other), mu, self.beta[player])
        return q, val

    def egv(self, x, y, mux, muy):
        """EGV(x, y) = phi_{mu_x}(y) - f_{mu_y}(x) = value(SBR_X(Ay)) + value(SBR_Y(-A^T x))."""
        _, phi = self.sbr(0, y, mux)
        _, negf = self.sbr(1, x, muy)
        return phi + negf

    def eps_sad(self, x, y):
        """max_y' x^T A y' - min_x' x'^T A y via the plain best responses."""
        _, vy, _ = T.best_response(self.tpx[1], self.loss_grad(1, x))   # min_y <y, -A^T x>
        _, vx, _ = T.best_response(self.tpx[0], self.loss_grad(0, y))   # min_x <x, A y>
        return -vy - vx

    def to_mbb(self, v):
        return v / self.game.spec.bb * 1000.0

    def theory_mu(self):
        return self.normA * math.sqrt(self.M[0] * self.M[1])


def step(P: Problem, me: int, mu_me: float, mu_other: float, v_me, v_other, tau: float,
         prox: str = "closed"):
    """Alg. 2 Step focused on player ``me``: returns (mu_me^+, v_me^+, v_other^+).

    Written for me = x; for me = y the same lines run with the roles swapped
    (A -> -A^T), which is what ``loss_grad`` / ``sbr`` do.
    """
    other = 1 - me
    s, _ = P.sbr(me, v_other, mu_me)                         # x_{mu_x}(y)
    v_hat = (1.0 - tau) * v_me + tau * s                     # x_hat
    o, _ = P.sbr(other, v_hat, mu_other)                     # y_{mu_y}(x_hat)
    v_other_plus = (1.0 - tau) * v_other + tau * o           # y_+
    if prox == "literal":
        # x_tilde = grad d*( grad d(x_{mu_x}(y)) - tau / ((1 - tau) mu_x) grad f_{mu_y}(x_hat) ),
        # grad f_{mu_y}(x_hat) = A y_{mu_y}(x_hat)
        grad_f = P.loss_grad(me, o)
        arg = T.grad_dgf(P.tpx[me], s, P.beta[me]) - tau / ((1.0 - tau) * mu_me) * grad_f
        v_tilde = T.conj_grad(P.tpx[me], arg, P.beta[me])
    elif prox == "closed":
        # same point, from the optimality condition of x_{mu_x}(y): grad d(x_{mu_x}(y)) equals
        # -A y / mu_x up to a term constant on X, so x_tilde = x_{(1-tau) mu_x}(y_+)
        v_tilde, _ = P.sbr(me, v_other_plus, (1.0 - tau) * mu_me)
    else:
        raise ValueError(prox)
    v_me_plus = (1.0 - tau) * v_me + tau * v_tilde           # x_+
    return (1.0 - tau) * mu_me, v_me_plus, v_other_plus


def decr(P: Problem, me: int, mux: float, muy: float, x, y, tau: float, prox: str = "closed"):
    """Alg. 4 Decr focused on player ``me``: Step at tau, halving tau while the excessive gap
    condition fails at the new point (reading: EGV of (x^+, y^+) with mu_me^+ and the other
    player's unchanged mu; every retry starts again from (x, y)).

    Returns (mux^+, muy^+, x^+, y^+, tau, attempts) with attempts = [(tau_k, EGV_k)] in order.
    """
    mu_me, mu_other = (mux, muy) if me == 0 else (muy, mux)
    v_me, v_other = (x, y) if me == 0 else (y, x)
    attempts = []
    while True:
        mu_me_p, v_me_p, v_other_p = step(P, me, mu_me, mu_other, v_me, v_other, tau, prox)
        xx, yy = (v_me_p, v_other_p) if me == 0 else (v_other_p, v_me_p)
        mx, my = (mu_me_p, mu_other) if me == 0 else (mu_other, mu_me_p)
        egv = P.egv(xx, yy, mx, my)
        attempts.append((tau, egv))
        if egv >= 0:
            return mx, my, xx, yy, tau, attempts
        tau *= 0.5
        if tau < TAU_MIN:
            raise FloatingPointError("tau underflow in Decr")


def initial_point(P: Problem, mux: float, muy: float):
    """Alg. 1 / 3 first two lines (sign reading in the module docstring)."""
    x_omega = uniform_behavioural(P.tpx[0], P.H)
    y0, _ = P.sbr(1, x_omega, muy)                          # y^0 = y_{mu_y}(x_omega)
    grad_f = P.loss_grad(0, y0)                             # grad f_{mu_y}(x_omega) = A y_{mu_y}(x_omega)
    x0 = T.conj_grad(P.tpx[0], -grad_f / mux, P.beta[0])    # grad d*(-mu_x^{-1} grad f)
    return x0, y0


@dataclass
class Result:
    x: np.ndarray
    y: np.ndarray
    mux: float
    muy: float
    iters: int
    gap_mbb: float
    products: int
    backoffs: int
    log: list = field(default_factory=list)
    schedule: list = field(default_factory=list)    # accepted (player, tau) per iteration


def solve(P: Problem, variant: str = "egt_as", alpha: float = 0.01, eps_mbb: float = 1.0,
          max_iters: int = 1000, prox: str = "closed", replay=None, mu0=None,
          gap_every: int = 1, log_egv: bool = False) -> Result:
    """Alg. 1 (variant 'theory'), practical EGT ('egt') or Alg. 3 / 4 ('egt_as').

    ``replay``: list of (player, tau) to follow instead of the schedule (no EGV check).
    ``mu0``: (mu_x, mu_y) initial smoothing, bypassing the choice and the guard.
    """
    if mu0 is not None:
        mux, muy = mu0
    elif variant == "theory":
        mux = muy = P.theory_mu()
    else:
        mux = muy = alpha * P.theory_mu()
    x, y = initial_point(P, mux, muy)
    if mu0 is None and variant != "theory":
        while P.egv(x, y, mux, muy) < 0:
            mux, muy = 2.0 * mux, 2.0 * muy
            x, y = initial_point(P, mux, muy)
    res = Result(x, y, mux, muy, 0, float("nan"), 0, 0)
    t, tau, backoffs = 0, 0.5, 0
    gap = float("inf")
    while True:
        if t % gap_every == 0 or t >= max_iters:
            gap = P.to_mbb(P.eps_sad(x, y))
        if gap <= eps_mbb or t >= max_iters or (replay is not None and t >= len(replay)):
            break
        if replay is not None:
            me, tau_t = replay[t]
        elif variant == "theory":
            me, tau_t = (0 if t % 2 == 0 else 1), 2.0 / (t + 3)
        else:
            me = 0 if mux > muy else 1
            tau_t = 2.0 / (t + 3) if variant == "egt" else tau
        if variant == "egt_as" and replay is None:
            # Alg. 4 Decr: halve tau until the excessive gap condition holds at the new point
            mux, muy, x, y, tau_t, attempts = decr(P, me, mux, muy, x, y, tau_t, prox)
            backoffs += len(attempts) - 1
            tau = tau_t
        else:
            mu_me, mu_other = (mux, muy) if me == 0 else (muy, mux)
            v_me, v_other = (x, y) if me == 0 else (y, x)
            mu_me_p, v_me_p, v_other_p = step(P, me, mu_me, mu_other, v_me, v_other, tau_t, prox)
            if me == 0:
                mux, x, y = mu_me_p, v_me_p, v_other_p
            else:
                muy, y, x = mu_me_p, v_me_p, v_other_p
        res.schedule.append((me, tau_t))
        entry = dict(t=t, player=me, tau=tau_t, mux=mux, muy=muy, gap_mbb=gap, products=P.products)
        if log_egv:
            entry["egv"] = P.egv(x, y, mux, muy)
        res.log.append(entry)
        t += 1
    res.x, res.y, res.mux, res.muy = x, y, mux, muy
    res.iters, res.gap_mbb, res.products, res.backoffs = t, gap, P.products, backoffs
    return res
