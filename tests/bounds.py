"""Error bounds of the FP32 GPU path against the FP64 oracle (test helpers).

All bounds are element-wise and follow the arithmetic (eps32 = 2^-24):

* product (63-bit fixed-point sums, exact, rounded once, then scaled):
  |err(A v)_i| <= 8 eps32 (|A| |v|)_i + floor_i, and an input error dv adds (|A| dv)_i;
* smoothed best response, FP32 rounding inside (exponent arguments carry an
  absolute error of a few eps32 times kappa = max |g_hat| / t, so each factor
  q_bar of q has a relative error of at most (8 kappa + 16) eps32):
  |dq| <= q expm1(L (8 kappa + 16) eps32), value |dV| <= 16 eps32 mag;
* smoothed best response, input error dg: log-sum-exp is 1-Lipschitz in the
  max norm, so at simplex j |d log q_bar_i| <= 2 max_k |d g_hat_k| / t_j and
  |d V_j| <= max_k |d g_hat_k|; q is the product of its ancestors' q_bar, so
  |dq| <= q (exp(sum of the path's |d log q_bar|) - 1) exactly, and the value
  moves by at most max over the treeplex of <q, |dg|> (a best response to |dg|);
* mixing (1 - tau) old + tau q in FP32: <= 4 eps32 (|old| + tau |q|).

``stage`` is one SBR stage of a Step (Alg. 2) taken from an input both sides
share exactly (a vector the GPU produced), so no error is carried from one
stage to the next: a Step at small mu amplifies FP32 rounding by about
kappa tau per stage, which makes a bound carried through a whole Step vacuous
late in a solve, while each stage on its own stays well conditioned.
"""
from __future__ import annotations

import numpy as np

from oracle import egt as OE
from oracle import treeplex as OT

EPS32 = 2.0 ** -24


def abs_apply(og, v, player):
    """(|A| v) for player 0 (v over y's sequences) or (|A|^T v) for player 1, by grouped GEMMs.

    |block_b| is |coef_b| P for a fold and |coef_b| (P o |sign|) for a showdown."""
    term = og.sf.terminals
    out = np.zeros((og.S[player], og.H))
    for kind, M in (("fold", og.P), ("showdown", og.P * np.abs(og.sign))):
        idx = [b for b, t in enumerate(term) if (t.kind == "fold") == (kind == "fold")]
        if not idx:
            continue
        src = np.array([term[b].seq[1 - player] for b in idx])
        dst = np.array([term[b].seq[player] for b in idx])
        c = np.abs(og.coef[idx])
        Mm = M if player == 0 else M.T
        res = (Mm @ v[src].T) * c[None, :]
        np.add.at(out, dst, res.T)
    return out


def fixed_point_floor(og, vec, player):
    """Absolute error floor of the products.  Each term r_opp v_opp enters its column's
    sums as an integer at the column scale 2^ex (|w| 2^ex < 2^52), off by at most 1.5
    units of 2^-ex <= 2^-50 of the column's largest |w| besides a relative 2^-47 (the
    integer sums are exact; the terms the card-removal algebra cancels cancel exactly), so
    an output built from at most H terms is off by at most H 1.5 2^-50 max|w|.  Bounded
    here by |coef_b| max(r_me) max(r_opp) / Z max|v_opp| H 2^-49 per output row."""
    r = og.spec.ranges
    out = np.zeros((og.S[player], og.H))
    for b, t in enumerate(og.sf.terminals):
        scale = abs(og.coef[b]) * r[player].max() * r[1 - player].max() / og.Z
        out[t.seq[player]] += scale * np.abs(vec[t.seq[1 - player]]).max() * og.H * 2.0 ** -49
    return out


def product_bound(og, v, dv, player):
    """Bound on |GPU(A v_gpu) - A v| for |v_gpu - v| <= dv (player 0: A y, player 1: A^T x)."""
    av = np.abs(v) + dv
    return 8 * EPS32 * abs_apply(og, av, player) + fixed_point_floor(og, av, player) + abs_apply(og, dv, player)


def sbr_conditioning(P, player, loss, mu):
    """(kappa, mag): kappa[h] = max over simplexes of |g_hat| / t for hand h (the absolute
    error of an FP32 exponent argument is a few eps32 times it); mag = sum over simplexes and
    hands of |min g_hat| + |V_j| (the size of the terms the FP32 value is built from)."""
    tpx, beta = P.tpx[player], P.beta[player]
    ch = tpx.children()
    V = np.zeros((tpx.n_infosets, loss.shape[1]))
    kappa = np.zeros(loss.shape[1])
    mag = 0.0
    for j in sorted(range(tpx.n_infosets), key=lambda j: -tpx.infoset_level[j]):
        gh = np.stack([loss[i] + sum((V[k] for k in ch[i]), 0) for i in tpx.infoset_seqs[j]])
        t = mu * beta[j]
        kappa = np.maximum(kappa, np.abs(gh).max(0) / t)
        m = gh.min(0)
        V[j] = m - t * np.log(np.exp(-(gh - m) / t).sum(0)) + t * np.log(len(tpx.infoset_seqs[j]))
        mag += float(np.abs(m).sum() + np.abs(V[j]).sum())
    return kappa, mag


def sbr_input_sensitivity(P, player, mu, dloss):
    """(dlq, dval): bound on |d log q| per (sequence, hand) and on the value when the SBR's
    input moves by at most dloss element-wise."""
    tpx, beta = P.tpx[player], P.beta[player]
    ch = tpx.children()
    H = dloss.shape[1]
    dV = np.zeros((tpx.n_infosets, H))
    dlqbar = np.zeros_like(dloss)
    for j in sorted(range(tpx.n_infosets), key=lambda j: -tpx.infoset_level[j]):
        seqs = tpx.infoset_seqs[j]
        dgh = np.stack([dloss[i] + sum((dV[k] for k in ch[i]), np.zeros(H)) for i in seqs])
        m = dgh.max(0)
        dV[j] = m
        dlqbar[seqs] = 2.0 * m / (mu * beta[j])
    dlq = np.zeros_like(dloss)
    for j in sorted(range(tpx.n_infosets), key=lambda j: tpx.infoset_level[j]):
        p = tpx.infoset_parent[j]
        for i in tpx.infoset_seqs[j]:
            dlq[i] = dlqbar[i] + (dlq[p] if p >= 0 else 0.0)
    _, v, _ = OT.best_response(tpx, -dloss)               # max over Q of <q, dloss>
    return dlq, -v


def sbr_with_bound(P, player, loss, mu, dloss):
    """Oracle SBR of ``loss`` (the minimised gradient) and the bounds of the GPU's FP32 SBR
    of an input within dloss of it: (q, value, dq, dval, kappa).

    q is the product of L factors q_bar, each with a relative error of at most
    (8 kappa_h + 16) eps32 from FP32 rounding plus 2 max |d g_hat| / t from the input, so
    |dq| <= q expm1(L (8 kappa_h + 16) eps32 + dlq)."""
    q, val, _ = OT.smoothed_br(P.tpx[player], loss, mu, P.beta[player])
    kappa, mag = sbr_conditioning(P, player, loss, mu)
    L = max(P.tpx[player].infoset_level) + 1
    dlq, dv_in = sbr_input_sensitivity(P, player, mu, dloss)
    rel = L * (8 * kappa[None, :] + 16) * EPS32 + dlq
    dq = np.minimum(q * np.expm1(np.minimum(rel, 700.0)) + 2.0 ** -100, 1.0)   # + FP32 underflow
    dval = 16 * EPS32 * mag + dv_in
    return q, val, dq, dval, float(kappa.max())


def mix_bound(old, q, dq, tau):
    """|d((1 - tau) old + tau q)| for a q within dq, computed in FP32."""
    return tau * dq + 4 * EPS32 * (np.abs(old) + tau * np.abs(q))


def loss_of(og, player, other):
    """Loss gradient of ``player`` at the other's iterate: A y (x) or -A^T x (y)."""
    return og.Ay(other) if player == 0 else -og.Atx(other)


def stage(P, og, player, other, mu, old, tau):
    """One SBR stage of a Step from a shared input: the oracle's (1 - tau) old + tau
    SBR_player(loss(other), mu) (or the SBR alone when old is None) with its bound, and the
    SBR's value with its bound.  Returns dict(v, dv, val, dval, kappa)."""
    g = loss_of(og, player, other)
    dg = product_bound(og, other, np.zeros_like(other), player)
    q, val, dq, dval, kappa = sbr_with_bound(P, player, g, mu, dg)
    if old is None:
        return dict(v=q, dv=dq, val=val, dval=dval, kappa=kappa)
    return dict(v=(1.0 - tau) * old + tau * q, dv=mix_bound(old, q, dq, tau), val=val, dval=dval,
                kappa=kappa)


def fp32_noise_floor(P, mu0, schedule, seed=0, variant="egt_as"):
    """The oracle's own trajectory when every product is perturbed by FP32-sized noise
    (relative 2^-24, iterates rounded to FP32) and the schedule is replayed: how far any FP32
    run of the same decisions may drift."""
    orig = P.loss_grad
    rng = np.random.default_rng(seed)

    def noisy(player, other):
        gv = orig(player, other.astype(np.float32).astype(np.float64))
        return (gv * (1 + EPS32 * rng.uniform(-1, 1, gv.shape))).astype(np.float32).astype(np.float64)

    P.loss_grad = noisy
    try:
        return OE.solve(P, variant=variant, eps_mbb=0.0, max_iters=len(schedule), mu0=mu0,
                        gap_every=10 ** 6, replay=schedule)
    finally:
        P.loss_grad = orig
