"""EGT/as pinned late in a solve: one Decr (Alg. 4) from the GPU's own state, stage by stage.

Comparing whole EGT/as trajectories cannot pin the small-mu arithmetic: mu
shrinks fast, the smoothed best responses become ill conditioned (kappa =
max |g_hat| / (mu beta) passes 1e3 after 100 iterations and 1e5 near 1
mbb/hand), and FP32 rounding, amplified by about kappa tau at each Step stage,
moves a trajectory far more than the arithmetic of any one stage.  Instead the
GPU runs to iteration t (100, 1000, the first iteration past 100 whose Decr
backs off, and the last iteration before its residual reaches 1 mbb/hand), and
from that state, which both sides then share exactly, one Decr is checked:

* each attempt tau_k = tau 2^-k of the Decr is run as a Step (egt_step), and
  each of its three SBR stages is compared element-wise with the oracle's stage
  computed from the GPU's own input to that stage -- x_hat (egt_step_point),
  y_+, x_+ -- within that stage's bound (``tests/bounds.py``): the product and
  the SBR at mu_x, at mu_y and at (1 - tau) mu_x, with tau and the mixing;
* the GPU's EGV of each attempt equals the oracle's EGV at the GPU's point
  within the bound of the two SBR values it is made of, so wherever the EGV is
  further from 0 than that bound the GPU takes the paper's decision (accept, or
  halve tau);
* the device-resident driver (the benchmark's kernel), run for one iteration
  from the same state, takes the same back-offs, tau and mu and ends on the
  same iterates, bit for bit, as the attempts run one by one;
* the FP64 residual of the new state equals the oracle's eps_sad of the GPU's
  iterates to 1e-9;
* the oracle's own Decr from the same state, FP64 throughout, takes the same
  number of back-offs.
"""
import numpy as np
import pytest

from oracle import egt as OE
from oracle import payoff
from paper_1810_03063_b300 import synth
from tests import bounds as B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPECS = {"tiny": synth.tiny, "full": synth.full_deck, "large": synth.large}
_CACHE = {}


@pytest.fixture(scope="module")
def egtlib():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_1810_03063_b300 import egt
    return egt


def game(name, egtlib):
    if name not in _CACHE:
        spec = SPECS[name]()
        og = payoff.make_game(spec)
        g = egtlib.Game(spec, device=0)
        rep = g.solve(variant=egtlib.EGT_AS, alpha=0.01, eps_mbb=1.0, max_iters=30000, gap_every=1,
                      log_cap=30000)
        assert rep["status"] == "EGT_OK", rep
        # the first iteration past 100 whose Decr backed off (its state is where Decr halves tau)
        t_back = next(e["t"] for e in rep["log"] if e["t"] >= 100 and e["backoffs"] > 0)
        _CACHE[name] = (spec, og, OE.Problem(og), g, rep["iters"], t_back)
    return _CACHE[name]


def vec(g, player):
    return torch.empty((g.S[player], g.ld), device="cuda")


def host(g, t):
    torch.cuda.synchronize()
    return g.unpack(t.double().cpu().numpy())


def check_stage(name, got, ref, bound):
    err = np.abs(got - ref)
    worst = float((err / bound).max())
    assert worst <= 1.0, f"{name}: error / bound = {worst:.3g} (max error {err.max():.3g})"
    return worst


@pytest.mark.parametrize("name", ["tiny", "full", "large"])
@pytest.mark.parametrize("when", ["t100", "t1000", "last", "backoff"])
def test_one_decr_from_gpu_state(egtlib, name, when):
    spec, og, P, g, n_solve, t_back = game(name, egtlib)
    t = {"t100": 100, "t1000": 1000, "last": n_solve - 1, "backoff": t_back}[when]
    g.solver_init(variant=egtlib.EGT_AS, alpha=0.01)
    g.iterate(t, variant=egtlib.EGT_AS, eps_mbb=0.0, gap_every=t)
    x, y = vec(g, 0), vec(g, 1)
    ck = g.checkpoint(x, y)
    assert ck["t"] == t
    xs, ys = host(g, x), host(g, y)
    mux, muy = ck["mu"]
    me = 0 if mux > muy else 1
    other = 1 - me
    mu_me, mu_o = (mux, muy) if me == 0 else (muy, mux)
    v_me, v_o = (xs, ys) if me == 0 else (ys, xs)

    # the benchmark's kernel: one EGT/as iteration of the device-resident driver
    eng = g.iterate(1, variant=egtlib.EGT_AS, eps_mbb=0.0, gap_every=1)
    xe, ye = vec(g, 0), vec(g, 1)
    mu_e = g.state_get(xe, ye)

    # the same Decr attempt by attempt, each stage against the oracle from the GPU's inputs
    worst = {}
    k = 0
    while True:
        tau_k = ck["tau"] * 0.5 ** k
        g.restore(x, y, ck)
        info = g.step(-1, tau_k, mode=egtlib.STEP_CHECK)
        assert info["player"] == me
        if not info["accepted"]:
            g.restore(x, y, ck)
            g.step(-1, tau_k, mode=egtlib.STEP_PLAIN)           # the same attempt, kept
        xp, yp, vh = vec(g, 0), vec(g, 1), vec(g, me)
        g.state_get(xp, yp)
        assert g.step_point(vh) == me
        xp_h, yp_h, vhat = host(g, xp), host(g, yp), host(g, vh)
        vm_plus, vo_plus = (xp_h, yp_h) if me == 0 else (yp_h, xp_h)

        a = B.stage(P, og, me, v_o, mu_me, v_me, tau_k)                 # v_hat
        worst["v_hat"] = check_stage("v_hat", vhat, a["v"], a["dv"])
        b = B.stage(P, og, other, vhat, mu_o, v_o, tau_k)               # other_+
        worst["other_plus"] = check_stage("other_+", vo_plus, b["v"], b["dv"])
        c = B.stage(P, og, me, vo_plus, (1.0 - tau_k) * mu_me, v_me, tau_k)   # me_+
        worst["me_plus"] = check_stage("me_+", vm_plus, c["v"], c["dv"])
        d = B.stage(P, og, other, vm_plus, mu_o, None, tau_k)           # other's value at me_+
        egv_ref, egv_tol = c["val"] + d["val"], c["dval"] + d["dval"]
        assert abs(info["egv"] - egv_ref) <= egv_tol, (info["egv"], egv_ref, egv_tol)
        if abs(egv_ref) > egv_tol:
            assert info["accepted"] == (egv_ref >= 0)
        assert info["accepted"] == (info["egv"] >= 0)
        if info["accepted"]:
            break
        k += 1
        assert k < 30

    if when == "backoff":
        assert k >= 1
    # the driver took the same decisions and ended on the same point
    assert eng["backoffs"] == k and eng["tau"] == tau_k, (eng, k, tau_k)
    assert mu_e == info["mu"] and info["mu"][me] == (1.0 - tau_k) * mu_me
    assert torch.equal(xe, xp) and torch.equal(ye, yp)

    # the FP64 residual of the new state
    gap = g.state_gap()
    ref_gap = P.to_mbb(P.eps_sad(xp_h, yp_h))
    assert abs(gap - ref_gap) <= 1e-9 * abs(ref_gap)

    # the oracle's own Decr from the same state, FP64 throughout
    *_, tau_o, attempts = OE.decr(P, me, mux, muy, xs, ys, ck["tau"])
    assert len(attempts) - 1 == k and tau_o == tau_k, (attempts, k)
    print(f"{name} t={t}: player {me}, tau {tau_k:.3g}, back-offs {k}, kappa {c['kappa']:.3g}, "
          f"error/bound {worst}, EGV {info['egv']:.3g} (oracle {egv_ref:.3g} +- {egv_tol:.2g}), "
          f"oracle Decr EGVs {[f'{e:.3g}' for _, e in attempts]}")
