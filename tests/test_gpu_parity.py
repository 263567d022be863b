"""GPU parity: every C-ABI call against the FP64 oracle on the same seeded inputs.

Tolerances are derived from the arithmetic (eps32 = 2^-24, eps64 = 2^-53):

* FP32 product: each term w = r_opp y enters its column's 63-bit fixed-point sums
  within 2^-47 |w| + 1.5 units of the column scale (`fixed_point_floor`: 1.5 units
  are at most 2^-50 of the column's largest term), the integer sums are exact and
  rounded once, then scaled and the sequence's one or two terminals added:
  |err_i| <= 8 eps32 (|A| |y|)_i + floor.
* FP64 product: the same sums rounded to FP64; the terms' relative 2^-47 dominates
  its rounding: |err_i| <= 128 eps64 (|A| |y|)_i + floor.
* FP32 SBR: an exponent argument (g_hat - m)/t carries a relative error of a
  few eps32, i.e. an absolute error of about eps32 * kappa with kappa =
  max |g_hat| / t; q_i is a product of L such factors, so
  |dq| <= L (8 kappa + 16) eps32 (q <= 1).
* Iterates after 100 plain EGT iterations: rel-L_inf <= 1e-5, gap within 1e-3
  relative; EGT/as in tau-replay mode the same at 30 iterations (later EGT/as
  states are pinned one Decr at a time in test_gpu_decr_pin.py).
"""
import zlib

import numpy as np
import pytest

from oracle import egt as OE
from oracle import payoff
from oracle import treeplex as OT
from paper_1810_03063_b300 import synth
from tests import bounds as B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24
EPS64 = 2.0 ** -53


@pytest.fixture(scope="module")
def egtlib():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_1810_03063_b300 import egt
    return egt


GAMES = {}


def zero_range_game():
    """12-card deck (21 hands, one 32-hand tile with 11 padding columns) where player 1
    never holds every third hand."""
    spec = synth.river_endgame(n_cards=12, bet_fracs=(1.0,), raise_cap=2, stack=2.0, alpha=1.0)
    r = spec.ranges.copy()
    r[0, ::3] = 0.0
    r[0] /= r[0].sum()
    return synth.GameSpec(**{**spec.__dict__, "ranges": r, "name": "zero_range12"})


def get(name, egtlib):
    if name not in GAMES:
        spec = {"kuhn": synth.kuhn, "tiny": synth.tiny, "full": synth.full_deck,
                "large": synth.large, "tiny7": lambda: synth.tiny(seed=7),
                "libratus": lambda: synth.libratus(n_cards=20, stack=2.0),
                "max": synth.max_size, "zero_range": zero_range_game}[name]()
        og = payoff.make_game(spec)
        GAMES[name] = (spec, og, OE.Problem(og), egtlib.Game(spec, device=0))
    return GAMES[name]


def dev(g, arr, dtype=torch.float32):
    return torch.tensor(g.pack(arr), dtype=dtype, device="cuda")


def host(g, t):
    torch.cuda.synchronize()
    return g.unpack(t.double().cpu().numpy())


def abs_product(og, vec, player):
    """(|A| |v|) of the oracle's matrix, for the error bound."""
    out = np.zeros((og.S[player], og.H))
    for b, t in enumerate(og.sf.terminals):
        B = np.abs(og.block(b))
        if player == 0:
            out[t.seq[0]] += B @ np.abs(vec[t.seq[1]])
        else:
            out[t.seq[1]] += B.T @ np.abs(vec[t.seq[0]])
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


def rand_vec(rng, S, H, kind):
    if kind == "uniform01":
        return rng.random((S, H))
    if kind == "signed":
        return rng.normal(size=(S, H))
    if kind == "spread":                  # 30 decades inside one column, both signs
        return rng.choice([-1.0, 1.0], size=(S, H)) * 10.0 ** rng.uniform(-30, 0, size=(S, H))
    return rng.random((S, H)) ** 8        # many tiny entries next to large ones


@pytest.mark.parametrize("name", ["kuhn", "tiny", "tiny7", "full", "libratus", "max", "zero_range"])
@pytest.mark.parametrize("kind", ["uniform01", "signed", "skewed", "spread"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_grad_f32_matches_oracle(egtlib, name, kind, seed):
    """Every output within 8 eps32 of the FP64 oracle relative to |A| |v| of that output,
    plus the fixed-point floor (about H 2^-49 of its terminals' largest term: it only shows
    on outputs more than ~8 decades under their column's, which the 30-decade input kind
    has)."""
    spec, og, P, g = get(name, egtlib)
    rng = np.random.default_rng([zlib.crc32(f"{name}/{kind}".encode()), seed])
    for player in (0, 1):
        vin = rand_vec(rng, og.S[1 - player], og.H, kind).astype(np.float32).astype(np.float64)
        ref = og.Ay(vin) if player == 0 else og.Atx(vin)
        bound = 8 * EPS32 * abs_product(og, vin, player) + fixed_point_floor(og, vin, player) + 1e-300
        tin = dev(g, vin)
        tout = torch.full((og.S[player], g.ld), float("nan"), device="cuda")
        g.grad(player, tin, tout)
        got = host(g, tout)
        err = np.abs(got - ref)
        assert (err <= bound).all(), (player, float((err / bound).max()))
        assert torch.all(tout[:, g.H:] == 0)


def test_grad_large_game_full_size(egtlib):
    """The large game (508 sequences, 677 terminals per player) at full size: both FP32
    products of random iterates, every output against the oracle's Kronecker-factored
    brute force."""
    spec, og, P, g = get("large", egtlib)
    rng = np.random.default_rng(11)
    for player in (0, 1):
        vin = rng.random((og.S[1 - player], og.H)).astype(np.float32).astype(np.float64)
        ref = og.Ay(vin) if player == 0 else og.Atx(vin)
        bound = 8 * EPS32 * abs_product(og, vin, player) + fixed_point_floor(og, vin, player) + 1e-300
        tout = torch.full((og.S[player], g.ld), float("nan"), device="cuda")
        g.grad(player, dev(g, vin), tout)
        err = np.abs(host(g, tout) - ref)
        assert (err <= bound).all(), (player, float((err / bound).max()))


@pytest.mark.parametrize("name", ["kuhn", "tiny", "full", "libratus", "max", "zero_range", "large"])
def test_grad_f64_matches_oracle(egtlib, name):
    spec, og, P, g = get(name, egtlib)
    rng = np.random.default_rng(5)
    for player in (0, 1):
        vin = rng.normal(size=(og.S[1 - player], og.H))
        ref = og.Ay(vin) if player == 0 else og.Atx(vin)
        bound = 128 * EPS64 * abs_product(og, vin, player) + fixed_point_floor(og, vin, player) + 1e-300
        tout = torch.empty((og.S[player], g.ld), dtype=torch.float64, device="cuda")
        g.grad_f64(player, dev(g, vin, torch.float64), tout)
        got = host(g, tout)
        assert (np.abs(got - ref) <= bound).all()


def test_grad_ignores_padding_columns(egtlib):
    spec, og, P, g = get("tiny", egtlib)
    rng = np.random.default_rng(9)
    vin = rng.random((og.S[1], og.H)).astype(np.float32)
    t_clean = dev(g, vin)
    t_dirty = t_clean.clone()
    t_dirty[:, g.H:] = float("nan")
    a = torch.empty((og.S[0], g.ld), device="cuda")
    b = torch.empty((og.S[0], g.ld), device="cuda")
    g.grad(0, t_clean, a)
    g.grad(0, t_dirty, b)
    assert torch.equal(a, b)


def test_grad_is_deterministic(egtlib):
    spec, og, P, g = get("full", egtlib)
    vin = dev(g, np.random.default_rng(3).random((og.S[1], og.H)))
    outs = []
    for _ in range(3):
        o = torch.empty((og.S[0], g.ld), device="cuda")
        g.grad(0, vin, o)
        outs.append(o)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[1], outs[2])


def sbr_conditioning(P, player, gvec, mu):
    """(kappa, mag) of the recursion: kappa = max |g_hat| / t, mag = sum over simplexes and
    hands of |min g_hat| + |V_j| (the size of the terms the FP32 value is built from)."""
    tpx, beta = P.tpx[player], P.beta[player]
    ch = tpx.children()
    V = np.zeros((tpx.n_infosets, gvec.shape[1]))
    kappa, mag = 0.0, 0.0
    for j in sorted(range(tpx.n_infosets), key=lambda j: -tpx.infoset_level[j]):
        gh = np.stack([gvec[i] + sum((V[k] for k in ch[i]), 0) for i in tpx.infoset_seqs[j]])
        t = mu * beta[j]
        kappa = max(kappa, float(np.abs(gh).max() / t))
        m = gh.min(0)
        V[j] = m - t * np.log(np.exp(-(gh - m) / t).sum(0)) + t * np.log(len(tpx.infoset_seqs[j]))
        mag += float(np.abs(m).sum() + np.abs(V[j]).sum())
    return kappa, mag


@pytest.mark.parametrize("name", ["kuhn", "tiny", "full", "libratus", "max", "zero_range", "large"])
@pytest.mark.parametrize("mu_scale", [1.0, 1e-2, 1e-4])
def test_smoothed_br_matches_oracle(egtlib, name, mu_scale):
    spec, og, P, g = get(name, egtlib)
    rng = np.random.default_rng(17)
    for player in (0, 1):
        # a realistic gradient: the product of a random strategy of the opponent
        opp = OT.smoothed_br(P.tpx[1 - player], rng.normal(size=(og.S[1 - player], og.H)), 1.0)[0]
        gv = (og.Ay(opp) if player == 0 else og.Atx(opp)).astype(np.float32).astype(np.float64)
        mu = mu_scale * P.theory_mu() * 0.01
        loss = gv if player == 0 else -gv
        q_ref, v_ref, per_hand = OT.smoothed_br(P.tpx[player], loss, mu, P.beta[player])
        val_ref = v_ref if player == 0 else -v_ref
        q = torch.full((og.S[player], g.ld), float("nan"), device="cuda")
        val = g.smoothed_br(player, dev(g, gv), mu, q)
        got = host(g, q)
        kappa, mag = sbr_conditioning(P, player, loss, mu)
        L = max(P.tpx[player].infoset_level) + 1
        tol_q = L * (8 * kappa + 16) * EPS32
        assert np.abs(got - q_ref).max() <= tol_q, (np.abs(got - q_ref).max(), tol_q)
        tol_v = 16 * EPS32 * mag + 1e-300
        assert abs(val - val_ref) <= tol_v, (val, val_ref, tol_v)
        assert torch.all(q[:, g.H:] == 0)


@pytest.mark.parametrize("name", ["kuhn", "tiny", "full", "libratus", "max", "zero_range", "large"])
def test_best_response_f64_matches_oracle(egtlib, name):
    spec, og, P, g = get(name, egtlib)
    rng = np.random.default_rng(23)
    for player in (0, 1):
        gv = rng.normal(size=(og.S[player], og.H))
        loss = gv if player == 0 else -gv
        _, v, _ = OT.best_response(P.tpx[player], loss)
        ref = v if player == 0 else -v
        got = g.best_response_f64(player, dev(g, gv, torch.float64))
        assert abs(got - ref) <= 64 * EPS64 * np.abs(gv).sum()


@pytest.mark.parametrize("name", ["kuhn", "tiny", "full", "libratus", "max", "zero_range", "large"])
def test_gap_matches_oracle(egtlib, name):
    spec, og, P, g = get(name, egtlib)
    rng = np.random.default_rng(29)
    x = OT.smoothed_br(P.tpx[0], rng.normal(size=(og.S[0], og.H)), 0.5)[0].astype(np.float32)
    y = OT.smoothed_br(P.tpx[1], rng.normal(size=(og.S[1], og.H)), 0.5)[0].astype(np.float32)
    ref = P.to_mbb(P.eps_sad(x.astype(np.float64), y.astype(np.float64)))
    got = g.gap(dev(g, x), dev(g, y))
    assert abs(got - ref) <= 1e-9 * abs(ref) + 1e-9


def rel_linf(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("name", ["tiny", "full", "libratus", "max", "zero_range", "large"])
@pytest.mark.parametrize("variant", ["theory", "egt"])
def test_trajectory_plain_egt_100_iterations(egtlib, name, variant):
    spec, og, P, g = get(name, egtlib)
    mu0 = (0.05 * P.theory_mu(), 0.05 * P.theory_mu()) if variant == "egt" else None
    r = OE.solve(P, variant=variant, eps_mbb=0.0, max_iters=100, mu0=mu0, gap_every=1000)
    x = torch.empty((og.S[0], g.ld), device="cuda")
    y = torch.empty((og.S[1], g.ld), device="cuda")
    rep = g.solve(x, y, variant={"theory": 0, "egt": 1}[variant], mu0=mu0, eps_mbb=0.0,
                  max_iters=100, gap_every=1000)
    assert rep["iters"] == 100
    xg, yg = host(g, x), host(g, y)
    assert rel_linf(xg, r.x) <= 1e-5, rel_linf(xg, r.x)
    assert rel_linf(yg, r.y) <= 1e-5, rel_linf(yg, r.y)
    assert abs(rep["gap_mbb"] - r.gap_mbb) <= 1e-3 * r.gap_mbb
    assert np.isclose(rep["mu"][0], r.mux, rtol=1e-14) and np.isclose(rep["mu"][1], r.muy, rtol=1e-14)


def replay_on_gpu(g, og, mu0, schedule):
    x = torch.empty((og.S[0], g.ld), device="cuda")
    y = torch.empty((og.S[1], g.ld), device="cuda")
    rep = g.solve(x, y, variant=2, mu0=mu0, eps_mbb=0.0, max_iters=len(schedule), gap_every=1000,
                  replay=schedule)
    return host(g, x), host(g, y), rep


@pytest.mark.parametrize("name", ["tiny", "full", "libratus", "large"])
def test_trajectory_egt_as_tau_replay_30(egtlib, name):
    """EGT/as in tau-replay mode while its smoothing is still well conditioned: within
    1e-5, or 3x the FP32 noise floor of the FP64 oracle where that floor (the largest
    drift of four FP32-perturbed oracle runs) already reaches a few 1e-6 after 30
    iterations, as it does on the Libratus-menu game (up to 1.0e-5)."""
    spec, og, P, g = get(name, egtlib)
    mu0 = (0.01 * P.theory_mu(),) * 2
    r = OE.solve(P, variant="egt_as", eps_mbb=0.0, max_iters=30, mu0=mu0, gap_every=1000)
    runs = [B.fp32_noise_floor(P, mu0, r.schedule, seed) for seed in range(4)]
    fx = max(rel_linf(f.x, r.x) for f in runs)
    fy = max(rel_linf(f.y, r.y) for f in runs)
    xg, yg, rep = replay_on_gpu(g, og, mu0, r.schedule)
    assert rel_linf(xg, r.x) <= max(1e-5, 3 * fx), (rel_linf(xg, r.x), fx)
    assert rel_linf(yg, r.y) <= max(1e-5, 3 * fy), (rel_linf(yg, r.y), fy)
    assert abs(rep["gap_mbb"] - r.gap_mbb) <= 1e-3 * r.gap_mbb


@pytest.mark.parametrize("name", ["tiny", "full", "libratus"])
def test_egt_as_100_iterations_stay_valid(egtlib, name):
    """After 100 EGT/as iterations (tau replayed from the oracle) mu is small and the smoothed
    best responses are ill conditioned (max |g_hat| / (mu beta) reaches 1e3-1e4), so iterates
    are not compared here: test_gpu_decr_pin.py checks the small-mu arithmetic from the GPU's
    own late states, stage by stage.  What holds at any conditioning is checked: the iterates
    satisfy the sequence-form constraints (Sec. 4) and the reported residual is the exact FP64
    eps_sad of the GPU's own iterates."""
    spec, og, P, g = get(name, egtlib)
    mu0 = (0.01 * P.theory_mu(),) * 2
    r = OE.solve(P, variant="egt_as", eps_mbb=0.0, max_iters=100, mu0=mu0, gap_every=1000)
    xg, yg, rep = replay_on_gpu(g, og, mu0, r.schedule)
    assert rep["iters"] == 100
    assert OT.is_in_treeplex(P.tpx[0], xg, 1e-5) and OT.is_in_treeplex(P.tpx[1], yg, 1e-5)
    assert abs(rep["gap_mbb"] - P.to_mbb(P.eps_sad(xg, yg))) <= 1e-9 * rep["gap_mbb"]


@pytest.mark.parametrize("name", ["tiny", "full", "libratus", "large"])
def test_egt_as_free_running_decisions(egtlib, name):
    """Free-running EGT/as: the tau / player decisions follow the oracle's (EGV signs agree)."""
    spec, og, P, g = get(name, egtlib)
    mu0 = (0.01 * P.theory_mu(),) * 2
    r = OE.solve(P, variant="egt_as", eps_mbb=0.0, max_iters=60, mu0=mu0, gap_every=1000)
    rep = g.solve(variant=2, mu0=mu0, eps_mbb=0.0, max_iters=60, gap_every=1000, log_cap=60)
    gpu_sched = [(e["player"], e["tau"]) for e in rep["log"]]
    first_diff = next((t for t, (a, b) in enumerate(zip(gpu_sched, r.schedule)) if a != b), None)
    assert first_diff is None, f"first differing decision at iteration {first_diff}"


def test_kuhn_solve_reaches_value(egtlib):
    spec, og, P, g = get("kuhn", egtlib)
    x = torch.empty((og.S[0], g.ld), device="cuda")
    y = torch.empty((og.S[1], g.ld), device="cuda")
    rep = g.solve(x, y, variant=2, eps_mbb=1.0, max_iters=5000)
    assert rep["status"] == "EGT_OK" and rep["gap_mbb"] <= 1.0
    xv, yv = host(g, x), host(g, y)
    eps = P.eps_sad(xv, yv)
    assert abs(og.value(xv, yv) - 1.0 / 18.0) <= eps + 1e-7


def test_step_api_and_state_roundtrip(egtlib):
    spec, og, P, g = get("tiny", egtlib)
    mu0 = (0.01 * P.theory_mu(),) * 2
    g.solver_init(variant=2, mu0=mu0)
    info = g.step(-1, 0.5, mode=2)
    assert info["accepted"] and info["egv"] >= 0 and info["products"] >= 3
    x = torch.empty((og.S[0], g.ld), device="cuda")
    y = torch.empty((og.S[1], g.ld), device="cuda")
    mu = g.state_get(x, y)
    a = g.step(-1, info["tau"], mode=0)
    x1 = torch.empty_like(x)
    g.state_get(x1, None)
    g.state_set(x, y, mu)               # resume from the snapshot: the same step again
    b = g.step(-1, info["tau"], mode=0)
    x2 = torch.empty_like(x)
    g.state_get(x2, None)
    assert a["player"] == b["player"] and torch.equal(x1, x2)


def test_invalid_pointers_are_rejected(egtlib):
    spec, og, P, g = get("tiny", egtlib)
    t = torch.zeros((og.S[1], g.ld), device="cuda")
    o = torch.zeros((og.S[0] * g.ld + 8,), device="cuda")
    with pytest.raises(egtlib.EGTError):
        g.grad(0, t, o[1:])               # 4-byte offset: misaligned
    with pytest.raises(egtlib.EGTError):
        g.grad(2, t, o)
    with pytest.raises(egtlib.EGTError):
        g.smoothed_br(0, t, -1.0)
