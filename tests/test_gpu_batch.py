"""Batched solving (egt_batch_*): many games in one device-resident launch.

A member's decisions come from the same fixed-order sums as when it runs
alone, whatever the group size and whatever else shares the launch, so each
member must end bit for bit where egt_solve takes the same game alone: same
iterates, mu, tau, residual and iteration count.  Each member stops at its own
target or iteration budget with its own status.
"""
import numpy as np
import pytest

from oracle import egt as OE
from oracle import payoff
from paper_1810_03063_b300 import synth
from tests import bounds as B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def egtlib():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_1810_03063_b300 import egt
    return egt


def mixed_specs():
    return [synth.tiny(), synth.kuhn(), synth.full_deck(seed=synth.BASE_SEED + 3),
            synth.tiny(seed=synth.BASE_SEED + 11), synth.large()]


def solo(egtlib, spec, variant, eps, max_iters, gap_every):
    g = egtlib.Game(spec, device=0)
    x = torch.empty((g.S[0], g.ld), device="cuda")
    y = torch.empty((g.S[1], g.ld), device="cuda")
    rep = g.solve(x, y, variant=variant, alpha=0.01, eps_mbb=eps, max_iters=max_iters,
                  gap_every=gap_every)
    torch.cuda.synchronize()
    g.close()
    return x, y, rep


def member_state(egtlib, g):
    x = torch.empty((g.S[0], g.ld), device="cuda")
    y = torch.empty((g.S[1], g.ld), device="cuda")
    mu = g.state_get(x, y)
    torch.cuda.synchronize()
    return x, y, mu


@pytest.mark.parametrize("group", [0, 1, 3])
def test_batch_members_equal_solo_solves_bitwise(egtlib, group):
    specs = mixed_specs()
    iters = [40, 40, 40, 25, 12]
    b = egtlib.Batch(0)
    games, slots = [], []
    for sp, n in zip(specs, iters):
        g = egtlib.Game(sp, device=0)
        g.solver_init(variant=egtlib.EGT_AS, alpha=0.01)
        slots.append(b.add(g, variant=egtlib.EGT_AS, eps_mbb=0.0, max_iters=n, gap_every=1))
        games.append(g)
    steps = b.run(n_iters=7, group=group)
    assert steps == 6                      # ceil(40 / 7) launches
    if group:
        assert b.launch_shape()[0] == group
    for sp, n, g, s in zip(specs, iters, games, slots):
        xs, ys, rs = solo(egtlib, sp, egtlib.EGT_AS, 0.0, n, 1)
        xb, yb, mu = member_state(egtlib, g)
        m = b.member(s)
        assert not m["active"] and m["status"] == "EGT_OK"
        assert m["iters"] == rs["iters"] == n
        assert torch.equal(xb, xs) and torch.equal(yb, ys), sp.name
        assert mu == rs["mu"] and m["tau"] == rs["tau"]
        assert m["gap_mbb"] == rs["gap_mbb"]
        # (the solo count also holds the initial point's products)
        assert m["backoffs"] == rs["backoffs"] and m["products"] == 3 * (n + m["backoffs"])
    b.close()


@pytest.mark.parametrize("variant", [0, 1])
def test_batch_plain_variants_equal_solo(egtlib, variant):
    specs = [synth.tiny(), synth.full_deck()]
    b = egtlib.Batch(0)
    games = []
    for sp in specs:
        g = egtlib.Game(sp, device=0)
        g.solver_init(variant=variant, alpha=0.01)
        games.append((b.add(g, variant=variant, eps_mbb=0.0, max_iters=30, gap_every=4), g))
    b.run(n_iters=11)
    for sp, (s, g) in zip(specs, games):
        xs, ys, rs = solo(egtlib, sp, variant, 0.0, 30, 4)
        xb, yb, mu = member_state(egtlib, g)
        assert torch.equal(xb, xs) and torch.equal(yb, ys)
        assert mu == rs["mu"] and b.member(s)["gap_mbb"] == rs["gap_mbb"]
    b.close()


def test_batch_members_stop_at_their_own_targets(egtlib):
    targets = [400.0, 150.0, 60.0]
    specs = [synth.tiny(seed=synth.BASE_SEED + k) for k in range(3)]
    b = egtlib.Batch(0)
    games = []
    for sp, eps in zip(specs, targets):
        g = egtlib.Game(sp, device=0)
        g.solver_init(variant=egtlib.EGT_AS, alpha=0.01)
        games.append((b.add(g, variant=egtlib.EGT_AS, eps_mbb=eps, max_iters=20000, gap_every=1), g))
    b.run(n_iters=50)
    for sp, eps, (s, g) in zip(specs, targets, games):
        m = b.member(s)
        xs, ys, rs = solo(egtlib, sp, egtlib.EGT_AS, eps, 20000, 1)
        assert m["status"] == rs["status"] == "EGT_OK"
        assert m["gap_mbb"] <= eps and m["gap_mbb"] == rs["gap_mbb"]
        assert m["iters"] == rs["iters"]
        xb, yb, _ = member_state(egtlib, g)
        assert torch.equal(xb, xs) and torch.equal(yb, ys)
    b.close()


def test_batch_budget_and_slots(egtlib):
    b = egtlib.Batch(0)
    g1 = egtlib.Game(synth.tiny(), device=0)
    g1.solver_init(variant=egtlib.EGT_AS, alpha=0.01)
    g2 = egtlib.Game(synth.kuhn(), device=0)
    g2.solver_init(variant=egtlib.EGT_AS, alpha=0.01)
    s1 = b.add(g1, eps_mbb=1e-9, max_iters=30)        # unreachable target
    s2 = b.add(g2, eps_mbb=0.0, max_iters=10)
    with pytest.raises(egtlib.EGTError):
        b.add(g1, max_iters=5)                        # already a member
    assert b.step(100) == 0
    assert b.member(s1)["status"] == "EGT_ERR_NOT_CONVERGED" and b.member(s1)["iters"] == 30
    assert b.member(s2)["status"] == "EGT_OK" and b.member(s2)["iters"] == 10
    b.remove(s1)
    with pytest.raises(egtlib.EGTError):
        b.member(s1)
    g3 = egtlib.Game(synth.tiny(seed=7), device=0)
    g3.solver_init(variant=egtlib.EGT_AS, alpha=0.01)
    assert b.add(g3, max_iters=5) == s1                # freed slot reused
    assert b.step(100) == 0 and b.member(s1)["iters"] == 5
    uninit = egtlib.Game(synth.tiny(), device=0)
    with pytest.raises(egtlib.EGTError):
        b.add(uninit, max_iters=5)
    b.close()


def test_batch_barrier_timeout_is_reported_per_member(egtlib, monkeypatch):
    b = egtlib.Batch(0)
    games = []
    for k in range(2):
        g = egtlib.Game(synth.tiny(seed=synth.BASE_SEED + k), device=0)
        g.solver_init(variant=egtlib.EGT_AS, alpha=0.01)
        games.append((b.add(g, max_iters=10), g))
    monkeypatch.setenv("EGT_TEST_BARRIER_EXTRA", "1")
    monkeypatch.setenv("EGT_BARRIER_TIMEOUT_MS", "50")
    assert b.step(5, group=2) == 0
    for s, _ in games:
        assert b.member(s)["status"] == "EGT_ERR_TIMEOUT"
    monkeypatch.delenv("EGT_TEST_BARRIER_EXTRA")
    # the context is still usable
    g = egtlib.Game(synth.tiny(), device=0)
    x = torch.empty((g.S[0], g.ld), device="cuda")
    y = torch.empty((g.S[1], g.ld), device="cuda")
    assert g.solve(x, y, variant=egtlib.EGT_AS, alpha=0.01, eps_mbb=0.0, max_iters=5)["iters"] == 5
    b.close()


def test_autotuned_shapes_leave_results_bitwise_unchanged(egtlib):
    """egt_batch_tune runs real steps under every candidate launch shape (CTA shares by a
    power 0-1 of the work; items paired on warp halves or not; all or 75 % of the co-resident
    CTAs) and keeps the fastest; members still end where solo solves end."""
    specs = mixed_specs()
    n = 60
    b = egtlib.Batch(0)
    games, slots = [], []
    for sp in specs:
        g = egtlib.Game(sp, device=0)
        g.solver_init(variant=egtlib.EGT_AS, alpha=0.01)
        slots.append(b.add(g, variant=egtlib.EGT_AS, eps_mbb=0.0, max_iters=n, gap_every=1))
        games.append(g)
    assert b.shape == dict(share=3, pairs=1, grid_pct=100, pack=0, wave_mb=128, wave_min=16)
    rep = b.tune(n_iters=3, reps=1)                # 13 candidates x 3 iterations = 39 of the 60
    cands = rep["candidates"]
    assert len(cands) == 13 and 0 <= rep["best"] < 13
    timed = [c for c in cands if c["iters"] > 0]
    assert all(c["iters"] == 3 * len(specs) for c in timed)    # every member ran every trial
    best = cands[rep["best"]]
    assert best["us_per_iter"] == min(c["us_per_iter"] for c in timed) > 0
    assert b.shape == {k: best[k] for k in ("share", "pairs", "grid_pct", "pack", "wave_mb", "wave_min")}
    b.run(n_iters=7)
    for sp, g, s in zip(specs, games, slots):
        xs, ys, rs = solo(egtlib, sp, egtlib.EGT_AS, 0.0, n, 1)
        xb, yb, mu = member_state(egtlib, g)
        m = b.member(s)
        assert not m["active"] and m["iters"] == rs["iters"] == n
        assert torch.equal(xb, xs) and torch.equal(yb, ys), sp.name
        assert mu == rs["mu"] and m["tau"] == rs["tau"] and m["gap_mbb"] == rs["gap_mbb"]
    # an idle batch: nothing timed, shape kept
    rep = b.tune(n_iters=3)
    assert rep["best"] == -1 and all(c["iters"] == 0 for c in rep["candidates"])
    with pytest.raises(egtlib.EGTError):
        b.shape = dict(share=5, pairs=1, grid_pct=100)
    with pytest.raises(egtlib.EGTError):
        b.shape = dict(share=2, pairs=1, grid_pct=0)
    with pytest.raises(egtlib.EGTError):
        b.shape = dict(wave_min=0)
    b.shape = dict(share=0, pairs=0, grid_pct=50, pack=1, wave_mb=3, wave_min=2)
    assert b.shape == dict(share=0, pairs=0, grid_pct=50, pack=1, wave_mb=3, wave_min=2)
    b.close()


def test_tuning_with_members_finishing_midway(egtlib):
    """Members that reach their budget during tuning drop out of the later trials (which then
    time fewer member-iterations) and still end exactly where their solo solves end."""
    specs = [synth.tiny(), synth.full_deck(seed=synth.BASE_SEED + 3)]
    budgets = [5, 50]
    b = egtlib.Batch(0)
    games, slots = [], []
    for sp, n in zip(specs, budgets):
        g = egtlib.Game(sp, device=0)
        g.solver_init(variant=egtlib.EGT_AS, alpha=0.01)
        slots.append(b.add(g, variant=egtlib.EGT_AS, eps_mbb=0.0, max_iters=n, gap_every=1))
        games.append(g)
    rep = b.tune(n_iters=3, reps=1)
    its = [c["iters"] for c in rep["candidates"]]
    assert its[:3] == [6, 5, 3] and all(i == 3 for i in its[3:])   # 13 trials x 3 = 39 < 50
    assert not b.member(slots[0])["active"] and b.member(slots[1])["active"]
    b.run(n_iters=7)
    for sp, n, g, s in zip(specs, budgets, games, slots):
        xs, ys, rs = solo(egtlib, sp, egtlib.EGT_AS, 0.0, n, 1)
        xb, yb, mu = member_state(egtlib, g)
        m = b.member(s)
        assert m["iters"] == rs["iters"] == n
        assert torch.equal(xb, xs) and torch.equal(yb, ys), sp.name
        assert mu == rs["mu"] and m["tau"] == rs["tau"] and m["gap_mbb"] == rs["gap_mbb"]
    b.close()


def test_launch_shape_fields_take_effect(egtlib):
    """grid_pct bounds the grid, share 0 gives equal groups, pairs = 0 keeps results unchanged."""
    specs = [synth.tiny(seed=synth.BASE_SEED + k) for k in range(4)]
    b = egtlib.Batch(0)
    games = []
    for sp in specs:
        g = egtlib.Game(sp, device=0)
        g.solver_init(variant=egtlib.EGT_AS, alpha=0.01)
        b.add(g, variant=egtlib.EGT_AS, eps_mbb=0.0, max_iters=30, gap_every=1)
        games.append(g)
    b.step(5)
    half = torch.cuda.get_device_properties(0).multi_processor_count // 2   # one CTA per SM
    b.shape = dict(share=0, pairs=0, grid_pct=50)
    b.step(5)
    group, grid = b.launch_shape()
    assert len(specs) <= grid <= half and group <= -(-half // len(specs))   # equal shares of half
    b.shape = dict(share=4, pairs=1, grid_pct=100)
    b.run(n_iters=7)
    for sp, g in zip(specs, games):
        xs, ys, rs = solo(egtlib, sp, egtlib.EGT_AS, 0.0, 30, 1)
        xb, yb, mu = member_state(egtlib, g)
        assert torch.equal(xb, xs) and torch.equal(yb, ys)
    b.close()


def test_packed_plan_runs_small_members_in_turn(egtlib):
    """pack = 1: members lighter than the balanced makespan share one-CTA groups run in turn
    (here many small games beside a large one); results still equal solo solves."""
    specs = [synth.large()] + [synth.tiny(seed=synth.BASE_SEED + k) for k in range(40)]
    n = 12
    b = egtlib.Batch(0)
    b.shape = dict(share=4, pairs=1, grid_pct=100, pack=1)
    games = []
    for sp in specs:
        g = egtlib.Game(sp, device=0)
        g.solver_init(variant=egtlib.EGT_AS, alpha=0.01)
        b.add(g, variant=egtlib.EGT_AS, eps_mbb=0.0, max_iters=n, gap_every=1)
        games.append(g)
    b.step(4)
    group, grid = b.launch_shape()
    assert grid <= torch.cuda.get_device_properties(0).multi_processor_count and group > 1
    b.run(n_iters=4)
    for sp, g in list(zip(specs, games))[:6]:
        xs, ys, rs = solo(egtlib, sp, egtlib.EGT_AS, 0.0, n, 1)
        xb, yb, mu = member_state(egtlib, g)
        assert torch.equal(xb, xs) and torch.equal(yb, ys), sp.name
        assert mu == rs["mu"]
    b.close()


def test_waves_keep_results(egtlib):
    """wave_mb: members in consecutive launches of bounded device bytes; same results."""
    specs = [synth.tiny(seed=synth.BASE_SEED + k) for k in range(6)] + [synth.full_deck()]
    n = 20
    b = egtlib.Batch(0)
    games = []
    for sp in specs:
        g = egtlib.Game(sp, device=0)
        g.solver_init(variant=egtlib.EGT_AS, alpha=0.01)
        b.add(g, variant=egtlib.EGT_AS, eps_mbb=0.0, max_iters=n, gap_every=1)
        games.append(g)
    b.shape = dict(share=3, pairs=1, grid_pct=100, pack=0, wave_mb=1, wave_min=1)   # about one member per wave
    b.run(n_iters=6)
    for sp, g in zip(specs, games):
        xs, ys, rs = solo(egtlib, sp, egtlib.EGT_AS, 0.0, n, 1)
        xb, yb, mu = member_state(egtlib, g)
        assert torch.equal(xb, xs) and torch.equal(yb, ys), sp.name
    b.close()


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


ORACLE_MIX = {"tiny": synth.tiny, "full": lambda: synth.full_deck(seed=synth.BASE_SEED + 3),
              "libratus20": lambda: synth.libratus(n_cards=20, stack=2.0), "large": synth.large}


@pytest.mark.parametrize("variant, n_iters", [("egt", 100), ("egt_as", 30)])
def test_batch_members_match_the_oracle(egtlib, variant, n_iters):
    """A mixed batch (tiny, full deck, 20-card Libratus menus, large) runs in batch launches of
    unequal length; every member's iterates match the FP64 oracle's solve of the same game at
    rel-L_inf 1e-5, mu to 1e-14 and the FP64 residual of its state to 1e-3: practical EGT for
    100 iterations, and free-running EGT/as for 30 iterations, where its smoothing is still well
    conditioned; there the iterate tolerance is 1e-5 or 3x the drift of the oracle's own run
    under FP32-sized noise on the same decisions, whichever is larger (that drift reaches a few
    1e-6 on the full deck by then, as in the solo tau-replay test)."""
    code = {"egt": egtlib.PRACTICAL, "egt_as": egtlib.EGT_AS}[variant]
    b = egtlib.Batch(0)
    members = []
    for name, make in ORACLE_MIX.items():
        spec = make()
        og = payoff.make_game(spec)
        P = OE.Problem(og)
        mu0 = ((0.05 if variant == "egt" else 0.01) * P.theory_mu(),) * 2
        g = egtlib.Game(spec, device=0)
        g.solver_init(variant=code, mu0=mu0)
        members.append((name, og, P, g, mu0, b.add(g, variant=code, eps_mbb=0.0, max_iters=n_iters,
                                                    gap_every=n_iters)))
    b.run(n_iters=17)
    for name, og, P, g, mu0, slot in members:
        r = OE.solve(P, variant=variant, eps_mbb=0.0, max_iters=n_iters, mu0=mu0, gap_every=10 ** 6)
        tx = ty = 1e-5
        if variant == "egt_as":
            runs = [B.fp32_noise_floor(P, mu0, r.schedule, seed) for seed in range(3)]
            tx = max(tx, 3 * max(rel_linf(f.x, r.x) for f in runs))
            ty = max(ty, 3 * max(rel_linf(f.y, r.y) for f in runs))
        m = b.member(slot)
        assert m["iters"] == n_iters
        xb, yb, mu = member_state(egtlib, g)
        xh, yh = g.unpack(xb.double().cpu().numpy()), g.unpack(yb.double().cpu().numpy())
        assert rel_linf(xh, r.x) <= tx, (name, rel_linf(xh, r.x), tx)
        assert rel_linf(yh, r.y) <= ty, (name, rel_linf(yh, r.y), ty)
        assert np.isclose(mu[0], r.mux, rtol=1e-14) and np.isclose(mu[1], r.muy, rtol=1e-14), name
        ref_gap = P.to_mbb(P.eps_sad(r.x, r.y))
        assert abs(g.state_gap() - ref_gap) <= 1e-3 * ref_gap, name
    b.close()
