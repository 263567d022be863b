"""The device-resident driver (egt_iterate, egt_solve with the device engine).

It runs the same kernel bodies and the same fixed-order FP64 reductions as the
host-driven loop, so its iterates, mu, tau, decisions and residuals must equal
the host loop's bit for bit; and that loop is the one held to the oracle in
test_gpu_parity.py.  Its grid barriers are bounded: a barrier that cannot
complete (phantom arrivals requested through the test hook) must end the
launch with EGT_ERR_TIMEOUT, leaving the context usable.
"""
import os

import numpy as np
import pytest

from paper_1810_03063_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def egtlib():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_1810_03063_b300 import egt
    return egt


GAMES = {}


def game(egtlib, name):
    if name not in GAMES:
        spec = {"tiny": synth.tiny, "full": synth.full_deck, "kuhn": synth.kuhn,
                "large": synth.large, "libratus": synth.libratus}[name]()
        GAMES[name] = egtlib.Game(spec, device=0)
    return GAMES[name]


def run(egtlib, g, engine, variant, iters, eps=0.0, gap_every=1, log_cap=0):
    x = torch.empty((g.S[0], g.ld), device="cuda")
    y = torch.empty((g.S[1], g.ld), device="cuda")
    rep = g.solve(x, y, variant=variant, alpha=0.01, eps_mbb=eps, max_iters=iters,
                  gap_every=gap_every, engine=engine, log_cap=log_cap)
    torch.cuda.synchronize()
    return x, y, rep


@pytest.mark.parametrize("name", ["kuhn", "tiny", "full", "libratus", "large"])
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_device_engine_equals_host_loop_bitwise(egtlib, name, variant):
    g = game(egtlib, name)
    xd, yd, rd = run(egtlib, g, egtlib.ENGINE_DEVICE, variant, 60, log_cap=60)
    xh, yh, rh = run(egtlib, g, egtlib.ENGINE_HOST, variant, 60, log_cap=60)
    assert torch.equal(xd, xh) and torch.equal(yd, yh)
    assert rd["iters"] == rh["iters"] == 60
    assert rd["mu"] == rh["mu"] and rd["tau"] == rh["tau"]
    assert rd["gap_mbb"] == rh["gap_mbb"]
    assert rd["backoffs"] == rh["backoffs"] and rd["products"] == rh["products"]
    assert rd["gap_checks"] == rh["gap_checks"]
    for a, b in zip(rd["log"], rh["log"]):
        assert (a["player"], a["tau"], a["mu"], a["backoffs"]) == (b["player"], b["tau"], b["mu"], b["backoffs"])
        assert a["gap_mbb"] == b["gap_mbb"]
        assert (np.isnan(a["egv"]) and np.isnan(b["egv"])) or a["egv"] == b["egv"]


def test_device_engine_stops_at_the_gap_target(egtlib):
    g = game(egtlib, "tiny")
    xd, yd, rd = run(egtlib, g, egtlib.ENGINE_DEVICE, 2, 20000, eps=200.0)
    xh, yh, rh = run(egtlib, g, egtlib.ENGINE_HOST, 2, 20000, eps=200.0)
    assert rd["status"] == rh["status"] == "EGT_OK"
    assert rd["iters"] == rh["iters"] and rd["gap_mbb"] == rh["gap_mbb"] <= 200.0
    assert torch.equal(xd, xh) and torch.equal(yd, yh)


def test_iterate_in_chunks_equals_one_launch(egtlib):
    g = game(egtlib, "full")
    g.solver_init(variant=2, alpha=0.01)
    g.iterate(25, variant=2, gap_every=5)
    g.iterate(15, variant=2, gap_every=5)
    x1 = torch.empty((g.S[0], g.ld), device="cuda")
    g.state_get(x1, None)
    g.solver_init(variant=2, alpha=0.01)
    rep = g.iterate(40, variant=2, gap_every=5)
    x2 = torch.empty((g.S[0], g.ld), device="cuda")
    g.state_get(x2, None)
    assert rep["iters"] == 40
    assert torch.equal(x1, x2)


def test_one_iteration_launches_with_backoffs_equal_one_launch(egtlib):
    """Every one-iteration launch ends with the deciding CTA's verdict on its last attempt
    pending: a rejection there must be redone inside the same launch (Alg. 4), so a run of
    one-iteration launches equals one launch bit for bit, back-offs included."""
    g = game(egtlib, "full")
    g.solver_init(variant=2, alpha=0.01)
    backoffs = 0
    for _ in range(200):
        rep = g.iterate(1, variant=2, gap_every=1)
        assert rep["iters"] == 1
        backoffs += rep["backoffs"]
    x1 = torch.empty((g.S[0], g.ld), device="cuda")
    y1 = torch.empty((g.S[1], g.ld), device="cuda")
    g.state_get(x1, y1)
    g.solver_init(variant=2, alpha=0.01)
    rep = g.iterate(200, variant=2, gap_every=1)
    x2 = torch.empty_like(x1)
    y2 = torch.empty_like(y1)
    g.state_get(x2, y2)
    assert rep["iters"] == 200 and rep["backoffs"] == backoffs
    assert backoffs > 0, "the window should contain a back-off"
    assert torch.equal(x1, x2) and torch.equal(y1, y2)


def test_iterate_gap_matches_state_gap(egtlib):
    g = game(egtlib, "full")
    g.solver_init(variant=2, alpha=0.01)
    rep = g.iterate(10, variant=2, gap_every=1)
    assert rep["gap_mbb"] == g.state_gap()


def test_large_game_runs_on_the_device_engine(egtlib):
    g = game(egtlib, "large")
    xd, yd, rd = run(egtlib, g, egtlib.ENGINE_DEVICE, 2, 20, gap_every=10)
    xh, yh, rh = run(egtlib, g, egtlib.ENGINE_HOST, 2, 20, gap_every=10)
    assert torch.equal(xd, xh) and rd["gap_mbb"] == rh["gap_mbb"]


def test_barrier_timeout_is_reported_and_context_survives(egtlib, monkeypatch):
    g = game(egtlib, "tiny")
    g.solver_init(variant=2, alpha=0.01)
    monkeypatch.setenv("EGT_TEST_BARRIER_EXTRA", "1")       # a CTA that never arrives
    monkeypatch.setenv("EGT_BARRIER_TIMEOUT_MS", "50")
    with pytest.raises(egtlib.EGTError) as e:
        g.iterate(3, variant=2)
    assert e.value.status == 7                              # EGT_ERR_TIMEOUT
    monkeypatch.delenv("EGT_TEST_BARRIER_EXTRA")
    monkeypatch.delenv("EGT_BARRIER_TIMEOUT_MS")
    # the device is still usable and the solver runs normally after re-initialisation
    xd, yd, rd = run(egtlib, g, egtlib.ENGINE_DEVICE, 2, 10)
    xh, yh, rh = run(egtlib, g, egtlib.ENGINE_HOST, 2, 10)
    assert torch.equal(xd, xh)


@pytest.mark.parametrize("variant", [1, 2])
def test_checkpoint_resume_in_a_fresh_game_is_bitwise(egtlib, tmp_path, variant):
    """A solve saved to a host .npz file (iterates + t, tau, mu, residual) and restored into a
    fresh game built from the same description continues exactly as the uninterrupted solve."""
    spec = synth.full_deck(seed=synth.BASE_SEED + 7)
    a = egtlib.Game(spec, device=0)
    a.solver_init(variant=variant, alpha=0.01)
    a.iterate(23, variant=variant, gap_every=4)
    path = str(tmp_path / "solve.npz")
    a.save(path)
    ra = a.iterate(31, variant=variant, gap_every=4)
    xa = torch.empty((a.S[0], a.ld), device="cuda")
    ya = torch.empty((a.S[1], a.ld), device="cuda")
    ca = a.checkpoint(xa, ya)
    b = egtlib.Game(spec, device=0)             # never initialised
    b.load(path)
    assert b.checkpoint()["t"] == 23
    rb = b.iterate(31, variant=variant, gap_every=4)
    xb = torch.empty_like(xa)
    yb = torch.empty_like(ya)
    cb = b.checkpoint(xb, yb)
    torch.cuda.synchronize()
    assert torch.equal(xa, xb) and torch.equal(ya, yb)
    assert ca == cb and ca["t"] == 54
    assert (ra["iters"], ra["backoffs"], ra["gap_mbb"], ra["mu"], ra["tau"]) == \
        (rb["iters"], rb["backoffs"], rb["gap_mbb"], rb["mu"], rb["tau"])
    bad = dict(cb, tau=0.0)
    with pytest.raises(egtlib.EGTError):
        b.restore(xb, yb, bad)
    a.close()
    b.close()


@pytest.mark.parametrize("engine", [0, 1])
def test_iteration_log_has_times_and_writes_jsonl(egtlib, tmp_path, engine):
    import json
    g = game(egtlib, "tiny")
    _, _, rep = run(egtlib, g, engine, 2, 40, log_cap=40)
    log = rep["log"]
    assert len(log) == 40 and [e["t"] for e in log] == list(range(40))
    times = [e["time_ns"] for e in log]
    assert all(b >= a for a, b in zip(times, times[1:])) and times[-1] > times[0]
    path = str(tmp_path / "solve.jsonl")
    egtlib.write_log_jsonl(path, log)
    recs = [json.loads(line) for line in open(path)]
    assert len(recs) == 40 and recs[0]["seconds"] == 0.0 and recs[-1]["seconds"] > 0
    assert recs[-1]["products"] == 3 * sum(1 + e["backoffs"] for e in log)
    assert all(r["egv"] is not None and r["egv"] >= 0 for r in recs)     # EGT/as accepts EGV >= 0 only
    # the residual of the iterates each iteration started from (gap_every = 1)
    assert all(r["gap_mbb"] is not None and r["gap_mbb"] > 0 for r in recs)


def test_whole_solves_are_deterministic(egtlib):
    """Two solves of the same game in separate game objects, one on a side stream, end with the
    same bits (iterates, mu, tau, residual, iteration and back-off counts)."""
    spec = synth.libratus(n_cards=52)
    runs = []
    for k in range(2):
        g = egtlib.Game(spec, device=0)
        x = torch.empty((g.S[0], g.ld), device="cuda")
        y = torch.empty((g.S[1], g.ld), device="cuda")
        s = torch.cuda.Stream() if k else torch.cuda.current_stream()
        with torch.cuda.stream(s):
            rep = g.solve(x, y, variant=2, alpha=0.01, eps_mbb=0.0, max_iters=400, gap_every=1,
                          stream=s.cuda_stream)
        torch.cuda.synchronize()
        runs.append((x, y, rep))
        g.close()
    (x0, y0, r0), (x1, y1, r1) = runs
    assert torch.equal(x0, x1) and torch.equal(y0, y1)
    for key in ("iters", "backoffs", "mu", "tau", "gap_mbb", "products"):
        assert r0[key] == r1[key], key
