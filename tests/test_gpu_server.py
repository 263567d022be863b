"""Serving (egt_server_*): continuous batching of solve requests.

A request admitted into a running batch keeps no trace of its neighbours: its
result must be bit for bit what egt_solve gives the same request alone, however
requests arrive, share launches and leave.  Admission is FIFO under the device
memory budget and the running cap.
"""
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


def solo(egtlib, spec, eps, max_iters):
    g = egtlib.Game(spec, device=0)
    x = torch.empty((g.S[0], g.ld), device="cuda")
    y = torch.empty((g.S[1], g.ld), device="cuda")
    rep = g.solve(x, y, variant=egtlib.EGT_AS, alpha=0.01, eps_mbb=eps, max_iters=max_iters, gap_every=1)
    torch.cuda.synchronize()
    g.close()
    return x.cpu().numpy(), y.cpu().numpy(), rep


def drain(srv, limit=10000):
    for _ in range(limit):
        st = srv.step()
        if st["queued"] == 0 and st["running"] == 0:
            return st
    raise AssertionError("server did not drain")


def test_requests_in_the_mix_equal_solo_solves(egtlib):
    srv = egtlib.Server(0, iters_per_step=37)
    first = [(synth.tiny(), 150.0), (synth.kuhn(), 5.0), (synth.full_deck(seed=synth.BASE_SEED + 5), 40.0)]
    later = [(synth.tiny(seed=synth.BASE_SEED + 9), 80.0), (synth.tiny(seed=synth.BASE_SEED + 2), 300.0),
             (synth.libratus(n_cards=20, stack=2.0), 100.0)]   # menus copied at submission
    ids = [(srv.submit(sp, eps_mbb=eps, max_iters=5000), sp, eps) for sp, eps in first]
    srv.step()
    srv.step()                                   # the first ones run while the others arrive
    ids += [(srv.submit(sp, eps_mbb=eps, max_iters=5000), sp, eps) for sp, eps in later]
    drain(srv)
    for rid, sp, eps in ids:
        r = srv.result(rid)
        xs, ys, rs = solo(egtlib, sp, eps, 5000)
        assert r["state"] == "done" and r["status"] == rs["status"] == "EGT_OK"
        assert r["iters"] == rs["iters"] and r["gap_mbb"] == rs["gap_mbb"] <= eps
        assert np.array_equal(r["x"], xs) and np.array_equal(r["y"], ys), sp.name
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
    with pytest.raises(egtlib.EGTError):
        srv.result(ids[0][0])                    # released
    srv.close()


def test_admission_respects_the_memory_budget_and_cap(egtlib):
    specs = [synth.tiny(seed=synth.BASE_SEED + k) for k in range(4)] + [synth.full_deck()]
    sizes = [egtlib.Game(sp, device=-1).device_bytes for sp in specs]
    budget = max(sizes) + min(sizes) // 2         # never two full-deck games, at most a tiny beside one
    srv = egtlib.Server(0, mem_budget_bytes=budget, iters_per_step=25)
    ids = [srv.submit(sp, eps_mbb=100.0, max_iters=3000) for sp in specs]
    seen_running = 0
    for _ in range(10000):
        st = srv.step()
        assert st["used_bytes"] <= budget
        seen_running = max(seen_running, st["running"])
        if st["queued"] == 0 and st["running"] == 0:
            break
    assert seen_running >= 1
    for rid in ids:
        assert srv.result(rid, iterates=False)["status"] == "EGT_OK"
    srv.close()

    srv = egtlib.Server(0, max_running=2, iters_per_step=10)
    ids = [srv.submit(synth.tiny(seed=synth.BASE_SEED + k), eps_mbb=100.0, max_iters=3000) for k in range(5)]
    st = srv.step()
    assert st["running"] <= 2 and st["queued"] >= 3
    drain(srv)
    assert all(srv.result(i, iterates=False)["status"] == "EGT_OK" for i in ids)
    srv.close()


def test_submit_rejects_what_cannot_run(egtlib):
    big = synth.large()
    srv = egtlib.Server(0, mem_budget_bytes=egtlib.Game(synth.tiny(), device=-1).device_bytes * 2)
    with pytest.raises(egtlib.EGTError) as e:
        srv.submit(big)
    assert e.value.status == 2                   # OOM: alone above the budget
    bad = synth.tiny()
    bad.hands[0, 0] = 99                         # card id outside the deck
    with pytest.raises(egtlib.EGTError):
        srv.submit(bad)
    st = srv.step()
    assert st["queued"] == 0 and st["running"] == 0 and st["launches"] == 0
    srv.close()


def test_unreachable_target_finishes_not_converged(egtlib):
    srv = egtlib.Server(0, iters_per_step=50)
    rid = srv.submit(synth.tiny(), eps_mbb=1e-9, max_iters=120)
    drain(srv)
    r = srv.result(rid)
    assert r["status"] == "EGT_ERR_NOT_CONVERGED" and r["iters"] == 120
    srv.close()


def test_served_requests_match_the_oracle(egtlib):
    """Requests served in a mix (a tiny and a full-deck game under practical EGT for 100
    iterations, admitted while an EGT/as request of another game is running) end where the
    FP64 oracle's solve of the same game ends: rel-L_inf 1e-5, mu to 1e-14, and the reported
    residual equal to the oracle's eps_sad of the returned iterates (1e-9) and within 1e-3 of
    the oracle trajectory's."""
    from oracle import egt as OE
    from oracle import payoff

    srv = egtlib.Server(0, iters_per_step=23)
    srv.submit(synth.tiny(seed=synth.BASE_SEED + 4), eps_mbb=20.0, max_iters=5000)
    srv.step()
    reqs = []
    for spec in (synth.tiny(), synth.full_deck(seed=synth.BASE_SEED + 6)):
        og = payoff.make_game(spec)
        P = OE.Problem(og)
        mu0 = (0.05 * P.theory_mu(),) * 2
        rid = srv.submit(spec, variant=egtlib.PRACTICAL, mu0=mu0, eps_mbb=0.0, max_iters=100, gap_every=1)
        reqs.append((rid, spec, og, P, mu0))
    drain(srv)
    for rid, spec, og, P, mu0 in reqs:
        r = srv.result(rid)
        assert r["iters"] == 100
        g = egtlib.Game(spec, device=-1)                       # host-only: the hand order
        xh, yh = g.unpack(r["x"].astype(np.float64)), g.unpack(r["y"].astype(np.float64))
        ref = OE.solve(P, variant="egt", eps_mbb=0.0, max_iters=100, mu0=mu0, gap_every=10 ** 6)
        rel = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
        assert rel(xh, ref.x) <= 1e-5 and rel(yh, ref.y) <= 1e-5, (spec.name, rel(xh, ref.x), rel(yh, ref.y))
        assert np.isclose(r["mu"][0], ref.mux, rtol=1e-14) and np.isclose(r["mu"][1], ref.muy, rtol=1e-14)
        own = P.to_mbb(P.eps_sad(xh, yh))
        assert abs(r["gap_mbb"] - own) <= 1e-9 * own
        ref_gap = P.to_mbb(P.eps_sad(ref.x, ref.y))
        assert abs(r["gap_mbb"] - ref_gap) <= 1e-3 * ref_gap
    srv.close()
