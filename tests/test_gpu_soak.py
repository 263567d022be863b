"""Randomised soak of the solver paths (fixed seed, fixed counts): random river endgames
(decks 12-52, 1-3 bet sizes, raise caps 1-4, stacks 2 or 10) through the device-resident
driver for all three variants, with a sample compared bit for bit against the host-driven
loop; random batch mixes with and without launch-shape tuning; servers with random request
sets.  No call may end in an error status."""
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


def random_game(rng):
    deck = int(rng.choice([12, 20, 32, 52]))
    fr = tuple(sorted(rng.choice([0.25, 0.5, 1.0, 2.0], size=int(rng.integers(1, 4)), replace=False).tolist()))
    return synth.river_endgame(n_cards=deck, bet_fracs=fr, raise_cap=int(rng.integers(1, 5)),
                               stack=float(rng.choice([2.0, 10.0])), alpha=float(rng.choice([0.5, 1.0])),
                               seed=int(rng.integers(1 << 30)), name=f"soak{deck}")


def test_random_solves_engine_equals_host_loop(egtlib):
    rng = np.random.default_rng(1810030630)
    for case in range(40):
        sp = random_game(rng)
        g = egtlib.Game(sp, device=0)
        variant, n, ge = int(rng.integers(3)), int(rng.integers(5, 150)), int(rng.integers(1, 6))
        x = torch.empty((g.S[0], g.ld), device="cuda")
        y = torch.empty((g.S[1], g.ld), device="cuda")
        rd = g.solve(x, y, variant=variant, alpha=0.01, eps_mbb=0.0, max_iters=n, gap_every=ge,
                     engine=egtlib.ENGINE_DEVICE)
        assert rd["status"] == "EGT_OK" and rd["iters"] == n, (case, sp.name)
        if case % 3 == 0:
            xh, yh = torch.empty_like(x), torch.empty_like(y)
            rh = g.solve(xh, yh, variant=variant, alpha=0.01, eps_mbb=0.0, max_iters=n, gap_every=ge,
                         engine=egtlib.ENGINE_HOST)
            torch.cuda.synchronize()
            assert torch.equal(x, xh) and torch.equal(y, yh), (case, sp.name)
            assert (rd["gap_mbb"], rd["mu"], rd["tau"]) == (rh["gap_mbb"], rh["mu"], rh["tau"]), case
        g.close()


def test_random_batches_and_servers(egtlib):
    rng = np.random.default_rng(7)
    for case in range(12):
        specs = synth.batch_mix(int(rng.integers(2, 24)), seed=int(rng.integers(1 << 30)))
        b = egtlib.Batch(0)
        games = []
        for sp in specs:
            g = egtlib.Game(sp, device=0)
            g.solver_init(variant=egtlib.EGT_AS, alpha=0.01)
            b.add(g, variant=egtlib.EGT_AS, eps_mbb=float(rng.choice([0.0, 5.0])),
                  max_iters=int(rng.integers(10, 120)))
            games.append(g)
        if case % 2 == 0:
            b.tune(n_iters=int(rng.integers(1, 4)))
        b.run(n_iters=int(rng.integers(5, 60)))
        for s in range(len(specs)):
            m = b.member(s)
            assert not m["active"] and m["status"] in ("EGT_OK", "EGT_ERR_NOT_CONVERGED"), (case, m)
        b.close()
        for g in games:
            g.close()
    for case in range(6):
        srv = egtlib.Server(0, iters_per_step=int(rng.integers(10, 100)))
        ids = [srv.submit(random_game(rng), eps_mbb=float(rng.choice([50.0, 200.0])), max_iters=2000)
               for _ in range(int(rng.integers(1, 8)))]
        for _ in range(10000):
            st = srv.step()
            if st["queued"] == 0 and st["running"] == 0:
                break
        for i in ids:
            r = srv.result(i, iterates=False)
            assert r["status"] in ("EGT_OK", "EGT_ERR_NOT_CONVERGED"), (case, r)
        srv.close()
