"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, validates descriptions, and its host-side game compiler
(device = -1) produces the same sequence form as the oracle."""
import numpy as np
import pytest

from oracle import egt as OE
from oracle import payoff
from paper_1810_03063_b300 import synth

egt = pytest.importorskip("paper_1810_03063_b300.egt", reason="libegt.so not built")


def test_exports_every_declared_symbol():
    names = egt.declared_symbols()
    assert len(names) >= 17
    for n in names:
        assert hasattr(egt.lib, n), n


SPECS = {
    "kuhn": synth.kuhn,
    "tiny": synth.tiny,
    "full": synth.full_deck,
    "full_stack2": lambda: synth.full_deck(stack=2.0),
    "large": synth.large,
    "libratus20": lambda: synth.libratus(n_cards=20, stack=2.0),
    "libratus52": synth.libratus,
}


@pytest.mark.parametrize("name", list(SPECS))
def test_host_compiler_matches_oracle(name):
    spec = SPECS[name]()
    g = egt.Game(spec, device=-1)
    og = payoff.make_game(spec, kind="factored" if spec.n_hands > 128 else "dense")
    P = OE.Problem(og)
    assert g.S == og.S and g.H == og.H and g.ld % 32 == 0 and g.ld >= g.H
    for p in range(2):
        tp = og.tpx[p]
        t = g.treeplex(p)
        assert list(t["parent"]) == list(tp.infoset_parent)
        assert list(t["first"]) == [s[0] for s in tp.infoset_seqs]
        assert list(t["n"]) == [len(s) for s in tp.infoset_seqs]
        assert list(t["level"]) == list(tp.infoset_level)
        assert np.array_equal(t["beta"], P.beta[p])
        assert np.isclose(g.M[p], P.M[p], rtol=1e-14)
        assert np.isclose(g.Omega[p], P.Omega[p], rtol=1e-12)
    term = g.terminals()
    assert g.T == len(og.sf.terminals)
    for b, t in enumerate(og.sf.terminals):
        assert (term["seq1"][b], term["seq2"][b]) == t.seq
        assert term["kind"][b] == (0 if t.kind == "fold" else 1)
        assert term["coef"][b] == og.coef[b]
    assert np.isclose(g.Z, og.Z, rtol=1e-12)
    assert np.isclose(g.normA, P.normA, rtol=1e-12)
    assert np.array_equal(g.order, np.argsort(spec.strength, kind="stable"))
    g.close()


def test_compute_calls_rejected_on_host_only_game():
    g = egt.Game(synth.tiny(), device=-1)
    with pytest.raises(egt.EGTError) as e:
        g.grad(0, 16, 32)
    assert e.value.status == 1
    with pytest.raises(egt.EGTError):
        g.solve(max_iters=1)
    g.close()


def _bad(**changes):
    base = synth.tiny()
    return synth.GameSpec(**{**base.__dict__, **changes})


@pytest.mark.parametrize("spec,msg", [
    (lambda: _bad(hands=np.where(synth.tiny().hands == synth.tiny().hands[0, 0], 99,
                                 synth.tiny().hands).astype(np.int32)), "card id"),
    (lambda: _bad(ranges=np.zeros((2, 105))), "all zero"),
    (lambda: _bad(ranges=np.full((2, 105), np.nan)), "finite"),
    (lambda: _bad(pot=0.0), "pot"),
    (lambda: _bad(bet_fracs=(-1.0,)), "bet fractions"),
    (lambda: _bad(hands=np.vstack([synth.tiny().hands[:-1], synth.tiny().hands[:1]])), "same cards"),
])
def test_invalid_descriptions_are_rejected(spec, msg):
    with pytest.raises(egt.EGTError) as e:
        egt.Game(spec(), device=-1)
    assert e.value.status == 1 and msg in str(e.value)


def test_disjoint_ranges_give_zero_chance_mass():
    """Every hand pair sharing a card: Z = 0 must be refused."""
    spec = synth.kuhn()
    r = np.zeros((2, 3))
    r[0, 0] = 1.0
    r[1, 0] = 1.0
    with pytest.raises(egt.EGTError) as e:
        egt.Game(synth.GameSpec(**{**spec.__dict__, "ranges": r}), device=-1)
    assert "Z = 0" in str(e.value)


def test_product_path_never_imports_the_oracle():
    """The library package and bench's own arm reach the oracle nowhere (it is test
    infrastructure; only tests, smoke() and bench's CPU legs may call it)."""
    import pathlib
    import re
    pkg = pathlib.Path(__file__).resolve().parents[1] / "paper_1810_03063_b300"
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)|[\"']oracle/", re.M)
    for f in pkg.rglob("*"):
        if f.suffix in (".py", ".cu", ".cuh", ".cpp", ".hpp", ".h"):
            assert not pat.search(f.read_text()), f


def test_size_limits():
    """1485 hands (ld 1504) compile and match the oracle's counts; a deck giving more than
    1536 hands is refused with its own message."""
    g = egt.Game(synth.max_size(), device=-1)
    assert g.H == 1485 and g.ld == 1504
    spec = synth.max_size()
    over = np.array([(a, b) for a in range(64) for b in range(a + 1, 64)][:1600], dtype=np.int32)
    big = synth.GameSpec(**{**spec.__dict__, "n_cards": 64, "hands": over,
                            "strength": np.arange(len(over), dtype=np.int32),
                            "ranges": np.full((2, len(over)), 1.0 / len(over))})
    with pytest.raises(egt.EGTError) as e:
        egt.Game(big, device=-1)
    assert "1536" in str(e.value)


def test_zero_range_hands_and_tiny_decks_compile():
    """Hands a player never holds (range 0) and a 12-card deck (21 hands, ld 32) are valid."""
    spec = synth.river_endgame(n_cards=12, bet_fracs=(1.0,), raise_cap=2, stack=2.0, alpha=1.0)
    r = spec.ranges.copy()
    r[0, ::3] = 0.0
    r[0] /= r[0].sum()
    g = egt.Game(synth.GameSpec(**{**spec.__dict__, "ranges": r}), device=-1)
    og = payoff.make_game(synth.GameSpec(**{**spec.__dict__, "ranges": r}))
    assert g.H == 21 and g.ld == 32 and g.S == og.S and np.isclose(g.Z, og.Z)
