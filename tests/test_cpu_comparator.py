"""The FP64 multi-core CPU comparator (libegt_cpu, include/egt_cpu.h) against the oracle.

The comparator restates the same method (EGT/as, Alg. 2-4, the Sec. 5 smoothed
best response, the structured O(T H) products) in C++ with OpenMP; it is the fair
CPU baseline that bench.py reports beside the GPU numbers.  Being FP64 throughout,
it must follow the oracle's trajectory to rounding: every decision equal and the
iterates within 1e-10 while the smoothing is well conditioned.
"""
import re

import numpy as np
import pytest

from oracle import egt as OE
from oracle import payoff
from paper_1810_03063_b300 import synth

cpu = pytest.importorskip("paper_1810_03063_b300.egt_cpu", reason="libegt_cpu.so not built")


def test_exports_every_declared_symbol():
    names = sorted(set(re.findall(r"\b(egt_cpu_[a-z0-9_]+)\s*\(", open(cpu.HEADER).read())))
    assert len(names) >= 5
    for n in names:
        assert hasattr(cpu.lib, n), n


def zero_range():
    spec = synth.river_endgame(n_cards=12, bet_fracs=(1.0,), raise_cap=2, stack=2.0, alpha=1.0)
    r = spec.ranges.copy()
    r[0, ::3] = 0.0
    r[0] /= r[0].sum()
    return synth.GameSpec(**{**spec.__dict__, "ranges": r, "name": "zero_range12"})


@pytest.mark.parametrize("make", [synth.kuhn, synth.tiny, zero_range,
                                  lambda: synth.libratus(n_cards=20, stack=2.0)])
def test_egt_as_follows_the_oracle(make):
    spec = make()
    P = OE.Problem(payoff.make_game(spec))
    r = OE.solve(P, variant="egt_as", alpha=0.01, eps_mbb=0.0, max_iters=30, gap_every=1)
    c = cpu.CpuGame(spec).solve(alpha=0.01, eps_mbb=0.0, max_iters=30, gap_every=1, threads=2, iterates=True)
    assert c["iters"] == 30 and c["backoffs"] == r.backoffs
    assert np.abs(c["x"] - r.x).max() <= 1e-10 and np.abs(c["y"] - r.y).max() <= 1e-10
    assert np.isclose(c["mu"][0], r.mux, rtol=1e-12) and np.isclose(c["mu"][1], r.muy, rtol=1e-12)
    assert abs(c["gap_mbb"] - r.gap_mbb) <= 1e-9 * r.gap_mbb


def test_full_deck_trajectory_and_thread_count_independence():
    spec = synth.full_deck()
    P = OE.Problem(payoff.make_game(spec))
    r = OE.solve(P, variant="egt_as", alpha=0.01, eps_mbb=0.0, max_iters=12, gap_every=1)
    g = cpu.CpuGame(spec)
    a = g.solve(alpha=0.01, eps_mbb=0.0, max_iters=12, gap_every=1, threads=1, iterates=True)
    b = g.solve(alpha=0.01, eps_mbb=0.0, max_iters=12, gap_every=1, threads=3, iterates=True)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["y"], b["y"])   # fixed-order sums
    assert a["gap_mbb"] == b["gap_mbb"] and a["mu"] == b["mu"] and b["threads"] == 3
    assert a["backoffs"] == r.backoffs
    assert np.abs(a["x"] - r.x).max() <= 1e-10 and np.abs(a["y"] - r.y).max() <= 1e-10
    assert abs(a["gap_mbb"] - r.gap_mbb) <= 1e-9 * r.gap_mbb


def test_reaches_the_target():
    c = cpu.CpuGame(synth.tiny()).solve(alpha=0.01, eps_mbb=50.0, max_iters=20000, gap_every=1)
    assert c["status"] == "EGT_OK" and c["gap_mbb"] <= 50.0 and c["iters"] > 0
    c = cpu.CpuGame(synth.tiny()).solve(alpha=0.01, eps_mbb=1e-9, max_iters=20, gap_every=1)
    assert c["status"] == "EGT_ERR_NOT_CONVERGED" and c["iters"] == 20
