"""egt_gap_noalloc against egt_gap, through the C-ABI.

egt_gap_noalloc serves callers that must not allocate device memory on their
path (device memory reserved up front by another allocator, or a loop that
cannot take the device-wide synchronisation of cudaMalloc / cudaFree): its
scratch is a static device array, so it allocates nothing.  It must give the
same residual as egt_gap, call after call, although every call reuses the same
array: both run the same kernels in the same order on the same data, only the
scratch differs, so the two residuals are equal bit for bit.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module")
def egtlib():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    from paper_1810_03063_b300 import egt
    return egt


def random_pair(g, rng):
    x = torch.tensor(rng.random((g.S[0], g.ld)), dtype=torch.float32, device="cuda")
    y = torch.tensor(rng.random((g.S[1], g.ld)), dtype=torch.float32, device="cuda")
    return x, y


@pytest.mark.parametrize("make", ["full_deck", "tiny"])
def test_gap_noalloc_matches_gap_on_consecutive_calls(egtlib, make):
    from paper_1810_03063_b300 import synth
    g = egtlib.Game(getattr(synth, make)(), device=0)
    rng = np.random.default_rng(2024)
    for _ in range(2):                     # two calls in a row share the static scratch
        x, y = random_pair(g, rng)
        ref = g.gap(x, y)
        got = g.gap_noalloc(x, y)
        assert got == ref, (got, ref)
    g.close()


def test_gap_noalloc_after_another_game(egtlib):
    """A smaller game after a larger one: nothing of the previous call leaks in."""
    from paper_1810_03063_b300 import synth
    big = egtlib.Game(synth.full_deck(seed=5), device=0)
    small = egtlib.Game(synth.kuhn(), device=0)
    rng = np.random.default_rng(7)
    xb, yb = random_pair(big, rng)
    xs, ys = random_pair(small, rng)
    for g, x, y in ((big, xb, yb), (small, xs, ys), (big, xb, yb)):
        ref = g.gap(x, y)
        assert g.gap_noalloc(x, y) == ref
    big.close()
    small.close()


def test_gap_noalloc_rejects_games_beyond_its_scratch(egtlib):
    from paper_1810_03063_b300 import synth
    g = egtlib.Game(synth.large(), device=0)       # 2 * 677 terminals * 1088 * 8 bytes > 2 MiB
    x, y = random_pair(g, np.random.default_rng(1))
    with pytest.raises(egtlib.EGTError) as e:
        g.gap_noalloc(x, y)
    assert e.value.status == 1 and "bytes of scratch" in str(e.value)
    g.close()
