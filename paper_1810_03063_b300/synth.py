"""Seeded synthetic river endgames (input generator only).

This module draws the *inputs* of a poker river endgame: the deck, the board,
the private hands, a strength preorder over the hands, each player's range
(the conditional hand distribution chance deals from), and the betting
parameters (pot, stack, bet-size menu, raise cap).  It holds none of the
method's arithmetic: no betting tree, no payoffs, no sequence form.  Both the
CUDA library (through the C-ABI) and the FP64 oracle consume what it returns.

The paper's workloads are Libratus river endgames (Sec. 7, "Experiments":
chance deals hands from the blueprint's conditional distribution, 5-card board,
pot, betting abstraction).  Their boards, ranges and bet trees are proprietary,
so these seeded games stand in for them with the same structure:

* deck of ``n_cards`` cards, card ``c`` has rank ``c // 4`` and suit ``c % 4``;
* board = first 5 cards of a seeded permutation of the deck;
* hands = all 2-card combinations of the remaining cards, lexicographic;
* strength = seeded total preorder: walk a random permutation of the hands,
  each hand opens a new strength class with probability ``1 - tie_prob`` or
  joins the previous class (about 25 % of hands tied by default);
* ranges = Dirichlet(alpha) over all ``C(n_cards, 2)`` combinations, combos
  touching the board zeroed, renormalised; independent per player.

RNG: ``numpy.random.Generator(PCG64(seed))``, draws in a fixed order (deck
permutation, strength permutation, class-opening uniforms, range of player 1,
range of player 2).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from itertools import combinations

import numpy as np

BASE_SEED = 1810030630


@dataclass(frozen=True)
class GameSpec:
    """Inputs of one river endgame (see module docstring)."""

    name: str
    n_cards: int
    hand_size: int
    board: tuple
    hands: np.ndarray          # [H, hand_size] int32 card ids, lexicographic order
    strength: np.ndarray       # [H] int32, higher wins, ties allowed
    ranges: np.ndarray         # [2, H] float64, each row sums to 1
    pot: float
    stack: float
    bb: float                  # big blind in chips; 1 mbb = bb / 1000
    bet_fracs: tuple
    allin: bool
    raise_cap: int
    seed: int = -1
    meta: dict = field(default_factory=dict)
    # None: the menu (bet_fracs, allin) everywhere.  Else menus[p][k] = (pot fractions, all-in
    # offered, fold offered when not facing a bet) for player p after k bets / raises (k = 3: 3+)
    menus: tuple = None

    @property
    def n_hands(self) -> int:
        return int(self.hands.shape[0])


def river_endgame(*, n_cards=52, bet_fracs=(0.5, 1.0), raise_cap=3, stack=10.0,
                  pot=1.0, alpha=0.5, tie_prob=0.25, seed=BASE_SEED, allin=True,
                  bb=None, name="river") -> GameSpec:
    """Draw one seeded river endgame with a 5-card board and 2-card hands."""
    # up to 60 cards (1485 hands, ld 1504): decks above 52 only exercise the library's size limit
    if n_cards < 9 or n_cards > 60 or n_cards % 4:
        raise ValueError("n_cards must be a multiple of 4 in [12, 60]")
    rng = np.random.Generator(np.random.PCG64(seed))
    deck_perm = rng.permutation(n_cards)
    board = tuple(sorted(int(c) for c in deck_perm[:5]))
    live = [c for c in range(n_cards) if c not in board]
    hands = np.array(list(combinations(live, 2)), dtype=np.int32)
    H = hands.shape[0]

    # strength preorder: random permutation, each hand opens a class w.p. 1 - tie_prob
    perm = rng.permutation(H)
    opens = rng.random(H) >= tie_prob
    strength = np.empty(H, dtype=np.int32)
    cls = -1
    for k, h in enumerate(perm):
        if k == 0 or opens[k]:
            cls += 1
        strength[h] = cls

    # ranges: Dirichlet over all combos of the full deck, board-touching combos zeroed
    all_combos = list(combinations(range(n_cards), 2))
    idx = {cmb: i for i, cmb in enumerate(all_combos)}
    live_idx = np.array([idx[(int(a), int(b))] for a, b in hands], dtype=np.int64)
    ranges = np.empty((2, H), dtype=np.float64)
    for p in range(2):
        full = rng.dirichlet(np.full(len(all_combos), alpha))
        r = full[live_idx]
        ranges[p] = r / r.sum()

    return GameSpec(name=name, n_cards=n_cards, hand_size=2, board=board, hands=hands,
                    strength=strength, ranges=ranges, pot=float(pot), stack=float(stack),
                    bb=float(0.05 * pot if bb is None else bb), bet_fracs=tuple(float(f) for f in bet_fracs),
                    allin=bool(allin), raise_cap=int(raise_cap), seed=int(seed),
                    meta=dict(alpha=alpha, tie_prob=tie_prob))


def tiny(seed=BASE_SEED) -> GameSpec:
    """20-card deck (5 ranks x 4 suits), 105 hands, bet {1 x pot} + all-in, cap 2, stack 2."""
    return river_endgame(n_cards=20, bet_fracs=(1.0,), raise_cap=2, stack=2.0, alpha=1.0,
                         seed=seed, name="tiny20")


def full_deck(seed=BASE_SEED, stack=10.0) -> GameSpec:
    """52 cards, 1081 hands, bets {0.5, 1} x pot + all-in, cap 3, stack 10."""
    return river_endgame(n_cards=52, bet_fracs=(0.5, 1.0), raise_cap=3, stack=stack, alpha=0.5,
                         seed=seed, name="full52")


def large(seed=BASE_SEED) -> GameSpec:
    """52 cards, 1081 hands, bets {0.25, 0.5, 1, 2} x pot + all-in, cap 4, stack 10."""
    return river_endgame(n_cards=52, bet_fracs=(0.25, 0.5, 1.0, 2.0), raise_cap=4, stack=10.0,
                         alpha=0.5, seed=seed, name="large52")


def max_size(seed=BASE_SEED) -> GameSpec:
    """60-card deck: 1485 hands per player (ld 1504, near the library's 1536 limit), bet {1} +
    all-in, cap 2, stack 2; a size-limit case, not a poker deck."""
    return river_endgame(n_cards=60, bet_fracs=(1.0,), raise_cap=2, stack=2.0, alpha=1.0,
                         seed=seed, name="max60")


def kuhn() -> GameSpec:
    """Kuhn poker as a river endgame: 3 one-card hands, ante pot 2, one bet of 1 chip.

    The betting rules of the library (bet = fraction x pot, sizes that reach
    the stack replaced by the all-in, cap on bets) generate exactly Kuhn's
    tree with pot 2, stack 1, cap 1.
    """
    hands = np.arange(3, dtype=np.int32).reshape(3, 1)
    return GameSpec(name="kuhn", n_cards=3, hand_size=1, board=(), hands=hands,
                    strength=np.arange(3, dtype=np.int32), ranges=np.full((2, 3), 1.0 / 3.0),
                    pot=2.0, stack=1.0, bb=1.0, bet_fracs=(0.5,), allin=True, raise_cap=1, seed=-1)


# Sec. 7's Libratus river abstraction (Libratus = player 1, first to act), per player and number
# of bets / raises so far: (pot fractions, all-in offered, fold offered when not facing a bet).
LIBRATUS_MENUS = (
    (((0.25, 0.5, 1.0, 2.0, 4.0, 8.0), True, True),   # opening: fold, check, six bets, all-in
     ((0.4, 0.7, 1.1, 2.0), True, False),              # after its check, facing the bet
     ((0.4, 0.7, 2.0), True, False),                   # after its bet, facing a raise
     ((0.7,), True, False)),                           # facing later raises
    (((0.5, 0.75, 1.0), True, True),                   # facing the check: fold, check, bets, all-in
     ((0.7, 1.1), True, False),                        # facing the initial bet
     ((0.7,), True, False),                            # facing later raises
     ((0.7,), True, False)),
)


def libratus(seed=BASE_SEED, n_cards=52, stack=9.0, alpha=0.5) -> GameSpec:
    """River endgame with Sec. 7's asymmetric Libratus bet menus, no raise cap besides the stack.

    stack 9 x pot is what remains of 200 big-blind stacks behind a 21 big-blind river pot
    (Endgame 2's pot, Sec. 7).
    """
    import dataclasses
    spec = river_endgame(n_cards=n_cards, bet_fracs=(), raise_cap=64, stack=stack, alpha=alpha,
                         seed=seed, name=f"libratus{n_cards}")
    return dataclasses.replace(spec, menus=LIBRATUS_MENUS)


def batch_mix(n_games=64, seed=BASE_SEED):
    """Ragged mix of river endgames: deck in {20, 52}, cap in {2, 3, 4}, 1-4 bet sizes."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    menu = (0.25, 0.5, 1.0, 2.0)
    out = []
    for i in range(n_games):
        deck = int(rng.choice([20, 52]))
        cap = int(rng.integers(2, 5))
        k = int(rng.integers(1, 5))
        fr = tuple(sorted(float(f) for f in rng.choice(menu, size=k, replace=False)))
        out.append(river_endgame(n_cards=deck, bet_fracs=fr, raise_cap=cap,
                                 stack=2.0 if deck == 20 else 10.0, alpha=1.0 if deck == 20 else 0.5,
                                 seed=seed + i, name=f"mix{i}"))
    return out
