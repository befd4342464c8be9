"""Pins of the random-walk oracle (Section 5.4) against facts fixed outside
it: the published SplitMix64 sequence, the closed form of the kept moves on
a uniform field, a brute-force ranking of all candidate moves, the exact
draw distribution, and invariants of a walk."""
import json
import os

import numpy as np
import pytest

import meshgen as mg
from oracle import walk as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_sequence():
    want = [int(x, 16) for x in json.load(open(os.path.join(GOLDEN, "splitmix64.json")))["state0_outputs"]]
    got, state = [], 0
    for _ in range(3):
        got.append(W.splitmix64(state))
        state = (state + 0x9E3779B97F4A7C15) & W.MASK64
    assert got == want


def test_candidate_count_is_the_lattice_disc():
    # the lattice points with 1 <= r^2 <= 256, counted directly
    brute = sum(1 for dx in range(-16, 17) for dy in range(-16, 17) if 1 <= dx * dx + dy * dy <= 256)
    assert len(W.candidate_offsets()) == brute == 796


def test_uniform_field_keeps_the_eight_neighbours():
    act = np.full((40, 40), 1000, dtype=np.uint32)
    moves = W.cell_moves(act, 5, 7)
    # r^2 = 1 (likelihood 1000 * 65536) in row-major order, then r^2 = 2 (x 32768)
    assert [(dx, dy) for dx, dy, _ in moves] == [(0, -1), (-1, 0), (1, 0), (0, 1), (-1, -1), (1, -1), (-1, 1), (1, 1)]
    assert [lk for *_, lk in moves] == [1000 * 65536] * 4 + [1000 * 32768] * 4


@pytest.mark.parametrize("seed", range(4))
def test_kept_moves_against_brute_force_ranking(seed):
    rng = np.random.default_rng(seed)
    act = rng.integers(0, 50, size=(23, 31)).astype(np.uint32)  # many equal likelihoods
    x, y = int(rng.integers(0, 31)), int(rng.integers(0, 23))
    allm = []
    for j, (dx, dy) in enumerate([(dx, dy) for dy in range(-16, 17) for dx in range(-16, 17)
                                  if 1 <= dx * dx + dy * dy <= 256]):
        lk = int(act[(y + dy) % 23, (x + dx) % 31]) * (65536 // (dx * dx + dy * dy))
        allm.append((lk, j, dx, dy))
    best = sorted(allm, key=lambda t: (-t[0], t[1]))[:8]
    assert W.cell_moves(act, x, y) == [(dx, dy, lk) for lk, _, dx, dy in best]


def test_draw_distribution_is_exactly_proportional():
    moves = [(1, 0, 5), (0, 1, 3), (-1, 0, 2), (0, -1, 0), (1, 1, 0), (2, 0, 0), (0, 2, 0), (3, 0, 0)]
    counts = {}
    for u in range(10 * 100):  # every residue mod 10 equally often
        m = W.choose(moves, u)
        counts[m] = counts.get(m, 0) + 1
    assert counts == {(1, 0): 500, (0, 1): 300, (-1, 0): 200}
    assert W.choose([(1, 0, 0)] * 8, 12345) == (0, 0)


def test_walk_invariants():
    act = mg.walk_activity(3, 48, 40)
    keys = mg.walk_agents(3, 500, 48, 40)
    new = W.step(act, keys, 0, 99)
    for k0, k1 in zip(keys.tolist(), new.tolist()):
        x0, y0, x1, y1 = k0 >> 16, k0 & 0xFFFF, k1 >> 16, k1 & 0xFFFF
        assert x1 < 48 and y1 < 40
        d = ((x1 - x0 + 24) % 48 - 24, (y1 - y0 + 20) % 40 - 20)
        assert d in [(dx, dy) for dx, dy, lk in W.cell_moves(act, x0, y0) if lk > 0]


def test_batch_counts():
    keys = np.array([5, 5, 6, 7] * 16 + [9] * 32, dtype=np.uint32)
    assert W.batch_invocations(keys, "naive", 64).tolist() == [64, 32]
    assert W.batch_invocations(keys, "hash", 64).tolist() == [3, 1]
    assert W.batch_invocations(keys, "warp", 64).tolist() == [6, 1]
