"""Pins for the oracle's batching and counting (CPU only).

Each test checks the oracle against something other than itself: hand-worked
cases from the paper's algorithms (tests/golden), closed forms, the paper's
printed Table 1 numbers, or an independent brute-force restatement.
"""
import json
import math
import os

import numpy as np
import pytest

import meshgen as mg
from oracle import batching as B

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _parse_count(s):
    return float(s[:-1]) * (1e3 if s[-1] == "k" else 1e6)


# --------------------------------------------------------------------------
# warp voting (Algorithm 1)
# --------------------------------------------------------------------------

def _case_indices(spec):
    if spec == "range(96)":
        return list(range(96))
    if spec == "[7]*96":
        return [7] * 96
    if spec == "strip32":
        return [t + k for t in range(32) for k in range(3)]
    raise ValueError(spec)


@pytest.mark.parametrize("case", _gold("warp_vote_cases.json")["cases"], ids=lambda c: c["name"])
def test_warp_vote_hand_worked(case):
    idx = _case_indices(case["indices"])
    rounds = B.warp_vote_batch(idx, 0, len(idx))
    assert [r["triangles"] for r in rounds] == case["round_triangles"]
    assert [len(r["held"]) for r in rounds] == case["round_invocations"]


def _held_list_replay(idx, lo, hi):
    """Independent restatement of a warp-voting round as a list of held ids:
    walk chunks of 32 positions; an id already held keeps its lane, a new id
    takes the next lane while fewer than 32 are held; the corners before the
    first one that finds no lane (or the batch end) are done."""
    rounds = []
    c = lo
    while c < hi:
        held, done, off = [], 0, c
        while off < hi and len(held) < 32:
            chunk = idx[off:min(off + 32, hi)]
            stop = None
            for k, x in enumerate(chunk):
                if x not in held:
                    if len(held) < 32:
                        held.append(x)
                    elif stop is None:
                        stop = k
            done += stop if stop is not None else len(chunk)
            off += 32
        tris = done // 3
        rounds.append((c, tuple(held), tris))
        c += 3 * tris
    return rounds


@pytest.mark.parametrize("seed", range(12))
def test_warp_vote_matches_held_list_restatement(seed):
    rng = np.random.default_rng(seed)
    n_tris = int(rng.integers(1, 70))
    vocab = int(rng.integers(1, 120))
    idx = [int(x) for x in rng.integers(0, vocab, size=3 * n_tris)]
    for lo, hi in B.static_batches(len(idx), 3 * int(rng.integers(1, 70))):
        got = [(r["start"], tuple(r["held"]), r["triangles"]) for r in B.warp_vote_batch(idx, lo, hi)]
        assert got == _held_list_replay(idx, lo, hi)


@pytest.mark.parametrize("seed", range(8))
def test_warp_vote_invariants(seed):
    rng = np.random.default_rng(100 + seed)
    idx = [int(x) for x in rng.integers(0, 60, size=3 * 64)]
    for lo, hi in B.static_batches(len(idx), 96):
        rounds = B.warp_vote_batch(idx, lo, hi)
        # rounds tile the batch exactly, in triangle units
        assert rounds[0]["start"] == lo
        assert sum(3 * r["triangles"] for r in rounds) == hi - lo
        inv = 0
        for r in rounds:
            held = r["held"]
            assert 1 <= len(held) <= 32 and len(set(held)) == len(held)
            assert r["triangles"] >= 1
            # each written corner is shaded from the vertex its index names
            for k, slot in enumerate(r["map"]):
                assert held[slot] == idx[r["start"] + k]
            inv += len(held)
        assert len(set(idx[lo:hi])) <= inv <= (hi - lo) + 2 * len(rounds)


# --------------------------------------------------------------------------
# sorting (Algorithm 2) and hashing (Algorithm 3)
# --------------------------------------------------------------------------

def test_sort_hand_worked():
    g = _gold("sort_hash_cases.json")
    map_, uniq, nv = B.sort_batch(g["ids"])
    assert map_ == g["sort_map"] and uniq == g["sort_unique_ids"] and nv == g["num_vertices"]


@pytest.mark.parametrize("seed", range(10))
def test_sort_and_hash_brute_force(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(1, 400))
    ids = [int(x) for x in rng.integers(0, int(rng.integers(1, 2 * n + 2)), size=n)]
    u = set(ids)
    map_, uniq, nv = B.sort_batch(ids)
    assert nv == len(u) and uniq == sorted(u)
    assert all(uniq[map_[i]] == ids[i] for i in range(n))
    size = 1 << max(0, math.ceil(math.log2(len(u))))
    for ts in (size, 2 * size):
        table, hmap, occ = B.hash_batch(ids, ts)
        assert occ == len(u)
        stored = [x for x in table if x != B.EMPTY]
        assert sorted(stored) == sorted(u)  # each id exactly once
        assert all(table[hmap[i]] == ids[i] for i in range(n))


def test_hash_table_overflow_raises():
    with pytest.raises(ValueError):
        B.hash_batch([1, 2, 3], 2)


def test_hash_slot_range_and_spread():
    for ts in (1, 2, 64, 256, 1024):
        slots = {B.hash_slot(i, ts) for i in range(4 * ts)}
        assert all(0 <= s < ts for s in slots)
        assert len(slots) >= min(ts, 4 * ts) * 0.6


# --------------------------------------------------------------------------
# batch formation
# --------------------------------------------------------------------------

def test_static_batches_closed_form():
    for n, S in [(0, 3), (3, 3), (96, 96), (97 * 3, 96), (23814, 255)]:
        bs = B.static_batches(n, S)
        assert len(bs) == math.ceil(n / S)
        assert sum(hi - lo for lo, hi in bs) == n
        assert all(hi - lo == S for lo, hi in bs[:-1])
    # tiny grid, 256 read as 255 indices: 93 full batches and one of 99 indices
    bs = B.static_batches(23814, 255)
    assert len(bs) == 94 and bs[-1][1] - bs[-1][0] == 99
    with pytest.raises(ValueError):
        B.static_batches(9, 256)


def test_static_starts_closed_form():
    """Static batch starts (Section 3.3) in triangles, against closed forms:
    ceil(T / (S/3)) batches, every one S/3 triangles but the last, which holds
    the remaining 1..S/3; T = 0 gives the single start 0."""
    assert B.static_starts(0, 255) == [0]
    # tiny grid (7,938 triangles) at S = 255: 93 batches of 85, one of 33
    st = B.static_starts(7938, 255)
    assert len(st) == 95 and st[0] == 0 and st[-1] == 7938
    assert st[-1] - st[-2] == 33 and st[-2] == 93 * 85
    # the 7.2M-triangle mesh at S = 255: 84,706 batches
    st = B.static_starts(7_200_000, 255)
    assert len(st) - 1 == 84_706 and st[-1] - st[-2] == 7_200_000 - 84_705 * 85
    # exact multiples leave no ragged batch; one triangle is one batch
    assert B.static_starts(170, 255) == [0, 85, 170]
    assert B.static_starts(1, 3) == [0, 1]
    assert B.static_starts(2, 3) == [0, 1, 2]
    for T, S in [(1, 96), (31, 96), (32, 96), (33, 96), (1000, 768), (4097, 63)]:
        per = S // 3
        st = B.static_starts(T, S)
        nb = -(-T // per)
        assert len(st) == nb + 1 and st[0] == 0 and st[-1] == T
        assert all(st[b + 1] - st[b] == per for b in range(nb - 1))
        assert 1 <= st[-1] - st[-2] <= per
        assert st[-1] - st[-2] == T - per * (nb - 1)
    for bad in (0, 256, -3):
        with pytest.raises(ValueError):
            B.static_starts(10, bad)


@pytest.mark.parametrize("case", _gold("dynamic_partition_cases.json")["cases"],
                         ids=lambda c: f"Nu{c['max_unique']}_max{c['max_tris']}_seg{c['segment_tris']}")
def test_dynamic_partition_hand_worked(case):
    idx = _gold("dynamic_partition_cases.json")["indices"]
    st = B.dynamic_partition(idx, case["max_unique"], case["max_tris"], case["segment_tris"])
    assert st == case["starts"]


def _check_partition_rule(idx, st, nu, mx, seg):
    """Brute-force statement of the greedy rule: every batch respects both
    limits and every cut not at a segment boundary is forced."""
    T = len(idx) // 3
    assert st[0] == 0 and st[-1] == T and all(a < b for a, b in zip(st, st[1:]))
    tri = [set(idx[3 * t:3 * t + 3]) for t in range(T)]
    for b in range(len(st) - 1):
        u = set().union(*tri[st[b]:st[b + 1]])
        assert len(u) <= nu and st[b + 1] - st[b] <= mx
        e = st[b + 1]
        if e < T and not (seg and e % seg == 0):
            assert len(u | tri[e]) > nu or st[b + 1] - st[b] == mx
        # no segment boundary strictly inside a batch
        if seg:
            assert all(t % seg for t in range(st[b] + 1, st[b + 1]))


@pytest.mark.parametrize("seed", range(10))
def test_dynamic_partition_rule_brute_force(seed):
    rng = np.random.default_rng(300 + seed)
    T = int(rng.integers(1, 300))
    idx = [int(x) for x in rng.integers(0, int(rng.integers(3, 200)), size=3 * T)]
    nu = int(rng.integers(3, 40))
    mx = int(rng.integers(1, 30))
    seg = int(rng.choice([0, 7, 50]))
    st = B.dynamic_partition(idx, nu, mx, seg)
    _check_partition_rule(idx, st, nu, mx, seg)


def test_dynamic_partition_grid():
    g = mg.grid_mesh(16)
    idx = [int(x) for x in g.indices]
    st = B.dynamic_partition(idx, 64, 85, 0)
    _check_partition_rule(idx, st, 64, 85, 0)
    assert B.dynamic_partition([], 256, 341) == [0]


def test_unique_per_batch_matches_sets():
    rng = np.random.default_rng(5)
    idx = rng.integers(0, 50, size=3 * 200)
    st = [0, 1, 17, 18, 90, 200]
    want = [len(set(idx[3 * a:3 * b].tolist())) for a, b in zip(st, st[1:])]
    assert B.unique_per_batch(idx, st).tolist() == want


def test_batch_invocations_variants_agree_on_sets():
    g = mg.grid_mesh(12)
    idx = g.indices
    st = B.static_starts(g.num_tris, 96)
    sets = B.unique_per_batch(idx, st)
    assert (B.batch_invocations(idx, st, "sort") == sets).all()
    assert (B.batch_invocations(idx, st, "hash") == sets).all()
    assert (B.batch_invocations(idx, st, "naive") == np.diff(st) * 3).all()
    assert (B.batch_invocations(idx, st, "warp") >= sets).all()


# --------------------------------------------------------------------------
# reuse metrics (Section 4.1, Table 1)
# --------------------------------------------------------------------------

def test_ideal_reuse_closed_forms():
    n = 64
    g = mg.grid_mesh(n)
    assert B.ideal_reuse(g.indices) == pytest.approx(1 - n * n / (6 * (n - 1) ** 2), abs=1e-15)
    f = 9
    s = mg.geodesic_sphere(f, 1)
    assert B.ideal_reuse(s.indices) == pytest.approx(1 - (10 * f * f + 2) / (60 * f * f), abs=1e-15)
    assert B.ideal_reuse([1, 2, 3]) == 0.0
    assert B.ideal_reuse([4, 4, 4, 4, 4, 4]) == pytest.approx(5 / 6)


def test_ideal_reuse_reproduces_table1():
    """Table 1's ideal column equals 1 - V/(3T) within the rounding of the
    printed V and T (half a unit of their last digit), +-0.005."""
    for name, v, t, ideal, _, _ in _gold("table1_reuse.json")["rows"]:
        V, T = _parse_count(v), _parse_count(t)
        unit_v = 1e3 if v.endswith("k") and "." not in v else (1e5 if v.endswith("M") else 1e2)
        unit_t = 1e3 if t.endswith("k") and "." not in t else (1e5 if t.endswith("M") else 1e2)
        lo = 1 - (V + unit_v / 2) / (3 * (T - unit_t / 2))
        hi = 1 - (V - unit_v / 2) / (3 * (T + unit_t / 2))
        assert lo - 0.005 <= ideal <= hi + 0.005, name
        # achieved reuse is a fraction of corners: converting the ideal back
        # through the invocation count is exact
        inv = (1 - ideal) * 3 * T
        assert B.achieved_reuse(inv, 3 * T) == pytest.approx(ideal)


def test_table1_text_claims_hold_on_printed_rows():
    g = _gold("table1_reuse.json")
    c = g["text_claims"]
    for name, _, _, ideal, warp, dyn in g["rows"]:
        assert dyn / ideal >= c["dyn_over_ideal_min"], name
        assert warp / ideal >= c["warp_over_ideal_min"], name
        assert warp <= ideal + 1e-9 and dyn <= ideal + 1e-9


def test_reuse_on_locality_ordered_sphere():
    """On a sphere shaped like the paper's 'sphere' row (about 40k vertices),
    warp voting at batch 96 and dynamic batching at 1023/256 fall below the
    ideal in the order the paper reports (Table 1: ideal > dyn > warp), with
    dynamic close to the ideal.  The synthetic mesh uses a Morton order
    instead of the paper's cache optimiser, so the margins are wider than the
    paper's 5% / 10-20% (measured: dyn/ideal 0.94, warp/ideal 0.79)."""
    s = mg.geodesic_sphere(45, 1)
    idx = s.indices
    T = s.num_tris
    ideal = B.ideal_reuse(idx)
    warp = B.achieved_reuse(B.batch_invocations(idx, B.static_starts(T, 96), "warp").sum(), idx.size)
    st = B.dynamic_partition(idx, 256, 341)
    dyn = B.achieved_reuse(B.unique_per_batch(idx, st).sum(), idx.size)
    assert ideal > dyn > warp
    assert dyn / ideal >= 0.92
    assert warp / ideal >= 0.74
    # shading rate of dynamic batching is below the 1.5 invocations/vertex target
    assert B.shading_rate(B.unique_per_batch(idx, st).sum(), s.num_vertices) <= 1.5
