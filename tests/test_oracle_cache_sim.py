"""Pins of the parallel LRU cache oracle (Section 5.1) against cases whose
answer is fixed independently: an unbounded sequential cache reaches the
ideal reuse (Section 5.1's definition), one cycle holding everything can hit
nothing (concurrent duplicates never hit), hand-worked streams, and a
brute-force LRU list for random streams."""
import numpy as np
import pytest

import meshgen as mg
from oracle import batching as B
from oracle import cache_sim as C


def test_unbounded_sequential_cache_reaches_ideal_reuse():
    mesh = mg.grid_mesh(20)
    n = len(mesh.indices)
    hits = C.parallel_cache_hits(mesh.indices, num_sms=1, concurrent=1, capacity=10 ** 9)
    assert hits / n == pytest.approx(B.ideal_reuse(mesh.indices), abs=0)
    assert hits == n - len(np.unique(mesh.indices))


def test_one_cycle_cannot_hit():
    mesh = mg.grid_mesh(10)
    assert C.parallel_cache_hits(mesh.indices, num_sms=1, concurrent=len(mesh.indices), capacity=10 ** 6) == 0


def test_hand_worked_streams():
    # capacity 1, one index per cycle: a a a b b -> miss hit hit miss hit
    assert C.parallel_cache_hits([1, 1, 1, 2, 2], 1, 1, 1) == 3
    # capacity 1 evicts: a b a -> all miss
    assert C.parallel_cache_hits([1, 2, 1], 1, 1, 1) == 0
    # capacity 2 keeps both: a b a b -> 2 hits
    assert C.parallel_cache_hits([1, 2, 1, 2], 1, 1, 2) == 2
    # two SMs, cycles of 2: SM0 works through [1,2 | 1,2], SM1 through [3,4 | 3,5]
    assert C.parallel_cache_hits([1, 2, 1, 2, 3, 4, 3, 5], 2, 2, 8) == 3
    # contiguous parts of ceil(7 / 2) = 4: SM0 [1,2 | 1,2], SM1 [1,2 | 1]
    assert C.parallel_cache_hits([1, 2, 1, 2, 1, 2, 1], 2, 2, 8) == 3
    # duplicates inside a cycle are shaded twice and inserted once
    assert C.parallel_cache_hits([7, 7, 7, 7], 1, 2, 4) == 2
    # LRU order: capacity 2, a b | a c | b  -> a hits in cycle 2 and becomes recent; c evicts b; b misses
    assert C.parallel_cache_hits([1, 2, 1, 3, 2], 1, 2, 2) == 1


def _brute(stream, sms, conc, cap):
    hits = 0
    part = (len(stream) + sms - 1) // sms
    for sm in range(sms):
        lru = []  # most recent last
        mine = stream[sm * part:(sm + 1) * part]
        for c in range(0, len(mine), conc):
            cyc = mine[c:c + conc]
            missed = []
            for v in cyc:
                if v in lru:
                    hits += 1
                    lru.remove(v)
                    lru.append(v)
                else:
                    missed.append(v)
            for v in missed:
                if v in lru:
                    lru.remove(v)
                lru.append(v)
                while len(lru) > cap:
                    lru.pop(0)
    return hits


@pytest.mark.parametrize("seed", range(8))
def test_random_streams_against_brute_force(seed):
    rng = np.random.default_rng(seed)
    stream = rng.integers(0, 12, size=int(rng.integers(1, 200))).tolist()
    sms, conc, cap = int(rng.integers(1, 4)), int(rng.integers(1, 9)), int(rng.integers(1, 10))
    assert C.parallel_cache_hits(stream, sms, conc, cap) == _brute(stream, sms, conc, cap)


def test_paper_setup_gives_little_reuse_on_a_large_mesh():
    # Section 5.1: the parallel cache stays below a fifth of the ideal reuse
    mesh = mg.geodesic_sphere(30, 1)
    r = C.parallel_cache_reuse(mesh.indices, 28, 1024, 64 * 1024)
    assert 0 <= r < 0.2 * B.ideal_reuse(mesh.indices)


# --- the native simulator (host code of the library; no GPU) against the oracle

@pytest.mark.parametrize("seed", range(6))
def test_native_simulator_matches_oracle_on_random_streams(seed):
    import paper_1805_08893_gb300 as gp
    rng = np.random.default_rng(100 + seed)
    stream = rng.integers(0, int(rng.integers(2, 3000)), size=int(rng.integers(1, 20000))).astype(np.uint32)
    sms, conc, cap = int(rng.integers(1, 40)), int(rng.integers(1, 300)), int(rng.integers(1, 700))
    want = C.parallel_cache_hits(stream, sms, conc, cap)
    for threads in (1, 0):
        assert gp.gp_simulate_parallel_cache(stream, sms, conc, cap, threads) == want


@pytest.mark.parametrize("kb", [16, 32, 64])
def test_native_simulator_matches_oracle_on_meshes(kb):
    import paper_1805_08893_gb300 as gp
    for mesh in (mg.grid_mesh(48), mg.geodesic_sphere(25, 3)):
        want = C.parallel_cache_hits(mesh.indices, 28, 1024, kb * 1024 // 32)
        assert gp.gp_simulate_parallel_cache(mesh.indices, 28, 1024, kb * 1024 // 32) == want


def test_native_simulator_rejects_bad_arguments():
    import paper_1805_08893_gb300 as gp
    with pytest.raises(gp.GpError):
        gp.gp_simulate_parallel_cache(np.arange(10, dtype=np.uint32), num_sms=0)
    with pytest.raises(gp.GpError):
        gp.gp_simulate_parallel_cache(np.arange(10, dtype=np.uint32), capacity_entries=0)
    assert gp.gp_simulate_parallel_cache(np.zeros(0, dtype=np.uint32)) == 0
