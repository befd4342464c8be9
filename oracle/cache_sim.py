"""Oracle of the parallel per-multiprocessor vertex cache of Section 5.1.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper compares batching against a simulated cache setup: a number of
multiprocessors, each running a fixed number of vertex-shader invocations at
a time and keeping their results in its own least-recently-used cache of a
given size (Section 5.1, Table 1 "Parallel Cache": 28 multiprocessors, 1024
concurrent invocations, 16/32/64 KB).  A duplicate index only hits the cache
if its vertex was shaded in an earlier shading cycle of the same
multiprocessor -- not if it is being shaded concurrently.

Readings (the paper does not fix them):

* Work distribution: the index buffer is split into num_sms contiguous parts
  of ceil(n / num_sms) indices (the last one shorter); each multiprocessor
  works through its part in shading cycles of ``concurrent`` consecutive
  indices.  (Dealing the cycles out round-robin instead gives reuse two
  orders of magnitude below Table 1's; contiguous parts land in its range.)
* Within a cycle each index is looked up in order; a hit refreshes its entry;
  every index that misses is shaded (one invocation each, also for
  duplicates inside the cycle).  At the end of the cycle the missed ids are
  inserted in index order (an id missed twice is inserted once, at its last
  miss), evicting least recently used entries beyond the capacity.
* Capacity in entries = cache bytes / 32 (one shaded vertex, 7 floats,
  padded to a 32-byte row).
* Reuse = hits / indices (Table 1's "average vertex reuse").
"""
from collections import OrderedDict


def parallel_cache_hits(index_buffer, num_sms: int, concurrent: int, capacity: int) -> int:
    """Number of indices served from a multiprocessor's LRU cache (Section 5.1)."""
    n = len(index_buffer)
    part = -(-n // num_sms)
    hits = 0
    for sm in range(num_sms):
        cache = OrderedDict()  # id -> None, least recently used first
        end = min(n, (sm + 1) * part)
        for lo in range(sm * part, end, concurrent):
            hi = min(lo + concurrent, end)
            missed = []
            for i in range(lo, hi):
                v = int(index_buffer[i])
                if v in cache:
                    hits += 1
                    cache.move_to_end(v)
                else:
                    missed.append(v)
            for v in missed:  # results of this cycle become visible afterwards
                if v in cache:
                    cache.move_to_end(v)
                else:
                    cache[v] = None
                    if len(cache) > capacity:
                        cache.popitem(last=False)
    return hits


def parallel_cache_reuse(index_buffer, num_sms: int = 28, concurrent: int = 1024, cache_bytes: int = 16 * 1024,
                         entry_bytes: int = 32) -> float:
    """Table 1's "Parallel Cache" reuse column: hits / indices."""
    n = len(index_buffer)
    if n == 0:
        return 0.0
    return parallel_cache_hits(index_buffer, num_sms, concurrent, cache_bytes // entry_bytes) / n
