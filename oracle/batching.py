"""Batch formation and per-batch shading-invocation counts, replayed on the CPU.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Each function takes the steps of one part of the method (Kenzel et al.,
Section 3) in the paper's order, restated from what the step computes.
Where the printed pseudocode is garbled or ambiguous the reading taken is
stated in the docstring; the full list of readings is kept with the design
notes.  Pure-Python loops: meant for small inputs or sampled batches of
large ones.
"""
from __future__ import annotations

import math

import numpy as np

WARP_SIZE = 32
EMPTY = -1  # the "-1" marker of Algorithms 1 and 3
HASH_MULTIPLIER = 2654435769  # Knuth's multiplicative constant, floor(2^32 / golden ratio)


def _ffs(x: int) -> int:
    """1-based position of the lowest set bit, 0 for x == 0 (CUDA ``ffs``)."""
    return (x & -x).bit_length()


# --------------------------------------------------------------------------
# batch formation
# --------------------------------------------------------------------------

def static_batches(num_indices: int, batch_indices: int):
    """Static batching (Section 3.3): consecutive windows of a fixed number of
    indices, the last one ragged.  The size must be a multiple of 3 so that no
    triangle straddles two batches.  Returns [(begin, end)) index ranges."""
    if batch_indices <= 0 or batch_indices % 3:
        raise ValueError("static batch size must be a positive multiple of 3")
    return [(b, min(b + batch_indices, num_indices)) for b in range(0, num_indices, batch_indices)]


def dynamic_partition(index_buffer, max_unique: int, max_tris: int, segment_tris: int = 0):
    """Dynamic batching preprocessing (Section 3.4).

    Scan the triangles front to back, counting the unique indices of the open
    batch; a triangle joins the batch while the batch then holds at most
    ``max_unique`` unique indices (the paper's N, reached inclusively) and at
    most ``max_tris`` triangles; otherwise the batch is closed and the
    triangle starts the next one.  The batch starts go to an auxiliary buffer.

    ``segment_tris`` > 0 additionally closes the open batch at every multiple
    of ``segment_tris`` triangles (the segmented reading that lets segments be
    scanned in parallel); 0 is the paper's single scan.

    Returns the batch starts in triangles with the triangle count appended:
    batch b covers triangles [starts[b], starts[b+1]).
    """
    if max_unique < 3 or max_tris < 1:
        raise ValueError("need max_unique >= 3 and max_tris >= 1")
    idx = [int(i) for i in index_buffer]
    T = len(idx) // 3
    starts = [0]
    if T == 0:
        return starts
    batch_set = set()
    count = 0
    for t in range(T):
        tri = {idx[3 * t], idx[3 * t + 1], idx[3 * t + 2]}
        at_segment = segment_tris > 0 and t % segment_tris == 0
        if count > 0 and (at_segment or len(batch_set | tri) > max_unique or count + 1 > max_tris):
            starts.append(t)
            batch_set = set()
            count = 0
        batch_set |= tri
        count += 1
    starts.append(T)
    return starts


# --------------------------------------------------------------------------
# per-batch deduplication
# --------------------------------------------------------------------------

def sort_batch(ids):
    """Deduplication of one batch by sorting (Section 3.4, Algorithm 2).

    The batch's (vertex id, position) pairs are sorted by id, stably, so
    equal ids form runs.  The last pair of every run is flagged (the end of
    the sorted list counts as a run boundary).  Summing the flags before each
    pair (an exclusive prefix sum) numbers the runs 0, 1, ... in ascending id
    order: that number is the slot of every position in the run, and the
    total is the number of distinct ids, i.e. the shader invocations of the
    batch.

    Returns (slot of each position, distinct ids in ascending order, count).
    """
    n = len(ids)
    order = sorted(range(n), key=lambda pos: int(ids[pos]))  # stable: positions stay in order within a run
    sorted_ids = [int(ids[pos]) for pos in order]
    run_end = [int(k == n - 1 or sorted_ids[k] != sorted_ids[k + 1]) for k in range(n)]
    runs_before = np.concatenate(([0], np.cumsum(run_end, dtype=np.int64)[:-1])).tolist() if n else []
    count = int(sum(run_end))
    slot_of = [0] * n
    distinct = [None] * count
    for k, pos in enumerate(order):
        slot_of[pos] = runs_before[k]
        distinct[runs_before[k]] = sorted_ids[k]
    return slot_of, distinct, count


def hash_slot(vertex_id: int, table_size: int) -> int:
    """Multiplicative hashing (Section 3.4): the top log2(size) bits of
    (id * A) mod 2^32, A = 2654435769 (the multiplier is not printed; this is
    the reading)."""
    bits = int(math.log2(table_size))
    if 1 << bits != table_size:
        raise ValueError("hash table size must be a power of two")
    return ((int(vertex_id) * HASH_MULTIPLIER) & 0xFFFFFFFF) >> (32 - bits) if bits else 0


def hash_batch(ids, table_size: int):
    """Deduplication of one batch by hashing (Section 3.4, Algorithm 3), the
    insertions taken one at a time in position order.

    The table starts with every slot empty.  Each position's id starts at its
    home slot (``hash_slot``) and walks forward one slot at a time (linear
    probing, wrapping around) until it finds either its own id, already
    stored by an earlier position, or an empty slot, which it then claims.
    The slot found is that position's entry of the map; every claimed slot is
    one shader invocation.  Readings of the printed algorithm: the
    compare-and-swap targets the probed slot, and a position is placed when
    the slot held nothing or held its own id.

    Returns (table, slot of each position, number of claimed slots).  On the
    GPU the slot an id ends up in depends on the order of concurrent
    insertions; the set of stored ids and the id behind each position do not.
    """
    table = [EMPTY] * table_size
    slot_of = []
    for vid in ids:
        vid = int(vid)
        s = hash_slot(vid, table_size)
        for _ in range(table_size):
            held = table[s]
            if held == EMPTY:
                table[s] = vid
            if held == EMPTY or held == vid:
                break
            s = (s + 1) % table_size
        else:
            raise ValueError("hash table full: more unique indices than slots")
        slot_of.append(s)
    return table, slot_of, sum(1 for x in table if x != EMPTY)


def warp_vote_batch(index_buffer, batch_begin: int, batch_end: int):
    """Deduplication of one static batch by warp voting (Section 3.3,
    Algorithm 1), for one warp of 32 lanes.

    The batch is worked through in rounds.  At the start of a round no lane
    holds a vertex.  The warp reads the batch 32 positions at a time; the
    positions of such a chunk are considered one after another, in lane
    order: a position whose id a lane already holds maps to that lane; a new
    id goes to the next free lane while one is left; otherwise the position
    gets no lane.  The positions of the chunk before the first one without a
    lane (or past the batch end) are finished.  The round reads chunks until
    every lane holds a vertex or the batch ends; then every held vertex is
    shaded once and the finished positions' whole triangles are written.
    The next round starts at the first position not written.

    Readings of the printed algorithm:
      * a 33rd new id in a round gets no lane (the printed shift by 32 is
        read as "no lane");
      * the finished count is 32 when every position of the chunk found a
        lane, else the index of the first one that did not (the printed
        minimum is unbalanced and its bit position is 1-based);
      * the round start advances from its current value by 3 x triangles;
      * all whole triangles of the round are written (the printed bound on
        the lane id only covers batches of at most 96 indices);
      * the corners of a triangle that a round cuts off are shaded again in
        the next round and count as further invocations.

    Returns a list of rounds, each a dict with ``start`` (first position of
    the round), ``held`` (the ids of lanes 0.. in the order they were taken,
    i.e. the round's shader invocations), ``map`` (the lane of each of the
    round's 3 x triangles corners) and ``triangles``.
    """
    rounds = []
    round_start = batch_begin
    while round_start < batch_end:
        n_held = 0        # lanes taken, counting ids that found none
        finished = 0      # positions of the round that found a lane, in whole chunks
        lane_holds = [EMPTY] * WARP_SIZE
        offset = round_start
        lane_of = {}
        while offset < batch_end and n_held < WARP_SIZE:
            chunk_ids = [int(index_buffer[offset + k]) if offset + k < batch_end else EMPTY
                         for k in range(WARP_SIZE)]
            slot_mask = [EMPTY] * WARP_SIZE
            for k in range(WARP_SIZE):
                vid = chunk_ids[k]
                holders = 0
                for lane in range(WARP_SIZE):  # which lanes hold this id
                    if lane_holds[lane] == vid:
                        holders |= 1 << lane
                if holders == 0:
                    if n_held < WARP_SIZE:
                        lane_holds[n_held] = vid
                        holders = 1 << n_held
                    n_held += 1
                slot_mask[k] = holders
            for k in range(WARP_SIZE):
                lane_of[finished + k] = _ffs(slot_mask[k]) - 1
            stops = 0
            for k in range(WARP_SIZE):
                if slot_mask[k] == 0 or chunk_ids[k] == EMPTY:
                    stops |= 1 << k
            finished += WARP_SIZE if stops == 0 else _ffs(stops) - 1
            offset += WARP_SIZE
        triangles = finished // 3
        held = lane_holds[:min(n_held, WARP_SIZE)]
        rounds.append({"start": round_start, "held": held,
                       "map": [lane_of[k] for k in range(3 * triangles)], "triangles": triangles})
        round_start += 3 * triangles
    return rounds


# --------------------------------------------------------------------------
# whole-buffer counts and reuse metrics
# --------------------------------------------------------------------------

def static_starts(num_tris: int, batch_indices: int):
    """Static batch starts in triangles (with the triangle count appended)."""
    if batch_indices <= 0 or batch_indices % 3:
        raise ValueError("static batch size must be a positive multiple of 3")
    per = batch_indices // 3
    return list(range(0, num_tris, per)) + [num_tris] if num_tris else [0]


def batch_invocations(index_buffer, starts, variant: str, table_size: int = 0):
    """Shader invocations of each batch for one method.

    ``starts`` are batch starts in triangles (from ``static_starts`` or
    ``dynamic_partition``).  variant: ``naive`` (Section 3.3: every corner
    shaded), ``warp`` (Algorithm 1), ``sort`` (Algorithm 2), ``hash`` /
    ``phash`` (Algorithm 3; the parallel variant of Section 3.4 changes how
    slots are found, not which ids are stored).
    """
    out = []
    for b in range(len(starts) - 1):
        lo, hi = 3 * starts[b], 3 * starts[b + 1]
        ids = [int(x) for x in index_buffer[lo:hi]]
        if variant == "naive":
            out.append(hi - lo)
        elif variant == "warp":
            out.append(sum(len(r["held"]) for r in warp_vote_batch(index_buffer, lo, hi)))
        elif variant == "sort":
            out.append(sort_batch(ids)[2])
        elif variant in ("hash", "phash"):
            size = table_size or (1 << max(0, math.ceil(math.log2(max(1, len(ids))))))
            out.append(hash_batch(ids, size)[2])
        else:
            raise ValueError(variant)
    return np.asarray(out, dtype=np.int64)


def unique_per_batch(index_buffer, starts):
    """|set(batch indices)| for every batch, by sorting (batch, id) pairs.

    This is the plain definition of the sort / hash / parallel-hash
    invocation count, usable on full-size buffers."""
    idx = np.asarray(index_buffer, dtype=np.int64)
    st = np.asarray(starts, dtype=np.int64)
    nb = st.size - 1
    if nb <= 0:
        return np.zeros(0, dtype=np.int64)
    tri_batch = np.repeat(np.arange(nb), np.diff(st))
    corner_batch = np.repeat(tri_batch, 3)
    key = corner_batch * (int(idx.max(initial=0)) + 1) + idx
    key = np.unique(key)
    return np.bincount(key // (int(idx.max(initial=0)) + 1), minlength=nb).astype(np.int64)


def ideal_reuse(index_buffer) -> float:
    """Ideal reuse rate (Section 4.1): duplicate indices over the length of the
    index buffer, i.e. 1 - |unique indices| / |indices|."""
    idx = np.asarray(index_buffer)
    if idx.size == 0:
        return 0.0
    return 1.0 - np.unique(idx).size / idx.size


def achieved_reuse(invocations: int, num_indices: int) -> float:
    """Reuse achieved by a method (Table 1, "equivalent to cache hit rates"):
    the fraction of referenced corners that did not need their own shader
    invocation, 1 - invocations / |indices|."""
    return 1.0 - invocations / num_indices if num_indices else 0.0


def shading_rate(invocations: int, referenced_vertices: int) -> float:
    """Shader invocations per referenced vertex (1 is ideal)."""
    return invocations / referenced_vertices if referenced_vertices else 0.0
