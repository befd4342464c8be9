"""Batch formation and per-batch shading-invocation counts, replayed on the CPU.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Each function follows one step of the paper (Kenzel et al., Section 3) in the
paper's order and notation.  Where the printed pseudocode is garbled or
ambiguous the reading taken is stated in the docstring; the full list of
readings is kept with the design notes.  Pure-Python loops: meant for small
inputs or sampled batches of large ones.
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
    """Dynamically batched sorting (Algorithm 2).

    ids[i] <- indexBuffer[BatchBegin + i], linIds[i] <- i; sort the pairs by
    id (stable, as a radix sort is); marks[i] = 1 where ids[i] != ids[i+1]
    (reading: ids[size] acts as a sentinel, so the last element is marked);
    an exclusive prefix sum of marks gives each element its group and
    numVertices; map[linIds[i]] <- group, uniqueIds[group] <- ids[i].

    Returns (map, uniqueIds, numVertices); uniqueIds is in ascending id order.
    """
    size = len(ids)
    pairs = sorted(((int(ids[i]), i) for i in range(size)), key=lambda p: p[0])
    s_ids = [p[0] for p in pairs]
    lin_ids = [p[1] for p in pairs]
    marks = [1 if (i == size - 1 or s_ids[i] != s_ids[i + 1]) else 0 for i in range(size)]
    prefix = []
    run = 0
    for m in marks:
        prefix.append(run)
        run += m
    num_vertices = run
    map_ = [0] * size
    unique_ids = [None] * num_vertices
    for i in range(size):
        map_[lin_ids[i]] = prefix[i]
        unique_ids[prefix[i]] = s_ids[i]
    return map_, unique_ids, num_vertices


def hash_slot(vertex_id: int, table_size: int) -> int:
    """Multiplicative hashing (Section 3.4): the top log2(size) bits of
    (id * A) mod 2^32, A = 2654435769 (the multiplier is not printed; this is
    the reading)."""
    bits = int(math.log2(table_size))
    if 1 << bits != table_size:
        raise ValueError("hash table size must be a power of two")
    return ((int(vertex_id) * HASH_MULTIPLIER) & 0xFFFFFFFF) >> (32 - bits) if bits else 0


def hash_batch(ids, table_size: int):
    """Dynamically batched hashing (Algorithm 3), insertions taken one at a
    time in index order.

    hashtable[.] <- -1; for each index: p <- hash(id); repeat
    prev <- atomicCAS(hashtable[p], -1, id) (reading: the printed
    ``hashtable[i]`` is ``hashtable[p]``); if prev = -1 or prev = id the
    index is placed at p (reading of the garbled ``prev - 1``), else p is
    advanced by linear probing.  map[i] <- p.  Every occupied slot is shaded.

    Returns (hashtable, map, number of occupied slots).  On the GPU the slot
    of an id depends on the order of concurrent insertions; the set of
    occupied ids and the id behind each map entry do not.
    """
    table = [EMPTY] * table_size
    map_ = []
    for vid in ids:
        vid = int(vid)
        p = hash_slot(vid, table_size)
        for _ in range(table_size):
            prev = table[p]
            if prev == EMPTY:
                table[p] = vid
            if prev == EMPTY or prev == vid:
                break
            p = (p + 1) % table_size
        else:
            raise ValueError("hash table full: more unique indices than slots")
        map_.append(p)
    return table, map_, sum(1 for x in table if x != EMPTY)


def warp_vote_batch(index_buffer, batch_begin: int, batch_end: int):
    """Statically batched warp voting (Algorithm 1), one warp of 32 lanes.

    Each outer iteration (a "round") starts with no lane holding a vertex.
    Chunks of 32 indices are read; for i = 0..31 the warp broadcasts lane i's
    index (shfl), asks which lane already holds it (ballot); if none does, the
    lowest free lane ``fill`` takes it.  outgoing[i] is lane i's slot mask.
    The corners before the first lane that found no slot (or lies past the
    batch end) are counted as done.  Chunks are read until every lane holds a
    vertex or the batch ends; then the held vertices are shaded and
    floor(done/3) triangles are written.

    Readings of the printed algorithm:
      * BitShift(1, fill) with fill >= 32 gives "no slot" (mask 0);
      * additional = 32 if firstmask = 0, else ffs(firstmask) - 1 (the
        printed min(WarpSize, ffs(firstmask)) is unbalanced and off by one);
      * cStart advances by 3 * triangles from its current value;
      * all floor(done/3) triangles are written (the printed
        ``laneId < triangles`` only covers batches of at most 96 indices);
      * a vertex of a cut-off triangle is shaded again in the next round and
        counts as another invocation.

    Returns a list of rounds, each a dict with ``start`` (first index of the
    round), ``held`` (the vertex ids of lanes 0..fill-1, i.e. the shader
    invocations), ``map`` (slot of each of the round's 3*triangles corners)
    and ``triangles``.
    """
    rounds = []
    c_start = batch_begin
    while c_start < batch_end:
        fill = 0
        done = 0
        my_id = [EMPTY] * WARP_SIZE
        offset = c_start
        map_ = {}
        while offset < batch_end and fill < WARP_SIZE:
            incoming = [int(index_buffer[offset + lane]) if offset + lane < batch_end else EMPTY
                        for lane in range(WARP_SIZE)]
            outgoing = [EMPTY] * WARP_SIZE
            for i in range(WARP_SIZE):
                current = incoming[i]
                match = 0
                for lane in range(WARP_SIZE):  # ballot(current = my_id)
                    if my_id[lane] == current:
                        match |= 1 << lane
                if match == 0:
                    if fill < WARP_SIZE:
                        my_id[fill] = current
                        match = 1 << fill
                    fill += 1
                outgoing[i] = match
            for lane in range(WARP_SIZE):
                map_[done + lane] = _ffs(outgoing[lane]) - 1
            firstmask = 0
            for lane in range(WARP_SIZE):
                if outgoing[lane] == 0 or incoming[lane] == EMPTY:
                    firstmask |= 1 << lane
            additional = WARP_SIZE if firstmask == 0 else _ffs(firstmask) - 1
            done += additional
            offset += WARP_SIZE
        triangles = done // 3
        held = my_id[:min(fill, WARP_SIZE)]
        rounds.append({"start": c_start, "held": held,
                       "map": [map_[k] for k in range(3 * triangles)], "triangles": triangles})
        c_start += 3 * triangles
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
