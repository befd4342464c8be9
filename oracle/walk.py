"""Oracle of the parallel random walk with on-the-fly reuse (Section 5.4).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper runs agents on a 256 x 256 grid with an activity field made of
overlaid Gaussians.  Per step, every agent evaluates all potential moves up
to a distance of 16, keeps the 8 most likely and draws one of them with
probability proportional to its likelihood.  The likelihoods depend only on
the agent's cell, so the agent's packed location ((x << 16) | y) serves as
the "index" whose expensive part (the 8 moves) the reuse methods compute once
per batch.

Readings (the paper leaves them open):

* The grid is a torus.  The candidate moves are the offsets (dx, dy) with
  1 <= dx^2 + dy^2 <= 16^2, in row-major order (dy, then dx, each from -16 to
  16); that order breaks ties.
* A move's likelihood is the integer A[target] * (65536 // r^2), with A the
  quantised activity field (``meshgen.walk_activity``) and r^2 = dx^2 + dy^2:
  the activity of the destination under an inverse-square (Levy-type) step
  length law.  Integers make every comparison exact on both sides.
* The 8 moves with the largest likelihoods are kept (equal ones: the earlier
  candidate first).
* Agent i at step s draws u = splitmix64(seed ^ ((s << 32) | i)) (SplitMix64,
  Steele, Lea & Flood, OOPSLA 2014; the finaliser of Vigna's reference code)
  and takes the first kept move whose running sum of likelihoods exceeds
  u mod (their total); with a total of 0 it stays.
"""
from functools import lru_cache

import numpy as np

RADIUS = 16
KEEP = 8
MASK64 = (1 << 64) - 1


@lru_cache(maxsize=None)
def candidate_offsets(radius: int = RADIUS):
    """The potential moves, in tie-breaking order: (dx, dy, r^2)."""
    out = []
    for dy in range(-radius, radius + 1):
        for dx in range(-radius, radius + 1):
            r2 = dx * dx + dy * dy
            if 1 <= r2 <= radius * radius:
                out.append((dx, dy, r2))
    return tuple(out)


def splitmix64(x: int) -> int:
    """SplitMix64 output for the state x (one increment, then the mix)."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def cell_moves(activity, x: int, y: int, radius: int = RADIUS, keep: int = KEEP):
    """The kept moves of cell (x, y): list of (dx, dy, likelihood), most likely first."""
    h, w = activity.shape
    cand = np.array(candidate_offsets(radius), dtype=np.int64)
    dx, dy, r2 = cand[:, 0], cand[:, 1], cand[:, 2]
    lik = activity[(y + dy) % h, (x + dx) % w].astype(np.int64) * (65536 // r2)
    order = np.lexsort((np.arange(len(cand)), -lik))[:keep]  # by likelihood, then candidate order
    return [(int(dx[j]), int(dy[j]), int(lik[j])) for j in order]


def choose(moves, u: int):
    """The move drawn with the 64-bit random number u ((0, 0) -- stay -- when
    no kept move has a positive likelihood)."""
    total = sum(m[2] for m in moves)
    if total == 0:
        return 0, 0
    r = u % total
    acc = 0
    for dx, dy, lk in moves:
        acc += lk
        if acc > r:
            return dx, dy
    raise AssertionError("unreachable: r < total")


def step(activity, keys, step_index: int, seed: int):
    """One step of every agent; keys are packed (x << 16) | y.  Returns the new keys."""
    h, w = activity.shape
    cache = {}
    out = np.empty_like(keys)
    for i, k in enumerate(keys.tolist()):
        if k not in cache:
            cache[k] = cell_moves(activity, k >> 16, k & 0xFFFF)
        dx, dy = choose(cache[k], splitmix64(seed ^ ((step_index << 32) | i)))
        out[i] = (((k >> 16) + dx) % w) << 16 | (((k & 0xFFFF) + dy) % h)
    return out


def run(activity, keys, steps: int, seed: int):
    """Positions after `steps` steps, and the keys of every step (for the counts)."""
    history = [keys]
    for s in range(steps):
        history.append(step(activity, history[-1], s, seed))
    return history[-1], history


def batch_invocations(keys, variant: str, batch: int):
    """Evaluations of the kept moves per batch of `batch` agents in one step:
    every agent (naive); the unique keys of each run of 32 agents, summed over
    the batch's runs (warp); the unique keys of the batch (sort / hash /
    phash).  For warp, `batch` is a multiple of 32."""
    n = len(keys)
    out = []
    for b in range(0, n, batch):
        chunk = keys[b:b + batch]
        if variant == "naive":
            out.append(len(chunk))
        elif variant == "warp":
            out.append(sum(len(np.unique(chunk[j:j + 32])) for j in range(0, len(chunk), 32)))
        else:
            out.append(len(np.unique(chunk)))
    return np.array(out, dtype=np.int64)
