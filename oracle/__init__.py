"""Plain CPU oracle for batch-based on-the-fly vertex reuse.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The library (``paper_1805_08893_gb300``) never imports it and shares
no code, table or constant with it; both sides only read the seeded inputs of
``meshgen``.

Two parts (Kenzel et al., "On-the-fly Vertex Reuse for Massively-Parallel
Software Geometry Processing"):

* ``shading`` -- the result every method must reach: corner k of triangle t
  is ``shade(vertexBuffer[indexBuffer[3t+k]])`` (Section 3: each referenced
  vertex is shaded, triangles are assembled from the results).  Written out
  in float64 from the definition; no reuse.
* ``batching`` -- the method's own bookkeeping that the plain definition does
  not fix: static and dynamic batch boundaries (Sections 3.3, 3.4), and the
  shading-invocation counts of warp voting (Algorithm 1), sorting
  (Algorithm 2) and hashing (Algorithm 3), replayed step by step.
* ``cache_sim`` -- the simulated per-multiprocessor LRU vertex cache the paper
  compares batching against (Section 5.1, Table 1).
* ``walk`` and ``loop`` -- the applications of Section 5: the parallel random
  walk (5.4) and Loop subdivision (5.2).

Every function's docstring cites the passage it follows.  Pins (closed forms,
hand-worked cases, brute force, the paper's printed numbers) live in
``tests/test_oracle_*.py`` and ``tests/golden/``.
"""
from . import batching, cache_sim, loop, shading, walk  # noqa: F401
