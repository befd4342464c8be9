// Adjacency for Loop subdivision (Section 5.2), built once per mesh on the
// host: the vertices' 1-rings and, for every triangle edge, the vertex
// opposite it in the neighbouring triangle.
//
// Rings: an interior vertex lists its distinct neighbours (in order of first
// appearance in the index buffer); a boundary vertex -- one with an edge used
// by a single triangle -- lists only its two boundary neighbours and is
// flagged, since Loop's boundary rule uses them alone.
#include <algorithm>
#include <cstdint>
#include <unordered_map>
#include <vector>

#include "gp.h"

namespace {
constexpr uint32_t kNone = 0xFFFFFFFFu;
inline uint64_t edge_key(uint32_t a, uint32_t b) { return ((uint64_t)a << 32) | b; }
}  // namespace

extern "C" gp_status gp_loop_adjacency(const uint32_t* indices, uint64_t num_indices, uint32_t num_vertices,
                                       uint32_t* ring_offsets, uint32_t* ring, uint64_t ring_capacity,
                                       uint32_t* opposite, uint32_t* vertex_flags, uint64_t* ring_count) {
  if ((num_indices && !indices) || num_indices % 3 || !ring_offsets || !vertex_flags || !ring_count ||
      (num_indices && !opposite))
    return GP_ERR_INVALID;
  const uint64_t T = num_indices / 3;
  for (uint64_t i = 0; i < num_indices; ++i)
    if (indices[i] >= num_vertices) return GP_ERR_INDEX_RANGE;
  // directed edge (a, b) of triangle t -> the third vertex of t
  std::unordered_map<uint64_t, uint32_t> third;
  third.reserve((size_t)num_indices * 2);
  for (uint64_t t = 0; t < T; ++t)
    for (int k = 0; k < 3; ++k) {
      const uint32_t a = indices[3 * t + k], b = indices[3 * t + (k + 1) % 3], c = indices[3 * t + (k + 2) % 3];
      third[edge_key(a, b)] = c;
    }
  // opposite vertex across each edge: the third vertex of the twin (b, a)
  std::vector<uint8_t> boundary(num_vertices, 0);
  std::vector<std::vector<uint32_t>> bnb(num_vertices);  // boundary neighbours
  for (uint64_t t = 0; t < T; ++t)
    for (int k = 0; k < 3; ++k) {
      const uint32_t a = indices[3 * t + k], b = indices[3 * t + (k + 1) % 3];
      const auto it = third.find(edge_key(b, a));
      opposite[3 * t + k] = it == third.end() ? kNone : it->second;
      if (it == third.end()) {
        boundary[a] = boundary[b] = 1;
        bnb[a].push_back(b);
        bnb[b].push_back(a);
      }
    }
  // rings
  std::vector<std::vector<uint32_t>> nb(num_vertices);
  for (uint64_t t = 0; t < T; ++t)
    for (int k = 0; k < 3; ++k) {
      const uint32_t a = indices[3 * t + k];
      for (int j = 1; j < 3; ++j) {
        const uint32_t b = indices[3 * t + (k + j) % 3];
        if (std::find(nb[a].begin(), nb[a].end(), b) == nb[a].end()) nb[a].push_back(b);
      }
    }
  uint64_t total = 0;
  for (uint32_t v = 0; v < num_vertices; ++v) {
    ring_offsets[v] = (uint32_t)std::min<uint64_t>(total, 0xFFFFFFFFu);
    const std::vector<uint32_t>& r = boundary[v] && bnb[v].size() == 2 ? bnb[v] : nb[v];
    vertex_flags[v] = boundary[v] && bnb[v].size() == 2 ? 1u : 0u;
    if (ring && total + r.size() <= ring_capacity) std::copy(r.begin(), r.end(), ring + total);
    total += r.size();
  }
  ring_offsets[num_vertices] = (uint32_t)std::min<uint64_t>(total, 0xFFFFFFFFu);
  *ring_count = total;
  if (total >= 0xFFFFFFFFull) return GP_ERR_UNSUPPORTED;
  if (ring && total > ring_capacity) return GP_ERR_INVALID;
  return GP_OK;
}
