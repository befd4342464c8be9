// Parallel per-multiprocessor LRU vertex cache, the cache-based setup the
// paper compares batching against (Section 5.1, Table 1 "Parallel Cache").
//
// The index buffer is split into num_sms contiguous parts; each simulated
// multiprocessor works through its part in shading cycles of `concurrent`
// consecutive indices.  Within
// a cycle every index is looked up in its multiprocessor's cache (a hit
// refreshes the entry); the ids that missed are shaded and inserted when the
// cycle ends, so concurrent duplicates never hit.  The multiprocessors are
// independent, so host threads simulate them side by side.
//
// Each cache is an LRU list over a fixed pool of `capacity` nodes with an
// open-addressing id -> node table (power-of-two size >= 2 x capacity,
// linear probing, backward-shift deletion).
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <thread>
#include <vector>

#include "gp.h"

namespace {

class LruCache {
 public:
  explicit LruCache(uint32_t capacity) : cap_(capacity) {
    uint32_t s = 16;
    while (s < 2 * capacity) s <<= 1;
    mask_ = s - 1;
    slot_.assign(s, kNone);
    id_.resize(capacity);
    prev_.resize(capacity);
    next_.resize(capacity);
  }

  // true (and the entry becomes most recent) if id is cached
  bool touch(uint32_t id) {
    const uint32_t n = find(id);
    if (n == kNone) return false;
    unlink(n);
    push_back(n);
    return true;
  }

  // caches id as the most recent entry, evicting the least recent if full
  void insert(uint32_t id) {
    if (touch(id)) return;
    uint32_t n;
    if (used_ < cap_) {
      n = used_++;
    } else {
      n = head_;
      unlink(n);
      erase(id_[n]);
    }
    id_[n] = id;
    push_back(n);
    uint32_t s = hash(id);
    while (slot_[s] != kNone) s = (s + 1) & mask_;
    slot_[s] = n;
  }

 private:
  static constexpr uint32_t kNone = 0xFFFFFFFFu;
  uint32_t hash(uint32_t id) const { return (id * 2654435769u) & mask_; }

  uint32_t find(uint32_t id) const {
    for (uint32_t s = hash(id);; s = (s + 1) & mask_) {
      const uint32_t n = slot_[s];
      if (n == kNone) return kNone;
      if (id_[n] == id) return n;
    }
  }

  void erase(uint32_t id) {  // backward-shift deletion keeps probe chains intact
    uint32_t s = hash(id);
    while (id_[slot_[s]] != id) s = (s + 1) & mask_;
    uint32_t hole = s;
    for (uint32_t t = (s + 1) & mask_; slot_[t] != kNone; t = (t + 1) & mask_) {
      const uint32_t home = hash(id_[slot_[t]]);
      // move the entry at t into the hole unless its home lies cyclically in (hole, t]
      const bool stays = hole <= t ? (home > hole && home <= t) : (home > hole || home <= t);
      if (!stays) {
        slot_[hole] = slot_[t];
        hole = t;
      }
    }
    slot_[hole] = kNone;
  }

  void unlink(uint32_t n) {
    if (prev_[n] != kNone) next_[prev_[n]] = next_[n]; else head_ = next_[n];
    if (next_[n] != kNone) prev_[next_[n]] = prev_[n]; else tail_ = prev_[n];
  }

  void push_back(uint32_t n) {
    prev_[n] = tail_;
    next_[n] = kNone;
    if (tail_ != kNone) next_[tail_] = n; else head_ = n;
    tail_ = n;
  }

  uint32_t cap_, mask_, used_ = 0, head_ = kNone, tail_ = kNone;
  std::vector<uint32_t> slot_, id_, prev_, next_;
};

uint64_t simulate_sm(const uint32_t* idx, uint64_t n, uint32_t sm, uint32_t num_sms, uint32_t conc,
                     uint32_t capacity) {
  LruCache cache(capacity);
  std::vector<uint32_t> missed;
  missed.reserve(conc);
  uint64_t hits = 0;
  const uint64_t part = (n + num_sms - 1) / num_sms;
  const uint64_t begin = std::min<uint64_t>(n, (uint64_t)sm * part), end = std::min<uint64_t>(n, begin + part);
  for (uint64_t lo = begin; lo < end; lo += conc) {
    const uint64_t hi = std::min<uint64_t>(lo + conc, end);
    missed.clear();
    for (uint64_t i = lo; i < hi; ++i) {
      if (cache.touch(idx[i])) ++hits;
      else missed.push_back(idx[i]);
    }
    for (uint32_t v : missed) cache.insert(v);
  }
  return hits;
}

}  // namespace

extern "C" gp_status gp_simulate_parallel_cache(const uint32_t* indices, uint64_t num_indices, uint32_t num_sms,
                                                uint32_t concurrent, uint32_t capacity_entries, uint32_t threads,
                                                uint64_t* hits) {
  if (!hits || (num_indices && !indices) || num_sms == 0 || concurrent == 0 || capacity_entries == 0 ||
      capacity_entries > (1u << 30))
    return GP_ERR_INVALID;
  const uint32_t hw = std::max(1u, std::thread::hardware_concurrency());
  const uint32_t nt = std::min(num_sms, threads ? threads : hw);
  std::vector<uint64_t> per_sm(num_sms, 0);
  std::atomic<uint32_t> next{0};
  auto worker = [&]() {
    for (uint32_t sm = next.fetch_add(1); sm < num_sms; sm = next.fetch_add(1))
      per_sm[sm] = simulate_sm(indices, num_indices, sm, num_sms, concurrent, capacity_entries);
  };
  std::vector<std::thread> pool;
  for (uint32_t t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (std::thread& t : pool) t.join();
  uint64_t total = 0;
  for (uint64_t h : per_sm) total += h;
  *hits = total;
  return GP_OK;
}
