// First-fit regions of one fixed arena (host code, no CUDA): the serving
// loop's workspace memory. Regions in use are kept sorted by offset; a free
// gap is the space between two of them (or before the first, after the last).
#ifndef ROIX_REGIONS_H_
#define ROIX_REGIONS_H_

#include <cstdint>
#include <utility>
#include <vector>

namespace roix {

struct Regions {
  uint64_t size = 0;                                 // bytes of the arena
  std::vector<std::pair<uint64_t, uint64_t>> used;  // (offset, bytes), by offset
  uint64_t in_use = 0;

  // Bytes of the largest free gap.
  uint64_t largest_gap() const {
    uint64_t best = 0, at = 0;
    for (const auto& r : used) {
      if (r.first > at && r.first - at > best) best = r.first - at;
      at = r.first + r.second;
    }
    if (size > at && size - at > best) best = size - at;
    return best;
  }

  // The first gap of at least `bytes` (lowest offset): its offset, now in
  // use; ~0 when no gap is large enough.
  uint64_t take(uint64_t bytes) {
    uint64_t at = 0;
    size_t k = 0;
    for (; k <= used.size(); ++k) {
      const uint64_t next = k < used.size() ? used[k].first : size;
      if (next >= at && next - at >= bytes) break;
      if (k < used.size()) at = used[k].first + used[k].second;
    }
    if (k > used.size()) return ~0ull;
    used.insert(used.begin() + (long)k, {at, bytes});
    in_use += bytes;
    return at;
  }

  // Frees the region that starts at `off` (false: no such region).
  bool give(uint64_t off) {
    for (size_t k = 0; k < used.size(); ++k)
      if (used[k].first == off) {
        in_use -= used[k].second;
        used.erase(used.begin() + (long)k);
        return true;
      }
    return false;
  }
};

}  // namespace roix

#endif  // ROIX_REGIONS_H_
