// Host check of the serving loop's arena regions (roix_regions.h): first fit,
// largest gap, exhaustion, reuse of freed gaps, accounting of bytes in use.
#include <cstdio>
#include <cstdlib>

#include "roix_regions.h"

#define CHECK(c)                                              \
  do {                                                        \
    if (!(c)) {                                               \
      std::printf("FAILED line %d: %s\n", __LINE__, #c);      \
      return 1;                                               \
    }                                                         \
  } while (0)

int main() {
  roix::Regions r;
  r.size = 1000;
  CHECK(r.largest_gap() == 1000);
  const uint64_t a = r.take(300), b = r.take(300), c = r.take(300);
  CHECK(a == 0 && b == 300 && c == 600);
  CHECK(r.in_use == 900 && r.largest_gap() == 100);
  CHECK(r.take(101) == ~0ull);           // nothing that large is free
  CHECK(r.give(b) && !r.give(b));        // a region is freed once
  CHECK(r.largest_gap() == 300 && r.in_use == 600);
  CHECK(r.take(200) == 300);             // first fit: the freed middle gap
  CHECK(r.take(100) == 500);             // the rest of that gap
  CHECK(r.take(100) == 900);             // then the tail
  CHECK(r.largest_gap() == 0 && r.in_use == 1000);
  CHECK(r.give(0) && r.give(300) && r.give(500));
  CHECK(r.largest_gap() == 600);         // 0..600 free again, 600..1000 in use
  CHECK(r.take(600) == 0 && r.take(1) == ~0ull);
  CHECK(r.give(0) && r.give(600) && r.give(900) && r.used.empty() && r.in_use == 0);
  // random sequences: regions stay disjoint, sorted, inside the arena, and
  // largest_gap() is the largest size take() can satisfy
  srand(7);
  roix::Regions q;
  q.size = 1 << 20;
  for (int it = 0; it < 20000; ++it) {
    if (rand() % 3 && !q.used.empty()) {
      q.give(q.used[(size_t)rand() % q.used.size()].first);
    } else {
      const uint64_t want = 1 + (uint64_t)(rand() % 70000);
      const uint64_t g = q.largest_gap();
      const uint64_t off = q.take(want);
      CHECK((off == ~0ull) == (want > g));
    }
    uint64_t at = 0, sum = 0;
    for (const auto& u : q.used) {
      CHECK(u.first >= at && u.first + u.second <= q.size);
      at = u.first + u.second;
      sum += u.second;
    }
    CHECK(sum == q.in_use);
  }
  std::printf("ok\n");
  return 0;
}
