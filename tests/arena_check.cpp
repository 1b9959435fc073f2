// Randomized check of the serving engine's range allocator against a plain
// byte-ownership model: allocations never overlap, stay inside the arena, are
// aligned, are refused only when no free range is large enough, and freeing
// everything merges the arena back into one range.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "lg_arena.h"

static int fail(const char* what, int step) {
  std::printf("FAIL %s at step %d\n", what, step);
  return 1;
}

int main(int argc, char** argv) {
  const uint64_t size = 1 << 16, align = 64;
  std::mt19937_64 rng(argc > 1 ? std::strtoull(argv[1], nullptr, 10) : 7);
  lg::RangeArena a;
  a.init(size, align);
  std::vector<int> owner(size, -1);  // model: byte -> live allocation id
  struct Live { uint64_t off, len; };
  std::vector<Live> live;
  for (int step = 0; step < 200000; step++) {
    if (live.empty() || rng() % 3 != 0) {
      const uint64_t want = 1 + rng() % (rng() % 8 == 0 ? 8192 : 600);
      uint64_t off;
      const uint64_t len = (want + align - 1) / align * align;
      // largest run of free bytes at aligned starts, from the model
      uint64_t best = 0;
      for (uint64_t o = 0; o < size; o += align) {
        uint64_t r = 0;
        while (o + r < size && owner[o + r] < 0) r++;
        if (r > best) best = r;
        o += r / align * align;
      }
      if (!a.alloc(want, &off)) {
        if (best >= len) return fail("refused although a range fits", step);
        continue;
      }
      if (off % align) return fail("misaligned", step);
      if (off + len > size) return fail("outside the arena", step);
      for (uint64_t b = off; b < off + len; b++) {
        if (owner[b] >= 0) return fail("overlap", step);
        owner[b] = step;
      }
      live.push_back({off, len});
    } else {
      const size_t i = rng() % live.size();
      if (!a.release(live[i].off)) return fail("release of a live range refused", step);
      for (uint64_t b = live[i].off; b < live[i].off + live[i].len; b++) owner[b] = -1;
      live[i] = live.back();
      live.pop_back();
    }
    uint64_t used = 0;
    for (auto& l : live) used += l.len;
    if (used != a.used()) return fail("used bytes", step);
  }
  if (a.release(12345)) return fail("release of an unknown offset accepted", -1);
  for (auto& l : live) a.release(l.off);
  if (a.used() != 0 || a.free_ranges() != 1 || a.largest_free() != size) return fail("final merge", -1);
  std::printf("ok peak=%llu\n", (unsigned long long)a.peak());
  return 0;
}
