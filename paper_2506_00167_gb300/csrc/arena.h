// Best-fit allocator of word ranges: the serving loop's device arena (host
// bookkeeping only; plain C++ so that it is tested on the CPU as well).
#pragma once

#include <stdint.h>

#include <limits>
#include <map>
#include <set>
#include <utility>

namespace ldpcgb {

// Device arena of the admitted requests' state, best fit in O(log n): free
// blocks indexed by offset (to merge neighbours) and by (length, offset).
// (A first-fit scan of the offset-ordered list cost a time linear in the
// number of holes, which grows with the requests in flight: under a burst the
// host could fall behind the arrivals and stay behind.)
struct Arena {
  std::map<int64_t, int64_t> by_off;               // free: offset -> length
  std::set<std::pair<int64_t, int64_t>> by_len;    // free: (length, offset)
  explicit Arena(int64_t words) { add(0, words); }
  void add(int64_t off, int64_t n) {
    by_off[off] = n;
    by_len.emplace(n, off);
  }
  void remove(int64_t off, int64_t n) {
    by_off.erase(off);
    by_len.erase({n, off});
  }
  int64_t alloc(int64_t n) {
    auto it = by_len.lower_bound({n, std::numeric_limits<int64_t>::min()});
    if (it == by_len.end()) return -1;
    const int64_t len = it->first, off = it->second;
    remove(off, len);
    if (len > n) add(off + n, len - n);
    return off;
  }
  void release(int64_t off, int64_t n) {
    auto nx = by_off.lower_bound(off);
    if (nx != by_off.end() && off + n == nx->first) {
      const int64_t o = nx->first, l = nx->second;
      remove(o, l);
      n += l;
    }
    auto pv = by_off.lower_bound(off);
    if (pv != by_off.begin()) {
      --pv;
      if (pv->first + pv->second == off) {
        const int64_t o = pv->first, l = pv->second;
        remove(o, l);
        off = o;
        n += l;
      }
    }
    add(off, n);
  }
};

}  // namespace ldpcgb
