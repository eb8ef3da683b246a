// Best-fit allocator of word ranges: the serving loop's device arena (host
// bookkeeping only; plain C++ so that it is tested on the CPU as well).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <functional>
#include <limits>
#include <map>
#include <new>
#include <set>
#include <utility>
#include <vector>

namespace ldpcgb {

// Fixed-size node storage for the arena's two indexes.  A service admits and
// releases requests in its steady-state loop; the indexes then take their tree
// nodes from here, all allocated when the arena is built, instead of from the
// heap, so that loop neither calls the allocator nor touches a page for the
// first time (a page fault there can stall it).  Past its capacity, or for a
// request larger than a node, it falls back to the heap.
class NodePool {
 public:
  static constexpr size_t kNode = 64;  // bytes per node (a tree node of two 64-bit words takes 48)
  explicit NodePool(size_t cap) : store_(cap * kNode) {
    free_.reserve(cap);
    for (size_t i = cap; i-- > 0;) free_.push_back(store_.data() + i * kNode);
  }
  NodePool(const NodePool&) = delete;
  NodePool& operator=(const NodePool&) = delete;
  void* take(size_t bytes) {
    if (bytes <= kNode && !free_.empty()) {
      unsigned char* p = free_.back();
      free_.pop_back();
      return p;
    }
    return ::operator new(bytes);
  }
  void give(void* p, size_t bytes) {
    unsigned char* c = static_cast<unsigned char*>(p);
    if (bytes <= kNode && !store_.empty() && c >= store_.data() && c < store_.data() + store_.size())
      free_.push_back(c);  // within the capacity reserved above: never reallocates
    else
      ::operator delete(p);
  }

 private:
  std::vector<unsigned char> store_;  // operator new's alignment; nodes at multiples of 64 bytes
  std::vector<unsigned char*> free_;
};

template <typename T>
struct PoolAlloc {
  using value_type = T;
  NodePool* pool;
  explicit PoolAlloc(NodePool* p) : pool(p) {}
  template <typename U>
  PoolAlloc(const PoolAlloc<U>& o) : pool(o.pool) {}
  T* allocate(size_t n) { return static_cast<T*>(pool->take(n * sizeof(T))); }
  void deallocate(T* p, size_t n) { pool->give(p, n * sizeof(T)); }
  template <typename U>
  bool operator==(const PoolAlloc<U>& o) const { return pool == o.pool; }
  template <typename U>
  bool operator!=(const PoolAlloc<U>& o) const { return pool != o.pool; }
};

// Device arena of the admitted requests' state, best fit in O(log n): free
// blocks indexed by offset (to merge neighbours) and by (length, offset).
// (A first-fit scan of the offset-ordered list cost a time linear in the
// number of holes, which grows with the requests in flight: under a burst the
// host could fall behind the arrivals and stay behind.)
struct Arena {
  using Off = std::map<int64_t, int64_t, std::less<int64_t>, PoolAlloc<std::pair<const int64_t, int64_t>>>;
  using Len = std::set<std::pair<int64_t, int64_t>, std::less<std::pair<int64_t, int64_t>>,
                       PoolAlloc<std::pair<int64_t, int64_t>>>;
  NodePool pool;  // (declared first: the indexes use it)
  Off by_off;     // free: offset -> length
  Len by_len;     // free: (length, offset)
  // node_cap: nodes held in reserve, two per free block (k live allocations leave at most k + 1)
  explicit Arena(int64_t words, size_t node_cap = 64)
      : pool(node_cap), by_off(Off::allocator_type(&pool)), by_len(Len::allocator_type(&pool)) {
    add(0, words);
  }
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;
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
