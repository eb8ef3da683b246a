"""Host logic: the serving arena's best-fit allocator (csrc/arena.h), compiled with the host compiler and
driven through random allocate / release sequences with requests completing out of order."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2506_00167_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <vector>
#include "arena.h"

int main() {
  const int64_t total = 1 << 20;
  ldpcgb::Arena a(total);
  std::mt19937_64 rng(7);
  std::map<int64_t, int64_t> live;  // offset -> length
  for (int step = 0; step < 200000; ++step) {
    if (live.empty() || rng() % 100 < 55) {
      const int64_t n = 1 + static_cast<int64_t>(rng() % 4300);
      // best fit expected: the smallest free block that holds n (lowest offset among equals)
      int64_t want = -1, want_len = 0;
      for (auto& f : a.by_off)
        if (f.second >= n && (want < 0 || f.second < want_len)) { want = f.first; want_len = f.second; }
      const int64_t off = a.alloc(n);
      if (off != want) { std::printf("best fit: got %lld want %lld\n", (long long)off, (long long)want); return 1; }
      if (off < 0) continue;
      auto nx = live.lower_bound(off);
      if (nx != live.end() && nx->first < off + n) { std::printf("overlap after\n"); return 1; }
      if (nx != live.begin()) { auto pv = std::prev(nx); if (pv->first + pv->second > off) { std::printf("overlap before\n"); return 1; } }
      live[off] = n;
    } else {
      auto it = live.begin();
      std::advance(it, static_cast<long>(rng() % live.size()));  // out of order
      a.release(it->first, it->second);
      live.erase(it);
    }
    // the free blocks never touch (they are merged), never overlap the live ones, and the books balance
    int64_t free_words = 0, prev_end = -1;
    for (auto& f : a.by_off) {
      if (f.first <= prev_end) { std::printf("unmerged or overlapping free blocks\n"); return 1; }
      prev_end = f.first + f.second;
      free_words += f.second;
    }
    if (a.by_len.size() != a.by_off.size()) { std::printf("index sizes differ\n"); return 1; }
    int64_t used = 0;
    for (auto& l : live) used += l.second;
    if (used + free_words != total) { std::printf("books do not balance\n"); return 1; }
  }
  for (auto& l : live) a.release(l.first, l.second);
  if (a.by_off.size() != 1 || a.by_off.begin()->second != total) { std::printf("not whole again\n"); return 1; }
  std::printf("ok\n");
  return 0;
}
"""


def test_arena_best_fit_invariants(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "arena_driver.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "arena_driver"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


DRIVER_NOALLOC = r"""
#include <cstdio>
#include <cstdlib>
#include <new>
#include <random>
#include <vector>
#include "arena.h"

static bool counting = false;
static long heap_calls = 0;
void* operator new(std::size_t n) {
  if (counting) ++heap_calls;
  if (void* p = std::malloc(n ? n : 1)) return p;
  throw std::bad_alloc();
}
void operator delete(void* p) noexcept { std::free(p); }
void operator delete(void* p, std::size_t) noexcept { std::free(p); }

int main() {
  const int max_live = 4000;
  ldpcgb::Arena a(1 << 24, 2 * max_live + 8);
  std::mt19937_64 rng(11);
  std::vector<std::pair<long long, long long>> live;
  live.reserve(max_live);
  for (int step = 0; step < 300000; ++step) {
    if (live.empty() || (live.size() < static_cast<size_t>(max_live) && rng() % 100 < 52)) {
      const long long n = 1 + static_cast<long long>(rng() % 3000);
      counting = true;
      const long long off = a.alloc(n);
      counting = false;
      if (off >= 0) live.emplace_back(off, n);
    } else {
      const size_t i = static_cast<size_t>(rng() % live.size());  // out of order
      counting = true;
      a.release(live[i].first, live[i].second);
      counting = false;
      live[i] = live.back();
      live.pop_back();
    }
  }
  std::printf("%ld\n", heap_calls);
  return 0;
}
"""


def test_arena_steady_state_allocates_nothing(tmp_path):
    """With its node pool sized for the requests in flight (two tree nodes per free block), admitting and
    releasing requests never calls the heap: the serving loop's host side stays allocation-free."""
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "arena_noalloc.cpp"
    src.write_text(DRIVER_NOALLOC)
    exe = tmp_path / "arena_noalloc"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "0", r.stdout + r.stderr
