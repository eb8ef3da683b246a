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
