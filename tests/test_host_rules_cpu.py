"""Host rules shared by the batch session and the serving loop (csrc/host_rules.h), compiled with the
host compiler: the redundancy versions' start and decoded columns against the oracle's geometry, the
serving loop's choice of the INT8 decode form (pairing by load, with hysteresis), and its completion-ring
consumer under injected faults (records missing, stale, corrupted or repeated)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import demap as odemap

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2506_00167_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstring>
#include "host_rules.h"

// "g nb npc Z rv E" -> "k0 cols" (cols -1 when k0 is -1)
// "p pairs always threshold release" starts a policy; "c inflight n_single fits_single fits_pair" -> 0/1
int main() {
  char op[4];
  ldpcgb::PairPolicy pol;
  while (std::scanf("%3s", op) == 1) {
    if (!std::strcmp(op, "g")) {
      int nb, npc, Z, rv, E;
      if (std::scanf("%d %d %d %d %d", &nb, &npc, &Z, &rv, &E) != 5) return 2;
      const int k0 = ldpcgb::rv_k0(nb - npc, rv, Z);
      const int cols = k0 < 0 ? -1 : ldpcgb::decoded_cols(nb, Z, npc * Z, k0, E);
      std::printf("%d %d\n", k0, cols);
    } else if (!std::strcmp(op, "p")) {
      int pairs, always;
      long long thr, rel;
      if (std::scanf("%d %d %lld %lld", &pairs, &always, &thr, &rel) != 4) return 2;
      pol = ldpcgb::PairPolicy();
      pol.pairs = pairs != 0;
      pol.always = always != 0;
      pol.threshold = thr;
      pol.release = rel;
    } else if (!std::strcmp(op, "c")) {
      long long inflight;
      int n_single, fs, fp;
      if (std::scanf("%lld %d %d %d", &inflight, &n_single, &fs, &fp) != 4) return 2;
      std::printf("%d\n", pol.choose(inflight, n_single, fs != 0, fp != 0) ? 1 : 0);
    } else {
      return 2;
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("host_rules")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(lines):
        r = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=60)
        assert r.returncode == 0, r.stderr
        return r.stdout.split("\n")[:-1]
    return run


def test_redundancy_version_start_and_columns_match_the_oracle(driver):
    # buffers of 66 Z (BG1-shaped: 68 columns, 2 punctured) and 50 Z (52, 2), and one of neither length
    rng = np.random.default_rng(31)
    cases = []
    for nb, npc in [(68, 2), (52, 2), (16, 0)]:
        for Z in (16, 32, 64, 384):
            ncb = nb * Z - npc * Z
            for rv in range(4):
                for E in list(rng.integers(1, 2 * ncb + 1, size=6)) + [ncb, ncb + 1, 2 * ncb]:
                    cases.append((nb, npc, Z, rv, int(E)))
    out = driver([f"g {nb} {npc} {Z} {rv} {E}" for nb, npc, Z, rv, E in cases])
    for (nb, npc, Z, rv, E), line in zip(cases, out):
        k0, cols = map(int, line.split())
        try:
            want_k0 = odemap.start_k0(nb, npc, Z, rv)
        except ValueError:
            assert (k0, cols) == (-1, -1), (nb, npc, Z, rv, E)
            continue
        assert k0 == want_k0, (nb, npc, Z, rv, E)
        # the oracle's column rule: n_eff = kb + m_eff with m_eff = cols - kb whenever cols - kb lies in
        # [mc, mb]; take kb = 0, mc = 0, mb = nb so that n_eff is the column count itself
        _, _, n_eff = odemap.geometry(nb, nb, 0, 0, npc, Z, E, rv)
        assert cols == n_eff, (nb, npc, Z, rv, E)


def _policy_reference(pairs, always, thr, rel, steps):
    """The rule restated: pairing starts when inflight + n_single exceeds thr and stops when it falls to
    rel or below; a request is paired if the paired form is available and fits, and the service pairs
    always, or only the paired form fits, or the load rule is pairing."""
    state, out = False, []
    for inflight, n_single, fs, fp in steps:
        load = inflight + n_single
        if load > thr:
            state = True
        elif load <= rel:
            state = False
        out.append(int(pairs and fp and (always or not fs or state)))
    return out


@pytest.mark.parametrize("pairs,always,thr,rel", [(1, 0, 304, 152), (1, 0, 152, 152), (1, 1, 304, 152),
                                                   (0, 0, 304, 152), (1, 0, 10, 2)])
def test_pairing_policy_follows_the_load_with_hysteresis(driver, pairs, always, thr, rel):
    rng = np.random.default_rng(thr + rel + 7 * always + 3 * pairs)
    steps = []
    inflight = 0
    for _ in range(4000):
        inflight = max(0, inflight + int(rng.integers(-40, 41)))
        steps.append((inflight, int(rng.integers(0, 17)), int(rng.random() < 0.95), int(rng.random() < 0.9)))
    lines = [f"p {pairs} {always} {thr} {rel}"] + [f"c {a} {b} {c} {d}" for a, b, c, d in steps]
    got = list(map(int, driver(lines)))
    assert got == _policy_reference(pairs, always, thr, rel, steps)


def test_pairing_policy_hysteresis_by_hand(driver):
    # threshold 300, release 150: single up to 300, paired above it, stays paired down to 151, single at 150
    seq = [(100, 0), (300, 0), (301, 0), (250, 0), (151, 0), (150, 0), (200, 0), (290, 11)]
    lines = ["p 1 0 300 150"] + [f"c {a} {b} 1 1" for a, b in seq]
    assert list(map(int, driver(lines))) == [0, 0, 1, 1, 1, 0, 0, 1]
    # only the paired form fits: paired at any load; only the single form fits: never paired
    assert list(map(int, driver(["p 1 0 300 150", "c 0 1 0 1", "c 999 1 1 0"]))) == [1, 0]


RING_DRIVER = r"""
#include <cstdio>
#include <cstring>
#include <set>
#include "host_rules.h"

struct Rec { unsigned long long tag; int req; unsigned seq; };

// A ring of 4 records.  Commands: "w q req" writes record number q (slot (q-1) % 4, sequence word
// last); "x slot word" overwrites a slot's sequence word; "d max" drains up to max records and prints
// "n rd bad taken-tags..."; a record is rejected when its request is not in flight, and taking one
// ends its request ("s req" puts a request in flight).
int main() {
  Rec ring[4];
  std::memset(ring, 0, sizeof ring);
  unsigned rd = 0;
  std::set<int> inflight;
  char op[4];
  while (std::scanf("%3s", op) == 1) {
    if (!std::strcmp(op, "s")) {
      int req;
      if (std::scanf("%d", &req) != 1) return 2;
      inflight.insert(req);
    } else if (!std::strcmp(op, "w")) {
      unsigned q;
      int req;
      if (std::scanf("%u %d", &q, &req) != 2) return 2;
      Rec& r = ring[(q - 1) % 4];
      r.tag = 1000 + q;
      r.req = req;
      r.seq = q;
    } else if (!std::strcmp(op, "x")) {
      unsigned slot, word;
      if (std::scanf("%u %u", &slot, &word) != 2) return 2;
      ring[slot].seq = word;
    } else if (!std::strcmp(op, "d")) {
      int max;
      if (std::scanf("%d", &max) != 1) return 2;
      bool bad = false;
      unsigned long long tags[16];
      int k = 0;
      const int n = ldpcgb::drain_ring(static_cast<volatile Rec*>(ring), 4u, rd, max, [&](volatile Rec* r) {
        const int req = r->req;
        if (!inflight.count(req)) return false;
        inflight.erase(req);
        tags[k++] = r->tag;
        return true;
      }, &bad);
      std::printf("%d %u %d", n, rd, bad ? 1 : 0);
      for (int i = 0; i < k; ++i) std::printf(" %llu", tags[i]);
      std::printf("\n");
    } else {
      return 2;
    }
  }
  return 0;
}
"""


def test_completion_ring_under_injected_faults(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "ring.cpp"
    src.write_text(RING_DRIVER)
    exe = tmp_path / "ring"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    script = [
        "s 0", "s 1", "s 2", "s 3", "s 4", "s 5", "s 6",
        "d 8",                 # nothing written yet
        "w 1 0", "w 2 1", "w 4 3",
        "d 8",                 # 1 and 2; record 3 is missing, so 4 waits
        "w 3 2",
        "d 1",                 # at most one per call
        "d 8",                 # then 4
        "d 8",                 # slot 0 still holds record 1 from the previous lap: not record 5
        "x 0 4294967295",      # a corrupted sequence word in the slot of record 5
        "d 8",
        "w 5 4", "w 6 1",      # record 6 repeats request 1, completed long ago
        "d 8",                 # 5 is taken, 6 is rejected and stays
        "d 8",                 # still rejected: the ring does not move past it
    ]
    r = subprocess.run([str(exe)], input="\n".join(script) + "\n", capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    assert r.stdout.split("\n")[:-1] == [
        "0 0 0",
        "2 2 0 1001 1002",
        "1 3 0 1003",
        "1 4 0 1004",
        "0 4 0",
        "0 4 0",
        "1 5 1 1005",
        "0 5 1",
    ]
