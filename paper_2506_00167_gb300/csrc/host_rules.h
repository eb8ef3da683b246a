// Host-side rules shared by the batch session and the serving loop: plain C++
// so that they are tested on the CPU as well.
#pragma once

#include <stdint.h>

#include <atomic>

namespace ldpcgb {

// Start k0 of redundancy version rv (0..3) in a circular buffer of buf_cols
// columns of Z positions: NR's table for buffers of 66 Z and 50 Z positions
// (the two base-graph sizes); -1 for versions 1-3 of any other buffer.
inline int rv_k0(int buf_cols, int rv, int Z) {
  static const int units66[4] = {0, 17, 33, 56}, units50[4] = {0, 13, 25, 43};
  if (rv == 0) return 0;
  if (rv < 0 || rv > 3) return -1;
  if (buf_cols == 66) return units66[rv] * Z;
  if (buf_cols == 50) return units50[rv] * Z;
  return -1;
}

// Columns decoded for a block sent from k0 with E bits: up to the last
// position sent (t0 + k0 + E), all nb when the bits wrap the buffer of
// nb * Z - t0 positions.
inline int decoded_cols(int nb, int Z, int t0, int k0, int E) {
  const int ncb = nb * Z - t0;
  return k0 + E > ncb ? nb : (t0 + k0 + E + Z - 1) / Z;
}

// The serving loop's per-request choice of the INT8 decode form.  Paired
// (two code blocks per thread group) once the work items in flight together
// with the request's own single-form items exceed `threshold`, and until they
// fall to `release`; always or never when the service fixes the form; the
// form that fits when the shape fits only one.
struct PairPolicy {
  bool pairs = false;      // the paired form is available at all (INT8, not fixed to single)
  bool always = false;     // fixed to paired
  int64_t threshold = 0;   // start pairing above this many items in flight
  int64_t release = 0;     // stop at or below this many (release <= threshold)
  bool pairing = false;    // state of the load rule

  // n_single: the request's items in the single form (0 if that form does not fit the shape);
  // fits_pair: the shape fits the paired form.
  bool choose(int64_t inflight, int n_single, bool fits_single, bool fits_pair) {
    const int64_t load = inflight + n_single;
    if (load > threshold)
      pairing = true;
    else if (load <= release)
      pairing = false;
    return pairs && fits_pair && (always || !fits_single || pairing);
  }
};

// Consumer of a device -> host completion ring: record number q (from 1)
// sits in slot (q - 1) mod cap and is complete once its sequence word reads q
// (the writer stores it last, after a system fence).  Records are taken in
// order from number rd + 1; a slot whose word is not the next number -- not
// yet written, left from the previous lap, or corrupted -- ends the drain, and
// so does a record whose contents `take` rejects (returns false): then *bad is
// set and rd stays on that record.  Returns the records taken.
template <typename Rec, typename Take>
int drain_ring(volatile Rec* ring, uint32_t cap, uint32_t& rd, int max, Take take, bool* bad) {
  int n = 0;
  *bad = false;
  while (n < max) {
    volatile Rec* r = ring + (rd % cap);
    if (r->seq != rd + 1u) break;
    std::atomic_thread_fence(std::memory_order_acquire);
    if (!take(r)) {
      *bad = true;
      break;
    }
    ++rd;
    ++n;
  }
  return n;
}

}  // namespace ldpcgb
