"""Plain CPU oracle for the punctured-eMBB receive path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import or run anything here; the
product path (the C-ABI library and its Python binding) never does and fails
loudly without its CUDA extension.

The oracle restates, step by step and in plain NumPy, what the receive path
computes (paper Sec. III-B eq. 1, Sec. V-A eq. 2, Sec. VI-D "UE"): puncture
flushing (LLR := 0), max-log soft demapping by brute force over the whole
constellation, layered offset-min-sum decoding in float64 and in exact
integer (INT8/INT16 saturating) arithmetic, the transport-block CRC-24 check,
goodput and reward.  It shares no code with the CUDA path; it reads the
seeded inputs that ``workload`` produces and recomputes its own geometry
(decoded rows, positions) from the base-graph sizes.

Floating point is float64 unless a function says otherwise (the float32 run
of the decoder exists to check the GPU's float32 decoder bit for bit).

Parity status per function (what pins it, in ``tests/test_oracle_*.py``):

* ``crc``: pinned -- algebra (remainder of msg||crc is 0, linearity, all-zero
  word, detection of every burst <= 24 bits), and agreement of bitwise long
  division with a byte-table implementation.
* ``encoder``: pinned -- H c = 0 over GF(2) for random information words.
* ``demap``: pinned -- QPSK closed form, odd symmetry, noiseless signs,
  per-axis separable minimum == full 2-D minimum.
* ``decoder``: pinned -- noiseless decoding, all-zero input, brute-force
  max-log ML on a tree code (float and exact integer), dropped-rows identity.
* ``goodput``: pinned -- closed-form eq. 1 and eq. 2 values and bounds.
* ``stats``: pinned -- Wilson interval against its textbook closed form.
* ``policy`` (URLLC puncturing allocations: RP, SeF, the KL-projection
  feasibility enforcer, SC masks): pinned -- RP and SeF reproduce the paper's
  Table VI columns (except one printed RP column, documented there);
  Huntington-Hill rounding is the brute-force minimum of its objective; the
  KL projection matches its closed form without caps, its KKT form, and a
  convex solver; feasible integer vectors are fixed points of the enforcer.
"""
from . import crc, demap, decoder, encoder, goodput, stats, path, policy  # noqa: F401
