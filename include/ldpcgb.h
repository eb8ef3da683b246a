/*
 * ldpcgb -- GB300 (sm_103a) receive path for URLLC-punctured eMBB transport
 * blocks: puncture flushing + max-log soft demapping, layered offset-min-sum
 * decoding of NR-style quasi-cyclic LDPC codes, and the transport-block CRC-24
 * check that yields d_e, the goodput (paper Sec. III-B, eq. 1) and the reward
 * r(t) (paper Sec. V-A, eq. 2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every call returns 0 (LDPC_OK) or a negative LDPC_E* code; on failure
 *   ldpc_last_error() returns a thread-local message.  No C++ exception and no
 *   abort crosses this interface.
 * - Compute calls only ENQUEUE work on the session's CUDA stream and return;
 *   results are ready once that stream is synchronised.
 * - "_dev" pointers are device memory OWNED BY THE CALLER (e.g. PyTorch
 *   tensors); the library never frees them.  Host pointers (descriptor
 *   arrays, base-graph tables) are read during the call and may be freed when
 *   it returns.  The library owns the session (shift tables, workspace, error
 *   word) and batch objects; destroy them with the matching *_destroy call.
 * - A session is bound to the device that was current at create time and to
 *   one stream; it is not thread-safe.
 * - Buffer sizes: ldpc_batch_info() reports how many elements each caller
 *   buffer must hold for a batch; the library cannot see allocation sizes and
 *   trusts the caller to provide at least that much.
 * - Device-side waits are bounded.  A kernel that gives up sets a bit in the
 *   session's device error word (read with ldpc_device_errors()) and returns.
 */
#ifndef LDPCGB_H
#define LDPCGB_H

#include <stdint.h>

#if defined(__GNUC__)
#define LDPC_API __attribute__((visibility("default")))
#else
#define LDPC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define LDPC_OK 0
#define LDPC_EINVAL (-1)   /* bad argument or descriptor (Z not allowed, E too large, misaligned offset) */
#define LDPC_ENOMEM (-2)   /* device-memory budget exceeded or cudaMalloc failed */
#define LDPC_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed */
#define LDPC_ETIMEOUT (-4) /* a bounded device wait gave up (serving) */
#define LDPC_EBUSY (-5)    /* serving ring full / not started */

/* Bits of the device error word. */
#define LDPC_DEVERR_TMA_TIMEOUT 0x1u   /* a bulk-copy wait hit its iteration limit */
#define LDPC_DEVERR_BAD_ITEM 0x2u      /* a work item failed its device-side check */
#define LDPC_DEVERR_SERVE_TIMEOUT 0x4u /* the serving loop's doorbell wait gave up */

typedef struct ldpc_session ldpc_session; /* opaque, owned by the library */
typedef struct ldpc_batch ldpc_batch;     /* opaque, owned by the library */

typedef enum { LDPC_F32 = 0, LDPC_I8 = 1, LDPC_I16 = 2 } ldpc_mode;

/* Decoder launch plan of a batch (see ldpc_session_set_strategy). */
#define LDPC_PLAN_MIXED 0 /* one persistent launch over every shape (plus one for global-message shapes) */
#define LDPC_PLAN_PER_Z 1 /* one persistent launch per lifting size */

typedef struct ldpc_graph ldpc_graph; /* opaque: an instantiated CUDA graph of one batch step */

/*
 * One base matrix.  Edges are listed in row-major (row, col) order; at most
 * one edge per (row, col).  Row k of the Z x Z block at (row, col) with raw
 * shift V connects to column (k + V mod Z) mod Z.  Columns [0, kb) carry
 * information, the next mc columns core parity (rows [0, mc) are the core
 * rows), the rest extension parity, one per extension row.  The first
 * n_punct_cols information columns are never transmitted.  The paper gives
 * no code parameters (Sec. III-B, Sec. VI-A "Tx Signal Processing"); callers
 * supply seeded matrices.  Host pointers, copied at ldpc_session_create.
 */
typedef struct {
  int32_t mb, nb, kb, mc;
  int32_t n_punct_cols;
  int32_t n_edges;
  const int16_t *row;
  const int16_t *col;
  const int16_t *V; /* raw shift in [0, 32767]; the lifted shift is V mod Z */
} ldpc_base_graph;

typedef struct {
  int32_t n_bg;
  const ldpc_base_graph *bgs; /* host array of n_bg */
  int32_t n_z;
  const int32_t *z_set;       /* allowed lifting sizes: 16 or a multiple of 32, <= 384 */
  int32_t mode;               /* ldpc_mode */
  int32_t max_iter;           /* 1..64 */
  int32_t early_term;         /* 1: stop a code block at the first zero syndrome */
  float offset_f32;           /* beta for LDPC_F32 (e.g. 0.5) */
  int32_t offset_lsb;         /* beta for the integer modes, in LSB (e.g. 1) */
  float q_scale;              /* integer modes: LSB per LLR unit (e.g. 4) */
  int32_t llr_sat;            /* |channel LLR| clamp after quantising (INT8 63, INT16 1023) */
  int32_t msg_sat;            /* |Q| clamp before the minimum (INT8 63, INT16 1023) */
  int32_t post_sat;           /* |Q|, |L| saturation (INT8 127, INT16 32767) */
  int32_t interleave;         /* 1: Qm-row block interleaver between rate matching and mapping */
  uint64_t device_mem_budget; /* bytes the session and its batches may allocate; 0 = unlimited */
  void *cuda_stream;          /* cudaStream_t; NULL = the legacy default stream */
} ldpc_session_desc;

/*
 * One code block.  Transmitted bit e is codeword position
 * t0 + ((k0 + e) mod Ncb), t0 = n_punct_cols * Z, Ncb = nb * Z - t0 (a
 * circular buffer read from the start k0 of the redundancy version; bits that
 * land on one position -- E > Ncb -- have their LLRs added; E <= 2 Ncb); the
 * decoder works on n_eff = kb + m_eff columns with
 * m_eff = min(mb, max(mc, ceil((t0 + last) / Z) - kb)) rows, last = Ncb if
 * k0 + E > Ncb, else k0 + E.  k0 = 0 for redundancy version 0; versions 1-3
 * (flags) follow NR's table: k0 = (17, 33, 56) * Z when Ncb = 66 Z and
 * (13, 25, 43) * Z when Ncb = 50 Z (other graphs: version 0 only).
 *   re_offset        first complex symbol (float2) of the block, E / Qm of them
 *   mask_word_offset first uint32 of its puncture mask: bit r % 32 of word
 *                    r / 32 set = resource element r was taken by URLLC
 *   llr_offset       first element of its n_eff * Z LLRs; a multiple of 16
 *   bits_word_offset first uint32 of its kb * Z / 32 decoded information
 *                    words: bit i of the block is bit i % 32 of word i / 32
 *   inv_sigma2       1 / noise variance per symbol
 *   flags            LDPC_CB_CRC24B: the block's last 24 information bits
 *                    are a CRC of its first K - 24 (K = kb * Z) under
 *                    g_B(x) = x^24 + x^23 + x^6 + x^5 + x + 1 (register from 0,
 *                    first bit highest degree), NR-style segmentation.  The
 *                    decoder then also stops a block whose hard decision
 *                    passes that CRC, and the TB check leaves those bits out.
 *                    Bits 1-2 (LDPC_CB_RV(rv)): the redundancy version sent.
 */
#define LDPC_CB_CRC24B 1
#define LDPC_CB_RV_SHIFT 1
#define LDPC_CB_RV_MASK (3 << LDPC_CB_RV_SHIFT)
#define LDPC_CB_RV(rv) ((rv) << LDPC_CB_RV_SHIFT)
typedef struct {
  int32_t bg, Z, Qm, E;
  int64_t re_offset;
  int64_t mask_word_offset;
  int64_t llr_offset;
  int64_t bits_word_offset;
  float inv_sigma2;
  int32_t flags; /* LDPC_CB_CRC24B | LDPC_CB_RV(rv) */
} ldpc_cb_desc;

/*
 * One transport block (one eMBB user in one slot): code blocks
 * [first_cb, first_cb + n_cb) carry its payload_bits + 24 CRC bits in order;
 * n_sc is n_e, the user's subcarriers; slot indexes the slot_N array.  Either
 * no block of the TB has LDPC_CB_CRC24B and payload_bits = sum(K) - 24, or
 * every block has it and payload_bits = sum(K - 24) - 24 (the TB's bits are
 * each block's first K - 24 bits, in block order).
 */
typedef struct {
  int32_t first_cb, n_cb, n_sc, slot, payload_bits;
} ldpc_tb_desc;

typedef struct {
  int64_t sym_elems;    /* float2 symbols the sym buffer must hold */
  int64_t mask_words;   /* uint32 mask words */
  int64_t llr_elems;    /* LLR elements (float / int8 / int16 by mode) */
  int64_t bits_words;   /* uint32 decoded-bit words */
  int32_t n_cb, n_tb, n_slots;
  int32_t n_items;      /* decoder work items (codeword groups) */
  int64_t info_bits;    /* sum of K over the code blocks */
} ldpc_batch_info;

/* Create a session: validates the base graphs (row degree 2..27, one entry per
 * (row, col)), builds the shift tables for every (base graph, Z) pair, and
 * allocates its workspace on the current device. */
LDPC_API int ldpc_session_create(const ldpc_session_desc *d, ldpc_session **out);
LDPC_API int ldpc_session_destroy(ldpc_session *s);
/* Rebind the session to another stream of the same device (NULL = legacy default). */
LDPC_API int ldpc_session_set_stream(ldpc_session *s, void *cuda_stream);

/* Work-item tile: code blocks of base graph `bg` at lifting size `Z` are decoded
 * `G` per thread block (G groups of Z threads).  Tiles set here override the
 * built-in default (256 / Z, at most 15 for Z > 32) for batches created
 * afterwards; G * Z <= 512.  The planner lowers G to G * Z <= 384 (two decoder
 * blocks share an SM) and further when shared memory requires it.
 * An autotuner chooses them by timing candidates (paper has no counterpart). */
typedef struct {
  int32_t bg, Z, G;
} ldpc_tile;
LDPC_API int ldpc_session_set_tiles(ldpc_session *s, const ldpc_tile *tiles, int32_t n);
/* LDPC_PLAN_MIXED (default) or LDPC_PLAN_PER_Z, for batches created afterwards. */
LDPC_API int ldpc_session_set_strategy(ldpc_session *s, int32_t strategy);

/* Validate host descriptor arrays and plan a batch: per-block geometry, the
 * decoder's work items (codeword groups of one shape), demap tiles and the
 * slot-to-TB lists.  cbs/tbs/slot_N are host arrays; slot_N[s] is N, the
 * subcarriers of slot s (the reward's normaliser).  n_tb may be 0 (decode
 * only); then tb_crc_goodput rejects the batch. */
LDPC_API int ldpc_batch_create(ldpc_session *s, const ldpc_cb_desc *cbs, int32_t n_cb,
                      const ldpc_tb_desc *tbs, int32_t n_tb, int32_t n_slots,
                      const int32_t *slot_N, ldpc_batch **out);
LDPC_API int ldpc_batch_destroy(ldpc_batch *b);
LDPC_API int ldpc_batch_info_get(const ldpc_batch *b, ldpc_batch_info *out);

/* One decoder launch of a batch's plan. */
typedef struct {
  int32_t block, grid, smem, n_items, global_messages, max_groups;
} ldpc_launch_info;
/* Copy up to `cap` launch records into `out`; *n_launches gets the total. */
LDPC_API int ldpc_batch_plan_get(const ldpc_batch *b, ldpc_launch_info *out, int32_t cap, int32_t *n_launches);

/*
 * Puncture flushing + max-log soft demapping + rate dematching (paper
 * Sec. VI-D "UE": the LLRs of bits on punctured resource elements are set to 0
 * after the soft demodulator; the demapper algorithm is not stated there,
 * this library uses max-log).  For each resource element r of each block:
 * if its mask bit is set all Qm LLRs are 0, otherwise
 *   lambda_i = inv_sigma2 * (min_{s: b_i=1} |y-s|^2 - min_{s: b_i=0} |y-s|^2)
 * over NR-style Gray QAM (Qm = 2, 4, 6, 8), written to codeword position
 * t0 + i * (E/Qm) + r (interleaved) or t0 + r * Qm + i.  Positions never
 * transmitted are written 0.  Integer modes store
 * clamp(round_half_away(q_scale * lambda), -llr_sat, llr_sat).
 *   sym_dev  float2 (re, im) symbols; mask_dev uint32 words;
 *   llr_dev  float (F32) / int8 (I8) / int16 (I16), batch info llr_elems.
 */
LDPC_API int puncture_demap(ldpc_session *s, const ldpc_batch *b, const void *sym_dev,
                   const uint32_t *mask_dev, void *llr_dev);

/*
 * Layered offset-min-sum decoding of every code block of the batch from the
 * LLR buffer.  Rows 0..m_eff-1 in order each iteration; check (l, k) over
 * edges j: Q_j = L[v_j] - R_j; R'_j = sign * max(min_{i != j} |Q_i| - beta, 0)
 * with sign the product of the other edges' signs (Q = 0 counts positive);
 * L[v_j] = Q_j + R'_j.  Integer modes saturate Q and L at post_sat and clamp
 * |Q| at msg_sat before the minimum.  After every iteration the hard decision
 * [L < 0] is checked against the m_eff rows; with early termination a block
 * stops at the first zero syndrome or, for a block with LDPC_CB_CRC24B, at the
 * first hard decision whose information bits pass its CRC.  Writes each
 * block's kb*Z information bits to bits_dev and status_dev[cb] = iterations |
 * (syndrome_zero << 16) | (cb_crc_passed << 17) (bit 17 only for blocks with
 * LDPC_CB_CRC24B, from the final hard decision).
 * The paper's decoder is a toolbox function (Sec. VI-D "UE"); this is the
 * algorithm this library fixes in its place.
 */
LDPC_API int decode_batch(ldpc_session *s, const ldpc_batch *b, const void *llr_dev,
                 uint32_t *bits_dev, int32_t *status_dev);

/*
 * decode_batch's latency form: each code block is decoded by a thread-block
 * cluster of cluster_ctas (2 or 4) CTAs on as many SMs, each CTA owning
 * Z / cluster_ctas of every layer's lifted checks and keeping a replica of the
 * block's posteriors (every new posterior is written into all replicas; a
 * cluster barrier separates the layers).  The same algorithm and arithmetic as
 * decode_batch (the paper's receiver decode, Sec. VI-D "UE"), so bits and
 * status are identical; for callers that decode one or a few large blocks and
 * want them back soonest.  Needs Z % (32 * cluster_ctas) == 0 and blocks
 * without LDPC_CB_CRC24B (LDPC_EINVAL otherwise); the first call per cluster
 * size builds the batch's cluster plan in device memory the batch owns.
 */
LDPC_API int ldpc_decode_cluster(ldpc_session *s, ldpc_batch *b, const void *llr_dev, uint32_t *bits_dev,
                                 int32_t *status_dev, int32_t cluster_ctas);

/*
 * Transport-block CRC-24 check and per-slot goodput and reward.  d_e = 1 iff
 * the TB's (payload_bits + 24) decoded bits are a multiple of
 * g(x) = 0x1864CFB (register from 0, first bit highest degree) -- the same
 * test as comparing received and recomputed CRC bits (Sec. VI-D "UE Feedback")
 * -- and, for a segmented TB with LDPC_CB_CRC24B, every block's K bits are a
 * multiple of g_B(x) = 0x1800063: every attached CRC bit must match.
 * Per slot t:  goodput_bits[t] = sum_e d_e * payload_bits_e;
 *              goodput_sc[t]   = sum_e d_e * n_e               (eq. 1)
 *              reward[t]       = (1/N_t) * sum_e (d_e - 1) n_e  (eq. 2)
 * d_dev: uint8 per TB; the other outputs one element per slot.
 */
LDPC_API int tb_crc_goodput(ldpc_session *s, const ldpc_batch *b, const uint32_t *bits_dev,
                   uint8_t *d_dev, uint64_t *goodput_bits_dev, uint32_t *goodput_sc_dev,
                   float *reward_dev);

/*
 * Capture one whole step of a batch -- puncture_demap, decode_batch and (if
 * the batch has TBs) tb_crc_goodput on the given buffers -- into a CUDA graph
 * and instantiate it, so a step is a single ldpc_graph_launch with no
 * per-kernel launch overhead (the decoder's work-queue reset is a memset node
 * inside the graph).  The buffers are baked into the graph: relaunching reads
 * and writes the same addresses.  Capture runs on a private stream; the
 * session's stream is unchanged afterwards.
 */
LDPC_API int ldpc_graph_create(ldpc_session *s, const ldpc_batch *b, const void *sym_dev,
                               const uint32_t *mask_dev, void *llr_dev, uint32_t *bits_dev,
                               int32_t *status_dev, uint8_t *d_dev, uint64_t *goodput_bits_dev,
                               uint32_t *goodput_sc_dev, float *reward_dev, ldpc_graph **out);
LDPC_API int ldpc_graph_launch(ldpc_graph *g, void *cuda_stream);
LDPC_API int ldpc_graph_destroy(ldpc_graph *g);

/*
 * Decode n_cb code blocks of one shape WITHOUT ALLOCATING any memory (the
 * paper has no counterpart; this is a deployment entry point).  For callers
 * that cannot call cudaMalloc: code under a memory pool or budget that
 * forbids growth once set up, a real-time receive loop where an allocation's
 * latency or failure is unacceptable, or a host application that owns all
 * device memory and hands the library only its buffers.  It needs no
 * session or batch: the base graph `g` (host arrays) and the decoder settings
 * are passed directly, with the same meaning and limits as in
 * ldpc_session_desc and ldpc_cb_desc.  Code block i's n_eff * Z LLRs start at
 * element i * n_eff * Z of llr_dev (float / int8 / int16 by `mode`, 16-byte
 * aligned); its kb*Z/32 information words are written at word
 * i * (kb*Z/32) of bits_dev and its status at status_dev[i], both as in
 * decode_batch.  Results equal decode_batch's for the same blocks.
 * Scratch: one fixed 24 MiB __device__ array inside the library, held by
 * every GPU that loads it until the process exits.  The first call on a
 * device looks up that array's address (make it before any stream capture).
 * n_cb above 32768, or a shape whose per-block message state does not fit
 * the array, is rejected with LDPC_EINVAL before any launch.  All calls share
 * the array and leave their contents in it: calls that overlap on the GPU
 * (other streams, other threads) race -- serialise them.  Enqueued on
 * `cuda_stream` (NULL = legacy default); never calls cudaMalloc/cudaFree.
 */
LDPC_API int decode_uniform_noalloc(const ldpc_base_graph *g, int32_t Z, int32_t E, int32_t n_cb,
                                    int32_t mode, int32_t max_iter, int32_t early_term,
                                    float offset_f32, int32_t offset_lsb, int32_t msg_sat,
                                    int32_t post_sat, const void *llr_dev, uint32_t *bits_dev,
                                    int32_t *status_dev, void *cuda_stream);
/* The no-allocation decoder's device error word on the current device (LDPC_DEVERR_* bits): each
 * decode_uniform_noalloc call clears it before it decodes; a work item whose bounded bulk-copy wait gave
 * up sets LDPC_DEVERR_TMA_TIMEOUT and leaves its blocks' bits and status unwritten.  Waits for
 * `cuda_stream`, stores the word in *flags_out (host) and clears it.  Allocates nothing. */
LDPC_API int decode_uniform_noalloc_errors(uint32_t *flags_out, void *cuda_stream);
/* Runs the decoder's bounded bulk-copy wait on an mbarrier that nothing completes, giving up after
 * `limit` polls (1..65536): it sets LDPC_DEVERR_TMA_TIMEOUT in the word above, exactly as a decode whose
 * copy never landed would.  For tests of the failure report; enqueued on `cuda_stream`. */
LDPC_API int decode_uniform_noalloc_wait_check(int32_t limit, void *cuda_stream);

/* ------------------------------------------------------------------ serving
 * Continuous batching of TB decode requests (the paper's per-TTI receiver
 * feedback loop, Sec. VI-D "UE", run as a service).  One persistent device
 * loop (one thread block per SM) takes work items -- up to G code blocks of
 * one TB -- from a ring in pinned host memory as soon as the host publishes
 * them, so requests that arrive while others are decoding start on the next
 * free SM; no kernel is launched per request.  Each item demaps its blocks'
 * symbols straight from the caller's pinned host pool into shared memory
 * (puncture flushing + max-log + quantisation fused into the decoder's
 * prologue), decodes them, and the last item of a TB runs its CRC-24 check,
 * copies the decoded bits to the caller's result pool and writes a
 * completion record to pinned host memory.  Admission: a request is admitted
 * only if its device-resident state (decoded bits, status words) fits the
 * arena of arena_bytes and the rings have room; otherwise submit stops and
 * reports how many were admitted, and the caller retries after completions
 * free space.  Every device wait is bounded: the loop exits after
 * idle_timeout_us without work (submit relaunches it) or when stopped.
 * Shapes whose decoder state does not fit shared memory are rejected
 * (LDPC_EINVAL); every mode fits every shape up to Z = 384 (an FP32 service
 * keeps its check messages in a device-memory slot per loop group, the
 * integer modes in shared memory; the INT8 single form holds its posteriors
 * as floats carrying the quantised integers).
 */
typedef struct ldpc_server ldpc_server;

typedef struct {
  uint64_t arena_bytes;      /* device-memory budget for admitted requests */
  int32_t max_inflight;      /* requests admitted at once, 1..65536 */
  int32_t idle_timeout_us;   /* device loop idles this long before exiting (e.g. 200000) */
  const void *host_pool;     /* pinned, mapped host memory holding the requests' symbols and masks */
  uint64_t host_pool_bytes;
  void *result_pool;         /* pinned, mapped host memory receiving decoded bits (may be NULL) */
  uint64_t result_pool_bytes;
  int32_t loops_per_sm;      /* 0 or 1: one device loop per SM.  2 (two
                              * loops per SM, messages in device memory) is withdrawn and returns
                              * LDPC_EINVAL: under load it once made an illegal access and once returned
                              * corrupted status words, cause not yet found */
  int32_t flags;             /* LDPC_SERVE_CB_CRC: accept TBs whose code blocks carry their own CRC (the
                              * loop then runs its variant with the code-block CRC exit).
                              * INT8 services decode a request's code blocks in one of two forms, chosen
                              * per request at admission: single (one block per thread group, check
                              * messages in shared memory: the lower latency per block) or paired (two
                              * blocks per thread group in half2 arithmetic, the batch decoder's paired
                              * form: more blocks in flight per SM).  By default a request is paired when
                              * the work items in flight together with its own single-form items would
                              * exceed pair_threshold (and, once pairing, until they fall to
                              * pair_release); LDPC_SERVE_UNPAIRED: never; LDPC_SERVE_PAIRED:
                              * always (where the shape allows it, Z a multiple of 32).  Results are the
                              * same bits either way; the two flags together are LDPC_EINVAL */
  int32_t pair_threshold;    /* work items in flight above which INT8 requests are paired; 0: twice the
                              * number of loop thread blocks (one per SM) */
  int32_t pair_release;      /* once pairing, keep pairing until the items in flight fall to this many
                              * (hysteresis); 0: the number of loop thread blocks; at most pair_threshold */
  /* URLLC puncturing codebook (Sec. III-A: URLLC packets preempt eMBB subcarriers for one mini-slot of
   * two OFDM symbols, seven mini-slots per slot).  A request names one entry and its band's place on
   * its slot's subcarrier grid; the loop expands the entry into the punctured resource elements of
   * the request's code blocks while it demaps them, so one slot's URLLC bursts hit exactly the users
   * whose bands lie under them.  codebook (host, copied at start; NULL when codebook_n = 0):
   * [codebook_n][7][ceil(codebook_prb / 32)] uint32 bitmaps; bit p % 32 of word p / 32 of
   * bitmap [id][m] set = PRB p (12 subcarriers) of the pattern grid is preempted in mini-slot m
   * (symbols 2m, 2m + 1).  The pattern repeats every codebook_prb PRBs along the slot's grid. */
  int32_t codebook_n;        /* entries, 0..65536 */
  int32_t codebook_prb;      /* pattern period in PRBs, 1..65536 (ignored when codebook_n = 0) */
  const uint32_t *codebook;
} ldpc_serve_desc;
#define LDPC_SERVE_CB_CRC 1
#define LDPC_SERVE_UNPAIRED 2
#define LDPC_SERVE_PAIRED 4

typedef struct {
  int32_t bg, Z, Qm, E, n_cb;   /* one shape for all of the TB's code blocks; n_cb in 1..16 */
  int32_t n_sc, payload_bits;   /* n_e; payload_bits = n_cb * kb * Z - 24, or, for n_cb > 1 with a CRC
                                 * per code block (LDPC_CB_CRC24B), n_cb * (kb * Z - 24) - 24 */
  float inv_sigma2;
  int32_t rv;                   /* redundancy version of every code block, 0..3, as LDPC_CB_RV in the
                                 * batch descriptors (1-3 need a buffer of 66 Z or 50 Z positions) */
  int32_t pattern;              /* which resource elements URLLC punctured: -1 = bit r % 32 of mask word
                                 * r / 32 at mask_offset, per code block; 0..codebook_n-1 = that codebook
                                 * entry on the slot's grid (mask_offset unused) */
  int64_t sym_offset;           /* bytes into host_pool (8-aligned): n_cb * E/Qm float2, block after block */
  int64_t mask_offset;          /* pattern -1: bytes into host_pool (4-aligned), n_cb * ceil(E/Qm/32) words */
  int64_t result_offset;        /* bytes into result_pool (4-aligned) for n_cb * kb*Z/32 words, or -1 */
  uint64_t tag;                 /* echoed in the completion */
  int32_t grid_sc;              /* pattern >= 0: the first subcarrier of the TB's band on its slot's grid.
                                 * Resource element i of the TB (code block i / (E/Qm), block after block)
                                 * sits on OFDM symbol i / n_sc and subcarrier grid_sc + i % n_sc; the TB
                                 * must fit its band in one slot: n_cb * E/Qm <= 14 * n_sc */
  int32_t reserved;             /* 0 */
} ldpc_serve_tb;

typedef struct {
  uint64_t tag;
  int32_t d;                    /* 1: the TB's CRC-24 check passed */
  int32_t max_iters;            /* most iterations any of its code blocks ran */
  int32_t all_syndrome_ok;      /* every code block ended with a zero syndrome */
  int32_t status;               /* 0, or LDPC_ETIMEOUT if the service stopped before it completed */
  int64_t t_submit_ns;          /* host steady clock at submission (replay: the scheduled arrival) */
  int64_t t_complete_ns;        /* host steady clock when the completion was collected */
  int64_t t_device_ns;          /* device global timer when the loop wrote the completion (own time base:
                                 * for differences between completions) */
  int64_t t_admit_ns;           /* host steady clock when the request was admitted */
} ldpc_serve_done;

/* Allocate the arena and rings and start the device loop on a private stream. */
LDPC_API int ldpc_serve_start(ldpc_session *s, const ldpc_serve_desc *d, ldpc_server **out);
/* Admit requests in order until one does not fit; *n_admitted says how many were taken. */
LDPC_API int ldpc_serve_submit(ldpc_server *srv, const ldpc_serve_tb *tbs, int32_t n, int32_t *n_admitted);
/* Collect up to cap completions (frees their arena space), in the order the loop wrote them; out[0..*n_out)
 * is valid whatever the return code.  A completion record that names no request in flight (corrupt or
 * repeated) stops the collection: the good records before it are returned with LDPC_OK, and the call that
 * starts on it returns LDPC_ECUDA with *n_out = 0 and leaves it in place -- the ring cannot advance past it,
 * so the caller stops the service (ldpc_serve_stop) and starts a new one. */
LDPC_API int ldpc_serve_poll(ldpc_server *srv, ldpc_serve_done *out, int32_t cap, int32_t *n_out);
/* Replay an arrival schedule: submit tbs[i] at arrival_ns[i] (ns after the call starts, non-decreasing),
 * retrying admission as space frees, and collect every completion into out[0..n) in completion order
 * (on an error return, the completions collected so far are in out, zeros after them).
 * Latency = t_complete_ns - t_submit_ns with t_submit_ns the scheduled arrival.  Gives up with
 * LDPC_ETIMEOUT if nothing completes for timeout_ms. */
LDPC_API int ldpc_serve_replay(ldpc_server *srv, const ldpc_serve_tb *tbs, const int64_t *arrival_ns, int32_t n,
                               ldpc_serve_done *out, int32_t timeout_ms);
/* Counters, out[0..n): since start, requests admitted, work items admitted in the single form, in
 * the paired form, device loop launches; then, for the last ldpc_serve_replay, the longest pass of
 * its host loop in ns, the number of passes longer than 1 ms, when the longest pass began (ns after
 * the replay started), and the replaying thread's involuntary and voluntary context switches and its
 * minor and major page faults during the replay (getrusage of the thread; 0 where unavailable).
 * Entries past these are 0. */
LDPC_API int ldpc_serve_stats(ldpc_server *srv, int64_t *out, int32_t n);
/* Stop the device loop (bounded wait) and free the server. */
LDPC_API int ldpc_serve_stop(ldpc_server *srv);

/* ---------------------------------------------------------------- puncturing allocations
 *
 * Which subcarriers URLLC takes from the eMBB users.  The paper compares its
 * learned policy with two fixed ones (Sec. VII-A) and repairs its policy's
 * output with a feasibility enforcer (Sec. V-B); these calls compute the
 * fixed policies, the enforcer and the per-subcarrier masks they imply,
 * batched, on the device.  They need no session; every pointer is a device
 * pointer owned by the caller, every call enqueues on `cuda_stream` (NULL =
 * legacy default stream) and returns LDPC_OK or LDPC_EINVAL (bad sizes, null
 * buffer) / LDPC_ECUDA (launch failure) without waiting for the kernel.
 * Per-problem failures are reported in status_dev (0 = ok) and leave that
 * problem's output zero.
 *
 * Integer rounding everywhere is Huntington-Hill: every value goes to its
 * floor or its ceiling (never above its cap), the units left after the
 * floors go one at a time to the largest q_e / sqrt(a_e (a_e + 1)) (infinite
 * for a_e = 0), equal priorities to the lower index.  Quotas, priorities and
 * the KL projection are float32, each operation rounded once in a fixed
 * order, so results are reproducible bit for bit. */
#define LDPC_POLICY_RP 0  /* "Resource Proportion": in proportion to the allocations */
#define LDPC_POLICY_SEF 1 /* "Smallest eMBB First": smallest allocations taken whole first (lower index on ties) */

/* SCs taken from each user, per (TTI, mini-slot).  alloc_dev: int32 [n_tti][n_users] SCs scheduled per
 * user (the eMBB schedule s(t)); demand_dev: int32 [n_tti][7] URLLC SCs per mini-slot; punct_dev (out):
 * int32 [n_tti][7][n_users]; status_dev (out): int32 [n_tti][7], 1 = demand above the TTI's total
 * allocation.  1 <= n_users <= 32. */
LDPC_API int ldpc_puncture_alloc(int32_t policy, int32_t n_tti, int32_t n_users, const int32_t *alloc_dev,
                                 const int32_t *demand_dev, int32_t *punct_dev, int32_t *status_dev,
                                 void *cuda_stream);

/* Feasibility enforcer (Sec. V-B): for each problem, the integer vector nearest a real puncturing vector
 * that may exceed the allocations.  First the projection x of m onto {0 <= x_e <= n_e, sum x = total}
 * minimising sum_e m_e log(m_e / x_e) (eq. 6, eq. 7; users with m_e > 0 get min(n_e, c m_e) with one scale
 * c, users with m_e <= 0 get 0 unless the others cannot hold the total, then the rest in proportion to
 * n_e), then Huntington-Hill rounding to integers summing to total.  punct_real_dev: float32
 * [n_prob][n_users]; alloc_dev: int32 [n_prob][n_users]; total_dev: int32 [n_prob] (j * L for branch j);
 * punct_dev (out): int32 [n_prob][n_users]; status_dev (out): int32 [n_prob], 1 = total above the
 * allocations, 2 = no rounding sums to the total. */
LDPC_API int ldpc_feasibility_enforce(int32_t n_prob, int32_t n_users, const float *punct_real_dev,
                                      const int32_t *alloc_dev, const int32_t *total_dev, int32_t *punct_dev,
                                      int32_t *status_dev, void *cuda_stream);

/* RT O-DU codebook B*(t) (Alg. 2), one TTI per thread block: for each branch j = 1 .. n_branch the
 * policy network's forward pass on input [s(t) / N, j / n_branch] (N = the TTI's total allocation): one
 * dense hidden layer of `hidden` ReLU units, outputs [mu_1..mu_E, s_1..s_E], sigma = softplus(s), the
 * reparameterised sample z = mu + sigma * noise, action (tanh(z) + 1) / 2 in [0, 1] read as the fraction
 * of each user's allocation to puncture; then the feasibility enforcer on each branch with total j * L.
 * The paper's network has trained weights (Sec. VII-B: one hidden layer of 128); none exist here, so the
 * caller supplies any weights (this is the timing form).  Layouts (row-major, float32): w1_dev
 * [hidden][n_users + 1], b1_dev [hidden], w2_dev [2 n_users][hidden], b2_dev [2 n_users]; noise_dev
 * [n_tti][n_branch][n_users] standard-normal draws (random numbers come from the caller).  alloc_dev:
 * int32 [n_tti][n_users]; outputs: codebook_dev int32 and action_dev float32 [n_tti][n_branch][n_users],
 * status_dev int32 [n_tti][n_branch] (enforcer status).  1 <= n_users <= 32, hidden <= 1024,
 * n_branch <= 32.  Sums start at the bias and add products in index order, each rounded once. */
LDPC_API int ldpc_rt_odu_codebook(int32_t n_tti, int32_t n_users, int32_t hidden, int32_t n_branch, int32_t L,
                                  const int32_t *alloc_dev, const float *w1_dev, const float *b1_dev,
                                  const float *w2_dev, const float *b2_dev, const float *noise_dev,
                                  int32_t *codebook_dev, float *action_dev, int32_t *status_dev, void *cuda_stream);

/* Puncture bitmap per (TTI, OFDM symbol): user e's band is the alloc SCs after users 0..e-1 (SC 0
 * first) and the lowest punct SCs of the band are punctured in both symbols of the mini-slot (a reading:
 * the paper does not say which SCs).  punct_dev as written by ldpc_puncture_alloc (each value at most its
 * allocation); mask_dev (out): uint32 [n_tti][14][words_per_symbol], bit b of word w = SC 32w + b; SCs
 * beyond 32 * words_per_symbol are dropped. */
LDPC_API int ldpc_sc_mask(int32_t n_tti, int32_t n_users, const int32_t *alloc_dev, const int32_t *punct_dev,
                          int32_t words_per_symbol, uint32_t *mask_dev, void *cuda_stream);

/* Synchronise the session stream and return (then clear) the device error word. */
LDPC_API int ldpc_device_errors(ldpc_session *s, uint32_t *flags_out);

/* Libraries built with -DLDPC_CHECKED test the indices their kernels trust
 * (posterior addresses, serving items and code-block records against the
 * shape, arena and host pool) and redirect a failing access to a safe slot.
 * out8 (host): the first failed check of the decoder kernels (words 0-3) and
 * of the serving loop (words 4-7), each {check id, value, limit,
 * block * 1024 + thread}; zeros when none failed or the library is not a
 * checked build.  Does not synchronise. */
LDPC_API int ldpc_check_log(uint32_t *out8);

/* Thread-local message for the last non-zero return on this thread. */
LDPC_API const char *ldpc_last_error(void);

/* Library version string. */
LDPC_API const char *ldpc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LDPCGB_H */
