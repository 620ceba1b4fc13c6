/*
 * rcg.h -- C ABI of librcg, a GB300 (sm_103a) implementation of the
 * cyclic-group RAID-6 code of Jackson, Rumynin and Zaboronski, "An approach to
 * RAID-6 based on cyclic groups" (arXiv cs/0611109).
 *
 * The code.  A strip is an element of R = F2[x]/(1 + x + ... + x^(p-1)) for an
 * odd prime p: multiplication by x is multiplication by the Sylvester matrix
 * S_p of Lemma 3.4.1, which has order p (Section 3.4).  For N data strips
 * d_0..d_{N-1} the two parity strips are (Corollary 3.2.4, equation
 * (znparity), 0-based data indices as in Section 4.1)
 *     P = d_0 + d_1 + ... + d_{N-1},      Q = d_0 + x d_1 + ... + x^(N-1) d_{N-1},
 * and any two lost strips are rebuilt by the case analysis of Lemma 3.1.2,
 * the two-data case by the elimination of Sections 4.3 and 4.6 with the
 * precomputed inverses (1 + x^z)^(-1).  Everything is XOR over GF(2): results
 * are exact and the solution of every erasure pair is unique (Lemma 3.1.2).
 *
 * Extended Q-parity (Section 3.3, equation (qext)).  For a prime p that
 * satisfies Theorem 3.3.3 (every 1 + x^u + x^v, 0 < u < v < p, is a unit of
 * R -- true for 5, 11, 13, 17, 19, 23, 29, ..., 59, 61 and false for 3, 7, 31)
 * a stripe may hold up to 2p - 1 data strips: data strip k >= p is weighted
 * in Q by 1 + x^(k-p+1), so
 *     Q = sum_{k<p} x^k d_k + sum_{k=p}^{N-1} (1 + x^(k-p+1)) d_k,
 * and P stays the plain XOR.  For N <= p this is the code above; every call
 * below accepts the extended range (rcg_prime_info gives the limit).
 *
 * Storage (bit-sliced).  A strip is p-1 rows of C bytes; row r holds the
 * coefficient of x^r of 8*C independent codewords, one per bit position.
 * Byte order, word width and bit order inside a row are irrelevant: every
 * operation is a row-level XOR plus a row-index remap.
 *
 * Stripe layout.  rcg_layout describes stripes in device memory: stripe s at
 * base + s*stripe_stride, its strip k (data k < N, P = strip N, Q = strip
 * N+1) at + k*strip_stride, row r at + r*row_stride; each row is row_bytes
 * bytes.  A zero stride means "packed".  base, strides and row_bytes must be
 * multiples of 16 bytes.  Any such layout is exact; the engine is fastest when
 * base and row_stride are multiples of 128 bytes (one L2 line), so that the
 * column tiles it copies start on line boundaries: with a packed layout whose
 * row_bytes is an odd multiple of 16, p = 59 launches measured about 10 % slower
 * on GB300 (pad the row stride to a multiple of 128 to avoid it).
 *
 * Ownership and asynchrony.  The caller owns every stripe buffer (device
 * memory, e.g. from PyTorch) and every output buffer.  Calls enqueue work on
 * the caller's CUDA stream (a cudaStream_t passed as void*; NULL = legacy
 * default stream) and return before it runs; the library keeps no pointer
 * past the call except as stated for rcg_batch_submit.  Argument errors are
 * returned synchronously and enqueue nothing.  Errors a kernel finds (an
 * invalid per-stripe erasure pair read from device memory, a bounded wait
 * that expired) are recorded in the context's device status word, read with
 * rcg_last_device_status.  No call aborts the process, traps on the device or
 * waits without a time limit.
 *
 * Overlap.  Work inside one call must not write memory another part of the
 * same call reads, except in place as documented (a recovery writes only the
 * erased strips, which it never reads).
 */
#ifndef RCG_H
#define RCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RCG_ABI_VERSION 1u

typedef enum rcg_status {
    RCG_OK = 0,
    RCG_EINVAL = 1,       /* invalid argument; nothing was enqueued */
    RCG_ENOMEM = 2,       /* a library allocation failed */
    RCG_ECUDA = 3,        /* a CUDA runtime call failed */
    RCG_ETIMEOUT = 4,     /* a bounded wait expired */
    RCG_EBUSY = 5,        /* a queue or slot table is full; retry later */
    RCG_EUNSUPPORTED = 6, /* the device is not sm_103 or a parameter is out of range */
    RCG_EDEVICE = 7       /* a kernel reported an error in the device status word */
} rcg_status;

/* Bits of the device status word (rcg_last_device_status). */
#define RCG_DEV_TIMEOUT 0x1u  /* a kernel's bounded wait on an mbarrier expired */
#define RCG_DEV_BADPAIR 0x2u  /* a per-stripe erasure pair read from device memory was invalid;
                                 that stripe was skipped */
#define RCG_DEV_BADJOB 0x4u   /* a batch descriptor failed the device-side check; skipped */

typedef struct rcg_ctx rcg_ctx;

typedef struct rcg_layout {
    void *base;             /* device address of stripe 0 */
    uint32_t p;             /* odd prime, 3 <= p <= 61; strips have p-1 rows */
    uint32_t n_data;        /* N, 1 <= N <= p (Corollary 3.2.4), or N <= 2p - 1 where
                               Theorem 3.3.3 holds (equation qext); strip N = P, N+1 = Q */
    uint64_t row_bytes;     /* C, bytes per row, a positive multiple of 16 */
    uint64_t row_stride;    /* bytes between rows of a strip; 0 = row_bytes */
    uint64_t strip_stride;  /* bytes between strips; 0 = (p-1)*row_stride */
    uint64_t stripe_stride; /* bytes between stripes; 0 = (N+2)*strip_stride */
} rcg_layout;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` (must be compute capability 10.3).
 * The context owns the per-p inverse tables (uploaded to the device), a
 * device status word and the batch descriptor buffers.  One context may be
 * used from one host thread at a time. */
rcg_status rcg_create(int device, rcg_ctx **out);
rcg_status rcg_destroy(rcg_ctx *ctx);

/* Upper limit, in nanoseconds, of every wait a kernel of this context makes
 * (default 2e9).  A wait that runs out sets RCG_DEV_TIMEOUT and the kernel
 * returns. */
rcg_status rcg_set_timeout(rcg_ctx *ctx, uint64_t timeout_ns);

/* How the engine moves strip tiles into shared memory.  RCG_COPY_AUTO (the
 * default): one 4-D tensor copy per strip tile wherever the driver accepts a
 * tensor map for the layout, per-row 1-D bulk copies otherwise.
 * RCG_COPY_ROWS: always per-row bulk copies.  Results are identical. */
#define RCG_COPY_AUTO 0
#define RCG_COPY_ROWS 1
rcg_status rcg_set_copy_mode(rcg_ctx *ctx, int mode);

/* How a two-data-strip erasure solves (1 + x^z) D_j = T, z = j - i, where
 * T = dP + x^(-i) dQ (Section 4.6).  The solution is unique (Lemma 3.1.2), so
 * both give identical bytes.
 * RCG_SOLVE_CHAIN (default): lift to F2[x]/(x^p - 1) and walk the rows
 * p-1, p-1+z, p-1+2z, ... (mod p) once, O(p) row XORs per column.
 * RCG_SOLVE_TABLE: the paper's closed form D_j = (1 + x^z)^(-1) T with the
 * per-p table (1 + x^z)^(-1) = sum_{t=0}^{(p-1)/2} x^(2tz), O(p^2/2). */
#define RCG_SOLVE_CHAIN 0
#define RCG_SOLVE_TABLE 1
rcg_status rcg_set_dd_solve(rcg_ctx *ctx, int solve);

/* Engine shape.  RCG_SHAPE_WIDE: one CTA per SM, 15 consumer warps, the
 * deepest shared-memory ring (best for large p such as 59).  RCG_SHAPE_PAIR:
 * two CTAs per SM, 6 consumer warps each, so one CTA's epilogue overlaps the
 * other's streaming (best for small and medium p).  RCG_SHAPE_AUTO (default)
 * picks pair for launches under 256 MB of traffic and wide above.
 * Results are identical. */
#define RCG_SHAPE_AUTO 0
#define RCG_SHAPE_WIDE 1
#define RCG_SHAPE_PAIR 2
rcg_status rcg_set_engine_shape(rcg_ctx *ctx, int shape);

/* Kernel for stripes of small primes.  RCG_COLUMN_AUTO (default): every
 * operation on p <= 7 -- single calls (encode, recover, recover_many, update,
 * degraded read, the host-memory calls) and the p <= 7 jobs of batches and of
 * the server -- runs in a column kernel: a thread owns a 16-byte column of
 * all p-1 rows of a stripe in registers, Q by Horner's rule, no shared memory,
 * one DRAM round trip per column, where the tile engine's stages would be
 * tiny (p = 5, 1 KiB rows: 4 KB).  RCG_COLUMN_OFF: always the tile engine.
 * Results are identical. */
#define RCG_COLUMN_AUTO 0
#define RCG_COLUMN_OFF 1
rcg_status rcg_set_column_kernel(rcg_ctx *ctx, int mode);

/* Where a batch's descriptor table travels (rcg_batch_launch, rcg_batch_submit
 * and the server's batches).  RCG_TABLES_AUTO (default): a table of at most
 * 31 744 bytes (about 240 column jobs, or a few dozen engine jobs with their
 * work items) is passed in the kernels' own parameter blocks -- no
 * host-to-device copy and no graph before the kernels start, the engine's
 * work items dealt round-robin -- and a larger one is copied to a device
 * buffer by a replayed CUDA graph.  RCG_TABLES_DEVICE: always the device
 * buffer and the graph.  Results are identical. */
#define RCG_TABLES_AUTO 0
#define RCG_TABLES_DEVICE 1
rcg_status rcg_set_batch_tables(rcg_ctx *ctx, int mode);

/* Synchronise the device and read, then clear, the device status word.
 * Returns RCG_EDEVICE when any bit was set (then *code holds the bits). */
rcg_status rcg_last_device_status(rcg_ctx *ctx, uint32_t *code);

const char *rcg_status_str(rcg_status s);
uint32_t rcg_abi_version(void);

/* Text of the last CUDA runtime error the library saw on the calling thread
 * (which call, the error name and message); "" if none.  The pointer stays
 * valid until the thread's next library call. */
const char *rcg_last_error(void);

/* ------------------------------------------------------------ stripe ops */

/* Encode: write P and Q of stripes [first_stripe, first_stripe + n_stripes)
 * from their data strips (Corollary 3.2.4, equation (znparity)).  One launch
 * for all stripes.  n_stripes == 0 is a no-op. */
rcg_status rcg_encode(rcg_ctx *ctx, const rcg_layout *L, uint64_t first_stripe,
                      uint64_t n_stripes, void *stream);

/* Recover strips i < j (0 <= i < j <= N+1) of one stripe in place from the
 * other N strips (Lemma 3.1.2): two data strips by Section 4.6's solve,
 * data + P through x^(-i) = x^(p-i), data + Q as in RAID-5, P + Q by
 * re-encoding.  The contents of strips i and j are not read.
 * With extended strips (i or j >= p, equation qext) the same four cases
 * hold with the weights w_k of Q: data i + P solves (1 + x^(i-p+1)) D_i = dQ;
 * two data strips solve (w_i + w_j) D_j = w_i dP + dQ, which the engine
 * brings to (1 + x^z) D_j = T when both are extended, and multiplies by the
 * inverse of a trinomial 1 + x^u + x^v (a unit by Theorem 3.3.3) when only
 * j is. */
rcg_status rcg_recover(rcg_ctx *ctx, const rcg_layout *L, uint64_t stripe, uint32_t i,
                       uint32_t j, void *stream);

/* Recover a per-stripe erasure pair for stripes [first_stripe, first_stripe +
 * n_stripes) in one launch.  pairs is a DEVICE array of 2*n_stripes bytes:
 * (i, j) of stripe first_stripe + s at pairs[2s], pairs[2s+1].  A stripe whose
 * pair is not 0 <= i < j <= N+1 is left untouched and sets RCG_DEV_BADPAIR. */
rcg_status rcg_recover_many(rcg_ctx *ctx, const rcg_layout *L, uint64_t first_stripe,
                            uint64_t n_stripes, const uint8_t *pairs, void *stream);

/* Small write (Section 3.4: updating Q needs no special instructions):
 * replace data strip i (< N) of one stripe by new_strip (device, p-1 rows of
 * C bytes, new_row_stride bytes apart; 0 = C) and update the parities by
 * P += d_i + new, Q += x^i (d_i + new).  Reads 4 strips, writes 3.  new_strip
 * must not overlap the stripe. */
rcg_status rcg_update(rcg_ctx *ctx, const rcg_layout *L, uint64_t stripe, uint32_t i,
                      const void *new_strip, uint64_t new_row_stride, void *stream);

/* Degraded read: rebuild strip j (0 <= j <= N+1) of one stripe without
 * reading it -- a data strip or P from the first parity equation (RAID-5),
 * Q from the second -- into out (device, p-1 rows of C bytes, out_row_stride
 * apart; 0 = C).  The stripe is not modified. */
rcg_status rcg_degraded_read(rcg_ctx *ctx, const rcg_layout *L, uint64_t stripe, uint32_t j,
                             void *out, uint64_t out_row_stride, void *stream);

/* ------------------------------------------- horizontal representation */

/* Section 4.5 keeps one ring element per machine word instead of bit-slicing
 * it over rows: for p = 17 a 16-bit word holds y_0..y_15, the coefficients of
 * x^0..x^15.  In this representation a strip is an array of elements, element
 * e being the little-endian bit field [e(p-1), (e+1)(p-1)) of the strip: for
 * p = 17 the 16-bit little-endian word e, for p = 5 a nibble, for p = 3 two
 * bits (bit r of the field = coefficient of x^r).  Multiplication by x^k is
 * the word formula of Section 4.6 applied lane by lane.  The code, the
 * erasure pairs (data 0..N-1, P = strip N, Q = strip N+1) and the extension
 * to 2p - 1 data strips (p = 5 and 17, equation qext) are those of the
 * bit-sliced calls; results are identical to encoding the transposed stripe.
 * Layout: stripe s at base + s*stripe_stride, strip k at + k*strip_stride,
 * strip_bytes bytes per strip.  base, strides and strip_bytes are multiples of
 * 16; zero strides mean packed.
 *
 * p = 257 (Z_257, named in Section 3.4 beside Z_17): an element is 256 bits,
 * the 32 little-endian bytes [32e, 32e + 32) of the strip.  base, strides and
 * strip_bytes are multiples of 32, N <= 257 (the base code: no extended
 * strips), and the per-stripe pairs of rcg_h_recover_many are two 16-bit
 * numbers per stripe (strip indices reach 258).  A recovery's inverse is not
 * tabulated: (1 + x^z)^(-1) = x^z (1 + x^(2z)) (1 + x^(4z)) ... (1 + x^(128z)),
 * because squaring has order 16 in R (Lemma 3.3.1: 2^16 = 1 and 2^8 = -1
 * modulo 257). */
typedef struct rcg_hlayout {
    void *base;             /* device address of stripe 0 */
    uint32_t p;             /* 3, 5, 17 or 257 */
    uint32_t n_data;        /* N, 1 <= N <= p (or 2p - 1 for p = 5, 17) */
    uint64_t strip_bytes;   /* bytes per strip, a positive multiple of 16 (32 for p = 257) */
    uint64_t strip_stride;  /* bytes between strips; 0 = strip_bytes */
    uint64_t stripe_stride; /* bytes between stripes; 0 = (N+2)*strip_stride */
} rcg_hlayout;

/* Encode P and Q of stripes [first_stripe, first_stripe + n_stripes)
 * (Corollary 3.2.4; Q by Horner's rule Q = d + xQ over the data strips from
 * the last to the first, Section 4.2).  One launch. */
rcg_status rcg_h_encode(rcg_ctx *ctx, const rcg_hlayout *L, uint64_t first_stripe, uint64_t n_stripes,
                        void *stream);

/* Recover strips i < j of one stripe in place (Lemma 3.1.2): two data strips
 * by (w_i + w_j) D_j = w_i dP + dQ with the inverse precomputed per pair (for
 * regular strips it is x^(-i) (1 + x^(j-i))^(-1), Section 4.6), data + P by
 * w_i^(-1) dQ, data + Q as RAID-5, P + Q by re-encoding.  Strips i and j are
 * not read. */
rcg_status rcg_h_recover(rcg_ctx *ctx, const rcg_hlayout *L, uint64_t stripe, uint32_t i, uint32_t j,
                         void *stream);

/* rcg_h_recover for a per-stripe pair: pairs is a DEVICE array of
 * 2*n_stripes bytes, as in rcg_recover_many (for p = 257: 2*n_stripes
 * little-endian 16-bit numbers, 4-byte aligned); an invalid pair leaves its
 * stripe untouched and sets RCG_DEV_BADPAIR. */
rcg_status rcg_h_recover_many(rcg_ctx *ctx, const rcg_hlayout *L, uint64_t first_stripe, uint64_t n_stripes,
                              const uint8_t *pairs, void *stream);

/* ------------------------------------------------- stripes in host memory */

/* rcg_encode and rcg_recover_many for stripes in HOST memory: L->base is a
 * host address of page-locked memory (cudaHostAlloc, cudaHostRegister, or a
 * pinned PyTorch tensor); pageable memory is RCG_EINVAL.  The stripes are
 * streamed through context-owned device staging (three 256 MB chunks,
 * allocated on first use) on three internal streams, so the upload of one
 * chunk, the engine on another and the download of a third overlap.
 *   encode:   uploads the data strips, downloads P and Q;
 *   recovery: uploads only the N surviving strips of each stripe (a gather
 *             kernel reads them through the stripes' mapped device
 *             addresses; the erased strips never cross the link), and writes
 *             only the two rebuilt strips of each stripe back into the host
 *             stripes, in place.  pairs is a HOST array of 2*n_stripes bytes.
 * Results are identical to the device calls.  The calls are ordered on
 * `stream`: the work starts after what is already queued there, and work
 * queued there afterwards sees the results. */
rcg_status rcg_encode_host(rcg_ctx *ctx, const rcg_layout *L, uint64_t first_stripe,
                           uint64_t n_stripes, void *stream);

/* Size of one staging chunk of the host-memory calls (default 256 MB, at
 * least 4096 bytes; a chunk always holds at least one stripe). */
rcg_status rcg_set_host_chunk(rcg_ctx *ctx, uint64_t bytes);
rcg_status rcg_recover_many_host(rcg_ctx *ctx, const rcg_layout *L, uint64_t first_stripe,
                                 uint64_t n_stripes, const uint8_t *pairs, void *stream);

/* ------------------------------------------------------------ batches */

typedef enum rcg_op {
    RCG_OP_ENCODE = 0,        /* encode n_stripes stripes */
    RCG_OP_RECOVER = 1,       /* recover pair (i, j) of n_stripes stripes */
    RCG_OP_DEGRADED_READ = 2, /* rebuild strip j of n_stripes stripes into aux */
    RCG_OP_UPDATE = 3         /* replace data strip i of n_stripes stripes by aux */
} rcg_op;

typedef struct rcg_job {
    rcg_layout layout;          /* stripes of this job (device memory) */
    uint64_t first_stripe;      /* first stripe of the layout this job touches */
    uint64_t n_stripes;         /* stripes in this job */
    uint32_t op;                /* rcg_op */
    uint32_t i, j;              /* recover: pair i < j; update: i; degraded read: j */
    const void *aux;            /* update: new strips; degraded read: output (device) */
    uint64_t aux_row_stride;    /* bytes between rows of aux; 0 = row_bytes */
    uint64_t aux_stripe_stride; /* bytes between stripes of aux; 0 = (p-1)*aux_row_stride */
} rcg_job;

/* Run a list of jobs of mixed p, N, C and op in ONE persistent-kernel launch:
 * jobs are cut into work items of roughly equal bytes, largest jobs first, and
 * the stages of all of them share each CTA's shared-memory ring (by default
 * equal slots sized for the batch's largest stage; a byte ring, where small
 * stages take less room, is a tuning choice -- rcg_set_batch_tuning).  The job list is validated on the
 * host, copied into a context-owned device descriptor table and replayed
 * through a CUDA graph captured once per context -- or, for a table of at
 * most 31 744 bytes, passed in the kernels' parameter blocks (see
 * rcg_set_batch_tables).  Jobs must not overlap in memory.  On return *ticket
 * identifies the batch for rcg_batch_wait.  The context keeps no pointer into
 * `jobs`.  Up to 16 batches may be in flight; a seventeenth waits (bounded)
 * for the oldest, or returns RCG_EBUSY. */
rcg_status rcg_batch_submit(rcg_ctx *ctx, const rcg_job *jobs, uint32_t n_jobs, void *stream,
                            uint64_t *ticket);

/* The two halves of rcg_batch_submit, for callers that overlap host work
 * with the GPU.  rcg_batch_prepare does all host work -- validation, tiling,
 * one TMA tensor map per job, the work-item list -- into an opaque batch that
 * holds no pointer into `jobs`; rcg_batch_launch copies it into a batch slot
 * and replays the slot's CUDA graph (same ticket semantics as
 * rcg_batch_submit).  A prepared batch may be launched any number of times
 * (it names the same device buffers each time) and is released with
 * rcg_batch_free.  The context that prepared a batch must launch it. */
typedef struct rcg_batch rcg_batch;
rcg_status rcg_batch_prepare(rcg_ctx *ctx, const rcg_job *jobs, uint32_t n_jobs, rcg_batch **out);
rcg_status rcg_batch_launch(rcg_ctx *ctx, const rcg_batch *batch, void *stream, uint64_t *ticket);
rcg_status rcg_batch_free(rcg_batch *batch);

/* How a batch's work items (runs of tiles of one job of roughly equal bytes,
 * largest jobs first) reach the CTAs.  RCG_SCHED_DYNAMIC (default): taken from a
 * global counter as CTAs free up.  RCG_SCHED_STATIC: dealt round-robin.
 * Either way a CTA requests its next item while the current one streams.
 * Results are identical. */
#define RCG_SCHED_STATIC 0
#define RCG_SCHED_DYNAMIC 1
rcg_status rcg_set_batch_schedule(rcg_ctx *ctx, int schedule);

/* Batch tuning (not in the paper).  How rcg_batch_prepare lays a batch out:
 * the engine shape of the launch, how work items reach the CTAs, the bytes per
 * work item, a narrowing of every job's tile (tile_div = 2 or 4 gives tiles
 * of 1/2 or 1/4 of the widest width the engine allows, so more stages fit the
 * ring), and how stages share each CTA's shared memory.  Results never depend
 * on the tuning. */
#define RCG_RING_FIXED 0  /* equal shared-memory slots sized for the batch's largest stage (default) */
#define RCG_RING_BYTES 1  /* a byte ring: stages of any size, up to 32 in flight */
typedef struct rcg_batch_tuning {
    uint32_t shape;       /* RCG_SHAPE_AUTO (by the batch's bytes), _WIDE or _PAIR */
    uint32_t schedule;    /* RCG_SCHED_DYNAMIC or RCG_SCHED_STATIC */
    uint64_t item_bytes;  /* bytes per work item, >= 64 KB; 0 = 1/16 of a CTA's share, 256 KB..2 MB */
    uint32_t tile_div;    /* 1 (widest tiles), 2 or 4 */
    uint32_t ring;        /* RCG_RING_FIXED or RCG_RING_BYTES */
    float ms;             /* rcg_batch_autotune: the chosen layout's time for the batch */
    uint32_t reserved;
} rcg_batch_tuning;

/* Autotune the batch layout on a real job list: runs the batch under the
 * current tuning and under candidate values of each knob in turn (engine
 * shape; schedule; item bytes 256 KB / 1 MB / 4 MB / default; tile_div
 * 1 / 2 / 4; ring discipline), each once untimed and twice timed with CUDA
 * events on `stream`,
 * keeps the fastest value of each knob, applies the result to the context
 * (later batches use it) and returns it.  The jobs run for real, about 30
 * times: every batch operation is idempotent on jobs that do not overlap in
 * memory (encode rewrites P and Q from the data, a recovery rewrites the same
 * bytes into the strips it never reads, a small write's second run changes
 * nothing, a degraded read rewrites its output), so the results are those of
 * one run.  Synchronous: returns when the timing is done. */
rcg_status rcg_batch_autotune(rcg_ctx *ctx, const rcg_job *jobs, uint32_t n_jobs, void *stream,
                              rcg_batch_tuning *out);

/* Apply a tuning (e.g. one saved from an earlier rcg_batch_autotune on the
 * same GPU model); NULL restores the defaults. */
rcg_status rcg_set_batch_tuning(rcg_ctx *ctx, const rcg_batch_tuning *tuning);

/* Wait at most timeout_ns for batch `ticket`; RCG_ETIMEOUT if it has not
 * finished (the batch keeps running). */
rcg_status rcg_batch_wait(rcg_ctx *ctx, uint64_t ticket, uint64_t timeout_ns);

/* ---------------------------------------------------------------- serving */

/* A request loop with continuous batching (not in the paper).  Requests are
 * rcg_jobs on caller-owned device stripes (the stripe and parity state stay
 * in device memory), each with an arrival time and an HBM footprint.  A
 * scheduler thread, started by rcg_serve_start, owns the context until
 * rcg_serve_destroy (do not use the context from other threads meanwhile) and
 * repeats:
 *  - retire launches whose completion event fired;
 *  - admit requests whose arrival time has passed, in arrival order, while
 *    the in-flight request count and the HBM budget allow.  Two requests
 *    conflict when the device bytes they touch overlap: the extent of the
 *    job's stripes ([first stripe, last byte of its last stripe]) and, for a
 *    degraded read or a small write, the extent of its aux buffer.  A request
 *    that conflicts with an admitted request, or with an earlier request
 *    still waiting, waits too (requests on the same bytes run in arrival
 *    order and never share a launch); requests behind it that do not
 *    conflict go ahead;
 *  - batched mode (default): launch everything admitted as ONE batch of the
 *    persistent engine while fewer than max_inflight_batches batches are in
 *    flight -- requests arriving meanwhile join the next batch, which is
 *    prepared on the host while the GPU runs;
 *  - per-job mode (per_job_launches = 1, the comparison): launch every
 *    admitted request at once with its own single-operation call (one kernel
 *    launch each); the number in flight is bounded only by max_inflight_jobs.
 *  Launches of both modes go round-robin over eight streams of the server's
 *  own, so small launches run at once and one batch's tail overlaps the next
 *  one's start; requests on the same bytes are never in flight together, so
 *  launches on different streams never touch the same bytes.
 *
 * The HBM budget is a counter, not a live reading: the budget is fixed when
 * the server is created (default min(120 GB, the device's free memory at that
 * moment)) and every admitted request's footprint counts against it until the
 * request completes.  The server itself allocates nothing per request. */
typedef struct rcg_server rcg_server;

typedef struct rcg_serve_config {
    uint64_t hbm_budget_bytes;   /* sum of footprints admitted at once; 0 = min(120 GB, free HBM) */
    uint32_t max_inflight_jobs;  /* admitted but not completed; 0 = 4 x max_batch_jobs */
    uint32_t max_batch_jobs;     /* requests per launch; 0 = 2048 */
    uint32_t per_job_launches;   /* 1: one single-operation launch per request */
    uint32_t max_inflight_batches; /* batched mode: batches in flight at once, 1..8; 0 = 8 */
} rcg_serve_config;

typedef struct rcg_serve_request {
    rcg_job job;                /* one stripe (n_stripes = 1) unless op = encode */
    uint64_t arrival_ns;        /* visible to the scheduler this long after rcg_serve_start */
    uint64_t footprint_bytes;   /* HBM working set while in flight; 0 = the default footprint:
                                   (n_data + 2) x strip stride x n_stripes, plus (p - 1) x row_bytes
                                   x n_stripes for a degraded read's output or a small write's
                                   new strips */
} rcg_serve_request;

typedef struct rcg_serve_result {
    uint64_t id;                /* submission index */
    uint64_t arrival_ns, admit_ns, launch_ns, complete_ns;  /* since rcg_serve_start */
    uint32_t status;            /* RCG_OK, or RCG_EBUSY while not completed */
    uint32_t batch;             /* number of the launch that carried the request (1, 2, ...) */
} rcg_serve_result;

typedef struct rcg_serve_stats {
    uint64_t kernel_launches;        /* GPU kernel launches issued (one per batch, or one per request) */
    uint64_t completed;              /* requests completed */
    uint64_t conflict_waits;         /* admissions put off by an overlapping request */
    uint32_t max_inflight_launches;  /* most launches in flight at once */
    uint32_t max_inflight_jobs;      /* most admitted, not completed requests at once */
} rcg_serve_stats;

rcg_status rcg_serve_create(rcg_ctx *ctx, const rcg_serve_config *cfg, rcg_server **out);
/* Queue n requests (before or after rcg_serve_start); *first_id = id of the
 * first.  All or nothing: when any request is invalid (an op other than
 * encode on more than one stripe, or a footprint above the budget, which could
 * never be admitted) none is queued and the call returns RCG_EINVAL. */
rcg_status rcg_serve_submit(rcg_server *s, const rcg_serve_request *reqs, uint32_t n, uint64_t *first_id);
rcg_status rcg_serve_start(rcg_server *s);
/* Wait (at most timeout_ns) until every submitted request has completed. */
rcg_status rcg_serve_drain(rcg_server *s, uint64_t timeout_ns);
/* Timings of requests [0, min(max, submitted)). */
rcg_status rcg_serve_results(rcg_server *s, rcg_serve_result *out, uint64_t max, uint64_t *n);
/* Counters of the server so far. */
rcg_status rcg_serve_get_stats(rcg_server *s, rcg_serve_stats *out);
/* Stop the scheduler (after the launches in flight finish) and free the server. */
rcg_status rcg_serve_destroy(rcg_server *s);

/* ------------------------------------------------ no-allocation batches */

/* The paper has no counterpart to this call: it exists for callers that may
 * not allocate device memory -- a framework whose caching allocator owns all
 * of the GPU's memory, or a submit path that cannot afford the implicit
 * device synchronisation of cudaMalloc/cudaFree.
 *
 * Runs jobs exactly as rcg_batch_submit does (one persistent launch, same
 * kernel, same results), but needs no rcg_ctx and allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine.  Its scratch (the
 * descriptor table, the tile counter and a fallback status word, about 165 KB)
 * is one file-scope device array that every GPU loading librcg holds until
 * the process exits.  The caller passes the inputs and outputs as in
 * rcg_job, plus optionally status_dev: a caller-owned device word that
 * receives the RCG_DEV_* bits of this call (OR-ed in; clear it first).  With
 * status_dev == NULL device-side errors are not reported.
 *
 * Limits and behaviour:
 *  - at most RCG_NOALLOC_MAX_JOBS jobs per call; more is RCG_EINVAL;
 *  - runs on the current device and the given stream, asynchronously;
 *  - the first call on a device also sets that device up (looks up the
 *    scratch array's device address, uploads the inverse tables, sets the
 *    kernel's shared-memory limit); make that first call before any stream
 *    capture;
 *  - a descriptor table of at most 31 744 bytes (as for rcg_batch_submit with
 *    RCG_TABLES_AUTO) travels in the kernels' parameter blocks and leaves the
 *    scratch untouched; a larger one is copied into the scratch;
 *  - every call reuses the same scratch, which keeps the previous call's
 *    contents (the tile counter is cleared on the stream before each launch):
 *    calls whose work overlaps on the GPU race on it, so keep them ordered
 *    (one stream, or events), and do not call it from two host threads at
 *    once. */
#define RCG_NOALLOC_MAX_JOBS 256u
rcg_status rcg_batch_submit_noalloc(const rcg_job *jobs, uint32_t n_jobs, uint32_t *status_dev,
                                    void *stream);

/* ----------------------------------------------------------- utilities */

/* Fill nbytes of device memory with the seeded test-data stream: word w (8
 * bytes little-endian) of stream `seed` is the (w+1)-th output of SplitMix64
 * started from state seed * 2^40; the buffer holds bytes [byte_offset,
 * byte_offset + nbytes) of that stream (byte_offset a multiple of 8). */
rcg_status rcg_fill_random(void *dev, uint64_t nbytes, uint64_t seed, uint64_t byte_offset,
                           void *stream);

/* Failure detection without a fault (not in the paper): launch one thread
 * that waits, with the same bounded mbarrier wait every engine kernel uses,
 * on a barrier nothing completes.  The wait runs out after timeout_ns (at
 * most 10 s), the kernel sets RCG_DEV_TIMEOUT in the context's status word
 * and returns; the context stays usable.  Read the bit with
 * rcg_last_device_status. */
rcg_status rcg_selftest_wait_timeout(rcg_ctx *ctx, uint64_t timeout_ns, void *stream);

/* Host: the per-p table of Section 4.6, (1 + x^z)^(-1) = sum_{j=0}^{(p-1)/2}
 * x^(2jz), for z = 1..p-1, as exponent sets modulo x^p - 1: bit m of masks[z]
 * set means the term x^m (0 <= m < p; x^(p-1) stands for its residue mod f).
 * masks[0] is set to 0.  masks must hold p entries. */
rcg_status rcg_inverse_table(uint32_t p, uint64_t *masks);

/* Host: facts about a prime p (3 <= p <= 61) that decide the code.
 * ord2: the order of 2 modulo p (Lemma 3.3.1: R is a product of
 * (p-1)/ord2 copies of GF(2^ord2)); is_field: ord2 == p - 1 (R is a field);
 * extends: Theorem 3.3.3 holds, checked as "every 1 + x^u + x^v with
 * 0 < u < v < p is a unit of R"; max_data: the largest N a layout may have,
 * 2p - 1 when extends, else p.  RCG_EINVAL for p not an odd prime <= 61. */
typedef struct rcg_prime_info_t {
    uint32_t ord2;
    uint32_t is_field;
    uint32_t extends;
    uint32_t max_data;
} rcg_prime_info_t;
rcg_status rcg_prime_info(uint32_t p, rcg_prime_info_t *out);

/* Host: the inverse in R = F2[x]/(1 + ... + x^(p-1)) of a (bit m = coefficient
 * of x^m, 0 <= m < p-1), computed as a^(2^d - 2), d = ord2 (Lemma 3.3.1), and
 * checked.  RCG_EINVAL when a is not a unit or not a residue (bit p-1 set). */
rcg_status rcg_ring_inverse(uint32_t p, uint64_t a, uint64_t *inv);

/* Host: the tiling the library uses for one stripe geometry. */
typedef struct rcg_plan_info {
    uint32_t tile_bytes;       /* W: column-tile width in bytes (multiple of 16, <= 2048) */
    uint32_t tiles_per_stripe; /* ceil(C / W) */
    uint32_t slot_bytes;       /* shared-memory ring slot: (p-1) rows x W */
    uint32_t n_slots;          /* ring depth */
    uint32_t max_items;        /* the engine's limit on p x W/16 per tile */
    uint32_t smem_bytes;       /* dynamic shared memory of one CTA for this plan */
    uint32_t ctas_per_sm;      /* resident CTAs per SM of the engine shape */
    uint32_t shape;            /* 0 = wide, 1 = pair (the shape RCG_SHAPE_AUTO picks for large launches) */
} rcg_plan_info;
rcg_status rcg_plan(uint32_t p, uint64_t row_bytes, rcg_plan_info *out);

#ifdef __cplusplus
}
#endif

#endif /* RCG_H */
