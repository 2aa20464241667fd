/*
 * zxp.h -- C ABI of libzxp: exact parametric-ZX stabilizer sums on GB300.
 *
 * Method: Sutcliffe & Kissinger, "Fast Classical Simulation of Quantum
 * Circuits via Parametric Rewriting in the ZX-Calculus" (QPL 2024).  A
 * Clifford+T amplitude (Sec. 2.2) is reduced once, on the host, to a
 * parametric scalar (Eq. 2) whose parameters are k Boolean decomposition
 * bits; the library then sums that scalar over all 2^k assignments on the
 * GPU, exactly, in the ring Z[w]/sqrt2^e (w = e^{i pi/4}).
 *
 * Conventions.
 *   - Scalars are (c0 + c1 w + c2 w^2 + c3 w^3) / sqrt2^e with c_j int64.
 *   - Qubit q <-> bit q of a basis index; out_bits[q] is qubit q's value.
 *   - Gates: H = (1/sqrt2)[[1,1],[1,-1]], S = diag(1,i), T = diag(1,w),
 *     CNOT(q0 = control, q1 = target), CZ(q0, q1); Sdg, Tdg their inverses.
 *   - The term of Gray-code index t in [0, 2^k) is the assignment
 *     x = t ^ (t >> 1); a range [first, first+count) sums those terms.
 *
 * Ownership.  Callers own every array they pass (copied during the call).
 * The library owns zxp_scalar and zxp_ctx objects (free with the matching
 * *_free / *_destroy).  Device memory is allocated by the library.
 *
 * Errors.  Every int-returning function returns ZXP_OK (0) or a negative
 * zxp_status; zxp_strerror() names it.  No function aborts the process.
 *
 * Threads.  A zxp_ctx may be used from one thread at a time; distinct
 * contexts (on one or several devices) are independent.  zxp_scalar objects
 * are read-only after creation and may be shared.
 */
#ifndef ZXP_C_API_H
#define ZXP_C_API_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ZXP_OK = 0,
    ZXP_EINVAL = -1,     /* bad argument: qubit, opcode, range beyond 2^k, blob */
    ZXP_ENOMEM = -2,     /* host or device allocation failed */
    ZXP_ETOOBIG = -3,    /* k > 62 or a table exceeds the kernel's limits */
    ZXP_EOVERFLOW = -4,  /* exponent e too large for exact numerators (64-bit
                            results: e > 124 and the value needs more; 128-bit:
                            e > 252) */
    ZXP_ECUDA = -5,      /* a CUDA runtime error (no device, launch failure) */
    ZXP_ETIMEDOUT = -6,  /* a wait budget expired */
    ZXP_EAGAIN = -7,     /* zxp_poll: not finished yet */
    ZXP_ENOTFOUND = -8   /* zxp_poll: unknown ticket */
} zxp_status;

/* Exact scalar (c0 + c1 w + c2 w^2 + c3 w^3) / sqrt2^e.  `flags` bit 0 is
 * set on a raw (not yet canonical) range partial; bit 1 marks a device
 * result that is not valid because a block's bounded wait for its table
 * copies gave up (the host entry points then return ZXP_ETIMEDOUT). */
typedef struct zxp_zomega {
    int64_t c[4];
    int32_t e;
    int32_t flags;
} zxp_zomega;

/* The same with 128-bit coefficients: coefficient j is the two's-complement
 * integer hi[j] * 2^64 + (uint64_t)c[j].  Exact sums of scalars with
 * 124 < e <= 252 (zxp_eval_wide). */
typedef struct zxp_zomega_wide {
    int64_t c[4];
    int64_t hi[4];
    int32_t e;
    int32_t flags;
} zxp_zomega_wide;

typedef enum {
    ZXP_H = 0, ZXP_S = 1, ZXP_T = 2, ZXP_CNOT = 3, ZXP_SDG = 4, ZXP_TDG = 5,
    ZXP_X = 6, ZXP_Z = 7, ZXP_CZ = 8
} zxp_op;

/* 8-byte gate record: op (zxp_op), q0 (qubit or control), q1 (target). */
typedef struct zxp_gate {
    uint8_t op;
    uint8_t reserved0;
    uint16_t q0, q1;
    uint16_t reserved1;
} zxp_gate;

typedef enum { ZXP_AMPLITUDE = 0, ZXP_MARGINAL_DOUBLED = 1 } zxp_kind;

typedef struct zxp_scalar zxp_scalar;  /* compiled parametric scalar */
typedef struct zxp_ctx zxp_ctx;        /* device + stream + workspaces */

/* Statistics of a compiled scalar. */
typedef struct {
    uint32_t k;          /* Boolean parameters a term index runs over: the sum
                            has 2^k terms (each summing 2^k_inner inner ones) */
    uint32_t n_lin;      /* linear phase rows (pi-pair rows with fixed Psi) */
    uint32_t n_quad;     /* quadratic rows (pi-pair rows, two parametric phases) */
    uint32_t n_node;     /* node rows (1 + e^{i Psi}) */
    uint32_t n_pair;     /* phase-pair rows (Eq. 3) */
    int32_t e0;          /* sqrt2 exponent of the denominator */
    uint32_t acc_bits;   /* 64: int64 numerators are provably exact (e0 <= 124);
                            128: zxp_amplitude sums modulo 2^128 (e0 <= 252);
                            0: no exact bound (e0 > 252) */
    uint32_t form_bits;  /* parity forms the kernel tracks per term */
    uint32_t t_count;    /* T-like gates in the input (0 for tables) */
    uint32_t node_words; /* 32-bit words of odd-node form bits per term */
    uint32_t other_words;/* 32-bit words of linear / zero / pair form bits */
    uint32_t device_bytes;       /* bytes of the tables a device evaluation keeps resident */
    uint32_t kernel_variant;     /* 0 table, 1 table + folded bits, 2 general, 3-8 counting
                                    (lane-private 32 / 16 bit, warp-shared; odd: no folded
                                    bits), 9/10 block lookup (10: with folded bits),
                                    11 block lookup with lane-private counters, 13 the
                                    same over two lookup tables; 14/15: 11/13 for a
                                    scalar with inner parameters */
    uint32_t k_inner;    /* inner parameters, summed inside every term (0: none) */
    uint32_t inner_bits; /* index bits of the inner table: k_inner + crossing forms
                            (2^inner_bits entries of 32 bytes on the device) */
    uint32_t upload_bytes;       /* bytes copied host -> device per upload (device_bytes
                                    less the inner table, which the device computes) */
} zxp_scalar_info_t;

/* ---- context --------------------------------------------------------- */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (e.g. a torch stream handle) or NULL for a stream the context creates.
 * Returns ZXP_ECUDA when no usable device is present. */
int zxp_ctx_create(int device, void *cuda_stream, zxp_ctx **out);
void zxp_ctx_destroy(zxp_ctx *ctx);

/* ---- compile (host only, Sec. 3.1-3.2) -------------------------------- */

/* Reduce a circuit to a parametric scalar.
 *   kind = ZXP_AMPLITUDE:          value = <out_bits| C |in_bits>
 *   kind = ZXP_MARGINAL_DOUBLED:   value = <in| C^dag (|b><b|_mask (x) I) C |in>,
 *        the probability that every qubit q in marg_mask reads out_bits[q]
 *        (the doubled diagram of Sec. 2.2; n_qubits <= 64).
 * in_bits may be NULL (all zero).  Arrays have n_qubits entries (0 or 1).
 * A reduction that leaves 32 or more parameters is split as by
 * zxp_scalar_split with default options (when that lowers the term count).
 * Errors: ZXP_EINVAL (qubit out of range, opcode, CNOT with q0 == q1),
 * ZXP_ETOOBIG (the reduction leaves more than 62 parameters). */
int zxp_compile(const zxp_gate *gates, size_t n_gates, int n_qubits,
                const uint8_t *in_bits, const uint8_t *out_bits,
                uint64_t marg_mask, int kind, zxp_scalar **out);

struct zxp_split_opts_s;
/* zxp_compile with the split chosen by the caller: `split` NULL leaves the
 * reduced scalar as it is (every parameter summed term by term, the
 * paper's form); otherwise the scalar is split as by zxp_scalar_split with
 * those options (zxp_split_opts).  Errors as zxp_compile, plus ZXP_EINVAL
 * for bad options. */
int zxp_compile_ex(const zxp_gate *gates, size_t n_gates, int n_qubits,
                   const uint8_t *in_bits, const uint8_t *out_bits,
                   uint64_t marg_mask, int kind, const struct zxp_split_opts_s *split,
                   zxp_scalar **out);

/* Build a scalar from the table layout (little endian):
 *   header  u32 magic 'ZXPS' (0x5350585A), u32 version (1, or 2 with inner
 *           parameters), u32 k, u32 n_lin, u32 n_quad, u32 n_node,
 *           u32 n_pair, i32 e0, i64 G[4]
 *   version 2: u32 k_inner (1..k), u32 0 -- the last k_inner parameters
 *           are inner: a term index runs over the first k - k_inner and each
 *           term sums every value of the inner ones (the value is unchanged);
 *           the outer parts of the forms that cross the two groups may not
 *           use parameters 0-3 (ZXP_EINVAL), and the inner parameters plus
 *           the distinct outer parts of crossing non-Clifford forms are at
 *           most 26 (ZXP_ETOOBIG)
 *   n_lin  x {u64 mask, u32 c, u32 0}        -> w^(c * l(x))
 *   n_quad x {u64 maskA, u64 maskB}          -> w^(4 lA(x) lB(x))
 *   n_node x {u64 mask, u32 g, u32 0}        -> 1 + w^(g + 4 l(x))
 *   n_pair x {u64 maskA, u64 maskB, u32 a, u32 b}
 *            -> 1 + w^(a+4lA) + w^(b+4lB) - w^(a+b+4(lA^lB))      (Eq. 3)
 * with l(x) = parity(mask & x); value = G / sqrt2^e0 * sum over x of the
 * product of all rows (Eq. 2).  Masks may not use bits >= k; k <= 62. */
int zxp_scalar_from_tables(const void *blob, size_t nbytes, zxp_scalar **out);
/* Write the table layout; *nbytes in: capacity, out: size needed.  With
 * buf == NULL only the size is returned. */
int zxp_scalar_to_tables(const zxp_scalar *s, void *buf, size_t *nbytes);
int zxp_scalar_info(const zxp_scalar *s, zxp_scalar_info_t *info);
void zxp_scalar_free(zxp_scalar *s);

/* ---- inner parameters -------------------------------------------------- */

/* Options of zxp_scalar_split (zero fields: defaults). */
typedef struct zxp_split_opts_s {
    uint32_t min_k;           /* scalars with fewer parameters are copied (32) */
    uint32_t max_inner;       /* inner parameters at most (22) */
    uint32_t max_index_bits;  /* inner parameters + crossing forms, <= 26 (24) */
    uint32_t max_cut;         /* crossing non-Clifford forms (3) */
    uint32_t low_free;        /* lowest outer parameters free of the cut, >= 4 (8) */
    uint32_t tries;           /* randomized attempts (24) */
    uint64_t seed;            /* (0: a fixed seed) */
    uint32_t reserved[4];
} zxp_split_opts;

/* Rewrite a scalar so that part of its parameters are summed inside every
 * term (host only; no counterpart in the paper's evaluation, which sums all
 * terms one by one).  The scalar's rows are functions of parity forms, so a
 * linear change of variables rewrites it exactly; in variables where the
 * non-Clifford rows sit on single coordinates (the graph form of the
 * diagram) the parameters are cut into inner ones, coupled to the rest only
 * by pi-pair (Clifford) terms and a few crossing forms, and outer ones.  For
 * every outer assignment the sum over the inner parameters is a
 * Walsh-Hadamard transform of the inner rows' product, read at the cut's
 * parities: one table of 2^inner_bits entries, computed on the device when
 * the scalar is first evaluated there (zxp_inner_sum).  The GPU then walks
 * 2^(k - k_inner) terms instead of 2^k.  Of the splits found, the one of
 * least estimated device time is taken (each more inner parameter halves the
 * walk and doubles the table).  *out has the same value as s (a version-2
 * scalar when the split lowers the term count, else a copy).
 * Errors: ZXP_EINVAL (s already split, bad options), ZXP_ENOMEM. */
int zxp_scalar_split(const zxp_scalar *s, const zxp_split_opts *opts, zxp_scalar **out);

/* Relabel a scalar's parameters (host only): the sum over all of them
 * (Eq. 2) does not depend on their order, but the Gray-code walk flips
 * parameters 0-2 in every aligned block of 8 steps, and its block lookup
 * (one table read per 8 terms) applies only when few parity forms hold them
 * and no phase-pair or zero-test form does.  *out has the same value as s:
 * the three parameters whose forms together are fewest (among those no
 * phase-pair or zero-test form holds, where possible) moved to positions
 * 0-2, the next lightest to 3, the others in their order, when that gives
 * the better block lookup (one table before two, two before none); else a
 * copy of s.  Range partials of *out refer to its order.  Scalars with inner
 * parameters: ZXP_EINVAL (their split already chooses the lowest outer
 * parameters so).  ZXP_ENOMEM. */
int zxp_scalar_reorder(const zxp_scalar *s, zxp_scalar **out);

/* Queue the computation of a split scalar's inner table on the context's
 * stream (a no-op for other scalars).  Evaluations do this once per device
 * by themselves; calling it again recomputes the table (e.g. to time it). */
int zxp_inner_sum(zxp_ctx *ctx, const zxp_scalar *s);

/* ---- evaluate (GPU, Sec. 3.3) ------------------------------------------ */

/* Sum the terms with Gray-code index in [first, first + count) (index t:
 * outer parameters gray(t), every inner value), multiplied
 * by G, into *out as a raw partial over sqrt2^e0 (flags bit 0 set).  The
 * call blocks until the result is on the host.  Partials of disjoint
 * ranges combine with zxp_zomega_add; the total over [0, 2^k) gives the
 * scalar after zxp_zomega_canon.  Errors: ZXP_EINVAL (range beyond 2^k),
 * ZXP_ECUDA, ZXP_ETIMEDOUT (flags bit 1). */
int zxp_eval(zxp_ctx *ctx, const zxp_scalar *s, uint64_t first, uint64_t count,
             zxp_zomega *out);

/* Device-side form of zxp_eval: queue the range on the context's stream
 * and write the raw partial (the 40-byte zxp_zomega layout, flags bit 0
 * set) to `dev_out`, a device pointer aligned to 8 bytes.  Returns without
 * waiting; the value is ready when the context's stream reaches this point
 * (synchronise that stream, or order work after it).  The call reuses the
 * context's workspace, so calls on one context must not overlap in time on
 * different streams.  Errors: ZXP_EINVAL (range, null or unaligned
 * pointer), ZXP_ECUDA. */
int zxp_eval_device(zxp_ctx *ctx, const zxp_scalar *s, uint64_t first, uint64_t count,
                    zxp_zomega *dev_out);

/* zxp_eval_device without any allocation (the paper has no counterpart;
 * scalars with inner parameters: ZXP_ETOOBIG).
 * For callers that cannot allocate device memory through the CUDA runtime:
 * code under a memory manager that owns the whole device (a framework's
 * caching allocator, a serving runtime's fixed arena) and latency-critical
 * loops, where cudaMalloc / cudaFree would synchronise the device.  It needs
 * no zxp_ctx.  The tables of `s` are staged, and the kernel's scratch (the
 * 4 x 64-bit accumulator and the completion counter) kept, in one
 * file-scope device array of 256 KB (the launch uses at most 2048 blocks),
 * held on every GPU that loads the library until the process exits.  The range is queued on `cuda_stream`
 * (NULL: the legacy default stream) of the current device, and the raw
 * partial (40-byte zxp_zomega layout, flags bit 0 set) lands at `dev_out`, a
 * caller-owned device pointer aligned to 8 bytes, when the stream reaches it.
 * Every call looks up the array's device address (cudaGetSymbolAddress, a
 * host-side lookup) with the current device, so calls stay valid after a
 * reset of the device's primary context; make the first call on a device
 * before any stream capture (it loads the library's device code).  Under
 * stream capture the table copies become graph nodes that read the
 * scalar's host tables at every replay: the scalar must then stay alive,
 * and unchanged, until the graph is destroyed.  No device allocation and no
 * cudaMalloc / cudaFree are made; on the host, the first call for a kernel
 * variant on a device fills the launch-shape caches (host allocations) and
 * the runtime stages the pageable table copies.  Every call shares the array and it keeps the
 * last call's contents (the counter is cleared at each call): calls that
 * overlap on the GPU, e.g. on two streams, race.  Errors: ZXP_EINVAL (range,
 * null or unaligned pointer), ZXP_ETOOBIG (tables larger than the array),
 * ZXP_ECUDA. */
int zxp_eval_noalloc(const zxp_scalar *s, uint64_t first, uint64_t count,
                     zxp_zomega *dev_out, void *cuda_stream);

/* The whole sum over [0, 2^k), canonical (the exact value of Eq. 2; for a
 * circuit amplitude N / sqrt2^e0 every |N_j| <= 2^(e0/2)).  e0 <= 124: summed
 * with 64-bit coefficients; 124 < e0 <= 252: summed modulo 2^128
 * (zxp_amplitude_wide) and returned when the canonical coefficients fit 64
 * bits.  Errors as zxp_eval, plus ZXP_EOVERFLOW when e0 > 252 (`out` then
 * holds the canonical form of the 64-bit sum, exact only if the true
 * numerator fits) or when the canonical value needs more than 64 bits (use
 * zxp_amplitude_wide). */
int zxp_amplitude(zxp_ctx *ctx, const zxp_scalar *s, zxp_zomega *out);

/* zxp_eval modulo 2^128 (any e0): the raw partial of [first, first + count)
 * with 128-bit coefficients, flags bit 0 set.  Each term is evaluated on its
 * own (the general per-term walk) from 128-bit tables that the first call
 * on a device uploads next to the 64-bit ones (with inner parameters also a
 * 128-bit inner table, 64 bytes per entry); they stay resident until the
 * scalar is freed.  Synchronous on the context's stream.  Errors as
 * zxp_eval. */
int zxp_eval_wide(zxp_ctx *ctx, const zxp_scalar *s, uint64_t first, uint64_t count,
                  zxp_zomega_wide *out);

/* The whole sum over [0, 2^k) in chunks of 2^chunk_log2 terms, resumable
 * across processes (the paper's exact sum, Eq. 2, for scalars whose full
 * evaluation outlasts one job).  After every chunk the running partial sum
 * (64-bit words, or 128-bit when e0 > 124) and the set of finished chunks
 * are written to the host file `path`: first to `path`.tmp, flushed to the
 * disk, then renamed over `path`, so the file always holds one complete
 * state and a process that ends between chunks loses at most the chunk in
 * flight.  A call that finds the file continues it: chunks already summed
 * are not run again.  The file names the scalar (a 64-bit FNV-1a digest of
 * its table bytes), k, chunk_log2 and e0; a file that differs, or is
 * damaged (a 64-bit checksum over its bytes), is ZXP_EINVAL and is left
 * alone.  At most max_chunks further chunks run (0: no limit); while chunks
 * remain the call returns ZXP_EAGAIN.  When all are summed it returns the
 * canonical amplitude in `out` with zxp_amplitude's status (the file stays:
 * a further call returns the value without running anything; delete it to
 * start again).  chunks_done / chunks_total (may be NULL) receive the
 * progress.  The layout of the file is documented in checkpoint.h.  Errors:
 * ZXP_EINVAL (arguments, a foreign or damaged file, a file that cannot be
 * written), the evaluation's errors. */
int zxp_sum_resumable(zxp_ctx *ctx, const zxp_scalar *s, uint32_t chunk_log2, const char *path,
                      uint64_t max_chunks, zxp_zomega *out, uint64_t *chunks_done, uint64_t *chunks_total);

/* Bounded table waits, for tests (no counterpart in the paper).  Every
 * block of a single-scalar sum kernel waits a bounded time (about a second)
 * for the bulk copies of its tables into shared memory; a block that gives
 * up skips its terms and marks the launch's result (flags bit 1), which the
 * host entry points report as ZXP_ETIMEDOUT.  enable != 0: the launches
 * queued from now on in this process expect 16 bytes more than their copies
 * deliver, so every block's wait runs to its limit (long after its copies
 * have landed) and gives up; enable = 0 restores normal launches. */
int zxp_test_table_timeout(int enable);

/* The whole sum modulo 2^128, canonical: exact for e0 <= 252 (the
 * numerator's coefficients are below 2^126 in magnitude).  ZXP_EOVERFLOW
 * when e0 > 252 (`out` then holds the canonical form of the 128-bit sum). */
int zxp_amplitude_wide(zxp_ctx *ctx, const zxp_scalar *s, zxp_zomega_wide *out);

/* Asynchronous form of zxp_eval: queue the range on the context's stream
 * and return a ticket.  The scalar must stay alive until the ticket is
 * polled to completion. */
int zxp_submit(zxp_ctx *ctx, const zxp_scalar *s, uint64_t first, uint64_t count,
               uint64_t *ticket);
/* Wait up to timeout_us (0: do not wait, < 0: wait without limit) for a
 * ticket.  ZXP_OK: *out holds the raw partial and the ticket is released.
 * ZXP_EAGAIN: not finished.  ZXP_ENOTFOUND: unknown ticket. */
int zxp_poll(zxp_ctx *ctx, uint64_t ticket, int64_t timeout_us, zxp_zomega *out);
/* One call for a client holding a scalar's table bytes (the layout of
 * zxp_scalar_from_tables): build the scalar, queue its whole sum [0, 2^k)
 * like zxp_submit and return a ticket.  The library owns that scalar and
 * frees it when the ticket is released by zxp_poll (or the context is
 * destroyed); the blob is copied at the call.  Errors: those of
 * zxp_scalar_from_tables and zxp_submit. */
int zxp_submit_tables(zxp_ctx *ctx, const void *blob, size_t nbytes, uint64_t *ticket);

/* ---- parametric scalars: one reduction for many bitstrings ---------------- */

/* The paper's own use (Sec. 3, Sec. 4): the output bits of the flagged
 * qubits (kind ZXP_AMPLITUDE), or the projected bits of the flagged qubits
 * inside marg_mask (kind ZXP_MARGINAL_DOUBLED), stay Boolean parameters
 * through the whole reduction.  The result is reduced once; zxp_bind then
 * turns it into an ordinary scalar for any values of the parameters (host
 * work linear in its size), whose value is exactly that of zxp_compile with
 * those bits.  Parameter j is the j-th flagged qubit in ascending order.
 * A parametric reduction can need more decomposition parameters k than a
 * reduction with fixed bits (fewer simplifications apply, Lemma 1). */
typedef struct zxp_pscalar zxp_pscalar;

typedef struct {
    uint32_t k;                  /* summed variables of every bound scalar */
    uint32_t n_params;
    uint32_t n_lin, n_quad, n_node, n_pair;
    int32_t e0;
    uint32_t t_count;
    uint32_t reserved[8];
} zxp_pscalar_info_t;

/* param_qubits: n_qubits entries, nonzero = parameter (at most 64 count);
 * out_bits gives the bits of the other qubits.  Errors as zxp_compile. */
int zxp_compile_param(const zxp_gate *gates, size_t n_gates, int n_qubits,
                      const uint8_t *in_bits, const uint8_t *out_bits,
                      const uint8_t *param_qubits, uint64_t marg_mask, int kind,
                      zxp_pscalar **out);
int zxp_pscalar_info(const zxp_pscalar *ps, zxp_pscalar_info_t *info);
/* qubits[j] = the qubit of parameter j (n_params entries). */
int zxp_pscalar_params(const zxp_pscalar *ps, uint32_t *qubits);
/* The scalar for parameter values `bits` (bit j = parameter j). */
int zxp_bind(const zxp_pscalar *ps, uint64_t bits, zxp_scalar **out);
void zxp_pscalar_free(zxp_pscalar *ps);

/* ---- batches: many scalars, one persistent launch per kernel variant ------ */

/* A batch evaluates the full sums of n scalars of uneven k together: every
 * scalar's range is cut into chunks that resident blocks take from one
 * work-stealing queue (App. E's reduction becomes 64-bit atomic adds into each
 * scalar's result).  zxp_batch_create uploads the descriptors, times a few
 * launch shapes (chunk size 2^12..2^20 terms, 128 or 256 threads per block)
 * on the actual batch, keeps the fastest, and captures the whole evaluation
 * (clears, launches, result copy) as a CUDA graph on the context's stream;
 * zxp_batch_run replays it.  The scalars must outlive the batch; the context
 * must not be used from another thread during create or run. */
typedef struct zxp_batch zxp_batch;

typedef struct {
    uint32_t n_scalars;
    uint32_t n_groups;           /* launches per run (one per kernel variant) */
    uint32_t n_chunks;
    uint32_t threads;            /* threads per block chosen by the tuner */
    uint32_t chunk_log2;         /* chunk length 2^chunk_log2 terms chosen by the tuner */
    uint32_t candidates;         /* launch shapes timed */
    double tuned_us;             /* device time of the chosen shape */
    double total_terms;          /* sum of 2^k */
    uint32_t reserved[6];
} zxp_batch_info_t;

/* Errors: ZXP_EINVAL (n == 0, null scalar, a scalar with inner
 * parameters), ZXP_ENOMEM, ZXP_ECUDA. */
int zxp_batch_create(zxp_ctx *ctx, const zxp_scalar *const *scalars, size_t n,
                     zxp_batch **out);
/* Run the batch and wait: out[i] receives scalar i's full raw sum (as
 * zxp_eval over [0, 2^k); canonicalise with zxp_zomega_canon). */
int zxp_batch_run(zxp_batch *b, zxp_zomega *out);
int zxp_batch_info(const zxp_batch *b, zxp_batch_info_t *info);
void zxp_batch_destroy(zxp_batch *b);

/* ---- request server: continuous batching ---------------------------------- */

/* A server owns a request loop on one context.  Requests (a circuit plus
 * output bits and kind, as for zxp_compile, or an already compiled scalar)
 * are accepted at any time from any thread.  Host worker threads compile
 * them; a scheduler thread admits compiled scalars to the device while the
 * device arena has room for their tables and a result slot is free, keeps
 * their tables and partial sums resident there, and runs steps: each step
 * gives every resident request a share of a term budget (small requests
 * whole, shortest first; what is left to the large ones, oldest first, so a
 * 2^40-term request proceeds in resumable chunks while small ones pass it)
 * and evaluates all shares together in one persistent launch per kernel
 * variant (the batch kernel).  Requests that arrive while steps are on the
 * device join the next step; finished values are copied back per step.
 * Two steps are in flight at a time.  The arithmetic is that of zxp_eval:
 * each value is exactly the one zxp_amplitude returns for the same scalar.
 *
 * policy ZXP_SERVE_PLAIN runs the same loop one request at a time, one
 * launch over its whole range (the one-scalar-per-launch baseline).
 *
 * The server is not part of the paper (its evaluation is offline); it is
 * the serving form of the sum in Sec. 4. */
typedef struct zxp_server zxp_server;

typedef enum { ZXP_SERVE_BATCHED = 0, ZXP_SERVE_PLAIN = 1 } zxp_serve_policy;

typedef struct {
    uint32_t policy;             /* zxp_serve_policy */
    uint32_t max_k;              /* admission: larger k completes with ZXP_ETOOBIG (0: 44) */
    uint32_t compile_threads;    /* host compile workers (0: hardware threads, at most 16) */
    uint32_t max_active;         /* requests resident on the device (0: 4096) */
    uint64_t arena_bytes;        /* device memory for resident tables (0: 64 MiB) */
    uint64_t step_terms;         /* term budget of one step (0: 2^30) */
    uint64_t small_terms;        /* requests with at most this many terms left run whole (0: 2^22) */
    uint32_t chunk_log2;         /* chunk length 2^chunk_log2 terms (0: 20) */
    uint32_t threads;            /* threads per block of the batch kernel (0: 128) */
    uint32_t reserved[8];
} zxp_server_opts;

typedef struct {
    const zxp_gate *gates;
    size_t n_gates;
    int32_t n_qubits;
    int32_t kind;                /* zxp_kind */
    const uint8_t *in_bits;      /* NULL: all zero */
    const uint8_t *out_bits;     /* n_qubits entries */
    uint64_t marg_mask;
} zxp_request;

/* Per-request record, times in microseconds since the server started. */
typedef struct {
    double submit_us;
    double compiled_us;          /* compile finished (submit time for scalars) */
    double admitted_us;          /* tables resident on the device */
    double done_us;              /* value back on the host */
    uint32_t k;
    uint32_t steps;              /* steps that carried part of its range */
    int32_t status;              /* ZXP_OK, or the error that ended it */
    uint32_t reserved;
} zxp_request_timing;

typedef struct {
    uint64_t submitted, completed, rejected;   /* rejected: ZXP_ETOOBIG at admission */
    uint64_t steps, launches;
    double terms;                /* terms evaluated */
    double device_busy_us;       /* sum of step device times */
    uint32_t active, peak_active;
    uint64_t arena_bytes, arena_peak;
    uint32_t reserved[8];
} zxp_server_stats_t;

/* opts may be NULL (all defaults).  Errors: ZXP_EINVAL, ZXP_ENOMEM, ZXP_ECUDA.
 * The context must outlive the server and is used only by its scheduler. */
int zxp_server_create(zxp_ctx *ctx, const zxp_server_opts *opts, zxp_server **out);
/* Copy the request and queue it; *ticket identifies it.  ZXP_EINVAL for a
 * malformed request (checked again, fully, by the compiler). */
int zxp_server_submit(zxp_server *srv, const zxp_request *req, uint64_t *ticket);
/* Queue a compiled scalar (borrowed: it must stay alive until its ticket
 * has been polled to completion).  ZXP_EINVAL for a scalar with inner
 * parameters (zxp_scalar_split), which only the single-scalar entry points
 * evaluate. */
int zxp_server_submit_scalar(zxp_server *srv, const zxp_scalar *s, uint64_t *ticket);
/* Queue the binding `bits` of a parametric scalar (borrowed: it must stay
 * alive until the ticket has been polled); a compile worker binds it. */
int zxp_server_submit_bind(zxp_server *srv, const zxp_pscalar *ps, uint64_t bits,
                           uint64_t *ticket);
/* Wait up to timeout_us (0: do not wait, < 0: without limit).  Returns
 * ZXP_EAGAIN while the request runs, ZXP_ENOTFOUND for an unknown ticket;
 * otherwise the request's own status (ZXP_OK: *out holds the canonical
 * value; ZXP_EOVERFLOW: as zxp_amplitude), and the ticket is released.
 * (A request with 124 < e0 <= 252 is summed again modulo 2^128 when its
 * step ends, synchronously on the server's stream, as zxp_amplitude does.)
 * out and timing may be NULL. */
int zxp_server_poll(zxp_server *srv, uint64_t ticket, int64_t timeout_us, zxp_zomega *out,
                    zxp_request_timing *timing);
int zxp_server_stats(zxp_server *srv, zxp_server_stats_t *stats);
/* Finish every queued request, then stop the threads and free everything. */
void zxp_server_destroy(zxp_server *srv);

/* ---- weak simulation and marginals by summing ----------------------------- */

/* Weak simulation by chained marginals (Sec. 2.2; App. F, Algorithm 2).
 * zxp_sampler_create reduces the n doubled diagrams P(a_0 .. a_j),
 * j = 0 .. n-1, once each with the bits a_0 .. a_j as parameters (n <= 64).
 * zxp_sampler_draw then draws n_samples bitstrings together: for each qubit
 * j in turn it evaluates P(B_i || 0) for every sample i on the device (one
 * step of continuous batching for all samples) and sets bit j of sample i to
 * 0 if u[i*n + j] < P(B_i || 0) / P(B_i), else to 1, where P(B_i) is the
 * exact probability of the prefix drawn so far.  The uniforms u in [0, 1)
 * are the caller's.  The comparison uses doubles computed from the exact
 * values as (c0 + (c1 - c3) / sqrt2) 2^(-e/2) (one more 1/sqrt2 for odd e),
 * in that order of IEEE operations.  The algorithm as printed compares u
 * with P(B_i || 0) alone; the ratio, which Sec. 2.2 states, is used.
 * out_bits: n_samples x n (row-major, bit j of sample i at [i*n + j]);
 * prob (nullable): the exact probability of each drawn bitstring.
 * The context must not be used by other threads while a sampler exists. */
typedef struct zxp_sampler zxp_sampler;
int zxp_sampler_create(zxp_ctx *ctx, const zxp_gate *gates, size_t n_gates, int n_qubits,
                       const uint8_t *in_bits, zxp_sampler **out);
/* k_per_prefix: n entries, the summed variables of each reduced marginal. */
int zxp_sampler_info(const zxp_sampler *s, uint32_t *k_per_prefix);
int zxp_sampler_draw(zxp_sampler *s, size_t n_samples, const double *u, uint8_t *out_bits,
                     zxp_zomega *prob);
void zxp_sampler_destroy(zxp_sampler *s);

/* The marginal probability that the qubits in mask read bits[q], by the
 * summing approach of Sec. 2.2: the amplitude is reduced once with the
 * other output bits as parameters and sum_b |<b|C|in>|^2 is taken exactly
 * over their 2^(n - |mask|) values (at most 2^30).  bits has n_qubits entries
 * (those outside mask are ignored).  Same value as zxp_compile with
 * ZXP_MARGINAL_DOUBLED and zxp_amplitude. */
int zxp_marginal_by_sum(zxp_ctx *ctx, const zxp_gate *gates, size_t n_gates, int n_qubits,
                        const uint8_t *in_bits, uint64_t mask, const uint8_t *bits,
                        zxp_zomega *out);

/* ---- measurement ------------------------------------------------------------ */

/* Integer throughput of the context's GPU (no counterpart in the paper; the
 * roofline denominator of the sum kernel, which is bound by integer issue).
 * A full resident grid runs eight chains of one instruction per thread:
 * kind 0 three-input logic (lop3), 1 add, 2 popcount, 3 multiply-add
 * (mad.lo), 4 logic and multiply-add in turn (the ALU and FMA pipes
 * together); *thread_instr_per_s receives the best of
 * three timed launches (thread instructions per second) and *ms (nullable)
 * that launch's time.  Errors: ZXP_EINVAL, ZXP_ENOMEM, ZXP_ECUDA. */
int zxp_int_peak(zxp_ctx *ctx, int kind, double *thread_instr_per_s, double *ms);

/* ---- exact scalar helpers (host) ---------------------------------------- */

/* a + b, after bringing both to the larger exponent (x sqrt2 per step). */
int zxp_zomega_add(const zxp_zomega *a, const zxp_zomega *b, zxp_zomega *out);
/* Canonical form: divide by sqrt2 while e > 0 and the numerator allows;
 * zero is (0,0,0,0; e = 0). */
int zxp_zomega_canon(const zxp_zomega *in, zxp_zomega *out);
void zxp_zomega_to_complex(const zxp_zomega *z, double *re, double *im);

const char *zxp_strerror(int status);
/* "zxp <version> sm_103a" */
const char *zxp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ZXP_C_API_H */
