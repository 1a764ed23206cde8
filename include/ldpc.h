/*
 * ldpc.h -- C ABI of libldpc: GF(2) systematic encoding and sum-product
 * (belief-propagation) decoding of binary LDPC codes on one GB300 GPU.
 *
 * Method: arXiv 2201.04265, "Distributed Processing for Encoding and
 * Decoding of Binary LDPC codes using MPI", Sec. II (Eqs. 1-8) and the
 * encoding/decoding procedures of Sec. III.  The paper's MPI split across
 * CPUs is not reproduced: frames are the data-parallel axis, as in its
 * batch processing (Sec. III-C).
 *
 * Conventions shared by every call
 *   - H is m x n (m checks, n bits), given in CSR form: row_ptr[m+1] and
 *     col_idx[nnz], column indices strictly increasing within a row.  The
 *     position e of an entry in this CSR order is its edge index.
 *   - Bits are packed 32 per uint32, least significant bit first; each frame
 *     occupies whole words (NW = ceil(n/32) for codewords, KW = ceil(k/32)
 *     for information words).  Pad bits must be 0 on input and are 0 on
 *     output.  Codeword bits are in H's column order.
 *   - LLRs are float32, frame-major (frame f at offset f*n), with the
 *     paper's sign: L = ln p(bit=1)/p(bit=0), so L >= 0 decides 1 (Eqs. 4, 8).
 *   - Pointers named d_* are device memory owned by the caller; they must
 *     stay valid until the work queued on `stream` has finished.  Host
 *     pointers (h_* or plain) are read before the call returns.
 *   - Every call except create/destroy/info is asynchronous on `stream`
 *     (NULL = the legacy default stream).  Errors in argument checking are
 *     returned at once; an asynchronous CUDA fault surfaces as LDPC_ECUDA from
 *     a later call or from the caller's own synchronisation.
 *   - Return value: LDPC_OK (0) or a negative ldpc_status; no exception
 *     crosses the ABI.  ldpc_last_error() gives a message for the calling
 *     thread's most recent failure.
 */
#ifndef LDPC_GB300_H
#define LDPC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ldpc_code ldpc_code;
typedef struct CUstream_st *ldpc_stream_t; /* identical to cudaStream_t */

typedef enum {
    LDPC_OK = 0,
    LDPC_EINVAL = -1,   /* bad shape, pointer, degree or option */
    LDPC_ENOMEM = -2,   /* host or device allocation failed */
    LDPC_ECUDA = -3,    /* a CUDA call or kernel launch failed */
    LDPC_ETIMEOUT = -4, /* reserved for a bounded wait inside a kernel that
                           gives up; no kernel of this version waits on
                           another, so no call returns it */
    LDPC_ENOTSUP = -5   /* valid request outside what the library supports */
} ldpc_status;

/* Optional quasi-cyclic description: an mb x nb base matrix of circulant
 * shifts (-1 = all-zero block) lifted by z; entry (i, j, s) connects check
 * i*z + r to bit j*z + (r + s) mod z.  When given, row_ptr/col_idx must be
 * NULL and n = nb*z, m = mb*z. */
typedef struct {
    int32_t mb, nb, z;
    const int16_t *shift; /* host, mb*nb */
} ldpc_qc_desc;

/* flags for ldpc_code_create */
#define LDPC_CREATE_HOST_ONLY 1u /* build host state only (no device tables);
                                    encode/decode with such a code fail */

/* Creates a code object from H (host arrays, copied).  A code created from
 * an ldpc_qc_desc combines the inputs of each check in ascending column order
 * (the same order for all z checks of a base row, which the cluster decoder
 * needs); otherwise each check's order comes from the shared-memory bank
 * schedule (ldpc_code_schedule).  Builds the Tanner
 * graph edge layouts (Sec. II-B, Fig. 1) and the systematic generator
 * (Eq. 2; Sec. III-B: G in standard form [I_k : P] after a column
 * permutation) by GF(2) Gauss-Jordan elimination that scans pivot columns
 * from right to left: the pivot columns are the parity positions, the other
 * k = n - rank(H) columns the information positions, both ascending.  With
 * H = [X | I] this puts the information bits first, as in Fig. 2.
 * Synchronous.  Returns LDPC_EINVAL for a malformed H (n < 1, m < 1, row_ptr
 * not monotone, a column out of range, repeated or unsorted columns in a
 * row) or rank(H) = n. */
int ldpc_code_create(int32_t n, int32_t m, const int32_t *row_ptr, const int32_t *col_idx,
                     const ldpc_qc_desc *qc, uint32_t flags, ldpc_code **out);

/* Sizes of a code: k information bits, rank = n - k parity bits, nnz edges.
 * Any output pointer may be NULL. */
int ldpc_code_info(const ldpc_code *code, int32_t *n, int32_t *m, int32_t *k, int32_t *rank,
                   int64_t *nnz);

/* Host copies of the information positions (k entries) and parity positions
 * (rank entries), both ascending.  Either pointer may be NULL. */
int ldpc_code_positions(const ldpc_code *code, int32_t *info_pos, int32_t *parity_pos);

/* Host copy of the parity map A = P^T: rank rows of KW words; bit i of row j
 * is the coefficient of information bit i in parity bit j (Eq. 3). */
int ldpc_code_parity_map(const ldpc_code *code, uint32_t *A);

/* Host copy of each check's evaluation order: eval_edge[row_ptr[c] + j] is the
 * CSR edge id of the j-th input check c combines (every decoder uses this
 * order, chosen at creation so that the shared-memory gathers of the resident
 * decoders are free of bank conflicts), and *unplaced the number of edges the
 * schedule could not place conflict-free (0 when every warp step touches 32
 * distinct banks).  The paper has no counterpart (the order of the inputs of
 * Eq. 5 does not change its value).  Either pointer may be NULL. */
int ldpc_code_schedule(const ldpc_code *code, int32_t *eval_edge, int64_t *unplaced);

/* Frees the code; NULL is ignored.  Must not race with work still queued
 * that uses it (synchronise the streams first). */
void ldpc_code_destroy(ldpc_code *code);

/* Systematic encoding m^T G = p^T (Eq. 3): d_info is F x KW words, d_code
 * receives F x NW words.  Information bit i lands at info position i;
 * parity bit j (at parity position j) is the XOR of the information bits
 * selected by row j of A.  Every output codeword satisfies H c^T = 0
 * (Eq. 1).  F = 0 is a no-op. */
int ldpc_encode(const ldpc_code *code, const uint32_t *d_info, uint32_t *d_code, int32_t F,
                ldpc_stream_t stream);

/* Four-Russians encoding tables (no counterpart in the paper, which states
 * only the product of Eq. 3).  For each group of 8 information bits and each
 * of the 256 byte values, the XOR of the selected columns of A, so that the
 * parity of a frame is one table row per group and 128 parity bits instead
 * of AND/XOR steps over every word of every row of A.  Builds the tables on
 * the code's device (synchronous; 4 KB per 128 parity bits per 8 information
 * bits: 66 MB for n = 8064 at rate 1/2, 600 MB for n = 26112 at rate 1/3);
 * from then on ldpc_encode uses them, with the same result bits.  *bytes
 * (may be NULL) receives the device memory held (0 when k or rank is 0:
 * nothing to look up, no tables).  Rebuilding replaces the tables.
 * Errors: LDPC_EINVAL (host-only code, wrong device), LDPC_ENOTSUP when
 * 4 ceil(rank/128) > ceil(n/32) (the lookup uses each codeword row as
 * scratch), LDPC_ENOMEM, LDPC_ECUDA.  Must not race with ldpc_encode calls
 * on the same code (synchronise first); so must ldpc_encode_tables_free,
 * which returns ldpc_encode to the AND/XOR form. */
int ldpc_encode_tables_build(ldpc_code *code, size_t *bytes);
int ldpc_encode_tables_free(ldpc_code *code);

/* Syndrome s = H z^T over GF(2) (Eq. 1) of F packed words d_bits (F x NW).
 * d_syn (F x ceil(m/32) words, bit c = check c) and d_ok (F bytes, 1 when
 * every check is satisfied) may each be NULL. */
int ldpc_syndrome(const ldpc_code *code, const uint32_t *d_bits, int32_t F, uint32_t *d_syn,
                  uint8_t *d_ok, ldpc_stream_t stream);

/* Decoder schedules. */
#define LDPC_SCHED_AUTO 0     /* resident when it fits on chip, else plain */
#define LDPC_SCHED_PLAIN 1    /* flooding, messages streamed through HBM,
                                 one check and one bit kernel per iteration */
#define LDPC_SCHED_RESIDENT 2 /* persistent kernel, frames held in shared
                                 memory for all iterations: rows of up to 16
                                 edges with columns of up to 4, or rows of
                                 10-12 with columns of up to 9, and a frame
                                 group that fits one SM (about n <= 8192
                                 for binary16 messages); LDPC_ENOTSUP
                                 otherwise.  With FP32 messages and no more
                                 frames than SMs, each frame gets more
                                 threads (lower latency, same bits) */
#define LDPC_SCHED_CLUSTER 3  /* persistent kernel for quasi-cyclic codes
                                 created from an ldpc_qc_desc whose frames do
                                 not fit one SM: a cluster of 2, 4 or 8 CTAs
                                 holds a frame group in its distributed
                                 shared memory for all iterations, each CTA
                                 owning whole base rows and columns; needs
                                 z a multiple of 32, base rows of at most 16
                                 ones and a part that fits one SM
                                 (LDPC_ENOTSUP otherwise) */

/* Cluster shape the LDPC_SCHED_CLUSTER schedule uses for this code with
 * binary16 (msg_fp16 = 1) or FP32 messages: *ctas CTAs per cluster,
 * *frames_per_group frames decoded together (2 with binary16 messages, one
 * binary16 pair per message word; 1 with FP32), and *local_fraction, the
 * share of base-matrix entries whose row and column the partition gives to
 * the same CTA (the rest are read from a peer CTA every iteration); all 0
 * when the code has no cluster layout.  No counterpart in the paper.  Any
 * pointer may be NULL. */
int ldpc_code_cluster_shape(const ldpc_code *code, int32_t msg_fp16, int32_t *ctas,
                            int32_t *frames_per_group, float *local_fraction);

typedef struct {
    int32_t max_iters;  /* T >= 0 iterations (an iteration = all check
                           updates, then all bit updates; Algorithm 1) */
    int32_t early_stop; /* 1: stop a frame after the first iteration whose
                           hard decisions satisfy H z^T = 0 */
    int32_t msg_fp16;   /* 1: check-to-bit messages stored as binary16
                           (computed and accumulated in FP32) */
    int32_t schedule;   /* LDPC_SCHED_* */
    float clip;         /* |message| clip (> 0): applied to bit-to-check
                           inputs of the check update and to its outputs */
} ldpc_decode_opts;

/* Bytes of device workspace ldpc_decode needs for F frames of this code
 * with these options (0 is possible). */
int ldpc_decode_workspace_size(const ldpc_code *code, int32_t F, const ldpc_decode_opts *opts,
                               size_t *bytes);

/* Sum-product decoding of F frames (Sec. II-B, Eqs. 4-8; flooding schedule
 * of Algorithm 1).  d_llr: F x n channel LLRs R_v.  Per iteration the check
 * update computes E_cv = (-1)^{d_c} 2 atanh( prod_{v' != v} tanh(L_v'c/2) )
 * (Eq. 5 with the sign its LLR convention requires) from the clipped
 * bit-to-check messages L_vc = R_v + sum_{c' != c} E_c'v (Eq. 6), and the
 * bit update forms L_v = R_v + sum_c E_cv (Eq. 7) and z_v = [L_v >= 0]
 * (Eq. 8).  Outputs (each may be NULL): d_post F x n total LLRs of the last
 * iteration performed, d_hard F x NW packed z, d_iters F iteration counts,
 * d_ok F flags (1 when H z^T = 0).  d_work must hold
 * ldpc_decode_workspace_size() bytes, 256-byte aligned. */
int ldpc_decode(const ldpc_code *code, const float *d_llr, int32_t F,
                const ldpc_decode_opts *opts, float *d_post, uint32_t *d_hard, int32_t *d_iters,
                uint8_t *d_ok, void *d_work, size_t work_bytes, ldpc_stream_t stream);

/* ---- Decoding straight from host memory.  F frames of channel LLRs in host
 * memory (h_llr, F x n; page-locked for the copies to overlap) are decoded
 * in chunks of `chunk` frames: chunks are copied to the device on a library
 * upload stream up to two ahead of the chunk being decoded on `stream`, and
 * every chunk's outputs (each host pointer may be NULL) are copied back as
 * soon as it is decoded.  When `stream` reaches the end of the queued work,
 * every output is in host memory.  d_work holds
 * ldpc_decode_host_workspace_size() bytes (three staging buffers and the
 * decoder's own workspace).  The library's upload and
 * download streams and their events are per device and shared: calls from several host threads at once
 * on one device must be serialised by the caller. */
int ldpc_decode_host_workspace_size(const ldpc_code *code, int32_t chunk, const ldpc_decode_opts *opts,
                                    size_t *bytes);
int ldpc_decode_host(const ldpc_code *code, const float *h_llr, int32_t F, const ldpc_decode_opts *opts,
                     float *h_post, uint32_t *h_hard, int32_t *h_iters, uint8_t *h_ok, int32_t chunk,
                     void *d_work, size_t work_bytes, ldpc_stream_t stream);

/* The same pipeline with a record of where the time goes (no counterpart in
 * the paper; a measurement aid): h_ms receives, for each of the
 * ceil(F / chunk) chunks, six times in milliseconds from the call's start on
 * `stream`: upload start and end, decode start and end, download start and
 * end.  Synchronises `stream` before it returns. */
int ldpc_decode_host_timeline(const ldpc_code *code, const float *h_llr, int32_t F,
                              const ldpc_decode_opts *opts, float *h_post, uint32_t *h_hard,
                              int32_t *h_iters, uint8_t *h_ok, int32_t chunk, void *d_work,
                              size_t work_bytes, ldpc_stream_t stream, float *h_ms);

/* ---- Mixed-code batches (serving): frames of several codes decoded in one
 * persistent launch.  A plan holds the codes (each regular with column weight
 * 3 and row weight 6, 9 or 12, at most 8192 bits, e.g. rates 1/2, 2/3, 3/4)
 * and a launch configuration.  ldpc_decode_mixed queues only device work
 * (memsets and kernels) on the stream, so it can be captured in a CUDA graph
 * and replayed; the same frame decoded alone by ldpc_decode gives the same
 * bits, whatever the configuration. */
typedef struct ldpc_mixed ldpc_mixed;

#define LDPC_MIXED_ORDER_LARGEST_FIRST 0 /* work on codes with most edges first */
#define LDPC_MIXED_ORDER_GIVEN 1         /* codes in the order given */
/* (In both orders the codes are then grouped by shape class -- row weight
 * and, with binary16 messages, plane size -- which the plan decodes with one
 * kernel each; the classes after the first run on streams the plan owns,
 * forked from and joined back to the caller's stream with events, so a call
 * stays one capturable sequence.  A plan must not be used by two host
 * threads at once.) */

typedef struct {
    int32_t order;           /* LDPC_MIXED_ORDER_* */
    int32_t groups_per_item; /* frame groups each team takes per work item (1..64) */
    int32_t ctas_per_sm;     /* persistent CTAs per SM (1..4, capped by occupancy) */
} ldpc_mixed_config;

/* codes[ncodes]: code objects on the current device (they must outlive the
 * plan).  msg_fp16 as in ldpc_decode_opts.  Synchronous; allocates the
 * plan's device tables. */
int ldpc_mixed_create(const ldpc_code *const *codes, int32_t ncodes, int32_t msg_fp16,
                      ldpc_mixed **out);
void ldpc_mixed_destroy(ldpc_mixed *plan);
int ldpc_mixed_workspace_size(const ldpc_mixed *plan, int32_t F, size_t *bytes);
int ldpc_mixed_get_config(const ldpc_mixed *plan, ldpc_mixed_config *cfg);
int ldpc_mixed_set_config(ldpc_mixed *plan, const ldpc_mixed_config *cfg);

/* Decodes F frames; frame f uses code d_frame_code[f] (an index into the
 * plan's codes), reads its n_f channel LLRs at d_llr + d_llr_off[f], writes its
 * total LLRs (if d_post) at d_post + d_llr_off[f] and its packed hard decisions
 * (if d_hard) at d_hard + d_hard_off[f] (ceil(n_f/32) words), and d_iters[f],
 * d_ok[f] (each may be NULL).  A frame whose code index is out of range is not
 * decoded and gets iters = -1, ok = 0.  Options as in ldpc_decode_opts. */
int ldpc_decode_mixed(const ldpc_mixed *plan, const int32_t *d_frame_code, const int64_t *d_llr_off,
                      const int64_t *d_hard_off, const float *d_llr, int32_t F, int32_t max_iters,
                      int32_t early_stop, float clip, float *d_post, uint32_t *d_hard,
                      int32_t *d_iters, uint8_t *d_ok, void *d_work, size_t work_bytes,
                      ldpc_stream_t stream);

/* Autotuner: decodes the given batch with every candidate configuration
 * (work order x groups per item x CTAs per SM), each captured in a CUDA graph
 * on a private stream that starts after the work queued on `stream`, and times
 * the graph's replays with CUDA events (`reps` timed replays per candidate
 * after an untimed one, in two passes over the candidates, the second in
 * reverse order); keeps the one with the lowest median time in the plan and
 * returns it in *chosen.  Returns when all its work is done; outputs hold the
 * last replay's (identical) results.  Not to be called during a stream capture. */
int ldpc_mixed_autotune(ldpc_mixed *plan, const int32_t *d_frame_code, const int64_t *d_llr_off,
                        const int64_t *d_hard_off, const float *d_llr, int32_t F, int32_t max_iters,
                        int32_t early_stop, float clip, float *d_post, uint32_t *d_hard,
                        int32_t *d_iters, uint8_t *d_ok, void *d_work, size_t work_bytes,
                        int32_t reps, ldpc_stream_t stream, ldpc_mixed_config *chosen);

/* ---- Weighted belief propagation (training a decoder; not in the paper,
 * which decodes with unit weights).  T unrolled flooding iterations in which
 * a weight w[t][e] (T x nnz, CSR edge order, float32) multiplies the check
 * message E_cv of edge e in iteration t in Eq. 6 and Eq. 7:
 *   L^t_v = R_v + sum_e w[t][e] E^t_e,   bit-to-check L^t_v - w[t][e] E^t_e.
 * With all weights 1 the result equals ldpc_decode with FP32 messages and no
 * early stop, bit for bit. */

/* Bytes of the checkpoint buffer (every iteration's messages and totals) that
 * ldpc_wbp_forward fills and ldpc_decode_backward reads. */
int ldpc_wbp_checkpoint_size(const ldpc_code *code, int32_t F, int32_t T, size_t *bytes);

/* Forward pass: d_llr F x n, d_w T x nnz, d_post F x n receives L^T (natural
 * units).  d_ckpt (>= ldpc_wbp_checkpoint_size bytes, 256-byte aligned) keeps
 * the per-iteration state for the backward pass.  Row degree <= 16, column
 * degree <= 32 (LDPC_ENOTSUP otherwise). */
int ldpc_wbp_forward(const ldpc_code *code, const float *d_llr, int32_t F, int32_t T,
                     const float *d_w, float clip, float *d_post, void *d_ckpt, size_t ckpt_bytes,
                     ldpc_stream_t stream);

/* Bytes of device workspace ldpc_decode_backward needs. */
int ldpc_decode_backward_workspace_size(const ldpc_code *code, int32_t F, int32_t T,
                                        size_t *bytes);

/* Adjoint of ldpc_wbp_forward: given d_grad_post = dloss/dL^T (F x n),
 * writes d_grad_w = dloss/dw (T x nnz, summed over frames in a fixed order, so
 * repeated calls give identical bits) and, if not NULL, d_grad_llr =
 * dloss/dR (F x n).  d_w, clip and the checkpoint must be those of the
 * forward call.  Clipping passes the gradient on the closed range |x| <= clip
 * and blocks it outside. */
int ldpc_decode_backward(const ldpc_code *code, int32_t F, int32_t T, const float *d_w, float clip,
                         const void *d_ckpt, size_t ckpt_bytes, const float *d_grad_post,
                         float *d_grad_w, float *d_grad_llr, void *d_work, size_t work_bytes,
                         ldpc_stream_t stream);

/* The paper has no counterpart to this call.  For callers that cannot
 * allocate device memory while decoding (for example a real-time receive
 * thread that must not block in an allocator, or a framework that owns all
 * device buffers): decodes exactly like ldpc_decode with LDPC_SCHED_PLAIN
 * (opts->schedule must be LDPC_SCHED_AUTO or LDPC_SCHED_PLAIN), but takes its
 * scratch from one static device array of LDPC_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library holds until exit, and allocates nothing.
 * The caller passes inputs and outputs as for ldpc_decode.  Returns
 * LDPC_EINVAL when F frames of this code need more scratch than the array
 * holds (ldpc_decode_workspace_size with the plain schedule gives the need).
 * The first call on a device looks up the array's address; make it before
 * any stream capture.  The address is kept for the life of the process: after
 * cudaDeviceReset on that device it is stale, so this call (like
 * ldpc_decode_host, whose streams are kept the same way) must not be used on
 * that device again in the same process.  All calls share the array: calls
 * whose work overlaps on the GPU race and must be serialised by the caller. */
#define LDPC_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int ldpc_decode_noalloc(const ldpc_code *code, const float *d_llr, int32_t F,
                        const ldpc_decode_opts *opts, float *d_post, uint32_t *d_hard,
                        int32_t *d_iters, uint8_t *d_ok, ldpc_stream_t stream);

/* Test hook, no counterpart in the paper: the device allocation that follows
 * `after` successful ones fails as if the device were out of memory (once;
 * a negative value cancels a pending failure).  Every call that allocates
 * (code creation, encoding tables, mixed plans) then returns LDPC_ENOMEM and
 * frees what it had taken.  Process-wide; for tests of those error paths. */
int ldpc_test_fail_allocation(int32_t after);

/* Status code to a static string. */
const char *ldpc_status_string(int status);

/* Message for the calling thread's most recent failed call ("" if none). */
const char *ldpc_last_error(void);

/* ---------------------------------------------------------------- probe --
 * No counterpart in the paper: a measurement aid.  Measures, on the current
 * device, how many results of ex2.approx, rcp.approx and lg2.approx (the three
 * transcendental instructions of every edge update) one SM delivers per
 * clock, and writes them to rates[0..2].  Synchronous; allocates and frees a
 * few hundred KB of device memory; takes a few milliseconds.  The resident
 * decoder's ALU roofline is built from these rates.
 * Errors: LDPC_EINVAL (rates NULL), LDPC_ECUDA. */
int ldpc_probe_xu_rates(float *rates);

#ifdef __cplusplus
}
#endif

#endif /* LDPC_GB300_H */
