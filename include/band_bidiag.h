/*
 * band_bidiag.h -- C ABI of the GB300 (sm_103a) band -> bidiagonal reducer.
 *
 * The library reduces an upper-banded n x n matrix A of bandwidth b to an
 * upper bidiagonal B = Q^T A P (Q, P orthogonal) by Householder bulge
 * chasing with successive bandwidth reduction: the second stage of the
 * three-stage SVD (arXiv 2510.12705, Section III, Algorithms 1 and 2).
 * B has the same singular values as A; only d = diag(B) and
 * e = superdiag(B) are returned (no singular vectors).
 *
 * Conventions shared by every entry point
 *   - Band storage (LAPACK 'U', 0-based, column-major):
 *         A[i][j] = band[(b + i - j) + j * ldab]   for 0 <= j - i <= b,
 *     ldab >= b + 1.  Entries of the first b columns that lie above row 0
 *     are ignored.  The input band is never modified.
 *   - Element type: BB_F64 (double), BB_F32 (float), BB_F16 (__half) or
 *     BB_BF16 (__nv_bfloat16) for band, d and e.  BB_F32 stores and updates
 *     in FP32 and generates every reflector (norm, beta, tau) in FP64 from the
 *     FP32 data (the precision split).  BB_F16 / BB_BF16 keep the working
 *     band in 16 bits and do everything else as BB_F32 does.
 *   - Device pointers: band, d_out (n elements), e_out (n-1 elements; may be
 *     NULL when n == 1) and workspace are CUDA device pointers on the
 *     current device; the caller owns them.  `stream` is a cudaStream_t
 *     (NULL = legacy default stream).  All work is enqueued on `stream`
 *     and the call returns without synchronising (except where stated).
 *   - b >= n is treated as b = n - 1.  b = 0 gives d = diag(A), e = 0;
 *     b = 1 copies the two diagonals.
 *   - Signs of d and e are those the reflectors produce (singular values are
 *     sign-invariant).
 *   - Return value: BB_OK or a BB_ERR_* code for errors detectable on the
 *     host (arguments, allocation, launch).  Errors found on the device
 *     (a bounded wait that ran out, non-finite input) are recorded in a
 *     sticky per-device status word read by bb_device_status().
 */
#ifndef BAND_BIDIAG_H
#define BAND_BIDIAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes (device status bits use the same values as flags: 1 << code) */
#define BB_OK 0
#define BB_ERR_ARG 1          /* invalid argument (n < 1, b < 0, ldab < b+1, NULL pointer, dtype, tuning) */
#define BB_ERR_ALLOC 2        /* stream-ordered allocation of the internal workspace failed */
#define BB_ERR_LAUNCH 3       /* a kernel launch or a CUDA call failed */
#define BB_ERR_TIMEOUT 4      /* device: a bounded spin-wait saw no progress within the time limit */
#define BB_ERR_NONFINITE 5    /* device: the input band holds NaN or Inf */
#define BB_ERR_WORKSPACE 6    /* caller workspace smaller than the size query returned */
#define BB_ERR_UNSUPPORTED 7  /* configuration outside the compiled kernels (shared memory, n >= 2^20) */

#define BB_F32 0
#define BB_F64 1
/* half-precision storage forms (band, working band and d, e in 16 bits;
 * panels and arithmetic in FP32, reflector generation in FP64, as in the FP32
 * form); entries and row norms must stay inside the storage type's range
 * (FP16: 65504, subnormal below 6.1e-5) */
#define BB_F16 2
#define BB_BF16 3

/* tuning flags */
#define BB_FLAG_INJECT_STALL 0x100   /* fault injection for tests: sweep 0 never reports
                                        progress, so the bounded waits of the other sweeps
                                        run out and the call records BB_ERR_TIMEOUT */

/*
 * Kernel hyperparameters (Section III-C): zero selects the built-in default.
 *   tw               inner tilewidth TW: bandwidth removed per stage (1..32)
 *   tpb              threads per bulge (CTA size: 64, 128, 256 or 512)
 *   sweeps_in_flight persistent CTAs, i.e. sweeps processed concurrently
 *                    (the paper's "max blocks"); capped at what fits on the GPU.
 *                    0 = every CTA that fits, except for FP64 stages of the
 *                    group kernel whose sweeps have at most 3 x (SM count)
 *                    row-bulges: one CTA per SM there
 *   flags            BB_FLAG_*
 *   timeout_s        limit on every device spin-wait without progress, seconds
 *                    (default 5 s)
 *   ev_start/ev_stop optional cudaEvent_t handles (NULL = none): recorded on the
 *                    call's stream immediately before and after the persistent
 *                    bulge-chasing kernels, so a caller can time them alone
 *   group            sweeps one CTA chases together through shared memory (the
 *                    paper's "max blocks" unrolled into one block): 0 = default
 *                    (24), -1 = one sweep per CTA on every stage, k >= 1 = at
 *                    most k (fewer when the window would not fit shared memory).
 *                    A stage (bw -> bw - d) takes min(k, (bw - d) / 3) sweeps per
 *                    CTA; other stages but the last run one sweep per CTA.
 *   teams            sweeps one CTA runs side by side on the last stage (the one
 *                    that ends at bandwidth 1), a team of four warps each, on a
 *                    shared-memory window: 0 = default (one sweep per CTA), -1 =
 *                    one sweep per CTA, k >= 1 = at most min(k, 4) (fewer when
 *                    the window would not fit shared memory)
 *   ev_launch/ev_count/launch_log  optional per-launch timing (NULL / 0 = none):
 *                    ev_launch is an array of ev_count cudaEvent_t handles;
 *                    launch i of the bulge-chasing kernels is bracketed by
 *                    events 2i and 2i+1 (while 2i+1 < ev_count), and, when
 *                    launch_log (host, ev_count / 2 ints) is given, its entry i
 *                    is set to 4 * stage + kernel (0 group, 1 team, 2 per-sweep)
 */
typedef struct {
    int tw;
    int tpb;
    int sweeps_in_flight;
    int flags;
    double timeout_s;
    void *ev_start;
    void *ev_stop;
    int group;
    int teams;
    void **ev_launch;
    int ev_count;
    int *launch_log;
} bb_tuning;

/* one problem of a batch: fields as in band_to_bidiag() */
typedef struct {
    int64_t n;
    int64_t b;
    const void *band;
    int64_t ldab;
    void *d_out;
    void *e_out;
} bb_problem;

/*
 * band_to_bidiag -- reduce one band matrix (Algorithm 1 over all stages:
 * a pack kernel, one persistent launch per stage, an extract kernel).  The
 * workspace (working band with fill rows of
 * height b + 2 TW + 1, Section IV storage format, plus progress counters) is
 * taken from CUDA's stream-ordered allocator on `stream` and released on it.
 */
int band_to_bidiag(int64_t n, int64_t b, int dtype, const void *band, int64_t ldab,
                   void *d_out, void *e_out, void *stream);

/*
 * band_to_bidiag_ex -- as band_to_bidiag with explicit tuning (NULL = default)
 * and an optional caller workspace (device, 256-byte aligned, at least
 * band_to_bidiag_workspace_size() bytes; NULL = stream-ordered allocation).
 * A caller workspace must not be used by two calls that overlap on the GPU.
 */
int band_to_bidiag_ex(int64_t n, int64_t b, int dtype, const void *band, int64_t ldab,
                      void *d_out, void *e_out, const bb_tuning *tuning,
                      void *workspace, size_t workspace_bytes, void *stream);

/* bytes of workspace band_to_bidiag_ex needs for this problem and tuning */
size_t band_to_bidiag_workspace_size(int64_t n, int64_t b, int dtype, const bb_tuning *tuning);

/*
 * dynamic shared memory per CTA of the bulge kernel for this problem and
 * tuning (both panels of a row-bulge); host only, 0 on invalid arguments.  A
 * tuning is usable on a device when this is at most the device's opt-in
 * shared memory per block (227 KB on sm_103a); otherwise the calls return
 * BB_ERR_UNSUPPORTED.
 */
size_t bb_shared_bytes(int64_t n, int64_t b, int dtype, const bb_tuning *tuning);

/*
 * band_to_bidiag_host -- end-to-end call on HOST buffers: copies the band
 * (ldab x n elements) to the device, reduces it, copies d and e back and
 * synchronises `stream`.  band, d_out, e_out are host pointers (pinned
 * memory gives the fastest copies).  Device memory comes from the
 * stream-ordered allocator.  Returns the first host- or device-side error
 * (the device status is read and cleared).
 */
int band_to_bidiag_host(int64_t n, int64_t b, int dtype, const void *band, int64_t ldab,
                        void *d_out, void *e_out, const bb_tuning *tuning, void *stream);

/*
 * Batched reduction of many independent band matrices of uneven n and b in
 * ONE persistent launch (plus a pack and an extract kernel).  A plan holds
 * the problem table in pinned host memory; bb_batch_execute enqueues only
 * stream operations (a host-to-device copy of the table, memsets and three
 * kernels), so it can be captured into a CUDA graph and replayed, as long as
 * the problems' pointers stay valid.
 */
typedef struct bb_batch_plan bb_batch_plan;
bb_batch_plan *bb_batch_plan_create(int count, const bb_problem *problems, int dtype,
                                    const bb_tuning *tuning);
size_t bb_batch_plan_workspace_size(const bb_batch_plan *plan);
int bb_batch_execute(const bb_batch_plan *plan, void *workspace, size_t workspace_bytes,
                     void *stream);
void bb_batch_plan_destroy(bb_batch_plan *plan);

/*
 * band_to_bidiag_batched -- the plan API in one call: plans the `count`
 * problems (host array of descriptors holding device pointers, one dtype),
 * takes the workspace from the stream-ordered allocator on `stream`, enqueues
 * the reduction (pack, one persistent launch per stage and kernel, extract)
 * and releases the workspace on `stream`.  The problem table is copied to the
 * device from pageable host memory, so the caller's array may be reused as
 * soon as the call returns.  Asynchronous; device-side errors go to the
 * status word.  Returns BB_OK, BB_ERR_ARG, BB_ERR_ALLOC, BB_ERR_UNSUPPORTED or
 * BB_ERR_LAUNCH.
 */
int band_to_bidiag_batched(int count, const bb_problem *problems, int dtype, void *stream);

/*
 * Device status: synchronises `stream`, returns the sticky status word of the
 * current device (bit (1 << code) set for each device-side error code seen
 * since the last reset) and clears it when `reset` is non-zero.
 */
int bb_device_status(void *stream, int reset);

/* bb_device_status(stream, 1): read and clear (blocks until `stream` is idle) */
int bb_last_device_status(void *stream);

/* human-readable name of a status code */
const char *bb_status_string(int code);

/*
 * Work model of the executed schedule (host only, no GPU needed): number of
 * stages and row-bulges, floating-point operations (4 m per reflector
 * application to a row or column of length m, plus generation), and
 * elements touched (|right panel U left panel| per row-bulge; algorithmic
 * bytes = 2 * elements * sizeof(element), one read and one write).
 */
int bb_schedule_counts(int64_t n, int64_t b, int tw, int64_t *stages, int64_t *steps,
                       double *flops, double *elements);

/* the same for stage `stage` only (0-based; *stages = total number of stages) */
int bb_stage_counts(int64_t n, int64_t b, int tw, int stage, int64_t *stages, int64_t *steps,
                    double *flops, double *elements);

/*
 * Order of the reflector store of band_to_bidiag_vectors (host only, no GPU
 * needed): *k = the ordinal of step s of sweep R in stage `stage` (0-based)
 * among all row-bulges of the reduction, counted stage by stage, sweep by
 * sweep, step by step -- the order in which the back-transformation applies
 * them.  Row-bulge k keeps its right reflector in slot 2k and its left one in
 * slot 2k + 1.  Returns BB_OK, or BB_ERR_ARG for bad sizes, a NULL k or a
 * row-bulge that the schedule does not have.
 */
int bb_reflector_index(int64_t n, int64_t b, int tw, int stage, int64_t R, int64_t s, int64_t *k);

/* built-in default tuning for (n, b, dtype) */
int bb_default_tuning(int64_t n, int64_t b, int dtype, bb_tuning *out);

/*
 * Microbenchmarks for the roofline denominators, run on `stream` of the
 * current device (synchronous):
 *   bb_measure_l2_bandwidth: read+write bytes/s of a copy kernel over a
 *       `bytes`-sized buffer pair that stays resident in L2, repeated `reps`
 *       times; returns GB/s.
 *   bb_measure_fma_peak: FMA throughput of independent FMA chains in every
 *       thread of a full-GPU grid; dtype BB_F32 or BB_F64; returns GFLOP/s
 *       (2 flops per FMA).
 * Both return a negative value on failure.
 */
double bb_measure_l2_bandwidth(size_t bytes, int reps, void *stream);
double bb_measure_fma_peak(int dtype, void *stream);

/*
 * Tuning (Section III-C hyperparameters; Section IV brute-force search;
 * automatic tuning is the paper's future work, Section VII).
 *
 * bb_autotune -- exhaustive search: reduces the caller's problem once untimed,
 * then `reps` times timed (CUDA events, median) for each of the `ncand`
 * candidate tunings (host array), writes the median times (ms) to times_ms
 * (host, ncand) and the index of the fastest to *best.  A candidate the
 * problem cannot use (BB_ERR_UNSUPPORTED, e.g. panels larger than shared
 * memory) gets time +inf; BB_ERR_UNSUPPORTED is returned only when no
 * candidate runs.  band/d_out/e_out as in band_to_bidiag (d_out, e_out are
 * overwritten).  Synchronous; allocates one workspace from the stream-ordered
 * allocator.
 */
int bb_autotune(int64_t n, int64_t b, int dtype, const void *band, int64_t ldab, void *d_out,
                void *e_out, const bb_tuning *candidates, int ncand, int reps, float *times_ms,
                int *best, void *stream);

/*
 * Learned tuner: a multilayer perceptron in_dim -> hidden -> hidden -> 1 with
 * ReLU activations, FP32, trained with mean squared error and Adam.  All
 * pointers are device pointers; all calls are asynchronous on `stream`.
 * Parameters (bb_mlp_param_count floats, row-major weights):
 *   W1[hidden][in_dim] | b1[hidden] | W2[hidden][hidden] | b2[hidden] | W3[hidden] | b3
 * Requires 1 <= in_dim <= 32 and in_dim <= hidden <= 128, hidden % 32 == 0.
 *   bb_mlp_forward:  X[N][in_dim] -> Y[N]; saves the activations H1, H2 [N][hidden].
 *   bb_mlp_backward: gradient of (1/N) sum (Y - T)^2 with respect to every
 *                    parameter into grads; scratch holds
 *                    bb_mlp_backward_scratch(hidden, N) floats.
 *   bb_mlp_adam:     one Adam step (bias-corrected, step >= 1) on `count`
 *                    parameters with moment buffers m, v.
 * Return BB_OK, BB_ERR_ARG or BB_ERR_LAUNCH.
 */
size_t bb_mlp_param_count(int in_dim, int hidden);
size_t bb_mlp_backward_scratch(int hidden, int N);
int bb_mlp_forward(int in_dim, int hidden, const float *params, const float *X, int N, float *Y,
                   float *H1, float *H2, void *stream);
int bb_mlp_backward(int in_dim, int hidden, const float *params, const float *X, const float *H1,
                    const float *H2, const float *Y, const float *T, int N, float *grads,
                    float *scratch, void *stream);
int bb_mlp_adam(int count, float *params, const float *grads, float *m, float *v, int step,
                float lr, float beta1, float beta2, float eps, void *stream);

/*
 * Singular vectors of the band stage (Section VII: the back-transformation of
 * the stored reflectors): band_to_bidiag_vectors -- the reduction of
 * band_to_bidiag (same arguments and outputs d_out, e_out), which also stores
 * every Householder reflector it builds, followed by the back-transformation
 * that forms the orthogonal Q (q_out) and P (p_out), n x n, column-major
 * (device, leading dimensions ldq, ldp >= n, `dtype`), with
 * Q^T A P = B = bidiag(d, e); Q and P have e1 as their first column and row.
 * The singular vectors of A are then Q and P times those of B.  The last
 * stage always runs one sweep per CTA here (teams are ignored).  workspace:
 * device, >= band_to_bidiag_vectors_workspace_size(n, b, dtype, tuning)
 * bytes, 256-byte aligned (the reduction's workspace plus two slots of
 * (MAXM + 1) values, rounded up to 4, per row-bulge); NULL = allocate it from
 * the stream-ordered allocator.  Cost: the reduction plus two passes over the
 * reflectors, one thread per row of Q and P.  Asynchronous on `stream`.
 * Returns the codes of band_to_bidiag_ex, BB_ERR_ARG also for NULL q_out /
 * p_out or ldq, ldp < n, and BB_ERR_UNSUPPORTED for 16-bit dtypes.  The
 * workspace-size query returns 0 for invalid arguments.
 */
size_t band_to_bidiag_vectors_workspace_size(int64_t n, int64_t b, int dtype, const bb_tuning *tuning);
int band_to_bidiag_vectors(int64_t n, int64_t b, int dtype, const void *band, int64_t ldab,
                           void *d_out, void *e_out, void *q_out, int64_t ldq, void *p_out,
                           int64_t ldp, const bb_tuning *tuning, void *workspace,
                           size_t workspace_bytes, void *stream);

/*
 * Stage 1 of the SVD (Section II: the dense matrix is reduced to band form
 * first; Section V-A: the accuracy experiments start from dense matrices):
 * dense_to_band -- the dense n x n matrix `a` (device, column-major,
 * leading dimension lda >= n, `dtype` BB_F64 or BB_F32; read, never written)
 * to upper band form B = Q^T A P with bandwidth b, written to band_out
 * (device, the LAPACK 'U' layout of band_to_bidiag's input:
 * B[i][j] at band_out[(b + i - j) + j * ldab], ldab >= b + 1; slots above row
 * 0 are set to zero), so its output can be passed to band_to_bidiag as is.
 * Method: Householder QR of b-wide column panels and LQ of b-wide row panels
 * (the larfg convention of the reduction above), the panels by this library's
 * kernels, the compact-WY trailing updates by cuBLAS GEMMs in `dtype`; b >= n-1
 * gives the R of a Householder QR.  The singular values of B are those of A
 * up to rounding.  workspace: device, >= dense_to_band_workspace_size(n, b,
 * dtype) bytes (a working copy of A plus O(n b)), 256-byte aligned; NULL =
 * allocate it from the stream-ordered allocator.  Calls on one device
 * serialise on the library's cuBLAS handle for that device.  Asynchronous on
 * `stream`.  Returns BB_OK, BB_ERR_ARG (n < 1, b < 1, lda < n, ldab < b + 1,
 * NULL pointers, bad dtype), BB_ERR_UNSUPPORTED (16-bit dtypes, n > 2^30),
 * BB_ERR_WORKSPACE, BB_ERR_ALLOC or BB_ERR_LAUNCH.  The workspace-size query
 * returns 0 for invalid arguments.
 */
size_t dense_to_band_workspace_size(int64_t n, int64_t b, int dtype);
int dense_to_band(int64_t n, int64_t b, int dtype, const void *a, int64_t lda, void *band_out,
                  int64_t ldab, void *workspace, size_t ws_bytes, void *stream);
/*
 * dense_to_band_qp -- dense_to_band (same arguments, same band, same
 * workspace size) that also forms its orthogonal factors Q (q_out) and P
 * (p_out), n x n, column-major, device, ldq, ldp >= n, with Q^T A P = B: each
 * panel's block of reflectors I - V T V^T multiplies them from the right, by
 * three GEMMs per panel and side.  With band_to_bidiag_vectors and the
 * bidiagonal's own singular vectors this gives the singular vectors of a
 * dense matrix.  Returns the codes of dense_to_band, BB_ERR_ARG also for NULL
 * q_out / p_out or ldq, ldp < n, BB_ERR_UNSUPPORTED also for ldq or ldp above
 * 2^31 - 1 (the GEMMs take 32-bit leading dimensions).
 */
int dense_to_band_qp(int64_t n, int64_t b, int dtype, const void *a, int64_t lda, void *band_out,
                     int64_t ldab, void *q_out, int64_t ldq, void *p_out, int64_t ldp, void *workspace,
                     size_t ws_bytes, void *stream);

/*
 * Singular values of the upper bidiagonal produced above (the third SVD
 * stage, which the paper hands to LAPACK: Sections V-A and VII), on the GPU.
 * bb_bidiag_sigma -- sigma_out[0..n-1] (device, FP64, descending) = the
 * singular values of B = bidiag(d, e); d (n) and e (n-1) are device arrays of
 * `dtype` BB_F64 or BB_F32 (widened to FP64; 16-bit outputs are converted by
 * the caller first).  Method: one thread per
 * singular value, bisection on the Sturm count of the Golub-Kahan matrix
 * (order 2n, zero diagonal, off-diagonal d0, e0, d1, e1, ...; three-term
 * recurrence without divisions on the squared couplings, computed once,
 * restarted at splits), started from a shared grid of counts over
 * [0, sigma bound] (about n/4 cells, at most 2^14), to an
 * absolute accuracy of about eps * sigma_max (the FP64 resolution for the
 * largest values).  Cost O(n^2 log(1/eps)); asynchronous
 * on `stream`.  workspace: device, >= bb_bidiag_sigma_workspace_size(n) bytes
 * (66048 + 16 n: bounds, grid counts and the 2n - 1 squared couplings),
 * 16-byte aligned.  Returns BB_OK, BB_ERR_ARG (n < 1, NULL pointers, dtype),
 * BB_ERR_WORKSPACE, BB_ERR_UNSUPPORTED (n >= 2^31) or BB_ERR_LAUNCH.
 */
size_t bb_bidiag_sigma_workspace_size(int64_t n);
int bb_bidiag_sigma(int64_t n, int dtype, const void *d, const void *e, double *sigma_out,
                    void *workspace, size_t ws_bytes, void *stream);

/*
 * band_to_bidiag_noalloc -- the paper has no counterpart; this is a library
 * convenience.  Same contract as band_to_bidiag (default tuning), but the call
 * allocates no device memory: its scratch is a statically sized device array
 * defined by this library, for callers that cannot allocate at call time
 * (inside a CUDA stream capture that must stay free of allocation nodes, under
 * an external allocator that owns all device memory, or from host code with no
 * allocation facility).  Limits:
 *   - every GPU that loads the library keeps band_to_bidiag_noalloc_max_bytes()
 *     (16 MiB) reserved until process exit;
 *   - a problem whose workspace (band_to_bidiag_workspace_size with default
 *     tuning) exceeds that size is rejected with BB_ERR_WORKSPACE before any
 *     GPU work;
 *   - all calls on a device share the array: calls whose GPU work may overlap
 *     race and corrupt each other; issue them on one stream;
 *   - the first call on each device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 */
int band_to_bidiag_noalloc(int64_t n, int64_t b, int dtype, const void *band, int64_t ldab,
                           void *d_out, void *e_out, void *stream);
size_t band_to_bidiag_noalloc_max_bytes(void);

#ifdef __cplusplus
}
#endif
#endif /* BAND_BIDIAG_H */
