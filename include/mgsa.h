/*
 * mgsa.h - A-orthonormal thin QR by modified Gram-Schmidt on GB300 (sm_103a).
 *
 * Computes, for a sparse symmetric positive definite A (m x m, CSR, FP64) and
 * a tall matrix Z (m x n, m >= n, FP64), the factorization
 *
 *     Z = Q R,   Q^T A Q = I_n,   R upper triangular with positive diagonal
 *
 * (Imakura & Yamamoto, arXiv 1703.10440, Section 1, eq. (1)), by modified
 * Gram-Schmidt under the A-inner product (x, y)_A = x^T A y, in one of three
 * forms (Section 2):
 *
 *   MGSA_NAIVE  Algorithms 3/4: two sparse matrix-vector products (MV) per
 *               column, x_i = A z_i and p_i = A q_i (2n MV in total).
 *   MGSA_HA     Algorithms 5/7 (high accuracy): one MV per column,
 *               x_i = A z_i, and p_i = x_i / r_ii (eq. (tec1)), n MV.
 *   MGSA_HP     Algorithms 6/8 (high performance): one block product X = A Z
 *               up front; the A-images are carried by the recurrence
 *               x_j <- x_j - r_ij p_i (eq. (tec2)), p_i = x_i / r_ii.
 *
 * All three run right-looking (the row-oriented Algorithms 4, 7, 8): step i
 * forms r_ii = sqrt(z_i^T x_i), q_i = z_i / r_ii, p_i, the row
 * r_ij = p_i^T z_j (j > i) and the rank-1 updates z_j <- z_j - r_ij q_i
 * (and x_j <- x_j - r_ij p_i for HP).  Every step runs in CUDA kernels of this
 * library; nothing runs on the host but argument checks and launches.
 *
 * Conventions shared by every entry point:
 *   - Matrices are column-major with a leading dimension (LAPACK style).
 *   - Pointers named *_dev / in mgsa_csr / Z, Q, R of mgsa_qr are device
 *     memory owned by the caller; the library never frees them.
 *   - The library owns its workspace (allocated by mgsa_create and grown by
 *     mgsa_reserve or by the first call that needs more).
 *   - Argument errors are detected on the host and returned synchronously,
 *     before anything is launched.  Numerical failures (breakdown) are
 *     recorded in a device status word that mgsa_get_info reads.
 *   - No exception crosses this interface and nothing is printed.
 *   - A handle is not thread-safe: use one handle per host thread / stream.
 *   - Results are deterministic: the same inputs, sizes and device give
 *     bitwise identical Q and R on every call.
 */
#ifndef MGSA_H
#define MGSA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (cudaStream_t is `struct CUstream_st *`); NULL is the legacy
 * default stream. */
typedef struct CUstream_st* mgsa_stream_t;

typedef struct mgsa_context* mgsa_handle;

typedef enum {
  MGSA_NAIVE = 0,     /* Algorithm 4: 2n MV */
  MGSA_HA = 1,        /* Algorithm 7: n MV, p_i = x_i / r_ii */
  MGSA_HP = 2,        /* Algorithm 8: X = AZ once, x-recurrence */
  /* Classical Gram-Schmidt counterparts (Section 2.3; recurrences in Section
   * 3.3): r_ij = p_i^T z_j^{(0)}, run column by column (left-looking).  Their
   * loss of A-orthogonality grows with kappa(A^{1/2} Z)^2 (Section 4.2), not
   * linearly as for MGS.  mgsa_qr / mgsa_qr_host / mgsa_reserve only. */
  MGSA_CGS_NAIVE = 3, /* 2n MV */
  MGSA_CGS_HA = 4,    /* n MV, p_j = x_j / r_jj */
  MGSA_CGS_HP = 5     /* X = AZ once, x-recurrence */
} mgsa_variant;

typedef enum {
  MGSA_OK = 0,
  MGSA_ERR_INVALID = 1,   /* bad argument; nothing was launched */
  MGSA_ERR_BREAKDOWN = 2, /* z_j^T x_j <= 0 at some column (A not SPD or Z rank deficient) */
  MGSA_ERR_NONFINITE = 3, /* z_j^T x_j is NaN or Inf at some column */
  MGSA_ERR_NOMEM = 4,     /* workspace allocation failed */
  MGSA_ERR_CUDA = 5,      /* a CUDA runtime call failed */
  MGSA_ERR_TIMEOUT = 6    /* a device-wide wait gave up (bounded spin); results undefined */
} mgsa_status;

/* Sparse symmetric positive definite A in CSR form, both triangles stored.
 * rowptr: m+1 int32, rowptr[0] = 0, non-decreasing, rowptr[m] = nnz.
 * col:    nnz int32 in [0, m).  val: nnz FP64.
 * All three arrays are device memory owned by the caller.  Entries of a row
 * are summed in the order stored. */
typedef struct {
  int64_t m;
  int64_t nnz;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
} mgsa_csr;

/* Largest n accepted by mgsa_qr. */
#define MGSA_MAX_N 2048

/* Create a handle bound to CUDA device `device`.  Allocates the control block
 * (status word and device-wide barrier state).  Returns MGSA_ERR_INVALID for a
 * NULL h or a bad device, MGSA_ERR_NOMEM / MGSA_ERR_CUDA on failure. */
mgsa_status mgsa_create(mgsa_handle* h, int device);

/* Release every allocation of the handle (synchronizes the device first).
 * NULL is accepted and ignored. */
mgsa_status mgsa_destroy(mgsa_handle h);

/* Grow the workspace so that mgsa_qr(m, n, v) allocates nothing; call it
 * before capturing mgsa_qr into a CUDA graph. */
mgsa_status mgsa_reserve(mgsa_handle h, int64_t m, int n, mgsa_variant v);

/* Bytes of device workspace mgsa_qr needs for (m, n, v). */
size_t mgsa_workspace_bytes(mgsa_handle h, int64_t m, int n, mgsa_variant v);

/* A-orthonormal thin QR of Z (Section 1, eq. (1)), right-looking MGS in the
 * form `v` (Algorithm 4, 7 or 8), or left-looking CGS (MGSA_CGS_*).
 *
 *   A      CSR matrix with A->m == m (device arrays, read only).
 *   Z      m x n input, column-major, leading dimension ldz >= m (read only).
 *   Q      m x n output, leading dimension ldq >= m.  Either Z itself (Q == Z
 *          and ldq == ldz: the factorisation runs in place) or not
 *          overlapping Z at all.
 *          Q is also the working storage of the z_j^{(i)} columns.
 *   R      n x n output, leading dimension ldr >= n; written in full, zeros
 *          below the diagonal.  The CTAs of one launch also pass the sums of
 *          each row (column for CGS) to each other through R; its contents
 *          are final once the queued work has completed.
 *   s      stream the work is queued on; the call returns without waiting.
 *
 * Requirements: 1 <= n <= MGSA_MAX_N, n <= m < 2^31, nnz < 2^31.
 * Q's columns q_i are formed as z_i * (1 / r_ii) (one reciprocal per column).
 * Returns MGSA_OK once queued; a numerical failure is reported later by
 * mgsa_get_info.  If the workspace must grow, this call allocates (and is then
 * not capturable into a CUDA graph); mgsa_reserve avoids that. */
mgsa_status mgsa_qr(mgsa_handle h, const mgsa_csr* A, const double* Z, int64_t m, int n, int64_t ldz,
                    mgsa_variant v, double* Q, int64_t ldq, double* R, int ldr, mgsa_stream_t s);

/* Time-sliced mgsa_qr: run steps [first, first + count) of the loop (step i
 * forms q_i and row i of R) as one launch, so that other work can run on the
 * GPU between slices.  Calls with first = 0, 1 * count, 2 * count, ... up to n
 * in order, on one stream, give bit for bit the results of one mgsa_qr call
 * on the whole GPU (slices never use a cluster: MGSA_PARAM_CLUSTER = 1).
 * The first slice (first == 0) reads Z; later ones continue from Q, R and the
 * handle's workspace, so between the slices of one QR the handle must run no
 * other QR and its parameters must not change.  A slice after a failed one
 * does nothing; mgsa_get_info reports the failure.  MGS forms only
 * (MGSA_NAIVE / MGSA_HA / MGSA_HP); arguments as for mgsa_qr. */
mgsa_status mgsa_qr_steps(mgsa_handle h, const mgsa_csr* A, const double* Z, int64_t m, int n, int64_t ldz,
                          mgsa_variant v, double* Q, int64_t ldq, double* R, int ldr, int first, int count,
                          mgsa_stream_t s);

/* Wait for stream s and report the outcome of the last mgsa_qr queued on h.
 * *info = 0 on success; otherwise the 1-based column j at which z_j^T x_j was
 * not positive (return MGSA_ERR_BREAKDOWN) or not finite (MGSA_ERR_NONFINITE),
 * or -1 with MGSA_ERR_TIMEOUT.  Columns >= j of Q and R are undefined after a
 * failure. */
mgsa_status mgsa_get_info(mgsa_handle h, mgsa_stream_t s, int* info);

/* Stream-ordered copy of the outcome of the last mgsa_qr queued on h into
 * device memory: info_dev[0] = 0 (success), 2 (breakdown), 3 (non-finite) or
 * 6 (timeout); info_dev[1] = the 1-based column (-1 for a timeout).  Queue it
 * on the same stream right after mgsa_qr to keep the status of that QR when
 * more QRs follow on the handle (mgsa_get_info only sees the latest one).
 * Does not wait. */
mgsa_status mgsa_copy_info(mgsa_handle h, int* info_dev, mgsa_stream_t s);

/* End-to-end call on HOST buffers (pageable or pinned): copies the CSR arrays
 * and Z to device buffers owned by the handle, runs mgsa_qr, copies Q and R
 * back, waits for stream s and returns the outcome as mgsa_get_info would
 * (with *info set).  Same sizes, layout and requirements as mgsa_qr; the
 * host arrays must hold rowptr[m+1], col[nnz], val[nnz], Z[ldz*n],
 * Q[ldq*n], R[ldr*n]. */
mgsa_status mgsa_qr_host(mgsa_handle h, const int32_t* rowptr, const int32_t* col, const double* val,
                         int64_t nnz, const double* Z, int64_t m, int n, int64_t ldz, mgsa_variant v,
                         double* Q, int64_t ldq, double* R, int ldr, mgsa_stream_t s, int* info);

/* Successive orthogonalisation (Section 2: the column-oriented, left-looking
 * MGS suits orthogonalising new columns against ones already orthonormalised).
 * Given k columns Qold (A-orthonormal) and Pold = A Qold (the p_i of the run
 * that produced them), orthonormalise the n columns of Z against them and
 * among themselves in the form `v`:
 *
 *   [Qold Z] = [Qold Q] [ I  R_top ]     R = [ R_top ]   (k + n) x n
 *                       [ 0  R_bot ]         [ R_bot ]
 *
 * with Q^T A Q = I, Qold^T A Q = 0 (in exact arithmetic); R_bot is upper
 * triangular.  The result equals mgsa_qr on [Qold Z] with the first k pivots
 * taken as given (one device-wide step per given column, no MV for it).
 *
 *   Qold, Pold  m x k device arrays, leading dimensions ldqo, ldpo >= m
 *               (read only; may be NULL when k == 0).  The p_i the form uses
 *               are Pold's columns as given (HA / naive / HP alike).
 *   Z, Q, A, s  as for mgsa_qr.
 *   P           m x n output p_j = A q_j of the new columns as the form forms
 *               them (naive: A q_j; HA / HP: the recurrence of eq. (tec1)),
 *               leading dimension ldp >= m; NULL = not returned.  Passing the
 *               (Q, P) of one call as (Qold, Pold) of the next grows a basis.
 *   R           (k + n) x n output, leading dimension ldr >= k + n.
 *
 * Requirements: v one of MGSA_NAIVE / MGSA_HA / MGSA_HP; 0 <= k, 1 <= n,
 * k + n <= MGSA_MAX_N, k + n <= m < 2^31; no output overlaps an input or
 * another output.  Status and info as for
 * mgsa_qr (info counts the columns of Z, 1-based).  mgsa_reserve(h, m, k + n,
 * v) makes the call allocation-free. */
mgsa_status mgsa_qr_append(mgsa_handle h, const mgsa_csr* A, const double* Qold, int64_t ldqo, const double* Pold,
                           int64_t ldpo, int k, const double* Z, int64_t m, int n, int64_t ldz, mgsa_variant v,
                           double* Q, int64_t ldq, double* P, int64_t ldp, double* R, int ldr, mgsa_stream_t s);

/* ---------------------------------------------------------------------- */
/* Batched QR: many independent instances in one call.                      */
/* ---------------------------------------------------------------------- */

/* One instance of a batch.  An array of these lives in DEVICE memory and is
 * read by the kernels (the host never dereferences it).  Every pointer is
 * device memory owned by the caller; A, Z, Q, R, ld* and variant mean what
 * they mean for mgsa_qr (rowptr/col/val form the CSR of the m x m SPD A).
 * work: mgsa_job_workspace_bytes(m, n, variant) bytes used by this job only. */
typedef struct {
  int64_t m;
  int32_t n;
  int32_t variant;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
  const double* Z;
  int64_t ldz;
  double* Q;
  int64_t ldq;
  double* R;
  int64_t ldr;
  double* work;
} mgsa_job;

/* Largest n of a batched job. */
#define MGSA_BATCH_MAX_N 256
/* info value of a job that failed the device-side checks (bad sizes,
 * NULL pointer, unknown variant); its outputs are untouched. */
#define MGSA_BATCH_INFO_INVALID (-2147483647)

/* Device workspace bytes one batched job of (m, n, v) needs (x / p columns):
 * 8 * round_up(m, 32) * (n for HP, 1 for HA, 2 for naive). */
size_t mgsa_job_workspace_bytes(int64_t m, int n, mgsa_variant v);

/* QR of `count` independent instances (Section 1, eq. (1); the same
 * right-looking Algorithms 4, 7, 8 as mgsa_qr) in one call on stream s.
 * Persistent kernels (one per variant) take jobs from a device work queue:
 * each CTA runs a whole instance with CTA-wide barriers, so instances of
 * different sizes run side by side and larger ones should come first in the
 * array for the best load balance.  info_dev[k] (device, count int32) gets 0,
 * the 1-based breakdown column j (z_j^T x_j <= 0), -j (not finite) or
 * MGSA_BATCH_INFO_INVALID.  The call allocates nothing and launches plain
 * kernels (no cooperative launch), so it can be captured into a CUDA graph.
 * Results are deterministic per instance; they may differ in the last bits
 * from mgsa_qr's (different reduction tree).  Returns MGSA_ERR_INVALID for
 * count < 0 or NULL arrays (count > 0); count == 0 does nothing. */
mgsa_status mgsa_qr_batched(mgsa_handle h, int count, const mgsa_job* jobs_dev, int* info_dev, mgsa_stream_t s);

/* ---------------------------------------------------------------------- */
/* Grouped launch: several QRs side by side on disjoint gangs of CTAs.      */
/* ---------------------------------------------------------------------- */

/* One member of a grouped launch: steps [first, first + count) of one QR (a
 * time slice, as for mgsa_qr_steps) on a gang of `ctas` CTAs of its own.
 *
 *   job    A, Z, Q, R, m, n, ld* as for mgsa_qr_batched (device pointers owned
 *          by the caller); job.variant must be the launch's variant.
 *          job.work: the member's workspace, mgsa_group_workspace_bytes(h, m,
 *          n, v) bytes of device memory, 256-byte aligned.  It carries the
 *          QR's state (x / p columns) between slices, with Q and R, so it and
 *          they must stay untouched between the slices of one QR.  Its first
 *          two int32 are the member's outcome once its last slice has run:
 *          status (0, 2 breakdown, 3 not finite, 6 timeout) and the 1-based
 *          column, as mgsa_copy_info reports them.
 *   ctas   CTAs asked for (>= 1); the gang uses at most that many, and fewer
 *          when the slabs would fall below the smallest slab size (128 rows,
 *          or MGSA_PARAM_MIN_ROWS_PER_CTA).  A member's results equal those of
 *          mgsa_qr / mgsa_qr_steps with MGSA_PARAM_MAX_CTAS = ctas and
 *          MGSA_PARAM_CLUSTER = 1 on a handle with the same settings, bit for
 *          bit, whatever else runs in the launch.  Slices of one QR may use
 *          different gang sizes (the last bits then depend on them).
 *   reserved  0. */
typedef struct {
  mgsa_job job;
  int32_t first;
  int32_t count;
  int32_t ctas;
  int32_t reserved;
} mgsa_group_member;

/* Most members of one grouped launch. */
#define MGSA_GROUP_MAX 64

/* Device workspace bytes of one member of a grouped launch on h's device. */
size_t mgsa_group_workspace_bytes(mgsa_handle h, int64_t m, int n, mgsa_variant v);

/* Grouped launch (Section 1, eq. (1); Algorithms 4, 7, 8, right-looking): one
 * cooperative launch runs `count` members (a HOST array, read before the call
 * returns), member k on CTAs of its own, with device-wide barriers that count
 * only its own gang, so QRs of very different sizes share the GPU without
 * waiting for each other.  The gangs' CTAs together may not exceed the number
 * the GPU holds at once (one per SM on GB300).  A slice after a failed slice
 * of the same QR does nothing.  MGS forms only; the CTA sum, sizes and
 * pointers are checked on the host (MGSA_ERR_INVALID).  Queues two launches on
 * s (a reset of the members' barrier words, then the grouped kernel) and
 * returns; allocates nothing. */
mgsa_status mgsa_qr_group(mgsa_handle h, mgsa_variant v, int count, const mgsa_group_member* members,
                          mgsa_stream_t s);

/* Launch parameters (0 restores the default).
 *   MGSA_PARAM_MAX_CTAS          cap on the number of CTAs of a single-instance
 *                                launch (default: one per SM that fits, i.e.
 *                                the co-resident maximum)
 *   MGSA_PARAM_CHUNK_ROWS        rows whose pivot vectors are staged in shared
 *                                memory at once (multiple of 32, <= 4096)
 *   MGSA_PARAM_MIN_ROWS_PER_CTA  smallest row slab given to one CTA (default 128,
 *                                or 32 when A averages >= 32 nonzeros per row)
 *   MGSA_PARAM_BATCH_CTAS        cap on the number of CTAs of mgsa_qr_batched
 *                                launches (default: one per SM).  With
 *                                MAX_CTAS on another handle, the two kinds of
 *                                launch can run side by side on disjoint SMs
 *                                (their CTA counts summing to at most the SM
 *                                count), which a server uses to keep small
 *                                requests from waiting behind large ones.
 *   MGSA_PARAM_ROW_MODE          rows per warp of the MVs and of the block
 *                                product: 0 = one warp per row when A averages
 *                                >= 32 nonzeros per row, else one thread per
 *                                row (default); 1 = one thread per row (32 rows
 *                                per warp); 2 = one warp per row
 *   MGSA_PARAM_CLUSTER           0 = automatic (default): a QR small enough
 *                                (at most 256 rows per CTA of the largest
 *                                cluster the GPU takes, and m * n <= 2^18)
 *                                runs on one thread-block cluster of up to 16
 *                                CTAs with hardware cluster barriers instead
 *                                of the whole GPU; 1 = never;
 *                                2..16 = always, on a cluster of that many CTAs
 *                                (MGSA_ERR_INVALID from mgsa_qr if the GPU
 *                                cannot co-schedule it).  MGS forms only.
 *   MGSA_PARAM_SPMM_PANEL        columns of Z per pass over A in the block
 *                                product X = A Z (HP): 4 or 8 (0 = 8), each
 *                                width a kernel of its own; every column's
 *                                sums are the same for either width
 *   MGSA_PARAM_WAIT_FAULT        failure-detection test hook, 0 (default) or
 *                                1: while set, each whole-GPU MGS launch of
 *                                this handle starts its device-wide barrier
 *                                counter one arrival short, so its first
 *                                device-wide wait never completes.  The wait
 *                                is bounded (4 s): the kernel records
 *                                MGSA_ERR_TIMEOUT, every CTA returns, and
 *                                mgsa_get_info reports it; the context stays
 *                                usable.  No effect on cluster, CGS, batched
 *                                or allocation-free launches.
 * Results stay deterministic for a fixed setting; different MAX_CTAS,
 * CHUNK_ROWS, MIN_ROWS_PER_CTA, ROW_MODE or CLUSTER settings change the reduction
 * tree and therefore the last bits of Q and R (BATCH_CTAS and SPMM_PANEL do
 * not).  The settings of a handle apply to its mgsa_qr, mgsa_qr_append and
 * (ROW_MODE, SPMM_PANEL, BATCH_CTAS) mgsa_qr_batched calls.  Returns MGSA_ERR_INVALID for an unknown parameter or an
 * out-of-range value. */
typedef enum {
  MGSA_PARAM_MAX_CTAS = 0,
  MGSA_PARAM_CHUNK_ROWS = 1,
  MGSA_PARAM_MIN_ROWS_PER_CTA = 2,
  MGSA_PARAM_BATCH_CTAS = 3,
  MGSA_PARAM_ROW_MODE = 4,
  MGSA_PARAM_SPMM_PANEL = 5,
  MGSA_PARAM_CLUSTER = 6,
  MGSA_PARAM_WAIT_FAULT = 7
} mgsa_param;
mgsa_status mgsa_set_param(mgsa_handle h, mgsa_param p, int64_t value);

/* Allocation-free QR.  The paper has no counterpart to this entry point; it
 * exists for callers that must not allocate device memory themselves: code
 * running under a memory manager that owns the whole device (a framework's
 * caching allocator, a server that admits work against a fixed memory
 * budget) and may not allocate behind its back, and latency-critical loops
 * where cudaMalloc / cudaFree would add device-wide synchronisation.  It
 * computes what mgsa_qr computes, with the same kernel, but needs no handle
 * and allocates nothing: its scratch (the x / p columns, the per-CTA
 * partial sums and the status / barrier words) lives in one static device
 * array of MGSA_NOALLOC_SCRATCH_BYTES bytes compiled into the library, which
 * every GPU that loads the library holds until the process exits.
 *
 *   A, Z, Q, R, m, n, ldz, ldq, ldr, v   as for mgsa_qr.
 *   info_dev  NULL, or device memory for two int32 written after the QR:
 *             info_dev[0] = 0 (success), 2 (z_j^T x_j <= 0), 3 (not finite)
 *             or 6 (a device-wide wait timed out); info_dev[1] = the 1-based
 *             column j of the failure (-1 for a timeout).
 *   s         stream; the call returns without waiting.
 *
 * Runs on the current CUDA device; every pointer must be on that device.
 * The first call on a device sets that device up (looks up the address of
 * the static array and sets the kernel's shared-memory limit); make that
 * first call before any stream capture.  That set-up belongs to the CUDA
 * context: each call checks the id of the current context, and the first
 * call in a new context on the device -- after cudaDeviceReset, for example --
 * repeats it, so it too should come before any stream capture.  Problems whose scratch does not fit
 * (about 8*(m*c + (2n+1)*G) bytes with c = n for HP, 1 for HA, 2 for naive and
 * G <= the number of SMs) are rejected with MGSA_ERR_INVALID and a message
 * in mgsa_last_error; nothing is launched then.  Every call uses the same
 * array and leaves its contents behind (the status and barrier words are
 * cleared at the start of each call), so calls whose work overlaps on the
 * GPU -- on different streams, or from different threads -- race and give
 * undefined results; order them on one stream. */
#define MGSA_NOALLOC_SCRATCH_BYTES (32u << 20)
mgsa_status mgsa_qr_noalloc(const mgsa_csr* A, const double* Z, int64_t m, int n, int64_t ldz, mgsa_variant v,
                            double* Q, int64_t ldq, double* R, int ldr, int* info_dev, mgsa_stream_t s);

/* ---------------------------------------------------------------------- */
/* Measurement.                                                             */
/* ---------------------------------------------------------------------- */

/* The FP64 fused multiply-add rate of device `device`, measured: a kernel in
 * which every thread runs 8 independent FMA chains for `iters` iterations on
 * 4 CTAs of 256 threads per SM, timed (after one untimed launch) with CUDA
 * events on a stream of its own.  *tflops = 2 * FMAs / time in TFLOP/s, *ms the
 * timed launch's duration.  The paper has no counterpart: this is the
 * ceiling against which the FP64-bound sweep kernels are measured.  It
 * allocates a small output buffer, synchronises the device's new stream and
 * restores the current device.  MGSA_ERR_INVALID for NULL outputs, iters < 1
 * or a bad device; MGSA_ERR_CUDA if a CUDA call fails. */
mgsa_status mgsa_fp64_probe(int device, int iters, double* tflops, double* ms);

/* Short static description of the most recent failure on this thread
 * (never NULL). */
const char* mgsa_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MGSA_H */
