/*
 * eeid -- squared eigenvector components of real symmetric FP64 matrices through
 * the eigenvector-eigenvalue identity, on one NVIDIA GB300 (sm_103a) GPU.
 *
 * The operation (Sec. 2, Eq. 1 of "Eigenvector Component Calculation Speedup over
 * NumPy for High-Performance Computing", arXiv 2002.04989): for a real symmetric
 * n x n matrix A with eigenvalues lam_1(A) <= ... <= lam_n(A) and unit eigenvectors
 * v_i, and M_j the (n-1) x (n-1) minor of A with row and column j removed,
 *
 *     |v_ij|^2 * prod_{k != i} (lam_i(A) - lam_k(A)) = prod_{k=1}^{n-1} (lam_i(A) - lam_k(M_j)).
 *
 * The paper's functions take (matrix, i, j) and return one component (Algorithms
 * 0 and 1, Sec. 3); this library takes whole sets of eigen-indices i ("rows") and
 * component indices j ("cols") and returns the grid.  Where the printed
 * algorithms and Eq. 1 disagree (which index is removed for the minor, which
 * product is the numerator), Eq. 1 is followed.
 *
 * Conventions for every entry point:
 *  - Indices are 0-based.  Eigen-index i = k means the (k+1)-th smallest
 *    eigenvalue; eigenvalue outputs are ascending.
 *  - Matrices are row-major FP64 with leading dimension lda >= n (in elements).
 *    Only the lower triangle (element (r, c), r >= c, at A[r*lda + c]) is read; the
 *    caller guarantees symmetry.  Entries must be finite.
 *  - "d_" pointers are device memory of the context's device; "h_" pointers are
 *    host memory.  The caller owns every buffer it passes; the library never
 *    frees or retains them beyond the call (asynchronous calls read/write them
 *    until the stream reaches that point).
 *  - Calls that take a stream (a cudaStream_t passed as void*; NULL = the legacy
 *    default stream) are asynchronous: they validate arguments and enqueue work,
 *    and return EEID_OK once enqueued.  Warnings and device-side errors found
 *    while the work runs are returned by the next eeid_sync() on that context.
 *  - A context's workspace is shared by its calls: issue the calls of one
 *    context on one stream (or order them yourself).  Contexts are not
 *    thread-safe; use one per host thread.
 *  - Deferred status is kept per stream: eeid_sync(ctx, s) returns and clears
 *    only what the context's calls on stream s raised (63 streams per context
 *    have a word of their own; further streams share one).
 *  - Status codes: negative = error (nothing, or only part, was enqueued),
 *    positive = warning (results written).  eeid_last_error() gives a message.
 */
#ifndef EEID_H
#define EEID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EEID_OK = 0,
  /* Two eigenvalues of A are exactly equal: Eq. 1 is 0/0 for those i.  The rows
   * of the affected eigen-indices are filled with NaN. */
  EEID_WARN_DEGENERATE = 1,
  /* The spectrum's minimum relative gap min_k (lam_{k+1}-lam_k)/max|lam| is below
   * 1e-4: results are computed but lie outside the accuracy contract. */
  EEID_WARN_SMALL_GAP = 2,
  EEID_ERR_INVALID = -1,   /* bad argument (NULL pointer, size, index, duplicate) */
  EEID_ERR_NOMEM = -2,     /* workspace would exceed the context's HBM budget */
  EEID_ERR_CUDA = -3,      /* a CUDA call failed (message in eeid_last_error) */
  EEID_ERR_TIMEOUT = -4,   /* a bounded wait ran out */
  EEID_ERR_BUSY = -5,      /* serving: admission refused (non-blocking submit) */
  EEID_ERR_NOT_FOUND = -6, /* serving: unknown ticket */
  EEID_ERR_CANCELLED = -7  /* serving: request cancelled before it ran */
} eeid_status;

typedef struct eeid_ctx eeid_ctx;

/* Create a context on CUDA device `device`.  `hbm_budget_bytes` caps the device
 * workspace the context may allocate (0 = half of the device's free memory at
 * creation).  *out receives the context.  Errors: EEID_ERR_INVALID (out NULL,
 * bad device), EEID_ERR_CUDA (no usable GPU). */
eeid_status eeid_ctx_create(int device, size_t hbm_budget_bytes, eeid_ctx** out);

/* Free the context and its workspace (waits for its outstanding work). NULL ok. */
void eeid_ctx_destroy(eeid_ctx* ctx);

/* Message for the last error or warning raised on the calling host thread. */
const char* eeid_last_error(void);

/* Return the worst deferred status of the context's calls on `stream` since the
 * previous eeid_sync on that stream (errors before warnings) and clear it.  The status
 * word is read and cleared on `stream` itself, after the calls, and the call then waits
 * for the stream; other streams' warnings are left for their own eeid_sync. */
eeid_status eeid_sync(eeid_ctx* ctx, void* stream);

/* Eigenvalues lam_1(A) <= ... <= lam_n(A) of A (Sec. 2: the first input of Eq. 1).
 * d_lambda: device, n doubles, written ascending.  n == 0 is a no-op. */
eeid_status eeid_eigvals(eeid_ctx* ctx, const double* dA, int64_t lda, int64_t n,
                         double* d_lambda, void* stream);

/* Eigenvalues of the minors M_j (A with row and column j removed; Sec. 2, the
 * second input of Eq. 1) for j = h_cols[c], c < ncols.  d_mu: device,
 * ncols x (n-1) doubles row-major, row c ascending.  h_cols: host, distinct
 * indices in [0, n).  ncols == 0 or n <= 1 is a no-op. */
eeid_status eeid_minor_eigvals(eeid_ctx* ctx, const double* dA, int64_t lda, int64_t n,
                               const int64_t* h_cols, int64_t ncols, double* d_mu,
                               void* stream);

/* Eq. 1 for the grid i = h_rows[r] (r < nrows), j = h_cols[c] (c < ncols):
 * d_out[r*ncols + c] = |v_ij|^2 (device, nrows x ncols doubles).
 * h_rows / h_cols: host, distinct indices in [0, n); NULL means "all" (then
 * nrows / ncols must equal n).  d_lambda_opt: optional device buffer of n doubles
 * that receives the eigenvalues of A.  n == 1 gives |v|^2 = 1; nrows == 0 or
 * ncols == 0 is a no-op.  Deferred warnings: EEID_WARN_DEGENERATE,
 * EEID_WARN_SMALL_GAP (see eeid_sync). */
eeid_status eeid_components(eeid_ctx* ctx, const double* dA, int64_t lda, int64_t n,
                            const int64_t* h_rows, int64_t nrows, const int64_t* h_cols,
                            int64_t ncols, double* d_out, double* d_lambda_opt, void* stream);

/* eeid_components on HOST buffers: copies hA (host, n x lda doubles, pinned or
 * pageable) into a device buffer the context keeps between calls (it is allocated
 * only when a call needs more than the last), runs the path on `stream`, copies
 * the nrows x ncols grid back into h_out (and the eigenvalues into h_lambda_opt),
 * and synchronises the stream.  Returns the call's final status (warnings
 * included).  Same index conventions as eeid_components. */
eeid_status eeid_components_host(eeid_ctx* ctx, const double* hA, int64_t lda, int64_t n,
                                 const int64_t* h_rows, int64_t nrows, const int64_t* h_cols,
                                 int64_t ncols, double* h_out, double* h_lambda_opt,
                                 void* stream);

/* Signed unit eigenvectors v_i for the eigen-indices i = h_rows[r] (r < nrows), every
 * component j: d_vec[r*n + j] = v_ij (device, nrows x n doubles).  Eq. 1 fixes only
 * |v_ij|; the signs come from applying it in a second basis (Sec. 2: the identity on
 * other bases gives the direction).  For a reference component r of v_i, rotating
 * coordinates r and j by 45 degrees and removing u = (e_r + e_j)/sqrt2 gives a minor
 * whose Eq. 1 value is q_ij = (v_ir + v_ij)^2 / 2; then
 *     v_ij = (q_ij - (|v_ir|^2 + |v_ij|^2) / 2) / |v_ir|   (v_ir > 0).
 * References are chosen on the device by a greedy cover with |v_ir| >= max_j |v_ij| / 4,
 * so the error of v_ij is about 2 delta / |v_ir| <= 8 sqrt(n) delta, delta being the
 * error of |v_ij|^2.  Each reference costs one rotated minor per component j whose
 * |v_ij|^2 is not exactly 0 for some row sharing it (at most n - 1 reductions); such
 * exactly-zero components are returned as 0.  A few eigenvectors often share one
 * reference, and a whole eigenbasis of a random matrix needs about ten.  Strongly
 * localised eigenvectors (nearly decoupled blocks) may each need their own reference,
 * up to n of them, so the cost grows toward n^2 reductions there.
 * Sign convention: the component of largest |v_ij|^2 (the first on exact ties) is
 * positive.  Rows of eigenvalues that are exactly degenerate are NaN.
 * h_rows: host, distinct indices in [0, n), NULL = all (nrows = n).  d_lambda_opt:
 * optional device buffer of n doubles for the eigenvalues of A.  The call runs on
 * `stream` and synchronises it once, midway, to read the chosen references back; it
 * returns with the last phase enqueued.  Deferred warnings as for eeid_components. */
eeid_status eeid_eigenvectors(eeid_ctx* ctx, const double* dA, int64_t lda, int64_t n,
                              const int64_t* h_rows, int64_t nrows, double* d_vec,
                              double* d_lambda_opt, void* stream);

/* Eq. 1 for a complex Hermitian A (Sec. 2 states the identity for Hermitian matrices):
 * d_out[r*ncols + c] = |v_ij|^2 for i = h_rows[r], j = h_cols[c], as eeid_components.
 * dA: device, row-major, interleaved (re, im) doubles, leading dimension lda >= n in
 * complex elements (16 bytes each); only the lower triangle is read, and the imaginary
 * parts of the diagonal are ignored (a Hermitian diagonal is real).  A and its minors are
 * reduced by unitary Householder reflections to real symmetric tridiagonals; bisection and
 * the identity are those of the real path.  n <= 2048 (the complex reduction keeps three
 * vectors of 16-byte entries in shared memory); larger n gives EEID_ERR_INVALID.
 * d_lambda_opt: optional device buffer of n doubles for the eigenvalues of A.  Same index
 * conventions, no-op cases and deferred warnings as eeid_components. */
eeid_status eeid_components_herm(eeid_ctx* ctx, const double* dA, int64_t lda, int64_t n,
                                 const int64_t* h_rows, int64_t nrows, const int64_t* h_cols,
                                 int64_t ncols, double* d_out, double* d_lambda_opt,
                                 void* stream);

/* One problem of a batch: the arguments of eeid_components.  h_rows / h_cols NULL
 * mean "all" (nrows / ncols = n). */
typedef struct {
  const double* dA;
  int64_t lda;
  int64_t n;
  const int64_t* h_rows;
  int64_t nrows;
  const int64_t* h_cols;
  int64_t ncols;
  double* d_out;      /* nrows x ncols */
  double* d_lambda;   /* optional, n */
} eeid_problem;

/* Eq. 1 for many matrices of uneven size in one pass: all tridiagonalisations,
 * bisections and identity evaluations of every problem are merged into
 * cost-sorted task lists run by persistent kernels, captured once per batch
 * shape into a CUDA graph.  Results are bitwise identical to calling
 * eeid_components on each problem alone.  probs: host array of `count`. */
eeid_status eeid_components_batched(eeid_ctx* ctx, const eeid_problem* probs, int64_t count,
                                    void* stream);

/* Enable (default) or disable CUDA-graph capture and replay for
 * eeid_components_batched.  With graphs off every batched call plans and launches
 * directly (better when batch shapes never repeat, as in serving). */
eeid_status eeid_set_graphs(eeid_ctx* ctx, int enable);

/* Enable (default) or disable the round plan of large calls.  When one call's
 * Householder reductions (A and its minors, Sec. 2) are near-equal in size and take
 * more than one round of the persistent grid, whole rounds may run as two 8-warp CTAs
 * per SM (hybrid rounds, when the size allows two per SM), and the last, partial
 * round is launched on an internal greatest-priority stream.  Meanwhile the caller's
 * stream bisects the eigenvalues of A and of the minors already reduced, on the SMs
 * that round leaves idle.  The two streams join before the last minors' bisection,
 * so the call still completes in the caller's stream order.  Results are bitwise the
 * same either way; with the plan on, the phase times of eeid_phase_times may
 * overlap. */
eeid_status eeid_set_overlap(eeid_ctx* ctx, int enable);

/* Latency mode: the cluster and group plans (both on by default).  When a call has few
 * Householder reductions (at most half as many as the device has SMs: one or a few
 * components, a few columns, or the eigenvalues of one large A -- the single-component
 * tasks of the paper's Table 1) of matrices with m >= 384, each reduction runs on a
 * thread-block cluster of up to 16 CTAs on as many SMs instead of on one CTA: the tiles
 * of every column step are split over the cluster, partial sums stay in the matrix's
 * workspace slot and the step vectors are exchanged through distributed shared memory.
 * When there are so few reductions of m >= 1536 that G = SMs / reductions exceeds 16
 * (one component of a large A: two reductions), the group plan runs each on G CTAs
 * launched cooperatively (all resident at once), which exchange the step vectors through
 * global memory and meet at bounded global-memory barriers.  A barrier that waits beyond
 * its limit (one second; only if the CTAs were not resident together) makes the group
 * stop, leaving its output incomplete, and eeid_sync return EEID_ERR_TIMEOUT.
 * mode 0 = both off; 1 = the cluster plan only; 2 (default) = both.  Results are bitwise
 * the same in every mode. */
eeid_status eeid_set_clusters(eeid_ctx* ctx, int mode);

/* Self-test of the bounded barrier wait of the group plan (see eeid_set_clusters): runs
 * the group variant of K-a on a 2 x 2 matrix as a group of two CTAs of which only one is
 * launched, so the group's first barrier never fills.  The launched CTA gives up after
 * the wait limit (one second of the GPU's global timer) and sets the timeout bit of
 * `stream`'s status word; the call returns once the stream is idle, and the next
 * eeid_sync(ctx, stream) returns EEID_ERR_TIMEOUT.  The context stays usable.  Takes a
 * little over a second. */
eeid_status eeid_check_barrier_timeout(eeid_ctx* ctx, void* stream);

/* Number of kernel launches the context has enqueued so far (for accounting). */
int64_t eeid_launch_count(const eeid_ctx* ctx);

/* Number of reference components the context's last eeid_eigenvectors call chose
 * (each costs n - 1 rotated-minor reductions); 0 before any such call. */
int64_t eeid_vector_refs(const eeid_ctx* ctx);

/* Tuning of the Householder kernel (K-a): matrices of size m in [m_lo, m_hi] are
 * reduced by the variant `path` (0 = working matrix resident in shared memory,
 * m <= 160; 1 = working matrix in a global-memory slot per CTA; 2 = the global-slot
 * variant built for high occupancy, at most 80 registers a thread so that three 8-warp
 * or six 4-warp CTAs share an SM) with `warps` warps per CTA (path 0: 1, 2, 4, 8;
 * path 1: 1, 2, 4, 8, 12, 16, where 1 and 2 are built for 16 and 8 CTAs per SM; path
 * 2: 4, 8).  Paths 1 and 2 run the same arithmetic.  Later rules take precedence.  A
 * call whose group of such matrices is too small to fill the SMs with a 1- or 2-warp
 * choice runs them with 4 warps instead (same results).
 * The warp count never changes a result: every instantiation of one path sums in
 * the same order, so the two paths' results are each bitwise fixed by m.  Changing
 * the path of a size changes the rounding order (not the accuracy class).  A rule
 * covering a size also keeps calls from switching it to the 8-warp two-CTAs-per-SM
 * rounds that are otherwise used for large near-equal groups (see eeid_set_overlap).
 * EEID_ERR_INVALID for an unsupported combination. */
eeid_status eeid_tune_tridiag(eeid_ctx* ctx, int m_lo, int m_hi, int path, int warps);

/* Drop all tuning rules (back to the built-in size table). */
eeid_status eeid_tune_reset(eeid_ctx* ctx);

/* Autotuner for the Householder kernel.  For size buckets up to min(max_m, 1024)
 * it times every supported variant (shared-memory or global-slot working matrix,
 * 1-16 warps per CTA, both builds of the global slot) on this device, on a wave of
 * synthetic minors whose sizes cover the bucket, largest first (as in a batch), keeps
 * the fastest per bucket, and installs the choices as tuning rules (larger sizes keep
 * the built-in choice).  With `cache_path` non-NULL the table is read
 * from that file when it exists and was made on the same device model, and
 * written there after tuning.  Runs synchronously on an internal stream; takes a
 * few seconds.  Errors: EEID_ERR_CUDA, EEID_ERR_NOMEM (workspace budget). */
eeid_status eeid_autotune(eeid_ctx* ctx, int max_m, const char* cache_path);

/* Phases of one call, in launch order, for eeid_phase_times. */
enum {
  EEID_PHASE_TRIDIAG = 0,       /* Householder reduction of A and of the minors */
  EEID_PHASE_BISECT_A = 1,      /* eigenvalues of A */
  EEID_PHASE_DENOMINATORS = 2,  /* prod_{k != i} (lam_i - lam_k), once per i */
  EEID_PHASE_BISECT_MINORS = 3, /* eigenvalues of the minors */
  EEID_PHASE_IDENTITY = 4,      /* Eq. 1 for the requested grid */
  EEID_NUM_PHASES = 5
};

/* Enable (1) or disable (0) per-phase device timing: each later call records CUDA
 * events on its stream around its phases (a small cost per launch). */
eeid_status eeid_set_timing(eeid_ctx* ctx, int enable);

/* Wait for the last timed call's events and write its per-phase device durations
 * in milliseconds into ms[0 .. min(cap, EEID_NUM_PHASES)) (0 for phases that call
 * did not run).  A phase's duration runs from the start of its first launch to the
 * end of its last; under the tail overlap (eeid_set_overlap) the reduction's
 * interval contains part of the bisection phases.  Returns the number of values
 * written, or a negative status. */
int eeid_phase_times(eeid_ctx* ctx, double* ms, int cap);

/* ------------------------------------------------------------------ serving
 * A request loop with continuous batching.  Callers on any thread submit a host
 * matrix and the components they want; a scheduler thread admits requests in
 * arrival order while the device budget allows, merges waiting requests of similar
 * cost (within a factor of 8 of n^3 (columns + 1)) into one batched launch (the work
 * of eeid_components_batched), and keeps up to `max_inflight` batches on the GPU at
 * once, each on its own stream and workspace, so requests arriving while a batch
 * runs start as soon as a slot and memory free up.  Each batch's reductions are
 * launched one round of the grid at a time, so a large request holds up a small one
 * by about one round, not its whole run.  A request's matrix, output and eigenvalues stay
 * resident on the device until its results are copied back.  Each result is
 * bitwise the same as eeid_components on that matrix alone.  (The paper serves one
 * component per call; this request loop is the library's own serving form of Eq. 1.) */
typedef struct eeid_server eeid_server;

typedef struct {
  size_t hbm_budget_bytes; /* device memory for the server (0 = half of free): half for
                              resident requests, half split over the batch workspaces */
  int max_batch;           /* most requests merged into one batch (0 = 64) */
  int max_inflight;        /* batches on the GPU at once (0 = 2) */
  int max_pending;         /* waiting requests before submit blocks / returns BUSY (0 = 4096) */
} eeid_server_opts;

typedef struct {
  double queue_ms;          /* submit -> batch launch */
  double total_ms;          /* submit -> results in the caller's buffers */
  int64_t batch_id;         /* batch that served the request (-1 if none) */
  int64_t batch_requests;   /* requests in that batch */
} eeid_req_stats;

typedef struct {
  int64_t pending;                 /* requests waiting for admission */
  int64_t inflight_batches;        /* batches on the GPU now */
  int64_t batches_launched;        /* since creation */
  int64_t max_overlapping_batches; /* most batches seen on the GPU at once */
  int64_t device_bytes_in_use;     /* resident request memory */
  int64_t device_budget_bytes;
} eeid_server_info_t;

/* Start a server on `device` (opts may be NULL for defaults).  The whole device
 * budget is taken here, not on demand: each batch workspace is allocated in full and
 * the request half warms a stream-ordered pool of the server's own.  A 1 GiB pinned
 * host pool for request staging is allocated too.  Nothing then allocates while batches
 * run, since an allocation would serialise the two batches' streams.  Errors:
 * EEID_ERR_INVALID, EEID_ERR_CUDA, EEID_ERR_NOMEM (the budget cannot be allocated). */
eeid_status eeid_server_create(int device, const eeid_server_opts* opts, eeid_server** out);

/* Stop: cancels requests not yet admitted, waits for the batches on the GPU, frees
 * everything (including results nobody waited for).  No other call on the server
 * may be in progress. */
void eeid_server_destroy(eeid_server* srv);

/* Submit |v_ij|^2 for all i and j in h_cols (NULL = all j, ncols = n) of the host
 * matrix hA (row-major, lda >= n, lower triangle read; copied at submit, so hA may be
 * reused at once).  Results will be written to h_out (n x ncols, row-major) and, if
 * non-NULL, the eigenvalues to h_lambda_opt (n); both must stay valid until
 * eeid_server_wait returns for the ticket.  With the queue full, nonblocking != 0
 * returns EEID_ERR_BUSY, otherwise the call waits for room.  A request larger than
 * the device budget returns EEID_ERR_NOMEM.  *ticket identifies the request. */
eeid_status eeid_server_submit(eeid_server* srv, const double* hA, int64_t lda, int64_t n,
                               const int64_t* h_cols, int64_t ncols, double* h_out,
                               double* h_lambda_opt, int nonblocking, uint64_t* ticket);

/* Wait up to timeout_ms (< 0: forever) for a request; on completion fills stats
 * (may be NULL), releases the ticket and returns the request's status (warnings
 * included; warnings are those of its whole batch).  EEID_ERR_TIMEOUT leaves the
 * request in place; EEID_ERR_CANCELLED if it was cancelled; EEID_ERR_NOT_FOUND for
 * an unknown or already-waited ticket. */
eeid_status eeid_server_wait(eeid_server* srv, uint64_t ticket, int64_t timeout_ms,
                             eeid_req_stats* stats);

/* Cancel a request that has not been admitted yet (EEID_ERR_BUSY once it runs).
 * Its wait then returns EEID_ERR_CANCELLED. */
eeid_status eeid_server_cancel(eeid_server* srv, uint64_t ticket);

/* Counters of the serving loop. */
eeid_status eeid_server_info(eeid_server* srv, eeid_server_info_t* info);

/* Bits of a device-side status word (OR-ed by the kernels while they run).  The context
 * calls report them through eeid_sync; eeid_eigvals_noalloc writes them to a word the
 * caller supplies. */
enum {
  EEID_DEV_DEGENERATE = 1u,       /* two eigenvalues of A exactly equal (Eq. 1 is 0/0) */
  EEID_DEV_SMALL_GAP = 2u,        /* minimum relative gap below 1e-4 */
  EEID_DEV_BRACKET_FALLBACK = 4u, /* a bisection bracket failed its check and restarted from
                                     the Gershgorin bracket (information only: the result
                                     is still correct) */
  EEID_DEV_BAD_TASK = 8u,         /* a kernel met a matrix beyond its size limit and skipped
                                     it: the output for that matrix was not written */
  EEID_DEV_TIMEOUT = 16u          /* a cooperative reduction's barrier wait ran out (group
                                     plan only): its group stopped, its output is invalid */
};

/* Eigenvalues of A, like eeid_eigvals, for callers that cannot allocate device
 * memory: for example code embedded in an application whose own memory pool owns
 * the whole device, or code on a latency-critical path where the implicit device
 * synchronisation of cudaMalloc/cudaFree is not acceptable.  It needs no context
 * and calls no cudaMalloc, cudaFree or other allocating routine.  (The paper has no
 * counterpart: this is an interface for such callers.)
 *
 * Scratch: one fixed file-scope device array of about 2.2 MB, present on every
 * GPU that loads the library for the life of the process, sized for n <= 512;
 * n > 512 returns EEID_ERR_INVALID with a message in eeid_last_error().  Every
 * call on a device uses the same array, so calls that overlap on the GPU (for
 * example on two streams without ordering) race and must be avoided; calls on one
 * stream are ordered and safe.
 *
 * First call on each device: it looks the array's address up (with that device
 * current) and caches it, and it loads the library's kernels and raises their
 * shared-memory limits.  Loading a module and changing a kernel attribute may wait
 * for work already queued on the device, so make that first call before any stream
 * capture and outside latency-critical sections; later calls do none of this.
 *
 * dA: device, row-major, lower triangle read, lda >= n.  d_lambda: device, n
 * doubles, ascending.  d_status_opt: optional device word (NULL = not reported).
 * The call sets it to 0 on `stream` before its kernels run; they OR in EEID_DEV_*
 * bits, which the caller reads once the stream has reached the end of the call.
 * EEID_DEV_BAD_TASK there means d_lambda was not written.  Without the word,
 * device-side conditions go unreported.  Asynchronous on `stream` (the calling
 * thread's current device); n == 0 is a no-op (d_status_opt untouched).  Results
 * agree with eeid_eigvals within the library's eigenvalue tolerance
 * (1e-12 * ||A||_2). */
eeid_status eeid_eigvals_noalloc(const double* dA, int64_t lda, int64_t n, double* d_lambda,
                                 unsigned* d_status_opt, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* EEID_H */
