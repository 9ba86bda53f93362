/*
 * idsketch.h -- C ABI of the pass-efficient interpolative decomposition (ID)
 * for one NVIDIA GB300 (sm_103a).
 *
 * Method: Dunton, Jofre, Iaccarino, Doostan, "Pass-efficient methods for
 * compression of high-dimensional turbulent flow data" (arXiv:1905.13257).
 *
 * Orientation.  The paper's data matrix has one time snapshot per ROW and is
 * compressed by a row ID  A ~ P A(I,:)  (Sec. 2.4, eq. eqn:id).  This library
 * stores one snapshot per COLUMN: A is m x n with m = grid points x velocity
 * components and n = snapshots, i.e. the paper's A transposed, and computes
 * the column ID  A ~ A(:,J) P,  P (k x n), P(:,J) = I.  J is the paper's I and
 * P is the paper's P transposed (Remark 2.1: row and column IDs are the same
 * construction on A^T).
 *
 * Conventions for every call
 *   - A and its column chunks are column-major: entry (i, j) at ptr[i + j*ld],
 *     ld >= m, element type given by id_config.dtype.  They live in device
 *     memory and stay owned by the caller.
 *   - J holds 0-based column indices in pivot order (int32).
 *   - P is row-major k x n FP64: entry (t, j) at P[t*n + j].
 *   - Outputs J and P may be device or host pointers (copied with
 *     cudaMemcpyDefault).  id_factor, id_coarse_factor and
 *     id_reconstruct_error synchronise the stream before returning (they
 *     read the pivot count or the error scalars on the host).
 *   - All GPU work is enqueued on the CUDA stream given to id_sketch_create.
 *   - Every call returns an id_status.  An argument error (ID_ERR_INVALID_ARG)
 *     or a call out of order (ID_ERR_STATE) changes nothing.  After
 *     ID_ERR_CUDA the handle is poisoned: every later call but
 *     id_sketch_destroy returns ID_ERR_CUDA.
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef IDSKETCH_H
#define IDSKETCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ID_OK = 0,
  ID_ERR_INVALID_ARG = 1,   /* bad pointer, size, stride or config field      */
  ID_ERR_STATE = 2,         /* call out of order (e.g. factor before columns) */
  ID_ERR_OOM = 3,           /* device allocation failed                      */
  ID_ERR_CUDA = 4,          /* a CUDA runtime call or kernel failed          */
  ID_ERR_RANK_DEFICIENT = 5,/* fewer than k pivots above the rank tolerance  */
  ID_ERR_TIMEOUT = 6,       /* a bounded device wait gave up                 */
  ID_ERR_UNSUPPORTED = 7    /* valid request this build does not implement   */
} id_status;

typedef enum { ID_F32 = 0, ID_F64 = 1 } id_dtype;

/* Arithmetic of the sketch products W = Psi A and Y = A Omega.
 *   ID_SKETCH_EXACT:   FP32-accurate (FP32 data) or FP64 (FP64 data) products.
 *   ID_SKETCH_BF16:    A rounded to bfloat16 once, FP32 accumulation.
 *   ID_SKETCH_FP8E4M3: FP32 data only, tensor-core path only.  Each column c
 *                      of a window is scaled by the power of two 2^e_c that
 *                      brings its largest magnitude closest to 448 without
 *                      passing it (e_c in [-100, 100], 0 for a zero column;
 *                      a scale pass reads the window once more), its entries
 *                      are rounded to FP8-E4M3 (nearest, ties to even), and
 *                      the products of the dequantised values with Psi and
 *                      Omega are accumulated in FP32 (the E4M3 values enter
 *                      the tensor cores exactly as bfloat16).
 * The pivoted QR and the solve for P are FP64 in every mode; A_c keeps the
 * data's own values. */
typedef enum { ID_SKETCH_EXACT = 0, ID_SKETCH_BF16 = 1, ID_SKETCH_FP8E4M3 = 2 } id_sketch_prec;

/* Rank tolerance of the pivoted QR: pivoting stops when every residual
 * column norm is <= ID_RANK_TOL_FACTOR * DBL_EPSILON * ||B||_F, B being the
 * matrix factored (the paper's pseudo-inverse R11^+ of Algorithm 3 step 4 is
 * then the inverse of the k_out x k_out non-singular R11). */
#define ID_RANK_TOL_FACTOR 64.0

typedef struct {
  int64_t m;               /* rows of A = ncomp * nx * ny * nz (or any m > 0)  */
  int64_t n_max;           /* column capacity: total columns streamed <= n_max */
  int32_t k;               /* target rank, 1 <= k <= l                          */
  int32_t l;               /* sketch width l = k + p, l <= 64; up to 96 for FP32
                              data without Y (see id_sketch_create)             */
  uint64_t seed;           /* seed of Psi and Omega (Philox4x32-10 key)         */
  int32_t dtype;           /* id_dtype of the streamed columns                  */
  int32_t prec;            /* id_sketch_prec                                    */
  int32_t grid[3];         /* nx, ny, nz; needed only for the coarse grid       */
  int32_t ncomp;           /* velocity components; grid/ncomp unused if 0       */
  int32_t coarse_stride[3];/* sx, sy, sz of the coarse grid (direct injection)  */
  int32_t want_Y;          /* 1: also form Y = A Omega (m x l)                  */
  int32_t want_coarse;     /* 1: copy A_c = A(rows_c, :) window by window        */
  int32_t window_cols;     /* columns aggregated per launch; 0 = process every
                              id_sketch_stream_columns call at once (no borrow) */
  int32_t reserved[4];     /* must be zero                                      */
} id_config;

typedef struct id_sketch id_sketch;   /* opaque, library-owned */

/* Create a sketch state on the current device for one stream of snapshots.
 * Draws Omega (n_max x l) from the counter generator, allocates W (l x n_max,
 * FP64), Y (m x l, dtype) and A_c (m_c x n_max, dtype) as requested.
 * Passage: Algorithm 4 steps 2-3 (Gaussian Omega, l = k + p; Sec. 2.2).
 * cuda_stream may be NULL (legacy default stream).
 * Sketch width: l <= 64 for every form.  FP32 data without Y may take
 * 64 < l <= 96 (k up to 86 at p = 10): the tensor-core sketch then forms W
 * in one pass with 96-wide accumulators when the window is one buffer with
 * 16-byte aligned columns, else in passes of 60 rows of Psi (one more read
 * of the window per pass); the pivoted QR and the solve take the wider W,
 * and the coarse-grid QR, the error pass and the single-pass ID keep
 * k <= 64.
 * Errors: ID_ERR_INVALID_ARG for an inconsistent config (m <= 0, n_max <= 0,
 * k < 1, k > l, l > 96, grid/ncomp not matching m when want_coarse, a coarse
 * stride < 1, reserved fields != 0), ID_ERR_UNSUPPORTED (l > 64 with FP64
 * data or want_Y; k > 64 with want_coarse; at id_sketch_stream_columns, l > 64
 * with columns that the tensor-core sketch cannot read: m < 128 or columns
 * not 16-byte aligned), ID_ERR_OOM, ID_ERR_CUDA. */
id_status id_sketch_create(const id_config* cfg, void* cuda_stream, id_sketch** out);

/* Stream ncols snapshot columns (device pointer, column-major, leading
 * dimension ld >= m) into the sketch: W(:, cols) = Psi A(:, cols) and
 * Y += A(:, cols) Omega(cols, :) in ONE read of the columns; the coarse rows
 * A_c(:, cols) are copied in the same window when want_coarse (FP32 data:
 * by a second kernel right after the window's sketch, which reads only the
 * row blocks holding coarse rows).
 * Passage: Sec. 2.1 (snapshots arrive one at a time, the count is not known
 * in advance) and Algorithm 4 step 3 / eq. eq:sampmatrix.
 * Ownership: with window_cols == 0 the columns are read before the call
 * returns (in stream order).  With window_cols > 0 the chunk is BORROWED until
 * the window is launched (window full, id_sketch_flush, id_factor,
 * id_coarse_factor, id_sketch_get or id_sketch_destroy): the caller must not
 * overwrite it before then.  Consecutive chunks of one buffer are merged into
 * one launch.  Streaming may continue after id_factor (the sketches are
 * linear in the columns); a later id_factor covers every column so far.
 * Errors: ID_ERR_INVALID_ARG (null pointer, ld < m, ncols < 0, total columns
 * > n_max). */
id_status id_sketch_stream_columns(id_sketch* h, const void* d_cols, int64_t ld, int64_t ncols);

/* Launch every pending (borrowed) chunk now.  Afterwards no chunk is borrowed. */
id_status id_sketch_flush(id_sketch* h);

/* Start a new stream of snapshots with the same config and buffers
 * (columns seen -> 0, W and Y cleared).  Pending chunks are dropped. */
id_status id_sketch_reset(id_sketch* h);

/* Randomized ID of the streamed columns from the small sketch W = Psi A:
 * k-step column-pivoted Householder QR of W (FP64) -> skeleton J, then
 * C = R11^{-1} R12 by back-substitution and P(:,J) = I, P(:,Jc) = C.
 * Passage: Algorithm 4 steps 4-8 (transposed orientation), Sec. 2.4.
 * J: k ints; P: k x n_seen FP64 row-major (host or device).  k_out (host, may
 * be NULL) receives the pivots taken.  n = columns streamed so far.
 * Pivot rule: largest residual column norm, recomputed at every step; ties go
 * to the lowest column index.
 * Returns ID_ERR_RANK_DEFICIENT when fewer than k pivots clear the rank
 * tolerance; J and the first k_out rows of P are still valid.
 * With want_coarse (FP32 data, cooperative coarse QR), the call also starts
 * id_coarse_factor's QR of the same columns on an internal stream of the
 * handle, on all SMs but one, and runs the QR of W in one CTA beside it; it
 * returns when J, P and k_out are ready.  The handle orders that work before
 * anything that would overwrite its inputs (new columns, a reset).
 * Errors: ID_ERR_STATE when no column was streamed. */
id_status id_factor(id_sketch* h, int32_t* J, double* P, int32_t* k_out);

/* Sub-sampled ID (Algorithm 5, transposed): deterministic k-step
 * column-pivoted QR (FP64) of the coarse matrix A_c = A(rows_c, :) gathered
 * during the pass, then P_c as in id_factor.  The pair induces the lifted ID
 * A ~ A(:, J_c) P_c of eq. eq:coarseregA.  rows_c = every stride-th grid index
 * in x, y, z from 0, all components, row r = ((c*ny + j)*nz + kz)*nx + i.
 * If id_factor already started this QR for the current columns, the call
 * waits for it instead of running it again.
 * Errors: ID_ERR_STATE without want_coarse or without columns. */
id_status id_coarse_factor(id_sketch* h, int32_t* Jc, double* Pc, int32_t* k_out);

/* Errors of the reconstruction A_hat = A(:,J) P over an m x n matrix in ONE
 * read of A (device, column-major, lda >= m, the handle's dtype):
 *   rel_fro = ||A - A_hat||_F / ||A||_F                (Sec. 3.3 metric)
 *   rel_max = max_ij |A_ij - A_hat_ij| / |A_ij| over A_ij != 0 (Sec. 3.1)
 * J (k ints) and P (k x n FP64 row-major) may be host or device pointers;
 * rel_fro / rel_max are host pointers (the call synchronises the stream);
 * either may be NULL.  k may be smaller than the handle's k (e.g. k_out).
 * Errors: ID_ERR_INVALID_ARG (null A, lda < m, n < 1, k < 1, k > 64,
 * J entry outside [0, n)). */
id_status id_reconstruct_error(id_sketch* h, const void* d_A, int64_t lda, int64_t n,
                               const int32_t* J, const double* P, int32_t k,
                               double* rel_fro, double* rel_max);

/* Largest k * n of P that id_reconstruct_error_noalloc accepts. */
#define ID_NOALLOC_MAX_KN 131072

/* The error pass of id_reconstruct_error for callers that must not allocate
 * device memory.  No counterpart in the paper: it exists for users whose own
 * allocator already holds the device's memory, who work to a fixed memory
 * budget, or who cannot accept the device-wide synchronisation that
 * cudaMalloc/cudaFree imply.  It needs no handle.  Inputs and outputs are as
 * in id_reconstruct_error; m is the number of rows and dtype the id_dtype of
 * A.  All scratch (per-CTA partial sums, result scalars, copies of J and P)
 * lives in one fixed device array of about 1.1 MB that every GPU loading the
 * library holds until the process exits.  The call allocates nothing.
 * Set-up: the first call on each device (with that device current) looks up
 * the array's device address; make that first call before any stream
 * capture.  All calls on a device share the array: calls that overlap on the
 * GPU race.  Synchronises cuda_stream before returning.  There is no handle,
 * so nothing is poisoned: after ID_ERR_TIMEOUT (a bounded device wait gave
 * up; the kernel has returned and the context stays usable) the next call
 * clears the flag and runs again, whereas a handle of id_reconstruct_error
 * refuses further work after a timeout.
 * Errors: ID_ERR_INVALID_ARG for the cases of id_reconstruct_error, a bad
 * dtype, or k * n > ID_NOALLOC_MAX_KN (the array's capacity for P). */
id_status id_reconstruct_error_noalloc(const void* d_A, int64_t lda, int64_t m, int64_t n,
                                       int32_t dtype, const int32_t* J, const double* P,
                                       int32_t k, double* rel_fro, double* rel_max,
                                       void* cuda_stream);

/* ---------------------------------------------------------------------
 * Single-pass ID (Algorithm 6, Sec. 2.6; eq. eqn:single_ID), column form:
 *   A ~ M A_c(:, J_c) P_c,
 * (J_c, P_c) from id_coarse_factor and M (m x m_c) the coarse-to-fine
 * interpolation of Algorithm 6 step 4: trilinear on the mesh, 8 coarse points
 * per fine point (a fine index on a coarse point takes it alone; between two
 * coarse points the weight follows the physical distance; past the last
 * coarse point a periodic direction wraps to point 0 at x_0 + period and a
 * non-periodic one extrapolates linearly from its last two coarse points).
 * The fine skeleton is never read from A: only A_c is kept.
 * ------------------------------------------------------------------- */

/* Mesh of the grid (host arrays, copied): x[nx], y[ny], z[nz] strictly
 * increasing coordinates of the grid indices; period[d] > 0 makes direction d
 * periodic with that length (x_0 + period > x_last), 0 leaves it open.
 * Requires want_coarse.  Allocates the interpolation tables and an
 * m_c x 64 skeleton buffer on the first call.  Errors: ID_ERR_STATE (no
 * coarse grid), ID_ERR_INVALID_ARG (NULL, non-increasing or non-finite
 * coordinates, bad period), ID_ERR_OOM. */
id_status id_set_mesh(id_sketch* h, const double* x, const double* y, const double* z,
                      const double period[3]);

/* S = M A_c(:, J_c): the single-pass ID's fine skeleton (m x kc, data type,
 * column-major, leading dimension m) written to the device buffer d_S.  J_c:
 * kc column indices of the streamed snapshots (host or device), 1 <= kc <= 64.
 * Synchronises the stream.  Errors: ID_ERR_STATE (no mesh, no coarse grid or
 * no columns yet), ID_ERR_INVALID_ARG (NULL, kc out of range, J_c outside
 * the streamed columns), ID_ERR_CUDA. */
id_status id_single_pass_lift(id_sketch* h, const int32_t* Jc, int32_t kc, void* d_S);

/* Errors of the single-pass ID A_hat = M A_c(:, J_c) P_c against A (device,
 * m x n, column-major, lda >= m, data type), one read of A: rel_fro =
 * ||A - A_hat||_F / ||A||_F and rel_max = max |A_ij - A_hat_ij| / |A_ij| over
 * A_ij != 0 (the metrics of Sec. 3).  P_c: kc x n FP64 row-major (host or
 * device).  Errors as id_single_pass_lift, plus ID_ERR_TIMEOUT. */
id_status id_single_pass_error(id_sketch* h, const void* d_A, int64_t lda, int64_t n,
                               const int32_t* Jc, const double* Pc, int32_t kc, double* rel_fro,
                               double* rel_max);

/* ---------------------------------------------------------------------
 * Batched form: many independent snapshot matrices, of uneven sizes, each
 * through the randomized ID (Algorithm 4, Sec. 2.4) in ONE CUDA-graph launch.
 * This serves the block-wise compression of Sec. 3.3 (a large snapshot
 * matrix split into column blocks, each compressed on its own) and many
 * variables or windows compressed side by side.  Problem b draws its own Psi
 * and Omega from its seed, so its result equals that of one id_sketch handle
 * with the same m, n, k, l, seed, dtype and prec that streams the whole
 * matrix and calls id_factor.
 * ------------------------------------------------------------------- */

/* Largest batch and largest n of one problem of the batched form. */
#define ID_BATCH_MAX_PROBLEMS 1024
#define ID_BATCH_MAX_COLS 512

typedef struct {
  const void* d_A;   /* device, column-major m x n, leading dimension lda;
                        read at every id_batch_run, caller-owned (the caller
                        keeps it alive and unchanged while a run is in flight) */
  int64_t lda;       /* >= m                                                  */
  int64_t m;         /* rows, >= 1                                            */
  int32_t n;         /* snapshots, 1 <= n <= ID_BATCH_MAX_COLS                */
  int32_t k;         /* target rank, 1 <= k <= min(l, n)                      */
  int32_t l;         /* sketch width, k <= l <= 64 (<= 96 for FP32 data)     */
  int32_t dtype;     /* id_dtype of A                                         */
  int32_t prec;      /* ID_SKETCH_EXACT or ID_SKETCH_BF16 (FP32 data only)     */
  int32_t reserved;  /* must be zero                                          */
  uint64_t seed;     /* seed of this problem's Psi and Omega                  */
} id_batch_problem;

typedef struct id_batch id_batch;   /* opaque, library-owned */

/* Create a batch on the current device: copies the problem list, creates one
 * sketch state per problem (and draws each Omega), and builds the work
 * list.  FP32 problems with m >= 128 whose A starts on a 16-byte boundary
 * with lda a multiple of 4 form the work list, run as one persistent
 * tensor-core launch (one CTA per SM): work items (row ranges of a few MB of
 * one problem; problems in order of decreasing QR work) are taken from a
 * device counter, and the CTA that completes a problem's last item sums W
 * from the items' partial slabs and runs the problem's pivoted QR and solve
 * for P while the other CTAs go on with later items.  Every other problem
 * (FP64 data, unaligned columns) keeps its own chain of kernels on a pool of
 * up to 8 worker streams (largest first, to balance the bytes).  cuda_stream: the stream id_batch_run enqueues on (NULL = legacy
 * default stream).  Errors: ID_ERR_INVALID_ARG (NULL, count outside
 * [1, ID_BATCH_MAX_PROBLEMS], a problem out of its ranges), ID_ERR_OOM,
 * ID_ERR_CUDA. */
id_status id_batch_create(const id_batch_problem* problems, int32_t count, void* cuda_stream,
                          id_batch** out);

/* Enqueue the whole batch on the batch's stream: per problem the fused sketch
 * W = Psi A of all n columns, the pivoted QR of W and the solve for P; no
 * host synchronisation.  Outputs (device memory, caller-owned):
 *   J    problem b's k_b pivots at J + sum_{c<b} k_c, pivot order, -1 past k_out
 *   P    problem b's k_b x n_b FP64 row-major at P + sum_{c<b} k_c n_c
 *   kout problem b's k_out at kout[b]
 * The first run (and a run with other output pointers) captures the work
 * into a CUDA graph, the work list and the worker streams as parallel
 * branches; later runs replay it.  The results of a work-list problem equal
 * those of one id_sketch handle up to the FP32 summation order of W (the
 * work items split its rows differently from one handle's CTAs).  Errors: ID_ERR_INVALID_ARG (NULL or host output pointers),
 * ID_ERR_CUDA (the batch is then poisoned: only destroy is valid). */
id_status id_batch_run(id_batch* b, int32_t* J, double* P, int32_t* kout);

/* Wait for the last run; kout_host (count entries, may be NULL) receives
 * every k_out.  Errors: ID_ERR_STATE (no run yet), ID_ERR_TIMEOUT (a device
 * wait of some problem gave up; poisoned), ID_ERR_RANK_DEFICIENT (some
 * k_out < k; the outputs are valid for the k_out pivots), ID_ERR_CUDA. */
id_status id_batch_wait(id_batch* b, int32_t* kout_host);

/* Synchronise the batch's stream and release everything it holds. */
void id_batch_destroy(id_batch* b);

/* Autotuner of the batched form: times the batch's graph with each of the
 * candidate work splits c in {0, 32, 16, 8, 4} -- one warm-up and three
 * timed replays each, CUDA events on the batch's private stream -- and keeps
 * the fastest for later id_batch_run calls (with the same output pointers as
 * here, device).  With a work list, c is the size of a work item in MB of A
 * (0: the work list's bytes over 16 items per SM, between 4 and 64 MB);
 * without one, a problem's sketch runs on at most ceil(row blocks / c) CTAs
 * (0: one CTA per SM).  Outputs: choice (the chosen c, may be NULL), ms (the
 * 5 average replay times in candidate order, host, may be NULL).  The
 * outputs J, P, kout hold a complete result of the batch on return.  No
 * counterpart in the paper.
 * Errors: as id_batch_run, and ID_ERR_TIMEOUT (a device wait of some candidate
 * gave up; poisoned). */
id_status id_batch_tune(id_batch* b, int32_t* J, double* P, int32_t* kout, int32_t* choice,
                        float* ms);

/* ID of the streamed columns with the skeleton chosen among candidates
 * (the learned proposal's): the pivoted QR of W(:, cand) gives J (pivot
 * order, indices of the streamed columns, -1 past k_out), and P (k x n FP64
 * row-major) is the least-squares fit of W on W(:, J) over all n streamed
 * columns -- for a pivoted QR the same as R11^-1 R12 (Sec. 2.4) -- with
 * P(:, J) = I exactly.  cand: ncand distinct column indices (host or
 * device), 1 <= ncand <= n.  Outputs as id_factor (host or device;
 * synchronises the stream).  Errors: ID_ERR_INVALID_ARG (NULL, ncand out of
 * range, a candidate outside the streamed columns or repeated), ID_ERR_STATE
 * (no columns yet), ID_ERR_RANK_DEFICIENT (fewer than k pivots above the
 * rank tolerance among the candidates), ID_ERR_TIMEOUT, ID_ERR_CUDA. */
id_status id_factor_restricted(id_sketch* h, const int32_t* cand, int32_t ncand, int32_t* J,
                               double* P, int32_t* k_out);

/* ---------------------------------------------------------------------
 * Learned skeleton proposal: the network's kernels.  No counterpart in the
 * paper (its conclusion motivates the ID as the selection of the most
 * important snapshots, Sec. 4).  The network scores snapshot columns from
 * coarse-grid features,
 *   s = w2 . gelu(x W1 + b1) + b2,  gelu(z) = z Phi(z)  (exact GELU),
 * and is trained on the skeletons the plain randomized ID picks, with the mean
 * binary cross entropy of sigmoid(s) (positives weighted by pos_weight).
 * All buffers are device FP32, row-major, caller-owned; the calls enqueue on
 * cuda_stream (NULL = legacy default stream) and do not synchronise.  Every
 * sum runs in a fixed order.  Errors: ID_ERR_INVALID_ARG (NULL pointer, a
 * size below 1 or too large), ID_ERR_CUDA.
 * ------------------------------------------------------------------- */

/* X (n x F): X[j * F + f] = scale * A(rows[f], j) for the n columns of A
 * (device, column-major m x n, lda >= m, dtype); rows: F device int64 row
 * indices (a row outside [0, m) gives a NaN feature, never an out-of-bounds
 * read). */
id_status id_mlp_features(const void* d_A, int64_t lda, int64_t m, int64_t n, int32_t dtype,
                          const int64_t* d_rows, int64_t F, float scale, float* d_X,
                          void* cuda_stream);

/* Forward pass on n feature rows X (n x F): Z = X W1 + b1 (n x H), G =
 * gelu(Z), s = G w2 + b2 (n).  W1: F x H; b1, w2: H; b2: 1 value.  The
 * product X W1 runs on the tensor cores with bfloat16 operands (X and W1 are
 * rounded to bfloat16 as they are staged: bfloat16 weights) and FP32
 * accumulation; the bias, GELU and score are FP32. */
id_status id_mlp_forward(const float* d_X, int64_t n, int64_t F, int32_t H, const float* d_W1,
                         const float* d_b1, const float* d_w2, const float* d_b2, float* d_Z,
                         float* d_G, float* d_s, void* cuda_stream);

/* Gradients of the loss for targets y (n values in {0, 1}) from a forward
 * pass's Z, G and s: gW1 (F x H), gb1 (H), gw2 (H), gb2 (1).  Scratch: ds (n),
 * dZ (n x H).  gW1 = X^T dZ runs on the tensor cores (bfloat16 operands, FP32
 * accumulation); the other gradients are FP32. */
id_status id_mlp_backward(const float* d_X, int64_t n, int64_t F, int32_t H, const float* d_Z,
                          const float* d_G, const float* d_w2, const float* d_s,
                          const float* d_y, float pos_weight, float* d_gW1, float* d_gb1,
                          float* d_gw2, float* d_gb2, float* d_ds, float* d_dZ,
                          void* cuda_stream);

/* Gradient step p -= lr g over count values (FP32 master parameters). */
id_status id_mlp_sgd(float* d_p, const float* d_g, int64_t count, float lr, void* cuda_stream);

/* The learned proposal's candidates: the count columns of highest score s
 * (n device values; ties to the lower column index; NaN below every number),
 * written to d_cand (count device int32) in increasing column order.
 * 1 <= count <= n <= 4096. */
id_status id_mlp_propose(const float* d_s, int64_t n, int32_t count, int32_t* d_cand,
                         void* cuda_stream);

/* The stratified proposal: the n columns form `strata` consecutive ranges
 * [q n / strata, (q + 1) n / strata) (snapshots in time order) and each range
 * gives its `per` columns of highest score (ties to the lower index, NaN
 * last).  The candidates go to d_cand (device int32, room for strata * per) in
 * increasing column order and their number (strata * per, or fewer when a
 * range holds fewer than per columns) to d_ncand (device int32, may be NULL).
 * 1 <= strata <= n <= 4096, per >= 1. */
id_status id_mlp_propose_stratified(const float* d_s, int64_t n, int32_t strata, int32_t per,
                                    int32_t* d_cand, int32_t* d_ncand, void* cuda_stream);

/* Synchronises cuda_stream and reports whether a bounded device wait of the
 * tensor-core products gave up since the last check (ID_ERR_TIMEOUT; the
 * affected outputs hold NaN, the flag is cleared) or ID_OK. */
id_status id_mlp_check(void* cuda_stream);

/* Borrow the device buffers of the sketch (valid until reset/destroy):
 *   W  l x n_max FP64, row-major (entry (s, j) at W[s*n_max + j])
 *   Y  m x l, dtype, column-major (entry (i, s) at Y[i + s*m]); NULL unless want_Y
 *   Ac m_c x n_max, dtype, column-major; NULL unless want_coarse
 * Any output pointer may be NULL.  Pending chunks are flushed first. */
id_status id_sketch_get(id_sketch* h, const double** d_W, const void** d_Y, const void** d_Ac,
                        int64_t* n_seen, int64_t* m_c);

/* Release every device buffer of the handle (synchronises its stream). */
void id_sketch_destroy(id_sketch* h);

/* Kernel timing, a measurement aid with no counterpart in the paper.
 * id_timing_enable(h, 1) makes the handle record CUDA events on its stream
 * around every launch of the fused tensor-core sketch kernel (which = 0) and
 * of the error-pass kernel (which = 1); id_timing_enable(h, 0) stops and
 * frees them.  id_timing_read waits for the last recorded launch of that
 * kernel, returns the summed launch durations (ms) and the number of
 * launches since the previous read, and starts a new accumulation.
 * Errors: ID_ERR_INVALID_ARG (bad which / NULL output), ID_ERR_STATE (timing
 * not enabled), ID_ERR_CUDA. */
id_status id_timing_enable(id_sketch* h, int32_t on);
id_status id_timing_read(id_sketch* h, int32_t which, double* total_ms, int64_t* launches);

/* Self-check of the device-side bounded waits, a fault-handling aid with no
 * counterpart in the paper.  Every wait in this library's kernels (mbarrier
 * phases, the coarse QR's grid barrier) gives up after a limit and raises a
 * status word that the host turns into ID_ERR_TIMEOUT, so that a stuck
 * kernel returns instead of hanging the GPU.  This call runs those same wait
 * routines, instantiated with a limit of about 1 ms, on device `device`:
 *   mode 0: an mbarrier phase that nothing completes   -> ID_ERR_TIMEOUT
 *   mode 1: the same phase, completed before the wait -> ID_OK
 *   mode 2: the grid barrier of a cooperative launch of 2 CTAs, one of which
 *           never reaches it                           -> ID_ERR_TIMEOUT
 *   mode 3: the same barrier reached by both CTAs       -> ID_OK
 * Nothing faults and the context stays usable.  Synchronous (its own
 * stream).  Errors: ID_ERR_INVALID_ARG (mode), ID_ERR_CUDA. */
id_status id_check_wait(int32_t device, int32_t mode);

/* Fill out[(i - first) * width + s] = G(i, s) for i in [first, first+count),
 * s in [0, width): the same counter-based Gaussian entries the sketch uses,
 * which = 1 for Psi (G(i,s) = Psi[s, i]) and which = 2 for Omega
 * (G(j,s) = Omega[j, s]).  Definition (the paper only asks for i.i.d.
 * Gaussian entries, Sec. 2.2): Philox4x32-10 with key (seed lo, seed hi),
 * counter (i lo, i hi, s / 10, which); field s % 10 (12 bits) of the 128-bit
 * output indexes the 4096 mid-point normal quantiles rounded to bfloat16.
 * d_out: device FP32 buffer of count*width entries; enqueued on cuda_stream. */
id_status id_gaussian_fill(int32_t which, uint64_t seed, int64_t first, int64_t count,
                           int32_t width, float* d_out, void* cuda_stream);

/* Host-only: the 4096-entry quantile table as bfloat16 bit patterns. */
id_status id_gaussian_table(uint16_t out[4096]);

/* Number of kernels this library has launched in the process so far (all
 * handles, all devices); for accounting in benchmarks. */
int64_t id_kernel_launches(void);

/* Text of the last CUDA error behind an ID_ERR_CUDA status in this process
 * ("no error" if none). */
const char* id_last_cuda_error(void);

/* Static string for a status code. */
const char* id_status_str(id_status s);

/* Library version (major*10000 + minor*100 + patch). */
int32_t id_version(void);

#ifdef __cplusplus
}
#endif

#endif /* IDSKETCH_H */
