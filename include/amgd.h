/*
 * amgd.h -- C ABI of the GB300 (sm_103a) algebraic-distance strength-of-
 * connection library.
 *
 * Method: Brandt, Brannick, Kahl, Livshits, "An algebraic distances measure
 * of AMG strength of connection".  Given a sparse matrix A (CSR) the library
 *   (a) draws K random test vectors and smooths them by nu relaxation sweeps
 *       on A x = 0                                   (§3; §5.2)
 *   (b) for every stored off-diagonal (i,j) fits the one-point least-squares
 *       interpolation p_ij of the target y_i from x_j and returns p_ij and
 *       the minimal functional LS_ij, whose reciprocal is the algebraic
 *       distance r_ij                          (§4.1, Eqs. (3.2), (4.1), (4.3))
 *   (c) keeps (i,j) when r_ij > theta * max_k r_ik and returns the kept
 *       edges as a strength CSR                        (§4.2, Eq. (4.4))
 * All arithmetic runs in hand-written CUDA kernels on the current device.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an int status (AMGD_OK or a negative AMGD_ERR_*);
 *   nothing throws across the ABI.  On error the handle keeps its previous
 *   state and amgd_last_error() holds a message.
 * - Ownership: the caller owns every array it passes.  amgd_create copies
 *   the matrix into device memory owned by the handle; outputs are written
 *   into caller buffers.  amgd_destroy frees everything the handle owns.
 * - mem = AMGD_MEM_HOST: the pointers are host memory; the call copies
 *   through the handle's stream and returns when the data is in place.
 *   mem = AMGD_MEM_DEVICE: the pointers are device memory of the current
 *   device; the call only enqueues work on the handle's stream.
 * - Ordering: every call is ordered on the handle's stream (default: the
 *   legacy default stream).  A handle is not thread-safe; distinct handles
 *   are independent.
 * - Sizes: 0 <= n < 2^31, nnz < 2^31, 1 <= K <= 64.
 * - Row order of A and the order of the columns inside each row are the
 *   caller's and are preserved: they fix the summation order of every row
 *   sum, and the order of the strength CSR.
 */
#ifndef AMGD_H
#define AMGD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amgd_ctx *amgd_handle;

/* status codes */
#define AMGD_OK               0
#define AMGD_ERR_ARG         -1   /* bad argument (size, pointer, enum, value)   */
#define AMGD_ERR_CSR         -2   /* row_ptr not monotone, column out of range,
                                     duplicate (i,j), non-finite value          */
#define AMGD_ERR_ZERO_DIAG   -3   /* a row without a stored nonzero diagonal    */
#define AMGD_ERR_CUDA        -4   /* a CUDA runtime error (text in last_error)  */
#define AMGD_ERR_OOM         -5   /* device allocation failed                   */
#define AMGD_ERR_STATE       -6   /* call out of order (e.g. strength before
                                     distances, MCGS without a coloring)        */
#define AMGD_ERR_CAPACITY    -7   /* output buffer too small                    */
#define AMGD_ERR_TIMEOUT     -8   /* a bounded device wait gave up; reported by the
                                     next call that synchronises the stream     */
#define AMGD_ERR_UNSUPPORTED -9   /* size or mode outside the supported range   */
#define AMGD_ERR_CHECK       -10  /* checked build only: a gather index (column
                                     index or row map) failed its bounds test;
                                     reported by the next call that synchronises
                                     the stream, the results are not valid      */

/* where caller arrays live */
#define AMGD_MEM_HOST   0
#define AMGD_MEM_DEVICE 1

/* relaxation sweep types (§3; §2 names Gauss-Seidel, §5.2 uses it) */
#define AMGD_SWEEP_JACOBI 0   /* x <- x - omega D^-1 A x, all rows at once          */
#define AMGD_SWEEP_MCGS   1   /* multicolor Gauss-Seidel / SOR over a given coloring */

/* LS target of the one-point fit */
#define AMGD_TARGET_RESIDUAL 0   /* y_i = x_i - (A x)_i / a_ii  (Eqs. (3.2), (4.1), (4.3)) */
#define AMGD_TARGET_PLAIN    1   /* y_i = x_i                   (Eq. (3.1))               */

/* test-vector storage precision */
#define AMGD_FP64 0   /* FP64 vectors, FP64 arithmetic                                  */
#define AMGD_FP32 1   /* FP32 vectors, FP32 arithmetic (LS sums: amgd_set_summation)   */
#define AMGD_BF16 2   /* BF16 vectors, FP32 arithmetic (LS sums: amgd_set_summation)   */

/* summation of the K-term LS sums on the mixed paths (amgd_set_summation) */
#define AMGD_SUM_PLAIN       0   /* FP32 fused multiply-add chains                  */
#define AMGD_SUM_COMPENSATED 1   /* compensated FP32 sums (default)                  */

/*
 * amgd_create -- build a handle for one n x n matrix A in CSR form.
 *   row_ptr[n+1] (int64, row_ptr[0] = 0, non-decreasing), col[nnz] (int32,
 *   0 <= col < n, no duplicate column inside a row), val[nnz] (finite
 *   doubles); every row must store its diagonal with a nonzero value.  This
 *   is the graph G_1 of A (§4.1, Eq. (4.2) with d = 1): the distances are
 *   evaluated on exactly the stored off-diagonals.
 *   K: number of test vectors (1..64).  seed: Philox4x64-10 key word 0 for
 *   the starting vectors; amgd_create leaves the vectors at that start
 *   (see amgd_init_vectors).  Storage starts as AMGD_FP64, target as
 *   AMGD_TARGET_RESIDUAL, LS weights as all ones.
 *   mem: where row_ptr/col/val live.  *out receives the handle (NULL on error).
 *   Errors: ARG, CSR, ZERO_DIAG, UNSUPPORTED, OOM, CUDA.
 */
int amgd_create(const int64_t *row_ptr, const int32_t *col, const double *val, int64_t n,
                int32_t K, uint64_t seed, int mem, amgd_handle *out);

/*
 * amgd_create_batch -- one handle over nmat independent matrices of uneven
 *   size, processed together by every kernel launch (block-diagonal
 *   concatenation: matrix b's rows follow matrix b-1's and its columns are
 *   shifted by the same offset).  row_ptr[b], col[b], val[b], n[b] describe
 *   matrix b exactly as in amgd_create.  Test vectors of matrix b use
 *   Philox key (seed, b) and the row index local to matrix b, so a batched
 *   build equals nmat separate builds bit for bit.  All outputs are in the
 *   concatenated numbering (amgd_batch_offsets gives the row and slot
 *   offsets of each matrix).  Errors as amgd_create.
 */
int amgd_create_batch(int32_t nmat, const int64_t *const *row_ptr, const int32_t *const *col,
                      const double *const *val, const int64_t *n, int32_t K, uint64_t seed,
                      int mem, amgd_handle *out);

/*
 * amgd_set_matrix_ids -- Philox key word 1 of the start vectors of each
 *   matrix of the handle: ids[nmat] (host, each >= 0; NULL restores the
 *   default, matrix b keyed b).  A process that builds a subset of a larger
 *   batch (one shard of its matrices, e.g. one GPU's share) passes the
 *   matrices' indices in the whole batch, so every matrix gets the same
 *   start vectors -- hence the same results bit for bit -- as in a build of
 *   the whole batch.  Takes effect at the next amgd_init_vectors or capture;
 *   synchronises the handle's stream and drops a captured graph.  The paper
 *   has no counterpart (it is the sharding of independent problems).
 *   Errors: ARG, STATE, OOM, CUDA.
 */
int amgd_set_matrix_ids(amgd_handle h, const int64_t *ids);

/* Row offsets (nmat+1) and CSR-slot offsets (nmat+1) of the matrices of a
 * batch handle, written to host arrays; a single-matrix handle has nmat 1. */
int amgd_batch_offsets(amgd_handle h, int64_t *row_off, int64_t *slot_off);

/* Sizes of a handle: n (total rows), nnz (stored entries), number of stored
 * off-diagonals E, K, nmat.  Any pointer may be NULL. */
int amgd_sizes(amgd_handle h, int64_t *n, int64_t *nnz, int64_t *E, int32_t *K, int32_t *nmat);

/* Make every later call of this handle use `stream` (a cudaStream_t of the
 * current device; NULL = legacy default stream). */
int amgd_set_stream(amgd_handle h, void *stream);

/* Storage precision of the test vectors (AMGD_FP64/FP32/BF16).  The current
 * vectors are converted by round-to-nearest-even; computed distances are
 * invalidated.  Errors: ARG, OOM, CUDA. */
int amgd_set_precision(amgd_handle h, int storage);

/* LS target: AMGD_TARGET_RESIDUAL (default) or AMGD_TARGET_PLAIN. */
int amgd_set_target(amgd_handle h, int target);

/*
 * amgd_set_summation -- how the mixed paths (FP32/BF16 storage, FP32
 *   arithmetic) form the K-term sums S_xx = sum w x_j^2, S_yx = sum w y_i x_j
 *   and LS_ij = sum w (y_i - a_ij x_j)^2 of the one-point fit (§4.1, Eq.
 *   (4.3)).  AMGD_SUM_COMPENSATED (the default): every lane keeps a running
 *   FP32 sum and the exact rounding error of each of its additions (TwoSum)
 *   in a second FP32 word (the Kahan-Babuska-Neumaier scheme), the lanes of a
 *   row combine their pairs with TwoSum in the shuffle reduction, and the two
 *   words are added once at the end.  AMGD_SUM_PLAIN: FP32 fused
 *   multiply-add chains.  Either way an edge whose LS falls below 1e-4 of
 *   sum_k w_k y_k^2 makes its row be redone in FP64 (cancellation).  Every
 *   distance kernel (each edge stage, any search depth) honours the
 *   setting; the FP64 path ignores it.  Drops computed distances and a
 *   captured graph.
 *   Errors: ARG.
 */
int amgd_set_summation(amgd_handle h, int mode);

/* LS weights w[K] (host doubles, each > 0 and finite; §3.1 weights
 * omega_kappa of Eq. (3.1)); NULL restores all ones. */
int amgd_set_weights(amgd_handle h, const double *w);

/*
 * amgd_set_coloring -- the coloring that fixes the Gauss-Seidel order of
 *   AMGD_SWEEP_MCGS: color[n] in 0..ncolors-1 (host or device per mem).
 *   Colors are swept in increasing order; a row of color c is updated from
 *   the new values of rows of smaller colors and the values from the start
 *   of the sweep of every other row, itself included.  For a proper
 *   coloring this is Gauss-Seidel (SOR) in color order; for an improper one
 *   (red-black on a 9-point stencil) it is the same well-defined rule.  The
 *   handle reorders its rows by color internally; results are returned in
 *   the caller's order.  The current vectors are kept.
 *   Errors: ARG (color out of range), OOM, CUDA.
 */
int amgd_set_coloring(amgd_handle h, const int32_t *color, int32_t ncolors, int mem);

/* Reset the test vectors to the Philox4x64-10 start for `seed`: element
 * (i, k) of matrix b is (2m + 1) 2^-32 - 1, where m is the 32-bit half
 * (k mod 2, low half first) of word ((k/2) mod 4) of Philox4x64-10 at counter
 * (i, k/8, 0, 0), key (seed, b); rounded to the storage precision.  (§3:
 * relaxation starts from random vectors.) */
int amgd_init_vectors(amgd_handle h, uint64_t seed);

/* Copy the test vectors in/out as an n x K row-major block of doubles
 * (caller's row order).  set rounds to the storage precision; get widens
 * exactly. */
int amgd_set_vectors(amgd_handle h, const double *X, int mem);
int amgd_get_vectors(amgd_handle h, double *X, int mem);

/* Replace the values of A (same pattern and slot order as at create;
 * val[nnz] host or device).  The values are staged on the device and checked
 * there (finite, nonzero diagonal) before they replace the old ones; the call
 * synchronises the handle's stream.  Errors: ARG, CSR, ZERO_DIAG, CUDA. */
int amgd_set_values(amgd_handle h, const double *val, int mem);

/*
 * Stream-ordered value updates and results, for a stream of matrices that
 * share one pattern (each replayed through a captured build).  No call below
 * synchronises; copies run on two copy streams of the handle, double-buffered,
 * so that the upload of the next values and the download of the last strength
 * graph overlap the build between them.
 * amgd_set_values_async -- like amgd_set_values: val[nnz] (host: page-locked
 *   memory for the copy to be asynchronous; or device) is copied into one of
 *   two staging buffers, checked on the device (finite, nonzero diagonal) and
 *   applied in the handle's stream order.  val must stay valid and unchanged
 *   until amgd_sync returns.  Values that fail the check are applied all the
 *   same (results computed from them are meaningless) and the next amgd_sync
 *   returns the error.
 * amgd_strength_async -- the current strength graph M^d (§4.2) as CSR, like
 *   amgd_strength: s_row_ptr[n+1] and the first min(cap, E) columns of s_col
 *   (E the stored off-diagonals of the pattern), in host or device memory
 *   (mem); valid after amgd_sync.  The next amgd_sync returns CAPACITY if the
 *   graph has more than cap columns.
 * amgd_sync -- waits for every asynchronous copy and kernel of the handle and
 *   reports the deferred errors.  Until it returns, calls that change the
 *   layout or the captured graph (precision, coloring, search depth, autotune,
 *   graph capture) return STATE.
 *   Errors: ARG, STATE (no distances yet, for amgd_strength_async), CSR,
 *   ZERO_DIAG, CAPACITY (at amgd_sync), CUDA.
 */
int amgd_set_values_async(amgd_handle h, const double *val, int mem);
int amgd_strength_async(amgd_handle h, int64_t *s_row_ptr, int32_t *s_col, int64_t cap, int mem);
int amgd_sync(amgd_handle h);

/*
 * amgd_relax -- nu sweeps on A x = 0 applied to all K vectors (§3):
 *   AMGD_SWEEP_JACOBI: x_i <- x_i - (omega / a_ii) sum_j a_ij x_j
 *   AMGD_SWEEP_MCGS:   as set by amgd_set_coloring, SOR weight omega
 *   Sweeps accumulate on the current vectors.  nu >= 0, omega finite.
 *   Errors: ARG, STATE (MCGS without coloring), CUDA.
 */
int amgd_relax(amgd_handle h, int32_t nu, double omega, int sweep_type);

/*
 * amgd_distances -- one-point LS fit for every stored off-diagonal slot p =
 *   (i,j) of A (§4.1, Eq. (4.3)) on the current vectors, and the strength
 *   flags for threshold theta (>= 0, finite; Eq. (4.4)).  Outputs are
 *   aligned with A's CSR slots (nnz long, caller's order) and any may be NULL
 *   (the values are kept on the device either way for amgd_strength):
 *     a[p]    the minimiser p_ij (0 on the diagonal)
 *     dist[p] the algebraic distance r_ij = 1 / LS_ij (+inf for LS = 0,
 *             NaN on the diagonal)
 *     ls[p]   the minimal LS functional LS_ij (NaN on the diagonal)
 *   For the residual target, a row with a single off-diagonal has
 *   y_i = -(a_ij/a_ii) x_j exactly: a = -a_ij/a_ii, LS = 0 are returned.
 *   With a search depth d > 1 (amgd_set_search_depth) the fits, the
 *   threshold and every per-slot output follow the entries of the graph G_d
 *   of A^d instead of A's (nnz_p entries, see amgd_distance_pattern); the
 *   target is still built from row i of A (Eq. (4.3)).
 *   Mixed precisions compute in FP32 -- the LS sums compensated or plain,
 *   see amgd_set_summation -- and redo in FP64 the row of an edge whose LS
 *   is below 1e-4 * sum_k w_k y_k^2 (cancellation).
 *   Errors: ARG, CUDA.
 */
int amgd_distances(amgd_handle h, double theta, double *a, double *dist, double *ls, int mem);

/*
 * amgd_set_search_depth -- d = 1 (default) measures the stored entries of A;
 *   d > 1 measures every pair (i, j) with (A^d)_ij != 0: the graph G_d of
 *   §4.1, Eq. (4.2), and the strength graph M^d of §4.2.  The pattern is
 *   structural (numerical cancellation in A^d is ignored) and is built from
 *   the graph of A alone (A^d is never formed): because every row holds its
 *   diagonal, it is every j within d steps of i, i itself included, columns
 *   ascending.  Setting d drops computed distances and any captured graph.
 *   1 <= d <= 16.  Errors: ARG, UNSUPPORTED (2^31 entries or more), OOM, CUDA.
 * amgd_distance_pattern -- the current pattern: row_ptr[n+1] (int64) and
 *   col[cap] (int32), either may be NULL; *nnz_p (may be NULL) receives its
 *   entry count.  Synchronous.  Errors: ARG, CAPACITY (cap < nnz_p), CUDA.
 */
int amgd_set_search_depth(amgd_handle h, int32_t d);
int amgd_distance_pattern(amgd_handle h, int64_t *row_ptr, int32_t *col, int64_t cap,
                          int64_t *nnz_p, int mem);

/*
 * amgd_strength -- the strength graph M^d (§4.2) from the flags of the last
 *   amgd_distances call: s_row_ptr[n+1] (int64), s_col[cap] (int32), kept
 *   edges row by row in the slot order of A (d = 1) or of G_d.
 *   mem = AMGD_MEM_DEVICE with cap >= E_p (the off-diagonal entries of the
 *     pattern: nnz_p - n; E for d = 1): enqueued without synchronising;
 *     the total is s_row_ptr[n] on the device; *nnz_s (may be NULL) is set
 *     after a synchronisation only if nnz_s is not NULL.
 *   otherwise the call synchronises, sets *nnz_s and returns
 *     AMGD_ERR_CAPACITY (nothing written to s_col) if cap is too small.
 *   Errors: ARG, STATE (no distances yet), CAPACITY, CUDA.
 */
int amgd_strength(amgd_handle h, int64_t *s_row_ptr, int32_t *s_col, int64_t cap,
                  int64_t *nnz_s, int mem);

/*
 * amgd_graph_capture -- record one whole build (vector start from `seed`,
 *   nu sweeps, distances for theta, strength CSR into the DEVICE buffers
 *   s_row_ptr[n+1], s_col[cap >= E_p]) as a CUDA graph owned by the handle;
 *   amgd_graph_launch replays it on the handle's stream.  Replaces any
 *   earlier graph.  Errors: ARG, STATE, CAPACITY (cap < E), CUDA.
 */
int amgd_graph_capture(amgd_handle h, uint64_t seed, int32_t nu, double omega, int sweep_type,
                       double theta, int64_t *s_row_ptr, int32_t *s_col, int64_t cap);
int amgd_graph_launch(amgd_handle h);

/*
 * Kernel shapes and the autotuner.  A row of test vectors is P = Kp/V
 *   sixteen-byte vectors (V = 2, 4, 8 elements for FP64, FP32, BF16); a
 *   shape spreads them over G lanes with NV vectors per lane (G*NV = P,
 *   NV in {1,2,4}) and gathers U nonzeros per batch (U in {4,8}; the
 *   distance pass also takes U = 2).  In these terms a warp holds 32/G
 *   rows and a lane's tile of K is NV*V components; a lane with an even NV
 *   holds its vectors side by side and moves two per 32-byte access, others
 *   move one per 16-byte access; the tuner picks all three.  For the
 *   relaxation, staged selects the kernel: 0 direct; 1 persistent, each
 *   tile's CSR slice copied into shared memory with TMA bulk copies ahead of
 *   use (waits bounded to about one second; a wait that runs out makes the
 *   next synchronising call return AMGD_ERR_TIMEOUT); 2 warp-pipelined, CSR
 *   slices and neighbour rows copied with cp.async two and one row groups
 *   ahead (U must be 4); 3 chunked, one 896-thread block per SM owning a
 *   contiguous run of rows, each warp asking the L2 for the row pointers
 *   and CSR lines of its next row groups ahead of use and loading the CSR
 *   with an evict-first and the vectors with an evict-last cache policy.
 *   For the distance pass, staged selects 0 the row
 *   kernel (G lanes per row), 1 the tile kernel (one thread per stored
 *   entry), 2 the row kernel reading the vectors in the sweeps' row order
 *   in place (search depth 1: no caller-order copy of the vectors; U in
 *   {2,4}; the default) or 3 the warp-staged kernel on that order (each
 *   warp gathers its rows' neighbour vectors once, G lanes per row, into a
 *   shared-memory window and fits one stored entry per lane; U in {4,8}).
 *   With search depth d > 1 a stage-2 or stage-3 shape runs as stage 0.  Shapes change speed only, never results beyond the order of
 *   the K-term LS sums.  kernel: AMGD_KERNEL_RELAX (the sweeps) or
 *   AMGD_KERNEL_EDGE (the distance pass); the shape applies to the current
 *   storage precision.
 * amgd_autotune times every valid shape of both kernels on the handle's own
 *   matrix and vectors (one sweep of sweep_type/omega into the spare vector
 *   buffer -- the current vectors are kept -- and one distance pass;
 *   computed distances are invalidated) and keeps the fastest.  cache_path
 *   (may be NULL): a text file of earlier results keyed by GPU name,
 *   storage, K, size buckets, sweep type and color count; a matching line
 *   is used without timing, a new result is appended.
 *   Errors: ARG, STATE (MCGS without coloring), CUDA.
 */
#define AMGD_KERNEL_RELAX 0
#define AMGD_KERNEL_EDGE  1
int amgd_set_kernel_shape(amgd_handle h, int kernel, int G, int NV, int U, int staged);
int amgd_get_kernel_shape(amgd_handle h, int kernel, int *G, int *NV, int *U, int *staged);
int amgd_autotune(amgd_handle h, int sweep_type, double omega, const char *cache_path);

/*
 * Phase timing of captured builds.  amgd_enable_phase_timing(h, 1) before
 *   amgd_graph_capture makes the captured graph record CUDA events (owned by
 *   the handle) on the stream it runs on at the boundaries
 *   start | vectors | sweeps | distances | strength.  amgd_phase_times waits
 *   for the last replay and writes the four phase durations in milliseconds
 *   (vector start, nu sweeps, distances, strength CSR).
 *   Errors: ARG, STATE (no timed graph has been captured), CUDA.
 */
int amgd_enable_phase_timing(amgd_handle h, int enable);
int amgd_phase_times(amgd_handle h, float *ms);

/*
 * amgd_ls_interpolation -- least-squares interpolation of caliber c (§4.3;
 *   the functional of Eq. (3.1), or of Eq. (3.2) for the residual target,
 *   over a set W of coarse points), from the current vectors (after
 *   amgd_relax) and the current target and weights.
 *   coarse[n] (coarse_mem): 1 for a coarse point, 0 for a fine point.
 *   For a fine row i the candidates are the coarse points among the entries
 *   of row i of the current pattern (A for search depth 1, the graph G_d of
 *   A^d after amgd_set_search_depth(d): the d_LS-ring of Eq. (4.5)); at most
 *   32 per row.  Every subset W with |W| <= c is fitted (weighted normal
 *   equations, Gaussian elimination with partial pivoting; a set whose
 *   pivot falls below 1e-13 of the largest diagonal entry is skipped) and
 *   scored by LS_W = sum_k w_k (y_ik - sum_{j in W} p_j x_jk)^2; the first
 *   set in lexicographic order with the smallest LS is kept for each size.
 *   Sizes then compete with the penalty of §4.3 on LS / S_yy (S_yy =
 *   sum_k w_k y_ik^2): starting from the empty set (1), size m replaces the
 *   current size m' < m when LS_m / S_yy < (LS_m' / S_yy)^(gamma (m - m')).
 *   A coarse row interpolates itself (weight 1).  Computed in FP64 from the
 *   vectors widened exactly, with the rounding order of the definition.
 *   Outputs (mem): p_row_ptr[n+1] (int64); p_col[cap] (int32, ascending per
 *   row) and p_val[cap] (double) -- both NULL to query the size; ls[n] (may
 *   be NULL): the chosen LS per row (0 for coarse rows).  *nnz_p (may be
 *   NULL): the entry count.  1 <= c <= 4, gamma >= 0.  Synchronous.
 *   Errors: ARG, CAPACITY (cap too small; p_row_ptr still written),
 *   UNSUPPORTED (a row with more than 32 candidates, K > 64), CUDA.
 */
int amgd_ls_interpolation(amgd_handle h, const uint8_t *coarse, int coarse_mem, int32_t caliber,
                          double gamma, int64_t *p_row_ptr, int32_t *p_col, double *p_val,
                          int64_t cap, int64_t *nnz_p, double *ls, int mem);

/*
 * amgd_cr_coarsen -- compatible-relaxation coarsening (§3.2 Eqs. (3.4),
 *   (3.5); §4.2 Eq. (4.4); Algorithm 1 with the candidate measure of the
 *   Remark after it).  coarse[n] (coarse_mem): C_0 on entry (nonzero =
 *   coarse; C_0 empty is allowed), C on exit (0/1).  Each stage:
 *   (1) nu F-relaxation sweeps of one vector from u = 1 on F, u = 0 held on
 *       C: the sweep of amgd_relax (sweep: AMGD_SWEEP_JACOBI with weight
 *       omega, or AMGD_SWEEP_MCGS over the coloring of amgd_set_coloring,
 *       SOR weight omega) restricted to the rows of F, in FP64 (row sums as
 *       fused multiply-adds in CSR order);
 *   (2) rho_f = ||u^nu||_inf^(1/nu) (Eq. (3.5) in the max norm; 0 when F is
 *       empty), written to rho[stage];
 *   (3) stop when rho_f <= delta or when max_sets sets have been added;
 *   (4) candidates Z = { i in F : |u_i| / ||u^nu||_inf > tol };
 *   (5) the strength graph on F: slot (i, j) of the current pattern (A, or
 *       G_d after amgd_set_search_depth) is strong iff i, j in F, j != i
 *       and LS_ij = 0 or theta LS_ij < min over the F neighbours k of LS_ik;
 *   (6) C gains the independent set of Z (strong slots in either direction
 *       are edges) that the greedy order selects: more candidates j with
 *       (j, i) strong first, then the larger key (word 0 of Philox4x64-10
 *       with counter (i, stage, 1, 0) and key (seed, 0)), then the smaller
 *       index.  It is computed by rounds of local maxima in that order.
 *   ls (ls_mem): FP64 LS per slot of the current pattern (nnz of the
 *   pattern, diagonal slots ignored), or NULL for the LS of the last
 *   amgd_distances (widened exactly).  rho: max_sets + 1 doubles on the host
 *   (may be NULL); *n_rho (may be NULL): the number of estimates written =
 *   the number of stages.  nu >= 1, max_sets >= 0.  Synchronous; one host
 *   read per stage and per batch of selection rounds.  Single-matrix
 *   handles only.
 *   Errors: ARG, STATE (no LS and no distances; MCGS without coloring),
 *   UNSUPPORTED (batched handle), CUDA.
 */
int amgd_cr_coarsen(amgd_handle h, uint8_t *coarse, int coarse_mem, const double *ls, int ls_mem,
                    int sweep, double omega, int32_t nu, double theta, double delta, double tol,
                    int32_t max_sets, uint64_t seed, double *rho, int32_t *n_rho);

/*
 * amgd_cr_stats -- counters of the last amgd_cr_coarsen on this handle:
 *   *rounds (may be NULL) the selection rounds launched over all stages
 *   (local-maximum rounds come in batches of 4 or 8, so this is at least the
 *   number needed); *launches (may be NULL) the kernels it launched.
 *   Errors: ARG.
 */
int amgd_cr_stats(amgd_handle h, int32_t *rounds, int64_t *launches);

/*
 * Reverse pass.  The paper differentiates nothing; these calls give the
 * gradient of a scalar loss on the LS values with respect to the values of A
 * and the Jacobi weight omega, by the chain rule through the steps of §3
 * (Jacobi sweeps on A x = 0), Eqs. (3.2), (4.1) (the LS target) and §4.1,
 * Eq. (4.3) (the one-point fits; a_ij minimises LS_ij, so the dependence
 * through a_ij drops out).  The start vectors are treated as constants.
 *
 * amgd_set_checkpointing -- every > 0: each later amgd_relax with
 *   AMGD_SWEEP_JACOBI (on a handle without a coloring) records its
 *   trajectory: the iterates X_0, X_every, X_2every, ... are kept in device
 *   memory owned by the handle (ceil(nu/every) blocks of n x Kp storage
 *   elements); amgd_backward recomputes the iterates between checkpoints
 *   (every - 1 more blocks).  every = 0 (the default) records nothing.
 *   Errors: ARG.
 *
 * amgd_backward -- reverse pass over the last recorded amgd_relax followed
 *   by amgd_distances (nothing else that changes the vectors, values,
 *   weights, target or precision in between).
 *   ls_bar[nnz] (mem): dL/dLS_p per slot, caller's slot order; entries on
 *     the diagonal and, for the residual target, in rows with one
 *     off-diagonal (where LS is the constant 0) are ignored.
 *     NULL: the loss is L = sum_p r_p^2 = sum_p LS_p^-2 over the slots the
 *     last amgd_distances kept (flags held fixed) with LS_p > 0.
 *   val_bar[nnz] (mem, written): dL/da_p for every stored value (a
 *     diagonal value enters both A and D: both parts are summed).
 *   omega_bar (host, may be NULL): dL/domega.
 *   loss (host, may be NULL): L for ls_bar == NULL, NaN otherwise.
 *   Arithmetic is that of the storage precision (FP64, or FP32 for the
 *   FP32/BF16 storages); sums have a fixed order (deterministic results).
 *   Synchronises when mem is AMGD_MEM_HOST or omega_bar / loss is given;
 *   otherwise it only enqueues work and amgd_backward_scalars fetches the
 *   two scalars later.
 *   Errors: ARG, STATE (no recorded trajectory or no distances after it),
 *   UNSUPPORTED (a coloring is set), CUDA.
 *
 * amgd_backward_scalars -- waits for the last reverse pass (eager or graph
 *   replay) and writes dL/domega and the loss (NaN unless the built-in loss
 *   was used); either pointer may be NULL.  Errors: ARG, STATE, CUDA.
 *
 * amgd_graph_capture_backward -- record one whole forward + reverse step as
 *   the handle's CUDA graph (replaces any earlier graph; replay with
 *   amgd_graph_launch): vector start from `seed`, nu recorded Jacobi sweeps
 *   with weight omega (checkpoint interval as set), distances for theta,
 *   and the reverse pass of the built-in loss with dL/dval written to the
 *   DEVICE buffer val_bar[nnz].  Phase timing, when enabled, records the
 *   boundaries start | vectors | sweeps | distances | reverse pass.
 *   Errors: ARG, STATE (checkpointing off), UNSUPPORTED (coloring set), CUDA.
 */
int amgd_set_checkpointing(amgd_handle h, int32_t every);
int amgd_backward(amgd_handle h, const double *ls_bar, int mem, double *val_bar,
                  double *omega_bar, double *loss);
int amgd_backward_scalars(amgd_handle h, double *omega_bar, double *loss);
int amgd_graph_capture_backward(amgd_handle h, uint64_t seed, int32_t nu, double omega,
                                double theta, double *val_bar);

/*
 * amgd_strength_noalloc -- the threshold of Eq. (4.4) and the strength CSR,
 *   computed from distances the caller already holds, without allocating
 *   any memory.  The paper has no counterpart to this entry point: it exists
 *   for callers that cannot call cudaMalloc (code running inside a memory
 *   pool or arena that owns every device allocation of the process, or a
 *   loop that must never take the CUDA driver's allocation lock), since every
 *   handle-based entry point allocates device memory for its handle.
 *
 *   All pointers are DEVICE memory of the current device:
 *     row_ptr[n+1] (int64) and col[nnz] (int32): the CSR pattern of A;
 *     ls[nnz]: LS_ij per slot (as written by amgd_distances; diagonal slots
 *       are recognised by col == row and ignored);
 *     s_row_ptr[n+1], s_col[cap]: the output CSR, rows in order, kept
 *       columns in slot order.  If s_row_ptr[n] > cap after the call, only
 *       the first cap columns were written.
 *   n >= 0 and theta >= 0 (else ARG).  stream: a cudaStream_t (NULL =
 *   legacy default stream); the call only enqueues work.
 *
 *   Working memory: a file-scope device array of 65536 int64 (512 KiB, one
 *   entry per tile of 4096 rows: the 64-bit offset of the tile's first kept
 *   edge, so strength graphs with 2^31 or more edges are counted exactly)
 *   that every GPU loading the library keeps until the process exits.  Hence
 *   n <= 268,435,456; larger n is rejected with AMGD_ERR_UNSUPPORTED before
 *   any GPU work.  The first call on a
 *   device looks up the array's device address with that device current
 *   (make this first call before any stream capture).  Every call reuses the
 *   same array; calls whose GPU work overlaps (other streams, other threads
 *   on the same device) race on it and must be serialised by the caller.
 *   Nothing is allocated or freed: no cudaMalloc, no cudaFree.
 *   Errors: ARG, UNSUPPORTED, CUDA (text in amgd_last_error(NULL)).
 */
int amgd_strength_noalloc(const int64_t *row_ptr, const int32_t *col, const double *ls,
                          int64_t n, double theta, int64_t *s_row_ptr, int32_t *s_col,
                          int64_t cap, void *stream);

/* Free everything the handle owns (synchronises its stream); NULL is a no-op. */
int amgd_destroy(amgd_handle h);

/* Static text of a status code. */
const char *amgd_status_string(int status);

/* 1 when this library is the checked build (libamgd_checked.so: every gather
 * index of the sweep and distance kernels is tested against the vector block
 * before its load; a failure is reported as AMGD_ERR_CHECK), else 0.  The
 * checked build is for tests; it is slower and computes the same results. */
int amgd_checked_build(void);

/* Message of the last error of h, or, when h is NULL, of the last failed
 * amgd_create / amgd_create_batch / amgd_strength_noalloc on this thread.
 * Valid until the next call on h. */
const char *amgd_last_error(amgd_handle h);

#ifdef __cplusplus
}
#endif
#endif /* AMGD_H */
