/*
 * sgks.h -- C ABI of the GB300 sGKS library (sketched generalized Krylov subspace method
 * for general-form Tikhonov regularization).
 *
 * Problem (paper Sec. 1, eq. tik):   min_x ||A x - b||^2 + lambda ||L x||^2,
 * A in R^{m x n}, L in R^{p x n}, lambda > 0.  The solver is Algorithm 2 (sGKS): the basis
 * W_k = [W_0, r_1, ..., r_k] is never orthogonalised; each new column r_{k+1} is the gradient
 * A^T (A x_k - b) + lambda L^T L x_k (eq. gradient); the projected problem is solved through
 * sketched QR factors S_A A W_k = Q_A R_A, S_L L W_k = Q_L R_L updated one column at a time
 * (eq. updqr, eq. projected_sketched_bis).  W_0 spans K_l(A^T A, A^T b), l = 3 (Sec. 4).
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers (CUDA global memory of the current device) unless
 *    the argument description says "host".  The caller owns them; the library never frees
 *    them.  Arrays passed to sgks_create must stay valid and unchanged until sgks_destroy.
 *  - Every function returns an int status: SGKS_OK (0), a negative error code, or a positive
 *    warning.  No function throws across the ABI.  A handle is not thread-safe.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream); all
 *    device work of a handle is ordered on that stream.
 *  - Images are row-major with x fastest (pixel (iy, ix) -> iy*nx + ix); space-time unknowns
 *    are frame-major (t*ny*nx + iy*nx + ix).
 */
#ifndef SGKS_H
#define SGKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define SGKS_OK             0
#define SGKS_BREAKDOWN      1   /* warning: new column numerically in the span of W (both sketched
                                   residual norms <= 1e-13 of the column norm, or exactly 0);
                                   it was not appended and the solve stopped early            */
#define SGKS_STOPPED        2   /* info: the relative-change test RC_k < tol stopped the solve */
#define SGKS_ERR_INVALID   -1   /* bad argument or descriptor                                  */
#define SGKS_ERR_CUDA      -2   /* a CUDA runtime call failed (see sgks_last_error)             */
#define SGKS_ERR_NONFINITE -3   /* NaN/Inf met in a sketched column or a residual norm         */
#define SGKS_ERR_STATE     -4   /* call not valid in the handle's state (e.g. basis full)       */
#define SGKS_ERR_NOMEM     -5   /* device allocation failed                                    */
#define SGKS_ERR_SKETCH    -6   /* sparse-sign draw limit (256 draws for one column) exceeded   */

/* ---- enums ------------------------------------------------------------------------------ */
enum { SGKS_F32 = 0, SGKS_F64 = 1 };
enum { SGKS_OP_DENSE = 1, SGKS_OP_CSR = 2, SGKS_OP_CONV2D = 3 };
enum { SGKS_REG_FD1 = 1, SGKS_REG_GRAD2D = 2, SGKS_REG_LAPLACE2D = 3, SGKS_REG_SPACETIME = 4 };
enum { SGKS_SKETCH_SPARSE_SIGN = 0, SGKS_SKETCH_GAUSSIAN = 1, SGKS_SKETCH_SRTT = 2 };
enum { SGKS_PREC_FP64 = 0, SGKS_PREC_FP32 = 1, SGKS_PREC_FP32X = 2, SGKS_PREC_FP32_PLAIN = 3, SGKS_PREC_FF = 4 };
enum { SGKS_FLAG_GLOBAL_SMALL = 1, SGKS_FLAG_RECORD = 2, SGKS_FLAG_GKS = 4, SGKS_FLAG_AUTOTUNE = 8,
       SGKS_FLAG_NO_TILES = 16, SGKS_FLAG_BW_HOST = 32 };

/* Forward operator A (m x n).
 *  SGKS_OP_CSR:    row_ptr[m+1], col[nnz] (int32, 0-based), val[nnz] of val_dtype.  Optional
 *                  transpose (the same matrix stored by columns): t_row_ptr[n+1], t_col[nnz]
 *                  (row indices of A, ascending within each column), t_val[nnz]; if all three
 *                  are NULL the library builds it on the device at sgks_create.
 *  SGKS_OP_DENSE:  dense[m*ld], row-major, ld >= n, of val_dtype.
 *  SGKS_OP_CONV2D: 2D convolution of an ny x nx image with the odd-sized kernel psf[kh*kw]
 *                  (row-major, val_dtype), zero boundary, same-size output (m = n = nx*ny):
 *                  (A x)[i,j] = sum_{a,c} psf[a*kw+c] * x[(i-a+kh/2)*nx + (j-c+kw/2)].
 * Values are converted to the solver precision on the device (FP32 form: rounded to float;
 * FP64 form: float values are widened exactly). */
typedef struct sgks_op {
    int32_t kind;
    int32_t val_dtype;
    int64_t m, n;
    int64_t nnz;
    const int32_t* row_ptr;
    const int32_t* col;
    const void* val;
    const int32_t* t_row_ptr;
    const int32_t* t_col;
    const void* t_val;
    const void* dense;
    int64_t ld;
    int32_t nx, ny, kh, kw;
    const void* psf;
} sgks_op;

/* Regularization operator L (p x n), a matrix-free finite-difference stencil.
 *  SGKS_REG_FD1:       D_n (rows [-1 1]), n = nx, p = nx-1               (Sec. 4, eq. reg_matrix)
 *  SGKS_REG_GRAD2D:    [I_ny (x) D_nx ; D_ny (x) I_nx], p = ny(nx-1)+(ny-1)nx (eq. reg_matrix)
 *  SGKS_REG_LAPLACE2D: 5-point Laplacian 4x_p - sum of the 4 neighbours, zero outside, p = nx ny
 *  SGKS_REG_SPACETIME: Psi of eq. spacetime_tik (Sec. 4.3), nt frames of ny x nx,
 *                      p = nt(ny(nx-1)+(ny-1)nx) + (nt-1)nx ny */
typedef struct sgks_reg {
    int32_t kind;
    int32_t nx, ny, nt;
} sgks_reg;

/* Options.  Zero-initialised fields take the defaults in brackets. */
typedef struct sgks_options {
    int32_t max_iters;    /* maximum number of appended columns; sizes W: d_max = ell + max_iters [100] */
    int32_t ell;          /* dimension of the initial Krylov basis W_0 [3]                          */
    int32_t n_refine;     /* refinement steps of the projected solve per iteration [0]              */
    int32_t precision;    /* SGKS_PREC_FP64: everything FP64.
                             SGKS_PREC_FP32: the basis W, the operator values and b in FP32;
                             the new column's A w and L w (the input of the sketched QR update),
                             x = W y, e = A W y - b and the gradient (basis column and refinement
                             residual) accumulated in compensated float-float arithmetic
                             (TwoProd/TwoSum, Dot2) on the FP32 units, A W, x and e kept as
                             float-float pairs; FP64 sketched QR, projected solve and refinement
                             solve.  Iterates stay within the FP32-storage floor of the FP64
                             ones.  SGKS_FLAG_GKS and SGKS_FLAG_RECORD run this form with the
                             FP32-accumulation kernels of SGKS_PREC_FP32_PLAIN.
                             SGKS_PREC_FP32X: the same form as SGKS_PREC_FP32.
                             SGKS_PREC_FP32_PLAIN: FP32 operators, sketch, W, A W, x and e with
                             FP32 accumulation; FP64 sketched QR, projected solve and refinement
                             reductions (its iterates drift from the FP64 ones once the basis
                             fills up).
                             SGKS_PREC_FF (batches only): the basis and every vector as
                             float-float pairs, compensated arithmetic on the FP32 units, FP64
                             small phase: FP64-class results (48-bit significand, FP32 exponent
                             range) at FP32-unit speed.
                             b, x_true and x_out are FP64 for FP64 and FF, FP32 otherwise; for
                             SGKS_PREC_FP32 sgks_get_buffer(SGKS_BUF_X / SGKS_BUF_AW) returns
                             (hi, lo) float pairs [FP64]                                         */
    int32_t sketch_kind;  /* SGKS_SKETCH_SPARSE_SIGN, SGKS_SKETCH_GAUSSIAN or SGKS_SKETCH_SRTT
                             (eq. sketching_trig: S = sqrt(h/s) D F E, F the orthonormal DCT-II;
                             built as a dense FP64 matrix on the device at create) [sparse-sign] */
    int32_t zeta;         /* nonzeros per sketch column, 1..16, <= sketch_rows [8]                  */
    int32_t cgs_passes;   /* 1 = the single projection printed under eq. updqr, 2 = CGS2 [2]       */
    int32_t flags;        /* bit 0 (SGKS_FLAG_GLOBAL_SMALL): run the FP64 QR append and projected
                             solve with the global-memory kernels instead of the on-chip cluster
                             kernels (chosen automatically when the on-chip slices do not fit).
                             bit 1 (SGKS_FLAG_RECORD): keep y_k of every iteration (and the
                             y after each refinement step) so that sgks_backward can
                             differentiate the solve; needs precision FP64 or FP32 and the
                             on-chip kernels.
                             bit 2 (SGKS_FLAG_GKS): run GKS (Algorithm 1) instead: orthonormal
                             basis V_k (gradient column orthogonalised, a second pass when the
                             loss ratio of eq. loss_criterion is >= 1e-10, normalised), full-size
                             thin QR factors of A V_k and L V_k updated by CGS2 (eq. updqr with
                             S = I), projected problem eq. projected_withQR.  The sketch options
                             are ignored; needs n_refine = 0, FP64 or FP32, ell + max_iters <=
                             1024; sgks_solve's tol applies the relative-change test of eq. RC.
                             bit 3 (SGKS_FLAG_AUTOTUNE, batches only): after the setup, time the
                             candidate tile choices of each group on its own data and keep the
                             fastest (bulk-copy slice 8 or 16 KB; lanes per CSR row of A and A^T;
                             instances per CTA of the tiled forward pass, the default or twice it),
                             a candidate replacing the default only when at least 5% faster;
                             results are cached per shape for the process.  Without it the
                             defaults are used (16 KB, 8, 8; 8 float-float or 16 FP32 instances
                             per tile CTA) and results are reproducible from run to run; the slice
                             and the tile instances keep every sum's order, the lanes per CSR row
                             change it (at the level of rounding).
                             bit 4 (SGKS_FLAG_NO_TILES, batches only): the compensated forms
                             (FP32, FF) compute A w of a CSR operator whose regularizer gives an
                             image geometry (2D stencils, space-time) through pixel tiles: each
                             tile of w is staged once in shared memory and the rays crossing it
                             leave one partial sum per (ray, tile), summed per ray in entry
                             order.  This flag keeps the CSR-row kernel instead.
                             bit 5 (SGKS_FLAG_BW_HOST, with SGKS_FLAG_RECORD): sgks_backward keeps
                             the adjoint of the basis (d_max x n values, the sweep's largest
                             array, as large as W itself) in pinned host memory mapped into the
                             device's address space, reached over the CPU-GPU link, for when the
                             device memory cannot hold a second basis-sized array; the result is
                             the same, bit for bit, as with device memory [0] */
    const double* gauss_SA; /* Gaussian sketch only: S_A, sketch_rows x m, row-major, FP64, device */
    const double* gauss_SL; /* Gaussian sketch only: S_L, sketch_rows x p, row-major, FP64, device */
    const void* x_true;     /* optional, n values of the solver precision: enables RRE records    */
    const int8_t* srtt_signs_A;  /* SRTT only (device): the Rademacher diagonal E of S_A, m entries +-1 */
    const int32_t* srtt_rows_A;  /* SRTT only (device): the s sampled rows D of S_A, in [0, m)         */
    const int8_t* srtt_signs_L;  /* SRTT only: E of S_L, p entries                                      */
    const int32_t* srtt_rows_L;  /* SRTT only: the s rows of S_L, in [0, p)                            */
} sgks_options;

/* Per-solve report (host memory).  rc / rre may be NULL; otherwise they receive one value per
 * iteration performed (index k-1 for iteration k): RC_k = ||x_k - x_{k-1}|| / ||x_{k-1}||
 * (eq. RC) and RRE_k = ||x_k - x_true|| / ||x_true|| (Sec. 4, needs opt.x_true). */
typedef struct sgks_report {
    int32_t iters_done;   /* iterations performed by this call                          */
    int32_t status;       /* SGKS_OK, SGKS_STOPPED, SGKS_BREAKDOWN or an error code     */
    int32_t subspace_dim; /* current d = ell + appended columns                         */
    int32_t reserved;
    double rc_last;
    double rre_last;      /* NaN if x_true was not given                                */
    double rre0;          /* RRE of x_0 (initial subspace)                              */
    double* rc;           /* host array of >= iters entries, or NULL                    */
    double* rre;          /* host array of >= iters entries, or NULL                    */
} sgks_report;

typedef struct sgks_handle sgks_handle;

/* Create a solver and run the setup (Algorithm 2 inputs, Sec. 4: W_0 = orthonormal basis of
 * K_l(A^T A, A^T b); S_A b; sketched QR of W_0; y_0; x_0).
 *  A, L:        descriptors as above (arrays: device, caller-owned, must outlive the handle).
 *  b:           m values of the solver precision (device).
 *  lambda:      regularization parameter, > 0 (eq. tik).
 *  sketch_rows: s = s_A = s_L, ell + max_iters <= s <= 2048 (Sec. 4: a small multiple of the
 *               maximum subspace dimension).
 *  seed:        seed of the sparse-sign sketches (S_A: stream 0, S_L: stream 1).
 *  opt:         options (host pointer, may be NULL for defaults).
 *  stream:      cudaStream_t (as void*) on which all work of the handle runs.
 * On success *h receives the handle (owned by the caller; release with sgks_destroy).
 * Errors: SGKS_ERR_INVALID (sizes, kinds, lambda <= 0, s out of range, zeta out of range,
 * CSR row_ptr not starting at 0 / not ending at nnz), SGKS_ERR_NOMEM, SGKS_ERR_CUDA. */
int sgks_create(sgks_handle** h, const sgks_op* A, const sgks_reg* L, const void* b,
                double lambda, int32_t sketch_rows, uint64_t seed, const sgks_options* opt,
                void* stream);

/* Re-run the setup for a new right-hand side b_new (device, m values of the solver precision;
 * may equal the previous pointer).  Operator preprocessing (transpose, conversions) and the
 * workspace are reused; the basis is discarded.  Asynchronous on the handle's stream. */
int sgks_reset(sgks_handle* h, const void* b_new);

/* One sGKS iteration (Algorithm 2, one pass of the loop): r_k from x_{k-1} (eq. gradient),
 * W_k = [W_{k-1}, r_k], sketch S_A A r_k and S_L L r_k, rank-one QR appends (eq. updqr) and
 * the d_A entry (eq. dA_update), y_k (eq. projected_sketched_bis), n_refine refinement steps,
 * x_k = W_k y_k, RC_k.  Asynchronous; returns SGKS_ERR_STATE if the basis is full.  Device
 * status (breakdown, non-finite values) is read by sgks_status. */
int sgks_step(sgks_handle* h);

/* Run `iters` iterations (replaying a captured CUDA graph of sgks_step), optionally stopping
 * when RC_k < tol (tol > 0; eq. RC), then copy x_k to x_out (device, n values of the solver
 * precision; NULL = do not copy) and fill *rep (host, may be NULL).  Synchronises the stream. */
int sgks_solve(sgks_handle* h, int32_t iters, double tol, void* x_out, sgks_report* rep);

/* Synchronise and read the device status word into *code (SGKS_OK, SGKS_BREAKDOWN,
 * SGKS_STOPPED, SGKS_ERR_NONFINITE or SGKS_ERR_SKETCH).  Returns SGKS_OK or an error. */
int sgks_status(sgks_handle* h, int32_t* code);

/* Human-readable description of the last error of h (or of the last failed sgks_create when h
 * is NULL).  The string is owned by the library and valid until the next call on h. */
const char* sgks_last_error(const sgks_handle* h);

/* Release handle-owned device memory and the captured graph.  NULL-safe.  Synchronises. */
void sgks_destroy(sgks_handle* h);

/* ---- inspection and building blocks (used by the parity tests) ------------------------- */

enum {
    SGKS_BUF_X = 1,     /* x_k (n, solver precision)                                         */
    SGKS_BUF_Y = 2,     /* y_k (d, FP64)                                                     */
    SGKS_BUF_W = 3,     /* W column-major (d columns of n values, solver precision)          */
    SGKS_BUF_QA = 4,    /* Q_A column-major (d columns of s, FP64)                           */
    SGKS_BUF_RA = 5,    /* R_A column-major, leading dimension d_max (FP64)                  */
    SGKS_BUF_QL = 6,
    SGKS_BUF_RL = 7,
    SGKS_BUF_DA = 8,    /* d_A (d, FP64)                                                     */
    SGKS_BUF_SB = 9,    /* S_A b (s, FP64)                                                   */
    SGKS_BUF_T = 10,    /* stacked triangular factor T, column-major, leading dim d_max      */
    SGKS_BUF_AW = 11    /* A W column-major (d columns of m values, solver precision)        */
};

/* Copy an internal buffer to dst (device) after synchronising; `bytes` is the capacity of
 * dst.  Writes the number of bytes copied to *copied.  Returns SGKS_ERR_INVALID if the buffer
 * id is unknown or dst is too small. */
int sgks_get_buffer(sgks_handle* h, int32_t which, void* dst, size_t bytes, size_t* copied);

/* Scalar state: out[0] = d (subspace dimension), out[1] = iterations done since the setup,
 * out[2] = device status code.  Host pointer, 3 entries.  Synchronises. */
int sgks_get_info(sgks_handle* h, int64_t* out);

enum { SGKS_APPLY_A = 1, SGKS_APPLY_AT = 2, SGKS_APPLY_L = 3, SGKS_APPLY_LT = 4,
       SGKS_APPLY_LTL = 5, SGKS_APPLY_SA = 6, SGKS_APPLY_SL = 7 };

/* Apply one operator of the handle: A (n -> m), A^T (m -> n), L (n -> p), L^T (p -> n),
 * L^T L (n -> n, the fused stencil used inside the gradient) in the solver precision, or a
 * sketch S_A (m -> s) / S_L (p -> s) with FP64 output.  in/out are device arrays of the sizes
 * stated; asynchronous on the handle's stream. */
int sgks_apply(sgks_handle* h, int32_t which, const void* in, void* out);

/* Sparse-sign sketch positions (paper Sec. 2.2 allows any oblivious embedding; this one is
 * defined here): for column j < h_cols, draws c = 0, 1, ... hash
 * hv = mix64(mix64(2*seed + stream) ^ (j*256 + c)) with mix64 the SplitMix64 finalizer,
 * row = ((hv >> 32) * s) >> 32, negative sign iff hv is odd; a repeated row is rejected.
 * Writes rows_out[j*zeta + k] (int32, device) and neg_out[j*zeta + k] (uint8 0/1, device) for
 * the k-th accepted draw.  Returns SGKS_ERR_SKETCH if some column needs more than 256 draws.
 * Synchronises `stream`. */
int sgks_sparse_sign_rows(uint64_t seed, int32_t stream_id, int64_t h_cols, int32_t s,
                          int32_t zeta, int32_t* rows_out, uint8_t* neg_out, void* stream);

/* Build the transpose of a CSR matrix on the device: the column-major storage of A, with
 * row indices ascending within each column (deterministic).  Inputs row_ptr[m+1], col[nnz],
 * val[nnz] (val_dtype); outputs t_row_ptr[n+1], t_col[nnz], t_val[nnz] (same dtype), all
 * device, caller-allocated.  Preconditions: 0 = row_ptr[0] <= row_ptr[1] <= ... <= row_ptr[m]
 * = nnz and every col[k] in [0, n).  Entries that break them are skipped by the kernels (nothing
 * is written outside the output and temporary arrays) and the call returns SGKS_ERR_INVALID;
 * the output is then not a transpose.  Temporary device memory is allocated and freed inside.
 * Synchronises `stream`. */
int sgks_csr_transpose(int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr,
                       const int32_t* col, const void* val, int32_t val_dtype,
                       int32_t* t_row_ptr, int32_t* t_col, void* t_val, void* stream);

/* The same CSR transpose, same arguments and the same output bit for bit, but without
 * allocating device memory: no cudaMalloc, cudaMallocAsync or cudaFree.  The paper has no
 * counterpart; this is for callers that cannot allocate.  One case is a process where another
 * allocator, such as a framework's caching allocator, has already reserved the device memory.
 * Another is a service that fixes its memory plan at start-up and must not have an allocation
 * fail or stall in the middle of a request.
 *
 * Its temporaries live in a fixed scratch array of 16 MiB (16,777,216 bytes) inside the
 * library.  With CUDA's lazy module loading the array is reserved on a device the first time
 * the library's kernels are used there, which may be this call: if the device memory is
 * already full that first use returns an allocation error (SGKS_ERR_CUDA), so make one warm-up
 * call at start-up, while memory is still free.  From then on the device holds the array until
 * the process exits.  The
 * array must hold 4*(n+1) + 4*nnz + es*nnz bytes, each of the three parts rounded up to 256
 * bytes, where es = 4 for SGKS_F32 values and 8 for SGKS_F64.  For example, n = 65,536 with
 * FP32 values fits nnz up to about 2.06 million.  Larger sizes return SGKS_ERR_INVALID, with
 * the sizes in sgks_last_error(NULL); use sgks_csr_transpose for those.
 *
 * The preconditions on row_ptr and col are those of sgks_csr_transpose, with the same
 * SGKS_ERR_INVALID when they do not hold (the error flag is a second, 4-byte array of the
 * library, so a malformed input cannot write into the scratch's neighbours).
 *
 * The first call on a device looks up the array's device address on the current device, which
 * must be the device of `stream` and of the buffers.  Make that first call before any stream
 * capture.  All calls share the one array, and each call overwrites what the previous one left
 * there.  Calls that overlap on the GPU (different streams, or host threads, at the same time)
 * race on it and give wrong results.  The call synchronises `stream` before it returns, so
 * calls made one after another from one thread are safe. */
int sgks_csr_transpose_noalloc(int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr,
                               const int32_t* col, const void* val, int32_t val_dtype,
                               int32_t* t_row_ptr, int32_t* t_col, void* t_val, void* stream);

/* Number of kernel launches the library has enqueued in this process so far (host-side count;
 * one replay of the captured step graph counts its kernel nodes). */
int64_t sgks_kernel_launches(void);

/* Per-kernel timing: run `iters` iterations (as sgks_step, without the graph) with a CUDA event
 * pair on the handle's stream around every kernel launch; each launch is synchronised, so the
 * call is for measurement only.  Host arrays of SGKS_PROFILE_CLASSES entries receive per kernel
 * class the total milliseconds, the number of launches and the sum over launches of the
 * subspace size d at launch (for per-launch byte models).  Classes:
 *   0 gradient -> new basis column   1 operator apply + sketch   2 sketched QR appends (K2)
 *   3 stacked QR + projected solve (K3; with SGKS_FLAG_GLOBAL_SMALL: K2 and K3 in one kernel)
 *   4 combine inside refinement      5 gradient + W^T r          6 refinement solve
 *   7 combine at the end of the iteration (x_k, e_k, RC, RRE) */
#define SGKS_PROFILE_CLASSES 8
int sgks_profile_steps(sgks_handle* h, int32_t iters, double* ms_out, int64_t* count_out, double* dsum_out);

/* The same per-class totals measured inside a CUDA graph: `iters` iterations are captured into
 * one graph with an event pair recorded as graph nodes around every kernel launch, the graph
 * is launched once, and each launch's time is the elapsed time of its pair.  Launches then
 * follow each other as in sgks_solve (no host round trip between kernels).  The iterations
 * count against the basis capacity like sgks_step.  Returns SGKS_ERR_STATE after
 * sgks_set_lambda without sgks_reset, SGKS_ERR_CUDA on a CUDA error. */
int sgks_profile_graph(sgks_handle* h, int32_t iters, double* ms_out, int64_t* count_out, double* dsum_out);

/* Average device time of one launch of a streaming kernel class in the handle's current state,
 * without per-launch events: `reps` launches are captured back to back into one CUDA graph,
 * which is launched once to warm up and once between two CUDA events on the handle's stream;
 * *us_out = elapsed microseconds / reps.  Classes (as sgks_profile_steps): 0 gradient -> next
 * basis column, 1 operator apply + sketch of the next column, 4 combine inside refinement,
 * 5 refinement gradient + W^T r.  These kernels write only the not-yet-appended column d,
 * scratch and the refinement's x, e and partials, which the next step recomputes, so the
 * iteration state is unchanged.  SGKS_ERR_INVALID for another class, for reps < 1 and for the
 * fp32x and GKS forms; SGKS_ERR_STATE after sgks_set_lambda without sgks_reset. */
int sgks_time_class(sgks_handle* h, int32_t cls, int32_t reps, double* us_out);

/* ---- differentiation ------------------------------------------------------------------- */
/* Reverse-mode derivative of the solve: for the x_K that the iterations since the last setup
 * (sgks_create / sgks_reset) produced, and xbar = dl/dx_K (device, n values of the solver
 * precision), write bbar = dl/db (device, m values of the solver precision) and *lambda_bar =
 * dl/dlambda (host).  This is the exact derivative of the map (b, lambda) -> x_K of Algorithm 2
 * with the handle's n_refine q = 0 refinement steps per iteration (Sec. 3.1: y^r = y^{r-1} -
 * G_k^{-1} W_k^T rho(W_k y^{r-1}), G_k = U_k^T U_k + lambda V_k^T V_k, rho the residual of the
 * normal equations), x_K = W_K y_K with every basis column r_j = A^T (A x_{j-1} - b) +
 * lambda L^T L x_{j-1} depending on the earlier iterates (eq. gradient) and W_0 spanning
 * K_l(A^T A, A^T b).  It is computed by a reverse sweep over the iterations that reuses the
 * stored basis W and the stored inverse of the stacked triangular factor of
 * eq. (projected_sketched_bis) (the leading block of which serves every earlier step, since the
 * factors only grow by columns, eq. updqr).  Needs a handle created with SGKS_FLAG_RECORD.  The
 * forward state is unchanged, so the call may be repeated.  Device scratch is allocated at the
 * first call.  Calls with the same K and lambda as the previous one capture the sweep's launches
 * into a CUDA graph (second call) and then replay it; the results are bit-identical to the
 * eager sweep.  Synchronises.  Errors: SGKS_ERR_STATE (no SGKS_FLAG_RECORD, or no iteration
 * recorded), SGKS_ERR_INVALID, SGKS_ERR_CUDA. */
int sgks_backward(sgks_handle* h, const void* xbar, void* bbar, double* lambda_bar);

/* Change lambda (> 0) of a handle.  The basis is discarded: call sgks_reset before the next
 * step or solve.  Synchronises. */
int sgks_set_lambda(sgks_handle* h, double lambda);

/* ---- batches: many independent problems in one handle ----------------------------------- */
/* Each instance i is a problem of its own (eq. tik with A_i, L_i, b_i, lambda_i) solved by
 * Algorithm 2 exactly as a single handle would solve it, with the same seed: the batch changes
 * the schedule, not the arithmetic of an instance.  Instances whose A and L descriptors are equal
 * field by field (the same device arrays) form groups that share the prepared operator and run
 * in one instance-interleaved pass over A per kernel; the group size is a power of two <= 256, a
 * larger set of equal instances is split (largest power of two first), and instances with
 * different operators (ragged sizes) form separate groups that run concurrently. */
typedef struct sgks_batch sgks_batch;

/* Create a batch of `count` instances and run the setup of each (as sgks_create).
 *  A, L:     host arrays of `count` descriptors (their device arrays as for sgks_create).
 *  b:        host array of `count` device pointers, b[i] holding m_i values of the solver
 *            precision.  Copied at create and at sgks_batch_reset.
 *  lambdas:  host array of `count` parameters, each > 0.
 *  x_true:   NULL, or a host array of `count` device pointers (n_i values each): RRE records.
 *  sketch_rows, seed, opt: as for sgks_create, shared by every instance; opt->x_true is ignored.
 *            Supported: precision SGKS_PREC_FP64, SGKS_PREC_FP32 (= SGKS_PREC_FP32X),
 *            SGKS_PREC_FP32_PLAIN or SGKS_PREC_FF; the sparse-sign sketch.
 * Errors as for sgks_create; SGKS_ERR_INVALID names the first bad instance. */
int sgks_batch_create(sgks_batch** h, int32_t count, const sgks_op* A, const sgks_reg* L,
                      const void* const* b, const double* lambdas, const void* const* x_true,
                      int32_t sketch_rows, uint64_t seed, const sgks_options* opt, void* stream);

/* Re-run the setup of every instance with new right-hand sides (host array of `count` device
 * pointers).  Asynchronous on the handle's stream. */
int sgks_batch_reset(sgks_batch* h, const void* const* b_new);

/* One iteration of every live instance (as sgks_step).  Asynchronous. */
int sgks_batch_step(sgks_batch* h);

/* Run `iters` iterations of every instance by replaying one captured graph, an instance leaving
 * the loop on its own when its RC_k < tol (tol > 0) or on breakdown / non-finite values.
 *  x_out: NULL, or a host array of `count` device pointers (NULL entries skipped) receiving x_k.
 *  reps:  NULL, or a host array of `count` reports (rc / rre pointers inside as for sgks_solve).
 * Synchronises.  Returns the most severe negative instance status, else SGKS_OK. */
int sgks_batch_solve(sgks_batch* h, int32_t iters, double tol, void* const* x_out, sgks_report* reps);

/* Copy the current iterate x_k of every instance to x_out (host array of `count` device
 * pointers, NULL entries skipped; n_i values of the solver precision each).  Synchronises. */
int sgks_batch_get_x(sgks_batch* h, void* const* x_out);

/* Synchronise and write each instance's status code (as sgks_status) to codes[count] (host). */
int sgks_batch_status(sgks_batch* h, int32_t* codes);

/* Number of groups; optionally the group index and group size of every instance (host arrays of
 * `count` entries, may be NULL). */
int sgks_batch_layout(sgks_batch* h, int32_t* group_of, int32_t* group_size);

/* Per-kernel timing of `iters` eager iterations of every group (groups one after another, each
 * launch timed with a CUDA event pair and synchronised: for measurement only).  Host arrays of
 * SGKS_BATCH_PROFILE_CLASSES entries receive the total milliseconds and the launch count per
 * kernel class: the classes of sgks_profile_steps, except that class 1 is the operator apply
 * alone (A w through pixel tiles: the tile pass and the per-ray sums), class 8 the sketch gather
 * (S_A A w) and class 9 S_L L w (L w formed and sketched in column chunks, never stored). */
#define SGKS_BATCH_PROFILE_CLASSES 10
int sgks_batch_profile_steps(sgks_batch* h, int32_t iters, double* ms_out, int64_t* count_out);

/* Description of the tile configuration of group `group` chosen by SGKS_FLAG_AUTOTUNE ("" when
 * the group was not tuned).  Owned by the handle. */
const char* sgks_batch_config(const sgks_batch* h, int32_t group);

/* Last error of h, or of the last failed sgks_batch_create when h is NULL. */
const char* sgks_batch_last_error(const sgks_batch* h);

/* Release the batch's device memory, streams and graph.  NULL-safe.  Synchronises. */
void sgks_batch_destroy(sgks_batch* h);

#ifdef __cplusplus
}
#endif
#endif /* SGKS_H */
