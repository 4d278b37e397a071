/*
 * bgs.h - C ABI of the GB300 block Gauss-Seidel / SA-AMG / FGMRES solver (libbgs.so).
 *
 * The library solves A x = b for a coupled multi-field system given as an F x F grid of
 * CSR blocks (F <= 8).  It is the method of "Multi-physics Preconditioning for Thermally
 * Activated Batteries" (Phillips): flexible GMRES (Sec. 2.2, flexible GMRES) right-
 * preconditioned by one forward block Gauss-Seidel sweep over a permutation of the fields
 * (Sec. 2.2, Eqs. hierarchical-bgs, non-voltage-bgs, voltage-bgs), with one smoothed-
 * aggregation AMG V-cycle per diagonal block (Sec. 2.2.1, Eq. galerkin: Chebyshev smoothing,
 * filtered prolongator smoothing, Galerkin coarse operators, a direct coarsest solve).
 *
 * Conventions for every entry point:
 *  - Return value: a status code (BGS_OK = 0, see below).  No C++ exception crosses the ABI.
 *  - Pointers marked "host or device" may point to either, on the handle's stream: pinned host
 *    memory (16-byte aligned) is read or written by the library's kernels over the host link, other
 *    host memory and device memory are copied with cudaMemcpyAsync (cudaMemcpyDefault).  Pointers
 *    marked "device" must be device memory.
 *  - Vectors over all fields are field-blocked: x = [x_0; x_1; ...; x_{F-1}], x_k of length
 *    field_sizes[k].
 *  - CSR: rowptr has nrows+1 int32 entries starting at 0; col/val have nnz entries; within a
 *    row the columns are strictly increasing and in [0, ncols).  nnz < 2^31.
 *  - The caller keeps ownership of everything it passes; the library copies what it keeps.
 *  - One handle is used from one host thread at a time; all work goes to the handle's stream.
 */
#ifndef BGS_H
#define BGS_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define BGS_OK 0
#define BGS_INVALID_ARG 1     /* malformed CSR, bad order, missing diagonal, size mismatch */
#define BGS_NOT_SETUP 2       /* solve before setup */
#define BGS_NO_CONVERGENCE 3  /* maxit reached; x holds the last iterate, info is filled */
#define BGS_BREAKDOWN 4       /* Arnoldi breakdown without convergence */
#define BGS_NAN_INF 5         /* NaN or Inf in the input or in a residual norm */
#define BGS_ZERO_PIVOT 6      /* the coarsest-level LU met a zero pivot */
#define BGS_CUDA_ERROR 7      /* a CUDA call failed */
#define BGS_OOM 8             /* device allocation failed */
#define BGS_INTERNAL 9        /* an internal consistency check failed */

typedef struct bgs_ctx *bgs_handle;

/* One CSR block; pointers host or device.  nrows == 0 and nnz == 0 with NULL pointers
 * denotes a zero block. */
typedef struct {
    int64_t nrows, ncols, nnz;
    const int32_t *rowptr;
    const int32_t *col;
    const double *val;
} bgs_csr;

typedef struct {
    int restart;            /* FGMRES restart length m (Sec. 2.2; default 50) */
    int maxit;              /* total FGMRES iterations (default 1000) */
    double rtol;            /* stop when ||b - A x|| / ||b|| <= rtol, true residual (default 1e-8) */
    int precision;          /* 0: FP64 hierarchy; 1: FP32 hierarchy + BF16 coupling values */
    int graph;              /* 1 (default): replay the preconditioner sweep as a captured CUDA graph */
    int autotune;           /* 1 (default): pick the SpMV form per stored operator by timing at setup, in the
                               precision the solve uses: field-interleaved F x F node blocks (the full
                               operator of equal fields), SELL-32 with diagonal offsets (structured
                               operators), SELL-32, or CSR with 1..32 lanes per row, each at 128, 256 or
                               512 threads per block; choices are cached per process by operator shape,
                               and in the text file named by the environment variable BGS_AUTOTUNE_CACHE
                               when it is set (BGS_AUTOTUNE_LOG set: every candidate's time is printed
                               to stderr).  0: the diagonal-offset form where built, else SELL-32
                               where built, else CSR with a lane count fixed by the row length */
    int cheb_degree[8];     /* Chebyshev degree per field id (Sec. 2.2.1: 2; voltage blocks 4, Sec. 3.1.5) */
    double theta[8];        /* strength drop tolerance per field id (Sec. 3.1.4: 0.04 for phi_s) */
    int max_coarse;         /* stop coarsening at this many rows (default 500; the paper uses 5000 with
                               a sparse direct solver, Sec. 2.2.1; here the coarsest solve is dense) */
    int max_levels;         /* at most this many levels, 1..16 (default 10) */
    double cheb_ratio;      /* lambda_min = lambda_max / ratio (default 30) */
    double cheb_boost;      /* lambda_max = boost * power-iteration estimate (default 1.1) */
    int power_iters;        /* power iterations for the eigenvalue estimates (default 10) */
    int filter_diag;        /* smoothing diagonal of the filtered matrix: 1 absolute row sum
                               (Sec. 2.2.1), 0 its plain diagonal */
    double reorth_eta;      /* Arnoldi: second Gram-Schmidt pass when ||w1|| < reorth_eta ||w|| (more than
                               log10(1/eta) digits cancelled); default 0.01; 1 always (CGS2),
                               1/sqrt(2) the DGKS test, 0 never */
    int jacobi;             /* 0 (default): forward block Gauss-Seidel sweep; 1: block Jacobi, the
                               couplings left out (the alternative Secs. 3.2 and 4 discuss): the
                               per-block V-cycles are independent and run concurrently */
    int subsolver[8];       /* per field id, the diagonal-block solver of the sweep: 0 (default) one
                               SA-AMG V-cycle; 1 DD(0)-ILU(0), i.e. restricted additive Schwarz without
                               overlap over subdomains of ilu_rows consecutive rows, one ILU(0) sweep
                               per subdomain (Sec. 2.1, Eq. one-level-schwarz; the species solver of
                               Sec. 3.1.1); 2 the diagonal solve z = diag(A_kk)^-1 r, exact for a
                               diagonal block such as the solid species A_s that Sec. 2.2 inverts
                               directly (one Jacobi step for any other block) */
    int ilu_rows;           /* DD(0)-ILU(0) subdomain size in rows, 1..8192 (default 4096) */
    int ngroups;            /* 0 (default): one flat sweep over the fields.  > 0: the nested variant
                               (Sec. 2.2, Eq. hierarchical-bgs over groups of fields): group g is the
                               order positions [group_end[g-1], group_end[g]) (group_end[ngroups-1] =
                               nfields; a group's field ids must be consecutive); the preconditioner
                               sweeps over the groups and solves each group's diagonal block by an inner
                               FGMRES(inner_restart), preconditioned by the group's own sweep, to a
                               relative residual inner_rtol or inner_maxit iterations.  The outer FGMRES
                               uses restart (the paper's nested solver: restart 5, inner FGMRES(30) to
                               1e-6, groups [phi_s, phi_e] and [p, c1, c2]).  No CUDA graph. */
    int group_end[8];
    int inner_restart;      /* 1..63 (default 30) */
    int inner_maxit;        /* default 30 */
    double inner_rtol;      /* default 1e-6 */
    int cheb_ellipse;       /* 1: Chebyshev smoothing on an ellipse (the nonsymmetric form Sec. 2.2.1 cites):
                               per level the real extent of the interval and an imaginary semi-axis
                               boost * rho(S), S the skew part of D^-1/2 A D^-1/2 (Bendixson); a level
                               whose radius is below 1e-10 lambda_max keeps the interval.  Default 0 */
} bgs_options;

typedef struct {
    int iters;              /* FGMRES iterations (preconditioner applications) */
    int converged;          /* 1 if the true relative residual reached rtol */
    int status;             /* same as the return value */
    int restarts;
    int reorth;             /* Arnoldi steps that ran the second Gram-Schmidt pass */
    double rel_true_resid;  /* ||b - A x|| / ||b|| of the returned x, in FP64 */
    double rel_est_resid;   /* last Arnoldi residual estimate */
    double t_setup_ms;      /* wall time of the last bgs_setup or bgs_update_values */
    double t_solve_ms;      /* this solve's wall time */
    int nlevels[8];         /* hierarchy levels per field id (1 for a field on DD(0)-ILU(0) or the diagonal
                               solve); entries past nfields are 0 */
} bgs_info;

/* Fills *opt with the defaults listed above. */
int bgs_default_options(bgs_options *opt);

/* Builds the block operator (Sec. 2.2, Eq. block-splitting).
 *  field_sizes: F entries (host).  blocks: F*F row-major bgs_csr (host array; block (r, c) has
 *  field_sizes[r] rows and field_sizes[c] columns, or is a zero block).  Every diagonal block
 *  is non-empty, square and stores its diagonal.  order: F entries (host), a permutation of
 *  0..F-1: the sweep visits fields in this order.  opt: NULL for defaults.  cuda_stream: a
 *  cudaStream_t or NULL for the default stream.  The CSR arrays are copied (host or device).
 *  On success *out owns device memory until bgs_destroy. */
int bgs_create(bgs_handle *out, int nfields, const int64_t *field_sizes, const bgs_csr *blocks,
               const int *order, const bgs_options *opt, void *cuda_stream);

/* Builds the SA-AMG hierarchy of every diagonal block (Sec. 2.2.1): strength filter, MIS-2
 * aggregation, smoothed prolongator, Galerkin coarse operators, Chebyshev bounds, coarsest LU. */
int bgs_setup(bgs_handle h);

/* Numeric re-set-up after the blocks' values changed on unchanged patterns, as in the nonlinear
 * iterations of a simulation (Sec. 3.2 notes that the symbolic phase of a factorisation can be
 * recycled across them while the numeric phase is redone).  values[r*F + c] points to the new
 * nnz(r, c) values of block (r, c) in the order of its stored entries (host or device memory,
 * read before the call returns; the caller keeps ownership); NULL keeps that block's values.
 * Every level keeps the strength flags and aggregates of the last bgs_setup (so all patterns, SELL
 * layouts and tuned kernels stay); the full operator, the couplings, the filtered matrices,
 * omega, P, R, the Galerkin operators, the Chebyshev bounds and the coarsest inverse are
 * recomputed from the new values.  The result equals a fresh bgs_setup on the new values whenever
 * that would make the same strength and aggregation decisions.  Returns BGS_NOT_SETUP before the
 * first bgs_setup, BGS_INVALID_ARG for values == NULL, BGS_ZERO_PIVOT if the new coarsest operator
 * is singular.  Captured CUDA graphs are dropped (they are re-captured by the next solve). */
int bgs_update_values(bgs_handle h, const double *const *values);

/* Solves A x = b by FGMRES(m) with the block Gauss-Seidel preconditioner, x0 = 0.
 * b, x: host or device, length sum(field_sizes).  info may be NULL. */
int bgs_solve(bgs_handle h, const double *b, double *x, bgs_info *info);

/* Solves A^T lambda = g with the transposed preconditioner: the sweep in reverse order over the
 * transposed couplings, V-cycles on the transposed diagonal blocks (same transfers).  This is an
 * extension; the paper has no adjoint.  g, lambda: host or device. */
int bgs_solve_adjoint(bgs_handle h, const double *g, double *lambda, bgs_info *info);

/* Gradient of a scalar loss through the solve with respect to the stored values of block
 * (row_field, col_field): dvals[e] = -lambda_i * x_j for stored entry e = (i, j) (extension,
 * no counterpart in the paper).  lambda, x: device, full length; dvals: device, nnz of the block. */
int bgs_grad_values(bgs_handle h, int row_field, int col_field, const double *lambda, const double *x,
                    double *dvals);

/* The same gradient for every stored block at once: dvals[r*F + c] receives nnz(r, c) values for block
 * (r, c) (device pointers; NULL skips that block, and zero blocks are skipped).  lambda, x: device,
 * full length. */
int bgs_grad_values_all(bgs_handle h, const double *lambda, const double *x, double *const *dvals);

/* One application of the preconditioner z = M^-1 v (device pointers, full length): the block sweep,
 * or with ngroups > 0 the nested preconditioner (inner FGMRES solves per group). */
int bgs_apply_preconditioner(bgs_handle h, const double *v, double *z);

/* The block solver of field k applied to b: one V-cycle of its hierarchy from x = 0, x = V_k(b),
 * or the DD(0)-ILU(0) sweep when subsolver[k] = 1 (device pointers, field length). */
int bgs_apply_vcycle(bgs_handle h, int field, const double *b, double *x);

/* y = A x with the assembled FP64 operator (device pointers, full length). */
int bgs_full_spmv(bgs_handle h, const double *x, double *y);

/* Hierarchy introspection (host outputs; any pointer may be NULL).  Level 0 is the block. */
int bgs_num_levels(bgs_handle h, int field, int *nlevels);
int bgs_level_info(bgs_handle h, int field, int level, int64_t *rows, int64_t *nnz, int64_t *p_nnz,
                   int *nagg, int *mis_rounds, double *omega, double *lmin, double *lmax);
/* which: 0 level operator A_l, 1 prolongator P_l, 2 restriction R_l.  rowptr/col/val: host
 * arrays sized by bgs_level_info (rows+1 / nnz / nnz; P_l has rows(l) rows and nagg columns). */
int bgs_level_copy(bgs_handle h, int field, int level, int which, int32_t *rowptr, int32_t *col, double *val);
/* Imaginary semi-axis of the smoother's ellipse on a level (0: the real interval). */
int bgs_level_ellipse(bgs_handle h, int field, int level, double *imag);
/* DD(0)-ILU(0) factors of a field whose subsolver is 1: the subdomain-restricted pattern of A_kk with
 * L (unit diagonal, strictly lower, not stored) and U in place.  *nnz receives the entry count; rowptr
 * (rows + 1), col and val (nnz each) are filled when not NULL (host or device).  BGS_INVALID_ARG for
 * a field on the V-cycle. */
int bgs_ilu_factors(bgs_handle h, int field, int64_t *nnz, int32_t *rowptr, int32_t *col, double *val);
/* SpMV kernel used for A_l (which 0), P_l (1), R_l (2), or the full operator (which 3; field and level
 * ignored; available from bgs_create on, the others after bgs_setup): -2 = field-interleaved node
 * blocks (full operator of equal fields only), -1 = SELL-32 with one diagonal offset per slice slot
 * (structured operators), 0 = SELL-32, k > 0 = CSR with k threads per row (chosen by the autotuner
 * when it is on); *threads_per_block (may be NULL) receives the block size of its launches. */
int bgs_level_format(bgs_handle h, int field, int level, int which, int *format, int *threads_per_block);
/* Aggregate id of every node of level `level` (host array of rows(level) entries). */
int bgs_level_aggregates(bgs_handle h, int field, int level, int32_t *agg);
/* Strength decision of every stored entry of A_l (Sec. 2.2.1 drop tolerance: 1 strong, 0 weak or the
 * diagonal), in CSR order, from the aggregation attempt that was kept (host array of nnz(A_l) bytes;
 * levels below the coarsest). */
int bgs_level_strength(bgs_handle h, int field, int level, uint8_t *strong);

/* Per-kernel-class timing of the last solve when enabled (bgs_set_profiling(h, 1)): launches,
 * summed CUDA-event milliseconds and algorithmic bytes.  kernel_class: 0 full SpMV, 1 Chebyshev
 * step on the finest level, 2 Arnoldi orthogonalisation, 3 coupling SpMV, 4 Chebyshev steps on
 * the coarser levels, 5 DD(0)-ILU(0) sweeps (factors read twice).  Algorithmic bytes: matrix values + column indices + row pointers + each
 * vector read or written once. */
int bgs_set_profiling(bgs_handle h, int on);
int bgs_kernel_stats(bgs_handle h, int kernel_class, int64_t *launches, double *ms, double *bytes);

/* Stateless y = A x for a device CSR in FP64 (K1): the same SpMV kernel the solver uses.
 * lanes: threads per row (1, 2, 4, 8, 16 or 32), or 0 for the built-in choice. */
int bgs_csr_spmv(int64_t nrows, int64_t nnz, const int32_t *rowptr, const int32_t *col, const double *val,
                 const double *x, double *y, int lanes, void *cuda_stream);

/* Block dot products of one Arnoldi step (K14, Sec. 2.2 flexible GMRES orthogonalisation):
 * h[k] = V_k . w for k < cnt and h[cnt] = w . w.  V: device, column-major, vector k at V + k*ld,
 * ld even and >= n; w: device, n entries; V and w 16-byte aligned (the kernel reads pairs of doubles;
 * anything else returns BGS_INVALID_ARG before any GPU work); h: device, cnt + 1 entries;
 * 1 <= cnt <= 64.  Per-block
 * partial sums go through device scratch that the call allocates and frees on the stream
 * (stream-ordered).  The sums are taken in a fixed order (run-to-run reproducible). */
int bgs_arnoldi_dots(const double *V, int64_t ld, int cnt, const double *w, int64_t n, double *h,
                     void *cuda_stream);

/* One classical Gram-Schmidt pass of the FGMRES orthogonalisation exactly as the solver runs it
 * (K14, Sec. 2.2 flexible GMRES): h[k] = V_k . w for k < cnt and h[cnt] = w . w, then
 * w <- w - sum_k h[k] V_k in place and *nw = w . w after the update.  On GB300 the FP64 pipe alone
 * caps these passes below the HBM rate, so the solver splits the products: in the dots, vectors
 * 0..2 of every group of 8 in FP64 and 3..7 in exact fixed point on the integer pipes; in the
 * update, the even rows in FP64 and the odd rows in fixed point.  A fixed-point sum truncates each
 * basis entry to a multiple of 2^-62 and each entry of the other factor to 56 bits below the
 * largest exponent among those one accumulator sees, sums exactly and rounds once to FP64.  This
 * needs |V_ik| < 2, as for the solver's unit basis vectors: a larger, infinite or NaN entry makes
 * its vector's fixed-point dot NaN (and with it the whole update), and an infinite or NaN w makes
 * every fixed-point dot NaN.  V: device, column-major, vector k
 * at V + k*ld, ld even and >= n; w: device, n entries; V and w 16-byte aligned; h: device, cnt + 1
 * entries; nw: device, 1 entry; 1 <= cnt <= 64 (anything else returns BGS_INVALID_ARG before any
 * GPU work).  Scratch is allocated and freed on the stream (stream-ordered); results are
 * run-to-run reproducible. */
int bgs_gram_schmidt_pass(const double *V, int64_t ld, int cnt, double *w, int64_t n, double *h, double *nw,
                          void *cuda_stream);

/* bgs_arnoldi_dots without any device allocation (the paper has no counterpart: this is a
 * library convenience).  For callers that cannot allocate device memory when they need the dots:
 * applications whose device memory is fully pre-reserved by their own pool manager, and embedded or
 * real-time hosts that forbid allocation after start-up.  Same arguments, results and limits
 * as bgs_arnoldi_dots (1 <= cnt <= 64, ld even and >= n, V and w 16-byte aligned; anything else
 * returns BGS_INVALID_ARG before any GPU work).  The partial sums go to one fixed array of 248,064
 * bytes inside the library's device image, held by every GPU that loads the library until the
 * process exits; on a GPU with more multiprocessors the kernel uses fewer blocks, never more
 * scratch.  The first call on each device looks up that array's address (cudaGetSymbolAddress with
 * the device current); with lazy module loading (the CUDA default) that first lookup is also when
 * the driver loads this part of the library and sets the array aside, so make the first call on
 * each device at start-up, before any stream capture.  Later calls allocate nothing.  The address is
 * kept for the life of the process: after cudaDeviceReset on a device, do not call this entry point
 * again on that device.  All calls share the array: calls whose GPU work overlaps (different
 * streams, threads or processes sharing the context) race and give wrong results; serialise them. */
int bgs_arnoldi_dots_noalloc(const double *V, int64_t ld, int cnt, const double *w, int64_t n, double *h,
                             void *cuda_stream);

/* The library allocates device memory stream-ordered from its own pool on each device; freed
 * memory stays cached there for later handles.  This returns the cached memory of the current
 * device to the driver (it synchronises the device first). */
int bgs_release_cached_memory(void);

/* Number of kernels this library has launched in the process so far (all handles). */
int64_t bgs_launch_count(void);

void bgs_destroy(bgs_handle h);
const char *bgs_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif
