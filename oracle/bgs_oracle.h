/*
 * Plain FP64 CPU oracle of the block Gauss-Seidel / SA-AMG / FGMRES solve.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library: only the
 * tests, the smoke check and the benchmark's CPU-baseline leg load it.  It shares no
 * header, helper or kernel with the CUDA path.  Everything is unblocked and in the order
 * the method states it (compiled with -ffp-contract=off).  Loops over independent rows may
 * run on several host threads (each row's arithmetic is unchanged); sums over whole vectors
 * (inner products, norms) are taken in consecutive blocks of 4096 terms, each block left to
 * right, then the block sums left to right, so no result depends on the thread count.
 *
 * What each part follows (paper sections and equations):
 *   strength / filter / aggregation / prolongator / Galerkin RAP  - Sec. 2.2.1, Eq. galerkin
 *   Chebyshev smoother, V-cycle, coarse direct solve              - Sec. 2.2.1
 *   block Gauss-Seidel sweep                                      - Sec. 2.2, Eqs. hierarchical-bgs,
 *                                                                   non-voltage-bgs, voltage-bgs
 *   flexible GMRES (right preconditioned, restarted)              - Sec. 2.2 (flexible GMRES)
 *   numeric re-set-up with the aggregation kept                    - Sec. 3.2 (symbolic reuse)
 *   DD(0)-ILU(0) subblock solver                                  - Sec. 2.1, Eq. one-level-schwarz;
 *                                                                   Sec. 3.1.1
 * The paper leaves the aggregation rule, the strength measure, eigenvalue estimation and
 * the filtered-diagonal form to the library it configures; the readings taken here are
 * spelled out next to each function in bgs_oracle.c.
 */
#ifndef BGS_ORACLE_H
#define BGS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n, m;          /* rows, columns */
    int nnz;
    int *rp, *ci;      /* row pointer (n+1), column index (nnz), rows sorted */
    double *v;         /* values (nnz) */
} or_csr;

typedef struct {
    int restart, maxit;
    double rtol;
    int cheb_degree[8];     /* per field id */
    double theta[8];        /* strength threshold per field id */
    int max_coarse, max_levels;
    double cheb_ratio, cheb_boost;
    int power_iters;
    int filter_diag;        /* 0: diag(A_F) ; 1: absolute row sum of A_F */
    int jacobi;             /* 1: block Jacobi (couplings left out of the sweep) */
    int subsolver[8];       /* per field id: 0 SA-AMG V-cycle, 1 DD(0)-ILU(0), 2 diagonal solve */
    int ilu_rows;           /* DD(0)-ILU(0) subdomain size in rows */
    int ngroups;            /* > 0: nested variant with groups [group_end[g-1], group_end[g]) of order positions */
    int group_end[8];
    int inner_restart, inner_maxit;
    double inner_rtol;      /* inner FGMRES relative tolerance per group solve */
    int cheb_ellipse;       /* 1: Chebyshev on an ellipse with a Bendixson imaginary extent */
} or_options;

typedef struct {
    int iters, converged, status;
    double rel_true_resid;
    double rel_est_resid;
} or_info;

/* host threads for the row loops (n <= 0: keep); returns the count in use */
int or_set_threads(int n);
/* sum_i a_i b_i in the fixed block order every whole-vector sum of the oracle uses */
double or_sum_prod(int n, const double *a, const double *b);

#define OR_MAX_LEVELS 16

typedef struct {
    int nlevels;                    /* levels 0..nlevels-1, last is the dense-LU level */
    or_csr *A[OR_MAX_LEVELS];       /* level operators */
    or_csr *P[OR_MAX_LEVELS];       /* prolongator level l -> from level l+1 */
    or_csr *R[OR_MAX_LEVELS];       /* restriction = P^T */
    int *agg[OR_MAX_LEVELS];        /* aggregate id per node of level l */
    unsigned char *strong[OR_MAX_LEVELS]; /* strength flag per stored entry of A_l (last attempt) */
    int nagg[OR_MAX_LEVELS];
    int mis_rounds[OR_MAX_LEVELS];
    double omega[OR_MAX_LEVELS];    /* prolongator damping */
    double *dinv[OR_MAX_LEVELS];    /* 1/diag(A_l) */
    double lmax[OR_MAX_LEVELS], lmin[OR_MAX_LEVELS];
    double lim[OR_MAX_LEVELS];       /* imaginary semi-axis of the smoother's ellipse (0: interval) */
    int degree;
    int nc;                          /* coarsest size */
    double *lu;                      /* dense LU of the coarsest, row-major */
    int *piv;
    int status;
} or_amg;

typedef struct {
    int rows;          /* subdomain size: rows [s*rows, (s+1)*rows) */
    or_csr *F;         /* subdomain-restricted pattern; L (unit, strictly lower) and U in place */
    int status;
} or_ilu;

typedef struct {
    int F;
    int sizes[8], offs[9];
    int order[8], pos[8];
    or_csr *blk[64];        /* F*F, NULL = zero */
    or_csr *full;           /* assembled full operator, field-blocked */
    or_amg *amg[8];
    or_ilu *ilu[8];         /* DD(0)-ILU(0) fields (amg[k] NULL there) */
    double *dgs[8];         /* diagonal-solve fields: 1 / diag(A_kk) (amg[k] NULL there) */
    or_options opt;
    int status;
} or_bgs;

/* CSR helpers */
or_csr *or_csr_new(int n, int m, int nnz);
or_csr *or_csr_from(int n, int m, const int *rp, const int *ci, const double *v);
void or_csr_free(or_csr *A);
void or_csr_info(const or_csr *A, int *n, int *m, int *nnz);
void or_csr_copy(const or_csr *A, int *rp, int *ci, double *v);
void or_spmv(const or_csr *A, const double *x, double *y);
or_csr *or_transpose(const or_csr *A);
or_csr *or_spgemm(const or_csr *A, const or_csr *B);

/* AMG pieces */
uint32_t or_fmix32(uint32_t h);
void or_strength_flags(const or_csr *A, double theta, unsigned char *strong);
or_csr *or_strength_graph(const or_csr *A, const unsigned char *strong);
int or_mis2(const or_csr *S, uint32_t salt, int *state);
int or_aggregate(const or_csr *S, const int *state, int *agg);
void or_filter(const or_csr *A, const unsigned char *strong, int filter_diag, double *vF, double *dF);
double or_power_lambda(const or_csr *A, const double *dinv, int iters);
or_csr *or_smooth_prolongator(const or_csr *AF, const double *dinvF, const int *agg, int nagg, double omega);
void or_chebyshev(const or_csr *A, const double *dinv, double lmin, double lmax, int deg,
                  const double *b, double *x, int x_is_zero);
double or_skew_radius(const or_csr *A, int iters);
void or_chebyshev_ellipse(const or_csr *A, const double *dinv, double theta, double c2, int deg,
                          const double *b, double *x, int x_is_zero);
int or_lu_factor(int n, double *a, int *piv);
void or_lu_solve(int n, const double *lu, const int *piv, const double *b, double *x);

or_amg *or_amg_setup(const or_csr *A, double theta, int degree, const or_options *opt);
void or_amg_free(or_amg *h);
int or_amg_update(or_amg *h, const double *v0, const or_options *opt);
void or_vcycle(const or_amg *h, const double *b, double *x);

/* DD(0)-ILU(0) */
or_ilu *or_ilu_setup(const or_csr *A, int rows);
int or_ilu_factor(or_ilu *m);
int or_ilu_update(or_ilu *m, const or_csr *A);
void or_ilu_apply(const or_ilu *m, const double *r, double *z);
void or_ilu_apply_transposed(const or_ilu *m, const double *r, double *z);
void or_ilu_free(or_ilu *m);

/* Block Gauss-Seidel and FGMRES */
void or_default_options(or_options *o);
or_bgs *or_bgs_create(int F, const int *sizes, const int *const *rps, const int *const *cis,
                      const double *const *vs, const int *nnzs, const int *order, const or_options *opt);
int or_bgs_setup(or_bgs *h);
int or_bgs_update_values(or_bgs *h, const double *const *vs);
void or_bgs_free(or_bgs *h);
void or_bgs_apply(const or_bgs *h, const double *v, double *z);
void or_bgs_apply_adjoint(const or_bgs *h, const double *v, double *z);
int or_bgs_solve(const or_bgs *h, const double *b, double *x, or_info *info);
int or_bgs_solve_adjoint(const or_bgs *h, const double *g, double *lam, or_info *info);
void or_full_spmv(const or_bgs *h, const double *x, double *y);
void or_grad_values(const or_csr *A, int roff, int coff, const double *lam, const double *x, double *g);

/* Generic FGMRES with a callback preconditioner (used by the tests on small systems) */
typedef void (*or_apply_fn)(void *ctx, const double *in, double *out);
int or_fgmres(int n, or_apply_fn amul, void *actx, or_apply_fn prec, void *pctx, const double *b, double *x,
              int restart, int maxit, double rtol, or_info *info);

#ifdef __cplusplus
}
#endif
#endif
