/*
 * Plain FP64 CPU oracle of the block Gauss-Seidel / SA-AMG / FGMRES solve.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the benchmark's
 * CPU-baseline leg, never by the library.  It shares no code with the CUDA path.
 * Compiled with -ffp-contract=off so that every product and sum is rounded on its own.
 * Independent row loops run on the host's threads (OpenMP) without changing any row's
 * arithmetic; whole-vector sums use the fixed block order of sum_prod below, so results do not
 * depend on the number of threads.
 *
 * Readings of the paper (it configures a library and does not spell these out):
 *  - strength (Sec. 2.2.1 drop tolerance theta; Sec. 3.1.4 theta = 0.04): j is strong for
 *    i != j iff a_ij^2 > theta^2 |a_ii a_jj| or a_ji^2 > theta^2 |a_ii a_jj| (symmetric test;
 *    a missing entry counts as 0).
 *  - coarsening that stalls (n_{l+1} > 0.9 n_l) while the level is above max_coarse is retried
 *    once with theta = 0 (no dropping); if that stalls too, the hierarchy stops there.
 *  - aggregation (not stated in the paper): distance-2 maximal independent set over the
 *    strength graph by synchronous rounds with keys (fmix32(i ^ salt), i); aggregates are a
 *    root plus its strong neighbours, the rest join the neighbouring phase-1 aggregate with the
 *    largest |a_ij| (ties to the smaller aggregate id); ids are roots ranked by node index.
 *  - tentative prolongator: one unnormalised 1 per row (constant near-nullspace).
 *  - filtered smoothing (Sec. 2.2.1, matrix filtering with an absolute-row-sum diagonal):
 *    A_F keeps the diagonal and the strong entries, dropped entries are added to the diagonal,
 *    D_F = sum_j |A_F,ij| (or diag(A_F)); P = P_tent - omega D_F^-1 A_F P_tent with
 *    omega = (4/3) / lambda_max(D_F^-1 A_F).
 *  - Galerkin coarse operator A_{l+1} = R_l A_l P_l, R_l = P_l^T (Eq. galerkin), l = 0..L-1.
 *  - Chebyshev smoother on D^-1 A over [boost*lmax/ratio, boost*lmax] (Sec. 2.2.1: degree 2,
 *    4 for the voltage blocks of the coupled solve, Sec. 3.1.5), three-term recurrence
 *    (Saad, Iterative Methods for Sparse Linear Systems, Alg. 12.1); degree k = k residual
 *    evaluations; lambda_max by power iteration.
 *  - coarsest level: dense LU with partial pivoting in place of the sparse direct solve.
 *  - block Gauss-Seidel (Sec. 2.2, Eqs. hierarchical-bgs ... voltage-bgs): a forward sweep over a
 *    permutation of the fields, one V-cycle per diagonal block, blocks after the current one ignored.
 *  - flexible GMRES(m), right preconditioned, x0 = 0, modified Gram-Schmidt, restarted on the
 *    true residual (Sec. 2.2, flexible GMRES).
 */
#include "bgs_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ST_OK 0
#define ST_INVALID 1
#define ST_NOCONV 3
#define ST_BREAKDOWN 4
#define ST_NANINF 5
#define ST_ZEROPIV 6

/* ------------------------------------------------------------------------------------ */
/* Host threads and whole-vector sums                                                    */
/* ------------------------------------------------------------------------------------ */
/* Loops whose iterations are independent rows (each row's arithmetic written once, in stored
 * order) may run on several host threads; a row's result is the same on any thread, so nothing
 * depends on the thread count.  A sum over a whole vector is the one place where the order of
 * the additions is a choice (the method states inner products and norms, not their summation
 * order): it is taken in consecutive blocks of OR_SUM_BLOCK terms, each block added left to
 * right, then the block sums left to right.  That order is fixed by n alone; for n up to
 * OR_SUM_BLOCK it is the plain left-to-right sum. */
#define OR_SUM_BLOCK 4096

int or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* sum_i a_i b_i in the fixed block order above */
static double sum_prod(int n, const double *a, const double *b) {
    int nb = (n + OR_SUM_BLOCK - 1) / OR_SUM_BLOCK;
    if (nb <= 1) {
        double s = 0.0;
        for (int i = 0; i < n; i++) s += a[i] * b[i];
        return s;
    }
    double *part = (double *)malloc(sizeof(double) * (size_t)nb);
#pragma omp parallel for schedule(static)
    for (int q = 0; q < nb; q++) {
        int lo = q * OR_SUM_BLOCK, hi = lo + OR_SUM_BLOCK < n ? lo + OR_SUM_BLOCK : n;
        double s = 0.0;
        for (int i = lo; i < hi; i++) s += a[i] * b[i];
        part[q] = s;
    }
    double s = 0.0;
    for (int q = 0; q < nb; q++) s += part[q];
    free(part);
    return s;
}

double or_sum_prod(int n, const double *a, const double *b) { return sum_prod(n, a, b); }

/* ------------------------------------------------------------------------------------ */
/* CSR helpers                                                                           */
/* ------------------------------------------------------------------------------------ */
or_csr *or_csr_new(int n, int m, int nnz) {
    or_csr *A = (or_csr *)calloc(1, sizeof(or_csr));
    A->n = n;
    A->m = m;
    A->nnz = nnz;
    A->rp = (int *)calloc((size_t)n + 1, sizeof(int));
    A->ci = (int *)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    A->v = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    return A;
}

or_csr *or_csr_from(int n, int m, const int *rp, const int *ci, const double *v) {
    int nnz = rp[n];
    or_csr *A = or_csr_new(n, m, nnz);
    memcpy(A->rp, rp, sizeof(int) * ((size_t)n + 1));
    memcpy(A->ci, ci, sizeof(int) * (size_t)nnz);
    memcpy(A->v, v, sizeof(double) * (size_t)nnz);
    return A;
}

void or_csr_free(or_csr *A) {
    if (!A) return;
    free(A->rp);
    free(A->ci);
    free(A->v);
    free(A);
}

void or_csr_info(const or_csr *A, int *n, int *m, int *nnz) {
    *n = A->n;
    *m = A->m;
    *nnz = A->nnz;
}

void or_csr_copy(const or_csr *A, int *rp, int *ci, double *v) {
    memcpy(rp, A->rp, sizeof(int) * ((size_t)A->n + 1));
    memcpy(ci, A->ci, sizeof(int) * (size_t)A->nnz);
    memcpy(v, A->v, sizeof(double) * (size_t)A->nnz);
}

/* y = A x, each row summed in stored order */
void or_spmv(const or_csr *A, const double *x, double *y) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < A->n; i++) {
        double s = 0.0;
        for (int e = A->rp[i]; e < A->rp[i + 1]; e++) s += A->v[e] * x[A->ci[e]];
        y[i] = s;
    }
}

/* Plain transpose; rows of the result are sorted because rows of A are visited in order. */
or_csr *or_transpose(const or_csr *A) {
    or_csr *T = or_csr_new(A->m, A->n, A->nnz);
    for (int e = 0; e < A->nnz; e++) T->rp[A->ci[e] + 1]++;
    for (int j = 0; j < A->m; j++) T->rp[j + 1] += T->rp[j];
    int *cur = (int *)malloc(sizeof(int) * ((size_t)A->m + 1));
    memcpy(cur, T->rp, sizeof(int) * ((size_t)A->m + 1));
    for (int i = 0; i < A->n; i++)
        for (int e = A->rp[i]; e < A->rp[i + 1]; e++) {
            int p = cur[A->ci[e]]++;
            T->ci[p] = i;
            T->v[p] = A->v[e];
        }
    free(cur);
    return T;
}

/* C = A B.  Row i of C: for each stored a_ik in order, for each stored b_kj in order,
 * acc[j] += a_ik * b_kj.  Every structural entry is kept; columns sorted. */
or_csr *or_spgemm(const or_csr *A, const or_csr *B) {
    int n = A->n, m = B->m;
    size_t mm = (size_t)(m > 0 ? m : 1);
    /* pass 1: count (each thread marks the columns of its own rows) */
    int *cnt = (int *)calloc((size_t)n + 1, sizeof(int));
#pragma omp parallel
    {
        int *mark = (int *)malloc(sizeof(int) * mm);
        for (int j = 0; j < m; j++) mark[j] = -1;
#pragma omp for schedule(dynamic, 256)
        for (int i = 0; i < n; i++) {
            int c = 0;
            for (int e = A->rp[i]; e < A->rp[i + 1]; e++) {
                int k = A->ci[e];
                for (int f = B->rp[k]; f < B->rp[k + 1]; f++) {
                    int j = B->ci[f];
                    if (mark[j] != i) {
                        mark[j] = i;
                        c++;
                    }
                }
            }
            cnt[i + 1] = c;
        }
        free(mark);
    }
    for (int i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    or_csr *C = or_csr_new(n, m, cnt[n]);
    memcpy(C->rp, cnt, sizeof(int) * ((size_t)n + 1));
    free(cnt);
    /* pass 2: accumulate in order, then emit sorted */
#pragma omp parallel
    {
        int *mark = (int *)malloc(sizeof(int) * mm);
        double *acc = (double *)malloc(sizeof(double) * mm);
        int *cols = (int *)malloc(sizeof(int) * mm);
        for (int j = 0; j < m; j++) mark[j] = -1;
#pragma omp for schedule(dynamic, 256)
        for (int i = 0; i < n; i++) {
            int c = 0;
            for (int e = A->rp[i]; e < A->rp[i + 1]; e++) {
                int k = A->ci[e];
                double a = A->v[e];
                for (int f = B->rp[k]; f < B->rp[k + 1]; f++) {
                    int j = B->ci[f];
                    if (mark[j] != i) {
                        mark[j] = i;
                        acc[j] = 0.0;
                        cols[c++] = j;
                    }
                    acc[j] += a * B->v[f];
                }
            }
            /* insertion sort of the (short) column list */
            for (int p = 1; p < c; p++) {
                int key = cols[p], q = p - 1;
                while (q >= 0 && cols[q] > key) {
                    cols[q + 1] = cols[q];
                    q--;
                }
                cols[q + 1] = key;
            }
            int base = C->rp[i];
            for (int p = 0; p < c; p++) {
                C->ci[base + p] = cols[p];
                C->v[base + p] = acc[cols[p]];
            }
        }
        free(mark);
        free(acc);
        free(cols);
    }
    return C;
}

static double lookup(const or_csr *A, int i, int j) {
    for (int e = A->rp[i]; e < A->rp[i + 1]; e++)
        if (A->ci[e] == j) return A->v[e];
    return 0.0;
}

static double diag_of(const or_csr *A, int i) { return lookup(A, i, i); }

/* ------------------------------------------------------------------------------------ */
/* Strength of connection, strength graph                                                */
/* ------------------------------------------------------------------------------------ */
uint32_t or_fmix32(uint32_t h) {
    /* MurmurHash3 32-bit finaliser (Appleby) */
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

/* strong[e] for each stored entry e of A: off-diagonal and passes the symmetric test */
void or_strength_flags(const or_csr *A, double theta, unsigned char *strong) {
    double t2 = theta * theta;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < A->n; i++) {
        double aii = diag_of(A, i);
        for (int e = A->rp[i]; e < A->rp[i + 1]; e++) {
            int j = A->ci[e];
            strong[e] = 0;
            if (j == i) continue;
            double ajj = diag_of(A, j);
            double aij = A->v[e];
            double aji = lookup(A, j, i);
            double rhs = t2 * fabs(aii * ajj);
            if (aij * aij > rhs || aji * aji > rhs) strong[e] = 1;
        }
    }
}

/* Undirected strength graph: edge {i, j} when a strong entry exists in row i or row j.
 * Values carry a_ij (0 when the entry is only present as a_ji). Rows sorted. */
or_csr *or_strength_graph(const or_csr *A, const unsigned char *strong) {
    int n = A->n;
    /* S_A: strong entries of A */
    int ns = 0;
    for (int e = 0; e < A->nnz; e++) ns += strong[e];
    or_csr *SA = or_csr_new(n, n, ns);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        int c = 0;
        for (int e = A->rp[i]; e < A->rp[i + 1]; e++) c += strong[e];
        SA->rp[i + 1] = c;
    }
    for (int i = 0; i < n; i++) SA->rp[i + 1] += SA->rp[i];
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        int p = SA->rp[i];
        for (int e = A->rp[i]; e < A->rp[i + 1]; e++)
            if (strong[e]) {
                SA->ci[p] = A->ci[e];
                SA->v[p] = A->v[e];
                p++;
            }
    }
    or_csr *ST = or_transpose(SA);
    /* union of row i of S_A and row i of S_A^T */
    int *cnt = (int *)calloc((size_t)n + 1, sizeof(int));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        int a = SA->rp[i], ae = SA->rp[i + 1], b = ST->rp[i], be = ST->rp[i + 1], c = 0;
        while (a < ae || b < be) {
            if (b >= be || (a < ae && SA->ci[a] < ST->ci[b])) a++;
            else if (a >= ae || ST->ci[b] < SA->ci[a]) b++;
            else { a++; b++; }
            c++;
        }
        cnt[i + 1] = c;
    }
    for (int i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    or_csr *S = or_csr_new(n, n, cnt[n]);
    memcpy(S->rp, cnt, sizeof(int) * ((size_t)n + 1));
    free(cnt);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        int a = SA->rp[i], ae = SA->rp[i + 1], b = ST->rp[i], be = ST->rp[i + 1], q = S->rp[i];
        while (a < ae || b < be) {
            if (b >= be || (a < ae && SA->ci[a] < ST->ci[b])) {
                S->ci[q] = SA->ci[a];
                S->v[q] = SA->v[a];
                a++;
            } else if (a >= ae || ST->ci[b] < SA->ci[a]) {
                S->ci[q] = ST->ci[b];
                S->v[q] = 0.0;
                b++;
            } else {
                S->ci[q] = SA->ci[a];
                S->v[q] = SA->v[a];
                a++;
                b++;
            }
            q++;
        }
    }
    or_csr_free(SA);
    or_csr_free(ST);
    return S;
}

/* ------------------------------------------------------------------------------------ */
/* Distance-2 maximal independent set by synchronous rounds                              */
/* ------------------------------------------------------------------------------------ */
static uint64_t mis_key(int i, uint32_t salt) {
    return ((uint64_t)or_fmix32((uint32_t)i ^ salt) << 32) | (uint64_t)(uint32_t)i;
}

/* state: 0 undecided, 1 in (root), 2 out.  Round: (i) an undecided v becomes a root iff its key
 * is larger than the key of every other undecided node within distance 2 (paths through any
 * node); (ii) every undecided node within distance 2 of a root leaves.  Returns the round count. */
int or_mis2(const or_csr *S, uint32_t salt, int *state) {
    int n = S->n;
    for (int i = 0; i < n; i++) state[i] = 0;
    int *newin = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int rounds = 0, undecided = n;
    while (undecided > 0) {
        rounds++;
        /* (i) by definition: scan the distance-2 ball of each undecided node */
#pragma omp parallel for schedule(static)
        for (int v = 0; v < n; v++) {
            newin[v] = 0;
            if (state[v] != 0) continue;
            uint64_t kv = mis_key(v, salt);
            int ok = 1;
            for (int e = S->rp[v]; e < S->rp[v + 1] && ok; e++) {
                int u = S->ci[e];
                if (u != v && state[u] == 0 && mis_key(u, salt) > kv) ok = 0;
                for (int f = S->rp[u]; f < S->rp[u + 1] && ok; f++) {
                    int w = S->ci[f];
                    if (w != v && state[w] == 0 && mis_key(w, salt) > kv) ok = 0;
                }
            }
            newin[v] = ok;
        }
#pragma omp parallel for schedule(static)
        for (int v = 0; v < n; v++)
            if (newin[v]) state[v] = 1;
        /* (ii) undecided nodes within distance 2 of a root leave */
#pragma omp parallel for schedule(static)
        for (int v = 0; v < n; v++) {
            if (state[v] != 0) continue;
            int near = 0;
            for (int e = S->rp[v]; e < S->rp[v + 1] && !near; e++) {
                int u = S->ci[e];
                if (state[u] == 1) near = 1;
                for (int f = S->rp[u]; f < S->rp[u + 1] && !near; f++)
                    if (state[S->ci[f]] == 1) near = 1;
            }
            newin[v] = near;
        }
        undecided = 0;
#pragma omp parallel for schedule(static) reduction(+ : undecided)
        for (int v = 0; v < n; v++) {
            if (state[v] == 0 && newin[v]) state[v] = 2;
            if (state[v] == 0) undecided++;
        }
    }
    free(newin);
    return rounds;
}

/* Aggregates from the roots: phase 1 = root + its strong neighbours; phase 2 = remaining nodes
 * join the phase-1 aggregate of the neighbour with the largest |a_ij| (ties: smaller id).
 * Ids: roots ranked by node index.  Returns the aggregate count, or -1 if a node is left over. */
int or_aggregate(const or_csr *S, const int *state, int *agg) {
    int n = S->n;
    int *rootid = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int nagg = 0;
    for (int i = 0; i < n; i++) rootid[i] = (state[i] == 1) ? nagg++ : -1;
    int *ph1 = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        ph1[i] = -1;
        if (state[i] == 1) {
            ph1[i] = rootid[i];
            continue;
        }
        for (int e = S->rp[i]; e < S->rp[i + 1]; e++) {
            int j = S->ci[e];
            if (state[j] == 1) ph1[i] = rootid[j];
        }
    }
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int i = 0; i < n; i++) {
        if (ph1[i] >= 0) {
            agg[i] = ph1[i];
            continue;
        }
        int best = -1;
        double bw = -1.0;
        for (int e = S->rp[i]; e < S->rp[i + 1]; e++) {
            int j = S->ci[e];
            if (j == i || ph1[j] < 0) continue;
            double w = fabs(S->v[e]);
            if (w > bw || (w == bw && ph1[j] < best)) {
                bw = w;
                best = ph1[j];
            }
        }
        agg[i] = best;
        if (best < 0) bad = 1;
    }
    free(rootid);
    free(ph1);
    return bad ? -1 : nagg;
}

/* Filtered matrix values vF (pattern of A) and its smoothing diagonal dF. */
void or_filter(const or_csr *A, const unsigned char *strong, int filter_diag, double *vF, double *dF) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < A->n; i++) {
        double lump = 0.0;
        int dpos = -1;
        for (int e = A->rp[i]; e < A->rp[i + 1]; e++) {
            int j = A->ci[e];
            if (j == i) {
                dpos = e;
                vF[e] = A->v[e];
            } else if (strong[e]) {
                vF[e] = A->v[e];
            } else {
                vF[e] = 0.0;
                lump += A->v[e];
            }
        }
        if (dpos >= 0) vF[dpos] = A->v[dpos] + lump;
        /* a row left with its lumped diagonal only, which is zero up to rounding (a zero row sum:
         * below 1e-12 of the row's absolute sum), is an exact zero row */
        int nstrong = 0;
        double rabs = 0.0;
        for (int e = A->rp[i]; e < A->rp[i + 1]; e++) {
            rabs += fabs(A->v[e]);
            nstrong += A->ci[e] != i && strong[e];
        }
        if (dpos >= 0 && nstrong == 0 && fabs(vF[dpos]) <= 1e-12 * rabs) vF[dpos] = 0.0;
        if (filter_diag) {
            double s = 0.0;
            for (int e = A->rp[i]; e < A->rp[i + 1]; e++)
                if (A->ci[e] == i || strong[e]) s += fabs(vF[e]);
            dF[i] = s;
        } else {
            dF[i] = dpos >= 0 ? vF[dpos] : 0.0;
        }
    }
}

/* lambda_max(D^-1 A) by power iteration from a hashed positive start vector.
 * v0_i = (fmix32(i ^ 0x7F4A7C15) >> 8 + 0.5) / 2^24, normalised; each step w = D^-1 A v,
 * lambda = ||w||, v = w / lambda.  Returns the last lambda. */
double or_power_lambda(const or_csr *A, const double *dinv, int iters) {
    int n = A->n;
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        uint32_t u = or_fmix32((uint32_t)i ^ 0x7F4A7C15u) >> 8;
        v[i] = ((double)u + 0.5) / 16777216.0;
    }
    double nv = sqrt(sum_prod(n, v, v));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) v[i] = v[i] / nv;
    double lam = 0.0;
    for (int it = 0; it < iters; it++) {
        or_spmv(A, v, w);
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; i++) w[i] = dinv[i] * w[i];
        lam = sqrt(sum_prod(n, w, w));
        if (lam == 0.0) break;
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; i++) v[i] = w[i] / lam;
    }
    free(v);
    free(w);
    return lam;
}

/* P = P_tent - omega D_F^-1 A_F P_tent, row by row: s_J = sum of A_F(i, j) over agg(j) = J in
 * stored order (this is A_F P_tent), p_iJ = [J == agg(i)] - c_i s_J with c_i = omega / D_F,ii. */
or_csr *or_smooth_prolongator(const or_csr *AF, const double *dinvF, const int *agg, int nagg, double omega) {
    int n = AF->n;
    or_csr *Pt = or_csr_new(n, nagg, n);
    for (int i = 0; i < n; i++) {
        Pt->rp[i + 1] = i + 1;
        Pt->ci[i] = agg[i];
        Pt->v[i] = 1.0;
    }
    or_csr *S = or_spgemm(AF, Pt);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        double c = omega * dinvF[i];
        for (int e = S->rp[i]; e < S->rp[i + 1]; e++) {
            double t = (S->ci[e] == agg[i]) ? 1.0 : 0.0;
            S->v[e] = t - c * S->v[e];
        }
    }
    or_csr_free(Pt);
    return S;
}

/* ------------------------------------------------------------------------------------ */
/* Chebyshev smoother on D^-1 A (Saad Alg. 12.1 form)                                    */
/* ------------------------------------------------------------------------------------ */
void or_chebyshev(const or_csr *A, const double *dinv, double lmin, double lmax, int deg,
                  const double *b, double *x, int x_is_zero) {
    int n = A->n;
    if (deg <= 0) return;
    double theta = (lmax + lmin) / 2.0, delta = (lmax - lmin) / 2.0;
    double sigma = theta / delta, rho = 1.0 / sigma;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    double inv_theta = 1.0 / theta;
    if (x_is_zero) {
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; i++) r[i] = b[i];
    } else {
        or_spmv(A, x, r);
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; i++) r[i] = b[i] - r[i];
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        d[i] = inv_theta * (dinv[i] * r[i]);
        x[i] = (x_is_zero ? 0.0 : x[i]) + d[i];
    }
    for (int k = 1; k < deg; k++) {
        double rho_new = 1.0 / (2.0 * sigma - rho);
        double c1 = rho_new * rho, c2 = 2.0 * rho_new / delta;
        or_spmv(A, x, r);
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; i++) {
            double ri = b[i] - r[i];
            d[i] = c1 * d[i] + c2 * (dinv[i] * ri);
            x[i] = x[i] + d[i];
        }
        rho = rho_new;
    }
    free(r);
    free(d);
}

/* ------------------------------------------------------------------------------------ */
/* Dense LU with partial pivoting (row-major, in place)                                  */
/* ------------------------------------------------------------------------------------ */
/* Radius of the skew-symmetric part of the diagonally scaled operator, rho(S) with
 * S = (M - M^T)/2 and M = D^-1/2 A D^-1/2 (D = diag(A), all positive; else 0).  M is similar to
 * D^-1 A, so by Bendixson's theorem every eigenvalue of D^-1 A has |Im| <= rho(S).  Power
 * iteration on S^T S = -S S from the same hashed start as or_power_lambda; returns sqrt of the
 * last estimate (0 for a symmetric A, where S = 0). */
double or_skew_radius(const or_csr *A, int iters) {
    int n = A->n;
    double *sc = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; i++) {
        double d = diag_of(A, i);
        if (!(d > 0.0)) {
            free(sc);
            return 0.0;
        }
        sc[i] = 1.0 / sqrt(d);
    }
    or_csr *AT = or_transpose(A);
    double *v = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *t = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *p = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *q = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *u = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        uint32_t h = or_fmix32((uint32_t)i ^ 0x7F4A7C15u) >> 8;
        v[i] = ((double)h + 0.5) / 16777216.0;
    }
    double nv = sqrt(sum_prod(n, v, v));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) v[i] = v[i] / nv;
    double lam = 0.0;
    for (int it = 0; it < iters; it++) {
        /* u = S v, then w = -S u; S x = (s .* (A (s .* x)) - s .* (A^T (s .* x))) / 2 */
        for (int pass = 0; pass < 2; pass++) {
            const double *in = pass == 0 ? v : u;
#pragma omp parallel for schedule(static)
            for (int i = 0; i < n; i++) t[i] = sc[i] * in[i];
            or_spmv(A, t, p);
            or_spmv(AT, t, q);
            double *out = pass == 0 ? u : t;
#pragma omp parallel for schedule(static)
            for (int i = 0; i < n; i++) out[i] = 0.5 * (sc[i] * p[i] - sc[i] * q[i]);
        }
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; i++) t[i] = -t[i];
        lam = sqrt(sum_prod(n, t, t));
        if (lam == 0.0) break;
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; i++) v[i] = t[i] / lam;
    }
    or_csr_free(AT);
    free(sc);
    free(v);
    free(t);
    free(p);
    free(q);
    free(u);
    return sqrt(lam);
}

/* Chebyshev smoothing for a spectrum of D^-1 A inside the ellipse with centre theta on the real axis
 * and focal parameter c2 = a^2 - b^2 (a real, b imaginary semi-axis; c2 < 0 when the ellipse is
 * taller than wide), the nonsymmetric form of Sec. 2.2.1 (Manteuffel).  The iteration of
 * or_chebyshev with tau_k = rho_k / delta, which keeps every coefficient real for any c2:
 * tau_0 = 1/theta, d = tau_0 D^-1 r; tau_k = 1/(2 theta - c2 tau_{k-1}),
 * d = c2 tau_k tau_{k-1} d + 2 tau_k D^-1 r, x += d.  The error is then multiplied by
 * T_k((theta - z)/c)/T_k(theta/c) on each eigenvalue z. */
void or_chebyshev_ellipse(const or_csr *A, const double *dinv, double theta, double c2, int deg,
                          const double *b, double *x, int x_is_zero) {
    int n = A->n;
    if (deg <= 0) return;
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *d = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double tau = 1.0 / theta;
    if (x_is_zero) {
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; i++) r[i] = b[i];
    } else {
        or_spmv(A, x, r);
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; i++) r[i] = b[i] - r[i];
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        d[i] = tau * (dinv[i] * r[i]);
        x[i] = (x_is_zero ? 0.0 : x[i]) + d[i];
    }
    for (int k = 1; k < deg; k++) {
        double tau_new = 1.0 / (2.0 * theta - c2 * tau);
        double c1 = c2 * tau_new * tau, cc = 2.0 * tau_new;
        or_spmv(A, x, r);
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; i++) {
            double ri = b[i] - r[i];
            d[i] = c1 * d[i] + cc * (dinv[i] * ri);
            x[i] = x[i] + d[i];
        }
        tau = tau_new;
    }
    free(r);
    free(d);
}

int or_lu_factor(int n, double *a, int *piv) {
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = fabs(a[(size_t)k * n + k]);
        for (int i = k + 1; i < n; i++) {
            double t = fabs(a[(size_t)i * n + k]);
            if (t > best) {
                best = t;
                p = i;
            }
        }
        piv[k] = p;
        if (best == 0.0) return ST_ZEROPIV;
        if (p != k)
            for (int j = 0; j < n; j++) {
                double t = a[(size_t)k * n + j];
                a[(size_t)k * n + j] = a[(size_t)p * n + j];
                a[(size_t)p * n + j] = t;
            }
        double akk = a[(size_t)k * n + k];
        for (int i = k + 1; i < n; i++) {
            double l = a[(size_t)i * n + k] / akk;
            a[(size_t)i * n + k] = l;
            for (int j = k + 1; j < n; j++) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
        }
    }
    return ST_OK;
}

void or_lu_solve(int n, const double *lu, const int *piv, const double *b, double *x) {
    for (int i = 0; i < n; i++) x[i] = b[i];
    for (int k = 0; k < n; k++)
        if (piv[k] != k) {
            double t = x[k];
            x[k] = x[piv[k]];
            x[piv[k]] = t;
        }
    for (int i = 0; i < n; i++) {
        double s = x[i];
        for (int j = 0; j < i; j++) s -= lu[(size_t)i * n + j] * x[j];
        x[i] = s;
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = x[i];
        for (int j = i + 1; j < n; j++) s -= lu[(size_t)i * n + j] * x[j];
        x[i] = s / lu[(size_t)i * n + i];
    }
}

/* A^T x = b with P A = L U: U^T y = b, L^T w = y, x = P^T w */
static void lu_solve_transposed(int n, const double *lu, const int *piv, const double *b, double *x) {
    for (int i = 0; i < n; i++) x[i] = b[i];
    for (int i = 0; i < n; i++) {
        double s = x[i];
        for (int j = 0; j < i; j++) s -= lu[(size_t)j * n + i] * x[j];
        x[i] = s / lu[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = x[i];
        for (int j = i + 1; j < n; j++) s -= lu[(size_t)j * n + i] * x[j];
        x[i] = s;
    }
    for (int k = n - 1; k >= 0; k--)
        if (piv[k] != k) {
            double t = x[k];
            x[k] = x[piv[k]];
            x[piv[k]] = t;
        }
}

/* ------------------------------------------------------------------------------------ */
/* SA-AMG hierarchy                                                                      */
/* ------------------------------------------------------------------------------------ */
/* Numeric part of one coarsening step, given the strength flags and aggregates of level l:
 * filtered matrix A_F (diagonal + strong entries, dropped entries lumped), D_F, omega from the
 * power iteration, P = P_tent - omega D_F^-1 A_F P_tent, R = P^T, A_{l+1} = R (A_l P).  The
 * full set-up and the numeric re-set-up both go through here. */
static void level_numeric(or_amg *h, int l, const unsigned char *strong, const or_options *opt) {
    or_csr *A = h->A[l];
    int n = A->n;
    double *vF = (double *)malloc(sizeof(double) * (size_t)(A->nnz > 0 ? A->nnz : 1));
    double *dF = (double *)malloc(sizeof(double) * (size_t)n);
    or_filter(A, strong, opt->filter_diag, vF, dF);
    /* A_F as its own matrix: the dropped entries leave the pattern (they would only add
     * structural zeros to P and to the coarse operators) */
    int *len = (int *)calloc((size_t)n + 1, sizeof(int));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        int c = 0;
        for (int e = A->rp[i]; e < A->rp[i + 1]; e++) c += (A->ci[e] == i) || strong[e];
        len[i + 1] = c;
    }
    for (int i = 0; i < n; i++) len[i + 1] += len[i];
    or_csr *AF = or_csr_new(n, n, len[n]);
    memcpy(AF->rp, len, sizeof(int) * ((size_t)n + 1));
    free(len);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        int q = AF->rp[i];
        for (int e = A->rp[i]; e < A->rp[i + 1]; e++)
            if (A->ci[e] == i || strong[e]) {
                AF->ci[q] = A->ci[e];
                AF->v[q] = vF[e];
                q++;
            }
    }
    double *dinvF = (double *)malloc(sizeof(double) * (size_t)n);
    /* a row whose filtered entries lump to zero (all its connections weak and a zero row sum)
     * takes no part in the smoothing: D_F^-1 = 0 there, so its row of P stays the P_tent row */
    for (int i = 0; i < n; i++) dinvF[i] = dF[i] != 0.0 ? 1.0 / dF[i] : 0.0;
    double lam = or_power_lambda(AF, dinvF, opt->power_iters);
    double omega = (4.0 / 3.0) / lam;
    or_csr *P = or_smooth_prolongator(AF, dinvF, h->agg[l], h->nagg[l], omega);
    or_csr_free(AF);
    or_csr *R = or_transpose(P);
    or_csr *AP = or_spgemm(A, P);
    or_csr *Ac = or_spgemm(R, AP);
    or_csr_free(AP);
    free(vF);
    free(dF);
    free(dinvF);
    or_csr_free(h->P[l]);
    or_csr_free(h->R[l]);
    or_csr_free(h->A[l + 1]);
    h->omega[l] = omega;
    h->P[l] = P;
    h->R[l] = R;
    h->A[l + 1] = Ac;
}

/* Smoother bounds on every level above the coarsest, and the dense LU of the coarsest. */
static void smoothers_and_lu(or_amg *h, const or_options *opt) {
    for (int k = 0; k + 1 < h->nlevels; k++) {
        or_csr *A = h->A[k];
        free(h->dinv[k]);
        h->dinv[k] = (double *)malloc(sizeof(double) * (size_t)A->n);
#pragma omp parallel for schedule(static)
        for (int i = 0; i < A->n; i++) h->dinv[k][i] = 1.0 / diag_of(A, i);
        double lam = or_power_lambda(A, h->dinv[k], opt->power_iters);
        h->lmax[k] = opt->cheb_boost * lam;
        h->lmin[k] = h->lmax[k] / opt->cheb_ratio;
        h->lim[k] = opt->cheb_ellipse ? opt->cheb_boost * or_skew_radius(A, opt->power_iters) : 0.0;
        /* below 1e-10 of lmax the skew part is rounding noise (e.g. a Galerkin product of a
         * symmetric operator summed in two orders): keep the real interval */
        if (h->lim[k] <= 1e-10 * h->lmax[k]) h->lim[k] = 0.0;
    }
    or_csr *Ac = h->A[h->nlevels - 1];
    int nc = Ac->n;
    h->nc = nc;
    free(h->lu);
    free(h->piv);
    h->lu = (double *)calloc((size_t)nc * nc, sizeof(double));
    h->piv = (int *)malloc(sizeof(int) * (size_t)(nc > 0 ? nc : 1));
    for (int i = 0; i < nc; i++)
        for (int e = Ac->rp[i]; e < Ac->rp[i + 1]; e++) h->lu[(size_t)i * nc + Ac->ci[e]] = Ac->v[e];
    int st = or_lu_factor(nc, h->lu, h->piv);
    if (st != ST_OK && h->status == ST_OK) h->status = st;
}

or_amg *or_amg_setup(const or_csr *A0, double theta, int degree, const or_options *opt) {
    or_amg *h = (or_amg *)calloc(1, sizeof(or_amg));
    h->degree = degree;
    h->A[0] = or_csr_from(A0->n, A0->m, A0->rp, A0->ci, A0->v);
    int l = 0;
    int maxlev = opt->max_levels < OR_MAX_LEVELS ? opt->max_levels : OR_MAX_LEVELS;
    for (;;) {
        or_csr *A = h->A[l];
        int n = A->n;
        if (n <= opt->max_coarse || l + 1 >= maxlev) break;
        unsigned char *strong = (unsigned char *)malloc((size_t)(A->nnz > 0 ? A->nnz : 1));
        or_csr *S = NULL;
        int *agg = (int *)malloc(sizeof(int) * (size_t)n);
        int nagg = -1;
        /* coarsening that stalls above max_coarse is retried once without dropping (theta = 0) */
        for (int attempt = 0; attempt < 2; attempt++) {
            double th = attempt == 0 ? theta : 0.0;
            if (attempt == 1 && (theta == 0.0 || nagg < 0 || (long long)nagg * 10 <= (long long)n * 9)) break;
            or_csr_free(S);
            or_strength_flags(A, th, strong);
            S = or_strength_graph(A, strong);
            int *state = (int *)malloc(sizeof(int) * (size_t)n);
            h->mis_rounds[l] = or_mis2(S, (uint32_t)l * 0x9E3779B9u, state);
            nagg = or_aggregate(S, state, agg);
            free(state);
        }
        or_csr_free(S);
        if (nagg < 0) {
            h->status = ST_INVALID;
            free(agg);
            free(strong);
            break;
        }
        if ((long long)nagg * 10 > (long long)n * 9) { /* coarsening stalled: stop here */
            free(agg);
            free(strong);
            break;
        }
        h->agg[l] = agg;
        h->nagg[l] = nagg;
        h->strong[l] = strong;   /* kept for the numeric re-set-up */
        level_numeric(h, l, strong, opt);
        l++;
    }
    h->nlevels = l + 1;
    smoothers_and_lu(h, opt);
    return h;
}

/* Numeric re-set-up: Sec. 3.2 notes that the symbolic phase of a factorisation can be recycled
 * across the linear solves of a simulation while the numeric phase is repeated every nonlinear
 * iteration.  The same split is taken here for the hierarchy: the level-0 operator takes new
 * values on its old pattern; every level keeps the strength flags and aggregates of the full
 * set-up (so every pattern stays the same), and all numeric quantities are recomputed. */
int or_amg_update(or_amg *h, const double *v0, const or_options *opt) {
    memcpy(h->A[0]->v, v0, sizeof(double) * (size_t)h->A[0]->nnz);
    h->status = ST_OK;
    for (int l = 0; l + 1 < h->nlevels; l++) level_numeric(h, l, h->strong[l], opt);
    smoothers_and_lu(h, opt);
    return h->status;
}

void or_amg_free(or_amg *h) {
    if (!h) return;
    for (int l = 0; l < OR_MAX_LEVELS; l++) {
        or_csr_free(h->A[l]);
        or_csr_free(h->P[l]);
        or_csr_free(h->R[l]);
        free(h->agg[l]);
        free(h->strong[l]);
        free(h->dinv[l]);
    }
    free(h->lu);
    free(h->piv);
    free(h);
}

/* the level's smoother: the real interval, or the ellipse when an imaginary extent was estimated
 * (the transposed operator has the conjugate spectrum, so the same ellipse) */
static void cheb_level(const or_amg *h, int l, const or_csr *A, const double *b, double *x, int x_is_zero) {
    if (h->lim[l] > 0.0) {
        double theta = (h->lmax[l] + h->lmin[l]) / 2.0, a = (h->lmax[l] - h->lmin[l]) / 2.0;
        or_chebyshev_ellipse(A, h->dinv[l], theta, a * a - h->lim[l] * h->lim[l], h->degree, b, x, x_is_zero);
    } else {
        or_chebyshev(A, h->dinv[l], h->lmin[l], h->lmax[l], h->degree, b, x, x_is_zero);
    }
}

static void vcycle_level(const or_amg *h, int l, const double *b, double *x, int transposed, or_csr **AT) {
    if (l == h->nlevels - 1) {
        if (transposed) lu_solve_transposed(h->nc, h->lu, h->piv, b, x);
        else or_lu_solve(h->nc, h->lu, h->piv, b, x);
        return;
    }
    const or_csr *A = transposed ? AT[l] : h->A[l];
    int n = A->n, nc = h->A[l + 1]->n;
    cheb_level(h, l, A, b, x, 1);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    or_spmv(A, x, r);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) r[i] = b[i] - r[i];
    double *bc = (double *)malloc(sizeof(double) * (size_t)nc);
    double *xc = (double *)malloc(sizeof(double) * (size_t)nc);
    or_spmv(h->R[l], r, bc);
    vcycle_level(h, l + 1, bc, xc, transposed, AT);
    or_spmv(h->P[l], xc, r);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) x[i] += r[i];
    cheb_level(h, l, A, b, x, 0);
    free(r);
    free(bc);
    free(xc);
}

void or_vcycle(const or_amg *h, const double *b, double *x) { vcycle_level(h, 0, b, x, 0, NULL); }

/* ------------------------------------------------------------------------------------ */
/* DD(0)-ILU(0) subblock solver                                                          */
/* ------------------------------------------------------------------------------------ */
/* One-level restricted additive Schwarz without overlap (Sec. 2.1, Eq. one-level-schwarz with
 * D_i = I) over subdomains of `rows` consecutive rows, each subdomain matrix A_i = R_i A R_i^T
 * approximated by one ILU(0) factorisation (the species solver of Sec. 3.1.1).  F holds A_i for
 * every subdomain (entries coupling two subdomains dropped), then L (unit, strictly lower) and U
 * (upper, with the diagonal) in its pattern. */
or_ilu *or_ilu_setup(const or_csr *A, int rows) {
    or_ilu *m = (or_ilu *)calloc(1, sizeof(or_ilu));
    int n = A->n;
    m->rows = rows > 0 ? rows : n;
    int nf = 0;
    for (int i = 0; i < n; i++)
        for (int e = A->rp[i]; e < A->rp[i + 1]; e++) nf += A->ci[e] / m->rows == i / m->rows;
    or_csr *F = or_csr_new(n, n, nf);
    nf = 0;
    for (int i = 0; i < n; i++) {
        for (int e = A->rp[i]; e < A->rp[i + 1]; e++)
            if (A->ci[e] / m->rows == i / m->rows) {
                F->ci[nf] = A->ci[e];
                F->v[nf] = A->v[e];
                nf++;
            }
        F->rp[i + 1] = nf;
    }
    m->F = F;
    m->status = or_ilu_factor(m);
    return m;
}

/* ILU(0) in place, row by row (IKJ): for each k < i stored in row i, l_ik = a_ik / u_kk, then
 * a_ij -= l_ik u_kj for every j > k stored in both row i and row k. */
int or_ilu_factor(or_ilu *m) {
    or_csr *F = m->F;
    int st = ST_OK;
    for (int i = 0; i < F->n; i++) {
        for (int e = F->rp[i]; e < F->rp[i + 1] && F->ci[e] < i; e++) {
            int k = F->ci[e];
            int dk = -1;
            for (int f = F->rp[k]; f < F->rp[k + 1]; f++)
                if (F->ci[f] == k) dk = f;
            if (dk < 0 || F->v[dk] == 0.0) {
                st = ST_ZEROPIV;
                continue;
            }
            double l = F->v[e] / F->v[dk];
            F->v[e] = l;
            /* merge the rest of row i with the upper part of row k */
            int f = dk + 1;
            for (int g = e + 1; g < F->rp[i + 1]; g++) {
                while (f < F->rp[k + 1] && F->ci[f] < F->ci[g]) f++;
                if (f < F->rp[k + 1] && F->ci[f] == F->ci[g]) F->v[g] = F->v[g] - l * F->v[f];
            }
        }
    }
    for (int i = 0; i < F->n; i++) {
        int has = 0;
        for (int e = F->rp[i]; e < F->rp[i + 1]; e++)
            if (F->ci[e] == i) has = F->v[e] != 0.0;
        if (!has) st = ST_ZEROPIV;
    }
    return st;
}

/* z = (L U)^-1 r, subdomain by subdomain: L y = r forward, U z = y backward (CSR order sums). */
void or_ilu_apply(const or_ilu *m, const double *r, double *z) {
    const or_csr *F = m->F;
    for (int i = 0; i < F->n; i++) {
        double t = r[i];
        for (int e = F->rp[i]; e < F->rp[i + 1] && F->ci[e] < i; e++) t = t - F->v[e] * z[F->ci[e]];
        z[i] = t;
    }
    for (int i = F->n - 1; i >= 0; i--) {
        double t = z[i], d = 0.0;
        for (int e = F->rp[i]; e < F->rp[i + 1]; e++) {
            if (F->ci[e] == i) d = F->v[e];
            else if (F->ci[e] > i) t = t - F->v[e] * z[F->ci[e]];
        }
        z[i] = t / d;
    }
}

/* z = (L U)^-T r: U^T w = r (forward, column sweeps of U), then L^T z = w (backward). */
void or_ilu_apply_transposed(const or_ilu *m, const double *r, double *z) {
    const or_csr *F = m->F;
    int n = F->n;
    double *t = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    memcpy(t, r, sizeof(double) * (size_t)n);
    for (int i = 0; i < n; i++) {
        double d = 0.0;
        for (int e = F->rp[i]; e < F->rp[i + 1]; e++)
            if (F->ci[e] == i) d = F->v[e];
        double w = t[i] / d;
        z[i] = w;
        for (int e = F->rp[i]; e < F->rp[i + 1]; e++)
            if (F->ci[e] > i) t[F->ci[e]] -= F->v[e] * w;
    }
    for (int i = n - 1; i >= 0; i--) {
        double w = z[i];
        for (int e = F->rp[i]; e < F->rp[i + 1] && F->ci[e] < i; e++) z[F->ci[e]] -= F->v[e] * w;
    }
    free(t);
}

/* numeric refactorisation after the values of A changed on the same pattern */
int or_ilu_update(or_ilu *m, const or_csr *A) {
    or_csr *F = m->F;
    int q = 0;
    for (int i = 0; i < A->n; i++)
        for (int e = A->rp[i]; e < A->rp[i + 1]; e++)
            if (A->ci[e] / m->rows == i / m->rows) F->v[q++] = A->v[e];
    m->status = or_ilu_factor(m);
    return m->status;
}

void or_ilu_free(or_ilu *m) {
    if (!m) return;
    or_csr_free(m->F);
    free(m);
}

/* ------------------------------------------------------------------------------------ */
/* Block Gauss-Seidel                                                                    */
/* ------------------------------------------------------------------------------------ */
void or_default_options(or_options *o) {
    memset(o, 0, sizeof(*o));
    o->restart = 50;
    o->maxit = 1000;
    o->rtol = 1e-8;
    for (int k = 0; k < 8; k++) {
        o->cheb_degree[k] = 2;
        o->theta[k] = 0.0;     /* no dropping: the library default the paper leaves in place */
    }
    o->theta[0] = 0.04;        /* phi_s: the grid-searched drop tolerance (Sec. 3.1.4) */
    o->cheb_degree[0] = 4;     /* voltage blocks: degree 4 in the coupled solve (Sec. 3.1.5) */
    o->cheb_degree[1] = 4;
    o->max_coarse = 500;       /* the coarsest level is a dense LU; the paper's 5000 suits a sparse solver */
    o->max_levels = 10;
    o->cheb_ratio = 30.0;
    o->cheb_boost = 1.1;
    o->power_iters = 10;
    o->filter_diag = 1;
    o->ilu_rows = 4096;
    o->ngroups = 0;
    o->inner_restart = 30;
    o->inner_maxit = 30;
    o->inner_rtol = 1e-6;
}

or_bgs *or_bgs_create(int F, const int *sizes, const int *const *rps, const int *const *cis,
                      const double *const *vs, const int *nnzs, const int *order, const or_options *opt) {
    (void)nnzs;
    or_bgs *h = (or_bgs *)calloc(1, sizeof(or_bgs));
    h->F = F;
    h->opt = *opt;
    h->offs[0] = 0;
    for (int k = 0; k < F; k++) {
        h->sizes[k] = sizes[k];
        h->offs[k + 1] = h->offs[k] + sizes[k];
        h->order[k] = order[k];
        h->pos[order[k]] = k;
    }
    for (int r = 0; r < F; r++)
        for (int c = 0; c < F; c++) {
            int b = r * F + c;
            if (rps[b]) h->blk[b] = or_csr_from(sizes[r], sizes[c], rps[b], cis[b], vs[b]);
        }
    /* full operator: row i of field r = blocks (r, 0..F-1) concatenated with column offsets */
    int n = h->offs[F];
    long long nnz = 0;
    for (int b = 0; b < F * F; b++)
        if (h->blk[b]) nnz += h->blk[b]->nnz;
    or_csr *A = or_csr_new(n, n, (int)nnz);
    /* row lengths, their running sum, then every row's entries (rows independent) */
    for (int r = 0; r < F; r++) {
#pragma omp parallel for schedule(static)
        for (int i = 0; i < sizes[r]; i++) {
            int len = 0;
            for (int c = 0; c < F; c++) {
                or_csr *B = h->blk[r * F + c];
                if (B) len += B->rp[i + 1] - B->rp[i];
            }
            A->rp[h->offs[r] + i + 1] = len;
        }
    }
    for (int i = 0; i < n; i++) A->rp[i + 1] += A->rp[i];
    for (int r = 0; r < F; r++) {
#pragma omp parallel for schedule(static)
        for (int i = 0; i < sizes[r]; i++) {
            int q = A->rp[h->offs[r] + i];
            for (int c = 0; c < F; c++) {
                or_csr *B = h->blk[r * F + c];
                if (!B) continue;
                for (int e = B->rp[i]; e < B->rp[i + 1]; e++) {
                    A->ci[q] = B->ci[e] + h->offs[c];
                    A->v[q] = B->v[e];
                    q++;
                }
            }
        }
    }
    h->full = A;
    return h;
}

int or_bgs_setup(or_bgs *h) {
    int st[8] = {0};
    /* the diagonal blocks are independent: each is set up on its own share of the host threads */
#ifdef _OPENMP
    int T = omp_get_max_threads(), outer = T < h->F ? T : h->F, inner = T / (outer > 0 ? outer : 1);
    omp_set_max_active_levels(2);
#pragma omp parallel for schedule(dynamic, 1) num_threads(outer > 0 ? outer : 1)
#endif
    for (int k = 0; k < h->F; k++) {
#ifdef _OPENMP
        omp_set_num_threads(inner > 0 ? inner : 1);
#endif
        or_csr *Akk = h->blk[k * h->F + k];
        if (h->opt.subsolver[k] == 2) {   /* the block's diagonal: exact for a diagonal block */
            int nk = h->sizes[k];
            h->dgs[k] = (double *)malloc(sizeof(double) * (size_t)(nk > 0 ? nk : 1));
            for (int i = 0; i < nk; i++) {
                double d = diag_of(Akk, i);
                if (d == 0.0) st[k] = ST_ZEROPIV;
                h->dgs[k][i] = 1.0 / d;
            }
            continue;
        }
        if (h->opt.subsolver[k] == 1) {   /* DD(0)-ILU(0) */
            h->ilu[k] = or_ilu_setup(Akk, h->opt.ilu_rows);
            st[k] = h->ilu[k]->status;
            continue;
        }
        h->amg[k] = or_amg_setup(Akk, h->opt.theta[k], h->opt.cheb_degree[k], &h->opt);
        st[k] = h->amg[k]->status;
    }
    for (int k = 0; k < h->F; k++)
        if (st[k]) h->status = st[k];
    return h->status;
}

/* New values for the stored blocks (same patterns; NULL keeps a block's values): the full
 * operator takes them, and every diagonal block's hierarchy is re-set-up numerically. */
int or_bgs_update_values(or_bgs *h, const double *const *vs) {
    int F = h->F;
    for (int b = 0; b < F * F; b++)
        if (h->blk[b] && vs[b]) memcpy(h->blk[b]->v, vs[b], sizeof(double) * (size_t)h->blk[b]->nnz);
    int q = 0;   /* the full operator's entries in the order or_bgs_create laid them out */
    for (int r = 0; r < F; r++)
        for (int i = 0; i < h->sizes[r]; i++)
            for (int c = 0; c < F; c++) {
                or_csr *B = h->blk[r * F + c];
                if (!B) continue;
                for (int e = B->rp[i]; e < B->rp[i + 1]; e++) h->full->v[q++] = B->v[e];
            }
    h->status = ST_OK;
    for (int k = 0; k < F; k++) {
        int st = ST_OK;
        if (h->dgs[k]) {
            for (int i = 0; i < h->sizes[k]; i++) {
                double d = diag_of(h->blk[k * F + k], i);
                if (d == 0.0) st = ST_ZEROPIV;
                h->dgs[k][i] = 1.0 / d;
            }
        } else {
            st = h->ilu[k] ? or_ilu_update(h->ilu[k], h->blk[k * F + k])
                           : or_amg_update(h->amg[k], h->blk[k * F + k]->v, &h->opt);
        }
        if (st) h->status = st;
    }
    return h->status;
}

void or_bgs_free(or_bgs *h) {
    if (!h) return;
    for (int b = 0; b < 64; b++) or_csr_free(h->blk[b]);
    or_csr_free(h->full);
    for (int k = 0; k < 8; k++) {
        or_amg_free(h->amg[k]);
        or_ilu_free(h->ilu[k]);
        free(h->dgs[k]);
    }
    free(h);
}

void or_full_spmv(const or_bgs *h, const double *x, double *y) { or_spmv(h->full, x, y); }

/* The solver of diagonal block k applied to r (z = V_k(r) or the DD(0)-ILU(0) sweep), or its
 * transpose for the adjoint (V-cycle on the transposed level operators, same transfers, LU solved
 * transposed; the transposed ILU sweep). */
static void block_solve(const or_bgs *h, int k, const double *r, double *z, int transposed) {
    if (h->dgs[k]) {   /* diagonal solve (its own transpose) */
#pragma omp parallel for schedule(static)
        for (int i = 0; i < h->sizes[k]; i++) z[i] = h->dgs[k][i] * r[i];
        return;
    }
    if (h->ilu[k]) {
        if (transposed) or_ilu_apply_transposed(h->ilu[k], r, z);
        else or_ilu_apply(h->ilu[k], r, z);
        return;
    }
    if (!transposed) {
        or_vcycle(h->amg[k], r, z);
        return;
    }
    const or_amg *g = h->amg[k];
    or_csr *AT[OR_MAX_LEVELS] = {0};
    for (int l = 0; l + 1 < g->nlevels; l++) AT[l] = or_transpose(g->A[l]);
    vcycle_level(g, 0, r, z, 1, AT);
    for (int l = 0; l + 1 < g->nlevels; l++) or_csr_free(AT[l]);
}

/* r_k -= A_kj z_j (or, transposed, r_k -= A_jk^T z_j); r and z indexed from the field starts */
static void sub_coupling(const or_bgs *h, int k, int j, const double *zj, double *rk, int transposed) {
    int F = h->F;
    if (!transposed) {
        or_csr *B = h->blk[k * F + j];
        if (!B) return;
#pragma omp parallel for schedule(static)
        for (int i = 0; i < B->n; i++) {
            double t = 0.0;
            for (int e = B->rp[i]; e < B->rp[i + 1]; e++) t += B->v[e] * zj[B->ci[e]];
            rk[i] -= t;
        }
    } else {
        or_csr *B = h->blk[j * F + k]; /* A_jk, applied transposed */
        if (!B) return;
        for (int i = 0; i < B->n; i++)
            for (int e = B->rp[i]; e < B->rp[i + 1]; e++) rk[B->ci[e]] -= B->v[e] * zj[i];
    }
}

/* One sweep over the order positions [p0, p1) on vectors indexed from offset `base`: forward,
 * r_k = v_k - sum over earlier positions of A_kj z_j, z_k = block solve (block Jacobi: no
 * couplings); transposed, the reverse order with the transposed couplings of later positions. */
static void sweep_range(const or_bgs *h, int p0, int p1, int base, const double *v, double *z, int transposed) {
    for (int t = p0; t < p1; t++) {
        int p = transposed ? p1 - 1 - (t - p0) : t;
        int k = h->order[p];
        int nk = h->sizes[k];
        double *r = (double *)malloc(sizeof(double) * (size_t)nk);
#pragma omp parallel for schedule(static)
        for (int i = 0; i < nk; i++) r[i] = v[h->offs[k] - base + i];
        if (!h->opt.jacobi) {
            if (!transposed)
                for (int q = p0; q < p; q++) sub_coupling(h, k, h->order[q], z + h->offs[h->order[q]] - base, r, 0);
            else
                for (int q = p + 1; q < p1; q++) sub_coupling(h, k, h->order[q], z + h->offs[h->order[q]] - base, r, 1);
        }
        block_solve(h, k, r, z + h->offs[k] - base, transposed);
        free(r);
    }
}

/* Nested variant (Sec. 2.2: the block-triangular preconditioner over the groups of Eq.
 * hierarchical-bgs, each group's diagonal block solved by an inner FGMRES, preconditioned by the
 * group's own sweep, Eqs. non-voltage-bgs and voltage-bgs; Sec. 3.2 runs the outer FGMRES(5)).
 * Group g is the order positions [group_end[g-1], group_end[g]); its fields have consecutive ids,
 * so its vector is one contiguous slice. */
typedef struct {
    const or_bgs *h;
    int p0, p1, base, n, transposed;
} grp_ctx;

static void amul_group(void *ctx, const double *in, double *out) {
    const grp_ctx *c = (const grp_ctx *)ctx;
    const or_bgs *h = c->h;
    for (int i = 0; i < c->n; i++) out[i] = 0.0;
    for (int p = c->p0; p < c->p1; p++) {
        int k = h->order[p];
        for (int q = c->p0; q < c->p1; q++) {
            int j = h->order[q];
            /* out_k += A_kj in_j  (transposed: out_k += A_jk^T in_j) */
            double *ok = out + h->offs[k] - c->base;
            const double *ij = in + h->offs[j] - c->base;
            int nk = h->sizes[k];
            double *t = (double *)calloc((size_t)nk, sizeof(double));
            sub_coupling(h, k, j, ij, t, c->transposed);
            for (int i = 0; i < nk; i++) ok[i] -= t[i];
            free(t);
        }
    }
}

static void prec_group(void *ctx, const double *in, double *out) {
    const grp_ctx *c = (const grp_ctx *)ctx;
    sweep_range(c->h, c->p0, c->p1, c->base, in, out, c->transposed);
}

static void apply_nested(const or_bgs *h, const double *v, double *z, int transposed) {
    int G = h->opt.ngroups, F = h->F;
    for (int t = 0; t < G; t++) {
        int g = transposed ? G - 1 - t : t;
        int p0 = g ? h->opt.group_end[g - 1] : 0, p1 = h->opt.group_end[g];
        int base = h->offs[h->order[p0]], n = 0;
        for (int p = p0; p < p1; p++) {
            if (h->offs[h->order[p]] < base) base = h->offs[h->order[p]];
            n += h->sizes[h->order[p]];
        }
        double *r = (double *)malloc(sizeof(double) * (size_t)n);
        for (int i = 0; i < n; i++) r[i] = v[base + i];
        /* couplings to the groups already solved in this sweep */
        for (int p = p0; p < p1; p++) {
            int k = h->order[p];
            double *rk = r + h->offs[k] - base;
            if (!transposed)
                for (int q = 0; q < p0; q++) sub_coupling(h, k, h->order[q], z + h->offs[h->order[q]], rk, 0);
            else
                for (int q = p1; q < F; q++) sub_coupling(h, k, h->order[q], z + h->offs[h->order[q]], rk, 1);
        }
        grp_ctx c = {h, p0, p1, base, n, transposed};
        or_info info;
        or_fgmres(n, amul_group, &c, prec_group, &c, r, z + base, h->opt.inner_restart, h->opt.inner_maxit,
                  h->opt.inner_rtol, &info);
        free(r);
    }
}

/* z = M^-1 v: for k in order, r_k = v_k - sum_{pos(j) < pos(k)} A_kj z_j, z_k = V-cycle_k(r_k).
 * With opt.jacobi the couplings are left out (block Jacobi, the alternative Secs. 3.2 and 4
 * discuss): z_k = V-cycle_k(v_k).  With opt.ngroups > 0: the nested variant above. */
void or_bgs_apply(const or_bgs *h, const double *v, double *z) {
    if (h->opt.ngroups > 0) apply_nested(h, v, z, 0);
    else sweep_range(h, 0, h->F, 0, v, z, 0);
}

/* Transposed preconditioner for A^T: reverse order, upper couplings transposed,
 * V-cycle on A_kk^T (level operators transposed, same transfers, LU solved transposed). */
void or_bgs_apply_adjoint(const or_bgs *h, const double *v, double *z) {
    if (h->opt.ngroups > 0) apply_nested(h, v, z, 1);
    else sweep_range(h, 0, h->F, 0, v, z, 1);
}

/* ------------------------------------------------------------------------------------ */
/* Flexible GMRES(m), right preconditioned, modified Gram-Schmidt                        */
/* ------------------------------------------------------------------------------------ */
static double nrm2(int n, const double *x) { return sqrt(sum_prod(n, x, x)); }

int or_fgmres(int n, or_apply_fn amul, void *actx, or_apply_fn prec, void *pctx, const double *b, double *x,
              int m, int maxit, double rtol, or_info *info) {
    memset(info, 0, sizeof(*info));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) x[i] = 0.0;
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) {
        info->converged = 1;
        return ST_OK;
    }
    if (!(bnorm == bnorm) || isinf(bnorm)) {
        info->status = ST_NANINF;
        return ST_NANINF;
    }
    double *Vb = (double *)malloc(sizeof(double) * (size_t)n * (m + 1));
    double *Zb = (double *)malloc(sizeof(double) * (size_t)n * m);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *H = (double *)calloc((size_t)(m + 1) * m, sizeof(double));
    double *cs = (double *)malloc(sizeof(double) * (size_t)m);
    double *sn = (double *)malloc(sizeof(double) * (size_t)m);
    double *g = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)m);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) r[i] = b[i];
    double beta = bnorm;
    int it = 0, status = ST_NOCONV;
    double rel = 1.0, est = 1.0;
    for (;;) {
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; i++) Vb[i] = r[i] / beta;
        for (int k = 0; k <= m; k++) g[k] = 0.0;
        g[0] = beta;
        int jend = 0, breakdown = 0, nan = 0;
        for (int j = 0; j < m; j++) {
            double *vj = Vb + (size_t)j * n, *zj = Zb + (size_t)j * n;
            prec(pctx, vj, zj);
            amul(actx, zj, w);
            for (int i = 0; i <= j; i++) {
                double *vi = Vb + (size_t)i * n;
                double hij = sum_prod(n, w, vi);
                H[(size_t)i * m + j] = hij;
#pragma omp parallel for schedule(static)
                for (int t = 0; t < n; t++) w[t] -= hij * vi[t];
            }
            double hn = nrm2(n, w);
            H[(size_t)(j + 1) * m + j] = hn;
            it++;
            if (hn == 0.0) breakdown = 1;
            else {
#pragma omp parallel for schedule(static)
                for (int t = 0; t < n; t++) Vb[(size_t)(j + 1) * n + t] = w[t] / hn;
            }
            for (int i = 0; i < j; i++) {
                double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
            double den = sqrt(a * a + c * c);
            cs[j] = den == 0.0 ? 1.0 : a / den;
            sn[j] = den == 0.0 ? 0.0 : c / den;
            H[(size_t)j * m + j] = den;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            est = fabs(g[j + 1]) / bnorm;
            jend = j + 1;
            if (!(est == est)) {
                nan = 1;
                break;
            }
            if (est <= rtol || it >= maxit || breakdown) break;
        }
        if (nan) {
            status = ST_NANINF;
            break;
        }
        for (int i = jend - 1; i >= 0; i--) {
            double s = g[i];
            for (int k = i + 1; k < jend; k++) s -= H[(size_t)i * m + k] * y[k];
            y[i] = s / H[(size_t)i * m + i];
        }
        /* x_t += y_k z_k,t for k = 0, 1, ... in that order for every entry t */
#pragma omp parallel for schedule(static)
        for (int t = 0; t < n; t++)
            for (int k = 0; k < jend; k++) x[t] += y[k] * Zb[(size_t)k * n + t];
        amul(actx, x, r);
#pragma omp parallel for schedule(static)
        for (int t = 0; t < n; t++) r[t] = b[t] - r[t];
        beta = nrm2(n, r);
        rel = beta / bnorm;
        if (!(rel == rel)) {
            status = ST_NANINF;
            break;
        }
        if (rel <= rtol) {
            status = ST_OK;
            break;
        }
        if (it >= maxit) {
            status = ST_NOCONV;
            break;
        }
        if (breakdown && beta == 0.0) {
            status = ST_BREAKDOWN;
            break;
        }
    }
    info->iters = it;
    info->converged = status == ST_OK;
    info->status = status;
    info->rel_true_resid = rel;
    info->rel_est_resid = est;
    free(Vb);
    free(Zb);
    free(w);
    free(r);
    free(H);
    free(cs);
    free(sn);
    free(g);
    free(y);
    return status;
}

static void amul_full(void *ctx, const double *in, double *out) { or_spmv(((const or_bgs *)ctx)->full, in, out); }
static void prec_bgs(void *ctx, const double *in, double *out) { or_bgs_apply((const or_bgs *)ctx, in, out); }

typedef struct {
    const or_bgs *h;
    or_csr *AT;
} adj_ctx;
static void amul_fullT(void *ctx, const double *in, double *out) { or_spmv(((adj_ctx *)ctx)->AT, in, out); }
static void prec_bgsT(void *ctx, const double *in, double *out) { or_bgs_apply_adjoint(((adj_ctx *)ctx)->h, in, out); }

int or_bgs_solve(const or_bgs *h, const double *b, double *x, or_info *info) {
    int n = h->offs[h->F];
    return or_fgmres(n, amul_full, (void *)h, prec_bgs, (void *)h, b, x, h->opt.restart, h->opt.maxit,
                     h->opt.rtol, info);
}

int or_bgs_solve_adjoint(const or_bgs *h, const double *g, double *lam, or_info *info) {
    int n = h->offs[h->F];
    adj_ctx c = {h, or_transpose(h->full)};
    int st = or_fgmres(n, amul_fullT, &c, prec_bgsT, &c, g, lam, h->opt.restart, h->opt.maxit, h->opt.rtol, info);
    or_csr_free(c.AT);
    return st;
}

/* dL/da_ij = -lambda_i x_j on the pattern of block A (row offset roff, column offset coff) */
void or_grad_values(const or_csr *A, int roff, int coff, const double *lam, const double *x, double *g) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < A->n; i++)
        for (int e = A->rp[i]; e < A->rp[i + 1]; e++) g[e] = -(lam[roff + i] * x[coff + A->ci[e]]);
}
