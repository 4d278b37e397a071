// Host-side interfaces between the translation units of libbgs.
#pragma once
#include "common.cuh"

namespace bgs {

// Non-owning CSR view (FP64 values).
struct CsrView {
    int n = 0, m = 0;
    int64_t nnz = 0;
    const int *rp = nullptr, *ci = nullptr;
    const double *v = nullptr;
};
inline CsrView view(const DCsr &A) { return CsrView{A.n, A.m, A.nnz, A.rp.p, A.ci.p, A.v.p}; }

// Reusable device scratch for reductions and flags (one per handle).
struct Scratch {
    DBuf<double> partial;   // per-block partial sums
    DBuf<double> scal;      // device scalars
    DBuf<int> flags;        // device integer flags / counters
    DBuf<int> iscan;        // scan block sums
    DBuf<double> pinned_dummy;
    double *h_scal = nullptr;  // pinned host mirror
    int *h_flags = nullptr;
    // a second stream for work that overlaps the owner's stream (forked and joined by events), at
    // the owner stream's priority
    cudaStream_t owner = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr;
    void init(cudaStream_t s);
    void ensure_side();
    ~Scratch();
};

// ---------------------------------------------------------------- util.cu
// One piece of a host <-> device (or device <-> device) copy.
struct XferSeg {
    const void *src;
    void *dst;
    size_t bytes;
};
// Enqueues the copies on s: pieces to or from pinned host memory (16-byte aligned) are moved by one
// kernel through the SMs over the host link; the others by cudaMemcpyAsync (cudaMemcpyDefault).
void transfer(const std::vector<XferSeg> &segs, cudaStream_t s);
long long launch_count();
void release_cached_memory();
// out[0..n] = exclusive scan of in[0..n-1] (out[n] = total); in and out may alias.
// Returns the total (synchronises the stream).  Throws if the total exceeds INT32_MAX.
int64_t scan_exclusive(const int *in, int *out, int64_t n, Scratch &sc, cudaStream_t s);
// a[0..n] = exclusive scan of a[0..n-1] in place (a has n + 1 entries; one block); returns a[n]
// (synchronises the stream)
long long scan_ll_inplace(long long *a, int n, cudaStream_t s);
// sum of squares / dot products into a device scalar (deterministic two-pass reduction).
void dev_dot(const double *a, const double *b, int64_t n, double *out, Scratch &sc, cudaStream_t s);
// the same, and out[1] = 1/sqrt(out[0]) (0 when out[0] is 0)
void dev_dot_rsqrt(const double *a, const double *b, int64_t n, double *out, Scratch &sc, cudaStream_t s);
// both with a caller's partial-sum buffer (num_sms() * 4 doubles) instead of the scratch's, for a
// second stream
void dev_dot(const double *a, const double *b, int64_t n, double *out, double *partial, cudaStream_t s);
void dev_dot_rsqrt(const double *a, const double *b, int64_t n, double *out, double *partial, cudaStream_t s);
void dev_fill_int(int *p, int value, int64_t n, cudaStream_t s);
void dev_fill_double(double *p, double value, int64_t n, cudaStream_t s);
// Validation of one CSR (device arrays); returns 0 or BGS_INVALID_ARG.  Checks monotone rowptr,
// rowptr[0] = 0, rowptr[n] = nnz, columns in range and strictly increasing, and (need_diag) that
// every row stores its diagonal.
int validate_csr(const CsrView &A, bool need_diag, Scratch &sc, cudaStream_t s);
// the validation kernel alone, its error bits in *flag (cleared first); validate_status maps them
void validate_csr_launch(const CsrView &A, bool need_diag, int *flag, cudaStream_t s);
int validate_status(int flag);
// C = row-wise concatenation of blocks: row i of C = row i of parts[0] (columns + offs[0]), then
// row i of parts[1] ... (all parts have n rows; columns stay sorted if offsets increase).
void concat_rows(int n, int nparts, const CsrView *parts, const int *col_offs, DCsr &C, Scratch &sc,
                 cudaStream_t s);
// the two passes of concat_rows into caller-owned arrays: the row lengths into cnt[0..n), then,
// given the row starts rp[0..n] (absolute positions in ci, v), the entries
void concat_count(int n, int nparts, const CsrView *parts, int *cnt, cudaStream_t s);
void concat_fill(int n, int nparts, const CsrView *parts, const int *col_offs, const int *rp, int *ci, double *v,
                 cudaStream_t s);
void convert_d2f(const double *in, float *out, int64_t n, cudaStream_t s);
void convert_d2bf(const double *in, __nv_bfloat16 *out, int64_t n, cudaStream_t s);
void copy_d2f(const double *in, float *out, int64_t n, cudaStream_t s);
void copy_f2d(const float *in, double *out, int64_t n, cudaStream_t s);
// out = (double) in and out_f = in (an FP32 output kept beside its FP64 copy)
void copy_f2d_keep(const float *in, double *out, float *out_f, int64_t n, cudaStream_t s);
void extract_diag(const CsrView &A, double *diag, cudaStream_t s);
void reciprocal(const double *in, double *out, int64_t n, cudaStream_t s);
// dvals[e] = -lam[roff + i] * x[coff + j]
void grad_outer(const CsrView &A, const double *lam, const double *x, double *dvals, cudaStream_t s);

// ---------------------------------------------------------------- spmv.cu
int choose_lanes(int64_t nrows, int64_t nnz);
// y = A x (FP64)
void spmv_f64(const CsrView &A, int lanes, const double *x, double *y, cudaStream_t s);
// Kernels on a stored operator; VT selects its value copy (double / float / bf16), XT the vector
// type.  SELL-32 is used when the matrix has it, CSR otherwise.
template <class VT, class XT>
void spmv_store(const DCsr &A, const XT *x, XT *y, cudaStream_t s);
template <class VT, class XT>
void spmv_resid(const DCsr &A, const XT *b, const XT *x, XT *r, cudaStream_t s);
template <class VT, class XT>
void spmv_addto(const DCsr &A, const XT *x, XT *y, cudaStream_t s);
template <class VT, class XT>
void cheb_step(const DCsr &A, const XT *b, const XT *dinv, const XT *xin, XT *xout, XT *e, double alpha,
               double scale, bool first, cudaStream_t s);
template <class XT>
void cheb_first(int n, const XT *b, const XT *dinv, double inv_theta, XT *x, XT *e, cudaStream_t s);
// r = v - L z (L with global columns into z), v FP64, z FP64 or its FP32 copy, output typed
template <class VT, class XT, class ZT>
void coupling_sub(const DCsr &L, const double *v, const ZT *z, XT *r, cudaStream_t s);
// The same products with the first Chebyshev step from x = 0 of the level they write the right-hand
// side of fused into the epilogue (e = D^-1 b, x = e / theta): the restriction y = R r onto a level,
// the coupling subtraction onto a block's finest level, and a plain copy b = v for a block without
// couplings.
template <class XT>
struct FirstStep {
    const XT *dinv;   // the level's D^-1
    XT *x, *e;        // the step's outputs
    double inv_theta;
};
template <class VT, class XT>
void spmv_store_first(const DCsr &A, const XT *x, XT *y, const FirstStep<XT> &f, cudaStream_t s);
template <class VT, class XT, class ZT>
void coupling_sub_first(const DCsr &L, const double *v, const ZT *z, XT *r, const FirstStep<XT> &f,
                        cudaStream_t s);
template <class XT>
void copy_in_first(const double *v, XT *b, int64_t n, const FirstStep<XT> &f, cudaStream_t s);
// w_i = dinv_i * (A v)_i (FP64, power iteration)
void spmv_scaled(const CsrView &A, const double *dinv, const double *v, double *w, cudaStream_t s);
// w_i = dinv_i * (A v)_i * (*rnorm), rnorm = 1/||v|| on the device (power iteration step on a
// normalised v; CSR with a lane count fixed by the shape, whatever format the operator is stored in)
void spmv_scaled_norm(const DCsr &A, const double *dinv, const double *v, const double *rnorm, double *w,
                      cudaStream_t s);
// y = W x, W dense row-major n x n in FP64
template <class XT>
void dense_gemv(int n, const double *W, const XT *x, XT *y, cudaStream_t s);
// Builds the SELL-32 copy when its padding stays within max_pad * nnz (returns whether built);
// sell_refresh re-gathers the FP32 / BF16 value copies after they are created.
bool build_sell(DCsr &A, double max_pad, Scratch &sc, cudaStream_t s);
// Builds the diagonal-offset SELL-32 copy when every slice has at most 32 distinct offsets and the
// slots stay within max_pad * nnz (returns whether built).  Only for operators whose input vectors
// are fully written when they are applied (a padded slot reads a neighbouring entry times 0).
bool build_dia(DCsr &A, double max_pad, Scratch &sc, cudaStream_t s);
void drop_dia(DCsr &A);
// re-gathers the FP32 / BF16 value copies of the SELL forms after those copies are created
void sell_refresh(DCsr &A, cudaStream_t s);
// After A.v changed in place: re-derive the FP32 / BF16 copies that exist and re-gather every
// SELL value copy (no allocation when the copies exist).
void refresh_values(DCsr &A, cudaStream_t s);
// Times the diagonal-offset SELL-32 and SELL-32 (if built) and CSR with 1..32 lanes per row, each at
// 128, 256 and 512 threads per block, and keeps the fastest for A (cached per shape); returns -1
// (diagonal-offset SELL), 0 (SELL-32) or the lane count.  value_bytes selects the precision timed
// (8 FP64, 4 FP32 hierarchy, 2 BF16 couplings).
// product: time y = A x instead of the Chebyshev step (an operator only ever applied as a product).
// BGS_TRACE=async: one timeline line (host clock since the first mark, stream) to stderr
void timeline_mark(const char *what, cudaStream_t s);
int autotune_spmv(DCsr &A, int value_bytes, Scratch &sc, cudaStream_t s, bool product = false);
// Builds the SpMV layouts an operator may run: the one the autotuner's cached choice for its shape
// names (use_cache), else SELL-32 and, with allow_dia, the diagonal-offset SELL-32 for the
// autotuner to time.  value_bytes as for autotune_spmv.
// bsr_fields: F > 0 for the full operator of F equal fields (the node-block layout is then a
// candidate too).
void build_formats(DCsr &A, int value_bytes, bool allow_dia, bool use_cache, Scratch &sc, cudaStream_t s,
                   bool product = false, int bsr_fields = 0);
// Builds the field-interleaved node-block copy of the full operator of F fields of equal size (F x F
// blocks per node pair, at most 32 block columns per node) when its stored block entries stay
// within max_pad * nnz (returns whether built).
bool build_bsr(DCsr &A, int F, double max_pad, Scratch &sc, cudaStream_t s);
void drop_bsr(DCsr &A);

// ---------------------------------------------------------------- krylov.cu
// h[k] = V_k . w for k < cnt and h[cnt] = w . w (V column-major, leading dimension ld, even; V and w
// 16-byte aligned), with a caller-provided partial-sum buffer of partial_cap doubles that needs
// arnoldi_dots_scratch(cnt, n, max_blocks) doubles and need not be cleared; max_blocks caps the
// grid (0: three blocks per multiprocessor).
void arnoldi_dots_into(const double *V, int64_t ld, int cnt, const double *w, int64_t n, double *h, double *partial,
                       size_t partial_cap, int max_blocks, cudaStream_t s);
size_t arnoldi_dots_scratch(int cnt, int64_t n, int max_blocks);
// One Gram-Schmidt pass of the FGMRES orthogonalisation with the solver's kernels (the FP64 /
// fixed-point split; basis entries below 2 in magnitude): h = V^T w (cnt + 1 entries, h[cnt] =
// ||w||^2), w -= V h, *nw = ||w||^2 after; partial holds gs_pass_scratch(cnt, n) doubles.
size_t gs_pass_scratch(int cnt, int64_t n);
void gs_pass(const double *V, int64_t ld, int cnt, double *w, int64_t n, double *h, double *nw, double *partial,
             size_t partial_cap, cudaStream_t s);

// FGMRES(m) state in device memory (one per Krylov workspace); m <= kMaxRestart.
constexpr int kMaxRestart = 63;
constexpr int kHld = kMaxRestart + 1;   // leading dimension of the Hessenberg matrix
struct FgState {
    int j;          // column of the current step within the cycle
    int cnt;        // j + 1: basis vectors the step orthogonalises against
    int it;         // iterations so far (all cycles)
    int jend;       // columns done in this cycle
    int stop;       // the cycle ends after this step
    int flag;       // why: 1 estimate <= rtol, 2 maxit, 3 breakdown, 4 NaN/Inf, 5 restart length
    int reorth;     // steps that ran the second Gram-Schmidt pass
    int need2;      // this step runs the second pass
    int m, maxit;
    double rtol, eta2, bnorm, est, inv_hn;
    double nw1, nw2;                 // ||w||^2 after the first / second pass
    double h1[kHld + 8], h2[kHld + 8];   // dots of the passes (h[cnt] = ||w||^2 before the pass)
    double cs[kHld], sn[kHld], g[kHld + 1], y[kHld];
    double H[(kHld + 1) * kHld];     // rotated Hessenberg matrix, row-major [i * kHld + j]
};
// start of a solve: restart length, iteration limit, tolerance, eta^2 of the re-orthogonalisation
// test, ||b||; iteration and re-orthogonalisation counts reset
void fg_init(FgState *st, int m, int maxit, double rtol, double eta2, double bnorm, cudaStream_t s);
// start of a cycle: state reset with g_0 = beta, V_0 = r / beta (and stage = V_0 when given)
void fg_begin(FgState *st, const double *r, double beta, double *V, double *stage, int64_t n, cudaStream_t s);
// column j of Z from the staging vector (j read on the device)
void fg_store_z(const FgState *st, const double *src, double *Z, int64_t ld, int64_t n, cudaStream_t s);
// the Gram-Schmidt passes of step j on w = A z_j (second pass by the re-orthogonalisation test, or
// always); m = the restart length (the largest basis a step can see)
void fg_orthogonalise(FgState *st, const double *V, int64_t ld, int m, double *w, int64_t n, bool always,
                      Scratch &sc, cudaStream_t s);
// the scalar part of the step and v_{j+1} = w / h_{j+1,j} (into stage too when given); with
// use_loop the step sets the WHILE condition of the captured cycle (0 when the cycle ends)
void fg_step(FgState *st, cudaGraphConditionalHandle loop, bool use_loop, const double *w, double *V, int64_t ld,
             double *stage, int64_t n, cudaStream_t s);
// after the cycle: y from the triangular system, x += Z y
void fg_finish_cycle(FgState *st, const double *Z, int64_t ld, double *x, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------- amg_setup.cu
struct Level {
    DCsr A, P, R, AT;
    DBuf<int> agg;
    DBuf<uint8_t> strong;   // strength flag per stored entry of A (the attempt that was kept)
    int nagg = 0, mis_rounds = 0;
    double omega = 0.0;
    DBuf<double> dinv;
    DBuf<float> dinvf;
    double lmin = 0.0, lmax = 0.0;
    double lim = 0.0;       // imaginary semi-axis of the smoother's ellipse (0: the real interval)
    // V-cycle work vectors (FP64 or FP32 by precision)
    DBuf<double> b, x0, x1, d, r;
    DBuf<float> fb, fx0, fx1, fd, fr;
};

// DD(0)-ILU(0) factors of one diagonal block: the subdomain-restricted pattern with L (unit,
// strictly lower) and U in place, and per subdomain of R rows the level schedules of the forward
// and backward sweeps (R + 1 level slots per subdomain).
constexpr int kIluMaxRows = 8192;
struct IluFactors {
    DCsr F;
    int R = 0, nsub = 0;
    DBuf<int> fptr, bptr, fsched, bsched, nlf, nlb;
};

struct Hier {
    std::vector<Level> L;
    int solver = 0;         // 0 SA-AMG V-cycle, 1 DD(0)-ILU(0) (then L holds level 0 only)
    IluFactors ilu, iluT;   // the DD(0)-ILU(0) factors and their transpose (adjoint, built on use)
    int degree = 2;
    int nc = 0;
    DBuf<double> inv;      // dense inverse of the coarsest operator, row-major nc x nc
    DBuf<double> invT;     // its transpose (adjoint V-cycle), built on first use
    int status = 0;
    const DBuf<double> &inv_T() const { return invT; }
    void build_inv_T(cudaStream_t s);
};

struct AmgParams {
    double theta;
    int degree, max_coarse, max_levels, power_iters, filter_diag;
    double cheb_ratio, cheb_boost;
    int cheb_ellipse;
    int fp32_galerkin;   // mixed precision: A P and R (A P) in FP32 from FP32 copies of A_l, P_l, R_l
};

constexpr int kMaxLevels = 16;
// ---------------------------------------------------------------- ilu.cu
void ilu_setup(IluFactors &M, const DCsr &A, int R, bool mixed, Scratch &sc, cudaStream_t s);
void ilu_update(IluFactors &M, const DCsr &A, Scratch &sc, cudaStream_t s);
void ilu_build_transposed(const IluFactors &M, IluFactors &T, Scratch &sc, cudaStream_t s);
// z = (L U)^-1 r per subdomain (transposed: the transposed factors T, (U^T)^-1 then (L^T)^-1)
template <class XT>
void ilu_apply(const IluFactors &M, bool transposed, const XT *r, XT *z, cudaStream_t s);

// Builds the hierarchy on the level-0 operator already stored in H.L[0].A.
void amg_build(Hier &H, const AmgParams &p, Scratch &sc, cudaStream_t s);
// Numeric re-set-up: H.L[0].A holds new values on its old pattern (value copies refreshed); the
// strength flags and aggregates of every level are kept and every numeric quantity is recomputed
// in place (P_l, R_l, A_l+1 values, smoother bounds, coarsest inverse).
void amg_update(Hier &H, const AmgParams &p, Scratch &sc, cudaStream_t s);
// dst takes src's values (same shape and pattern; a pattern difference sets device flag slot 10 of
// sc, which the caller clears before and reads after) and refreshes its value copies.
void take_values(DCsr &dst, const DCsr &src, Scratch &sc, cudaStream_t s);
void transpose_csr(const CsrView &A, DCsr &T, Scratch &sc, cudaStream_t s);
// SELL-32 is used for an operator when its padding adds at most this factor to the stored entries
constexpr double kMaxPad = 2.0;
// the diagonal-offset SELL-32 copy is built when its slots stay within this factor of the entries
constexpr double kMaxPadDia = 1.5;
// The node-block copy stores F^2 values per block, and its kernel multiplies every one of them: it is
// built as an autotuner candidate while that stays within this factor of the stored entries (the
// 128^3 workload's full operator, with 5 x 5 blocks of which the off-node ones hold their diagonal
// only, is at 3.1x and timed 2.7x slower than the diagonal-offset SELL-32), and up to the larger
// factor when a cached choice names it.
constexpr double kMaxPadBsr = 1.5;
constexpr double kMaxPadBsrForced = 8.0;

}  // namespace bgs
