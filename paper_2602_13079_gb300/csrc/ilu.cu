// DD(0)-ILU(0) subblock solver (Sec. 2.1, Eq. one-level-schwarz with no overlap, D_i = I; the species
// solver of Sec. 3.1.1): the rows are cut into subdomains of R consecutive rows, each subdomain
// matrix A_i = R_i A R_i^T (entries coupling two subdomains dropped) is factored by ILU(0), and one
// application is L_i y = r_i, U_i z_i = y for every subdomain at once.
//
// GPU form: one CTA per subdomain.  The triangular dependencies inside a subdomain are scheduled by
// level (level(i) = 1 + max level(k) over the stored k < i of row i; the backward sweep likewise
// over k > i), computed once at set-up; a CTA then sweeps its levels in order with the rows of a
// level in parallel, the subdomain's vector in shared memory.  The factorisation runs on the same
// schedule, row by row in the order and with the unfused operations of the plain IKJ algorithm, so
// its factors are bit-identical to a sequential ILU(0).
#include <mutex>

#include "internal.h"

namespace bgs {

namespace {

constexpr int kSchedT = 32;    // threads of the scheduling kernel (lane 0 works)
constexpr int kFactT = 128;    // threads per subdomain in the factorisation
constexpr int kSolveT = 64;    // threads per subdomain in the sweeps

__global__ void k_dd_count(int n, int R, const int *rp, const int *ci, int *cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = i / R;
        int c = 0;
        for (int e = rp[i]; e < rp[i + 1]; e++) c += ci[e] / R == s;
        cnt[i] = c;
    }
}

__global__ void k_dd_fill(int n, int R, const int *rp, const int *ci, const double *v, const int *frp, int *fci,
                          double *fv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = i / R;
        int q = frp[i];
        for (int e = rp[i]; e < rp[i + 1]; e++)
            if (ci[e] / R == s) {
                fci[q] = ci[e];
                if (fv) fv[q] = v[e];
                q++;
            }
    }
}

// values of A restricted to the subdomains, in the stored order of F (same pattern)
__global__ void k_dd_values(int n, int R, const int *rp, const int *ci, const double *v, const int *frp, double *fv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = i / R;
        int q = frp[i];
        for (int e = rp[i]; e < rp[i + 1]; e++)
            if (ci[e] / R == s) fv[q++] = v[e];
    }
}

// One CTA per subdomain, lane 0 working: forward levels over the strictly lower entries, backward
// levels over the strictly upper ones, then a counting sort of the rows by level.  ptr has R + 1
// slots per subdomain (level l of subdomain s: rows sched[ptr[s(R+1)+l] .. ptr[s(R+1)+l+1]) ).
__global__ void k_dd_schedule(int n, int R, const int *rp, const int *ci, int *fptr, int *fsched, int *nlf,
                              int *bptr, int *bsched, int *nlb) {
    extern __shared__ int lv[];        // R levels, then R counters
    int *cnt = lv + R;
    if (threadIdx.x != 0) return;
    const int s = blockIdx.x, r0 = s * R, r1 = min(n, r0 + R), m = r1 - r0;
    for (int pass = 0; pass < 2; pass++) {
        const bool fwd = pass == 0;
        int maxl = 0;
        for (int t = 0; t < m; t++) {
            const int i = fwd ? r0 + t : r1 - 1 - t;
            int l = 0;
            for (int e = rp[i]; e < rp[i + 1]; e++) {
                const int c = ci[e];
                if (fwd ? c < i : c > i) l = max(l, lv[c - r0] + 1);
            }
            lv[i - r0] = l;
            maxl = max(maxl, l);
        }
        const int nl = maxl + 1;
        for (int l = 0; l < nl; l++) cnt[l] = 0;
        for (int t = 0; t < m; t++) cnt[lv[t]]++;
        int *ptr = (fwd ? fptr : bptr) + (size_t)s * (R + 1);
        int *sched = fwd ? fsched : bsched;
        int p = r0;
        for (int l = 0; l < nl; l++) {
            ptr[l] = p;
            const int c = cnt[l];
            cnt[l] = p;      // cursor
            p += c;
        }
        ptr[nl] = p;
        for (int t = 0; t < m; t++) {
            const int i = fwd ? r0 + t : r1 - 1 - t;
            sched[cnt[lv[i - r0]]++] = i;
        }
        (fwd ? nlf : nlb)[s] = nl;
    }
}

// ILU(0) in place on the forward schedule: row i (all its lower neighbours already final) takes
// l_ik = a_ik / u_kk for each stored k < i in column order, then a_ij -= l_ik u_kj for the later
// entries j of row i that row k also stores.  Products and differences are separately rounded,
// as in the sequential algorithm.
__global__ void __launch_bounds__(kFactT) k_ilu0(int R, const int *rp, const int *ci, double *v, const int *fptr,
                                                 const int *fsched, const int *nlf, int *status) {
    const int s = blockIdx.x;
    const int *ptr = fptr + (size_t)s * (R + 1);
    const int nl = nlf[s];
    for (int l = 0; l < nl; l++) {
        for (int t = ptr[l] + threadIdx.x; t < ptr[l + 1]; t += blockDim.x) {
            const int i = fsched[t];
            const int ie = rp[i + 1];
            for (int e = rp[i]; e < ie && ci[e] < i; e++) {
                const int k = ci[e], ke = rp[k + 1];
                int dk = -1;
                for (int f = rp[k]; f < ke; f++)
                    if (ci[f] == k) dk = f;
                if (dk < 0 || v[dk] == 0.0) {
                    *status = 1;
                    continue;
                }
                const double lik = v[e] / v[dk];
                v[e] = lik;
                int f = dk + 1;
                for (int g = e + 1; g < ie; g++) {
                    const int cg = ci[g];
                    while (f < ke && ci[f] < cg) f++;
                    if (f < ke && ci[f] == cg) v[g] = __dsub_rn(v[g], __dmul_rn(lik, v[f]));
                }
            }
        }
        __syncthreads();
    }
}

__global__ void k_ilu0_diag_check(int n, const int *rp, const int *ci, const double *v, int *status) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        bool ok = false;
        for (int e = rp[i]; e < rp[i + 1]; e++)
            if (ci[e] == i) ok = v[e] != 0.0;
        if (!ok) *status = 1;
    }
}

// sweep arithmetic type: FP64 for FP64 vectors, FP32 for FP32 vectors
template <class XT>
struct SweepT { using T = double; };
template <>
struct SweepT<float> { using T = float; };

__device__ __forceinline__ double mulsub(double acc, double a, double b) { return __dsub_rn(acc, __dmul_rn(a, b)); }
__device__ __forceinline__ float mulsub(float acc, float a, float b) { return acc - a * b; }

// Both triangular sweeps of one subdomain per CTA.  UNIT_L: the forward sweep's diagonal is 1
// (L of LU); otherwise it divides by the stored diagonal (U^T of the transposed factors).  UNIT_U
// likewise for the backward sweep.  Each row sums its terms in stored (column) order.
template <class VT, class XT, bool UNIT_L, bool UNIT_U>
__global__ void __launch_bounds__(kSolveT) k_dd_solve(int n, int R, const int *__restrict__ rp, const int *__restrict__ ci,
                                                      const VT *__restrict__ val, const int *__restrict__ fptr,
                                                      const int *__restrict__ fsched, const int *__restrict__ nlf,
                                                      const int *__restrict__ bptr, const int *__restrict__ bsched,
                                                      const int *__restrict__ nlb, const XT *__restrict__ r,
                                                      XT *__restrict__ z) {
    using CT = typename SweepT<XT>::T;
    extern __shared__ unsigned char smraw[];
    CT *y = reinterpret_cast<CT *>(smraw);
    const int s = blockIdx.x, r0 = s * R, r1 = min(n, r0 + R), m = r1 - r0;
    for (int t = threadIdx.x; t < m; t += blockDim.x) y[t] = (CT)r[r0 + t];
    __syncthreads();
    const int *fp = fptr + (size_t)s * (R + 1);
    const int nf = nlf[s];
    for (int l = 0; l < nf; l++) {
        for (int t = fp[l] + threadIdx.x; t < fp[l + 1]; t += blockDim.x) {
            const int i = fsched[t];
            CT acc = y[i - r0], d = (CT)1;
            for (int e = rp[i]; e < rp[i + 1]; e++) {
                const int c = ci[e];
                if (c < i) acc = mulsub(acc, (CT)to_d(val[e]), y[c - r0]);
                else {
                    if (!UNIT_L && c == i) d = (CT)to_d(val[e]);
                    break;
                }
            }
            y[i - r0] = UNIT_L ? acc : acc / d;
        }
        __syncthreads();
    }
    const int *bp = bptr + (size_t)s * (R + 1);
    const int nb = nlb[s];
    for (int l = 0; l < nb; l++) {
        for (int t = bp[l] + threadIdx.x; t < bp[l + 1]; t += blockDim.x) {
            const int i = bsched[t];
            CT acc = y[i - r0], d = (CT)1;
            for (int e = rp[i]; e < rp[i + 1]; e++) {
                const int c = ci[e];
                if (c == i) d = (CT)to_d(val[e]);
                else if (c > i) acc = mulsub(acc, (CT)to_d(val[e]), y[c - r0]);
            }
            y[i - r0] = UNIT_U ? acc : acc / d;
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < m; t += blockDim.x) z[r0 + t] = (XT)y[t];
}

template <class VT, class XT, bool UL, bool UU>
void set_solve_smem() {
    CK(cudaFuncSetAttribute(k_dd_solve<VT, XT, UL, UU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)(sizeof(double) * kIluMaxRows)));
}

void set_attributes() {
    static std::once_flag once;
    std::call_once(once, [] {
        CK(cudaFuncSetAttribute(k_dd_schedule, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(int) * 2 * kIluMaxRows)));
        set_solve_smem<double, double, true, false>();
        set_solve_smem<double, double, false, true>();
        set_solve_smem<float, float, true, false>();
        set_solve_smem<float, float, false, true>();
    });
}

void schedule(IluFactors &M, cudaStream_t s) {
    const int n = M.F.n, R = M.R;
    M.nsub = (n + R - 1) / R;
    const size_t slots = (size_t)M.nsub * (R + 1);
    M.fptr.alloc(slots, s);
    M.bptr.alloc(slots, s);
    M.fsched.alloc((size_t)std::max(n, 1), s);
    M.bsched.alloc((size_t)std::max(n, 1), s);
    M.nlf.alloc((size_t)M.nsub, s);
    M.nlb.alloc((size_t)M.nsub, s);
    k_dd_schedule<<<M.nsub, kSchedT, sizeof(int) * 2 * (size_t)R, s>>>(n, R, M.F.rp.p, M.F.ci.p, M.fptr.p, M.fsched.p,
                                                                         M.nlf.p, M.bptr.p, M.bsched.p, M.nlb.p);
    CK_LAUNCH();
}

void factor(IluFactors &M, Scratch &sc, cudaStream_t s) {
    const int n = M.F.n;
    CK(cudaMemsetAsync(sc.flags.p + 11, 0, sizeof(int), s));
    k_ilu0<<<M.nsub, kFactT, 0, s>>>(M.R, M.F.rp.p, M.F.ci.p, M.F.v.p, M.fptr.p, M.fsched.p, M.nlf.p,
                                      sc.flags.p + 11);
    CK_LAUNCH();
    k_ilu0_diag_check<<<grid_for(n, 256), 256, 0, s>>>(n, M.F.rp.p, M.F.ci.p, M.F.v.p, sc.flags.p + 11);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(sc.h_flags + 11, sc.flags.p + 11, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (sc.h_flags[11]) throw Error(BGS_ZERO_PIVOT, "zero pivot in the ILU(0) factorisation");
}

}  // namespace

void ilu_setup(IluFactors &M, const DCsr &A, int R, bool mixed, Scratch &sc, cudaStream_t s) {
    set_attributes();
    if (R < 1 || R > kIluMaxRows) throw Error(BGS_INVALID_ARG, "ilu_rows outside 1..8192");
    const int n = A.n;
    M = IluFactors();
    M.R = R;
    DCsr &F = M.F;
    F.n = F.m = n;
    F.rp.alloc((size_t)n + 1, s);
    k_dd_count<<<grid_for(n, 256), 256, 0, s>>>(n, R, A.rp.p, A.ci.p, F.rp.p);
    CK_LAUNCH();
    F.nnz = scan_exclusive(F.rp.p, F.rp.p, n, sc, s);
    F.ci.alloc((size_t)F.nnz, s);
    F.v.alloc((size_t)F.nnz, s);
    k_dd_fill<<<grid_for(n, 256), 256, 0, s>>>(n, R, A.rp.p, A.ci.p, A.v.p, F.rp.p, F.ci.p, F.v.p);
    CK_LAUNCH();
    schedule(M, s);
    factor(M, sc, s);
    if (mixed) {
        F.vf.alloc((size_t)F.nnz, s);
        convert_d2f(F.v.p, F.vf.p, F.nnz, s);
    }
}

void ilu_update(IluFactors &M, const DCsr &A, Scratch &sc, cudaStream_t s) {
    const int n = A.n;
    k_dd_values<<<grid_for(n, 256), 256, 0, s>>>(n, M.R, A.rp.p, A.ci.p, A.v.p, M.F.rp.p, M.F.v.p);
    CK_LAUNCH();
    factor(M, sc, s);
    if (M.F.vf.p) convert_d2f(M.F.v.p, M.F.vf.p, M.F.nnz, s);
}

void ilu_build_transposed(const IluFactors &M, IluFactors &T, Scratch &sc, cudaStream_t s) {
    T = IluFactors();
    T.R = M.R;
    transpose_csr(view(M.F), T.F, sc, s);
    schedule(T, s);
    if (M.F.vf.p) {
        T.F.vf.alloc((size_t)T.F.nnz, s);
        convert_d2f(T.F.v.p, T.F.vf.p, T.F.nnz, s);
    }
}

template <class XT>
void ilu_apply(const IluFactors &M, bool transposed, const XT *r, XT *z, cudaStream_t s) {
    const DCsr &F = M.F;
    if (F.n <= 0) return;
    const size_t smem = sizeof(typename SweepT<XT>::T) * (size_t)M.R;
    if (sizeof(XT) == sizeof(double)) {
        const double *v = F.v.p;
        if (!transposed)
            k_dd_solve<double, XT, true, false><<<M.nsub, kSolveT, smem, s>>>(
                F.n, M.R, F.rp.p, F.ci.p, v, M.fptr.p, M.fsched.p, M.nlf.p, M.bptr.p, M.bsched.p, M.nlb.p, r, z);
        else
            k_dd_solve<double, XT, false, true><<<M.nsub, kSolveT, smem, s>>>(
                F.n, M.R, F.rp.p, F.ci.p, v, M.fptr.p, M.fsched.p, M.nlf.p, M.bptr.p, M.bsched.p, M.nlb.p, r, z);
    } else {
        const float *v = F.vf.p;
        if (!transposed)
            k_dd_solve<float, XT, true, false><<<M.nsub, kSolveT, smem, s>>>(
                F.n, M.R, F.rp.p, F.ci.p, v, M.fptr.p, M.fsched.p, M.nlf.p, M.bptr.p, M.bsched.p, M.nlb.p, r, z);
        else
            k_dd_solve<float, XT, false, true><<<M.nsub, kSolveT, smem, s>>>(
                F.n, M.R, F.rp.p, F.ci.p, v, M.fptr.p, M.fsched.p, M.nlf.p, M.bptr.p, M.bsched.p, M.nlb.p, r, z);
    }
    CK_LAUNCH();
}

template void ilu_apply<double>(const IluFactors &, bool, const double *, double *, cudaStream_t);
template void ilu_apply<float>(const IluFactors &, bool, const float *, float *, cudaStream_t);

}  // namespace bgs
