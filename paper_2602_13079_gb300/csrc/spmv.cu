// SpMV with fused epilogues (K1, K2, K10, K11, K13).
//
// Three storage paths share every epilogue:
//  * SELL-32 (the fine-level operators, the full operator, prolongators): one thread per row,
//    a warp owns a slice of 32 rows stored column-major, so entry j of the 32 rows is one
//    contiguous 256-byte (FP64) / 128-byte (index) run; no row-pointer round trip; the epilogue
//    (residual, Chebyshev step, prolongation add, coupling subtraction) is fully coalesced.
//  * SELL-32 with diagonal offsets (structured operators): the same slices, but slot k of a slice
//    stores one offset o for its 32 rows (column = row + o) instead of 32 column indices, so the
//    index stream (a third of the FP64 CSR bytes, half of the FP32 ones) shrinks 32-fold; rows
//    missing an offset hold 0 there.  The entries of a row are still summed in column order.
//  * CSR with L threads per row (coarse levels with long, irregular rows): rows are taken in
//    warp-uniform strips of 32/L rows, the L lanes stride over the row and reduce by shuffles.
// Every path is instantiated for 128, 256 and 512 threads per block (rows per block = threads / L
// for CSR, = threads for the SELL forms); the autotuner picks the format and the block size.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include <climits>
#include <type_traits>

#include "spmv_dev.cuh"

namespace bgs {

// ------------------------------------------------------------------------------------------ CSR
template <int L, class VT, class XT, class AT, class Epi, int TPB>
__global__ void __launch_bounds__(TPB) k_spmv(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                              const VT *__restrict__ val, const XT *__restrict__ x, Epi epi) {
    spmv_rows<L, VT, XT, AT>(n, rp, ci, val, x, epi);
}

// ------------------------------------------------------------------------------------------ SELL-32
template <class VT, class XT, class AT, class Epi, int TPB>
__global__ void __launch_bounds__(TPB) k_sell(int n, const int *__restrict__ sptr, const int *__restrict__ sci,
                                              const VT *__restrict__ sv, const XT *__restrict__ x, Epi epi) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int slice = row >> 5;
    if ((slice << 5) >= n) return;          // whole warp past the end
    const int lane = row & 31;
    const int s0 = __ldg(sptr + slice);
    const int w = (__ldg(sptr + slice + 1) - s0) >> 5;
    const int *c = sci + s0 + lane;
    const VT *v = sv + s0 + lane;
    constexpr bool S = Epi::kSub;
    AT acc = row < n ? epi.template start<AT>(row) : (AT)0;
    if constexpr (sizeof(AT) == 4 && sizeof(VT) == 4) {
        // FP32 values and sums: batches of eight slots, the slot index clamped to the slice width
        // and a slot past it taken as 0 (as in the one-thread-per-row CSR form)
#pragma unroll 1
        for (int j = 0; j < w; j += 8) {
            int cc[8];
            AT a[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int jj = min(j + u, w - 1) - j;
                cc[u] = __ldg(c + jj * 32);
                a[u] = j + u < w ? Cvt<AT>::f(ldg(v + jj * 32)) : (AT)0;
            }
#pragma unroll
            for (int u = 0; u < 8; u++) acc = mac<S>(acc, a[u], Cvt<AT>::f(ldg(x + cc[u])));
            c += 8 * 32;
            v += 8 * 32;
        }
        if (row < n) epi(row, acc);
        return;
    }
    // FP64: batches of 8 slots (all index and value loads, then all gathers, in flight together:
    // the long rows of the coarse levels wait on fewer dependent rounds), then of 4, then single
    int j = 0;
#pragma unroll 1
    for (; j + 8 <= w; j += 8) {
        int cc[8];
        AT a[8], xv[8];
#pragma unroll
        for (int u = 0; u < 8; u++) { cc[u] = __ldg(c + u * 32); a[u] = Cvt<AT>::f(ldg(v + u * 32)); }
#pragma unroll
        for (int u = 0; u < 8; u++) xv[u] = Cvt<AT>::f(ldg(x + cc[u]));
#pragma unroll
        for (int u = 0; u < 8; u++) acc = mac<S>(acc, a[u], xv[u]);
        c += 8 * 32;
        v += 8 * 32;
    }
#pragma unroll 1
    for (; j + 4 <= w; j += 4) {
        const int c0 = __ldg(c + 0 * 32), c1 = __ldg(c + 1 * 32), c2 = __ldg(c + 2 * 32), c3 = __ldg(c + 3 * 32);
        const AT a0 = Cvt<AT>::f(ldg(v + 0 * 32)), a1 = Cvt<AT>::f(ldg(v + 1 * 32));
        const AT a2 = Cvt<AT>::f(ldg(v + 2 * 32)), a3 = Cvt<AT>::f(ldg(v + 3 * 32));
        acc = mac<S>(acc, a0, Cvt<AT>::f(ldg(x + c0)));
        acc = mac<S>(acc, a1, Cvt<AT>::f(ldg(x + c1)));
        acc = mac<S>(acc, a2, Cvt<AT>::f(ldg(x + c2)));
        acc = mac<S>(acc, a3, Cvt<AT>::f(ldg(x + c3)));
        c += 4 * 32;
        v += 4 * 32;
    }
    for (; j < w; j++) {
        acc = mac<S>(acc, Cvt<AT>::f(ldg(v)), Cvt<AT>::f(ldg(x + __ldg(c))));
        c += 32;
        v += 32;
    }
    if (row < n) epi(row, acc);
}

// ------------------------------------------------------------------------------------------ SELL-32, diagonal offsets
// The row sum of one row over its slice's w slots (offsets in myo across the warp's lanes), added
// to acc.  CLAMP: the column row + offset is clamped into [0, last] (a padded slot may point
// outside; its value is 0); a slice whose rows all stay inside for every offset skips it.
template <bool CLAMP, class VT, class XT, class AT, bool S>
__device__ __forceinline__ AT dia_row_sum(AT acc, int row, int w, int myo, int last, const VT *__restrict__ v,
                                          const XT *__restrict__ x) {
    auto col = [&](int o) { return CLAMP ? min(max(row + o, 0), last) : row + o; };
    if constexpr (sizeof(AT) == 4 && sizeof(VT) == 4) {
        // FP32: batches of 4 slots, all loads of a batch in flight together; a slot past the slice
        // width re-reads the last one (a cached duplicate) and its product is skipped (w is
        // warp-uniform).  Batches of 8 took 40 registers (48 warps per SM) against 32 (64 warps)
        // and timed 3% slower in the solve.
        constexpr int U = 4;
#pragma unroll 1
        for (int k = 0; k < w; k += U) {
            AT a[U], xv[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int kk = min(k + u, w - 1);
                const int c = col(__shfl_sync(0xffffffffu, myo, kk));
                a[u] = Cvt<AT>::f(ldg(v + kk * 32));
                xv[u] = Cvt<AT>::f(ldg(x + c));
            }
#pragma unroll
            for (int u = 0; u < U; u++)
                if (k + u < w) acc = mac<S>(acc, a[u], xv[u]);
        }
    } else {
        // FP64: full batches of 4 slots, then the rest one by one (no duplicate loads; this timed
        // faster than predicated batches for the FP64 operators)
        constexpr int U = 4;
        int k = 0;
#pragma unroll 1
        for (; k + U <= w; k += U) {
            AT a[U], xv[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int c = col(__shfl_sync(0xffffffffu, myo, k + u));
                a[u] = Cvt<AT>::f(ldg(v + (k + u) * 32));
                xv[u] = Cvt<AT>::f(ldg(x + c));
            }
#pragma unroll
            for (int u = 0; u < U; u++) acc = mac<S>(acc, a[u], xv[u]);
        }
#pragma unroll 1
        for (; k < w; k++) {
            const int c = col(__shfl_sync(0xffffffffu, myo, k));
            acc = mac<S>(acc, Cvt<AT>::f(ldg(v + k * 32)), Cvt<AT>::f(ldg(x + c)));
        }
    }
    return acc;
}

// Slice of 32 rows per warp; lane k holds the slice's k-th offset (w <= wmax <= 32), broadcast by
// shuffle.  The offsets sit at a fixed stride of wmax per slice, so their load does not wait for the
// slice's slot pointer: a warp's loads take two dependent rounds (pointers, offsets and the start
// value; then values and x), not three.
template <class VT, class XT, class AT, class Epi, int TPB>
__global__ void __launch_bounds__(TPB) k_dia(int n, int m, int wmax, const int *__restrict__ dptr,
                                             const int *__restrict__ doff, const VT *__restrict__ dv,
                                             const XT *__restrict__ x, Epi epi) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int slice = row >> 5;
    if ((slice << 5) >= n) return;          // whole warp past the end
    const int lane = row & 31;
    const int s0 = __ldg(dptr + slice);
    const int w = (__ldg(dptr + slice + 1) - s0) >> 5;
    const int myo = lane < wmax ? __ldg(doff + (int64_t)slice * wmax + lane) : 0;
    const VT *v = dv + s0 + lane;
    const int last = m - 1;
    AT acc = row < n ? epi.template start<AT>(row) : (AT)0;
    // every row of the slice, shifted by every offset it stores (and 0), inside [0, m): no clamping
    const int omin = __reduce_min_sync(0xffffffffu, myo), omax = __reduce_max_sync(0xffffffffu, myo);
    const int64_t first = (int64_t)slice << 5;
    if (first + omin >= 0 && first + 31 + omax <= (int64_t)last)
        acc = dia_row_sum<false, VT, XT, AT, Epi::kSub>(acc, row, w, myo, last, v, x);
    else
        acc = dia_row_sum<true, VT, XT, AT, Epi::kSub>(acc, row, w, myo, last, v, x);
    if (row < n) epi(row, acc);
}

// ------------------------------------------------------------------------------------------ field-interleaved node blocks
// The full operator of F fields on nc nodes as F x F node blocks (the block-sparse form the
// coupled unknowns of one node suggest): one thread per node computes the F rows f * nc + I, each
// block slot one block column J with its F x F values (stored lane-innermost, so every value load of
// a warp is one contiguous run) and F gathers x[g * nc + J].  A row's products are summed block by
// block (ascending J), within a block by field g.
template <int F, class Epi, int TPB>
__global__ void __launch_bounds__(TPB) k_bsr(int nc, const int *__restrict__ bptr, const int *__restrict__ bcol,
                                             const double *__restrict__ bval, const double *__restrict__ x, Epi epi) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int slice = I >> 5;
    if ((slice << 5) >= nc) return;
    const int lane = I & 31;
    const int s0 = __ldg(bptr + slice);
    const int w = (__ldg(bptr + slice + 1) - s0) >> 5;
    constexpr bool S = Epi::kSub;
    double acc[F];
#pragma unroll
    for (int f = 0; f < F; f++) acc[f] = I < nc ? epi.template start<double>(f * nc + I) : 0.0;
    const double *vb = bval + (size_t)s0 * F * F + lane;
#pragma unroll 1
    for (int k = 0; k < w; k++) {
        const int J = __ldg(bcol + s0 + k * 32 + lane);
        double xg[F];
#pragma unroll
        for (int g = 0; g < F; g++) xg[g] = __ldg(x + (size_t)g * nc + J);
#pragma unroll
        for (int f = 0; f < F; f++)
#pragma unroll
            for (int g = 0; g < F; g++)
                acc[f] = mac<S>(acc[f], __ldg(vb + ((size_t)k * F * F + f * F + g) * 32), xg[g]);
    }
    if (I < nc)
#pragma unroll
        for (int f = 0; f < F; f++) epi(f * nc + I, acc[f]);
}

// value arrays of a matrix by element type (CSR order / SELL order / diagonal-offset order)
template <class VT>
struct Vals;
template <>
struct Vals<double> {
    static const double *csr(const DCsr &A) { return A.v.p; }
    static const double *sell(const DCsr &A) { return A.sv.p; }
    static const double *dia(const DCsr &A) { return A.dv.p; }
};
template <>
struct Vals<float> {
    static const float *csr(const DCsr &A) { return A.vf.p; }
    static const float *sell(const DCsr &A) { return A.svf.p; }
    static const float *dia(const DCsr &A) { return A.dvf.p; }
};
template <>
struct Vals<__nv_bfloat16> {
    static const __nv_bfloat16 *csr(const DCsr &A) { return A.vb.p; }
    static const __nv_bfloat16 *sell(const DCsr &A) { return A.svb.p; }
    static const __nv_bfloat16 *dia(const DCsr &A) { return A.dvb.p; }
};

template <class VT, class XT, class AT, class Epi, int TPB>
static void launch_csr_tpb(int lanes, int n, const int *rp, const int *ci, const VT *val, const XT *x, Epi epi,
                           cudaStream_t s) {
    const int rows_per_block = TPB / lanes;
    const int g = grid_for(n, rows_per_block, num_sms() * (8192 / TPB));
    switch (lanes) {
        case 1: k_spmv<1, VT, XT, AT, Epi, TPB><<<g, TPB, 0, s>>>(n, rp, ci, val, x, epi); break;
        case 2: k_spmv<2, VT, XT, AT, Epi, TPB><<<g, TPB, 0, s>>>(n, rp, ci, val, x, epi); break;
        case 4: k_spmv<4, VT, XT, AT, Epi, TPB><<<g, TPB, 0, s>>>(n, rp, ci, val, x, epi); break;
        case 8: k_spmv<8, VT, XT, AT, Epi, TPB><<<g, TPB, 0, s>>>(n, rp, ci, val, x, epi); break;
        case 16: k_spmv<16, VT, XT, AT, Epi, TPB><<<g, TPB, 0, s>>>(n, rp, ci, val, x, epi); break;
        default: k_spmv<32, VT, XT, AT, Epi, TPB><<<g, TPB, 0, s>>>(n, rp, ci, val, x, epi); break;
    }
    CK_LAUNCH();
}

template <class VT, class XT, class AT, class Epi>
static void launch_csr(int lanes, int n, const int *rp, const int *ci, const VT *val, const XT *x, Epi epi,
                       cudaStream_t s, int tpb = 256) {
    if (n <= 0) return;
    if (tpb == 128) launch_csr_tpb<VT, XT, AT, Epi, 128>(lanes, n, rp, ci, val, x, epi, s);
    else if (tpb == 512) launch_csr_tpb<VT, XT, AT, Epi, 512>(lanes, n, rp, ci, val, x, epi, s);
    else launch_csr_tpb<VT, XT, AT, Epi, 256>(lanes, n, rp, ci, val, x, epi, s);
}

int choose_lanes(int64_t nrows, int64_t nnz) {
    double avg = nrows > 0 ? (double)nnz / (double)nrows : 0.0;
    if (avg <= 2.0) return 2;
    if (avg <= 6.0) return 4;
    if (avg <= 14.0) return 8;
    if (avg <= 40.0) return 16;
    return 32;
}

static int lanes_of(const DCsr &A) { return A.lanes ? A.lanes : choose_lanes(A.n, A.nnz); }

// dispatch: SELL when built, CSR otherwise

template <class VT, class XT, class AT, class Epi, int TPB>
static void launch_sliced(const DCsr &A, const XT *x, Epi epi, cudaStream_t s) {
    const int g = (int)(((int64_t)A.n + TPB - 1) / TPB);
    if (A.dia)
        k_dia<VT, XT, AT, Epi, TPB><<<g, TPB, 0, s>>>(A.n, A.m, A.dia_wmax, A.dptr.p, A.doff.p, Vals<VT>::dia(A), x, epi);
    else k_sell<VT, XT, AT, Epi, TPB><<<g, TPB, 0, s>>>(A.n, A.sptr.p, A.sci.p, Vals<VT>::sell(A), x, epi);
    CK_LAUNCH();
}

template <int F, class Epi, int TPB>
static void launch_bsr_f(const DCsr &A, const double *x, Epi epi, cudaStream_t s) {
    const int g = (int)(((int64_t)A.bsr_nc + TPB - 1) / TPB);
    k_bsr<F, Epi, TPB><<<g, TPB, 0, s>>>(A.bsr_nc, A.bptr.p, A.bcol.p, A.bval.p, x, epi);
    CK_LAUNCH();
}

template <class Epi, int TPB>
static void launch_bsr_tpb(const DCsr &A, const double *x, Epi epi, cudaStream_t s) {
    switch (A.bsr_F) {
        case 2: launch_bsr_f<2, Epi, TPB>(A, x, epi, s); break;
        case 3: launch_bsr_f<3, Epi, TPB>(A, x, epi, s); break;
        case 4: launch_bsr_f<4, Epi, TPB>(A, x, epi, s); break;
        case 5: launch_bsr_f<5, Epi, TPB>(A, x, epi, s); break;
        case 6: launch_bsr_f<6, Epi, TPB>(A, x, epi, s); break;
        default: throw Error(BGS_INTERNAL, "node blocks built for an unsupported field count");
    }
}

// the node-block form serves the full operator's plain product and residual only
template <class VT, class XT, class Epi>
constexpr bool kBsrEpi = std::is_same<VT, double>::value && std::is_same<XT, double>::value &&
                         (std::is_same<Epi, EStore<double>>::value || std::is_same<Epi, EResid<double>>::value);

template <class VT, class XT, class Epi>
static void run(const DCsr &A, const XT *x, Epi epi, cudaStream_t s) {
    using AT = typename AccT<VT, XT>::T;
    if (A.n <= 0) return;
    if (A.bsr_active()) {
        if constexpr (kBsrEpi<VT, XT, Epi>) {
            if (A.tpb == 128) launch_bsr_tpb<Epi, 128>(A, x, epi, s);
            else if (A.tpb == 512) launch_bsr_tpb<Epi, 512>(A, x, epi, s);
            else launch_bsr_tpb<Epi, 256>(A, x, epi, s);
            return;
        } else {
            throw Error(BGS_INTERNAL, "node-block layout applied with an unsupported epilogue");
        }
    }
    if (A.dia || A.sell) {
        if (A.tpb == 128) launch_sliced<VT, XT, AT, Epi, 128>(A, x, epi, s);
        else if (A.tpb == 512) launch_sliced<VT, XT, AT, Epi, 512>(A, x, epi, s);
        else launch_sliced<VT, XT, AT, Epi, 256>(A, x, epi, s);
    } else {
        launch_csr<VT, XT, AT>(lanes_of(A), A.n, A.rp.p, A.ci.p, Vals<VT>::csr(A), x, epi, s, A.tpb);
    }
}

void spmv_f64(const CsrView &A, int lanes, const double *x, double *y, cudaStream_t s) {
    if (lanes <= 0) lanes = choose_lanes(A.n, A.nnz);
    launch_csr<double, double, double>(lanes, A.n, A.rp, A.ci, A.v, x, EStore<double>{y}, s);
}

void spmv_scaled(const CsrView &A, const double *dinv, const double *v, double *w, cudaStream_t s) {
    launch_csr<double, double, double>(choose_lanes(A.n, A.nnz), A.n, A.rp, A.ci, A.v, v, EScale{dinv, w}, s);
}

void spmv_scaled_norm(const DCsr &A, const double *dinv, const double *v, const double *rnorm, double *w,
                      cudaStream_t s) {
    // a summation order fixed by the shape alone (not by the autotuned format), so that a set-up
    // and a later numeric re-set-up sum alike: short rows left to right, one thread per row (from
    // the diagonal-offset layout when the operator has one: its slots run in column order and its
    // padded slots add exact zeros), longer rows over L lanes
    const double avg = A.n > 0 ? (double)A.nnz / (double)A.n : 0.0;
    const int lanes = avg <= 12.0 ? 1 : (avg <= 64.0 ? 4 : 8);
    if (lanes == 1 && A.dia && A.n > 0) {
        launch_sliced<double, double, double, EScaleNorm, 256>(A, v, EScaleNorm{dinv, rnorm, w}, s);
        return;
    }
    launch_csr<double, double, double>(lanes, A.n, A.rp.p, A.ci.p, A.v.p, v, EScaleNorm{dinv, rnorm, w}, s);
}

template <class VT, class XT>
void spmv_store(const DCsr &A, const XT *x, XT *y, cudaStream_t s) {
    run<VT, XT>(A, x, EStore<XT>{y}, s);
}
template <class VT, class XT>
void spmv_resid(const DCsr &A, const XT *b, const XT *x, XT *r, cudaStream_t s) {
    run<VT, XT>(A, x, EResid<XT>{b, r}, s);
}
template <class VT, class XT>
void spmv_addto(const DCsr &A, const XT *x, XT *y, cudaStream_t s) {
    run<VT, XT>(A, x, EAdd<XT>{y}, s);
}
template <class VT, class XT>
void cheb_step(const DCsr &A, const XT *b, const XT *dinv, const XT *xin, XT *xout, XT *e, double alpha,
               double scale, bool first, cudaStream_t s) {
    using CT = typename AccOf<XT>::T;
    run<VT, XT>(A, xin, ECheb<XT, CT>{b, dinv, xin, xout, e, (CT)alpha, (CT)scale, first ? 1 : 0}, s);
}
template <class VT, class XT, class ZT>
void coupling_sub(const DCsr &L, const double *v, const ZT *z, XT *r, cudaStream_t s) {
    run<VT, ZT>(L, z, ESub<XT>{v, r}, s);
}
template <class VT, class XT>
void spmv_store_first(const DCsr &A, const XT *x, XT *y, const FirstStep<XT> &f, cudaStream_t s) {
    using CT = typename AccOf<XT>::T;
    run<VT, XT>(A, x, EThenFirst<EStore<XT>, XT, CT>{EStore<XT>{y}, f.dinv, f.x, f.e, (CT)f.inv_theta}, s);
}
template <class VT, class XT, class ZT>
void coupling_sub_first(const DCsr &L, const double *v, const ZT *z, XT *r, const FirstStep<XT> &f,
                        cudaStream_t s) {
    using CT = typename AccOf<XT>::T;
    run<VT, ZT>(L, z, EThenFirst<ESub<XT>, XT, CT>{ESub<XT>{v, r}, f.dinv, f.x, f.e, (CT)f.inv_theta}, s);
}
// b = v (converted to XT) and the first Chebyshev step from it, for a block without couplings
template <class XT>
__global__ void k_copy_first(int64_t n, const double *__restrict__ v, XT *__restrict__ b, const XT *__restrict__ dinv,
                             double inv_theta, XT *__restrict__ x, XT *__restrict__ e) {
    using CT = typename AccOf<XT>::T;
    const CT it = (CT)inv_theta;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const XT bi = (XT)v[i];
        b[i] = bi;
        const CT t = (CT)dinv[i] * (CT)bi;
        e[i] = (XT)t;
        x[i] = (XT)(it * t);
    }
}
template <class XT>
void copy_in_first(const double *v, XT *b, int64_t n, const FirstStep<XT> &f, cudaStream_t s) {
    if (n <= 0) return;
    k_copy_first<XT><<<grid_for(n, 256, num_sms() * 32), 256, 0, s>>>(n, v, b, f.dinv, f.inv_theta, f.x, f.e);
    CK_LAUNCH();
}

template <class XT>
__global__ void k_cheb_first(int n, const XT *__restrict__ b, const XT *__restrict__ dinv, double inv_theta,
                             XT *__restrict__ x, XT *__restrict__ e) {
    cheb_first_rows<XT>(n, b, dinv, inv_theta, x, e);
}
template <class XT>
void cheb_first(int n, const XT *b, const XT *dinv, double inv_theta, XT *x, XT *e, cudaStream_t s) {
    if (n <= 0) return;
    k_cheb_first<XT><<<grid_for(n, 256, num_sms() * 32), 256, 0, s>>>(n, b, dinv, inv_theta, x, e);
    CK_LAUNCH();
}

template <class XT>
__global__ void k_dense_gemv(int n, const double *__restrict__ W, const XT *__restrict__ x, XT *__restrict__ y) {
    dense_gemv_rows<XT>(n, W, x, y);
}
template <class XT>
void dense_gemv(int n, const double *W, const XT *x, XT *y, cudaStream_t s) {
    if (n <= 0) return;
    k_dense_gemv<XT><<<grid_for((int64_t)n * 32, 256, num_sms() * 16), 256, 0, s>>>(n, W, x, y);
    CK_LAUNCH();
}

// ------------------------------------------------------------------------------------------ SELL build
__global__ void k_sell_width(int n, const int *rp, int *wslot) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int slice = row >> 5;
    if ((slice << 5) >= n) return;
    const int len = row < n ? rp[row + 1] - rp[row] : 0;
    const int w = __reduce_max_sync(0xffffffffu, len);
    if ((row & 31) == 0) wslot[slice] = w * 32;
}

// Padded slots get value 0 and the first stored column of their slice: a column the slice reads
// anyway, so the padding never touches an entry of x outside the columns the matrix references
// (x may hold unwritten entries there, e.g. the sweep output while later fields are still to be
// computed, and 0 times such an entry need not be 0).
__global__ void k_sell_fill(int n, const int *rp, const int *ci, const int *sptr, int *sci, int *sperm) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int slice = row >> 5;
    if ((slice << 5) >= n) return;
    const int lane = row & 31;
    const int s0 = sptr[slice];
    const int w = (sptr[slice + 1] - s0) >> 5;
    const int b = row < n ? rp[row] : 0, len = row < n ? rp[row + 1] - b : 0;
    // the slice's first stored column (w > 0 means some row of the slice stores an entry)
    const unsigned has = __ballot_sync(0xffffffffu, len > 0);
    const int src = has ? __ffs(has) - 1 : 0;
    const int pad = __shfl_sync(0xffffffffu, len > 0 ? ci[b] : 0, src);
    for (int j = 0; j < w; j++) {
        const int slot = s0 + j * 32 + lane;
        if (j < len) {
            sci[slot] = ci[b + j];
            sperm[slot] = b + j;
        } else {
            sci[slot] = pad;
            sperm[slot] = -1;
        }
    }
}

template <class T>
__global__ void k_gather_vals(int64_t m, const int *perm, const T *src, T *dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int p = perm[i];
        dst[i] = p >= 0 ? src[p] : (T)0.0f;
    }
}

template <class T>
static void gather_into(const DCsr &A, const T *src, DBuf<T> &dst, cudaStream_t s) {
    if (dst.n != (size_t)A.sell_nnz || !dst.p) dst.alloc((size_t)A.sell_nnz, s);
    k_gather_vals<T><<<grid_for(A.sell_nnz, 256), 256, 0, s>>>(A.sell_nnz, A.sperm.p, src, dst.p);
    CK_LAUNCH();
}

bool build_sell(DCsr &A, double max_pad, Scratch &sc, cudaStream_t s) {
    if (A.sell) return true;
    if (A.n <= 0 || A.nnz <= 0) return false;
    const int nsl = (A.n + 31) / 32;
    DBuf<int> sptr((size_t)nsl + 1, s);
    k_sell_width<<<(unsigned)(((int64_t)nsl * 32 + 255) / 256), 256, 0, s>>>(A.n, A.rp.p, sptr.p);
    CK_LAUNCH();
    const int64_t tot = scan_exclusive(sptr.p, sptr.p, nsl, sc, s);
    if ((double)tot > max_pad * (double)A.nnz) return false;
    A.sptr = std::move(sptr);
    A.sell_nnz = tot;
    A.sci.alloc((size_t)tot, s);
    A.sperm.alloc((size_t)tot, s);
    k_sell_fill<<<(unsigned)(((int64_t)nsl * 32 + 255) / 256), 256, 0, s>>>(A.n, A.rp.p, A.ci.p, A.sptr.p, A.sci.p,
                                                                           A.sperm.p);
    CK_LAUNCH();
    gather_into(A, A.v.p, A.sv, s);
    A.sell = true;
    sell_refresh(A, s);
    return true;
}

// ------------------------------------------------------------------------------------------ diagonal-offset SELL build
// One warp per slice of 32 rows: the union of the rows' diagonal offsets (column - row), found by
// merging the 32 sorted lists (each step takes the warp minimum of the lanes' next offsets).  The
// width pass writes 32 * (union size), or -1 when a slice has more than 32 distinct offsets; the
// fill pass writes the offsets and, per slot, the CSR index of the row's entry there (-1: none).
__global__ void k_dia_width(int n, const int *rp, const int *ci, int *wslot) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int slice = row >> 5;
    if ((slice << 5) >= n) return;
    int p = row < n ? rp[row] : 0;
    const int e = row < n ? rp[row + 1] : 0;
    int w = 0;
    for (;;) {
        const int cand = p < e ? ci[p] - row : INT_MAX;
        const int mn = __reduce_min_sync(0xffffffffu, cand);
        if (mn == INT_MAX) break;
        if (cand == mn) p++;
        if (++w > 32) break;
    }
    if ((row & 31) == 0) wslot[slice] = w > 32 ? -1 : w * 32;
}
__global__ void k_dia_fill(int n, int wmax, const int *rp, const int *ci, const int *dptr, int *doff, int *dperm) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int slice = row >> 5;
    if ((slice << 5) >= n) return;
    const int lane = row & 31;
    const int s0 = dptr[slice];
    int p = row < n ? rp[row] : 0;
    const int e = row < n ? rp[row + 1] : 0;
    int k = 0;
    for (;; k++) {
        const int cand = p < e ? ci[p] - row : INT_MAX;
        const int mn = __reduce_min_sync(0xffffffffu, cand);
        if (mn == INT_MAX) break;
        if (lane == 0) doff[(int64_t)slice * wmax + k] = mn;
        dperm[s0 + k * 32 + lane] = cand == mn ? p : -1;
        if (cand == mn) p++;
    }
    if (lane == 0)
        for (; k < wmax; k++) doff[(int64_t)slice * wmax + k] = 0;   // past the slice's width: unused
}
// min and max of a[0..n) into out[0], out[1] (out preset to INT_MAX, INT_MIN)
__global__ void k_minmax_int(int n, const int *a, int *out) {
    int lo = INT_MAX, hi = INT_MIN;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        lo = min(lo, a[i]);
        hi = max(hi, a[i]);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(out, lo);
        atomicMax(out + 1, hi);
    }
}

template <class T>
static void gather_dia(const DCsr &A, const T *src, DBuf<T> &dst, cudaStream_t s) {
    if (dst.n != (size_t)A.dia_nnz || !dst.p) dst.alloc((size_t)A.dia_nnz, s);
    k_gather_vals<T><<<grid_for(A.dia_nnz, 256), 256, 0, s>>>(A.dia_nnz, A.dperm.p, src, dst.p);
    CK_LAUNCH();
}

bool build_dia(DCsr &A, double max_pad, Scratch &sc, cudaStream_t s) {
    if (A.dia) return true;
    if (A.n <= 0 || A.nnz <= 0 || A.m <= 0 || A.m > INT_MAX - 64) return false;
    const int nsl = (A.n + 31) / 32;
    const unsigned g = (unsigned)(((int64_t)nsl * 32 + 255) / 256);
    DBuf<int> dptr((size_t)nsl + 1, s);
    k_dia_width<<<g, 256, 0, s>>>(A.n, A.rp.p, A.ci.p, dptr.p);
    CK_LAUNCH();
    dev_fill_int(sc.flags.p + 16, INT_MAX, 1, s);
    dev_fill_int(sc.flags.p + 17, INT_MIN, 1, s);
    k_minmax_int<<<grid_for(nsl, 256), 256, 0, s>>>(nsl, dptr.p, sc.flags.p + 16);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(sc.h_flags + 16, sc.flags.p + 16, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (sc.h_flags[16] < 0) return false;                 // a slice with more than 32 offsets
    const int wmax = std::max(sc.h_flags[17] / 32, 1);
    const int64_t tot = scan_exclusive(dptr.p, dptr.p, nsl, sc, s);
    if ((double)tot > max_pad * (double)A.nnz) return false;
    A.dptr = std::move(dptr);
    A.dia_nnz = tot;
    A.dia_wmax = wmax;
    A.doff.alloc((size_t)nsl * wmax, s);
    A.dperm.alloc((size_t)tot, s);
    k_dia_fill<<<g, 256, 0, s>>>(A.n, wmax, A.rp.p, A.ci.p, A.dptr.p, A.doff.p, A.dperm.p);
    CK_LAUNCH();
    gather_dia(A, A.v.p, A.dv, s);
    A.dia = true;
    sell_refresh(A, s);
    return true;
}

// ------------------------------------------------------------------------------------------ node-block build
constexpr int kBsrMaxBlocks = 32;   // distinct block columns per node

// the distinct block columns of node I over its F rows, ascending, into lc; the count, or -1 past
// kBsrMaxBlocks
__device__ int bsr_node_cols(int I, int F, int nc, const int *rp, const int *ci, int *lc) {
    int c = 0;
    for (int f = 0; f < F; f++) {
        const int r = f * nc + I;
        for (int e = rp[r]; e < rp[r + 1]; e++) {
            const int J = ci[e] % nc;
            int p = c - 1;
            while (p >= 0 && lc[p] > J) p--;
            if (p >= 0 && lc[p] == J) continue;
            if (c == kBsrMaxBlocks) return -1;
            for (int q = c; q > p + 1; q--) lc[q] = lc[q - 1];
            lc[p + 1] = J;
            c++;
        }
    }
    return c;
}

__global__ void k_bsr_width(int nc, int F, const int *rp, const int *ci, int *wslot, int *fail) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int slice = I >> 5;
    if ((slice << 5) >= nc) return;
    int lc[kBsrMaxBlocks];
    int c = I < nc ? bsr_node_cols(I, F, nc, rp, ci, lc) : 0;
    if (c < 0) {
        atomicOr(fail, 1);
        c = 0;
    }
    const int w = __reduce_max_sync(0xffffffffu, c);
    if ((I & 31) == 0) wslot[slice] = w * 32;
}

// block columns (a padded slot repeats the node's first block column, values 0) and values
__global__ void k_bsr_fill(int nc, int F, const int *rp, const int *ci, const double *v, const int *bptr, int *bcol,
                           double *bval) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int slice = I >> 5;
    if ((slice << 5) >= nc) return;
    const int lane = I & 31;
    const int s0 = bptr[slice], w = (bptr[slice + 1] - s0) >> 5;
    int lc[kBsrMaxBlocks];
    const int c = I < nc ? bsr_node_cols(I, F, nc, rp, ci, lc) : 0;
    const int pad = c > 0 ? lc[0] : 0;
    const size_t FF = (size_t)F * F;
    for (int k = 0; k < w; k++) {
        bcol[s0 + k * 32 + lane] = k < c ? lc[k] : pad;
        for (size_t fg = 0; fg < FF; fg++) bval[((size_t)s0 + (size_t)k * 32) * FF + fg * 32 + lane] = 0.0;
    }
    if (I >= nc) return;
    for (int f = 0; f < F; f++) {
        const int r = f * nc + I;
        for (int e = rp[r]; e < rp[r + 1]; e++) {
            const int g = ci[e] / nc, J = ci[e] - g * nc;
            int lo = 0, hi = c - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (lc[mid] < J) lo = mid + 1;
                else hi = mid;
            }
            bval[((size_t)s0 + (size_t)lo * 32) * FF + (size_t)(f * F + g) * 32 + lane] = v[e];
        }
    }
}

static void bsr_fill(DCsr &A, cudaStream_t s) {
    const int nsl = (A.bsr_nc + 31) / 32;
    k_bsr_fill<<<(unsigned)(((int64_t)nsl * 32 + 255) / 256), 256, 0, s>>>(A.bsr_nc, A.bsr_F, A.rp.p, A.ci.p, A.v.p,
                                                                         A.bptr.p, A.bcol.p, A.bval.p);
    CK_LAUNCH();
}

bool build_bsr(DCsr &A, int F, double max_pad, Scratch &sc, cudaStream_t s) {
    if (A.bsr) return true;
    if (F < 2 || F > 6 || A.n <= 0 || A.nnz <= 0 || A.n % F || A.m != A.n) return false;
    const int nc = A.n / F;
    const int nsl = (nc + 31) / 32;
    DBuf<int> bptr((size_t)nsl + 1, s);
    CK(cudaMemsetAsync(sc.flags.p + 15, 0, sizeof(int), s));
    k_bsr_width<<<(unsigned)(((int64_t)nsl * 32 + 255) / 256), 256, 0, s>>>(nc, F, A.rp.p, A.ci.p, bptr.p,
                                                                           sc.flags.p + 15);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(sc.h_flags + 15, sc.flags.p + 15, sizeof(int), cudaMemcpyDeviceToHost, s));
    const int64_t tot = scan_exclusive(bptr.p, bptr.p, nsl, sc, s);   // synchronises
    if (sc.h_flags[15]) return false;                                // a node with too many block columns
    if ((double)tot * F * F > max_pad * (double)A.nnz) return false;
    A.bptr = std::move(bptr);
    A.bsr_slots = tot;
    A.bsr_F = F;
    A.bsr_nc = nc;
    A.bcol.alloc((size_t)tot, s);
    A.bval.alloc((size_t)tot * F * F, s);
    bsr_fill(A, s);
    A.bsr = true;
    return true;
}

void drop_bsr(DCsr &A) {
    A.bsr = false;
    A.bsr_slots = 0;
    A.bptr.release(); A.bcol.release(); A.bval.release();
}

void drop_dia(DCsr &A) {
    A.dia = false;
    A.dia_nnz = 0;
    A.dia_wmax = 0;
    A.dptr.release(); A.doff.release(); A.dperm.release(); A.dv.release(); A.dvf.release(); A.dvb.release();
}

void sell_refresh(DCsr &A, cudaStream_t s) {
    if (A.sell) {
        if (A.vf.p) gather_into(A, A.vf.p, A.svf, s);
        if (A.vb.p) gather_into(A, A.vb.p, A.svb, s);
    }
    if (A.dia) {
        if (A.vf.p) gather_dia(A, A.vf.p, A.dvf, s);
        if (A.vb.p) gather_dia(A, A.vb.p, A.dvb, s);
    }
}

void refresh_values(DCsr &A, cudaStream_t s) {
    if (A.nnz <= 0) return;
    if (A.vf.p) convert_d2f(A.v.p, A.vf.p, A.nnz, s);
    if (A.vb.p) convert_d2bf(A.v.p, A.vb.p, A.nnz, s);
    if (A.sell) gather_into(A, A.v.p, A.sv, s);
    if (A.dia) gather_dia(A, A.v.p, A.dv, s);
    if (A.bsr) bsr_fill(A, s);
    sell_refresh(A, s);
}

// ------------------------------------------------------------------------------------------ autotuner
// Picks the SpMV kernel of one stored operator by timing it with every candidate: the diagonal-
// offset SELL-32 and SELL-32 (when built) and CSR with 1, 2, 4, 8, 16, 32 threads per row, each at
// 128, 256 and 512 threads per block.  The timed launch is the fused Chebyshev step (the epilogue
// most launches of a level operator run: b, D^-1, x and e read, e and x' written, five distinct
// vectors) or, for an operator applied only as a plain product (the full operator), y = A x; one
// warm-up and
// the fastest of five timed launches each, CUDA events on the stream.  The choice is cached for the
// process, keyed by (rows, columns, stored entries, value bytes, epilogue), so repeated set-ups of operators
// with the same shape reuse it without timing, and build only the layout the choice needs.
// a choice: format (-2 node blocks, -1 diagonal-offset SELL, 0 SELL-32, k > 0 CSR with k threads per
// row) and block size
struct Choice {
    int format = 0, tpb = 256;
    int code() const {
        const int f = format == -2 ? 8 : (format < 0 ? 0 : (format == 0 ? 1 : 2 + __builtin_ctz((unsigned)format)));
        return f * 4 + (tpb == 128 ? 0 : (tpb == 512 ? 2 : 1));
    }
    static Choice from(int c) {
        Choice ch;
        const int f = c / 4, t = c % 4;
        ch.format = f == 8 ? -2 : (f == 0 ? -1 : (f == 1 ? 0 : 1 << (f - 2)));
        ch.tpb = t == 0 ? 128 : (t == 2 ? 512 : 256);
        return ch;
    }
};

using TuneKey = std::tuple<int, int, int64_t, int, int>;   // rows, columns, entries, value bytes, epilogue
static std::mutex g_tune_mu;
static std::map<TuneKey, int> g_tune;   // -> Choice::code()
static bool g_tune_loaded = false;

// BGS_AUTOTUNE_CACHE=<file>: choices are read from and appended to this text file, so another
// process (or a profiled run) reuses them instead of timing again.
static void tune_cache_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("BGS_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    int n, m, vb, ep, c;
    long long nnz;
    while (fscanf(f, "%d %d %lld %d %d %d", &n, &m, &nnz, &vb, &ep, &c) == 6)
        g_tune[std::make_tuple(n, m, (int64_t)nnz, vb, ep)] = c;
    fclose(f);
}

static void tune_cache_append(const TuneKey &k, int c) {
    const char *path = getenv("BGS_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%d %d %lld %d %d %d\n", std::get<0>(k), std::get<1>(k), (long long)std::get<2>(k), std::get<3>(k),
            std::get<4>(k), c);
    fclose(f);
}

template <class VT, class XT>
static Choice time_candidates(DCsr &A, bool product, cudaStream_t s) {
    using CT = typename AccOf<XT>::T;
    // distinct vectors for b, D^-1, x, x' and e, as in a smoothing step (one shared vector would be
    // read from L2 and favour the layouts with the fewest matrix bytes over what a step sees)
    const size_t nx = (size_t)std::max(A.m, A.n) + 1;
    DBuf<XT> x(nx, s), y(nx, s), e(nx, s), bv(nx, s), dv(nx, s);
    XT *const bufs[5] = {x.p, y.p, e.p, bv.p, dv.p};
    for (XT *p : bufs) CK(cudaMemsetAsync(p, 0, sizeof(XT) * nx, s));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    Choice choice;
    const bool had_sell = A.sell, had_dia = A.dia, had_bsr = A.bsr;
    const bool log = getenv("BGS_AUTOTUNE_LOG") != nullptr;   // every candidate's time to stderr
    const int formats[9] = {-2, -1, 0, 1, 2, 4, 8, 16, 32};
    for (int f : formats) {
        if ((f == -2 && !(had_bsr && product && kBsrEpi<VT, XT, EStore<XT>>)) || (f == -1 && !had_dia) ||
            (f == 0 && !had_sell))
            continue;
        for (int tpb : {128, 256, 512}) {
            A.bsr = f == -2;
            A.dia = f == -1;
            A.sell = f == 0;
            A.lanes = f > 0 ? f : 0;
            A.tpb = tpb;
            float fastest = 1e30f;
            for (int rep = 0; rep < 6; rep++) {
                CK(cudaEventRecord(e0, s));
                if (product) run<VT, XT>(A, x.p, EStore<XT>{y.p}, s);
                else run<VT, XT>(A, x.p, ECheb<XT, CT>{bv.p, dv.p, x.p, y.p, e.p, (CT)0.5, (CT)0.5, 0}, s);
                CK(cudaEventRecord(e1, s));
                CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                if (rep) fastest = std::min(fastest, ms);
            }
            if (log) fprintf(stderr, "bgs-autotune n %d m %d nnz %lld vbytes %d product %d format %d tpb %d ms %.5f\n",
                             A.n, A.m, (long long)A.nnz, (int)sizeof(VT), product ? 1 : 0, f, tpb, fastest);
            if (fastest < best) {
                best = fastest;
                choice.format = f;
                choice.tpb = tpb;
            }
        }
    }
    A.sell = had_sell;
    A.dia = had_dia;
    A.bsr = had_bsr;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return choice;
}

static void apply_choice(DCsr &A, Choice c) {
    A.tpb = c.tpb;
    A.lanes = c.format > 0 ? c.format : 0;
    if (c.format != -2 && A.bsr) drop_bsr(A);
    if (c.format != -1 && A.dia) drop_dia(A);
    if (c.format != 0 && A.sell) {
        A.sell = false;
        A.sptr.release(); A.sci.release(); A.sperm.release(); A.sv.release(); A.svf.release(); A.svb.release();
    }
}

static int cached_code(const TuneKey &key) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_cache_load();
    auto it = g_tune.find(key);
    return it != g_tune.end() ? it->second : -1;
}

void build_formats(DCsr &A, int value_bytes, bool allow_dia, bool use_cache, Scratch &sc, cudaStream_t s,
                   bool product, int bsr_fields) {
    if (A.n <= 0 || A.nnz <= 0) return;
    const int code = use_cache ? cached_code(std::make_tuple(A.n, A.m, A.nnz, value_bytes, product ? 1 : 0)) : -1;
    if (code >= 0) {
        const Choice c = Choice::from(code);
        if (c.format != -1 && A.dia) drop_dia(A);   // built earlier for the set-up's own products
        A.tpb = c.tpb;
        A.lanes = c.format > 0 ? c.format : 0;
        if (c.format == -2 && bsr_fields && build_bsr(A, bsr_fields, kMaxPadBsrForced, sc, s)) return;
        if (c.format == -1 && allow_dia && build_dia(A, kMaxPadDia, sc, s)) return;
        if (c.format <= 0) build_sell(A, kMaxPad, sc, s);
        return;
    }
    build_sell(A, kMaxPad, sc, s);
    if (allow_dia) build_dia(A, kMaxPadDia, sc, s);
    if (bsr_fields) build_bsr(A, bsr_fields, kMaxPadBsr, sc, s);
}

int autotune_spmv(DCsr &A, int value_bytes, Scratch &sc, cudaStream_t s, bool product) {
    if (A.n <= 0 || A.nnz <= 0) return 0;
    const TuneKey key = std::make_tuple(A.n, A.m, A.nnz, value_bytes, product ? 1 : 0);
    const int code = cached_code(key);
    Choice c;
    if (code >= 0) {
        c = Choice::from(code);
        // the layout the choice names was not built for this operator: the fastest one that was
        if ((c.format == -2 && !A.bsr) || (c.format == -1 && !A.dia) || (c.format == 0 && !A.sell))
            c = Choice{A.dia ? -1 : (A.sell ? 0 : 1), 256};
    } else {
        // time the kernels in the precision the solve will use
        if (value_bytes == 2 && A.vb.p) c = time_candidates<__nv_bfloat16, double>(A, product, s);
        else if (value_bytes == 4 && A.vf.p) c = time_candidates<float, float>(A, product, s);
        else c = time_candidates<double, double>(A, product, s);
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[key] = c.code();
        tune_cache_append(key, c.code());
    }
    apply_choice(A, c);
    return c.format;
}

// explicit instantiations
#define BGS_INST(VT, XT)                                                                                    \
    template void spmv_store<VT, XT>(const DCsr &, const XT *, XT *, cudaStream_t);                       \
    template void spmv_store_first<VT, XT>(const DCsr &, const XT *, XT *, const FirstStep<XT> &,         \
                                           cudaStream_t);                                                 \
    template void copy_in_first<XT>(const double *, XT *, int64_t, const FirstStep<XT> &, cudaStream_t);  \
    template void spmv_resid<VT, XT>(const DCsr &, const XT *, const XT *, XT *, cudaStream_t);           \
    template void spmv_addto<VT, XT>(const DCsr &, const XT *, XT *, cudaStream_t);                       \
    template void cheb_step<VT, XT>(const DCsr &, const XT *, const XT *, const XT *, XT *, XT *, double, \
                                    double, bool, cudaStream_t);
BGS_INST(double, double)
BGS_INST(float, float)
#undef BGS_INST
template void coupling_sub<double, double, double>(const DCsr &, const double *, const double *, double *,
                                                   cudaStream_t);
template void coupling_sub<__nv_bfloat16, float, double>(const DCsr &, const double *, const double *, float *,
                                                         cudaStream_t);
template void coupling_sub<__nv_bfloat16, float, float>(const DCsr &, const double *, const float *, float *,
                                                        cudaStream_t);
template void coupling_sub_first<double, double, double>(const DCsr &, const double *, const double *, double *,
                                                         const FirstStep<double> &, cudaStream_t);
template void coupling_sub_first<__nv_bfloat16, float, double>(const DCsr &, const double *, const double *,
                                                               float *, const FirstStep<float> &, cudaStream_t);
template void coupling_sub_first<__nv_bfloat16, float, float>(const DCsr &, const double *, const float *, float *,
                                                              const FirstStep<float> &, cudaStream_t);
template void cheb_first<double>(int, const double *, const double *, double, double *, double *, cudaStream_t);
template void cheb_first<float>(int, const float *, const float *, double, float *, float *, cudaStream_t);
template void dense_gemv<double>(int, const double *, const double *, double *, cudaStream_t);
template void dense_gemv<float>(int, const double *, const float *, float *, cudaStream_t);

}  // namespace bgs
