// Device code of the SpMV kernels: value conversions, the fused epilogues, and the per-row bodies
// of the CSR SpMV, the first Chebyshev step and the dense coarsest-level product.
#pragma once
#include "internal.h"

namespace bgs {

template <class AT>
struct Cvt;
template <>
struct Cvt<double> {
    template <class T>
    __device__ __forceinline__ static double f(T x) { return to_d(x); }
};
template <>
struct Cvt<float> {
    template <class T>
    __device__ __forceinline__ static float f(T x) { return to_f(x); }
};

// acc + a x (or acc - a x) as one fused multiply-add.  Every epilogue names the value the row sum
// starts from (b for a residual, y for an update in place, 0 for a plain product) and whether the
// products are subtracted, so r = b - A x costs one FMA per stored entry and nothing after it.
template <bool SUB>
__device__ __forceinline__ double mac(double acc, double a, double x) { return SUB ? fma(-a, x, acc) : fma(a, x, acc); }
template <bool SUB>
__device__ __forceinline__ float mac(float acc, float a, float x) { return SUB ? fmaf(-a, x, acc) : fmaf(a, x, acc); }

// ------------------------------------------------------------------------------------------ epilogues
// start(i): the value the row sum of row i starts from; kSub: the products are subtracted from it;
// operator()(i, s): consumes the finished sum.
template <class XT>
struct EStore {   // y = A x
    XT *y;
    static constexpr bool kSub = false;
    template <class AT>
    __device__ AT start(int) const { return (AT)0; }
    template <class AT>
    __device__ void operator()(int i, AT s) const { y[i] = (XT)s; }
};
template <class XT>
struct EResid {   // r = b - A x
    const XT *b;
    XT *r;
    static constexpr bool kSub = true;
    template <class AT>
    __device__ AT start(int i) const { return (AT)b[i]; }
    template <class AT>
    __device__ void operator()(int i, AT s) const { r[i] = (XT)s; }
};
template <class XT>
struct EAdd {   // y = y + A x
    XT *y;
    static constexpr bool kSub = false;
    template <class AT>
    __device__ AT start(int i) const { return (AT)y[i]; }
    template <class AT>
    __device__ void operator()(int i, AT s) const { y[i] = (XT)s; }
};
template <class XT>
struct ESub {   // r = v - A z with FP64 v
    const double *v;
    XT *r;
    static constexpr bool kSub = true;
    template <class AT>
    __device__ AT start(int i) const { return (AT)v[i]; }
    template <class AT>
    __device__ void operator()(int i, AT s) const { r[i] = (XT)s; }
};
struct EScale {   // w = D^-1 A v
    const double *dinv;
    double *w;
    static constexpr bool kSub = false;
    template <class AT>
    __device__ AT start(int) const { return (AT)0; }
    __device__ void operator()(int i, double s) const { w[i] = dinv[i] * s; }
};
struct EScaleNorm {   // w = dinv (A v) / ||v||, 1/||v|| read from device memory (w = dinv (A v) without it)
    const double *dinv;
    const double *rnorm;
    double *w;
    static constexpr bool kSub = false;
    template <class AT>
    __device__ AT start(int) const { return (AT)0; }
    __device__ void operator()(int i, double s) const { w[i] = rnorm ? dinv[i] * (s * *rnorm) : dinv[i] * s; }
};
// One Chebyshev step in scaled form.  The recurrence d' = c1 d + c2 D^-1 r, x' = x + d' is carried
// as e = d / c2 (the step's own c2): e' = alpha e + D^-1 r with alpha = c1 c2_prev / c2, and
// x' = x + c2 e'.  After the row sum r = b - A x that is one multiply and two FMAs per row.
template <class XT, class CT>
struct ECheb {
    const XT *b, *dinv, *xin;
    XT *xout, *e;
    CT alpha, scale;
    int first;   // e is not read (alpha = 0)
    static constexpr bool kSub = true;
    template <class AT>
    __device__ AT start(int i) const { return (AT)b[i]; }
    template <class AT>
    __device__ void operator()(int i, AT r) const {
        CT t = (CT)dinv[i] * (CT)r;
        if (!first) t = mac<false>(t, alpha, (CT)e[i]);
        e[i] = (XT)t;
        xout[i] = (XT)mac<false>((CT)xin[i], scale, t);
    }
};

// The first Chebyshev step from x = 0 of the level whose right-hand side b a product writes (the
// restriction onto a level, or the coupling subtraction onto a block's finest level), fused into
// that product's epilogue: after the base epilogue stores b_i, e_i = D^-1_i b_i and
// x_i = e_i / theta, from the stored (rounded) b_i as the separate first-step kernel computes them.
template <class Base, class XT, class CT>
struct EThenFirst {
    Base base;
    const XT *dinv;
    XT *x, *e;
    CT inv_theta;
    static constexpr bool kSub = Base::kSub;
    template <class AT>
    __device__ AT start(int i) const { return base.template start<AT>(i); }
    template <class AT>
    __device__ void operator()(int i, AT s) const {
        base(i, s);
        const CT t = (CT)dinv[i] * (CT)(XT)s;
        e[i] = (XT)t;
        x[i] = (XT)(inv_theta * t);
    }
};

template <class XT>
struct AccOf { using T = double; };
template <>
struct AccOf<float> { using T = float; };

// y = A x with L threads per row over the whole grid: rows in warp-uniform strips of 32/L rows, the
// L lanes stride over the row and reduce by shuffles.
template <int L, class VT, class XT, class AT, class Epi>
__device__ __forceinline__ void spmv_rows(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                          const VT *__restrict__ val, const XT *__restrict__ x, Epi epi) {
    constexpr int RPW = 32 / L;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (L - 1);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * RPW; base < n; base += nwarps * RPW) {
        const int row = (int)(base + lane / L);
        AT acc = (AT)0;
        if (row < n) {
            if (sub == 0) acc = epi.template start<AT>(row);
            const int s = __ldg(rp + row), e = __ldg(rp + row + 1);
            if constexpr (L == 1 && sizeof(AT) == 4 && sizeof(VT) == 4) {
                // FP32 values and sums, one thread per row: batches of eight entries with the index clamped to
                // the row's last entry and the value of a slot past the end taken as 0 (an exact
                // no-op in the sum), so all loads of a batch are in flight together; the selects
                // run on the integer / FP32 pipes (faster on a 7-point fine level; the FP64 form
                // gains nothing, its FP64 pipe being the other limit, nor do BF16 values)
                for (int k = s; k < e; k += 8) {
                    int c[8];
                    AT a[8];
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int kk = min(k + u, e - 1);
                        c[u] = __ldg(ci + kk);
                        a[u] = k + u < e ? Cvt<AT>::f(ldg(val + kk)) : (AT)0;
                    }
#pragma unroll
                    for (int u = 0; u < 8; u++) acc = mac<Epi::kSub>(acc, a[u], Cvt<AT>::f(ldg(x + c[u])));
                }
            } else {
                for (int k = s + sub; k < e; k += L)
                    acc = mac<Epi::kSub>(acc, Cvt<AT>::f(ldg(val + k)), Cvt<AT>::f(ldg(x + __ldg(ci + k))));
            }
        }
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (sub == 0 && row < n) epi(row, acc);
    }
}

// The first Chebyshev step from x = 0 in the scaled form of ECheb: e = D^-1 b, x = e / theta.
template <class XT>
__device__ __forceinline__ void cheb_first_rows(int n, const XT *__restrict__ b, const XT *__restrict__ dinv,
                                                double inv_theta, XT *__restrict__ x, XT *__restrict__ e) {
    using CT = typename AccOf<XT>::T;
    const CT it = (CT)inv_theta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const CT t = (CT)dinv[i] * (CT)b[i];
        e[i] = (XT)t;
        x[i] = (XT)(it * t);
    }
}

// Dense GEMV with a row-major matrix: one warp per row, y_i = sum_j W_ij x_j (FP64 accumulation).
template <class XT>
__device__ __forceinline__ void dense_gemv_rows(int n, const double *__restrict__ W, const XT *__restrict__ x,
                                                XT *__restrict__ y) {
    const int lane = threadIdx.x & 31;
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += (gridDim.x * blockDim.x) >> 5) {
        const double *w = W + (size_t)row * n;
        double acc = 0.0;
        for (int j = lane; j < n; j += 32) acc += w[j] * (double)x[j];
        acc = warp_sum(acc);
        if (lane == 0) y[row] = (XT)acc;
    }
}

// accumulation type: FP64 for FP64 vectors, FP32 for FP32 vectors and for BF16 coupling values
template <class VT, class XT>
struct AccT { using T = typename AccOf<XT>::T; };
template <>
struct AccT<__nv_bfloat16, double> { using T = float; };

}  // namespace bgs
