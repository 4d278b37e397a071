// Arnoldi orthogonalisation kernels of FGMRES (K14, K15): classical Gram-Schmidt with one
// re-orthogonalisation (CGS2) in three passes over the basis V (column-major, leading dim ld):
//   pass 1: h1 = V^T w
//   pass 2: w -= V h1, then h2 = V^T w on the updated entries (same thread re-reads V from L1)
//   pass 3: w -= V h2, ||w||^2
// Each pass reduces per-block partials, then one block sums them in a fixed order, so the
// results do not depend on scheduling.
#include "internal.h"

namespace bgs {

constexpr int KT = 256;          // threads per block
constexpr int KG = kSMs * 2;     // blocks

template <int K>
__device__ void block_reduce_store(double (&acc)[K + 1], int cnt, double *part) {
    __shared__ double sm[KT / 32][K + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k <= K; k++) {
        if (k < cnt || k == K) {
            double v = warp_sum(acc[k]);
            if (lane == 0) sm[w][k] = v;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k <= K; k += blockDim.x) {
        if (k < cnt || k == K) {
            double t = 0.0;
            for (int q = 0; q < KT / 32; q++) t += sm[q][k];
            part[(size_t)blockIdx.x * (K + 1) + k] = t;
        }
    }
}

template <int K>
__global__ void __launch_bounds__(KT) k_mdot(const double *__restrict__ V, int64_t ld, int cnt,
                                             const double *__restrict__ w, int64_t n, double *part) {
    double acc[K + 1];
#pragma unroll
    for (int k = 0; k <= K; k++) acc[k] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int k = 0; k < K; k++)
            if (k < cnt) acc[k] += V[k * ld + i] * wi;
        acc[K] += wi * wi;
    }
    block_reduce_store<K>(acc, cnt, part);
}

template <int K>
__global__ void __launch_bounds__(KT) k_mupdate_dot(const double *__restrict__ V, int64_t ld, int cnt,
                                                    const double *__restrict__ h, double *__restrict__ w, int64_t n,
                                                    double *part) {
    __shared__ double hs[K];
    for (int k = threadIdx.x; k < K; k += blockDim.x) hs[k] = k < cnt ? h[k] : 0.0;
    __syncthreads();
    double acc[K + 1];
#pragma unroll
    for (int k = 0; k <= K; k++) acc[k] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double wi = w[i];
#pragma unroll
        for (int k = 0; k < K; k++)
            if (k < cnt) wi -= V[k * ld + i] * hs[k];
        w[i] = wi;
#pragma unroll
        for (int k = 0; k < K; k++)
            if (k < cnt) acc[k] += V[k * ld + i] * wi;
        acc[K] += wi * wi;
    }
    block_reduce_store<K>(acc, cnt, part);
}

template <int K>
__global__ void __launch_bounds__(KT) k_mupdate_norm(const double *__restrict__ V, int64_t ld, int cnt,
                                                     const double *__restrict__ h, double *__restrict__ w, int64_t n,
                                                     double *part) {
    __shared__ double hs[K];
    for (int k = threadIdx.x; k < K; k += blockDim.x) hs[k] = k < cnt ? h[k] : 0.0;
    __syncthreads();
    double acc[K + 1];
#pragma unroll
    for (int k = 0; k <= K; k++) acc[k] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double wi = w[i];
#pragma unroll
        for (int k = 0; k < K; k++)
            if (k < cnt) wi -= V[k * ld + i] * hs[k];
        w[i] = wi;
        acc[K] += wi * wi;
    }
    block_reduce_store<K>(acc, 0, part);
}

// out[k] = sum over blocks of part[b][k] for k < cnt; out[cnt] = sum of part[b][K]
template <int K>
__global__ void k_mreduce(const double *part, int g, int cnt, double *out) {
    const int k = threadIdx.x;
    if (k > K) return;
    if (k < cnt || k == K) {
        double t = 0.0;
        for (int b = 0; b < g; b++) t += part[(size_t)b * (K + 1) + k];
        out[k == K ? cnt : k] = t;
    }
}

template <int K>
static void run_mdot(int mode, const double *V, int64_t ld, int cnt, const double *h, double *w, int64_t n,
                     double *out, Scratch &sc, cudaStream_t s) {
    int g = grid_for(n, KT, KG);
    if ((size_t)g * (K + 1) > sc.partial.n) throw Error(BGS_INTERNAL, "partial scratch");
    if (mode == 0) k_mdot<K><<<g, KT, 0, s>>>(V, ld, cnt, w, n, sc.partial.p);
    else if (mode == 1) k_mupdate_dot<K><<<g, KT, 0, s>>>(V, ld, cnt, h, w, n, sc.partial.p);
    else k_mupdate_norm<K><<<g, KT, 0, s>>>(V, ld, cnt, h, w, n, sc.partial.p);
    CK_LAUNCH();
    k_mreduce<K><<<1, K + 1 > 32 ? ((K + 1 + 31) / 32) * 32 : 32, 0, s>>>(sc.partial.p, g, mode == 2 ? 0 : cnt, out);
    CK_LAUNCH();
}

static void dispatch(int mode, const double *V, int64_t ld, int cnt, const double *h, double *w, int64_t n,
                     double *out, Scratch &sc, cudaStream_t s) {
    if (cnt <= 8) run_mdot<8>(mode, V, ld, cnt, h, w, n, out, sc, s);
    else if (cnt <= 16) run_mdot<16>(mode, V, ld, cnt, h, w, n, out, sc, s);
    else if (cnt <= 32) run_mdot<32>(mode, V, ld, cnt, h, w, n, out, sc, s);
    else if (cnt <= 64) run_mdot<64>(mode, V, ld, cnt, h, w, n, out, sc, s);
    else throw Error(BGS_INVALID_ARG, "restart length above 63");
}

void arnoldi_dots(const double *V, int64_t ld, int cnt, const double *w, int64_t n, double *h, Scratch &sc,
                  cudaStream_t s) {
    dispatch(0, V, ld, cnt, nullptr, const_cast<double *>(w), n, h, sc, s);
}
void arnoldi_update_dots(const double *V, int64_t ld, int cnt, const double *h, double *w, int64_t n, double *h2,
                         Scratch &sc, cudaStream_t s) {
    dispatch(1, V, ld, cnt, h, w, n, h2, sc, s);
}
void arnoldi_update_norm(const double *V, int64_t ld, int cnt, const double *h, double *w, int64_t n,
                         double *nrm2, Scratch &sc, cudaStream_t s) {
    dispatch(2, V, ld, cnt, h, w, n, nrm2, sc, s);
}

struct Coefs {
    double y[64];
};

__global__ void k_multi_axpy(const double *__restrict__ Z, int64_t ld, int cnt, Coefs c, double *__restrict__ x,
                             int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double xi = x[i];
        for (int k = 0; k < cnt; k++) xi += c.y[k] * Z[k * ld + i];
        x[i] = xi;
    }
}

void multi_axpy(const double *Z, int64_t ld, int cnt, const double *y_host, double *x, int64_t n, cudaStream_t s) {
    if (cnt <= 0 || n <= 0) return;
    if (cnt > 64) throw Error(BGS_INVALID_ARG, "restart length above 64");
    Coefs c{};
    for (int k = 0; k < cnt; k++) c.y[k] = y_host[k];
    k_multi_axpy<<<grid_for(n, 256, kSMs * 8), 256, 0, s>>>(Z, ld, cnt, c, x, n);
    CK_LAUNCH();
}

__global__ void k_scale_copy(const double *in, double a, double *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] * a;
}
void scale_copy(const double *in, double alpha, double *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_scale_copy<<<grid_for(n, 256, kSMs * 8), 256, 0, s>>>(in, alpha, out, n);
    CK_LAUNCH();
}

__global__ void k_scale_inv_dev(const double *in, const double *sc, double *out, int64_t n, int sq) {
    const double d = sq ? sqrt(*sc) : *sc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] / d;
}
void scale_by_inv_dev(const double *in, const double *dev_scalar, double *out, int64_t n, bool sqrt_first,
                      cudaStream_t s) {
    if (n <= 0) return;
    k_scale_inv_dev<<<grid_for(n, 256, kSMs * 8), 256, 0, s>>>(in, dev_scalar, out, n, sqrt_first ? 1 : 0);
    CK_LAUNCH();
}

}  // namespace bgs
