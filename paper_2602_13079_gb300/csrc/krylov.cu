// Arnoldi orthogonalisation of FGMRES (K14, K15): classical Gram-Schmidt with selective
// re-orthogonalisation (Daniel-Gragg-Kaufman-Stewart test, "twice is enough").
//   dots:   h = V^T w and ||w||^2 in one pass over V (column-major, leading dimension ld);
//           the basis is split over gridDim.y in chunks of KC vectors so a thread keeps KC + 1
//           accumulators, and each thread reads two rows per load (16-byte loads along a column).
//   update: w_out = w_in - V h and ||w_out||^2 in one pass (one accumulator per row pair).
// Every reduction goes through per-block partials summed by one block in a fixed order, so the
// results do not depend on scheduling.
#include "internal.h"

namespace bgs {

constexpr int KT = 256;          // threads per block
constexpr int KC = 16;           // basis vectors per dot chunk
constexpr int KG = kSMs * 4;     // blocks along x (update)
constexpr int KGD = kSMs * 3;    // blocks along x (dots): one wave at the 3 blocks per SM that
                                 // k_mdot's registers allow, so no SM runs a lone fourth block

// Sums each of the NACC per-thread accumulators over the block; thread k writes sum k to out[k].
template <int NACC>
__device__ void block_reduce_to(const double (&acc)[NACC], int nvalid, double *out) {
    __shared__ double sm[KT / 32][NACC];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NACC; k++) {
        if (k < nvalid) {
            const double v = warp_sum(acc[k]);
            if (lane == 0) sm[w][k] = v;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nvalid; k += blockDim.x) {
        double t = 0.0;
        for (int q = 0; q < KT / 32; q++) t += sm[q][k];
        out[k] = t;
    }
}

// part layout: [chunk][block][KC + 1]; slot KC holds ||w||^2 (chunk 0 only)
__global__ void __launch_bounds__(KT, 3) k_mdot(const double *__restrict__ V, int64_t ld, int cnt,
                                             const double *__restrict__ w, int64_t n, double *part) {
    const int k0 = blockIdx.y * KC;
    const int kc = min(KC, cnt - k0);
    double acc[KC + 1];
#pragma unroll
    for (int k = 0; k <= KC; k++) acc[k] = 0.0;
    const int64_t npair = n >> 1;
    const double2 *w2 = reinterpret_cast<const double2 *>(w);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npair; p += (int64_t)gridDim.x * blockDim.x) {
        const double2 wi = w2[p];
#pragma unroll
        for (int k = 0; k < KC; k++)
            if (k < kc) {
                const double2 v = reinterpret_cast<const double2 *>(V + (int64_t)(k0 + k) * ld)[p];
                acc[k] = fma(v.x, wi.x, acc[k]);   // two FMAs per pair: FP64 issue rate is the limit
                acc[k] = fma(v.y, wi.y, acc[k]);
            }
        acc[KC] = fma(wi.x, wi.x, acc[KC]);
        acc[KC] = fma(wi.y, wi.y, acc[KC]);
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {   // odd tail row
        const int64_t i = n - 1;
        const double wi = w[i];
        for (int k = 0; k < kc; k++) acc[k] += V[(int64_t)(k0 + k) * ld + i] * wi;
        acc[KC] += wi * wi;
    }
    if (blockIdx.y != 0) acc[KC] = 0.0;
    block_reduce_to<KC + 1>(acc, KC + 1, part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * (KC + 1));
}

// one warp per output: out[t] = sum over blocks of the partials (fixed order per lane, then a
// fixed shuffle tree)
__global__ void k_mdot_reduce(const double *part, int g, int nchunk, int cnt, double *out) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (t > cnt) return;
    double s = 0.0;
    if (t < cnt) {
        const int c = t / KC, k = t % KC;
        for (int b = lane; b < g; b += 32) s += part[((size_t)c * g + b) * (KC + 1) + k];
    } else {
        for (int b = lane; b < g; b += 32) s += part[(size_t)b * (KC + 1) + KC];
    }
    s = warp_sum(s);
    if (lane == 0) out[t] = s;
}

// w_out = w_in - V h ; partial ||w_out||^2 per block
__global__ void __launch_bounds__(KT) k_mupdate(const double *__restrict__ V, int64_t ld, int cnt,
                                                const double *__restrict__ h, const double *w_in, double *w_out,
                                                int64_t n, double *part) {
    __shared__ double hs[64];
    for (int k = threadIdx.x; k < 64; k += blockDim.x) hs[k] = k < cnt ? h[k] : 0.0;
    __syncthreads();
    double nrm = 0.0;
    const int64_t npair = n >> 1;
    const double2 *wi2 = reinterpret_cast<const double2 *>(w_in);
    double2 *wo2 = reinterpret_cast<double2 *>(w_out);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npair; p += (int64_t)gridDim.x * blockDim.x) {
        double2 a = wi2[p];
#pragma unroll 8
        for (int k = 0; k < cnt; k++) {
            const double2 v = reinterpret_cast<const double2 *>(V + (int64_t)k * ld)[p];
            a.x -= v.x * hs[k];
            a.y -= v.y * hs[k];
        }
        wo2[p] = a;
        nrm = fma(a.x, a.x, nrm);
        nrm = fma(a.y, a.y, nrm);
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t i = n - 1;
        double a = w_in[i];
        for (int k = 0; k < cnt; k++) a -= V[(int64_t)k * ld + i] * hs[k];
        w_out[i] = a;
        nrm += a * a;
    }
    double acc[1] = {nrm};
    block_reduce_to<1>(acc, 1, part + blockIdx.x);
}

__global__ void k_sum_partials(const double *part, int g, double *out) {
    double s = 0.0;
    for (int b = threadIdx.x; b < g; b += 32) s += part[b];
    s = warp_sum(s);
    if (threadIdx.x == 0) *out = s;
}

size_t arnoldi_dots_scratch(int cnt, int64_t n) {
    const int nchunk = (cnt + KC - 1) / KC;
    const int g = grid_for(n / 2 + 1, KT, KGD);
    return (size_t)nchunk * g * (KC + 1);
}

void arnoldi_dots_into(const double *V, int64_t ld, int cnt, const double *w, int64_t n, double *h, double *partial,
                       size_t partial_cap, cudaStream_t s) {
    if (cnt < 1 || cnt > 64) throw Error(BGS_INVALID_ARG, "basis size outside 1..64");
    if (ld & 1) throw Error(BGS_INVALID_ARG, "basis leading dimension must be even");
    const int nchunk = (cnt + KC - 1) / KC;
    const int g = grid_for(n / 2 + 1, KT, KGD);
    if ((size_t)nchunk * g * (KC + 1) > partial_cap) throw Error(BGS_INTERNAL, "partial scratch too small");
    k_mdot<<<dim3(g, nchunk), KT, 0, s>>>(V, ld, cnt, w, n, partial);
    CK_LAUNCH();
    k_mdot_reduce<<<(cnt + 1 + 7) / 8, 256, 0, s>>>(partial, g, nchunk, cnt, h);
    CK_LAUNCH();
}

void arnoldi_dots(const double *V, int64_t ld, int cnt, const double *w, int64_t n, double *h, Scratch &sc,
                  cudaStream_t s) {
    arnoldi_dots_into(V, ld, cnt, w, n, h, sc.partial.p, sc.partial.n, s);
}

void arnoldi_update(const double *V, int64_t ld, int cnt, const double *h, const double *w_in, double *w_out,
                    int64_t n, double *nrm2, Scratch &sc, cudaStream_t s) {
    if (cnt < 1 || cnt > 64) throw Error(BGS_INVALID_ARG, "basis size outside 1..64");
    if (ld & 1) throw Error(BGS_INTERNAL, "basis leading dimension must be even");
    const int g = grid_for(n / 2 + 1, KT, KG);
    k_mupdate<<<g, KT, 0, s>>>(V, ld, cnt, h, w_in, w_out, n, sc.partial.p);
    CK_LAUNCH();
    k_sum_partials<<<1, 32, 0, s>>>(sc.partial.p, g, nrm2);
    CK_LAUNCH();
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
