// Flexible GMRES on the device (Sec. 2.2, flexible GMRES): the Arnoldi orthogonalisation (K14,
// K15), the Givens rotations of the Hessenberg column, the residual estimate and the stopping test.
//
// Orthogonalisation: classical Gram-Schmidt with selective re-orthogonalisation (Daniel-Gragg-
// Kaufman-Stewart test, "twice is enough").
//   dots:   h = V^T w and ||w||^2 in one pass over V (column-major, leading dimension ld);
//           the basis is split over gridDim.y in chunks of KC vectors so a thread keeps KC + 1
//           accumulators, and each thread reads two rows per load (16-byte loads along a column).
//   update: w_out = w_in - V h and ||w_out||^2 in one pass (one accumulator per row pair).
// Every reduction goes through per-block partials summed in a fixed order, so the results do not
// depend on scheduling.
//
// The step kernels read the basis size (cnt = j + 1) from the solver state in device memory, and
// the scalar work of a step (Hessenberg column, rotations, estimate, stop decision) runs in one
// single-thread kernel, so a whole restart cycle can be replayed as one CUDA graph whose WHILE
// node the step kernel ends; launched one by one, the same kernels give the same bits.
#include "internal.h"

namespace bgs {

constexpr int KT = 256;   // threads per block
constexpr int KC = 16;    // basis vectors per dot chunk
// blocks along x: the dots run one wave at the 3 blocks per multiprocessor that k_mdot's
// registers allow (so no multiprocessor runs a lone fourth block); the update 4 per multiprocessor
static int kg_dots() { return num_sms() * 3; }
static int kg_update() { return num_sms() * 4; }

// basis size of a launch: the fixed value, or the solver state's (device) count
__device__ __forceinline__ int basis_count(int cnt, const int *cntp) { return cntp ? *cntp : cnt; }

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

// part layout: [chunk][block][KC + 1]; slot KC holds ||w||^2 (chunk 0 only).  A launch whose gate
// reads 0 does nothing (the second Gram-Schmidt pass when the test does not ask for it).
__global__ void __launch_bounds__(KT, 3) k_mdot(const double *__restrict__ V, int64_t ld, int cnt0, const int *cntp,
                                             const int *gate, const double *__restrict__ w, int64_t n, double *part) {
    if (gate && !*gate) return;
    const int cnt = basis_count(cnt0, cntp);
    const int k0 = blockIdx.y * KC;
    if (k0 >= cnt) return;                 // chunk past the basis (launched for the largest count)
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
// fixed shuffle tree); out[cnt] = ||w||^2
__global__ void k_mdot_reduce(const double *part, int g, int cnt0, const int *cntp, const int *gate, double *out) {
    if (gate && !*gate) return;
    const int cnt = basis_count(cnt0, cntp);
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
__global__ void __launch_bounds__(KT) k_mupdate(const double *__restrict__ V, int64_t ld, int cnt0, const int *cntp,
                                                const int *gate, const double *__restrict__ h, const double *w_in,
                                                double *w_out, int64_t n, double *part) {
    if (gate && !*gate) return;
    const int cnt = basis_count(cnt0, cntp);
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

__global__ void k_sum_partials(const double *part, int g, const int *gate, double *out) {
    if (gate && !*gate) return;
    double s = 0.0;
    for (int b = threadIdx.x; b < g; b += 32) s += part[b];
    s = warp_sum(s);
    if (threadIdx.x == 0) *out = s;
}

size_t arnoldi_dots_scratch(int cnt, int64_t n, int max_blocks) {
    const int nchunk = (cnt + KC - 1) / KC;
    const int g = grid_for(n / 2 + 1, KT, max_blocks > 0 ? max_blocks : kg_dots());
    return (size_t)nchunk * g * (KC + 1);
}

static void dots_launch(const double *V, int64_t ld, int cnt, const int *cntp, int cnt_max, const int *gate,
                        const double *w, int64_t n, double *h, double *partial, size_t partial_cap, int max_blocks,
                        cudaStream_t s) {
    const int nchunk = (cnt_max + KC - 1) / KC;
    const int g = grid_for(n / 2 + 1, KT, max_blocks > 0 ? max_blocks : kg_dots());
    if ((size_t)nchunk * g * (KC + 1) > partial_cap) throw Error(BGS_INTERNAL, "partial scratch too small");
    k_mdot<<<dim3(g, nchunk), KT, 0, s>>>(V, ld, cnt, cntp, gate, w, n, partial);
    CK_LAUNCH();
    k_mdot_reduce<<<(cnt_max + 1 + 7) / 8, 256, 0, s>>>(partial, g, cnt, cntp, gate, h);
    CK_LAUNCH();
}

void arnoldi_dots_into(const double *V, int64_t ld, int cnt, const double *w, int64_t n, double *h, double *partial,
                       size_t partial_cap, int max_blocks, cudaStream_t s) {
    if (cnt < 1 || cnt > 64) throw Error(BGS_INVALID_ARG, "basis size outside 1..64");
    if (ld & 1) throw Error(BGS_INVALID_ARG, "basis leading dimension must be even");
    dots_launch(V, ld, cnt, nullptr, cnt, nullptr, w, n, h, partial, partial_cap, max_blocks, s);
}

// ------------------------------------------------------------------------------------------
// FGMRES step kernels
// ------------------------------------------------------------------------------------------
// Start of a restart cycle: v_0 = r / beta into V_0 (and the graph's staging vector when given).
__global__ void k_fg_first(const double *r, double inv_beta, double *v0, double *stage, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = r[i] * inv_beta;
        v0[i] = v;
        if (stage) stage[i] = v;
    }
}

__global__ void k_fg_begin(FgState *st, double beta) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    st->j = 0;
    st->cnt = 1;
    st->stop = 0;
    st->flag = 0;
    st->jend = 0;
    for (int k = 0; k <= kMaxRestart; k++) st->g[k] = 0.0;
    st->g[0] = beta;
}

// z_j (the graph's staging output) into column j of Z
__global__ void k_fg_store_z(const FgState *st, const double *src, double *Z, int64_t ld, int64_t n) {
    double *dst = Z + (int64_t)st->j * ld;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// the re-orthogonalisation test: a second pass when ||w1|| < eta ||w|| (always for eta >= 1)
__global__ void k_fg_check(FgState *st, int always) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int need = always || st->nw1 < st->eta2 * st->h1[st->cnt];
    st->need2 = need;
    st->reorth += need;
}

// Column j of the Hessenberg matrix from the dots, the earlier rotations applied to it, the new
// rotation, the residual estimate |g_{j+1}| / ||b||, and the stop decision; then the next column.
__global__ void k_fg_step(FgState *st, cudaGraphConditionalHandle loop, int use_loop) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int j = st->j, m = st->m;
    double *H = st->H;
    for (int i = 0; i <= j; i++) {
        double v = st->h1[i];
        if (st->need2) v += st->h2[i];
        H[i * kHld + j] = v;
    }
    const double nw = st->need2 ? st->nw2 : st->nw1;
    const double hn = sqrt(nw);
    H[(j + 1) * kHld + j] = hn;
    st->it++;
    const int breakdown = hn == 0.0;
    st->inv_hn = breakdown ? 0.0 : 1.0 / hn;
    for (int i = 0; i < j; i++) {
        const double a = H[i * kHld + j], c = H[(i + 1) * kHld + j];
        H[i * kHld + j] = st->cs[i] * a + st->sn[i] * c;
        H[(i + 1) * kHld + j] = -st->sn[i] * a + st->cs[i] * c;
    }
    const double a = H[j * kHld + j], c = H[(j + 1) * kHld + j];
    const double den = sqrt(a * a + c * c);
    st->cs[j] = den == 0.0 ? 1.0 : a / den;
    st->sn[j] = den == 0.0 ? 0.0 : c / den;
    H[j * kHld + j] = den;
    H[(j + 1) * kHld + j] = 0.0;
    st->g[j + 1] = -st->sn[j] * st->g[j];
    st->g[j] = st->cs[j] * st->g[j];
    const double est = fabs(st->g[j + 1]) / st->bnorm;
    st->est = est;
    st->jend = j + 1;
    int flag = 0;
    if (!isfinite(est)) flag = 4;
    else if (est <= st->rtol) flag = 1;
    else if (st->it >= st->maxit) flag = 2;
    else if (breakdown) flag = 3;
    else if (j + 1 >= m) flag = 5;
    st->flag = flag;
    st->stop = flag != 0;
    if (!flag) {
        st->j = j + 1;
        st->cnt = j + 2;
    }
    if (use_loop) cudaGraphSetConditional(loop, flag ? 0u : 1u);
}

// v_{j+1} = w / h_{j+1,j} into the next column (and the staging vector), unless the cycle stopped
__global__ void k_fg_next(const FgState *st, const double *w, double *V, int64_t ld, double *stage, int64_t n) {
    if (st->stop) return;
    const double s = st->inv_hn;
    double *dst = V + (int64_t)st->j * ld;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = w[i] * s;
        dst[i] = v;
        if (stage) stage[i] = v;
    }
}

// y from the triangular system H(0:jend, 0:jend) y = g(0:jend) (back substitution)
__global__ void k_fg_backsolve(FgState *st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int je = st->jend;
    for (int i = je - 1; i >= 0; i--) {
        double t = st->g[i];
        for (int k = i + 1; k < je; k++) t -= st->H[i * kHld + k] * st->y[k];
        st->y[i] = t / st->H[i * kHld + i];
    }
}

// x += sum_k y_k Z_k, k < jend (y on the device)
__global__ void k_fg_update_x(const FgState *st, const double *__restrict__ Z, int64_t ld, double *__restrict__ x,
                              int64_t n) {
    __shared__ double ys[kMaxRestart + 1];
    const int je = st->jend;
    for (int k = threadIdx.x; k < je; k += blockDim.x) ys[k] = st->y[k];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double xi = x[i];
        for (int k = 0; k < je; k++) xi += ys[k] * Z[k * ld + i];
        x[i] = xi;
    }
}

__global__ void k_fg_init(FgState *st, int m, int maxit, double rtol, double eta2, double bnorm) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    st->m = m;
    st->maxit = maxit;
    st->rtol = rtol;
    st->eta2 = eta2;
    st->bnorm = bnorm;
    st->it = 0;
    st->reorth = 0;
    st->est = 1.0;
}

void fg_init(FgState *st, int m, int maxit, double rtol, double eta2, double bnorm, cudaStream_t s) {
    k_fg_init<<<1, 32, 0, s>>>(st, m, maxit, rtol, eta2, bnorm);
    CK_LAUNCH();
}

void fg_begin(FgState *st, const double *r, double beta, double *V, double *stage, int64_t n, cudaStream_t s) {
    k_fg_begin<<<1, 32, 0, s>>>(st, beta);
    CK_LAUNCH();
    k_fg_first<<<grid_for(n, 256, num_sms() * 8), 256, 0, s>>>(r, 1.0 / beta, V, stage, n);
    CK_LAUNCH();
}

void fg_store_z(const FgState *st, const double *src, double *Z, int64_t ld, int64_t n, cudaStream_t s) {
    k_fg_store_z<<<grid_for(n, 256, num_sms() * 8), 256, 0, s>>>(st, src, Z, ld, n);
    CK_LAUNCH();
}

void fg_orthogonalise(FgState *st, const double *V, int64_t ld, int m, double *w, int64_t n, bool always,
                      Scratch &sc, cudaStream_t s) {
    const int cnt_max = m;   // the step of column j orthogonalises against j + 1 <= m vectors
    const int gu = grid_for(n / 2 + 1, KT, kg_update());
    // first pass: h1 = V^T w, ||w||^2; w1 = w - V h1, ||w1||^2
    dots_launch(V, ld, 0, &st->cnt, cnt_max, nullptr, w, n, st->h1, sc.partial.p, sc.partial.n, 0, s);
    k_mupdate<<<gu, KT, 0, s>>>(V, ld, 0, &st->cnt, nullptr, st->h1, w, w, n, sc.partial.p);
    CK_LAUNCH();
    k_sum_partials<<<1, 32, 0, s>>>(sc.partial.p, gu, nullptr, &st->nw1);
    CK_LAUNCH();
    k_fg_check<<<1, 32, 0, s>>>(st, always ? 1 : 0);
    CK_LAUNCH();
    // second pass when the test asks for it (the kernels read the decision on the device)
    dots_launch(V, ld, 0, &st->cnt, cnt_max, &st->need2, w, n, st->h2, sc.partial.p, sc.partial.n, 0, s);
    k_mupdate<<<gu, KT, 0, s>>>(V, ld, 0, &st->cnt, &st->need2, st->h2, w, w, n, sc.partial.p);
    CK_LAUNCH();
    k_sum_partials<<<1, 32, 0, s>>>(sc.partial.p, gu, &st->need2, &st->nw2);
    CK_LAUNCH();
}

void fg_step(FgState *st, cudaGraphConditionalHandle loop, bool use_loop, const double *w, double *V, int64_t ld,
             double *stage, int64_t n, cudaStream_t s) {
    k_fg_step<<<1, 32, 0, s>>>(st, loop, use_loop ? 1 : 0);
    CK_LAUNCH();
    k_fg_next<<<grid_for(n, 256, num_sms() * 8), 256, 0, s>>>(st, w, V, ld, stage, n);
    CK_LAUNCH();
}

void fg_finish_cycle(FgState *st, const double *Z, int64_t ld, double *x, int64_t n, cudaStream_t s) {
    k_fg_backsolve<<<1, 32, 0, s>>>(st);
    CK_LAUNCH();
    k_fg_update_x<<<grid_for(n, 256, num_sms() * 8), 256, 0, s>>>(st, Z, ld, x, n);
    CK_LAUNCH();
}

}  // namespace bgs
