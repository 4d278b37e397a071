// Scans, reductions, validation, block assembly and small element-wise kernels.
#include <atomic>
#include <climits>
#include <cstdlib>
#include <mutex>

#include "internal.h"

namespace bgs {

static std::atomic<long long> g_launches{0};
cudaMemPool_t device_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[128] = {};
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        CK(cudaMemPoolCreate(&pools[dev], &props));
        uint64_t keep = UINT64_MAX;
        CK(cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep));
    }
    return pools[dev];
}

void release_cached_memory() {
    if (!plain_alloc()) {
        CK(cudaDeviceSynchronize());
        CK(cudaMemPoolTrimTo(device_pool(), 0));
    }
}

bool plain_alloc() {
    static const bool v = [] {
        const char *e = getenv("BGS_PLAIN_ALLOC");
        return e && e[0] == '1';
    }();
    return v;
}
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int num_sms() {
    static std::atomic<int> cache[128] = {};
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) dev = 0;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    CK(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    if (v < 1) v = 1;
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

void Scratch::init(cudaStream_t s) {
    owner = s;
    partial.alloc(num_sms() * 8 * 72, s);
    scal.alloc(256, s);
    flags.alloc(64, s);
    iscan.alloc(1 << 16, s);
    CK(cudaMallocHost((void **)&h_scal, 256 * sizeof(double)));
    CK(cudaMallocHost((void **)&h_flags, 64 * sizeof(int)));
}

void Scratch::ensure_side() {
    if (side) return;
    int prio = 0;
    if (owner) CK(cudaStreamGetPriority(owner, &prio));
    CK(cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, prio));
    CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
}

Scratch::~Scratch() {
    if (side) {
        cudaStreamSynchronize(side);
        cudaStreamDestroy(side);
        cudaEventDestroy(fork);
    }
    if (h_scal) cudaFreeHost(h_scal);
    if (h_flags) cudaFreeHost(h_flags);
}

// ------------------------------------------------------------------------------------------
// Host transfers: pinned host memory is read or written by the SMs over the host link (one
// kernel for every piece of a call) instead of by the copy engines, whose host transfers on this
// platform ran at a fifth of the link rate on some calls; other memory goes through cudaMemcpyAsync.
// ------------------------------------------------------------------------------------------
constexpr int kXferMax = 96;
struct XferParams {
    int nseg;
    uint64_t start[kXferMax + 1];   // first 16-byte unit of each piece, then the total
    const uint4 *src[kXferMax];
    uint4 *dst[kXferMax];
};

__global__ void k_xfer(XferParams p) {
    const uint64_t total = p.start[p.nseg];
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += (uint64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = p.nseg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.start[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        const uint64_t off = u - p.start[lo];
        p.dst[lo][off] = p.src[lo][off];
    }
}

// device-usable address of pinned host memory, or nullptr for device / pageable memory
static void *pinned_device_address(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

void transfer(const std::vector<XferSeg> &segs, cudaStream_t s) {
    XferParams prm{};
    auto flush = [&]() {
        if (prm.nseg == 0) return;
        const uint64_t total = prm.start[prm.nseg];
        k_xfer<<<grid_for((int64_t)total, 256, num_sms() * 8), 256, 0, s>>>(prm);
        CK_LAUNCH();
        prm.nseg = 0;
    };
    for (const XferSeg &g : segs) {
        if (g.bytes == 0) continue;
        const void *hs = pinned_device_address(g.src);
        void *hd = pinned_device_address(g.dst);
        const void *src = hs ? hs : g.src;
        void *dst = hd ? hd : g.dst;
        const bool aligned = (((uintptr_t)src | (uintptr_t)dst | (uintptr_t)g.bytes) & 15) == 0;
        if ((hs || hd) && aligned) {
            if (prm.nseg == kXferMax) flush();
            prm.src[prm.nseg] = (const uint4 *)src;
            prm.dst[prm.nseg] = (uint4 *)dst;
            prm.start[prm.nseg + 1] = prm.start[prm.nseg] + g.bytes / 16;
            prm.nseg++;
        } else {
            CK(cudaMemcpyAsync(g.dst, g.src, g.bytes, cudaMemcpyDefault, s));
        }
    }
    flush();
}

// ------------------------------------------------------------------------------------------
// Exclusive scan (int32 counts -> int32 offsets, int64 block totals)
// ------------------------------------------------------------------------------------------
constexpr int SCAN_T = 1024, SCAN_I = 4, SCAN_B = SCAN_T * SCAN_I;

__device__ long long block_excl_scan(long long v, long long *sm_warp, long long *total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        long long t = (lane < (int)(blockDim.x >> 5)) ? sm_warp[lane] : 0;
        long long u = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o) u += y;
        }
        if (lane < (int)(blockDim.x >> 5)) sm_warp[lane] = u - t;
        if (lane == 31) *total = u;
    }
    __syncthreads();
    long long r = sm_warp[w] + x - v;
    __syncthreads();
    return r;
}

__global__ void k_scan_sums(const int *__restrict__ in, int64_t n, long long *bsums) {
    __shared__ long long sw[32];
    __shared__ long long tot;
    int64_t base = (int64_t)blockIdx.x * SCAN_B + threadIdx.x * SCAN_I;
    long long v = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; k++)
        if (base + k < n) v += in[base + k];
    block_excl_scan(v, sw, &tot);
    if (threadIdx.x == 0) bsums[blockIdx.x] = tot;
}

__global__ void k_scan_ll_single(long long *a, int n) {
    // exclusive scan of n long longs in one block, chunk by chunk with a running carry
    __shared__ long long sw[32];
    __shared__ long long tot;
    long long carry = 0;
    for (int c0 = 0; c0 < n; c0 += SCAN_B) {
        const int base = c0 + threadIdx.x * SCAN_I;
        long long v[SCAN_I], s = 0;
#pragma unroll
        for (int k = 0; k < SCAN_I; k++) {
            v[k] = (base + k < n) ? a[base + k] : 0;
            s += v[k];
        }
        long long off = block_excl_scan(s, sw, &tot) + carry;
#pragma unroll
        for (int k = 0; k < SCAN_I; k++) {
            if (base + k < n) a[base + k] = off;
            off += v[k];
        }
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) a[n] = carry;
}

__global__ void k_scan_apply(const int *in, int *out, int64_t n, const long long *boffs, long long *total) {
    __shared__ long long sw[32];
    __shared__ long long tot;
    int64_t base = (int64_t)blockIdx.x * SCAN_B + threadIdx.x * SCAN_I;
    int v[SCAN_I];
    long long s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; k++) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    long long off = block_excl_scan(s, sw, &tot) + boffs[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_I; k++) {
        if (base + k < n) out[base + k] = (int)off;
        off += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        long long t = boffs[blockIdx.x] + tot;
        *total = t;
        out[n] = (int)(t > INT_MAX ? INT_MAX : t);
    }
}

long long scan_ll_inplace(long long *a, int n, cudaStream_t s) {
    k_scan_ll_single<<<1, SCAN_T, 0, s>>>(a, n);
    CK_LAUNCH();
    long long h = 0;
    CK(cudaMemcpyAsync(&h, a + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return h;
}

int64_t scan_exclusive(const int *in, int *out, int64_t n, Scratch &sc, cudaStream_t s) {
    if (n == 0) {
        CK(cudaMemsetAsync(out, 0, sizeof(int), s));
        return 0;
    }
    const int64_t nb = (n + SCAN_B - 1) / SCAN_B;
    long long *bs = (long long *)sc.iscan.p;   // nb + 1 block offsets, then the total
    if ((size_t)(nb + 2) * sizeof(long long) > sc.iscan.bytes()) throw Error(BGS_INTERNAL, "scan too large");
    long long *total = bs + nb + 1;
    k_scan_sums<<<(unsigned)nb, SCAN_T, 0, s>>>(in, n, bs);
    CK_LAUNCH();
    k_scan_ll_single<<<1, SCAN_T, 0, s>>>(bs, (int)nb);
    CK_LAUNCH();
    k_scan_apply<<<(unsigned)nb, SCAN_T, 0, s>>>(in, out, n, bs, total);
    CK_LAUNCH();
    long long h = 0;
    CK(cudaMemcpyAsync(&h, total, sizeof(long long), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h > INT_MAX) throw Error(BGS_INVALID_ARG, "more than 2^31-1 entries");
    return h;
}

// ------------------------------------------------------------------------------------------
// Deterministic dot product
// ------------------------------------------------------------------------------------------
__device__ double block_sum(double v) {
    __shared__ double sw[32];
    v = warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sw[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = (lane < (int)(blockDim.x >> 5)) ? sw[lane] : 0.0;
        t = warp_sum(t);
    }
    return t;  // valid in thread 0
}

__global__ void k_dot_partial(const double *__restrict__ a, const double *__restrict__ b, int64_t n, double *part) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += a[i] * b[i];
    double t = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_reduce_final(const double *part, int g, double *out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < g; i += blockDim.x) acc += part[i];
    double t = block_sum(acc);
    if (threadIdx.x == 0) *out = t;
}

__global__ void k_reduce_final_rsqrt(const double *part, int g, double *out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < g; i += blockDim.x) acc += part[i];
    double t = block_sum(acc);
    if (threadIdx.x == 0) {
        out[0] = t;
        out[1] = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
    }
}

void dev_dot_rsqrt(const double *a, const double *b, int64_t n, double *out, double *partial, cudaStream_t s) {
    int g = grid_for(n, 256, num_sms() * 4);
    k_dot_partial<<<g, 256, 0, s>>>(a, b, n, partial);
    CK_LAUNCH();
    k_reduce_final_rsqrt<<<1, 256, 0, s>>>(partial, g, out);
    CK_LAUNCH();
}
void dev_dot_rsqrt(const double *a, const double *b, int64_t n, double *out, Scratch &sc, cudaStream_t s) {
    dev_dot_rsqrt(a, b, n, out, sc.partial.p, s);
}

void dev_dot(const double *a, const double *b, int64_t n, double *out, double *partial, cudaStream_t s) {
    int g = grid_for(n, 256, num_sms() * 4);
    k_dot_partial<<<g, 256, 0, s>>>(a, b, n, partial);
    CK_LAUNCH();
    k_reduce_final<<<1, 256, 0, s>>>(partial, g, out);
    CK_LAUNCH();
}
void dev_dot(const double *a, const double *b, int64_t n, double *out, Scratch &sc, cudaStream_t s) {
    dev_dot(a, b, n, out, sc.partial.p, s);
}

// ------------------------------------------------------------------------------------------
// Small element-wise kernels
// ------------------------------------------------------------------------------------------
template <class T>
__global__ void k_fill(T *p, T v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}
void dev_fill_int(int *p, int value, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_fill<int><<<grid_for(n, 256), 256, 0, s>>>(p, value, n);
    CK_LAUNCH();
}
void dev_fill_double(double *p, double value, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_fill<double><<<grid_for(n, 256), 256, 0, s>>>(p, value, n);
    CK_LAUNCH();
}

template <class A, class B>
__global__ void k_convert(const A *in, B *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (B)in[i];
}
__global__ void k_convert_bf(const double *in, __nv_bfloat16 *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __double2bfloat16(in[i]);
}
void convert_d2f(const double *in, float *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_convert<double, float><<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
    CK_LAUNCH();
}
void copy_d2f(const double *in, float *out, int64_t n, cudaStream_t s) { convert_d2f(in, out, n, s); }
void copy_f2d(const float *in, double *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_convert<float, double><<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
    CK_LAUNCH();
}
__global__ void k_copy_f2d_keep(const float *in, double *out, float *out_f, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = in[i];
        out[i] = (double)v;
        out_f[i] = v;
    }
}
void copy_f2d_keep(const float *in, double *out, float *out_f, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_copy_f2d_keep<<<grid_for(n, 256), 256, 0, s>>>(in, out, out_f, n);
    CK_LAUNCH();
}
void convert_d2bf(const double *in, __nv_bfloat16 *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_convert_bf<<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
    CK_LAUNCH();
}

__global__ void k_reciprocal(const double *in, double *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = 1.0 / in[i];
}
void reciprocal(const double *in, double *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_reciprocal<<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
    CK_LAUNCH();
}

__global__ void k_extract_diag(int n, const int *rp, const int *ci, const double *v, double *d) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double x = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; e++)
            if (ci[e] == i) {
                x = v[e];
                break;
            }
        d[i] = x;
    }
}
void extract_diag(const CsrView &A, double *diag, cudaStream_t s) {
    if (A.n <= 0) return;
    k_extract_diag<<<grid_for(A.n, 256), 256, 0, s>>>(A.n, A.rp, A.ci, A.v, diag);
    CK_LAUNCH();
}

__global__ void k_grad_outer(int n, const int *rp, const int *ci, const double *lam, const double *x, double *g) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double li = lam[i];
        for (int e = rp[i]; e < rp[i + 1]; e++) g[e] = -(li * x[ci[e]]);
    }
}
void grad_outer(const CsrView &A, const double *lam, const double *x, double *dvals, cudaStream_t s) {
    if (A.n <= 0) return;
    k_grad_outer<<<grid_for(A.n, 256), 256, 0, s>>>(A.n, A.rp, A.ci, lam, x, dvals);
    CK_LAUNCH();
}

// ------------------------------------------------------------------------------------------
// Validation
// ------------------------------------------------------------------------------------------
__global__ void k_validate(int n, int m, int64_t nnz, const int *rp, const int *ci, const double *v, int need_diag,
                           int *flag) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (rp[0] != 0 || (int64_t)rp[n] != nnz) atomicOr(flag, 1);
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int s = rp[i], e = rp[i + 1];
        if (s < 0 || e < s || (int64_t)e > nnz) {
            atomicOr(flag, 2);
            continue;
        }
        int prev = -1, has_diag = 0;
        for (int k = s; k < e; k++) {
            int c = ci[k];
            if (c < 0 || c >= m || c <= prev) atomicOr(flag, 4);
            double x = v[k];
            if (!(x == x) || x - x != 0.0) atomicOr(flag, 16);
            if (c == i) has_diag = 1;
            prev = c;
        }
        if (need_diag && !has_diag) atomicOr(flag, 8);
    }
}

void validate_csr_launch(const CsrView &A, bool need_diag, int *flag, cudaStream_t s) {
    CK(cudaMemsetAsync(flag, 0, sizeof(int), s));
    if (A.n > 0) {
        k_validate<<<grid_for(A.n, 256), 256, 0, s>>>(A.n, A.m, A.nnz, A.rp, A.ci, A.v, need_diag ? 1 : 0, flag);
        CK_LAUNCH();
    }
}

int validate_status(int flag) {
    if (flag & 16) return BGS_NAN_INF;
    return flag ? BGS_INVALID_ARG : BGS_OK;
}

int validate_csr(const CsrView &A, bool need_diag, Scratch &sc, cudaStream_t s) {
    validate_csr_launch(A, need_diag, sc.flags.p, s);
    CK(cudaMemcpyAsync(sc.h_flags, sc.flags.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return validate_status(sc.h_flags[0]);
}

// ------------------------------------------------------------------------------------------
// Row-wise concatenation of blocks (assembly of the full operator / coupling rows)
// ------------------------------------------------------------------------------------------
struct Parts {
    const int *rp[8];
    const int *ci[8];
    const double *v[8];
    int off[8];
    int np;
};

__global__ void k_concat_count(int n, Parts P, int *cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int c = 0;
        for (int p = 0; p < P.np; p++) c += P.rp[p][i + 1] - P.rp[p][i];
        cnt[i] = c;
    }
}

// One warp per 32 consecutive rows: for each part the lanes walk the part's entries of those rows
// (one contiguous range of the source) 32 apart, so the reads are coalesced and the writes land in
// runs; an entry's row within the group comes from a search over the group's row starts in shared
// memory, its destination from that row's start plus the row's entries of the earlier parts.
constexpr int kConcatWarps = 8;
__global__ void __launch_bounds__(kConcatWarps * 32) k_concat_fill(int n, Parts P, const int *rp, int *ci, double *v) {
    __shared__ int sst[kConcatWarps][33], sdst[kConcatWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t g0 = ((int64_t)blockIdx.x * kConcatWarps + w) * 32; g0 < n;
         g0 += (int64_t)gridDim.x * kConcatWarps * 32) {
        const int rows = (int)min((int64_t)32, n - g0);
        const int i = (int)g0 + lane;
        int dst = lane < rows ? rp[i] : 0;   // where row i's entries of part p start
        for (int p = 0; p < P.np; p++) {
            const int *prp = P.rp[p];
            const int st = lane < rows ? prp[i] : 0, en = lane < rows ? prp[i + 1] : 0;
            if (lane < rows) {
                sst[w][lane] = st;
                sdst[w][lane] = dst;
            }
            if (lane == rows - 1) sst[w][rows] = en;
            __syncwarp();
            const int e0 = sst[w][0], e1 = sst[w][rows];
            const int *pci = P.ci[p];
            const double *pv = P.v[p];
            const int off = P.off[p];
            for (int e = e0 + lane; e < e1; e += 32) {
                int lo = 0, hi = rows - 1;   // the last row whose start is <= e (it holds e)
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (sst[w][mid] <= e) lo = mid;
                    else hi = mid - 1;
                }
                const int q = sdst[w][lo] + (e - sst[w][lo]);
                ci[q] = pci[e] + off;
                v[q] = pv[e];
            }
            __syncwarp();
            dst += en - st;
        }
    }
}

static Parts make_parts(int nparts, const CsrView *parts, const int *col_offs) {
    Parts P{};
    if (nparts > 8) throw Error(BGS_INVALID_ARG, "more than 8 blocks in one block row");
    P.np = nparts;
    for (int p = 0; p < nparts; p++) {
        P.rp[p] = parts[p].rp;
        P.ci[p] = parts[p].ci;
        P.v[p] = parts[p].v;
        P.off[p] = col_offs[p];
    }
    return P;
}

void concat_count(int n, int nparts, const CsrView *parts, int *cnt, cudaStream_t s) {
    if (n <= 0) return;
    if (nparts == 0) {
        CK(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)n, s));
        return;
    }
    const int zero = 0;
    k_concat_count<<<grid_for(n, 256), 256, 0, s>>>(n, make_parts(nparts, parts, &zero), cnt);
    CK_LAUNCH();
}

void concat_fill(int n, int nparts, const CsrView *parts, const int *col_offs, const int *rp, int *ci, double *v,
                 cudaStream_t s) {
    if (n <= 0 || nparts == 0) return;
    const int g = (int)std::min<int64_t>(((int64_t)n + kConcatWarps * 32 - 1) / (kConcatWarps * 32),
                                         (int64_t)num_sms() * 16);
    k_concat_fill<<<g, kConcatWarps * 32, 0, s>>>(n, make_parts(nparts, parts, col_offs), rp, ci, v);
    CK_LAUNCH();
}

void concat_rows(int n, int nparts, const CsrView *parts, const int *col_offs, DCsr &C, Scratch &sc,
                 cudaStream_t s) {
    C.n = n;
    C.rp.alloc((size_t)n + 1, s);
    if (nparts == 0 || n == 0) {
        CK(cudaMemsetAsync(C.rp.p, 0, sizeof(int) * ((size_t)n + 1), s));
        C.nnz = 0;
        return;
    }
    concat_count(n, nparts, parts, C.rp.p, s);
    C.nnz = scan_exclusive(C.rp.p, C.rp.p, n, sc, s);
    C.ci.alloc((size_t)C.nnz, s);
    C.v.alloc((size_t)C.nnz, s);
    concat_fill(n, nparts, parts, col_offs, C.rp.p, C.ci.p, C.v.p, s);
}

}  // namespace bgs
