// SA-AMG setup on the device (Sec. 2.2.1, Eq. galerkin): strength filter (K3), MIS-2 rounds
// (K4), aggregation (K5), tentative + smoothed prolongator (K6), transpose (K8), two-pass
// hash SpGEMM for A_F P_tent, A P and R (A P) (K7), power iteration (K9) and the coarsest dense
// LU with an explicit inverse (K12).
//
// Integer decisions (strength, MIS-2, aggregates) follow the exact rules:
//  * j strong for i != j iff a_ij^2 > theta^2 |a_ii a_jj| or a_ji^2 > theta^2 |a_ii a_jj|, each
//    product rounded separately (no fused multiply-add), a missing entry counting as 0;
//  * MIS-2 by synchronous rounds with keys (fmix32(i ^ salt), i), salt = level * 0x9E3779B9;
//  * aggregates = root + strong neighbours, then the leftover nodes join the neighbouring
//    phase-1 aggregate with the largest |a_ij| (ties to the smaller id); ids by root index.
// SpGEMM accumulates every output entry in the order of the left operand's row, so the
// products are summed in a fixed order (mul and add rounded separately).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <cmath>
#include <cstdlib>
#include <mutex>

#include <climits>

#include "internal.h"

namespace bgs {

// Set-up phase tracing to stderr.  BGS_TRACE set: each phase's wall time, the stream synchronised
// at every mark.  BGS_TRACE=async: no synchronisation; each mark prints the host clock since the
// process's first mark and the stream, a timeline of the concurrent per-block set-ups (host-side,
// so it runs ahead of the GPU between the set-up's own synchronisations).
static std::chrono::steady_clock::time_point trace_origin() {
    static const std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    return t0;
}
static void timeline_print(const char *what, cudaStream_t s, int level, long long n) {
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - trace_origin()).count();
    fprintf(stderr, "bgs-timeline %10.3f ms stream %p level %d n %lld %s\n", ms, (void *)s, level, n, what);
}
struct Trace {
    bool on, async;
    cudaStream_t s;
    std::chrono::steady_clock::time_point t;
    explicit Trace(cudaStream_t st) : on(getenv("BGS_TRACE") != nullptr), async(false), s(st) {
        if (on) {
            async = strcmp(getenv("BGS_TRACE"), "async") == 0;
            if (!async) cudaStreamSynchronize(s);
            t = std::chrono::steady_clock::now();
            trace_origin();
            if (async) timeline_print("start", s, -1, 0);
        }
    }
    void mark(const char *what, int level, long long n) {
        if (!on) return;
        if (async) {
            timeline_print(what, s, level, n);
            return;
        }
        cudaStreamSynchronize(s);
        auto now = std::chrono::steady_clock::now();
        fprintf(stderr, "bgs-trace level %d n %lld %-18s %8.3f ms\n", level, n, what,
                std::chrono::duration<double, std::milli>(now - t).count());
        t = now;
    }
};

void timeline_mark(const char *what, cudaStream_t s) {
    const char *t = getenv("BGS_TRACE");
    if (t && strcmp(t, "async") == 0) timeline_print(what, s, -1, 0);
}

// ==========================================================================================
// Strength of connection
// ==========================================================================================
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ int find_in_row(const int *ci, int s, int e, int col) {
    int lo = s, hi = e - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int c = ci[mid];
        if (c == col) return mid;
        if (c < col) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

__global__ void k_strength(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ v,
                           const double *__restrict__ diag, double t2, uint8_t *strong, int *flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double aii = diag[i];
        if (aii == 0.0) atomicOr(flags, 2);
        for (int e = rp[i]; e < rp[i + 1]; e++) {
            const int j = ci[e];
            if (j == i) {
                strong[e] = 0;
                continue;
            }
            const int f = find_in_row(ci, rp[j], rp[j + 1], i);
            if (f < 0) atomicOr(flags, 1);   // structurally non-symmetric
            const double aji = f >= 0 ? v[f] : 0.0;
            const double aij = v[e];
            const double rhs = __dmul_rn(t2, fabs(__dmul_rn(aii, diag[j])));
            strong[e] = (__dmul_rn(aij, aij) > rhs || __dmul_rn(aji, aji) > rhs) ? 1 : 0;
        }
    }
}

__global__ void k_count_flag(int n, const int *rp, const uint8_t *flag, int *cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int c = 0;
        for (int e = rp[i]; e < rp[i + 1]; e++) c += flag[e];
        cnt[i] = c;
    }
}

__global__ void k_fill_flag(int n, const int *rp, const int *ci, const double *v, const uint8_t *flag, const int *orp,
                            int *oci, double *ov) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int q = orp[i];
        for (int e = rp[i]; e < rp[i + 1]; e++)
            if (flag[e]) {
                oci[q] = ci[e];
                ov[q] = v[e];
                q++;
            }
    }
}

// union of two sorted rows (A, B); values from A, 0 where only B has the column
__global__ void k_merge_count(int n, const int *arp, const int *aci, const int *brp, const int *bci, int *cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int a = arp[i], ae = arp[i + 1], b = brp[i], be = brp[i + 1], c = 0;
        while (a < ae || b < be) {
            if (b >= be || (a < ae && aci[a] < bci[b])) a++;
            else if (a >= ae || bci[b] < aci[a]) b++;
            else { a++; b++; }
            c++;
        }
        cnt[i] = c;
    }
}
__global__ void k_merge_fill(int n, const int *arp, const int *aci, const double *av, const int *brp, const int *bci,
                             const int *orp, int *oci, double *ov) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int a = arp[i], ae = arp[i + 1], b = brp[i], be = brp[i + 1], q = orp[i];
        while (a < ae || b < be) {
            if (b >= be || (a < ae && aci[a] < bci[b])) { oci[q] = aci[a]; ov[q] = av[a]; a++; }
            else if (a >= ae || bci[b] < aci[a]) { oci[q] = bci[b]; ov[q] = 0.0; b++; }
            else { oci[q] = aci[a]; ov[q] = av[a]; a++; b++; }
            q++;
        }
    }
}

// ==========================================================================================
// Transpose with sorted rows
// ==========================================================================================
__global__ void k_tr_count(int64_t nnz, const int *ci, int *cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[ci[e]], 1);
}
__global__ void k_tr_fill(int n, const int *rp, const int *ci, const double *v, const int *trp, int *cur, int *tci,
                          double *tv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int e = rp[i]; e < rp[i + 1]; e++) {
            int c = ci[e];
            int p = trp[c] + atomicAdd(&cur[c], 1);
            tci[p] = i;
            if (v) tv[p] = v[e];
        }
}
// rank sort of each row (keys distinct): one warp per row, reading the unsorted copy
__global__ void k_row_rank_sort(int n, const int *rp, const int *ici, const double *iv, int *oci, double *ov) {
    const int lane = threadIdx.x & 31;
    for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += (gridDim.x * blockDim.x) >> 5) {
        const int s = rp[r], e = rp[r + 1];
        for (int t = s + lane; t < e; t += 32) {
            const int k = ici[t];
            int rank = 0;
            for (int q = s; q < e; q++) rank += ici[q] < k;
            oci[s + rank] = k;
            if (iv) ov[s + rank] = iv[t];
        }
    }
}

void transpose_csr(const CsrView &A, DCsr &T, Scratch &sc, cudaStream_t s) {
    T.n = A.m;
    T.m = A.n;
    T.nnz = A.nnz;
    T.rp.alloc((size_t)A.m + 1, s);
    CK(cudaMemsetAsync(T.rp.p, 0, sizeof(int) * ((size_t)A.m + 1), s));
    if (A.nnz > 0) {
        k_tr_count<<<grid_for(A.nnz, 256), 256, 0, s>>>(A.nnz, A.ci, T.rp.p);
        CK_LAUNCH();
    }
    scan_exclusive(T.rp.p, T.rp.p, A.m, sc, s);
    DBuf<int> cur((size_t)A.m + 1, s), tci((size_t)std::max<int64_t>(A.nnz, 1), s);
    DBuf<double> tv;
    if (A.v) tv.alloc((size_t)std::max<int64_t>(A.nnz, 1), s);
    CK(cudaMemsetAsync(cur.p, 0, sizeof(int) * ((size_t)A.m + 1), s));
    T.ci.alloc((size_t)A.nnz, s);
    if (A.v) T.v.alloc((size_t)A.nnz, s);
    if (A.n > 0 && A.nnz > 0) {
        k_tr_fill<<<grid_for(A.n, 256), 256, 0, s>>>(A.n, A.rp, A.ci, A.v, T.rp.p, cur.p, tci.p, tv.p);
        CK_LAUNCH();
        k_row_rank_sort<<<grid_for((int64_t)A.m * 32, 256), 256, 0, s>>>(A.m, T.rp.p, tci.p, tv.p, T.ci.p, T.v.p);
        CK_LAUNCH();
    }
}

// ==========================================================================================
// Strength graph
// ==========================================================================================
// S: undirected strength graph without the diagonal, values a_ij (0 where only a_ji is stored).
static void strength_graph(const CsrView &A, const uint8_t *strong, bool asym, DCsr &S, Scratch &sc,
                           cudaStream_t s) {
    const int n = A.n;
    DCsr SA;
    SA.n = SA.m = n;
    SA.rp.alloc((size_t)n + 1, s);
    k_count_flag<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp, strong, SA.rp.p);
    CK_LAUNCH();
    SA.nnz = scan_exclusive(SA.rp.p, SA.rp.p, n, sc, s);
    SA.ci.alloc((size_t)SA.nnz, s);
    SA.v.alloc((size_t)SA.nnz, s);
    k_fill_flag<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp, A.ci, A.v, strong, SA.rp.p, SA.ci.p, SA.v.p);
    CK_LAUNCH();
    if (!asym) {   // symmetric pattern: the symmetric test makes S_A symmetric already
        S = std::move(SA);
        return;
    }
    DCsr ST;
    transpose_csr(view(SA), ST, sc, s);
    S.n = S.m = n;
    S.rp.alloc((size_t)n + 1, s);
    k_merge_count<<<grid_for(n, 256), 256, 0, s>>>(n, SA.rp.p, SA.ci.p, ST.rp.p, ST.ci.p, S.rp.p);
    CK_LAUNCH();
    S.nnz = scan_exclusive(S.rp.p, S.rp.p, n, sc, s);
    S.ci.alloc((size_t)S.nnz, s);
    S.v.alloc((size_t)S.nnz, s);
    k_merge_fill<<<grid_for(n, 256), 256, 0, s>>>(n, SA.rp.p, SA.ci.p, SA.v.p, ST.rp.p, ST.ci.p, S.rp.p, S.ci.p,
                                                   S.v.p);
    CK_LAUNCH();
}

// ==========================================================================================
// MIS-2 rounds and aggregation
// ==========================================================================================
__device__ __forceinline__ unsigned long long mis_key1(int i, uint32_t salt) {
    return ((((unsigned long long)fmix32((uint32_t)i ^ salt)) << 32) | (unsigned long long)(uint32_t)i) + 1ull;
}

// m1[v] = max key over undecided nodes of the closed neighbourhood of v (0: none)
__global__ void k_mis_m1(int n, const int *rp, const int *ci, const int *state, uint32_t salt,
                         unsigned long long *m1) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        unsigned long long m = state[v] == 0 ? mis_key1(v, salt) : 0ull;
        for (int e = rp[v]; e < rp[v + 1]; e++) {
            int u = ci[e];
            if (state[u] == 0) {
                unsigned long long k = mis_key1(u, salt);
                m = k > m ? k : m;
            }
        }
        m1[v] = m;
    }
}
// undecided v becomes a root iff the maximum over its distance-2 ball is its own key
__global__ void k_mis_select(int n, const int *rp, const int *ci, int *state, uint32_t salt,
                             const unsigned long long *m1) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (state[v] != 0) continue;
        unsigned long long m = m1[v];
        for (int e = rp[v]; e < rp[v + 1]; e++) {
            unsigned long long k = m1[ci[e]];
            m = k > m ? k : m;
        }
        if (m == mis_key1(v, salt)) state[v] = 1;
    }
}
__global__ void k_mis_f1(int n, const int *rp, const int *ci, const int *state, int *f1) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int f = state[v] == 1;
        for (int e = rp[v]; e < rp[v + 1] && !f; e++) f = state[ci[e]] == 1;
        f1[v] = f;
    }
}
__global__ void k_mis_out(int n, const int *rp, const int *ci, int *state, const int *f1, int *undecided) {
    int local = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (state[v] != 0) continue;
        int f = f1[v];
        for (int e = rp[v]; e < rp[v + 1] && !f; e++) f = f1[ci[e]];
        if (f) state[v] = 2;
        else local++;
    }
    if (local) atomicAdd(undecided, local);
}

// Rounds are launched in batches with one read-back per batch (each round leaves its count of
// undecided nodes in its own slot); a round after the last one changes nothing, so the round count
// is the first round that left no node undecided.
static int mis2(const DCsr &S, uint32_t salt, int *state, Scratch &sc, cudaStream_t s) {
    const int n = S.n;
    DBuf<unsigned long long> m1((size_t)n, s);
    DBuf<int> f1((size_t)n, s);
    constexpr int kBatch = 4;
    DBuf<int> left((size_t)kBatch, s);
    CK(cudaMemsetAsync(state, 0, sizeof(int) * (size_t)n, s));
    const int g = grid_for(n, 256);
    int rounds = 0;
    for (;;) {
        CK(cudaMemsetAsync(left.p, 0, sizeof(int) * kBatch, s));
        for (int b = 0; b < kBatch; b++) {
            k_mis_m1<<<g, 256, 0, s>>>(n, S.rp.p, S.ci.p, state, salt, m1.p);
            CK_LAUNCH();
            k_mis_select<<<g, 256, 0, s>>>(n, S.rp.p, S.ci.p, state, salt, m1.p);
            CK_LAUNCH();
            k_mis_f1<<<g, 256, 0, s>>>(n, S.rp.p, S.ci.p, state, f1.p);
            CK_LAUNCH();
            k_mis_out<<<g, 256, 0, s>>>(n, S.rp.p, S.ci.p, state, f1.p, left.p + b);
            CK_LAUNCH();
        }
        CK(cudaMemcpyAsync(sc.h_flags + 20, left.p, sizeof(int) * kBatch, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int b = 0; b < kBatch; b++) {
            rounds++;
            if (sc.h_flags[20 + b] == 0) return rounds;
        }
        if (rounds > n + 1) throw Error(BGS_INTERNAL, "MIS-2 did not terminate");
    }
}

__global__ void k_root_flag(int n, const int *state, int *f) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) f[i] = state[i] == 1;
}
__global__ void k_phase1(int n, const int *rp, const int *ci, const int *state, const int *rootid, int *ph1) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int a = -1;
        if (state[i] == 1) a = rootid[i];
        else
            for (int e = rp[i]; e < rp[i + 1]; e++)
                if (state[ci[e]] == 1) a = rootid[ci[e]];
        ph1[i] = a;
    }
}
__global__ void k_phase2(int n, const int *rp, const int *ci, const double *v, const int *ph1, int *agg, int *bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int a = ph1[i];
        if (a < 0) {
            double bw = -1.0;
            for (int e = rp[i]; e < rp[i + 1]; e++) {
                int j = ci[e];
                int pj = ph1[j];
                if (j == i || pj < 0) continue;
                double w = fabs(v[e]);
                if (w > bw || (w == bw && pj < a)) {
                    bw = w;
                    a = pj;
                }
            }
            if (a < 0) atomicOr(bad, 1);
        }
        agg[i] = a;
    }
}

static int aggregate(const DCsr &S, const int *state, int *agg, Scratch &sc, cudaStream_t s) {
    const int n = S.n;
    DBuf<int> rootid((size_t)n + 1, s), ph1((size_t)n, s);
    const int g = grid_for(n, 256);
    k_root_flag<<<g, 256, 0, s>>>(n, state, rootid.p);
    CK_LAUNCH();
    int nagg = (int)scan_exclusive(rootid.p, rootid.p, n, sc, s);
    k_phase1<<<g, 256, 0, s>>>(n, S.rp.p, S.ci.p, state, rootid.p, ph1.p);
    CK_LAUNCH();
    CK(cudaMemsetAsync(sc.flags.p + 5, 0, sizeof(int), s));
    k_phase2<<<g, 256, 0, s>>>(n, S.rp.p, S.ci.p, S.v.p, ph1.p, agg, sc.flags.p + 5);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(sc.h_flags + 5, sc.flags.p + 5, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return sc.h_flags[5] ? -1 : nagg;
}

// ==========================================================================================
// Filtered matrix (compact: diagonal + strong entries, dropped entries lumped on the diagonal)
// ==========================================================================================
__global__ void k_filter_count(int n, const int *rp, const int *ci, const uint8_t *strong, int *cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int c = 0;
        for (int e = rp[i]; e < rp[i + 1]; e++) c += (ci[e] == i) || strong[e];
        cnt[i] = c;
    }
}
__global__ void k_filter_fill(int n, const int *rp, const int *ci, const double *v, const uint8_t *strong,
                              const int *frp, int *fci, double *fv, double *dinvF, int filter_diag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double lump = 0.0, rabs = 0.0;
        int nstrong = 0;
        for (int e = rp[i]; e < rp[i + 1]; e++) {
            if (ci[e] != i && !strong[e]) lump += v[e];
            rabs += fabs(v[e]);
            nstrong += ci[e] != i && strong[e];
        }
        int q = frp[i];
        double dg = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; e++) {
            if (ci[e] == i) {
                fci[q] = i;
                fv[q] = v[e] + lump;
                // only the lumped diagonal left and zero up to rounding (a zero row sum, below
                // 1e-12 of the row's absolute sum): an exact zero row
                if (nstrong == 0 && fabs(fv[q]) <= 1e-12 * rabs) fv[q] = 0.0;
                dg = fv[q];
                q++;
            } else if (strong[e]) {
                fci[q] = ci[e];
                fv[q] = v[e];
                q++;
            }
        }
        if (filter_diag) {
            double sabs = 0.0;
            for (int t = frp[i]; t < q; t++) sabs += fabs(fv[t]);
            dg = sabs;
        }
        // a row whose lumped filtered entries are all zero takes no part in the smoothing
        dinvF[i] = dg != 0.0 ? 1.0 / dg : 0.0;
    }
}

// ==========================================================================================
// Power iteration: lambda_max(D^-1 A), start v0_i = ((fmix32(i ^ 0x7F4A7C15) >> 8) + 0.5) / 2^24
// ==========================================================================================
__global__ void k_power_start(int n, double *v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t u = fmix32((uint32_t)i ^ 0x7F4A7C15u) >> 8;
        v[i] = ((double)u + 0.5) / 16777216.0;
    }
}

// The iterates u_k = (D^-1 A)^k u_0 are left unnormalised and the estimate is ||u_k|| / ||u_k-1||
// from the last two, which equals ||D^-1 A v|| for the normalised v = u_k-1 / ||u_k-1|| of the
// textbook iteration.  Every 8 steps (never on the last) the iterate is rescaled to unit norm, so
// its size stays far from FP64's range limits however many steps are asked for.
// The steps, enqueued on s with no read-back: out[0] = ||u_k||^2, out[2] = ||u_k-1||^2 (out[0..1]
// also hold (||v||^2, 1/||v||) for the rescaling steps); partial: num_sms() * 4 doubles.
static void power_enqueue(const DCsr &A, const double *dinv, int iters, double *partial, double *out,
                          cudaStream_t s) {
    const int n = A.n;
    DBuf<double> v((size_t)n, s), w((size_t)n, s);
    k_power_start<<<grid_for(n, 256), 256, 0, s>>>(n, v.p);
    CK_LAUNCH();
    double *nv = out, *nw = out + 2;
    for (int it = 0; it < iters; it++) {
        if (it > 0 && it % 8 == 0 && it < iters - 1) {
            dev_dot_rsqrt(v.p, v.p, n, nv, partial, s);      // (||v||^2, 1/||v||)
            spmv_scaled_norm(A, dinv, v.p, nv + 1, w.p, s);  // w = D^-1 A (v / ||v||)
        } else {
            spmv_scaled_norm(A, dinv, v.p, nullptr, w.p, s); // w = D^-1 A v
        }
        std::swap(v.p, w.p);
    }
    dev_dot(v.p, v.p, n, nv, partial, s);   // ||u_k||^2
    dev_dot(w.p, w.p, n, nw, partial, s);   // ||u_k-1||^2
}

static double power_estimate(double a, double b) { return b > 0.0 ? std::sqrt(a / b) : 0.0; }

static double power_lambda(const DCsr &A, const double *dinv, int iters, Scratch &sc, cudaStream_t s) {
    double *out = sc.scal.p + 20;
    power_enqueue(A, dinv, iters, sc.partial.p, out, s);
    CK(cudaMemcpyAsync(sc.h_scal + 1, out, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(sc.h_scal + 2, out + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return power_estimate(sc.h_scal[1], sc.h_scal[2]);
}

// ==========================================================================================
// Hash SpGEMM C = A B (two passes; warp per row; shared-memory tables, global tables for big rows)
// ==========================================================================================
constexpr int SG_WARPS = 8;
constexpr int SG_SYM_T = 2048;
constexpr int SG_NUM_T = 1024;
constexpr int SG_LOCAL = 48;       // thread-per-row path: at most this many distinct columns
constexpr int SG_LOCAL_UB = 128;   // and at most this many products; other rows use the warp-hash path
constexpr int SG_SMALL_T = 256;    // warp-hash tables up to this size run with small shared tables

__device__ __forceinline__ unsigned nextpow2u(unsigned x) {
    x = x < 2 ? 2 : x;
    return 1u << (32 - __clz(x - 1));
}

__device__ __forceinline__ int tbl_insert(int *keys, unsigned mask, int col, bool &ins) {
    unsigned h = ((unsigned)col * 2654435761u) & mask;
    for (unsigned t = 0; t <= mask; t++) {
        int k = ((volatile int *)keys)[h];
        if (k == col) { ins = false; return (int)h; }
        if (k == -1) {
            int old = atomicCAS(&keys[h], -1, col);
            if (old == -1) { ins = true; return (int)h; }
            if (old == col) { ins = false; return (int)h; }
        }
        h = (h + 1) & mask;
    }
    ins = false;
    return -1;
}


// Accumulate the products of one row into a hash table, one warp: lanes take 32 entries of the
// left operand's row at a time and walk their right-operand rows in step.  Lanes of one step that
// hit the same column are grouped (__match_any_sync); the group leader owns the column's slot
// and adds the group's products to it in lane order (= left-operand order), each as one fused
// multiply-add, so no two lanes race on a slot and the sums are reproducible.  sv holds 64
// doubles per warp: the lanes' left values (per chunk) and right values (per step).  Returns
// this lane's count of new columns; sets over if the table's limit is passed (symbolic pass with
// a capped shared table).
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }

template <bool NUM, class VT>
__device__ int sg_accumulate(int row, int *keys, VT *vals, unsigned T, bool capped, VT *sv, const int *arp,
                             const int *aci, const VT *av, const int *brp, const int *bci, const VT *bv,
                             bool &over) {
    const int lane = threadIdx.x & 31;
    const unsigned mask = T - 1;
    int mine = 0;
    const int rb = arp[row], re = arp[row + 1];
    for (int e0 = rb; e0 < re; e0 += 32) {
        const int e = e0 + lane;
        const bool has = e < re;
        const int k = has ? aci[e] : 0;
        const VT a = (NUM && has) ? av[e] : (VT)0;
        const int bs = has ? brp[k] : 0;
        const int len = has ? brp[k + 1] - bs : 0;
        const int maxlen = __reduce_max_sync(0xffffffffu, len);
        if (NUM) sv[lane] = a;   // read by the leaders after the first step's __syncwarp
        // lane l walks its right-operand row starting at entry l mod len: the rows of neighbouring
        // left entries share most of their columns in sorted order, so stepping them in lockstep
        // from their first entries made most lanes of a step hit the same column (long serial
        // group sums); the rotated walks spread a step's lanes over the row's columns
        const int rot = len > 0 ? lane % len : 0;
        for (int q = 0; q < maxlen; q++) {
            const bool act = q < len;
            const int qq = act ? (q + rot < len ? q + rot : q + rot - len) : 0;
            const int j = act ? bci[bs + qq] : -1;
            const unsigned grp = __match_any_sync(0xffffffffu, j);
            const int leader = __ffs(grp) - 1;
            if (NUM && act) sv[32 + lane] = bv[bs + qq];
            __syncwarp();
            if (act && lane == leader) {
                bool ins;
                const int sl = tbl_insert(keys, mask, j, ins);
                if (sl < 0) over = true;
                else {
                    if (NUM) {
                        VT v = vals[sl];
                        for (unsigned g = grp; g; g &= g - 1) {
                            const int m = __ffs(g) - 1;
                            v = vfma(sv[m], sv[32 + m], v);
                        }
                        vals[sl] = v;
                    }
                    mine += ins;
                }
            }
            __syncwarp();
            if (capped) {
                const int total = __reduce_add_sync(0xffffffffu, mine);
                if (__any_sync(0xffffffffu, over) || total > (int)(T / 2)) {
                    over = true;
                    return mine;
                }
            }
        }
    }
    over = __any_sync(0xffffffffu, over);
    return mine;
}

__global__ void k_sg_ub(int n, const int *arp, const int *aci, const int *brp, int *ub) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        long long u = 0;
        for (int e = arp[i]; e < arp[i + 1]; e++) u += brp[aci[e] + 1] - brp[aci[e]];
        ub[i] = (int)(u > 0x3fffffff ? 0x3fffffff : u);
    }
}

// symbolic: distinct column count per row; rows that overflow the shared table get -1
template <int TMAX>
__global__ void __launch_bounds__(SG_WARPS * 32) k_sg_sym(int n, const int *rows, const int *arp, const int *aci,
                                                          const int *brp, const int *bci, const int *ub, int *cnt) {
    extern __shared__ int sg_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int *keys = sg_smem + wib * TMAX;
    for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < n; it += (gridDim.x * blockDim.x) >> 5) {
        const int row = rows ? rows[it] : it;
        const int u = ub[row];
        if (u == 0) {
            if (lane == 0) cnt[row] = 0;
            continue;
        }
        const unsigned T = min((unsigned)TMAX, nextpow2u(2u * (unsigned)u));
        for (unsigned t = lane; t < T; t += 32) keys[t] = -1;
        __syncwarp();
        bool over = false;
        const int mine = sg_accumulate<false, double>(row, keys, nullptr, T, T == (unsigned)TMAX && u > (int)(TMAX / 2),
                                              nullptr, arp, aci, nullptr, brp, bci, nullptr, over);
        const int total = __reduce_add_sync(0xffffffffu, mine);
        if (lane == 0) cnt[row] = over ? -1 : total;
        __syncwarp();
    }
}

// symbolic for big rows: global table per row
// (open_only: rows whose count is already there, cnt[row] >= 0, are skipped)
__global__ void k_sg_sym_big(int nbig, const int *rows, const long long *toff, int *gkeys, const int *arp,
                             const int *aci, const int *brp, const int *bci, int *cnt, int open_only) {
    const int lane = threadIdx.x & 31;
    for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nbig; b += (gridDim.x * blockDim.x) >> 5) {
        const int row = rows[b];
        if (open_only && cnt[row] >= 0) continue;
        int *keys = gkeys + toff[b];
        const unsigned T = (unsigned)(toff[b + 1] - toff[b]);
        for (unsigned t = lane; t < T; t += 32) keys[t] = -1;
        __syncwarp();
        bool over = false;
        const int mine = sg_accumulate<false, double>(row, keys, nullptr, T, false, nullptr, arp, aci, nullptr, brp, bci,
                                              nullptr, over);
        const int total = __reduce_add_sync(0xffffffffu, mine);
        if (lane == 0) cnt[row] = total;
    }
}

// numeric accumulate + in-place compaction + rank sort into the output row
template <class VT>
__device__ void sg_numeric_row(int row, int *keys, VT *vals, unsigned T, VT *sv, const int *arp, const int *aci,
                               const VT *av, const int *brp, const int *bci, const VT *bv, const int *crp, int *cci,
                               VT *cv, int *err) {
    const int lane = threadIdx.x & 31;
    for (unsigned t = lane; t < T; t += 32) {
        keys[t] = -1;
        vals[t] = (VT)0;
    }
    __syncwarp();
    bool over = false;
    sg_accumulate<true, VT>(row, keys, vals, T, false, sv, arp, aci, av, brp, bci, bv, over);
    if (over) {
        if (lane == 0) atomicOr(err, 1);
        return;
    }
    int wpos = 0;
    for (unsigned base = 0; base < T; base += 32) {
        const unsigned sl = base + lane;
        const int k = sl < T ? keys[sl] : -1;
        const VT v = sl < T ? vals[sl] : (VT)0;
        const unsigned bal = __ballot_sync(0xffffffffu, k != -1);
        const int pos = wpos + __popc(bal & ((1u << lane) - 1u));
        __syncwarp();
        if (k != -1) {
            keys[pos] = k;
            vals[pos] = v;
        }
        wpos += __popc(bal);
        __syncwarp();
    }
    const int c = wpos;
    const int out = crp[row];
    if (c != crp[row + 1] - out) {   // must equal the symbolic count; never write past the row
        if (lane == 0) atomicOr(err, 1);
        return;
    }
    for (int t = lane; t < c; t += 32) {
        const int kt = keys[t];
        int rank = 0;
        for (int q = 0; q < c; q++) rank += keys[q] < kt;
        cci[out + rank] = kt;
        cv[out + rank] = vals[t];
    }
    __syncwarp();
}

// shared memory of k_sg_num per block: SG_WARPS tables of TMAX values and keys, 64 staged values
template <int TMAX, class VT>
constexpr int sg_num_smem() {
    return (int)(sizeof(VT) * SG_WARPS * (TMAX + 64) + sizeof(int) * SG_WARPS * TMAX);
}

template <int TMAX, class VT>
__global__ void __launch_bounds__(SG_WARPS * 32) k_sg_num(int n, const int *rows, const int *arp, const int *aci,
                                                          const VT *av, const int *brp, const int *bci, const VT *bv,
                                                          const int *crp, int *cci, VT *cv, int *err) {
    extern __shared__ __align__(16) unsigned char sg_nsm_raw[];
    VT *sg_nsm = reinterpret_cast<VT *>(sg_nsm_raw);
    const int wib = threadIdx.x >> 5;
    VT *vals = sg_nsm + wib * TMAX;
    VT *sv = sg_nsm + SG_WARPS * TMAX + wib * 64;
    int *keys = (int *)(sg_nsm + SG_WARPS * (TMAX + 64)) + wib * TMAX;
    for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < n; it += (gridDim.x * blockDim.x) >> 5) {
        const int row = rows ? rows[it] : it;
        const int c = crp[row + 1] - crp[row];
        if (c == 0 || c > TMAX / 2) continue;
        const unsigned T = nextpow2u(2u * (unsigned)c);
        sg_numeric_row(row, keys, vals, T, sv, arp, aci, av, brp, bci, bv, crp, cci, cv, err);
    }
}

template <class VT>
// (rows of at most min_c columns are skipped: a shared-table kernel made them)
__global__ void k_sg_num_big(int nbig, const int *rows, const long long *toff, int *gkeys, VT *gvals, const int *arp,
                             const int *aci, const VT *av, const int *brp, const int *bci, const VT *bv,
                             const int *crp, int *cci, VT *cv, int *err, int min_c) {
    __shared__ VT svb[8][64];
    for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nbig; b += (gridDim.x * blockDim.x) >> 5) {
        if (crp[rows[b] + 1] - crp[rows[b]] <= min_c) continue;
        const unsigned T = (unsigned)(toff[b + 1] - toff[b]);
        sg_numeric_row(rows[b], gkeys + toff[b], gvals + toff[b], T, svb[(threadIdx.x >> 5) & 7], arp, aci, av, brp,
                       bci, bv, crp, cci, cv, err);
    }
}

__global__ void k_big_mark(int n, const int *cnt, int limit, int *flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flag[i] = (cnt[i] < 0 || cnt[i] > limit) ? 1 : 0;
}
__global__ void k_big_list(int n, const int *flag, const int *pos, int *rows) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (flag[i]) rows[pos[i]] = i;
}
// table sizes nextpow2(2 * size) for the big rows (size = ub for symbolic, cnt for numeric)
__global__ void k_big_tsize(int nbig, const int *rows, const int *size, long long *toff) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbig; b += gridDim.x * blockDim.x) {
        unsigned s = (unsigned)size[rows[b]];
        unsigned t = 2;
        while (t < 2u * s) t <<= 1;
        toff[b] = (long long)t;
    }
}
__global__ void k_ll_excl_scan_small(long long *a, int n) {
    // n is small (number of big rows); one thread
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        long long s = 0;
        for (int i = 0; i < n; i++) {
            long long t = a[i];
            a[i] = s;
            s += t;
        }
        a[n] = s;
    }
}

static int collect_flag(int n, const int *flag, DBuf<int> &rows, Scratch &sc, cudaStream_t s) {
    DBuf<int> pos((size_t)n + 1, s);
    int nb = (int)scan_exclusive(flag, pos.p, n, sc, s);
    rows.alloc((size_t)std::max(nb, 1), s);
    if (nb) {
        k_big_list<<<grid_for(n, 256), 256, 0, s>>>(n, flag, pos.p, rows.p);
        CK_LAUNCH();
    }
    return nb;
}

static int collect_big(int n, const int *cnt, int limit, DBuf<int> &rows, Scratch &sc, cudaStream_t s) {
    DBuf<int> flag((size_t)n + 1, s);
    k_big_mark<<<grid_for(n, 256), 256, 0, s>>>(n, cnt, limit, flag.p);
    CK_LAUNCH();
    DBuf<int> pos((size_t)n + 1, s);
    int nbig = (int)scan_exclusive(flag.p, pos.p, n, sc, s);
    rows.alloc((size_t)std::max(nbig, 1), s);
    if (nbig) {
        k_big_list<<<grid_for(n, 256), 256, 0, s>>>(n, flag.p, pos.p, rows.p);
        CK_LAUNCH();
    }
    return nbig;
}

static long long big_tables(int nbig, const int *rows, const int *size, DBuf<long long> &toff, cudaStream_t s) {
    toff.alloc((size_t)nbig + 1, s);
    k_big_tsize<<<grid_for(nbig, 256), 256, 0, s>>>(nbig, rows, size, toff.p);
    CK_LAUNCH();
    if (nbig > 100000) throw Error(BGS_INTERNAL, "too many long SpGEMM rows");
    k_ll_excl_scan_small<<<1, 1, 0, s>>>(toff.p, nbig);
    CK_LAUNCH();
    long long total = 0;
    CK(cudaMemcpyAsync(&total, toff.p + nbig, sizeof(long long), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return total;
}

// symbolic rows still open (cnt < 0) whose table for ub products fits in hi slots
__global__ void k_sym_class(int n, const int *cnt, const int *ub, unsigned hi, int *flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned t = 2;
        while (t < 2u * (unsigned)ub[i]) t <<= 1;
        flag[i] = (cnt[i] < 0 && t <= hi) ? 1 : 0;
    }
}

// flag rows whose needed table size nextpow2(2 * size[i]) lies in (lo, hi] (size[i] < 0: use ub)
__global__ void k_table_class(int n, const int *size, const int *ub, unsigned lo, unsigned hi, int *flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int sz = size[i] < 0 ? ub[i] : size[i];
        unsigned t = 2;
        while (t < 2u * (unsigned)sz) t <<= 1;
        flag[i] = (sz > 0 && t > lo && t <= hi) ? 1 : 0;
    }
}

__global__ void k_hash_rows(int n, const int *cnt, const int *ub, int *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (ub[i] > SG_LOCAL_UB || cnt[i] > SG_LOCAL) ? cnt[i] : 0;
}

__global__ void k_row_lengths(int n, const int *rp, int *len) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) len[i] = rp[i + 1] - rp[i];
}

// Short rows (at most SG_LOCAL_UB products), one thread per row.  Symbolic: the distinct output
// columns of the row in an insertion-sorted local list (at most SG_LOCAL entries), written to the
// row's SG_LOCAL slots of cols; rows with more distinct columns report -1 and go to the warp-hash
// kernels.  Numeric: the row's sorted columns are copied into C, its values start at 0, and every
// product, in the order of the left operand's row, is added in place at its column (binary search
// in the row), so each output entry is summed in that order.
__global__ void __launch_bounds__(128) k_sg_local_sym(int n, const int *__restrict__ arp, const int *__restrict__ aci,
                                                      const int *__restrict__ brp, const int *__restrict__ bci,
                                                      const int *__restrict__ ub, int *cnt, int *cols) {
    int lc[SG_LOCAL];
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
        if (ub[row] > SG_LOCAL_UB) {
            cnt[row] = -1;
            continue;
        }
        int c = 0;
        bool over = false;
        for (int e = arp[row]; e < arp[row + 1] && !over; e++) {
            const int k = aci[e];
            for (int f = brp[k]; f < brp[k + 1]; f++) {
                const int j = bci[f];
                int p = c - 1;
                while (p >= 0 && lc[p] > j) p--;
                if (p >= 0 && lc[p] == j) continue;
                if (c == SG_LOCAL) {
                    over = true;
                    break;
                }
                for (int q = c; q > p + 1; q--) lc[q] = lc[q - 1];
                lc[p + 1] = j;
                c++;
            }
        }
        cnt[row] = over ? -1 : c;
        if (!over) {
            int *out = cols + (size_t)row * SG_LOCAL;
            for (int q = 0; q < c; q++) out[q] = lc[q];
        }
    }
}

// acc + a b with the product rounded on its own (no fused multiply-add), as the oracle sums
__device__ __forceinline__ double add_mul_rn(double acc, double a, double b) { return __dadd_rn(acc, __dmul_rn(a, b)); }
__device__ __forceinline__ float add_mul_rn(float acc, float a, float b) { return __fadd_rn(acc, __fmul_rn(a, b)); }

template <class VT>
__global__ void __launch_bounds__(128) k_sg_local_num(int n, const int *__restrict__ arp, const int *__restrict__ aci,
                                                      const VT *__restrict__ av, const int *__restrict__ brp,
                                                      const int *__restrict__ bci, const VT *__restrict__ bv,
                                                      const int *__restrict__ ub, const int *__restrict__ cols,
                                                      const int *__restrict__ crp, int *cci, VT *cv, int *err) {
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
        const int o = crp[row], c = crp[row + 1] - o;
        if (ub[row] > SG_LOCAL_UB || c > SG_LOCAL) continue;   // handled by the hash path
        const int *in = cols + (size_t)row * SG_LOCAL;
        int *rc = cci + o;
        VT *rv = cv + o;
        for (int q = 0; q < c; q++) {
            rc[q] = in[q];
            rv[q] = (VT)0;
        }
        for (int e = arp[row]; e < arp[row + 1]; e++) {
            const int k = aci[e];
            const VT a = av[e];
            for (int f = brp[k]; f < brp[k + 1]; f++) {
                const int j = bci[f];
                int lo = 0, hi = c;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (rc[mid] < j) lo = mid + 1;
                    else hi = mid;
                }
                if (lo >= c || rc[lo] != j) {   // not in the symbolic pattern: never write outside it
                    atomicOr(err, 1);
                    continue;
                }
                rv[lo] = add_mul_rn(rv[lo], a, bv[f]);
            }
        }
    }
}

__global__ void k_iota(int n, int *a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = i;
}

// Products with few rows (the coarse levels): every row first through the shared-memory hash
// kernels (a symbolic table of SG_SYM_T slots, capped; a numeric table sized from the row's column
// count, up to SG_NUM_T slots), and the rows that do not fit through global-memory tables sized
// from their product counts, all launched over every row without classifying them first: three
// read-backs in all (table total, row counts, error flag).  The coarsest products have few rows of
// thousands of products but a few dozen columns, which the shared tables serve.
constexpr int kSgSmallRows = 16384;
template <class VT>
static void spgemm_small(const CsrView &A, const VT *av, const CsrView &B, const VT *bv, DCsr &C, DBuf<VT> &cv,
                         const int *ub, Scratch &sc, cudaStream_t s) {
    const int n = A.n;
    DBuf<int> rows((size_t)n, s);
    k_iota<<<grid_for(n, 256), 256, 0, s>>>(n, rows.p);
    CK_LAUNCH();
    DBuf<long long> toff((size_t)n + 1, s);
    k_big_tsize<<<grid_for(n, 256), 256, 0, s>>>(n, rows.p, ub, toff.p);
    CK_LAUNCH();
    const long long tot = scan_ll_inplace(toff.p, n, s);
    DBuf<int> gk((size_t)tot, s);
    DBuf<VT> gv((size_t)tot, s);
    k_sg_sym<SG_SYM_T><<<grid_for((int64_t)n * 32, SG_WARPS * 32, num_sms() * 8), SG_WARPS * 32,
                         sizeof(int) * SG_WARPS * SG_SYM_T, s>>>(n, nullptr, A.rp, A.ci, B.rp, B.ci, ub, C.rp.p);
    CK_LAUNCH();
    k_sg_sym_big<<<grid_for((int64_t)n * 32, 256), 256, 0, s>>>(n, rows.p, toff.p, gk.p, A.rp, A.ci, B.rp, B.ci,
                                                                 C.rp.p, 1);
    CK_LAUNCH();
    C.nnz = scan_exclusive(C.rp.p, C.rp.p, n, sc, s);
    C.ci.alloc((size_t)C.nnz, s);
    cv.alloc((size_t)C.nnz, s);
    CK(cudaMemsetAsync(sc.flags.p + 8, 0, sizeof(int), s));
    k_sg_num<SG_NUM_T, VT><<<grid_for((int64_t)n * 32, SG_WARPS * 32, num_sms() * 8), SG_WARPS * 32,
                             sg_num_smem<SG_NUM_T, VT>(), s>>>(n, nullptr, A.rp, A.ci, av, B.rp, B.ci, bv, C.rp.p,
                                                               C.ci.p, cv.p, sc.flags.p + 8);
    CK_LAUNCH();
    k_sg_num_big<VT><<<grid_for((int64_t)n * 32, 256), 256, 0, s>>>(n, rows.p, toff.p, gk.p, gv.p, A.rp, A.ci, av,
                                                                     B.rp, B.ci, bv, C.rp.p, C.ci.p, cv.p,
                                                                     sc.flags.p + 8, SG_NUM_T / 2);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(sc.h_flags + 8, sc.flags.p + 8, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (sc.h_flags[8]) throw Error(BGS_INTERNAL, "SpGEMM numeric count differs from the symbolic count");
}

// C = A B with values of type VT (av, bv: the operands' values in that type; cv receives C's)
template <class VT>
static void spgemm_t(const CsrView &A, const VT *av, const CsrView &B, const VT *bv, DCsr &C, DBuf<VT> &cv,
                     Scratch &sc, cudaStream_t s) {
    const int n = A.n;
    C.n = n;
    C.m = B.m;
    C.rp.alloc((size_t)n + 1, s);
    if (n == 0) {
        C.nnz = 0;
        CK(cudaMemsetAsync(C.rp.p, 0, sizeof(int), s));
        return;
    }
    DBuf<int> ub((size_t)n, s);
    k_sg_ub<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp, A.ci, B.rp, ub.p);
    CK_LAUNCH();
    if (n <= kSgSmallRows) {
        spgemm_small<VT>(A, av, B, bv, C, cv, ub.p, sc, s);
        return;
    }
    // symbolic: short rows per thread, the rest per warp (shared table), then global tables
    const int gl = grid_for(n, 128, num_sms() * 32);
    DBuf<int> lcols((size_t)n * SG_LOCAL, s);   // sorted columns of the short rows
    k_sg_local_sym<<<gl, 128, 0, s>>>(n, A.rp, A.ci, B.rp, B.ci, ub.p, C.rp.p, lcols.p);
    CK_LAUNCH();
    {
        // every open row first tries a small table (capped: a row with more than SG_SMALL_T / 2
        // distinct columns gives up and stays open, whatever its product count), then the rows
        // still open with large tables, then rows past the shared table
        DBuf<int> flag((size_t)n, s), rows;
        k_sym_class<<<grid_for(n, 256), 256, 0, s>>>(n, C.rp.p, ub.p, 0xffffffffu, flag.p);
        CK_LAUNCH();
        const int nbA = collect_flag(n, flag.p, rows, sc, s);
        if (nbA) {
            k_sg_sym<SG_SMALL_T><<<grid_for((int64_t)nbA * 32, SG_WARPS * 32, num_sms() * 32), SG_WARPS * 32,
                                   sizeof(int) * SG_WARPS * SG_SMALL_T, s>>>(nbA, rows.p, A.rp, A.ci, B.rp, B.ci,
                                                                             ub.p, C.rp.p);
            CK_LAUNCH();
        }
        k_sym_class<<<grid_for(n, 256), 256, 0, s>>>(n, C.rp.p, ub.p, 1024, flag.p);
        CK_LAUNCH();
        DBuf<int> rowsM;
        const int nbM = collect_flag(n, flag.p, rowsM, sc, s);
        if (nbM) {
            k_sg_sym<1024><<<grid_for((int64_t)nbM * 32, SG_WARPS * 32, num_sms() * 16), SG_WARPS * 32,
                             sizeof(int) * SG_WARPS * 1024, s>>>(nbM, rowsM.p, A.rp, A.ci, B.rp, B.ci, ub.p, C.rp.p);
            CK_LAUNCH();
        }
        DBuf<int> rows1;
        const int nb1 = collect_big(n, C.rp.p, 1 << 30, rows1, sc, s);
        if (nb1) {
            k_sg_sym<SG_SYM_T><<<grid_for((int64_t)nb1 * 32, SG_WARPS * 32, num_sms() * 8), SG_WARPS * 32,
                                 sizeof(int) * SG_WARPS * SG_SYM_T, s>>>(nb1, rows1.p, A.rp, A.ci, B.rp, B.ci, ub.p,
                                                                         C.rp.p);
            CK_LAUNCH();
            DBuf<int> rows2;
            const int nb2 = collect_big(n, C.rp.p, 1 << 30, rows2, sc, s);
            if (nb2) {
                DBuf<long long> toff;
                long long tot = big_tables(nb2, rows2.p, ub.p, toff, s);
                DBuf<int> gk((size_t)tot, s);
                k_sg_sym_big<<<grid_for((int64_t)nb2 * 32, 256), 256, 0, s>>>(nb2, rows2.p, toff.p, gk.p, A.rp, A.ci,
                                                                               B.rp, B.ci, C.rp.p, 0);
                CK_LAUNCH();
            }
        }
    }
    C.nnz = scan_exclusive(C.rp.p, C.rp.p, n, sc, s);
    C.ci.alloc((size_t)C.nnz, s);
    cv.alloc((size_t)C.nnz, s);
    // numeric
    CK(cudaMemsetAsync(sc.flags.p + 8, 0, sizeof(int), s));
    k_sg_local_num<VT><<<gl, 128, 0, s>>>(n, A.rp, A.ci, av, B.rp, B.ci, bv, ub.p, lcols.p, C.rp.p, C.ci.p, cv.p,
                                          sc.flags.p + 8);
    CK_LAUNCH();
    lcols.release();
    {
        DBuf<int> cnt((size_t)n, s), rows;
        k_row_lengths<<<grid_for(n, 256), 256, 0, s>>>(n, C.rp.p, cnt.p);
        CK_LAUNCH();
        DBuf<int> hashcnt((size_t)n, s);   // row length for rows the hash path owns, else 0
        k_hash_rows<<<grid_for(n, 256), 256, 0, s>>>(n, cnt.p, ub.p, hashcnt.p);
        CK_LAUNCH();
        DBuf<int> flag((size_t)n, s);
        // rows by table size: up to 128 slots (8 blocks of 8 warps per SM fit the shared memory),
        // up to SG_SMALL_T, up to SG_NUM_T; a row's table size follows from its own count, so the
        // class only sets the shared memory reserved per warp
        const unsigned cls[4] = {0u, 128u, (unsigned)SG_SMALL_T, (unsigned)SG_NUM_T};
        for (int c = 0; c < 3; c++) {
            k_table_class<<<grid_for(n, 256), 256, 0, s>>>(n, hashcnt.p, ub.p, cls[c], cls[c + 1], flag.p);
            CK_LAUNCH();
            DBuf<int> rl;
            const int nb = collect_flag(n, flag.p, rl, sc, s);
            if (!nb) continue;
            if (c == 0) {
                k_sg_num<128, VT><<<grid_for((int64_t)nb * 32, SG_WARPS * 32, num_sms() * 32), SG_WARPS * 32,
                                    sg_num_smem<128, VT>(), s>>>(nb, rl.p, A.rp, A.ci, av, B.rp, B.ci, bv, C.rp.p,
                                                                 C.ci.p, cv.p, sc.flags.p + 8);
            } else if (c == 1) {
                k_sg_num<SG_SMALL_T, VT><<<grid_for((int64_t)nb * 32, SG_WARPS * 32, num_sms() * 32), SG_WARPS * 32,
                                           sg_num_smem<SG_SMALL_T, VT>(), s>>>(nb, rl.p, A.rp, A.ci, av, B.rp, B.ci,
                                                                               bv, C.rp.p, C.ci.p, cv.p,
                                                                               sc.flags.p + 8);
            } else {
                k_sg_num<SG_NUM_T, VT><<<grid_for((int64_t)nb * 32, SG_WARPS * 32, num_sms() * 8), SG_WARPS * 32,
                                         sg_num_smem<SG_NUM_T, VT>(), s>>>(nb, rl.p, A.rp, A.ci, av, B.rp, B.ci, bv,
                                                                           C.rp.p, C.ci.p, cv.p, sc.flags.p + 8);
            }
            CK_LAUNCH();
        }
        {
            DBuf<int> rows2;
            const int nb2 = collect_big(n, cnt.p, SG_NUM_T / 2, rows2, sc, s);
            if (nb2) {
                DBuf<long long> toff;
                long long tot = big_tables(nb2, rows2.p, cnt.p, toff, s);
                DBuf<int> gk((size_t)tot, s);
                DBuf<VT> gv((size_t)tot, s);
                k_sg_num_big<VT><<<grid_for((int64_t)nb2 * 32, 256), 256, 0, s>>>(
                    nb2, rows2.p, toff.p, gk.p, gv.p, A.rp, A.ci, av, B.rp, B.ci, bv, C.rp.p, C.ci.p, cv.p,
                    sc.flags.p + 8, -1);
                CK_LAUNCH();
            }
        }
    }
    CK(cudaMemcpyAsync(sc.h_flags + 8, sc.flags.p + 8, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (sc.h_flags[8]) throw Error(BGS_INTERNAL, "SpGEMM numeric count differs from the symbolic count");
}

static void spgemm(const CsrView &A, const CsrView &B, DCsr &C, Scratch &sc, cudaStream_t s) {
    spgemm_t<double>(A, A.v, B, B.v, C, C.v, sc, s);
}

// ==========================================================================================
// Prolongator: P_tent (iota, agg, 1) and the damped smoothing transform
// ==========================================================================================
__global__ void k_ptent(int n, const int *agg, int *rp, int *ci, double *v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) {
        rp[i] = i;
        if (i < n) {
            ci[i] = agg[i];
            v[i] = 1.0;
        }
    }
}
// p_iJ = [J == agg(i)] - (omega * dinvF_i) * s_iJ
__global__ void k_psmooth(int n, const int *rp, const int *ci, double *v, const int *agg, const double *dinvF,
                          double omega) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double c = omega * dinvF[i];
        const int a = agg[i];
        for (int e = rp[i]; e < rp[i + 1]; e++) {
            const double t = ci[e] == a ? 1.0 : 0.0;
            v[e] = t - __dmul_rn(c, v[e]);
        }
    }
}

// ==========================================================================================
// Coarsest level: explicit inverse by Gauss-Jordan elimination with partial (row) pivoting
// ==========================================================================================
// In-place Gauss-Jordan on the row-major n x n matrix: step k takes the pivot row p (largest
// |a_ik| for i >= k, ties to the smaller row), moves it to row k, scales it by 1/a_pk and
// eliminates column k from every other row, leaving column k of the running inverse in column k.
// After the last step the columns are unscrambled by undoing the row interchanges in reverse.
// GB300 issues about two FP64 FMAs per clock per SM, so every step spreads its n^2 updates over
// the whole GPU: one launch per step, reading the state before the step (S) and writing the state
// after it (D), so no block ever waits on another.  Each launch also leaves one (|value|, row)
// pivot candidate per block for the next column; every block of the next launch reduces them in
// the same fixed order and so all agree on the pivot.
constexpr int GJ_T = 256;

__global__ void k_to_dense_rm(int n, const int *rp, const int *ci, const double *v, double *a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int e = rp[i]; e < rp[i + 1]; e++) a[(size_t)i * n + ci[e]] = v[e];
}

__device__ __forceinline__ bool gj_better(double v, int i, double bv, int bi) {
    return v > bv || (v == bv && i < bi);
}

// block-wide (|value|, row) maximum, written by thread 0 to cv[blockIdx.x], ci[blockIdx.x]
__device__ void gj_block_best(double best, int bi, double *cv, int *cidx) {
    __shared__ double sv[GJ_T / 32];
    __shared__ int si[GJ_T / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (gj_better(ov, oi, best, bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { sv[w] = best; si[w] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < GJ_T / 32; q++)
            if (gj_better(sv[q], si[q], best, bi)) { best = sv[q]; bi = si[q]; }
        cv[blockIdx.x] = best;
        cidx[blockIdx.x] = bi;
    }
}

__global__ void __launch_bounds__(GJ_T) k_gj_first(int n, const double *a, double *cv, int *cidx) {
    double best = -1.0;
    int bi = INT_MAX;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double t = fabs(a[(size_t)i * n]);
        if (gj_better(t, i, best, bi)) { best = t; bi = i; }
    }
    gj_block_best(best, bi, cv, cidx);
}

__global__ void __launch_bounds__(GJ_T) k_gj_step(int n, int k, const double *__restrict__ S, double *__restrict__ D,
                                                  const double *cv_in, const int *ci_in, int g_in, double *cv_out,
                                                  int *ci_out, int *perm, int *status) {
    __shared__ int sp;
    __shared__ double srp;
    if (threadIdx.x < 32) {
        double best = -1.0;
        int bi = INT_MAX;
        for (int b = threadIdx.x; b < g_in; b += 32)
            if (gj_better(cv_in[b], ci_in[b], best, bi)) { best = cv_in[b]; bi = ci_in[b]; }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (gj_better(ov, oi, best, bi)) { best = ov; bi = oi; }
        }
        if (threadIdx.x == 0) {
            if (!(best > 0.0) || bi >= n) {   // singular: continue on row k with a unit pivot
                bi = k;
                srp = 1.0;
                if (blockIdx.x == 0) *status = 1;
            } else {
                srp = 1.0 / S[(size_t)bi * n + k];
            }
            sp = bi;
            if (blockIdx.x == 0) perm[k] = bi;
        }
    }
    __syncthreads();
    const int p = sp;
    const double rpiv = srp;
    const int kn = k + 1;
    double best = -1.0;
    int bi = INT_MAX;
    const unsigned un = (unsigned)n;
    const unsigned total = un * un;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int i = (int)(t / un), j = (int)(t - (unsigned)i * un);
        const double pk = S[(size_t)p * n + j] * rpiv;   // entry j of the scaled pivot row
        double out;
        if (i == k) {
            out = (j == k) ? rpiv : pk;
        } else {
            const size_t src = (size_t)(i == p ? k : i) * n;
            const double f = S[src + k];
            out = (j == k) ? -f * rpiv : S[src + j] - f * pk;
        }
        D[t] = out;
        if (j == kn && i >= kn && gj_better(fabs(out), i, best, bi)) { best = fabs(out); bi = i; }
    }
    gj_block_best(best, bi, cv_out, ci_out);
}

// tau = the column order that undoes the row interchanges (applied in reverse order)
__global__ void k_gj_tau(int n, const int *perm, int *tau) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int c = 0; c < n; c++) tau[c] = c;
    for (int k = n - 1; k >= 0; k--) {
        const int p = perm[k];
        const int t = tau[k];
        tau[k] = tau[p];
        tau[p] = t;
    }
}

__global__ void k_gj_unscramble(int n, const double *D, const int *tau, double *W) {
    const unsigned un = (unsigned)n, total = un * un;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const unsigned i = t / un, c = t - i * un;
        W[t] = D[(size_t)i * n + tau[c]];
    }
}

// Blocked form: GJB_R pivot steps per pair of launches.  The panel kernel (one block) takes the
// columns K = [k, k+R) of the state before the steps, chooses the R pivots by partial pivoting on an
// LU-eliminated FP32 working copy (in R sequential Gauss-Jordan steps the rows at and below each
// pivot hold the values LU gives them; FP32 rounding can only swap the choice between two entries of
// nearly the same size, which leaves the pivoting as stable) and computes D = A_KK^-1 of the
// interchanged pivot rows (Gauss-Jordan on R x R, one thread per entry, pivots on the diagonal).
// The update kernel (one block per row) writes the state after the R steps: columns K: D (pivot
// rows) and F = -A_IK D (other rows); other columns: D A_KJ (pivot rows) and A_IJ + F A_KJ (other
// rows), A_KJ the interchanged pivot rows.  In exact arithmetic this is the state R sequential steps
// leave.  GB300's FP64 tensor path (mma.sync f64) runs at the FP64 FMA rate, so these small
// products stay on the FP64 pipe.
constexpr int GJB_R = 16;
constexpr int GJB_T = 256;       // = GJB_R * GJB_R: one thread per entry of the pivot block
constexpr int GJB_MAXN = 2560;   // the panel's working copy (n x R floats) in shared memory

// position q after the block's row interchanges (pk[t]: the row exchanged with row k + t) holds row
// src(q) of the state before them
__device__ __forceinline__ int gjb_src(int q, int k, int R, const int *pk) {
    for (int t = R - 1; t >= 0; t--) {
        const int p = pk[t];
        if (q == k + t) q = p;
        else if (q == p) q = k + t;
    }
    return q;
}

__global__ void __launch_bounds__(GJB_T) k_gjb_panel(int n, int k, int R, const double *__restrict__ S, int *perm,
                                                      double *Dk, int *status) {
    extern __shared__ float gjb_sm[];
    // n x R, row-major [i * R + t]: the panel, rows interchanged, eliminated below the pivots.  It
    // only chooses the pivots, so it is kept in FP32 (one SM's FP64 rate made the FP64 copy the
    // slowest part of the inverse); every value the inverse is made of comes from the FP64 state
    float *Cw = gjb_sm;
    __shared__ double bv_s[GJB_T / 32];
    __shared__ int bi_s[GJB_T / 32];
    __shared__ int piv_s[GJB_R];
    __shared__ double M[GJB_R * GJB_R];
    __shared__ double prow[GJB_R], pcol[GJB_R];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int t = 0; t < R; t++) Cw[i * R + t] = (float)S[(size_t)i * n + k + t];
    __syncthreads();
    for (int t = 0; t < R; t++) {
        const int c = k + t;
        double best = -1.0;
        int bi = INT_MAX;
        for (int i = c + threadIdx.x; i < n; i += blockDim.x) {
            const double a = fabsf(Cw[i * R + t]);
            if (gj_better(a, i, best, bi)) { best = a; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (gj_better(ov, oi, best, bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { bv_s[w] = best; bi_s[w] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = 1; q < GJB_T / 32; q++)
                if (gj_better(bv_s[q], bi_s[q], best, bi)) { best = bv_s[q]; bi = bi_s[q]; }
            if (!(best > 0.0) || bi >= n) {   // singular: keep row c, report (the results are not used)
                bi = c;
                *status = 1;
            }
            piv_s[t] = bi;
            perm[c] = bi;
        }
        __syncthreads();
        const int p = piv_s[t];
        if (p != c && threadIdx.x < R) {
            const float a = Cw[c * R + threadIdx.x];
            Cw[c * R + threadIdx.x] = Cw[p * R + threadIdx.x];
            Cw[p * R + threadIdx.x] = a;
        }
        __syncthreads();
        if (t + 1 < R) {   // each thread eliminates its own rows below the pivot
            const float rpv = 1.0f / Cw[c * R + t];
            for (int i = c + 1 + threadIdx.x; i < n; i += blockDim.x) {
                const float l = Cw[i * R + t] * rpv;
                for (int u = t + 1; u < R; u++) Cw[i * R + u] -= l * Cw[c * R + u];
            }
        }
        __syncthreads();
    }
    // A_KK: the interchanged pivot rows of the state before the steps; D = A_KK^-1 in place
    const int r = threadIdx.x / GJB_R, q = threadIdx.x % GJB_R;
    if (r < R && q < R) {
        M[r * GJB_R + q] = S[(size_t)gjb_src(k + r, k, R, piv_s) * n + k + q];
    }
    __syncthreads();
    for (int t = 0; t < R; t++) {
        // stage row t and column t: every thread then reads only staged values and its own entry
        if (threadIdx.x < R) prow[threadIdx.x] = M[t * GJB_R + threadIdx.x];
        else if (threadIdx.x < 2 * R) pcol[threadIdx.x - R] = M[(threadIdx.x - R) * GJB_R + t];
        __syncthreads();
        if (threadIdx.x == 0 && prow[t] == 0.0) *status = 1;   // an exactly singular pivot block
        const double rp = 1.0 / prow[t];
        if (r < R && q < R) {
            const double f = pcol[r];
            double v;
            if (r == t) v = q == t ? rp : prow[q] * rp;
            else v = q == t ? -f * rp : M[r * GJB_R + q] - f * (prow[q] * rp);
            M[r * GJB_R + q] = v;
        }
        __syncthreads();
    }
    if (r < R && q < R) Dk[r * R + q] = M[r * GJB_R + q];
}

__global__ void __launch_bounds__(GJB_T) k_gjb_update(int n, int k, int R, const double *__restrict__ S,
                                                       double *__restrict__ Dout, const int *perm,
                                                       const double *__restrict__ Dk) {
    __shared__ int pk[GJB_R], srck[GJB_R];
    __shared__ double Ds[GJB_R * GJB_R];
    __shared__ double Fr[GJB_R], rowK[GJB_R];
    if (threadIdx.x < R) pk[threadIdx.x] = perm[k + threadIdx.x];
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) Ds[e] = Dk[e];
    __syncthreads();
    if (threadIdx.x < R) srck[threadIdx.x] = gjb_src(k + threadIdx.x, k, R, pk);
    __syncthreads();
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const bool piv_row = i >= k && i < k + R;
        const int si = gjb_src(i, k, R, pk);   // every thread, from shared memory
        if (threadIdx.x < R) rowK[threadIdx.x] = S[(size_t)si * n + k + threadIdx.x];
        __syncthreads();
        // this row's factors F = -A_iK D (other rows) or the row of D (pivot rows)
        if (threadIdx.x < R) {
            double f;
            if (piv_row) {
                f = Ds[(i - k) * R + threadIdx.x];
            } else {
                f = 0.0;
                for (int q = 0; q < R; q++) f -= rowK[q] * Ds[q * R + threadIdx.x];
            }
            Fr[threadIdx.x] = f;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            double out;
            if (j >= k && j < k + R) {
                out = Fr[j - k];
            } else {
                out = piv_row ? 0.0 : S[(size_t)si * n + j];
                for (int q = 0; q < R; q++) out += Fr[q] * S[(size_t)srck[q] * n + j];
            }
            Dout[(size_t)i * n + j] = out;
        }
        __syncthreads();
    }
}

// Radius of the skew-symmetric part S = (M - M^T)/2 of M = D^-1/2 A D^-1/2 (D = diag(A), all
// positive, else 0): a Bendixson bound on |Im| of the eigenvalues of D^-1 A.  Power iteration on
// S^T S = -S S from the hashed start, CSR kernels fixed by the shape, no host round trip until the
// end (a zero vector stays zero and gives 0, as for a symmetric A).
__global__ void k_skew_scale(int n, const double *diag, double *sc, int *bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double d = diag[i];
        if (!(d > 0.0)) *bad = 1;
        sc[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    }
}
__global__ void k_vmul(int n, const double *a, const double *b, double *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = a[i] * b[i];
}
__global__ void k_skew_out(int n, const double *sc, const double *p, const double *q, double *out, double sgn) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = sgn * (0.5 * (sc[i] * p[i] - sc[i] * q[i]));
}
__global__ void k_normalise_safe(int n, const double *in, const double *nrm2, double *out) {
    const double d = sqrt(*nrm2);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = d > 0.0 ? in[i] / d : 0.0;
}

static double skew_radius(const DCsr &A, int iters, Scratch &sc, cudaStream_t s) {
    const int n = A.n;
    if (n <= 0) return 0.0;
    const int g = grid_for(n, 256);
    DBuf<double> diag((size_t)n, s), scl((size_t)n, s), v((size_t)n, s), u((size_t)n, s), t((size_t)n, s),
        p((size_t)n, s), q((size_t)n, s);
    extract_diag(view(A), diag.p, s);
    CK(cudaMemsetAsync(sc.flags.p + 12, 0, sizeof(int), s));
    k_skew_scale<<<g, 256, 0, s>>>(n, diag.p, scl.p, sc.flags.p + 12);
    CK_LAUNCH();
    DCsr AT;
    transpose_csr(view(A), AT, sc, s);
    const int la = choose_lanes(A.n, A.nnz);
    double *nr = sc.scal.p + 18;
    k_power_start<<<g, 256, 0, s>>>(n, v.p);
    CK_LAUNCH();
    dev_dot(v.p, v.p, n, nr, sc, s);
    k_normalise_safe<<<g, 256, 0, s>>>(n, v.p, nr, v.p);
    CK_LAUNCH();
    for (int it = 0; it < iters; it++) {
        for (int pass = 0; pass < 2; pass++) {
            k_vmul<<<g, 256, 0, s>>>(n, scl.p, pass == 0 ? v.p : u.p, t.p);
            CK_LAUNCH();
            spmv_f64(view(A), la, t.p, p.p, s);
            spmv_f64(view(AT), la, t.p, q.p, s);
            k_skew_out<<<g, 256, 0, s>>>(n, scl.p, p.p, q.p, pass == 0 ? u.p : t.p, pass == 0 ? 1.0 : -1.0);
            CK_LAUNCH();
        }
        dev_dot(t.p, t.p, n, nr, sc, s);
        k_normalise_safe<<<g, 256, 0, s>>>(n, t.p, nr, v.p);
        CK_LAUNCH();
    }
    CK(cudaMemcpyAsync(sc.h_scal + 2, nr, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(sc.h_flags + 12, sc.flags.p + 12, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (sc.h_flags[12]) return 0.0;
    return std::sqrt(std::sqrt(sc.h_scal[2]));
}

// Enqueues the inverse of Ac into W (allocated by the caller) on stream s without waiting; a zero
// pivot sets device flag slot 6 of sc (cleared here).
static void dense_inverse_async(const DCsr &Ac, double *W, Scratch &sc, cudaStream_t s) {
    const int n = Ac.n;
    CK(cudaMemsetAsync(sc.flags.p + 6, 0, sizeof(int), s));
    if (n == 0) return;
    DBuf<double> a((size_t)n * n, s), b((size_t)n * n, s);
    // about eight matrix entries per thread in each step: fewer blocks keep the pivot reduction
    // at the start of every step short
    const int g = grid_for((int64_t)n * n, GJ_T * 8, num_sms());
    DBuf<double> cv((size_t)2 * g, s);
    DBuf<int> cidx((size_t)2 * g, s), perm((size_t)n, s), tau((size_t)n, s);
    CK(cudaMemsetAsync(a.p, 0, sizeof(double) * (size_t)n * n, s));
    k_to_dense_rm<<<grid_for(n, 256), 256, 0, s>>>(n, Ac.rp.p, Ac.ci.p, Ac.v.p, a.p);
    CK_LAUNCH();
    double *S = a.p, *D = b.p;
    if (n <= GJB_MAXN) {
        // blocked: GJB_R pivot steps per panel launch and update launch
        DBuf<double> Dk((size_t)GJB_R * GJB_R, s);
        const size_t smem = sizeof(float) * (size_t)n * GJB_R;
        const int gu = std::min(n, num_sms() * 4);
        for (int k = 0; k < n; k += GJB_R) {
            const int R = std::min(GJB_R, n - k);
            k_gjb_panel<<<1, GJB_T, smem, s>>>(n, k, R, S, perm.p, Dk.p, sc.flags.p + 6);
            CK_LAUNCH();
            k_gjb_update<<<gu, GJB_T, 0, s>>>(n, k, R, S, D, perm.p, Dk.p);
            CK_LAUNCH();
            std::swap(S, D);
        }
    } else {
        const int g0 = std::min(g, grid_for(n, GJ_T, num_sms()));
        k_gj_first<<<g0, GJ_T, 0, s>>>(n, a.p, cv.p, cidx.p);
        CK_LAUNCH();
        int gin = g0;
        for (int k = 0; k < n; k++) {
            const int in = k & 1, out = in ^ 1;
            k_gj_step<<<g, GJ_T, 0, s>>>(n, k, S, D, cv.p + (size_t)in * g, cidx.p + (size_t)in * g, gin,
                                         cv.p + (size_t)out * g, cidx.p + (size_t)out * g, perm.p, sc.flags.p + 6);
            CK_LAUNCH();
            std::swap(S, D);
            gin = g;
        }
    }
    k_gj_tau<<<1, 1, 0, s>>>(n, perm.p, tau.p);
    CK_LAUNCH();
    k_gj_unscramble<<<g, GJ_T, 0, s>>>(n, S, tau.p, W);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(sc.h_flags + 6, sc.flags.p + 6, sizeof(int), cudaMemcpyDeviceToHost, s));
}

__global__ void k_dense_transpose(int n, const double *in, double *out) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)n * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), j = (int)(t % n);
        out[(size_t)j * n + i] = in[t];
    }
}

void Hier::build_inv_T(cudaStream_t s) {
    invT.alloc((size_t)nc * nc, s);
    if (nc > 0) {
        k_dense_transpose<<<grid_for((int64_t)nc * nc, 256), 256, 0, s>>>(nc, inv.p, invT.p);
        CK_LAUNCH();
    }
}

// ==========================================================================================
// Hierarchy construction
// ==========================================================================================
static void set_attributes() {
    static std::once_flag attrs;
    std::call_once(attrs, [] {
        CK(cudaFuncSetAttribute(k_sg_sym<SG_SYM_T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(int) * SG_WARPS * SG_SYM_T)));
        CK(cudaFuncSetAttribute(k_sg_num<SG_NUM_T, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                sg_num_smem<SG_NUM_T, double>()));
        CK(cudaFuncSetAttribute(k_sg_num<SG_NUM_T, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                sg_num_smem<SG_NUM_T, float>()));
        CK(cudaFuncSetAttribute(k_gjb_panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(float) * GJB_MAXN * GJB_R)));
    });
}

__global__ void k_same_pattern(int n, int64_t nnz, const int *rp1, const int *ci1, const int *rp2, const int *ci2,
                               int *flag) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= n || t < nnz;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t <= n && rp1[t] != rp2[t]) *flag = 1;
        if (t < nnz && ci1[t] != ci2[t]) *flag = 1;
    }
}

void take_values(DCsr &dst, const DCsr &src, Scratch &sc, cudaStream_t s) {
    if (dst.n != src.n || dst.m != src.m || dst.nnz != src.nnz)
        throw Error(BGS_INTERNAL, "numeric re-set-up produced a different operator shape");
    k_same_pattern<<<grid_for(std::max<int64_t>(dst.nnz, dst.n + 1), 256), 256, 0, s>>>(
        dst.n, dst.nnz, dst.rp.p, dst.ci.p, src.rp.p, src.ci.p, sc.flags.p + 10);
    CK_LAUNCH();
    if (dst.nnz)
        CK(cudaMemcpyAsync(dst.v.p, src.v.p, sizeof(double) * (size_t)dst.nnz, cudaMemcpyDeviceToDevice, s));
    refresh_values(dst, s);
}

// Numeric part of coarsening step l, given the level's strength flags and aggregates: the
// filtered matrix A_F and D_F, omega from the power iteration, P = P_tent - omega D_F^-1 A_F P_tent,
// R = P^T and A_{l+1} = R (A_l P).  With `update` the results replace the values of the stored
// P_l, R_l and A_{l+1}, whose patterns come out the same because flags and aggregates are kept.
static void level_numeric(Hier &H, int l, const AmgParams &p, Scratch &sc, cudaStream_t s, Trace &tr,
                          bool update) {
    Level &Lv = H.L[l];
    DCsr &A = Lv.A;
    const int n = A.n;
    const int nagg = Lv.nagg;
    DCsr AF;
    AF.n = AF.m = n;
    AF.rp.alloc((size_t)n + 1, s);
    k_filter_count<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp.p, A.ci.p, Lv.strong.p, AF.rp.p);
    CK_LAUNCH();
    AF.nnz = scan_exclusive(AF.rp.p, AF.rp.p, n, sc, s);
    AF.ci.alloc((size_t)AF.nnz, s);
    AF.v.alloc((size_t)AF.nnz, s);
    DBuf<double> dinvF((size_t)n, s);
    k_filter_fill<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp.p, A.ci.p, A.v.p, Lv.strong.p, AF.rp.p, AF.ci.p, AF.v.p,
                                                   dinvF.p, p.filter_diag);
    CK_LAUNCH();
    tr.mark("filter", l, AF.nnz);
    // nothing filtered out (A_F has every entry of A_l, so the same values): the iteration runs on
    // A_l and its layouts
    const double lamF = power_lambda(AF.nnz == A.nnz ? A : AF, dinvF.p, p.power_iters, sc, s);
    const double omega = (4.0 / 3.0) / lamF;
    tr.mark("power(omega)", l, n);
    DCsr Pt;
    Pt.n = n;
    Pt.m = nagg;
    Pt.nnz = n;
    Pt.rp.alloc((size_t)n + 1, s);
    Pt.ci.alloc((size_t)n, s);
    Pt.v.alloc((size_t)n, s);
    k_ptent<<<grid_for(n + 1, 256), 256, 0, s>>>(n, Lv.agg.p, Pt.rp.p, Pt.ci.p, Pt.v.p);
    CK_LAUNCH();
    DCsr P, R, AP, Ac;
    spgemm(view(AF), view(Pt), P, sc, s);
    k_psmooth<<<grid_for(n, 256), 256, 0, s>>>(n, P.rp.p, P.ci.p, P.v.p, Lv.agg.p, dinvF.p, omega);
    CK_LAUNCH();
    tr.mark("prolongator", l, P.nnz);
    transpose_csr(view(P), R, sc, s);
    tr.mark("transpose", l, R.nnz);
    if (p.fp32_galerkin) {
        // the FP32 hierarchy's operator: A P and R (A P) in FP32 arithmetic from FP32 copies of A_l
        // (kept from the previous level's product, or converted on the finest level), P_l and R_l
        // (the copies the FP32 solve uses); A_l+1 keeps the FP32 product and its FP64 widening
        if (A.vf.n != (size_t)A.nnz) {
            A.vf.alloc((size_t)A.nnz, s);
            convert_d2f(A.v.p, A.vf.p, A.nnz, s);
        }
        P.vf.alloc((size_t)P.nnz, s);
        convert_d2f(P.v.p, P.vf.p, P.nnz, s);
        R.vf.alloc((size_t)R.nnz, s);
        convert_d2f(R.v.p, R.vf.p, R.nnz, s);
        spgemm_t<float>(view(A), A.vf.p, view(P), P.vf.p, AP, AP.vf, sc, s);
        tr.mark("spgemm AP", l, AP.nnz);
        spgemm_t<float>(view(R), R.vf.p, view(AP), AP.vf.p, Ac, Ac.vf, sc, s);
        Ac.v.alloc((size_t)Ac.nnz, s);
        copy_f2d(Ac.vf.p, Ac.v.p, Ac.nnz, s);
        tr.mark("spgemm R(AP)", l, Ac.nnz);
    } else {
        spgemm(view(A), view(P), AP, sc, s);
        tr.mark("spgemm AP", l, AP.nnz);
        spgemm(view(R), view(AP), Ac, sc, s);
        tr.mark("spgemm R(AP)", l, Ac.nnz);
    }
    Lv.omega = omega;
    if (update) {
        take_values(Lv.P, P, sc, s);
        take_values(Lv.R, R, sc, s);
        take_values(H.L[l + 1].A, Ac, sc, s);
    } else {
        Lv.P = std::move(P);
        Lv.R = std::move(R);
        H.L[l + 1].A = std::move(Ac);
    }
}

// Chebyshev power iterations started early: level l's estimate is enqueued on the scratch's side
// stream as soon as A_l is final (and known not to be the coarsest), so it overlaps the coarsening
// of the levels below it; the results are read back once, at the end of the build.  The same
// kernels in the same order as power_lambda, so the same estimates.
struct EarlyCheb {
    std::vector<int> levels;   // levels whose estimate is enqueued
    DBuf<double> partial;      // dot partials of the side stream
    DBuf<double> out;          // 4 doubles per level (power_enqueue's out)
};

static void cheb_power_early(Hier &H, int l, const AmgParams &p, Scratch &sc, cudaStream_t s, EarlyCheb &ec) {
    Level &Lv = H.L[l];
    const int n = Lv.A.n;
    cudaStream_t side = sc.side;
    CK(cudaEventRecord(sc.fork, s));
    CK(cudaStreamWaitEvent(side, sc.fork, 0));
    DBuf<double> diag((size_t)n, side);
    extract_diag(view(Lv.A), diag.p, side);
    Lv.dinv.alloc((size_t)n, side);
    reciprocal(diag.p, Lv.dinv.p, n, side);
    power_enqueue(Lv.A, Lv.dinv.p, p.power_iters, ec.partial.p, ec.out.p + 4 * l, side);
    ec.levels.push_back(l);
}

static void set_cheb_bounds(Level &Lv, double lam, const AmgParams &p, Scratch &sc, cudaStream_t s) {
    Lv.lmax = p.cheb_boost * lam;
    Lv.lmin = Lv.lmax / p.cheb_ratio;
    Lv.lim = p.cheb_ellipse ? p.cheb_boost * skew_radius(Lv.A, p.power_iters, sc, s) : 0.0;
    // below 1e-10 of lmax the skew part is rounding noise (e.g. a Galerkin product of a symmetric
    // operator summed in two orders): keep the real interval
    if (Lv.lim <= 1e-10 * Lv.lmax) Lv.lim = 0.0;
}

// Chebyshev bounds on every level above the coarsest and the coarsest dense inverse; the inverse
// runs on the scratch's side stream (after the early estimates queued there, if any) while the
// remaining power iterations run on s.
static void smoothers_and_inverse(Hier &H, const AmgParams &p, Scratch &sc, cudaStream_t s, Trace &tr,
                                  EarlyCheb *ec) {
    H.nc = H.L.back().A.n;
    if (H.nc > 16384) throw Error(BGS_INTERNAL, "coarsest level too large for the dense direct solve");
    H.inv.alloc((size_t)H.nc * H.nc, s);
    sc.ensure_side();
    CK(cudaEventRecord(sc.fork, s));
    CK(cudaStreamWaitEvent(sc.side, sc.fork, 0));
    dense_inverse_async(H.L.back().A, H.inv.p, sc, sc.side);
    std::vector<char> early(H.L.size(), 0);
    if (ec)
        for (int l : ec->levels) early[(size_t)l] = 1;
    for (size_t k = 0; k + 1 < H.L.size(); k++) {
        if (early[k]) continue;
        Level &Lv = H.L[k];
        const int n = Lv.A.n;
        DBuf<double> diag((size_t)n, s);
        extract_diag(view(Lv.A), diag.p, s);
        if (Lv.dinv.n != (size_t)n) Lv.dinv.alloc((size_t)n, s);
        reciprocal(diag.p, Lv.dinv.p, n, s);
        set_cheb_bounds(Lv, power_lambda(Lv.A, Lv.dinv.p, p.power_iters, sc, s), p, sc, s);
        tr.mark("power(cheb)", (int)k, n);
    }
    CK(cudaStreamSynchronize(sc.side));
    if (ec && !ec->levels.empty()) {
        std::vector<double> h(ec->out.n);
        CK(cudaMemcpy(h.data(), ec->out.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
        for (int l : ec->levels) {
            if (l + 1 >= (int)H.L.size()) continue;   // cannot happen: enqueued levels are not the coarsest
            set_cheb_bounds(H.L[(size_t)l], power_estimate(h[4 * (size_t)l], h[4 * (size_t)l + 2]), p, sc, s);
            tr.mark("power(cheb)", l, H.L[(size_t)l].A.n);
        }
    }
    // the inverse is used on s from here on
    CK(cudaEventRecord(sc.fork, sc.side));
    CK(cudaStreamWaitEvent(s, sc.fork, 0));
    H.status = sc.h_flags[6] ? BGS_ZERO_PIVOT : BGS_OK;
    tr.mark("dense LU+inverse", (int)H.L.size() - 1, H.nc);
}

void amg_build(Hier &H, const AmgParams &p, Scratch &sc, cudaStream_t s) {
    set_attributes();
    H.degree = p.degree;
    H.L.reserve(kMaxLevels + 1);
    const double t2 = p.theta * p.theta;
    Trace tr(s);
    // the finest operator's diagonal-offset layout (the solve's likely choice) serves the
    // set-up's power iterations on it already (spmv_scaled_norm)
    build_dia(H.L[0].A, kMaxPadDia, sc, s);
    sc.ensure_side();
    EarlyCheb ec;
    ec.partial.alloc((size_t)num_sms() * 4, s);
    ec.out.alloc(4 * (size_t)(kMaxLevels + 1), s);
    // on every exit (an exception included), the side stream's work ends before ec's buffers go
    struct SideJoin {
        cudaStream_t st;
        ~SideJoin() { cudaStreamSynchronize(st); }
    } join{sc.side};
    for (int l = 0;; l++) {
        const int n = H.L[l].A.n;
        if (n <= p.max_coarse || l + 1 >= std::min(p.max_levels, kMaxLevels)) break;
        DCsr &A = H.L[l].A;
        DBuf<double> diag((size_t)n, s);
        extract_diag(view(A), diag.p, s);
        DBuf<uint8_t> strong((size_t)std::max<int64_t>(A.nnz, 1), s);
        DCsr S;
        DBuf<int> agg((size_t)n, s);
        int nagg = -1, rounds = 0;
        // coarsening that stalls above max_coarse is retried once without dropping (theta = 0)
        for (int attempt = 0; attempt < 2; attempt++) {
            const double th2 = attempt == 0 ? t2 : 0.0;
            if (attempt == 1 && (t2 == 0.0 || (long long)nagg * 10 <= (long long)n * 9)) break;
            CK(cudaMemsetAsync(sc.flags.p + 7, 0, sizeof(int), s));
            k_strength<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp.p, A.ci.p, A.v.p, diag.p, th2, strong.p,
                                                         sc.flags.p + 7);
            CK_LAUNCH();
            CK(cudaMemcpyAsync(sc.h_flags + 7, sc.flags.p + 7, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            const int sflags = sc.h_flags[7];
            if (sflags & 2) throw Error(BGS_ZERO_PIVOT, "zero diagonal entry in a level operator");
            S = DCsr();
            strength_graph(view(A), strong.p, (sflags & 1) != 0, S, sc, s);
            tr.mark("strength", l, n);
            DBuf<int> state((size_t)n, s);
            const uint32_t salt = (uint32_t)l * 0x9E3779B9u;
            rounds = mis2(S, salt, state.p, sc, s);
            tr.mark("mis2", l, rounds);
            nagg = aggregate(S, state.p, agg.p, sc, s);
            tr.mark("aggregate", l, nagg);
            if (nagg < 0) throw Error(BGS_INTERNAL, "aggregation left a node unassigned");
        }
        if ((long long)nagg * 10 > (long long)n * 9) break;   // coarsening stalled
        H.L.emplace_back();
        cheb_power_early(H, l, p, sc, s, ec);   // level l is not the coarsest: its smoother's estimate
        Level &Lv = H.L[l];
        Lv.strong = std::move(strong);   // kept for the numeric re-set-up
        Lv.agg = std::move(agg);
        Lv.nagg = nagg;
        Lv.mis_rounds = rounds;
        level_numeric(H, l, p, sc, s, tr, false);
    }
    smoothers_and_inverse(H, p, sc, s, tr, &ec);
}

void amg_update(Hier &H, const AmgParams &p, Scratch &sc, cudaStream_t s) {
    set_attributes();
    Trace tr(s);
    CK(cudaMemsetAsync(sc.flags.p + 10, 0, sizeof(int), s));
    for (int l = 0; l + 1 < (int)H.L.size(); l++) level_numeric(H, l, p, sc, s, tr, true);
    smoothers_and_inverse(H, p, sc, s, tr, nullptr);
    CK(cudaMemcpyAsync(sc.h_flags + 10, sc.flags.p + 10, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (sc.h_flags[10]) throw Error(BGS_INTERNAL, "numeric re-set-up produced a different operator pattern");
}

}  // namespace bgs
