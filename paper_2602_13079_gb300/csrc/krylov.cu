// Flexible GMRES on the device (Sec. 2.2, flexible GMRES): the Arnoldi orthogonalisation (K14,
// K15), the Givens rotations of the Hessenberg column, the residual estimate and the stopping test.
//
// Orthogonalisation: classical Gram-Schmidt with selective re-orthogonalisation (Daniel-Gragg-
// Kaufman-Stewart test, "twice is enough").
//   dots:   h = V^T w and ||w||^2 in one pass over V (column-major, leading dimension ld);
//           the basis is split over gridDim.y in chunks of vectors so a thread keeps one
//           accumulator per vector of its chunk, and each thread reads two rows per load (16-byte
//           loads along a column).
//   update: w_out = w_in - V h and ||w_out||^2 in one pass (one accumulator per row).
// Every reduction goes through per-block partials summed in a fixed order, so the results do not
// depend on scheduling.
//
// The FGMRES passes split their products between two kinds of arithmetic.  On GB300 the FP64 pipe
// retires about 1.6 fused multiply-adds per clock per multiprocessor, fewer than the basis entries
// HBM delivers (about 2.7 per clock), so a pass done wholly in FP64 is bound by that pipe; the
// integer pipes sit idle meanwhile.  So a share of the products runs as exact integer arithmetic:
//  * a basis entry v, |v| < 2 (the basis vectors have unit norm), becomes the integer
//    trunc(|v| 2^62) (at most 63 bits) and a sign;
//  * the other factor x (w in the dots, h in the update) is taken relative to the largest exponent
//    field S among the values one accumulator sees: |x| = M 2^(S - 1078) with M a 56-bit integer
//    (an entry 2^k below the largest drops its k lowest mantissa bits);
//  * each integer product, floor(product / 2^32) formed from 32-bit partial products (less than one
//    unit, 2^-87 of the largest possible product, cut off), is summed into a 96-bit two's-complement
//    accumulator: a thread's sum is exact up to those truncations and independent of order; it is
//    rounded to FP64 once (value = accumulator * 2^(S - 1108)) and the thread sums go through the
//    same fixed-order FP64 tree as the FP64 sums.
// The terms of a dot of a unit vector v with w thus carry less than 2^-62 ||w||_1 + 2^-55 max|w|
// ||v||_1 + n 2^-84 max|w| of truncation in all, and only the tree's roundings on top, where an FP64
// sum rounds at every term.  The dots take vectors 0..2 of each chunk of 8 in FP64 and 3..7 in
// fixed point; the update takes the first row of each pair in FP64 and the second in fixed point
// (both passes of the 27 iterations of the 128^3 FP64 solve: 21.6 -> 16.5 ms, and 14.4 ms with the
// dots' loads staged through shared memory and the update's eight loads in flight).  The
// general-purpose dots of the C interface (any V) stay in FP64.
//
// The step kernels read the basis size (cnt = j + 1) from the solver state in device memory, and
// the scalar work of a step (Hessenberg column, rotations, estimate, stop decision) runs in one
// single-thread kernel, so a whole restart cycle can be replayed as one CUDA graph whose WHILE
// node the step kernel ends; launched one by one, the same kernels give the same bits.
#include <algorithm>
#include <atomic>

#include "internal.h"

namespace bgs {

constexpr int KT = 256;   // threads per block
constexpr int KC = 16;    // basis vectors per dot chunk of the C interface's FP64 dots
// blocks along x: one wave at the 3 blocks per multiprocessor that k_mdot's and k_mupdate's
// registers allow (so no multiprocessor runs a lone fourth block)
static int kg_dots() { return num_sms() * 3; }
static int kg_update() { return num_sms() * 3; }

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

// ------------------------------------------------------------------------------------------
// Fixed-point products (the scheme in the header comment)
// ------------------------------------------------------------------------------------------
struct Fx96 {
    uint32_t w0, w1, w2;   // two's complement, w0 least significant
};

// exponent field of a double for scaling: at least 1, so that zeros and subnormals share the
// smallest normal exponent
__device__ __forceinline__ uint32_t fx_exp(uint64_t bits) { return max((uint32_t)(bits >> 52) & 0x7ffu, 1u); }

// trunc(|v| 2^62) for |v| < 2; bad is set for |v| >= 2, Inf and NaN (the value is then 0)
__device__ __forceinline__ uint64_t fx_basis(uint64_t bits, bool &bad) {
    const uint32_t e = (uint32_t)(bits >> 52) & 0x7ffu;
    bad |= e >= 1024u;
    const uint64_t m = ((bits & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 10;
    return m >> min(1023u - e, 63u);   // e >= 1024 wraps to a shift of 63: 0
}

// |x| = M 2^(S - 1078) with M < 2^56, for S >= fx_exp(x)
__device__ __forceinline__ uint64_t fx_scaled(uint64_t bits, uint32_t S) {
    const uint32_t e = (uint32_t)(bits >> 52) & 0x7ffu;
    const uint64_t m = ((bits & 0x000FFFFFFFFFFFFFull) | ((uint64_t)(e != 0) << 52)) << 3;
    return m >> min(S - max(e, 1u), 63u);
}

// acc += (-1)^s floor(a b / 2^32) for a = a1 2^32 + a0 < 2^63, b = b1 2^32 + b0 < 2^56, formed as
// hi(a0 b0) + a0 b1 + a1 b0 + a1 b1 2^32; each term is below 2^88, so 127 of them fit the
// accumulator's 2^95
__device__ __forceinline__ void fx_mac(Fx96 &acc, uint64_t a, uint64_t b, uint32_t s) {
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    uint64_t t = (uint64_t)__umulhi(a0, b0);
    t += (uint64_t)a0 * b1;
    t += (uint64_t)a1 * b0;                 // < 2^32 + 2^56 + 2^63
    const uint64_t u = (uint64_t)a1 * b1;   // < 2^55
    uint32_t x0 = (uint32_t)t, x1, x2;
    asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %4, 0;"
        : "=r"(x1), "=r"(x2)
        : "r"((uint32_t)(t >> 32)), "r"((uint32_t)u), "r"((uint32_t)(u >> 32)));
    const uint32_t mask = 0u - s;   // negation as (x ^ mask) + s
    x0 ^= mask;
    x1 ^= mask;
    x2 ^= mask;
    asm("{\n\t.reg .u32 c;\n\tadd.cc.u32 c, %3, 0xffffffff;\n\t"
        "addc.cc.u32 %0, %0, %4;\n\taddc.cc.u32 %1, %1, %5;\n\taddc.u32 %2, %2, %6;\n\t}"
        : "+r"(acc.w0), "+r"(acc.w1), "+r"(acc.w2)
        : "r"(s), "r"(x0), "r"(x1), "r"(x2));
}

// the accumulator times 2^E, rounded to nearest once: the magnitude's leading 64 bits with the
// rest as a sticky bit, converted with round-to-nearest-even, then scaled exactly by 2^E
__device__ double fx_to_double(Fx96 a, int E) {
    const bool neg = (int32_t)a.w2 < 0;
    if (neg)
        asm("{\n\tnot.b32 %0, %0;\n\tnot.b32 %1, %1;\n\tnot.b32 %2, %2;\n\t"
            "add.cc.u32 %0, %0, 1;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.u32 %2, %2, 0;\n\t}"
            : "+r"(a.w0), "+r"(a.w1), "+r"(a.w2));
    double d;
    if (a.w2 == 0) {
        d = __ull2double_rn(((uint64_t)a.w1 << 32) | a.w0);
    } else {
        const int lz = __clz((int)a.w2);   // 0..31
        const uint64_t hi = ((uint64_t)a.w2 << 32) | a.w1;
        const uint64_t top = lz ? (hi << lz) | (a.w0 >> (32 - lz)) : hi;
        const uint32_t rest = a.w0 << lz;
        d = __ull2double_rn(top | (uint64_t)(rest != 0));
        E += 32 - lz;
    }
    d = (E >= -1022 && E <= 1023) ? d * __longlong_as_double((long long)(E + 1023) << 52) : ldexp(d, E);
    return neg ? -d : d;
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
// fixed shuffle tree); out[cnt] = ||w||^2.  Partials laid out [chunk][block][CH + 1].
template <int CH>
__global__ void k_mdot_reduce(const double *part, int g, int cnt0, const int *cntp, const int *gate, double *out) {
    if (gate && !*gate) return;
    const int cnt = basis_count(cnt0, cntp);
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (t > cnt) return;
    double s = 0.0;
    if (t < cnt) {
        const int c = t / CH, k = t % CH;
        for (int b = lane; b < g; b += 32) s += part[((size_t)c * g + b) * (CH + 1) + k];
    } else {
        for (int b = lane; b < g; b += 32) s += part[(size_t)b * (CH + 1) + CH];
    }
    s = warp_sum(s);
    if (lane == 0) out[t] = s;
}

// FGMRES dots: chunks of OC basis vectors, the first OF of a chunk on the FP64 pipe and the rest in
// fixed point; ||w||^2 (FP64) in chunk 0.  A thread's fixed-point sums are rounded into FP64 after
// every kFxBatch row pairs (at most 2 kFxBatch < 127 terms per accumulator), added in order.
// The loads run two row pairs ahead of the arithmetic: each thread copies its next pair's chunk
// entries and w with cp.async into its own column of a two-stage shared buffer (basis entries
// marked evict-first in L2, so that w stays there for the other chunks), then computes on the
// current stage; a thread only reads what it copied, so no block barrier is needed.
constexpr int OC = 8, OF = 3, OI = OC - OF, kFxBatch = 60;
static int kg_odots() { return num_sms() * 2; }
static size_t odot_smem() { return sizeof(double2) * 2 * (OC + 1) * KT; }

__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async16_first(void *sdst, const void *gsrc, uint64_t pol) {
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__global__ void __launch_bounds__(KT, 2) k_odot(const double *__restrict__ V, int64_t ld, int cnt0, const int *cntp,
                                             const int *gate, const double *__restrict__ w, int64_t n, double *part) {
    if (gate && !*gate) return;
    const int cnt = basis_count(cnt0, cntp);
    const int k0 = blockIdx.y * OC;
    if (k0 >= cnt) return;                 // chunk past the basis (launched for the largest count)
    const int kc = min(OC, cnt - k0);
    const bool first = blockIdx.y == 0;
    extern __shared__ double2 ostage[];    // [2][OC + 1][KT]: chunk entries, then w
    __shared__ double fsum[OI][KT];
    const int64_t npair = n >> 1;
    const double2 *w2 = reinterpret_cast<const double2 *>(w);
    const int64_t p0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, ps = (int64_t)gridDim.x * blockDim.x;
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
    auto issue = [&](int st, int64_t p) {
        double2 *b = ostage + (size_t)st * (OC + 1) * KT + threadIdx.x;
        cp_async16(b + OC * KT, w2 + p);
#pragma unroll
        for (int i = 0; i < OC; i++)
            if (i < kc) cp_async16_first(b + i * KT, reinterpret_cast<const double2 *>(V + (int64_t)(k0 + i) * ld) + p, pol);
    };
    if (p0 < npair) issue(0, p0);
    cp_async_commit();
    // the thread's scale: the largest exponent field among its rows of w (eight loads in flight)
    uint32_t S = 1;
    {
        int64_t p = p0;
        for (; p + 7 * ps < npair; p += 8 * ps) {
            uint64_t t[16];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const double2 v = w2[p + u * ps];
                t[2 * u] = __double_as_longlong(v.x);
                t[2 * u + 1] = __double_as_longlong(v.y);
            }
#pragma unroll
            for (int u = 0; u < 16; u++) S = max(S, fx_exp(t[u]));
        }
        for (; p < npair; p += ps) {
            const double2 v = w2[p];
            S = max(S, max(fx_exp(__double_as_longlong(v.x)), fx_exp(__double_as_longlong(v.y))));
        }
    }
    const bool wbad = S == 2047u;   // w holds an Inf or NaN
    uint32_t badm = 0;              // bit i: vector OF + i has an entry outside (-2, 2)
    const int E = (int)S - 1108;
    double accd[OF], nrm = 0.0;
#pragma unroll
    for (int i = 0; i < OF; i++) accd[i] = 0.0;
#pragma unroll
    for (int i = 0; i < OI; i++) fsum[i][threadIdx.x] = 0.0;
    Fx96 acc[OI];
#pragma unroll
    for (int i = 0; i < OI; i++) acc[i] = Fx96{0, 0, 0};
    int st = 0, inbatch = 0;
    for (int64_t p = p0; p < npair; p += ps) {
        if (p + ps < npair) issue(st ^ 1, p + ps);
        cp_async_commit();
        cp_async_wait1();   // this pair's copies are complete
        const double2 *b = ostage + (size_t)st * (OC + 1) * KT + threadIdx.x;
        const double2 wi = b[OC * KT];
        const uint64_t bx = __double_as_longlong(wi.x), by = __double_as_longlong(wi.y);
        const uint64_t Wx = fx_scaled(bx, S), Wy = fx_scaled(by, S);
        const uint32_t sx = (uint32_t)(bx >> 63), sy = (uint32_t)(by >> 63);
#pragma unroll
        for (int i = 0; i < OF; i++)
            if (i < kc) {
                const double2 v = b[i * KT];
                accd[i] = fma(v.x, wi.x, accd[i]);
                accd[i] = fma(v.y, wi.y, accd[i]);
            }
#pragma unroll
        for (int i = 0; i < OI; i++)
            if (OF + i < kc) {
                const double2 v = b[(OF + i) * KT];
                const uint64_t vx = __double_as_longlong(v.x), vy = __double_as_longlong(v.y);
                bool bi = false;
                fx_mac(acc[i], fx_basis(vx, bi), Wx, sx ^ (uint32_t)(vx >> 63));
                fx_mac(acc[i], fx_basis(vy, bi), Wy, sy ^ (uint32_t)(vy >> 63));
                badm |= (uint32_t)bi << i;
            }
        if (first) {
            nrm = fma(wi.x, wi.x, nrm);
            nrm = fma(wi.y, wi.y, nrm);
        }
        st ^= 1;
        if (++inbatch == kFxBatch) {
            inbatch = 0;
#pragma unroll
            for (int i = 0; i < OI; i++) {
                fsum[i][threadIdx.x] += fx_to_double(acc[i], E);
                acc[i] = Fx96{0, 0, 0};
            }
        }
    }
#pragma unroll
    for (int i = 0; i < OI; i++) fsum[i][threadIdx.x] += fx_to_double(acc[i], E);
    double out[OC + 1];
#pragma unroll
    for (int i = 0; i < OF; i++) out[i] = accd[i];
#pragma unroll
    for (int i = 0; i < OI; i++)
        out[OF + i] = wbad || ((badm >> i) & 1u) ? __longlong_as_double(0x7ff8000000000000ll) : fsum[i][threadIdx.x];
    out[OC] = nrm;
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {   // odd tail row, in FP64
        const int64_t r = n - 1;
        const double wr = w[r];
        for (int k = 0; k < kc; k++) out[k] += V[(int64_t)(k0 + k) * ld + r] * wr;
        if (first) out[OC] += wr * wr;
    }
    block_reduce_to<OC + 1>(out, OC + 1, part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * (OC + 1));
}

// k_odot's dynamic shared memory above the default limit, once per device
static void odot_attributes() {
    static std::atomic<bool> done[128] = {};
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) dev = 0;
    if (done[dev].load(std::memory_order_acquire)) return;
    CK(cudaFuncSetAttribute(k_odot, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)odot_smem()));
    done[dev].store(true, std::memory_order_release);
}

// w_out = w_in - V h; partial ||w_out||^2 per block.  The first row of each pair on the FP64 pipe,
// the second in fixed point (h scaled by its largest exponent field; at most 64 terms per row).
// Eight basis vectors' loads in flight per thread, three blocks per multiprocessor.
__global__ void __launch_bounds__(KT, 3) k_mupdate(const double *__restrict__ V, int64_t ld, int cnt0, const int *cntp,
                                                const int *gate, const double *__restrict__ h, const double *w_in,
                                                double *w_out, int64_t n, double *part) {
    if (gate && !*gate) return;
    const int cnt = basis_count(cnt0, cntp);
    __shared__ double hs[64];
    __shared__ uint64_t hm[64];
    __shared__ uint32_t hsg[64];
    __shared__ uint32_t Sh;
    if (threadIdx.x < 32) {
        uint32_t e = 1;
        for (int k = threadIdx.x; k < cnt; k += 32) e = max(e, fx_exp(__double_as_longlong(h[k])));
        for (int o = 16; o; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
        if (threadIdx.x == 0) Sh = e;
    }
    __syncthreads();
    const uint32_t S = Sh;
    for (int k = threadIdx.x; k < 64; k += blockDim.x) {
        const double hk = k < cnt ? h[k] : 0.0;
        const uint64_t b = __double_as_longlong(hk);
        hs[k] = hk;
        hm[k] = fx_scaled(b, S);
        hsg[k] = (uint32_t)(b >> 63);
    }
    __syncthreads();
    const bool hbad = S == 2047u;   // h holds an Inf or NaN
    const int E = (int)S - 1108;
    double nrm = 0.0;
    const int64_t npair = n >> 1;
    const double2 *wi2 = reinterpret_cast<const double2 *>(w_in);
    double2 *wo2 = reinterpret_cast<double2 *>(w_out);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npair; p += (int64_t)gridDim.x * blockDim.x) {
        double2 a = wi2[p];
        Fx96 ay{0, 0, 0};
        bool bad = hbad;   // per row: an entry of this row outside (-2, 2)
#pragma unroll 8
        for (int k = 0; k < cnt; k++) {
            const double2 v = __ldcs(reinterpret_cast<const double2 *>(V + (int64_t)k * ld) + p);
            a.x -= v.x * hs[k];
            const uint64_t vy = __double_as_longlong(v.y);
            fx_mac(ay, fx_basis(vy, bad), hm[k], hsg[k] ^ (uint32_t)(vy >> 63));
        }
        a.y = bad ? __longlong_as_double(0x7ff8000000000000ll) : a.y - fx_to_double(ay, E);
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
    k_mdot_reduce<KC><<<(cnt_max + 1 + 7) / 8, 256, 0, s>>>(partial, g, cnt, cntp, gate, h);
    CK_LAUNCH();
}

void arnoldi_dots_into(const double *V, int64_t ld, int cnt, const double *w, int64_t n, double *h, double *partial,
                       size_t partial_cap, int max_blocks, cudaStream_t s) {
    if (cnt < 1 || cnt > 64) throw Error(BGS_INVALID_ARG, "basis size outside 1..64");
    if (ld & 1) throw Error(BGS_INVALID_ARG, "basis leading dimension must be even");
    dots_launch(V, ld, cnt, nullptr, cnt, nullptr, w, n, h, partial, partial_cap, max_blocks, s);
}

// the FGMRES dots (basis of unit vectors): k_odot, then the same fixed-order reduction
static void odots_launch(const double *V, int64_t ld, int cnt0, const int *cntp, int cnt_max, const int *gate,
                         const double *w, int64_t n, double *h, double *partial, size_t partial_cap, cudaStream_t s) {
    const int nchunk = (cnt_max + OC - 1) / OC;
    const int g = grid_for(n / 2 + 1, KT, kg_odots());
    if ((size_t)nchunk * g * (OC + 1) > partial_cap) throw Error(BGS_INTERNAL, "partial scratch too small");
    odot_attributes();
    k_odot<<<dim3(g, nchunk), KT, odot_smem(), s>>>(V, ld, cnt0, cntp, gate, w, n, partial);
    CK_LAUNCH();
    k_mdot_reduce<OC><<<(cnt_max + 1 + 7) / 8, 256, 0, s>>>(partial, g, cnt0, cntp, gate, h);
    CK_LAUNCH();
}

size_t gs_pass_scratch(int cnt, int64_t n) {
    const size_t dots = (size_t)((cnt + OC - 1) / OC) * grid_for(n / 2 + 1, KT, kg_odots()) * (OC + 1);
    return std::max(dots, (size_t)grid_for(n / 2 + 1, KT, kg_update()));
}

void gs_pass(const double *V, int64_t ld, int cnt, double *w, int64_t n, double *h, double *nw, double *partial,
             size_t partial_cap, cudaStream_t s) {
    if (cnt < 1 || cnt > 64) throw Error(BGS_INVALID_ARG, "basis size outside 1..64");
    if (ld & 1) throw Error(BGS_INVALID_ARG, "basis leading dimension must be even");
    odots_launch(V, ld, cnt, nullptr, cnt, nullptr, w, n, h, partial, partial_cap, s);
    const int gu = grid_for(n / 2 + 1, KT, kg_update());
    if ((size_t)gu > partial_cap) throw Error(BGS_INTERNAL, "partial scratch too small");
    k_mupdate<<<gu, KT, 0, s>>>(V, ld, cnt, nullptr, nullptr, h, w, w, n, partial);
    CK_LAUNCH();
    k_sum_partials<<<1, 32, 0, s>>>(partial, gu, nullptr, nw);
    CK_LAUNCH();
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
    odots_launch(V, ld, 0, &st->cnt, cnt_max, nullptr, w, n, st->h1, sc.partial.p, sc.partial.n, s);
    k_mupdate<<<gu, KT, 0, s>>>(V, ld, 0, &st->cnt, nullptr, st->h1, w, w, n, sc.partial.p);
    CK_LAUNCH();
    k_sum_partials<<<1, 32, 0, s>>>(sc.partial.p, gu, nullptr, &st->nw1);
    CK_LAUNCH();
    k_fg_check<<<1, 32, 0, s>>>(st, always ? 1 : 0);
    CK_LAUNCH();
    // second pass when the test asks for it (the kernels read the decision on the device)
    odots_launch(V, ld, 0, &st->cnt, cnt_max, &st->need2, w, n, st->h2, sc.partial.p, sc.partial.n, s);
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
