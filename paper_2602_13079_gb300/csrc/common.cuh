// Shared device/host utilities of libbgs (GB300, sm_103a).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "../../include/bgs.h"

namespace bgs {

// ------------------------------------------------------------------------------------------
// Errors: thrown inside the library, turned into status codes at the C ABI.
// ------------------------------------------------------------------------------------------
struct Error : std::runtime_error {
    int status;
    Error(int s, const std::string &m) : std::runtime_error(m), status(s) {}
};

inline void cuda_check(cudaError_t e, const char *file, int line) {
    if (e == cudaSuccess) return;
    char buf[256];
    snprintf(buf, sizeof(buf), "%s at %s:%d", cudaGetErrorString(e), file, line);
    throw Error(e == cudaErrorMemoryAllocation ? BGS_OOM : BGS_CUDA_ERROR, buf);
}
#define CK(x) ::bgs::cuda_check((x), __FILE__, __LINE__)
// every kernel launch is followed by CK_LAUNCH(): it checks the launch and counts it
void count_launch();
#define CK_LAUNCH() (::bgs::count_launch(), ::bgs::cuda_check(cudaGetLastError(), __FILE__, __LINE__))

// ------------------------------------------------------------------------------------------
// Device buffers: stream-ordered allocation, freed on the stream they were allocated on.
// ------------------------------------------------------------------------------------------
// Device allocations are stream-ordered, from a memory pool the library owns (one per device)
// that keeps freed memory cached for the next allocation instead of returning it to the driver
// at every synchronisation (bgs_release_cached_memory() trims it).  BGS_PLAIN_ALLOC=1 switches to
// cudaMalloc / cudaFree (synchronous).
bool plain_alloc();
cudaMemPool_t device_pool();

template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    DBuf() = default;
    DBuf(size_t count, cudaStream_t st) { alloc(count, st); }
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n; s = o.s;
            o.p = nullptr; o.n = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t count, cudaStream_t st) {
        release();
        s = st;
        n = count;
        if (count) {
            if (plain_alloc()) CK(cudaMalloc((void **)&p, count * sizeof(T)));
            else CK(cudaMallocFromPoolAsync((void **)&p, count * sizeof(T), device_pool(), st));
        }
    }
    void release() {
        if (p) {
            if (plain_alloc()) {
                cudaStreamSynchronize(s);
                cudaFree(p);
            } else {
                cudaFreeAsync(p, s);
            }
        }
        p = nullptr;
        n = 0;
    }
    T *get() const { return p; }
    size_t bytes() const { return n * sizeof(T); }
};

// A device CSR matrix.  Values in FP64 always; FP32 / BF16 copies exist in mixed precision.
// Optionally also stored as SELL-32: rows in slices of 32 (one warp), each slice padded to its
// longest row and stored column-major (entry j of the 32 rows contiguous), so that a warp's
// loads of values and column indices are single contiguous 128/256-byte runs.
struct DCsr {
    int n = 0, m = 0;       // rows, columns
    int64_t nnz = 0;
    DBuf<int> rp, ci;
    DBuf<double> v;
    DBuf<float> vf;
    DBuf<__nv_bfloat16> vb;
    int lanes = 0;          // CSR SpMV threads per row chosen for this matrix
    int tpb = 256;          // threads per block of its SpMV launches (autotuned: 128, 256 or 512)
    // SELL-32 copy (sell == true when built): slice offsets, columns (a padded slot repeats
    // its slice's first stored column, with value 0), CSR index of each slot (-1 pad)
    bool sell = false;
    int64_t sell_nnz = 0;
    DBuf<int> sptr, sci, sperm;
    DBuf<double> sv;
    DBuf<float> svf;
    DBuf<__nv_bfloat16> svb;
    // SELL-32 with one diagonal offset per slot (dia == true when built): slice s of 32 rows holds
    // w_s <= 32 slots, slot k one offset o for all its rows (entry column = row + o), so no column
    // index is stored per entry; a row without an entry at that offset holds value 0 there.  Used for
    // the structured operators (stencil blocks, the full operator), where the offsets repeat.
    bool dia = false;
    int64_t dia_nnz = 0;            // value slots (32 per slice and offset)
    int dia_wmax = 0;               // the widest slice's offset count (the stride of doff)
    DBuf<int> dptr, doff, dperm;    // slot start per slice (multiple of 32); offset k of slice s at
                                    // doff[s * dia_wmax + k]; CSR index of each slot (-1: padding)
    DBuf<double> dv;
    DBuf<float> dvf;
    DBuf<__nv_bfloat16> dvb;
    // Field-interleaved node blocks (bsr == true when built; the full operator of F fields of equal
    // size nc only): node I gathers rows f*nc + I (f < F); its block columns J (ascending) each hold an
    // F x F block, entry (f, g) = A(f*nc + I, g*nc + J) or 0.  Nodes in slices of 32 (one warp), slice
    // s holding w_s block slots; bcol[slot*32 + lane], bval[((slot*F + f)*F + g)*32 + lane].
    bool bsr = false;
    // the node-block kernel runs when it is the only sliced layout (the autotuner's choice, or the
    // one built); untuned, the diagonal-offset and SELL-32 forms come first
    bool bsr_active() const { return bsr && !dia && !sell; }
    int bsr_F = 0, bsr_nc = 0;
    int64_t bsr_slots = 0;          // block slots (32 per slice and slot)
    DBuf<int> bptr, bcol;           // slot start per slice (multiple of 32), block column per slot
    DBuf<double> bval;
};

// ------------------------------------------------------------------------------------------
// Launch helpers
// ------------------------------------------------------------------------------------------
// Multiprocessors of the current device (cudaDevAttrMultiProcessorCount, looked up once per
// device): every grid cap below is a multiple of it (152 on a GB300).
int num_sms();

// Blocks for `work` items of `block` each, capped at max_blocks (default: 16 per multiprocessor).
inline int grid_for(int64_t work, int block, int max_blocks = 0) {
    if (max_blocks <= 0) max_blocks = num_sms() * 16;
    int64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(double x) { return (float)x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return (double)x; }
__device__ __forceinline__ double to_d(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

template <class T>
__device__ __forceinline__ T from_d(double x);
template <>
__device__ __forceinline__ double from_d<double>(double x) { return x; }
template <>
__device__ __forceinline__ float from_d<float>(double x) { return (float)x; }

// read-only cached load
template <class T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }
template <>
__device__ __forceinline__ __nv_bfloat16 ldg(const __nv_bfloat16 *p) { return *p; }

}  // namespace bgs
