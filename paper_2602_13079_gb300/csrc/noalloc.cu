// Arnoldi block dot products for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point where they need
// this operation: applications whose device memory is fully pre-reserved by their own pool
// manager, or embedded/real-time hosts that forbid allocation after start-up.
// bgs_arnoldi_dots() allocates its per-block partial-sum scratch on every call;
// bgs_arnoldi_dots_noalloc() below instead uses one fixed scratch array that lives in this
// library's device image, so a call allocates nothing.
#include <mutex>

#include "internal.h"

namespace {

// The dot kernel's grid is capped at kNoAllocBlocks blocks here (the kernel strides over the rows,
// so any grid gives the same sums up to their fixed summation order).  Its partial sums then need
// at most 4 chunks of 16 vectors (cnt <= 64) times kNoAllocBlocks blocks times 17 sums = 31,008
// doubles (248,064 bytes).  Every GPU that loads the library holds this array until the process
// exits.
constexpr int kNoAllocBlocks = 456;
constexpr size_t kNoAllocPartials = 4 * (size_t)kNoAllocBlocks * 17;
static_assert(kNoAllocPartials * sizeof(double) == 248064, "scratch size stated in bgs.h");

static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[128] = {};   // device address of the array, per device ordinal

}  // namespace

extern "C" int bgs_arnoldi_dots_noalloc(const double *V, int64_t ld, int cnt, const double *w, int64_t n, double *h,
                                        void *stream) {
    if (!V || !w || !h || n < 1 || cnt < 1 || cnt > 64 || ld < n || (ld & 1)) return BGS_INVALID_ARG;
    if (((uintptr_t)V | (uintptr_t)w) & 15) return BGS_INVALID_ARG;   // read as 16-byte pairs
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return BGS_CUDA_ERROR;
    double *scratch = nullptr;
    {
        // First call on a device: look up the array's device address with that device current.
        // In host code the symbol name is only a host-side stand-in, never a device address.
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) {
                cudaGetLastError();   // leave no sticky error for the caller's next launch check
                return BGS_CUDA_ERROR;
            }
            g_noalloc_ptr[dev] = (double *)p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    try {
        // every partial sum the reduction reads is written earlier in the same call, so nothing in
        // the shared array has to be cleared first
        bgs::arnoldi_dots_into(V, ld, cnt, w, n, h, scratch, kNoAllocPartials, kNoAllocBlocks,
                               (cudaStream_t)stream);
    } catch (const bgs::Error &e) {
        return e.status;
    } catch (...) {
        return BGS_INTERNAL;
    }
    return BGS_OK;
}
