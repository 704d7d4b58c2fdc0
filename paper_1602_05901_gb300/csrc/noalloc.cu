// rsv_mdot_noalloc: a multi-vector dot product that allocates no memory.
//
// rsv_dot and the solvers obtain their reduction scratch (per-CTA partial
// sums and a completion ticket) from the CUDA allocator.  Some callers cannot
// allocate at the moment they need a reduction: code that has handed its
// whole device-memory budget to a memory pool or to other libraries, code
// running inside a callback of another library that forbids allocation, and
// latency-critical loops that must not risk an allocator synchronisation.
// For them this entry point keeps its scratch in one file-scope device array
// of fixed size, shared by every call in the process.
#include <mutex>

#include "common.cuh"

namespace rsv {
namespace {

constexpr int kNoallocMaxK = 64;  // most basis vectors one call may reduce against

// Partial sums [kNoallocMaxK][kRedBlocks], outputs [kNoallocMaxK], completion ticket.
struct NoallocScratch {
    double partial[kNoallocMaxK * kRedBlocks];
    double out[kNoallocMaxK];
    unsigned counter[4];
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
NoallocScratch *g_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device.  The first call on a
// device resolves it (cudaGetSymbolAddress) and caches it; the name
// g_noalloc_scratch itself is only a host-side stand-in and must never reach a
// kernel as an argument.
cudaError_t scratch_on_current_device(NoallocScratch **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_ptr[dev] = static_cast<NoallocScratch *>(p);
    }
    *out = g_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace rsv

using namespace rsv;

extern "C" rsv_status rsv_mdot_noalloc(void *stream, int64_t n, const double *w, const double *V, int64_t ldv, int k,
                                       double *result) {
    if (n < 0 || k < 1 || k > kNoallocMaxK || !result || (n > 0 && (!w || !V)) || ldv < n) return RSV_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    NoallocScratch *sc = nullptr;
    RSV_CUDA_TRY(scratch_on_current_device(&sc));
    // The ticket must start at zero; the partials and outputs are overwritten.
    RSV_CUDA_TRY(cudaMemsetAsync(sc->counter, 0, sizeof(sc->counter), st));
    RSV_CUDA_TRY(launch_mdot<double>(st, n, w, V, ldv, k, sc->partial, sc->out, &sc->counter[0], nullptr));
    RSV_CUDA_TRY(cudaMemcpyAsync(result, sc->out, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    RSV_CUDA_TRY(cudaStreamSynchronize(st));
    return RSV_OK;
}
