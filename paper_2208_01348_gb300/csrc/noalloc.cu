// Matrix-vector product for callers that cannot allocate device memory.
//
// eels_matvec_dev keeps its FFT scratch in the context, which grows it with
// the device allocator on demand.  Some callers cannot let a library call
// the allocator at that point: real-time or latency-critical loops that
// must not hit the allocator's implicit synchronisation, and hosts (plugins
// inside a larger application, frameworks with their own caching pool) that
// own all device memory and forbid foreign allocations.  eels_matvec_dev_noalloc
// applies the same prepared operator with the same kernels, but its FFT
// scratch is one fixed array compiled into the library: a file-scope
// __device__ array of EELS_NOALLOC_SCRATCH_BYTES (64 MiB) that every GPU which
// loads the library holds until the process exits.  The call itself
// allocates nothing.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/eelsdda.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = EELS_NOALLOC_SCRATCH_BYTES;

// The shared scratch.  Its host-side name is only a stand-in for the symbol:
// the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[256] = {};   // device address of g_noalloc_scratch per device ordinal

// Device address of the scratch on device `dev` (the context's device):
// looked up once per device (the first call on that device) with that
// device made current for the lookup, then the caller's current device is
// restored.
int scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= 256) return EELS_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        int cur = 0;
        if (cudaGetDevice(&cur) != cudaSuccess) {
            cudaGetLastError();
            return EELS_E_CUDA;
        }
        void* p = nullptr;
        cudaError_t e = cudaSetDevice(dev);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        const cudaError_t e2 = cudaSetDevice(cur);
        if (e != cudaSuccess || e2 != cudaSuccess || !p) {
            cudaGetLastError();
            return EELS_E_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return EELS_OK;
}

}  // namespace

// Engine-side helpers (engine.cu): the context's device ordinal, and the
// launch of the prepared operator with the given scratch (it validates the
// context, refuses a call whose current device is not the context's, returns
// an EELS_* code and sets the context's error text on failure).
int eels_internal_device(const eels_ctx* ctx);
int eels_internal_matvec_with_scratch(eels_ctx* ctx, int precision, const void* x, void* y, int n_sys, void* stream,
                                      void* scratch, size_t scratch_bytes);

extern "C" int eels_matvec_dev_noalloc(eels_ctx* ctx, int precision, const void* x, void* y, int n_sys,
                                       void* cuda_stream) {
    if (!ctx) return EELS_E_INVALID_ARG;
    void* scratch = nullptr;
    const int rc = scratch_address(eels_internal_device(ctx), &scratch);
    if (rc != EELS_OK) return rc;
    return eels_internal_matvec_with_scratch(ctx, precision, x, y, n_sys, cuda_stream, scratch, kScratchBytes);
}
