// sdrt_residual_noalloc: the residual entry point for callers that cannot
// allocate device memory.
//
// sdrt_residual keeps the face states exchanged between elements in a
// workspace that the library allocates with cudaMalloc on first use.  Some
// callers cannot let a library do that: a solver embedded as a plugin inside
// another framework whose memory pool owns the whole device budget, or a
// time-critical loop that cannot accept cudaMalloc's implicit device-wide
// synchronisation.  This entry point runs the same kernels with the face
// states in a fixed buffer that is part of the library image (a file-scope
// __device__ array), so the call itself allocates nothing.
#include <cuda_runtime.h>

#include "internal.hpp"
#include "sdrt.h"

namespace {

// Face-state scratch of sdrt_residual_noalloc.  Every GPU on which the library
// is loaded holds it until the process exits.  Every call overwrites it
// completely before reading it (each external flux point of each element is
// written by the interpolation kernel, and the residual kernel reads only
// points that exist), so nothing has to be cleared between calls.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SDRT_NOALLOC_SCRATCH_BYTES];

}  // namespace

namespace sdrt {

int internal_noalloc_scratch_address(void** addr) {
    *addr = nullptr;
    // Host code cannot use the symbol itself: on the host it names a
    // stand-in, not device memory.  The device address is looked up with the
    // context's device current; the lookup loads this file's module.
    return (int)cudaGetSymbolAddress(addr, g_noalloc_scratch);
}

}  // namespace sdrt

extern "C" int sdrt_residual_noalloc(sdrt_ctx* ctx, int mesh_id, const void* U_dev, void* R_dev) {
    if (!ctx) return SDRT_ERR_ARG;
    if (sdrt::internal_device(ctx) < 0)
        return sdrt::internal_fail(ctx, SDRT_ERR_STATE, "host-only context: no device computation");
    void* scratch = sdrt::internal_noalloc_scratch(ctx);
    if (!scratch) return sdrt::internal_fail(ctx, SDRT_ERR_STATE, "static scratch buffer not resolved");
    return sdrt::internal_residual_with_scratch(ctx, mesh_id, U_dev, R_dev, scratch, SDRT_NOALLOC_SCRATCH_BYTES);
}
