// Library-internal hooks between the C ABI translation units.
#pragma once

#include <cstddef>

#include "sdrt.h"

namespace sdrt {

// CUDA device of a context, or -1 for a host-only context.
int internal_device(const sdrt_ctx* ctx);

// Record an error message on the context and return code.
int internal_fail(sdrt_ctx* ctx, int code, const char* msg);

// Device address of sdrt_residual_noalloc's static scratch buffer on the
// current device (cudaGetSymbolAddress, which also loads the module holding
// it).  Called by sdrt_create with the context's device current.
int internal_noalloc_scratch_address(void** addr);

// The address sdrt_create stored for the context's device (null for a
// host-only context).
void* internal_noalloc_scratch(const sdrt_ctx* ctx);

// Residual of a mesh whose face states are kept in the caller-provided device
// buffer `scratch` (scratch_bytes long) instead of the mesh's own workspace.
// Launches the same kernels as sdrt_residual; allocates nothing.
int internal_residual_with_scratch(sdrt_ctx* ctx, int mesh_id, const void* U, void* R, void* scratch,
                                   size_t scratch_bytes);

}  // namespace sdrt
