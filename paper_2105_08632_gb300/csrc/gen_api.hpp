// Host-side interface of the operator-specialised kernels (gen_stage.cuh,
// instantiated per element type by the translation units that
// csrc/gen/opgen.cpp writes at build time).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kargs.hpp"

namespace sdrt {

// Face records ("FR"): the states at the external flux points of every
// element, in tiles of 32 consecutive elements, each tile point-major,
// variables innermost: value (point sigma of element e of a block, variable
// v) at (fe_base + (e / 32) 32 N_fe + sigma 32 + e % 32) * V + v, fe_base the
// block's first external point (a multiple of 32).  A tile's records are one
// contiguous block (written as a stream), and within it the records of one
// point of consecutive elements are next to each other, so the partners of
// a tile's consecutive elements -- often consecutive themselves -- are read
// from a few cache lines.
//
// One launch works on one block (one element type):
//   kind 0  interpolation: FRout = M0 U at every external point;
//   kind 1  stage: per tile of 32 elements, [u_fe; u_fiu] = [M0; M12] U, the
//           common fluxes with the partners' states read from FRin (Sec. 2.1),
//           the transformed internal fluxes (Eq. "normal_transformed_flux"),
//           R~ = [M14 | M13] F~ (Eq. "residual_sdrt_matrices"),
//           dU/dt = -R~ / det J and the epilogue E; with FRout non-null the
//           epilogue's new state (the next RK stage, or the new U of the last
//           stage) is interpolated to the external points and written to FRout.
struct GenArgs {
    int nelem, ld;
    int64_t u_off;           // element offset of the block in the state arrays
    int64_t fr_base;         // FR index of the block's first record (fe_base * V)
    const float* metric;     // [NM][ld] (kargs.hpp KBlock layout)
    const int* pmap;         // [N_fe][ld] FR index of each external point's partner
    const float* U;          // stage input state (whole state array)
    const float* FRin;       // face records of the stage input (whole array)
    float* FRout;            // face records of the epilogue's new state (whole array) or null
    KPhys<float> P;
    KEpi<float> E;
};

// Launcher of one element type: returns 0, or -1 if (V, system, Riemann) is
// not instantiated.
typedef int (*GenLauncher)(int kind, const GenArgs& a, int V, int sys, int rie, int nsm, cudaStream_t st);

// Launcher of the specialised kernels of (shape, degree), or null.
GenLauncher gen_launcher(int shape, int p);

}  // namespace sdrt
