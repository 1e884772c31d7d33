// Launchers of the operators on a solved potential (outside the V-cycle).
#pragma once
#include "sg_internal.cuh"

namespace sg {

// out[d][cell] = c[d] (8 (phi_{+1} - phi_{-1}) - (phi_{+2} - phi_{-2})) along axis d
// (c[d] = -1 / (12 h_d): g = -grad phi to fourth order, Sec. 3); out holds
// three arrays of the grid's size, x component first.  With scratch (one
// unsigned word on the device) and a 16-byte aligned phi the combination is
// formed exactly in 64-bit fixed point on the level's scale (a pre-pass
// kernel finds it) and rounded to FP64 once; otherwise in FP64.  *nkernels:
// the kernels launched.
cudaError_t launch_gravity(const LevelGeom& g, const double* phi, double* out, const double c[3], unsigned* scratch,
                           int* nkernels, cudaStream_t st);

}  // namespace sg
