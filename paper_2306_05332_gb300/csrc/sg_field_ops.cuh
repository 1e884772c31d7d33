// Launchers of the operators on a solved potential (outside the V-cycle).
#pragma once
#include "sg_internal.cuh"

namespace sg {

// out[d][cell] = c[d] (8 (phi_{+1} - phi_{-1}) - (phi_{+2} - phi_{-2})) along axis d
// (c[d] = -1 / (12 h_d): g = -grad phi to fourth order, Sec. 3), FP64; out holds
// three arrays of the grid's size, x component first.
cudaError_t launch_gravity(const LevelGeom& g, const double* phi, double* out, const double c[3], cudaStream_t st);

}  // namespace sg
