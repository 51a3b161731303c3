// Conversion of an uploaded FP32 state (hs_set_spins_async) into a lattice's
// layout.  Internal to the library.
#pragma once

#include <cuda_runtime.h>

#include "hs_impl.h"

namespace hs {

// d_xyz: device, 3 * n_sites floats in natural order; stored into the planes
// (sc) or the 4-vector table (other lattices) in the lattice's precision.
cudaError_t launch_scatter_f32(int precision, const Layout &L, const float *d_xyz, cudaStream_t s);

}  // namespace hs
