// Device side of the multi-process z-slab decomposition (slab.cu): the
// per-sweep observables of Eq. 2 from the sums of all slabs, added to one
// handle's accumulator on the device.  Internal to the library.
#pragma once

#include <cuda_runtime.h>

#include "hs_impl.h"

namespace hs {

// tot = {E, sum S_x, sum S_y, sum S_z, accepted} of one sweep of the whole
// lattice (device memory); n_sites its present spins, e the unit easy axis.
cudaError_t launch_slab_apply(DevAccum *acc, const double *tot, double n_sites, const double e[3], cudaStream_t s);

}  // namespace hs
