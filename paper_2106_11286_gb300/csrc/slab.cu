// One sweep of a lattice split over several processes: each slab's fused
// sums (E share, spin sum, accepted moves) are summed across the processes
// (an allreduce of five doubles, outside the library); this kernel takes the
// totals, derives the sweep's observables (Eq. 2: M = sum S / N, |M|, M^2,
// M^4, |M.e|) and adds them to one handle's moments, as the single-lattice
// sweep does with its own totals.  One thread; stream-ordered.
#include "slab.h"

#include "device.cuh"

namespace hs {
namespace {

struct ApplyArgs {
    DevAccum *acc;
    const double *tot;
    double n_sites;
    double e[3];
};

__global__ void slab_apply_kernel(const ApplyArgs a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double tot[kPartials];
#pragma unroll
    for (int q = 0; q < kPartials; ++q) tot[q] = a.tot[q];
    double o[8];
    sweep_observables(tot, a.n_sites, a.e, o);
    DevAccum &A = *a.acc;
#pragma unroll
    for (int q = 0; q < 8; ++q) A.last[q] = o[q];
    A.moments[HS_SUM_E] += o[0];
    A.moments[HS_SUM_E2] += o[0] * o[0];
    A.moments[HS_SUM_ABSM] += o[4];
    A.moments[HS_SUM_M2] += o[5];
    A.moments[HS_SUM_M4] += o[6];
    A.moments[HS_SUM_MX] += o[1];
    A.moments[HS_SUM_MY] += o[2];
    A.moments[HS_SUM_MZ] += o[3];
    A.moments[HS_SUM_ABSME] += o[7];
    A.count += 1.0;
}

}  // namespace

cudaError_t launch_slab_apply(DevAccum *acc, const double *tot, double n_sites, const double e[3], cudaStream_t s) {
    ApplyArgs a{acc, tot, n_sites, {e[0], e[1], e[2]}};
    slab_apply_kernel<<<1, 32, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace hs
