// Natural-order FP32 spins to the lattice's layout, for the pipelined upload
// hs_set_spins_async.  A float widens exactly, so each stored value is the
// one an FP64 input of the same number would give.
#include "upload.h"

#include "device.cuh"

namespace hs {
namespace {

// sc planes [colour][xyz][z][y][x/2]; a z-slab stores its own planes from
// array plane 1 (its halos are planes 0 and nz + 1).
template <int P>
__global__ void sc_scatter_f32_kernel(void *planes, const float *xyz, int Lx, int Ly, int nz, int Lz_arr, int z_off,
                                      int z0, int Lh) {
    using S = typename Tr<P>::S;
    S *pl = (S *)planes;
    const int64_t plane = (int64_t)Lz_arr * Ly * Lh;
    const int64_t n = (int64_t)Lx * Ly * nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % Lx);
        const int64_t r = i / Lx;
        const int y = (int)(r % Ly), z = (int)(r / Ly);
        const int c = (x + y + z + z0) & 1;
        const int64_t idx = (r + (int64_t)z_off * Ly) * Lh + (x >> 1);
#pragma unroll
        for (int q = 0; q < 3; ++q)
            pl[(int64_t)(3 * c + q) * plane + idx] = store_from_double<S>((double)xyz[3 * i + q]);
    }
}

// Neighbour-table layout: present site i (renumbered) holds natural site nat[i].
template <int P>
__global__ void table_scatter_f32_kernel(void *spins4, const uint32_t *nat, int64_t n_present, const float *xyz) {
    using S = typename Tr<P>::S;
    using S4 = Vec<S, 4>;
    S4 *sp = reinterpret_cast<S4 *>(spins4);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_present;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t site = nat[i];
        S4 s;
        s.v[0] = store_from_double<S>((double)xyz[3 * site]);
        s.v[1] = store_from_double<S>((double)xyz[3 * site + 1]);
        s.v[2] = store_from_double<S>((double)xyz[3 * site + 2]);
        s.v[3] = store_from_double<S>(0.0);
        sp[i] = s;
    }
}

int grid_of(int64_t n) {
    int64_t g = (n + kBlock - 1) / kBlock;
    return (int)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

template <int P>
cudaError_t scatter_f32(const Layout &L, const float *d_xyz, cudaStream_t s) {
    if (L.structured)
        sc_scatter_f32_kernel<P><<<grid_of(L.n_sites), kBlock, 0, s>>>(L.planes, d_xyz, L.Lx, L.Ly, L.nz, L.Lz,
                                                                       L.slab ? 1 : 0, L.z0, L.Lh);
    else
        table_scatter_f32_kernel<P><<<grid_of(L.n_present), kBlock, 0, s>>>(L.spins4, L.nat, L.n_present, d_xyz);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_scatter_f32(int precision, const Layout &L, const float *d_xyz, cudaStream_t s) {
    switch (precision) {
    case HS_FP64: return scatter_f32<HS_FP64>(L, d_xyz, s);
    case HS_FP32: return scatter_f32<HS_FP32>(L, d_xyz, s);
    case HS_FP16: return scatter_f32<HS_FP16>(L, d_xyz, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hs
