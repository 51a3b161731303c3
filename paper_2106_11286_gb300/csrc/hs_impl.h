// Internal declarations of the GB300 Metropolis library (not part of the ABI).
//
// Device layouts (all in HBM, allocated by the lattice handle):
//  * stencil path (unmasked periodic sc, Lx/2 divisible by the vector width):
//    colour-major SoA.  Plane (colour c, component a) is an array
//    [Lz][Ly][Lx/2] of the storage type; site (x,y,z) of colour
//    c = (x+y+z)&1 sits at xh = x/2 in row (z,y).  Planes are ordered
//    c0x c0y c0z c1x c1y c1z so that one colour is 3 contiguous planes.
//  * table path (everything else): present sites renumbered colour by colour
//    (ascending natural index inside a class); spins as 4-vectors (x,y,z,0)
//    of the storage type, one per renumbered site plus one zero dummy at the
//    end; neighbour table [width][n_pad] of renumbered indices, padded with
//    the dummy; nat[i] = natural index of renumbered site i.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/hs.h"

namespace hs {

constexpr int kPartials = 5;  // E, Sx, Sy, Sz, accepted
constexpr int kRingMax = 64;  // sweeps whose slots a ring fold takes at most
constexpr int kSweepRecord = kPartials + 8;  // a ring fold's per-sweep record: totals, observables
constexpr int kBlock = 256;   // threads per CTA of the sweep kernels
// partial-sum sets per colour of a z-slab: first own plane, last own plane,
// the planes between them, the whole slab in one launch
constexpr int kSlabSets = 4;

// Division by a runtime constant d (1 <= d < 2^31) of numerators n < 2^31
// by multiply-high and shift: with l = ceil(log2 d) and m = ceil(2^(31+l)/d)
// (m < 2^32), floor(n m / 2^(31+l)) = floor(n / d) because the rounding
// excess n (m - 2^(31+l)/d) / 2^(31+l) stays below 2^-l <= 1/d.
#ifdef __CUDACC__
#define HS_HOST_DEVICE __host__ __device__
#else
#define HS_HOST_DEVICE
#endif

struct FastDiv {
    uint32_t d, m, l;
    HS_HOST_DEVICE FastDiv() : d(1), m(0), l(0) {}
    explicit FastDiv(uint32_t div) : d(div), l(0) {
        while ((1ull << l) < div) ++l;
        m = (l == 0) ? 0u : (uint32_t)(((1ull << (31 + l)) + div - 1) / div);
    }
#ifdef __CUDACC__
    __device__ __forceinline__ uint32_t div(uint32_t n) const { return l == 0 ? n : (__umulhi(n, m) >> (l - 1)); }
#endif
};

// Device-resident accumulator block of one lattice.
struct DevAccum {
    double moments[HS_N_MOMENTS];
    double count;          // accumulated sweeps
    double accepted;       // accepted moves since the last hs_sweep began
    double last[8];        // E, Mx, My, Mz, |M|, M2, M4, |M.e| of the last finalised reduction
    unsigned int done;     // CTA arrival counter of the finishing pass
    int error;             // latched device error code (0 = none)
    double sums[5];        // E, sum S_x, sum S_y, sum S_z, accepted moves of the last finalised reduction
};

// Parameters of one colour pass.
struct PassArgs {
    // stencil layout
    void *own[3];
    const void *oth[3];
    int Lx, Ly, Lz, Lh;
    FastDiv div_nxv, div_ly;   // row = t / (Lh/V), z = row / Ly
    int nz, z_off;             // planes updated, array plane of the first (1 for a z-slab: plane 0 is a halo)
    int zpar;                  // parity of (global z - array z), for the colour of a row
    uint32_t site_off;         // global natural index - (array row Lx + x), mod 2^32
    uint32_t rank_off;         // colour rank of a site - (array row Lh + x / 2), mod 2^32
    int ty;                    // z-march stencil: rows per plane-slab
    uint32_t rev;              // register stencil: nonzero = work items in descending order, item t taken as
                               // rev - t (rev = items - 1)
    // table layout
    void *spins4;           // 4-vectors, renumbered order
    const int32_t *nbr;     // [width][n_pad]
    const uint32_t *nat;    // natural index per renumbered site
    int width;
    int64_t n_pad;
    int64_t begin, end;     // renumbered range of this colour
    int64_t colour_begin;   // first renumbered index of this colour (energy split)
    // common
    int colour;
    int n_colours;
    double J, K, e[3];
    double beta;
    float fJ, fK, fe[3], fbeta;  // the same in FP32 for the FP32 / FP16 kernels
    int tensor;             // 1: the on-site anisotropy tensor term is on
    double A[6];            // its symmetric tensor (xx, yy, zz, xy, xz, yz)
    float fA[6];
    const double2 *sc_tab;  // FP64 trial: sin, cos(pi j / 1024), j = 0..2047
    int zaxis;              // 1: e = (0, 0, 1) exactly (the FP64 stencil takes S.e = S_z)
    uint32_t key0, key1, replica, sweep;
    double *partials;       // [ring slots][n_colours][n_blocks][kPartials]; a slab has kSlabSets sets per colour
                            // (pass = kSlabSets colour + set, n_colours = 2 kSlabSets); a launch of fewer CTAs
                            // than n_blocks leaves the rest of its set zero
    double *sweep_tot;      // [ring slots][kSweepRecord]: per-sweep records of a ring fold
    int pass;               // colour index = partial slot
    int slot;               // ring slot: the sweep's index within its fold group (0 for single passes)
    int n_blocks;
    int finish;             // 1: last launch of the sequence, its last CTA to arrive reduces and finalises
    uint64_t skip_sets;     // finaliser: partial sets of the slot left out (bit p = set p; not written this sweep)
    int accumulate;         // 0: no fused measurement; 1: measure and add the moments to the accumulator;
                            // 2: measure only (the sums; a slab whose moments come from all slabs' sums)
    double n_present;
    DevAccum *acc;
};

// codes as in hs_kernel (include/hs.h)
enum KernelKind { kStencil = 1, kTable = 3, kMarch = 4, kPipe = 5 };

struct Layout {
    bool structured;
    bool slab;              // z-slab of a periodic sc lattice: Lz = nz + 2 array planes, halos at 0 and nz + 1
    int z0, nz, Lz_glob;    // first global plane, own planes, global Lz (slab); 0, Lz, Lz otherwise
    int kernel;             // KernelKind
    int vec;                // vector width of the stencil kernels
    int prefetch;           // register stencil: 0 none, 1 next work item in registers, 2 split prefetch
    int tensor;             // 1: the on-site anisotropy tensor term is on (register stencil without
                            //    prefetch, or the neighbour table)
    int ty;                 // z-march stencil: rows per plane-slab
    int order;              // register stencil: 1 ascending passes, 2 alternating (colour 1 descending)
    bool plain;             // register stencil: the ascending-only variant (lattices beyond 2^31 sites)
    int n_colours;
    int64_t n_sites, n_present;
    // stencil
    int Lx, Ly, Lz, Lh;
    void *planes;           // 6 planes of Lz*Ly*Lh elements
    // table
    void *spins4;
    int32_t *nbr;
    uint32_t *nat;
    int width;
    int64_t n_pad;
    int64_t colour_begin[65];  // renumbered colour ranges (n_colours + 1 entries)
};

size_t storage_size(int precision);

// Record the thread-local message returned by hs_last_error; returns code.
int set_last_error(int code, const std::string &msg);

// Kernel launchers (kernels.cu).  All return cudaError_t of the launch.
cudaError_t launch_pass(int precision, const Layout &L, const PassArgs &a, int n_blocks, cudaStream_t s);
cudaError_t launch_init(int precision, const Layout &L, int mode, const double e[3], uint32_t key0,
                        uint32_t key1, uint32_t replica, cudaStream_t s);
cudaError_t launch_gather_sites(int precision, const Layout &L, int64_t n, const int64_t *d_sites, double *d_out,
                                cudaStream_t s);
cudaError_t launch_scatter(int precision, const Layout &L, const double *d_xyz, cudaStream_t s);
cudaError_t launch_gather(int precision, const Layout &L, double *d_xyz, cudaStream_t s);
cudaError_t launch_measure(int precision, const Layout &L, const PassArgs &a, int n_blocks, cudaStream_t s);
// Fold ring slots 0 .. n_slots-1 (sweeps of a.n_colours passes each, in sweep
// order) into the accumulator: one CTA per slot sums it, then one thread
// applies the totals in order.  1 <= n_slots <= kRingMax.
cudaError_t launch_fold(const PassArgs &a, int n_slots, cudaStream_t s);
int pass_blocks(int precision, const Layout &L, int n_sm, int blocks_per_sm);
int pass_occupancy(int precision, const Layout &L, int accumulate);
size_t pipe_smem_bytes(int precision, int vec);  // dynamic shared memory of the pipelined stencil

}  // namespace hs
