// Colour-pass Metropolis kernels for sm_103a (arXiv 2106.11286: Eq. 1, the
// Metropolis steps (i)-(iii), Eq. 2), plus initialisation, layout
// conversion and measurement.
//
// Every kernel here is HBM- or ALU-bound elementwise work over one colour
// class: no dense contraction exists, so no tensor-core path is used.  The
// stencil pass reads its own colour and the other colour with 128-bit
// coalesced loads (own values, plus the other colour's rows at y+-1, z+-1 and
// the same row for the x neighbours, all at the same xh); the neighbour rows
// are shared by adjacent rows of the grid through L1/L2.  Random numbers come
// from an in-register Philox4x32-10 keyed by (seed, replica, sweep, colour,
// site): nothing of the generator lives in memory.
//
// Reductions: per-thread partials -> warp shuffle -> CTA (FP64) -> one slot
// per CTA and pass; the last CTA of the finishing pass sums the slots in a
// fixed order (bit-reproducible) and updates the FP64 accumulator.
#include <cuda_fp16.h>
#include <stdint.h>

#include <algorithm>

#include "device.cuh"

namespace hs {
namespace {

// Register stencil: every operand is loaded from global memory (L1/L2 serve
// the neighbour rows shared by adjacent work items).  With PF the loads of
// the thread's next work item are issued before the current one is
// computed (two items in flight, unrolled by hand so no operand is copied).
template <int P, int V, bool MEAS, bool PF>
__global__ void __launch_bounds__(kBlock) sc_pass_kernel(const PassArgs a) {
    using S = typename Tr<P>::S;
    using C = typename Tr<P>::C;
    using VT = Vec<S, V>;
    const uint32_t n_items = (uint32_t)a.Lz * a.Ly * (a.Lh / V);  // < 2^31: n_sites < 2^32
    const int c = a.colour;
    C J, K, ex, ey, ez, beta;
    load_params(a, J, K, ex, ey, ez, beta);
    S *own_w[3] = {(S *)a.own[0], (S *)a.own[1], (S *)a.own[2]};
    const S *const own[3] = {(const S *)a.own[0], (const S *)a.own[1], (const S *)a.own[2]};
    const S *const oth[3] = {(const S *)a.oth[0], (const S *)a.oth[1], (const S *)a.oth[2]};
    C accE = C(0), accX = C(0), accY = C(0), accZ = C(0);
    unsigned nacc = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    auto compute = [&](StencilItem<P, V> &it) {
        if (update_item<P, V, MEAS>(it.s, it.o, it.nym, it.nyp, it.nzm, it.nzp, it.ed, it.p, it.site0, c, a, J, K,
                                    ex, ey, ez, beta, accE, accX, accY, accZ, nacc)) {
#pragma unroll
            for (int q = 0; q < 3; ++q) *reinterpret_cast<VT *>(own_w[q] + it.b0) = it.s[q];
        }
    };
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (!PF) {
        for (; t < n_items; t += stride) {
            StencilItem<P, V> it;
            load_item<P, V>(a, t, own, oth, it);
            compute(it);
        }
    } else if (t < n_items) {
        StencilItem<P, V> A, B;
        load_item<P, V>(a, t, own, oth, A);
        while (true) {
            if (t + stride < n_items) load_item<P, V>(a, t + stride, own, oth, B);
            compute(A);
            t += stride;
            if (t >= n_items) break;
            if (t + stride < n_items) load_item<P, V>(a, t + stride, own, oth, A);
            compute(B);
            t += stride;
            if (t >= n_items) break;
        }
    }
    write_partials<C, MEAS>(a, accE, accX, accY, accZ, nacc);
}

// ----------------------------------------------------------------- staged stencil pass
// The other colour's planes are staged in shared memory by the bulk-copy
// (TMA) engine.  A CTA owns a slab of ty rows (full x) and marches through a
// chunk of z planes.  Shared memory holds a ring of 4 other-colour plane
// slabs (z-1, z, z+1 and z+2 arriving), each ty+2 rows (halo rows y0-1 and
// y0+ty wrap periodically), and 2 own-colour slabs (z, z+1 arriving).  Every
// copy group completes on an mbarrier with an expected byte count; waits are
// bounded (timeout -> device error word, uniform abort of the CTA).

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait on one phase of an mbarrier: about one second of clock, or
// 2^26 polls, whichever comes first.
constexpr long long kWaitCycles = 2000000000LL;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (mbar_try(bar, parity)) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Issue one copy group from warp 0: n_oth other-colour planes starting at
// plane zo (ring slots so..so+n_oth-1) and optionally the own plane zw into
// own slot sw.  Lane l issues copy l: other copies are (plane, component,
// {main rows, low halo row, high halo row}), own copies one per component.
template <typename S>
__device__ __forceinline__ void issue_group(uint64_t *bar, S *oth_s, S *own_s, const PassArgs &a, int ty, int y0,
                                            int zo, int n_oth, int so, int zw, int sw) {
    const int lane = threadIdx.x & 31;
    const uint32_t row_bytes = (uint32_t)a.Lh * sizeof(S);
    const int n_own = (zw >= 0) ? 3 : 0;
    if (lane == 0) {
        const uint32_t bytes = (uint32_t)(n_oth * 3 * (ty + 2) + n_own * ty) * row_bytes;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, bytes);
    }
    __syncwarp();
    const int n_copies = n_oth * 9 + n_own;
    const int Ly = a.Ly, Lz = a.Lz, Lh = a.Lh;
    for (int l = lane; l < n_copies; l += 32) {
        if (l < n_oth * 9) {
            const int pl = l / 9, q = (l % 9) / 3, part = l % 3;
            int z = zo + pl;
            z = (z % Lz + Lz) % Lz;
            const int slot = (so + pl) & 3;
            const S *plane = static_cast<const S *>(a.oth[q]);
            S *dst = oth_s + ((size_t)(slot * 3 + q) * (ty + 2)) * Lh;
            if (part == 0) {
                bulk_g2s(dst + Lh, plane + ((size_t)z * Ly + y0) * Lh, (uint32_t)ty * row_bytes, bar);
            } else if (part == 1) {
                const int y = (y0 == 0) ? Ly - 1 : y0 - 1;
                bulk_g2s(dst, plane + ((size_t)z * Ly + y) * Lh, row_bytes, bar);
            } else {
                const int y = (y0 + ty == Ly) ? 0 : y0 + ty;
                bulk_g2s(dst + (size_t)(ty + 1) * Lh, plane + ((size_t)z * Ly + y) * Lh, row_bytes, bar);
            }
        } else {
            const int q = l - n_oth * 9;
            const S *plane = static_cast<const S *>(a.own[q]);
            S *dst = own_s + ((size_t)(sw * 3 + q) * ty) * Lh;
            bulk_g2s(dst, plane + ((size_t)zw * Ly + y0) * Lh, (uint32_t)ty * row_bytes, bar);
        }
    }
}

template <int P, int V, bool MEAS>
__global__ void __launch_bounds__(kBlock) sc_staged_kernel(const PassArgs a) {
    using S = typename Tr<P>::S;
    using C = typename Tr<P>::C;
    using VT = Vec<S, V>;
    extern __shared__ __align__(128) unsigned char hs_dyn_smem[];
    __shared__ __align__(8) uint64_t bars[2];
    const int Lh = a.Lh, Ly = a.Ly, Lx = a.Lx;
    const int ty = a.ty;
    const int nxv = Lh / V;
    const int items = ty * nxv;
    const int n_yslab = Ly / ty;
    const int c = a.colour;
    S *oth_s = reinterpret_cast<S *>(hs_dyn_smem);               // [4][3][ty+2][Lh]
    S *own_s = oth_s + (size_t)4 * 3 * (ty + 2) * Lh;            // [2][3][ty][Lh]
    S *own_g[3] = {(S *)a.own[0], (S *)a.own[1], (S *)a.own[2]};
    C J, K, ex, ey, ez, beta;
    load_params(a, J, K, ex, ey, ez, beta);
    C accE = C(0), accX = C(0), accY = C(0), accZ = C(0);
    unsigned nacc = 0;
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t G = 0;  // copy groups issued so far by this CTA (barrier G&1, phase G>>1)
    bool abort = false;
    for (int unit = blockIdx.x; unit < a.n_units && !abort; unit += gridDim.x) {
        const int ys = unit % n_yslab;
        const int y0 = ys * ty;
        const int z0 = (unit / n_yslab) * a.zchunk;
        const int z1 = min(a.Lz, z0 + a.zchunk);
        // prologue: other planes z0-1, z0, z0+1 into slots 0..2, own plane z0 into slot 0
        if (threadIdx.x < 32) issue_group<S>(&bars[G & 1], oth_s, own_s, a, ty, y0, z0 - 1, 3, 0, z0, 0);
        for (int z = z0; z < z1; ++z) {
            const int j = z - z0;
            const bool ok = mbar_wait_bounded(&bars[G & 1], (G >> 1) & 1);
            if (__syncthreads_or(!ok)) {
                abort = true;
                break;
            }
            ++G;
            if (z + 1 < z1 && threadIdx.x < 32)
                issue_group<S>(&bars[G & 1], oth_s, own_s, a, ty, y0, z + 2, 1, (j + 3) & 3, z + 1, (j + 1) & 1);
            const S *Om = oth_s + (size_t)((j & 3) * 3) * (ty + 2) * Lh;        // plane z-1
            const S *O0 = oth_s + (size_t)(((j + 1) & 3) * 3) * (ty + 2) * Lh;  // plane z
            const S *Op = oth_s + (size_t)(((j + 2) & 3) * 3) * (ty + 2) * Lh;  // plane z+1
            const S *W = own_s + (size_t)((j & 1) * 3) * ty * Lh;               // own plane z
            const size_t cs = (size_t)(ty + 2) * Lh;                            // component stride (other)
            const size_t ws = (size_t)ty * Lh;                                  // component stride (own)
            for (int it = threadIdx.x; it < items; it += kBlock) {
                const int yl = (int)a.div_nxv.div((uint32_t)it);
                const int xh0 = (it - yl * nxv) * V;
                const int y = y0 + yl;
                const uint32_t p = (uint32_t)(y + z + c) & 1u;
                const int xe = p ? ((xh0 + V == Lh) ? 0 : xh0 + V) : ((xh0 == 0) ? Lh - 1 : xh0 - 1);
                VT s[3], o[3], nym[3], nyp[3], nzm[3], nzp[3];
                C ed[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const S *r0 = O0 + q * cs + (size_t)(yl + 1) * Lh;
                    s[q] = *reinterpret_cast<const VT *>(W + q * ws + (size_t)yl * Lh + xh0);
                    o[q] = *reinterpret_cast<const VT *>(r0 + xh0);
                    nym[q] = *reinterpret_cast<const VT *>(r0 - Lh + xh0);
                    nyp[q] = *reinterpret_cast<const VT *>(r0 + Lh + xh0);
                    nzm[q] = *reinterpret_cast<const VT *>(Om + q * cs + (size_t)(yl + 1) * Lh + xh0);
                    nzp[q] = *reinterpret_cast<const VT *>(Op + q * cs + (size_t)(yl + 1) * Lh + xh0);
                    ed[q] = to_c(r0[xe]);
                }
                const uint32_t site0 = (uint32_t)((z * Ly + y) * Lx + 2 * xh0) + p;
                if (update_item<P, V, MEAS>(s, o, nym, nyp, nzm, nzp, ed, p, site0, c, a, J, K, ex, ey, ez, beta,
                                            accE, accX, accY, accZ, nacc)) {
                    const size_t gi = ((size_t)z * Ly + y) * Lh + xh0;
#pragma unroll
                    for (int q = 0; q < 3; ++q) *reinterpret_cast<VT *>(own_g[q] + gi) = s[q];
                }
            }
            __syncthreads();  // every thread is done with the slots the next group overwrites
        }
    }
    if (abort) {
        if (threadIdx.x == 0) atomicExch(&a.acc->error, 1);
        // the group that timed out may still land: give it one more bounded wait
        mbar_wait_bounded(&bars[G & 1], (G >> 1) & 1);
        __syncthreads();
    }
    write_partials<C, MEAS>(a, accE, accX, accY, accZ, nacc);
}

// ----------------------------------------------------------------- table pass
// One colour pass over renumbered sites [begin, end) with a neighbour table.
// Neighbours sum in stored order; padding points at a zero dummy spin.
template <int P, bool MEAS>
__global__ void __launch_bounds__(kBlock) table_pass_kernel(const PassArgs a) {
    using S = typename Tr<P>::S;
    using C = typename Tr<P>::C;
    using S4 = Vec<S, 4>;
    S4 *spins = reinterpret_cast<S4 *>(a.spins4);
    C J, K, ex, ey, ez, beta;
    load_params(a, J, K, ex, ey, ez, beta);
    C accE = C(0), accX = C(0), accY = C(0), accZ = C(0);
    unsigned nacc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = a.begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.end; i += stride) {
        C hx = C(0), hy = C(0), hz = C(0);
        C lx = C(0), ly = C(0), lz = C(0);
        for (int k = 0; k < a.width; ++k) {
            const int32_t j = __ldg(a.nbr + (int64_t)k * a.n_pad + i);
            const S4 n = spins[j];
            const C nx = to_c(n.v[0]), ny = to_c(n.v[1]), nz = to_c(n.v[2]);
            hx += nx;
            hy += ny;
            hz += nz;
            if (MEAS && j < a.colour_begin) {
                lx += nx;
                ly += ny;
                lz += nz;
            }
        }
        S4 s = spins[i];
        C sx = to_c(s.v[0]), sy = to_c(s.v[1]), sz = to_c(s.v[2]);
        C tx, ty, tz, u;
        if constexpr (P == HS_FP64)
            draw_trial<P>(__ldg(a.nat + i), a.sweep, (uint32_t)a.colour, a.replica, a.key0, a.key1, tx, ty, tz, u);
        else
            draw_trial_rank<P>((uint32_t)(i - a.colour_begin), a.sweep, (uint32_t)a.colour, a.replica, a.key0,
                               a.key1, tx, ty, tz, u);
        if (metropolis<C>(sx, sy, sz, tx, ty, tz, hx, hy, hz, J, K, ex, ey, ez, beta, u).acc) {
            sx = tx;
            sy = ty;
            sz = tz;
            s.v[0] = to_store<S, C>(tx);
            s.v[1] = to_store<S, C>(ty);
            s.v[2] = to_store<S, C>(tz);
            spins[i] = s;
            ++nacc;
        }
        if (MEAS) {
            const C se = sx * ex + sy * ey + sz * ez;
            accE += -J * (sx * lx + sy * ly + sz * lz) - K * se * se;
            accX += sx;
            accY += sy;
            accZ += sz;
        }
    }
    write_partials<C, MEAS>(a, accE, accX, accY, accZ, nacc);
}

// ----------------------------------------------------------------- measure
// Standalone Eq. 1 / Eq. 2 of the current state in FP64: every site adds
// -J/2 S_i.h_i - K (S_i.e)^2, so each bond is counted once overall.
template <int P>
__global__ void __launch_bounds__(kBlock) sc_measure_kernel(const PassArgs a, const void *planes) {
    using S = typename Tr<P>::S;
    const S *pl = (const S *)planes;
    const int Lh = a.Lh, Ly = a.Ly, Lz = a.Lz;
    const int64_t plane = (int64_t)Lz * Ly * Lh;
    double accE = 0, accX = 0, accY = 0, accZ = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 2 * plane; t += stride) {
        const int c = (int)(t / plane);
        const int64_t idx = t - c * plane;
        const int xh = (int)(idx % Lh);
        const int64_t row = idx / Lh;
        const int y = (int)(row % Ly), z = (int)(row / Ly);
        const int p = (y + z + c) & 1;
        const S *me = pl + (int64_t)(3 * c) * plane;
        const S *ot = pl + (int64_t)(3 * (1 - c)) * plane;
        const int xm = p ? xh : (xh == 0 ? Lh - 1 : xh - 1);
        const int xp = p ? (xh == Lh - 1 ? 0 : xh + 1) : xh;
        const int ym = (y == 0) ? Ly - 1 : y - 1, yp = (y == Ly - 1) ? 0 : y + 1;
        const int zm = (z == 0) ? Lz - 1 : z - 1, zp = (z == Lz - 1) ? 0 : z + 1;
        const int64_t nb[6] = {row * Lh + xm,
                               row * Lh + xp,
                               ((int64_t)z * Ly + ym) * Lh + xh,
                               ((int64_t)z * Ly + yp) * Lh + xh,
                               ((int64_t)zm * Ly + y) * Lh + xh,
                               ((int64_t)zp * Ly + y) * Lh + xh};
        double s[3], h[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < 3; ++q) {
            s[q] = (double)to_c(me[q * plane + idx]);
            for (int k = 0; k < 6; ++k) h[q] += (double)to_c(ot[q * plane + nb[k]]);
        }
        const double se = s[0] * a.e[0] + s[1] * a.e[1] + s[2] * a.e[2];
        accE += -0.5 * a.J * (s[0] * h[0] + s[1] * h[1] + s[2] * h[2]) - a.K * se * se;
        accX += s[0];
        accY += s[1];
        accZ += s[2];
    }
    write_partials<double, true>(a, accE, accX, accY, accZ, 0u);
}

template <int P>
__global__ void __launch_bounds__(kBlock) table_measure_kernel(const PassArgs a, int64_t n_present) {
    using S = typename Tr<P>::S;
    using S4 = Vec<S, 4>;
    const S4 *spins = reinterpret_cast<const S4 *>(a.spins4);
    double accE = 0, accX = 0, accY = 0, accZ = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_present; i += stride) {
        double h[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < a.width; ++k) {
            const S4 n = spins[a.nbr[(int64_t)k * a.n_pad + i]];
            for (int q = 0; q < 3; ++q) h[q] += (double)to_c(n.v[q]);
        }
        const S4 sv = spins[i];
        const double s0 = to_c(sv.v[0]), s1 = to_c(sv.v[1]), s2 = to_c(sv.v[2]);
        const double se = s0 * a.e[0] + s1 * a.e[1] + s2 * a.e[2];
        accE += -0.5 * a.J * (s0 * h[0] + s1 * h[1] + s2 * h[2]) - a.K * se * se;
        accX += s0;
        accY += s1;
        accZ += s2;
    }
    write_partials<double, true>(a, accE, accX, accY, accZ, 0u);
}

// ----------------------------------------------------------------- init / layout
template <int P>
__global__ void sc_init_kernel(void *planes, int Lx, int Ly, int Lz, int Lh, int mode, double e0, double e1,
                               double e2, uint32_t k0, uint32_t k1, uint32_t replica) {
    using S = typename Tr<P>::S;
    S *pl = (S *)planes;
    const int64_t plane = (int64_t)Lz * Ly * Lh;
    const int64_t n = (int64_t)Lx * Ly * Lz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % Lx);
        const int64_t row = i / Lx;
        const int y = (int)(row % Ly), z = (int)(row / Ly);
        const int c = (x + y + z) & 1;
        const int64_t idx = row * Lh + (x >> 1);
        double v[3] = {e0, e1, e2};
        if (mode == HS_INIT_RANDOM) {
            const uint4 w = philox10(make_uint4((uint32_t)i, 0u, kTagInit << 24, replica), k0, k1);
            sphere_fp64(w, v[0], v[1], v[2]);
        }
        for (int q = 0; q < 3; ++q) pl[(int64_t)(3 * c + q) * plane + idx] = store_from_double<S>(v[q]);
    }
}

template <int P>
__global__ void table_init_kernel(void *spins4, const uint32_t *nat, int64_t n_present, int mode, double e0,
                                  double e1, double e2, uint32_t k0, uint32_t k1, uint32_t replica) {
    using S = typename Tr<P>::S;
    using S4 = Vec<S, 4>;
    S4 *sp = reinterpret_cast<S4 *>(spins4);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_present;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v[3] = {e0, e1, e2};
        if (mode == HS_INIT_RANDOM) {
            const uint4 w = philox10(make_uint4(nat[i], 0u, kTagInit << 24, replica), k0, k1);
            sphere_fp64(w, v[0], v[1], v[2]);
        }
        S4 s;
        s.v[0] = store_from_double<S>(v[0]);
        s.v[1] = store_from_double<S>(v[1]);
        s.v[2] = store_from_double<S>(v[2]);
        s.v[3] = store_from_double<S>(0.0);
        sp[i] = s;
    }
}

template <int P>
__global__ void sc_convert_kernel(void *planes, double *xyz, int Lx, int Ly, int Lz, int Lh, int to_layout) {
    using S = typename Tr<P>::S;
    S *pl = (S *)planes;
    const int64_t plane = (int64_t)Lz * Ly * Lh;
    const int64_t n = (int64_t)Lx * Ly * Lz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % Lx);
        const int64_t row = i / Lx;
        const int y = (int)(row % Ly), z = (int)(row / Ly);
        const int c = (x + y + z) & 1;
        const int64_t idx = row * Lh + (x >> 1);
        for (int q = 0; q < 3; ++q) {
            S *d = pl + (int64_t)(3 * c + q) * plane + idx;
            if (to_layout)
                *d = store_from_double<S>(xyz[3 * i + q]);
            else
                xyz[3 * i + q] = (double)to_c(*d);
        }
    }
}

template <int P>
__global__ void table_convert_kernel(void *spins4, const uint32_t *nat, int64_t n_present, double *xyz,
                                     int to_layout) {
    using S = typename Tr<P>::S;
    using S4 = Vec<S, 4>;
    S4 *sp = reinterpret_cast<S4 *>(spins4);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_present;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t site = nat[i];
        if (to_layout) {
            S4 s;
            s.v[0] = store_from_double<S>(xyz[3 * site]);
            s.v[1] = store_from_double<S>(xyz[3 * site + 1]);
            s.v[2] = store_from_double<S>(xyz[3 * site + 2]);
            s.v[3] = store_from_double<S>(0.0);
            sp[i] = s;
        } else {
            const S4 s = sp[i];
            xyz[3 * site] = (double)to_c(s.v[0]);
            xyz[3 * site + 1] = (double)to_c(s.v[1]);
            xyz[3 * site + 2] = (double)to_c(s.v[2]);
        }
    }
}

inline int grid_for(int64_t n, int cap = 152 * 16) {
    int64_t g = (n + kBlock - 1) / kBlock;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

template <int P, int V>
cudaError_t launch_sc_v(const PassArgs &a, int n_blocks, cudaStream_t s, bool meas, bool pf) {
    if (pf) {
        if (meas)
            sc_pass_kernel<P, V, true, true><<<n_blocks, kBlock, 0, s>>>(a);
        else
            sc_pass_kernel<P, V, false, true><<<n_blocks, kBlock, 0, s>>>(a);
    } else {
        if (meas)
            sc_pass_kernel<P, V, true, false><<<n_blocks, kBlock, 0, s>>>(a);
        else
            sc_pass_kernel<P, V, false, false><<<n_blocks, kBlock, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <int P, int V>
cudaError_t launch_staged_v(const Layout &L, const PassArgs &a, cudaStream_t s, bool meas) {
    const size_t smem = staged_smem_bytes(P, L.ty, L.Lh);
    if (meas)
        sc_staged_kernel<P, V, true><<<L.grid, kBlock, smem, s>>>(a);
    else
        sc_staged_kernel<P, V, false><<<L.grid, kBlock, smem, s>>>(a);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_pass_p(const Layout &L, const PassArgs &a, int n_blocks, cudaStream_t s) {
    const bool meas = a.accumulate != 0;
    if (L.kernel == kStaged) {
        switch (L.vec) {
        case 1: return launch_staged_v<P, 1>(L, a, s, meas);
        case 2: return launch_staged_v<P, 2>(L, a, s, meas);
        case 4: if constexpr (P != HS_FP64) return launch_staged_v<P, 4>(L, a, s, meas); break;
        case 8: if constexpr (P == HS_FP16) return launch_staged_v<P, 8>(L, a, s, meas); break;
        default: break;
        }
        return cudaErrorInvalidValue;
    }
    if (L.kernel == kStencil) {
        switch (L.vec) {
        case 1: return launch_sc_v<P, 1>(a, n_blocks, s, meas, L.prefetch);
        case 2: return launch_sc_v<P, 2>(a, n_blocks, s, meas, L.prefetch);
        case 4: if constexpr (P != HS_FP64) return launch_sc_v<P, 4>(a, n_blocks, s, meas, L.prefetch); break;
        case 8: if constexpr (P == HS_FP16) return launch_sc_v<P, 8>(a, n_blocks, s, meas, L.prefetch); break;
        default: break;
        }
        return cudaErrorInvalidValue;
    }
    if (meas)
        table_pass_kernel<P, true><<<n_blocks, kBlock, 0, s>>>(a);
    else
        table_pass_kernel<P, false><<<n_blocks, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

template <int P>
const void *staged_ptr(int vec, bool meas) {
    switch (vec) {
    case 1: return meas ? (const void *)sc_staged_kernel<P, 1, true> : (const void *)sc_staged_kernel<P, 1, false>;
    case 2: return meas ? (const void *)sc_staged_kernel<P, 2, true> : (const void *)sc_staged_kernel<P, 2, false>;
    case 4:
        if constexpr (P != HS_FP64)
            return meas ? (const void *)sc_staged_kernel<P, 4, true> : (const void *)sc_staged_kernel<P, 4, false>;
        break;
    case 8:
        if constexpr (P == HS_FP16)
            return meas ? (const void *)sc_staged_kernel<P, 8, true> : (const void *)sc_staged_kernel<P, 8, false>;
        break;
    default: break;
    }
    return nullptr;
}

}  // namespace

size_t storage_size(int precision) {
    return precision == HS_FP64 ? 8 : (precision == HS_FP32 ? 4 : 2);
}

// 4 other-colour slabs of ty+2 rows and 2 own-colour slabs of ty rows, 3
// components each, rows of Lh elements.
size_t staged_smem_bytes(int precision, int ty, int Lh) {
    return (size_t)(4 * 3 * (ty + 2) + 2 * 3 * ty) * (size_t)Lh * storage_size(precision);
}

int staged_occupancy(int precision, int vec, size_t smem_bytes) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    if (smem_bytes + 2048 > (size_t)optin) return 0;
    int occ = 8;
    for (int m = 0; m < 2; ++m) {
        const void *k = nullptr;
        switch (precision) {
        case HS_FP64: k = staged_ptr<HS_FP64>(vec, m != 0); break;
        case HS_FP32: k = staged_ptr<HS_FP32>(vec, m != 0); break;
        case HS_FP16: k = staged_ptr<HS_FP16>(vec, m != 0); break;
        default: break;
        }
        if (!k) return 0;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes) != cudaSuccess)
            return 0;
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, kBlock, smem_bytes) != cudaSuccess) return 0;
        occ = std::min(occ, b);
    }
    return occ;
}

static int64_t pass_items(const Layout &L) {
    if (L.structured) return (int64_t)L.Lz * L.Ly * (L.Lh / L.vec);
    int64_t items = 0;
    for (int c = 0; c < L.n_colours; ++c)
        items = std::max<int64_t>(items, L.colour_begin[c + 1] - L.colour_begin[c]);
    return items;
}

template <int P, int V>
static const void *sc_ptr(bool meas, bool pf) {
    if (pf) return meas ? (const void *)sc_pass_kernel<P, V, true, true> : (const void *)sc_pass_kernel<P, V, false, true>;
    return meas ? (const void *)sc_pass_kernel<P, V, true, false> : (const void *)sc_pass_kernel<P, V, false, false>;
}

template <int P>
static const void *pass_kernel_ptr(const Layout &L, bool meas) {
    if (L.kernel == kStencil) {
        switch (L.vec) {
        case 1: return sc_ptr<P, 1>(meas, L.prefetch);
        case 2: return sc_ptr<P, 2>(meas, L.prefetch);
        case 4:
            if constexpr (P != HS_FP64) return sc_ptr<P, 4>(meas, L.prefetch);
            break;
        case 8:
            if constexpr (P == HS_FP16) return sc_ptr<P, 8>(meas, L.prefetch);
            break;
        default: break;
        }
        return nullptr;
    }
    return meas ? (const void *)table_pass_kernel<P, true> : (const void *)table_pass_kernel<P, false>;
}

int pass_occupancy(int precision, const Layout &L, int accumulate) {
    const void *k = nullptr;
    switch (precision) {
    case HS_FP64: k = pass_kernel_ptr<HS_FP64>(L, accumulate != 0); break;
    case HS_FP32: k = pass_kernel_ptr<HS_FP32>(L, accumulate != 0); break;
    case HS_FP16: k = pass_kernel_ptr<HS_FP16>(L, accumulate != 0); break;
    default: break;
    }
    int blocks = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, kBlock, 0) != cudaSuccess) return 1;
    return blocks > 0 ? blocks : 1;
}

// Persistent-style grid: resident CTAs per SM x SMs, never more CTAs than
// work items need.
int pass_blocks(int precision, const Layout &L, int n_sm, int blocks_per_sm) {
    (void)precision;
    return grid_for(pass_items(L), n_sm * std::max(blocks_per_sm, 1));
}

cudaError_t launch_pass(int precision, const Layout &L, const PassArgs &a, int n_blocks, cudaStream_t s) {
    switch (precision) {
    case HS_FP64: return launch_pass_p<HS_FP64>(L, a, n_blocks, s);
    case HS_FP32: return launch_pass_p<HS_FP32>(L, a, n_blocks, s);
    case HS_FP16: return launch_pass_p<HS_FP16>(L, a, n_blocks, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_measure(int precision, const Layout &L, const PassArgs &a, int n_blocks, cudaStream_t s) {
    if (L.structured) {
        switch (precision) {
        case HS_FP64: sc_measure_kernel<HS_FP64><<<n_blocks, kBlock, 0, s>>>(a, L.planes); break;
        case HS_FP32: sc_measure_kernel<HS_FP32><<<n_blocks, kBlock, 0, s>>>(a, L.planes); break;
        case HS_FP16: sc_measure_kernel<HS_FP16><<<n_blocks, kBlock, 0, s>>>(a, L.planes); break;
        default: return cudaErrorInvalidValue;
        }
    } else {
        switch (precision) {
        case HS_FP64: table_measure_kernel<HS_FP64><<<n_blocks, kBlock, 0, s>>>(a, L.n_present); break;
        case HS_FP32: table_measure_kernel<HS_FP32><<<n_blocks, kBlock, 0, s>>>(a, L.n_present); break;
        case HS_FP16: table_measure_kernel<HS_FP16><<<n_blocks, kBlock, 0, s>>>(a, L.n_present); break;
        default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_init(int precision, const Layout &L, int mode, const double e[3], uint32_t key0, uint32_t key1,
                        uint32_t replica, cudaStream_t s) {
    if (L.structured) {
        const int g = grid_for(L.n_sites);
        switch (precision) {
        case HS_FP64:
            sc_init_kernel<HS_FP64><<<g, kBlock, 0, s>>>(L.planes, L.Lx, L.Ly, L.Lz, L.Lh, mode, e[0], e[1], e[2],
                                                          key0, key1, replica);
            break;
        case HS_FP32:
            sc_init_kernel<HS_FP32><<<g, kBlock, 0, s>>>(L.planes, L.Lx, L.Ly, L.Lz, L.Lh, mode, e[0], e[1], e[2],
                                                          key0, key1, replica);
            break;
        case HS_FP16:
            sc_init_kernel<HS_FP16><<<g, kBlock, 0, s>>>(L.planes, L.Lx, L.Ly, L.Lz, L.Lh, mode, e[0], e[1], e[2],
                                                          key0, key1, replica);
            break;
        default: return cudaErrorInvalidValue;
        }
    } else {
        const int g = grid_for(L.n_present);
        switch (precision) {
        case HS_FP64:
            table_init_kernel<HS_FP64><<<g, kBlock, 0, s>>>(L.spins4, L.nat, L.n_present, mode, e[0], e[1], e[2],
                                                             key0, key1, replica);
            break;
        case HS_FP32:
            table_init_kernel<HS_FP32><<<g, kBlock, 0, s>>>(L.spins4, L.nat, L.n_present, mode, e[0], e[1], e[2],
                                                             key0, key1, replica);
            break;
        case HS_FP16:
            table_init_kernel<HS_FP16><<<g, kBlock, 0, s>>>(L.spins4, L.nat, L.n_present, mode, e[0], e[1], e[2],
                                                             key0, key1, replica);
            break;
        default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

static cudaError_t launch_convert(int precision, const Layout &L, double *xyz, int to_layout, cudaStream_t s) {
    if (L.structured) {
        const int g = grid_for(L.n_sites);
        switch (precision) {
        case HS_FP64: sc_convert_kernel<HS_FP64><<<g, kBlock, 0, s>>>(L.planes, xyz, L.Lx, L.Ly, L.Lz, L.Lh, to_layout); break;
        case HS_FP32: sc_convert_kernel<HS_FP32><<<g, kBlock, 0, s>>>(L.planes, xyz, L.Lx, L.Ly, L.Lz, L.Lh, to_layout); break;
        case HS_FP16: sc_convert_kernel<HS_FP16><<<g, kBlock, 0, s>>>(L.planes, xyz, L.Lx, L.Ly, L.Lz, L.Lh, to_layout); break;
        default: return cudaErrorInvalidValue;
        }
    } else {
        const int g = grid_for(L.n_present);
        switch (precision) {
        case HS_FP64: table_convert_kernel<HS_FP64><<<g, kBlock, 0, s>>>(L.spins4, L.nat, L.n_present, xyz, to_layout); break;
        case HS_FP32: table_convert_kernel<HS_FP32><<<g, kBlock, 0, s>>>(L.spins4, L.nat, L.n_present, xyz, to_layout); break;
        case HS_FP16: table_convert_kernel<HS_FP16><<<g, kBlock, 0, s>>>(L.spins4, L.nat, L.n_present, xyz, to_layout); break;
        default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_scatter(int precision, const Layout &L, const double *d_xyz, cudaStream_t s) {
    return launch_convert(precision, L, const_cast<double *>(d_xyz), 1, s);
}

cudaError_t launch_gather(int precision, const Layout &L, double *d_xyz, cudaStream_t s) {
    return launch_convert(precision, L, d_xyz, 0, s);
}

}  // namespace hs
