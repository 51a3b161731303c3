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
// per CTA and pass, in a ring of slot sets, one per sweep of a group of up to
// 64.  Within hs_sweep the passes only write slots; after each full group
// (and after the loop) a ring fold sums every sweep's slots in a fixed order
// (bit-reproducible), one CTA per sweep, and one thread applies the totals to
// the FP64 accumulator in sweep order, so no pass carries a serial reduction
// (a last-arriving CTA reducing inside the finishing pass cost 8 % at 256^3,
// a fold in the next sweep's first pass 5 %).  Single passes and standalone
// measurements keep the last-arriving-CTA form.
#include <cuda_fp16.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "device.cuh"

namespace hs {
namespace {

// Register stencil: every operand is loaded from global memory (L1/L2 serve
// the neighbour rows shared by adjacent work items).  Launch bounds of two
// resident CTAs per SM (128 registers) measured fastest on GB300.  Prefetch
// modes (PF):
//   0  none;
//   1  the loads of the thread's next work item are issued before the
//      current one is computed (two items in flight in registers, unrolled by
//      hand so no operand is copied);
//   2  split prefetch: as soon as the current item's local fields are summed
//      (its neighbour vectors are dead then), the next item's own row,
//      same-row and z-1 / z+1 rows -- the operands most often in DRAM -- are
//      loaded, so they travel during the current item's Metropolis
//      arithmetic; the y-1 / y+1 rows (the rows of neighbouring work items
//      of the same CTA, usually in L1 or L2) are loaded when an item is
//      taken up.
//   TEN adds the on-site anisotropy tensor term (built with PF = 0 only).
//   AX = 1: the FP32 variant chosen at launch when e = (0, 0, 1) exactly:
//   S.e = S_z, three packed instructions fewer per site pair, with no branch
//   in the item loop (a run-time branch there measured slower).
//   DIR = false: a variant with ascending passes only, whose item indices
//   never refer to PassArgs::rev (built for FP32 V = 4 and FP16 V = 8 with
//   PF = 0, the launches of lattices beyond 2^31 sites, where it measured
//   faster: 137 against 103-112 attempts/ns at 2048^3 FP32, while the
//   direction-capable code is faster at 256^3 to 1024^3).
template <int P, int V, bool MEAS, int PF, bool TEN = false, bool DIR = true, int AX = 0>
__global__ void __launch_bounds__(kBlock, 2) sc_pass_kernel(const PassArgs a) {
    pdl_enter();
    using S = typename Tr<P>::S;
    using C = typename Tr<P>::C;
    using VT = Vec<S, V>;
    const uint32_t n_items = (uint32_t)a.nz * a.Ly * (a.Lh / V);  // own planes only; < 2^31
    const int c = a.colour;
    C J, K, ex, ey, ez, beta;
    load_params(a, J, K, ex, ey, ez, beta);
    S *own_w[3] = {(S *)a.own[0], (S *)a.own[1], (S *)a.own[2]};
    const S *const own[3] = {(const S *)a.own[0], (const S *)a.own[1], (const S *)a.own[2]};
    const S *const oth[3] = {(const S *)a.oth[0], (const S *)a.oth[1], (const S *)a.oth[2]};
    SiteAcc<P> acc;
    const uint32_t stride = gridDim.x * blockDim.x;
    auto compute = [&](StencilItem<P, V> &it) {
        if (update_item<P, V, MEAS, TEN, AX>(it.s, it.o, it.nym, it.nyp, it.nzm, it.nzp, it.ed, it.p, it.site0, it.rank0,
                                             c, a, J, K, ex, ey, ez, beta, acc)) {
#pragma unroll
            for (int q = 0; q < 3; ++q) *reinterpret_cast<VT *>(own_w[q] + it.b0) = it.s[q];
        }
    };
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (PF == 0) {
        for (; t < n_items; t += stride) {
            StencilItem<P, V> it;
            load_item<P, V, false, DIR>(a, t, own, oth, it);
            compute(it);
        }
    } else if (PF == 2) {
        if (t < n_items) {
            SplitItem<P, V> A;
            load_split_a<P, V, false, DIR>(a, t, own, oth, A);
            while (true) {
                VT nym[3], nyp[3];
                load_split_b<P, V>(A, oth, nym, nyp);
                C h[3][V];
                item_fields<P, V>(A.o, nym, nyp, A.nzm, A.nzp, A.ed, A.f.p, h);
                VT sv[3] = {A.s[0], A.s[1], A.s[2]};
                const uint32_t b0 = A.f.b0, site0 = A.f.site0, rank0 = A.f.rank0;
                const uint32_t tn = t + stride;
                const bool more = tn < n_items;
                if (more) load_split_a<P, V, false, DIR>(a, tn, own, oth, A);  // the neighbour vectors are dead now
                if (update_item_h<P, V, MEAS, TEN, AX>(sv, h, site0, rank0, c, a, J, K, ex, ey, ez, beta, acc)) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) *reinterpret_cast<VT *>(own_w[q] + b0) = sv[q];
                }
                if (!more) break;
                t = tn;
            }
        }
    } else if (t < n_items) {
        StencilItem<P, V> A, B;
        load_item<P, V, false, DIR>(a, t, own, oth, A);
        while (true) {
            if (t + stride < n_items) load_item<P, V, false, DIR>(a, t + stride, own, oth, B);
            compute(A);
            t += stride;
            if (t >= n_items) break;
            if (t + stride < n_items) load_item<P, V, false, DIR>(a, t + stride, own, oth, A);
            compute(B);
            t += stride;
            if (t >= n_items) break;
        }
    }
    write_partials<C, MEAS>(a, acc.E(J, K), acc.X(), acc.Y(), acc.Z(), acc.n);
}

// ----------------------------------------------------------------- pipelined stencil pass
// The register stencil with one landing slot per thread in shared memory: the
// operands of the thread's next work item travel global -> shared through
// cp.async while the current item, already in registers, is computed.  Each
// thread thus keeps one item of loads in flight during its arithmetic without
// holding a second item in registers (which would not fit in 128 registers).
// Only the issuing thread reads its slot, so cp.async.wait_all alone orders
// the copy before the reads (no CTA barrier).  The slot is refilled after the
// reads of the previous item: a thread's shared-memory reads and its later
// cp.async go through the load/store pipe in program order, and the copy's
// shared-memory write lands only when its global data returns.
//
// Slot layout (structure of arrays over the CTA's threads, so a warp's
// accesses to one operand are consecutive): 18 vectors (own s[3], other
// colour o[3], y-1, y+1, z-1, z+1 rows) at [j][thread], then 3 edge words at
// [q][thread].  An edge word is one element, or for 2-byte storage the
// aligned 4-byte pair holding it (cp.async copies 4, 8 or 16 bytes).
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

template <int B>
__device__ __forceinline__ void cp_async_ca(uint32_t dst, const void *src) {
    static_assert(B == 4 || B == 8 || B == 16, "cp.async copies 4, 8 or 16 bytes");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(B) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int P>
struct PipeEdge {
    using S = typename Tr<P>::S;
    using W = typename std::conditional<(sizeof(S) >= 4), S, uint32_t>::type;
};

template <int P, int V>
struct PipeSlot {
    using S = typename Tr<P>::S;
    using VT = Vec<S, V>;
    using W = typename PipeEdge<P>::W;
    static constexpr size_t kVecBytes = 18u * kBlock * sizeof(VT);
    static constexpr size_t kBytes = kVecBytes + 3u * kBlock * sizeof(W);
};

// Issue the copies of work item t's operands into this thread's slot.
template <int P, int V>
__device__ __forceinline__ ItemOffsets pipe_issue(const PassArgs &a, uint32_t t, const typename Tr<P>::S *const (&own)[3],
                                                  const typename Tr<P>::S *const (&oth)[3], uint32_t slot_v,
                                                  uint32_t slot_e) {
    using S = typename Tr<P>::S;
    using Sl = PipeSlot<P, V>;
    constexpr int VB = (int)sizeof(typename Sl::VT);
    constexpr int WB = (int)sizeof(typename Sl::W);
    const uint32_t nxv = a.Lh / V;
    const uint32_t row = a.div_nxv.div(t);
    const uint32_t xv = t - row * nxv;
    const uint32_t z = a.div_ly.div(row);
    const uint32_t y = row - z * a.Ly;
    const ItemOffsets f = item_offsets<V>(a, y, z, xv);
    // for 2-byte storage the edge word starts at the even element of the pair
    const uint32_t bed_w = (sizeof(S) >= 4) ? f.bed : (f.bed & ~1u);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        cp_async_ca<VB>(slot_v + (uint32_t)((0 + q) * kBlock * VB), own[q] + f.b0);
        cp_async_ca<VB>(slot_v + (uint32_t)((3 + q) * kBlock * VB), oth[q] + f.b0);
        cp_async_ca<VB>(slot_v + (uint32_t)((6 + q) * kBlock * VB), oth[q] + f.bym);
        cp_async_ca<VB>(slot_v + (uint32_t)((9 + q) * kBlock * VB), oth[q] + f.byp);
        cp_async_ca<VB>(slot_v + (uint32_t)((12 + q) * kBlock * VB), oth[q] + f.bzm);
        cp_async_ca<VB>(slot_v + (uint32_t)((15 + q) * kBlock * VB), oth[q] + f.bzp);
        cp_async_ca<WB>(slot_e + (uint32_t)(q * kBlock * WB), oth[q] + bed_w);
    }
    cp_async_commit();
    return f;
}

// Read this thread's slot (after cp.async.wait_all) into registers.
template <int P, int V>
__device__ __forceinline__ void pipe_read(const typename PipeSlot<P, V>::VT *sv, const typename PipeSlot<P, V>::W *se,
                                          const ItemOffsets &f, StencilItem<P, V> &it) {
    using S = typename Tr<P>::S;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        it.s[q] = sv[(0 + q) * kBlock];
        it.o[q] = sv[(3 + q) * kBlock];
        it.nym[q] = sv[(6 + q) * kBlock];
        it.nyp[q] = sv[(9 + q) * kBlock];
        it.nzm[q] = sv[(12 + q) * kBlock];
        it.nzp[q] = sv[(15 + q) * kBlock];
        if constexpr (sizeof(S) >= 4) {
            it.ed[q] = to_c(se[q * kBlock]);
        } else {
            const uint32_t w = se[q * kBlock];
            const unsigned short bits = (unsigned short)((f.bed & 1u) ? (w >> 16) : (w & 0xffffu));
            it.ed[q] = to_c(__ushort_as_half(bits));
        }
    }
    it.b0 = f.b0;
    it.p = f.p;
    it.site0 = f.site0;
    it.rank0 = f.rank0;
}

template <int P, int V, bool MEAS, int AX = 0>
__global__ void __launch_bounds__(kBlock, 2) sc_pipe_kernel(const PassArgs a) {
    pdl_enter();
    using S = typename Tr<P>::S;
    using C = typename Tr<P>::C;
    using Sl = PipeSlot<P, V>;
    using VT = typename Sl::VT;
    using W = typename Sl::W;
    extern __shared__ __align__(16) unsigned char pipe_smem[];
    const uint32_t n_items = (uint32_t)a.Lz * a.Ly * (a.Lh / V);
    const int c = a.colour;
    C J, K, ex, ey, ez, beta;
    load_params(a, J, K, ex, ey, ez, beta);
    S *own_w[3] = {(S *)a.own[0], (S *)a.own[1], (S *)a.own[2]};
    const S *const own[3] = {(const S *)a.own[0], (const S *)a.own[1], (const S *)a.own[2]};
    const S *const oth[3] = {(const S *)a.oth[0], (const S *)a.oth[1], (const S *)a.oth[2]};
    const VT *sv = reinterpret_cast<const VT *>(pipe_smem) + threadIdx.x;
    const W *se = reinterpret_cast<const W *>(pipe_smem + Sl::kVecBytes) + threadIdx.x;
    const uint32_t slot_v = smem_addr(sv);
    const uint32_t slot_e = smem_addr(se);
    SiteAcc<P> acc;
    const uint32_t stride = gridDim.x * blockDim.x;
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_items) {
        ItemOffsets f = pipe_issue<P, V>(a, t, own, oth, slot_v, slot_e);
        while (true) {
            cp_async_wait_all();
            StencilItem<P, V> it;
            pipe_read<P, V>(sv, se, f, it);
            const uint32_t tn = t + stride;
            const bool more = tn < n_items;
            if (more) f = pipe_issue<P, V>(a, tn, own, oth, slot_v, slot_e);
            if (update_item<P, V, MEAS, false, AX>(it.s, it.o, it.nym, it.nyp, it.nzm, it.nzp, it.ed, it.p, it.site0,
                                                   it.rank0, c, a, J, K, ex, ey, ez, beta, acc)) {
#pragma unroll
                for (int q = 0; q < 3; ++q) *reinterpret_cast<VT *>(own_w[q] + it.b0) = it.s[q];
            }
            if (!more) break;
            t = tn;
        }
    }
    write_partials<C, MEAS>(a, acc.E(J, K), acc.X(), acc.Y(), acc.Z(), acc.n);
}

// ----------------------------------------------------------------- z-marching stencil pass
// Register stencil in slab order: the plane-slabs (ty rows of one z plane)
// of every y slab, z fastest, are split into equal contiguous ranges, one per
// CTA, so a CTA walks along z.  On small lattices it spreads a pass over more
// SMs than the grid-stride stencil, whose CTAs each take 256 work items (the
// autotuner picks it for the 16^3 FP64 lattice, which is bound by the FP64
// pipe of the SMs it runs on).  The other colour's rows at z and z+1, loaded
// as the z+-1 neighbours of plane z, come back from L1 for plane z+1; only
// the own plane z+1 and the other colour's plane z+2 are new, and thread 0
// asks the bulk-copy engine to prefetch those into L2 one plane ahead.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int P, int V, bool MEAS>
__global__ void __launch_bounds__(kBlock, 2) sc_march_kernel(const PassArgs a) {
    pdl_enter();
    using S = typename Tr<P>::S;
    using C = typename Tr<P>::C;
    using VT = Vec<S, V>;
    const int c = a.colour;
    const uint32_t Lh = a.Lh, Ly = a.Ly, Lz = a.Lz;
    const uint32_t ty = (uint32_t)a.ty;
    const uint32_t nxv = Lh / V;
    const uint32_t items = ty * nxv;
    const uint32_t n_slabs = Ly / ty;
    const uint64_t total = (uint64_t)n_slabs * Lz;  // plane-slabs
    const uint32_t q0 = (uint32_t)(total * blockIdx.x / gridDim.x);
    const uint32_t q1 = (uint32_t)(total * (blockIdx.x + 1) / gridDim.x);
    C J, K, ex, ey, ez, beta;
    load_params(a, J, K, ex, ey, ez, beta);
    S *own_w[3] = {(S *)a.own[0], (S *)a.own[1], (S *)a.own[2]};
    const S *const own[3] = {(const S *)a.own[0], (const S *)a.own[1], (const S *)a.own[2]};
    const S *const oth[3] = {(const S *)a.oth[0], (const S *)a.oth[1], (const S *)a.oth[2]};
    const uint32_t slab_bytes = ty * Lh * (uint32_t)sizeof(S);
    const bool pf = (slab_bytes % 16u) == 0u;
    SiteAcc<P> acc;
    for (uint32_t q = q0; q < q1; ++q) {
        const uint32_t slab = q / Lz;  // once per plane-slab: plain division is fine
        const uint32_t z = q - slab * Lz;
        const uint32_t y0 = slab * ty;
        if (pf && threadIdx.x == 0 && q + 1 < q1) {
            const uint32_t z1 = (z + 1 == Lz) ? 0 : z + 1;
            const uint32_t z2 = (z1 + 1 == Lz) ? 0 : z1 + 1;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                prefetch_l2(own[k] + ((size_t)z1 * Ly + y0) * Lh, slab_bytes);
                prefetch_l2(oth[k] + ((size_t)z2 * Ly + y0) * Lh, slab_bytes);
            }
        }
        for (uint32_t it = threadIdx.x; it < items; it += kBlock) {
            const uint32_t yl = a.div_nxv.div(it);
            const uint32_t xv = it - yl * nxv;
            StencilItem<P, V> item;
            load_item_at<P, V>(a, y0 + yl, z, xv, own, oth, item);
            if (update_item<P, V, MEAS>(item.s, item.o, item.nym, item.nyp, item.nzm, item.nzp, item.ed, item.p,
                                        item.site0, item.rank0, c, a, J, K, ex, ey, ez, beta, acc)) {
#pragma unroll
                for (int k = 0; k < 3; ++k) *reinterpret_cast<VT *>(own_w[k] + item.b0) = item.s[k];
            }
        }
    }
    write_partials<C, MEAS>(a, acc.E(J, K), acc.X(), acc.Y(), acc.Z(), acc.n);
}

// ----------------------------------------------------------------- table pass
// One colour pass over renumbered sites [begin, end) with a neighbour table.
// Neighbours sum in stored order; padding points at a zero dummy spin.
// Each site waits on two dependent gathers (its table row, then the
// neighbours' spins), so resident warps set the throughput: FP32 / FP16 fit
// five CTAs per SM in 48 registers without spilling (measured 51.8 -> 56.0
// attempts/ns on the FP32 bcc nanoparticle, 45.2 -> 48.0 on bcc 128^3,
// 65.0 -> 68.3 FP16); FP64 would spill and keeps four.
// TEN adds the on-site anisotropy tensor term.  PFL2 asks L2 for the next
// site's table row and own spin (prefetch instructions, no registers held)
// while the current site waits for its gathers: the table is streamed from
// DRAM once, so its first-hop latency is otherwise exposed at every site
// (measured 56.0 -> 62.4 attempts/ns on the FP32 bcc nanoparticle; slower
// for FP16 and for the 12-neighbour fcc table, so the autotuner decides).
// W > 0: a table of exactly W neighbours, unrolled: the W row entries load
// together, then the W gathers, then the sums in stored order (the same
// sums), so each site waits two round trips instead of 2 W.  It needs 64
// registers (four CTAs per SM): at 48 the compiler issues the gathers one
// after another again.  Measured on the FP32 bcc nanoparticle at W = 8:
// 65.9 -> 76.9 attempts/ns without PFL2 (74.9 with it); a version that also
// loaded the next site's row into registers measured lower.
template <int P, bool MEAS, bool TEN = false, bool PFL2 = false, int W = 0>
__global__ void __launch_bounds__(kBlock, P == HS_FP64 ? 1 : (W > 0 ? 4 : 5)) table_pass_kernel(const PassArgs a) {
    pdl_enter();
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
        if (PFL2 && i + stride < a.end) {
            for (int k = 0; k < a.width; ++k)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(a.nbr + (int64_t)k * a.n_pad + i + stride));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(spins + i + stride));
        }
        if constexpr (W > 0) {
            int32_t jj[W];
            S4 nn[W];
#pragma unroll
            for (int k = 0; k < W; ++k) jj[k] = __ldg(a.nbr + (int64_t)k * a.n_pad + i);
#pragma unroll
            for (int k = 0; k < W; ++k) nn[k] = spins[jj[k]];
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const C nx = to_c(nn[k].v[0]), ny = to_c(nn[k].v[1]), nz = to_c(nn[k].v[2]);
                hx += nx;
                hy += ny;
                hz += nz;
                if (MEAS && jj[k] < a.colour_begin) {
                    lx += nx;
                    ly += ny;
                    lz += nz;
                }
            }
        } else {
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
        }
        S4 s = spins[i];
        C sx = to_c(s.v[0]), sy = to_c(s.v[1]), sz = to_c(s.v[2]);
        C tx, ty, tz, u;
        bool accepted;
        if constexpr (P == HS_FP64) {
            float uf;
            draw_trial64(__ldg(a.nat + i), a.sweep, (uint32_t)a.colour, a.replica, a.key0, a.key1, a.sc_tab, tx, ty,
                         tz, u, uf);
            accepted = metropolis<C, TEN>(sx, sy, sz, tx, ty, tz, hx, hy, hz, J, K, ex, ey, ez, beta, u, uf, a.A).acc;
        } else {
            draw_trial_rank<P>((uint32_t)(i - a.colour_begin), a.sweep, (uint32_t)a.colour, a.replica, a.key0,
                               a.key1, tx, ty, tz, u);
            const Dots32<float> d =
                site_math32<float, TEN>(sx, sy, sz, tx, ty, tz, hx, hy, hz, J, K, ex, ey, ez, a.fA);
            accepted = accept32(d.dH, u, neg_beta_log2e(beta));
        }
        if (accepted) {
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
            if constexpr (TEN) {
                if constexpr (P == HS_FP64)
                    accE -= quad64(sx, sy, sz, a.A);
                else
                    accE -= quad32<float>(sx, sy, sz, a.fA);
            }
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
    pdl_enter();
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
        if (a.tensor) accE -= quad64(s[0], s[1], s[2], a.A);
        accX += s[0];
        accY += s[1];
        accZ += s[2];
    }
    write_partials<double, true>(a, accE, accX, accY, accZ, 0u);
}

template <int P>
__global__ void __launch_bounds__(kBlock) table_measure_kernel(const PassArgs a, int64_t n_present) {
    pdl_enter();
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
        if (a.tensor) accE -= quad64(s0, s1, s2, a.A);
        accX += s0;
        accY += s1;
        accZ += s2;
    }
    write_partials<double, true>(a, accE, accX, accY, accZ, 0u);
}

// ----------------------------------------------------------------- fold
// Ring fold, after the last pass of a group of sweeps: CTA i sums ring slot i
// (sweep i of the group) and writes that sweep's record (its totals and
// observables) ...
__global__ void __launch_bounds__(kBlock) fold_sum_kernel(const PassArgs a) {
    double tot[kPartials];
    slot_totals<kBlock>(a, blockIdx.x, tot);
    if (threadIdx.x == 0) {
        double o[8];
        sweep_observables(tot, a.n_present, a.e, o);
        double *rec = a.sweep_tot + (size_t)blockIdx.x * kSweepRecord;
#pragma unroll
        for (int q = 0; q < kPartials; ++q) rec[q] = tot[q];
#pragma unroll
        for (int q = 0; q < 8; ++q) rec[kPartials + q] = o[q];
    }
}

// ... and one thread applies the records to the accumulator in sweep order,
// the accumulator held in registers over the group.
__global__ void fold_apply_kernel(const PassArgs a, int n_slots) {
    if (threadIdx.x != 0) return;
    AccRegs R;
    R.load(a.acc);
    const bool acc = a.accumulate == 1;
    for (int i = 0; i < n_slots; ++i) {
        const double *rec = a.sweep_tot + (size_t)i * kSweepRecord;
        double tot[kPartials], o[8];
#pragma unroll
        for (int q = 0; q < kPartials; ++q) tot[q] = rec[q];
#pragma unroll
        for (int q = 0; q < 8; ++q) o[q] = rec[kPartials + q];
        apply_sweep(R, tot, o, acc, acc);
    }
    R.store(a.acc);
}

// ----------------------------------------------------------------- init / layout
// Own sites of a periodic sc lattice or z-slab (nz planes from global plane
// z0, stored from array plane z_off of Lz_arr): index i runs over them in
// natural order; the global natural index is i + z0 Ly Lx.
template <int P>
__global__ void sc_init_kernel(void *planes, int Lx, int Ly, int nz, int Lz_arr, int z_off, int z0, int Lh, int mode,
                               double e0, double e1, double e2, uint32_t k0, uint32_t k1, uint32_t replica) {
    using S = typename Tr<P>::S;
    S *pl = (S *)planes;
    const int64_t plane = (int64_t)Lz_arr * Ly * Lh;
    const int64_t n = (int64_t)Lx * Ly * nz;
    const int64_t glob0 = (int64_t)z0 * Ly * Lx;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % Lx);
        const int64_t r = i / Lx;
        const int y = (int)(r % Ly), z = (int)(r / Ly);
        const int c = (x + y + z + z0) & 1;
        const int64_t idx = (r + (int64_t)z_off * Ly) * Lh + (x >> 1);
        double v[3] = {e0, e1, e2};
        if (mode == HS_INIT_RANDOM) {
            // counter (index lo, index hi, tag 1, replica): an initial spin has no sweep
            const uint64_t gi = (uint64_t)(i + glob0);
            const uint4 w = philox10(make_uint4((uint32_t)gi, (uint32_t)(gi >> 32), kTagInit << 24, replica), k0, k1);
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
__global__ void sc_convert_kernel(void *planes, double *xyz, int Lx, int Ly, int nz, int Lz_arr, int z_off, int z0,
                                  int Lh, int to_layout) {
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
        for (int q = 0; q < 3; ++q) {
            S *d = pl + (int64_t)(3 * c + q) * plane + idx;
            if (to_layout)
                *d = store_from_double<S>(xyz[3 * i + q]);
            else
                xyz[3 * i + q] = (double)to_c(*d);
        }
    }
}

// Spins of selected sites (global natural indices, own sites of the lattice
// or slab), in FP64, for lattices too large to copy whole.
template <int P>
__global__ void sc_gather_kernel(const void *planes, int Lx, int Ly, int Lz_arr, int z_off, int z0, int Lh, int64_t n,
                                 const int64_t *sites, double *out) {
    using S = typename Tr<P>::S;
    const S *pl = (const S *)planes;
    const int64_t plane = (int64_t)Lz_arr * Ly * Lh;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = sites[t];
        const int x = (int)(i % Lx);
        const int64_t r = i / Lx;
        const int y = (int)(r % Ly), z = (int)(r / Ly);
        const int c = (x + y + z) & 1;
        const int64_t idx = ((int64_t)(z - z0 + z_off) * Ly + y) * Lh + (x >> 1);
        for (int q = 0; q < 3; ++q) out[3 * t + q] = (double)to_c(pl[(int64_t)(3 * c + q) * plane + idx]);
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

// Launch with programmatic stream serialisation (see pdl_enter).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int P, int V, int PF>
cudaError_t launch_sc_pf(const PassArgs &a, int n_blocks, cudaStream_t s, bool meas) {
    return meas ? launch_pdl(sc_pass_kernel<P, V, true, PF>, n_blocks, kBlock, 0, s, a)
                : launch_pdl(sc_pass_kernel<P, V, false, PF>, n_blocks, kBlock, 0, s, a);
}

// the precisions and widths that have the ascending-only stencil variant
template <int P, int V>
constexpr bool has_plain_variant() {
    return (P == HS_FP32 && V == 4) || (P == HS_FP16 && V == 8);
}

template <int P, int V>
cudaError_t launch_sc_v(const PassArgs &a, int n_blocks, cudaStream_t s, bool meas, int pf, bool ten, bool plain) {
    // e = (0, 0, 1): the AX = 1 variant of the direction-capable stencil (lattices up to 2^31 sites).  The
    // ascending-only variant beyond keeps the general products: with AX = 1 it measured 120 against
    // 132-137 attempts/ns at 2048^3.
    if constexpr (P == HS_FP32 && V == 4)
        if (a.zaxis && pf == 0 && !ten && !plain)
            return meas ? launch_pdl(sc_pass_kernel<P, V, true, 0, false, true, 1>, n_blocks, kBlock, 0, s, a)
                        : launch_pdl(sc_pass_kernel<P, V, false, 0, false, true, 1>, n_blocks, kBlock, 0, s, a);
    if constexpr (has_plain_variant<P, V>())
        if (plain && pf == 0 && !ten)
            return meas ? launch_pdl(sc_pass_kernel<P, V, true, 0, false, false>, n_blocks, kBlock, 0, s, a)
                        : launch_pdl(sc_pass_kernel<P, V, false, 0, false, false>, n_blocks, kBlock, 0, s, a);
    if (ten)
        return meas ? launch_pdl(sc_pass_kernel<P, V, true, 0, true>, n_blocks, kBlock, 0, s, a)
                    : launch_pdl(sc_pass_kernel<P, V, false, 0, true>, n_blocks, kBlock, 0, s, a);
    if (pf == 1) return launch_sc_pf<P, V, 1>(a, n_blocks, s, meas);
    if (pf == 2) return launch_sc_pf<P, V, 2>(a, n_blocks, s, meas);
    return launch_sc_pf<P, V, 0>(a, n_blocks, s, meas);
}

// FP16 V = 8 (the pipelined kernel the FP16 workloads run) has the S.e = S_z
// variant for e = (0, 0, 1), chosen here rather than per work item.
template <int P, int V>
constexpr bool has_pipe_ax_variant() { return P == HS_FP16 && V == 8; }

template <int P, int V>
cudaError_t launch_pipe_v(const PassArgs &a, int n_blocks, cudaStream_t s, bool meas) {
    const size_t smem = PipeSlot<P, V>::kBytes;
    if constexpr (has_pipe_ax_variant<P, V>())
        if (a.zaxis)
            return meas ? launch_pdl(sc_pipe_kernel<P, V, true, 1>, n_blocks, kBlock, smem, s, a)
                        : launch_pdl(sc_pipe_kernel<P, V, false, 1>, n_blocks, kBlock, smem, s, a);
    return meas ? launch_pdl(sc_pipe_kernel<P, V, true>, n_blocks, kBlock, smem, s, a)
                : launch_pdl(sc_pipe_kernel<P, V, false>, n_blocks, kBlock, smem, s, a);
}

template <int P, int V>
cudaError_t launch_march_v(const PassArgs &a, int n_blocks, cudaStream_t s, bool meas) {
    return meas ? launch_pdl(sc_march_kernel<P, V, true>, n_blocks, kBlock, 0, s, a)
                : launch_pdl(sc_march_kernel<P, V, false>, n_blocks, kBlock, 0, s, a);
}

template <int P>
cudaError_t launch_pass_p(const Layout &L, const PassArgs &a, int n_blocks, cudaStream_t s) {
    const bool meas = a.accumulate != 0;
    if (L.kernel == kMarch) {
        switch (L.vec) {
        case 1: return launch_march_v<P, 1>(a, n_blocks, s, meas);
        case 2: return launch_march_v<P, 2>(a, n_blocks, s, meas);
        case 4: if constexpr (P != HS_FP64) return launch_march_v<P, 4>(a, n_blocks, s, meas); break;
        case 8: if constexpr (P == HS_FP16) return launch_march_v<P, 8>(a, n_blocks, s, meas); break;
        default: break;
        }
        return cudaErrorInvalidValue;
    }
    if (L.kernel == kPipe) {
        switch (L.vec) {
        case 1: if constexpr (P != HS_FP16) return launch_pipe_v<P, 1>(a, n_blocks, s, meas); break;
        case 2: return launch_pipe_v<P, 2>(a, n_blocks, s, meas);
        case 4: if constexpr (P != HS_FP64) return launch_pipe_v<P, 4>(a, n_blocks, s, meas); break;
        case 8: if constexpr (P == HS_FP16) return launch_pipe_v<P, 8>(a, n_blocks, s, meas); break;
        default: break;
        }
        return cudaErrorInvalidValue;
    }
    if (L.kernel == kStencil) {
        switch (L.vec) {
        case 1: return launch_sc_v<P, 1>(a, n_blocks, s, meas, L.prefetch, L.tensor != 0, L.plain);
        case 2: return launch_sc_v<P, 2>(a, n_blocks, s, meas, L.prefetch, L.tensor != 0, L.plain);
        case 4: if constexpr (P != HS_FP64) return launch_sc_v<P, 4>(a, n_blocks, s, meas, L.prefetch, L.tensor != 0, L.plain); break;
        case 8: if constexpr (P == HS_FP16) return launch_sc_v<P, 8>(a, n_blocks, s, meas, L.prefetch, L.tensor != 0, L.plain); break;
        default: break;
        }
        return cudaErrorInvalidValue;
    }
    if (L.tensor)
        return meas ? launch_pdl(table_pass_kernel<P, true, true>, n_blocks, kBlock, 0, s, a)
                    : launch_pdl(table_pass_kernel<P, false, true>, n_blocks, kBlock, 0, s, a);
    if constexpr (P == HS_FP32)
        if (L.width == 8) {  // the unrolled 8-neighbour table (bcc, the nanoparticle's CSR)
            if (L.prefetch == 1)
                return meas ? launch_pdl(table_pass_kernel<P, true, false, true, 8>, n_blocks, kBlock, 0, s, a)
                            : launch_pdl(table_pass_kernel<P, false, false, true, 8>, n_blocks, kBlock, 0, s, a);
            return meas ? launch_pdl(table_pass_kernel<P, true, false, false, 8>, n_blocks, kBlock, 0, s, a)
                        : launch_pdl(table_pass_kernel<P, false, false, false, 8>, n_blocks, kBlock, 0, s, a);
        }
    if (L.prefetch == 1)
        return meas ? launch_pdl(table_pass_kernel<P, true, false, true>, n_blocks, kBlock, 0, s, a)
                    : launch_pdl(table_pass_kernel<P, false, false, true>, n_blocks, kBlock, 0, s, a);
    return meas ? launch_pdl(table_pass_kernel<P, true>, n_blocks, kBlock, 0, s, a)
                : launch_pdl(table_pass_kernel<P, false>, n_blocks, kBlock, 0, s, a);
}

}  // namespace

cudaError_t launch_fold(const PassArgs &a, int n_slots, cudaStream_t s) {
    if (n_slots < 1 || n_slots > kRingMax) return cudaErrorInvalidValue;
    fold_sum_kernel<<<n_slots, kBlock, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fold_apply_kernel<<<1, 32, 0, s>>>(a, n_slots);
    return cudaGetLastError();
}

size_t storage_size(int precision) {
    return precision == HS_FP64 ? 8 : (precision == HS_FP32 ? 4 : 2);
}

static int64_t pass_items(const Layout &L) {
    if (L.structured) return (int64_t)L.nz * L.Ly * (L.Lh / L.vec);
    int64_t items = 0;
    for (int c = 0; c < L.n_colours; ++c)
        items = std::max<int64_t>(items, L.colour_begin[c + 1] - L.colour_begin[c]);
    return items;
}

template <int P, int V, int PF>
static const void *sc_ptr_pf(bool meas) {
    return meas ? (const void *)sc_pass_kernel<P, V, true, PF> : (const void *)sc_pass_kernel<P, V, false, PF>;
}

template <int P, int V>
static const void *sc_ptr(bool meas, int pf, bool ten, bool plain) {
    if constexpr (has_plain_variant<P, V>())
        if (plain && pf == 0 && !ten)
            return meas ? (const void *)sc_pass_kernel<P, V, true, 0, false, false>
                        : (const void *)sc_pass_kernel<P, V, false, 0, false, false>;
    if (ten)
        return meas ? (const void *)sc_pass_kernel<P, V, true, 0, true> : (const void *)sc_pass_kernel<P, V, false, 0, true>;
    if (pf == 1) return sc_ptr_pf<P, V, 1>(meas);
    if (pf == 2) return sc_ptr_pf<P, V, 2>(meas);
    return sc_ptr_pf<P, V, 0>(meas);
}

template <int P, int V>
static const void *march_ptr(bool meas) {
    return meas ? (const void *)sc_march_kernel<P, V, true> : (const void *)sc_march_kernel<P, V, false>;
}

template <int P, int V>
static const void *pipe_ptr(bool meas) {
    return meas ? (const void *)sc_pipe_kernel<P, V, true> : (const void *)sc_pipe_kernel<P, V, false>;
}

// the S.e = S_z twin of the pipelined kernel for this precision and width, or nullptr
static const void *pipe_ax_ptr(int precision, int vec, bool meas) {
    if (precision == HS_FP16 && vec == 8)
        return meas ? (const void *)sc_pipe_kernel<HS_FP16, 8, true, 1> : (const void *)sc_pipe_kernel<HS_FP16, 8, false, 1>;
    return nullptr;
}

template <int P>
static size_t pipe_bytes(int vec) {
    switch (vec) {
    case 1: if constexpr (P != HS_FP16) return PipeSlot<P, 1>::kBytes; break;
    case 2: return PipeSlot<P, 2>::kBytes;
    case 4: if constexpr (P != HS_FP64) return PipeSlot<P, 4>::kBytes; break;
    case 8: if constexpr (P == HS_FP16) return PipeSlot<P, 8>::kBytes; break;
    default: break;
    }
    return 0;
}

// 0 when the pipelined stencil has no variant for this precision and width
// (a slot vector must be 4, 8 or 16 bytes).
size_t pipe_smem_bytes(int precision, int vec) {
    switch (precision) {
    case HS_FP64: return pipe_bytes<HS_FP64>(vec);
    case HS_FP32: return pipe_bytes<HS_FP32>(vec);
    case HS_FP16: return pipe_bytes<HS_FP16>(vec);
    default: return 0;
    }
}

template <int P>
static const void *pass_kernel_ptr(const Layout &L, bool meas) {
    if (L.kernel == kMarch) {
        switch (L.vec) {
        case 1: return march_ptr<P, 1>(meas);
        case 2: return march_ptr<P, 2>(meas);
        case 4:
            if constexpr (P != HS_FP64) return march_ptr<P, 4>(meas);
            break;
        case 8:
            if constexpr (P == HS_FP16) return march_ptr<P, 8>(meas);
            break;
        default: break;
        }
        return nullptr;
    }
    if (L.kernel == kPipe) {
        switch (L.vec) {
        case 1:
            if constexpr (P != HS_FP16) return pipe_ptr<P, 1>(meas);
            break;
        case 2: return pipe_ptr<P, 2>(meas);
        case 4:
            if constexpr (P != HS_FP64) return pipe_ptr<P, 4>(meas);
            break;
        case 8:
            if constexpr (P == HS_FP16) return pipe_ptr<P, 8>(meas);
            break;
        default: break;
        }
        return nullptr;
    }
    if (L.kernel == kStencil) {
        switch (L.vec) {
        case 1: return sc_ptr<P, 1>(meas, L.prefetch, L.tensor != 0, L.plain);
        case 2: return sc_ptr<P, 2>(meas, L.prefetch, L.tensor != 0, L.plain);
        case 4:
            if constexpr (P != HS_FP64) return sc_ptr<P, 4>(meas, L.prefetch, L.tensor != 0, L.plain);
            break;
        case 8:
            if constexpr (P == HS_FP16) return sc_ptr<P, 8>(meas, L.prefetch, L.tensor != 0, L.plain);
            break;
        default: break;
        }
        return nullptr;
    }
    if (L.tensor)
        return meas ? (const void *)table_pass_kernel<P, true, true> : (const void *)table_pass_kernel<P, false, true>;
    if constexpr (P == HS_FP32)
        if (L.width == 8) {
            if (L.prefetch == 1)
                return meas ? (const void *)table_pass_kernel<P, true, false, true, 8>
                            : (const void *)table_pass_kernel<P, false, false, true, 8>;
            return meas ? (const void *)table_pass_kernel<P, true, false, false, 8>
                        : (const void *)table_pass_kernel<P, false, false, false, 8>;
        }
    if (L.prefetch == 1)
        return meas ? (const void *)table_pass_kernel<P, true, false, true>
                    : (const void *)table_pass_kernel<P, false, false, true>;
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
    if (!k) return 1;
    size_t smem = 0;
    if (L.kernel == kPipe) {
        // opt in to the slots' dynamic shared memory and ask for a carveout
        // that holds two CTAs' slots, leaving the rest of the SM's 256 KB to
        // L1 (the neighbour rows shared by adjacent items)
        smem = pipe_smem_bytes(precision, L.vec);
        int dev = 0, per_sm = 0;
        if (smem == 0 || cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            per_sm <= 0)
            return 0;
        cudaFuncAttributes fa{};
        if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return 0;
        const size_t per_cta = smem + fa.sharedSizeBytes + 1024;  // + the driver's reserved 1 KB
        const int pct = std::min(100, (int)((200 * per_cta + (size_t)per_sm - 1) / (size_t)per_sm));
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
            cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess)
            return 0;
        // the launch may take the kernel's S.e = S_z twin (same slots and registers): the same opt-in
        if (const void *kx = pipe_ax_ptr(precision, L.vec, accumulate != 0))
            if (cudaFuncSetAttribute(kx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
                cudaFuncSetAttribute(kx, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess)
                return 0;
    }
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, kBlock, smem) != cudaSuccess) return 1;
    if (L.kernel == kPipe) return blocks;
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
            sc_init_kernel<HS_FP64><<<g, kBlock, 0, s>>>(L.planes, L.Lx, L.Ly, L.nz, L.Lz, L.slab ? 1 : 0, L.z0, L.Lh, mode, e[0], e[1], e[2],
                                                          key0, key1, replica);
            break;
        case HS_FP32:
            sc_init_kernel<HS_FP32><<<g, kBlock, 0, s>>>(L.planes, L.Lx, L.Ly, L.nz, L.Lz, L.slab ? 1 : 0, L.z0, L.Lh, mode, e[0], e[1], e[2],
                                                          key0, key1, replica);
            break;
        case HS_FP16:
            sc_init_kernel<HS_FP16><<<g, kBlock, 0, s>>>(L.planes, L.Lx, L.Ly, L.nz, L.Lz, L.slab ? 1 : 0, L.z0, L.Lh, mode, e[0], e[1], e[2],
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
        case HS_FP64:
            sc_convert_kernel<HS_FP64><<<g, kBlock, 0, s>>>(L.planes, xyz, L.Lx, L.Ly, L.nz, L.Lz, L.slab ? 1 : 0, L.z0,
                                                          L.Lh, to_layout);
            break;
        case HS_FP32:
            sc_convert_kernel<HS_FP32><<<g, kBlock, 0, s>>>(L.planes, xyz, L.Lx, L.Ly, L.nz, L.Lz, L.slab ? 1 : 0, L.z0,
                                                          L.Lh, to_layout);
            break;
        case HS_FP16:
            sc_convert_kernel<HS_FP16><<<g, kBlock, 0, s>>>(L.planes, xyz, L.Lx, L.Ly, L.nz, L.Lz, L.slab ? 1 : 0, L.z0,
                                                          L.Lh, to_layout);
            break;
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

cudaError_t launch_gather_sites(int precision, const Layout &L, int64_t n, const int64_t *d_sites, double *d_out,
                                cudaStream_t s) {
    const int g = grid_for(n);
    const int z_off = L.slab ? 1 : 0;
    switch (precision) {
    case HS_FP64:
        sc_gather_kernel<HS_FP64><<<g, kBlock, 0, s>>>(L.planes, L.Lx, L.Ly, L.Lz, z_off, L.z0, L.Lh, n, d_sites, d_out);
        break;
    case HS_FP32:
        sc_gather_kernel<HS_FP32><<<g, kBlock, 0, s>>>(L.planes, L.Lx, L.Ly, L.Lz, z_off, L.z0, L.Lh, n, d_sites, d_out);
        break;
    case HS_FP16:
        sc_gather_kernel<HS_FP16><<<g, kBlock, 0, s>>>(L.planes, L.Lx, L.Ly, L.Lz, z_off, L.z0, L.Lh, n, d_sites, d_out);
        break;
    default: return cudaErrorInvalidValue;
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
