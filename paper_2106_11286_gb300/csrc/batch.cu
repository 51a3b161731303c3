// Batched replicas in one persistent kernel: many periodic sc lattices of one
// precision (FP64, FP32 or FP16) and uneven size, each at its own beta,
// advanced sweep by sweep (Metropolis steps (i)-(iii) of arXiv 2106.11286,
// colour class by colour class) with the E / M moments of Eq. 1 / Eq. 2
// accumulated per member in FP64.
//
// Work split: the members' items (2 FP64 or 4 FP32 / FP16 sites of a row of one colour) are
// concatenated and cut into equal contiguous chunks, one per CTA; a chunk may
// cover several members, and each (CTA, member) piece is a segment with its
// own FP64 reduction slot, so the per-member sums are taken in a fixed order
// (bit-reproducible).  Colour passes are separated by a grid barrier (the
// launch is cooperative, so every CTA is resident); every wait on it is
// bounded and a timeout latches an error word that the host reports.  A
// sweep's per-member finalise runs inside the next barrier's wait.  Data
// written by other CTAs in the same launch is read L2-only (measured faster
// here than cached loads behind the barrier's GPU-scope fences).
#include <cuda_runtime.h>

#include "batch.h"
#include "device.cuh"

namespace hs {
namespace {

constexpr long long kBarrierCycles = 2000000000LL;  // about one second

// Grid-wide barrier on a monotonic 64-bit arrival count (zeroed before the
// launch): barrier k completes when the count reaches n_ctas (k + 1), so
// nothing is reset inside the kernel.  Arrival: the CTA's threads meet, and
// thread 0 fences (its CTA's earlier writes become visible GPU-wide first)
// and adds 1.  Wait: thread 0 polls the count with acquire loads, bounded;
// on a timeout it latches the error word.  The two halves are separate so a
// CTA can do work that needs no other CTA between arriving and waiting.
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void barrier_arrive(unsigned long long *cnt, bool skip_arrival) {
    __syncthreads();
    if (threadIdx.x == 0 && !skip_arrival) {  // (test hook: a skipped arrival runs every wait out)
        __threadfence();
        atomicAdd(cnt, 1ull);
    }
}

__device__ bool barrier_wait(const unsigned long long *cnt, unsigned long long target, int *error) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        if (ld_acquire_gpu(cnt) < target) {
            const long long t0 = clock64();
            for (uint32_t it = 0; ld_acquire_gpu(cnt) < target; ++it) {
                if (it > (1u << 30) || clock64() - t0 > kBarrierCycles) {
                    ok = 0;
                    atomicExch(error, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ PassArgs member_args(const BatchMember &m, int colour, uint32_t sweep) {
    PassArgs a{};
    a.Lx = m.Lx;
    a.Ly = m.Ly;
    a.Lz = m.Lz;
    a.Lh = m.Lh;
    a.div_nxv = m.div_nxv;
    a.div_ly = m.div_ly;
    a.colour = colour;
    a.fJ = m.fJ;
    a.fK = m.fK;
    a.fe[0] = m.fe[0];
    a.fe[1] = m.fe[1];
    a.fe[2] = m.fe[2];
    a.fbeta = m.fbeta;
    a.J = m.J;
    a.K = m.K;
    a.e[0] = m.e[0];
    a.e[1] = m.e[1];
    a.e[2] = m.e[2];
    a.beta = m.beta;
    a.sc_tab = m.sc_tab;
    a.zaxis = m.zaxis;
    a.key0 = m.key0;
    a.key1 = m.key1;
    a.replica = m.replica;
    a.sweep = sweep;
    return a;
}

// Add one sweep of a member, its five FP64 totals (E share, sum S, accepted
// moves), to its accumulator (one thread): the raw sums, Eq. 2's
// observables, and in the measurement phase their moments.
__device__ void member_apply_sweep(const BatchMember &m, const double (&tot)[kPartials], bool measured) {
    DevAccum *A = m.acc;
    A->accepted += tot[4];
#pragma unroll
    for (int q = 0; q < kPartials; ++q) A->sums[q] = tot[q];
    const double mx = tot[1] / m.n_present, my = tot[2] / m.n_present, mz = tot[3] / m.n_present;
    const double m2 = mx * mx + my * my + mz * mz;
    const double am = sqrt(m2);
    const double me = fabs(mx * m.e[0] + my * m.e[1] + mz * m.e[2]);
    A->last[0] = tot[0];
    A->last[1] = mx;
    A->last[2] = my;
    A->last[3] = mz;
    A->last[4] = am;
    A->last[5] = m2;
    A->last[6] = m2 * m2;
    A->last[7] = me;
    if (measured) {
        A->moments[HS_SUM_E] += tot[0];
        A->moments[HS_SUM_E2] += tot[0] * tot[0];
        A->moments[HS_SUM_ABSM] += am;
        A->moments[HS_SUM_M2] += m2;
        A->moments[HS_SUM_M4] += m2 * m2;
        A->moments[HS_SUM_MX] += mx;
        A->moments[HS_SUM_MY] += my;
        A->moments[HS_SUM_MZ] += mz;
        A->moments[HS_SUM_ABSME] += me;
        A->count += 1.0;
    }
}

// Finalise sweep s for the members this CTA owns, one warp per member: sum
// the member's segment slots of both colour passes in a fixed order and
// update its FP64 accumulator.  Reads slot parity s & 1, which sweep s + 2
// rewrites only after two more grid barriers that this CTA reaches after
// finishing here.
__device__ void finalize_sweep(const BatchArgs &b, int s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int par = s & 1;
    for (int r = blockIdx.x * (kBlock / 32) + warp; r < b.n_members; r += gridDim.x * (kBlock / 32)) {
        const BatchMember &m = b.members[r];
        double tot[kPartials] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int c = 0; c < 2; ++c)
            for (int si = m.seg_begin + lane; si < m.seg_end; si += 32)
#pragma unroll
                for (int q = 0; q < kPartials; ++q)
                    tot[q] += __ldcg(b.slots + (((size_t)par * 2 + c) * b.n_segs + si) * kPartials + q);
#pragma unroll
        for (int q = 0; q < kPartials; ++q) tot[q] = warp_sum(tot[q]);
        if (lane == 0) member_apply_sweep(m, tot, s >= b.n_equil);
    }
}

// One colour pass c of batch sweep s over this CTA's segments: every item of
// each segment (Metropolis steps (i)-(iii) of one member), then the
// segment's partial sums -> its FP64 slot.  CG: L2-only loads, for the
// persistent kernel, which reads data other CTAs wrote earlier in the same
// launch; a launch per pass loads through L1 (kernel boundaries keep it
// coherent).  PF = 2: split prefetch inside a segment, as in the
// single-lattice stencil: once the current item's local fields are summed,
// the next item's own row, same-row, z-1 and z+1 rows are loaded and travel
// during the current item's arithmetic.  PF = 0: one item of loads at a time.
template <int P>
constexpr int kBatchVec = (P == HS_FP64) ? 2 : 4;  // batch_vec()

// AX = 1: every member's easy axis is (0, 0, 1), so S.e = S_z (the FP32 and
// FP16 kernels' variant chosen at launch, as for a single lattice); AX = 2:
// every member's K is +0 as well, so the uniaxial term is left out.
template <int P, int PF, bool CG, int AX = 0>
__device__ __forceinline__ void batch_pass(const BatchArgs &b, int s, int c) {
    constexpr int V = kBatchVec<P>;
    using S = typename Tr<P>::S;
    using VT = Vec<S, V>;
    using C = typename Tr<P>::C;
    __shared__ double s_red[kBlock / 32][kPartials];
    // the current segment's member parameters and plane pointers (own colour
    // x, y, z, then the other colour's), read from shared memory where used
    // rather than held in registers
    __shared__ PassArgs s_args;
    __shared__ S *s_planes[6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int par = s & 1;  // slot parity this sweep writes
    for (int si = b.cta_seg[blockIdx.x]; si < b.cta_seg[blockIdx.x + 1]; ++si) {
        const BatchSeg sg = b.segs[si];
        const BatchMember &m = b.members[sg.member];
        // the previous segment's last use of s_args is before its reduction's barriers
        if (threadIdx.x == 0) {
            s_args = member_args(m, c, m.sweep0 + (uint32_t)s);
            const size_t plane = (size_t)m.Lz * m.Ly * m.Lh;
            S *const base = static_cast<S *>(m.planes);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                s_planes[q] = base + (size_t)(3 * c + q) * plane;
                s_planes[3 + q] = base + (size_t)(3 * (1 - c) + q) * plane;
            }
        }
        __syncthreads();
        const PassArgs &a = s_args;
        S *const(&own_w)[3] = *reinterpret_cast<S *const(*)[3]>(&s_planes[0]);
        const S *const(&own)[3] = *reinterpret_cast<const S *const(*)[3]>(&s_planes[0]);
        const S *const(&oth)[3] = *reinterpret_cast<const S *const(*)[3]>(&s_planes[3]);
        C J, K, ex, ey, ez, beta;
        load_params(a, J, K, ex, ey, ez, beta);
        SiteAcc<P> acc;
        if constexpr (PF == 2) {
            uint32_t t = sg.begin + threadIdx.x;
            if (t < sg.end) {
                SplitItem<P, V> A;
                load_split_a<P, V, CG>(a, t, own, oth, A);
                while (true) {
                    VT nym[3], nyp[3];
                    load_split_b<P, V, CG>(A, oth, nym, nyp);
                    C h[3][V];
                    item_fields<P, V>(A.o, nym, nyp, A.nzm, A.nzp, A.ed, A.f.p, h);
                    VT sv[3] = {A.s[0], A.s[1], A.s[2]};
                    const uint32_t b0 = A.f.b0, site0 = A.f.site0, rank0 = A.f.rank0;
                    const uint32_t tn = t + sg.stride;
                    const bool more = tn < sg.end;
                    if (more) load_split_a<P, V, CG>(a, tn, own, oth, A);  // the neighbour vectors are dead
                    if (update_item_h<P, V, true, false, AX>(sv, h, site0, rank0, c, a, J, K, ex, ey, ez, beta, acc)) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) *reinterpret_cast<VT *>(own_w[q] + b0) = sv[q];
                    }
                    if (!more) break;
                    t = tn;
                }
            }
        } else {
            for (uint32_t t = sg.begin + threadIdx.x; t < sg.end; t += sg.stride) {
                StencilItem<P, V> it;
                load_item<P, V, CG>(a, t, own, oth, it);
                if (update_item<P, V, true, false, AX>(it.s, it.o, it.nym, it.nyp, it.nzm, it.nzp, it.ed, it.p, it.site0,
                                                       it.rank0, c, a, J, K, ex, ey, ez, beta, acc)) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) *reinterpret_cast<VT *>(own_w[q] + it.b0) = it.s[q];
                }
            }
        }
        // segment partials: warp shuffle -> CTA (FP64) -> slot
        const C accE = warp_sum(acc.E(J, K));
        const C accX = warp_sum(acc.X());
        const C accY = warp_sum(acc.Y());
        const C accZ = warp_sum(acc.Z());
        const unsigned nacc = __reduce_add_sync(0xffffffffu, acc.n);
        if (lane == 0) {
            s_red[warp][0] = accE;
            s_red[warp][1] = accX;
            s_red[warp][2] = accY;
            s_red[warp][3] = accZ;
            s_red[warp][4] = (double)nacc;
        }
        __syncthreads();
        if (threadIdx.x < kPartials) {
            double t = 0.0;
            for (int w = 0; w < kBlock / 32; ++w) t += s_red[w][threadIdx.x];
            b.slots[(((size_t)par * 2 + c) * b.n_segs + si) * kPartials + threadIdx.x] = t;
        }
        __syncthreads();
    }
}

// The persistent schedule: every sweep and colour pass in one cooperative
// launch, passes separated by the bounded grid barrier.
template <int P, int PF, int AX = 0>
__global__ void __launch_bounds__(kBlock, 2) batch_kernel(const BatchArgs b) {
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(b.bar);
    for (int s = 0; s < b.n_total; ++s) {
        for (int c = 0; c < 2; ++c) {
            batch_pass<P, PF, true, AX>(b, s, c);
            const bool skip = b.inject_skip && blockIdx.x == 0 && s == 0 && c == 0;
            barrier_arrive(cnt, skip);
            // the previous sweep's finalise runs while this CTA waits for the
            // others to finish the first pass of this sweep
            if (c == 0 && s > 0) finalize_sweep(b, s - 1);
            const unsigned long long k = 2ull * (unsigned long long)s + (unsigned long long)c;
            if (!barrier_wait(cnt, (k + 1ull) * gridDim.x, b.error)) {  // uniform per CTA
                if (threadIdx.x == 0)
                    for (int r = 0; r < b.n_members; ++r) atomicExch(&b.members[r].acc->error, 1);
                return;
            }
        }
    }
    // the last sweep's finalise, after its last barrier
    if (b.n_total > 0) finalize_sweep(b, b.n_total - 1);
}

// The per-pass schedule: one launch per colour pass of every member, the
// launches chained by programmatic dependent launch (a launch's CTAs are
// scheduled as the previous one's retire and wait for its completion before
// touching memory).  Pass 0 of sweep s first finalises sweep s - 1, whose
// passes have completed by then; the slots it reads (parity (s-1) & 1) are
// rewritten only by pass 0 of sweep s + 1, two completed launches later.
template <int P, int PF, int AX = 0>
__global__ void __launch_bounds__(kBlock, 2) batch_pass_kernel(const BatchArgs b, int s, int c) {
    pdl_enter();
    if (c == 0 && s > 0) finalize_sweep(b, s - 1);
    batch_pass<P, PF, false, AX>(b, s, c);
}

// The last sweep's finalise of the per-pass schedule.
__global__ void __launch_bounds__(kBlock) batch_finalize_kernel(const BatchArgs b, int s) {
    pdl_enter();
    finalize_sweep(b, s);
}

// The resident schedule: one CTA per member, whose six planes are copied into
// the CTA's shared memory once and stay there for every sweep of the run
// (small lattices, up to the per-CTA shared memory).  A colour pass reads only
// the other colour, so a CTA barrier between passes is the only ordering the
// chain needs: no grid barrier, no global traffic between the first load and
// the final store.  The work items, loads and Metropolis update are those of
// the streaming kernels, on generic pointers into shared memory, so the chain
// is bit-identical; each sweep's FP64 totals (the two passes' CTA sums, in a
// fixed order) go straight to the member's accumulator.
constexpr int kResidentRing = 32;  // sweeps whose totals the resident kernel folds at once

// Fold sweeps s0 .. s0 + n - 1 of a resident member (totals in s_tot) into its
// accumulator, by one warp: lane k derives sweep k's observables (Eq. 2),
// then lane 0 adds them to the moments in sweep order, holding the
// accumulator in registers, as member_apply_sweep would sweep by sweep.
__device__ void resident_fold(const BatchMember &m, const double (*s_tot)[kPartials], double (*s_obs)[8], int s0,
                              int n, int n_equil) {
    const int lane = threadIdx.x & 31;
    if (lane < n) {
        double tot[kPartials], o[8];
#pragma unroll
        for (int q = 0; q < kPartials; ++q) tot[q] = s_tot[lane][q];
        sweep_observables(tot, m.n_present, m.e, o);
#pragma unroll
        for (int q = 0; q < 8; ++q) s_obs[lane][q] = o[q];
    }
    __syncwarp();
    if (lane == 0) {
        AccRegs R;
        R.load(m.acc);
        for (int k = 0; k < n; ++k) {
            const double *o = s_obs[k];
            R.accepted += s_tot[k][4];
            if (s0 + k >= n_equil) {
                R.moments[HS_SUM_E] += o[0];
                R.moments[HS_SUM_E2] += o[0] * o[0];
                R.moments[HS_SUM_ABSM] += o[4];
                R.moments[HS_SUM_M2] += o[5];
                R.moments[HS_SUM_M4] += o[6];
                R.moments[HS_SUM_MX] += o[1];
                R.moments[HS_SUM_MY] += o[2];
                R.moments[HS_SUM_MZ] += o[3];
                R.moments[HS_SUM_ABSME] += o[7];
                R.count += 1.0;
            }
        }
#pragma unroll
        for (int q = 0; q < kPartials; ++q) R.sums[q] = s_tot[n - 1][q];
#pragma unroll
        for (int q = 0; q < 8; ++q) R.last[q] = s_obs[n - 1][q];
        R.store(m.acc);
    }
    __syncwarp();
}

template <int P, int AX = 0>
__global__ void __launch_bounds__(kBlock, 2) batch_resident_kernel(const BatchArgs b) {
    constexpr int V = kBatchVec<P>;
    using S = typename Tr<P>::S;
    using VT = Vec<S, V>;
    using C = typename Tr<P>::C;
    extern __shared__ uint4 s_state[];
    __shared__ C s_red[kBlock / 32][kPartials];          // the warps' sums of one pass
    __shared__ double s_tot[kResidentRing][kPartials];   // per-sweep totals awaiting the fold
    __shared__ double s_obs[kResidentRing][8];
    __shared__ PassArgs s_args;
    const BatchMember &m = b.members[blockIdx.x];
    const uint32_t plane = (uint32_t)m.Lz * m.Ly * m.Lh;  // elements of one component plane; Lh % V == 0
    // six planes in 16-byte chunks (6 plane sizeof(S) is a multiple of 48 bytes)
    const uint32_t n16 = (uint32_t)(6u * (size_t)plane * sizeof(S) / 16u);
    const uint4 *g16 = static_cast<const uint4 *>(m.planes);
    for (uint32_t i = threadIdx.x; i < n16; i += kBlock) s_state[i] = __ldcg(g16 + i);
    if (threadIdx.x == 0) s_args = member_args(m, 0, m.sweep0);  // per pass only the colour and sweep change
    S *const st = reinterpret_cast<S *>(s_state);
    const uint32_t n_items = plane / V;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double sweep_tot = 0.0;  // warp 0, lane q < kPartials: quantity q of the current sweep
    for (int s = 0; s < b.n_total; ++s) {
        for (int c = 0; c < 2; ++c) {
            if (threadIdx.x == 0) {
                s_args.colour = c;
                s_args.sweep = m.sweep0 + (uint32_t)s;
            }
            __syncthreads();  // the parameters, and every store of the previous pass (or the initial copy)
            const PassArgs &a = s_args;
            S *own_w[3];
            const S *own[3], *oth[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                own_w[q] = st + (size_t)(3 * c + q) * plane;
                own[q] = own_w[q];
                oth[q] = st + (size_t)(3 * (1 - c) + q) * plane;
            }
            C J, K, ex, ey, ez, beta;
            load_params(a, J, K, ex, ey, ez, beta);
            SiteAcc<P> acc;
            for (uint32_t t = threadIdx.x; t < n_items; t += kBlock) {
                StencilItem<P, V> it;
                load_item<P, V>(a, t, own, oth, it);
                if (update_item<P, V, true, false, AX>(it.s, it.o, it.nym, it.nyp, it.nzm, it.nzp, it.ed, it.p, it.site0,
                                                       it.rank0, c, a, J, K, ex, ey, ez, beta, acc)) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) *reinterpret_cast<VT *>(own_w[q] + it.b0) = it.s[q];
                }
            }
            // the pass's sums: warp shuffle, then the warps' sums added in FP64 in warp order by warp 0, one
            // lane per quantity, into the sweep's totals
            const C accE = warp_sum(acc.E(J, K));
            const C accX = warp_sum(acc.X());
            const C accY = warp_sum(acc.Y());
            const C accZ = warp_sum(acc.Z());
            const unsigned nacc = __reduce_add_sync(0xffffffffu, acc.n);
            if (lane == 0) {
                s_red[warp][0] = accE;
                s_red[warp][1] = accX;
                s_red[warp][2] = accY;
                s_red[warp][3] = accZ;
                s_red[warp][4] = (C)nacc;  // an integer far below 2^24: exact
            }
            __syncthreads();
            if (warp == 0 && lane < kPartials)
                for (int w = 0; w < kBlock / 32; ++w) sweep_tot += (double)s_red[w][lane];
        }
        if (warp == 0) {
            const int slot = s % kResidentRing;
            if (lane < kPartials) s_tot[slot][lane] = sweep_tot;
            sweep_tot = 0.0;
            __syncwarp();
            if (slot == kResidentRing - 1 || s == b.n_total - 1)
                resident_fold(m, s_tot, s_obs, s - slot, slot + 1, b.n_equil);
        }
    }
    __syncthreads();
    uint4 *w16 = static_cast<uint4 *>(m.planes);
    for (uint32_t i = threadIdx.x; i < n16; i += kBlock) w16[i] = s_state[i];
}

// Zero every member's accepted-move counter (hs_batch_run's count covers its
// own sweeps): one launch for the whole batch.
__global__ void batch_reset_kernel(const BatchMember *members, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) members[i].acc->accepted = 0.0;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*kernel)(KArgs...), int grid, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace

namespace {
template <int P>
int occupancy_p(int prefetch) {
    int blocks = 0, blocks_pass = 0;
    const void *k = prefetch ? (const void *)batch_kernel<P, 2> : (const void *)batch_kernel<P, 0>;
    const void *kp = prefetch ? (const void *)batch_pass_kernel<P, 2> : (const void *)batch_pass_kernel<P, 0>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, kBlock, 0) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_pass, kp, kBlock, 0) != cudaSuccess) return 0;
    int occ = blocks < blocks_pass ? blocks : blocks_pass;
    if constexpr (P == HS_FP32 || P == HS_FP16) {  // the launch may take the axis variants: the grid must fit each
        const void *ks[4] = {
            prefetch ? (const void *)batch_kernel<P, 2, 1> : (const void *)batch_kernel<P, 0, 1>,
            prefetch ? (const void *)batch_pass_kernel<P, 2, 1> : (const void *)batch_pass_kernel<P, 0, 1>,
            prefetch ? (const void *)batch_kernel<P, 2, 2> : (const void *)batch_kernel<P, 0, 2>,
            prefetch ? (const void *)batch_pass_kernel<P, 2, 2> : (const void *)batch_pass_kernel<P, 0, 2>};
        for (const void *kx : ks) {
            int bx = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bx, kx, kBlock, 0) != cudaSuccess) return 0;
            occ = occ < bx ? occ : bx;
        }
    }
    return occ;
}

// the axis variant a batch takes: 0 general, 1 e = z for every member, 2 also K = +0 (FP32 and FP16)
inline int batch_ax(const BatchArgs &b) { return b.zaxis_all ? (b.kzero_all ? 2 : 1) : 0; }

// the axis twins serve FP32 and FP16 batches whose members all have e = (0, 0, 1)
template <int P>
constexpr bool batch_has_ax() { return P == HS_FP32 || P == HS_FP16; }

template <int P>
cudaError_t passes_p(const BatchArgs &b, int grid, cudaStream_t s, int prefetch) {
    for (int sw = 0; sw < b.n_total; ++sw)
        for (int c = 0; c < 2; ++c) {
            cudaError_t e = cudaSuccess;
            const int ax = batch_has_ax<P>() ? batch_ax(b) : 0;
            if constexpr (batch_has_ax<P>())
                if (ax == 2)
                    e = prefetch ? launch_chained(batch_pass_kernel<P, 2, 2>, grid, s, b, sw, c)
                                 : launch_chained(batch_pass_kernel<P, 0, 2>, grid, s, b, sw, c);
            if constexpr (batch_has_ax<P>())
                if (ax == 1)
                    e = prefetch ? launch_chained(batch_pass_kernel<P, 2, 1>, grid, s, b, sw, c)
                                 : launch_chained(batch_pass_kernel<P, 0, 1>, grid, s, b, sw, c);
            if (ax == 0)
                e = prefetch ? launch_chained(batch_pass_kernel<P, 2>, grid, s, b, sw, c)
                             : launch_chained(batch_pass_kernel<P, 0>, grid, s, b, sw, c);
            if (e != cudaSuccess) return e;
        }
    if (b.n_total > 0) return launch_chained(batch_finalize_kernel, grid, s, b, b.n_total - 1);
    return cudaSuccess;
}

template <int P>
size_t resident_limit_p() {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, batch_resident_kernel<P>) != cudaSuccess)
        return 0;
    return optin > (int)fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
}

template <int P, int AX>
cudaError_t resident_ax(const BatchArgs &b, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(batch_resident_kernel<P, AX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    batch_resident_kernel<P, AX><<<b.n_members, kBlock, smem, s>>>(b);
    return cudaGetLastError();
}

template <int P>
cudaError_t resident_p(const BatchArgs &b, size_t smem, cudaStream_t s) {
    if constexpr (batch_has_ax<P>()) {
        if (batch_ax(b) == 2) return resident_ax<P, 2>(b, smem, s);
        if (batch_ax(b) == 1) return resident_ax<P, 1>(b, smem, s);
    }
    return resident_ax<P, 0>(b, smem, s);
}

template <int P>
cudaError_t persistent_p(const BatchArgs &b, int grid, cudaStream_t s, int prefetch) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if constexpr (batch_has_ax<P>()) {
        if (batch_ax(b) == 2)
            return prefetch ? cudaLaunchKernelEx(&cfg, batch_kernel<P, 2, 2>, b)
                            : cudaLaunchKernelEx(&cfg, batch_kernel<P, 0, 2>, b);
        if (batch_ax(b) == 1)
            return prefetch ? cudaLaunchKernelEx(&cfg, batch_kernel<P, 2, 1>, b)
                            : cudaLaunchKernelEx(&cfg, batch_kernel<P, 0, 1>, b);
    }
    return prefetch ? cudaLaunchKernelEx(&cfg, batch_kernel<P, 2>, b) : cudaLaunchKernelEx(&cfg, batch_kernel<P, 0>, b);
}
}  // namespace

cudaError_t launch_batch_reset(const BatchArgs &b, cudaStream_t s) {
    if (b.n_members < 1) return cudaSuccess;
    batch_reset_kernel<<<(b.n_members + kBlock - 1) / kBlock, kBlock, 0, s>>>(b.members, b.n_members);
    return cudaGetLastError();
}

int batch_occupancy(int precision, int prefetch) {
    switch (precision) {
    case HS_FP64: return occupancy_p<HS_FP64>(prefetch);
    case HS_FP32: return occupancy_p<HS_FP32>(prefetch);
    case HS_FP16: return occupancy_p<HS_FP16>(prefetch);
    default: return 0;
    }
}

cudaError_t launch_batch_passes(int precision, const BatchArgs &b, int grid, cudaStream_t s, int prefetch) {
    switch (precision) {
    case HS_FP64: return passes_p<HS_FP64>(b, grid, s, prefetch);
    case HS_FP32: return passes_p<HS_FP32>(b, grid, s, prefetch);
    case HS_FP16: return passes_p<HS_FP16>(b, grid, s, prefetch);
    default: return cudaErrorInvalidValue;
    }
}

size_t batch_resident_limit(int precision) {
    switch (precision) {
    case HS_FP64: return resident_limit_p<HS_FP64>();
    case HS_FP32: return resident_limit_p<HS_FP32>();
    case HS_FP16: return resident_limit_p<HS_FP16>();
    default: return 0;
    }
}

cudaError_t launch_batch_resident(int precision, const BatchArgs &b, size_t smem, cudaStream_t s) {
    switch (precision) {
    case HS_FP64: return resident_p<HS_FP64>(b, smem, s);
    case HS_FP32: return resident_p<HS_FP32>(b, smem, s);
    case HS_FP16: return resident_p<HS_FP16>(b, smem, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch(int precision, const BatchArgs &b, int grid, cudaStream_t s, int prefetch) {
    switch (precision) {
    case HS_FP64: return persistent_p<HS_FP64>(b, grid, s, prefetch);
    case HS_FP32: return persistent_p<HS_FP32>(b, grid, s, prefetch);
    case HS_FP16: return persistent_p<HS_FP16>(b, grid, s, prefetch);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hs
