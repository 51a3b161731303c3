// Wavefront colour passes for the periodic sc lattice (Metropolis steps
// (i)-(iii) of arXiv 2106.11286 with the fused Eq. 1 / Eq. 2 sums): many
// passes, whole sweeps, in one persistent launch instead of one launch per
// pass.
//
// A pass needs, at plane z, the other colour's planes z-1, z, z+1 as the
// previous pass left them -- nothing more.  So the passes of a group of D
// follow each other through the lattice a few planes apart, and a plane that
// the first pass of the group brought into L2 is still there when the others
// reach it: HBM sees each spin about once per group instead of three times
// per pass, and no pass waits for the whole previous pass to drain.
//
// Work unit: (pass p, plane z, a range of work items of that colour plane).
// Units have tickets; CTA b runs tickets b, b + grid, b + 2 grid, ... in
// order.  Inside a group, pass d (0 <= d < D) visits its planes in the order
// k = 0, 1, ..., Lz-1 starting at plane p mod Lz (so consecutive passes start
// one plane apart and the periodic wrap never makes a pass wait for the end of
// the previous one), and plane-units are ordered by (k + lag d, d).  Unit
// (p, k) needs pass p-1 at positions k, k+1, k+2; with lag >= 3 those have
// smaller tickets, and so has everything of an earlier group.  Every CTA is
// resident (cooperative launch) and runs its tickets in order, so the
// smallest unfinished ticket can always proceed: no deadlock.
//
// A CTA is 15 compute warps and one control warp.  The control warp polls
// the per-plane completion counters for the next units (relaxed loads, then an
// acquire fence), publishes each through an mbarrier (up to four tickets
// ahead, so compute warps rarely wait and drift apart instead of stalling
// together), collects the compute warps' partial sums when they arrive on a
// second mbarrier, and releases a unit by adding 1 to its plane's counter
// after a release fence.  Counter
// cnt[z] reaches p U once passes 0 .. p-1 have finished plane z: a pass
// cannot start a plane before the previous pass finished it.  Every wait is
// bounded; a timeout latches the device error word and the CTA retires.
//
// Reductions: each CTA adds its units' partial sums per pass in ticket order
// (FP64, shared memory), flushed to its own slot when its tickets leave a
// group; a one-CTA kernel after the launch sums the slots of each sweep in a
// fixed order and updates the FP64 accumulator sweep by sweep.  The result is
// bit-reproducible for a given configuration.
#include <cuda_runtime.h>

#include "device.cuh"

namespace hs {
namespace {

constexpr int kWaveCompute = kWaveComputeWarps;
constexpr int kWaveCT = 32 * kWaveCompute;        // compute threads
constexpr int kWaveThreads = kWaveCT + 32;        // + the control warp
constexpr int kWaveMaxD = 32;                     // passes per group, at most
constexpr int kWaveRing = 4;                      // tickets a CTA holds ready or in progress

struct WaveUnit {
    uint32_t p, z, ib, ie;  // pass, array plane, item range within the colour plane
};

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Non-blocking test of one mbarrier phase (acquire at CTA scope when true).
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ WaveUnit wave_decode(const WaveArgs &w, uint32_t t) {
    const uint32_t Lz = (uint32_t)w.a.Lz;
    const uint32_t per_group = w.D * Lz * w.U;
    const uint32_t g = t / per_group;
    const uint32_t r = t - g * per_group;
    const uint32_t q = r / w.U;
    const uint32_t yb = r - q * w.U;
    const uint32_t e = (g < w.n_full) ? w.order_full[q] : w.order_last[q];
    WaveUnit u;
    u.p = g * w.D + (e >> 20);
    u.z = (u.p % Lz + (e & 0xFFFFFu)) % Lz;
    u.ib = yb * w.ipu;
    u.ie = min(u.ib + w.ipu, w.n_pi);
    return u;
}

// Control warp: keep up to kWaveRing tickets ready ahead of the oldest
// unreleased one, release finished ones, keep the per-pass sums.  One
// iteration: test which of the pending units the compute warps have finished
// (mbarrier, acquire at CTA scope) and poll the counters of the next tickets
// (relaxed loads); then one acq_rel fence at GPU scope serves both directions
// -- it orders the finished units' stores before the counter increments that
// follow it, and the polled counter values before the loads of the units made
// ready after it.
template <bool MEAS>
__device__ void wave_control(const WaveArgs &w, uint32_t n_mine, uint64_t *ready, uint64_t *done, WaveUnit *desc,
                             double (*part)[kWaveCompute][kPartials], double (*pacc)[kPartials],
                             volatile int *abort_flag) {
    const int lane = threadIdx.x & 31;
    const uint32_t G = gridDim.x;
    const uint32_t Lz = (uint32_t)w.a.Lz;
    uint32_t j_ready = 0, j_done = 0;
    uint32_t group = 0;  // group of the sums held in pacc
    auto flush = [&](uint32_t g) {
        const uint32_t Dg = (g < w.n_full) ? w.D : w.D_last;
        if (lane < kPartials)
            for (uint32_t d = 0; d < Dg; ++d) {
                w.slots[((size_t)(g * w.D + d) * G + blockIdx.x) * kPartials + lane] = pacc[d][lane];
                pacc[d][lane] = 0.0;
            }
        __syncwarp();
    };
    long long t_last = clock64();
    uint32_t idle = 0;
    WaveUnit cand = {0, 0, 0, 0};
    bool have_cand = false;
    while (j_done < n_mine) {
        // finished units, oldest first (lane 0 decides, the warp stays converged)
        uint32_t n_fin = 0;
        if (lane == 0)
            while (j_done + n_fin < j_ready &&
                   mbar_test(&done[(j_done + n_fin) % kWaveRing], ((j_done + n_fin) / kWaveRing) & 1))
                ++n_fin;
        n_fin = __shfl_sync(0xffffffffu, n_fin, 0);
        // the next ticket's inputs
        int ok = 0;
        if (j_ready < n_mine && j_ready - j_done < kWaveRing) {
            if (!have_cand) {
                cand = wave_decode(w, blockIdx.x + j_ready * G);
                have_cand = true;
            }
            ok = 1;
            if (cand.p > 0 && lane == 0) {
                const uint32_t need = cand.p * w.U;
                const uint32_t zm = (cand.z == 0) ? Lz - 1 : cand.z - 1;
                const uint32_t zp = (cand.z == Lz - 1) ? 0 : cand.z + 1;
                const uint32_t c0 = ld_relaxed_u32(w.cnt + zm), c1 = ld_relaxed_u32(w.cnt + cand.z),
                               c2 = ld_relaxed_u32(w.cnt + zp);
                ok = (int)(c0 - need) >= 0 && (int)(c1 - need) >= 0 && (int)(c2 - need) >= 0;
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
        }
        if (n_fin == 0 && !ok) {
            ++idle;
            int bad = 0, stop = 0;
            if (lane == 0) {
                stop = *abort_flag;
                bad = clock64() - t_last > kWaitCycles;
                if ((idle & 255u) == 0 && *(volatile int *)w.error != 0) bad = 1;
            }
            if (__shfl_sync(0xffffffffu, stop, 0)) break;
            if (__shfl_sync(0xffffffffu, bad, 0)) {
                if (lane == 0) {
                    *abort_flag = 1;
                    atomicExch(w.error, 1);
                }
                __syncwarp();
                break;
            }
            __nanosleep(20);
            continue;
        }
        t_last = clock64();
        idle = 0;
        if (lane == 0) asm volatile("fence.acq_rel.gpu;" ::: "memory");
        __syncwarp();
        for (uint32_t f = 0; f < n_fin; ++f, ++j_done) {
            const uint32_t slot = j_done % kWaveRing;
            const WaveUnit u = desc[slot];
            const bool skip = w.inject_skip && blockIdx.x == 0 && j_done == 0;  // test hook
            if (lane == 0 && !skip) asm volatile("red.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(w.cnt + u.z) : "memory");
            const uint32_t g = u.p / w.D;
            if (g != group) {
                flush(group);
                group = g;
            }
            if (lane < kPartials) {
                double v = 0.0;
#pragma unroll
                for (int q = 0; q < kWaveCompute; ++q) v += part[slot][q][lane];
                pacc[u.p - g * w.D][lane] += v;
            }
            __syncwarp();
        }
        if (ok) {
            if (lane == 0) {
                desc[j_ready % kWaveRing] = cand;
                mbar_arrive(&ready[j_ready % kWaveRing]);
            }
            __syncwarp();
            ++j_ready;
            have_cand = false;
        }
    }
    int stop = 0;
    if (lane == 0) stop = *abort_flag;
    if (!__shfl_sync(0xffffffffu, stop, 0)) flush(group);
}

template <int P, int V, bool MEAS>
__global__ void __launch_bounds__(kWaveThreads, 1) sc_wave_kernel(const WaveArgs w) {
    using S = typename Tr<P>::S;
    using C = typename Tr<P>::C;
    using VT = Vec<S, V>;
    __shared__ __align__(8) uint64_t ready[kWaveRing];
    __shared__ __align__(8) uint64_t done[kWaveRing];
    __shared__ WaveUnit desc[kWaveRing];
    __shared__ double part[kWaveRing][kWaveCompute][kPartials];
    __shared__ double pacc[kWaveMaxD][kPartials];
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int r = 0; r < kWaveRing; ++r) {
            mbar_init(&ready[r], 1);
            mbar_init(&done[r], kWaveCompute);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < kWaveMaxD * kPartials; i += blockDim.x) (&pacc[0][0])[i] = 0.0;
    __syncthreads();
    const uint32_t G = gridDim.x;
    const uint32_t n_mine = (w.n_tickets > blockIdx.x) ? (w.n_tickets - blockIdx.x + G - 1) / G : 0u;
    if (warp == kWaveCompute) {
        wave_control<MEAS>(w, n_mine, ready, done, desc, part, pacc, &abort_flag);
        return;
    }
    C J, K, ex, ey, ez, beta;
    load_params(w.a, J, K, ex, ey, ez, beta);
    const size_t plane = (size_t)w.a.Lz * w.a.Ly * w.a.Lh;
    S *const base = static_cast<S *>(w.planes);
    const uint32_t tc = threadIdx.x;
    for (uint32_t j = 0; j < n_mine; ++j) {
        if (!mbar_wait(&ready[j % kWaveRing], (j / kWaveRing) & 1, &abort_flag)) break;
        const WaveUnit u = desc[j % kWaveRing];
        const int c = (int)(u.p & 1u);
        PassArgs a = w.a;
        a.colour = c;
        a.sweep = w.sweep0 + (u.p >> 1);
        S *own_w[3];
        const S *own[3], *oth[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            own_w[q] = base + (size_t)(3 * c + q) * plane;
            own[q] = own_w[q];
            oth[q] = base + (size_t)(3 * (1 - c) + q) * plane;
        }
        SiteAcc<P> acc;
        const uint32_t t0 = u.z * w.n_pi;
        uint32_t i = u.ib + tc;
        if (i < u.ie) {  // split prefetch, as in the register stencil
            SplitItem<P, V> A;
            load_split_a<P, V>(a, t0 + i, own, oth, A);
            while (true) {
                VT nym[3], nyp[3];
                load_split_b<P, V>(A, oth, nym, nyp);
                C h[3][V];
                item_fields<P, V>(A.o, nym, nyp, A.nzm, A.nzp, A.ed, A.f.p, h);
                VT sv[3] = {A.s[0], A.s[1], A.s[2]};
                const uint32_t b0 = A.f.b0, site0 = A.f.site0, rank0 = A.f.rank0;
                const uint32_t in = i + kWaveCT;
                const bool more = in < u.ie;
                if (more) load_split_a<P, V>(a, t0 + in, own, oth, A);
                if (update_item_h<P, V, MEAS>(sv, h, site0, rank0, c, a, J, K, ex, ey, ez, beta, acc)) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) *reinterpret_cast<VT *>(own_w[q] + b0) = sv[q];
                }
                if (!more) break;
                i = in;
            }
        }
        // unit partials: warp shuffle -> this warp's slot
        float e = 0.f, x = 0.f, y = 0.f, z = 0.f;
        if (MEAS) {
            e = warp_sum((float)acc.E());
            x = warp_sum((float)acc.X());
            y = warp_sum((float)acc.Y());
            z = warp_sum((float)acc.Z());
        }
        const unsigned n = __reduce_add_sync(0xffffffffu, acc.n);
        if (lane == 0) {
            double *pp = part[j % kWaveRing][warp];
            pp[0] = e;
            pp[1] = x;
            pp[2] = y;
            pp[3] = z;
            pp[4] = (double)n;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&done[j % kWaveRing]);
    }
}

// Per-sweep totals of a launch: warp w sums sweeps w, w + 8, ... (both passes,
// CTA slots in ascending order, then a fixed shuffle tree) into the first slot
// of the sweep's first pass; thread 0 then applies them to the accumulator in
// sweep order, as the per-pass kernels' last CTA does.
__global__ void __launch_bounds__(256) wave_finalize_kernel(const WaveArgs w, int grid) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t n_sweeps = w.n_pass / 2;
    for (uint32_t s = warp; s < n_sweeps; s += 8) {
        double tot[kPartials] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int c = 0; c < 2; ++c)
            for (int b = lane; b < grid; b += 32)
#pragma unroll
                for (int q = 0; q < kPartials; ++q) tot[q] += w.slots[((size_t)(2 * s + c) * grid + b) * kPartials + q];
#pragma unroll
        for (int q = 0; q < kPartials; ++q) tot[q] = warp_sum(tot[q]);
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < kPartials; ++q) w.slots[(size_t)(2 * s) * grid * kPartials + q] = tot[q];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    DevAccum *A = w.acc;
    for (uint32_t s = 0; s < n_sweeps; ++s) {
        const double *tot = w.slots + (size_t)(2 * s) * grid * kPartials;
        A->accepted += tot[4];
        for (int q = 0; q < kPartials; ++q) A->sums[q] = tot[q];
        if (w.accumulate) {
            const double E = tot[0];
            const double mx = tot[1] / w.n_present, my = tot[2] / w.n_present, mz = tot[3] / w.n_present;
            const double m2 = mx * mx + my * my + mz * mz;
            const double am = sqrt(m2);
            const double me = fabs(mx * w.e[0] + my * w.e[1] + mz * w.e[2]);
            A->last[0] = E;
            A->last[1] = mx;
            A->last[2] = my;
            A->last[3] = mz;
            A->last[4] = am;
            A->last[5] = m2;
            A->last[6] = m2 * m2;
            A->last[7] = me;
            A->moments[HS_SUM_E] += E;
            A->moments[HS_SUM_E2] += E * E;
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
}

template <int P, int V>
const void *wave_ptr(bool meas) {
    return meas ? (const void *)sc_wave_kernel<P, V, true> : (const void *)sc_wave_kernel<P, V, false>;
}

const void *wave_kernel_ptr(int precision, int vec, bool meas) {
    if (precision == HS_FP32 && vec == 4) return wave_ptr<HS_FP32, 4>(meas);
    if (precision == HS_FP16 && vec == 8) return wave_ptr<HS_FP16, 8>(meas);
    return nullptr;
}

}  // namespace

int wave_occupancy(int precision, int vec) {
    int occ = 8;
    for (int m = 0; m < 2; ++m) {
        const void *k = wave_kernel_ptr(precision, vec, m != 0);
        if (!k) return 0;
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, kWaveThreads, 0) != cudaSuccess) return 0;
        occ = b < occ ? b : occ;
    }
    return occ;
}

cudaError_t launch_wave(int precision, int vec, const WaveArgs &w, int grid, cudaStream_t s) {
    const void *k = wave_kernel_ptr(precision, vec, w.accumulate != 0);
    if (!k) return cudaErrorInvalidValue;
    void *args[] = {const_cast<WaveArgs *>(&w)};
    return cudaLaunchCooperativeKernel(k, dim3((unsigned)grid), dim3(kWaveThreads), args, 0, s);
}

cudaError_t launch_wave_finalize(const WaveArgs &w, int grid, cudaStream_t s) {
    wave_finalize_kernel<<<1, 256, 0, s>>>(w, grid);
    return cudaGetLastError();
}

}  // namespace hs
