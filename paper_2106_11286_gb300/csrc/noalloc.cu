// Allocation-free sweep entry point: hs_sweep_sc_fp32_noalloc (see
// include/hs.h).  It runs the library's FP32 sc stencil colour pass with its
// fused reductions on a lattice the caller holds in device memory, and keeps
// the reduction scratch (per-CTA slots, accumulator, arrival counter) in the
// file-scope device array below instead of memory from cudaMalloc.
//
// Why: some callers cannot allocate device memory themselves -- a host
// framework whose caching allocator or fixed budget owns all device memory,
// or a latency-critical loop that cannot afford cudaMalloc's implicit
// device-wide synchronisation.  They pass their own buffers for the spins
// and the results; this file supplies the rest from static storage.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "hs_impl.h"

namespace {

constexpr int kMaxCtas = HS_NOALLOC_MAX_CTAS;
constexpr size_t kSlotBytes = (size_t)2 * kMaxCtas * hs::kPartials * sizeof(double);  // 2 colour passes
constexpr size_t kAccumOffset = (kSlotBytes + 255) / 256 * 256;
constexpr size_t kScratchBytes = kAccumOffset + (sizeof(hs::DevAccum) + 255) / 256 * 256;

// Shared by every call on a device and kept until the process exits; holds
// what the last call left in it.
static __device__ __align__(256) unsigned char hs_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch[kMaxDevices] = {};  // device address of the array, per device

int fail(int code, const std::string &msg) { return hs::set_last_error(code, msg); }

// Device address of the scratch array on the current device, looked up once
// per device (host code only sees a stand-in symbol, not a device address).
// The cached address belongs to the module as loaded in the device's
// current context; cudaDeviceReset unloads it, so after a reset the entry
// point must not be called again in this process.
int scratch_address(int dev, void **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, hs_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return fail(HS_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return HS_OK;
}

}  // namespace

extern "C" int hs_sweep_sc_fp32_noalloc(float *planes, const int32_t dims[3], const hs_params *p, double beta,
                                        uint64_t seed, uint32_t replica, uint64_t first_sweep, int64_t n_sweeps,
                                        double *d_out, void *cuda_stream) {
    if (!planes || !dims || !p || !d_out) return fail(HS_E_INVALID, "null argument");
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 2 || dims[a] % 2 != 0) return fail(HS_E_INVALID, "dims must be even and >= 2");
    if ((double)dims[0] * dims[1] * dims[2] >= 2147483647.0) return fail(HS_E_INVALID, "more than 2^31 - 1 sites");
    if (!(beta >= 0.0) || !std::isfinite(beta)) return fail(HS_E_INVALID, "beta must be finite and >= 0");
    if (n_sweeps < 0) return fail(HS_E_INVALID, "n_sweeps must be >= 0");
    const double en = std::sqrt(p->e[0] * p->e[0] + p->e[1] * p->e[1] + p->e[2] * p->e[2]);
    if (!(en > 0.0)) return fail(HS_E_INVALID, "easy axis must be non-zero");
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return fail(HS_E_DEVICE, "no device");
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(HS_E_CUDA, "cudaDeviceGetAttribute failed");
    void *scratch = nullptr;
    int st = scratch_address(dev, &scratch);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    hs::Layout L{};
    L.structured = true;
    L.kernel = hs::kStencil;
    L.n_colours = 2;
    L.Lx = dims[0];
    L.Ly = dims[1];
    L.Lz = dims[2];
    L.nz = dims[2];
    L.Lz_glob = dims[2];
    L.Lh = dims[0] / 2;
    L.vec = (L.Lh % 4 == 0) ? 4 : ((L.Lh % 2 == 0) ? 2 : 1);
    // the kernel moves vec floats per vector load and store, so every plane
    // (a multiple of vec floats from the base) must start on that boundary
    if ((uintptr_t)planes % (sizeof(float) * (size_t)L.vec) != 0)
        return fail(HS_E_INVALID, "planes must be aligned to " + std::to_string(4 * L.vec) +
                                      " bytes for this Lx (vector width " + std::to_string(L.vec) + ")");
    if ((uintptr_t)d_out % alignof(double) != 0) return fail(HS_E_INVALID, "d_out must be 8-byte aligned");
    // as a handle's automatic launch: no prefetch, the colour-1 pass descending (each pass starts on the
    // planes the previous one touched last, still in L2)
    L.prefetch = 0;
    L.n_sites = L.n_present = (int64_t)dims[0] * dims[1] * dims[2];
    L.planes = planes;
    const int occ = hs::pass_occupancy(HS_FP32, L, 1);
    const int grid = hs::pass_blocks(HS_FP32, L, n_sm, occ);
    if (grid > kMaxCtas) return fail(HS_E_INVALID, "launch needs more CTAs than the static scratch holds (1024)");

    double *slots = static_cast<double *>(scratch);
    hs::DevAccum *acc = reinterpret_cast<hs::DevAccum *>(static_cast<unsigned char *>(scratch) + kAccumOffset);
    // the array keeps the previous call's contents: zero the accumulator and
    // the arrival counter (the slots are written before they are read)
    if (cudaMemsetAsync(acc, 0, sizeof(hs::DevAccum), s) != cudaSuccess)
        return fail(HS_E_CUDA, "cudaMemsetAsync failed");

    hs::PassArgs a{};
    a.Lx = L.Lx;
    a.Ly = L.Ly;
    a.Lz = L.Lz;
    a.nz = L.nz;
    a.Lh = L.Lh;
    a.div_nxv = hs::FastDiv((uint32_t)(L.Lh / L.vec));
    a.div_ly = hs::FastDiv((uint32_t)L.Ly);
    a.n_colours = 2;
    a.J = p->J;
    a.K = p->K;
    for (int q = 0; q < 3; ++q) a.e[q] = p->e[q] / en;
    a.zaxis = (a.e[0] == 0.0 && a.e[1] == 0.0 && a.e[2] == 1.0) ? 1 : 0;
    a.beta = beta;
    a.fJ = (float)a.J;
    a.fK = (float)a.K;
    for (int q = 0; q < 3; ++q) a.fe[q] = (float)a.e[q];
    a.fbeta = (float)beta;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.replica = replica;
    a.partials = slots;
    a.n_blocks = grid;
    a.accumulate = 1;
    a.n_present = (double)L.n_present;
    a.acc = acc;
    const size_t plane = (size_t)L.Lz * L.Ly * L.Lh;
    for (int64_t k = 0; k < n_sweeps; ++k) {
        a.sweep = (uint32_t)(first_sweep + (uint64_t)k);
        for (int c = 0; c < 2; ++c) {
            a.colour = c;
            a.pass = c;
            a.finish = (c == 1);
            a.rev = (c == 1) ? (uint32_t)((size_t)L.nz * L.Ly * (L.Lh / L.vec) - 1) : 0u;
            for (int q = 0; q < 3; ++q) {
                a.own[q] = planes + (size_t)(3 * c + q) * plane;
                a.oth[q] = planes + (size_t)(3 * (1 - c) + q) * plane;
            }
            const cudaError_t e = hs::launch_pass(HS_FP32, L, a, grid, s);
            if (e != cudaSuccess) return fail(HS_E_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
        }
    }
    // moments, sweep count and accepted moves are contiguous in DevAccum
    if (cudaMemcpyAsync(d_out, acc->moments, (HS_N_MOMENTS + 2) * sizeof(double), cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
        return fail(HS_E_CUDA, "cudaMemcpyAsync failed");
    return HS_OK;
}
