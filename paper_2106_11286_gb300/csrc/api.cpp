// C ABI of the GB300 Metropolis library (declarations and contract in
// include/hs.h).  Host side: argument checks, lattice geometry, colouring,
// colour-sorted renumbering, device allocation and the sweep schedule.
//
// Geometry (arXiv 2106.11286 states the method for "any crystal lattice";
// the nearest-neighbour sets below are the sc / bcc / fcc coordination
// shells, z = 6 / 8 / 12).  Neighbour order of each site, which is also the
// order of the local-field sum:
//   sc : -x, +x, -y, +y, -z, +z
//   bcc: the 8 partner cells ordered by (dz, dy, dx) ascending; a corner
//        (basis 0) pairs with the centres of cells c + {-1,0}^3, a centre
//        with the corners of cells c + {0,1}^3
//   fcc: the 12 displacements (two half-integer components, one zero)
//        ordered by (dz, dy, dx) ascending
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <string>
#include <vector>

#include "batch.h"
#include "hs_impl.h"
#include "slab.h"
#include "upload.h"

namespace {
std::string &g_error_ref();
}

int hs::set_last_error(int code, const std::string &msg) {
    g_error_ref() = msg;
    return code;
}

using hs::DevAccum;
using hs::Layout;
using hs::PassArgs;

namespace {

thread_local std::string g_error;

std::string &g_error_ref() { return g_error; }

int fail(int code, const std::string &msg) {
    g_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    g_error = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return HS_E_OOM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return HS_E_DEVICE;
    return HS_E_CUDA;
}

#define HS_CUDA(call)                                        \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
    } while (0)

// ---------------------------------------------------------------- geometry
struct Offset {
    int dx, dy, dz, basis;
};

// Neighbour offsets (cell offset + partner basis) of each basis site.
std::vector<std::vector<Offset>> lattice_offsets(int type) {
    std::vector<std::vector<Offset>> off;
    if (type == HS_SC) {
        off.push_back({{-1, 0, 0, 0}, {1, 0, 0, 0}, {0, -1, 0, 0}, {0, 1, 0, 0}, {0, 0, -1, 0}, {0, 0, 1, 0}});
    } else if (type == HS_BCC) {
        for (int b = 0; b < 2; ++b) {
            std::vector<Offset> o;
            const int base = b == 0 ? -1 : 0;
            for (int k = 0; k < 8; ++k)  // k = dz*4 + dy*2 + dx in {0,1}^3, dz slowest
                o.push_back({base + (k & 1), base + ((k >> 1) & 1), base + (k >> 2), 1 - b});
            off.push_back(o);
        }
    } else {  // fcc: basis in half units
        const int B[4][3] = {{0, 0, 0}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};
        std::vector<std::array<int, 3>> disp;
        for (int k = 0; k < 27; ++k) {
            const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
            if ((dx != 0) + (dy != 0) + (dz != 0) == 2) disp.push_back({dx, dy, dz});
        }
        for (int b = 0; b < 4; ++b) {
            std::vector<Offset> o;
            for (auto &d : disp) {
                int q[3], cell[3];
                for (int a = 0; a < 3; ++a) {
                    q[a] = B[b][a] + d[a];
                    cell[a] = (q[a] >= 0) ? q[a] / 2 : -((1 - q[a]) / 2);
                    q[a] -= 2 * cell[a];
                }
                int nb = -1;
                for (int t = 0; t < 4; ++t)
                    if (B[t][0] == q[0] && B[t][1] == q[1] && B[t][2] == q[2]) nb = t;
                o.push_back({cell[0], cell[1], cell[2], nb});
            }
            off.push_back(o);
        }
    }
    return off;
}

struct Graph {
    int64_t n = 0;
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col;
    std::vector<int32_t> colour;  // natural index -> class (-1 absent)
    int n_colours = 0;
};

void build_structured(int type, const int32_t d[3], int periodic, Graph &g) {
    const auto off = lattice_offsets(type);
    const int nb = (int)off.size();
    const int64_t Lx = d[0], Ly = d[1], Lz = d[2];
    g.n = Lx * Ly * Lz * nb;
    g.row_ptr.assign(g.n + 1, 0);
    g.col.clear();
    g.col.reserve((size_t)g.n * off[0].size());
    g.colour.assign(g.n, 0);
    int64_t i = 0;
    for (int64_t cz = 0; cz < Lz; ++cz)
        for (int64_t cy = 0; cy < Ly; ++cy)
            for (int64_t cx = 0; cx < Lx; ++cx)
                for (int b = 0; b < nb; ++b, ++i) {
                    for (const Offset &o : off[b]) {
                        int64_t x = cx + o.dx, y = cy + o.dy, z = cz + o.dz;
                        const bool inside = x >= 0 && x < Lx && y >= 0 && y < Ly && z >= 0 && z < Lz;
                        if (!inside) {
                            if (!periodic) continue;
                            x = (x + Lx) % Lx;
                            y = (y + Ly) % Ly;
                            z = (z + Lz) % Lz;
                        }
                        g.col.push_back((int32_t)(((z * Ly + y) * Lx + x) * nb + o.basis));
                    }
                    g.row_ptr[i + 1] = (int64_t)g.col.size();
                    g.colour[i] = (type == HS_SC) ? (int32_t)((cx + cy + cz) & 1) : b;
                }
    g.n_colours = (type == HS_FCC) ? 4 : 2;
}

int greedy(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *mask, int32_t *colour) {
    std::vector<int64_t> seen;  // seen[c] == i marks colour c taken for site i
    int n_colours = 0;
    for (int64_t i = 0; i < n; ++i) colour[i] = -1;
    for (int64_t i = 0; i < n; ++i) {
        if (mask && !mask[i]) continue;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            const int32_t c = colour[col[k]];
            if (c < 0) continue;
            if ((size_t)c >= seen.size()) seen.resize((size_t)c + 1, -1);
            seen[(size_t)c] = i;
        }
        int32_t c = 0;
        while ((size_t)c < seen.size() && seen[(size_t)c] == i) ++c;
        colour[i] = c;
        n_colours = std::max(n_colours, c + 1);
    }
    return n_colours;
}

int check_csr(int64_t n, const int64_t *row_ptr, const int32_t *col) {
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(HS_E_INVALID, "n_sites must be in [0, 2^31)");
    if (!row_ptr || (n > 0 && !col && row_ptr[n] > 0)) return fail(HS_E_INVALID, "row_ptr/col_idx missing");
    if (row_ptr[0] != 0) return fail(HS_E_INVALID, "row_ptr[0] must be 0");
    for (int64_t i = 0; i < n; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return fail(HS_E_INVALID, "row_ptr must be non-decreasing");
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            if (col[k] < 0 || col[k] >= n) return fail(HS_E_INVALID, "col_idx out of range");
            if (col[k] == i) return fail(HS_E_INVALID, "self loop in neighbour list");
        }
    return HS_OK;
}

}  // namespace

// ---------------------------------------------------------------- handle
struct hs_lattice {
    int type = 0, precision = 0, periodic = 0, device = 0, n_sm = 0;
    int32_t dims[3] = {0, 0, 0};
    hs_params p{};
    uint64_t seed = 0;
    uint32_t replica = 0;
    cudaStream_t stream = nullptr;
    uint64_t sweep = 0;
    int accumulate = 0;
    int64_t last_n_sweeps = 0;
    double2 *sc_tab = nullptr;     // FP64: sin, cos(pi j / 1024) table of the trial orientation
    int tensor = 0;                // on-site anisotropy tensor term on
    double tA[6] = {0, 0, 0, 0, 0, 0};
    Layout L{};
    int n_blocks = 1;
    hs_launch req{};        // requested launch configuration (0 = automatic)
    int max_blocks = 1;     // capacity of the partials buffer
    int fold_ring = 1;      // sweeps per ring fold (slot sets of the partials buffer)
    double *partials = nullptr;
    DevAccum *acc = nullptr;
    double *stage = nullptr;  // 3 * n_sites doubles, lazily for host copies
    // hs_set_spins_async: two upload buffers (3 * n_sites doubles each), filled
    // on a copy stream of the handle's own and converted on the handle's stream
    void *up_buf[2] = {nullptr, nullptr};
    cudaStream_t up_stream = nullptr;
    cudaEvent_t up_filled[2] = {nullptr, nullptr};  // buffer's copy done
    cudaEvent_t up_free[2] = {nullptr, nullptr};    // buffer's conversion done
    int up_next = 0;
    // z-slab: parts of colour passes and the halo copies
    uint64_t sets_written = 0;      // partial sets written in the current sweep
    int interior_due = -1;          // colour whose interior part must come next (-1: none)
    int reserve = 0;                // CTAs the interior part leaves unlaunched
    cudaStream_t comm = nullptr;    // stream of the pack / unpack / plane copies
    int64_t max_pitch = 0;          // largest pitch of a strided copy (device attribute)
    int64_t device_bytes = 0;
    std::vector<void *> allocations;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    double timed_ms = 0.0;
    int64_t timed_launches = 0;

    ~hs_lattice() {
        cudaStreamSynchronize(stream);
        for (void *a : allocations) cudaFree(a);
        if (stage) cudaFree(stage);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (up_stream) cudaStreamSynchronize(up_stream);
        for (int b = 0; b < 2; ++b) {
            if (up_buf[b]) cudaFree(up_buf[b]);
            if (up_filled[b]) cudaEventDestroy(up_filled[b]);
            if (up_free[b]) cudaEventDestroy(up_free[b]);
        }
        if (up_stream) cudaStreamDestroy(up_stream);
    }
    template <typename T>
    int alloc(T **ptr, size_t bytes) {
        void *p_ = nullptr;
        cudaError_t e = cudaMalloc(&p_, bytes ? bytes : 16);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        allocations.push_back(p_);
        device_bytes += (int64_t)bytes;
        *ptr = static_cast<T *>(p_);
        return HS_OK;
    }
};

namespace {

PassArgs base_args(const hs_lattice *h) {
    PassArgs a{};
    const Layout &L = h->L;
    a.Lx = L.Lx;
    a.Ly = L.Ly;
    a.Lz = L.Lz;
    a.Lh = L.Lh;
    if (L.structured) {
        a.div_nxv = hs::FastDiv((uint32_t)(L.Lh / L.vec));
        a.div_ly = hs::FastDiv((uint32_t)L.Ly);
        // a z-slab's array plane z holds global plane z - z_off + z0
        a.nz = L.nz;
        a.z_off = L.slab ? 1 : 0;
        a.zpar = (L.z0 - a.z_off) & 1;
        a.site_off = (uint32_t)((int64_t)(L.z0 - a.z_off) * L.Ly * L.Lx);
        a.rank_off = (uint32_t)((int64_t)(L.z0 - a.z_off) * L.Ly * L.Lh);
        a.ty = L.ty;
    }
    a.spins4 = L.spins4;
    a.nbr = L.nbr;
    a.nat = L.nat;
    a.width = L.width;
    a.n_pad = L.n_pad;
    a.n_colours = L.n_colours;
    a.J = h->p.J;
    a.K = h->p.K;
    a.e[0] = h->p.e[0];
    a.e[1] = h->p.e[1];
    a.e[2] = h->p.e[2];
    a.fJ = (float)h->p.J;
    a.fK = (float)h->p.K;
    for (int q = 0; q < 3; ++q) a.fe[q] = (float)h->p.e[q];
    a.key0 = (uint32_t)h->seed;
    a.key1 = (uint32_t)(h->seed >> 32);
    a.replica = h->replica;
    a.sc_tab = h->sc_tab;
    a.tensor = h->tensor;
    a.zaxis = (h->p.e[0] == 0.0 && h->p.e[1] == 0.0 && h->p.e[2] == 1.0) ? 1 : 0;
    for (int q = 0; q < 6; ++q) {
        a.A[q] = h->tA[q];
        a.fA[q] = (float)h->tA[q];
    }
    a.partials = h->partials;
    a.sweep_tot = h->partials + (size_t)h->fold_ring * L.n_colours * h->max_blocks * hs::kPartials;
    a.n_blocks = h->n_blocks;
    a.n_present = (double)L.n_present;
    a.acc = h->acc;
    return a;
}

int setup_structured(hs_lattice *h) {
    Layout &L = h->L;
    const size_t es = hs::storage_size(h->precision);
    L.Lx = h->dims[0];
    L.Ly = h->dims[1];
    L.Lz = h->dims[2];
    L.Lh = L.Lx / 2;
    L.vec = 1;
    if (!L.slab) {
        L.nz = L.Lz;
        L.z0 = 0;
        L.Lz_glob = L.Lz;
    } else {
        L.Lz = L.nz + 2;  // halo planes at array planes 0 and nz + 1
    }
    const int64_t plane = (int64_t)L.Lz * L.Ly * L.Lh;
    int st = h->alloc(&L.planes, (size_t)plane * 6 * es);
    if (st == HS_OK && L.slab) {  // halos read as zero until the first exchange
        cudaError_t e = cudaMemsetAsync(L.planes, 0, (size_t)plane * 6 * es, h->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync");
    }
    return st;
}

int setup_table(hs_lattice *h, Graph &g, const uint8_t *mask) {
    Layout &L = h->L;
    const int64_t n = g.n;
    // colour classes must be independent sets among present sites
    for (int64_t i = 0; i < n; ++i) {
        if (mask && !mask[i]) continue;
        for (int64_t k = g.row_ptr[i]; k < g.row_ptr[i + 1]; ++k) {
            const int32_t j = g.col[k];
            if (mask && !mask[j]) continue;
            if (g.colour[i] == g.colour[j])
                return fail(HS_E_COLOUR, "colouring is not proper (periodic sc needs even dimensions)");
        }
    }
    if (g.n_colours > 64) return fail(HS_E_INVALID, "more than 64 colour classes");
    // renumber: class by class, ascending natural index inside a class
    std::vector<int64_t> count(g.n_colours + 1, 0);
    int64_t n_present = 0;
    for (int64_t i = 0; i < n; ++i)
        if (!mask || mask[i]) {
            ++count[g.colour[i] + 1];
            ++n_present;
        }
    for (int c = 0; c < g.n_colours; ++c) count[c + 1] += count[c];
    for (int c = 0; c <= g.n_colours; ++c) L.colour_begin[c] = count[c];
    std::vector<int64_t> renum(n, -1);
    std::vector<uint32_t> nat(n_present);
    std::vector<int64_t> cursor(count.begin(), count.end() - 1);
    int width = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (mask && !mask[i]) continue;
        const int64_t r = cursor[g.colour[i]]++;
        renum[i] = r;
        nat[r] = (uint32_t)i;
        int deg = 0;
        for (int64_t k = g.row_ptr[i]; k < g.row_ptr[i + 1]; ++k)
            if (!mask || mask[g.col[k]]) ++deg;
        width = std::max(width, deg);
    }
    L.n_present = n_present;
    L.width = width;
    L.n_pad = n_present + 1;
    const int32_t dummy = (int32_t)n_present;
    std::vector<int32_t> table((size_t)width * L.n_pad, dummy);
    for (int64_t r = 0; r < n_present; ++r) {
        const int64_t i = nat[r];
        int k2 = 0;
        for (int64_t k = g.row_ptr[i]; k < g.row_ptr[i + 1]; ++k) {
            const int32_t j = g.col[k];
            if (mask && !mask[j]) continue;
            table[(size_t)k2 * L.n_pad + r] = (int32_t)renum[j];
            ++k2;
        }
    }
    const size_t es = hs::storage_size(h->precision);
    int st;
    if ((st = h->alloc(&L.spins4, (size_t)L.n_pad * 4 * es))) return st;
    if ((st = h->alloc(&L.nbr, std::max<size_t>(table.size(), 1) * sizeof(int32_t)))) return st;
    if ((st = h->alloc(&L.nat, std::max<size_t>(nat.size(), 1) * sizeof(uint32_t)))) return st;
    HS_CUDA(cudaMemsetAsync(L.spins4, 0, (size_t)L.n_pad * 4 * es, h->stream));
    if (!table.empty())
        HS_CUDA(cudaMemcpyAsync(L.nbr, table.data(), table.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    if (!nat.empty())
        HS_CUDA(cudaMemcpyAsync(L.nat, nat.data(), nat.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, h->stream));
    HS_CUDA(cudaStreamSynchronize(h->stream));  // host vectors die on return
    return HS_OK;
}

bool vec_ok(const hs_lattice *h, int v) {
    const int es = (int)hs::storage_size(h->precision);
    return (v == 1 || v == 2 || v == 4 || v == 8) && v * es <= 16 && h->L.Lh % v == 0;
}

// Widest vector of at most 16 bytes dividing Lx/2; FP16 stops at 4 sites
// (8 bytes), which measured faster than 8 on GB300 (fewer registers).
int default_vec(const hs_lattice *h) {
    const int es = (int)hs::storage_size(h->precision);
    const int vmax = std::min(16 / es, 4);
    for (int v = vmax; v > 1; v /= 2)
        if (h->L.Lh % v == 0) return v;
    return 1;
}

// Zero a slab's partial sets: a launch of fewer CTAs than the set's stride
// relies on the rest of its set reading zero.
int clear_slab_sets(hs_lattice *h) {
    if (!h->L.slab || !h->partials) return HS_OK;
    const size_t n = (size_t)2 * hs::kSlabSets * h->max_blocks * hs::kPartials;
    HS_CUDA(cudaMemsetAsync(h->partials, 0, n * sizeof(double), h->stream));
    return HS_OK;
}

int configure_launch(hs_lattice *h) {
    Layout &L = h->L;
    if (L.slab && (h->sets_written != 0 || h->interior_due >= 0))
        return fail(HS_E_INVALID, "a slab's sweep is in progress");
    const hs_launch &r = h->req;
    L.tensor = h->tensor;
    if (!L.structured) {
        L.kernel = hs::kTable;
        // request 1 = L2 prefetch of the next site's table row, 2 = off, 0 = automatic (on for FP32 tables of
        // fewer than 8 neighbours: measured faster there, slower for FP16 and for fcc's 12; off for 8, whose
        // unrolled kernel measured 76.9 against 74.9 attempts/ns with it on the bcc nanoparticle)
        if (r.prefetch == 3) return fail(HS_E_INVALID, "split prefetch is a stencil option");
        L.prefetch = r.prefetch == 0 ? ((h->precision == HS_FP32 && L.width < 8) ? 1 : 0) : (r.prefetch == 1 ? 1 : 0);
        int bps = r.blocks_per_sm;
        const int occ = std::min(hs::pass_occupancy(h->precision, L, 0), hs::pass_occupancy(h->precision, L, 1));
        if (bps <= 0 || bps > occ) bps = occ;
        h->n_blocks = std::min(hs::pass_blocks(h->precision, L, h->n_sm, bps), h->max_blocks);
        return HS_OK;
    }
    L.vec = r.vec_width ? r.vec_width : default_vec(h);
    int kind = r.kernel;
    if (L.n_sites > 2147483647LL) {  // beyond 2^31 sites: the register stencil, with 32-bit work items
        if (kind != HS_KERNEL_AUTO && kind != HS_KERNEL_STENCIL)
            return fail(HS_E_INVALID, "lattices beyond 2^31 sites run the register stencil");
        if ((int64_t)L.nz * L.Ly * (L.Lh / L.vec) >= 4294967296LL)
            return fail(HS_E_INVALID, "vector width too small: more than 2^32 work items");
    }
    // automatic choice: the register stencil (hs_autotune also times the pipelined one)
    if (kind == HS_KERNEL_AUTO) kind = HS_KERNEL_STENCIL;
    if (h->tensor && (kind != HS_KERNEL_STENCIL || r.prefetch == 1 || r.prefetch == 3))
        return fail(HS_E_INVALID, "the anisotropy tensor term runs on the register stencil without prefetch");
    if (kind == HS_KERNEL_MARCH) {
        const int nxv = L.Lh / L.vec;
        int ty = r.tile_y;
        if (ty == 0) {  // smallest slab with one work item per thread
            for (int c : {1, 2, 4, 8, 16, 32})
                if (L.Ly % c == 0 && c * nxv >= hs::kBlock) {
                    ty = c;
                    break;
                }
            if (ty == 0) ty = L.Ly;
        }
        if (ty < 1 || L.Ly % ty != 0) return fail(HS_E_INVALID, "tile_y must divide Ly");
        L.kernel = hs::kMarch;
        L.ty = ty;
        int bps = r.blocks_per_sm;
        const int occ = std::min(hs::pass_occupancy(h->precision, L, 0), hs::pass_occupancy(h->precision, L, 1));
        if (bps <= 0 || bps > occ) bps = occ;
        const int64_t slabs = (int64_t)(L.Ly / ty) * L.Lz;
        h->n_blocks = (int)std::min<int64_t>(std::min<int64_t>(slabs, (int64_t)h->n_sm * bps), h->max_blocks);
        return HS_OK;
    }
    if (kind == HS_KERNEL_PIPE) {
        if (hs::pipe_smem_bytes(h->precision, L.vec) == 0)
            return fail(HS_E_INVALID, "pipelined stencil needs 4 to 16 bytes of storage per vector");
        L.kernel = hs::kPipe;
        const int occ = std::min(hs::pass_occupancy(h->precision, L, 0), hs::pass_occupancy(h->precision, L, 1));
        if (occ < 1) return fail(HS_E_INVALID, "pipelined stencil slots do not fit in shared memory");
        int bps = r.blocks_per_sm;
        if (bps <= 0 || bps > occ) bps = occ;
        h->n_blocks = std::min(hs::pass_blocks(h->precision, L, h->n_sm, bps), h->max_blocks);
        return HS_OK;
    }
    L.kernel = hs::kStencil;  // before the occupancy query, which looks at the kind
    // request 1 = next item in registers, 3 = split prefetch, 2 = off; automatic: off (with the alternating
    // order, which lets each pass start on data in L2, no prefetch measured fastest at 256^3 and 464^3 FP32)
    if (h->tensor || r.prefetch == 0)
        L.prefetch = 0;
    else
        L.prefetch = r.prefetch == 1 ? 1 : (r.prefetch == 3 ? 2 : 0);
    // automatic order: alternating, except with the split prefetch, which measured slower in descending passes,
    // and beyond 2^31 sites, where the ascending-only variant of the kernel is faster (137 against 103-112
    // attempts/ns at 2048^3 FP32; the direction-capable code is faster from 256^3 to 1024^3)
    const bool wide = L.n_sites > 2147483647LL;
    L.order = r.order != 0 ? r.order : ((L.prefetch == 2 || wide) ? 1 : 2);
    L.plain = wide && L.order == 1 && L.prefetch == 0 && !h->tensor &&
              ((h->precision == HS_FP32 && L.vec == 4) || (h->precision == HS_FP16 && L.vec == 8));
    int bps = r.blocks_per_sm;
    const int occ = std::min(hs::pass_occupancy(h->precision, L, 0), hs::pass_occupancy(h->precision, L, 1));
    if (bps <= 0 || bps > occ) bps = occ;
    h->n_blocks = std::min(hs::pass_blocks(h->precision, L, h->n_sm, bps), h->max_blocks);
    return clear_slab_sets(h);  // the parts' grids follow the launch configuration
}

int flush_timing(hs_lattice *h) {
    if (h->ev_used == 0) return HS_OK;
    HS_CUDA(cudaStreamSynchronize(h->stream));
    for (size_t k = 0; k + 1 < h->ev_used; k += 2) {
        float ms = 0.f;
        HS_CUDA(cudaEventElapsedTime(&ms, h->ev[k], h->ev[k + 1]));
        h->timed_ms += ms;
        ++h->timed_launches;
    }
    h->ev_used = 0;
    return HS_OK;
}

int record_event(hs_lattice *h) {
    if (h->ev_used == h->ev.size()) {
        if (h->ev.size() >= 8192) {
            if (h->ev_used % 2 != 0) return fail(HS_E_INVALID, "timing events unbalanced");
            int st = flush_timing(h);
            if (st) return st;
        } else {
            cudaEvent_t e;
            HS_CUDA(cudaEventCreate(&e));
            h->ev.push_back(e);
        }
    }
    HS_CUDA(cudaEventRecord(h->ev[h->ev_used++], h->stream));
    return HS_OK;
}

int check_device_error(hs_lattice *h) {
    int err = 0;
    HS_CUDA(cudaMemcpyAsync(&err, &h->acc->error, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    HS_CUDA(cudaStreamSynchronize(h->stream));
    if (err != 0) {
        HS_CUDA(cudaMemsetAsync(&h->acc->error, 0, sizeof(int), h->stream));
        return fail(HS_E_TIMEOUT, "a bounded device-side wait timed out");
    }
    return HS_OK;
}

}  // namespace

extern "C" {

const char *hs_last_error(void) { return g_error.c_str(); }

int hs_api_version(void) { return HS_API_VERSION; }

int hs_colour_greedy(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const uint8_t *site_mask,
                     int32_t *colour_out, int *n_colours) {
    if (!colour_out || !n_colours) return fail(HS_E_INVALID, "null output");
    int st = check_csr(n, row_ptr, col_idx);
    if (st) return st;
    *n_colours = greedy(n, row_ptr, col_idx, site_mask, colour_out);
    return HS_OK;
}

namespace {
// z-slab of a periodic sc lattice: own global planes z0 .. z0 + nz - 1
struct SlabSpec {
    int z0, nz;
};

int lattice_create(hs_lattice **out, int type, const int32_t dims[3], int periodic, const int64_t *row_ptr,
                   const int32_t *col_idx, int64_t n_sites, const uint8_t *site_mask, const hs_params *p,
                   int precision, uint64_t seed, uint32_t replica, void *cuda_stream, const SlabSpec *slab) {
    if (!out) return fail(HS_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!p) return fail(HS_E_INVALID, "params are NULL");
    if (precision < HS_FP64 || precision > HS_FP16) return fail(HS_E_INVALID, "unknown precision");
    if (type < HS_SC || type > HS_CSR) return fail(HS_E_INVALID, "unknown lattice type");
    const double en = std::sqrt(p->e[0] * p->e[0] + p->e[1] * p->e[1] + p->e[2] * p->e[2]);
    if (!(en > 0.0) || !std::isfinite(en) || !std::isfinite(p->J) || !std::isfinite(p->K))
        return fail(HS_E_INVALID, "J, K must be finite and e non-zero");
    Graph g;
    bool structured = false;
    if (type == HS_CSR) {
        if (row_ptr == nullptr) return fail(HS_E_INVALID, "HS_CSR needs row_ptr and col_idx");
        int st = check_csr(n_sites, row_ptr, col_idx);
        if (st) return st;
    } else {
        if (!dims || row_ptr || col_idx) return fail(HS_E_INVALID, "structured lattices take dims, not a CSR");
        const int nb = type == HS_SC ? 1 : (type == HS_BCC ? 2 : 4);
        for (int a = 0; a < 3; ++a)
            if (dims[a] < 1) return fail(HS_E_INVALID, "dims must be >= 1");
        const double total = (double)dims[0] * dims[1] * dims[2] * nb;
        // FP32 / FP16 periodic sc: 32-bit element offsets within a colour plane
        // and 32-bit colour ranks (up to 2^33 sites); everything else: 32-bit
        // signed site indices
        const bool wide = type == HS_SC && periodic && site_mask == nullptr && precision != HS_FP64;
        if (wide) {
            const double rows = slab ? (double)(slab->nz + 2) : (double)dims[2];
            if ((double)dims[2] * dims[1] * (dims[0] / 2) > 4294967296.0 || rows * dims[1] * (dims[0] / 2) > 4294967296.0)
                return fail(HS_E_INVALID, "more than 2^32 sites of one colour");
        } else if (total >= 2147483647.0) {
            return fail(HS_E_INVALID, "more than 2^31 - 1 sites");
        }
        if (type == HS_SC && periodic) {
            for (int a = 0; a < 3; ++a)
                if (dims[a] % 2 != 0)
                    return fail(HS_E_COLOUR, "periodic sc with an odd dimension is not two-colourable");
        }
        structured = (type == HS_SC && periodic && site_mask == nullptr);
    }
    int dev = 0;
    {
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    }
    hs_lattice *h = new (std::nothrow) hs_lattice();
    if (!h) return fail(HS_E_OOM, "host allocation failed");
    h->type = type;
    h->precision = precision;
    h->periodic = periodic ? 1 : 0;
    h->device = dev;
    if (dims) std::memcpy(h->dims, dims, sizeof(h->dims));
    h->p = *p;
    for (int a = 0; a < 3; ++a) h->p.e[a] = p->e[a] / en;
    h->seed = seed;
    h->replica = replica;
    h->stream = (cudaStream_t)cuda_stream;
    h->comm = h->stream;
    {
        int pitch = 0;
        cudaError_t e = cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&pitch, cudaDevAttrMaxPitch, dev);
        if (e != cudaSuccess) {
            delete h;
            return cuda_fail(e, "cudaDeviceGetAttribute");
        }
        h->max_pitch = pitch;
    }
    int st = HS_OK;
    Layout &L = h->L;
    L.structured = structured;
    if (slab) {
        L.slab = true;
        L.z0 = slab->z0;
        L.nz = slab->nz;
        L.Lz_glob = dims[2];
    }
    try {
        if (structured) {
            L.n_colours = 2;
            L.n_sites = L.n_present = (int64_t)dims[0] * dims[1] * (slab ? slab->nz : dims[2]);
            st = setup_structured(h);
        } else {
            if (type == HS_CSR) {
                g.n = n_sites;
                g.row_ptr.assign(row_ptr, row_ptr + n_sites + 1);
                g.col.assign(col_idx, col_idx + row_ptr[n_sites]);
                g.colour.assign(n_sites, -1);
                g.n_colours = greedy(n_sites, row_ptr, col_idx, site_mask, g.colour.data());
            } else {
                build_structured(type, dims, periodic, g);
            }
            L.n_sites = g.n;
            L.n_colours = std::max(g.n_colours, 1);
            st = setup_table(h, g, site_mask);
        }
    } catch (const std::bad_alloc &) {
        st = fail(HS_E_OOM, "host allocation failed");
    }
    if (st == HS_OK) {
        h->max_blocks = h->n_sm * (2048 / hs::kBlock);
        // ring of per-sweep slot sets (at most 8 MB, at most kRingMax sweeps),
        // then the ring fold's per-sweep records
        const size_t slot_doubles = (size_t)L.n_colours * h->max_blocks * hs::kPartials;
        const size_t fit = (size_t)(8u << 20) / (slot_doubles * sizeof(double));
        h->fold_ring = (int)std::max<size_t>(1, std::min<size_t>(hs::kRingMax, fit));
        // a slab sweeps pass by pass (no ring) but keeps kSlabSets partial sets per colour in slot 0
        if (L.slab) h->fold_ring = std::max(h->fold_ring, hs::kSlabSets);
        st = h->alloc(&h->partials, (slot_doubles + hs::kSweepRecord) * (size_t)h->fold_ring * sizeof(double));
        if (st == HS_OK) st = configure_launch(h);
    }
    if (st == HS_OK) st = h->alloc(&h->acc, sizeof(DevAccum));
    if (st == HS_OK && precision == HS_FP64) {
        // sin, cos(pi j / 1024) for the FP64 trial's table lookup, from long double on the host
        const long double pi = 3.141592653589793238462643383279502884L;
        std::vector<double2> tab(2048);
        for (int j = 0; j < 2048; ++j) {
            const long double a = pi * (long double)j / 1024.0L;
            tab[j] = make_double2((double)sinl(a), (double)cosl(a));
        }
        st = h->alloc(&h->sc_tab, tab.size() * sizeof(double2));
        if (st == HS_OK) {
            cudaError_t e = cudaMemcpy(h->sc_tab, tab.data(), tab.size() * sizeof(double2), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) st = cuda_fail(e, "cudaMemcpy");
        }
    }
    if (st == HS_OK) {
        cudaError_t e = cudaMemsetAsync(h->acc, 0, sizeof(DevAccum), h->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync");
    }
    if (st == HS_OK) st = hs_init_spins(h, HS_INIT_ALIGNED);
    if (st == HS_OK) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
    }
    if (st != HS_OK) {
        delete h;
        return st;
    }
    *out = h;
    return HS_OK;
}
}  // namespace

int hs_lattice_create(hs_lattice **out, int type, const int32_t dims[3], int periodic, const int64_t *row_ptr,
                      const int32_t *col_idx, int64_t n_sites, const uint8_t *site_mask, const hs_params *p,
                      int precision, uint64_t seed, uint32_t replica, void *cuda_stream) {
    return lattice_create(out, type, dims, periodic, row_ptr, col_idx, n_sites, site_mask, p, precision, seed,
                          replica, cuda_stream, nullptr);
}

int hs_slab_create(hs_lattice **out, const int32_t dims[3], int32_t z0, int32_t nz, const hs_params *p,
                   int precision, uint64_t seed, uint32_t replica, void *cuda_stream) {
    if (!out) return fail(HS_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!dims) return fail(HS_E_INVALID, "dims are NULL");
    if (nz < 1 || z0 < 0 || (int64_t)z0 + nz > dims[2]) return fail(HS_E_INVALID, "slab planes must lie in [0, Lz)");
    const SlabSpec spec{z0, nz};
    return lattice_create(out, HS_SC, dims, 1, nullptr, nullptr, 0, nullptr, p, precision, seed, replica,
                          cuda_stream, &spec);
}

void hs_lattice_destroy(hs_lattice *h) { delete h; }

int hs_init_spins(hs_lattice *h, int mode) {
    if (!h) return fail(HS_E_INVALID, "null handle");
    if (mode != HS_INIT_RANDOM && mode != HS_INIT_ALIGNED) return fail(HS_E_INVALID, "unknown init mode");
    if (h->L.n_present == 0) return HS_OK;
    HS_CUDA(hs::launch_init(h->precision, h->L, mode, h->p.e, (uint32_t)h->seed, (uint32_t)(h->seed >> 32),
                            h->replica, h->stream));
    return HS_OK;
}

namespace {
// Launch colour pass c of sweep index `sweep`.  Its CTAs' partial sums go to
// ring slot `slot`.  deferred = 0 (slot 0): the last colour's last CTA to
// arrive finalises the sweep inside the kernel.  deferred = 1 (hs_sweep): the
// caller folds the ring after each full group of sweeps and after its loop.
int run_pass(hs_lattice *h, PassArgs &a, uint32_t sweep, int c, bool deferred = false, int slot = 0) {
    const Layout &L = h->L;
    a.sweep = sweep;
    a.colour = c;
    a.pass = c;
    a.slot = slot;
    a.finish = deferred ? 0 : (c == L.n_colours - 1);
    if (L.structured) {
        const size_t es = hs::storage_size(h->precision);
        const int64_t plane = (int64_t)L.Lz * L.Ly * L.Lh;
        char *base = static_cast<char *>(L.planes);
        for (int q = 0; q < 3; ++q) {
            a.own[q] = base + (size_t)(3 * c + q) * plane * es;
            a.oth[q] = base + (size_t)(3 * (1 - c) + q) * plane * es;
        }
        // alternating order: colour 1 runs from the last work item down, so it starts on the planes that
        // colour 0 touched last (in L2), and the next sweep's colour 0 starts where colour 1 ended
        a.rev = (L.kernel == hs::kStencil && L.order == 2 && c == 1)
                    ? (uint32_t)((int64_t)a.nz * L.Ly * (L.Lh / L.vec) - 1)
                    : 0u;
    } else {
        a.begin = L.colour_begin[c];
        a.end = L.colour_begin[c + 1];
        a.colour_begin = L.colour_begin[c];
    }
    if (h->timing) {
        int st = record_event(h);
        if (st) return st;
    }
    HS_CUDA(hs::launch_pass(h->precision, L, a, h->n_blocks, h->stream));
    if (h->timing) {
        int st = record_event(h);
        if (st) return st;
    }
    return HS_OK;
}

int check_beta(double beta) {
    if (!(beta >= 0.0) || !std::isfinite(beta)) return fail(HS_E_INVALID, "beta must be finite and >= 0");
    return HS_OK;
}
}  // namespace

int hs_sweep(hs_lattice *h, double beta, int64_t n_sweeps) {
    if (!h) return fail(HS_E_INVALID, "null handle");
    if (int st = check_beta(beta)) return st;
    if (n_sweeps < 0) return fail(HS_E_INVALID, "n_sweeps must be >= 0");
    if (h->L.slab && n_sweeps > 0)
        return fail(HS_E_INVALID, "a slab sweeps pass by pass (hs_sweep_pass), its halos refreshed in between");
    h->last_n_sweeps = n_sweeps;
    HS_CUDA(cudaMemsetAsync(&h->acc->accepted, 0, sizeof(double), h->stream));
    if (n_sweeps == 0 || h->L.n_present == 0) {
        h->sweep += (uint64_t)n_sweeps;
        return HS_OK;
    }
    PassArgs a = base_args(h);
    a.beta = beta;
    a.fbeta = (float)beta;
    a.accumulate = h->accumulate;
    // sweep s writes ring slot s mod ring; each full ring, and the rest after
    // the loop, is folded into the accumulator in sweep order
    int pending = 0;
    for (int64_t s = 0; s < n_sweeps; ++s) {
        for (int c = 0; c < h->L.n_colours; ++c)
            if (int st = run_pass(h, a, (uint32_t)(h->sweep + (uint64_t)s), c, true, pending)) return st;
        if (++pending == h->fold_ring) {
            HS_CUDA(hs::launch_fold(a, pending, h->stream));
            pending = 0;
        }
    }
    if (pending > 0) HS_CUDA(hs::launch_fold(a, pending, h->stream));
    h->sweep += (uint64_t)n_sweeps;
    return HS_OK;
}

namespace {
// CTAs of a stencil launch over n_planes own planes of a slab, at most cap.
int plane_grid(const hs_lattice *h, int n_planes, int cap) {
    const int64_t items = (int64_t)n_planes * h->L.Ly * (h->L.Lh / h->L.vec);
    return (int)std::max<int64_t>(1, std::min<int64_t>((items + hs::kBlock - 1) / hs::kBlock, cap));
}

// One launch of colour c of a slab over its own array planes z_first ..
// z_first + n_planes - 1 (1 .. nz), on `grid` CTAs, its partials in set
// `set` of that colour.  finish: this launch completes the sweep, so its
// last CTA folds the sets written in it.
int run_slab_launch(hs_lattice *h, PassArgs a, int c, int set, int z_first, int n_planes, int grid, bool finish) {
    const Layout &L = h->L;
    a.sweep = (uint32_t)h->sweep;
    a.colour = c;
    a.n_colours = 2 * hs::kSlabSets;
    a.pass = hs::kSlabSets * c + set;
    a.slot = 0;
    a.z_off = z_first;
    a.nz = n_planes;
    h->sets_written |= 1ull << a.pass;
    a.finish = finish ? 1 : 0;
    a.skip_sets = ~h->sets_written;
    const size_t es = hs::storage_size(h->precision);
    const int64_t plane = (int64_t)L.Lz * L.Ly * L.Lh;
    char *base = static_cast<char *>(L.planes);
    for (int q = 0; q < 3; ++q) {
        a.own[q] = base + (size_t)(3 * c + q) * plane * es;
        a.oth[q] = base + (size_t)(3 * (1 - c) + q) * plane * es;
    }
    if (h->timing) {
        int st = record_event(h);
        if (st) return st;
    }
    HS_CUDA(hs::launch_pass(h->precision, L, a, grid, h->stream));
    if (h->timing) {
        int st = record_event(h);
        if (st) return st;
    }
    return HS_OK;
}

}  // namespace

int hs_sweep_pass(hs_lattice *h, double beta, int colour) { return hs_sweep_pass_part(h, beta, colour, HS_PART_WHOLE); }

int hs_sweep_pass_part(hs_lattice *h, double beta, int colour, int part) {
    if (!h) return fail(HS_E_INVALID, "null handle");
    if (int st = check_beta(beta)) return st;
    if (colour < 0 || colour >= h->L.n_colours) return fail(HS_E_INVALID, "colour out of range");
    if (part != HS_PART_WHOLE && part != HS_PART_BOUNDARY && part != HS_PART_INTERIOR)
        return fail(HS_E_INVALID, "part must be HS_PART_WHOLE, HS_PART_BOUNDARY or HS_PART_INTERIOR");
    const Layout &L = h->L;
    if (part != HS_PART_WHOLE && !L.slab) return fail(HS_E_INVALID, "boundary and interior parts are slab passes");
    if (part == HS_PART_INTERIOR ? h->interior_due != colour : h->interior_due >= 0)
        return fail(HS_E_INVALID, "a boundary part must be followed by the interior part of its colour");
    const bool last = colour == L.n_colours - 1;
    if (colour == 0 && part != HS_PART_INTERIOR) {
        h->last_n_sweeps = 1;
        h->sets_written = 0;
        HS_CUDA(cudaMemsetAsync(&h->acc->accepted, 0, sizeof(double), h->stream));
    }
    if (L.n_present > 0) {
        PassArgs a = base_args(h);
        a.beta = beta;
        a.fbeta = (float)beta;
        // a slab always measures its fused sums (the observables of a lattice split into slabs come from
        // all slabs' sums); only accumulation adds its own moments
        a.accumulate = h->accumulate ? 1 : (L.slab ? 2 : 0);
        if (!L.slab) {
            if (int st = run_pass(h, a, (uint32_t)h->sweep, colour)) return st;
        } else if (part == HS_PART_WHOLE) {
            if (int st = run_slab_launch(h, a, colour, 3, 1, L.nz, h->n_blocks, last)) return st;
        } else if (part == HS_PART_BOUNDARY) {
            if (L.nz <= 2) {  // the boundary planes are the whole slab: one launch, no interior
                if (int st = run_slab_launch(h, a, colour, 0, 1, L.nz, plane_grid(h, L.nz, h->n_blocks), last))
                    return st;
            } else {
                const int g = plane_grid(h, 1, h->n_blocks);
                if (int st = run_slab_launch(h, a, colour, 0, 1, 1, g, false)) return st;
                if (int st = run_slab_launch(h, a, colour, 1, L.nz, 1, g, false)) return st;
            }
        } else if (L.nz > 2) {
            const int g = plane_grid(h, L.nz - 2, std::max(1, h->n_blocks - h->reserve));
            if (int st = run_slab_launch(h, a, colour, 2, 2, L.nz - 2, g, last)) return st;
        }
    }
    h->interior_due = part == HS_PART_BOUNDARY ? colour : -1;
    if (last && part != HS_PART_BOUNDARY) {
        h->sweep += 1;
        h->sets_written = 0;
    }
    return HS_OK;
}

int hs_slab_reserve_ctas(hs_lattice *h, int32_t ctas) {
    if (!h) return fail(HS_E_INVALID, "null handle");
    if (!h->L.slab) return fail(HS_E_INVALID, "not a slab");
    if (ctas < 0 || ctas >= h->n_blocks) return fail(HS_E_INVALID, "reserve 0 .. the pass's CTAs - 1");
    if (h->sets_written != 0 || h->interior_due >= 0) return fail(HS_E_INVALID, "a sweep is in progress");
    h->reserve = ctas;
    return clear_slab_sets(h);
}

int hs_slab_set_comm_stream(hs_lattice *h, void *cuda_stream) {
    if (!h) return fail(HS_E_INVALID, "null handle");
    if (!h->L.slab) return fail(HS_E_INVALID, "not a slab");
    h->comm = (cudaStream_t)cuda_stream;
    return HS_OK;
}

int hs_slab_plane(const hs_lattice *h, int colour, int component, int which, void **dev_ptr, size_t *bytes) {
    if (!h || !dev_ptr || !bytes) return fail(HS_E_INVALID, "null argument");
    const Layout &L = h->L;
    if (!L.slab) return fail(HS_E_INVALID, "not a slab");
    if (colour < 0 || colour > 1 || component < 0 || component > 2 || which < 0 || which > 3)
        return fail(HS_E_INVALID, "colour 0/1, component 0..2, which 0..3");
    const size_t es = hs::storage_size(h->precision);
    const size_t plane_elems = (size_t)L.Ly * L.Lh;
    const int z = which == 0 ? 0 : (which == 1 ? 1 : (which == 2 ? L.nz : L.nz + 1));
    *dev_ptr = static_cast<char *>(L.planes) + ((size_t)(3 * colour + component) * L.Lz + z) * plane_elems * es;
    *bytes = plane_elems * es;
    return HS_OK;
}

namespace {
// Copy the three component planes of one colour at one z plane between
// (dst, dst_pitch) and (src, src_pitch) -- addresses of component x, pitch
// = bytes from one component's plane to the next -- as one strided copy, or
// three when a pitch exceeds the device's largest.
int copy_components(const hs_lattice *h, void *dst, size_t dst_pitch, const void *src, size_t src_pitch,
                    size_t bytes, cudaStream_t s) {
    if ((int64_t)std::max(dst_pitch, src_pitch) <= h->max_pitch) {
        HS_CUDA(cudaMemcpy2DAsync(dst, dst_pitch, src, src_pitch, bytes, 3, cudaMemcpyDeviceToDevice, s));
        return HS_OK;
    }
    for (int q = 0; q < 3; ++q)
        HS_CUDA(cudaMemcpyAsync(static_cast<char *>(dst) + q * dst_pitch, static_cast<const char *>(src) + q * src_pitch,
                                bytes, cudaMemcpyDeviceToDevice, s));
    return HS_OK;
}

// bytes from one component's plane array to the next (the colour-major layout)
size_t component_pitch(const hs_lattice *h) {
    return (size_t)h->L.Lz * h->L.Ly * h->L.Lh * hs::storage_size(h->precision);
}
}  // namespace

int hs_slab_copy_plane(hs_lattice *dst, int dst_which, const hs_lattice *src, int src_which, int colour) {
    if (!dst || !src) return fail(HS_E_INVALID, "null handle");
    if (!dst->L.slab || !src->L.slab) return fail(HS_E_INVALID, "not a slab");
    if (dst->precision != src->precision || dst->L.Lx != src->L.Lx || dst->L.Ly != src->L.Ly ||
        dst->device != src->device)
        return fail(HS_E_INVALID, "slabs of different lattices or devices");
    void *d = nullptr, *sp = nullptr;
    size_t nb = 0, ns = 0;
    if (int st = hs_slab_plane(dst, colour, 0, dst_which, &d, &nb)) return st;
    if (int st = hs_slab_plane(src, colour, 0, src_which, &sp, &ns)) return st;
    return copy_components(dst, d, component_pitch(dst), sp, component_pitch(src), nb, dst->comm);
}

int hs_slab_pack(const hs_lattice *h, int colour, int which, void *d_buf) {
    if (!h || !d_buf) return fail(HS_E_INVALID, "null argument");
    void *sp = nullptr;
    size_t nb = 0;
    if (int st = hs_slab_plane(h, colour, 0, which, &sp, &nb)) return st;
    return copy_components(h, d_buf, nb, sp, component_pitch(h), nb, h->comm);
}

int hs_slab_unpack(hs_lattice *h, int colour, int which, const void *d_buf) {
    if (!h || !d_buf) return fail(HS_E_INVALID, "null argument");
    void *dp = nullptr;
    size_t nb = 0;
    if (int st = hs_slab_plane(h, colour, 0, which, &dp, &nb)) return st;
    return copy_components(h, dp, component_pitch(h), d_buf, nb, nb, h->comm);
}

int hs_read_sums_device(hs_lattice *h, double *d_out) {
    if (!h || !d_out) return fail(HS_E_INVALID, "null argument");
    HS_CUDA(cudaMemcpyAsync(d_out, h->acc->sums, 5 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    return HS_OK;
}

int hs_accumulate_sums(hs_lattice *h, const double *d_tot, int64_t n_sites) {
    if (!h || !d_tot) return fail(HS_E_INVALID, "null argument");
    if (n_sites < 1) return fail(HS_E_INVALID, "n_sites must be >= 1");
    HS_CUDA(hs::launch_slab_apply(h->acc, d_tot, (double)n_sites, h->p.e, h->stream));
    return HS_OK;
}

int hs_get_sites(hs_lattice *h, int64_t n, const int64_t *sites, double *out) {
    if (!h || (n > 0 && (!sites || !out))) return fail(HS_E_INVALID, "null argument");
    if (n < 0) return fail(HS_E_INVALID, "negative count");
    const Layout &L = h->L;
    if (!L.structured) return fail(HS_E_INVALID, "site gathers need a periodic sc lattice or slab");
    const int64_t plane = (int64_t)L.Lx * L.Ly;
    for (int64_t t = 0; t < n; ++t) {
        const int64_t z = sites[t] / plane;
        if (sites[t] < 0 || z < L.z0 || z >= (int64_t)L.z0 + L.nz) return fail(HS_E_INVALID, "site not owned");
    }
    if (n == 0) return HS_OK;
    int64_t *d_sites = nullptr;
    double *d_out = nullptr;
    cudaError_t e = cudaMalloc(&d_sites, (size_t)n * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_out, (size_t)n * 3 * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_sites, sites, (size_t)n * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = hs::launch_gather_sites(h->precision, L, n, d_sites, d_out, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, d_out, (size_t)n * 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(d_sites);
    cudaFree(d_out);
    if (e != cudaSuccess) return cuda_fail(e, "hs_get_sites");
    return HS_OK;
}

int hs_read_sums(hs_lattice *h, double out[5]) {
    if (!h || !out) return fail(HS_E_INVALID, "null argument");
    HS_CUDA(cudaMemcpyAsync(out, h->acc->sums, 5 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return check_device_error(h);
}

int hs_measure(hs_lattice *h, hs_measurement *out) {
    if (!h || !out) return fail(HS_E_INVALID, "null argument");
    if (h->L.slab) return fail(HS_E_INVALID, "a slab measures through its fused sums (hs_read_sums)");
    std::memset(out, 0, sizeof(*out));
    out->n_sites = h->L.n_present;
    if (h->L.n_present == 0) return HS_OK;
    PassArgs a = base_args(h);
    a.n_colours = 1;
    a.pass = 0;
    a.finish = 1;
    a.accumulate = 0;
    HS_CUDA(hs::launch_measure(h->precision, h->L, a, h->n_blocks, h->stream));
    double last[8], accepted = 0.0;
    HS_CUDA(cudaMemcpyAsync(last, h->acc->last, sizeof(last), cudaMemcpyDeviceToHost, h->stream));
    HS_CUDA(cudaMemcpyAsync(&accepted, &h->acc->accepted, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    int st = check_device_error(h);
    if (st) return st;
    out->E = last[0];
    out->M[0] = last[1];
    out->M[1] = last[2];
    out->M[2] = last[3];
    out->absM = last[4];
    out->M2 = last[5];
    out->M4 = last[6];
    const double attempts = (double)h->last_n_sweeps * (double)h->L.n_present;
    out->accept_rate = attempts > 0 ? accepted / attempts : 0.0;
    return HS_OK;
}

int hs_accumulate(hs_lattice *h, int on) {
    if (!h) return fail(HS_E_INVALID, "null handle");
    h->accumulate = on ? 1 : 0;
    return HS_OK;
}

int hs_reset_accumulator(hs_lattice *h) {
    if (!h) return fail(HS_E_INVALID, "null handle");
    HS_CUDA(cudaMemsetAsync(h->acc->moments, 0, sizeof(h->acc->moments) + sizeof(double), h->stream));
    return HS_OK;
}

int hs_read_accumulator(hs_lattice *h, double moments[HS_N_MOMENTS], int64_t *count) {
    if (!h || !moments || !count) return fail(HS_E_INVALID, "null argument");
    double buf[HS_N_MOMENTS + 1];
    HS_CUDA(cudaMemcpyAsync(buf, h->acc->moments, sizeof(buf), cudaMemcpyDeviceToHost, h->stream));
    int st = check_device_error(h);
    if (st) return st;
    std::memcpy(moments, buf, sizeof(double) * HS_N_MOMENTS);
    *count = (int64_t)buf[HS_N_MOMENTS];
    return HS_OK;
}

static int ensure_stage(hs_lattice *h) {
    if (h->stage) return HS_OK;
    cudaError_t e = cudaMalloc(&h->stage, (size_t)std::max<int64_t>(h->L.n_sites, 1) * 3 * sizeof(double));
    if (e != cudaSuccess) {
        h->stage = nullptr;
        return cuda_fail(e, "cudaMalloc(stage)");
    }
    return HS_OK;
}

int hs_get_spins_device(hs_lattice *h, double *d_xyz) {
    if (!h || !d_xyz) return fail(HS_E_INVALID, "null argument");
    if (!h->L.structured)
        HS_CUDA(cudaMemsetAsync(d_xyz, 0, (size_t)h->L.n_sites * 3 * sizeof(double), h->stream));
    if (h->L.n_present == 0) return HS_OK;
    HS_CUDA(hs::launch_gather(h->precision, h->L, d_xyz, h->stream));
    return HS_OK;
}

int hs_set_spins_device(hs_lattice *h, const double *d_xyz) {
    if (!h || !d_xyz) return fail(HS_E_INVALID, "null argument");
    if (h->L.n_present == 0) return HS_OK;
    HS_CUDA(hs::launch_scatter(h->precision, h->L, d_xyz, h->stream));
    return HS_OK;
}

int hs_get_spins(hs_lattice *h, double *xyz) {
    if (!h || !xyz) return fail(HS_E_INVALID, "null argument");
    int st = ensure_stage(h);
    if (st) return st;
    if ((st = hs_get_spins_device(h, h->stage))) return st;
    HS_CUDA(cudaMemcpyAsync(xyz, h->stage, (size_t)h->L.n_sites * 3 * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
    HS_CUDA(cudaStreamSynchronize(h->stream));
    return HS_OK;
}

int hs_set_spins(hs_lattice *h, const double *xyz) {
    if (!h || !xyz) return fail(HS_E_INVALID, "null argument");
    int st = ensure_stage(h);
    if (st) return st;
    HS_CUDA(cudaMemcpyAsync(h->stage, xyz, (size_t)h->L.n_sites * 3 * sizeof(double), cudaMemcpyHostToDevice,
                            h->stream));
    if ((st = hs_set_spins_device(h, h->stage))) return st;
    HS_CUDA(cudaStreamSynchronize(h->stream));
    return HS_OK;
}

// The upload buffers, copy stream and events of hs_set_spins_async, made on
// the first call (the only one that allocates).
static int ensure_upload(hs_lattice *h) {
    if (h->up_stream) return HS_OK;
    const size_t bytes = (size_t)std::max<int64_t>(h->L.n_sites, 1) * 3 * sizeof(double);
    for (int b = 0; b < 2; ++b) {  // a failed set-up keeps what it made for the next try
        cudaError_t e = cudaSuccess;
        if (!h->up_buf[b]) {
            void *p_ = nullptr;
            e = cudaMalloc(&p_, bytes);
            if (e == cudaSuccess) h->up_buf[b] = p_;
        }
        if (e == cudaSuccess && !h->up_filled[b]) e = cudaEventCreateWithFlags(&h->up_filled[b], cudaEventDisableTiming);
        if (e == cudaSuccess && !h->up_free[b]) e = cudaEventCreateWithFlags(&h->up_free[b], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "hs_set_spins_async set-up");
    }
    cudaError_t e = cudaStreamCreateWithFlags(&h->up_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        h->up_stream = nullptr;
        return cuda_fail(e, "cudaStreamCreate(upload)");
    }
    return HS_OK;
}

int hs_set_spins_async(hs_lattice *h, const void *xyz, int dtype) {
    if (!h || !xyz) return fail(HS_E_INVALID, "null argument");
    if (dtype != HS_FP64 && dtype != HS_FP32) return fail(HS_E_INVALID, "dtype must be HS_FP64 or HS_FP32");
    int st = ensure_upload(h);
    if (st) return st;
    if (h->L.n_present == 0) return HS_OK;
    const int b = h->up_next;
    h->up_next ^= 1;
    const size_t bytes = (size_t)h->L.n_sites * 3 * (dtype == HS_FP64 ? sizeof(double) : sizeof(float));
    // the copy may start once the conversion that last read this buffer is done
    HS_CUDA(cudaStreamWaitEvent(h->up_stream, h->up_free[b], 0));
    HS_CUDA(cudaMemcpyAsync(h->up_buf[b], xyz, bytes, cudaMemcpyHostToDevice, h->up_stream));
    HS_CUDA(cudaEventRecord(h->up_filled[b], h->up_stream));
    // the conversion into the layout follows the work already on the handle's stream
    HS_CUDA(cudaStreamWaitEvent(h->stream, h->up_filled[b], 0));
    if (dtype == HS_FP64)
        HS_CUDA(hs::launch_scatter(h->precision, h->L, (const double *)h->up_buf[b], h->stream));
    else
        HS_CUDA(hs::launch_scatter_f32(h->precision, h->L, (const float *)h->up_buf[b], h->stream));
    HS_CUDA(cudaEventRecord(h->up_free[b], h->stream));
    return HS_OK;
}

int hs_set_sweep_counter(hs_lattice *h, uint64_t sweep) {
    if (!h) return fail(HS_E_INVALID, "null handle");
    h->sweep = sweep;
    return HS_OK;
}

int hs_get_info(const hs_lattice *h, hs_info *out) {
    if (!h || !out) return fail(HS_E_INVALID, "null argument");
    out->type = h->type;
    out->precision = h->precision;
    out->n_colours = h->L.n_colours;
    out->structured = h->L.structured ? 1 : 0;
    out->n_sites = h->L.n_sites;
    out->n_present = h->L.n_present;
    out->device_bytes = h->device_bytes;
    out->sweep = h->sweep;
    out->fold_sweeps = h->fold_ring;
    return HS_OK;
}

int hs_enable_timing(hs_lattice *h, int on) {
    if (!h) return fail(HS_E_INVALID, "null handle");
    int st = flush_timing(h);
    if (st) return st;
    h->timing = on != 0;
    h->timed_ms = 0.0;
    h->timed_launches = 0;
    return HS_OK;
}

int hs_read_timing(hs_lattice *h, double *ms, int64_t *launches) {
    if (!h || !ms || !launches) return fail(HS_E_INVALID, "null argument");
    int st = flush_timing(h);
    if (st) return st;
    *ms = h->timed_ms;
    *launches = h->timed_launches;
    return HS_OK;
}

// ---------------------------------------------------------------- launch configuration
int hs_set_launch(hs_lattice *h, const hs_launch *cfg) {
    if (!h || !cfg) return fail(HS_E_INVALID, "null argument");
    if (cfg->kernel != HS_KERNEL_AUTO && cfg->kernel != HS_KERNEL_STENCIL && cfg->kernel != HS_KERNEL_TABLE &&
        cfg->kernel != HS_KERNEL_MARCH && cfg->kernel != HS_KERNEL_PIPE)
        return fail(HS_E_INVALID, "unknown kernel kind");
    if (h->L.slab && cfg->kernel != HS_KERNEL_AUTO && cfg->kernel != HS_KERNEL_STENCIL)
        return fail(HS_E_INVALID, "a slab runs the register stencil");
    if (h->L.structured) {
        if (cfg->kernel == HS_KERNEL_TABLE) return fail(HS_E_INVALID, "sc stencil lattices have no table kernel");
        if (cfg->vec_width != 0 && !vec_ok(h, cfg->vec_width))
            return fail(HS_E_INVALID, "vector width must divide Lx/2, 16 bytes at most");
    } else if (cfg->kernel == HS_KERNEL_STENCIL || cfg->kernel == HS_KERNEL_MARCH || cfg->kernel == HS_KERNEL_PIPE) {
        return fail(HS_E_INVALID, "stencil kernels need an unmasked periodic sc lattice");
    }
    if (cfg->blocks_per_sm < 0 || cfg->blocks_per_sm > 2048 / hs::kBlock)
        return fail(HS_E_INVALID, "blocks_per_sm out of range");
    if (cfg->tile_y < 0) return fail(HS_E_INVALID, "negative tile_y");
    if (cfg->prefetch < 0 || cfg->prefetch > 3) return fail(HS_E_INVALID, "prefetch must be 0, 1, 2 or 3");
    if (cfg->order < 0 || cfg->order > 2) return fail(HS_E_INVALID, "order must be 0, 1 or 2");
    const hs_launch keep = h->req;
    const Layout keep_l = h->L;
    const int keep_b = h->n_blocks;
    h->req = *cfg;
    int st = configure_launch(h);
    if (st) {
        h->req = keep;
        h->L = keep_l;
        h->n_blocks = keep_b;
    }
    return st;
}

int hs_set_anisotropy_tensor(hs_lattice *h, const double A[6]) {
    if (!h) return fail(HS_E_INVALID, "null handle");
    double t[6] = {0, 0, 0, 0, 0, 0};
    if (A)
        for (int q = 0; q < 6; ++q) {
            if (!std::isfinite(A[q])) return fail(HS_E_INVALID, "tensor entries must be finite");
            t[q] = A[q];
        }
    int on = 0;
    for (int q = 0; q < 6; ++q) on |= (t[q] != 0.0);
    const int keep_on = h->tensor;
    double keep_t[6];
    for (int q = 0; q < 6; ++q) keep_t[q] = h->tA[q];
    const hs_launch keep_req = h->req;
    const Layout keep_l = h->L;
    const int keep_b = h->n_blocks;
    h->tensor = on;
    for (int q = 0; q < 6; ++q) h->tA[q] = t[q];
    h->req = hs_launch{};  // back to the automatic launch, which takes the tensor into account
    int st = configure_launch(h);
    if (st) {
        h->tensor = keep_on;
        for (int q = 0; q < 6; ++q) h->tA[q] = keep_t[q];
        h->req = keep_req;
        h->L = keep_l;
        h->n_blocks = keep_b;
    }
    return st;
}

int hs_get_anisotropy_tensor(const hs_lattice *h, double A[6]) {
    if (!h || !A) return fail(HS_E_INVALID, "null argument");
    for (int q = 0; q < 6; ++q) A[q] = h->tensor ? h->tA[q] : 0.0;
    return HS_OK;
}

int hs_get_launch(const hs_lattice *h, hs_launch *out) {
    if (!h || !out) return fail(HS_E_INVALID, "null argument");
    const Layout &L = h->L;
    out->kernel = L.kernel;
    out->vec_width = L.structured ? L.vec : 1;
    out->blocks_per_sm = (h->n_blocks + h->n_sm - 1) / std::max(h->n_sm, 1);
    out->tile_y = L.kernel == hs::kMarch ? L.ty : 0;
    out->prefetch = (L.kernel == hs::kStencil || L.kernel == hs::kTable)
                        ? (L.prefetch == 1 ? 1 : (L.prefetch == 2 ? 3 : 2))
                        : 0;
    out->order = L.kernel == hs::kStencil ? L.order : 0;
    return HS_OK;
}

namespace {
struct TuneKey {
    int precision, structured, accumulate, tensor;
    int64_t a, b, c, d;
    bool operator<(const TuneKey &o) const {
        return std::tie(precision, structured, accumulate, tensor, a, b, c, d) <
               std::tie(o.precision, o.structured, o.accumulate, o.tensor, o.a, o.b, o.c, o.d);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, hs_launch> g_tune_cache;

// Candidate configurations of one lattice.
std::vector<hs_launch> tune_candidates(hs_lattice *h) {
    std::vector<hs_launch> out;
    const Layout &L = h->L;
    if (!L.structured) {
        for (int b = 1; b <= 8; ++b)
            for (int pf : {1, 2}) out.push_back({HS_KERNEL_TABLE, 1, b, 0, pf});
        return out;
    }
    for (int v : {1, 2, 4, 8}) {
        if (!vec_ok(h, v)) continue;
        for (int b = 1; b <= 8; ++b)
            for (int pf : {1, 2, 3}) out.push_back({HS_KERNEL_STENCIL, v, b, 0, pf});
        if (hs::pipe_smem_bytes(h->precision, v) != 0)
            for (int b = 1; b <= 2; ++b) out.push_back({HS_KERNEL_PIPE, v, b, 0, 0});
        for (int ty : {2, 4, 8, 16})
            if (L.Ly % ty == 0 && ty * (L.Lh / v) >= 64)
                for (int b : {1, 2}) out.push_back({HS_KERNEL_MARCH, v, b, ty, 0});
    }
    return out;
}
}  // namespace

int hs_autotune(hs_lattice *h, double beta, int n_trial_sweeps) {
    if (!h) return fail(HS_E_INVALID, "null handle");
    if (n_trial_sweeps < 1) return fail(HS_E_INVALID, "n_trial_sweeps must be >= 1");
    if (h->L.n_present == 0 || h->L.slab) return HS_OK;  // a slab keeps the register stencil
    const Layout &L = h->L;
    const TuneKey key{h->precision, L.structured ? 1 : 0, h->accumulate, h->tensor, L.structured ? L.Lx : L.n_present,
                      L.structured ? L.Ly : L.width, L.structured ? L.Lz : L.n_colours, h->n_sm};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) return hs_set_launch(h, &it->second);
    }
    // save state: spins, accumulator, sweep counter
    const size_t es = hs::storage_size(h->precision);
    void *state = L.structured ? L.planes : L.spins4;
    const size_t bytes = L.structured ? (size_t)L.Lz * L.Ly * L.Lh * 6 * es : (size_t)L.n_pad * 4 * es;
    void *saved = nullptr;
    HS_CUDA(cudaMalloc(&saved, bytes));
    DevAccum acc_saved;
    const uint64_t sweep_saved = h->sweep;
    const int64_t last_saved = h->last_n_sweeps;
    const bool timing_saved = h->timing;
    const hs_launch req_saved = h->req;
    h->timing = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best_ms = 1e30f;
    hs_launch best = h->req;
    // every candidate runs the same sweeps from the same state (the acceptance
    // rate, and with it the store traffic, drifts along a chain); the three
    // fastest are timed again over twice the sweeps
    auto trial = [&](const hs_launch &cand, int n, float &ms) -> int {
        HS_CUDA(cudaMemcpyAsync(state, saved, bytes, cudaMemcpyDeviceToDevice, h->stream));
        h->sweep = sweep_saved;
        int r;
        if ((r = hs_sweep(h, beta, 1))) return r;  // warm-up
        HS_CUDA(cudaEventRecord(e0, h->stream));
        if ((r = hs_sweep(h, beta, n))) return r;
        HS_CUDA(cudaEventRecord(e1, h->stream));
        HS_CUDA(cudaEventSynchronize(e1));
        HS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        (void)cand;
        return HS_OK;
    };
    auto run = [&]() -> int {
        HS_CUDA(cudaMemcpyAsync(saved, state, bytes, cudaMemcpyDeviceToDevice, h->stream));
        HS_CUDA(cudaMemcpyAsync(&acc_saved, h->acc, sizeof(DevAccum), cudaMemcpyDeviceToHost, h->stream));
        HS_CUDA(cudaStreamSynchronize(h->stream));
        HS_CUDA(cudaEventCreate(&e0));
        HS_CUDA(cudaEventCreate(&e1));
        std::vector<std::pair<float, hs_launch>> timed;
        for (const hs_launch &cand : tune_candidates(h)) {
            if (hs_set_launch(h, &cand) != HS_OK) continue;  // e.g. more CTAs per SM than fit
            float ms = 0.f;
            if (int r = trial(cand, n_trial_sweeps, ms)) return r;
            timed.push_back({ms, cand});
        }
        std::stable_sort(timed.begin(), timed.end(),
                         [](const std::pair<float, hs_launch> &x, const std::pair<float, hs_launch> &y) {
                             return x.first < y.first;
                         });
        for (size_t i = 0; i < timed.size() && i < 3; ++i) {
            if (hs_set_launch(h, &timed[i].second) != HS_OK) continue;
            float ms = 0.f;
            if (int r = trial(timed[i].second, 2 * n_trial_sweeps, ms)) return r;
            if (ms < best_ms) {
                best_ms = ms;
                best = timed[i].second;
            }
        }
        return HS_OK;
    };
    int st = run();
    // restore the chain exactly
    cudaMemcpyAsync(state, saved, bytes, cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync(h->acc, &acc_saved, sizeof(DevAccum), cudaMemcpyHostToDevice, h->stream);
    cudaStreamSynchronize(h->stream);
    cudaFree(saved);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    h->sweep = sweep_saved;
    h->last_n_sweeps = last_saved;
    h->timing = timing_saved;
    if (st) {
        hs_set_launch(h, &req_saved);
        return st;
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    return hs_set_launch(h, &best);
}

// ---------------------------------------------------------------- batch
struct hs_batch {
    std::vector<hs_lattice *> members;
    cudaStream_t stream = nullptr;
    int grid = 0, n_segs = 0;
    std::vector<hs::BatchMember> host_members;
    hs::BatchMember *d_members = nullptr;
    hs::BatchSeg *d_segs = nullptr;
    int *d_cta_seg = nullptr;
    double *d_slots = nullptr;
    unsigned int *d_bar = nullptr;
    int *d_error = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_total = -1, graph_equil = -1;
    bool graph_failed = false;
    int inject_timeout = 0;  // test hook, consumed by the next run
    int occ = 1, ctas_per_sm = 1, align_rows = 0;  // work split (batch_layout)
    int prefetch = 0;                              // 1: split prefetch variant of the kernel
    int schedule = 0;                              // 0: one persistent launch, 1: a launch per colour pass,
                                                   // 2: resident (one CTA per member, in shared memory)
    size_t resident_bytes = 0;                     // the largest member's six planes
    int precision = HS_FP32;                       // every member's
    ~hs_batch() {
        cudaStreamSynchronize(stream);
        if (exec) cudaGraphExecDestroy(exec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        cudaFree(d_members);
        cudaFree(d_segs);
        cudaFree(d_cta_seg);
        cudaFree(d_slots);
        cudaFree(d_bar);
        cudaFree(d_error);
    }
};

namespace {
hs::BatchArgs batch_args(const hs_batch *b, int n_total, int n_equil) {
    hs::BatchArgs a{};
    a.members = b->d_members;
    a.n_members = (int)b->members.size();
    a.segs = b->d_segs;
    a.cta_seg = b->d_cta_seg;
    a.n_segs = b->n_segs;
    a.slots = b->d_slots;
    a.bar = b->d_bar;
    a.error = b->d_error;
    a.n_total = n_total;
    a.n_equil = n_equil;
    a.zaxis_all = 1;
    a.kzero_all = 1;
    for (const hs::BatchMember &m : b->host_members) {
        a.zaxis_all &= m.zaxis;
        a.kzero_all &= (m.K == 0.0 && !std::signbit(m.K)) ? 1 : 0;
    }
    return a;
}
}  // namespace

namespace {
// Work split of a batch (the batch's tile shape): the members' work items (4
// sites of one row of one colour), concatenated, are cut into one contiguous
// range per CTA, ctas_per_sm CTAs per SM; with align_rows the cuts are moved
// to the nearest row boundary of the member they fall in, so no row is split
// between two CTAs.  Segment = (CTA, member) piece, with its own FP64 slot.
// Interleaved split (align_rows 2): a contiguous split at whole blocks of
// kBlock items, cut at equal estimated cost per CTA (an item of a member with
// r work items per row weighs 1 + 3 / r: on the 64-replica batch of L = 16 ...
// 96, weights of 1 + 2 / r, 1 + 3 / r and 1 + 4.5 / r measured 133.7, 136.4
// and 135.9 attempts/ns, equal weights 128.1), then, within each member, the blocks of the CTAs that hold
// nothing but that member are dealt out to them round-robin (CTA j of G takes
// blocks j, j + G, ...), so those CTAs sweep the member side by side in
// grid-stride order, as one lattice's grid-stride loop does, instead of on
// separate fronts; a CTA shared with another member keeps its contiguous
// piece.  Every CTA keeps its share (to within one block).  segs come
// out member by member in ascending CTA order, seg_cta holds each one's CTA.
void interleaved_layout(int grid, const std::vector<int64_t> &items, const std::vector<int64_t> &row,
                        std::vector<hs::BatchSeg> &segs, std::vector<int> &seg_cta) {
    const int n = (int)items.size();
    const int64_t K = hs::kBlock;
    std::vector<int64_t> nb(n), A(n + 1, 0);
    std::vector<double> w(n), cw(n + 1, 0.0);
    for (int m = 0; m < n; ++m) {
        nb[m] = (items[m] + K - 1) / K;
        A[m + 1] = A[m] + nb[m];
        // estimated cost of an item: short rows (small members) cost more per
        // site (their operands stay in L2 latency, their rows have more edges)
        w[m] = 1.0 + 3.0 / (double)row[m];
        cw[m + 1] = cw[m] + (double)nb[m] * w[m];
    }
    const int64_t B = A[n];
    // cut points in blocks at equal estimated cost per CTA
    std::vector<int64_t> cut(grid + 1, 0);
    for (int c = 1, m = 0; c < grid; ++c) {
        const double T = (double)c * cw[n] / grid;
        while (m < n - 1 && cw[m + 1] <= T) ++m;
        const int64_t blk = A[m] + (int64_t)((T - cw[m]) / w[m] + 0.5);
        cut[c] = std::min(B, std::max(cut[c - 1], blk));
    }
    cut[grid] = B;
    int c = 0;
    for (int m = 0; m < n; ++m) {
        const int64_t a0 = A[m], a1 = A[m + 1];
        while (cut[c + 1] <= a0) ++c;
        struct Piece { int cta; int64_t p0, p1; bool full; };
        std::vector<Piece> pieces;
        for (int cc = c; cc < grid && cut[cc] < a1; ++cc) {
            const int64_t p0 = std::max(cut[cc], a0), p1 = std::min(cut[cc + 1], a1);
            if (p1 > p0) pieces.push_back({cc, p0, p1, p0 == cut[cc] && p1 == cut[cc + 1]});
        }
        int G = 0;
        int64_t F0 = 0, F1 = 0;
        for (const Piece &p : pieces)
            if (p.full) {
                if (G == 0) F0 = p.p0;
                F1 = p.p1;
                ++G;
            }
        int j = 0;
        for (const Piece &p : pieces) {
            if (p.full && G >= 2) {
                segs.push_back({m, (uint32_t)((F0 - a0 + j) * K), (uint32_t)std::min((F1 - a0) * K, items[m]),
                                (uint32_t)(G * K)});
                ++j;
            } else {
                segs.push_back({m, (uint32_t)((p.p0 - a0) * K), (uint32_t)std::min((p.p1 - a0) * K, items[m]),
                                (uint32_t)K});
            }
            seg_cta.push_back(p.cta);
        }
    }
}

int batch_layout(hs_batch *b, int ctas_per_sm, int align_rows) {
    const int n = (int)b->members.size();
    const int grid = b->members[0]->n_sm * ctas_per_sm;
    std::vector<int64_t> items(n), offset(n + 1, 0), row(n);
    for (int r = 0; r < n; ++r) {
        const Layout &L = b->members[r]->L;
        row[r] = L.Lh / hs::batch_vec(b->precision);
        items[r] = (int64_t)L.Lz * L.Ly * row[r];
        offset[r + 1] = offset[r] + items[r];
    }
    const int64_t total = offset[n];
    std::vector<hs::BatchSeg> segs;
    std::vector<int> cta_seg(grid + 1, 0);
    if (align_rows == 2) {
        // segments member by member and in ascending CTA order: each CTA's and
        // each member's are contiguous (kernel and finalise)
        std::vector<int> seg_cta;
        interleaved_layout(grid, items, row, segs, seg_cta);
        for (int m = 0; m < n; ++m) b->host_members[m].seg_begin = b->host_members[m].seg_end = 0;
        for (size_t k = 0; k < segs.size(); ++k) {
            hs::BatchMember &hm = b->host_members[segs[k].member];
            if (k == 0 || segs[k - 1].member != segs[k].member) hm.seg_begin = (int)k;
            hm.seg_end = (int)k + 1;
            ++cta_seg[seg_cta[k] + 1];
        }
    } else {
    const int64_t chunk = (total + grid - 1) / grid;
    std::vector<int64_t> bnd(grid + 1);
    bnd[0] = 0;
    bnd[grid] = total;
    int r = 0;
    for (int c = 1; c < grid; ++c) {
        int64_t pos = std::min<int64_t>((int64_t)c * chunk, total);
        if (align_rows && pos < total) {
            while (offset[r + 1] <= pos) ++r;
            const int64_t rel = pos - offset[r];
            pos = offset[r] + std::min<int64_t>(items[r], (rel + row[r] / 2) / row[r] * row[r]);
        }
        bnd[c] = std::max(pos, bnd[c - 1]);
    }
    int c = 0;
    for (int m = 0; m < n; ++m) {
        b->host_members[m].seg_begin = (int)segs.size();
        for (int64_t g = offset[m]; g < offset[m + 1];) {
            while (bnd[c + 1] <= g) ++c;
            const int64_t g_end = std::min(offset[m + 1], bnd[c + 1]);
            segs.push_back({m, (uint32_t)(g - offset[m]), (uint32_t)(g_end - offset[m]), (uint32_t)hs::kBlock});
            ++cta_seg[c + 1];
            g = g_end;
        }
        b->host_members[m].seg_end = (int)segs.size();
    }
    }
    for (int k = 0; k < grid; ++k) cta_seg[k + 1] += cta_seg[k];
    HS_CUDA(cudaStreamSynchronize(b->stream));
    cudaFree(b->d_segs);
    cudaFree(b->d_cta_seg);
    cudaFree(b->d_slots);
    b->d_segs = nullptr;
    b->d_cta_seg = nullptr;
    b->d_slots = nullptr;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    b->graph_total = b->graph_equil = -1;
    b->grid = grid;
    b->n_segs = (int)segs.size();
    b->ctas_per_sm = ctas_per_sm;
    b->align_rows = align_rows;
    cudaError_t e;
    if ((e = cudaMalloc(&b->d_segs, sizeof(hs::BatchSeg) * segs.size())) != cudaSuccess ||
        (e = cudaMalloc(&b->d_cta_seg, sizeof(int) * cta_seg.size())) != cudaSuccess ||
        (e = cudaMalloc(&b->d_slots, sizeof(double) * 4 * segs.size() * hs::kPartials)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(batch)");
    if ((e = cudaMemcpyAsync(b->d_segs, segs.data(), sizeof(hs::BatchSeg) * segs.size(), cudaMemcpyHostToDevice,
                             b->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b->d_cta_seg, cta_seg.data(), sizeof(int) * cta_seg.size(), cudaMemcpyHostToDevice,
                             b->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
        return cuda_fail(e, "batch upload");
    return HS_OK;
}
}  // namespace

namespace {
constexpr int kResidentMinMembers = 16;  // hs_batch_create's choice of the resident schedule
}  // namespace

int hs_batch_create(hs_batch **out, hs_lattice *const *members, int n_members) {
    if (!out) return fail(HS_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!members || n_members < 1) return fail(HS_E_INVALID, "need at least one member");
    for (int r = 0; r < n_members; ++r) {
        const hs_lattice *h = members[r];
        if (!h) return fail(HS_E_INVALID, "null member");
        if (h->stream != members[0]->stream || h->device != members[0]->device)
            return fail(HS_E_INVALID, "members must share one stream and device");
        if (!h->L.structured || h->L.slab || h->L.Lh % hs::batch_vec(h->precision) != 0)
            return fail(HS_E_INVALID,
                        "batch members must be unmasked periodic sc with Lx divisible by 8 (FP32, FP16) or 4 (FP64)");
        if (h->precision != members[0]->precision) return fail(HS_E_INVALID, "batch members must share one precision");
        if (h->tensor) return fail(HS_E_INVALID, "batch members take no anisotropy tensor term");
        for (int q = 0; q < r; ++q)
            if (members[q] == h) return fail(HS_E_INVALID, "a lattice appears twice in the batch");
    }
    const int precision = members[0]->precision;
    const int occ = std::min(hs::batch_occupancy(precision, 0), hs::batch_occupancy(precision, 1));
    if (occ < 1) return fail(HS_E_CUDA, "batch kernel does not fit on an SM");
    hs_batch *b = new (std::nothrow) hs_batch();
    if (!b) return fail(HS_E_OOM, "host allocation failed");
    b->members.assign(members, members + n_members);
    b->stream = members[0]->stream;
    b->precision = precision;
    b->occ = occ;
    b->host_members.resize(n_members);
    for (int r = 0; r < n_members; ++r) {
        hs::BatchMember &m = b->host_members[r];
        const hs_lattice *h = members[r];
        const Layout &L = h->L;
        m.planes = L.planes;
        m.Lx = L.Lx;
        m.Ly = L.Ly;
        m.Lz = L.Lz;
        m.Lh = L.Lh;
        m.div_nxv = hs::FastDiv((uint32_t)(L.Lh / hs::batch_vec(precision)));
        m.div_ly = hs::FastDiv((uint32_t)L.Ly);
        m.fJ = (float)h->p.J;
        m.fK = (float)h->p.K;
        m.J = h->p.J;
        m.K = h->p.K;
        for (int q = 0; q < 3; ++q) {
            m.fe[q] = (float)h->p.e[q];
            m.e[q] = h->p.e[q];
        }
        m.sc_tab = h->sc_tab;
        m.zaxis = (h->p.e[0] == 0.0 && h->p.e[1] == 0.0 && h->p.e[2] == 1.0) ? 1 : 0;
        m.key0 = (uint32_t)h->seed;
        m.key1 = (uint32_t)(h->seed >> 32);
        m.replica = h->replica;
        m.n_present = (double)L.n_present;
        m.acc = h->acc;
        b->resident_bytes = std::max(b->resident_bytes, (size_t)6 * L.Lz * L.Ly * L.Lh * hs::storage_size(precision));
    }
    cudaError_t e;
    if ((e = cudaMalloc(&b->d_members, sizeof(hs::BatchMember) * n_members)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_bar, 2 * sizeof(unsigned int))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_error, sizeof(int))) != cudaSuccess) {
        delete b;
        return cuda_fail(e, "cudaMalloc(batch)");
    }
    if ((e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        delete b;
        return cuda_fail(e, "cudaStreamCreate");
    }
    if (int st = batch_layout(b, occ, 2)) {  // the interleaved split, measured fastest on every tested batch
        delete b;
        return st;
    }
    // many small members: the resident schedule (measured 3.2x the persistent one on 304 members of 16^3,
    // 2.5x on 152 of 24^3, 1.2x on 16 of 24^3, which leave most SMs idle)
    if (n_members >= kResidentMinMembers && b->resident_bytes <= hs::batch_resident_limit(precision)) b->schedule = 2;
    *out = b;
    return HS_OK;
}

int hs_batch_run(hs_batch *b, const double *betas, int64_t n_sweeps, int64_t n_equil) {
    if (!b || !betas) return fail(HS_E_INVALID, "null argument");
    if (n_sweeps < 0 || n_equil < 0 || n_sweeps + n_equil > (int64_t)1 << 30)
        return fail(HS_E_INVALID, "sweep counts must be >= 0 and below 2^30");
    const int n = (int)b->members.size();
    for (int r = 0; r < n; ++r)
        if (!(betas[r] >= 0.0) || !std::isfinite(betas[r])) return fail(HS_E_INVALID, "betas must be finite, >= 0");
    const int n_total = (int)(n_sweeps + n_equil), n_eq = (int)n_equil;
    for (int r = 0; r < n; ++r) {
        hs_lattice *h = b->members[r];
        b->host_members[r].fbeta = (float)betas[r];
        b->host_members[r].beta = betas[r];
        b->host_members[r].sweep0 = (uint32_t)h->sweep;
        h->last_n_sweeps = n_total;
    }
    HS_CUDA(cudaMemcpyAsync(b->d_members, b->host_members.data(), sizeof(hs::BatchMember) * n,
                            cudaMemcpyHostToDevice, b->stream));
    hs::BatchArgs args = batch_args(b, n_total, n_eq);
    HS_CUDA(hs::launch_batch_reset(args, b->stream));  // the accepted counts cover this run's sweeps
    if (n_total == 0) return HS_OK;
    HS_CUDA(cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned int), b->stream));
    HS_CUDA(cudaMemsetAsync(b->d_error, 0, sizeof(int), b->stream));
    if (b->schedule == 1 && !b->inject_timeout) {  // chained launches on the stream, no graph
        HS_CUDA(hs::launch_batch_passes(b->precision, args, b->grid, b->stream, b->prefetch));
        for (int r = 0; r < n; ++r) b->members[r]->sweep += (uint64_t)n_total;
        return HS_OK;
    }
    if (b->inject_timeout) {  // test hook: launched directly, never captured
        args.inject_skip = 1;
        b->inject_timeout = 0;
        HS_CUDA(hs::launch_batch(b->precision, args, b->grid, b->stream, b->prefetch));
        for (int r = 0; r < n; ++r) b->members[r]->sweep += (uint64_t)n_total;
        return HS_OK;
    }
    if (b->schedule == 2) {  // one launch: every member resident in its CTA's shared memory
        HS_CUDA(hs::launch_batch_resident(b->precision, args, b->resident_bytes, b->stream));
        for (int r = 0; r < n; ++r) b->members[r]->sweep += (uint64_t)n_total;
        return HS_OK;
    }
    // the persistent kernel runs as one node of a CUDA graph, captured once per
    // (sweeps, equilibration) pair; without graph support it is launched directly
    if (!b->graph_failed && (b->graph_total != n_total || b->graph_equil != n_eq || !b->exec)) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        bool ok = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            const cudaError_t le = hs::launch_batch(b->precision, args, b->grid, b->cap_stream, b->prefetch);
            ok = (cudaStreamEndCapture(b->cap_stream, &graph) == cudaSuccess) && le == cudaSuccess;
        }
        if (ok) ok = cudaGraphInstantiate(&b->exec, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        if (!ok) {
            cudaGetLastError();
            b->exec = nullptr;
            b->graph_failed = true;
        } else {
            b->graph_total = n_total;
            b->graph_equil = n_eq;
        }
    }
    if (b->exec) {
        HS_CUDA(cudaGraphLaunch(b->exec, b->stream));
    } else {
        HS_CUDA(hs::launch_batch(b->precision, args, b->grid, b->stream, b->prefetch));
    }
    for (int r = 0; r < n; ++r) b->members[r]->sweep += (uint64_t)n_total;
    return HS_OK;
}

// Batch autotuner: time every work split (1 .. occupancy CTAs per SM, cuts
// at any item or at row boundaries), load schedule and colour schedule, and
// the resident schedule where every member fits one CTA's shared memory, for
// n_trial_sweeps sweeps after one warm-up sweep, keep the fastest, and put
// every member's spins, sweep counter and accumulator back as they were.
int hs_batch_autotune(hs_batch *b, const double *betas, int n_trial_sweeps) {
    if (!b || !betas) return fail(HS_E_INVALID, "null argument");
    if (n_trial_sweeps < 1) return fail(HS_E_INVALID, "n_trial_sweeps must be >= 1");
    const int n = (int)b->members.size();
    struct Saved {
        void *planes = nullptr;
        size_t bytes = 0;
        uint64_t sweep = 0;
        int64_t last_n = 0;
        DevAccum acc{};
    };
    std::vector<Saved> saved(n);
    auto release = [&]() {
        for (Saved &sv : saved) cudaFree(sv.planes);
    };
    for (int r = 0; r < n; ++r) {
        hs_lattice *h = b->members[r];
        const Layout &L = h->L;
        saved[r].bytes = (size_t)6 * L.Lz * L.Ly * L.Lh * hs::storage_size(b->precision);
        saved[r].sweep = h->sweep;
        saved[r].last_n = h->last_n_sweeps;
        cudaError_t e = cudaMalloc(&saved[r].planes, saved[r].bytes);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(saved[r].planes, L.planes, saved[r].bytes, cudaMemcpyDeviceToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&saved[r].acc, h->acc, sizeof(DevAccum), cudaMemcpyDeviceToHost, b->stream);
        if (e != cudaSuccess) {
            release();
            return cuda_fail(e, "batch autotune backup");
        }
    }
    auto restore = [&]() -> int {
        for (int r = 0; r < n; ++r) {
            hs_lattice *h = b->members[r];
            HS_CUDA(cudaMemcpyAsync(h->L.planes, saved[r].planes, saved[r].bytes, cudaMemcpyDeviceToDevice,
                                    b->stream));
            HS_CUDA(cudaMemcpyAsync(h->acc, &saved[r].acc, sizeof(DevAccum), cudaMemcpyHostToDevice, b->stream));
            h->sweep = saved[r].sweep;
            h->last_n_sweeps = saved[r].last_n;
        }
        HS_CUDA(cudaStreamSynchronize(b->stream));
        return HS_OK;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = HS_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = fail(HS_E_CUDA, "events");
    int best_c = b->ctas_per_sm, best_a = b->align_rows, best_pf = b->prefetch, best_sc = b->schedule;
    float best_ms = 0.f;
    bool have = false;
    if (st == HS_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) st = fail(HS_E_CUDA, "synchronise");
    const int max_sc = b->resident_bytes <= hs::batch_resident_limit(b->precision) ? 2 : 1;
    for (int sc = 0; st == HS_OK && sc <= max_sc; ++sc)
    for (int pf = 0; st == HS_OK && pf <= (sc == 2 ? 0 : 1); ++pf)
    for (int c = (sc == 2 ? b->occ : 1); st == HS_OK && c <= b->occ; ++c)
        for (int al = (sc == 2 ? 2 : 0); st == HS_OK && al <= 2; ++al) {  // the resident schedule: one candidate
            b->prefetch = pf;
            b->schedule = sc;
            if ((st = batch_layout(b, c, al))) break;
            if ((st = hs_batch_run(b, betas, 1, 0))) break;
            if ((st = hs_batch_run(b, betas, n_trial_sweeps, 0))) break;  // graph capture for this count
            cudaEventRecord(e0, b->stream);
            if ((st = hs_batch_run(b, betas, n_trial_sweeps, 0))) break;
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = fail(HS_E_CUDA, "batch autotune timing");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (!have || ms < best_ms) {
                have = true;
                best_ms = ms;
                best_c = c;
                best_a = al;
                best_pf = pf;
                best_sc = sc;
            }
            if ((st = restore())) break;
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    b->prefetch = best_pf;
    b->schedule = best_sc;
    if (st == HS_OK) st = batch_layout(b, best_c, best_a);
    const int st2 = restore();
    release();
    return st ? st : st2;
}

int hs_batch_set_layout(hs_batch *b, int ctas_per_sm, int align_rows, int prefetch, int schedule) {
    if (!b) return fail(HS_E_INVALID, "null handle");
    if (ctas_per_sm < 1 || ctas_per_sm > b->occ) return fail(HS_E_INVALID, "ctas_per_sm out of range");
    if (align_rows < 0 || align_rows > 2 || (prefetch != 0 && prefetch != 1) || schedule < 0 || schedule > 2)
        return fail(HS_E_INVALID, "align_rows must be 0, 1 or 2, prefetch 0 or 1, schedule 0, 1 or 2");
    if (schedule == 2 && b->resident_bytes > hs::batch_resident_limit(b->precision))
        return fail(HS_E_INVALID, "the resident schedule needs every member's spins in one CTA's shared memory");
    b->prefetch = prefetch;
    b->schedule = schedule;
    return batch_layout(b, ctas_per_sm, align_rows);
}

int hs_batch_get_layout(const hs_batch *b, int *ctas_per_sm, int *align_rows, int *prefetch, int *schedule) {
    if (!b || !ctas_per_sm || !align_rows || !prefetch || !schedule) return fail(HS_E_INVALID, "null argument");
    *ctas_per_sm = b->ctas_per_sm;
    *align_rows = b->align_rows;
    *prefetch = b->prefetch;
    *schedule = b->schedule;
    return HS_OK;
}

void hs_batch_destroy(hs_batch *b) { delete b; }

int hs_batch_inject_timeout(hs_batch *b, int on) {
    if (!b) return fail(HS_E_INVALID, "null handle");
    b->inject_timeout = on ? 1 : 0;
    return HS_OK;
}

}  // extern "C"
