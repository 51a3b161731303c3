/*
 * hs.h -- C ABI of the GB300 single-spin Metropolis library for the classical
 * anisotropic Heisenberg model (arXiv 2106.11286).
 *
 * The method (all citations are to the paper):
 *   Eq. 1   H = -J sum_<ij> S_i.S_j - K sum_i (S_i.e)^2, |S_i| = 1, each
 *           nearest-neighbour bond counted once, e the uniaxial easy axis.
 *   Metropolis steps (i)-(iii): pick a site, propose a random orientation,
 *           accept if dH <= 0, else accept iff P <= exp(-beta dH), P uniform
 *           in [0,1).
 *   Eq. 2   M = (1 / (N |S|)) sum_i S_i with N the number of present spins.
 *   Optional on-site tensor term -sum_i S_i^T A S_i (one symmetric 3x3 A
 *           for all sites): the effective shape anisotropy the paper offers
 *           in place of dipolar coupling (introduction), read as a general
 *           quadratic on-site anisotropy; see hs_set_anisotropy_tensor.
 *
 * Parallel decomposition (the paper's own racy block scheme is replaced):
 * the neighbour graph is split into colour classes (independent sets); a
 * sweep updates class 0, then class 1, ..., each class fully in parallel.
 * Sites inside a class share no bond and random numbers are keyed by site,
 * so the result of a class update does not depend on the visiting order.
 *   sc:  2 classes, colour = (x+y+z) mod 2  (periodic dims must be even)
 *   bcc: 2 classes, colour = basis index (0 cube corner, 1 body centre)
 *   fcc: 4 classes, colour = basis index
 *   CSR: greedy colouring, present sites in ascending natural index each
 *        take the smallest colour unused by an earlier-coloured neighbour.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
 *   counter = (index, sweep, tag<<24 | colour<<8 | call, replica)
 *   key     = (seed & 0xffffffff, seed >> 32)
 * tag 0 = trial move, tag 1 = initial spin.  The FP64 path draws two blocks
 * per trial keyed by the natural site index (calls 0 and 1): u_z from words
 * 0,1, u_phi from words 2,3 of call 0 and P from words 0,1 of call 1, each
 * u = ((a>>5) 2^26 + (b>>6)) 2^-53.  The FP32 and FP16 paths share one block
 * between two sites of the same colour: the site whose rank among the
 * present sites of its colour (ascending natural index) is r uses block
 * index r >> 1 and its half r & 1, words (a, b) = 2(r&1), 2(r&1)+1;
 * u_z = (a>>11) 2^-21, u_phi = (b>>11) 2^-21,
 * P = (((a & 0x7ff) << 11) | (b & 0x7ff)) 2^-22.  On a periodic sc lattice
 * r = natural index >> 1.  Initial spins always use one FP64-schedule block
 * keyed by the natural index.
 * Trial orientation: z = 2u_z - 1, phi = pi (2u_phi - 1),
 * r = sqrt((1-z)(1+z)), S' = (r cos phi, r sin phi, z).
 * There is no random-number state in memory.
 *
 * Conventions for every call:
 *   - Return HS_OK (0) or a negative hs_status; hs_last_error() gives a
 *     thread-local message for the last failure on the calling thread.
 *     Nothing aborts the process.
 *   - Host arrays passed in are copied before the call returns; the caller
 *     keeps ownership (hs_set_spins_async reads its array later, see there).
 *   - The lattice handle owns all device memory it allocates.  A handle is
 *     used by one host thread at a time.
 *   - Device work is ordered on the CUDA stream given at creation (NULL =
 *     the legacy default stream).  Calls that return data to host memory
 *     synchronise that stream before returning.
 *   - Spins cross the boundary in FP64 (hs_set_spins_async also takes FP32),
 *     natural site order, 3 values per site (x, y, z), for all n_sites
 *     natural indices; absent (masked) sites read back as 0 and are ignored
 *     on input.
 *   - A device-side error (a bounded wait that timed out) is latched on the
 *     device and reported by the next call that synchronises.
 */
#ifndef HS_H
#define HS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HS_API_VERSION 1

typedef struct hs_lattice hs_lattice;
typedef struct hs_batch hs_batch;

enum hs_lattice_type { HS_SC = 0, HS_BCC = 1, HS_FCC = 2, HS_CSR = 3 };
enum hs_precision { HS_FP64 = 0, HS_FP32 = 1, HS_FP16 = 2 };
enum hs_init_mode { HS_INIT_RANDOM = 0, HS_INIT_ALIGNED = 1 };
enum hs_status {
    HS_OK = 0,
    HS_E_INVALID = -1, /* bad argument or unsupported shape */
    HS_E_CUDA = -2,    /* a CUDA runtime call failed */
    HS_E_OOM = -3,     /* device or host allocation failed */
    HS_E_COLOUR = -4,  /* the requested structural colouring is not proper */
    HS_E_TIMEOUT = -5, /* a bounded device-side wait gave up */
    HS_E_DEVICE = -6   /* no usable CUDA device */
};

/* Hamiltonian parameters of Eq. 1.  e need not be normalised: the library
 * normalises it (a zero vector is HS_E_INVALID). */
typedef struct {
    double J;
    double K;
    double e[3];
} hs_params;

/* Instantaneous observables (FP64), Eq. 1 and Eq. 2. */
typedef struct {
    double E;           /* total energy, each bond once */
    double M[3];        /* M vector = sum S_i / N (|S| = 1) */
    double absM;        /* |M| */
    double M2;          /* |M|^2 */
    double M4;          /* |M|^4 */
    int64_t n_sites;    /* N: present spins */
    double accept_rate; /* accepted / attempted moves of the last hs_sweep call */
} hs_measurement;

/* Layout of the per-sweep accumulator read by hs_read_accumulator. */
#define HS_N_MOMENTS 9
enum hs_moment {
    HS_SUM_E = 0,     /* sum E            */
    HS_SUM_E2 = 1,    /* sum E^2          */
    HS_SUM_ABSM = 2,  /* sum |M|          */
    HS_SUM_M2 = 3,    /* sum |M|^2        */
    HS_SUM_M4 = 4,    /* sum |M|^4        */
    HS_SUM_MX = 5,    /* sum M_x          */
    HS_SUM_MY = 6,    /* sum M_y          */
    HS_SUM_MZ = 7,    /* sum M_z          */
    HS_SUM_ABSME = 8  /* sum |M . e|      */
};

typedef struct {
    int type;          /* hs_lattice_type */
    int precision;     /* hs_precision */
    int n_colours;     /* colour classes per sweep */
    int structured;    /* 1: sc stencil kernel, 0: neighbour-table kernel */
    int64_t n_sites;   /* natural indices */
    int64_t n_present; /* N */
    int64_t device_bytes; /* device memory held by the handle */
    uint64_t sweep;    /* next sweep index (Philox counter word 1) */
    int fold_sweeps;   /* hs_sweep folds the fused per-sweep sums into the accumulator
                          after every fold_sweeps sweeps (1..64) and after its last one */
} hs_info;

/*
 * Create a lattice, copy its geometry to the device and set all spins along
 * +e (call hs_init_spins for a random start).
 *   type      HS_SC / HS_BCC / HS_FCC: dims[3] = cells (Lx, Ly, Lz) and
 *             periodic (0/1); row_ptr, col_idx must be NULL and n_sites is
 *             ignored.  Natural index sc (z*Ly+y)*Lx+x, bcc/fcc
 *             ((cz*Ly+cy)*Lx+cx)*B+b.  Periodic sc needs even dims >= 2.
 *             Unmasked periodic sc with Lx/2 a multiple of the vector width
 *             runs the stencil kernel; every other case runs the
 *             neighbour-table kernel.
 *             HS_CSR: row_ptr[n_sites+1] (int64, row_ptr[0] = 0) and
 *             col_idx[row_ptr[n_sites]] (int32 in [0, n_sites), no self
 *             loops) give a symmetric neighbour list; its stored order is
 *             the order of the neighbour sum.  dims and periodic are ignored.
 *   site_mask n_sites bytes, 0 = vacancy (removed from the graph), or NULL.
 *   p         Eq. 1 parameters.
 *   precision HS_FP64 / HS_FP32 / HS_FP16 spin storage and arithmetic (FP16
 *             stores binary16 and computes in FP32); reductions are FP64.
 *   seed, replica  Philox key and counter word 3.
 *   cuda_stream    cudaStream_t to order all work on (NULL = default).
 * Errors: HS_E_INVALID (shape, neighbour list), HS_E_COLOUR (odd periodic
 * sc), HS_E_OOM, HS_E_CUDA, HS_E_DEVICE.  On error *out is NULL.
 */
int hs_lattice_create(hs_lattice **out, int type, const int32_t dims[3], int periodic,
                      const int64_t *row_ptr, const int32_t *col_idx, int64_t n_sites,
                      const uint8_t *site_mask, const hs_params *p, int precision, uint64_t seed,
                      uint32_t replica, void *cuda_stream);

/* Free the handle and its device memory (NULL is a no-op).  Synchronises
 * the stream first. */
void hs_lattice_destroy(hs_lattice *h);

/* Initial state.  HS_INIT_RANDOM: every present site gets an independent
 * uniform point on the sphere from the tag-1 Philox block of its natural
 * index (sweep 0, colour 0), computed in FP64 and rounded to the storage
 * precision.  HS_INIT_ALIGNED: every spin = +e.  Does not change the sweep
 * counter. */
int hs_init_spins(hs_lattice *h, int mode);

/* n_sweeps Metropolis sweeps (Metropolis steps (i)-(iii), every present site
 * attempted once per sweep, colour classes in order) at inverse temperature
 * beta >= 0.  Sweep k of the call uses Philox counter word 1 = the sweep
 * counter + k; the counter then advances by n_sweeps.  With accumulation on
 * (hs_accumulate), every sweep also adds its E and M moments (computed
 * inside the colour passes, FP64 totals) to the accumulator.  Asynchronous:
 * returns after queueing the work on the stream. */
int hs_sweep(hs_lattice *h, double beta, int64_t n_sweeps);

/* Recompute E (Eq. 1) and M (Eq. 2) of the current state and copy them to
 * *out; accept_rate refers to the last hs_sweep call.  Synchronous. */
int hs_measure(hs_lattice *h, hs_measurement *out);

/* Switch per-sweep accumulation of the moments on (1) or off (0). */
int hs_accumulate(hs_lattice *h, int on);

/* Zero the accumulator and its sweep count. */
int hs_reset_accumulator(hs_lattice *h);

/* Copy the HS_N_MOMENTS sums (hs_moment order) and the number of
 * accumulated sweeps.  Synchronous. */
int hs_read_accumulator(hs_lattice *h, double moments[HS_N_MOMENTS], int64_t *count);

/* Spins to / from host memory: xyz is 3 * n_sites doubles in natural order.
 * hs_set_spins normalises nothing: callers pass unit vectors.  Both are
 * synchronous (the host buffer may be reused on return). */
int hs_get_spins(hs_lattice *h, double *xyz);
int hs_set_spins(hs_lattice *h, const double *xyz);

/* Same with a device pointer (3 * n_sites doubles, device memory); ordered
 * on the handle's stream, asynchronous. */
int hs_get_spins_device(hs_lattice *h, double *d_xyz);
int hs_set_spins_device(hs_lattice *h, const double *d_xyz);

/* Asynchronous upload of a whole state from host memory, for callers that
 * feed a new state every few sweeps and want the copy to run while earlier
 * sweeps do (the state is what Eq. 1 and the Metropolis steps act on; the
 * paper loads one initial state, so the pipelining is this library's own).
 *   xyz    host, 3 * n_sites values in natural order (unit vectors; nothing is
 *          normalised), FP64 when dtype = HS_FP64, FP32 when dtype = HS_FP32
 *          (widened exactly, so an FP32 lattice stores the given values).
 *          Page-locked memory lets the copy overlap the device's work;
 *          pageable memory works but the copy may then block the caller.
 * The copy runs on a stream of the handle's own into one of two device
 * buffers (used alternately); the conversion into the lattice's layout is
 * ordered on the handle's stream after the work already queued there, so
 * the sweeps queued before this call see the old state and those queued
 * after it the new one.  The call returns without waiting.  Keep xyz
 * unchanged until a later synchronous call on the handle (hs_read_accumulator,
 * hs_measure, hs_get_spins, ...) has returned or the handle's stream has been
 * synchronised.  The first call allocates the two buffers (2 * 3 * n_sites
 * doubles); later calls allocate nothing.  Errors: HS_E_INVALID for a null
 * argument or another dtype, a CUDA error code for a failed allocation or
 * launch. */
int hs_set_spins_async(hs_lattice *h, const void *xyz, int dtype);

/* Set the next sweep index (checkpoint / resume: spins + sweep counter +
 * seed + replica fix the rest of the chain bit for bit). */
int hs_set_sweep_counter(hs_lattice *h, uint64_t sweep);

int hs_get_info(const hs_lattice *h, hs_info *out);

/* Per-kernel timing of the colour passes: when enabled, hs_sweep brackets
 * each colour-pass launch with CUDA events on the handle's stream.
 * hs_read_timing synchronises, returns the summed kernel time in ms and the
 * number of timed launches since the last enable, and keeps counting. */
int hs_enable_timing(hs_lattice *h, int on);
int hs_read_timing(hs_lattice *h, double *ms, int64_t *launches);

/* Launch configuration of the colour-pass kernels (the autotuner's knobs).
 * Results never depend on it: a site's random numbers and arithmetic are
 * fixed by its natural index, so every configuration gives bit-identical
 * spins.  Zero fields mean "choose automatically". */
enum hs_kernel {
    HS_KERNEL_AUTO = 0,
    HS_KERNEL_STENCIL = 1, /* sc: operands loaded through L1/L2 into registers */
    HS_KERNEL_TABLE = 3,   /* neighbour-table kernel (bcc, fcc, CSR, masked) */
    HS_KERNEL_MARCH = 4,   /* sc: register stencil walking each CTA's slab of
                              tile_y rows along z (rows reused from L1, next
                              plane prefetched into L2); spreads a small
                              lattice's pass over more SMs */
    HS_KERNEL_PIPE = 5     /* sc: register stencil whose next work item is copied
                              global -> shared (cp.async, one slot per thread)
                              while the current one is computed; needs 4..16
                              bytes of storage per vector */
};
typedef struct {
    int kernel;        /* hs_kernel; the table kernel is the only one for non-sc */
    int vec_width;     /* sc kernels: sites per thread, 1/2/4/8, dividing Lx/2,
                          at most 16 bytes of storage per load */
    int blocks_per_sm; /* resident CTAs per SM (0 = max) */
    int tile_y;        /* z-march: rows per CTA slab (divides Ly; 0 = automatic) */
    int prefetch;      /* stencil: 1 = issue the next work item's loads before
                          computing the current one, 3 = split prefetch (the
                          next item's own, same-row and z+-1 rows loaded once
                          the current item's fields are summed), 2 = off,
                          0 = automatic (off);
                          table: 1 = ask L2 for the next site's table row
                          and spin ahead, 2 = off, 0 = automatic (on for FP32
                          tables of fewer than 8 neighbours) */
    int order;         /* stencil: order of the work items over a sweep:
                          1 = every pass in ascending (z, y, x) order,
                          2 = alternating (the passes of colour 1 descending,
                          so each pass begins on the planes that the pass
                          before it touched last, which are still in L2),
                          0 = automatic (alternating; ascending with the
                          split prefetch) */
} hs_launch;

/* Set (fields 0 = automatic) or read the launch configuration.  Kernel
 * codes 2 and 6 are not used (HS_E_INVALID). */
int hs_set_launch(hs_lattice *h, const hs_launch *cfg);
int hs_get_launch(const hs_lattice *h, hs_launch *out);

/* On-site anisotropy tensor: adds -sum_i S_i^T A S_i to Eq. 1 (to dH in
 * Metropolis step (iii), to E in hs_measure and in the fused per-sweep
 * reductions), with A symmetric, given as its six entries
 * A = (Axx, Ayy, Azz, Axy, Axz, Ayz); S^T A S = Axx x^2 + Ayy y^2 + Azz z^2
 * + 2 (Axy xy + Axz xz + Ayz yz).  A = NULL or all zeros removes the term.
 * The uniaxial term is the special case A = K e e^T.  Kernels: the register
 * stencil without prefetch (periodic sc) and the neighbour table (everything
 * else); the pipelined and z-march kernels and hs_batch_create reject a
 * lattice that has the term.  Setting the tensor resets the launch
 * configuration to automatic.  Entries must be finite (HS_E_INVALID
 * otherwise; nothing changes then).  The FP32 / FP16 kernels use the entries
 * rounded to FP32.  hs_get_anisotropy_tensor reads them back (zeros when
 * the term is off). */
int hs_set_anisotropy_tensor(hs_lattice *h, const double A[6]);
int hs_get_anisotropy_tensor(const hs_lattice *h, double A[6]);

/* Autotuner: time every valid launch configuration (kernel, vector width,
 * CTAs per SM, z-march slab rows, prefetch) for
 * n_trial_sweeps sweeps at beta, each from the same saved state and sweep
 * counter (one warm-up sweep first); the three fastest are timed again over
 * twice the sweeps and the fastest of those is kept.  The spins, the
 * accumulator and the sweep counter are restored afterwards, so the chain is
 * exactly as if the call had not happened.  Choices are cached per
 * (precision, shape, SM count) for the life of the process.  Synchronous. */
int hs_autotune(hs_lattice *h, double beta, int n_trial_sweeps);

/* Host-only helper (no device needed): the greedy colouring the library
 * uses for HS_CSR lattices.  colour_out[n] gets the class of each present
 * site (-1 for masked sites); *n_colours the number of classes. */
int hs_colour_greedy(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                     const uint8_t *site_mask, int32_t *colour_out, int *n_colours);

/* Batched replicas: many independent lattices advanced together by one
 * persistent kernel (cooperative launch, captured once in a CUDA graph per
 * (n_sweeps, n_equil) pair), each member at its own beta, with its own seed,
 * replica, sweep counter and accumulator.  Members must be unmasked periodic
 * sc lattices of one precision (FP64, FP32 or FP16; any sizes, mixed) with
 * Lx divisible by 8 (FP32, FP16) or 4 (FP64), created on one stream and
 * device; they stay owned by the caller and must outlive the batch.  hs_batch_run performs n_equil sweeps, then n_sweeps sweeps whose
 * moments are added to each member's accumulator (as hs_sweep with
 * accumulation on would), with the same random numbers and arithmetic as
 * hs_sweep on each member alone.  Colour passes are separated by a grid-wide
 * barrier whose waits are bounded: a timeout is latched in every member and
 * reported (HS_E_TIMEOUT) by the next synchronising call on a member.
 * Asynchronous. */
int hs_batch_create(hs_batch **out, hs_lattice *const *members, int n_members);
int hs_batch_run(hs_batch *b, const double *betas, int64_t n_sweeps, int64_t n_equil);
void hs_batch_destroy(hs_batch *b);

/* Batch autotuner: the batch's work split -- its members' work items (4
 * sites of one row of one colour), concatenated and cut into one contiguous
 * range per CTA, or interleaved -- is timed for every CTA count per SM (1 up
 * to the kernel's occupancy), the three splits (align_rows 0: contiguous
 * ranges cut at any item; 1: cut at the nearest row boundary; 2: contiguous
 * ranges of whole 256-item blocks cut at equal estimated cost (an item of a
 * member with r work items per row weighs 1 + 3 / r), then the blocks of the
 * CTAs that hold nothing but one member dealt out to them round-robin, so
 * they sweep that member side by side in grid-stride order), both load
 * schedules of the kernel (one work item of loads at a
 * time, or split prefetch: the next item's own, same-row and z+-1 rows load
 * during the current item's arithmetic) and both colour schedules (schedule
 * 0: every sweep in one persistent cooperative launch, passes separated by
 * the bounded grid barrier, captured in a CUDA graph; schedule 1: one launch
 * per colour pass of every member, consecutive launches chained by
 * programmatic dependent launch), and, when every member's six planes fit
 * in one CTA's shared memory (on GB300 cubes up to L = 24 in FP32, 20 in
 * FP64, 32 in FP16), schedule 2:
 * one launch with one CTA per member, whose planes are copied into shared
 * memory once and stay there for every sweep, the colour passes separated
 * by CTA barriers only (no grid barrier, no global traffic between the
 * first load and the final store; the work split and load schedule do not
 * apply), for n_trial_sweeps sweeps at the given
 * betas after one warm-up sweep; the fastest is kept.  Colour 0 then colour
 * 1 in every sweep under all of them.  Every member's spins, sweep counter
 * and accumulator are restored, so the members' chains are as if the call
 * had not happened (spins are identical under every choice; the FP64 sums
 * are taken in each split's own fixed order).  Synchronous.
 * hs_batch_get_layout reads the choice in use (hs_batch_create starts with
 * the maximum CTAs per SM, the interleaved split (align_rows 2), no
 * prefetch, and schedule 2 when there are at least 16 members and every one
 * fits in a CTA's shared memory, else schedule 0). */
int hs_batch_autotune(hs_batch *b, const double *betas, int n_trial_sweeps);
int hs_batch_get_layout(const hs_batch *b, int *ctas_per_sm, int *align_rows, int *prefetch, int *schedule);
/* Set the choice by hand: ctas_per_sm in 1 .. the kernel's occupancy,
 * align_rows 0, 1 or 2, prefetch 0 or 1, schedule 0, 1 or 2, the last only
 * when every member fits in one CTA's shared memory (HS_E_INVALID otherwise).
 * The members' chains do not depend on it.  The timeout test hook always
 * runs the persistent schedule.  Synchronises the batch's stream. */
int hs_batch_set_layout(hs_batch *b, int ctas_per_sm, int align_rows, int prefetch, int schedule);

/* Allocation-free sweep (the paper has no counterpart; it is a service to
 * callers that cannot allocate device memory themselves: a host framework
 * whose caching allocator or fixed budget owns all device memory, or a
 * latency-critical loop that cannot afford cudaMalloc's implicit device-wide
 * synchronisation).
 * Runs n_sweeps sweeps (sweep indices first_sweep, first_sweep+1, ...) of the
 * FP32 sc stencil kernel, with the same random numbers and arithmetic as a
 * handle created with HS_SC, periodic, HS_FP32, seed and replica, on spins
 * the caller holds in device memory:
 *   planes  device, 6 planes of Lz*Ly*(Lx/2) floats in the order colour 0
 *           x, y, z, colour 1 x, y, z; site (x,y,z) of colour (x+y+z)&1 at
 *           index (z*Ly + y)*(Lx/2) + x/2 of its colour's planes.  Updated
 *           in place.  dims all even and >= 2, fewer than 2^31 sites.
 *   d_out   device, HS_N_MOMENTS + 2 doubles, overwritten with the moment
 *           sums of this call's sweeps (hs_moment order), the number of
 *           sweeps and the number of accepted moves.
 * It calls no cudaMalloc, cudaFree or allocating library routine.  Its
 * reduction scratch (per-CTA slots for at most HS_NOALLOC_MAX_CTAS CTAs, the
 * accumulator and an arrival counter, about 80 KB) is one static device
 * array that every GPU loading the library holds until the process exits.
 * Each call zeroes what must start at zero; every call shares the array, so
 * calls whose work overlaps on the GPU (on different streams, or from
 * several threads) race and must be serialised by the caller.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress,
 * once per device, with that device current); make that first call before
 * any stream capture.  A device that would need more CTAs than the scratch
 * holds is rejected with HS_E_INVALID.  planes must start on a 4 * vec byte
 * boundary, vec being the vector width the kernel takes for this Lx (4 when
 * Lx/2 is a multiple of 4, else 2 when it is even, else 1), and d_out on an
 * 8-byte boundary; a misaligned pointer (a view with a storage offset, say)
 * is rejected with HS_E_INVALID before anything is launched.  The device
 * address is cached for the life of the process: after cudaDeviceReset do
 * not call this entry point again.  Asynchronous on cuda_stream; errors are
 * reported through hs_last_error. */
#define HS_NOALLOC_MAX_CTAS 1024
int hs_sweep_sc_fp32_noalloc(float *planes, const int32_t dims[3], const hs_params *p, double beta,
                             uint64_t seed, uint32_t replica, uint64_t first_sweep, int64_t n_sweeps,
                             double *d_out, void *cuda_stream);

/* One colour pass of the current sweep (Metropolis steps (i)-(iii) over
 * colour class `colour`); the pass of the last colour finalises the sweep's
 * fused reductions and advances the sweep counter.  hs_sweep(h, beta, 1) is
 * the passes 0 .. C-1 in order.  A z-slab (below) sweeps this way, its halo
 * planes refreshed between the passes. */
int hs_sweep_pass(hs_lattice *h, double beta, int colour);

/* Domain decomposition of a periodic sc lattice along z: a slab handle owns
 * the global planes z0 .. z0+nz-1 of an Lx x Ly x Lz lattice (dims as for
 * hs_lattice_create, all even) and stores one halo plane of each colour
 * below and above them.  Every own site keeps its global natural index,
 * colour, neighbour order and random numbers, so a set of slabs that
 * exchanges halos between colour passes reproduces the whole lattice's
 * chain bit for bit.  A slab runs the register stencil; hs_sweep,
 * hs_measure and hs_batch_create reject it, and hs_autotune leaves it
 * unchanged.  hs_get_spins / hs_set_spins / hs_init_spins work on its own
 * planes (Lx Ly nz spins in natural order).  Halos read as zero until
 * first written. */
int hs_slab_create(hs_lattice **out, const int32_t dims[3], int32_t z0, int32_t nz, const hs_params *p,
                   int precision, uint64_t seed, uint32_t replica, void *cuda_stream);
/* Device address and size of one component plane of a slab:
 * which = 0 halo below, 1 first own plane, 2 last own plane, 3 halo above.
 * Planes are [Ly][Lx/2] of the storage type in the colour-major layout; a
 * multi-device run sends these (own 1 / 2 to the neighbours' halos 3 / 0). */
int hs_slab_plane(const hs_lattice *h, int colour, int component, int which, void **dev_ptr, size_t *bytes);
/* Copy the three component planes of colour `colour` from plane src_which of
 * src to plane dst_which of dst (same lattice and device), on dst's
 * communication stream (hs_slab_set_comm_stream; by default its stream):
 * the halo exchange of slabs that share a device. */
int hs_slab_copy_plane(hs_lattice *dst, int dst_which, const hs_lattice *src, int src_which, int colour);
/* One message per halo transfer between processes: hs_slab_pack copies the
 * three component planes (x, y, z) of colour `colour` at plane `which` (as
 * for hs_slab_plane) back to back into the caller's device buffer d_buf
 * (3 x the plane bytes hs_slab_plane reports); hs_slab_unpack copies such a
 * buffer into plane `which` of this slab.  One strided device-to-device copy
 * each, ordered on the handle's communication stream (hs_slab_set_comm_stream;
 * by default its stream), so a stream-ordered send (NCCL) of d_buf needs no
 * host synchronisation. */
int hs_slab_pack(const hs_lattice *h, int colour, int which, void *d_buf);
int hs_slab_unpack(hs_lattice *h, int colour, int which, const void *d_buf);

/* Boundary-first colour pass of a slab.  A colour pass updates only sites of
 * its colour and reads only the other colour, so its order over the planes
 * does not change the result: the pass may run as part HS_PART_BOUNDARY
 * (the first and last own planes) followed by HS_PART_INTERIOR (the planes
 * between them), both on the slab's stream.  Once the boundary part is done
 * the colour's boundary planes are final, so their messages can travel
 * (hs_slab_pack on the communication stream, a send, hs_slab_unpack of the
 * received halos of the same colour) while the interior part runs: the
 * interior part reads and writes neither those planes nor the halos of its
 * own colour.  The next colour's pass must follow both the interior part
 * (stream order) and the unpacked halos (the caller's event).
 * HS_PART_WHOLE is the whole pass in one launch (= hs_sweep_pass).  Each
 * part keeps its own partial sums; the launch that completes the last
 * colour's pass finalises the sweep from the parts run in it, so the fused
 * sums and the spins equal those of whole passes bit for bit.
 * HS_E_INVALID: a part other than HS_PART_WHOLE on a non-slab lattice, an
 * interior part not directly after the boundary part of the same colour,
 * or a boundary or whole part while an interior part is due.  A slab of one
 * or two planes has no interior: its boundary part covers it and its
 * interior part launches nothing. */
#define HS_PART_WHOLE 0
#define HS_PART_BOUNDARY 1
#define HS_PART_INTERIOR 2
int hs_sweep_pass_part(hs_lattice *h, double beta, int colour, int part);
/* CTAs that the interior part leaves unlaunched (0 <= ctas < the pass's CTA
 * count; default 0), so that the communication's copy and send kernels find
 * free SMs beside it instead of waiting for its persistent CTAs to retire. */
int hs_slab_reserve_ctas(hs_lattice *h, int32_t ctas);
/* Stream on which hs_slab_pack, hs_slab_unpack and hs_slab_copy_plane (into
 * this slab) run: by default the slab's own stream; NULL selects the legacy
 * default stream, as elsewhere in this API.  With a separate stream the
 * caller orders those copies against the passes with events, keeps the
 * stream alive while the slab uses it, and synchronises it before
 * hs_lattice_destroy (which waits only for the slab's own stream). */
int hs_slab_set_comm_stream(hs_lattice *h, void *cuda_stream);

/* Stream-ordered forms of the sums exchange of a multi-process lattice:
 * hs_read_sums_device copies the last finalised sweep's five sums (as
 * hs_read_sums) to device memory d_out; after the caller's allreduce over
 * the processes, hs_accumulate_sums takes the five totals d_tot (device
 * memory) of one sweep of the whole lattice of n_sites present spins and adds
 * that sweep's E and M moments (Eq. 1, Eq. 2) to this handle's accumulator,
 * as a single lattice does with its own sums; hs_read_accumulator reads them.
 * Keep the slab's own accumulation off (hs_accumulate(h, 0)), or its
 * per-slab observables are added too.  Asynchronous. */
int hs_read_sums_device(hs_lattice *h, double *d_out);
int hs_accumulate_sums(hs_lattice *h, const double *d_tot, int64_t n_sites);

/* Spins of n selected sites in FP64: out[3t .. 3t+2] = S of the site with
 * global natural index sites[t] (host arrays, the caller's).  Periodic sc
 * lattices and slabs (own sites only); HS_E_INVALID for any other site.
 * Synchronises the handle's stream.  For lattices too large to copy whole. */
int hs_get_sites(hs_lattice *h, int64_t n, const int64_t *sites, double *out);

/* FP64 sums of the last finalised fused reduction (the last hs_sweep or
 * hs_sweep_pass sweep, or hs_measure): out = {E share, sum S_x, sum S_y,
 * sum S_z, accepted moves of that sweep}.  Summed over the slabs of a
 * lattice they give its E (every bond is counted at its colour-1 end, which
 * one slab owns) and M = sum S / N. */
int hs_read_sums(hs_lattice *h, double out[5]);

/* Measured arithmetic peak of the current device, for the roofline of a
 * path bound by arithmetic rather than memory (the FP64 sweep: the paper
 * runs in double precision, and GB300's FP64 rate, not its HBM, bounds it).
 * kind 0: FP64 fused multiply-add (DFMA); 1: FP32 FFMA; 2: packed FP32
 * (two lanes per instruction, the form the FP32 / FP16 sweep kernels use).
 * Runs independent FMA chains on every SM (8 CTAs of 256 threads per SM,
 * 8 chains per thread), a warm-up launch, then one launch timed with CUDA
 * events on cuda_stream; *flops_per_s = 2 x FMAs / time.  Allocates and
 * frees a small device buffer; synchronous.  HS_E_INVALID for another kind. */
int hs_measure_alu_peak(int kind, void *cuda_stream, double *flops_per_s);

/* Test hook for the bounded device-side waits (failure detection without a
 * GPU fault): in the next hs_batch_run (persistent schedule) one CTA skips
 * its first grid-barrier arrival, so every other CTA's bounded wait runs out
 * (about one second).  The kernel latches its error word and returns; the
 * next synchronising call on each member reports HS_E_TIMEOUT and clears it,
 * the CUDA context stays usable, and the spins of the interrupted sweep are
 * left part-updated. */
int hs_batch_inject_timeout(hs_batch *b, int on);

const char *hs_last_error(void);
int hs_api_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HS_H */
