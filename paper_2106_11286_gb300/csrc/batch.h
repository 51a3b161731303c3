// Declarations of the batched kernels (batch.cu), shared with the host code
// that builds a batch (api.cpp); not part of the ABI.
#pragma once

#include "hs_impl.h"

namespace hs {

// ---- batched persistent kernel (batch.cu)
// One member lattice (periodic sc, stencil layout; every member of a batch in
// one precision, vector width batch_vec(precision)).
struct BatchMember {
    void *planes;           // six planes of the storage type
    int Lx, Ly, Lz, Lh;
    FastDiv div_nxv, div_ly;
    float fJ, fK, fe[3], fbeta;
    double J, K, beta;      // the same in FP64 (FP64 members)
    double e[3];
    const double2 *sc_tab;  // FP64 members: sin, cos(pi j / 1024) of the trial
    int zaxis;              // 1: e = (0, 0, 1) exactly
    uint32_t key0, key1, replica;
    uint32_t sweep0;        // the member's sweep index at batch sweep 0
    double n_present;
    DevAccum *acc;
    int seg_begin, seg_end;  // the member's segments (contiguous)
};

// Items begin, begin + stride, ... (< end) of one member's colour pass,
// each the first of kBlock consecutive items that one CTA's threads take
// together: stride kBlock for a contiguous range; a multiple of kBlock when
// several CTAs sweep one member side by side.
struct BatchSeg {
    int member;
    uint32_t begin, end, stride;
};

struct BatchArgs {
    const BatchMember *members;
    int n_members;
    const BatchSeg *segs;
    const int *cta_seg;      // CTA c owns segments [cta_seg[c], cta_seg[c+1])
    int n_segs;
    double *slots;           // [sweep parity][colour][segment][kPartials]
    unsigned int *bar;       // grid barrier: one 64-bit arrival count (two words, 8-byte aligned)
    int *error;              // latched device error (barrier timeout)
    int n_total, n_equil;    // sweeps, of which the first n_equil unmeasured
    int inject_skip;         // test hook: 1 = CTA 0 skips its first barrier arrival
    int zaxis_all;           // 1: every member's easy axis is (0, 0, 1): FP32 / FP16 run the S.e = S_z kernels
    int kzero_all;           // 1: besides, every member's K is +0: they run the kernels without the K term
};

// sites per work item of a batch member: 16-byte loads for FP64 and FP32,
// 8-byte loads for FP16
inline int batch_vec(int precision) { return precision == HS_FP64 ? 2 : 4; }
// prefetch 0: one work item of loads at a time; 1: split prefetch (the
// next item's DRAM-heavy rows load during the current item's arithmetic)
cudaError_t launch_batch(int precision, const BatchArgs &b, int grid, cudaStream_t s, int prefetch);
// the per-pass schedule: 2 n_total chained pass launches and a finalise launch
cudaError_t launch_batch_passes(int precision, const BatchArgs &b, int grid, cudaStream_t s, int prefetch);
int batch_occupancy(int precision, int prefetch);
// the resident schedule: one CTA per member, its planes in dynamic shared
// memory (smem bytes, at most batch_resident_limit(precision)) for the whole run
cudaError_t launch_batch_resident(int precision, const BatchArgs &b, size_t smem, cudaStream_t s);
size_t batch_resident_limit(int precision);
// zero every member's accepted-move counter (reads b.members on the device)
cudaError_t launch_batch_reset(const BatchArgs &b, cudaStream_t s);

}  // namespace hs
