// Device building blocks shared by the colour-pass kernels (kernels.cu) and
// the batched persistent kernel (batch.cu): Philox4x32-10, the trial
// orientation, the Metropolis test of Eq. 1, the fused reductions and the
// stencil work item.  Internal to the library.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>
#include <string.h>

#include "hs_impl.h"

namespace hs {
namespace {


// ----------------------------------------------------------------- Philox
// Philox4x32-10 as published (Salmon et al., SC'11): ten rounds of two
// 32x32->64 multiplies with fixed odd multipliers, a cross-lane swap of the
// high halves xored with the round key, and a Weyl key schedule.
constexpr uint32_t kMulA = 0xD2511F53u;
constexpr uint32_t kMulB = 0xCD9E8D57u;
constexpr uint32_t kWeylA = 0x9E3779B9u;
constexpr uint32_t kWeylB = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t pa = (uint64_t)kMulA * c.x;  // one 32x32->64 multiply per lane pair
        const uint64_t pb = (uint64_t)kMulB * c.z;
        c = make_uint4((uint32_t)(pb >> 32) ^ c.y ^ k0, (uint32_t)pb, (uint32_t)(pa >> 32) ^ c.w ^ k1, (uint32_t)pa);
        k0 += kWeylA;
        k1 += kWeylB;
    }
    return c;
}

// Programmatic dependent launch: a pass kernel lets the next kernel in the
// stream be scheduled as its own CTAs retire, then waits until the previous
// kernel has completed and its writes are visible before touching memory.
// Without a programmatic dependency both instructions are no-ops.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

constexpr uint32_t kTagTrial = 0u;
constexpr uint32_t kTagInit = 1u;

// ----------------------------------------------------------------- precision
template <int P> struct Tr;
template <> struct Tr<HS_FP64> { using S = double; using C = double; };
template <> struct Tr<HS_FP32> { using S = float; using C = float; };
template <> struct Tr<HS_FP16> { using S = __half; using C = float; };

__device__ __forceinline__ double to_c(double v) { return v; }
__device__ __forceinline__ float to_c(float v) { return v; }
__device__ __forceinline__ float to_c(__half v) { return __half2float(v); }

template <typename S> __device__ __forceinline__ S store_from_double(double v);
template <> __device__ __forceinline__ double store_from_double<double>(double v) { return v; }
template <> __device__ __forceinline__ float store_from_double<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ __half store_from_double<__half>(double v) { return __double2half(v); }

template <typename T, int V>
struct alignas(sizeof(T) * V) Vec {
    T v[V];
};

// Uniform point on the sphere in FP64 from one Philox block (words 0,1 -> u_z,
// words 2,3 -> u_phi, 53 bits each): z = 2u_z - 1 and v = 2u_phi - 1 are
// formed exactly from the integers, r = sqrt((1-z)(1+z)) is correctly
// rounded, phi = pi v.
__device__ __forceinline__ void sphere_fp64(uint4 w, double &x, double &y, double &z) {
    const int64_t two52 = int64_t(1) << 52;
    const int64_t iz = (int64_t)((((uint64_t)(w.x >> 5)) << 26) | (uint64_t)(w.y >> 6));
    const int64_t iv = (int64_t)((((uint64_t)(w.z >> 5)) << 26) | (uint64_t)(w.w >> 6));
    z = (double)(iz - two52) * 0x1p-52;
    const double v = (double)(iv - two52) * 0x1p-52;
    const double r = sqrt((1.0 - z) * (1.0 + z));
    double sn, cs;
    sincospi(v, &sn, &cs);
    x = r * cs;
    y = r * sn;
}

// sin(pi t), cos(pi t) for t = m 2^-52 in [0, 2) (m < 2^53), by table lookup
// and angle addition (Tang, "Table-lookup algorithms for elementary functions
// and their error analysis", 1991): j = m 2^-42 rounded to the nearest
// integer (0 .. 2048; j = 2048 is j = 0, the period being 2) and b = m - j 2^42
// in [-2^41, 2^41), so t = j/1024 + b 2^-52 exactly.  sin, cos(pi j/1024) come
// from a 2048-entry table (correctly rounded on the host); x = pi b 2^-52
// (|x| <= pi 2^-11 < 0.00154) takes sin x = x - x^3/6 (first omitted term
// below 7.2e-17) and cos x = 1 - c, c = x^2/2 - x^4/24 (first omitted below
// 1.8e-20); then sin(a + x) = sin a + (cos a sin x - sin a c) and
// cos(a + x) = cos a - (sin a sin x + cos a c).  Error below two units in the
// last place, for 10 FP64 operations.
constexpr double kPiTwoM52 = 3.141592653589793 * 0x1p-52;  // pi (FP64) 2^-52, exact scaling

__device__ __forceinline__ void sincospi_tab(uint64_t m, const double2 *tab, double &sn, double &cs) {
    const uint64_t j = (m + (1ull << 41)) >> 42;
    const int64_t b = (int64_t)m - (int64_t)(j << 42);
    const double x = (double)b * kPiTwoM52;
    const double x2 = x * x;
    const double sx = fma(x * x2, -1.0 / 6.0, x);
    const double c = x2 * fma(x2, -1.0 / 24.0, 0.5);
    const double2 t = __ldg(tab + (j & 2047u));
    sn = fma(t.y, sx, fma(-t.x, c, t.x));
    cs = fma(-t.x, sx, fma(-t.y, c, t.y));
}

// k 2^-s exactly, for an integer |k| < 2^53 and 0 < s <= 53: k converted
// (exact), then s taken off its exponent field, which stays positive for
// |k| >= 1; k = 0 gives +0.  Integer instructions in place of an FP64 multiply.
__device__ __forceinline__ double scaled_int(int64_t k, int s) {
    const double d = (double)k;
    const double r = __hiloint2double(__double2hiint(d) - (s << 20), __double2loint(d));
    return k == 0 ? 0.0 : r;
}

// Trial orientation and acceptance uniform of one site, FP64 schedule
// (Metropolis step (ii)); the sphere point of sphere_fp64 up to rounding:
// 1 - z^2 is formed with one rounding (fma), and phi = pi v = pi t - pi
// (t = v + 1) from the table: sin(pi v) = -sin(pi t), cos(pi v) = -cos(pi t).
// uf is the acceptance uniform's top 24 bits: uf <= u < uf + 2^-24.
__device__ __forceinline__ void draw_trial64(uint32_t site, uint32_t sweep, uint32_t colour, uint32_t replica,
                                             uint32_t k0, uint32_t k1, const double2 *tab, double &tx, double &ty,
                                             double &tz, double &u, float &uf) {
    const uint32_t w2 = (kTagTrial << 24) | (colour << 8);
    const uint4 a = philox10(make_uint4(site, sweep, w2, replica), k0, k1);
    const uint4 b = philox10(make_uint4(site, sweep, w2 | 1u, replica), k0, k1);
    const int64_t two52 = int64_t(1) << 52;
    const int64_t iz = (int64_t)((((uint64_t)(a.x >> 5)) << 26) | (uint64_t)(a.y >> 6));
    const uint64_t iv = (((uint64_t)(a.z >> 5)) << 26) | (uint64_t)(a.w >> 6);
    tz = scaled_int(iz - two52, 52);
    const double r = sqrt(fma(-tz, tz, 1.0));
    double sn, cs;
    sincospi_tab(iv, tab, sn, cs);
    tx = -(r * cs);
    ty = -(r * sn);
    const uint64_t ip = (((uint64_t)(b.x >> 5)) << 26) | (uint64_t)(b.y >> 6);
    u = scaled_int((int64_t)ip, 53);
    uf = (float)(uint32_t)(ip >> 29) * 0x1p-24f;
}

// ---- FP32 arithmetic of one site (float) or of the two sites of a Philox
// pair (float2, packed sm_100+ instructions).  Every operation is rounded
// explicitly and identically in both forms, so a site's result never depends
// on whether it was processed alone or as a lane of a pair.
__device__ __forceinline__ float f_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float f_sub(float a, float b) { return __fadd_rn(a, -b); }
__device__ __forceinline__ float f_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float f_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 f_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f_sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 f_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <typename T> __device__ __forceinline__ T splat(float v);
template <> __device__ __forceinline__ float splat<float>(float v) { return v; }
template <> __device__ __forceinline__ float2 splat<float2>(float v) { return make_float2(v, v); }

// 2^x from the hardware base-2 exponential (relative error about 2^-22).
__device__ __forceinline__ float ex2_hw(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_l(float x) { return ex2_hw(x); }
__device__ __forceinline__ float2 ex2_l(float2 x) { return make_float2(ex2_hw(x.x), ex2_hw(x.y)); }
__device__ __forceinline__ float rsqrt_l(float x) { return rsqrtf(x); }
__device__ __forceinline__ float2 rsqrt_l(float2 x) { return make_float2(rsqrtf(x.x), rsqrtf(x.y)); }
__device__ __forceinline__ float pos_or_zero(float w, float r) { return w > 0.0f ? r : 0.0f; }
__device__ __forceinline__ float2 pos_or_zero(float2 w, float2 r) {
    return make_float2(w.x > 0.0f ? r.x : 0.0f, w.y > 0.0f ? r.y : 0.0f);
}
__device__ __forceinline__ void sincos_l(float a, float &s, float &c) { __sincosf(a, &s, &c); }
__device__ __forceinline__ void sincos_l(float2 a, float2 &s, float2 &c) {
    __sincosf(a.x, &s.x, &c.x);
    __sincosf(a.y, &s.y, &c.y);
}
__device__ __forceinline__ float half_round(float x) { return __half2float(__float2half_rn(x)); }
__device__ __forceinline__ float half_round_l(float x) { return half_round(x); }
// both lanes rounded to binary16 by one packed conversion (each lane rounded
// to nearest even, as the scalar form), then widened exactly
__device__ __forceinline__ float2 half_round_l(float2 x) { return __half22float2(__float22half2_rn(x)); }

// c + a for a binary16 a, with one rounding: the mixed-precision add widens a
// exactly, so the result equals f_add(c, (float)a) bit for bit.
__device__ __forceinline__ float add_half(float c, __half a) {
    float d;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(__half_as_ushort(a)), "f"(c));
    return d;
}

// FP32 schedule: one Philox block serves two sites of the same colour.  The
// site of rank r within its colour class (ascending natural index) uses
// block r >> 1 and the half r & 1: words (a, b) = (x, y) or (z, w).
// u_z and u_phi are the top 21 bits of a and b, P the two low 11-bit fields
// (22 bits).
__device__ __forceinline__ uint4 trial_block(uint32_t rank_pair, uint32_t sweep, uint32_t colour, uint32_t replica,
                                             uint32_t k0, uint32_t k1) {
    return philox10(make_uint4(rank_pair, sweep, (kTagTrial << 24) | (colour << 8), replica), k0, k1);
}

// The three integers of one half (a, b): z index, azimuth index, P index.
__device__ __forceinline__ void half_ints(uint32_t a, uint32_t b, float &zi, float &vi, float &ui) {
    zi = (float)((int)(a >> 11) - (1 << 20));
    vi = (float)((int)(b >> 11) - (1 << 20));
    ui = (float)(((a & 0x7FFu) << 11) | (b & 0x7FFu));
}

// Trial orientation and acceptance uniform (Metropolis step (ii)) from the
// integers: z and v = 2u - 1 are exact, r = w / sqrt(w) with w = (1-z)(1+z)
// >= 0 from the hardware reciprocal square root, the azimuth pi v from the
// hardware sine / cosine on [-pi, pi) (absolute error about 4e-7, below what
// a 21-bit proposal resolves).  FP16 storage renormalises and rounds the trial
// to binary16; the rounded vector is the one tested and stored, so the chain
// samples the stored state.
template <int P, typename T>
__device__ __forceinline__ void trial32(T zi, T vi, T ui, T &tx, T &ty, T &tz, T &u) {
    tz = f_mul(zi, splat<T>(0x1p-20f));
    const T v = f_mul(vi, splat<T>(0x1p-20f));
    u = f_mul(ui, splat<T>(0x1p-22f));
    const T w2 = f_mul(f_sub(splat<T>(1.0f), tz), f_add(splat<T>(1.0f), tz));
    const T r = pos_or_zero(w2, f_mul(w2, rsqrt_l(w2)));
    T sn, cs;
    sincos_l(f_mul(splat<T>(3.14159265358979f), v), sn, cs);
    tx = f_mul(r, cs);
    ty = f_mul(r, sn);
    if constexpr (P == HS_FP16) {
        const T inv = rsqrt_l(f_fma(tz, tz, f_fma(ty, ty, f_mul(tx, tx))));
        tx = half_round_l(f_mul(tx, inv));
        ty = half_round_l(f_mul(ty, inv));
        tz = half_round_l(f_mul(tz, inv));
    }
}

// One site's trial, FP32 / FP16 schedule, from its rank in the colour class.
template <int P>
__device__ __forceinline__ void draw_trial_rank(uint32_t rank, uint32_t sweep, uint32_t colour, uint32_t replica,
                                                uint32_t k0, uint32_t k1, float &tx, float &ty, float &tz, float &u) {
    const uint4 w = trial_block(rank >> 1, sweep, colour, replica, k0, k1);
    float zi, vi, ui;
    if (rank & 1u)
        half_ints(w.z, w.w, zi, vi, ui);
    else
        half_ints(w.x, w.y, zi, vi, ui);
    trial32<P, float>(zi, vi, ui, tx, ty, tz, u);
}

// Metropolis step (iii), FP32 (one site or a pair of lanes): dH of Eq. 1
// restricted to the terms containing S_i, dH = J (S.h - S'.h) +
// K ((S.e)^2 - (S'.e)^2); the dot products are kept for the fused energy.
// Acceptance: dH <= 0 or P <= exp(-beta dH) = 2^(-beta log2(e) dH).
template <typename T>
struct Dots32 {
    T sh, th, se, pe, dH;
    T qs, qt;  // S^T A S and S'^T A S' (tensor term only)
};

// The on-site anisotropy tensor term S^T A S of a general symmetric A (the
// effective shape anisotropy the paper offers in place of dipolar coupling),
// A = (xx, yy, zz, xy, xz, yz): the product A S row by row, then its dot
// product with S.
template <typename T>
__device__ __forceinline__ T quad32(T x, T y, T z, const float (&A)[6]) {
    const T ax = f_fma(splat<T>(A[4]), z, f_fma(splat<T>(A[3]), y, f_mul(splat<T>(A[0]), x)));
    const T ay = f_fma(splat<T>(A[5]), z, f_fma(splat<T>(A[1]), y, f_mul(splat<T>(A[3]), x)));
    const T az = f_fma(splat<T>(A[2]), z, f_fma(splat<T>(A[5]), y, f_mul(splat<T>(A[4]), x)));
    return f_fma(z, az, f_fma(y, ay, f_mul(x, ax)));
}
__device__ __forceinline__ double quad64(double x, double y, double z, const double (&A)[6]) {
    const double ax = A[0] * x + A[3] * y + A[4] * z;
    const double ay = A[3] * x + A[1] * y + A[5] * z;
    const double az = A[4] * x + A[5] * y + A[2] * z;
    return x * ax + y * ay + z * az;
}

// TEN adds the tensor term: dH += S^T A S - S'^T A S'.  ZAX: the easy axis is
// e = (0, 0, 1) exactly, so S.e = S_z (what the three products give for it).
// KZ: K = +0, so the uniaxial term, +0 times a finite number, adds nothing
// (dH may differ only in the sign of a zero, which dH <= 0 does not see).
template <typename T, bool TEN = false, bool ZAX = false, bool KZ = false>
__device__ __forceinline__ Dots32<T> site_math32(T sx, T sy, T sz, T tx, T ty, T tz, T hx, T hy, T hz, float J,
                                                 float K, float ex, float ey, float ez, const float *A = nullptr) {
    Dots32<T> d;
    d.sh = f_fma(sz, hz, f_fma(sy, hy, f_mul(sx, hx)));
    d.th = f_fma(tz, hz, f_fma(ty, hy, f_mul(tx, hx)));
    if constexpr (ZAX) {
        d.se = sz;
        d.pe = tz;
    } else {
        d.se = f_fma(sz, splat<T>(ez), f_fma(sy, splat<T>(ey), f_mul(sx, splat<T>(ex))));
        d.pe = f_fma(tz, splat<T>(ez), f_fma(ty, splat<T>(ey), f_mul(tx, splat<T>(ex))));
    }
    if constexpr (KZ)
        d.dH = f_mul(splat<T>(J), f_sub(d.sh, d.th));
    else
        d.dH = f_fma(splat<T>(K), f_mul(f_sub(d.se, d.pe), f_add(d.se, d.pe)), f_mul(splat<T>(J), f_sub(d.sh, d.th)));
    if constexpr (TEN) {
        const float(&At)[6] = *reinterpret_cast<const float(*)[6]>(A);
        d.qs = quad32<T>(sx, sy, sz, At);
        d.qt = quad32<T>(tx, ty, tz, At);
        d.dH = f_add(d.dH, f_sub(d.qs, d.qt));
    }
    return d;
}

__device__ __forceinline__ bool accept32(float dH, float u, float neg_beta_log2e) {
    return (dH <= 0.0f) || (u <= ex2_hw(f_mul(neg_beta_log2e, dH)));
}

template <typename S, typename C> __device__ __forceinline__ S to_store(C v);
template <> __device__ __forceinline__ double to_store<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float to_store<float, float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_store<__half, float>(float v) { return __float2half_rn(v); }


// Metropolis step (iii) for one site in FP64: dH of Eq. 1 restricted to the
// terms that contain S_i, dH = J (S.h - S'.h) + K ((S.e)^2 - (S'.e)^2), then
// dH <= 0 or P <= exp(-beta dH).  The dot products are returned for the
// fused energy measurement.
template <typename C>
struct SiteDots {
    C sh, th, se, pe;
    C qs, qt;  // tensor term only
    bool acc;
};

// The FP64 acceptance P <= exp(x), x = -beta dH < 0, decided first in FP32:
// e = 2^(x log2(e)) from the hardware base-2 exponential has, for |x| <= 80,
// a relative error of at most 2^-22 (ex2) + 3 |x| 2^-24 (rounding x, log2(e)
// and their product to FP32) < 1.5e-5.  P lies in [uf, uf + 2^-24) (uf its
// top 24 bits, exact in FP32); the bounds e (1 -+ 3e-5), rounded to FP32, keep
// a margin over both errors, so outside that band the outcome of the FP64
// comparison is known.  Inside the band (or for |x| > 80) the FP64
// exponential decides, so the decision always equals the plain FP64 rule.
__device__ __forceinline__ bool accept64(double x, double u, float uf) {
    const float xf = (float)x;
    if (xf >= -80.0f) {
        const float y = __fmul_rn(xf, 1.44269504088896341f);
        float e;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(y));
        if (__fadd_rn(uf, 0x1p-24f) < __fmul_rn(e, 1.0f - 3e-5f)) return true;
        if (uf > __fmul_rn(e, 1.0f + 3e-5f)) return false;
    }
    return u <= exp(x);
}

// ZAX: the easy axis is e = (0, 0, 1) exactly, so S.e = S_z (what the three
// products give for that e, without them).
template <typename C, bool TEN = false, bool ZAX = false>
__device__ __forceinline__ SiteDots<C> metropolis(C sx, C sy, C sz, C tx, C ty, C tz, C hx, C hy, C hz, C J, C K,
                                                  C ex, C ey, C ez, C beta, C u, float uf,
                                                  const double *A = nullptr) {
    SiteDots<C> d;
    d.sh = sx * hx + sy * hy + sz * hz;
    d.th = tx * hx + ty * hy + tz * hz;
    if constexpr (ZAX) {
        d.se = sz;
        d.pe = tz;
    } else {
        d.se = sx * ex + sy * ey + sz * ez;
        d.pe = tx * ex + ty * ey + tz * ez;
    }
    // the uniaxial term K ((S.e)^2 - (S'.e)^2): for e = z as S_z^2 - S'_z^2 with one
    // rounding of S'_z^2 (an fma), else as the product of difference and sum
    C dH;
    if constexpr (ZAX)
        dH = fma(K, fma(d.se, d.se, -(d.pe * d.pe)), J * (d.sh - d.th));
    else
        dH = J * (d.sh - d.th) + K * ((d.se - d.pe) * (d.se + d.pe));
    if constexpr (TEN) {
        const double(&At)[6] = *reinterpret_cast<const double(*)[6]>(A);
        d.qs = quad64(sx, sy, sz, At);
        d.qt = quad64(tx, ty, tz, At);
        dH += d.qs - d.qt;
    }
    d.acc = (dH <= C(0)) || accept64(-beta * dH, u, uf);
    return d;
}

__device__ __forceinline__ void load_params(const PassArgs &a, double &J, double &K, double &ex, double &ey,
                                            double &ez, double &beta) {
    J = a.J;
    K = a.K;
    ex = a.e[0];
    ey = a.e[1];
    ez = a.e[2];
    beta = a.beta;
}
__device__ __forceinline__ void load_params(const PassArgs &a, float &J, float &K, float &ex, float &ey, float &ez,
                                            float &beta) {
    J = a.fJ;
    K = a.fK;
    ex = a.fe[0];
    ey = a.fe[1];
    ez = a.fe[2];
    beta = a.fbeta;
}

// ----------------------------------------------------------------- reduction
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Totals of one ring slot (one sweep of a.n_colours passes, or a standalone
// measurement), executed by one whole CTA: every CTA's partials of every
// partial set not in a.skip_sets, summed in a fixed order (so the FP64
// totals do not depend on scheduling); the result is valid in thread 0.
template <int NT = kBlock>
__device__ void slot_totals(const PassArgs &a, int slot, double (&tot)[kPartials]) {
    __shared__ double s_fin[NT / 32][kPartials];
    double t[kPartials] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const double *base = a.partials + (size_t)slot * a.n_colours * a.n_blocks * kPartials;
    for (int p = 0; p < a.n_colours; ++p) {
        if ((a.skip_sets >> p) & 1ull) continue;
        for (int b = threadIdx.x; b < a.n_blocks; b += NT) {
            const double *ps = base + ((size_t)p * a.n_blocks + b) * kPartials;
#pragma unroll
            for (int q = 0; q < kPartials; ++q) t[q] += __ldcg(ps + q);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kPartials; ++q) t[q] = warp_sum(t[q]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < kPartials; ++q) s_fin[warp][q] = t[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPartials; ++q) tot[q] = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w)
#pragma unroll
            for (int q = 0; q < kPartials; ++q) tot[q] += s_fin[w][q];
}

// Eq. 2 with |S| = 1 from one sweep's totals: o = E, Mx, My, Mz, |M|, M2, M4,
// |M.e| with M = sum S / N.
__device__ __forceinline__ void sweep_observables(const double (&tot)[kPartials], double n_present,
                                                  const double (&e)[3], double (&o)[8]) {
    const double mx = tot[1] / n_present;
    const double my = tot[2] / n_present;
    const double mz = tot[3] / n_present;
    const double m2 = mx * mx + my * my + mz * mz;
    o[0] = tot[0];
    o[1] = mx;
    o[2] = my;
    o[3] = mz;
    o[4] = sqrt(m2);
    o[5] = m2;
    o[6] = m2 * m2;
    o[7] = fabs(mx * e[0] + my * e[1] + mz * e[2]);
}

// Apply one sweep to an accumulator (one thread): the accepted count, the raw
// sums and, when measured, the observables o of sweep_observables and their
// moments.  Acc is DevAccum in device memory or AccRegs, a register copy of
// its fields.
template <class Acc>
__device__ __forceinline__ void apply_sweep(Acc &A, const double (&tot)[kPartials], const double (&o)[8],
                                            bool measured, bool accumulate) {
    A.accepted += tot[4];
#pragma unroll
    for (int q = 0; q < kPartials; ++q) A.sums[q] = tot[q];
    if (!measured) return;
#pragma unroll
    for (int q = 0; q < 8; ++q) A.last[q] = o[q];
    if (accumulate) {
        A.moments[HS_SUM_E] += o[0];
        A.moments[HS_SUM_E2] += o[0] * o[0];
        A.moments[HS_SUM_ABSM] += o[4];
        A.moments[HS_SUM_M2] += o[5];
        A.moments[HS_SUM_M4] += o[6];
        A.moments[HS_SUM_MX] += o[1];
        A.moments[HS_SUM_MY] += o[2];
        A.moments[HS_SUM_MZ] += o[3];
        A.moments[HS_SUM_ABSME] += o[7];
        A.count += 1.0;
    }
}

// The fields of DevAccum that apply_sweep updates, held in registers while
// one thread applies many sweeps (one read and one write of device memory).
struct AccRegs {
    double moments[HS_N_MOMENTS];
    double count, accepted;
    double last[8];
    double sums[kPartials];
    __device__ __forceinline__ void load(const DevAccum *A) {
#pragma unroll
        for (int q = 0; q < HS_N_MOMENTS; ++q) moments[q] = A->moments[q];
        count = A->count;
        accepted = A->accepted;
#pragma unroll
        for (int q = 0; q < 8; ++q) last[q] = A->last[q];
#pragma unroll
        for (int q = 0; q < kPartials; ++q) sums[q] = A->sums[q];
    }
    __device__ __forceinline__ void store(DevAccum *A) const {
#pragma unroll
        for (int q = 0; q < HS_N_MOMENTS; ++q) A->moments[q] = moments[q];
        A->count = count;
        A->accepted = accepted;
#pragma unroll
        for (int q = 0; q < 8; ++q) A->last[q] = last[q];
#pragma unroll
        for (int q = 0; q < kPartials; ++q) A->sums[q] = sums[q];
    }
};

// Finalise a single colour pass sequence or a standalone measurement inside
// its last kernel: the last of its CTAs to arrive folds the slots.  Every
// earlier launch of the sequence ran on the same stream and has completed
// (griddepcontrol.wait at kernel entry), so only this launch's CTAs count.
template <int NT = kBlock>
__device__ void finish_reduction(const PassArgs &a, bool measured) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned ticket = atomicAdd(&a.acc->done, 1u);
        s_last = (ticket == gridDim.x - 1u);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double tot[kPartials];
    slot_totals<NT>(a, a.slot, tot);
    if (threadIdx.x == 0) {
        double o[8];
        sweep_observables(tot, a.n_present, a.e, o);
        apply_sweep(*a.acc, tot, o, measured, a.accumulate == 1);
        a.acc->done = 0u;
    }
}

// NT = threads of the CTA (a multiple of 32).
template <typename C, bool MEAS, int NT = kBlock>
__device__ __forceinline__ void write_partials(const PassArgs &a, C e, C x, C y, C z, unsigned nacc) {
    __shared__ double s_w[NT / 32][kPartials];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (MEAS) {
        e = warp_sum(e);
        x = warp_sum(x);
        y = warp_sum(y);
        z = warp_sum(z);
    }
    nacc = __reduce_add_sync(0xffffffffu, nacc);
    if (lane == 0) {
        s_w[warp][0] = MEAS ? (double)e : 0.0;
        s_w[warp][1] = MEAS ? (double)x : 0.0;
        s_w[warp][2] = MEAS ? (double)y : 0.0;
        s_w[warp][3] = MEAS ? (double)z : 0.0;
        s_w[warp][4] = (double)nacc;
    }
    __syncthreads();
    if (threadIdx.x < kPartials) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) s += s_w[w][threadIdx.x];
        a.partials[(((size_t)a.slot * a.n_colours + a.pass) * a.n_blocks + blockIdx.x) * kPartials + threadIdx.x] = s;
    }
    if (a.finish) finish_reduction<NT>(a, MEAS);
}

// ----------------------------------------------------------------- stencil pass
// One colour pass of the periodic sc lattice in colour-major SoA layout.
// Work item = V consecutive sites of one row of the updated colour.  Row
// parity p = (y+z+c)&1 fixes where the x neighbours sit in the other colour's
// row: p = 0 -> (xh-1, xh), p = 1 -> (xh, xh+1); the +-y and +-z neighbours
// sit at the same xh in the adjacent rows.  Neighbour order of the local
// field sum: -x, +x, -y, +y, -z, +z.

// Per-thread partial sums of the fused measurement (E, S) and accepted moves.
// FP32 / FP16 accumulate in float2 lanes (even / odd site of a pair).
template <int P>
struct SiteAcc {
    float2 e = make_float2(0.f, 0.f), x = make_float2(0.f, 0.f), y = make_float2(0.f, 0.f),
           z = make_float2(0.f, 0.f);
    unsigned n = 0;
    __device__ __forceinline__ float E(float, float) const { return e.x + e.y; }
    __device__ __forceinline__ float X() const { return x.x + x.y; }
    __device__ __forceinline__ float Y() const { return y.x + y.y; }
    __device__ __forceinline__ float Z() const { return z.x + z.y; }
};
// FP64: the energy as its two sums, scaled once by -K and -J at the end:
// k = sum (S.e)^2 over the sites, j = sum S.h over the later colour's sites,
// e = the tensor term's share.
template <>
struct SiteAcc<HS_FP64> {
    double e = 0.0, k = 0.0, j = 0.0, x = 0.0, y = 0.0, z = 0.0;
    unsigned n = 0;
    __device__ __forceinline__ double E(double J, double K) const { return e - J * j - K * k; }
    __device__ __forceinline__ double X() const { return x; }
    __device__ __forceinline__ double Y() const { return y; }
    __device__ __forceinline__ double Z() const { return z; }
};

// -beta log2(e), rounded once; every FP32 path uses this same value.
__device__ __forceinline__ float neg_beta_log2e(float beta) { return f_mul(-beta, 1.44269504088896341f); }

// Step (i) for the V sites of one work item: the local field h[q][k] of site
// k, the sum of its neighbours in the order -x, +x, -y, +y, -z, +z, from the
// other colour's same row o (+ the edge element ed beyond it; row parity p
// picks (xh-1, xh) or (xh, xh+1) for the x neighbours) and its rows at y-1,
// y+1, z-1, z+1.  FP32 / FP16 add two sites at a time as the lanes of float2
// (identical per lane to the scalar adds).
template <int P, int V>
__device__ __forceinline__ void item_fields(const Vec<typename Tr<P>::S, V> (&o)[3],
                                            const Vec<typename Tr<P>::S, V> (&nym)[3],
                                            const Vec<typename Tr<P>::S, V> (&nyp)[3],
                                            const Vec<typename Tr<P>::S, V> (&nzm)[3],
                                            const Vec<typename Tr<P>::S, V> (&nzp)[3], const typename Tr<P>::C (&ed)[3],
                                            uint32_t p, typename Tr<P>::C (&h)[3][V]) {
    using C = typename Tr<P>::C;
    auto xm_of = [&](int k, int q) -> C { return p ? to_c(o[q].v[k]) : (k == 0 ? ed[q] : to_c(o[q].v[k - 1])); };
    auto xp_of = [&](int k, int q) -> C { return p ? (k == V - 1 ? ed[q] : to_c(o[q].v[k + 1])) : to_c(o[q].v[k]); };
    if constexpr (P == HS_FP64) {
#pragma unroll
        for (int k = 0; k < V; ++k)
#pragma unroll
            for (int q = 0; q < 3; ++q)
                h[q][k] = ((((xm_of(k, q) + xp_of(k, q)) + to_c(nym[q].v[k])) + to_c(nyp[q].v[k])) +
                           to_c(nzm[q].v[k])) +
                          to_c(nzp[q].v[k]);
    } else if constexpr (P == HS_FP16) {
        // binary16 operands added straight into the FP32 sum (add_half: one
        // rounding per add, the same sums as widening each operand first)
#pragma unroll
        for (int k = 0; k < V; ++k)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                float t = xm_of(k, q);
                if (k == V - 1)
                    t = p ? f_add(t, ed[q]) : add_half(t, o[q].v[k]);
                else
                    t = add_half(t, p ? o[q].v[k + 1] : o[q].v[k]);
                t = add_half(t, nym[q].v[k]);
                t = add_half(t, nyp[q].v[k]);
                t = add_half(t, nzm[q].v[k]);
                h[q][k] = add_half(t, nzp[q].v[k]);
            }
    } else if constexpr (V >= 2) {
#pragma unroll
        for (int j = 0; j < V / 2; ++j) {
            const int k0 = 2 * j, k1 = 2 * j + 1;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float2 xm = make_float2(xm_of(k0, q), xm_of(k1, q));
                const float2 xp = make_float2(xp_of(k0, q), xp_of(k1, q));
                const float2 ym = make_float2(to_c(nym[q].v[k0]), to_c(nym[q].v[k1]));
                const float2 yp = make_float2(to_c(nyp[q].v[k0]), to_c(nyp[q].v[k1]));
                const float2 zm = make_float2(to_c(nzm[q].v[k0]), to_c(nzm[q].v[k1]));
                const float2 zp = make_float2(to_c(nzp[q].v[k0]), to_c(nzp[q].v[k1]));
                const float2 hh = f_add(f_add(f_add(f_add(f_add(xm, xp), ym), yp), zm), zp);
                h[q][k0] = hh.x;
                h[q][k1] = hh.y;
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < 3; ++q)
            h[q][0] = f_add(f_add(f_add(f_add(f_add(xm_of(0, q), xp_of(0, q)), to_c(nym[q].v[0])), to_c(nyp[q].v[0])),
                                  to_c(nzm[q].v[0])),
                            to_c(nzp[q].v[0]));
    }
}

// Metropolis steps (ii)-(iii) for the V sites of one FP64 work item (see
// update_item_h); ZAX as in metropolis.
template <int V, bool MEAS, bool TEN, bool ZAX>
__device__ __forceinline__ bool update_fp64(Vec<double, V> (&s)[3], const double (&h)[3][V], uint32_t site0, int c,
                                            const PassArgs &a, double J, double K, double ex, double ey, double ez,
                                            double beta, SiteAcc<HS_FP64> &acc) {
    using C = double;
    bool any = false;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        C tx, ty, tz, u;
        float uf;
        draw_trial64(site0 + 2u * k, a.sweep, (uint32_t)c, a.replica, a.key0, a.key1, a.sc_tab, tx, ty, tz, u,
                     uf);
        C sx = s[0].v[k], sy = s[1].v[k], sz = s[2].v[k];
        const SiteDots<C> d = metropolis<C, TEN, ZAX>(sx, sy, sz, tx, ty, tz, h[0][k], h[1][k], h[2][k], J, K,
                                                      ex, ey, ez, beta, u, uf, a.A);
        if (d.acc) {
            sx = tx;
            sy = ty;
            sz = tz;
            s[0].v[k] = tx;
            s[1].v[k] = ty;
            s[2].v[k] = tz;
            any = true;
            ++acc.n;
        }
        if (MEAS) {
            // bond energy counted at the later colour's end: pass 1 owns
            // every sc bond, pass 0 only the anisotropy term
            const C e_new = d.acc ? d.pe : d.se;
            acc.k = fma(e_new, e_new, acc.k);
            if (TEN) acc.e -= d.acc ? d.qt : d.qs;
            if (c == 1) acc.j += d.acc ? d.th : d.sh;
            acc.x += sx;
            acc.y += sy;
            acc.z += sz;
        }
    }
    return any;
}

// Metropolis steps (ii)-(iii) for the V sites of one work item, given the
// item's own spins s and the local fields h of step (i).  site0 is the
// natural index of the item's first site (the FP64 schedule's counter), rank0
// its rank within its colour class (the FP32 / FP16 schedule's; on a periodic
// sc lattice the natural index halved, kept separately so that it stays exact
// beyond 2^32 sites).  Updates s in place; returns whether any site was
// accepted.
// Metropolis steps (ii)-(iii) for the V sites of one FP32 / FP16 work item
// (see update_item_h); ZAX as in site_math32.
// KZ (with ZAX): K = +0, whose energy share -K (S.e)^2 is -0 (written as such,
// so every sum takes the same values; adding -0 changes none).
template <int P, int V, bool MEAS, bool TEN, bool ZAX, bool KZ = false>
__device__ __forceinline__ bool update_f32(Vec<typename Tr<P>::S, V> (&s)[3], const float (&h)[3][V], uint32_t rank0,
                                           int c, const PassArgs &a, float J, float K, float ex, float ey, float ez,
                                           float beta, SiteAcc<P> &acc) {
    using S = typename Tr<P>::S;
    using C = float;
    bool any = false;
    const float nb = neg_beta_log2e(beta);
    // one site in lane x of the accumulators
    auto single = [&](int k, float tx, float ty, float tz, float u) {
        const float sx = to_c(s[0].v[k]), sy = to_c(s[1].v[k]), sz = to_c(s[2].v[k]);
        const Dots32<float> d = site_math32<float, TEN, ZAX, KZ>(sx, sy, sz, tx, ty, tz, h[0][k], h[1][k], h[2][k], J, K,
                                                        ex, ey, ez, a.fA);
        const bool ac = accept32(d.dH, u, nb);
        if (ac) {
            s[0].v[k] = to_store<S, C>(tx);
            s[1].v[k] = to_store<S, C>(ty);
            s[2].v[k] = to_store<S, C>(tz);
            any = true;
            ++acc.n;
        }
        if (MEAS) {
            const float en = ac ? d.pe : d.se;
            float ei = KZ ? -0.0f : f_mul(-K, f_mul(en, en));
            if (TEN) ei = f_sub(ei, ac ? d.qt : d.qs);
            if (c == 1) ei = f_fma(-J, ac ? d.th : d.sh, ei);
            acc.e.x = f_add(acc.e.x, ei);
            acc.x.x = f_add(acc.x.x, ac ? tx : sx);
            acc.y.x = f_add(acc.y.x, ac ? ty : sy);
            acc.z.x = f_add(acc.z.x, ac ? tz : sz);
        }
    };
    // ranks of the item's sites in their colour class: rank0 + k
    if (V >= 2 && (rank0 & 1u) == 0u) {
#pragma unroll
        for (int j = 0; j < V / 2; ++j) {  // one Philox block and packed arithmetic per pair
            const int k0 = 2 * j, k1 = 2 * j + 1;
            const uint4 w = trial_block((rank0 >> 1) + j, a.sweep, (uint32_t)c, a.replica, a.key0, a.key1);
            float2 zi, vi, ui;
            half_ints(w.x, w.y, zi.x, vi.x, ui.x);
            half_ints(w.z, w.w, zi.y, vi.y, ui.y);
            float2 tx, ty, tz, u;
            trial32<P, float2>(zi, vi, ui, tx, ty, tz, u);
            float2 hp[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) hp[q] = make_float2(h[q][k0], h[q][k1]);
            const float2 sx = make_float2(to_c(s[0].v[k0]), to_c(s[0].v[k1]));
            const float2 sy = make_float2(to_c(s[1].v[k0]), to_c(s[1].v[k1]));
            const float2 sz = make_float2(to_c(s[2].v[k0]), to_c(s[2].v[k1]));
            const Dots32<float2> d =
                site_math32<float2, TEN, ZAX, KZ>(sx, sy, sz, tx, ty, tz, hp[0], hp[1], hp[2], J, K, ex, ey, ez, a.fA);
            const bool a0 = accept32(d.dH.x, u.x, nb);
            const bool a1 = accept32(d.dH.y, u.y, nb);
            if (a0) {
                s[0].v[k0] = to_store<S, C>(tx.x);
                s[1].v[k0] = to_store<S, C>(ty.x);
                s[2].v[k0] = to_store<S, C>(tz.x);
                ++acc.n;
            }
            if (a1) {
                s[0].v[k1] = to_store<S, C>(tx.y);
                s[1].v[k1] = to_store<S, C>(ty.y);
                s[2].v[k1] = to_store<S, C>(tz.y);
                ++acc.n;
            }
            any = any || a0 || a1;
            if (MEAS) {
                const float2 en = make_float2(a0 ? d.pe.x : d.se.x, a1 ? d.pe.y : d.se.y);
                float2 ei = KZ ? make_float2(-0.0f, -0.0f) : f_mul(splat<float2>(-K), f_mul(en, en));
                if (TEN) ei = f_sub(ei, make_float2(a0 ? d.qt.x : d.qs.x, a1 ? d.qt.y : d.qs.y));
                if (c == 1)
                    ei = f_fma(splat<float2>(-J), make_float2(a0 ? d.th.x : d.sh.x, a1 ? d.th.y : d.sh.y), ei);
                acc.e = f_add(acc.e, ei);
                acc.x = f_add(acc.x, make_float2(a0 ? tx.x : sx.x, a1 ? tx.y : sx.y));
                acc.y = f_add(acc.y, make_float2(a0 ? ty.x : sy.x, a1 ? ty.y : sy.y));
                acc.z = f_add(acc.z, make_float2(a0 ? tz.x : sz.x, a1 ? tz.y : sz.y));
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k) {
            float tx, ty, tz, u;
            draw_trial_rank<P>(rank0 + k, a.sweep, (uint32_t)c, a.replica, a.key0, a.key1, tx, ty, tz, u);
            single(k, tx, ty, tz, u);
        }
    }
    return any;
}

// AX = 1: the kernel was chosen for e = (0, 0, 1) at launch, so S.e = S_z
// with no branch (the FP32 register stencil's form); AX = 2: the same with
// K = +0 (the FP32 and FP16 batch kernels); AX = 0: FP64 and FP16 decide per
// work item from PassArgs::zaxis, FP32 takes the general products.
template <int P, int V, bool MEAS, bool TEN = false, int AX = 0>
__device__ __forceinline__ bool update_item_h(Vec<typename Tr<P>::S, V> (&s)[3], const typename Tr<P>::C (&h)[3][V],
                                              uint32_t site0, uint32_t rank0, int c, const PassArgs &a,
                                              typename Tr<P>::C J, typename Tr<P>::C K, typename Tr<P>::C ex,
                                              typename Tr<P>::C ey, typename Tr<P>::C ez, typename Tr<P>::C beta,
                                              SiteAcc<P> &acc) {
    if constexpr (P == HS_FP64) {
        // one uniform branch per work item: the item body with S.e = S_z
        // (e = (0, 0, 1), the FP64 pipe spared six operations per site) or
        // with the general dot products
        if constexpr (!TEN)
            if (a.zaxis) return update_fp64<V, MEAS, false, true>(s, h, site0, c, a, J, K, ex, ey, ez, beta, acc);
        return update_fp64<V, MEAS, TEN, false>(s, h, site0, c, a, J, K, ex, ey, ez, beta, acc);
    } else {
        if constexpr (AX >= 1 && !TEN)
            return update_f32<P, V, MEAS, false, true, AX == 2>(s, h, rank0, c, a, J, K, ex, ey, ez, beta, acc);
        // FP16 (bound by instruction issue, its loads decoupled by the
        // pipelined landing slots) takes the same branch; the FP32 register
        // stencil, bound by load latency, measured slower with it (the branch
        // between an item's loads and its arithmetic costs more than the three
        // instructions per site it saves) and keeps the general products
        if constexpr (!TEN && P == HS_FP16)
            if (a.zaxis) return update_f32<P, V, MEAS, false, true>(s, h, rank0, c, a, J, K, ex, ey, ez, beta, acc);
        return update_f32<P, V, MEAS, TEN, false>(s, h, rank0, c, a, J, K, ex, ey, ez, beta, acc);
    }
}

// The same from the raw operands: step (i) then steps (ii)-(iii).
template <int P, int V, bool MEAS, bool TEN = false, int AX = 0>
__device__ __forceinline__ bool update_item(Vec<typename Tr<P>::S, V> (&s)[3], const Vec<typename Tr<P>::S, V> (&o)[3],
                                            const Vec<typename Tr<P>::S, V> (&nym)[3],
                                            const Vec<typename Tr<P>::S, V> (&nyp)[3],
                                            const Vec<typename Tr<P>::S, V> (&nzm)[3],
                                            const Vec<typename Tr<P>::S, V> (&nzp)[3], const typename Tr<P>::C (&ed)[3],
                                            uint32_t p, uint32_t site0, uint32_t rank0, int c, const PassArgs &a,
                                            typename Tr<P>::C J, typename Tr<P>::C K, typename Tr<P>::C ex,
                                            typename Tr<P>::C ey, typename Tr<P>::C ez, typename Tr<P>::C beta,
                                            SiteAcc<P> &acc) {
    typename Tr<P>::C h[3][V];
    item_fields<P, V>(o, nym, nyp, nzm, nzp, ed, p, h);
    return update_item_h<P, V, MEAS, TEN, AX>(s, h, site0, rank0, c, a, J, K, ex, ey, ez, beta, acc);
}

// Vector load, optionally L2-only (ld.global.cg).  A kernel that reads data
// other CTAs wrote earlier in the same launch must not be served from a
// stale line of its SM's L1 (L1 is not coherent across SMs).
template <typename T, bool CG>
__device__ __forceinline__ T ld_val(const T *p) {
    if constexpr (!CG) {
        return *p;
    } else {
        T out;
        if constexpr (sizeof(T) == 16) {
            const uint4 v = __ldcg(reinterpret_cast<const uint4 *>(p));
            memcpy(&out, &v, 16);
        } else if constexpr (sizeof(T) == 8) {
            const uint2 v = __ldcg(reinterpret_cast<const uint2 *>(p));
            memcpy(&out, &v, 8);
        } else if constexpr (sizeof(T) == 4) {
            const unsigned int v = __ldcg(reinterpret_cast<const unsigned int *>(p));
            memcpy(&out, &v, 4);
        } else {
            const unsigned short v = __ldcg(reinterpret_cast<const unsigned short *>(p));
            memcpy(&out, &v, 2);
        }
        return out;
    }
}

// Operands of one work item of the register stencil.
template <int P, int V>
struct StencilItem {
    Vec<typename Tr<P>::S, V> s[3], o[3], nym[3], nyp[3], nzm[3], nzp[3];
    typename Tr<P>::C ed[3];
    uint32_t b0, p, site0, rank0;
};

// Element offsets (within a colour plane) of the operands of the work item at
// row (y, z), vector xv: the own vector b0 (and the other colour's same-row
// vector at the same offset), the other colour's rows at y-1, y+1, z-1, z+1,
// and the edge element beyond the row vector on the side parity p picks.
struct ItemOffsets {
    uint32_t b0, bym, byp, bzm, bzp, bed, p, site0, rank0;
};

template <int V>
__device__ __forceinline__ ItemOffsets item_offsets(const PassArgs &a, uint32_t y, uint32_t z, uint32_t xv) {
    const uint32_t Lh = a.Lh, Ly = a.Ly, Lz = a.Lz, Lx = a.Lx;
    const uint32_t row = z * Ly + y;
    const uint32_t xh0 = xv * V;
    const uint32_t ym = (y == 0) ? Ly - 1 : y - 1;
    const uint32_t yp = (y == Ly - 1) ? 0 : y + 1;
    const uint32_t zm = (z == 0) ? Lz - 1 : z - 1;
    const uint32_t zp = (z == Lz - 1) ? 0 : z + 1;
    ItemOffsets o;
    o.p = (y + z + (uint32_t)a.colour + (uint32_t)a.zpar) & 1u;
    o.b0 = row * Lh + xh0;
    o.bym = (z * Ly + ym) * Lh + xh0;
    o.byp = (z * Ly + yp) * Lh + xh0;
    o.bzm = (zm * Ly + y) * Lh + xh0;
    o.bzp = (zp * Ly + y) * Lh + xh0;
    o.bed = row * Lh + (o.p ? ((xh0 + V == Lh) ? 0 : xh0 + V) : ((xh0 == 0) ? Lh - 1 : xh0 - 1));
    o.site0 = row * Lx + 2 * xh0 + o.p + a.site_off;
    o.rank0 = row * Lh + xh0 + a.rank_off;  // (row Lx + 2 xh0 + p) / 2 + the slab's offset
    return o;
}

// Load the operands of the work item at row (y, z), vector xv.
template <int P, int V, bool CG = false>
__device__ __forceinline__ void load_item_at(const PassArgs &a, uint32_t y, uint32_t z, uint32_t xv,
                                             const typename Tr<P>::S *const (&own)[3],
                                             const typename Tr<P>::S *const (&oth)[3], StencilItem<P, V> &it) {
    using S = typename Tr<P>::S;
    using VT = Vec<S, V>;
    const ItemOffsets f = item_offsets<V>(a, y, z, xv);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        it.s[q] = ld_val<VT, CG>(reinterpret_cast<const VT *>(own[q] + f.b0));
        it.o[q] = ld_val<VT, CG>(reinterpret_cast<const VT *>(oth[q] + f.b0));
        it.nym[q] = ld_val<VT, CG>(reinterpret_cast<const VT *>(oth[q] + f.bym));
        it.nyp[q] = ld_val<VT, CG>(reinterpret_cast<const VT *>(oth[q] + f.byp));
        it.nzm[q] = ld_val<VT, CG>(reinterpret_cast<const VT *>(oth[q] + f.bzm));
        it.nzp[q] = ld_val<VT, CG>(reinterpret_cast<const VT *>(oth[q] + f.bzp));
        it.ed[q] = to_c(ld_val<S, CG>(oth[q] + f.bed));
    }
    it.b0 = f.b0;
    it.p = f.p;
    it.site0 = f.site0;
    it.rank0 = f.rank0;
}

// The work item with linear index t = (z Ly + y) (Lh/V) + xv (rev - t in a
// descending pass; DIR = false: always ascending, with no reference to rev).
template <int P, int V, bool CG = false, bool DIR = true>
__device__ __forceinline__ void load_item(const PassArgs &a, uint32_t t, const typename Tr<P>::S *const (&own)[3],
                                          const typename Tr<P>::S *const (&oth)[3], StencilItem<P, V> &it) {
    if constexpr (DIR) t = a.rev ? a.rev - t : t;  // a descending pass
    const uint32_t nxv = a.Lh / V;
    const uint32_t r = a.div_nxv.div(t);
    const uint32_t xv = t - r * nxv;
    const uint32_t row = r + (uint32_t)(a.z_off * a.Ly);  // a z-slab's own rows start after its halo plane
    const uint32_t z = a.div_ly.div(row);
    const uint32_t y = row - z * a.Ly;
    load_item_at<P, V, CG>(a, y, z, xv, own, oth, it);
}

// Split loading of the work item with linear index t (see the split
// prefetch of the stencil kernels): part A -- the own row, the other colour's
// same row (+ edge element) and its rows at z-1 and z+1 -- is loaded ahead;
// part B -- the rows at y-1 and y+1 -- when the item is taken up.
template <int P, int V>
struct SplitItem {
    Vec<typename Tr<P>::S, V> s[3], o[3], nzm[3], nzp[3];
    typename Tr<P>::C ed[3];
    ItemOffsets f;
};

template <int P, int V, bool CG = false, bool DIR = true>
__device__ __forceinline__ void load_split_a(const PassArgs &a, uint32_t t, const typename Tr<P>::S *const (&own)[3],
                                             const typename Tr<P>::S *const (&oth)[3], SplitItem<P, V> &A) {
    using S = typename Tr<P>::S;
    using VT = Vec<S, V>;
    if constexpr (DIR) t = a.rev ? a.rev - t : t;  // a descending pass
    const uint32_t nxv = a.Lh / V;
    const uint32_t r = a.div_nxv.div(t);
    const uint32_t xv = t - r * nxv;
    const uint32_t row = r + (uint32_t)(a.z_off * a.Ly);
    const uint32_t z = a.div_ly.div(row);
    A.f = item_offsets<V>(a, row - z * a.Ly, z, xv);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        A.s[q] = ld_val<VT, CG>(reinterpret_cast<const VT *>(own[q] + A.f.b0));
        A.o[q] = ld_val<VT, CG>(reinterpret_cast<const VT *>(oth[q] + A.f.b0));
        A.nzm[q] = ld_val<VT, CG>(reinterpret_cast<const VT *>(oth[q] + A.f.bzm));
        A.nzp[q] = ld_val<VT, CG>(reinterpret_cast<const VT *>(oth[q] + A.f.bzp));
        A.ed[q] = to_c(ld_val<S, CG>(oth[q] + A.f.bed));
    }
}

template <int P, int V, bool CG = false>
__device__ __forceinline__ void load_split_b(const SplitItem<P, V> &A, const typename Tr<P>::S *const (&oth)[3],
                                             Vec<typename Tr<P>::S, V> (&nym)[3], Vec<typename Tr<P>::S, V> (&nyp)[3]) {
    using VT = Vec<typename Tr<P>::S, V>;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        nym[q] = ld_val<VT, CG>(reinterpret_cast<const VT *>(oth[q] + A.f.bym));
        nyp[q] = ld_val<VT, CG>(reinterpret_cast<const VT *>(oth[q] + A.f.byp));
    }
}

}  // namespace
}  // namespace hs
