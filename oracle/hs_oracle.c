/*
 * hs_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for the
 * single-spin Metropolis sweep of the classical anisotropic Heisenberg model.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or helper
 * with the CUDA library; the two are written separately and compared.
 *
 * What it follows (arXiv 2106.11286):
 *   - Eq. 1:  H = -J sum_<ij> S_i.S_j - K sum_i (S_i.e)^2, |S_i| = 1
 *             (each nearest-neighbour bond counted once).
 *   - The effective shape anisotropy the paper names as the stand-in for
 *             dipolar coupling (introduction, GPU implementation paragraph),
 *             read as a general on-site quadratic term -sum_i S_i^T A S_i
 *             with one symmetric 3x3 tensor A for every site, stored as
 *             (Axx, Ayy, Azz, Axy, Axz, Ayz); A = NULL means no such term.
 *   - Metropolis steps (i)-(iii): pick a site, propose a new orientation at
 *             random, accept if dH <= 0, else accept iff P <= exp(-beta dH)
 *             with P uniform in [0,1).
 *   - Eq. 2:  M = (1 / (N |S|)) sum_i S_i.
 * Readings where the paper is silent (all listed in the design notes):
 *   - sites are visited colour class by colour class (independent sets of
 *     the neighbour graph), ascending natural index inside a class;
 *   - the trial orientation is uniform on the sphere: z = 2u-1,
 *     phi = pi (2u'-1), r = sqrt((1-z)(1+z)), S' = (r cos phi, r sin phi, z);
 *   - random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11), counter
 *     (index, sweep, tag<<24 | colour<<8 | call, replica), key (seed lo, hi);
 *     index = natural site index (FP64 schedule, initial spins) or the
 *     site's rank within its colour class halved (FP32 schedule).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no FMA
 * contraction, so every product and sum is the one written here; OpenMP only
 * shares one colour class among threads in or_sweep_parallel).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition (SC'11, Sec. 4 / Table 2):  */
/* a round multiplies words 0 and 2 by two fixed odd constants, swaps the   */
/* high/low halves across lanes and xors in the round key; the key is       */
/* bumped by the two Weyl constants between rounds.                          */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform in [0,1) on the 2^-53 grid from two words (27 + 26 top bits).   */
double or_u53(uint32_t a, uint32_t b)
{
    double hi = (double)(a >> 5);
    double lo = (double)(b >> 6);
    return (hi * 67108864.0 + lo) / 9007199254740992.0; /* 2^26, 2^53 */
}

/* Uniform in [0,1) on the 2^-24 grid from the top 24 bits of one word.     */
double or_u24(uint32_t a)
{
    return (double)(a >> 8) / 16777216.0; /* 2^24 */
}

enum { OR_TAG_TRIAL = 0, OR_TAG_INIT = 1 };

/* Counter/key schedule of one Philox call. */
static void or_draw(uint64_t seed, uint32_t replica, uint64_t site, uint64_t sweep,
                    uint32_t tag, uint32_t colour, uint32_t call, uint32_t out[4])
{
    uint32_t ctr[4], key[2];
    ctr[0] = (uint32_t)site;
    ctr[1] = (uint32_t)sweep;
    ctr[2] = (tag << 24) | (colour << 8) | call;
    ctr[3] = replica;
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
    or_philox4x32_10(ctr, key, out);
}

/* Uniform point on the unit sphere from two uniforms (Archimedes: z is
 * uniform on [-1,1), the azimuth uniform on [-pi,pi)). */
static void or_sphere_point(double uz, double uphi, double s[3])
{
    double z = 2.0 * uz - 1.0;
    double v = 2.0 * uphi - 1.0;
    double phi = M_PI * v;
    double r = sqrt((1.0 - z) * (1.0 + z));
    s[0] = r * cos(phi);
    s[1] = r * sin(phi);
    s[2] = z;
}

/* Draw the two uniforms (u_z, u_phi) and the acceptance uniform P of one
 * trial move.
 * mode 0 (FP64 schedule): two Philox blocks keyed by the natural site index
 *   (calls 0 and 1), three 53-bit uniforms: u_z from words 0,1 and u_phi
 *   from words 2,3 of call 0, P from words 0,1 of call 1.
 * mode 1 and 2 (FP32 schedule): one Philox block serves two sites of the
 *   same colour: the site whose rank among the present sites of its colour
 *   (ascending natural index) is r uses block r >> 1 (counter word 0) and
 *   its half r & 1, i.e. words a = 2(r&1) and b = a+1.  u_z and u_phi are
 *   the top 21 bits of a and b, P the two low 11-bit fields (a's above b's),
 *   22 bits: u = k 2^-21, P = k 2^-22. */
void or_trial_uniforms(int mode, uint64_t seed, uint32_t replica, uint64_t site, uint64_t rank, uint64_t sweep,
                       uint32_t colour, double u[3])
{
    uint32_t r[4];
    if (mode == 0) {
        or_draw(seed, replica, site, sweep, OR_TAG_TRIAL, colour, 0, r);
        u[0] = or_u53(r[0], r[1]);
        u[1] = or_u53(r[2], r[3]);
        or_draw(seed, replica, site, sweep, OR_TAG_TRIAL, colour, 1, r);
        u[2] = or_u53(r[0], r[1]);
    } else {
        or_draw(seed, replica, rank >> 1, sweep, OR_TAG_TRIAL, colour, 0, r);
        uint32_t a = r[2 * (rank & 1)];
        uint32_t b = r[2 * (rank & 1) + 1];
        u[0] = (double)(a >> 11) / 2097152.0;                               /* 2^21 */
        u[1] = (double)(b >> 11) / 2097152.0;
        u[2] = (double)(((a & 0x7FFu) << 11) | (b & 0x7FFu)) / 4194304.0;  /* 2^22 */
    }
}

/* Round a double to the nearest binary16 value (round half to even),
 * returned as a double.  Written from the IEEE 754 binary16 definition:
 * 11 significant bits for |x| >= 2^-14, a fixed 2^-24 spacing below. */
double or_round_half(double x)
{
    if (x == 0.0 || !isfinite(x))
        return x;
    double a = fabs(x);
    int e;
    frexp(a, &e); /* a = f * 2^e, f in [0.5,1) */
    int exp_unbiased = e - 1; /* a in [2^(e-1), 2^e) */
    double quantum;
    if (exp_unbiased < -14)
        quantum = ldexp(1.0, -24);
    else
        quantum = ldexp(1.0, exp_unbiased - 10);
    double q = a / quantum;            /* exact: power-of-two scaling */
    double n = nearbyint(q);           /* default rounding: half to even */
    double rounded = n * quantum;
    if (rounded > 65504.0)
        rounded = INFINITY;
    return x < 0 ? -rounded : rounded;
}

/* ------------------------------------------------------------------------ */
/* Lattices.  Natural index:                                                 */
/*   sc : i = (z*Ly + y)*Lx + x                                              */
/*   bcc: i = ((cz*Ly + cy)*Lx + cx)*2 + b, b=0 cube corner, b=1 centre      */
/*   fcc: i = ((cz*Ly + cy)*Lx + cx)*4 + b, basis (0,0,0),(0,h,h),(h,0,h),   */
/*        (h,h,0) with h = 1/2                                               */
/* Neighbour order of each site is fixed:                                    */
/*   sc : -x, +x, -y, +y, -z, +z                                             */
/*   bcc: the 8 diagonal offsets with dz, then dy, then dx ascending         */
/*   fcc: the 12 offsets (two half-integer components) with dz, dy, dx       */
/*        ascending                                                          */
/* Open boundaries drop the missing neighbours; periodic ones wrap.          */
/* Each builder fills row_ptr[n+1]; col may be NULL to count only.           */
/* ------------------------------------------------------------------------ */
static int wrap(int v, int L, int periodic, int *ok)
{
    if (v >= 0 && v < L)
        return v;
    if (!periodic) {
        *ok = 0;
        return 0;
    }
    return ((v % L) + L) % L;
}

/* Neighbours of sc site i in the fixed order -x, +x, -y, +y, -z, +z;
 * returns how many exist (6 when periodic). */
int or_sc_site_neighbours(int Lx, int Ly, int Lz, int periodic, int64_t i, int64_t *out)
{
    static const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    const int x = (int)(i % Lx);
    const int y = (int)((i / Lx) % Ly);
    const int z = (int)(i / ((int64_t)Lx * Ly));
    int n = 0;
    for (int k = 0; k < 6; ++k) {
        int ok = 1;
        int nx = wrap(x + off[k][0], Lx, periodic, &ok);
        int ny = wrap(y + off[k][1], Ly, periodic, &ok);
        int nz = wrap(z + off[k][2], Lz, periodic, &ok);
        if (!ok)
            continue;
        out[n++] = ((int64_t)nz * Ly + ny) * Lx + nx;
    }
    return n;
}

/* The same for m sites: out[6t..6t+5] (unused slots -1), returns nothing. */
void or_sc_sites_neighbours(int Lx, int Ly, int Lz, int periodic, int64_t m, const int64_t *sites, int64_t *out)
{
    for (int64_t t = 0; t < m; ++t) {
        const int n = or_sc_site_neighbours(Lx, Ly, Lz, periodic, sites[t], &out[6 * t]);
        for (int k = n; k < 6; ++k)
            out[6 * t + k] = -1;
    }
}

int64_t or_sc_neighbours(int Lx, int Ly, int Lz, int periodic, int64_t *row_ptr, int32_t *col)
{
    const int64_t n_sites = (int64_t)Lx * Ly * Lz;
    int64_t nnz = 0;
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n_sites; ++i) {
        int64_t nb[6];
        const int n = or_sc_site_neighbours(Lx, Ly, Lz, periodic, i, nb);
        for (int k = 0; k < n; ++k) {
            if (col)
                col[nnz] = (int32_t)nb[k];
            ++nnz;
        }
        row_ptr[i + 1] = nnz;
    }
    return nnz;
}

int64_t or_bcc_neighbours(int Lx, int Ly, int Lz, int periodic, int64_t *row_ptr, int32_t *col)
{
    int64_t nnz = 0;
    int64_t i = 0;
    row_ptr[0] = 0;
    for (int cz = 0; cz < Lz; ++cz)
        for (int cy = 0; cy < Ly; ++cy)
            for (int cx = 0; cx < Lx; ++cx)
                for (int b = 0; b < 2; ++b, ++i) {
                    /* corner (b=0) sees the centres of the 8 cells around it,
                     * i.e. cell offsets in {-1,0}; a centre (b=1) sees the 8
                     * corners of its own cell, i.e. offsets in {0,1}. */
                    int lo = (b == 0) ? -1 : 0;
                    for (int dz = lo; dz <= lo + 1; ++dz)
                        for (int dy = lo; dy <= lo + 1; ++dy)
                            for (int dx = lo; dx <= lo + 1; ++dx) {
                                int ok = 1;
                                int nx = wrap(cx + dx, Lx, periodic, &ok);
                                int ny = wrap(cy + dy, Ly, periodic, &ok);
                                int nz = wrap(cz + dz, Lz, periodic, &ok);
                                if (!ok)
                                    continue;
                                if (col)
                                    col[nnz] = (int32_t)((((int64_t)nz * Ly + ny) * Lx + nx) * 2 + (1 - b));
                                ++nnz;
                            }
                    row_ptr[i + 1] = nnz;
                }
    return nnz;
}

/* fcc basis in half-lattice-constant units. */
static const int fcc_basis[4][3] = {{0, 0, 0}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};

static int fcc_basis_index(int px, int py, int pz)
{
    for (int b = 0; b < 4; ++b)
        if (fcc_basis[b][0] == px && fcc_basis[b][1] == py && fcc_basis[b][2] == pz)
            return b;
    return -1;
}

static int floor_div2(int v) { return (v >= 0) ? v / 2 : -((-v + 1) / 2); }

int64_t or_fcc_neighbours(int Lx, int Ly, int Lz, int periodic, int64_t *row_ptr, int32_t *col)
{
    int64_t nnz = 0;
    int64_t i = 0;
    row_ptr[0] = 0;
    for (int cz = 0; cz < Lz; ++cz)
        for (int cy = 0; cy < Ly; ++cy)
            for (int cx = 0; cx < Lx; ++cx)
                for (int b = 0; b < 4; ++b, ++i) {
                    /* position in half units */
                    int px = 2 * cx + fcc_basis[b][0];
                    int py = 2 * cy + fcc_basis[b][1];
                    int pz = 2 * cz + fcc_basis[b][2];
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                int nonzero = (dx != 0) + (dy != 0) + (dz != 0);
                                if (nonzero != 2)
                                    continue;
                                int qx = px + dx, qy = py + dy, qz = pz + dz;
                                int ncx = floor_div2(qx), ncy = floor_div2(qy), ncz = floor_div2(qz);
                                int nb = fcc_basis_index(qx - 2 * ncx, qy - 2 * ncy, qz - 2 * ncz);
                                int ok = (nb >= 0);
                                ncx = wrap(ncx, Lx, periodic, &ok);
                                ncy = wrap(ncy, Ly, periodic, &ok);
                                ncz = wrap(ncz, Lz, periodic, &ok);
                                if (!ok)
                                    continue;
                                if (col)
                                    col[nnz] = (int32_t)((((int64_t)ncz * Ly + ncy) * Lx + ncx) * 4 + nb);
                                ++nnz;
                            }
                    row_ptr[i + 1] = nnz;
                }
    return nnz;
}

/* Structured colouring: sc (x+y+z) mod 2, bcc and fcc the basis index.
 * kind: 0 sc, 1 bcc, 2 fcc. */
void or_colour_structured(int kind, int Lx, int Ly, int Lz, int32_t *colour)
{
    int64_t i = 0;
    int nb = (kind == 0) ? 1 : (kind == 1 ? 2 : 4);
    for (int z = 0; z < Lz; ++z)
        for (int y = 0; y < Ly; ++y)
            for (int x = 0; x < Lx; ++x)
                for (int b = 0; b < nb; ++b, ++i)
                    colour[i] = (kind == 0) ? ((x + y + z) & 1) : b;
}

/* For sampled sites of an Lx x Ly x Lz sc lattice (no vacancies): the colour
 * (x + y + z) & 1 of or_colour_structured and the rank of the site among the
 * sites of its colour in ascending natural index, the count or_sweep keeps.
 * With Lx even, every pair of natural indices (2k, 2k+1) lies in one row and
 * holds one site of each colour, so the sites of either colour before site i
 * number floor(i / 2). */
void or_sc_sites_colour_rank(int Lx, int Ly, int Lz, int64_t m, const int64_t *sites, int32_t *colour, int64_t *rank)
{
    (void)Lz;
    for (int64_t t = 0; t < m; ++t) {
        const int64_t i = sites[t];
        const int x = (int)(i % Lx);
        const int y = (int)((i / Lx) % Ly);
        const int64_t z = i / ((int64_t)Lx * Ly);
        colour[t] = (int32_t)((x + y + z) & 1);
        rank[t] = i / 2;
    }
}

/* Greedy colouring: present vertices in ascending natural index each take
 * the smallest colour not held by an already-coloured present neighbour.
 * Absent vertices get colour -1.  Returns the number of colours. */
int or_colour_greedy(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *mask,
                     int32_t *colour)
{
    int n_colours = 0;
    int cap = 64;
    char *used = (char *)malloc((size_t)cap);
    for (int64_t i = 0; i < n; ++i)
        colour[i] = -1;
    for (int64_t i = 0; i < n; ++i) {
        if (mask && !mask[i])
            continue;
        int64_t deg = row_ptr[i + 1] - row_ptr[i];
        if (deg + 1 > cap) {
            cap = (int)(deg + 1);
            used = (char *)realloc(used, (size_t)cap);
        }
        memset(used, 0, (size_t)cap);
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int32_t c = colour[col[k]];
            if (c >= 0 && c < cap)
                used[c] = 1;
        }
        int c = 0;
        while (used[c])
            ++c;
        colour[i] = c;
        if (c + 1 > n_colours)
            n_colours = c + 1;
    }
    free(used);
    return n_colours;
}

/* ------------------------------------------------------------------------ */
/* Initial state: each present site gets an independent uniform point on   */
/* the sphere from one Philox call with tag INIT at sweep 0, colour 0.     */
/* Absent sites are zero.  S is n x 3, natural order.                       */
/* ------------------------------------------------------------------------ */
/* Initial spin of natural site i: a sphere point from one Philox block,
 * counter (index lo, index hi, tag 1, replica); an initial spin has no
 * sweep, so the sweep word carries the index's high half. */
static void or_init_site(uint64_t seed, uint32_t replica, uint64_t i, double s[3])
{
    uint32_t r[4];
    or_draw(seed, replica, i, i >> 32, OR_TAG_INIT, 0, 0, r);
    or_sphere_point(or_u53(r[0], r[1]), or_u53(r[2], r[3]), s);
}

void or_init_spins(int64_t n, const uint8_t *mask, uint64_t seed, uint32_t replica, double *S)
{
    for (int64_t i = 0; i < n; ++i) {
        if (mask && !mask[i]) {
            S[3 * i] = S[3 * i + 1] = S[3 * i + 2] = 0.0;
            continue;
        }
        or_init_site(seed, replica, (uint64_t)i, &S[3 * i]);
    }
}

/* The same for m sampled natural indices (no vacancies). */
void or_init_sites(int64_t m, const int64_t *sites, uint64_t seed, uint32_t replica, double *S)
{
    for (int64_t t = 0; t < m; ++t)
        or_init_site(seed, replica, (uint64_t)sites[t], &S[3 * t]);
}

/* S^T A S for the symmetric tensor A = (Axx, Ayy, Azz, Axy, Axz, Ayz):
 * the matrix-vector product A S, then its dot product with S. */
static double quad_form(const double A[6], const double s[3])
{
    double As0 = A[0] * s[0] + A[3] * s[1] + A[4] * s[2];
    double As1 = A[3] * s[0] + A[1] * s[1] + A[5] * s[2];
    double As2 = A[4] * s[0] + A[5] * s[1] + A[2] * s[2];
    return s[0] * As0 + s[1] * As1 + s[2] * As2;
}

/* Single-site energy -J S.h - K (S.e)^2 - S^T A S for a given local field h
 * (the last term only when A is given). */
static double site_energy(const double s[3], const double h[3], double J, double K, const double e[3],
                          const double *A)
{
    double sh = s[0] * h[0] + s[1] * h[1] + s[2] * h[2];
    double se = s[0] * e[0] + s[1] * e[1] + s[2] * e[2];
    double E = -J * sh - K * se * se;
    if (A)
        E -= quad_form(A, s);
    return E;
}

/* ------------------------------------------------------------------------ */
/* Metropolis steps (ii)-(iii) at one site whose local field h (the sum of  */
/* its present neighbours' spins, step (i)) is given: draw the trial from   */
/* the schedule of `mode` (see or_sweep), take dH from Eq. 1 and accept if  */
/* dH <= 0, else iff P <= exp(-beta dH).  Updates s in place on acceptance; */
/* returns 1 if accepted.  *dH_out gets dH; *in_band is 1 for a decision   */
/* with P > 0 and |beta dH + ln P| < band, on either side of dH = 0: a dH   */
/* just below zero with P just below 1 is as close to the acceptance        */
/* boundary exp(-beta dH) = P as a dH just above zero.                      */
/* ------------------------------------------------------------------------ */
int or_site_update(int mode, uint64_t seed, uint32_t replica, uint64_t site, uint64_t rank, uint64_t sweep,
                   uint32_t colour, double J, double K, const double e[3], const double *A, double beta,
                   double band, const double h[3], double s[3], double *dH_out, int *in_band)
{
    double u[3];
    or_trial_uniforms(mode, seed, replica, site, rank, sweep, colour, u);
    double trial[3];
    or_sphere_point(u[0], u[1], trial);
    if (mode == 2) {
        trial[0] = or_round_half(trial[0]);
        trial[1] = or_round_half(trial[1]);
        trial[2] = or_round_half(trial[2]);
    }
    double dH = site_energy(trial, h, J, K, e, A) - site_energy(s, h, J, K, e, A);
    double P = u[2];
    int accept;
    if (dH <= 0.0)
        accept = 1;
    else
        accept = (P <= exp(-beta * dH));
    *in_band = (band > 0.0 && P > 0.0 && fabs(beta * dH + log(P)) < band);
    if (accept) {
        s[0] = trial[0];
        s[1] = trial[1];
        s[2] = trial[2];
    }
    *dH_out = dH;
    return accept;
}

/* The same for m sampled sites at once (site t: natural index site[t],
 * rank rank[t] among the present sites of its colour colour[t], local field
 * h[3t..3t+2], spin s[3t..3t+2] updated in place); accepted[t] and
 * in_band[t] get the decisions. */
void or_sites_update(int64_t m, const int64_t *site, const int64_t *rank, const int32_t *colour, const double *h,
                     double *s, int mode, uint64_t seed, uint32_t replica, uint64_t sweep, double J, double K,
                     const double e[3], const double *A, double beta, double band, uint8_t *accepted,
                     uint8_t *in_band)
{
    for (int64_t t = 0; t < m; ++t) {
        double dH;
        int b;
        accepted[t] = (uint8_t)or_site_update(mode, seed, replica, (uint64_t)site[t], (uint64_t)rank[t], sweep,
                                              (uint32_t)colour[t], J, K, e, A, beta, band, &h[3 * t], &s[3 * t],
                                              &dH, &b);
        in_band[t] = (uint8_t)b;
    }
}

/* ------------------------------------------------------------------------ */
/* One Metropolis sweep: colour classes 0..n_colours-1 in order, present    */
/* sites of the class in ascending natural index.                           */
/*   mode 0: FP64 random-number schedule, spins kept in FP64               */
/*   mode 1: FP32 random-number schedule (a block per two same-colour      */
/*           sites), spins kept in FP64                                     */
/*   mode 2: FP32 schedule, the trial spin rounded to binary16 per          */
/*           component before dH (the stored state is the rounded one)     */
/* Outputs: returns accepted moves; *sum_dH gets the sum of accepted dH;    */
/* *n_band counts decisions with |beta dH + ln P| < band (either sign of    */
/* dH); band_site (optional, n bytes) is set to 1 at those sites.           */
/* ------------------------------------------------------------------------ */
int64_t or_sweep(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *colour,
                 int n_colours, const uint8_t *mask, double J, double K, const double e[3], const double *A,
                 double beta, uint64_t seed, uint32_t replica, uint64_t sweep, int mode, double band,
                 double *S, double *sum_dH, int64_t *n_band, uint8_t *band_site)
{
    int64_t accepted = 0;
    double dH_total = 0.0;
    int64_t bands = 0;
    for (int c = 0; c < n_colours; ++c) {
        uint64_t rank = 0; /* rank of site i among the present sites of colour c */
        for (int64_t i = 0; i < n; ++i) {
            if (colour[i] != c)
                continue;
            if (mask && !mask[i])
                continue;
            uint64_t my_rank = rank++;
            /* step (i): site i; local field from present neighbours */
            double h[3] = {0.0, 0.0, 0.0};
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                int32_t j = col[k];
                if (mask && !mask[j])
                    continue;
                h[0] += S[3 * (int64_t)j];
                h[1] += S[3 * (int64_t)j + 1];
                h[2] += S[3 * (int64_t)j + 2];
            }
            /* steps (ii)-(iii) */
            double dH;
            int in_band;
            if (or_site_update(mode, seed, replica, (uint64_t)i, my_rank, sweep, (uint32_t)c, J, K, e, A, beta,
                               band, h, &S[3 * i], &dH, &in_band)) {
                dH_total += dH;
                ++accepted;
            }
            if (in_band) {
                ++bands;
                if (band_site)
                    band_site[i] = 1;
            }
        }
    }
    if (sum_dH)
        *sum_dH = dH_total;
    if (n_band)
        *n_band = bands;
    return accepted;
}

/* ------------------------------------------------------------------------ */
/* The same sweep with the sites of one colour class shared among          */
/* n_threads OpenMP threads.  A class is an independent set: its sites     */
/* read only other classes' spins, which do not change during the class,  */
/* and every random number is keyed by the site (or by its class rank,     */
/* counted here before the class starts), so the spins, the accepted count */
/* and the band flags equal or_sweep's bit for bit whatever the thread     */
/* count; only *sum_dH is added in another order.                          */
/* ------------------------------------------------------------------------ */
int64_t or_sweep_parallel(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *colour,
                          int n_colours, const uint8_t *mask, double J, double K, const double e[3],
                          const double *A, double beta, uint64_t seed, uint32_t replica, uint64_t sweep, int mode,
                          double band, double *S, double *sum_dH, int64_t *n_band, uint8_t *band_site,
                          int n_threads)
{
    int64_t accepted = 0;
    double dH_total = 0.0;
    int64_t bands = 0;
    int64_t *rank = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!rank)
        return -1;
    if (n_threads < 1)
        n_threads = 1;
    for (int c = 0; c < n_colours; ++c) {
        int64_t count = 0;
        for (int64_t i = 0; i < n; ++i)
            rank[i] = (colour[i] == c && !(mask && !mask[i])) ? count++ : -1;
#pragma omp parallel for schedule(static) num_threads(n_threads) reduction(+ : accepted, dH_total, bands)
        for (int64_t i = 0; i < n; ++i) {
            if (rank[i] < 0)
                continue;
            double h[3] = {0.0, 0.0, 0.0};
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                int32_t j = col[k];
                if (mask && !mask[j])
                    continue;
                h[0] += S[3 * (int64_t)j];
                h[1] += S[3 * (int64_t)j + 1];
                h[2] += S[3 * (int64_t)j + 2];
            }
            double dH;
            int in_band;
            if (or_site_update(mode, seed, replica, (uint64_t)i, (uint64_t)rank[i], sweep, (uint32_t)c, J, K, e, A,
                               beta, band, h, &S[3 * i], &dH, &in_band)) {
                dH_total += dH;
                ++accepted;
            }
            if (in_band) {
                ++bands;
                if (band_site)
                    band_site[i] = 1;
            }
        }
    }
    free(rank);
    if (sum_dH)
        *sum_dH = dH_total;
    if (n_band)
        *n_band = bands;
    return accepted;
}

/* Total energy, Eq. 1, full recompute: every undirected bond once (pairs
 * listed as j > i in a symmetric neighbour list), plus the anisotropy of
 * every present site (and its tensor term when A is given). */
double or_energy(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *mask, double J,
                 double K, const double e[3], const double *A, const double *S)
{
    double exch = 0.0, anis = 0.0, tens = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (mask && !mask[i])
            continue;
        const double *si = &S[3 * i];
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t j = col[k];
            if (j <= i)
                continue;
            if (mask && !mask[j])
                continue;
            const double *sj = &S[3 * j];
            exch += si[0] * sj[0] + si[1] * sj[1] + si[2] * sj[2];
        }
        double se = si[0] * e[0] + si[1] * e[1] + si[2] * e[2];
        anis += se * se;
        if (A)
            tens += quad_form(A, si);
    }
    return -J * exch - K * anis - tens;
}

/* Sum of the present spins (numerator of Eq. 2); returns the count N. */
int64_t or_spin_sum(int64_t n, const uint8_t *mask, const double *S, double out[3])
{
    int64_t count = 0;
    out[0] = out[1] = out[2] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (mask && !mask[i])
            continue;
        out[0] += S[3 * i];
        out[1] += S[3 * i + 1];
        out[2] += S[3 * i + 2];
        ++count;
    }
    return count;
}
