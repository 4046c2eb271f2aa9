/*
 * crk_oracle.c -- plain, slow, FP64 CPU oracle for the short-range
 * particle-particle solver of CRK-HACC (arXiv 2510.03557, Sec. IV).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  The product path never
 * calls it and shares no code with it (no headers, no helpers, no tables).
 *
 * What it computes, pass by pass, for particles in a periodic cube of side L:
 *   density      rho_i = sum_{j in N_i + {i}} m_j W(r_ij, h_i)          (CRKSPH, Sec. IV-A)
 *   moments      m0, m1, m2 and their x_i-gradients (40 sums per gas particle)
 *   corrections  A, B, dA, dB of the linear reproducing kernel (3x3 inverse of m2)
 *   hydro        pairwise-antisymmetric CRKSPH momentum and energy rates with
 *                Monaghan artificial viscosity (Eq. 1-2 give the pair-sum form)
 *   gravity      short-range part of a Gaussian long/short split (Sec. IV-A)
 *   KDK          fixed-step kick-drift-kick
 * The paper cites but does not print these formulas; the readings used are:
 *   - smoothing kernel: 3-D Wendland C4 with compact support H = 2h;
 *   - neighbour predicate: r^2 < H_i^2 (strict), r^2 = (dx*dx + dy*dy) + dz*dz
 *     with dx = x_j - x_i wrapped once to [-L/2, L/2), no FMA contraction
 *     (built with -ffp-contract=off);
 *   - hydro pair set: r^2 < H_i^2 or r^2 < H_j^2; gravity set: r^2 < r_cut^2;
 *   - split: S(r) = erfc(r / 2 r_s) + r / (sqrt(pi) r_s) exp(-r^2 / 4 r_s^2);
 *   - u floored at u_floor after each kick, floor events counted;
 *   friends-of-friends groups (in situ halo finding, Sec. IV-B3): particles
 *   of the chosen species linked when r^2 < b^2 (the same predicate), groups
 *   the connected components, each labelled by its smallest index.
 * The neighbour search is a cell list of side >= the largest search radius
 * (or all pairs when the box holds fewer than three such cells); no tree,
 * no leaves, no leaf pairs.  Every per-particle sum runs in a fixed order.
 *
 * Parity pins for every function are in the oracle tests: kernel
 * normalisation by quadrature and gradient by finite differences, lattice
 * neighbour counts, the reproducing identities of the corrected kernel,
 * finite-difference derivatives of A and B, pairwise antisymmetry,
 * momentum and energy conservation, the textbook-SPH limit, and direct
 * summation minus the analytic long-range part for gravity.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_ESINGULAR -5

#define ORC_GAS 1

typedef struct {
    double L;          /* box side */
    double G;          /* gravitational constant */
    double gamma;      /* adiabatic index */
    double r_cut;      /* short-range gravity cut-off radius */
    double r_split;    /* Gaussian split scale r_s */
    double eps_soft;   /* Plummer softening length */
    double av_alpha;   /* viscosity alpha */
    double av_beta;    /* viscosity beta */
    double av_eps2;    /* viscosity epsilon^2 */
    double u_floor;    /* floor on the specific thermal energy */
    int brute;         /* 1: all-pairs search instead of the cell list */
    int nthreads;      /* 0: OpenMP default */
} orc_params;

/* ------------------------------------------------------------------ */
/* Smoothing kernel: Wendland C4 in 3-D, support H = 2h, q = r/H.       */
/*   W(r,h) = 495 / (32 pi H^3) (1-q)^6 (1 + 6q + 35q^2/3)             */
/* dW/dq = -(56/3) q (1+5q) (1-q)^5 times the same prefactor, so        */
/*   grad_i W = W'(r) x_ij / r = -(56/3) 495/(32 pi H^5) (1+5q)(1-q)^5 x_ij */
/* which is finite at r = 0 (the limit is taken analytically).          */
/* ------------------------------------------------------------------ */
static const double ORC_PI = 3.14159265358979323846;

double orc_W(double r, double h)
{
    double H = 2.0 * h;
    double q = r / H;
    if (q >= 1.0) return 0.0;
    double omq = 1.0 - q;
    double omq2 = omq * omq;
    double omq6 = omq2 * omq2 * omq2;
    double norm = 495.0 / (32.0 * ORC_PI * H * H * H);
    return norm * omq6 * (1.0 + 6.0 * q + 35.0 * q * q / 3.0);
}

/* Returns g such that grad_i W(x_ij, h) = g * x_ij. */
double orc_gradW_factor(double r, double h)
{
    double H = 2.0 * h;
    double q = r / H;
    if (q >= 1.0) return 0.0;
    double omq = 1.0 - q;
    double omq2 = omq * omq;
    double omq5 = omq2 * omq2 * omq;
    double norm = 495.0 / (32.0 * ORC_PI * H * H * H * H * H);
    return -(56.0 / 3.0) * norm * (1.0 + 5.0 * q) * omq5;
}

/* Short-range factor of the Gaussian split; the long-range part is 1 - S. */
double orc_S(double r, double r_s)
{
    double t = r / (2.0 * r_s);
    return erfc(t) + r / (sqrt(ORC_PI) * r_s) * exp(-t * t);
}

/* SplitMix64 output function (Steele, Lea & Flood 2014). */
static uint64_t orc_mix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Minimum-image component of x_j - x_i (one wrap). */
static double orc_wrap_d(double d, double L)
{
    if (d >= 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}

/* dx = x_j - x_i (minimum image), returns r^2 in the fixed order. */
static double orc_sep(const double *pos, int64_t i, int64_t j, double L, double dx[3])
{
    for (int a = 0; a < 3; ++a) dx[a] = orc_wrap_d(pos[3 * j + a] - pos[3 * i + a], L);
    return (dx[0] * dx[0] + dx[1] * dx[1]) + dx[2] * dx[2];
}

/* ------------------------------------------------------------------ */
/* Cell list                                                          */
/* ------------------------------------------------------------------ */
typedef struct {
    int nc;             /* cells per side (1 = all pairs) */
    int64_t *start;     /* nc^3 + 1 */
    int64_t *idx;       /* particle indices grouped by cell, ascending within a cell */
} orc_cells;

static int orc_cell_of(double x, double L, int nc)
{
    int c = (int)(x / L * (double)nc);
    if (c < 0) c = 0;
    if (c >= nc) c = nc - 1;
    return c;
}

/* Cells at least R (1 + 1e-9) wide: a cell index is rounded, so with cells
 * exactly R wide a pair with r just below R could land two cells apart; the
 * margin keeps every pair with r < R in neighbouring cells. */
static int orc_cells_build(orc_cells *cl, int64_t n, const double *pos, double L, double R, int brute)
{
    double Rm = R * (1.0 + 1e-9);
    int nc = (R > 0.0) ? (int)floor(L / Rm) : 1;
    while (nc > 1 && L / (double)nc < Rm) --nc;
    if (brute || nc < 3) nc = 1;
    if (nc > 1024) nc = 1024;
    int64_t ncell = (int64_t)nc * nc * nc;
    cl->nc = nc;
    cl->start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    cl->idx = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *cid = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!cl->start || !cl->idx || !cid) { free(cl->start); free(cl->idx); free(cid); return ORC_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) {
        int cx = orc_cell_of(pos[3 * i + 0], L, nc);
        int cy = orc_cell_of(pos[3 * i + 1], L, nc);
        int cz = orc_cell_of(pos[3 * i + 2], L, nc);
        cid[i] = ((int64_t)cz * nc + cy) * nc + cx;
        cl->start[cid[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) cl->start[c + 1] += cl->start[c];
    int64_t *fill = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
    if (!fill) { free(cl->start); free(cl->idx); free(cid); return ORC_ENOMEM; }
    memcpy(fill, cl->start, (size_t)ncell * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) cl->idx[fill[cid[i]]++] = i;
    free(fill);
    free(cid);
    return ORC_OK;
}

static void orc_cells_free(orc_cells *cl)
{
    free(cl->start);
    free(cl->idx);
}

/* The distinct cells around particle i: 27 when nc >= 3, else the single cell. */
static int orc_cells_around(const orc_cells *cl, const double *pos, int64_t i, double L, int64_t out[27])
{
    int nc = cl->nc;
    if (nc == 1) { out[0] = 0; return 1; }
    int cx = orc_cell_of(pos[3 * i + 0], L, nc);
    int cy = orc_cell_of(pos[3 * i + 1], L, nc);
    int cz = orc_cell_of(pos[3 * i + 2], L, nc);
    int k = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int x = (cx + dx + nc) % nc, y = (cy + dy + nc) % nc, z = (cz + dz + nc) % nc;
                out[k++] = ((int64_t)z * nc + y) * nc + x;
            }
    return k;
}

static double orc_max_H(int64_t n, const double *h, const uint8_t *species)
{
    double m = 0.0;
    for (int64_t i = 0; i < n; ++i)
        if (species[i] == ORC_GAS && 2.0 * h[i] > m) m = 2.0 * h[i];
    return m;
}

static void orc_set_threads(const orc_params *p)
{
#ifdef _OPENMP
    if (p->nthreads > 0) omp_set_num_threads(p->nthreads);
#else
    (void)p;
#endif
}

/* The neighbour predicate in FP64; dx = x_j - x_i. */
static int orc_in_gather(double r2, double hi)
{
    double H = 2.0 * hi;
    return r2 < H * H;
}

/* ------------------------------------------------------------------ */
/* Neighbour sets: count and order-independent hash of original ids    */
/* kind 0: hydro gather set  {gas j != i : r^2 < H_i^2}, gas i only     */
/* kind 1: hydro pair set    {gas j != i : r^2 < H_i^2 or r^2 < H_j^2}  */
/* kind 2: gravity set       {j != i : r^2 < r_cut^2}, every species    */
/* ------------------------------------------------------------------ */
int orc_neighbours(int64_t n, const double *pos, const double *h, const uint8_t *species,
                   const orc_params *p, int kind, int32_t *count, uint64_t *hash)
{
    if (n < 0 || kind < 0 || kind > 2) return ORC_EINVAL;
    orc_set_threads(p);
    double R = (kind == 2) ? p->r_cut : orc_max_H(n, h, species);
    orc_cells cl;
    int rc = orc_cells_build(&cl, n, pos, p->L, R, p->brute);
    if (rc) return rc;
    double rc2 = p->r_cut * p->r_cut;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        int32_t cnt = 0;
        uint64_t hs = 0;
        if (kind == 2 || species[i] == ORC_GAS) {
            int64_t cells[27];
            int nc = orc_cells_around(&cl, pos, i, p->L, cells);
            for (int c = 0; c < nc; ++c)
                for (int64_t k = cl.start[cells[c]]; k < cl.start[cells[c] + 1]; ++k) {
                    int64_t j = cl.idx[k];
                    if (j == i) continue;
                    if (kind != 2 && species[j] != ORC_GAS) continue;
                    double dx[3];
                    double r2 = orc_sep(pos, i, j, p->L, dx);
                    int in;
                    if (kind == 0) in = orc_in_gather(r2, h[i]);
                    else if (kind == 1) in = orc_in_gather(r2, h[i]) || orc_in_gather(r2, h[j]);
                    else in = r2 < rc2;
                    if (in) { cnt++; hs += orc_mix64((uint64_t)j); }
                }
        }
        count[i] = cnt;
        hash[i] = hs;
    }
    orc_cells_free(&cl);
    return ORC_OK;
}

/* Adds to mask_out every gas particle in the hydro pair set of a masked gas
 * particle (and the masked particles themselves).  Used to evaluate a sample
 * of outputs without computing the whole box. */
int orc_expand_mask(int64_t n, const double *pos, const double *h, const uint8_t *species,
                    const orc_params *p, const uint8_t *mask_in, uint8_t *mask_out)
{
    orc_set_threads(p);
    double R = orc_max_H(n, h, species);
    orc_cells cl;
    int rc = orc_cells_build(&cl, n, pos, p->L, R, p->brute);
    if (rc) return rc;
    for (int64_t i = 0; i < n; ++i) mask_out[i] = mask_in[i];
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        if (!mask_in[i] || species[i] != ORC_GAS) continue;
        int64_t cells[27];
        int nc = orc_cells_around(&cl, pos, i, p->L, cells);
        for (int c = 0; c < nc; ++c)
            for (int64_t k = cl.start[cells[c]]; k < cl.start[cells[c] + 1]; ++k) {
                int64_t j = cl.idx[k];
                if (species[j] != ORC_GAS) continue;
                double dx[3];
                double r2 = orc_sep(pos, i, j, p->L, dx);
                if (orc_in_gather(r2, h[i]) || orc_in_gather(r2, h[j])) mask_out[j] = 1;
            }
    }
    orc_cells_free(&cl);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Density pass: rho_i = sum over j in N_i plus i itself of m_j W(r, h_i) */
/* V = m / rho, P = (gamma - 1) rho u, c = sqrt(gamma (gamma - 1) u)    */
/* ------------------------------------------------------------------ */
int orc_density(int64_t n, const double *pos, const double *mass, const double *u,
                const double *h, const uint8_t *species, const orc_params *p,
                const uint8_t *mask, double *rho, double *V, double *P, double *c)
{
    orc_set_threads(p);
    orc_cells cl;
    int rc = orc_cells_build(&cl, n, pos, p->L, orc_max_H(n, h, species), p->brute);
    if (rc) return rc;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        if (species[i] != ORC_GAS || (mask && !mask[i])) continue;
        double sum = 0.0;
        int64_t cells[27];
        int nc = orc_cells_around(&cl, pos, i, p->L, cells);
        for (int cc = 0; cc < nc; ++cc)
            for (int64_t k = cl.start[cells[cc]]; k < cl.start[cells[cc] + 1]; ++k) {
                int64_t j = cl.idx[k];
                if (species[j] != ORC_GAS) continue;
                double dx[3];
                double r2 = orc_sep(pos, i, j, p->L, dx);
                if (j != i && !orc_in_gather(r2, h[i])) continue;
                sum += mass[j] * orc_W(sqrt(r2), h[i]);
            }
        rho[i] = sum;
        V[i] = mass[i] / sum;
        P[i] = (p->gamma - 1.0) * sum * u[i];
        c[i] = sqrt(p->gamma * (p->gamma - 1.0) * u[i]);
    }
    orc_cells_free(&cl);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Moments (sums over j in N_i plus i, W_ij = W(r, h_i), x_ij = x_i - x_j, */
/* d_g = d/dx_i^g):                                                    */
/*   m0 = sum V_j W_ij          m1^a = sum V_j x^a W_ij                 */
/*   m2^ab = sum V_j x^a x^b W_ij                                       */
/*   d_g m0 = sum V_j d_gW_ij   d_g m1^a = sum V_j (x^a d_gW + delta_ag W) */
/*   d_g m2^ab = sum V_j (x^a x^b d_gW + (delta_ag x^b + delta_bg x^a) W) */
/* Layout of the 40 values per particle:                               */
/*   [0] m0, [1..3] m1^a, [4..9] m2 (xx xy xz yy yz zz), [10..12] d_g m0, */
/*   [13..21] d_g m1^a at 13 + 3a + g, [22..39] d_g m2^ab at 22 + 3s + g  */
/*   with s the packed (ab) index above.                              */
/* ------------------------------------------------------------------ */
static const int ORC_SYM_A[6] = {0, 0, 0, 1, 1, 2};
static const int ORC_SYM_B[6] = {0, 1, 2, 1, 2, 2};

int orc_moments(int64_t n, const double *pos, const double *V, const double *h,
                const uint8_t *species, const orc_params *p, const uint8_t *mask, double *mom)
{
    orc_set_threads(p);
    orc_cells cl;
    int rc = orc_cells_build(&cl, n, pos, p->L, orc_max_H(n, h, species), p->brute);
    if (rc) return rc;
#pragma omp parallel for schedule(dynamic, 128)
    for (int64_t i = 0; i < n; ++i) {
        if (species[i] != ORC_GAS || (mask && !mask[i])) continue;
        double m[40];
        for (int t = 0; t < 40; ++t) m[t] = 0.0;
        int64_t cells[27];
        int nc = orc_cells_around(&cl, pos, i, p->L, cells);
        for (int cc = 0; cc < nc; ++cc)
            for (int64_t k = cl.start[cells[cc]]; k < cl.start[cells[cc] + 1]; ++k) {
                int64_t j = cl.idx[k];
                if (species[j] != ORC_GAS) continue;
                double dx[3];
                double r2 = orc_sep(pos, i, j, p->L, dx);
                if (j != i && !orc_in_gather(r2, h[i])) continue;
                double r = sqrt(r2);
                double x[3] = {-dx[0], -dx[1], -dx[2]};
                double W = orc_W(r, h[i]);
                double gf = orc_gradW_factor(r, h[i]);
                double dW[3] = {gf * x[0], gf * x[1], gf * x[2]};
                double Vj = V[j];
                m[0] += Vj * W;
                for (int a = 0; a < 3; ++a) m[1 + a] += Vj * x[a] * W;
                for (int s = 0; s < 6; ++s) m[4 + s] += Vj * x[ORC_SYM_A[s]] * x[ORC_SYM_B[s]] * W;
                for (int g = 0; g < 3; ++g) m[10 + g] += Vj * dW[g];
                for (int a = 0; a < 3; ++a)
                    for (int g = 0; g < 3; ++g)
                        m[13 + 3 * a + g] += Vj * (x[a] * dW[g] + (a == g ? W : 0.0));
                for (int s = 0; s < 6; ++s) {
                    int a = ORC_SYM_A[s], b = ORC_SYM_B[s];
                    for (int g = 0; g < 3; ++g)
                        m[22 + 3 * s + g] += Vj * (x[a] * x[b] * dW[g] +
                                                   ((a == g ? x[b] : 0.0) + (b == g ? x[a] : 0.0)) * W);
                }
            }
        for (int t = 0; t < 40; ++t) mom[40 * i + t] = m[t];
    }
    orc_cells_free(&cl);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Corrections (per particle, FP64):                                   */
/*   M = m2^{-1} (explicit cofactor inverse), singular if              */
/*       |det m2| < 1e-30 ||m2||_F^3                                    */
/*   A = 1 / (m0 - m1^T M m1),  B = -M m1                               */
/*   d_g M = -M (d_g m2) M,  d_g B = -M (d_g m1) - (d_g M) m1            */
/*   d_g A = -A^2 (d_g m0 + 2 B . d_g m1 + B^T (d_g m2) B)              */
/* Outputs: A[i], B[3i+a], dA[3i+g], dB[9i + 3a + g] = d_g B^a.         */
/* ------------------------------------------------------------------ */
static void orc_unpack_sym(const double *s6, double M[3][3])
{
    for (int s = 0; s < 6; ++s) {
        M[ORC_SYM_A[s]][ORC_SYM_B[s]] = s6[s];
        M[ORC_SYM_B[s]][ORC_SYM_A[s]] = s6[s];
    }
}

int orc_corrections(int64_t n, const double *mom, const uint8_t *species, const uint8_t *mask,
                    double *A, double *B, double *dA, double *dB, int64_t *bad)
{
    int64_t first_bad = -1;
    for (int64_t i = 0; i < n; ++i) {
        if (species[i] != ORC_GAS || (mask && !mask[i])) continue;
        const double *m = mom + 40 * i;
        double m2[3][3];
        orc_unpack_sym(m + 4, m2);
        double c00 = m2[1][1] * m2[2][2] - m2[1][2] * m2[2][1];
        double c01 = m2[1][2] * m2[2][0] - m2[1][0] * m2[2][2];
        double c02 = m2[1][0] * m2[2][1] - m2[1][1] * m2[2][0];
        double det = m2[0][0] * c00 + m2[0][1] * c01 + m2[0][2] * c02;
        double fro = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) fro += m2[a][b] * m2[a][b];
        fro = sqrt(fro);
        if (!(fabs(det) >= 1e-30 * fro * fro * fro) || fro == 0.0) {
            if (first_bad < 0) first_bad = i;
            A[i] = 0.0;
            for (int a = 0; a < 3; ++a) { B[3 * i + a] = 0.0; dA[3 * i + a] = 0.0; }
            for (int t = 0; t < 9; ++t) dB[9 * i + t] = 0.0;
            continue;
        }
        /* cofactor inverse: M[a][b] = cof[b][a] / det */
        double cof[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                int a1 = (a + 1) % 3, a2 = (a + 2) % 3, b1 = (b + 1) % 3, b2 = (b + 2) % 3;
                cof[a][b] = m2[a1][b1] * m2[a2][b2] - m2[a1][b2] * m2[a2][b1];
            }
        double M[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) M[a][b] = cof[b][a] / det;
        const double m0 = m[0];
        const double m1[3] = {m[1], m[2], m[3]};
        double Mm1[3];
        for (int a = 0; a < 3; ++a) Mm1[a] = M[a][0] * m1[0] + M[a][1] * m1[1] + M[a][2] * m1[2];
        double m1Mm1 = m1[0] * Mm1[0] + m1[1] * Mm1[1] + m1[2] * Mm1[2];
        double Ai = 1.0 / (m0 - m1Mm1);
        double Bi[3] = {-Mm1[0], -Mm1[1], -Mm1[2]};
        A[i] = Ai;
        for (int a = 0; a < 3; ++a) B[3 * i + a] = Bi[a];
        for (int g = 0; g < 3; ++g) {
            double dm0 = m[10 + g];
            double dm1[3], dm2[3][3], dm2s[6];
            for (int a = 0; a < 3; ++a) dm1[a] = m[13 + 3 * a + g];
            for (int s = 0; s < 6; ++s) dm2s[s] = m[22 + 3 * s + g];
            orc_unpack_sym(dm2s, dm2);
            /* dM = -M dm2 M */
            double T[3][3], dM[3][3];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    T[a][b] = dm2[a][0] * M[0][b] + dm2[a][1] * M[1][b] + dm2[a][2] * M[2][b];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    dM[a][b] = -(M[a][0] * T[0][b] + M[a][1] * T[1][b] + M[a][2] * T[2][b]);
            /* dB = -M dm1 - dM m1 */
            for (int a = 0; a < 3; ++a) {
                double v = 0.0;
                for (int b = 0; b < 3; ++b) v += -M[a][b] * dm1[b] - dM[a][b] * m1[b];
                dB[9 * i + 3 * a + g] = v;
            }
            /* dA = -A^2 (dm0 + 2 B.dm1 + B^T dm2 B) */
            double Bdm1 = Bi[0] * dm1[0] + Bi[1] * dm1[1] + Bi[2] * dm1[2];
            double BdmB = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) BdmB += Bi[a] * dm2[a][b] * Bi[b];
            dA[3 * i + g] = -Ai * Ai * (dm0 + 2.0 * Bdm1 + BdmB);
        }
    }
    if (bad) *bad = first_bad;
    return first_bad >= 0 ? ORC_ESINGULAR : ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Corrected kernel gradient of particle i evaluated at separation x   */
/* (x = x_i - x_other), with i's smoothing length and corrections:      */
/*   d_g W^R = A (1 + B.x) d_gW + d_gA (1 + B.x) W + A (d_gB . x + B^g) W */
/* ------------------------------------------------------------------ */
static void orc_corrected_grad(const double x[3], double r, double hi, double Ai,
                               const double *Bi, const double *dAi, const double *dBi,
                               double out[3], double *WR)
{
    double W = orc_W(r, hi);
    double gf = orc_gradW_factor(r, hi);
    double lin = 1.0 + Bi[0] * x[0] + Bi[1] * x[1] + Bi[2] * x[2];
    for (int g = 0; g < 3; ++g) {
        double dBx = dBi[0 * 3 + g] * x[0] + dBi[1 * 3 + g] * x[1] + dBi[2 * 3 + g] * x[2];
        out[g] = Ai * lin * gf * x[g] + dAi[g] * lin * W + Ai * (dBx + Bi[g]) * W;
    }
    if (WR) *WR = Ai * lin * W;
}

/* Monaghan viscous pressure for one side: eta = x / h, v = v_self - v_other */
static double orc_visc_Q(const double x[3], const double v[3], double hs, double rho, double c,
                         const orc_params *p)
{
    double eta[3] = {x[0] / hs, x[1] / hs, x[2] / hs};
    double ve = v[0] * eta[0] + v[1] * eta[1] + v[2] * eta[2];
    double ee = eta[0] * eta[0] + eta[1] * eta[1] + eta[2] * eta[2];
    double mu = ve / (ee + p->av_eps2);
    if (mu > 0.0) mu = 0.0;
    return rho * (-p->av_alpha * c * mu + p->av_beta * mu * mu);
}

/* Hydro pair force F_ij (force on i from j), x_ij = x_i - x_j:
 *   F_ij = -1/2 V_i V_j (P_i + P_j + Q_i + Q_j) (dW^R_ij - dW^R_ji)
 * with dW^R_ji j's corrected gradient at x_ji = -x_ij using h_j. */
static void orc_hydro_pair_force(int64_t i, int64_t j, const double xij[3], double r,
                                 const double *vel, const double *h, const double *rho,
                                 const double *V, const double *P, const double *c,
                                 const double *A, const double *B, const double *dA,
                                 const double *dB, const orc_params *p, double F[3])
{
    double xji[3] = {-xij[0], -xij[1], -xij[2]};
    double vij[3] = {vel[3 * i] - vel[3 * j], vel[3 * i + 1] - vel[3 * j + 1], vel[3 * i + 2] - vel[3 * j + 2]};
    double vji[3] = {-vij[0], -vij[1], -vij[2]};
    double gi[3], gj[3];
    orc_corrected_grad(xij, r, h[i], A[i], B + 3 * i, dA + 3 * i, dB + 9 * i, gi, NULL);
    orc_corrected_grad(xji, r, h[j], A[j], B + 3 * j, dA + 3 * j, dB + 9 * j, gj, NULL);
    double Qi = orc_visc_Q(xij, vij, h[i], rho[i], c[i], p);
    double Qj = orc_visc_Q(xji, vji, h[j], rho[j], c[j], p);
    double pre = -0.5 * V[i] * V[j] * (P[i] + P[j] + Qi + Qj);
    for (int g = 0; g < 3; ++g) F[g] = pre * (gi[g] - gj[g]);
}

/* ------------------------------------------------------------------ */
/* Hydro rates: m_i a_i = sum_j F_ij,  m_i du_i = -1/2 sum_j F_ij.(v_i - v_j) */
/* over the hydro pair set (j != i).  vel holds the velocities that enter  */
/* the viscosity (the KDK predictor).  acc and dudt are overwritten for    */
/* gas particles in the mask.                                           */
/* ------------------------------------------------------------------ */
int orc_hydro(int64_t n, const double *pos, const double *vel, const double *mass,
              const double *h, const uint8_t *species, const double *rho, const double *V,
              const double *P, const double *c, const double *A, const double *B,
              const double *dA, const double *dB, const orc_params *p, const uint8_t *mask,
              double *acc, double *dudt)
{
    orc_set_threads(p);
    orc_cells cl;
    int rc = orc_cells_build(&cl, n, pos, p->L, orc_max_H(n, h, species), p->brute);
    if (rc) return rc;
#pragma omp parallel for schedule(dynamic, 128)
    for (int64_t i = 0; i < n; ++i) {
        if (species[i] != ORC_GAS || (mask && !mask[i])) continue;
        double a[3] = {0.0, 0.0, 0.0}, du = 0.0;
        int64_t cells[27];
        int nc = orc_cells_around(&cl, pos, i, p->L, cells);
        for (int cc = 0; cc < nc; ++cc)
            for (int64_t k = cl.start[cells[cc]]; k < cl.start[cells[cc] + 1]; ++k) {
                int64_t j = cl.idx[k];
                if (j == i || species[j] != ORC_GAS) continue;
                double dx[3];
                double r2 = orc_sep(pos, i, j, p->L, dx);
                if (!(orc_in_gather(r2, h[i]) || orc_in_gather(r2, h[j]))) continue;
                double xij[3] = {-dx[0], -dx[1], -dx[2]};
                double F[3];
                orc_hydro_pair_force(i, j, xij, sqrt(r2), vel, h, rho, V, P, c, A, B, dA, dB, p, F);
                double vij[3] = {vel[3 * i] - vel[3 * j], vel[3 * i + 1] - vel[3 * j + 1],
                                 vel[3 * i + 2] - vel[3 * j + 2]};
                for (int g = 0; g < 3; ++g) a[g] += F[g];
                du += -0.5 * (F[0] * vij[0] + F[1] * vij[1] + F[2] * vij[2]);
            }
        for (int g = 0; g < 3; ++g) acc[3 * i + g] = a[g] / mass[i];
        dudt[i] = du / mass[i];
    }
    orc_cells_free(&cl);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Short-range gravity: a_i = sum_{j != i, r < r_cut} F_ij / m_i with    */
/*   F_ij = -G m_i m_j x_ij (r^2 + eps^2)^{-3/2} S(r)                    */
/* over every species pair.  acc is overwritten for masked particles.   */
/* ------------------------------------------------------------------ */
int orc_gravity(int64_t n, const double *pos, const double *mass, const uint8_t *species,
                const orc_params *p, const uint8_t *mask, double *acc)
{
    (void)species;
    orc_set_threads(p);
    orc_cells cl;
    int rc = orc_cells_build(&cl, n, pos, p->L, p->r_cut, p->brute);
    if (rc) return rc;
    double rc2 = p->r_cut * p->r_cut;
    double e2 = p->eps_soft * p->eps_soft;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        if (mask && !mask[i]) continue;
        double a[3] = {0.0, 0.0, 0.0};
        int64_t cells[27];
        int nc = orc_cells_around(&cl, pos, i, p->L, cells);
        for (int cc = 0; cc < nc; ++cc)
            for (int64_t k = cl.start[cells[cc]]; k < cl.start[cells[cc] + 1]; ++k) {
                int64_t j = cl.idx[k];
                if (j == i) continue;
                double dx[3];
                double r2 = orc_sep(pos, i, j, p->L, dx);
                if (!(r2 < rc2)) continue;
                double r = sqrt(r2);
                double s2 = r2 + e2;
                double f = -p->G * mass[j] * orc_S(r, p->r_split) / (s2 * sqrt(s2));
                for (int g = 0; g < 3; ++g) a[g] += f * (-dx[g]);
            }
        for (int g = 0; g < 3; ++g) acc[3 * i + g] = a[g];
    }
    orc_cells_free(&cl);
    return ORC_OK;
}

/* Hydro and gravity pair forces of one pair (i, j), force on i. */
int orc_pair_forces(int64_t n, const double *pos, const double *vel, const double *mass,
                    const double *h, const uint8_t *species, const double *rho, const double *V,
                    const double *P, const double *c, const double *A, const double *B,
                    const double *dA, const double *dB, const orc_params *p, int64_t i, int64_t j,
                    double *F_hydro, double *F_grav)
{
    if (i < 0 || j < 0 || i >= n || j >= n || i == j) return ORC_EINVAL;
    double dx[3];
    double r2 = orc_sep(pos, i, j, p->L, dx);
    double r = sqrt(r2);
    double xij[3] = {-dx[0], -dx[1], -dx[2]};
    for (int g = 0; g < 3; ++g) { F_hydro[g] = 0.0; F_grav[g] = 0.0; }
    if (species[i] == ORC_GAS && species[j] == ORC_GAS &&
        (orc_in_gather(r2, h[i]) || orc_in_gather(r2, h[j])))
        orc_hydro_pair_force(i, j, xij, r, vel, h, rho, V, P, c, A, B, dA, dB, p, F_hydro);
    if (r2 < p->r_cut * p->r_cut) {
        double s2 = r2 + p->eps_soft * p->eps_soft;
        double f = -p->G * mass[i] * mass[j] * orc_S(r, p->r_split) / (s2 * sqrt(s2));
        for (int g = 0; g < 3; ++g) F_grav[g] = f * xij[g];
    }
    return ORC_OK;
}

/* Reproducing-kernel diagnostics per gas particle i (sums over j in N_i + {i}):
 *   out[16i + 0]          = sum V_j W^R_ij                       (should be 1)
 *   out[16i + 1 + a]      = sum V_j x_ij^a W^R_ij                (should be 0)
 *   out[16i + 4 + g]      = sum V_j d_g W^R_ij                   (should be 0)
 *   out[16i + 7 + 3b + g] = sum V_j x_ij^b d_g W^R_ij            (should be -delta_bg) */
int orc_crk_identities(int64_t n, const double *pos, const double *V, const double *h,
                       const uint8_t *species, const double *A, const double *B,
                       const double *dA, const double *dB, const orc_params *p,
                       const uint8_t *mask, double *out)
{
    orc_set_threads(p);
    orc_cells cl;
    int rc = orc_cells_build(&cl, n, pos, p->L, orc_max_H(n, h, species), p->brute);
    if (rc) return rc;
#pragma omp parallel for schedule(dynamic, 128)
    for (int64_t i = 0; i < n; ++i) {
        if (species[i] != ORC_GAS || (mask && !mask[i])) continue;
        double s[16];
        for (int t = 0; t < 16; ++t) s[t] = 0.0;
        int64_t cells[27];
        int nc = orc_cells_around(&cl, pos, i, p->L, cells);
        for (int cc = 0; cc < nc; ++cc)
            for (int64_t k = cl.start[cells[cc]]; k < cl.start[cells[cc] + 1]; ++k) {
                int64_t j = cl.idx[k];
                if (species[j] != ORC_GAS) continue;
                double dx[3];
                double r2 = orc_sep(pos, i, j, p->L, dx);
                if (j != i && !orc_in_gather(r2, h[i])) continue;
                double x[3] = {-dx[0], -dx[1], -dx[2]};
                double g[3], WR;
                orc_corrected_grad(x, sqrt(r2), h[i], A[i], B + 3 * i, dA + 3 * i, dB + 9 * i, g, &WR);
                s[0] += V[j] * WR;
                for (int a = 0; a < 3; ++a) s[1 + a] += V[j] * x[a] * WR;
                for (int q = 0; q < 3; ++q) s[4 + q] += V[j] * g[q];
                for (int b = 0; b < 3; ++b)
                    for (int q = 0; q < 3; ++q) s[7 + 3 * b + q] += V[j] * x[b] * g[q];
            }
        for (int t = 0; t < 16; ++t) out[16 * i + t] = s[t];
    }
    orc_cells_free(&cl);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* All passes: density, moments, corrections, hydro, gravity.          */
/* vel / u are the values that enter the force (KDK predictor).        */
/* acc = hydro + gravity; gas outputs rho, V, P, c, A, B, dA, dB, dudt; */
/* DM rows of the gas-only outputs are zero.  mask (optional) restricts */
/* the outputs to masked particles; the caller expands the mask so that */
/* every quantity a masked output needs is computed.                   */
/* ------------------------------------------------------------------ */
int orc_forces(int64_t n, const double *pos, const double *vel, const double *mass,
               const double *u, const double *h, const uint8_t *species, const orc_params *p,
               const uint8_t *mask_hydro, const uint8_t *mask_moments, const uint8_t *mask_density,
               double *acc, double *dudt, double *rho, double *V, double *P, double *c,
               double *mom, double *A, double *B, double *dA, double *dB, int64_t *bad)
{
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *ag = (double *)calloc(3 * nn, sizeof(double));
    if (!ag) return ORC_ENOMEM;
    memset(acc, 0, 3 * nn * sizeof(double));
    memset(dudt, 0, nn * sizeof(double));
    memset(rho, 0, nn * sizeof(double));
    memset(V, 0, nn * sizeof(double));
    memset(P, 0, nn * sizeof(double));
    memset(c, 0, nn * sizeof(double));
    memset(mom, 0, 40 * nn * sizeof(double));
    memset(A, 0, nn * sizeof(double));
    memset(B, 0, 3 * nn * sizeof(double));
    memset(dA, 0, 3 * nn * sizeof(double));
    memset(dB, 0, 9 * nn * sizeof(double));
    int rc = orc_density(n, pos, mass, u, h, species, p, mask_density, rho, V, P, c);
    if (!rc) rc = orc_moments(n, pos, V, h, species, p, mask_moments, mom);
    if (!rc) rc = orc_corrections(n, mom, species, mask_moments, A, B, dA, dB, bad);
    if (!rc) rc = orc_hydro(n, pos, vel, mass, h, species, rho, V, P, c, A, B, dA, dB, p,
                            mask_hydro, acc, dudt);
    if (!rc) rc = orc_gravity(n, pos, mass, species, p, mask_hydro, ag);
    if (!rc)
        for (int64_t i = 0; i < 3 * n; ++i) acc[i] += ag[i];
    free(ag);
    return rc;
}

/* Position wrap into [0, L) after a drift; a value that rounds up to L maps to 0. */
static double orc_wrap_pos(double x, double L)
{
    if (x >= L) x -= L;
    if (x < 0.0) {
        x += L;
        if (x >= L) x = 0.0;
    }
    return x;
}

/* ------------------------------------------------------------------ */
/* Fixed-step kick-drift-kick, nsteps steps:                            */
/*   v_half = v + dt/2 a;  u_half = u + dt/2 du   (gas u floored)         */
/*   x <- wrap(x + dt v_half)                                            */
/*   predictor v^ = v_half + dt/2 a_old, u^ = u_half + dt/2 du_old (floored) */
/*   forces at (x, v^, u^) -> a, du                                      */
/*   v = v_half + dt/2 a;  u = u_half + dt/2 du   (gas u floored)         */
/* If have_forces is 0, acc/dudt are first evaluated at (x, v, u).      */
/* Returns the number of floor events in *nfloor.                      */
/* ------------------------------------------------------------------ */
static void orc_floor_u(int64_t n, const uint8_t *species, double *u, double fl, int64_t *nfloor)
{
    for (int64_t i = 0; i < n; ++i)
        if (species[i] == ORC_GAS && u[i] < fl) { u[i] = fl; (*nfloor)++; }
}

int orc_kdk(int64_t n, double *pos, double *vel, const double *mass, double *u, const double *h,
            const uint8_t *species, const orc_params *p, double dt, int nsteps,
            double *acc, double *dudt, int have_forces, int64_t *nfloor)
{
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *rho = malloc(nn * sizeof(double)), *V = malloc(nn * sizeof(double));
    double *P = malloc(nn * sizeof(double)), *c = malloc(nn * sizeof(double));
    double *mom = malloc(40 * nn * sizeof(double)), *A = malloc(nn * sizeof(double));
    double *B = malloc(3 * nn * sizeof(double)), *dA = malloc(3 * nn * sizeof(double));
    double *dB = malloc(9 * nn * sizeof(double));
    double *vp = malloc(3 * nn * sizeof(double)), *up = malloc(nn * sizeof(double));
    int rc = ORC_OK;
    int64_t bad = -1, floors = 0;
    if (!rho || !V || !P || !c || !mom || !A || !B || !dA || !dB || !vp || !up) { rc = ORC_ENOMEM; goto done; }
    if (!have_forces) {
        rc = orc_forces(n, pos, vel, mass, u, h, species, p, NULL, NULL, NULL, acc, dudt, rho, V, P, c,
                        mom, A, B, dA, dB, &bad);
        if (rc) goto done;
    }
    double hdt = 0.5 * dt;
    for (int s = 0; s < nsteps; ++s) {
        for (int64_t i = 0; i < 3 * n; ++i) vel[i] = vel[i] + hdt * acc[i];
        for (int64_t i = 0; i < n; ++i) u[i] = u[i] + hdt * dudt[i];
        orc_floor_u(n, species, u, p->u_floor, &floors);
        for (int64_t i = 0; i < 3 * n; ++i) pos[i] = orc_wrap_pos(pos[i] + dt * vel[i], p->L);
        for (int64_t i = 0; i < 3 * n; ++i) vp[i] = vel[i] + hdt * acc[i];
        for (int64_t i = 0; i < n; ++i) up[i] = u[i] + hdt * dudt[i];
        orc_floor_u(n, species, up, p->u_floor, &floors);
        rc = orc_forces(n, pos, vp, mass, up, h, species, p, NULL, NULL, NULL, acc, dudt, rho, V, P, c,
                        mom, A, B, dA, dB, &bad);
        if (rc) goto done;
        for (int64_t i = 0; i < 3 * n; ++i) vel[i] = vel[i] + hdt * acc[i];
        for (int64_t i = 0; i < n; ++i) u[i] = u[i] + hdt * dudt[i];
        orc_floor_u(n, species, u, p->u_floor, &floors);
    }
done:
    if (nfloor) *nfloor = floors;
    free(rho); free(V); free(P); free(c); free(mom); free(A); free(B); free(dA); free(dB);
    free(vp); free(up);
    return rc;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Friends-of-friends groups (in situ halo finding, Sec. IV-B3)        */
/* ------------------------------------------------------------------ */
/* Root of x with path halving. */
static int64_t orc_find(int64_t *par, int64_t x)
{
    while (par[x] != x) {
        par[x] = par[par[x]];
        x = par[x];
    }
    return x;
}

/* Particles whose species bit is set in species_mask (bit 0: CRK_DM, bit 1:
 * CRK_GAS) are linked when r^2 < b^2, r^2 formed as for every neighbour set;
 * groups are the connected components of the links.  group[i] = the smallest
 * index in i's group, -1 for particles of the other species; *ngroups counts
 * the groups, singletons included.  Sequential union-find over a cell list;
 * unions always hang the larger root under the smaller, so a root is the
 * smallest index of its tree. */
int orc_fof(int64_t n, const double *pos, const uint8_t *species, double L, double b, int species_mask,
            int64_t *group, int64_t *ngroups)
{
    if (!(b > 0.0) || !(b < 0.5 * L)) return ORC_EINVAL;
    int64_t *par = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!par) return ORC_ENOMEM;
    for (int64_t i = 0; i < n; ++i) par[i] = i;
    orc_cells cl;
    int rc = orc_cells_build(&cl, n, pos, L, b, 0);
    if (rc) { free(par); return rc; }
    const double b2 = b * b;
    for (int64_t i = 0; i < n; ++i) {
        if (!((species_mask >> species[i]) & 1)) continue;
        int64_t cells[27];
        int nci = orc_cells_around(&cl, pos, i, L, cells);
        for (int c = 0; c < nci; ++c)
            for (int64_t q = cl.start[cells[c]]; q < cl.start[cells[c] + 1]; ++q) {
                int64_t j = cl.idx[q];
                if (j <= i || !((species_mask >> species[j]) & 1)) continue;
                double dx[3];
                if (!(orc_sep(pos, i, j, L, dx) < b2)) continue;
                int64_t ri = orc_find(par, i), rj = orc_find(par, j);
                if (ri == rj) continue;
                if (ri < rj) par[rj] = ri;
                else par[ri] = rj;
            }
    }
    int64_t ng = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!((species_mask >> species[i]) & 1)) {
            group[i] = -1;
            continue;
        }
        group[i] = orc_find(par, i);
        if (group[i] == i) ++ng;
    }
    *ngroups = ng;
    orc_cells_free(&cl);
    free(par);
    return ORC_OK;
}
