/*
 * oracle.c -- plain FP64 CPU oracle for the Velocity Jumps (JUMP) MD path.
 *
 * TEST INFRASTRUCTURE: see oracle.h. Slow on purpose: every nonbonded sum is a
 * brute-force loop over all pairs with the minimum image, every list is built
 * by testing every pair, and each algorithm runs in the order the paper gives.
 *
 * Sources (Gouraud, Lagardere, Adjoua, Ple, Monmarche, Piquemal, "Velocity
 * Jumps for Molecular Dynamics", arXiv 2412.15073):
 *   Sec. 2.1  Langevin SDE and the split grad U = sum_i F_i
 *   Sec. 2.2  jump rate (MRZ form), jump kernel, density f_eta, BPS limit
 *   Sec. 2.3  splittings BAOAB-like BJAOAJB, CAOAC, C'J'AOAJ'C', RESPA, RESPA1
 *   Sec. 2.4  Poisson thinning, Algorithms 1-3, rejection sampling of G~
 *   Sec. 3.1  pair jumps for direct electrostatics, Algorithm 4, ring technique
 *   Sec. 3.2  Lennard-Jones BPS jumps, Algorithm 5
 * Readings where the paper is silent:
 *   electrostatics: damped shifted force (DSF) Coulomb in place of Ewald;
 *   switch chi: quintic smoothstep on [r_c-h, r_c];
 *   rate bounds: numerical max of |d/dr (1-chi)U| on a grid, rounded up;
 *   acceptance p = lambda / bar-lambda_Y, with the sqrt(beta) that Algorithm 4 omits;
 *   adaptive eps: eps = eps0 |g| in the rate, bound and kernel;
 *   the jump partner J is drawn before eta is formed.
 */
#include "oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- physical constants (kcal/mol, A, ps, amu, e) ---------------------- */
#define OR_KB        0.0019872042586      /* Boltzmann constant, kcal/mol/K   */
#define OR_COULOMB   332.0637             /* kcal A / (mol e^2)               */
#define OR_KCAL_AMU  418.4                /* 1 kcal/mol = 418.4 amu A^2/ps^2  */
#define OR_PI        3.14159265358979323846
#define OR_KMAX      (1 << 20)            /* proposal cap per atom and phase  */
#define OR_SAMPLER_CAP 64                 /* attempt cap of the G~ sampler    */

/* Philox counter tags (word 2, bits 24..31) */
#define TAG_O 1u
#define TAG_C 2u
#define TAG_J 3u
#define TAG_S 4u

enum { W_FULL = 0, W_SHORT = 1, W_LONG = 2 };
#define OR_MAX_RINGS 4
enum { K_LJ = 4, K_NKIND = 5 };            /* kinds 0..3: rings, 4: LJ partners */

typedef struct { int *off, *idx; int cap; } or_list;

struct or_sys {
    int n;
    or_params p;
    double L;
    double *x, *v, *xb;      /* positions (wrapped), velocities, positions at last list build */
    int *img;
    double *m, *mt, *q;      /* mass (amu), reduced mass m/418.4, charge */
    int *type;
    int ntypes;
    double *eps, *sig;       /* ntypes x ntypes */
    int nb, na;
    int *bonds; double *bk, *br0;
    int *angles; double *ak, *at0;
    int *exoff, *exidx;      /* per-atom excluded partners */
    /* derived */
    double beta;
    int nr;                              /* number of rings */
    double edge[OR_MAX_RINGS + 1];       /* ring edges: r_c - h, ..., r_E */
    double lhat[OR_MAX_RINGS], qmax;
    double *LY, *LLJ;                    /* per-atom rate bounds (n x 4), LJ bound */
    or_list lists[K_NKIND];
    int lazy;                /* lists built per atom on demand (see or_params.lazy_lists) */
    int alist_atom;          /* atom whose lists the per-atom cache holds (-1: none) */
    int* alist[K_NKIND];     /* that atom's lists */
    int alist_n[K_NKIND];
    int ncell;
    int *cellm;              /* cell of each atom at the last outer rebuild */
    double *xo;              /* positions at the last outer rebuild */
    /* forces (as accelerations a = -grad/m~) */
    double *a0, *ab, *as, *al;
    int64_t step;
    int64_t cnt[OR_NCOUNTERS];
    uint32_t err;
    /* event log */
    int64_t ev_cap, ev_n;
    int64_t *ev;
    /* velocity record for spectra: v after each innermost step */
    int64_t vr_cap, vr_n;
    double* vr;
};

/* store v as the state after the innermost step that just ended (up to vr_cap samples) */
static void vrec(or_sys* s)
{
    if (s->vr && s->vr_n < s->vr_cap)
        memcpy(s->vr + 3 * (size_t)s->n * (size_t)s->vr_n, s->v, sizeof(double) * 3 * (size_t)s->n);
    if (s->vr) s->vr_n++;
}

/* ======================================================================== */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two     */
/* 32x32->64 multiplications, key bumped by the Weyl constants between     */
/* rounds.                                                                  */
/* ======================================================================== */
void or_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* draw of one Philox block in the stream of (atom, s, tag, half, attempt, k) */
static void draw(const or_sys* s, uint32_t atom, uint32_t s0, uint32_t tag, int half,
                 uint32_t attempt, uint32_t k, uint32_t* u)
{
    uint32_t ctr[4] = { atom, s0, (tag << 24) | ((uint32_t)half << 20) | (attempt << 8), k };
    uint32_t key[2] = { s->p.seed, s->p.replica };
    or_philox(ctr, key, u);
}

/* uniform on (0,1) from 32 random bits: (b + 1/2) 2^-32 */
static double unif(uint32_t b) { return ((double)b + 0.5) * (1.0 / 4294967296.0); }

/* uniform index in [0, n) from 32 random bits: floor(b n / 2^32) */
static int pick(uint32_t b, int n) { return (int)(((uint64_t)b * (uint64_t)n) >> 32); }

/* ======================================================================== */
/* Normal law and Theta(eta) = E[(eta+G)_+] (Sec. 2.2, below the rate).     */
/* Closed form: eta Phi(eta) + phi(eta).                                    */
/* ======================================================================== */
static double nphi(double y) { return exp(-0.5 * y * y) / sqrt(2.0 * OR_PI); }
static double nPhi(double y) { return 0.5 * erfc(-y / sqrt(2.0)); }

double or_theta(double eta)
{
    double t = eta * nPhi(eta) + nphi(eta);
    return t > 0.0 ? t : 0.0;
}

/* ======================================================================== */
/* G~ with density f_eta(y) = (eta+y)_+ exp(-y^2/2) / (Theta(eta) sqrt(2pi)) */
/* by rejection (Sec. 2.4, the four proposal families by eta). With         */
/* z = eta + y > 0 the target is proportional to z exp(-z^2/2 + eta z).     */
/*   eta > 0        : proposal  eta phi(y) + y_+ phi-like Rayleigh mixture, */
/*                    ratio (eta+y)_+ / (eta + y_+)                          */
/*   -1 <= eta <= 0 : z ~ Rayleigh(1), ratio exp(eta z)                     */
/*   -2.5 <= eta < -1: z ~ Exp(|eta|), ratio z exp((1 - z^2)/2)             */
/*   eta < -2.5     : z ~ Gamma(2, |eta|), ratio exp(-z^2/2)                */
/* ======================================================================== */
static double gtilde_draw(double eta, const uint32_t u[4], int* ok)
{
    *ok = 0;
    if (eta > 0.0) {
        double y;
        double pg = eta / (eta + 1.0 / sqrt(2.0 * OR_PI));
        if (unif(u[0]) < pg)
            y = sqrt(-2.0 * log(unif(u[1]))) * cos(2.0 * OR_PI * unif(u[2]));
        else
            y = sqrt(-2.0 * log(unif(u[1])));
        if (y >= 0.0) { *ok = 1; return y; }
        double r = (eta + y) > 0.0 ? (eta + y) / eta : 0.0;
        if (unif(u[3]) <= r) { *ok = 1; return y; }
        return 0.0;
    } else if (eta >= -1.0) {
        double z = sqrt(-2.0 * log(unif(u[0])));
        if (unif(u[1]) <= exp(eta * z)) { *ok = 1; return z - eta; }
        return 0.0;
    } else if (eta >= -2.5) {
        double z = -log(unif(u[0])) / (-eta);
        if (unif(u[1]) <= z * exp(0.5 * (1.0 - z * z))) { *ok = 1; return z - eta; }
        return 0.0;
    } else {
        double z = -(log(unif(u[0])) + log(unif(u[1]))) / (-eta);
        if (unif(u[2]) <= exp(-0.5 * z * z)) { *ok = 1; return z - eta; }
        return 0.0;
    }
}

static double gtilde(const or_sys* s, double eta, uint32_t atom, uint32_t s0, int half,
                     uint32_t k, int* attempts, int* fail)
{
    *fail = 0;
    for (int a = 0; a < OR_SAMPLER_CAP; ++a) {
        uint32_t u[4];
        int ok;
        draw(s, atom, s0, TAG_S, half, (uint32_t)a, k, u);
        double y = gtilde_draw(eta, u, &ok);
        if (ok) { *attempts = a + 1; return y; }
    }
    *attempts = OR_SAMPLER_CAP;
    *fail = 1;
    return 0.0;
}

double or_sample_gtilde(double eta, uint32_t seed, uint32_t replica, uint32_t atom,
                        uint32_t s0, int half, uint32_t k, int* attempts)
{
    or_sys tmp;
    memset(&tmp, 0, sizeof tmp);
    tmp.p.seed = seed;
    tmp.p.replica = replica;
    int fail;
    double y = gtilde(&tmp, eta, atom, s0, half, k, attempts, &fail);
    if (fail) *attempts = -1;
    return y;
}

/* ======================================================================== */
/* Pair potentials.                                                         */
/* chi: quintic switch, 1 on r <= r_c-h, 0 on r >= r_c (Sec. 3.1, the split */
/*      U_ij = chi U_ij + (1-chi) U_ij).                                    */
/* DSF Coulomb (Fennell-Gezelter 2006), cut and shifted in value and slope  */
/*      at R = r_E.                                                         */
/* LJ 4 eps [(s/r)^12 - (s/r)^6], shifted in value and slope at R = r_E.    */
/* ======================================================================== */
static double chi(const or_sys* s, double r)
{
    double lo = s->p.r_split - s->p.h_switch;
    if (r <= lo) return 1.0;
    if (r >= s->p.r_split) return 0.0;
    double t = (r - lo) / s->p.h_switch;
    return 1.0 - t * t * t * (10.0 - 15.0 * t + 6.0 * t * t);
}

static double dchi(const or_sys* s, double r)
{
    double lo = s->p.r_split - s->p.h_switch;
    if (r <= lo || r >= s->p.r_split) return 0.0;
    double t = (r - lo) / s->p.h_switch;
    return -30.0 * t * t * (1.0 - t) * (1.0 - t) / s->p.h_switch;
}

static double u_dsf(const or_sys* s, double r)
{
    double a = s->p.dsf_alpha, R = s->p.r_cut;
    if (r >= R) return 0.0;
    double eR = erfc(a * R) / R;
    double fR = erfc(a * R) / (R * R) + 2.0 * a / sqrt(OR_PI) * exp(-a * a * R * R) / R;
    return erfc(a * r) / r - eR + fR * (r - R);
}

static double du_dsf(const or_sys* s, double r)
{
    double a = s->p.dsf_alpha, R = s->p.r_cut;
    if (r >= R) return 0.0;
    double fR = erfc(a * R) / (R * R) + 2.0 * a / sqrt(OR_PI) * exp(-a * a * R * R) / R;
    double fr = erfc(a * r) / (r * r) + 2.0 * a / sqrt(OR_PI) * exp(-a * a * r * r) / r;
    return -fr + fR;
}

/* real-space Coulomb per unit C q_i q_j: DSF, or the Ewald erfc(alpha r)/r,
 * both zero from r_cut on */
static double u_coul(const or_sys* s, double r)
{
    if (s->p.coulomb_mode == 1) return r < s->p.r_cut ? erfc(s->p.dsf_alpha * r) / r : 0.0;
    return u_dsf(s, r);
}

static double du_coul(const or_sys* s, double r)
{
    if (s->p.coulomb_mode == 1) {
        if (r >= s->p.r_cut) return 0.0;
        double a = s->p.dsf_alpha;
        return -(erfc(a * r) / r + 2.0 * a / sqrt(OR_PI) * exp(-a * a * r * r)) / r;
    }
    return du_dsf(s, r);
}

static double u_lj(double e, double sg, double r)
{
    double s6 = pow(sg / r, 6.0);
    return 4.0 * e * (s6 * s6 - s6);
}

static double du_lj(double e, double sg, double r)
{
    double s6 = pow(sg / r, 6.0);
    return 4.0 * e * (-12.0 * s6 * s6 + 6.0 * s6) / r;
}

static double u_ljsf(const or_sys* s, double e, double sg, double r)
{
    double R = s->p.r_cut;
    if (r >= R || e == 0.0) return 0.0;
    return u_lj(e, sg, r) - u_lj(e, sg, R) - (r - R) * du_lj(e, sg, R);
}

static double du_ljsf(const or_sys* s, double e, double sg, double r)
{
    double R = s->p.r_cut;
    if (r >= R || e == 0.0) return 0.0;
    return du_lj(e, sg, r) - du_lj(e, sg, R);
}

/* weighted radial derivative d/dr [w(r) U(r)] = w' U + w U' */
static double wdudr(const or_sys* s, double u, double du, double r, int weight)
{
    if (weight == W_FULL) return du;
    if (weight == W_SHORT) return dchi(s, r) * u + chi(s, r) * du;
    return -dchi(s, r) * u + (1.0 - chi(s, r)) * du;
}

static double wu(const or_sys* s, double u, double r, int weight)
{
    if (weight == W_FULL) return u;
    if (weight == W_SHORT) return chi(s, r) * u;
    return (1.0 - chi(s, r)) * u;
}

double or_pair_dudr(const or_sys* s, int ti, int tj, double qiqj, double r, int weight)
{
    double e = s->eps[ti * s->ntypes + tj], sg = s->sig[ti * s->ntypes + tj];
    double u = OR_COULOMB * qiqj * u_coul(s, r) + u_ljsf(s, e, sg, r);
    double du = OR_COULOMB * qiqj * du_coul(s, r) + du_ljsf(s, e, sg, r);
    return wdudr(s, u, du, r, weight);
}

double or_pair_u(const or_sys* s, int ti, int tj, double qiqj, double r, int weight)
{
    double e = s->eps[ti * s->ntypes + tj], sg = s->sig[ti * s->ntypes + tj];
    double u = OR_COULOMB * qiqj * u_coul(s, r) + u_ljsf(s, e, sg, r);
    return wu(s, u, r, weight);
}

/* radial derivative of the long-range Coulomb part (1-chi) U_DSF per unit
 * C q_i q_j (the part handled by the C' jumps) */
static double coul_long_dudr(const or_sys* s, double r)
{
    return -dchi(s, r) * u_coul(s, r) + (1.0 - chi(s, r)) * du_coul(s, r);
}

/* radial derivative of the long-range LJ part (1-chi) U_LJ (J' jumps) */
static double lj_long_dudr(const or_sys* s, double e, double sg, double r)
{
    return -dchi(s, r) * u_ljsf(s, e, sg, r) + (1.0 - chi(s, r)) * du_ljsf(s, e, sg, r);
}

/* ======================================================================== */
/* geometry                                                                 */
/* ======================================================================== */
static void minimage(const or_sys* s, int i, int j, double* d)
{
    for (int c = 0; c < 3; ++c) {
        double t = s->x[3 * i + c] - s->x[3 * j + c];
        d[c] = t - s->L * nearbyint(t / s->L);
    }
}

static int excluded(const or_sys* s, int i, int j)
{
    for (int e = s->exoff[i]; e < s->exoff[i + 1]; ++e)
        if (s->exidx[e] == j) return 1;
    return 0;
}

/* ======================================================================== */
/* bounds on |F_ij| (Sec. 3.1: analytic bounds uniform in j; ring technique */
/* bounds L_M on [r_c-h, r_M] and L_L on [r_M, r_E], generalised to rings   */
/* with edges r_c-h = e_0 < e_1 < ... < e_n = r_E). Reading: grid max,      */
/* times (1 + 1e-4), rounded up to 9 significant bits.                      */
/* ======================================================================== */
static double round_up_bound(double x)
{
    if (!(x > 0.0)) return 0.0;
    int e;
    double f = frexp(x * (1.0 + 1e-4), &e);   /* f in [0.5, 1) */
    f = ceil(f * 512.0) / 512.0;
    return ldexp(f, e);
}

#define OR_NGRID 20001

static double grid_max_coul(const or_sys* s, double lo, double hi)
{
    double m = 0.0;
    if (!(hi > lo)) return 0.0;
    for (int k = 0; k < OR_NGRID; ++k) {
        double r = lo + (hi - lo) * (double)k / (double)(OR_NGRID - 1);
        double f = fabs(coul_long_dudr(s, r));
        if (f > m) m = f;
    }
    return m;
}

static double grid_max_lj(const or_sys* s, double e, double sg, double lo, double hi)
{
    double m = 0.0;
    if (!(hi > lo) || e == 0.0) return 0.0;
    for (int k = 0; k < OR_NGRID; ++k) {
        double r = lo + (hi - lo) * (double)k / (double)(OR_NGRID - 1);
        double f = fabs(lj_long_dudr(s, e, sg, r));
        if (f > m) m = f;
    }
    return m;
}

static void compute_bounds(or_sys* s)
{
    double lo = s->p.r_split - s->p.h_switch, R = s->p.r_cut;
    /* ring edges */
    s->edge[0] = lo;
    if (s->p.n_rings >= 1) {
        s->nr = s->p.n_rings > OR_MAX_RINGS ? OR_MAX_RINGS : s->p.n_rings;
        for (int y = 1; y < s->nr; ++y) s->edge[y] = s->p.ring_r[y - 1];
    } else {
        s->nr = (s->p.r_mid > lo && s->p.r_mid < R) ? 2 : 1;
        if (s->nr == 2) s->edge[1] = s->p.r_mid;
    }
    s->edge[s->nr] = R;
    for (int y = 0; y < s->nr; ++y) s->lhat[y] = grid_max_coul(s, s->edge[y], s->edge[y + 1]);
    for (int y = s->nr; y < OR_MAX_RINGS; ++y) s->lhat[y] = 0.0;
    s->qmax = 0.0;
    for (int i = 0; i < s->n; ++i) if (fabs(s->q[i]) > s->qmax) s->qmax = fabs(s->q[i]);
    int nt = s->ntypes;
    double* ljhat = (double*)calloc((size_t)nt * nt, sizeof(double));
    int* present = (int*)calloc((size_t)nt, sizeof(int));
    for (int i = 0; i < s->n; ++i) present[s->type[i]] = 1;
    for (int a = 0; a < nt; ++a)
        for (int b = 0; b < nt; ++b)
            ljhat[a * nt + b] = grid_max_lj(s, s->eps[a * nt + b], s->sig[a * nt + b], lo, R);
    for (int i = 0; i < s->n; ++i) {
        double cq = OR_COULOMB * fabs(s->q[i]) * s->qmax;
        for (int y = 0; y < OR_MAX_RINGS; ++y)
            s->LY[OR_MAX_RINGS * i + y] = y < s->nr ? round_up_bound(cq * s->lhat[y]) : 0.0;
        double m = 0.0;
        for (int b = 0; b < nt; ++b)
            if (present[b] && ljhat[s->type[i] * nt + b] > m) m = ljhat[s->type[i] * nt + b];
        s->LLJ[i] = round_up_bound(m);
    }
    free(ljhat);
    free(present);
}

void or_bounds(const or_sys* s, double* lhat, double* qmax, double* edges, int* nrings, double* LY, double* LLJ)
{
    if (lhat) for (int y = 0; y < OR_MAX_RINGS; ++y) lhat[y] = s->lhat[y];
    if (qmax) *qmax = s->qmax;
    if (edges) for (int y = 0; y <= OR_MAX_RINGS; ++y) edges[y] = y <= s->nr ? s->edge[y] : 0.0;
    if (nrings) *nrings = s->nr;
    for (int i = 0; i < s->n; ++i) {
        if (LY) for (int y = 0; y < OR_MAX_RINGS; ++y) LY[OR_MAX_RINGS * i + y] = s->LY[OR_MAX_RINGS * i + y];
        if (LLJ) LLJ[i] = s->LLJ[i];
    }
}
/* ======================================================================== */
/* jump lists (Sec. 3.1 remark: middle and long neighbour lists with counts */
/* N_M(i), N_L(i), one list per ring; Sec. 3.2: LJ partners). Membership by */
/* distance at the    */
/* build positions widened by the skin. Order: by (cell of j at the last    */
/* outer rebuild, j) on the grid of n_c = floor(2 L / (r_E + skin_outer))   */
/* cells per edge. An outer rebuild happens when some atom moved more than  */
/* (skin_outer - skin)/2 since the last one; it only refreshes the cells    */
/* that order the lists.                                                    */
/* ======================================================================== */
static int cell_of(const or_sys* s, int j)
{
    int nc = s->ncell;
    double cs = s->L / (double)nc;
    int c[3];
    for (int d = 0; d < 3; ++d) {
        int t = (int)floor(s->x[3 * j + d] / cs);
        if (t < 0) t = 0;
        if (t >= nc) t = nc - 1;
        c[d] = t;
    }
    return (c[2] * nc + c[1]) * nc + c[0];
}

typedef struct { int cell, j; } cj_t;
static int cmp_cj(const void* a, const void* b)
{
    const cj_t* x = (const cj_t*)a;
    const cj_t* y = (const cj_t*)b;
    if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
    return x->j < y->j ? -1 : (x->j > y->j);
}

static int in_kind(const or_sys* s, int kind, int i, int j, double r2)
{
    double lo, hi;
    double sk = s->p.skin, sw = s->p.r_split - s->p.h_switch, R = s->p.r_cut;
    if (kind < OR_MAX_RINGS) {
        if (kind >= s->nr || sw >= R || s->q[i] * s->q[j] == 0.0) return 0;
        lo = s->edge[kind] - sk; hi = s->edge[kind + 1] + sk;
    } else {
        if (sw >= R || s->eps[s->type[i] * s->ntypes + s->type[j]] == 0.0) return 0;
        lo = sw - sk; hi = R + sk;
    }
    if (lo < 0.0) lo = 0.0;
    return r2 >= lo * lo && r2 < hi * hi;
}

typedef struct { cj_t* e; int n, cap; } cj_vec;
static void cj_push(cj_vec* v, int cell, int j)
{
    if (v->n == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 64;
        v->e = (cj_t*)realloc(v->e, sizeof(cj_t) * (size_t)v->cap);
    }
    v->e[v->n].cell = cell;
    v->e[v->n].j = j;
    v->n++;
}

/* the lists of atom i: a brute-force pass over all j, then the (cell, j) order */
static void atom_lists(const or_sys* s, int i, cj_vec* out)
{
    const int* cell = s->cellm;
    double hi = s->p.r_cut + s->p.skin;
    for (int j = 0; j < s->n; ++j) {
        if (j == i) continue;
        double d[3];
        minimage(s, i, j, d);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (r2 >= hi * hi || excluded(s, i, j)) continue;
        for (int kind = 0; kind < K_NKIND; ++kind)
            if (in_kind(s, kind, i, j, r2)) cj_push(&out[kind], cell[j], j);
    }
    for (int kind = 0; kind < K_NKIND; ++kind) qsort(out[kind].e, (size_t)out[kind].n, sizeof(cj_t), cmp_cj);
}

/* list `kind` of atom i: from the lists of all atoms, or built for atom i
 * alone in lazy mode (one atom cached at a time; not for parallel callers) */
static const int* list_of(or_sys* s, int kind, int i, int* n)
{
    if (!s->lazy) {
        const or_list* l = &s->lists[kind];
        *n = l->off[i + 1] - l->off[i];
        return l->idx + l->off[i];
    }
    if (s->alist_atom != i) {
        cj_vec tmp[K_NKIND];
        memset(tmp, 0, sizeof tmp);
        atom_lists(s, i, tmp);
        for (int k = 0; k < K_NKIND; ++k) {
            free(s->alist[k]);
            s->alist[k] = (int*)malloc(sizeof(int) * (size_t)(tmp[k].n > 0 ? tmp[k].n : 1));
            for (int t = 0; t < tmp[k].n; ++t) s->alist[k][t] = tmp[k].e[t].j;
            s->alist_n[k] = tmp[k].n;
            free(tmp[k].e);
        }
        s->alist_atom = i;
    }
    *n = s->alist_n[kind];
    return s->alist[kind];
}

/* one brute-force pass over all pairs fills the jump lists of every atom */
static void build_lists(or_sys* s)
{
    int n = s->n;
    cj_vec* tmp = (cj_vec*)calloc((size_t)n * K_NKIND, sizeof(cj_vec));
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) atom_lists(s, i, &tmp[(size_t)i * K_NKIND]);
    for (int kind = 0; kind < K_NKIND; ++kind) {
        or_list* l = &s->lists[kind];
        free(l->off);
        free(l->idx);
        l->off = (int*)malloc(sizeof(int) * (size_t)(n + 1));
        l->off[0] = 0;
        for (int i = 0; i < n; ++i) l->off[i + 1] = l->off[i] + tmp[(size_t)i * K_NKIND + kind].n;
        l->idx = (int*)malloc(sizeof(int) * (size_t)(l->off[n] > 0 ? l->off[n] : 1));
        for (int i = 0; i < n; ++i) {
            cj_vec* v = &tmp[(size_t)i * K_NKIND + kind];
            for (int k = 0; k < v->n; ++k) l->idx[l->off[i] + k] = v->e[k].j;
        }
    }
    for (size_t t = 0; t < (size_t)n * K_NKIND; ++t) free(tmp[t].e);
    free(tmp);
    memcpy(s->xb, s->x, sizeof(double) * 3 * (size_t)n);
    s->cnt[5]++;
}

static void outer_rebuild(or_sys* s)
{
    for (int j = 0; j < s->n; ++j) s->cellm[j] = cell_of(s, j);
    memcpy(s->xo, s->x, sizeof(double) * 3 * (size_t)s->n);
}

static double max_disp2(const or_sys* s, const double* ref)
{
    double m = 0.0;
    for (int i = 0; i < s->n; ++i) {
        double d2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            double t = s->x[3 * i + c] - ref[3 * i + c];
            t -= s->L * nearbyint(t / s->L);
            d2 += t * t;
        }
        if (d2 > m) m = d2;
    }
    return m;
}

void or_rebuild(or_sys* s) { outer_rebuild(s); build_lists(s); }

/* before each nonbonded evaluation: outer rebuild when some atom moved more
 * than (skin_outer - skin)/2 since the last outer rebuild, list rebuild when
 * some atom moved more than skin/2 since the last list build */
static void maybe_rebuild(or_sys* s)
{
    double lo = 0.5 * (s->p.skin_outer - s->p.skin), li = 0.5 * s->p.skin;
    if (max_disp2(s, s->xo) > lo * lo) {
        outer_rebuild(s);
        build_lists(s);
    } else if (max_disp2(s, s->xb) > li * li) {
        build_lists(s);
    }
}

void or_list_counts(or_sys* s, int kind, int* counts)
{
    for (int i = 0; i < s->n; ++i) list_of(s, kind, i, &counts[i]);
}

int or_list_get(or_sys* s, int kind, int i, int* out)
{
    int c;
    const int* l = list_of(s, kind, i, &c);
    for (int k = 0; k < c; ++k) out[k] = l[k];
    return c;
}

/* ======================================================================== */
/* forces                                                                   */
/* ======================================================================== */
static void bonded_gradient(const or_sys* s, double* g, double* eb, double* ea)
{
    double ebond = 0.0, eang = 0.0;
    for (int b = 0; b < s->nb; ++b) {
        int i = s->bonds[2 * b], j = s->bonds[2 * b + 1];
        double d[3];
        minimage(s, i, j, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double dr = r - s->br0[b];
        ebond += 0.5 * s->bk[b] * dr * dr;
        double f = r > 0.0 ? s->bk[b] * dr / r : 0.0;
        for (int c = 0; c < 3; ++c) { g[3 * i + c] += f * d[c]; g[3 * j + c] -= f * d[c]; }
    }
    for (int t = 0; t < s->na; ++t) {
        int i = s->angles[3 * t], j = s->angles[3 * t + 1], k = s->angles[3 * t + 2];
        double a[3], b[3];
        minimage(s, i, j, a);
        minimage(s, k, j, b);
        double ra = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        double rb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
        double cth = (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) / (ra * rb);
        if (cth > 1.0) cth = 1.0;
        if (cth < -1.0) cth = -1.0;
        double th = acos(cth);
        double sth = sin(th);
        double dth = th - s->at0[t];
        eang += 0.5 * s->ak[t] * dth * dth;
        if (sth < 1e-12) continue;
        double pre = s->ak[t] * dth;
        for (int c = 0; c < 3; ++c) {
            /* d theta / d a = (cos th a/|a| - b/|b|) / (|a| sin th) */
            double ga = (cth * a[c] / ra - b[c] / rb) / (ra * sth);
            double gb = (cth * b[c] / rb - a[c] / ra) / (rb * sth);
            g[3 * i + c] += pre * ga;
            g[3 * k + c] += pre * gb;
            g[3 * j + c] -= pre * (ga + gb);
        }
    }
    if (eb) *eb = ebond;
    if (ea) *ea = eang;
}

/* nonbonded gradient on atom i, brute force over all j */
static void nonbonded_atom(const or_sys* s, int i, int weight, double* g3, double* e_lj, double* e_c)
{
    double gx = 0, gy = 0, gz = 0, elj = 0, ec = 0;
    double R2 = s->p.r_cut * s->p.r_cut;
    for (int j = 0; j < s->n; ++j) {
        if (j == i) continue;
        double d[3];
        minimage(s, i, j, d);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (r2 >= R2 || excluded(s, i, j)) continue;
        double r = sqrt(r2);
        int ti = s->type[i], tj = s->type[j];
        double e = s->eps[ti * s->ntypes + tj], sg = s->sig[ti * s->ntypes + tj];
        double uc = OR_COULOMB * s->q[i] * s->q[j] * u_coul(s, r);
        double duc = OR_COULOMB * s->q[i] * s->q[j] * du_coul(s, r);
        double ul = u_ljsf(s, e, sg, r), dul = du_ljsf(s, e, sg, r);
        double f;
        if (s->p.lj_long_mode == 1 && weight != W_FULL) {
            /* LJ wholly deterministic: all of it in the short part, none in the long */
            double flj = weight == W_SHORT ? dul : 0.0;
            f = (wdudr(s, uc, duc, r, weight) + flj) / r;
            elj += weight == W_SHORT ? ul : 0.0;
        } else {
            f = wdudr(s, uc + ul, duc + dul, r, weight) / r;
            elj += wu(s, ul, r, weight);
        }
        gx += f * d[0]; gy += f * d[1]; gz += f * d[2];
        ec += wu(s, uc, r, weight);
    }
    g3[0] = gx; g3[1] = gy; g3[2] = gz;
    if (e_lj) *e_lj = elj;
    if (e_c) *e_c = ec;
}


/* the (1 - chi) LJ gradient of atom i, pair by pair (lj_long_mode 2: the LJ
 * long part deterministic at the slow level of the multiple-time-step schemes) */
static void lj_long_atom(const or_sys* s, int i, double* g3)
{
    double R2 = s->p.r_cut * s->p.r_cut;
    for (int j = 0; j < s->n; ++j) {
        if (j == i) continue;
        double d[3];
        minimage(s, i, j, d);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (r2 >= R2 || excluded(s, i, j)) continue;
        double r = sqrt(r2);
        int ti = s->type[i], tj = s->type[j];
        double e = s->eps[ti * s->ntypes + tj], sg = s->sig[ti * s->ntypes + tj];
        double f = wdudr(s, u_ljsf(s, e, sg, r), du_ljsf(s, e, sg, r), r, W_LONG) / r;
        for (int c = 0; c < 3; ++c) g3[c] += f * d[c];
    }
}

/* ======================================================================== */
/* Ewald electrostatics (coulomb_mode 1). The real-space pairs erfc(a r)/r  */
/* are split by chi like any pair term (Sec. 3.1); the rest is smooth and  */
/* deterministic: the reciprocal sum, the self term -C a/sqrt(pi) sum q^2, */
/* and, for excluded pairs (which the reciprocal sum still couples), the   */
/* correction -C q_i q_j erf(a r)/r.                                        */
/* ======================================================================== */
static void ewald_excl_self(const or_sys* s, double* grad, double* energy)
{
    double a = s->p.dsf_alpha, e = 0.0;
    for (int i = 0; i < s->n; ++i) {
        e -= OR_COULOMB * a / sqrt(OR_PI) * s->q[i] * s->q[i];
        for (int k = s->exoff[i]; k < s->exoff[i + 1]; ++k) {
            int j = s->exidx[k];
            double d[3];
            minimage(s, i, j, d);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double qq = OR_COULOMB * s->q[i] * s->q[j];
            if (j > i) e -= qq * erf(a * r) / r;
            /* d/dr [-erf(a r)/r] = erf(a r)/r^2 - (2a/sqrt(pi)) exp(-a^2 r^2)/r */
            double dudr = qq * (erf(a * r) / (r * r) - 2.0 * a / sqrt(OR_PI) * exp(-a * a * r * r) / r);
            if (grad)
                for (int c = 0; c < 3; ++c) grad[3 * i + c] += dudr * d[c] / r;
        }
    }
    if (energy) *energy += e;
}

void or_ewald_recip_plain(const or_sys* s, int kmax, double* grad, double* energy)
{
    int n = s->n;
    double L = s->L, V = L * L * L, a = s->p.dsf_alpha, e = 0.0;
    if (grad) memset(grad, 0, sizeof(double) * 3 * (size_t)n);
    double* cs = (double*)malloc(sizeof(double) * (size_t)n);
    double* sn = (double*)malloc(sizeof(double) * (size_t)n);
    for (int n1 = -kmax; n1 <= kmax; ++n1)
        for (int n2 = -kmax; n2 <= kmax; ++n2)
            for (int n3 = -kmax; n3 <= kmax; ++n3) {
                if (n1 * n1 + n2 * n2 + n3 * n3 > kmax * kmax || (n1 == 0 && n2 == 0 && n3 == 0)) continue;
                double m[3] = { n1 / L, n2 / L, n3 / L };
                double m2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
                double w = exp(-OR_PI * OR_PI * m2 / (a * a)) / m2;
                /* S(m) = sum_j q_j exp(2 pi i m.x_j) */
                double Sr = 0.0, Si = 0.0;
                for (int j = 0; j < n; ++j) {
                    double th = 2.0 * OR_PI * (m[0] * s->x[3 * j] + m[1] * s->x[3 * j + 1] + m[2] * s->x[3 * j + 2]);
                    cs[j] = cos(th);
                    sn[j] = sin(th);
                    Sr += s->q[j] * cs[j];
                    Si += s->q[j] * sn[j];
                }
                e += OR_COULOMB / (2.0 * OR_PI * V) * w * (Sr * Sr + Si * Si);
                if (grad)
                    for (int j = 0; j < n; ++j) {
                        /* d|S|^2/dx_j = -4 pi q_j m (Sr sin - Si cos) */
                        double f = -OR_COULOMB / (2.0 * OR_PI * V) * w * 4.0 * OR_PI * s->q[j] * (Sr * sn[j] - Si * cs[j]);
                        for (int c = 0; c < 3; ++c) grad[3 * j + c] += f * m[c];
                    }
            }
    free(cs);
    free(sn);
    if (energy) *energy = e;
    ewald_excl_self(s, grad, energy);
}

/* smooth PME: the cardinal B-spline M_p and its derivative */
static double bspline(int p, double u)
{
    if (u <= 0.0 || u >= p) return 0.0;
    if (p == 2) return 1.0 - fabs(u - 1.0);
    return (u * bspline(p - 1, u) + (p - u) * bspline(p - 1, u - 1.0)) / (p - 1);
}

static double dbspline(int p, double u) { return bspline(p - 1, u) - bspline(p - 1, u - 1.0); }

/* grid points per edge: the smallest 2,3,5-smooth integer >= L / spacing (at least 2 p) */
static int pme_grid(double L, double spacing, int p)
{
    int K = (int)ceil(L / spacing);
    if (K < 2 * p) K = 2 * p;
    for (;; ++K) {
        int m = K;
        while (m % 2 == 0) m /= 2;
        while (m % 3 == 0) m /= 3;
        while (m % 5 == 0) m /= 5;
        if (m == 1) return K;
    }
}

/* one pass of a separable DFT along an axis of a K^3 complex grid:
 * out(m) = sum_k in(k) exp(sign 2 pi i m k / K) */
static void dft_axis(double* re, double* im, int K, int axis, int sign)
{
    double* tr = (double*)malloc(sizeof(double) * (size_t)K);
    double* ti = (double*)malloc(sizeof(double) * (size_t)K);
    size_t stride = axis == 0 ? 1 : (axis == 1 ? (size_t)K : (size_t)K * K);
    for (int a = 0; a < K; ++a)
        for (int b = 0; b < K; ++b) {
            size_t base = axis == 0 ? ((size_t)a * K + b) * K : (axis == 1 ? (size_t)a * K * K + b : (size_t)a * K + b);
            for (int m = 0; m < K; ++m) {
                double sr = 0.0, si = 0.0;
                for (int k = 0; k < K; ++k) {
                    double th = sign * 2.0 * OR_PI * (double)((long)m * k % K) / K;
                    double c = cos(th), sv = sin(th);
                    double xr = re[base + k * stride], xi = im[base + k * stride];
                    sr += xr * c - xi * sv;
                    si += xr * sv + xi * c;
                }
                tr[m] = sr;
                ti[m] = si;
            }
            for (int m = 0; m < K; ++m) { re[base + m * stride] = tr[m]; im[base + m * stride] = ti[m]; }
        }
    free(tr);
    free(ti);
}

void or_ewald_recip_pme(const or_sys* s, double* grad, double* energy, int* Kout)
{
    int n = s->n, p = s->p.pme_order;
    double L = s->L, V = L * L * L, a = s->p.dsf_alpha;
    int K = pme_grid(L, s->p.pme_spacing, p);
    if (Kout) *Kout = K;
    size_t G = (size_t)K * K * K;
    double* Q = (double*)calloc(G, sizeof(double));
    double* im = (double*)calloc(G, sizeof(double));
    /* charges spread with M_p: point k gets q M_p(u - k) for k = floor(u) - t, t = 0..p-1 */
    for (int i = 0; i < n; ++i) {
        double u[3];
        int k0[3];
        for (int c = 0; c < 3; ++c) {
            double x = s->x[3 * i + c] - L * floor(s->x[3 * i + c] / L);
            u[c] = K * x / L;
            k0[c] = (int)floor(u[c]);
        }
        for (int t0 = 0; t0 < p; ++t0)
            for (int t1 = 0; t1 < p; ++t1)
                for (int t2 = 0; t2 < p; ++t2) {
                    int k[3] = { k0[0] - t0, k0[1] - t1, k0[2] - t2 };
                    double w = s->q[i];
                    int t[3] = { t0, t1, t2 };
                    for (int c = 0; c < 3; ++c) {
                        w *= bspline(p, u[c] - k0[c] + t[c]);
                        k[c] = ((k[c] % K) + K) % K;
                    }
                    Q[((size_t)k[2] * K + k[1]) * K + k[0]] += w;
                }
    }
    /* F(Q)(m) = sum_k Q(k) exp(-2 pi i m.k / K) */
    double* re = (double*)malloc(sizeof(double) * G);
    memcpy(re, Q, sizeof(double) * G);
    for (int ax = 0; ax < 3; ++ax) dft_axis(re, im, K, ax, -1);
    /* E = 1/2 sum_m G(m) |F(Q)(m)|^2, G = (C / (pi V)) exp(-pi^2 m^2 / a^2) / m^2 B(m) */
    double* bmod = (double*)malloc(sizeof(double) * (size_t)K);
    for (int m = 0; m < K; ++m) {
        double sr = 0.0, si = 0.0;
        for (int k = 0; k <= p - 2; ++k) {
            double th = 2.0 * OR_PI * (double)m * k / K;
            sr += bspline(p, k + 1.0) * cos(th);
            si += bspline(p, k + 1.0) * sin(th);
        }
        double d2 = sr * sr + si * si;
        bmod[m] = d2 > 1e-300 ? 1.0 / d2 : 0.0;
    }
    double e = 0.0;
    for (int m2 = 0; m2 < K; ++m2)
        for (int m1 = 0; m1 < K; ++m1)
            for (int m0 = 0; m0 < K; ++m0) {
                size_t g = ((size_t)m2 * K + m1) * K + m0;
                int mm[3] = { m0, m1, m2 };
                double msq = 0.0;
                for (int c = 0; c < 3; ++c) {
                    double mc = (mm[c] <= K / 2 ? mm[c] : mm[c] - K) / L;
                    msq += mc * mc;
                }
                double Gm = 0.0;
                if (msq > 0.0)
                    Gm = OR_COULOMB / (OR_PI * V) * exp(-OR_PI * OR_PI * msq / (a * a)) / msq * bmod[m0] * bmod[m1] * bmod[m2];
                e += 0.5 * Gm * (re[g] * re[g] + im[g] * im[g]);
                re[g] *= Gm;
                im[g] *= Gm;
            }
    if (energy) *energy = e;
    if (grad) {
        /* phi(k) = sum_m G(m) F(Q)(m) exp(+2 pi i m.k / K) = dE/dQ(k) */
        for (int ax = 0; ax < 3; ++ax) dft_axis(re, im, K, ax, +1);
        memset(grad, 0, sizeof(double) * 3 * (size_t)n);
        for (int i = 0; i < n; ++i) {
            double u[3];
            int k0[3];
            for (int c = 0; c < 3; ++c) {
                double x = s->x[3 * i + c] - L * floor(s->x[3 * i + c] / L);
                u[c] = K * x / L;
                k0[c] = (int)floor(u[c]);
            }
            for (int t0 = 0; t0 < p; ++t0)
                for (int t1 = 0; t1 < p; ++t1)
                    for (int t2 = 0; t2 < p; ++t2) {
                        int t[3] = { t0, t1, t2 }, k[3];
                        double M[3], dM[3];
                        for (int c = 0; c < 3; ++c) {
                            M[c] = bspline(p, u[c] - k0[c] + t[c]);
                            dM[c] = dbspline(p, u[c] - k0[c] + t[c]);
                            k[c] = (((k0[c] - t[c]) % K) + K) % K;
                        }
                        double ph = re[((size_t)k[2] * K + k[1]) * K + k[0]];
                        /* dQ(k)/dx_c = q (K / L) M'_p(u_c - k_c) prod_{d != c} M_p(u_d - k_d) */
                        grad[3 * i + 0] += s->q[i] * K / L * dM[0] * M[1] * M[2] * ph;
                        grad[3 * i + 1] += s->q[i] * K / L * M[0] * dM[1] * M[2] * ph;
                        grad[3 * i + 2] += s->q[i] * K / L * M[0] * M[1] * dM[2] * ph;
                    }
        }
    }
    free(Q); free(im); free(re); free(bmod);
    ewald_excl_self(s, grad, energy);
}

/* the reciprocal part of a gradient mode in Ewald mode (modes 0, 2, 4, 5, 6) */
static int mode_has_recip(const or_sys* s, int mode)
{
    return s->p.coulomb_mode == 1 && (mode == 0 || mode == 2 || mode == 4 || mode == 5 || mode == 6);
}

void or_gradient(or_sys* s, int mode, double* grad, double* energy)
{
    int n = s->n;
    memset(grad, 0, sizeof(double) * 3 * (size_t)n);
    double eb = 0, ea = 0, elj = 0, ec = 0;
    int weight = W_FULL, nb = 0, bo = 0;
    switch (mode) {
    case 0: weight = W_FULL; nb = 1; bo = 1; break;
    case 1: bo = 1; break;
    case 2: weight = W_FULL; nb = 1; break;
    case 3: weight = W_SHORT; nb = 1; break;
    case 4: weight = W_LONG; nb = 1; break;
    case 5: weight = W_SHORT; nb = 1; bo = 1; break;
    default: break;       /* 6: reciprocal part only (Ewald mode) */
    }
    if (nb) {
#pragma omp parallel for schedule(dynamic, 16) reduction(+:elj,ec)
        for (int i = 0; i < n; ++i) {
            double el, e2;
            nonbonded_atom(s, i, weight, &grad[3 * i], &el, &e2);
            elj += el;
            ec += e2;
        }
    }
    if (bo) bonded_gradient(s, grad, &eb, &ea);
    if (s->p.lj_long_mode == 2 && (mode == 5 || mode == 6)) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int i = 0; i < n; ++i) lj_long_atom(s, i, &grad[3 * i]);
    }
    double erec = 0.0;
    if (mode_has_recip(s, mode)) {
        double* g = (double*)malloc(sizeof(double) * 3 * (size_t)n);
        or_ewald_recip_pme(s, g, &erec, NULL);
        for (size_t k = 0; k < 3 * (size_t)n; ++k) grad[k] += g[k];
        free(g);
    }
    if (energy) *energy = eb + ea + 0.5 * (elj + ec) + erec;
}

void or_gradient_atom(or_sys* s, int mode, int i, double* g3)
{
    int weight = mode == 3 || mode == 5 ? W_SHORT : (mode == 4 ? W_LONG : W_FULL);
    g3[0] = g3[1] = g3[2] = 0.0;
    if (mode != 1 && mode != 6) nonbonded_atom(s, i, weight, g3, NULL, NULL);
    if (mode == 0 || mode == 1 || mode == 5) {
        double* g = (double*)calloc(3 * (size_t)s->n, sizeof(double));
        bonded_gradient(s, g, NULL, NULL);
        for (int c = 0; c < 3; ++c) g3[c] += g[3 * i + c];
        free(g);
    }
    if (s->p.lj_long_mode == 2 && (mode == 5 || mode == 6)) lj_long_atom(s, i, g3);
    if (mode_has_recip(s, mode)) {
        double* g = (double*)malloc(sizeof(double) * 3 * (size_t)s->n);
        or_ewald_recip_pme(s, g, NULL, NULL);
        for (int c = 0; c < 3; ++c) g3[c] += g[3 * i + c];
        free(g);
    }
}

void or_energy(or_sys* s, double* terms)
{
    double* g = (double*)calloc(3 * (size_t)s->n, sizeof(double));
    double eb, ea, elj = 0, ec = 0;
    bonded_gradient(s, g, &eb, &ea);
#pragma omp parallel for schedule(dynamic, 16) reduction(+:elj,ec)
    for (int i = 0; i < s->n; ++i) {
        double g3[3], el, e2;
        nonbonded_atom(s, i, W_FULL, g3, &el, &e2);
        elj += el;
        ec += e2;
    }
    double erec = 0.0;
    if (s->p.coulomb_mode == 1) or_ewald_recip_pme(s, NULL, &erec, NULL);
    terms[0] = eb; terms[1] = ea; terms[2] = 0.5 * elj; terms[3] = 0.5 * ec + erec;
    free(g);
}

/* acceleration a = -grad / m~ of a gradient mode */
static void accel(or_sys* s, int mode, double* a)
{
    or_gradient(s, mode, a, NULL);
    for (int i = 0; i < s->n; ++i)
        for (int c = 0; c < 3; ++c) a[3 * i + c] = -a[3 * i + c] / s->mt[i];
}

/* ======================================================================== */
/* B, A, O parts of the splitting (Sec. 2.3, JUMP integrator)              */
/* ======================================================================== */
static void kick(or_sys* s, const double* a, double h)
{
    for (int i = 0; i < 3 * s->n; ++i) s->v[i] += h * a[i];
}

static void drift(or_sys* s, double h)
{
    for (int i = 0; i < 3 * s->n; ++i) s->x[i] += h * s->v[i];
}

static void wrap(or_sys* s)
{
    for (int i = 0; i < 3 * s->n; ++i) {
        if (s->x[i] < 0.0) { s->x[i] += s->L; s->img[i] -= 1; }
        if (s->x[i] >= s->L) { s->x[i] -= s->L; s->img[i] += 1; }
    }
}

/* O: v <- e^{-gamma tau} v + sqrt((1 - e^{-2 gamma tau}) / (beta m~)) G, G from Box-Muller */
static void ostep(or_sys* s, double tau, uint32_t s0)
{
    double c1 = exp(-s->p.gamma * tau);
    double one_m = -expm1(-2.0 * s->p.gamma * tau);
    for (int i = 0; i < s->n; ++i) {
        uint32_t u[4];
        draw(s, (uint32_t)i, s0, TAG_O, 0, 0, 0, u);
        double r0 = sqrt(-2.0 * log(unif(u[0])));
        double r1 = sqrt(-2.0 * log(unif(u[2])));
        double G[3] = { r0 * cos(2.0 * OR_PI * unif(u[1])),
                        r0 * sin(2.0 * OR_PI * unif(u[1])),
                        r1 * cos(2.0 * OR_PI * unif(u[3])) };
        double c2 = sqrt(one_m / (s->beta * s->mt[i]));
        for (int c = 0; c < 3; ++c) s->v[3 * i + c] = c1 * s->v[3 * i + c] + c2 * G[c];
    }
}

static void log_event(or_sys* s, int64_t s0, int half, int tag, int atom, int64_t k, int J)
{
    if (s->ev_cap <= 0) return;
#pragma omp critical(or_event_log)
    {
        if (s->ev_n < s->ev_cap) {
            int64_t* e = &s->ev[6 * s->ev_n];
            e[0] = s0; e[1] = half; e[2] = tag; e[3] = atom; e[4] = k; e[5] = J;
            s->ev_n++;
        }
    }
}

/* ======================================================================== */
/* Step C' for one atom (Algorithm 4, adaptive eps, ring technique with     */
/* any number of rings up to four).                                         */
/* x is fixed, a = -grad U_short / m~ is the drift between jumps.           */
/* ======================================================================== */
static void cprime_atom(or_sys* s, int i, double* v, const double* a, double tau2,
                        uint32_t s0, int half, int64_t* nprop, int64_t* nacc, int64_t* natt,
                        uint32_t* err)
{
    int nr = s->nr;
    int N[OR_MAX_RINGS];
    const int* lidx[OR_MAX_RINGS];
    int ntot = 0;
    for (int y = 0; y < nr; ++y) {
        lidx[y] = list_of(s, y, i, &N[y]);
        ntot += N[y];
    }
    double beta = s->beta, mt = s->mt[i], eps0 = s->p.eps0;
    double t = 0.0;
    uint32_t k = 0;
    if (ntot == 0) {
        for (int c = 0; c < 3; ++c) v[c] += tau2 * a[c];
        return;
    }
    const double* LY = &s->LY[OR_MAX_RINGS * i];
    double aa = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    for (;;) {
        /* bound on |v| over the rest of the phase, then the rate bound per ring */
        double sr = tau2 - t;
        double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        double va = v[0] * a[0] + v[1] * a[1] + v[2] * a[2];
        double B = sqrt(vv + sr * sr * aa + 2.0 * sr * (va > 0.0 ? va : 0.0));
        double LamY[OR_MAX_RINGS], w[OR_MAX_RINGS], Lam = 0.0;
        for (int y = 0; y < nr; ++y) {
            if (s->p.eps_mode == 1) {
                double c0 = sqrt(beta / mt) / (eps0 * sqrt(2.0 * OR_PI));
                LamY[y] = beta * LY[y] * B + c0;
            } else {
                double c0 = sqrt(beta / (2.0 * OR_PI * mt)) / eps0;
                LamY[y] = LY[y] * (beta * B + c0);
            }
            w[y] = (double)N[y] * LamY[y];
            Lam += w[y];
        }
        uint32_t u[4];
        draw(s, (uint32_t)i, s0, TAG_C, half, 0, k, u);
        double T = -log(unif(u[0])) / Lam;
        if (!(Lam > 0.0) || t + T > tau2) {
            for (int c = 0; c < 3; ++c) v[c] += (tau2 - t) * a[c];
            break;
        }
        t += T;
        for (int c = 0; c < 3; ++c) v[c] += T * a[c];
        (*nprop)++;
        /* ring Y with probability w_Y / Lam (first ring whose cumulative
         * weight exceeds U1 Lam), then J uniform in ring Y */
        double target = unif(u[1]) * Lam, cum = 0.0;
        int Y = nr - 1;
        for (int y = 0; y < nr; ++y) {
            cum += w[y];
            if (target < cum) { Y = y; break; }
        }
        int J = lidx[Y][pick(u[2], N[Y])];
        double d[3];
        minimage(s, i, J, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        int inside = r >= s->edge[Y] && r < s->edge[Y + 1];
        double g[3] = { 0.0, 0.0, 0.0 };
        if (inside) {
            double f = OR_COULOMB * s->q[i] * s->q[J] * coul_long_dudr(s, r) / r;
            for (int c = 0; c < 3; ++c) g[c] = f * d[c];
        }
        double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        if (gn > 0.0) {
            double vg = v[0] * g[0] + v[1] * g[1] + v[2] * g[2];
            double eps, eta, p;
            if (s->p.eps_mode == 1) {
                eps = eps0 * gn;
                eta = eps0 * sqrt(beta * mt) * vg;
                p = sqrt(beta / mt) * or_theta(eta) / eps0 / LamY[Y];
            } else {
                eps = eps0;
                eta = eps0 * sqrt(beta * mt) * vg / gn;
                p = gn * or_theta(eta) / (LY[Y] * (eps0 * sqrt(beta * mt) * B + 1.0 / sqrt(2.0 * OR_PI)));
            }
            if (p > 1.0) *err |= OR_E_BOUND;
            if (unif(u[3]) <= p) {
                int att, fail;
                double Gt = gtilde(s, eta, (uint32_t)i, s0, half, k, &att, &fail);
                *natt += att;
                if (fail) *err |= OR_E_LIMIT;
                double coef = 2.0 * eps / (sqrt(beta * mt) * (1.0 + eps * eps)) * (eta + Gt) / gn;
                for (int c = 0; c < 3; ++c) v[c] -= coef * g[c];
                (*nacc)++;
                log_event(s, s0, half, (int)TAG_C, i, k, J);
            }
        }
        ++k;
        if (k >= OR_KMAX) {
            *err |= OR_E_LIMIT;
            for (int c = 0; c < 3; ++c) v[c] += (tau2 - t) * a[c];
            break;
        }
    }
}

/* ======================================================================== */
/* Step J' for one atom (Algorithm 5): BPS on the long-range LJ part. The   */
/* Poisson(N beta |v| L tau/2) count is drawn as the exponential arrivals   */
/* in [0, tau/2]; each proposal picks J uniformly and reflects with         */
/* probability (v . g)_+ / (|v| L).                                         */
/* ======================================================================== */
static void jprime_atom(or_sys* s, int i, double* v, double tau2, uint32_t s0, int half,
                        int64_t* nprop, int64_t* nacc, uint32_t* err)
{
    int N;
    const int* lidx = list_of(s, K_LJ, i, &N);
    double V = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double Li = s->LLJ[i];
    if (N == 0 || !(V > 0.0) || !(Li > 0.0)) return;
    double Lam = (double)N * s->beta * V * Li;
    double lo = s->p.r_split - s->p.h_switch, R = s->p.r_cut;
    double t = 0.0;
    uint32_t k = 0;
    for (;;) {
        uint32_t u[4];
        draw(s, (uint32_t)i, s0, TAG_J, half, 0, k, u);
        double T = -log(unif(u[0])) / Lam;
        if (t + T > tau2) break;
        t += T;
        (*nprop)++;
        int J = lidx[pick(u[2], N)];
        double d[3];
        minimage(s, i, J, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double g[3] = { 0.0, 0.0, 0.0 };
        if (r >= lo && r < R) {
            int ti = s->type[i], tj = s->type[J];
            double f = lj_long_dudr(s, s->eps[ti * s->ntypes + tj], s->sig[ti * s->ntypes + tj], r) / r;
            for (int c = 0; c < 3; ++c) g[c] = f * d[c];
        }
        double vg = v[0] * g[0] + v[1] * g[1] + v[2] * g[2];
        double p = (vg > 0.0 ? vg : 0.0) / (V * Li);
        if (p > 1.0) *err |= OR_E_BOUND;
        if (unif(u[3]) <= p) {
            double gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
            for (int c = 0; c < 3; ++c) v[c] -= 2.0 * vg / gg * g[c];
            (*nacc)++;
            log_event(s, s0, half, (int)TAG_J, i, k, J);
        }
        ++k;
        if (k >= OR_KMAX) { *err |= OR_E_LIMIT; break; }
    }
}

/* phase over all atoms: which = 0 C' only, 1 J' only */
static void cphase(or_sys* s, const double* a, double tau2, uint32_t s0, int half)
{
    int64_t np = 0, na = 0, nt = 0;
    uint32_t err = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+:np,na,nt) reduction(|:err)
    for (int i = 0; i < s->n; ++i)
        cprime_atom(s, i, &s->v[3 * i], &a[3 * i], tau2, s0, half, &np, &na, &nt, &err);
    s->cnt[0] += np; s->cnt[1] += na; s->cnt[4] += nt;
    s->err |= err;
}

static void jphase(or_sys* s, double tau2, uint32_t s0, int half)
{
    if (s->p.lj_long_mode) return;   /* the LJ long part is deterministic: no LJ jump mechanism */
    int64_t np = 0, na = 0;
    uint32_t err = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+:np,na) reduction(|:err)
    for (int i = 0; i < s->n; ++i)
        jprime_atom(s, i, &s->v[3 * i], tau2, s0, half, &np, &na, &err);
    s->cnt[2] += np; s->cnt[3] += na;
    s->err |= err;
}

void or_cprime_one(or_sys* s, int i, const double* v_in, const double* a_in, double tau2,
                   uint32_t s0, int half, double* v_out, int64_t* nprop, int64_t* nacc)
{
    double v[3] = { v_in[0], v_in[1], v_in[2] };
    int64_t np = 0, na = 0, nt = 0;
    uint32_t err = 0;
    cprime_atom(s, i, v, a_in, tau2, s0, half, &np, &na, &nt, &err);
    s->err |= err;
    for (int c = 0; c < 3; ++c) v_out[c] = v[c];
    if (nprop) *nprop = np;
    if (nacc) *nacc = na;
}

void or_jprime_one(or_sys* s, int i, const double* v_in, double tau2,
                   uint32_t s0, int half, double* v_out, int64_t* nprop, int64_t* nacc)
{
    double v[3] = { v_in[0], v_in[1], v_in[2] };
    int64_t np = 0, na = 0;
    uint32_t err = 0;
    jprime_atom(s, i, v, tau2, s0, half, &np, &na, &err);
    s->err |= err;
    for (int c = 0; c < 3; ++c) v_out[c] = v[c];
    if (nprop) *nprop = np;
    if (nacc) *nacc = na;
}

int or_sample_atom_work(or_sys* s, int n, const int* atoms, int mode, int n_grad, int n_phase,
                        double tau2, uint32_t s0, int nthreads)
{
    if (s->lazy) return -1;
    int used = 1;
    int weight = mode == 3 ? W_SHORT : W_FULL;
#ifdef _OPENMP
    int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int k = 0; k < n; ++k) {
        int i = atoms[k];
        double g[3] = { 0.0, 0.0, 0.0 }, v[3], a[3];
        for (int r = 0; r < n_grad; ++r) nonbonded_atom(s, i, weight, g, NULL, NULL);
        for (int c = 0; c < 3; ++c) { v[c] = s->v[3 * i + c]; a[c] = -g[c] / s->mt[i]; }
        int64_t np = 0, na = 0, nat = 0;
        uint32_t err = 0;
        for (int ph = 0; ph < n_phase; ++ph) {
            cprime_atom(s, i, v, a, tau2, s0, ph & 1, &np, &na, &nat, &err);
            if (!s->p.lj_long_mode) jprime_atom(s, i, v, tau2, s0, ph & 1, &np, &na, &err);
        }
#ifdef _OPENMP
        if (k == 0) used = omp_get_num_threads();
#endif
    }
    (void)nthreads;
    return used;
}

static void check_finite(or_sys* s)
{
    for (int i = 0; i < 3 * s->n; ++i)
        if (!isfinite(s->x[i]) || !isfinite(s->v[i])) { s->err |= OR_E_NONFIN; return; }
}

/* ======================================================================== */
/* integrators (Sec. 2.3 and Sec. 3.3). tau in ps.                          */
/* ======================================================================== */
/* inner A O A with a wrap of the positions */
static void aoa(or_sys* s, double tau, uint32_t s0)
{
    drift(s, 0.5 * tau);
    ostep(s, tau, s0);
    drift(s, 0.5 * tau);
    wrap(s);
}

/* BAOAB: B A O A [grad] B on the full potential */
int or_step_baoab(or_sys* s, int64_t nsteps, double dt_fs)
{
    if (s->lazy) return -1;   /* the steps rebuild the lists of every atom */
    double tau = dt_fs * 1e-3;
    accel(s, 0, s->a0);
    for (int64_t st = 0; st < nsteps; ++st) {
        uint32_t s0 = (uint32_t)s->step;
        kick(s, s->a0, 0.5 * tau);
        aoa(s, tau, s0);
        maybe_rebuild(s);
        accel(s, 0, s->a0);
        kick(s, s->a0, 0.5 * tau);
        s->step++;
        vrec(s);
    }
    check_finite(s);
    return (int)s->err;
}

/* JUMP: C' J' A O A J' C' with F0 = bonded + chi-weighted pairs */
int or_step_jump(or_sys* s, int64_t nsteps, double dt_fs)
{
    if (s->lazy) return -1;   /* the steps rebuild the lists of every atom */
    double tau = dt_fs * 1e-3;
    accel(s, 5, s->a0);
    for (int64_t st = 0; st < nsteps; ++st) {
        uint32_t s0 = (uint32_t)s->step;
        cphase(s, s->a0, 0.5 * tau, s0, 0);
        jphase(s, 0.5 * tau, s0, 0);
        aoa(s, tau, s0);
        maybe_rebuild(s);
        accel(s, 5, s->a0);
        jphase(s, 0.5 * tau, s0, 1);
        cphase(s, s->a0, 0.5 * tau, s0, 1);
        s->step++;
        vrec(s);
    }
    check_finite(s);
    return (int)s->err;
}

int or_step_bjaoajb(or_sys* s, int64_t nsteps, double dt_fs)
{
    if (s->lazy) return -1;
    double tau = dt_fs * 1e-3;
    double* zero = (double*)calloc(3 * (size_t)s->n, sizeof(double));
    accel(s, 5, s->a0);
    for (int64_t st = 0; st < nsteps; ++st) {
        uint32_t s0 = (uint32_t)s->step;
        kick(s, s->a0, 0.5 * tau);
        cphase(s, zero, 0.5 * tau, s0, 0);
        jphase(s, 0.5 * tau, s0, 0);
        aoa(s, tau, s0);
        maybe_rebuild(s);
        accel(s, 5, s->a0);
        jphase(s, 0.5 * tau, s0, 1);
        cphase(s, zero, 0.5 * tau, s0, 1);
        kick(s, s->a0, 0.5 * tau);
        s->step++;
        vrec(s);
    }
    free(zero);
    check_finite(s);
    return (int)s->err;
}

/* innermost RESPA step on the bonded force: B A O A [grad] B */
static void inner_bonded(or_sys* s, double dt, int record)
{
    uint32_t s0 = (uint32_t)s->step;
    kick(s, s->ab, 0.5 * dt);
    aoa(s, dt, s0);
    accel(s, 1, s->ab);
    kick(s, s->ab, 0.5 * dt);
    s->step++;
    if (record) vrec(s);
}

/* BAOAB-RESPA: B_nb(D/2) [n x inner bonded] B_nb(D/2), D = n dt */
int or_step_baoab_respa(or_sys* s, int64_t nouter, double dt_inner_fs, int n_inner)
{
    if (s->lazy) return -1;   /* the steps rebuild the lists of every atom */
    double dt = dt_inner_fs * 1e-3, D = dt * n_inner;
    accel(s, 1, s->ab);
    accel(s, 2, s->al);
    for (int64_t o = 0; o < nouter; ++o) {
        kick(s, s->al, 0.5 * D);
        for (int k = 0; k < n_inner; ++k) inner_bonded(s, dt, k < n_inner - 1);
        maybe_rebuild(s);
        accel(s, 2, s->al);
        kick(s, s->al, 0.5 * D);
        vrec(s);
    }
    check_finite(s);
    return (int)s->err;
}

/* BAOAB-RESPA1: B_long(D/2) [n x (B_short(k/2) [m x inner] B_short(k/2))] B_long(D/2) */
int or_step_baoab_respa1(or_sys* s, int64_t nouter, double dt_inner_fs, int m_mid, int n_outer)
{
    if (s->lazy) return -1;   /* the steps rebuild the lists of every atom */
    double dt = dt_inner_fs * 1e-3, kap = dt * m_mid, D = kap * n_outer;
    accel(s, 1, s->ab);
    accel(s, 3, s->as);
    accel(s, 4, s->al);
    for (int64_t o = 0; o < nouter; ++o) {
        kick(s, s->al, 0.5 * D);
        for (int j = 0; j < n_outer; ++j) {
            kick(s, s->as, 0.5 * kap);
            for (int k = 0; k < m_mid; ++k) inner_bonded(s, dt, k < m_mid - 1);
            maybe_rebuild(s);
            accel(s, 3, s->as);
            kick(s, s->as, 0.5 * kap);
            if (j < n_outer - 1) vrec(s);
        }
        maybe_rebuild(s);
        accel(s, 4, s->al);
        kick(s, s->al, 0.5 * D);
        vrec(s);
    }
    check_finite(s);
    return (int)s->err;
}

/* JUMP-RESPA: C'(D/2) J'(D/2) [n x inner bonded] J'(D/2) C'(D/2), the
 * C' drift being the short-range nonbonded acceleration */
int or_step_jump_respa(or_sys* s, int64_t nouter, double dt_inner_fs, int n_inner)
{
    if (s->lazy) return -1;   /* the steps rebuild the lists of every atom */
    double dt = dt_inner_fs * 1e-3, D = dt * n_inner;
    /* the slow deterministic force (the Ewald reciprocal part, and the LJ long
     * part in lj_long_mode 2) is kicked at D (Sec. 2.3) */
    int ew = s->p.coulomb_mode == 1 || s->p.lj_long_mode == 2;
    accel(s, 1, s->ab);
    accel(s, 3, s->as);
    if (ew) accel(s, 6, s->al);
    for (int64_t o = 0; o < nouter; ++o) {
        uint32_t s0 = (uint32_t)s->step;
        if (ew) kick(s, s->al, 0.5 * D);
        cphase(s, s->as, 0.5 * D, s0, 0);
        jphase(s, 0.5 * D, s0, 0);
        for (int k = 0; k < n_inner; ++k) inner_bonded(s, dt, k < n_inner - 1);
        maybe_rebuild(s);
        accel(s, 3, s->as);
        jphase(s, 0.5 * D, s0, 1);
        cphase(s, s->as, 0.5 * D, s0, 1);
        if (ew) { accel(s, 6, s->al); kick(s, s->al, 0.5 * D); }
        vrec(s);
    }
    check_finite(s);
    return (int)s->err;
}

/* JUMP-RESPA1: the outer level holds the slow many-body force: the Ewald
 * reciprocal part (absent with DSF electrostatics, the level is then empty);
 * the mid level kappa = m dt carries the short-range pairs and the jumps, the
 * inner level the bonded terms. */
int or_step_jump_respa1(or_sys* s, int64_t nouter, double dt_inner_fs, int m_mid, int n_outer)
{
    if (s->lazy) return -1;   /* the steps rebuild the lists of every atom */
    double dt = dt_inner_fs * 1e-3, kap = dt * m_mid, D = kap * n_outer;
    int ew = s->p.coulomb_mode == 1 || s->p.lj_long_mode == 2;
    accel(s, 1, s->ab);
    accel(s, 3, s->as);
    if (ew) accel(s, 6, s->al);
    for (int64_t o = 0; o < nouter; ++o) {
        if (ew) kick(s, s->al, 0.5 * D);
        for (int j = 0; j < n_outer; ++j) {
            uint32_t s0 = (uint32_t)s->step;
            cphase(s, s->as, 0.5 * kap, s0, 0);
            jphase(s, 0.5 * kap, s0, 0);
            for (int k = 0; k < m_mid; ++k) inner_bonded(s, dt, k < m_mid - 1);
            maybe_rebuild(s);
            accel(s, 3, s->as);
            jphase(s, 0.5 * kap, s0, 1);
            cphase(s, s->as, 0.5 * kap, s0, 1);
            if (j < n_outer - 1) vrec(s);
        }
        if (ew) { accel(s, 6, s->al); kick(s, s->al, 0.5 * D); }
        vrec(s);
    }
    check_finite(s);
    return (int)s->err;
}

/* ======================================================================== */
/* construction and state                                                   */
/* ======================================================================== */
or_sys* or_create(int n, const or_params* p,
                  const double* x, const double* v,
                  const double* mass, const double* charge, const int* type,
                  int ntypes, const double* lj_eps, const double* lj_sigma,
                  int nbonds, const int* bonds, const double* bond_k, const double* bond_r0,
                  int nangles, const int* angles, const double* angle_k, const double* angle_t0,
                  int nexcl, const int* excl_pairs)
{
    or_sys* s = (or_sys*)calloc(1, sizeof(or_sys));
    s->n = n;
    s->p = *p;
    s->L = p->box;
    size_t n3 = 3 * (size_t)n;
    s->x = (double*)malloc(sizeof(double) * n3);
    s->v = (double*)malloc(sizeof(double) * n3);
    s->xb = (double*)malloc(sizeof(double) * n3);
    s->img = (int*)calloc(n3, sizeof(int));
    memcpy(s->x, x, sizeof(double) * n3);
    memcpy(s->v, v, sizeof(double) * n3);
    s->m = (double*)malloc(sizeof(double) * (size_t)n);
    s->mt = (double*)malloc(sizeof(double) * (size_t)n);
    s->q = (double*)malloc(sizeof(double) * (size_t)n);
    s->type = (int*)malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        s->m[i] = mass[i];
        s->mt[i] = mass[i] / OR_KCAL_AMU;
        s->q[i] = charge[i];
        s->type[i] = type[i];
    }
    s->ntypes = ntypes;
    s->eps = (double*)malloc(sizeof(double) * (size_t)(ntypes * ntypes));
    s->sig = (double*)malloc(sizeof(double) * (size_t)(ntypes * ntypes));
    memcpy(s->eps, lj_eps, sizeof(double) * (size_t)(ntypes * ntypes));
    memcpy(s->sig, lj_sigma, sizeof(double) * (size_t)(ntypes * ntypes));
    s->nb = nbonds;
    s->bonds = (int*)malloc(sizeof(int) * (size_t)(2 * nbonds + 1));
    s->bk = (double*)malloc(sizeof(double) * (size_t)(nbonds + 1));
    s->br0 = (double*)malloc(sizeof(double) * (size_t)(nbonds + 1));
    if (nbonds) {
        memcpy(s->bonds, bonds, sizeof(int) * 2 * (size_t)nbonds);
        memcpy(s->bk, bond_k, sizeof(double) * (size_t)nbonds);
        memcpy(s->br0, bond_r0, sizeof(double) * (size_t)nbonds);
    }
    s->na = nangles;
    s->angles = (int*)malloc(sizeof(int) * (size_t)(3 * nangles + 1));
    s->ak = (double*)malloc(sizeof(double) * (size_t)(nangles + 1));
    s->at0 = (double*)malloc(sizeof(double) * (size_t)(nangles + 1));
    if (nangles) {
        memcpy(s->angles, angles, sizeof(int) * 3 * (size_t)nangles);
        memcpy(s->ak, angle_k, sizeof(double) * (size_t)nangles);
        memcpy(s->at0, angle_t0, sizeof(double) * (size_t)nangles);
    }
    /* per-atom exclusion lists (both directions) */
    s->exoff = (int*)calloc((size_t)(n + 1), sizeof(int));
    for (int e = 0; e < nexcl; ++e) {
        s->exoff[excl_pairs[2 * e] + 1]++;
        s->exoff[excl_pairs[2 * e + 1] + 1]++;
    }
    for (int i = 0; i < n; ++i) s->exoff[i + 1] += s->exoff[i];
    s->exidx = (int*)malloc(sizeof(int) * (size_t)(2 * nexcl + 1));
    int* fill = (int*)calloc((size_t)n, sizeof(int));
    for (int e = 0; e < nexcl; ++e) {
        int a = excl_pairs[2 * e], b = excl_pairs[2 * e + 1];
        s->exidx[s->exoff[a] + fill[a]++] = b;
        s->exidx[s->exoff[b] + fill[b]++] = a;
    }
    free(fill);
    s->beta = 1.0 / (OR_KB * p->temperature);
    s->LY = (double*)malloc(sizeof(double) * OR_MAX_RINGS * (size_t)n);
    s->LLJ = (double*)malloc(sizeof(double) * (size_t)n);
    compute_bounds(s);
    if (s->p.skin_outer < s->p.skin) s->p.skin_outer = s->p.skin;
    int nc = (int)floor(2.0 * s->L / (s->p.r_cut + s->p.skin_outer));
    s->ncell = nc < 1 ? 1 : nc;
    s->cellm = (int*)malloc(sizeof(int) * (size_t)n);
    s->xo = (double*)malloc(sizeof(double) * n3);
    s->a0 = (double*)calloc(n3, sizeof(double));
    s->ab = (double*)calloc(n3, sizeof(double));
    s->as = (double*)calloc(n3, sizeof(double));
    s->al = (double*)calloc(n3, sizeof(double));
    wrap(s);
    memset(s->img, 0, sizeof(int) * n3);
    outer_rebuild(s);
    s->lazy = p->lazy_lists != 0;
    s->alist_atom = -1;
    if (!s->lazy) build_lists(s);
    s->cnt[5] = 0;
    return s;
}

void or_destroy(or_sys* s)
{
    if (!s) return;
    free(s->x); free(s->v); free(s->xb); free(s->img);
    free(s->m); free(s->mt); free(s->q); free(s->type);
    free(s->eps); free(s->sig);
    free(s->bonds); free(s->bk); free(s->br0);
    free(s->angles); free(s->ak); free(s->at0);
    free(s->exoff); free(s->exidx);
    free(s->LY); free(s->LLJ);
    for (int k = 0; k < K_NKIND; ++k) { free(s->lists[k].off); free(s->lists[k].idx); free(s->alist[k]); }
    free(s->a0); free(s->ab); free(s->as); free(s->al);
    free(s->cellm); free(s->xo);
    free(s->vr);
    free(s->ev);
    free(s);
}

void or_set_threads(int nthreads)
{
#ifdef _OPENMP
    omp_set_num_threads(nthreads > 0 ? nthreads : omp_get_num_procs());
#else
    (void)nthreads;
#endif
}

int or_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_get_state(const or_sys* s, double* x, double* v, int* img, double* x_build,
                  double* x_outer)
{
    size_t n3 = 3 * (size_t)s->n;
    if (x) memcpy(x, s->x, sizeof(double) * n3);
    if (v) memcpy(v, s->v, sizeof(double) * n3);
    if (img) memcpy(img, s->img, sizeof(int) * n3);
    if (x_build) memcpy(x_build, s->xb, sizeof(double) * n3);
    if (x_outer) memcpy(x_outer, s->xo, sizeof(double) * n3);
}

/* restore a state; with x_build (list build positions) and x_outer (outer
 * rebuild positions) the lists are rebuilt as they were, so that a resumed
 * run repeats the uninterrupted one */
void or_set_state(or_sys* s, const double* x, const double* v, const int* img,
                  const double* x_build, const double* x_outer, int64_t step)
{
    size_t n3 = 3 * (size_t)s->n;
    memcpy(s->x, x_outer ? x_outer : (x_build ? x_build : x), sizeof(double) * n3);
    outer_rebuild(s);
    if (x_build) memcpy(s->x, x_build, sizeof(double) * n3);
    if (!s->lazy) {
        build_lists(s);
        s->cnt[5]--;
    }
    s->alist_atom = -1;
    memcpy(s->x, x, sizeof(double) * n3);
    memcpy(s->v, v, sizeof(double) * n3);
    if (img) memcpy(s->img, img, sizeof(int) * n3);
    s->step = step;
}

int64_t or_step_count(const or_sys* s) { return s->step; }

void or_counters(const or_sys* s, int64_t* out)
{
    for (int k = 0; k < OR_NCOUNTERS; ++k) out[k] = s->cnt[k];
}

uint32_t or_errors(const or_sys* s) { return s->err; }

void or_events_enable(or_sys* s, int64_t cap)
{
    free(s->ev);
    s->ev = cap > 0 ? (int64_t*)malloc(sizeof(int64_t) * 6 * (size_t)cap) : NULL;
    s->ev_cap = cap;
    s->ev_n = 0;
}

int64_t or_events_get(const or_sys* s, int64_t* out6)
{
    if (out6 && s->ev_n) memcpy(out6, s->ev, sizeof(int64_t) * 6 * (size_t)s->ev_n);
    return s->ev_n;
}

void or_vrec_enable(or_sys* s, int64_t cap)
{
    free(s->vr);
    s->vr = cap > 0 ? (double*)malloc(sizeof(double) * 3 * (size_t)s->n * (size_t)cap) : NULL;
    s->vr_cap = cap;
    s->vr_n = 0;
}

int64_t or_vrec_get(const or_sys* s, double* out)
{
    const int64_t k = s->vr_n < s->vr_cap ? s->vr_n : s->vr_cap;
    if (out && k) memcpy(out, s->vr, sizeof(double) * 3 * (size_t)s->n * (size_t)k);
    return k;
}

/* mass-weighted velocity autocorrelation, by its definition: the average
 * over the time origins t of sum_i m_i v_i(t) . v_i(t + k) */
void or_vacf(const double* v, const double* mass, int n, int64_t T, int64_t nlags, double* out)
{
    for (int64_t k = 0; k < nlags; ++k) {
        double acc = 0.0;
        if (k < T) {
            for (int64_t t = 0; t + k < T; ++t) {
                const double* a = v + 3 * (size_t)n * (size_t)t;
                const double* b = v + 3 * (size_t)n * (size_t)(t + k);
                for (int i = 0; i < n; ++i)
                    acc += mass[i] * (a[3 * i] * b[3 * i] + a[3 * i + 1] * b[3 * i + 1] + a[3 * i + 2] * b[3 * i + 2]);
            }
            acc /= (double)(T - k);
        }
        out[k] = acc;
    }
}

/* Hann-windowed cosine transform of an autocorrelation C(0..K-1):
 * S_j = C(0) + 2 sum_{k=1}^{K-1} w_k C(k) cos(pi j k / K), w_k = (1 + cos(pi k / K)) / 2,
 * j = 0..K-1; with samples dt apart, bin j is the frequency j / (2 K dt) */
void or_vacf_spectrum(const double* C, int64_t K, double* S)
{
    for (int64_t j = 0; j < K; ++j) {
        double acc = C[0];
        for (int64_t k = 1; k < K; ++k) {
            const double w = 0.5 * (1.0 + cos(OR_PI * (double)k / (double)K));
            acc += 2.0 * w * C[k] * cos(OR_PI * (double)((j * k) % (2 * K)) / (double)K);
        }
        S[j] = acc;
    }
}
