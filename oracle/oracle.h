/*
 * oracle.h -- plain FP64 CPU oracle for the Velocity Jumps (JUMP) MD path.
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load or call this library. The product
 * path (the CUDA library behind include/md.h) never does, and the two share
 * no code: this file and oracle.c are written independently from the paper
 * ("Velocity Jumps for Molecular Dynamics", Gouraud et al., arXiv 2412.15073).
 *
 * Units: kcal/mol, Angstrom, ps, amu, elementary charge. The paper's F_i are
 * gradients of U (Sec. 2.1, the decomposition of grad U); everything here that
 * is called "grad" is a gradient, the force is its negative.
 *
 * Parity status (pins live in tests/test_oracle_*.py):
 *   philox, uniforms ............ pinned (statistics)
 *   pair potentials, gradients .. pinned (finite differences, closed forms)
 *   Theta, G~ sampler ........... pinned (quadrature, exact CDF, KS test)
 *   thinning (C', J') ........... pinned (survival laws, BPS bounce law)
 *   JUMP invariance ............. pinned (Boltzmann law of a 2-body system)
 *   BAOAB ....................... pinned (exact harmonic variance, Verlet order)
 *   RESPA / RESPA1 drivers ...... pinned by reduction (n = 1 equals BAOAB) and
 *                                 by their energy error at gamma 0 (second order)
 *   JUMP-RESPA, JUMP-RESPA1 ..... pinned (Boltzmann laws of the three bond
 *                                 lengths of a harmonic chain whose bonded pair
 *                                 also jumps; with an LJ slow level as well)
 *   LJ long modes 1, 2 .......... pinned by reduction (moved part = pair sum)
 *   Ewald, plain reciprocal sum . pinned (rock-salt Madelung constant; the
 *                                 full gradient is the derivative of its energy)
 *   smooth PME .................. pinned (plain sum per order, grid refinement,
 *                                 finite differences of its energy)
 *   VACF, spectrum .............. pinned (closed forms, numpy correlate)
 */
#ifndef MD_ORACLE_H
#define MD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double box;          /* cubic periodic box edge (A) */
    double r_cut;        /* r_E: outer cutoff of LJ and DSF Coulomb (A) */
    double r_split;      /* r_c: short/long split radius (A) */
    double h_switch;     /* h: width of the switch, chi goes 1 -> 0 on [r_c-h, r_c] */
    double r_mid;        /* r_M: ring boundary when n_rings == 0; <= r_c-h or >= r_E means one ring */
    double dsf_alpha;    /* DSF damping (1/A) */
    double gamma;        /* friction (1/ps) */
    double temperature;  /* K */
    double eps0;         /* jump parameter: eps = eps0*|g| (adaptive) or eps0 (constant) */
    double skin;         /* Verlet skin (A); lists are rebuilt when an atom moved > skin/2 */
    double skin_outer;   /* skin of the outer candidate grid (>= skin); it fixes the list order */
    int eps_mode;        /* 1 adaptive (the paper's choice), 0 constant */
    int n_rings;         /* 0: rings from r_mid; 1..4: ring edges r_c-h, ring_r[0..n-2], r_E */
    double ring_r[3];    /* interior ring edges, increasing, inside (r_c-h, r_E) */
    uint32_t seed;       /* Philox key word 0 */
    uint32_t replica;    /* Philox key word 1 */
    int lazy_lists;      /* nonzero: no list build at creation; the lists of one atom are built
                          * when a per-atom call needs them (for very large systems whose O(N^2)
                          * list build is out of reach); the or_step_* calls then return -1 */
    int lj_long_mode;    /* 0: the long-range LJ part (1-chi) U_LJ is handled by BPS jumps (J');
                          * 1: it is deterministic, in F0 (the paper's GPU runs): gradient modes
                          * 3 and 5 carry the whole LJ, mode 4 only (1-chi) Coulomb, no J';
                          * 2: deterministic at the slow level: modes 3 and 4 split LJ by chi as
                          * in mode 0, mode 5 adds the (1-chi) LJ part (F0 of JUMP), mode 6 holds
                          * it (with the Ewald reciprocal part), JUMP-RESPA(1) kick mode 6 at
                          * their outer step, no J' */
    int coulomb_mode;    /* 0: DSF Coulomb (damping dsf_alpha); 1: Ewald: real-space pairs
                          * erfc(alpha r)/r to r_cut (alpha = dsf_alpha) split by chi as in
                          * Sec. 3.1, plus a smooth-PME reciprocal sum (Essmann et al. 1995),
                          * the self term and the exclusion correction */
    int pme_order;       /* B-spline order p of the reciprocal sum (Ewald mode) */
    double pme_spacing;  /* target grid spacing (A); K = smallest 2,3,5-smooth integer >= L/spacing */
} or_params;

typedef struct or_sys or_sys;

/* Counters: [0] C' proposals [1] C' accepts [2] J' proposals [3] J' accepts
 *           [4] sampler attempts [5] list rebuilds */
#define OR_NCOUNTERS 6

/* error flags (bitwise OR) */
#define OR_E_BOUND   1u   /* thinning ratio p > 1: a rate bound was violated */
#define OR_E_LIMIT   2u   /* sampler attempt cap or proposal cap reached */
#define OR_E_NONFIN  4u   /* non-finite state */

or_sys* or_create(int n, const or_params* p,
                  const double* x, const double* v,
                  const double* mass, const double* charge, const int* type,
                  int ntypes, const double* lj_eps, const double* lj_sigma,
                  int nbonds, const int* bonds, const double* bond_k, const double* bond_r0,
                  int nangles, const int* angles, const double* angle_k, const double* angle_t0,
                  int nexcl, const int* excl_pairs);
void or_destroy(or_sys* s);
void or_set_threads(int nthreads);
int  or_get_threads(void);

/* state */
void    or_get_state(const or_sys* s, double* x, double* v, int* img, double* x_build,
                     double* x_outer);
void    or_set_state(or_sys* s, const double* x, const double* v, const int* img,
                     const double* x_build, const double* x_outer, int64_t step);
int64_t or_step_count(const or_sys* s);
void    or_counters(const or_sys* s, int64_t* out);
uint32_t or_errors(const or_sys* s);

/* forces: mode 0 full (bonded + all pairs), 1 bonded only, 2 nonbonded full,
 * 3 nonbonded short (chi-weighted), 4 nonbonded long ((1-chi)-weighted),
 * 5 F0 of JUMP (bonded + short). Brute force over all pairs, minimum image.
 * grad is 3n (row-major xyz). energy (may be NULL) gets the matching energy. */
void or_gradient(or_sys* s, int mode, double* grad, double* energy);
/* full potential energy terms: [bond, angle, lj, coulomb] */
void or_energy(or_sys* s, double* terms);
/* per-atom gradient of the chosen mode for one atom only (O(N)) */
void or_gradient_atom(or_sys* s, int mode, int i, double* g3);

/* rate bounds: lhat[4] the per-ring max of |d/dr (1-chi) u_DSF| (unit
 * charges, per C q_i q_j), qmax, edges[5] the ring edges, nrings; per atom
 * LY (n x 4, row-major) and LLJ arrays (any may be NULL) */
void or_bounds(const or_sys* s, double* lhat, double* qmax, double* edges, int* nrings, double* LY, double* LLJ);

/* jump lists: kind 0..3 ring 0..3 (inner to outer), 4 LJ. counts[n]; list of one atom */
void or_list_counts(or_sys* s, int kind, int* counts);
int  or_list_get(or_sys* s, int kind, int i, int* out);
/* force a rebuild now */
void or_rebuild(or_sys* s);

/* single-phase primitives (x fixed) for one atom, used by pins and by the
 * sampled parity at full size. They read the lists of atom i. */
void or_cprime_one(or_sys* s, int i, const double* v_in, const double* a_in, double tau2,
                   uint32_t s0, int half, double* v_out, int64_t* nprop, int64_t* nacc);
void or_jprime_one(or_sys* s, int i, const double* v_in, double tau2,
                   uint32_t s0, int half, double* v_out, int64_t* nprop, int64_t* nacc);

/* timing workload of the CPU baseline: the per-atom work of one step for a
 * sample of atoms. For each listed atom: n_grad brute-force evaluations of its
 * nonbonded gradient of weight mode (2 full, 3 short), then n_phase C' phases
 * over tau2 (drift by the last gradient over m~), each followed by a J' phase
 * when the LJ long part jumps. Velocities and counters are left untouched.
 * The atoms are spread over nthreads OpenMP threads (<= 0: all available);
 * returns the number of threads that ran. Needs lists of all atoms (not lazy). */
int or_sample_atom_work(or_sys* s, int n, const int* atoms, int mode, int n_grad, int n_phase,
                        double tau2, uint32_t s0, int nthreads);

/* integrators (dt in fs) */
int or_step_baoab(or_sys* s, int64_t nsteps, double dt_fs);
int or_step_baoab_respa(or_sys* s, int64_t nouter, double dt_inner_fs, int n_inner);
int or_step_baoab_respa1(or_sys* s, int64_t nouter, double dt_inner_fs, int m_mid, int n_outer);
int or_step_jump(or_sys* s, int64_t nsteps, double dt_fs);
/* Ewald mode: the reciprocal-space gradient and energy by the plain Ewald
 * sum over the integer vectors n with |n| <= kmax (m = n / L), no
 * interpolation; the self term and the exclusion correction are included.
 * The reference the smooth-PME sum of the integrators is checked against. */
void or_ewald_recip_plain(const or_sys* s, int kmax, double* grad, double* energy);
/* the same quantities from the smooth-PME sum used by the integrators; K the grid */
void or_ewald_recip_pme(const or_sys* s, double* grad, double* energy, int* K);

/* BJAOAJB (Sec. 2.3): B(dt/2) with F0, then the jump processes alone over
 * dt/2 (C' with zero drift, then J'), A O A, F0, J', C' (zero drift), B. */
int or_step_bjaoajb(or_sys* s, int64_t nsteps, double dt_fs);
int or_step_jump_respa(or_sys* s, int64_t nouter, double dt_inner_fs, int n_inner);
int or_step_jump_respa1(or_sys* s, int64_t nouter, double dt_inner_fs, int m_mid, int n_outer);

/* accepted-jump log: records (s, half, tag, atom, k, J) of every accepted jump */
void    or_events_enable(or_sys* s, int64_t cap);
int64_t or_events_get(const or_sys* s, int64_t* out6);

/* velocity record for spectra (Sec. 4, the velocity autocorrelation spectra
 * of the multiple-time-step integrators): v after each innermost step, taken
 * after the closing kicks and phases of every level that ends at that step;
 * at most cap samples are kept (later ones are counted, not stored) */
void    or_vrec_enable(or_sys* s, int64_t cap);
int64_t or_vrec_get(const or_sys* s, double* out);     /* T x 3n; returns T */
/* mass-weighted VACF of a series v[T][n][3]: out[k] = (1 / (T - k))
 * sum_{t=0}^{T-1-k} sum_i m_i v_i(t) . v_i(t + k), k < nlags (0 for k >= T) */
void or_vacf(const double* v, const double* mass, int n, int64_t T, int64_t nlags, double* out);
/* Hann-windowed cosine transform S_j = C(0) + 2 sum_{k=1}^{K-1} w_k C(k) cos(pi j k / K),
 * w_k = (1 + cos(pi k / K)) / 2, j < K */
void or_vacf_spectrum(const double* C, int64_t K, double* S);

/* primitives */
void   or_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out);
double or_theta(double eta);
double or_sample_gtilde(double eta, uint32_t seed, uint32_t replica, uint32_t atom,
                        uint32_t s0, int half, uint32_t k, int* attempts);
double or_pair_dudr(const or_sys* s, int ti, int tj, double qiqj, double r, int weight);
double or_pair_u(const or_sys* s, int ti, int tj, double qiqj, double r, int weight);

#ifdef __cplusplus
}
#endif
#endif
