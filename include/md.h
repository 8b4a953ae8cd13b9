/*
 * md.h -- C ABI of the GB300 (sm_103a) Velocity Jumps molecular-dynamics
 * library (libmdjump.so).
 *
 * What it computes: Langevin dynamics of fixed-charge systems with
 * Lennard-Jones + damped-shifted-force (DSF) Coulomb pairs and harmonic bonds
 * and angles, integrated by BAOAB / BAOAB-RESPA / BAOAB-RESPA1 or by the
 * Velocity Jumps integrators JUMP / JUMP-RESPA / JUMP-RESPA1 of Gouraud et
 * al., "Velocity Jumps for Molecular Dynamics" (arXiv 2412.15073):
 *   - the Langevin SDE and the split grad U = F_0 + sum_i F_i (Sec. 2.1);
 *   - the jump rate, jump kernel and density f_eta of G~ (Sec. 2.2);
 *   - the splittings BAOAB-like, C'J'AOAJ'C', RESPA and RESPA1 (Sec. 2.3);
 *   - Poisson thinning and rejection sampling of G~ (Sec. 2.4, Alg. 1-3);
 *   - pair jumps on the long-range electrostatics with adaptive eps and the
 *     ring technique (Sec. 3.1, Alg. 4) and BPS jumps on the long-range LJ
 *     part (Sec. 3.2, Alg. 5).
 *
 * Units: kcal/mol, Angstrom, ps (time steps are passed in fs), amu, e.
 *
 * Conventions for every entry point:
 *   - Return value: MD_OK (0) or a negative MD_E* code. After an error,
 *     md_last_error(ctx) gives a one-line message. Errors raised by the GPU
 *     (bound violated, overflow, non-finite state) are sticky: they stay in
 *     the context's error flags until md_set_system is called again.
 *   - Pointers named host_* or documented as host pointers are read or written
 *     with ordinary CPU accesses; the library copies what it needs and never
 *     keeps caller pointers after the call returns.
 *   - Arrays of atoms are row-major (atom, xyz) doubles: 3*n_atoms values.
 *   - All device memory is owned by the context, allocated stream-ordered on
 *     md_config.cuda_stream and released by md_finalize.
 *   - Calls on one context must not overlap (no internal locking).
 */
#ifndef MDJUMP_MD_H
#define MDJUMP_MD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MD_OK           0
#define MD_EINVAL      -1   /* an argument is out of range or inconsistent */
#define MD_ECUDA       -2   /* a CUDA runtime call failed */
#define MD_EOVERFLOW   -3   /* a pair term outside the fixed-point range (|component| >= 2^20 kcal/mol/A,
                             * or not finite), or a neighbour-list capacity exceeded */
#define MD_EBOUND      -4   /* thinning ratio p > 1: a rate bound was violated */
#define MD_ELIMIT      -5   /* sampler attempt cap or per-phase proposal cap reached */
#define MD_ENONFINITE  -6   /* NaN or Inf in positions or velocities */
#define MD_ENOSYSTEM   -7   /* replica has no system (md_set_system not called) */
#define MD_ENOMEM      -8   /* device allocation failed */

/* GPU error flag bits, as reported in md_obs.error_flags */
#define MD_FLAG_BOUND     1u
#define MD_FLAG_LIMIT     2u
#define MD_FLAG_NONFINITE 4u
#define MD_FLAG_OVERFLOW  8u

typedef struct md_ctx md_ctx;

/* Arithmetic of the hot path.
 *   MD_FP64:  every step in double precision (parity mode).
 *   MD_MIXED: FP32 pair arithmetic and jump loops, pair forces summed in
 *             64-bit fixed point (2^-32 kcal/mol/A; order independent), FP64
 *             positions, velocities, integration, O-step and acceptance near
 *             ties (|U - p| < 2e-6 is decided again in FP64). */
enum { MD_FP64 = 0, MD_MIXED = 1 };

typedef struct {
    int precision;         /* MD_FP64 or MD_MIXED */
    uint64_t seed;         /* Philox key word 0 = low 32 bits of seed, word 1 = replica */
    int device;            /* CUDA device ordinal */
    void* cuda_stream;     /* cudaStream_t used for every launch and copy; NULL = default stream */
    int max_replicas;      /* replicas advanced together by each md_step_* call (>= 1) */
    int64_t event_log_cap; /* capacity of the accepted-jump log (0 = off) */
    int threads_per_atom;  /* pair kernel: 0 = autotune at the first step, else 1, 2, 4 or 8 */
    int no_graphs;         /* 0: md_step_* calls replay CUDA graphs of chunks of about four innermost
                            * steps (four steps, two RESPA cycles of two, or one longer cycle),
                            * captured on a private stream ordered after cuda_stream the first time a
                            * call of that integrator, time step and system layout has more than one
                            * chunk's worth of steps; later calls of at least one chunk replay the
                            * graph from their first step on. Nonzero: plain launches. Results are
                            * identical either way. */
} md_config;

/* One periodic system (cubic box). All pointers are host pointers, copied. */
typedef struct {
    int n_atoms;
    double box;                                  /* edge (A); needs r_cut + skin_outer <= box/2 */
    const double* x;                             /* 3n positions (A) */
    const double* v;                             /* 3n velocities (A/ps) */
    const double* mass;                          /* n (amu) */
    const double* charge;                        /* n (e) */
    const int* type;                             /* n LJ types in [0, n_types) */
    int n_types;                                 /* <= 8 */
    const double* lj_eps;                        /* n_types^2 (kcal/mol), mixing done by the caller */
    const double* lj_sigma;                      /* n_types^2 (A) */
    int n_bonds;   const int* bonds;   const double* bond_k;  const double* bond_r0;   /* 1/2 k (r - r0)^2 */
    int n_angles;  const int* angles;  const double* angle_k; const double* angle_t0;  /* 1/2 k (t - t0)^2, centre in the middle */
    int n_excl;    const int* excl_pairs;        /* pairs with no nonbonded interaction */
    double r_cut;      /* r_E: cutoff of LJ and DSF Coulomb, both shifted in value and slope */
    double r_split;    /* r_c: short-range part chi U, long-range part (1 - chi) U (Sec. 3.1) */
    double h_switch;   /* h: chi is a quintic step from 1 at r_c - h to 0 at r_c */
    double r_mid;      /* r_M: ring boundary (Sec. 3.1 ring technique); outside (r_c-h, r_E) = one ring */
    double dsf_alpha;  /* DSF damping (1/A) */
    double gamma;      /* Langevin friction (1/ps) */
    double temperature;/* K */
    double eps0;       /* jump parameter eps0 */
    int eps_mode;      /* 1: adaptive eps = eps0 |F_ij| (the paper's choice), 0: constant eps = eps0 */
    double skin;       /* list skin (A): lists are rebuilt when an atom moved more than skin/2 */
    double skin_outer; /* outer candidate skin (A, >= skin); it also fixes the order of the jump lists */
    int n_rings;       /* 0: rings from r_mid; 1..4: rings with edges r_c-h, ring_r[0..n_rings-2], r_E */
    double ring_r[3];  /* interior ring edges (A), strictly increasing inside (r_c-h, r_E); MD_EINVAL otherwise */
    int lj_long_mode;  /* 0: the long-range LJ part (1-chi) U_LJ jumps (BPS, J', Sec. 3.2);
                        * 1: it is deterministic in F0, as in the paper's GPU runs (Sec. 4):
                        * gradient modes 3 and 5 carry the whole LJ, mode 4 only (1-chi) Coulomb;
                        * 2: deterministic at the slow level (the paper's RESPA1 splits van der
                        * Waals into a short and a long range): modes 3 and 4 split LJ by chi as
                        * in mode 0, mode 5 (F0 of JUMP, BJAOAJB) adds the (1-chi) LJ part, mode 6
                        * holds it, and JUMP-RESPA / JUMP-RESPA1 kick it at their outer step.
                        * No J' in modes 1 and 2. */
    int coulomb_mode;  /* 0: damped shifted force Coulomb (DSF, dsf_alpha);
                        * 1: Ewald (Sec. 3.1 splits its real-space part like DSF): pair term
                        *    erfc(a r)/r cut at r_cut with a = dsf_alpha > 0, no shift; the
                        *    reciprocal part by smooth PME (cardinal B-splines of order pme_order
                        *    4, 6 or 8 (an odd order has |b(m)| = 0 at m = K/2 on even grids),
                        *    grid of K^3 points, K the smallest 2,3,5-smooth integer
                        *    >= max(box / pme_spacing, 2 pme_order)), the self energy
                        *    -C a / sqrt(pi) sum q^2 and, for excluded pairs, -C q_i q_j erf(a r)/r.
                        *    The reciprocal part is deterministic: it belongs to F0 (gradient
                        *    mode 5), to modes 0, 2 and 4, and alone to mode 6; JUMP-RESPA and
                        *    JUMP-RESPA1 kick it at their outer period (Sec. 2.3). */
    int pme_order;     /* B-spline order p (coulomb_mode 1) */
    double pme_spacing;/* target grid spacing (A, coulomb_mode 1) */
} md_system;

typedef struct {
    double ke, temperature;              /* kcal/mol, K (3N degrees of freedom) */
    double pe_bond, pe_angle, pe_lj, pe_coul;   /* full potential (no split), kcal/mol */
    int64_t step;                        /* innermost steps taken since md_set_system (+ md_set_state step) */
    int64_t jump_proposals, jump_accepts;        /* C' (electrostatic pair jumps) */
    int64_t bps_proposals, bps_accepts;          /* J' (LJ bounces) */
    int64_t sampler_attempts, list_rebuilds, outer_rebuilds, guarded_accepts;
    uint32_t error_flags;                /* MD_FLAG_* */
} md_obs;

/* Create a context on cfg->device. *out receives the handle. Errors:
 * MD_EINVAL (bad config), MD_ECUDA. */
int md_init(md_ctx** out, const md_config* cfg);

/* Copy one replica's system to the device, build its neighbour and jump
 * lists and reset its step counter to 0. replica in [0, max_replicas).
 * Errors: MD_EINVAL (sizes, box too small for r_cut + skin_outer, types),
 * MD_ENOMEM, MD_ECUDA. */
int md_set_system(md_ctx* ctx, int replica, const md_system* sys);

/* Overwrite positions and velocities of a replica (host pointers, 3n each)
 * and set its step counter. img (3n ints, may be NULL = zeros) are periodic
 * image counts. x_build / x_outer (may be NULL = x) are the positions at which
 * the lists and the outer candidate grid were last built; passing the values
 * from md_get_state makes a resumed run repeat an uninterrupted one bit for
 * bit. The values are taken as given: a non-finite position or velocity is
 * reported by the next step call as MD_ENONFINITE (the device check of the
 * A O A update), without a fault. Errors: MD_EINVAL (replica, NULL x or v),
 * MD_ENOSYSTEM, MD_ECUDA. */
int md_set_state(md_ctx* ctx, int replica, const double* x, const double* v, const int* img,
                 const double* x_build, const double* x_outer, int64_t step);

/* Integrators. Each advances every replica. dt in fs. Errors: MD_EINVAL,
 * MD_ENOSYSTEM, MD_ECUDA, and the sticky GPU errors (MD_EBOUND, MD_ELIMIT,
 * MD_EOVERFLOW, MD_ENONFINITE), checked once at the end of the call.
 *   baoab:        B A O A B on the full potential (Sec. 2.3, BAOAB).
 *   baoab_respa:  nonbonded kicks at Delta = n_inner dt around n_inner
 *                 bonded BAOAB steps (Sec. 2.3, RESPA).
 *   baoab_respa1: long-range (1-chi) pairs at Delta = n_outer kappa, short
 *                 chi pairs at kappa = m_mid dt, bonded at dt (RESPA1).
 *   jump:         C'(dt/2) J'(dt/2) A O A J'(dt/2) C'(dt/2), F_0 = bonded +
 *                 chi pairs, electrostatic (1-chi) part by pair jumps (C',
 *                 Alg. 4 with rings), LJ (1-chi) part by BPS (J', Alg. 5).
 *   jump_respa:   C'J' at Delta = n_inner dt around bonded inner steps.
 *   jump_respa1:  C'J' at kappa = m_mid dt around bonded inner steps; the
 *                 outer level of period n_outer kappa carries the slow
 *                 many-body force: the Ewald reciprocal part (coulomb_mode 1;
 *                 DSF electrostatics have none). jump_respa kicks it at
 *                 Delta = n_inner dt. */
int md_step_baoab(md_ctx* ctx, int64_t nsteps, double dt_fs);
int md_step_baoab_respa(md_ctx* ctx, int64_t n_outer, double dt_inner_fs, int n_inner);
int md_step_baoab_respa1(md_ctx* ctx, int64_t n_outer, double dt_inner_fs, int m_mid, int n_outer_ratio);
int md_step_jump(md_ctx* ctx, int64_t nsteps, double dt_fs);

/* The BJAOAJB splitting of Sec. 2.3 with the same jump mechanisms: B(dt/2)
 * with F0, the jump processes alone over dt/2 (Coulomb pair jumps with no
 * drift, then LJ bounces), A(dt/2) O(dt) A(dt/2), F0, LJ bounces, pair jumps,
 * B(dt/2). Same streams and counters as md_step_jump. */
int md_step_bjaoajb(md_ctx* ctx, int64_t nsteps, double dt_fs);
int md_step_jump_respa(md_ctx* ctx, int64_t n_outer, double dt_inner_fs, int n_inner);
int md_step_jump_respa1(md_ctx* ctx, int64_t n_outer, double dt_inner_fs, int m_mid, int n_outer_ratio);

/* Observables of one replica (synchronises the stream). */
int md_observables(md_ctx* ctx, int replica, md_obs* out);

/* Copy a replica's state to host buffers (3n each; any may be NULL). */
int md_get_state(md_ctx* ctx, int replica, double* x, double* v, int* img,
                 double* x_build, double* x_outer);

/* Gradient of one part of the potential at the current positions, into a
 * host buffer of 3n doubles. mode: 0 full, 1 bonded, 2 nonbonded full,
 * 3 nonbonded short (chi-weighted), 4 nonbonded long ((1-chi)-weighted),
 * 5 F_0 of JUMP (bonded + short), 6 the slow level of JUMP-RESPA(1): the Ewald
 * reciprocal part with the exclusion correction, plus the (1-chi) LJ part with
 * lj_long_mode 2 (zero with DSF and lj_long_mode 0 or 1). With coulomb_mode 1,
 * modes 0, 2, 4 and 5 include the reciprocal part. Uses the current lists (rebuilt first when an atom moved
 * more than skin/2). */
int md_gradient(md_ctx* ctx, int replica, int mode, double* host_grad);

/* One velocity phase at fixed positions, for testing the jump kernels: phase
 * 0 = C' (drift by the acceleration of gradient mode accel_mode, which the
 * call computes first), 1 = J'. tau2 in ps, s0 and half select the random
 * streams exactly as inside the integrators. Applies to every replica. */
int md_run_phase(md_ctx* ctx, int phase, double tau2_ps, int64_t s0, int half, int accel_mode);

/* Jump list of one atom: kind 0..3 ring 0..3 (inner to outer; rings past the
 * system's ring count are empty), 4 LJ. Writes up to cap
 * partner indices (local to the replica, in list order) into host_out and
 * returns the list length (or a negative error). */
int md_get_list(md_ctx* ctx, int replica, int kind, int atom, int* host_out, int cap);

/* Accepted-jump log (needs event_log_cap > 0): rows of 6 int64
 * (s, half, tag 2 = C' / 3 = J', atom, proposal index k, partner J), in no
 * particular order. Returns the number of rows written (<= cap); clear != 0
 * empties the log. */
int64_t md_get_events(md_ctx* ctx, int replica, int64_t* host_out6, int64_t cap, int clear);

/* Kernel launch accounting of this context. Classes (MD_PROFILE_CLASSES):
 * 0 pair force, 1 bonded force, 2 velocity phases (the C' and J' jump
 * kernels), 3 kicks and A-O-A updates, 4 list rebuild: cell grid, outer
 * candidates and flag reset, 5 bookkeeping (step counters, energies), 6 Ewald
 * reciprocal part (PME kernels; the cuFFT transforms are not counted),
 * 7 list rebuild: the inner list filter, 8 rate ordering of the atoms before
 * a mixed-mode C' phase. launches_out[MD_PROFILE_CLASSES] (may be NULL)
 * receives the cumulative number of kernels launched per class since md_init
 * (kernels replayed inside CUDA graphs included). enable = 1 starts timing
 * every launch group with CUDA events on the context's stream (graphs are
 * not used while timing is on), 0 stops it, -1 leaves it as it is;
 * ms_out[MD_PROFILE_CLASSES] (may be NULL) receives the accumulated device
 * time per class while timing was on (summed at the end of each md_step_*
 * call) and groups_out[MD_PROFILE_CLASSES] (may be NULL) the number of timed
 * launch groups. reset != 0 clears the times. */
#define MD_PROFILE_CLASSES 9
int md_profile(md_ctx* ctx, int enable, int reset, double* ms_out, int64_t* groups_out,
               int64_t* launches_out);

/* Nonbonded gradient without allocation.
 *
 * The paper has no counterpart: this is a service entry point for callers
 * that cannot allocate device memory. Examples are a host framework whose own
 * allocator has reserved the GPU's memory and forbids other allocations, and
 * a real-time loop that cannot afford the device-wide synchronisation that
 * cudaMalloc / cudaFree imply. Such callers pass their own device arrays for
 * inputs and output; the call itself allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).
 *
 * It computes, for one periodic cubic system, the gradient of the LJ + DSF
 * pair potential with weight 0 full, 1 short (chi U), 2 long ((1 - chi) U),
 * the same quantity as md_gradient modes 2, 3 and 4, in FP64, from a cell
 * grid built on every call. Pairs whose d_mol entries are equal are excluded
 * (d_mol may be NULL: no exclusions).
 *   d_x (3n doubles, A), d_charge (n doubles, e), d_type (n ints), d_mol
 *   (n ints or NULL), d_grad (3n doubles, output): device pointers of the
 *   current device; lj_eps, lj_sigma: host arrays of n_types^2 doubles.
 *   r_cut, r_split, h_switch, dsf_alpha: as in md_system; box >= 2 r_cut.
 *   cuda_stream: the stream the kernels run on (NULL = default stream).
 * Returns MD_OK or MD_EINVAL (null pointer, n_atoms outside
 * [1, MD_NOALLOC_MAX_ATOMS], more than MD_NOALLOC_MAX_CELLS cells of edge
 * >= r_cut, bad parameters) or MD_ECUDA; the message is md_last_error(NULL).
 *
 * The atoms of each cell are put in increasing index order before the pair
 * sums, so every call sums the pairs of an atom in the same order: two calls
 * on the same input return the same bits.
 *
 * Scratch: one static device array (about 2 MB, every GPU that loads the
 * library holds it until the process exits) shared by all calls. It keeps the
 * last call's contents; each call clears what must start at zero. Calls that
 * overlap on the GPU (different streams, or different host threads on the
 * same device) race on it and must be serialised by the caller. The first
 * call on a device looks up the array's device address with
 * cudaGetSymbolAddress (once per device, with that device current); make that
 * first call before any stream capture. */
#define MD_NOALLOC_MAX_ATOMS 131072
#define MD_NOALLOC_MAX_CELLS 32768
int md_nb_gradient_noalloc(const double* d_x, const double* d_charge, const int* d_type, const int* d_mol,
                           int n_atoms, double box, int n_types, const double* lj_eps, const double* lj_sigma,
                           double r_cut, double r_split, double h_switch, double dsf_alpha, int weight,
                           double* d_grad, void* cuda_stream);

/* Velocity record for spectra (Sec. 4: the velocity autocorrelation spectra
 * that show the resonances of the multiple-time-step integrators). From this
 * call on, every md_step_* call stores the velocities of all atoms of all
 * replicas after each innermost step, taken after the closing kicks and
 * phases of every level that ends at that step, until n_samples steps are
 * stored (later steps are not stored). Adjacent C' phases of JUMP and
 * JUMP-RESPA(1) then run as separate launches (same results). The record
 * holds n_samples x 3N values on the device (FP64 in MD_FP64, FP32 in
 * MD_MIXED). n_samples = 0 ends the record; md_set_system, md_set_state and a
 * new md_vacf_start end it too. Errors: MD_EINVAL, MD_ENOMEM, MD_ECUDA. */
int md_vacf_start(md_ctx* ctx, int64_t n_samples);

/* Mass-weighted velocity autocorrelation of one replica from the record:
 *   vacf_out[k] = (1 / (T - k)) sum_{t=0}^{T-1-k} sum_i m_i v_i(t) . v_i(t + k)
 * (amu A^2 / ps^2, 0 for k >= T), k < n_lags, T = samples stored (*n_stored;
 * 0 when nothing is recorded), computed on the device through FFTs of the
 * zero-padded series (Wiener-Khinchin, exact up to rounding); and its
 * Hann-windowed cosine transform
 *   spectrum_out[j] = C(0) + 2 sum_{k=1}^{K-1} w_k C(k) cos(pi j k / K),
 *   w_k = (1 + cos(pi k / K)) / 2, K = n_lags, j < K,
 * whose bin j is the frequency j / (2 K dt) for samples dt apart. Host
 * buffers of n_lags doubles; either may be NULL. Synchronises the stream. */
int md_vacf_get(md_ctx* ctx, int replica, int64_t n_lags, double* vacf_out, double* spectrum_out,
                int64_t* n_stored);

/* Release every device buffer and the context. */
int md_finalize(md_ctx* ctx);

/* Message of the last error on ctx (or of the last md_init failure when ctx
 * is NULL). Never NULL. */
const char* md_last_error(const md_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
