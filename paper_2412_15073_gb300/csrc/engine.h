// engine.h -- internal interface between the host engine (md_api.cu) and the
// kernel translation units of libmdjump.so. Not installed.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace mdj {

// launch classes of the accounting (md_profile): 0 pair force, 1 bonded, 2 velocity
// phases (C', J' kernels), 3 kicks and A-O-A, 4 cell grid and outer candidates of the
// list rebuild, 5 bookkeeping, 6 Ewald reciprocal (PME), 7 inner list filter,
// 8 rate ordering of the velocity phases
constexpr int NPROF = 9;

// Device pointers of one context, passed by value to every kernel. All atom
// arrays are concatenated over replicas (replica r owns [atom_off, atom_off+n)).
struct Dev {
    int N, R;
    const RepParams* P;
    const int* rep;                 // atom -> replica
    int* vorder;                    // visiting order of the velocity phases (grouped by jump rate)
    const int* vorder0;             // the order fixed at set-up (expected rates at the thermal speed)
    int *vkey, *vhist, *vofs;       // rate sort: bucket per atom, counts and offsets per (replica, bucket)
    // state (FP64 master copies)
    double *x, *v, *xb, *xo;        // positions, velocities, positions at list build / outer build
    int* img;                       // periodic image counts
    double *a0, *ab, *as, *al;      // accelerations: F0 (or full), bonded, short pairs, long pairs
    double* gout;                   // gradient output of md_gradient
    // scaled 32-bit coordinates (x, y, z) and the charge as float bits in w
    uint4* pos;
    // per-atom constants
    const double *mt, *isqmt, *q;   // m/418.4, 1/sqrt(m~), charge
    const double* nimt;             // -1/m~ (acceleration from gradient without an FP64 division per use)
    const int* type;
    const double *LY, *LLJ;         // rate bounds per atom: rings (n x MAX_RINGS), LJ
    const float *LYf, *LLJf;
    // bonded terms: per-atom items (kind | role << 4, term index)
    const int* bi_off;
    const int2* bitem;
    const int2* bond_ij;
    const double *bond_k, *bond_r0;
    const int4* ang;                // (end a, centre, end b, 0)
    const double *ang_k, *ang_t0;
    int nbond, nang;
    double* bterm;                  // per bond: gradient on its first atom (3)
    double* aterm;                  // per angle: gradients on its two ends (6)
    // exclusions (both directions)
    const int* ex_off;
    const int* ex_idx;
    // outer grid cells
    int *cell_start, *cell_cnt, *cell_atoms, *atom_cell, *cell_rep;
    int total_cells;
    // outer candidate list (global indices, ordered by (cell, j))
    uint32_t* olist;
    int* ocnt;
    int ocap;
    const uint16_t* shell_tab;      // [R][SHELL_BINS]
    // inner lists (packed entries)
    uint32_t* list[NKIND];
    int* lcnt[NKIND];
    int lcap[NKIND];
    // per replica
    int* flags;                     // [R][2]: inner rebuild, outer rebuild
    uint32_t* err;                  // [R]
    uint32_t* ovf;                  // [R] which capacity overflowed: bit = list kind, OVF_OUTER, OVF_CELL
    unsigned long long* cnt;        // [R][NCOUNT]
    double* energy;                 // [R][6]: bond, angle, lj, coul, ke, spare
    long long* step_base;           // [R]
    double* stepc;                  // [R][2]: exp(-gamma tau), sqrt((1 - exp(-2 gamma tau)) / beta)
    // smooth PME (Ewald replicas): fixed-point charge grid, real grid, spectrum, influence function
    unsigned long long* pme_qi;
    double* pme_q;
    double2* pme_spec;
    const double* pme_G;
    const float* pme_Gf;            // G in FP32 (mixed mode; pme_q and pme_spec then hold FP32 data)
    double* pme_e;                  // [R] reciprocal energy of the last md_observables
    int *pme_brick, *pme_slot, *pme_sorted;   // per atom: brick, slot in it; atoms ordered by brick
    int *pme_bcnt, *pme_bstart;     // per brick: atom count, first sorted position ([nbricks + 1])
    const int* pme_brick_rep;       // brick -> replica
    int pme_nbricks;
    // accepted-jump log
    long long* ev;
    unsigned long long* ev_n;
    long long ev_cap;
    int* qctr;                      // work counter of the queue-fed velocity-phase kernel
    long long* facc;                // [N][3] fixed-point pair sums of the half-list force kernels (kept at zero)
    int lj_long_mask;               // bit 0: some replica has lj_long_mode 1, bit 1: lj_long_mode 2
    const int* ib_start;            // blocks of whole bonded groups for the fused inner steps ([n_ib + 1])
    const int *ib_bond_off, *ib_bond;   // per block: its bonds (global term indices)
    const int *ib_ang_off, *ib_ang;     // per block: its angles
    const int* item_slot;           // per bonded item: slot of its term in its block's list
    int n_ib;                       // 0: the bonded groups do not allow the fused inner steps
    int lj_symmetric;               // every replica's LJ tables are symmetric (eps_ab = eps_ba, sigma_ab = sigma_ba)
    const int* lj_perm;             // [N] atoms with an LJ partner type, then the others (each ascending)
    // cluster tiles of the mixed-mode pair kernels (k_lists.cu builds them):
    // the atoms of each outer cell in clusters of TILE_CL, ordered by sub-cell
    // (Morton code) and index; replica r owns clusters [cl_roff[r], cl_roff[r + 1])
    int ncl_cap;
    const int* cl_roff;             // [R + 1]
    int* cl_start;                  // [total_cells] first cluster of each cell
    int* cl_atom;                   // [ncl_cap][TILE_CL] atom in each slot (-1: empty)
    int* cl_of;                     // [N] cluster of each atom
    int* cl_slot;                   // [N] its slot
    int* cl_cell;                   // [ncl_cap] cell of each cluster (-1: unused)
    uint4* cl_ref;                  // [ncl_cap] scaled position of slot 0
    int4 *cl_lo, *cl_hi;            // [ncl_cap] box of the members, scaled units relative to cl_ref
    // half lists of cluster pairs (J >= I) at the short (0) and full (1) list radii
    int* cpl_j[2];
    unsigned long long* cpl_mask[2];
    int* cpl_n[2];
    int cpl_cap[2];
    int tiles;                      // bit t: list t is kept up to date with the lists
};

constexpr int TILE_CL = 8;          // atoms per cluster

// can gradient mode `mode` run as half-list kernels? (full, short and long
// pair weights and the (1 - chi) LJ part alone (7); not the short weight of
// replicas whose short force also runs over the LJ list: lj_long_mode 1 in
// modes 3 and 5, lj_long_mode 2 in mode 5)
inline bool force_half_ok(const Dev& d, int mode)
{
    if (!d.lj_symmetric) return false;
    if (mode == 0 || mode == 2 || mode == 4 || mode == 7) return true;
    if (mode == 3) return !(d.lj_long_mask & 1);
    if (mode == 5) return d.lj_long_mask == 0;
    return false;
}

// ---- lists (k_lists.cu) ---------------------------------------------------------
void launch_check(const Dev& d, int force_inner, int force_outer, cudaStream_t s);
void launch_rebuild(const Dev& d, int kinds, int fp64, int keep_refs, int exact_outer,
                    int max_cells_per_rep, cudaStream_t s);
// the same chain in three parts: cells and outer candidates (5 kernels), the
// inner list filter (1 kernel, none when kinds is 0), the flag reset (1 kernel)
void launch_rebuild_cells(const Dev& d, int keep_refs, int exact_outer, cudaStream_t s);
void launch_rebuild_inner(const Dev& d, int kinds, int exact, cudaStream_t s);
void launch_rebuild_done(const Dev& d, cudaStream_t s);
void launch_late_lists(const Dev& d, int kinds, cudaStream_t s);
// cluster tiles: clusters of the outer cells (where an outer rebuild happens),
// then their boxes and the cluster-pair lists `tiles` (bit 0 short, bit 1 full)
// where an inner rebuild happens
void launch_tiles(const Dev& d, int tiles, cudaStream_t s);
void launch_tiles_late(const Dev& d, int tiles, cudaStream_t s);     // whatever the flags say
constexpr uint32_t OVF_TILE = 1u << 19;

// ---- forces and integrators (k_force.cu) -----------------------------------------
// mode: 0 full, 1 bonded, 2 nb full, 3 nb short, 4 nb long, 5 F0 (bonded + short),
// 7 the (1 - chi) LJ part alone (replicas with lj_long_mode 2, zero elsewhere)
// tpa: threads per atom (1, 2, 4, 8), | FORCE_HALF for the half-list kernels
// (mixed mode; the same values bit for bit, see k_force_half).
// returns the number of kernels launched
constexpr int FORCE_HALF = 16;
constexpr int FORCE_TILE = 32;      // the cluster-tile kernels (mixed mode; the same values bit for bit)
int launch_force(const Dev& d, int mode, double* out, int as_grad, int fp64, int tpa, cudaStream_t s);
void launch_kick(const Dev& d, const double* a, double h, cudaStream_t s);
void launch_kick2(const Dev& d, const double* a, double h, const double* b, double hb, cudaStream_t s);
// pre_a (may be null): the kick v += pre_h pre_a that precedes the A O A, in the same launch
void launch_aoa(const Dev& d, double tau, uint32_t s_off, int do_check, int fp64, cudaStream_t s,
                const double* pre_a = nullptr, double pre_h = 0.0);
// the bonded acceleration into out, then the kick v += kick_h out (one launch after the terms)
void launch_bonded_kick(const Dev& d, double* out, double kick_h, cudaStream_t s);
// nsteps inner steps B A O A [bonded] B at dt in one launch (blocks of whole
// bonded groups, d.n_ib > 0); the list check runs on the last step when check_last
constexpr int IB_MAX = 128;
constexpr int IB_TERMS = 256;       // bonds, and angles, of one block at most
void launch_inner_steps(const Dev& d, double dt, uint32_t s_off, int nsteps, int check_last, int fp64, cudaStream_t s);
void launch_energy(const Dev& d, cudaStream_t s);
void launch_advance(const Dev& d, long long nsteps, cudaStream_t s);

// ---- smooth PME (k_pme.cu) -----------------------------------------------------------------
// Reciprocal part of Ewald electrostatics for the replicas with coul_mode 1; the host runs
// the cuFFT transforms between these launches:
//   bin (atoms ordered by grid brick, 3 kernels) -> spread (per brick in shared memory, then
//   added to the fixed-point grid) -> tofloat (real grid; clears the fixed-point one)
//   -> forward FFT -> convolve (times G; energy != 0 also sums the energy into pme_e)
//   -> inverse FFT (potential grid) -> gather (per brick: gradient + exclusion correction
//   added to out, as -grad / m~ unless as_grad).
// spread and gather run once per B-spline order present (order: its replicas only).
void launch_pme_bin(const Dev& d, int fp64, cudaStream_t s);
void launch_pme_spread(const Dev& d, int order, int fp64, cudaStream_t s);
void launch_pme_tofloat(const Dev& d, long long total, int fp64, cudaStream_t s);
void launch_pme_convolve_grid(const Dev& d, int energy, long long max_spec, int fp64, cudaStream_t s);
void launch_pme_gather(const Dev& d, int order, double* out, int as_grad, int fp64, cudaStream_t s);
// exclusion-correction energy of each Ewald replica, added to d.energy[6 r + 3]
void launch_pme_excl_energy(const Dev& d, cudaStream_t s);

// ---- velocity record and autocorrelation (k_vacf.cu) -----------------------------------
// record: v into row step_base[0] + s_local - origin of buf (skipped outside [0, cap))
void launch_vacf_record(const Dev& d, void* buf, int fp64, long long origin, long long cap, uint32_t s_local,
                        cudaStream_t s);
// series s0 .. s0 + nb of a [T][n3] record into zero-padded [nb][2T] rows
void launch_vacf_gather(const void* buf, void* pad, int fp64, long long T, int n3, int s0, int nb, cudaStream_t s);
// P(j) += sum over the nb transformed series of m~ |X(j)|^2, j < nj
void launch_vacf_power(const void* X, int fp64, const double* mass_of_atom, int s0, int nb, long long nj, double* P,
                       cudaStream_t s);
void launch_vacf_to_complex(const double* P, double2* Z, long long nj, cudaStream_t s);
void launch_vacf_finish(const double* r, double* C, long long T, long long nlags, cudaStream_t s);
void launch_vacf_spectrum(const double* C, double* S, long long K, cudaStream_t s);

// ---- jumps (k_jump.cu) --------------------------------------------------------------
// order 0: C' then J' (first half of a step), 1: J' then C' (second half)
// variant of the mixed-mode C' kernel: occupancy targets of 3, 4, 5, 6 blocks
// of 128 threads. Every variant computes the same values. In mixed mode a C'
// phase first orders the atoms by their expected number of proposals, and
// J' runs as a kernel of its own.
constexpr int NVPHASE_VARIANTS = 4;
// launch variants of the mixed velocity phase, v in [0, NVPHASE_LAUNCH_VARIANTS):
// occupancy variant v % NVPHASE_VARIANTS; with the rate ordering of the current
// velocities ((v / NVPHASE_VARIANTS) % 2 == 0) or in the order fixed at set-up
// (where proposals are few, sorting costs more than it saves); one thread per
// atom (v < 2 NVPHASE_VARIANTS) or lanes fed from a queue of atoms (the rest)
constexpr int NVPHASE_LAUNCH_VARIANTS = 4 * NVPHASE_VARIANTS;
inline bool vphase_sorted(int v) { return (v / NVPHASE_VARIANTS) % 2 == 0; }
inline bool vphase_queue(int v) { return v >= 2 * NVPHASE_VARIANTS; }
constexpr int RATE_BUCKETS = 128;
// order 2 (mixed mode only): J' (s_off, half 1), C' (s_off, 1), C' (s_off2, 0), J' (s_off2, 0).
// hp0: host copy of the parameters of replica 0 when the context holds one
// replica (its constants then travel as a kernel parameter), else null.
// presorted: the caller has already run launch_rate_order for this phase (mixed
// mode, variants < NVPHASE_VARIANTS); otherwise the launch orders the atoms itself.
void launch_vphase(const Dev& d, const double* a, double tau2, uint32_t s_off, int half, int order,
                   int doC, int doJ, int fp64, int variant, cudaStream_t s, uint32_t s_off2, const RepParams* hp0,
                   int presorted = 0);
// same with an absolute stream index s0 (md_run_phase)
void launch_vphase_abs(const Dev& d, const double* a, double tau2, uint32_t s0, int half, int order,
                       int doC, int doJ, int fp64, int variant, cudaStream_t s, const RepParams* hp0,
                       int presorted = 0);
// visiting order of a mixed-mode C' phase over tau2_total (3 kernels)
void launch_rate_order(const Dev& d, const double* a, double tau2_total, cudaStream_t s);

}  // namespace mdj
