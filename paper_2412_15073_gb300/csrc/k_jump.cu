// k_jump.cu -- velocity phases at fixed positions: the C' step (pair jumps on
// the long-range electrostatics with the drift of the short-range
// acceleration, Algorithm 4 with adaptive eps and the ring technique of
// Sec. 3.1) and the J' step (BPS bounces on the long-range LJ part,
// Algorithm 5 of Sec. 3.2).
//
// One thread per atom: each atom's proposals form its own sequential Poisson
// thinning chain (the jumps of F_ij change v_i only, Sec. 3.1), so atoms run
// in parallel. Between proposals the velocity drifts as v0 + t a + J, with J
// the sum of the jumps so far; the phase ends at v0 + (tau/2) a + J.
#include <algorithm>

#include "engine.h"

namespace mdj {

namespace {

__device__ __forceinline__ double mimg(double t, const RepParams& P)
{
    return t - P.L * rint(t * P.invL);
}

// displacement x_i - x_j of a list entry, in the arithmetic type
template <typename T> struct JD;
template <> struct JD<float> {
    __device__ static void get(const Dev& d, const RepParams& P, int i, const uint4& pi, int j,
                               float& dx, float& dy, float& dz)
    {
        sdisp(pi, d.pos[j], P.sclf, P.sclf_lo, dx, dy, dz);
    }
};
template <> struct JD<double> {
    __device__ static void get(const Dev& d, const RepParams& P, int i, const uint4&, int j,
                               double& dx, double& dy, double& dz)
    {
        dx = mimg(d.x[3 * i] - d.x[3 * j], P);
        dy = mimg(d.x[3 * i + 1] - d.x[3 * j + 1], P);
        dz = mimg(d.x[3 * i + 2] - d.x[3 * j + 2], P);
    }
};

// radial derivative of (1 - chi) U per unit C q_i q_j (DSF) or of (1 - chi) U_LJ
template <typename T>
__device__ __forceinline__ T coul_long(const RepParams& P, T r)
{
    T u, du, c, dc;
    dsf<T>(P, r, T(1) / r, u, du);
    chi_and_slope<T>(r, T(P.sw), T(P.h), c, dc);
    return -dc * u + (T(1) - c) * du;
}

template <typename T>
__device__ __forceinline__ T lj_long(const RepParams& P, const LJPair& l, T r)
{
    T u, du, c, dc;
    ljsf<T>(P, l, r, T(1) / r, u, du);
    chi_and_slope<T>(r, T(P.sw), T(P.h), c, dc);
    return -dc * u + (T(1) - c) * du;
}

__device__ void log_event(const Dev& d, long long s0, int half, int tag, int rep, int atom, long long k, int J)
{
    if (d.ev_cap <= 0) return;
    const unsigned long long idx = atomicAdd(d.ev_n, 1ull);
    if ((long long)idx >= d.ev_cap) return;
    long long* e = d.ev + 6 * idx;
    e[0] = s0; e[1] = half; e[2] = tag | (rep << 8); e[3] = atom; e[4] = k; e[5] = J;
}

struct Tally {
    unsigned int cprop = 0, cacc = 0, jprop = 0, jacc = 0, satt = 0, guard = 0;
};

// acceptance probability of a C' proposal in FP64 from the FP64 positions
// (mixed mode only, when U is within 2e-6 of the FP32 value)
__device__ __noinline__ double cprime_p64(const Dev& d, const RepParams& P, int i, int J, int Y,
                             const double v0[3], const double a[3], double tprev, double t,
                             const float jac[3], double aa, double tau2)
{
    double vp[3], vt[3];
    for (int c = 0; c < 3; ++c) {
        vp[c] = v0[c] + tprev * a[c] + double(jac[c]);
        vt[c] = v0[c] + t * a[c] + double(jac[c]);
    }
    const double s = tau2 - tprev;
    const double vv = vp[0] * vp[0] + vp[1] * vp[1] + vp[2] * vp[2];
    const double va = vp[0] * a[0] + vp[1] * a[1] + vp[2] * a[2];
    const double B = sqrt(vv + s * s * aa + 2.0 * s * fmax(va, 0.0));
    const double mt = d.mt[i], beta = P.beta, eps0 = P.eps0;
    const double LY = d.LY[MAX_RINGS * i + Y];
    double dx = mimg(d.x[3 * i] - d.x[3 * J], P), dy = mimg(d.x[3 * i + 1] - d.x[3 * J + 1], P),
           dz = mimg(d.x[3 * i + 2] - d.x[3 * J + 2], P);
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (!(r >= P.edge[Y] && r < P.edge[Y + 1])) return 0.0;
    const double f = COULOMB * d.q[i] * d.q[J] * coul_long<double>(P, r) / r;
    const double gx = f * dx, gy = f * dy, gz = f * dz;
    const double gn = sqrt(gx * gx + gy * gy + gz * gz);
    if (!(gn > 0.0)) return 0.0;
    const double vg = vt[0] * gx + vt[1] * gy + vt[2] * gz;
    if (P.eps_mode == 1) {
        const double LamY = beta * LY * B + sqrt(beta / mt) / (eps0 * sqrt(2.0 * PI));
        const double eta = eps0 * sqrt(beta * mt) * vg;
        return sqrt(beta / mt) * theta<double>(eta) / eps0 / LamY;
    }
    const double eta = eps0 * sqrt(beta * mt) * vg / gn;
    return gn * theta<double>(eta) / (LY * (eps0 * sqrt(beta * mt) * B + 1.0 / sqrt(2.0 * PI)));
}

static_assert(MAX_RINGS == 4, "ring selection below is written for four ring slots");

// v[Y] for a ring index held in a register (selects instead of indexing local memory)
template <typename A>
__device__ __forceinline__ A ring_sel(const A (&v)[MAX_RINGS], int Y)
{
    return Y == 0 ? v[0] : (Y == 1 ? v[1] : (Y == 2 ? v[2] : v[3]));
}

// partner counts of the rings of atom i (0 for ring slots past the replica's count)
__device__ __forceinline__ int ring_counts(const Dev& d, const RepParams& P, int i, int (&N)[MAX_RINGS])
{
    int ntot = 0;
#pragma unroll
    for (int y = 0; y < MAX_RINGS; ++y) {
        N[y] = y < P.nr ? min(d.lcnt[L_R0 + y][i], d.lcap[L_R0 + y]) : 0;
        ntot += N[y];
    }
    return ntot;
}

// ring of a proposal: the first ring whose cumulative weight exceeds U Lam
// (ring Y with probability w_Y / Lam, Sec. 3.1 ring technique)
template <typename T>
__device__ __forceinline__ int ring_pick(const T (&w)[MAX_RINGS], T target, int nr)
{
    int Y = nr - 1;
    bool found = false;
    T cum = T(0);
#pragma unroll
    for (int y = 0; y < MAX_RINGS; ++y) {
        cum += w[y];
        if (!found && y < nr && target < cum) { Y = y; found = true; }
    }
    return Y;
}

// C' for atom i over tau2 (Algorithm 4, adaptive or constant eps, up to four rings)
template <typename T>
__device__ void cprime(const Dev& d, const RepParams& P, int i, int il, double v[3], const double a[3],
                       double tau2, uint32_t s0, int half, Tally& tl, uint32_t& err)
{
    int N[MAX_RINGS];
    if (ring_counts(d, P, i, N) == 0) {
        for (int c = 0; c < 3; ++c) v[c] += tau2 * a[c];
        return;
    }
    const T beta = T(P.beta), eps0 = T(P.eps0);
    const double mt64 = d.mt[i];
    const T mt = T(mt64);
    const T sbm = d_sqrt(beta * mt), sbom = d_sqrt(beta / mt);
    T LYv[MAX_RINGS];
#pragma unroll
    for (int y = 0; y < MAX_RINGS; ++y) LYv[y] = T(d.LY[MAX_RINGS * i + y]);
    const T qiC = T(COULOMB * d.q[i]);
    const bool adaptive = P.eps_mode == 1;
    const T c0 = adaptive ? sbom / (eps0 * T(2.5066282746310002)) : sbom / (T(2.5066282746310002) * eps0);
    const T ax = T(a[0]), ay = T(a[1]), az = T(a[2]);
    const T aa = ax * ax + ay * ay + az * az;
    const double aa64 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    const T T2 = T(tau2);
    const T vx0 = T(v[0]), vy0 = T(v[1]), vz0 = T(v[2]);
    const uint4 pi = sizeof(T) == 4 ? d.pos[i] : make_uint4(0, 0, 0, 0);
    T t = T(0);
    T jx = T(0), jy = T(0), jz = T(0);
    // velocity at time t: v0 + t a + J (the telescoped drift of Algorithm 4)
    T vx = vx0, vy = vy0, vz = vz0;
    uint32_t k = 0;
    for (;;) {
        const T s = T2 - t;
        const T vv = vx * vx + vy * vy + vz * vz;
        const T va = vx * ax + vy * ay + vz * az;
        const T B = d_sqrt(vv + s * s * aa + T(2) * s * (va > T(0) ? va : T(0)));
        T LamYv[MAX_RINGS], w[MAX_RINGS], Lam = T(0);
#pragma unroll
        for (int y = 0; y < MAX_RINGS; ++y) {
            LamYv[y] = adaptive ? beta * LYv[y] * B + c0 : LYv[y] * (beta * B + c0);
            w[y] = T(N[y]) * LamYv[y];
            Lam += w[y];
        }
        const U4 u = draw(P, uint32_t(il), s0, TAG_C, half, 0, k);
        const T Tn = -d_log(unif<T>(u.x)) / Lam;
        if (!(Lam > T(0)) || t + Tn > T2) break;
        const T tprev = t;
        t += Tn;
        vx = T(v[0]) + t * ax + jx;
        vy = T(v[1]) + t * ay + jy;
        vz = T(v[2]) + t * az + jz;
        if (sizeof(T) == 8) {   // FP64: the same sums as the definition, without rounding to float
            vx = T(v[0] + double(t) * a[0] + double(jx));
            vy = T(v[1] + double(t) * a[1] + double(jy));
            vz = T(v[2] + double(t) * a[2] + double(jz));
        }
        tl.cprop++;
        const int Y = ring_pick<T>(w, unif<T>(u.y) * Lam, P.nr);
        const uint32_t* row = d.list[L_R0 + Y] + (size_t)i * d.lcap[L_R0 + Y];
        // an empty ring only from an infinite bound (flagged as non-finite): the atom itself, outside every ring
        const uint32_t NY = uint32_t(ring_sel(N, Y));
        const int J = NY ? int(row[__umulhi(u.z, NY)]) : i;
        T dx, dy, dz;
        JD<T>::get(d, P, i, pi, J, dx, dy, dz);
        const T r = d_sqrt(dx * dx + dy * dy + dz * dz);
        const bool inside = r >= T(P.edge[Y]) && r < T(P.edge[Y + 1]);
        if (inside) {
            const T f = qiC * T(d.q[J]) * coul_long<T>(P, r) / r;
            const T gx = f * dx, gy = f * dy, gz = f * dz;
            const T gn = d_sqrt(gx * gx + gy * gy + gz * gz);
            if (gn > T(0)) {
                const T vg = vx * gx + vy * gy + vz * gz;
                const T LamY = ring_sel(LamYv, Y);
                T eps, eta, p;
                if (adaptive) {
                    eps = eps0 * gn;
                    eta = eps0 * sbm * vg;
                    p = sbom * theta<T>(eta) / eps0 / LamY;
                } else {
                    const T LY = ring_sel(LYv, Y);
                    eps = eps0;
                    eta = eps0 * sbm * vg / gn;
                    p = gn * theta<T>(eta) / (LY * (eps0 * sbm * B + T(0.3989422804014327)));
                }
                bool acc;
                if (sizeof(T) == 4 && fabs(double(unif<T>(u.w)) - double(p)) < 2e-6) {
                    const float jac[3] = {float(jx), float(jy), float(jz)};
                    const double p64 = cprime_p64(d, P, i, J, Y, v, a, double(tprev), double(t), jac,
                                                  aa64, tau2);
                    acc = unif<double>(u.w) <= p64;
                    if (p64 > 1.0) err |= F_BOUND;
                    tl.guard++;
                } else {
                    acc = unif<T>(u.w) <= p;
                    if (p > T(1) + (sizeof(T) == 4 ? T(P_TOL32) : T(0))) err |= F_BOUND;
                }
                if (acc) {
                    // G~ by rejection, streams (S, half, attempt, k)
                    T G = T(0);
                    int att = 0;
                    bool ok = false;
                    for (; att < SAMPLER_CAP && !ok; ++att) {
                        const U4 us = draw(P, uint32_t(il), s0, TAG_S, half, uint32_t(att), k);
                        ok = gtilde_attempt<T>(eta, us, G);
                    }
                    tl.satt += att;
                    if (!ok) { err |= F_LIMIT; G = T(0); }
                    const T coef = T(2) * eps / (sbm * (T(1) + eps * eps)) * (eta + G) / gn;
                    jx -= coef * gx; jy -= coef * gy; jz -= coef * gz;
                    vx -= coef * gx; vy -= coef * gy; vz -= coef * gz;
                    tl.cacc++;
                    log_event(d, (long long)s0, half, int(TAG_C), d.rep[i], il, k, J - P.atom_off);
                }
            }
        }
        ++k;
        if (k >= uint32_t(KMAX)) { err |= F_LIMIT; break; }
    }
    for (int c = 0; c < 3; ++c) v[c] += tau2 * a[c];
    v[0] += double(jx); v[1] += double(jy); v[2] += double(jz);
}

// J' for atom i over tau2 (Algorithm 5: Poisson(N beta |v| L tau/2)
// proposals as exponential arrivals, uniform partner, reflection)
template <typename T>
__device__ __noinline__ void jprime(const Dev& d, const RepParams& P, int i, int il, double v[3], double tau2,
                       uint32_t s0, int half, Tally& tl, uint32_t& err)
{
    const int N = min(d.lcnt[L_LJ][i], d.lcap[L_LJ]);
    if (N == 0) return;
    const double V64 = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const double Li64 = d.LLJ[i];
    if (!(V64 > 0.0) || !(Li64 > 0.0)) return;
    const uint32_t* row = d.list[L_LJ] + (size_t)i * d.lcap[L_LJ];
    const T V = T(V64), Li = T(Li64);
    const T Lam = T(N) * T(P.beta) * V * Li;
    const T T2 = T(tau2);
    const uint4 pi = sizeof(T) == 4 ? d.pos[i] : make_uint4(0, 0, 0, 0);
    const int ti = d.type[i];
    T t = T(0);
    uint32_t k = 0;
    for (;;) {
        const U4 u = draw(P, uint32_t(il), s0, TAG_J, half, 0, k);
        const T Tn = -d_log(unif<T>(u.x)) / Lam;
        if (t + Tn > T2) break;
        t += Tn;
        tl.jprop++;
        const int J = int(row[__umulhi(u.z, uint32_t(N))]);
        T dx, dy, dz;
        JD<T>::get(d, P, i, pi, J, dx, dy, dz);
        const T r = d_sqrt(dx * dx + dy * dy + dz * dz);
        if (r >= T(P.sw) && r < T(P.R)) {
            const T f = lj_long<T>(P, P.lj[ti * MAX_TYPES + d.type[J]], r) / r;
            const double gx = double(f * dx), gy = double(f * dy), gz = double(f * dz);
            const double vg = v[0] * gx + v[1] * gy + v[2] * gz;
            const double p = (vg > 0.0 ? vg : 0.0) / (V64 * Li64);
            if (p > 1.0) err |= F_BOUND;
            if (unif<double>(u.w) <= p) {
                const double gg = gx * gx + gy * gy + gz * gz;
                const double c = 2.0 * vg / gg;
                v[0] -= c * gx; v[1] -= c * gy; v[2] -= c * gz;
                tl.jacc++;
                log_event(d, (long long)s0, half, int(TAG_J), d.rep[i], il, k, J - P.atom_off);
            }
        }
        ++k;
        if (k >= uint32_t(KMAX)) { err |= F_LIMIT; break; }
    }
}

__device__ __forceinline__ void warp_add(unsigned long long* dst, unsigned int v32, bool uniform, int lane)
{
    unsigned long long v = v32;
    if (uniform) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0 && v) atomicAdd(dst, v);
    } else if (v) {
        atomicAdd(dst, v);
    }
}


// ---- mixed-mode fast path ----------------------------------------------------------
// G~ by rejection for one accepted proposal (streams (S, half, attempt, k))
__device__ __forceinline__ float sample_gtilde_f(const RepParams& P, uint32_t il, uint32_t s0, int half,
                                               uint32_t k, float eta, int* att_out, bool* ok_out)
{
    float G = 0.f;
    bool ok = false;
    int att = 0;
    for (; att < SAMPLER_CAP && !ok; ++att) {
        const U4 us = draw(P, il, s0, TAG_S, half, uint32_t(att), k);
        ok = gtilde_attempt<float>(eta, us, G);
    }
    *att_out = att;
    *ok_out = ok;
    return ok ? G : 0.f;
}

// radial derivative of (1 - chi) U_DSF per unit C q_i q_j in FP32, from
// per-replica constants held in registers (r >= r_c - h, the jump range)
__device__ __forceinline__ float coul_long_f(float r, float rinv, float alpha, float kexp, float eR, float fR,
                                             float R, float sw, float h)
{
    const float e = erfcf(alpha * r);
    const float g = kexp * expf(-alpha * alpha * r * r);
    const float du = -(e * rinv + g) * rinv + fR;
    if (r >= sw + h) return du;                 // chi = 0 past the switch
    const float u = e * rinv - eR + fR * (r - R);
    float c, dc;
    chi_and_slope<float>(r, sw, h, c, dc);
    return -dc * u + (1.f - c) * du;
}

// per-replica constants of the FP32 C' loop. A single-system launch passes
// them as a grid-constant kernel parameter (read straight from the constant
// bank, no registers); batched launches copy them from RepParams.
struct JC {
    float sc, sclo;                        // L / 2^32 as two floats
    uint32_t key0, key1;                   // Philox key (seed, replica)
    int nr, atom_off, adaptive, pad;
    float elo[MAX_RINGS], ehi[MAX_RINGS];  // ring y is [elo[y], ehi[y])
    float alpha, kexp, eR, fR, R, sw, h;   // DSF and switch
    float beta, eps0;
};

__host__ __device__ inline JC make_jc(const RepParams& P)
{
    JC c;
    c.sc = P.sclf; c.sclo = P.sclf_lo;
    c.key0 = P.seed; c.key1 = P.replica;
    c.nr = P.nr; c.atom_off = P.atom_off; c.adaptive = P.eps_mode == 1; c.pad = 0;
    for (int y = 0; y < MAX_RINGS; ++y) { c.elo[y] = P.edgef[y]; c.ehi[y] = P.edgef[y + 1]; }
    c.alpha = P.alphaf; c.kexp = P.kexpf; c.eR = P.eRf; c.fR = P.fRf;
    c.R = float(P.R); c.sw = float(P.sw); c.h = float(P.h);
    c.beta = float(P.beta); c.eps0 = float(P.eps0);
    return c;
}

// C' for atom i in FP32 (Algorithm 4, adaptive or constant eps, up to four rings),
// written as an initialisation and a step so that a lane can run a chain one
// proposal at a time (the queue kernel below interleaves the chains of the
// atoms a lane takes one after the other). Software-pipelined: right after
// proposal k is placed in time, the bound at the new state and the ring of
// proposal k+1 are computed and the list entry of k+1 is fetched; its
// position is fetched once proposal k is decided. If proposal k jumps, the
// bound and ring of k+1 are recomputed (and the entry refetched when the ring
// changed), so the sequence is that of Algorithm 4. Only B and Lam of the
// bound are kept; ring weights are recomputed from B.
struct CAtom {                             // constants of one atom's C' pass
    int i, il;
    int N[MAX_RINGS];
    float LYv[MAX_RINGS];
    uint4 pi;
    float qiC, sbm, sbom, c0, aa, T2;
    float3 v0, a;
    uint32_t s0, ctag;
    int half;
};
struct CChain {                            // running state of the chain
    float t, B, Lam, vx, vy, vz;
    float3 jv;
    uint32_t k, Jn;
    U4 u;
    int Yn;
    uint4 pjn;
};

// per-pair rate bound of ring y at speed bound B
__device__ __forceinline__ float c_lamy(const JC& c, const CAtom& A, float Ly, float B)
{
    return c.adaptive ? fmaf(c.beta * Ly, B, A.c0) : Ly * fmaf(c.beta, B, A.c0);
}

// bound at the current state: B and Lam = sum_y N_y Lam_y
__device__ __forceinline__ void c_bound(const JC& c, const CAtom& A, CChain& S)
{
    const float s = A.T2 - S.t;
    const float vv = S.vx * S.vx + S.vy * S.vy + S.vz * S.vz;
    const float va = S.vx * A.a.x + S.vy * A.a.y + S.vz * A.a.z;
    S.B = sqrtf(vv + s * s * A.aa + 2.f * s * fmaxf(va, 0.f));
    float Lam = 0.f;
#pragma unroll
    for (int y = 0; y < MAX_RINGS; ++y) Lam += float(A.N[y]) * c_lamy(c, A, A.LYv[y], S.B);
    S.Lam = Lam;
}

// ring of a proposal: first ring whose cumulative weight exceeds U Lam; a
// target that rounds up to Lam falls back to the outermost ring with weight
__device__ __forceinline__ int c_pick(const JC& c, const CAtom& A, const CChain& S, uint32_t uy)
{
    const float target = unif<float>(uy) * S.Lam;
    int Y = -1, last = 0;
    float cum = 0.f;
#pragma unroll
    for (int y = 0; y < MAX_RINGS; ++y) {
        const float wy = float(A.N[y]) * c_lamy(c, A, A.LYv[y], S.B);
        cum += wy;
        if (y < c.nr && A.N[y] > 0) last = y;     // for finite bounds: exactly the rings with weight
        if (Y < 0 && y < c.nr && target < cum) Y = y;
    }
    return Y < 0 ? last : Y;
}

// list entry of a proposal; an empty ring (reachable only from a non-finite
// state, which the A O A update flags) gives the atom itself: outside every ring
__device__ __forceinline__ uint32_t c_entry(const Dev& d, const CAtom& A, int Y, uint32_t uz)
{
    const uint32_t* row = d.list[L_R0 + Y] + (size_t)A.i * d.lcap[L_R0 + Y];
    const uint32_t NY = uint32_t(ring_sel(A.N, Y));
    return NY ? __ldg(row + __umulhi(uz, NY)) : uint32_t(A.i);
}

// constants of atom i's pass and the first proposal's draw, bound, ring and
// partner; returns false when the atom has no ring partner (no proposal)
__device__ __forceinline__ bool c_init(const Dev& d, const JC& c, int i, int il, float3 v0, float3 a, float T2,
                                       uint32_t s0, int half, CAtom& A, CChain& S)
{
    int ntot = 0;
#pragma unroll
    for (int y = 0; y < MAX_RINGS; ++y) {
        A.N[y] = y < c.nr ? min(d.lcnt[L_R0 + y][i], d.lcap[L_R0 + y]) : 0;
        ntot += A.N[y];
    }
    if (ntot == 0) return false;
    A.i = i; A.il = il; A.s0 = s0; A.half = half;
    A.ctag = (uint32_t(TAG_C) << 24) | (uint32_t(half) << 20);
    const float mt = float(d.mt[i]);
    A.sbm = sqrtf(c.beta * mt);
    A.sbom = sqrtf(c.beta / mt);
    const float4 ly4 = __ldg(reinterpret_cast<const float4*>(d.LYf) + i);
    A.LYv[0] = ly4.x; A.LYv[1] = ly4.y; A.LYv[2] = ly4.z; A.LYv[3] = ly4.w;
    A.pi = d.pos[i];
    A.qiC = float(COULOMB) * __uint_as_float(A.pi.w);
    A.c0 = A.sbom / (c.eps0 * 2.5066282746310002f);
    A.aa = a.x * a.x + a.y * a.y + a.z * a.z;
    A.T2 = T2; A.v0 = v0; A.a = a;
    S.t = 0.f;
    S.jv = make_float3(0.f, 0.f, 0.f);
    S.vx = v0.x; S.vy = v0.y; S.vz = v0.z;
    S.k = 0;
    S.u = philox(uint32_t(il), s0, A.ctag, 0, c.key0, c.key1);
    c_bound(c, A, S);
    S.Yn = c_pick(c, A, S, S.u.y);
    S.Jn = c_entry(d, A, S.Yn, S.u.z);
    S.pjn = __ldg(d.pos + S.Jn);
    return true;
}

// proposal k of the chain (its time, ring, partner and position are ready):
// place it, prepare proposal k+1, decide proposal k. Returns true when the
// pass has ended (the next arrival falls past tau/2, or the proposal cap)
__device__ __forceinline__ bool c_step(const Dev& d, const JC& c, const RepParams& P, const CAtom& A, CChain& S,
                                       Tally& tl, uint32_t& err)
{
    const float Tn = __fdividef(-__logf(unif<float>(S.u.x)), S.Lam);
    if (!(S.Lam > 0.f) || S.t + Tn > A.T2) return true;
    const float tprev = S.t;
    S.t += Tn;
    S.vx = fmaf(S.t, A.a.x, A.v0.x) + S.jv.x;
    S.vy = fmaf(S.t, A.a.y, A.v0.y) + S.jv.y;
    S.vz = fmaf(S.t, A.a.z, A.v0.z) + S.jv.z;
    tl.cprop++;
    const int Y = S.Yn;
    const int J = int(S.Jn);
    const uint4 pj = S.pjn;
    const float Bk = S.B;
    const uint32_t uacc = S.u.w;
    const uint32_t kk = S.k;
    ++S.k;
    // next proposal: draw, bound at the new state, ring and list entry
    S.u = philox(uint32_t(A.il), A.s0, A.ctag, S.k, c.key0, c.key1);
    c_bound(c, A, S);
    S.Yn = c_pick(c, A, S, S.u.y);
    S.Jn = c_entry(d, A, S.Yn, S.u.z);
    // decide proposal kk
    float dx, dy, dz;
    sdisp(A.pi, pj, c.sc, c.sclo, dx, dy, dz);
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    if (r >= ring_sel(c.elo, Y) && r < ring_sel(c.ehi, Y)) {
        const float f = A.qiC * __uint_as_float(pj.w) *
                        coul_long_f(r, rinv, c.alpha, c.kexp, c.eR, c.fR, c.R, c.sw, c.h) * rinv;
        const float gx = f * dx, gy = f * dy, gz = f * dz;
        const float gn = fabsf(f) * r;
        if (gn > 0.f) {
            const float vg = S.vx * gx + S.vy * gy + S.vz * gz;
            float eps, eta, p;
            if (c.adaptive) {
                eps = c.eps0 * gn;
                eta = c.eps0 * A.sbm * vg;
                p = __fdividef(A.sbom * theta<float>(eta), c.eps0 * c_lamy(c, A, ring_sel(A.LYv, Y), Bk));
            } else {
                eps = c.eps0;
                eta = __fdividef(c.eps0 * A.sbm * vg, gn);
                p = __fdividef(gn * theta<float>(eta), ring_sel(A.LYv, Y) * (c.eps0 * A.sbm * Bk + 0.3989422804014327f));
            }
            bool acc;
            const float U = unif<float>(uacc);
            if (fabsf(U - p) < 2e-6f) {
                const double v0d[3] = {d.v[3 * A.i], d.v[3 * A.i + 1], d.v[3 * A.i + 2]};
                const double ad[3] = {double(A.a.x), double(A.a.y), double(A.a.z)};
                const float jac[3] = {S.jv.x, S.jv.y, S.jv.z};
                const double p64 = cprime_p64(d, P, A.i, J, Y, v0d, ad, double(tprev), double(S.t), jac,
                                              double(A.aa), double(A.T2));
                acc = unif<double>(uacc) <= p64;
                if (p64 > 1.0) err |= F_BOUND;
                tl.guard++;
            } else {
                acc = U <= p;
                if (p > 1.f + P_TOL32) err |= F_BOUND;
            }
            if (acc) {
                int att;
                bool ok;
                const float G = sample_gtilde_f(P, uint32_t(A.il), A.s0, A.half, kk, eta, &att, &ok);
                tl.satt += att;
                if (!ok) err |= F_LIMIT;
                const float coef = 2.f * eps / (A.sbm * (1.f + eps * eps)) * (eta + G) / gn;
                S.jv.x -= coef * gx; S.jv.y -= coef * gy; S.jv.z -= coef * gz;
                S.vx -= coef * gx; S.vy -= coef * gy; S.vz -= coef * gz;
                tl.cacc++;
                log_event(d, (long long)A.s0, A.half, int(TAG_C), d.rep[A.i], A.il, kk, J - c.atom_off);
                // the velocity changed: bound and ring of the next proposal again
                c_bound(c, A, S);
                const int Y2 = c_pick(c, A, S, S.u.y);
                if (Y2 != S.Yn) { S.Yn = Y2; S.Jn = c_entry(d, A, S.Yn, S.u.z); }
            }
        }
    }
    S.pjn = __ldg(d.pos + S.Jn);
    if (S.k >= uint32_t(KMAX)) { err |= F_LIMIT; return true; }
    return false;
}

// C' for atom i in FP32: the whole chain in one loop; jv receives the sum of the jumps
__device__ __forceinline__ void cprime_f(const Dev& d, const JC& c, const RepParams& P, int i, int il, float3& jv,
                                         const float3 v0, const float3 a, float T2, uint32_t s0, int half,
                                         Tally& tl, uint32_t& err)
{
    CAtom A;
    CChain S;
    if (!c_init(d, c, i, il, v0, a, T2, s0, half, A, S)) return;
    while (!c_step(d, c, P, A, S, tl, err)) {}
    jv = S.jv;
}

// mixed-mode velocity phase; threads visit atoms in the order vorder (atoms
// ordered by expected number of proposals so that the lanes of a warp do
// similar work). jmode places the J' phases (LJ bounces) around the C'
// passes: 0 none, 1 after (s_off, half), 2 before (s_off, half), 3 before
// (s_off, half) and after (s_off2, 0).
// npass = 2 runs two consecutive C' phases at the same positions: the second
// half of the step at s_off (half 1) and the first half of the next step at
// s_off2 (half 0), which are adjacent in the C'J'AOAJ'C' sequence when no J'
// acts between them (the J' phases of the two steps run before and after).
template <int MINB, bool SINGLE>
__global__ void __launch_bounds__(128, MINB) k_cphase_f(Dev d, const __grid_constant__ JC jc0, const double* a,
                                                        double tau2, uint32_t s_off, int s_abs, int half, int npass,
                                                        uint32_t s_off2, int jmode)
{
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = t0 < d.N;
    const int i = d.vorder[live ? t0 : d.N - 1];
    const int r = d.rep[i];
    const RepParams& P = d.P[r];
    Tally tl;
    uint32_t err = 0;
    if (live) {
        const int il = i - P.atom_off;
        const uint32_t sb = s_abs ? 0u : uint32_t(d.step_base[r]);
        double v[3] = {d.v[3 * i], d.v[3 * i + 1], d.v[3 * i + 2]};
        double ad[3] = {a ? a[3 * i] : 0.0, a ? a[3 * i + 1] : 0.0, a ? a[3 * i + 2] : 0.0};
        if ((jmode & 2) && P.lj_jump) jprime<float>(d, P, i, il, v, tau2, sb + s_off, half, tl, err);
        for (int pass = 0; pass < npass; ++pass) {
            const uint32_t s0 = sb + (pass ? s_off2 : s_off);
            const int hp = pass ? 0 : half;
            float3 jv = make_float3(0.f, 0.f, 0.f);
            if (P.rings_on) {
                const float3 v0 = make_float3(float(v[0]), float(v[1]), float(v[2]));
                const float3 af = make_float3(float(ad[0]), float(ad[1]), float(ad[2]));
                // the FP64 guard of an acceptance reads the velocity at the start of the pass
                d.v[3 * i] = v[0]; d.v[3 * i + 1] = v[1]; d.v[3 * i + 2] = v[2];
                if (SINGLE) {
                    cprime_f(d, jc0, P, i, il, jv, v0, af, float(tau2), s0, hp, tl, err);
                } else {
                    const JC jc = make_jc(P);
                    cprime_f(d, jc, P, i, il, jv, v0, af, float(tau2), s0, hp, tl, err);
                }
                // the FP64 velocity and acceleration come back from memory after the
                // chain instead of occupying registers during it
                v[0] = d.v[3 * i]; v[1] = d.v[3 * i + 1]; v[2] = d.v[3 * i + 2];
                ad[0] = a ? a[3 * i] : 0.0; ad[1] = a ? a[3 * i + 1] : 0.0; ad[2] = a ? a[3 * i + 2] : 0.0;
            }
            // FP64 end of the phase: (v0 + (tau/2) a) + sum of the jumps; the
            // first sum rounds like a B kick, so a phase without jumps is one
            v[0] = fma(tau2, ad[0], v[0]) + double(jv.x);
            v[1] = fma(tau2, ad[1], v[1]) + double(jv.y);
            v[2] = fma(tau2, ad[2], v[2]) + double(jv.z);
        }
        if (jmode & 1 && P.lj_jump)
            jprime<float>(d, P, i, il, v, tau2, sb + (jmode == 3 ? s_off2 : s_off), jmode == 3 ? 0 : half, tl, err);
        d.v[3 * i] = v[0]; d.v[3 * i + 1] = v[1]; d.v[3 * i + 2] = v[2];
        if (err) atomicOr(&d.err[r], err);
    }
    const int lane = threadIdx.x & 31;
    const int r0 = __shfl_sync(0xffffffffu, r, 0);
    const bool uniform = __all_sync(0xffffffffu, r == r0);
    unsigned long long* C = d.cnt + (size_t)r * NCOUNT;
    warp_add(&C[C_CPROP], tl.cprop, uniform, lane);
    warp_add(&C[C_CACC], tl.cacc, uniform, lane);
    warp_add(&C[C_SATT], tl.satt, uniform, lane);
    warp_add(&C[C_GUARD], tl.guard, uniform, lane);
    warp_add(&C[C_JPROP], tl.jprop, uniform, lane);
    warp_add(&C[C_JACC], tl.jacc, uniform, lane);
}

// The same velocity phase with lanes fed from a queue. In the kernel above a
// warp runs 32 chains to the end of the longest one: the Poisson counts of
// the 32 atoms differ even when their expected counts match, so lanes idle.
// Here every lane runs one proposal per loop turn, and a lane whose atom is
// finished (J' before, its C' passes, J' after) takes the next atom of the
// visiting order from a warp pool refilled 32 atoms at a time from a global
// counter (qctr, zero at launch). Each atom's chain is the same sequence of
// draws and decisions as above, so the results are identical; only the
// assignment of atoms to lanes differs. Counters are flushed whenever a lane
// moves to another replica (the order groups atoms by replica).
template <int MINB, bool SINGLE>
__global__ void __launch_bounds__(128, MINB) k_cphase_q(Dev d, const __grid_constant__ JC jc0, const double* a,
                                                        double tau2, uint32_t s_off, int s_abs, int half, int npass,
                                                        uint32_t s_off2, int jmode, int* qctr)
{
    const int lane = threadIdx.x & 31;
    const unsigned lower = (1u << lane) - 1u;
    int pool_base = 0, pool_left = 0;          // warp-uniform
    bool drained = false;                      // warp-uniform
    int i = -1, pass = 0, tr = -1;             // atom, pass, replica of the tallied work
    bool chain = false;                        // the current pass has been set up
    bool live = false;                         // ... and has proposals to run
    double v[3] = {0.0, 0.0, 0.0}, ad[3] = {0.0, 0.0, 0.0};
    JC jcl{};
    CAtom A;
    CChain S;
    Tally tl;
    uint32_t err = 0;
    const RepParams* P = d.P;
    auto flush = [&](int r) {
        unsigned long long* C = d.cnt + (size_t)r * NCOUNT;
        if (tl.cprop) atomicAdd(&C[C_CPROP], (unsigned long long)tl.cprop);
        if (tl.cacc) atomicAdd(&C[C_CACC], (unsigned long long)tl.cacc);
        if (tl.satt) atomicAdd(&C[C_SATT], (unsigned long long)tl.satt);
        if (tl.guard) atomicAdd(&C[C_GUARD], (unsigned long long)tl.guard);
        if (tl.jprop) atomicAdd(&C[C_JPROP], (unsigned long long)tl.jprop);
        if (tl.jacc) atomicAdd(&C[C_JACC], (unsigned long long)tl.jacc);
        tl = Tally();
    };
    for (;;) {
        // idle lanes take the next atoms of the order
        unsigned need = __ballot_sync(0xffffffffu, i < 0);
        while (need && !drained) {
            if (pool_left == 0) {
                int b = 0;
                if (lane == 0) b = atomicAdd(qctr, 32);
                b = __shfl_sync(0xffffffffu, b, 0);
                pool_base = b;
                pool_left = b < d.N ? min(32, d.N - b) : 0;
                if (pool_left == 0) { drained = true; break; }
            }
            const int take = min(__popc(need), pool_left);
            const int rank = __popc(need & lower);
            if (((need >> lane) & 1u) && rank < take) i = d.vorder[pool_base + rank];
            pool_base += take;
            pool_left -= take;
            need = __ballot_sync(0xffffffffu, i < 0);
        }
        if (!__any_sync(0xffffffffu, i >= 0)) break;
        if (i >= 0 && !chain) {
            // a new atom (pass 0), or the next pass of the current one
            const int r = d.rep[i];
            P = d.P + r;
            const int il = i - P->atom_off;
            const uint32_t sb = s_abs ? 0u : uint32_t(d.step_base[r]);
            if (pass == 0) {
                if (tr != r) {
                    if (tr >= 0) flush(tr);
                    tr = r;
                }
                v[0] = d.v[3 * i]; v[1] = d.v[3 * i + 1]; v[2] = d.v[3 * i + 2];
                ad[0] = a ? a[3 * i] : 0.0; ad[1] = a ? a[3 * i + 1] : 0.0; ad[2] = a ? a[3 * i + 2] : 0.0;
                if ((jmode & 2) && P->lj_jump) jprime<float>(d, *P, i, il, v, tau2, sb + s_off, half, tl, err);
                if (!SINGLE) jcl = make_jc(*P);
            }
            const uint32_t s0 = sb + (pass ? s_off2 : s_off);
            const int hp = pass ? 0 : half;
            live = false;
            if (P->rings_on) {
                // the FP64 guard of an acceptance reads the velocity at the start of the pass
                d.v[3 * i] = v[0]; d.v[3 * i + 1] = v[1]; d.v[3 * i + 2] = v[2];
                const float3 v0 = make_float3(float(v[0]), float(v[1]), float(v[2]));
                const float3 af = make_float3(float(ad[0]), float(ad[1]), float(ad[2]));
                live = c_init(d, SINGLE ? jc0 : jcl, i, il, v0, af, float(tau2), s0, hp, A, S);
            }
            if (!live) S.jv = make_float3(0.f, 0.f, 0.f);    // no partner: the pass is a plain drift
            chain = true;
        }
        bool ended = false;
        if (i >= 0) ended = !live || c_step(d, SINGLE ? jc0 : jcl, *P, A, S, tl, err);
        if (ended) {
            // FP64 end of the pass: (v0 + (tau/2) a) + sum of the jumps
            v[0] = fma(tau2, ad[0], v[0]) + double(S.jv.x);
            v[1] = fma(tau2, ad[1], v[1]) + double(S.jv.y);
            v[2] = fma(tau2, ad[2], v[2]) + double(S.jv.z);
            chain = false;
            if (++pass >= npass) {
                const int r = d.rep[i];
                if (jmode & 1 && P->lj_jump) {
                    const uint32_t sb = s_abs ? 0u : uint32_t(d.step_base[r]);
                    jprime<float>(d, *P, i, i - P->atom_off, v, tau2, sb + (jmode == 3 ? s_off2 : s_off),
                                  jmode == 3 ? 0 : half, tl, err);
                }
                d.v[3 * i] = v[0]; d.v[3 * i + 1] = v[1]; d.v[3 * i + 2] = v[2];
                if (err) { atomicOr(&d.err[r], err); err = 0; }
                i = -1;
                pass = 0;
            }
        }
    }
    // counters: one reduction per warp when its lanes' last work was on one replica
    const unsigned has = __ballot_sync(0xffffffffu, tr >= 0);
    if (!has) return;
    const int t0 = __shfl_sync(0xffffffffu, tr, __ffs(has) - 1);
    if (__all_sync(0xffffffffu, tr == t0 || tr < 0)) {
        unsigned long long* C = d.cnt + (size_t)t0 * NCOUNT;
        warp_add(&C[C_CPROP], tl.cprop, true, lane);
        warp_add(&C[C_CACC], tl.cacc, true, lane);
        warp_add(&C[C_SATT], tl.satt, true, lane);
        warp_add(&C[C_GUARD], tl.guard, true, lane);
        warp_add(&C[C_JPROP], tl.jprop, true, lane);
        warp_add(&C[C_JACC], tl.jacc, true, lane);
    } else if (tr >= 0) {
        flush(tr);
    }
}

// mixed-mode J' phase: one thread per atom (BPS bounces, FP64 velocity)
__global__ void __launch_bounds__(128) k_jphase_f(Dev d, double tau2, uint32_t s_off, int s_abs, int half)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < d.N;
    const int ic = live ? i : d.N - 1;
    const int r = d.rep[ic];
    const RepParams& P = d.P[r];
    Tally tl;
    uint32_t err = 0;
    if (live && P.lj_jump) {
        const uint32_t s0 = (s_abs ? 0u : uint32_t(d.step_base[r])) + s_off;
        double v[3] = {d.v[3 * i], d.v[3 * i + 1], d.v[3 * i + 2]};
        jprime<float>(d, P, i, i - P.atom_off, v, tau2, s0, half, tl, err);
        d.v[3 * i] = v[0]; d.v[3 * i + 1] = v[1]; d.v[3 * i + 2] = v[2];
        if (err) atomicOr(&d.err[r], err);
    }
    const int lane = threadIdx.x & 31;
    const int r0 = __shfl_sync(0xffffffffu, r, 0);
    const bool uniform = __all_sync(0xffffffffu, r == r0);
    unsigned long long* C = d.cnt + (size_t)r * NCOUNT;
    warp_add(&C[C_JPROP], tl.jprop, uniform, lane);
    warp_add(&C[C_JACC], tl.jacc, uniform, lane);
}

template <typename T>
__global__ void __launch_bounds__(128) k_vphase(Dev d, const double* a, double tau2, uint32_t s_off, int s_abs,
                                                int half, int order, int doC, int doJ)
{
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i0 < d.N;
    const int i = live ? i0 : d.N - 1;
    const int r = d.rep[i];
    const RepParams& P = d.P[r];
    Tally tl;
    uint32_t err = 0;
    if (live) {
        const uint32_t s0 = (s_abs ? 0u : uint32_t(d.step_base[r])) + s_off;
        const int il = i - P.atom_off;
        double v[3] = {d.v[3 * i], d.v[3 * i + 1], d.v[3 * i + 2]};
        double acc[3] = {0, 0, 0};
        if (a) { acc[0] = a[3 * i]; acc[1] = a[3 * i + 1]; acc[2] = a[3 * i + 2]; }
        const bool c_on = doC && P.rings_on;
        const bool j_on = doJ && P.lj_jump;
        for (int step = 0; step < 2; ++step) {
            const bool isC = (order == 0) ? step == 0 : step == 1;
            if (isC) {
                if (doC) {
                    if (c_on) cprime<T>(d, P, i, il, v, acc, tau2, s0, half, tl, err);
                    else for (int c = 0; c < 3; ++c) v[c] += tau2 * acc[c];
                }
            } else if (j_on) {
                jprime<T>(d, P, i, il, v, tau2, s0, half, tl, err);
            }
        }
        d.v[3 * i] = v[0]; d.v[3 * i + 1] = v[1]; d.v[3 * i + 2] = v[2];
        if (err) atomicOr(&d.err[r], err);
    }
    const int lane = threadIdx.x & 31;
    const int r0 = __shfl_sync(0xffffffffu, r, 0);
    const bool uniform = __all_sync(0xffffffffu, r == r0);
    unsigned long long* C = d.cnt + (size_t)r * NCOUNT;
    warp_add(&C[C_CPROP], tl.cprop, uniform, lane);
    warp_add(&C[C_CACC], tl.cacc, uniform, lane);
    warp_add(&C[C_JPROP], tl.jprop, uniform, lane);
    warp_add(&C[C_JACC], tl.jacc, uniform, lane);
    warp_add(&C[C_SATT], tl.satt, uniform, lane);
    warp_add(&C[C_GUARD], tl.guard, uniform, lane);
}

// expected number of C' proposals of atom i in the coming phase (the bound
// Lam at its start times tau/2), as a bucket; high rates get low keys
__global__ void k_rate_key(Dev d, const double* a, double tau2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const int r = d.rep[i];
    const RepParams& P = d.P[r];
    int N[MAX_RINGS];
    float mu = 0.f;
    if (P.rings_on && ring_counts(d, P, i, N) > 0) {
        const float vx = float(d.v[3 * i]), vy = float(d.v[3 * i + 1]), vz = float(d.v[3 * i + 2]);
        const float ax = a ? float(a[3 * i]) : 0.f, ay = a ? float(a[3 * i + 1]) : 0.f, az = a ? float(a[3 * i + 2]) : 0.f;
        const float s = float(tau2);
        const float va = vx * ax + vy * ay + vz * az;
        const float B = sqrtf(vx * vx + vy * vy + vz * vz + s * s * (ax * ax + ay * ay + az * az) + 2.f * s * fmaxf(va, 0.f));
        const float beta = float(P.beta), mt = float(d.mt[i]);
        const float c0 = sqrtf(beta / mt) / (float(P.eps0) * 2.5066282746310002f);
        const float4 ly = __ldg(reinterpret_cast<const float4*>(d.LYf) + i);
        const float LYv[MAX_RINGS] = {ly.x, ly.y, ly.z, ly.w};
        float lam = 0.f;
#pragma unroll
        for (int y = 0; y < MAX_RINGS; ++y)
            lam += float(N[y]) * (P.eps_mode == 1 ? beta * LYv[y] * B + c0 : LYv[y] * (beta * B + c0));
        mu = lam * s;
    }
    // a non-finite velocity (flagged by the A O A update) gives mu = NaN: bucket 0
    const int b = mu > 0.f ? min(RATE_BUCKETS - 1, int(mu * 0.25f)) : 0;
    const int key = r * RATE_BUCKETS + (RATE_BUCKETS - 1 - b);
    d.vkey[i] = key;
    // one atomic per distinct key in the warp
    const unsigned peers = __match_any_sync(__activemask(), key);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&d.vhist[key], __popc(peers));
}

// exclusive scan of the bucket counts into offsets (one block); clears the counts
__global__ void __launch_bounds__(1024) k_rate_scan(Dev d)
{
    __shared__ int warp_tot[32];
    __shared__ int carry;
    const int nk = d.R * RATE_BUCKETS;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nk; base += 1024) {
        const int k = base + threadIdx.x;
        const int c = k < nk ? d.vhist[k] : 0;
        int x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        const int before = carry + (wid ? warp_tot[wid - 1] : 0) + x - c;
        if (k < nk) { d.vofs[k] = before; d.vhist[k] = 0; }
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + c;
        __syncthreads();
    }
}

__global__ void k_rate_scatter(Dev d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const int key = d.vkey[i];
    const unsigned peers = __match_any_sync(__activemask(), key);
    const int lane = threadIdx.x & 31, lead = __ffs(peers) - 1;
    int base = 0;
    if (lane == lead) base = atomicAdd(&d.vofs[key], __popc(peers));
    base = __shfl_sync(peers, base, lead);
    d.vorder[base + __popc(peers & ((1u << lane) - 1u))] = i;
}

}  // namespace

// visiting order of a mixed-mode C' phase: atoms by replica, then by their
// expected number of proposals (descending), so that the lanes of a warp run
// chains of similar length. The order within a bucket does not matter: each
// atom's chain depends on its own counter-based draws only.
static void rate_order(const Dev& d, const double* a, double tau2, cudaStream_t st)
{
    const int nb = (d.N + 255) / 256;
    k_rate_key<<<nb, 256, 0, st>>>(d, a, tau2);
    k_rate_scan<<<1, 1024, 0, st>>>(d);
    k_rate_scatter<<<nb, 256, 0, st>>>(d);
}

// resident blocks of a queue kernel over the whole GPU (the grid of a
// persistent launch), at most the blocks a plain launch would take
template <int MINB, bool SINGLE>
static int queue_blocks()
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cphase_q<MINB, SINGLE>, 128, 0);
    return std::max(1, sms * std::max(per, 1));
}

static int queue_grid(int occ, bool single, int nb)
{
    static int cache[2][NVPHASE_VARIANTS] = {};
    int& g = cache[single ? 1 : 0][occ];
    if (!g) {
        switch (occ) {
        case 1: g = single ? queue_blocks<4, true>() : queue_blocks<4, false>(); break;
        case 2: g = single ? queue_blocks<5, true>() : queue_blocks<5, false>(); break;
        case 3: g = single ? queue_blocks<6, true>() : queue_blocks<6, false>(); break;
        default: g = single ? queue_blocks<3, true>() : queue_blocks<3, false>(); break;
        }
    }
    return std::min(g, nb);
}

void launch_rate_order(const Dev& d, const double* a, double tau2_total, cudaStream_t st)
{
    rate_order(d, a, tau2_total, st);
}

static void vphase_any(const Dev& d, const double* a, double tau2, uint32_t s, uint32_t s2, int s_abs, int half,
                       int order, int doC, int doJ, int fp64, int variant, cudaStream_t st, const RepParams* hp0,
                       int presorted)
{
    const int nb = (d.N + 127) / 128;
    if (fp64) {
        k_vphase<double><<<nb, 128, 0, st>>>(d, a, tau2, s, s_abs, half, order, doC, doJ);
        return;
    }
    // order 0: C' then J'; 1: J' then C'; 2: J' (s, 1), C' (s, 1), C' (s2, 0), J' (s2, 0)
    if (!doC) {
        if (doJ) k_jphase_f<<<(d.N + 127) / 128, 128, 0, st>>>(d, tau2, s, s_abs, half);
        return;
    }
    const int npass = order == 2 ? 2 : 1;
    const int jmode = !doJ ? 0 : (order == 0 ? 1 : (order == 1 ? 2 : 3));
    // any visiting order gives the same values: each atom's chain depends on its own draws
    Dev dv = d;
    if (vphase_sorted(variant)) {
        if (!presorted) rate_order(d, a, tau2 * npass, st);
    } else {
        dv.vorder = const_cast<int*>(d.vorder0);
    }
    const bool queue = vphase_queue(variant);
    const int occ = variant % NVPHASE_VARIANTS;
    const JC jc = hp0 ? make_jc(*hp0) : JC{};
    if (queue) {
        cudaMemsetAsync(d.qctr, 0, sizeof(int), st);
        const int g = queue_grid(occ, hp0 != nullptr, nb);
        if (hp0) {
            switch (occ) {
            case 1: k_cphase_q<4, true><<<g, 128, 0, st>>>(dv, jc, a, tau2, s, s_abs, half, npass, s2, jmode, d.qctr); break;
            case 2: k_cphase_q<5, true><<<g, 128, 0, st>>>(dv, jc, a, tau2, s, s_abs, half, npass, s2, jmode, d.qctr); break;
            case 3: k_cphase_q<6, true><<<g, 128, 0, st>>>(dv, jc, a, tau2, s, s_abs, half, npass, s2, jmode, d.qctr); break;
            default: k_cphase_q<3, true><<<g, 128, 0, st>>>(dv, jc, a, tau2, s, s_abs, half, npass, s2, jmode, d.qctr); break;
            }
        } else {
            switch (occ) {
            case 1: k_cphase_q<4, false><<<g, 128, 0, st>>>(dv, jc, a, tau2, s, s_abs, half, npass, s2, jmode, d.qctr); break;
            case 2: k_cphase_q<5, false><<<g, 128, 0, st>>>(dv, jc, a, tau2, s, s_abs, half, npass, s2, jmode, d.qctr); break;
            case 3: k_cphase_q<6, false><<<g, 128, 0, st>>>(dv, jc, a, tau2, s, s_abs, half, npass, s2, jmode, d.qctr); break;
            default: k_cphase_q<3, false><<<g, 128, 0, st>>>(dv, jc, a, tau2, s, s_abs, half, npass, s2, jmode, d.qctr); break;
            }
        }
        return;
    }
    if (hp0) {
        switch (occ) {
        case 1: k_cphase_f<4, true><<<nb, 128, 0, st>>>(dv, jc, a, tau2, s, s_abs, half, npass, s2, jmode); break;
        case 2: k_cphase_f<5, true><<<nb, 128, 0, st>>>(dv, jc, a, tau2, s, s_abs, half, npass, s2, jmode); break;
        case 3: k_cphase_f<6, true><<<nb, 128, 0, st>>>(dv, jc, a, tau2, s, s_abs, half, npass, s2, jmode); break;
        default: k_cphase_f<3, true><<<nb, 128, 0, st>>>(dv, jc, a, tau2, s, s_abs, half, npass, s2, jmode); break;
        }
    } else {
        switch (occ) {
        case 1: k_cphase_f<4, false><<<nb, 128, 0, st>>>(dv, jc, a, tau2, s, s_abs, half, npass, s2, jmode); break;
        case 2: k_cphase_f<5, false><<<nb, 128, 0, st>>>(dv, jc, a, tau2, s, s_abs, half, npass, s2, jmode); break;
        case 3: k_cphase_f<6, false><<<nb, 128, 0, st>>>(dv, jc, a, tau2, s, s_abs, half, npass, s2, jmode); break;
        default: k_cphase_f<3, false><<<nb, 128, 0, st>>>(dv, jc, a, tau2, s, s_abs, half, npass, s2, jmode); break;
        }
    }
}

void launch_vphase(const Dev& d, const double* a, double tau2, uint32_t s_off, int half, int order,
                   int doC, int doJ, int fp64, int variant, cudaStream_t s, uint32_t s_off2, const RepParams* hp0,
                   int presorted)
{
    vphase_any(d, a, tau2, s_off, s_off2, 0, half, order, doC, doJ, fp64, variant, s, hp0, presorted);
}

void launch_vphase_abs(const Dev& d, const double* a, double tau2, uint32_t s0, int half, int order,
                       int doC, int doJ, int fp64, int variant, cudaStream_t s, const RepParams* hp0,
                       int presorted)
{
    vphase_any(d, a, tau2, s0, 0, 1, half, order, doC, doJ, fp64, variant, s, hp0, presorted);
}

}  // namespace mdj
