// common.cuh -- device-side building blocks of the GB300 JUMP engine.
//
// Internal header of libmdjump.so (not installed). Holds the per-replica
// parameter block, the counter-based Philox4x32-10 generator, the pair terms
// (DSF Coulomb, shifted-force LJ, the quintic switch chi of Sec. 3.1), the
// normal-law helpers for Theta(eta) and the G~ sampler (Sec. 2.2, 2.4).
// Every function is templated on the arithmetic type T: double for the FP64
// parity mode, float for the mixed-precision mode.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mdj {

// ---- physical constants (kcal/mol, A, ps, amu, e) --------------------------
constexpr double KB = 0.0019872042586;     // kcal/mol/K
constexpr double COULOMB = 332.0637;       // kcal A / (mol e^2)
constexpr double KCAL_AMU = 418.4;         // 1 kcal/mol = 418.4 amu A^2 / ps^2
constexpr double PI = 3.14159265358979323846;

constexpr int MAX_TYPES = 8;
constexpr int KMAX = 1 << 20;              // proposal cap per atom and phase
constexpr int SAMPLER_CAP = 64;            // attempts of the G~ sampler

// Philox stream tags (counter word 2, bits 24..31)
constexpr uint32_t TAG_O = 1, TAG_C = 2, TAG_J = 3, TAG_S = 4;

// error flag bits (match MD_FLAG_* in md.h)
constexpr uint32_t F_BOUND = 1, F_LIMIT = 2, F_NONFIN = 4, F_OVERFLOW = 8;

// list kinds: short and full neighbour lists, up to four jump rings, LJ partners
constexpr int MAX_RINGS = 4;
enum ListKind { L_SHORT = 0, L_FULL = 1, L_R0 = 2, L_LJ = L_R0 + MAX_RINGS, NKIND = L_LJ + 1 };

// counters per replica
enum Counter { C_CPROP = 0, C_CACC, C_JPROP, C_JACC, C_SATT, C_REBUILD, C_OUTER, C_GUARD, NCOUNT };

// pair weight: full U, short chi U, long (1 - chi) U
enum Weight { W_FULL = 0, W_SHORT = 1, W_LONG = 2, W_LJLONG = 3 };   // W_LJLONG: (1 - chi) LJ alone

struct alignas(16) LJPair {
    double c12, c6, uR, duR;   // 4 eps s^12, 4 eps s^6, U_LJ(R), U_LJ'(R)
    float c12f, c6f, uRf, duRf;   // the same in FP32 (one 16-byte load)
    int on;                    // eps > 0
    int pad[3];
};

// Everything a kernel needs about one replica. Device resident, one per replica.
struct RepParams {
    double L, invL;
    int atom_off, n;
    // outer candidate grid (fixes the order of the jump lists)
    int nc, cell_off;
    double cs;
    // scaled coordinates: x = s L / 2^32 with s a 32-bit integer, so that
    // integer differences give the minimum image exactly
    double scl, inv_scl;       // L / 2^32, 2^32 / L
    float sclf, sclf_lo;       // L / 2^32 as a sum of two floats (hi + lo)
    float scl2f;               // (L / 2^32)^2
    unsigned long long sw2u;   // (r_c - h)^2 in squared scaled units, rounded
    // cutoffs
    double R, rc, h, sw;       // r_E, r_c, h, r_c - h
    double edge[MAX_RINGS + 1];// ring edges: sw = edge[0] < ... < edge[nr] = R
    float edgef[MAX_RINGS + 1];
    int nr, rings_on, lj_on, eps_mode;
    int lj_long, lj_jump;      // lj_long_mode (0 jumped, 1 in F0, 2 at the slow level); LJ bounces (J') on
    double skin, skin_o;
    // DSF: u(r) = erfc(a r)/r - eR + fR (r - R); u'(r) = -erfc(a r)/r^2 - k exp(-a^2 r^2)/r + fR
    double alpha, eR, fR, kexp;     // kexp = 2 a / sqrt(pi)
    float alphaf, eRf, fRf, kexpf;
    // thermostat / jumps
    double beta, gamma, eps0;
    uint32_t seed, replica;
    int ntypes, pad2;
    // shell table of the inner list build: bins of r^2 on [0, (r_E + skin_outer)^2)
    float shell_invw;          // bins per A^2
    int pad3;
    // squared limits of the ring (y < MAX_RINGS) and LJ (y = MAX_RINGS) shells:
    // [lo2, hi2) widened by the skin; empty shells have lo2 = hi2 = 0
    double shell_lo2[MAX_RINGS + 1], shell_hi2[MAX_RINGS + 1];
    float shell_lo2f[MAX_RINGS + 1], shell_hi2f[MAX_RINGS + 1];
    float r2s, r2f;            // (r_c + skin)^2, (r_E + skin)^2: short and full lists
    // Ewald electrostatics (coul_mode 1): real space is the DSF form with eR = fR = 0
    // (erfc(a r)/r cut at r_E); the reciprocal part is a smooth-PME sum on a K^3 grid
    int coul_mode, pme_p, pme_K;
    int pme_nb, pme_boff;               // bricks of PME_BRICK^3 grid points per edge, first brick
    int pad4;
    long long pme_goff, pme_soff;       // offsets of this replica's real grid and spectrum
    double pme_self;                    // -C a / sqrt(pi) sum q^2 (kcal/mol)
    LJPair lj[MAX_TYPES * MAX_TYPES];
};

// shell table: per bin of r^2, the ring and LJ lists that contain the whole
// bin (bit = list kind), or SHELL_AMB when a ring or LJ shell limit lies
// within the bin or its tolerance margin (decided in FP64 then)
// FP32 acceptance ratios: as eta -> 0 (pairs whose force is tiny beside the
// 1/(eps0 sqrt(2 pi)) floor of the adaptive bound) the exact p tends to 1 from
// below by less than FP32 rounding, and the FP32 quotient can land a few ulps
// above 1. Such a p is no evidence of a violated bound: the decision is exact
// anyway (U within 2e-6 of p is decided again in FP64, where the check is
// strict), so the FP32 check flags p above 1 + P_TOL32 only.
constexpr float P_TOL32 = 4e-6f;
constexpr int SHELL_BINS = 2048;
// smooth PME: the grid is processed in bricks of PME_BRICK^3 points; atoms are
// binned by the brick that holds floor(u), u = K x / L
constexpr int PME_BRICK = 8;

// bits of the per-replica overflow word: list kind k sets bit k; these two
// are the outer candidate list and a cell above the in-block sort capacity
constexpr uint32_t OVF_OUTER = 1u << 16, OVF_CELL = 1u << 17;
// a pair term outside the range of the 64-bit fixed-point sums (or not finite)
constexpr uint32_t OVF_FIX = 1u << 18;
constexpr uint16_t SHELL_AMB = 0x8000;

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ---------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

__device__ __forceinline__ U4 draw(const RepParams& P, uint32_t atom, uint32_t s0, uint32_t tag,
                                   int half, uint32_t attempt, uint32_t k)
{
    return philox(atom, s0, (tag << 24) | (uint32_t(half) << 20) | (attempt << 8), k,
                  P.seed, P.replica);
}

// uniform on (0,1): (b + 1/2) 2^-32
template <typename T> __device__ __forceinline__ T unif(uint32_t b);
template <> __device__ __forceinline__ double unif<double>(uint32_t b)
{
    return ((double)b + 0.5) * (1.0 / 4294967296.0);
}
template <> __device__ __forceinline__ float unif<float>(uint32_t b)
{
    // exact 24-bit rounding of (b + 1/2) 2^-32 through the double path would
    // cost FP64; take the top 24 bits plus a half step instead: (b>>8 + 1/2) 2^-24
    return ((float)(b >> 8) + 0.5f) * (1.0f / 16777216.0f);
}

// ---- math shims --------------------------------------------------------------
__device__ __forceinline__ double d_erfc(double x) { return erfc(x); }
__device__ __forceinline__ float d_erfc(float x) { return erfcf(x); }
__device__ __forceinline__ double d_exp(double x) { return exp(x); }
__device__ __forceinline__ float d_exp(float x) { return expf(x); }
__device__ __forceinline__ double d_log(double x) { return log(x); }
__device__ __forceinline__ float d_log(float x) { return logf(x); }
__device__ __forceinline__ double d_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double d_rint(double x) { return rint(x); }
__device__ __forceinline__ float d_rint(float x) { return rintf(x); }
__device__ __forceinline__ void d_sincospi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ void d_sincospi(float x, float* s, float* c) { sincospif(x, s, c); }

template <typename T> struct PT;
template <> struct PT<double> {
    __device__ static double alpha(const RepParams& P) { return P.alpha; }
    __device__ static double eR(const RepParams& P) { return P.eR; }
    __device__ static double fR(const RepParams& P) { return P.fR; }
    __device__ static double kexp(const RepParams& P) { return P.kexp; }
    __device__ static double c12(const LJPair& l) { return l.c12; }
    __device__ static double c6(const LJPair& l) { return l.c6; }
    __device__ static double uR(const LJPair& l) { return l.uR; }
    __device__ static double duR(const LJPair& l) { return l.duR; }
};
template <> struct PT<float> {
    __device__ static float alpha(const RepParams& P) { return P.alphaf; }
    __device__ static float eR(const RepParams& P) { return P.eRf; }
    __device__ static float fR(const RepParams& P) { return P.fRf; }
    __device__ static float kexp(const RepParams& P) { return P.kexpf; }
    __device__ static float c12(const LJPair& l) { return l.c12f; }
    __device__ static float c6(const LJPair& l) { return l.c6f; }
    __device__ static float uR(const LJPair& l) { return l.uRf; }
    __device__ static float duR(const LJPair& l) { return l.duRf; }
};

// ---- switch chi (quintic step on [r_c - h, r_c]) ----------------------------
// chi and its slope at s = (r - sw) / h in [0, 1]
template <typename T>
__device__ __forceinline__ void chi_of_s(T s, T h, T& c, T& dc)
{
    const T s2 = s * s;
    c = T(1) - s2 * s * (T(10) - T(15) * s + T(6) * s2);
    const T om = T(1) - s;
    dc = T(-30) * s2 * om * om / h;
}

template <typename T>
__device__ __forceinline__ void chi_and_slope(T r, T sw, T h, T& c, T& dc)
{
    if (r <= sw) { c = T(1); dc = T(0); return; }
    if (r >= sw + h) { c = T(0); dc = T(0); return; }
    chi_of_s<T>((r - sw) / h, h, c, dc);
}

// The same in FP32 for a pair given by its scaled coordinates a, b, with s
// taken from the exact integer displacement: r - sw = (r^2 - sw^2) / (r + sw),
// where r^2 - sw^2 is formed exactly in 64-bit integers (three 32 x 32 -> 64
// bit products; the squared length of a displacement shorter than L/2 stays
// below 2^62) and rounded once. An FP32 distance near sw is off by up to half
// an ulp of r (2.4e-7 A at 4.5 A), and the switch's slope (up to 15/(8h) per
// unit of s) turns that into the largest error of a chi-weighted pair force,
// chi' U; this form leaves about a tenth of it. r is the FP32 distance that
// decides the region; hinv = 1/h.
__device__ __forceinline__ void chi_and_slope_x(const uint4& a, const uint4& b, const RepParams& P, float r,
                                                float sw, float h, float hinv, float& c, float& dc)
{
    if (r <= sw) { c = 1.f; dc = 0.f; return; }
    if (r >= sw + h) { c = 0.f; dc = 0.f; return; }
    const int ix = int(a.x - b.x), iy = int(a.y - b.y), iz = int(a.z - b.z);
    const long long q = (long long)ix * ix + (long long)iy * iy + (long long)iz * iz;
    const float dq = __ll2float_rn(q - (long long)P.sw2u);
    const float s = fminf(1.f, fmaxf(0.f, __fdividef(dq * P.scl2f, r + sw) * hinv));
    const float s2 = s * s;
    c = 1.f - s2 * s * (10.f - 15.f * s + 6.f * s2);
    const float om = 1.f - s;
    dc = -30.f * s2 * om * om * hinv;
}

// DSF Coulomb per unit C q_i q_j: value and radial derivative, r < R
template <typename T>
__device__ __forceinline__ void dsf(const RepParams& P, T r, T rinv, T& u, T& du)
{
    const T a = PT<T>::alpha(P);
    const T e = d_erfc(a * r);
    const T g = PT<T>::kexp(P) * d_exp(-a * a * r * r);
    u = e * rinv - PT<T>::eR(P) + PT<T>::fR(P) * (r - T(P.R));
    du = -(e * rinv + g) * rinv + PT<T>::fR(P);
}

// shifted-force LJ: value and radial derivative, r < R
template <typename T>
__device__ __forceinline__ void ljsf(const RepParams& P, const LJPair& l, T r, T rinv, T& u, T& du)
{
    const T r2i = rinv * rinv;
    const T r6i = r2i * r2i * r2i;
    const T c12 = PT<T>::c12(l), c6 = PT<T>::c6(l);
    u = r6i * (c12 * r6i - c6) - PT<T>::uR(l) - (r - T(P.R)) * PT<T>::duR(l);
    du = r6i * rinv * (T(6) * c6 - T(12) * c12 * r6i) - PT<T>::duR(l);
}
template <>
__device__ __forceinline__ void ljsf<float>(const RepParams& P, const LJPair& l, float r, float rinv, float& u,
                                            float& du)
{
    const float4 c = *reinterpret_cast<const float4*>(&l.c12f);    // c12, c6, U(R), U'(R)
    const float r2i = rinv * rinv;
    const float r6i = r2i * r2i * r2i;
    u = r6i * (c.x * r6i - c.y) - c.z - (r - float(P.R)) * c.w;
    du = r6i * rinv * (6.f * c.y - 12.f * c.x * r6i) - c.w;
}

// distance and its reciprocal from r^2, by the correctly rounded square root
// and division in both precisions (an approximate reciprocal square root in
// FP32 costs about 2e-6 of relative force error per pair)
__device__ __forceinline__ void rdist(double r2, double& r, double& rinv)
{
    r = sqrt(r2);
    rinv = 1.0 / r;
}
__device__ __forceinline__ void rdist(float r2, float& r, float& rinv)
{
    r = sqrtf(r2);
    rinv = 1.f / r;
}

// ---- normal law --------------------------------------------------------------
template <typename T> __device__ __forceinline__ T nphi(T y)
{
    return d_exp(T(-0.5) * y * y) * T(0.3989422804014327);
}
template <typename T> __device__ __forceinline__ T nPhi(T y)
{
    return T(0.5) * d_erfc(-y * T(0.7071067811865476));
}
// Theta(eta) = E[(eta + G)_+] = eta Phi(eta) + phi(eta)
template <typename T> __device__ __forceinline__ T theta(T eta)
{
    const T t = eta * nPhi(eta) + nphi(eta);
    return t > T(0) ? t : T(0);
}

// one attempt of the G~ rejection sampler (Sec. 2.4); returns true on accept
template <typename T>
__device__ __forceinline__ bool gtilde_attempt(T eta, const U4& u, T& y)
{
    if (eta > T(0)) {
        const T pg = eta / (eta + T(0.3989422804014327));
        const T rad = d_sqrt(T(-2) * d_log(unif<T>(u.y)));
        if (unif<T>(u.x) < pg) {
            T s, c;
            d_sincospi(T(2) * unif<T>(u.z), &s, &c);
            y = rad * c;
        } else {
            y = rad;
        }
        if (y >= T(0)) return true;
        const T ratio = (eta + y) > T(0) ? (eta + y) / eta : T(0);
        return unif<T>(u.w) <= ratio;
    } else if (eta >= T(-1)) {
        const T z = d_sqrt(T(-2) * d_log(unif<T>(u.x)));
        y = z - eta;
        return unif<T>(u.y) <= d_exp(eta * z);
    } else if (eta >= T(-2.5)) {
        const T z = -d_log(unif<T>(u.x)) / (-eta);
        y = z - eta;
        return unif<T>(u.y) <= z * d_exp(T(0.5) * (T(1) - z * z));
    } else {
        const T z = -(d_log(unif<T>(u.x)) + d_log(unif<T>(u.y))) / (-eta);
        y = z - eta;
        return unif<T>(u.z) <= d_exp(T(-0.5) * z * z);
    }
}

// ---- fixed point (2^32 units of kcal/mol/A) -----------------------------------
constexpr double FIX_SCALE = 4294967296.0;
constexpr double FIX_INV = 1.0 / 4294967296.0;
// largest |component| of one pair term that the sums accept: 2^20 kcal/mol/A
// is 2^52 fixed-point units, so 2^11 terms per atom stay inside int64 (list
// rows are far shorter); a term at or above it, or a non-finite one, is
// flagged as an overflow (real forces stay below ~10^4 kcal/mol/A)
constexpr float FIX_TERM_MAX = 1048576.0f;

__device__ __forceinline__ long long to_fix(float f)
{
    return __float2ll_rn(f * 4294967296.0f);
}

// ---- scaled 32-bit coordinates ----------------------------------------------------
// position in [0, L) -> integer in [0, 2^32) (wraps at L, which is the periodic box)
__device__ __forceinline__ uint32_t to_scaled(double x, const RepParams& P)
{
    return (uint32_t)(unsigned long long)llrint(x * P.inv_scl);
}
// FP32 minimum-image displacement a - b: exact integer difference, rounded
// once to FP32 and scaled by L / 2^32 carried as two floats (no systematic
// scale error)
__device__ __forceinline__ void sdisp(const uint4& a, const uint4& b, float s, float slo, float& dx, float& dy,
                                      float& dz)
{
    const float fx = __int2float_rn(int(a.x - b.x));
    const float fy = __int2float_rn(int(a.y - b.y));
    const float fz = __int2float_rn(int(a.z - b.z));
    dx = fmaf(fx, s, fx * slo);
    dy = fmaf(fy, s, fy * slo);
    dz = fmaf(fz, s, fz * slo);
}

// ---- list rows into L2 ahead of their use ---------------------------------------
// Lists are far larger than L2 and are read row by row: a whole row is asked
// into L2 with one bulk prefetch (a hint: no completion to wait for, nothing
// is written) before the loop that reads it, so the loop's loads wait on L2
// instead of DRAM. `row` is 16-byte aligned (rows start at multiples of 32
// entries) and the size is rounded up to 16 bytes within the row's capacity.
__device__ __forceinline__ void prefetch_row_l2(const uint32_t* row, int n)
{
    if (n <= 0) return;
    const uint32_t bytes = uint32_t((n + 3) & ~3) * 4u;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(row)), "r"(bytes)
                 : "memory");
}

}  // namespace mdj
