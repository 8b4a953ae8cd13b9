// k_force.cu -- pair and bonded gradients, kicks, the A O A update, energies.
//
// Pair terms (LJ shifted in value and slope at r_E, DSF Coulomb) weighted by
// 1, chi or 1 - chi (the split U = chi U + (1 - chi) U of Sec. 3.1); bonded
// terms 1/2 k (r - r0)^2 and 1/2 k (theta - theta0)^2. One thread per atom
// owns its gradient (full neighbour lists, no atomics); in the mixed mode each
// pair contribution is rounded to 64-bit fixed point (2^-32 kcal/mol/A) before
// it is summed, so the sum does not depend on the order of the list.
// The B, A and O parts follow the splitting of Sec. 2.3: B kicks the
// velocity, A moves positions, O is the exact Ornstein-Uhlenbeck step with
// Philox normals.
#include "engine.h"

namespace mdj {

namespace {

__device__ __forceinline__ double3 ld3(const double* p, int i)
{
    return make_double3(p[3 * i], p[3 * i + 1], p[3 * i + 2]);
}

__device__ __forceinline__ double mimg(double t, const RepParams& P)
{
    return t - P.L * rint(t * P.invL);
}

// displacement x_i - x_j at the current positions
template <typename T> struct Disp;
template <> struct Disp<double> {
    __device__ static void get(const Dev& d, const RepParams& P, int i, int j, double& dx, double& dy,
                               double& dz)
    {
        const double3 a = ld3(d.x, i), b = ld3(d.x, j);
        dx = mimg(a.x - b.x, P); dy = mimg(a.y - b.y, P); dz = mimg(a.z - b.z, P);
    }
};

// bonded terms, FP64 in both modes (with k_b ~ 10^3 kcal/mol/A^2 an FP32 bond
// length would put ~10^-4 kcal/mol/A of error on the force). bond_term: the
// gradient on the bond's first atom; angle_term: the gradients on the two end
// atoms (the centre takes minus their sum)
__device__ __forceinline__ void bond_term_x(const RepParams& P, const double* xa, const double* xb, double k,
                                            double r0, double o[3])
{
    const double dx = mimg(xa[0] - xb[0], P), dy = mimg(xa[1] - xb[1], P), dz = mimg(xa[2] - xb[2], P);
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    const double f = r > 0.0 ? k * (r - r0) / r : 0.0;
    o[0] = f * dx; o[1] = f * dy; o[2] = f * dz;
}

// xa, xc: the end atoms, xm: the centre
__device__ __forceinline__ void angle_term_x(const RepParams& P, const double* xa, const double* xm, const double* xc,
                                             double k, double t0, double o[6])
{
    const double ax = mimg(xa[0] - xm[0], P), ay = mimg(xa[1] - xm[1], P), az = mimg(xa[2] - xm[2], P);
    const double bx = mimg(xc[0] - xm[0], P), by = mimg(xc[1] - xm[1], P), bz = mimg(xc[2] - xm[2], P);
    // FP64 division and the trigonometric functions run at a small fraction of
    // the FP32 rate on this GPU: one reciprocal per length, sin(theta) as
    // sqrt(1 - cos^2) (theta stays far from 0 and pi in these molecules; the
    // guard below covers the degenerate case), and one division for the prefactor
    const double ra = sqrt(ax * ax + ay * ay + az * az), rb = sqrt(bx * bx + by * by + bz * bz);
    const double ira = 1.0 / ra, irb = 1.0 / rb;
    double cth = (ax * bx + ay * by + az * bz) * (ira * irb);
    cth = fmin(1.0, fmax(-1.0, cth));
    const double th = acos(cth);
    const double sth = sqrt(fmax(0.0, 1.0 - cth * cth));
    if (sth < 1e-12) {
        for (int c = 0; c < 6; ++c) o[c] = 0.0;
        return;
    }
    const double q = k * (th - t0) / sth;
    const double ia = q * ira, ib = q * irb;
    const double ux = ax * ira, uy = ay * ira, uz = az * ira, vx = bx * irb, vy = by * irb, vz = bz * irb;
    o[0] = (cth * ux - vx) * ia; o[1] = (cth * uy - vy) * ia; o[2] = (cth * uz - vz) * ia;
    o[3] = (cth * vx - ux) * ib; o[4] = (cth * vy - uy) * ib; o[5] = (cth * vz - uz) * ib;
}

__device__ __forceinline__ void bond_term(const Dev& d, int t, double o[3])
{
    const int2 ij = d.bond_ij[t];
    bond_term_x(d.P[d.rep[ij.x]], d.x + 3 * ij.x, d.x + 3 * ij.y, d.bond_k[t], d.bond_r0[t], o);
}

__device__ __forceinline__ void angle_term(const Dev& d, int ta, double o[6])
{
    const int4 a = d.ang[ta];
    angle_term_x(d.P[d.rep[a.y]], d.x + 3 * a.x, d.x + 3 * a.y, d.x + 3 * a.z, d.ang_k[ta], d.ang_t0[ta], o);
}

// one thread per term; the per-term gradients are gathered per atom
// afterwards, so every atom sums its terms in a fixed order
__global__ void k_bonded_terms(Dev d)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < d.nbond) {
        double o[3];
        bond_term(d, t, o);
        d.bterm[3 * t] = o[0]; d.bterm[3 * t + 1] = o[1]; d.bterm[3 * t + 2] = o[2];
        return;
    }
    const int ta = t - d.nbond;
    if (ta >= d.nang) return;
    double o[6];
    angle_term(d, ta, o);
    double* out = d.aterm + 6 * (size_t)ta;
    for (int c = 0; c < 6; ++c) out[c] = o[c];
}

// sum of the bonded gradients on atom i (items in a fixed order)
__device__ __forceinline__ void bonded_gather(const Dev& d, int i, double& gx, double& gy, double& gz)
{
    const int b0 = d.bi_off[i], b1 = d.bi_off[i + 1];
    for (int it = b0; it < b1; ++it) {
        const int2 item = d.bitem[it];
        const int kind = item.x & 15, role = item.x >> 4, t = item.y;
        if (kind == 0) {
            const double sgn = role == 0 ? 1.0 : -1.0;
            // sgn = +-1: the product is exact and the fused form adds it with one rounding, as before
            gx = fma(sgn, d.bterm[3 * t], gx); gy = fma(sgn, d.bterm[3 * t + 1], gy); gz = fma(sgn, d.bterm[3 * t + 2], gz);
        } else {
            const double* o = d.aterm + 6 * (size_t)t;
            if (role == 0) { gx += o[0]; gy += o[1]; gz += o[2]; }
            else if (role == 2) { gx += o[3]; gy += o[4]; gz += o[5]; }
            else { gx -= o[0] + o[3]; gy -= o[1] + o[4]; gz -= o[2] + o[5]; }
        }
    }
}

// switch of a pair: FP32 from the exact integer displacement, FP64 from r
__device__ __forceinline__ void chi_t(const uint4& a, const uint4& b, const RepParams& P, float r, float sw, float h,
                                      float hinv, float& c, float& dc)
{
    chi_and_slope_x(a, b, P, r, sw, h, hinv, c, dc);
}
__device__ __forceinline__ void chi_t(const uint4&, const uint4&, const RepParams&, double r, double sw, double h,
                                      double, double& c, double& dc)
{
    chi_and_slope<double>(r, sw, h, c, dc);
}

// pair gradient accumulators: fixed point for float, double for double
template <typename T> struct Acc;
template <> struct Acc<float> {
    long long x = 0, y = 0, z = 0;
    bool bad = false;          // a term outside the fixed-point range (or not finite)
    // the term (f dx, f dy, f dz) with f = (dU/dr) / r; fr = dU/dr is its length
    __device__ void add(float f, float dx, float dy, float dz, float fr)
    {
        bad |= !(fabsf(fr) < 0.5f * FIX_TERM_MAX);      // each component, and their sum, below the limit
        x += to_fix(f * dx); y += to_fix(f * dy); z += to_fix(f * dz);
    }
    __device__ bool overflow() const { return bad; }
    __device__ void combine_shfl(int tpa)
    {
        for (int o = tpa >> 1; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o, tpa);
            y += __shfl_down_sync(0xffffffffu, y, o, tpa);
            z += __shfl_down_sync(0xffffffffu, z, o, tpa);
        }
    }
    __device__ double gx() const { return double(x) * FIX_INV; }
    __device__ double gy() const { return double(y) * FIX_INV; }
    __device__ double gz() const { return double(z) * FIX_INV; }
};
template <> struct Acc<double> {
    double x = 0, y = 0, z = 0;
    __device__ void add(double f, double dx, double dy, double dz, double)
    {
        x += f * dx; y += f * dy; z += f * dz;
    }
    __device__ bool overflow() const { return false; }
    __device__ void combine_shfl(int tpa)
    {
        for (int o = tpa >> 1; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o, tpa);
            y += __shfl_down_sync(0xffffffffu, y, o, tpa);
            z += __shfl_down_sync(0xffffffffu, z, o, tpa);
        }
    }
    __device__ double gx() const { return x; }
    __device__ double gy() const { return y; }
    __device__ double gz() const { return z; }
};

// pair gradient over the list of atom i; TPA threads per atom stride the list
template <typename T, int W, bool BONDED, int TPA>
__global__ void __launch_bounds__(256) k_force(Dev d, int lk, double* out, int as_grad)
{
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = gt / TPA, sub = gt % TPA;
    const bool live = t < d.N;
    // the LJ part alone visits the atoms with LJ partners first (warps without idle atoms)
    const int i = (W == W_LJLONG && live) ? d.lj_perm[t] : t;
    const int ii = live ? i : d.N - 1;
    const int r = d.rep[ii];
    const RepParams& P = d.P[r];
    Acc<T> acc;
    if (live) {
        const int ti = d.type[i];
        const T qi = T(d.q[i]);
        const T cut = W == W_SHORT ? T(fmin(P.rc, P.R)) : T(P.R);
        const T cut2 = cut * cut;
        const T sw = T(P.sw), h = T(P.h), sw2 = sw * sw, hinv = T(1) / h;
        const T C = T(COULOMB);
        const uint32_t* row = d.list[lk] + (size_t)i * d.lcap[lk];
        const int n = W == W_LJLONG ? 0 : min(d.lcnt[lk][i], d.lcap[lk]);
        if (sub == 0) prefetch_row_l2(row, n);
        // position of i in the arithmetic type
        uint4 pi = make_uint4(0, 0, 0, 0);
        double3 xi = make_double3(0, 0, 0);
        if (sizeof(T) == 4) pi = d.pos[i];
        else xi = ld3(d.x, i);
        const float sc = P.sclf;
        for (int k = sub; k < n; k += TPA) {
            const int j = int(row[k]);
            T dx, dy, dz, qj;
            uint4 pj = make_uint4(0, 0, 0, 0);
            if (sizeof(T) == 4) {
                pj = d.pos[j];
                float fx, fy, fz;
                sdisp(pi, pj, sc, P.sclf_lo, fx, fy, fz);
                dx = T(fx); dy = T(fy); dz = T(fz);
                qj = T(__uint_as_float(pj.w));
            } else {
                const double3 xj = ld3(d.x, j);
                dx = T(mimg(xi.x - xj.x, P)); dy = T(mimg(xi.y - xj.y, P)); dz = T(mimg(xi.z - xj.z, P));
                qj = T(d.q[j]);
            }
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= cut2) continue;
            if (W == W_LONG && r2 <= sw2) continue;
            T rr, rinv;
            rdist(r2, rr, rinv);
            T u = T(0), du = T(0);
            const T qq = qi * qj;
            if (qq != T(0)) {
                T uc, duc;
                dsf<T>(P, rr, rinv, uc, duc);
                u = C * qq * uc;
                du = C * qq * duc;
            }
            const LJPair& lj = P.lj[ti * MAX_TYPES + d.type[j]];
            if (lj.on && !(W == W_LONG && P.lj_long == 1)) {   // LJ long part in F0: not in the long weight
                T ul, dul;
                ljsf<T>(P, lj, rr, rinv, ul, dul);
                u += ul;
                du += dul;
            }
            T f;
            if (W == W_FULL) {
                f = du;
            } else {
                T c, dc;
                chi_t(pi, pj, P, rr, sw, h, hinv, c, dc);
                f = W == W_SHORT ? dc * u + c * du : -dc * u + (T(1) - c) * du;
            }
            acc.add(f * rinv, dx, dy, dz, f);
        }
        if ((W == W_SHORT && (P.lj_long == 1 || (P.lj_long == 2 && BONDED))) || (W == W_LJLONG && P.lj_long == 2)) {
            // the (1 - chi) LJ part over the LJ list: in the short force with
            // lj_long_mode 1 (the paper's GPU runs), in F0 and alone at the slow
            // level with lj_long_mode 2
            const uint32_t* lrow = d.list[L_LJ] + (size_t)i * d.lcap[L_LJ];
            const int nl = min(d.lcnt[L_LJ][i], d.lcap[L_LJ]);
            if (sub == 0) prefetch_row_l2(lrow, nl);
            const T R2 = T(P.R) * T(P.R);
            for (int k = sub; k < nl; k += TPA) {
                const int j = int(lrow[k]);
                T dx, dy, dz;
                uint4 pj = make_uint4(0, 0, 0, 0);
                if (sizeof(T) == 4) {
                    pj = d.pos[j];
                    float fx, fy, fz;
                    sdisp(pi, pj, sc, P.sclf_lo, fx, fy, fz);
                    dx = T(fx); dy = T(fy); dz = T(fz);
                } else {
                    const double3 xj = ld3(d.x, j);
                    dx = T(mimg(xi.x - xj.x, P)); dy = T(mimg(xi.y - xj.y, P)); dz = T(mimg(xi.z - xj.z, P));
                }
                const T r2 = dx * dx + dy * dy + dz * dz;
                if (r2 >= R2 || r2 <= sw2) continue;
                const LJPair& lj = P.lj[ti * MAX_TYPES + d.type[j]];
                if (!lj.on) continue;
                T rr, rinv;
                rdist(r2, rr, rinv);
                T ul, dul, c, dc;
                ljsf<T>(P, lj, rr, rinv, ul, dul);
                chi_t(pi, pj, P, rr, sw, h, hinv, c, dc);
                const T fl = -dc * ul + (T(1) - c) * dul;
                acc.add(fl * rinv, dx, dy, dz, fl);
            }
        }
    }
    if (live && acc.overflow()) {
        atomicOr(&d.err[r], F_OVERFLOW);
        atomicOr(&d.ovf[r], OVF_FIX);
    }
    if (TPA > 1) acc.combine_shfl(TPA);
    if (!live || sub != 0) return;
    double gx = acc.gx(), gy = acc.gy(), gz = acc.gz();
    if (BONDED) bonded_gather(d, i, gx, gy, gz);
    if (as_grad) {
        out[3 * i] = gx; out[3 * i + 1] = gy; out[3 * i + 2] = gz;
    } else {
        const double s = d.nimt[i];
        out[3 * i] = s * gx; out[3 * i + 1] = s * gy; out[3 * i + 2] = s * gz;
    }
}

// One pair of the half-list and tile kernels (mixed mode), i - j from the
// scaled coordinates: false when it does not contribute (beyond the cutoff of
// the weight, inside r_c - h for the long weight, no LJ pair for the LJ part
// alone); else f = (dU/dr)/r, fr = dU/dr and the displacement (dx, dy, dz).
template <int W>
__device__ __forceinline__ bool pair_term(const Dev& d, const RepParams& P, const uint4& pi, int ti, const uint4& pj,
                                          int j, float sc, float cut2, float sw, float h, float sw2, float hinv,
                                          float R2, float& dx, float& dy, float& dz, float& f, float& fr)
{
    const float C = float(COULOMB);
    sdisp(pi, pj, sc, P.sclf_lo, dx, dy, dz);
    const float qi = __uint_as_float(pi.w), qj = __uint_as_float(pj.w);
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (W == W_LJLONG) {
        if (r2 >= R2 || r2 <= sw2) return false;
        const LJPair& lj = P.lj[ti * MAX_TYPES + d.type[j]];
        if (!lj.on) return false;
        float rr, rinv;
        rdist(r2, rr, rinv);
        float ul, dul, c, dc;
        ljsf<float>(P, lj, rr, rinv, ul, dul);
        chi_and_slope_x(pi, pj, P, rr, sw, h, hinv, c, dc);
        fr = -dc * ul + (1.f - c) * dul;
        f = fr * rinv;
        return true;
    }
    if (r2 >= cut2) return false;
    if (W == W_LONG && r2 <= sw2) return false;
    float rr, rinv;
    rdist(r2, rr, rinv);
    float u = 0.f, du = 0.f;
    const float qq = qi * qj;
    if (qq != 0.f) {
        float uc, duc;
        dsf<float>(P, rr, rinv, uc, duc);
        u = C * qq * uc;
        du = C * qq * duc;
    }
    const LJPair& lj = P.lj[ti * MAX_TYPES + d.type[j]];
    if (lj.on && !(W == W_LONG && P.lj_long == 1)) {
        float ul, dul;
        ljsf<float>(P, lj, rr, rinv, ul, dul);
        u += ul;
        du += dul;
    }
    if (W == W_FULL) {
        fr = du;
    } else {
        float c, dc;
        chi_and_slope_x(pi, pj, P, rr, sw, h, hinv, c, dc);
        fr = W == W_SHORT ? dc * u + c * du : -dc * u + (1.f - c) * du;
    }
    f = fr * rinv;
    return true;
}

// The same pair gradient over half of each list: the threads of atom i take
// only the partners j > i and add the pair's fixed-point contribution to both
// atoms (64-bit integer atomics into d.facc), so every unique pair is
// evaluated once. The lists are symmetric (j is in the list of i exactly when
// i is in the list of j: membership is decided from r^2, which the exact
// integer displacement makes the same both ways), the displacement j - i is
// the exact negation of i - j, the pair terms depend on r, q_i q_j and the
// (symmetric) LJ table only, and round-to-nearest conversion to fixed point
// is odd, so each atom receives exactly the terms the full-list kernel sums,
// and integer sums do not depend on their order: the results are bit for bit
// those of k_force<float>. k_force_finish converts the sums and clears d.facc.
template <int W, int TPA>
__global__ void __launch_bounds__(256) k_force_half(Dev d, int lk)
{
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = gt / TPA, sub = gt % TPA;
    const bool live = t < d.N;
    const int i = (W == W_LJLONG && live) ? d.lj_perm[t] : t;
    const int ii = live ? i : d.N - 1;
    const int r = d.rep[ii];
    const RepParams& P = d.P[r];
    Acc<float> acc;
    if (live) {
        const int ti = d.type[i];
        const uint4 pi = d.pos[i];
        const float cut = W == W_SHORT ? float(fmin(P.rc, P.R)) : float(P.R);
        const float cut2 = cut * cut;
        const float sw = float(P.sw), h = float(P.h), sw2 = sw * sw, hinv = 1.f / h;
        const uint32_t* row = d.list[lk] + (size_t)i * d.lcap[lk];
        // the (1 - chi) LJ part alone (W_LJLONG) runs over the LJ list of replicas
        // with lj_long_mode 2 only (zero elsewhere, as in k_force)
        const int n = (W == W_LJLONG && P.lj_long != 2) ? 0 : min(d.lcnt[lk][i], d.lcap[lk]);
        if (sub == 0) prefetch_row_l2(row, n);
        const float sc = P.sclf;
        const float R2 = float(P.R) * float(P.R);
        for (int k = sub; k < n; k += TPA) {
            const int j = int(row[k]);
            if (j <= i) continue;
            const uint4 pj = d.pos[j];
            float dx, dy, dz, f, fr;
            if (!pair_term<W>(d, P, pi, ti, pj, j, sc, cut2, sw, h, sw2, hinv, R2, dx, dy, dz, f, fr)) continue;
            const float gx = f * dx, gy = f * dy, gz = f * dz;
            acc.add(f, dx, dy, dz, fr);
            unsigned long long* fj = reinterpret_cast<unsigned long long*>(d.facc) + 3 * (size_t)j;
            atomicAdd(fj, (unsigned long long)(-to_fix(gx)));
            atomicAdd(fj + 1, (unsigned long long)(-to_fix(gy)));
            atomicAdd(fj + 2, (unsigned long long)(-to_fix(gz)));
        }
    }
    if (live && acc.overflow()) {
        atomicOr(&d.err[r], F_OVERFLOW);
        atomicOr(&d.ovf[r], OVF_FIX);
    }
    if (TPA > 1) acc.combine_shfl(TPA);
    if (!live || sub != 0) return;
    unsigned long long* fi = reinterpret_cast<unsigned long long*>(d.facc) + 3 * (size_t)i;
    if (acc.x) atomicAdd(fi, (unsigned long long)acc.x);
    if (acc.y) atomicAdd(fi + 1, (unsigned long long)acc.y);
    if (acc.z) atomicAdd(fi + 2, (unsigned long long)acc.z);
}

// The same half-list pair gradient over cluster tiles. The atoms of each
// outer cell form clusters of TILE_CL (k_lists.cu); list `tl` holds, for each
// cluster I, the clusters J >= I whose boxes come within the list radius, with
// a 64-bit mask of the slot pairs (a, b) to take (both slots occupied, not an
// excluded pair, b > a when J = I). One warp per cluster I: lane (a, g) holds
// atom a of I and takes slots b = g and g + 4 of each J, so the eight i atoms
// and a J's positions are loaded once per tile instead of once per pair. Each
// pair is the pair_term of k_force_half with the displacement i - j, and each
// atom receives the same fixed-point terms (the j side negated exactly) into
// d.facc: the sums are bit for bit those of the per-atom kernels.
// Measured on 96,000-atom water: 2-2.5 times slower than the per-atom
// half-list kernels (short list 0.27 against 0.11 ms, full list 0.70 against
// 0.36 ms). Most of a tile's 64 slot pairs lie beyond the cutoff (clusters of
// eight atoms span ~4 A; 15-35 % of the slots are pairs within it), and every
// slot pays the j-side shuffle reduction whether it contributes or not; a
// version that loaded the next tile's atoms ahead was slower still. The
// tiles are therefore opt-in (MDJ_TILES) and the autotuner times them only
// then.
template <int W>
__global__ void __launch_bounds__(128) k_force_tile(Dev d, int tl)
{
    const int lane = threadIdx.x & 31, a = lane & 7, g = lane >> 3;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int I = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); I < d.ncl_cap; I += nw) {
        const int cell = d.cl_cell[I];
        if (cell < 0) continue;
        const int r = d.cell_rep[cell];
        const RepParams& P = d.P[r];
        const int i = d.cl_atom[TILE_CL * (size_t)I + a];
        const uint4 pi = i >= 0 ? d.pos[i] : make_uint4(0, 0, 0, 0);
        const int ti = i >= 0 ? d.type[i] : 0;
        const float cut = W == W_SHORT ? float(fmin(P.rc, P.R)) : float(P.R);
        const float cut2 = cut * cut;
        const float sw = float(P.sw), h = float(P.h), sw2 = sw * sw, hinv = 1.f / h;
        const float sc = P.sclf;
        const float R2 = float(P.R) * float(P.R);
        const int n = min(d.cpl_n[tl][I], d.cpl_cap[tl]);
        const int* jrow = d.cpl_j[tl] + (size_t)I * d.cpl_cap[tl];
        const unsigned long long* mrow = d.cpl_mask[tl] + (size_t)I * d.cpl_cap[tl];
        Acc<float> acc;
        for (int t = 0; t < n; ++t) {
            const int J = jrow[t];
            const unsigned long long mask = mrow[t];
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
                const int b = g + 4 * pass;
                const int j = d.cl_atom[TILE_CL * (size_t)J + b];
                long long jx = 0, jy = 0, jz = 0;
                if ((mask >> (TILE_CL * a + b)) & 1ull) {
                    const uint4 pj = d.pos[j];
                    float dx, dy, dz, f, fr;
                    if (pair_term<W>(d, P, pi, ti, pj, j, sc, cut2, sw, h, sw2, hinv, R2, dx, dy, dz, f, fr)) {
                        const float gx = f * dx, gy = f * dy, gz = f * dz;
                        acc.add(f, dx, dy, dz, fr);
                        jx = -to_fix(gx); jy = -to_fix(gy); jz = -to_fix(gz);
                    }
                }
                // the terms on atom j, summed over the eight i atoms of its lane group
#pragma unroll
                for (int o = 1; o < TILE_CL; o <<= 1) {
                    jx += __shfl_xor_sync(0xffffffffu, jx, o);
                    jy += __shfl_xor_sync(0xffffffffu, jy, o);
                    jz += __shfl_xor_sync(0xffffffffu, jz, o);
                }
                if (a == 0 && j >= 0 && (jx | jy | jz)) {
                    unsigned long long* fj = reinterpret_cast<unsigned long long*>(d.facc) + 3 * (size_t)j;
                    if (jx) atomicAdd(fj, (unsigned long long)jx);
                    if (jy) atomicAdd(fj + 1, (unsigned long long)jy);
                    if (jz) atomicAdd(fj + 2, (unsigned long long)jz);
                }
            }
        }
        if (acc.overflow()) {
            atomicOr(&d.err[r], F_OVERFLOW);
            atomicOr(&d.ovf[r], OVF_FIX);
        }
        // the terms on atom i, summed over its four lane groups
        long long ix = acc.x, iy = acc.y, iz = acc.z;
        ix += __shfl_xor_sync(0xffffffffu, ix, 8); iy += __shfl_xor_sync(0xffffffffu, iy, 8);
        iz += __shfl_xor_sync(0xffffffffu, iz, 8);
        ix += __shfl_xor_sync(0xffffffffu, ix, 16); iy += __shfl_xor_sync(0xffffffffu, iy, 16);
        iz += __shfl_xor_sync(0xffffffffu, iz, 16);
        if (g == 0 && i >= 0) {
            unsigned long long* fi = reinterpret_cast<unsigned long long*>(d.facc) + 3 * (size_t)i;
            if (ix) atomicAdd(fi, (unsigned long long)ix);
            if (iy) atomicAdd(fi + 1, (unsigned long long)iy);
            if (iz) atomicAdd(fi + 2, (unsigned long long)iz);
        }
    }
}

// fixed-point sums of k_force_half to the output (plus the bonded terms),
// clearing the sums for the next evaluation
template <bool BONDED>
__global__ void k_force_finish(Dev d, double* out, int as_grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    long long* f = d.facc + 3 * (size_t)i;
    double gx = double(f[0]) * FIX_INV, gy = double(f[1]) * FIX_INV, gz = double(f[2]) * FIX_INV;
    f[0] = 0; f[1] = 0; f[2] = 0;
    if (BONDED) bonded_gather(d, i, gx, gy, gz);
    if (as_grad) {
        out[3 * i] = gx; out[3 * i + 1] = gy; out[3 * i + 2] = gz;
    } else {
        const double s = d.nimt[i];
        out[3 * i] = s * gx; out[3 * i + 1] = s * gy; out[3 * i + 2] = s * gz;
    }
}

// the bonded gradient of each atom; with kick_h != 0 (as an acceleration),
// also the kick v += kick_h a that follows it in an inner step, with the same
// rounding as k_kick
__global__ void k_bonded(Dev d, double* out, int as_grad, double kick_h)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    double gx = 0, gy = 0, gz = 0;
    bonded_gather(d, i, gx, gy, gz);
    if (as_grad) {
        out[3 * i] = gx; out[3 * i + 1] = gy; out[3 * i + 2] = gz;
    } else {
        const double s = d.nimt[i];
        const double a[3] = {s * gx, s * gy, s * gz};
        out[3 * i] = a[0]; out[3 * i + 1] = a[1]; out[3 * i + 2] = a[2];
        if (kick_h != 0.0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) d.v[3 * i + c] = fma(kick_h, a[c], d.v[3 * i + c]);
        }
    }
}

__global__ void k_kick(Dev d, const double* a, double h)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 3 * d.N) return;
    d.v[k] = fma(h, a[k], d.v[k]);
}

__global__ void k_kick2(Dev d, const double* a, double h, const double* b, double hb)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 3 * d.N) return;
    const double v = fma(h, a[k], d.v[k]);
    d.v[k] = fma(hb, b[k], v);
}

// A(tau/2) O(tau) A(tau/2), wrap, refresh the FP32 mirror, optional list check
template <typename T>
__global__ void k_aoa(Dev d, double tau, uint32_t s_off, int do_check, const double* pre_a, double pre_h)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const int r = d.rep[i];
    const RepParams& P = d.P[r];
    const uint32_t s0 = uint32_t(d.step_base[r]) + s_off;
    const double h = 0.5 * tau;
    double x[3] = {d.x[3 * i], d.x[3 * i + 1], d.x[3 * i + 2]};
    double v[3] = {d.v[3 * i], d.v[3 * i + 1], d.v[3 * i + 2]};
    // the kick that precedes the A O A in an inner step (as k_kick)
    if (pre_a) {
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] = fma(pre_h, pre_a[3 * i + a], v[a]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = fma(h, v[a], x[a]);
    const U4 u = draw(P, uint32_t(i - P.atom_off), s0, TAG_O, 0, 0, 0);
    const T r0 = d_sqrt(T(-2) * d_log(unif<T>(u.x)));
    const T r1 = d_sqrt(T(-2) * d_log(unif<T>(u.z)));
    T s1, c1v, s2, c2v;
    d_sincospi(T(2) * unif<T>(u.y), &s1, &c1v);
    d_sincospi(T(2) * unif<T>(u.w), &s2, &c2v);
    const double G[3] = {double(r0 * c1v), double(r0 * s1), double(r1 * c2v)};
    const double c1 = d.stepc[2 * r], c2 = d.stepc[2 * r + 1] * d.isqmt[i];
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = fma(c1, v[a], c2 * G[a]);
    int im[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        x[a] = fma(h, v[a], x[a]);
        if (x[a] < 0.0) { x[a] += P.L; im[a] -= 1; }
        if (x[a] >= P.L) { x[a] -= P.L; im[a] += 1; }
    }
    bool fin = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        fin = fin && isfinite(x[a]) && isfinite(v[a]);
        d.x[3 * i + a] = x[a];
        d.v[3 * i + a] = v[a];
        if (im[a]) d.img[3 * i + a] += im[a];
    }
    if (!fin) atomicOr(&d.err[r], F_NONFIN);
    // scaled 32-bit coordinates for the FP32 kernels (w keeps the charge)
    uint4 sp = d.pos[i];
    sp.x = to_scaled(x[0], P); sp.y = to_scaled(x[1], P); sp.z = to_scaled(x[2], P);
    d.pos[i] = sp;
    if (do_check) {
        const double lo = 0.5 * (P.skin_o - P.skin), li = 0.5 * P.skin;
        double t0 = mimg(x[0] - d.xo[3 * i], P), t1 = mimg(x[1] - d.xo[3 * i + 1], P),
               t2 = mimg(x[2] - d.xo[3 * i + 2], P);
        if (t0 * t0 + t1 * t1 + t2 * t2 > lo * lo) {
            d.flags[2 * r + 1] = 1;
            d.flags[2 * r] = 1;
        }
        t0 = mimg(x[0] - d.xb[3 * i], P); t1 = mimg(x[1] - d.xb[3 * i + 1], P);
        t2 = mimg(x[2] - d.xb[3 * i + 2], P);
        if (t0 * t0 + t1 * t1 + t2 * t2 > li * li) d.flags[2 * r] = 1;
    }
}

// Inner steps of the multiple-time-step drivers, fused: n steps of B(dt/2)
// A(dt/2) O(dt) A(dt/2) [bonded gradient] B(dt/2) on the bonded force alone
// (the innermost level of Sec. 2.3). Bonded terms couple only the atoms of
// one connected group (a molecule), so a block that holds whole groups runs
// all n steps with block barriers and no grid-wide step: positions stay in
// shared memory, velocities and accelerations in registers, each term of the
// block is evaluated once per step into shared memory and every atom sums its
// terms in its item order. The operations are those of the separate kicks,
// A-O-A update, term-parallel bonded kernel and gather, in the same order, so
// the results are the same bits. Blocks: atoms [ib_start[b], ib_start[b+1])
// (at most IB_MAX), their bonds ib_bond[ib_bond_off[b] ...] and angles
// ib_ang[ib_ang_off[b] ...] (at most IB_TERMS each); item_slot gives the slot
// of an item's term within its block's list.
template <typename T>
__global__ void __launch_bounds__(IB_MAX) k_inner_steps(Dev d, double dt, uint32_t s_off, int nsteps, int check_last)
{
    __shared__ double sx[IB_MAX][3];
    __shared__ double sb[IB_TERMS][3];
    __shared__ double sa[IB_TERMS][6];
    const int blk = blockIdx.x, tid = threadIdx.x;
    const int b0 = d.ib_start[blk], b1 = d.ib_start[blk + 1];
    const int tb0 = d.ib_bond_off[blk], nbt = d.ib_bond_off[blk + 1] - tb0;
    const int ta0 = d.ib_ang_off[blk], nat = d.ib_ang_off[blk + 1] - ta0;
    const int i = b0 + tid;
    const bool live = i < b1;
    const int ic = live ? i : b0;
    const int r = d.rep[ic];
    const RepParams& P = d.P[r];
    const double h = 0.5 * dt;
    double x[3], v[3], ab[3];
    int img[3] = {0, 0, 0};
    bool fin = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        x[a] = d.x[3 * ic + a];
        v[a] = d.v[3 * ic + a];
        ab[a] = d.ab[3 * ic + a];
    }
    const double c1 = d.stepc[2 * r], c2 = d.stepc[2 * r + 1] * d.isqmt[ic];
    const double smt = d.nimt[ic];
    for (int st = 0; st < nsteps; ++st) {
        if (live) {
            // B: the kick of the bonded acceleration of the previous step
#pragma unroll
            for (int a = 0; a < 3; ++a) v[a] = fma(h, ab[a], v[a]);
            // A O A and wrap (as k_aoa)
            const uint32_t s0 = uint32_t(d.step_base[r]) + s_off + uint32_t(st);
#pragma unroll
            for (int a = 0; a < 3; ++a) x[a] = fma(h, v[a], x[a]);
            const U4 u = draw(P, uint32_t(i - P.atom_off), s0, TAG_O, 0, 0, 0);
            const T r0 = d_sqrt(T(-2) * d_log(unif<T>(u.x)));
            const T r1 = d_sqrt(T(-2) * d_log(unif<T>(u.z)));
            T s1, c1v, s2, c2v;
            d_sincospi(T(2) * unif<T>(u.y), &s1, &c1v);
            d_sincospi(T(2) * unif<T>(u.w), &s2, &c2v);
            const double G[3] = {double(r0 * c1v), double(r0 * s1), double(r1 * c2v)};
#pragma unroll
            for (int a = 0; a < 3; ++a) v[a] = fma(c1, v[a], c2 * G[a]);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                x[a] = fma(h, v[a], x[a]);
                if (x[a] < 0.0) { x[a] += P.L; img[a] -= 1; }
                if (x[a] >= P.L) { x[a] -= P.L; img[a] += 1; }
                fin = fin && isfinite(x[a]) && isfinite(v[a]);
                sx[tid][a] = x[a];
            }
        }
        __syncthreads();                // the block's new positions are in shared memory
        for (int k = tid; k < nbt; k += IB_MAX) {
            const int t = d.ib_bond[tb0 + k];
            const int2 ij = d.bond_ij[t];
            bond_term_x(d.P[d.rep[ij.x]], sx[ij.x - b0], sx[ij.y - b0], d.bond_k[t], d.bond_r0[t], sb[k]);
        }
        for (int k = tid; k < nat; k += IB_MAX) {
            const int t = d.ib_ang[ta0 + k];
            const int4 an = d.ang[t];
            angle_term_x(d.P[d.rep[an.y]], sx[an.x - b0], sx[an.y - b0], sx[an.z - b0], d.ang_k[t], d.ang_t0[t], sa[k]);
        }
        __syncthreads();                // every term of the block is evaluated
        if (live) {
            // bonded gradient of atom i: its items in order (as bonded_gather)
            double gx = 0, gy = 0, gz = 0;
            for (int it = d.bi_off[i]; it < d.bi_off[i + 1]; ++it) {
                const int2 item = d.bitem[it];
                const int kind = item.x & 15, role = item.x >> 4, sl = d.item_slot[it];
                if (kind == 0) {
                    const double sgn = role == 0 ? 1.0 : -1.0;
                    gx = fma(sgn, sb[sl][0], gx); gy = fma(sgn, sb[sl][1], gy); gz = fma(sgn, sb[sl][2], gz);
                } else {
                    const double* o = sa[sl];
                    if (role == 0) { gx += o[0]; gy += o[1]; gz += o[2]; }
                    else if (role == 2) { gx += o[3]; gy += o[4]; gz += o[5]; }
                    else { gx -= o[0] + o[3]; gy -= o[1] + o[4]; gz -= o[2] + o[5]; }
                }
            }
            ab[0] = smt * gx; ab[1] = smt * gy; ab[2] = smt * gz;
#pragma unroll
            for (int a = 0; a < 3; ++a) v[a] = fma(h, ab[a], v[a]);
        }
    }
    if (!live) return;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        d.x[3 * i + a] = x[a];
        d.v[3 * i + a] = v[a];
        d.ab[3 * i + a] = ab[a];
        if (img[a]) d.img[3 * i + a] += img[a];
    }
    if (!fin) atomicOr(&d.err[r], F_NONFIN);
    uint4 sp = d.pos[i];
    sp.x = to_scaled(x[0], P); sp.y = to_scaled(x[1], P); sp.z = to_scaled(x[2], P);
    d.pos[i] = sp;
    if (check_last) {
        const double lo = 0.5 * (P.skin_o - P.skin), li = 0.5 * P.skin;
        double t0 = mimg(x[0] - d.xo[3 * i], P), t1 = mimg(x[1] - d.xo[3 * i + 1], P),
               t2 = mimg(x[2] - d.xo[3 * i + 2], P);
        if (t0 * t0 + t1 * t1 + t2 * t2 > lo * lo) {
            d.flags[2 * r + 1] = 1;
            d.flags[2 * r] = 1;
        }
        t0 = mimg(x[0] - d.xb[3 * i], P); t1 = mimg(x[1] - d.xb[3 * i + 1], P);
        t2 = mimg(x[2] - d.xb[3 * i + 2], P);
        if (t0 * t0 + t1 * t1 + t2 * t2 > li * li) d.flags[2 * r] = 1;
    }
}

// energies of the full potential (FP64), kinetic energy; one pass per atom
__global__ void k_energy(Dev d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const int r = d.rep[i];
    const RepParams& P = d.P[r];
    double eb = 0, ea = 0, elj = 0, ec = 0, ke = 0;
    const double3 v = ld3(d.v, i);
    ke = 0.5 * d.mt[i] * (v.x * v.x + v.y * v.y + v.z * v.z);
    for (int it = d.bi_off[i]; it < d.bi_off[i + 1]; ++it) {
        const int2 item = d.bitem[it];
        const int kind = item.x & 15, role = item.x >> 4, t = item.y;
        if (kind == 0 && role == 0) {
            const int2 ij = d.bond_ij[t];
            double dx, dy, dz;
            Disp<double>::get(d, P, ij.x, ij.y, dx, dy, dz);
            const double rr = sqrt(dx * dx + dy * dy + dz * dz) - d.bond_r0[t];
            eb += 0.5 * d.bond_k[t] * rr * rr;
        } else if (kind == 1 && role == 1) {
            const int4 a = d.ang[t];
            double ax, ay, az, bx, by, bz;
            Disp<double>::get(d, P, a.x, a.y, ax, ay, az);
            Disp<double>::get(d, P, a.z, a.y, bx, by, bz);
            double cth = (ax * bx + ay * by + az * bz) /
                         (sqrt(ax * ax + ay * ay + az * az) * sqrt(bx * bx + by * by + bz * bz));
            cth = fmin(1.0, fmax(-1.0, cth));
            const double dt = acos(cth) - d.ang_t0[t];
            ea += 0.5 * d.ang_k[t] * dt * dt;
        }
    }
    const int n = min(d.ocnt[i], d.ocap);
    const uint32_t* row = d.olist + (size_t)i * d.ocap;
    const int ti = d.type[i];
    for (int k = 0; k < n; ++k) {
        const int j = int(row[k]);
        if (j <= i) continue;
        double dx, dy, dz;
        Disp<double>::get(d, P, i, j, dx, dy, dz);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= P.R * P.R) continue;
        const double rr = sqrt(r2), rinv = 1.0 / rr;
        const double qq = d.q[i] * d.q[j];
        if (qq != 0.0) {
            double uc, duc;
            dsf<double>(P, rr, rinv, uc, duc);
            ec += COULOMB * qq * uc;
        }
        const LJPair& lj = P.lj[ti * MAX_TYPES + d.type[j]];
        if (lj.on) {
            double ul, dul;
            ljsf<double>(P, lj, rr, rinv, ul, dul);
            elj += ul;
        }
    }
    double* E = d.energy + 6 * r;
    if (eb != 0) atomicAdd(&E[0], eb);
    if (ea != 0) atomicAdd(&E[1], ea);
    if (elj != 0) atomicAdd(&E[2], elj);
    if (ec != 0) atomicAdd(&E[3], ec);
    atomicAdd(&E[4], ke);
}

__global__ void k_advance(Dev d, long long n)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < d.R) d.step_base[r] += n;
}

inline int blocks(long long n, int b) { return int((n + b - 1) / b); }

template <typename T, int W, bool B>
void force_tpa(const Dev& d, int lk, double* out, int as_grad, int tpa, cudaStream_t s)
{
    const long long threads = (long long)d.N * tpa;
    switch (tpa) {
    case 1: k_force<T, W, B, 1><<<blocks(threads, 128), 128, 0, s>>>(d, lk, out, as_grad); break;
    case 2: k_force<T, W, B, 2><<<blocks(threads, 128), 128, 0, s>>>(d, lk, out, as_grad); break;
    case 4: k_force<T, W, B, 4><<<blocks(threads, 128), 128, 0, s>>>(d, lk, out, as_grad); break;
    default: k_force<T, W, B, 8><<<blocks(threads, 128), 128, 0, s>>>(d, lk, out, as_grad); break;
    }
}

// half-list form (mixed mode): the pair kernel, then the conversion
template <int W, bool B>
void force_half(const Dev& d, int lk, double* out, int as_grad, int tpa, cudaStream_t s)
{
    const long long threads = (long long)d.N * tpa;
    switch (tpa) {
    case 1: k_force_half<W, 1><<<blocks(threads, 128), 128, 0, s>>>(d, lk); break;
    case 2: k_force_half<W, 2><<<blocks(threads, 128), 128, 0, s>>>(d, lk); break;
    case 4: k_force_half<W, 4><<<blocks(threads, 128), 128, 0, s>>>(d, lk); break;
    default: k_force_half<W, 8><<<blocks(threads, 128), 128, 0, s>>>(d, lk); break;
    }
    k_force_finish<B><<<blocks(d.N, 256), 256, 0, s>>>(d, out, as_grad);
}

// cluster-tile list of a gradient mode: 0 short radius, 1 full radius, -1 none
inline int tile_list_of(int mode)
{
    if (mode == 3 || mode == 5) return 0;
    if (mode == 0 || mode == 2 || mode == 4) return 1;
    return -1;
}

template <int W, bool B>
void force_tile(const Dev& d, int tl, double* out, int as_grad, cudaStream_t s)
{
    static int per_sm = 0, sms = 0;
    if (!per_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_force_tile<W>, 128, 0);
        per_sm = per_sm > 0 ? per_sm : 1;
    }
    const int want = (d.ncl_cap + 3) / 4;
    const int g = want < sms * per_sm ? want : sms * per_sm;
    k_force_tile<W><<<g > 0 ? g : 1, 128, 0, s>>>(d, tl);
    k_force_finish<B><<<blocks(d.N, 256), 256, 0, s>>>(d, out, as_grad);
}

template <typename T>
int force_t(const Dev& d, int mode, double* out, int as_grad, int tpa, cudaStream_t s)
{
    const bool bonded = mode == 0 || mode == 1 || mode == 5;
    if (bonded && d.nbond + d.nang > 0)
        k_bonded_terms<<<blocks(d.nbond + d.nang, 128), 128, 0, s>>>(d);
    int nk = (bonded && d.nbond + d.nang > 0) ? 2 : 1;
    // the half-list kernels (tpa | FORCE_HALF) serve the full, short and long
    // pair weights of mixed mode; the short weight of replicas that keep the LJ
    // long part deterministic also runs over the LJ list and stays full
    const int tl = tile_list_of(mode);
    const bool tile = (tpa & FORCE_TILE) && sizeof(T) == 4 && force_half_ok(d, mode) && tl >= 0 &&
                      ((d.tiles >> tl) & 1);
    if (tile) {
        nk += 2;
        switch (mode) {
        case 0: force_tile<W_FULL, true>(d, tl, out, as_grad, s); break;
        case 2: force_tile<W_FULL, false>(d, tl, out, as_grad, s); break;
        case 3: force_tile<W_SHORT, false>(d, tl, out, as_grad, s); break;
        case 4: force_tile<W_LONG, false>(d, tl, out, as_grad, s); break;
        default: force_tile<W_SHORT, true>(d, tl, out, as_grad, s); break;
        }
        return nk;
    }
    const bool half = (tpa & FORCE_HALF) && sizeof(T) == 4 && force_half_ok(d, mode);
    const int t = tpa & ~(FORCE_HALF | FORCE_TILE);
    if (half) {
        nk += 1;
        switch (mode) {
        case 0: force_half<W_FULL, true>(d, L_FULL, out, as_grad, t, s); break;
        case 2: force_half<W_FULL, false>(d, L_FULL, out, as_grad, t, s); break;
        case 3: force_half<W_SHORT, false>(d, L_SHORT, out, as_grad, t, s); break;
        case 4: force_half<W_LONG, false>(d, L_FULL, out, as_grad, t, s); break;
        case 7: force_half<W_LJLONG, false>(d, L_LJ, out, as_grad, t, s); break;
        default: force_half<W_SHORT, true>(d, L_SHORT, out, as_grad, t, s); break;
        }
        return nk;
    }
    switch (mode) {
    case 0: force_tpa<T, W_FULL, true>(d, L_FULL, out, as_grad, t, s); break;
    case 1: k_bonded<<<blocks(d.N, 256), 256, 0, s>>>(d, out, as_grad, 0.0); break;
    case 2: force_tpa<T, W_FULL, false>(d, L_FULL, out, as_grad, t, s); break;
    case 3: force_tpa<T, W_SHORT, false>(d, L_SHORT, out, as_grad, t, s); break;
    case 4: force_tpa<T, W_LONG, false>(d, L_FULL, out, as_grad, t, s); break;
    case 7: force_tpa<T, W_LJLONG, false>(d, L_LJ, out, as_grad, t, s); break;
    default: force_tpa<T, W_SHORT, true>(d, L_SHORT, out, as_grad, t, s); break;
    }
    return nk;
}

}  // namespace

int launch_force(const Dev& d, int mode, double* out, int as_grad, int fp64, int tpa, cudaStream_t s)
{
    return fp64 ? force_t<double>(d, mode, out, as_grad, tpa, s) : force_t<float>(d, mode, out, as_grad, tpa, s);
}

void launch_kick(const Dev& d, const double* a, double h, cudaStream_t s)
{
    k_kick<<<blocks(3LL * d.N, 256), 256, 0, s>>>(d, a, h);
}

void launch_kick2(const Dev& d, const double* a, double h, const double* b, double hb, cudaStream_t s)
{
    k_kick2<<<blocks(3LL * d.N, 256), 256, 0, s>>>(d, a, h, b, hb);
}

void launch_inner_steps(const Dev& d, double dt, uint32_t s_off, int nsteps, int check_last, int fp64, cudaStream_t s)
{
    if (fp64) k_inner_steps<double><<<d.n_ib, IB_MAX, 0, s>>>(d, dt, s_off, nsteps, check_last);
    else k_inner_steps<float><<<d.n_ib, IB_MAX, 0, s>>>(d, dt, s_off, nsteps, check_last);
}

void launch_aoa(const Dev& d, double tau, uint32_t s_off, int do_check, int fp64, cudaStream_t s,
                const double* pre_a, double pre_h)
{
    if (fp64) k_aoa<double><<<blocks(d.N, 256), 256, 0, s>>>(d, tau, s_off, do_check, pre_a, pre_h);
    else k_aoa<float><<<blocks(d.N, 256), 256, 0, s>>>(d, tau, s_off, do_check, pre_a, pre_h);
}

void launch_bonded_kick(const Dev& d, double* out, double kick_h, cudaStream_t s)
{
    if (d.nbond + d.nang > 0) k_bonded_terms<<<blocks(d.nbond + d.nang, 128), 128, 0, s>>>(d);
    k_bonded<<<blocks(d.N, 256), 256, 0, s>>>(d, out, 0, kick_h);
}

void launch_energy(const Dev& d, cudaStream_t s)
{
    k_energy<<<blocks(d.N, 128), 128, 0, s>>>(d);
}

void launch_advance(const Dev& d, long long nsteps, cudaStream_t s)
{
    k_advance<<<blocks(d.R, 128), 128, 0, s>>>(d, nsteps);
}

}  // namespace mdj
