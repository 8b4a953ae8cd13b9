// k_pme.cu -- the reciprocal part of Ewald electrostatics by smooth particle
// mesh Ewald (Essmann et al., J. Chem. Phys. 103, 8577 (1995)), for replicas
// whose pair Coulomb is the Ewald real-space term erfc(a r)/r of Sec. 3.1.
// The reciprocal part is a slow many-body force: it is not jumped but kept
// deterministic (in F0 for JUMP, at the outer step of JUMP-RESPA1, Sec. 2.3).
// Spread and gather take their B-spline weights in the path's precision
// (FP64, or FP32 in mixed mode); grids, transforms and G are FP64.
//
// Charges are spread with cardinal B-splines M_p onto a K^3 grid in 64-bit
// fixed point (order independent), converted to a real grid, transformed
// (cuFFT, driven by the host), multiplied by
//   G(m) = (C / (pi V)) exp(-pi^2 |m|^2 / a^2) / |m|^2 |b(m)|^2,
// transformed back to the potential grid phi = dE/dQ, and the gradient of
// each atom gathered from phi with the derivative of M_p. Excluded pairs,
// which the reciprocal sum still couples, get -C q_i q_j erf(a r)/r back.
#include "engine.h"

namespace mdj {

namespace {

// fixed-point unit of the charge grid: 2^-48 e (grid values up to 2^15 e in magnitude)
constexpr double PME_FIX = 281474976710656.0;
constexpr int PME_PMAX = 8;

// M_p(u) and M_p'(u) for u = f + t, t = 0 .. p-1, f in [0, 1): the p weights
// of one coordinate, by the B-spline recursion
template <typename T>
__device__ __forceinline__ void bspline_weights(int p, T f, T* M, T* dM)
{
    // order 2: M_2(f + t) = {f, 1 - f} for t = 0, 1 (t indexes the distance k0 - k)
    T w[PME_PMAX];
    w[0] = f;
    w[1] = T(1) - f;
    for (int n = 3; n <= p; ++n) {
        if (n == p)
            for (int t = 0; t < n; ++t) dM[t] = (t < n - 1 ? w[t] : T(0)) - (t > 0 ? w[t - 1] : T(0));
        // M_n(u) = (u M_{n-1}(u) + (n - u) M_{n-1}(u - 1)) / (n - 1), u = f + t
        T nw[PME_PMAX];
        for (int t = 0; t < n; ++t) {
            const T u = f + T(t);
            const T a = t < n - 1 ? w[t] : T(0);        // M_{n-1}(u)
            const T b = t > 0 ? w[t - 1] : T(0);        // M_{n-1}(u - 1)
            nw[t] = (u * a + (T(n) - u) * b) / T(n - 1);
        }
        for (int t = 0; t < n; ++t) w[t] = nw[t];
    }
    for (int t = 0; t < p; ++t) M[t] = w[t];
}

template <typename T>
__global__ void k_pme_spread(Dev d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const RepParams& P = d.P[d.rep[i]];
    if (P.coul_mode != 1) return;
    const int p = P.pme_p, K = P.pme_K;
    const double q = d.q[i];
    if (q == 0.0) return;
    int k0[3];
    T M[3][PME_PMAX], dM[3][PME_PMAX];
    for (int c = 0; c < 3; ++c) {
        double x = d.x[3 * i + c];
        x -= P.L * floor(x * P.invL);
        const double u = K * x * P.invL;
        k0[c] = int(floor(u));
        bspline_weights<T>(p, T(u - k0[c]), M[c], dM[c]);
    }
    unsigned long long* g = d.pme_qi + P.pme_goff;
    for (int t2 = 0; t2 < p; ++t2) {
        const int z = ((k0[2] - t2) % K + K) % K;
        for (int t1 = 0; t1 < p; ++t1) {
            const int y = ((k0[1] - t1) % K + K) % K;
            const T w21 = M[2][t2] * M[1][t1];
            for (int t0 = 0; t0 < p; ++t0) {
                const int x = ((k0[0] - t0) % K + K) % K;
                const double w = double(w21 * M[0][t0]) * q;
                atomicAdd(&g[((long long)z * K + y) * K + x], (unsigned long long)(long long)llrint(w * PME_FIX));
            }
        }
    }
}

// fixed point to the real grid of the forward transform; clears the fixed-point grid
__global__ void k_pme_tofloat(Dev d, long long total)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total) return;
    d.pme_q[k] = double((long long)d.pme_qi[k]) / PME_FIX;
    d.pme_qi[k] = 0ull;
}

// one block per (replica, plane m2): spectrum times G; the energy sums the
// full spectrum through the half the real-to-complex transform keeps
__global__ void k_pme_convolve(Dev d, int energy)
{
    const int r = blockIdx.y;
    const RepParams& P = d.P[r];
    if (P.coul_mode != 1) return;
    const int K = P.pme_K, Kh = K / 2 + 1;
    const int m2 = blockIdx.x;
    if (m2 >= K) return;
    double e = 0.0;
    for (int t = threadIdx.x; t < K * Kh; t += blockDim.x) {
        const long long k = P.pme_soff + ((long long)m2 * K) * Kh + t;
        const double G = d.pme_G[k];
        double2 z = d.pme_spec[k];
        if (energy) {
            const int m0 = t % Kh;
            const double w = (m0 == 0 || (K % 2 == 0 && m0 == K / 2)) ? 1.0 : 2.0;
            e += 0.5 * w * G * (z.x * z.x + z.y * z.y);
        }
        z.x *= G;
        z.y *= G;
        d.pme_spec[k] = z;
    }
    if (energy) {
        for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&d.pme_e[r], e);
    }
}

// gradient of atom i: reciprocal sum from phi (the inverse transform, which
// holds dE/dQ) plus the exclusion correction; added to out
template <typename T>
__global__ void k_pme_gather(Dev d, double* out, int as_grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const RepParams& P = d.P[d.rep[i]];
    if (P.coul_mode != 1) return;
    const int p = P.pme_p, K = P.pme_K;
    const double q = d.q[i];
    double gx = 0.0, gy = 0.0, gz = 0.0;
    if (q != 0.0) {
        int k0[3];
        T M[3][PME_PMAX], dM[3][PME_PMAX];
        for (int c = 0; c < 3; ++c) {
            double x = d.x[3 * i + c];
            x -= P.L * floor(x * P.invL);
            const double u = K * x * P.invL;
            k0[c] = int(floor(u));
            bspline_weights<T>(p, T(u - k0[c]), M[c], dM[c]);
        }
        const double* phi = d.pme_q + P.pme_goff;
        T ax = T(0), ay = T(0), az = T(0);
        for (int t2 = 0; t2 < p; ++t2) {
            const int z = ((k0[2] - t2) % K + K) % K;
            for (int t1 = 0; t1 < p; ++t1) {
                const int y = ((k0[1] - t1) % K + K) % K;
                for (int t0 = 0; t0 < p; ++t0) {
                    const int x = ((k0[0] - t0) % K + K) % K;
                    const T ph = T(phi[((long long)z * K + y) * K + x]);
                    ax += dM[0][t0] * M[1][t1] * M[2][t2] * ph;
                    ay += M[0][t0] * dM[1][t1] * M[2][t2] * ph;
                    az += M[0][t0] * M[1][t1] * dM[2][t2] * ph;
                }
            }
        }
        // dQ(k)/dx = q (K / L) M_p'(u - k) ...: dM above is dM/du, and u - k = f + t
        const double s = q * K * P.invL;
        gx = s * double(ax); gy = s * double(ay); gz = s * double(az);
        // excluded partners: d/dr [-C q_i q_j erf(a r)/r]
        const double a = P.alpha;
        for (int e = d.ex_off[i]; e < d.ex_off[i + 1]; ++e) {
            const int j = d.ex_idx[e];
            double dx = d.x[3 * i] - d.x[3 * j], dy = d.x[3 * i + 1] - d.x[3 * j + 1], dz = d.x[3 * i + 2] - d.x[3 * j + 2];
            dx -= P.L * rint(dx * P.invL); dy -= P.L * rint(dy * P.invL); dz -= P.L * rint(dz * P.invL);
            const double r = sqrt(dx * dx + dy * dy + dz * dz);
            const double qq = COULOMB * q * d.q[j];
            const double dudr = qq * (erf(a * r) / (r * r) - P.kexp * exp(-a * a * r * r) / r);
            gx += dudr * dx / r; gy += dudr * dy / r; gz += dudr * dz / r;
        }
    }
    const double sc = as_grad ? 1.0 : -1.0 / d.mt[i];
    out[3 * i] += sc * gx; out[3 * i + 1] += sc * gy; out[3 * i + 2] += sc * gz;
}

__global__ void k_pme_excl_energy(Dev d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const int r = d.rep[i];
    const RepParams& P = d.P[r];
    if (P.coul_mode != 1) return;
    double e = 0.0;
    for (int k = d.ex_off[i]; k < d.ex_off[i + 1]; ++k) {
        const int j = d.ex_idx[k];
        if (j <= i) continue;
        double dx = d.x[3 * i] - d.x[3 * j], dy = d.x[3 * i + 1] - d.x[3 * j + 1], dz = d.x[3 * i + 2] - d.x[3 * j + 2];
        dx -= P.L * rint(dx * P.invL); dy -= P.L * rint(dy * P.invL); dz -= P.L * rint(dz * P.invL);
        const double rr = sqrt(dx * dx + dy * dy + dz * dz);
        e -= COULOMB * d.q[i] * d.q[j] * erf(P.alpha * rr) / rr;
    }
    if (e != 0.0) atomicAdd(&d.energy[6 * r + 3], e);
}

inline int blocks(long long n, int b) { return int((n + b - 1) / b); }

}  // namespace

void launch_pme_spread(const Dev& d, int fp64, cudaStream_t s)
{
    if (fp64) k_pme_spread<double><<<blocks(d.N, 128), 128, 0, s>>>(d);
    else k_pme_spread<float><<<blocks(d.N, 128), 128, 0, s>>>(d);
}

void launch_pme_tofloat(const Dev& d, long long total, cudaStream_t s)
{
    k_pme_tofloat<<<blocks(total, 256), 256, 0, s>>>(d, total);
}

void launch_pme_convolve_grid(const Dev& d, int energy, int kmax, cudaStream_t s)
{
    k_pme_convolve<<<dim3(kmax, d.R), 256, 0, s>>>(d, energy);
}

void launch_pme_gather(const Dev& d, double* out, int as_grad, int fp64, cudaStream_t s)
{
    if (fp64) k_pme_gather<double><<<blocks(d.N, 128), 128, 0, s>>>(d, out, as_grad);
    else k_pme_gather<float><<<blocks(d.N, 128), 128, 0, s>>>(d, out, as_grad);
}

void launch_pme_excl_energy(const Dev& d, cudaStream_t s)
{
    k_pme_excl_energy<<<blocks(d.N, 128), 128, 0, s>>>(d);
}

}  // namespace mdj
