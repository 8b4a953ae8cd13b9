// k_pme.cu -- the reciprocal part of Ewald electrostatics by smooth particle
// mesh Ewald (Essmann et al., J. Chem. Phys. 103, 8577 (1995)), for replicas
// whose pair Coulomb is the Ewald real-space term erfc(a r)/r of Sec. 3.1.
// The reciprocal part is a slow many-body force: it is not jumped but kept
// deterministic (in F0 for JUMP, at the outer step of JUMP-RESPA1, Sec. 2.3).
// FP64 mode runs every step in double precision. Mixed mode has no FP64
// arithmetic in the hot loops (FP64 runs at a small fraction of the FP32 rate
// on this GPU): grid coordinates come exactly from the 32-bit scaled
// positions, B-spline weights and the gather are FP32, charge contributions
// are summed exactly in split 32-bit integers in shared memory, and the grid,
// the transforms and G are FP32.
//
// Charges are spread with cardinal B-splines M_p onto a K^3 grid in 64-bit
// fixed point (order independent), converted to a real grid, transformed
// (cuFFT, driven by the host), multiplied by
//   G(m) = (C / (pi V)) exp(-pi^2 |m|^2 / a^2) / |m|^2 |b(m)|^2,
// transformed back to the potential grid phi = dE/dQ, and the gradient of
// each atom gathered from phi with the derivative of M_p. Excluded pairs,
// which the reciprocal sum still couples, get -C q_i q_j erf(a r)/r back.
#include <algorithm>

#include "engine.h"

namespace mdj {

namespace {

// fixed-point unit of the FP64 charge grid: 2^-50 e (grid values up to 2^13 e in
// magnitude: hundreds of times the charge a grid point gathers in a liquid)
constexpr double PME_FIX = 1125899906842624.0;
constexpr int PME_THREADS = 128;
constexpr int PME_CHUNK = 64;           // atoms staged in shared memory at a time

// M_p(f + t) and M_p'(f + t), t = 0 .. P-1, f in [0, 1]: the weights of one
// coordinate, by the B-spline recursion M_n(u) = (u M_{n-1}(u) + (n - u) M_{n-1}(u - 1)) / (n - 1)
// from M_2(f) = f, M_2(1 + f) = 1 - f, and M_n'(u) = M_{n-1}(u) - M_{n-1}(u - 1)
template <typename T, int P>
__device__ __forceinline__ void bspline_weights(T f, T* M, T* dM)
{
    T w[P];
    w[0] = f;
    w[1] = T(1) - f;
#pragma unroll
    for (int n = 3; n <= P; ++n) {
        if (n == P) {
#pragma unroll
            for (int t = 0; t < n; ++t) dM[t] = (t < n - 1 ? w[t] : T(0)) - (t > 0 ? w[t - 1] : T(0));
        }
        T nw[P];
#pragma unroll
        for (int t = 0; t < n; ++t) {
            const T u = f + T(t);
            const T a = t < n - 1 ? w[t] : T(0);
            const T b = t > 0 ? w[t - 1] : T(0);
            nw[t] = (u * a + (T(n) - u) * b) / T(n - 1);
        }
#pragma unroll
        for (int t = 0; t < n; ++t) w[t] = nw[t];
    }
#pragma unroll
    for (int t = 0; t < P; ++t) M[t] = w[t];
}

// grid coordinate of one axis: u = K x / L with x wrapped into the box, k0 = floor(u) in [0, K)
__device__ __forceinline__ void grid_coord(const RepParams& P, double x, int& k0, double& f)
{
    x -= P.L * floor(x * P.invL);
    const double u = P.pme_K * x * P.invL;
    const double fl = floor(u);
    k0 = int(fl);
    f = u - fl;
    if (k0 >= P.pme_K) k0 -= P.pme_K;     // x rounded up to L: the point 0, same weights
    if (!(k0 >= 0 && k0 < P.pme_K)) k0 = 0;   // non-finite x (flagged by the A O A update): in range
}

__device__ __forceinline__ int wrap_k(int g, int K) { return g < 0 ? g + K : (g >= K ? g - K : g); }

// mixed mode: the same from the 32-bit scaled coordinate s = x 2^32 / L
// (exact integer k0; f rounded once to FP32, f in [0, 1])
__device__ __forceinline__ void grid_coord_fix(const RepParams& P, uint32_t s, int& k0, float& f)
{
    const unsigned long long prod = (unsigned long long)s * (unsigned long long)P.pme_K;
    k0 = int(prod >> 32);
    f = __uint2float_rn(uint32_t(prod)) * 2.3283064365386963e-10f;
}

__device__ __forceinline__ uint32_t comp(const uint4& p, int c) { return c == 0 ? p.x : (c == 1 ? p.y : p.z); }

// ---- binning: atoms ordered by brick (count, scan, place) ----------------------------------
template <bool FIX>
__global__ void k_pme_count(Dev d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const RepParams& P = d.P[d.rep[i]];
    if (P.coul_mode != 1) { d.pme_brick[i] = -1; return; }
    const uint4 ps = FIX ? d.pos[i] : make_uint4(0, 0, 0, 0);
    int b = 0;
    for (int c = 2; c >= 0; --c) {
        int k0;
        if (FIX) {
            float f;
            grid_coord_fix(P, comp(ps, c), k0, f);
        } else {
            double f;
            grid_coord(P, d.x[3 * i + c], k0, f);
        }
        b = b * P.pme_nb + k0 / PME_BRICK;
    }
    b += P.pme_boff;
    d.pme_brick[i] = b;
    d.pme_slot[i] = atomicAdd(&d.pme_bcnt[b], 1);
}

// one block: exclusive scan of the brick counts into pme_bstart; clears the counts
__global__ void __launch_bounds__(1024) k_pme_scan(Dev d)
{
    __shared__ int part[1024];
    const int nb = d.pme_nbricks, t = threadIdx.x;
    const int per = (nb + 1023) / 1024;
    const int lo = min(nb, t * per), hi = min(nb, lo + per);
    int sum = 0;
    for (int b = lo; b < hi; ++b) sum += d.pme_bcnt[b];
    part[t] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - sum;
    for (int b = lo; b < hi; ++b) {
        d.pme_bstart[b] = run;
        run += d.pme_bcnt[b];
        d.pme_bcnt[b] = 0;
    }
    if (t == 1023) d.pme_bstart[nb] = part[1023];
}

__global__ void k_pme_place(Dev d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const int b = d.pme_brick[i];
    if (b >= 0) d.pme_sorted[d.pme_bstart[b] + d.pme_slot[i]] = i;
}

// brick of a block and the origin of its region: the region holds the grid
// points k0 - t (t < P) of the atoms whose k0 lies in the brick
struct BrickRegion {
    int o[3];
    int start, end;
};

__device__ __forceinline__ BrickRegion brick_region(const Dev& d, const RepParams& P, int b, int order)
{
    BrickRegion R;
    const int lb = b - P.pme_boff, nb = P.pme_nb;
    R.o[0] = (lb % nb) * PME_BRICK - (order - 1);
    R.o[1] = ((lb / nb) % nb) * PME_BRICK - (order - 1);
    R.o[2] = (lb / (nb * nb)) * PME_BRICK - (order - 1);
    R.start = d.pme_bstart[b];
    R.end = d.pme_bstart[b + 1];
    return R;
}

// ---- spread: block per brick, shared fixed-point accumulation ------------------------------
template <typename T, int P>
__global__ void __launch_bounds__(PME_THREADS) k_pme_spread(Dev d)
{
    constexpr int S = PME_BRICK + P - 1;
    __shared__ unsigned long long acc[S * S * S];
    __shared__ T wsh[PME_CHUNK][3][P];
    __shared__ int ksh[PME_CHUNK][3];
    __shared__ double qsh[PME_CHUNK];
    const int b = blockIdx.x;
    const RepParams& Pr = d.P[d.pme_brick_rep[b]];
    if (Pr.pme_p != P) return;
    const BrickRegion R = brick_region(d, Pr, b, P);
    if (R.end == R.start) return;
    for (int k = threadIdx.x; k < S * S * S; k += PME_THREADS) acc[k] = 0ull;
    for (int c0 = R.start; c0 < R.end; c0 += PME_CHUNK) {
        const int n = min(PME_CHUNK, R.end - c0);
        __syncthreads();
        if (threadIdx.x < n) {
            const int i = d.pme_sorted[c0 + threadIdx.x];
            for (int c = 0; c < 3; ++c) {
                int k0;
                double f;
                grid_coord(Pr, d.x[3 * i + c], k0, f);
                T M[P], dM[P];
                bspline_weights<T, P>(T(f), M, dM);
#pragma unroll
                for (int t = 0; t < P; ++t) wsh[threadIdx.x][c][t] = M[t];
                ksh[threadIdx.x][c] = k0 - R.o[c];      // in [P - 1, P - 1 + PME_BRICK)
            }
            qsh[threadIdx.x] = d.q[i];
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < n * P * P; idx += PME_THREADS) {
            const int a = idx / (P * P), rem = idx - a * (P * P);
            const int t2 = rem / P, t1 = rem - t2 * P;
            const int base = ((ksh[a][2] - t2) * S + (ksh[a][1] - t1)) * S + ksh[a][0];
            const T wzy = wsh[a][2][t2] * wsh[a][1][t1];
            const double q = qsh[a];
#pragma unroll
            for (int t0 = 0; t0 < P; ++t0) {
                const double w = double(wzy * wsh[a][0][t0]) * q;
                atomicAdd(&acc[base - t0], (unsigned long long)(long long)llrint(w * PME_FIX));
            }
        }
    }
    __syncthreads();
    const int K = Pr.pme_K;
    unsigned long long* g = d.pme_qi + Pr.pme_goff;
    for (int k = threadIdx.x; k < S * S * S; k += PME_THREADS) {
        const unsigned long long v = acc[k];
        if (!v) continue;
        const int rz = k / (S * S), ry = (k / S) % S, rx = k % S;
        const int gz = wrap_k(R.o[2] + rz, K), gy = wrap_k(R.o[1] + ry, K), gx = wrap_k(R.o[0] + rx, K);
        atomicAdd(&g[((long long)gz * K + gy) * K + gx], v);
    }
}

// mixed mode: FP32 weights; each contribution w (units of e) is rounded once
// to a multiple of 2^-40 e and split as a 2^-16 + b 2^-40, a = rint(w 2^16),
// b = rint((w 2^16 - a) 2^24) (|b| <= 2^23; the subtraction is exact), summed
// in two 32-bit shared counters: exact, so independent of the order. The low
// counter is folded into the high one after each chunk of atoms.
template <int P>
__global__ void __launch_bounds__(PME_THREADS) k_pme_spread_fix(Dev d)
{
    constexpr int S = PME_BRICK + P - 1;
    static_assert(PME_CHUNK < 256, "low counters hold fewer than 256 contributions");
    __shared__ int hi[S * S * S];
    __shared__ int lo[S * S * S];
    __shared__ float wsh[PME_CHUNK][3][P];
    __shared__ int ksh[PME_CHUNK][3];
    __shared__ float qsh[PME_CHUNK];
    const int b = blockIdx.x;
    const RepParams& Pr = d.P[d.pme_brick_rep[b]];
    if (Pr.pme_p != P) return;
    const BrickRegion R = brick_region(d, Pr, b, P);
    if (R.end == R.start) return;
    for (int k = threadIdx.x; k < S * S * S; k += PME_THREADS) { hi[k] = 0; lo[k] = 0; }
    for (int c0 = R.start; c0 < R.end; c0 += PME_CHUNK) {
        const int n = min(PME_CHUNK, R.end - c0);
        __syncthreads();
        if (c0 > R.start)
            for (int k = threadIdx.x; k < S * S * S; k += PME_THREADS) {
                hi[k] += lo[k] >> 24;
                lo[k] &= 0xffffff;
            }
        if (threadIdx.x < n) {
            const int i = d.pme_sorted[c0 + threadIdx.x];
            const uint4 ps = d.pos[i];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                int k0;
                float f;
                grid_coord_fix(Pr, comp(ps, c), k0, f);
                float M[P], dM[P];
                bspline_weights<float, P>(f, M, dM);
#pragma unroll
                for (int t = 0; t < P; ++t) wsh[threadIdx.x][c][t] = M[t];
                ksh[threadIdx.x][c] = k0 - R.o[c];
            }
            qsh[threadIdx.x] = __uint_as_float(ps.w);
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < n * P * P; idx += PME_THREADS) {
            const int a = idx / (P * P), rem = idx - a * (P * P);
            const int t2 = rem / P, t1 = rem - t2 * P;
            const int base = ((ksh[a][2] - t2) * S + (ksh[a][1] - t1)) * S + ksh[a][0];
            const float wzyq = wsh[a][2][t2] * wsh[a][1][t1] * qsh[a];
#pragma unroll
            for (int t0 = 0; t0 < P; ++t0) {
                const float t = wzyq * wsh[a][0][t0] * 65536.0f;
                const float ah = rintf(t);
                atomicAdd(&hi[base - t0], __float2int_rn(ah));
                atomicAdd(&lo[base - t0], __float2int_rn((t - ah) * 16777216.0f));
            }
        }
    }
    __syncthreads();
    const int K = Pr.pme_K;
    unsigned long long* g = d.pme_qi + Pr.pme_goff;
    for (int k = threadIdx.x; k < S * S * S; k += PME_THREADS) {
        const long long v = (long long)hi[k] * 16777216ll + (long long)lo[k];
        if (!v) continue;
        const int rz = k / (S * S), ry = (k / S) % S, rx = k % S;
        const int gz = wrap_k(R.o[2] + rz, K), gy = wrap_k(R.o[1] + ry, K), gx = wrap_k(R.o[0] + rx, K);
        atomicAdd(&g[((long long)gz * K + gy) * K + gx], (unsigned long long)v);
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

// mixed mode: fixed point (units 2^-40 e) to an FP32 real grid
__global__ void k_pme_tofloat_fix(Dev d, long long total)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total) return;
    reinterpret_cast<float*>(d.pme_q)[k] = __ll2float_rn((long long)d.pme_qi[k]) * 9.094947017729282e-13f;
    d.pme_qi[k] = 0ull;
}

// spectrum times G, one replica per grid row y; the energy sums the full
// spectrum through the half the real-to-complex transform keeps
__global__ void k_pme_convolve(Dev d, int energy)
{
    const int r = blockIdx.y;
    const RepParams& P = d.P[r];
    if (P.coul_mode != 1) return;
    const int K = P.pme_K, Kh = K / 2 + 1;
    const long long n = (long long)K * K * Kh;
    double e = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const long long k = P.pme_soff + t;
        const double G = d.pme_G[k];
        double2 z = d.pme_spec[k];
        if (energy) {
            const int m0 = int(t % Kh);
            const double w = (m0 == 0 || (K % 2 == 0 && m0 == K / 2)) ? 1.0 : 2.0;
            e += 0.5 * w * G * (z.x * z.x + z.y * z.y);
        }
        z.x *= G;
        z.y *= G;
        d.pme_spec[k] = z;
    }
    if (energy) {
        for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
        if ((threadIdx.x & 31) == 0 && e != 0.0) atomicAdd(&d.pme_e[r], e);
    }
}

// mixed mode: FP32 spectrum times FP32 G (the energy, for observables only, in FP64)
__global__ void k_pme_convolve_fix(Dev d, int energy)
{
    const int r = blockIdx.y;
    const RepParams& P = d.P[r];
    if (P.coul_mode != 1) return;
    const int K = P.pme_K, Kh = K / 2 + 1;
    const long long n = (long long)K * K * Kh;
    float2* spec = reinterpret_cast<float2*>(d.pme_spec) + P.pme_soff;
    const float* G = d.pme_Gf + P.pme_soff;
    double e = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const float g = G[t];
        float2 z = spec[t];
        if (energy) {
            const int m0 = int(t % Kh);
            const double w = (m0 == 0 || (K % 2 == 0 && m0 == K / 2)) ? 1.0 : 2.0;
            e += 0.5 * w * double(g) * (double(z.x) * z.x + double(z.y) * z.y);
        }
        z.x *= g;
        z.y *= g;
        spec[t] = z;
    }
    if (energy) {
        for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
        if ((threadIdx.x & 31) == 0 && e != 0.0) atomicAdd(&d.pme_e[r], e);
    }
}

template <typename T> __device__ __forceinline__ T erf_t(T x);
template <> __device__ __forceinline__ double erf_t<double>(double x) { return erf(x); }
template <> __device__ __forceinline__ float erf_t<float>(float x) { return erff(x); }
template <typename T> __device__ __forceinline__ T exp_t(T x);
template <> __device__ __forceinline__ double exp_t<double>(double x) { return exp(x); }
template <> __device__ __forceinline__ float exp_t<float>(float x) { return expf(x); }
template <typename T> __device__ __forceinline__ T sqrt_t(T x);
template <> __device__ __forceinline__ double sqrt_t<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float sqrt_t<float>(float x) { return sqrtf(x); }

// ---- gather: block per brick, the potential grid of the region in shared memory ------------
// gradient of atom i: reciprocal sum from phi (which holds dE/dQ) plus the
// exclusion correction d/dr [-C q_i q_j erf(a r)/r]; added to out
template <typename T, int P>
__global__ void __launch_bounds__(PME_THREADS) k_pme_gather(Dev d, double* out, int as_grad)
{
    constexpr int S = PME_BRICK + P - 1;
    __shared__ T ph[S * S * S];
    const int b = blockIdx.x;
    const RepParams& Pr = d.P[d.pme_brick_rep[b]];
    if (Pr.pme_p != P) return;
    const BrickRegion R = brick_region(d, Pr, b, P);
    if (R.end == R.start) return;
    const int K = Pr.pme_K;
    const double* phi = d.pme_q + Pr.pme_goff;
    for (int k = threadIdx.x; k < S * S * S; k += PME_THREADS) {
        const int rz = k / (S * S), ry = (k / S) % S, rx = k % S;
        const int gz = wrap_k(R.o[2] + rz, K), gy = wrap_k(R.o[1] + ry, K), gx = wrap_k(R.o[0] + rx, K);
        ph[k] = T(phi[((long long)gz * K + gy) * K + gx]);
    }
    __syncthreads();
    for (int a = R.start + threadIdx.x; a < R.end; a += PME_THREADS) {
        const int i = d.pme_sorted[a];
        const double q = d.q[i];
        double gx = 0.0, gy = 0.0, gz = 0.0;
        if (q != 0.0) {
            T M[3][P], dM[3][P];
            int kr[3];
            for (int c = 0; c < 3; ++c) {
                int k0;
                double f;
                grid_coord(Pr, d.x[3 * i + c], k0, f);
                bspline_weights<T, P>(T(f), M[c], dM[c]);
                kr[c] = k0 - R.o[c];
            }
            T ax = T(0), ay = T(0), az = T(0);
#pragma unroll
            for (int t2 = 0; t2 < P; ++t2) {
#pragma unroll
                for (int t1 = 0; t1 < P; ++t1) {
                    const T* row = ph + ((kr[2] - t2) * S + (kr[1] - t1)) * S + kr[0];
                    T sx = T(0), s0 = T(0);
#pragma unroll
                    for (int t0 = 0; t0 < P; ++t0) {
                        const T v = row[-t0];
                        sx += dM[0][t0] * v;
                        s0 += M[0][t0] * v;
                    }
                    ax += sx * M[1][t1] * M[2][t2];
                    ay += s0 * dM[1][t1] * M[2][t2];
                    az += s0 * M[1][t1] * dM[2][t2];
                }
            }
            // dQ(k)/dx = q (K / L) M_p'(u - k) ...: dM above is dM/du, and u - k = f + t
            const double sc = q * K * Pr.invL;
            gx = sc * double(ax); gy = sc * double(ay); gz = sc * double(az);
            const T al = T(Pr.alpha), kx = T(Pr.kexp);
            for (int e = d.ex_off[i]; e < d.ex_off[i + 1]; ++e) {
                const int j = d.ex_idx[e];
                double dx = d.x[3 * i] - d.x[3 * j], dy = d.x[3 * i + 1] - d.x[3 * j + 1], dz = d.x[3 * i + 2] - d.x[3 * j + 2];
                dx -= Pr.L * rint(dx * Pr.invL); dy -= Pr.L * rint(dy * Pr.invL); dz -= Pr.L * rint(dz * Pr.invL);
                const T x = T(dx), y = T(dy), z = T(dz);
                const T r2 = x * x + y * y + z * z, r = sqrt_t<T>(r2);
                const T qq = T(COULOMB * q * d.q[j]);
                const T dudr = qq * (erf_t<T>(al * r) / r2 - kx * exp_t<T>(-al * al * r2) / r);
                const T s = dudr / r;
                gx += double(s * x); gy += double(s * y); gz += double(s * z);
            }
        }
        const double m = as_grad ? 1.0 : d.nimt[i];
        out[3 * i] += m * gx; out[3 * i + 1] += m * gy; out[3 * i + 2] += m * gz;
    }
}

// mixed mode gather: FP32 potential grid, weights from the scaled positions,
// exclusion displacements from their exact integer differences
template <int P>
__global__ void __launch_bounds__(PME_THREADS) k_pme_gather_fix(Dev d, double* out, int as_grad)
{
    constexpr int S = PME_BRICK + P - 1;
    __shared__ float ph[S * S * S];
    const int b = blockIdx.x;
    const RepParams& Pr = d.P[d.pme_brick_rep[b]];
    if (Pr.pme_p != P) return;
    const BrickRegion R = brick_region(d, Pr, b, P);
    if (R.end == R.start) return;
    const int K = Pr.pme_K;
    const float* phi = reinterpret_cast<const float*>(d.pme_q) + Pr.pme_goff;
    for (int k = threadIdx.x; k < S * S * S; k += PME_THREADS) {
        const int rz = k / (S * S), ry = (k / S) % S, rx = k % S;
        const int gz = wrap_k(R.o[2] + rz, K), gy = wrap_k(R.o[1] + ry, K), gx = wrap_k(R.o[0] + rx, K);
        ph[k] = phi[((long long)gz * K + gy) * K + gx];
    }
    __syncthreads();
    const float scl = float(K) * float(Pr.invL);
    for (int a = R.start + threadIdx.x; a < R.end; a += PME_THREADS) {
        const int i = d.pme_sorted[a];
        const uint4 ps = d.pos[i];
        const float q = __uint_as_float(ps.w);
        float gx = 0.f, gy = 0.f, gz = 0.f;
        if (q != 0.f) {
            float M[3][P], dM[3][P];
            int kr[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                int k0;
                float f;
                grid_coord_fix(Pr, comp(ps, c), k0, f);
                bspline_weights<float, P>(f, M[c], dM[c]);
                kr[c] = k0 - R.o[c];
            }
            float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
            for (int t2 = 0; t2 < P; ++t2) {
#pragma unroll
                for (int t1 = 0; t1 < P; ++t1) {
                    const float* row = ph + ((kr[2] - t2) * S + (kr[1] - t1)) * S + kr[0];
                    float sx = 0.f, s0 = 0.f;
#pragma unroll
                    for (int t0 = 0; t0 < P; ++t0) {
                        const float v = row[-t0];
                        sx = fmaf(dM[0][t0], v, sx);
                        s0 = fmaf(M[0][t0], v, s0);
                    }
                    ax = fmaf(sx, M[1][t1] * M[2][t2], ax);
                    ay = fmaf(s0, dM[1][t1] * M[2][t2], ay);
                    az = fmaf(s0, M[1][t1] * dM[2][t2], az);
                }
            }
            const float sc = q * scl;
            gx = sc * ax; gy = sc * ay; gz = sc * az;
            const float al = Pr.alphaf, kx = Pr.kexpf;
            for (int e = d.ex_off[i]; e < d.ex_off[i + 1]; ++e) {
                const uint4 pj = d.pos[d.ex_idx[e]];
                float x, y, z;
                sdisp(ps, pj, Pr.sclf, Pr.sclf_lo, x, y, z);
                const float r2 = x * x + y * y + z * z, r = sqrtf(r2);
                const float qq = float(COULOMB) * q * __uint_as_float(pj.w);
                const float s = qq * (erff(al * r) / r2 - kx * expf(-al * al * r2) / r) / r;
                gx = fmaf(s, x, gx); gy = fmaf(s, y, gy); gz = fmaf(s, z, gz);
            }
        }
        const double m = as_grad ? 1.0 : -d.isqmt[i] * d.isqmt[i];
        out[3 * i] += m * double(gx); out[3 * i + 1] += m * double(gy); out[3 * i + 2] += m * double(gz);
    }
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

template <int P>
void spread_p(const Dev& d, int fp64, cudaStream_t s)
{
    if (fp64) k_pme_spread<double, P><<<d.pme_nbricks, PME_THREADS, 0, s>>>(d);
    else k_pme_spread_fix<P><<<d.pme_nbricks, PME_THREADS, 0, s>>>(d);
}

template <int P>
void gather_p(const Dev& d, double* out, int as_grad, int fp64, cudaStream_t s)
{
    if (fp64) k_pme_gather<double, P><<<d.pme_nbricks, PME_THREADS, 0, s>>>(d, out, as_grad);
    else k_pme_gather_fix<P><<<d.pme_nbricks, PME_THREADS, 0, s>>>(d, out, as_grad);
}

}  // namespace

void launch_pme_bin(const Dev& d, int fp64, cudaStream_t s)
{
    if (fp64) k_pme_count<false><<<blocks(d.N, 256), 256, 0, s>>>(d);
    else k_pme_count<true><<<blocks(d.N, 256), 256, 0, s>>>(d);
    k_pme_scan<<<1, 1024, 0, s>>>(d);
    k_pme_place<<<blocks(d.N, 256), 256, 0, s>>>(d);
}

void launch_pme_spread(const Dev& d, int order, int fp64, cudaStream_t s)
{
    // even orders only: the host refuses odd ones (|b(m)| vanishes at m = K/2)
    switch (order) {
    case 4: spread_p<4>(d, fp64, s); break;
    case 6: spread_p<6>(d, fp64, s); break;
    default: spread_p<8>(d, fp64, s); break;
    }
}

void launch_pme_tofloat(const Dev& d, long long total, int fp64, cudaStream_t s)
{
    if (fp64) k_pme_tofloat<<<blocks(total, 256), 256, 0, s>>>(d, total);
    else k_pme_tofloat_fix<<<blocks(total, 256), 256, 0, s>>>(d, total);
}

void launch_pme_convolve_grid(const Dev& d, int energy, long long max_spec, int fp64, cudaStream_t s)
{
    const int bx = std::max(1, std::min(4 * 152, blocks(max_spec, 256 * 4)));
    if (fp64) k_pme_convolve<<<dim3(bx, d.R), 256, 0, s>>>(d, energy);
    else k_pme_convolve_fix<<<dim3(bx, d.R), 256, 0, s>>>(d, energy);
}

void launch_pme_gather(const Dev& d, int order, double* out, int as_grad, int fp64, cudaStream_t s)
{
    switch (order) {
    case 4: gather_p<4>(d, out, as_grad, fp64, s); break;
    case 6: gather_p<6>(d, out, as_grad, fp64, s); break;
    default: gather_p<8>(d, out, as_grad, fp64, s); break;
    }
}

void launch_pme_excl_energy(const Dev& d, cudaStream_t s)
{
    k_pme_excl_energy<<<blocks(d.N, 128), 128, 0, s>>>(d);
}

}  // namespace mdj
