// k_vacf.cu -- velocity record and velocity autocorrelation spectra (the
// spectra of the multiple-time-step integrators in Sec. 4: resonance peaks of
// BAOAB-RESPA1 against JUMP-RESPA1).
//
// Recording stores v after every innermost step in a [sample][3N] buffer
// (one coalesced row per step, FP64 in FP64 mode, FP32 in mixed mode). The
// mass-weighted autocorrelation of one replica,
//   C(k) = (1 / (T - k)) sum_{t=0}^{T-1-k} sum_i m_i v_i(t) . v_i(t + k),
// is computed by the Wiener-Khinchin route: each of the replica's 3n series is
// zero-padded to 2T and transformed (cuFFT, batched), the mass-weighted power
// sum_s m_s |X_s(j)|^2 is summed over series, and its inverse transform is the
// lag sum R(k) = sum_t x(t) x(t + k) exactly (the padding removes wrap-around).
// The spectrum is the Hann-windowed cosine transform of C.
#include <algorithm>

#include "engine.h"

namespace mdj {

namespace {

template <typename T>
__global__ void k_vacf_record(const double* v, T* buf, const long long* step_base, long long origin,
                              long long cap, uint32_t s_local, int n3)
{
    const long long slot = step_base[0] + (long long)s_local - origin;
    if (slot < 0 || slot >= cap) return;
    T* row = buf + slot * (long long)n3;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n3; k += gridDim.x * blockDim.x) row[k] = T(v[k]);
}

// series s0 .. s0 + nb of the record, transposed into [nb][2T] rows, zero-padded
template <typename T>
__global__ void k_vacf_gather(const T* buf, T* pad, long long T_, int n3, int s0, int nb)
{
    __shared__ T tile[32][33];
    const long long t0 = (long long)blockIdx.x * 32;
    const int b0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const long long t = t0 + r;
        const int b = b0 + threadIdx.x;
        tile[r][threadIdx.x] = (t < T_ && b < nb) ? buf[t * n3 + s0 + b] : T(0);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int b = b0 + r;
        const long long t = t0 + threadIdx.x;
        if (b < nb && t < 2 * T_) pad[(long long)b * 2 * T_ + t] = tile[threadIdx.x][r];
    }
}

// P(j) += sum_b m~_b |X_b(j)|^2, j = 0 .. T (m~ = m / 418.4 of the series' atom)
template <typename C>
__global__ void k_vacf_power(const C* X, const double* mass_of_atom, int s0, int nb, long long nj, double* P)
{
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nj) return;
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) {
        const C z = X[(long long)b * nj + j];
        acc += mass_of_atom[(s0 + b) / 3] * (double(z.x) * double(z.x) + double(z.y) * double(z.y));
    }
    P[j] += acc;
}

__global__ void k_vacf_to_complex(const double* P, double2* Z, long long nj)
{
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nj) Z[j] = make_double2(P[j], 0.0);
}

// C(k) = R(k) / (T - k), R(k) = r(k) / (2T) (the inverse transform is unnormalised);
// the power was weighted by m~ = m / 418.4, so C is scaled back to amu A^2 / ps^2
__global__ void k_vacf_finish(const double* r, double* C, long long T_, long long nlags)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nlags) return;
    C[k] = k < T_ ? r[k] * KCAL_AMU / (2.0 * double(T_)) / double(T_ - k) : 0.0;
}

// S(j) = C(0) + 2 sum_{k=1}^{K-1} w_k C(k) cos(pi j k / K), w_k = (1 + cos(pi k / K)) / 2
__global__ void k_vacf_spectrum(const double* C, double* S, long long K)
{
    const long long j = blockIdx.x;
    double acc = 0.0;
    for (long long k = 1 + threadIdx.x; k < K; k += blockDim.x) {
        const double w = 0.5 * (1.0 + cospi(double(k) / double(K)));
        acc += 2.0 * w * C[k] * cospi(double((j * k) % (2 * K)) / double(K));
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) S[j] = C[0] + red[0];
}

inline int blocks(long long n, int b) { return int((n + b - 1) / b); }

}  // namespace

void launch_vacf_record(const Dev& d, void* buf, int fp64, long long origin, long long cap, uint32_t s_local,
                        cudaStream_t s)
{
    const int n3 = 3 * d.N;
    const int nb = std::min(blocks(n3, 256), 4 * 152);
    if (fp64) k_vacf_record<double><<<nb, 256, 0, s>>>(d.v, (double*)buf, d.step_base, origin, cap, s_local, n3);
    else k_vacf_record<float><<<nb, 256, 0, s>>>(d.v, (float*)buf, d.step_base, origin, cap, s_local, n3);
}

void launch_vacf_gather(const void* buf, void* pad, int fp64, long long T, int n3, int s0, int nb, cudaStream_t s)
{
    const dim3 grid(unsigned((2 * T + 31) / 32), unsigned((nb + 31) / 32));
    const dim3 block(32, 8);
    if (fp64) k_vacf_gather<double><<<grid, block, 0, s>>>((const double*)buf, (double*)pad, T, n3, s0, nb);
    else k_vacf_gather<float><<<grid, block, 0, s>>>((const float*)buf, (float*)pad, T, n3, s0, nb);
}

void launch_vacf_power(const void* X, int fp64, const double* mass_of_atom, int s0, int nb, long long nj, double* P,
                       cudaStream_t s)
{
    if (fp64) k_vacf_power<double2><<<blocks(nj, 128), 128, 0, s>>>((const double2*)X, mass_of_atom, s0, nb, nj, P);
    else k_vacf_power<float2><<<blocks(nj, 128), 128, 0, s>>>((const float2*)X, mass_of_atom, s0, nb, nj, P);
}

void launch_vacf_to_complex(const double* P, double2* Z, long long nj, cudaStream_t s)
{
    k_vacf_to_complex<<<blocks(nj, 256), 256, 0, s>>>(P, Z, nj);
}

void launch_vacf_finish(const double* r, double* C, long long T, long long nlags, cudaStream_t s)
{
    k_vacf_finish<<<blocks(nlags, 256), 256, 0, s>>>(r, C, T, nlags);
}

void launch_vacf_spectrum(const double* C, double* S, long long K, cudaStream_t s)
{
    k_vacf_spectrum<<<unsigned(K), 256, 0, s>>>(C, S, K);
}

}  // namespace mdj
