// noalloc.cu -- md_nb_gradient_noalloc: the nonbonded gradient of one system
// computed from caller-owned device arrays without allocating anything.
//
// It is a variant of the pair-gradient kernel of k_force.cu. Instead of the
// context's neighbour lists (device memory the context allocates), it uses a
// cell grid whose scratch lives in one file-scope __device__ array of fixed,
// modest size that every GPU loading this library keeps until the process
// exits. Pair arithmetic is FP64, as in the FP64 mode of the context path.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/md.h"
#include "common.cuh"

namespace mdj {
void set_global_error(const std::string& msg);
}

namespace {

using namespace mdj;

constexpr int NA_MAX_ATOMS = MD_NOALLOC_MAX_ATOMS;
constexpr int NA_MAX_CELLS = MD_NOALLOC_MAX_CELLS;
// layout (ints): count[C] | cursor[C] | start[C + 1] | atoms[N] | cell of atom[N] | fill[N]
constexpr size_t NA_INTS = 3 * (size_t)NA_MAX_CELLS + 1 + 3 * (size_t)NA_MAX_ATOMS;

static __device__ __align__(256) int g_na_scratch[NA_INTS];

struct NaParams {
    int n, nc, ncell, ntypes, weight, has_mol;
    double L, invL, cs, R, rc, sw, h;
    double alpha, eR, fR, kexp;
    double c12[MAX_TYPES * MAX_TYPES], c6[MAX_TYPES * MAX_TYPES];
    double uR[MAX_TYPES * MAX_TYPES], duR[MAX_TYPES * MAX_TYPES];
    int on[MAX_TYPES * MAX_TYPES];
};

struct Scratch {
    int *count, *cursor, *start, *atoms, *cell, *fill;
};

__device__ __forceinline__ Scratch view(int* base)
{
    Scratch s;
    s.count = base;
    s.cursor = base + NA_MAX_CELLS;
    s.start = base + 2 * NA_MAX_CELLS;
    s.atoms = base + 3 * NA_MAX_CELLS + 1;
    s.cell = s.atoms + NA_MAX_ATOMS;
    s.fill = s.cell + NA_MAX_ATOMS;
    return s;
}

__global__ void k_na_clear(int* base, int ncell)
{
    const Scratch s = view(base);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
        s.count[c] = 0;
        s.cursor[c] = 0;
    }
}

__global__ void k_na_count(const double* x, int* base, NaParams p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const Scratch s = view(base);
    int c3[3];
    for (int a = 0; a < 3; ++a) {
        double t = x[3 * i + a];
        t -= p.L * floor(t * p.invL);
        int c = (int)floor(t / p.cs);
        c3[a] = c < 0 ? 0 : (c >= p.nc ? p.nc - 1 : c);
    }
    const int c = (c3[2] * p.nc + c3[1]) * p.nc + c3[0];
    s.cell[i] = c;
    atomicAdd(&s.count[c], 1);
}

// one block: exclusive scan of the cell counts
__global__ void k_na_scan(int* base, int ncell)
{
    const Scratch s = view(base);
    __shared__ int warp_sum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int b = 0; b < ncell; b += blockDim.x) {
        const int c = b + threadIdx.x;
        const int v = c < ncell ? s.count[c] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_sum[w] = incl;
        __syncthreads();
        if (w == 0) {
            const int nw = blockDim.x >> 5;
            int t = lane < nw ? warp_sum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += u;
            }
            if (lane < nw) warp_sum[lane] = t;
        }
        __syncthreads();
        const int before = (w > 0 ? warp_sum[w - 1] : 0) + incl - v;
        if (c < ncell) s.start[c] = carry + before;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) s.start[ncell] = carry;
}

// atoms into their cells' ranges of `fill`, in the order the atomics give
__global__ void k_na_fill(int* base, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Scratch s = view(base);
    const int c = s.cell[i];
    s.fill[s.start[c] + atomicAdd(&s.cursor[c], 1)] = i;
}

// one warp per cell: the cell's atoms into `atoms` in increasing index (rank
// sort), so that every call sums the pairs of an atom in the same order
__global__ void k_na_sort(int* base, int ncell)
{
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (c >= ncell) return;
    const Scratch s = view(base);
    const int b = s.start[c], n = s.start[c + 1] - b;
    for (int k = lane; k < n; k += 32) {
        const int v = s.fill[b + k];
        int rank = 0;
        for (int m = 0; m < n; ++m) rank += s.fill[b + m] < v;
        s.atoms[b + rank] = v;
    }
}

// pair gradient of atom i over the 27 (or fewer, unique) neighbour cells
__global__ void k_na_force(const double* x, const double* q, const int* type, const int* mol, const int* base,
                           NaParams p, double* grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const Scratch s = view(const_cast<int*>(base));
    const int ci = s.cell[i];
    const int cc[3] = {ci % p.nc, (ci / p.nc) % p.nc, ci / (p.nc * p.nc)};
    const int nax = p.nc >= 3 ? 3 : p.nc;
    const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    const double qi = q[i];
    const int ti = type[i];
    const int mi = p.has_mol ? mol[i] : -1;
    const double cut = p.weight == W_SHORT ? fmin(p.rc, p.R) : p.R;
    double gx = 0, gy = 0, gz = 0;
    for (int qz = 0; qz < nax; ++qz)
        for (int qy = 0; qy < nax; ++qy)
            for (int qx = 0; qx < nax; ++qx) {
                const int q3[3] = {qx, qy, qz};
                int cv[3];
                for (int a = 0; a < 3; ++a) cv[a] = p.nc >= 3 ? (cc[a] + q3[a] - 1 + p.nc) % p.nc : q3[a];
                const int c = (cv[2] * p.nc + cv[1]) * p.nc + cv[0];
                for (int k = s.start[c]; k < s.start[c + 1]; ++k) {
                    const int j = s.atoms[k];
                    if (j == i || (p.has_mol && mol[j] == mi)) continue;
                    double dx = xi - x[3 * j], dy = yi - x[3 * j + 1], dz = zi - x[3 * j + 2];
                    dx -= p.L * rint(dx * p.invL);
                    dy -= p.L * rint(dy * p.invL);
                    dz -= p.L * rint(dz * p.invL);
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 >= cut * cut) continue;
                    if (p.weight == W_LONG && r2 <= p.sw * p.sw) continue;
                    const double r = sqrt(r2), rinv = 1.0 / r;
                    double u = 0, du = 0;
                    const double qq = qi * q[j];
                    if (qq != 0.0) {
                        const double e = erfc(p.alpha * r);
                        const double g = p.kexp * exp(-p.alpha * p.alpha * r2);
                        u = COULOMB * qq * (e * rinv - p.eR + p.fR * (r - p.R));
                        du = COULOMB * qq * (-(e * rinv + g) * rinv + p.fR);
                    }
                    const int tp = ti * MAX_TYPES + type[j];
                    if (p.on[tp]) {
                        const double r6i = rinv * rinv * rinv * rinv * rinv * rinv;
                        u += r6i * (p.c12[tp] * r6i - p.c6[tp]) - p.uR[tp] - (r - p.R) * p.duR[tp];
                        du += r6i * rinv * (6.0 * p.c6[tp] - 12.0 * p.c12[tp] * r6i) - p.duR[tp];
                    }
                    double f = du;
                    if (p.weight != W_FULL) {
                        double ch, dch;
                        chi_and_slope<double>(r, p.sw, p.h, ch, dch);
                        f = p.weight == W_SHORT ? dch * u + ch * du : -dch * u + (1.0 - ch) * du;
                    }
                    f *= rinv;
                    gx += f * dx; gy += f * dy; gz += f * dz;
                }
            }
    grad[3 * i] = gx; grad[3 * i + 1] = gy; grad[3 * i + 2] = gz;
}

// device address of the scratch array, looked up once per device
std::mutex g_na_mutex;
int* g_na_ptr[256] = {};

int scratch_for(int dev, int** out)
{
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (dev < 0 || dev >= 256) return MD_EINVAL;
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) {
            set_global_error(std::string("md_nb_gradient_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return MD_ECUDA;
        }
        g_na_ptr[dev] = (int*)p;
    }
    *out = g_na_ptr[dev];
    return MD_OK;
}

int fail(int code, const char* msg)
{
    set_global_error(std::string("md_nb_gradient_noalloc: ") + msg);
    return code;
}

}  // namespace

extern "C" int md_nb_gradient_noalloc(const double* d_x, const double* d_charge, const int* d_type,
                                      const int* d_mol, int n_atoms, double box, int n_types,
                                      const double* lj_eps, const double* lj_sigma, double r_cut,
                                      double r_split, double h_switch, double dsf_alpha, int weight,
                                      double* d_grad, void* cuda_stream)
{
    if (!d_x || !d_charge || !d_type || !d_grad || !lj_eps || !lj_sigma)
        return fail(MD_EINVAL, "null array");
    if (n_atoms < 1 || n_atoms > NA_MAX_ATOMS)
        return fail(MD_EINVAL, "n_atoms must be in [1, MD_NOALLOC_MAX_ATOMS]");
    if (n_types < 1 || n_types > MAX_TYPES) return fail(MD_EINVAL, "n_types must be in [1, 8]");
    if (weight < 0 || weight > 2) return fail(MD_EINVAL, "weight must be 0 (full), 1 (short) or 2 (long)");
    if (!(r_cut > 0) || !(h_switch > 0) || !(r_split > h_switch) || !(dsf_alpha >= 0) || !(box >= 2.0 * r_cut))
        return fail(MD_EINVAL, "need r_cut > 0, r_split > h_switch > 0, dsf_alpha >= 0, box >= 2 r_cut");
    NaParams p;
    std::memset(&p, 0, sizeof p);
    p.n = n_atoms;
    p.nc = std::max(1, int(std::floor(box / r_cut)));
    if ((long long)p.nc * p.nc * p.nc > NA_MAX_CELLS)
        return fail(MD_EINVAL, "box / r_cut gives more cells than MD_NOALLOC_MAX_CELLS");
    p.ncell = p.nc * p.nc * p.nc;
    p.ntypes = n_types;
    p.weight = weight;
    p.has_mol = d_mol != nullptr;
    p.L = box; p.invL = 1.0 / box; p.cs = box / p.nc;
    p.R = r_cut; p.rc = r_split; p.h = h_switch; p.sw = r_split - h_switch;
    p.alpha = dsf_alpha;
    p.eR = std::erfc(dsf_alpha * r_cut) / r_cut;
    p.kexp = 2.0 * dsf_alpha / std::sqrt(PI);
    p.fR = std::erfc(dsf_alpha * r_cut) / (r_cut * r_cut) + p.kexp * std::exp(-dsf_alpha * dsf_alpha * r_cut * r_cut) / r_cut;
    for (int a = 0; a < n_types; ++a)
        for (int b = 0; b < n_types; ++b) {
            const double e = lj_eps[a * n_types + b], sg = lj_sigma[a * n_types + b];
            const int t = a * MAX_TYPES + b;
            p.c12[t] = 4.0 * e * std::pow(sg, 12);
            p.c6[t] = 4.0 * e * std::pow(sg, 6);
            p.uR[t] = p.c12[t] / std::pow(r_cut, 12) - p.c6[t] / std::pow(r_cut, 6);
            p.duR[t] = -12.0 * p.c12[t] / std::pow(r_cut, 13) + 6.0 * p.c6[t] / std::pow(r_cut, 7);
            p.on[t] = e > 0.0;
        }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(MD_ECUDA, cudaGetErrorString(e));
    int* scratch = nullptr;
    int rc = scratch_for(dev, &scratch);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int nb = (n_atoms + 127) / 128;
    k_na_clear<<<(p.ncell + 255) / 256, 256, 0, s>>>(scratch, p.ncell);
    k_na_count<<<nb, 128, 0, s>>>(d_x, scratch, p);
    k_na_scan<<<1, 1024, 0, s>>>(scratch, p.ncell);
    k_na_fill<<<nb, 128, 0, s>>>(scratch, n_atoms);
    k_na_sort<<<(p.ncell + 3) / 4, 128, 0, s>>>(scratch, p.ncell);
    k_na_force<<<nb, 128, 0, s>>>(d_x, d_charge, d_type, d_mol, scratch, p, d_grad);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MD_ECUDA, cudaGetErrorString(e));
    return MD_OK;
}
