// k_lists.cu -- neighbour and jump lists.
//
// Two levels (the ring technique of Sec. 3.1 needs per-atom "middle" and
// "long" lists with their counts N_M(i), N_L(i), and Sec. 3.2 an LJ list):
//   outer: every partner within r_E + skin_outer, found through a cell grid
//          of floor(L / (r_E + skin_outer)) cells per edge and stored in
//          (cell, j) order: neighbour cells in increasing linear index, atoms
//          of a cell in increasing index. Rebuilt when an atom moved more
//          than (skin_outer - skin)/2 since the last outer build.
//   inner: short (r_c + skin), full (r_E + skin), ring M, ring L and LJ lists
//          filtered from the outer list in its order, at the build positions
//          x_b, when an atom moved more than skin/2 since the last build.
// Every rebuild kernel reads the per-replica flags and returns at once when
// its replica does not rebuild, so the chain can be launched every step.
#include "engine.h"

namespace mdj {

namespace {

constexpr int WARPS = 4;              // warps per block in warp-per-item kernels
constexpr int SORT_CAP = 1024;        // atoms per cell the in-block sort handles

__device__ __forceinline__ double3 ld3(const double* p, int i)
{
    return make_double3(p[3 * i], p[3 * i + 1], p[3 * i + 2]);
}

__device__ __forceinline__ double mimg(double t, const RepParams& P)
{
    return t - P.L * rint(t * P.invL);
}

__device__ __forceinline__ double dist2_fp64(const double* X, int i, int j, const RepParams& P)
{
    const double3 a = ld3(X, i), b = ld3(X, j);
    const double dx = mimg(a.x - b.x, P), dy = mimg(a.y - b.y, P), dz = mimg(a.z - b.z, P);
    return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ float sdist2(const Dev& d, const RepParams& P, const uint4& pi, int j)
{
    float dx, dy, dz;
    sdisp(pi, d.pos[j], P.sclf, P.sclf_lo, dx, dy, dz);
    return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ bool is_excluded(const Dev& d, int i, int j)
{
    const int e0 = d.ex_off[i], e1 = d.ex_off[i + 1];
    for (int e = e0; e < e1; ++e)
        if (d.ex_idx[e] == j) return true;
    return false;
}

// ---- displacement check -------------------------------------------------------
__global__ void k_check(Dev d, int force_inner, int force_outer)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const int r = d.rep[i];
    const RepParams& P = d.P[r];
    if (force_inner || force_outer) {
        if (i == P.atom_off) {
            d.flags[2 * r] = 1;
            if (force_outer) d.flags[2 * r + 1] = 1;
        }
        return;
    }
    const double lo = 0.5 * (P.skin_o - P.skin), li = 0.5 * P.skin;
    const double3 x = ld3(d.x, i), xo = ld3(d.xo, i), xb = ld3(d.xb, i);
    double t0 = mimg(x.x - xo.x, P), t1 = mimg(x.y - xo.y, P), t2 = mimg(x.z - xo.z, P);
    if (t0 * t0 + t1 * t1 + t2 * t2 > lo * lo) {
        d.flags[2 * r + 1] = 1;
        d.flags[2 * r] = 1;
    }
    t0 = mimg(x.x - xb.x, P); t1 = mimg(x.y - xb.y, P); t2 = mimg(x.z - xb.z, P);
    if (t0 * t0 + t1 * t1 + t2 * t2 > li * li) d.flags[2 * r] = 1;
}

// ---- refresh the scaled coordinates; assign outer cells ----------------------------
__global__ void k_rehome(Dev d, int keep_refs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const int r = d.rep[i];
    if (!d.flags[2 * r]) return;
    const int fo = d.flags[2 * r + 1];
    const RepParams& P = d.P[r];
    const double3 x = ld3(d.x, i);
    if (!keep_refs) {
        d.xb[3 * i] = x.x; d.xb[3 * i + 1] = x.y; d.xb[3 * i + 2] = x.z;
        if (fo) { d.xo[3 * i] = x.x; d.xo[3 * i + 1] = x.y; d.xo[3 * i + 2] = x.z; }
    }
    d.pos[i] = make_uint4(to_scaled(x.x, P), to_scaled(x.y, P), to_scaled(x.z, P),
                          __float_as_uint((float)d.q[i]));
    if (fo) {
        const double3 xo = ld3(d.xo, i);
        const double oo[3] = {xo.x, xo.y, xo.z};
        int c3[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int c = (int)floor(oo[a] / P.cs);
            c3[a] = c < 0 ? 0 : (c >= P.nc ? P.nc - 1 : c);
        }
        const int cell = P.cell_off + (c3[2] * P.nc + c3[1]) * P.nc + c3[0];
        d.atom_cell[i] = cell;
        atomicAdd(&d.cell_cnt[cell], 1);
    }
}

// ---- per-replica exclusive scan of the cell counts ------------------------------
__global__ void k_cell_scan(Dev d)
{
    const int r = blockIdx.x;
    if (!d.flags[2 * r + 1]) return;
    const RepParams& P = d.P[r];
    const int ncell = P.nc * P.nc * P.nc;
    __shared__ int warp_sum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = P.atom_off;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < ncell; base += blockDim.x) {
        const int c = base + threadIdx.x;
        const int v = c < ncell ? d.cell_cnt[P.cell_off + c] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_sum[w] = incl;
        __syncthreads();
        if (w == 0) {
            const int nw = blockDim.x >> 5;
            int s = lane < nw ? warp_sum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += t;
            }
            if (lane < nw) warp_sum[lane] = s;
        }
        __syncthreads();
        const int before = (w > 0 ? warp_sum[w - 1] : 0) + incl - v;
        if (c < ncell) {
            d.cell_start[P.cell_off + c] = carry + before;
            d.cell_cnt[P.cell_off + c] = 0;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) d.cell_start[P.cell_off + ncell] = carry;
}

__global__ void k_cell_fill(Dev d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.N) return;
    const int r = d.rep[i];
    if (!d.flags[2 * r + 1]) return;
    const int c = d.atom_cell[i];
    const int pos = d.cell_start[c] + atomicAdd(&d.cell_cnt[c], 1);
    d.cell_atoms[pos] = i;
}

// one warp per cell: order the atoms of the cell by index (rank sort)
__global__ void k_cell_sort(Dev d)
{
    __shared__ int buf[WARPS][SORT_CAP];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * WARPS + w;
    if (c >= d.total_cells) return;
    const int r = d.cell_rep[c];
    if (r < 0 || !d.flags[2 * r + 1]) return;
    const int s = d.cell_start[c], e = d.cell_start[c + 1], n = e - s;
    if (n > SORT_CAP) {
        if (lane == 0) { atomicOr(&d.err[r], F_OVERFLOW); atomicOr(&d.ovf[r], 1u << 6); d.cell_cnt[c] = 0; }
        return;
    }
    for (int k = lane; k < n; k += 32) buf[w][k] = d.cell_atoms[s + k];
    __syncwarp();
    for (int k = lane; k < n; k += 32) {
        const int v = buf[w][k];
        int rank = 0;
        for (int m = 0; m < n; ++m) rank += buf[w][m] < v;
        d.cell_atoms[s + rank] = v;
    }
    if (lane == 0) d.cell_cnt[c] = 0;
}

// one block per cell: the candidates of the (sorted) neighbour cells are staged
// in shared memory once per cell, in (cell, j) order, and every warp scans them
// for one atom of the cell at a time. Neighbour cells whose box lies farther
// than r_E + skin_outer from the atom are skipped.
constexpr int OCAP = 4096;                  // staged candidates per chunk
constexpr int OUTER_THREADS = 256;
constexpr int OUTER_SMEM = OCAP * (16 + 4) + 1024 * 4;

__global__ void __launch_bounds__(OUTER_THREADS) k_outer_cells(Dev d, int exact)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint4* cpos = (uint4*)smem;
    int* cidx = (int*)(cpos + OCAP);
    int* acnt = cidx + OCAP;                // running list length of each atom of the cell
    __shared__ int nb[27], nboff[27], nbstart[27], nbsize[27], nbpre[28];
    __shared__ int nnb;
    const int c = blockIdx.x;
    if (c >= d.total_cells) return;
    const int r = d.cell_rep[c];
    if (r < 0 || !d.flags[2 * r + 1]) return;
    const RepParams& P = d.P[r];
    const int nc = P.nc;
    const int lin = c - P.cell_off;
    const int cc[3] = {lin % nc, (lin / nc) % nc, lin / (nc * nc)};
    const int nax = nc >= 3 ? 3 : nc;
    const int ncell = nax * nax * nax;
    const int s_i = d.cell_start[c], e_i = d.cell_start[c + 1];
    const int natoms = e_i - s_i;
    if (natoms > 1024) {
        if (threadIdx.x == 0) { atomicOr(&d.err[r], F_OVERFLOW); atomicOr(&d.ovf[r], 1u << 6); }
        return;
    }
    if (natoms == 0) return;
    // neighbour cells in increasing linear index, with their offset code
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int mine = 0, off = 0;
        if (lane < ncell) {
            const int q[3] = {lane % nax, (lane / nax) % nax, lane / (nax * nax)};
            int cv[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) cv[a] = nc >= 3 ? (cc[a] + q[a] - 1 + nc) % nc : q[a];
            mine = (cv[2] * nc + cv[1]) * nc + cv[0];
            off = nc >= 3 ? (q[0] | (q[1] << 2) | (q[2] << 4)) : 0x3f;   // 0x3f: no pruning
            nb[lane] = mine;
        }
        __syncwarp();
        int rank = 0;
        for (int m = 0; m < ncell; ++m) rank += nb[m] < mine;
        __syncwarp();
        if (lane < ncell) {
            nb[rank] = mine;
            nboff[rank] = off;
        }
        __syncwarp();
        if (lane < ncell) {
            const int gc = P.cell_off + nb[lane];
            nbstart[lane] = d.cell_start[gc];
            nbsize[lane] = d.cell_start[gc + 1] - d.cell_start[gc];
        }
        __syncwarp();
        if (lane == 0) {
            int acc = 0;
            for (int m = 0; m < ncell; ++m) { nbpre[m] = acc; acc += nbsize[m]; }
            nbpre[ncell] = acc;
            nnb = ncell;
        }
    }
    for (int a = threadIdx.x; a < natoms; a += blockDim.x) acnt[a] = 0;
    __syncthreads();
    const int total = nbpre[nnb];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const double ro = P.R + P.skin_o;
    const float r2of = float(ro * ro * (1.0 + 4e-6));
    const float rof = float(ro * (1.0 + 2e-6));
    const float csf = float(P.cs);
    for (int base = 0; base < total; base += OCAP) {
        const int len = min(OCAP, total - base);
        // stage candidates [base, base + len) in (cell, j) order
        for (int k = threadIdx.x; k < len; k += blockDim.x) {
            const int g = base + k;
            int m = 0;
            while (nbpre[m + 1] <= g) ++m;
            const int j = d.cell_atoms[nbstart[m] + (g - nbpre[m])];
            cidx[k] = j;
            cpos[k] = d.pos[j];
        }
        __syncthreads();
        for (int a = w; a < natoms; a += nw) {
            const int i = d.cell_atoms[s_i + a];
            const uint4 pi = d.pos[i];
            // position of i inside its cell, per axis (for the pruning of far cells)
            float f3[3];
            {
                const double3 xo = ld3(d.xo, i);
                const double xx[3] = {xo.x, xo.y, xo.z};
#pragma unroll
                for (int q = 0; q < 3; ++q) f3[q] = float(xx[q] - cc[q] * P.cs);
            }
            uint32_t* row = d.olist + (size_t)i * d.ocap;
            int cnt = acnt[a];
            for (int m = 0; m < nnb; ++m) {
                const int lo = max(nbpre[m], base) - base, hi = min(nbpre[m + 1], base + len) - base;
                if (lo >= hi) continue;
                const int oc = nboff[m];
                if (oc != 0x3f) {
                    float dd2 = 0.f;
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const int o = (oc >> (2 * q)) & 3;      // 0: cell below, 1: same, 2: above
                        const float t = o == 0 ? f3[q] : (o == 2 ? csf - f3[q] : 0.f);
                        dd2 += t > 0.f ? t * t : 0.f;
                    }
                    if (dd2 > rof * rof) continue;
                }
                for (int k0 = lo; k0 < hi; k0 += 32) {
                    const int k = k0 + lane;
                    bool ok = false;
                    int j = -1;
                    if (k < hi) {
                        j = cidx[k];
                        if (j != i) {
                            if (exact) {
                                ok = dist2_fp64(d.xo, i, j, P) < ro * ro;
                            } else {
                                float dx, dy, dz;
                                sdisp(pi, cpos[k], P.sclf, P.sclf_lo, dx, dy, dz);
                                ok = dx * dx + dy * dy + dz * dz < r2of;
                            }
                            if (ok) ok = !is_excluded(d, i, j);
                        }
                    }
                    const unsigned b = __ballot_sync(0xffffffffu, ok);
                    const int pos = cnt + __popc(b & ((1u << lane) - 1u));
                    if (ok && pos < d.ocap) row[pos] = (uint32_t)j;
                    cnt += __popc(b);
                }
            }
            if (lane == 0) acnt[a] = cnt;
            __syncwarp();
        }
        __syncthreads();
    }
    for (int a = threadIdx.x; a < natoms; a += blockDim.x) {
        const int i = d.cell_atoms[s_i + a];
        const int cnt = acnt[a];
        d.ocnt[i] = cnt;
        if (cnt > d.ocap) {
            atomicOr(&d.err[r], F_OVERFLOW);
            atomicOr(&d.ovf[r], 1u << 5);
        }
    }
}

// one warp per atom: filter the outer list into the inner lists
__global__ void k_inner_lists(Dev d, int kinds, int exact, int late)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * WARPS + w;
    if (i >= d.N) return;
    const int r = d.rep[i];
    if (!late && !d.flags[2 * r]) return;
    const RepParams& P = d.P[r];
    const uint4 pi = d.pos[i];
    const float qi = __uint_as_float(pi.w);
    const int ti = d.type[i];
    const double sk = P.skin;
    const double lo_m = fmax(0.0, P.sw - sk), hi_m = P.rM + sk;
    const double lo_l = P.rM - sk, hi_l = P.R + sk;
    const double lo_j = fmax(0.0, P.sw - sk), hi_j = P.R + sk;
    // ring and LJ shell limits (squared), FP64 and FP32 copies
    const double b2[6] = {lo_m * lo_m, hi_m * hi_m, lo_l * lo_l, hi_l * hi_l, lo_j * lo_j, hi_j * hi_j};
    float b2f[6];
#pragma unroll
    for (int t = 0; t < 6; ++t) b2f[t] = float(b2[t]);
    const float r2s = float((P.rc + sk) * (P.rc + sk)), r2f = float((P.R + sk) * (P.R + sk));
    const bool ringm_on = P.rings_on && !P.one_ring;
    const bool ringl_on = P.rings_on && P.rM < P.R;
    const bool lj_on = P.lj_on;
    int cnt[NKIND] = {0, 0, 0, 0, 0};
    const int n_o = d.ocnt[i] < d.ocap ? d.ocnt[i] : d.ocap;
    const uint32_t* orow = d.olist + (size_t)i * d.ocap;
    for (int base = 0; base < n_o; base += 32) {
        const int k = base + lane;
        bool m[NKIND] = {false, false, false, false, false};
        uint32_t entry = 0;
        if (k < n_o) {
            const int j = (int)orow[k];
            entry = (uint32_t)j;
            const uint4 pj = d.pos[j];
            const bool qq = qi != 0.f && __uint_as_float(pj.w) != 0.f;
            const bool ljp = lj_on && P.lj[ti * MAX_TYPES + d.type[j]].on;
            if (exact) {
                const double r2 = dist2_fp64(d.xb, i, j, P);
                m[L_SHORT] = r2 < double(r2s);
                m[L_FULL] = r2 < double(r2f);
                m[L_RM] = ringm_on && qq && r2 >= b2[0] && r2 < b2[1];
                m[L_RL] = ringl_on && qq && r2 >= b2[2] && r2 < b2[3];
                m[L_LJ] = ljp && r2 >= b2[4] && r2 < b2[5];
            } else {
                float dx, dy, dz;
                sdisp(pi, pj, P.sclf, P.sclf_lo, dx, dy, dz);
                const float r2 = dx * dx + dy * dy + dz * dz;
                m[L_SHORT] = r2 < r2s;
                m[L_FULL] = r2 < r2f;
                // ring and LJ membership decides which partner a jump picks:
                // within 2e-5 (relative, in r^2) of a shell limit it is decided in FP64
                bool near = false;
#pragma unroll
                for (int t = 0; t < 6; ++t) near |= fabsf(r2 - b2f[t]) < 2e-5f * b2f[t] + 1e-6f;
                if (near) {
                    const double r2d = dist2_fp64(d.xb, i, j, P);
                    m[L_RM] = ringm_on && qq && r2d >= b2[0] && r2d < b2[1];
                    m[L_RL] = ringl_on && qq && r2d >= b2[2] && r2d < b2[3];
                    m[L_LJ] = ljp && r2d >= b2[4] && r2d < b2[5];
                } else {
                    m[L_RM] = ringm_on && qq && r2 >= b2f[0] && r2 < b2f[1];
                    m[L_RL] = ringl_on && qq && r2 >= b2f[2] && r2 < b2f[3];
                    m[L_LJ] = ljp && r2 >= b2f[4] && r2 < b2f[5];
                }
            }
        }
#pragma unroll
        for (int kind = 0; kind < NKIND; ++kind) {
            if (!(kinds & (1 << kind))) continue;
            const unsigned b = __ballot_sync(0xffffffffu, m[kind]);
            const int pos = cnt[kind] + __popc(b & ((1u << lane) - 1u));
            if (m[kind] && pos < d.lcap[kind]) d.list[kind][(size_t)i * d.lcap[kind] + pos] = entry;
            cnt[kind] += __popc(b);
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int kind = 0; kind < NKIND; ++kind) {
            if (!(kinds & (1 << kind))) continue;
            d.lcnt[kind][i] = cnt[kind];
            if (cnt[kind] > d.lcap[kind]) {
                atomicOr(&d.err[r], F_OVERFLOW);
                atomicOr(&d.ovf[r], 1u << kind);
            }
        }
    }
}

__global__ void k_flags_clear(Dev d)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.R) return;
    if (d.flags[2 * r]) d.cnt[(size_t)r * NCOUNT + C_REBUILD] += 1;
    if (d.flags[2 * r + 1]) d.cnt[(size_t)r * NCOUNT + C_OUTER] += 1;
    d.flags[2 * r] = 0;
    d.flags[2 * r + 1] = 0;
}

inline int blocks(int n, int b) { return (n + b - 1) / b; }

}  // namespace

void launch_check(const Dev& d, int force_inner, int force_outer, cudaStream_t s)
{
    k_check<<<blocks(d.N, 256), 256, 0, s>>>(d, force_inner, force_outer);
}

void launch_rebuild(const Dev& d, int kinds, int exact, int keep_refs, int exact_outer,
                    int /*max_cells_per_rep*/, cudaStream_t s)
{
    k_rehome<<<blocks(d.N, 256), 256, 0, s>>>(d, keep_refs);
    k_cell_scan<<<d.R, 1024, 0, s>>>(d);
    k_cell_fill<<<blocks(d.N, 256), 256, 0, s>>>(d);
    k_cell_sort<<<blocks(d.total_cells, WARPS), 32 * WARPS, 0, s>>>(d);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_outer_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, OUTER_SMEM);
        attr = true;
    }
    k_outer_cells<<<d.total_cells, OUTER_THREADS, OUTER_SMEM, s>>>(d, exact_outer);
    if (kinds) k_inner_lists<<<blocks(d.N, WARPS), 32 * WARPS, 0, s>>>(d, kinds, exact, 0);
    k_flags_clear<<<blocks(d.R, 128), 128, 0, s>>>(d);
}

void launch_late_lists(const Dev& d, int kinds, cudaStream_t s)
{
    if (kinds) k_inner_lists<<<blocks(d.N, WARPS), 32 * WARPS, 0, s>>>(d, kinds, 1, 1);
}

}  // namespace mdj
