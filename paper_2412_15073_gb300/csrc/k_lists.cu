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
#include <algorithm>

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
    if (d.R == 1 && !d.flags[0]) return;        // the only replica does not rebuild
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
    if (d.R == 1 && !d.flags[1]) return;
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
    if (d.R == 1 && !d.flags[1]) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * WARPS + w;
    if (c >= d.total_cells) return;
    const int r = d.cell_rep[c];
    if (r < 0 || !d.flags[2 * r + 1]) return;
    const int s = d.cell_start[c], e = d.cell_start[c + 1], n = e - s;
    if (n > SORT_CAP) {
        if (lane == 0) { atomicOr(&d.err[r], F_OVERFLOW); atomicOr(&d.ovf[r], OVF_CELL); d.cell_cnt[c] = 0; }
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

// Outer candidate lists. A cell's atoms are split over OUTER_GROUPS warps
// (home atoms); each warp streams the candidates of the 125 neighbour cells
// (cells in increasing linear index, atoms of a cell in increasing index), 32
// per batch, one per lane, and for each home atom in turn ballots which
// candidates lie within r_E + skin_outer: the matches are appended to that
// atom's row with coalesced stores, so every row comes out in (cell, j)
// order. The next batch's candidates load while the current one is tested.
// Cells have an edge of at least (r_E + skin_outer)/2, so the neighbourhood
// is +-2 cells per axis.
constexpr int OUTER_WARPS = 4;
constexpr int OUTER_GROUPS = 2;                           // warps per cell, each with a share of its atoms

__global__ void __launch_bounds__(32 * OUTER_WARPS) k_outer_cells(Dev d, int exact)
{
    __shared__ int nbs[OUTER_WARPS][128];
    __shared__ int cpre[OUTER_WARPS][129];     // candidates before each sorted neighbour cell
    __shared__ int cbeg[OUTER_WARPS][128];     // first atom of each sorted neighbour cell
    __shared__ uint4 home[OUTER_WARPS][32];    // (x, y, z, i) of the home atoms of a pass
    __shared__ int4 hex[OUTER_WARPS][32];      // their first four excluded partners (-1: none)
    __shared__ uint32_t* hrow[OUTER_WARPS][32];  // their rows of the outer list
    __shared__ int hmore[OUTER_WARPS][32];     // 1: more than four excluded partners, else -1
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (d.R == 1 && !d.flags[1]) return;        // the only replica does not rebuild its outer list
    const int ntask = d.total_cells * OUTER_GROUPS;
    // the warps stride over the tasks (cell, share of its atoms): a launch in
    // which no replica rebuilds costs one flag read per task
    for (int task = blockIdx.x * OUTER_WARPS + w; task < ntask; task += gridDim.x * OUTER_WARPS) {
    const int c = task / OUTER_GROUPS, g = task % OUTER_GROUPS;
    const int r = d.cell_rep[c];
    if (r < 0 || !d.flags[2 * r + 1]) continue;
    const int s_i = d.cell_start[c], e_i = d.cell_start[c + 1];
    const int natoms = e_i - s_i;
    if (g == 0 && natoms > 1024 && lane == 0) { atomicOr(&d.err[r], F_OVERFLOW); atomicOr(&d.ovf[r], OVF_CELL); }
    const int nlim = min(natoms, 1024);
    const int share = (nlim + OUTER_GROUPS - 1) / OUTER_GROUPS;
    const int h_lo = g * share, h_hi = min(nlim, h_lo + share);
    if (h_lo >= h_hi) continue;
    const RepParams& P = d.P[r];
    const int nc = P.nc;
    const int lin = c - P.cell_off;
    const int cc[3] = {lin % nc, (lin / nc) % nc, lin / (nc * nc)};
    const int nax = nc >= 5 ? 5 : nc;
    const int ncell = nax * nax * nax;
    // neighbour cells in increasing linear index
    for (int t = lane; t < ncell; t += 32) {
        const int q[3] = {t % nax, (t / nax) % nax, t / (nax * nax)};
        int cv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) cv[a] = nc >= 5 ? (cc[a] + q[a] - 2 + nc) % nc : q[a];
        nbs[w][t] = (cv[2] * nc + cv[1]) * nc + cv[0];
    }
    __syncwarp();
    int mine[4], rk[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int t = lane + 32 * u;
        mine[u] = t < ncell ? nbs[w][t] : 0;
        rk[u] = 0;
        if (t < ncell)
            for (int m = 0; m < ncell; ++m) rk[u] += nbs[w][m] < mine[u];
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (lane + 32 * u < ncell) nbs[w][rk[u]] = mine[u];
    __syncwarp();
    // candidate ranges: lane l holds sorted cells 4l .. 4l+3; warp scan of their counts
    int cntc[4], sum = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int m = 4 * lane + u;
        cntc[u] = 0;
        if (m < ncell) {
            const int gc = P.cell_off + nbs[w][m];
            const int b0 = d.cell_start[gc];
            cbeg[w][m] = b0;
            cntc[u] = d.cell_start[gc + 1] - b0;
        }
        sum += cntc[u];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    {
        int run = incl - sum;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int m = 4 * lane + u;
            if (m <= ncell) cpre[w][m] = run;
            run += cntc[u];
        }
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (lane == 31) cpre[w][ncell] = total;
    __syncwarp();
    // FP32 test in units of the scaled coordinates (no scale multiplies),
    // FP32 test in units of the scaled coordinates (no scale multiplies),
    // widened by 4e-6 so that rounding never drops a partner
    const double ro = P.R + P.skin_o;
    const float r2ou = float(ro * ro * (1.0 + 4e-6) * P.inv_scl * P.inv_scl);
    const double r2o = ro * ro;
    const unsigned below = (1u << lane) - 1u;
    // candidate q of the stream: its atom index (-1 past the end)
    auto cand_of = [&](int q) -> int {
        if (q >= total) return -1;
        int lo = 0, hi = ncell - 1;               // last cell m with cpre[m] <= q
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cpre[w][mid] <= q) lo = mid; else hi = mid - 1;
        }
        return d.cell_atoms[cbeg[w][lo] + (q - cpre[w][lo])];
    };
    for (int h0 = h_lo; h0 < h_hi; h0 += 32) {
        const int nh = min(32, h_hi - h0);
        // home atoms of this pass: lane h holds atom h's count
        int cnt = 0;
        __syncwarp();
        if (lane < nh) {
            const int i = d.cell_atoms[s_i + h0 + lane];
            const uint4 pi = d.pos[i];
            home[w][lane] = make_uint4(pi.x, pi.y, pi.z, uint32_t(i));
            const int e0 = d.ex_off[i], e1 = d.ex_off[i + 1];
            hex[w][lane] = make_int4(e0 < e1 ? d.ex_idx[e0] : -1, e0 + 1 < e1 ? d.ex_idx[e0 + 1] : -1,
                                     e0 + 2 < e1 ? d.ex_idx[e0 + 2] : -1, e0 + 3 < e1 ? d.ex_idx[e0 + 3] : -1);
            hmore[w][lane] = e1 - e0 > 4 ? 1 : -1;
            hrow[w][lane] = d.olist + (size_t)i * d.ocap;
        }
        __syncwarp();
        int jn = cand_of(lane);
        uint4 pn = jn >= 0 ? d.pos[jn] : make_uint4(0, 0, 0, 0);
        for (int qb = 0; qb < total; qb += 32) {
            const int j = jn;
            const uint4 pj = pn;
            if (qb + 32 < total) {
                jn = cand_of(qb + 32 + lane);
                pn = jn >= 0 ? d.pos[jn] : make_uint4(0, 0, 0, 0);
            }
            for (int h = 0; h < nh; ++h) {
                const uint4 hp = home[w][h];
                const int i = int(hp.w);
                bool ok;
                if (exact) {            // uniform: the set-up builds
                    ok = j >= 0 && j != i && dist2_fp64(d.xo, i, j >= 0 ? j : 0, P) < r2o;
                } else {
                    const float dx = float(int(hp.x - pj.x)), dy = float(int(hp.y - pj.y)),
                                dz = float(int(hp.z - pj.z));
                    ok = (j >= 0) & (j != i) & (dx * dx + dy * dy + dz * dz < r2ou);
                }
                const int4 ex = hex[w][h];
                ok &= (j != ex.x) & (j != ex.y) & (j != ex.z) & (j != ex.w);
                if (hmore[w][h] >= 0) {         // uniform and rare: more than four exclusions
                    const int e1 = d.ex_off[i + 1];
                    for (int e = d.ex_off[i] + 4; e < e1; ++e) ok &= d.ex_idx[e] != j;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, ok);
                const int pos = __shfl_sync(0xffffffffu, cnt, h) + __popc(bal & below);
                if (ok && pos < d.ocap) hrow[w][h][pos] = (uint32_t)j;
                if (lane == h) cnt += __popc(bal);
            }
        }
        if (lane < nh) {
            const int i = int(home[w][lane].w);
            d.ocnt[i] = cnt;
            if (cnt > d.ocap) {
                atomicOr(&d.err[r], F_OVERFLOW);
                atomicOr(&d.ovf[r], OVF_OUTER);
            }
        }
    }
    }
}

// one warp per atom: filter the outer list into the inner lists, keeping its
// order. Ring and LJ membership (which decides the partner a jump picks) comes
// from the replica's shell table; candidates in a bin that holds a shell limit
// are decided in FP64 from the build positions, as in exact mode. KM is the
// set of list kinds the context builds, known at compile time for the usual
// sets (0: any, read from `kinds`). The warps stride over the atoms, so a
// launch in which no replica rebuilds costs one flag read per atom and no
// block of its own.
template <uint32_t KM>
__global__ void __launch_bounds__(32 * WARPS) k_inner_lists(Dev d, int kinds_rt, int exact, int late)
{
    // a single replica that does not rebuild: every thread sees the same flag
    if (!late && d.R == 1 && !d.flags[0]) return;
    const uint32_t kinds = KM ? KM : uint32_t(kinds_rt);
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * WARPS;
    const int i0 = blockIdx.x * WARPS + (threadIdx.x >> 5);
    for (int i = i0; i < d.N; i += nw) {
        const int r = d.rep[i];
        if (!late && !d.flags[2 * r]) continue;
        // the outer rows stream from DRAM: this warp's next row goes to L2
        // while the current one is filtered (and the first row right away)
        if (lane == 0) {
            if (i == i0) prefetch_row_l2(d.olist + (size_t)i * d.ocap, min(d.ocnt[i], d.ocap));
            const int nx = i + nw;
            if (nx < d.N && (late || d.flags[2 * d.rep[nx]]))
                prefetch_row_l2(d.olist + (size_t)nx * d.ocap, min(d.ocnt[nx], d.ocap));
        }
        const RepParams& P = d.P[r];
        const uint4 pi = d.pos[i];
        const float qi = __uint_as_float(pi.w);
        const int ti = d.type[i];
        constexpr uint32_t RING_BITS = ((1u << MAX_RINGS) - 1u) << L_R0;
        // lists this atom takes: rings (y < nr) need a charge, LJ an LJ type pair
        uint32_t want = kinds & ((1u << L_SHORT) | (1u << L_FULL));
#pragma unroll
        for (int y = 0; y < MAX_RINGS; ++y)
            if ((kinds & (1u << (L_R0 + y))) && y < P.nr && P.rings_on && qi != 0.f) want |= 1u << (L_R0 + y);
        unsigned ljmask = 0;
        if ((kinds & (1u << L_LJ)) && P.lj_on) {
            for (int t = 0; t < P.ntypes; ++t) ljmask |= (P.lj[ti * MAX_TYPES + t].on ? 1u : 0u) << t;
            if (ljmask) want |= 1u << L_LJ;
        }
        const bool need_type = (want >> L_LJ) & 1u;
        const float r2s = P.r2s, r2f = P.r2f;
        const uint16_t* tab = d.shell_tab + (size_t)r * SHELL_BINS;
        const float invw = P.shell_invw;
        const float sc = P.sclf, sclo = P.sclf_lo;
        int cnt[NKIND] = {};
        uint32_t* row[NKIND];
#pragma unroll
        for (int kind = 0; kind < NKIND; ++kind)
            row[kind] = (kinds >> kind) & 1u ? d.list[kind] + (size_t)i * d.lcap[kind] : nullptr;
        const int n_o = min(d.ocnt[i], d.ocap);
        const uint32_t* orow = d.olist + (size_t)i * d.ocap;
        // three batches of 32 candidates in flight: the entries of batch b+2 and
        // the positions (and types) of batch b+1 load while batch b is filtered
        uint32_t j1 = lane < n_o ? __ldg(orow + lane) : 0u;
        uint32_t j2 = lane + 32 < n_o ? __ldg(orow + lane + 32) : 0u;
        uint4 p1 = lane < n_o ? d.pos[j1] : make_uint4(0, 0, 0, 0);
        int t1 = (lane < n_o && need_type) ? __ldg(d.type + j1) : 0;
        for (int base = 0; base < n_o; base += 32) {
            const int k = base + lane;
            const uint32_t j = j1;
            const uint4 pj = p1;
            const int tj = t1;
            j1 = j2;
            if (k + 64 < n_o) j2 = __ldg(orow + k + 64);
            if (k + 32 < n_o) {
                p1 = d.pos[j1];
                if (need_type) t1 = __ldg(d.type + j1);
            }
            uint32_t m = 0;
            if (k < n_o) {
                uint32_t cand = want;
                if (__uint_as_float(pj.w) == 0.f) cand &= ~RING_BITS;
                if (need_type && !((ljmask >> tj) & 1u)) cand &= ~(1u << L_LJ);
                bool fp64 = exact != 0;
                if (!fp64) {
                    float dx, dy, dz;
                    sdisp(pi, pj, sc, sclo, dx, dy, dz);
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    m = (r2 < r2s ? 1u << L_SHORT : 0u) | (r2 < r2f ? 1u << L_FULL : 0u);
                    if (kinds & ~((1u << L_SHORT) | (1u << L_FULL))) {
                        const uint16_t t = __ldg(tab + min(SHELL_BINS - 1, int(r2 * invw)));
                        if (!(t & SHELL_AMB)) {
                            m |= t;
                        } else if (cand & ~((1u << L_SHORT) | (1u << L_FULL))) {
                            // a shell limit is near this bin: decide in FP32 unless r^2 is
                            // within 2e-6 (relative) of a limit, far above its FP32 error
                            bool near = false;
#pragma unroll
                            for (int y = 0; y <= MAX_RINGS; ++y) {
                                const float lo = P.shell_lo2f[y], hi = P.shell_hi2f[y];
                                near |= fabsf(r2 - lo) <= 2e-6f * lo + 1e-7f || fabsf(r2 - hi) <= 2e-6f * hi + 1e-7f;
                                if (r2 >= lo && r2 < hi) m |= 1u << (y < MAX_RINGS ? L_R0 + y : L_LJ);
                            }
                            if (near) {
                                fp64 = true;
                                m &= (1u << L_SHORT) | (1u << L_FULL);
                            }
                        }
                    }
                }
                if (fp64) {
                    const double r2 = dist2_fp64(d.xb, i, (int)j, P);
                    if (exact) m = (r2 < double(r2s) ? 1u << L_SHORT : 0u) | (r2 < double(r2f) ? 1u << L_FULL : 0u);
#pragma unroll
                    for (int y = 0; y <= MAX_RINGS; ++y)
                        if (r2 >= P.shell_lo2[y] && r2 < P.shell_hi2[y]) m |= 1u << (y < MAX_RINGS ? L_R0 + y : L_LJ);
                }
                m &= cand;
            }
            const unsigned below = (1u << lane) - 1u;
#pragma unroll
            for (int kind = 0; kind < NKIND; ++kind) {
                if (!((kinds >> kind) & 1u) || !((want >> kind) & 1u)) continue;   // warp-uniform
                const bool in = (m >> kind) & 1u;
                const unsigned b = __ballot_sync(0xffffffffu, in);
                const int pos = cnt[kind] + __popc(b & below);
                if (in && pos < d.lcap[kind]) row[kind][pos] = j;
                cnt[kind] += __popc(b);
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int kind = 0; kind < NKIND; ++kind) {
                if (!((kinds >> kind) & 1u)) continue;
                d.lcnt[kind][i] = cnt[kind];
                if (cnt[kind] > d.lcap[kind]) {
                    atomicOr(&d.err[r], F_OVERFLOW);
                    atomicOr(&d.ovf[r], 1u << kind);
                }
            }
        }
    }
}

// the usual kind sets of the drivers (BAOAB; BAOAB-RESPA1, with the LJ list
// when the LJ long part is deterministic; the JUMP family; all kinds)
constexpr uint32_t KM_FULL = 1u << L_FULL;
constexpr uint32_t KM_RESPA1 = (1u << L_FULL) | (1u << L_SHORT);
constexpr uint32_t KM_RESPA1_LJ = KM_RESPA1 | (1u << L_LJ);
constexpr uint32_t KM_JUMP = (1u << L_SHORT) | (((1u << MAX_RINGS) - 1u) << L_R0) | (1u << L_LJ);
constexpr uint32_t KM_JUMP1 = (1u << L_SHORT) | (1u << L_R0) | (1u << L_LJ);          // one ring
constexpr uint32_t KM_JUMP2 = KM_JUMP1 | (1u << (L_R0 + 1));                           // two rings
constexpr uint32_t KM_ALL = (1u << NKIND) - 1u;

// warps of a strided launch over the atoms: the resident warps of the GPU,
// at most one per atom
int inner_grid(const Dev& d)
{
    static int per_sm = 0, sms = 0;
    if (!per_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_inner_lists<KM_JUMP>, 32 * WARPS, 0);
        per_sm = std::max(per_sm, 1);
    }
    return std::max(1, std::min((d.N + WARPS - 1) / WARPS, sms * per_sm));
}

void inner_lists(const Dev& d, int kinds, int exact, int late, cudaStream_t s)
{
    if (!kinds) return;
    const int g = inner_grid(d);
    switch (uint32_t(kinds)) {
    case KM_FULL: k_inner_lists<KM_FULL><<<g, 32 * WARPS, 0, s>>>(d, kinds, exact, late); break;
    case KM_RESPA1: k_inner_lists<KM_RESPA1><<<g, 32 * WARPS, 0, s>>>(d, kinds, exact, late); break;
    case KM_RESPA1_LJ: k_inner_lists<KM_RESPA1_LJ><<<g, 32 * WARPS, 0, s>>>(d, kinds, exact, late); break;
    case KM_JUMP: k_inner_lists<KM_JUMP><<<g, 32 * WARPS, 0, s>>>(d, kinds, exact, late); break;
    case KM_JUMP1: k_inner_lists<KM_JUMP1><<<g, 32 * WARPS, 0, s>>>(d, kinds, exact, late); break;
    case KM_JUMP2: k_inner_lists<KM_JUMP2><<<g, 32 * WARPS, 0, s>>>(d, kinds, exact, late); break;
    case KM_ALL: k_inner_lists<KM_ALL><<<g, 32 * WARPS, 0, s>>>(d, kinds, exact, late); break;
    default: k_inner_lists<0><<<g, 32 * WARPS, 0, s>>>(d, kinds, exact, late); break;
    }
}

// ---- cluster tiles of the pair kernels ---------------------------------------------
// Cluster layout (at an outer rebuild): the atoms of each outer cell, ordered
// by the Morton code of the quarter-cell they sit in (from the outer-build
// positions) and then by index, cut into clusters of TILE_CL; a replica's
// clusters follow its cells. Cluster pairs (at an inner rebuild): every pair of clusters of a
// replica whose member boxes, at the current positions, come closer than the
// list radius; since a cluster's atoms lie in one cell, the candidate J of a
// cluster I are the clusters of the +-2 cells around I's cell, as for the
// outer candidates.

// per replica: first cluster of each cell; clusters past the replica's count unused
__global__ void k_cluster_scan(Dev d, int late)
{
    const int r = blockIdx.x;
    if (!late && !d.flags[2 * r + 1]) return;
    const RepParams& P = d.P[r];
    const int ncell = P.nc * P.nc * P.nc;
    const int c0 = d.cl_roff[r], c1 = d.cl_roff[r + 1];
    for (int k = c0 + threadIdx.x; k < c1; k += blockDim.x) d.cl_cell[k] = -1;
    __shared__ int warp_sum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = c0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < ncell; base += blockDim.x) {
        const int c = base + threadIdx.x;
        const int gc = P.cell_off + c;
        const int v = c < ncell ? (d.cell_start[gc + 1] - d.cell_start[gc] + TILE_CL - 1) / TILE_CL : 0;
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
            int sv = lane < nw ? warp_sum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, sv, o);
                if (lane >= o) sv += t;
            }
            if (lane < nw) warp_sum[lane] = sv;
        }
        __syncthreads();
        const int before = (w > 0 ? warp_sum[w - 1] : 0) + incl - v;
        if (c < ncell) d.cl_start[gc] = carry + before;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += before + v;
        __syncthreads();
    }
}

// one warp per cell: its atoms ordered by (sub-cell, index) into its clusters
__global__ void k_cluster_form(Dev d, int late)
{
    __shared__ long long key[WARPS][SORT_CAP];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * WARPS + w;
    if (c >= d.total_cells) return;
    const int r = d.cell_rep[c];
    if (r < 0 || (!late && !d.flags[2 * r + 1])) return;
    const RepParams& P = d.P[r];
    const int s0 = d.cell_start[c], n = d.cell_start[c + 1] - s0;
    if (n > SORT_CAP) return;               // the cell sort has flagged the overflow
    const int lin = c - P.cell_off;
    const double inv_q = 4.0 / P.cs;        // quarter-cell units
    const double o3[3] = {(lin % P.nc) * P.cs, ((lin / P.nc) % P.nc) * P.cs, (lin / (P.nc * P.nc)) * P.cs};
    for (int k = lane; k < n; k += 32) {
        const int i = d.cell_atoms[s0 + k];
        // Morton order of the 4 x 4 x 4 sub-cells: eight consecutive atoms stay close
        int code = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int q = min(3, max(0, int((d.xo[3 * i + a] - o3[a]) * inv_q)));
            code |= ((q & 1) << a) | (((q >> 1) & 1) << (3 + a));
        }
        key[w][k] = ((long long)code << 32) | (long long)i;
    }
    __syncwarp();
    const int first = d.cl_start[c];
    const int ncl = (n + TILE_CL - 1) / TILE_CL;
    for (int k = lane; k < ncl * TILE_CL; k += 32) {
        const int cl = first + k / TILE_CL, slot = k % TILE_CL;
        if (slot == 0) d.cl_cell[cl] = c;
        if (k >= n) d.cl_atom[TILE_CL * (size_t)cl + slot] = -1;
    }
    for (int k = lane; k < n; k += 32) {
        const long long v = key[w][k];
        int rank = 0;
        for (int m = 0; m < n; ++m) rank += key[w][m] < v;
        const int i = int(v & 0xffffffffll);
        const int cl = first + rank / TILE_CL, slot = rank % TILE_CL;
        d.cl_atom[TILE_CL * (size_t)cl + slot] = i;
        d.cl_of[i] = cl;
        d.cl_slot[i] = slot;
    }
}

// one thread per cluster: reference position (slot 0) and the members' box
// relative to it, from the current scaled coordinates
__global__ void k_cluster_boxes(Dev d, int late)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= d.ncl_cap) return;
    const int cell = d.cl_cell[I];
    if (cell < 0) return;
    const int r = d.cell_rep[cell];
    if (!late && !d.flags[2 * r]) return;
    const int* at = d.cl_atom + TILE_CL * (size_t)I;
    const uint4 ref = d.pos[at[0]];
    int4 lo = make_int4(0, 0, 0, 0), hi = make_int4(0, 0, 0, 0);
    for (int s = 1; s < TILE_CL; ++s) {
        const int i = at[s];
        if (i < 0) continue;
        const uint4 p = d.pos[i];
        const int dx = int(p.x - ref.x), dy = int(p.y - ref.y), dz = int(p.z - ref.z);
        lo.x = min(lo.x, dx); lo.y = min(lo.y, dy); lo.z = min(lo.z, dz);
        hi.x = max(hi.x, dx); hi.y = max(hi.y, dy); hi.z = max(hi.z, dz);
    }
    d.cl_ref[I] = ref;
    d.cl_lo[I] = lo;
    d.cl_hi[I] = hi;
}

// the gap between two boxes along one axis, in scaled units: I's box
// [lo, hi] and J's box [dr + loj, dr + hij] relative to I's reference
__device__ __forceinline__ float box_gap(int dr, int lo, int hi, int loj, int hij)
{
    const long long a = (long long)dr + loj - hi, b = (long long)lo - ((long long)dr + hij);
    return float(max(0ll, max(a, b)));
}

// one warp per cluster I: the clusters J >= I of the +-2 cells around I's
// cell (lanes over the candidates, the next batch loading while the current
// one is tested) whose boxes come within the radius of list tl, with the
// mask of the slot pairs to take
__global__ void __launch_bounds__(32 * WARPS) k_cluster_pairs(Dev d, int tl, int late)
{
    __shared__ int nbs[WARPS][128];
    __shared__ int cpre[WARPS][129];
    __shared__ int cbeg[WARPS][128];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    for (int I = blockIdx.x * WARPS + w; I < d.ncl_cap; I += gridDim.x * WARPS) {
        const int cell = d.cl_cell[I];
        if (cell < 0) continue;
        const int r = d.cell_rep[cell];
        if (!late && !d.flags[2 * r]) continue;
        const RepParams& P = d.P[r];
        const int nc = P.nc;
        const int lin = cell - P.cell_off;
        const int cc[3] = {lin % nc, (lin / nc) % nc, lin / (nc * nc)};
        const int nax = nc >= 5 ? 5 : nc;
        const int ncell = nax * nax * nax;
        __syncwarp();
        for (int t = lane; t < ncell; t += 32) {
            const int q[3] = {t % nax, (t / nax) % nax, t / (nax * nax)};
            int cv[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) cv[a] = nc >= 5 ? (cc[a] + q[a] - 2 + nc) % nc : q[a];
            const int gc = P.cell_off + (cv[2] * nc + cv[1]) * nc + cv[0];
            nbs[w][t] = gc;
        }
        __syncwarp();
        // candidate clusters: lane l holds neighbour cells 4l .. 4l+3; warp scan of their counts
        int cntc[4], sum = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int m = 4 * lane + u;
            cntc[u] = 0;
            if (m < ncell) {
                const int gc = nbs[w][m];
                cbeg[w][m] = d.cl_start[gc];
                cntc[u] = (d.cell_start[gc + 1] - d.cell_start[gc] + TILE_CL - 1) / TILE_CL;
            }
            sum += cntc[u];
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        {
            int run = incl - sum;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int m = 4 * lane + u;
                if (m <= ncell) cpre[w][m] = run;
                run += cntc[u];
            }
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (lane == 31) cpre[w][ncell] = total;
        __syncwarp();
        const double rl = (tl == 0 ? fmin(P.rc, P.R) : P.R) + P.skin;
        // FP32 test in Angstrom, widened by 1e-5 so that rounding never drops a pair
        const float rl2 = float(rl * rl * (1.0 + 1e-5));
        const float sc = P.sclf;
        const uint4 refI = d.cl_ref[I];
        const int4 loI = d.cl_lo[I], hiI = d.cl_hi[I];
        const int* atI = d.cl_atom + TILE_CL * (size_t)I;
        const int cap = d.cpl_cap[tl];
        int* jrow = d.cpl_j[tl] + (size_t)I * cap;
        unsigned long long* mrow = d.cpl_mask[tl] + (size_t)I * cap;
        int cnt = 0;
        for (int qb = 0; qb < total; qb += 32) {
            const int q = qb + lane;
            int J = -1;
            if (q < total) {
                int lo = 0, hi = ncell - 1;               // last cell m with cpre[m] <= q
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (cpre[w][mid] <= q) lo = mid; else hi = mid - 1;
                }
                J = cbeg[w][lo] + (q - cpre[w][lo]);
            }
            bool ok = J >= I;
            unsigned long long mask = 0;
            if (ok) {
                const uint4 refJ = d.cl_ref[J];
                const int4 loJ = d.cl_lo[J], hiJ = d.cl_hi[J];
                const float gx = box_gap(int(refJ.x - refI.x), loI.x, hiI.x, loJ.x, hiJ.x) * sc;
                const float gy = box_gap(int(refJ.y - refI.y), loI.y, hiI.y, loJ.y, hiJ.y) * sc;
                const float gz = box_gap(int(refJ.z - refI.z), loI.z, hiI.z, loJ.z, hiJ.z) * sc;
                ok = gx * gx + gy * gy + gz * gz < rl2;
            }
            if (ok) {
                const int* atJ = d.cl_atom + TILE_CL * (size_t)J;
                unsigned occI = 0, occJ = 0;
#pragma unroll
                for (int s = 0; s < TILE_CL; ++s) {
                    occI |= (atI[s] >= 0 ? 1u : 0u) << s;
                    occJ |= (atJ[s] >= 0 ? 1u : 0u) << s;
                }
#pragma unroll
                for (int a = 0; a < TILE_CL; ++a) {
                    if (!((occI >> a) & 1u)) continue;
                    unsigned row = occJ;
                    if (J == I) row &= ~((2u << a) - 1u);      // b > a within one cluster
                    mask |= (unsigned long long)row << (TILE_CL * a);
                    const int i = atI[a];
                    for (int e = d.ex_off[i]; e < d.ex_off[i + 1]; ++e) {
                        const int x = d.ex_idx[e];
                        if (d.cl_of[x] == J) mask &= ~(1ull << (TILE_CL * a + d.cl_slot[x]));
                    }
                }
                ok = mask != 0;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, ok);
            const int pos = cnt + __popc(bal & below);
            if (ok && pos < cap) {
                jrow[pos] = J;
                mrow[pos] = mask;
            }
            cnt += __popc(bal);
        }
        if (lane == 0) {
            d.cpl_n[tl][I] = cnt;
            if (cnt > cap) {
                atomicOr(&d.err[r], F_OVERFLOW);
                atomicOr(&d.ovf[r], OVF_TILE);
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

// blocks of a strided outer-candidate launch: the resident blocks of the GPU,
// at most one warp per task
static int outer_grid(long long tasks)
{
    static int per_sm = 0, sms = 0;
    if (!per_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_outer_cells, 32 * OUTER_WARPS, 0);
        per_sm = std::max(per_sm, 1);
    }
    return (int)std::max(1LL, std::min((tasks + OUTER_WARPS - 1) / OUTER_WARPS, (long long)sms * per_sm));
}

void launch_rebuild_cells(const Dev& d, int keep_refs, int exact_outer, cudaStream_t s)
{
    k_rehome<<<blocks(d.N, 256), 256, 0, s>>>(d, keep_refs);
    k_cell_scan<<<d.R, 1024, 0, s>>>(d);
    k_cell_fill<<<blocks(d.N, 256), 256, 0, s>>>(d);
    k_cell_sort<<<blocks(d.total_cells, WARPS), 32 * WARPS, 0, s>>>(d);
    // OUTER_GROUPS warps per cell, each looping over its groups of 32 atoms
    const long long tasks = (long long)d.total_cells * OUTER_GROUPS;
    k_outer_cells<<<outer_grid(tasks), 32 * OUTER_WARPS, 0, s>>>(d, exact_outer);
}

void launch_rebuild_inner(const Dev& d, int kinds, int exact, cudaStream_t s)
{
    inner_lists(d, kinds, exact, 0, s);
}

void launch_rebuild_done(const Dev& d, cudaStream_t s)
{
    k_flags_clear<<<blocks(d.R, 128), 128, 0, s>>>(d);
}

void launch_rebuild(const Dev& d, int kinds, int exact, int keep_refs, int exact_outer,
                    int /*max_cells_per_rep*/, cudaStream_t s)
{
    launch_rebuild_cells(d, keep_refs, exact_outer, s);
    launch_rebuild_inner(d, kinds, exact, s);
    launch_tiles(d, d.tiles, s);
    launch_rebuild_done(d, s);
}

void launch_late_lists(const Dev& d, int kinds, cudaStream_t s)
{
    inner_lists(d, kinds, 1, 1, s);
}

static void tiles_chain(const Dev& d, int tiles, int late, cudaStream_t s)
{
    if (!tiles || !d.ncl_cap) return;
    k_cluster_scan<<<d.R, 1024, 0, s>>>(d, late);
    k_cluster_form<<<blocks(d.total_cells, WARPS), 32 * WARPS, 0, s>>>(d, late);
    k_cluster_boxes<<<blocks(d.ncl_cap, 128), 128, 0, s>>>(d, late);
    static int per_sm = 0, sms = 0;
    if (!per_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cluster_pairs, 32 * WARPS, 0);
        per_sm = std::max(per_sm, 1);
    }
    const int g = std::max(1, std::min(blocks(d.ncl_cap, WARPS), sms * per_sm));
    for (int t = 0; t < 2; ++t)
        if ((tiles >> t) & 1) k_cluster_pairs<<<g, 32 * WARPS, 0, s>>>(d, t, late);
}

void launch_tiles(const Dev& d, int tiles, cudaStream_t s)
{
    tiles_chain(d, tiles, 0, s);
}

void launch_tiles_late(const Dev& d, int tiles, cudaStream_t s)
{
    tiles_chain(d, tiles, 1, s);
}

}  // namespace mdj
