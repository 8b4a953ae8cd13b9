// md_api.cu -- host engine and C ABI of libmdjump.so (declared in include/md.h).
//
// The context keeps a host copy of every replica's topology and parameters,
// lays all replicas out end to end in device memory (one launch advances all
// of them), computes the per-atom rate bounds of the jump rings on the host,
// and drives the integrators of Sec. 2.3 as sequences of kernel launches on
// one CUDA stream. Device memory is allocated stream-ordered on that stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cufft.h>

#include "../../include/md.h"
#include "engine.h"

using namespace mdj;

static_assert(NPROF == MD_PROFILE_CLASSES, "launch classes of md_profile");

namespace {

// ---- host pair terms for the rate bounds (FP64) --------------------------------
struct HostPair {
    double R, sw, h, alpha;
    int ewald = 0;          // 1: Ewald real space erfc(a r)/r, no value or slope shift
    double chi(double r) const
    {
        if (r <= sw) return 1.0;
        if (r >= sw + h) return 0.0;
        const double s = (r - sw) / h;
        return 1.0 - s * s * s * (10.0 - 15.0 * s + 6.0 * s * s);
    }
    double dchi(double r) const
    {
        if (r <= sw || r >= sw + h) return 0.0;
        const double s = (r - sw) / h;
        return -30.0 * s * s * (1.0 - s) * (1.0 - s) / h;
    }
    double fR() const
    {
        if (ewald) return 0.0;
        return std::erfc(alpha * R) / (R * R) + 2.0 * alpha / std::sqrt(PI) * std::exp(-alpha * alpha * R * R) / R;
    }
    double u_dsf(double r) const
    {
        if (r >= R) return 0.0;
        if (ewald) return std::erfc(alpha * r) / r;
        return std::erfc(alpha * r) / r - std::erfc(alpha * R) / R + fR() * (r - R);
    }
    double du_dsf(double r) const
    {
        if (r >= R) return 0.0;
        return -(std::erfc(alpha * r) / (r * r) + 2.0 * alpha / std::sqrt(PI) * std::exp(-alpha * alpha * r * r) / r) + fR();
    }
    static double lj(double c12, double c6, double r) { return c12 / std::pow(r, 12) - c6 / std::pow(r, 6); }
    static double dlj(double c12, double c6, double r) { return -12.0 * c12 / std::pow(r, 13) + 6.0 * c6 / std::pow(r, 7); }
    double u_ljsf(double c12, double c6, double r) const
    {
        if (r >= R) return 0.0;
        return lj(c12, c6, r) - lj(c12, c6, R) - (r - R) * dlj(c12, c6, R);
    }
    double du_ljsf(double c12, double c6, double r) const
    {
        if (r >= R) return 0.0;
        return dlj(c12, c6, r) - dlj(c12, c6, R);
    }
};

constexpr int NGRID = 20001;

// max of |d/dr (1 - chi) U| on [lo, hi] sampled at NGRID points
template <class F> double grid_max(F f, double lo, double hi)
{
    if (!(hi > lo)) return 0.0;
    double m = 0.0;
    for (int k = 0; k < NGRID; ++k) {
        const double r = lo + (hi - lo) * (double)k / (double)(NGRID - 1);
        const double v = std::fabs(f(r));
        if (v > m) m = v;
    }
    return m;
}

// bound rounded up to 9 significant bits after a 1e-4 safety factor
double round_up_bound(double x)
{
    if (!(x > 0.0)) return 0.0;
    int e;
    double f = std::frexp(x * (1.0 + 1e-4), &e);
    f = std::ceil(f * 512.0) / 512.0;
    return std::ldexp(f, e);
}

struct RepHost {
    bool set = false;
    bool fresh = true;      // state comes from md_set_system, not from the device
    int n = 0;
    double box = 0;
    std::vector<double> x, v, xb, xo, mass, charge, lj_eps, lj_sig, bond_k, bond_r0, ang_k, ang_t0;
    std::vector<int> img, type, bonds, angles, excl;
    int ntypes = 0;
    md_system sys{};
    long long step = 0;
    std::vector<unsigned long long> cnt;
    uint32_t err = 0;
};

}  // namespace

struct md_ctx {
    md_config cfg{};
    cudaStream_t s = nullptr;
    std::string msg;
    std::vector<RepHost> reps;
    bool dirty = true;
    bool on_device = false;
    int kinds = 0;          // inner list kinds built so far
    int fp64 = 0;
    int tpa_cfg = 0;
    int tpa[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // pair kernel choice per gradient mode (7: the LJ long part alone)
    int vvar = -1;          // chosen variant of the mixed-mode velocity-phase kernel
    bool tune_log = false;  // report the autotuners' choices on stderr (MDJ_TUNE_LOG)
    bool fuse_inner = false;      // run the inner steps fused (MDJ_FUSED_INNER; separate launches otherwise)
    Dev d{};
    std::vector<void*> bufs;
    std::vector<RepParams> hp;
    std::vector<int> rep_atom_off;
    // launch accounting and optional per-class timing
    long long nlaunch[NPROF] = {};
    bool prof = false;
    double prof_ms[NPROF] = {};
    long long prof_groups[NPROF] = {};
    std::vector<cudaEvent_t> ev_pool;
    struct Pend { int cls; cudaEvent_t a, b; };
    std::vector<Pend> pend;
    // CUDA graphs of driver chunks (see run_units); gen changes whenever the
    // device layout does, which invalidates every captured graph
    cudaStream_t gs = nullptr;
    // second stream of the reciprocal sum: forked from the main stream once the
    // positions of a slow step are final, joined before the slow kick
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool recip_open = false;
    double* arecip = nullptr;       // [N][3] reciprocal acceleration of the slow level
    long long gen = 0;
    struct Graph { long long gen; int key; double tau; int n_inner, units; cudaGraphExec_t exec;
                   long long launches[NPROF]; };
    std::vector<Graph> graphs;
    bool graphs_broken = false;
    long long ngraph_launches = 0;  // graph replays issued (each replays a chunk of a driver)
    // smooth PME: one pair of cuFFT plans (real to complex, complex to real) per grid size
    struct FftPlan { int K; cufftHandle d2z, z2d; };
    std::vector<FftPlan> fft;
    std::vector<int> ewald_reps;
    std::vector<int> pme_orders;    // B-spline orders present
    long long pme_total = 0;        // grid points over all Ewald replicas
    long long pme_max_spec = 0;     // largest half spectrum
    // velocity record (md_vacf_start): [cap][3N] values, FP64 or FP32 as the precision
    void* vr = nullptr;
    long long vr_cap = 0, vr_origin = 0;
    // error of a call made inside a driver body (cuFFT), reported at the end of the call
    int deferred = MD_OK;
    // pinned staging
    double* h_stepc = nullptr;
    uint32_t* h_err = nullptr;
};

static std::string g_init_msg = "no error";
static std::mutex g_msg_mutex;

namespace mdj {
// message of the last failed call that has no context (md_init, the no-allocation entry)
void set_global_error(const std::string& msg)
{
    std::lock_guard<std::mutex> lock(g_msg_mutex);
    g_init_msg = msg;
}
}

#define FAIL(code, ...)                                                   \
    do {                                                                  \
        char _b[512];                                                     \
        std::snprintf(_b, sizeof _b, __VA_ARGS__);                        \
        ctx->msg = _b;                                                    \
        return code;                                                      \
    } while (0)

#define CK(call)                                                          \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) FAIL(MD_ECUDA, "%s: %s", #call, cudaGetErrorString(_e)); \
    } while (0)

namespace {

template <typename T> int dalloc(md_ctx* ctx, T** p, size_t count)
{
    const size_t bytes = (count ? count : 1) * sizeof(T);
    cudaError_t e = cudaMallocAsync((void**)p, bytes, ctx->s);
    if (e != cudaSuccess) {
        ctx->msg = std::string("device allocation failed: ") + cudaGetErrorString(e);
        return MD_ENOMEM;
    }
    ctx->bufs.push_back((void*)*p);
    ctx->gen++;
    return MD_OK;
}

// release a buffer that a larger one replaced (stream-ordered: launches
// already queued, and graphs already launched, still see it)
void dfree(md_ctx* ctx, void* p)
{
    auto it = std::find(ctx->bufs.begin(), ctx->bufs.end(), p);
    if (it == ctx->bufs.end()) return;
    cudaFreeAsync(p, ctx->s);
    ctx->bufs.erase(it);
}

template <typename T> int upload(md_ctx* ctx, T* dst, const T* src, size_t count)
{
    if (!count) return MD_OK;
    cudaError_t e = cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, ctx->s);
    if (e != cudaSuccess) {
        ctx->msg = std::string("upload failed: ") + cudaGetErrorString(e);
        return MD_ECUDA;
    }
    return MD_OK;
}

// end a velocity record (its buffer is freed; captured graphs that record are dropped)
void vacf_stop(md_ctx* ctx)
{
    if (ctx->vr) cudaFreeAsync(ctx->vr, ctx->s);
    ctx->vr = nullptr;
    ctx->vr_cap = 0;
    ctx->gen++;
}

void free_device(md_ctx* ctx)
{
    for (void* p : ctx->bufs) cudaFreeAsync(p, ctx->s);
    ctx->bufs.clear();
    ctx->on_device = false;
}

// does some replica keep the LJ long part at the slow level (lj_long_mode 2)?
bool any_lj_slow(const md_ctx* ctx)
{
    for (const RepParams& P : ctx->hp)
        if (P.lj_long == 2) return true;
    return false;
}

// does some replica keep the LJ long part deterministic (its short gradient
// then also runs over the LJ list)?
bool any_lj_long(const md_ctx* ctx)
{
    for (const RepParams& P : ctx->hp)
        if (P.lj_long) return true;
    return false;
}

int lists_needed(const md_ctx* ctx, int family)
{
    // 0 BAOAB / BAOAB-RESPA, 1 BAOAB-RESPA1, 2 JUMP family
    const int lj = any_lj_long(ctx) ? 1 << L_LJ : 0;
    if (family == 0) return 1 << L_FULL;
    if (family == 1) return (1 << L_FULL) | (1 << L_SHORT) | lj;
    // the rings some replica has (the list filter is compiled for the usual sets)
    int nr = 0;
    for (const RepParams& P : ctx->hp) nr = std::max(nr, P.nr);
    int k = (1 << L_SHORT) | (1 << L_LJ);
    for (int y = 0; y < std::max(nr, 1); ++y) k |= 1 << (L_R0 + y);
    return k;
}

int mode_list(const md_ctx* ctx, int mode)
{
    if (mode == 1) return 0;
    if (mode == 6) return any_lj_slow(ctx) ? 1 << L_LJ : 0;
    if (mode == 3 || mode == 5) return (1 << L_SHORT) | (any_lj_long(ctx) ? 1 << L_LJ : 0);
    return 1 << L_FULL;
}

// estimated per-atom capacity of a list with shell [lo, hi] at density rho
int cap_of(double rho, double lo, double hi)
{
    lo = std::max(lo, 0.0);
    const double vol = 4.0 / 3.0 * PI * (hi * hi * hi - lo * lo * lo);
    int c = int(vol * rho * 1.5) + 64;
    return (c + 31) / 32 * 32;
}

// skin-widened shell [lo, hi) of list kind k in one replica (hi <= lo: empty)
void shell_of(const RepParams& P, int k, double& lo, double& hi)
{
    const double sk = P.skin;
    lo = 0.0; hi = 0.0;
    if (k == L_SHORT) hi = P.rc + sk;
    else if (k == L_FULL) hi = P.R + sk;
    else if (k == L_LJ) { lo = P.sw - sk; hi = P.R + sk; }
    else if (k - L_R0 < P.nr) { lo = P.edge[k - L_R0] - sk; hi = P.edge[k - L_R0 + 1] + sk; }
}

// per-atom capacity of list kind k over all replicas (32 when every shell is empty)
int kind_cap(const md_ctx* ctx, int k)
{
    double rho = 0, lo = 1e300, hi = 0;
    for (const RepParams& P : ctx->hp) {
        double a, b;
        shell_of(P, k, a, b);
        if (b <= a) continue;
        rho = std::max(rho, P.n / (P.L * P.L * P.L));
        lo = std::min(lo, a); hi = std::max(hi, b);
    }
    return hi > 0 ? cap_of(rho, lo, hi) : 32;
}

// shell table of one replica (see SHELL_BINS): bins of r^2 over [0, (r_E +
// skin_outer)^2); a bin is ambiguous when a ring or LJ shell limit lies within
// it or within a margin of 2e-5 r^2 + 1e-6 A^2 of it (far wider than the FP32
// error of r^2), otherwise it lists the ring and LJ kinds that contain it
void make_shell_table(const RepParams& P, uint16_t* tab)
{
    const double r2max = (P.R + P.skin_o) * (P.R + P.skin_o);
    const double w = r2max / SHELL_BINS;
    double lo2[NKIND], hi2[NKIND];
    bool use[NKIND];
    for (int k = 0; k < NKIND; ++k) {
        double lo, hi;
        shell_of(P, k, lo, hi);
        lo = std::max(lo, 0.0);
        use[k] = k != L_SHORT && k != L_FULL && hi > lo;
        lo2[k] = lo * lo;
        hi2[k] = hi * hi;
    }
    for (int b = 0; b < SHELL_BINS; ++b) {
        const double a = b * w, e = b == SHELL_BINS - 1 ? 1e300 : (b + 1) * w;
        const double ma = 2e-5 * a + 1e-6, me = 2e-5 * std::min(e, 1e30) + 1e-6;
        uint16_t t = 0;
        bool amb = b == SHELL_BINS - 1;
        for (int k = 0; k < NKIND; ++k) {
            if (!use[k]) continue;
            for (double lim : {lo2[k], hi2[k]})
                if (lim > 0.0 && lim >= a - ma && lim <= e + me) amb = true;
            if (lo2[k] <= a && e <= hi2[k]) t |= uint16_t(1u << k);
        }
        tab[b] = amb ? SHELL_AMB : t;
    }
}

// smooth PME grid points per edge: the smallest 2,3,5-smooth K >= max(L / spacing, 2 p)
int pme_grid_size(double L, double spacing, int p)
{
    int K = std::max((int)std::ceil(L / spacing), 2 * p);
    for (;; ++K) {
        int m = K;
        while (m % 2 == 0) m /= 2;
        while (m % 3 == 0) m /= 3;
        while (m % 5 == 0) m /= 5;
        if (m == 1) return K;
    }
}

// cardinal B-spline M_p at u (zero outside (0, p)), by its recursion in p
double host_bspline(int p, double u)
{
    if (u <= 0.0 || u >= p) return 0.0;
    if (p == 2) return 1.0 - std::fabs(u - 1.0);
    return (u * host_bspline(p - 1, u) + (p - u) * host_bspline(p - 1, u - 1.0)) / (p - 1);
}

// influence function of one replica on the half spectrum [m2][m1][m0 <= K/2]:
// G(m) = (C / (pi V)) exp(-pi^2 |m|^2 / a^2) / |m|^2 / |b1 b2 b3|^2, G(0) = 0, with
// |b(m)|^-2 = |sum_{k=0}^{p-2} M_p(k + 1) exp(2 pi i m k / K)|^2 (Essmann et al. 1995)
void make_pme_G(const RepParams& P, double* G)
{
    const int K = P.pme_K, Kh = K / 2 + 1, p = P.pme_p;
    std::vector<double> bm(K);
    for (int m = 0; m < K; ++m) {
        double sr = 0.0, si = 0.0;
        for (int k = 0; k <= p - 2; ++k) {
            const double th = 2.0 * PI * m * k / K;
            sr += host_bspline(p, k + 1.0) * std::cos(th);
            si += host_bspline(p, k + 1.0) * std::sin(th);
        }
        const double d2 = sr * sr + si * si;
        bm[m] = d2 > 1e-300 ? 1.0 / d2 : 0.0;
    }
    const double V = P.L * P.L * P.L, a = P.alpha;
    for (int m2 = 0; m2 < K; ++m2)
        for (int m1 = 0; m1 < K; ++m1)
            for (int m0 = 0; m0 < Kh; ++m0) {
                const double f2 = (m2 <= K / 2 ? m2 : m2 - K) / P.L, f1 = (m1 <= K / 2 ? m1 : m1 - K) / P.L;
                const double f0 = m0 / P.L;
                const double msq = f0 * f0 + f1 * f1 + f2 * f2;
                double g = 0.0;
                if (msq > 0.0) g = COULOMB / (PI * V) * std::exp(-PI * PI * msq / (a * a)) / msq * bm[m0] * bm[m1] * bm[m2];
                G[((size_t)m2 * K + m1) * Kh + m0] = g;
            }
}

RepParams make_params(const md_ctx* ctx, const RepHost& h, int r, int atom_off, int cell_off)
{
    const md_system& s = h.sys;
    RepParams P;
    std::memset(&P, 0, sizeof P);
    P.L = h.box; P.invL = 1.0 / h.box;
    P.atom_off = atom_off; P.n = h.n;
    const double skin_o = std::max(s.skin, s.skin_outer);
    P.nc = std::max(1, int(std::floor(2.0 * h.box / (s.r_cut + skin_o))));
    P.cs = h.box / P.nc;
    P.cell_off = cell_off;
    P.scl = h.box / 4294967296.0;
    P.inv_scl = 4294967296.0 / h.box;
    P.sclf = float(P.scl);
    P.sclf_lo = float(P.scl - double(P.sclf));
    P.R = s.r_cut; P.rc = s.r_split; P.h = s.h_switch; P.sw = s.r_split - s.h_switch;
    P.scl2f = float(P.scl * P.scl);
    {
        const double t = std::max(P.sw, 0.0) * P.inv_scl;      // below 2^31: sw < r_E < L / 2
        P.sw2u = (unsigned long long)std::llrint(t * t);
    }
    // ring edges (Sec. 3.1 ring technique): explicit interior edges, else r_M
    // when it lies inside (r_c - h, r_E), else one ring
    P.edge[0] = P.sw;
    if (s.n_rings >= 1) {
        P.nr = std::min(s.n_rings, MAX_RINGS);
        for (int y = 1; y < P.nr; ++y) P.edge[y] = s.ring_r[y - 1];
    } else {
        P.nr = (s.r_mid > P.sw && s.r_mid < P.R) ? 2 : 1;
        if (P.nr == 2) P.edge[1] = s.r_mid;
    }
    P.edge[P.nr] = P.R;
    for (int y = P.nr + 1; y <= MAX_RINGS; ++y) P.edge[y] = P.R;
    for (int y = 0; y <= MAX_RINGS; ++y) P.edgef[y] = float(P.edge[y]);
    double qmax = 0;
    for (double q : h.charge) qmax = std::max(qmax, std::fabs(q));
    bool any_lj = false;
    for (double e : h.lj_eps) any_lj |= e > 0.0;
    P.rings_on = (P.sw < P.R) && qmax > 0.0;
    P.lj_on = (P.sw < P.R) && any_lj;
    P.lj_long = s.lj_long_mode;
    P.lj_jump = P.lj_on && P.lj_long == 0;
    P.eps_mode = s.eps_mode;
    P.skin = s.skin; P.skin_o = skin_o;
    HostPair hpair{s.r_cut, P.sw, s.h_switch, s.dsf_alpha, s.coulomb_mode};
    P.alpha = s.dsf_alpha;
    // Ewald real space: the same pair code with no value or slope shift at r_E
    P.eR = s.coulomb_mode == 1 ? 0.0 : std::erfc(s.dsf_alpha * s.r_cut) / s.r_cut;
    P.fR = hpair.fR();
    P.coul_mode = s.coulomb_mode;
    if (s.coulomb_mode == 1) {
        P.pme_p = s.pme_order;
        P.pme_K = pme_grid_size(h.box, s.pme_spacing, s.pme_order);
        double q2 = 0.0;
        for (double q : h.charge) q2 += q * q;
        P.pme_self = -COULOMB * s.dsf_alpha / std::sqrt(PI) * q2;
    }
    P.kexp = 2.0 * s.dsf_alpha / std::sqrt(PI);
    P.alphaf = float(P.alpha); P.eRf = float(P.eR); P.fRf = float(P.fR); P.kexpf = float(P.kexp);
    P.shell_invw = float(SHELL_BINS / ((s.r_cut + skin_o) * (s.r_cut + skin_o)));
    for (int y = 0; y <= MAX_RINGS; ++y) {
        double lo, hi;
        if (y < MAX_RINGS) { lo = y < P.nr ? P.edge[y] - s.skin : 0.0; hi = y < P.nr ? P.edge[y + 1] + s.skin : 0.0; }
        else { lo = P.sw - s.skin; hi = P.R + s.skin; }
        lo = std::max(lo, 0.0);
        P.shell_lo2[y] = lo * lo; P.shell_hi2[y] = hi * hi;
        P.shell_lo2f[y] = float(P.shell_lo2[y]); P.shell_hi2f[y] = float(P.shell_hi2[y]);
    }
    P.r2s = float((s.r_split + s.skin) * (s.r_split + s.skin));
    P.r2f = float((s.r_cut + s.skin) * (s.r_cut + s.skin));
    P.beta = 1.0 / (KB * s.temperature);
    P.gamma = s.gamma;
    P.eps0 = s.eps0;
    P.seed = uint32_t(ctx->cfg.seed & 0xffffffffull);
    P.replica = uint32_t(r);
    P.ntypes = h.ntypes;
    for (int a = 0; a < h.ntypes; ++a)
        for (int b = 0; b < h.ntypes; ++b) {
            const double e = h.lj_eps[a * h.ntypes + b], sg = h.lj_sig[a * h.ntypes + b];
            LJPair& l = P.lj[a * MAX_TYPES + b];
            l.c12 = 4.0 * e * std::pow(sg, 12);
            l.c6 = 4.0 * e * std::pow(sg, 6);
            l.uR = HostPair::lj(l.c12, l.c6, s.r_cut);
            l.duR = HostPair::dlj(l.c12, l.c6, s.r_cut);
            l.c12f = float(l.c12); l.c6f = float(l.c6); l.uRf = float(l.uR); l.duRf = float(l.duR);
            l.on = e > 0.0;
        }
    return P;
}

// per-atom bounds of a replica: L_Y per ring (C |q_i| qmax Lhat_Y, n x MAX_RINGS) and L_LJ
void make_bounds(const RepHost& h, const RepParams& P, double* LY, double* LLJ)
{
    HostPair hp{P.R, P.sw, P.h, P.alpha, P.coul_mode};
    auto coul = [&](double r) { return -hp.dchi(r) * hp.u_dsf(r) + (1.0 - hp.chi(r)) * hp.du_dsf(r); };
    double Lh[MAX_RINGS] = {};
    for (int y = 0; y < P.nr; ++y) Lh[y] = grid_max(coul, P.edge[y], P.edge[y + 1]);
    double qmax = 0;
    for (double q : h.charge) qmax = std::max(qmax, std::fabs(q));
    const int nt = h.ntypes;
    std::vector<double> ljhat(nt * nt, 0.0);
    std::vector<int> present(nt, 0);
    for (int t : h.type) present[t] = 1;
    for (int a = 0; a < nt; ++a)
        for (int b = 0; b < nt; ++b) {
            const LJPair& l = P.lj[a * MAX_TYPES + b];
            if (!l.on) continue;
            auto f = [&](double r) {
                return -hp.dchi(r) * hp.u_ljsf(l.c12, l.c6, r) + (1.0 - hp.chi(r)) * hp.du_ljsf(l.c12, l.c6, r);
            };
            ljhat[a * nt + b] = grid_max(f, P.sw, P.R);
        }
    for (int i = 0; i < h.n; ++i) {
        const double cq = COULOMB * std::fabs(h.charge[i]) * qmax;
        for (int y = 0; y < MAX_RINGS; ++y)
            LY[MAX_RINGS * i + y] = y < P.nr ? round_up_bound(cq * Lh[y]) : 0.0;
        double m = 0;
        for (int b = 0; b < nt; ++b)
            if (present[b]) m = std::max(m, ljhat[h.type[i] * nt + b]);
        LLJ[i] = round_up_bound(m);
    }
}

int check_sys(md_ctx* ctx, const md_system* s)
{
    if (!s || s->n_atoms <= 0 || !s->x || !s->v || !s->mass || !s->charge || !s->type)
        FAIL(MD_EINVAL, "md_set_system: missing atom arrays");
    if (s->n_types < 1 || s->n_types > MAX_TYPES || !s->lj_eps || !s->lj_sigma)
        FAIL(MD_EINVAL, "md_set_system: n_types must be in [1, %d] with LJ tables", MAX_TYPES);
    if (!(s->r_cut > 0) || !(s->h_switch > 0) || !(s->r_split > s->h_switch) || !(s->skin >= 0) ||
        !(s->dsf_alpha >= 0) || !(s->gamma >= 0) || !(s->temperature > 0) || !(s->eps0 > 0) ||
        (s->eps_mode != 0 && s->eps_mode != 1))
        FAIL(MD_EINVAL, "md_set_system: invalid cutoff, switch, thermostat or jump parameters");
    if (s->lj_long_mode < 0 || s->lj_long_mode > 2)
        FAIL(MD_EINVAL, "md_set_system: lj_long_mode must be 0, 1 or 2");
    if (s->coulomb_mode != 0 && s->coulomb_mode != 1)
        FAIL(MD_EINVAL, "md_set_system: coulomb_mode must be 0 (DSF) or 1 (Ewald)");
    if (s->coulomb_mode == 1) {
        // an odd order makes the B-spline factor |b(m)|^2 vanish at m = K/2 on an even grid
        if (!(s->dsf_alpha > 0) || (s->pme_order != 4 && s->pme_order != 6 && s->pme_order != 8) ||
            !(s->pme_spacing > 0))
            FAIL(MD_EINVAL, "md_set_system: Ewald needs dsf_alpha > 0, pme_order 4, 6 or 8, pme_spacing > 0");
        if (!(s->box / s->pme_spacing <= 1024))
            FAIL(MD_EINVAL, "md_set_system: PME grid above 1024 points per edge");
    }
    if (s->n_rings < 0 || s->n_rings > MAX_RINGS)
        FAIL(MD_EINVAL, "md_set_system: n_rings must be in [0, %d]", MAX_RINGS);
    for (int y = 1; y < s->n_rings; ++y) {
        const double lo = y == 1 ? s->r_split - s->h_switch : s->ring_r[y - 2];
        if (!(s->ring_r[y - 1] > lo && s->ring_r[y - 1] < s->r_cut))
            FAIL(MD_EINVAL, "md_set_system: ring_r must increase strictly inside (r_split - h_switch, r_cut)");
    }
    const double skin_o = std::max(s->skin, s->skin_outer);
    if (!(s->box >= 2.0 * (s->r_cut + skin_o)))
        FAIL(MD_EINVAL, "md_set_system: box %.4f must be at least 2 (r_cut + skin_outer) = %.4f", s->box,
             2.0 * (s->r_cut + skin_o));
    for (int i = 0; i < s->n_atoms; ++i) {
        if (s->type[i] < 0 || s->type[i] >= s->n_types) FAIL(MD_EINVAL, "md_set_system: atom %d has type %d", i, s->type[i]);
        if (!(s->mass[i] > 0)) FAIL(MD_EINVAL, "md_set_system: atom %d has mass <= 0", i);
        for (int c = 0; c < 3; ++c)
            if (!std::isfinite(s->x[3 * i + c]) || !std::isfinite(s->v[3 * i + c]))
                FAIL(MD_EINVAL, "md_set_system: non-finite coordinate of atom %d", i);
    }
    auto idx_ok = [&](const int* a, int cnt, int per) {
        for (int k = 0; k < cnt * per; ++k)
            if (a[k] < 0 || a[k] >= s->n_atoms) return false;
        return true;
    };
    if ((s->n_bonds && (!s->bonds || !s->bond_k || !s->bond_r0 || !idx_ok(s->bonds, s->n_bonds, 2))) ||
        (s->n_angles && (!s->angles || !s->angle_k || !s->angle_t0 || !idx_ok(s->angles, s->n_angles, 3))) ||
        (s->n_excl && (!s->excl_pairs || !idx_ok(s->excl_pairs, s->n_excl, 2))))
        FAIL(MD_EINVAL, "md_set_system: bonded or exclusion indices out of range");
    return MD_OK;
}

// copy the device state of every replica back to its host record
int download_all(md_ctx* ctx)
{
    if (!ctx->on_device) return MD_OK;
    CK(cudaStreamSynchronize(ctx->s));
    const Dev& d = ctx->d;
    std::vector<long long> sb(d.R);
    std::vector<unsigned long long> cnt((size_t)d.R * NCOUNT);
    std::vector<uint32_t> err(d.R);
    CK(cudaMemcpy(sb.data(), d.step_base, sizeof(long long) * d.R, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(cnt.data(), d.cnt, sizeof(unsigned long long) * cnt.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(err.data(), d.err, sizeof(uint32_t) * d.R, cudaMemcpyDeviceToHost));
    for (int r = 0; r < (int)ctx->reps.size(); ++r) {
        RepHost& h = ctx->reps[r];
        if (!h.set || h.fresh || r >= d.R) continue;
        const size_t o = 3 * (size_t)ctx->rep_atom_off[r], n3 = 3 * (size_t)h.n;
        CK(cudaMemcpy(h.x.data(), d.x + o, n3 * sizeof(double), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(h.v.data(), d.v + o, n3 * sizeof(double), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(h.xb.data(), d.xb + o, n3 * sizeof(double), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(h.xo.data(), d.xo + o, n3 * sizeof(double), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(h.img.data(), d.img + o, n3 * sizeof(int), cudaMemcpyDeviceToHost));
        h.step = sb[r];
        h.cnt.assign(cnt.begin() + (size_t)r * NCOUNT, cnt.begin() + (size_t)(r + 1) * NCOUNT);
        h.err = err[r];
    }
    return MD_OK;
}

int read_max(md_ctx* ctx, const int* dev_counts, int n, int& mx)
{
    std::vector<int> c(n);
    CK(cudaMemcpyAsync(c.data(), dev_counts, sizeof(int) * n, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    mx = 0;
    for (int v : c) mx = std::max(mx, v);
    return MD_OK;
}

// cluster-tile lists kept with the lists (mixed mode): the short radius with
// the short kind, the full radius with the full kind
int tile_bits(const md_ctx* ctx, int kinds)
{
    if (ctx->fp64 || !ctx->d.ncl_cap) return 0;
    return ((kinds >> L_SHORT) & 1) | (((kinds >> L_FULL) & 1) << 1);
}

// estimated cluster pairs of one cluster within list radius t (J >= I and J < I
// alike, with room for clusters of a whole cell's extent)
int tile_cap(const md_ctx* ctx, int t)
{
    double rho = 0, rl = 0, cs = 0;
    for (const RepParams& P : ctx->hp) {
        rho = std::max(rho, P.n / (P.L * P.L * P.L));
        rl = std::max(rl, (t == 0 ? std::min(P.rc, P.R) : P.R) + P.skin);
        cs = std::max(cs, P.cs);
    }
    const double reach = rl + cs;
    const int c = int(4.0 / 3.0 * PI * reach * reach * reach * rho / TILE_CL) + 32;
    return (c + 31) / 32 * 32;
}

// grow list capacities that came close to or over their limit, then rebuild
int fit_caps(md_ctx* ctx, int kinds_to_check, bool outer)
{
    Dev& d = ctx->d;
    for (int round = 0; round < 4; ++round) {
        bool grow = false;
        int mx;
        if (outer) {
            int rc = read_max(ctx, d.ocnt, d.N, mx);
            if (rc) return rc;
            if (mx > d.ocap * 0.9) {
                const int cap = (int(mx * 1.4) + 64 + 31) / 32 * 32;
                uint32_t* p;
                if ((rc = dalloc(ctx, &p, (size_t)d.N * cap))) return rc;
                dfree(ctx, d.olist);
                d.olist = p; d.ocap = cap;
                grow = true;
            }
        }
        for (int k = 0; k < NKIND; ++k) {
            if (!(kinds_to_check & (1 << k))) continue;
            int rc = read_max(ctx, d.lcnt[k], d.N, mx);
            if (rc) return rc;
            if (mx > d.lcap[k] * 0.9) {
                const int cap = (int(mx * 1.4) + 64 + 31) / 32 * 32;
                uint32_t* p;
                if ((rc = dalloc(ctx, &p, (size_t)d.N * cap))) return rc;
                dfree(ctx, d.list[k]);
                d.list[k] = p; d.lcap[k] = cap;
                grow = true;
            }
        }
        bool tiles_grew = false;
        for (int t = 0; t < 2; ++t) {
            if (!((d.tiles >> t) & 1)) continue;
            int rc = read_max(ctx, d.cpl_n[t], d.ncl_cap, mx);
            if (rc) return rc;
            if (mx > d.cpl_cap[t] * 0.9) {
                const int cap = (int(mx * 1.4) + 32 + 31) / 32 * 32;
                int* pj;
                unsigned long long* pm;
                if ((rc = dalloc(ctx, &pj, (size_t)d.ncl_cap * cap)) ||
                    (rc = dalloc(ctx, &pm, (size_t)d.ncl_cap * cap)))
                    return rc;
                dfree(ctx, d.cpl_j[t]);
                dfree(ctx, d.cpl_mask[t]);
                d.cpl_j[t] = pj; d.cpl_mask[t] = pm; d.cpl_cap[t] = cap;
                grow = tiles_grew = true;
            }
        }
        if (!grow) return MD_OK;
        // rebuild at the stored build positions (exact, keeps the references)
        CK(cudaMemsetAsync(d.err, 0, sizeof(uint32_t) * d.R, ctx->s));
        if (outer) {
            launch_check(d, 1, 1, ctx->s);
            launch_rebuild(d, ctx->kinds & ~kinds_to_check, 1, 1, 1, 0, ctx->s);
        } else if (tiles_grew) {
            launch_tiles_late(d, d.tiles, ctx->s);
        }
        launch_late_lists(d, kinds_to_check, ctx->s);
        CK(cudaGetLastError());
    }
    FAIL(MD_EOVERFLOW, "neighbour-list capacity could not be fitted");
}

int commit(md_ctx* ctx)
{
    if (!ctx->dirty) return MD_OK;
    int R = 0;
    for (int r = 0; r < (int)ctx->reps.size(); ++r)
        if (ctx->reps[r].set) R = r + 1;
    if (R == 0) FAIL(MD_ENOSYSTEM, "no replica has a system");
    for (int r = 0; r < R; ++r)
        if (!ctx->reps[r].set) FAIL(MD_ENOSYSTEM, "replica %d has no system (replicas 0..%d must be set)", r, R - 1);
    int rc = download_all(ctx);
    if (rc) return rc;
    vacf_stop(ctx);
    free_device(ctx);
    // layout
    int N = 0, cells = 0;
    ctx->rep_atom_off.assign(R, 0);
    ctx->hp.assign(R, RepParams{});
    double rho = 0;
    for (int r = 0; r < R; ++r) {
        RepHost& h = ctx->reps[r];
        ctx->rep_atom_off[r] = N;
        ctx->hp[r] = make_params(ctx, h, r, N, cells);
        const RepParams& P = ctx->hp[r];
        cells += P.nc * P.nc * P.nc + 1;
        N += h.n;
        rho = std::max(rho, h.n / (h.box * h.box * h.box));
    }

    Dev& d = ctx->d;
    d = Dev{};
    d.N = N; d.R = R;
    // host arrays
    std::vector<double> x(3 * N), v(3 * N), xb(3 * N), xo(3 * N), mt(N), isqmt(N), nimt(N), q(N), LY(MAX_RINGS * N),
        LLJ(N);
    std::vector<float> LYf(MAX_RINGS * N), LLJf(N);
    std::vector<int> img(3 * N), type(N), rep(N), cell_rep(cells, -1);
    std::vector<int> bi_off(N + 1, 0), ex_off(N + 1, 0), ex_idx;
    std::vector<int2> bitem, bond_ij;
    std::vector<double> bond_k, bond_r0, ang_k, ang_t0;
    std::vector<int4> ang;
    std::vector<std::vector<int2>> items(N);
    std::vector<std::vector<int>> exl(N);
    double rmax_o = 0;
    for (int r = 0; r < R; ++r) {
        RepHost& h = ctx->reps[r];
        const RepParams& P = ctx->hp[r];
        const int o = P.atom_off;
        const int ncell = P.nc * P.nc * P.nc;
        for (int c = 0; c < ncell; ++c) cell_rep[P.cell_off + c] = r;
        std::memcpy(&x[3 * o], h.x.data(), sizeof(double) * 3 * h.n);
        std::memcpy(&v[3 * o], h.v.data(), sizeof(double) * 3 * h.n);
        std::memcpy(&xb[3 * o], h.xb.data(), sizeof(double) * 3 * h.n);
        std::memcpy(&xo[3 * o], h.xo.data(), sizeof(double) * 3 * h.n);
        std::memcpy(&img[3 * o], h.img.data(), sizeof(int) * 3 * h.n);
        make_bounds(h, P, &LY[MAX_RINGS * o], &LLJ[o]);
        for (int i = 0; i < h.n; ++i) {
            mt[o + i] = h.mass[i] / KCAL_AMU;
            isqmt[o + i] = 1.0 / std::sqrt(mt[o + i]);
            nimt[o + i] = -1.0 / mt[o + i];
            q[o + i] = h.charge[i];
            type[o + i] = h.type[i];
            rep[o + i] = r;
            for (int y = 0; y < MAX_RINGS; ++y) LYf[MAX_RINGS * (o + i) + y] = float(LY[MAX_RINGS * (o + i) + y]);
            LLJf[o + i] = float(LLJ[o + i]);
        }
        const int nb = (int)h.bond_k.size();
        for (int b = 0; b < nb; ++b) {
            const int t = (int)bond_ij.size();
            const int a0 = o + h.bonds[2 * b], a1 = o + h.bonds[2 * b + 1];
            bond_ij.push_back(make_int2(a0, a1));
            bond_k.push_back(h.bond_k[b]);
            bond_r0.push_back(h.bond_r0[b]);
            items[a0].push_back(make_int2(0 | (0 << 4), t));
            items[a1].push_back(make_int2(0 | (1 << 4), t));
        }
        const int na = (int)h.ang_k.size();
        for (int a = 0; a < na; ++a) {
            const int t = (int)ang.size();
            const int e0 = o + h.angles[3 * a], c = o + h.angles[3 * a + 1], e1 = o + h.angles[3 * a + 2];
            ang.push_back(make_int4(e0, c, e1, 0));
            ang_k.push_back(h.ang_k[a]);
            ang_t0.push_back(h.ang_t0[a]);
            items[e0].push_back(make_int2(1 | (0 << 4), t));
            items[c].push_back(make_int2(1 | (1 << 4), t));
            items[e1].push_back(make_int2(1 | (2 << 4), t));
        }
        const int ne = (int)h.excl.size() / 2;
        for (int e = 0; e < ne; ++e) {
            const int a0 = o + h.excl[2 * e], a1 = o + h.excl[2 * e + 1];
            exl[a0].push_back(a1);
            exl[a1].push_back(a0);
        }
        rmax_o = std::max(rmax_o, P.R + P.skin_o);
    }
    // visiting order of the velocity phases: by replica, then grouped by an
    // estimate of the proposal rate (per-pair bound at the thermal speed plus
    // the adaptive-eps floor), stable in index inside a group
    std::vector<int> vorder(N);
    {
        std::vector<double> est(N);
        for (int i = 0; i < N; ++i) {
            const RepParams& P = ctx->hp[rep[i]];
            const double vth = std::sqrt(3.0 / (P.beta * mt[i]));
            double ly = 0;
            for (int y = 0; y < MAX_RINGS; ++y) ly += LY[MAX_RINGS * i + y];
            est[i] = ly * P.beta * vth + 2.0 * std::sqrt(P.beta / mt[i]) / P.eps0 + LLJ[i];
            vorder[i] = i;
        }
        std::stable_sort(vorder.begin(), vorder.end(), [&](int x, int y) {
            return rep[x] != rep[y] ? rep[x] < rep[y] : est[x] > est[y];
        });
    }
    // blocks of whole bonded groups (connected by bonds and angles) for the
    // fused inner steps: each group must be a contiguous index range of at
    // most IB_MAX atoms; groups are packed in index order
    std::vector<int> ib_start;
    {
        std::vector<int> root(N);
        for (int i = 0; i < N; ++i) root[i] = i;
        auto find = [&](int a) {
            while (root[a] != a) { root[a] = root[root[a]]; a = root[a]; }
            return a;
        };
        auto unite = [&](int a, int b) {
            a = find(a); b = find(b);
            if (a != b) root[std::max(a, b)] = std::min(a, b);
        };
        for (const int2& bij : bond_ij) unite(bij.x, bij.y);
        for (const int4& an : ang) { unite(an.x, an.y); unite(an.z, an.y); }
        bool ok = true;
        int start = 0;
        ib_start.push_back(0);
        for (int i = 0; i < N && ok;) {
            // group of i: the contiguous run of atoms with the same root
            const int g = find(i);
            int j = i + 1;
            while (j < N && find(j) == g) ++j;
            if (g != i || j - i > IB_MAX) ok = false;          // a group must start its run and fit a block
            if (j - start > IB_MAX) { ib_start.push_back(i); start = i; }
            i = j;
        }
        // a group that reappears after another one is not contiguous
        if (ok) {
            std::vector<int> last(N, -1);
            for (int i = 0; i < N && ok; ++i) {
                const int g = find(i);
                if (last[g] >= 0 && last[g] != i - 1) ok = false;
                last[g] = i;
            }
        }
        ib_start.push_back(N);
        if (!ok) ib_start.clear();
    }
    // the terms of each block, and the slot of every item's term in its block's list
    std::vector<int> ib_bond_off, ib_bond, ib_ang_off, ib_ang, item_slot;
    if (!ib_start.empty()) {
        const int nb = (int)ib_start.size() - 1;
        std::vector<int> blk(N);
        for (int b = 0; b < nb; ++b)
            for (int i = ib_start[b]; i < ib_start[b + 1]; ++i) blk[i] = b;
        std::vector<std::vector<int>> bl(nb), al(nb);
        std::vector<int> bslot(bond_ij.size()), aslot(ang.size());
        for (int t = 0; t < (int)bond_ij.size(); ++t) {
            const int b = blk[bond_ij[t].x];
            bslot[t] = (int)bl[b].size();
            bl[b].push_back(t);
        }
        for (int t = 0; t < (int)ang.size(); ++t) {
            const int b = blk[ang[t].y];
            aslot[t] = (int)al[b].size();
            al[b].push_back(t);
        }
        bool fit = true;
        ib_bond_off.push_back(0);
        ib_ang_off.push_back(0);
        for (int b = 0; b < nb; ++b) {
            fit = fit && (int)bl[b].size() <= IB_TERMS && (int)al[b].size() <= IB_TERMS;
            ib_bond.insert(ib_bond.end(), bl[b].begin(), bl[b].end());
            ib_ang.insert(ib_ang.end(), al[b].begin(), al[b].end());
            ib_bond_off.push_back((int)ib_bond.size());
            ib_ang_off.push_back((int)ib_ang.size());
        }
        for (int i = 0; i < N; ++i)
            for (const int2& it : items[i]) item_slot.push_back((it.x & 15) == 0 ? bslot[it.y] : aslot[it.y]);
        if (!fit) ib_start.clear();
    }
    for (int i = 0; i < N; ++i) {
        bi_off[i + 1] = bi_off[i] + (int)items[i].size();
        for (auto& it : items[i]) bitem.push_back(it);
        ex_off[i + 1] = ex_off[i] + (int)exl[i].size();
        for (int j : exl[i]) ex_idx.push_back(j);
    }
    // device arrays
    RepParams* dP;
    int *drep, *dvorder, *dvorder0, *dtype, *dimg, *dbi_off, *dex_off, *dex_idx;
    double *dmt, *disqmt, *dq, *dLY, *dLLJ, *dbk, *dbr0, *dak, *dat0;
    float *dLYf, *dLLJf;
    int2 *dbitem, *dbij;
    int4* dang;
#define AL(p, n) if ((rc = dalloc(ctx, &(p), (n)))) return rc
    AL(dP, R); AL(drep, N); AL(dvorder, N); AL(dvorder0, N); AL(dtype, N); AL(dimg, 3 * N); AL(dbi_off, N + 1);
    AL(dex_off, N + 1); AL(dex_idx, ex_idx.size());
    AL(dmt, N); AL(disqmt, N); AL(dq, N); AL(dLY, MAX_RINGS * N); AL(dLLJ, N);
    {
        double* dnimt;
        AL(dnimt, N);
        if ((rc = upload(ctx, dnimt, nimt.data(), N))) return rc;
        d.nimt = dnimt;
    }
    AL(dLYf, MAX_RINGS * N); AL(dLLJf, N);
    AL(dbitem, bitem.size()); AL(dbij, bond_ij.size()); AL(dbk, bond_k.size()); AL(dbr0, bond_r0.size());
    AL(dang, ang.size()); AL(dak, ang_k.size()); AL(dat0, ang_t0.size());
    AL(d.bterm, 3 * bond_k.size()); AL(d.aterm, 6 * ang_k.size());
    d.nbond = (int)bond_k.size();
    d.nang = (int)ang_k.size();
    AL(d.x, 3 * N); AL(d.v, 3 * N); AL(d.xb, 3 * N); AL(d.xo, 3 * N);
    AL(d.a0, 3 * N); AL(d.ab, 3 * N); AL(d.as, 3 * N); AL(d.al, 3 * N); AL(d.gout, 3 * N);
    AL(d.pos, N);
    AL(d.cell_start, cells + 1); AL(d.cell_cnt, cells + 1); AL(d.cell_atoms, N); AL(d.atom_cell, N);
    AL(d.cell_rep, cells);
    d.total_cells = cells;
    d.ocap = cap_of(rho, 0, rmax_o);
    AL(d.olist, (size_t)N * d.ocap); AL(d.ocnt, N);
    for (int k = 0; k < NKIND; ++k) {
        d.lcap[k] = (ctx->kinds & (1 << k)) ? kind_cap(ctx, k) : 32;
        AL(d.list[k], (size_t)N * d.lcap[k]);
        AL(d.lcnt[k], N);
    }
    AL(d.flags, 2 * R); AL(d.err, R); AL(d.ovf, R); AL(d.cnt, (size_t)R * NCOUNT); AL(d.energy, 6 * R);
    AL(d.step_base, R); AL(d.stepc, 2 * R);
    AL(d.vkey, N); AL(d.vhist, (size_t)R * RATE_BUCKETS); AL(d.vofs, (size_t)R * RATE_BUCKETS); AL(d.qctr, 1);
    AL(d.facc, 3 * (size_t)N);
    d.ncl_cap = 0;
    d.tiles = 0;
    // the box test of a cluster pair takes the minimum image of the two
    // clusters' reference atoms; every member pair then shares it only when
    // half the box exceeds the list radius plus the clusters' extent (a cell,
    // widened by the outer skin, corner to corner); smaller boxes keep the
    // per-atom kernels
    // (opt-in: MDJ_TILES set; on 96,000-atom water they measured 2-2.5 times
    // slower than the per-atom half-list kernels, see k_force_tile)
    bool tiles_fit = !ctx->fp64 && std::getenv("MDJ_TILES") != nullptr;
    for (const RepParams& P : ctx->hp)
        tiles_fit = tiles_fit && 0.5 * P.L > P.R + P.skin + std::sqrt(3.0) * (P.cs + P.skin_o);
    if (tiles_fit) {
        // cluster tiles: replica r owns ceil(n_r / TILE_CL) + (its cells) clusters,
        // enough for ceil(n_c / TILE_CL) in each of its cells
        std::vector<int> roff(R + 1, 0);
        for (int r = 0; r < R; ++r) {
            const RepParams& P = ctx->hp[r];
            roff[r + 1] = roff[r] + (P.n + TILE_CL - 1) / TILE_CL + P.nc * P.nc * P.nc;
        }
        d.ncl_cap = roff[R];
        int* droff;
        AL(droff, R + 1);
        if ((rc = upload(ctx, droff, roff.data(), R + 1))) return rc;
        d.cl_roff = droff;
        AL(d.cl_start, cells); AL(d.cl_atom, (size_t)TILE_CL * d.ncl_cap); AL(d.cl_of, N); AL(d.cl_slot, N);
        AL(d.cl_cell, d.ncl_cap); AL(d.cl_ref, d.ncl_cap); AL(d.cl_lo, d.ncl_cap); AL(d.cl_hi, d.ncl_cap);
        CK(cudaMemsetAsync(d.cl_cell, 0xff, sizeof(int) * (size_t)d.ncl_cap, ctx->s));
        for (int t = 0; t < 2; ++t) {
            d.cpl_cap[t] = tile_cap(ctx, t);
            AL(d.cpl_j[t], (size_t)d.ncl_cap * d.cpl_cap[t]);
            AL(d.cpl_mask[t], (size_t)d.ncl_cap * d.cpl_cap[t]);
            AL(d.cpl_n[t], d.ncl_cap);
            CK(cudaMemsetAsync(d.cpl_n[t], 0, sizeof(int) * (size_t)d.ncl_cap, ctx->s));
        }
        d.tiles = tile_bits(ctx, ctx->kinds);
    }
    {
        int *dib, *dbo, *dbl, *dao, *dal, *dsl;
        const bool on = !ib_start.empty();
        AL(dib, std::max<size_t>(ib_start.size(), 1)); AL(dbo, std::max<size_t>(ib_bond_off.size(), 1));
        AL(dbl, std::max<size_t>(ib_bond.size(), 1)); AL(dao, std::max<size_t>(ib_ang_off.size(), 1));
        AL(dal, std::max<size_t>(ib_ang.size(), 1)); AL(dsl, std::max<size_t>(item_slot.size(), 1));
        if (on && ((rc = upload(ctx, dib, ib_start.data(), ib_start.size())) ||
                   (rc = upload(ctx, dbo, ib_bond_off.data(), ib_bond_off.size())) ||
                   (rc = upload(ctx, dbl, ib_bond.data(), ib_bond.size())) ||
                   (rc = upload(ctx, dao, ib_ang_off.data(), ib_ang_off.size())) ||
                   (rc = upload(ctx, dal, ib_ang.data(), ib_ang.size())) ||
                   (rc = upload(ctx, dsl, item_slot.data(), item_slot.size()))))
            return rc;
        d.ib_start = dib; d.ib_bond_off = dbo; d.ib_bond = dbl; d.ib_ang_off = dao; d.ib_ang = dal; d.item_slot = dsl;
        d.n_ib = on ? (int)ib_start.size() - 1 : 0;
    }
    {
        // atoms with an LJ partner type first, the others after (each in index
        // order): the launches of the (1 - chi) LJ part alone run over this order,
        // so their warps hold LJ atoms only
        std::vector<int> perm;
        perm.reserve(N);
        for (int pass = 0; pass < 2; ++pass)
            for (int r = 0; r < R; ++r) {
                const RepHost& h = ctx->reps[r];
                const int o = ctx->hp[r].atom_off;
                for (int i = 0; i < h.n; ++i) {
                    bool lj = false;
                    for (int b = 0; b < h.ntypes; ++b) lj |= h.lj_eps[h.type[i] * h.ntypes + b] != 0.0;
                    if (lj == (pass == 0)) perm.push_back(o + i);
                }
            }
        int* dperm;
        AL(dperm, N);
        if ((rc = upload(ctx, dperm, perm.data(), N))) return rc;
        d.lj_perm = dperm;
    }
    d.lj_long_mask = 0;
    d.lj_symmetric = 1;
    for (int r = 0; r < R; ++r) {
        const RepHost& h = ctx->reps[r];
        if (h.sys.lj_long_mode == 1) d.lj_long_mask |= 1;
        if (h.sys.lj_long_mode == 2) d.lj_long_mask |= 2;
        for (int a = 0; a < h.ntypes; ++a)
            for (int b = 0; b < h.ntypes; ++b)
                if (h.lj_eps[a * h.ntypes + b] != h.lj_eps[b * h.ntypes + a] ||
                    h.lj_sig[a * h.ntypes + b] != h.lj_sig[b * h.ntypes + a])
                    d.lj_symmetric = 0;
    }
    // smooth PME grids of the Ewald replicas, each part starting on a 512-byte boundary
    ctx->ewald_reps.clear();
    ctx->pme_orders.clear();
    long long gtot = 0, stot = 0;
    int nbricks = 0;
    ctx->pme_max_spec = 0;
    for (int r = 0; r < R; ++r) {
        RepParams& P = ctx->hp[r];
        if (P.coul_mode != 1) continue;
        const long long K = P.pme_K;
        P.pme_goff = gtot;
        P.pme_soff = stot;
        P.pme_nb = (P.pme_K + PME_BRICK - 1) / PME_BRICK;
        P.pme_boff = nbricks;
        nbricks += P.pme_nb * P.pme_nb * P.pme_nb;
        gtot += (K * K * K + 63) / 64 * 64;
        stot += (K * K * (K / 2 + 1) + 31) / 32 * 32;
        ctx->ewald_reps.push_back(r);
        ctx->pme_max_spec = std::max(ctx->pme_max_spec, K * K * (K / 2 + 1));
        if (std::find(ctx->pme_orders.begin(), ctx->pme_orders.end(), P.pme_p) == ctx->pme_orders.end())
            ctx->pme_orders.push_back(P.pme_p);
    }
    ctx->pme_total = gtot;
    if (!ctx->ewald_reps.empty()) {
        AL(ctx->arecip, 3 * (size_t)N);
        if (!ctx->s2) {
            // the higher priority lets its blocks in as soon as the main stream's free an SM
            int lo = 0, hi = 0;
            CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            CK(cudaStreamCreateWithPriority(&ctx->s2, cudaStreamNonBlocking, hi));
        }
        if (!ctx->ev_fork) CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
        if (!ctx->ev_join) CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    }
    {
        double* dG;
        float* dGf;
        int* dbrep;
        AL(d.pme_qi, gtot); AL(d.pme_q, gtot); AL(d.pme_spec, stot); AL(dG, stot); AL(dGf, stot); AL(d.pme_e, R);
        AL(d.pme_brick, N); AL(d.pme_slot, N); AL(d.pme_sorted, N);
        AL(d.pme_bcnt, nbricks); AL(d.pme_bstart, nbricks + 1); AL(dbrep, nbricks);
        d.pme_G = dG;
        d.pme_Gf = dGf;
        d.pme_brick_rep = dbrep;
        d.pme_nbricks = nbricks;
        if (nbricks) {
            std::vector<int> brep(nbricks);
            for (int r : ctx->ewald_reps) {
                const RepParams& P = ctx->hp[r];
                for (int b = 0; b < P.pme_nb * P.pme_nb * P.pme_nb; ++b) brep[P.pme_boff + b] = r;
            }
            if ((rc = upload(ctx, dbrep, brep.data(), brep.size()))) return rc;
            CK(cudaMemsetAsync(d.pme_bcnt, 0, sizeof(int) * nbricks, ctx->s));
        }
        if (gtot) {
            std::vector<double> G(stot, 0.0);
            for (int r : ctx->ewald_reps) make_pme_G(ctx->hp[r], &G[ctx->hp[r].pme_soff]);
            std::vector<float> Gf(G.begin(), G.end());
            if ((rc = upload(ctx, dG, G.data(), G.size())) || (rc = upload(ctx, dGf, Gf.data(), Gf.size()))) return rc;
            CK(cudaMemsetAsync(d.pme_qi, 0, sizeof(unsigned long long) * gtot, ctx->s));
        }
        for (int r : ctx->ewald_reps) {
            const int K = ctx->hp[r].pme_K;
            bool have = false;
            for (auto& f : ctx->fft) have |= f.K == K;
            if (have) continue;
            // FP64 transforms in FP64 mode, FP32 in mixed mode
            md_ctx::FftPlan f{K, 0, 0};
            const cufftType fw = ctx->fp64 ? CUFFT_D2Z : CUFFT_R2C, bw = ctx->fp64 ? CUFFT_Z2D : CUFFT_C2R;
            if (cufftPlan3d(&f.d2z, K, K, K, fw) != CUFFT_SUCCESS) FAIL(MD_ECUDA, "cufftPlan3d (forward, K = %d) failed", K);
            if (cufftPlan3d(&f.z2d, K, K, K, bw) != CUFFT_SUCCESS) {
                cufftDestroy(f.d2z);
                FAIL(MD_ECUDA, "cufftPlan3d (inverse, K = %d) failed", K);
            }
            ctx->fft.push_back(f);
        }
    }
    uint16_t* dtab;
    AL(dtab, (size_t)R * SHELL_BINS);
    d.shell_tab = dtab;
    std::vector<uint16_t> tab((size_t)R * SHELL_BINS);
    for (int r = 0; r < R; ++r) make_shell_table(ctx->hp[r], &tab[(size_t)r * SHELL_BINS]);
    if ((rc = upload(ctx, dtab, tab.data(), tab.size()))) return rc;
    const long long evcap = ctx->cfg.event_log_cap > 0 ? ctx->cfg.event_log_cap : 0;
    AL(d.ev, (size_t)6 * (evcap ? evcap : 1)); AL(d.ev_n, 1);
#undef AL
    d.ev_cap = evcap;
    d.P = dP; d.rep = drep; d.vorder = dvorder; d.vorder0 = dvorder0; d.type = dtype; d.img = dimg; d.bi_off = dbi_off; d.ex_off = dex_off;
    d.ex_idx = dex_idx; d.mt = dmt; d.isqmt = disqmt; d.q = dq; d.LY = dLY; d.LLJ = dLLJ;
    d.LYf = dLYf; d.LLJf = dLLJf; d.bitem = dbitem; d.bond_ij = dbij; d.bond_k = dbk;
    d.bond_r0 = dbr0; d.ang = dang; d.ang_k = dak; d.ang_t0 = dat0;
    if ((rc = upload(ctx, dP, ctx->hp.data(), R)) || (rc = upload(ctx, drep, rep.data(), N)) ||
        (rc = upload(ctx, dvorder, vorder.data(), N)) || (rc = upload(ctx, dvorder0, vorder.data(), N)) ||
        (rc = upload(ctx, dtype, type.data(), N)) || (rc = upload(ctx, dimg, img.data(), 3 * (size_t)N)) ||
        (rc = upload(ctx, dbi_off, bi_off.data(), N + 1)) || (rc = upload(ctx, dex_off, ex_off.data(), N + 1)) ||
        (rc = upload(ctx, dex_idx, ex_idx.data(), ex_idx.size())) || (rc = upload(ctx, dmt, mt.data(), N)) ||
        (rc = upload(ctx, disqmt, isqmt.data(), N)) || (rc = upload(ctx, dq, q.data(), N)) ||
        (rc = upload(ctx, dLY, LY.data(), (size_t)MAX_RINGS * N)) || (rc = upload(ctx, dLLJ, LLJ.data(), N)) ||
        (rc = upload(ctx, dLYf, LYf.data(), (size_t)MAX_RINGS * N)) || (rc = upload(ctx, dLLJf, LLJf.data(), N)) ||
        (rc = upload(ctx, dbitem, bitem.data(), bitem.size())) ||
        (rc = upload(ctx, dbij, bond_ij.data(), bond_ij.size())) ||
        (rc = upload(ctx, dbk, bond_k.data(), bond_k.size())) ||
        (rc = upload(ctx, dbr0, bond_r0.data(), bond_r0.size())) ||
        (rc = upload(ctx, dang, ang.data(), ang.size())) || (rc = upload(ctx, dak, ang_k.data(), ang_k.size())) ||
        (rc = upload(ctx, dat0, ang_t0.data(), ang_t0.size())) || (rc = upload(ctx, d.x, x.data(), 3 * (size_t)N)) ||
        (rc = upload(ctx, d.v, v.data(), 3 * (size_t)N)) || (rc = upload(ctx, d.xb, xb.data(), 3 * (size_t)N)) ||
        (rc = upload(ctx, d.xo, xo.data(), 3 * (size_t)N)) || (rc = upload(ctx, d.cell_rep, cell_rep.data(), cells)))
        return rc;
    CK(cudaMemsetAsync(d.cell_cnt, 0, sizeof(int) * (cells + 1), ctx->s));
    CK(cudaMemsetAsync(d.flags, 0, sizeof(int) * 2 * R, ctx->s));
    CK(cudaMemsetAsync(d.ev_n, 0, sizeof(unsigned long long), ctx->s));
    CK(cudaMemsetAsync(d.a0, 0, sizeof(double) * 3 * N, ctx->s));
    CK(cudaMemsetAsync(d.ab, 0, sizeof(double) * 3 * N, ctx->s));
    CK(cudaMemsetAsync(d.as, 0, sizeof(double) * 3 * N, ctx->s));
    CK(cudaMemsetAsync(d.al, 0, sizeof(double) * 3 * N, ctx->s));
    CK(cudaMemsetAsync(d.err, 0, sizeof(uint32_t) * R, ctx->s));
    CK(cudaMemsetAsync(d.ovf, 0, sizeof(uint32_t) * R, ctx->s));
    CK(cudaMemsetAsync(d.vhist, 0, sizeof(int) * R * RATE_BUCKETS, ctx->s));
    CK(cudaMemsetAsync(d.facc, 0, sizeof(long long) * 3 * (size_t)N, ctx->s));
    ctx->on_device = true;
    // initial build at the stored reference positions
    launch_check(d, 1, 1, ctx->s);
    launch_rebuild(d, ctx->kinds, 1, 1, 1, 0, ctx->s);
    CK(cudaGetLastError());
    if ((rc = fit_caps(ctx, ctx->kinds, true))) return rc;
    // restore per-replica counters, errors and step counters
    std::vector<long long> sb(R);
    std::vector<unsigned long long> cnt((size_t)R * NCOUNT, 0);
    std::vector<uint32_t> err(R, 0);
    for (int r = 0; r < R; ++r) {
        RepHost& h = ctx->reps[r];
        sb[r] = h.step;
        if (!h.fresh && (int)h.cnt.size() == NCOUNT)
            std::copy(h.cnt.begin(), h.cnt.end(), cnt.begin() + (size_t)r * NCOUNT);
        err[r] = h.fresh ? 0 : h.err;
        h.fresh = false;
    }
    if ((rc = upload(ctx, d.step_base, sb.data(), R)) || (rc = upload(ctx, d.cnt, cnt.data(), cnt.size())) ||
        (rc = upload(ctx, d.err, err.data(), R)))
        return rc;
    CK(cudaStreamSynchronize(ctx->s));
    ctx->dirty = false;
    return MD_OK;
}

int ensure_kinds(md_ctx* ctx, int mask)
{
    const int add = mask & ~ctx->kinds;
    if (!add) return MD_OK;
    Dev& d = ctx->d;
    // capacities for the new kinds
    int rc;
    for (int k = 0; k < NKIND; ++k) {
        if (!(add & (1 << k))) continue;
        uint32_t* p;
        if ((rc = dalloc(ctx, &p, (size_t)d.N * kind_cap(ctx, k)))) return rc;
        dfree(ctx, d.list[k]);
        d.list[k] = p;
        d.lcap[k] = kind_cap(ctx, k);
    }
    launch_late_lists(d, add, ctx->s);
    const int tnew = tile_bits(ctx, ctx->kinds | add) & ~d.tiles;
    if (tnew) launch_tiles_late(d, tnew, ctx->s);
    d.tiles |= tnew;
    CK(cudaGetLastError());
    if ((rc = fit_caps(ctx, add, false))) return rc;
    ctx->kinds |= add;
    return MD_OK;
}

cudaEvent_t take_event(md_ctx* ctx)
{
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// scope of one launch group: counts its kernels, times it when profiling
struct Prof {
    md_ctx* ctx;
    int cls;
    cudaEvent_t a = nullptr;
    Prof(md_ctx* c, int k, int nkernels) : ctx(c), cls(k)
    {
        ctx->nlaunch[k] += nkernels;
        if (ctx->prof) {
            a = take_event(ctx);
            cudaEventRecord(a, ctx->s);
        }
    }
    ~Prof()
    {
        if (a) {
            cudaEvent_t b = take_event(ctx);
            cudaEventRecord(b, ctx->s);
            ctx->pend.push_back({cls, a, b});
        }
    }
};

void collect_profile(md_ctx* ctx)
{
    for (auto& p : ctx->pend) {
        float ms = 0;
        cudaEventElapsedTime(&ms, p.a, p.b);
        ctx->prof_ms[p.cls] += ms;
        ctx->prof_groups[p.cls] += 1;
        ctx->ev_pool.push_back(p.a);
        ctx->ev_pool.push_back(p.b);
    }
    ctx->pend.clear();
}

// can gradient mode `mode` run on the cluster tiles? (mixed mode, a half-list
// mode whose tile list is kept)
bool tile_ok(const md_ctx* ctx, int mode)
{
    if (ctx->fp64 || !force_half_ok(ctx->d, mode)) return false;
    const int tl = (mode == 3 || mode == 5) ? 0 : (mode == 0 || mode == 2 || mode == 4) ? 1 : -1;
    return tl >= 0 && ((ctx->d.tiles >> tl) & 1);
}

int tpa_for(md_ctx* ctx, int mode)
{
    if (ctx->fp64) return 1;
    if (ctx->tpa_cfg > 0) return ctx->tpa_cfg;
    if (ctx->tpa[mode]) return ctx->tpa[mode];
    if (const char* env = std::getenv("MDJ_FORCE_VARIANT")) {
        // a fixed kernel choice (tests): threads per atom, | 16 for the half-list kernels
        int t = std::atoi(env);
        if (!force_half_ok(ctx->d, mode)) t &= ~(FORCE_HALF | FORCE_TILE);
        if (!tile_ok(ctx, mode)) t &= ~FORCE_TILE;
        const int w = t & ~(FORCE_HALF | FORCE_TILE);
        ctx->tpa[mode] = (w == 1 || w == 2 || w == 4 || w == 8) ? t : 1;
        return ctx->tpa[mode];
    }
    // autotune: time each width, with the full and (where allowed) the
    // half-list kernels, on the current lists (results do not depend on it)
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int pick = 1;
    std::vector<int> cands = {1, 2, 4, 8};
    if (force_half_ok(ctx->d, mode))
        for (int t : {1, 2, 4, 8}) cands.push_back(t | FORCE_HALF);
    if (tile_ok(ctx, mode)) cands.push_back(1 | FORCE_TILE);
    for (int t : cands) {
        launch_force(ctx->d, mode, ctx->d.gout, 1, 0, t, ctx->s);
        cudaEventRecord(e0, ctx->s);
        for (int k = 0; k < 5; ++k) launch_force(ctx->d, mode, ctx->d.gout, 1, 0, t, ctx->s);
        cudaEventRecord(e1, ctx->s);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ctx->tune_log) std::fprintf(stderr, "mdjump tune:   mode %d variant %d: %.4f ms\n", mode, t, ms);
        if (ms < best) { best = ms; pick = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tpa[mode] = pick;
    if (ctx->tune_log)
        std::fprintf(stderr, "mdjump tune: gradient mode %d: %s%d threads per atom%s (%.4f ms for 5 evaluations)\n",
                     mode, (pick & FORCE_TILE) ? "cluster tiles, " : "", pick & ~(FORCE_HALF | FORCE_TILE),
                     (pick & FORCE_HALF) ? ", half list" : "", best);
    return pick;
}

// does gradient mode `mode` carry the Ewald reciprocal part in some replica?
bool mode_has_recip(const md_ctx* ctx, int mode)
{
    return !ctx->ewald_reps.empty() && (mode == 0 || mode == 2 || mode == 4 || mode == 5 || mode == 6);
}

const md_ctx::FftPlan* fft_plan(const md_ctx* ctx, int K)
{
    for (const auto& f : ctx->fft)
        if (f.K == K) return &f;
    return nullptr;
}

// smooth PME on every Ewald replica: with out, the gradient (added to out, as
// -grad / m~ unless as_grad); with energy, the reciprocal energies into d.pme_e
int pme(md_ctx* ctx, double* out, int as_grad, int energy, cudaStream_t st = nullptr)
{
    Dev& d = ctx->d;
    const cudaStream_t S = st ? st : ctx->s;
    const int no = (int)ctx->pme_orders.size();
    Prof p(ctx, 6, 5 + no + (out ? no : 0));
    launch_pme_bin(d, ctx->fp64, S);
    for (int order : ctx->pme_orders) launch_pme_spread(d, order, ctx->fp64, S);
    launch_pme_tofloat(d, ctx->pme_total, ctx->fp64, S);
    // the FP32 grids of mixed mode live in the same buffers, at the same element offsets
    float* qf = reinterpret_cast<float*>(d.pme_q);
    cufftComplex* sf = reinterpret_cast<cufftComplex*>(d.pme_spec);
    for (int r : ctx->ewald_reps) {
        const RepParams& P = ctx->hp[r];
        const md_ctx::FftPlan* f = fft_plan(ctx, P.pme_K);
        const cufftResult e = cufftSetStream(f->d2z, S) != CUFFT_SUCCESS ? CUFFT_INTERNAL_ERROR
            : ctx->fp64 ? cufftExecD2Z(f->d2z, d.pme_q + P.pme_goff, (cufftDoubleComplex*)(d.pme_spec + P.pme_soff))
                        : cufftExecR2C(f->d2z, qf + P.pme_goff, sf + P.pme_soff);
        if (e != CUFFT_SUCCESS) FAIL(MD_ECUDA, "cuFFT forward transform failed (%d)", (int)e);
    }
    launch_pme_convolve_grid(d, energy, ctx->pme_max_spec, ctx->fp64, S);
    if (!out) return MD_OK;
    for (int r : ctx->ewald_reps) {
        const RepParams& P = ctx->hp[r];
        const md_ctx::FftPlan* f = fft_plan(ctx, P.pme_K);
        const cufftResult e = cufftSetStream(f->z2d, S) != CUFFT_SUCCESS ? CUFFT_INTERNAL_ERROR
            : ctx->fp64 ? cufftExecZ2D(f->z2d, (cufftDoubleComplex*)(d.pme_spec + P.pme_soff), d.pme_q + P.pme_goff)
                        : cufftExecC2R(f->z2d, sf + P.pme_soff, qf + P.pme_goff);
        if (e != CUFFT_SUCCESS) FAIL(MD_ECUDA, "cuFFT inverse transform failed (%d)", (int)e);
    }
    for (int order : ctx->pme_orders) launch_pme_gather(d, order, out, as_grad, ctx->fp64, S);
    return MD_OK;
}

// gradient mode into out (as -grad / m~ unless as_grad); mode 6 = the reciprocal part alone
void force_into(md_ctx* ctx, int mode, double* out, int as_grad, bool with_recip = true)
{
    if (mode == 6) {
        // the slow level: the (1 - chi) LJ part of lj_long_mode 2 replicas (zero elsewhere), then PME
        if (any_lj_slow(ctx)) {
            const int t = tpa_for(ctx, 7);
            const bool half = !ctx->fp64 && (t & FORCE_HALF) && force_half_ok(ctx->d, 7);
            Prof p(ctx, 0, half ? 2 : 1);
            launch_force(ctx->d, 7, out, as_grad, ctx->fp64, t, ctx->s);
        } else {
            cudaMemsetAsync(out, 0, sizeof(double) * 3 * (size_t)ctx->d.N, ctx->s);
        }
    } else {
        const int t = mode == 1 ? 1 : tpa_for(ctx, mode);
        const bool bonded = mode == 0 || mode == 1 || mode == 5;
        const bool half = !ctx->fp64 && (t & FORCE_HALF) && force_half_ok(ctx->d, mode);
        Prof p(ctx, mode == 1 ? 1 : 0, ((bonded && ctx->d.nbond + ctx->d.nang > 0) ? 2 : 1) + (half ? 1 : 0));
        launch_force(ctx->d, mode, out, as_grad, ctx->fp64, t, ctx->s);
    }
    if (with_recip && mode_has_recip(ctx, mode)) {
        const int rc = pme(ctx, out, as_grad, 0);
        if (rc && !ctx->deferred) ctx->deferred = rc;
    }
}

void force(md_ctx* ctx, int mode, double* out) { force_into(ctx, mode, out, 0); }

// The slow level of the multiple-time-step drivers with a reciprocal part:
// the pair part goes to `al`, the reciprocal part to ctx->arecip, and the slow
// kick adds both. recip_begin starts the reciprocal sum at the current
// positions; unless per-class times are being taken, it runs on the second
// stream, overlapping what the main stream runs meanwhile (the velocity phase
// and the slow pair part; it reads only positions and its own grids). recip_end joins it back before its result is used. The
// arithmetic is the same either way.
void recip_begin(md_ctx* ctx)
{
    if (ctx->ewald_reps.empty()) return;
    const bool side = !ctx->prof && ctx->s2;
    const cudaStream_t st = side ? ctx->s2 : ctx->s;
    if (side) {
        cudaEventRecord(ctx->ev_fork, ctx->s);
        cudaStreamWaitEvent(ctx->s2, ctx->ev_fork, 0);
    }
    cudaMemsetAsync(ctx->arecip, 0, sizeof(double) * 3 * (size_t)ctx->d.N, st);
    const int rc = pme(ctx, ctx->arecip, 0, 0, st);
    if (rc && !ctx->deferred) ctx->deferred = rc;
    if (side) {
        cudaEventRecord(ctx->ev_join, ctx->s2);
        ctx->recip_open = true;
    }
}

void recip_end(md_ctx* ctx)
{
    if (!ctx->recip_open) return;
    cudaStreamWaitEvent(ctx->s, ctx->ev_join, 0);
    ctx->recip_open = false;
}

// the slow kick: the pair part, plus the reciprocal part when there is one
void slow_kick(md_ctx* ctx, double h)
{
    Prof p(ctx, 3, 1);
    if (ctx->ewald_reps.empty()) launch_kick(ctx->d, ctx->d.al, h, ctx->s);
    else launch_kick2(ctx->d, ctx->d.al, h, ctx->arecip, h, ctx->s);
}

// the error a driver body left behind (its message is already in ctx->msg)
int take_deferred(md_ctx* ctx)
{
    const int rc = ctx->deferred;
    ctx->deferred = MD_OK;
    return rc;
}

void rebuild_step(md_ctx* ctx)
{
    {
        Prof p(ctx, 4, 5);
        launch_rebuild_cells(ctx->d, 0, ctx->fp64, ctx->s);
    }
    if (ctx->kinds) {
        Prof p(ctx, 7, 1);
        launch_rebuild_inner(ctx->d, ctx->kinds, ctx->fp64, ctx->s);
    }
    if (ctx->d.tiles) {
        Prof p(ctx, 7, 3 + __builtin_popcount(ctx->d.tiles));
        launch_tiles(ctx->d, ctx->d.tiles, ctx->s);
    }
    Prof p(ctx, 4, 1);
    launch_rebuild_done(ctx->d, ctx->s);
}

void kick(md_ctx* ctx, const double* a, double h)
{
    Prof p(ctx, 3, 1);
    launch_kick(ctx->d, a, h, ctx->s);
}

void aoa(md_ctx* ctx, double tau, uint32_t s_off, int check)
{
    Prof p(ctx, 3, 1);
    launch_aoa(ctx->d, tau, s_off, check, ctx->fp64, ctx->s);
}

// parameters of the only replica, for launches that pass them by value
const RepParams* single_params(const md_ctx* ctx)
{
    return ctx->d.R == 1 ? &ctx->hp[0] : nullptr;
}

// autotune the velocity-phase kernel variant on a saved copy of the state:
// velocities, counters, event log and error flags are restored afterwards, so
// tuning leaves no trace in the trajectory
int tune_vphase(md_ctx* ctx, const double* a, double tau2)
{
    if (ctx->fp64 || ctx->vvar >= 0) return MD_OK;
    Dev& d = ctx->d;
    const char* env = std::getenv("MDJ_VPHASE_VARIANT");
    if (env) {
        ctx->vvar = std::max(0, std::min(NVPHASE_LAUNCH_VARIANTS - 1, std::atoi(env)));
        return MD_OK;
    }
    double* vs;
    unsigned long long *cs, *evs;
    uint32_t* es;
    int rc;
    if ((rc = dalloc(ctx, &vs, 3 * (size_t)d.N)) || (rc = dalloc(ctx, &cs, (size_t)d.R * NCOUNT)) ||
        (rc = dalloc(ctx, &evs, 1)) || (rc = dalloc(ctx, &es, d.R)))
        return rc;
    CK(cudaMemcpyAsync(vs, d.v, sizeof(double) * 3 * d.N, cudaMemcpyDeviceToDevice, ctx->s));
    CK(cudaMemcpyAsync(cs, d.cnt, sizeof(unsigned long long) * d.R * NCOUNT, cudaMemcpyDeviceToDevice, ctx->s));
    CK(cudaMemcpyAsync(evs, d.ev_n, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, ctx->s));
    CK(cudaMemcpyAsync(es, d.err, sizeof(uint32_t) * d.R, cudaMemcpyDeviceToDevice, ctx->s));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // each variant: one warm-up launch, then the fastest of three (robust to
    // interference); the set-up order replaces the rate ordering only when it
    // is clearly (2 %) faster, since the tuned phase is a single one
    float best[2] = {1e30f, 1e30f};
    int pick[2] = {0, NVPHASE_VARIANTS};
    for (int v = 0; v < NVPHASE_LAUNCH_VARIANTS; ++v) {
        float tmin = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            CK(cudaMemcpyAsync(d.v, vs, sizeof(double) * 3 * d.N, cudaMemcpyDeviceToDevice, ctx->s));
            cudaEventRecord(e0, ctx->s);
            launch_vphase(d, a, tau2, 0, 0, 0, 1, 1, 0, v, ctx->s, 0, single_params(ctx));
            cudaEventRecord(e1, ctx->s);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep) tmin = std::min(tmin, ms);
        }
        const int g = vphase_sorted(v) ? 0 : 1;
        if (tmin < best[g]) { best[g] = tmin; pick[g] = v; }
    }
    const int pick_v = best[1] < 0.98f * best[0] ? pick[1] : pick[0];
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaMemcpyAsync(d.v, vs, sizeof(double) * 3 * d.N, cudaMemcpyDeviceToDevice, ctx->s));
    CK(cudaMemcpyAsync(d.cnt, cs, sizeof(unsigned long long) * d.R * NCOUNT, cudaMemcpyDeviceToDevice, ctx->s));
    CK(cudaMemcpyAsync(d.ev_n, evs, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, ctx->s));
    CK(cudaMemcpyAsync(d.err, es, sizeof(uint32_t) * d.R, cudaMemcpyDeviceToDevice, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    for (void* p : {(void*)vs, (void*)cs, (void*)evs, (void*)es}) dfree(ctx, p);
    ctx->vvar = pick_v;
    if (ctx->tune_log)
        std::fprintf(stderr, "mdjump tune: velocity phase variant %d (%s, %s, occupancy %d): best rate-ordered %.4f ms, "
                     "best set-up order %.4f ms\n", pick_v, vphase_queue(pick_v) ? "queue" : "thread per atom",
                     vphase_sorted(pick_v) ? "rate order" : "set-up order", pick_v % NVPHASE_VARIANTS, best[0], best[1]);
    return MD_OK;
}

void vphase(md_ctx* ctx, const double* a, double tau2, uint32_t s_off, int half, int order, uint32_t s_off2 = 0)
{
    if (ctx->vvar < 0) tune_vphase(ctx, a, tau2);
    const int var = ctx->vvar < 0 ? 0 : ctx->vvar;
    // mixed: the rate order (3 kernels, unless the variant keeps the set-up order), then the phase kernel
    const bool sort = !ctx->fp64 && vphase_sorted(var);
    if (sort) {
        Prof p(ctx, 8, 3);
        launch_rate_order(ctx->d, a, tau2 * (order == 2 ? 2 : 1), ctx->s);
    }
    Prof p(ctx, 2, 1);
    launch_vphase(ctx->d, a, tau2, s_off, half, order, 1, 1, ctx->fp64, var, ctx->s, s_off2, single_params(ctx),
                  sort ? 1 : 0);
}

int set_stepc(md_ctx* ctx, double tau)
{
    const int R = ctx->d.R;
    for (int r = 0; r < R; ++r) {
        const RepParams& P = ctx->hp[r];
        ctx->h_stepc[2 * r] = std::exp(-P.gamma * tau);
        ctx->h_stepc[2 * r + 1] = std::sqrt(-std::expm1(-2.0 * P.gamma * tau) / P.beta);
    }
    CK(cudaMemcpyAsync(ctx->d.stepc, ctx->h_stepc, sizeof(double) * 2 * R, cudaMemcpyHostToDevice, ctx->s));
    return MD_OK;
}

int finish(md_ctx* ctx, long long inner_steps)
{
    {
        Prof p(ctx, 5, 1);
        launch_advance(ctx->d, inner_steps, ctx->s);
    }
    CK(cudaGetLastError());
    if (int rc = take_deferred(ctx)) return rc;
    CK(cudaMemcpyAsync(ctx->h_err, ctx->d.err, sizeof(uint32_t) * ctx->d.R, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    collect_profile(ctx);
    uint32_t f = 0;
    for (int r = 0; r < ctx->d.R; ++r) f |= ctx->h_err[r];
    if (f & F_NONFIN) FAIL(MD_ENONFINITE, "non-finite positions or velocities");
    if (f & F_BOUND) FAIL(MD_EBOUND, "a thinning acceptance ratio exceeded 1 (rate bound violated)");
    if (f & F_LIMIT) FAIL(MD_ELIMIT, "sampler attempt cap or proposal cap reached");
    if (f & F_OVERFLOW) {
        std::vector<uint32_t> o(ctx->d.R);
        CK(cudaMemcpy(o.data(), ctx->d.ovf, sizeof(uint32_t) * ctx->d.R, cudaMemcpyDeviceToHost));
        uint32_t m = 0;
        for (uint32_t v : o) m |= v;
        static const char* names[NKIND] = {"short", "full", "ring 0", "ring 1", "ring 2", "ring 3", "LJ"};
        static_assert(NKIND == 7, "list kind names");
        std::string which;
        for (int b = 0; b < NKIND; ++b)
            if (m & (1u << b)) which += std::string(which.empty() ? "" : ", ") + names[b];
        if (m & OVF_OUTER) which += std::string(which.empty() ? "" : ", ") + "outer";
        if (m & OVF_CELL) which += std::string(which.empty() ? "" : ", ") + "cell";
        if (m & OVF_TILE) which += std::string(which.empty() ? "" : ", ") + "cluster pairs";
        if (m & OVF_FIX)
            FAIL(MD_EOVERFLOW, "a pair force term left the range of the 64-bit fixed-point sums "
                               "(|component| >= 2^20 kcal/mol/A, or not finite)%s%s",
                 which.empty() ? "" : "; capacity exceeded too: ", which.c_str());
        FAIL(MD_EOVERFLOW, "capacity exceeded: %s (lists are sized at set-up; an unstable run "
                           "packs atoms denser than that)", which.c_str());
    }
    return MD_OK;
}

int prepare(md_ctx* ctx, int family, double dt_fs)
{
    if (!ctx) return MD_EINVAL;
    if (!(dt_fs > 0) || !std::isfinite(dt_fs)) FAIL(MD_EINVAL, "time step must be positive");
    int rc = commit(ctx);
    if (rc) return rc;
    if ((rc = ensure_kinds(ctx, lists_needed(ctx, family)))) return rc;
    CK(cudaMemsetAsync(ctx->d.flags, 0, sizeof(int) * 2 * ctx->d.R, ctx->s));
    return MD_OK;
}

// ---- CUDA graphs ------------------------------------------------------------
void drop_graphs(md_ctx* ctx)
{
    for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
}

// Runs `units` units of a driver (a step, or a RESPA cycle of spu inner
// steps). body(u0, n) issues n units whose random streams are offset from
// the replicas' step bases by u0 units. With graphs on, chunks of G units
// (about four innermost steps) replay a graph captured once per time step,
// driver and device layout. The first call of a kind runs its first unit as
// plain launches (it runs the autotuners, which time real launches) and
// advances the step bases, then captures the chunk (at offset 0, with the
// step bases advanced by G units inside it); later calls, such as the timed
// steps after a warm-up, replay it from their first unit on. What is left
// runs plainly at offset 0 and finish() advances the step bases past it. The
// streams, and so the results, are those of a plain run.
template <typename Body>
int run_units(md_ctx* ctx, int key, double tau, int spu, long long units, Body body)
{
    Dev& d = ctx->d;
    const long long G = std::max(1, 4 / spu);
    long long done = 0;
    if (!ctx->cfg.no_graphs && !ctx->prof && !ctx->graphs_broken && units >= G) {
        // graphs of an older device layout can never replay again: release them
        // (every earlier call ended with a synchronisation; the private stream is idle)
        for (size_t k = 0; k < ctx->graphs.size();) {
            if (ctx->graphs[k].gen != ctx->gen) {
                cudaGraphExecDestroy(ctx->graphs[k].exec);
                ctx->graphs.erase(ctx->graphs.begin() + (long)k);
            } else {
                ++k;
            }
        }
        const md_ctx::Graph* g = nullptr;
        for (const auto& x : ctx->graphs)
            if (x.gen == ctx->gen && x.key == key && x.tau == tau && x.n_inner == spu && x.units == G) g = &x;
        if (!g && units >= G + 1) {
            body(0, 1);
            launch_advance(d, spu, ctx->s);
            ctx->nlaunch[5] += 1;
            done = 1;
            if (!ctx->gs) CK(cudaStreamCreateWithFlags(&ctx->gs, cudaStreamNonBlocking));
            // capture on the private stream (the caller's may be the legacy default stream)
            cudaEvent_t e = take_event(ctx);
            CK(cudaEventRecord(e, ctx->s));
            CK(cudaStreamWaitEvent(ctx->gs, e, 0));
            ctx->ev_pool.push_back(e);
            cudaStream_t s0 = ctx->s;
            long long before[NPROF];
            std::copy(ctx->nlaunch, ctx->nlaunch + NPROF, before);
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            ctx->s = ctx->gs;
            cudaError_t ce = cudaStreamBeginCapture(ctx->gs, cudaStreamCaptureModeThreadLocal);
            if (ce == cudaSuccess) {
                body(0, G);
                launch_advance(d, G * spu, ctx->s);
                ce = cudaStreamEndCapture(ctx->gs, &graph);
            }
            ctx->s = s0;
            if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (ce != cudaSuccess) {
                // no graph: fall back to plain launches for good
                cudaGetLastError();
                ctx->graphs_broken = true;
                std::copy(before, before + NPROF, ctx->nlaunch);
                CK(cudaStreamSynchronize(ctx->gs));
            } else {
                md_ctx::Graph ng{ctx->gen, key, tau, spu, (int)G, exec, {}};
                for (int c = 0; c < NPROF; ++c) ng.launches[c] = ctx->nlaunch[c] - before[c] + (c == 5 ? 1 : 0);
                std::copy(before, before + NPROF, ctx->nlaunch);
                ctx->graphs.push_back(ng);
                g = &ctx->graphs.back();
            }
        }
        if (g) {
            cudaEvent_t e = take_event(ctx);
            CK(cudaEventRecord(e, ctx->s));
            CK(cudaStreamWaitEvent(ctx->gs, e, 0));
            while (units - done >= G) {
                CK(cudaGraphLaunch(g->exec, ctx->gs));
                for (int c = 0; c < NPROF; ++c) ctx->nlaunch[c] += g->launches[c];
                ctx->ngraph_launches += 1;
                done += G;
            }
            CK(cudaEventRecord(e, ctx->gs));
            CK(cudaStreamWaitEvent(ctx->s, e, 0));
            ctx->ev_pool.push_back(e);
        }
    }
    // the step bases already count the units done above: offsets restart at 0
    body(0, units - done);
    return finish(ctx, (units - done) * spu);
}

// velocity record of the innermost step s_off (relative to the step bases) that just ended
void record(md_ctx* ctx, uint32_t s_off)
{
    if (!ctx->vr) return;
    Prof p(ctx, 5, 1);
    launch_vacf_record(ctx->d, ctx->vr, ctx->fp64, ctx->vr_origin, ctx->vr_cap, s_off, ctx->s);
}

// inner bonded step of the RESPA family: B A O A [grad] B at dt
void inner_bonded(md_ctx* ctx, double dt, uint32_t s_off, int check)
{
    Dev& d = ctx->d;
    // the two kicks ride in the A O A and bonded-gather launches (same arithmetic)
    {
        Prof p(ctx, 3, 1);
        launch_aoa(d, dt, s_off, check, ctx->fp64, ctx->s, d.ab, 0.5 * dt);
    }
    Prof p(ctx, 1, d.nbond + d.nang > 0 ? 2 : 1);
    launch_bonded_kick(d, d.ab, 0.5 * dt, ctx->s);
}

// n inner steps from s_off: fused into one launch when the bonded groups
// allow it and no velocity record needs the steps one by one; the list check
// runs on the last step
void inner_steps(md_ctx* ctx, double dt, uint32_t s_off, int n)
{
    if (ctx->d.n_ib > 0 && !ctx->vr && ctx->fuse_inner) {
        Prof p(ctx, 3, 1);
        launch_inner_steps(ctx->d, dt, s_off, n, 1, ctx->fp64, ctx->s);
        return;
    }
    for (int k = 0; k < n; ++k) {
        inner_bonded(ctx, dt, s_off + uint32_t(k), k == n - 1);
        if (k < n - 1) record(ctx, s_off + uint32_t(k));
    }
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

int md_init(md_ctx** out, const md_config* cfg)
{
    if (!out || !cfg) { set_global_error("md_init: null argument"); return MD_EINVAL; }
    *out = nullptr;
    if (cfg->precision != MD_FP64 && cfg->precision != MD_MIXED) { set_global_error("md_init: precision must be MD_FP64 or MD_MIXED"); return MD_EINVAL; }
    if (cfg->max_replicas < 1 || cfg->max_replicas > 65536) { set_global_error("md_init: max_replicas out of range"); return MD_EINVAL; }
    if (cfg->threads_per_atom != 0 && cfg->threads_per_atom != 1 && cfg->threads_per_atom != 2 &&
        cfg->threads_per_atom != 4 && cfg->threads_per_atom != 8) { set_global_error("md_init: threads_per_atom must be 0, 1, 2, 4 or 8"); return MD_EINVAL; }
    if (cfg->event_log_cap < 0) { set_global_error("md_init: event_log_cap < 0"); return MD_EINVAL; }
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess) { set_global_error(std::string("md_init: cudaSetDevice: ") + cudaGetErrorString(e)); return MD_ECUDA; }
    md_ctx* ctx = new md_ctx();
    ctx->cfg = *cfg;
    ctx->s = (cudaStream_t)cfg->cuda_stream;
    ctx->fp64 = cfg->precision == MD_FP64;
    ctx->tpa_cfg = cfg->threads_per_atom;
    ctx->fuse_inner = std::getenv("MDJ_FUSED_INNER") != nullptr;
    ctx->tune_log = std::getenv("MDJ_TUNE_LOG") != nullptr;
    ctx->reps.resize(cfg->max_replicas);
    bool ok = cudaMallocHost((void**)&ctx->h_stepc, sizeof(double) * 2 * cfg->max_replicas) == cudaSuccess;
    if (ok && cudaMallocHost((void**)&ctx->h_err, sizeof(uint32_t) * cfg->max_replicas) != cudaSuccess) {
        cudaFreeHost(ctx->h_stepc);
        ok = false;
    }
    if (!ok) {
        set_global_error("md_init: pinned host allocation failed");
        delete ctx;
        return MD_ENOMEM;
    }
    *out = ctx;
    return MD_OK;
}

int md_set_system(md_ctx* ctx, int replica, const md_system* sys)
{
    if (!ctx) return MD_EINVAL;
    if (replica < 0 || replica >= (int)ctx->reps.size()) FAIL(MD_EINVAL, "replica %d out of range", replica);
    int rc = check_sys(ctx, sys);
    if (rc) return rc;
    if ((rc = download_all(ctx))) return rc;
    RepHost& h = ctx->reps[replica];
    const int n = sys->n_atoms;
    h = RepHost();
    h.set = true;
    h.fresh = true;
    h.n = n;
    h.box = sys->box;
    h.sys = *sys;
    h.x.assign(sys->x, sys->x + 3 * n);
    h.v.assign(sys->v, sys->v + 3 * n);
    h.img.assign(3 * n, 0);
    for (int k = 0; k < 3 * n; ++k) {       // wrap into [0, L), images start at zero
        double t = h.x[k];
        t -= h.box * std::floor(t / h.box);
        if (t >= h.box) t -= h.box;
        h.x[k] = t;
    }
    h.xb = h.x;
    h.xo = h.x;
    h.mass.assign(sys->mass, sys->mass + n);
    h.charge.assign(sys->charge, sys->charge + n);
    h.type.assign(sys->type, sys->type + n);
    h.ntypes = sys->n_types;
    h.lj_eps.assign(sys->lj_eps, sys->lj_eps + sys->n_types * sys->n_types);
    h.lj_sig.assign(sys->lj_sigma, sys->lj_sigma + sys->n_types * sys->n_types);
    h.bonds.assign(sys->bonds, sys->bonds + 2 * sys->n_bonds);
    h.bond_k.assign(sys->bond_k, sys->bond_k + sys->n_bonds);
    h.bond_r0.assign(sys->bond_r0, sys->bond_r0 + sys->n_bonds);
    h.angles.assign(sys->angles, sys->angles + 3 * sys->n_angles);
    h.ang_k.assign(sys->angle_k, sys->angle_k + sys->n_angles);
    h.ang_t0.assign(sys->angle_t0, sys->angle_t0 + sys->n_angles);
    h.excl.assign(sys->excl_pairs, sys->excl_pairs + 2 * sys->n_excl);
    // keep no caller pointers
    h.sys.x = h.sys.v = h.sys.mass = h.sys.charge = nullptr;
    h.sys.type = nullptr;
    h.sys.lj_eps = h.sys.lj_sigma = nullptr;
    h.sys.bonds = h.sys.angles = h.sys.excl_pairs = nullptr;
    h.sys.bond_k = h.sys.bond_r0 = h.sys.angle_k = h.sys.angle_t0 = nullptr;
    h.step = 0;
    ctx->dirty = true;
    return commit(ctx);
}

int md_set_state(md_ctx* ctx, int replica, const double* x, const double* v, const int* img,
                 const double* x_build, const double* x_outer, int64_t step)
{
    if (!ctx) return MD_EINVAL;
    int rc = commit(ctx);
    if (rc) return rc;
    if (replica < 0 || replica >= ctx->d.R) FAIL(MD_EINVAL, "replica %d out of range", replica);
    if (!x || !v) FAIL(MD_EINVAL, "md_set_state: x and v are required");
    Dev& d = ctx->d;
    vacf_stop(ctx);     // the record assumes uninterrupted steps
    const RepHost& h = ctx->reps[replica];
    const size_t o = 3 * (size_t)ctx->rep_atom_off[replica], n3 = 3 * (size_t)h.n;
    std::vector<int> zero;
    if (!img) { zero.assign(n3, 0); img = zero.data(); }
    const double* xb = x_build ? x_build : x;
    const double* xo = x_outer ? x_outer : xb;
    CK(cudaStreamSynchronize(ctx->s));
    CK(cudaMemcpy(d.x + o, x, n3 * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.v + o, v, n3 * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.img + o, img, n3 * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.xb + o, xb, n3 * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.xo + o, xo, n3 * sizeof(double), cudaMemcpyHostToDevice));
    long long st = step;
    CK(cudaMemcpy(d.step_base + replica, &st, sizeof st, cudaMemcpyHostToDevice));
    const int fl[2] = {1, 1};
    CK(cudaMemsetAsync(d.flags, 0, sizeof(int) * 2 * d.R, ctx->s));
    CK(cudaMemcpyAsync(d.flags + 2 * replica, fl, sizeof fl, cudaMemcpyHostToDevice, ctx->s));
    // lists at the given build positions; in mixed mode the run's own decisions
    // (FP32, with the ring and LJ limits re-decided in FP64), which give the
    // same ring and LJ lists as the exact set-up build at a fraction of its
    // cost (FP64 runs at a small fraction of the FP32 rate on this GPU)
    launch_rebuild(d, ctx->kinds, ctx->fp64, 1, ctx->fp64, 0, ctx->s);
    CK(cudaGetLastError());
    // the list build is not a rebuild of the run: undo the counter increments
    std::vector<unsigned long long> c(NCOUNT);
    CK(cudaMemcpyAsync(c.data(), d.cnt + (size_t)replica * NCOUNT, sizeof(unsigned long long) * NCOUNT,
                       cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    c[C_REBUILD] -= 1;
    c[C_OUTER] -= 1;
    CK(cudaMemcpy(d.cnt + (size_t)replica * NCOUNT, c.data(), sizeof(unsigned long long) * NCOUNT,
                  cudaMemcpyHostToDevice));
    return MD_OK;
}

int md_step_baoab(md_ctx* ctx, int64_t nsteps, double dt_fs)
{
    int rc = prepare(ctx, 0, dt_fs);
    if (rc) return rc;
    if (nsteps < 0) FAIL(MD_EINVAL, "nsteps < 0");
    Dev& d = ctx->d;
    const double tau = dt_fs * 1e-3;
    if ((rc = set_stepc(ctx, tau))) return rc;
    force(ctx, 0, d.a0);
    return run_units(ctx, 0, tau, 1, nsteps, [&](long long u0, long long n) {
        for (long long k = u0; k < u0 + n; ++k) {
            kick(ctx, d.a0, 0.5 * tau);
            aoa(ctx, tau, uint32_t(k), 1);
            rebuild_step(ctx);
            force(ctx, 0, d.a0);
            kick(ctx, d.a0, 0.5 * tau);
            record(ctx, uint32_t(k));
        }
    });
}

int md_step_jump(md_ctx* ctx, int64_t nsteps, double dt_fs)
{
    int rc = prepare(ctx, 2, dt_fs);
    if (rc) return rc;
    if (nsteps < 0) FAIL(MD_EINVAL, "nsteps < 0");
    Dev& d = ctx->d;
    const double tau = dt_fs * 1e-3;
    if ((rc = set_stepc(ctx, tau))) return rc;
    force(ctx, 5, d.a0);
    // C'J' A O A [F0] J'C', step after step. In mixed mode the C' of the second
    // half of step k and the C' of the first half of step k+1 (adjacent, at the
    // same positions and acceleration) run in one launch, unless velocities are
    // recorded between the two.
    const bool fuse = !ctx->fp64 && !ctx->vr;
    return run_units(ctx, 1, tau, 1, nsteps, [&](long long u0, long long n) {
        for (long long k = u0; k < u0 + n; ++k) {
            if (k == u0 || !fuse) vphase(ctx, d.a0, 0.5 * tau, uint32_t(k), 0, 0);
            aoa(ctx, tau, uint32_t(k), 1);
            rebuild_step(ctx);
            force(ctx, 5, d.a0);
            if (fuse && k + 1 < u0 + n) vphase(ctx, d.a0, 0.5 * tau, uint32_t(k), 1, 2, uint32_t(k + 1));
            else vphase(ctx, d.a0, 0.5 * tau, uint32_t(k), 1, 1);
            record(ctx, uint32_t(k));
        }
    });
}

int md_step_bjaoajb(md_ctx* ctx, int64_t nsteps, double dt_fs)
{
    int rc = prepare(ctx, 2, dt_fs);
    if (rc) return rc;
    if (nsteps < 0) FAIL(MD_EINVAL, "nsteps < 0");
    Dev& d = ctx->d;
    const double tau = dt_fs * 1e-3;
    if ((rc = set_stepc(ctx, tau))) return rc;
    force(ctx, 5, d.a0);
    // B J A O A [F0] J B: the velocity phases run the jump processes alone (no drift)
    return run_units(ctx, 5, tau, 1, nsteps, [&](long long u0, long long n) {
        for (long long k = u0; k < u0 + n; ++k) {
            kick(ctx, d.a0, 0.5 * tau);
            vphase(ctx, nullptr, 0.5 * tau, uint32_t(k), 0, 0);
            aoa(ctx, tau, uint32_t(k), 1);
            rebuild_step(ctx);
            force(ctx, 5, d.a0);
            vphase(ctx, nullptr, 0.5 * tau, uint32_t(k), 1, 1);
            kick(ctx, d.a0, 0.5 * tau);
            record(ctx, uint32_t(k));
        }
    });
}

int md_step_baoab_respa(md_ctx* ctx, int64_t n_outer, double dt_inner_fs, int n_inner)
{
    int rc = prepare(ctx, 0, dt_inner_fs);
    if (rc) return rc;
    if (n_outer < 0 || n_inner < 1) FAIL(MD_EINVAL, "n_outer >= 0 and n_inner >= 1 required");
    Dev& d = ctx->d;
    const double dt = dt_inner_fs * 1e-3, D = dt * n_inner;
    if ((rc = set_stepc(ctx, dt))) return rc;
    force(ctx, 1, d.ab);
    force(ctx, 2, d.al);
    return run_units(ctx, 2, dt, n_inner, n_outer, [&](long long u0, long long n) {
        uint32_t s = uint32_t(u0 * n_inner);
        for (long long o = 0; o < n; ++o) {
            kick(ctx, d.al, 0.5 * D);
            inner_steps(ctx, dt, s, n_inner);
            s += n_inner;
            rebuild_step(ctx);
            force(ctx, 2, d.al);
            kick(ctx, d.al, 0.5 * D);
            record(ctx, s - 1);
        }
    });
}

int md_step_baoab_respa1(md_ctx* ctx, int64_t n_outer, double dt_inner_fs, int m_mid, int n_outer_ratio)
{
    int rc = prepare(ctx, 1, dt_inner_fs);
    if (rc) return rc;
    if (n_outer < 0 || m_mid < 1 || n_outer_ratio < 1) FAIL(MD_EINVAL, "n_outer >= 0, m_mid >= 1, n_outer_ratio >= 1 required");
    Dev& d = ctx->d;
    const double dt = dt_inner_fs * 1e-3, kap = dt * m_mid, D = kap * n_outer_ratio;
    if ((rc = set_stepc(ctx, dt))) return rc;
    force(ctx, 1, d.ab);
    force(ctx, 3, d.as);
    force_into(ctx, 4, d.al, 0, false);
    recip_begin(ctx);
    recip_end(ctx);
    const int spu = n_outer_ratio * m_mid;
    return run_units(ctx, 3 | (m_mid << 8), dt, spu, n_outer, [&](long long u0, long long n) {
        uint32_t s = uint32_t(u0 * spu);
        for (long long o = 0; o < n; ++o) {
            slow_kick(ctx, 0.5 * D);
            for (int j = 0; j < n_outer_ratio; ++j) {
                kick(ctx, d.as, 0.5 * kap);
                inner_steps(ctx, dt, s, m_mid);
                s += m_mid;
                rebuild_step(ctx);
                force(ctx, 3, d.as);
                if (j == n_outer_ratio - 1) recip_begin(ctx);     // positions of the slow step are final
                kick(ctx, d.as, 0.5 * kap);
                if (j < n_outer_ratio - 1) record(ctx, s - 1);
            }
            force_into(ctx, 4, d.al, 0, false);
            recip_end(ctx);
            slow_kick(ctx, 0.5 * D);
            record(ctx, s - 1);
        }
    });
}

// JUMP-RESPA (ratio 1, outer period Delta = n_inner dt) and JUMP-RESPA1
// (mid period kappa = n_inner dt, outer Delta = ratio kappa): C'J' at the mid
// level around bonded inner steps; the Ewald reciprocal part, when a replica
// has one, is kicked at the outer level around each group of `ratio` cycles.
static int jump_respa_cycles(md_ctx* ctx, int64_t n_outer, double dt_inner_fs, int n_inner, int ratio)
{
    Dev& d = ctx->d;
    // a slow level exists when some replica has a reciprocal part or keeps its LJ long part there
    const bool ew = !ctx->ewald_reps.empty() || any_lj_slow(ctx);
    const double dt = dt_inner_fs * 1e-3, kap = dt * n_inner, D = kap * ratio;
    int rc;
    if ((rc = set_stepc(ctx, dt))) return rc;
    force(ctx, 1, d.ab);
    force(ctx, 3, d.as);
    if (ew) {
        force_into(ctx, 6, d.al, 0, false);
        recip_begin(ctx);
        recip_end(ctx);
    }
    // with no outer force a unit is one mid cycle; else one outer step of ratio cycles
    const int per = ew ? ratio : 1;
    const long long units = ew ? n_outer : n_outer * ratio;
    // as in md_step_jump, adjacent C' phases of consecutive cycles share a launch in
    // mixed mode (not across an outer kick, which changes the velocities in between)
    const bool fuse = !ctx->fp64 && !ctx->vr;
    return run_units(ctx, 4 | (n_inner << 8), dt, per * n_inner, units, [&](long long u0, long long n) {
        uint32_t s = uint32_t(u0 * per * n_inner);
        for (long long o = 0; o < n; ++o) {
            if (ew) slow_kick(ctx, 0.5 * D);
            for (int j = 0; j < per; ++j) {
                const uint32_t s0 = s;
                const bool carried = fuse && (ew ? j > 0 : o > 0);
                const bool pass_on = fuse && (ew ? j + 1 < per : o + 1 < n);
                if (!carried) vphase(ctx, d.as, 0.5 * kap, s0, 0, 0);
                inner_steps(ctx, dt, s, n_inner);
                s += n_inner;
                rebuild_step(ctx);
                force(ctx, 3, d.as);
                if (ew && j == per - 1) recip_begin(ctx);        // positions of the slow step are final
                if (pass_on) vphase(ctx, d.as, 0.5 * kap, s0, 1, 2, s);
                else vphase(ctx, d.as, 0.5 * kap, s0, 1, 1);
                if (j < per - 1) record(ctx, s - 1);
            }
            if (ew) {
                force_into(ctx, 6, d.al, 0, false);
                recip_end(ctx);
                slow_kick(ctx, 0.5 * D);
            }
            record(ctx, s - 1);
        }
    });
}

int md_step_jump_respa(md_ctx* ctx, int64_t n_outer, double dt_inner_fs, int n_inner)
{
    int rc = prepare(ctx, 2, dt_inner_fs);
    if (rc) return rc;
    if (n_outer < 0 || n_inner < 1) FAIL(MD_EINVAL, "n_outer >= 0 and n_inner >= 1 required");
    return jump_respa_cycles(ctx, n_outer, dt_inner_fs, n_inner, 1);
}

int md_step_jump_respa1(md_ctx* ctx, int64_t n_outer, double dt_inner_fs, int m_mid, int n_outer_ratio)
{
    int rc = prepare(ctx, 2, dt_inner_fs);
    if (rc) return rc;
    if (n_outer < 0 || m_mid < 1 || n_outer_ratio < 1) FAIL(MD_EINVAL, "n_outer >= 0, m_mid >= 1, n_outer_ratio >= 1 required");
    return jump_respa_cycles(ctx, n_outer, dt_inner_fs, m_mid, n_outer_ratio);
}

int md_observables(md_ctx* ctx, int replica, md_obs* out)
{
    if (!ctx || !out) return MD_EINVAL;
    int rc = commit(ctx);
    if (rc) return rc;
    if (replica < 0 || replica >= ctx->d.R) FAIL(MD_EINVAL, "replica %d out of range", replica);
    Dev& d = ctx->d;
    CK(cudaMemsetAsync(d.energy, 0, sizeof(double) * 6 * d.R, ctx->s));
    launch_energy(d, ctx->s);
    double erec = 0.0;
    const bool ew = ctx->hp[replica].coul_mode == 1;
    if (ew) {
        CK(cudaMemsetAsync(d.pme_e, 0, sizeof(double) * d.R, ctx->s));
        if ((rc = pme(ctx, nullptr, 0, 1))) return rc;
        launch_pme_excl_energy(d, ctx->s);
        CK(cudaMemcpyAsync(&erec, d.pme_e + replica, sizeof erec, cudaMemcpyDeviceToHost, ctx->s));
    }
    CK(cudaGetLastError());
    double e[6];
    unsigned long long c[NCOUNT];
    long long st;
    uint32_t err;
    CK(cudaMemcpyAsync(e, d.energy + 6 * replica, sizeof e, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaMemcpyAsync(c, d.cnt + (size_t)replica * NCOUNT, sizeof c, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaMemcpyAsync(&st, d.step_base + replica, sizeof st, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaMemcpyAsync(&err, d.err + replica, sizeof err, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    const int n = ctx->reps[replica].n;
    std::memset(out, 0, sizeof *out);
    out->pe_bond = e[0]; out->pe_angle = e[1]; out->pe_lj = e[2]; out->pe_coul = e[3];
    if (ew) out->pe_coul += erec + ctx->hp[replica].pme_self;
    out->ke = e[4];
    out->temperature = 2.0 * e[4] / (3.0 * n * KB);
    out->step = st;
    out->jump_proposals = (int64_t)c[C_CPROP]; out->jump_accepts = (int64_t)c[C_CACC];
    out->bps_proposals = (int64_t)c[C_JPROP]; out->bps_accepts = (int64_t)c[C_JACC];
    out->sampler_attempts = (int64_t)c[C_SATT]; out->list_rebuilds = (int64_t)c[C_REBUILD];
    out->outer_rebuilds = (int64_t)c[C_OUTER]; out->guarded_accepts = (int64_t)c[C_GUARD];
    out->error_flags = err;
    return MD_OK;
}

int md_get_state(md_ctx* ctx, int replica, double* x, double* v, int* img, double* x_build, double* x_outer)
{
    if (!ctx) return MD_EINVAL;
    int rc = commit(ctx);
    if (rc) return rc;
    if (replica < 0 || replica >= ctx->d.R) FAIL(MD_EINVAL, "replica %d out of range", replica);
    Dev& d = ctx->d;
    const size_t o = 3 * (size_t)ctx->rep_atom_off[replica], n3 = 3 * (size_t)ctx->reps[replica].n;
    if (x) CK(cudaMemcpyAsync(x, d.x + o, n3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    if (v) CK(cudaMemcpyAsync(v, d.v + o, n3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    if (img) CK(cudaMemcpyAsync(img, d.img + o, n3 * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    if (x_build) CK(cudaMemcpyAsync(x_build, d.xb + o, n3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    if (x_outer) CK(cudaMemcpyAsync(x_outer, d.xo + o, n3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    return MD_OK;
}

int md_gradient(md_ctx* ctx, int replica, int mode, double* host_grad)
{
    if (!ctx || !host_grad) return MD_EINVAL;
    if (mode < 0 || mode > 6) FAIL(MD_EINVAL, "gradient mode %d out of range", mode);
    int rc = commit(ctx);
    if (rc) return rc;
    if (replica < 0 || replica >= ctx->d.R) FAIL(MD_EINVAL, "replica %d out of range", replica);
    if ((rc = ensure_kinds(ctx, mode_list(ctx, mode)))) return rc;
    Dev& d = ctx->d;
    force_into(ctx, mode, d.gout, 1);
    CK(cudaGetLastError());
    if ((rc = take_deferred(ctx))) return rc;
    const size_t o = 3 * (size_t)ctx->rep_atom_off[replica], n3 = 3 * (size_t)ctx->reps[replica].n;
    CK(cudaMemcpyAsync(host_grad, d.gout + o, n3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    return MD_OK;
}

int md_run_phase(md_ctx* ctx, int phase, double tau2_ps, int64_t s0, int half, int accel_mode)
{
    if (!ctx) return MD_EINVAL;
    if ((phase != 0 && phase != 1) || (half != 0 && half != 1) || !(tau2_ps >= 0) || accel_mode < 0 || accel_mode > 5)
        FAIL(MD_EINVAL, "md_run_phase: bad phase, half, tau2 or accel_mode");
    int rc = commit(ctx);
    if (rc) return rc;
    int rings = 0;
    for (int y = 0; y < MAX_RINGS; ++y) rings |= 1 << (L_R0 + y);
    const int need = (phase == 0 ? rings | mode_list(ctx, accel_mode) : (1 << L_LJ));
    if ((rc = ensure_kinds(ctx, need))) return rc;
    Dev& d = ctx->d;
    if (phase == 0) force(ctx, accel_mode, d.a0);
    {
        // phase 0: rate order (3 kernels, unless the variant keeps the set-up order), then C'; phase 1: J' only
        const int var = ctx->vvar < 0 ? 0 : ctx->vvar;
        const bool sort = !ctx->fp64 && phase == 0 && vphase_sorted(var);
        if (sort) {
            Prof p(ctx, 8, 3);
            launch_rate_order(d, d.a0, tau2_ps, ctx->s);
        }
        Prof p(ctx, 2, 1);
        launch_vphase_abs(d, phase == 0 ? d.a0 : nullptr, tau2_ps, uint32_t(s0), half, 0, phase == 0, phase == 1,
                          ctx->fp64, var, ctx->s, single_params(ctx), sort ? 1 : 0);
    }
    CK(cudaGetLastError());
    if ((rc = take_deferred(ctx))) return rc;
    CK(cudaMemcpyAsync(ctx->h_err, d.err, sizeof(uint32_t) * d.R, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    return MD_OK;
}

int md_get_list(md_ctx* ctx, int replica, int kind, int atom, int* host_out, int cap)
{
    if (!ctx) return MD_EINVAL;
    int rc = commit(ctx);
    if (rc) return rc;
    if (replica < 0 || replica >= ctx->d.R || kind < 0 || kind > MAX_RINGS || atom < 0 ||
        atom >= ctx->reps[replica].n)
        FAIL(MD_EINVAL, "md_get_list: bad replica, kind or atom");
    const int k = kind < MAX_RINGS ? L_R0 + kind : L_LJ;
    if ((rc = ensure_kinds(ctx, 1 << k))) return rc;
    Dev& d = ctx->d;
    const int gi = ctx->rep_atom_off[replica] + atom;
    int n;
    CK(cudaMemcpyAsync(&n, d.lcnt[k] + gi, sizeof n, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    const int m = std::min(std::min(n, d.lcap[k]), std::max(cap, 0));
    if (m > 0 && host_out) {
        std::vector<uint32_t> e(m);
        CK(cudaMemcpy(e.data(), d.list[k] + (size_t)gi * d.lcap[k], sizeof(uint32_t) * m, cudaMemcpyDeviceToHost));
        for (int t = 0; t < m; ++t) host_out[t] = int(e[t]) - ctx->rep_atom_off[replica];
    }
    return n;
}

int64_t md_get_events(md_ctx* ctx, int replica, int64_t* host_out6, int64_t cap, int clear)
{
    if (!ctx) return MD_EINVAL;
    int rc = commit(ctx);
    if (rc) return rc;
    Dev& d = ctx->d;
    unsigned long long n = 0;
    CK(cudaMemcpyAsync(&n, d.ev_n, sizeof n, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    const long long m = std::min<long long>((long long)n, d.ev_cap);
    std::vector<long long> ev((size_t)6 * (m > 0 ? m : 1));
    if (m > 0) CK(cudaMemcpy(ev.data(), d.ev, sizeof(long long) * 6 * m, cudaMemcpyDeviceToHost));
    int64_t w = 0;
    for (long long t = 0; t < m && w < cap; ++t) {
        if ((ev[6 * t + 2] >> 8) != replica) continue;
        if (host_out6) {
            for (int c = 0; c < 6; ++c) host_out6[6 * w + c] = ev[6 * t + c];
            host_out6[6 * w + 2] &= 0xff;
        }
        ++w;
    }
    if (clear) CK(cudaMemsetAsync(d.ev_n, 0, sizeof(unsigned long long), ctx->s));
    if ((long long)n > d.ev_cap) FAIL(MD_EOVERFLOW, "event log overflowed (%llu events, capacity %lld)", n, d.ev_cap);
    return w;
}

int md_profile(md_ctx* ctx, int enable, int reset, double* ms_out, int64_t* groups_out,
               int64_t* launches_out)
{
    if (!ctx) return MD_EINVAL;
    if (!ctx->pend.empty()) {
        CK(cudaStreamSynchronize(ctx->s));
        collect_profile(ctx);
    }
    if (reset) {
        for (int k = 0; k < NPROF; ++k) { ctx->prof_ms[k] = 0; ctx->prof_groups[k] = 0; }
    }
    if (enable == 0 || enable == 1) ctx->prof = enable == 1;
    for (int k = 0; k < NPROF; ++k) {
        if (ms_out) ms_out[k] = ctx->prof_ms[k];
        if (groups_out) groups_out[k] = ctx->prof_groups[k];
        if (launches_out) launches_out[k] = ctx->nlaunch[k];
    }
    return MD_OK;
}

int md_vacf_start(md_ctx* ctx, int64_t n_samples)
{
    if (!ctx) return MD_EINVAL;
    if (n_samples < 0) FAIL(MD_EINVAL, "md_vacf_start: n_samples < 0");
    int rc = commit(ctx);
    if (rc) return rc;
    vacf_stop(ctx);
    if (n_samples == 0) return MD_OK;
    const size_t bytes = (size_t)n_samples * 3 * (size_t)ctx->d.N * (ctx->fp64 ? sizeof(double) : sizeof(float));
    if (cudaMallocAsync(&ctx->vr, bytes, ctx->s) != cudaSuccess) {
        cudaGetLastError();
        ctx->vr = nullptr;
        FAIL(MD_ENOMEM, "md_vacf_start: %zu bytes for %lld samples", bytes, (long long)n_samples);
    }
    long long sb = 0;
    CK(cudaMemcpyAsync(&sb, ctx->d.step_base, sizeof sb, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    ctx->vr_cap = n_samples;
    ctx->vr_origin = sb;
    return MD_OK;
}

int md_vacf_get(md_ctx* ctx, int replica, int64_t n_lags, double* vacf_out, double* spectrum_out, int64_t* n_stored)
{
    if (!ctx) return MD_EINVAL;
    if (n_lags < 1) FAIL(MD_EINVAL, "md_vacf_get: n_lags < 1");
    int rc = commit(ctx);
    if (rc) return rc;
    if (replica < 0 || replica >= ctx->d.R) FAIL(MD_EINVAL, "replica %d out of range", replica);
    Dev& d = ctx->d;
    long long T = 0;
    if (ctx->vr) {
        long long sb = 0;
        CK(cudaMemcpyAsync(&sb, d.step_base, sizeof sb, cudaMemcpyDeviceToHost, ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
        T = std::max(0LL, std::min(ctx->vr_cap, sb - ctx->vr_origin));
    }
    if (n_stored) *n_stored = T;
    if (T == 0) {
        if (vacf_out) std::fill(vacf_out, vacf_out + n_lags, 0.0);
        if (spectrum_out) std::fill(spectrum_out, spectrum_out + n_lags, 0.0);
        return MD_OK;
    }
    const int fp64 = ctx->fp64;
    const size_t e = fp64 ? sizeof(double) : sizeof(float);
    const int n3 = 3 * d.N, s_lo = 3 * ctx->rep_atom_off[replica], s_hi = s_lo + 3 * ctx->reps[replica].n;
    const long long nj = T + 1;
    // series per transform batch: about 2 GB of padded input and spectrum at most
    const int nb = (int)std::max(1LL, std::min((long long)(s_hi - s_lo), (long long)(2e9 / (4.0 * T * e))));
    void *pad = nullptr, *X = nullptr;
    double *P = nullptr, *r = nullptr, *C = nullptr, *S = nullptr;
    double2* Z = nullptr;
    cufftHandle fw = 0, bw = 0;
    auto cleanup = [&]() {
        if (fw) cufftDestroy(fw);
        if (bw) cufftDestroy(bw);
        for (void* p : {pad, X, (void*)P, (void*)r, (void*)C, (void*)S, (void*)Z})
            if (p) cudaFreeAsync(p, ctx->s);
    };
    auto fail = [&](const char* what) {
        cleanup();
        cudaGetLastError();
        FAIL(MD_ECUDA, "md_vacf_get: %s failed", what);
    };
    if (cudaMallocAsync(&pad, (size_t)nb * 2 * T * e, ctx->s) != cudaSuccess ||
        cudaMallocAsync(&X, (size_t)nb * nj * 2 * e, ctx->s) != cudaSuccess ||
        cudaMallocAsync((void**)&P, nj * sizeof(double), ctx->s) != cudaSuccess ||
        cudaMallocAsync((void**)&Z, nj * sizeof(double2), ctx->s) != cudaSuccess ||
        cudaMallocAsync((void**)&r, 2 * T * sizeof(double), ctx->s) != cudaSuccess ||
        cudaMallocAsync((void**)&C, n_lags * sizeof(double), ctx->s) != cudaSuccess ||
        cudaMallocAsync((void**)&S, n_lags * sizeof(double), ctx->s) != cudaSuccess)
        return fail("device allocation");
    int len = int(2 * T);
    if (cufftPlanMany(&fw, 1, &len, nullptr, 1, len, nullptr, 1, int(nj), fp64 ? CUFFT_D2Z : CUFFT_R2C, nb) != CUFFT_SUCCESS ||
        cufftPlan1d(&bw, len, CUFFT_Z2D, 1) != CUFFT_SUCCESS ||
        cufftSetStream(fw, ctx->s) != CUFFT_SUCCESS || cufftSetStream(bw, ctx->s) != CUFFT_SUCCESS)
        return fail("cuFFT plan");
    if (cudaMemsetAsync(P, 0, nj * sizeof(double), ctx->s) != cudaSuccess) return fail("memset");
    for (int s0 = s_lo; s0 < s_hi; s0 += nb) {
        const int cnt = std::min(nb, s_hi - s0);
        launch_vacf_gather(ctx->vr, pad, fp64, T, n3, s0, cnt, ctx->s);
        const cufftResult fr = fp64 ? cufftExecD2Z(fw, (double*)pad, (cufftDoubleComplex*)X)
                                    : cufftExecR2C(fw, (float*)pad, (cufftComplex*)X);
        if (fr != CUFFT_SUCCESS) return fail("forward transform");
        launch_vacf_power(X, fp64, d.mt, s0, cnt, nj, P, ctx->s);
    }
    launch_vacf_to_complex(P, Z, nj, ctx->s);
    if (cufftExecZ2D(bw, (cufftDoubleComplex*)Z, r) != CUFFT_SUCCESS) return fail("inverse transform");
    launch_vacf_finish(r, C, T, n_lags, ctx->s);
    launch_vacf_spectrum(C, S, n_lags, ctx->s);
    if (cudaGetLastError() != cudaSuccess) return fail("kernel launch");
    if ((vacf_out && cudaMemcpyAsync(vacf_out, C, n_lags * sizeof(double), cudaMemcpyDeviceToHost, ctx->s) != cudaSuccess) ||
        (spectrum_out && cudaMemcpyAsync(spectrum_out, S, n_lags * sizeof(double), cudaMemcpyDeviceToHost, ctx->s) != cudaSuccess))
        return fail("copy to host");
    const cudaError_t se = cudaStreamSynchronize(ctx->s);
    cleanup();
    if (se != cudaSuccess) FAIL(MD_ECUDA, "md_vacf_get: %s", cudaGetErrorString(se));
    return MD_OK;
}

int md_finalize(md_ctx* ctx)
{
    if (!ctx) return MD_EINVAL;
    if (ctx->gs) cudaStreamSynchronize(ctx->gs);
    drop_graphs(ctx);
    vacf_stop(ctx);
    free_device(ctx);
    cudaStreamSynchronize(ctx->s);
    for (auto& f : ctx->fft) { cufftDestroy(f.d2z); cufftDestroy(f.z2d); }
    if (ctx->gs) cudaStreamDestroy(ctx->gs);
    if (ctx->s2) { cudaStreamSynchronize(ctx->s2); cudaStreamDestroy(ctx->s2); }
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    for (auto& p : ctx->pend) { ctx->ev_pool.push_back(p.a); ctx->ev_pool.push_back(p.b); }
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    cudaFreeHost(ctx->h_stepc);
    cudaFreeHost(ctx->h_err);
    delete ctx;
    return MD_OK;
}

const char* md_last_error(const md_ctx* ctx)
{
    return ctx ? ctx->msg.c_str() : g_init_msg.c_str();
}

}  // extern "C"
