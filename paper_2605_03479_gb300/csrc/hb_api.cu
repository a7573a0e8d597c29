// C ABI of the GB300 HB-UGKS library (declared in include/hbugks.h): workspace layout, case tables, graph
// capture of the pseudo-time iteration, state and field conversions.  All device memory lives in the
// caller's workspace; the library allocates none.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hbugks.h"
#include "hb_kernels.cuh"
#include "hb_cells.cuh"

using namespace hb;

namespace {

#define HB_CK(x)                                             \
    do {                                                     \
        cudaError_t e_ = (x);                                \
        if (e_ != cudaSuccess) {                             \
            last_cuda_error() = e_;                          \
            return HBUGKS_ECUDA;                             \
        }                                                    \
    } while (0)

cudaError_t& last_cuda_error()
{
    static thread_local cudaError_t e = cudaSuccess;
    return e;
}

constexpr int CHUNK = 16;   // iterations per captured graph

// NVTX range (header-only NVTX 3): a tracing tool attached to the process (Nsight Systems, or any library named
// by NVTX_INJECTION64_PATH) sees every call of the C ABI, and every kernel stage that an iteration enqueues, as
// a named range on the calling thread.  With no tool attached a push or pop is one test of a null pointer.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

// timing events destroyed on every return path
struct Events {
    std::vector<cudaEvent_t> ev;
    cudaError_t create(int n)
    {
        ev.assign(n, nullptr);
        for (auto& e : ev) {
            const cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) { e = nullptr; return r; }
        }
        return cudaSuccess;
    }
    ~Events()
    {
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
    }
};

// bump allocator over the workspace; with base == nullptr it only measures
struct Carver {
    char* base;
    size_t off = 0;
    template <class X>
    X* take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        X* p = base ? reinterpret_cast<X*>(base + off) : nullptr;
        off += count * sizeof(X);
        return p;
    }
};

struct HostCase {
    hbugks_case src;
    int nx, ny, nu, nv, nvel, nvb, nvp, nt, nh, nfx, nf, nc;
    std::vector<double> xn, yn, u, wu, v, wv;
    double mu0, omega;
    int nslot;                      // wall-state slots: nt (harmonic balance) or time steps per period
    double dt_fixed;                // > 0: time-domain mode, the global physical step
    std::vector<double> wall_tab;   // [4][nslot][3]
    // stored velocity order: sign classes 0 (u > 0, v > 0), 1 (u < 0, v > 0), 2 (u > 0, v < 0), 3 (u < 0, v < 0),
    // each padded to whole blocks; per slot the canonical index jv * nu + iu (-1: padding) and the share of the
    // node's weight (1/2 or 1/4 for a node with u = 0 or v = 0, stored in two or four classes)
    std::vector<int> vcan, vcls;
    std::vector<double> vfac;
    int k1b, k2b, k3b, k4b, ksb, ktb;
    int k4shape;
    int k1sep;                      // face sums by v-moments: no zero node, every sign class 1..32 u-nodes wide
    int pairs;                      // every sign class holds an even number of velocity blocks
};

// K1 tile (TX x TY cells, one warp each) and velocity blocks staged per pass, per storage precision
template <typename T> constexpr int K1_TX = 4;
template <typename T> constexpr int K1_TY = 2;
template <typename T> constexpr int K1_G = std::is_same<T, float>::value ? 6 : 4;
template <typename T> constexpr int K1_S = 3;   // pipeline stages of the staged velocity blocks

template <typename T>
constexpr size_t k1_smem_of()
{
    return k1_cells_smem<T, K1_TX<T>, K1_TY<T>, K1_G<T>, K1_S<T>>();
}
template <typename T, bool SEP>
constexpr auto k1_kernel()
{
    return k1_cells<T, K1_TX<T>, K1_TY<T>, K1_G<T>, K1_S<T>, SEP>;
}

// K4 tile shapes (TX, TY, warps per CTA)
// K4 variants: tile (TX, TY), warps per CTA, velocity blocks per CTA (2: single precision only, and only for
// cases whose sign classes each hold an even number of blocks)
struct Shape {
    int tx, ty, nw, vpl;
};
constexpr Shape K4_SHAPES[] = {{4, 4, 8, 1}, {4, 2, 8, 1}, {2, 2, 4, 1}, {8, 4, 16, 1}, {4, 2, 8, 2}};
constexpr int N_K4_SHAPES = 5;

template <typename T>
size_t k4_smem_of(int shape, int nt)
{
    switch (shape) {
        case 0: return k4_cells_smem<T, 4, 4, 1>(nt);
        case 1: return k4_cells_smem<T, 4, 2, 1>(nt);
        case 2: return k4_cells_smem<T, 2, 2, 1>(nt);
        case 3: return k4_cells_smem<T, 8, 4, 1>(nt);
        default: return k4_cells_smem<T, 4, 2, 2>(nt);
    }
}

constexpr size_t SMEM_MAX = 219 * 1024;   // dynamic shared memory per CTA, leaving room for the static arrays

// largest tile whose shared memory lets two CTAs share an SM, else the largest that fits at all
template <typename T>
int pick_k4_shape(int nt)
{
    for (int s = 0; s < N_K4_SHAPES; ++s)
        if (K4_SHAPES[s].vpl == 1 && k4_smem_of<T>(s, nt) <= 113 * 1024) return s;
    for (int s = 0; s < N_K4_SHAPES; ++s)
        if (K4_SHAPES[s].vpl == 1 && k4_smem_of<T>(s, nt) <= SMEM_MAX) return s;
    return -1;
}

// a K4 variant a case of this precision can run: its shared memory fits a CTA, and two velocity blocks per
// CTA need single precision and sign classes of an even number of blocks (the CTA's blocks share one class)
template <typename T>
bool k4_shape_ok(int shape, int nt, bool pairs)
{
    if (shape < 0 || shape >= N_K4_SHAPES || k4_smem_of<T>(shape, nt) > SMEM_MAX) return false;
    return K4_SHAPES[shape].vpl == 1 || (sizeof(T) == 4 && pairs);
}

// finite and strictly positive
inline bool pos(double x) { return std::isfinite(x) && x > 0; }

bool validate(const hbugks_case& c)
{
    const hbugks_mesh& m = c.mesh;
    const hbugks_vgrid& g = c.vgrid;
    const hbugks_physics& p = c.phys;
    if (m.nx < 1 || m.ny < 1 || !m.xnodes || !m.ynodes) return false;
    if (g.nu < 1 || g.nv < 1 || !g.u || !g.v || !g.wu || !g.wv) return false;
    if (p.n_harmonics < 0 || 2 * p.n_harmonics + 1 > MAXNT) return false;
    if (!pos(p.kn) || !pos(p.cfl) || !(std::isfinite(p.st) && p.st >= 0) || !pos(p.gamma)) return false;
    if (!pos(p.pr) || !std::isfinite(p.w_vss) || !pos(p.alpha_vss) || !pos(g.umax) || !pos(g.vmax)) return false;
    if (p.precision != 0 && p.precision != 1) return false;
    if (p.face_step != 0 && p.face_step != 1) return false;
    if (p.td_steps < 0 || (p.td_steps > 0 && (p.n_harmonics != 0 || !(p.st > 0)))) return false;
    if (p.spectral_implicit != 0 && p.spectral_implicit != 1) return false;
    // the kernels index the per-face and per-cell expm1 tables ([nf][nt][nu + nv], [nc][nt][2][nu + nv]) and a
    // cell's 32-lane rows with 32-bit element offsets
    {
        const long long nc = (long long)m.nx * m.ny, nt = 2LL * p.n_harmonics + 1, nuv = (long long)g.nu + g.nv;
        const long long nf = (long long)m.ny * (m.nx + 1) + (long long)(m.ny + 1) * m.nx;
        if (nf * nt * nuv > INT_MAX || nc * nt * 2 * nuv > INT_MAX || nc * VB > INT_MAX) return false;
    }
    if (!std::isfinite(m.xnodes[0]) || !std::isfinite(m.ynodes[0])) return false;
    for (int i = 0; i < m.nx; ++i) if (!(m.xnodes[i + 1] > m.xnodes[i]) || !std::isfinite(m.xnodes[i + 1])) return false;
    for (int j = 0; j < m.ny; ++j) if (!(m.ynodes[j + 1] > m.ynodes[j]) || !std::isfinite(m.ynodes[j + 1])) return false;
    for (int i = 0; i < g.nu; ++i) if (!pos(g.wu[i]) || !std::isfinite(g.u[i])) return false;
    for (int j = 0; j < g.nv; ++j) if (!pos(g.wv[j]) || !std::isfinite(g.v[j])) return false;
    const int nslot = p.td_steps > 0 ? p.td_steps : 2 * p.n_harmonics + 1;
    for (int w = 0; w < 4; ++w) {
        const hbugks_wall& wl = c.walls[w];
        const double vals[9] = {wl.u_mean, wl.v_mean, wl.T_mean, wl.u_re, wl.u_im, wl.v_re, wl.v_im, wl.T_re, wl.T_im};
        for (double x : vals) if (!std::isfinite(x)) return false;
        for (int n = 0; n < nslot; ++n) {
            double th = p.td_steps > 0 ? 2.0 * M_PI * (n + 0.5) / nslot : 2.0 * M_PI * n / nslot;
            if (!(wl.T_mean + wl.T_re * cos(th) - wl.T_im * sin(th) > 0)) return false;
        }
    }
    return true;
}

void fill_host(HostCase& h, const hbugks_case& c)
{
    h.src = c;
    h.nx = c.mesh.nx; h.ny = c.mesh.ny; h.nu = c.vgrid.nu; h.nv = c.vgrid.nv;
    h.nvel = h.nu * h.nv;
    h.vcan.clear(); h.vcls.clear(); h.vfac.clear();
    for (int cls = 0; cls < 4; ++cls) {
        const size_t first = h.vcan.size();
        for (int jv = 0; jv < h.nv; ++jv)
            for (int iu = 0; iu < h.nu; ++iu) {
                const double uu = c.vgrid.u[iu], vv = c.vgrid.v[jv];
                if ((cls & 1) ? uu > 0 : uu < 0) continue;
                if ((cls & 2) ? vv > 0 : vv < 0) continue;
                h.vcan.push_back(jv * h.nu + iu);
                h.vfac.push_back((uu == 0 ? 0.5 : 1.0) * (vv == 0 ? 0.5 : 1.0));
            }
        while ((h.vcan.size() - first) % VB) { h.vcan.push_back(-1); h.vfac.push_back(0.0); }
        for (size_t k = first; k < h.vcan.size(); k += VB) h.vcls.push_back(cls);
    }
    h.nvp = (int)h.vcan.size();
    h.nvb = h.nvp / VB;
    {
        int cnt[4] = {0, 0, 0, 0};
        for (int c : h.vcls) ++cnt[c];
        h.pairs = cnt[0] % 2 == 0 && cnt[1] % 2 == 0 && cnt[2] % 2 == 0 && cnt[3] % 2 == 0;
    }
    {
        int upos = 0, uneg = 0, zero = 0;
        for (int iu = 0; iu < h.nu; ++iu) {
            const double uu = c.vgrid.u[iu];
            upos += uu > 0; uneg += uu < 0; zero += uu == 0;
        }
        for (int jv = 0; jv < h.nv; ++jv) zero += c.vgrid.v[jv] == 0;
        // in a class of k u-nodes with k dividing 32, lane l of every block holds u-node l mod k
        h.k1sep = !zero && upos > 0 && uneg > 0 && 32 % upos == 0 && 32 % uneg == 0;
    }
    h.nh = c.phys.n_harmonics;
    h.nt = 2 * h.nh + 1;
    h.nfx = h.ny * (h.nx + 1);
    h.nf = h.nfx + (h.ny + 1) * h.nx;
    h.nc = h.nx * h.ny;
    h.xn.assign(c.mesh.xnodes, c.mesh.xnodes + h.nx + 1);
    h.yn.assign(c.mesh.ynodes, c.mesh.ynodes + h.ny + 1);
    h.u.assign(c.vgrid.u, c.vgrid.u + h.nu);
    h.wu.assign(c.vgrid.wu, c.vgrid.wu + h.nu);
    h.v.assign(c.vgrid.v, c.vgrid.v + h.nv);
    h.wv.assign(c.vgrid.wv, c.vgrid.wv + h.nv);
    // Eq. def_Kn with H = rho0 = 1, sqrt(2 R T0) = 1:  mu(T0) = Kn sqrt(pi) / F(alpha, w)
    const double a = c.phys.alpha_vss, w = c.phys.w_vss;
    const double F = 4.0 * a * (5.0 - 2.0 * w) * (7.0 - 2.0 * w) / (5.0 * (a + 1.0) * (a + 2.0));
    h.mu0 = c.phys.kn * sqrt(M_PI) / F;
    h.omega = c.phys.st;   // Eq. def_St with H = 1, sqrt(2 R T0) = 1
    // wall states per level (Eqs. bc_vel, bc_temp at t_n = nT/N_T), or, in time-domain mode, per step of a
    // period at the step's midpoint
    const bool td = c.phys.td_steps > 0;
    h.nslot = td ? c.phys.td_steps : h.nt;
    h.dt_fixed = td ? 2.0 * M_PI / (h.omega * c.phys.td_steps) : 0.0;
    h.wall_tab.assign(4 * h.nslot * 3, 0.0);
    for (int wl = 0; wl < 4; ++wl)
        for (int n = 0; n < h.nslot; ++n) {
            const hbugks_wall& W = h.src.walls[wl];
            double th = td ? 2.0 * M_PI * (n + 0.5) / h.nslot : 2.0 * M_PI * n / h.nt;
            double cs = cos(th), sn = sin(th);
            double* o = &h.wall_tab[(wl * h.nslot + n) * 3];
            o[0] = W.u_mean + W.u_re * cs - W.u_im * sn;   // Eq. bc_vel
            o[1] = W.v_mean + W.v_re * cs - W.v_im * sn;
            o[2] = W.T_mean + W.T_re * cs - W.T_im * sn;   // Eq. bc_temp
        }
    h.k2b = (h.nf * h.nt + 127) / 128;
    h.k3b = (h.nc + K3_THREADS - 1) / K3_THREADS;
    h.ksb = (h.nc + 127) / 128;
    h.ktb = (h.nc * h.nt + KT_ITEMS - 1) / KT_ITEMS;
}

template <typename T>
void layout_case(Carver& cv, const HostCase& h, CaseDev<T>& d)
{
    d.nx = h.nx; d.ny = h.ny; d.nu = h.nu; d.nv = h.nv; d.nvel = h.nvel; d.nvb = h.nvb;
    for (int c = 0, e = 0; c < 4; ++c) {
        for (int cl : h.vcls) e += cl == c;
        d.cls_end[c] = e;
    }
    d.nt = h.nt; d.nh = h.nh; d.nfx = h.nfx; d.nf = h.nf; d.nc = h.nc;
    d.face_step = h.src.phys.face_step;
    d.omega = h.omega; d.mu0 = h.mu0; d.w_vss = h.src.phys.w_vss; d.pr = h.src.phys.pr;
    d.cfl = h.src.phys.cfl; d.gam = h.src.phys.gamma; d.umax = h.src.vgrid.umax; d.vmax = h.src.vgrid.vmax;
    d.lam0 = 1.0;
    for (int k = 0; k < 8; ++k) d.e[k] = 0.0;
    for (int dd = 1; dd <= h.nh; ++dd) d.e[dd] = ((dd & 1) ? -0.5 : 0.5) / sin(M_PI * dd / h.nt);   // Eq. D_explicit
    for (int k = 0; k < 8; ++k) d.et[k] = T(d.e[k]);
    d.spectral_implicit = h.src.phys.spectral_implicit;
    d.minv = cv.take<T>((size_t)h.nc * h.nt * h.nt);
    d.nslot = h.nslot;
    d.dt_fixed = h.dt_fixed;
    d.wall = cv.take<double>((size_t)4 * h.nslot * 3);
    d.xn = cv.take<double>(h.nx + 1); d.yn = cv.take<double>(h.ny + 1);
    d.xc = cv.take<double>(h.nx); d.yc = cv.take<double>(h.ny);
    d.hx = cv.take<double>(h.nx); d.hy = cv.take<double>(h.ny);
    d.rdx = cv.take<double>(h.nx); d.rdy = cv.take<double>(h.ny);
    d.vu = cv.take<double>(h.nvp); d.vv = cv.take<double>(h.nvp); d.vw = cv.take<double>(h.nvp);
    d.tu = cv.take<T>(h.nvp); d.tv = cv.take<T>(h.nvp); d.tw = cv.take<T>(h.nvp); d.thref = cv.take<T>(h.nvp);
    d.twu = cv.take<T>(h.nvp); d.twv = cv.take<T>(h.nvp);
    d.u1 = cv.take<double>(h.nu); d.wu1 = cv.take<double>(h.nu);
    d.v1 = cv.take<double>(h.nv); d.wv1 = cv.take<double>(h.nv);
    d.tu1 = cv.take<T>(h.nu); d.tv1 = cv.take<T>(h.nv);
    d.refmom = cv.take<double>(5 * 13);
    const size_t ns = (size_t)h.nvb * h.nc * h.nt * VB;
    for (int k = 0; k < 2; ++k) {
        d.f[k] = cv.take<P2<T>>(ns);
        d.W[k] = cv.take<double>((size_t)h.nt * h.nc * 4);
    }
    d.dG = cv.take<double>(h.nc);
    d.hmom = cv.take<double>((size_t)h.nc * h.nt * 4 * NM);
    d.cmom = cv.take<double>((size_t)h.nc * h.nt * NCM);
    d.fpar = cv.take<T>((size_t)h.nf * h.nt * NP);
    d.ftab = cv.take<T>((size_t)h.nf * h.nt * (h.nu + h.nv));
    d.wtab = cv.take<T>((size_t)4 * h.nslot * (h.nu + h.nv));
    d.wxr = cv.take<T>((size_t)9 * h.nu);
    d.wyr = cv.take<T>((size_t)9 * h.nv);
    d.xr0 = cv.take<double>(36);
    d.yr0 = cv.take<double>(36);
    d.xr0t = cv.take<T>(36);
    d.yr0t = cv.take<T>(36);
    d.wconst = cv.take<double>((size_t)4 * h.nslot * WCN);
    d.oconst = cv.take<double>(32);
    d.ctab = cv.take<T>((size_t)h.nc * h.nt * 2 * (h.nu + h.nv));
    d.viu = cv.take<int>(h.nvp);
    d.viv = cv.take<int>(h.nvp);
    d.vcan = cv.take<int>(h.nvp);
    d.vcls = cv.take<int>(h.nvb);
    d.shakhov = h.src.phys.pr != 1.0;
    d.fflux = cv.take<double>((size_t)h.nf * h.nt * 4);
    d.cpar = cv.take<T>((size_t)h.nc * h.nt * NCP);
    d.rpart = cv.take<double>((size_t)h.k3b * 4);
    d.rhist = cv.take<double>((size_t)RING * 4);
    size_t stage = std::max((size_t)h.nc * h.nvp, (size_t)(h.nt * 8 + 16) * h.nc);
    d.stage = cv.take<double>(stage);
}

}  // namespace

// ====================================================================================== solver

// one kernel launch of the iteration covering every case it applies to
struct LaunchSpec {
    int kind;      // 0 K1 tile, 1 K2, 2 K3, 3 tables, 4 K4 tile, 5 steps
    int shape;     // tile shape index (K1, K4)
    int table;     // block offset table index
    int total;     // total blocks
    size_t smem;   // dynamic shared memory bytes
};

template <typename T>
struct Impl {
    std::vector<HostCase> hc;
    std::vector<CaseDev<T>> dc;
    CaseDev<T>* d_cases = nullptr;
    CaseStatus* d_status = nullptr;
    double* d_tol = nullptr;
    int* d_err = nullptr;            // [0] error word (a bounded wait expired), [1] test hook: expire the next wait
    int* d_loop = nullptr;           // iterations left in the device-side loop of the current call
    int* d_off = nullptr;            // [table][ncases + 1]
    int* d_tune_off = nullptr;       // block offsets of a single-case launch (autotuning)
    std::vector<int> off_host;
    std::vector<LaunchSpec> specs;   // in launch order (without the residual kernel)
    int k3_table = 0, steps_table = 0;
    bool any_implicit = false;       // some case takes the spectral source at the new iterate
};

struct hbugks_solver {
    int ncases = 0;
    int precision = 0;
    cudaStream_t user = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t g1 = nullptr, gN = nullptr;
    cudaGraphExec_t gW = nullptr;     // device-side loop: a while node over one iteration and the loop test
    int loop_mode = 0;                // 0: device-side loop (gW), 1: host-polled graphs of CHUNK iterations
    char* ws = nullptr;
    size_t bytes = 0;
    Impl<float>* f = nullptr;
    Impl<double>* d = nullptr;
    double tol_host = 0.0;
    std::vector<CaseStatus> st_host;
};

namespace {

template <typename T>
void fill_offsets(Impl<T>& im, int ncases);

void set_k4_blocks(HostCase& h)
{
    if (h.k4shape < 0) { h.k4b = 0; return; }
    const Shape s4 = K4_SHAPES[h.k4shape];
    h.k4b = ((h.nx + s4.tx - 1) / s4.tx) * ((h.ny + s4.ty - 1) / s4.ty) * (h.nvb / s4.vpl);
}

template <typename T>
size_t plan(Impl<T>& im, int ncases, const hbugks_case* cases, char* base)
{
    Carver cv{base};
    im.hc.resize(ncases);
    im.dc.resize(ncases);
    for (int k = 0; k < ncases; ++k) {
        HostCase& h = im.hc[k];
        fill_host(h, cases[k]);
        h.k4shape = pick_k4_shape<T>(h.nt);
        h.k1b = ((h.nx + K1_TX<T> - 1) / K1_TX<T>) * ((h.ny + K1_TY<T> - 1) / K1_TY<T>) * h.nt;
        set_k4_blocks(h);
    }
    im.d_cases = cv.take<CaseDev<T>>(ncases);
    im.d_status = cv.take<CaseStatus>(ncases);
    im.d_tol = cv.take<double>(1);
    im.d_err = cv.take<int>(2);
    im.d_loop = cv.take<int>(2);
    im.d_tune_off = cv.take<int>(2);
    // launch specs: K1 per shape, K2, K3, tables, K4 per shape; plus the step kernel (state setting only)
    im.specs.clear();
    auto add = [&](int kind, int shape) { im.specs.push_back(LaunchSpec{kind, shape, (int)im.specs.size(), 0, 0}); };
    add(0, 0);
    add(0, 1);
    add(1, 0);
    add(2, 0);
    im.k3_table = (int)im.specs.size() - 1;
    add(3, 0);
    for (int sh = 0; sh < N_K4_SHAPES; ++sh) add(4, sh);
    add(5, 0);
    im.steps_table = (int)im.specs.size() - 1;
    const int ntab = (int)im.specs.size();
    im.d_off = cv.take<int>((size_t)ntab * (ncases + 1));
    for (int k = 0; k < ncases; ++k) {
        layout_case(cv, im.hc[k], im.dc[k]);
        im.dc[k].st = im.d_status + k;
        im.dc[k].tol = im.d_tol;
        im.dc[k].err = im.d_err;
        im.dc[k].expire = im.d_err + 1;
    }
    fill_offsets(im, ncases);
    return cv.off + 256;
}

// block offset tables of every launch from the cases' block counts and K4 shapes
template <typename T>
void fill_offsets(Impl<T>& im, int ncases)
{
    const int ntab = (int)im.specs.size();
    im.off_host.assign((size_t)ntab * (ncases + 1), 0);
    for (auto& sp : im.specs) {
        int acc = 0;
        size_t smem = 0;
        for (int k = 0; k < ncases; ++k) {
            im.off_host[(size_t)sp.table * (ncases + 1) + k] = acc;
            const HostCase& h = im.hc[k];
            int nb = 0;
            switch (sp.kind) {
                case 0: nb = h.k1sep == sp.shape ? h.k1b : 0; smem = k1_smem_of<T>(); break;
                case 1: nb = h.k2b; break;
                case 2: nb = h.k3b; break;
                case 3: nb = h.ktb; break;
                case 4: if (h.k4shape == sp.shape) { nb = h.k4b; smem = std::max(smem, k4_smem_of<T>(sp.shape, h.nt)); } break;
                case 5: nb = h.ksb; break;
            }
            acc += nb;
        }
        im.off_host[(size_t)sp.table * (ncases + 1) + ncases] = acc;
        sp.total = acc;
        sp.smem = smem;
    }
}

// Constants of the diffuse walls, FP64 on the host (they depend only on the wall waveforms):
//   wconst[w][n]: raw moments of the unit-density wall Maxwellian H_w (and B_w = H_w / (2 lam_w)) over the
//                 reflected velocities (13), sum_refl w |u_n| H_w, and the reflected flux moments of (H_w, B_w) (4);
//   oconst[w]:    incident and reflected flux moments of (H_ref, B_ref);
//   wtab[w][n]:   expm1(lam0 x^2 - lam_w (x - U_w)^2) over the 1-D nodes (separable wall Maxwellian).
template <typename T>
void wall_constants(const HostCase& h, std::vector<double>& wconst, std::vector<double>& oconst, std::vector<T>& wtab)
{
    const int nt = h.nslot, nuv = h.nu + h.nv;      // one set per wall-state slot
    wconst.assign((size_t)4 * nt * WCN, 0.0);
    oconst.assign(32, 0.0);
    wtab.assign((size_t)4 * nt * nuv, T(0));
    for (int wl = 0; wl < 4; ++wl) {
        const int ax = (wl == 1 || wl == 3) ? 0 : 1;        // right/left walls are x-normal
        const double nin = (wl == 0 || wl == 3) ? 1.0 : -1.0;
        for (int n = 0; n < nt; ++n) {
            const double* ws = &h.wall_tab[(wl * nt + n) * 3];
            const double Uw = ws[0], Vw = ws[1], lamw = 1.0 / ws[2];
            double* o = &wconst[((size_t)wl * nt + n) * WCN];
            for (int jv = 0; jv < h.nv; ++jv)
                for (int iu = 0; iu < h.nu; ++iu) {
                    const double u = h.u[iu], v = h.v[jv], w = h.wu[iu] * h.wv[jv];
                    const double un = ax == 0 ? u : v;
                    if (!(un * nin > 0)) continue;
                    const double H = lamw / M_PI * exp(-lamw * ((u - Uw) * (u - Uw) + (v - Vw) * (v - Vw)));
                    const double B = H * 0.5 / lamw;
                    const double m[13] = {H, u * H, v * H, u * u * H, u * v * H, v * v * H, u * u * u * H,
                                          u * u * v * H, u * v * v * H, v * v * v * H, B, u * B, v * B};
                    for (int k = 0; k < 13; ++k) o[k] += w * m[k];
                    o[13] += w * fabs(un) * H;
                    o[14] += w * un * H;
                    o[15] += w * un * u * H;
                    o[16] += w * un * v * H;
                    o[17] += w * un * 0.5 * ((u * u + v * v) * H + B);
                }
            T* tb = &wtab[((size_t)wl * nt + n) * nuv];
            for (int k = 0; k < h.nu; ++k) tb[k] = T(expm1(h.u[k] * h.u[k] - lamw * (h.u[k] - Uw) * (h.u[k] - Uw)));
            for (int k = 0; k < h.nv; ++k) tb[h.nu + k] = T(expm1(h.v[k] * h.v[k] - lamw * (h.v[k] - Vw) * (h.v[k] - Vw)));
        }
        double* oc = &oconst[wl * 8];
        for (int jv = 0; jv < h.nv; ++jv)
            for (int iu = 0; iu < h.nu; ++iu) {
                const double u = h.u[iu], v = h.v[jv], w = h.wu[iu] * h.wv[jv];
                const double un = ax == 0 ? u : v;
                const double H = (1.0 / M_PI) * exp(-(u * u + v * v)), B = 0.5 * H;
                const double f[4] = {un * H, un * u * H, un * v * H, un * 0.5 * ((u * u + v * v) * H + B)};
                const int o = un * nin < 0 ? 0 : (un * nin > 0 ? 4 : -1);
                if (o < 0) continue;
                for (int k = 0; k < 4; ++k) oc[o + k] += w * f[k];
            }
    }
}

// host tables of one case uploaded into the workspace
template <typename T>
cudaError_t upload_case(const HostCase& h, const CaseDev<T>& d, cudaStream_t s, std::vector<std::vector<char>>& keep)
{
    auto put = [&](const void* dst, const void* src, size_t n) -> cudaError_t {
        keep.emplace_back((const char*)src, (const char*)src + n);
        return cudaMemcpyAsync(const_cast<void*>(dst), keep.back().data(), n, cudaMemcpyHostToDevice, s);
    };
    cudaError_t e;
    std::vector<double> xc(h.nx), yc(h.ny), hx(h.nx), hy(h.ny), rdx(h.nx, 0.0), rdy(h.ny, 0.0);
    for (int i = 0; i < h.nx; ++i) { xc[i] = 0.5 * (h.xn[i] + h.xn[i + 1]); hx[i] = 0.5 * (h.xn[i + 1] - h.xn[i]); }
    for (int j = 0; j < h.ny; ++j) { yc[j] = 0.5 * (h.yn[j] + h.yn[j + 1]); hy[j] = 0.5 * (h.yn[j + 1] - h.yn[j]); }
    for (int i = 0; i + 1 < h.nx; ++i) rdx[i] = 1.0 / (xc[i + 1] - xc[i]);
    for (int j = 0; j + 1 < h.ny; ++j) rdy[j] = 1.0 / (yc[j + 1] - yc[j]);
    std::vector<double> vu(h.nvp, 0.0), vv(h.nvp, 0.0), vw(h.nvp, 0.0);
    std::vector<T> tu(h.nvp, T(0)), tv(h.nvp, T(0)), tw(h.nvp, T(0)), th(h.nvp, T(0)), twu(h.nvp, T(0)),
        twv(h.nvp, T(0));
    double ref[5][13];
    memset(ref, 0, sizeof ref);
    std::vector<int> iu_(h.nvp, 0), iv_(h.nvp, 0);
    for (int a = 0; a < h.nvp; ++a) {
        const int can = h.vcan[a];
        if (can < 0) continue;             // padding: zero velocity, weight and reference
        const int iu = can % h.nu, jv = can / h.nu;
        const double u = h.u[iu], v = h.v[jv], w = h.wu[iu] * h.wv[jv] * h.vfac[a];
        vu[a] = u; vv[a] = v; vw[a] = w;
        tu[a] = T(u); tv[a] = T(v); tw[a] = T(w); th[a] = T((1.0 / M_PI) * exp(-(u * u + v * v)));
        twu[a] = T(h.wu[iu]); twv[a] = T(h.wv[jv] * h.vfac[a]);
        iu_[a] = iu; iv_[a] = jv;
    }
    for (int jv = 0; jv < h.nv; ++jv)
        for (int iu = 0; iu < h.nu; ++iu) {
            double u = h.u[iu], v = h.v[jv], w = h.wu[iu] * h.wv[jv];
            double href = (1.0 / M_PI) * exp(-(u * u + v * v));
            double bref = 0.5 * href;
            double m[13] = {href, u * href, v * href, u * u * href, u * v * href, v * v * href, u * u * u * href,
                            u * u * v * href, u * v * v * href, v * v * v * href, bref, u * bref, v * bref};
            bool in[5] = {true, u > 0, u < 0, v > 0, v < 0};
            for (int s5 = 0; s5 < 5; ++s5)
                if (in[s5])
                    for (int k = 0; k < 13; ++k) ref[s5][k] += w * m[k];
        }
    if ((e = put(d.wall, h.wall_tab.data(), sizeof(double) * h.wall_tab.size()))) return e;
    if ((e = put(d.xn, h.xn.data(), sizeof(double) * h.xn.size()))) return e;
    if ((e = put(d.yn, h.yn.data(), sizeof(double) * h.yn.size()))) return e;
    if ((e = put(d.xc, xc.data(), sizeof(double) * h.nx))) return e;
    if ((e = put(d.yc, yc.data(), sizeof(double) * h.ny))) return e;
    if ((e = put(d.hx, hx.data(), sizeof(double) * h.nx))) return e;
    if ((e = put(d.hy, hy.data(), sizeof(double) * h.ny))) return e;
    if ((e = put(d.rdx, rdx.data(), sizeof(double) * h.nx))) return e;
    if ((e = put(d.rdy, rdy.data(), sizeof(double) * h.ny))) return e;
    if ((e = put(d.vu, vu.data(), sizeof(double) * h.nvp))) return e;
    if ((e = put(d.vv, vv.data(), sizeof(double) * h.nvp))) return e;
    if ((e = put(d.vw, vw.data(), sizeof(double) * h.nvp))) return e;
    if ((e = put(d.tu, tu.data(), sizeof(T) * h.nvp))) return e;
    if ((e = put(d.tv, tv.data(), sizeof(T) * h.nvp))) return e;
    if ((e = put(d.tw, tw.data(), sizeof(T) * h.nvp))) return e;
    if ((e = put(d.thref, th.data(), sizeof(T) * h.nvp))) return e;
    if ((e = put(d.twu, twu.data(), sizeof(T) * h.nvp))) return e;
    if ((e = put(d.twv, twv.data(), sizeof(T) * h.nvp))) return e;
    if ((e = put(d.u1, h.u.data(), sizeof(double) * h.nu))) return e;
    if ((e = put(d.wu1, h.wu.data(), sizeof(double) * h.nu))) return e;
    if ((e = put(d.v1, h.v.data(), sizeof(double) * h.nv))) return e;
    if ((e = put(d.wv1, h.wv.data(), sizeof(double) * h.nv))) return e;
    if ((e = put(d.refmom, &ref[0][0], sizeof ref))) return e;
    // reference 1-D sums w x^p exp(-lam0 x^2) per node and over node subsets (all, positive, negative, zero)
    std::vector<T> wxr((size_t)9 * h.nu), wyr((size_t)9 * h.nv);
    std::vector<double> xr0(36, 0.0), yr0(36, 0.0);
    std::vector<T> xr0t(36), yr0t(36);
    for (int k = 0; k < h.nu; ++k) {
        const double x = h.u[k], g = h.wu[k] * exp(-x * x);
        const int row = x > 0 ? 1 : (x < 0 ? 2 : 3);
        double pw = g;
        for (int q = 0; q < 9; ++q) { wxr[(size_t)q * h.nu + k] = T(pw); xr0[row * 9 + q] += pw; xr0[q] += pw; pw *= x; }
    }
    for (int k = 0; k < h.nv; ++k) {
        const double y = h.v[k], g = h.wv[k] * exp(-y * y);
        const int row = y > 0 ? 1 : (y < 0 ? 2 : 3);
        double pw = g;
        for (int q = 0; q < 9; ++q) { wyr[(size_t)q * h.nv + k] = T(pw); yr0[row * 9 + q] += pw; yr0[q] += pw; pw *= y; }
    }
    for (int k = 0; k < 36; ++k) { xr0t[k] = T(xr0[k]); yr0t[k] = T(yr0[k]); }
    if ((e = put(d.wxr, wxr.data(), sizeof(T) * wxr.size()))) return e;
    if ((e = put(d.wyr, wyr.data(), sizeof(T) * wyr.size()))) return e;
    if ((e = put(d.xr0, xr0.data(), sizeof(double) * 36))) return e;
    if ((e = put(d.yr0, yr0.data(), sizeof(double) * 36))) return e;
    if ((e = put(d.xr0t, xr0t.data(), sizeof(T) * 36))) return e;
    if ((e = put(d.yr0t, yr0t.data(), sizeof(T) * 36))) return e;
    {
        std::vector<double> wconst, oconst;
        std::vector<T> wtab;
        wall_constants<T>(h, wconst, oconst, wtab);
        if ((e = put(d.wconst, wconst.data(), sizeof(double) * wconst.size()))) return e;
        if ((e = put(d.oconst, oconst.data(), sizeof(double) * oconst.size()))) return e;
        if ((e = put(d.wtab, wtab.data(), sizeof(T) * wtab.size()))) return e;
    }
    std::vector<T> tu1(h.nu), tv1(h.nv);
    for (int i = 0; i < h.nu; ++i) tu1[i] = T(h.u[i]);
    for (int j = 0; j < h.nv; ++j) tv1[j] = T(h.v[j]);
    if ((e = put(d.tu1, tu1.data(), sizeof(T) * h.nu))) return e;
    if ((e = put(d.tv1, tv1.data(), sizeof(T) * h.nv))) return e;
    if ((e = put(d.viu, iu_.data(), sizeof(int) * h.nvp))) return e;
    if ((e = put(d.viv, iv_.data(), sizeof(int) * h.nvp))) return e;
    if ((e = put(d.vcan, h.vcan.data(), sizeof(int) * h.nvp))) return e;
    if ((e = put(d.vcls, h.vcls.data(), sizeof(int) * h.nvb))) return e;
    return cudaSuccess;
}

__global__ void k_status_reset(CaseStatus* st, int ncases, int which, int user_active)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncases || (which >= 0 && k != which)) return;
    st[k].active = 0;
    st[k].parity = 0;
    st[k].diverged = 0;
    st[k].iters = 0;
    st[k].iters_call = 0;
    if (user_active >= 0) st[k].user_active = user_active;
    for (int q = 0; q < 4; ++q) st[k].last[q] = 0.0;
}

__global__ void k_begin_call(CaseStatus* st, int ncases)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncases) return;
    st[k].active = st[k].user_active && !st[k].diverged;
    st[k].iters_call = 0;
}

__global__ void k_set_int(int* p, int v) { *p = v; }

// End of one pass of the device-side loop: one iteration fewer left; the loop goes on while iterations are left,
// some case is still iterating (not converged, not diverged) and no device wait has failed.  Every pass
// decrements the count, so the loop ends after at most the requested number of iterations.
__global__ void k_loop_test(cudaGraphConditionalHandle hc, int* left, const CaseStatus* st, int ncases, const int* err)
{
    if (threadIdx.x != 0) return;
    const int r = *left - 1;
    *left = r;
    int any = 0;
    for (int k = 0; k < ncases; ++k) any |= st[k].active;
    cudaGraphSetConditional(hc, (r > 0 && any && *(volatile const int*)err == 0) ? 1u : 0u);
}

// state of one case copied between handles of possibly different precision (same grid and velocity layout)
template <typename TS, typename TD>
__global__ void k_convert_state(const P2<TS>* src, P2<TD>* dst, size_t n)
{
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const P2<TS> a = src[k];
    dst[k] = pk(TD(a.x), TD(a.y));
}

template <typename T>
void launch_k1(int shape, int total, size_t smem, Batch<T> b, cudaStream_t s)
{
    if (shape == 1) k1_kernel<T, true>()<<<total, K1_TX<T> * K1_TY<T> * 32, smem, s>>>(b);
    else k1_kernel<T, false>()<<<total, K1_TX<T> * K1_TY<T> * 32, smem, s>>>(b);
}

template <typename T, bool IMP>
void launch_k4_(int shape, int total, size_t smem, Batch<T> b, cudaStream_t s)
{
    switch (shape) {
        case 0: k4_cells<T, 4, 4, 8, IMP, 1><<<total, 8 * 32, smem, s>>>(b); break;
        case 1: k4_cells<T, 4, 2, 8, IMP, 1><<<total, 8 * 32, smem, s>>>(b); break;
        case 2: k4_cells<T, 2, 2, 4, IMP, 1><<<total, 4 * 32, smem, s>>>(b); break;
        case 3: k4_cells<T, 8, 4, 16, IMP, 1><<<total, 16 * 32, smem, s>>>(b); break;
        default:
            if constexpr (sizeof(T) == 4) k4_cells<T, 4, 2, 8, IMP, 2><<<total, 8 * 32, smem, s>>>(b);
            break;
    }
}

// the explicit-only kernels unless a case of the handle takes the spectral source at the new iterate
template <typename T>
void launch_k4(bool imp, int shape, int total, size_t smem, Batch<T> b, cudaStream_t s)
{
    if (imp) launch_k4_<T, true>(shape, total, smem, b, s);
    else launch_k4_<T, false>(shape, total, smem, b, s);
}

// every K4 shape may be chosen later (autotuning), so each gets the largest dynamic shared memory it can use
template <typename T>
cudaError_t set_smem_attributes()
{
    const int big = (int)SMEM_MAX;
    cudaError_t e = cudaFuncSetAttribute(k1_kernel<T, false>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)k1_smem_of<T>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k1_kernel<T, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)k1_smem_of<T>());
    auto set = [&](auto k) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    };
    set(k4_cells<T, 4, 4, 8, false, 1>); set(k4_cells<T, 4, 2, 8, false, 1>);
    set(k4_cells<T, 2, 2, 4, false, 1>); set(k4_cells<T, 8, 4, 16, false, 1>);
    set(k4_cells<T, 4, 4, 8, true, 1>); set(k4_cells<T, 4, 2, 8, true, 1>);
    set(k4_cells<T, 2, 2, 4, true, 1>); set(k4_cells<T, 8, 4, 16, true, 1>);
    if constexpr (sizeof(T) == 4) {
        set(k4_cells<T, 4, 2, 8, false, 2>);
        set(k4_cells<T, 4, 2, 8, true, 2>);
    }
    return e;
}

// Kernel kinds reported by the profiler: 0 face moments, 1 face parameters, 2 macro update (with the
// equilibrium tables), 3 micro update, 4 residual.
inline int profile_slot(int kind) { return kind == 0 ? 0 : kind == 1 ? 1 : (kind == 2 || kind == 3) ? 2 : 3; }

// one iteration; with `ev` (2 events per kernel kind, 5 kinds) each kind is bracketed by an event pair
template <typename T>
void enqueue_iteration(Impl<T>& im, int ncases, cudaStream_t s, cudaEvent_t* ev = nullptr)
{
    const int stride = ncases + 1;
    int open_slot = -1;
    for (auto& sp : im.specs) {
        if (sp.kind == 5 || sp.total == 0) continue;
        const int slot = profile_slot(sp.kind);
        if (ev && slot != open_slot) {
            if (open_slot >= 0) cudaEventRecord(ev[2 * open_slot + 1], s);
            cudaEventRecord(ev[2 * slot], s);
            open_slot = slot;
        }
        Batch<T> b{im.d_cases, ncases, im.d_off + (size_t)sp.table * stride};
        static const char* const names[5] = {"k1_cells", "k2_face_params", "k3_macro", "k_tables", "k4_cells"};
        Range r(names[sp.kind]);
        switch (sp.kind) {
            case 0: launch_k1<T>(sp.shape, sp.total, sp.smem, b, s); break;
            case 1: k2_face_params<T><<<sp.total, 128, 0, s>>>(b); break;
            case 2: k3_macro<T><<<sp.total, K3_THREADS, 0, s>>>(b); break;
            case 3: k_tables<T><<<sp.total, KT_ITEMS, 0, s>>>(b); break;
            case 4: launch_k4<T>(im.any_implicit, sp.shape, sp.total, sp.smem, b, s); break;
        }
    }
    if (ev) {
        cudaEventRecord(ev[2 * open_slot + 1], s);
        cudaEventRecord(ev[8], s);
    }
    {
        Range r("k5_finish");
        k5_finish<T><<<ncases, 32, 0, s>>>(im.d_cases, ncases, im.d_off + (size_t)im.k3_table * stride);
    }
    if (ev) cudaEventRecord(ev[9], s);
}

template <typename T>
void enqueue_steps(Impl<T>& im, int ncases, cudaStream_t s)
{
    const LaunchSpec& sp = im.specs[im.steps_table];
    if (sp.total) k_steps<T><<<sp.total, 128, 0, s>>>(Batch<T>{im.d_cases, ncases, im.d_off + (size_t)sp.table * (ncases + 1)});
}

hbugks_status begin(hbugks_t h)
{
    HB_CK(cudaEventRecord(h->ev_in, h->user));
    HB_CK(cudaStreamWaitEvent(h->s, h->ev_in, 0));
    return HBUGKS_OK;
}

hbugks_status end(hbugks_t h)
{
    HB_CK(cudaEventRecord(h->ev_out, h->s));
    HB_CK(cudaStreamWaitEvent(h->user, h->ev_out, 0));
    HB_CK(cudaGetLastError());
    return HBUGKS_OK;
}

template <typename T>
hbugks_status capture(hbugks_t h, Impl<T>& im)
{
    for (int which = 0; which < 2; ++which) {
        int n = which == 0 ? 1 : CHUNK;
        cudaGraph_t g;
        HB_CK(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < n; ++k) enqueue_iteration(im, h->ncases, h->s);
        HB_CK(cudaStreamEndCapture(h->s, &g));
        cudaGraphExec_t ex;
        HB_CK(cudaGraphInstantiate(&ex, g, 0));
        cudaGraphDestroy(g);
        (which == 0 ? h->g1 : h->gN) = ex;
    }
    // The pseudo-time loop on the device: a graph holding one conditional while node, whose body is one
    // iteration followed by the loop test; one launch runs up to the requested number of iterations and stops
    // by itself once every case has converged (or diverged, or a wait failed), with no host round trip.
    cudaGraph_t g;
    HB_CK(cudaGraphCreate(&g, 0));
    struct GraphGuard {
        cudaGraph_t g;
        ~GraphGuard() { cudaGraphDestroy(g); }
    } guard{g};
    cudaGraphConditionalHandle hc;
    HB_CK(cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault));
    // the parameter struct holds a union of non-trivial members: zeroed raw storage stands in for a constructor
    alignas(cudaGraphNodeParams) unsigned char np_raw[sizeof(cudaGraphNodeParams)];
    memset(np_raw, 0, sizeof np_raw);
    cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_raw);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hc;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    HB_CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    HB_CK(cudaStreamBeginCaptureToGraph(h->s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    enqueue_iteration(im, h->ncases, h->s);
    k_loop_test<<<1, 32, 0, h->s>>>(hc, im.d_loop, im.d_status, h->ncases, im.d_err);
    HB_CK(cudaStreamEndCapture(h->s, &body));
    HB_CK(cudaGraphInstantiate(&h->gW, g, 0));
    return HBUGKS_OK;
}

// every case at rest (rho 1, T0) on every level, fresh status, local steps of that state
template <typename T>
hbugks_status reset_rest(hbugks_t h, Impl<T>& im, int ncases)
{
    HB_CK(cudaMemsetAsync(im.d_tol, 0, sizeof(double), h->s));
    HB_CK(cudaMemsetAsync(im.d_err, 0, 2 * sizeof(int), h->s));
    k_status_reset<<<(ncases + 127) / 128, 128, 0, h->s>>>(im.d_status, ncases, -1, 1);
    for (int k = 0; k < ncases; ++k) {
        const CaseDev<T>& d = im.dc[k];
        size_t tot = (size_t)d.nc * d.nvb * VB * d.nt;
        k_init_uniform<T><<<(unsigned)((tot + 255) / 256), 256, 0, h->s>>>(d, 1.0, 0.0, 0.0, 1.0);
    }
    enqueue_steps(im, ncases, h->s);
    return HBUGKS_OK;
}

template <typename T>
hbugks_status upload_offsets(hbugks_t h, Impl<T>& im)
{
    fill_offsets(im, h->ncases);
    HB_CK(cudaMemcpyAsync(im.d_off, im.off_host.data(), sizeof(int) * im.off_host.size(), cudaMemcpyHostToDevice, h->s));
    return HBUGKS_OK;
}

// ------------------------------------------------------------------------------ autotuner of the K4 variant
// The micro update's variant (cells per CTA, velocity blocks per CTA) trades halo re-reads, pass-1 work and the
// indices and parameters shared by a CTA's blocks against shared memory per CTA and so against CTAs per SM;
// which wins depends on the level count, the velocity grid, the mesh and the GPU.  Each variant the case can
// run is timed on the case itself (one warm-up launch, then three), after one iteration from rest has filled
// the parameters the kernel reads.  Choices are cached per process by everything that sets the launch: mesh
// size, velocity grid, blocks, levels, precision, SM count and the form of the spectral source.

struct TuneCache {
    std::mutex mu;
    std::map<std::vector<int>, int> best;
};
TuneCache& tune_cache()
{
    static TuneCache c;
    return c;
}

template <typename T>
hbugks_status autotune(hbugks_t h, Impl<T>& im, int ncases)
{
    int dev = 0, sms = 0;
    HB_CK(cudaGetDevice(&dev));
    HB_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    std::vector<std::vector<int>> keys(ncases);
    bool need = false;
    {
        std::lock_guard<std::mutex> lk(tune_cache().mu);
        for (int k = 0; k < ncases; ++k) {
            const HostCase& hc = im.hc[k];
            keys[k] = {hc.nx, hc.ny, hc.nu, hc.nv, hc.nvb, hc.nt, (int)sizeof(T), sms, hc.src.phys.spectral_implicit};
            auto it = tune_cache().best.find(keys[k]);
            if (it != tune_cache().best.end()) im.hc[k].k4shape = it->second;
            else need = true;
        }
    }
    if (need) {
        k_begin_call<<<(ncases + 127) / 128, 128, 0, h->s>>>(im.d_status, ncases);
        enqueue_iteration(im, ncases, h->s);
        k_begin_call<<<(ncases + 127) / 128, 128, 0, h->s>>>(im.d_status, ncases);
        Events evs;
        HB_CK(evs.create(2));
        const cudaEvent_t e0 = evs.ev[0], e1 = evs.ev[1];
        for (int k = 0; k < ncases; ++k) {
            {
                std::lock_guard<std::mutex> lk(tune_cache().mu);
                auto it = tune_cache().best.find(keys[k]);
                if (it != tune_cache().best.end()) { im.hc[k].k4shape = it->second; continue; }
            }
            HostCase& hc = im.hc[k];
            int best = -1;
            float best_ms = 0.f;
            for (int sh = 0; sh < N_K4_SHAPES; ++sh) {
                if (!k4_shape_ok<T>(sh, hc.nt, hc.pairs != 0)) continue;
                const size_t smem = k4_smem_of<T>(sh, hc.nt);
                const Shape S = K4_SHAPES[sh];
                const int off[2] = {0, ((hc.nx + S.tx - 1) / S.tx) * ((hc.ny + S.ty - 1) / S.ty) * (hc.nvb / S.vpl)};
                HB_CK(cudaMemcpyAsync(im.d_tune_off, off, sizeof off, cudaMemcpyHostToDevice, h->s));
                const Batch<T> b{im.d_cases + k, 1, im.d_tune_off};
                const bool imp = hc.src.phys.spectral_implicit != 0;
                launch_k4<T>(imp, sh, off[1], smem, b, h->s);
                HB_CK(cudaEventRecord(e0, h->s));
                for (int r = 0; r < 3; ++r) launch_k4<T>(imp, sh, off[1], smem, b, h->s);
                HB_CK(cudaEventRecord(e1, h->s));
                HB_CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                HB_CK(cudaEventElapsedTime(&ms, e0, e1));
                if (best < 0 || ms < best_ms) { best = sh; best_ms = ms; }
            }
            hc.k4shape = best;
            std::lock_guard<std::mutex> lk(tune_cache().mu);
            tune_cache().best[keys[k]] = best;
        }
        HB_CK(cudaGetLastError());
    }
    for (auto& hc : im.hc) set_k4_blocks(hc);
    return upload_offsets(h, im);
}

template <typename T>
hbugks_status do_create(hbugks_t h, Impl<T>& im, int ncases, const hbugks_case* cases)
{
    plan(im, ncases, cases, h->ws);
    for (auto& hc : im.hc) {
        if (hc.k4shape < 0) return HBUGKS_EINVAL;
        if (hc.src.phys.spectral_implicit) im.any_implicit = true;
    }
    HB_CK(set_smem_attributes<T>());
    std::vector<std::vector<char>> keep;
    for (int k = 0; k < ncases; ++k) HB_CK(upload_case(im.hc[k], im.dc[k], h->s, keep));
    HB_CK(cudaMemcpyAsync(im.d_cases, im.dc.data(), sizeof(CaseDev<T>) * ncases, cudaMemcpyHostToDevice, h->s));
    HB_CK(cudaMemcpyAsync(im.d_off, im.off_host.data(), sizeof(int) * im.off_host.size(), cudaMemcpyHostToDevice, h->s));
    hbugks_status rc = reset_rest(h, im, ncases);
    if (rc == HBUGKS_OK) rc = autotune(h, im, ncases);
    if (rc == HBUGKS_OK) rc = reset_rest(h, im, ncases);
    if (rc != HBUGKS_OK) return rc;
    HB_CK(cudaStreamSynchronize(h->s));
    HB_CK(cudaGetLastError());
    return capture(h, im);
}

// runs fn on the handle's precision; a status-returning fn reports a C++ exception (host allocation) as a status,
// so that none crosses the C ABI
template <class F>
auto dispatch(hbugks_t h, F&& fn) -> decltype(fn(*h->d))
{
    using R = decltype(fn(*h->d));
    if constexpr (std::is_same<R, hbugks_status>::value) {
        try {
            if (h->f) return fn(*h->f);
            return fn(*h->d);
        } catch (const std::bad_alloc&) {
            return HBUGKS_ENOMEM;
        } catch (...) {
            return HBUGKS_EINVAL;
        }
    } else {
        if (h->f) return fn(*h->f);
        return fn(*h->d);
    }
}

}  // namespace

namespace {

// up to n iterations in one launch of the device-side loop (stream-ordered: the count is set on the stream)
template <typename T>
hbugks_status launch_loop(hbugks_t h, Impl<T>& im, int n)
{
    if (n <= 0) return HBUGKS_OK;
    k_set_int<<<1, 1, 0, h->s>>>(im.d_loop, n);
    HB_CK(cudaGraphLaunch(h->gW, h->s));
    return HBUGKS_OK;
}

}  // namespace

// ====================================================================================== no-allocation harmonic

namespace {

// fixed scratch of the no-allocation entry point: per-level fields [nt][8][nc]
static __device__ __align__(256) double g_noalloc_scratch[HBUGKS_NOALLOC_MAX_DOUBLES];

// fields of every level from a canonical FP64 state (h, b [nt][nc][nu*nv]); one warp per (cell, level)
__global__ void k_fields_canonical(int nc, int nu, int nv, int nt, const double* u, const double* wu, const double* v,
                                   const double* wv, const double* h, const double* b, double* lv)
{
    const int lane = threadIdx.x & 31;
    const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= nc * nt) return;
    const int n = item / nc, c = item - n * nc;
    const int nvel = nu * nv;
    const double* hc = h + ((size_t)n * nc + c) * nvel;
    const double* bc = b + ((size_t)n * nc + c) * nvel;
    double A[13];
    for (int q = 0; q < 13; ++q) A[q] = 0.0;
    for (int a = lane; a < nvel; a += 32) {
        const int iu = a % nu, jv = a / nu;
        const double uu = u[iu], vv = v[jv], w = wu[iu] * wv[jv];
        const double wd = w * hc[a], we = w * bc[a];
        A[0] += wd; A[1] += wd * uu; A[2] += wd * vv; A[3] += wd * uu * uu; A[4] += wd * uu * vv;
        A[5] += wd * vv * vv; A[6] += wd * uu * uu * uu; A[7] += wd * uu * uu * vv; A[8] += wd * uu * vv * vv;
        A[9] += wd * vv * vv * vv; A[10] += we; A[11] += we * uu; A[12] += we * vv;
    }
    for (int q = 0; q < 13; ++q) A[q] = warp_sum(A[q]);
    if (lane == 0) {
        double Wm[4] = {A[0], A[1], A[2], 0.5 * (A[3] + A[5] + A[10])};
        double rho, U, V, lam, qx, qy;
        prim(Wm, rho, U, V, lam);
        heat_flux_raw(A, U, V, qx, qy);
        double* o = lv + (size_t)n * 8 * nc;
        o[0 * nc + c] = rho;
        o[1 * nc + c] = U;
        o[2 * nc + c] = V;
        o[3 * nc + c] = 1.0 / lam;
        o[4 * nc + c] = A[4] - V * A[1] - U * A[2] + U * V * A[0];
        o[5 * nc + c] = qx;
        o[6 * nc + c] = qy;
        o[7 * nc + c] = rho / (2.0 * lam);
    }
}

// the calling thread's current CUDA context, through the driver entry point the runtime hands out (the library
// does not link the driver library itself); nullptr if it cannot be queried
void* current_context()
{
    using Fn = int (*)(void**);
    static Fn fn = []() -> Fn {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<Fn>(p);
    }();
    void* ctx = nullptr;
    if (!fn || fn(&ctx) != 0) return nullptr;
    return ctx;
}

// Device address of the scratch array, looked up once per device and context: the address belongs to the
// context the module was loaded into, so after a context is torn down and rebuilt (cudaDeviceReset, a new
// primary context) it is looked up again.
double* noalloc_scratch(int dev)
{
    struct Entry { void* ctx; double* ptr; };
    static std::mutex mu;
    static Entry tab[256] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 256) return nullptr;
    void* ctx = current_context();
    if (!tab[dev].ptr || ctx == nullptr || ctx != tab[dev].ctx) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
        tab[dev] = Entry{ctx, static_cast<double*>(p)};
    }
    return tab[dev].ptr;
}

}  // namespace

// ====================================================================================== ABI

extern "C" {

size_t hbugks_workspace_bytes(int ncases, const hbugks_case* cases)
{
    Range range_("hbugks_workspace_bytes");
    if (ncases < 1 || !cases) return 0;
    for (int k = 0; k < ncases; ++k)
        if (!validate(cases[k]) || cases[k].phys.precision != cases[0].phys.precision) return 0;
    try {
        if (cases[0].phys.precision == 1) {
            Impl<float> im;
            return plan(im, ncases, cases, nullptr);
        }
        Impl<double> im;
        return plan(im, ncases, cases, nullptr);
    } catch (...) {
        return 0;
    }
}

hbugks_status hbugks_create(int ncases, const hbugks_case* cases, void* d_workspace, size_t bytes,
                            void* cuda_stream, hbugks_t* out)
{
    Range range_("hbugks_create");
    if (!out || !d_workspace || ((uintptr_t)d_workspace & 255)) return HBUGKS_EINVAL;
    size_t need = hbugks_workspace_bytes(ncases, cases);
    if (need == 0) return HBUGKS_EINVAL;
    if (bytes < need) return HBUGKS_ENOMEM;
    hbugks_t h = new (std::nothrow) hbugks_solver;
    if (!h) return HBUGKS_ENOMEM;
    h->ncases = ncases;
    h->precision = cases[0].phys.precision;
    h->user = (cudaStream_t)cuda_stream;
    h->ws = (char*)d_workspace;
    h->bytes = bytes;
    hbugks_status rc = HBUGKS_OK;
    if (cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        hbugks_destroy(h);
        return HBUGKS_ECUDA;
    }
    if ((rc = begin(h)) != HBUGKS_OK) { hbugks_destroy(h); return rc; }
    try {
        h->st_host.resize(ncases);
        if (h->precision == 1) {
            h->f = new Impl<float>;
            rc = do_create(h, *h->f, ncases, cases);
        } else {
            h->d = new Impl<double>;
            rc = do_create(h, *h->d, ncases, cases);
        }
    } catch (const std::bad_alloc&) {
        rc = HBUGKS_ENOMEM;
    } catch (...) {
        rc = HBUGKS_EINVAL;
    }
    if (rc == HBUGKS_OK) rc = end(h);
    if (rc != HBUGKS_OK) { hbugks_destroy(h); return rc; }
    *out = h;
    return HBUGKS_OK;
}

void hbugks_destroy(hbugks_t h)
{
    Range range_("hbugks_destroy");
    if (!h) return;
    if (h->s) cudaStreamSynchronize(h->s);
    if (h->g1) cudaGraphExecDestroy(h->g1);
    if (h->gN) cudaGraphExecDestroy(h->gN);
    if (h->gW) cudaGraphExecDestroy(h->gW);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->s) cudaStreamDestroy(h->s);
    delete h->f;
    delete h->d;
    delete h;
}

hbugks_status hbugks_set_wall(hbugks_t h, int ci, int wall, const hbugks_wall* w)
{
    Range range_("hbugks_set_wall");
    if (!h || !w || ci < 0 || ci >= h->ncases || wall < 0 || wall > 3) return HBUGKS_EINVAL;
    return dispatch(h, [&](auto& im) -> hbugks_status {
        HostCase hc = im.hc[ci];
        hc.src.walls[wall] = *w;
        if (!validate(hc.src)) return HBUGKS_EINVAL;
        fill_host(im.hc[ci], hc.src);
        hbugks_status rc = begin(h);
        if (rc) return rc;
        HB_CK(cudaMemcpyAsync((void*)im.dc[ci].wall, im.hc[ci].wall_tab.data(),
                              sizeof(double) * im.hc[ci].wall_tab.size(), cudaMemcpyHostToDevice, h->s));
        using TT = std::remove_const_t<typename std::remove_pointer<decltype(im.dc[ci].tu)>::type>;
        std::vector<double> wconst, oconst;
        std::vector<TT> wtab;
        wall_constants<TT>(im.hc[ci], wconst, oconst, wtab);
        HB_CK(cudaMemcpyAsync((void*)im.dc[ci].wconst, wconst.data(), sizeof(double) * wconst.size(),
                              cudaMemcpyHostToDevice, h->s));
        HB_CK(cudaMemcpyAsync((void*)im.dc[ci].wtab, wtab.data(), sizeof(TT) * wtab.size(), cudaMemcpyHostToDevice, h->s));
        HB_CK(cudaStreamSynchronize(h->s));
        return end(h);
    });
}

hbugks_status hbugks_init_uniform(hbugks_t h, int ci, double rho, double u, double v, double T)
{
    Range range_("hbugks_init_uniform");
    if (!h || ci < -1 || ci >= h->ncases || !(rho > 0) || !(T > 0)) return HBUGKS_EINVAL;
    return dispatch(h, [&](auto& im) -> hbugks_status {
        hbugks_status rc = begin(h);
        if (rc) return rc;
        k_status_reset<<<(h->ncases + 127) / 128, 128, 0, h->s>>>(im.d_status, h->ncases, ci, -1);
        for (int k = 0; k < h->ncases; ++k) {
            if (ci >= 0 && k != ci) continue;
            auto& d = im.dc[k];
            size_t tot = (size_t)d.nc * d.nvb * VB * d.nt;
            using TT = typename std::remove_pointer<decltype(d.tu)>::type;
            k_init_uniform<std::remove_const_t<TT>><<<(unsigned)((tot + 255) / 256), 256, 0, h->s>>>(d, rho, u, v, T);
        }
        enqueue_steps(im, h->ncases, h->s);
        return end(h);
    });
}

hbugks_status hbugks_set_state(hbugks_t h, int ci, const double* W, const double* hh, const double* bb)
{
    Range range_("hbugks_set_state");
    if (!h || ci < 0 || ci >= h->ncases || !W || !hh || !bb) return HBUGKS_EINVAL;
    return dispatch(h, [&](auto& im) -> hbugks_status {
        auto& d = im.dc[ci];
        using TT = std::remove_const_t<typename std::remove_pointer<decltype(d.tu)>::type>;
        hbugks_status rc = begin(h);
        if (rc) return rc;
        k_status_reset<<<(h->ncases + 127) / 128, 128, 0, h->s>>>(im.d_status, h->ncases, ci, -1);
        HB_CK(cudaMemcpyAsync(d.W[0], W, sizeof(double) * d.nt * d.nc * 4, cudaMemcpyHostToDevice, h->s));
        const size_t lvl = (size_t)d.nc * d.nvel;
        const size_t tot = (size_t)d.nc * d.nvb * VB;
        for (int n = 0; n < d.nt; ++n)
            for (int which = 0; which < 2; ++which) {
                const double* src = (which == 0 ? hh : bb) + (size_t)n * lvl;
                HB_CK(cudaMemcpyAsync(d.stage, src, sizeof(double) * lvl, cudaMemcpyHostToDevice, h->s));
                k_set_level<TT><<<(unsigned)((tot + 255) / 256), 256, 0, h->s>>>(d, n, which, d.stage);
            }
        enqueue_steps(im, h->ncases, h->s);
        HB_CK(cudaStreamSynchronize(h->s));
        return end(h);
    });
}

hbugks_status hbugks_get_state(hbugks_t h, int ci, double* W, double* hh, double* bb)
{
    Range range_("hbugks_get_state");
    if (!h || ci < 0 || ci >= h->ncases || !W || (!hh != !bb)) return HBUGKS_EINVAL;
    return dispatch(h, [&](auto& im) -> hbugks_status {
        auto& d = im.dc[ci];
        using TT = std::remove_const_t<typename std::remove_pointer<decltype(d.tu)>::type>;
        hbugks_status rc = begin(h);
        if (rc) return rc;
        CaseStatus st;
        HB_CK(cudaMemcpyAsync(&st, im.d_status + ci, sizeof st, cudaMemcpyDeviceToHost, h->s));
        HB_CK(cudaStreamSynchronize(h->s));
        HB_CK(cudaMemcpyAsync(W, d.W[st.parity], sizeof(double) * d.nt * d.nc * 4, cudaMemcpyDeviceToHost, h->s));
        const size_t lvl = (size_t)d.nc * d.nvel;
        const size_t tot = (size_t)d.nc * d.nvb * VB;
        for (int n = 0; hh && n < d.nt; ++n)
            for (int which = 0; which < 2; ++which) {
                k_get_level<TT><<<(unsigned)((tot + 255) / 256), 256, 0, h->s>>>(d, n, which, d.stage);
                double* dst = (which == 0 ? hh : bb) + (size_t)n * lvl;
                HB_CK(cudaMemcpyAsync(dst, d.stage, sizeof(double) * lvl, cudaMemcpyDeviceToHost, h->s));
            }
        HB_CK(cudaStreamSynchronize(h->s));
        return end(h);
    });
}

hbugks_status hbugks_set_active(hbugks_t h, const int* flags)
{
    Range range_("hbugks_set_active");
    if (!h || !flags) return HBUGKS_EINVAL;
    return dispatch(h, [&](auto& im) -> hbugks_status {
        hbugks_status rc = begin(h);
        if (rc) return rc;
        std::vector<CaseStatus> st(h->ncases);
        HB_CK(cudaMemcpyAsync(st.data(), im.d_status, sizeof(CaseStatus) * h->ncases, cudaMemcpyDeviceToHost, h->s));
        HB_CK(cudaStreamSynchronize(h->s));
        for (int k = 0; k < h->ncases; ++k) st[k].user_active = flags[k] ? 1 : 0;
        HB_CK(cudaMemcpyAsync(im.d_status, st.data(), sizeof(CaseStatus) * h->ncases, cudaMemcpyHostToDevice, h->s));
        HB_CK(cudaStreamSynchronize(h->s));
        return end(h);
    });
}

static hbugks_status launch_iters(hbugks_t h, int n)
{
    while (n >= CHUNK) {
        HB_CK(cudaGraphLaunch(h->gN, h->s));
        n -= CHUNK;
    }
    while (n-- > 0) HB_CK(cudaGraphLaunch(h->g1, h->s));
    return HBUGKS_OK;
}


hbugks_status hbugks_enqueue_iterations(hbugks_t h, int n)
{
    Range range_("hbugks_enqueue_iterations");
    if (!h || n < 0) return HBUGKS_EINVAL;
    return dispatch(h, [&](auto& im) -> hbugks_status {
        hbugks_status rc = begin(h);
        if (rc) return rc;
        HB_CK(cudaMemsetAsync(im.d_tol, 0, sizeof(double), h->s));
        k_begin_call<<<(h->ncases + 127) / 128, 128, 0, h->s>>>(im.d_status, h->ncases);
        if ((rc = h->loop_mode == 0 ? launch_loop(h, im, n) : launch_iters(h, n))) return rc;
        return end(h);
    });
}

hbugks_status hbugks_iterate(hbugks_t h, int max_iters, double tol_rho, int* iters_done, double* resid_out)
{
    Range range_("hbugks_iterate");
    if (!h || max_iters < 0) return HBUGKS_EINVAL;
    return dispatch(h, [&](auto& im) -> hbugks_status {
        hbugks_status rc = begin(h);
        if (rc) return rc;
        h->tol_host = tol_rho > 0 ? tol_rho : 0.0;
        HB_CK(cudaMemcpyAsync(im.d_tol, &h->tol_host, sizeof(double), cudaMemcpyHostToDevice, h->s));
        k_begin_call<<<(h->ncases + 127) / 128, 128, 0, h->s>>>(im.d_status, h->ncases);
        int done = 0;
        std::vector<CaseStatus>& st = h->st_host;
        // statuses and the error word after every chunk of iterations: a wait that ran out ends the call at once
        // (the kernels of later iterations return without work while the word is set)
        auto poll = [&](int& err) -> hbugks_status {
            HB_CK(cudaMemcpyAsync(st.data(), im.d_status, sizeof(CaseStatus) * h->ncases, cudaMemcpyDeviceToHost, h->s));
            HB_CK(cudaMemcpyAsync(&err, im.d_err, sizeof(int), cudaMemcpyDeviceToHost, h->s));
            HB_CK(cudaStreamSynchronize(h->s));
            return HBUGKS_OK;
        };
        int err = 0;
        if (h->loop_mode == 0) {
            // one launch of the device-side loop, one read of the statuses at its end
            if ((rc = launch_loop(h, im, max_iters))) return rc;
            done = max_iters;
        } else {
            while (done < max_iters) {
                int n = std::min(CHUNK, max_iters - done);
                if ((rc = launch_iters(h, n))) return rc;
                done += n;
                if ((rc = poll(err))) return rc;
                if (err) break;
                bool any = false;
                for (int k = 0; k < h->ncases; ++k) any = any || st[k].active;
                if (!any) break;
            }
        }
        if ((h->loop_mode == 0 || done == 0) && (rc = poll(err))) return rc;
        if (err) {
            // the state is the one before the failed iteration (its residual kernel did not run, so the state
            // buffers did not swap); clear the error word and the test hook, and recompute the local steps of
            // that state (the macro update had already replaced them with those of the abandoned iterate), so
            // that the next call iterates normally
            HB_CK(cudaMemsetAsync(im.d_err, 0, 2 * sizeof(int), h->s));
            enqueue_steps(im, h->ncases, h->s);
            HB_CK(cudaStreamSynchronize(h->s));
            end(h);
            return HBUGKS_TIMEOUT;
        }
        bool diverged = false, all = true;
        for (int k = 0; k < h->ncases; ++k) {
            if (iters_done) iters_done[k] = (int)st[k].iters_call;
            if (resid_out)
                for (int q = 0; q < 4; ++q) resid_out[k * 4 + q] = st[k].last[q];
            if (st[k].diverged) diverged = true;
            if (tol_rho > 0 && st[k].user_active && !(st[k].last[0] <= tol_rho && st[k].iters >= 10)) all = false;
        }
        if ((rc = end(h))) return rc;
        if (diverged) return HBUGKS_DIVERGED;
        return all ? HBUGKS_OK : HBUGKS_NOT_CONVERGED;
    });
}

hbugks_status hbugks_residual_history(hbugks_t h, int ci, int n, double* out)
{
    Range range_("hbugks_residual_history");
    if (!h || ci < 0 || ci >= h->ncases || n < 0 || n > RING || !out) return HBUGKS_EINVAL;
    return dispatch(h, [&](auto& im) -> hbugks_status {
        hbugks_status rc = begin(h);
        if (rc) return rc;
        std::vector<double> ring((size_t)RING * 4);
        CaseStatus st;
        HB_CK(cudaMemcpyAsync(ring.data(), im.dc[ci].rhist, sizeof(double) * ring.size(), cudaMemcpyDeviceToHost, h->s));
        HB_CK(cudaMemcpyAsync(&st, im.d_status + ci, sizeof st, cudaMemcpyDeviceToHost, h->s));
        HB_CK(cudaStreamSynchronize(h->s));
        if (n > st.iters) return HBUGKS_EINVAL;
        for (int k = 0; k < n; ++k) {
            long long it = st.iters - n + k;
            for (int q = 0; q < 4; ++q) out[k * 4 + q] = ring[(it % RING) * 4 + q];
        }
        return end(h);
    });
}

hbugks_status hbugks_get_level_fields(hbugks_t h, int ci, int level, double* out)
{
    Range range_("hbugks_get_level_fields");
    if (!h || ci < 0 || ci >= h->ncases || !out) return HBUGKS_EINVAL;
    return dispatch(h, [&](auto& im) -> hbugks_status {
        auto& d = im.dc[ci];
        using TT = std::remove_const_t<typename std::remove_pointer<decltype(d.tu)>::type>;
        if (level < 0 || level >= d.nt) return HBUGKS_EINVAL;
        hbugks_status rc = begin(h);
        if (rc) return rc;
        k_fields<TT><<<(d.nc + 7) / 8, 256, 0, h->s>>>(d, level, d.stage);
        HB_CK(cudaMemcpyAsync(out, d.stage, sizeof(double) * 8 * d.nc, cudaMemcpyDeviceToHost, h->s));
        HB_CK(cudaStreamSynchronize(h->s));
        return end(h);
    });
}

hbugks_status hbugks_get_harmonic(hbugks_t h, int ci, int k, double* re, double* im_out)
{
    Range range_("hbugks_get_harmonic");
    if (!h || ci < 0 || ci >= h->ncases || !re || !im_out) return HBUGKS_EINVAL;
    return dispatch(h, [&](auto& im) -> hbugks_status {
        auto& d = im.dc[ci];
        using TT = std::remove_const_t<typename std::remove_pointer<decltype(d.tu)>::type>;
        if (k < 0 || k > d.nh) return HBUGKS_EINVAL;
        hbugks_status rc = begin(h);
        if (rc) return rc;
        for (int n = 0; n < d.nt; ++n)
            k_fields<TT><<<(d.nc + 7) / 8, 256, 0, h->s>>>(d, n, d.stage + (size_t)n * 8 * d.nc);
        double* ore = d.stage + (size_t)d.nt * 8 * d.nc;
        double* oim = ore + 8 * d.nc;
        k_dft<<<(8 * d.nc + 127) / 128, 128, 0, h->s>>>(d.stage, d.nt, d.nc, k, ore, oim);
        HB_CK(cudaMemcpyAsync(re, ore, sizeof(double) * 8 * d.nc, cudaMemcpyDeviceToHost, h->s));
        HB_CK(cudaMemcpyAsync(im_out, oim, sizeof(double) * 8 * d.nc, cudaMemcpyDeviceToHost, h->s));
        HB_CK(cudaStreamSynchronize(h->s));
        return end(h);
    });
}

long long hbugks_iteration_count(hbugks_t h, int ci)
{
    if (!h || ci < 0 || ci >= h->ncases) return -1;
    CaseStatus st;
    const CaseStatus* src = h->f ? h->f->d_status + ci : h->d->d_status + ci;
    if (begin(h) != HBUGKS_OK) return -1;
    if (cudaMemcpyAsync(&st, src, sizeof st, cudaMemcpyDeviceToHost, h->s) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(h->s) != cudaSuccess) return -1;
    if (end(h) != HBUGKS_OK) return -1;
    return st.iters;
}

hbugks_status hbugks_profile_kernels(hbugks_t h, int n, double* ms)
{
    Range range_("hbugks_profile_kernels");
    if (!h || n < 1 || !ms) return HBUGKS_EINVAL;
    return dispatch(h, [&](auto& im) -> hbugks_status {
        hbugks_status rc = begin(h);
        if (rc) return rc;
        Events evs;
        HB_CK(evs.create(10));
        cudaEvent_t* ev = evs.ev.data();
        HB_CK(cudaMemsetAsync(im.d_tol, 0, sizeof(double), h->s));
        k_begin_call<<<(h->ncases + 127) / 128, 128, 0, h->s>>>(im.d_status, h->ncases);
        double acc[5] = {0, 0, 0, 0, 0};
        for (int it = 0; it < n; ++it) {
            enqueue_iteration(im, h->ncases, h->s, ev);
            HB_CK(cudaEventSynchronize(ev[9]));
            for (int k = 0; k < 5; ++k) {
                float t = 0.f;
                HB_CK(cudaEventElapsedTime(&t, ev[2 * k], ev[2 * k + 1]));
                acc[k] += t;
            }
        }
        for (int k = 0; k < 5; ++k) ms[k] = acc[k] / n;
        return end(h);
    });
}

hbugks_status hbugks_harmonic_noalloc(int nx, int ny, int nu, int nv, const double* u, const double* wu, const double* v,
                                      const double* wv, int nt, const double* h, const double* b, int k, double* re,
                                      double* im, void* cuda_stream)
{
    Range range_("hbugks_harmonic_noalloc");
    if (nx < 1 || ny < 1 || nu < 1 || nv < 1 || nt < 1 || !(nt & 1) || !u || !wu || !v || !wv || !h || !b || !re || !im)
        return HBUGKS_EINVAL;
    if (k < 0 || k > (nt - 1) / 2) return HBUGKS_EINVAL;
    const long long nc = (long long)nx * ny;
    if (8LL * nt * nc > (long long)HBUGKS_NOALLOC_MAX_DOUBLES) return HBUGKS_EINVAL;
    int dev = 0;
    HB_CK(cudaGetDevice(&dev));
    double* scratch = noalloc_scratch(dev);
    if (!scratch) return HBUGKS_ECUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int items = (int)(nc * nt);
    k_fields_canonical<<<(items + 7) / 8, 256, 0, s>>>((int)nc, nu, nv, nt, u, wu, v, wv, h, b, scratch);
    k_dft<<<(int)((8 * nc + 127) / 128), 128, 0, s>>>(scratch, nt, (int)nc, k, re, im);
    HB_CK(cudaGetLastError());
    return HBUGKS_OK;
}

hbugks_status hbugks_copy_state(hbugks_t dst, int dst_case, hbugks_t src, int src_case)
{
    Range range_("hbugks_copy_state");
    if (!dst || !src || dst == src || dst_case < 0 || dst_case >= dst->ncases || src_case < 0 ||
        src_case >= src->ncases)
        return HBUGKS_EINVAL;
    return dispatch(src, [&](auto& is) -> hbugks_status {
        return dispatch(dst, [&](auto& id) -> hbugks_status {
            const HostCase& hs = is.hc[src_case];
            const HostCase& hd = id.hc[dst_case];
            if (hs.nx != hd.nx || hs.ny != hd.ny || hs.nu != hd.nu || hs.nv != hd.nv || hs.nt != hd.nt ||
                hs.nvp != hd.nvp || hs.xn != hd.xn || hs.yn != hd.yn || hs.u != hd.u || hs.v != hd.v ||
                hs.wu != hd.wu || hs.wv != hd.wv)
                return HBUGKS_EINVAL;
            const auto& ds = is.dc[src_case];
            const auto& dd = id.dc[dst_case];
            // everything enqueued on src so far, then the current buffer of the source case
            hbugks_status rc = begin(src);
            if (rc) return rc;
            CaseStatus st;
            HB_CK(cudaMemcpyAsync(&st, is.d_status + src_case, sizeof st, cudaMemcpyDeviceToHost, src->s));
            HB_CK(cudaStreamSynchronize(src->s));
            if ((rc = end(src))) return rc;
            if ((rc = begin(dst))) return rc;
            const size_t n = (size_t)hd.nvb * hd.nc * hd.nt * VB;
            using TS = std::remove_const_t<typename std::remove_pointer<decltype(ds.tu)>::type>;
            using TD = std::remove_const_t<typename std::remove_pointer<decltype(dd.tu)>::type>;
            k_status_reset<<<(dst->ncases + 127) / 128, 128, 0, dst->s>>>(id.d_status, dst->ncases, dst_case, -1);
            k_convert_state<TS, TD><<<(unsigned)((n + 255) / 256), 256, 0, dst->s>>>(ds.f[st.parity], dd.f[0], n);
            HB_CK(cudaMemcpyAsync(dd.W[0], ds.W[st.parity], sizeof(double) * hd.nt * hd.nc * 4,
                                  cudaMemcpyDeviceToDevice, dst->s));
            enqueue_steps(id, dst->ncases, dst->s);
            HB_CK(cudaStreamSynchronize(dst->s));
            return end(dst);
        });
    });
}

hbugks_status hbugks_test_expire_wait(hbugks_t h)
{
    Range range_("hbugks_test_expire_wait");
    if (!h) return HBUGKS_EINVAL;
    return dispatch(h, [&](auto& im) -> hbugks_status {
        hbugks_status rc = begin(h);
        if (rc) return rc;
        const int one = 1;
        HB_CK(cudaMemcpyAsync(im.d_err + 1, &one, sizeof(int), cudaMemcpyHostToDevice, h->s));
        HB_CK(cudaStreamSynchronize(h->s));
        return end(h);
    });
}

hbugks_status hbugks_get_micro_variant(hbugks_t h, int case_index, int* tx, int* ty, int* vpl)
{
    if (!h || case_index < 0 || case_index >= h->ncases || !tx || !ty || !vpl) return HBUGKS_EINVAL;
    const int sh = dispatch(h, [&](auto& im) { return im.hc[case_index].k4shape; });
    *tx = K4_SHAPES[sh].tx;
    *ty = K4_SHAPES[sh].ty;
    *vpl = K4_SHAPES[sh].vpl;
    return HBUGKS_OK;
}

hbugks_status hbugks_set_micro_variant(hbugks_t h, int case_index, int tx, int ty, int vpl)
{
    Range range_("hbugks_set_micro_variant");
    if (!h || case_index < 0 || case_index >= h->ncases) return HBUGKS_EINVAL;
    int sh = -1;
    for (int k = 0; k < N_K4_SHAPES; ++k)
        if (K4_SHAPES[k].tx == tx && K4_SHAPES[k].ty == ty && K4_SHAPES[k].vpl == vpl) sh = k;
    if (sh < 0) return HBUGKS_EINVAL;
    return dispatch(h, [&](auto& im) -> hbugks_status {
        using T = typename std::remove_reference<decltype(*im.d_cases)>::type::value_type;
        HostCase& hc = im.hc[case_index];
        if (!k4_shape_ok<T>(sh, hc.nt, hc.pairs != 0)) return HBUGKS_EINVAL;
        hbugks_status rc = begin(h);
        if (rc) return rc;
        hc.k4shape = sh;
        set_k4_blocks(hc);
        if ((rc = upload_offsets(h, im)) != HBUGKS_OK) return rc;
        HB_CK(cudaStreamSynchronize(h->s));
        if (h->g1) { cudaGraphExecDestroy(h->g1); h->g1 = nullptr; }
        if (h->gN) { cudaGraphExecDestroy(h->gN); h->gN = nullptr; }
        if (h->gW) { cudaGraphExecDestroy(h->gW); h->gW = nullptr; }
        if ((rc = capture(h, im)) != HBUGKS_OK) return rc;
        return end(h);
    });
}

hbugks_status hbugks_get_tile_shape(hbugks_t h, int case_index, int* tx, int* ty)
{
    int vpl = 0;
    return hbugks_get_micro_variant(h, case_index, tx, ty, &vpl);
}

hbugks_status hbugks_set_tile_shape(hbugks_t h, int case_index, int tx, int ty)
{
    return hbugks_set_micro_variant(h, case_index, tx, ty, 1);
}

int hbugks_launches_per_iteration(hbugks_t h)
{
    if (!h) return -1;
    return dispatch(h, [&](auto& im) -> int {
        int n = h->loop_mode == 0 ? 2 : 1;   // residual kernel (and the loop test of the device-side loop)
        for (auto& sp : im.specs)
            if (sp.kind != 5 && sp.total) ++n;
        return n;
    });
}

hbugks_status hbugks_set_loop_mode(hbugks_t h, int mode)
{
    Range range_("hbugks_set_loop_mode");
    if (!h || (mode != 0 && mode != 1)) return HBUGKS_EINVAL;
    h->loop_mode = mode;
    return HBUGKS_OK;
}

const char* hbugks_status_string(hbugks_status s)
{
    switch (s) {
        case HBUGKS_OK: return "ok";
        case HBUGKS_NOT_CONVERGED: return "not converged";
        case HBUGKS_EINVAL: return "invalid argument";
        case HBUGKS_ECUDA: return "CUDA error";
        case HBUGKS_ENOMEM: return "workspace too small or host memory exhausted";
        case HBUGKS_DIVERGED: return "diverged";
        case HBUGKS_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char* hbugks_cuda_error_string(void)
{
    return cudaGetErrorString(last_cuda_error());
}

}  // extern "C"
