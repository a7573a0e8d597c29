// Kernels of one HB-UGKS pseudo-time iteration (Sec 2.2 - 2.4) and of the state/field conversions.
//
// One iteration, for every active case of a batch (each kernel covers all cases through a per-case block
// offset table):
//   K1 face_moments : per (face, level): velocity sums of the limited, upwinded interface reconstruction
//                     (kinetic average, heat-flux moments, tangential slopes, free-transport flux moments);
//                     per (cell, level): raw moments of h^k for the heat flux q^k
//   K2 face_params  : per (face, level): interface Maxwellian, tau, dG_f (Eq. dt_face), C1..C5 (Eq. C_coeffs),
//                     slopes a^L, a^R, a_t and A (compatibility), diffuse-wall density (Eq. rho_wall), the
//                     macro flux (Eq. macro_flux) and the parameters the micro update needs
//   K3 macro_update : per cell: W^{k+1} (Eq. fv_W with the spectral source), the collision coefficients of
//                     Eq. fv_h, the next local step (Eqs. dt_hb, nu_conv) and the level-0 residual partials
//   K4 micro_update : per (cell, 32 velocities): interface micro fluxes (Eq. micro_flux), spectral source
//                     across levels and the semi-implicit collision update (Eq. fv_h)
//   K5 finish       : per case: residual (Eq. benchmark_residuals), convergence / divergence status
#pragma once
#include "hb_common.cuh"

namespace hb {

template <typename T>
struct Batch {
    const CaseDev<T>* cases;
    int ncases;
    const int* off;   // block offsets per case for this kernel, ncases + 1 entries
};

// ------------------------------------------------------------------------------ geometry helpers

struct FaceGeo {
    int axis;            // 0: normal along x, 1: normal along y
    int iL, jL, iR, jR;  // low-side and high-side cells
    bool hasL, hasR;
    int wall;            // wall id when one side is missing
};

template <typename T>
__device__ __forceinline__ FaceGeo face_geo(const CaseDev<T>& cd, int f)
{
    FaceGeo g;
    if (f < cd.nfx) {
        int j = f / (cd.nx + 1), i = f - j * (cd.nx + 1);
        g.axis = 0;
        g.iL = i - 1; g.jL = j; g.iR = i; g.jR = j;
        g.hasL = i > 0; g.hasR = i < cd.nx;
        g.wall = (i == 0) ? 3 : 1;
    } else {
        int ff = f - cd.nfx;
        int j = ff / cd.nx, i = ff - j * cd.nx;
        g.axis = 1;
        g.iL = i; g.jL = j - 1; g.iR = i; g.jR = j;
        g.hasL = j > 0; g.hasR = j < cd.ny;
        g.wall = (j == 0) ? 0 : 2;
    }
    return g;
}

// van Leer limited slope from backward / forward divided differences
template <typename T>
__device__ __forceinline__ T van_leer(T s1, T s2)
{
    T p = s1 * s2;
    return p > T(0) ? T(2) * p / (s1 + s2) : T(0);
}

template <typename T>
struct Rec {
    T f, sx, sy;   // value and limited slopes of one array at one cell, level, velocity
};

// value and x / y slopes of array `a` at cell (i, j); a wall-adjacent cell uses its one-sided difference
template <typename T>
__device__ __forceinline__ Rec<T> rec(const CaseDev<T>& cd, const T* a, int vb, int i, int j, int n, int lane)
{
    const int nc = cd.nc, nt = cd.nt, nx = cd.nx, ny = cd.ny;
    int c = j * nx + i;
    Rec<T> r;
    r.f = a[sidx(nc, nt, vb, c, n, lane)];
    if (nx > 1) {
        T s1 = 0, s2 = 0;
        if (i > 0) s1 = (r.f - a[sidx(nc, nt, vb, c - 1, n, lane)]) * T(cd.rdx[i - 1]);
        if (i < nx - 1) s2 = (a[sidx(nc, nt, vb, c + 1, n, lane)] - r.f) * T(cd.rdx[i]);
        if (i == 0) s1 = s2;
        if (i == nx - 1) s2 = s1;
        r.sx = van_leer(s1, s2);
    } else {
        r.sx = 0;
    }
    if (ny > 1) {
        T s1 = 0, s2 = 0;
        if (j > 0) s1 = (r.f - a[sidx(nc, nt, vb, c - nx, n, lane)]) * T(cd.rdy[j - 1]);
        if (j < ny - 1) s2 = (a[sidx(nc, nt, vb, c + nx, n, lane)] - r.f) * T(cd.rdy[j]);
        if (j == 0) s1 = s2;
        if (j == ny - 1) s2 = s1;
        r.sy = van_leer(s1, s2);
    } else {
        r.sy = 0;
    }
    return r;
}

template <typename T>
struct Up {
    T d0, e0;      // reconstructed deviations of h and b at the face
    T sn, st;      // normal / tangential slopes of h in the upwind cell
    T snb, stb;    // same for b
    int mode;      // 1: carried by the reconstruction (interior, or incident at a wall); 2: reflected at a
                   // wall; 0: zero normal velocity at a wall
};

// Upwind reconstruction of (h, b) at face g for one velocity with normal component un (Sec 2.2)
template <typename T>
__device__ __forceinline__ Up<T> upwind(const CaseDev<T>& cd, const T* dh, const T* db, const FaceGeo& g, int vb,
                                        int n, int lane, T un)
{
    Up<T> o;
    const bool wall = !(g.hasL && g.hasR);
    auto one = [&](bool left) {
        int i = left ? g.iL : g.iR, j = left ? g.jL : g.jR;
        Rec<T> rh = rec(cd, dh, vb, i, j, n, lane);
        Rec<T> rb = rec(cd, db, vb, i, j, n, lane);
        T off = g.axis == 0 ? T(left ? cd.hx[i] : -cd.hx[i]) : T(left ? cd.hy[j] : -cd.hy[j]);
        Up<T> u;
        if (g.axis == 0) {
            u.sn = rh.sx; u.st = rh.sy; u.snb = rb.sx; u.stb = rb.sy;
        } else {
            u.sn = rh.sy; u.st = rh.sx; u.snb = rb.sy; u.stb = rb.sx;
        }
        u.d0 = rh.f + u.sn * off;
        u.e0 = rb.f + u.snb * off;
        u.mode = 1;
        return u;
    };
    if (wall) {
        bool left = g.hasL;                 // interior cell side
        o = one(left);
        T nin = left ? T(-1) : T(1);        // normal pointing into the fluid
        T s = un * nin;
        o.mode = s < T(0) ? 1 : (s > T(0) ? 2 : 0);
        return o;
    }
    if (un > T(0)) return one(true);
    if (un < T(0)) return one(false);
    Up<T> a = one(true), b = one(false);
    o.d0 = T(0.5) * (a.d0 + b.d0); o.e0 = T(0.5) * (a.e0 + b.e0);
    o.sn = T(0.5) * (a.sn + b.sn); o.st = T(0.5) * (a.st + b.st);
    o.snb = T(0.5) * (a.snb + b.snb); o.stb = T(0.5) * (a.stb + b.stb);
    o.mode = 1;
    return o;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------------------------ K1 face / cell moments

template <typename T>
__global__ void __launch_bounds__(256) k1_moments(Batch<T> B)
{
    int cs = find_case(B.off, B.ncases, blockIdx.x);
    const CaseDev<T>& cd = B.cases[cs];
    if (!cd.st->active) return;
    const int lane = threadIdx.x & 31;
    const int item = (blockIdx.x - B.off[cs]) * 8 + (threadIdx.x >> 5);
    const int nt = cd.nt;
    const int p = cd.st->parity;
    const T* dh = cd.dh[p];
    const T* db = cd.db[p];
    if (item < cd.nf * nt) {
        const int f = item / nt, n = item - f * nt;
        const FaceGeo g = face_geo(cd, f);
        T acc[NM];
#pragma unroll
        for (int k = 0; k < NM; ++k) acc[k] = T(0);
        for (int vb = 0; vb < cd.nvb; ++vb) {
            const int a = vb * VB + lane;
            const T u = cd.tu[a], v = cd.tv[a], w = cd.tw[a];
            const T un = g.axis == 0 ? u : v, ut = g.axis == 0 ? v : u;
            Up<T> r = upwind(cd, dh, db, g, vb, n, lane, un);
            const T u2 = u * u + v * v;
            // tangential slopes: every velocity of the upwind / interior cell
            acc[13] += w * r.st;
            acc[14] += w * u * r.st;
            acc[15] += w * v * r.st;
            acc[16] += w * u2 * r.st;
            acc[17] += w * r.stb;
            if (r.mode == 1) {
                const T wd = w * r.d0, we = w * r.e0;
                acc[0] += wd;
                acc[1] += wd * u;
                acc[2] += wd * v;
                acc[3] += wd * u * u;
                acc[4] += wd * u * v;
                acc[5] += wd * v * v;
                acc[6] += wd * u * u * u;
                acc[7] += wd * u * u * v;
                acc[8] += wd * u * v * v;
                acc[9] += wd * v * v * v;
                acc[10] += we;
                acc[11] += we * u;
                acc[12] += we * v;
                const T s = un * r.sn + ut * r.st, sb = un * r.snb + ut * r.stb;
                const T wus = w * un * s;
                acc[18] += wus;
                acc[19] += wus * u;
                acc[20] += wus * v;
                acc[21] += wus * u2;
                acc[22] += w * un * sb;
            }
        }
        double* out = cd.fmom + (size_t)item * NM;
#pragma unroll
        for (int k = 0; k < NM; ++k) {
            double s = warp_sum((double)acc[k]);
            if (lane == 0) out[k] = s;
        }
    } else if (item < (cd.nf + cd.nc) * nt) {
        const int it2 = item - cd.nf * nt;
        const int c = it2 / nt, n = it2 - c * nt;
        T acc[NCM];
#pragma unroll
        for (int k = 0; k < NCM; ++k) acc[k] = T(0);
        for (int vb = 0; vb < cd.nvb; ++vb) {
            const int a = vb * VB + lane;
            const T u = cd.tu[a], v = cd.tv[a], w = cd.tw[a];
            const size_t id = sidx(cd.nc, nt, vb, c, n, lane);
            const T wd = w * dh[id], we = w * db[id];
            acc[0] += wd;
            acc[1] += wd * u;
            acc[2] += wd * v;
            acc[3] += wd * u * u;
            acc[4] += wd * u * v;
            acc[5] += wd * v * v;
            acc[6] += wd * u * u * u;
            acc[7] += wd * u * u * v;
            acc[8] += wd * u * v * v;
            acc[9] += wd * v * v * v;
            acc[10] += we;
            acc[11] += we * u;
            acc[12] += we * v;
        }
        double* out = cd.cmom + (size_t)it2 * NCM;
#pragma unroll
        for (int k = 0; k < NCM; ++k) {
            double s = warp_sum((double)acc[k]);
            if (lane == 0) out[k] = s;
        }
    }
}

// heat flux from the 13 raw moments (h: 1,u,v,uu,uv,vv,uuu,uuv,uvv,vvv; b: 1,u,v) about (U, V):
// q = 1/2 sum w c (|c|^2 h + b)  (Eq. heatflux, reduced)
__device__ __forceinline__ void heat_flux_raw(const double* A, double U, double V, double& qx, double& qy)
{
    double cx3 = A[6] - 3.0 * U * A[3] + 3.0 * U * U * A[1] - U * U * U * A[0];
    double cxcy2 = A[8] - 2.0 * V * A[4] + V * V * A[1] - U * A[5] + 2.0 * U * V * A[2] - U * V * V * A[0];
    double cy3 = A[9] - 3.0 * V * A[5] + 3.0 * V * V * A[2] - V * V * V * A[0];
    double cycx2 = A[7] - 2.0 * U * A[4] + U * U * A[2] - V * A[3] + 2.0 * U * V * A[1] - V * U * U * A[0];
    qx = 0.5 * (cx3 + cxcy2 + A[11] - U * A[10]);
    qy = 0.5 * (cy3 + cycx2 + A[12] - V * A[10]);
}

// ------------------------------------------------------------------------------ K2 face parameters

template <typename T>
__global__ void __launch_bounds__(128) k2_face_params(Batch<T> B)
{
    int cs = find_case(B.off, B.ncases, blockIdx.x);
    const CaseDev<T>& cd = B.cases[cs];
    if (!cd.st->active) return;
    const int item = (blockIdx.x - B.off[cs]) * blockDim.x + threadIdx.x;
    const int nt = cd.nt;
    if (item >= cd.nf * nt) return;
    const int f = item / nt, n = item - f * nt;
    const FaceGeo g = face_geo(cd, f);
    const int p = cd.st->parity;
    const double* W = cd.W[p];
    const double* m = cd.fmom + (size_t)item * NM;
    const bool wall = !(g.hasL && g.hasR);
    const double nin = wall ? (g.hasL ? -1.0 : 1.0) : 0.0;
    const int ax = g.axis;
    // velocity-subset rows of the 1-D sums along the normal axis
    const int inc_row = nin > 0 ? 2 : 1;      // incident: u_n nin < 0
    const int ref_row = nin > 0 ? 1 : 2;      // reflected: u_n nin > 0
    int refset = 0;
    if (wall) refset = ax == 0 ? (nin > 0 ? 2 : 1) : (nin > 0 ? 4 : 3);
    double A[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) A[k] = m[k] + cd.refmom[refset * 13 + k];

    // ---- diffuse wall: Maxwellian of the wall, free-transport density estimate, mixed kinetic average
    double Uw = 0, Vw = 0, lamw = 1, prefw = 0, i2lw = 0, Dw = 1, rhow0 = 0;
    Sums1D Xw, Yw;
    double Amix[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) Amix[k] = A[k];
    if (wall) {
        const double* ws = cd.wall + ((size_t)g.wall * nt + n) * 3;
        Uw = ws[0]; Vw = ws[1]; lamw = cd.lam0 / ws[2];
        sums1d(cd.u1, cd.wu1, cd.nu, lamw, Uw, Xw);
        sums1d(cd.v1, cd.wv1, cd.nv, lamw, Vw, Yw);
        prefw = lamw / M_PI;
        i2lw = 0.5 / lamw;
        const int rx = ax == 0 ? ref_row : 0, ry = ax == 0 ? 0 : ref_row;
        double Aw[13];
        Aw[0] = Xw.s[rx][0] * Yw.s[ry][0];
        Aw[1] = Xw.s[rx][1] * Yw.s[ry][0];
        Aw[2] = Xw.s[rx][0] * Yw.s[ry][1];
        Aw[3] = Xw.s[rx][2] * Yw.s[ry][0];
        Aw[4] = Xw.s[rx][1] * Yw.s[ry][1];
        Aw[5] = Xw.s[rx][0] * Yw.s[ry][2];
        Aw[6] = Xw.s[rx][3] * Yw.s[ry][0];
        Aw[7] = Xw.s[rx][2] * Yw.s[ry][1];
        Aw[8] = Xw.s[rx][1] * Yw.s[ry][2];
        Aw[9] = Xw.s[rx][0] * Yw.s[ry][3];
#pragma unroll
        for (int k = 0; k < 10; ++k) Aw[k] *= prefw;
        Aw[10] = i2lw * Aw[0]; Aw[11] = i2lw * Aw[1]; Aw[12] = i2lw * Aw[2];
        Dw = nin * (ax == 0 ? Aw[1] : Aw[2]);                 // sum_refl w |u_n| H_w
        rhow0 = -nin * (ax == 0 ? A[1] : A[2]) / Dw;          // Eq. rho_wall with the free-transport part
#pragma unroll
        for (int k = 0; k < 13; ++k) Amix[k] = A[k] + rhow0 * Aw[k];
    }

    // ---- interface Maxwellian from the kinetic average, heat flux, relaxation time
    double W0[4] = {Amix[0], Amix[1], Amix[2], 0.5 * (Amix[3] + Amix[5] + Amix[10])};
    double rho0, U0, V0, lam0f;
    prim(W0, rho0, U0, V0, lam0f);
    double q0x, q0y;
    heat_flux_raw(Amix, U0, V0, q0x, q0y);
    const double tau = relax_time(cd.mu0, cd.w_vss, cd.lam0, rho0, lam0f);

    // ---- face step (Eq. dt_face) and time-integration weights (Eq. C_coeffs)
    const int cL = g.jL * cd.nx + g.iL, cR = g.jR * cd.nx + g.iR;
    double dGf;
    if (!g.hasL) dGf = cd.dG[cR];
    else if (!g.hasR) dGf = cd.dG[cL];
    else if (cd.face_step == 1) dGf = 2.0 * cd.dG[cL] * cd.dG[cR] / (cd.dG[cL] + cd.dG[cR]);
    else dGf = fmin(cd.dG[cL], cd.dG[cR]);
    double C[5];
    ugks_coeffs(dGf, tau, C);

    // ---- equilibrium slopes
    double aL[4], aR[4], at[4], Aa[4], w[4];
    if (g.hasL) {
        const double* WL = W + ((size_t)n * cd.nc + cL) * 4;
        double d = ax == 0 ? cd.hx[g.iL] : cd.hy[g.jL];
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = (W0[k] - WL[k]) / d / rho0;
        micro_slope(w, U0, V0, lam0f, aL);
    }
    if (g.hasR) {
        const double* WR = W + ((size_t)n * cd.nc + cR) * 4;
        double d = ax == 0 ? cd.hx[g.iR] : cd.hy[g.jR];
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = (WR[k] - W0[k]) / d / rho0;
        micro_slope(w, U0, V0, lam0f, aR);
    }
    if (!g.hasL) {
#pragma unroll
        for (int k = 0; k < 4; ++k) aL[k] = aR[k];
    }
    if (!g.hasR) {
#pragma unroll
        for (int k = 0; k < 4; ++k) aR[k] = aL[k];
    }
    w[0] = m[13] / rho0; w[1] = m[14] / rho0; w[2] = m[15] / rho0; w[3] = 0.5 * (m[16] + m[17]) / rho0;
    micro_slope(w, U0, V0, lam0f, at);

    // ---- analytic velocity sums of polynomial x interface Maxwellian
    Sums1D X, Y;
    sums1d(cd.u1, cd.wu1, cd.nu, lam0f, U0, X);
    sums1d(cd.v1, cd.wv1, cd.nv, lam0f, V0, Y);
    const double pref = rho0 * lam0f / M_PI, i2l = 0.5 / lam0f;
    auto rows = [&](int r, int& rx, int& ry) { rx = ax == 0 ? r : 0; ry = ax == 0 ? 0 : r; };
    Poly un, ut;
    un.zero(); ut.zero();
    if (ax == 0) { un.c[1][0] = 1.0; ut.c[0][1] = 1.0; } else { un.c[0][1] = 1.0; ut.c[1][0] = 1.0; }
    Poly PhL, PbL, PhR, PbR, Pht, Pbt, t1, t2;
    poly_P(aL, i2l, false, PhL); poly_P(aL, i2l, true, PbL);
    poly_P(aR, i2l, false, PhR); poly_P(aR, i2l, true, PbR);
    poly_P(at, i2l, false, Pht); poly_P(at, i2l, true, Pbt);
    // Q_side = u_n P_h(a_side) + u_t P_h(a_t),  R_side likewise with P_b
    Poly QL, RL, QR, RR, Q0, R0;
    poly_mul(un, PhL, QL); poly_mul(ut, Pht, t1);
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b < 5; ++b) QL.c[a][b] += t1.c[a][b];
    poly_mul(un, PbL, RL); poly_mul(ut, Pbt, t2);
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b < 5; ++b) RL.c[a][b] += t2.c[a][b];
    poly_mul(un, PhR, QR);
    poly_mul(un, PbR, RR);
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            QR.c[a][b] += t1.c[a][b];
            RR.c[a][b] += t2.c[a][b];
            Q0.c[a][b] = 0.5 * (QL.c[a][b] + QR.c[a][b]);
            R0.c[a][b] = 0.5 * (RL.c[a][b] + RR.c[a][b]);
        }
    // compatibility: moments of (A.psi) g0 = - moments of (u_n a_n + u_t a_t) g0
    double M[4], tmp[4];
    int rx, ry;
    if (!wall) {
        rows(1, rx, ry); mom4(QL, RL, X, rx, Y, ry, pref, i2l, M);
        rows(2, rx, ry); mom4(QR, RR, X, rx, Y, ry, pref, i2l, tmp);
#pragma unroll
        for (int k = 0; k < 4; ++k) M[k] += tmp[k];
        rows(3, rx, ry); mom4(Q0, R0, X, rx, Y, ry, pref, i2l, tmp);
#pragma unroll
        for (int k = 0; k < 4; ++k) M[k] += tmp[k];
    } else {
        mom4(QL, RL, X, 0, Y, 0, pref, i2l, M);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = -M[k] / rho0;
    micro_slope(w, U0, V0, lam0f, Aa);

    // ---- macro flux: velocity moments of the time-integrated interface distribution (Eq. macro_flux)
    // C1 term: u_n (1 + Shakhov) ; Shakhov factor s (c.q)(2 lam |c|^2 - 4) for h and (... - 2) for b
    const double sk = (1.0 - cd.pr) * 4.0 * lam0f * lam0f / (5.0 * rho0);
    Poly cq, c2, sh, sb, q1, r1;
    cq.zero(); c2.zero();
    cq.c[1][0] = sk * q0x; cq.c[0][1] = sk * q0y; cq.c[0][0] = -sk * (q0x * U0 + q0y * V0);
    c2.c[2][0] = 2.0 * lam0f; c2.c[0][2] = 2.0 * lam0f; c2.c[1][0] = -4.0 * lam0f * U0;
    c2.c[0][1] = -4.0 * lam0f * V0; c2.c[0][0] = 2.0 * lam0f * (U0 * U0 + V0 * V0);
    c2.c[0][0] -= 4.0;
    poly_mul(cq, c2, sh);                 // s (c.q)(2 lam |c|^2 - 4)
    sb = sh;
    sb.c[1][0] += 2.0 * cq.c[1][0]; sb.c[0][1] += 2.0 * cq.c[0][1]; sb.c[0][0] += 2.0 * cq.c[0][0];
    sh.c[0][0] += 1.0; sb.c[0][0] += 1.0;
    poly_mul(un, sh, q1); poly_mul(un, sb, r1);
    const int half = wall ? inc_row : 0;  // velocities carried by the integral solution
    double F1[4], F2[4], F3[4], F4[4], F5[4];
    rows(half, rx, ry);
    mom4(q1, r1, X, rx, Y, ry, pref, i2l, F1);
    // C2 term: u_n (u_n P(a_bar) + u_t P(a_t)) with a_bar = a^L for u_n > 0, a^R for u_n < 0
    Poly uQ, uR;
    if (!wall) {
        poly_mul(un, QL, uQ); poly_mul(un, RL, uR);
        rows(1, rx, ry); mom4(uQ, uR, X, rx, Y, ry, pref, i2l, F2);
        poly_mul(un, QR, uQ); poly_mul(un, RR, uR);
        rows(2, rx, ry); mom4(uQ, uR, X, rx, Y, ry, pref, i2l, tmp);
#pragma unroll
        for (int k = 0; k < 4; ++k) F2[k] += tmp[k];
    } else {
        poly_mul(un, QL, uQ); poly_mul(un, RL, uR);
        rows(inc_row, rx, ry); mom4(uQ, uR, X, rx, Y, ry, pref, i2l, F2);
    }
    // C3 term: u_n P(A)
    Poly PhA, PbA;
    poly_P(Aa, i2l, false, PhA); poly_P(Aa, i2l, true, PbA);
    poly_mul(un, PhA, uQ); poly_mul(un, PbA, uR);
    rows(half, rx, ry);
    mom4(uQ, uR, X, rx, Y, ry, pref, i2l, F3);
    // C4 term: u_n psi h_0 (reconstruction; incident velocities only at a wall)
    if (ax == 0) { F4[0] = A[1]; F4[1] = A[3]; F4[2] = A[4]; F4[3] = 0.5 * (A[6] + A[8] + A[11]); }
    else { F4[0] = A[2]; F4[1] = A[4]; F4[2] = A[5]; F4[3] = 0.5 * (A[7] + A[9] + A[12]); }
    // C5 term: u_n (u_n sigma_n + u_t sigma_t) psi
    F5[0] = m[18]; F5[1] = m[19]; F5[2] = m[20]; F5[3] = 0.5 * (m[21] + m[22]);
    double I[4], F[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) I[k] = C[0] * F1[k] + C[1] * F2[k] + C[2] * F3[k] + C[3] * F4[k] + C[4] * F5[k];
    double rhow = 0.0;
    if (!wall) {
#pragma unroll
        for (int k = 0; k < 4; ++k) F[k] = I[k] / dGf;
    } else {
        // impermeability (Eq. rho_wall) with the time-integrated incident flux; reflected part rho_w H_w
        rhow = -nin * I[0] / (dGf * Dw);
        Poly one;
        one.zero();
        one.c[0][0] = 1.0;
        Poly uu;
        poly_mul(un, one, uu);
        int wx = ax == 0 ? ref_row : 0, wy = ax == 0 ? 0 : ref_row;
        mom4(uu, uu, Xw, wx, Yw, wy, prefw, i2lw, tmp);
#pragma unroll
        for (int k = 0; k < 4; ++k) F[k] = I[k] / dGf + rhow * tmp[k];
    }
    double* fo = cd.fflux + (size_t)item * 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) fo[k] = F[k];

    // ---- parameters of the micro flux
    T* pp = cd.fpar + (size_t)item * NP;
    double e[13];
    eq_params(rho0, U0, V0, lam0f, cd.lam0, cd.pr, q0x, q0y, e);
#pragma unroll
    for (int k = 0; k < 13; ++k) pp[k] = T(e[k]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        pp[F_AL + k] = T(aL[k]);
        pp[F_AR + k] = T(aR[k]);
        pp[F_AT + k] = T(at[k]);
        pp[F_A + k] = T(Aa[k]);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) pp[F_C + k] = T(C[k] / dGf);
    if (wall) {
        eq_params(rhow, Uw, Vw, lamw, cd.lam0, 1.0, 0.0, 0.0, e);
#pragma unroll
        for (int k = 0; k < 8; ++k) pp[F_WR + k] = T(e[k]);
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) pp[F_WR + k] = T(0);
    }
    pp[F_NIN] = T(nin);
}

// ------------------------------------------------------------------------------ local pseudo-time step

// Eqs. dt_hb, nu_conv: dG_i = CFL / (max_n nu_conv,i,n + omega N_H)
template <typename T>
__device__ __forceinline__ double local_step(const CaseDev<T>& cd, const double* W, int c, int i, int j)
{
    const double dx = 2.0 * cd.hx[i], dy = 2.0 * cd.hy[j];
    double numax = 0.0;
    for (int n = 0; n < cd.nt; ++n) {
        double rho, U, V, lam;
        prim(W + ((size_t)n * cd.nc + c) * 4, rho, U, V, lam);
        double cs = sqrt(cd.gam / (2.0 * lam));
        double ut = fmax(fabs(cd.umax), fabs(U)) + cs;
        double vt = fmax(fabs(cd.vmax), fabs(V)) + cs;
        numax = fmax(numax, (dy * ut + dx * vt) / (dx * dy));
    }
    return cd.cfl / (numax + cd.omega * cd.nh);
}

template <typename T>
__global__ void k_steps(Batch<T> B)
{
    int cs = find_case(B.off, B.ncases, blockIdx.x);
    const CaseDev<T>& cd = B.cases[cs];
    int c = (blockIdx.x - B.off[cs]) * blockDim.x + threadIdx.x;
    if (c >= cd.nc) return;
    cd.dG[c] = local_step(cd, cd.W[cd.st->parity], c, c % cd.nx, c / cd.nx);
}

// ------------------------------------------------------------------------------ K3 macro update

template <typename T>
__global__ void __launch_bounds__(K3_THREADS) k3_macro(Batch<T> B)
{
    int cs = find_case(B.off, B.ncases, blockIdx.x);
    const CaseDev<T>& cd = B.cases[cs];
    if (!cd.st->active) return;
    const int lb = blockIdx.x - B.off[cs];
    const int c = lb * K3_THREADS + threadIdx.x;
    const int nt = cd.nt, nc = cd.nc;
    const int p = cd.st->parity;
    double r2[4] = {0, 0, 0, 0};
    if (c < nc) {
        const int i = c % cd.nx, j = c / cd.nx;
        const double* W = cd.W[p];
        double* Wn = cd.W[p ^ 1];
        const int fL = j * (cd.nx + 1) + i, fR = fL + 1, fB = cd.nfx + j * cd.nx + i, fT = fB + cd.nx;
        const double dx = 2.0 * cd.hx[i], dy = 2.0 * cd.hy[j], area = dx * dy;
        const double dG = cd.dG[c];
        double Wc[MAXNT][4];
        for (int n = 0; n < nt; ++n)
#pragma unroll
            for (int k = 0; k < 4; ++k) Wc[n][k] = W[((size_t)n * nc + c) * 4 + k];
        for (int n = 0; n < nt; ++n) {
            const double* FL = cd.fflux + ((size_t)fL * nt + n) * 4;
            const double* FR = cd.fflux + ((size_t)fR * nt + n) * 4;
            const double* FB = cd.fflux + ((size_t)fB * nt + n) * 4;
            const double* FT = cd.fflux + ((size_t)fT * nt + n) * 4;
            double wn[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                double div = (dy * (FR[k] - FL[k]) + dx * (FT[k] - FB[k])) / area;
                double ew = 0.0;
                for (int d = 1; d <= cd.nh; ++d) {
                    int nm = n - d; if (nm < 0) nm += nt;
                    int np = n + d; if (np >= nt) np -= nt;
                    ew += cd.e[d] * (Wc[nm][k] - Wc[np][k]);
                }
                wn[k] = Wc[n][k] - dG * (div + cd.omega * ew);
                Wn[((size_t)n * nc + c) * 4 + k] = wn[k];
            }
            if (n == 0) {
#pragma unroll
                for (int k = 0; k < 4; ++k) { double d = wn[k] - Wc[0][k]; r2[k] = d * d; }
            }
            // collision coefficients of Eq. fv_h with h+ from W^k and W^{k+1} and the heat flux q^k
            double A[13];
            const double* cm = cd.cmom + ((size_t)c * nt + n) * NCM;
#pragma unroll
            for (int k = 0; k < 13; ++k) A[k] = cm[k] + cd.refmom[k];
            double r0, U0, V0, l0, r1, U1, V1, l1, qx, qy;
            prim(Wc[n], r0, U0, V0, l0);
            prim(wn, r1, U1, V1, l1);
            heat_flux_raw(A, U0, V0, qx, qy);
            const double t0 = relax_time(cd.mu0, cd.w_vss, cd.lam0, r0, l0);
            const double t1 = relax_time(cd.mu0, cd.w_vss, cd.lam0, r1, l1);
            double e0[13], e1[13];
            eq_params(r0, U0, V0, l0, cd.lam0, cd.pr, qx, qy, e0);
            eq_params(r1, U1, V1, l1, cd.lam0, cd.pr, qx, qy, e1);
            T* cp = cd.cpar + ((size_t)c * nt + n) * NCP;
#pragma unroll
            for (int k = 0; k < 13; ++k) { cp[C_EQ0 + k] = T(e0[k]); cp[C_EQ1 + k] = T(e1[k]); }
            const double D = 1.0 + 0.5 * dG / t1;
            cp[C_KSELF] = T((1.0 - 0.5 * dG / t0) / D);
            cp[C_KE] = T(dG * cd.omega / D);
            cp[C_KP1] = T(0.5 * dG / (t1 * D));
            cp[C_KP0] = T(0.5 * dG / (t0 * D));
            cp[C_KDX] = T(dG / (dx * D));
            cp[C_KDY] = T(dG / (dy * D));
        }
        cd.dG[c] = local_step(cd, Wn, c, i, j);
    }
    // deterministic block reduction of the level-0 residual partials
    __shared__ double red[K3_THREADS][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) red[threadIdx.x][k] = r2[k];
    __syncthreads();
    for (int s = K3_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < 4; ++k) red[threadIdx.x][k] += red[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) cd.rpart[lb * 4 + k] = red[0][k];
}

// ------------------------------------------------------------------------------ K4 micro update

template <typename T>
struct FluxOut {
    T h, b;
};

// micro flux of one face at one velocity, delta form (Eq. micro_flux minus u_n H_ref)
template <typename T>
__device__ __forceinline__ FluxOut<T> micro_flux(const CaseDev<T>& cd, const T* dh, const T* db, int f, int n, int vb,
                                                 int lane, T u, T v, T u2, T href)
{
    const FaceGeo g = face_geo(cd, f);
    const T* fp = cd.fpar + ((size_t)f * cd.nt + n) * NP;
    const T un = g.axis == 0 ? u : v, ut = g.axis == 0 ? v : u;
    FluxOut<T> o;
    Up<T> r = upwind(cd, dh, db, g, vb, n, lane, un);
    if (r.mode == 1) {
        T H, dH, dB, Hp, Bp;
        eq_eval(fp, u, v, u2, href, H, dH, dB, Hp, Bp);
        const T* ab = un > T(0) ? fp + F_AL : fp + F_AR;
        const T* at = fp + F_AT;
        const T* A = fp + F_A;
        const T q = T(0.5) * (u2 + fp[F_I2L]);
        const T Pa = ab[0] + ab[1] * u + ab[2] * v + ab[3] * q;
        const T Pt = at[0] + at[1] * u + at[2] * v + at[3] * q;
        const T PA = A[0] + A[1] * u + A[2] * v + A[3] * q;
        const T C2 = fp[F_C + 1], C3 = fp[F_C + 2];
        const T Ph = C2 * (un * Pa + ut * Pt) + C3 * PA;
        const T Pb = Ph + (C2 * (un * ab[3] + ut * at[3]) + C3 * A[3]) * fp[F_I2L];
        o.h = un * (fp[F_C] * (dH + Hp) + Ph * H + fp[F_C + 3] * r.d0 + fp[F_C + 4] * (un * r.sn + ut * r.st));
        o.b = un * (fp[F_C] * (dB + Bp) + Pb * H * fp[F_I2L] + fp[F_C + 3] * r.e0 +
                    fp[F_C + 4] * (un * r.snb + ut * r.stb));
    } else if (r.mode == 2) {
        const T* w = fp + F_WR;
        T D = w[2] * u2 + w[3] * u + w[4] * v - w[5];
        T dHw = href * (w[1] + w[0] * t_expm1<T>(D));
        o.h = un * dHw;
        o.b = un * (dHw * w[6] + href * w[7]);
    } else {
        o.h = T(0);
        o.b = T(0);
    }
    return o;
}

template <typename T>
__global__ void __launch_bounds__(256) k4_micro(Batch<T> B)
{
    int cs = find_case(B.off, B.ncases, blockIdx.x);
    const CaseDev<T>& cd = B.cases[cs];
    if (!cd.st->active) return;
    const int lane = threadIdx.x & 31;
    const int item = (blockIdx.x - B.off[cs]) * 8 + (threadIdx.x >> 5);
    if (item >= cd.nc * cd.nvb) return;
    const int c = item % cd.nc, vb = item / cd.nc;
    const int i = c % cd.nx, j = c / cd.nx;
    const int nc = cd.nc, nt = cd.nt, nh = cd.nh;
    const int p = cd.st->parity;
    const T* dh = cd.dh[p];
    const T* db = cd.db[p];
    T* oh = cd.dh[p ^ 1];
    T* ob = cd.db[p ^ 1];
    const int a = vb * VB + lane;
    const T u = cd.tu[a], v = cd.tv[a], href = cd.thref[a];
    const T u2 = u * u + v * v;
    const int fL = j * (cd.nx + 1) + i, fR = fL + 1, fB = cd.nfx + j * cd.nx + i, fT = fB + cd.nx;
    const T* hcell = dh + sidx(nc, nt, vb, c, 0, lane);     // level n at hcell[32 n]
    const T* bcell = db + sidx(nc, nt, vb, c, 0, lane);
#pragma unroll 1
    for (int n = 0; n < nt; ++n) {
        const T* cp = cd.cpar + ((size_t)c * nt + n) * NCP;
        FluxOut<T> xl = micro_flux(cd, dh, db, fL, n, vb, lane, u, v, u2, href);
        FluxOut<T> xr = micro_flux(cd, dh, db, fR, n, vb, lane, u, v, u2, href);
        FluxOut<T> yb = micro_flux(cd, dh, db, fB, n, vb, lane, u, v, u2, href);
        FluxOut<T> yt = micro_flux(cd, dh, db, fT, n, vb, lane, u, v, u2, href);
        // spectral source (E dh)_n = sum_d e_d (dh_{n-d} - dh_{n+d})
        T eh = T(0), eb = T(0);
        for (int d = 1; d <= nh; ++d) {
            int nm = n - d; if (nm < 0) nm += nt;
            int np = n + d; if (np >= nt) np -= nt;
            eh += T(cd.e[d]) * (hcell[nm * VB] - hcell[np * VB]);
            eb += T(cd.e[d]) * (bcell[nm * VB] - bcell[np * VB]);
        }
        T H1, dH1, dB1, Hp1, Bp1, H0, dH0, dB0, Hp0, Bp0;
        eq_eval(cp + C_EQ1, u, v, u2, href, H1, dH1, dB1, Hp1, Bp1);
        eq_eval(cp + C_EQ0, u, v, u2, href, H0, dH0, dB0, Hp0, Bp0);
        const T kdx = cp[C_KDX], kdy = cp[C_KDY];
        const T h0 = hcell[n * VB], b0 = bcell[n * VB];
        T nh_ = cp[C_KSELF] * h0 - kdx * (xr.h - xl.h) - kdy * (yt.h - yb.h) - cp[C_KE] * eh +
                cp[C_KP1] * (dH1 + Hp1) + cp[C_KP0] * (dH0 + Hp0);
        T nb_ = cp[C_KSELF] * b0 - kdx * (xr.b - xl.b) - kdy * (yt.b - yb.b) - cp[C_KE] * eb +
                cp[C_KP1] * (dB1 + Bp1) + cp[C_KP0] * (dB0 + Bp0);
        oh[sidx(nc, nt, vb, c, n, lane)] = nh_;
        ob[sidx(nc, nt, vb, c, n, lane)] = nb_;
    }
}

// ------------------------------------------------------------------------------ K5 residual / status

template <typename T>
__global__ void k5_finish(const CaseDev<T>* cases, int ncases, const int* k3off)
{
    int cs = blockIdx.x;
    if (cs >= ncases) return;
    const CaseDev<T>& cd = cases[cs];
    CaseStatus* st = cd.st;
    if (!st->active) return;
    const int nb = k3off[cs + 1] - k3off[cs];
    __shared__ double part[4][32];
    const int lane = threadIdx.x;      // 32 threads
    double s[4] = {0, 0, 0, 0};
    for (int b = lane; b < nb; b += 32)
#pragma unroll
        for (int k = 0; k < 4; ++k) s[k] += cd.rpart[b * 4 + k];
#pragma unroll
    for (int k = 0; k < 4; ++k) part[k][lane] = s[k];
    __syncwarp();
    if (lane == 0) {
        double R[4];
        bool bad = false;
        for (int k = 0; k < 4; ++k) {
            double t = 0.0;
            for (int l = 0; l < 32; ++l) t += part[k][l];
            R[k] = sqrt(t / cd.nc);
            if (!(R[k] <= 1e10)) bad = true;   // also catches NaN
            st->last[k] = R[k];
            cd.rhist[(st->iters % RING) * 4 + k] = R[k];
        }
        st->iters += 1;
        st->iters_call += 1;
        st->parity ^= 1;
        if (bad) {
            st->diverged = 1;
            st->active = 0;
        } else if (*cd.tol > 0.0 && st->iters >= 10 && R[0] <= *cd.tol) {
            st->active = 0;
        }
    }
}

// ------------------------------------------------------------------------------ conversions and fields

// canonical FP64 level array (stage[c][a], a < nvel) -> delta-form internal layout of one level
template <typename T>
__global__ void k_set_level(CaseDev<T> cd, int n, int which, const double* stage)
{
    size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t tot = (size_t)cd.nc * cd.nvb * VB;
    if (k >= tot) return;
    int lane = k & 31;
    size_t r = k >> 5;
    int c = r % cd.nc, vb = r / cd.nc;
    int a = vb * VB + lane;
    double val = 0.0;
    if (a < cd.nvel) {
        double href = (cd.lam0 / M_PI) * exp(-cd.lam0 * (cd.vu[a] * cd.vu[a] + cd.vv[a] * cd.vv[a]));
        double rv = which == 0 ? href : href * 0.5 / cd.lam0;
        val = stage[(size_t)c * cd.nvel + a] - rv;
    }
    T* dst = which == 0 ? cd.dh[cd.st->parity] : cd.db[cd.st->parity];
    dst[sidx(cd.nc, cd.nt, vb, c, n, lane)] = T(val);
}

template <typename T>
__global__ void k_get_level(CaseDev<T> cd, int n, int which, double* stage)
{
    size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t tot = (size_t)cd.nc * cd.nvb * VB;
    if (k >= tot) return;
    int lane = k & 31;
    size_t r = k >> 5;
    int c = r % cd.nc, vb = r / cd.nc;
    int a = vb * VB + lane;
    if (a >= cd.nvel) return;
    double href = (cd.lam0 / M_PI) * exp(-cd.lam0 * (cd.vu[a] * cd.vu[a] + cd.vv[a] * cd.vv[a]));
    double rv = which == 0 ? href : href * 0.5 / cd.lam0;
    const T* src = which == 0 ? cd.dh[cd.st->parity] : cd.db[cd.st->parity];
    stage[(size_t)c * cd.nvel + a] = (double)src[sidx(cd.nc, cd.nt, vb, c, n, lane)] + rv;
}

// uniform reduced Maxwellian (rho, U, V, T) on every level, delta form; W = its continuous moments
template <typename T>
__global__ void k_init_uniform(CaseDev<T> cd, double rho, double U, double V, double Tt)
{
    size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t tot = (size_t)cd.nc * cd.nvb * VB * cd.nt;
    const int p = cd.st->parity;
    if (k < (size_t)cd.nc * cd.nt) {
        double* W = cd.W[p] + k * 4;
        W[0] = rho; W[1] = rho * U; W[2] = rho * V; W[3] = 0.5 * rho * (U * U + V * V) + 0.75 * rho * Tt;
    }
    if (k >= tot) return;
    int lane = k & 31;
    size_t r = k >> 5;
    int n = r % cd.nt;
    r /= cd.nt;
    int c = r % cd.nc, vb = r / cd.nc;
    int a = vb * VB + lane;
    double dhv = 0.0, dbv = 0.0;
    if (a < cd.nvel) {
        double uu = cd.vu[a], vv = cd.vv[a];
        double lam = cd.lam0 / Tt;
        double H = rho * (lam / M_PI) * exp(-lam * ((uu - U) * (uu - U) + (vv - V) * (vv - V)));
        double href = (cd.lam0 / M_PI) * exp(-cd.lam0 * (uu * uu + vv * vv));
        dhv = H - href;
        dbv = H * 0.5 / lam - href * 0.5 / cd.lam0;
    }
    cd.dh[p][sidx(cd.nc, cd.nt, vb, c, n, lane)] = T(dhv);
    cd.db[p][sidx(cd.nc, cd.nt, vb, c, n, lane)] = T(dbv);
}

// fields of one level from the moments of h, b: out[f * nc + c], f = rho, U, V, T, tau_xy, qx, qy, p
template <typename T>
__global__ void k_fields(CaseDev<T> cd, int n, double* out)
{
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= cd.nc) return;
    const int p = cd.st->parity;
    double A[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) A[k] = 0.0;
    for (int vb = 0; vb < cd.nvb; ++vb) {
        int a = vb * VB + lane;
        double w = cd.vw[a], u = cd.vu[a], v = cd.vv[a];
        size_t id = sidx(cd.nc, cd.nt, vb, c, n, lane);
        double wd = w * (double)cd.dh[p][id], we = w * (double)cd.db[p][id];
        A[0] += wd; A[1] += wd * u; A[2] += wd * v; A[3] += wd * u * u; A[4] += wd * u * v; A[5] += wd * v * v;
        A[6] += wd * u * u * u; A[7] += wd * u * u * v; A[8] += wd * u * v * v; A[9] += wd * v * v * v;
        A[10] += we; A[11] += we * u; A[12] += we * v;
    }
#pragma unroll
    for (int k = 0; k < 13; ++k) A[k] = warp_sum(A[k]) + cd.refmom[k];
    if (lane == 0) {
        double Wm[4] = {A[0], A[1], A[2], 0.5 * (A[3] + A[5] + A[10])};
        double rho, U, V, lam, qx, qy;
        prim(Wm, rho, U, V, lam);
        heat_flux_raw(A, U, V, qx, qy);
        double txy = A[4] - V * A[1] - U * A[2] + U * V * A[0];
        const int nc = cd.nc;
        out[0 * nc + c] = rho;
        out[1 * nc + c] = U;
        out[2 * nc + c] = V;
        out[3 * nc + c] = cd.lam0 / lam;
        out[4 * nc + c] = txy;
        out[5 * nc + c] = qx;
        out[6 * nc + c] = qy;
        out[7 * nc + c] = rho / (2.0 * lam);
    }
}

// Eq. dft_general on fields of all levels (lv[n][8][nc]) -> re/im of harmonic k
__global__ void k_dft(const double* lv, int nt, int nc, int k, double* re, double* im)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8 * nc) return;
    double sr = 0.0, si = 0.0;
    for (int n = 0; n < nt; ++n) {
        double th = 2.0 * M_PI * (double)k * (double)n / (double)nt;
        double val = lv[(size_t)n * 8 * nc + idx];
        sr += val * cos(th);
        si -= val * sin(th);
    }
    re[idx] = sr / nt;
    im[idx] = si / nt;
}

}  // namespace hb
