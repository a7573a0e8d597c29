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

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
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

// delta-form velocity sum sum_a w_a u^p v^q (H0 - H_ref) over the subset given by the rows (rx, ry), from the
// reference 1-D sums X0, Y0 (FP64) and the table sums dX, dY = sum w x^p e^{-lam0 x^2} expm1(..):
//   (lam0/pi) [(r - 1) X0 Y0 + r (dX Y0 + X0 dY + dX dY)]
template <typename T>
__device__ __forceinline__ double dsum(const double* X0, const double* Y0, const SumsT<T>& dX, const SumsT<T>& dY,
                                       int rx, int ry, int p, int q, double r, double lam0)
{
    const double x0 = X0[rx * 9 + p], y0 = Y0[ry * 9 + q];
    const double dx = (double)dX.s[rx][p], dy = (double)dY.s[ry][q];
    return lam0 / M_PI * ((r - 1.0) * x0 * y0 + r * (dx * y0 + x0 * dy + dx * dy));
}

// Velocity sums of the upwinded reconstruction at face g, level n, from the half-face sums of its cells: at an
// interior face the low-side cell's u_n > 0 class plus the high-side cell's u_n < 0 class; at a wall the
// interior cell's class moving into the wall, with the tangential-slope sums (13..17) over both classes.
template <typename T>
__device__ __forceinline__ void face_sums(const CaseDev<T>& cd, const FaceGeo& g, int n, double* m)
{
    const int sp = g.axis == 0 ? 0 : 2;                  // half-face slot of the u_n > 0 class, sp + 1: u_n < 0
    const size_t stride = (size_t)cd.nt * 4 * NM;
    const double* L = g.hasL ? cd.hmom + (size_t)(g.jL * cd.nx + g.iL) * stride + (size_t)n * 4 * NM : nullptr;
    const double* R = g.hasR ? cd.hmom + (size_t)(g.jR * cd.nx + g.iR) * stride + (size_t)n * 4 * NM : nullptr;
    if (g.hasL && g.hasR) {
        for (int k = 0; k < NM; ++k) m[k] = L[sp * NM + k] + R[(sp + 1) * NM + k];
    } else if (g.hasR) {
        for (int k = 0; k < NM; ++k) m[k] = R[(sp + 1) * NM + k];
        for (int k = 13; k < 18; ++k) m[k] += R[sp * NM + k];
    } else {
        for (int k = 0; k < NM; ++k) m[k] = L[sp * NM + k];
        for (int k = 13; k < 18; ++k) m[k] += L[(sp + 1) * NM + k];
    }
}

template <typename T>
__global__ void __launch_bounds__(128) k2_face_params(Batch<T> B)
{
    int cs = find_case(B.off, B.ncases, blockIdx.x);
    const CaseDev<T>& cd = B.cases[cs];
    if (!cd.st->active || *(volatile int*)cd.err) return;
    const int item = (blockIdx.x - B.off[cs]) * blockDim.x + threadIdx.x;
    const int nt = cd.nt;
    if (item >= cd.nf * nt) return;
    const int f = item / nt, n = item - f * nt;
    const FaceGeo g = face_geo(cd, f);
    const int p = cd.st->parity;
    const double* W = cd.W[p];
    double m[NM];                                        // velocity sums of the reconstructed deviations
    face_sums(cd, g, n, m);
    const bool wall = !(g.hasL && g.hasR);
    const double nin = wall ? (g.hasL ? -1.0 : 1.0) : 0.0;
    const int ax = g.axis;
    const int inc_row = nin > 0 ? 2 : 1;      // incident: u_n nin < 0
    int refset = 0;
    if (wall) refset = ax == 0 ? (nin > 0 ? 2 : 1) : (nin > 0 ? 4 : 3);
    double A[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) A[k] = m[k] + cd.refmom[refset * 13 + k];

    // ---- diffuse wall: free-transport density estimate (Eq. rho_wall) and the mixed kinetic average
    const int wsl = wall_slot(cd, n);
    const double* wc = wall ? cd.wconst + ((size_t)g.wall * cd.nslot + wsl) * WCN : nullptr;
    double Amix[13], Dw = 1.0, rhow0 = 0.0;
#pragma unroll
    for (int k = 0; k < 13; ++k) Amix[k] = A[k];
    if (wall) {
        Dw = wc[13];                                        // sum over reflected velocities of w |u_n| H_w
        rhow0 = -nin * (ax == 0 ? A[1] : A[2]) / Dw;
#pragma unroll
        for (int k = 0; k < 13; ++k) Amix[k] = A[k] + rhow0 * wc[k];
    }

    // ---- interface Maxwellian from the kinetic average, heat flux, relaxation time
    double W0[4] = {Amix[0], Amix[1], Amix[2], 0.5 * (Amix[3] + Amix[5] + Amix[10])};
    double rho0, U0, V0, lamf;
    prim(W0, rho0, U0, V0, lamf);
    double q0x, q0y;
    heat_flux_raw(Amix, U0, V0, q0x, q0y);
    const double tau = relax_time(cd.mu0, cd.w_vss, cd.lam0, rho0, lamf);

    // ---- face step (Eq. dt_face) and time-integration weights (Eq. C_coeffs)
    const int cL = g.jL * cd.nx + g.iL, cR = g.jR * cd.nx + g.iR;
    double dGf;
    if (!g.hasL) dGf = cd.dG[cR];
    else if (!g.hasR) dGf = cd.dG[cL];
    else if (cd.face_step == 1) dGf = 2.0 * cd.dG[cL] * cd.dG[cR] / (cd.dG[cL] + cd.dG[cR]);
    else dGf = fmin(cd.dG[cL], cd.dG[cR]);
    T Ct[5];
    ugks_coeffs<T>(T(dGf), T(tau), Ct);
    double C[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) C[k] = (double)Ct[k];

    // ---- equilibrium slopes a^L, a^R (normal), a_t (tangential)
    double aL[4], aR[4], at[4], Aa[4], w[4];
    if (g.hasL) {
        const double* WL = W + ((size_t)n * cd.nc + cL) * 4;
        const double d = ax == 0 ? cd.hx[g.iL] : cd.hy[g.jL];
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = (W0[k] - WL[k]) / d / rho0;
        micro_slope(w, U0, V0, lamf, aL);
    }
    if (g.hasR) {
        const double* WR = W + ((size_t)n * cd.nc + cR) * 4;
        const double d = ax == 0 ? cd.hx[g.iR] : cd.hy[g.jR];
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = (WR[k] - W0[k]) / d / rho0;
        micro_slope(w, U0, V0, lamf, aR);
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
    micro_slope(w, U0, V0, lamf, at);

    // ---- separable table of the interface Maxwellian and its 1-D sums
    const int nu = cd.nu, nv = cd.nv, nuv = nu + nv;
    T* tb = cd.ftab + (size_t)item * nuv;
    SumsT<T> dX, dY;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 9; ++q) { dX.s[r][q] = T(0); dY.s[r][q] = T(0); }
    {
        const T dl = T(cd.lam0 - lamf);
        T tl = T(2.0 * lamf * U0), l2 = T(lamf * U0 * U0);
        // the sums of the three node classes (positive, negative, zero) in registers: a node adds its term to
        // its own class and zero to the other two
        T sp_[9], sn_[9], sz_[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) { sp_[q] = T(0); sn_[q] = T(0); sz_[q] = T(0); }
        for (int k = 0; k < nu; ++k) {
            const T x = cd.tu1[k];
            const T e = t_expm1<T>(dl * x * x + tl * x - l2);
            tb[k] = e;
            const T ep = x > T(0) ? e : T(0), en = x < T(0) ? e : T(0), ez = x == T(0) ? e : T(0);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const T wq = cd.wxr[q * nu + k];
                sp_[q] += wq * ep; sn_[q] += wq * en; sz_[q] += wq * ez;
            }
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) { dX.s[1][q] = sp_[q]; dX.s[2][q] = sn_[q]; dX.s[3][q] = sz_[q]; }
#pragma unroll
        for (int q = 0; q < 9; ++q) { sp_[q] = T(0); sn_[q] = T(0); sz_[q] = T(0); }
        tl = T(2.0 * lamf * V0);
        l2 = T(lamf * V0 * V0);
        for (int k = 0; k < nv; ++k) {
            const T y = cd.tv1[k];
            const T e = t_expm1<T>(dl * y * y + tl * y - l2);
            tb[nu + k] = e;
            const T ep = y > T(0) ? e : T(0), en = y < T(0) ? e : T(0), ez = y == T(0) ? e : T(0);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const T wq = cd.wyr[q * nv + k];
                sp_[q] += wq * ep; sn_[q] += wq * en; sz_[q] += wq * ez;
            }
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) { dY.s[1][q] = sp_[q]; dY.s[2][q] = sn_[q]; dY.s[3][q] = sz_[q]; }
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            dX.s[0][q] = dX.s[1][q] + dX.s[2][q] + dX.s[3][q];
            dY.s[0][q] = dY.s[1][q] + dY.s[2][q] + dY.s[3][q];
        }
    }
    // full 1-D sums of the interface Maxwellian (reference + table part)
    SumsT<T> X, Y;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            X.s[r][q] = cd.xr0t[r * 9 + q] + dX.s[r][q];
            Y.s[r][q] = cd.yr0t[r * 9 + q] + dY.s[r][q];
        }
    const T pref = T(rho0 * lamf / M_PI), i2l = T(0.5 / lamf);
    auto rows = [&](int r, int& rx, int& ry) { rx = ax == 0 ? r : 0; ry = ax == 0 ? 0 : r; };
    // u_n and u_t as the axis a product by them shifts a polynomial along (0: u, 1: v)
    const int axn = ax, axt = 1 - ax;
    PolyT<T> PhL, PbL, PhR, PbR, Pht, Pbt, t1, t2;
    poly_P<T>(aL, 0.5 / lamf, false, PhL); poly_P<T>(aL, 0.5 / lamf, true, PbL);
    poly_P<T>(aR, 0.5 / lamf, false, PhR); poly_P<T>(aR, 0.5 / lamf, true, PbR);
    poly_P<T>(at, 0.5 / lamf, false, Pht); poly_P<T>(at, 0.5 / lamf, true, Pbt);
    // Q_side = u_n P_h(a_side) + u_t P_h(a_t),  R_side likewise with P_b
    PolyT<T> QL, RL, QR, RR, Q0, R0;
    poly_shift(axn, PhL, QL); poly_shift(axt, Pht, t1);
    poly_shift(axn, PbL, RL); poly_shift(axt, Pbt, t2);
    poly_shift(axn, PhR, QR);
    poly_shift(axn, PbR, RR);
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            QL.c[a][b] += t1.c[a][b];
            RL.c[a][b] += t2.c[a][b];
            QR.c[a][b] += t1.c[a][b];
            RR.c[a][b] += t2.c[a][b];
            Q0.c[a][b] = T(0.5) * (QL.c[a][b] + QR.c[a][b]);
            R0.c[a][b] = T(0.5) * (RL.c[a][b] + RR.c[a][b]);
        }
    // compatibility: moments of (A.psi) g0 = - moments of (u_n a_n + u_t a_t) g0
    T M[4], tmp[4];
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
    for (int k = 0; k < 4; ++k) w[k] = -(double)M[k] / rho0;
    micro_slope(w, U0, V0, lamf, Aa);

    // ---- macro flux deviation (Eq. macro_flux minus the flux of H_ref, which cancels in every cell balance)
    // Shakhov factor s (c.q)(2 lam |c|^2 - 4) and the b-part addition 2 s (c.q)
    double sp[13];
    shakhov_poly((1.0 - cd.pr) * 4.0 * lamf * lamf / (5.0 * rho0), q0x, q0y, U0, V0, lamf, sp);
    PolyT<T> shk, cq2, sb;
    shk.zero(); cq2.zero();
    shk.c[0][0] = T(sp[0]); shk.c[1][0] = T(sp[1]); shk.c[0][1] = T(sp[2]); shk.c[2][0] = T(sp[3]);
    shk.c[1][1] = T(sp[4]); shk.c[0][2] = T(sp[5]); shk.c[3][0] = T(sp[6]); shk.c[2][1] = T(sp[7]);
    shk.c[1][2] = T(sp[8]); shk.c[0][3] = T(sp[9]);
    cq2.c[0][0] = T(sp[10]); cq2.c[1][0] = T(sp[11]); cq2.c[0][1] = T(sp[12]);
    sb = shk;
    sb.c[0][0] += cq2.c[0][0]; sb.c[1][0] += cq2.c[1][0]; sb.c[0][1] += cq2.c[0][1];
    const int half = wall ? inc_row : 0;  // velocities carried by the integral solution
    PolyT<T> q1, r1;
    poly_shift(axn, shk, q1); poly_shift(axn, sb, r1);
    T F1s[4], F2[4], F3[4];
    rows(half, rx, ry);
    mom4(q1, r1, X, rx, Y, ry, pref, i2l, F1s);
    // C2 term: u_n (u_n P(a_bar) + u_t P(a_t)) with a_bar = a^L for u_n > 0, a^R for u_n < 0
    PolyT<T> uQ, uR;
    if (!wall) {
        poly_shift(axn, QL, uQ); poly_shift(axn, RL, uR);
        rows(1, rx, ry); mom4(uQ, uR, X, rx, Y, ry, pref, i2l, F2);
        poly_shift(axn, QR, uQ); poly_shift(axn, RR, uR);
        rows(2, rx, ry); mom4(uQ, uR, X, rx, Y, ry, pref, i2l, tmp);
#pragma unroll
        for (int k = 0; k < 4; ++k) F2[k] += tmp[k];
    } else {
        poly_shift(axn, QL, uQ); poly_shift(axn, RL, uR);
        rows(inc_row, rx, ry); mom4(uQ, uR, X, rx, Y, ry, pref, i2l, F2);
    }
    // C3 term: u_n P(A)
    PolyT<T> PhA, PbA;
    poly_P<T>(Aa, 0.5 / lamf, false, PhA); poly_P<T>(Aa, 0.5 / lamf, true, PbA);
    poly_shift(axn, PhA, uQ); poly_shift(axn, PbA, uR);
    rows(half, rx, ry);
    mom4(uQ, uR, X, rx, Y, ry, pref, i2l, F3);
    // C1 term, Maxwellian part: moments of u_n psi (H0 - H_ref, B0 - B_ref), in FP64 from the reference sums
    const double rr = rho0 * lamf / cd.lam0, i2ld = 0.5 / lamf, di2l = 0.5 / lamf - 0.5 / cd.lam0;
    double dF1[4];
    {
        rows(half, rx, ry);
        auto S = [&](int pp, int qq) { return dsum(cd.xr0, cd.yr0, dX, dY, rx, ry, pp, qq, rr, cd.lam0); };
        auto Sr = [&](int pp, int qq) { return cd.lam0 / M_PI * cd.xr0[rx * 9 + pp] * cd.yr0[ry * 9 + qq]; };
        if (ax == 0) {
            const double s10 = S(1, 0);
            dF1[0] = s10; dF1[1] = S(2, 0); dF1[2] = S(1, 1);
            dF1[3] = 0.5 * (S(3, 0) + S(1, 2)) + 0.5 * (i2ld * s10 + di2l * Sr(1, 0));
        } else {
            const double s01 = S(0, 1);
            dF1[0] = s01; dF1[1] = S(1, 1); dF1[2] = S(0, 2);
            dF1[3] = 0.5 * (S(2, 1) + S(0, 3)) + 0.5 * (i2ld * s01 + di2l * Sr(0, 1));
        }
    }
    // C4 term: u_n psi (h_0 - H_ref) (reconstruction; incident velocities only at a wall); C5 term
    double F4[4], F5[4];
    if (ax == 0) { F4[0] = m[1]; F4[1] = m[3]; F4[2] = m[4]; F4[3] = 0.5 * (m[6] + m[8] + m[11]); }
    else { F4[0] = m[2]; F4[1] = m[4]; F4[2] = m[5]; F4[3] = 0.5 * (m[7] + m[9] + m[12]); }
    F5[0] = m[18]; F5[1] = m[19]; F5[2] = m[20]; F5[3] = 0.5 * (m[21] + m[22]);
    double I[4], F[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        I[k] = C[0] * (dF1[k] + (double)F1s[k]) + C[1] * (double)F2[k] + C[2] * (double)F3[k] + C[3] * F4[k] + C[4] * F5[k];
    double rhow = 0.0;
    if (!wall) {
#pragma unroll
        for (int k = 0; k < 4; ++k) F[k] = I[k] / dGf;
    } else {
        // impermeability (Eq. rho_wall) with the time-integrated incident mass flux; reflected part rho_w H_w
        const double* oc = cd.oconst + g.wall * 8;           // [0..3] incident flux of H_ref, [4..7] reflected
        const double Iinc0 = dGf * oc[0] + I[0];
        rhow = -nin * Iinc0 / (dGf * Dw);
#pragma unroll
        for (int k = 0; k < 4; ++k) F[k] = I[k] / dGf + rhow * wc[14 + k] - oc[4 + k];
    }
    double* fo = cd.fflux + (size_t)item * 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) fo[k] = F[k];

    // ---- parameters of the micro flux (delta form, divided by dG_f): for each upwind side the cubic
    // Q = C1' s(c.q)(2 lam |c|^2 - 4) + C2' (u_n P_h(a_side) + u_t P_h(a_t)) + C3' P_h(A) and the linear b-part
    // difference C1' 2 s (c.q) + C2' (u_n a_side,3 + u_t a_t,3)/(2 lam) + C3' A_3/(2 lam)
    T* pp = cd.fpar + ((size_t)n * cd.nf + f) * NP;      // level-major: a tile's faces of one level are rows
    const T C1p = T(C[0] / dGf), C2p = T(C[1] / dGf), C3p = T(C[2] / dGf);
    for (int side = 0; side < 2; ++side) {
        const PolyT<T>& Qs = side == 0 ? QL : QR;
        const PolyT<T>& Rs = side == 0 ? RL : RR;
        PolyT<T> qf, lb;
#pragma unroll
        for (int a = 0; a < 5; ++a)
#pragma unroll
            for (int b = 0; b < 5; ++b) {
                qf.c[a][b] = C1p * shk.c[a][b] + C2p * Qs.c[a][b] + C3p * PhA.c[a][b];
                lb.c[a][b] = C1p * cq2.c[a][b] + C2p * (Rs.c[a][b] - Qs.c[a][b]) + C3p * (PbA.c[a][b] - PhA.c[a][b]);
            }
        T* q = pp + (side == 0 ? F_QL : F_QR);
        q[0] = qf.c[0][0]; q[1] = qf.c[1][0]; q[2] = qf.c[0][1]; q[3] = qf.c[2][0]; q[4] = qf.c[1][1];
        q[5] = qf.c[0][2]; q[6] = qf.c[3][0]; q[7] = qf.c[2][1]; q[8] = qf.c[1][2]; q[9] = qf.c[0][3];
        T* l = pp + (side == 0 ? F_LBL : F_LBR);
        l[0] = lb.c[0][0]; l[1] = lb.c[1][0]; l[2] = lb.c[0][1];
    }
    pp[F_RM1] = T(rr - 1.0);
    pp[F_R] = T(rr);
    pp[F_I2L] = T(i2ld);
    pp[F_DI2L] = T(di2l);
    pp[F_C1] = C1p;
    pp[F_C4] = T(C[3] / dGf);
    pp[F_C5] = T(C[4] / dGf);
    pp[F_NIN] = T(nin);
    if (wall) {
        const double* ws = cd.wall + ((size_t)g.wall * cd.nslot + wsl) * 3;
        const double lamw = cd.lam0 / ws[2];
        const double rw = rhow * lamw / cd.lam0;
        pp[F_WRM1] = T(rw - 1.0);
        pp[F_WR] = T(rw);
        pp[F_WI2L] = T(0.5 / lamw);
        pp[F_WDI2L] = T(0.5 / lamw - 0.5 / cd.lam0);
    } else {
        pp[F_WRM1] = pp[F_WR] = pp[F_WI2L] = pp[F_WDI2L] = T(0);
    }
}

// ------------------------------------------------------------------------------ separable Maxwellian tables

// Tables of expm1(lam0 x^2 - lam (x - U)^2) over the 1-D velocity nodes, so that for a Maxwellian of density
// rho: H - H_ref = H_ref [(r - 1) + r (ex + ey + ex ey)], r = rho lam / lam0.  The cell-level tables of W^k and
// W^{k+1}: a CTA takes 128 cell-levels; each thread first forms the exponent coefficients of one of them in
// FP64 (one thread per cell-level, so the slow FP64 divisions run on every lane), then each warp writes the
// tables of 32 of them with its lanes over the nodes.  (The interface and wall tables are formed in
// k2_face_params.)
constexpr int KT_ITEMS = 128;   // cell-levels per CTA of k_tables (one per thread)

template <typename T>
__global__ void __launch_bounds__(KT_ITEMS) k_tables(Batch<T> B)
{
    const int cs = find_case(B.off, B.ncases, blockIdx.x);
    const CaseDev<T>& cd = B.cases[cs];
    if (!cd.st->active || *(volatile int*)cd.err) return;
    __shared__ T coef[KT_ITEMS][2][5];
    const int nt = cd.nt, nuv = cd.nu + cd.nv, nitems = cd.nc * nt;
    const int first = (blockIdx.x - B.off[cs]) * KT_ITEMS;   // cell-level pairs first.., item = c * nt + n
    const int p = cd.st->parity;
    {
        const int item = first + threadIdx.x;
        if (item < nitems) {
            for (int e = 0; e < 2; ++e) {
                double rho, U, V, lam;
                prim((e == 0 ? cd.W[p] : cd.W[p ^ 1]) + ((size_t)(item % nt) * cd.nc + item / nt) * 4, rho, U, V, lam);
                T* q = coef[threadIdx.x][e];
                q[0] = T(cd.lam0 - lam);
                q[1] = T(2.0 * lam * U);
                q[2] = T(lam * U * U);
                q[3] = T(2.0 * lam * V);
                q[4] = T(lam * V * V);
            }
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = 0; r < 32; ++r) {
        const int li = warp * 32 + r, item = first + li;
        if (item >= nitems) break;
        for (int e = 0; e < 2; ++e) {
            const T* c = coef[li][e];
            T* dst = cd.ctab + ((size_t)item * 2 + e) * nuv;
            for (int k = lane; k < cd.nu; k += 32) {
                const T x = cd.tu1[k];
                dst[k] = t_expm1<T>(c[0] * x * x + c[1] * x - c[2]);
            }
            for (int k = lane; k < cd.nv; k += 32) {
                const T y = cd.tv1[k];
                dst[cd.nu + k] = t_expm1<T>(c[0] * y * y + c[3] * y - c[4]);
            }
        }
    }
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
    cd.dG[c] = cd.dt_fixed > 0.0 ? cd.dt_fixed : local_step(cd, cd.W[cd.st->parity], c, c % cd.nx, c / cd.nx);
}

// ------------------------------------------------------------------------------ K3 macro update

// A = diag(D) + dG omega E (D = 1 when null), E of Eq. D_explicit from the paired offsets e_d:
// E_{n, n-d} = e_d, E_{n, n+d} = -e_d (levels cyclic)
template <typename T>
__device__ void spectral_matrix(const CaseDev<T>& cd, double dG, const double* D, double (&A)[MAXNT][MAXNT])
{
    const int nt = cd.nt;
    for (int n = 0; n < nt; ++n)
        for (int m = 0; m < nt; ++m) A[n][m] = n == m ? (D ? D[n] : 1.0) : 0.0;
    for (int n = 0; n < nt; ++n)
        for (int d = 1; d <= cd.nh; ++d) {
            int nm = n - d; if (nm < 0) nm += nt;
            int np = n + d; if (np >= nt) np -= nt;
            A[n][nm] += dG * cd.omega * cd.e[d];
            A[n][np] -= dG * cd.omega * cd.e[d];
        }
}

// Solve A X = R in place for the columns of R (R becomes X), A destroyed: Gaussian elimination with partial
// pivoting over the levels
template <int NR>
__device__ void solve_levels(int nt, double (&A)[MAXNT][MAXNT], double (&R)[MAXNT][NR])
{
    for (int k = 0; k < nt; ++k) {
        int piv = k;
        for (int i = k + 1; i < nt; ++i)
            if (fabs(A[i][k]) > fabs(A[piv][k])) piv = i;
        if (piv != k) {
            for (int j = 0; j < nt; ++j) { const double t = A[k][j]; A[k][j] = A[piv][j]; A[piv][j] = t; }
            for (int j = 0; j < NR; ++j) { const double t = R[k][j]; R[k][j] = R[piv][j]; R[piv][j] = t; }
        }
        for (int i = k + 1; i < nt; ++i) {
            const double f = A[i][k] / A[k][k];
            for (int j = k; j < nt; ++j) A[i][j] -= f * A[k][j];
            for (int j = 0; j < NR; ++j) R[i][j] -= f * R[k][j];
        }
    }
    for (int k = nt - 1; k >= 0; --k)
        for (int j = 0; j < NR; ++j) {
            double s = R[k][j];
            for (int m = k + 1; m < nt; ++m) s -= A[k][m] * R[m][j];
            R[k][j] = s / A[k][k];
        }
}

template <typename T>
__global__ void __launch_bounds__(K3_THREADS) k3_macro(Batch<T> B)
{
    int cs = find_case(B.off, B.ncases, blockIdx.x);
    const CaseDev<T>& cd = B.cases[cs];
    if (!cd.st->active || *(volatile int*)cd.err) return;
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
        const bool implicit = cd.spectral_implicit != 0;
        double Wi[MAXNT][4];
        if (implicit) {
            // spectral source at the new iterate: (I + dG omega E) W^{k+1} = W^k - dG div F for every variable
            double A[MAXNT][MAXNT];
            spectral_matrix(cd, dG, nullptr, A);
            for (int n = 0; n < nt; ++n) {
                const double* FL = cd.fflux + ((size_t)fL * nt + n) * 4;
                const double* FR = cd.fflux + ((size_t)fR * nt + n) * 4;
                const double* FB = cd.fflux + ((size_t)fB * nt + n) * 4;
                const double* FT = cd.fflux + ((size_t)fT * nt + n) * 4;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    Wi[n][k] = Wc[n][k] - dG * (dy * (FR[k] - FL[k]) + dx * (FT[k] - FB[k])) / area;
            }
            solve_levels(nt, A, Wi);
        }
        double Dn[MAXNT];
        for (int n = 0; n < nt; ++n) {
            const double* FL = cd.fflux + ((size_t)fL * nt + n) * 4;
            const double* FR = cd.fflux + ((size_t)fR * nt + n) * 4;
            const double* FB = cd.fflux + ((size_t)fB * nt + n) * 4;
            const double* FT = cd.fflux + ((size_t)fT * nt + n) * 4;
            double wn[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (implicit) {
                    wn[k] = Wi[n][k];
                } else {
                    double div = (dy * (FR[k] - FL[k]) + dx * (FT[k] - FB[k])) / area;
                    double ew = 0.0;
                    for (int d = 1; d <= cd.nh; ++d) {
                        int nm = n - d; if (nm < 0) nm += nt;
                        int np = n + d; if (np >= nt) np -= nt;
                        ew += cd.e[d] * (Wc[nm][k] - Wc[np][k]);
                    }
                    wn[k] = Wc[n][k] - dG * (div + cd.omega * ew);
                }
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
            T* cp = cd.cpar + ((size_t)n * cd.nc + c) * NCP;
            eq_cell(r0, U0, V0, l0, cd.lam0, cd.pr, qx, qy, cp + C_EQ0);
            eq_cell(r1, U1, V1, l1, cd.lam0, cd.pr, qx, qy, cp + C_EQ1);
            // explicit: the update of Eq. fv_h divided by D; implicit: its right-hand side, which the micro
            // update then multiplies by minv across levels
            const double D = 1.0 + 0.5 * dG / t1;
            Dn[n] = D;
            const double s_ = implicit ? 1.0 : D;
            // kself, -kE, kp1, kp0, -kdx, -kdy, each stored twice (broadcast pairs for the (h, b) update)
            const double kk[6] = {(1.0 - 0.5 * dG / t0) / s_, implicit ? 0.0 : -dG * cd.omega / D,
                                  0.5 * dG / (t1 * s_), 0.5 * dG / (t0 * s_), -dG / (dx * s_), -dG / (dy * s_)};
#pragma unroll
            for (int q = 0; q < 6; ++q) cp[C_K + 2 * q] = cp[C_K + 2 * q + 1] = T(kk[q]);
        }
        if (implicit) {
            // inverse of diag(D_n) + dG omega E for the micro update of this cell (every velocity)
            double A[MAXNT][MAXNT], X[MAXNT][MAXNT];
            spectral_matrix(cd, dG, Dn, A);
            for (int n = 0; n < nt; ++n)
                for (int m = 0; m < nt; ++m) X[n][m] = n == m ? 1.0 : 0.0;
            solve_levels(nt, A, X);
            T* mo = cd.minv + (size_t)c * nt * nt;
            for (int n = 0; n < nt; ++n)
                for (int m = 0; m < nt; ++m) mo[n * nt + m] = T(X[n][m]);
        }
        cd.dG[c] = cd.dt_fixed > 0.0 ? cd.dt_fixed : local_step(cd, Wn, c, i, j);
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

// ------------------------------------------------------------------------------ K5 residual / status

template <typename T>
__global__ void k5_finish(const CaseDev<T>* cases, int ncases, const int* k3off)
{
    int cs = blockIdx.x;
    if (cs >= ncases) return;
    const CaseDev<T>& cd = cases[cs];
    CaseStatus* st = cd.st;
    if (!st->active || *(volatile int*)cd.err) return;   // a failed wait leaves the iteration unfinished
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

// sign class in which a node is stored first (classes in order 0..3: u > 0 first, then v > 0 first)
template <typename T>
__device__ __forceinline__ int first_class(const CaseDev<T>& cd, int can)
{
    const double u = cd.u1[can % cd.nu], v = cd.v1[can / cd.nu];
    return (u < 0 ? 1 : 0) | (v < 0 ? 2 : 0);
}

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
    const int can = cd.vcan[a];
    if (can >= 0) {
        double href = (cd.lam0 / M_PI) * exp(-cd.lam0 * (cd.vu[a] * cd.vu[a] + cd.vv[a] * cd.vv[a]));
        double rv = which == 0 ? href : href * 0.5 / cd.lam0;
        val = stage[(size_t)c * cd.nvel + can] - rv;
    }
    T* dst = reinterpret_cast<T*>(cd.f[cd.st->parity]);
    dst[2 * sidx(cd.nc, cd.nt, vb, c, n, lane) + which] = T(val);
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
    const int can = cd.vcan[a];
    // a node stored in several sign classes holds the same value in each; the first copy is read
    if (can < 0 || cd.vcls[vb] != first_class(cd, can)) return;
    double href = (cd.lam0 / M_PI) * exp(-cd.lam0 * (cd.vu[a] * cd.vu[a] + cd.vv[a] * cd.vv[a]));
    double rv = which == 0 ? href : href * 0.5 / cd.lam0;
    const T* src = reinterpret_cast<const T*>(cd.f[cd.st->parity]);
    stage[(size_t)c * cd.nvel + can] = (double)src[2 * sidx(cd.nc, cd.nt, vb, c, n, lane) + which] + rv;
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
    if (cd.vcan[a] >= 0) {
        double uu = cd.vu[a], vv = cd.vv[a];
        double lam = cd.lam0 / Tt;
        double H = rho * (lam / M_PI) * exp(-lam * ((uu - U) * (uu - U) + (vv - V) * (vv - V)));
        double href = (cd.lam0 / M_PI) * exp(-cd.lam0 * (uu * uu + vv * vv));
        dhv = H - href;
        dbv = H * 0.5 / lam - href * 0.5 / cd.lam0;
    }
    cd.f[p][sidx(cd.nc, cd.nt, vb, c, n, lane)] = pk(T(dhv), T(dbv));
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
        const P2<T> fv = cd.f[p][sidx(cd.nc, cd.nt, vb, c, n, lane)];
        double wd = w * (double)fv.x, we = w * (double)fv.y;
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
