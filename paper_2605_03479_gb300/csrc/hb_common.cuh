// Shared device definitions of the GB300 HB-UGKS path.
//
// State layout (per case), velocity-blocked "delta form":
//   dh[vb][cell][level][32]   dh = h - H_ref  (T = double or float),  same for db = b - B_ref
// with vb the block of 32 consecutive discrete velocities (one warp lane per velocity), cell = j*nx + i and
// H_ref = (lam0/pi) exp(-lam0 |u|^2), B_ref = H_ref / (2 lam0), the reduced Maxwellian at rest at T0
// (lam0 = 1).  Every update is applied to the deviations, which is algebraically identical to the update of
// h itself: E annihilates level-constant vectors, the reference parts of the collision terms cancel, and the
// reference part of every interface flux is u_n H_ref (C1 + C4 = dG_f), which cancels in each cell's flux
// balance because the signed face lengths of a rectangle sum to zero.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hb {

constexpr int VB = 32;        // velocities per block (= warp width)
constexpr int MAXNT = 15;     // N_H <= 7
constexpr int NM = 23;        // face moments per (face, level)
constexpr int NCM = 13;       // cell moments per (cell, level)
constexpr int NP = 48;        // face parameters per (face, level)
constexpr int NCP = 32;       // cell parameters per (cell, level)
constexpr int RING = 4096;    // residual history slots per case
constexpr int K3_THREADS = 128;

// face parameter slots
enum FP {
    F_R = 0, F_RM1, F_DL, F_TLU, F_TLV, F_LU2, F_I2L, F_DI2L, F_U, F_V, F_TL, F_SQX, F_SQY,
    F_AL = 13, F_AR = 17, F_AT = 21, F_A = 25, F_C = 29,
    F_WR = 34, F_WRM1, F_WDL, F_WTLU, F_WTLV, F_WLU2, F_WI2L, F_WDI2L, F_NIN
};
// cell parameter slots: equilibrium of W^k at 0..12, of W^{k+1} at 13..25, update coefficients 26..31
enum CP { C_EQ0 = 0, C_EQ1 = 13, C_KSELF = 26, C_KE, C_KP1, C_KP0, C_KDX, C_KDY };
// equilibrium sub-slots (same order as the first 13 face slots)
enum EQ { E_R = 0, E_RM1, E_DL, E_TLU, E_TLV, E_LU2, E_I2L, E_DI2L, E_U, E_V, E_TL, E_SQX, E_SQY };

struct CaseStatus {
    int active;          // iterating in the current call
    int user_active;     // allowed to iterate at all
    int parity;          // which of the two state buffers is current
    int diverged;
    long long iters;     // iterations since the state was set
    long long iters_call;
    double last[4];      // last residual
};

template <typename T>
struct CaseDev {
    int nx, ny, nu, nv, nvel, nvb, nt, nh, nfx, nf, nc;
    int face_step;
    double omega, mu0, w_vss, pr, cfl, gam, umax, vmax, lam0;
    double e[8];                       // e_d = (-1)^d / (2 sin(pi d / N_T)), d = 1..N_H
    const double* wall;                // [4][nt][3]  U_w, V_w, T_w per level
    const double *xn, *yn, *xc, *yc, *hx, *hy, *rdx, *rdy;   // rdx[i] = 1/(xc[i+1]-xc[i])
    const double *vu, *vv, *vw;        // per padded velocity
    const T *tu, *tv, *tw, *thref;     // per padded velocity
    const double *u1, *wu1, *v1, *wv1; // 1-D grids
    const double* refmom;              // [5][13]: full, u>0, u<0, v>0, v<0 moments of (H_ref, B_ref)
    T* dh[2];
    T* db[2];
    double* W[2];
    double* dG;
    double* fmom;                      // [nf][nt][NM]
    double* cmom;                      // [nc][nt][NCM]
    T* fpar;                           // [nf][nt][NP]
    double* fflux;                     // [nf][nt][4]
    T* cpar;                           // [nc][nt][NCP]
    double* rpart;                     // [k3 blocks][4]
    double* rhist;                     // [RING][4]
    double* stage;                     // conversion staging (>= nc * nvel_pad doubles)
    CaseStatus* st;
    const double* tol;                 // shared residual target of the handle
};

// --------------------------------------------------------------------------------- small helpers

__device__ __forceinline__ int find_case(const int* off, int ncases, int blk)
{
    int lo = 0, hi = ncases - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= blk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ size_t sidx(int nc, int nt, int vb, int c, int n, int lane)
{
    return ((((size_t)vb * nc + c) * nt + n) << 5) + lane;
}

template <typename T> __device__ __forceinline__ T t_expm1(T x);
template <> __device__ __forceinline__ double t_expm1<double>(double x) { return expm1(x); }
template <> __device__ __forceinline__ float t_expm1<float>(float x) { return expm1f(x); }

// primitive variables from W = (rho, rho U, rho V, rho E) with D + K = 3
__device__ __forceinline__ void prim(const double* W, double& rho, double& U, double& V, double& lam)
{
    rho = W[0];
    U = W[1] / rho;
    V = W[2] / rho;
    lam = 0.75 * rho / (W[3] - 0.5 * rho * (U * U + V * V));
}

// tau = mu/p, mu = mu0 (T/T0)^w, T/T0 = lam0/lam, p = rho/(2 lam)
__device__ __forceinline__ double relax_time(double mu0, double w, double lam0, double rho, double lam)
{
    return mu0 * pow(lam0 / lam, w) * 2.0 * lam / rho;
}

// Coefficients of Eq. C_coeffs: Taylor series in x = dG/tau below x = 1 (the printed forms cancel there),
// printed forms with 1 - e^-x = -expm1(-x) above.
__device__ __noinline__ void ugks_coeffs(double dG, double tau, double C[5])
{
    double x = dG / tau;
    if (x < 1.0) {
        // terms t_j = x^j / j!, summed from the highest order down
        double t[27];
        t[0] = 1.0;
#pragma unroll
        for (int j = 1; j <= 26; ++j) t[j] = t[j - 1] * x * (1.0 / j);
        double s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0, s5 = 0.0;
#pragma unroll
        for (int j = 26; j >= 1; --j) {
            double sg = (j & 1) ? 1.0 : -1.0;
            s4 += sg * t[j];
            if (j >= 2) s1 -= sg * t[j];
            if (j >= 3) { s2 += sg * (2.0 - j) * t[j]; s3 += sg * t[j]; }
            s5 += sg * (j - 1.0) * t[j];
        }
        C[0] = tau * s1;
        C[1] = tau * tau * s2;
        C[2] = tau * tau * s3;
        C[3] = tau * s4;
        C[4] = tau * tau * s5;
    } else {
        double phi = -expm1(-x), ex = exp(-x);
        C[0] = dG - tau * phi;
        C[1] = 2.0 * tau * tau * phi - tau * dG - tau * dG * ex;
        C[2] = 0.5 * dG * dG - tau * dG + tau * tau * phi;
        C[3] = tau * phi;
        C[4] = tau * dG * ex - tau * tau * phi;
    }
}

// Coefficients a of (a.psi) g whose moments per unit density are w (continuous Maxwellian, K = 1).
__device__ __forceinline__ void micro_slope(const double w[4], double U, double V, double lam, double a[4])
{
    double R2 = w[1] - U * w[0];
    double R3 = w[2] - V * w[0];
    double e = U * U + V * V + 1.5 / lam;
    double R4 = 2.0 * w[3] - e * w[0];
    a[3] = (4.0 / 3.0) * lam * lam * (R4 - 2.0 * U * R2 - 2.0 * V * R3);
    a[2] = 2.0 * lam * R3 - V * a[3];
    a[1] = 2.0 * lam * R2 - U * a[3];
    a[0] = w[0] - U * a[1] - V * a[2] - 0.5 * a[3] * e;
}

// Parameters of the delta-form equilibrium for the Maxwellian (rho, U, V, lam) with Shakhov heat flux q:
// H - H_ref = H_ref [ r e^D - 1 ], D = (lam0 - lam)|u|^2 + 2 lam (uU + vV) - lam |U|^2, r = rho lam / lam0.
__device__ inline void eq_params(double rho, double U, double V, double lam, double lam0, double pr,
                                 double qx, double qy, double* o)
{
    double r = rho * lam / lam0;
    o[E_R] = r;
    o[E_RM1] = r - 1.0;
    o[E_DL] = lam0 - lam;
    o[E_TLU] = 2.0 * lam * U;
    o[E_TLV] = 2.0 * lam * V;
    o[E_LU2] = lam * (U * U + V * V);
    o[E_I2L] = 0.5 / lam;
    o[E_DI2L] = 0.5 / lam - 0.5 / lam0;
    o[E_U] = U;
    o[E_V] = V;
    o[E_TL] = 2.0 * lam;
    // Shakhov (Eq. shakhov reduced over xi): H+ = s (c.q)(2 lam |c|^2 - 4) H, s = (1 - Pr) 4 lam^2 / (5 rho)
    double s = (1.0 - pr) * 4.0 * lam * lam / (5.0 * rho);
    o[E_SQX] = s * qx;
    o[E_SQY] = s * qy;
}

// delta-form reduced equilibrium at one velocity: returns dH = H - H_ref, dB = B - B_ref and the Shakhov
// corrections Hp, Bp, plus H itself (needed by the slope terms of the interface flux).
template <typename T>
__device__ __forceinline__ void eq_eval(const T* p, T u, T v, T u2, T href, T& H, T& dH, T& dB, T& Hp, T& Bp)
{
    T D = p[E_DL] * u2 + p[E_TLU] * u + p[E_TLV] * v - p[E_LU2];
    T em1 = t_expm1<T>(D);
    dH = href * (p[E_RM1] + p[E_R] * em1);
    H = href + dH;
    dB = dH * p[E_I2L] + href * p[E_DI2L];
    T cx = u - p[E_U], cy = v - p[E_V];
    T c2 = cx * cx + cy * cy;
    T cq = p[E_SQX] * cx + p[E_SQY] * cy;
    Hp = cq * (p[E_TL] * c2 - T(4)) * H;
    Bp = cq * (p[E_TL] * c2 - T(2)) * (H * p[E_I2L]);
}

// ----------------------------------------------------------------------- analytic velocity sums
// Discrete sums of polynomial x Maxwellian over the tensor velocity grid factor into 1-D sums
//   X[p] = sum_i wu_i u_i^p exp(-lam (u_i - U)^2)  (restricted to u_i > 0, u_i < 0 or all),
//   Y[q] likewise in v,  so  sum_a w_a u^p v^q rho (lam/pi) e^{-lam |u - U|^2} = rho lam/pi X[p] Y[q].

struct Sums1D {
    double s[4][9];   // [0] all, [1] positive nodes, [2] negative nodes, [3] zero nodes; powers 0..8
};

__device__ __noinline__ void sums1d(const double* x, const double* w, int n, double lam, double U, Sums1D& S)
{
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int p = 0; p < 9; ++p) S.s[r][p] = 0.0;
    for (int k = 0; k < n; ++k) {
        double xv = x[k], d = xv - U;
        double g = w[k] * exp(-lam * d * d);
        int r = xv > 0.0 ? 1 : (xv < 0.0 ? 2 : 3);
        double pw = g;
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            S.s[r][p] += pw;
            pw *= xv;
        }
    }
#pragma unroll
    for (int p = 0; p < 9; ++p) S.s[0][p] = S.s[1][p] + S.s[2][p] + S.s[3][p];
}

// polynomial in (u, v) of total degree <= 4
struct Poly {
    double c[5][5];
    __device__ void zero()
    {
#pragma unroll
        for (int p = 0; p < 5; ++p)
#pragma unroll
            for (int q = 0; q < 5; ++q) c[p][q] = 0.0;
    }
};

__device__ __noinline__ void poly_mul(const Poly& A, const Poly& B, Poly& C)
{
    C.zero();
#pragma unroll
    for (int p = 0; p < 5; ++p)
#pragma unroll
        for (int q = 0; q < 5 - p; ++q) {
            double a = A.c[p][q];
            if (a == 0.0) continue;
#pragma unroll
            for (int r = 0; r < 5 - p; ++r)
#pragma unroll
                for (int s = 0; s < 5 - p - q - r; ++s)
                    if (s >= 0) C.c[p + r][q + s] += a * B.c[r][s];
        }
}

// P_h(a) = a0 + a1 u + a2 v + a3/2 (u^2 + v^2 + 1/(2 lam)),  P_b(a) = P_h(a) + a3/(2 lam)
__device__ inline void poly_P(const double* a, double i2l, bool for_b, Poly& P)
{
    P.zero();
    P.c[0][0] = a[0] + 0.5 * a[3] * i2l + (for_b ? a[3] * i2l : 0.0);
    P.c[1][0] = a[1];
    P.c[0][1] = a[2];
    P.c[2][0] = 0.5 * a[3];
    P.c[0][2] = 0.5 * a[3];
}

// moments sum w psi [Q H ; R B] over the grid part selected by (rx, ry), H = pref e^{..}, B = H i2l:
//   (sum Q H, sum u Q H, sum v Q H, 1/2 sum (|u|^2 Q H + R B))
__device__ __noinline__ void mom4(const Poly& Q, const Poly& R, const Sums1D& X, int rx, const Sums1D& Y, int ry,
                            double pref, double i2l, double out[4])
{
    double o0 = 0, o1 = 0, o2 = 0, o3 = 0, ob = 0;
#pragma unroll
    for (int p = 0; p < 5; ++p)
#pragma unroll
        for (int q = 0; q < 5 - p; ++q) {
            double a = Q.c[p][q], r = R.c[p][q];
            if (a != 0.0) {
                o0 += a * X.s[rx][p] * Y.s[ry][q];
                o1 += a * X.s[rx][p + 1] * Y.s[ry][q];
                o2 += a * X.s[rx][p] * Y.s[ry][q + 1];
                o3 += a * (X.s[rx][p + 2] * Y.s[ry][q] + X.s[rx][p] * Y.s[ry][q + 2]);
            }
            if (r != 0.0) ob += r * X.s[rx][p] * Y.s[ry][q];
        }
    out[0] = pref * o0;
    out[1] = pref * o1;
    out[2] = pref * o2;
    out[3] = 0.5 * pref * (o3 + i2l * ob);
}

}  // namespace hb
