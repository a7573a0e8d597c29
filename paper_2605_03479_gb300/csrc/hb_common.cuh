// Shared device definitions of the GB300 HB-UGKS path.
//
// State layout (per case), velocity-blocked "delta form":
//   f[vb][level][cell][32] = (h - H_ref, b - B_ref)   pairs of T = double or float, h and b side by side
// with vb the block of 32 consecutive discrete velocities (one warp lane per velocity), cell = j*nx + i and
// H_ref = (lam0/pi) exp(-lam0 |u|^2), B_ref = H_ref / (2 lam0), the reduced Maxwellian at rest at T0
// (lam0 = 1).  Every update is applied to the deviations, which is algebraically identical to the update of
// h itself: E annihilates level-constant vectors, the reference parts of the collision terms cancel, and the
// reference part of every interface flux is u_n H_ref (C1 + C4 = dG_f), which cancels in each cell's flux
// balance because the signed face lengths of a rectangle sum to zero.
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace hb {

constexpr int VB = 32;        // velocities per block (= warp width)
constexpr int MAXNT = 15;     // N_H <= 7
constexpr int NM = 23;        // face moments per (face, level)
constexpr int NCM = 13;       // cell moments per (cell, level)
constexpr int NP = 44;        // face parameters per (face, level), 16-byte aligned blocks
constexpr int NCP = 36;       // cell parameters per (cell, level)
constexpr int RING = 4096;    // residual history slots per case
constexpr int K3_THREADS = 128;
constexpr int WCN = 18;       // per wall and level: Aw[13] (reflected-half raw moments, unit density), Dw, Gw[4]

// ------------------------------------------------------------------ (h, b) pairs and packed arithmetic
// The reduced distributions h and b of one velocity go through the same transport, reconstruction, spectral and
// update arithmetic, so they are stored and processed as a pair.  For float a pair is one 64-bit register pair
// and every operation below is a single packed FP32x2 instruction of sm_100+ (both halves rounded as the
// scalar instruction would); for double they are two scalar operations.
template <typename T> struct PairOf;
template <> struct PairOf<float> { using type = float2; };
template <> struct PairOf<double> { using type = double2; };
template <typename T> using P2 = typename PairOf<T>::type;

__device__ __forceinline__ float2 pk(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double2 pk(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float2 bc(float x) { return make_float2(x, x); }
__device__ __forceinline__ double2 bc(double x) { return make_double2(x, x); }

__device__ __forceinline__ uint64_t f2u(float2 a) { return *reinterpret_cast<uint64_t*>(&a); }
__device__ __forceinline__ float2 u2f(uint64_t a) { return *reinterpret_cast<float2*>(&a); }

// a * b + c
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 psub(float2 a, float2 b)
{
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(d);
}
__device__ __forceinline__ double2 psub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// Face parameter slots of the micro flux (delta form).  For an interface velocity u = (u, v) with normal
// component u_n, the Maxwellian part of the time-integrated flux divided by dG_f is
//   h: C1' dH + H Q(u, v),   b: C1' dB + B (Q(u, v) + l0 + l1 u + l2 v)
// where dH = H - H_ref = H_ref [(r - 1) + r (ex + ey + ex ey)] with the separable factors ex(u), ey(v) of the
// face table, Q is the bivariate cubic C1' s (c.q)(2 lam |c|^2 - 4) + C2' (u_n P(a_n) + u_t P(a_t)) + C3' P(A)
// (a_n = a^L for u_n > 0, a^R for u_n < 0) and the linear term is the b-part difference.
// Cubic monomial order: 1, u, v, u^2, uv, v^2, u^3, u^2 v, u v^2, v^3.  Blocks start on multiples of 4.
enum FP {
    F_QL = 0, F_QR = 12, F_LBL = 24, F_LBR = 28, F_RM1 = 32, F_R = 33, F_I2L = 34, F_DI2L = 35,
    F_C1 = 36, F_C4 = 37, F_C5 = 38, F_NIN = 39, F_WRM1 = 40, F_WR = 41, F_WI2L = 42, F_WDI2L = 43
};
// Cell parameter slots: equilibrium of W^k at 0..11, of W^{k+1} at 12..23, each: r - 1, r, 1/(2 lam),
// 1/(2 lam) - 1/(2 lam0), then the Shakhov factor s (c.q)(2 lam |c|^2 - 4) = L(u, v) Q(u, v) as
// L = a0 + a1 u + a2 v (slots 4..6; 7 unused) and Q = b0 + b1 u + b2 v + b3 (u^2 + v^2) (slots 8..11): the reduced
// corrections are H+ = L Q H and B+ = (L Q + 2 L) B.  From 24 on, the update coefficients of Eq. fv_h as
// broadcast pairs (each value twice): kself, -kE, kp1, kp0, -kdx, -kdy.
enum CP { C_EQ0 = 0, C_EQ1 = 12, C_K = 24 };
enum EQ { E_RM1 = 0, E_R, E_I2L, E_DI2L, E_L = 4, E_Q = 8 };

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
    using value_type = T;
    int nx, ny, nu, nv, nvel, nvb, nt, nh, nfx, nf, nc;
    int face_step;
    double omega, mu0, w_vss, pr, cfl, gam, umax, vmax, lam0;
    double e[8];                       // e_d = (-1)^d / (2 sin(pi d / N_T)), d = 1..N_H
    T et[8];                           // the same in the storage precision
    int spectral_implicit;             // spectral source at the new pseudo-time iterate
    T* minv;                           // [nc][nt][nt] inverse of diag(1 + dG/(2 tau_n^{k+1})) + dG omega E (implicit)
    int nslot;                         // wall-state slots: nt, or time steps per period (time-domain mode)
    double dt_fixed;                   // > 0: time-domain mode, one global physical step for every cell and face
    const double* wall;                // [4][nslot][3]  U_w, V_w, T_w per level (per step in time-domain mode)
    const double *xn, *yn, *xc, *yc, *hx, *hy, *rdx, *rdy;   // rdx[i] = 1/(xc[i+1]-xc[i])
    const double *vu, *vv, *vw;        // per padded velocity
    const T *tu, *tv, *tw, *thref;     // per padded velocity
    const T *twu, *twv;                // per padded velocity: the factors w_u, w_v of its weight (0 for padding)
    const double *u1, *wu1, *v1, *wv1; // 1-D grids
    const T *tu1, *tv1;                // 1-D nodes in the storage precision
    const double* refmom;              // [5][13]: full, u>0, u<0, v>0, v<0 moments of (H_ref, B_ref)
    const T *wxr, *wyr;                // [9][nu], [9][nv]: w x^p exp(-lam0 x^2) per 1-D node
    const double *xr0, *yr0;           // [4][9]: sums of the above over all / positive / negative / zero nodes
    const T *xr0t, *yr0t;              // the same in the storage precision
    const double* wconst;              // [4][nslot][WCN] reflected-half constants of each wall Maxwellian
    const double* oconst;              // [4][8]: incident and reflected flux moments of (H_ref, B_ref) per wall
    P2<T>* f[2];                       // the two state buffers (current: st->parity)
    double* W[2];
    double* dG;
    double* hmom;                      // [nc][nt][4][NM] half-face sums of the reconstruction per sign class
    double* cmom;                      // [nc][nt][NCM]
    T* fpar;                           // [nt][nf][NP]
    T* ftab;                           // [nf][nt][nu + nv]   expm1 factors of the interface Maxwellian
    T* wtab;                           // [4][nslot][nu + nv]  expm1 factors of each wall's Maxwellian
    T* ctab;                           // [nc][nt][2][nu + nv] expm1 factors of the cell equilibria (W^k, W^{k+1})
    const int* viu;                    // per stored velocity: u index (0 for padding)
    const int* viv;                    // per stored velocity: v index
    const int* vcan;                   // per stored velocity: canonical index jv * nu + iu, -1 for padding
    const int* vcls;                   // per velocity block: sign class (bit 0: u < 0, bit 1: v < 0)
    int cls_end[4];                    // one past the last block of sign classes 0..c (classes are consecutive)
    int shakhov;                       // Pr != 1
    double* fflux;                     // [nf][nt][4]
    T* cpar;                           // [nt][nc][NCP]
    double* rpart;                     // [k3 blocks][4]
    double* rhist;                     // [RING][4]
    double* stage;                     // conversion staging (>= nc * nvel_pad doubles)
    CaseStatus* st;
    const double* tol;                 // shared residual target of the handle
    int* err;                          // device error word of the handle (1: a bounded wait expired); every
                                       // kernel of the iteration returns at once while it is set
    const int* expire;                 // test hook of the handle: nonzero makes the micro update report its
                                       // first completed wait as expired (no copy in flight is abandoned)
};

template <typename T>
struct Batch {
    const CaseDev<T>* cases;
    int ncases;
    const int* off;   // block offsets per case for this kernel, ncases + 1 entries
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

// wall-state slot of level n in the current iteration: the level itself, or in time-domain mode the step
// within the forcing period
template <typename T>
__device__ __forceinline__ int wall_slot(const CaseDev<T>& cd, int n)
{
    return cd.dt_fixed > 0.0 ? (int)(cd.st->iters % cd.nslot) : n;
}

__device__ __forceinline__ size_t sidx(int nc, int nt, int vb, int c, int n, int lane)
{
    return ((((size_t)vb * nt + n) * nc + c) << 5) + lane;
}

// ---------------------------------------------------------------- bulk copies (TMA) with an mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// arrive on the barrier and add `bytes` to the transaction count its current phase waits for
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// plain arrival (no transaction bytes)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16) completing on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// the same with the destination given as a shared-memory address
__device__ __forceinline__ void bulk_g2s_at(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// nanoseconds of the GPU's global timer
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// A bulk copy lands in microseconds; a wait that lasts this long has failed.
constexpr uint64_t WAIT_LIMIT_NS = 500000000ull;

// Wait for phase `phase` of `bar`, bounded by elapsed time.  On expiry record the failure in *err (and in the
// CTA's abort flag, if given) and return false.  A wait also gives up, without recording anything, once another
// warp of the CTA has set the abort flag, so that one failed wait stops the whole CTA within one limit.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, int* err, volatile int* abort = nullptr)
{
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(bar, phase)) return true;
        if ((it & 31) == 0) {
            if (abort && *abort) return false;
            if (global_ns() - t0 > WAIT_LIMIT_NS) {
                atomicExch(err, 1);
                if (abort) *abort = 1;
                return false;
            }
        }
    }
}

// After a failed wait: bounded wait for a batch of bulk copies that was issued and not yet seen complete, so
// that no copy is still writing into the CTA's shared memory when it exits.  If that wait runs out too (the
// copies themselves failed), the CTA exits regardless; the handle's error word is already set.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t phase)
{
    const uint64_t t0 = global_ns();
    for (unsigned it = 0;; ++it) {
        if (mbar_try_wait(bar, phase)) return;
        if ((it & 31) == 31 && global_ns() - t0 > WAIT_LIMIT_NS) return;
    }
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
// printed forms with 1 - e^-x = -expm1(-x) above.  Evaluated in the precision P of their use.
template <typename P>
__device__ __noinline__ void ugks_coeffs(P dG, P tau, P C[5])
{
    P x = dG / tau;
    if (x < P(1)) {
        P t[27];
        t[0] = P(1);
#pragma unroll
        for (int j = 1; j <= 26; ++j) t[j] = t[j - 1] * x * (P(1) / P(j));
        P s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0;
#pragma unroll
        for (int j = 26; j >= 1; --j) {
            P sg = (j & 1) ? P(1) : P(-1);
            s4 += sg * t[j];
            if (j >= 2) s1 -= sg * t[j];
            if (j >= 3) { s2 += sg * P(2 - j) * t[j]; s3 += sg * t[j]; }
            s5 += sg * P(j - 1) * t[j];
        }
        C[0] = tau * s1;
        C[1] = tau * tau * s2;
        C[2] = tau * tau * s3;
        C[3] = tau * s4;
        C[4] = tau * tau * s5;
    } else {
        P phi = -t_expm1<P>(-x), ex = P(1) + t_expm1<P>(-x);
        C[0] = dG - tau * phi;
        C[1] = P(2) * tau * tau * phi - tau * dG - tau * dG * ex;
        C[2] = P(0.5) * dG * dG - tau * dG + tau * tau * phi;
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

// Shakhov factor s (c.q)(2 lam |c|^2 - 4), s = (1 - Pr) 4 lam^2 / (5 rho), c = u - U, as a cubic in (u, v)
// (monomials 1, u, v, u^2, uv, v^2, u^3, u^2 v, u v^2, v^3), followed by the linear form 2 s (c.q) (1, u, v):
// the reduced corrections are H+ = cubic * H and B+ = (cubic + linear) * B (Eq. shakhov integrated over xi).
__device__ inline void shakhov_poly(double s, double qx, double qy, double U, double V, double lam, double* o)
{
    const double a0 = -s * (qx * U + qy * V), a1 = s * qx, a2 = s * qy;      // s (c.q) = a0 + a1 u + a2 v
    const double b3 = 2.0 * lam, b1 = -4.0 * lam * U, b2 = -4.0 * lam * V;
    const double b0 = 2.0 * lam * (U * U + V * V) - 4.0;                       // 2 lam |c|^2 - 4
    o[0] = a0 * b0;
    o[1] = a0 * b1 + a1 * b0;
    o[2] = a0 * b2 + a2 * b0;
    o[3] = a0 * b3 + a1 * b1;
    o[4] = a1 * b2 + a2 * b1;
    o[5] = a0 * b3 + a2 * b2;
    o[6] = a1 * b3;
    o[7] = a2 * b3;
    o[8] = a1 * b3;
    o[9] = a2 * b3;
    o[10] = 2.0 * a0;
    o[11] = 2.0 * a1;
    o[12] = 2.0 * a2;
}

// Cell equilibrium parameters (slots E_*) of the Maxwellian (rho, U, V, lam) with heat flux q: the Shakhov
// factor s (c.q)(2 lam |c|^2 - 4), s = (1 - Pr) 4 lam^2 / (5 rho), c = u - U, kept as its linear factor
// L = s (c.q) and quadratic factor 2 lam |c|^2 - 4 (Eq. shakhov integrated over xi)
template <typename T>
__device__ inline void eq_cell(double rho, double U, double V, double lam, double lam0, double pr, double qx, double qy,
                               T* o)
{
    const double r = rho * lam / lam0;
    o[E_RM1] = T(r - 1.0);
    o[E_R] = T(r);
    o[E_I2L] = T(0.5 / lam);
    o[E_DI2L] = T(0.5 / lam - 0.5 / lam0);
    const double s = (1.0 - pr) * 4.0 * lam * lam / (5.0 * rho);
    o[E_L] = T(-s * (qx * U + qy * V));
    o[E_L + 1] = T(s * qx);
    o[E_L + 2] = T(s * qy);
    o[E_L + 3] = T(0);
    o[E_Q] = T(2.0 * lam * (U * U + V * V) - 4.0);
    o[E_Q + 1] = T(-4.0 * lam * U);
    o[E_Q + 2] = T(-4.0 * lam * V);
    o[E_Q + 3] = T(2.0 * lam);
}

// Horner evaluation of the bivariate cubic with monomials 1, u, v, u^2, uv, v^2, u^3, u^2 v, u v^2, v^3
template <typename T>
__device__ __forceinline__ T cubic(const T* c, T u, T v)
{
    T yv = c[0] + v * (c[2] + v * (c[5] + v * c[9]));
    T ux = (c[1] + v * (c[4] + v * c[8])) + u * ((c[3] + v * c[7]) + u * c[6]);
    return yv + u * ux;
}

// ----------------------------------------------------------------------- analytic velocity sums
// Discrete sums of polynomial x Maxwellian over the tensor velocity grid factor into 1-D sums
//   X[p] = sum_i wu_i u_i^p exp(-lam (u_i - U)^2)  (over u_i > 0, u_i < 0, u_i = 0 or all),
//   Y[q] likewise in v,  so  sum_a w_a u^p v^q rho (lam/pi) e^{-lam |u - U|^2} = rho lam/pi X[p] Y[q].

template <typename P>
struct SumsT {
    P s[4][9];   // [0] all, [1] positive nodes, [2] negative nodes, [3] zero nodes; powers 0..8
};

// polynomial in (u, v) of total degree <= 4
template <typename P>
struct PolyT {
    P c[5][5];
    __device__ void zero()
    {
#pragma unroll
        for (int p = 0; p < 5; ++p)
#pragma unroll
            for (int q = 0; q < 5; ++q) c[p][q] = P(0);
    }
};

// C = u A (dir 0) or v A (dir 1), truncated at total degree 4: every product in the face parameters has a
// monomial u_n or u_t as one factor, so it shifts the coefficients by one power
template <typename P>
__device__ __forceinline__ void poly_shift(int dir, const PolyT<P>& A, PolyT<P>& C)
{
    C.zero();
    if (dir == 0) {
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4 - p; ++q)
                if (A.c[p][q] != P(0)) C.c[p + 1][q] = A.c[p][q];
    } else {
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4 - p; ++q)
                if (A.c[p][q] != P(0)) C.c[p][q + 1] = A.c[p][q];
    }
}

// P_h(a) = a0 + a1 u + a2 v + a3/2 (u^2 + v^2 + 1/(2 lam)),  P_b(a) = P_h(a) + a3/(2 lam)
template <typename P>
__device__ inline void poly_P(const double* a, double i2l, bool for_b, PolyT<P>& out)
{
    out.zero();
    out.c[0][0] = P(a[0] + 0.5 * a[3] * i2l + (for_b ? a[3] * i2l : 0.0));
    out.c[1][0] = P(a[1]);
    out.c[0][1] = P(a[2]);
    out.c[2][0] = P(0.5 * a[3]);
    out.c[0][2] = P(0.5 * a[3]);
}

// moments sum w psi [Q H ; R B] over the grid part selected by (rx, ry), H = pref e^{..}, B = H i2l:
//   (sum Q H, sum u Q H, sum v Q H, 1/2 sum (|u|^2 Q H + R B)).  The selected rows of the 1-D sums are copied
// through constant indices first, so that everything stays in registers.
template <typename P>
__device__ __forceinline__ void sum_row(const SumsT<P>& X, int r, P (&o)[9])
{
#pragma unroll
    for (int q = 0; q < 9; ++q) o[q] = r == 0 ? X.s[0][q] : r == 1 ? X.s[1][q] : r == 2 ? X.s[2][q] : X.s[3][q];
}

template <typename P>
__device__ __forceinline__ void mom4(const PolyT<P>& Q, const PolyT<P>& R, const SumsT<P>& X, int rx, const SumsT<P>& Y,
                                     int ry, P pref, P i2l, P out[4])
{
    P xr[9], yr[9];
    sum_row(X, rx, xr);
    sum_row(Y, ry, yr);
    P o0 = 0, o1 = 0, o2 = 0, o3 = 0, ob = 0;
#pragma unroll
    for (int p = 0; p < 5; ++p)
#pragma unroll
        for (int q = 0; q < 5 - p; ++q) {
            const P a = Q.c[p][q], r = R.c[p][q];
            if (a != P(0)) {
                o0 += a * xr[p] * yr[q];
                o1 += a * xr[p + 1] * yr[q];
                o2 += a * xr[p] * yr[q + 1];
                o3 += a * (xr[p + 2] * yr[q] + xr[p] * yr[q + 2]);
            }
            if (r != P(0)) ob += r * xr[p] * yr[q];
        }
    out[0] = pref * o0;
    out[1] = pref * o1;
    out[2] = pref * o2;
    out[3] = P(0.5) * pref * (o3 + i2l * ob);
}

}  // namespace hb
