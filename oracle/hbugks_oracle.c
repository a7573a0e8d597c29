/*
 * HB-UGKS CPU oracle — plain, scalar, FP64.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this file: it is built and
 * loaded only by tests/, by __graft_entry__.smoke() and by bench.py's cpu_baseline / reference leg.
 * It shares no source, header, table or helper with the CUDA path (paper_2605_03479_gb300/csrc).
 *
 * What it computes: one pseudo-time iteration of the time-domain harmonic balance unified gas-kinetic
 * scheme (Zhu, Wu, Wei, Xu, arXiv 2605.03479), Section 2, in the order of the paper's text:
 *   local pseudo-time steps (Eq. dt_hb, nu_conv, dt_face)                 -> cell_steps()
 *   limited reconstruction + kinetic averaging at the interface (Sec 2.2) -> face_flux()
 *   interface Maxwellian, slopes a_n, a_t, A, coefficients C1..C5 (Eq. C_coeffs)
 *   micro flux (Eq. micro_flux), macro flux as its velocity moments (Eq. macro_flux)
 *   diffuse multiscale wall with impermeability density (Eqs. bc_vel, bc_temp, bc_diffuse, rho_wall)
 *   macro update with spectral source (Eq. fv_W), micro update, implicit collision (Eq. fv_h)
 *   level-0 residual (Eq. benchmark_residuals)
 * Everything is evaluated per velocity on the full 2-D discrete grid; every velocity sum is a plain
 * sum over that grid.
 *
 * Units: lengths in cavity heights H, velocities in sqrt(2 R T0) (so R T0 = 1/2), temperatures in T0.
 * lambda = 1/(2RT); lam_ref = lambda(T0) (= 1 in these units).  D = 2, K = 1 (Sec 2.1).
 *
 * Readings of points the paper leaves open (the CUDA path takes the same ones):
 *   - reduced Shakhov terms H+, B+ : g+ of Eq. shakhov integrated over the internal variable xi;
 *   - heat flux for the Shakhov term of the cell update taken from h^k (q^k);
 *   - limiter = van Leer on non-uniform spacing; one-sided difference in wall-adjacent cells;
 *   - a_n^{L,R} from one-sided differences of W between the cell centres and the kinetic average W_0;
 *     a_t from the velocity moments of the upwind tangential slopes; A from the compatibility condition;
 *     each inverted with the continuous-Maxwellian closed form;
 *   - C1..C5 by their Taylor series in x = dG/tau for x < 1, by the printed forms otherwise;
 *   - one dG per cell (max over levels of nu_conv), u_max = truncation bound of the velocity grid;
 *   - wall: incident part from the interior reconstruction through the same integral solution, with
 *     the wall-side equilibrium taken from the mixed (incident + free-transport-reflected) distribution
 *     (pinned by zero wall mass flux, the rest fixed point, mirror and transpose symmetries and the
 *     collisionless limits of the oscillating lid; the choice of that equilibrium itself has no closed form
 *     to compare with);
 *   - velocity nodes with u_n == 0 at an interior face take the average of the two reconstructions.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, ny;
    const double *xn, *yn;      /* mesh nodes, nx+1 and ny+1 values */
    int nu, nv;
    const double *u, *wu;       /* 1-D velocity nodes and weights (x component) */
    const double *v, *wv;       /* 1-D velocity nodes and weights (y component) */
    double umax, vmax;          /* truncation bounds of the velocity grid (Eq. nu_conv) */
    int nt;                     /* number of sub-time levels N_T = 2 N_H + 1 */
    double omega;               /* angular frequency */
    double mu0;                 /* viscosity at T0 */
    double w_vss;               /* viscosity index: mu = mu0 (T/T0)^w */
    double pr;                  /* Prandtl number of the Shakhov model */
    double cfl;
    int face_step;              /* 0: min(dG_L, dG_R); 1: harmonic mean (Eq. dt_face) */
    double gam;                 /* ratio of specific heats in the sound speed */
    double lam_ref;             /* lambda at T0 */
    double wall[4][9];          /* walls 0 bottom, 1 right, 2 top, 3 left: mean U, V, T; Re/Im of U, V, T amplitudes */
    double theta0;              /* phase of level 0 in radians (0 for HB) */
    double dt_fixed;            /* > 0: one global step for every cell and face (time-domain mode) */
    int first_order;            /* 1: zero slopes (debug / test mode) */
    int spectral_implicit;      /* 1: the spectral source at the new iterate (solved across levels per cell and
                                   velocity); 0: at the old iterate, as printed in Eqs. fv_W, fv_h */
} orc_problem;

/* ---------------------------------------------------------------- spectral derivative matrix */

/* Eq. D_explicit: E_nm = 1/2 (-1)^(n-m) csc(pi (n-m)/N_T), E_nn = 0, for odd N_T. */
void orc_E_matrix(int nt, double *E)
{
    for (int n = 0; n < nt; n++)
        for (int m = 0; m < nt; m++) {
            if (n == m) { E[n * nt + m] = 0.0; continue; }
            int d = n - m;
            double sgn = (d % 2 == 0) ? 1.0 : -1.0;
            E[n * nt + m] = 0.5 * sgn / sin(M_PI * (double)d / (double)nt);
        }
}

/* ------------------------------------------------------------- UGKS time-integration weights */

/* Eq. C_coeffs.  For x = dG/tau < 1 the printed forms cancel, so each is summed from its Taylor
 * series in x (derived by expanding exp(-x) in the printed forms); otherwise the printed forms are used
 * with 1 - exp(-x) = -expm1(-x). */
void orc_ugks_coeffs(double dG, double tau, double C[5])
{
    double x = dG / tau;
    if (x < 1.0) {
        /* t_j = x^j / j!  (j = 1..NTERM) */
        enum { NTERM = 26 };
        double t[NTERM + 1];
        t[0] = 1.0;
        for (int j = 1; j <= NTERM; j++) t[j] = t[j - 1] * x / (double)j;
        double s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0;
        /* sum from the smallest term up */
        for (int j = NTERM; j >= 1; j--) {
            double sg = (j % 2 == 1) ? 1.0 : -1.0;          /* (-1)^(j+1) */
            s4 += sg * t[j];                                 /* 1 - e^-x            */
            if (j >= 2) s1 += -sg * t[j];                    /* x - (1 - e^-x)      */
            if (j >= 3) s2 += sg * (double)(2 - j) * t[j];   /* 2(1-e^-x) - x - x e^-x */
            if (j >= 3) s3 += sg * t[j];                     /* x^2/2 - x + (1-e^-x) */
            s5 += sg * (double)(j - 1) * t[j];               /* x e^-x - (1-e^-x)   */
        }
        C[0] = tau * s1;
        C[1] = tau * tau * s2;
        C[2] = tau * tau * s3;
        C[3] = tau * s4;
        C[4] = tau * tau * s5;
    } else {
        double phi = -expm1(-x);
        double ex = exp(-x);
        C[0] = dG - tau * phi;
        C[1] = 2.0 * tau * tau * phi - tau * dG - tau * dG * ex;
        C[2] = 0.5 * dG * dG - tau * dG + tau * tau * phi;
        C[3] = tau * phi;
        C[4] = tau * dG * ex - tau * tau * phi;
    }
}

/* ------------------------------------------------------- Maxwellian slope coefficients a */

/* Given w = (dW)/rho, the velocity moments (per unit density) of (a . psi) g for the Maxwellian g with
 * (U, V, lambda), D = 2, K = 1, solve for a = (a1, a2, a3, a4) where
 * a . psi = a1 + a2 u + a3 v + a4 (u^2 + v^2 + xi^2)/2 (Sec 2.2, Taylor expansion of the Maxwellian).
 * Closed form of the 4x4 moment system of the continuous Maxwellian. */
void orc_micro_slope(const double w[4], double U, double V, double lam, double a[4])
{
    const double K = 1.0;
    double R2 = w[1] - U * w[0];
    double R3 = w[2] - V * w[0];
    double R4 = 2.0 * w[3] - (U * U + V * V + (K + 2.0) / (2.0 * lam)) * w[0];
    a[3] = 4.0 * lam * lam / (K + 2.0) * (R4 - 2.0 * U * R2 - 2.0 * V * R3);
    a[2] = 2.0 * lam * R3 - V * a[3];
    a[1] = 2.0 * lam * R2 - U * a[3];
    a[0] = w[0] - U * a[1] - V * a[2] - 0.5 * a[3] * (U * U + V * V + (K + 2.0) / (2.0 * lam));
}

/* (a . psi) integrated over xi against g (for h) and against xi^2 g (for b), divided by H resp. B:
 *   h: a1 + a2 u + a3 v + a4/2 (u^2 + v^2 + 1/(2 lam))
 *   b: a1 + a2 u + a3 v + a4/2 (u^2 + v^2 + 3/(2 lam))  */
static double poly_h(const double a[4], double u, double v, double lam)
{
    return a[0] + a[1] * u + a[2] * v + 0.5 * a[3] * (u * u + v * v + 1.0 / (2.0 * lam));
}
static double poly_b(const double a[4], double u, double v, double lam)
{
    return a[0] + a[1] * u + a[2] * v + 0.5 * a[3] * (u * u + v * v + 3.0 / (2.0 * lam));
}

/* ------------------------------------------------------------ equilibria and moments */

/* primitive variables from W = (rho, rho U, rho V, rho E), rho E = rho |U|^2/2 + 3 rho / (4 lambda) */
static void prim(const double W[4], double *rho, double *U, double *V, double *lam)
{
    *rho = W[0];
    *U = W[1] / W[0];
    *V = W[2] / W[0];
    *lam = 0.75 * W[0] / (W[3] - 0.5 * W[0] * ((*U) * (*U) + (*V) * (*V)));
}

/* tau = mu / p, mu = mu0 (T/T0)^w, T/T0 = lam_ref/lam, p = rho/(2 lam) */
static double relax_time(const orc_problem *P, double rho, double lam)
{
    double mu = P->mu0 * pow(P->lam_ref / lam, P->w_vss);
    return mu / (rho / (2.0 * lam));
}

/* reduced Maxwellian H = int g dxi and B = int xi^2 g dxi (Eq. maxwellian with K = 1) */
static void maxwell(double rho, double U, double V, double lam, double u, double v, double *H, double *B)
{
    double c2 = (u - U) * (u - U) + (v - V) * (v - V);
    *H = rho * (lam / M_PI) * exp(-lam * c2);
    *B = *H / (2.0 * lam);
}

/* reduced Shakhov corrections (Eq. shakhov integrated over xi with K = 1):
 *   H+ = (1-Pr) c.q /(5 p RT) (|c|^2/RT - 4) H,  B+ = (1-Pr) c.q /(5 p RT) (|c|^2/RT - 2) B  */
static void shakhov(const orc_problem *P, double rho, double U, double V, double lam, double qx, double qy,
                    double u, double v, double H, double B, double *Hp, double *Bp)
{
    double RT = 1.0 / (2.0 * lam);
    double p = rho * RT;
    double cx = u - U, cy = v - V;
    double c2 = cx * cx + cy * cy;
    double s = (1.0 - P->pr) * (cx * qx + cy * qy) / (5.0 * p * RT);
    *Hp = s * (c2 / RT - 4.0) * H;
    *Bp = s * (c2 / RT - 2.0) * B;
}

/* conservative moments (Eq. moment, reduced form): W = sum w (h, u h, v h, (|u|^2 h + b)/2) */
static void moments_W(const orc_problem *P, const double *h, const double *b, double W[4])
{
    W[0] = W[1] = W[2] = W[3] = 0.0;
    for (int jv = 0; jv < P->nv; jv++)
        for (int iu = 0; iu < P->nu; iu++) {
            int a = jv * P->nu + iu;
            double u = P->u[iu], v = P->v[jv], w = P->wu[iu] * P->wv[jv];
            W[0] += w * h[a];
            W[1] += w * u * h[a];
            W[2] += w * v * h[a];
            W[3] += w * 0.5 * ((u * u + v * v) * h[a] + b[a]);
        }
}

/* heat flux (Eq. heatflux, reduced form): q = 1/2 sum w c (|c|^2 h + b), c = u - U */
static void heat_flux(const orc_problem *P, const double *h, const double *b, double U, double V, double q[2])
{
    q[0] = q[1] = 0.0;
    for (int jv = 0; jv < P->nv; jv++)
        for (int iu = 0; iu < P->nu; iu++) {
            int a = jv * P->nu + iu;
            double cx = P->u[iu] - U, cy = P->v[jv] - V, w = P->wu[iu] * P->wv[jv];
            double e = (cx * cx + cy * cy) * h[a] + b[a];
            q[0] += 0.5 * w * cx * e;
            q[1] += 0.5 * w * cy * e;
        }
}

/* ---------------------------------------------------------------------------- geometry */

typedef struct {
    double *xc, *dx, *yc, *dy;
} geom;

static void make_geom(const orc_problem *P, geom *g)
{
    g->xc = malloc(sizeof(double) * P->nx);
    g->dx = malloc(sizeof(double) * P->nx);
    g->yc = malloc(sizeof(double) * P->ny);
    g->dy = malloc(sizeof(double) * P->ny);
    for (int i = 0; i < P->nx; i++) { g->xc[i] = 0.5 * (P->xn[i] + P->xn[i + 1]); g->dx[i] = P->xn[i + 1] - P->xn[i]; }
    for (int j = 0; j < P->ny; j++) { g->yc[j] = 0.5 * (P->yn[j] + P->yn[j + 1]); g->dy[j] = P->yn[j + 1] - P->yn[j]; }
}
static void free_geom(geom *g) { free(g->xc); free(g->dx); free(g->yc); free(g->dy); }

/* wall state at level n (Eqs. bc_vel, bc_temp): mean + Re(amp e^{i theta}), theta = theta0 + 2 pi n / N_T */
static void wall_state(const orc_problem *P, int wall, int n, double *Uw, double *Vw, double *Tw)
{
    const double *p = P->wall[wall];
    double th = P->theta0 + 2.0 * M_PI * (double)n / (double)P->nt;
    double c = cos(th), s = sin(th);
    *Uw = p[0] + (p[3] * c - p[4] * s);
    *Vw = p[1] + (p[5] * c - p[6] * s);
    *Tw = p[2] + (p[7] * c - p[8] * s);
}

/* ------------------------------------------------------------------- local pseudo-time steps */

/* Solve A x = r in place (r becomes x) for an n x n matrix A (row-major, overwritten): Gaussian elimination with
 * partial pivoting, the textbook algorithm. */
static void solve_dense(int n, double* A, double* r)
{
    for (int k = 0; k < n; k++) {
        int piv = k;
        for (int i = k + 1; i < n; i++)
            if (fabs(A[i * n + k]) > fabs(A[piv * n + k])) piv = i;
        if (piv != k) {
            for (int j = 0; j < n; j++) { double t = A[k * n + j]; A[k * n + j] = A[piv * n + j]; A[piv * n + j] = t; }
            double t = r[k]; r[k] = r[piv]; r[piv] = t;
        }
        for (int i = k + 1; i < n; i++) {
            double f = A[i * n + k] / A[k * n + k];
            for (int j = k; j < n; j++) A[i * n + j] -= f * A[k * n + j];
            r[i] -= f * r[k];
        }
    }
    for (int k = n - 1; k >= 0; k--) {
        double s = r[k];
        for (int j = k + 1; j < n; j++) s -= A[k * n + j] * r[j];
        r[k] = s / A[k * n + k];
    }
}

/* Eqs. dt_hb, nu_conv: dG_i = CFL / (nu_conv,i + omega N_H), one value per cell (largest nu over levels) */
static void cell_steps(const orc_problem *P, const geom *g, const double *W, double *dG)
{
    int Nc = P->nx * P->ny;
    int NH = (P->nt - 1) / 2;
    for (int j = 0; j < P->ny; j++)
        for (int i = 0; i < P->nx; i++) {
            int c = j * P->nx + i;
            if (P->dt_fixed > 0.0) { dG[c] = P->dt_fixed; continue; }
            double numax = 0.0;
            for (int n = 0; n < P->nt; n++) {
                double rho, U, V, lam;
                prim(&W[(n * Nc + c) * 4], &rho, &U, &V, &lam);
                double cs = sqrt(P->gam / (2.0 * lam));
                double ut = fmax(fabs(P->umax), fabs(U)) + cs;
                double vt = fmax(fabs(P->vmax), fabs(V)) + cs;
                double nu = (g->dy[j] * ut + g->dx[i] * vt) / (g->dx[i] * g->dy[j]);
                if (nu > numax) numax = nu;
            }
            dG[c] = P->cfl / (numax + P->omega * (double)NH);
        }
}

/* ---------------------------------------------------------------------------- slopes */

/* van Leer limited slope from backward and forward divided differences */
static double van_leer(double s1, double s2)
{
    double den = fabs(s1) + fabs(s2);
    if (den == 0.0) return 0.0;
    double sg1 = (s1 > 0) - (s1 < 0), sg2 = (s2 > 0) - (s2 < 0);
    return (sg1 + sg2) * fabs(s1) * fabs(s2) / den;
}

/* slopes of one level's array f[c*Nv + a] in x (sx) and y (sy) */
static void slopes(const orc_problem *P, const geom *g, const double *f, double *sx, double *sy)
{
    int Nv = P->nu * P->nv, nx = P->nx, ny = P->ny;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int c = j * nx + i;
            for (int a = 0; a < Nv; a++) {
                if (P->first_order) { sx[(size_t)c * Nv + a] = 0.0; sy[(size_t)c * Nv + a] = 0.0; continue; }
                double f0 = f[(size_t)c * Nv + a];
                double s1 = 0.0, s2 = 0.0;
                /* x */
                if (i > 0) s1 = (f0 - f[(size_t)(c - 1) * Nv + a]) / (g->xc[i] - g->xc[i - 1]);
                if (i < nx - 1) s2 = (f[(size_t)(c + 1) * Nv + a] - f0) / (g->xc[i + 1] - g->xc[i]);
                if (i == 0) s1 = s2;
                if (i == nx - 1) s2 = s1;
                sx[(size_t)c * Nv + a] = (nx == 1) ? 0.0 : van_leer(s1, s2);
                /* y */
                if (j > 0) s1 = (f0 - f[(size_t)(c - nx) * Nv + a]) / (g->yc[j] - g->yc[j - 1]);
                if (j < ny - 1) s2 = (f[(size_t)(c + nx) * Nv + a] - f0) / (g->yc[j + 1] - g->yc[j]);
                if (j == 0) s1 = s2;
                if (j == ny - 1) s2 = s1;
                sy[(size_t)c * Nv + a] = (ny == 1) ? 0.0 : van_leer(s1, s2);
            }
        }
}

/* -------------------------------------------------------------------------- face flux */

typedef struct {
    const orc_problem *P;
    int n;                       /* level */
    const double *h, *b;         /* level-n arrays [c*Nv + a] */
    const double *sxh, *syh, *sxb, *syb;
    const double *W;             /* all levels [ (n Nc + c) 4 + p ] */
    const double *dG;
    int Nc, Nv;
    /* scratch per velocity */
    double *h0, *b0, *snh, *sth, *snb, *stb, *Hf, *Bf;
    int *side;                   /* +1: from L, -1: from R, 0: average */
} face_ctx;

/*
 * Flux through one face with unit normal along `axis` (0: x, 1: y), between cell L (low side) and
 * cell R (high side).  L < 0 (wall below) or R < 0 (wall above) marks a wall face; `wall` is its id.
 * xf: face coordinate along the normal; xL, xR: cell-centre coordinates along the normal.
 * Outputs: Hf[a], Bf[a] = micro flux rates (Eq. micro_flux divided by dG_f), F[4] = macro flux rate.
 */
static void face_flux(face_ctx *X, int axis, int L, int R, double xf, double xL, double xR, int wall, double F[4])
{
    const orc_problem *P = X->P;
    int Nv = X->Nv, Nc = X->Nc;
    const double *sn_h = axis == 0 ? X->sxh : X->syh, *st_h = axis == 0 ? X->syh : X->sxh;
    const double *sn_b = axis == 0 ? X->sxb : X->syb, *st_b = axis == 0 ? X->syb : X->sxb;
    int is_wall = (L < 0 || R < 0);
    int I = L >= 0 ? L : R;                /* interior cell of a wall face */
    double xI = L >= 0 ? xL : xR;
    /* inward normal sign of a wall face: +1 if the fluid is on the high side */
    double nin = (L < 0) ? 1.0 : -1.0;

    /* --- reconstruction at the interface and upwind selection (Sec 2.2) */
    for (int jv = 0; jv < P->nv; jv++)
        for (int iu = 0; iu < P->nu; iu++) {
            int a = jv * P->nu + iu;
            double un = axis == 0 ? P->u[iu] : P->v[jv];
            if (is_wall) {
                size_t k = (size_t)I * Nv + a;
                X->h0[a] = X->h[k] + sn_h[k] * (xf - xI);
                X->b0[a] = X->b[k] + sn_b[k] * (xf - xI);
                X->snh[a] = sn_h[k]; X->sth[a] = st_h[k];
                X->snb[a] = sn_b[k]; X->stb[a] = st_b[k];
                X->side[a] = (un * nin < 0.0) ? 1 : ((un * nin > 0.0) ? -1 : 0); /* 1: incident */
                continue;
            }
            size_t kL = (size_t)L * Nv + a, kR = (size_t)R * Nv + a;
            double hL = X->h[kL] + sn_h[kL] * (xf - xL), hR = X->h[kR] + sn_h[kR] * (xf - xR);
            double bL = X->b[kL] + sn_b[kL] * (xf - xL), bR = X->b[kR] + sn_b[kR] * (xf - xR);
            if (un > 0.0) {
                X->h0[a] = hL; X->b0[a] = bL;
                X->snh[a] = sn_h[kL]; X->sth[a] = st_h[kL]; X->snb[a] = sn_b[kL]; X->stb[a] = st_b[kL];
                X->side[a] = 1;
            } else if (un < 0.0) {
                X->h0[a] = hR; X->b0[a] = bR;
                X->snh[a] = sn_h[kR]; X->sth[a] = st_h[kR]; X->snb[a] = sn_b[kR]; X->stb[a] = st_b[kR];
                X->side[a] = -1;
            } else {
                X->h0[a] = 0.5 * (hL + hR); X->b0[a] = 0.5 * (bL + bR);
                X->snh[a] = 0.5 * (sn_h[kL] + sn_h[kR]); X->sth[a] = 0.5 * (st_h[kL] + st_h[kR]);
                X->snb[a] = 0.5 * (sn_b[kL] + sn_b[kR]); X->stb[a] = 0.5 * (st_b[kL] + st_b[kR]);
                X->side[a] = 0;
            }
        }

    /* --- wall: Maxwellian of the wall and free-transport estimate of the wall density */
    double Uw = 0, Vw = 0, Tw = 1, lamw = 1, rhow0 = 0;
    if (is_wall) {
        wall_state(P, wall, X->n, &Uw, &Vw, &Tw);
        lamw = P->lam_ref / Tw;
        double num = 0.0, den = 0.0;
        for (int jv = 0; jv < P->nv; jv++)
            for (int iu = 0; iu < P->nu; iu++) {
                int a = jv * P->nu + iu;
                double un = axis == 0 ? P->u[iu] : P->v[jv];
                double w = P->wu[iu] * P->wv[jv];
                double Hw, Bw;
                maxwell(1.0, Uw, Vw, lamw, P->u[iu], P->v[jv], &Hw, &Bw);
                if (un * nin < 0.0) num += w * fabs(un) * X->h0[a];
                else if (un * nin > 0.0) den += w * fabs(un) * Hw;
            }
        rhow0 = num / den;
    }

    /* --- kinetic average W_0 at the interface (wall: incident reconstruction + reflected rho_w0 H_w) */
    double W0[4] = {0, 0, 0, 0};
    for (int jv = 0; jv < P->nv; jv++)
        for (int iu = 0; iu < P->nu; iu++) {
            int a = jv * P->nu + iu;
            double u = P->u[iu], v = P->v[jv], w = P->wu[iu] * P->wv[jv];
            double hh = X->h0[a], bb = X->b0[a];
            if (is_wall && X->side[a] != 1) {
                double Hw, Bw;
                maxwell(1.0, Uw, Vw, lamw, u, v, &Hw, &Bw);
                hh = (X->side[a] == -1) ? rhow0 * Hw : 0.0;
                bb = (X->side[a] == -1) ? rhow0 * Bw : 0.0;
            }
            W0[0] += w * hh;
            W0[1] += w * u * hh;
            W0[2] += w * v * hh;
            W0[3] += w * 0.5 * ((u * u + v * v) * hh + bb);
        }
    double rho0, U0, V0, lam0;
    prim(W0, &rho0, &U0, &V0, &lam0);
    /* heat flux of the same distribution (Shakhov part of the interface equilibrium) */
    double q0[2] = {0, 0};
    for (int jv = 0; jv < P->nv; jv++)
        for (int iu = 0; iu < P->nu; iu++) {
            int a = jv * P->nu + iu;
            double u = P->u[iu], v = P->v[jv], w = P->wu[iu] * P->wv[jv];
            double hh = X->h0[a], bb = X->b0[a];
            if (is_wall && X->side[a] != 1) {
                double Hw, Bw;
                maxwell(1.0, Uw, Vw, lamw, u, v, &Hw, &Bw);
                hh = (X->side[a] == -1) ? rhow0 * Hw : 0.0;
                bb = (X->side[a] == -1) ? rhow0 * Bw : 0.0;
            }
            double cx = u - U0, cy = v - V0;
            double e = (cx * cx + cy * cy) * hh + bb;
            q0[0] += 0.5 * w * cx * e;
            q0[1] += 0.5 * w * cy * e;
        }
    double tau = relax_time(P, rho0, lam0);

    /* --- face step (Eq. dt_face) and time-integration weights (Eq. C_coeffs) */
    double dGf;
    if (is_wall) dGf = X->dG[I];
    else if (P->face_step == 1) dGf = 2.0 * X->dG[L] * X->dG[R] / (X->dG[L] + X->dG[R]);
    else dGf = fmin(X->dG[L], X->dG[R]);
    double C[5];
    orc_ugks_coeffs(dGf, tau, C);

    /* --- equilibrium slopes: normal a^L, a^R from W at cell centres and W_0; tangential a_t; A */
    double aL[4] = {0, 0, 0, 0}, aR[4] = {0, 0, 0, 0}, at[4], A[4];
    {
        double w[4];
        if (L >= 0) {
            const double *WL = &X->W[((size_t)X->n * Nc + L) * 4];
            for (int p = 0; p < 4; p++) w[p] = (W0[p] - WL[p]) / (xf - xL) / rho0;
            orc_micro_slope(w, U0, V0, lam0, aL);
        }
        if (R >= 0) {
            const double *WR = &X->W[((size_t)X->n * Nc + R) * 4];
            for (int p = 0; p < 4; p++) w[p] = (WR[p] - W0[p]) / (xR - xf) / rho0;
            orc_micro_slope(w, U0, V0, lam0, aR);
        }
        if (is_wall) { if (L < 0) memcpy(aL, aR, sizeof aL); else memcpy(aR, aL, sizeof aR); }
        double Wt[4] = {0, 0, 0, 0};
        for (int jv = 0; jv < P->nv; jv++)
            for (int iu = 0; iu < P->nu; iu++) {
                int a = jv * P->nu + iu;
                double u = P->u[iu], v = P->v[jv], wt = P->wu[iu] * P->wv[jv];
                Wt[0] += wt * X->sth[a];
                Wt[1] += wt * u * X->sth[a];
                Wt[2] += wt * v * X->sth[a];
                Wt[3] += wt * 0.5 * ((u * u + v * v) * X->sth[a] + X->stb[a]);
            }
        for (int p = 0; p < 4; p++) w[p] = Wt[p] / rho0;
        orc_micro_slope(w, U0, V0, lam0, at);
        /* compatibility: moments of (A.psi) g0 = - moments of (u_n a_n + u_t a_t) g0 */
        double M[4] = {0, 0, 0, 0};
        for (int jv = 0; jv < P->nv; jv++)
            for (int iu = 0; iu < P->nu; iu++) {
                double u = P->u[iu], v = P->v[jv], wt = P->wu[iu] * P->wv[jv];
                double un = axis == 0 ? u : v, ut = axis == 0 ? v : u;
                const double *an = (un > 0.0) ? aL : ((un < 0.0) ? aR : NULL);
                double H0, B0;
                maxwell(rho0, U0, V0, lam0, u, v, &H0, &B0);
                double ph, pb;
                if (an) {
                    ph = un * poly_h(an, u, v, lam0) + ut * poly_h(at, u, v, lam0);
                    pb = un * poly_b(an, u, v, lam0) + ut * poly_b(at, u, v, lam0);
                } else {
                    ph = 0.5 * un * (poly_h(aL, u, v, lam0) + poly_h(aR, u, v, lam0)) + ut * poly_h(at, u, v, lam0);
                    pb = 0.5 * un * (poly_b(aL, u, v, lam0) + poly_b(aR, u, v, lam0)) + ut * poly_b(at, u, v, lam0);
                }
                M[0] += wt * ph * H0;
                M[1] += wt * u * ph * H0;
                M[2] += wt * v * ph * H0;
                M[3] += wt * 0.5 * ((u * u + v * v) * ph * H0 + pb * B0);
            }
        for (int p = 0; p < 4; p++) w[p] = -M[p] / rho0;
        orc_micro_slope(w, U0, V0, lam0, A);
    }

    /* --- time-integrated interface distribution (Eq. integral_solution integrated over [0, dG_f]) */
    for (int jv = 0; jv < P->nv; jv++)
        for (int iu = 0; iu < P->nu; iu++) {
            int a = jv * P->nu + iu;
            double u = P->u[iu], v = P->v[jv];
            double un = axis == 0 ? u : v, ut = axis == 0 ? v : u;
            double H0, B0, Hp, Bp;
            maxwell(rho0, U0, V0, lam0, u, v, &H0, &B0);
            shakhov(P, rho0, U0, V0, lam0, q0[0], q0[1], u, v, H0, B0, &Hp, &Bp);
            double ph, pb;
            if (X->side[a] == 0 && !is_wall) {
                ph = 0.5 * un * (poly_h(aL, u, v, lam0) + poly_h(aR, u, v, lam0)) + ut * poly_h(at, u, v, lam0);
                pb = 0.5 * un * (poly_b(aL, u, v, lam0) + poly_b(aR, u, v, lam0)) + ut * poly_b(at, u, v, lam0);
            } else {
                const double *an = (un > 0.0) ? aL : aR;
                ph = un * poly_h(an, u, v, lam0) + ut * poly_h(at, u, v, lam0);
                pb = un * poly_b(an, u, v, lam0) + ut * poly_b(at, u, v, lam0);
            }
            double Ih = C[0] * (H0 + Hp) + C[1] * ph * H0 + C[2] * poly_h(A, u, v, lam0) * H0
                      + C[3] * X->h0[a] + C[4] * (un * X->snh[a] + ut * X->sth[a]);
            double Ib = C[0] * (B0 + Bp) + C[1] * pb * B0 + C[2] * poly_b(A, u, v, lam0) * B0
                      + C[3] * X->b0[a] + C[4] * (un * X->snb[a] + ut * X->stb[a]);
            X->Hf[a] = Ih;   /* time integral over [0, dG_f]; turned into a rate below */
            X->Bf[a] = Ib;
        }

    if (is_wall) {
        /* impermeability (Eq. rho_wall) with the time-integrated incident distribution */
        double num = 0.0, den = 0.0;
        for (int jv = 0; jv < P->nv; jv++)
            for (int iu = 0; iu < P->nu; iu++) {
                int a = jv * P->nu + iu;
                double un = axis == 0 ? P->u[iu] : P->v[jv];
                double w = P->wu[iu] * P->wv[jv];
                double Hw, Bw;
                maxwell(1.0, Uw, Vw, lamw, P->u[iu], P->v[jv], &Hw, &Bw);
                if (X->side[a] == 1) num += w * fabs(un) * X->Hf[a];
                else if (X->side[a] == -1) den += w * fabs(un) * Hw * dGf;
            }
        double rhow = num / den;
        for (int jv = 0; jv < P->nv; jv++)
            for (int iu = 0; iu < P->nu; iu++) {
                int a = jv * P->nu + iu;
                double un = axis == 0 ? P->u[iu] : P->v[jv];
                double Hw, Bw;
                maxwell(1.0, Uw, Vw, lamw, P->u[iu], P->v[jv], &Hw, &Bw);
                if (X->side[a] == 1) { X->Hf[a] = un * X->Hf[a] / dGf; X->Bf[a] = un * X->Bf[a] / dGf; }
                else if (X->side[a] == -1) { X->Hf[a] = un * rhow * Hw; X->Bf[a] = un * rhow * Bw; }
                else { X->Hf[a] = 0.0; X->Bf[a] = 0.0; }
            }
    } else {
        for (int jv = 0; jv < P->nv; jv++)
            for (int iu = 0; iu < P->nu; iu++) {
                int a = jv * P->nu + iu;
                double un = axis == 0 ? P->u[iu] : P->v[jv];
                X->Hf[a] = un * X->Hf[a] / dGf;   /* Eq. micro_flux */
                X->Bf[a] = un * X->Bf[a] / dGf;
            }
    }

    /* --- macro flux = conservative moments of the micro flux (Eq. macro_flux) */
    F[0] = F[1] = F[2] = F[3] = 0.0;
    for (int jv = 0; jv < P->nv; jv++)
        for (int iu = 0; iu < P->nu; iu++) {
            int a = jv * P->nu + iu;
            double u = P->u[iu], v = P->v[jv], w = P->wu[iu] * P->wv[jv];
            F[0] += w * X->Hf[a];
            F[1] += w * u * X->Hf[a];
            F[2] += w * v * X->Hf[a];
            F[3] += w * 0.5 * ((u * u + v * v) * X->Hf[a] + X->Bf[a]);
        }
}

/* ------------------------------------------------------------------------- one iteration */

/*
 * Advance W, h, b by `niter` pseudo-time iterations in place.
 * Layouts: W[(n Nc + c) 4 + p], h[(n Nc + c) Nv + a], b likewise, c = j nx + i, a = jv nu + iu.
 * resid (may be NULL): niter x 4 values of Eq. benchmark_residuals (level 0).
 * Returns 0.
 */
int orc_hb_iterate(const orc_problem *P, double *W, double *h, double *b, int niter, double *resid)
{
    int nx = P->nx, ny = P->ny, Nc = nx * ny, Nv = P->nu * P->nv, nt = P->nt;
    size_t NS = (size_t)Nc * Nv;
    geom g;
    make_geom(P, &g);
    double *E = malloc(sizeof(double) * nt * nt);
    orc_E_matrix(nt, E);
    double *dG = malloc(sizeof(double) * Nc);
    double *sxh = malloc(sizeof(double) * NS), *syh = malloc(sizeof(double) * NS);
    double *sxb = malloc(sizeof(double) * NS), *syb = malloc(sizeof(double) * NS);
    double *divh = calloc((size_t)nt * NS, sizeof(double)), *divb = calloc((size_t)nt * NS, sizeof(double));
    double *divW = calloc((size_t)nt * Nc * 4, sizeof(double));
    double *q = malloc(sizeof(double) * nt * Nc * 2);
    double *Wn = malloc(sizeof(double) * nt * Nc * 4);
    double *hn = malloc(sizeof(double) * nt * NS), *bn = malloc(sizeof(double) * nt * NS);
    face_ctx X;
    X.P = P; X.Nc = Nc; X.Nv = Nv; X.W = W; X.dG = dG;
    X.h0 = malloc(sizeof(double) * Nv); X.b0 = malloc(sizeof(double) * Nv);
    X.snh = malloc(sizeof(double) * Nv); X.sth = malloc(sizeof(double) * Nv);
    X.snb = malloc(sizeof(double) * Nv); X.stb = malloc(sizeof(double) * Nv);
    X.Hf = malloc(sizeof(double) * Nv); X.Bf = malloc(sizeof(double) * Nv);
    X.side = malloc(sizeof(int) * Nv);

    for (int it = 0; it < niter; it++) {
        /* (1) local pseudo-time steps from W^k */
        cell_steps(P, &g, W, dG);
        memset(divh, 0, sizeof(double) * nt * NS);
        memset(divb, 0, sizeof(double) * nt * NS);
        memset(divW, 0, sizeof(double) * nt * Nc * 4);

        /* (2) interface fluxes, level by level; accumulate sum_f |L_f| (flux . outward normal) */
        for (int n = 0; n < nt; n++) {
            const double *hl = h + (size_t)n * NS, *bl = b + (size_t)n * NS;
            slopes(P, &g, hl, sxh, syh);
            slopes(P, &g, bl, sxb, syb);
            X.n = n; X.h = hl; X.b = bl; X.sxh = sxh; X.syh = syh; X.sxb = sxb; X.syb = syb;
            double *dh = divh + (size_t)n * NS, *db = divb + (size_t)n * NS, *dW = divW + (size_t)n * Nc * 4;
            double F[4];
            /* faces normal to x: i = 0 .. nx, between cells (i-1, j) and (i, j) */
            for (int j = 0; j < ny; j++)
                for (int i = 0; i <= nx; i++) {
                    int L = (i > 0) ? j * nx + i - 1 : -1;
                    int R = (i < nx) ? j * nx + i : -1;
                    int wall = (i == 0) ? 3 : 1;
                    double xL = (i > 0) ? g.xc[i - 1] : 0.0, xR = (i < nx) ? g.xc[i] : 0.0;
                    face_flux(&X, 0, L, R, P->xn[i], xL, xR, wall, F);
                    double len = g.dy[j];
                    for (int a = 0; a < Nv; a++) {
                        if (L >= 0) { dh[(size_t)L * Nv + a] += len * X.Hf[a]; db[(size_t)L * Nv + a] += len * X.Bf[a]; }
                        if (R >= 0) { dh[(size_t)R * Nv + a] -= len * X.Hf[a]; db[(size_t)R * Nv + a] -= len * X.Bf[a]; }
                    }
                    for (int p = 0; p < 4; p++) {
                        if (L >= 0) dW[L * 4 + p] += len * F[p];
                        if (R >= 0) dW[R * 4 + p] -= len * F[p];
                    }
                }
            /* faces normal to y: j = 0 .. ny, between cells (i, j-1) and (i, j) */
            for (int j = 0; j <= ny; j++)
                for (int i = 0; i < nx; i++) {
                    int L = (j > 0) ? (j - 1) * nx + i : -1;
                    int R = (j < ny) ? j * nx + i : -1;
                    int wall = (j == 0) ? 0 : 2;
                    double yL = (j > 0) ? g.yc[j - 1] : 0.0, yR = (j < ny) ? g.yc[j] : 0.0;
                    face_flux(&X, 1, L, R, P->yn[j], yL, yR, wall, F);
                    double len = g.dx[i];
                    for (int a = 0; a < Nv; a++) {
                        if (L >= 0) { dh[(size_t)L * Nv + a] += len * X.Hf[a]; db[(size_t)L * Nv + a] += len * X.Bf[a]; }
                        if (R >= 0) { dh[(size_t)R * Nv + a] -= len * X.Hf[a]; db[(size_t)R * Nv + a] -= len * X.Bf[a]; }
                    }
                    for (int p = 0; p < 4; p++) {
                        if (L >= 0) dW[L * 4 + p] += len * F[p];
                        if (R >= 0) dW[R * 4 + p] -= len * F[p];
                    }
                }
        }

        /* (3) heat flux of h^k for the Shakhov equilibria of the cell update */
        for (int n = 0; n < nt; n++)
            for (int c = 0; c < Nc; c++) {
                double rho, U, V, lam;
                prim(&W[((size_t)n * Nc + c) * 4], &rho, &U, &V, &lam);
                heat_flux(P, h + (size_t)n * NS + (size_t)c * Nv, b + (size_t)n * NS + (size_t)c * Nv, U, V,
                          &q[(n * Nc + c) * 2]);
            }

        /* (4) macro update with the spectral source (Eq. fv_W) */
        for (int n = 0; n < nt; n++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    int c = j * nx + i;
                    double area = g.dx[i] * g.dy[j];
                    for (int p = 0; p < 4; p++) {
                        double src = 0.0;
                        if (!P->spectral_implicit)
                            for (int m = 0; m < nt; m++) src += E[n * nt + m] * W[((size_t)m * Nc + c) * 4 + p];
                        Wn[((size_t)n * Nc + c) * 4 + p] = W[((size_t)n * Nc + c) * 4 + p]
                            - dG[c] * (divW[((size_t)n * Nc + c) * 4 + p] / area + P->omega * src);
                    }
                }
        if (P->spectral_implicit) {
            /* spectral source at the new iterate: (I + dG omega E) W^{k+1} = W^k - dG div F, per cell and variable */
            double* A = (double*)malloc(sizeof(double) * nt * nt);
            double* r = (double*)malloc(sizeof(double) * nt);
            for (int c = 0; c < Nc; c++)
                for (int p = 0; p < 4; p++) {
                    for (int n = 0; n < nt; n++) {
                        for (int m = 0; m < nt; m++) A[n * nt + m] = (n == m ? 1.0 : 0.0) + dG[c] * P->omega * E[n * nt + m];
                        r[n] = Wn[((size_t)n * Nc + c) * 4 + p];
                    }
                    solve_dense(nt, A, r);
                    for (int n = 0; n < nt; n++) Wn[((size_t)n * Nc + c) * 4 + p] = r[n];
                }
            free(A);
            free(r);
        }

        /* (5) micro update with implicit collision (Eq. fv_h) */
        for (int n = 0; n < nt; n++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    int c = j * nx + i;
                    double area = g.dx[i] * g.dy[j];
                    double r0, U0, V0, l0, r1, U1, V1, l1;
                    prim(&W[((size_t)n * Nc + c) * 4], &r0, &U0, &V0, &l0);
                    prim(&Wn[((size_t)n * Nc + c) * 4], &r1, &U1, &V1, &l1);
                    double t0 = relax_time(P, r0, l0), t1 = relax_time(P, r1, l1);
                    double qx = q[(n * Nc + c) * 2], qy = q[(n * Nc + c) * 2 + 1];
                    double d = dG[c];
                    for (int jv = 0; jv < P->nv; jv++)
                        for (int iu = 0; iu < P->nu; iu++) {
                            int a = jv * P->nu + iu;
                            double u = P->u[iu], v = P->v[jv];
                            size_t k = (size_t)n * NS + (size_t)c * Nv + a;
                            double Hk, Bk, Hpk, Bpk, H1, B1, Hp1, Bp1;
                            maxwell(r0, U0, V0, l0, u, v, &Hk, &Bk);
                            shakhov(P, r0, U0, V0, l0, qx, qy, u, v, Hk, Bk, &Hpk, &Bpk);
                            maxwell(r1, U1, V1, l1, u, v, &H1, &B1);
                            shakhov(P, r1, U1, V1, l1, qx, qy, u, v, H1, B1, &Hp1, &Bp1);
                            double Eh = 0.0, Eb = 0.0;
                            for (int m = 0; m < nt && !P->spectral_implicit; m++) {
                                size_t km = (size_t)m * NS + (size_t)c * Nv + a;
                                Eh += E[n * nt + m] * h[km];
                                Eb += E[n * nt + m] * b[km];
                            }
                            hn[k] = (h[k] - d / area * divh[k] - d * P->omega * Eh
                                     + 0.5 * d * ((H1 + Hp1) / t1 + (Hk + Hpk - h[k]) / t0)) / (1.0 + 0.5 * d / t1);
                            bn[k] = (b[k] - d / area * divb[k] - d * P->omega * Eb
                                     + 0.5 * d * ((B1 + Bp1) / t1 + (Bk + Bpk - b[k]) / t0)) / (1.0 + 0.5 * d / t1);
                        }
                }

        if (P->spectral_implicit) {
            /* spectral source at the new iterate: the update above divided by (1 + dG/(2 tau^{k+1})) is
             * D h^{k+1} = rhs with D = diag(1 + dG/(2 tau_n^{k+1})); with the source it becomes
             * (D + dG omega E) h^{k+1} = D (update above), solved per cell and velocity (same for b) */
            double* A = (double*)malloc(sizeof(double) * nt * nt);
            double* r = (double*)malloc(sizeof(double) * nt);
            double* Dn = (double*)malloc(sizeof(double) * nt);
            for (int c = 0; c < Nc; c++) {
                for (int n = 0; n < nt; n++) {
                    double r1, U1, V1, l1;
                    prim(&Wn[((size_t)n * Nc + c) * 4], &r1, &U1, &V1, &l1);
                    Dn[n] = 1.0 + 0.5 * dG[c] / relax_time(P, r1, l1);
                }
                for (int arr = 0; arr < 2; arr++) {
                    double* x = arr == 0 ? hn : bn;
                    for (int a = 0; a < Nv; a++) {
                        for (int n = 0; n < nt; n++) {
                            for (int m = 0; m < nt; m++)
                                A[n * nt + m] = (n == m ? Dn[n] : 0.0) + dG[c] * P->omega * E[n * nt + m];
                            r[n] = Dn[n] * x[(size_t)n * NS + (size_t)c * Nv + a];
                        }
                        solve_dense(nt, A, r);
                        for (int n = 0; n < nt; n++) x[(size_t)n * NS + (size_t)c * Nv + a] = r[n];
                    }
                }
            }
            free(A);
            free(r);
            free(Dn);
        }

        /* (6) level-0 residual (Eq. benchmark_residuals) */
        if (resid) {
            for (int p = 0; p < 4; p++) {
                double s = 0.0;
                for (int c = 0; c < Nc; c++) {
                    double dd = Wn[(size_t)c * 4 + p] - W[(size_t)c * 4 + p];
                    s += dd * dd;
                }
                resid[it * 4 + p] = sqrt(s / (double)Nc);
            }
        }
        memcpy(W, Wn, sizeof(double) * nt * Nc * 4);
        memcpy(h, hn, sizeof(double) * nt * NS);
        memcpy(b, bn, sizeof(double) * nt * NS);
    }

    free(X.h0); free(X.b0); free(X.snh); free(X.sth); free(X.snb); free(X.stb); free(X.Hf); free(X.Bf); free(X.side);
    free(E); free(dG); free(sxh); free(syh); free(sxb); free(syb); free(divh); free(divb); free(divW); free(q);
    free(Wn); free(hn); free(bn);
    free_geom(&g);
    return 0;
}

/* ----------------------------------------------------------------- fields and probes */

/*
 * Macroscopic fields of one level from the moments of h, b (Sec 3.1.1): out[f * Nc + c] for
 * f = 0 rho, 1 U, 2 V, 3 T/T0, 4 tau_xy (Eq. shear_stress_eval), 5 q_x, 6 q_y, 7 p.
 */
void orc_fields(const orc_problem *P, const double *h, const double *b, int level, double *out)
{
    int Nc = P->nx * P->ny, Nv = P->nu * P->nv;
    for (int c = 0; c < Nc; c++) {
        const double *hc = h + ((size_t)level * Nc + c) * Nv, *bc = b + ((size_t)level * Nc + c) * Nv;
        double W[4], rho, U, V, lam, q[2];
        moments_W(P, hc, bc, W);
        prim(W, &rho, &U, &V, &lam);
        heat_flux(P, hc, bc, U, V, q);
        double txy = 0.0;
        for (int jv = 0; jv < P->nv; jv++)
            for (int iu = 0; iu < P->nu; iu++) {
                int a = jv * P->nu + iu;
                txy += P->wu[iu] * P->wv[jv] * (P->u[iu] - U) * (P->v[jv] - V) * hc[a];
            }
        out[0 * Nc + c] = rho;
        out[1 * Nc + c] = U;
        out[2 * Nc + c] = V;
        out[3 * Nc + c] = P->lam_ref / lam;
        out[4 * Nc + c] = txy;
        out[5 * Nc + c] = q[0];
        out[6 * Nc + c] = q[1];
        out[7 * Nc + c] = rho / (2.0 * lam);
    }
}

/* Probe entry points used by the pin tests (single evaluations of the building blocks). */
void orc_maxwell_grid(const orc_problem *P, double rho, double U, double V, double lam, double *H, double *B)
{
    for (int jv = 0; jv < P->nv; jv++)
        for (int iu = 0; iu < P->nu; iu++) {
            int a = jv * P->nu + iu;
            maxwell(rho, U, V, lam, P->u[iu], P->v[jv], &H[a], &B[a]);
        }
}

void orc_shakhov_grid(const orc_problem *P, double rho, double U, double V, double lam, double qx, double qy,
                      double *Hp, double *Bp)
{
    for (int jv = 0; jv < P->nv; jv++)
        for (int iu = 0; iu < P->nu; iu++) {
            int a = jv * P->nu + iu;
            double H, B;
            maxwell(rho, U, V, lam, P->u[iu], P->v[jv], &H, &B);
            shakhov(P, rho, U, V, lam, qx, qy, P->u[iu], P->v[jv], H, B, &Hp[a], &Bp[a]);
        }
}

void orc_moments(const orc_problem *P, const double *h, const double *b, double W[4], double q[2])
{
    double rho, U, V, lam;
    moments_W(P, h, b, W);
    prim(W, &rho, &U, &V, &lam);
    heat_flux(P, h, b, U, V, q);
}

void orc_cell_steps(const orc_problem *P, const double *W, double *dG)
{
    geom g;
    make_geom(P, &g);
    cell_steps(P, &g, W, dG);
    free_geom(&g);
}

double orc_van_leer(double s1, double s2) { return van_leer(s1, s2); }

double orc_relax_time(const orc_problem *P, double rho, double lam) { return relax_time(P, rho, lam); }
