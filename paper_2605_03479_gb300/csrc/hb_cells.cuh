// Per-velocity kernels of one HB-UGKS iteration on sign-pure velocity blocks.
//
// The discrete velocities are stored in blocks of 32 (one warp lane each) in which u and v each keep one sign
// (a zero node is stored once in each of the adjacent sign classes with its weight split between the copies).
// The upwind side of every x-face is then the same for all lanes of a block, and so is that of every y-face,
// so each cell reconstructs once per velocity block and the result serves the one x-face and the one y-face
// lying downwind of it (Sec 2.2, upwind interface reconstruction):
//   k1_cells : per (cell, level): velocity sums of the reconstruction of h^k at the cell's downwind faces,
//              kept per sign class (half-face sums), and the raw moments of h^k;
//   k4_cells : per (cell, level, 32 velocities): interface micro fluxes (Eq. micro_flux), spectral source and
//              the semi-implicit collision update (Eq. fv_h).
// A CTA of k1_cells owns a tile of cells and one level and runs over all velocity blocks; a CTA of k4_cells
// owns a tile of cells and one velocity block and runs over all levels.  Both stage the tile and its halo in
// shared memory with bulk copies (TMA) completing on an mbarrier.
#pragma once
#include "hb_common.cuh"

namespace hb {

template <typename T>
__device__ __forceinline__ T vleer(T s1, T s2);
template <>
__device__ __forceinline__ double vleer<double>(double s1, double s2)
{
    double p = s1 * s2;
    return p > 0.0 ? (p + p) / (s1 + s2) : 0.0;
}
// single precision: the limited slope needs no correctly rounded division (2-ulp reciprocal form)
template <>
__device__ __forceinline__ float vleer<float>(float s1, float s2)
{
    float p = s1 * s2;
    return p > 0.f ? __fdividef(p + p, s1 + s2) : 0.f;
}

// van Leer slope of a cell from its two neighbours along one axis; a missing neighbour (wall) makes the
// available one-sided difference the slope, a single cell along the axis has none
template <typename T>
__device__ __forceinline__ T slope(T fm, T f0, T fp, T wm, T wp, bool has_m, bool has_p, bool several)
{
    T s1 = (f0 - fm) * wm, s2 = (fp - f0) * wp;
    if (!has_m) s1 = s2;
    if (!has_p) s2 = s1;
    return several ? vleer(s1, s2) : T(0);
}

// 16-byte read-only vector loads of N consecutive parameters (N a multiple of 16 / sizeof(T), p 16-byte aligned)
template <int N>
__device__ __forceinline__ void ldv(const float* p, float* o)
{
#pragma unroll
    for (int k = 0; k < N; k += 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p + k));
        o[k] = v.x; o[k + 1] = v.y; o[k + 2] = v.z; o[k + 3] = v.w;
    }
}
template <int N>
__device__ __forceinline__ void ldv(const double* p, double* o)
{
#pragma unroll
    for (int k = 0; k < N; k += 2) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p + k));
        o[k] = v.x; o[k + 1] = v.y;
    }
}

// spectral source of one cell and lane: sum_d e_d (f_{n-d} - f_{n+d}) for h and b (Eq. D_explicit in paired
// form), levels lv elements apart in shared memory
template <int NH, typename T>
__device__ __forceinline__ void spectral(const T* hc, const T* bc, int n, int nt, int lv, const T* et, T& eh, T& eb)
{
    eh = T(0);
    eb = T(0);
#pragma unroll
    for (int d = 1; d <= NH; ++d) {
        int nm = n - d; nm += nm < 0 ? nt : 0;
        int np = n + d; np -= np >= nt ? nt : 0;
        eh += et[d] * (hc[nm * lv] - hc[np * lv]);
        eb += et[d] * (bc[nm * lv] - bc[np * lv]);
    }
}

__device__ __forceinline__ void mbar_setup(uint64_t* bars, int n)
{
    if (threadIdx.x == 0) {
        for (int k = 0; k < n; ++k) mbar_init(bars + k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

__host__ __device__ constexpr size_t round16(size_t b) { return (b + 15) / 16 * 16; }

// Sum over the 32 lanes of each of v[0..N-1] (N <= 32), recursive halving: after the step with distance d the
// lanes with bit d set hold the upper half of the remaining values.  Returns, on lane l, the total of v[l]
// (0 for l >= N).  v is destroyed.
template <int N, typename T>
__device__ __forceinline__ T lane_totals(T (&v)[N], int lane)
{
    T x[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) x[k] = k < N ? v[k] : T(0);
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const bool hi = (lane & d) != 0;
#pragma unroll
        for (int k = 0; k < d; ++k) {
            const T send = hi ? x[k] : x[k + d];
            const T keep = hi ? x[k + d] : x[k];
            x[k] = keep + __shfl_xor_sync(0xffffffffu, send, d);
        }
    }
    return x[0];
}

// ------------------------------------------------------------------------------ K1: half-face sums

// Velocity sums of one cell's reconstruction at its downwind faces.  Slots of the 23 sums (as for an
// interface with normal n and tangent t, u_n = u.n):
//   0..9   w d0 (1, u, v, u^2, uv, v^2, u^3, u^2 v, u v^2, v^3),  d0 the reconstructed h deviation at the face
//   10..12 w e0 (1, u, v),                                         e0 the same for b
//   13..16 w s_t (1, u, v, |u|^2), 17 w s_t^b                      tangential slopes of h and b
//   18..21 w u_n (u_n s_n + u_t s_t) (1, u, v, |u|^2), 22 the same for b
// A wall face takes 0..12 and 18..22 from the velocities moving into the wall only and 13..17 from all.
// Half-face slots per (cell, level): 0 x-face of the u > 0 class (the right face), 1 u < 0 (left face),
// 2 v > 0 (top face), 3 v < 0 (bottom face).
template <typename T, int TX, int TY, int G, int S>
__global__ void __launch_bounds__(TX * TY * 32, 1) k1_cells(Batch<T> B)
{
    constexpr int PX = TX + 2, PY = TY + 2, NR = PX * PY, NWC = TX * TY;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bars[S], empty[S];
    __shared__ T sacc[NWC][4][NM];
    __shared__ int abort_flag;                               // set by the first warp whose wait runs out
    const int cs = find_case(B.off, B.ncases, blockIdx.x);
    const CaseDev<T>& cd = B.cases[cs];
    if (!cd.st->active) return;
    // another CTA may set the error word while this one starts: decide for the whole CTA at once
    if (__syncthreads_or(*(volatile int*)cd.err != 0)) return;
    const int lb = blockIdx.x - B.off[cs];
    const int ntx = (cd.nx + TX - 1) / TX, nty = (cd.ny + TY - 1) / TY;
    const int tx = lb % ntx, ty = (lb / ntx) % nty, n = lb / (ntx * nty);
    const int i0 = tx * TX, j0 = ty * TY;
    const int nt = cd.nt, nc = cd.nc, nx = cd.nx, ny = cd.ny, nvb = cd.nvb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ti = warp % TX, tj = warp / TX, i = i0 + ti, j = j0 + tj;
    const bool valid = i < nx && j < ny;
    for (int k = lane; k < 4 * NM; k += 32) sacc[warp][k / NM][k % NM] = T(0);
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int k = 0; k < S; ++k) mbar_init(empty + k, NWC);   // one arrival per warp: slot read
    }
    mbar_setup(bars, S);
    // staged rectangle: columns i0-1 .. i0+TX, rows j0-1 .. j0+TY; S buffers [G][h, b][NR][32] in a ring
    constexpr size_t blk = (size_t)NR * VB;
    T* buf = reinterpret_cast<T*>(smem_raw);
    const int p = cd.st->parity;
    const T* gh = cd.dh[p];
    const T* gb = cd.db[p];
    const int c0 = max(i0 - 1, 0), c1 = min(i0 + TX + 1, nx);
    uint32_t rbytes = 0;
    for (int r = 0; r < PY; ++r) {
        const int jj = j0 - 1 + r;
        if (jj >= 0 && jj < ny) rbytes += (uint32_t)((c1 - c0) * VB * sizeof(T));
    }
    const int nchunk = (nvb + G - 1) / G;
    int* err = cd.err;
    auto issue = [&](int k) {
        const int vb0 = k * G, gk = min(G, nvb - vb0);
        T* dst = buf + (size_t)(k % S) * G * 2 * blk;
        if (lane == 0) mbar_arrive_expect(&bars[k % S], (uint32_t)(2 * gk) * rbytes);
        __syncwarp();
        for (int q = lane; q < gk * 2 * PY; q += 32) {
            const int r = q % PY, ga = q / PY;   // ga = 2 g + array
            const int jj = j0 - 1 + r;
            if (jj < 0 || jj >= ny) continue;
            const size_t src = ((size_t)(vb0 + (ga >> 1)) * nt + n) * nc * VB + ((size_t)jj * nx + c0) * VB;
            bulk_g2s(dst + (size_t)ga * blk + (size_t)(r * PX + c0 - (i0 - 1)) * VB, ((ga & 1) ? gb : gh) + src,
                     (uint32_t)((c1 - c0) * VB * sizeof(T)), &bars[k % S]);
        }
    };
    if (warp == 0)
        for (int k = 0; k < S - 1 && k < nchunk; ++k) issue(k);
    int issued = min(S - 1, nchunk);                         // chunks warp 0 has issued (kept on warp 0)
    // a wait ran out: warp 0, which issued the copies, waits (bounded) for every chunk from k on that it has not
    // seen complete, so that none still lands in shared memory after the CTA exits; the other warps just leave
    auto give_up = [&](int k) {
        if (warp == 0)
            for (int q = k; q < issued; ++q) mbar_drain(&bars[q % S], (uint32_t)((q / S) & 1));
    };

    // the warp's cell: neighbours, spacings, half widths (uniform over the warp)
    const bool hm = i > 0, hp = i < nx - 1, vm = j > 0, vp = j < ny - 1, sx = nx > 1, sy = ny > 1;
    const T wxm = valid && hm ? T(cd.rdx[i - 1]) : T(0), wxp = valid && hp ? T(cd.rdx[i]) : T(0);
    const T wym = valid && vm ? T(cd.rdy[j - 1]) : T(0), wyp = valid && vp ? T(cd.rdy[j]) : T(0);
    const T hxh = valid ? T(cd.hx[i]) : T(0), hyh = valid ? T(cd.hy[j]) : T(0);
    const int kc = (tj + 1) * PX + ti + 1;
    const T* __restrict__ tu = cd.tu;
    const T* __restrict__ tv = cd.tv;
    const T* __restrict__ tw = cd.tw;
    const int* __restrict__ vcls = cd.vcls;

    T ax[NM], ay[NM], ac[NCM];
#pragma unroll
    for (int q = 0; q < NM; ++q) { ax[q] = T(0); ay[q] = T(0); }
#pragma unroll
    for (int q = 0; q < NCM; ++q) ac[q] = T(0);
    int cur = -1;
    // add the sums of the current sign class to its two half-face slots
    auto flush = [&]() {
        const T tx_ = lane_totals<NM>(ax, lane);
        const T ty_ = lane_totals<NM>(ay, lane);
        if (lane < NM) {
            sacc[warp][(cur & 1) ? 1 : 0][lane] += tx_;
            sacc[warp][(cur & 2) ? 3 : 2][lane] += ty_;
        }
#pragma unroll
        for (int q = 0; q < NM; ++q) { ax[q] = T(0); ay[q] = T(0); }
    };

    // Ring of S slots: chunk k lands in slot k % S (mbarrier bars); each warp arrives on empty once it has
    // read the slot, and warp 0 refills a slot only after every warp has released it, so warps run up to
    // S - 1 chunks apart instead of meeting at a CTA barrier per chunk.
    for (int k = 0; k < nchunk; ++k) {
        if (warp == 0 && k + S - 1 < nchunk) {
            const int kk = k + S - 1;
            if (kk >= S && !mbar_wait(&empty[kk % S], (uint32_t)((kk / S - 1) & 1), err, &abort_flag)) {
                give_up(k);
                return;
            }
            issue(kk);
            issued = kk + 1;
        }
        if (!mbar_wait(&bars[k % S], (uint32_t)((k / S) & 1), err, &abort_flag)) {
            give_up(k);
            return;
        }
        const T* cb = buf + (size_t)(k % S) * G * 2 * blk;
        const int vb0 = k * G, gk = min(G, nvb - vb0);
        if (valid) {
            // the velocities of block g + 1 are loaded while block g is summed
            int ncls = __ldg(vcls + vb0);
            T nu_ = __ldg(tu + vb0 * VB + lane), nv_ = __ldg(tv + vb0 * VB + lane), nw_ = __ldg(tw + vb0 * VB + lane);
            for (int g = 0; g < gk; ++g) {
                const int cls = ncls;
                const T u = nu_, v = nv_, w = nw_;
                if (g + 1 < gk) {
                    const int a1 = (vb0 + g + 1) * VB + lane;
                    ncls = __ldg(vcls + vb0 + g + 1);
                    nu_ = __ldg(tu + a1); nv_ = __ldg(tv + a1); nw_ = __ldg(tw + a1);
                }
                if (cls != cur) {
                    if (cur >= 0) flush();
                    cur = cls;
                }
                const T* ph = cb + (size_t)(2 * g) * blk + (size_t)kc * VB + lane;
                const T* pb = ph + blk;
                const T f0 = ph[0], g0 = pb[0];
                const T sxh = slope(ph[-VB], f0, ph[VB], wxm, wxp, hm, hp, sx);
                const T syh = slope(ph[-PX * VB], f0, ph[PX * VB], wym, wyp, vm, vp, sy);
                const T sxb = slope(pb[-VB], g0, pb[VB], wxm, wxp, hm, hp, sx);
                const T syb = slope(pb[-PX * VB], g0, pb[PX * VB], wym, wyp, vm, vp, sy);
                const bool xn = (cls & 1) != 0, yn = (cls & 2) != 0;
                const T offx = xn ? -hxh : hxh, offy = yn ? -hyh : hyh;
                T d0x = f0 + sxh * offx, e0x = g0 + sxb * offx;
                T d0y = f0 + syh * offy, e0y = g0 + syb * offy;
                // a velocity parallel to a wall carries nothing into it
                if ((xn ? !hm : !hp) && u == T(0)) { d0x = T(0); e0x = T(0); }
                if ((yn ? !vm : !vp) && v == T(0)) { d0y = T(0); e0y = T(0); }
                const T wu = w * u, wv = w * v, wuu = wu * u, wuv = wu * v, wvv = wv * v;
                const T m[10] = {w, wu, wv, wuu, wuv, wvv, wuu * u, wuu * v, wvv * u, wvv * v};
                const T wq = wuu + wvv;
#pragma unroll
                for (int q = 0; q < 10; ++q) {
                    ax[q] += d0x * m[q];
                    ay[q] += d0y * m[q];
                    ac[q] += f0 * m[q];
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    ax[10 + q] += e0x * m[q];
                    ay[10 + q] += e0y * m[q];
                    ac[10 + q] += g0 * m[q];
                }
                ax[13] += syh * w; ax[14] += syh * wu; ax[15] += syh * wv; ax[16] += syh * wq; ax[17] += syb * w;
                ay[13] += sxh * w; ay[14] += sxh * wu; ay[15] += sxh * wv; ay[16] += sxh * wq; ay[17] += sxb * w;
                const T txh = u * (u * sxh + v * syh), tyh = v * (v * syh + u * sxh);
                ax[18] += txh * w; ax[19] += txh * wu; ax[20] += txh * wv; ax[21] += txh * wq;
                ay[18] += tyh * w; ay[19] += tyh * wu; ay[20] += tyh * wv; ay[21] += tyh * wq;
                ax[22] += u * (u * sxb + v * syb) * w;
                ay[22] += v * (v * syb + u * sxb) * w;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[k % S]);
    }
    if (!valid) return;
    if (cur >= 0) flush();
    const T cm = lane_totals<NCM>(ac, lane);
    __syncwarp();
    const int c = j * nx + i;
    if (lane < NCM) cd.cmom[((size_t)c * nt + n) * NCM + lane] = (double)cm;
    double* hmo = cd.hmom + ((size_t)c * nt + n) * 4 * NM;
    for (int k = lane; k < 4 * NM; k += 32) hmo[k] = (double)sacc[warp][k / NM][k % NM];
}

template <typename T, int TX, int TY, int G, int S>
constexpr size_t k1_cells_smem()
{
    return (size_t)S * G * 2 * (TX + 2) * (TY + 2) * VB * sizeof(T);
}

// ------------------------------------------------------------------------------ K4: micro update

// Micro flux (delta form, divided by dG_f) through the downwind face of the reconstructing cell, for one lane:
// u_n [C1' dH + H Q + C4' d0 + C5' (u_n s_n + u_t s_t)] and the b counterpart, from the face's parameters fp
// (shared memory; the cubic at qo and linear term at lo belong to the upwind side) and the expm1 factors
// (ex, ey) of the interface Maxwellian at the lane's velocity.
template <typename T>
__device__ __forceinline__ void flux_down(const T* fp, int qo, int lo, T ex, T ey, T href, T u, T v, T un, T ut, T d0,
                                          T e0, T sn, T st, T snb, T stb, T& Hf, T& Bf)
{
    const T* sc = fp + F_RM1;      // r - 1, r, 1/(2 lam), 1/(2 lam) - 1/(2 lam0), C1', C4', C5', nin
    const T E = ex + ey + ex * ey;
    const T dH = href * (sc[0] + sc[1] * E);
    const T H = href + dH;
    const T i2l = sc[2];
    const T dB = dH * i2l + href * sc[3];
    const T* l = fp + lo;
    const T Q = cubic(fp + qo, u, v);
    const T Qb = Q + l[0] + l[1] * u + l[2] * v;
    Hf = un * (sc[4] * dH + H * Q + sc[5] * d0 + sc[6] * (un * sn + ut * st));
    Bf = un * (sc[4] * dB + H * i2l * Qb + sc[5] * e0 + sc[6] * (un * snb + ut * stb));
    if (un == T(0)) { Hf = T(0); Bf = T(0); }
}

// Flux (delta form, divided by dG_f) of the distribution a diffuse wall re-emits, rho_w H_w u_n: velocities of
// the block leave the wall.
template <typename T>
__device__ __forceinline__ void flux_wall(const T* fp, const T* __restrict__ tb, int iu, int ivn, T href, T un, T& Hf,
                                          T& Bf)
{
    const T* wp = fp + F_WRM1;
    const T ex = __ldg(tb + iu), ey = __ldg(tb + ivn);
    const T E = ex + ey + ex * ey;
    const T dHw = href * (wp[0] + wp[1] * E);
    Hf = un * dHw;
    Bf = un * (dHw * wp[2] + href * wp[3]);
}

// Shared-memory layout of k4_cells (element offsets in T, each block 16-byte aligned):
//   own   [nt][h, b][NCT][32]      the tile's own cells on every level (spectral source, h^k of the update)
//   rect  [2][h, b][NR][32]        per level: the tile with its halo, (TX+3) x (TY+3) cells, two cells on the
//                                  upwind side of each axis and one on the downwind side (ring of 2 levels)
//   fp    [2][NFT][NP]             per level: parameters of the tile's faces (ring of 2 levels)
//   cp    [2][NCT][NCP]            per level: update coefficients of the tile's cells (ring of 2 levels)
//   flux  [2][h, b][NFT][32]       per level: micro fluxes of the tile's faces (double buffered)
template <typename T, int TX, int TY>
struct K4Layout {
    static constexpr int PX = TX + 3, PY = TY + 3, NR = PX * PY, NCT = TX * TY;
    static constexpr int NFX = TY * (TX + 1), NFY = (TY + 1) * TX, NFT = NFX + NFY;
    static constexpr size_t RECT = (size_t)2 * NR * VB;                 // one ring slot, h and b
    static constexpr size_t FP = (size_t)NFT * NP, CP = (size_t)NCT * NCP, FLUX = (size_t)2 * NFT * VB;
    __host__ __device__ static constexpr size_t own_elems(int nt) { return (size_t)nt * 2 * NCT * VB; }
    __host__ __device__ static constexpr size_t rect_off(int nt) { return own_elems(nt); }
    __host__ __device__ static constexpr size_t fp_off(int nt) { return rect_off(nt) + 2 * RECT; }
    __host__ __device__ static constexpr size_t cp_off(int nt) { return fp_off(nt) + 2 * FP; }
    __host__ __device__ static constexpr size_t flux_off(int nt) { return cp_off(nt) + 2 * CP; }
    __host__ __device__ static constexpr size_t bytes(int nt) { return (flux_off(nt) + 2 * FLUX) * sizeof(T); }
};

// A CTA: a TX x TY tile of cells, one velocity block, all levels.  Per level, the first pass reconstructs
// every tile cell and the upwind halo cells and evaluates the flux through each one's downwind face (every
// face of the tile exactly once); the second pass applies Eq. fv_h to the tile cells.  The second pass of
// level n runs together with the first pass of level n + 1 (fluxes double buffered), so one barrier separates
// the levels.  With IMP and a case that asks for it, the spectral source is taken at the new iterate: pass 2
// leaves each level's right-hand side in the own-cell store and a last pass applies the per-cell inverse
// across levels.  Batch k of bulk copies (the halo rectangle and face parameters of level k, the cell
// coefficients of level k - 1; batch 0 also every level of the tile's own cells) completes on mbarrier k & 1
// and is issued one level ahead of its use.
template <typename T, int TX, int TY, int NW, bool IMP>
__global__ void __launch_bounds__(NW * 32) k4_cells(Batch<T> B)
{
    using L = K4Layout<T, TX, TY>;
    constexpr int PX = L::PX, PY = L::PY, NR = L::NR, NCT = L::NCT, NFX = L::NFX, NFT = L::NFT;
    constexpr int NIT = NCT + TY + TX, NPASS = (NIT + NW - 1) / NW;
    constexpr int lv = NR * VB;                               // one array of one rectangle slot
    constexpr int SROWS = 4;                                  // tile rows per strip of the CTA order
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bars[2];
    __shared__ T gxr[PX], gxh[PX], gyr[PY], gyh[PY];
    const int cs = find_case(B.off, B.ncases, blockIdx.x);
    const CaseDev<T>& cd = B.cases[cs];
    if (!cd.st->active) return;
    // another CTA may set the error word while this one starts: decide for the whole CTA at once
    if (__syncthreads_or(*(volatile int*)cd.err != 0)) return;
    const bool expire = *(volatile const int*)cd.expire != 0;
    const int nvb = cd.nvb, nx = cd.nx, ny = cd.ny;
    // CTA order: velocity block fastest (the CTAs of one tile share its parameters in L2), then tiles in
    // strips of SROWS tile rows, column by column (neighbour tiles, whose halos overlap, run close in time)
    const int lb = blockIdx.x - B.off[cs];
    const int vb = lb % nvb, tile = lb / nvb;
    const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY;
    const int strip = tile / (ntx * SROWS), rows = min(SROWS, nty - strip * SROWS);
    const int rem = tile - strip * ntx * SROWS;
    const int i0 = (rem / rows) * TX, j0 = (strip * SROWS + rem % rows) * TY;
    const int nt = cd.nt, nc = cd.nc, nh = cd.nh, nfx = cd.nfx, nf = cd.nf;
    const int nuv = cd.nu + cd.nv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cls = __ldg(cd.vcls + vb);
    const bool xneg = (cls & 1) != 0, yneg = (cls & 2) != 0;
    const int xlo = xneg ? -1 : -2, ylo = yneg ? -1 : -2;
    const int iend = min(i0 + TX, nx), jend = min(j0 + TY, ny);
    T* const sm = reinterpret_cast<T*>(smem_raw);
    T* const own = sm;
    T* const rect = sm + L::rect_off(nt);
    T* const fps = sm + L::fp_off(nt);
    T* const cps = sm + L::cp_off(nt);
    T* const fbuf = sm + L::flux_off(nt);
    mbar_setup(bars, 2);
    const int p = cd.st->parity;
    const T* gh = cd.dh[p];
    const T* gb = cd.db[p];
    // bulk copies of the rectangle rows (clipped to the domain)
    const int c0 = max(i0 + xlo, 0), c1 = min(i0 + xlo + PX, nx);
    const int nfr = iend - i0;                                // valid cells per tile row
    const uint32_t row_b = (uint32_t)((c1 - c0) * VB * sizeof(T));
    int rrows = 0;
    for (int r = 0; r < PY; ++r) {
        const int jj = j0 + ylo + r;
        rrows += (jj >= 0 && jj < ny) ? 1 : 0;
    }
    const uint32_t rect_b = 2u * rrows * row_b;
    const uint32_t fp_b = (uint32_t)(((jend - j0) * (nfr + 1) + (jend - j0 + 1) * nfr) * NP * sizeof(T));
    const uint32_t cp_b = (uint32_t)((jend - j0) * nfr * NCP * sizeof(T));
    // batch k: rectangle and face parameters of level k (k < nt), cell coefficients of level k - 1 (k >= 1)
    auto issue = [&](int k) {
        const bool lvl = k < nt, cel = k >= 1;
        uint32_t bytes = (lvl ? rect_b + fp_b : 0u) + (cel ? cp_b : 0u);
        if (k == 0) bytes += (uint32_t)(2 * nt * (jend - j0) * nfr * VB * sizeof(T));
        uint64_t* bar = &bars[k & 1];
        if (lane == 0) mbar_arrive_expect(bar, bytes);
        __syncwarp();
        const int nrect = lvl ? 2 * PY : 0, nfpr = lvl ? 2 * TY + 1 : 0, ncpr = cel ? TY : 0;
        const int nown = k == 0 ? 2 * nt * TY : 0;
        for (int q = lane; q < nrect + nfpr + ncpr + nown; q += 32) {
            if (q < nrect) {
                const int r = q % PY, a = q / PY;
                const int jj = j0 + ylo + r;
                if (jj < 0 || jj >= ny) continue;
                const size_t src = ((size_t)vb * nt + k) * nc * VB + ((size_t)jj * nx + c0) * VB;
                bulk_g2s(rect + (size_t)(k & 1) * L::RECT + (size_t)a * lv + (r * PX + c0 - (i0 + xlo)) * VB,
                         (a ? gb : gh) + src, row_b, bar);
            } else if (q < nrect + nfpr) {
                const int r = q - nrect;
                if (r < TY) {                                 // x-faces of tile row r
                    const int jj = j0 + r;
                    if (jj >= ny) continue;
                    bulk_g2s(fps + (size_t)(k & 1) * L::FP + (size_t)r * (TX + 1) * NP,
                             cd.fpar + ((size_t)k * nf + jj * (nx + 1) + i0) * NP,
                             (uint32_t)((nfr + 1) * NP * sizeof(T)), bar);
                } else {                                      // y-faces of face row r - TY
                    const int fr = r - TY, jj = j0 + fr;
                    if (jj > jend) continue;
                    bulk_g2s(fps + (size_t)(k & 1) * L::FP + (size_t)(NFX + fr * TX) * NP,
                             cd.fpar + ((size_t)k * nf + nfx + jj * nx + i0) * NP, (uint32_t)(nfr * NP * sizeof(T)),
                             bar);
                }
            } else if (q < nrect + nfpr + ncpr) {
                const int r = q - nrect - nfpr, jj = j0 + r;  // cells of tile row r, level k - 1
                if (jj >= ny) continue;
                bulk_g2s(cps + (size_t)((k - 1) & 1) * L::CP + (size_t)r * TX * NCP,
                         cd.cpar + ((size_t)(k - 1) * nc + jj * nx + i0) * NCP, (uint32_t)(nfr * NCP * sizeof(T)), bar);
            } else {
                const int o = q - nrect - nfpr - ncpr;        // own cells: row, array, level
                const int r = o % TY, a = (o / TY) & 1, n = o / (2 * TY), jj = j0 + r;
                if (jj >= ny) continue;
                bulk_g2s(own + ((size_t)(n * 2 + a) * NCT + r * TX) * VB,
                         (a ? gb : gh) + ((size_t)vb * nt + n) * nc * VB + ((size_t)jj * nx + i0) * VB,
                         (uint32_t)(nfr * VB * sizeof(T)), bar);
            }
        }
    };
    if (warp == 0) issue(0);
    for (int k = threadIdx.x; k < PX; k += blockDim.x) {
        const int ii = i0 + xlo + k;
        gxr[k] = (ii >= 0 && ii < nx - 1) ? T(cd.rdx[ii]) : T(0);
        gxh[k] = (ii >= 0 && ii < nx) ? T(cd.hx[ii]) : T(0);
    }
    for (int k = threadIdx.x; k < PY; k += blockDim.x) {
        const int jj = j0 + ylo + k;
        gyr[k] = (jj >= 0 && jj < ny - 1) ? T(cd.rdy[jj]) : T(0);
        gyh[k] = (jj >= 0 && jj < ny) ? T(cd.hy[jj]) : T(0);
    }
    const int av = vb * VB + lane;
    const T u = __ldg(cd.tu + av), v = __ldg(cd.tv + av), href = __ldg(cd.thref + av);
    const int iu = __ldg(cd.viu + av), ivn = cd.nu + __ldg(cd.viv + av);
    T et[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) et[d] = cd.et[d];
    const T* __restrict__ ftab = cd.ftab;
    const T* __restrict__ wtab = cd.wtab;
    const T* __restrict__ ctab = cd.ctab;
    const bool shakhov = cd.shakhov != 0;
    const int NTf = nt * nuv;                                 // per-face stride of the expm1 tables
    const int qoff = xneg ? F_QR : F_QL, loff = xneg ? F_LBR : F_LBL;
    const int qoffy = yneg ? F_QR : F_QL, loffy = yneg ? F_LBR : F_LBL;
    int* err = cd.err;

    const bool implicit = IMP && cd.spectral_implicit != 0;   // IMP = false compiles the explicit form alone
    // a tile none of whose cells touches a wall: every stencil neighbour exists
    const bool interior = i0 >= 1 && j0 >= 1 && i0 + TX <= nx - 1 && j0 + TY <= ny - 1;
    constexpr bool PAIRED = NCT == 2 * NW;                    // each warp owns two tile cells in pass 1

    for (int s = 0; s <= nt; ++s) {
        if (warp == 0 && s < nt) issue(s + 1);
        // the test hook reports the first wait as expired only after it has completed
        const int fail = !mbar_wait(&bars[s & 1], (uint32_t)((s >> 1) & 1), err) || expire;
        if (__syncthreads_or(fail)) {
            // every thread agrees; warp 0, which issued them, waits (bounded) for batches s and s + 1, so that
            // no bulk copy still lands in shared memory after the CTA exits
            if (threadIdx.x == 0 && expire) atomicExch(err, 1);
            if (warp == 0) {
                mbar_drain(&bars[s & 1], (uint32_t)((s >> 1) & 1));
                if (s < nt) mbar_drain(&bars[(s + 1) & 1], (uint32_t)(((s + 1) >> 1) & 1));
            }
            return;
        }
        if (s < nt) {
            // ---- pass 1, level s: reconstruction and downwind-face fluxes
            const int n = s;
            T* Fh = fbuf + (size_t)(n & 1) * L::FLUX + lane;
            T* Fb = Fh + NFT * VB;
            const T* rh = rect + (size_t)(n & 1) * L::RECT + lane;
            const T* fpn = fps + (size_t)(n & 1) * L::FP;
            const T* ftn = ftab + n * nuv;
            int rfirst = 0;
            if (PAIRED && interior) {
                // both tile cells of the warp as one straight-line block, stores last, so that the two
                // independent chains interleave
                T fx[2][4];
                int sl[2][2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int it = warp + q * NW, ti = it % TX, tj = it / TX;
                    const int i = i0 + ti, j = j0 + tj;
                    const int kx = ti - xlo, ky = tj - ylo;
                    const int fix = xneg ? i : i + 1, fjy = yneg ? j : j + 1;
                    sl[q][0] = tj * (TX + 1) + fix - i0;
                    sl[q][1] = NFX + (fjy - j0) * TX + ti;
                    const T* tbx = ftn + (j * (nx + 1) + fix) * NTf;
                    const T* tby = ftn + (nfx + fjy * nx + i) * NTf;
                    const T exx = __ldg(tbx + iu), eyx = __ldg(tbx + ivn);
                    const T exy = __ldg(tby + iu), eyy = __ldg(tby + ivn);
                    const T* ph = rh + (ky * PX + kx) * VB;
                    const T* pb = ph + lv;
                    const T f0 = ph[0], g0 = pb[0];
                    const T wxm = gxr[kx - 1], wxp = gxr[kx], wym = gyr[ky - 1], wyp = gyr[ky];
                    const T sxh = slope(ph[-VB], f0, ph[VB], wxm, wxp, true, true, true);
                    const T sxb = slope(pb[-VB], g0, pb[VB], wxm, wxp, true, true, true);
                    const T syh = slope(ph[-PX * VB], f0, ph[PX * VB], wym, wyp, true, true, true);
                    const T syb = slope(pb[-PX * VB], g0, pb[PX * VB], wym, wyp, true, true, true);
                    const T offx = xneg ? -gxh[kx] : gxh[kx], offy = yneg ? -gyh[ky] : gyh[ky];
                    flux_down(fpn + sl[q][0] * NP, qoff, loff, exx, eyx, href, u, v, u, v, f0 + sxh * offx,
                              g0 + sxb * offx, sxh, syh, sxb, syb, fx[q][0], fx[q][1]);
                    flux_down(fpn + sl[q][1] * NP, qoffy, loffy, exy, eyy, href, u, v, v, u, f0 + syh * offy,
                              g0 + syb * offy, syh, sxh, syb, sxb, fx[q][2], fx[q][3]);
                }
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    Fh[sl[q][0] * VB] = fx[q][0];
                    Fb[sl[q][0] * VB] = fx[q][1];
                    Fh[sl[q][1] * VB] = fx[q][2];
                    Fb[sl[q][1] * VB] = fx[q][3];
                }
                rfirst = 2;
            }
#pragma unroll
            for (int r = 0; r < NPASS; ++r) {
                if (r < rfirst) continue;
                const int it = warp + r * NW;
                if (it >= NIT) break;
                int ti, tj;
                bool dox = true, doy = true;
                if ((r + 1) * NW <= NCT || it < NCT) {
                    ti = it % TX; tj = it / TX;
                    if (i0 + ti >= nx || j0 + tj >= ny) continue;
                } else if (it < NCT + TY) {
                    tj = it - NCT; ti = xneg ? iend - i0 : -1; doy = false;
                    if (j0 + tj >= ny) continue;
                } else {
                    ti = it - NCT - TY; tj = yneg ? jend - j0 : -1; dox = false;
                    if (i0 + ti >= nx) continue;
                }
                const int i = i0 + ti, j = j0 + tj;
                if (i < 0 || i >= nx || j < 0 || j >= ny) {
                    // upwind face of the tile on a wall: the re-emitted distribution
                    T Hf, Bf;
                    int slot;
                    if (dox) {
                        const int fi = i < 0 ? 0 : nx;
                        slot = tj * (TX + 1) + fi - i0;
                        flux_wall(fpn + slot * NP, wtab + ((i < 0 ? 3 : 1) * cd.nslot + wall_slot(cd, n)) * nuv, iu,
                                  ivn, href, u, Hf, Bf);
                    } else {
                        const int fj = j < 0 ? 0 : ny;
                        slot = NFX + (fj - j0) * TX + ti;
                        flux_wall(fpn + slot * NP, wtab + ((j < 0 ? 0 : 2) * cd.nslot + wall_slot(cd, n)) * nuv, iu,
                                  ivn, href, v, Hf, Bf);
                    }
                    Fh[slot * VB] = Hf;
                    Fb[slot * VB] = Bf;
                    continue;
                }
                const int kx = ti - xlo, ky = tj - ylo;
                const int fix = xneg ? i : i + 1, fjy = yneg ? j : j + 1;
                const int slx = tj * (TX + 1) + fix - i0, sly = NFX + (fjy - j0) * TX + ti;
                // expm1 factors of the interface Maxwellians first: their latency overlaps the reconstruction
                const T* tbx = ftn + (j * (nx + 1) + fix) * NTf;
                const T* tby = ftn + (nfx + fjy * nx + i) * NTf;
                T exx = T(0), eyx = T(0), exy = T(0), eyy = T(0);
                if (dox) { exx = __ldg(tbx + iu); eyx = __ldg(tbx + ivn); }
                if (doy) { exy = __ldg(tby + iu); eyy = __ldg(tby + ivn); }
                const T* ph = rh + (ky * PX + kx) * VB;
                const T* pb = ph + lv;
                const T f0 = ph[0], g0 = pb[0];
                const bool hm = i > 0, hp = i < nx - 1, vm = j > 0, vp = j < ny - 1;
                const T wxm = gxr[kx - 1], wxp = gxr[kx], wym = gyr[ky - 1], wyp = gyr[ky];
                const T sxh = slope(ph[-VB], f0, ph[VB], wxm, wxp, hm, hp, nx > 1);
                const T sxb = slope(pb[-VB], g0, pb[VB], wxm, wxp, hm, hp, nx > 1);
                const T syh = slope(ph[-PX * VB], f0, ph[PX * VB], wym, wyp, vm, vp, ny > 1);
                const T syb = slope(pb[-PX * VB], g0, pb[PX * VB], wym, wyp, vm, vp, ny > 1);
                if (dox) {
                    const T off = xneg ? -gxh[kx] : gxh[kx];
                    T Hf, Bf;
                    flux_down(fpn + slx * NP, qoff, loff, exx, eyx, href, u, v, u, v, f0 + sxh * off, g0 + sxb * off,
                              sxh, syh, sxb, syb, Hf, Bf);
                    Fh[slx * VB] = Hf;
                    Fb[slx * VB] = Bf;
                }
                if (doy) {
                    const T off = yneg ? -gyh[ky] : gyh[ky];
                    T Hf, Bf;
                    flux_down(fpn + sly * NP, qoffy, loffy, exy, eyy, href, u, v, v, u, f0 + syh * off, g0 + syb * off,
                              syh, sxh, syb, sxb, Hf, Bf);
                    Fh[sly * VB] = Hf;
                    Fb[sly * VB] = Bf;
                }
            }
        }
        if (s > 0) {
            // ---- pass 2, level s - 1: Eq. fv_h with the spectral source (delta form)
            const int n = s - 1;
            const T* Fh = fbuf + (size_t)(n & 1) * L::FLUX + lane;
            const T* Fb = Fh + NFT * VB;
            T* on = cd.dh[p ^ 1] + ((size_t)vb * nt + n) * nc * VB + lane;
            T* onb = cd.db[p ^ 1] + ((size_t)vb * nt + n) * nc * VB + lane;
            const T* cpn = cps + (size_t)(n & 1) * L::CP;
            const T* ctn = ctab + n * 2 * nuv;
            constexpr int lvo = 2 * NCT * VB;                 // level stride of the own-cell store
#pragma unroll
            for (int r = 0; r < (NCT + NW - 1) / NW; ++r) {
                const int ct = warp + r * NW;
                if (ct >= NCT) break;
                const int ti = ct % TX, tj = ct / TX;
                const int i = i0 + ti, j = j0 + tj;
                if (i >= nx || j >= ny) continue;
                const int c = j * nx + i;
                const T* tb = ctn + c * nt * 2 * nuv;
                const T ex0 = __ldg(tb + iu), ey0 = __ldg(tb + ivn);
                const T ex1 = __ldg(tb + nuv + iu), ey1 = __ldg(tb + nuv + ivn);
                const int fL = tj * (TX + 1) + ti, fB = NFX + tj * TX + ti;
                const T dxh = Fh[(fL + 1) * VB] - Fh[fL * VB];
                const T dyh = Fh[(fB + TX) * VB] - Fh[fB * VB];
                const T dxb = Fb[(fL + 1) * VB] - Fb[fL * VB];
                const T dyb = Fb[(fB + TX) * VB] - Fb[fB * VB];
                T* hc = own + ct * VB + lane;                // level m, array a at hc[m * lvo + a * NCT * VB]
                T* bc = hc + NCT * VB;
                T eh, eb;
                switch (implicit ? 0 : nh) {
                    case 0: eh = T(0); eb = T(0); break;
                    case 1: spectral<1>(hc, bc, n, nt, lvo, et, eh, eb); break;
                    case 2: spectral<2>(hc, bc, n, nt, lvo, et, eh, eb); break;
                    case 3: spectral<3>(hc, bc, n, nt, lvo, et, eh, eb); break;
                    case 4: spectral<4>(hc, bc, n, nt, lvo, et, eh, eb); break;
                    case 5: spectral<5>(hc, bc, n, nt, lvo, et, eh, eb); break;
                    case 6: spectral<6>(hc, bc, n, nt, lvo, et, eh, eb); break;
                    default: spectral<7>(hc, bc, n, nt, lvo, et, eh, eb); break;
                }
                // equilibria of W^{k+1} (slot 1) and W^k (slot 0): dH = H - H_ref from the cell table, Shakhov cubic
                const T* cp = cpn + ct * NCP;
                T dhp[2], dbp[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const T* q = cp + (e == 0 ? C_EQ0 : C_EQ1);
                    const T ex = e == 0 ? ex0 : ex1, ey = e == 0 ? ey0 : ey1;
                    const T E = ex + ey + ex * ey;
                    const T dH = href * (q[E_RM1] + q[E_R] * E);
                    const T dB = dH * q[E_I2L] + href * q[E_DI2L];
                    if (shakhov) {
                        const T H = href + dH;
                        const T sk = cubic(q + E_SH, u, v);
                        const T skb = sk + q[E_SHB] + q[E_SHB + 1] * u + q[E_SHB + 2] * v;
                        dhp[e] = dH + H * sk;
                        dbp[e] = dB + H * q[E_I2L] * skb;
                    } else {
                        dhp[e] = dH;
                        dbp[e] = dB;
                    }
                }
                const T* k = cp + C_KSELF;                    // kself, kE, kp1, kp0, kdx, kdy
                const T h0 = hc[n * lvo], b0 = bc[n * lvo];
                const T xh = k[0] * h0 - k[4] * dxh - k[5] * dyh - k[1] * eh + k[2] * dhp[1] + k[3] * dhp[0];
                const T xb = k[0] * b0 - k[4] * dxb - k[5] * dyb - k[1] * eb + k[2] * dbp[1] + k[3] * dbp[0];
                if (implicit) {
                    // right-hand side of level n; h^k of this level is no longer needed
                    hc[n * lvo] = xh;
                    bc[n * lvo] = xb;
                } else {
                    on[c * VB] = xh;
                    onb[c * VB] = xb;
                }
            }
        }
        __syncthreads();
    }
    if (implicit) {
        // spectral source at the new iterate: h^{k+1} = minv (right-hand sides over the levels), per cell and lane
        constexpr int lvo = 2 * NCT * VB;
        for (int ct = warp; ct < NCT; ct += NW) {
            const int ti = ct % TX, tj = ct / TX;
            const int i = i0 + ti, j = j0 + tj;
            if (i >= nx || j >= ny) continue;
            const int c = j * nx + i;
            const T* hc = own + ct * VB + lane;
            const T* bc = hc + NCT * VB;
            T rh[MAXNT], rb[MAXNT];
#pragma unroll
            for (int m = 0; m < MAXNT; ++m) {
                rh[m] = m < nt ? hc[m * lvo] : T(0);
                rb[m] = m < nt ? bc[m * lvo] : T(0);
            }
            const T* Mi = cd.minv + (size_t)c * nt * nt;
            T* oh = cd.dh[p ^ 1] + (size_t)vb * nt * nc * VB + (size_t)c * VB + lane;
            T* ob = cd.db[p ^ 1] + (size_t)vb * nt * nc * VB + (size_t)c * VB + lane;
#pragma unroll
            for (int n = 0; n < MAXNT; ++n) {
                if (n >= nt) break;
                T sh = T(0), sb = T(0);
#pragma unroll
                for (int m = 0; m < MAXNT; ++m)
                    if (m < nt) {
                        const T w = __ldg(Mi + n * nt + m);
                        sh += w * rh[m];
                        sb += w * rb[m];
                    }
                oh[(size_t)n * nc * VB] = sh;
                ob[(size_t)n * nc * VB] = sb;
            }
        }
    }
}

template <typename T, int TX, int TY>
constexpr size_t k4_cells_smem(int nt)
{
    return K4Layout<T, TX, TY>::bytes(nt);
}

}  // namespace hb
