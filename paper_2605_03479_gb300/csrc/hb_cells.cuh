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
// owns a tile of cells and one or two velocity blocks of one sign class and runs over all levels.  Both stage
// the tile and its halo in shared memory with bulk copies (TMA) completing on an mbarrier.  The distributions
// h and b of a velocity are stored side by side and carried as one pair (hb_common.cuh): one 8-byte access
// and, in single precision, one packed FP32x2 instruction for both wherever they see the same arithmetic
// (differences, limited slopes, reconstruction, the flux combination, velocity sums with a common weight,
// spectral source and update).
#pragma once
#include "hb_common.cuh"

namespace hb {

// van Leer limiter of a pair: 2 s1 s2 / (s1 + s2) where s1 s2 > 0, else 0.  Single precision: the limited slope
// needs no correctly rounded division (approximate reciprocal, 2 ulp)
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float2 vleer2(float2 s1, float2 s2)
{
    const float2 p = pmul(s1, s2);
    const float2 den = padd(s1, s2);
    const float2 q = pmul(padd(p, p), make_float2(rcp_approx(den.x), rcp_approx(den.y)));
    return make_float2(p.x > 0.f ? q.x : 0.f, p.y > 0.f ? q.y : 0.f);
}
__device__ __forceinline__ double2 vleer2(double2 s1, double2 s2)
{
    const double px = s1.x * s2.x, py = s1.y * s2.y;
    return make_double2(px > 0.0 ? (px + px) / (s1.x + s2.x) : 0.0, py > 0.0 ? (py + py) / (s1.y + s2.y) : 0.0);
}

// Limited slope of (h, b) of a cell from its two neighbours along one axis, wm = 1/(x_i - x_{i-1}),
// wp = 1/(x_{i+1} - x_i) (non-uniform spacing); a missing neighbour (wall) makes the available one-sided
// difference the slope, a single cell along the axis has none
template <typename V, typename T>
__device__ __forceinline__ V slope2(V fm, V f0, V fp, T wm, T wp, bool has_m, bool has_p, bool several)
{
    V s1 = pmul(psub(f0, fm), bc(wm)), s2 = pmul(psub(fp, f0), bc(wp));
    if (!has_m) s1 = s2;
    if (!has_p) s2 = s1;
    return several ? vleer2(s1, s2) : bc(T(0));
}
// both neighbours present
template <typename V, typename T>
__device__ __forceinline__ V slope2i(V fm, V f0, V fp, T wm, T wp)
{
    return vleer2(pmul(psub(f0, fm), bc(wm)), pmul(psub(fp, f0), bc(wp)));
}

// spectral source of one cell and lane: sum_d e_d (f_{n-d} - f_{n+d}) for (h, b) (Eq. D_explicit in paired
// form), levels lv pairs apart in shared memory, e_d as broadcast pairs (etb[0] = 0)
template <int NH, typename V>
__device__ __forceinline__ V spectral2(const V* fc, int n, int nt, int lv, const V* etb)
{
    V e = etb[0];
#pragma unroll
    for (int d = 1; d <= NH; ++d) {
        int nm = n - d; nm += nm < 0 ? nt : 0;
        int np = n + d; np -= np >= nt ? nt : 0;
        e = pfma(etb[d], psub(fc[nm * lv], fc[np * lv]), e);
    }
    return e;
}

// spectral source of every level of one cell and lane, in place: the pair of level n (levels lv pairs apart)
// becomes sum_d e_d (f_{n-d} - f_{n+d}), with the operations of spectral2 in the same order
template <int NH, typename V, typename T>
__device__ __forceinline__ void spectral_all(V* fc, int lv, const T* et)
{
    constexpr int NT = 2 * NH + 1;
    V f[NT], eb[NH + 1];
#pragma unroll
    for (int m = 0; m < NT; ++m) f[m] = fc[m * lv];
#pragma unroll
    for (int d = 0; d <= NH; ++d) eb[d] = bc(et[d]);
#pragma unroll
    for (int n = 0; n < NT; ++n) {
        V e = eb[0];
#pragma unroll
        for (int d = 1; d <= NH; ++d) e = pfma(eb[d], psub(f[(n - d + NT) % NT], f[(n + d) % NT]), e);
        fc[n * lv] = e;
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
// With SEP the case's velocity grid has no zero node and each sign class has 1, 2, 4, 8, 16 or 32 u-nodes, so a
// lane sees the same u in every block of a class (blocks hold whole rows of the class, u fastest): every sum
// w u^a v^b d factors into w_u u^a (the lane's) times sum over the lane's velocities of w_v v^b d, and the lane
// keeps only those v-moments (34 sums instead of 59), multiplying by w_u u^a when the class changes.
template <typename T, int TX, int TY, int G, int S, bool SEP>
__global__ void __launch_bounds__(TX * TY * 32, (sizeof(T) == 4 && TX * TY == 8) ? 2 : 1) k1_cells(Batch<T> B)
{
    using V = P2<T>;
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
    // staged rectangle: columns i0-1 .. i0+TX, rows j0-1 .. j0+TY; S buffers [G][NR][32] of (h, b) pairs
    constexpr size_t blk = (size_t)NR * VB;
    V* buf = reinterpret_cast<V*>(smem_raw);
    const int p = cd.st->parity;
    const V* gf = cd.f[p];
    const int c0 = max(i0 - 1, 0), c1 = min(i0 + TX + 1, nx);
    const uint32_t row_b = (uint32_t)((c1 - c0) * VB * sizeof(V));
    uint32_t rbytes = 0;
    for (int r = 0; r < PY; ++r) {
        const int jj = j0 - 1 + r;
        if (jj >= 0 && jj < ny) rbytes += row_b;
    }
    const int nchunk = (nvb + G - 1) / G;
    int* err = cd.err;
    auto issue = [&](int k) {
        const int vb0 = k * G, gk = min(G, nvb - vb0);
        V* dst = buf + (size_t)(k % S) * G * blk;
        if (lane == 0) mbar_arrive_expect(&bars[k % S], (uint32_t)gk * rbytes);
        __syncwarp();
        for (int q = lane; q < gk * PY; q += 32) {
            const int r = q % PY, g = q / PY;
            const int jj = j0 - 1 + r;
            if (jj < 0 || jj >= ny) continue;
            const size_t src = ((size_t)(vb0 + g) * nt + n) * nc * VB + ((size_t)jj * nx + c0) * VB;
            bulk_g2s(dst + (size_t)g * blk + (size_t)(r * PX + c0 - (i0 - 1)) * VB, gf + src, row_b, &bars[k % S]);
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
    const bool inner = hm && hp && vm && vp;                 // every neighbour present: no wall branches
    const int kc = (tj + 1) * PX + ti + 1;
    const T* __restrict__ tu = cd.tu;
    const T* __restrict__ tv = cd.tv;
    const T* __restrict__ tw = SEP ? cd.twv : cd.tw;       // SEP: the v-factor w_v of each weight

    // general: the 23 + 23 + 13 sums per lane; SEP: v-moments per lane (x-face h: 4, b: 2, tangential h: 3,
    // b: 1, normal-flux h: 3, b: 1; the y-face alike; cell h: 4, b: 2), folded into the 23 + 23 + 13 at a
    // class change.  A sum of h and the sum of b with the same weight are kept as one pair (one packed FMA):
    //   SEP      xp: (0, 4) (1, 5) (6, 9) (10, 13) of the 14 v-moments, xs: 2 3 7 8 11 12;  cp: (0, 4) (1, 5),
    //            csm: 2 3 of the 6 cell v-moments
    //   general  xp: (0, 10) (1, 11) (2, 12) (13, 17) (18, 22) of the 23 sums, xs: 3..9, 14..16, 19..21;
    //            cp: (0, 10) (1, 11) (2, 12), csm: 3..9 of the 13 cell sums
    constexpr int NXP = SEP ? 4 : 5, NXS = SEP ? 6 : 13, NCP2 = SEP ? 2 : 3, NCS = SEP ? 2 : 7;
    V xp[NXP], yp[NXP], cp2[NCP2];
    T xs[NXS], ys[NXS], csm[NCS], ac[NCM];
    auto zero_faces = [&]() {
#pragma unroll
        for (int q = 0; q < NXP; ++q) { xp[q] = bc(T(0)); yp[q] = bc(T(0)); }
#pragma unroll
        for (int q = 0; q < NXS; ++q) { xs[q] = T(0); ys[q] = T(0); }
    };
    auto zero_cell = [&]() {
#pragma unroll
        for (int q = 0; q < NCP2; ++q) cp2[q] = bc(T(0));
#pragma unroll
        for (int q = 0; q < NCS; ++q) csm[q] = T(0);
    };
    zero_faces();
    zero_cell();
#pragma unroll
    for (int q = 0; q < NCM; ++q) ac[q] = T(0);
    int cur = -1, cend = 0;                                  // current sign class, the first block past it
    T ul = T(0), wul = T(0);                                 // SEP: the lane's u and w_u in the current class
    // the 14 v-moments of a face (SEP) or its 23 sums (general) in slot order
    auto face_sums = [&](const V (&P)[NXP], const T (&S_)[NXS], T (&m)[SEP ? 14 : NM]) {
        if constexpr (SEP) {
            m[0] = P[0].x; m[1] = P[1].x; m[2] = S_[0]; m[3] = S_[1]; m[4] = P[0].y; m[5] = P[1].y;
            m[6] = P[2].x; m[7] = S_[2]; m[8] = S_[3]; m[9] = P[2].y; m[10] = P[3].x; m[11] = S_[4];
            m[12] = S_[5]; m[13] = P[3].y;
        } else {
            m[0] = P[0].x; m[1] = P[1].x; m[2] = P[2].x;
#pragma unroll
            for (int q = 0; q < 7; ++q) m[3 + q] = S_[q];
            m[10] = P[0].y; m[11] = P[1].y; m[12] = P[2].y; m[13] = P[3].x;
            m[14] = S_[7]; m[15] = S_[8]; m[16] = S_[9]; m[17] = P[3].y; m[18] = P[4].x;
            m[19] = S_[10]; m[20] = S_[11]; m[21] = S_[12]; m[22] = P[4].y;
        }
    };
    // the 23 face sums of one face from its v-moments m (SEP)
    auto unfold = [&](const T (&m)[14], T (&o)[NM]) {
        const T w1 = wul, w2 = w1 * ul, w3 = w2 * ul, w4 = w3 * ul;     // w_u u^a
        o[0] = w1 * m[0]; o[1] = w2 * m[0]; o[2] = w1 * m[1]; o[3] = w3 * m[0]; o[4] = w2 * m[1];
        o[5] = w1 * m[2]; o[6] = w4 * m[0]; o[7] = w3 * m[1]; o[8] = w2 * m[2]; o[9] = w1 * m[3];
        o[10] = w1 * m[4]; o[11] = w2 * m[4]; o[12] = w1 * m[5];
        o[13] = w1 * m[6]; o[14] = w2 * m[6]; o[15] = w1 * m[7]; o[16] = w3 * m[6] + w1 * m[8];
        o[17] = w1 * m[9];
        o[18] = w1 * m[10]; o[19] = w2 * m[10]; o[20] = w1 * m[11]; o[21] = w3 * m[10] + w1 * m[12];
        o[22] = w1 * m[13];
    };
    // add the sums of the current sign class to its two half-face slots
    auto flush = [&]() {
        T tx_, ty_;
        if constexpr (SEP) {
            T mx[14], my[14], ox[NM], oy[NM];
            face_sums(xp, xs, mx);
            face_sums(yp, ys, my);
            unfold(mx, ox);
            unfold(my, oy);
            const T c0 = cp2[0].x, c1 = cp2[1].x, c2 = csm[0], c3 = csm[1], c4 = cp2[0].y, c5 = cp2[1].y;
            const T w1 = wul, w2 = w1 * ul, w3 = w2 * ul, w4 = w3 * ul;
            ac[0] += w1 * c0; ac[1] += w2 * c0; ac[2] += w1 * c1; ac[3] += w3 * c0;
            ac[4] += w2 * c1; ac[5] += w1 * c2; ac[6] += w4 * c0; ac[7] += w3 * c1;
            ac[8] += w2 * c2; ac[9] += w1 * c3;
            ac[10] += w1 * c4; ac[11] += w2 * c4; ac[12] += w1 * c5;
            zero_cell();
            tx_ = lane_totals<NM>(ox, lane);
            ty_ = lane_totals<NM>(oy, lane);
        } else {
            T ox[NM], oy[NM];
            face_sums(xp, xs, ox);
            face_sums(yp, ys, oy);
            tx_ = lane_totals<NM>(ox, lane);
            ty_ = lane_totals<NM>(oy, lane);
        }
        if (lane < NM) {
            sacc[warp][(cur & 1) ? 1 : 0][lane] += tx_;
            sacc[warp][(cur & 2) ? 3 : 2][lane] += ty_;
        }
        zero_faces();
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
        const V* cb = buf + (size_t)(k % S) * G * blk;
        const int vb0 = k * G, gk = min(G, nvb - vb0);
        // the blocks of the chunk; INNER: every neighbour of the warp's cell exists (no wall branches)
        auto run_blocks = [&](auto inner_tag) {
            constexpr bool INNER = decltype(inner_tag)::value;
            // the velocities of block g + 1 are loaded while block g is summed
            T nu_ = __ldg(tu + vb0 * VB + lane), nv_ = __ldg(tv + vb0 * VB + lane), nw_ = __ldg(tw + vb0 * VB + lane);
            for (int g = 0; g < gk; ++g) {
                const T u = nu_, v = nv_, w = nw_;
                if (g + 1 < gk) {
                    const int a1 = (vb0 + g + 1) * VB + lane;
                    nu_ = __ldg(tu + a1); nv_ = __ldg(tv + a1); nw_ = __ldg(tw + a1);
                }
                // the classes occupy consecutive blocks: a new one starts where the current one ends
                if (vb0 + g >= cend) {
                    if (cur >= 0) flush();
                    do {
                        ++cur;
                        cend = cd.cls_end[cur];
                    } while (vb0 + g >= cend);
                    if (SEP) {
                        ul = u;
                        wul = __ldg(cd.twu + (vb0 + g) * VB + lane);
                    }
                }
                const int cls = cur;
                const V* ph = cb + (size_t)g * blk + (size_t)kc * VB + lane;
                const V f0 = ph[0];
                V sxv, syv;
                if constexpr (INNER) {
                    sxv = slope2i(ph[-VB], f0, ph[VB], wxm, wxp);
                    syv = slope2i(ph[-PX * VB], f0, ph[PX * VB], wym, wyp);
                } else {
                    sxv = slope2(ph[-VB], f0, ph[VB], wxm, wxp, hm, hp, sx);
                    syv = slope2(ph[-PX * VB], f0, ph[PX * VB], wym, wyp, vm, vp, sy);
                }
                const bool xn = (cls & 1) != 0, yn = (cls & 2) != 0;
                V dx = pfma(sxv, bc(xn ? -hxh : hxh), f0);       // reconstruction at the downwind x-face
                V dy = pfma(syv, bc(yn ? -hyh : hyh), f0);
                if constexpr (!INNER) {
                    // a velocity parallel to a wall carries nothing into it
                    if ((xn ? !hm : !hp) && u == T(0)) dx = bc(T(0));
                    if ((yn ? !vm : !vp) && v == T(0)) dy = bc(T(0));
                }
                const T sxh = sxv.x, syh = syv.x;
                if constexpr (SEP) {
                    // w is w_v here; v-moments of every summand
                    const T c1 = w * v, c2 = c1 * v, c3 = c2 * v;
                    const V bw = bc(w), bc1 = bc(c1);
                    const V tx = pmul(bc(ul), pfma(bc(ul), sxv, pmul(bc(v), syv)));   // u_n (u_n s_n + u_t s_t)
                    const V ty = pmul(bc(v), pfma(bc(v), syv, pmul(bc(ul), sxv)));
                    xp[0] = pfma(dx, bw, xp[0]); xp[1] = pfma(dx, bc1, xp[1]);
                    xs[0] += dx.x * c2; xs[1] += dx.x * c3;
                    yp[0] = pfma(dy, bw, yp[0]); yp[1] = pfma(dy, bc1, yp[1]);
                    ys[0] += dy.x * c2; ys[1] += dy.x * c3;
                    xp[2] = pfma(syv, bw, xp[2]); xs[2] += syh * c1; xs[3] += syh * c2;
                    yp[2] = pfma(sxv, bw, yp[2]); ys[2] += sxh * c1; ys[3] += sxh * c2;
                    xp[3] = pfma(tx, bw, xp[3]); xs[4] += tx.x * c1; xs[5] += tx.x * c2;
                    yp[3] = pfma(ty, bw, yp[3]); ys[4] += ty.x * c1; ys[5] += ty.x * c2;
                    cp2[0] = pfma(f0, bw, cp2[0]); cp2[1] = pfma(f0, bc1, cp2[1]);
                    csm[0] += f0.x * c2; csm[1] += f0.x * c3;
                    continue;
                }
                if constexpr (!SEP) {
                    const T wu = w * u, wv = w * v, wuu = wu * u, wuv = wu * v, wvv = wv * v;
                    const T m[10] = {w, wu, wv, wuu, wuv, wvv, wuu * u, wuu * v, wvv * u, wvv * v};
                    const T wq = wuu + wvv;
                    const V tx = pmul(bc(u), pfma(bc(u), sxv, pmul(bc(v), syv)));
                    const V ty = pmul(bc(v), pfma(bc(v), syv, pmul(bc(u), sxv)));
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        xp[q] = pfma(dx, bc(m[q]), xp[q]);
                        yp[q] = pfma(dy, bc(m[q]), yp[q]);
                        cp2[q] = pfma(f0, bc(m[q]), cp2[q]);
                    }
#pragma unroll
                    for (int q = 3; q < 10; ++q) {
                        xs[q - 3] += dx.x * m[q];
                        ys[q - 3] += dy.x * m[q];
                        csm[q - 3] += f0.x * m[q];
                    }
                    xp[3] = pfma(syv, bc(w), xp[3]); xs[7] += syh * wu; xs[8] += syh * wv; xs[9] += syh * wq;
                    yp[3] = pfma(sxv, bc(w), yp[3]); ys[7] += sxh * wu; ys[8] += sxh * wv; ys[9] += sxh * wq;
                    xp[4] = pfma(tx, bc(w), xp[4]); xs[10] += tx.x * wu; xs[11] += tx.x * wv; xs[12] += tx.x * wq;
                    yp[4] = pfma(ty, bc(w), yp[4]); ys[10] += ty.x * wu; ys[11] += ty.x * wv; ys[12] += ty.x * wq;
                }
            }
        };
        if (valid) {
            if (inner) run_blocks(std::true_type{});
            else run_blocks(std::false_type{});
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[k % S]);
    }
    if (!valid) return;
    if (cur >= 0) flush();
    if constexpr (!SEP) {
#pragma unroll
        for (int q = 0; q < 3; ++q) { ac[q] = cp2[q].x; ac[10 + q] = cp2[q].y; }
#pragma unroll
        for (int q = 0; q < 7; ++q) ac[3 + q] = csm[q];
    }
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
    return (size_t)S * G * (TX + 2) * (TY + 2) * VB * sizeof(P2<T>);
}

// ------------------------------------------------------------------------------ K4: micro update

// Micro flux pair (delta form, divided by dG_f) through the downwind face of the reconstructing cell, for one
// lane: u_n [C1' dH + H Q + C4' d0 + C5' (u_n s_n + u_t s_t)] for h and u_n [C1' dB + B (Q + lin) + C4' e0 +
// C5' (...)] for b, from the face's parameters fp (shared memory; the cubic at qo and linear term at lo belong to
// the upwind side), the expm1 factors (ex, ey) of the interface Maxwellian at the lane's velocity, the
// reconstructed pair d0 and the normal and tangential slope pairs; unb, utb are (u_n, u_n) and (u_t, u_t).
template <typename T, typename V>
__device__ __forceinline__ V flux2(const T* fp, int qo, int lo, T ex, T ey, T href, T u, T v, V unb, V utb, V d0,
                                   V sn, V st)
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
    V m = pk(sc[4] * dH + H * Q, sc[4] * dB + (H * i2l) * Qb);
    m = pfma(bc(sc[5]), d0, m);
    m = pfma(bc(sc[6]), pfma(unb, sn, pmul(utb, st)), m);
    return pmul(unb, m);
}

// Flux pair (delta form, divided by dG_f) of the distribution a diffuse wall re-emits, rho_w H_w u_n: velocities
// of the block leave the wall.
template <typename T, typename V>
__device__ __forceinline__ V flux_wall2(const T* fp, const T* __restrict__ tb, int iu, int ivn, T href, V unb)
{
    const T* wp = fp + F_WRM1;
    const T ex = __ldg(tb + iu), ey = __ldg(tb + ivn);
    const T E = ex + ey + ex * ey;
    const T dHw = href * (wp[0] + wp[1] * E);
    return pmul(unb, pk(dHw, dHw * wp[2] + href * wp[3]));
}

// Equilibrium pair (H+ - H_ref, B+ - B_ref) of one cell-parameter slot q at the lane's velocity: the Maxwellian
// from the cell table factors (ex, ey), and with the Shakhov model the correction (L Q) H for h and (L Q + 2 L) B
// for b (L, Q the linear and quadratic factors of s (c.q)(2 lam |c|^2 - 4); r2 = u^2 + v^2).
template <typename T>
__device__ __forceinline__ P2<T> eq2(const T* q, T ex, T ey, T href, T u, T v, T r2, bool shakhov)
{
    const T E = ex + ey + ex * ey;
    const T dH = href * (q[E_RM1] + q[E_R] * E);
    const T dB = dH * q[E_I2L] + href * q[E_DI2L];
    if (!shakhov) return pk(dH, dB);
    const T H = href + dH;
    const T L = q[E_L] + q[E_L + 1] * u + q[E_L + 2] * v;
    const T Qs = q[E_Q] + q[E_Q + 1] * u + q[E_Q + 2] * v + q[E_Q + 3] * r2;
    const T sk = L * Qs;
    return pfma(pk(H, H * q[E_I2L]), pk(sk, sk + T(2) * L), pk(dH, dB));
}

// One bulk copy of the per-level batches of k4_cells, formed once per CTA: level l's copy reads src + l sstride
// and lands in ring slot l & 1 (dst + (l & 1) dslot).  kind 0: a row of the halo rectangle, 1: a row of face
// parameters (both of level k in batch k), 2: a row of cell coefficients (level k - 1 in batch k); bytes 0: the
// row lies outside the domain.
struct alignas(16) K4Copy {
    const char* src;
    long long sstride;
    uint32_t dst, dslot, bytes;
    int kind;
};

// Shared-memory layout of k4_cells (byte offsets, pairs for distributions, each block 16-byte aligned).  A CTA
// owns VPL velocity blocks of one sign class (h = 0..VPL-1 below), and each lane one velocity of every block:
//   own   [nt][VPL][NCT][32] pairs   the tile's own cells on every level: h^k as loaded; in the explicit form
//                                    replaced once by the spectral source of every level
//   rect  [2][VPL][NR][32] pairs     per level: the tile with its halo, (TX+3) x (TY+3) cells, two cells on
//                                    the upwind side of each axis and one on the downwind side (ring of 2)
//   fp    [2][NFT][NP] T             per level: parameters of the tile's faces (ring of 2 levels)
//   cp    [2][NCT][NCP] T            per level: update coefficients of the tile's cells (ring of 2 levels)
//   flux  [2][VPL][NFT][32] pairs    per level: micro fluxes of the tile's faces (double buffered)
template <typename T, int TX, int TY, int VPL>
struct K4Layout {
    using V = P2<T>;
    static constexpr int PX = TX + 3, PY = TY + 3, NR = PX * PY, NCT = TX * TY;
    static constexpr int NFX = TY * (TX + 1), NFY = (TY + 1) * TX, NFT = NFX + NFY;
    static constexpr size_t RECT = (size_t)VPL * NR * VB;               // pairs per ring slot
    static constexpr size_t FP = (size_t)NFT * NP, CP = (size_t)NCT * NCP, FLUX = (size_t)VPL * NFT * VB;
    __host__ __device__ static constexpr size_t own_bytes(int nt) { return (size_t)nt * VPL * NCT * VB * sizeof(V); }
    __host__ __device__ static constexpr size_t rect_off(int nt) { return own_bytes(nt); }
    __host__ __device__ static constexpr size_t fp_off(int nt) { return rect_off(nt) + 2 * RECT * sizeof(V); }
    __host__ __device__ static constexpr size_t cp_off(int nt) { return fp_off(nt) + 2 * FP * sizeof(T); }
    __host__ __device__ static constexpr size_t flux_off(int nt) { return cp_off(nt) + 2 * CP * sizeof(T); }
    __host__ __device__ static constexpr size_t bytes(int nt) { return flux_off(nt) + 2 * FLUX * sizeof(V); }
};

// A CTA: a TX x TY tile of cells, VPL velocity blocks of one sign class, all levels.  Per level, the first pass
// reconstructs every tile cell and the upwind halo cells and evaluates the flux through each one's downwind
// face (every face of the tile exactly once); the second pass applies Eq. fv_h to the tile cells.  Each item
// (a cell of a pass) forms its indices, addresses and face or cell parameters once and serves the lane's
// velocity in each of the VPL blocks.  The second pass of level n runs in the same barrier interval as the
// first pass of level n + 1 (fluxes double buffered), so one barrier separates the levels.  In the explicit
// form the spectral source of every level is formed once per CTA, in place in the own-cell store, and each
// warp keeps h^k of its pass-2 cells from pass 1.  With IMP and a case that asks for it, the spectral source is
// taken at the new iterate instead: pass 2 leaves each level's right-hand side in the own-cell store and a last
// pass applies the per-cell inverse across levels.  Batch k of bulk copies (the halo rectangle and face
// parameters of level k, the cell coefficients of level k - 1; batch 0 also every level of the tile's own
// cells) completes on mbarrier k & 1 and is issued one level ahead of its use.
template <typename T, int TX, int TY, int NW, bool IMP, int VPL>
__global__ void __launch_bounds__(NW * 32) k4_cells(Batch<T> B)
{
    using L = K4Layout<T, TX, TY, VPL>;
    using V = P2<T>;
    constexpr int PX = L::PX, PY = L::PY, NR = L::NR, NCT = L::NCT, NFX = L::NFX, NFT = L::NFT;
    constexpr int NIT = NCT + TY + TX, NPASS = (NIT + NW - 1) / NW;
    constexpr int NP2 = (NCT + NW - 1) / NW;                  // tile cells per warp in pass 2
    constexpr int SROWS = 4;                                  // tile rows per strip of the CTA order
    constexpr int LVO = VPL * NCT * VB;                       // level stride of the own-cell store (pairs)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bars[2];
    __shared__ T gxr[PX], gxh[PX], gyr[PY], gyh[PY];
    const int cs = find_case(B.off, B.ncases, blockIdx.x);
    const CaseDev<T>& cd = B.cases[cs];
    if (!cd.st->active) return;
    // another CTA may set the error word while this one starts: decide for the whole CTA at once
    if (__syncthreads_or(*(volatile int*)cd.err != 0)) return;
    const bool expire = *(volatile const int*)cd.expire != 0;
    const int nvg = cd.nvb / VPL, nx = cd.nx, ny = cd.ny;
    // CTA order: velocity group fastest (the CTAs of one tile share its parameters in L2), then tiles in
    // strips of SROWS tile rows, column by column (neighbour tiles, whose halos overlap, run close in time)
    const int lb = blockIdx.x - B.off[cs];
    const int vb = (lb % nvg) * VPL, tile = lb / nvg;         // vb: the CTA's first velocity block
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
    V* const own = reinterpret_cast<V*>(smem_raw);
    V* const rect = reinterpret_cast<V*>(smem_raw + L::rect_off(nt));
    T* const fps = reinterpret_cast<T*>(smem_raw + L::fp_off(nt));
    T* const cps = reinterpret_cast<T*>(smem_raw + L::cp_off(nt));
    V* const fbuf = reinterpret_cast<V*>(smem_raw + L::flux_off(nt));
    mbar_setup(bars, 2);
    const int p = cd.st->parity;
    const V* gf = cd.f[p];
    const size_t bstride = (size_t)nt * nc * VB;              // pairs between consecutive velocity blocks
    // bulk copies of the rectangle rows (clipped to the domain)
    const int c0 = max(i0 + xlo, 0), c1 = min(i0 + xlo + PX, nx);
    const int nfr = iend - i0;                                // valid cells per tile row
    const uint32_t row_b = (uint32_t)((c1 - c0) * VB * sizeof(V));
    int rrows = 0;
    for (int r = 0; r < PY; ++r) {
        const int jj = j0 + ylo + r;
        rrows += (jj >= 0 && jj < ny) ? 1 : 0;
    }
    const uint32_t rect_b = (uint32_t)(VPL * rrows) * row_b;
    const uint32_t fp_b = (uint32_t)(((jend - j0) * (nfr + 1) + (jend - j0 + 1) * nfr) * NP * sizeof(T));
    const uint32_t cp_b = (uint32_t)((jend - j0) * nfr * NCP * sizeof(T));
    // batch 0 (warp 0): rectangle and face parameters of level 0, every level of the own cells
    {
        constexpr int NRECT = VPL * PY, NFPR = 2 * TY + 1;
        const int nown = nt * VPL * TY;
        if (warp == 0) {
            if (lane == 0)
                mbar_arrive_expect(&bars[0], rect_b + fp_b + (uint32_t)(nt * VPL * (jend - j0) * nfr * VB * sizeof(V)));
            __syncwarp();
            for (int q = lane; q < NRECT + NFPR + nown; q += 32) {
                if (q < NRECT) {
                    const int h = q / PY, r = q % PY, jj = j0 + ylo + r;
                    if (jj < 0 || jj >= ny) continue;
                    bulk_g2s(rect + (size_t)(h * NR + r * PX + c0 - (i0 + xlo)) * VB,
                             gf + (vb + h) * bstride + ((size_t)jj * nx + c0) * VB, row_b, &bars[0]);
                } else if (q < NRECT + NFPR) {
                    const int r = q - NRECT;
                    if (r < TY) {                             // x-faces of tile row r
                        const int jj = j0 + r;
                        if (jj >= ny) continue;
                        bulk_g2s(fps + (size_t)r * (TX + 1) * NP, cd.fpar + ((size_t)jj * (nx + 1) + i0) * NP,
                                 (uint32_t)((nfr + 1) * NP * sizeof(T)), &bars[0]);
                    } else {                                  // y-faces of face row r - TY
                        const int fr = r - TY, jj = j0 + fr;
                        if (jj > jend) continue;
                        bulk_g2s(fps + (size_t)(NFX + fr * TX) * NP, cd.fpar + ((size_t)nfx + (size_t)jj * nx + i0) * NP,
                                 (uint32_t)(nfr * NP * sizeof(T)), &bars[0]);
                    }
                } else {
                    const int o = q - NRECT - NFPR;           // own cells: row, block, level
                    const int r = o % TY, h = (o / TY) % VPL, n = o / (TY * VPL), jj = j0 + r;
                    if (jj >= ny) continue;
                    bulk_g2s(own + ((size_t)(n * VPL + h) * NCT + r * TX) * VB,
                             gf + (vb + h) * bstride + (size_t)n * nc * VB + ((size_t)jj * nx + i0) * VB,
                             (uint32_t)(nfr * VB * sizeof(V)), &bars[0]);
                }
            }
        }
    }
    // the copies of batches 1..nt, formed once: at each level warp 0 then only offsets them
    constexpr int NQ = VPL * PY + 2 * TY + 1 + TY;
    static_assert(NQ <= 32, "one lane of warp 0 per copy of a batch");
    __shared__ K4Copy cpy[32];
    if (warp == 0 && lane < NQ) {
        K4Copy c;
        c.bytes = 0;
        c.src = nullptr;
        c.sstride = 0;
        c.dst = 0;
        c.dslot = 0;
        c.kind = 0;
        if (lane < VPL * PY) {
            const int h = lane / PY, r = lane % PY, jj = j0 + ylo + r;
            if (jj >= 0 && jj < ny) {
                c.src = reinterpret_cast<const char*>(gf + (vb + h) * bstride + ((size_t)jj * nx + c0) * VB);
                c.sstride = (long long)nc * VB * sizeof(V);
                c.dst = smem_u32(rect + (size_t)(h * NR + r * PX + c0 - (i0 + xlo)) * VB);
                c.dslot = (uint32_t)(L::RECT * sizeof(V));
                c.bytes = row_b;
            }
        } else if (lane < VPL * PY + 2 * TY + 1) {
            const int r = lane - VPL * PY;
            c.kind = 1;
            c.sstride = (long long)nf * NP * sizeof(T);
            c.dslot = (uint32_t)(L::FP * sizeof(T));
            if (r < TY) {                                     // x-faces of tile row r
                const int jj = j0 + r;
                if (jj < ny) {
                    c.src = reinterpret_cast<const char*>(cd.fpar + ((size_t)jj * (nx + 1) + i0) * NP);
                    c.dst = smem_u32(fps + (size_t)r * (TX + 1) * NP);
                    c.bytes = (uint32_t)((nfr + 1) * NP * sizeof(T));
                }
            } else {                                          // y-faces of face row r - TY
                const int fr = r - TY, jj = j0 + fr;
                if (jj <= jend) {
                    c.src = reinterpret_cast<const char*>(cd.fpar + ((size_t)nfx + (size_t)jj * nx + i0) * NP);
                    c.dst = smem_u32(fps + (size_t)(NFX + fr * TX) * NP);
                    c.bytes = (uint32_t)(nfr * NP * sizeof(T));
                }
            }
        } else {
            const int r = lane - VPL * PY - 2 * TY - 1, jj = j0 + r;   // cells of tile row r
            c.kind = 2;
            if (jj < ny) {
                c.src = reinterpret_cast<const char*>(cd.cpar + ((size_t)jj * nx + i0) * NCP);
                c.sstride = (long long)nc * NCP * sizeof(T);
                c.dst = smem_u32(cps + (size_t)r * TX * NCP);
                c.dslot = (uint32_t)(L::CP * sizeof(T));
                c.bytes = (uint32_t)(nfr * NCP * sizeof(T));
            }
        }
        cpy[lane] = c;
    }
    __syncwarp();
    // batch k >= 1 (warp 0): rectangle and face parameters of level k (k < nt), cell coefficients of level k - 1
    auto issue_next = [&](int k) {
        const bool lvl = k < nt;
        uint64_t* bar = &bars[k & 1];
        if (lane == 0) mbar_arrive_expect(bar, (lvl ? rect_b + fp_b : 0u) + cp_b);
        __syncwarp();
        if (lane < NQ) {
            const K4Copy c = cpy[lane];
            if (c.bytes != 0 && (lvl || c.kind == 2)) {
                const int l = c.kind == 2 ? k - 1 : k;
                bulk_g2s_at(c.dst + (uint32_t)(l & 1) * c.dslot, c.src + (long long)l * c.sstride, c.bytes, bar);
            }
        }
    };
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
    // the lane's velocity in each of the CTA's blocks
    T u[VPL], v[VPL], href[VPL], r2[VPL];
    int iu[VPL], ivn[VPL];
#pragma unroll
    for (int h = 0; h < VPL; ++h) {
        const int av = (vb + h) * VB + lane;
        u[h] = __ldg(cd.tu + av);
        v[h] = __ldg(cd.tv + av);
        href[h] = __ldg(cd.thref + av);
        r2[h] = u[h] * u[h] + v[h] * v[h];
        iu[h] = __ldg(cd.viu + av);
        ivn[h] = cd.nu + __ldg(cd.viv + av);
    }
    V etb[IMP ? 8 : 1];                                       // implicit-capable kernels: e_d as pairs
#pragma unroll
    for (int d = 0; d < (IMP ? 8 : 1); ++d) etb[d] = bc(cd.et[d]);
    const T* __restrict__ ftab = cd.ftab;
    const T* __restrict__ wtab = cd.wtab;
    const T* __restrict__ ctab = cd.ctab;
    const bool shakhov = cd.shakhov != 0;
    const int NTf = nt * nuv;                                 // per-face stride of the expm1 tables
    const int qoff = xneg ? F_QR : F_QL, loff = xneg ? F_LBR : F_LBL;
    const int qoffy = yneg ? F_QR : F_QL, loffy = yneg ? F_LBR : F_LBL;
    int* err = cd.err;

    const bool implicit = IMP && cd.spectral_implicit != 0;   // IMP = false compiles the explicit form alone
    // a tile none of whose first-pass cells (tile cells and upwind halo) touches a wall: every stencil neighbour
    // of each exists
    const bool interior = i0 >= 2 && j0 >= 2 && i0 + TX <= nx - 2 && j0 + TY <= ny - 2;
    constexpr bool PAIRED = NCT == 2 * NW;                    // each warp owns two tile cells in pass 1
    V f0k[NP2][VPL];                                          // h^k of the warp's pass-2 cells (explicit form)
#pragma unroll
    for (int r = 0; r < NP2; ++r)
#pragma unroll
        for (int h = 0; h < VPL; ++h) f0k[r][h] = bc(T(0));

    __syncthreads();                                          // the spacing tables above, for every warp
    for (int s = 0; s <= nt; ++s) {
        if (warp == 0 && s < nt) issue_next(s + 1);
        // the test hook reports the first wait as expired only after it has completed
        const int fail = !mbar_wait(&bars[s & 1], (uint32_t)((s >> 1) & 1), err) || expire;
        if (!fail) {
            if (!IMP && s == 0) {
                // the spectral source of every level of the warp's own cells, once, in place of h^k
#pragma unroll
                for (int r = 0; r < NP2; ++r) {
                    const int ct = warp + r * NW;
                    if (ct >= NCT) break;
                    if (i0 + ct % TX >= nx || j0 + ct / TX >= ny) continue;
#pragma unroll
                    for (int h = 0; h < VPL; ++h) {
                        V* fc = own + (size_t)(h * NCT + ct) * VB + lane;
                        switch (nh) {
                            case 0: spectral_all<0>(fc, LVO, cd.et); break;
                            case 1: spectral_all<1>(fc, LVO, cd.et); break;
                            case 2: spectral_all<2>(fc, LVO, cd.et); break;
                            case 3: spectral_all<3>(fc, LVO, cd.et); break;
                            case 4: spectral_all<4>(fc, LVO, cd.et); break;
                            case 5: spectral_all<5>(fc, LVO, cd.et); break;
                            case 6: spectral_all<6>(fc, LVO, cd.et); break;
                            default: spectral_all<7>(fc, LVO, cd.et); break;
                        }
                    }
                }
                __syncwarp();
            }
            if (s > 0) {
                // ---- pass 2, level s - 1 (ahead of pass 1 of level s, which refills f0k): Eq. fv_h with the
                // spectral source (delta form)
                const int n = s - 1;
                const V* F = fbuf + (size_t)(n & 1) * L::FLUX + lane;
                V* on = cd.f[p ^ 1] + vb * bstride + (size_t)n * nc * VB + lane;
                const T* cpn = cps + (size_t)(n & 1) * L::CP;
                const T* ctn = ctab + n * 2 * nuv;
#pragma unroll
                for (int r = 0; r < NP2; ++r) {
                    const int ct = warp + r * NW;
                    if (ct >= NCT) break;
                    const int ti = ct % TX, tj = ct / TX;
                    const int i = i0 + ti, j = j0 + tj;
                    if (i >= nx || j >= ny) continue;
                    const int c = j * nx + i;
                    const T* tb = ctn + c * nt * 2 * nuv;
                    const int fL = tj * (TX + 1) + ti, fB = NFX + tj * TX + ti;
                    const T* cp = cpn + ct * NCP;
                    const V* k = reinterpret_cast<const V*>(cp + C_K);   // kself, -kE, kp1, kp0, -kdx, -kdy
#pragma unroll
                    for (int h = 0; h < VPL; ++h) {
                        const T ex0 = __ldg(tb + iu[h]), ey0 = __ldg(tb + ivn[h]);
                        const T ex1 = __ldg(tb + nuv + iu[h]), ey1 = __ldg(tb + nuv + ivn[h]);
                        const V* Fh = F + (size_t)h * NFT * VB;
                        const V dX = psub(Fh[(fL + 1) * VB], Fh[fL * VB]);
                        const V dY = psub(Fh[(fB + TX) * VB], Fh[fB * VB]);
                        V* fc = own + (size_t)(h * NCT + ct) * VB + lane;   // level m at fc[m * LVO]
                        V e, f0;
                        if constexpr (!IMP) {
                            e = fc[n * LVO];                  // precomputed
                            f0 = f0k[r][h];
                        } else {
                            switch (implicit ? 0 : nh) {
                                case 0: e = etb[0]; break;
                                case 1: e = spectral2<1>(fc, n, nt, LVO, etb); break;
                                case 2: e = spectral2<2>(fc, n, nt, LVO, etb); break;
                                case 3: e = spectral2<3>(fc, n, nt, LVO, etb); break;
                                case 4: e = spectral2<4>(fc, n, nt, LVO, etb); break;
                                case 5: e = spectral2<5>(fc, n, nt, LVO, etb); break;
                                case 6: e = spectral2<6>(fc, n, nt, LVO, etb); break;
                                default: e = spectral2<7>(fc, n, nt, LVO, etb); break;
                            }
                            f0 = fc[n * LVO];
                        }
                        // equilibria of W^{k+1} (slot 1) and W^k (slot 0), delta form
                        const V q1 = eq2(cp + C_EQ1, ex1, ey1, href[h], u[h], v[h], r2[h], shakhov);
                        const V q0 = eq2(cp + C_EQ0, ex0, ey0, href[h], u[h], v[h], r2[h], shakhov);
                        V x = pmul(k[0], f0);
                        x = pfma(k[4], dX, x);
                        x = pfma(k[5], dY, x);
                        x = pfma(k[1], e, x);
                        x = pfma(k[2], q1, x);
                        x = pfma(k[3], q0, x);
                        if (implicit) fc[n * LVO] = x;       // right-hand side of level n; h^k no longer needed
                        else on[h * bstride + (size_t)c * VB] = x;
                    }
                }
            }
            if (s < nt) {
                // ---- pass 1, level s: reconstruction and downwind-face fluxes
                const int n = s;
                V* F = fbuf + (size_t)(n & 1) * L::FLUX + lane;
                const V* rh = rect + (size_t)(n & 1) * L::RECT + lane;
                const T* fpn = fps + (size_t)(n & 1) * L::FP;
                const T* ftn = ftab + n * nuv;
                int rfirst = 0;
                if (PAIRED && interior) {
                    // both tile cells of the warp, every block, as one straight-line block, stores last, so that
                    // the independent chains interleave
                    V fl[2][VPL][2];
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
                        const T wxm = gxr[kx - 1], wxp = gxr[kx], wym = gyr[ky - 1], wyp = gyr[ky];
                        const V hx = bc(xneg ? -gxh[kx] : gxh[kx]), hy = bc(yneg ? -gyh[ky] : gyh[ky]);
#pragma unroll
                        for (int h = 0; h < VPL; ++h) {
                            const T exx = __ldg(tbx + iu[h]), eyx = __ldg(tbx + ivn[h]);
                            const T exy = __ldg(tby + iu[h]), eyy = __ldg(tby + ivn[h]);
                            const V* ph = rh + (size_t)(h * NR + ky * PX + kx) * VB;
                            const V f0 = ph[0];
                            f0k[q][h] = f0;
                            const V sxv = slope2i(ph[-VB], f0, ph[VB], wxm, wxp);
                            const V syv = slope2i(ph[-PX * VB], f0, ph[PX * VB], wym, wyp);
                            const V dx0 = pfma(sxv, hx, f0);
                            const V dy0 = pfma(syv, hy, f0);
                            const V ub = bc(u[h]), vbb = bc(v[h]);
                            fl[q][h][0] = flux2(fpn + sl[q][0] * NP, qoff, loff, exx, eyx, href[h], u[h], v[h], ub, vbb,
                                                dx0, sxv, syv);
                            fl[q][h][1] = flux2(fpn + sl[q][1] * NP, qoffy, loffy, exy, eyy, href[h], u[h], v[h], vbb,
                                                ub, dy0, syv, sxv);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 2; ++q)
#pragma unroll
                        for (int h = 0; h < VPL; ++h) {
                            F[(h * NFT + sl[q][0]) * VB] = fl[q][h][0];
                            F[(h * NFT + sl[q][1]) * VB] = fl[q][h][1];
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
                    if (!interior && (i < 0 || i >= nx || j < 0 || j >= ny)) {
                        // upwind face of the tile on a wall: the re-emitted distribution
                        int slot;
                        const T* wt;
                        if (dox) {
                            const int fi = i < 0 ? 0 : nx;
                            slot = tj * (TX + 1) + fi - i0;
                            wt = wtab + ((i < 0 ? 3 : 1) * cd.nslot + wall_slot(cd, n)) * nuv;
                        } else {
                            const int fj = j < 0 ? 0 : ny;
                            slot = NFX + (fj - j0) * TX + ti;
                            wt = wtab + ((j < 0 ? 0 : 2) * cd.nslot + wall_slot(cd, n)) * nuv;
                        }
#pragma unroll
                        for (int h = 0; h < VPL; ++h)
                            F[(h * NFT + slot) * VB] = flux_wall2(fpn + slot * NP, wt, iu[h], ivn[h], href[h],
                                                                  bc(dox ? u[h] : v[h]));
                        continue;
                    }
                    const int kx = ti - xlo, ky = tj - ylo;
                    const int fix = xneg ? i : i + 1, fjy = yneg ? j : j + 1;
                    const int slx = tj * (TX + 1) + fix - i0, sly = NFX + (fjy - j0) * TX + ti;
                    const T* tbx = ftn + (j * (nx + 1) + fix) * NTf;
                    const T* tby = ftn + (nfx + fjy * nx + i) * NTf;
                    const T wxm = gxr[kx - 1], wxp = gxr[kx], wym = gyr[ky - 1], wyp = gyr[ky];
#pragma unroll
                    for (int h = 0; h < VPL; ++h) {
                        // expm1 factors of the interface Maxwellians first: their latency overlaps the
                        // reconstruction
                        T exx = T(0), eyx = T(0), exy = T(0), eyy = T(0);
                        if (dox) { exx = __ldg(tbx + iu[h]); eyx = __ldg(tbx + ivn[h]); }
                        if (doy) { exy = __ldg(tby + iu[h]); eyy = __ldg(tby + ivn[h]); }
                        const V* ph = rh + (size_t)(h * NR + ky * PX + kx) * VB;
                        const V f0 = ph[0];
                        if (r < NP2 && it < NCT) f0k[r][h] = f0;
                        V sxv, syv;
                        if (interior) {
                            sxv = slope2i(ph[-VB], f0, ph[VB], wxm, wxp);
                            syv = slope2i(ph[-PX * VB], f0, ph[PX * VB], wym, wyp);
                        } else {
                            sxv = slope2(ph[-VB], f0, ph[VB], wxm, wxp, i > 0, i < nx - 1, nx > 1);
                            syv = slope2(ph[-PX * VB], f0, ph[PX * VB], wym, wyp, j > 0, j < ny - 1, ny > 1);
                        }
                        const V ub = bc(u[h]), vbb = bc(v[h]);
                        if (dox) {
                            const V d0 = pfma(sxv, bc(xneg ? -gxh[kx] : gxh[kx]), f0);
                            F[(h * NFT + slx) * VB] = flux2(fpn + slx * NP, qoff, loff, exx, eyx, href[h], u[h], v[h],
                                                            ub, vbb, d0, sxv, syv);
                        }
                        if (doy) {
                            const V d0 = pfma(syv, bc(yneg ? -gyh[ky] : gyh[ky]), f0);
                            F[(h * NFT + sly) * VB] = flux2(fpn + sly * NP, qoffy, loffy, exy, eyy, href[h], u[h],
                                                            v[h], vbb, ub, d0, syv, sxv);
                        }
                    }
                }
            }
        }
        // one barrier per level: it publishes this level's fluxes, frees the ring slots read here, and makes
        // the CTA agree on a failed wait
        if (__syncthreads_or(fail)) {
            // warp 0, which issued them, waits (bounded) for batches s and s + 1, so that no bulk copy still
            // lands in shared memory after the CTA exits
            if (threadIdx.x == 0 && expire) atomicExch(err, 1);
            if (warp == 0) {
                mbar_drain(&bars[s & 1], (uint32_t)((s >> 1) & 1));
                if (s < nt) mbar_drain(&bars[(s + 1) & 1], (uint32_t)(((s + 1) >> 1) & 1));
            }
            return;
        }
    }
    if (implicit) {
        // spectral source at the new iterate: f^{k+1} = minv (right-hand sides over the levels), per cell, block
        // and lane
        for (int ct = warp; ct < NCT; ct += NW) {
            const int ti = ct % TX, tj = ct / TX;
            const int i = i0 + ti, j = j0 + tj;
            if (i >= nx || j >= ny) continue;
            const int c = j * nx + i;
            const T* Mi = cd.minv + (size_t)c * nt * nt;
#pragma unroll
            for (int h = 0; h < VPL; ++h) {
                const V* fc = own + (size_t)(h * NCT + ct) * VB + lane;
                V rr[MAXNT];
#pragma unroll
                for (int m = 0; m < MAXNT; ++m) rr[m] = m < nt ? fc[m * LVO] : bc(T(0));
                V* o = cd.f[p ^ 1] + (vb + h) * bstride + (size_t)c * VB + lane;
#pragma unroll
                for (int n = 0; n < MAXNT; ++n) {
                    if (n >= nt) break;
                    V acc = bc(T(0));
#pragma unroll
                    for (int m = 0; m < MAXNT; ++m)
                        if (m < nt) acc = pfma(bc(__ldg(Mi + n * nt + m)), rr[m], acc);
                    o[(size_t)n * nc * VB] = acc;
                }
            }
        }
    }
}

template <typename T, int TX, int TY, int VPL>
constexpr size_t k4_cells_smem(int nt)
{
    return K4Layout<T, TX, TY, VPL>::bytes(nt);
}

}  // namespace hb
