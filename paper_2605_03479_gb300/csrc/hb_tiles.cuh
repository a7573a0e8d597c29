// Tiled kernels of the per-velocity work of one HB-UGKS iteration:
//   k1_tile : velocity sums of the upwinded, limited interface reconstruction (per face and level) and raw
//             moments of h^k (per cell and level);
//   k4_tile : interface micro fluxes (Eq. micro_flux), spectral source and semi-implicit collision update
//             (Eq. fv_h) of every cell, velocity and level.
// A CTA owns a TX x TY tile of cells.  The tile and the halo its stencil needs (two cells along each axis,
// one across the diagonal) are staged in shared memory by bulk copies (TMA) once per level block; every face
// flux is then evaluated once per level and velocity and shared by the two cells it separates.  Lanes of a
// warp are 32 consecutive discrete velocities.
#pragma once
#include "hb_common.cuh"

namespace hb {

// Staged region of a tile, row by row.  Row r holds j = j0 + r - 2 and the columns the stencil reaches:
// rows -2 and TY + 1 need [0, TX), rows -1 and TY need [-1, TX + 1), the tile rows need [-2, TX + 2).
template <int TX, int TY>
struct Tile {
    static constexpr int clo(int r) { return (r == 0 || r == TY + 3) ? 0 : ((r == 1 || r == TY + 2) ? -1 : -2); }
    static constexpr int chi(int r) { return (r == 0 || r == TY + 3) ? TX : ((r == 1 || r == TY + 2) ? TX + 1 : TX + 2); }
    static constexpr int rowoff(int r)
    {
        int s = 0;
        for (int k = 0; k < r; ++k) s += chi(k) - clo(k);
        return s;
    }
    static constexpr int NCELL = rowoff(TY + 4);
    // staged index of tile cell (ti, tj): closed form of rowoff(tj + 2) - clo(tj + 2) + ti
    __host__ __device__ static constexpr int idx(int ti, int tj)
    {
        return tj < -1 ? ti
             : tj == -1 ? TX + 1 + ti
             : tj < TY ? 2 * TX + 4 + tj * (TX + 4) + ti
             : tj == TY ? 2 * TX + 3 + TY * (TX + 4) + ti
             : 3 * TX + 4 + TY * (TX + 4) + ti;
    }
    static constexpr int NXF = (TX + 1) * TY;
    static constexpr int NF = NXF + TX * (TY + 1);
    static constexpr int NCT = TX * TY;
};

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

// 16-byte vector loads of N consecutive parameters (N a multiple of 16 / sizeof(T), p 16-byte aligned)
template <int N>
__device__ __forceinline__ void ldv(const float* p, float* o)
{
#pragma unroll
    for (int k = 0; k < N; k += 4) {
        const float4 v = *reinterpret_cast<const float4*>(p + k);
        o[k] = v.x; o[k + 1] = v.y; o[k + 2] = v.z; o[k + 3] = v.w;
    }
}
template <int N>
__device__ __forceinline__ void ldv(const double* p, double* o)
{
#pragma unroll
    for (int k = 0; k < N; k += 2) {
        const double2 v = *reinterpret_cast<const double2*>(p + k);
        o[k] = v.x; o[k + 1] = v.y;
    }
}

// A face of the tile: fidx < NXF are x-normal faces (a = 0..TX, r = 0..TY-1), the rest y-normal.
struct TFace {
    int axis, tiL, tjL, tiR, tjR, i, j, gface;
    bool valid, hasL, hasR;
    int wall;
};

template <typename T, int TX, int TY>
__device__ __forceinline__ TFace tface(const CaseDev<T>& cd, int fidx, int i0, int j0)
{
    using S = Tile<TX, TY>;
    TFace f;
    if (fidx < S::NXF) {
        int a = fidx % (TX + 1), r = fidx / (TX + 1);
        f.axis = 0;
        f.i = i0 + a; f.j = j0 + r;
        f.valid = f.i <= cd.nx && f.j < cd.ny;
        f.tiL = a - 1; f.tjL = r; f.tiR = a; f.tjR = r;
        f.hasL = f.i > 0; f.hasR = f.i < cd.nx;
        f.gface = f.j * (cd.nx + 1) + f.i;
        f.wall = f.i == 0 ? 3 : 1;
    } else {
        int ff = fidx - S::NXF;
        int a = ff % TX, r = ff / TX;
        f.axis = 1;
        f.i = i0 + a; f.j = j0 + r;
        f.valid = f.i < cd.nx && f.j <= cd.ny;
        f.tiL = a; f.tjL = r - 1; f.tiR = a; f.tjR = r;
        f.hasL = f.j > 0; f.hasR = f.j < cd.ny;
        f.gface = cd.nfx + f.j * cd.nx + f.i;
        f.wall = f.j == 0 ? 0 : 2;
    }
    return f;
}

// One candidate upwind cell of a face: staged indices of the cell and its axis neighbours (the cell itself
// where a neighbour is outside the domain), presence flags, inverse centre distances, and the signed offset
// from the cell centre to the face along the face normal.
template <typename T>
struct FSide {
    int c, xm, xp, ym, yp, flags;   // flags: 1 x-, 2 x+, 4 y-, 8 y+ neighbours present; 16 nx > 1; 32 ny > 1
    T wxm, wxp, wym, wyp, off;
};

template <typename T>
struct FStencil {
    FSide<T> s[2];                  // [0] low-side cell (upwind for u_n > 0), [1] high-side cell
    int gface, wall, axis, valid, hasL, hasR;
};

// Tile geometry in shared memory (local index k <-> global index i0 - 2 + k)
template <typename T, int TX, int TY>
struct TileGeo {
    T rdx[TX + 4], rdy[TY + 4], hx[TX + 4], hy[TY + 4];
};

template <typename T, int TX, int TY>
__device__ __forceinline__ void load_geo(const CaseDev<T>& cd, int i0, int j0, TileGeo<T, TX, TY>& g)
{
    for (int k = threadIdx.x; k < TX + 4; k += blockDim.x) {
        int i = i0 - 2 + k;
        bool ok = i >= 0 && i < cd.nx;
        g.rdx[k] = ok ? T(cd.rdx[i]) : T(0);
        g.hx[k] = ok ? T(cd.hx[i]) : T(0);
    }
    for (int k = threadIdx.x; k < TY + 4; k += blockDim.x) {
        int j = j0 - 2 + k;
        bool ok = j >= 0 && j < cd.ny;
        g.rdy[k] = ok ? T(cd.rdy[j]) : T(0);
        g.hy[k] = ok ? T(cd.hy[j]) : T(0);
    }
}

// Face stencils of a tile into shared memory (call after the geometry is loaded and synchronised)
template <typename T, int TX, int TY>
__device__ __forceinline__ void build_stencils(const CaseDev<T>& cd, const TileGeo<T, TX, TY>& g, int i0, int j0,
                                               FStencil<T>* st)
{
    using S = Tile<TX, TY>;
    for (int fi = threadIdx.x; fi < S::NF; fi += blockDim.x) {
        const TFace f = tface<T, TX, TY>(cd, fi, i0, j0);
        FStencil<T> o;
        o.gface = f.gface; o.wall = f.wall; o.axis = f.axis; o.valid = f.valid; o.hasL = f.hasL; o.hasR = f.hasR;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            FSide<T>& s = o.s[side];
            const bool present = side == 0 ? f.hasL : f.hasR;
            const int ti = side == 0 ? f.tiL : f.tiR, tj = side == 0 ? f.tjL : f.tjR;
            if (!present || !f.valid) {
                s.c = s.xm = s.xp = s.ym = s.yp = 0; s.flags = 0;
                s.wxm = s.wxp = s.wym = s.wyp = s.off = T(0);
                continue;
            }
            const int i = i0 + ti, j = j0 + tj;
            const bool hm = i > 0, hp = i < cd.nx - 1, vm = j > 0, vp = j < cd.ny - 1;
            s.c = S::idx(ti, tj);
            s.xm = hm ? S::idx(ti - 1, tj) : s.c;
            s.xp = hp ? S::idx(ti + 1, tj) : s.c;
            s.ym = vm ? S::idx(ti, tj - 1) : s.c;
            s.yp = vp ? S::idx(ti, tj + 1) : s.c;
            s.flags = (hm ? 1 : 0) | (hp ? 2 : 0) | (vm ? 4 : 0) | (vp ? 8 : 0) | (cd.nx > 1 ? 16 : 0) |
                      (cd.ny > 1 ? 32 : 0);
            s.wxm = g.rdx[ti + 1]; s.wxp = g.rdx[ti + 2];
            s.wym = g.rdy[tj + 1]; s.wyp = g.rdy[tj + 2];
            const T hw = f.axis == 0 ? g.hx[ti + 2] : g.hy[tj + 2];
            s.off = side == 0 ? hw : -hw;
        }
        st[fi] = o;
    }
}

// value and van Leer slopes of a staged array at a stencil cell (a: the lane's element of cell 0, cells VB apart);
// a wall-adjacent cell uses its one-sided difference
template <typename T>
__device__ __forceinline__ void slopes_at(const T* a, const FSide<T>& s, T& f0, T& sx, T& sy)
{
    f0 = a[s.c * VB];
    const T fxm = a[s.xm * VB], fxp = a[s.xp * VB], fym = a[s.ym * VB], fyp = a[s.yp * VB];
    T s1 = (f0 - fxm) * s.wxm, s2 = (fxp - f0) * s.wxp;
    if (!(s.flags & 1)) s1 = s2;
    if (!(s.flags & 2)) s2 = s1;
    sx = (s.flags & 16) ? vleer(s1, s2) : T(0);
    s1 = (f0 - fym) * s.wym;
    s2 = (fyp - f0) * s.wyp;
    if (!(s.flags & 4)) s1 = s2;
    if (!(s.flags & 8)) s2 = s1;
    sy = (s.flags & 32) ? vleer(s1, s2) : T(0);
}

// Upwind reconstruction at a face for one lane: mode 1 carried by the reconstruction (interior face, or
// incident at a wall), 2 reflected at a wall, 0 no contribution (wall velocity parallel to the wall).
template <typename T>
struct URec {
    T d0, e0, sn, st, snb, stb;
    int mode;
};

template <typename T>
__device__ __forceinline__ URec<T> recon_side(const T* sh, const T* sb, const FStencil<T>& fs, int side)
{
    const FSide<T>& s = fs.s[side];
    T fh, sxh, syh, fb, sxb, syb;
    slopes_at(sh, s, fh, sxh, syh);
    slopes_at(sb, s, fb, sxb, syb);
    URec<T> r;
    if (fs.axis == 0) { r.sn = sxh; r.st = syh; r.snb = sxb; r.stb = syb; }
    else { r.sn = syh; r.st = sxh; r.snb = syb; r.stb = sxb; }
    r.d0 = fh + r.sn * s.off;
    r.e0 = fb + r.snb * s.off;
    r.mode = 1;
    return r;
}

template <typename T>
__device__ __forceinline__ URec<T> urec(const T* sh, const T* sb, const FStencil<T>& fs, T un, bool average_ties)
{
    const bool wallf = !(fs.hasL && fs.hasR);
    // upwind side per lane without branching: the low-side cell for u_n > 0
    const int side = wallf ? (fs.hasL ? 0 : 1) : (un > T(0) ? 0 : 1);
    URec<T> o = recon_side(sh, sb, fs, side);
    if (wallf) {
        const T s = fs.hasL ? -un : un;            // u . n_in
        o.mode = s < T(0) ? 1 : (s > T(0) ? 2 : 0);
        return o;
    }
    if (average_ties && un == T(0)) {              // zero normal velocity: average of the two reconstructions
        URec<T> a = recon_side(sh, sb, fs, 0);
        o.d0 = T(0.5) * (a.d0 + o.d0); o.e0 = T(0.5) * (a.e0 + o.e0);
        o.sn = T(0.5) * (a.sn + o.sn); o.st = T(0.5) * (a.st + o.st);
        o.snb = T(0.5) * (a.snb + o.snb); o.stb = T(0.5) * (a.stb + o.stb);
    }
    return o;
}

template <typename T>
__device__ __forceinline__ T wsum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Staged region of one level: each region row is a run of consecutive cells, contiguous both in global memory
// (cell-major within a level) and in shared memory, so it moves with one bulk copy.  region_bytes() sizes the
// region of one level block; row_seg() gives the copy of one row.
template <typename T, int TX, int TY>
__device__ __forceinline__ uint32_t region_bytes(const CaseDev<T>& cd, int i0, int j0)
{
    using S = Tile<TX, TY>;
    uint32_t bytes = 0;
    for (int r = 0; r < TY + 4; ++r) {
        const int j = j0 + r - 2;
        if (j < 0 || j >= cd.ny) continue;
        int c0 = S::clo(r), c1 = S::chi(r);
        if (i0 + c0 < 0) c0 = -i0;
        if (i0 + c1 > cd.nx) c1 = cd.nx - i0;
        if (c1 > c0) bytes += (uint32_t)((c1 - c0) * VB * sizeof(T));
    }
    return bytes;
}

// Bulk copy of staged row r of one level block: global element offset within the level, shared element offset,
// bytes; false if the row lies outside the domain.
template <typename T, int TX, int TY>
__device__ __forceinline__ bool row_seg(int nx, int ny, int i0, int j0, int r, size_t& goff, int& soff, uint32_t& bytes)
{
    using S = Tile<TX, TY>;
    const int j = j0 + r - 2;
    if (j < 0 || j >= ny) return false;
    int c0 = S::clo(r), c1 = S::chi(r);
    if (i0 + c0 < 0) c0 = -i0;
    if (i0 + c1 > nx) c1 = nx - i0;
    if (c1 <= c0) return false;
    goff = ((size_t)j * nx + i0 + c0) * VB;
    soff = S::idx(c0, r - 2) * VB;
    bytes = (uint32_t)((c1 - c0) * VB * sizeof(T));
    return true;
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

// ------------------------------------------------------------------------------ K1: velocity sums

template <typename T, int TX, int TY, int G>
__global__ void __launch_bounds__(256) k1_tile(Batch<T> B)
{
    using S = Tile<TX, TY>;
    constexpr int NITEM = S::NF + S::NCT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bars[2];
    const int cs = find_case(B.off, B.ncases, blockIdx.x);
    const CaseDev<T>& cd = B.cases[cs];
    if (!cd.st->active) return;
    const int lb = blockIdx.x - B.off[cs];
    const int ntx = (cd.nx + TX - 1) / TX, nty = (cd.ny + TY - 1) / TY;
    const int tx = lb % ntx, ty = (lb / ntx) % nty, n = lb / (ntx * nty);
    const int i0 = tx * TX, j0 = ty * TY;
    const int nt = cd.nt, nc = cd.nc, nx = cd.nx, ny = cd.ny;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // shared memory: staged blocks [2 buffers][G][h, b][NCELL][32] | accumulators [NITEM][NM] | stencils | geometry
    constexpr size_t blk = (size_t)S::NCELL * VB;
    T* buf = reinterpret_cast<T*>(smem_raw);
    T* acc = buf + 2 * G * 2 * blk;
    FStencil<T>* fst = reinterpret_cast<FStencil<T>*>(smem_raw + round16((2 * G * 2 * blk + NITEM * NM) * sizeof(T)));
    TileGeo<T, TX, TY>* geo = reinterpret_cast<TileGeo<T, TX, TY>*>(fst + S::NF);
    for (int k = threadIdx.x; k < NITEM * NM; k += blockDim.x) acc[k] = T(0);
    load_geo<T, TX, TY>(cd, i0, j0, *geo);
    mbar_setup(bars, 2);
    build_stencils<T, TX, TY>(cd, *geo, i0, j0, fst);
    const int p = cd.st->parity;
    const T* gh = cd.dh[p];
    const T* gb = cd.db[p];
    const int nchunk = (cd.nvb + G - 1) / G, nvb = cd.nvb;
    const T* __restrict__ tu = cd.tu;
    const T* __restrict__ tv = cd.tv;
    const T* __restrict__ tw = cd.tw;
    int* err = cd.err;
    const uint32_t rbytes = region_bytes<T, TX, TY>(cd, i0, j0);
    // staged copies of chunk k (G velocity blocks of level n, h and b), issued by the lanes of warp 0
    auto issue = [&](int k) {
        const int vb0 = k * G;
        const int gk = min(G, nvb - vb0);
        T* dst = buf + (size_t)(k & 1) * G * 2 * blk;
        if (lane == 0) mbar_arrive_expect(&bars[k & 1], (uint32_t)(2 * gk) * rbytes);
        __syncwarp();
        for (int q = lane; q < gk * 2 * (TY + 4); q += 32) {
            const int r = q % (TY + 4), ga = q / (TY + 4);   // ga = 2 g + array
            size_t goff;
            int soff;
            uint32_t bytes;
            if (!row_seg<T, TX, TY>(nx, ny, i0, j0, r, goff, soff, bytes)) continue;
            const size_t src = ((size_t)(vb0 + (ga >> 1)) * nt + n) * nc * VB + goff;
            bulk_g2s(dst + (size_t)ga * blk + soff, ((ga & 1) ? gb : gh) + src, bytes, &bars[k & 1]);
        }
    };
    if (warp == 0) issue(0);
    for (int k = 0; k < nchunk; ++k) {
        if (warp == 0 && k + 1 < nchunk) issue(k + 1);
        const int fail = !mbar_wait(&bars[k & 1], (uint32_t)((k >> 1) & 1), err);
        if (__syncthreads_or(fail)) return;
        const T* cb = buf + (size_t)(k & 1) * G * 2 * blk;
        const int vb0 = k * G;
        const int gk = min(G, nvb - vb0);
        for (int item = warp; item < NITEM; item += blockDim.x >> 5) {
            T a[NM];
#pragma unroll
            for (int q = 0; q < NM; ++q) a[q] = T(0);
            if (item < S::NF) {
                const FStencil<T>& fs = fst[item];
                if (!fs.valid) continue;
                for (int g = 0; g < gk; ++g) {
                    const int av = (vb0 + g) * VB + lane;
                    const T u = tu[av], v = tv[av], w = tw[av];
                    const T un = fs.axis == 0 ? u : v, ut = fs.axis == 0 ? v : u;
                    const URec<T> r = urec(cb + (size_t)(2 * g) * blk + lane, cb + (size_t)(2 * g + 1) * blk + lane,
                                           fs, un, true);
                    const T u2 = u * u + v * v;
                    const T wst = w * r.st;
                    a[13] += wst;
                    a[14] += wst * u;
                    a[15] += wst * v;
                    a[16] += wst * u2;
                    a[17] += w * r.stb;
                    if (r.mode == 1) {
                        const T wd = w * r.d0, we = w * r.e0;
                        const T wdu = wd * u, wdv = wd * v;
                        const T wduu = wdu * u, wdvv = wdv * v;
                        a[0] += wd;
                        a[1] += wdu;
                        a[2] += wdv;
                        a[3] += wduu;
                        a[4] += wdu * v;
                        a[5] += wdvv;
                        a[6] += wduu * u;
                        a[7] += wduu * v;
                        a[8] += wdvv * u;
                        a[9] += wdvv * v;
                        a[10] += we;
                        a[11] += we * u;
                        a[12] += we * v;
                        const T wus = w * un * (un * r.sn + ut * r.st);
                        a[18] += wus;
                        a[19] += wus * u;
                        a[20] += wus * v;
                        a[21] += wus * u2;
                        a[22] += w * un * (un * r.snb + ut * r.stb);
                    }
                }
#pragma unroll
                for (int q = 0; q < NM; ++q) {
                    const T sm = wsum(a[q]);
                    if (lane == 0) acc[item * NM + q] += sm;
                }
            } else {
                const int ct = item - S::NF;
                const int ti = ct % TX, tj = ct / TX;
                if (i0 + ti >= nx || j0 + tj >= ny) continue;
                const int ci = S::idx(ti, tj);
                for (int g = 0; g < gk; ++g) {
                    const int av = (vb0 + g) * VB + lane;
                    const T u = tu[av], v = tv[av], w = tw[av];
                    const T wd = w * cb[(size_t)(2 * g) * blk + ci * VB + lane];
                    const T we = w * cb[(size_t)(2 * g + 1) * blk + ci * VB + lane];
                    const T wdu = wd * u, wdv = wd * v;
                    const T wduu = wdu * u, wdvv = wdv * v;
                    a[0] += wd;
                    a[1] += wdu;
                    a[2] += wdv;
                    a[3] += wduu;
                    a[4] += wdu * v;
                    a[5] += wdvv;
                    a[6] += wduu * u;
                    a[7] += wduu * v;
                    a[8] += wdvv * u;
                    a[9] += wdvv * v;
                    a[10] += we;
                    a[11] += we * u;
                    a[12] += we * v;
                }
#pragma unroll
                for (int q = 0; q < NCM; ++q) {
                    const T sm = wsum(a[q]);
                    if (lane == 0) acc[item * NM + q] += sm;
                }
            }
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < NITEM * NM; k += blockDim.x) {
        const int item = k / NM, m = k - item * NM;
        if (item < S::NF) {
            const FStencil<T>& fs = fst[item];
            if (fs.valid) cd.fmom[((size_t)fs.gface * nt + n) * NM + m] = (double)acc[k];
        } else if (m < NCM) {
            const int ct = item - S::NF;
            const int i = i0 + ct % TX, j = j0 + ct / TX;
            if (i < nx && j < ny) cd.cmom[((size_t)(j * nx + i) * nt + n) * NCM + m] = (double)acc[k];
        }
    }
}

template <typename T, int TX, int TY, int G>
constexpr size_t k1_smem()
{
    using S = Tile<TX, TY>;
    return round16(((size_t)2 * G * 2 * S::NCELL * VB + (S::NF + S::NCT) * NM) * sizeof(T)) +
           S::NF * sizeof(FStencil<T>) + sizeof(TileGeo<T, TX, TY>);
}

// ------------------------------------------------------------------------------ K4: micro update

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(256) k4_tile(Batch<T> B)
{
    using S = Tile<TX, TY>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar[1];
    const int cs = find_case(B.off, B.ncases, blockIdx.x);
    const CaseDev<T>& cd = B.cases[cs];
    if (!cd.st->active) return;
    const int lb = blockIdx.x - B.off[cs];
    const int ntx = (cd.nx + TX - 1) / TX, nty = (cd.ny + TY - 1) / TY;
    const int tx = lb % ntx, ty = (lb / ntx) % nty, vb = lb / (ntx * nty);
    const int i0 = tx * TX, j0 = ty * TY;
    const int nt = cd.nt, nc = cd.nc, nx = cd.nx, ny = cd.ny, nh = cd.nh, nu = cd.nu;
    const int nuv = cd.nu + cd.nv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    // shared memory: staged h and b [level][NCELL][32] each | face fluxes of one level [NF][32] x 2 | stencils | geo
    constexpr size_t blk = (size_t)S::NCELL * VB;
    T* sh = reinterpret_cast<T*>(smem_raw);
    T* sb = sh + (size_t)nt * blk;
    T* fh = sb + (size_t)nt * blk;
    T* fb = fh + (size_t)S::NF * VB;
    FStencil<T>* fst =
        reinterpret_cast<FStencil<T>*>(smem_raw + round16(((size_t)2 * nt * blk + 2 * S::NF * VB) * sizeof(T)));
    TileGeo<T, TX, TY>* geo = reinterpret_cast<TileGeo<T, TX, TY>*>(fst + S::NF);
    mbar_setup(bar, 1);
    const int p = cd.st->parity;
    if (warp == 0) {
        // staged copies of every level of h and b, issued by the lanes of warp 0
        if (lane == 0) mbar_arrive_expect(bar, (uint32_t)(2 * nt) * region_bytes<T, TX, TY>(cd, i0, j0));
        __syncwarp();
        const T* gh = cd.dh[p];
        const T* gb = cd.db[p];
        for (int q = lane; q < 2 * nt * (TY + 4); q += 32) {
            const int r = q % (TY + 4), na = q / (TY + 4);   // na = 2 n + array
            size_t goff;
            int soff;
            uint32_t bytes;
            if (!row_seg<T, TX, TY>(nx, ny, i0, j0, r, goff, soff, bytes)) continue;
            const int n = na >> 1;
            const size_t src = ((size_t)vb * nt + n) * nc * VB + goff;
            bulk_g2s(((na & 1) ? sb : sh) + (size_t)n * blk + soff, ((na & 1) ? gb : gh) + src, bytes, bar);
        }
    }
    load_geo<T, TX, TY>(cd, i0, j0, *geo);
    __syncthreads();
    build_stencils<T, TX, TY>(cd, *geo, i0, j0, fst);
    T* oh = cd.dh[p ^ 1];
    T* ob = cd.db[p ^ 1];
    const int av = vb * VB + lane;
    const T u = cd.tu[av], v = cd.tv[av], href = cd.thref[av];
    const int iu = cd.viu[av], iv = cd.viv[av];
    T et[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) et[d] = cd.et[d];
    const T* __restrict__ fpar = cd.fpar;
    const T* __restrict__ ftab = cd.ftab;
    const T* __restrict__ wtab = cd.wtab;
    const T* __restrict__ cpar = cd.cpar;
    const T* __restrict__ ctab = cd.ctab;
    const bool shakhov = cd.shakhov != 0;
    const int fail = !mbar_wait(bar, 0u, cd.err);
    if (__syncthreads_or(fail)) return;
    for (int n = 0; n < nt; ++n) {
        const T* shn = sh + (size_t)n * blk + lane;
        const T* sbn = sb + (size_t)n * blk + lane;
        // ---- face fluxes of level n (Eq. micro_flux, delta form, divided by dG_f)
        for (int fi = warp; fi < S::NF; fi += nwarp) {
            const FStencil<T>& fs = fst[fi];
            if (!fs.valid) continue;
            const T un = fs.axis == 0 ? u : v, ut = fs.axis == 0 ? v : u;
            const T* fp = fpar + ((size_t)fs.gface * nt + n) * NP;
            T Hf = T(0), Bf = T(0);
            const URec<T> r = urec(shn, sbn, fs, un, false);
            if (r.mode == 1 && un != T(0)) {
                T sc[8];
                ldv<8>(fp + F_RM1, sc);        // r - 1, r, 1/(2 lam), 1/(2 lam) - 1/(2 lam0), C1', C4', C5', nin
                const T* tb = ftab + ((size_t)fs.gface * nt + n) * nuv;
                const T ex = tb[iu], ey = tb[nu + iv];
                const T E = ex + ey + ex * ey;
                const T dH = href * (sc[0] + sc[1] * E);
                const T H = href + dH;
                const T i2l = sc[2];
                const T dB = dH * i2l + href * sc[3];
                const bool pos = un > T(0);
                T q[12], l[4];
                ldv<12>(fp + (pos ? F_QL : F_QR), q);
                ldv<4>(fp + (pos ? F_LBL : F_LBR), l);
                const T Q = cubic(q, u, v);
                const T Qb = Q + l[0] + l[1] * u + l[2] * v;
                Hf = un * (sc[4] * dH + H * Q + sc[5] * r.d0 + sc[6] * (un * r.sn + ut * r.st));
                Bf = un * (sc[4] * dB + H * i2l * Qb + sc[5] * r.e0 + sc[6] * (un * r.snb + ut * r.stb));
            } else if (r.mode == 2) {
                T wp[4];
                ldv<4>(fp + F_WRM1, wp);
                const T* tb = wtab + ((size_t)fs.wall * nt + n) * nuv;
                const T ex = tb[iu], ey = tb[nu + iv];
                const T E = ex + ey + ex * ey;
                const T dHw = href * (wp[0] + wp[1] * E);
                Hf = un * dHw;
                Bf = un * (dHw * wp[2] + href * wp[3]);
            }
            fh[fi * VB + lane] = Hf;
            fb[fi * VB + lane] = Bf;
        }
        __syncthreads();
        // ---- cell update of level n (Eq. fv_h with the spectral source, delta form)
        for (int ct = warp; ct < S::NCT; ct += nwarp) {
            const int ti = ct % TX, tj = ct / TX;
            const int i = i0 + ti, j = j0 + tj;
            if (i >= nx || j >= ny) continue;
            const int c = j * nx + i;
            const T* cp = cpar + ((size_t)c * nt + n) * NCP;
            const T* hc = sh + (size_t)S::idx(ti, tj) * VB + lane;     // level m at hc[m * blk]
            const T* bc = sb + (size_t)S::idx(ti, tj) * VB + lane;
            const int fL = tj * (TX + 1) + ti, fB = S::NXF + tj * TX + ti;
            const T dxh = fh[(fL + 1) * VB + lane] - fh[fL * VB + lane];
            const T dyh = fh[(fB + TX) * VB + lane] - fh[fB * VB + lane];
            const T dxb = fb[(fL + 1) * VB + lane] - fb[fL * VB + lane];
            const T dyb = fb[(fB + TX) * VB + lane] - fb[fB * VB + lane];
            T eh = T(0), eb = T(0);
#pragma unroll
            for (int d = 1; d < 8; ++d) {
                if (d > nh) break;
                int nm = n - d; if (nm < 0) nm += nt;
                int np = n + d; if (np >= nt) np -= nt;
                eh += et[d] * (hc[nm * blk] - hc[np * blk]);
                eb += et[d] * (bc[nm * blk] - bc[np * blk]);
            }
            // equilibria of W^{k+1} (slot 1) and W^k (slot 0): dH = H - H_ref from the cell table, Shakhov cubic
            const T* tb = ctab + ((size_t)c * nt + n) * 2 * nuv;
            T dhp[2], dbp[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                T q[20];
                ldv<20>(cp + (e == 0 ? C_EQ0 : C_EQ1), q);
                const T ex = tb[e * nuv + iu], ey = tb[e * nuv + nu + iv];
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
            T k[8];
            ldv<8>(cp + C_KSELF, k);           // kself, kE, kp1, kp0, kdx, kdy
            const T h0 = hc[n * blk], b0 = bc[n * blk];
            const size_t o = sidx(nc, nt, vb, c, n, lane);
            oh[o] = k[0] * h0 - k[4] * dxh - k[5] * dyh - k[1] * eh + k[2] * dhp[1] + k[3] * dhp[0];
            ob[o] = k[0] * b0 - k[4] * dxb - k[5] * dyb - k[1] * eb + k[2] * dbp[1] + k[3] * dbp[0];
        }
        __syncthreads();
    }
}

template <typename T, int TX, int TY>
size_t k4_smem(int nt)
{
    using S = Tile<TX, TY>;
    return round16(((size_t)2 * S::NCELL * nt * VB + (size_t)2 * S::NF * VB) * sizeof(T)) +
           S::NF * sizeof(FStencil<T>) + sizeof(TileGeo<T, TX, TY>);
}

}  // namespace hb
