// mhd_kernels.cuh -- kernels of one VL / CTU + CT step on a batch of periodic
// boxes (one box is the batch of one).
//
// HBM layout (structure of arrays).  Every box's cells are concatenated:
// box b owns cells [off_b, off_b + n_b) of every field array, x fastest
// inside a box (c = off + (k*ny + j)*nx + i).  Field f of an array starts at
// f * N, N the total cell count of the batch.
//   state   rho, Mx, My, Mz (type TU), e (type TE), Bx, By, Bz (type TE);
//           B_d[c] is the face c - 1/2 e_d (Eq. 14), no duplicated face.
//   W       8 primitives (R): rho, vx, vy, vz, P, Bx, By, Bz (cell centre).
//   F[d]    7 flux components per face, sweep frame of axis d (R).
//   E[c]    edge field along axis c at the lower (a,b) corner, a=c+1, b=c+2
//           (Ez at (i-1/2,j-1/2,k), Ex at (i,j-1/2,k-1/2), Ey at (i-1/2,j,k-1/2)).
//   WM/WP   CTU traced face states (7 per cell per axis, R).
// Per-cell kernels run one thread per cell over "virtual blocks" of 256
// cells that never straddle two boxes; the sweeps run a persistent grid over
// the batch's list of face tiles.
#pragma once
#include <stdint.h>
#include "mhd_dev.cuh"

namespace mhd {

constexpr int CELL_THREADS = 256;
constexpr int TX = 32;             // sweep tile extent along x
constexpr int SWEEP_THREADS = 256;
constexpr int TL_MAX = 16;         // largest tile extent along the second tiled axis

struct BoxDev {
    int nx, ny, nz, pad;
    long long off;      // first cell of the box in the batch arrays
    long long n;        // cells of the box
    long long vblk0;    // first virtual block of the box
    double dx;
    int tile0[3];       // first sweep tile of the box, per axis
    float inv_dx;       // 1/dx in single precision
};

// dt of a box and its ratios to dx, in both precisions; written once per
// step so that no kernel divides by dx (FP64 is slow on this part)
struct DtBox {
    double dt, hdt, dtdx, hdtdx;
    float fdt, fhdt, fdtdx, fhdtdx;
};

template <class T> struct DtOf;
template <> struct DtOf<double> {
    static __device__ __forceinline__ double dt(const DtBox& d) { return d.dt; }
    static __device__ __forceinline__ double hdt(const DtBox& d) { return d.hdt; }
    static __device__ __forceinline__ double dtdx(const DtBox& d) { return d.dtdx; }
    static __device__ __forceinline__ double hdtdx(const DtBox& d) { return d.hdtdx; }
};
template <> struct DtOf<float> {
    static __device__ __forceinline__ float dt(const DtBox& d) { return d.fdt; }
    static __device__ __forceinline__ float hdt(const DtBox& d) { return d.fhdt; }
    static __device__ __forceinline__ float dtdx(const DtBox& d) { return d.fdtdx; }
    static __device__ __forceinline__ float hdtdx(const DtBox& d) { return d.fhdtdx; }
};

__device__ __forceinline__ void write_dtbox(DtBox* o, double dt, double dx)
{
    DtBox d;
    d.dt = dt;
    d.hdt = 0.5 * dt;
    d.dtdx = dt / dx;
    d.hdtdx = 0.5 * d.dtdx;   // = (dt/2)/dx exactly: halving commutes with rounding
    d.fdt = (float)d.dt;
    d.fhdt = (float)d.hdt;
    d.fdtdx = (float)d.dtdx;
    d.fhdtdx = (float)d.hdtdx;
    *o = d;
}

struct Boxes {
    const BoxDev* b;    // device table, nbox entries
    int nbox;
    int tl;             // sweep tile extent along the second tiled axis
    long long N;        // cells of the batch (field stride)
    long long nvblk;    // virtual blocks of the batch
    int ntile[3];       // sweep tiles of the batch, per axis
    int pad;
};

template <class TU, class TE> struct StateP {
    TU* rho;
    TU* m[3];
    TE* e;
    TE* b[3];
};

// periodic wrap; one add or subtract for offsets within a period, the
// modulo only for the rare larger ones (boxes thinner than the stencil)
__device__ __forceinline__ int wrapi(int i, int n)
{
    if (i < 0) i += n;
    else if (i >= n) i -= n;
    if ((unsigned)i >= (unsigned)n) {
        i %= n;
        if (i < 0) i += n;
    }
    return i;
}

__device__ __forceinline__ long long cell_of(const BoxDev& g, int i, int j, int k)
{
    return g.off + ((long long)k * g.ny + j) * g.nx + i;
}

// neighbour of (i,j,k) shifted by s along axis d (periodic in the box)
__device__ __forceinline__ long long nbr(const BoxDev& g, int i, int j, int k, int d, int s)
{
    if (d == 0) i = wrapi(i + s, g.nx);
    else if (d == 1) j = wrapi(j + s, g.ny);
    else k = wrapi(k + s, g.nz);
    return cell_of(g, i, j, k);
}

// (i, j, k) of the local cell index lc (< 2^31 cells per box): 32-bit division
__device__ __forceinline__ void coords(const BoxDev& g, long long lc, int& i, int& j, int& k)
{
    const unsigned u = (unsigned)lc, nx = (unsigned)g.nx, ny = (unsigned)g.ny;
    const unsigned t = u / nx;
    const unsigned kk = t / ny;
    i = (int)(u - t * nx);
    j = (int)(t - kk * ny);
    k = (int)kk;
}

// box of a virtual block / of a sweep tile (binary search, block-uniform)
__device__ __forceinline__ int box_of_vblk(const Boxes& B, long long v)
{
    int lo = 0, hi = B.nbox - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (B.b[mid].vblk0 <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int box_of_tile(const Boxes& B, int d, int t)
{
    int lo = 0, hi = B.nbox - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (B.b[mid].tile0[d] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <class R>
__device__ __forceinline__ void load_rot(const R* __restrict__ W, long long N, long long c, int d, R w[7], R& bn)
{
    const int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
    w[0] = W[c];
    w[1] = W[(1 + d) * N + c];
    w[2] = W[(1 + t1) * N + c];
    w[3] = W[(1 + t2) * N + c];
    w[4] = W[4 * N + c];
    w[5] = W[(5 + t1) * N + c];
    w[6] = W[(5 + t2) * N + c];
    bn = W[(5 + d) * N + c];
}

// positive doubles order like unsigned integers: max-reduce their bits
__device__ __forceinline__ void atomic_max_pos(unsigned long long* p, double v)
{
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------
// a1 + a2: primitives of every cell, the per-box CFL signal-speed maximum and
// a record of the first cell with rho <= 0 or P <= 0 (or not finite).
// ---------------------------------------------------------------------------
template <class R, class TU, class TE>
__global__ void __launch_bounds__(CELL_THREADS) k_prim(Boxes B, StateP<TU, TE> s, R* __restrict__ W, double gam,
                                                       double* smax_part, unsigned long long* bad_cell,
                                                       double pfloor = 0.0, unsigned long long* nfloor = nullptr)
{
    const long long N = B.N;
    __shared__ double red[CELL_THREADS];
    for (long long v = blockIdx.x; v < B.nvblk; v += gridDim.x) {
        const int bi = box_of_vblk(B, v);
        const BoxDev g = B.b[bi];
        const long long lc = (v - g.vblk0) * CELL_THREADS + threadIdx.x;
        double local = 0.0;
        if (lc < g.n) {
            int i, j, k;
            coords(g, lc, i, j, k);
            const long long c = g.off + lc;
            TE bx = TE(0.5) * (s.b[0][c] + s.b[0][nbr(g, i, j, k, 0, 1)]);
            TE by = TE(0.5) * (s.b[1][c] + s.b[1][nbr(g, i, j, k, 1, 1)]);
            TE bz = TE(0.5) * (s.b[2][c] + s.b[2][nbr(g, i, j, k, 2, 1)]);
            TE rho = TE(s.rho[c]);
            TE mx = TE(s.m[0][c]), my = TE(s.m[1][c]), mz = TE(s.m[2][c]);
            TE vx = mx / rho, vy = my / rho, vz = mz / rho;
            // pressure recovery in the precision of the stored energy
            TE p = TE(gam - 1.0) * (s.e[c] - TE(0.5) * rho * (vx * vx + vy * vy + vz * vz)
                                    - TE(0.5) * (bx * bx + by * by + bz * bz));
            if (pfloor > 0.0 && p < TE(pfloor)) {
                // optional pressure floor.  At the start of a step (nfloor given)
                // e is raised so that P = pfloor (not conservative); read-only
                // passes only use the floored value.
                if (nfloor) {
                    s.e[c] = s.e[c] + (TE(pfloor) - p) / TE(gam - 1.0);
                    atomicAdd(nfloor, 1ull);
                }
                p = TE(pfloor);
            }
            R w[8] = {R(rho), R(vx), R(vy), R(vz), R(p), R(bx), R(by), R(bz)};
#pragma unroll
            for (int f = 0; f < 8; f++) W[f * N + c] = w[f];
            if (!(w[0] > R(0)) || !(w[4] > R(0))) atomicMin(bad_cell, (unsigned long long)c);
            if (smax_part) {
                R a2 = R(gam) * w[4] / w[0];
                R sm = R(0);
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    const int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
                    R cf = fast_speed(w[0], a2, w[5 + d], w[5 + t1], w[5 + t2]);
                    sm = rmax(sm, Num<R>::abs_(w[1 + d]) + cf);
                }
                local = (double)sm;
            }
        }
        if (smax_part) {
            // virtual-block maximum (the block lies in one box); no atomics
            red[threadIdx.x] = local;
            __syncthreads();
            for (int o = CELL_THREADS / 2; o > 0; o >>= 1) {
                if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
                __syncthreads();
            }
            if (threadIdx.x == 0) smax_part[v] = red[0];
            __syncthreads();
        }
    }
}

// dt of every box from the maxima of its virtual blocks (one block per box)
static __global__ void k_finalize_dt(Boxes B, const double* __restrict__ smax_part, double cfl, double* dt,
                                     double* smax_box, DtBox* dtb)
{
    const int b = blockIdx.x;
    if (b >= B.nbox) return;
    const long long v0 = B.b[b].vblk0;
    const long long v1 = b + 1 < B.nbox ? B.b[b + 1].vblk0 : B.nvblk;
    __shared__ double red[256];
    double m = 0.0;
    for (long long v = v0 + threadIdx.x; v < v1; v += blockDim.x) m = fmax(m, smax_part[v]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double sm = red[0];
        if (smax_box) smax_box[b] = sm;
        const double d = sm > 0.0 ? cfl * B.b[b].dx / sm : 0.0;
        if (dt) dt[b] = d;
        if (dtb) write_dtbox(dtb + b, d, B.b[b].dx);
    }
}

// dt of every box from a host value (v > 0) or from dt[] (v <= 0)
static __global__ void k_set_dt(Boxes B, double* dt, double v, DtBox* dtb)
{
    for (int b = threadIdx.x; b < B.nbox; b += blockDim.x) {
        if (v > 0.0) dt[b] = v;
        write_dtbox(dtb + b, dt[b], B.b[b].dx);
    }
}

// ---------------------------------------------------------------------------
// Sweep along axis d over tiles of faces: reconstruct every cell of the tile
// (plus one cell below it along d) once into shared memory, then solve one
// Riemann problem per face.  Persistent: the grid loops over the batch's
// tiles.  MODE 0: first-order states (VL predictor); MODE 1: reconstruction
// (VL corrector); MODE 2: reconstruction + tracing + the d B_n/dn source
// terms (CTU predictor), the traced states also kept in HBM for the
// transverse correction.
// ---------------------------------------------------------------------------
struct Tile {
    int ex, ey, ez;      // tile extents (faces)
    int rx, ry, rz;      // reconstruction region (tile + 1 below along d)
    int sx, sy, sz;      // slope region (region + 1 on both sides along d)
};

// The reconstruction region is always TX x tl cells (x by the second tiled
// axis), so with tl = 8 one 256-thread pass reconstructs it exactly; the
// tile of faces is the region minus its first cell row along d.
__host__ __device__ __forceinline__ Tile tile_of(int d, int tl)
{
    Tile t;
    t.rx = TX;
    t.ry = d == 2 ? 1 : tl;
    t.rz = d == 2 ? tl : 1;
    t.ex = t.rx - (d == 0);
    t.ey = t.ry - (d == 1);
    t.ez = t.rz - (d == 2);
    t.sx = t.rx + 2 * (d == 0);
    t.sy = t.ry + 2 * (d == 1);
    t.sz = t.rz + 2 * (d == 2);
    return t;
}

inline int tiles_of_box(int nx, int ny, int nz, int d, int tl)
{
    Tile t = tile_of(d, tl);
    return ((nx + t.ex - 1) / t.ex) * ((ny + t.ey - 1) / t.ey) * ((nz + t.ez - 1) / t.ez);
}

template <class R>
size_t sweep_smem_bytes(int recon, int tl)
{
    size_t region = (size_t)TX * tl;
    size_t slopes = (size_t)((TX + 2) * tl > TX * (tl + 2) ? (TX + 2) * tl : TX * (tl + 2));
    size_t b = region * 14 * sizeof(R);
    if (recon == PPM) b += slopes * 7 * sizeof(R);
    return b;
}

template <class R, int RECON, int SOLVER, int MODE, class TE>
__global__ void __launch_bounds__(SWEEP_THREADS) k_sweep(Boxes B, int d, const R* __restrict__ W,
                                                         const TE* __restrict__ Bd, R* __restrict__ F,
                                                         R* __restrict__ WMg, R* __restrict__ WPg,
                                                         const DtBox* __restrict__ dtb, double gam,
                                                         const int* __restrict__ tile_list = nullptr,
                                                         const int* __restrict__ tile_count = nullptr)
{
    extern __shared__ unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);
    const long long N = B.N;
    const Tile t = tile_of(d, B.tl);
    const R gr = R(gam), gm1 = R(gam - 1.0);
    const int nreg = t.rx * t.ry * t.rz;
    R* SMs = sm;                 // [nreg][7] state on the cell's face -1/2
    R* SPs = sm + nreg * 7;      // [nreg][7] state on the cell's face +1/2
    R* DWs = sm + nreg * 14;     // [nslope][7] PPM slopes

    // all tiles of the batch, or only those of a list (the learned selector's)
    const int ntile = tile_list ? *tile_count : B.ntile[d];
    for (int it = blockIdx.x; it < ntile; it += gridDim.x) {
        const int tile = tile_list ? tile_list[it] : it;
        const int bi = box_of_tile(B, d, tile);
        const BoxDev g = B.b[bi];
        const int ntx = (g.nx + t.ex - 1) / t.ex;
        const int nty = (g.ny + t.ey - 1) / t.ey;
        int bl = tile - g.tile0[d];
        const int tx = bl % ntx; bl /= ntx;
        const int ty = bl % nty; bl /= nty;
        const int tz = bl;
        const int x0 = tx * t.ex, y0 = ty * t.ey, z0 = tz * t.ez;
        const R dtdx = MODE == 2 ? DtOf<R>::dtdx(dtb[bi]) : R(0);

        if (MODE != 0) {
            // region origin: one cell below the tile along d
            const int ox = x0 - (d == 0), oy = y0 - (d == 1), oz = z0 - (d == 2);
            if (RECON == PPM) {
                const int nsl = t.sx * t.sy * t.sz;
                const int sx0 = ox - (d == 0), sy0 = oy - (d == 1), sz0 = oz - (d == 2);
                for (int q = threadIdx.x; q < nsl; q += blockDim.x) {
                    int qx = q % t.sx, qy = (q / t.sx) % t.sy, qz = q / (t.sx * t.sy);
                    int i = wrapi(sx0 + qx, g.nx), j = wrapi(sy0 + qy, g.ny), k = wrapi(sz0 + qz, g.nz);
                    R wm[7], w0[7], wp[7], bn, bdum;
                    load_rot(W, N, cell_of(g, i, j, k), d, w0, bn);
                    load_rot(W, N, nbr(g, i, j, k, d, -1), d, wm, bdum);
                    load_rot(W, N, nbr(g, i, j, k, d, 1), d, wp, bdum);
                    R dw[7];
                    char_slope(wm, w0, wp, bn, gr, dw);
#pragma unroll
                    for (int m = 0; m < 7; m++) DWs[q * 7 + m] = dw[m];
                }
                __syncthreads();
            }
            for (int q = threadIdx.x; q < nreg; q += blockDim.x) {
                int qx = q % t.rx, qy = (q / t.rx) % t.ry, qz = q / (t.rx * t.ry);
                int gi = ox + qx, gj = oy + qy, gk = oz + qz;
                int i = wrapi(gi, g.nx), j = wrapi(gj, g.ny), k = wrapi(gk, g.nz);
                long long c = cell_of(g, i, j, k);
                R wm1[7], w0[7], wp1[7], bn, bdum;
                load_rot(W, N, c, d, w0, bn);
                load_rot(W, N, nbr(g, i, j, k, d, -1), d, wm1, bdum);
                load_rot(W, N, nbr(g, i, j, k, d, 1), d, wp1, bdum);
                R dwm[7], dw0[7], dwp[7];
                if (RECON == PPM) {
                    // slope-region index of this cell and its two neighbours along d
                    int sxq = qx + (d == 0), syq = qy + (d == 1), szq = qz + (d == 2);
                    int sq = (szq * t.sy + syq) * t.sx + sxq;
                    int st = d == 0 ? 1 : (d == 1 ? t.sx : t.sx * t.sy);
#pragma unroll
                    for (int m = 0; m < 7; m++) {
                        dwm[m] = DWs[(sq - st) * 7 + m];
                        dw0[m] = DWs[sq * 7 + m];
                        dwp[m] = DWs[(sq + st) * 7 + m];
                    }
                }
                R wmf[7], wpf[7];
                recon_cell<RECON, MODE == 2>(wm1, w0, wp1, bn, gr, dwm, dw0, dwp, dtdx, wmf, wpf);
                if (MODE == 2) {
                    // d B_n / dn source terms of the 1-D sweep, over dt/2
                    long long cp = nbr(g, i, j, k, d, 1);
                    R dbn = sizeof(R) == 8 ? R((double)(Bd[cp] - Bd[c]) / g.dx) : R(Bd[cp] - Bd[c]) * R(g.inv_dx);
                    R hdt = DtOf<R>::hdt(dtb[bi]);
                    R vb = w0[1] * bn + w0[2] * w0[5] + w0[3] * w0[6];
                    R src[7] = {R(0), bn / w0[0], w0[5] / w0[0], w0[6] / w0[0], -gm1 * vb, w0[2], w0[3]};
#pragma unroll
                    for (int m = 0; m < 7; m++) {
                        wmf[m] = wmf[m] + hdt * src[m] * dbn;
                        wpf[m] = wpf[m] + hdt * src[m] * dbn;
                    }
                    bool own = qx >= (d == 0) && qy >= (d == 1) && qz >= (d == 2) && gi < g.nx && gj < g.ny && gk < g.nz;
                    if (own) {
#pragma unroll
                        for (int m = 0; m < 7; m++) {
                            WMg[(long long)m * N + c] = wmf[m];
                            WPg[(long long)m * N + c] = wpf[m];
                        }
                    }
                }
#pragma unroll
                for (int m = 0; m < 7; m++) {
                    SMs[q * 7 + m] = wmf[m];
                    SPs[q * 7 + m] = wpf[m];
                }
            }
            __syncthreads();
        }
        const int nface = t.ex * t.ey * t.ez;
        for (int q = threadIdx.x; q < nface; q += blockDim.x) {
            int qx = q % t.ex, qy = (q / t.ex) % t.ey, qz = q / (t.ex * t.ey);
            int i = x0 + qx, j = y0 + qy, k = z0 + qz;
            if (i >= g.nx || j >= g.ny || k >= g.nz) continue;
            long long c = cell_of(g, i, j, k);
            R wl[7], wr[7], bdum;
            if (MODE == 0) {
                load_rot(W, N, nbr(g, i, j, k, d, -1), d, wl, bdum);
                load_rot(W, N, c, d, wr, bdum);
            } else {
                // region index of this cell; the left state is the cell below's "+" state
                int rq = ((qz + (d == 2)) * t.ry + (qy + (d == 1))) * t.rx + (qx + (d == 0));
                int st = d == 0 ? 1 : (d == 1 ? t.rx : t.rx * t.ry);
#pragma unroll
                for (int m = 0; m < 7; m++) {
                    wl[m] = SPs[(rq - st) * 7 + m];
                    wr[m] = SMs[rq * 7 + m];
                }
            }
            R f[7];
            riemann<SOLVER>(wl, wr, R(Bd[c]), gm1, gr, f);
#pragma unroll
            for (int m = 0; m < 7; m++) F[(long long)m * N + c] = f[m];
        }
        if (MODE != 0) __syncthreads();   // the next tile reuses shared memory
    }
}

// ---------------------------------------------------------------------------
// a7: edge electric fields, upwinded corner average (one cell -> its three
// lower edges).  F[d] = F + d*7*N.
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R upwind(R f, R xm, R xp)
{
    if (f > R(0)) return xm;
    if (f < R(0)) return xp;
    return R(0.5) * (xm + xp);
}

template <class R>
__global__ void __launch_bounds__(CELL_THREADS) k_emf(Boxes B, const R* __restrict__ F, const R* __restrict__ W,
                                                      R* __restrict__ E)
{
    const long long N = B.N;
    for (long long v = blockIdx.x; v < B.nvblk; v += gridDim.x) {
    const BoxDev g = B.b[box_of_vblk(B, v)];
    const long long lc = (v - g.vblk0) * CELL_THREADS + threadIdx.x;
    if (lc >= g.n) continue;
    int i, j, k;
    coords(g, lc, i, j, k);
    const long long q = g.off + lc;
#pragma unroll
    for (int cax = 0; cax < 3; cax++) {
        const int a = cax == 2 ? 0 : cax + 1, bb = cax == 0 ? 2 : cax - 1;
        const R* Fa = F + (long long)a * 7 * N;
        const R* Fb = F + (long long)bb * 7 * N;
        long long c11 = q;
        long long c01 = nbr(g, i, j, k, a, -1);
        long long c10 = nbr(g, i, j, k, bb, -1);
        int i2 = i, j2 = j, k2 = k;
        if (a == 0) i2 = wrapi(i - 1, g.nx); else if (a == 1) j2 = wrapi(j - 1, g.ny); else k2 = wrapi(k - 1, g.nz);
        long long c00 = nbr(g, i2, j2, k2, bb, -1);
        R ea0 = -Fa[5 * N + c10], ea1 = -Fa[5 * N + c11];
        R eb0 = Fb[6 * N + c01], eb1 = Fb[6 * N + c11];
        R fa0 = Fa[c10], fa1 = Fa[c11];
        R fb0 = Fb[c01], fb1 = Fb[c11];
        R cc00 = -(W[(1 + a) * N + c00] * W[(5 + bb) * N + c00] - W[(1 + bb) * N + c00] * W[(5 + a) * N + c00]);
        R cc10 = -(W[(1 + a) * N + c10] * W[(5 + bb) * N + c10] - W[(1 + bb) * N + c10] * W[(5 + a) * N + c10]);
        R cc01 = -(W[(1 + a) * N + c01] * W[(5 + bb) * N + c01] - W[(1 + bb) * N + c01] * W[(5 + a) * N + c01]);
        R cc11 = -(W[(1 + a) * N + c11] * W[(5 + bb) * N + c11] - W[(1 + bb) * N + c11] * W[(5 + a) * N + c11]);
        R hib = upwind(fa1, cc01 - eb0, cc11 - eb1);
        R lob = upwind(fa0, eb0 - cc00, eb1 - cc10);
        R hia = upwind(fb1, cc10 - ea0, cc11 - ea1);
        R loa = upwind(fb0, ea0 - cc00, ea1 - cc01);
        E[cax * N + q] = R(0.25) * (ea0 + ea1 + eb0 + eb1) + R(0.25) * (lob - hib) + R(0.25) * (loa - hia);
    }
    }
}

// curl_d E on the face d of cell (i,j,k): (E_t2(+t1) - E_t2) - (E_t1(+t2) - E_t1),
// formed in the face-field type TE: every edge value is widened before the
// differences, so the four faces sharing an edge cancel exactly in div B
template <class TE, class R>
__device__ __forceinline__ TE curl_face(const BoxDev& g, long long N, const R* __restrict__ E, int i, int j, int k, int d)
{
    const int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
    long long c = cell_of(g, i, j, k);
    return (TE(E[t2 * N + nbr(g, i, j, k, t1, 1)]) - TE(E[t2 * N + c])) -
           (TE(E[t1 * N + nbr(g, i, j, k, t2, 1)]) - TE(E[t1 * N + c]));
}

// ---------------------------------------------------------------------------
// a8 + a1: half-step face field B^{n+1/2} = B^n - (dt/2) curl E (Eq. 13) and
// the half-step cell primitives from U^{n+1/2} = U^n - (dt/2) div F (Eq. 10)
// with the cell-centre B of the updated faces.  Only Bh and Wh are stored.
// ---------------------------------------------------------------------------
template <class R, class TU, class TE>
__global__ void __launch_bounds__(CELL_THREADS) k_half(Boxes B, StateP<TU, TE> s, const R* __restrict__ F,
                                                       const R* __restrict__ E, const DtBox* __restrict__ dtb,
                                                       double gam, TE* __restrict__ Bh0, TE* __restrict__ Bh1,
                                                       TE* __restrict__ Bh2, R* __restrict__ Wh, double pfloor = 0.0)
{
    const long long N = B.N;
    for (long long v = blockIdx.x; v < B.nvblk; v += gridDim.x) {
    const int bi = box_of_vblk(B, v);
    const BoxDev g = B.b[bi];
    const long long lc = (v - g.vblk0) * CELL_THREADS + threadIdx.x;
    if (lc >= g.n) continue;
    const TE r = DtOf<TE>::hdtdx(dtb[bi]);
    TE* Bh[3] = {Bh0, Bh1, Bh2};
    int i, j, k;
    coords(g, lc, i, j, k);
    const long long c = g.off + lc;
    TE bc[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        TE lo = s.b[d][c] - r * curl_face<TE>(g, N, E, i, j, k, d);
        int i2 = i, j2 = j, k2 = k;
        if (d == 0) i2 = wrapi(i + 1, g.nx); else if (d == 1) j2 = wrapi(j + 1, g.ny); else k2 = wrapi(k + 1, g.nz);
        TE hi = s.b[d][cell_of(g, i2, j2, k2)] - r * curl_face<TE>(g, N, E, i2, j2, k2, d);
        Bh[d][c] = lo;
        bc[d] = TE(0.5) * (lo + hi);
    }
    // divergence of the fluxes, sweep frames back to x, y, z
    TE du[5] = {TE(0), TE(0), TE(0), TE(0), TE(0)};
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
        const R* Fd = F + (long long)d * 7 * N;
        long long cp = nbr(g, i, j, k, d, 1);
        du[0] += TE(Fd[cp] - Fd[c]);
        du[1 + d] += TE(Fd[N + cp] - Fd[N + c]);
        du[1 + t1] += TE(Fd[2 * N + cp] - Fd[2 * N + c]);
        du[1 + t2] += TE(Fd[3 * N + cp] - Fd[3 * N + c]);
        du[4] += TE(Fd[4 * N + cp] - Fd[4 * N + c]);
    }
    TE rho = TE(s.rho[c]) - r * du[0];
    TE mx = TE(s.m[0][c]) - r * du[1], my = TE(s.m[1][c]) - r * du[2], mz = TE(s.m[2][c]) - r * du[3];
    TE e = s.e[c] - r * du[4];
    TE vx = mx / rho, vy = my / rho, vz = mz / rho;
    TE p = TE(gam - 1.0) * (e - TE(0.5) * rho * (vx * vx + vy * vy + vz * vz)
                            - TE(0.5) * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]));
    if (pfloor > 0.0 && p < TE(pfloor)) p = TE(pfloor);
    Wh[c] = R(rho); Wh[N + c] = R(vx); Wh[2 * N + c] = R(vy); Wh[3 * N + c] = R(vz);
    Wh[4 * N + c] = R(p); Wh[5 * N + c] = R(bc[0]); Wh[6 * N + c] = R(bc[1]); Wh[7 * N + c] = R(bc[2]);
    }
}

// ---------------------------------------------------------------------------
// a10: full update U^{n+1} = U^n - dt div F (Eq. 10), B^{n+1} = B^n - dt curl E
// (Eq. 13), in place.
// ---------------------------------------------------------------------------
template <class R, class TU, class TE>
__global__ void __launch_bounds__(CELL_THREADS) k_full(Boxes B, StateP<TU, TE> s, const R* __restrict__ F,
                                                       const R* __restrict__ E, const DtBox* __restrict__ dtb)
{
    const long long N = B.N;
    for (long long v = blockIdx.x; v < B.nvblk; v += gridDim.x) {
    const int bi = box_of_vblk(B, v);
    const BoxDev g = B.b[bi];
    const long long lc = (v - g.vblk0) * CELL_THREADS + threadIdx.x;
    if (lc >= g.n) continue;
    const TE r = DtOf<TE>::dtdx(dtb[bi]);
    int i, j, k;
    coords(g, lc, i, j, k);
    const long long c = g.off + lc;
    TE du[5] = {TE(0), TE(0), TE(0), TE(0), TE(0)};
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
        const R* Fd = F + (long long)d * 7 * N;
        long long cp = nbr(g, i, j, k, d, 1);
        du[0] += TE(Fd[cp] - Fd[c]);
        du[1 + d] += TE(Fd[N + cp] - Fd[N + c]);
        du[1 + t1] += TE(Fd[2 * N + cp] - Fd[2 * N + c]);
        du[1 + t2] += TE(Fd[3 * N + cp] - Fd[3 * N + c]);
        du[4] += TE(Fd[4 * N + cp] - Fd[4 * N + c]);
    }
    s.rho[c] = TU(TE(s.rho[c]) - r * du[0]);
    s.m[0][c] = TU(TE(s.m[0][c]) - r * du[1]);
    s.m[1][c] = TU(TE(s.m[1][c]) - r * du[2]);
    s.m[2][c] = TU(TE(s.m[2][c]) - r * du[3]);
    s.e[c] = s.e[c] - r * du[4];
#pragma unroll
    for (int d = 0; d < 3; d++) s.b[d][c] = s.b[d][c] - r * curl_face<TE>(g, N, E, i, j, k, d);
    }
}

// ---------------------------------------------------------------------------
// a9 + a6: CTU transverse correction of the traced states of the two cells
// on each d-face, then the corrector Riemann solve with the half-step B_n.
// ---------------------------------------------------------------------------
template <class R, int SOLVER, class TE>
__global__ void __launch_bounds__(CELL_THREADS) k_ctu_correct(Boxes B, int d, const R* __restrict__ WM,
                                                              const R* __restrict__ WP, const R* __restrict__ W,
                                                              const R* __restrict__ F1, const TE* __restrict__ Bhd,
                                                              R* __restrict__ F2, const DtBox* __restrict__ dtb,
                                                              double gam)
{
    const long long N = B.N;
    for (long long v = blockIdx.x; v < B.nvblk; v += gridDim.x) {
    const int bi = box_of_vblk(B, v);
    const BoxDev g = B.b[bi];
    const long long lc = (v - g.vblk0) * CELL_THREADS + threadIdx.x;
    if (lc >= g.n) continue;
    const int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
    const R gm1 = R(gam - 1.0), gr = R(gam);
    const R r = DtOf<R>::hdtdx(dtb[bi]);
    int i, j, k;
    coords(g, lc, i, j, k);
    const long long c = g.off + lc;
    R wf[2][7];
#pragma unroll
    for (int side = 0; side < 2; side++) {
        int si = i, sj = j, sk = k;
        if (side == 0) {
            if (d == 0) si = wrapi(i - 1, g.nx); else if (d == 1) sj = wrapi(j - 1, g.ny); else sk = wrapi(k - 1, g.nz);
        }
        long long sc = cell_of(g, si, sj, sk);
        const R* src = side == 0 ? WP : WM;
        R w[7];
#pragma unroll
        for (int m = 0; m < 7; m++) w[m] = src[(long long)m * N + sc];
        // global-frame conserved state with the cell-centre B_n of the cell
        R v[3], bg[3];
        v[d] = w[1]; v[t1] = w[2]; v[t2] = w[3];
        bg[d] = W[(5 + d) * N + sc]; bg[t1] = w[5]; bg[t2] = w[6];
        R q[8];
        q[0] = w[0];
        q[1] = w[0] * v[0]; q[2] = w[0] * v[1]; q[3] = w[0] * v[2];
        q[4] = w[4] / gm1 + R(0.5) * w[0] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2])
               + R(0.5) * (bg[0] * bg[0] + bg[1] * bg[1] + bg[2] * bg[2]);
        q[5] = bg[0]; q[6] = bg[1]; q[7] = bg[2];
#pragma unroll
        for (int mm = 0; mm < 2; mm++) {
            const int e = mm == 0 ? t1 : t2;
            const int e1 = e == 2 ? 0 : e + 1, e2 = e == 0 ? 2 : e - 1;
            const R* Fe = F1 + (long long)e * 7 * N;
            long long sp = nbr(g, si, sj, sk, e, 1);
            R df[7];
#pragma unroll
            for (int m = 0; m < 7; m++) df[m] = Fe[(long long)m * N + sp] - Fe[(long long)m * N + sc];
            q[0] -= r * df[0];
            q[1 + e] -= r * df[1];
            q[1 + e1] -= r * df[2];
            q[1 + e2] -= r * df[3];
            q[4] -= r * df[4];
            q[5 + e1] -= r * df[5];
            q[5 + e2] -= r * df[6];
        }
        R rho = q[0];
        R vx = q[1] / rho, vy = q[2] / rho, vz = q[3] / rho;
        R p = gm1 * (q[4] - R(0.5) * rho * (vx * vx + vy * vy + vz * vz)
                     - R(0.5) * (q[5] * q[5] + q[6] * q[6] + q[7] * q[7]));
        R vg[3] = {vx, vy, vz};
        wf[side][0] = rho;
        wf[side][1] = vg[d];
        wf[side][2] = vg[t1];
        wf[side][3] = vg[t2];
        wf[side][4] = p;
        wf[side][5] = q[5 + t1];
        wf[side][6] = q[5 + t2];
    }
    R f[7];
    riemann<SOLVER>(wf[0], wf[1], R(Bhd[c]), gm1, gr, f);
#pragma unroll
    for (int m = 0; m < 7; m++) F2[(long long)m * N + c] = f[m];
    }
}

// ---------------------------------------------------------------------------
// a11: per virtual block: |div B| dx maximum, sum of |B_cc|^2 and sums of
// the conserved fields; finished per box in fixed order by k_finish_diag.
// ---------------------------------------------------------------------------
template <class TU, class TE>
__global__ void __launch_bounds__(CELL_THREADS) k_diag(Boxes B, StateP<TU, TE> s, double* __restrict__ part)
{
    // part: [nvblk][10]: maxdiv, sum b2, rho, mx, my, mz, e, bx, by, bz
    __shared__ double red[CELL_THREADS];
    for (long long v = blockIdx.x; v < B.nvblk; v += gridDim.x) {
    const BoxDev g = B.b[box_of_vblk(B, v)];
    const long long lc = (v - g.vblk0) * CELL_THREADS + threadIdx.x;
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (lc < g.n) {
        int i, j, k;
        coords(g, lc, i, j, k);
        const long long c = g.off + lc;
        double dv = 0.0, b2 = 0.0;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            double bp = (double)s.b[d][nbr(g, i, j, k, d, 1)], b0 = (double)s.b[d][c];
            dv += bp - b0;
            double bcc = 0.5 * (bp + b0);
            b2 += bcc * bcc;
        }
        acc[0] = fabs(dv);
        acc[1] = b2;
        acc[2] = (double)s.rho[c];
        acc[3] = (double)s.m[0][c];
        acc[4] = (double)s.m[1][c];
        acc[5] = (double)s.m[2][c];
        acc[6] = (double)s.e[c];
        acc[7] = (double)s.b[0][c];
        acc[8] = (double)s.b[1][c];
        acc[9] = (double)s.b[2][c];
    }
    for (int f = 0; f < 10; f++) {
        red[threadIdx.x] = acc[f];
        __syncthreads();
        for (int o = CELL_THREADS / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o)
                red[threadIdx.x] = f == 0 ? fmax(red[threadIdx.x], red[threadIdx.x + o]) : red[threadIdx.x] + red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[v * 10 + f] = red[0];
        __syncthreads();
    }
    }
}

// one block per box, one thread per quantity, fixed order: deterministic
static __global__ void k_finish_diag(Boxes B, const double* __restrict__ part, double* __restrict__ out)
{
    const int b = blockIdx.x;
    const int f = threadIdx.x;
    if (b >= B.nbox || f >= 10) return;
    const long long v0 = B.b[b].vblk0;
    const long long v1 = b + 1 < B.nbox ? B.b[b + 1].vblk0 : B.nvblk;
    double a = 0.0;
    for (long long v = v0; v < v1; v++) {
        double x = part[v * 10 + f];
        a = f == 0 ? fmax(a, x) : a + x;
    }
    out[b * 10 + f] = a;
}

// ---------------------------------------------------------------------------
// state conversion for the mixed layout (double interface <-> float rho, M)
// ---------------------------------------------------------------------------
template <class TO, class TI>
__global__ void k_convert(TO* __restrict__ out, const TI* __restrict__ in, long long n)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        out[c] = TO(in[c]);
}

}  // namespace mhd
