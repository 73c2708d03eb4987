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
constexpr int PENCIL_THREADS = 128;

// Resident blocks per SM asked of the register allocator for the pencil and
// x-warp sweeps (0: no bound).  Unbounded, the FP32 Roe sweeps take 123-128
// registers with PLM (4 blocks of 128 threads per SM) and 157-167 with PPM
// (3 blocks).  At 96 registers (5 blocks) for PLM, and at 128 (4 blocks) for
// the PPM tracing pencils of CTU, they spill at most 148 bytes a thread and
// the extra warps hide more latency than the spills cost (measured at 256^3;
// the VL PPM sweeps lose 1 % at 4 blocks and stay unbounded).  The HLLD and
// HLLE sweeps already fit 5 blocks or more, and the FP64 sweeps (194-230
// registers) are bound by the FP64 rate.
template <class R, int RECON, int SOLVER, int MODE>
constexpr int xwarp_min_blocks()
{
    if (sizeof(R) != 4 || SOLVER != ROE) return 0;
    return RECON == PPM ? (MODE == 2 ? 4 : 0) : 5;
}

// The pencils load the next cell while they solve the current face (the
// first-order walk always, the PLM walk of the VL corrector with Roe and of
// the CTU tracing); with Roe that takes 124-128 registers, and at the 96 of
// the 5-block bound it spilled and lost to the walk without the prefetch, so
// the FP32 Roe pencils other than PPM get 4 blocks (y and z predictor at
// 256^3: 0.303 -> 0.268 ms).
template <class R, int RECON, int SOLVER, int MODE>
constexpr int sweep_min_blocks()
{
    if (sizeof(R) == 4 && SOLVER == ROE && (MODE == 0 || RECON != PPM)) return 4;
    return xwarp_min_blocks<R, RECON, SOLVER, MODE>();
}

struct BoxDev {
    int nx, ny, nz, pad;
    long long off;      // first cell of the box in the batch arrays
    long long n;        // cells of the box
    long long vblk0;    // first virtual block of the box
    double dx;
    int tile0[3];       // first sweep tile of the box, per axis
    float inv_dx;       // 1/dx in single precision
    int etile0;         // first edge-field tile of the box
    int bc;             // bit d set: outflow (zero-gradient) boundaries along axis d, else periodic
    int ftile0;         // first tile of the box in the fused VL predictor
    long long pth0[3];  // first pencil-segment thread of the box, per axis
    long long xw0[3];   // first x-warp item of the box: predictor, PLM corrector, PPM corrector
    long long xr0;      // first grid row (j, k) of the box
    long long xp0;      // first x-pencil thread of the box
    long long vq0;      // first virtual block of the box in the x-quad kernels
    int quad;           // 1: those kernels take the box's cells four along x per thread (16-byte aligned)
    int qpad;
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
    int netile;         // edge-field tiles of the batch
    int pl;             // pencil segment length (faces per thread)
    long long npth[3];  // pencil-segment threads of the batch, per axis
    long long nxw[3];   // x-warp items of the batch: predictor, PLM corrector, PPM corrector
    long long nxr;      // grid rows of the batch
    long long nxp;      // x-pencil threads of the batch
    long long nvq;      // virtual blocks of the x-quad kernels
    int nftile;         // fused VL predictor tiles of the batch
    int fz;             // their extent along z (planes per tile)
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

// index along an axis of n cells: periodic wrap, or for an outflow axis the
// nearest cell (zero-gradient ghosts; a face or edge beyond the last one is
// the last one)
__device__ __forceinline__ int bidx(int i, int n, int outflow)
{
    if (outflow) return i < 0 ? 0 : (i >= n ? n - 1 : i);
    return wrapi(i, n);
}

__device__ __forceinline__ long long cell_of(const BoxDev& g, int i, int j, int k)
{
    return g.off + ((long long)k * g.ny + j) * g.nx + i;
}

// neighbour of (i,j,k) shifted by s along axis d (periodic in the box)
__device__ __forceinline__ long long nbr(const BoxDev& g, int i, int j, int k, int d, int s)
{
    if (d == 0) i = bidx(i + s, g.nx, g.bc & 1);
    else if (d == 1) j = bidx(j + s, g.ny, g.bc & 2);
    else k = bidx(k + s, g.nz, g.bc & 4);
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

// four consecutive elements from / to a 16-byte aligned address (FP32: one
// 16-byte access; FP64: two)
template <class T>
__device__ __forceinline__ void ld4(const T* __restrict__ p, T v[4])
{
    if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
}

template <class T>
__device__ __forceinline__ void st4(T* __restrict__ p, const T v[4])
{
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    }
}

// box of a virtual block of the x-quad kernels
__device__ __forceinline__ int box_of_vq(const Boxes& B, long long v)
{
    int lo = 0, hi = B.nbox - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (B.b[mid].vq0 <= v) lo = mid; else hi = mid - 1;
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

// FP32 operand widened to the energy and face-field type TE (FP64 in the mixed
// form) on the integer units.  A hardware FP32 -> FP64 conversion issues on the
// FP64 pipe, which runs at 1/64 of the FP32 rate on this part and bounds the
// mixed per-cell kernels; the IEEE-754 binary32 and binary64 layouts give the
// same exact value with a few integer instructions: the sign stays, the
// exponent is re-biased by 1023 - 127 = 896 (by 2047 - 255 = 1792 for
// infinities and NaNs, which keep their class) and the 23 fraction bits become
// the top of the 52.  Zeros and FP32 subnormals (which this build's FP32
// arithmetic flushes) give a signed zero.
template <class TE, class R>
__device__ __forceinline__ TE widen(R x)
{
    if constexpr (sizeof(TE) == 8 && sizeof(R) == 4) {
        const unsigned u = __float_as_uint(x);
        const unsigned a = u & 0x7fffffffu, sgn = u & 0x80000000u;
        const bool tiny = a < 0x00800000u;
        const unsigned hi = tiny ? sgn : (sgn | ((a >> 3) + (a >= 0x7f800000u ? 0x70000000u : 0x38000000u)));
        const unsigned lo = tiny ? 0u : (a << 29);
        return __hiloint2double((int)hi, (int)lo);
    } else {
        return TE(x);
    }
}

// FP64 value rounded to the FP32 arithmetic type R on the integer units (the
// counterpart of widen, for the same reason): round to nearest, ties to even,
// on the 29 fraction bits that FP32 drops; a carry out of the fraction moves
// into the exponent, and past the largest finite FP32 value to infinity.
// Results below the FP32 normal range give a signed zero (this build flushes
// subnormals); NaNs stay NaNs.
template <class R, class TE>
__device__ __forceinline__ R narrow(TE x)
{
    if constexpr (sizeof(TE) == 8 && sizeof(R) == 4) {
        const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
        const unsigned sgn = hi & 0x80000000u, ex = (hi >> 20) & 0x7ffu;
        unsigned v = ((ex - 896u) << 23) + (((hi & 0xfffffu) << 3) | (lo >> 29));
        const unsigned rem = lo & 0x1fffffffu;
        v += (rem > 0x10000000u || (rem == 0x10000000u && (v & 1u))) ? 1u : 0u;
        v = ex <= 896u ? 0u : (ex >= 1151u ? 0x7f800000u : v);
        if (ex == 0x7ffu && ((hi & 0xfffffu) | lo)) v = 0x7fc00000u;
        return __uint_as_float(sgn | v);
    } else {
        return R(x);
    }
}

// kinetic energy |M|^2 / (2 rho) in the energy's type TE: from the velocities
// when the state has one type, else (the mixed form: FP32 rho, M with an
// FP64 energy) in FP64 from the stored FP32 momentum, so the pressure
// recovery keeps FP64 accuracy.  There 1/rho is the FP32 reciprocal irho
// refined by one Newton step in FP64, y <- y + y (1 - rho y), which squares
// its relative error: below (2.4e-7)^2 + 2e-16 < 1e-13, against a full FP64
// division that costs several more FP64-pipe instructions.
template <class TU, class TE>
__device__ __forceinline__ TE kinetic(TU rho, TU irho, TU mx, TU my, TU mz, TU vx, TU vy, TU vz)
{
    if (sizeof(TU) == sizeof(TE))
        return TE(0.5) * (TE(mx) * TE(vx) + TE(my) * TE(vy) + TE(mz) * TE(vz));
    const TE dx = widen<TE>(mx), dy = widen<TE>(my), dz = widen<TE>(mz);
    const TE y0 = widen<TE>(irho);
    const TE y = fma(y0, fma(-widen<TE>(rho), y0, TE(1)), y0);
    return (TE(0.5) * (dx * dx + dy * dy + dz * dz)) * y;
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
// block maximum of the threads' values v >= 0, folded into *acc by an atomic
// maximum on the bits of the double (monotone for values >= 0); every thread
// of the block calls it
__device__ __forceinline__ void block_max_to(double v, double* red, unsigned long long* acc)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double m = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (!(m > 0.0)) m = 0.0;      // -0 (and NaN) as +0: the bits then order as the values
        if (threadIdx.x == 0) atomicMax(acc, (unsigned long long)__double_as_longlong(m));
    }
    __syncthreads();
}

// Pressure recovery (Eq. 5) of one cell in the precision of the stored
// energy, from rho, M (TU), their quotient v, e (TE) and twice the
// cell-centred field (the sum of the cell's two faces per axis): the halving
// is folded into the magnetic energy's factor and done in the arithmetic type
// for the primitives, both exact (powers of two), which saves three FP64
// multiplications in the mixed form.
template <class TU, class TE>
__device__ __forceinline__ TE cell_pressure(TU rho, TU irho, TU mx, TU my, TU mz, TU vx, TU vy, TU vz, TE e, TE sx,
                                            TE sy, TE sz, double gam)
{
    return TE(gam - 1.0) * (e - kinetic<TU, TE>(rho, irho, mx, my, mz, vx, vy, vz)
                            - TE(0.125) * (sx * sx + sy * sy + sz * sz));
}

// CFL signal speed of one cell's primitives: max over axes of |v_d| + c_f,d
template <class R>
__device__ __forceinline__ R cell_signal(const R w[8], double gam)
{
    const R iw0 = R(1) / w[0];
    R a2 = sizeof(R) == 4 ? R(gam) * w[4] * iw0 : R(gam) * w[4] / w[0];
    R sm = R(0);
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
        R cf = fast_speed(w[0], iw0, a2, w[5 + d], w[5 + t1], w[5 + t2]);
        sm = rmax(sm, Num<R>::abs_(w[1 + d]) + cf);
    }
    return sm;
}

// CT face update (Eq. 13): b - r * circulation
template <class TE>
__device__ __forceinline__ TE ct_face(TE b, TE r, TE circ)
{
    return b - r * circ;
}

template <class R, class TU, class TE, bool OUT = false>
__global__ void __launch_bounds__(CELL_THREADS) k_prim(Boxes B, StateP<TU, TE> s, R* __restrict__ W, double gam,
                                                       unsigned long long* smax_acc, unsigned long long* bad_cell,
                                                       double pfloor = 0.0, unsigned long long* nfloor = nullptr)
{
    const long long N = B.N;
    __shared__ double red[CELL_THREADS / 32];
    // CFL signal speeds: a running maximum per thread over the cells of one
    // box, folded into the box's accumulator when the (block-uniform) box
    // changes and at the end; no barrier per virtual block
    double run = 0.0;
    int cur = -1;
    for (long long v = blockIdx.x; v < B.nvblk; v += gridDim.x) {
        const int bi = box_of_vblk(B, v);
        if (smax_acc && bi != cur) {
            if (cur >= 0) block_max_to(run, red, smax_acc + cur);
            run = 0.0;
            cur = bi;
        }
        BoxDev g = B.b[bi];
        if (!OUT) g.bc = 0;     // periodic instantiation: the wrap is compiled in
        const long long lc = (v - g.vblk0) * CELL_THREADS + threadIdx.x;
        double local = 0.0;
        if (lc < g.n) {
            int i, j, k;
            coords(g, lc, i, j, k);
            const long long c = g.off + lc;
            // twice the cell-centred field (the sum of the two faces)
            const TE sx = s.b[0][c] + s.b[0][nbr(g, i, j, k, 0, 1)];
            const TE sy = s.b[1][c] + s.b[1][nbr(g, i, j, k, 1, 1)];
            const TE sz = s.b[2][c] + s.b[2][nbr(g, i, j, k, 2, 1)];
            const TU rho = s.rho[c];
            const TU mx = s.m[0][c], my = s.m[1][c], mz = s.m[2][c];
            const TU irho = TU(1) / rho;     // one division (FP64 is slow on this part)
            const TU vx = mx * irho, vy = my * irho, vz = mz * irho;
            TE p = cell_pressure<TU, TE>(rho, irho, mx, my, mz, vx, vy, vz, s.e[c], sx, sy, sz, gam);
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
            R w[8] = {R(rho), R(vx), R(vy), R(vz), narrow<R>(p), R(0.5) * narrow<R>(sx), R(0.5) * narrow<R>(sy),
                      R(0.5) * narrow<R>(sz)};
#pragma unroll
            for (int f = 0; f < 8; f++) W[f * N + c] = w[f];
            if (!(w[0] > R(0)) || !(w[4] > R(0))) atomicMin(bad_cell, (unsigned long long)c);
            if (smax_acc) local = (double)cell_signal(w, gam);
        }
        run = fmax(run, local);
    }
    if (smax_acc && cur >= 0) block_max_to(run, red, smax_acc + cur);
}

// a1 + a2 by x-quads (periodic boxes, FP32 state): k_prim's arithmetic for
// four consecutive cells along x per thread, 16-byte loads and stores, the x
// neighbour faces from the same vectors; one cell per thread in a box that
// is not 16-byte aligned.  The CFL maximum runs per box as in k_prim (the
// quad virtual blocks never straddle two boxes).
template <class R, class TU, class TE>
__global__ void __launch_bounds__(CELL_THREADS) k_prim4(Boxes B, StateP<TU, TE> s, R* __restrict__ W, double gam,
                                                        unsigned long long* smax_acc, unsigned long long* bad_cell,
                                                        double pfloor = 0.0, unsigned long long* nfloor = nullptr)
{
    const long long N = B.N;
    __shared__ double red[CELL_THREADS / 32];
    double run = 0.0;
    int cur = -1;
    // one cell: the primitives (Eq. 5) from rho, M, e and twice the
    // cell-centred field, the optional floor, the stores and the checks;
    // returns its CFL signal speed
    auto cell = [&](long long c, TU rho, TU mx, TU my, TU mz, TE e, TE sx, TE sy, TE sz, R w[8]) -> double {
        const TU irho = TU(1) / rho;
        const TU vx = mx * irho, vy = my * irho, vz = mz * irho;
        TE p = cell_pressure<TU, TE>(rho, irho, mx, my, mz, vx, vy, vz, e, sx, sy, sz, gam);
        if (pfloor > 0.0 && p < TE(pfloor)) {
            if (nfloor) {
                s.e[c] = e + (TE(pfloor) - p) / TE(gam - 1.0);
                atomicAdd(nfloor, 1ull);
            }
            p = TE(pfloor);
        }
        w[0] = R(rho); w[1] = R(vx); w[2] = R(vy); w[3] = R(vz); w[4] = narrow<R>(p);
        w[5] = R(0.5) * narrow<R>(sx); w[6] = R(0.5) * narrow<R>(sy); w[7] = R(0.5) * narrow<R>(sz);
        if (!(w[0] > R(0)) || !(w[4] > R(0))) atomicMin(bad_cell, (unsigned long long)c);
        return smax_acc ? (double)cell_signal(w, gam) : 0.0;
    };
    for (long long v = blockIdx.x; v < B.nvq; v += gridDim.x) {
        const int bi = box_of_vq(B, v);
        if (smax_acc && bi != cur) {
            if (cur >= 0) block_max_to(run, red, smax_acc + cur);
            run = 0.0;
            cur = bi;
        }
        BoxDev g = B.b[bi];
        g.bc = 0;
        double local = 0.0;
        if (!g.quad) {                                     // one cell per thread
            const long long lc = (v - g.vq0) * CELL_THREADS + threadIdx.x;
            if (lc < g.n) {
                int i, j, k;
                coords(g, lc, i, j, k);
                const long long c = g.off + lc;
                const TE sx = s.b[0][c] + s.b[0][nbr(g, i, j, k, 0, 1)];
                const TE sy = s.b[1][c] + s.b[1][nbr(g, i, j, k, 1, 1)];
                const TE sz = s.b[2][c] + s.b[2][nbr(g, i, j, k, 2, 1)];
                R w[8];
                local = cell(c, s.rho[c], s.m[0][c], s.m[1][c], s.m[2][c], s.e[c], sx, sy, sz, w);
#pragma unroll
                for (int f = 0; f < 8; f++) W[f * N + c] = w[f];
            }
        } else {
            const long long lc = 4 * ((v - g.vq0) * CELL_THREADS + threadIdx.x);
            if (lc < g.n) {
                int i, j, k;
                coords(g, lc, i, j, k);                    // i: a multiple of 4
                const long long c = g.off + lc;
                const long long cx = cell_of(g, i + 4 < g.nx ? i + 4 : 0, j, k);
                const long long cy = nbr(g, i, j, k, 1, 1), cz = nbr(g, i, j, k, 2, 1);
                TE b0[4], b1[4], b2[4], b1y[4], b2z[4], e[4];
                TU rho[4], mx[4], my[4], mz[4];
                ld4(s.b[0] + c, b0);
                ld4(s.b[1] + c, b1);
                ld4(s.b[2] + c, b2);
                ld4(s.b[1] + cy, b1y);
                ld4(s.b[2] + cz, b2z);
                const TE b0x = s.b[0][cx];
                ld4(s.rho + c, rho);
                ld4(s.m[0] + c, mx);
                ld4(s.m[1] + c, my);
                ld4(s.m[2] + c, mz);
                ld4(s.e + c, e);
                R w[8][4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const TE sx = b0[q] + (q < 3 ? b0[q + 1] : b0x);
                    const TE sy = b1[q] + b1y[q];
                    const TE sz = b2[q] + b2z[q];
                    R wq[8];
                    local = fmax(local, cell(c + q, rho[q], mx[q], my[q], mz[q], e[q], sx, sy, sz, wq));
#pragma unroll
                    for (int f = 0; f < 8; f++) w[f][q] = wq[f];
                }
#pragma unroll
                for (int f = 0; f < 8; f++) st4(W + f * N + c, w[f]);
            }
        }
        run = fmax(run, local);
    }
    if (smax_acc && cur >= 0) block_max_to(run, red, smax_acc + cur);
}

// dt of every box from its signal-speed maximum (the accumulator, which is
// cleared for the next primitive pass); one thread per box
static __global__ void k_finalize_dt(Boxes B, unsigned long long* __restrict__ smax_acc, double cfl, double* dt,
                                     double* smax_box, DtBox* dtb)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B.nbox) return;
    const double sm = __longlong_as_double((long long)smax_acc[b]);
    smax_acc[b] = 0ull;
    if (smax_box) smax_box[b] = sm;
    const double d = sm > 0.0 ? cfl * B.b[b].dx / sm : 0.0;
    if (dt) dt[b] = d;
    if (dtb) write_dtbox(dtb + b, d, B.b[b].dx);
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

// D >= 0 fixes the sweep axis at compile time (the CTU tracing launches):
// with the run-time axis the compiler keeps per-thread arrays in local memory.
template <class R, int RECON, int SOLVER, int MODE, class TE, int D = -1>
__global__ void __launch_bounds__(SWEEP_THREADS) k_sweep(Boxes B, int d_run, const R* __restrict__ W,
                                                         const TE* __restrict__ Bd, R* __restrict__ F,
                                                         R* __restrict__ WMg, R* __restrict__ WPg,
                                                         const DtBox* __restrict__ dtb, double gam,
                                                         const int* __restrict__ tile_list = nullptr,
                                                         const int* __restrict__ tile_count = nullptr,
                                                         const unsigned char* __restrict__ skip = nullptr)
{
    const int d = D >= 0 ? D : d_run;
    extern __shared__ unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);
    const long long N = B.N;
    const Tile t = tile_of(d, B.tl);
    const R gr = R(gam), gm1 = R(gam - 1.0);
    const int nreg = t.rx * t.ry * t.rz;
    R* SMs = sm;                 // [nreg][7] state on the cell's face -1/2
    R* SPs = sm + nreg * 7;      // [nreg][7] state on the cell's face +1/2
    R* DWs = sm + nreg * 14;     // [nslope][7] PPM slopes

    // all tiles of the batch, or only those of a list, or all but those
    // marked in skip (the learned selector's full and cheap tiles)
    const int ntile = tile_list ? *tile_count : B.ntile[d];
    for (int it = blockIdx.x; it < ntile; it += gridDim.x) {
        const int tile = tile_list ? tile_list[it] : it;
        if (skip && skip[tile]) continue;     // block-uniform
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
                    int i = bidx(sx0 + qx, g.nx, g.bc & 1), j = bidx(sy0 + qy, g.ny, g.bc & 2),
                        k = bidx(sz0 + qz, g.nz, g.bc & 4);
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
                int i = bidx(gi, g.nx, g.bc & 1), j = bidx(gj, g.ny, g.bc & 2), k = bidx(gk, g.nz, g.bc & 4);
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
// a3/a4 + a6 by pencils (VL predictor and corrector): one thread walks pl
// consecutive faces of one grid line along the sweep axis d, keeping the
// states of the cells around the current face in registers, so every cell
// is loaded and reconstructed once per segment (plus the segment's one- or
// two-cell lead-in) and no shared memory or barrier is involved.  Lanes run
// along the first transverse axis (x for d = 1, 2; y for d = 0).
// ---------------------------------------------------------------------------
struct Pencil {
    long long base, stride;   // cell of line position i: base + bidx(i) * stride
    int n;                    // cells along the line
    int out;                  // outflow ends (else periodic)
};

__host__ __device__ __forceinline__ void pencil_dims(int nx, int ny, int nz, int d, int pl, int& na, int& nb, int& ns)
{
    if (d == 0) { na = ny; nb = nz; ns = (nx + pl - 1) / pl; }
    else if (d == 1) { na = nx; nb = nz; ns = (ny + pl - 1) / pl; }
    else { na = nx; nb = ny; ns = (nz + pl - 1) / pl; }
}

__host__ __device__ __forceinline__ long long pencil_threads_of_box(int nx, int ny, int nz, int d, int pl)
{
    int na, nb, ns;
    pencil_dims(nx, ny, nz, d, pl, na, nb, ns);
    return (long long)na * nb * ns;
}

__device__ __forceinline__ int box_of_pth(const Boxes& B, int d, long long t)
{
    int lo = 0, hi = B.nbox - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (B.b[mid].pth0[d] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ long long pcell(const Pencil& p, int i)
{
    return p.base + (long long)bidx(i, p.n, p.out) * p.stride;
}

// CTU tracing (Sec. 3.2, steps 1-2): the dB_n/dn source terms of a cell
// (state w0, cell-centre B_n bn) over dt/2, added to both traced states;
// dbn = (B_n(upper face) - B_n(lower face)) / dx
template <class R>
__device__ __forceinline__ void trace_source(const R w0[7], R bn, R dbn, R hdt, R gm1, R wm[7], R wp[7])
{
    R vb = w0[1] * bn + w0[2] * w0[5] + w0[3] * w0[6];
    R src[7] = {R(0), bn / w0[0], w0[5] / w0[0], w0[6] / w0[0], -gm1 * vb, w0[2], w0[3]};
#pragma unroll
    for (int m = 0; m < 7; m++) {
        wm[m] = wm[m] + hdt * src[m] * dbn;
        wp[m] = wp[m] + hdt * src[m] * dbn;
    }
}

// (B_n(c1) - B_n(c0)) / dx of the face field, in the arithmetic type
template <class R, class TE>
__device__ __forceinline__ R face_gradient(const TE* __restrict__ Bd, long long c0, long long c1, const BoxDev& g)
{
    return sizeof(R) == 8 ? R((double)(Bd[c1] - Bd[c0]) / g.dx) : R(Bd[c1] - Bd[c0]) * R(g.inv_dx);
}

template <class R>
__device__ __forceinline__ void copy7(R d[7], const R s[7])
{
#pragma unroll
    for (int m = 0; m < 7; m++) d[m] = s[m];
}

// seg_list / seg_count: only the segments of a list (the learned selector's
// full ones); skip: every segment but those marked (its cheap ones: the grid
// covers every segment of the axis, so adjacent lanes keep adjacent
// segments and coalesced loads)
// The sweep axis D is a template parameter: with a run-time axis the
// compiler kept the cell windows in local memory (a 240-byte stack frame).
// MODE 2 (CTU step 1-2): the states are traced to t + dt/2 (recon_cell with
// tracing, plus the dB_n/dn source terms of the 1-D sweep, as in k_sweep);
// each owned cell's lower and upper traced states go to WMg / WPg, and the
// face flux uses the previous cell's upper and this cell's lower state.
template <class R, int RECON, int SOLVER, int MODE, class TE, int D>
__global__ void __launch_bounds__(PENCIL_THREADS, (sweep_min_blocks<R, RECON, SOLVER, MODE>())) k_pencil(Boxes B, const R* __restrict__ W,
                                                           const TE* __restrict__ Bd, R* __restrict__ F, double gam,
                                                           const int* __restrict__ seg_list = nullptr,
                                                           const int* __restrict__ seg_count = nullptr,
                                                           R* __restrict__ WMg = nullptr, R* __restrict__ WPg = nullptr,
                                                           const DtBox* __restrict__ dtb = nullptr,
                                                           const unsigned char* __restrict__ skip = nullptr)
{
    constexpr int d = D;
    // one segment per thread, or with a list a grid-stride loop over it (the
    // list's grid is capped: most of the axis's segments are not on it)
    const long long gstride = (long long)gridDim.x * blockDim.x;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x;; it += gstride) {
    long long gt = it;
    if (seg_list) {
        if (it >= *seg_count) return;
        gt = seg_list[it];
    }
    if (gt >= B.npth[d]) return;
    if (skip && skip[gt]) return;
    const int bi = box_of_pth(B, d, gt);
    const BoxDev g = B.b[bi];
    int na, nb, ns;
    pencil_dims(g.nx, g.ny, g.nz, d, B.pl, na, nb, ns);
    long long t = gt - g.pth0[d];
    const int ia = (int)(t % na);
    t /= na;
    const int ib = (int)(t % nb);
    const int sg = (int)(t / nb);
    Pencil p;
    if (d == 0) { p.base = g.off + ((long long)ib * g.ny + ia) * g.nx; p.stride = 1; p.n = g.nx; }
    else if (d == 1) { p.base = g.off + (long long)ib * g.ny * g.nx + ia; p.stride = g.nx; p.n = g.ny; }
    else { p.base = g.off + (long long)ib * g.nx + ia; p.stride = (long long)g.nx * g.ny; p.n = g.nz; }
    p.out = g.bc >> d & 1;
    const int i0 = sg * B.pl;
    const int i1 = i0 + B.pl < p.n ? i0 + B.pl : p.n;
    const long long N = B.N;
    const R gr = R(gam), gm1 = R(gam - 1.0);
    constexpr bool TR = MODE == 2;
    const R dtdx = TR ? DtOf<R>::dtdx(dtb[bi]) : R(0);
    const R hdt = TR ? DtOf<R>::hdt(dtb[bi]) : R(0);
    // MODE 2: the dB_n/dn source terms of cell i (state w0, cell-centre B_n
    // bn) over dt/2, added to both traced states
    auto trace_src = [&](int i, const R w0[7], R bn, R wm[7], R wp[7]) {
        trace_source(w0, bn, face_gradient<R>(Bd, pcell(p, i), pcell(p, i + 1), g), hdt, gm1, wm, wp);
    };
    R f[7];
    if (MODE == 0) {
        // first-order states: the face i sees cells i-1 and i; cell i+1 is
        // loaded while face i is solved
        R wl[7], wr[7], wn[7], bdum;
        load_rot(W, N, pcell(p, i0 - 1), d, wl, bdum);
        load_rot(W, N, p.base + (long long)i0 * p.stride, d, wn, bdum);
        TE bnn = Bd[p.base + (long long)i0 * p.stride];
        for (int i = i0; i < i1; i++) {
            const long long ci = p.base + (long long)i * p.stride;
            copy7(wr, wn);
            const R bnf = R(bnn);
            if (i + 1 < i1) {
                load_rot(W, N, ci + p.stride, d, wn, bdum);
                bnn = Bd[ci + p.stride];
            }
            riemann<SOLVER>(wl, wr, bnf, gm1, gr, f);
#pragma unroll
            for (int m = 0; m < 7; m++) F[(long long)m * N + ci] = f[m];
            copy7(wl, wr);
        }
    } else if (RECON != PPM) {
        // PLM: cells i-1, i, i+1 in registers; wpp the "+" state of cell i-1
        R wa[7], wb[7], wc[7], bna, bnb, bnc, wpp[7], wm[7], wp[7], dum[7];
        // lead-in: the "+" state of cell i0-1, i.e. of the cell it maps to (at
        // a lower outflow side, cell 0 with its own stencil and source term)
        const int li = bidx(i0 - 1, p.n, p.out);
        load_rot(W, N, pcell(p, li - 1), d, wa, bna);
        load_rot(W, N, pcell(p, li), d, wb, bnb);
        load_rot(W, N, pcell(p, li + 1), d, wc, bnc);
        recon_cell<RECON, TR>(wa, wb, wc, bnb, gr, dum, dum, dum, dtdx, wm, wpp);
        if (TR) trace_src(li, wb, bnb, wm, wpp);
        load_rot(W, N, pcell(p, i0 - 1), d, wa, bna);
        load_rot(W, N, pcell(p, i0), d, wb, bnb);
        // cell i+2 is loaded while face i is computed, where that measured
        // faster at 256^3 FP32: the VL corrector with Roe (at 4 blocks per
        // SM, y and z 0.492 -> 0.47 ms) and the CTU tracing with Roe and HLLD
        // (0.70 -> 0.62 ms); the VL corrector with HLLE lost 7 % and with
        // HLLD 1 %
        constexpr bool PF = (MODE == 1 && SOLVER == ROE) || (MODE == 2 && SOLVER != HLLE);
        R wn[7], bnn;
        if (PF) load_rot(W, N, pcell(p, i0 + 1), d, wn, bnn);
        for (int i = i0; i < i1; i++) {
            const long long ci = p.base + (long long)i * p.stride;
            if (PF) {
                copy7(wc, wn);
                bnc = bnn;
                if (i + 1 < i1) load_rot(W, N, pcell(p, i + 2), d, wn, bnn);
            } else {
                load_rot(W, N, pcell(p, i + 1), d, wc, bnc);
            }
            recon_cell<RECON, TR>(wa, wb, wc, bnb, gr, dum, dum, dum, dtdx, wm, wp);
            if (TR) {
                trace_src(i, wb, bnb, wm, wp);
#pragma unroll
                for (int m = 0; m < 7; m++) {
                    WMg[(long long)m * N + ci] = wm[m];
                    WPg[(long long)m * N + ci] = wp[m];
                }
            }
            riemann<SOLVER>(wpp, wm, R(Bd[ci]), gm1, gr, f);
#pragma unroll
            for (int m = 0; m < 7; m++) F[(long long)m * N + ci] = f[m];
            copy7(wpp, wp);
            copy7(wa, wb); bna = bnb;
            copy7(wb, wc); bnb = bnc;
        }
    } else {
        // PPM: cells i-1 .. i+2 and the characteristic slopes of i-1 .. i+1
        R w0[7], w1[7], w2[7], w3[7], b0, b1, b2, b3;      // cells i-1, i, i+1, i+2
        R s0[7], s1[7], s2[7];                              // slopes of i-1, i, i+1
        R wpp[7], wm[7], wp[7];
        {
            // lead-in: the "+" state of cell i0-1, i.e. of the cell li it maps to
            // (at a lower outflow side, cell 0 with its own stencil and source)
            const int li = bidx(i0 - 1, p.n, p.out);
            R wq[7], bq;
            load_rot(W, N, pcell(p, li - 2), d, wq, bq);
            load_rot(W, N, pcell(p, li - 1), d, w0, b0);
            load_rot(W, N, pcell(p, li), d, w1, b1);
            load_rot(W, N, pcell(p, li + 1), d, w2, b2);
            load_rot(W, N, pcell(p, li + 2), d, w3, b3);
            char_slope(wq, w0, w1, b0, gr, s0);             // slope of li-1
            char_slope(w0, w1, w2, b1, gr, s1);             // li
            char_slope(w1, w2, w3, b2, gr, s2);             // li+1
            recon_cell<PPM, TR>(w0, w1, w2, b1, gr, s0, s1, s2, dtdx, wm, wpp);
            if (TR) trace_src(li, w1, b1, wm, wpp);
        }
        // window of the loop: w0..w2 = cells i0-1 .. i0+1, s0, s1 = slopes of
        // i0-1, i0
        {
            R wq[7], bq;
            load_rot(W, N, pcell(p, i0 - 2), d, wq, bq);
            load_rot(W, N, pcell(p, i0 - 1), d, w0, b0);
            load_rot(W, N, pcell(p, i0), d, w1, b1);
            load_rot(W, N, pcell(p, i0 + 1), d, w2, b2);
            char_slope(wq, w0, w1, b0, gr, s0);
            char_slope(w0, w1, w2, b1, gr, s1);
        }
        // the VL corrector loads cell i+3 while face i is computed (256^3
        // FP32: y and z 0.81 -> 0.75 ms with Roe, -> 0.77 with HLLD); the CTU
        // tracing lost 4-6 % with it
        R wn[7], bnn;
        constexpr bool PFP = MODE == 1;
        if (PFP) load_rot(W, N, pcell(p, i0 + 2), d, wn, bnn);
        for (int i = i0; i < i1; i++) {
            const long long ci = p.base + (long long)i * p.stride;
            if (PFP) {
                copy7(w3, wn);
                b3 = bnn;
                if (i + 1 < i1) load_rot(W, N, pcell(p, i + 3), d, wn, bnn);
            } else {
                load_rot(W, N, pcell(p, i + 2), d, w3, b3);
            }
            char_slope(w1, w2, w3, b2, gr, s2);             // slope of i+1
            recon_cell<PPM, TR>(w0, w1, w2, b1, gr, s0, s1, s2, dtdx, wm, wp);
            if (TR) {
                trace_src(i, w1, b1, wm, wp);
#pragma unroll
                for (int m = 0; m < 7; m++) {
                    WMg[(long long)m * N + ci] = wm[m];
                    WPg[(long long)m * N + ci] = wp[m];
                }
            }
            riemann<SOLVER>(wpp, wm, R(Bd[ci]), gm1, gr, f);
#pragma unroll
            for (int m = 0; m < 7; m++) F[(long long)m * N + ci] = f[m];
            copy7(wpp, wp);
            copy7(w0, w1); b0 = b1;
            copy7(w1, w2); b1 = b2;
            copy7(w2, w3); b2 = b3;
            copy7(s0, s1);
            copy7(s1, s2);
        }
    }
    if (!seg_list) return;
    }
}

// launch the pencil sweep along a run-time axis d
template <class R, int RECON, int SOLVER, int MODE, class TE>
inline void launch_pencil(int d, int grid, cudaStream_t st, const Boxes& g, const R* W, const TE* Bd, R* F,
                          double gam, const int* seg_list = nullptr, const int* seg_count = nullptr,
                          R* WMg = nullptr, R* WPg = nullptr, const DtBox* dtb = nullptr,
                          const unsigned char* skip = nullptr)
{
    if (d == 0)
        k_pencil<R, RECON, SOLVER, MODE, TE, 0><<<grid, PENCIL_THREADS, 0, st>>>(g, W, Bd, F, gam, seg_list, seg_count,
                                                                              WMg, WPg, dtb, skip);
    else if (d == 1)
        k_pencil<R, RECON, SOLVER, MODE, TE, 1><<<grid, PENCIL_THREADS, 0, st>>>(g, W, Bd, F, gam, seg_list, seg_count,
                                                                              WMg, WPg, dtb, skip);
    else
        k_pencil<R, RECON, SOLVER, MODE, TE, 2><<<grid, PENCIL_THREADS, 0, st>>>(g, W, Bd, F, gam, seg_list, seg_count,
                                                                              WMg, WPg, dtb, skip);
}

// ---------------------------------------------------------------------------
// a3/a4 + a6 along x by warps: the lanes of a warp hold 32 consecutive cells
// of one grid row (coalesced loads, x fastest in memory) and take their
// neighbours' states and slopes by register shuffles, so the x sweep also
// runs without shared memory or barriers.  A warp item yields XW_FW faces:
// 31 for the first-order predictor (lanes 1..31), 29 for PLM (reconstruction
// valid on lanes 1..30, faces on lanes 2..30), 27 for PPM (slopes on lanes
// 1..30, reconstruction on 2..29, faces on 3..29).
// ---------------------------------------------------------------------------
template <int RECON, int MODE> struct XW {
    static constexpr int slot = MODE == 0 ? 0 : (RECON == PPM ? 2 : 1);
    static constexpr int lead = MODE == 0 ? 1 : (RECON == PPM ? 3 : 2);   // lane 0's cell: x0 - lead
};
__host__ __device__ constexpr int xw_faces(int slot) { return slot == 0 ? 31 : (slot == 1 ? 29 : 27); }

__host__ __device__ __forceinline__ long long xwarp_items_of_box(int nx, int ny, int nz, int slot)
{
    const int fw = xw_faces(slot);
    return (long long)ny * nz * ((nx + fw - 1) / fw);
}

__device__ __forceinline__ int box_of_xw(const Boxes& B, int slot, long long t)
{
    int lo = 0, hi = B.nbox - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (B.b[mid].xw0[slot] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <class R>
__device__ __forceinline__ void shfl7(R o[7], const R v[7], int up)
{
#pragma unroll
    for (int m = 0; m < 7; m++)
        o[m] = up ? __shfl_up_sync(0xffffffffu, v[m], 1) : __shfl_down_sync(0xffffffffu, v[m], 1);
}

__device__ __forceinline__ int box_of_row(const Boxes& B, long long t)
{
    int lo = 0, hi = B.nbox - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (B.b[mid].xr0 <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One warp per grid row, marching its segments of xw_faces(dslot) faces
// (dslot: the segment length, at most the kernel's own), the next segment's
// cell loaded while the current one is computed; with skip, the segments
// marked there are left out of the march.  With item_list / item_count the
// warps stride over the listed segments instead, one at a time (the learned
// selector's lists, whose cheap and full kernels share one decomposition).
//
// MODE 2 (CTU steps 1-2, x periodic): the lanes reconstruct with tracing and
// add the dB_n/dn source terms, as the tracing pencils do; each face lane
// writes its cell's traced lower and upper states to WMg / WPg.  (At a lower
// outflow side the lanes left of x = 0 would see a clamped stencil, where the
// CTU lead-in is cell 0 with its own stencil and source term; such boxes
// keep the tile sweep along x.)
template <class R, int RECON, int SOLVER, int MODE, class TE>
__global__ void __launch_bounds__(PENCIL_THREADS, (xwarp_min_blocks<R, RECON, SOLVER, MODE>())) k_xwarp(Boxes B, const R* __restrict__ W,
                                                          const TE* __restrict__ Bd, R* __restrict__ F, double gam,
                                                          int dslot, const int* __restrict__ item_list = nullptr,
                                                          const int* __restrict__ item_count = nullptr,
                                                          R* __restrict__ WMg = nullptr, R* __restrict__ WPg = nullptr,
                                                          const DtBox* __restrict__ dtb = nullptr,
                                                          const unsigned char* __restrict__ skip = nullptr)
{
    constexpr bool TR = MODE == 2;
    constexpr int LEAD = XW<RECON, MODE>::lead;
    const int FW = xw_faces(dslot);
    const int lane = threadIdx.x & 31;
    // one row per warp, or with a list a grid-stride loop over its items (the
    // list's grid is capped: most items are not on it).  One body serves both,
    // so a listed segment is computed with the very instructions of a march.
    const long long wstride = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;; wid += wstride) {
    int bi, j, k, sg0, sg1;
    long long item0 = 0;                             // item of segment 0 of the row (skip)
    if (item_list) {
        if (wid >= *item_count) return;              // uniform over the warp
        const long long item = item_list[wid];
        bi = box_of_xw(B, dslot, item);
        const BoxDev& gb = B.b[bi];
        const int nseg = (gb.nx + FW - 1) / FW;
        long long t = item - gb.xw0[dslot];
        sg0 = (int)(t % nseg);
        sg1 = sg0 + 1;
        t /= nseg;
        j = (int)(t % gb.ny);
        k = (int)(t / gb.ny);
    } else {
        if (wid >= B.nxr) return;
        bi = box_of_row(B, wid);
        const BoxDev& gb = B.b[bi];
        const long long t = wid - gb.xr0;
        j = (int)(t % gb.ny);
        k = (int)(t / gb.ny);
        sg0 = 0;
        sg1 = (gb.nx + FW - 1) / FW;
        item0 = gb.xw0[dslot] + t * sg1;
    }
    const int nx = B.b[bi].nx, xout = B.b[bi].bc & 1;
    const long long row = B.b[bi].off + ((long long)k * B.b[bi].ny + j) * nx;
    const long long N = B.N;
    const R gr = R(gam), gm1 = R(gam - 1.0);
    const R dtdx = TR ? DtOf<R>::dtdx(dtb[bi]) : R(0);
    const R hdt = TR ? DtOf<R>::hdt(dtb[bi]) : R(0);
    const bool face = lane >= LEAD && lane < LEAD + FW;
    R w[7], bn, f[7];
    load_rot(W, N, row + bidx(sg0 * FW - LEAD + lane, nx, xout), 0, w, bn);
    for (int sg = sg0; sg < sg1; sg++) {
        const int xi = sg * FW - LEAD + lane;        // this lane's cell (and the face below it)
        const long long ci = row + bidx(xi, nx, xout);
        R wn[7], bnn;
        if (sg + 1 < sg1) load_rot(W, N, row + bidx(xi + FW, nx, xout), 0, wn, bnn);
        if (skip && skip[item0 + sg]) {              // warp-uniform: another launch's segment
            if (sg + 1 < sg1) {
                copy7(w, wn);
                bn = bnn;
            }
            continue;
        }
        R wl[7], wr[7];
        if (MODE == 0) {
            shfl7(wl, w, 1);
            copy7(wr, w);
        } else {
            R wm1[7], wp1[7], wpf[7];
            shfl7(wm1, w, 1);
            shfl7(wp1, w, 0);
            if (RECON == PPM) {
                // the lane's cell eigensystem serves its slope and its reconstruction
                R s0[7], sm1[7], sp1[7];
                Eig<R> e;
                cell_eig(w, bn, gr, e);
                char_slope_e(e, wm1, w, wp1, s0);
                shfl7(sm1, s0, 1);
                shfl7(sp1, s0, 0);
                recon_cell_e<PPM, TR>(e, wm1, w, wp1, sm1, s0, sp1, dtdx, wr, wpf);
            } else {
                R dum[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};   // slopes: unused by PLM
                recon_cell<RECON, TR>(wm1, w, wp1, bn, gr, dum, dum, dum, dtdx, wr, wpf);
            }
            if (TR) {
                trace_source(w, bn, face_gradient<R>(Bd, ci, row + bidx(xi + 1, nx, xout), B.b[bi]), hdt, gm1, wr,
                             wpf);
                if (face && xi < nx) {
#pragma unroll
                    for (int m = 0; m < 7; m++) {
                        WMg[(long long)m * N + ci] = wr[m];
                        WPg[(long long)m * N + ci] = wpf[m];
                    }
                }
            }
            shfl7(wl, wpf, 1);                       // the "+" state of the cell below
        }
        if (face && xi < nx) {
            riemann<SOLVER>(wl, wr, R(Bd[ci]), gm1, gr, f);
#pragma unroll
            for (int m = 0; m < 7; m++) F[(long long)m * N + ci] = f[m];
        }
        if (sg + 1 < sg1) {
            copy7(w, wn);
            bn = bnn;
        }
    }
    if (!item_list) return;
    }
}

// ---------------------------------------------------------------------------
// a7: edge electric fields, upwinded corner average (Sec. 2, Eqs. 13-14 with
// the Gardiner-Stone reference field).  Every cell gets its three lower
// edges: E_c at the corner of the faces a = c+1, b = c+2,
//   E = (ea0 + ea1 + eb0 + eb1)/4 + (lob - hib)/4 + (loa - hia)/4,
// the face values ea = -F_a[B_b], eb = F_b[B_a], the corrections upwinded by
// the sign of the mass flux through the face (mean on a tie), against the
// cell-centre reference -(v x B).
//
// Tiled: a block owns 32 x 16 cells of an x-y slab and marches EZC planes
// along z.  Each plane is staged once in shared memory with a one-cell halo
// on its lower x and y sides (561 cells x 12 values: the three reference
// components and, per axis, the mass flux and the two B fluxes), three plane
// slots deep so that one barrier per plane suffices.  F[d] = F + d*7*N.
// ---------------------------------------------------------------------------
constexpr int ETX = 32, ETY = 16, EZC = 16;
constexpr int EHX = ETX + 1, EPL = EHX * (ETY + 1);   // halo'd plane cells
constexpr int ENV = 12;                               // values per staged cell
constexpr int EMF_THREADS = 576;                     // >= EPL: one staged cell per thread

__host__ __device__ __forceinline__ int emf_tiles_of_box(int nx, int ny, int nz)
{
    return ((nx + ETX - 1) / ETX) * ((ny + ETY - 1) / ETY) * ((nz + EZC - 1) / EZC);
}

template <class R>
constexpr size_t emf_smem_bytes()
{
    return (size_t)3 * ENV * EPL * sizeof(R);
}

__device__ __forceinline__ int box_of_etile(const Boxes& B, int t)
{
    int lo = 0, hi = B.nbox - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (B.b[mid].etile0 <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <class R>
__device__ __forceinline__ R upwind(R f, R xm, R xp)
{
    if (f > R(0)) return xm;
    if (f < R(0)) return xp;
    return R(0.5) * (xm + xp);
}

// one edge from the staged planes: P1 the cell's plane, P0 the plane below;
// sa / sb the staged offsets of the shift by -1 along a / b (plane shifts
// select P0 instead)
template <class R>
__device__ __forceinline__ R edge_e(const R* cc11, const R* cc01, const R* cc10, const R* cc00,
                                    R ea0, R ea1, R eb0, R eb1, R fa0, R fa1, R fb0, R fb1)
{
    R hib = upwind(fa1, *cc01 - eb0, *cc11 - eb1);
    R lob = upwind(fa0, eb0 - *cc00, eb1 - *cc10);
    R hia = upwind(fb1, *cc10 - ea0, *cc11 - ea1);
    R loa = upwind(fb0, ea0 - *cc00, ea1 - *cc01);
    return R(0.25) * (ea0 + ea1 + eb0 + eb1) + R(0.25) * (lob - hib) + R(0.25) * (loa - hia);
}

// staged values of one cell: the reference field -(v x B) and, per axis d,
// the mass flux and the two B fluxes of F_d
template <class R>
struct EmfStage {
    R v[ENV];
};

// the cell-centre reference field -(v x B) (both staging forms)
template <class R>
__device__ __forceinline__ void ref_field(R v0, R v1, R v2, R b0, R b1, R b2, R& e0, R& e1, R& e2)
{
    e0 = -(v1 * b2 - v2 * b1);
    e1 = -(v2 * b0 - v0 * b2);
    e2 = -(v0 * b1 - v1 * b0);
}

template <class R>
__device__ __forceinline__ void emf_load(const R* __restrict__ F, const R* __restrict__ W, long long N, long long c,
                                         EmfStage<R>& s)
{
    const R v0 = W[N + c], v1 = W[2 * N + c], v2 = W[3 * N + c];
    const R b0 = W[5 * N + c], b1 = W[6 * N + c], b2 = W[7 * N + c];
    ref_field(v0, v1, v2, b0, b1, b2, s.v[0], s.v[1], s.v[2]);
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const R* Fd = F + (long long)d * 7 * N;
        s.v[3 + 3 * d] = Fd[c];
        s.v[4 + 3 * d] = Fd[5 * N + c];
        s.v[5 + 3 * d] = Fd[6 * N + c];
    }
}

// EMF_THREADS = 576 >= EPL = 561: one staged cell per thread, so a plane
// is one round of loads; the loads of plane k+1 are issued before the edges
// of plane k are computed and stored to shared memory after them.
template <class R>
__global__ void __launch_bounds__(EMF_THREADS) k_emf(Boxes B, const R* __restrict__ F, const R* __restrict__ W,
                                                     R* __restrict__ E)
{
    extern __shared__ unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>(smem_raw);    // [3 slots][ENV][EPL]
    const long long N = B.N;
    const int tid = threadIdx.x;
    const int tx = tid % ETX, ty = tid / ETX;  // edge cell of the threads tid < ETX * ETY
    const int q = (ty + 1) * EHX + (tx + 1);   // its index in the staged plane
    const bool stager = tid < EPL;
    const int hx = tid % EHX, hy = tid / EHX;  // staged cell of the threads tid < EPL
    for (int tile = blockIdx.x; tile < B.netile; tile += gridDim.x) {
        const BoxDev g = B.b[box_of_etile(B, tile)];
        const int ntx = (g.nx + ETX - 1) / ETX, nty = (g.ny + ETY - 1) / ETY;
        int bl = tile - g.etile0;
        const int x0 = (bl % ntx) * ETX;
        bl /= ntx;
        const int y0 = (bl % nty) * ETY;
        const int z0 = (bl / nty) * EZC;
        const int z1 = z0 + EZC < g.nz ? z0 + EZC : g.nz;
        const bool mine = tid < ETX * ETY && x0 + tx < g.nx && y0 + ty < g.ny;
        const int si = bidx(x0 - 1 + hx, g.nx, g.bc & 1), sj = bidx(y0 - 1 + hy, g.ny, g.bc & 2);
        EmfStage<R> st;
        if (stager) emf_load(F, W, N, cell_of(g, si, sj, bidx(z0 - 1, g.nz, g.bc & 4)), st);
        for (int k = z0 - 1; k < z1; k++) {
            R* P = sm + ((k + 3) % 3) * ENV * EPL;
            if (stager) {
#pragma unroll
                for (int f = 0; f < ENV; f++) P[f * EPL + tid] = st.v[f];
            }
            __syncthreads();
            if (stager && k + 1 < z1) emf_load(F, W, N, cell_of(g, si, sj, k + 1), st);
            if (k >= z0 && mine) {
                const R* P1 = P;
                const R* P0 = sm + ((k + 2) % 3) * ENV * EPL;
                const long long c = cell_of(g, x0 + tx, y0 + ty, k);
                // Ex: a = y, b = z.  c01 = y-1, c10 = z-1
                {
                    const R* X1 = P1 + 0 * EPL; const R* X0 = P0 + 0 * EPL;
                    R ea0 = -P0[7 * EPL + q], ea1 = -P1[7 * EPL + q];            // -F_y[B_z]
                    R eb0 = P1[11 * EPL + q - EHX], eb1 = P1[11 * EPL + q];      //  F_z[B_y]
                    R fa0 = P0[6 * EPL + q], fa1 = P1[6 * EPL + q];
                    R fb0 = P1[9 * EPL + q - EHX], fb1 = P1[9 * EPL + q];
                    E[c] = edge_e(X1 + q, X1 + q - EHX, X0 + q, X0 + q - EHX, ea0, ea1, eb0, eb1, fa0, fa1, fb0, fb1);
                }
                // Ey: a = z, b = x.  c01 = z-1, c10 = x-1
                {
                    const R* Y1 = P1 + 1 * EPL; const R* Y0 = P0 + 1 * EPL;
                    R ea0 = -P1[10 * EPL + q - 1], ea1 = -P1[10 * EPL + q];      // -F_z[B_x]
                    R eb0 = P0[5 * EPL + q], eb1 = P1[5 * EPL + q];              //  F_x[B_z]
                    R fa0 = P1[9 * EPL + q - 1], fa1 = P1[9 * EPL + q];
                    R fb0 = P0[3 * EPL + q], fb1 = P1[3 * EPL + q];
                    E[N + c] = edge_e(Y1 + q, Y0 + q, Y1 + q - 1, Y0 + q - 1, ea0, ea1, eb0, eb1, fa0, fa1, fb0, fb1);
                }
                // Ez: a = x, b = y.  c01 = x-1, c10 = y-1
                {
                    const R* Z1 = P1 + 2 * EPL;
                    R ea0 = -P1[4 * EPL + q - EHX], ea1 = -P1[4 * EPL + q];      // -F_x[B_y]
                    R eb0 = P1[8 * EPL + q - 1], eb1 = P1[8 * EPL + q];          //  F_y[B_x]
                    R fa0 = P1[3 * EPL + q - EHX], fa1 = P1[3 * EPL + q];
                    R fb0 = P1[6 * EPL + q - 1], fb1 = P1[6 * EPL + q];
                    E[2 * N + c] = edge_e(Z1 + q, Z1 + q - 1, Z1 + q - EHX, Z1 + q - 1 - EHX, ea0, ea1, eb0, eb1, fa0,
                                          fa1, fb0, fb1);
                }
            }
        }
        __syncthreads();   // the next tile restages every slot
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

// Flux through the outer face of the last cell along an outflow axis d: the
// Riemann flux between the cell and its zero-gradient copy (the limited slope
// against the copy is zero, so both face states are the cell's stage state
// Wst), with the normal field of the last face.  One thread per cell of the
// last layer of a one-box context; Fout[d][7][cs], cs = the largest
// cross-section, the layer's cell (a, b) at a + b * n_a (a, b the two other
// axes in increasing order).
__host__ __device__ __forceinline__ int cross_size(int nx, int ny, int nz)
{
    int a = ny * nz, b = nx * nz, c = nx * ny;
    return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

template <class R, int SOLVER, class TE>
__global__ void k_outer_flux(BoxDev g, int d, const R* __restrict__ Wst, const TE* __restrict__ bface, double gam,
                             long long N, R* __restrict__ Fout, int cs)
{
    const int na = d == 0 ? g.ny : g.nx, nb = d == 2 ? g.ny : g.nz;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= na * nb) return;
    const int a = q % na, b = q / na;
    int i, j, k;
    if (d == 0) { i = g.nx - 1; j = a; k = b; }
    else if (d == 1) { i = a; j = g.ny - 1; k = b; }
    else { i = a; j = b; k = g.nz - 1; }
    const long long c = cell_of(g, i, j, k);
    R w[7], bdum, f[7];
    load_rot(Wst, N, c, d, w, bdum);
    riemann<SOLVER>(w, w, R(bface[c]), R(gam - 1.0), R(gam), f);
    R* Fd = Fout + (long long)d * 7 * cs;
#pragma unroll
    for (int m = 0; m < 7; m++) Fd[(long long)m * cs + q] = f[m];
}

// Dirichlet sides (the shock tubes of Sec. 5.1 hold the left and right
// states at the ends of the box): the nl outermost cells at each end of axis
// d are ghost cells put back to a fixed state after every step; beyond them
// the outflow rule holds.  A ghost cell gets the fixed conserved state and
// its three lower faces the fixed field, except the lower face along d of the
// first upper ghost cell: that is the interior's upper boundary face, which
// CT advances.  One thread per ghost cell (2 nl layers of the cross-section,
// a + b * n_a as in k_outer_flux).
struct FixedState {
    double u[5];   // rho, Mx, My, Mz, e
    double b[3];   // Bx, By, Bz
};

template <class TU, class TE>
__global__ void k_fix_layers(BoxDev g, int d, int nl, FixedState lo, FixedState hi, StateP<TU, TE> s)
{
    const int nd = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
    const int na = d == 0 ? g.ny : g.nx, nb = d == 2 ? g.ny : g.nz;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 2LL * nl * na * nb) return;
    const int a = (int)(q % na);
    const long long r = q / na;
    const int b = (int)(r % nb);
    const int l = (int)(r / nb);                 // 0 .. 2 nl - 1
    const bool up = l >= nl;
    const int p = up ? nd - 2 * nl + l : l;      // position along d
    int i, j, k;
    if (d == 0) { i = p; j = a; k = b; }
    else if (d == 1) { i = a; j = p; k = b; }
    else { i = a; j = b; k = p; }
    const long long c = cell_of(g, i, j, k);
    const FixedState& f = up ? hi : lo;
    s.rho[c] = TU(f.u[0]);
    s.m[0][c] = TU(f.u[1]);
    s.m[1][c] = TU(f.u[2]);
    s.m[2][c] = TU(f.u[3]);
    s.e[c] = TE(f.u[4]);
#pragma unroll
    for (int m = 0; m < 3; m++)
        if (m != d || p != nd - nl) s.b[m][c] = TE(f.b[m]);
}

// CTU stage 1: the outer face's states are the last cell's own traced upper
// (WP) and lower (WM) states along d (sweep frame; the ghost beyond it is the
// cell itself), with the normal field of the last face
template <class R, int SOLVER, class TE>
__global__ void k_outer_flux_traced(BoxDev g, int d, const R* __restrict__ WPd, const R* __restrict__ WMd,
                                    const TE* __restrict__ bface, double gam, long long N, R* __restrict__ Fout, int cs)
{
    const int na = d == 0 ? g.ny : g.nx, nb = d == 2 ? g.ny : g.nz;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= na * nb) return;
    const int a = q % na, b = q / na;
    int i, j, k;
    if (d == 0) { i = g.nx - 1; j = a; k = b; }
    else if (d == 1) { i = a; j = g.ny - 1; k = b; }
    else { i = a; j = b; k = g.nz - 1; }
    const long long c = cell_of(g, i, j, k);
    R wl[7], wr[7], f[7];
#pragma unroll
    for (int m = 0; m < 7; m++) {
        wl[m] = WPd[(long long)m * N + c];
        wr[m] = WMd[(long long)m * N + c];
    }
    riemann<SOLVER>(wl, wr, R(bface[c]), R(gam - 1.0), R(gam), f);
    R* Fd = Fout + (long long)d * 7 * cs;
#pragma unroll
    for (int m = 0; m < 7; m++) Fd[(long long)m * cs + q] = f[m];
}

// index of cell (i, j, k) in the last layer along d (a + b * n_a, as in
// k_outer_flux), and whether it is in that layer along an outflow axis
__device__ __forceinline__ bool outer_cell(const BoxDev& g, int d, int i, int j, int k, int& q)
{
    const int p = d == 0 ? i : (d == 1 ? j : k);
    const int nd = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
    q = d == 0 ? j + k * g.ny : (d == 1 ? i + k * g.nx : i + j * g.nx);
    return (g.bc >> d & 1) && p == nd - 1;
}

// outflow: for each outflow axis along which (i, j, k) is the last cell, add
// the outer-face flux minus the cell's own lower-face flux to the divergence
// (the stencil saw the cell as its own upper neighbour)
template <class R, class TU, class TE>
__device__ __forceinline__ void outer_divergence(const BoxDev& g, int i, int j, int k, long long c, long long N,
                                                 const R* __restrict__ F, const R* __restrict__ Fout, int cs,
                                                 TU du[4], TE& due)
{
#pragma unroll 1
    for (int d = 0; d < 3; d++) {
        if (!(g.bc >> d & 1) || (d == 0 ? i : (d == 1 ? j : k)) != (d == 0 ? g.nx : (d == 1 ? g.ny : g.nz)) - 1)
            continue;
        const int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
        const int na = d == 0 ? g.ny : g.nx;
        const int q = d == 0 ? j + k * na : (d == 1 ? i + k * na : i + j * na);
        const R* Fo = Fout + (long long)d * 7 * cs;
        const R* Fd = F + (long long)d * 7 * N;
        const R f0 = Fo[q], f1 = Fo[cs + q], f2 = Fo[2 * cs + q], f3 = Fo[3 * cs + q], f4 = Fo[4 * cs + q];
        du[0] += TU(f0 - Fd[c]);
        du[1 + d] += TU(f1 - Fd[N + c]);
        du[1 + t1] += TU(f2 - Fd[2 * N + c]);
        du[1 + t2] += TU(f3 - Fd[3 * N + c]);
        due += TE(f4 - Fd[4 * N + c]);
    }
}

// half-step face field (Eq. 13 with dt/2) of a cell's lower faces lo[d] and
// twice its cell-centred field bc[d] (the sum of the updated lower and upper
// faces, see k_prim), each circulation in the order of curl_face.  ec[m]:
// E_m at the cell's own edges; en[m][a]: E_m at the cell shifted by +1 along
// a != m; on the diagonals the upper faces' circulations need, E_2 at
// (i+1, j+1, k), E_1 at (i+1, j, k+1), E_0 at (i, j+1, k+1); blo / bhi the
// face field of the lower / upper faces; r = (dt/2)/dx.
template <class TE, class R>
__device__ __forceinline__ void half_faces(const R ec[3], const R en[3][3], R e2xy, R e1xz, R e0yz, const TE blo[3],
                                           const TE bhi[3], TE r, TE lo[3], TE bc[3])
{
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
        // E_t2 at c + e_d + e_t1 and E_t1 at c + e_d + e_t2
        const R et2d = d == 0 ? e2xy : (d == 1 ? e0yz : e1xz);
        const R et1d = d == 0 ? e1xz : (d == 1 ? e2xy : e0yz);
        const TE clo = (widen<TE>(en[t2][t1]) - widen<TE>(ec[t2])) - (widen<TE>(en[t1][t2]) - widen<TE>(ec[t1]));
        const TE chi = (widen<TE>(et2d) - widen<TE>(en[t2][d])) - (widen<TE>(et1d) - widen<TE>(en[t1][d]));
        lo[d] = blo[d] - r * clo;
        const TE hi = bhi[d] - r * chi;
        bc[d] = lo[d] + hi;
    }
}

// divergence of the hydrodynamic fluxes (Eq. 10) of a cell from its lower
// (fc) and upper (fn) faces per axis, sweep frames back to x, y, z: rho and
// M in their storage type TU, the energy in TE
// the contribution of axis d (lower face fc, upper face fn) to the divergence
template <class R, class TU, class TE>
__device__ __forceinline__ void flux_divergence_axis(int d, const R fc[5], const R fn[5], TU du[4], TE& due)
{
    const int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
    du[0] += TU(fn[0] - fc[0]);
    du[1 + d] += TU(fn[1] - fc[1]);
    du[1 + t1] += TU(fn[2] - fc[2]);
    du[1 + t2] += TU(fn[3] - fc[3]);
    due += widen<TE>(fn[4] - fc[4]);
}

template <class R, class TU, class TE>
__device__ __forceinline__ void flux_divergence(const R fc[3][5], const R fn[3][5], TU du[4], TE& due)
{
    du[0] = du[1] = du[2] = du[3] = TU(0);
    due = TE(0);
#pragma unroll
    for (int d = 0; d < 3; d++) flux_divergence_axis<R, TU, TE>(d, fc[d], fn[d], du, due);
}

// half-step cell state U^{n+1/2} = U^n - (dt/2) div F (Eq. 10) and its
// primitives (Eq. 5) with twice the cell-centred half-step field bc;
// ru, r = (dt/2)/dx in the types TU and TE
template <class R, class TU, class TE>
__device__ __forceinline__ void half_prims(TU rho0, TU mx0, TU my0, TU mz0, TE e0, const TU du[4], TE due, TU ru, TE r,
                                           const TE bc[3], double gam, double pfloor, R w[8])
{
    TU rho = rho0 - ru * du[0];
    TU mx = mx0 - ru * du[1], my = my0 - ru * du[2], mz = mz0 - ru * du[3];
    TE e = e0 - r * due;
    const TU irho = TU(1) / rho;
    TU vx = mx * irho, vy = my * irho, vz = mz * irho;
    TE p = TE(gam - 1.0) * (e - kinetic<TU, TE>(rho, irho, mx, my, mz, vx, vy, vz)
                            - TE(0.125) * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]));
    if (pfloor > 0.0 && p < TE(pfloor)) p = TE(pfloor);
    w[0] = R(rho); w[1] = R(vx); w[2] = R(vy); w[3] = R(vz);
    w[4] = narrow<R>(p); w[5] = R(0.5) * narrow<R>(bc[0]);
    w[6] = R(0.5) * narrow<R>(bc[1]); w[7] = R(0.5) * narrow<R>(bc[2]);
}

// ---------------------------------------------------------------------------
// a8 + a1: half-step face field B^{n+1/2} = B^n - (dt/2) curl E (Eq. 13) and
// the half-step cell primitives from U^{n+1/2} = U^n - (dt/2) div F (Eq. 10)
// with the cell-centre B of the updated faces.  Only Bh and Wh are stored.
// ---------------------------------------------------------------------------
template <class R, class TU, class TE, bool OUT = false>
__global__ void __launch_bounds__(CELL_THREADS) k_half(Boxes B, StateP<TU, TE> s, const R* __restrict__ F,
                                                       const R* __restrict__ E, const DtBox* __restrict__ dtb,
                                                       double gam, TE* __restrict__ Bh0, TE* __restrict__ Bh1,
                                                       TE* __restrict__ Bh2, R* __restrict__ Wh, double pfloor = 0.0,
                                                       const R* __restrict__ Fout = nullptr, int cs = 0)
{
    const long long N = B.N;
    for (long long v = blockIdx.x; v < B.nvblk; v += gridDim.x) {
    const int bi = box_of_vblk(B, v);
    BoxDev g = B.b[bi];
    if (!OUT) g.bc = 0;     // periodic instantiation: the wrap is compiled in
    const long long lc = (v - g.vblk0) * CELL_THREADS + threadIdx.x;
    if (lc >= g.n) continue;
    const TE r = DtOf<TE>::hdtdx(dtb[bi]);
    TE* Bh[3] = {Bh0, Bh1, Bh2};
    int i, j, k;
    coords(g, lc, i, j, k);
    const long long c = g.off + lc;
    // every operand is loaded before any arithmetic (independent loads
    // issued together, as in k_full).  Edge fields: E_m at the cell (ec),
    // shifted by +1 along a != m (en), and on the three diagonals the upper
    // faces' circulations need: E_2 at (i+1, j+1, k), E_1 at (i+1, j, k+1),
    // E_0 at (i, j+1, k+1)
    const int ip = bidx(i + 1, g.nx, g.bc & 1), jp = bidx(j + 1, g.ny, g.bc & 2), kp = bidx(k + 1, g.nz, g.bc & 4);
    const long long cp[3] = {cell_of(g, ip, j, k), cell_of(g, i, jp, k), cell_of(g, i, j, kp)};
    R fc[3][5], fn[3][5];
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
        for (int m = 0; m < 5; m++) {
            fc[d][m] = F[((long long)d * 7 + m) * N + c];
            fn[d][m] = F[((long long)d * 7 + m) * N + cp[d]];
        }
    R ec[3], en[3][3];
#pragma unroll
    for (int m = 0; m < 3; m++) {
        ec[m] = E[m * N + c];
#pragma unroll
        for (int a = 0; a < 3; a++)
            if (a != m) en[m][a] = E[m * N + cp[a]];
    }
    const R e2xy = E[2 * N + cell_of(g, ip, jp, k)], e1xz = E[N + cell_of(g, ip, j, kp)],
            e0yz = E[cell_of(g, i, jp, kp)];
    TE blo[3], bhi[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        blo[d] = s.b[d][c];
        bhi[d] = s.b[d][cp[d]];
    }
    const TU rho0 = s.rho[c], mx0 = s.m[0][c], my0 = s.m[1][c], mz0 = s.m[2][c];
    const TE e0 = s.e[c];
    TE lo[3], bc[3];
    half_faces<TE, R>(ec, en, e2xy, e1xz, e0yz, blo, bhi, r, lo, bc);
#pragma unroll
    for (int d = 0; d < 3; d++) Bh[d][c] = lo[d];
    TU du[4];
    TE due;
    flux_divergence<R, TU, TE>(fc, fn, du, due);
    // outflow: the last cell's upper neighbour is the cell itself (a zero
    // difference above); add its outer-face flux instead
    if (g.bc) outer_divergence(g, i, j, k, c, N, F, Fout, cs, du, due);
    R w[8];
    half_prims<R, TU, TE>(rho0, mx0, my0, mz0, e0, du, due, DtOf<TU>::hdtdx(dtb[bi]), r, bc, gam, pfloor, w);
#pragma unroll
    for (int f = 0; f < 8; f++) Wh[f * N + c] = w[f];
    }
}

// full update of one cell: rho and M in their storage type, the energy in
// TE (Eq. 10) from the flux divergence du, due; the face field by CT (Eq. 13),
// the circulation of E around each lower face d in the order of curl_face
// (ec, en as in half_faces); ru, r = dt/dx in the types TU and TE.  u: the
// updated rho, Mx, My, Mz; eb: e and the three lower faces.
template <class R, class TU, class TE>
__device__ __forceinline__ void full_values(TU rho0, TU mx0, TU my0, TU mz0, TE e0, const TE bo[3], const TU du[4],
                                            TE due, const R ec[3], const R en[3][3], TU ru, TE r, TU u[4], TE eb[4])
{
    u[0] = rho0 - ru * du[0];
    u[1] = mx0 - ru * du[1];
    u[2] = my0 - ru * du[2];
    u[3] = mz0 - ru * du[3];
    eb[0] = e0 - r * due;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
        const TE curl = (widen<TE>(en[t2][t1]) - widen<TE>(ec[t2])) - (widen<TE>(en[t1][t2]) - widen<TE>(ec[t1]));
        eb[1 + d] = ct_face(bo[d], r, curl);
    }
}

// full update of cell c in place (full_values, stored)
template <class R, class TU, class TE>
__device__ __forceinline__ void full_cell(const StateP<TU, TE>& s, long long c, TU rho0, TU mx0, TU my0, TU mz0, TE e0,
                                          const TE bo[3], const TU du[4], TE due, const R ec[3], const R en[3][3],
                                          TU ru, TE r)
{
    TU u[4];
    TE eb[4];
    full_values<R, TU, TE>(rho0, mx0, my0, mz0, e0, bo, du, due, ec, en, ru, r, u, eb);
    s.rho[c] = u[0];
    s.m[0][c] = u[1];
    s.m[1][c] = u[2];
    s.m[2][c] = u[3];
    s.e[c] = eb[0];
#pragma unroll
    for (int d = 0; d < 3; d++) s.b[d][c] = eb[1 + d];
}

// ---------------------------------------------------------------------------
// a8 + a1 by x-quads (periodic boxes): k_half's arithmetic for four
// consecutive cells along x per thread, 16-byte loads and stores, the x
// neighbours from the same vectors (as k_full4); one cell per thread in a
// box that is not 16-byte aligned.
// ---------------------------------------------------------------------------
template <class R, class TU, class TE>
__global__ void __launch_bounds__(CELL_THREADS) k_half4(Boxes B, StateP<TU, TE> s, const R* __restrict__ F,
                                                        const R* __restrict__ E, const DtBox* __restrict__ dtb,
                                                        double gam, TE* __restrict__ Bh0, TE* __restrict__ Bh1,
                                                        TE* __restrict__ Bh2, R* __restrict__ Wh, double pfloor)
{
    const long long N = B.N;
    TE* Bh[3] = {Bh0, Bh1, Bh2};
    for (long long v = blockIdx.x; v < B.nvq; v += gridDim.x) {
        const int bi = box_of_vq(B, v);
        BoxDev g = B.b[bi];
        g.bc = 0;
        const TE r = DtOf<TE>::hdtdx(dtb[bi]);
        const TU ru = DtOf<TU>::hdtdx(dtb[bi]);
        if (!g.quad) {                                     // one cell per thread, as k_half
            const long long lc = (v - g.vq0) * CELL_THREADS + threadIdx.x;
            if (lc >= g.n) continue;
            int i, j, k;
            coords(g, lc, i, j, k);
            const long long c = g.off + lc;
            const int ip = wrapi(i + 1, g.nx), jp = wrapi(j + 1, g.ny), kp = wrapi(k + 1, g.nz);
            const long long cp[3] = {cell_of(g, ip, j, k), cell_of(g, i, jp, k), cell_of(g, i, j, kp)};
            R fc[3][5], fn[3][5];
#pragma unroll
            for (int d = 0; d < 3; d++)
#pragma unroll
                for (int m = 0; m < 5; m++) {
                    fc[d][m] = F[((long long)d * 7 + m) * N + c];
                    fn[d][m] = F[((long long)d * 7 + m) * N + cp[d]];
                }
            R ec[3], en[3][3];
#pragma unroll
            for (int m = 0; m < 3; m++) {
                ec[m] = E[m * N + c];
#pragma unroll
                for (int a = 0; a < 3; a++)
                    if (a != m) en[m][a] = E[m * N + cp[a]];
            }
            const R e2xy = E[2 * N + cell_of(g, ip, jp, k)], e1xz = E[N + cell_of(g, ip, j, kp)],
                    e0yz = E[cell_of(g, i, jp, kp)];
            TE blo[3], bhi[3];
#pragma unroll
            for (int d = 0; d < 3; d++) {
                blo[d] = s.b[d][c];
                bhi[d] = s.b[d][cp[d]];
            }
            TE lo[3], bc[3];
            half_faces<TE, R>(ec, en, e2xy, e1xz, e0yz, blo, bhi, r, lo, bc);
#pragma unroll
            for (int d = 0; d < 3; d++) Bh[d][c] = lo[d];
            TU du[4];
            TE due;
            flux_divergence<R, TU, TE>(fc, fn, du, due);
            R w[8];
            half_prims<R, TU, TE>(s.rho[c], s.m[0][c], s.m[1][c], s.m[2][c], s.e[c], du, due, ru, r, bc, gam, pfloor,
                                  w);
#pragma unroll
            for (int f = 0; f < 8; f++) Wh[f * N + c] = w[f];
            continue;
        }
        const long long lc = 4 * ((v - g.vq0) * CELL_THREADS + threadIdx.x);
        if (lc >= g.n) continue;
        int i, j, k;
        coords(g, lc, i, j, k);                            // i: a multiple of 4
        const long long c = g.off + lc;
        const int ix = i + 4 < g.nx ? i + 4 : 0;           // beyond the quad's last cell
        const int jp = wrapi(j + 1, g.ny), kp = wrapi(k + 1, g.nz);
        const long long cx = cell_of(g, ix, j, k), cy = cell_of(g, i, jp, k), cz = cell_of(g, i, j, kp);
        TU du[4][4];
        TE due[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            du[q][0] = du[q][1] = du[q][2] = du[q][3] = TU(0);
            due[q] = TE(0);
        }
#pragma unroll
        for (int d = 0; d < 3; d++) {
            R fc[5][4], fn[5][4];
#pragma unroll
            for (int m = 0; m < 5; m++) {
                const R* Fm = F + ((long long)d * 7 + m) * N;
                ld4(Fm + c, fc[m]);
                if (d == 0) {
                    fn[m][0] = fc[m][1];
                    fn[m][1] = fc[m][2];
                    fn[m][2] = fc[m][3];
                    fn[m][3] = Fm[cx];
                } else {
                    ld4(Fm + (d == 1 ? cy : cz), fn[m]);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const R a[5] = {fc[0][q], fc[1][q], fc[2][q], fc[3][q], fc[4][q]};
                const R b[5] = {fn[0][q], fn[1][q], fn[2][q], fn[3][q], fn[4][q]};
                flux_divergence_axis<R, TU, TE>(d, a, b, du[q], due[q]);
            }
        }
        // edge fields: at the cells' edges, shifted by +1 along a != m, and on
        // the diagonals the upper faces' circulations need
        R ec[3][4], exy[4], exz[4], eyz[4], ezy[4], eyzd[4];
#pragma unroll
        for (int m = 0; m < 3; m++) ld4(E + m * N + c, ec[m]);
        ld4(E + cy, exy);                                   // E_x at y+1
        ld4(E + cz, exz);                                   // E_x at z+1
        ld4(E + N + cz, eyz);                               // E_y at z+1
        ld4(E + 2 * N + cy, ezy);                           // E_z at y+1
        ld4(E + cell_of(g, i, jp, kp), eyzd);               // E_x at (y+1, z+1)
        const R eyx = E[N + cx], ezx = E[2 * N + cx];        // E_y, E_z beyond the quad along x
        const R ezxy = E[2 * N + cell_of(g, ix, jp, k)];     // E_z at (x+1, y+1) beyond the quad
        const R eyxz = E[N + cell_of(g, ix, j, kp)];         // E_y at (x+1, z+1) beyond the quad
        TE b0[4], b1[4], b2[4], b1y[4], b2z[4];
        ld4(s.b[0] + c, b0);
        ld4(s.b[1] + c, b1);
        ld4(s.b[2] + c, b2);
        ld4(s.b[1] + cy, b1y);
        ld4(s.b[2] + cz, b2z);
        const TE b0x = s.b[0][cx];
        TU rho[4], mx[4], my[4], mz[4];
        TE e[4];
        ld4(s.rho + c, rho);
        ld4(s.m[0] + c, mx);
        ld4(s.m[1] + c, my);
        ld4(s.m[2] + c, mz);
        ld4(s.e + c, e);
        TE lo0[4], lo1[4], lo2[4];
        R w[8][4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const R ecq[3] = {ec[0][q], ec[1][q], ec[2][q]};
            R en[3][3];
            en[0][1] = exy[q];
            en[0][2] = exz[q];
            en[1][0] = q < 3 ? ec[1][q + 1] : eyx;
            en[1][2] = eyz[q];
            en[2][0] = q < 3 ? ec[2][q + 1] : ezx;
            en[2][1] = ezy[q];
            en[0][0] = en[1][1] = en[2][2] = R(0);   // unused
            const R e2xy = q < 3 ? ezy[q + 1] : ezxy, e1xz = q < 3 ? eyz[q + 1] : eyxz, e0yz = eyzd[q];
            const TE blo[3] = {b0[q], b1[q], b2[q]};
            const TE bhi[3] = {q < 3 ? b0[q + 1] : b0x, b1y[q], b2z[q]};
            TE lo[3], bc[3];
            half_faces<TE, R>(ecq, en, e2xy, e1xz, e0yz, blo, bhi, r, lo, bc);
            lo0[q] = lo[0];
            lo1[q] = lo[1];
            lo2[q] = lo[2];
            R wq[8];
            half_prims<R, TU, TE>(rho[q], mx[q], my[q], mz[q], e[q], du[q], due[q], ru, r, bc, gam, pfloor, wq);
#pragma unroll
            for (int f = 0; f < 8; f++) w[f][q] = wq[f];
        }
        st4(Bh0 + c, lo0);
        st4(Bh1 + c, lo1);
        st4(Bh2 + c, lo2);
#pragma unroll
        for (int f = 0; f < 8; f++) st4(Wh + f * N + c, w[f]);
    }
}

// ---------------------------------------------------------------------------
// a10: full update U^{n+1} = U^n - dt div F (Eq. 10), B^{n+1} = B^n - dt curl E
// (Eq. 13), in place.
// ---------------------------------------------------------------------------
template <class R, class TU, class TE, bool OUT = false>
__global__ void __launch_bounds__(CELL_THREADS) k_full(Boxes B, StateP<TU, TE> s, const R* __restrict__ F,
                                                       const R* __restrict__ E, const DtBox* __restrict__ dtb,
                                                       const R* __restrict__ Fout = nullptr, int cs = 0)
{
    const long long N = B.N;
    for (long long v = blockIdx.x; v < B.nvblk; v += gridDim.x) {
    const int bi = box_of_vblk(B, v);
    BoxDev g = B.b[bi];
    if (!OUT) g.bc = 0;     // periodic instantiation: the wrap is compiled in
    const long long lc = (v - g.vblk0) * CELL_THREADS + threadIdx.x;
    if (lc >= g.n) continue;
    const TE r = DtOf<TE>::dtdx(dtb[bi]);
    int i, j, k;
    coords(g, lc, i, j, k);
    const long long c = g.off + lc;
    const long long cp[3] = {nbr(g, i, j, k, 0, 1), nbr(g, i, j, k, 1, 1), nbr(g, i, j, k, 2, 1)};
    // every operand is loaded before any arithmetic: the ~45 loads are
    // independent, and issued together they keep the memory system busy
    // (interleaved with the arithmetic, a few at a time, the kernel waited
    // on each group in turn)
    R fc[3][5], fn[3][5];
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
        for (int m = 0; m < 5; m++) {
            fc[d][m] = F[((long long)d * 7 + m) * N + c];
            fn[d][m] = F[((long long)d * 7 + m) * N + cp[d]];
        }
    R ec[3], en[3][3];      // E_m at the cell's edges and at those shifted by +1 along a != m
#pragma unroll
    for (int m = 0; m < 3; m++) {
        ec[m] = E[m * N + c];
#pragma unroll
        for (int a = 0; a < 3; a++)
            if (a != m) en[m][a] = E[m * N + cp[a]];
    }
    const TU rho0 = s.rho[c], mx0 = s.m[0][c], my0 = s.m[1][c], mz0 = s.m[2][c];
    const TE e0 = s.e[c], b00 = s.b[0][c], b10 = s.b[1][c], b20 = s.b[2][c];
    TU du[4];
    TE due;
    flux_divergence<R, TU, TE>(fc, fn, du, due);
    // outflow: the last cell's upper neighbour is the cell itself (a zero
    // difference above); add its outer-face flux instead
    if (g.bc) outer_divergence(g, i, j, k, c, N, F, Fout, cs, du, due);
    const TE bo[3] = {b00, b10, b20};
    full_cell<R, TU, TE>(s, c, rho0, mx0, my0, mz0, e0, bo, du, due, ec, en, DtOf<TU>::dtdx(dtb[bi]), r);
    }
}

// ---------------------------------------------------------------------------
// a10 by x-quads (periodic boxes): each thread updates four consecutive
// cells along x with 16-byte loads and stores, taking the x neighbours of the
// quad's cells from the same vectors (one more element for the last), so a
// load instruction moves four times the bytes of k_full's.  The fluxes come
// axis by axis (the divergence in flux_divergence's order of operations),
// then the edge fields and the state; the arithmetic per cell is k_full's.
// A box that is not 16-byte aligned in every field array (quad = 0) takes
// one cell per thread.
// ---------------------------------------------------------------------------
template <class R, class TU, class TE>
__global__ void __launch_bounds__(CELL_THREADS) k_full4(Boxes B, StateP<TU, TE> s, const R* __restrict__ F,
                                                        const R* __restrict__ E, const DtBox* __restrict__ dtb)
{
    const long long N = B.N;
    for (long long v = blockIdx.x; v < B.nvq; v += gridDim.x) {
        const int bi = box_of_vq(B, v);
        BoxDev g = B.b[bi];
        g.bc = 0;
        const TE r = DtOf<TE>::dtdx(dtb[bi]);
        const TU ru = DtOf<TU>::dtdx(dtb[bi]);
        if (!g.quad) {                                     // one cell per thread
            const long long lc = (v - g.vq0) * CELL_THREADS + threadIdx.x;
            if (lc >= g.n) continue;
            int i, j, k;
            coords(g, lc, i, j, k);
            const long long c = g.off + lc;
            const long long cp[3] = {nbr(g, i, j, k, 0, 1), nbr(g, i, j, k, 1, 1), nbr(g, i, j, k, 2, 1)};
            R fc[3][5], fn[3][5];
#pragma unroll
            for (int d = 0; d < 3; d++)
#pragma unroll
                for (int m = 0; m < 5; m++) {
                    fc[d][m] = F[((long long)d * 7 + m) * N + c];
                    fn[d][m] = F[((long long)d * 7 + m) * N + cp[d]];
                }
            R ec[3], en[3][3];
#pragma unroll
            for (int m = 0; m < 3; m++) {
                ec[m] = E[m * N + c];
#pragma unroll
                for (int a = 0; a < 3; a++)
                    if (a != m) en[m][a] = E[m * N + cp[a]];
            }
            const TE bo[3] = {s.b[0][c], s.b[1][c], s.b[2][c]};
            TU du[4];
            TE due;
            flux_divergence<R, TU, TE>(fc, fn, du, due);
            full_cell<R, TU, TE>(s, c, s.rho[c], s.m[0][c], s.m[1][c], s.m[2][c], s.e[c], bo, du, due, ec, en, ru, r);
            continue;
        }
        const long long lc = 4 * ((v - g.vq0) * CELL_THREADS + threadIdx.x);
        if (lc >= g.n) continue;
        int i, j, k;
        coords(g, lc, i, j, k);                            // i: a multiple of 4
        const long long c = g.off + lc;
        const long long cx = cell_of(g, i + 4 < g.nx ? i + 4 : 0, j, k);   // beyond the quad's last cell
        const long long cy = nbr(g, i, j, k, 1, 1), cz = nbr(g, i, j, k, 2, 1);
        TU du[4][4];
        TE due[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            du[q][0] = du[q][1] = du[q][2] = du[q][3] = TU(0);
            due[q] = TE(0);
        }
#pragma unroll
        for (int d = 0; d < 3; d++) {
            R fc[5][4], fn[5][4];
#pragma unroll
            for (int m = 0; m < 5; m++) {
                const R* Fm = F + ((long long)d * 7 + m) * N;
                ld4(Fm + c, fc[m]);
                if (d == 0) {
                    fn[m][0] = fc[m][1];
                    fn[m][1] = fc[m][2];
                    fn[m][2] = fc[m][3];
                    fn[m][3] = Fm[cx];
                } else {
                    ld4(Fm + (d == 1 ? cy : cz), fn[m]);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const R a[5] = {fc[0][q], fc[1][q], fc[2][q], fc[3][q], fc[4][q]};
                const R b[5] = {fn[0][q], fn[1][q], fn[2][q], fn[3][q], fn[4][q]};
                flux_divergence_axis<R, TU, TE>(d, a, b, du[q], due[q]);
            }
        }
        // edge fields at the cells' edges and at those shifted by +1 along a != m
        R ec[3][4], ey1[4], ez1[4], exy[4], exz[4], eyz[4], ezy[4];
#pragma unroll
        for (int m = 0; m < 3; m++) ld4(E + m * N + c, ec[m]);
        ld4(E + cy, exy);                                   // E_x at y+1
        ld4(E + cz, exz);                                   // E_x at z+1
        ld4(E + N + cz, eyz);                               // E_y at z+1
        ld4(E + 2 * N + cy, ezy);                           // E_z at y+1
        const R eyx = E[N + cx], ezx = E[2 * N + cx];        // E_y, E_z beyond the quad along x
        ey1[0] = ec[1][1]; ey1[1] = ec[1][2]; ey1[2] = ec[1][3]; ey1[3] = eyx;   // E_y at x+1
        ez1[0] = ec[2][1]; ez1[1] = ec[2][2]; ez1[2] = ec[2][3]; ez1[3] = ezx;   // E_z at x+1
        TU rho[4], mx[4], my[4], mz[4];
        TE e[4], b0[4], b1[4], b2[4];
        ld4(s.rho + c, rho);
        ld4(s.m[0] + c, mx);
        ld4(s.m[1] + c, my);
        ld4(s.m[2] + c, mz);
        ld4(s.e + c, e);
        ld4(s.b[0] + c, b0);
        ld4(s.b[1] + c, b1);
        ld4(s.b[2] + c, b2);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const R ecq[3] = {ec[0][q], ec[1][q], ec[2][q]};
            R en[3][3];
            en[0][1] = exy[q];
            en[0][2] = exz[q];
            en[1][0] = ey1[q];
            en[1][2] = eyz[q];
            en[2][0] = ez1[q];
            en[2][1] = ezy[q];
            en[0][0] = en[1][1] = en[2][2] = R(0);   // unused
            const TE bo[3] = {b0[q], b1[q], b2[q]};
            TU u[4];
            TE eb[4];
            full_values<R, TU, TE>(rho[q], mx[q], my[q], mz[q], e[q], bo, du[q], due[q], ecq, en, ru, r, u, eb);
            rho[q] = u[0]; mx[q] = u[1]; my[q] = u[2]; mz[q] = u[3];
            e[q] = eb[0]; b0[q] = eb[1]; b1[q] = eb[2]; b2[q] = eb[3];
        }
        st4(s.rho + c, rho);
        st4(s.m[0] + c, mx);
        st4(s.m[1] + c, my);
        st4(s.m[2] + c, mz);
        st4(s.e + c, e);
        st4(s.b[0] + c, b0);
        st4(s.b[1] + c, b1);
        st4(s.b[2] + c, b2);
    }
}

// ---------------------------------------------------------------------------
// a9 + a6: CTU transverse correction of the traced states of the two cells
// on each d-face, then the corrector Riemann solve with the half-step B_n.
// ---------------------------------------------------------------------------
// the transverse flux differences of cell (si, sj, sk) along the two axes
// other than d, df[0] along t1 and df[1] along t2: F_e(+1) - F_e, or at the
// last cell of an outflow axis e the outer flux minus F_e
template <class R, bool OUT, int d>
__device__ __forceinline__ void ctu_tdiff(const BoxDev& g, int si, int sj, int sk, long long sc,
                                          const R* __restrict__ F1, const R* __restrict__ Fo1, int cs, long long N,
                                          R df[2][7])
{
    const int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
#pragma unroll
    for (int mm = 0; mm < 2; mm++) {
        const int e = mm == 0 ? t1 : t2;
        const R* Fe = F1 + (long long)e * 7 * N;
        int qe;
        if (OUT && outer_cell(g, e, si, sj, sk, qe)) {
            const R* Fo = Fo1 + (long long)e * 7 * cs;
#pragma unroll
            for (int m = 0; m < 7; m++) df[mm][m] = Fo[(long long)m * cs + qe] - Fe[(long long)m * N + sc];
        } else {
            long long sp = nbr(g, si, sj, sk, e, 1);
#pragma unroll
            for (int m = 0; m < 7; m++) df[mm][m] = Fe[(long long)m * N + sp] - Fe[(long long)m * N + sc];
        }
    }
}

// the corrected state of a traced state w (frame of d) of a cell with
// cell-centre B_n bnc and transverse flux differences df: to conserved
// variables in the global frame, minus r = dt/(2 dx) times each difference,
// back to primitive variables in the frame of d
template <class R, int d>
__device__ __forceinline__ void ctu_apply(const R w[7], R bnc, const R df[2][7], R r, R gm1, R wf[7])
{
    const int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
    R v[3], bg[3];
    v[d] = w[1]; v[t1] = w[2]; v[t2] = w[3];
    bg[d] = bnc; bg[t1] = w[5]; bg[t2] = w[6];
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
        q[0] -= r * df[mm][0];
        q[1 + e] -= r * df[mm][1];
        q[1 + e1] -= r * df[mm][2];
        q[1 + e2] -= r * df[mm][3];
        q[4] -= r * df[mm][4];
        q[5 + e1] -= r * df[mm][5];
        q[5 + e2] -= r * df[mm][6];
    }
    R rho = q[0];
    const R irho = R(1) / rho;
    R vx = q[1] * irho, vy = q[2] * irho, vz = q[3] * irho;
    R p = gm1 * (q[4] - R(0.5) * rho * (vx * vx + vy * vy + vz * vz)
                 - R(0.5) * (q[5] * q[5] + q[6] * q[6] + q[7] * q[7]));
    R vg[3] = {vx, vy, vz};
    wf[0] = rho;
    wf[1] = vg[d];
    wf[2] = vg[t1];
    wf[3] = vg[t2];
    wf[4] = p;
    wf[5] = q[5 + t1];
    wf[6] = q[5 + t2];
}

// the traced state w (from WM or WP along d) of cell (si, sj, sk), as 8
// global-frame conserved components with the cell-centre B_n of the cell,
// minus dt/2 times the divergence of the other two axes' stage-1 fluxes
// across the cell (along an outflow axis the last cell's upper face flux is
// the outer one, Fo1), back to sweep-frame primitives
template <class R, bool OUT, int d>
__device__ __forceinline__ void ctu_corrected(const BoxDev& g, int si, int sj, int sk, long long sc,
                                              const R* __restrict__ src, const R* __restrict__ W,
                                              const R* __restrict__ F1, const R* __restrict__ Fo1, int cs,
                                              long long N, R r, R gm1, R wf[7])
{
    R w[7], df[2][7];
#pragma unroll
    for (int m = 0; m < 7; m++) w[m] = src[(long long)m * N + sc];
    ctu_tdiff<R, OUT, d>(g, si, sj, sk, sc, F1, Fo1, cs, N, df);
    ctu_apply<R, d>(w, W[(5 + d) * N + sc], df, r, gm1, wf);
}

// Outflow instantiation (OUT): the transverse corrections of last cells take
// the stage-1 outer fluxes Fo1, and the last cell along an outflow d also
// writes the stage-2 flux of its outer face into Fo2: the Riemann flux of
// its own corrected upper and lower states with the half-step B_n of the
// last face.  The axis d is a template parameter: every frame rotation is
// then static, and the per-state arrays stay in registers.
template <class R, int SOLVER, class TE, int d, bool OUT = false>
__global__ void __launch_bounds__(CELL_THREADS) k_ctu_correct(Boxes B, const R* __restrict__ WM,
                                                              const R* __restrict__ WP, const R* __restrict__ W,
                                                              const R* __restrict__ F1, const TE* __restrict__ Bhd,
                                                              R* __restrict__ F2, const DtBox* __restrict__ dtb,
                                                              double gam, const R* __restrict__ Fo1 = nullptr,
                                                              int cs = 0, R* __restrict__ Fo2 = nullptr)
{
    const long long N = B.N;
    for (long long v = blockIdx.x; v < B.nvblk; v += gridDim.x) {
    const int bi = box_of_vblk(B, v);
    BoxDev g = B.b[bi];
    if (!OUT) g.bc = 0;     // periodic instantiation: the wrap is compiled in
    const long long lc = (v - g.vblk0) * CELL_THREADS + threadIdx.x;
    if (lc >= g.n) continue;
    const R gm1 = R(gam - 1.0), gr = R(gam);
    const R r = DtOf<R>::hdtdx(dtb[bi]);
    int i, j, k;
    coords(g, lc, i, j, k);
    const long long c = g.off + lc;
    R wf[2][7];
    {
        int si = i, sj = j, sk = k;
        if (d == 0) si = bidx(i - 1, g.nx, g.bc & 1); else if (d == 1) sj = bidx(j - 1, g.ny, g.bc & 2);
        else sk = bidx(k - 1, g.nz, g.bc & 4);
        ctu_corrected<R, OUT, d>(g, si, sj, sk, cell_of(g, si, sj, sk), WP, W, F1, Fo1, cs, N, r, gm1, wf[0]);
    }
    ctu_corrected<R, OUT, d>(g, i, j, k, c, WM, W, F1, Fo1, cs, N, r, gm1, wf[1]);
    R f[7];
    riemann<SOLVER>(wf[0], wf[1], R(Bhd[c]), gm1, gr, f);
#pragma unroll
    for (int m = 0; m < 7; m++) F2[(long long)m * N + c] = f[m];
    int qd;
    if (OUT && outer_cell(g, d, i, j, k, qd)) {
        R wu[7], fo[7];
        ctu_corrected<R, OUT, d>(g, i, j, k, c, WP, W, F1, Fo1, cs, N, r, gm1, wu);
        riemann<SOLVER>(wu, wf[1], R(Bhd[c]), gm1, gr, fo);
        R* Fo = Fo2 + (long long)d * 7 * cs;
#pragma unroll
        for (int m = 0; m < 7; m++) Fo[(long long)m * cs + qd] = fo[m];
    }
    }
}

// Pencil form of steps 5-6 along y or z (D = 1, 2), selected by the pencil
// mask as the tracing sweeps are: a thread walks a segment of pencil_len
// faces of a grid line, with lanes along x so that every load is coalesced.
// Each cell's transverse flux differences are loaded once and correct both
// of its traced states (the per-cell form loads and applies them for each
// of the two faces of the cell); the corrected upper state is carried to
// the next face.  The lead-in is the upper state of the cell that i0 - 1
// maps to.  Same arithmetic per state as k_ctu_correct.  The FP32 Roe form
// takes 124-159 registers unbounded (3 blocks of 128 threads per SM along
// y); bounded to 4 blocks it spills at most 36 bytes, and the y pass at 256^3
// went from 0.71 to 0.59 ms.
template <class R, int SOLVER, class TE, int D, bool OUT = false>
__global__ void __launch_bounds__(PENCIL_THREADS, (sizeof(R) == 4 && SOLVER == ROE ? 4 : 0)) k_ctu_pencil(Boxes B, const R* __restrict__ WM,
                                                               const R* __restrict__ WP, const R* __restrict__ W,
                                                               const R* __restrict__ F1, const TE* __restrict__ Bhd,
                                                               R* __restrict__ F2, const DtBox* __restrict__ dtb,
                                                               double gam, const R* __restrict__ Fo1 = nullptr,
                                                               int cs = 0, R* __restrict__ Fo2 = nullptr)
{
    static_assert(D == 1 || D == 2, "the x axis keeps the per-cell form");
    constexpr int d = D;
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gt >= B.npth[d]) return;
    const int bi = box_of_pth(B, d, gt);
    BoxDev g = B.b[bi];
    if (!OUT) g.bc = 0;     // periodic instantiation: the wrap is compiled in
    int na, nb, ns;
    pencil_dims(g.nx, g.ny, g.nz, d, B.pl, na, nb, ns);
    long long t = gt - g.pth0[d];
    const int ia = (int)(t % na);
    t /= na;
    const int ib = (int)(t % nb);
    const int sg = (int)(t / nb);
    const int n = d == 1 ? g.ny : g.nz;
    const bool out = g.bc >> d & 1;
    const int i0 = sg * B.pl;
    const int i1 = i0 + B.pl < n ? i0 + B.pl : n;
    const long long N = B.N;
    const R gm1 = R(gam - 1.0), gr = R(gam);
    const R r = DtOf<R>::hdtdx(dtb[bi]);
    // cell p of the line: x = ia, and (y, z) = (p, ib) or (ib, p)
    auto at = [&](int p, int& i, int& j, int& k) {
        i = ia;
        if (d == 1) { j = p; k = ib; } else { j = ib; k = p; }
    };
    R df[2][7], w[7], wpp[7];
    {
        int si, sj, sk;
        at(bidx(i0 - 1, n, out), si, sj, sk);
        const long long sc = cell_of(g, si, sj, sk);
#pragma unroll
        for (int m = 0; m < 7; m++) w[m] = WP[(long long)m * N + sc];
        ctu_tdiff<R, OUT, d>(g, si, sj, sk, sc, F1, Fo1, cs, N, df);
        ctu_apply<R, d>(w, W[(5 + d) * N + sc], df, r, gm1, wpp);
    }
    for (int p = i0; p < i1; p++) {
        int i, j, k;
        at(p, i, j, k);
        const long long c = cell_of(g, i, j, k);
        ctu_tdiff<R, OUT, d>(g, i, j, k, c, F1, Fo1, cs, N, df);
        const R bnc = W[(5 + d) * N + c];
        const R bface = R(Bhd[c]);
        R wm[7], f[7];
#pragma unroll
        for (int m = 0; m < 7; m++) w[m] = WM[(long long)m * N + c];
        ctu_apply<R, d>(w, bnc, df, r, gm1, wm);
        riemann<SOLVER>(wpp, wm, bface, gm1, gr, f);
#pragma unroll
        for (int m = 0; m < 7; m++) F2[(long long)m * N + c] = f[m];
#pragma unroll
        for (int m = 0; m < 7; m++) w[m] = WP[(long long)m * N + c];
        ctu_apply<R, d>(w, bnc, df, r, gm1, wpp);
        int qd;
        if (OUT && outer_cell(g, d, i, j, k, qd)) {
            riemann<SOLVER>(wpp, wm, bface, gm1, gr, f);
            R* Fo = Fo2 + (long long)d * 7 * cs;
#pragma unroll
            for (int m = 0; m < 7; m++) Fo[(long long)m * cs + qd] = f[m];
        }
    }
}

// Warp form of steps 5-6 along x (x periodic), selected by bit 0 of the
// pencil mask: one warp per grid row marches segments of 31 faces; lane l
// holds cell x0 - 1 + l, loads its transverse flux differences once and
// corrects both of its traced states; the corrected upper state goes to the
// next lane by a shuffle, and lanes 1-31 solve their lower faces.  Same
// arithmetic per state as k_ctu_correct.
template <class R, int SOLVER, class TE, bool OUT = false>
__global__ void __launch_bounds__(PENCIL_THREADS, (sizeof(R) == 4 && SOLVER == ROE ? 4 : 0))
    k_ctu_xwarp(Boxes B, const R* __restrict__ WM, const R* __restrict__ WP, const R* __restrict__ W,
                const R* __restrict__ F1, const TE* __restrict__ Bhd, R* __restrict__ F2,
                const DtBox* __restrict__ dtb, double gam, const R* __restrict__ Fo1 = nullptr, int cs = 0)
{
    constexpr int FW = 31;
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= B.nxr) return;                        // uniform over the warp
    const int bi = box_of_row(B, wid);
    BoxDev g = B.b[bi];
    if (!OUT) g.bc = 0;     // periodic instantiation: the wrap is compiled in
    const long long t = wid - g.xr0;
    const int j = (int)(t % g.ny), k = (int)(t / g.ny);
    const long long N = B.N;
    const R gm1 = R(gam - 1.0), gr = R(gam);
    const R r = DtOf<R>::hdtdx(dtb[bi]);
    const int nseg = (g.nx + FW - 1) / FW;
    for (int sg = 0; sg < nseg; sg++) {
        const int xi = sg * FW - 1 + lane;           // this lane's cell (and the face below it)
        const int i = wrapi(xi, g.nx);
        const long long c = cell_of(g, i, j, k);
        R df[2][7], w[7], wm[7], wp[7], wl[7];
        ctu_tdiff<R, OUT, 0>(g, i, j, k, c, F1, Fo1, cs, N, df);
        const R bnc = W[5 * N + c];
#pragma unroll
        for (int m = 0; m < 7; m++) w[m] = WM[(long long)m * N + c];
        ctu_apply<R, 0>(w, bnc, df, r, gm1, wm);
#pragma unroll
        for (int m = 0; m < 7; m++) w[m] = WP[(long long)m * N + c];
        ctu_apply<R, 0>(w, bnc, df, r, gm1, wp);
        shfl7(wl, wp, 1);                            // the corrected upper state of the cell below
        if (lane >= 1 && xi < g.nx) {
            R f[7];
            riemann<SOLVER>(wl, wm, R(Bhd[c]), gm1, gr, f);
#pragma unroll
            for (int m = 0; m < 7; m++) F2[(long long)m * N + c] = f[m];
        }
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
// Diagnostics of the ABC relaxation and the refinement tests (Sec. 4.3, 4.5):
// per virtual block the sums of e, of B_f^2/2 over the cell's three faces and
// of |M|^2/(2 rho), the maximum of dx |J_cc| / |B_cc| and of dx |J_cc|, and
// the count of cells with dx |J_cc| / |B_cc| > thr.  dx J on an edge along a
// is (B_c(c) - B_c(c - e_b)) - (B_b(c) - B_b(c - e_c)), b = a+1, c = a+2
// (Stokes on the four faces around the edge); J_cc is the mean of the cell's
// four edges along each axis.  All in FP64.
// ---------------------------------------------------------------------------
template <class TE>
__device__ __forceinline__ double edge_j(const BoxDev& g, TE* const* b, int i, int j, int k, int a)
{
    const int bb = a == 2 ? 0 : a + 1, cc = a == 0 ? 2 : a - 1;
    const long long c = cell_of(g, i, j, k);
    return ((double)b[cc][c] - (double)b[cc][nbr(g, i, j, k, bb, -1)])
         - ((double)b[bb][c] - (double)b[bb][nbr(g, i, j, k, cc, -1)]);
}

// block reduction of NF per-thread values (bit f of maxmask: maximum, else
// sum; fixed order) stored at out[0 .. NF-1] by thread 0
template <int NF>
__device__ __forceinline__ void block_reduce_store(const double* acc, unsigned maxmask, double* red, double* out)
{
    for (int f = 0; f < NF; f++) {
        red[threadIdx.x] = acc[f];
        __syncthreads();
        const bool mx = maxmask >> f & 1;
        for (int o = CELL_THREADS / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o)
                red[threadIdx.x] = mx ? fmax(red[threadIdx.x], red[threadIdx.x + o]) : red[threadIdx.x] + red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[f] = red[0];
        __syncthreads();
    }
}

template <class TU, class TE>
__global__ void __launch_bounds__(CELL_THREADS) k_energies(Boxes B, StateP<TU, TE> s, double thr,
                                                           double* __restrict__ part)
{
    // part: [nvblk][6]: sum e, sum B_f^2/2, sum |M|^2/(2 rho), max dx|J|/|B|, count, max dx|J|
    __shared__ double red[CELL_THREADS];
    for (long long v = blockIdx.x; v < B.nvblk; v += gridDim.x) {
        const BoxDev g = B.b[box_of_vblk(B, v)];
        const long long lc = (v - g.vblk0) * CELL_THREADS + threadIdx.x;
        double acc[6] = {0, 0, 0, 0, 0, 0};
        if (lc < g.n) {
            int i, j, k;
            coords(g, lc, i, j, k);
            const long long c = g.off + lc;
            const double rho = (double)s.rho[c];
            const double m0 = (double)s.m[0][c], m1 = (double)s.m[1][c], m2 = (double)s.m[2][c];
            acc[0] = (double)s.e[c];
            acc[2] = 0.5 * (m0 * m0 + m1 * m1 + m2 * m2) / rho;
            double jc2 = 0.0, bc2 = 0.0, ub = 0.0;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const int bb = a == 2 ? 0 : a + 1, cc = a == 0 ? 2 : a - 1;
                const double bf = (double)s.b[a][c];
                ub += 0.5 * bf * bf;
                int ib = i, jb = j, kb = k, ic = i, jc = j, kc = k;
                if (bb == 0) ib = bidx(i + 1, g.nx, g.bc & 1); else if (bb == 1) jb = bidx(j + 1, g.ny, g.bc & 2);
                else kb = bidx(k + 1, g.nz, g.bc & 4);
                if (cc == 0) ic = bidx(i + 1, g.nx, g.bc & 1); else if (cc == 1) jc = bidx(j + 1, g.ny, g.bc & 2);
                else kc = bidx(k + 1, g.nz, g.bc & 4);
                int ibc = ib, jbc = jb, kbc = kb;
                if (cc == 0) ibc = bidx(ib + 1, g.nx, g.bc & 1); else if (cc == 1) jbc = bidx(jb + 1, g.ny, g.bc & 2);
                else kbc = bidx(kb + 1, g.nz, g.bc & 4);
                const double ja = 0.25 * (edge_j(g, s.b, i, j, k, a) + edge_j(g, s.b, ib, jb, kb, a) +
                                          edge_j(g, s.b, ic, jc, kc, a) + edge_j(g, s.b, ibc, jbc, kbc, a));
                const double bcen = 0.5 * (bf + (double)s.b[a][nbr(g, i, j, k, a, 1)]);
                jc2 += ja * ja;
                bc2 += bcen * bcen;
            }
            acc[1] = ub;
            const double jm = sqrt(jc2), r = jm / sqrt(bc2);
            acc[3] = r;
            acc[4] = r > thr ? 1.0 : 0.0;
            acc[5] = jm;
        }
        block_reduce_store<6>(acc, 0x28u, red, part + v * 6);
    }
}

// per-box totals of per-virtual-block parts [nvblk][nf] (bit f of maxmask:
// maximum, else sum), in block order
static __global__ void k_finish_parts(Boxes B, const double* __restrict__ part, int nf, unsigned maxmask,
                                      double* __restrict__ out)
{
    const int b = blockIdx.x;
    const int f = threadIdx.x;
    if (b >= B.nbox || f >= nf) return;
    const long long v0 = B.b[b].vblk0;
    const long long v1 = b + 1 < B.nbox ? B.b[b + 1].vblk0 : B.nvblk;
    const bool mx = maxmask >> f & 1;
    double a = 0.0;
    for (long long v = v0; v < v1; v++) {
        double x = part[v * nf + f];
        a = mx ? fmax(a, x) : a + x;
    }
    out[b * nf + f] = a;
}

// ---------------------------------------------------------------------------
// Pressure-gradient refinement indicator of the magnetised blast run
// (Sec. 5.1): the FP64 gas pressure of every cell from the stored state
// (cell-centre B the mean of the two faces), then per cell
// scale |grad P| / P with grad P by centred differences over 2 dx (a
// neighbour beyond an outflow side is the cell itself), reduced per box to
// its maximum and the numbers of cells above thr * 2^l, l < nlev <= 4.
// ---------------------------------------------------------------------------
template <class TU, class TE, bool OUT>
__global__ void __launch_bounds__(CELL_THREADS) k_pressure(Boxes B, StateP<TU, TE> s, double gam,
                                                           double* __restrict__ P)
{
    for (long long v = blockIdx.x; v < B.nvblk; v += gridDim.x) {
        BoxDev g = B.b[box_of_vblk(B, v)];
        if (!OUT) g.bc = 0;
        const long long lc = (v - g.vblk0) * CELL_THREADS + threadIdx.x;
        if (lc >= g.n) continue;
        int i, j, k;
        coords(g, lc, i, j, k);
        const long long c = g.off + lc;
        const double bx = 0.5 * ((double)s.b[0][c] + (double)s.b[0][nbr(g, i, j, k, 0, 1)]);
        const double by = 0.5 * ((double)s.b[1][c] + (double)s.b[1][nbr(g, i, j, k, 1, 1)]);
        const double bz = 0.5 * ((double)s.b[2][c] + (double)s.b[2][nbr(g, i, j, k, 2, 1)]);
        const double rho = (double)s.rho[c];
        const double mx = (double)s.m[0][c], my = (double)s.m[1][c], mz = (double)s.m[2][c];
        P[c] = (gam - 1.0) * ((double)s.e[c] - 0.5 * (mx * mx + my * my + mz * mz) / rho
                              - 0.5 * (bx * bx + by * by + bz * bz));
    }
}

template <bool OUT>
__global__ void __launch_bounds__(CELL_THREADS) k_pgrad(Boxes B, const double* __restrict__ P, double scale,
                                                        double thr, int nlev, double* __restrict__ part)
{
    // part: [nvblk][5]: max score, then the counts above thr * 2^l
    __shared__ double red[CELL_THREADS];
    for (long long v = blockIdx.x; v < B.nvblk; v += gridDim.x) {
        BoxDev g = B.b[box_of_vblk(B, v)];
        if (!OUT) g.bc = 0;
        const long long lc = (v - g.vblk0) * CELL_THREADS + threadIdx.x;
        double acc[5] = {0, 0, 0, 0, 0};
        if (lc < g.n) {
            int i, j, k;
            coords(g, lc, i, j, k);
            const long long c = g.off + lc;
            double g2 = 0.0;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const double df = P[nbr(g, i, j, k, d, 1)] - P[nbr(g, i, j, k, d, -1)];
                g2 += df * df;
            }
            const double sc = scale * (sqrt(g2) * (0.5 / g.dx)) / P[c];
            acc[0] = sc;
            double t = thr;
#pragma unroll
            for (int l = 0; l < 4; l++, t *= 2.0) acc[1 + l] = l < nlev && sc > t ? 1.0 : 0.0;
        }
        block_reduce_store<5>(acc, 0x1u, red, part + v * 5);
    }
}

// ---------------------------------------------------------------------------
// Magnetic helicity (Sec. 4.5) of one box: the cell-centre field in FP64
// (mean of the two faces per axis) is transformed by a real-to-complex 3-D
// DFT (cuFFT); on the half spectrum, A_k = i k x B_k / |k|^2 (Coulomb gauge,
// no A for k = 0) and H = dx^3 / n sum_k w_k Re(conj(A_k) . B_k), w_k = 2 for
// the modes whose conjugates the half spectrum leaves out, else 1.
// ---------------------------------------------------------------------------
template <class TE>
__global__ void k_bcc(BoxDev g, const TE* __restrict__ b0, const TE* __restrict__ b1, const TE* __restrict__ b2,
                      double* __restrict__ out)
{
    for (long long lc = blockIdx.x * (long long)blockDim.x + threadIdx.x; lc < g.n;
         lc += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        coords(g, lc, i, j, k);
        const long long c = g.off + lc;
        out[lc] = 0.5 * ((double)b0[c] + (double)b0[nbr(g, i, j, k, 0, 1)]);
        out[g.n + lc] = 0.5 * ((double)b1[c] + (double)b1[nbr(g, i, j, k, 1, 1)]);
        out[2 * g.n + lc] = 0.5 * ((double)b2[c] + (double)b2[nbr(g, i, j, k, 2, 1)]);
    }
}

// Bk: 3 half spectra of nz x ny x (nx/2+1) complex values (re, im pairs)
static __global__ void k_helicity_part(int nx, int ny, int nz, double dx, const double2* __restrict__ Bk,
                                       double* __restrict__ part)
{
    __shared__ double red[256];
    const int nxh = nx / 2 + 1;
    const long long m = (long long)nz * ny * nxh;
    const double two_pi = 6.283185307179586;
    const double kfx = two_pi / (nx * dx), kfy = two_pi / (ny * dx), kfz = two_pi / (nz * dx);
    double acc = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < m; q += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(q % nxh);
        const long long r = q / nxh;
        const int iy = (int)(r % ny), iz = (int)(r / ny);
        const int my = iy <= ny / 2 ? iy : iy - ny, mz = iz <= nz / 2 ? iz : iz - nz;
        if (ix == 0 && my == 0 && mz == 0) continue;
        const double kx = kfx * ix, ky = kfy * my, kz = kfz * mz;
        const double k2 = kx * kx + ky * ky + kz * kz;
        const double2 bx = Bk[q], by = Bk[m + q], bz = Bk[2 * m + q];
        // c = k x B (complex); A = i c / k2 = (-Im c, Re c) / k2
        const double cxr = ky * bz.x - kz * by.x, cxi = ky * bz.y - kz * by.y;
        const double cyr = kz * bx.x - kx * bz.x, cyi = kz * bx.y - kx * bz.y;
        const double czr = kx * by.x - ky * bx.x, czi = kx * by.y - ky * bx.y;
        // Re(conj(A).B) = (A_re B_re + A_im B_im) summed, A_re = -c_im/k2, A_im = c_re/k2
        const double v = (-cxi * bx.x + cxr * bx.y - cyi * by.x + cyr * by.y - czi * bz.x + czr * bz.y) / k2;
        const double w = (ix == 0 || (nx % 2 == 0 && ix == nx / 2)) ? 1.0 : 2.0;
        acc += w * v;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
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
