// mhd_yhalf.cuh -- per-cell passes inside the y and z pencils of the step
// (VL, and the CTU dt/2 update).
//
// k_yhalf: the VL half update (Sec. 3.2, VL step 3: B^{n+1/2} by
// Eq. 13 and U^{n+1/2} by Eq. 10 with dt/2, and their primitives, Eq. 5)
// computed inside the corrector's y pencils (VL steps 4-5 along y: PLM
// reconstruction of the half-step state and the Riemann fluxes).
//
// The corrector's face sweeps are bound by instruction issue and the half
// update by HBM bandwidth; as two kernels their times add.  Here each pencil
// thread forms the half-step state of every cell its walk reconstructs from
// U^n, B^n and the predictor's fluxes and edge fields, so that the loads of
// the half update overlap the arithmetic of the reconstruction and the
// Riemann solves of other warps.  The thread stores the half-step
// primitives and the three lower half-step faces of the cells it owns (the
// x and z corrector sweeps and the corrector's edge fields read them), and
// the y fluxes.  A segment of pl faces forms pl + 3 half-step states with
// PLM (its lead-in cells i0 - 2, i0 - 1 and the cell past its end), pl + 5
// with PPM (three lead-in cells, two past its end): the extra ones are
// recomputed where the neighbouring segment owns them.
//
// The arithmetic of each half-step state is k_half's (half_faces,
// flux_divergence, half_prims on the same operands), and of each face the
// PLM pencil's.  The compiler may pair multiplications and additions into
// fused multiply-adds differently in the two kernels, so the states agree
// with the separate kernels' to rounding, not bit for bit (FP64: 1e-14 after
// two steps of a 64 x 48 x 40 ABC box, the most any value moved).
//
// The predictor's y fluxes are still being read (by the lead-in and
// look-ahead cells of neighbouring segments) while the y corrector fluxes
// are written, so these go to a second flux array; the x and z correctors
// then write theirs there too, and the corrector's edge fields and the full
// update read it.
//
// Periodic boxes (one or a batch), PLM and PPM reconstructions.
//
// k_yprim: the primitives at t^n (Eq. 5, with the cell-centred field the
// mean of the two faces) and the CFL signal speeds (Sec. 3.2) inside the
// first-order y predictor pencils, by the same reasoning: each thread forms
// the primitives of its segment's cells and of the one lead-in cell, stores
// those of its own cells (the x and z predictors and the predictor's edge
// fields read them), folds their signal speeds into the box's maximum and
// solves its y faces.  Periodic boxes without a pressure floor (a floored
// cell's energy is raised in place by its owner while a neighbouring
// segment's lead-in may be reading it).
//
// k_zfull: the conservative part of the VL full update (Eq. 10 for rho, M
// and e with dt) inside the corrector's z pencils, the last corrector sweep:
// each thread, having solved the z faces below and above a cell of its
// segment, updates that cell's rho, M and e in place from U^n, the x and y
// corrector fluxes and its own two z fluxes, and stores only the three z
// flux components the corrector's edge fields read (the mass flux and the
// two field fluxes).  The face field then advances by CT (Eq. 13) in k_ct
// or k_ct4, which read only E and B.  A segment of pl faces solves pl + 1
// (its last cell's upper face is the next segment's first).  PLM and PPM;
// in the learned selector's step it is the cheap z corrector, after the full
// scheme's list pass, whose faces it reads for the segments marked full.
//
// k_ctu_yhalf: the CTU dt/2 update (steps 3-4) inside the y pencils of the
// transverse correction and corrector solve, each owned cell's half-step
// state formed once (the y correction needs only the cells' own half-step
// normal field).
#pragma once
#include "mhd_kernels.cuh"

namespace mhd {

// what a cell's half-step state takes from the cell below it along y: the
// predictor's y flux (5 hydrodynamic components), its lower y face, E_x and
// E_z at its edges, E_z at its x + 1 neighbour and E_x at its z + 1
// neighbour.  They are the upper-y operands of the cell below, so a walk
// loads them once.
template <class R, class TE>
struct YCarry {
    R fy[5];
    TE by;
    R ex, ez, ezx, exz;
};

// the half-step state of cell c (its y + 1 neighbour cy, x + 1 and z + 1
// offsets ox, oz) with k_half's arithmetic: the primitives w8 and the three
// lower half-step faces lo; Y holds what it shares with the cell below along
// y and leaves what the cell above takes from it
template <class R, class TU, class TE>
__device__ __forceinline__ void yhalf_state(const StateP<TU, TE>& s, const R* __restrict__ Fp,
                                            const R* __restrict__ E, long long N, long long c, long long cy,
                                            long long ox, long long oz, TE r, TU ru, double gam, double pfloor,
                                            YCarry<R, TE>& Y, R w8[8], TE lo[3])
{
    R fc[3][5], fn[3][5];
#pragma unroll
    for (int m = 0; m < 5; m++) {
        fc[0][m] = Fp[(long long)m * N + c];
        fn[0][m] = Fp[(long long)m * N + c + ox];
        fc[1][m] = Y.fy[m];
        fn[1][m] = Fp[(7LL + m) * N + cy];
        fc[2][m] = Fp[(14LL + m) * N + c];
        fn[2][m] = Fp[(14LL + m) * N + c + oz];
    }
    const R ec[3] = {Y.ex, E[N + c], Y.ez};
    R en[3][3];
    en[0][1] = E[cy];
    en[0][2] = Y.exz;
    en[1][0] = E[N + c + ox];
    en[1][2] = E[N + c + oz];
    en[2][0] = Y.ezx;
    en[2][1] = E[2 * N + cy];
    en[0][0] = en[1][1] = en[2][2] = R(0);   // unused
    const R e2xy = E[2 * N + cy + ox], e1xz = E[N + c + ox + oz], e0yz = E[cy + oz];
    const TE blo[3] = {s.b[0][c], Y.by, s.b[2][c]};
    const TE bhi[3] = {s.b[0][c + ox], s.b[1][cy], s.b[2][c + oz]};
    const TU rho0 = s.rho[c], mx0 = s.m[0][c], my0 = s.m[1][c], mz0 = s.m[2][c];
    const TE e0 = s.e[c];
    TE bc[3];
    half_faces<TE, R>(ec, en, e2xy, e1xz, e0yz, blo, bhi, r, lo, bc);
    TU du[4];
    TE due;
    flux_divergence<R, TU, TE>(fc, fn, du, due);
    half_prims<R, TU, TE>(rho0, mx0, my0, mz0, e0, du, due, ru, r, bc, gam, pfloor, w8);
    // the next cell's operands from below
#pragma unroll
    for (int m = 0; m < 5; m++) Y.fy[m] = fn[1][m];
    Y.by = bhi[1];
    Y.ex = en[0][1];
    Y.ez = en[2][1];
    Y.ezx = e2xy;
    Y.exz = e0yz;
}

// the carry of the walk's first cell c
template <class R, class TU, class TE>
__device__ __forceinline__ void yhalf_carry(const StateP<TU, TE>& s, const R* __restrict__ Fp,
                                            const R* __restrict__ E, long long N, long long c, long long ox,
                                            long long oz, YCarry<R, TE>& Y)
{
#pragma unroll
    for (int m = 0; m < 5; m++) Y.fy[m] = Fp[(7LL + m) * N + c];
    Y.by = s.b[1][c];
    Y.ex = E[c];
    Y.ez = E[2 * N + c];
    Y.ezx = E[2 * N + c + ox];
    Y.exz = E[c + oz];
}

// register bound: as the PLM corrector pencils it extends (FP32 Roe: 4
// blocks of 128 threads, 128 registers with 16 bytes spilled; at 3 blocks
// and 167 registers it ran 0.760 against 0.708 ms at 256^3, at 5 blocks and
// 96 registers, 128 bytes spilled, 0.835 against 0.705; the z and CTU forms
// lost likewise at 5 blocks: 0.84 against 0.68 ms, CTU step 5.67 against
// 5.18 ms)
template <class R, int RECON, int SOLVER>
constexpr int yhalf_min_blocks()
{
    return sweep_min_blocks<R, RECON, SOLVER, 1>();
}

template <class R, class TU, class TE, int RECON, int SOLVER>
__global__ void __launch_bounds__(PENCIL_THREADS, (yhalf_min_blocks<R, RECON, SOLVER>()))
k_yhalf(Boxes B, StateP<TU, TE> s, const R* __restrict__ Fp, const R* __restrict__ E,
        const DtBox* __restrict__ dtb, double gam, double pfloor, TE* __restrict__ Bh0, TE* __restrict__ Bh1,
        TE* __restrict__ Bh2, R* __restrict__ Wh, R* __restrict__ Fy)
{
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gt >= B.npth[1]) return;
    const int bi = box_of_pth(B, 1, gt);
    const BoxDev g = B.b[bi];
    int na, nb, ns;
    pencil_dims(g.nx, g.ny, g.nz, 1, B.pl, na, nb, ns);
    long long t = gt - g.pth0[1];
    const int ix = (int)(t % na);          // the line's x
    t /= na;
    const int iz = (int)(t % nb);          // and z
    const int sg = (int)(t / nb);
    const long long N = B.N;
    const int nx = g.nx, ny = g.ny;
    const long long plane = (long long)nx * ny;
    const long long base = g.off + (long long)iz * plane + ix;     // cell (x, 0, z)
    const long long ox = ix + 1 < nx ? 1 : 1 - nx;                   // to x + 1 (periodic)
    const long long oz = iz + 1 < g.nz ? plane : plane - (long long)g.nz * plane;   // to z + 1
    const int i0 = sg * B.pl;
    const int i1 = i0 + B.pl < ny ? i0 + B.pl : ny;
    const TE r = DtOf<TE>::hdtdx(dtb[bi]);
    const TU ru = DtOf<TU>::hdtdx(dtb[bi]);
    const R gr = R(gam), gm1 = R(gam - 1.0);

    YCarry<R, TE> Y;   // the walk's first cell: two lead-in cells for PLM, three for PPM
    yhalf_carry<R, TU, TE>(s, Fp, E, N, base + (long long)wrapi(i0 - (RECON == PPM ? 3 : 2), ny) * nx, ox, oz, Y);
    // the half-step state of line cell i (the next one along the walk after
    // the previous call): w and bn in the y sweep frame, lo the lower y face;
    // stored when the segment owns the cell
    auto half_cell = [&](int i, R w[7], R& bn, TE& lo_y) {
        const long long c = base + (long long)wrapi(i, ny) * nx;
        const long long cy = base + (long long)wrapi(i + 1, ny) * nx;
        R w8[8];
        TE lo[3];
        yhalf_state<R, TU, TE>(s, Fp, E, N, c, cy, ox, oz, r, ru, gam, pfloor, Y, w8, lo);
        if (i >= i0 && i < i1) {
            Bh0[c] = lo[0];
            Bh1[c] = lo[1];
            Bh2[c] = lo[2];
#pragma unroll
            for (int f = 0; f < 8; f++) Wh[f * N + c] = w8[f];
        }
        // the y sweep frame (as load_rot with d = 1)
        w[0] = w8[0]; w[1] = w8[2]; w[2] = w8[3]; w[3] = w8[1];
        w[4] = w8[4]; w[5] = w8[7]; w[6] = w8[5];
        bn = w8[6];
        lo_y = lo[1];
    };

    if constexpr (RECON == PPM) {
        // PPM walk as the corrector pencil: cells i-1 .. i+2 and the
        // characteristic slopes of i-1 .. i+1 in registers, wpp the "+" state
        // of cell i-1; a segment forms pl + 5 half-step states (cells i0 - 3
        // .. i1 + 1), the lead-in's slopes serving the window as they are
        R w0[7], w1[7], w2[7], w3[7], wq[7], b0, b1, b2, b3, bq;
        R s0[7], s1[7], s2[7], wpp[7], wm[7], wp[7], f[7];
        TE l1, l2, l3, ldum;
        half_cell(i0 - 3, wq, bq, ldum);
        half_cell(i0 - 2, w0, b0, ldum);
        half_cell(i0 - 1, w1, b1, l1);
        half_cell(i0, w2, b2, l2);
        half_cell(i0 + 1, w3, b3, l3);
        char_slope(wq, w0, w1, b0, gr, s0);                 // slope of i0 - 2
        char_slope(w0, w1, w2, b1, gr, s1);                 // i0 - 1
        char_slope(w1, w2, w3, b2, gr, s2);                 // i0
        recon_cell<PPM, false>(w0, w1, w2, b1, gr, s0, s1, s2, R(0), wm, wpp);   // "+" of cell i0 - 1
        copy7(w0, w1); b0 = b1;
        copy7(w1, w2); b1 = b2; l1 = l2;
        copy7(w2, w3); b2 = b3; l2 = l3;
        copy7(s0, s1);
        copy7(s1, s2);
        for (int i = i0; i < i1; i++) {
            const long long ci = base + (long long)i * nx;
            half_cell(i + 2, w3, b3, l3);
            char_slope(w1, w2, w3, b2, gr, s2);             // slope of i + 1
            recon_cell<PPM, false>(w0, w1, w2, b1, gr, s0, s1, s2, R(0), wm, wp);
            riemann<SOLVER>(wpp, wm, R(l1), gm1, gr, f);
#pragma unroll
            for (int m = 0; m < 7; m++) Fy[(long long)m * N + ci] = f[m];
            copy7(wpp, wp);
            copy7(w0, w1); b0 = b1;
            copy7(w1, w2); b1 = b2; l1 = l2;
            copy7(w2, w3); b2 = b3; l2 = l3;
            copy7(s0, s1);
            copy7(s1, s2);
        }
        (void)bq;
        (void)b0;
        return;
    }
    // PLM walk as the corrector pencil: cells i-1, i, i+1 in registers, wpp
    // the "+" state of cell i-1.  The cell i+1 is formed just before face i
    // is solved: forming cell i+2 one face ahead (as the plain pencil loads
    // it) held more registers and ran slower, 0.789 against 0.708 ms at
    // 256^3 FP32 Roe, the other warps hiding the loads' latency instead
    R wa[7], wb[7], wc[7], bna, bnb, bnc, wpp[7], wm[7], wp[7];
    TE lb, lc, ldum;
    R dum[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};   // slopes: unused by PLM
    half_cell(i0 - 2, wa, bna, ldum);
    half_cell(i0 - 1, wb, bnb, ldum);
    half_cell(i0, wc, bnc, lc);
    recon_cell<RECON, false>(wa, wb, wc, bnb, gr, dum, dum, dum, R(0), wm, wpp);   // "+" of cell i0 - 1
    copy7(wa, wb); bna = bnb;
    copy7(wb, wc); bnb = bnc; lb = lc;
    R f[7];
    for (int i = i0; i < i1; i++) {
        const long long ci = base + (long long)i * nx;
        half_cell(i + 1, wc, bnc, lc);
        recon_cell<RECON, false>(wa, wb, wc, bnb, gr, dum, dum, dum, R(0), wm, wp);
        riemann<SOLVER>(wpp, wm, R(lb), gm1, gr, f);
#pragma unroll
        for (int m = 0; m < 7; m++) Fy[(long long)m * N + ci] = f[m];
        copy7(wpp, wp);
        copy7(wa, wb); bna = bnb;
        copy7(wb, wc); bnb = bnc; lb = lc;
    }
    (void)bna;
}

// the primitives of one cell (Eq. 5) from rho, M, e and twice its
// cell-centred field, as k_prim forms them
template <class R, class TU, class TE>
__device__ __forceinline__ void cell_prims(TU rho, TU mx, TU my, TU mz, TE e, TE sx, TE sy, TE sz, double gam,
                                           R w[8])
{
    const TU irho = TU(1) / rho;
    const TU vx = mx * irho, vy = my * irho, vz = mz * irho;
    const TE p = cell_pressure<TU, TE>(rho, irho, mx, my, mz, vx, vy, vz, e, sx, sy, sz, gam);
    w[0] = R(rho); w[1] = R(vx); w[2] = R(vy); w[3] = R(vz); w[4] = narrow<R>(p);
    w[5] = R(0.5) * narrow<R>(sx); w[6] = R(0.5) * narrow<R>(sy); w[7] = R(0.5) * narrow<R>(sz);
}

template <class R, class TU, class TE, int SOLVER>
__global__ void __launch_bounds__(PENCIL_THREADS, (sweep_min_blocks<R, PLM, SOLVER, 0>()))
k_yprim(Boxes B, StateP<TU, TE> s, R* __restrict__ W, double gam, unsigned long long* __restrict__ smax_acc,
        unsigned long long* __restrict__ bad_cell, R* __restrict__ Fy)
{
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool live = gt < B.npth[1];      // the live threads are a prefix of each warp
    int bi = -1;
    double smax = 0.0;
    if (live) {
        bi = box_of_pth(B, 1, gt);
        const BoxDev g = B.b[bi];
        int na, nb, ns;
        pencil_dims(g.nx, g.ny, g.nz, 1, B.pl, na, nb, ns);
        long long t = gt - g.pth0[1];
        const int ix = (int)(t % na);
        t /= na;
        const int iz = (int)(t % nb);
        const int sg = (int)(t / nb);
        const long long N = B.N;
        const int nx = g.nx, ny = g.ny;
        const long long plane = (long long)nx * ny;
        const long long base = g.off + (long long)iz * plane + ix;
        const long long ox = ix + 1 < nx ? 1 : 1 - nx;
        const long long oz = iz + 1 < g.nz ? plane : plane - (long long)g.nz * plane;
        const int i0 = sg * B.pl;
        const int i1 = i0 + B.pl < ny ? i0 + B.pl : ny;
        const R gr = R(gam), gm1 = R(gam - 1.0);
        // the lower y face of the walk's next cell (the upper face of the one before)
        TE by = s.b[1][base + (long long)wrapi(i0 - 1, ny) * nx];
        // the primitives of line cell i in the y sweep frame (as load_rot with
        // d = 1), its lower y face in fb; stored, checked and counted in the
        // CFL maximum when the segment owns the cell
        auto prim_cell = [&](int i, R w[7], TE& fb) {
            const long long c = base + (long long)wrapi(i, ny) * nx;
            const long long cy = base + (long long)wrapi(i + 1, ny) * nx;
            const TE byu = s.b[1][cy];
            const TE sx = s.b[0][c] + s.b[0][c + ox];
            const TE sy = by + byu;
            const TE sz = s.b[2][c] + s.b[2][c + oz];
            R w8[8];
            cell_prims<R, TU, TE>(s.rho[c], s.m[0][c], s.m[1][c], s.m[2][c], s.e[c], sx, sy, sz, gam, w8);
            if (i >= i0 && i < i1) {
#pragma unroll
                for (int f = 0; f < 8; f++) W[f * N + c] = w8[f];
                if (!(w8[0] > R(0)) || !(w8[4] > R(0))) atomicMin(bad_cell, (unsigned long long)c);
                if (smax_acc) smax = fmax(smax, (double)cell_signal(w8, gam));
            }
            w[0] = w8[0]; w[1] = w8[2]; w[2] = w8[3]; w[3] = w8[1];
            w[4] = w8[4]; w[5] = w8[7]; w[6] = w8[5];
            fb = by;
            by = byu;
        };
        // first-order states: face i sees cells i - 1 and i
        R wl[7], wr[7], f[7];
        TE fdum, fb;
        prim_cell(i0 - 1, wl, fdum);
        for (int i = i0; i < i1; i++) {
            prim_cell(i, wr, fb);
            riemann<SOLVER>(wl, wr, R(fb), gm1, gr, f);
            const long long ci = base + (long long)i * nx;
#pragma unroll
            for (int m = 0; m < 7; m++) Fy[(long long)m * N + ci] = f[m];
            copy7(wl, wr);
        }
    }
    if (!smax_acc) return;
    // the warp's maximum into its box's accumulator (the bits of a double
    // >= 0 order as its value); a warp across two boxes folds lane by lane
    const int b0 = __shfl_sync(0xffffffffu, bi, 0);
    if (__all_sync(0xffffffffu, !live || bi == b0)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
        if (!(smax > 0.0)) smax = 0.0;
        if ((threadIdx.x & 31) == 0 && b0 >= 0)
            atomicMax(smax_acc + b0, (unsigned long long)__double_as_longlong(smax));
    } else if (live) {
        if (!(smax > 0.0)) smax = 0.0;
        atomicMax(smax_acc + bi, (unsigned long long)__double_as_longlong(smax));
    }
}

// the conservative full update of one cell from its U^n and flux
// divergence (full_values without the face field)
template <class TU, class TE>
__device__ __forceinline__ void full_hydro(TU rho0, TU mx0, TU my0, TU mz0, TE e0, const TU du[4], TE due, TU ru,
                                           TE r, TU u[4], TE& e)
{
    u[0] = rho0 - ru * du[0];
    u[1] = mx0 - ru * du[1];
    u[2] = my0 - ru * du[2];
    u[3] = mz0 - ru * du[3];
    e = e0 - r * due;
}

template <class R, class TU, class TE, int RECON, int SOLVER>
__global__ void __launch_bounds__(PENCIL_THREADS, (sweep_min_blocks<R, RECON, SOLVER, 1>()))
k_zfull(Boxes B, StateP<TU, TE> s, const R* __restrict__ Wh, const TE* __restrict__ Bhz, R* __restrict__ F,
        const DtBox* __restrict__ dtb, double gam, const unsigned char* __restrict__ skip = nullptr)
{
    constexpr int d = 2;
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gt >= B.npth[d]) return;
    const int bi = box_of_pth(B, d, gt);
    const BoxDev g = B.b[bi];
    int na, nb, ns;
    pencil_dims(g.nx, g.ny, g.nz, d, B.pl, na, nb, ns);
    long long t = gt - g.pth0[d];
    const int ix = (int)(t % na);          // the line's x
    t /= na;
    const int iy = (int)(t % nb);          // and y
    const int sg = (int)(t / nb);
    Pencil p;
    p.base = g.off + (long long)iy * g.nx + ix;
    p.stride = (long long)g.nx * g.ny;
    p.n = g.nz;
    p.out = 0;
    const long long N = B.N;
    const long long ox = ix + 1 < g.nx ? 1 : 1 - g.nx;                               // to x + 1
    const long long oy = iy + 1 < g.ny ? g.nx : g.nx - (long long)g.ny * g.nx;        // to y + 1
    const int i0 = sg * B.pl;
    const int i1 = i0 + B.pl < p.n ? i0 + B.pl : p.n;
    const TE r = DtOf<TE>::dtdx(dtb[bi]);
    const TU ru = DtOf<TU>::dtdx(dtb[bi]);
    const R gr = R(gam), gm1 = R(gam - 1.0);
    R* Fz = F + 14 * N;
    // The learned selector's step (skip given): the segments it marks full
    // had their faces solved by the full scheme's list pass, launched before
    // this kernel; their fluxes are read from F instead of this walk's, and
    // not stored.  The face past a segment belongs to the next segment of the
    // line (the first one past the line's end), and is read from F when that
    // one is marked.
    const bool full = skip && skip[gt];
    const bool next_full = skip && skip[g.pth0[d] + ix + (long long)na * (iy + (long long)nb * ((sg + 1) % ns))];
    // cell c (line cell i - 1) from its two z fluxes fl (lower) and fu (upper)
    auto update = [&](long long c, const R fl[7], const R fu[7]) {
        R fc[3][5], fn[3][5];
#pragma unroll
        for (int m = 0; m < 5; m++) {
            fc[0][m] = F[(long long)m * N + c];
            fn[0][m] = F[(long long)m * N + c + ox];
            fc[1][m] = F[(7LL + m) * N + c];
            fn[1][m] = F[(7LL + m) * N + c + oy];
            fc[2][m] = fl[m];
            fn[2][m] = fu[m];
        }
        const TU rho0 = s.rho[c], mx0 = s.m[0][c], my0 = s.m[1][c], mz0 = s.m[2][c];
        const TE e0 = s.e[c];
        TU du[4];
        TE due;
        flux_divergence<R, TU, TE>(fc, fn, du, due);
        TU u[4];
        TE e;
        full_hydro<TU, TE>(rho0, mx0, my0, mz0, e0, du, due, ru, r, u, e);
        s.rho[c] = u[0];
        s.m[0][c] = u[1];
        s.m[1][c] = u[2];
        s.m[2][c] = u[3];
        s.e[c] = e;
    };
    // face i's flux f: the full scheme's (read) or this walk's (its own
    // faces' components stored); then the update of cell i - 1
    R f[7], fprev[7];
    auto face_done = [&](int i, long long ci) {
        if (i < i1 ? full : next_full) {    // the full scheme's face
#pragma unroll
            for (int m = 0; m < 5; m++) f[m] = Fz[(long long)m * N + ci];
        } else if (i < i1) {                // the components the edge fields read
            Fz[ci] = f[0];
            Fz[5 * N + ci] = f[5];
            Fz[6 * N + ci] = f[6];
        }
        if (i > i0) update(pcell(p, i - 1), fprev, f);
        copy7(fprev, f);
    };
    if constexpr (RECON == PPM) {
        // PPM walk as the corrector pencil, one face further: cells i-1 ..
        // i+2 and the slopes of i-1 .. i+1, wpp the "+" state of cell i-1;
        // the cell i+3 loaded while face i is solved
        R w0[7], w1[7], w2[7], w3[7], wq[7], b0, b1, b2, b3, bq, s0[7], s1[7], s2[7], wpp[7], wm[7], wp[7];
        load_rot(Wh, N, pcell(p, i0 - 3), d, wq, bq);
        load_rot(Wh, N, pcell(p, i0 - 2), d, w0, b0);
        load_rot(Wh, N, pcell(p, i0 - 1), d, w1, b1);
        load_rot(Wh, N, pcell(p, i0), d, w2, b2);
        load_rot(Wh, N, pcell(p, i0 + 1), d, w3, b3);
        char_slope(wq, w0, w1, b0, gr, s0);                 // slope of i0 - 2
        char_slope(w0, w1, w2, b1, gr, s1);                 // i0 - 1
        char_slope(w1, w2, w3, b2, gr, s2);                 // i0
        recon_cell<PPM, false>(w0, w1, w2, b1, gr, s0, s1, s2, R(0), wm, wpp);   // "+" of cell i0 - 1
        copy7(w0, w1); b0 = b1;
        copy7(w1, w2); b1 = b2;
        copy7(w2, w3); b2 = b3;
        copy7(s0, s1);
        copy7(s1, s2);
        R wn[7], bnn;
        load_rot(Wh, N, pcell(p, i0 + 2), d, wn, bnn);
        for (int i = i0; i <= i1; i++) {
            const long long ci = pcell(p, i);
            copy7(w3, wn);
            b3 = bnn;
            if (i < i1) load_rot(Wh, N, pcell(p, i + 3), d, wn, bnn);
            char_slope(w1, w2, w3, b2, gr, s2);             // slope of i + 1
            recon_cell<PPM, false>(w0, w1, w2, b1, gr, s0, s1, s2, R(0), wm, wp);
            riemann<SOLVER>(wpp, wm, R(Bhz[ci]), gm1, gr, f);
            face_done(i, ci);
            copy7(wpp, wp);
            copy7(w0, w1); b0 = b1;
            copy7(w1, w2); b1 = b2;
            copy7(w2, w3); b2 = b3;
            copy7(s0, s1);
            copy7(s1, s2);
        }
        (void)bq;
        (void)b0;
        return;
    }
    // PLM walk as the corrector pencil, one face further: cells i-1, i, i+1
    // in registers, wpp the "+" state of cell i-1; the cell i+2 loaded while
    // face i is solved
    R wa[7], wb[7], wc[7], bna, bnb, bnc, wpp[7], wm[7], wp[7];
    R dum[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};   // slopes: unused by PLM
    load_rot(Wh, N, pcell(p, i0 - 2), d, wa, bna);
    load_rot(Wh, N, pcell(p, i0 - 1), d, wb, bnb);
    load_rot(Wh, N, pcell(p, i0), d, wc, bnc);
    recon_cell<RECON, false>(wa, wb, wc, bnb, gr, dum, dum, dum, R(0), wm, wpp);   // "+" of cell i0 - 1
    copy7(wa, wb); bna = bnb;
    copy7(wb, wc); bnb = bnc;
    R wn[7], bnn;
    load_rot(Wh, N, pcell(p, i0 + 1), d, wn, bnn);
    for (int i = i0; i <= i1; i++) {
        const long long ci = pcell(p, i);
        copy7(wc, wn);
        bnc = bnn;
        if (i < i1) load_rot(Wh, N, pcell(p, i + 2), d, wn, bnn);
        recon_cell<RECON, false>(wa, wb, wc, bnb, gr, dum, dum, dum, R(0), wm, wp);
        riemann<SOLVER>(wpp, wm, R(Bhz[ci]), gm1, gr, f);
        face_done(i, ci);
        copy7(wpp, wp);
        copy7(wa, wb); bna = bnb;
        copy7(wb, wc); bnb = bnc;
    }
    (void)bna;
}

// CT (Eq. 13) of the three lower faces of every cell with dt, from E and
// B^n, in place: full_values' face arithmetic, for the step whose
// conservative update ran in the z corrector (k_zfull).  By x-quads (16-byte
// loads, the x neighbours from the same vectors) in boxes that are 16-byte
// aligned with an FP32 field, one cell per thread elsewhere.
template <class R, class TE>
__device__ __forceinline__ void ct_faces(const R ec[3], const R en[3][3], const TE bo[3], TE r, TE bn[3])
{
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const int t1 = d == 2 ? 0 : d + 1, t2 = d == 0 ? 2 : d - 1;
        const TE curl = (widen<TE>(en[t2][t1]) - widen<TE>(ec[t2])) - (widen<TE>(en[t1][t2]) - widen<TE>(ec[t1]));
        bn[d] = ct_face(bo[d], r, curl);
    }
}

// one cell of k_ct / k_ct4's one-cell path: its three lower faces
template <class R, class TU, class TE>
__device__ __forceinline__ void ct_cell(const BoxDev& g, long long N, const StateP<TU, TE>& s,
                                        const R* __restrict__ E, long long lc, TE r)
{
    int i, j, k;
    coords(g, lc, i, j, k);
    const long long c = g.off + lc;
    const long long cp[3] = {nbr(g, i, j, k, 0, 1), nbr(g, i, j, k, 1, 1), nbr(g, i, j, k, 2, 1)};
    R ec[3], en[3][3];
#pragma unroll
    for (int m = 0; m < 3; m++) {
        ec[m] = E[m * N + c];
#pragma unroll
        for (int a = 0; a < 3; a++)
            if (a != m) en[m][a] = E[m * N + cp[a]];
    }
    const TE bo[3] = {s.b[0][c], s.b[1][c], s.b[2][c]};
    TE bn[3];
    ct_faces<R, TE>(ec, en, bo, r, bn);
#pragma unroll
    for (int d = 0; d < 3; d++) s.b[d][c] = bn[d];
}

template <class R, class TU, class TE>
__global__ void __launch_bounds__(CELL_THREADS) k_ct(Boxes B, StateP<TU, TE> s, const R* __restrict__ E,
                                                     const DtBox* __restrict__ dtb)
{
    for (long long v = blockIdx.x; v < B.nvblk; v += gridDim.x) {
        const int bi = box_of_vblk(B, v);
        BoxDev g = B.b[bi];
        g.bc = 0;
        const long long lc = (v - g.vblk0) * CELL_THREADS + threadIdx.x;
        if (lc < g.n) ct_cell<R, TU, TE>(g, B.N, s, E, lc, DtOf<TE>::dtdx(dtb[bi]));
    }
}

template <class R, class TU, class TE>
__global__ void __launch_bounds__(CELL_THREADS) k_ct4(Boxes B, StateP<TU, TE> s, const R* __restrict__ E,
                                                      const DtBox* __restrict__ dtb)
{
    static_assert(sizeof(TE) == 4, "x-quads of the FP32 field");
    const long long N = B.N;
    for (long long v = blockIdx.x; v < B.nvq; v += gridDim.x) {
        const int bi = box_of_vq(B, v);
        BoxDev g = B.b[bi];
        g.bc = 0;
        const TE r = DtOf<TE>::dtdx(dtb[bi]);
        if (!g.quad) {                                     // one cell per thread
            const long long lc = (v - g.vq0) * CELL_THREADS + threadIdx.x;
            if (lc < g.n) ct_cell<R, TU, TE>(g, N, s, E, lc, r);
            continue;
        }
        const long long lc = 4 * ((v - g.vq0) * CELL_THREADS + threadIdx.x);
        if (lc >= g.n) continue;
        int i, j, k;
        coords(g, lc, i, j, k);                            // i: a multiple of 4
        const long long c = g.off + lc;
        const long long cx = cell_of(g, i + 4 < g.nx ? i + 4 : 0, j, k);
        const long long cy = nbr(g, i, j, k, 1, 1), cz = nbr(g, i, j, k, 2, 1);
        R ec[3][4], exy[4], exz[4], eyz[4], ezy[4];
#pragma unroll
        for (int m = 0; m < 3; m++) ld4(E + m * N + c, ec[m]);
        ld4(E + cy, exy);                                   // E_x at y+1
        ld4(E + cz, exz);                                   // E_x at z+1
        ld4(E + N + cz, eyz);                               // E_y at z+1
        ld4(E + 2 * N + cy, ezy);                           // E_z at y+1
        const R eyx = E[N + cx], ezx = E[2 * N + cx];        // E_y, E_z beyond the quad along x
        TE b0[4], b1[4], b2[4];
        ld4(s.b[0] + c, b0);
        ld4(s.b[1] + c, b1);
        ld4(s.b[2] + c, b2);
        TE o0[4], o1[4], o2[4];
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
            const TE bo[3] = {b0[q], b1[q], b2[q]};
            TE bn[3];
            ct_faces<R, TE>(ecq, en, bo, r, bn);
            o0[q] = bn[0];
            o1[q] = bn[1];
            o2[q] = bn[2];
        }
        st4(s.b[0] + c, o0);
        st4(s.b[1] + c, o1);
        st4(s.b[2] + c, o2);
    }
}

// CTU (Sec. 3.2, steps 3-6 along y): the dt/2 update (k_half's arithmetic,
// through yhalf_state) inside the y pencils of the transverse correction and
// corrector solve (k_ctu_pencil's arithmetic).  The correction of a y face
// takes the half-step normal field of the face's cell, which the walk forms
// with the cell's whole half-step state; each cell is formed once, by the
// segment that owns it, which stores its half-step primitives and faces for
// the x and z corrections and the corrector's edge fields.  Periodic boxes.
template <class R, class TU, class TE, int SOLVER>
__global__ void __launch_bounds__(PENCIL_THREADS, (sizeof(R) == 4 && SOLVER == ROE ? 4 : 0))
k_ctu_yhalf(Boxes B, StateP<TU, TE> s, const R* __restrict__ WM, const R* __restrict__ WP, const R* __restrict__ W,
            const R* __restrict__ F1, const R* __restrict__ E, R* __restrict__ F2, const DtBox* __restrict__ dtb,
            double gam, double pfloor, TE* __restrict__ Bh0, TE* __restrict__ Bh1, TE* __restrict__ Bh2,
            R* __restrict__ Wh)
{
    constexpr int d = 1;
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gt >= B.npth[d]) return;
    const int bi = box_of_pth(B, d, gt);
    BoxDev g = B.b[bi];
    g.bc = 0;
    int na, nb, ns;
    pencil_dims(g.nx, g.ny, g.nz, d, B.pl, na, nb, ns);
    long long t = gt - g.pth0[d];
    const int ia = (int)(t % na);          // x
    t /= na;
    const int ib = (int)(t % nb);          // z
    const int sg = (int)(t / nb);
    const int n = g.ny, nx = g.nx;
    const int i0 = sg * B.pl;
    const int i1 = i0 + B.pl < n ? i0 + B.pl : n;
    const long long N = B.N;
    const long long plane = (long long)nx * n;
    const long long base = g.off + (long long)ib * plane + ia;
    const long long ox = ia + 1 < nx ? 1 : 1 - nx;
    const long long oz = ib + 1 < g.nz ? plane : plane - (long long)g.nz * plane;
    const R gm1 = R(gam - 1.0), gr = R(gam);
    const R r = DtOf<R>::hdtdx(dtb[bi]);
    const TE rh = DtOf<TE>::hdtdx(dtb[bi]);
    const TU ruh = DtOf<TU>::hdtdx(dtb[bi]);
    R df[2][7], w[7], wpp[7];
    {
        const int sj = wrapi(i0 - 1, n);
        const long long sc = base + (long long)sj * nx;
#pragma unroll
        for (int m = 0; m < 7; m++) w[m] = WP[(long long)m * N + sc];
        ctu_tdiff<R, false, d>(g, ia, sj, ib, sc, F1, nullptr, 0, N, df);
        ctu_apply<R, d>(w, W[(5 + d) * N + sc], df, r, gm1, wpp);
    }
    YCarry<R, TE> Y;
    yhalf_carry<R, TU, TE>(s, F1, E, N, base + (long long)i0 * nx, ox, oz, Y);
    for (int p = i0; p < i1; p++) {
        const long long c = base + (long long)p * nx;
        const long long cy = base + (long long)wrapi(p + 1, n) * nx;
        R w8[8];
        TE lo[3];
        yhalf_state<R, TU, TE>(s, F1, E, N, c, cy, ox, oz, rh, ruh, gam, pfloor, Y, w8, lo);
        Bh0[c] = lo[0];
        Bh1[c] = lo[1];
        Bh2[c] = lo[2];
#pragma unroll
        for (int f = 0; f < 8; f++) Wh[f * N + c] = w8[f];
        ctu_tdiff<R, false, d>(g, ia, p, ib, c, F1, nullptr, 0, N, df);
        const R bnc = W[(5 + d) * N + c];
        const R bface = R(lo[1]);
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
    }
}

// CTU (steps 5-7 along z): the transverse correction and corrector solve of
// the z faces (k_ctu_pencil's arithmetic) with the conservative part of the
// full update, as k_zfull does for VL: one face past the segment, each cell
// updated in place once its two z faces are solved, from U^n, the x and y
// corrector fluxes and its own z fluxes; only the three z flux components
// the edge fields read are stored.  Periodic boxes.
template <class R, class TU, class TE, int SOLVER>
__global__ void __launch_bounds__(PENCIL_THREADS, (sizeof(R) == 4 && SOLVER == ROE ? 4 : 0))
k_ctu_zfull(Boxes B, StateP<TU, TE> s, const R* __restrict__ WM, const R* __restrict__ WP, const R* __restrict__ W,
            const R* __restrict__ F1, const TE* __restrict__ Bhz, R* __restrict__ F2, const DtBox* __restrict__ dtb,
            double gam)
{
    constexpr int d = 2;
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gt >= B.npth[d]) return;
    const int bi = box_of_pth(B, d, gt);
    BoxDev g = B.b[bi];
    g.bc = 0;
    int na, nb, ns;
    pencil_dims(g.nx, g.ny, g.nz, d, B.pl, na, nb, ns);
    long long t = gt - g.pth0[d];
    const int ia = (int)(t % na);          // x
    t /= na;
    const int ib = (int)(t % nb);          // y
    const int sg = (int)(t / nb);
    const int n = g.nz;
    const int i0 = sg * B.pl;
    const int i1 = i0 + B.pl < n ? i0 + B.pl : n;
    const long long N = B.N;
    const long long plane = (long long)g.nx * g.ny;
    const long long base = g.off + (long long)ib * g.nx + ia;      // cell (x, y, 0)
    const long long ox = ia + 1 < g.nx ? 1 : 1 - g.nx;
    const long long oy = ib + 1 < g.ny ? g.nx : g.nx - (long long)g.ny * g.nx;
    const R gm1 = R(gam - 1.0), gr = R(gam);
    const R r = DtOf<R>::hdtdx(dtb[bi]);
    const TE rf = DtOf<TE>::dtdx(dtb[bi]);
    const TU ruf = DtOf<TU>::dtdx(dtb[bi]);
    const R* WMd = WM + 14 * N;
    const R* WPd = WP + 14 * N;
    R* Fz = F2 + 14 * N;
    R df[2][7], w[7], wpp[7], f[7], fprev[7];
    {
        const int sk = wrapi(i0 - 1, n);
        const long long sc = base + (long long)sk * plane;
#pragma unroll
        for (int m = 0; m < 7; m++) w[m] = WPd[(long long)m * N + sc];
        ctu_tdiff<R, false, d>(g, ia, ib, sk, sc, F1, nullptr, 0, N, df);
        ctu_apply<R, d>(w, W[(5 + d) * N + sc], df, r, gm1, wpp);
    }
    for (int p = i0; p <= i1; p++) {
        const int k = p < n ? p : p - n;
        const long long c = base + (long long)k * plane;
        ctu_tdiff<R, false, d>(g, ia, ib, k, c, F1, nullptr, 0, N, df);
        const R bnc = W[(5 + d) * N + c];
        R wm[7];
#pragma unroll
        for (int m = 0; m < 7; m++) w[m] = WMd[(long long)m * N + c];
        ctu_apply<R, d>(w, bnc, df, r, gm1, wm);
        riemann<SOLVER>(wpp, wm, R(Bhz[c]), gm1, gr, f);
        if (p < i1) {                       // the components the edge fields read
            Fz[c] = f[0];
            Fz[5 * N + c] = f[5];
            Fz[6 * N + c] = f[6];
        }
        if (p > i0) {                       // cell p - 1 between faces p - 1 and p
            const long long cc = base + (long long)(p - 1) * plane;
            R fc[3][5], fn[3][5];
#pragma unroll
            for (int m = 0; m < 5; m++) {
                fc[0][m] = F2[(long long)m * N + cc];
                fn[0][m] = F2[(long long)m * N + cc + ox];
                fc[1][m] = F2[(7LL + m) * N + cc];
                fn[1][m] = F2[(7LL + m) * N + cc + oy];
                fc[2][m] = fprev[m];
                fn[2][m] = f[m];
            }
            const TU rho0 = s.rho[cc], mx0 = s.m[0][cc], my0 = s.m[1][cc], mz0 = s.m[2][cc];
            const TE e0 = s.e[cc];
            TU du[4];
            TE due;
            flux_divergence<R, TU, TE>(fc, fn, du, due);
            TU u[4];
            TE e;
            full_hydro<TU, TE>(rho0, mx0, my0, mz0, e0, du, due, ruf, rf, u, e);
            s.rho[cc] = u[0];
            s.m[0][cc] = u[1];
            s.m[1][cc] = u[2];
            s.m[2][cc] = u[3];
            s.e[cc] = e;
        }
        copy7(fprev, f);
        if (p < i1) {
#pragma unroll
            for (int m = 0; m < 7; m++) w[m] = WPd[(long long)m * N + c];
            ctu_apply<R, d>(w, bnc, df, r, gm1, wpp);
        }
    }
}

}  // namespace mhd
