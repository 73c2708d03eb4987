// mhd_yhalf.cuh -- per-cell passes inside the y pencils of the VL step.
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
// the y fluxes.  A segment of pl faces forms pl + 3 half-step states (its
// lead-in cells i0 - 2, i0 - 1 and the cell past its end): the three extra
// ones are recomputed where the neighbouring segment owns them.
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
// Periodic boxes (one or a batch), PLM reconstructions.
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

// register bound: as the PLM corrector pencils it extends (FP32 Roe: 4
// blocks of 128 threads, 128 registers with 16 bytes spilled; at 3 blocks
// and 167 registers it ran 0.760 against 0.708 ms at 256^3)
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
    static_assert(RECON != PPM, "the fused walk reconstructs PLM stencils only");
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

    YCarry<R, TE> Y;
    {
        const long long c = base + (long long)wrapi(i0 - 2, ny) * nx;
#pragma unroll
        for (int m = 0; m < 5; m++) Y.fy[m] = Fp[(7LL + m) * N + c];
        Y.by = s.b[1][c];
        Y.ex = E[c];
        Y.ez = E[2 * N + c];
        Y.ezx = E[2 * N + c + ox];
        Y.exz = E[c + oz];
    }
    // the half-step state of line cell i (the next one along the walk after
    // the previous call): w and bn in the y sweep frame, lo the lower y face;
    // stored when the segment owns the cell
    auto half_cell = [&](int i, R w[7], R& bn, TE& lo_y) {
        const long long c = base + (long long)wrapi(i, ny) * nx;
        const long long cy = base + (long long)wrapi(i + 1, ny) * nx;
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
        TE lo[3], bc[3];
        half_faces<TE, R>(ec, en, e2xy, e1xz, e0yz, blo, bhi, r, lo, bc);
        TU du[4];
        TE due;
        flux_divergence<R, TU, TE>(fc, fn, du, due);
        R w8[8];
        half_prims<R, TU, TE>(rho0, mx0, my0, mz0, e0, du, due, ru, r, bc, gam, pfloor, w8);
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
        // the next cell's operands from below
#pragma unroll
        for (int m = 0; m < 5; m++) Y.fy[m] = fn[1][m];
        Y.by = bhi[1];
        Y.ex = en[0][1];
        Y.ez = en[2][1];
        Y.ezx = e2xy;
        Y.exz = e0yz;
    };

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

}  // namespace mhd
