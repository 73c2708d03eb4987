// mhd_xpencil.cuh -- the VL face sweeps along x (Sec. 3.2: the first-order
// predictor fluxes and the reconstructed corrector fluxes) by pencils.
//
// The 32 lanes of a warp walk 32 consecutive grid rows (j, then k) of one
// box, each thread the pencil_len faces of one segment of its row, with the
// cells around the current face in registers, exactly as the y and z
// pencils do: one reconstruction and one Riemann solve per face, no lane
// that reconstructs without producing a face and no register shuffles (the
// costs of the x-warp form).  Along x a row is contiguous in memory, so
// 32 lanes on 32 rows would load and store 32 scattered words per
// instruction; instead both directions pass through per-warp shared-memory
// chunks of XC cells x 32 rows:
//   cells   lane l copies (cp.async) cell l % XC of rows l / XC + 8 m,
//           m = 0 .. XC-1, of the 8 primitives and the face field: 16-byte
//           row pieces; each lane then reads its own row (stride XST, odd,
//           so the 32 rows fall in 32 banks);
//   fluxes  each lane writes its faces' 7 components into its row, and
//           every XC faces the warp stores the chunk with the same pattern.
// The walk is warp-uniform (every lane of a warp has the same segment), so
// the chunk refills and flushes need only __syncwarp.
//
// Measured at 256^3 (VL + PLM + Roe): in FP64 the x sweeps run at the y and
// z pencils' rate (corrector 27.7 ms against 30.3 ms by warps, predictor
// 14.7 against 16.9), so this is the FP64 default.  In FP32 arithmetic the
// x-warps stay faster (0.62 against 1.8 ms): there the staging, not the
// arithmetic, sets the pace -- every copy instruction touches 8 rows in
// 16-byte half sectors, the buffers leave little of the SM's L1, and the
// flux stores' half sectors double the DRAM writes.
#pragma once
#include "mhd_kernels.cuh"
#include "mhd_fused.cuh"

namespace mhd {

constexpr int XC = 4;            // cells per staged chunk along x
constexpr int XST = XC + 1;      // row stride of a chunk (odd: conflict-free row reads)
constexpr int XCH = 32 * XST;    // one field of a chunk for the warp's 32 rows

// shared memory of one warp: the face field (TE), 8 primitives, 7 fluxes
template <class R, class TE>
__host__ __device__ constexpr size_t xpencil_warp_bytes()
{
    return (size_t)XCH * sizeof(TE) + (size_t)(8 + 7) * XCH * sizeof(R);
}

// pencil threads of a box: its rows rounded up to whole warps, per segment
__host__ __device__ __forceinline__ long long xpencil_threads_of_box(int nx, int ny, int nz, int pl)
{
    const long long rows = ((long long)ny * nz + 31) / 32 * 32;
    return rows * ((nx + pl - 1) / pl);
}

__device__ __forceinline__ int box_of_xp(const Boxes& B, long long t)
{
    int lo = 0, hi = B.nbox - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (B.b[mid].xp0 <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// MODE 0: first-order states (the VL predictor); MODE 1: reconstructed
// (the corrector).  Periodic or outflow x (the outflow lead-in as in
// k_pencil: the "+" state of cell 0 with its own clamped stencil).
template <class R, int RECON, int SOLVER, int MODE, class TE>
__global__ void __launch_bounds__(PENCIL_THREADS, (sweep_min_blocks<R, RECON, SOLVER, MODE>()))
k_xpencil(Boxes B, const R* __restrict__ W, const TE* __restrict__ Bd, R* __restrict__ F, double gam)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    unsigned char* base = smem_raw + (threadIdx.x >> 5) * xpencil_warp_bytes<R, TE>();
    TE* const sfb = reinterpret_cast<TE*>(base);
    R* const sw = reinterpret_cast<R*>(base + XCH * sizeof(TE));
    R* const sfo = sw + 8 * XCH;
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gt >= B.nxp) return;                     // whole warps: every box's share is a multiple of 32
    const int bi = box_of_xp(B, gt);
    const BoxDev& gb = B.b[bi];
    const int nx = gb.nx, out = gb.bc & 1;
    const int nrow = gb.ny * gb.nz;
    const long long prow = ((long long)nrow + 31) / 32 * 32;
    const long long t = gt - gb.xp0;
    const int sg = (int)(t / prow);
    const int rw0 = (int)(t - sg * prow) - lane;  // the warp's first row
    const long long off = gb.off;
    const int i0 = sg * B.pl, i1 = i0 + B.pl < nx ? i0 + B.pl : nx;
    const long long N = B.N;
    const R gr = R(gam), gm1 = R(gam - 1.0);
    const int kx = lane % XC, rl0 = lane / XC;    // this lane's place in the chunk copies
    int cbase = 0, obase = i0;
    // stage logical cells [c0, c0 + XC) of the warp's rows (rows past the
    // box: its last row, never stored)
    auto refill = [&](int c0) {
        cbase = c0;
        __syncwarp();                             // every lane is done with the previous chunk
        const int phys = bidx(c0 + kx, nx, out);
#pragma unroll
        for (int m = 0; m < XC; m++) {
            const int rl = rl0 + (32 / XC) * m;
            const int row = rw0 + rl < nrow ? rw0 + rl : nrow - 1;
            const long long c = off + (long long)row * nx + phys;
            const int o = rl * XST + kx;
#pragma unroll
            for (int f = 0; f < 8; f++) cp_async_el(sw + f * XCH + o, W + f * N + c);
            cp_async_el(sfb + o, Bd + c);
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncwarp();                             // every lane's copies have landed
    };
    // logical cell j (j >= cbase; warp-uniform) of this lane's row in the x
    // sweep frame, with its cell-centre B_x and its lower x face field
    auto cell = [&](int j, R w[7], R& bn, TE& fb) {
        if (j >= cbase + XC) refill(cbase + XC);
        const int o = lane * XST + (j - cbase);
        w[0] = sw[o];
        w[1] = sw[XCH + o];
        w[2] = sw[2 * XCH + o];
        w[3] = sw[3 * XCH + o];
        w[4] = sw[4 * XCH + o];
        w[5] = sw[6 * XCH + o];
        w[6] = sw[7 * XCH + o];
        bn = sw[5 * XCH + o];
        fb = sfb[o];
    };
    // the flux of face i (i from i0 in order) into the chunk; a full chunk,
    // or the segment's last face, is stored
    auto put = [&](int i, const R f[7]) {
        const int o = lane * XST + (i - obase);
#pragma unroll
        for (int m = 0; m < 7; m++) sfo[m * XCH + o] = f[m];
        if (i - obase == XC - 1 || i == i1 - 1) {
            __syncwarp();
            const int ix = obase + kx;
#pragma unroll
            for (int m = 0; m < XC; m++) {
                const int rl = rl0 + (32 / XC) * m;
                if (ix < i1 && rw0 + rl < nrow) {
                    const long long c = off + (long long)(rw0 + rl) * nx + ix;
                    const int oo = rl * XST + kx;
#pragma unroll
                    for (int q = 0; q < 7; q++) F[q * N + c] = sfo[q * XCH + oo];
                }
            }
            __syncwarp();
            obase += XC;
        }
    };
    R f[7];
    if (MODE == 0) {
        // first-order states: the face i sees cells i-1 and i
        refill(i0 - 1);
        R wl[7], wr[7], bd;
        TE fd;
        cell(i0 - 1, wl, bd, fd);
        for (int i = i0; i < i1; i++) {
            cell(i, wr, bd, fd);
            riemann<SOLVER>(wl, wr, R(fd), gm1, gr, f);
            put(i, f);
            copy7(wl, wr);
        }
    } else if (RECON != PPM) {
        // PLM: cells i-1, i, i+1 in registers; wpp the "+" state of cell i-1
        refill(i0 - 2);
        R wa[7], wb[7], wc[7], bna, bnb, bnc, wpp[7], wm[7], wp[7];
        R dum[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};   // slopes: unused by PLM
        TE fa, fb, fc;
        // lead-in: the "+" state of logical cell li (i0 - 1; at a lower
        // outflow side cell 0 with its own stencil)
        const int li = (out && i0 == 0) ? 0 : i0 - 1;
        cell(li - 1, wa, bna, fa);
        cell(li, wb, bnb, fb);
        cell(li + 1, wc, bnc, fc);
        recon_cell<RECON, false>(wa, wb, wc, bnb, gr, dum, dum, dum, R(0), wm, wpp);
        // the loop's window, cells i0 - 1 and i0 (at a lower outflow side the
        // lead-in cells -1 and 0 already)
        if (li == i0 - 1) {
            copy7(wa, wb); bna = bnb; fa = fb;
            copy7(wb, wc); bnb = bnc; fb = fc;
        }
        for (int i = i0; i < i1; i++) {
            cell(i + 1, wc, bnc, fc);
            recon_cell<RECON, false>(wa, wb, wc, bnb, gr, dum, dum, dum, R(0), wm, wp);
            riemann<SOLVER>(wpp, wm, R(fb), gm1, gr, f);
            put(i, f);
            copy7(wpp, wp);
            copy7(wa, wb); bna = bnb; fa = fb;
            copy7(wb, wc); bnb = bnc; fb = fc;
        }
    } else {
        // PPM: cells i-1 .. i+2 and the characteristic slopes of i-1 .. i+1
        refill(i0 - 3);
        R w0[7], w1[7], w2[7], w3[7], b0, b1, b2, b3;
        R s0[7], s1[7], s2[7], wpp[7], wm[7], wp[7];
        TE f0, f1, f2, f3;
        const int li = (out && i0 == 0) ? 0 : i0 - 1;
        {
            R wq[7], bq;
            TE fq;
            cell(li - 2, wq, bq, fq);
            cell(li - 1, w0, b0, f0);
            cell(li, w1, b1, f1);
            cell(li + 1, w2, b2, f2);
            cell(li + 2, w3, b3, f3);
            char_slope(wq, w0, w1, b0, gr, s0);             // slope of li-1
            char_slope(w0, w1, w2, b1, gr, s1);             // li
            char_slope(w1, w2, w3, b2, gr, s2);             // li+1
            recon_cell<PPM, false>(w0, w1, w2, b1, gr, s0, s1, s2, R(0), wm, wpp);
        }
        // window: w0..w2 = cells i0-1 .. i0+1, s0, s1 = slopes of i0-1, i0
        if (li == i0 - 1) {
            copy7(w0, w1); b0 = b1; f0 = f1;
            copy7(w1, w2); b1 = b2; f1 = f2;
            copy7(w2, w3); b2 = b3; f2 = f3;
            copy7(s0, s1);
            copy7(s1, s2);
        }
        for (int i = i0; i < i1; i++) {
            cell(i + 2, w3, b3, f3);
            char_slope(w1, w2, w3, b2, gr, s2);             // slope of i+1
            recon_cell<PPM, false>(w0, w1, w2, b1, gr, s0, s1, s2, R(0), wm, wp);
            riemann<SOLVER>(wpp, wm, R(f1), gm1, gr, f);
            put(i, f);
            copy7(wpp, wp);
            copy7(w0, w1); b0 = b1; f0 = f1;
            copy7(w1, w2); b1 = b2; f1 = f2;
            copy7(w2, w3); b2 = b3; f2 = f3;
            copy7(s0, s1);
            copy7(s1, s2);
        }
    }
}

}  // namespace mhd
