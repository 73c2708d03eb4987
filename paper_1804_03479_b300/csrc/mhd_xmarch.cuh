// mhd_xmarch.cuh -- the VL face sweeps along x (Sec. 3.2: the first-order
// predictor fluxes and the PLM corrector fluxes) by warps marching their row
// in segments of 32 cells aligned to the row's start.
//
// Lane l of segment s owns cell x = 32 s + l and the face below it: it
// reconstructs that cell (the corrector) and solves the Riemann problem at
// its lower face.  Every lane produces a face, and the warp's flux stores
// start on the row's first cell, so a row that starts on a 128-byte line
// (FP32, nx and the box offset multiples of 32) stores whole lines.  The
// stencil's neighbours across a segment's ends come from registers kept
// from the previous segment:
//   predictor  lane l takes cell x, and lane 0 the previous segment's last
//              cell.  FP32 rows of whole 16-byte-aligned segments come
//              through shared memory by asynchronous copies, three segments
//              in flight per warp; other rows load cell x one segment ahead
//              into registers;
//   corrector  lane l loads cell x + 1, one segment ahead, so that the
//              stencil x - 1 .. x + 1 of every lane lies in this segment's
//              loads or, for lanes 0 and 1, the previous segment's; lane 0
//              takes the previous segment's last "+" state.
// (An unshifted corrector needs the next segment's first cell in the
// current iteration, so two segments in flight: at 256^3 FP32 Roe it
// spilled 60 bytes and took 0.62 ms.  The shifted one took 0.60 ms in a
// plain loop over the row's segments (20 bytes spilled) and 0.51 ms in the
// loop below, which ptxas fits in 128 registers without spilling.)
// The corrector starts with a lead-in segment -1 (cells -32 .. -1, periodic
// or clamped), reconstructed but not solved, whose lane 31 gives face 0 its
// lower state, exactly as the x-warp lane of cell -1 does.
//
// The x-warp form (k_xwarp) overlaps its segments by the stencil's reach
// instead: 31 (predictor) or 29 (PLM corrector) of its 32 lanes produce a
// face, a 256-cell row takes 9 segments where this form takes 8 (plus the
// corrector's lead-in), and its loads and stores start off a line boundary.
// At 256^3 FP32 this form takes 0.266 ms for the Roe predictor (x-warps
// 0.449; 0.356 with the register prefetch of one segment) and 0.510 / 0.509
// ms for the PLM corrector with Roe and HLLD (x-warps 0.616 / 0.574).
#pragma once
#include "mhd_kernels.cuh"

namespace mhd {

// lane l gets v of lane l - 1; lane 0 gets c of lane 31 (the previous
// segment's last cell)
template <class R>
__device__ __forceinline__ void from_below(R o[7], const R v[7], const R c[7])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int m = 0; m < 7; m++) o[m] = __shfl_sync(0xffffffffu, lane == 31 ? c[m] : v[m], (lane + 31) & 31);
}

// lane l gets v of lane l + 1; lane 31 gets n of lane 0 (the next segment's
// first cell)
template <class R>
__device__ __forceinline__ void from_above(R o[7], const R v[7], const R n[7])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int m = 0; m < 7; m++) o[m] = __shfl_sync(0xffffffffu, lane == 0 ? n[m] : v[m], (lane + 1) & 31);
}

// register bound: four resident blocks for the FP32 Roe walks (122 and 128
// registers; at the x-warps' five blocks the predictor spilled and ran
// slower, 0.375 against 0.356 ms at 256^3)
template <class R, int RECON, int SOLVER, int MODE>
constexpr int xmarch_min_blocks()
{
    return sizeof(R) == 4 && SOLVER == ROE ? 4 : xwarp_min_blocks<R, RECON, SOLVER, MODE>();
}

// 16-byte asynchronous copy global -> shared (cache at L2 only)
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_group()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// wait until at most N of this thread's committed copy groups are pending
template <int N>
__device__ __forceinline__ void cp_async_wait_pending()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// the staged predictor: segments in flight per warp, and the arrays of a
// segment (the 7 primitives of the x frame and the face field)
constexpr int XM_SLOTS = 3, XM_ARR = 8;

// grid rows marched by one warp.  The corrector's loop chains them (the
// next row's lead-in loads issued while the current row's last segment is
// solved); more than one row a warp measured slower at 256^3 FP32 Roe
// (corrector 0.510 / 0.512 / 0.514 / 0.520 ms for 1 / 2 / 4 / 8 rows,
// predictor chained likewise 0.368 to 0.405 ms): fewer warps, and no
// latency left to hide at a row's start.  So one row a warp.
constexpr int XMARCH_ROWS = 1;

__host__ __device__ __forceinline__ long long xmarch_warps(long long nrows)
{
    return (nrows + XMARCH_ROWS - 1) / XMARCH_ROWS;
}

// one grid row: its box, x length, outflow flag and first cell
struct XRow {
    int bi, nx, out, nseg;
    long long base;
};

__device__ __forceinline__ XRow xrow_of(const Boxes& B, long long r)
{
    const int bi = box_of_row(B, r);
    XRow q;
    q.bi = bi;
    q.nx = B.b[bi].nx;
    q.out = B.b[bi].bc & 1;
    q.nseg = (q.nx + 31) >> 5;
    q.base = B.b[bi].off + (r - B.b[bi].xr0) * q.nx;
    return q;
}

// MODE 0: first-order states (the VL predictor); MODE 1: PLM-reconstructed
// (the VL corrector); MODE 2: PLM-reconstructed with the characteristic
// tracing and the dB_n/dn source terms (CTU steps 1-2, as the tracing
// pencils do), each cell's traced lower and upper states also written to
// WMg / WPg.  Warp w marches grid rows w XMARCH_ROWS .. (w + 1) XMARCH_ROWS
// - 1 of the whole batch (B.nxr rows, each of its own box); x periodic or
// (MODE 0 and 1) outflow, with clamped cells as in the x-warps.
template <class R, int RECON, int SOLVER, int MODE, class TE>
__global__ void __launch_bounds__(PENCIL_THREADS, (xmarch_min_blocks<R, RECON, SOLVER, MODE>()))
k_xmarch(Boxes B, const R* __restrict__ W, const TE* __restrict__ Bd, R* __restrict__ F, double gam,
         R* __restrict__ WMg = nullptr, R* __restrict__ WPg = nullptr, const DtBox* __restrict__ dtb = nullptr)
{
    static_assert(MODE == 0 || RECON != PPM, "the march reconstructs PLM stencils only");
    constexpr bool TR = MODE == 2;
    const int lane = threadIdx.x & 31;
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    long long r = wid * XMARCH_ROWS;
    if (r >= B.nxr) return;                          // uniform over the warp
    const long long rend = r + XMARCH_ROWS < B.nxr ? r + XMARCH_ROWS : B.nxr;
    const long long N = B.N;
    const R gr = R(gam), gm1 = R(gam - 1.0);
    XRow q = xrow_of(B, r);
    R f[7];
    TE fb, fbn;
    if (MODE == 0) {
        // face x sees cells x - 1 and x; wc: the previous segment's cells
        // (at the row's start its cell -1, in every lane).  One row a warp:
        // an outer loop over rows cost registers and time (0.375 against
        // 0.356 ms at 256^3 FP32 Roe, even at one row)
        static_assert(XMARCH_ROWS == 1, "the predictor marches one row a warp");
        if constexpr (sizeof(R) == 4 && sizeof(TE) == 4) {
            // FP32 rows of whole 16-byte-aligned segments (periodic x, a quad
            // box: nx, the offset and the field stride multiples of 4 cells,
            // nx a multiple of 32): the segments come through shared memory,
            // XM_SLOTS of them in flight per warp, by asynchronous copies that
            // hold no registers; one register segment in flight left the
            // kernel waiting on memory (long_scoreboard first): 0.266 against
            // 0.356 ms at 256^3 (Roe), the y/z pencils' rate
            __shared__ __align__(16) float xm_buf[PENCIL_THREADS / 32][XM_SLOTS][XM_ARR][32];
            if (!q.out && q.nx % 32 == 0 && B.b[q.bi].quad) {
                float (*buf)[XM_ARR][32] = xm_buf[threadIdx.x >> 5];
                // segment sg into slot sl: lane l copies pieces l and l + 32
                // of the 8 x 8 16-byte pieces (array a = piece / 8)
                auto stage = [&](int sg, int sl) {
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const int pc = lane + 32 * h, a = pc >> 3, o = (pc & 7) * 4;
                        const int fld = a < 5 ? a : a + 1;             // W fields 0-4, 6, 7
                        const float* src = a < 7 ? (const float*)W + (long long)fld * N : (const float*)Bd;
                        cp_async16(&buf[sl][a][o], src + q.base + 32 * sg + o);
                    }
                };
                R wc[7], bdum;
                load_rot(W, N, q.base + q.nx - 1, 0, wc, bdum);      // cell -1: the row's last cell
#pragma unroll
                for (int k = 0; k < XM_SLOTS; k++) {
                    if (k < q.nseg) stage(k, k);
                    cp_async_group();                                // one group per segment, empty past the row
                }
                for (int sg = 0; sg < q.nseg; sg++) {
                    const int sl = sg % XM_SLOTS;
                    cp_async_wait_pending<XM_SLOTS - 1>();           // segment sg has landed (this lane's part)
                    __syncwarp();                                    // ... and every lane's
                    R w[7];
#pragma unroll
                    for (int m = 0; m < 7; m++) w[m] = buf[sl][m][lane];
                    const R fbv = buf[sl][7][lane];
                    __syncwarp();                                    // every lane is done with the slot
                    if (sg + XM_SLOTS < q.nseg) stage(sg + XM_SLOTS, sl);
                    cp_async_group();
                    R wl[7];
                    from_below(wl, w, wc);
                    riemann<SOLVER>(wl, w, fbv, gm1, gr, f);
#pragma unroll
                    for (int m = 0; m < 7; m++) F[(long long)m * N + q.base + 32 * sg + lane] = f[m];
                    copy7(wc, w);
                }
                cp_async_wait_pending<0>();
                return;
            }
        }
        R w[7], bn, wn[7], bnn, wc[7], bdum;
        load_rot(W, N, q.base + bidx(-1, q.nx, q.out), 0, wc, bdum);
        {
            const long long c0 = q.base + bidx(lane, q.nx, q.out);
            load_rot(W, N, c0, 0, w, bn);
            fb = Bd[c0];
        }
        for (int s = 0; s < q.nseg; s++) {
            const int x = 32 * s + lane;
            if (s + 1 < q.nseg) {
                const long long cn = q.base + bidx(x + 32, q.nx, q.out);
                load_rot(W, N, cn, 0, wn, bnn);
                fbn = Bd[cn];
            }
            R wl[7];
            from_below(wl, w, wc);
            if (x < q.nx) {
                riemann<SOLVER>(wl, w, R(fb), gm1, gr, f);
#pragma unroll
                for (int m = 0; m < 7; m++) F[(long long)m * N + q.base + x] = f[m];
            }
            if (s + 1 < q.nseg) {
                copy7(wc, w);
                copy7(w, wn);
                fb = fbn;
            }
        }
    } else {
        // cell x is reconstructed from x - 1, x, x + 1; face x takes the "+"
        // state of cell x - 1 and the "-" state of cell x.  Lane l holds
        // cell x + 1 (v; one cell past its own, loaded one segment ahead), so
        // that its whole stencil is in this segment's lanes or, for lanes 0
        // and 1, the previous segment's (vc); wpc: the previous segment's
        // "+" states.  Each row starts with its lead-in segment -1.  The
        // tracing form loads the face field shifted by one as well (fs: face
        // x + 1; face x from the lane below, or for lane 0 the previous
        // segment's fsc), which gives each cell its dB_n/dn.
        R dum[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};   // slopes: unused by PLM
        R v[7], bv, vc[7], bvc, wpc[7];
        TE fs, fsc, fsn;
        R dtdx = R(0), hdt = R(0);
        load_rot(W, N, q.base + bidx(lane - 31, q.nx, q.out), 0, v, bv);
        copy7(vc, v);                                // (lanes 0 and 1 in a lead-in: not used)
        bvc = bv;
        copy7(wpc, v);
        if constexpr (TR) {
            fs = Bd[q.base + bidx(lane - 31, q.nx, q.out)];
            fsc = fs;
            dtdx = DtOf<R>::dtdx(dtb[q.bi]);
            hdt = DtOf<R>::hdt(dtb[q.bi]);
        }
        int s = -1;
        for (;;) {
            const int x = 32 * s + lane;
            // the next segment: of this row, else the next row's lead-in
            int sn = s + 1;
            long long rn = r;
            XRow qn = q;
            if (sn == q.nseg) {
                sn = -1;
                rn = r + 1;
                if (rn < rend) qn = xrow_of(B, rn);
            }
            const bool more = rn < rend;
            R vn[7], bvn;
            if (more) {                              // its cells (shifted by one) and faces
                const long long cv = qn.base + bidx(32 * sn + lane + 1, qn.nx, qn.out);
                load_rot(W, N, cv, 0, vn, bvn);
                if constexpr (TR)
                    fsn = Bd[cv];
                else if (sn >= 0)
                    fbn = Bd[qn.base + bidx(32 * sn + lane, qn.nx, qn.out)];
            }
            R w[7], bn, wm1[7], wm[7], wp[7];
#pragma unroll
            for (int m = 0; m < 7; m++) {
                w[m] = __shfl_sync(0xffffffffu, lane == 31 ? vc[m] : v[m], (lane + 31) & 31);
                wm1[m] = __shfl_sync(0xffffffffu, lane >= 30 ? vc[m] : v[m], (lane + 30) & 31);
            }
            bn = __shfl_sync(0xffffffffu, lane == 31 ? bvc : bv, (lane + 31) & 31);
            recon_cell<RECON, TR>(wm1, w, v, bn, gr, dum, dum, dum, dtdx, wm, wp);
            if constexpr (TR) {
                fb = __shfl_sync(0xffffffffu, lane == 31 ? fsc : fs, (lane + 31) & 31);   // face x
                const R dbn = sizeof(R) == 8 ? R((double)(fs - fb) / B.b[q.bi].dx)
                                             : R(fs - fb) * R(B.b[q.bi].inv_dx);   // as face_gradient
                trace_source(w, bn, dbn, hdt, gm1, wm, wp);
            }
            if (s >= 0) {
                R wl[7];
                from_below(wl, wp, wpc);
                if (x < q.nx) {
                    if constexpr (TR) {
#pragma unroll
                        for (int m = 0; m < 7; m++) {
                            WMg[(long long)m * N + q.base + x] = wm[m];
                            WPg[(long long)m * N + q.base + x] = wp[m];
                        }
                    }
                    riemann<SOLVER>(wl, wm, R(fb), gm1, gr, f);
#pragma unroll
                    for (int m = 0; m < 7; m++) F[(long long)m * N + q.base + x] = f[m];
                }
            }
            if (!more) break;
            copy7(wpc, wp);
            copy7(vc, v);
            bvc = bv;
            copy7(v, vn);
            bv = bvn;
            if constexpr (TR) {
                fsc = fs;
                fs = fsn;
                if (qn.bi != q.bi) {
                    dtdx = DtOf<R>::dtdx(dtb[qn.bi]);
                    hdt = DtOf<R>::hdt(dtb[qn.bi]);
                }
            } else if (sn >= 0) {
                fb = fbn;
            }
            s = sn;
            r = rn;
            q = qn;
        }
    }
}

}  // namespace mhd
