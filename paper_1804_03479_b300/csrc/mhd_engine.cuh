// mhd_engine.cuh -- context and the launch sequence of one step.
#pragma once
#include <cuda_runtime.h>
#include <stdio.h>
#include "mhd.h"
#include "mhd_kernels.cuh"
#include "mhd_fused.cuh"
#include "mhd_xpencil.cuh"
#include "mhd_xmarch.cuh"
#include "mhd_tma.cuh"
#include "mhd_yhalf.cuh"

struct mhd_ctx;
struct mhd_mlp;
typedef void (*mhd_step_fn)(mhd_ctx*, bool device_dt);

struct mhd_ctx {
    mhd_grid grid;                  // box 0
    mhd_scheme sch;
    double gamma;
    cudaStream_t stream;
    bool own_stream;
    int nbox;
    mhd::BoxDev* hbox;              // host copy of the box table
    mhd::BoxDev* dbox;              // device copy
    mhd::Boxes B;                   // kernel view (points at dbox)
    int nsm;                        // SMs of the device
    int sweep_bps;                  // persistent sweep blocks per SM
    int bc;                         // outflow axes (bit d), one-box contexts; 0 = periodic
    void* fout;                     // [3][7][cross-section] outer-face fluxes of the outflow axes
    int fix_nl[3];                  // Dirichlet sides: fixed ghost layers at each end of axis d (0: none)
    mhd::FixedState fix[3][2];      // their states, lower and upper end
    int pencil_mask;                // VL sweeps by pencils on the axes of bits 0-2; bit 3: fused VL
                                    // predictor; bit 4: x by staged pencils instead of warps (VL)
    int emf_stage_req;              // edge fields: 0 = k_emf, 1 = planes by the tensor memory accelerator
                                    // where eligible, 2 = fused with the update (k_emf_update) where eligible
    int emf_tma;                    // 1 when the context runs k_emf_tma
    int emf_tma_grid;               // its grid: min(SMs, tiles)
    CUtensorMap* tmaps;             // [6] 64-byte aligned 4-D tensors of k_emf_tma: W, Wh (3-field copies),
                                    // F1 (1-, 2-field copies), F2 (the same)
    unsigned* perr;                 // device: bit 0 = a staged-plane wait of k_emf_tma gave up
    int pencil_len;                 // faces per pencil-segment thread
    size_t szu, sze, szr;          // element sizes: rho/M storage, e/B storage, arithmetic
    void* rho;
    void* m[3];
    void* e;
    void* b[3];
    void* W;                        // 8 primitives at t^n
    void* Wh;                       // 8 primitives at t^{n+1/2}
    void* F1;                       // 3 x 7 face fluxes
    void* F2;                       // 3 x 7 face fluxes (CTU corrector)
    void* E;                        // 3 edge fields
    void* Bh[3];                    // half-step face field
    void* WM;                       // 3 x 7 traced states (CTU)
    void* WP;
    void* stage;                    // staging for the mixed layout
    double* dt;                     // [nbox]
    mhd::DtBox* dtc;                // [nbox] dt and its ratios to dx
    double* smax;                   // [nbox] signal-speed maximum of each box
    unsigned long long* smax_part;  // [nbox] signal-speed maximum accumulators (bits of a double >= 0;
                                    // cleared by k_finalize_dt)
    int cell_grid;                  // persistent grid of the per-cell kernels
    int quad_grid;                  // persistent grid of the x-quad kernels
    unsigned long long* bad;
    unsigned long long* nfloor;     // cells raised to the pressure floor
    double* part;                   // [nvblk][10]
    double* diag;                   // [nbox][10]
    long long bytes;
    mhd_step_fn step;
    mhd_step_fn plain_step;         // the scheme's own step (without selector)
    int launches;
    // learned path selector (FP32 VL, one box)
    mhd_mlp* sel;
    float* sel_feats;               // [nblocks][48]
    cudaStream_t sel_st;            // the selector's passes, beside the cheap predictor sweeps
    cudaEvent_t sel_fork, sel_join; // (created with the selector; no timing)
    unsigned char* sel_flags;       // [nblocks], 1 = full path
    int* sel_cnt;                   // per list: entries
    int* sel_list[8];               // per axis d: [2d] one byte per unit (tile, pencil segment or x-warp
                                    // item), 1 = full path, in the units' order; [2d+1] the list of the
                                    // full units; [6], [7] the same for the x corrector's items when x
                                    // runs by warps (sel_cnt[2q + 1]: the entries of list 2q + 1)
    long long sel_cap;              // entries of each list
    cudaGraphExec_t gexec;
    bool have_graph;
    // kernel-group timing (CUDA events on the context stream)
    cudaEvent_t* prof_ev;           // [prof_cap][MHD_NGROUPS + 1]
    int prof_cap, prof_steps;
    bool prof_on;
    mhd_status sticky;
    char err[256];
};

#define MHD_NGROUPS 11  // prim+dt, predictor sweeps x/y/z, emf, half, corrector sweeps x/y/z, emf, full

// record the boundary event `b` of the current step when timing is on
inline void prof_mark(mhd_ctx* c, int b)
{
    if (c->prof_on && c->prof_steps < c->prof_cap)
        cudaEventRecord(c->prof_ev[c->prof_steps * (MHD_NGROUPS + 1) + b], c->stream);
}

namespace mhd {

template <class TU, class TE>
inline StateP<TU, TE> state_of(mhd_ctx* c)
{
    StateP<TU, TE> s;
    s.rho = (TU*)c->rho;
    for (int d = 0; d < 3; d++) s.m[d] = (TU*)c->m[d];
    s.e = (TE*)c->e;
    for (int d = 0; d < 3; d++) s.b[d] = (TE*)c->b[d];
    return s;
}

inline int xrow_grid(const mhd_ctx* c)
{
    return (int)((c->B.nxr * 32 + PENCIL_THREADS - 1) / PENCIL_THREADS);
}

// the aligned x-march: XMARCH_ROWS rows per warp
inline int xmarch_grid(const mhd_ctx* c)
{
    return (int)((xmarch_warps(c->B.nxr) * 32 + PENCIL_THREADS - 1) / PENCIL_THREADS);
}

inline int xwarp_grid(const mhd_ctx* c, int slot)
{
    return (int)((c->B.nxw[slot] * 32 + PENCIL_THREADS - 1) / PENCIL_THREADS);
}

inline int pencil_grid(const mhd_ctx* c, int d)
{
    return (int)((c->B.npth[d] + PENCIL_THREADS - 1) / PENCIL_THREADS);
}

// grids of the list forms of the pencil and x-warp sweeps (the learned
// selector's full units): capped at 8 blocks per SM, the kernels stride over
// the list, so that a short list does not pay for a grid of idle blocks
inline int list_grid_pencil(const mhd_ctx* c, int d)
{
    const int cap = 8 * c->nsm, g = pencil_grid(c, d);
    return g < cap ? g : cap;
}

inline int list_grid_xwarp(const mhd_ctx* c, int slot)
{
    const int cap = 8 * c->nsm, g = xwarp_grid(c, slot);
    return g < cap ? g : cap;
}

inline int sweep_grid(const mhd_ctx* c, int d)
{
    int cap = c->sweep_bps * c->nsm;
    return c->B.ntile[d] < cap ? c->B.ntile[d] : cap;
}

// put the ghost layers of the Dirichlet sides back to their fixed states
template <class TU, class TE>
void fix_layers(mhd_ctx* c, const StateP<TU, TE>& s, cudaStream_t st)
{
    for (int d = 0; d < 3; d++) {
        const int nl = c->fix_nl[d];
        if (!nl) continue;
        const BoxDev& g = c->hbox[0];
        const int na = d == 0 ? g.ny : g.nx, nb = d == 2 ? g.ny : g.nz;
        const long long nt = 2LL * nl * na * nb;
        k_fix_layers<TU, TE><<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(g, d, nl, c->fix[d][0], c->fix[d][1], s);
    }
}

// the edge fields of one stage: by k_emf_tma when the context runs it (FP32
// arithmetic, one box), else by k_emf
//
// Every compilation unit that launches these kernels holds its own instance of
// them, while the linker keeps a single copy of this inline function for all
// units with the same R (the FP32, mixed and learned steps share R = float).
// The instance launched here may therefore belong to another unit than the
// one whose step function raised its shared-memory limit, so the limit is
// raised here, on the instance this copy launches (a host-side attribute
// call, not a stream operation), and the occupancy is asked of it too.
template <class R>
void launch_emf(mhd_ctx* c, const Boxes& g, const R* F, const R* W, R* E, cudaStream_t st)
{
    if constexpr (sizeof(R) == 4) {
        if (c->emf_tma) {
            cudaFuncSetAttribute(k_emf_tma<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)emf_tma_smem_bytes());
            const CUtensorMap& mw = c->tmaps[W == (const R*)c->W ? 0 : 1];
            const int f = F == (const R*)c->F1 ? 2 : 4;
            k_emf_tma<R><<<c->emf_tma_grid, EMF_TMA_THREADS, emf_tma_smem_bytes(), st>>>(
                g, mw, c->tmaps[f], c->tmaps[f + 1], F, W, E, c->perr);
            return;
        }
    }
    cudaFuncSetAttribute(k_emf<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)emf_smem_bytes<R>());
    // persistent grid: the blocks one SM keeps resident (registers and shared
    // memory) times the SMs
    static int per = 0;
    if (per <= 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_emf<R>, EMF_THREADS, emf_smem_bytes<R>()) !=
                cudaSuccess || nb < 1)
            nb = 1;
        per = nb;
    }
    const long long cap = (long long)per * c->nsm;
    const int grid = (int)(g.netile < cap ? g.netile : cap);
    k_emf<R><<<grid, EMF_THREADS, emf_smem_bytes<R>(), st>>>(g, F, W, E);
}

// the VL x sweeps by staged pencils (k_xpencil) instead of warps
inline bool x_pencils(const mhd_ctx* c)
{
    return (c->pencil_mask & 17) == 17;
}

template <class R, int RECON, int SOLVER, int MODE, class TE>
void launch_xpencil(mhd_ctx* c, const Boxes& g, const R* W, const TE* Bd, R* F, cudaStream_t st)
{
    constexpr size_t smem = (PENCIL_THREADS / 32) * xpencil_warp_bytes<R, TE>();
    cudaFuncSetAttribute(k_xpencil<R, RECON, SOLVER, MODE, TE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    const int grid = (int)((g.nxp + PENCIL_THREADS - 1) / PENCIL_THREADS);
    k_xpencil<R, RECON, SOLVER, MODE, TE><<<grid, PENCIL_THREADS, smem, st>>>(g, W, Bd, F, c->gamma);
}

// the x sweeps by aligned marching warps (k_xmarch) instead of the
// overlapping x-warps: the VL predictor with pencil-mask bits 0 and 5, the VL
// corrector with bits 0 and 6 and a PLM stencil (the PPM corrector keeps its
// x-warp; bit 4, staged x pencils, takes precedence); the CTU tracing (MODE
// 2) with bits 0 and 5, a PLM stencil and a periodic x (the caller checks
// the boundary)
template <int RECON, int MODE>
inline bool x_march(const mhd_ctx* c)
{
    if (MODE == 0) return (c->pencil_mask & 33) == 33;
    if (MODE == 2) return (c->pencil_mask & 33) == 33 && RECON != PPM;
    return (c->pencil_mask & 65) == 65 && RECON != PPM;
}

template <class R, int RECON, int SOLVER, int MODE, class TE>
void launch_xmarch(mhd_ctx* c, const Boxes& g, const R* W, const TE* Bd, R* F, cudaStream_t st, R* WM = nullptr,
                   R* WP = nullptr)
{
    if constexpr (MODE == 0 || RECON != PPM)
        k_xmarch<R, RECON, SOLVER, MODE, TE><<<xmarch_grid(c), PENCIL_THREADS, 0, st>>>(g, W, Bd, F, c->gamma, WM,
                                                                                         WP, c->dtc);
}

// the VL predictor runs fused (k_vl_predictor) when the pencil mask has bit 3,
// the scheme is VL without a learned selector and every box is periodic
inline bool fused_predictor(const mhd_ctx* c)
{
    return (c->pencil_mask & 8) && c->sch.integrator == MHD_VL && !c->bc;
}

// The periodic half and full updates: by x-quads (k_half4, k_full4) when the
// state is FP32 throughout; in the mixed and FP64 forms one cell per thread
// (their FP64 per-cell arithmetic ran slower with four cells a thread:
// 1.88 against 1.46 ms for the mixed half update at 256^3).
template <class R, class TU, class TE>
void launch_half(mhd_ctx* c, const Boxes& g, const StateP<TU, TE>& s, const R* F, const R* E, TE* const Bh[3], R* Wh,
                 cudaStream_t st)
{
    if constexpr (sizeof(TU) == 4 && sizeof(TE) == 4)
        k_half4<R, TU, TE><<<c->quad_grid, CELL_THREADS, 0, st>>>(g, s, F, E, c->dtc, c->gamma, Bh[0], Bh[1], Bh[2],
                                                                   Wh, c->sch.pfloor);
    else
        k_half<R, TU, TE><<<c->cell_grid, CELL_THREADS, 0, st>>>(g, s, F, E, c->dtc, c->gamma, Bh[0], Bh[1], Bh[2],
                                                                  Wh, c->sch.pfloor);
}

template <class R, class TU, class TE>
void launch_full(mhd_ctx* c, const Boxes& g, const StateP<TU, TE>& s, const R* F, const R* E, cudaStream_t st)
{
    if constexpr (sizeof(TU) == 4 && sizeof(TE) == 4)
        k_full4<R, TU, TE><<<c->quad_grid, CELL_THREADS, 0, st>>>(g, s, F, E, c->dtc);
    else
        k_full<R, TU, TE><<<c->cell_grid, CELL_THREADS, 0, st>>>(g, s, F, E, c->dtc);
}

// the edge-field form a step runs: 1 = k_emf_tma, 2 = k_emf_update (the
// edge fields fused with the update; periodic boxes), 0 = k_emf followed by
// the update kernel
inline int emf_form(const mhd_ctx* c)
{
    if (c->emf_tma) return 1;
    return c->emf_stage_req == 2 && !c->bc ? 2 : 0;
}

// the VL half update fused into the corrector's y pencils (k_yhalf) with
// pencil-mask bits 1 and 7: periodic boxes without a learned
// selector, the predictor and the edge fields as separate kernels, and the
// second flux array allocated (the corrector's fluxes go there)
inline bool y_half(const mhd_ctx* c)
{
    return (c->pencil_mask & 130) == 130 && c->sch.integrator == MHD_VL && !c->bc && !c->sel && c->F2 &&
           !fused_predictor(c) && emf_form(c) == 0;
}

// CTU: the dt/2 update inside the y pencils of the transverse correction
// (k_ctu_yhalf) with pencil-mask bits 1 and 7: periodic boxes, the edge
// fields as their own kernel
inline bool ctu_y_half(const mhd_ctx* c)
{
    return c->sch.integrator == MHD_CTU && (c->pencil_mask & 130) == 130 && !c->bc && emf_form(c) == 0;
}

// CTU: the conservative update inside the z pencils of the transverse
// correction (k_ctu_zfull), CT alone after the edge fields, with pencil-mask
// bits 2 and 9: periodic boxes, the edge fields as their own kernel
inline bool ctu_z_full(const mhd_ctx* c)
{
    return c->sch.integrator == MHD_CTU && (c->pencil_mask & 516) == 516 && !c->bc && emf_form(c) == 0;
}

// the learned selector's step: the half update inside the cheap y corrector
// pencils with pencil-mask bits 1 and 7 (the second flux array allocated,
// the edge fields as their own kernel)
inline bool sel_y_half(const mhd_ctx* c)
{
    return (c->pencil_mask & 130) == 130 && c->F2 && emf_form(c) != 2;
}

// the t^n primitives and CFL signal speeds inside the VL predictor's y
// pencils (k_yprim) with pencil-mask bits 1 and 8: periodic boxes without a
// learned selector or a pressure floor, bit 3 clear
inline bool y_prim(const mhd_ctx* c)
{
    return (c->pencil_mask & 258) == 258 && c->sch.integrator == MHD_VL && !c->bc && !c->sel &&
           !(c->sch.pfloor > 0.0) && !fused_predictor(c);
}

// the conservative part of the VL full update inside the corrector's z
// pencils (k_zfull), the face field by CT alone after the edge fields (k_ct /
// k_ct4), with pencil-mask bits 2 and 9: as y_half (periodic boxes, no
// selector, the predictor and the edge fields as separate kernels)
inline bool z_full(const mhd_ctx* c)
{
    return (c->pencil_mask & 516) == 516 && c->sch.integrator == MHD_VL && !c->bc && !c->sel &&
           !fused_predictor(c) && emf_form(c) == 0;
}

template <class R, class TU, class TE>
void launch_ct(mhd_ctx* c, const Boxes& g, const StateP<TU, TE>& s, const R* E, cudaStream_t st)
{
    if constexpr (sizeof(TU) == 4 && sizeof(TE) == 4)
        k_ct4<R, TU, TE><<<c->quad_grid, CELL_THREADS, 0, st>>>(g, s, E, c->dtc);
    else
        k_ct<R, TU, TE><<<c->cell_grid, CELL_THREADS, 0, st>>>(g, s, E, c->dtc);
}

template <class R, class TU, class TE, int RECON, int SOLVER>
void launch_yhalf(mhd_ctx* c, const Boxes& g, const StateP<TU, TE>& s, const R* F, const R* E, TE* const Bh[3],
                  R* Wh, R* Fc, cudaStream_t st)
{
    k_yhalf<R, TU, TE, RECON, SOLVER><<<pencil_grid(c, 1), PENCIL_THREADS, 0, st>>>(
            g, s, F, E, c->dtc, c->gamma, c->sch.pfloor, Bh[0], Bh[1], Bh[2], Wh, Fc + 7 * g.N);
}

// k_emf_update: the edge fields of F and W, then the half (HALF: into Bh and
// Wh) or full update; persistent grid as launch_vl_predictor
template <class R, class TU, class TE, bool HALF>
void launch_emf_update(mhd_ctx* c, const Boxes& g, const StateP<TU, TE>& s, const R* F, const R* W, TE* const* Bh,
                       R* Wh, cudaStream_t st)
{
    constexpr size_t smem = emf_update_smem_bytes<R>();
    cudaFuncSetAttribute(k_emf_update<R, TU, TE, HALF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    static int per = 0;
    if (per <= 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_emf_update<R, TU, TE, HALF>, EU_THREADS, smem) !=
                cudaSuccess || nb < 1)
            nb = 1;
        per = nb;
    }
    const long long cap = (long long)per * c->nsm;
    const int grid = (int)(g.nftile < cap ? g.nftile : cap);
    k_emf_update<R, TU, TE, HALF><<<grid, EU_THREADS, smem, st>>>(g, s, F, W, c->dtc, c->gamma, HALF ? Bh[0] : nullptr,
                                                                 HALF ? Bh[1] : nullptr, HALF ? Bh[2] : nullptr, Wh,
                                                                 c->sch.pfloor);
}

// VL steps 1-3 in one launch: persistent grid of the blocks one SM keeps
// resident (registers and the kernel's shared memory) times the SMs; the
// shared-memory limit is raised on the instance this copy launches (see
// launch_emf)
template <class R, class TU, class TE, int SOLVER>
void launch_vl_predictor(mhd_ctx* c, const Boxes& g, const StateP<TU, TE>& s, const R* W, TE* const Bh[3], R* Wh,
                         cudaStream_t st)
{
    constexpr size_t smem = PredSmem<R, TE>::bytes;
    cudaFuncSetAttribute(k_vl_predictor<R, TU, TE, SOLVER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    static int per = 0;
    if (per <= 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_vl_predictor<R, TU, TE, SOLVER>, PRED_THREADS,
                                                          smem) != cudaSuccess || nb < 1)
            nb = 1;
        per = nb;
    }
    const long long cap = (long long)per * c->nsm;
    const int grid = (int)(g.nftile < cap ? g.nftile : cap);
    k_vl_predictor<R, TU, TE, SOLVER><<<grid, PRED_THREADS, smem, st>>>(g, s, W, c->dtc, c->gamma, Bh[0], Bh[1], Bh[2],
                                                                       Wh, c->sch.pfloor);
}

// CTU steps 5-6 along axis D (periodic or outflow instantiation): by
// pencils along y and z and by warps along a periodic x where the pencil
// mask has the axis, else per cell
template <class R, int SOLVER, class TE, int D>
void ctu_correct_axis(mhd_ctx* c, const Boxes& g, const R* WM, const R* WP, const R* W, const R* F1, const TE* BhD,
                      R* F2, double gam, const R* fo1, int cs, R* fo2, cudaStream_t st)
{
    const long long o = (long long)D * 7 * g.N;
    if constexpr (D == 0) {
        if ((c->pencil_mask & 1) && !(c->bc & 1)) {   // by warps along a periodic x
            if (c->bc)
                k_ctu_xwarp<R, SOLVER, TE, true><<<xrow_grid(c), PENCIL_THREADS, 0, st>>>(
                    g, WM, WP, W, F1, BhD, F2, c->dtc, gam, fo1, cs);
            else
                k_ctu_xwarp<R, SOLVER, TE><<<xrow_grid(c), PENCIL_THREADS, 0, st>>>(g, WM, WP, W, F1, BhD, F2,
                                                                                   c->dtc, gam);
            return;
        }
    }
    if constexpr (D > 0) {
        if (c->pencil_mask >> D & 1) {
            if (c->bc)
                k_ctu_pencil<R, SOLVER, TE, D, true><<<pencil_grid(c, D), PENCIL_THREADS, 0, st>>>(
                    g, WM + o, WP + o, W, F1, BhD, F2 + o, c->dtc, gam, fo1, cs, fo2);
            else
                k_ctu_pencil<R, SOLVER, TE, D><<<pencil_grid(c, D), PENCIL_THREADS, 0, st>>>(
                    g, WM + o, WP + o, W, F1, BhD, F2 + o, c->dtc, gam);
            return;
        }
    }
    if (c->bc)
        k_ctu_correct<R, SOLVER, TE, D, true><<<c->cell_grid, CELL_THREADS, 0, st>>>(
            g, WM + o, WP + o, W, F1, BhD, F2 + o, c->dtc, gam, fo1, cs, fo2);
    else
        k_ctu_correct<R, SOLVER, TE, D><<<c->cell_grid, CELL_THREADS, 0, st>>>(g, WM + o, WP + o, W, F1, BhD, F2 + o,
                                                                           c->dtc, gam);
}

template <class R, class TU, class TE, int INTEG, int RECON, int SOLVER>
void run_step(mhd_ctx* c, bool device_dt)
{
    const Boxes g = c->B;
    const long long n = g.N;
    const int nb = c->cell_grid;
    cudaStream_t st = c->stream;
    StateP<TU, TE> s = state_of<TU, TE>(c);
    R* W = (R*)c->W;
    R* Wh = (R*)c->Wh;
    R* F1 = (R*)c->F1;
    R* F2 = (R*)c->F2;
    R* E = (R*)c->E;
    TE* Bh[3] = {(TE*)c->Bh[0], (TE*)c->Bh[1], (TE*)c->Bh[2]};
    const double gam = c->gamma;
    const size_t smem = sweep_smem_bytes<R>(RECON, g.tl);

    // VL with pencil-mask bit 8: the primitives inside the y predictor (its
    // time goes to the primitive group)
    const bool yp = INTEG == VL && y_prim(c);
    prof_mark(c, 0);
    if (yp)
        k_yprim<R, TU, TE, SOLVER><<<pencil_grid(c, 1), PENCIL_THREADS, 0, st>>>(
            g, s, W, gam, device_dt ? c->smax_part : nullptr, c->bad, F1 + 7 * n);
    else if (c->bc)
        k_prim<R, TU, TE, true><<<nb, CELL_THREADS, 0, st>>>(g, s, W, gam, device_dt ? c->smax_part : nullptr,
                                                             c->bad, c->sch.pfloor, c->nfloor);
    else if constexpr (sizeof(TU) == 4 && sizeof(TE) == 4)
        k_prim4<R, TU, TE><<<c->quad_grid, CELL_THREADS, 0, st>>>(g, s, W, gam, device_dt ? c->smax_part : nullptr,
                                                                   c->bad, c->sch.pfloor, c->nfloor);
    else
        k_prim<R, TU, TE><<<nb, CELL_THREADS, 0, st>>>(g, s, W, gam, device_dt ? c->smax_part : nullptr, c->bad,
                                                       c->sch.pfloor, c->nfloor);
    if (device_dt) k_finalize_dt<<<(c->nbox + 127) / 128, 128, 0, st>>>(g, c->smax_part, c->sch.cfl, c->dt, c->smax, c->dtc);
    prof_mark(c, 1);

    if (INTEG == VL) {
        const int cs = c->bc ? cross_size(c->hbox[0].nx, c->hbox[0].ny, c->hbox[0].nz) : 0;
        const bool yh = y_half(c);
        if (fused_predictor(c)) {
            // VL steps 1-3 in one kernel (its time goes to the half-update group)
            for (int b = 2; b <= 5; b++) prof_mark(c, b);
            launch_vl_predictor<R, TU, TE, SOLVER>(c, g, s, W, Bh, Wh, st);
            prof_mark(c, 6);
        } else {
            // VL steps 1-3: first-order fluxes with the face B_n, edge E, half update
            for (int d = 0; d < 3; d++) {
                if (d == 1 && yp)
                    ;                                   // done with the primitives
                else if (d == 0 && x_pencils(c))
                    launch_xpencil<R, RECON, SOLVER, 0, TE>(c, g, W, s.b[0], F1, st);
                else if (d == 0 && x_march<RECON, 0>(c))
                    launch_xmarch<R, RECON, SOLVER, 0, TE>(c, g, W, s.b[0], F1, st);
                else if ((c->pencil_mask >> d & 1) && d == 0)
                    k_xwarp<R, RECON, SOLVER, 0, TE><<<xrow_grid(c), PENCIL_THREADS, 0, st>>>(
                        g, W, s.b[d], F1, gam, XW<RECON, 0>::slot);
                else if (c->pencil_mask >> d & 1)
                    launch_pencil<R, RECON, SOLVER, 0, TE>(d, pencil_grid(c, d), st, g, W, s.b[d],
                                                           F1 + (long long)d * 7 * n, gam);
                else
                    k_sweep<R, RECON, SOLVER, 0, TE><<<sweep_grid(c, d), SWEEP_THREADS, 0, st>>>(
                        g, d, W, s.b[d], F1 + (long long)d * 7 * n, nullptr, nullptr, c->dtc, gam);
                prof_mark(c, 2 + d);
            }
            if (emf_form(c) == 2) {   // edge fields and half update in one kernel (its time: the half group)
                prof_mark(c, 5);
                launch_emf_update<R, TU, TE, true>(c, g, s, F1, W, Bh, Wh, st);
            } else {
                launch_emf<R>(c, g, F1, W, E, st);
                prof_mark(c, 5);
                for (int d = 0; d < 3; d++)
                    if (c->bc >> d & 1)
                        k_outer_flux<R, SOLVER, TE><<<(cs + 127) / 128, 128, 0, st>>>(c->hbox[0], d, W, s.b[d],
                                                                                     gam, n, (R*)c->fout, cs);
                if (c->bc)
                    k_half<R, TU, TE, true><<<nb, CELL_THREADS, 0, st>>>(g, s, F1, E, c->dtc, gam, Bh[0], Bh[1],
                                                                         Bh[2], Wh, c->sch.pfloor,
                                                                         (const R*)c->fout, cs);
                else if (yh)     // the half update inside the y corrector pencils (its time: the half group)
                    launch_yhalf<R, TU, TE, RECON, SOLVER>(c, g, s, F1, E, Bh, Wh, F2, st);
                else
                    launch_half<R, TU, TE>(c, g, s, F1, E, Bh, Wh, st);
            }
            prof_mark(c, 6);
        }
        // VL steps 4-7: reconstruct at the half step, Riemann, edge E, full
        // update; the corrector's fluxes go to F2 when the y sweep ran fused
        // with the half update (the predictor's F1 was read while it ran)
        R* Fc = yh ? F2 : F1;
        const bool zf = z_full(c);
        for (int d = 0; d < 3; d++) {
            if (d == 1 && yh)
                ;                                       // done with the half update
            else if (d == 2 && zf)                      // with the conservative full update
                k_zfull<R, TU, TE, RECON, SOLVER><<<pencil_grid(c, 2), PENCIL_THREADS, 0, st>>>(
                    g, s, Wh, Bh[2], Fc, c->dtc, gam);
            else if (d == 0 && x_pencils(c))
                launch_xpencil<R, RECON, SOLVER, 1, TE>(c, g, Wh, Bh[0], Fc, st);
            else if (d == 0 && x_march<RECON, 1>(c))
                launch_xmarch<R, RECON, SOLVER, 1, TE>(c, g, Wh, Bh[0], Fc, st);
            else if ((c->pencil_mask >> d & 1) && d == 0)
                k_xwarp<R, RECON, SOLVER, 1, TE><<<xrow_grid(c), PENCIL_THREADS, 0, st>>>(
                    g, Wh, Bh[d], Fc, gam, XW<RECON, 1>::slot);
            else if (c->pencil_mask >> d & 1)
                launch_pencil<R, RECON, SOLVER, 1, TE>(d, pencil_grid(c, d), st, g, Wh, Bh[d],
                                                       Fc + (long long)d * 7 * n, gam);
            else
                k_sweep<R, RECON, SOLVER, 1, TE><<<sweep_grid(c, d), SWEEP_THREADS, smem, st>>>(
                    g, d, Wh, Bh[d], Fc + (long long)d * 7 * n, nullptr, nullptr, c->dtc, gam);
            prof_mark(c, 7 + d);
        }
        if (emf_form(c) == 2) {       // edge fields and full update in one kernel (the full group)
            prof_mark(c, 10);
            launch_emf_update<R, TU, TE, false>(c, g, s, F1, Wh, nullptr, nullptr, st);
        } else {
            launch_emf<R>(c, g, Fc, Wh, E, st);
            prof_mark(c, 10);
            for (int d = 0; d < 3; d++)
                if (c->bc >> d & 1)
                    k_outer_flux<R, SOLVER, TE><<<(cs + 127) / 128, 128, 0, st>>>(c->hbox[0], d, Wh, Bh[d], gam,
                                                                                 n, (R*)c->fout, cs);
            if (c->bc)
                k_full<R, TU, TE, true><<<nb, CELL_THREADS, 0, st>>>(g, s, F1, E, c->dtc, (const R*)c->fout, cs);
            else if (zf)
                launch_ct<R, TU, TE>(c, g, s, E, st);
            else
                launch_full<R, TU, TE>(c, g, s, Fc, E, st);
        }
        fix_layers(c, s, st);
        prof_mark(c, 11);
    } else {
        R* WM = (R*)c->WM;
        R* WP = (R*)c->WP;
        // CTU steps 1-2: traced states (+ source terms) and their fluxes, by
        // pencils on y and z and warps on x (x periodic) where the pencil
        // mask has the axis, else by tiles
        for (int d = 0; d < 3; d++) {
            if (d == 0 && x_march<RECON, 2>(c) && !(c->bc & 1))
                launch_xmarch<R, RECON, SOLVER, 2, TE>(c, g, W, s.b[0], F1, st, WM, WP);
            else if ((c->pencil_mask & 1) && d == 0 && !(c->bc & 1))
                k_xwarp<R, RECON, SOLVER, 2, TE><<<xrow_grid(c), PENCIL_THREADS, 0, st>>>(
                    g, W, s.b[0], F1, gam, XW<RECON, 2>::slot, nullptr, nullptr, WM, WP, c->dtc);
            else if ((c->pencil_mask >> d & 1) && d > 0)
                launch_pencil<R, RECON, SOLVER, 2, TE>(d, pencil_grid(c, d), st, g, W, s.b[d],
                                                       F1 + (long long)d * 7 * n, gam, nullptr, nullptr,
                                                       WM + (long long)d * 7 * n, WP + (long long)d * 7 * n, c->dtc);
            else if (d == 0)
                k_sweep<R, RECON, SOLVER, 2, TE, 0><<<sweep_grid(c, d), SWEEP_THREADS, smem, st>>>(
                    g, d, W, s.b[d], F1, WM, WP, c->dtc, gam);
            else if (d == 1)
                k_sweep<R, RECON, SOLVER, 2, TE, 1><<<sweep_grid(c, d), SWEEP_THREADS, smem, st>>>(
                    g, d, W, s.b[d], F1 + (long long)7 * n, WM + (long long)7 * n, WP + (long long)7 * n, c->dtc,
                    gam);
            else
                k_sweep<R, RECON, SOLVER, 2, TE, 2><<<sweep_grid(c, d), SWEEP_THREADS, smem, st>>>(
                    g, d, W, s.b[d], F1 + (long long)14 * n, WM + (long long)14 * n, WP + (long long)14 * n,
                    c->dtc, gam);
            prof_mark(c, 2 + d);
        }
        // steps 3-4: edge E at t^n, dt/2 update of face B and cell state
        const bool eu = emf_form(c) == 2;
        if (eu) {
            prof_mark(c, 5);
            launch_emf_update<R, TU, TE, true>(c, g, s, F1, W, Bh, Wh, st);
        } else {
            launch_emf<R>(c, g, F1, W, E, st);
            prof_mark(c, 5);
        }
        // outflow: stage-1 fluxes through the outer faces (the last cells'
        // own traced states) into the first half of the outer-flux buffer;
        // the corrections write the stage-2 ones into the second half
        const int cs = c->bc ? cross_size(c->hbox[0].nx, c->hbox[0].ny, c->hbox[0].nz) : 0;
        R* fo1 = (R*)c->fout;
        R* fo2 = c->bc ? fo1 + (long long)21 * cs : nullptr;
        for (int d = 0; d < 3; d++)
            if (c->bc >> d & 1)
                k_outer_flux_traced<R, SOLVER, TE><<<(cs + 127) / 128, 128, 0, st>>>(
                    c->hbox[0], d, WP + (long long)d * 7 * n, WM + (long long)d * 7 * n, s.b[d], gam, n, fo1, cs);
        const bool cyh = ctu_y_half(c);
        if (c->bc)
            k_half<R, TU, TE, true><<<nb, CELL_THREADS, 0, st>>>(g, s, F1, E, c->dtc, gam, Bh[0], Bh[1], Bh[2], Wh,
                                                                 c->sch.pfloor, fo1, cs);
        else if (cyh)           // the dt/2 update with the y correction (its time: the half group)
            k_ctu_yhalf<R, TU, TE, SOLVER><<<pencil_grid(c, 1), PENCIL_THREADS, 0, st>>>(
                g, s, WM + (long long)7 * n, WP + (long long)7 * n, W, F1, E, F2 + (long long)7 * n, c->dtc, gam,
                c->sch.pfloor, Bh[0], Bh[1], Bh[2], Wh);
        else if (!eu)
            launch_half<R, TU, TE>(c, g, s, F1, E, Bh, Wh, st);
        prof_mark(c, 6);
        // steps 5-6: transverse correction and corrector fluxes
        ctu_correct_axis<R, SOLVER, TE, 0>(c, g, WM, WP, W, F1, Bh[0], F2, gam, fo1, cs, fo2, st);
        prof_mark(c, 7);
        if (!cyh) ctu_correct_axis<R, SOLVER, TE, 1>(c, g, WM, WP, W, F1, Bh[1], F2, gam, fo1, cs, fo2, st);
        prof_mark(c, 8);
        const bool czf = ctu_z_full(c);
        if (czf)                // with the conservative full update
            k_ctu_zfull<R, TU, TE, SOLVER><<<pencil_grid(c, 2), PENCIL_THREADS, 0, st>>>(g, s, WM, WP, W, F1, Bh[2],
                                                                                     F2, c->dtc, gam);
        else
            ctu_correct_axis<R, SOLVER, TE, 2>(c, g, WM, WP, W, F1, Bh[2], F2, gam, fo1, cs, fo2, st);
        prof_mark(c, 9);
        // steps 7-8
        if (eu) {
            prof_mark(c, 10);
            launch_emf_update<R, TU, TE, false>(c, g, s, F2, Wh, nullptr, nullptr, st);
        } else {
            launch_emf<R>(c, g, F2, Wh, E, st);
            prof_mark(c, 10);
            if (c->bc)
                k_full<R, TU, TE, true><<<nb, CELL_THREADS, 0, st>>>(g, s, F2, E, c->dtc, fo2, cs);
            else if (czf)
                launch_ct<R, TU, TE>(c, g, s, E, st);
            else
                launch_full<R, TU, TE>(c, g, s, F2, E, st);
        }
        fix_layers(c, s, st);
        prof_mark(c, 11);
    }
    if (c->prof_on && c->prof_steps < c->prof_cap) c->prof_steps++;
}

template <class R, class TE, int RECON, int SOLVER, int MODE>
inline cudaError_t allow_smem()
{
    size_t b = sweep_smem_bytes<R>(RECON, TL_MAX);
    cudaError_t e = cudaFuncSetAttribute(k_emf<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)emf_smem_bytes<R>());
    if constexpr (sizeof(R) == 4) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_emf_tma<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)emf_tma_smem_bytes());
    }
    if (e != cudaSuccess || MODE == 0) return e;
    if constexpr (MODE == 2) {   // the CTU tracing sweeps run with the axis fixed at compile time
        e = cudaFuncSetAttribute(k_sweep<R, RECON, SOLVER, MODE, TE, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)b);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_sweep<R, RECON, SOLVER, MODE, TE, 1>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_sweep<R, RECON, SOLVER, MODE, TE, 2>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
        return e;
    } else {
        return cudaFuncSetAttribute(k_sweep<R, RECON, SOLVER, MODE, TE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)b);
    }
}

// pick the step function of one precision; returns nullptr if not built
template <class R, class TU, class TE>
mhd_step_fn pick_step(int integ, int recon, int solver, cudaError_t* attr)
{
#define MHD_CASE(I, RC, S)                                                              \
    if (integ == I && recon == RC && solver == S) {                                     \
        *attr = allow_smem<R, TE, RC, S, (I == VL ? 1 : 2)>();                          \
        return &run_step<R, TU, TE, I, RC, S>;                                          \
    }
    MHD_CASE(VL, PLM, ROE) MHD_CASE(VL, PLM, HLLD) MHD_CASE(VL, PLM, HLLE)
    MHD_CASE(VL, PPM, ROE) MHD_CASE(VL, PPM, HLLD) MHD_CASE(VL, PPM, HLLE)
    MHD_CASE(VL, PLM_PRIM, ROE) MHD_CASE(VL, PLM_PRIM, HLLD) MHD_CASE(VL, PLM_PRIM, HLLE)
    MHD_CASE(CTU, PLM, ROE) MHD_CASE(CTU, PLM, HLLD) MHD_CASE(CTU, PLM, HLLE)
    MHD_CASE(CTU, PPM, ROE) MHD_CASE(CTU, PPM, HLLD) MHD_CASE(CTU, PPM, HLLE)
#undef MHD_CASE
    *attr = cudaSuccess;
    return nullptr;
}

}  // namespace mhd

// per-precision entry points (one compilation unit each)
mhd_step_fn mhd_pick_fp64(int integ, int recon, int solver, cudaError_t* attr);
mhd_step_fn mhd_pick_fp32(int integ, int recon, int solver, cudaError_t* attr);
mhd_step_fn mhd_pick_mixed(int integ, int recon, int solver, cudaError_t* attr);
