// mhd_capi.cu -- the C ABI declared in include/mhd.h.
#include <stdarg.h>
#include <cmath>
#include <stdlib.h>
#include <string.h>
#include <cufft.h>
#include <cudaTypedefs.h>
#include "mhd_engine.cuh"

using namespace mhd;

static mhd_status fail(mhd_ctx* c, mhd_status s, const char* fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
        if (c->sticky == MHD_OK) c->sticky = s;
    }
    return s;
}

#define CK(call)                                                                                \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(c, MHD_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static const char* g_init_err = "no error";

// lets the allocation-free entry point report argument errors through
// mhd_last_error(NULL)
void mhd_internal_set_init_error(const char* msg) { g_init_err = msg; }

// the learned selector's lists follow the sweep layout (mhd_learned.cu)
mhd_status mhd_internal_selector_lists(mhd_ctx* c);

static void release(mhd_ctx* c)
{
    void* bufs[] = {c->rho, c->m[0], c->m[1], c->m[2], c->e, c->b[0], c->b[1], c->b[2], c->W, c->Wh,
                    c->F1, c->F2, c->E, c->Bh[0], c->Bh[1], c->Bh[2], c->WM, c->WP, c->stage,
                    c->dt, c->dtc, c->smax, c->smax_part, c->bad, c->nfloor, c->part, c->diag, c->dbox, c->sel_feats,
                    c->sel_flags, c->sel_cnt, c->sel_list[0], c->sel_list[1], c->sel_list[2], c->sel_list[3],
                    c->sel_list[4], c->sel_list[5], c->sel_list[6], c->sel_list[7], c->fout, c->perr};
    for (void* p : bufs)
        if (p) cudaFree(p);
    free(c->tmaps);
    if (c->have_graph) cudaGraphExecDestroy(c->gexec);
    if (c->prof_ev) {
        for (int q = 0; q < c->prof_cap * (MHD_NGROUPS + 1); q++) cudaEventDestroy(c->prof_ev[q]);
        free(c->prof_ev);
    }
    free(c->hbox);
    if (c->sel_fork) cudaEventDestroy(c->sel_fork);
    if (c->sel_join) cudaEventDestroy(c->sel_join);
    if (c->sel_st) cudaStreamDestroy(c->sel_st);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

static cudaError_t dalloc(mhd_ctx* c, void** p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) c->bytes += (long long)bytes;
    return e;
}

// the second flux array of a VL context, on first use: the corrector's
// fluxes when its y sweep runs fused with the half update (pencil-mask bit 7)
static cudaError_t ensure_f2(mhd_ctx* c)
{
    if (c->F2 || c->sch.integrator != MHD_VL) return cudaSuccess;
    cudaError_t e = dalloc(c, &c->F2, 21 * (size_t)c->B.N * c->szr);
    if (e != cudaSuccess) {
        c->F2 = nullptr;
        cudaGetLastError();   // an allocation failure is not sticky: clear it for the next check
    }
    return e;
}

// the driver's tensor-map encoder, looked up once through the runtime (no
// link against the driver library)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// nf fields of a one-box array of 4-byte values as a 4-D tensor
// (nx, ny, nz, nf), copied in boxes of one staged plane of bf fields
static bool encode_planes(CUtensorMap* m, void* base, const BoxDev& b, int nf, int bf)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || !base) return false;
    const cuuint64_t dim[4] = {(cuuint64_t)b.nx, (cuuint64_t)b.ny, (cuuint64_t)b.nz, (cuuint64_t)nf};
    const cuuint64_t stride[3] = {(cuuint64_t)b.nx * 4, (cuuint64_t)b.nx * b.ny * 4, (cuuint64_t)b.n * 4};
    const cuuint32_t box[4] = {(cuuint32_t)TMA_X, (cuuint32_t)TmaPlane<TMA_TY>::Y, 1, (cuuint32_t)bf};
    const cuuint32_t step[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dim, stride, box, step, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// k_emf_tma where the context allows it: one box, 4-byte arithmetic, rows a
// multiple of 16 bytes (nx % 4 == 0; every stride of the tensors is then one
// too) and planes at least one staged plane wide; else k_emf
static void setup_emf_tma(mhd_ctx* c)
{
    const int was = c->emf_tma;
    c->emf_tma = 0;
    if (c->emf_stage_req == 1 && c->nbox == 1 && c->szr == 4) {
        const BoxDev& b = c->hbox[0];
        if (b.nx % 4 == 0 && b.nx >= TMA_X && b.ny >= TmaPlane<TMA_TY>::Y) {
            if (!c->tmaps) c->tmaps = (CUtensorMap*)aligned_alloc(64, 6 * sizeof(CUtensorMap));
            // W, Wh: 3 fields a copy (v, B); F1, F2: the mass flux, then the two B fluxes
            bool ok = c->tmaps && encode_planes(&c->tmaps[0], c->W, b, 8, 3) &&
                      encode_planes(&c->tmaps[1], c->Wh, b, 8, 3) && encode_planes(&c->tmaps[2], c->F1, b, 21, 1) &&
                      encode_planes(&c->tmaps[3], c->F1, b, 21, 2);
            if (ok && c->F2)
                ok = encode_planes(&c->tmaps[4], c->F2, b, 21, 1) && encode_planes(&c->tmaps[5], c->F2, b, 21, 2);
            else if (ok) {
                c->tmaps[4] = c->tmaps[2];
                c->tmaps[5] = c->tmaps[3];
            }
            // resident blocks per SM, by this unit's instance (the others have
            // the same resources and get the same attribute where they launch)
            int per = 0;
            ok = ok &&
                 cudaFuncSetAttribute(k_emf_tma<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)emf_tma_smem_bytes()) == cudaSuccess &&
                 cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_emf_tma<float>, EMF_TMA_THREADS,
                                                               emf_tma_smem_bytes()) == cudaSuccess &&
                 per >= 1;
            if (ok) {
                const long long nt = (long long)((b.nx + ETX - 1) / ETX) * ((b.ny + TMA_TY - 1) / TMA_TY) *
                                     ((b.nz + EZC - 1) / EZC);
                const long long cap = (long long)per * c->nsm;
                c->emf_tma_grid = (int)(nt < cap ? nt : cap);
                c->emf_tma = 1;
            }
        }
    }
    if (c->emf_tma != was && c->have_graph) {   // a captured step holds the other kernel
        cudaGraphExecDestroy(c->gexec);
        c->have_graph = false;
    }
}

// tile prefix sums of the box table for tile length tl; uploads the table
static void apply_fixed_layers(mhd_ctx* c);
static void count_launches(mhd_ctx* c);

static cudaError_t layout_tiles(mhd_ctx* c, int tl)
{
    int t0[3] = {0, 0, 0}, e0 = 0, f0 = 0;
    long long p0[3] = {0, 0, 0}, w0[3] = {0, 0, 0}, r0 = 0, xq = 0;
    for (int b = 0; b < c->nbox; b++) {
        BoxDev& x = c->hbox[b];
        for (int d = 0; d < 3; d++) {
            x.tile0[d] = t0[d];
            t0[d] += tiles_of_box(x.nx, x.ny, x.nz, d, tl);
        }
        x.etile0 = e0;
        e0 += emf_tiles_of_box(x.nx, x.ny, x.nz);
        x.ftile0 = f0;
        f0 += pred_tiles_of_box(x.nx, x.ny, x.nz, PRED_FZ);
        for (int d = 0; d < 3; d++) {
            x.pth0[d] = p0[d];
            p0[d] += pencil_threads_of_box(x.nx, x.ny, x.nz, d, c->pencil_len);
        }
        for (int q = 0; q < 3; q++) {
            x.xw0[q] = w0[q];
            w0[q] += xwarp_items_of_box(x.nx, x.ny, x.nz, q);
        }
        x.xr0 = r0;
        r0 += (long long)x.ny * x.nz;
        x.xp0 = xq;
        xq += xpencil_threads_of_box(x.nx, x.ny, x.nz, c->pencil_len);
    }
    c->B.nxp = xq;
    c->B.nxr = r0;
    c->B.pl = c->pencil_len;
    for (int d = 0; d < 3; d++) c->B.npth[d] = p0[d];
    for (int q = 0; q < 3; q++) c->B.nxw[q] = w0[q];
    c->B.tl = tl;
    for (int d = 0; d < 3; d++) c->B.ntile[d] = t0[d];
    c->B.netile = e0;
    c->B.nftile = f0;
    c->B.fz = PRED_FZ;
    count_launches(c);
    if (c->have_graph) {   // a captured step holds the old tile layout
        cudaGraphExecDestroy(c->gexec);
        c->have_graph = false;
    }
    cudaError_t e = cudaMemcpyAsync(c->dbox, c->hbox, sizeof(BoxDev) * c->nbox, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e;
}

// nx*ny*nz < limit, decided without forming a product that could wrap
static bool cells_below(int nx, int ny, int nz, long long limit)
{
    const long long a = nx, b = ny, c = nz;
    if (a >= limit) return false;
    if (b >= (limit + a - 1) / a) return false;            // a*b < limit, a*b fits
    const long long ab = a * b;
    return c < (limit + ab - 1) / ab;                       // a*b*c < limit
}

static mhd_status init_common(int nbox, const mhd_grid* grids, double gamma, const mhd_scheme* scheme, void* stream,
                              mhd_ctx** out)
{
    if (!out) return MHD_EINVAL;
    *out = nullptr;
    if (nbox < 1 || !grids || !scheme) { g_init_err = "null grid or scheme, or no box"; return MHD_EINVAL; }
    for (int b = 0; b < nbox; b++)
        if (grids[b].nx < 1 || grids[b].ny < 1 || grids[b].nz < 1 || !(grids[b].dx > 0.0) ||
            !cells_below(grids[b].nx, grids[b].ny, grids[b].nz, 1LL << 31)) {
            g_init_err = "bad grid (sides >= 1, dx > 0, fewer than 2^31 cells per box)";
            return MHD_EINVAL;
        }
    if (!(gamma > 1.0)) { g_init_err = "gamma must exceed 1"; return MHD_EINVAL; }
    if (scheme->integrator < 0 || scheme->integrator > 1 || scheme->recon < 0 || scheme->recon > 2 ||
        scheme->riemann < 0 || scheme->riemann > 2 || scheme->precision < 0 || scheme->precision > 2) {
        g_init_err = "bad scheme enum";
        return MHD_EINVAL;
    }
    if (!(scheme->pfloor >= 0.0)) { g_init_err = "pfloor must be >= 0"; return MHD_EINVAL; }
    if (scheme->integrator == MHD_CTU && scheme->recon == MHD_PLM_PRIM) {
        g_init_err = "PLM_PRIM is built for VL only";
        return MHD_EUNSUPPORTED;
    }
    mhd_ctx* c = (mhd_ctx*)calloc(1, sizeof(mhd_ctx));
    if (!c) return MHD_ENOMEM;
    strcpy(c->err, "no error");
    c->grid = grids[0];
    c->sch = *scheme;
    c->gamma = gamma;
    c->nbox = nbox;
    c->hbox = (BoxDev*)calloc((size_t)nbox, sizeof(BoxDev));
    if (!c->hbox) { free(c); return MHD_ENOMEM; }
    long long off = 0, vb = 0;
    for (int b = 0; b < nbox; b++) {
        BoxDev& x = c->hbox[b];
        x.nx = grids[b].nx; x.ny = grids[b].ny; x.nz = grids[b].nz;
        x.n = (long long)x.nx * x.ny * x.nz;
        x.off = off;
        x.vblk0 = vb;
        x.dx = grids[b].dx;
        x.inv_dx = (float)(1.0 / grids[b].dx);
        off += x.n;
        vb += (x.n + CELL_THREADS - 1) / CELL_THREADS;
    }
    const long long n = off;
    // the x-quad kernels: a box whose rows, offset and field stride are all
    // multiples of 4 cells (16-byte aligned in every field array) takes four
    // cells along x per thread, any other box one
    long long vq = 0;
    for (int b = 0; b < nbox; b++) {
        BoxDev& x = c->hbox[b];
        x.quad = x.nx % 4 == 0 && x.off % 4 == 0 && n % 4 == 0;
        x.vq0 = vq;
        vq += x.quad ? (x.n / 4 + CELL_THREADS - 1) / CELL_THREADS : (x.n + CELL_THREADS - 1) / CELL_THREADS;
    }
    c->B.nbox = nbox;
    c->B.N = n;
    c->B.nvblk = vb;
    c->B.nvq = vq;
    cudaError_t attr = cudaSuccess;
    switch (scheme->precision) {
        case MHD_FP64: c->szu = 8; c->sze = 8; c->szr = 8; c->step = mhd_pick_fp64(scheme->integrator, scheme->recon, scheme->riemann, &attr); break;
        case MHD_FP32: c->szu = 4; c->sze = 4; c->szr = 4; c->step = mhd_pick_fp32(scheme->integrator, scheme->recon, scheme->riemann, &attr); break;
        default:       c->szu = 4; c->sze = 8; c->szr = 4; c->step = mhd_pick_mixed(scheme->integrator, scheme->recon, scheme->riemann, &attr); break;
    }
    if (!c->step) { free(c->hbox); free(c); g_init_err = "scheme combination not built"; return MHD_EUNSUPPORTED; }
    c->plain_step = c->step;
    if (attr != cudaSuccess) { free(c->hbox); free(c); g_init_err = "cudaFuncSetAttribute failed"; return MHD_ECUDA; }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev);
    c->sweep_bps = 4;
    // register sweeps on every axis: pencils along y and z, warps along x
    // (CTU with an outflow x axis: tiles along x).  VL: for FP64 x by staged
    // pencils (bit 4); for FP32 and mixed x by aligned marching warps (bits
    // 5 and 6; the PPM corrector keeps its overlapping warps).  CTU: the
    // PLM tracing along x by aligned marching warps (bit 5).  The fused
    // predictor (bit 3) is not a default: at 256^3 it ties the sweeps it
    // replaces (its halo solves and plane barriers cost what it saves in
    // traffic).  FP32 and mixed PLM: the half update inside the y corrector
    // pencils (bit 7; 256^3 FP32 Roe: 0.708 ms against 0.439 + 0.475 for the
    // two kernels, mixed 1.90 against 1.46 + 0.49); FP64 keeps the two (its
    // corrector is bound by the FP64 pipe: 30.8 against 2.8 + 27.5 ms).  The
    // mixed form also forms the t^n primitives inside the y predictor pencils
    // (bit 8; 256^3 PLM + Roe: 0.718 ms against 0.644 + 0.307, whose FP64
    // per-cell arithmetic then overlaps the sweep's); in FP32 and FP64 that
    // ties the two kernels (0.451 against 0.179 + 0.267 ms; 20.2 against
    // 5.4 + 14.8 ms).  FP32 PPM takes the half update in the y corrector too
    // (256^3 Roe: step 4.86 -> 4.71 ms, HLLD 4.87 -> 4.67); the mixed PPM
    // form ties with it (6.47 against 6.48 ms).  FP32 PLM also runs the conservative part of the full
    // update inside the z corrector pencils and the face field by CT alone
    // (bit 9; 256^3 Roe: z corrector 0.468 -> 0.685 ms, full update 0.412 ->
    // 0.098, step 3.67 -> 3.58 ms); the mixed form (5.43 -> 5.51 ms) and FP64
    // (144.0 -> 144.8 ms) lose with it.  CTU FP32 and mixed run the dt/2
    // update inside the y pencils of the transverse correction (bit 7; 256^3
    // PLM + Roe 5.32 -> 5.22 ms, PPM + HLLD 6.23 -> 6.09, mixed 7.11 -> 6.79);
    // FP64 ties (128^3: 24.65 against 24.69 ms) and keeps 39.  CTU FP32 also
    // runs the conservative update inside the z correction pencils (bit 9;
    // 5.23 -> 5.18 ms, PPM + HLLD 6.09 -> 6.06); mixed loses with it (6.79 ->
    // 6.93 ms).  The autotuner may change the mask.
    if (scheme->integrator != MHD_VL)   // FP32, mixed: the dt/2 update in the y correction (bit 7),
        c->pencil_mask = scheme->precision == MHD_FP64 ? 39 : (scheme->precision == MHD_FP32 ? 679 : 167);   // FP32:
                                        // and the conservative update in the z correction (bit 9)
    else if (scheme->precision == MHD_FP64)
        c->pencil_mask = 23;
    else if (scheme->precision == MHD_FP32)   // PLM: the half update in the y corrector, the conservative
        c->pencil_mask = 743;                    // update in the z corrector (PLM, or a selector's cheap sweep)
    else
        c->pencil_mask = scheme->recon != MHD_PPM ? 487 : 359;   // mixed: and the primitives in the y predictor
    c->pencil_len = 32;
    c->cell_grid = (int)(vb < 16LL * c->nsm ? vb : 16LL * c->nsm);
    if (c->cell_grid < 1) c->cell_grid = 1;
    c->quad_grid = (int)(vq < 16LL * c->nsm ? vq : 16LL * c->nsm);
    if (c->quad_grid < 1) c->quad_grid = 1;
    if (e == cudaSuccess) {
        if (stream) {
            c->stream = (cudaStream_t)stream;
        } else {
            e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
            c->own_stream = true;
        }
    }
    const bool ctu = scheme->integrator == MHD_CTU;
    if (e == cudaSuccess) e = dalloc(c, &c->rho, n * c->szu);
    for (int d = 0; d < 3 && e == cudaSuccess; d++) e = dalloc(c, &c->m[d], n * c->szu);
    if (e == cudaSuccess) e = dalloc(c, &c->e, n * c->sze);
    for (int d = 0; d < 3 && e == cudaSuccess; d++) e = dalloc(c, &c->b[d], n * c->sze);
    if (e == cudaSuccess) e = dalloc(c, &c->W, 8 * n * c->szr);
    if (e == cudaSuccess) e = dalloc(c, &c->Wh, 8 * n * c->szr);
    if (e == cudaSuccess) e = dalloc(c, &c->F1, 21 * n * c->szr);
    // (VL: the second flux array for the y corrector fused with the half
    // update, pencil-mask bit 7, the FP32 and mixed PLM default)
    if (e == cudaSuccess && (ctu || (c->pencil_mask & 128))) e = dalloc(c, &c->F2, 21 * n * c->szr);
    if (e == cudaSuccess) e = dalloc(c, &c->E, 3 * n * c->szr);
    for (int d = 0; d < 3 && e == cudaSuccess; d++) e = dalloc(c, &c->Bh[d], n * c->sze);
    if (e == cudaSuccess && ctu) e = dalloc(c, &c->WM, 21 * n * c->szr);
    if (e == cudaSuccess && ctu) e = dalloc(c, &c->WP, 21 * n * c->szr);
    if (e == cudaSuccess && scheme->precision == MHD_MIXED) e = dalloc(c, &c->stage, 4 * n * sizeof(double));
    if (e == cudaSuccess) e = dalloc(c, (void**)&c->dt, sizeof(double) * nbox);
    if (e == cudaSuccess) e = dalloc(c, (void**)&c->dtc, sizeof(DtBox) * nbox);
    if (e == cudaSuccess) e = dalloc(c, (void**)&c->smax, sizeof(double) * nbox);
    if (e == cudaSuccess) e = dalloc(c, (void**)&c->smax_part, sizeof(unsigned long long) * nbox);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->smax_part, 0, sizeof(unsigned long long) * nbox, c->stream);
    if (e == cudaSuccess) e = dalloc(c, (void**)&c->bad, sizeof(unsigned long long));
    if (e == cudaSuccess) e = dalloc(c, (void**)&c->nfloor, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->nfloor, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = dalloc(c, (void**)&c->part, (size_t)vb * 10 * sizeof(double));
    if (e == cudaSuccess) e = dalloc(c, (void**)&c->diag, (size_t)nbox * 10 * sizeof(double));
    if (e == cudaSuccess) e = dalloc(c, (void**)&c->dbox, sizeof(BoxDev) * nbox);
    c->B.b = c->dbox;
    if (e == cudaSuccess) e = cudaMemsetAsync(c->bad, 0xff, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = dalloc(c, (void**)&c->perr, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->perr, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dt, 0, sizeof(double) * nbox, c->stream);
    // edge fields by their own kernel with per-thread loads: on the B300 the
    // faster of the three forms (see mhd_set_emf_staging)
    c->emf_stage_req = 0;
    if (e == cudaSuccess) e = layout_tiles(c, 8);   // (counts the launches of the step)
    if (e != cudaSuccess) {
        g_init_err = e == cudaErrorMemoryAllocation ? "device allocation failed" : cudaGetErrorString(e);
        mhd_status s = e == cudaErrorMemoryAllocation ? MHD_ENOMEM : MHD_ECUDA;
        release(c);
        free(c);
        return s;
    }
    *out = c;
    return MHD_OK;
}

extern "C" mhd_status mhd_init(const mhd_grid* grid, double gamma, const mhd_scheme* scheme, void* stream,
                               mhd_ctx** out)
{
    return init_common(1, grid, gamma, scheme, stream, out);
}

extern "C" mhd_status mhd_init_batch(int nbox, const mhd_grid* grids, double gamma, const mhd_scheme* scheme,
                                     void* stream, mhd_ctx** out)
{
    return init_common(nbox, grids, gamma, scheme, stream, out);
}

extern "C" int mhd_nbox(mhd_ctx* c) { return c ? c->nbox : 0; }

static mhd_status check_device_flags(mhd_ctx* c)
{
    unsigned long long bad = ~0ull;
    unsigned perr = 0;
    CK(cudaMemcpyAsync(&bad, c->bad, sizeof(bad), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&perr, c->perr, sizeof(perr), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (perr) return fail(c, MHD_ETIMEOUT, "a staged-plane wait of the edge-field kernel gave up (flags %u)", perr);
    if (bad != ~0ull) return fail(c, MHD_ENEGATIVE, "rho <= 0 or P <= 0 in cell %llu", bad);
    return c->sticky;
}

extern "C" mhd_status mhd_set_state_box(mhd_ctx* c, int box, const void* U, const void* B, int on_device)
{
    if (!c || !U || !B || box < 0 || box >= c->nbox) return fail(c, MHD_EINVAL, "bad arguments");
    const long long n = c->hbox[box].n, off = c->hbox[box].off, N = c->B.N;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (c->sch.precision != MHD_MIXED) {
        const size_t sz = c->szu;  // == sze for the uniform layouts
        const char* u = (const char*)U;
        const char* b = (const char*)B;
        char* dst[5] = {(char*)c->rho, (char*)c->m[0], (char*)c->m[1], (char*)c->m[2], (char*)c->e};
        for (int f = 0; f < 5; f++) CK(cudaMemcpyAsync(dst[f] + off * sz, u + f * n * sz, n * sz, k, c->stream));
        for (int d = 0; d < 3; d++) CK(cudaMemcpyAsync((char*)c->b[d] + off * sz, b + d * n * sz, n * sz, k, c->stream));
    } else {
        const double* u = (const double*)U;
        const double* b = (const double*)B;
        double* stg = (double*)c->stage;
        for (int f = 0; f < 4; f++) CK(cudaMemcpyAsync(stg + f * N + off, u + f * n, n * sizeof(double), k, c->stream));
        CK(cudaMemcpyAsync((double*)c->e + off, u + 4 * n, n * sizeof(double), k, c->stream));
        for (int d = 0; d < 3; d++) CK(cudaMemcpyAsync((double*)c->b[d] + off, b + d * n, n * sizeof(double), k, c->stream));
        float* dst[4] = {(float*)c->rho, (float*)c->m[0], (float*)c->m[1], (float*)c->m[2]};
        for (int f = 0; f < 4; f++)
            k_convert<float, double><<<1184, 256, 0, c->stream>>>(dst[f] + off, stg + f * N + off, n);
        CK(cudaGetLastError());
    }
    if (c->fix_nl[0] | c->fix_nl[1] | c->fix_nl[2]) {   // the ghost layers hold their fixed states
        apply_fixed_layers(c);
        CK(cudaGetLastError());
    }
    if (!on_device) CK(cudaStreamSynchronize(c->stream));
    return MHD_OK;
}

extern "C" mhd_status mhd_get_state_box(mhd_ctx* c, int box, void* U, void* B, int on_device)
{
    if (!c || !U || !B || box < 0 || box >= c->nbox) return fail(c, MHD_EINVAL, "bad arguments");
    const long long n = c->hbox[box].n, off = c->hbox[box].off, N = c->B.N;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (c->sch.precision != MHD_MIXED) {
        const size_t sz = c->szu;
        char* u = (char*)U;
        char* b = (char*)B;
        const char* src[5] = {(const char*)c->rho, (const char*)c->m[0], (const char*)c->m[1], (const char*)c->m[2],
                              (const char*)c->e};
        for (int f = 0; f < 5; f++) CK(cudaMemcpyAsync(u + f * n * sz, src[f] + off * sz, n * sz, k, c->stream));
        for (int d = 0; d < 3; d++) CK(cudaMemcpyAsync(b + d * n * sz, (const char*)c->b[d] + off * sz, n * sz, k, c->stream));
    } else {
        double* u = (double*)U;
        double* b = (double*)B;
        double* stg = (double*)c->stage;
        const float* src[4] = {(const float*)c->rho, (const float*)c->m[0], (const float*)c->m[1], (const float*)c->m[2]};
        for (int f = 0; f < 4; f++)
            k_convert<double, float><<<1184, 256, 0, c->stream>>>(stg + f * N + off, src[f] + off, n);
        CK(cudaGetLastError());
        for (int f = 0; f < 4; f++) CK(cudaMemcpyAsync(u + f * n, stg + f * N + off, n * sizeof(double), k, c->stream));
        CK(cudaMemcpyAsync(u + 4 * n, (const double*)c->e + off, n * sizeof(double), k, c->stream));
        for (int d = 0; d < 3; d++) CK(cudaMemcpyAsync(b + d * n, (const double*)c->b[d] + off, n * sizeof(double), k, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return check_device_flags(c);
}

extern "C" mhd_status mhd_set_state(mhd_ctx* c, const void* U, const void* B, int on_device)
{
    return mhd_set_state_box(c, 0, U, B, on_device);
}

extern "C" mhd_status mhd_get_state(mhd_ctx* c, void* U, void* B, int on_device)
{
    return mhd_get_state_box(c, 0, U, B, on_device);
}

// primitives and per-box signal-speed maxima of the current state (no floor
// raise of e), with the boundary handling the context was set to
template <class R, class TU, class TE>
static void prim_pass(mhd_ctx* c)
{
    const int nb = c->cell_grid;
    if (c->bc)
        k_prim<R, TU, TE, true><<<nb, CELL_THREADS, 0, c->stream>>>(c->B, state_of<TU, TE>(c), (R*)c->W, c->gamma,
                                                                    c->smax_part, c->bad, c->sch.pfloor);
    else
        k_prim<R, TU, TE><<<nb, CELL_THREADS, 0, c->stream>>>(c->B, state_of<TU, TE>(c), (R*)c->W, c->gamma,
                                                              c->smax_part, c->bad, c->sch.pfloor);
}

extern "C" mhd_status mhd_cfl_dt(mhd_ctx* c, double* dt)
{
    if (!c || !dt) return fail(c, MHD_EINVAL, "null pointer");
    switch (c->sch.precision) {
        case MHD_FP64: prim_pass<double, double, double>(c); break;
        case MHD_FP32: prim_pass<float, float, float>(c); break;
        default:       prim_pass<float, float, double>(c); break;
    }
    k_finalize_dt<<<(c->nbox + 127) / 128, 128, 0, c->stream>>>(c->B, c->smax_part, c->sch.cfl, nullptr, c->smax, nullptr);
    CK(cudaGetLastError());
    double* s = (double*)malloc(sizeof(double) * c->nbox);
    if (!s) return fail(c, MHD_ENOMEM, "host allocation failed");
    cudaError_t e = cudaMemcpyAsync(s, c->smax, sizeof(double) * c->nbox, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { free(s); return fail(c, MHD_ECUDA, "cfl readback: %s", cudaGetErrorString(e)); }
    mhd_status st = check_device_flags(c);
    for (int b = 0; b < c->nbox && st == MHD_OK; b++) {
        if (!(s[b] > 0.0)) st = fail(c, MHD_ENEGATIVE, "no positive signal speed in box %d", b);
        else dt[b] = c->sch.cfl * c->hbox[b].dx / s[b];
    }
    free(s);
    return st;
}

extern "C" mhd_status mhd_step(mhd_ctx* c, double dt)
{
    if (!c) return MHD_EINVAL;
    if (!(dt > 0.0) || !(dt < 1e300)) return fail(c, MHD_EINVAL, "dt must be positive and finite");
    k_set_dt<<<1, 256, 0, c->stream>>>(c->B, c->dt, dt, c->dtc);
    c->step(c, false);
    CK(cudaGetLastError());
    return MHD_OK;
}

extern "C" mhd_status mhd_step_boxes(mhd_ctx* c, const double* dt)
{
    if (!c || !dt) return fail(c, MHD_EINVAL, "null pointer");
    for (int b = 0; b < c->nbox; b++)
        if (!(dt[b] > 0.0) || !(dt[b] < 1e300)) return fail(c, MHD_EINVAL, "dt of box %d must be positive and finite", b);
    CK(cudaMemcpyAsync(c->dt, dt, sizeof(double) * c->nbox, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));   // dt is the caller's host array
    k_set_dt<<<1, 256, 0, c->stream>>>(c->B, c->dt, 0.0, c->dtc);
    c->step(c, false);
    CK(cudaGetLastError());
    return MHD_OK;
}

extern "C" mhd_status mhd_advance(mhd_ctx* c, int nsteps, int use_graph)
{
    if (!c || nsteps < 0) return fail(c, MHD_EINVAL, "bad arguments");
    if (!use_graph) {
        for (int s = 0; s < nsteps; s++) c->step(c, true);
        CK(cudaGetLastError());
        return MHD_OK;
    }
    if (!c->have_graph) {
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        c->step(c, true);
        cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        if (e != cudaSuccess) return fail(c, MHD_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&c->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(c, MHD_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        c->have_graph = true;
    }
    for (int s = 0; s < nsteps; s++) CK(cudaGraphLaunch(c->gexec, c->stream));
    return MHD_OK;
}

extern "C" mhd_status mhd_last_dt(mhd_ctx* c, double* dt)
{
    if (!c || !dt) return fail(c, MHD_EINVAL, "null pointer");
    CK(cudaMemcpyAsync(dt, c->dt, sizeof(double) * c->nbox, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MHD_OK;
}

static mhd_status run_diag(mhd_ctx* c, double* out)
{
    const int nb = c->cell_grid;
    switch (c->sch.precision) {
        case MHD_FP64: k_diag<double, double><<<nb, CELL_THREADS, 0, c->stream>>>(c->B, state_of<double, double>(c), c->part); break;
        case MHD_FP32: k_diag<float, float><<<nb, CELL_THREADS, 0, c->stream>>>(c->B, state_of<float, float>(c), c->part); break;
        default:       k_diag<float, double><<<nb, CELL_THREADS, 0, c->stream>>>(c->B, state_of<float, double>(c), c->part); break;
    }
    k_finish_diag<<<c->nbox, 32, 0, c->stream>>>(c->B, c->part, c->diag);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, c->diag, (size_t)c->nbox * 10 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return check_device_flags(c);
}

extern "C" mhd_status mhd_divB(mhd_ctx* c, double* maxabs, double* brms)
{
    if (!c || !maxabs || !brms) return fail(c, MHD_EINVAL, "null pointer");
    double* d = (double*)malloc(sizeof(double) * 10 * c->nbox);
    if (!d) return fail(c, MHD_ENOMEM, "host allocation failed");
    mhd_status s = run_diag(c, d);
    for (int b = 0; b < c->nbox; b++) {
        maxabs[b] = d[b * 10];
        brms[b] = sqrt(d[b * 10 + 1] / (double)c->hbox[b].n);
    }
    free(d);
    return s;
}

extern "C" mhd_status mhd_sums(mhd_ctx* c, double* sums8)
{
    if (!c || !sums8) return fail(c, MHD_EINVAL, "null pointer");
    double* d = (double*)malloc(sizeof(double) * 10 * c->nbox);
    if (!d) return fail(c, MHD_ENOMEM, "host allocation failed");
    mhd_status s = run_diag(c, d);
    for (int b = 0; b < c->nbox; b++)
        for (int f = 0; f < 8; f++) sums8[b * 8 + f] = d[b * 10 + 2 + f];
    free(d);
    return s;
}

extern "C" mhd_status mhd_energies(mhd_ctx* c, double jb_threshold, double* out)
{
    if (!c || !out) return fail(c, MHD_EINVAL, "null pointer");
    if (!(jb_threshold >= 0.0)) return fail(c, MHD_EINVAL, "jb_threshold must be >= 0");
    const int nb = c->cell_grid;
    switch (c->sch.precision) {
        case MHD_FP64: k_energies<double, double><<<nb, CELL_THREADS, 0, c->stream>>>(c->B, state_of<double, double>(c), jb_threshold, c->part); break;
        case MHD_FP32: k_energies<float, float><<<nb, CELL_THREADS, 0, c->stream>>>(c->B, state_of<float, float>(c), jb_threshold, c->part); break;
        default:       k_energies<float, double><<<nb, CELL_THREADS, 0, c->stream>>>(c->B, state_of<float, double>(c), jb_threshold, c->part); break;
    }
    k_finish_parts<<<c->nbox, 32, 0, c->stream>>>(c->B, c->part, 6, 0x28u, c->diag);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, c->diag, (size_t)c->nbox * 6 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int b = 0; b < c->nbox; b++) {
        const double dx = c->hbox[b].dx, v = dx * dx * dx;
        out[b * 6 + 0] *= v;
        out[b * 6 + 1] *= v;
        out[b * 6 + 2] *= v;
        out[b * 6 + 5] /= dx;
    }
    return check_device_flags(c);
}

template <class TU, class TE>
static void pressure_pass(mhd_ctx* c, double* P)
{
    if (c->bc) k_pressure<TU, TE, true><<<c->cell_grid, CELL_THREADS, 0, c->stream>>>(c->B, state_of<TU, TE>(c), c->gamma, P);
    else k_pressure<TU, TE, false><<<c->cell_grid, CELL_THREADS, 0, c->stream>>>(c->B, state_of<TU, TE>(c), c->gamma, P);
}

extern "C" mhd_status mhd_pressure_gradient(mhd_ctx* c, double scale, double thr, int nlev, double* out)
{
    if (!c || !out) return fail(c, MHD_EINVAL, "null pointer");
    if (!(scale > 0.0) || !(thr >= 0.0) || nlev < 1 || nlev > 4)
        return fail(c, MHD_EINVAL, "mhd_pressure_gradient: scale > 0, thr >= 0 and 1 <= nlev <= 4 required");
    // the cell pressures (FP64) go to the primitive scratch, which every step
    // and every CFL pass rewrite before reading
    double* P = (double*)c->W;
    switch (c->sch.precision) {
        case MHD_FP64: pressure_pass<double, double>(c, P); break;
        case MHD_FP32: pressure_pass<float, float>(c, P); break;
        default:       pressure_pass<float, double>(c, P); break;
    }
    if (c->bc) k_pgrad<true><<<c->cell_grid, CELL_THREADS, 0, c->stream>>>(c->B, P, scale, thr, nlev, c->part);
    else k_pgrad<false><<<c->cell_grid, CELL_THREADS, 0, c->stream>>>(c->B, P, scale, thr, nlev, c->part);
    k_finish_parts<<<c->nbox, 32, 0, c->stream>>>(c->B, c->part, 5, 0x1u, c->diag);
    CK(cudaGetLastError());
    double d[5];
    for (int b = 0; b < c->nbox; b++) {
        CK(cudaMemcpyAsync(d, c->diag + (size_t)b * 5, sizeof(d), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (int f = 0; f <= nlev; f++) out[(size_t)b * (nlev + 1) + f] = d[f];
    }
    return check_device_flags(c);
}

extern "C" mhd_status mhd_helicity(mhd_ctx* c, double* h)
{
    if (!c || !h) return fail(c, MHD_EINVAL, "null pointer");
    if (c->bc) return fail(c, MHD_EUNSUPPORTED, "mhd_helicity: the Coulomb gauge needs a periodic box");
    const size_t rsz = c->sch.precision == MHD_FP64 ? sizeof(double) : sizeof(float);
    const size_t f1_bytes = (size_t)21 * (size_t)c->B.N * rsz;
    const int nblk = (int)(c->B.nvblk * 10 < 1024 ? c->B.nvblk * 10 : 1024);   // c->part holds nvblk * 10
    double parts[1024];
    for (int b = 0; b < c->nbox; b++) {
        const BoxDev& g = c->hbox[b];
        const long long n = g.n;
        const long long m = (long long)g.nz * g.ny * (g.nx / 2 + 1);
        const size_t in_bytes = ((size_t)3 * n * sizeof(double) + 255) / 256 * 256;
        if (in_bytes + (size_t)3 * m * sizeof(double2) > f1_bytes)
            return fail(c, MHD_ENOMEM, "mhd_helicity: box %d does not fit the flux scratch", b);
        double* in = (double*)c->F1;
        double2* out = (double2*)((char*)c->F1 + in_bytes);
        switch (c->sch.precision) {
            case MHD_FP32: k_bcc<float><<<256, 256, 0, c->stream>>>(g, (float*)c->b[0], (float*)c->b[1], (float*)c->b[2], in); break;
            default:       k_bcc<double><<<256, 256, 0, c->stream>>>(g, (double*)c->b[0], (double*)c->b[1], (double*)c->b[2], in); break;
        }
        CK(cudaGetLastError());
        cufftHandle plan;
        int dims[3] = {g.nz, g.ny, g.nx};
        if (cufftPlanMany(&plan, 3, dims, nullptr, 1, (int)n, nullptr, 1, (int)m, CUFFT_D2Z, 3) != CUFFT_SUCCESS)
            return fail(c, MHD_ECUDA, "mhd_helicity: cuFFT plan failed for box %d", b);
        cufftResult fr = cufftSetStream(plan, c->stream);
        if (fr == CUFFT_SUCCESS) fr = cufftExecD2Z(plan, in, (cufftDoubleComplex*)out);
        if (fr != CUFFT_SUCCESS) {
            cufftDestroy(plan);
            return fail(c, MHD_ECUDA, "mhd_helicity: cuFFT transform failed for box %d", b);
        }
        k_helicity_part<<<nblk, 256, 0, c->stream>>>(g.nx, g.ny, g.nz, g.dx, out, c->part);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(parts, c->part, nblk * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cufftDestroy(plan);
        if (e != cudaSuccess) return fail(c, MHD_ECUDA, "mhd_helicity: %s", cudaGetErrorString(e));
        double s = 0.0;
        for (int q = 0; q < nblk; q++) s += parts[q];
        h[b] = s * g.dx * g.dx * g.dx / (double)n;
    }
    return check_device_flags(c);
}

extern "C" mhd_status mhd_sync(mhd_ctx* c)
{
    if (!c) return MHD_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaGetLastError());
    return check_device_flags(c);
}

extern "C" mhd_status mhd_set_sweep_config(mhd_ctx* c, int tile_len, int blocks_per_sm)
{
    if (!c) return MHD_EINVAL;
    if (!(tile_len == 4 || tile_len == 8 || tile_len == 16) || blocks_per_sm < 1 || blocks_per_sm > 64)
        return fail(c, MHD_EINVAL, "tile_len must be 4, 8 or 16 and blocks_per_sm in [1, 64]");
    c->sweep_bps = blocks_per_sm;
    CK(layout_tiles(c, tile_len));
    return MHD_OK;
}

extern "C" mhd_status mhd_get_sweep_config(mhd_ctx* c, int* tile_len, int* blocks_per_sm)
{
    if (!c || !tile_len || !blocks_per_sm) return fail(c, MHD_EINVAL, "null pointer");
    *tile_len = c->B.tl;
    *blocks_per_sm = c->sweep_bps;
    return MHD_OK;
}

// kernels per step of a one-box context: the scheme's 12 (8 with the fused
// VL predictor: prim, dt, predictor, 3 sweeps, emf, full; one fewer per
// edge-field kernel fused with its update), an outer-face flux pass per
// outflow axis and stage, a layer reset per Dirichlet axis.  With a learned
// selector: the scheme's 12, the features, the network, the three lists and
// the other path's six sweeps.
static void count_launches(mhd_ctx* c)
{
    if (c->sel) {
        c->launches = 12 + 3 + 3 + 6 - (emf_form(c) == 2 ? 2 : 0) - (sel_y_half(c) ? 1 : 0);
        return;
    }
    // (CTU: one stage-1 outer-face pass per outflow axis; the stage-2 ones
    // are part of the corrections)
    // (the y corrector takes the half update, the y predictor the primitives)
    int n = fused_predictor(c) ? 8 : 12 - (y_half(c) || ctu_y_half(c) ? 1 : 0) - (y_prim(c) ? 1 : 0);
    if (emf_form(c) == 2) n -= fused_predictor(c) ? 1 : 2;   // each edge-field kernel takes its update
    const int per_axis = c->sch.integrator == MHD_VL ? 2 : 1;
    for (int d = 0; d < 3; d++) n += per_axis * (c->bc >> d & 1) + (c->fix_nl[d] > 0);
    c->launches = n;
}

void mhd_internal_count_launches(mhd_ctx* c) { count_launches(c); }

static void apply_fixed_layers(mhd_ctx* c)
{
    switch (c->sch.precision) {
        case MHD_FP64: fix_layers<double, double>(c, state_of<double, double>(c), c->stream); break;
        case MHD_FP32: fix_layers<float, float>(c, state_of<float, float>(c), c->stream); break;
        default:       fix_layers<float, double>(c, state_of<float, double>(c), c->stream); break;
    }
}

extern "C" mhd_status mhd_set_boundary(mhd_ctx* c, int outflow_mask)
{
    if (!c) return MHD_EINVAL;
    if (outflow_mask < 0 || outflow_mask > 7) return fail(c, MHD_EINVAL, "outflow_mask must be in [0, 7]");
    if (outflow_mask && (c->nbox != 1 || c->sel))
        return fail(c, MHD_EUNSUPPORTED, "outflow boundaries are built for one-box contexts without a selector");
    if (outflow_mask && !c->fout) {
        // two stages of outer-face fluxes (CTU keeps the first while the
        // corrections write the second; VL uses the first half only)
        const BoxDev& b = c->hbox[0];
        CK(dalloc(c, &c->fout, (size_t)2 * 3 * 7 * cross_size(b.nx, b.ny, b.nz) * c->szr));
    }
    c->bc = outflow_mask;
    c->hbox[0].bc = outflow_mask;
    for (int d = 0; d < 3; d++)
        if (!(outflow_mask >> d & 1)) c->fix_nl[d] = 0;   // a Dirichlet side needs the clamp beyond it
    count_launches(c);
    CK(layout_tiles(c, c->B.tl));   // uploads the box table (and drops a captured step)
    return MHD_OK;
}

extern "C" mhd_status mhd_set_dirichlet(mhd_ctx* c, int axis, int nlayers, const double* w_lo, const double* w_hi)
{
    if (!c) return MHD_EINVAL;
    if (axis < 0 || axis > 2) return fail(c, MHD_EINVAL, "axis must be 0, 1 or 2");
    if (nlayers == 0) {
        c->fix_nl[axis] = 0;
        count_launches(c);
        CK(layout_tiles(c, c->B.tl));
        return MHD_OK;
    }
    if (!w_lo || !w_hi) return fail(c, MHD_EINVAL, "null pointer");
    if (c->nbox != 1 || c->sel)
        return fail(c, MHD_EUNSUPPORTED, "Dirichlet sides are built for one-box contexts without a selector");
    // layers the interior needs to see an unbounded fixed region: VL's
    // half-step PPM reads one cell further
    const int need = c->sch.integrator == MHD_VL && c->sch.recon == MHD_PPM ? 3 : 2;
    const BoxDev& g = c->hbox[0];
    const int nd = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
    if (nlayers < need || 2 * nlayers + 1 > nd)
        return fail(c, MHD_EINVAL, "nlayers must be >= %d for this reconstruction and leave an interior (2 nlayers < %d)",
                    need, nd);
    const double* w[2] = {w_lo, w_hi};
    FixedState f[2];
    for (int side = 0; side < 2; side++) {
        const double* q = w[side];
        for (int m = 0; m < 8; m++)
            if (!std::isfinite(q[m])) return fail(c, MHD_EINVAL, "non-finite Dirichlet state");
        if (!(q[0] > 0.0) || !(q[4] > 0.0)) return fail(c, MHD_EINVAL, "Dirichlet state needs rho > 0 and P > 0");
        f[side].u[0] = q[0];
        f[side].u[1] = q[0] * q[1];
        f[side].u[2] = q[0] * q[2];
        f[side].u[3] = q[0] * q[3];
        f[side].u[4] = q[4] / (c->gamma - 1.0) + 0.5 * q[0] * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3])
                     + 0.5 * (q[5] * q[5] + q[6] * q[6] + q[7] * q[7]);
        for (int m = 0; m < 3; m++) f[side].b[m] = q[5 + m];
    }
    if (!(c->bc >> axis & 1)) {
        mhd_status st = mhd_set_boundary(c, c->bc | (1 << axis));
        if (st != MHD_OK) return st;
    }
    c->fix[axis][0] = f[0];
    c->fix[axis][1] = f[1];
    c->fix_nl[axis] = nlayers;
    count_launches(c);
    CK(layout_tiles(c, c->B.tl));   // drops a captured step
    apply_fixed_layers(c);
    CK(cudaGetLastError());
    return MHD_OK;
}

extern "C" mhd_status mhd_get_dirichlet(mhd_ctx* c, int axis, int* nlayers)
{
    if (!c || !nlayers || axis < 0 || axis > 2) return fail(c, MHD_EINVAL, "bad arguments");
    *nlayers = c->fix_nl[axis];
    return MHD_OK;
}

extern "C" mhd_status mhd_get_boundary(mhd_ctx* c, int* outflow_mask)
{
    if (!c || !outflow_mask) return fail(c, MHD_EINVAL, "null pointer");
    *outflow_mask = c->bc;
    return MHD_OK;
}

extern "C" mhd_status mhd_set_sweep_pencils(mhd_ctx* c, int pencil_mask, int pencil_len)
{
    if (!c) return MHD_EINVAL;
    if (pencil_mask < 0 || pencil_mask > 1023 || pencil_len < 1 || pencil_len > 1024)
        return fail(c, MHD_EINVAL, "pencil_mask must be in [0, 1023] and pencil_len in [1, 1024]");
    if ((pencil_mask & 128) && ensure_f2(c) != cudaSuccess)
        return fail(c, MHD_ENOMEM, "second flux array for the fused y corrector");
    c->pencil_mask = pencil_mask;
    c->pencil_len = pencil_len;
    CK(layout_tiles(c, c->B.tl));
    if (c->sel && mhd_internal_selector_lists(c) != MHD_OK) return fail(c, MHD_ENOMEM, "selector lists");
    return MHD_OK;
}

extern "C" mhd_status mhd_get_sweep_pencils(mhd_ctx* c, int* pencil_mask, int* pencil_len)
{
    if (!c || !pencil_mask || !pencil_len) return fail(c, MHD_EINVAL, "null pointer");
    *pencil_mask = c->pencil_mask;
    *pencil_len = c->pencil_len;
    return MHD_OK;
}

extern "C" mhd_status mhd_set_emf_staging(mhd_ctx* c, int mode)
{
    if (!c) return MHD_EINVAL;
    if (mode < 0 || mode > 2) return fail(c, MHD_EINVAL, "mode must be 0, 1 or 2");
    const int was = emf_form(c);
    c->emf_stage_req = mode;
    setup_emf_tma(c);
    if (emf_form(c) != was && c->have_graph) {   // a captured step holds the other kernels
        cudaGraphExecDestroy(c->gexec);
        c->have_graph = false;
    }
    count_launches(c);
    return MHD_OK;
}

extern "C" mhd_status mhd_get_emf_staging(mhd_ctx* c, int* mode, int* active)
{
    if (!c || !mode || !active) return fail(c, MHD_EINVAL, "null pointer");
    *mode = c->emf_stage_req;
    *active = emf_form(c);
    return MHD_OK;
}

// time `reps` directly launched steps of the current configuration
static mhd_status time_steps(mhd_ctx* c, int reps, float* ms)
{
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    CK(cudaEventRecord(a, c->stream));
    for (int r = 0; r < reps; r++) c->step(c, true);
    CK(cudaEventRecord(b, c->stream));
    CK(cudaEventSynchronize(b));
    CK(cudaEventElapsedTime(ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    CK(cudaGetLastError());
    return MHD_OK;
}

// Try every (tile length, blocks per SM) pair on the context's own batch;
// the state is copied aside first and restored after every trial.
extern "C" mhd_status mhd_autotune(mhd_ctx* c, int reps, int* tile_len, int* blocks_per_sm, double* ms_best)
{
    if (!c || reps < 1) return fail(c, MHD_EINVAL, "bad arguments");
    const long long N = c->B.N;
    void* saved = nullptr;
    const size_t ub = 4 * N * c->szu, eb = 4 * N * c->sze;
    CK(cudaMalloc(&saved, ub + eb));
    char* sv = (char*)saved;
    void* fu[4] = {c->rho, c->m[0], c->m[1], c->m[2]};
    void* fe[4] = {c->e, c->b[0], c->b[1], c->b[2]};
    cudaError_t e = cudaSuccess;
    for (int f = 0; f < 4 && e == cudaSuccess; f++)
        e = cudaMemcpyAsync(sv + f * N * c->szu, fu[f], N * c->szu, cudaMemcpyDeviceToDevice, c->stream);
    for (int f = 0; f < 4 && e == cudaSuccess; f++)
        e = cudaMemcpyAsync(sv + ub + f * N * c->sze, fe[f], N * c->sze, cudaMemcpyDeviceToDevice, c->stream);
    const int tls[3] = {4, 8, 16};
    const int bpss[4] = {1, 2, 4, 8};
    float best = 1e30f;
    int btl = c->B.tl, bbps = c->sweep_bps, bmask = 0, blen = c->pencil_len;
    mhd_status st = e == cudaSuccess ? MHD_OK : fail(c, MHD_ECUDA, "autotune copy: %s", cudaGetErrorString(e));
    // one trial: warm-up step, `reps` timed steps, state restored
    auto trial = [&](float* ms) -> mhd_status {
        mhd_status s2 = time_steps(c, 1, ms);
        if (s2 == MHD_OK) s2 = time_steps(c, reps, ms);
        for (int f = 0; f < 4; f++)
            cudaMemcpyAsync(fu[f], sv + f * N * c->szu, N * c->szu, cudaMemcpyDeviceToDevice, c->stream);
        for (int f = 0; f < 4; f++)
            cudaMemcpyAsync(fe[f], sv + ub + f * N * c->sze, N * c->sze, cudaMemcpyDeviceToDevice, c->stream);
        return s2;
    };
    // tiles on every axis: (tile length, blocks per SM)
    c->pencil_mask = 0;
    for (int i = 0; i < 3 && st == MHD_OK; i++)
        for (int j = 0; j < 4 && st == MHD_OK; j++) {
            c->sweep_bps = bpss[j];
            if (layout_tiles(c, tls[i]) != cudaSuccess) { st = fail(c, MHD_ECUDA, "autotune layout"); break; }
            float ms = 0.0f;
            st = trial(&ms);
            if (st == MHD_OK && ms < best) { best = ms; btl = tls[i]; bbps = bpss[j]; }
        }
    // pencils on all axes or on y and z only (x keeps the best tiles), per
    // segment length (VL: x by warps; CTU: x by pencil threads)
    {
        // (VL without a selector: also with x by staged pencils, bit 4, by
        // aligned marching warps, bits 5 and 6, and for periodic boxes with
        // the fused predictor, bit 3)
        // (CTU: also with the x tracing by aligned marching warps, bit 5)
        // (VL, periodic, no selector: also with the primitives inside the y
        // predictor pencils, bit 8, with the half update inside the y
        // corrector pencils, bit 7, when its flux array can be had, and for
        // PLM with the conservative update inside the z corrector, bit 9)
        int vl_masks[12] = {7, 6, 23, 103, 15, 31, 111, 359, 0, 0, 0, 0};
        // (167: bit 7, the dt/2 update in the y correction; 679: and bit 9, the
        // conservative update in the z correction)
        const int ctu_masks[5] = {7, 6, 39, 167, 679};
        const bool ctu = c->sch.integrator != MHD_VL;
        const int* masks = ctu ? ctu_masks : vl_masks;
        const int lens[3] = {8, 16, 32};
        int nvl = 8;
        if (!c->sel && !c->bc && ensure_f2(c) == cudaSuccess) {
            if (c->sch.recon != MHD_PPM) {
                vl_masks[7] = 151;
                vl_masks[8] = 231;
                vl_masks[9] = 487;
                vl_masks[10] = 743;        // (bit 9: the conservative update in the z corrector)
                vl_masks[11] = 999;
                nvl = 12;
            } else {
                vl_masks[8] = 231;
                vl_masks[9] = 487;
                vl_masks[10] = 743;
                vl_masks[11] = 999;
                nvl = 12;
            }
        }
        const int nmask = ctu ? (!c->bc ? 5 : 3) : (c->sel ? 2 : (!c->bc ? nvl : 4));
        c->sweep_bps = bbps;
        for (int i = 0; i < nmask && st == MHD_OK; i++)
            for (int j = 0; j < 3 && st == MHD_OK; j++) {
                c->pencil_mask = masks[i];
                c->pencil_len = lens[j];
                if (layout_tiles(c, btl) != cudaSuccess) { st = fail(c, MHD_ECUDA, "autotune layout"); break; }
                if (c->sel && mhd_internal_selector_lists(c) != MHD_OK) { st = fail(c, MHD_ENOMEM, "selector lists"); break; }
                float ms = 0.0f;
                st = trial(&ms);
                if (st == MHD_OK && ms < best) { best = ms; bmask = masks[i]; blen = lens[j]; }
            }
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(saved);
    if (st != MHD_OK) return st;
    c->sweep_bps = bbps;
    c->pencil_mask = bmask;
    c->pencil_len = blen;
    CK(layout_tiles(c, btl));
    if (tile_len) *tile_len = btl;
    if (blocks_per_sm) *blocks_per_sm = bbps;
    if (ms_best) *ms_best = best / reps;
    return MHD_OK;
}

extern "C" mhd_status mhd_profile_begin(mhd_ctx* c, int max_steps)
{
    if (!c || max_steps < 1 || max_steps > 100000) return fail(c, MHD_EINVAL, "bad arguments");
    if (c->prof_ev) {
        for (int q = 0; q < c->prof_cap * (MHD_NGROUPS + 1); q++) cudaEventDestroy(c->prof_ev[q]);
        free(c->prof_ev);
        c->prof_ev = nullptr;
    }
    int ne = max_steps * (MHD_NGROUPS + 1);
    c->prof_ev = (cudaEvent_t*)calloc((size_t)ne, sizeof(cudaEvent_t));
    if (!c->prof_ev) return fail(c, MHD_ENOMEM, "host allocation failed");
    c->prof_cap = max_steps;
    for (int q = 0; q < ne; q++) CK(cudaEventCreate(&c->prof_ev[q]));
    c->prof_steps = 0;
    c->prof_on = true;
    return MHD_OK;
}

extern "C" mhd_status mhd_profile_end(mhd_ctx* c, double* ms, int ngroups, int* steps)
{
    if (!c || !ms || ngroups < 1) return fail(c, MHD_EINVAL, "bad arguments");
    c->prof_on = false;
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < ngroups; k++) ms[k] = 0.0;
    for (int st = 0; st < c->prof_steps; st++) {
        cudaEvent_t* e = c->prof_ev + st * (MHD_NGROUPS + 1);
        for (int k = 0; k < ngroups && k < MHD_NGROUPS; k++) {
            float t = 0.0f;
            CK(cudaEventElapsedTime(&t, e[k], e[k + 1]));
            ms[k] += t;
        }
    }
    if (steps) *steps = c->prof_steps;
    return MHD_OK;
}

extern "C" long long mhd_floor_count(mhd_ctx* c)
{
    if (!c) return -1;
    unsigned long long v = 0;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return -1;
    if (cudaMemcpy(&v, c->nfloor, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    return (long long)v;
}

extern "C" long long mhd_bad_cell(mhd_ctx* c)
{
    if (!c) return -1;
    unsigned long long bad = ~0ull;
    if (cudaMemcpy(&bad, c->bad, sizeof(bad), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    return bad == ~0ull ? -1 : (long long)bad;
}

extern "C" void mhd_clear_error(mhd_ctx* c)
{
    if (!c) return;
    cudaMemsetAsync(c->bad, 0xff, sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(c->perr, 0, sizeof(unsigned), c->stream);
    cudaStreamSynchronize(c->stream);
    c->sticky = MHD_OK;
    strcpy(c->err, "no error");
}

extern "C" mhd_status mhd_inject_wait_flag(mhd_ctx* c, unsigned bits)
{
    if (!c || bits == 0u || bits > 3u) return fail(c, MHD_EINVAL, "bits must be 1, 2 or 3");
    // the word a kernel's bounded wait sets when it gives up, written from the
    // host: the error path is exercised without making any device wait fail
    CK(cudaMemcpyAsync(c->perr, &bits, sizeof(bits), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MHD_OK;
}

extern "C" const char* mhd_last_error(mhd_ctx* c) { return c ? c->err : g_init_err; }

extern "C" long long mhd_device_bytes(mhd_ctx* c) { return c ? c->bytes : 0; }

extern "C" int mhd_launches_per_step(mhd_ctx* c) { return c ? c->launches : 0; }

extern "C" void mhd_free(mhd_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    release(c);
    free(c);
}
