// mhd_noalloc.cu -- one FP64 VL step for callers that cannot allocate.
//
// Some callers may not call cudaMalloc at all: a plug-in running inside a
// host application whose allocator owns every byte of device memory, or a
// latency-critical loop that cannot afford the device-wide synchronisation
// cudaMalloc/cudaFree can imply.  mhd_step_noalloc serves them.  It runs the
// same kernels as mhd_step, but its scratch (primitives, fluxes, edge fields,
// half-step faces, dt and a flag word) lives in the file-scope array below,
// of fixed size.  The caller still owns and passes the state.
#include <mutex>
#include <stdio.h>
#include <string.h>
#include "mhd_engine.cuh"

using namespace mhd;

void mhd_internal_set_init_error(const char* msg);   // defined with the other entry points

// per cell: W (8) + Wh (8) + fluxes (21) + edge E (3) + half-step faces (3);
// then dt, the CFL word, the flag word, the floor count and the one-entry
// box table
static constexpr size_t kDoublesPerCell = 43;
static constexpr size_t kScratchBytes = kDoublesPerCell * MHD_NOALLOC_MAX_CELLS * sizeof(double) + 1024;
static_assert(sizeof(mhd::BoxDev) <= 256 && sizeof(mhd::DtBox) <= 256, "tables must fit the slack");

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host code cannot use g_noalloc_scratch as an address (on the host it is a
// stand-in symbol); its device address is looked up once per device.
static constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;

static void* scratch_address(int dev, cudaError_t* err)
{
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // the current device is `dev`
        if (*err != cudaSuccess) return nullptr;
        g_scratch_addr[dev] = p;
    }
    *err = cudaSuccess;
    return g_scratch_addr[dev];
}

// Writes this call's box table, dt and its ratios, and resets the flag word
// and the floor count: everything the array must hold before the step, set
// from kernel arguments, so no host buffer is read after the call returns.
static __global__ void k_noalloc_setup(BoxDev hb, BoxDev* dbox, double* dt, double v, DtBox* dtb,
                                       unsigned long long* bad, unsigned long long* nfloor)
{
    if (threadIdx.x != 0) return;
    *dbox = hb;
    dt[0] = v;
    write_dtbox(dtb, v, hb.dx);
    *bad = ~0ULL;       // no anomaly recorded
    *nfloor = 0ULL;
}

static mhd_status reject(mhd_status s, const char* msg)
{
    mhd_internal_set_init_error(msg);
    return s;
}

extern "C" mhd_status mhd_step_noalloc(const mhd_grid* grid, double gamma, const mhd_scheme* scheme, double dt,
                                       void* U, void* B, void* stream)
{
    if (!grid || !scheme || !U || !B) return reject(MHD_EINVAL, "mhd_step_noalloc: null argument");
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->dx > 0.0))
        return reject(MHD_EINVAL, "mhd_step_noalloc: bad grid");
    // bound each side before forming the product, so that it cannot wrap
    const long long lim = MHD_NOALLOC_MAX_CELLS;
    if (grid->nx > lim || grid->ny > lim / grid->nx || grid->nz > lim / ((long long)grid->nx * grid->ny)) {
        static char msg[200];
        snprintf(msg, sizeof(msg), "mhd_step_noalloc: %d x %d x %d cells exceed the fixed scratch of %d cells",
                 grid->nx, grid->ny, grid->nz, MHD_NOALLOC_MAX_CELLS);
        return reject(MHD_EINVAL, msg);
    }
    const long long n = (long long)grid->nx * grid->ny * grid->nz;
    if (!(gamma > 1.0)) return reject(MHD_EINVAL, "mhd_step_noalloc: gamma must exceed 1");
    if (!(dt > 0.0) || !(dt < 1e300)) return reject(MHD_EINVAL, "mhd_step_noalloc: dt must be positive and finite");
    if (scheme->integrator != MHD_VL || scheme->precision != MHD_FP64)
        return reject(MHD_EUNSUPPORTED, "mhd_step_noalloc: only the FP64 VL scheme is built");
    if (scheme->recon < 0 || scheme->recon > 2 || scheme->riemann < 0 || scheme->riemann > 2)
        return reject(MHD_EINVAL, "mhd_step_noalloc: bad scheme enum");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return reject(MHD_ECUDA, "mhd_step_noalloc: no usable current device");
    cudaError_t e = cudaSuccess;
    unsigned char* base = (unsigned char*)scratch_address(dev, &e);
    if (!base) return reject(MHD_ECUDA, "mhd_step_noalloc: cudaGetSymbolAddress failed");

    // a context on the stack: the caller's state, scratch carved from the array
    mhd_ctx c;
    memset(&c, 0, sizeof(c));
    c.grid = *grid;
    c.sch = *scheme;
    c.gamma = gamma;
    c.stream = (cudaStream_t)stream;
    c.nbox = 1;
    c.szu = c.sze = c.szr = sizeof(double);
    double* u = (double*)U;
    double* b = (double*)B;
    c.rho = u;
    for (int d = 0; d < 3; d++) c.m[d] = u + (1 + d) * n;
    c.e = u + 4 * n;
    for (int d = 0; d < 3; d++) c.b[d] = b + d * n;
    double* s = (double*)base;
    c.W = s;
    c.Wh = s + 8 * n;
    c.F1 = s + 16 * n;
    c.E = s + 37 * n;
    for (int d = 0; d < 3; d++) c.Bh[d] = s + (40 + d) * n;
    c.dt = s + 43 * n;
    c.smax = nullptr;          // steps with the caller's dt: no CFL reduction
    c.smax_part = nullptr;
    c.bad = (unsigned long long*)(s + 43 * n + 2);
    c.nfloor = (unsigned long long*)(s + 43 * n + 3);   // pfloor > 0 raises e as mhd_step does
    // the one-entry box table lives in the array too, 64-byte aligned
    size_t tab = ((43 * (size_t)n + 4) * sizeof(double) + 63) / 64 * 64;
    BoxDev* dbox = (BoxDev*)(base + tab);
    c.dtc = (DtBox*)(base + tab + 256);
    BoxDev hb;
    memset(&hb, 0, sizeof(hb));
    hb.nx = grid->nx; hb.ny = grid->ny; hb.nz = grid->nz;
    hb.n = n;
    hb.dx = grid->dx;
    hb.inv_dx = (float)(1.0 / grid->dx);
    const int tl = 8;
    hb.tile0[0] = hb.tile0[1] = hb.tile0[2] = 0;
    hb.etile0 = 0;
    c.B.b = dbox;
    c.B.nbox = 1;
    c.B.tl = tl;
    c.B.N = n;
    c.B.nvblk = (n + CELL_THREADS - 1) / CELL_THREADS;
    hb.quad = 0;                       // the caller's arrays: one cell per thread in the x-quad kernels
    hb.vq0 = 0;
    c.B.nvq = c.B.nvblk;
    for (int d = 0; d < 3; d++) c.B.ntile[d] = tiles_of_box(hb.nx, hb.ny, hb.nz, d, tl);
    c.B.netile = emf_tiles_of_box(hb.nx, hb.ny, hb.nz);
    c.pencil_mask = 0;                 // tile sweeps only
    c.pencil_len = 16;
    c.B.pl = 16;
    for (int d = 0; d < 3; d++) {
        hb.pth0[d] = 0;
        c.B.npth[d] = pencil_threads_of_box(hb.nx, hb.ny, hb.nz, d, 16);
        hb.xw0[d] = 0;
        c.B.nxw[d] = xwarp_items_of_box(hb.nx, hb.ny, hb.nz, d);
    }
    hb.xr0 = 0;
    c.B.nxr = (long long)hb.ny * hb.nz;
    hb.ftile0 = 0;                     // (the fused predictor and the x pencils are off: mask 0)
    hb.xp0 = 0;
    c.B.nxp = xpencil_threads_of_box(hb.nx, hb.ny, hb.nz, 16);
    c.B.nftile = pred_tiles_of_box(hb.nx, hb.ny, hb.nz, PRED_FZ);
    c.B.fz = PRED_FZ;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return reject(MHD_ECUDA, "mhd_step_noalloc: device query failed");
    c.nsm = nsm;
    c.sweep_bps = 4;
    c.cell_grid = (int)(c.B.nvblk < 16LL * nsm ? c.B.nvblk : 16LL * nsm);
    c.quad_grid = c.cell_grid;
    cudaError_t attr = cudaSuccess;
    c.step = mhd_pick_fp64(scheme->integrator, scheme->recon, scheme->riemann, &attr);
    if (!c.step || attr != cudaSuccess) return reject(MHD_ECUDA, "mhd_step_noalloc: kernel set-up failed");
    // the array keeps the previous call's contents: the set-up kernel writes
    // the table and dt and resets the flag word and the floor count
    k_noalloc_setup<<<1, 32, 0, c.stream>>>(hb, dbox, c.dt, dt, c.dtc, c.bad, c.nfloor);
    c.step(&c, false);
    e = cudaGetLastError();
    if (e != cudaSuccess) return reject(MHD_ECUDA, cudaGetErrorString(e));
    return MHD_OK;
}
