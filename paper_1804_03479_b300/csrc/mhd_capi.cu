// mhd_capi.cu -- the C ABI declared in include/mhd.h.
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>
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

static void release(mhd_ctx* c)
{
    void* bufs[] = {c->rho, c->m[0], c->m[1], c->m[2], c->e, c->b[0], c->b[1], c->b[2], c->W, c->Wh,
                    c->F1, c->F2, c->E, c->Bh[0], c->Bh[1], c->Bh[2], c->WM, c->WP, c->stage,
                    c->dt, c->smax, c->bad, c->part, c->diag};
    for (void* p : bufs)
        if (p) cudaFree(p);
    if (c->have_graph) cudaGraphExecDestroy(c->gexec);
    if (c->prof_ev) {
        for (int q = 0; q < c->prof_cap * (MHD_NGROUPS + 1); q++) cudaEventDestroy(c->prof_ev[q]);
        free(c->prof_ev);
    }
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

static cudaError_t dalloc(mhd_ctx* c, void** p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) c->bytes += (long long)bytes;
    return e;
}

extern "C" mhd_status mhd_init(const mhd_grid* grid, double gamma, const mhd_scheme* scheme, void* stream,
                               mhd_ctx** out)
{
    if (!out) return MHD_EINVAL;
    *out = nullptr;
    if (!grid || !scheme) { g_init_err = "null grid or scheme"; return MHD_EINVAL; }
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->dx > 0.0)) { g_init_err = "bad grid"; return MHD_EINVAL; }
    if (!(gamma > 1.0)) { g_init_err = "gamma must exceed 1"; return MHD_EINVAL; }
    if (scheme->integrator < 0 || scheme->integrator > 1 || scheme->recon < 0 || scheme->recon > 2 ||
        scheme->riemann < 0 || scheme->riemann > 2 || scheme->precision < 0 || scheme->precision > 2) {
        g_init_err = "bad scheme enum";
        return MHD_EINVAL;
    }
    if (scheme->integrator == MHD_CTU && scheme->recon == MHD_PLM_PRIM) {
        g_init_err = "PLM_PRIM is built for VL only";
        return MHD_EUNSUPPORTED;
    }
    mhd_ctx* c = (mhd_ctx*)calloc(1, sizeof(mhd_ctx));
    if (!c) return MHD_ENOMEM;
    strcpy(c->err, "no error");
    c->grid = *grid;
    c->sch = *scheme;
    c->gamma = gamma;
    c->g.nx = grid->nx; c->g.ny = grid->ny; c->g.nz = grid->nz;
    c->g.n = (long long)grid->nx * grid->ny * grid->nz;
    c->g.dx = grid->dx;
    const long long n = c->g.n;
    cudaError_t attr = cudaSuccess;
    switch (scheme->precision) {
        case MHD_FP64: c->szu = 8; c->sze = 8; c->szr = 8; c->step = mhd_pick_fp64(scheme->integrator, scheme->recon, scheme->riemann, &attr); break;
        case MHD_FP32: c->szu = 4; c->sze = 4; c->szr = 4; c->step = mhd_pick_fp32(scheme->integrator, scheme->recon, scheme->riemann, &attr); break;
        default:       c->szu = 4; c->sze = 8; c->szr = 4; c->step = mhd_pick_mixed(scheme->integrator, scheme->recon, scheme->riemann, &attr); break;
    }
    if (!c->step) { free(c); g_init_err = "scheme combination not built"; return MHD_EUNSUPPORTED; }
    if (attr != cudaSuccess) { free(c); g_init_err = "cudaFuncSetAttribute failed"; return MHD_ECUDA; }
    c->launches = 12;   // prim, dt, 3 sweeps, emf, half, 3 sweeps or corrections, emf, full
    cudaError_t e = cudaSuccess;
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        c->own_stream = true;
    }
    const bool ctu = scheme->integrator == MHD_CTU;
    if (e == cudaSuccess) e = dalloc(c, &c->rho, n * c->szu);
    for (int d = 0; d < 3 && e == cudaSuccess; d++) e = dalloc(c, &c->m[d], n * c->szu);
    if (e == cudaSuccess) e = dalloc(c, &c->e, n * c->sze);
    for (int d = 0; d < 3 && e == cudaSuccess; d++) e = dalloc(c, &c->b[d], n * c->sze);
    if (e == cudaSuccess) e = dalloc(c, &c->W, 8 * n * c->szr);
    if (e == cudaSuccess) e = dalloc(c, &c->Wh, 8 * n * c->szr);
    if (e == cudaSuccess) e = dalloc(c, &c->F1, 21 * n * c->szr);
    if (e == cudaSuccess && ctu) e = dalloc(c, &c->F2, 21 * n * c->szr);
    if (e == cudaSuccess) e = dalloc(c, &c->E, 3 * n * c->szr);
    for (int d = 0; d < 3 && e == cudaSuccess; d++) e = dalloc(c, &c->Bh[d], n * c->sze);
    if (e == cudaSuccess && ctu) e = dalloc(c, &c->WM, 21 * n * c->szr);
    if (e == cudaSuccess && ctu) e = dalloc(c, &c->WP, 21 * n * c->szr);
    if (e == cudaSuccess && scheme->precision == MHD_MIXED) e = dalloc(c, &c->stage, 5 * n * sizeof(double));
    if (e == cudaSuccess) e = dalloc(c, (void**)&c->dt, sizeof(double));
    if (e == cudaSuccess) e = dalloc(c, (void**)&c->smax, sizeof(unsigned long long));
    if (e == cudaSuccess) e = dalloc(c, (void**)&c->bad, sizeof(unsigned long long));
    c->nblk = (int)((n + 255) / 256 < 148 * 16 ? (n + 255) / 256 : 148 * 16);
    if (e == cudaSuccess) e = dalloc(c, (void**)&c->part, (size_t)c->nblk * 10 * sizeof(double));
    if (e == cudaSuccess) e = dalloc(c, (void**)&c->diag, 10 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->bad, 0xff, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dt, 0, sizeof(double), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
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

static mhd_status check_device_flags(mhd_ctx* c)
{
    unsigned long long bad = ~0ull;
    CK(cudaMemcpyAsync(&bad, c->bad, sizeof(bad), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (bad != ~0ull) return fail(c, MHD_ENEGATIVE, "rho <= 0 or P <= 0 in cell %llu", bad);
    return c->sticky;
}

extern "C" mhd_status mhd_set_state(mhd_ctx* c, const void* U, const void* B, int on_device)
{
    if (!c || !U || !B) return fail(c, MHD_EINVAL, "null pointer");
    const long long n = c->g.n;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (c->sch.precision != MHD_MIXED) {
        const size_t sz = c->szu;  // == sze for the uniform layouts
        const char* u = (const char*)U;
        const char* b = (const char*)B;
        void* dst[5] = {c->rho, c->m[0], c->m[1], c->m[2], c->e};
        for (int f = 0; f < 5; f++) CK(cudaMemcpyAsync(dst[f], u + f * n * sz, n * sz, k, c->stream));
        for (int d = 0; d < 3; d++) CK(cudaMemcpyAsync(c->b[d], b + d * n * sz, n * sz, k, c->stream));
    } else {
        const double* u = (const double*)U;
        const double* b = (const double*)B;
        CK(cudaMemcpyAsync(c->stage, u, 4 * n * sizeof(double), k, c->stream));
        CK(cudaMemcpyAsync(c->e, u + 4 * n, n * sizeof(double), k, c->stream));
        for (int d = 0; d < 3; d++) CK(cudaMemcpyAsync(c->b[d], b + d * n, n * sizeof(double), k, c->stream));
        void* dst[4] = {c->rho, c->m[0], c->m[1], c->m[2]};
        for (int f = 0; f < 4; f++)
            k_convert<float, double><<<c->nblk, 256, 0, c->stream>>>((float*)dst[f], (const double*)c->stage + f * n, n);
        CK(cudaGetLastError());
    }
    if (!on_device) CK(cudaStreamSynchronize(c->stream));
    return MHD_OK;
}

extern "C" mhd_status mhd_get_state(mhd_ctx* c, void* U, void* B, int on_device)
{
    if (!c || !U || !B) return fail(c, MHD_EINVAL, "null pointer");
    const long long n = c->g.n;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (c->sch.precision != MHD_MIXED) {
        const size_t sz = c->szu;
        char* u = (char*)U;
        char* b = (char*)B;
        void* src[5] = {c->rho, c->m[0], c->m[1], c->m[2], c->e};
        for (int f = 0; f < 5; f++) CK(cudaMemcpyAsync(u + f * n * sz, src[f], n * sz, k, c->stream));
        for (int d = 0; d < 3; d++) CK(cudaMemcpyAsync(b + d * n * sz, c->b[d], n * sz, k, c->stream));
    } else {
        double* u = (double*)U;
        double* b = (double*)B;
        void* src[4] = {c->rho, c->m[0], c->m[1], c->m[2]};
        for (int f = 0; f < 4; f++)
            k_convert<double, float><<<c->nblk, 256, 0, c->stream>>>((double*)c->stage + f * n, (const float*)src[f], n);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(u, c->stage, 4 * n * sizeof(double), k, c->stream));
        CK(cudaMemcpyAsync(u + 4 * n, c->e, n * sizeof(double), k, c->stream));
        for (int d = 0; d < 3; d++) CK(cudaMemcpyAsync(b + d * n, c->b[d], n * sizeof(double), k, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return check_device_flags(c);
}

extern "C" mhd_status mhd_cfl_dt(mhd_ctx* c, double* dt)
{
    if (!c || !dt) return fail(c, MHD_EINVAL, "null pointer");
    CK(cudaMemsetAsync(c->smax, 0, sizeof(unsigned long long), c->stream));
    switch (c->sch.precision) {
        case MHD_FP64: k_prim<double, double, double><<<c->nblk, 256, 0, c->stream>>>(c->g, state_of<double, double>(c), (double*)c->W, c->gamma, c->smax, c->bad); break;
        case MHD_FP32: k_prim<float, float, float><<<c->nblk, 256, 0, c->stream>>>(c->g, state_of<float, float>(c), (float*)c->W, c->gamma, c->smax, c->bad); break;
        default:       k_prim<float, float, double><<<c->nblk, 256, 0, c->stream>>>(c->g, state_of<float, double>(c), (float*)c->W, c->gamma, c->smax, c->bad); break;
    }
    CK(cudaGetLastError());
    unsigned long long s = 0;
    CK(cudaMemcpyAsync(&s, c->smax, sizeof(s), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    double smax;
    memcpy(&smax, &s, sizeof(double));
    mhd_status st = check_device_flags(c);
    if (st != MHD_OK) return st;
    if (!(smax > 0.0)) return fail(c, MHD_ENEGATIVE, "no positive signal speed");
    *dt = c->sch.cfl * c->g.dx / smax;
    return MHD_OK;
}

extern "C" mhd_status mhd_step(mhd_ctx* c, double dt)
{
    if (!c) return MHD_EINVAL;
    if (!(dt > 0.0) || !(dt < 1e300)) return fail(c, MHD_EINVAL, "dt must be positive and finite");
    k_set_dt<<<1, 1, 0, c->stream>>>(c->dt, dt);
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
    CK(cudaMemcpyAsync(dt, c->dt, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MHD_OK;
}

static mhd_status run_diag(mhd_ctx* c, double out[10])
{
    switch (c->sch.precision) {
        case MHD_FP64: k_diag<double, double><<<c->nblk, 256, 0, c->stream>>>(c->g, state_of<double, double>(c), c->part); break;
        case MHD_FP32: k_diag<float, float><<<c->nblk, 256, 0, c->stream>>>(c->g, state_of<float, float>(c), c->part); break;
        default:       k_diag<float, double><<<c->nblk, 256, 0, c->stream>>>(c->g, state_of<float, double>(c), c->part); break;
    }
    k_finish_diag<<<1, 32, 0, c->stream>>>(c->part, c->nblk, c->diag);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, c->diag, 10 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return check_device_flags(c);
}

extern "C" mhd_status mhd_divB(mhd_ctx* c, double* maxabs, double* brms)
{
    if (!c || !maxabs || !brms) return fail(c, MHD_EINVAL, "null pointer");
    double d[10];
    mhd_status s = run_diag(c, d);
    *maxabs = d[0];
    *brms = sqrt(d[1] / (double)c->g.n);
    return s;
}

extern "C" mhd_status mhd_sums(mhd_ctx* c, double* sums8)
{
    if (!c || !sums8) return fail(c, MHD_EINVAL, "null pointer");
    double d[10];
    mhd_status s = run_diag(c, d);
    for (int f = 0; f < 8; f++) sums8[f] = d[2 + f];
    return s;
}

extern "C" mhd_status mhd_sync(mhd_ctx* c)
{
    if (!c) return MHD_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaGetLastError());
    return check_device_flags(c);
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
    cudaStreamSynchronize(c->stream);
    c->sticky = MHD_OK;
    strcpy(c->err, "no error");
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
