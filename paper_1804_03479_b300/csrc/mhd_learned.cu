// mhd_learned.cu -- the learned path selector: MLP, training kernels'
// driver, block features and errors, and the selected VL step (FP32).
#include <stdlib.h>
#include <string.h>
#include "mhd_engine.cuh"
#include "mhd_learned.cuh"

using namespace mhd;

void mhd_internal_set_init_error(const char* msg);
void mhd_internal_count_launches(mhd_ctx* c);

struct mhd_mlp {
    cudaStream_t stream;
    float* p;            // FP32 master parameters
    float* mom;          // Adam moments
    float* vel;
    float* grad;
    float* loss;
    unsigned short* w1t; // bf16 operand copies
    unsigned short* w2t;
    unsigned short* w2n;
    // training scratch (grown on demand)
    long long cap;
    uint32_t* xq;
    uint32_t* h1q;
    uint32_t* dh2q;
    uint32_t* dh1q;
    long long step;
};

static MlpDev mlp_dev(const mhd_mlp* m)
{
    MlpDev d;
    d.p = m->p;
    d.w1t = (const uint32_t*)m->w1t;
    d.w2t = (const uint32_t*)m->w2t;
    d.w2n = (const uint32_t*)m->w2n;
    return d;
}

static void mlp_release(mhd_mlp* m)
{
    void* bufs[] = {m->p, m->mom, m->vel, m->grad, m->loss, m->w1t, m->w2t, m->w2n, m->xq, m->h1q, m->dh2q, m->dh1q};
    for (void* b : bufs)
        if (b) cudaFree(b);
}

// splitmix64: the seeded stream of the initial weights
static unsigned long long splitmix64(unsigned long long& s)
{
    unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" mhd_status mhd_mlp_create(void* stream, unsigned long long seed, mhd_mlp** out)
{
    if (!out) return MHD_EINVAL;
    *out = nullptr;
    mhd_mlp* m = (mhd_mlp*)calloc(1, sizeof(mhd_mlp));
    if (!m) return MHD_ENOMEM;
    m->stream = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    float** fb[] = {&m->p, &m->mom, &m->vel, &m->grad};
    for (float** b : fb)
        if (e == cudaSuccess) e = cudaMalloc((void**)b, NPARAM * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->w1t, NF * NH * 2);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->w2t, NH * NH * 2);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->w2n, NH * NH * 2);
    if (e != cudaSuccess) {
        mlp_release(m);
        free(m);
        mhd_internal_set_init_error("mhd_mlp_create: device allocation failed");
        return MHD_ENOMEM;
    }
    // He-uniform weights, zero biases (seeded)
    float* h = (float*)calloc(NPARAM, sizeof(float));
    unsigned long long s = seed;
    for (int i = 0; i < NPARAM; i++) {
        float bound = 0.f;
        if (i < P_B1) bound = sqrtf(6.f / NF);
        else if (i >= P_W2 && i < P_B2) bound = sqrtf(6.f / NH);
        else if (i >= P_W3 && i < P_B3) bound = sqrtf(6.f / NH);
        double u = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
        h[i] = bound * (float)(2.0 * u - 1.0);
    }
    e = cudaMemcpyAsync(m->p, h, NPARAM * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->mom, 0, NPARAM * sizeof(float), m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->vel, 0, NPARAM * sizeof(float), m->stream);
    if (e == cudaSuccess) {
        k_mlp_refresh<<<32, 256, 0, m->stream>>>(m->p, m->w1t, m->w2t, m->w2n);
        e = cudaStreamSynchronize(m->stream);
    }
    free(h);
    if (e != cudaSuccess) {
        mlp_release(m);
        free(m);
        return MHD_ECUDA;
    }
    *out = m;
    return MHD_OK;
}

extern "C" void mhd_mlp_free(mhd_mlp* m)
{
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    mlp_release(m);
    free(m);
}

extern "C" int mhd_mlp_nparam(void) { return NPARAM; }

extern "C" mhd_status mhd_mlp_set_weights(mhd_mlp* m, const float* w, int on_device)
{
    if (!m || !w) return MHD_EINVAL;
    if (cudaMemcpyAsync(m->p, w, NPARAM * sizeof(float), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        m->stream) != cudaSuccess)
        return MHD_ECUDA;
    cudaMemsetAsync(m->mom, 0, NPARAM * sizeof(float), m->stream);
    cudaMemsetAsync(m->vel, 0, NPARAM * sizeof(float), m->stream);
    m->step = 0;
    k_mlp_refresh<<<32, 256, 0, m->stream>>>(m->p, m->w1t, m->w2t, m->w2n);
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? MHD_OK : MHD_ECUDA;
}

extern "C" mhd_status mhd_mlp_get_weights(mhd_mlp* m, float* w, int on_device)
{
    if (!m || !w) return MHD_EINVAL;
    if (cudaMemcpyAsync(w, m->p, NPARAM * sizeof(float), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        m->stream) != cudaSuccess)
        return MHD_ECUDA;
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? MHD_OK : MHD_ECUDA;
}

static mhd_status ensure_train_cap(mhd_mlp* m, long long npad)
{
    if (npad <= m->cap) return MHD_OK;
    uint32_t** bufs[] = {&m->xq, &m->h1q, &m->dh2q, &m->dh1q};
    for (uint32_t** b : bufs)
        if (*b) { cudaFree(*b); *b = nullptr; }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->xq, npad * NF * 2);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->h1q, npad * NH * 2);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->dh2q, npad * NH * 2);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->dh1q, npad * NH * 2);
    if (e != cudaSuccess) { m->cap = 0; return MHD_ENOMEM; }
    m->cap = npad;
    return MHD_OK;
}

// gradient of the weighted mean BCE loss over n samples into m->grad
static mhd_status mlp_gradient(mhd_mlp* m, const float* X, const float* y, const float* wgt, long long n, double wsum,
                               float* loss_host)
{
    const long long npad = (n + 15) / 16 * 16;
    mhd_status st = ensure_train_cap(m, npad);
    if (st != MHD_OK) return st;
    cudaMemsetAsync(m->grad, 0, NPARAM * sizeof(float), m->stream);
    cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream);
    const int grid = (int)((npad / 16 + 7) / 8 < 1184 ? (npad / 16 + 7) / 8 : 1184);
    k_mlp_train_act<<<grid, 256, 0, m->stream>>>(mlp_dev(m), X, y, wgt, n, npad, (float)(1.0 / wsum), m->xq, m->h1q,
                                                 m->dh2q, m->dh1q, m->grad, m->loss);
    const long long nw = 56 * ((npad + 255) / 256);
    const int grid2 = (int)((nw + 7) / 8 < 1184 ? (nw + 7) / 8 : 1184);
    k_mlp_wgrad<<<grid2, 256, 0, m->stream>>>((const unsigned short*)m->xq, (const unsigned short*)m->h1q,
                                              (const unsigned short*)m->dh1q, (const unsigned short*)m->dh2q, npad,
                                              m->grad);
    if (cudaGetLastError() != cudaSuccess) return MHD_ECUDA;
    if (loss_host) {
        if (cudaMemcpyAsync(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
            return MHD_ECUDA;
        if (cudaStreamSynchronize(m->stream) != cudaSuccess) return MHD_ECUDA;
    }
    return MHD_OK;
}

extern "C" mhd_status mhd_mlp_grad(mhd_mlp* m, const float* X, const float* y, const float* wgt, long long n,
                                   double wsum, float* grad_out, float* loss)
{
    if (!m || !X || !y || n < 1 || !(wsum > 0.0) || !grad_out) return MHD_EINVAL;
    mhd_status st = mlp_gradient(m, X, y, wgt, n, wsum, loss);
    if (st != MHD_OK) return st;
    if (cudaMemcpyAsync(grad_out, m->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToDevice, m->stream) != cudaSuccess)
        return MHD_ECUDA;
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? MHD_OK : MHD_ECUDA;
}

extern "C" mhd_status mhd_mlp_train_step(mhd_mlp* m, const float* X, const float* y, const float* wgt, long long n,
                                         double wsum, double lr, float* loss)
{
    if (!m || !X || !y || n < 1 || !(wsum > 0.0) || !(lr > 0.0)) return MHD_EINVAL;
    mhd_status st = mlp_gradient(m, X, y, wgt, n, wsum, nullptr);
    if (st != MHD_OK) return st;
    m->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
    k_adam<<<32, 256, 0, m->stream>>>(m->p, m->mom, m->vel, m->grad, (float)lr, b1, b2, 1e-8f, c1, c2);
    k_mlp_refresh<<<32, 256, 0, m->stream>>>(m->p, m->w1t, m->w2t, m->w2n);
    if (cudaGetLastError() != cudaSuccess) return MHD_ECUDA;
    if (loss) {
        if (cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
            return MHD_ECUDA;
        if (cudaStreamSynchronize(m->stream) != cudaSuccess) return MHD_ECUDA;
    }
    return MHD_OK;
}

extern "C" mhd_status mhd_mlp_predict(mhd_mlp* m, const float* X, long long n, float* logits)
{
    if (!m || !X || !logits || n < 1) return MHD_EINVAL;
    const int grid = (int)((n / 16 + 8) / 8 < 1184 ? (n / 16 + 8) / 8 : 1184);
    k_mlp_infer<<<grid, 256, 0, m->stream>>>(mlp_dev(m), X, n, logits, nullptr);
    if (cudaGetLastError() != cudaSuccess) return MHD_ECUDA;
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? MHD_OK : MHD_ECUDA;
}

// ---------------------------------------------------------------------------
// block features and block errors of single-box contexts
// ---------------------------------------------------------------------------
static bool blockable(const mhd_ctx* c)
{
    return c && c->nbox == 1 && c->hbox[0].nx % 4 == 0 && c->hbox[0].ny % 4 == 0 && c->hbox[0].nz % 4 == 0;
}

extern "C" long long mhd_nblocks(mhd_ctx* c)
{
    if (!blockable(c)) return -1;
    return (long long)(c->hbox[0].nx / 4) * (c->hbox[0].ny / 4) * (c->hbox[0].nz / 4);
}

static void launch_features(mhd_ctx* c, float* feats)
{
    const long long nblk = mhd_nblocks(c);
    const int grid = features_grid(c->hbox[0]);
    (void)nblk;
    const int nb = c->cell_grid;
    if (c->sch.precision == MHD_FP64) {
        k_prim<double, double, double><<<nb, CELL_THREADS, 0, c->stream>>>(c->B, state_of<double, double>(c), (double*)c->W, c->gamma, nullptr, c->bad, c->sch.pfloor);
        k_block_features<double><<<grid, 256, 0, c->stream>>>(c->hbox[0], (const double*)c->W, c->B.N, (float)c->gamma, feats);
    } else if (c->sch.precision == MHD_FP32) {
        k_prim<float, float, float><<<nb, CELL_THREADS, 0, c->stream>>>(c->B, state_of<float, float>(c), (float*)c->W, c->gamma, nullptr, c->bad, c->sch.pfloor);
        k_block_features<float><<<grid, 256, 0, c->stream>>>(c->hbox[0], (const float*)c->W, c->B.N, (float)c->gamma, feats);
    } else {
        k_prim<float, float, double><<<nb, CELL_THREADS, 0, c->stream>>>(c->B, state_of<float, double>(c), (float*)c->W, c->gamma, nullptr, c->bad, c->sch.pfloor);
        k_block_features<float><<<grid, 256, 0, c->stream>>>(c->hbox[0], (const float*)c->W, c->B.N, (float)c->gamma, feats);
    }
}

extern "C" mhd_status mhd_block_features(mhd_ctx* c, float* feats)
{
    if (!blockable(c) || !feats) {
        mhd_internal_set_init_error("mhd_block_features: one box with sides divisible by 4 and a device buffer");
        return MHD_EINVAL;
    }
    launch_features(c, feats);
    if (cudaGetLastError() != cudaSuccess) return MHD_ECUDA;
    return cudaStreamSynchronize(c->stream) == cudaSuccess ? MHD_OK : MHD_ECUDA;
}

extern "C" mhd_status mhd_block_error(mhd_ctx* a, mhd_ctx* b, float* err)
{
    if (!blockable(a) || !blockable(b) || !err || a->sch.precision != b->sch.precision ||
        a->hbox[0].nx != b->hbox[0].nx || a->hbox[0].ny != b->hbox[0].ny || a->hbox[0].nz != b->hbox[0].nz) {
        mhd_internal_set_init_error("mhd_block_error: two single-box contexts of one shape and precision");
        return MHD_EINVAL;
    }
    const long long nblk = mhd_nblocks(a);
    const int grid = (int)((nblk + 7) / 8 < 148 * 8 ? (nblk + 7) / 8 : 148 * 8);   // one warp per block
    cudaStreamSynchronize(b->stream);
    switch (a->sch.precision) {
        case MHD_FP64: k_block_err<double, double><<<grid, 256, 0, a->stream>>>(a->hbox[0], state_of<double, double>(a), state_of<double, double>(b), (float)a->gamma, err); break;
        case MHD_FP32: k_block_err<float, float><<<grid, 256, 0, a->stream>>>(a->hbox[0], state_of<float, float>(a), state_of<float, float>(b), (float)a->gamma, err); break;
        default:       k_block_err<float, double><<<grid, 256, 0, a->stream>>>(a->hbox[0], state_of<float, double>(a), state_of<float, double>(b), (float)a->gamma, err); break;
    }
    if (cudaGetLastError() != cudaSuccess) return MHD_ECUDA;
    return cudaStreamSynchronize(a->stream) == cudaSuccess ? MHD_OK : MHD_ECUDA;
}

// ---------------------------------------------------------------------------
// the selected step: features -> MLP -> flags -> tile lists -> cheap (PLM in
// primitives + HLLE) and full (characteristic PPM + HLLD) sweeps
// ---------------------------------------------------------------------------
// the selector's skip bytes of unit kind q (0: x predictor items, 6: x
// corrector items, 2d: the tiles or pencil segments of axis d), one byte per
// unit in a buffer sized in ints
static inline unsigned char* sel_of(mhd_ctx* c, int q) { return (unsigned char*)c->sel_list[q]; }

static void run_step_learned(mhd_ctx* c, bool device_dt)
{
    typedef float R;
    const Boxes g = c->B;
    const long long n = g.N;
    cudaStream_t st = c->stream;
    StateP<float, float> s = state_of<float, float>(c);
    R* W = (R*)c->W;
    R* Wh = (R*)c->Wh;
    R* F1 = (R*)c->F1;
    R* E = (R*)c->E;
    float* Bh[3] = {(float*)c->Bh[0], (float*)c->Bh[1], (float*)c->Bh[2]};
    const double gam = c->gamma;
    const long long nblk = mhd_nblocks(c);
    const size_t smem = sweep_smem_bytes<R>(PPM, g.tl);

    prof_mark(c, 0);
    k_prim4<R, float, float><<<c->quad_grid, CELL_THREADS, 0, st>>>(g, s, W, gam, device_dt ? c->smax_part : nullptr,
                                                                     c->bad, c->sch.pfloor, c->nfloor);
    if (device_dt) k_finalize_dt<<<(c->nbox + 127) / 128, 128, 0, st>>>(g, c->smax_part, c->sch.cfl, c->dt, c->smax, c->dtc);
    const bool xw = c->pencil_mask & 1;
    // x by aligned marching warps (bits 5 / 6): the cheap kernel solves every
    // face of the sweep (its segments are not the x-warp items of the lists)
    // and the full kernel, launched after it, overwrites the listed items
    const bool xm0 = xw && (c->pencil_mask & 32), xm1 = xw && (c->pencil_mask & 64);
    // With the x predictor marching and y, z by pencils the cheap predictor
    // sweeps need no list: they solve every face, the full list passes
    // overwrite theirs after them.  The selector's passes (features,
    // inference, classification) then run on the selector's stream beside
    // them, and the full passes wait for it.
    const bool ov = xm0 && (c->pencil_mask & 6) == 6 && c->sel_st;
    cudaStream_t ss = st;
    if (ov) {
        cudaEventRecord(c->sel_fork, st);
        cudaStreamWaitEvent(c->sel_st, c->sel_fork, 0);
        ss = c->sel_st;
    }
    // selector: features of the current state, one inference, tile lists
    const int fgrid = features_grid(c->hbox[0]);
    k_block_features<R><<<fgrid, 256, 0, ss>>>(c->hbox[0], W, n, (float)gam, c->sel_feats);
    const int igrid = (int)((nblk / 16 + 8) / 8 < 1184 ? (nblk / 16 + 8) / 8 : 1184);
    k_mlp_infer<<<igrid, 256, 0, ss>>>(mlp_dev(c->sel), c->sel_feats, nblk, nullptr, c->sel_flags);
    cudaMemsetAsync(c->sel_cnt, 0, 8 * sizeof(int), ss);
    // unit q (2d: axis d; 6: the x corrector's items): skip bytes sel_of(c, q),
    // full list sel_list[q + 1] with its count sel_cnt[q + 1]
    for (int d = 0; d < 3; d++) {
        if (d == 0 && xw) {
            // x by warps: the predictor's items (31 faces) in 0/1, the
            // corrector's (27 faces, shared by the cheap PLM and full PPM kernels) in 6/7
            k_xw_classify<<<(int)((g.nxw[0] + 255) / 256 < 4096 ? (g.nxw[0] + 255) / 256 : 4096), 256, 0, ss>>>(
                c->hbox[0], 0, c->sel_flags, sel_of(c, 0), c->sel_list[1], c->sel_cnt + 1, g.nxw[0]);
            k_xw_classify<<<(int)((g.nxw[2] + 255) / 256 < 4096 ? (g.nxw[2] + 255) / 256 : 4096), 256, 0, ss>>>(
                c->hbox[0], 2, c->sel_flags, sel_of(c, 6), c->sel_list[7], c->sel_cnt + 7, g.nxw[2]);
        } else if (c->pencil_mask >> d & 1)
            k_seg_classify<<<(int)((g.npth[d] + 255) / 256 < 4096 ? (g.npth[d] + 255) / 256 : 4096), 256, 0, ss>>>(
                c->hbox[0], d, g.pl, c->sel_flags, sel_of(c, 2 * d), c->sel_list[2 * d + 1],
                c->sel_cnt + 2 * d + 1, g.npth[d]);
        else
            k_tile_classify<<<(g.ntile[d] + 255) / 256, 256, 0, ss>>>(c->hbox[0], d, g.tl, c->sel_flags,
                                                                       sel_of(c, 2 * d), c->sel_list[2 * d + 1],
                                                                       c->sel_cnt + 2 * d + 1, g.ntile[d]);
    }
    if (ov) cudaEventRecord(c->sel_join, c->sel_st);
    prof_mark(c, 1);
    // VL steps 1-3: the cheap kernel over every unit but the marked ones
    // (x: warps marching their rows), the full kernel over the full list
    if (ov) {
        // the cheap sweeps over every face (their time goes to the x group),
        // then the full passes once the lists are there
        k_xmarch<R, PLM_PRIM, HLLE, 0, float><<<xmarch_grid(c), PENCIL_THREADS, 0, st>>>(g, W, s.b[0], F1, gam);
        for (int d = 1; d < 3; d++)
            launch_pencil<R, PLM_PRIM, HLLE, 0, float>(d, pencil_grid(c, d), st, g, W, s.b[d],
                                                          F1 + (long long)d * 7 * n, gam);
        cudaStreamWaitEvent(st, c->sel_join, 0);
        k_xwarp<R, PPM, HLLD, 0, float><<<list_grid_xwarp(c, 0), PENCIL_THREADS, 0, st>>>(
            g, W, s.b[0], F1, gam, 0, c->sel_list[1], c->sel_cnt + 1);
        prof_mark(c, 2);
        for (int d = 1; d < 3; d++) {
            launch_pencil<R, PPM, HLLD, 0, float>(d, list_grid_pencil(c, d), st, g, W, s.b[d],
                                                  F1 + (long long)d * 7 * n, gam, c->sel_list[2 * d + 1],
                                                  c->sel_cnt + 2 * d + 1);
            prof_mark(c, 2 + d);
        }
    }
    for (int d = 0; d < 3 && !ov; d++) {
        if (d == 0 && xw) {
            if (xm0)
                k_xmarch<R, PLM_PRIM, HLLE, 0, float><<<xmarch_grid(c), PENCIL_THREADS, 0, st>>>(g, W, s.b[0], F1,
                                                                                               gam);
            else
                k_xwarp<R, PLM_PRIM, HLLE, 0, float><<<xrow_grid(c), PENCIL_THREADS, 0, st>>>(
                    g, W, s.b[0], F1, gam, 0, nullptr, nullptr, nullptr, nullptr, nullptr, sel_of(c, 0));
            k_xwarp<R, PPM, HLLD, 0, float><<<list_grid_xwarp(c, 0), PENCIL_THREADS, 0, st>>>(
                g, W, s.b[0], F1, gam, 0, c->sel_list[1], c->sel_cnt + 1);
        } else if (c->pencil_mask >> d & 1) {
            launch_pencil<R, PLM_PRIM, HLLE, 0, float>(d, pencil_grid(c, d), st, g, W, s.b[d],
                                                          F1 + (long long)d * 7 * n, gam, nullptr, nullptr, nullptr,
                                                          nullptr, nullptr, sel_of(c, 2 * d));
            launch_pencil<R, PPM, HLLD, 0, float>(d, list_grid_pencil(c, d), st, g, W, s.b[d],
                                                          F1 + (long long)d * 7 * n, gam, c->sel_list[2 * d + 1],
                                                          c->sel_cnt + 2 * d + 1);
        } else {
            k_sweep<R, PLM_PRIM, HLLE, 0, float><<<sweep_grid(c, d), SWEEP_THREADS, 0, st>>>(
                g, d, W, s.b[d], F1 + (long long)d * 7 * n, nullptr, nullptr, c->dtc, gam, nullptr, nullptr,
                sel_of(c, 2 * d));
            k_sweep<R, PPM, HLLD, 0, float><<<sweep_grid(c, d), SWEEP_THREADS, 0, st>>>(
                g, d, W, s.b[d], F1 + (long long)d * 7 * n, nullptr, nullptr, c->dtc, gam, c->sel_list[2 * d + 1],
                c->sel_cnt + 2 * d + 1);
        }
        prof_mark(c, 2 + d);
    }
    const bool eu = emf_form(c) == 2;   // edge fields fused with the update that uses them
    // pencil-mask bits 1 and 7: the half update inside the cheap y corrector
    // pencils, which then solve every y face (the full list pass overwrites
    // its faces after them); the corrector's fluxes go to the second array
    const bool yh = sel_y_half(c);
    R* Fc = yh ? (R*)c->F2 : F1;
    // pencil-mask bits 2 and 9: the conservative update inside the cheap z
    // corrector pencils, after the full z list pass, whose faces they read;
    // the face field then by CT alone
    const bool zf = yh && (c->pencil_mask & 516) == 516;
    if (eu) {
        prof_mark(c, 5);
        launch_emf_update<R, float, float, true>(c, g, s, F1, W, Bh, Wh, st);
    } else {
        launch_emf<R>(c, g, F1, W, E, st);
        prof_mark(c, 5);
        if (yh)
            launch_yhalf<R, float, float, PLM_PRIM, HLLE>(c, g, s, F1, E, Bh, Wh, (R*)c->F2, st);
        else
            k_half4<R, float, float><<<c->quad_grid, CELL_THREADS, 0, st>>>(g, s, F1, E, c->dtc, gam, Bh[0], Bh[1],
                                                                             Bh[2], Wh, c->sch.pfloor);
    }
    prof_mark(c, 6);
    // VL steps 4-7
    for (int d = 0; d < 3; d++) {
        if (d == 0 && xw) {
            if (xm1)
                k_xmarch<R, PLM_PRIM, HLLE, 1, float><<<xmarch_grid(c), PENCIL_THREADS, 0, st>>>(g, Wh, Bh[0], Fc,
                                                                                               gam);
            else
                k_xwarp<R, PLM_PRIM, HLLE, 1, float><<<xrow_grid(c), PENCIL_THREADS, 0, st>>>(
                    g, Wh, Bh[0], Fc, gam, 2, nullptr, nullptr, nullptr, nullptr, nullptr, sel_of(c, 6));
            k_xwarp<R, PPM, HLLD, 1, float><<<list_grid_xwarp(c, 2), PENCIL_THREADS, 0, st>>>(
                g, Wh, Bh[0], Fc, gam, 2, c->sel_list[7], c->sel_cnt + 7);
        } else if (d == 2 && zf) {
            launch_pencil<R, PPM, HLLD, 1, float>(d, list_grid_pencil(c, d), st, g, Wh, Bh[d],
                                                  Fc + (long long)d * 7 * n, gam, c->sel_list[2 * d + 1],
                                                  c->sel_cnt + 2 * d + 1);
            k_zfull<R, float, float, PLM_PRIM, HLLE><<<pencil_grid(c, 2), PENCIL_THREADS, 0, st>>>(
                g, s, Wh, Bh[2], Fc, c->dtc, gam, sel_of(c, 2 * d));
        } else if (c->pencil_mask >> d & 1) {
            if (!(d == 1 && yh))     // (y: the cheap faces were solved with the half update)
                launch_pencil<R, PLM_PRIM, HLLE, 1, float>(d, pencil_grid(c, d), st, g, Wh, Bh[d],
                                                              Fc + (long long)d * 7 * n, gam, nullptr, nullptr,
                                                              nullptr, nullptr, nullptr, sel_of(c, 2 * d));
            launch_pencil<R, PPM, HLLD, 1, float>(d, list_grid_pencil(c, d), st, g, Wh, Bh[d],
                                                          Fc + (long long)d * 7 * n, gam, c->sel_list[2 * d + 1],
                                                          c->sel_cnt + 2 * d + 1);
        } else {
            k_sweep<R, PLM_PRIM, HLLE, 1, float><<<sweep_grid(c, d), SWEEP_THREADS,
                                                   sweep_smem_bytes<R>(PLM_PRIM, g.tl), st>>>(
                g, d, Wh, Bh[d], Fc + (long long)d * 7 * n, nullptr, nullptr, c->dtc, gam, nullptr, nullptr,
                sel_of(c, 2 * d));
            k_sweep<R, PPM, HLLD, 1, float><<<sweep_grid(c, d), SWEEP_THREADS, smem, st>>>(
                g, d, Wh, Bh[d], Fc + (long long)d * 7 * n, nullptr, nullptr, c->dtc, gam, c->sel_list[2 * d + 1],
                c->sel_cnt + 2 * d + 1);
        }
        prof_mark(c, 7 + d);
    }
    if (eu) {
        prof_mark(c, 10);
        launch_emf_update<R, float, float, false>(c, g, s, Fc, Wh, nullptr, nullptr, st);
    } else {
        launch_emf<R>(c, g, Fc, Wh, E, st);
        prof_mark(c, 10);
        if (zf)
            k_ct4<R, float, float><<<c->quad_grid, CELL_THREADS, 0, st>>>(g, s, E, c->dtc);
        else
            k_full4<R, float, float><<<c->quad_grid, CELL_THREADS, 0, st>>>(g, s, Fc, E, c->dtc);
    }
    prof_mark(c, 11);
    if (c->prof_on && c->prof_steps < c->prof_cap) c->prof_steps++;
}

// selector unit buffers large enough for the current sweep layout:
// the tiles of the shortest tile length and the pencil segments of the
// current length, whichever is more (grown when the layout needs more)
mhd_status mhd_internal_selector_lists(mhd_ctx* c)
{
    long long need = 0;
    const BoxDev& b0 = c->hbox[0];
    for (int d = 0; d < 3; d++) {
        long long nt = tiles_of_box(b0.nx, b0.ny, b0.nz, d, 4);
        long long np = pencil_threads_of_box(b0.nx, b0.ny, b0.nz, d, c->pencil_len);
        long long nw = xwarp_items_of_box(b0.nx, b0.ny, b0.nz, d);
        need = nt > need ? nt : need;
        need = np > need ? np : need;
        need = nw > need ? nw : need;
    }
    if (c->sel_list[0] && need <= c->sel_cap) return MHD_OK;
    if (c->have_graph) { cudaGraphExecDestroy(c->gexec); c->have_graph = false; }
    cudaStreamSynchronize(c->stream);
    for (int q = 0; q < 8; q++)
        if (c->sel_list[q]) {
            cudaFree(c->sel_list[q]);
            c->sel_list[q] = nullptr;
            c->bytes -= c->sel_cap * 4;
        }
    c->sel_cap = 0;
    for (int q = 0; q < 8; q++) {
        if (cudaMalloc((void**)&c->sel_list[q], (size_t)need * sizeof(int)) != cudaSuccess) return MHD_ENOMEM;
        c->bytes += need * 4;
    }
    c->sel_cap = need;
    return MHD_OK;
}

extern "C" mhd_status mhd_set_selector(mhd_ctx* c, mhd_mlp* m)
{
    if (!c) return MHD_EINVAL;
    if (!m) {   // back to the plain scheme
        c->sel = nullptr;
        c->step = c->plain_step;
        mhd_internal_count_launches(c);
        if (c->have_graph) { cudaGraphExecDestroy(c->gexec); c->have_graph = false; }
        return MHD_OK;
    }
    if (!blockable(c) || c->sch.precision != MHD_FP32 || c->sch.integrator != MHD_VL || c->bc) {
        snprintf(c->err, sizeof(c->err), "the selector needs one periodic FP32 VL box with sides divisible by 4");
        return MHD_EUNSUPPORTED;
    }
    if (!c->sel_feats) {
        const long long nblk = mhd_nblocks(c);
        cudaError_t e = cudaMalloc((void**)&c->sel_feats, nblk * NF * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->sel_flags, nblk);
        if (e == cudaSuccess) e = cudaMalloc((void**)&c->sel_cnt, 8 * sizeof(int));
        if (e != cudaSuccess) return MHD_ENOMEM;
        c->bytes += nblk * (NF * 4 + 1) + 24;
        cudaFuncSetAttribute(k_sweep<float, PPM, HLLD, 1, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sweep_smem_bytes<float>(PPM, TL_MAX));
    }
    // this unit's own instantiations of the edge-field kernels (their planes
    // take more than the default 48 KB of shared memory)
    if (cudaFuncSetAttribute(k_emf<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)emf_smem_bytes<float>()) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_emf_tma<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)emf_tma_smem_bytes()) != cudaSuccess)
        return MHD_ECUDA;
    if (mhd_internal_selector_lists(c) != MHD_OK) return MHD_ENOMEM;
    if (!c->sel_st) {
        if (cudaStreamCreateWithFlags(&c->sel_st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->sel_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->sel_join, cudaEventDisableTiming) != cudaSuccess)
            return MHD_ECUDA;
    }
    c->sel = m;
    c->step = run_step_learned;
    mhd_internal_count_launches(c);
    if (c->have_graph) { cudaGraphExecDestroy(c->gexec); c->have_graph = false; }
    return MHD_OK;
}

// fraction of 4^3 blocks and of sweep tiles the last selected step ran cheap
extern "C" mhd_status mhd_selector_stats(mhd_ctx* c, double* frac_blocks, double* frac_tiles)
{
    if (!c || !c->sel || !frac_blocks || !frac_tiles) return MHD_EINVAL;
    const long long nblk = mhd_nblocks(c);
    unsigned char* f = (unsigned char*)malloc((size_t)nblk);
    int cnt[6];
    if (!f) return MHD_ENOMEM;
    cudaError_t e = cudaMemcpyAsync(f, c->sel_flags, nblk, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, c->sel_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { free(f); return MHD_ECUDA; }
    long long cheap = 0;
    for (long long i = 0; i < nblk; i++) cheap += f[i] == 0;
    free(f);
    *frac_blocks = (double)cheap / (double)nblk;
    // the predictor's units of each axis (x-warp items, pencil segments or
    // tiles, by the sweep configuration): all of them, and the full ones
    long long tot = 0, tf = cnt[1] + cnt[3] + cnt[5];
    for (int d = 0; d < 3; d++)
        tot += (d == 0 && (c->pencil_mask & 1)) ? c->B.nxw[0] : ((c->pencil_mask >> d & 1) ? c->B.npth[d] : c->B.ntile[d]);
    *frac_tiles = tot > 0 ? (double)(tot - tf) / (double)tot : 0.0;
    return MHD_OK;
}
