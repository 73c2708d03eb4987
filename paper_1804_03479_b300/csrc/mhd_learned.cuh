// mhd_learned.cuh -- device code of the learned path selector.
//
// Per 4^3 block of cells a small MLP (48 features -> 64 -> 64 -> 1, ReLU,
// logit out) predicts whether the cheap path (primitive PLM + HLLE) stays
// within a stated error of the full path (characteristic PPM + HLLD) for one
// step.  The two dense layers run on the tensor cores as warp-level
// mma.m16n8k16 with BF16 operands and FP32 accumulation; a warp owns 16 rows
// (blocks or training samples) and keeps each layer's output in registers
// as the next layer's A fragments.
//
// Quantisation points (mirrored by the CPU reference of the tests):
//   X_q = bf16(X), W1_q = bf16(W1), W2_q = bf16(W2); b1, b2, w3, b3 FP32
//   A1 = X_q W1_q + b1, H1 = relu(A1), H1_q = bf16(H1)
//   A2 = H1_q W2_q + b2, H2 = relu(A2) (FP32), z = H2 . w3 + b3
//   dz = (sigmoid(z) - y) wgt / sum(wgt)
//   dH2 = dz w3 [A2 > 0], dH2_q = bf16(dH2)
//   dH1 = (dH2_q W2_q^T) [A1 > 0], dH1_q = bf16(dH1)
//   dW1 = X_q^T dH1_q, dW2 = H1_q^T dH2_q, dw3 = H2^T dz,
//   db1 = sum dH1, db2 = sum dH2, db3 = sum dz
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>
#include "mhd_kernels.cuh"

namespace mhd {

constexpr int NF = 48;         // features per block
constexpr int NH = 64;         // hidden width
// packed FP32 parameters: W1[48][64], b1[64], W2[64][64], b2[64], w3[64], b3
constexpr int P_W1 = 0, P_B1 = NF * NH, P_W2 = P_B1 + NH, P_B2 = P_W2 + NH * NH, P_W3 = P_B2 + NH,
              P_B3 = P_W3 + NH, NPARAM = P_B3 + 1;

struct MlpDev {
    const float* p;            // FP32 master parameters [NPARAM]
    const uint32_t* w1t;       // bf16 W1^T [64][48] as 24 words per row
    const uint32_t* w2t;       // bf16 W2^T [64][64] as 32 words per row
    const uint32_t* w2n;       // bf16 W2   [64][64] as 32 words per row
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x (low half) = lo
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Forward pass of the 16 rows of one warp.  X rows r0 = row0 + g, r1 = r0 + 8
// (g = lane/4, t = lane%4); rows >= n read as zero.  Returns the C fragments
// of A1 and A2 (pre-activation, bias included) and the logits of rows r0, r1.
struct Frag {
    float a1[8][4];
    float a2[8][4];
    uint32_t x[3][4];
    float z0, z1;
};

__device__ __forceinline__ void mlp_forward16(const MlpDev& m, const float* __restrict__ X, long long n, long long row0,
                                              Frag& F)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const long long r0 = row0 + g, r1 = row0 + g + 8;
#pragma unroll
    for (int kk = 0; kk < 3; kk++) {
        const int col = 16 * kk + 2 * t;
        float x00 = 0, x01 = 0, x10 = 0, x11 = 0, x02 = 0, x03 = 0, x12 = 0, x13 = 0;
        if (r0 < n) {
            const float* xr = X + r0 * NF;
            x00 = xr[col]; x01 = xr[col + 1]; x02 = xr[col + 8]; x03 = xr[col + 9];
        }
        if (r1 < n) {
            const float* xr = X + r1 * NF;
            x10 = xr[col]; x11 = xr[col + 1]; x12 = xr[col + 8]; x13 = xr[col + 9];
        }
        F.x[kk][0] = pack_bf16(x00, x01);
        F.x[kk][1] = pack_bf16(x10, x11);
        F.x[kk][2] = pack_bf16(x02, x03);
        F.x[kk][3] = pack_bf16(x12, x13);
    }
    // layer 1
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const float bb0 = m.p[P_B1 + 8 * j + 2 * t], bb1 = m.p[P_B1 + 8 * j + 2 * t + 1];
        F.a1[j][0] = bb0; F.a1[j][1] = bb1; F.a1[j][2] = bb0; F.a1[j][3] = bb1;
        const uint32_t* wrow = m.w1t + (8 * j + g) * 24;
#pragma unroll
        for (int kk = 0; kk < 3; kk++) mma_bf16(F.a1[j], F.x[kk], wrow[8 * kk + t], wrow[8 * kk + 4 + t]);
    }
    // H1_q as the A fragments of layer 2
    uint32_t h1[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; kk++) {
        h1[kk][0] = pack_bf16(fmaxf(F.a1[2 * kk][0], 0.f), fmaxf(F.a1[2 * kk][1], 0.f));
        h1[kk][1] = pack_bf16(fmaxf(F.a1[2 * kk][2], 0.f), fmaxf(F.a1[2 * kk][3], 0.f));
        h1[kk][2] = pack_bf16(fmaxf(F.a1[2 * kk + 1][0], 0.f), fmaxf(F.a1[2 * kk + 1][1], 0.f));
        h1[kk][3] = pack_bf16(fmaxf(F.a1[2 * kk + 1][2], 0.f), fmaxf(F.a1[2 * kk + 1][3], 0.f));
    }
    // layer 2
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const float bb0 = m.p[P_B2 + 8 * j + 2 * t], bb1 = m.p[P_B2 + 8 * j + 2 * t + 1];
        F.a2[j][0] = bb0; F.a2[j][1] = bb1; F.a2[j][2] = bb0; F.a2[j][3] = bb1;
        const uint32_t* wrow = m.w2t + (8 * j + g) * 32;
#pragma unroll
        for (int kk = 0; kk < 4; kk++) mma_bf16(F.a2[j], h1[kk], wrow[8 * kk + t], wrow[8 * kk + 4 + t]);
    }
    // layer 3 (FP32): each thread holds 16 columns of rows r0 and r1
    float p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const float w0 = m.p[P_W3 + 8 * j + 2 * t], w1 = m.p[P_W3 + 8 * j + 2 * t + 1];
        p0 += fmaxf(F.a2[j][0], 0.f) * w0 + fmaxf(F.a2[j][1], 0.f) * w1;
        p1 += fmaxf(F.a2[j][2], 0.f) * w0 + fmaxf(F.a2[j][3], 0.f) * w1;
    }
    p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
    p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
    F.z0 = p0 + m.p[P_B3];
    F.z1 = p1 + m.p[P_B3];
}

// inference: logits of n rows (one warp per 16 rows, grid-stride)
__global__ void __launch_bounds__(256) k_mlp_infer(MlpDev m, const float* __restrict__ X, long long n,
                                                   float* __restrict__ logits, unsigned char* __restrict__ full_flag)
{
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long w = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); w * 16 < n; w += warps) {
        Frag F;
        mlp_forward16(m, X, n, w * 16, F);
        if ((lane & 3) == 0) {
            const long long r0 = w * 16 + (lane >> 2), r1 = r0 + 8;
            if (r0 < n) {
                if (logits) logits[r0] = F.z0;
                if (full_flag) full_flag[r0] = F.z0 > 0.f ? 0 : 1;   // logit > 0: the cheap path is predicted safe
            }
            if (r1 < n) {
                if (logits) logits[r1] = F.z1;
                if (full_flag) full_flag[r1] = F.z1 > 0.f ? 0 : 1;
            }
        }
    }
}

// sum over the 8 lanes sharing t (lanes t, t+4, ..., t+28)
__device__ __forceinline__ float sum_over_g(float v)
{
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
}

// Training forward + backward through the activations (one warp per 16
// samples).  Writes X_q, H1_q, dH2_q, dH1_q (bf16, zero rows past n) for the
// weight-gradient kernel and accumulates the bias and w3 gradients and the
// loss into grad / loss with atomics.
__global__ void __launch_bounds__(256) k_mlp_train_act(MlpDev m, const float* __restrict__ X, const float* __restrict__ y,
                                                       const float* __restrict__ wgt, long long n, long long npad,
                                                       float inv_wsum, uint32_t* __restrict__ Xq, uint32_t* __restrict__ H1q,
                                                       uint32_t* __restrict__ dH2q, uint32_t* __restrict__ dH1q,
                                                       float* __restrict__ grad, float* __restrict__ loss)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long w = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); w * 16 < npad; w += warps) {
        Frag F;
        mlp_forward16(m, X, n, w * 16, F);
        const long long r0 = w * 16 + g, r1 = r0 + 8;
        const float y0 = r0 < n ? y[r0] : 0.f, y1 = r1 < n ? y[r1] : 0.f;
        const float q0 = r0 < n ? (wgt ? wgt[r0] : 1.f) : 0.f, q1 = r1 < n ? (wgt ? wgt[r1] : 1.f) : 0.f;
        const float s0 = 1.f / (1.f + expf(-F.z0)), s1 = 1.f / (1.f + expf(-F.z1));
        const float dz0 = (s0 - y0) * q0 * inv_wsum, dz1 = (s1 - y1) * q1 * inv_wsum;
        // loss: sum of wgt * BCE(z, y) / sum(wgt), stable form
        if (t == 0) {
            float l0 = fmaxf(F.z0, 0.f) - F.z0 * y0 + log1pf(expf(-fabsf(F.z0)));
            float l1 = fmaxf(F.z1, 0.f) - F.z1 * y1 + log1pf(expf(-fabsf(F.z1)));
            float l = (l0 * q0 + l1 * q1) * inv_wsum;
            l += __shfl_xor_sync(0x11111111u, l, 4);
            l += __shfl_xor_sync(0x11111111u, l, 8);
            l += __shfl_xor_sync(0x11111111u, l, 16);
            if (lane == 0) atomicAdd(loss, l);
        }
        float db3 = (t == 0) ? dz0 + dz1 : 0.f;
        // dH2 = dz w3 [A2 > 0]; w3 and b2 gradients
        float dh2[8][4];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int c0 = 8 * j + 2 * t;
            const float w0 = m.p[P_W3 + c0], w1 = m.p[P_W3 + c0 + 1];
            dh2[j][0] = F.a2[j][0] > 0.f ? dz0 * w0 : 0.f;
            dh2[j][1] = F.a2[j][1] > 0.f ? dz0 * w1 : 0.f;
            dh2[j][2] = F.a2[j][2] > 0.f ? dz1 * w0 : 0.f;
            dh2[j][3] = F.a2[j][3] > 0.f ? dz1 * w1 : 0.f;
            float gw0 = sum_over_g(fmaxf(F.a2[j][0], 0.f) * dz0 + fmaxf(F.a2[j][2], 0.f) * dz1);
            float gw1 = sum_over_g(fmaxf(F.a2[j][1], 0.f) * dz0 + fmaxf(F.a2[j][3], 0.f) * dz1);
            float gb0 = sum_over_g(dh2[j][0] + dh2[j][2]);
            float gb1 = sum_over_g(dh2[j][1] + dh2[j][3]);
            if (g == 0) {
                atomicAdd(grad + P_W3 + c0, gw0);
                atomicAdd(grad + P_W3 + c0 + 1, gw1);
                atomicAdd(grad + P_B2 + c0, gb0);
                atomicAdd(grad + P_B2 + c0 + 1, gb1);
            }
        }
        db3 += __shfl_xor_sync(0xffffffffu, db3, 4);
        db3 += __shfl_xor_sync(0xffffffffu, db3, 8);
        db3 += __shfl_xor_sync(0xffffffffu, db3, 16);
        if (lane == 0) atomicAdd(grad + P_B3, db3);
        // dH2_q as A fragments; dH1 = dH2_q W2_q^T [A1 > 0]
        uint32_t a3[4][4];
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
            a3[kk][0] = pack_bf16(dh2[2 * kk][0], dh2[2 * kk][1]);
            a3[kk][1] = pack_bf16(dh2[2 * kk][2], dh2[2 * kk][3]);
            a3[kk][2] = pack_bf16(dh2[2 * kk + 1][0], dh2[2 * kk + 1][1]);
            a3[kk][3] = pack_bf16(dh2[2 * kk + 1][2], dh2[2 * kk + 1][3]);
        }
#pragma unroll
        for (int j = 0; j < 8; j++) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            const uint32_t* wrow = m.w2n + (8 * j + g) * 32;
#pragma unroll
            for (int kk = 0; kk < 4; kk++) mma_bf16(acc, a3[kk], wrow[8 * kk + t], wrow[8 * kk + 4 + t]);
            const int c0 = 8 * j + 2 * t;
            float d0 = F.a1[j][0] > 0.f ? acc[0] : 0.f, d1 = F.a1[j][1] > 0.f ? acc[1] : 0.f;
            float d2 = F.a1[j][2] > 0.f ? acc[2] : 0.f, d3 = F.a1[j][3] > 0.f ? acc[3] : 0.f;
            float gb0 = sum_over_g(d0 + d2), gb1 = sum_over_g(d1 + d3);
            if (g == 0) {
                atomicAdd(grad + P_B1 + c0, gb0);
                atomicAdd(grad + P_B1 + c0 + 1, gb1);
            }
            // stores: word of (row, cols c0, c0+1) in a [rows][64] bf16 array is row*32 + 4j + t
            dH1q[r0 * 32 + 4 * j + t] = pack_bf16(d0, d1);
            dH1q[r1 * 32 + 4 * j + t] = pack_bf16(d2, d3);
            dH2q[r0 * 32 + 4 * j + t] = a3[j >> 1][(j & 1) * 2];
            dH2q[r1 * 32 + 4 * j + t] = a3[j >> 1][(j & 1) * 2 + 1];
            H1q[r0 * 32 + 4 * j + t] = pack_bf16(fmaxf(F.a1[j][0], 0.f), fmaxf(F.a1[j][1], 0.f));
            H1q[r1 * 32 + 4 * j + t] = pack_bf16(fmaxf(F.a1[j][2], 0.f), fmaxf(F.a1[j][3], 0.f));
        }
#pragma unroll
        for (int kk = 0; kk < 3; kk++) {
            Xq[r0 * 24 + 8 * kk + t] = F.x[kk][0];
            Xq[r1 * 24 + 8 * kk + t] = F.x[kk][1];
            Xq[r0 * 24 + 8 * kk + 4 + t] = F.x[kk][2];
            Xq[r1 * 24 + 8 * kk + 4 + t] = F.x[kk][3];
        }
    }
}

__device__ __forceinline__ uint32_t pack_raw(unsigned short lo, unsigned short hi)
{
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

// Weight gradients on the tensor cores: dW1 = X_q^T dH1_q (48 x 64),
// dW2 = H1_q^T dH2_q (64 x 64), summed over the (padded) batch.  One warp per
// (16 x 8 output tile, 256-sample chunk); FP32 partial sums go to grad with
// atomics.  A(m, k) = act[k][m] and B(k, n) = dact[k][n] are gathered from the
// row-major bf16 arrays.
__global__ void __launch_bounds__(256) k_mlp_wgrad(const unsigned short* __restrict__ Xq, const unsigned short* __restrict__ H1q,
                                                   const unsigned short* __restrict__ dH1q,
                                                   const unsigned short* __restrict__ dH2q, long long npad,
                                                   float* __restrict__ grad)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int ntile1 = 3 * 8, ntile = ntile1 + 4 * 8;
    const long long nchunk = (npad + 255) / 256;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long w = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); w < ntile * nchunk; w += warps) {
        const int tile = (int)(w % ntile);
        const long long chunk = w / ntile;
        const bool first = tile < ntile1;
        const int mt = first ? tile / 8 : (tile - ntile1) / 8, nt = first ? tile % 8 : (tile - ntile1) % 8;
        const unsigned short* act = first ? Xq : H1q;
        const unsigned short* dact = first ? dH1q : dH2q;
        const int ma = first ? NF : NH;      // row length of act
        const int m0 = 16 * mt, n0 = 8 * nt;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const long long k1 = (chunk + 1) * 256 < npad ? (chunk + 1) * 256 : npad;
        for (long long k0 = chunk * 256; k0 < k1; k0 += 16) {
            uint32_t a[4];
            const long long ka = k0 + 2 * t;
            a[0] = pack_raw(act[ka * ma + m0 + g], act[(ka + 1) * ma + m0 + g]);
            a[1] = pack_raw(act[ka * ma + m0 + g + 8], act[(ka + 1) * ma + m0 + g + 8]);
            a[2] = pack_raw(act[(ka + 8) * ma + m0 + g], act[(ka + 9) * ma + m0 + g]);
            a[3] = pack_raw(act[(ka + 8) * ma + m0 + g + 8], act[(ka + 9) * ma + m0 + g + 8]);
            uint32_t b0 = pack_raw(dact[ka * NH + n0 + g], dact[(ka + 1) * NH + n0 + g]);
            uint32_t b1 = pack_raw(dact[(ka + 8) * NH + n0 + g], dact[(ka + 9) * NH + n0 + g]);
            mma_bf16(acc, a, b0, b1);
        }
        const int base = first ? P_W1 : P_W2;
        const int r0 = m0 + g, c0 = n0 + 2 * t;
        atomicAdd(grad + base + r0 * NH + c0, acc[0]);
        atomicAdd(grad + base + r0 * NH + c0 + 1, acc[1]);
        atomicAdd(grad + base + (r0 + 8) * NH + c0, acc[2]);
        atomicAdd(grad + base + (r0 + 8) * NH + c0 + 1, acc[3]);
    }
}

// Adam on the FP32 master parameters, then the bf16 operand copies
__global__ void k_adam(float* __restrict__ p, float* __restrict__ mom, float* __restrict__ vel,
                       const float* __restrict__ grad, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) {
        float gi = grad[i];
        float m = b1 * mom[i] + (1.f - b1) * gi;
        float v = b2 * vel[i] + (1.f - b2) * gi * gi;
        mom[i] = m;
        vel[i] = v;
        p[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

__global__ void k_mlp_refresh(const float* __restrict__ p, unsigned short* __restrict__ w1t, unsigned short* __restrict__ w2t,
                              unsigned short* __restrict__ w2n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NF * NH + 2 * NH * NH; i += gridDim.x * blockDim.x) {
        if (i < NF * NH) {
            int k = i / NH, n = i % NH;           // W1[k][n]
            w1t[n * NF + k] = __bfloat16_as_ushort(__float2bfloat16_rn(p[P_W1 + i]));
        } else if (i < NF * NH + NH * NH) {
            int q = i - NF * NH, k = q / NH, n = q % NH;   // W2[k][n]
            w2t[n * NH + k] = __bfloat16_as_ushort(__float2bfloat16_rn(p[P_W2 + q]));
        } else {
            int q = i - NF * NH - NH * NH;
            w2n[q] = __bfloat16_as_ushort(__float2bfloat16_rn(p[P_W2 + q]));
        }
    }
}

// ---------------------------------------------------------------------------
// Features of every 4^3 block of one box.  For each primitive q (rho, vx, vy,
// vz, P, Bx, By, Bz): mean, range, the largest jump between face neighbours along x, y and z (the block and one
// cell beyond each of its faces), standard deviation; each divided by a scale
// of the block (rho: mean rho; v: c_ref = sqrt((gamma P + B^2)/rho);
// P: mean P; B: B_ref = sqrt(B^2 + P)).  The mean slots of rho and P, which
// that scaling makes trivial, carry log10(beta)/6 and |v|/c_ref instead.
// ---------------------------------------------------------------------------
// Lane pairs own the blocks: a warp covers 64 consecutive cells along x (16
// blocks) of one row of blocks, lanes 2b and 2b + 1 the block of cells
// x0 .. x0 + 3, x0 = 4 (16 s + b), the first its z planes k0, k0 + 1, the
// second k0 + 2, k0 + 3; each row of 4 cells along x (one per (y, z)) is one
// 16-byte load, so a load instruction of a field fetches whole 128-byte
// lines, and every load of a field is issued before its arithmetic (one
// round trip per field).  A block's statistics are sums in the lane and one
// shuffle with its partner; the x neighbours across its faces come from the
// lanes two away (a load at the warp's ends), the y neighbours from loads of
// the rows beyond its faces, the z pair across the middle from the partner
// and the z neighbours from loads.  The raw statistics wait in shared memory
// until the block's scales are known.  Measured per 384^3 pass: 0.68 ms.
// (A lane per x column of a block, loading one field and one halo at a
// time, took 1.0 ms; a lane per z plane of a block, 0.82 ms: more shuffles.)
constexpr int FEAT_THREADS = 256;

template <class R>
__device__ __forceinline__ void load_row4(const R* __restrict__ p, float v[4])
{
    if constexpr (sizeof(R) == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p));
        const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
        v[0] = (float)a.x; v[1] = (float)a.y; v[2] = (float)b.x; v[3] = (float)b.y;
    }
}

template <class R>
__global__ void __launch_bounds__(FEAT_THREADS, 2) k_block_features(BoxDev g, const R* __restrict__ W, long long N,
                                                                    float gam, float* __restrict__ feats)
{
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ float sraw[FEAT_THREADS / 32][NF][16];   // per warp: each block's 48 raw entries
    const int lane = threadIdx.x & 31, hb = lane & 1, bl = lane >> 1;
    float (*raw)[16] = sraw[threadIdx.x >> 5];
    const int nbx = g.nx / 4, nby = g.ny / 4, nbz = g.nz / 4;
    const int nseg = (nbx + 15) / 16;
    const long long nitem = (long long)nseg * nby * nbz;
    const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
    // the loop bound is warp-uniform, so every lane takes part in the shuffles
    for (long long it = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; it < nitem; it += nwarp) {
        const int xs = (int)(it % nseg);
        const long long r = it / nseg;
        const int jb = (int)(r % nby), kb = (int)(r / nby);
        const int ib = 16 * xs + bl;
        const bool valid = ib < nbx;
        const int x0 = 4 * (valid ? ib : nbx - 1);     // lanes past the row read a valid block, unused
        const int j0 = 4 * jb, k0 = 4 * kb, kz = k0 + 2 * hb;   // this lane's planes kz, kz + 1
        const int jm = wrapi(j0 - 1, g.ny), jp = wrapi(j0 + 4, g.ny);
        const int kh = hb ? wrapi(k0 + 4, g.nz) : wrapi(k0 - 1, g.nz);   // the z neighbour plane on this lane's side
        // x neighbours outside the warp's reach: below the first block, and
        // above the last block of the row or of the warp
        const bool own_l = bl == 0, own_r = bl == 15 || ib + 1 >= nbx;
        const int xl = wrapi(x0 - 1, g.nx), xr = wrapi(x0 + 4, g.nx);
        float b2l = 0.f, mrho = 0.f, mP = 0.f;
#pragma unroll 1
        for (int f = 0; f < 8; f++) {
            const R* Wf = W + (long long)f * N;
            // every load of the field first: the lane's 8 rows (y j0 + (q & 3),
            // z kz + (q >> 2)), the rows beyond the block's y faces on its
            // planes, the plane beyond its z face on its side, and at the
            // warp's ends the x neighbour columns
            float v[8][4], hy[2][2][4], hz[4][4], xlo[8], xhi[8];
#pragma unroll
            for (int q = 0; q < 8; q++) load_row4(Wf + cell_of(g, x0, j0 + (q & 3), kz + (q >> 2)), v[q]);
#pragma unroll
            for (int p = 0; p < 2; p++) {
                load_row4(Wf + cell_of(g, x0, jm, kz + p), hy[p][0]);
                load_row4(Wf + cell_of(g, x0, jp, kz + p), hy[p][1]);
            }
#pragma unroll
            for (int jj = 0; jj < 4; jj++) load_row4(Wf + cell_of(g, x0, j0 + jj, kh), hz[jj]);
#pragma unroll
            for (int q = 0; q < 8; q++) {
                xlo[q] = own_l ? (float)Wf[cell_of(g, xl, j0 + (q & 3), kz + (q >> 2))] : 0.f;
                xhi[q] = own_r ? (float)Wf[cell_of(g, xr, j0 + (q & 3), kz + (q >> 2))] : 0.f;
            }
            float sum = 0.f, mn = 3e38f, mx = -3e38f, dx = 0.f, dy = 0.f, dz = 0.f;
#pragma unroll
            for (int q = 0; q < 8; q++) {
#pragma unroll
                for (int a = 0; a < 4; a++) {
                    sum += v[q][a];
                    mn = fminf(mn, v[q][a]);
                    mx = fmaxf(mx, v[q][a]);
                    if (a > 0) dx = fmaxf(dx, fabsf(v[q][a] - v[q][a - 1]));
                    if ((q & 3) > 0) dy = fmaxf(dy, fabsf(v[q][a] - v[q - 1][a]));
                    if (q >= 4) dz = fmaxf(dz, fabsf(v[q][a] - v[q - 4][a]));
                    if (f >= 5) b2l += v[q][a] * v[q][a];
                }
            }
            // x pairs across the block's faces: the blocks beside it are two lanes away
#pragma unroll
            for (int q = 0; q < 8; q++) {
                float left = __shfl_up_sync(FULL, v[q][3], 2);
                float right = __shfl_down_sync(FULL, v[q][0], 2);
                if (own_l) left = xlo[q];
                if (own_r) right = xhi[q];
                dx = fmaxf(dx, fmaxf(fabsf(v[q][0] - left), fabsf(right - v[q][3])));
            }
            // y pairs across the faces, for this lane's two planes
#pragma unroll
            for (int p = 0; p < 2; p++)
#pragma unroll
                for (int a = 0; a < 4; a++)
                    dy = fmaxf(dy, fmaxf(fabsf(v[4 * p][a] - hy[p][0][a]), fabsf(hy[p][1][a] - v[4 * p + 3][a])));
            // z pairs: across the block's middle (k0 + 1, k0 + 2; the partner's
            // planes) and across the face on this lane's side
#pragma unroll
            for (int jj = 0; jj < 4; jj++) {
#pragma unroll
                for (int a = 0; a < 4; a++) {
                    // the first lane sends its upper plane, the second its lower one
                    const float mine = hb ? v[jj][a] : v[4 + jj][a];
                    const float other = __shfl_xor_sync(FULL, mine, 1);
                    dz = fmaxf(dz, fabsf(mine - other));
                    dz = fmaxf(dz, fabsf(hb ? hz[jj][a] - v[4 + jj][a] : v[jj][a] - hz[jj][a]));
                }
            }
            sum += __shfl_xor_sync(FULL, sum, 1);
            mn = fminf(mn, __shfl_xor_sync(FULL, mn, 1));
            mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, 1));
            dx = fmaxf(dx, __shfl_xor_sync(FULL, dx, 1));
            dy = fmaxf(dy, __shfl_xor_sync(FULL, dy, 1));
            dz = fmaxf(dz, __shfl_xor_sync(FULL, dz, 1));
            const float m = sum * (1.f / 64.f);
            float sq = 0.f;
#pragma unroll
            for (int q = 0; q < 8; q++)
#pragma unroll
                for (int a = 0; a < 4; a++) {
                    const float e = v[q][a] - m;
                    sq += e * e;
                }
            sq += __shfl_xor_sync(FULL, sq, 1);
            if (f == 0) mrho = m;
            if (f == 4) mP = m;
            if (hb == 0) {
                raw[f * 6][bl] = m;
                raw[f * 6 + 1][bl] = mx - mn;
                raw[f * 6 + 2][bl] = dx;
                raw[f * 6 + 3][bl] = dy;
                raw[f * 6 + 4][bl] = dz;
                raw[f * 6 + 5][bl] = sqrtf(sq * (1.f / 64.f));
            }
        }
        // mean |v| over the block: the three velocity fields again (L1/L2),
        // every row in one round trip
        float vabs = 0.f;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const long long c = cell_of(g, x0, j0 + (q & 3), kz + (q >> 2));
            float vx[4], vy[4], vz[4];
            load_row4(W + N + c, vx);
            load_row4(W + 2 * N + c, vy);
            load_row4(W + 3 * N + c, vz);
#pragma unroll
            for (int a = 0; a < 4; a++) vabs += sqrtf(vx[a] * vx[a] + vy[a] * vy[a] + vz[a] * vz[a]);
        }
        vabs += __shfl_xor_sync(FULL, vabs, 1);
        b2l += __shfl_xor_sync(FULL, b2l, 1);
        __syncwarp();                                 // the raw entries are in shared memory
        if (valid) {
            const float inv = 1.f / 64.f;
            const float rho = mrho, P = fmaxf(mP, 1e-30f);
            const float b2 = b2l * inv;
            const float cref = sqrtf((gam * P + b2) / fmaxf(rho, 1e-30f));
            const float bref = sqrtf(b2 + P);
            // each lane of the pair scales and stores half of the block's row
            float o[NF / 2];
#pragma unroll
            for (int k = 0; k < NF / 2; k++) {
                const int e = hb * (NF / 2) + k, f = e / 6;
                const float is = 1.f / fmaxf(f == 0 ? rho : (f < 4 ? cref : (f == 4 ? P : bref)), 1e-30f);
                o[k] = raw[e][bl] * is;
            }
            if (hb == 0) o[0] = fminf(fmaxf(log10f(2.f * P / fmaxf(b2, 1e-30f)), -6.f), 6.f) / 6.f;
            else o[0] = vabs * inv / cref;            // entry 24: the mean slot of P
            float4* out = reinterpret_cast<float4*>(feats + (((long long)kb * nby + jb) * nbx + ib) * NF + hb * (NF / 2));
#pragma unroll
            for (int k = 0; k < NF / 8; k++) out[k] = make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
        }
        __syncwarp();                                 // the raw entries are rewritten by the next item
    }
}

// launch grid of k_block_features: one warp per row segment of 16 blocks
inline int features_grid(const BoxDev& g)
{
    const long long warps = (long long)((g.nx / 4 + 15) / 16) * (g.ny / 4) * (g.nz / 4);
    const long long blocks = (warps * 32 + FEAT_THREADS - 1) / FEAT_THREADS;
    return (int)(blocks < 148 * 16 ? blocks : 148 * 16);
}

// ---------------------------------------------------------------------------
// Per-block difference of two states of one box (the label of a training
// pair): max over the 8 stored fields of mean |a - b| over the block's 64
// cells divided by the field's scale in state a (rho: mean rho; momentum:
// mean rho times c_ref; e: mean e; face B: B_ref).
// ---------------------------------------------------------------------------
template <class TU, class TE>
__global__ void __launch_bounds__(256) k_block_err(BoxDev g, StateP<TU, TE> a, StateP<TU, TE> bb, float gam,
                                                   float* __restrict__ err)
{
    const int lane = threadIdx.x & 31;
    const int nbx = g.nx / 4, nby = g.ny / 4, nbz = g.nz / 4;
    const long long nblk = (long long)nbx * nby * nbz;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long b = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); b < nblk; b += warps) {
        const int ib = (int)(b % nbx), jb = (int)((b / nbx) % nby), kb = (int)(b / ((long long)nbx * nby));
        float d[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        float srho = 0.f, se = 0.f, sp = 0.f, sb2 = 0.f;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int i = 4 * ib + (lane & 3), j = 4 * jb + ((lane >> 2) & 3), k = 4 * kb + (lane >> 4) + 2 * h;
            const long long c = cell_of(g, i, j, k);
            float qa[8] = {(float)a.rho[c], (float)a.m[0][c], (float)a.m[1][c], (float)a.m[2][c], (float)a.e[c],
                           (float)a.b[0][c], (float)a.b[1][c], (float)a.b[2][c]};
            float qb[8] = {(float)bb.rho[c], (float)bb.m[0][c], (float)bb.m[1][c], (float)bb.m[2][c], (float)bb.e[c],
                           (float)bb.b[0][c], (float)bb.b[1][c], (float)bb.b[2][c]};
#pragma unroll
            for (int f = 0; f < 8; f++) d[f] += fabsf(qa[f] - qb[f]);
            const float bx = 0.5f * (qa[5] + (float)a.b[0][nbr(g, i, j, k, 0, 1)]);
            const float by = 0.5f * (qa[6] + (float)a.b[1][nbr(g, i, j, k, 1, 1)]);
            const float bz = 0.5f * (qa[7] + (float)a.b[2][nbr(g, i, j, k, 2, 1)]);
            const float bsq = bx * bx + by * by + bz * bz;
            const float ke = 0.5f * (qa[1] * qa[1] + qa[2] * qa[2] + qa[3] * qa[3]) / qa[0];
            srho += qa[0];
            se += qa[4];
            sp += (gam - 1.f) * (qa[4] - ke - 0.5f * bsq);
            sb2 += bsq;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int f = 0; f < 8; f++) d[f] += __shfl_xor_sync(0xffffffffu, d[f], o);
            srho += __shfl_xor_sync(0xffffffffu, srho, o);
            se += __shfl_xor_sync(0xffffffffu, se, o);
            sp += __shfl_xor_sync(0xffffffffu, sp, o);
            sb2 += __shfl_xor_sync(0xffffffffu, sb2, o);
        }
        if (lane == 0) {
            const float rho = srho / 64.f, e = fabsf(se / 64.f), P = fmaxf(sp / 64.f, 1e-30f), b2 = sb2 / 64.f;
            const float cref = sqrtf((gam * P + b2) / fmaxf(rho, 1e-30f));
            const float bref = sqrtf(b2 + P);
            const float scale[8] = {rho, rho * cref, rho * cref, rho * cref, e, bref, bref, bref};
            float m = 0.f;
#pragma unroll
            for (int f = 0; f < 8; f++) m = fmaxf(m, d[f] / 64.f / fmaxf(scale[f], 1e-30f));
            err[b] = m;
        }
    }
}

// ---------------------------------------------------------------------------
// Unit selection of the learned step: a sweep unit (tile, pencil segment or
// x-warp segment) along d is "full" when any 4^3 block holding a cell next to
// one of its faces is flagged full (so a face takes the full path whenever
// either neighbouring block asks for it), else "cheap".  One byte per unit
// (1 = full), in the units' own order, and a list of the full units: the
// cheap kernel runs over every unit and skips the marked ones, so adjacent
// lanes keep adjacent units and their loads stay coalesced (most units are
// cheap); the full kernel runs over the list only, its warps busy with full
// units.
// ---------------------------------------------------------------------------
// mark a unit and list it if full: one atomic per warp that has full units
// (the cheap units are counted by difference, so the many warps without a
// full unit touch no counter)
__device__ __forceinline__ void select_unit(long long t, bool full, unsigned char* sel, int* list_full, int* cnt_full)
{
    sel[t] = full;
    const unsigned act = __activemask();
    const unsigned fm = __ballot_sync(act, full);
    if (fm) {
        const int lane = threadIdx.x & 31, leader = __ffs(fm) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(cnt_full, __popc(fm));
        base = __shfl_sync(act, base, leader);
        if (full) list_full[base + __popc(fm & ((1u << lane) - 1u))] = (int)t;
    }
}

__global__ void k_tile_classify(BoxDev g, int d, int tl, const unsigned char* __restrict__ full_flag,
                                unsigned char* __restrict__ sel, int* __restrict__ list_full,
                                int* __restrict__ cnt_full, int ntile)
{
    const Tile T = tile_of(d, tl);
    const int ntx = (g.nx + T.ex - 1) / T.ex, nty = (g.ny + T.ey - 1) / T.ey;
    const int nbx = g.nx / 4, nby = g.ny / 4;
    for (int tile = blockIdx.x * blockDim.x + threadIdx.x; tile < ntile; tile += gridDim.x * blockDim.x) {
        int bl = tile;
        const int tx = bl % ntx; bl /= ntx;
        const int ty = bl % nty; bl /= nty;
        const int tz = bl;
        // cells beside the tile's faces: [x0 - 1, x0 + ex - 1] along d, the tile's extent across
        const int x0 = tx * T.ex - (d == 0), y0 = ty * T.ey - (d == 1), z0 = tz * T.ez - (d == 2);
        const int x1 = tx * T.ex + T.ex - 1, y1 = ty * T.ey + T.ey - 1, z1 = tz * T.ez + T.ez - 1;
        // block index ranges (floor division: the cell -1 lies in block -1, wrapped)
        const int nbz = g.nz / 4;
        const int kb0 = (z0 + 4) / 4 - 1, kb1 = z1 / 4;
        const int jb0 = (y0 + 4) / 4 - 1, jb1 = y1 / 4;
        const int ib0 = (x0 + 4) / 4 - 1, ib1 = x1 / 4;
        bool full = false;
        for (int kq = kb0; kq <= kb1 && !full; kq++)
            for (int jq = jb0; jq <= jb1 && !full; jq++)
                for (int iq = ib0; iq <= ib1 && !full; iq++) {
                    const int kb = wrapi(kq, nbz), jb = wrapi(jq, nby), ib = wrapi(iq, nbx);
                    full = full_flag[((long long)kb * nby + jb) * nbx + ib] != 0;
                }
        select_unit(tile, full, sel, list_full, cnt_full);
    }
}

// pencil segments of axis d (length pl) into cheap and full lists: full when
// any 4^3 block holding one of the cells beside the segment's faces (cells
// i0-1 .. i1-1 of its line) is flagged
__global__ void k_seg_classify(BoxDev g, int d, int pl, const unsigned char* __restrict__ full_flag,
                               unsigned char* __restrict__ sel, int* __restrict__ list_full,
                               int* __restrict__ cnt_full, long long nseg)
{
    int na, nb, ns;
    pencil_dims(g.nx, g.ny, g.nz, d, pl, na, nb, ns);
    const int nbx = g.nx / 4, nby = g.ny / 4;
    const int nd = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
    const int nbd = nd / 4;
    for (long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; t0 < nseg;
         t0 += (long long)gridDim.x * blockDim.x) {
        long long t = t0;
        const int ia = (int)(t % na);
        t /= na;
        const int ib = (int)(t % nb);
        const int sg = (int)(t / nb);
        const int i0 = sg * pl, i1 = i0 + pl < nd ? i0 + pl : nd;
        const int q0 = (i0 + 3) / 4 - 1, q1 = (i1 - 1) / 4;     // blocks of cells i0-1 and i1-1
        bool full = false;
        for (int q = q0; q <= q1 && !full; q++) {
            const int qb = wrapi(q, nbd);
            int bi, bj, bk;
            if (d == 0) { bi = qb; bj = ia / 4; bk = ib / 4; }
            else if (d == 1) { bi = ia / 4; bj = qb; bk = ib / 4; }
            else { bi = ia / 4; bj = ib / 4; bk = qb; }
            full = full_flag[((long long)bk * nby + bj) * nbx + bi] != 0;
        }
        select_unit(t0, full, sel, list_full, cnt_full);
    }
}

// x-warp items (decomposition dslot) into cheap and full lists: full when any
// 4^3 block holding one of the cells beside the item's faces (cells x0-1 ..
// x1-1 of its row) is flagged
__global__ void k_xw_classify(BoxDev g, int dslot, const unsigned char* __restrict__ full_flag,
                              unsigned char* __restrict__ sel, int* __restrict__ list_full,
                              int* __restrict__ cnt_full, long long nitem)
{
    const int fw = xw_faces(dslot);
    const int nseg = (g.nx + fw - 1) / fw;
    const int nbx = g.nx / 4, nby = g.ny / 4;
    for (long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; t0 < nitem;
         t0 += (long long)gridDim.x * blockDim.x) {
        long long t = t0;
        const int sg = (int)(t % nseg);
        t /= nseg;
        const int j = (int)(t % g.ny), k = (int)(t / g.ny);
        const int x0 = sg * fw, x1 = x0 + fw < g.nx ? x0 + fw : g.nx;
        const int q0 = (x0 + 3) / 4 - 1, q1 = (x1 - 1) / 4;
        bool full = false;
        for (int q = q0; q <= q1 && !full; q++)
            full = full_flag[((long long)(k / 4) * nby + j / 4) * nbx + wrapi(q, nbx)] != 0;
        select_unit(t0, full, sel, list_full, cnt_full);
    }
}

}  // namespace mhd
