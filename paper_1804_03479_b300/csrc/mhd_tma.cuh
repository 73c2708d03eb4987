// mhd_tma.cuh -- edge electric fields with the planes staged by the tensor
// memory accelerator (one-box FP32 and mixed contexts; mhd_set_emf_staging
// mode 1).
//
// The same edges as k_emf (Sec. 2, Eqs. 13-14 with the Gardiner-Stone
// reference field), with the same arithmetic per edge; only the staging
// differs.  k_emf has each of its threads load one staged cell per plane
// into registers, one plane ahead.  Here a producer warp issues bulk tensor
// copies (cp.async.bulk.tensor) of whole field planes into a ring of
// TMA_SLOTS plane slots in shared memory; an mbarrier per slot counts the
// bytes in, and a second one per slot counts the compute warps out.
//
// Measured on the B300 at 256^3 (per launch): 0.45 ms for 32 x 8 tiles with
// three slots (three blocks per SM), against 0.30 ms for k_emf.  Deeper rings
// cost resident blocks and were slower (32 x 16 tiles, five slots, one block
// per SM: 0.55 ms; 32 x 8, four slots, two blocks: 0.69 ms); line-aligned
// rows, a polling wait and leaving out the proxy fence changed nothing.  The
// per-plane compute of a block, with its barriers, bounds both forms, and
// k_emf keeps more of it in flight per SM.  k_emf is the default.
#pragma once
#include <cuda.h>
#include <stdint.h>
#include "mhd_kernels.cuh"

namespace mhd {

// ---- mbarrier and bulk-tensor primitives (inline PTX) ----------------------
__device__ __forceinline__ unsigned smem_addr(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// make the initialised barriers visible to the tensor memory accelerator
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic-proxy accesses of shared memory (made
// block-wide by a preceding barrier) before its later bulk copies into it
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// one arrival plus the transaction bytes the copies of this phase will bring
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// about 2 s at the B300's 2.03 GHz: far beyond any plane copy
constexpr long long TMA_WAIT_CYCLES = 4000000000LL;

// wait for the phase of the given parity.  After TMA_WAIT_CYCLES it gives
// up: sets bit `site` of *err and clears `live`, after which this thread
// waits no more (the kernel runs to its end on whatever the slots hold, in
// about one limit rather than one per plane, and the host reports the error)
__device__ __forceinline__ void mbar_wait_bounded(unsigned long long* bar, unsigned parity, unsigned* err, int site,
                                                  bool& live)
{
    if (!live) return;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > TMA_WAIT_CYCLES) {
            atomicOr(err, 1u << site);
            live = false;
            return;
        }
    }
}

// tiled 4-D bulk tensor copy global -> shared, completing on `bar`
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int f,
                                            unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(f), "r"(smem_addr(bar))
        : "memory");
}

// ---- the staged plane ------------------------------------------------------
// A tile is ETX x TY cells of an x-y slab, marched along z over EZC planes
// (plus the plane below).  A staged plane holds, per field, the cells
// x0 - 4 .. x0 + 35 (the copy starts on a 16-byte boundary; x0 - 1 is the
// halo) by y0 - 1 .. y0 + TY - 1: 40 x (TY + 1) values.  Its 15 fields, by
// logical index (the slots of 0-11 are those of k_emf's staged cell):
//   0-2   the velocity (W 1-3), replaced in place by the reference field
//         -(v x B) once the plane has arrived
//   3+3d  the mass flux of F_d (F_d 0); 4+3d, 5+3d its B fluxes (F_d 5, 6)
//   12-14 the cell-centred field (W 5-7)
// They arrive in 8 copies (fields adjacent in global memory share one copy,
// dense in shared memory): v, B, and per axis the mass flux and the two B
// fluxes.  Each copy lands on a 128-byte boundary.
constexpr int TMA_X = 40;
constexpr int TMA_TY = 8;                // tile rows of the staged form (k_emf: ETY = 16)
constexpr int TMA_SLOTS = 3;             // ring depth: 2 planes in flight while one is computed

__host__ __device__ constexpr int tma_round(int v) { return (v + 31) / 32 * 32; }   // 128 bytes of 4-byte values

template <int TY>
struct TmaPlane {
    static constexpr int Y = TY + 1;
    static constexpr int P = TMA_X * Y;                       // values per field plane
    static constexpr int V = 0;                               // v: 3 fields
    static constexpr int B = tma_round(3 * P);                // B: 3 fields
    static constexpr int FM0 = B + tma_round(3 * P);          // F_0 mass flux
    static constexpr int FB0 = FM0 + tma_round(P);            // F_0 B fluxes: 2 fields
    static constexpr int FAX = tma_round(P) + tma_round(2 * P);   // per-axis step of the flux copies
    static constexpr int SLOT = FM0 + 3 * FAX;                // values per slot
    static constexpr unsigned BYTES = 15u * P * 4u;           // one plane's copies
    static constexpr int THREADS = ETX * TY;                  // compute threads: one edge cell each
    __host__ __device__ static constexpr int off(int f)
    {
        return f < 3 ? V + f * P
                     : (f >= 12 ? B + (f - 12) * P
                                : ((f - 3) % 3 == 0 ? FM0 + (f - 3) / 3 * FAX
                                                    : FB0 + (f - 3) / 3 * FAX + ((f - 3) % 3 - 1) * P));
    }
};

static_assert(TmaPlane<TMA_TY>::off(14) + TmaPlane<TMA_TY>::P <= TmaPlane<TMA_TY>::FM0 &&
                  TmaPlane<TMA_TY>::off(11) + TmaPlane<TMA_TY>::P <= TmaPlane<TMA_TY>::SLOT,
              "the field planes of a slot do not overlap");
static_assert(TmaPlane<TMA_TY>::B % 32 == 0 && TmaPlane<TMA_TY>::FM0 % 32 == 0 && TmaPlane<TMA_TY>::FB0 % 32 == 0 &&
                  TmaPlane<TMA_TY>::FAX % 32 == 0 && TmaPlane<TMA_TY>::SLOT % 32 == 0,
              "every copy lands on a 128-byte boundary");

constexpr int EMF_TMA_THREADS = TmaPlane<TMA_TY>::THREADS + 32;   // the compute threads, then one producer warp

// the copies are 128-byte aligned in shared memory; the dynamic block is
// aligned up inside the kernel.  Then 2 x TMA_SLOTS barriers: full, empty.
constexpr size_t emf_tma_smem_bytes()
{
    return (size_t)TMA_SLOTS * TmaPlane<TMA_TY>::SLOT * 4 + 128 + 2 * TMA_SLOTS * sizeof(unsigned long long);
}

// barrier 1 over the NT compute threads (the producer warp is not in it)
template <int NT>
__device__ __forceinline__ void compute_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// mW: W (or W at t + dt/2) as a 4-D tensor (nx, ny, nz, 8 fields), box
// 40 x (TMA_TY + 1) x 1 x 3; mFm / mFb: the stage's fluxes as (nx, ny, nz,
// 21 = 3 axes x 7 fields), boxes 40 x (TMA_TY + 1) x 1 x 1 (mass flux) and
// x 2 (B fluxes).  F and
// W are the same arrays, read directly for the halo fix-ups.  One box
// (B.b[0]); grid = min(resident blocks, tiles), persistent over the tiles.
//
// The jobs of a block, in order: for each of its tiles (blockIdx.x,
// + gridDim.x, ...) the planes q = 0 .. nq - 1 (q = 0: the plane below the
// tile).  Job j fills slot j % TMA_SLOTS: the producer warp waits until the
// slot is empty (use j / TMA_SLOTS - 1 released), then arms full[slot] with
// the plane's bytes and issues its copies.  The compute threads wait for
// full[slot], put in the halo fix-ups and the reference field, compute the
// edges of the plane from it and the previous slot, then release the
// previous slot (one arrival per compute warp on empty[slot]).
template <class R>
__global__ void __launch_bounds__(EMF_TMA_THREADS)
    k_emf_tma(Boxes B, const __grid_constant__ CUtensorMap mW, const __grid_constant__ CUtensorMap mFm,
              const __grid_constant__ CUtensorMap mFb, const R* __restrict__ F, const R* __restrict__ W,
              R* __restrict__ E, unsigned* __restrict__ err)
{
    static_assert(sizeof(R) == 4, "the staged planes are laid out for 4-byte values");
    using L = TmaPlane<TMA_TY>;
    constexpr int NT = L::THREADS;
    extern __shared__ unsigned char smem_raw[];
    R* sm = reinterpret_cast<R*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    unsigned long long* full = reinterpret_cast<unsigned long long*>(sm + TMA_SLOTS * L::SLOT);
    unsigned long long* empty = full + TMA_SLOTS;
    const BoxDev g = B.b[0];
    const long long N = B.N;
    const int tid = threadIdx.x;
    const int ntx = (g.nx + ETX - 1) / ETX, nty = (g.ny + TMA_TY - 1) / TMA_TY, ntz = (g.nz + EZC - 1) / EZC;
    const int ntile = ntx * nty * ntz;
    auto tile_of = [&](int t, int& x0, int& y0, int& z0, int& nq) {
        x0 = (t % ntx) * ETX;
        const int r = t / ntx;
        y0 = (r % nty) * TMA_TY;
        z0 = (r / nty) * EZC;
        nq = (z0 + EZC < g.nz ? z0 + EZC : g.nz) - z0 + 1;
    };
    // the plane of job q of a tile (at a lower z boundary, q = 0 is the one
    // -1 maps to)
    auto plane_of = [&](int z0, int q) { return q == 0 ? bidx(z0 - 1, g.nz, g.bc & 4) : z0 - 1 + q; };

    if (tid == 0) {
        for (int s = 0; s < TMA_SLOTS; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NT / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();
    bool live = true;

    if (tid >= NT) {
        // producer warp: lane 0 issues every job of the block
        if (tid != NT) return;
        long long p = 0;
        for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
            int x0, y0, z0, nq;
            tile_of(t, x0, y0, z0, nq);
            const int xs = x0 - 4, ys = y0 - 1;
            for (int q = 0; q < nq; q++, p++) {
                const int s = (int)(p % TMA_SLOTS);
                if (p >= TMA_SLOTS) mbar_wait_bounded(&empty[s], (unsigned)((p / TMA_SLOTS - 1) & 1), err, 1, live);
                const int kk = plane_of(z0, q);
                R* P = sm + s * L::SLOT;
                unsigned long long* b = &full[s];
                mbar_arrive_expect_tx(b, L::BYTES);
                tma_load_4d(P + L::V, &mW, xs, ys, kk, 1, b);      // v: W 1-3
                tma_load_4d(P + L::B, &mW, xs, ys, kk, 5, b);      // B: W 5-7
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    tma_load_4d(P + L::FM0 + d * L::FAX, &mFm, xs, ys, kk, 7 * d, b);       // F_d 0
                    tma_load_4d(P + L::FB0 + d * L::FAX, &mFb, xs, ys, kk, 7 * d + 5, b);   // F_d 5-6
                }
            }
        }
        return;
    }

    const int tx = tid % ETX, ty = tid / ETX;      // edge cell of the threads tid < NT
    constexpr int o0 = L::off(0), o1 = L::off(1), o2 = L::off(2), o3 = L::off(3), o4 = L::off(4),
                  o5 = L::off(5), o6 = L::off(6), o7 = L::off(7), o8 = L::off(8), o9 = L::off(9),
                  o10 = L::off(10), o11 = L::off(11), o12 = L::off(12), o13 = L::off(13), o14 = L::off(14);
    long long j = 0;
    for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
        int x0, y0, z0, nq;
        tile_of(t, x0, y0, z0, nq);
        const bool mine = tid < NT && x0 + tx < g.nx && y0 + ty < g.ny;
        for (int q = 0; q < nq; q++, j++) {
            const int kk = plane_of(z0, q);
            const int s = (int)(j % TMA_SLOTS);
            R* P1 = sm + s * L::SLOT;
            mbar_wait_bounded(&full[s], (unsigned)((j / TMA_SLOTS) & 1), err, 0, live);
            if (x0 == 0 || y0 == 0) {
                // the lower x column / y row of a tile at the box's lower side
                // came in as fill values: put in the cells -1 maps to (periodic
                // wrap or outflow clamp), as k_emf stages them
                for (int h = tid; h < L::Y + ETX + 1; h += NT) {
                    int lx, ly;
                    if (h < L::Y) {
                        if (x0 != 0) continue;
                        lx = 3;
                        ly = h;
                    } else {
                        if (y0 != 0) continue;
                        lx = 3 + (h - L::Y);
                        ly = 0;
                    }
                    const int gi = bidx(x0 - 4 + lx, g.nx, g.bc & 1), gj = bidx(y0 - 1 + ly, g.ny, g.bc & 2);
                    const long long c = cell_of(g, gi, gj, kk);
                    const int o = ly * TMA_X + lx;
#pragma unroll
                    for (int f = 0; f < 3; f++) {
                        P1[L::off(f) + o] = W[(1 + f) * N + c];
                        P1[L::off(12 + f) + o] = W[(5 + f) * N + c];
                    }
#pragma unroll
                    for (int d = 0; d < 3; d++) {
                        const R* Fd = F + (long long)d * 7 * N;
                        P1[L::off(3 + 3 * d) + o] = Fd[c];
                        P1[L::off(4 + 3 * d) + o] = Fd[5 * N + c];
                        P1[L::off(5 + 3 * d) + o] = Fd[6 * N + c];
                    }
                }
                compute_sync<NT>();
            }
            // the reference field of the used cells (x0 - 1 .. x0 + 31 by the
            // plane's 17 rows), in place of the velocity
            for (int h = tid; h < (ETX + 1) * L::Y; h += NT) {
                const int o = (h / (ETX + 1)) * TMA_X + 3 + h % (ETX + 1);
                const R v0 = P1[o0 + o], v1 = P1[o1 + o], v2 = P1[o2 + o];
                const R b0 = P1[o12 + o], b1 = P1[o13 + o], b2 = P1[o14 + o];
                ref_field(v0, v1, v2, b0, b1, b2, P1[o0 + o], P1[o1 + o], P1[o2 + o]);
            }
            // this thread's generic writes to the slot come before the
            // copies that will refill it
            fence_proxy_async_smem();
            compute_sync<NT>();
            if (q > 0 && mine) {
                const int k = z0 - 1 + q;
                const R* P0 = sm + (int)((j - 1) % TMA_SLOTS) * L::SLOT;
                const long long c = cell_of(g, x0 + tx, y0 + ty, k);
                const int o = (ty + 1) * TMA_X + tx + 4;
                // Ex: a = y, b = z.  c01 = y-1, c10 = z-1
                {
                    const R* X1 = P1 + o0; const R* X0 = P0 + o0;
                    R ea0 = -P0[o7 + o], ea1 = -P1[o7 + o];                  // -F_y[B_z]
                    R eb0 = P1[o11 + o - TMA_X], eb1 = P1[o11 + o];          //  F_z[B_y]
                    R fa0 = P0[o6 + o], fa1 = P1[o6 + o];
                    R fb0 = P1[o9 + o - TMA_X], fb1 = P1[o9 + o];
                    E[c] = edge_e(X1 + o, X1 + o - TMA_X, X0 + o, X0 + o - TMA_X, ea0, ea1, eb0, eb1, fa0, fa1, fb0,
                                  fb1);
                }
                // Ey: a = z, b = x.  c01 = z-1, c10 = x-1
                {
                    const R* Y1 = P1 + o1; const R* Y0 = P0 + o1;
                    R ea0 = -P1[o10 + o - 1], ea1 = -P1[o10 + o];            // -F_z[B_x]
                    R eb0 = P0[o5 + o], eb1 = P1[o5 + o];                    //  F_x[B_z]
                    R fa0 = P1[o9 + o - 1], fa1 = P1[o9 + o];
                    R fb0 = P0[o3 + o], fb1 = P1[o3 + o];
                    E[N + c] = edge_e(Y1 + o, Y0 + o, Y1 + o - 1, Y0 + o - 1, ea0, ea1, eb0, eb1, fa0, fa1, fb0, fb1);
                }
                // Ez: a = x, b = y.  c01 = x-1, c10 = y-1
                {
                    const R* Z1 = P1 + o2;
                    R ea0 = -P1[o4 + o - TMA_X], ea1 = -P1[o4 + o];          // -F_x[B_y]
                    R eb0 = P1[o8 + o - 1], eb1 = P1[o8 + o];                //  F_y[B_x]
                    R fa0 = P1[o3 + o - TMA_X], fa1 = P1[o3 + o];
                    R fb0 = P1[o6 + o - 1], fb1 = P1[o6 + o];
                    E[2 * N + c] = edge_e(Z1 + o, Z1 + o - 1, Z1 + o - TMA_X, Z1 + o - 1 - TMA_X, ea0, ea1, eb0, eb1,
                                          fa0, fa1, fb0, fb1);
                }
            }
            // done with the previous slot (read as P0 above, or not at all on
            // a tile's first plane): one arrival per compute warp releases it
            if (j > 0) {
                __syncwarp();
                if ((tid & 31) == 0) mbar_arrive(&empty[(j - 1) % TMA_SLOTS]);
            }
        }
    }
}

}  // namespace mhd
