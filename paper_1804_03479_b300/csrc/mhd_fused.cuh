// mhd_fused.cuh -- fused kernels of the step: the VL predictor (Sec. 3.2,
// VL steps 1-3) as one kernel, and the edge fields fused with the half or
// full update that uses them (k_emf_update, after the file's first kernel;
// an opt-in form).
//
// The first-order fluxes of the three axes (the face B_n in the Riemann
// problem), the upwinded corner edge fields (Eqs. 13-14) and the dt/2 update
// of the face field and the cell state with the half-step primitives, for a
// tile of PX x PY cells of an x-y slab marched along z through shared memory.
// At step q of a tile (z plane p = z0 - 1 + q; every plane is staged with a
// one-cell halo ring by cp.async while the plane before it is computed):
//   fluxes   F_x and F_y of plane p on every face the tile's edges and cells
//            use, F_z at the level p - 1/2 (between the planes p-1 and p);
//   edges    E_z of plane p, E_x and E_y at the level p - 1/2;
//   update   the cells of plane p - 1, whose fluxes and edge fields are then
//            all in shared memory: Bh and Wh are written, nothing else.
// The predictor's fluxes and edge fields never reach HBM: the kernel reads W,
// the face field and the state once and writes Bh and Wh once, where the
// three sweeps, k_emf and k_half move 21 flux values and 3 edge values per
// cell out and back.  The faces of the halo ring are solved by both tiles
// that use them: per cell 5/PX + 5/PY + 5/FZ Riemann solves beyond the
// method's three (about a third more).  Measured on the B300 at 256^3 FP32
// it ties the five kernels it replaces (1.87 against 1.85 ms with Roe;
// issue-bound at 58 % of cycles, 16 resident warps per SM, barrier stalls
// between its phases; 32 x 16 tiles at one block per SM the same), so it is
// an opt-in form (pencil-mask bit 3).
//
// Shared memory (one block):
//   sB  [3 planes][3][HP]  face field B_d at the lower faces (type TE)
//   sW  [3 planes][8][HP]  primitives
//   sFx [2 planes][7][NFX] x fluxes: faces i in [x0, x0+PX], rows j in [y0-1, y0+PY]
//   sFy [2 planes][7][NFY] y fluxes: cells i in [x0-1, x0+PX], faces j in [y0, y0+PY]
//   sFz [2 levels][7][HP]  z fluxes of every cell of the halo'd plane
//   sEz [2 planes][NEZ]    E_z at i in [x0, x0+PX], j in [y0, y0+PY]
//   sEx [2 levels][NEX]    E_x at i in [x0, x0+PX), j in [y0, y0+PY]
//   sEy [2 levels][NEY]    E_y at i in [x0, x0+PX], j in [y0, y0+PY)
// Periodic boxes only (contexts with an outflow axis keep the sweeps).
#pragma once
#include "mhd_kernels.cuh"

#ifndef MHD_PRED_FZ
#define MHD_PRED_FZ 32
#endif

namespace mhd {

constexpr int PX = 32, PY = 8;            // tile extent along x and y (cells)
constexpr int PRED_FZ = MHD_PRED_FZ;      // planes of a tile along z
constexpr int PRED_THREADS = 256;
constexpr int PHX = PX + 2, PHY = PY + 2, PHP = PHX * PHY;   // the halo'd plane
constexpr int NFX = (PX + 1) * (PY + 2);
constexpr int NFY = (PX + 2) * (PY + 1);
constexpr int NEZ = (PX + 1) * (PY + 1);
constexpr int NEX = PX * (PY + 1);
constexpr int NEY = (PX + 1) * PY;

__host__ __device__ __forceinline__ int pred_tiles_of_box(int nx, int ny, int nz, int fz)
{
    return ((nx + PX - 1) / PX) * ((ny + PY - 1) / PY) * ((nz + fz - 1) / fz);
}

// byte offsets of the shared arrays (the TE array first: 8-byte aligned)
template <class R, class TE>
struct PredSmem {
    static constexpr size_t b = 0;
    static constexpr size_t w = b + (size_t)9 * PHP * sizeof(TE);
    static constexpr size_t fx = w + (size_t)24 * PHP * sizeof(R);
    static constexpr size_t fy = fx + (size_t)14 * NFX * sizeof(R);
    static constexpr size_t fz = fy + (size_t)14 * NFY * sizeof(R);
    static constexpr size_t ez = fz + (size_t)14 * PHP * sizeof(R);
    static constexpr size_t ex = ez + (size_t)2 * NEZ * sizeof(R);
    static constexpr size_t ey = ex + (size_t)2 * NEX * sizeof(R);
    static constexpr size_t bytes = ey + (size_t)2 * NEY * sizeof(R);
};

__device__ __forceinline__ int box_of_ftile(const Boxes& B, int t)
{
    int lo = 0, hi = B.nbox - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (B.b[mid].ftile0 <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// one element global -> shared without a register round trip (cp.async; the
// 4- and 8-byte forms need only the element's own alignment)
template <class T>
__device__ __forceinline__ void cp_async_el(T* dst, const T* src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// the reference field -(v x B) of the staged cell h (plane arrays Wp)
template <class R>
__device__ __forceinline__ void ref_of(const R* Wp, int h, R& e0, R& e1, R& e2)
{
    ref_field(Wp[PHP + h], Wp[2 * PHP + h], Wp[3 * PHP + h], Wp[5 * PHP + h], Wp[6 * PHP + h], Wp[7 * PHP + h], e0,
              e1, e2);
}

template <class R, class TU, class TE, int SOLVER>
__global__ void __launch_bounds__(PRED_THREADS, (sizeof(R) == 4 ? 2 : 1))
k_vl_predictor(Boxes B, StateP<TU, TE> s, const R* __restrict__ W, const DtBox* __restrict__ dtb, double gam,
               TE* __restrict__ Bh0, TE* __restrict__ Bh1, TE* __restrict__ Bh2, R* __restrict__ Wh,
               double pfloor)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using SM = PredSmem<R, TE>;
    TE* const sB = reinterpret_cast<TE*>(smem_raw + SM::b);
    R* const sW = reinterpret_cast<R*>(smem_raw + SM::w);
    R* const sFx = reinterpret_cast<R*>(smem_raw + SM::fx);
    R* const sFy = reinterpret_cast<R*>(smem_raw + SM::fy);
    R* const sFz = reinterpret_cast<R*>(smem_raw + SM::fz);
    R* const sEz = reinterpret_cast<R*>(smem_raw + SM::ez);
    R* const sEx = reinterpret_cast<R*>(smem_raw + SM::ex);
    R* const sEy = reinterpret_cast<R*>(smem_raw + SM::ey);
    const long long N = B.N;
    const int tid = threadIdx.x;
    const R gr = R(gam), gm1 = R(gam - 1.0);
    for (int tile = blockIdx.x; tile < B.nftile; tile += gridDim.x) {
        const int bi = box_of_ftile(B, tile);
        const BoxDev g = B.b[bi];
        const int ntx = (g.nx + PX - 1) / PX, nty = (g.ny + PY - 1) / PY;
        int bl = tile - g.ftile0;
        const int x0 = (bl % ntx) * PX;
        bl /= ntx;
        const int y0 = (bl % nty) * PY;
        const int z0 = (bl / nty) * B.fz;
        const int z1 = z0 + B.fz < g.nz ? z0 + B.fz : g.nz;
        const int nq = z1 - z0 + 2;              // steps: planes z0-1 .. z1
        const TE r = DtOf<TE>::hdtdx(dtb[bi]);
        const TU ru = DtOf<TU>::hdtdx(dtb[bi]);
        // stage plane z0 - 1 + qq (wrapped) into ring slot qq % 3
        auto stage = [&](int qq) {
            const int kk = wrapi(z0 - 1 + qq, g.nz);
            R* dW = sW + (qq % 3) * 8 * PHP;
            TE* dB = sB + (qq % 3) * 3 * PHP;
            for (int h = tid; h < PHP; h += PRED_THREADS) {
                const int hy = h / PHX, hx = h - hy * PHX;
                const long long c = cell_of(g, wrapi(x0 - 1 + hx, g.nx), wrapi(y0 - 1 + hy, g.ny), kk);
#pragma unroll
                for (int f = 0; f < 8; f++) cp_async_el(dW + f * PHP + h, W + f * N + c);
#pragma unroll
                for (int d = 0; d < 3; d++) cp_async_el(dB + d * PHP + h, s.b[d] + c);
            }
            cp_async_commit();
        };
        __syncthreads();                         // the previous tile's reads of every slot are done
        stage(0);
        for (int q = 0; q < nq; q++) {
            cp_async_wait_all();
            __syncthreads();                     // plane q staged; step q-1 finished with its slots
            if (q + 1 < nq) stage(q + 1);
            const R* Wc = sW + (q % 3) * 8 * PHP;            // plane q
            const R* Wb = sW + ((q + 2) % 3) * 8 * PHP;      // plane q - 1
            const TE* Bc = sB + (q % 3) * 3 * PHP;
            // ---- fluxes: F_x, F_y of plane q; F_z at its lower level (q >= 1)
            {
                R* Fx = sFx + (q & 1) * 7 * NFX;
                R* Fy = sFy + (q & 1) * 7 * NFY;
                R* Fz = sFz + (q & 1) * 7 * PHP;
                const int nit = q == 0 ? NFX + NFY : NFX + NFY + PHP;
                for (int it = tid; it < nit; it += PRED_THREADS) {
                    int ax, hl, hr, stride;
                    R* dst;
                    const R* WL = Wc;
                    if (it < NFX) {                   // x face i - 1/2 of row j: cells i-1, i
                        const int jy = it / (PX + 1), ix = it - jy * (PX + 1);
                        hl = jy * PHX + ix;
                        hr = hl + 1;
                        ax = 0;
                        dst = Fx + it;
                        stride = NFX;
                    } else if (it < NFX + NFY) {      // y face j - 1/2 of column i: cells j-1, j
                        const int t = it - NFX;
                        const int jy = t / (PX + 2), ix = t - jy * (PX + 2);
                        hl = jy * PHX + ix;
                        hr = hl + PHX;
                        ax = 1;
                        dst = Fy + t;
                        stride = NFY;
                    } else {                          // z face below cell h: planes q-1, q
                        const int t = it - NFX - NFY;
                        hl = hr = t;
                        ax = 2;
                        WL = Wb;
                        dst = Fz + t;
                        stride = PHP;
                    }
                    const int t1 = ax == 2 ? 0 : ax + 1, t2 = ax == 0 ? 2 : ax - 1;
                    R wl[7], wr[7], f[7];
                    wl[0] = WL[hl];                  wr[0] = Wc[hr];
                    wl[1] = WL[(1 + ax) * PHP + hl]; wr[1] = Wc[(1 + ax) * PHP + hr];
                    wl[2] = WL[(1 + t1) * PHP + hl]; wr[2] = Wc[(1 + t1) * PHP + hr];
                    wl[3] = WL[(1 + t2) * PHP + hl]; wr[3] = Wc[(1 + t2) * PHP + hr];
                    wl[4] = WL[4 * PHP + hl];        wr[4] = Wc[4 * PHP + hr];
                    wl[5] = WL[(5 + t1) * PHP + hl]; wr[5] = Wc[(5 + t1) * PHP + hr];
                    wl[6] = WL[(5 + t2) * PHP + hl]; wr[6] = Wc[(5 + t2) * PHP + hr];
                    riemann<SOLVER>(wl, wr, R(Bc[ax * PHP + hr]), gm1, gr, f);
#pragma unroll
                    for (int m = 0; m < 7; m++) dst[m * stride] = f[m];
                }
            }
            __syncthreads();
            // ---- edges: E_z of plane q (q < nq - 1), E_x and E_y at its lower level
            if (q >= 1) {
                const R* Fx1 = sFx + (q & 1) * 7 * NFX;
                const R* Fx0 = sFx + ((q - 1) & 1) * 7 * NFX;
                const R* Fy1 = sFy + (q & 1) * 7 * NFY;
                const R* Fy0 = sFy + ((q - 1) & 1) * 7 * NFY;
                const R* Fz1 = sFz + (q & 1) * 7 * PHP;
                R* Ez = sEz + (q & 1) * NEZ;
                R* Ex = sEx + (q & 1) * NEX;
                R* Ey = sEy + (q & 1) * NEY;
                const int nez = q < nq - 1 ? NEZ : 0;
                for (int it = tid; it < nez + NEX + NEY; it += PRED_THREADS) {
                    R c11, c01, c10, c00, u, v;
                    if (it < nez) {                   // E_z at (i-1/2, j-1/2): a = x, b = y
                        const int jy = it / (PX + 1), ix = it - jy * (PX + 1);
                        const int h = (jy + 1) * PHX + ix + 1;                 // cell (i, j)
                        ref_of(Wc, h, u, v, c11);
                        ref_of(Wc, h - 1, u, v, c01);
                        ref_of(Wc, h - PHX, u, v, c10);
                        ref_of(Wc, h - PHX - 1, u, v, c00);
                        const int a0 = jy * (PX + 1) + ix, a1 = a0 + (PX + 1);  // x faces of rows j-1, j
                        const int b0 = jy * (PX + 2) + ix, b1 = b0 + 1;         // y faces of columns i-1, i
                        Ez[it] = edge_e(&c11, &c01, &c10, &c00, -Fx1[5 * NFX + a0], -Fx1[5 * NFX + a1],
                                        Fy1[6 * NFY + b0], Fy1[6 * NFY + b1], Fx1[a0], Fx1[a1], Fy1[b0], Fy1[b1]);
                    } else if (it < nez + NEX) {      // E_x at (i, j-1/2, q-1/2): a = y, b = z
                        const int t = it - nez;
                        const int jy = t / PX, ix = t - jy * PX;
                        const int h = (jy + 1) * PHX + ix + 1;
                        ref_of(Wc, h, c11, u, v);
                        ref_of(Wc, h - PHX, c01, u, v);
                        ref_of(Wb, h, c10, u, v);
                        ref_of(Wb, h - PHX, c00, u, v);
                        const int a = jy * (PX + 2) + ix + 1;                   // y face (i, j-1/2)
                        Ex[t] = edge_e(&c11, &c01, &c10, &c00, -Fy0[5 * NFY + a], -Fy1[5 * NFY + a],
                                       Fz1[6 * PHP + h - PHX], Fz1[6 * PHP + h], Fy0[a], Fy1[a], Fz1[h - PHX],
                                       Fz1[h]);
                    } else {                          // E_y at (i-1/2, j, q-1/2): a = z, b = x
                        const int t = it - nez - NEX;
                        const int jy = t / (PX + 1), ix = t - jy * (PX + 1);
                        const int h = (jy + 1) * PHX + ix + 1;
                        ref_of(Wc, h, u, c11, v);
                        ref_of(Wb, h, u, c01, v);
                        ref_of(Wc, h - 1, u, c10, v);
                        ref_of(Wb, h - 1, u, c00, v);
                        const int a = (jy + 1) * (PX + 1) + ix;                 // x face (i-1/2, j)
                        Ey[t] = edge_e(&c11, &c01, &c10, &c00, -Fz1[5 * PHP + h - 1], -Fz1[5 * PHP + h],
                                       Fx0[6 * NFX + a], Fx1[6 * NFX + a], Fz1[h - 1], Fz1[h], Fx0[a], Fx1[a]);
                    }
                }
            }
            __syncthreads();
            // ---- update of plane q - 1 (z = z0 + q - 2)
            if (q >= 2) {
                const int qc = q - 1;
                const R* Fx0 = sFx + (qc & 1) * 7 * NFX;
                const R* Fy0 = sFy + (qc & 1) * 7 * NFY;
                const R* Fzl = sFz + (qc & 1) * 7 * PHP;
                const R* Fzu = sFz + (q & 1) * 7 * PHP;
                const R* Ez0 = sEz + (qc & 1) * NEZ;
                const R* Ex0 = sEx + (qc & 1) * NEX;
                const R* Ex1 = sEx + (q & 1) * NEX;
                const R* Ey0 = sEy + (qc & 1) * NEY;
                const R* Ey1 = sEy + (q & 1) * NEY;
                const TE* Bl = sB + (qc % 3) * 3 * PHP;
                const int k = z0 + q - 2;
                for (int u = tid; u < PX * PY; u += PRED_THREADS) {
                    const int jy = u / PX, ix = u - jy * PX;
                    const int i = x0 + ix, j = y0 + jy;
                    if (i >= g.nx || j >= g.ny) continue;
                    const int h = (jy + 1) * PHX + ix + 1;
                    const long long c = cell_of(g, i, j, k);
                    const TU rho0 = s.rho[c], mx0 = s.m[0][c], my0 = s.m[1][c], mz0 = s.m[2][c];
                    const TE e0 = s.e[c];
                    R fc[3][5], fn[3][5];
                    const int ax0 = (jy + 1) * (PX + 1) + ix, ay0 = jy * (PX + 2) + ix + 1;
#pragma unroll
                    for (int m = 0; m < 5; m++) {
                        fc[0][m] = Fx0[m * NFX + ax0];
                        fn[0][m] = Fx0[m * NFX + ax0 + 1];
                        fc[1][m] = Fy0[m * NFY + ay0];
                        fn[1][m] = Fy0[m * NFY + ay0 + PX + 2];
                        fc[2][m] = Fzl[m * PHP + h];
                        fn[2][m] = Fzu[m * PHP + h];
                    }
                    const int iz = jy * (PX + 1) + ix, ixe = jy * PX + ix;
                    R ec[3], en[3][3];
                    ec[0] = Ex0[ixe];
                    ec[1] = Ey0[iz];
                    ec[2] = Ez0[iz];
                    en[0][1] = Ex0[ixe + PX];
                    en[0][2] = Ex1[ixe];
                    en[1][0] = Ey0[iz + 1];
                    en[1][2] = Ey1[iz];
                    en[2][0] = Ez0[iz + 1];
                    en[2][1] = Ez0[iz + PX + 1];
                    en[0][0] = en[1][1] = en[2][2] = R(0);   // unused
                    const R e2xy = Ez0[iz + PX + 2], e1xz = Ey1[iz + 1], e0yz = Ex1[ixe + PX];
                    const TE blo[3] = {Bl[h], Bl[PHP + h], Bl[2 * PHP + h]};
                    const TE bhi[3] = {Bl[h + 1], Bl[PHP + h + PHX], Bc[2 * PHP + h]};
                    TE lo[3], bc[3];
                    half_faces<TE, R>(ec, en, e2xy, e1xz, e0yz, blo, bhi, r, lo, bc);
                    Bh0[c] = lo[0];
                    Bh1[c] = lo[1];
                    Bh2[c] = lo[2];
                    TU du[4];
                    TE due;
                    flux_divergence<R, TU, TE>(fc, fn, du, due);
                    R w[8];
                    half_prims<R, TU, TE>(rho0, mx0, my0, mz0, e0, du, due, ru, r, bc, gam, pfloor, w);
#pragma unroll
                    for (int f = 0; f < 8; f++) Wh[f * N + c] = w[f];
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The edge fields (Eqs. 13-14) fused with the update that uses them: the
// dt/2 update to B^{n+1/2} and the half-step primitives (HALF; VL steps 2-3,
// CTU steps 3-4), or the full update of U and B in place (VL steps 6-7, CTU
// steps 7-8).  The same tiles and z march as k_vl_predictor; per plane the
// halo'd cells' v, B and the mass and B fluxes of the three axes are staged
// by cp.async (ring of three planes), the edge fields go to shared memory
// and the cells of the plane below are updated with their fluxes read from
// F (the neighbours' from cache).  The edge fields never reach HBM, and F,
// W and the state are read once: 43 values per FP32 cell-update against 52
// for k_emf followed by k_half or k_full.  Periodic boxes; the in-place full
// update is race-free because a cell's update reads only its own state and
// its own lower faces (the edge fields come from F and W).
// It is an opt-in form (edge-field staging mode 2): at 256^3 on the B300 the
// corrector's pair takes 0.83 ms here against 0.74 ms for k_emf and k_full,
// which stream at close to the copy bandwidth with 64 resident warps per SM;
// this kernel keeps 24, issues about three times their instructions per
// cell (per-element copies, edge items) and waits at its plane barriers.
// ---------------------------------------------------------------------------
constexpr int EU_THREADS = 256;
static_assert(PX * PY == EU_THREADS, "k_emf_update: one updated cell per thread and plane");

// shared memory of k_emf_update: sF [3 planes][9][PHP] the mass flux and the
// two B fluxes of each axis (F_d components 0, 5, 6 at 3d + 0, 1, 2); sV
// [6][PHP] v and B of the plane being staged (each cell read back only by
// the thread that copied it); sR [3 planes][3][PHP] the reference field
// -(v x B) of every staged cell; the edge fields as in k_vl_predictor.
// (Copying two planes ahead, with a fourth flux slot and a second v, B slot,
// measured slower: two resident blocks per SM instead of three.)
template <class R>
constexpr size_t emf_update_smem_bytes()
{
    return ((size_t)(27 + 6 + 9) * PHP + 2 * (NEZ + NEX + NEY)) * sizeof(R);
}

template <class R, class TU, class TE, bool HALF>
__global__ void __launch_bounds__(EU_THREADS) k_emf_update(Boxes B, StateP<TU, TE> s, const R* __restrict__ F,
                                                           const R* __restrict__ W, const DtBox* __restrict__ dtb,
                                                           double gam, TE* __restrict__ Bh0, TE* __restrict__ Bh1,
                                                           TE* __restrict__ Bh2, R* __restrict__ Wh, double pfloor)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* const sF = reinterpret_cast<R*>(smem_raw);
    R* const sV = sF + 27 * PHP;
    R* const sR = sV + 6 * PHP;
    R* const sEz = sR + 9 * PHP;                               // [2][NEZ]
    R* const sEx = sEz + 2 * NEZ;                              // [2][NEX]
    R* const sEy = sEx + 2 * NEX;                              // [2][NEY]
    const long long N = B.N;
    const int tid = threadIdx.x;
    for (int tile = blockIdx.x; tile < B.nftile; tile += gridDim.x) {
        const int bi = box_of_ftile(B, tile);
        BoxDev g = B.b[bi];
        g.bc = 0;
        const int ntx = (g.nx + PX - 1) / PX, nty = (g.ny + PY - 1) / PY;
        int bl = tile - g.ftile0;
        const int x0 = (bl % ntx) * PX;
        bl /= ntx;
        const int y0 = (bl % nty) * PY;
        const int z0 = (bl / nty) * B.fz;
        const int z1 = z0 + B.fz < g.nz ? z0 + B.fz : g.nz;
        const int nq = z1 - z0 + 2;
        const TE r = HALF ? DtOf<TE>::hdtdx(dtb[bi]) : DtOf<TE>::dtdx(dtb[bi]);
        const TU ru = HALF ? DtOf<TU>::hdtdx(dtb[bi]) : DtOf<TU>::dtdx(dtb[bi]);
        // copy plane z0 - 1 + qq (wrapped): fluxes into slot qq % 3, v and B into sV
        auto stage = [&](int qq) {
            const int kk = wrapi(z0 - 1 + qq, g.nz);
            R* dF = sF + (qq % 3) * 9 * PHP;
            R* dV = sV;
            for (int h = tid; h < PHP; h += EU_THREADS) {
                const int hy = h / PHX, hx = h - hy * PHX;
                const long long c = cell_of(g, wrapi(x0 - 1 + hx, g.nx), wrapi(y0 - 1 + hy, g.ny), kk);
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    const R* Fd = F + (long long)d * 7 * N;
                    cp_async_el(dF + (3 * d) * PHP + h, Fd + c);
                    cp_async_el(dF + (3 * d + 1) * PHP + h, Fd + 5 * N + c);
                    cp_async_el(dF + (3 * d + 2) * PHP + h, Fd + 6 * N + c);
                }
                cp_async_el(dV + h, W + N + c);
                cp_async_el(dV + PHP + h, W + 2 * N + c);
                cp_async_el(dV + 2 * PHP + h, W + 3 * N + c);
                cp_async_el(dV + 3 * PHP + h, W + 5 * N + c);
                cp_async_el(dV + 4 * PHP + h, W + 6 * N + c);
                cp_async_el(dV + 5 * PHP + h, W + 7 * N + c);
            }
            cp_async_commit();
        };
        // the reference fields of the thread's own staged cells of plane qq,
        // from its own copies once they have landed (so no barrier before;
        // the next one publishes them)
        auto refs = [&](int qq) {
            cp_async_wait_all();
            const R* V = sV;
            R* dR = sR + (qq % 3) * 3 * PHP;
            for (int h = tid; h < PHP; h += EU_THREADS)
                ref_field(V[h], V[PHP + h], V[2 * PHP + h], V[3 * PHP + h], V[4 * PHP + h], V[5 * PHP + h], dR[h],
                          dR[PHP + h], dR[2 * PHP + h]);
        };
        // the cell this thread updates in every plane (PX * PY = EU_THREADS)
        const int ujy = tid / PX, uix = tid - ujy * PX;
        const int ui = x0 + uix, uj = y0 + ujy;
        const bool uown = ui < g.nx && uj < g.ny;
        __syncthreads();                         // the previous tile's reads of every slot are done
        stage(0);
        refs(0);
        for (int q = 0; q < nq; q++) {
            __syncthreads();                     // plane q staged with its reference fields; step q-1 done
            if (q + 1 < nq) stage(q + 1);
            // the update's operands of plane q - 1 from device memory, loaded
            // now so that they arrive while the edge fields are computed
            const bool upd = q >= 2 && uown;
            const int k = z0 + q - 2;
            long long c = 0;
            R fc[3][5], fn[3][5];
            TE bo[3], bhi[3];
            TU rho0 = TU(0), mx0 = TU(0), my0 = TU(0), mz0 = TU(0);
            TE e0 = TE(0);
            if (upd) {
                c = cell_of(g, ui, uj, k);
                const long long cp[3] = {nbr(g, ui, uj, k, 0, 1), nbr(g, ui, uj, k, 1, 1), nbr(g, ui, uj, k, 2, 1)};
#pragma unroll
                for (int d = 0; d < 3; d++)
#pragma unroll
                    for (int m = 0; m < 5; m++) {
                        fc[d][m] = F[((long long)d * 7 + m) * N + c];
                        fn[d][m] = F[((long long)d * 7 + m) * N + cp[d]];
                    }
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    bo[d] = s.b[d][c];
                    if (HALF) bhi[d] = s.b[d][cp[d]];
                }
                rho0 = s.rho[c];
                mx0 = s.m[0][c];
                my0 = s.m[1][c];
                mz0 = s.m[2][c];
                e0 = s.e[c];
            }
            // ---- edges: E_z of plane q (q < nq - 1), E_x and E_y at its lower level.
            // Items in rows of 32 (conflict-free shared loads): E_z at i < x0 + PX,
            // E_x, E_y at i < x0 + PX, then the column i = x0 + PX of E_z and E_y.
            if (q >= 1) {
                const R* F1 = sF + (q % 3) * 9 * PHP;
                const R* F0 = sF + ((q + 2) % 3) * 9 * PHP;
                const R* R1 = sR + (q % 3) * 3 * PHP;
                const R* R0 = sR + ((q + 2) % 3) * 3 * PHP;
                R* Ez = sEz + (q & 1) * NEZ;
                R* Ex = sEx + (q & 1) * NEX;
                R* Ey = sEy + (q & 1) * NEY;
                constexpr int EZM = PX * (PY + 1), EYM = PX * PY;        // 32-wide parts
                constexpr int NIT = EZM + NEX + EYM + (PY + 1) + PY;      // = NEZ + NEX + NEY
                const bool doz = q < nq - 1;                              // E_z of the last plane: unused
                const int nit = doz ? NIT : NIT - EZM - (PY + 1);
                for (int it0 = tid; it0 < nit; it0 += EU_THREADS) {
                    int it = it0;
                    if (!doz) it = it0 < NEX + EYM ? it0 + EZM : it0 - (NEX + EYM) + EZM + NEX + EYM + PY + 1;
                    int kind, ix, jy;
                    if (it < EZM) { kind = 0; jy = it / PX; ix = it - jy * PX; }
                    else if (it < EZM + NEX) { kind = 1; const int t = it - EZM; jy = t / PX; ix = t - jy * PX; }
                    else if (it < EZM + NEX + EYM) { kind = 2; const int t = it - EZM - NEX; jy = t / PX; ix = t - jy * PX; }
                    else if (it < EZM + NEX + EYM + PY + 1) { kind = 0; jy = it - (EZM + NEX + EYM); ix = PX; }
                    else { kind = 2; jy = it - (EZM + NEX + EYM + PY + 1); ix = PX; }
                    const int h = (jy + 1) * PHX + ix + 1;                    // cell (i, j) of the edge
                    if (kind == 0) {                  // E_z at (i-1/2, j-1/2): a = x, b = y
                        const R* Rz = R1 + 2 * PHP;
                        Ez[jy * (PX + 1) + ix] = edge_e(Rz + h, Rz + h - 1, Rz + h - PHX, Rz + h - PHX - 1,
                                                        -F1[PHP + h - PHX], -F1[PHP + h], F1[5 * PHP + h - 1],
                                                        F1[5 * PHP + h], F1[h - PHX], F1[h], F1[3 * PHP + h - 1],
                                                        F1[3 * PHP + h]);
                    } else if (kind == 1) {           // E_x at (i, j-1/2, q-1/2): a = y, b = z
                        Ex[jy * PX + ix] = edge_e(R1 + h, R1 + h - PHX, R0 + h, R0 + h - PHX, -F0[4 * PHP + h],
                                                  -F1[4 * PHP + h], F1[8 * PHP + h - PHX], F1[8 * PHP + h],
                                                  F0[3 * PHP + h], F1[3 * PHP + h], F1[6 * PHP + h - PHX],
                                                  F1[6 * PHP + h]);
                    } else {                          // E_y at (i-1/2, j, q-1/2): a = z, b = x
                        const R* Ry1 = R1 + PHP;
                        const R* Ry0 = R0 + PHP;
                        Ey[jy * (PX + 1) + ix] = edge_e(Ry1 + h, Ry0 + h, Ry1 + h - 1, Ry0 + h - 1,
                                                        -F1[7 * PHP + h - 1], -F1[7 * PHP + h], F0[2 * PHP + h],
                                                        F1[2 * PHP + h], F1[6 * PHP + h - 1], F1[6 * PHP + h],
                                                        F0[h], F1[h]);
                    }
                }
            }
            __syncthreads();
            // ---- update of plane q - 1 (z = z0 + q - 2)
            if (upd) {
                const int qc = q - 1;
                const R* Ez0 = sEz + (qc & 1) * NEZ;
                const R* Ex0 = sEx + (qc & 1) * NEX;
                const R* Ex1 = sEx + (q & 1) * NEX;
                const R* Ey0 = sEy + (qc & 1) * NEY;
                const R* Ey1 = sEy + (q & 1) * NEY;
                const int iz = ujy * (PX + 1) + uix, ixe = ujy * PX + uix;
                R ec[3], en[3][3];
                ec[0] = Ex0[ixe];
                ec[1] = Ey0[iz];
                ec[2] = Ez0[iz];
                en[0][1] = Ex0[ixe + PX];
                en[0][2] = Ex1[ixe];
                en[1][0] = Ey0[iz + 1];
                en[1][2] = Ey1[iz];
                en[2][0] = Ez0[iz + 1];
                en[2][1] = Ez0[iz + PX + 1];
                en[0][0] = en[1][1] = en[2][2] = R(0);   // unused
                TU du[4];
                TE due;
                flux_divergence<R, TU, TE>(fc, fn, du, due);
                if constexpr (HALF) {
                    const R e2xy = Ez0[iz + PX + 2], e1xz = Ey1[iz + 1], e0yz = Ex1[ixe + PX];
                    TE lo[3], bc[3];
                    half_faces<TE, R>(ec, en, e2xy, e1xz, e0yz, bo, bhi, r, lo, bc);
                    Bh0[c] = lo[0];
                    Bh1[c] = lo[1];
                    Bh2[c] = lo[2];
                    R w[8];
                    half_prims<R, TU, TE>(rho0, mx0, my0, mz0, e0, du, due, ru, r, bc, gam, pfloor, w);
#pragma unroll
                    for (int f = 0; f < 8; f++) Wh[f * N + c] = w[f];
                } else {
                    full_cell<R, TU, TE>(s, c, rho0, mx0, my0, mz0, e0, bo, du, due, ec, en, ru, r);
                }
            }
            if (q + 1 < nq) refs(q + 1);
        }
    }
}

}  // namespace mhd
