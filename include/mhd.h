/*
 * mhd.h -- C ABI of the B300 (sm_103a) ideal-MHD patch advance.
 *
 * The library advances the ideal-MHD equations (Eqs. 1-9 of "Magnetohydro-
 * dynamics with GAMER", Zhang, Schive & Chiueh 2018) on a periodic uniform
 * grid with dx = dy = dz (Sec. 3.1), using the unsplit VL or CTU scheme
 * with constrained transport (Sec. 3.2, Eqs. 10-16).  Every step runs in
 * hand-written CUDA kernels on the stream given at mhd_init.
 *
 * State layout (what mhd_set_state / mhd_get_state exchange), C order:
 *   U: 5 arrays of n = nx*ny*nz cell averages (Eq. 11), in the order
 *      rho, Mx, My, Mz, e; cell c = (k*ny + j)*nx + i, x fastest.
 *   B: 3 arrays of n face averages (Eq. 14): B[0][c] is Bx on the face
 *      x_{i-1/2} of cell c, B[1][c] is By on y_{j-1/2}, B[2][c] is Bz on
 *      z_{k-1/2}.  Periodic: the face x_{nx-1/2} is B[0] of cell i = 0.
 *   Element type: double for MHD_FP64 and MHD_MIXED, float for MHD_FP32.
 *
 * Errors: no call throws or aborts.  Every call returns an mhd_status;
 * mhd_last_error() gives a one-line description.  Kernels run
 * asynchronously; a device-side anomaly (rho <= 0 or P <= 0 at the start
 * of a step) is recorded on the device and reported as MHD_ENEGATIVE by
 * the next call that synchronises (mhd_cfl_dt, mhd_divB, mhd_sums,
 * mhd_get_state, mhd_sync).  An error stays until mhd_clear_error.
 *
 * Ownership: the library allocates the state and all scratch on the
 * device in mhd_init and frees them in mhd_free.  Pointers passed in are
 * only read or written during the call (copies are stream-ordered and
 * complete before the call returns when they touch host memory).
 * Thread safety: one context must not be used from two threads at once.
 */
#ifndef MHD_H
#define MHD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MHD_OK = 0,
    MHD_EINVAL = 1,        /* bad argument (size, enum, null pointer, dt)      */
    MHD_ENOMEM = 2,        /* device allocation failed                          */
    MHD_ECUDA = 3,         /* a CUDA runtime call failed                        */
    MHD_ENEGATIVE = 4,     /* rho <= 0 or P <= 0 (or not finite) in some cell   */
    MHD_ETIMEOUT = 5,      /* a bounded device wait gave up                     */
    MHD_EUNSUPPORTED = 6   /* combination not built                             */
} mhd_status;

enum { MHD_VL = 0, MHD_CTU = 1 };                     /* integrator, Sec. 3.2 */
enum { MHD_PLM = 0, MHD_PPM = 1, MHD_PLM_PRIM = 2 };  /* reconstruction: PLM / PPM in
                                                         characteristic variables;
                                                         PLM_PRIM = primitive-variable
                                                         PLM (VL only)            */
enum { MHD_ROE = 0, MHD_HLLD = 1, MHD_HLLE = 2 };     /* Riemann solver, Sec. 3.2 */
enum { MHD_FP64 = 0, MHD_FP32 = 1, MHD_MIXED = 2 };   /* MIXED: FP32 arithmetic and
                                                         rho, M storage; FP64 e, face B,
                                                         pressure recovery, CT and
                                                         energy accumulation       */

typedef struct {
    int nx, ny, nz;   /* cells per axis, each >= 1                        */
    double dx;        /* cell size, dx = dy = dz (Sec. 3.1)               */
} mhd_grid;

typedef struct {
    int integrator;   /* MHD_VL or MHD_CTU                                */
    int recon;        /* MHD_PLM, MHD_PPM, MHD_PLM_PRIM                   */
    int riemann;      /* MHD_ROE, MHD_HLLD, MHD_HLLE                      */
    int precision;    /* MHD_FP64, MHD_FP32, MHD_MIXED                    */
    double cfl;       /* Courant number for mhd_cfl_dt / mhd_advance      */
    double pfloor;    /* pressure floor, 0 = none (the paper's scheme has
                         none; > 0 raises e where P < pfloor at the start
                         of a step and floors the half-step P: not
                         conservative, counted by mhd_floor_count)        */
} mhd_scheme;

typedef struct mhd_ctx mhd_ctx;

/* Create a context for one periodic box: grid, adiabatic index gamma
 * (Eq. 5) and scheme.  stream is a cudaStream_t (NULL = a stream the
 * library creates).  Allocates the state and scratch on the current device.
 * On failure *out is NULL and the status says why. */
mhd_status mhd_init(const mhd_grid* grid, double gamma, const mhd_scheme* scheme, void* stream,
                    mhd_ctx** out);

/* Batch of independent periodic boxes (each its own grid and dt) advanced
 * together: every kernel of a step is one launch over all boxes, the face
 * sweeps run a persistent grid over the batch's tile list (tile shape set
 * by mhd_set_sweep_config or mhd_autotune).  mhd_init is the batch of one.
 * The paper advances many patch groups per GPU call (Sec. 4); here the
 * groups are whole boxes. */
mhd_status mhd_init_batch(int nbox, const mhd_grid* grids, double gamma, const mhd_scheme* scheme,
                          void* stream, mhd_ctx** out);
int mhd_nbox(mhd_ctx* ctx);

/* Copy the state of box `box` in (U: 5*n, B: 3*n elements of the layout
 * above, n the box's cell count).  on_device != 0: U, B are device
 * pointers; else host pointers.  mhd_set_state is box 0. */
mhd_status mhd_set_state_box(mhd_ctx* ctx, int box, const void* U, const void* B, int on_device);
mhd_status mhd_set_state(mhd_ctx* ctx, const void* U, const void* B, int on_device);

/* Copy the state of a box out (same layout); synchronises the stream. */
mhd_status mhd_get_state_box(mhd_ctx* ctx, int box, void* U, void* B, int on_device);
mhd_status mhd_get_state(mhd_ctx* ctx, void* U, void* B, int on_device);

/* CFL time step of every box (Sec. 3.2): dt[b] = cfl * dx_b / max over the
 * box's cells and axes of |v_d| + c_f,d, from the current state.
 * dt has nbox entries.  Synchronises. */
mhd_status mhd_cfl_dt(mhd_ctx* ctx, double* dt);

/* One step of the scheme (Sec. 3.2, CTU steps 1-8 or VL steps 1-7) with the
 * same dt > 0 for every box (mhd_step) or dt[b] per box (mhd_step_boxes).
 * Asynchronous. */
mhd_status mhd_step(mhd_ctx* ctx, double dt);
mhd_status mhd_step_boxes(mhd_ctx* ctx, const double* dt);

/* nsteps steps, each with every box's CFL dt computed and used on the
 * device (no host round trip).  Asynchronous.  With use_graph != 0 one step
 * is captured once into a CUDA graph and replayed. */
mhd_status mhd_advance(mhd_ctx* ctx, int nsteps, int use_graph);

/* dt of every box used by the most recent step (nbox entries).  Synchronises. */
mhd_status mhd_last_dt(mhd_ctx* ctx, double* dt);

/* Discrete divergence (Eq. 16) per box: maxabs[b] = max over the box's
 * cells of |sum_d B_d(c + e_d) - B_d(c)| (= max |div B| dx), brms[b] = rms
 * of the box's cell-centre field (nbox entries each).  Synchronises. */
mhd_status mhd_divB(mhd_ctx* ctx, double* maxabs, double* brms);

/* Sums per box (FP64, fixed-order reduction): rho, Mx, My, Mz, e over cells,
 * Bx, By, Bz over faces; sums8 has 8 * nbox entries.  Synchronises. */
mhd_status mhd_sums(mhd_ctx* ctx, double* sums8);

/* Diagnostics of Sec. 4.3 / 4.5 per box (FP64, fixed-order reduction), out
 * has 6 * nbox entries:
 *   [0] E_T = sum e dx^3            [1] U_B = sum over faces B_f^2/2 dx^3
 *   [2] U_V = sum |M|^2/(2 rho) dx^3
 *   [3] max over cells of dx |J| / |B|   (J = curl B: dx J on an edge is the
 *       circulation of the face B around it; the cell value is the mean of
 *       its four edges per axis, |B| the mean of its two faces per axis)
 *   [4] number of cells with dx |J| / |B| > jb_threshold (the refinement
 *       test |J|/|B| > thr / dx of the Orszag-Tang and ABC runs)
 *   [5] max over cells of |J|.
 * jb_threshold >= 0, else MHD_EINVAL.  Synchronises. */
mhd_status mhd_energies(mhd_ctx* ctx, double jb_threshold, double* out);

/* Pressure-gradient refinement indicator of the magnetised blast run
 * (Sec. 5.1) per box, in FP64 from the stored state: per cell
 * scale * |grad P| / P (scale = 100 r0 there), grad P by centred
 * differences of the cell pressure over 2 dx (cell-centre B the mean of the
 * two faces; a neighbour beyond an outflow side is the cell itself).  out
 * has (1 + nlev) * nbox entries: per box the maximum, then for l < nlev the
 * number of cells above thr * 2^l (the run refines to level n above
 * 1.25 * 2^(n-1)).  scale > 0, thr >= 0 and 1 <= nlev <= 4, else
 * MHD_EINVAL.  Uses the primitive scratch, which every step rewrites
 * before reading (the state is not touched).  Synchronises. */
mhd_status mhd_pressure_gradient(mhd_ctx* ctx, double scale, double thr, int nlev, double* out);

/* Magnetic helicity H = sum A.B dx^3 per box (Sec. 4.5; h has nbox entries),
 * of the cell-centre field (mean of the two faces per axis), with A in the
 * Coulomb gauge of the periodic box: A_k = i k x B_k / |k|^2 from the
 * discrete Fourier transform (cuFFT, FP64), the mean field carrying no A;
 * H by Parseval.  Uses the flux scratch (no state is touched); cuFFT
 * allocates its work area.  MHD_ENOMEM if a box's transform does not fit
 * the scratch (3n doubles + 3 half spectra).  Synchronises. */
mhd_status mhd_helicity(mhd_ctx* ctx, double* h);

/* Face-sweep tiling: tiles of 32 x tile_len faces (tile_len 4, 8 or 16),
 * blocks_per_sm x SMs persistent blocks.  mhd_autotune times every pair on
 * the context's own batch (reps steps each, the state restored after each
 * trial), and for the VL integrator also the pencil sweeps below (on all
 * axes or on y and z, segment lengths 8, 16, 32, with x by overlapping
 * warps, staged pencils or aligned marching warps, and with the fused
 * predictor where it applies); it keeps the fastest and
 * reports the tiling (ms per step in *ms_best; the pencil choice through
 * mhd_get_sweep_pencils).  The autotuner allocates a temporary copy of the
 * state. */
mhd_status mhd_set_sweep_config(mhd_ctx* ctx, int tile_len, int blocks_per_sm);
mhd_status mhd_get_sweep_config(mhd_ctx* ctx, int* tile_len, int* blocks_per_sm);
mhd_status mhd_autotune(mhd_ctx* ctx, int reps, int* tile_len, int* blocks_per_sm, double* ms_best);

/* Boundaries.  Every axis is periodic by default.  mhd_set_boundary makes
 * the axes of the bits of outflow_mask (bit d: axis d) outflow boundaries
 * (zero gradient): a cell, face or edge beyond the last one is the last one,
 * and the flux through the outer face of the last cell is the Riemann flux
 * between that cell and its copy (for CTU, of the cell's own upper and
 * lower traced states, corrected in the second stage); CT then keeps the
 * divergence of every cell.  One-box contexts (VL or CTU) without a selector
 * (else MHD_EUNSUPPORTED); outflow_mask in [0, 7] (else MHD_EINVAL).
 * mhd_helicity needs a periodic box. */
mhd_status mhd_set_boundary(mhd_ctx* ctx, int outflow_mask);
mhd_status mhd_get_boundary(mhd_ctx* ctx, int* outflow_mask);

/* Dirichlet sides (the shock tubes of Sec. 5.1 hold the left and right
 * states at the ends of the box), held as ghost layers inside the box: the
 * nlayers outermost cells at each end of `axis` are put back to a fixed
 * state when the call is made, after every mhd_set_state and after every
 * step, and the axis becomes an outflow axis (the outflow rule holds beyond
 * the layers).  w_lo, w_hi: 8 doubles each, (rho, vx, vy, vz, P, Bx, By, Bz)
 * in box axes, for the lower and upper end (host memory, copied).  A ghost
 * cell gets the conserved state of w and its three lower faces the field of
 * w, except the lower face along `axis` of the first upper ghost cell: that
 * is the interior's upper boundary face, which CT advances.  With nlayers
 * >= 2 (VL with PPM: >= 3) the interior sees an unbounded region of the
 * fixed state; fewer is MHD_EINVAL, as is 2 nlayers >= the cells along
 * `axis`, rho <= 0, P <= 0 or a non-finite value.  nlayers = 0 removes the
 * side (the axis stays outflow).  One-box contexts (VL or CTU) without a
 * selector (else MHD_EUNSUPPORTED).  mhd_set_boundary with the axis's bit
 * cleared removes the side too.  mhd_get_dirichlet reports nlayers. */
mhd_status mhd_set_dirichlet(mhd_ctx* ctx, int axis, int nlayers, const double* w_lo, const double* w_hi);
mhd_status mhd_get_dirichlet(mhd_ctx* ctx, int axis, int* nlayers);

/* Pencil sweeps: on every axis d with bit d of pencil_mask set, the face
 * sweeps (VL predictor and corrector; CTU tracing sweeps) keep the cells
 * around each face in registers (no shared memory): one thread walks a
 * segment of pencil_len consecutive faces of a grid line.  For CTU the bits
 * also select the register forms of the transverse correction and corrector
 * solve (pencils on y and z, warps on a periodic x; each cell's transverse
 * flux differences loaded once for both of its traced states).  The x axis runs by warps instead (VL; CTU
 * where x is periodic, else by tiles): the 32 lanes of a warp hold 32
 * consecutive cells of a row and exchange neighbour states by shuffles (27
 * to 31 faces per warp).  The results are those of the tile sweeps (the
 * same arithmetic per face).
 * Bit 3 (VL, every box periodic, no learned selector; ignored otherwise):
 * the predictor (Sec. 3.2, VL steps 1-3: first-order fluxes with the face
 * B_n on all three axes, the corner edge fields of Eqs. 13-14 and the dt/2
 * update to B^{n+1/2} and the half-step primitives) runs as one kernel that
 * marches z planes of 32 x 8-cell tiles through shared memory; the
 * predictor's fluxes and edge fields then never leave the chip, and the
 * step is 8 launches instead of 12.  The faces of each tile's one-cell halo
 * ring are solved by both tiles that use them (the same arithmetic): about
 * a third more Riemann solves, which with the plane barriers cost what the
 * traffic saves -- on the B300 at 256^3 FP32 it ties the sweeps, k_emf and
 * k_half it replaces (1.87 against 1.85 ms with Roe, 32 x 16 tiles the
 * same), so it is not a default.
 * Bit 4 with bit 0 (VL without a learned selector; ignored otherwise): x
 * runs by pencils as y and z do -- the lanes of a warp walk 32 consecutive
 * grid rows, one segment of pencil_len faces each -- with the cells and
 * the fluxes passing through per-warp shared-memory chunks of 4 cells x 32
 * rows, so that the loads and stores along the contiguous x rows stay
 * coalesced; one reconstruction per face and no register shuffles.  In
 * FP64 that runs x at the y and z rate (at 256^3: 27.7 against 30.3 ms for
 * the corrector by warps); in FP32 arithmetic the staging sets the pace and
 * the warps are faster (0.62 against 1.8 ms).
 * Bits 5 and 6 with bit 0 (VL; ignored otherwise and where bit 4 applies): the x predictor (bit 5) and the PLM x corrector
 * (bit 6; the PPM corrector keeps its warps) run by aligned marching warps:
 * one warp per row, lane l of segment s on cell 32 s + l, every lane
 * producing a face, the neighbours across a segment's ends from the
 * previous segment's registers and the next segment's prefetch (the
 * overlapping warps above produce 27 to 31 faces per 32 lanes from loads
 * that start off a line boundary; FP32 predictor rows of whole aligned
 * segments stream three segments per warp through shared memory by
 * asynchronous copies).  At 256^3 FP32 the predictor takes 0.27 ms where the
 * overlapping warps take 0.45 (Roe), the PLM corrector 0.51 / 0.51 / 0.44 ms
 * against 0.62 / 0.57 / 0.50 (Roe / HLLD / HLLE).  With a
 * learned selector the cheap x sweep marches every face and the full
 * scheme's x-warp items, launched after it, overwrite theirs.
 * For CTU, bit 5 with bit 0 runs the PLM tracing along a periodic x (CTU
 * steps 1-2: the traced states with their dB_n/dn source, and their fluxes)
 * by the same aligned march: at 256^3 FP32 0.64 ms where the overlapping
 * warps take 0.81 (Roe); the PPM tracing and the transverse correction keep
 * their warps.
 * Bit 7 with bit 1 (VL, every box periodic, no
 * learned selector, bit 3 clear and the edge fields as their own kernel;
 * ignored otherwise): the half update (Sec. 3.2, VL step 3: B^{n+1/2} by
 * Eq. 13, U^{n+1/2} by Eq. 10 with dt/2, and its primitives) runs inside
 * the corrector's y pencils: each pencil thread forms the half-step state
 * of every cell its walk reconstructs (its segment's cells, two lead-in
 * cells and one past its end), stores the half-step primitives and faces
 * of the cells it owns and solves its y faces; the x and z correctors
 * follow.  The half update's loads then overlap the corrector's arithmetic
 * (256^3 FP32 PLM + Roe: 0.708 ms for what the two kernels take 0.439 +
 * 0.475; PPM + Roe: step 4.86 -> 4.71 ms)
 * and the step is 11 launches.  The corrector's fluxes go to a second flux
 * array (21 values per cell in the arithmetic type), allocated on first
 * use (MHD_ENOMEM if that fails).  The states agree with the separate
 * kernels' to rounding.
 * Bit 8 with bit 1 (VL, every box periodic, no learned selector, no
 * pressure floor, bit 3 clear; ignored otherwise): the primitives at t^n
 * (Eq. 5) and the CFL signal speeds (Sec. 3.2) are formed inside the
 * predictor's y pencils (each thread: its segment's cells and one lead-in
 * cell; it stores its own cells' primitives and folds their signal speeds
 * into the box's maximum), one launch fewer.  It pays in the mixed form,
 * whose FP64 primitive arithmetic then overlaps the sweep (256^3 PLM +
 * Roe: 0.718 ms against 0.644 + 0.307); in FP32 and FP64 it ties the two
 * kernels.
 * Bit 9 with bit 2 (VL, every box periodic, bit 3 clear, the edge fields as
 * their own kernel; with a learned selector and bit 7 as well, its cheap
 * PLM z corrector, which runs after the full z list pass and reads the
 * marked segments' faces; ignored otherwise):
 * the conservative part of the full update (Eq. 10 for rho, M
 * and e with dt) runs inside the corrector's z pencils, the last corrector
 * sweep: each thread updates the cells of its segment in place once it has
 * solved their lower and upper z faces (pl + 1 faces a segment), from the x
 * and y corrector fluxes and its own z fluxes, and stores only the three z
 * flux components the edge fields read; after the edge fields the face
 * field advances by CT (Eq. 13) in a kernel that reads only E and B.  At
 * 256^3 FP32 Roe the step takes 3.58 ms against 3.67.
 * For CTU, bit 7 with bit 1 (every box periodic, the edge fields as their
 * own kernel) runs the dt/2 update (Sec. 3.2, CTU steps 3-4) inside the y
 * pencils of the transverse correction and corrector solve: each thread
 * forms the half-step state of its segment's cells, stores their half-step
 * primitives and faces and corrects its y faces with the cells' half-step
 * normal field; the x and z corrections follow (256^3 FP32 PLM + Roe: 5.32
 * -> 5.22 ms; mixed 7.11 -> 6.79).  For CTU, bit 9 with bit 2 (the same
 * conditions) runs the conservative update inside the z pencils of the
 * transverse correction, as for VL (FP32: 5.23 -> 5.18 ms).
 * pencil_mask in [0, 1023] (0: tiles everywhere), pencil_len in [1, 1024],
 * else MHD_EINVAL.  Defaults (pencil_len 32): VL FP64 23; VL FP32 743; VL
 * mixed 487 with PLM, 359 with PPM; CTU FP32 679, mixed 167, FP64 39. */
mhd_status mhd_set_sweep_pencils(mhd_ctx* ctx, int pencil_mask, int pencil_len);
mhd_status mhd_get_sweep_pencils(mhd_ctx* ctx, int* pencil_mask, int* pencil_len);

/* Staging of the edge-field kernel (Sec. 2, Eqs. 13-14; the corner-averaged
 * edge fields of both stages).  mode 2: the edge fields are
 * computed by the kernel of the update that uses them (the dt/2 update to
 * B^{n+1/2} with the half-step primitives, or the full update): tiles of
 * 32 x 8 cells march along z, each plane's v, B and mass and B fluxes are
 * staged in shared memory by asynchronous copies, the edge fields stay in
 * shared memory and the cells below are updated from them, so the edge
 * fields never pass through device memory and the step has one launch
 * fewer per stage.  That needs periodic boxes; elsewhere mode 2 runs as mode
 * 0.  It moves 43 values per FP32 cell-update against 52, but on the B300
 * it is the slower form (0.86 against 0.74 ms for the corrector's edge
 * fields and full update at 256^3): with 16 resident warps per SM it issues
 * about three times the instructions of the two separate kernels and
 * waits on its plane barriers, where the separate kernels stream at close
 * to the copy bandwidth.  mode 0 (the default): a separate
 * edge-field kernel in which each thread loads its staged cell of every
 * plane (32 x 16 cells per block, two blocks per SM), then the update
 * kernel.  mode 1: the planes of that separate kernel are staged by the
 * tensor memory accelerator where the context allows it -- bulk tensor
 * copies of whole field planes into a ring of three shared-memory plane
 * slots per block (32 x 8 cells, three blocks per SM), refilled by a
 * producer warp while the block computes.  That needs one box, FP32 or
 * MIXED precision, nx a multiple of 4, nx >= 40 and ny >= 9; elsewhere
 * mode 1 runs as mode 0.  Modes 0 and 1 give the same edge fields bit for
 * bit; on the B300 the per-thread form is the faster of the two (0.30
 * against 0.45 ms per launch at 256^3).  mode in {0, 1, 2}, else
 * MHD_EINVAL.  mhd_get_emf_staging reports the requested mode and the form
 * in use (active: 0 separate kernel with per-thread loads, 1 tensor copies,
 * 2 fused with the update).  A plane wait of the tensor-copy form that
 * gives up (after about 2 s) sets a device flag (bit 0: a consumer's wait
 * for a filled slot, bit 1: the producer's wait for a free one), and the
 * next call that reads the device flags (mhd_sync, mhd_cfl_dt, mhd_divB,
 * mhd_sums, mhd_get_state, ...) returns MHD_ETIMEOUT until
 * mhd_clear_error. */
mhd_status mhd_set_emf_staging(mhd_ctx* ctx, int mode);
mhd_status mhd_get_emf_staging(mhd_ctx* ctx, int* mode, int* active);

/* Wait for all work queued on the context's stream; reports recorded
 * device-side anomalies. */
mhd_status mhd_sync(mhd_ctx* ctx);

/* Kernel-group timing.  mhd_profile_begin arms CUDA events (on the
 * context's stream) at the boundaries of the 11 kernel groups of each of
 * the next max_steps directly launched steps (not graph replays):
 * 0 primitives + CFL dt, 1-3 predictor sweep along x, y, z (CTU: the
 * traced first-stage sweeps), 4 edge E, 5 half update, 6-8 corrector sweep
 * along x, y, z (CTU: transverse corrections), 9 edge E, 10 full update.
 * mhd_profile_end synchronises, stops recording and writes the summed
 * milliseconds of each group (ms[ngroups], ngroups <= 11) and the number
 * of steps recorded. */
mhd_status mhd_profile_begin(mhd_ctx* ctx, int max_steps);
mhd_status mhd_profile_end(mhd_ctx* ctx, double* ms, int ngroups, int* steps);

/* Cell-steps raised to the pressure floor since mhd_init.  Synchronises. */
long long mhd_floor_count(mhd_ctx* ctx);

/* Host-side fault injection for tests of the error path: writes `bits`
 * (1, 2 or 3) into the context's device wait flag, exactly as a bounded
 * device wait that gave up would, so that the mapping to MHD_ETIMEOUT can be
 * checked without making any wait on the GPU fail.  Synchronises. */
mhd_status mhd_inject_wait_flag(mhd_ctx* ctx, unsigned bits);

/* Cell index of the first anomaly found (or -1) and reset of the error. */
long long mhd_bad_cell(mhd_ctx* ctx);
void mhd_clear_error(mhd_ctx* ctx);

/* One-line description of the last error (never NULL). */
const char* mhd_last_error(mhd_ctx* ctx);

/* Measured fused multiply-add throughput of the current device in TFLOP/s
 * (2 flops per FMA), the arithmetic peak the benchmark's roofline divides
 * by: a grid of one full wave of 256-thread blocks, each thread running 8
 * independent FMA chains, timed with CUDA events (best of `reps` launches
 * after one warm-up) at the clocks the device is running.  precision
 * MHD_FP32 or MHD_FP64, 1 <= reps <= 1000, else MHD_EINVAL.  Not part of
 * the method (the paper has no counterpart); it allocates nothing on the
 * device.  Synchronises. */
mhd_status mhd_fma_peak(int precision, int reps, double* tflops);

/* Device memory the context holds, in bytes. */
long long mhd_device_bytes(mhd_ctx* ctx);

/* Number of kernel launches one step issues for this context's scheme. */
int mhd_launches_per_step(mhd_ctx* ctx);

/* Free the context and its device memory (NULL is allowed). */
void mhd_free(mhd_ctx* ctx);

/* ---- learned path selector ---------------------------------------------
 * Per 4^3 block of cells a small MLP (48 features -> 64 -> 64 -> 1, ReLU,
 * BF16 weights on the tensor cores, FP32 accumulation) predicts whether the
 * cheap path (PLM in primitive variables + HLLE) stays within a stated error
 * of the full path (characteristic PPM + HLLD) for one step.  Not in the
 * paper: the paper's method is the full path everywhere; this is an
 * acceleration judged against it.  All arrays are DEVICE pointers. */
typedef struct mhd_mlp mhd_mlp;

/* Network with seeded He-uniform weights, zero biases; Adam state zero. */
mhd_status mhd_mlp_create(void* stream, unsigned long long seed, mhd_mlp** out);
void mhd_mlp_free(mhd_mlp* mlp);
/* Packed FP32 parameter count (7361): W1[48][64], b1[64], W2[64][64],
 * b2[64], w3[64], b3. */
int mhd_mlp_nparam(void);
mhd_status mhd_mlp_set_weights(mhd_mlp* mlp, const float* w, int on_device);
mhd_status mhd_mlp_get_weights(mhd_mlp* mlp, float* w, int on_device);
/* Gradient of the weighted mean binary cross-entropy of the logits against
 * y (0/1) over n samples X[n][48]; wgt[n] may be NULL (all 1); wsum is the
 * sum of the weights.  grad_out: device [nparam]; *loss: host, may be NULL. */
mhd_status mhd_mlp_grad(mhd_mlp* mlp, const float* X, const float* y, const float* wgt, long long n,
                        double wsum, float* grad_out, float* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on that gradient. */
mhd_status mhd_mlp_train_step(mhd_mlp* mlp, const float* X, const float* y, const float* wgt, long long n,
                              double wsum, double lr, float* loss);
/* Logits of n feature rows (logit > 0: the cheap path is predicted safe). */
mhd_status mhd_mlp_predict(mhd_mlp* mlp, const float* X, long long n, float* logits);
/* 4^3 blocks of a one-box context whose sides are multiples of 4 (else -1). */
long long mhd_nblocks(mhd_ctx* ctx);
/* Features of every block of the current state, feats[nblocks][48]. */
mhd_status mhd_block_features(mhd_ctx* ctx, float* feats);
/* Per block, max over the 8 stored fields of mean |a - b| over the block
 * divided by the field's scale in a (rho; rho c_ref for momentum; e; B_ref
 * for the face B): the label metric of a training pair. */
mhd_status mhd_block_error(mhd_ctx* a, mhd_ctx* b, float* err);
/* Attach a trained network to a one-box FP32 VL context (NULL detaches):
 * every following step computes the features, runs the network and steps
 * each sweep tile on the full path when any block next to one of its faces
 * is predicted unsafe, else on the cheap path. */
mhd_status mhd_set_selector(mhd_ctx* ctx, mhd_mlp* mlp);
/* Fractions of blocks and of sweep tiles the last selected step ran cheap. */
mhd_status mhd_selector_stats(mhd_ctx* ctx, double* frac_blocks, double* frac_tiles);

/* ---- stepping without any device allocation ---------------------------
 * The paper has no counterpart: this is a service for callers that may not
 * allocate device memory themselves or through this library (for example a
 * plug-in inside another application whose allocator owns all device
 * memory, or a loop that cannot afford the device-wide synchronisation
 * cudaMalloc / cudaFree can cause).  It advances the caller's state by one
 * FP64 VL step (any recon, any Riemann solver, scheme->pfloor as in
 * mhd_step) with the given dt, in place: U and B are DEVICE pointers in the
 * layout above (double).  All scratch lives in one fixed array built into
 * the library, sized for at most MHD_NOALLOC_MAX_CELLS cells (about 11 MB,
 * held on every GPU that has loaded the library's device code until the
 * process exits).  The call allocates nothing and calls no allocating
 * routine.
 *   - Larger grids: MHD_EINVAL (each side is bounded before the cell count
 *     is formed); other integrators or precisions: MHD_EUNSUPPORTED; the
 *     reason is in mhd_last_error(NULL).
 *   - The first call on a device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *     Under CUDA's default lazy module loading that first lookup is also
 *     when the driver loads the library's device code on that device and
 *     reserves the array, which can synchronise the device: a caller whose
 *     allocator will take all free memory makes one warm-up call per device
 *     before it does (or sets CUDA_MODULE_LOADING=EAGER, which reserves the
 *     array when the context is created).
 *   - Every call, on any stream, shares the one array, which keeps the last
 *     call's contents: calls that overlap on the GPU race and corrupt each
 *     other.  Serialise them (one stream, or events).  Each call resets
 *     what must start at zero (the flag word and the floor count) from its
 *     own kernel arguments.
 *   - Asynchronous on `stream` (NULL = the default stream); a cell with
 *     rho <= 0 or P <= 0 is not reported by this call. */
#define MHD_NOALLOC_MAX_CELLS 32768
mhd_status mhd_step_noalloc(const mhd_grid* grid, double gamma, const mhd_scheme* scheme, double dt,
                            void* U, void* B, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MHD_H */
