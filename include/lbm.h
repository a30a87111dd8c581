/*
 * lbm.h - C ABI of the GB300 (sm_103a) solver for the effective thermal
 * conductivity of heterogeneous anisotropic media with the D3Q7
 * multiple-relaxation-time lattice Boltzmann model and an off-diagonal
 * relaxation block (Fang et al., arXiv 1503.08718).
 *
 * Problem statement (Section 2.1, Eq. 1-4; Section 2.3): a voxel phase map,
 * one symmetric conductivity tensor per phase, a temperature difference
 * applied across two opposite faces (Dirichlet, Eq. 23) and either periodic
 * (Eq. 25) or adiabatic (Eq. 24 with zero flux) conditions on the four other
 * faces.  The solver iterates the lattice Boltzmann map (Eq. 5-13, 21) to its
 * steady state and returns the effective conductivity of Eq. 22.
 *
 * Conventions shared by every call:
 *   - Lattice units dx = dt = 1; gamma = 1/8 and eps = 2 gamma (Section 2.2);
 *     relaxation times tau_0 = tau_4 = tau_5 = tau_6 = 1.
 *   - The diffusivity is D = s * lambda (unit heat capacity, Eq. 20) with a
 *     lattice scale s; tau = I/2 + D/eps (Eq. 13).  s is chosen so the largest
 *     diagonal tau equals opts.tau_max, unless opts.lattice_scale > 0 sets it.
 *   - Arrays of voxels are x fastest: index = (z * ny + y) * nx + x.
 *   - Tensors are 6 doubles per phase in the order xx, yy, zz, yz, xz, xy.
 *   - The hot wall (t_hot) is the face at the axis minimum, walls sit half a
 *     spacing outside the first and last node, L = N_axis and A = N_b N_c.
 *   - Pointers documented as "host" are read (or written) during the call
 *     only and never retained.  Every buffer the library needs on the device
 *     is allocated and owned by the context, with two exceptions:
 *     lbm_create_with_workspace carves them from the caller's block instead,
 *     and lbm_braid_voxelize_noalloc works in caller memory plus one small
 *     file-scope device array of its own.
 *   - A call that fails returns a non-zero lbm_status and records a message
 *     retrievable with lbm_last_error().  After LBM_ERR_CUDA the context is
 *     poisoned: only lbm_last_error() and lbm_destroy() remain valid.
 *   - One context per host thread; contexts are independent.
 *   - The collision is FP32.  The reduced collision leaves every node's
 *     seven populations fixed by four numbers, so the state is stored (FP32,
 *     or BF16 / FP16 with opts.storage) as four fields per node,
 *     th = T - R(z) and jhat / 2; each step rebuilds the populations it
 *     pulls exactly.  R(z) is a per-plane reference temperature along the
 *     temperature-difference axis: the plane mean of T at the previous
 *     check, rounded to a power-of-two grid so that every change of frame
 *     is exact in FP32.  The map is linear, so the frame changes no result
 *     in exact arithmetic; it keeps the stored values small.  Plane-flux and residual
 *     reductions are FP64.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque, owned by the library */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = 1,   /* bad size, pointer, id or tensor */
    LBM_ERR_STATE = 2,         /* call out of order (e.g. solve before set_tensors) */
    LBM_ERR_CUDA = 3,          /* CUDA runtime error; context poisoned */
    LBM_ERR_OUT_OF_MEMORY = 4, /* device allocation failed */
    LBM_ERR_NOT_CONVERGED = 5, /* max_iters reached; results still readable */
    LBM_ERR_DIVERGED = 6,      /* non-finite residual or flux */
    LBM_ERR_STALLED = 7,       /* residual did not improve for stall_checks checks */
    LBM_ERR_TIMEOUT = 8,       /* reserved for bounded device-side waits */
    LBM_ERR_INTERNAL = 9
} lbm_status;

typedef enum { LBM_AXIS_X = 0, LBM_AXIS_Y = 1, LBM_AXIS_Z = 2 } lbm_axis;
typedef enum { LBM_LATERAL_PERIODIC = 0, LBM_LATERAL_ADIABATIC = 1 } lbm_lateral;
/* Storage of the state (four fields per node) between steps; the collision
 * is FP32 in every mode.  BF16 and FP16 halve the memory traffic (17 instead
 * of 33 bytes per lattice update) and are rounded stochastically on store. */
typedef enum { LBM_STORE_F32 = 0, LBM_STORE_BF16 = 1, LBM_STORE_F16 = 2 } lbm_storage;

typedef struct {
    double t_hot, t_cold;   /* wall temperatures (defaults 1, 0); t_hot != t_cold */
    double tau_max;         /* largest diagonal relaxation time (default 1.5), > 0.5 */
    double lattice_scale;   /* > 0 overrides tau_max: D = lattice_scale * lambda */
    double tol;             /* stop when R_T <= tol at a check (default 1e-8) */
    int64_t max_iters;      /* iteration cap (default 50 000 000) */
    int32_t check_every;    /* K: steps per check interval, even, in [2, 4096] (default 100) */
    int32_t stall_checks;   /* stop with LBM_ERR_STALLED after this many checks
                               without a new smallest R_T; 0 disables (default 0) */
    int32_t storage;        /* lbm_storage (default LBM_STORE_F32) */
    int32_t host_loop;      /* 0 (default): lbm_run drives the check intervals with one
                               CUDA graph and a device-side while condition; 1: the host
                               launches each interval and reads the stop flag after it
                               (same kernels and results; for tools that cannot trace
                               conditional graphs) */
    int32_t fuse;           /* 1 (default): FP32 plain steps run two at a time in one
                               kernel (temporal blocking) when the canonical rows hold a
                               multiple of 4 nodes (lbm_start orders the lateral axes to
                               allow it) and the cell gives every SM at least one block
                               of four warps; identical results; a batch's autotuner
                               also times single steps and keeps the faster.  2: two
                               steps per launch whenever the rows allow it, however
                               small the cell (and in a batch whenever every solve
                               allows it).  0: single steps only.  The layout does not
                               depend on this field. */
    int32_t reserved;
    const float* t_init;    /* host, nx*ny*nz initial T field in the original axis
                               order, or NULL for the linear profile between walls */
    void* stream;           /* cudaStream_t for all work, or NULL for the context's */
} lbm_solve_opts;

typedef struct {
    int64_t iters;          /* iterations performed since lbm_start */
    double k_eff;           /* Eq. 22 at the last check */
    double residual_T;      /* R_T = sum|T^n - T^(n-m)| / (m sum|T^n|) at the last check,
                               m = iterations since the previous check (or start) */
    double residual_Q;      /* R_Q = (max_k Q - min_k Q) / |mean Q| at the last check */
    double elapsed_ms;      /* device time of the call's iterations (CUDA events) */
    double lattice_scale;   /* s used */
    int32_t status;         /* lbm_status of the solve */
    int32_t checks;         /* number of checks performed since lbm_start */
} lbm_solve_info;

/* Fills o with the defaults listed in lbm_solve_opts (wall temperatures of
 * Eq. 23, the lattice scale of Eq. 13 through tau_max, the R_T stop rule,
 * which the paper leaves open). */
void lbm_default_opts(lbm_solve_opts* o);

/* Creates a context for an nx*ny*nz cell (the voxel lattice of Section 2.3,
 * one node per voxel) on CUDA device cuda_device.  Sizes must be >= 2 and
 * nx*ny*nz < 2^31.  *out receives the context; the context owns its device
 * memory until lbm_destroy.  LBM_ERR_INVALID_ARG for bad sizes or device,
 * LBM_ERR_OUT_OF_MEMORY if an allocation fails. */
lbm_status lbm_create(int nx, int ny, int nz, int cuda_device, lbm_ctx** out);

/* No counterpart in the paper (device memory ownership).
 * Device bytes a context for an nx*ny*nz cell needs when all of its device
 * memory comes from the caller (lbm_create_with_workspace): the cell's
 * buffers, one solve along any axis with the given storage (lbm_storage) and
 * up to 255 phases, and the voxeliser's scratch.  0 for invalid sizes or
 * storage.  Host-only: needs no GPU. */
size_t lbm_workspace_bytes(int nx, int ny, int nz, int storage);

/* No counterpart in the paper (device memory ownership).
 * Like lbm_create, but every device buffer of the context is carved from the
 * caller's block dev_ptr[0 .. bytes): for callers whose device memory belongs
 * to another allocator (a framework's caching pool, e.g. a torch tensor) or
 * to a fixed budget.  dev_ptr must be device memory of cuda_device, 256-byte
 * aligned, and stay valid and untouched by the caller until lbm_destroy,
 * which does not free it.  bytes >= lbm_workspace_bytes(nx, ny, nz, storage)
 * holds every solve with that storage; a smaller block fails at lbm_start of
 * a solve that does not fit (LBM_ERR_OUT_OF_MEMORY).  lbm_set_geometry_braid
 * then keeps its scratch in the block too (n_max <= 4096).  The context still
 * creates its streams, events and CUDA graphs and a small pinned host block.
 * Errors: LBM_ERR_INVALID_ARG for bad sizes, a null, misaligned or non-device
 * pointer, or bytes below what the cell's own buffers need. */
lbm_status lbm_create_with_workspace(int nx, int ny, int nz, int cuda_device, void* dev_ptr, size_t bytes,
                                     lbm_ctx** out);

/* Voxel phase map (step-wise material description, Sections 3.2 and 5).
 * phase: host, nx*ny*nz uint8 phase ids, each < n_phases; 1 <= n_phases <= 255.
 * Copied to the device.  Invalidates any solve state. */
lbm_status lbm_set_geometry(lbm_ctx* c, const uint8_t* phase, int n_phases);

/* Per-phase conductivity tensors (Eq. 26 rotated into xyz; Eq. 31).
 * lambda: host, n_phases*6 doubles (xx, yy, zz, yz, xz, xy); each tensor must
 * be symmetric positive definite (checked by Cholesky in FP64).
 * n_phases must equal the geometry's. */
lbm_status lbm_set_tensors(lbm_ctx* c, const double* lambda, int n_phases);

/* Prepares a solve with the temperature difference along `axis` and the
 * given lateral faces: computes s, tau and the relaxation block S_b = tau^-1
 * per phase (Eq. 12-13) in FP64, lays the cell out with `axis` slowest, and
 * writes the initial distributions f^eq(T0) (Eq. 6).  Iterations restart at 0.
 * The axis must have at most 65535 nodes.
 * o may be NULL for defaults. */
lbm_status lbm_start(lbm_ctx* c, lbm_axis axis, lbm_lateral lateral, const lbm_solve_opts* o);

/* Advances n_steps fused collide-stream iterations (Eq. 5, 21, 23-25) with
 * no convergence check, asynchronously on the solve's stream. */
lbm_status lbm_advance(lbm_ctx* c, int64_t n_steps);

/* Runs one iteration as a check step: the fused step plus FP64 plane sums of
 * the axial heat flux (Eq. 15-16) and the residual R_T, then Eq. 22.
 * Synchronises the stream; info (nullable) receives the results. */
lbm_status lbm_check(lbm_ctx* c, lbm_solve_info* info);

/* Iterates the lattice (Eq. 5, 21, 23-25) toward the steady state of
 * Section 2.3 from the current state in whole check intervals (CUDA graph
 * with a device-side while condition, no host round trip per check; each
 * check evaluates the flux of Eq. 16 and k_eff of Eq. 22) until R_T <= tol,
 * max_iters, a stall or a non-finite value.  Synchronous. */
lbm_status lbm_run(lbm_ctx* c, lbm_solve_info* info);

/* lbm_start followed by lbm_run: the whole method of Section 2 on one cell
 * (Eq. 5-25 to the steady state, k_eff by Eq. 22). */
lbm_status lbm_solve(lbm_ctx* c, lbm_axis axis, lbm_lateral lateral,
                     const lbm_solve_opts* o, lbm_solve_info* info);

/* Effective conductivity (Eq. 22) of the last check. */
lbm_status lbm_k_eff(const lbm_ctx* c, double* out);

/* Current temperature T = sum f (Eq. 14) into host_out (nx*ny*nz floats,
 * original axis order). Synchronous. */
lbm_status lbm_get_temperature(lbm_ctx* c, float* host_out);

/* Convergence history of the current solve (k_eff of Eq. 22 and the
 * residuals at each check): for each of the most recent
 * min(checks, max_entries, 65536) checks, oldest first, four doubles
 * (iteration, k_eff, R_T, R_Q) into host_out.  *n_out (nullable) receives
 * the number of entries written.  Synchronous. */
lbm_status lbm_get_history(lbm_ctx* c, double* host_out, int max_entries, int* n_out);

/* No counterpart in the paper (checkpoint and resume of the iteration).
 * Bytes of a snapshot of the current solve: its distributions (four stored
 * fields per node, th = T - R(z) and jhat / 2, from which the seven
 * post-collision populations follow exactly), reference frames, residual
 * snapshot, control block, check history and last plane fluxes.  0 without a started solve (or for NULL / a poisoned context). */
size_t lbm_state_bytes(const lbm_ctx* c);

/* No counterpart in the paper.  Writes the snapshot of the current solve
 * (lbm_state_bytes bytes) to host_out (caller-owned).  Synchronous.
 * LBM_ERR_STATE without a started solve, LBM_ERR_INVALID_ARG if host_out is
 * NULL or bytes is too small. */
lbm_status lbm_get_state(lbm_ctx* c, void* host_out, size_t bytes);

/* No counterpart in the paper.  Resumes from a snapshot taken by
 * lbm_get_state: the context must have the same geometry and tensors and a
 * solve started (lbm_start) with the same axis, lateral type, storage,
 * check interval and walls; the snapshot replaces that solve's state, so a
 * following lbm_run / lbm_advance continues the saved iteration (bit for
 * bit the iterates of an uninterrupted run driven the same way).  host_in
 * is read during the call only.  Synchronous.  LBM_ERR_INVALID_ARG for a
 * snapshot of another solve or a truncated one. */
lbm_status lbm_set_state(lbm_ctx* c, const void* host_in, size_t bytes);

/* No counterpart in the paper (how the solve is laid out and launched).
 * After lbm_start: the canonical layout (rows of nx nodes, the temperature
 * axis nz last; pitch = padded row length) and the kernel plan of the plain
 * steps: steps_per_launch 2 when FP32 plain steps run as fused pairs
 * (temporal blocking) with tiles of tile_rows rows, zchunk planes and
 * block_threads threads per block, else 1 (single steps; tile fields 0). */
typedef struct {
    int32_t nx, ny, nz, pitch;
    int32_t steps_per_launch;
    int32_t tile_rows, zchunk, block_threads;
} lbm_launch_plan;

lbm_status lbm_get_launch_plan(const lbm_ctx* c, lbm_launch_plan* out);

/* Plane sums Q[k] of the axial flux of Eq. 16 at the last check, the
 * integrand of Eq. 22 (n == N_axis doubles, host_out caller-owned). */
lbm_status lbm_get_plane_flux(const lbm_ctx* c, double* host_out, int n);

/* Synthetic four-directional braided cell (yarns along
 * (sx sin g / sqrt 2, sy sin g / sqrt 2, cos g), Section 4.1) voxelised on
 * the device by a voxel-centre test in FP64 without contraction (the
 * step-wise approximation of Section 3.2).  anchors: host, n_max (x0, y0)
 * pairs; yarn i belongs to family i mod 4 with signs (+,+), (-,+), (-,-),
 * (+,-) and elliptic section with semi-axes A (horizontal) and B.  Yarns are
 * added in order until the yarn fraction reaches phi; a voxel takes the
 * family (1..4) of the first yarn containing it, else 0.  Sets the geometry
 * with n_phases = 5.  n_used and fraction (host, nullable) receive the yarn
 * count and the achieved fraction. Returns LBM_ERR_INVALID_ARG if phi is not
 * reached with n_max yarns or g is not in (0, pi/2). */
lbm_status lbm_set_geometry_braid(lbm_ctx* c, double g_rad, double A, double B,
                                  const double* anchors, int n_max, double phi,
                                  int* n_used, double* fraction);

/* ---- Batched solves (the paper's sweeps over fibre fraction, braiding
 * angle and direction, Section 5 and Fig. 9) ------------------------------ */

typedef struct lbm_batch lbm_batch; /* opaque, owned by the library */

typedef struct {
    int32_t n_solves;       /* solves in the batch */
    int32_t n_converged;    /* solves that met R_T <= tol */
    int64_t total_updates;  /* lattice updates performed (voxels x iterations, summed) */
    double elapsed_ms;      /* device time of the graph launch (CUDA events) */
    int32_t block_threads;  /* block size the autotuner picked for the plain steps: single
                               steps (128, 256 or 512 threads) or FP32 two-step launches
                               (256 .. 640 threads; see lbm_batch_solve) */
    int32_t status;         /* LBM_OK if every solve converged, else LBM_ERR_NOT_CONVERGED */
    int32_t steps_per_launch; /* 2 if the plain steps ran as two-step launches, else 1 */
    int32_t reserved;
} lbm_batch_info;

/* Creates an empty batch (for the sweeps of Section 5) on CUDA device
 * cuda_device. */
lbm_status lbm_batch_create(int cuda_device, lbm_batch** out);

/* Adds one steady solve of Section 2 to the sweep: an nx*ny*nz cell (phase
 * map and n_phases tensors, host, copied; same layout and checks as
 * lbm_set_geometry / lbm_set_tensors) with the temperature difference along
 * `axis`.  *id (nullable) receives the solve's index. */
lbm_status lbm_batch_add(lbm_batch* b, int nx, int ny, int nz, const uint8_t* phase, int n_phases,
                         const double* lambda, lbm_axis axis, int* id);

/* Solves every added problem (the sweeps of Section 5, Fig. 9) with one
 * lateral type and one set of options (each solve takes its own lattice
 * scale from its tensors unless opts.lattice_scale is set; opts.t_init must
 * be NULL: per-solve start fields come from lbm_batch_set_initial).  All
 * solves stay resident
 * in device memory; one CUDA graph launch advances every unconverged solve by
 * whole check intervals until each has met tol or max_iters.  Before the
 * launch an autotuner times six plain steps of the batch itself for each
 * candidate and keeps the fastest: single steps with 128, 256 or 512 threads
 * per block, and (FP32 storage with opts.fuse, every solve's canonical rows a
 * multiple of 4 nodes) two steps per launch with 256 .. 640 threads per
 * block (tile height from the row width) and z chunks of 8, 16 or 32 planes.
 * Every candidate computes the same iterates bit for bit.  Synchronous. */
lbm_status lbm_batch_solve(lbm_batch* b, lbm_lateral lateral, const lbm_solve_opts* o,
                           lbm_batch_info* info);

/* Result of solve `id` after lbm_batch_solve (iterations, k_eff of Eq. 22,
 * residuals, lattice scale, status). */
lbm_status lbm_batch_result(const lbm_batch* b, int id, lbm_solve_info* info);

/* Final temperature (Eq. 14) of solve `id` (nx*ny*nz floats, original axis
 * order, host_out caller-owned). */
lbm_status lbm_batch_get_temperature(lbm_batch* b, int id, float* host_out);

/* Initial temperature of solve `id` (host, nx*ny*nz floats in the original
 * axis order, copied; NULL restores the linear profile): the solve starts
 * from f^eq of this field (Eq. 6), e.g. a learned prediction of the steady
 * field (the method needs only the steady state, Section 2.3).  Applies to
 * the next lbm_batch_solve. */
lbm_status lbm_batch_set_initial(lbm_batch* b, int id, const float* t_init);

/* Convergence history of solve `id` after lbm_batch_solve: for each of its
 * most recent min(checks, max_entries, 4096) checks, oldest first, five
 * doubles (iteration, k_eff of Eq. 22, R_T, R_Q, device time in ms from the
 * start of the batch's iteration to the end of that check) into host_out.
 * *n_out (nullable) receives the number of entries.  Synchronous. */
lbm_status lbm_batch_get_history(lbm_batch* b, int id, double* host_out, int max_entries, int* n_out);

/* No counterpart in the paper.  Message of the last failed batch call
 * (batch-owned string). NULL-safe. */
const char* lbm_batch_last_error(const lbm_batch* b);

/* No counterpart in the paper.  Frees the batch and its device memory.
 * NULL-safe. */
void lbm_batch_destroy(lbm_batch* b);

/* ---- Learned warm start: layers of the 3D convolutional network ---------
 * The paper's method only needs the steady state (Section 2.3, Eq. 20), so
 * the iteration may start from any field; these layers predict that field
 * from the material so the iteration starts near it.  The converged lattice
 * Boltzmann solve remains the answer.  All tensors are device pointers in
 * caller memory, channels last: element [v][c] at v * C + c with the voxel
 * index v = ((n * d + z) * h + y) * w + x over a batch of n cells of d x h x w
 * (z the temperature-difference axis).  Activations and weights are BF16,
 * accumulation FP32.  stream: cudaStream_t (NULL = legacy default stream).
 * Calls are asynchronous; they return LBM_ERR_INVALID_ARG on a bad size or
 * NULL pointer and LBM_ERR_CUDA on a launch error.  The paper has no
 * network: none of these layers has a counterpart in it. */

/* y = act(bias + conv(x, w)): ksize 3 (27 taps, periodic in x and y, zero
 * outside in z) or 1.  x [V][cin] (cin a multiple of 16), w [taps][cin][cout]
 * (tap = (dz*3 + dy)*3 + dx), bias [cout] FP32 or NULL, y [V][cout] BF16, or
 * FP32 if out_f32 (cout a multiple of 32).  relu != 0 applies the leaky
 * ReLU max(., 0) + 0.01 min(., 0).
 * Runs on the tensor cores (mma.sync m16n8k16, implicit GEMM). */
lbm_status lbm_nn_conv3d(const void* x, int cin, const void* w, const float* bias, void* y, int cout,
                         int n, int d, int h, int wdt, int ksize, int relu, int out_f32,
                         void* stream);

/* The same 3x3x3 convolution (bias, leaky ReLU, BF16 or FP32 output) on the
 * fifth-generation tensor cores: tcgen05.mma with the accumulators in
 * tensor memory, persistent blocks (one per SM) walking tiles of 16 x 8
 * output voxels of one or more planes, each tile's halo staged once in
 * shared memory and read by every tap's MMA through its own descriptor, the
 * taps' weight slabs streamed by cp.async.bulk through a ring of
 * shared-memory stages, the epilogue of one tile overlapping the MMAs of the
 * next.  wk: the weight slabs lbm_nn_weights_kmajor writes
 * (27 * cin * cout BF16).
 * Requires cin and cout multiples of 16, cout <= 256, h a multiple of 16 and
 * w a multiple of 8 (lbm_nn_conv3d_tc_supported); else LBM_ERR_INVALID_ARG.
 * Each block bounds its waits; a timeout is recorded for lbm_nn_tc_error. */
lbm_status lbm_nn_conv3d_tc(const void* x, int cin, const void* wk, const float* bias, void* y, int cout,
                            int n, int d, int h, int wdt, int relu, int out_f32, void* stream);

/* Weight gradient of the 3x3x3 convolution on the tcgen05 tensor cores,
 * dw[tap][ci][co] += sum_v x[v + tap][ci] g[v][co] (FP32 atomics into dw;
 * zero it first): per tap a GEMM over the voxels with both operands read
 * channels-last (MN-major) from shared memory, the accumulators of a group
 * of taps in tensor memory.  Same layouts and padding as lbm_nn_conv3d.
 * Requires cin a multiple of 16, cout a multiple of 8 and at most 128, h a
 * multiple of 16 and w of 8 (lbm_nn_conv3d_wgrad_tc_supported). */
lbm_status lbm_nn_conv3d_wgrad_tc(const void* x, int cin, const void* g, int cout, float* dw, int n, int d,
                                  int h, int wdt, void* stream);

/* 1 if lbm_nn_conv3d_wgrad_tc takes these sizes, else 0.  Host-only. */
int lbm_nn_conv3d_wgrad_tc_supported(int cin, int cout, int n, int d, int h, int w);

/* lbm_nn_conv3d_tc with an explicit launch configuration: tz output planes
 * per tile (1, 2 or 4: the planes share every weight slab) and ns weight
 * stages in shared memory (>= 2); 0 lets the library choose, as
 * lbm_nn_conv3d_tc does.  LBM_ERR_INVALID_ARG if the sizes or the
 * configuration do not fit (d must be a multiple of tz; the two accumulator
 * buffers of tz planes must fit 512 tensor-memory columns; the stages must
 * fit shared memory). */
lbm_status lbm_nn_conv3d_tc_cfg(const void* x, int cin, const void* wk, const float* bias, void* y, int cout,
                                int n, int d, int h, int wdt, int relu, int out_f32, int tz, int ns, void* stream);

/* 1 if lbm_nn_conv3d_tc takes these sizes, else 0.  Host-only. */
int lbm_nn_conv3d_tc_supported(int cin, int cout, int n, int d, int h, int w);

/* Weight slabs for lbm_nn_conv3d_tc from w [27][cin][cout] (27 * cin * cout
 * BF16 into wk).  The conv that uses them has K input and N output channels:
 * flip = 0 gives the forward conv (K = cin, N = cout); flip = 1 the data
 * gradient's conv (K = cout, N = cin, taps reversed: tap t uses
 * w[26 - t]).  The K channels are split into groups of G = 32 if 32 divides
 * K, else 16; slab (tap, group) is
 * [G/8][N][8] (input channel group*G + 8*k8 + e, output channel n), each slab
 * contiguous, slabs in (tap, group) order: the image of one shared-memory
 * weight stage, K-major core matrices of 8 x 8 elements. */
lbm_status lbm_nn_weights_kmajor(const void* w, void* wk, int cin, int cout, int flip, void* stream);

/* First error recorded by a lbm_nn_conv3d_tc block since the last clear (0:
 * none; 1: a bounded wait on the tensor core expired).  clear != 0 resets it.
 * Synchronous. */
lbm_status lbm_nn_tc_error(int* out, int clear);

/* dw[tap][ci][co] += sum_v x[v + tap][ci] g[v][co] (FP32 accumulation into dw;
 * zero dw first).  Same layouts and padding as lbm_nn_conv3d. */
lbm_status lbm_nn_conv3d_wgrad(const void* x, int cin, const void* g, int cout, float* dw, int n,
                               int d, int h, int wdt, int ksize, void* stream);

/* wf[tap][co][ci] = w[taps-1-tap][ci][co]: with it lbm_nn_conv3d computes the
 * gradient with respect to the conv's input. */
lbm_status lbm_nn_flip_weights(const void* w, void* wf, int cin, int cout, int ksize, void* stream);

/* db[c] += sum_v g[v][c] (c <= 1024). */
lbm_status lbm_nn_bias_grad(const void* g, int c, long long nvox, float* db, void* stream);

/* g = dy where y > 0, else 0.01 dy (backward of the fused leaky ReLU whose
 * output is y). */
lbm_status lbm_nn_relu_mask(const void* dy, const void* y, void* g, long long count, void* stream);

/* y[parent] = scale * sum of the 8 children of x; (d, h, w) are x's sizes
 * (even).  scale 1/8 is 2x2x2 average pooling, 1 the backward of upsampling. */
lbm_status lbm_nn_pool2(const void* x, void* y, int c, int n, int d, int h, int w, float scale,
                        void* stream);

/* y[child] = scale * x[parent]; (d, h, w) are y's sizes (even).  scale 1 is
 * nearest upsampling, 1/8 the backward of average pooling. */
lbm_status lbm_nn_upsample2(const void* x, void* y, int c, int n, int d, int h, int w, float scale,
                            void* stream);

/* y[v] = [a[v] (ca channels), b[v] (cb channels)]. */
lbm_status lbm_nn_concat(const void* a, int ca, const void* b, int cb, void* y, long long nvox,
                         void* stream);

/* dst[v][0:c] = src[v][coff:coff+c] (+ dst if accumulate); src has csrc channels. */
lbm_status lbm_nn_slice(const void* src, int csrc, int coff, void* dst, int c, long long nvox,
                        int accumulate, void* stream);

/* Output head: pred[v] = t_lin[v] + b + w . h[v] (h: 32 BF16 channels, w, b
 * FP32).  With target != NULL also the squared-error loss and its gradients:
 * loss += sum_v (pred - target)^2, dT = 2 (pred - target) / nvox,
 * dh = dT w (BF16), dw += sum dT h, db += sum dT. */
lbm_status lbm_nn_head(const void* h, const float* w, const float* b, const float* t_lin,
                       const float* target, float* pred, void* dh, float* dw, float* db,
                       double* loss, long long nvox, void* stream);

/* Network input x [V][16] BF16: channels 0..5 = table[phase[v]] (six tensor
 * components per phase, FP32), channel 6 = t_lin_z[z], 7..15 = 0. */
lbm_status lbm_nn_input(const uint8_t* phase, const float* table, const float* t_lin_z, void* x,
                        int n, int d, int h, int w, void* stream);

/* One Adam step on FP32 master weights p with gradient g and moments m, v
 * (step counts from 1); p_bf16 (nullable) receives the BF16 copy. */
lbm_status lbm_nn_adam(float* p, const float* g, float* m, float* v, void* p_bf16, long long count,
                       float lr, float beta1, float beta2, float eps, int step, void* stream);

/* Largest n_max accepted by lbm_braid_voxelize_noalloc. */
#define LBM_NOALLOC_MAX_YARNS 1024

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory.  It produces the same phase map as
 * lbm_set_geometry_braid (bit for bit), but writes it into caller memory and
 * allocates nothing: no cudaMalloc, no cudaFree, no context.  Callers that
 * need it are processes whose device memory belongs to another allocator
 * (e.g. a framework's caching pool holding most of the GPU), services under a
 * fixed memory budget, and loops that must not stall on the device-wide
 * synchronisation that cudaMalloc and cudaFree imply.
 *
 * Its scratch (a yarn histogram) is a file-scope __device__ array of
 * LBM_NOALLOC_MAX_YARNS + 1 64-bit bins (8.2 KB) that every GPU loading the
 * library holds until the process exits.  The first call on a device (the
 * current device) looks up that array's device address once; make that first
 * call before any stream capture, and do not call it again on a device after
 * cudaDeviceReset (the cached address would be stale).  Every call on a device shares the array
 * and clears the bins it uses; calls that overlap on the GPU (concurrent
 * streams or threads) race on it and must be serialised by the caller.
 *
 * nx, ny, nz: cell size (>= 1, product < 2^31).
 * g_rad, A, B, phi: as lbm_set_geometry_braid.
 * d_anchors: device, 16-byte aligned, n_max (x0, y0) double pairs.
 *            d_anchors and d_phase must be device (or managed) memory of the
 *            current device; anything else (a host pointer, say) returns
 *            LBM_ERR_INVALID_ARG before any kernel runs.
 * n_max: 1 .. LBM_NOALLOC_MAX_YARNS; larger values return
 *        LBM_ERR_INVALID_ARG with a message saying so.
 * d_phase: device, nx*ny*nz uint8 output (x fastest), written on `stream`.
 * n_used, fraction: host, nullable; set before return.
 * stream: cudaStream_t (NULL = legacy default stream).  The call
 *         synchronises the stream once (to read the histogram); the phase map
 *         is written asynchronously after that on the same stream.
 * err, err_len: host buffer (nullable) for a message on failure.
 * Returns LBM_OK, LBM_ERR_INVALID_ARG or LBM_ERR_CUDA. */
lbm_status lbm_braid_voxelize_noalloc(int nx, int ny, int nz, double g_rad, double A, double B,
                                      const double* d_anchors, int n_max, double phi,
                                      uint8_t* d_phase, int* n_used, double* fraction,
                                      void* stream, char* err, int err_len);

/* Yarn conductivities from the fibre and matrix conductivities (Section 4.2):
 * longitudinal lam_L = lam_fL phi_fy + lam_m (1 - phi_fy) (Eq. 36) and
 * transverse lam_T = lam_m + phi_fy / (1/(lam_fT - lam_m) + (1 - phi_fy)/(2 lam_m))
 * (Eq. 37, whose printed numerator 1 - phi_fy contradicts Table II; phi_fy
 * reproduces it).  phi_fy: fibre fraction inside the yarn, in (0, 1).
 * Host-only, no device work.  Returns LBM_ERR_INVALID_ARG on non-positive
 * conductivities, lam_fT == lam_m or phi_fy outside (0, 1). */
lbm_status lbm_yarn_conductivity(double lam_fL, double lam_fT, double lam_m, double phi_fy,
                                 double* lam_L, double* lam_T);

/* Unit cell of the four-directional braid (Section 4.1, Eq. 32-35): yarn
 * volume fraction phi_y = pi sqrt(3) / 8 (Eq. 35), phi_fy = phi_f / phi_y, yarn
 * section area A = n_f pi d_f^2 / 4 / phi_fy = pi d c (Eq. 34) with
 * c = d sqrt(3) cos(gamma) (Eq. 33), cell side a = 8 d (Eq. 32) and braiding
 * pitch h = a / tan(gamma) (the paper takes h from its reference [17]; this
 * relation reproduces its worked example).  Lengths in the unit of d_f.
 * Host-only.  Outputs (host, nullable): a, h, c (semi-major), d (semi-minor),
 * phi_fy.  Returns LBM_ERR_INVALID_ARG unless 0 < phi_f < phi_y, n_f >= 1,
 * d_f > 0 and 0 < gamma < pi/2. */
lbm_status lbm_braid_unit_cell(double phi_f, int n_f, double d_f, double gamma_rad, double* a,
                               double* h, double* c, double* d, double* phi_fy);

/* Copies the phase map (the voxelised cell of Section 5, Fig. 7; nx*ny*nz
 * uint8, original order) to host_out (caller-owned). */
lbm_status lbm_get_geometry(lbm_ctx* c, uint8_t* host_out);

/* No counterpart in the paper (a stand-in for a memory checker).  1 if this
 * library was built with bounds checks (LBM_DEBUG): every global and ring
 * access of the step kernels is checked against its buffer, an access outside
 * records a code (and touches the buffer's first element instead), and the
 * solver calls that synchronise (lbm_check, lbm_run, lbm_solve,
 * lbm_batch_solve) then fail with LBM_ERR_INTERNAL.  0 for the normal build. */
int lbm_debug_build(void);

/* The recorded bounds-check code of the context kernels (0: none; always 0
 * in the normal build); clear != 0 resets it.  Synchronous. */
lbm_status lbm_debug_error(unsigned* out, int clear);

/* No counterpart in the paper.  Message of the last failed call on this
 * context (context-owned string, valid until the next call).  NULL-safe. */
const char* lbm_last_error(const lbm_ctx* c);

/* No counterpart in the paper.  Frees the context and all device memory it
 * owns (a caller's workspace stays the caller's). NULL-safe. */
void lbm_destroy(lbm_ctx* c);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
