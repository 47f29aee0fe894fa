/* hlbm.h -- C ABI of the GB300 moving-grid hybrid lattice Boltzmann solver.
 *
 * The solver advances the flow around a rigid lamina that moves through a
 * viscous fluid, as in Di Ilio, Chiappini, Ubertini, Bella, Succi, "A
 * moving-grid approach for fluid-structure interaction problems with hybrid
 * lattice Boltzmann method":
 *   - D2Q9 BGK stream-collide on a fixed Cartesian lattice (Sec. 3, eq. LBE,
 *     eq. local_eq) with no-slip side walls and outflow top/bottom (Sec. 5);
 *   - a cell-vertex finite-volume LB update on a triangular patch fitted to
 *     the body, sub-cycled n times per lattice step (Sec. 3, eq. ulbe);
 *   - the coupling of the two grids at interpolation nodes (eq.
 *     postcollision2_s, eq. postcollision2_u);
 *   - the per-step relocation of the patch and the refill of its nodes
 *     (Sec. 4, types 1/2/3, eq. continuity_stresses);
 *   - the force on the lamina and the complex hydrodynamic function
 *     Theta (Sec. 2.1, eq. force_phasor).
 *
 * Conventions for every call:
 *   - Lattice units: dx = dt = 1 on the Cartesian lattice, c_s^2 = 1/3.
 *   - Every pointer argument is HOST memory unless stated otherwise.  Input
 *     arrays are copied during the call; the caller keeps ownership.
 *   - All device memory belongs to the solver.  It is obtained from the
 *     allocator installed with hlbm_set_allocator (cudaMalloc otherwise) and
 *     released by hlbm_destroy.
 *   - Calls return HLBM_OK (0) or a negative HLBM_E* code; the message of
 *     the last failure is available from hlbm_last_error.  Nothing aborts
 *     the process.
 *   - hlbm_step only enqueues work on the solver's stream and returns;
 *     the hlbm_get_* / hlbm_force / hlbm_gamma / hlbm_status calls
 *     synchronise that stream.
 *   - A handle is used from one host thread at a time.
 */
#ifndef HLBM_H
#define HLBM_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define HLBM_OK 0
#define HLBM_EINVAL (-1)    /* invalid argument or configuration          */
#define HLBM_ECUDA (-2)     /* a CUDA runtime call failed                 */
#define HLBM_EUNSTABLE (-3) /* NaN/Inf in the force: the run diverged     */
#define HLBM_EGEOM (-4)     /* a geometric precondition failed on device  */
#define HLBM_ENOMEM (-5)    /* device allocation failed                   */
#define HLBM_EIO (-6)       /* a checkpoint file could not be read/written */
#define HLBM_ETIMEOUT (-7)  /* an FV neighbour wait ran out: step abandoned */

/* boundary kinds of the Cartesian domain sides (Sec. 5) */
#define HLBM_BC_WALL 0     /* half-way bounce-back no-slip wall          */
#define HLBM_BC_OUTFLOW 1  /* zero-gradient outflow                      */
#define HLBM_BC_PERIODIC 2

/* storage and arithmetic precision of the populations */
#define HLBM_F64 0  /* FP64 storage and arithmetic                               */
#define HLBM_F32 1  /* FP32 storage and arithmetic                               */
#define HLBM_F16 2  /* lattice populations stored as FP16 (scaled by 2^10)       */
                    /* deviations; FP32 arithmetic and patch; FP64 force and fit */
#define HLBM_BF16 3 /* as HLBM_F16 with BF16 lattice storage (no scaling)        */

/* patch node kinds (Sec. 4) */
#define HLBM_NODE_INTERIOR 0 /* discretization node                       */
#define HLBM_NODE_OUTER 1    /* outer boundary = interpolation node        */
#define HLBM_NODE_WALL 2     /* on the lamina surface                      */

/* motion kinds (Sec. 2: y(t) = A sin(w t)) */
#define HLBM_MOTION_STATIC 0
#define HLBM_MOTION_HARMONIC 1 /* X = 0, Y = A sin(w t)                   */
#define HLBM_MOTION_UNIFORM 2  /* X = vx t, Y = vy t                      */
#define HLBM_MOTION_INDUCED 3  /* X = 0, m Y'' + c Y' + k Y = F_y (below)  */

/* status bits reported by hlbm_status (device-side checks) */
#define HLBM_ST_FILL_NOT_LOCATED 1u   /* eq. 178 node outside the patch     */
#define HLBM_ST_DONOR_NOT_COMPUTED 2u /* bilinear donor not a computed node */
#define HLBM_ST_NONFINITE 8u          /* NaN/Inf in the lamina force        */
#define HLBM_ST_UNUSED_TO_DISC 16u    /* lattice node skipped a class       */
#define HLBM_ST_SYNC_TIMEOUT 32u      /* FV tiles waited too long: aborted  */

/* Cartesian lattice: nx*ny nodes at integer positions (x, y), row-major.
 * rho_init / ux_init / uy_init: optional host arrays [ny*nx] of the initial
 * density and velocity (the state starts at equilibrium); NULL selects rho0
 * and (u0x, u0y) everywhere. */
/* One coarser lattice level around the solver's lattice (level 0).  Level k
 * (levels[k-1]) has twice the spacing and time step of level k-1, nx x ny
 * nodes, and holds node (0, 0) of level k-1 at its node (ox, oy); its
 * relaxation time is tau_k = 1/2 + (tau_s - 1/2)/2^k (same viscosity).
 * Each step of level k-1's box, its outermost ring is rebuilt from level k
 * (rho, u and post-collision f^neq rescaled by (tau_{k-1} - 1)/(2 (tau_k - 1));
 * the four-point cubic midpoint rule along the box edge; at odd times of
 * level k-1 the mean of level k's two times around it), and whenever level
 * k-1 has caught up with level k, level k's nodes strictly inside the box
 * take level k-1's post-collision state with f^neq rescaled back.  Every
 * level inside another has odd nx, ny; the boundary kinds of hlbm_grid_t
 * apply to the coarsest level.  Level k starts at equilibrium with rho_init,
 * ux_init, uy_init ([ny*nx], NULL: rho0, u0x, u0y) and then takes level
 * k-1's initial state inside the box.  hlbm_create fails with HLBM_EINVAL
 * unless each box has odd sizes of at least 9 and keeps to the edges of the
 * level around it a margin of one node (two when that level is itself inside
 * another: the cubic rule must not reach a ring), n_levels <=
 * HLBM_MAX_LEVELS, and every tau_k (k = 0 .. n_levels) differs from 1 by
 * more than 1e-3. */
#define HLBM_MAX_LEVELS 4
typedef struct {
    int32_t nx, ny;
    int32_t ox, oy;
    const double* rho_init;
    const double* ux_init;
    const double* uy_init;
} hlbm_level_t;

typedef struct {
    int32_t nx, ny;
    int32_t bc_x, bc_y; /* sides x = 0, nx-1 and y = 0, ny-1 */
    int32_t dtype;      /* HLBM_F64 | HLBM_F32 | HLBM_F16 | HLBM_BF16 */
    double rho0;
    double u0x, u0y;
    const double* rho_init;
    const double* ux_init;
    const double* uy_init;
    /* Nested structured refinement levels (Sec. 5 runs its lattice on four
     * levels; the coupling is not given there): n_levels coarser lattices,
     * levels[0] first (see hlbm_level_t).  0 = one uniform lattice. */
    int32_t n_levels;
    const hlbm_level_t* levels;
    /* Non-reflecting outflow (the second reading of Sec. 5's unspecified
     * outflow; 0 rows = the zero-gradient copy alone): along each outflow
     * side of the lattice that carries the domain boundary (the coarsest
     * level), the post-collision populations of the sponge_rows rows next
     * to it relax towards the rest state, f <- w rho0 + (1 - s(d)) (f -
     * w rho0) at d rows from the side, s(d) = sponge_sigma ((N - d)/N)^2.
     * 0 <= sponge_rows < half the lattice side it lies along,
     * 0 <= sponge_sigma < 1. */
    int32_t sponge_rows;
    double sponge_sigma;
} hlbm_grid_t;

/* Body-fitted triangular patch around the lamina (Sec. 3, Sec. 4).
 * xy: [n_nodes*2] node coordinates in the body frame (origin at the lamina
 * centre); tri: [n_tris*3] node indices; kind: [n_nodes] HLBM_NODE_*.
 * The lamina is the rectangle |x| <= L/2, |y| <= T/2 of the body frame,
 * centred at (x_c, y_c) at t = 0.  Lattice nodes inside the rounded
 * rectangle at offset delta_f (the fictitious curve) are unused.  n_sub FV
 * sub-steps are taken per lattice step (dt_s = n_sub dt_u).  lumped = 1
 * replaces the consistent collision matrix C_ik by the identity.
 * outer_fv selects the update of the outer (interpolation) patch nodes,
 * eq. postcollision2_u: 0 takes its interpolated part only,
 * f = f^eq,s + (1 - dt_s/(2 tau_s)) f^neq,s, bilinear from the lattice and
 * linear in time over the lattice step; 1 adds its FV sums over the node's
 * truncated control volume, with the starred values of the paper
 * (interpolated at interpolation nodes, the patch state elsewhere).
 * fv_kernel picks the kernel of the FV sub-steps, HLBM_FV_*: AUTO takes the
 * first that applies of DEEP and TMEM (rows of at most 7 off-diagonal
 * entries, outer_fv = 0), SMEM and GLOBAL; the others are for testing and
 * hlbm_create fails with HLBM_EINVAL when the one asked for cannot run the
 * patch.  All give the same results bit for bit. */
typedef struct {
    int32_t n_nodes, n_tris;
    const double* xy;
    const int32_t* tri;
    const int8_t* kind;
    double lamina_L, lamina_T;
    double x_c, y_c;
    double delta_f;
    int32_t n_sub;
    int32_t lumped;
    int32_t outer_fv;
    int32_t fv_kernel;
} hlbm_patch_t;

/* kernels of the FV sub-steps (hlbm_patch_t.fv_kernel) */
#define HLBM_FV_AUTO 0
#define HLBM_FV_GLOBAL 1 /* records in global memory, any tile size          */
#define HLBM_FV_SMEM 2   /* tiles in shared memory, records updated in place */
#define HLBM_FV_TMEM 3   /* rows in tensor memory, records double-buffered   */
#define HLBM_FV_DEEP 4   /* as TMEM with ghost layers: one exchange between   */
                         /* tiles every K sub-steps (hlbm_set_fv_depth)       */

/* Lamina motion.  HARMONIC: A, omega; UNIFORM: vx, vy.  INDUCED (the paper's
 * outlook towards fluid-structure interaction, Sec. 7): a rigid lamina on a
 * spring and damper moved by the fluid, m Y'' + c Y' + k Y = F_y per unit
 * length (lattice units, rho0 = 1), Y(0) = y0, Y'(0) = v0.  Each lattice step
 * t takes one symplectic Euler step with the force at t:
 * v(t+1) = v(t) + (F_y(t) - c v(t) - k Y(t)) / m, Y(t+1) = Y(t) + v(t+1);
 * the patch sits at Y(t) during step t and the wall velocity of sub-step j
 * is v(t) + (j+1)/n (v(t+1) - v(t)).  hlbm_step then reads F_y(t) back from
 * the device every step (it synchronises the stream) and fails with
 * HLBM_EINVAL when |v| would take the patch's outer nodes past their
 * donors (|v| > outer-boundary distance - delta_f - 1.5) or the window off
 * the lattice. */
typedef struct {
    int32_t kind; /* HLBM_MOTION_* */
    double A, omega;
    double vx, vy;
    double mass, stiffness, damping, y0, v0;
} hlbm_motion_t;

typedef struct hlbm hlbm_t;

/* Device allocator hook used by every later hlbm_create.  alloc returns a
 * device pointer of at least `bytes` usable on `stream` (NULL on failure);
 * release frees it.  Passing NULLs restores cudaMalloc/cudaFree. */
typedef void* (*hlbm_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*hlbm_free_fn)(void* ptr, void* stream, void* ctx);
int hlbm_set_allocator(hlbm_alloc_fn alloc, hlbm_free_fn release, void* ctx);

/* Build a solver (Sec. 2 problem statement): copies the mesh, derives the FV
 * matrices S_ik = c_i . g_Pk and C_ik of eq. ulbe on median-dual control
 * volumes, the wall segments and the point-location bins, sets the initial
 * equilibrium state and fills the patch from the lattice by the type-1
 * rule of Sec. 4.  tau_s is the lattice relaxation time; the patch uses
 * tau_u = tau_s - 1/2 (same viscosity, Sec. 3).  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream) on which all work is queued.
 * Returns HLBM_EINVAL when the time step is unstable (dt_u >= 2 tau_u,
 * Sec. 7), when the patch is too thin for the per-step displacement, or
 * when the patch can come closer than 4 nodes to the lattice edge. */
int hlbm_create(const hlbm_grid_t* grid, const hlbm_patch_t* patch, double tau_s,
                const hlbm_motion_t* motion, void* cuda_stream, hlbm_t** out);

/* Advance nsteps lattice steps (asynchronous).  Each step: move the patch
 * to y(t) and refill it (Sec. 4), reclassify the lattice nodes, feed the
 * lattice interpolation nodes from the patch (eq. postcollision2_s), one
 * stream-collide of eq. LBE, n_sub FV sub-steps of eq. ulbe with the outer
 * patch nodes fed from the lattice (eq. postcollision2_u), and the force on
 * the lamina at the new time.
 * Device status bits (HLBM_ST_*) are errors.  Once the host has seen one --
 * through hlbm_status, hlbm_force or hlbm_gamma, or through the copy of the
 * status word that each hlbm_step call queues at its end, which the next
 * call reads if it has arrived (without waiting for it) -- hlbm_step steps
 * nothing and returns HLBM_ETIMEOUT (SYNC_TIMEOUT), HLBM_EUNSTABLE
 * (NONFINITE) or HLBM_EGEOM (the others) until hlbm_clear_status or
 * hlbm_load. */
int hlbm_step(hlbm_t* h, int64_t nsteps);

/* Acknowledge the device status bits: synchronises the solver's stream,
 * clears the status word and the FV kernels' abort flag, and restarts
 * their progress counters at the current step, so that hlbm_step runs
 * again.  The state is left as it is: after HLBM_ETIMEOUT the patch holds
 * the sub-steps the abandoned step completed, tile by tile (restore a
 * checkpoint with hlbm_load to go on from a consistent state). */
int hlbm_clear_status(hlbm_t* h);

/* Fault injection from the host, for tests of the error paths (nothing
 * faults, traps or hangs the GPU):
 *   HLBM_FAULT_STALL_TILE: during the next hlbm_step's FV launch, tile
 *     `arg` never releases its progress counter, and the neighbour waits
 *     give up after 4096 polls; its neighbours then set
 *     HLBM_ST_SYNC_TIMEOUT and the abort flag and every tile returns.
 *   HLBM_FAULT_NAN_LATTICE: NaN is copied (cudaMemcpy from the host) into
 *     the nine populations of lattice node `arg` (= y * nx + x) that the
 *     next stream-collide reads; it reaches the force within some steps
 *     when the node is near the patch.
 * HLBM_EINVAL for another kind or an argument out of range. */
#define HLBM_FAULT_STALL_TILE 1
#define HLBM_FAULT_NAN_LATTICE 2
int hlbm_inject_fault(hlbm_t* h, int32_t kind, int64_t arg);

/* Copy the force history (per unit length, fluid on lamina) for times
 * first .. first+count-1 into fx, fy.  Time 0 is the initial state.
 * Synchronises the stream; returns the error of any device status bit
 * (see hlbm_step) after the copy. */
int hlbm_force(hlbm_t* h, int64_t first, int64_t count, double* fx, double* fy);

/* Hydrodynamic function Theta = F-hat / ((pi/4) rho0 w^2 L^2 A) from a
 * least-squares fit F_y(t) = a sin(w t) + b cos(w t) over
 * t in [discard_periods, discard_periods + fit_periods] periods (Sec. 2.1;
 * the paper discards 1 period and fits 3).  re = a/N, im = b/N; rms is the
 * fit residual in the same units.  HARMONIC motion only.  Returns the error
 * of any device status bit (see hlbm_step). */
int hlbm_gamma(hlbm_t* h, double discard_periods, double fit_periods, double* re, double* im,
               double* rms);

/* Macroscopic fields at the current time: lattice [ny*nx] (values at
 * nodes that are not discretization nodes are unspecified) and patch
 * [n_nodes].  Any pointer may be NULL. */
int hlbm_get_fields(hlbm_t* h, double* rho_s, double* ux_s, double* uy_s, double* rho_u,
                    double* ux_u, double* uy_u);

/* Coarser lattice level k (1 .. n_levels): rho, ux, uy [ny_k*nx_k] at its
 * current time (the solver's time rounded down to a multiple of 2^k).
 * Nodes over a node of the finer level that was not computed (under the
 * lamina) hold rho0 and zero velocity.  HLBM_EINVAL for another k. */
int hlbm_get_level_fields(hlbm_t* h, int32_t level, double* rho, double* ux, double* uy);

/* Node classes of the last step on the whole lattice [ny*nx]:
 * 0 discretization, 1 interpolation, 2 unused (Sec. 4). */
int hlbm_get_class(hlbm_t* h, int8_t* cls);

/* Refill record of the last relocation, per patch node: type 0 (wall),
 * 1, 2 or 3 (Sec. 4); donor = enclosing triangle (type 3), lattice cell
 * iy*nx+ix of the bilinear stencil (type 1), else -1. */
int hlbm_get_refill(hlbm_t* h, int32_t* type, int32_t* donor);

/* Patch populations at the current time, [n_nodes*9] node-major. */
int hlbm_get_patch_f(hlbm_t* h, double* f9);

/* FV matrices as built on the device: CSR rows per node (pivot first),
 * S_ik = c_i . (gx, gy), C_ik = cc.  Sizes from hlbm_info. */
int hlbm_get_fv(hlbm_t* h, int32_t* row_ptr, int32_t* col, double* gx, double* gy, double* cc);

typedef struct {
    int64_t time;          /* current time (steps taken)                  */
    int64_t n_struct;      /* nx*ny                                        */
    int64_t n_struct_disc; /* discretization nodes in the last step       */
    int32_t n_nodes, n_tris, nnz, n_outer, n_wall_segments;
    int32_t box_w, box_h;  /* lattice window that follows the patch       */
    int32_t launches_per_step; /* kernels per step (with levels: the most)     */
    int32_t dtype;
    int32_t fv_kernel; /* HLBM_FV_* in use                                */
    int32_t n_tiles;   /* FV tiles (blocks of the FV launch)               */
    double y, vy;      /* lamina displacement and velocity at `time`       */
    int32_t n_levels;       /* coarser lattice levels                     */
    int64_t n_coarse;       /* nodes of all coarser levels                */
    double coarse_updates;  /* their node updates per step, sum N_k / 2^k */
    int32_t fv_depth;       /* HLBM_FV_DEEP: sub-steps between exchanges (else 1) */
    int32_t fv_slots;       /* HLBM_FV_DEEP: most slots (own and ghost nodes) of a tile */
} hlbm_info_t;
int hlbm_info(hlbm_t* h, hlbm_info_t* info);

/* Exchange interval of the HLBM_FV_DEEP kernel.  The method's FV sub-steps
 * (Sec. 3, eq. ulbe) are unchanged; this sets how the GPU's tiles share
 * their boundary data.  Each FV tile keeps `depth` layers of ghost
 * nodes around its own nodes and recomputes them, so that tiles exchange
 * records once every `depth` sub-steps instead of every sub-step; deeper
 * layers cost redundant work and shared memory.  The tiles are rebuilt
 * with the largest interval up to `depth` (1 .. HLBM_FV_MAX_DEPTH) that
 * fits on the device (default 2); the results do not change, bit for bit.
 * Synchronises the stream.  HLBM_EINVAL for another depth. */
#define HLBM_FV_MAX_DEPTH 4
int hlbm_set_fv_depth(hlbm_t* h, int32_t depth);

/* Overlap of the lattice and the patch (enable = 1, the default): with an
 * FP32 lattice, the deep-tile FV kernel, one lattice level and a prescribed
 * motion, the FV launch of step t also runs step t+1's stream-collide of
 * every lattice node outside step t+1's window and the nodes pulling from it
 * (the only nodes that step t+1's relocation, classification and eq. 178
 * feed change), on warps of its own; step t+1's stream-collide then covers
 * that rectangle alone.  The results are the same bits either way.  Across
 * hlbm_step calls the precomputed part is kept (hlbm_load, hlbm_clear_status
 * and an injected lattice fault drop it).  enable = 0 runs each step's
 * stream-collide whole, before its FV launch. */
int hlbm_set_overlap(hlbm_t* h, int32_t enable);

/* The share (0, 1] of the lattice rows, from y = 0, whose part away from the
 * patch the FV launch streams under the overlap; the next step's
 * stream-collide covers the other rows with its rectangle (default 0.85:
 * the FV launch then ends about when its far lattice does).  Results do not
 * change.  HLBM_EINVAL outside (0, 1]. */
int hlbm_set_overlap_share(hlbm_t* h, double share);

/* Per-phase device time, measured with CUDA events recorded on the
 * solver's stream around each phase of hlbm_step while profiling is on.
 * hlbm_profile(h, 1) starts recording and clears the totals; (h, 0) stops.
 * hlbm_profile_read fills ms[HLBM_N_PHASES] (summed milliseconds) and
 * launches[HLBM_N_PHASES] (kernel launches) and synchronises the stream. */
#define HLBM_PHASE_MOVE 0   /* refill, classification, eq. 178 feed      */
#define HLBM_PHASE_STREAM 1 /* lattice stream-collide (eq. LBE)          */
#define HLBM_PHASE_FV 2     /* outer-node feed and FV sub-steps          */
#define HLBM_PHASE_FORCE 3  /* force on the lamina                       */
#define HLBM_N_PHASES 4
int hlbm_profile(hlbm_t* h, int enable);
int hlbm_profile_read(hlbm_t* h, double* ms, int64_t* launches);

/* Device status bits (HLBM_ST_*), accumulated since creation. */
int hlbm_status(hlbm_t* h, uint32_t* bits);

/* ---- batched sweep: independent solvers stepped together ----------------
 * The paper runs a parametric study over (beta, eps) (Sec. 2, Sec. 6);
 * a sweep steps many solvers with one call.  Each lattice step, every
 * instance issues its lattice part (relocation, classification, eq. 178
 * feed, stream-collide) on a stream of its own; the FV sub-steps of the
 * instances follow one another on a single stream, each starting as soon
 * as its instance's lattice part is done; each instance then issues its
 * force.  The solvers stay owned by the caller (destroy them after the
 * sweep) and keep their own force history, fields and status; their own
 * streams are ordered after the sweep's work when a sweep call returns.
 * All work starts after, and cuda_stream waits for, the sweep's calls. */
typedef struct hlbm_sweep hlbm_sweep_t;
int hlbm_sweep_create(int32_t n, hlbm_t* const* solvers, void* cuda_stream, hlbm_sweep_t** out);
int hlbm_sweep_step(hlbm_sweep_t* w, int64_t nsteps);
/* Tile-size autotuner for the FV kernels: for each candidate size (256,
 * 512, 1024, 1536 nodes per tile) every instance is re-tiled and
 * trial_steps sweep steps are timed per instance; each instance keeps the
 * fastest.  The trial steps advance the solvers like hlbm_sweep_step.
 * tile_nodes (may be NULL) receives the chosen size per instance. */
int hlbm_sweep_tune(hlbm_sweep_t* w, int32_t trial_steps, int32_t* tile_nodes);
/* nsteps sweep steps with the FV time of each instance summed into fv_ms[n]. */
int hlbm_sweep_fv_time(hlbm_sweep_t* w, int64_t nsteps, double* fv_ms);
/* Packs the sweep's solvers into shared FV launches (enable = 1): solvers of
 * the same precision whose sub-step counts lie within 25 % of each other,
 * up to 16, are retiled so that together they take one block per SM, and
 * each lattice step runs their FV sub-steps in one cooperative launch of the
 * tensor-memory kernel (each solver keeps its own tables, counters and
 * buffers).  Solvers with outer_fv = 1 or a forced fv_kernel stay alone.
 * A group whose tiles the tensor-memory kernel cannot hold even with more,
 * smaller tiles stays unpacked.  enable = 0 undoes it (the tuner's tiling,
 * or the default one before hlbm_sweep_tune).  n_packs (may be NULL) receives
 * the number of packs.  Results do not change: a node's arithmetic does not
 * depend on its tile or launch.  hlbm_sweep_tune after this call undoes it. */
int hlbm_sweep_pack(hlbm_sweep_t* w, int32_t enable, int32_t* n_packs);
const char* hlbm_sweep_last_error(const hlbm_sweep_t* w);
void hlbm_sweep_destroy(hlbm_sweep_t* w);

/* Gradient of the hydrodynamic function with respect to the motion's A and
 * omega and to tau_s, by central differences: seven solvers (the base point
 * and each parameter moved by -/+ rel_step times its value) are created from
 * the given inputs (as hlbm_create), stepped nsteps together as one sweep
 * (hlbm_sweep_*), and each fitted over the same steps
 * [ceil(discard_periods T), floor((discard_periods + fit_periods) T)] of the
 * base period T = 2 pi / omega, with its own omega and A in the fit and the
 * normalisation (Sec. 2.1).  theta[2] receives (Re, Im) Theta at the base
 * point; grad[6] receives d(Re, Im)/dA, d(Re, Im)/domega, d(Re, Im)/dtau_s.
 * sweep_ms (may be NULL) receives the device time of the seven solves.
 * HARMONIC motion only; 0 < rel_step < 0.1.  The discrete decisions of the
 * method (node classes, donors) make Theta piecewise smooth in A and omega:
 * the quotient is that of the moved runs, jumps included.  Errors as for
 * hlbm_create (message: hlbm_last_error(NULL)); everything created is
 * released before the call returns. */
int hlbm_theta_gradient(const hlbm_grid_t* grid, const hlbm_patch_t* patch, double tau_s,
                        const hlbm_motion_t* motion, int64_t nsteps, double discard_periods, double fit_periods,
                        double rel_step, void* cuda_stream, double* theta, double* grad, double* sweep_ms);

/* Gradient of the hydrodynamic function by the adjoint (reverse mode) of the
 * discrete hybrid step.  A solver is created from the inputs (as
 * hlbm_create), stepped nsteps with its dynamic state checkpointed in
 * device memory every checkpoint_every steps, and Theta is fitted over the
 * steps [ceil(discard_periods T), floor((discard_periods + fit_periods) T)],
 * T = 2 pi / omega (Sec. 2.1, eq. force_phasor).  For the objective
 * L = w_re Re Theta + w_im Im Theta, the reverse sweep then visits the
 * segments between checkpoints from the last to the first: each is stepped
 * again from its checkpoint keeping what every step's reverse needs, and
 * the steps are reversed one by one -- force, the n FV sub-steps of eq. ulbe
 * (recomputed), the outer-node feed (eq. postcollision2_u), stream-collide
 * (eq. LBE), the eq. postcollision2_s fill and the refill of Sec. 4 -- with
 * every decision of the forward step held fixed (node classes, refill types,
 * donor cells and triangles; Theta is smooth in the parameters between
 * them).  theta[2] receives (Re, Im) Theta, grad[3] dL/dA, dL/domega,
 * dL/dtau_s (A and omega through the positions y(t) = A sin(w t), the wall
 * velocity and the fit; tau_s through 1/tau_s, 1/tau_u, and the interface
 * factors 2 (tau_s - 1)/(2 tau_s - 1) and 1 - 1/(2 tau_s)).  fwd_ms and bwd_ms
 * (may be NULL) receive the device time of the checkpointed forward run and
 * of the reverse sweep.  HARMONIC motion, one lattice level, outer_fv = 0,
 * no absorbing layer (sponge_rows = 0), FP64 or FP32 populations (adjoints
 * in the population type, the parameter sums in FP64).  Device memory: one lattice
 * copy per checkpoint and per step of a segment, released before the call
 * returns.  Errors as for hlbm_create (message: hlbm_last_error(NULL)). */
int hlbm_theta_adjoint(const hlbm_grid_t* grid, const hlbm_patch_t* patch, double tau_s, const hlbm_motion_t* motion,
                       int64_t nsteps, double discard_periods, double fit_periods, double w_re, double w_im,
                       int32_t checkpoint_every, void* cuda_stream, double* theta, double* grad, double* fwd_ms,
                       double* bwd_ms);

/* Least-squares fit F(t) = a sin(w t) + b cos(w t) over t = t0..t1 of the
 * samples F(t) = samples[t * stride] (DEVICE memory, caller-owned, at least
 * t1 * stride + 1 doubles), the fit hlbm_gamma performs, for callers that
 * must not allocate device memory: code running under a fixed
 * device-memory budget or inside a framework that owns all allocations, and
 * loops that cannot take the device-wide synchronisation of cudaMalloc /
 * cudaFree.  The paper has no counterpart; it is an interface of this
 * library.  (A solver's force history interleaves F_x and F_y: pass its F_y
 * column with stride 2.)
 *
 * Allocates nothing: its intermediate sums live in a file-scope device
 * array of 257 x 8 doubles that every GPU loading the library holds until
 * the process exits.  The first call on a device (and the first after the
 * device's context was destroyed, e.g. by cudaDeviceReset) looks up that
 * array's device address with cudaGetSymbolAddress.  Calls share the array:
 * every value a call reads is written earlier in the same call, but calls
 * that overlap on the GPU (other streams or host threads) race and must be
 * serialised by the caller.  Work is queued on cuda_stream (a cudaStream_t,
 * NULL = legacy default stream), which is synchronised before a, b and rms
 * (host pointers; rms may be NULL) are written.  Returns HLBM_EINVAL for
 * more than 2^26 samples, t1 <= t0, t0 < 0, stride < 1, omega not finite
 * and positive, a stream that is being captured (the call reads its
 * results back to the host), or sin(w t) and cos(w t) nearly dependent over
 * the window (det of the normal equations below 1e-12 n^2 for n samples,
 * e.g. w a multiple of pi); HLBM_ECUDA when a CUDA call or a launch fails. */
int hlbm_fit_static(const double* samples, int64_t stride, int64_t t0, int64_t t1, double omega,
                    void* cuda_stream, double* a, double* b, double* rms);

/* Checkpoint and restart.  hlbm_save writes the solver's dynamic state at
 * its current step t to the file `path` (a host path; the file is replaced):
 * both lattice population buffers, the window classes and states, both
 * patch record buffers, the latest refill record, the force history
 * 0..t, the status word, and the step counters.  It synchronises the
 * solver's stream first.  hlbm_load restores such a file into a solver
 * created from the same inputs (lattice, boundaries, dtype, patch mesh,
 * physics and motion, checked against the file's header and a hash of the
 * mesh); stepping on from there gives bit for bit the fields, refill
 * records and forces the saved solver would have given.  Geometry, FV
 * matrices and tile tables are not stored: hlbm_create rebuilds them.
 * The file is in the host's byte order and holds, after a fixed header,
 * about 18 * nx * ny * sizeof(population) bytes.
 * Returns HLBM_EIO when the file cannot be opened, written or read, is
 * not a checkpoint or is not complete; HLBM_EINVAL when it belongs to other
 * inputs; HLBM_ENOMEM when the longer force history cannot be allocated --
 * in these cases before anything of the solver is changed; HLBM_ECUDA on a
 * failed copy, which leaves the solver's state undefined. */
int hlbm_save(hlbm_t* h, const char* path);
int hlbm_load(hlbm_t* h, const char* path);

/* Message of the last failed call on h; with h == NULL, of the last failed
 * hlbm_create on this thread. */
const char* hlbm_last_error(const hlbm_t* h);
void hlbm_destroy(hlbm_t* h);

#ifdef __cplusplus
}
#endif
#endif
