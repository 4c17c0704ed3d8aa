/*
 * lbm.h -- C ABI of the GB300 LBGK-LPT bubble-column library (liblbm.so).
 *
 * The library advances one liquid column, discretised with the D3Q19 BGK
 * lattice Boltzmann model, two-way coupled to Lagrangian point bubbles, as
 * stated in arXiv:1710.07073:
 *   - liquid: BGK collision with Guo forcing and streaming (Sec. 2.2,
 *     Eq. 5-16), half-way bounce-back on wall faces (Sec. 3.3);
 *   - bubbles: Newton's law with buoyancy, drag and added mass
 *     (Sec. 2.1, Eq. 1-4, Table 1), sub-stepped as in Table 2;
 *   - coupling: clipped fourth-order polynomial mapping (Sec. 3.2,
 *     Eq. 18-21) for interpolation to the bubbles and spreading back;
 *   - order of operations: Algorithm 1.
 *
 * Units are lattice units: dx = dt_l = 1, lattice speed e = 1.  Gravity acts
 * along -z.  Every array crossing this ABI is a HOST array owned by the
 * caller; the library copies in and out.  The library owns all device memory
 * (allocated with cudaMalloc, or with the caller's allocator when one is set
 * with lbm_set_allocator before the first device use).
 *
 * Layouts.  Site (i, j, k), 0 <= i < nx etc., has linear index
 * s = (k * ny + j) * nx + i (x fastest).  Scalar fields are double[S],
 * S = nx*ny*nz.  Vector fields are structure-of-arrays double[3*S]
 * (all x components, then y, then z).  Per-bubble vectors are
 * interleaved double[3*n] (x0, y0, z0, x1, ...).  Populations are
 * double[19*S], direction-major, in the order returned by lbm_velocity_set.
 *
 * Errors.  Every int-returning call returns LBM_OK (0) or a negative
 * LBM_ERR_* code; the context keeps a message readable with
 * lbm_last_error.  LBM_ERR_UNSTABLE is sticky: once the liquid solver has
 * flagged a non-finite value or |u| >= 0.3 (beyond the low-Mach range of
 * Eq. 6), or a bubble has moved more than 4 cells along an axis in one step
 * (a lattice speed of 4), every later lbm_step returns it until the state is
 * reset with lbm_set_fields or lbm_set_populations.
 *
 * Threads.  A context may be used from one host thread at a time.  All work
 * is enqueued on the context's CUDA stream (lbm_set_stream); calls that
 * return host data synchronise that stream.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define LBM_OK            0
#define LBM_ERR_ARG      -1   /* invalid argument; nothing was changed        */
#define LBM_ERR_ALLOC    -2   /* device allocation failed                     */
#define LBM_ERR_UNSTABLE -3   /* liquid solver produced NaN/Inf or |u|>=0.3  */
#define LBM_ERR_TIMEOUT  -4   /* reserved: a bounded device wait ran out      */
#define LBM_ERR_CUDA     -5   /* a CUDA runtime call failed                   */
#define LBM_ERR_STATE    -6   /* call not valid in the current state          */

/* ---- walls: one bit per box face; a set bit is a half-way bounce-back
 * no-slip wall (Sec. 3.3), a clear bit makes the axis periodic.  Both faces
 * of an axis must agree.  LBM_TOP_FREE_SLIP, with LBM_WALL_ZP set, makes the
 * +z face a free-slip plane half-way above the top layer instead (Sec. 3.3:
 * free-slip top): a population leaving through it is reflected specularly,
 * c_z reversed and the tangential components kept, into the top layer one
 * tangential step along; a link that also crosses a no-slip face bounces
 * back.  Bubbles treat the face like a wall (clipped windows, clamped
 * centres, the stop at the top).  LBM_WALL_ALL_FREE_TOP: no-slip everywhere
 * but the free-slip top. --------------------------------------------------- */
#define LBM_WALL_XM  0x01
#define LBM_WALL_XP  0x02
#define LBM_WALL_YM  0x04
#define LBM_WALL_YP  0x08
#define LBM_WALL_ZM  0x10
#define LBM_WALL_ZP  0x20
#define LBM_WALL_ALL 0x3F
#define LBM_TOP_FREE_SLIP 0x40
#define LBM_WALL_ALL_FREE_TOP 0x7F

/* ---- population storage precision (collision arithmetic is always FP32).
 * Populations are stored shifted by their rest-state value w_j * rho_l:
 *   F32 : f_j - w_j rho_l
 *   F16 / BF16 : (f_j - w_j rho_l) * scale / w_j, rounded to nearest even. */
#define LBM_STORE_F32  0
#define LBM_STORE_F16  1
#define LBM_STORE_BF16 2

/* Largest bubble diameter accepted (lattice units); the mapping window
 * n = width_factor * d must fit the library's fixed tile bookkeeping. */
#define LBM_MAX_DIAMETER 6.0

typedef struct lbm_ctx lbm_ctx;

/* Closure and coupling parameters, lattice units (Table 1, Table 2, Eq. 3). */
typedef struct lbm_params {
    double g;             /* gravity magnitude, acting along -z            */
    double rho_l;         /* liquid density; also the storage shift rho_0   */
    double rho_ratio;     /* rho_b / rho_l                                  */
    double sigma;         /* surface tension (enters Eo, Eq. 3)             */
    double c_added_mass;  /* C_A of the virtual-mass force (Table 1: 0.5)   */
    double drag_scale;    /* multiplies F_D (1.0 = Table 1)                 */
    double sn_coeff;      /* a in 24/Re (1 + a Re^b) (0.15)                 */
    double sn_exp;        /* b in 24/Re (1 + a Re^b) (0.687)                */
    double width_factor;  /* mapping half-width n = width_factor * d_b (1.5)*/
    int    substeps;      /* bubble sub-steps per liquid step (Table 2: 10) */
    int    two_way;       /* 1: spread the reaction onto the liquid (Eq. 21)*/
    int    forces;        /* LBM_FORCE_* bits: the Table 1 forces beyond    */
                          /* buoyancy, drag and virtual mass (0: none)      */
    int    mapping;       /* LBM_MAP_CELL (Eq. 19) or LBM_MAP_POINT         */
    int    reaction;      /* LBM_REACTION_DRAG_LIFT or LBM_REACTION_ALL     */
} lbm_params;

/* Mapping weights (lbm_params.mapping), for interpolation (Eq. 20) and
 * spreading (Eq. 21) alike, renormalised over the in-box nodes either way:
 *   LBM_MAP_CELL   the cell integral of Z over the node's cell (Eq. 19);
 *   LBM_MAP_POINT  Z sampled at the node, times the cell width.  The node
 *                  samples sum to one only up to the midpoint rule's error
 *                  (below 0.15 n^-3), which the renormalisation removes.
 *                  Needs n = width_factor d_b > 1/2 for every bubble, so
 *                  that the nearest node lies inside the window
 *                  (lbm_set_bubbles returns LBM_ERR_ARG otherwise).
 * The mapping can change only while the context holds no bubbles
 * (LBM_ERR_STATE otherwise). */
#define LBM_MAP_CELL  0
#define LBM_MAP_POINT 1

/* Reaction spread onto the liquid (lbm_params.reaction), averaged over the
 * bubble sub-steps of a liquid step:
 *   LBM_REACTION_DRAG_LIFT  psi_b = -(F_D + F_L) (Algorithm 1 step 6);
 *   LBM_REACTION_ALL        psi_b = -sum F over the interphase forces of
 *                           Table 1 (Sec. 3.2): F_D + F_L + F_S + F_VM with
 *                           F_VM = C_A rho_l V_b (D_t u_l - D_t u_b), D_t u_b
 *                           the sub-step's acceleration.  Gravity and the
 *                           hydrostatic part of F_B are not passed back, so
 *                           psi_b = F_B - m_b (u_b^{n+1} - u_b^n)/dt_l, and
 *                           the mixture's momentum grows by sum F_B per step. */
#define LBM_REACTION_DRAG_LIFT 0
#define LBM_REACTION_ALL       1

/* Optional interface forces of Table 1 (lbm_params.forces):
 *   LBM_FORCE_LIFT    F_L = -C_L rho_l V_b (u_b - u_l) x (curl u_l) with
 *                     Table 1's C_L(Re, Eo_d) (f(Eo_d) carries the published
 *                     constant 0.474 that the printed table drops); the
 *                     liquid vorticity is the central difference of the
 *                     Eq. 10 velocity at the nodes (ghost -u beyond a no-slip
 *                     wall, +u tangential beyond a free-slip top), interpolated
 *                     with Eq. 19-20 like the velocity (Algorithm 1 step 3).
 *                     The reaction is -(F_D + F_L) (Algorithm 1 step 6).  The
 *                     windows reach one cell further, so on a periodic axis
 *                     2n + 4 <= L.
 *   LBM_FORCE_STRESS  F_S = rho_l V_b D_t u_l, with the virtual mass's
 *                     D_t u_l. */
#define LBM_FORCE_LIFT   0x1
#define LBM_FORCE_STRESS 0x2

typedef void* (*lbm_alloc_fn)(size_t bytes, void* user);
typedef void  (*lbm_free_fn)(void* ptr, size_t bytes, void* user);

/* Fill *p with the defaults: g=1e-5, rho_l=1, rho_ratio=1e-3,
 * sigma=5.84e-6, C_A=0.5, drag_scale=1, sn_coeff=0.15, sn_exp=0.687,
 * width_factor=1.5, substeps=10, two_way=1, forces=0, mapping=LBM_MAP_CELL,
 * reaction=LBM_REACTION_DRAG_LIFT. */
void lbm_default_params(lbm_params* p);

/* Velocity set and weights in the library's direction order (Eq. 7-8):
 * c[3*j + a] is component a of c_j, w[j] its weight.  Either may be NULL. */
void lbm_velocity_set(int* c57, double* w19);

/* ---- physical units (Appendix A) -------------------------------------------
 * A physical set-up (SI units) and its lattice: Delta x_lu = Delta t_lu = 1,
 * so the conversion factors lattice-per-physical are LCF = 1/dx, TCF = 1/dt
 * and, from rho_pu = rho_lu LCF^3 / MCF, MCF = rho_lu LCF^3 / rho_pu.  A
 * quantity of dimension m^a s^b kg^c converts as x_lu = x_pu LCF^a TCF^b
 * MCF^c: lengths by LCF, times by TCF, velocities by LCF/TCF, g by
 * LCF/TCF^2, kinematic viscosity by LCF^2/TCF, surface tension (kg/s^2) by
 * MCF/TCF^2. */
typedef struct lbm_physical {
    double dx;        /* grid spacing Delta x, m                          */
    double dt;        /* liquid time step Delta t_l, s                    */
    double rho_l;     /* liquid density, kg/m^3                           */
    double rho_b;     /* bubble density, kg/m^3                           */
    double mu_l;      /* liquid dynamic viscosity, kg/(m s)               */
    double sigma;     /* surface tension, N/m                             */
    double g;         /* gravity, m/s^2                                   */
    double rho_l_lu;  /* liquid density in lattice units (Appendix A: 1)  */
} lbm_physical;

typedef struct lbm_units {
    double lcf, tcf, mcf;   /* lattice per physical: length, time, mass     */
} lbm_units;

/* Convert a physical set-up to lattice units (Appendix A).  Fills *u with
 * the factors; *p (if not NULL) gets g, rho_l = rho_l_lu, rho_ratio, sigma in
 * lattice units, the other fields untouched (call lbm_default_params first);
 * *omega (if not NULL) gets the relaxation frequency of nu_lu = (mu_l/rho_l)
 * LCF^2/TCF by Eq. 9, omega = 1/(3 nu_lu + 1/2).  Returns LBM_ERR_ARG for a
 * non-positive or non-finite input or rho_b >= rho_l.  A set-up with water's
 * viscosity at millimetre cells gives omega just below 2 (Appendix A's 4 mm
 * case: nu_lu = 4e-6, omega = 1.99995); the conversion does not check
 * stability. */
int lbm_units_from_physical(const lbm_physical* ph, lbm_units* u, lbm_params* p,
                            double* omega);

/* Create a context for an nx*ny*nz column with relaxation frequency omega
 * (Eq. 9: nu = (1/omega - 1/2)/3; omega must lie in (0, 2)) and the given
 * wall bits, FP32 storage.  The liquid starts at f = f^eq(rho_l, 0)
 * (Algorithm 1 initialisation).  Device memory is allocated on first use.
 * Returns LBM_ERR_ARG for non-positive sizes, 19 S >= 2^32, omega out of
 * range or mismatched wall bits. */
int lbm_create(int nx, int ny, int nz, double omega, unsigned walls, lbm_ctx** out);

/* As lbm_create with a storage precision (LBM_STORE_*) and, for the 16-bit
 * formats, the scale applied after dividing by w_j (ignored for F32). */
int lbm_create_storage(int nx, int ny, int nz, double omega, unsigned walls,
                       int storage, double scale, lbm_ctx** out);

/* Free the context and all device memory it owns.  NULL is ignored. */
void lbm_destroy(lbm_ctx* ctx);

/* Use this CUDA stream (a cudaStream_t passed as void*) for all work. */
int lbm_set_stream(lbm_ctx* ctx, void* stream);

/* Route device allocations through alloc/free (e.g. a framework's caching
 * allocator).  Must come before the first call that touches the device. */
int lbm_set_allocator(lbm_ctx* ctx, lbm_alloc_fn alloc, lbm_free_fn free_fn, void* user);

int lbm_set_params(lbm_ctx* ctx, const lbm_params* p);
int lbm_get_params(const lbm_ctx* ctx, lbm_params* p);

/* Set the liquid to f = f^eq(rho, u) (Eq. 6; Algorithm 1 initialisation).
 * rho: double[S] or NULL for rho_l everywhere; u3: double[3*S] SoA or NULL
 * for rest.  Clears the sticky instability flag. */
int lbm_set_fields(lbm_ctx* ctx, const double* rho, const double* u3);

/* Set the pre-collision populations f_j(x, t) directly (double[19*S] in
 * lbm_velocity_set order).  Clears the sticky instability flag. */
int lbm_set_populations(lbm_ctx* ctx, const double* f);

/* Read the pre-collision populations f_j(x, t) (double[19*S]). */
int lbm_get_populations(lbm_ctx* ctx, double* f);

/* Replace all bubbles.  pos3/vel3: double[3*n] interleaved; diam: double[n].
 * Each centre must lie inside the box, 0 < d <= LBM_MAX_DIAMETER, and on a
 * periodic axis the window must not wrap onto itself (2n + 2 <= L).  All
 * bubbles start active with no liquid-velocity history (D_t u_l = 0 on
 * their first step).  n = 0 removes all bubbles. */
int lbm_set_bubbles(lbm_ctx* ctx, int n, const double* pos3, const double* vel3,
                    const double* diam);

/* Advance nsteps coupled steps (Algorithm 1 loop body), each:
 *   1. per active bubble: interpolate the bare Eq. 10 liquid velocity of the
 *      current populations to the centre (Eq. 19-20, window renormalised
 *      over in-box nodes), run `substeps` explicit Newton updates (Eq. 4)
 *      with m_eff = m_b + C_A rho_l V_b, form psi_b = -mean F_D;
 *   2. bin the bubbles' windows to lattice tiles (Algorithm 1 step 2);
 *   3. one fused collide-stream sweep: each node gathers its force Phi from
 *      the bubbles binned to its tile (Eq. 21, fixed order, no atomics),
 *      applies Eq. 13, 6, 14, 12, 15 and streams (Eq. 16) with bounce-back;
 *   4. a bubble whose centre reached nz - r_b under a +z wall is deactivated
 *      (Algorithm 1, stop at the top) after spreading this step.
 * With few bubbles (the single-launch binning) on even-nx lattices, a step's
 * sweep may start while its bubble update still runs: lattice z layers that
 * no bubble can reach this step (support widened by 4 cells) do not wait for
 * it.  Results are the same bits as with the two in stream order (which the
 * library keeps while kernel timing is on).  With many bubbles, or few
 * bubbles in a lattice of 2^24 sites or more, on even-nx lattices whose z
 * axis is wall-bounded, a step forks from the context stream into two
 * library streams: a high-priority one for the bubble update, the binning
 * and the sweep of the z blocks bubble forces can reach, and a low-priority
 * one for the sweep of the other blocks, which needs no forces; the step
 * joins the context stream again before it ends.  The reachable blocks are
 * those of the binning (many bubbles) or of the update's guard (few) two
 * steps before, widened by one tile layer per step (a bubble moving farther
 * is flagged).  Same bits as stream order.  psi_b is -mean(F_D + F_L) unless lbm_params.reaction says
 * otherwise.
 * Returns after the work has completed, with LBM_ERR_UNSTABLE if flagged. */
int lbm_step(lbm_ctx* ctx, int nsteps);

/* Liquid density and bare Eq. 10 velocity u = sum c f / rho of the current
 * pre-collision populations.  Either pointer may be NULL. */
int lbm_get_fields(lbm_ctx* ctx, double* rho, double* u3);

/* Copy out up to `cap` bubbles.  Any output pointer may be NULL.
 * pos3, vel3: state after the last step; ul3: liquid velocity interpolated at
 * the start of the last step; psi3: reaction spread in the last step;
 * active: 1 while the bubble is coupled.  *n receives the bubble count. */
int lbm_get_bubbles(lbm_ctx* ctx, int cap, int* n, double* pos3, double* vel3,
                    double* ul3, double* psi3, int* active);

/* FP64 totals over the box: out4 = {sum rho, sum rho u_x, sum rho u_y,
 * sum rho u_z} of the current pre-collision populations (Eq. 10). */
int lbm_get_totals(lbm_ctx* ctx, double* out4);

/* Binning of the last step (Algorithm 1 step 2), for inspection.
 * cell: int[n] linear id of the cell holding each bubble after its update
 * (-1 when inactive); tile3: the tile shape (tx, ty, tz); *ntiles: tile
 * count; offsets: int[ntiles+1]; items: int[cap_items] bubble ids, per tile in
 * ascending order; *nitems: number of ids.  Any pointer may be NULL. */
int lbm_get_bins(lbm_ctx* ctx, int* cell, int* tile3, int* ntiles, int* offsets,
                 int* items, int cap_items, int* nitems);

/* Number of lattice sites and bytes of population storage per site and step
 * (read + write of all 19 populations). */
long long lbm_sites(const lbm_ctx* ctx);
int lbm_bytes_per_site(const lbm_ctx* ctx);

/* Per-launch timing of the fused collide-stream kernel: when on, each launch
 * is bracketed by CUDA events on the context stream; lbm_get_kernel_time
 * returns the summed milliseconds and the launch count since timing was
 * switched on (synchronises the stream). */
int lbm_set_kernel_timing(lbm_ctx* ctx, int on);
int lbm_get_kernel_time(lbm_ctx* ctx, double* ms, int* launches);

/* ---- Reverse mode: gradients of a terminal-velocity mismatch ----------------
 * Objective: L = (ubar - target)^2, where ubar is the bubble rise velocity
 * u_b,z averaged over all bubbles and over the last `window` of `nsteps`
 * coupled steps (the terminal velocity of Sec. 4.1 / Table 4).
 *
 * lbm_adj_forward advances the context by nsteps steps exactly as lbm_step
 * does, keeping a checkpoint of the full state every `checkpoint_every`
 * steps, and returns L.  lbm_adj_backward then runs the hand-written adjoint
 * of every step in reverse (each segment between checkpoints is recomputed
 * forward first) and returns, scaled by dloss (= dOuter/dL):
 *   grad_drag_scale  dL/ds_D, s_D the drag scale of lbm_params;
 *   grad_diam        double[n] dL/dd_b per bubble (volume, mass, buoyancy,
 *                    drag closure and the mapping window n = width_factor d_b);
 *   grad_u0          double[3*S] SoA dL/du0, the initial liquid velocity, for
 *                    initial populations f = f^eq(rho, u0) as lbm_set_fields
 *                    sets them (NULL to skip).
 * Wall contacts of the bubble (clamped centre) and the stop at the top are
 * treated as fixed switches.  Needs FP32 storage, 1..256 bubbles.  After the
 * backward the context is back at the state the forward ended in.  Any call
 * that changes the state between the two (lbm_step, lbm_set_*) discards the
 * record; lbm_adj_backward then returns LBM_ERR_STATE.  A free-slip top
 * (LBM_TOP_FREE_SLIP), the optional forces (lbm_params.forces), point-sampled
 * mapping and the -sum F reaction are not covered: lbm_adj_forward returns
 * LBM_ERR_STATE.
 * Each reverse step runs the bubbles' spreading adjoint and sub-step reverse
 * (a CTA per bubble) on a second, library-owned stream alongside the per-node
 * sweep, and joins them through events before the interpolation adjoint.
 * Memory: one state per
 * checkpoint plus checkpoint_every states during the backward.  With kernel
 * timing on (lbm_set_kernel_timing), lbm_adj_backward times each launch of
 * the per-node adjoint sweep instead of the forward collide-stream. */
int lbm_adj_forward(lbm_ctx* ctx, int nsteps, int checkpoint_every, int window, double target,
                    double* loss);
int lbm_adj_backward(lbm_ctx* ctx, double dloss, double* grad_drag_scale, double* grad_diam,
                     double* grad_u0);

/* ---- Batches: many independent columns in one launch ---------------------
 * The grid-independence and stability studies of the paper (Sec. 4.2-4.3,
 * Tables 5-6, Fig. 5) run the same single-bubble problem on many columns of
 * different size and relaxation frequency.  A batch advances such columns
 * together: per coupled step one bubble-update launch for all columns (binning
 * fused behind it) and one persistent collide-stream launch over all columns'
 * work items; pairs of steps are captured into a CUDA graph and replayed.
 * Each column follows exactly the single-column step (the results are
 * identical to lbm_step on that column alone).
 *
 * Limits: every nx must be even; at most 256 columns; the (tile, bubble)
 * pairs of all bubbles must fit 4096 (about 80 bubbles of d <= 4).  Storage
 * precision as in lbm_create_storage.  A batch runs on its own non-blocking
 * stream unless lbm_batch_set_stream gives one (the default stream cannot be
 * captured). */
typedef struct lbm_batch lbm_batch;

/* dims3: int[3*ncols] (nx, ny, nz per column); omegas: double[ncols] in
 * (0, 2); walls: unsigned[ncols] or NULL for bounce-back on all faces. */
int lbm_batch_create(int ncols, const int* dims3, const double* omegas, const unsigned* walls,
                     int storage, double scale, lbm_batch** out);
void lbm_batch_destroy(lbm_batch* b);
int lbm_batch_set_stream(lbm_batch* b, void* stream);
int lbm_batch_set_allocator(lbm_batch* b, lbm_alloc_fn alloc, lbm_free_fn free_fn, void* user);
/* Closure parameters shared by all columns (rho_l only before first use). */
int lbm_batch_set_params(lbm_batch* b, const lbm_params* p);
/* counts: int[ncols] bubbles per column; pos3/vel3/diam hold them column
 * after column (positions in each column's own coordinates). */
int lbm_batch_set_bubbles(lbm_batch* b, const int* counts, const double* pos3, const double* vel3,
                          const double* diam);
/* Advance every column by nsteps coupled steps (graph replays). */
int lbm_batch_step(lbm_batch* b, int nsteps);
/* Autotuner: times each candidate launch shape -- CTA tile 32 x 4 x P nodes
 * with P in {1, 2, 4} z-planes, work-item depth in z-blocks {1, 2, 4, 8},
 * and half, one or two times the resident CTAs per SM -- for trial_steps
 * steps on this batch, keeps the fastest, and restores the state the trials
 * advanced.  Results do not depend on the shape (bit for bit).  Either output
 * may be NULL; lbm_batch_launch_shape reads the whole shape. */
int lbm_batch_tune(lbm_batch* b, int trial_steps, int* depth_out, int* grid_out);
/* The batch's current launch shape: z-planes per CTA (the CTA tile is
 * 32 x 4 x planes nodes), z-blocks per work item and persistent CTAs.  Before
 * lbm_batch_tune: planes 2, depth 2 and a grid of the resident CTAs (set on
 * first device use).  Any output may be NULL. */
int lbm_batch_launch_shape(const lbm_batch* b, int* planes, int* depth, int* grid);
/* Fix the launch shape without tuning: planes 1, 2 or 4, depth 1..64, grid
 * the persistent CTAs (0: the resident CTAs per SM times the SM count).
 * LBM_ERR_ARG otherwise. */
int lbm_batch_set_launch_shape(lbm_batch* b, int planes, int depth, int grid);
/* Fields of one column (as lbm_get_fields). */
int lbm_batch_get_fields(lbm_batch* b, int col, double* rho, double* u3);
/* All bubbles, column after column (as lbm_get_bubbles). */
int lbm_batch_get_bubbles(lbm_batch* b, int cap, int* n, double* pos3, double* vel3, double* ul3,
                          double* psi3, int* active);
long long lbm_batch_sites(const lbm_batch* b);
/* Per-launch timing of the persistent collide-stream (steps then run without
 * the graph); as lbm_set_kernel_timing / lbm_get_kernel_time. */
int lbm_batch_set_kernel_timing(lbm_batch* b, int on);
int lbm_batch_get_kernel_time(lbm_batch* b, double* ms, int* launches);
long long lbm_batch_launch_count(const lbm_batch* b);
int lbm_batch_sync(lbm_batch* b);
const char* lbm_batch_last_error(const lbm_batch* b);

/* ---- Binning that allocates nothing -------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory when they need the binning: code running while
 * a stream is captured into a CUDA graph in global capture mode (cudaMalloc is
 * an error there), runtimes that hand all device memory to their own pool at
 * start-up, and tight loops that cannot pay for the device-wide
 * synchronisation of a cudaMalloc.  It bins bubbles into tiles exactly as
 * lbm_step does (the result equals lbm_get_bins for the same centres) but
 * keeps its scratch -- LBM_NOALLOC_MAX_TILES tile counters plus the scan's
 * block sums, about 1 MiB -- in a fixed array inside the library, which every
 * GPU that loads the library holds until the process exits.  It calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *
 * All pointers are DEVICE memory owned by the caller:
 *   pos3        double[3*n]  interleaved bubble centres (inside the box);
 *   half_width  double[n]    window half-widths n_b = width_factor * d_b;
 *   active      int[n]       non-zero for bubbles to bin;
 *   tile_offsets int[T+1]    out: per-tile start into tile_items, tiles of the
 *                            shape lbm_get_bins reports, T = ceil(nx/32) *
 *                            ceil(ny/4) * ceil(nz/4), numbered x-fastest;
 *   tile_items  int[cap_items] out: bubble ids, ascending within each tile;
 *   status      int[1]       out: bit flags, 0 when all is well:
 *                            1  more than cap_items ids were due (the list
 *                               is cut);
 *                            2  a bubble was skipped: a non-finite centre or
 *                               half-width, a half-width outside
 *                               (0, LBM_NOALLOC_MAX_HALF_WIDTH], or a centre
 *                               outside [0, L) on some axis.
 * The work is enqueued on `stream` (a cudaStream_t, may be NULL) and is
 * complete when that stream is.  The first call on a device looks up the
 * scratch array's device address for that device (a CUDA runtime query);
 * make that first call before any stream capture begins.  Every call shares
 * the one scratch array and clears what it needs at its start, so calls that
 * overlap on the GPU (other streams, other host threads) race.
 * Returns LBM_ERR_ARG for bad sizes or walls, or when T exceeds
 * LBM_NOALLOC_MAX_TILES; LBM_ERR_CUDA if a CUDA call fails. */
#define LBM_NOALLOC_MAX_TILES 262144
#define LBM_NOALLOC_MAX_HALF_WIDTH 9.0
#define LBM_NOALLOC_STATUS_OVERFLOW 1
#define LBM_NOALLOC_STATUS_SKIPPED  2
int lbm_bin_bubbles_noalloc(int nx, int ny, int nz, unsigned walls, int n,
                            const double* pos3, const double* half_width, const int* active,
                            int* tile_offsets, int* tile_items, int cap_items, int* status,
                            void* stream);

/* Number of kernels this context has launched since it was created. */
long long lbm_launch_count(const lbm_ctx* ctx);

/* Name of the collide-stream kernel (step 3 of lbm_step) that the next step
 * of this context launches, for reports that pair timings with profiles:
 * the two-node sweep "k_collide_stream_pair<S,T>" (even nx with two-way
 * coupled bubbles; S the storage code, T = 1 for the tabulated force gather
 * of long tile lists), "k_collide_stream_free<S>" (even nx, no tile lists:
 * no bubbles or no two-way coupling; the many-bubble step also launches it
 * for the blocks no bubble force reaches) or "k_collide_stream<S>" (odd nx).
 * A static string; "" for NULL. */
const char* lbm_sweep_kernel(const lbm_ctx* ctx);

/* Wait for all work enqueued by this context. */
int lbm_sync(lbm_ctx* ctx);

/* Message of the last error on this context ("" if none); never NULL. */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Static name of a status code. */
const char* lbm_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
