/*
 * adg.h -- C ABI of libadg: one ADER-DG time step with a-posteriori subcell
 * (MOOD) limiting for the compressible Euler equations on 2D/3D Cartesian
 * grids, after Dumbser, Zanotti, Loubere, Diot, "A posteriori subcell limiting
 * of the discontinuous Galerkin finite element method for hyperbolic
 * conservation laws" (arXiv 1406.7416).
 *
 * Conventions shared by every entry point
 *   - Every call returns int: 0 = ADG_OK, < 0 an error, > 0 a warning.  No C++
 *     exception crosses this boundary.  adg_last_error() gives the message of
 *     the last failed call on a state.
 *   - The library owns all device memory of a state; the caller owns every
 *     host buffer it passes (read during the call only, never retained).
 *   - Work is enqueued on the state's CUDA stream (adg_set_stream; default:
 *     the legacy default stream).  Calls that copy to the host synchronize that
 *     stream before returning; adg_step does not synchronize.
 *   - Host array layouts (double unless stated):
 *       cell index   c = i + n0 * (j + n1 * k)          (x fastest)
 *       node index   l = a + n * (b + n * c3)           (x fastest), n = N + 1
 *       subcell idx  s = sx + Ns * (sy + Ns * sz)       (x fastest), Ns = 2N + 1
 *       DOFs         dofs[c][v][l],  v = 0..nvar-1, nvar = dim + 2
 *                    (rho, rho*u, rho*v, [rho*w], rho*E), nodal values at the
 *                    tensor Gauss-Legendre points of each cell (Sec. 2.1
 *                    Eq. ansatz.uh)
 *       subcells     sub[c][v][s]: subcell averages (Sec. 4.2 Eq. subcell.p)
 *       flags        beta[c]: uint8, 1 = troubled cell (Sec. 4.3)
 *
 * Precision modes (adg_create `prec`)
 *   ADG_PREC_FP64        every step of the path in FP64.
 *   ADG_PREC_MIXED_FP32  the predictor's Picard sweeps (Eq. pde.nc.dg2) run in
 *                        FP32.  For N <= 5 no FP64 sweep follows: the last
 *                        FP32 sweep yields only the space-time correction
 *                        dq = q - u, and the final stage adds it to the FP64 u
 *                        term by term (face traces as FP64 trace(u) + FP32
 *                        trace(dq); time-averaged fluxes as FP64 F(u) + FP32
 *                        flux changes).  For N >= 6 one FP64 sweep follows
 *                        the FP32 ones and the final stage is FP64
 *                        (ADG_OPT_FP64_SWEEPS changes either default).  FP64:
 *                        the corrector accumulation (Eq. pde.nc.gw2), the
 *                        detector's comparisons, the projection P and the
 *                        reconstruction R, the finite volume update of the
 *                        subcells and the neighbour flux correction.  The
 *                        detector's P(u*) is the kept FP64 P(u^n) plus an FP32
 *                        projection of the change (ADG_OPT_PROJECT_DELTA).
 *                        FP32: the subcell scheme's WENO3 reconstruction,
 *                        degree-2 predictor and sub-face fluxes
 *                        (ADG_OPT_SUBCELL_FP32); the wave speeds of the CFL
 *                        step, from the FP64 rho E - |m|^2 / 2.
 *                        Conservation stays at FP64 round-off.
 *   ADG_PREC_MIXED_TF32  ADG_PREC_MIXED_FP32 with the predictor's Picard
 *                        contractions on the tensor pipe (ADG_PRED_WARP4_TC:
 *                        TF32 operands split into high and low parts, three
 *                        mma products per tile, FP32 accumulation, which keeps
 *                        them FP32-accurate); 2D N <= 5 and 3D.
 *   (A BF16 mode is not provided: BF16 operands need three-way splits and six
 *   products per tile to reach FP32 accuracy, which the mixed scheme's final
 *   stage needs, and the contractions here are n x n with n <= 10.)
 * Accuracy bar of the mixed modes (tested on the benchmark workloads): the
 * relative L1 distance to the FP64 path per conserved variable after the same
 * steps is at most 1% of the FP64 scheme's own L1 error on that workload.
 */
#ifndef ADG_H
#define ADG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADG_OK 0
#define ADG_ERR_ARG (-1)          /* invalid argument or call order          */
#define ADG_ERR_OOM (-2)          /* device allocation failed                */
#define ADG_ERR_CUDA (-3)         /* a CUDA runtime call failed              */
#define ADG_ERR_TIMEOUT (-4)      /* a bounded device wait gave up           */
#define ADG_ERR_CAPACITY (-5)     /* more troubled cells than subcell slots  */
#define ADG_ERR_STATE (-6)        /* no admissible wave speed (dt undefined) */
#define ADG_WARN_SUBCELL_INADMISSIBLE 1 /* a subcell average left the
                                           admissible set after the limiter */

/* Boundary kinds, one per face (adg_create `bc[2k]` low, `bc[2k+1]` high side
 * of axis k).  The paper's tests use periodic, transmissive (outflow),
 * reflecting-wall and inflow (Dirichlet) boundaries (Sec. 5.1, 5.4, 5.5)
 * without printing their discrete form; this library's rules:
 *   PERIODIC      wrap (both faces of an axis, or neither);
 *   TRANSMISSIVE  ghost = copy of the interior (DG traces and subcells);
 *   REFLECTIVE    ghost = mirror image with the wall-normal momentum negated
 *                 (subcells mirror across the wall); the mirror images of the
 *                 boundary cells take part in the detector's neighbourhood V_i;
 *   INFLOW        ghost = the face's fixed conserved state
 *                 (adg_set_boundary_state); no cell beyond it joins V_i
 *                 (nor beyond a transmissive face);
 *   FRONT         the face is split at a point moving along one tangential
 *                 axis, x_f(t) = a + b t (adg_set_boundary_front): points with
 *                 x < x_f(t) follow one transmissive / reflective / inflow rule,
 *                 the others another -- the double-Mach boundaries of Sec. 5.4.
 *                 DG face nodes use their own position and time t^n + tau dt,
 *                 ghost subcells their centre at t^n; no cell beyond it joins
 *                 V_i. */
#define ADG_BC_PERIODIC 0
#define ADG_BC_TRANSMISSIVE 1
#define ADG_BC_REFLECTIVE 2
#define ADG_BC_INFLOW 3
#define ADG_BC_FRONT 4

#define ADG_PREC_FP64 0
#define ADG_PREC_MIXED_FP32 1
#define ADG_PREC_MIXED_TF32 2

/* adg_set_option keys */
#define ADG_OPT_DMP_EPS 1         /* eps of Eq. (relax), default 1e-3                 */
#define ADG_OPT_DMP_FLOOR 2       /* floor of delta, default 1e-4 (relative to
                                     max(1,|M|,|m|)); 0 gives the literal Eq. (relax) */
#define ADG_OPT_FORCE_LIMITER 3   /* 1: flag every cell every step (testing)          */
#define ADG_OPT_PICARD_ITERS 4    /* Picard sweeps of Eq. (pde.nc.dg2), default N+1   */
#define ADG_OPT_SLOT_CAPACITY 5   /* max troubled cells per step (before first load)  */
#define ADG_OPT_PROFILE 6         /* 1: time the phases of every step with CUDA events */
#define ADG_OPT_FP64_SWEEPS 7     /* mixed precision: final Picard sweeps run in FP64
                                     (the others in FP32); 0: none, the last FP32
                                     sweep's space-time correction is subtracted from
                                     the FP64 u.  Default 0 for N <= 5, 1 for N >= 6  */
#define ADG_OPT_END_TIME 8        /* end time of the run: steps are cut to reach it and
                                     the state idles afterwards (0: none, default)    */
#define ADG_OPT_CFL 9             /* the state's CFL number for batched CFL steps
                                     called with cfl <= 0 (includes 1/(d(2N+1)))      */
#define ADG_OPT_SCRATCH_BYTES 10  /* limiter scratch budget in bytes (before the first
                                     load; default an eighth of the free device memory
                                     at the first load, clamped to 2..32 GiB; used up to
                                     a quarter of the cells per limiter pass)         */
#define ADG_OPT_CASCADE 11        /* 1 (default): the extra MOOD layer of Sec. 6
                                     (Fig. algo2): a troubled cell whose WENO3 subcell
                                     result fails the admissibility test of
                                     Eq. (positivity) is recomputed from v^n by a
                                     first-order Rusanov step on its subgrid, and its
                                     WENO3 face neighbours take that flux on the shared
                                     face; 0: the two-level scheme (DG or WENO3), where
                                     such a cell raises ADG_WARN_SUBCELL_INADMISSIBLE */
#define ADG_OPT_FLUX 12           /* numerical flux of the DG faces and the WENO3
                                     sub-faces (Sec. 2.3): ADG_FLUX_RUSANOV (default)
                                     or ADG_FLUX_OSHER, the universal Osher-type flux
                                     of Dumbser and Toro (three-point Gauss-Legendre
                                     path integral), used for the vortex table of
                                     Sec. 5.2; the first-order layer keeps Rusanov */

#define ADG_OPT_HOST_PASSES 13    /* 0 (default): each adg_step / adg_step_cfl is one
                                     CUDA graph launch with no host wait; the limiter
                                     passes run in a conditional loop of the graph
                                     whose trip count the device takes from the
                                     step's troubled count.  1: the host waits once
                                     per step, after the DG phase, for that count and
                                     launches the passes itself.  Batched steps are
                                     always graphs.                                   */

#define ADG_OPT_SUBCELL_FP64_SWEEPS 14  /* mixed precision: how many of the three
                                     Picard sweeps of the degree-2 subcell predictor
                                     run in FP64 after the FP32 ones (0..3, default
                                     0: all FP32; the finite volume update stays
                                     FP64, the sub-face fluxes follow
                                     ADG_OPT_SUBCELL_FP32).  States batched
                                     together share one launch per value.          */

#define ADG_OPT_SUBCELL_FP32 15   /* mixed precision: the subcell scheme's WENO3
                                     reconstruction (weights in the ratio form
                                     ((sigma_min+eps)/(sigma_k+eps))^8, which cannot
                                     underflow to 0/0) and its sub-face Rusanov fluxes
                                     run in FP32 (default 1); the finite volume update,
                                     R and the flux correction stay FP64, and each
                                     sub-face flux is one value for both sides, so the
                                     scheme stays conservative.  0: FP64.  With the
                                     Osher-type flux the sub-faces stay FP64.        */

#define ADG_OPT_PROJECT_DELTA 16  /* mixed precision: the detector forms the subcell
                                     averages of the candidate, P(u*), as the P(u^n)
                                     kept from the previous step plus an FP32
                                     projection of the step's change u* - u^n, where
                                     P(u^n) is known (cells not limited, fixed or
                                     loaded since); FP64 P everywhere every 16th
                                     step.  1 (default) or 0; before the first load.
                                     Needs nv Ns^d doubles per cell.                 */

#define ADG_OPT_PREDICTOR 17       /* launch shape of the space-time predictor
                                     (Eq. pde.nc.dg2); every shape computes the same
                                     outputs.  -1 (default): after the state's first
                                     step the autotuner times the shapes whose
                                     outputs are bit for bit the default's (both
                                     block widths, or WARP1, WARP2 and WARP4 where
                                     the warp-per-cell shapes apply) and
                                     keeps the fastest (adg_autotune); -2: the same
                                     over every shape that applies, including those
                                     that round differently in FP32 (the tensor-pipe
                                     contractions, the block-per-cell mixed kernel);
                                     or one of:
                                       ADG_PRED_BLOCK       one block per cell
                                       ADG_PRED_BLOCK_ALT   one block per cell at the
                                                            other block width
                                       ADG_PRED_WARP1 / 2 / 4  mixed precision with
                                                            no FP64 sweep (2D N <= 5,
                                                            3D): one warp per cell for
                                                            the FP32 sweeps, 1, 2 or 4
                                                            cells per block sharing
                                                            the FP64 terms
                                       ADG_PRED_WARP4_TC    the same, with the sweeps'
                                                            contractions on the tensor
                                                            pipe (TF32 operands split
                                                            in high and low parts,
                                                            three products per tile:
                                                            FP32-accurate)
                                     A shape that does not apply is refused with
                                     ADG_ERR_ARG.                                     */
#define ADG_PRED_BLOCK 0
#define ADG_PRED_BLOCK_ALT 1
#define ADG_PRED_WARP2 2
#define ADG_PRED_WARP4 3
#define ADG_PRED_WARP4_TC 4
#define ADG_PRED_WARP1 5

#define ADG_OPT_SUBCELL_REGISTERS 18  /* mixed precision with the FP32 subcell
                                     predictor (the default subcell options): 1
                                     (default) the subcell's space-time nodes in
                                     registers -- each lane holds a spatial node
                                     and its three time nodes, three subcells per
                                     warp in 2D, one in 3D (27 spatial nodes);
                                     warp shuffles, no shared memory -- and, with
                                     the Rusanov flux, face traces handed to a
                                     warp-per-sub-face flux kernel; 0: one warp
                                     per subcell with the nodes in shared memory
                                     and the thread-per-sub-face flux kernel.
                                     Both give the same results bit for bit.    */

#define ADG_FLUX_RUSANOV 0
#define ADG_FLUX_OSHER 1

/* Cartesian grid (Sec. 2.1): cells n[k] of size dx[k] from corner x0[k]. */
typedef struct {
  int dim;        /* 2 or 3 */
  int n[3];       /* cells per axis; n[2] ignored for dim == 2 */
  double x0[3];   /* lower corner */
  double dx[3];   /* cell size per axis */
} adg_grid;

/* Test-problem initial data (Sec. 5.2, 5.6, 5.8), projected on the device by
 * adg_init_problem.  States are primitive: (rho, u, v, [w], p). */
#define ADG_IC_RADIAL 0   /* inner state for |x - center| <= radius, else outer */
#define ADG_IC_QUADRANT 1 /* 2D: state 1 x>xc,y>yc; 2 x<=xc,y>yc; 3 x<=xc,y<=yc; 4 x>xc,y<=yc */
#define ADG_IC_PLANAR 2   /* inner state where normal . x < offset (a planar front, e.g. the
                             oblique shock of Sec. 5.4), else outer */
typedef struct {
  int kind;
  double center[3];
  double radius;
  double inner[5];
  double outer[5];
  double quad[4][4];              /* (rho, u, v, p) of quadrants 1..4            */
  int vortex;                     /* 1: superpose the isentropic vortex          */
  double vortex_center[2];
  double vortex_strength;         /* beta of Sec. 5.2                            */
  const double* cell_rho_factor;  /* host [cells] density factor, or NULL        */
  double normal[3];               /* ADG_IC_PLANAR: front normal and offset      */
  double offset;
} adg_problem;

typedef struct adg_state adg_state;

/* Create a solver state for `grid`, polynomial degree N (1..9 in 2D, 1..3 in
 * 3D), ideal-gas gamma > 1, boundary kind per face bc[2*k] (low side of axis
 * k), bc[2*k+1] (high side): periodic faces must come in pairs.  No device
 * memory is touched until the first load.  Errors: ADG_ERR_ARG. */
int adg_create(const adg_grid* grid, int N, double gamma, const int* bc, int prec,
               adg_state** out);

/* Device allocator used for every buffer of this state (call before the first
 * load).  alloc(bytes, ctx) returns a device pointer or NULL; free(ptr, ctx).
 * Default: cudaMalloc / cudaFree. */
int adg_set_allocator(adg_state* st, void* (*alloc)(size_t, void*),
                      void (*free_fn)(void*, void*), void* ctx);

/* CUDA stream (a cudaStream_t passed as void*) for all work of this state. */
int adg_set_stream(adg_state* st, void* stream);

/* Numerical options, keys ADG_OPT_*.  Errors: ADG_ERR_ARG. */
int adg_set_option(adg_state* st, int key, double value);

/* Load the DG DOFs (host dofs[cells][nvar][n^dim]) as u^n.  With
 * exact_subcell_avgs (host sub[cells][nvar][Ns^dim]) the detector of Sec. 4.3
 * is applied to P(u^0) against bounds from the exact averages (Sec. 4.4, last
 * paragraph); flagged cells keep the exact averages as subcell data and their
 * DOFs become R(exact averages).  With NULL every cell starts unflagged.
 * Errors: ADG_ERR_ARG, ADG_ERR_OOM, ADG_ERR_CUDA, ADG_ERR_CAPACITY. */
int adg_load(adg_state* st, const double* dofs, const double* exact_subcell_avgs);

/* Project a test problem on the device: composite Gauss-Legendre rule of
 * Ns subintervals x (N+2) points per axis and cell for the L2 projection and
 * the exact subcell averages, then the same initial detection as adg_load. */
int adg_init_problem(adg_state* st, const adg_problem* problem);

/* Load / read a complete state (checkpoint-resume and testing): DOFs, flags
 * and the subcell data of flagged cells (host sub[cells][nvar][Ns^dim]; rows
 * of unflagged cells are ignored on load and written as NaN on read). */
int adg_load_full(adg_state* st, const double* dofs, const uint8_t* beta,
                  const double* subcells);
int adg_read_full(adg_state* st, double* dofs, uint8_t* beta, double* subcells);

/* One full time step of size dt > 0 (Sec. 4.4): predictor (Eq. pde.nc.dg2),
 * corrector (Eq. pde.nc.gw2), detection (Eqs. positivity, dmp, relax),
 * subcell ADER-WENO3 recomputation of troubled cells (Eq. aderweno with the
 * data of Eq. ader.icbc), reconstruction R, the flux correction of their
 * unlimited face neighbours, and with ADG_OPT_CASCADE the first-order layer.
 * Asynchronous (one CUDA graph launch) unless ADG_OPT_HOST_PASSES is 1 (then
 * one wait for the step's troubled count after the DG phase).  Errors: ADG_ERR_ARG (dt <= 0,
 * nothing loaded), ADG_ERR_CUDA.  Device-side conditions (capacity overflow,
 * inadmissible subcells) surface on the next synchronizing call. */
int adg_step(adg_state* st, double dt);

/* Same step with dt = min(cfl * min_k dx_k / lambda_max, dt_max) computed on
 * the device from the current state (Eq. cfl); nothing returns to the host. */
int adg_step_cfl(adg_state* st, double cfl, double dt_max);

/* Simulated time t of the state and the number of steps it has taken since
 * the last load (either may be NULL); synchronizes. */
int adg_time(adg_state* st, double* t, int64_t* steps);

/* Batched stepping of many independent states (no counterpart in the
 * paper, which steps one grid): states of the same
 * dimension, degree and precision share every kernel launch, each launch
 * covering all their cells, faces or troubled cells.  All states must be
 * loaded; their streams are set to the batch's stream (`stream`, or a stream
 * the batch creates when NULL).  A state may belong to one live batch at a
 * time and must not be stepped on its own while it does.
 *   adg_batch_step with dts (host [count]) takes those steps; with dts = NULL
 *   every state takes the CFL step of Eq. (cfl) with the number `cfl`, or
 *   with its own ADG_OPT_CFL when cfl <= 0, cut at its end time
 *   (ADG_OPT_END_TIME); states past their end time idle.  CFL steps run as
 *   one CUDA graph, captured on the first and replayed while cfl is
 *   unchanged; each group's limiter passes loop on the device.
 * Asynchronous; errors of device-side conditions surface in adg_status of
 * the states. */
typedef struct adg_batch adg_batch;
int adg_batch_create(adg_state* const* states, int count, void* stream, adg_batch** out);
int adg_batch_step(adg_batch* b, const double* dts, double cfl);
void adg_batch_destroy(adg_batch* b);

/* One step of `count` states with host steps dts[count] in shared launches
 * (a batch created and destroyed around the call). */
int adg_step_batch(adg_state* const* states, const double* dts, int count);

/* Eq. (cfl): dt = cfl * min_k dx_k / lambda_max with lambda_max over the
 * subcell averages v^n of every cell; cfl includes 1/(d (2N+1)).
 * Synchronizes.  Errors: ADG_ERR_STATE when no admissible wave speed exists. */
int adg_max_dt(adg_state* st, double cfl, double* dt_out);

/* Flags beta^{n+1} of the last step (or beta^0 after a load), host uint8[cells]. */
int adg_flags(adg_state* st, uint8_t* beta);

/* Current DOFs, host dofs[cells][nvar][n^dim]. */
int adg_read(adg_state* st, double* dofs);

/* Number of troubled cells of the last step. */
int adg_troubled_count(adg_state* st, int64_t* out);

/* Troubled-cell counts (beta^{n+1} = 1, Sec. 4.3) of the last steps since the
 * last load, oldest first: out[i] (host int64[max]) for the min(max, steps,
 * 4096) most recent steps; *written receives their number.  The device keeps
 * the counts as the steps run, so reading them costs the steps nothing.
 * Synchronizes.  Errors: ADG_ERR_ARG (nothing loaded, bad pointers). */
int adg_troubled_history(adg_state* st, int64_t* out, int max, int* written);

/* The fixed conserved state q[nvar] of inflow face `face` (2k low, 2k+1 high
 * side of axis k), host memory, copied.  Needed for every ADG_BC_INFLOW face
 * before the first load.  Errors: ADG_ERR_ARG (face out of range or not an
 * inflow face, rho <= 0 or p <= 0). */
int adg_set_boundary_state(adg_state* st, int face, const double* q);

/* The moving split of front face `face`: points whose coordinate along
 * tangential axis `axis` is below a + b t follow `kind_before` (with state
 * q_before[nvar] if it is ADG_BC_INFLOW, else NULL), the others `kind_after`.
 * Needed for every ADG_BC_FRONT face before the first load.  Errors:
 * ADG_ERR_ARG (not a front face, axis not tangential, a part not transmissive /
 * reflective / inflow, an inflow part without an admissible state). */
int adg_set_boundary_front(adg_state* st, int face, int axis, double a, double b, int kind_before,
                           const double* q_before, int kind_after, const double* q_after);

/* Set the simulated time (time-dependent boundaries, restarts from adg_load_full,
 * which starts the clock at 0).  Needs a loaded state. */
int adg_set_time(adg_state* st, double t);

/* Cells recomputed by the first-order layer (ADG_OPT_CASCADE): in the last
 * step, and since the last load.  Either pointer may be null. */
int adg_fallback_count(adg_state* st, int64_t* last_step, int64_t* total);

/* Synchronize and report pending device-side conditions of earlier steps
 * (ADG_ERR_CAPACITY, ADG_WARN_SUBCELL_INADMISSIBLE); clears them. */
int adg_status(adg_state* st);

/* Counts of the per-state scalars: cells, nvar, nodes per cell (n^dim),
 * subcells per cell (Ns^dim). */
int adg_sizes(const adg_state* st, int64_t* cells, int* nvar, int* nodes, int* subcells);

/* Autotuner of the predictor's launch shape (no counterpart in the paper):
 * times the predictor in every shape among which ADG_OPT_PREDICTOR lets it
 * choose (-1, -2; with a fixed shape every shape that applies, for the
 * report), `reps` launches each (after one warm-up launch) with CUDA events on
 * the state's stream, on the current level with the dt of the last step, and
 * keeps the fastest for the following steps unless ADG_OPT_PREDICTOR fixes a
 * shape.  The state's data are unchanged (the predictor's outputs are
 * rewritten by the next step).  ms[k] (host, k < cap) receives the
 * milliseconds per launch of shape k, NaN for shapes not timed.
 * Runs automatically after the first step of a state whose ADG_OPT_PREDICTOR
 * is -1 or -2.  Synchronizes.  Errors: ADG_ERR_ARG (nothing loaded, no step taken
 * yet, reps < 1), ADG_ERR_CUDA. */
int adg_autotune(adg_state* st, int reps, double* ms, int cap);

/* Launch layout after the first load: out[0] = subcell slot capacity,
 * out[1] = troubled cells per limiter chunk, out[2] = kernels launched by one
 * adg_step at most (every limiter pass the capacity allows, in the state's
 * launch mode), out[3] = device bytes held by the state, and with cap >= 5,
 * out[4] = kernels issued by this state's steps so far, the passes of the
 * device-sized loops counted on the device (batched steps count on the first
 * state of each group of one dimension, degree and precision; synchronizes
 * the state's stream); with cap >= 7, out[5] = Picard
 * sweeps of the predictor, out[6] = how many of them run in FP64; with
 * cap >= 8, out[7] = the predictor's launch shape in effect (ADG_PRED_*).
 * Needs cap >= 4. */
int adg_info(const adg_state* st, int64_t* out, int cap);

/* Phase timing (ADG_OPT_PROFILE = 1): accumulated milliseconds of the steps
 * since the last call, measured with CUDA events on the state's stream, in
 * the order predictor, face fluxes, corrector + detector, subcell limiter,
 * neighbour flux correction; ms[5] = number of steps timed.  Synchronizes and
 * resets the sums.  Needs cap >= 6. */
int adg_phase_times(adg_state* st, double* ms, int cap);

const char* adg_last_error(const adg_state* st);

/* Subcell ADER-WENO3 update of caller-owned patches that allocates nothing.
 * The paper has no counterpart: it is a variant, for one batch of patches, of
 * the limiter that adg_step runs on its troubled cells.
 *
 * Who needs it: callers that cannot call cudaMalloc -- code running inside a
 * host application that owns all device memory, or a loop that must never
 * reach an allocator -- but can hand over device buffers they already own.
 *
 * Inputs (device pointers; the caller owns them):
 *   patches [count][dim+2][L^dim], L = 2N+7: the subcell averages of the
 *           target cell (local subcells 0..2N) and of three ghost layers
 *           around it (-3..-1 and 2N+1..2N+3 per axis), x fastest;
 *   h[dim]  subcell widths (host array), dt > 0, gamma > 1, N 1..9 (2D) or
 *           1..3 (3D).
 * Outputs (device pointers): vnew [count][dim+2][(2N+1)^dim] the updated
 * subcell averages; faces [count][dim][2][dim+2][(2N+1)^(dim-1)] the sub-face
 * fluxes on the low / high faces of each cell, or NULL.
 * Work is enqueued on `stream` (a cudaStream_t, NULL for the default stream);
 * the call uploads the operator table of degree N and synchronizes that stream
 * once before launching.
 *
 * Scratch: one static device array of 32 MiB, held by every GPU that loads
 * the library until the process exits; its address is looked up on the first
 * call made on each device (make that first call before any stream capture).
 * count is limited by that size (e.g. about 146 patches for dim 2, N 5); a
 * larger count returns ADG_ERR_CAPACITY with the limit in `err`.  Every call
 * shares the array and leaves its contents behind: calls that overlap on the
 * GPU (other streams, other threads) race and must be serialized by the caller.
 * No cudaMalloc, cudaFree or allocating library routine is called.
 * err (may be NULL) receives a message of at most errlen bytes on failure.
 * Returns ADG_OK, ADG_ERR_ARG, ADG_ERR_CAPACITY or ADG_ERR_CUDA. */
int adg_subcell_update_noalloc(int dim, int N, double gamma, const double* h, double dt,
                               const double* patches, int count, double* vnew, double* faces,
                               void* stream, char* err, size_t errlen);

/* Halo exchange of a domain decomposition (the paper runs its largest tests
 * on many processes, each owning a block of the grid, Sec. 5.8; the flux
 * correction of Sec. 4.4 couples cells across a block edge).  A subdomain is a
 * state whose grid holds its own cells plus halo layers copied from the
 * states that own them before every step; a step needs the level-n data of
 * the cells within two cells of the owned ones (face traces and detector
 * bounds of the face neighbours, and the troubled status and sub-face fluxes
 * of neighbours that feed the flux correction), so two halo layers make the
 * owned cells' new level exactly the single-domain one.
 *
 * A box is the cells with lo[k] <= index_k < hi[k] along every axis k < dim
 * (cell coordinates of the state's own grid).  The packed form of `count`
 * cells, in box order (x fastest), is the byte buffer
 *   dofs [count][nvar][n^dim] double | sub [count][nvar][Ns^dim] double |
 *   cmm [count][nvar][2] double | beta [count] uint8
 * (the DOFs, the stored subcell data of flagged cells -- other rows are
 * unspecified -- the per-cell min / max of the subcell data, the flags).
 *
 * adg_halo_bytes: bytes of the packed form of `count` cells of this state's
 *   degree and dimension.
 * adg_pack_cells: the current level of the box into `buf` (device memory of
 *   at least adg_halo_bytes, 8-byte aligned, owned by the caller).
 * adg_unpack_cells: the packed cells of `buf` become the current level of the
 *   box (a box of the same shape in another state of the same dimension and
 *   degree); the troubled list, subcell slots and kept averages are rebuilt
 *   and the wave speeds are recomputed at the next CFL query.
 * Both are enqueued on the state's stream (calls on states with different
 * streams are ordered by the caller).  Errors: ADG_ERR_ARG (nothing loaded,
 * box outside the grid or empty, unaligned buffer), ADG_ERR_CUDA; more
 * flagged cells than subcell slots surfaces in adg_status as ADG_ERR_CAPACITY. */
int adg_halo_bytes(const adg_state* st, int64_t count, int64_t* bytes);
int adg_pack_cells(adg_state* st, const int* lo, const int* hi, void* buf);
int adg_unpack_cells(adg_state* st, const int* lo, const int* hi, const void* buf);

/* Arithmetic-pipe rates of the current device (no counterpart in the paper;
 * the step's kernels are bound by these pipes, and they are the denominators
 * the roofline figures are checked against): out[0] FP64 FMA, out[1] FP32 FMA,
 * out[2] FP64 -> FP32 conversion, out[3] FP64 comparison, and with cap >= 6
 * out[4] the FP64 reciprocal by division (1.0 / x) and out[5] the same by the
 * library's Newton-Raphson form (an FP32 seed and two FP64 steps, used on the
 * mixed-precision path), each in thread operations per second (an FMA is two
 * flop), from 3 timed runs of a dependency-chain kernel over 8 blocks of 256
 * threads per multiprocessor (best of the last two).  With cap >= 8 it also
 * compares the Newton form with 1.0 / x on 2^22 values (mantissas from a
 * hash, magnitudes 2^-60 .. 2^60, both signs): out[6] the largest difference
 * in units of the last place, out[7] the fraction of values that differ.
 * Allocates and frees scratch buffers; synchronizes the device.  Needs
 * cap >= 4.  Errors: ADG_ERR_ARG, ADG_ERR_OOM, ADG_ERR_CUDA. */
int adg_pipe_rates(double* out, int cap);

/* Free every device buffer of the state and the state itself. */
void adg_destroy(adg_state* st);

#ifdef __cplusplus
}
#endif
#endif /* ADG_H */
