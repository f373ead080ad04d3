/*
 * moses.h -- C-ABI of the GB300 (sm_103a) implementation of one explicit time
 * step of the depth-integrated two-phase (solid grains + interstitial fluid)
 * shallow-flow model of MoSES_2PDF (arXiv:2104.06784) over a DEM.
 *
 * What the library computes, per step (Sect. 2.2 and App. A):
 *   dt   = CFL min(dx, dy) / a_max,  a_max = largest per-phase wave speed over
 *          all cells (the CFL reduction of Sect. 3.1.2, Stage 2)
 *   U*   = U^n + dt L(U^n),   U** = U* + dt L(U*),   U^{n+1} = (U^n + U**)/2
 *          (two-step modified Euler, Sect. 2.2)
 *   L    = central (Kurganov-Tadmor) fluxes of Eqs. FluxEqSxi_Topo ..
 *          FluxEqFeta_Topo with minmod reconstruction (Sect. 2.2) plus the
 *          sources of Eqs. Src_nd_Topo, Src_f_Topo, Src_v_Topo, SrcF_nd_Topo,
 *          SrcF_f_Topo, SrcF_v_Topo, SrcF_vis_Topo; Coulomb friction with a
 *          stopping condition; positivity of both depths.
 * The conserved state per cell is U = (J h^s, J h^s v_X^s, J h^s v_Y^s,
 * J h^f, J h^f v_X^f, J h^f v_Y^f) (App. A, Eqs. MassEq_TopoS0/F0,
 * MomentumEqS_Topo/F_Topo), h the thickness normal to the bed, v_X, v_Y the
 * horizontal projections of the phase velocities, J = J_b = det Omega_b.
 *
 * Conventions for every call:
 *  - Grids are row-major [j * nx + i]; j = 0 is the southern row (Y grows
 *    northwards), i = 0 the western column.  Cells are dx by dy metres.
 *  - Host pointers unless a name ends in _device.  The library copies every
 *    input; it never keeps a caller's pointer after a call returns.
 *  - Device work runs on the CUDA stream given to moses_create (NULL = the
 *    legacy default stream).  Calls that return values to the host
 *    synchronise that stream before returning.
 *  - Every int-returning call returns MOSES_OK (0) or a negative MOSES_E*
 *    code; moses_last_error() gives the message.  No call throws.
 *  - A moses_sim is not thread-safe; distinct sims are independent.
 */
#ifndef MOSES_H
#define MOSES_H

#ifdef __cplusplus
extern "C" {
#endif

#define MOSES_OK 0
#define MOSES_EINVAL (-1)     /* bad argument (size, pointer, parameter)       */
#define MOSES_ENOMEM (-2)     /* device or host allocation failed               */
#define MOSES_ECUDA (-3)      /* a CUDA call failed (message has the CUDA error) */
#define MOSES_ENONFINITE (-4) /* the state or the time step became non-finite   */
#define MOSES_ETIMEOUT (-5)   /* a bounded device-side wait gave up             */
#define MOSES_ESTATE (-6)     /* call out of order (e.g. step before a state)   */

#define MOSES_BC_CLOSED 0       /* wall: mirror, normal momentum negated      */
#define MOSES_BC_TRANSMISSIVE 1 /* the paper's "no reflection" (Sect. 3.1.2):
                                   zero-gradient copy into the ghost cells      */

#define MOSES_SIDE_W 0
#define MOSES_SIDE_E 1
#define MOSES_SIDE_S 2
#define MOSES_SIDE_N 3

#define MOSES_FP64 0 /* state, geometry and flux arithmetic in FP64            */
#define MOSES_FP32 1 /* state, geometry and fluxes in FP32; budgets and the
                        friction stopping test in FP64                          */

#define MOSES_BUDGET_LEN 13

/* Model and scheme parameters, SI units.  The paper's equations are
 * dimensionless (App. A); g = 1 recovers them.  Every pressure carries g c,
 * c = n_Z (App. A, below Eq. FluxEqFeta_Topo). */
typedef struct {
    double g;            /* gravity [m s^-2]                                      */
    double eps;          /* aspect ratio epsilon in the pressure terms (1 in SI)  */
    double eps_chi;      /* epsilon^chi in front of kappa in p_b (1 in SI)        */
    double rho_s, rho_f; /* densities; alpha_rho = rho_f / rho_s                 */
    double delta_b_deg;  /* basal friction angle delta_b (Sect. 3.1.2 (a))        */
    double phi_int_deg;  /* internal friction angle phi_int (k_mode 1 only)       */
    int k_mode;          /* 0: earth-pressure coefficient 1, the solid pressure of
                            App. A (below Eq. FluxEqFeta_Topo); 1: Savage-Hutter
                            coefficients K_act/pass = 2 sec^2(phi_int) (1 -/+
                            sqrt(1 - cos^2(phi_int) sec^2(delta_b))) - 1 on the
                            solid pressure of each direction and the solid
                            celerity: a cell is passive where it and its two
                            neighbours along the axis carry solid and the solid
                            velocity along the axis drops by more than
                            1e-6 (|v+| + |v-|) + 1e-6 m/s, active otherwise;
                            each side of a face takes its cell's K; the CFL
                            celerity takes K_pass.  Needs delta_b <= phi_int
                            < 90 deg, the central flux, minmod and nu_f = 0;
                            not accepted by moses_batch_create or
                            moses_step_static                                    */
    double c_d;          /* interphase drag c_D [s^-1] (Eqs. Src_v_Topo, SrcF_v)  */
    double nu_f;         /* fluid viscosity eps/N_R [m^2 s^-1] (Eq. SrcF_vis_Topo);
                            > 0 runs the 32 x 8 viscous form of the stage; not
                            accepted by moses_batch_create, moses_adjoint_misfit,
                            moses_step_static                                    */
    double k_f;          /* fluid basal friction vartheta_b/(eps N_R) [s^-1]      */
    double cfl;          /* Courant number (the paper uses 0.1, Sect. 2.2)        */
    double dt_max;       /* time step cap, and the step of a dry domain [s]       */
    double h_dry;        /* depth below which a phase has no velocity [m]         */
    int bc[4];           /* W, E, S, N: MOSES_BC_CLOSED or MOSES_BC_TRANSMISSIVE  */
    int fluid_pg_mode;   /* 0: fluid pressure-gradient source with phi^s (the
                            reaction of the solid buoyancy); 1: phi^f as printed
                            in Eq. SrcF_f_Topo                                    */
    int precision;       /* MOSES_FP64 or MOSES_FP32                              */
    int scheme;          /* MOSES_SCHEME_CENTRAL: the central flux of Sect. 2.2
                            (the paper's); MOSES_SCHEME_CENTRAL_UPWIND: the
                            central-upwind flux with one-sided local speeds of
                            the second-order scheme Sect. 2.2 cites (32 x 8
                            tiles; not accepted by moses_batch_create,
                            moses_adjoint_misfit, moses_step_static)          */
    int recon;           /* MOSES_RECON_MINMOD: minmod TVD slopes (Sect. 2.2, the
                            paper's); MOSES_RECON_WENO3: third-order WENO face
                            values, the option Sect. 2.2 names (32 x 8 tiles)   */
    int rk;              /* 0 or 2: the two-step modified Euler (Sect. 2.2, the
                            paper's); 3: three-stage SSP Runge-Kutta, the
                            multi-step option Sect. 2.2 names.  recon and rk
                            other than the paper's are not accepted by
                            moses_batch_create, moses_adjoint_misfit,
                            moses_stage_adjoint, moses_step_static             */
} moses_params;

#define MOSES_SCHEME_CENTRAL 0
#define MOSES_SCHEME_CENTRAL_UPWIND 1
#define MOSES_RECON_MINMOD 0
#define MOSES_RECON_WENO3 1

typedef struct moses_sim moses_sim; /* opaque; owns all its device memory */

/* Create a simulation over a DEM (Sect. 2.1; Sect. 3.1.2 Stage 0-1).
 * dem: nx*ny bed elevations [m] at cell centres (host).  nx, ny >= 1;
 * dx, dy > 0.  Runs the one-time geometry pass (basal basis, J_b, Omega_b^-1,
 * slope and curvature terms) on the GPU.  stream: a cudaStream_t or NULL.
 * On success *out owns ~ (6 + 6 + 20) nx ny words of device memory.
 * The state starts dry at t = 0.  Errors: EINVAL, ENOMEM, ECUDA. */
int moses_create(const double *dem, int nx, int ny, double dx, double dy, const moses_params *p,
                 void *stream, moses_sim **out);

/* Mode-I release (Sect. 3.1.2 Stage 0): finite masses placed in the domain.
 * h: normal flow thickness [m]; phi_s: solid volume fraction (NULL = 0.5);
 * vx_s .. vy_f: phase velocities, horizontal projections [m s^-1] (NULL = 0).
 * All nx*ny, host.  Replaces the state; keeps t and the inflow segments.
 * Errors: EINVAL (NULL h, h < 0, phi_s outside [0, 1], non-finite), ECUDA. */
int moses_set_release(moses_sim *s, const double *h, const double *phi_s, const double *vx_s,
                      const double *vy_s, const double *vx_f, const double *vy_f);

/* Mode-II inflow (Sect. 3.1.2 Stage 0): a hydrograph on boundary cells
 * [i0, i1) of `side` (indices along that side).  t, Q, phi_s: npts samples
 * (host) of time [s], total discharge [m^3 s^-1] and solid fraction; linear in
 * between, zero outside [t[0], t[npts-1]].  The ghost cells of the segment
 * hold the mixture at critical depth for the unit discharge Q / width,
 * moving inward.  Up to 8 segments, npts <= 64, t non-decreasing.
 * Errors: EINVAL, ECUDA. */
int moses_set_inflow(moses_sim *s, int side, int i0, int i1, int npts, const double *t,
                     const double *Q, const double *phi_s);

/* Advance nsteps CFL-limited steps (Sect. 2.2; Stage 2 of Sect. 3.1.2).
 * Tiles with no mass within the stencil's reach are not computed: their
 * stage result, the zero state, is written directly, and not written again
 * while the buffer holds it from an earlier step of these calls (wet/dry
 * masking with per-tile known-zero flags; the result is the same).  Any other
 * call that may write the state, or moses_set_tile, makes the next step write
 * every dry tile once.  t_out (may be NULL) receives the time after the last step.  Synchronises
 * the stream once at the end.  Errors: ESTATE, ENONFINITE (a kernel saw a
 * non-finite value; the state is left as computed and every later step
 * reports it again until a new state is set), ECUDA. */
int moses_step(moses_sim *s, int nsteps, double *t_out);

/* moses_step with CUDA events recorded on the stream around every stage
 * launch: stage_ms[0] / stage_ms[1] receive the summed device time of the
 * stage-1 / stage-2 launches [ms] (the two launches of each step).  For
 * per-kernel throughput measurements; otherwise identical to moses_step. */
int moses_step_timed(moses_sim *s, int nsteps, double *t_out, double *stage_ms);

/* Tile shape of the stage kernel (not in the paper, which gives none):
 * MOSES_TILE_32x8 (the default), MOSES_TILE_32x4 or MOSES_TILE_32x16 cells
 * per CTA, or MOSES_TILE_32x4_2T: 32 x 4 cells with two threads per cell on
 * the listed wet tiles of the plain form (one thread takes the cell's x-face,
 * the other its y-face; the cell update runs on the first of the two), for
 * steps with few wet tiles per SM, whose time is the latency of one tile.
 * Every tile computes the same values (the state after a step is
 * bit-identical); only the speed differs.  Errors: EINVAL for another value. */
#define MOSES_TILE_32x8 0
#define MOSES_TILE_32x4 1
#define MOSES_TILE_32x16 2
#define MOSES_TILE_32x4_2T 3
#define MOSES_NTILES 4
int moses_set_tile(moses_sim *s, int tile);

/* Autotuner: times `reps` (>= 1; 0 = 5) first stages of a step from the
 * current state, launched as moses_step launches them in a run (classified
 * from the per-tile mass bits, dry tiles that hold the zero state left
 * unwritten), with each tile shape (CUDA events on the simulation's stream,
 * after one untimed stage each that classifies from the data and sets those
 * records up; two rounds over the shapes; the state, time and budgets are
 * not changed), selects the shape with the fastest launch and returns it in
 * *tile_out (may be NULL).  ms_out (may be NULL) receives the fastest launch
 * of each tile [ms], indexed by MOSES_TILE_*.  The choice
 * is cached per process by (device, SM count, precision, nx, ny): a later call
 * with ms_out == NULL on a simulation with the same key takes the cached tile
 * without timing.  Errors: EINVAL, ESTATE (no state), ECUDA. */
int moses_autotune(moses_sim *s, int reps, int *tile_out, double *ms_out);

/* Advance with a prescribed time step dt > 0 (same stages, no CFL search).
 * Errors: EINVAL, ESTATE, ENONFINITE, ECUDA. */
int moses_step_dt(moses_sim *s, int nsteps, double dt, double *t_out);

/* Advance until t >= t_end (the last step is shortened to land on t_end) or
 * max_steps steps.  *nsteps_out (may be NULL) gets the steps taken. */
int moses_run_until(moses_sim *s, double t_end, int max_steps, int *nsteps_out);

/* The time step the next moses_step would take, and the current time. */
int moses_next_dt(moses_sim *s, double *dt, double *t);

/* Output fields of Sect. 3.1.2 Stage 3: total normal thickness h, solid
 * fraction phi_s, phase velocities (horizontal projections).  Each pointer
 * may be NULL; non-NULL ones receive nx*ny doubles (host). */
int moses_get_state(moses_sim *s, double *h, double *phi_s, double *vx_s, double *vy_s,
                    double *vx_f, double *vy_f);

/* Conserved state U, 6 planes of nx*ny doubles, plane k holding U_{k+1}
 * (host).  get: copy out (FP32 state widened).  set: replace (rounded to
 * FP32 in that form); does not change t.  Errors: EINVAL (negative depth,
 * non-finite), ECUDA. */
int moses_get_conserved(moses_sim *s, double *U);
int moses_set_conserved(moses_sim *s, const double *U);

/* The same on device memory owned by the caller (6*nx*ny doubles, same plane
 * order), for zero-copy use from frameworks that hold tensors in HBM. */
int moses_get_conserved_device(moses_sim *s, double *U_device);
int moses_set_conserved_device(moses_sim *s, const double *U_device);

/* One stage U + dt L(U) from the current state at time t (friction, clamp
 * and dry-momentum rule included), written to U_out (6*nx*ny doubles, host).
 * The state is unchanged.  For stage-level parity checks. */
int moses_stage(moses_sim *s, double t, double dt, double *U_out);

/* Largest cell-centre wave speed of the current state (the a_max of the CFL
 * step), reduced exactly on the GPU. */
int moses_max_speed(moses_sim *s, double *amax);

/* ---- One strip of a row-decomposed domain ------------------------------
 *
 * The paper runs one simulation per GPU (Sect. 3.2).  A domain too large for
 * one GPU is split into strips of whole rows, one simulation per strip, each
 * created on its own rows plus `o` rows of overlap on every side that meets
 * another strip (its window), with that strip's slice of the DEM and
 * release.  o = 2 x (stages per step) + 1: a stage reads state and bed
 * geometry two cells away, and the geometry of a window's last row comes
 * from a bed extrapolated past the window.  Every step each strip steps its
 * whole window,
 * then receives the o overlap rows from the strips that own them
 * (moses_get_rows_device there, moses_set_rows_device here), and the
 * strips agree on the CFL maximum (the largest moses_max_speed of all
 * strips, written back with moses_set_max_speed).  The owned rows then
 * evolve bit for bit as in the undecomposed run: their stencils see only
 * exact values, and the maximum is the same exact maximum.  The host side
 * of this (row split, exchange over torch.distributed, maximum) is
 * paper_2104_06784_gb300/decomp.py. */

/* Rows [j0, j1) of this simulation are its own: only their cells enter the
 * CFL maximum, the clamp counts and the volume sums of moses_get_budget,
 * only their boundary faces the boundary inflow.  Default: every row.
 * A strip with owned rows set joins no batch and has no adjoint (EINVAL). */
int moses_set_owned_rows(moses_sim *s, int j0, int j1);

/* Planes per row of the row buffers: 6 (FP64 state) or 8 (FP32 state and
 * its two mass remainder planes).  0 for NULL. */
int moses_row_planes(const moses_sim *s);

/* Rows [j0, j0 + nrows) of the state to / from a device buffer owned by the
 * caller, moses_row_planes(s) * nrows * nx doubles, [plane][row][i] (exact
 * in both directions for values of the simulation's precision).  get is
 * asynchronous on the simulation's stream.  set takes the values as given
 * (no validation: a non-finite value raises MOSES_ENONFINITE at the next
 * step), refills the ghost cells those rows own at the current time, and
 * updates the stepping launches' per-tile records (known-zero flags, mass
 * bits) of the tiles it touches; it is asynchronous too.  EINVAL: rows
 * outside the grid; ESTATE: no state set yet. */
int moses_get_rows_device(moses_sim *s, int j0, int nrows, double *rows_device);
int moses_set_rows_device(moses_sim *s, int j0, int nrows, const double *rows_device);

/* Replace the CFL maximum the next step takes its time step from (finite,
 * >= 0; the maximum over all strips).  Synchronous. */
int moses_set_max_speed(moses_sim *s, double amax);

/* FP64 budgets, reduced on the GPU: out[0..1] solid / fluid volume
 * sum(U1), sum(U4) dx dy [m^3]; out[2..5] momenta sum(U2, U3, U5, U6) dx dy;
 * out[6..7] time-integrated boundary volume inflow per phase (the computed
 * face fluxes with the stage weights of the step); out[8..9] volume added by the positivity clamp
 * per phase; out[10] clamp events; out[11] t; out[12] steps taken. */
int moses_get_budget(moses_sim *s, double out[MOSES_BUDGET_LEN]);

/* Message of the last error on s (or of the last failed moses_create when
 * s is NULL).  Valid until the next call on s. */
const char *moses_last_error(const moses_sim *s);

/* Release all device memory of s.  NULL is ignored. */
void moses_destroy(moses_sim *s);

/* ---- Ensembles --------------------------------------------------------------
 * Many independent simulations advanced together, for the "abundant plausible
 * scenarios" and parameter back-calculation use of Sect. 5: each member keeps
 * its own DEM, grid size, parameters, time and CFL time step.  A call of
 * moses_batch_step is one cooperative launch of every CTA that fits on the
 * GPU at once, which runs all its steps for every member: per Heun stage the
 * wet tiles of every member are classified (from the data on the call's first
 * stage, then from the per-tile mass bits the stage keeps) and the stage runs
 * on them, with the CTAs meeting on a grid barrier between the phases.  Every
 * wait of that barrier is bounded (0.5 s): one that runs out ends the launch
 * and the call returns MOSES_ETIMEOUT.  The tile shape (32 x 4, 32 x 8 or
 * 32 x 16) is the fastest of one first stage per shape on the members' states,
 * timed by moses_batch_create (the members' control blocks are restored; their
 * U* scratch buffers are overwritten).  Members are ordinary moses_sim objects
 * created on the same stream with the same precision form; their states and
 * budgets are read with the per-simulation calls.  The batch does not own
 * them: destroy the batch before its members.  Errors (moses_batch_last_error):
 * EINVAL, ESTATE, ENONFINITE, ETIMEOUT, ECUDA. */
typedef struct moses_batch moses_batch;
int moses_batch_create(int n, moses_sim *const *sims, moses_batch **out);
/* every member advances nsteps CFL-limited steps (one launch); synchronises at
 * the end */
int moses_batch_step(moses_batch *b, int nsteps);
/* the same, with CUDA events on the batch's stream around the launch: *ms
 * receives its device time [ms] */
int moses_batch_step_timed(moses_batch *b, int nsteps, double *ms);
/* number of tiles of all members in the chosen tile shape */
int moses_batch_tiles(const moses_batch *b);
/* rows of the chosen tile shape (4, 8 or 16; 0 for NULL); ms_out (may be
 * NULL) receives the timed first stage of the 32 x 4, 32 x 8 and 32 x 16
 * shapes [ms] */
int moses_batch_tile_rows(const moses_batch *b, double ms_out[3]);
/* replace the chosen tile shape by 32 x rows (4, 8 or 16); EINVAL else */
int moses_batch_set_tile_rows(moses_batch *b, int rows);
/* testing only: on != 0 makes the launch's grid barrier wait for one CTA
 * more than the grid holds, so that every wait runs out (no fault); the call
 * then returns MOSES_ETIMEOUT.  0 restores normal steps. */
int moses_batch_debug_timeout(moses_batch *b, int on);
const char *moses_batch_last_error(const moses_batch *b);
void moses_batch_destroy(moses_batch *b);

/* ---- Adjoint: gradients of a deposit misfit --------------------------------
 * For the parameter back-calculation of Sect. 5: runs nsteps CFL steps from
 * the current state and returns L = sum_cells (h^s - h^s_target)^2 dx dy at
 * the end (h^s = J h^s / J, the solid's normal thickness) with its gradient.
 * The adjoint holds the recorded time steps fixed and uses the derivative of
 * the branch the forward took at every kink (minmod, max of the local speeds,
 * Coulomb stopping -> 0, positivity clamp and dry rule -> 0).  The state is
 * checkpointed every ckpt_every steps (<= 0: ceil(sqrt(nsteps))) and each
 * segment is recomputed before it is swept backwards.
 *   hs_target    nx*ny target solid thickness [m] (host)
 *   loss         L [m^4]; may be NULL
 *   g_params     [0] dL/d delta_b per degree (through tan(delta_b) and, with
 *                k_mode 1, through K_act and K_pass), [1] dL/d phi_int per
 *                degree (k_mode 1; 0 for k_mode 0, whose model has no
 *                internal friction), [2] dL/d c_D
 *   g_state0     6*nx*ny dL/dU at the start (host) or NULL
 *   g_release_h  nx*ny dL/dh of the release thickness (host) or NULL, with
 *                release_phi the release's solid fraction (NULL: U1/(U1+U4))
 *   timing_ms    [0] forward run, [1] recompute + backward sweep (CUDA
 *                events), or NULL
 * The regime of the earth-pressure coefficient (k_mode 1) is a kink like the
 * others: the derivative holds it fixed.  Afterwards the state and the time
 * are those at the end of the forward run.  Not available with nu_f > 0; with
 * k_mode 1 it needs delta_b < phi_int.  Errors: EINVAL, ESTATE, ENOMEM,
 * ECUDA. */
int moses_adjoint_misfit(moses_sim *s, int nsteps, int ckpt_every, const double *hs_target, double *loss,
                         double g_params[3], double *g_state0, double *g_release_h, const double *release_phi,
                         double timing_ms[2]);

/* Adjoint of one stage at the current state (the reverse of moses_stage with
 * the time step dt held fixed): lam_in = (dS/dU)^T lam_out, both 6*nx*nx
 * doubles on the host in the plane order of moses_get_conserved;
 * g_param[0..2] (may be NULL) receive lam_out . dS/d tan(delta_b) (with
 * k_mode 1 including its effect on K_act and K_pass), lam_out . dS/d c_D and
 * lam_out . dS/d phi_int [per radian; 0 for k_mode 0].  For stage-level
 * gradient checks. */
int moses_stage_adjoint(moses_sim *s, double t, double dt, const double *lam_out, double *lam_in,
                        double *g_param);

/* ---- Step without device allocation --------------------------------------
 * The paper has no counterpart to this call.  It is for callers that cannot
 * let a library allocate device memory: host programs that reserve all device
 * memory in their own pool (a foreign cudaMalloc fails or fragments it),
 * processes under a hard device-memory limit, and loops that may not stall
 * on the allocator (cudaMalloc and cudaFree synchronise the device).  It
 * advances one FP64 Heun step
 * of a grid of at most MOSES_STATIC_MAX_NX x MOSES_STATIC_MAX_NY cells and
 * calls no cudaMalloc, cudaFree or allocating library routine: its scratch
 * (extended DEM, geometry, padded state, Heun intermediate, control block,
 * about 7.7 MB) is a statically sized device array that every GPU loading the
 * library holds until the process exits.
 *   dem_device   nx*ny bed elevations (device memory, caller's)
 *   U_in_device  6*nx*ny conserved state, same plane order as
 *                moses_get_conserved (device memory, caller's)
 *   U_out_device 6*nx*ny, receives U^{n+1}; may equal U_in_device
 *   t            time of U_in (start of the step); closed / transmissive
 *                boundaries only (no inflow segments); p->precision must be
 *                MOSES_FP64 and p->nu_f 0
 *   dt_out       host pointer receiving the time step taken, or NULL.
 *                Non-NULL: the call synchronises the stream, reads the time
 *                step and the device status word, and returns ENONFINITE
 *                when the input or the result holds a non-finite value.
 *                NULL: nothing is read back, the call returns as soon as its
 *                work is queued, and a non-finite result is not reported.
 *   stream       cudaStream_t or NULL
 * The first call on a device looks up that device's copy of the array
 * (cudaGetSymbolAddress) and keeps the address for the rest of the process;
 * make that first call before any stream capture, and do not use this call
 * again on a device after cudaDeviceReset in the same process (the kept
 * address would be stale).  Every call shares the array and overwrites it, so
 * calls that overlap on the GPU (other streams, other threads) race;
 * serialise them.  Errors (read with moses_last_error(NULL)): EINVAL for
 * sizes beyond the limit or bad arguments, ENONFINITE (dt_out non-NULL
 * only), ECUDA. */
#define MOSES_STATIC_MAX_NX 128
#define MOSES_STATIC_MAX_NY 128
int moses_step_static(const double *dem_device, int nx, int ny, double dx, double dy,
                      const moses_params *p, const double *U_in_device, double *U_out_device,
                      double t, double *dt_out, void *stream);

/* Testing the failure path of the one device-side wait: with on != 0 the
 * wet/dry classification of the following steps waits for 16 bytes that no
 * copy delivers, so its bounded wait (about 0.5 s per CTA, twice) runs out;
 * the step then returns MOSES_ETIMEOUT, and a later step does so again until
 * a new state is set.  No fault is raised: the wait simply ends.  on = 0
 * restores normal stepping.  Errors: EINVAL. */
int moses_debug_timeout(moses_sim *s, int on);

/* Debugging aid (not in the paper): fills every element of the simulation's
 * device buffers that no kernel may read -- the pitch padding to the right of
 * the second ghost column, in every plane of the state, the Heun intermediate
 * and the geometry -- with a quiet NaN.  A later run that gives the same
 * result as an unpoisoned one shows that no stencil reads outside its cells
 * (the canary test of the test suite).  Errors: EINVAL, ECUDA. */
int moses_debug_poison(moses_sim *s);

/* Testing the arithmetic the stage kernels build on (not in the paper): for
 * each of the n host values x[k] (1 <= n <= 2^24), out (9 n doubles, host)
 * receives, plane by plane: the kernels' FP64 reciprocal 1/x, CUDA's 1.0/x,
 * the kernels' FP64 square root, CUDA's sqrt, the kernels' FP64 reciprocal
 * square root, CUDA's rsqrt, and the kernels' FP32 reciprocal, square root
 * and reciprocal square root of (float)x.  The FP64 functions start from the
 * hardware approximations and take one third-order refinement step each
 * (series of (1-e)^-1 and (1-d)^-1/2); the reciprocal is defined for x whose
 * reciprocal is a normal number, the square root gives 0 for x <= 0 or
 * subnormal.  Uses the current device; allocates and frees a scratch buffer.
 * Errors (moses_last_error(NULL)): EINVAL, ECUDA. */
int moses_debug_math(const double *x, int n, double *out);

/* Measuring the FP64 roof the stage kernel's FP64 form runs against (not in
 * the paper): times `reps` launches (1..1000, after one warm-up) of a kernel
 * that runs eight independent FP64 FMA chains per thread in registers on
 * 4 CTAs of 256 threads per SM, and returns the best rate in *tflops
 * [TFLOP/s, 2 flops per FMA].  Uses the current device and the legacy default
 * stream.  Errors (moses_last_error(NULL)): EINVAL, ECUDA. */
int moses_debug_fp64_rate(int reps, double *tflops);

/* Evaluating a double-float flux phase (not in the paper; the arithmetic is
 * NOT IEEE FP64): the stage's central flux through one face (twice the flux
 * of Sect. 2.2 with the fluxes of App. A) on n synthetic x-faces
 * (1 <= n <= 2^22; masses, velocities and pressure coefficients of a release
 * event, one side and phase in eight dry), computed in FP64 and in
 * double-float arithmetic (each value a pair of FP32 numbers, about 48
 * significant bits, on the FP32 pipes).  The inputs are made once in both
 * types before the timed launches, which only load them, run the flux and
 * store the results in their own type.  Each form runs `reps` (4..64)
 * dependent repetitions per face; the rate counts the difference between
 * `reps` and 2 repetitions (CUDA events, the fastest of three launches each),
 * so that the loads and the stores cancel.  res (4 doubles, host):
 * [0] FP64 face fluxes per second over the GPU [1e9 / s], [1] the same in
 * double-float, [2] the relative max-norm of the double-float fluxes against
 * the FP64 ones (over the seven flux components, max |difference| / max |FP64
 * value|), [3] the largest relative difference of one component where the
 * FP64 value exceeds 1e-6 of its component's largest.  Uses the current
 * device; allocates and frees 472 n bytes.
 * Errors (moses_last_error(NULL)): EINVAL, ENOMEM, ECUDA. */
int moses_debug_flux_eval(long long n, int reps, double *res);

/* Library build identification (architecture, precision forms). */
const char *moses_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MOSES_H */
