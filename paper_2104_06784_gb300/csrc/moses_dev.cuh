// moses_dev.cuh -- device-side data layout shared by the kernels of the
// two-phase shallow-flow step (arXiv:2104.06784, App. A and Sect. 2.2).
//
// HBM layout of one simulation (nx x ny interior cells, G = 2 ghost layers):
//   plane     : (ny + 4) rows of `pitch` elements, pitch = nx + 4 rounded up
//               to 32 elements; interior cell (i, j) at (j + 2) * pitch + i + 2
//   state U   : 6 planes, U1..U6 (structure of arrays), element type T
//   scratch U*: 6 planes (the Heun intermediate state)
//   FP32 form : 2 more planes after each of U and U*, the FP32 rounding
//               remainders of the two mass components (compensated mass)
//   geometry  : GEO_PLANES planes of T, computed once per DEM
//   control   : one Ctl block (time, dt, a_max bits, FP64 budgets, status)
#pragma once
#include <cstdint>

namespace moses {

constexpr int GH = 2;          // ghost layers of the state
constexpr int MAX_INFLOW = 8;  // inflow segments per simulation
constexpr int MAX_HYD = 64;    // samples per hydrograph

// Geometry planes, computed once per DEM and parameter set (cell centres and
// faces; faces indexed by their lower cell).  kap_s = eps g (1 - alpha) / 2,
// kap_f = eps g / 2; A = (A_ij) the 2x2 block of Omega_b^-1; c = n_Z = 1/J.
enum GeoPlane : int {
    GC_J = 0,   // J_b = sqrt(1 + bX^2 + bY^2)
    GC_C,       // c = n_Z
    GC_JHD,     // J h_dry            (dry test of a phase: U > J h_dry)
    GC_GC1,     // g (1 - alpha) c    (J p_b^s = U1 (g (1 - alpha) c - eps^chi kappa^s))
    GC_GCF,     // g c                (J p_b^f = U4 (g c - eps^chi kappa^f))
    GC_BX,      // dB/dX (central difference)
    GC_BY,      // dB/dY
    GC_MNX,     // -c bX = n_X        (s_n = J p_b (n_X, n_Y))
    GC_MNY,     // -c bY = n_Y
    GC_A11,     // (1 + bY^2) / J^2
    GC_A12,     // -bX bY / J^2 (= A21)
    GC_A22,     // (1 + bX^2) / J^2
    GC_KXX,     // c bXX     kappa = -(KXX vX^2 + KXY2 vX vY + KYY vY^2)
    GC_KXY2,    // 2 c bXY
    GC_KYY,     // c bYY
    GC_SXS,     // kap_s K_pass A11 c^2   cell-centre wave speeds (CFL; K_pass = 1 unless k_mode 1)
    GC_SXF,     // 2 kap_f A11 c^2
    GC_SYS,     // kap_s K_pass A22 c^2
    GC_SYF,     // 2 kap_f A22 c^2
    GX_JHD,     // x-face (i+1/2, j): J h_dry
    GX_SN,      //   kap_s A11 c^2 : solid X-momentum pressure coefficient, solid speed
    GX_ST,      //   kap_s A12 c^2 : solid Y-momentum pressure coefficient
    GX_FN,      //   kap_f A11 c^2 : fluid X-momentum
    GX_FT,      //   kap_f A12 c^2 : fluid Y-momentum
    GX_FN2,     //   2 kap_f A11 c^2 : fluid speed
    GX_HG,      //   (g/2) c^2 : P = J h pbar^f = (g/2) c^2 (J h)^2
    GY_JHD,     // y-face (i, j+1/2)
    GY_SN,      //   kap_s A22 c^2 : solid Y-momentum, solid speed
    GY_ST,      //   kap_s A21 c^2 : solid X-momentum
    GY_FN,      //   kap_f A22 c^2
    GY_FT,      //   kap_f A21 c^2
    GY_FN2,     //   2 kap_f A22 c^2
    GY_HG,      //   (g/2) c^2
    GEO_PLANES
};
// FP32 form (and FP64 with the viscous term): four more planes from which the
// stage kernel rebuilds the cell and face geometry in the tile (the same
// formulas as the geometry pass): the cell's central slopes bX, bY and the face-normal differences
// (b_{i+1,j} - b_{i,j}) / dx, (b_{i,j+1} - b_{i,j}) / dy.  Curvatures follow
// as differences of these: bXX from DBX, bYY from DBY, bXY from SY along X.
enum SlopePlane : int { GS_SX = GEO_PLANES, GS_SY, GS_DBX, GS_DBY, GEO_PLANES_F32 };

// Device control block, one per simulation (or per ensemble member).
struct Ctl {
    double t;                     // time of the current state
    double dt;                    // time step of the step in progress
    unsigned long long amax;      // IEEE bits of a_max of the current state
    unsigned long long amax_acc;  // accumulator for a_max of the next state
    unsigned int ticket;          // blocks finished in the step's last kernel
    int status;                   // STATUS_* bits raised on the device
    long long steps;              // steps taken
    double bnd_in[2];             // time-integrated boundary volume inflow
    double clamp_vol[2];          // volume added by the positivity clamp
    unsigned long long clamp_cells;
    double dt_fixed;              // > 0: prescribed time step
    double t_end;                 // > 0: shorten the step to land on t_end
};

enum Status : int { STATUS_NONFINITE = 1, STATUS_TIMEOUT = 2 };

struct InflowSeg {
    int side, i0, i1, npts;
    double t[MAX_HYD], Q[MAX_HYD], phi[MAX_HYD];
};

// Physical constants of the step (all derived on the host from moses_params)
struct Phys {
    double kap_s;      // eps g (1 - alpha) / 2 : solid pressure factor
    double kap_f;      // eps g / 2             : fluid pressure factor
    double half_g;     // g / 2                 : P = half_g c^2 Ut^2
    double g_1ma;      // g (1 - alpha)
    double g;
    double eps_chi;
    double eps_alpha;  // eps alpha
    double eps;
    double alpha;
    double c_d, k_f, nu_f, tan_delta, h_dry;
    double cfl, dt_max, dmin;
    double dx, dy, inv_dx, inv_dy;
    double cell_area;  // dx dy
    int pg_mode;       // 0: phi^s (reaction reading), 1: phi^f (as printed)
    int scheme;        // 0: central flux, 1: central-upwind flux
    int recon;         // 0: minmod slopes, 1: third-order WENO
    int rk;            // 2: two-step modified Euler, 3: three-stage SSP Runge-Kutta
    int bc[4];
    // internal friction (reading R10): k_mode 1 scales the solid pressure of
    // each direction by the Savage-Hutter coefficient K_act or K_pass (both 1
    // in the paper's form, k_mode 0); the CFL celerity takes K_pass
    int k_mode;
    double K_act, K_pass;
};

// Constants of the stage kernel in its arithmetic type, prepared on the host
// (the FP32 form then runs no FP64 conversions per thread).
template <typename T>
struct KT {
    T eps_chi, eps_alpha, eps, alpha, c_d, k_f, hinv_dx, hinv_dy, tan_delta;
    // geometry rebuilt from slopes (FP32 form)
    T kap_s, kap_f, kap_f2, half_g, g_1ma, g, h_dry, inv_dx, inv_dy, inv_2dx;
    // viscous term (Eq. SrcF_vis_Topo): nu_f, 1/(2 dy)
    T nu_f, inv_2dy;
    // earth-pressure coefficients (k_mode 1) and the CFL celerity's solid
    // pressure factor kap_s K_pass (FP32 form)
    T Ka, Kp, kap_s_cfl;
    double tan_delta_d;
};

template <typename T>
inline KT<T> make_kt(const Phys &p)
{
    KT<T> k;
    k.eps_chi = (T)p.eps_chi;
    k.eps_alpha = (T)p.eps_alpha;
    k.eps = (T)p.eps;
    k.alpha = (T)p.alpha;
    k.c_d = (T)p.c_d;
    k.k_f = (T)p.k_f;
    k.hinv_dx = (T)(0.5 * p.inv_dx);
    k.hinv_dy = (T)(0.5 * p.inv_dy);
    k.tan_delta = (T)p.tan_delta;
    k.kap_s = (T)p.kap_s;
    k.kap_f = (T)p.kap_f;
    k.kap_f2 = (T)(2.0 * p.kap_f);
    k.half_g = (T)p.half_g;
    k.g_1ma = (T)p.g_1ma;
    k.g = (T)p.g;
    k.h_dry = (T)p.h_dry;
    k.inv_dx = (T)p.inv_dx;
    k.inv_dy = (T)p.inv_dy;
    k.inv_2dx = (T)(0.5 * p.inv_dx);
    k.nu_f = (T)p.nu_f;
    k.inv_2dy = (T)(0.5 * p.inv_dy);
    k.Ka = (T)p.K_act;
    k.Kp = (T)p.K_pass;
    k.kap_s_cfl = (T)(p.kap_s * p.K_pass);
    k.tan_delta_d = p.tan_delta;
    return k;
}

// Everything a stage kernel needs.
template <typename T>
struct alignas(8) StageArgs {
    const T *Uin;      // stage input (ghosts valid on the four sides)
    const T *Un;       // stage 2: U^n for the Heun average (interior); else null
    T *Uout;           // stage output (may equal Un in stage 2: same cell only)
    // FP32 form only: rounding remainders of the two mass components (2 planes
    // each; the mass of a cell is U + R); null in the FP64 form
    const T *Rin;
    const T *Rn;
    T *Rout;
    const T *geo;
    Ctl *ctl;
    const InflowSeg *inflow;
    int n_inflow;
    int nx, ny, pitch;
    // rows [own_j0, own_j1) are this simulation's own (all rows, unless it is
    // one strip of a decomposed domain): only their cells enter the CFL
    // maximum and the clamp counts, only their boundary faces the boundary
    // budget
    int own_j0, own_j1;
    long long plane;   // elements per plane
    Phys ph;
    KT<T> k;
    int stage;         // 1 or 2
    int want_amax;     // stage 2: reduce a_max of U^{n+1}
    int debug_stage;   // 1: single stage to Uout with a given dt (no Heun)
    double dbg_t, dbg_dt;
    // three-stage SSP Runge-Kutta: 0 for the two-step Euler, else the stage
    // (1, 2, 3; `stage` is 1 for the first, 2 for the others, which combine
    // with Un); rk3_bw is the stage's weight in the budgets (1/6, 1/6, 2/3)
    int rk3;
    double rk3_bw;
    // recording form only (the adjoint's recompute): per interior cell the
    // trial masses and solid momenta before friction and the clamp, and the
    // gradient of P (6 planes: U1*, U2*, U3*, U4*, dP/dxi, dP/deta)
    T *rec;
    // wet-tile list of the stepping launches (plain form): classify_kernel
    // writes the dry tiles' zero state and lists the tiles that hold mass,
    // which the stage kernel then runs; wl_n[0] entries, wl_n[1] CTAs done.
    // Null: every tile tests itself.
    int *wl;
    unsigned int *wl_n;
    // per tile of the launch's shape (row-major, ceil(nx/32) across): 1 where
    // the stage's classification found work.  The first stage of a step tests
    // the data and writes tw_next; a later stage (tw_prev non-null) takes a
    // tile as wet where it or a neighbouring tile was wet in the stage before
    // (its input has mass only there, and the 2-cell halo lies in the
    // neighbours), reading no state, and writes tw_next.
    const unsigned char *tw_prev;
    unsigned char *tw_next;
    // known-zero flags of the output buffer, per tile of the launch's shape
    // (null: every dry tile is written).  1 where the buffer's tile -- the
    // state, the FP32 remainders and the ghost cells the tile's cells own --
    // holds the zero state of an earlier write of the classification; such a
    // tile, dry again, is not written again.  The classification keeps them:
    // 1 for a dry tile, 0 for a tile with work and for a tile on a side with
    // an inflow segment (its ghost state follows the hydrograph).
    unsigned char *zk;
    // per-tile mass bits (MB_* below), so that a stage can be classified
    // without reading the state.  mb_out: the bits of Uout, written for every
    // tile (the classification zeroes a dry tile's, the stage kernel sets a
    // wet tile's from the values it stores).  mb_in: the bits of Uin; with
    // mb_ok the classification takes the wet tiles from them, otherwise the
    // data classification of a first stage writes them.  mb_n: the bits of
    // U^n in a combining stage.  All null outside the stepping launches.
    unsigned short *mb_in, *mb_out;
    const unsigned short *mb_n;
    int mb_ok;
    // testing only: extra bytes the classification's copy barrier expects and
    // no copy delivers, so that its bounded wait runs out (0 normally)
    unsigned int dbg_stall_tx;
    // the adjoint's runs: fix != 0 makes the step's first stage start at fix_t
    // with the time step fix_dt (a recomputed step, as the forward took it)
    // instead of the control block's time and CFL step; with t_log non-null
    // the first stage writes the step's start time and time step to
    // t_log[log_idx], dt_log[log_idx] (the forward run's record)
    int fix;
    double fix_t, fix_dt;
    double *t_log, *dt_log;
    int log_idx;
    // with wbox non-null the classification also widens wbox (x min, y min,
    // x max, y max of the launch's tiles) to every tile it lists: the box of
    // the stage's work, which the adjoint's kernels then cover
    int *wbox;
};

// Mass bits of a 32 x TY tile: where its cells hold mass (U1 or U4 non-zero,
// NaN included, or a non-zero FP32 mass remainder).  MB_ANY: some cell; the
// others: a cell within two cells of a side (W: columns 0-1, E: columns
// 30-31, S: rows 0-1, N: the last two rows) or of a corner (both).  A tile
// needs its stage where its own bits have MB_ANY or a neighbour's bits have
// the side or corner that faces it (the stencil's 2-cell reach).
enum : unsigned short {
    MB_ANY = 1u, MB_W = 2u, MB_E = 4u, MB_S = 8u, MB_N = 16u,
    MB_SW = 32u, MB_SE = 64u, MB_NW = 128u, MB_NE = 256u
};

__host__ __device__ inline long long cell_index(int i, int j, int pitch)
{
    return (long long)(j + GH) * pitch + (i + GH);
}

}  // namespace moses

// launchers of the templated stage kernels (one translation unit per type)
namespace moses {
struct BatchTile;
struct BatchStrip;
// the wet/dry classification works on strips of 32 columns by kStripRows rows,
// one CTA of kStripWarps warps each
constexpr int kStripRows = 16, kStripWarps = 4;
template <typename T>
int launch_stage(const StageArgs<T> &a, int tile, void *stream);
// the same stage (tile 32 x 8) that also writes a.rec
template <typename T>
int launch_stage_rec(const StageArgs<T> &a, void *stream);
// an ensemble run (BatchRun, stage.cuh) with 32 x ty tiles (ty 4, 8 or 16):
// one cooperative launch of every CTA that fits at once; *grid (may be NULL)
// gets that grid; with r.nstages == 0 nothing is launched
template <typename T>
struct BatchRun;
template <typename T>
int launch_batch(const BatchRun<T> &r, int ty, int *grid, void *stream);
}  // namespace moses
