// moses_dev.cuh -- device-side data layout shared by the kernels of the
// two-phase shallow-flow step (arXiv:2104.06784, App. A and Sect. 2.2).
//
// HBM layout of one simulation (nx x ny interior cells, G = 2 ghost layers):
//   plane     : (ny + 4) rows of `pitch` elements, pitch = nx + 4 rounded up
//               to 32 elements; interior cell (i, j) at (j + 2) * pitch + i + 2
//   state U   : 6 planes, U1..U6 (structure of arrays), element type T
//   scratch U*: 6 planes (the Heun intermediate state)
//   geometry  : GEO_PLANES planes of T, computed once per DEM
//   control   : one Ctl block (time, dt, a_max bits, FP64 budgets, status)
#pragma once
#include <cstdint>

namespace moses {

constexpr int GH = 2;          // ghost layers of the state
constexpr int MAX_INFLOW = 8;  // inflow segments per simulation
constexpr int MAX_HYD = 64;    // samples per hydrograph

// geometry planes (cell centres and faces; faces indexed by their lower cell)
enum GeoPlane : int {
    GC_J = 0,   // J_b = sqrt(1 + bX^2 + bY^2)
    GC_C,       // c = n_Z = 1 / J_b
    GC_BX,      // dB/dX (central difference)
    GC_BY,      // dB/dY
    GC_A11,     // (Omega_b^-1)_11 = (1 + bY^2) / J^2
    GC_A12,     // (Omega_b^-1)_12 = (Omega_b^-1)_21 = -bX bY / J^2
    GC_A22,     // (Omega_b^-1)_22 = (1 + bX^2) / J^2
    GC_KXX,     // c bXX   (curvature of the bed; kappa = -(KXX vX^2 + 2 KXY vX vY + KYY vY^2))
    GC_KXY,     // c bXY
    GC_KYY,     // c bYY
    GC_G11,     // A11 c^2 (cell-centre wave speed along xi)
    GC_G22,     // A22 c^2 (along eta)
    GX_J,       // x-face (i+1/2, j): J_b
    GX_GN,      //   A11 c^2 : pressure coefficient of the X-momentum flux
    GX_GT,      //   A12 c^2 : pressure coefficient of the Y-momentum flux
    GX_C2,      //   c^2     : P = J h pbar^f = (g/2) c^2 (J h)^2
    GY_J,       // y-face (i, j+1/2): J_b
    GY_GN,      //   A22 c^2 : Y-momentum flux
    GY_GT,      //   A21 c^2 : X-momentum flux
    GY_C2,
    GEO_PLANES
};

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
    int bc[4];
};

// Everything a stage kernel needs.
template <typename T>
struct StageArgs {
    const T *Uin;      // stage input (ghosts valid on the four sides)
    const T *Un;       // stage 2: U^n for the Heun average (interior); else null
    T *Uout;           // stage output (may equal Un in stage 2: same cell only)
    const T *geo;
    Ctl *ctl;
    const InflowSeg *inflow;
    int n_inflow;
    int nx, ny, pitch;
    long long plane;   // elements per plane
    Phys ph;
    int stage;         // 1 or 2
    int want_amax;     // stage 2: reduce a_max of U^{n+1}
    int debug_stage;   // 1: single stage to Uout with a given dt (no Heun)
    double dbg_t, dbg_dt;
};

__host__ __device__ inline long long cell_index(int i, int j, int pitch)
{
    return (long long)(j + GH) * pitch + (i + GH);
}

}  // namespace moses

// launchers of the templated stage kernels (one translation unit per type)
namespace moses {
template <typename T>
int launch_stage(const StageArgs<T> &a, int tile, void *stream);
int stage_tiles_available(int *tiles, int max);
}  // namespace moses
