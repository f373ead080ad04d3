// internal.cuh -- the simulation object and host helpers shared by the
// translation units of the library (not part of the public C-ABI).
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/moses.h"
#include "moses_dev.cuh"

using namespace moses;

struct moses_sim {
    int nx = 0, ny = 0, pitch = 0;
    long long plane = 0;  // elements per plane
    double dx = 0, dy = 0;
    moses_params p{};
    Phys ph{};
    int prec = MOSES_FP64;
    size_t esz = 8;  // bytes per state element
    cudaStream_t stream = nullptr;
    void *U = nullptr;     // state, 6 planes
    void *Us = nullptr;    // Heun intermediate, 6 planes
    void *geo = nullptr;   // geo_planes(s) planes
    void *Us2 = nullptr;   // second intermediate of the three-stage Runge-Kutta (rk = 3 only)
    int *wl = nullptr;              // wet-tile list of the stepping launches (one entry per 32 x 4 tile)
    unsigned int *wl_n = nullptr;   // its two counters
    unsigned char *tw[2] = {nullptr, nullptr};  // per-tile wet flags of the stages (ping-pong)
    // known-zero tile flags of U, Us and Us2 (three arrays of one byte per
    // 32 x 4 tile), kept by the stepping launches.  They describe the buffers
    // only while the stepping launches are their sole writer: every other call
    // that may write a buffer, or that changes the tile shape, clears
    // zk_valid, and the next step starts from all-zero flags.
    unsigned char *zk = nullptr;
    bool zk_valid = false;
    // mass bits of U, Us and Us2 (StageArgs::mb_in), valid with zk_valid: the
    // first stage of a step then classifies from U's bits
    unsigned short *mb = nullptr;
    int dbg_stall = 0;              // moses_debug_timeout: the classification's copy wait runs out
    Ctl *ctl = nullptr;    // device control block
    InflowSeg *inflow_d = nullptr;
    InflowSeg inflow_h[MAX_INFLOW];
    int n_inflow = 0;
    double *stage_buf = nullptr;  // dense 6*nx*ny doubles (host <-> device staging)
    double *red = nullptr;        // 8 doubles for reductions
    bool have_state = false;
    int tile = 0;
    int own_j0 = 0, own_j1 = 0;  // owned rows (moses_set_owned_rows; all rows by default)
    std::string err;
};

// rows of the tiles of a MOSES_TILE_* shape
inline int tile_rows(int tile) { return tile == 1 || tile == 3 ? 4 : tile == 2 ? 16 : 8; }

extern std::string g_create_err;

// ---------------------------------------------------------------------------
// error helpers

// the known-zero tile flags no longer describe the buffers (see moses_sim::zk)
inline void zk_reset(moses_sim *s)
{
    if (s) s->zk_valid = false;
}

// declared first in a call that may write the state buffers by another route
// than the stepping launches: clears zk_valid when the call returns
struct ZkReset {
    moses_sim *s;
    ~ZkReset() { zk_reset(s); }
};

inline int fail(moses_sim *s, int code, const std::string &msg)
{
    if (s) s->err = msg;
    else g_create_err = msg;
    return code;
}

#define CK(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(s, e_ == cudaErrorMemoryAllocation ? MOSES_ENOMEM : MOSES_ECUDA,              \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                          \
    } while (0)


// the simulation is one strip of a decomposed domain (moses_set_owned_rows)
inline bool is_strip(const moses_sim *s) { return s->own_j0 != 0 || s->own_j1 != s->ny; }

inline int grid_for(long long n, int block = 256)
{
    long long b = (n + block - 1) / block;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

// the slope planes: always in FP32 (its stage rebuilds the geometry from
// them), in FP64 only for the viscous term (face metric in the tile)
inline bool has_slopes(const moses_sim *s) { return s->prec == MOSES_FP32 || s->p.nu_f > 0.0; }
inline int geo_planes(const moses_sim *s) { return has_slopes(s) ? (int)GEO_PLANES_F32 : (int)GEO_PLANES; }

// remainder planes (FP32 form) that follow the six state planes of a buffer
template <typename T>
inline T *rem(moses_sim *s, void *buf)
{
    return s->prec == MOSES_FP32 ? (T *)buf + 6 * s->plane : nullptr;
}

template <typename T>
inline StageArgs<T> base_args(moses_sim *s)
{
    StageArgs<T> a{};
    a.geo = (const T *)s->geo;
    a.ctl = s->ctl;
    a.inflow = s->inflow_d;
    a.n_inflow = s->n_inflow;
    a.nx = s->nx;
    a.ny = s->ny;
    a.own_j0 = s->own_j0;
    a.own_j1 = s->own_j1;
    a.pitch = s->pitch;
    a.plane = s->plane;
    a.ph = s->ph;
    a.k = make_kt<T>(s->ph);
    a.dbg_stall_tx = s->dbg_stall ? 16u : 0u;
    return a;
}

