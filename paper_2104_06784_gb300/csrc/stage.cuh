// stage.cuh -- one stage U + dt L(U) of the two-phase shallow-flow scheme on
// sm_103a, templated on the storage/arithmetic type T (double or float).
//
// L(U) is the semi-discrete central (Kurganov-Tadmor) scheme of Sect. 2.2
// with minmod reconstruction of the conserved variables, the fluxes of
// App. A (Eqs. FluxEqSxi_Topo .. FluxEqFeta_Topo) and the sources of App. A
// (Eqs. Src_nd_Topo, Src_f_Topo, Src_v_Topo, SrcF_nd_Topo, SrcF_f_Topo,
// SrcF_v_Topo).  Coulomb friction is applied semi-implicitly with a stopping
// condition, then the positivity clamp and the dry-momentum rule.
//
// Work decomposition: one CTA per TX x TY tile.  The CTA stages the 6 state
// planes of the tile plus a 2-cell halo in shared memory (coalesced loads),
// computes every x-face and y-face flux of the tile exactly once into shared
// memory, then updates its cells.  In stage 2 it also forms the Heun average
// in place, writes the ghost cells of the new state (boundary conditions
// fused into the producer), and reduces the CFL wave speed: warp shuffle max,
// CTA max, one atomicMax on the IEEE bits of a non-negative double (exact and
// independent of order).  The last CTA to finish (ticket counter, no waiting)
// turns the maximum into the next time step.
#pragma once
#include <cuda_runtime.h>

#include "moses_dev.cuh"

namespace moses {

template <typename T>
struct K {  // constants in the arithmetic type
    T kap_s, kap_f2, kap_f, half_g, g_1ma, g, eps_chi, eps_alpha, eps, alpha, c_d, k_f, h_dry, inv_dx,
        inv_dy;
    double tan_delta;
    __device__ explicit K(const Phys &p)
        : kap_s((T)p.kap_s), kap_f2((T)(2.0 * p.kap_f)), kap_f((T)p.kap_f), half_g((T)p.half_g),
          g_1ma((T)p.g_1ma), g((T)p.g), eps_chi((T)p.eps_chi), eps_alpha((T)p.eps_alpha), eps((T)p.eps),
          alpha((T)p.alpha), c_d((T)p.c_d), k_f((T)p.k_f), h_dry((T)p.h_dry), inv_dx((T)p.inv_dx),
          inv_dy((T)p.inv_dy), tan_delta(p.tan_delta)
    {
    }
};

__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double tabs(double x) { return fabs(x); }
__device__ __forceinline__ float tabs(float x) { return fabsf(x); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }

__device__ __forceinline__ bool nonfinite(double x)
{
    return (__double2hiint(x) & 0x7ff00000) == 0x7ff00000;
}
__device__ __forceinline__ bool nonfinite(float x) { return (__float_as_int(x) & 0x7f800000) == 0x7f800000; }

// minmod of two one-sided undivided differences (Sect. 2.2)
template <typename T>
__device__ __forceinline__ T minmod(T a, T b)
{
    if (a * b <= T(0)) return T(0);
    return a > T(0) ? tmin(a, b) : tmax(a, b);
}

template <typename T>
struct FaceGeo {
    T J, gn, gt, c2;
};

// Physical flux of one reconstructed state through a face of direction d
// (0: xi = X, 1: eta = Y), the per-phase local speeds and P = J h pbar^f.
// With xi = X, eta = Y the tangential velocity v_xi equals v_X, the mass flux
// J h^p v_xi^p is the momentum component U_{2+d}, and the pressure terms
// eps J h A_dk Nbar^s, eps J h A_dk pbar^f become (A_dk c^2) kap (J h) U.
template <typename T>
__device__ __forceinline__ void side_flux(const T u[6], const FaceGeo<T> &G, int d, const K<T> &k, T F[6],
                                          T &as, T &af, T &P)
{
    const T Ut = u[0] + u[3];
    const T hd = G.J * k.h_dry;
    const bool ws = u[0] > hd, wf = u[3] > hd;
    const T rs = ws ? T(1) / u[0] : T(0);
    const T rf = wf ? T(1) / u[3] : T(0);
    const T vns = (d == 0 ? u[1] : u[2]) * rs;
    const T vnf = (d == 0 ? u[4] : u[5]) * rf;
    const T cX = d == 0 ? G.gn : G.gt;
    const T cY = d == 0 ? G.gt : G.gn;
    const T ps = k.kap_s * Ut * u[0];
    const T pf = k.kap_f * Ut * Ut;
    F[0] = ws ? (d == 0 ? u[1] : u[2]) : T(0);
    F[1] = u[1] * vns + cX * ps;
    F[2] = u[2] * vns + cY * ps;
    F[3] = wf ? (d == 0 ? u[4] : u[5]) : T(0);
    F[4] = u[4] * vnf + cX * pf;
    F[5] = u[5] * vnf + cY * pf;
    as = tabs(vns) + tsqrt(G.gn * k.kap_s * (Ut + u[0]));
    af = tabs(vnf) + tsqrt(G.gn * k.kap_f2 * Ut);
    P = k.half_g * G.c2 * Ut * Ut;
}

// Central flux through one face from the four cells a | b || c | d along the
// face normal (values um = b + slope_b/2, up = c - slope_c/2).
template <typename T>
__device__ __forceinline__ void face_flux(const T *s0, int stride_c, int o_a, int o_b, int o_c, int o_d,
                                          const FaceGeo<T> &G, int d, const K<T> &k, T H[7])
{
    T um[6], up[6];
#pragma unroll
    for (int c = 0; c < 6; c++) {
        const T *p = s0 + c * stride_c;
        const T ua = p[o_a], ub = p[o_b], uc = p[o_c], ud = p[o_d];
        const T dC = uc - ub;
        um[c] = ub + T(0.5) * minmod(ub - ua, dC);
        up[c] = uc - T(0.5) * minmod(dC, ud - uc);
    }
    T Fm[6], Fp[6], asm_, afm, asp, afp, Pm, Pp;
    side_flux(um, G, d, k, Fm, asm_, afm, Pm);
    side_flux(up, G, d, k, Fp, asp, afp, Pp);
    const T as = tmax(asm_, asp), af = tmax(afm, afp);
#pragma unroll
    for (int c = 0; c < 6; c++) {
        const T a = c < 3 ? as : af;
        H[c] = T(0.5) * (Fm[c] + Fp[c]) - T(0.5) * a * (up[c] - um[c]);
    }
    H[6] = T(0.5) * (Pm + Pp);
}

__device__ __forceinline__ double interp_series(const double *t, const double *v, int n, double tt)
{
    if (n <= 0 || tt < t[0] || tt > t[n - 1]) return 0.0;
    for (int q = 0; q < n - 1; q++) {
        if (tt <= t[q + 1]) {
            double w = (t[q + 1] > t[q]) ? (tt - t[q]) / (t[q + 1] - t[q]) : 1.0;
            return v[q] + w * (v[q + 1] - v[q]);
        }
    }
    return v[n - 1];
}

// Ghost state of an inflow segment (Sect. 3.1.2 Mode-II): the mixture at
// critical depth for the unit discharge q = Q / width, moving inward.
// J, c, Ann: geometry of the ghost cell (Ann = A11 on W/E, A22 on S/N).
template <typename T>
__device__ void inflow_state(const InflowSeg &f, double J, double c, double Ann, const Phys &ph, double tt,
                             T u[6])
{
#pragma unroll
    for (int q = 0; q < 6; q++) u[q] = T(0);
    const double W = (f.i1 - f.i0) * ((f.side < 2) ? ph.dy : ph.dx);
    const double Q = interp_series(f.t, f.Q, f.npts, tt);
    const double phs = interp_series(f.t, f.phi, f.npts, tt);
    if (!(Q > 0.0) || W <= 0.0) return;
    const double q = Q / W;
    const double hc = cbrt(q * q / (J * J * ph.eps * ph.g * c * Ann));
    const double vn = q / (J * hc);
    const double sgn = (f.side == 0 || f.side == 2) ? 1.0 : -1.0;
    const double U1 = J * hc * phs, U4 = J * hc * (1.0 - phs);
    u[0] = (T)U1;
    u[3] = (T)U4;
    if (f.side < 2) {
        u[1] = (T)(U1 * sgn * vn);
        u[4] = (T)(U4 * sgn * vn);
    } else {
        u[2] = (T)(U1 * sgn * vn);
        u[5] = (T)(U4 * sgn * vn);
    }
}

template <typename T>
__device__ __forceinline__ void store6(T *U, long long plane, long long idx, const T v[6])
{
#pragma unroll
    for (int c = 0; c < 6; c++) U[c * plane + idx] = v[c];
}

// Ghost cells of the state just written for cell (i, j) (R4: closed = mirror
// with negated normal momentum, transmissive = zero-gradient copy; inflow
// segments override their side's rule).  The thread owning each mirror or
// copy source writes the ghost, so no other pass over the boundary is needed.
template <typename T>
__device__ void write_ghosts(T *U, const T *geo, const StageArgs<T> &a, int i, int j, const T v[6], double tg)
{
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    const long long plane = a.plane;
    const Phys &ph = a.ph;
    if (i < 2 || i >= nx - 2) {
#pragma unroll
        for (int side = 0; side < 2; side++) {
            // inflow rows on this side
            int seg = -1;
            for (int f = 0; f < a.n_inflow; f++)
                if (a.inflow[f].side == side && j >= a.inflow[f].i0 && j < a.inflow[f].i1) seg = f;
            const bool closed = ph.bc[side] == 0;
            for (int kk = 0; kk < GH; kk++) {
                const int gi = side == 0 ? -1 - kk : nx + kk;
                int src;
                if (side == 0) src = closed ? (kk < nx ? kk : nx - 1) : 0;
                else src = closed ? (nx - 1 - kk >= 0 ? nx - 1 - kk : 0) : nx - 1;
                if (seg >= 0) {
                    if (i != (side == 0 ? 0 : nx - 1)) continue;
                    const long long gidx = cell_index(gi, j, pitch);
                    T u[6];
                    inflow_state<T>(a.inflow[seg], (double)geo[GC_J * plane + gidx], (double)geo[GC_C * plane + gidx],
                                    (double)geo[GC_A11 * plane + gidx], ph, tg, u);
                    store6(U, plane, gidx, u);
                } else if (src == i) {
                    T u[6] = {v[0], v[1], v[2], v[3], v[4], v[5]};
                    if (closed) {
                        u[1] = -u[1];
                        u[4] = -u[4];
                    }
                    store6(U, plane, cell_index(gi, j, pitch), u);
                }
            }
        }
    }
    if (j < 2 || j >= ny - 2) {
#pragma unroll
        for (int side = 2; side < 4; side++) {
            int seg = -1;
            for (int f = 0; f < a.n_inflow; f++)
                if (a.inflow[f].side == side && i >= a.inflow[f].i0 && i < a.inflow[f].i1) seg = f;
            const bool closed = ph.bc[side] == 0;
            for (int kk = 0; kk < GH; kk++) {
                const int gj = side == 2 ? -1 - kk : ny + kk;
                int src;
                if (side == 2) src = closed ? (kk < ny ? kk : ny - 1) : 0;
                else src = closed ? (ny - 1 - kk >= 0 ? ny - 1 - kk : 0) : ny - 1;
                if (seg >= 0) {
                    if (j != (side == 2 ? 0 : ny - 1)) continue;
                    const long long gidx = cell_index(i, gj, pitch);
                    T u[6];
                    inflow_state<T>(a.inflow[seg], (double)geo[GC_J * plane + gidx], (double)geo[GC_C * plane + gidx],
                                    (double)geo[GC_A22 * plane + gidx], ph, tg, u);
                    store6(U, plane, gidx, u);
                } else if (src == j) {
                    T u[6] = {v[0], v[1], v[2], v[3], v[4], v[5]};
                    if (closed) {
                        u[2] = -u[2];
                        u[5] = -u[5];
                    }
                    store6(U, plane, cell_index(i, gj, pitch), u);
                }
            }
        }
    }
}

// largest cell-centre wave speed of a state (R7), both phases, both axes
template <typename T>
__device__ __forceinline__ double cell_speed(const T u[6], T J, T g11, T g22, const K<T> &k)
{
    const T Ut = u[0] + u[3];
    const T hd = J * k.h_dry;
    const T rs = u[0] > hd ? T(1) / u[0] : T(0);
    const T rf = u[3] > hd ? T(1) / u[3] : T(0);
    const T cs = k.kap_s * (Ut + u[0]);
    const T cf = k.kap_f2 * Ut;
    T m = tabs(u[1] * rs) + tsqrt(g11 * cs);
    m = tmax(m, tabs(u[4] * rf) + tsqrt(g11 * cf));
    m = tmax(m, tabs(u[2] * rs) + tsqrt(g22 * cs));
    m = tmax(m, tabs(u[5] * rf) + tsqrt(g22 * cf));
    return (double)m;
}

__device__ __forceinline__ double dt_from(const Ctl *ctl, const Phys &ph, double amax)
{
    double dt;
    if (ctl->dt_fixed > 0.0) {
        dt = ctl->dt_fixed;
    } else {
        dt = (amax > 0.0) ? ph.cfl * ph.dmin / amax : ph.dt_max;
        if (dt > ph.dt_max) dt = ph.dt_max;
    }
    if (ctl->t_end > 0.0 && ctl->t + dt > ctl->t_end) dt = ctl->t_end > ctl->t ? ctl->t_end - ctl->t : 0.0;
    return dt;
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) stage_kernel(const StageArgs<T> a)
{
    constexpr int NT = TX * TY;
    constexpr int SW = TX + 4, SH = TY + 4, SP = SW * SH;
    constexpr int NXF = (TX + 1) * TY, NYF = TX * (TY + 1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sU = reinterpret_cast<T *>(smem_raw);
    T *sHx = sU + 6 * SP;   // [7][TY][TX+1]
    T *sHy = sHx + 7 * NXF; // [7][TY+1][TX]
    __shared__ double red_d[NT / 32];
    __shared__ double acc[4];
    __shared__ unsigned int acc_n;
    __shared__ bool last_block;

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    const long long plane = a.plane;
    const K<T> k(a.ph);
    const T *geo = a.geo;
    Ctl *ctl = a.ctl;

    double t_now, dt;
    if (a.debug_stage) {
        t_now = a.dbg_t;
        dt = a.dbg_dt;
    } else if (a.stage == 1) {
        t_now = ctl->t;
        dt = dt_from(ctl, a.ph, __longlong_as_double((long long)ctl->amax));
    } else {
        t_now = ctl->t;
        dt = ctl->dt;
    }
    const T dtT = (T)dt;
    if (tid < 4) acc[tid] = 0.0;
    if (tid == 0) acc_n = 0;

    // ---- stage the tile + 2-cell halo of the six state planes -------------
    for (int e = tid; e < 6 * SP; e += NT) {
        const int c = e / SP, r = e - c * SP;
        const int ly = r / SW, lx = r - ly * SW;
        const int gi = x0 - 2 + lx, gj = y0 - 2 + ly;
        T v = T(0);
        if (gi < nx + 2 && gj < ny + 2) v = a.Uin[c * plane + cell_index(gi, gj, pitch)];
        sU[e] = v;
    }
    __syncthreads();

    // ---- x-faces (i+1/2, j), i = x0-1 .. x0+TX-1 ---------------------------
    for (int f = tid; f < NXF; f += NT) {
        const int ly = f / (TX + 1), lx = f - ly * (TX + 1);
        const int i = x0 + lx - 1, j = y0 + ly;
        if (j >= ny || i >= nx) continue;
        const long long gidx = cell_index(i, j, pitch);
        FaceGeo<T> G{geo[GX_J * plane + gidx], geo[GX_GN * plane + gidx], geo[GX_GT * plane + gidx],
                     geo[GX_C2 * plane + gidx]};
        const int ob = (ly + 2) * SW + lx + 1;  // left cell in smem
        T H[7];
        face_flux(sU, SP, ob - 1, ob, ob + 1, ob + 2, G, 0, k, H);
#pragma unroll
        for (int c = 0; c < 7; c++) sHx[c * NXF + f] = H[c];
        if (!a.debug_stage && (i == -1 || i == nx - 1)) {
            const double w = 0.5 * dt * a.ph.dy * (i == -1 ? 1.0 : -1.0);
            atomicAdd(&acc[0], w * (double)H[0]);
            atomicAdd(&acc[1], w * (double)H[3]);
        }
    }
    // ---- y-faces (i, j+1/2), j = y0-1 .. y0+TY-1 ---------------------------
    for (int f = tid; f < NYF; f += NT) {
        const int ly = f / TX, lx = f - ly * TX;
        const int i = x0 + lx, j = y0 + ly - 1;
        if (i >= nx || j >= ny) continue;
        const long long gidx = cell_index(i, j, pitch);
        FaceGeo<T> G{geo[GY_J * plane + gidx], geo[GY_GN * plane + gidx], geo[GY_GT * plane + gidx],
                     geo[GY_C2 * plane + gidx]};
        const int ob = (ly + 1) * SW + lx + 2;  // lower cell in smem
        T H[7];
        face_flux(sU, SP, ob - SW, ob, ob + SW, ob + 2 * SW, G, 1, k, H);
#pragma unroll
        for (int c = 0; c < 7; c++) sHy[c * NYF + f] = H[c];
        if (!a.debug_stage && (j == -1 || j == ny - 1)) {
            const double w = 0.5 * dt * a.ph.dx * (j == -1 ? 1.0 : -1.0);
            atomicAdd(&acc[0], w * (double)H[0]);
            atomicAdd(&acc[1], w * (double)H[3]);
        }
    }
    __syncthreads();

    // ---- cell update --------------------------------------------------------
    const int lx = tid % TX, ly = tid / TX;
    const int i = x0 + lx, j = y0 + ly;
    double speed = 0.0;
    bool bad = false;
    if (i < nx && j < ny) {
        const long long gidx = cell_index(i, j, pitch);
        const int os = (ly + 2) * SW + lx + 2;
        T u[6];
#pragma unroll
        for (int c = 0; c < 6; c++) u[c] = sU[c * SP + os];
        const T J = geo[GC_J * plane + gidx], c0 = geo[GC_C * plane + gidx];
        const T bX = geo[GC_BX * plane + gidx], bY = geo[GC_BY * plane + gidx];
        const T A11 = geo[GC_A11 * plane + gidx], A12 = geo[GC_A12 * plane + gidx],
                A22 = geo[GC_A22 * plane + gidx];
        const T kXX = geo[GC_KXX * plane + gidx], kXY = geo[GC_KXY * plane + gidx],
                kYY = geo[GC_KYY * plane + gidx];
        const T hd = J * k.h_dry;
        const T Ut = u[0] + u[3];
        // volume fractions phi^s, phi^f of the mixture (0 when h <= h_dry)
        const bool wet = Ut * c0 > k.h_dry;
        const T rUt = wet ? T(1) / Ut : T(0);
        const T phs = u[0] * rUt, phf = u[3] * rUt;
        const bool ws = u[0] > hd, wf = u[3] > hd;
        const T rs = ws ? T(1) / u[0] : T(0), rf = wf ? T(1) / u[3] : T(0);
        const T vXs = u[1] * rs, vYs = u[2] * rs, vXf = u[4] * rf, vYf = u[5] * rf;
        // kappa = v . (dn/dxi v_xi + dn/deta v_eta) = -c (bXX vX^2 + 2 bXY vX vY + bYY vY^2)
        const T ks = -(kXX * vXs * vXs + T(2) * kXY * vXs * vYs + kYY * vYs * vYs);
        const T kf = -(kXX * vXf * vXf + T(2) * kXY * vXf * vYf + kYY * vYf * vYf);
        // J p_b for each phase, clamped at 0 (lift-off)
        const T Jpbs = tmax(T(0), u[0] * (k.g_1ma * c0 - k.eps_chi * ks));
        const T Jpbf = tmax(T(0), u[3] * (k.g * c0 - k.eps_chi * kf));
        // s_n = J p_b (n_X, n_Y) = J p_b c (-bX, -bY)
        const T nsX = -c0 * bX, nsY = -c0 * bY;
        // gradient of P = J h pbar^f from its face values
        const int fx = ly * (TX + 1) + lx, fy = ly * TX + lx;
        const T dPx = (sHx[6 * NXF + fx + 1] - sHx[6 * NXF + fx]) * k.inv_dx;
        const T dPy = (sHy[6 * NYF + fy + TX] - sHy[6 * NYF + fy]) * k.inv_dy;
        const T gX = A11 * dPx + A12 * dPy, gY = A12 * dPx + A22 * dPy;
        const T fpg = a.ph.pg_mode == 1 ? phf : phs;
        const T bs = -k.eps_alpha * phs, bf = k.eps * fpg;
        // interphase drag J c_D phi^s phi^f h = c_D phi^s phi^f (J h)
        const T D = k.c_d * phs * phf * Ut;
        const T dvX = vXf - vXs, dvY = vYf - vYs;
        const T ff = k.k_f * phf * Ut;  // fluid basal friction J phi^f h k_f
        T S[6];
        S[0] = T(0);
        S[3] = T(0);
        S[1] = Jpbs * nsX + bs * gX + k.alpha * D * dvX;
        S[2] = Jpbs * nsY + bs * gY + k.alpha * D * dvY;
        S[4] = Jpbf * nsX + bf * gX - D * dvX - ff * vXf;
        S[5] = Jpbf * nsY + bf * gY - D * dvY - ff * vYf;
        T out[6];
#pragma unroll
        for (int c = 0; c < 6; c++) {
            const T divx = (sHx[c * NXF + fx + 1] - sHx[c * NXF + fx]) * k.inv_dx;
            const T divy = (sHy[c * NYF + fy + TX] - sHy[c * NYF + fy]) * k.inv_dy;
            out[c] = u[c] + dtT * (S[c] - (divx + divy));
        }
        // Coulomb friction with stopping (semi-implicit, direction from q*),
        // decided in FP64 in both precision forms
        {
            const double qX = (double)out[1], qY = (double)out[2];
            const double qZ = (double)bX * qX + (double)bY * qY;
            const double qn = sqrt(qX * qX + qY * qY + qZ * qZ);
            const double Fr = dt * (double)Jpbs * k.tan_delta;
            if (qn <= Fr) {
                out[1] = T(0);
                out[2] = T(0);
            } else {
                const double r = 1.0 - Fr / qn;
                out[1] = (T)(qX * r);
                out[2] = (T)(qY * r);
            }
        }
        // positivity clamp (counted) and dry momentum
#pragma unroll
        for (int ph = 0; ph < 2; ph++) {
            const int c = 3 * ph;
            if (out[c] < T(0)) {
                if (!a.debug_stage) {
                    atomicAdd(&acc[2 + ph], -0.5 * (double)out[c] * a.ph.cell_area);
                    atomicAdd(&acc_n, 1u);
                }
                out[c] = T(0);
            }
            if (out[c] <= hd) {
                out[c + 1] = T(0);
                out[c + 2] = T(0);
            }
        }
        if (a.stage == 2 && !a.debug_stage) {
            // Heun average with U^n (same cell), dry momentum again
#pragma unroll
            for (int c = 0; c < 6; c++) out[c] = T(0.5) * (a.Un[c * plane + gidx] + out[c]);
#pragma unroll
            for (int ph = 0; ph < 2; ph++)
                if (out[3 * ph] <= hd) {
                    out[3 * ph + 1] = T(0);
                    out[3 * ph + 2] = T(0);
                }
            if (a.want_amax)
                speed = cell_speed(out, J, geo[GC_G11 * plane + gidx], geo[GC_G22 * plane + gidx], k);
        }
#pragma unroll
        for (int c = 0; c < 6; c++) bad |= nonfinite(out[c]);
        if (a.debug_stage) {
            store6(a.Uout, plane, gidx, out);
        } else {
            store6(a.Uout, plane, gidx, out);
            write_ghosts(a.Uout, geo, a, i, j, out, t_now + dt);
        }
    }

    if (a.debug_stage) return;

    // ---- CTA reductions -----------------------------------------------------
    if (bad) atomicOr(&ctl->status, (int)STATUS_NONFINITE);
    if (a.stage == 2 && a.want_amax) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) speed = fmax(speed, __shfl_xor_sync(0xffffffffu, speed, o));
        if ((tid & 31) == 0) red_d[tid >> 5] = speed;
    }
    __syncthreads();
    if (tid == 0) {
        if (acc[0] != 0.0) atomicAdd(&ctl->bnd_in[0], acc[0]);
        if (acc[1] != 0.0) atomicAdd(&ctl->bnd_in[1], acc[1]);
        if (acc_n) {
            atomicAdd(&ctl->clamp_vol[0], acc[2]);
            atomicAdd(&ctl->clamp_vol[1], acc[3]);
            atomicAdd(&ctl->clamp_cells, (unsigned long long)acc_n);
        }
        if (a.stage == 1 && blockIdx.x == 0 && blockIdx.y == 0) ctl->dt = dt;
        if (a.stage == 2) {
            if (a.want_amax) {
                double m = 0.0;
                for (int w = 0; w < NT / 32; w++) m = fmax(m, red_d[w]);
                atomicMax(&ctl->amax_acc, (unsigned long long)__double_as_longlong(m));
            }
            __threadfence();
            const unsigned int nb = gridDim.x * gridDim.y;
            last_block = (atomicAdd(&ctl->ticket, 1u) == nb - 1);
        }
    }
    if (a.stage != 2) return;
    __syncthreads();
    if (last_block && tid == 0) {
        __threadfence();
        const unsigned long long m = atomicExch(&ctl->amax_acc, 0ull);
        if (a.want_amax) ctl->amax = m;
        ctl->ticket = 0;
        if (ctl->dt > 0.0) {
            ctl->t = ctl->t + ctl->dt;
            ctl->steps += 1;
        }
        const double am = __longlong_as_double((long long)m);
        if (a.want_amax && am != am) atomicOr(&ctl->status, (int)STATUS_NONFINITE);
    }
}

template <typename T, int TX, int TY>
constexpr size_t stage_smem_bytes()
{
    return sizeof(T) * (6 * (TX + 4) * (TY + 4) + 7 * (TX + 1) * TY + 7 * TX * (TY + 1));
}

}  // namespace moses
