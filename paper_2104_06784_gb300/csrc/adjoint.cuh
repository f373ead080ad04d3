// adjoint.cuh -- reverse (vector-Jacobian) form of one stage of the
// two-phase shallow-flow scheme, for gradients of a deposit misfit with respect
// to the basal friction, the drag coefficient and the initial state.
//
// The stage U -> S(U) of stage.cuh is differentiated with the time step held
// fixed (it is recorded by the forward run).  Where the scheme has kinks the
// derivative of the branch the forward took is used: minmod -> the selected
// difference (0 when the limiter returns 0); max of the two local speeds -> the
// selected side; Coulomb stopping -> 0 for a stopped cell; positivity clamp
// and dry rule -> 0 for the clamped or zeroed values; |v| -> sign(v).
//
// The adjoint of a stage is computed by three kernels so that every tile
// gathers (no scatter across tiles):
//   A  per cell, pointwise: from the stage input, the trial state before
//      friction and the pressure gradient that the recording forward stage
//      kept (StageArgs::rec), reverse the masks, the friction, the sources and
//      the update.  Writes the adjoint of the pre-friction output lam_pre (6),
//      of the pressure gradient (dP/dxi, dP/deta), the cell's own
//      contributions (identity + sources + friction, and the direct Heun
//      term) into lam_in, and the parameter partials (tan delta_b, c_D)
//      reduced per CTA.
//   B  per face: recompute the face states (halo 3), form the flux adjoints
//      from lam_pre and the pressure adjoints of the two neighbours, reverse
//      the central flux and the minmod reconstruction, and gather per cell:
//      lam_in += face terms; ghost cells at the boundary get theirs.
//   C  fold the ghost cells' adjoints into their mirror / copy sources
//      (inflow ghosts are constants).
// Heun: U^{n+1} = dry(1/2 (U^n + S(S(U^n)))).  With lam^{n+1} given, the
// second stage's A takes lam_out = 1/2 lam^{n+1} with the momenta zeroed where
// U^{n+1} is dry, and the first stage's A adds that same term to its cell
// result, writing lam^n over lam^{n+1} in place (each cell reads its own
// value before it writes it; no other thread reads it).
#pragma once
#include "stage.cuh"

namespace moses {

__device__ __forceinline__ double tsgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }
__device__ __forceinline__ float tsgn(float x) { return x > 0.0f ? 1.0f : (x < 0.0f ? -1.0f : 0.0f); }

// adjoint of side_flux: given the adjoints of F (6), as, af and P, add the
// adjoint of the reconstructed state u to lu
template <typename T, int D>
__device__ __forceinline__ void side_flux_vjp(const T u[6], const FaceGeo<T> &G, const T lF[6], T las, T laf, T lP,
                                              T lu[6])
{
    const T Ut = u[0] + u[3];
    const bool ws = gtp(u[0], G.jhd), wf = gtp(u[3], G.jhd);
    const T rs = ws ? frcp(u[0]) : T(0);
    const T rf = wf ? frcp(u[3]) : T(0);
    const T uns = D == 0 ? u[1] : u[2];
    const T unf = D == 0 ? u[4] : u[5];
    const T vns = uns * rs, vnf = unf * rf;
    const T sX = D == 0 ? G.sn : G.st, sY = D == 0 ? G.st : G.sn;
    const T fX = D == 0 ? G.fn : G.ft, fY = D == 0 ? G.ft : G.fn;
    const T qs = fsqrt(G.sn * (Ut + u[0])), qf = fsqrt(G.fn2 * Ut);
    // F1 = sX Ps + u1 vns, F2 = sY Ps + u2 vns, F4 = fX Pf + u4 vnf, F5 = fY Pf + u5 vnf
    const T lvns = lF[1] * u[1] + lF[2] * u[2] + las * tsgn(vns);
    const T lvnf = lF[4] * u[4] + lF[5] * u[5] + laf * tsgn(vnf);
    const T lPs = lF[1] * sX + lF[2] * sY;
    const T lPf = lF[4] * fX + lF[5] * fY + lP * G.hg;
    // Ps = Ut u0, Pf = Ut^2, as = |vns| + sqrt(sn (Ut + u0)), af = |vnf| + sqrt(fn2 Ut)
    T lUt = lPs * u[0] + T(2) * Ut * lPf;
    T lu0 = lPs * Ut;
    if (qs > T(0)) {
        const T t = las * G.sn / (T(2) * qs);
        lUt += t;
        lu0 += t;
    }
    if (qf > T(0)) lUt += laf * G.fn2 / (T(2) * qf);
    lu[1] += lF[1] * vns;
    lu[2] += lF[2] * vns;
    lu[4] += lF[4] * vnf;
    lu[5] += lF[5] * vnf;
    // vns = uns / u0 (wet), F0 = uns (wet)
    const T luns = lvns * rs + (ws ? lF[0] : T(0));
    const T lunf = lvnf * rf + (wf ? lF[3] : T(0));
    T lu3 = T(0);
    if (ws) lu0 -= lvns * vns * rs;
    if (wf) lu3 -= lvnf * vnf * rf;
    lu[0] += lu0 + lUt;
    lu[3] += lu3 + lUt;
    lu[1 + D] += luns;
    lu[4 + D] += lunf;
}

// adjoint of face_flux2 (H2 = F(um) + F(up) - a (up - um), H2[6] = P(um) + P(up));
// Gm, Gp: the face geometry of each side (solid pressure coefficients scaled
// by that side's earth-pressure coefficient with k_mode 1).  With KM it also
// returns lH . dH2/dK for each side's coefficient (G: the unscaled geometry):
// dF1/dK = sX Ps, dF2/dK = sY Ps, and the solid speed's
// d sqrt(K sn (Ut + u0))/dK = sn (Ut + u0) / (2 sqrt(..)) where that side
// gives the face its speed.
template <typename T, int D, bool KM = false>
__device__ __forceinline__ void face_flux2_vjp(const T um[6], const T up[6], const FaceGeo<T> &Gm, const FaceGeo<T> &Gp,
                                               const T lH[6], T lP2, T lum[6], T lup[6], const FaceGeo<T> *G = nullptr,
                                               T *lKm = nullptr, T *lKp = nullptr)
{
    T Fm[6], Fp[6], asm_, afm, asp, afp, Pm, Pp;
    side_flux<T, D>(um, Gm, Fm, asm_, afm, Pm);
    side_flux<T, D>(up, Gp, Fp, asp, afp, Pp);
    const bool ms = ibits(asm_) >= ibits(asp), mf = ibits(afm) >= ibits(afp);  // maxnn picks the first on ties
    const T as = ms ? asm_ : asp, af = mf ? afm : afp;
    T las = T(0), laf = T(0);
#pragma unroll
    for (int c = 0; c < 6; c++) {
        const T a = c < 3 ? as : af;
        const T d = up[c] - um[c];
        if (c < 3) las -= lH[c] * d;
        else laf -= lH[c] * d;
        lum[c] = a * lH[c];
        lup[c] = -a * lH[c];
    }
    side_flux_vjp<T, D>(um, Gm, lH, ms ? las : T(0), mf ? laf : T(0), lP2, lum);
    side_flux_vjp<T, D>(up, Gp, lH, ms ? T(0) : las, mf ? T(0) : laf, lP2, lup);
    if constexpr (KM) {
        const T sX = D == 0 ? G->sn : G->st, sY = D == 0 ? G->st : G->sn;
        const auto dK = [&](const T u[6], const FaceGeo<T> &Gs, const bool sel) -> T {
            const T Ut = u[0] + u[3], Ps = Ut * u[0], w = Ut + u[0];
            T r = lH[1] * (sX * Ps) + lH[2] * (sY * Ps);
            const T cs = fsqrt(Gs.sn * w);
            if (sel && cs > T(0)) r += las * (G->sn * w / (T(2) * cs));
            return r;
        };
        *lKm = dK(um, Gm, ms);
        *lKp = dK(up, Gp, !ms);
    }
}

// minmod selection: 0 -> returned 0, 1 -> returned a, 2 -> returned b
__device__ __forceinline__ int minmod_sel(double a, double b)
{
    const long long ia = ibits(a), ib = ibits(b);
    const long long ma = ia & 0x7fffffffffffffffll, mb = ib & 0x7fffffffffffffffll;
    if ((ia ^ ib) < 0 || ma == 0 || mb == 0) return 0;
    return ma < mb ? 1 : 2;
}
__device__ __forceinline__ int minmod_sel(float a, float b)
{
    if (!(a * b > 0.0f)) return 0;  // as the FP32 minmod
    return fabsf(a) < fabsf(b) ? 1 : 2;
}

// Arguments of the adjoint kernels
template <typename T>
struct AdjArgs {
    StageArgs<T> f;   // the forward stage (Uin = the stage input, rec = its record; geometry, constants)
    const T *lam_out; // adjoint of the stage output (6 planes, interior); unused when heun == 2
    T *lam_pre;       // A -> B: adjoint of the pre-friction output (6 planes)
    T *lam_dp;        // A -> B: adjoint of dP/dxi, dP/deta (2 planes)
    T *lam_in;        // adjoint of the stage input (6 planes, ghosts included): A writes the
                      // cells' own contributions, B adds the face terms and sets the ghosts
    double *g_param;  // [0] d/d tan(delta_b), [1] d/d c_D; with k_mode 1 also
                      // [2] d/d K_act, [3] d/d K_pass (FP64 accumulators)
    // Heun: 2 = second stage (A reads lam_next), 1 = first stage (B adds the
    // direct term; lam_in == lam_next), 0 = a lone stage
    int heun;
    const T *lam_next;  // lam^{n+1} (6 planes, interior)
    const T *U_next;    // U^{n+1} (its dry mask)
    // Tiles far from any mass (the run of many steps): tw is the stage's
    // tile-wet map of the recording recompute (32 x 8 tiles, tgx x tgy; null:
    // every tile computes).  A tile with no wet tile within two tiles has no
    // mass near its cells, the face tiles that read its cells' lam_pre and
    // lam_dp are dry too, and the exact reverse there is the identity on the
    // mass adjoints with zero momentum adjoints: the second Heun stage skips
    // it (its lam_in is read only where the first stage computes), the first
    // stage leaves lam in place and zeroes its momentum planes unless lamz
    // (one byte per tile: the tile's momentum adjoints of lam are 0) says so.
    const unsigned char *tw;
    int tgx, tgy;
    unsigned char *lamz;
    // the face kernel folds the ghost adjoints its tile owns into their
    // sources itself (every source lies in the owning tile: the last tile
    // along each axis holds two cells or more), and no fold kernel runs
    int fold_inline;
    // the launch covers a box of tiles: CTA (blockIdx.x, blockIdx.y) takes
    // the 32 x 8 tile (bx0 + blockIdx.x, by0 + blockIdx.y)
    int bx0, by0;
};

// the tile (bx, by) of the adjoint kernels lies two tiles or more from every
// wet tile of the stage (see AdjArgs::tw)
// (the 25 flags are loaded together, one memory latency, and OR-ed: an early
// exit would chain the loads, and most CTAs of a step are such far tiles)
template <typename T>
__device__ __forceinline__ bool adj_far_from_mass(const AdjArgs<T> &q, int bx, int by)
{
    unsigned int any = 0u;
#pragma unroll
    for (int dy = -2; dy <= 2; dy++)
#pragma unroll
        for (int dx = -2; dx <= 2; dx++) {
            const int xx = bx + dx, yy = by + dy;
            if (xx >= 0 && xx < q.tgx && yy >= 0 && yy < q.tgy) any |= q.tw[yy * q.tgx + xx];
        }
    return any == 0u;
}

// 1/2 lam^{n+1}, momenta zeroed where U^{n+1} is dry (adjoint of the Heun
// average followed by the dry rule), component c of cell g
template <typename T>
__device__ __forceinline__ T heun_half(const AdjArgs<T> &q, long long g, int c, T jhd)
{
    const long long plane = q.f.plane;
    const int ph = c / 3;
    if (c != 3 * ph && !gtp(q.U_next[3 * ph * plane + g], jhd)) return T(0);
    return T(0.5) * q.lam_next[c * plane + g];
}

}  // namespace moses

namespace moses {

// J h_dry of cell g as the stage kernel computes it (FP32: from the slopes)
template <typename T>
__device__ __forceinline__ T cell_jhd(const StageArgs<T> &a, long long g)
{
    if constexpr (sizeof(T) == 4) {
        const T sX = a.geo[GS_SX * a.plane + g], sY = a.geo[GS_SY * a.plane + g];
        const T s2 = fma(sX, sX, fma(sY, sY, T(1)));
        return s2 * frsqrt(s2) * a.k.h_dry;
    } else {
        return a.geo[GC_JHD * a.plane + g];
    }
}

// ---- kernel A: cell adjoint (pointwise) --------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) adj_cell_kernel(const AdjArgs<T> q)
{
    constexpr int NT = 256;
    __shared__ double red[2][NT / 32];
    wait_prior_grid();  // launched after the kernel before it (launch_after)
    const StageArgs<T> &a = q.f;
    const int tid = threadIdx.x;
    const int tbx = q.bx0 + (int)blockIdx.x, tby = q.by0 + (int)blockIdx.y;  // the tile (AdjArgs::bx0)
    const int i = tbx * 32 + (tid & 31), j = tby * 8 + (tid >> 5);
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    const long long plane = a.plane;
    const KT<T> &k = a.k;
    const T *geo = a.geo;
    const double dt = a.dbg_dt;
    const T dtT = (T)dt;
    if (q.tw && adj_far_from_mass(q, tbx, tby)) {  // CTA-uniform (AdjArgs::tw)
        if (q.heun != 1) return;
        const int tile = tby * q.tgx + tbx;
        if (q.lamz[tile]) return;
        if (i < nx && j < ny) {
            const long long g = cell_index(i, j, pitch);
#pragma unroll
            for (int c = 0; c < 6; c++)
                if (c != 0 && c != 3) q.lam_in[c * plane + g] = T(0);
        }
        if (tid == 0) q.lamz[tile] = 1;
        return;
    }
    if (q.lamz && q.heun == 1 && tid == 0) q.lamz[tby * q.tgx + tbx] = 0;
    // parameter partials: per cell and across the warp in T, per CTA and
    // globally in FP64 (the FP64 pipe of GB300 is 1/64 of its FP32 rate)
    T g_tan = T(0), g_cd = T(0);
    bool dry_cell = false;
    if (i < nx && j < ny) {
        // no mass before the stage nor in its trial output: velocities,
        // pressures, sources and friction are 0 and the dry rule zeroes the
        // momenta, so the reverse passes the mass adjoints through and gives 0
        // for the rest (what the full computation below gives for such a cell)
        const long long g = cell_index(i, j, pitch);
        const T m0 = a.Uin[g], m3 = a.Uin[3 * plane + g], p0 = a.rec[g], p3 = a.rec[3 * plane + g];
        if (!(nonzero(m0) | nonzero(m3) | nonzero(p0) | nonzero(p3))) {
            dry_cell = true;
            const T l0 = q.heun == 2 ? T(0.5) * q.lam_next[g] : q.lam_out[g];
            const T l3 = q.heun == 2 ? T(0.5) * q.lam_next[3 * plane + g] : q.lam_out[3 * plane + g];
            const T lp[6] = {l0, T(0), T(0), l3, T(0), T(0)};
            const T jhd1 = q.heun == 1 ? cell_jhd(a, g) : T(0);
#pragma unroll
            for (int c = 0; c < 6; c++) {
                q.lam_pre[c * plane + g] = lp[c];
                q.lam_in[c * plane + g] = q.heun == 1 ? lp[c] + heun_half(q, g, c, jhd1) : lp[c];
            }
            q.lam_dp[g] = T(0);
            q.lam_dp[plane + g] = T(0);
        }
    }
    if (i < nx && j < ny && !dry_cell) {
        const long long g = cell_index(i, j, pitch);
        T u[6], pre4[4];
#pragma unroll
        for (int c = 0; c < 6; c++) u[c] = a.Uin[c * plane + g];
#pragma unroll
        for (int c = 0; c < 4; c++) pre4[c] = a.rec[c * plane + g];
        const T dPx = a.rec[4 * plane + g], dPy = a.rec[5 * plane + g];
        // ---- forward quantities of the cell (as in stage_tile) ----
        // the cell geometry: FP32 rebuilt from the slope planes exactly as the
        // FP32 stage does, FP64 read from the geometry planes
        T jhd, kXX, kXY2, kYY, gc1, gcf, nX, nY, bX, bY, A11, A12, A22;
        if constexpr (sizeof(T) == 4) {
            const T *sl = geo + GS_SX * plane + g;
            const CellGeo32 G = cell_geo32(sl[0], sl[plane], (sl[2 * plane] - sl[2 * plane - 1]) * k.inv_dx,
                                           (sl[plane + 1] - sl[plane - 1]) * k.inv_2dx,
                                           (sl[3 * plane] - sl[3 * plane - pitch]) * k.inv_dy, k);
            jhd = G.jhd, kXX = G.kXX, kXY2 = G.kXY2, kYY = G.kYY, gc1 = G.gc1, gcf = G.gcf;
            nX = G.nX, nY = G.nY, bX = G.bX, bY = G.bY, A11 = G.A11, A12 = G.A12, A22 = G.A22;
        } else {
            jhd = geo[GC_JHD * plane + g];
            kXX = geo[GC_KXX * plane + g], kXY2 = geo[GC_KXY2 * plane + g], kYY = geo[GC_KYY * plane + g];
            gc1 = geo[GC_GC1 * plane + g], gcf = geo[GC_GCF * plane + g];
            nX = geo[GC_MNX * plane + g], nY = geo[GC_MNY * plane + g];
            bX = geo[GC_BX * plane + g], bY = geo[GC_BY * plane + g];
            A11 = geo[GC_A11 * plane + g], A12 = geo[GC_A12 * plane + g], A22 = geo[GC_A22 * plane + g];
        }
        const T Ut = u[0] + u[3];
        const bool wmix = gtp(Ut, jhd), ws = gtp(u[0], jhd), wf = gtp(u[3], jhd);
        const T rUt = wmix ? frcp(Ut) : T(0);
        const T phs = u[0] * rUt, phf = u[3] * rUt;
        const T rs = ws ? frcp(u[0]) : T(0), rf = wf ? frcp(u[3]) : T(0);
        const T vXs = u[1] * rs, vYs = u[2] * rs, vXf = u[4] * rf, vYf = u[5] * rf;
        const T nks = fma(kXX, vXs * vXs, fma(kXY2, vXs * vYs, kYY * (vYs * vYs)));
        const T nkf = fma(kXX, vXf * vXf, fma(kXY2, vXf * vYf, kYY * (vYf * vYf)));
        const T ps_raw = u[0] * fma(k.eps_chi, nks, gc1), pf_raw = u[3] * fma(k.eps_chi, nkf, gcf);
        const T Jpbs = pos(ps_raw);
        const T gX = fma(A11, dPx, A12 * dPy), gY = fma(A12, dPx, A22 * dPy);
        const bool pgf = a.ph.pg_mode == 1;
        const T bs = -k.eps_alpha * phs;
        const T bf = k.eps * (pgf ? phf : phs);
        const T D = k.c_d * phs * phf * Ut;
        const T aD = k.alpha * D;
        const T dvX = vXf - vXs, dvY = vYf - vYs;
        const T ff = k.k_f * phf * Ut;
        // friction on the recorded trial momentum
        const T Fr = dtT * Jpbs * k.tan_delta;
        const T q1 = pre4[1], q2 = pre4[2];
        const T qZ = fma(bX, q1, bY * q2);
        const T qn2 = fma(q1, q1, fma(q2, q2, qZ * qZ));
        bool stopped;  // the forward's decision (FP32: with its FP64 tie-break)
        if constexpr (sizeof(T) == 4) stopped = coulomb_stops(q1, q2, bX, bY, Fr, qn2, dt, Jpbs, k.tan_delta_d);
        else stopped = !gtp(qn2, Fr * Fr);
        const bool rubs = !stopped && ibits(Fr) > 0;  // friction acts
        const T rr = rubs ? frsqrt(qn2) : T(0);
        const T r = rubs ? fma(-Fr, rr, T(1)) : T(1);
        bool clamped[2], dry[2];
#pragma unroll
        for (int ph = 0; ph < 2; ph++) {
            clamped[ph] = negative(pre4[3 * ph]);
            const T m = clamped[ph] ? T(0) : pre4[3 * ph];
            dry[ph] = !gtp(m, jhd);
        }
        // ---- reverse ----
        T lo[6];
#pragma unroll
        for (int c = 0; c < 6; c++) lo[c] = q.heun == 2 ? heun_half(q, g, c, jhd) : q.lam_out[c * plane + g];
        // clamp and dry rule
#pragma unroll
        for (int ph = 0; ph < 2; ph++) {
            if (clamped[ph]) lo[3 * ph] = T(0);
            if (dry[ph]) {
                lo[3 * ph + 1] = T(0);
                lo[3 * ph + 2] = T(0);
            }
        }
        // friction
        T lpre[6] = {lo[0], T(0), T(0), lo[3], lo[4], lo[5]};
        T lFr = T(0);
        if (!stopped && !rubs) {
            lpre[1] = lo[1];
            lpre[2] = lo[2];
        }
        if (rubs) {
            const T sq = lo[1] * q1 + lo[2] * q2;
            const T t = ((sq * rr) * rr) * (Fr * rr);  // sq rr <= |lo|: no overflow for tiny |q*|
            lpre[1] = fma(r, lo[1], t * fma(qZ, bX, q1));
            lpre[2] = fma(r, lo[2], t * fma(qZ, bY, q2));
            lFr = -sq * rr;
        }
        T lJpbs = lFr * dtT * k.tan_delta;
        g_tan += lFr * dtT * Jpbs;
        // update pre = u + dt (S - div): identity, sources; div goes to faces via lam_pre
        T lu[6], lS[6];
#pragma unroll
        for (int c = 0; c < 6; c++) {
            lu[c] = lpre[c];
            lS[c] = dtT * lpre[c];
        }
        lJpbs += lS[1] * nX + lS[2] * nY;
        const T lJpbf = lS[4] * nX + lS[5] * nY;
        const T lbs = lS[1] * gX + lS[2] * gY;
        const T lbf = lS[4] * gX + lS[5] * gY;
        const T lgX = lS[1] * bs + lS[4] * bf, lgY = lS[2] * bs + lS[5] * bf;
        const T laD = lS[1] * dvX + lS[2] * dvY;
        const T lD = -(lS[4] * dvX + lS[5] * dvY) + laD * k.alpha;
        const T ldvX = lS[1] * aD - lS[4] * D, ldvY = lS[2] * aD - lS[5] * D;
        const T lff = -(lS[4] * vXf + lS[5] * vYf);
        T lvXf = -lS[4] * ff + ldvX, lvYf = -lS[5] * ff + ldvY;
        T lvXs = -ldvX, lvYs = -ldvY;
        T lphs = T(0), lphf = T(0), lUt = T(0);
        // ff = k_f phf Ut ; D = c_D phs phf Ut
        lphf += lff * k.k_f * Ut;
        lUt += lff * k.k_f * phf;
        g_cd += lD * phs * phf * Ut;
        lphs += lD * k.c_d * phf * Ut;
        lphf += lD * k.c_d * phs * Ut;
        lUt += lD * k.c_d * phs * phf;
        // bs = -eps alpha phs ; bf = eps phi
        lphs -= lbs * k.eps_alpha;
        if (pgf) lphf += lbf * k.eps;
        else lphs += lbf * k.eps;
        // gX, gY -> the pressure-gradient adjoints (to faces)
        const T ldPx = lgX * A11 + lgY * A12, ldPy = lgX * A12 + lgY * A22;
        // J p_b = max(0, U (g c - eps_chi kappa))
        T lnks = T(0), lnkf = T(0);
        if (ibits(ps_raw) > 0) {
            lu[0] += lJpbs * fma(k.eps_chi, nks, gc1);
            lnks = lJpbs * u[0] * k.eps_chi;
        }
        if (ibits(pf_raw) > 0) {
            lu[3] += lJpbf * fma(k.eps_chi, nkf, gcf);
            lnkf = lJpbf * u[3] * k.eps_chi;
        }
        lvXs += lnks * fma(T(2) * kXX, vXs, kXY2 * vYs);
        lvYs += lnks * fma(kXY2, vXs, T(2) * kYY * vYs);
        lvXf += lnkf * fma(T(2) * kXX, vXf, kXY2 * vYf);
        lvYf += lnkf * fma(kXY2, vXf, T(2) * kYY * vYf);
        // velocities v = q / U
        lu[1] += lvXs * rs;
        lu[2] += lvYs * rs;
        lu[4] += lvXf * rf;
        lu[5] += lvYf * rf;
        if (ws) lu[0] -= (lvXs * vXs + lvYs * vYs) * rs;
        if (wf) lu[3] -= (lvXf * vXf + lvYf * vYf) * rf;
        // volume fractions phi = U / Ut
        lu[0] += lphs * rUt;
        lu[3] += lphf * rUt;
        if (wmix) lUt -= (lphs * phs + lphf * phf) * rUt;
        lu[0] += lUt;
        lu[3] += lUt;
#pragma unroll
        for (int c = 0; c < 6; c++) {
            q.lam_pre[c * plane + g] = lpre[c];
            q.lam_in[c * plane + g] = q.heun == 1 ? lu[c] + heun_half(q, g, c, jhd) : lu[c];
        }
        q.lam_dp[g] = ldPx;
        q.lam_dp[plane + g] = ldPy;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        g_tan += __shfl_xor_sync(0xffffffffu, g_tan, o);
        g_cd += __shfl_xor_sync(0xffffffffu, g_cd, o);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = (double)g_tan;
        red[1][tid >> 5] = (double)g_cd;
    }
    __syncthreads();
    if (tid == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < NT / 32; w++) {
            s0 += red[0][w];
            s1 += red[1][w];
        }
        if (s0 != 0.0) atomicAdd(&q.g_param[0], s0);
        if (s1 != 0.0) atomicAdd(&q.g_param[1], s1);
    }
}

}  // namespace moses

namespace moses {

// ---- kernel B: face adjoint and gather ----------------------------------------
// D = 0: x-faces over rows of the tile; D = 1: y-faces over columns.  Along the
// face normal the tile covers cells [o0 - 2, o0 + L + 1] with slopes, faces with
// lower cell in [o0 - 2, o0 + L], slope adjoints for cells [o0 - 1, o0 + L].
// In the FP32 form the bed slopes (4 planes, from which the face geometry is
// rebuilt as the FP32 stage does) and the cell adjoints lam_pre, lam_dp of
// the tile and a 2-cell halo are staged in shared memory up front, so that
// the face loop reads no global memory; FP64 reads its face geometry and the
// cell adjoints in the loop (its shared memory is full at two CTAs per SM).
template <typename T, int TX, int TY, bool KM = false>
struct FaceAdjSmem {
    static constexpr bool STAGE = sizeof(T) == 4;
    static constexpr int SW3 = TX + 6, SH3 = TY + 6, SP3 = SW3 * SH3;
    static constexpr int NS = (TY * (TX + 4) > (TY + 4) * TX) ? TY * (TX + 4) : (TY + 4) * TX;
    static constexpr int NF = (TY * (TX + 3) > (TY + 3) * TX) ? TY * (TX + 3) : (TY + 3) * TX;
    static constexpr int NL = (TY * (TX + 2) > (TY + 2) * TX) ? TY * (TX + 2) : (TY + 2) * TX;
    static constexpr int LW = TX + 4, LP = LW * (TY + 4);  // lam box: tile + 2-cell halo
    static constexpr size_t sel_bytes = (6 * NS + 15) / 16 * 16;
    static constexpr size_t base = sizeof(T) * (6 * SP3 + 6 * NS + 12 * NF + 6 * NL) + sel_bytes;
    static constexpr size_t staged = base + (STAGE ? sizeof(T) * (8 * LP + 4 * LP) : 0);
    // earth-pressure form: solid velocities (v_X, v_Y) of the state box
    static constexpr size_t bytes = staged + (KM ? sizeof(T) * 2 * SP3 : 0);
};

// Cell h (0 <= h < (TX + 2 HW)(TY + 2 HW) - TX TY) of the halo of width HW
// around a TX x TY tile, in tile coordinates: the HW rows below, the HW rows
// above, then HW columns on each side of the tile's rows.
template <int TX, int TY, int HW>
__device__ __forceinline__ void halo_cell(int h, int &tx, int &ty)
{
    constexpr int W = TX + 2 * HW, RW = HW * W;
    if (h < RW) {
        ty = h / W - HW;
        tx = h - (ty + HW) * W - HW;
    } else if (h < 2 * RW) {
        h -= RW;
        ty = h / W;
        tx = h - ty * W - HW;
        ty += TY;
    } else {
        h -= 2 * RW;
        ty = h / (2 * HW);
        const int k = h - ty * (2 * HW);
        tx = k < HW ? k - HW : TX + k - HW;
    }
}

template <typename T, int TX, int TY, int D, bool KM = false>
__device__ __forceinline__ void adj_face_dir(const AdjArgs<T> &q, T *sU, T *sS, unsigned char *sSel, T *sLum,
                                             T *sLup, T *sLs, const T *sLam, const T *sBs, const T *sVs, T lres[6],
                                             T &gKa, T &gKp)
{
    using SM = FaceAdjSmem<T, TX, TY, KM>;
    constexpr int NT = TX * TY, SW3 = SM::SW3, SP3 = SM::SP3, LW = SM::LW, LP = SM::LP;
    constexpr int L = D == 0 ? TX : TY;   // cells of the tile along the normal
    constexpr int M = D == 0 ? TY : TX;   // lines of the tile
    constexpr int NSl = L + 4, NFl = L + 3, NLl = L + 2;
    constexpr int NS = M * NSl, NF = M * NFl, NL = M * NLl;
    constexpr int STEP = D == 0 ? 1 : SW3;  // smem stride along the normal
    const StageArgs<T> &a = q.f;
    const int tid = threadIdx.x;
    const int x0 = (q.bx0 + (int)blockIdx.x) * TX, y0 = (q.by0 + (int)blockIdx.y) * TY;
    const int o0 = D == 0 ? x0 : y0;
    const int n = D == 0 ? a.nx : a.ny, nt = D == 0 ? a.ny : a.nx;  // along, across
    const int pitch = a.pitch;
    const long long plane = a.plane;
    const T *geo = a.geo;
    const T hinv = D == 0 ? a.k.hinv_dx : a.k.hinv_dy;
    const T dtT = (T)a.dbg_dt;
    auto sidx = [&](int m, int p) {  // smem index of cell at line m, normal position p (tile coords)
        return D == 0 ? (m + 3) * SW3 + (p + 3) : (p + 3) * SW3 + (m + 3);
    };
    auto gidx = [&](int m, int p) {  // global (i, j) of line m, normal position p (tile coords)
        return D == 0 ? cell_index(x0 + p, y0 + m, pitch) : cell_index(x0 + m, y0 + p, pitch);
    };
    auto lidx = [&](int m, int p) {  // lam box index of line m, normal position p
        return D == 0 ? (m + 2) * LW + (p + 2) : (p + 2) * LW + (m + 2);
    };
    // Positions (m, p): each thread takes the one of its own cell, p in [0, L),
    // then a share of those outside the tile along the normal, p in
    // [-nlo, 0) and [L, L + nhi), over all lines (index arithmetic only there).
    const int m_own = D == 0 ? tid / TX : tid % TX, p_own = D == 0 ? tid % TX : tid / TX;
    const auto extra = [&](const int nlo, const int nhi, const auto &fn) {
        for (int e = tid; e < (nlo + nhi) * M; e += NT) {
            const int kk = e / M, m = e - kk * M;
            fn(m, kk < nlo ? kk - nlo : L + kk - nlo);
        }
    };
    // slopes and their selections, cells p = -2 .. L+1
    const auto slope = [&](const int m, const int p) {
        const int e = m * NSl + p + 2;
        const T *u = sU + sidx(m, p);
#pragma unroll
        for (int c = 0; c < 6; c++) {
            const T *uc = u + c * SP3;
            const T d1 = uc[0] - uc[-STEP], d2 = uc[STEP] - uc[0];
            sS[c * NS + e] = minmod(d1, d2);
            sSel[c * NS + e] = (unsigned char)minmod_sel(d1, d2);
        }
    };
    slope(m_own, p_own);
    extra(2, 2, slope);
    __syncthreads();
    // face adjoints, faces with lower cell p = -2 .. L
    const auto face = [&](const int m, const int p) {
        const int e = m * NFl + p + 2;
        const int lo = o0 + p;                       // lower cell index along the normal
        const int line = (D == 0 ? y0 : x0) + m;     // index across
        const bool exists = lo >= -1 && lo <= n - 1 && line < nt;
        T lum[6] = {T(0), T(0), T(0), T(0), T(0), T(0)}, lup[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        if (exists) {
            FaceGeo<T> G;
            T lH[6], d0, d1;
            if constexpr (SM::STAGE) {
                // cells outside the domain hold 0 in the lam box; the slope box
                // has the same layout (planes SX, SY, DBX, DBY)
                const int bl = lidx(m, p), bh = lidx(m, p + 1);
                if constexpr (D == 0)
                    G = face_geo32(sBs[2 * LP + bl], T(0.5) * (sBs[LP + bl] + sBs[LP + bh]), q.f.k);
                else
                    G = face_geo32(sBs[3 * LP + bl], T(0.5) * (sBs[bl] + sBs[bh]), q.f.k);
#pragma unroll
                for (int c = 0; c < 6; c++) lH[c] = dtT * hinv * (sLam[c * LP + bh] - sLam[c * LP + bl]);
                d0 = sLam[(6 + D) * LP + bl];
                d1 = sLam[(6 + D) * LP + bh];
            } else {
                const long long g = gidx(m, p);
                if (D == 0)
                    G = FaceGeo<T>{geo[GX_JHD * plane + g], geo[GX_SN * plane + g], geo[GX_ST * plane + g],
                                   geo[GX_FN * plane + g],  geo[GX_FT * plane + g], geo[GX_FN2 * plane + g],
                                   geo[GX_HG * plane + g]};
                else
                    G = FaceGeo<T>{geo[GY_JHD * plane + g], geo[GY_SN * plane + g], geo[GY_ST * plane + g],
                                   geo[GY_FN * plane + g],  geo[GY_FT * plane + g], geo[GY_FN2 * plane + g],
                                   geo[GY_HG * plane + g]};
                const bool in_lo = lo >= 0, in_hi = lo + 1 <= n - 1;
                const long long gl = g, gh = D == 0 ? g + 1 : g + pitch;
#pragma unroll
                for (int c = 0; c < 6; c++) {
                    const T a1 = in_hi ? q.lam_pre[c * plane + gh] : T(0);
                    const T a0 = in_lo ? q.lam_pre[c * plane + gl] : T(0);
                    lH[c] = dtT * hinv * (a1 - a0);
                }
                d0 = in_lo ? q.lam_dp[D * plane + gl] : T(0);
                d1 = in_hi ? q.lam_dp[D * plane + gh] : T(0);
            }
            const T lP2 = hinv * (d0 - d1);
            T um[6], up[6];
            const int sl = m * NSl + (p + 2);  // slope index of the lower cell
#pragma unroll
            for (int c = 0; c < 6; c++) {
                um[c] = fma(T(0.5), sS[c * NS + sl], sU[c * SP3 + sidx(m, p)]);
                up[c] = fma(T(-0.5), sS[c * NS + sl + 1], sU[c * SP3 + sidx(m, p + 1)]);
            }
            if constexpr (KM) {
                // each side with its cell's coefficient, as the forward stage;
                // the coefficient partials of the faces this tile owns (lower
                // cell in the tile, or the domain's first face)
                const bool pm = cell_passive(sVs + D * SP3, sidx(m, p), STEP);
                const bool pp = cell_passive(sVs + D * SP3, sidx(m, p + 1), STEP);
                const T Km = pm ? a.k.Kp : a.k.Ka, Kq = pp ? a.k.Kp : a.k.Ka;
                FaceGeo<T> Gm = G, Gp = G;
                Gm.sn *= Km;
                Gm.st *= Km;
                Gp.sn *= Kq;
                Gp.st *= Kq;
                T lKm, lKp;
                face_flux2_vjp<T, D, true>(um, up, Gm, Gp, lH, lP2, lum, lup, &G, &lKm, &lKp);
                if ((p >= 0 && p < L) || lo == -1) {
                    (pm ? gKp : gKa) += lKm;
                    (pp ? gKp : gKa) += lKp;
                }
            } else {
                face_flux2_vjp<T, D>(um, up, G, G, lH, lP2, lum, lup);
            }
        }
#pragma unroll
        for (int c = 0; c < 6; c++) {
            sLum[c * NF + e] = lum[c];
            sLup[c * NF + e] = lup[c];
        }
    };
    face(m_own, p_own);
    extra(2, 1, face);
    __syncthreads();
    // slope adjoints, cells p = -1 .. L: lam_sigma = (lam_um(face p) - lam_up(face p-1)) / 2
    const auto slope_adj = [&](const int m, const int p) {
        const int e = m * NLl + p + 1;
        const int f = m * NFl + (p + 2);  // face with lower cell p
#pragma unroll
        for (int c = 0; c < 6; c++) sLs[c * NL + e] = T(0.5) * (sLum[c * NF + f] - sLup[c * NF + f - 1]);
    };
    slope_adj(m_own, p_own);
    extra(1, 1, slope_adj);
    __syncthreads();
    // gather for cell p at line m
    // p in [-2, L+1]: faces p (lower cell p) and p-1 exist in the tile's range for
    // p in [-1, L]; slope adjoints exist for cells [-1, L]
    auto gather = [&](int m, int p, int c) -> T {
        const int f = m * NFl + (p + 2);
        T v = T(0);
        if (p <= L) v += sLum[c * NF + f];
        if (p >= -1) v += sLup[c * NF + f - 1];
        const int sl = m * NSl + (p + 2);
        const int lidx = m * NLl + (p + 1);
        if (p >= -1 && p <= L) {
            const unsigned char s0 = sSel[c * NS + sl];
            if (s0 == 1) v += sLs[c * NL + lidx];
            else if (s0 == 2) v -= sLs[c * NL + lidx];
        }
        if (p + 1 >= -1 && p + 1 <= L && sSel[c * NS + sl + 1] == 1) v -= sLs[c * NL + lidx + 1];
        if (p - 1 >= -1 && p - 1 <= L && sSel[c * NS + sl - 1] == 2) v += sLs[c * NL + lidx - 1];
        return v;
    };
    // interior cell of this thread
#pragma unroll
    for (int c = 0; c < 6; c++) lres[c] += gather(m_own, p_own, c);
    // ghost cells beyond the domain boundary along this direction
    for (int e = tid; e < 4 * M; e += NT) {
        const int m = e / 4, w = e - m * 4;
        const int line = (D == 0 ? y0 : x0) + m;
        if (line >= nt) continue;
        const int gpos = w < 2 ? -1 - w : n + (w - 2);  // -1, -2, n, n+1
        // owners: the first tile for -1, -2; the tile holding cell n-1 for n, n+1
        if (w < 2 ? o0 != 0 : !(o0 <= n - 1 && n - 1 < o0 + L)) continue;
        const int p = gpos - o0;
        const long long g = D == 0 ? cell_index(gpos, line, pitch) : cell_index(line, gpos, pitch);
#pragma unroll
        for (int c = 0; c < 6; c++) q.lam_in[c * plane + g] = gather(m, p, c);
    }
    __syncthreads();
}

// The ghost-cell adjoints a tile owns along direction D (as adj_face_dir
// writes them), set to 0: a tile without face terms
template <typename T, int TX, int TY, int D>
__device__ __forceinline__ void adj_ghost_zero(const AdjArgs<T> &q)
{
    constexpr int NT = TX * TY;
    constexpr int L = D == 0 ? TX : TY, M = D == 0 ? TY : TX;
    const StageArgs<T> &a = q.f;
    const int x0 = (q.bx0 + (int)blockIdx.x) * TX, y0 = (q.by0 + (int)blockIdx.y) * TY;
    const int o0 = D == 0 ? x0 : y0;
    const int n = D == 0 ? a.nx : a.ny, nt = D == 0 ? a.ny : a.nx;
    for (int e = threadIdx.x; e < 4 * M; e += NT) {
        const int m = e / 4, w = e - m * 4;
        const int line = (D == 0 ? y0 : x0) + m;
        if (line >= nt) continue;
        const int gpos = w < 2 ? -1 - w : n + (w - 2);
        if (w < 2 ? o0 != 0 : !(o0 <= n - 1 && n - 1 < o0 + L)) continue;
        const long long g = D == 0 ? cell_index(gpos, line, a.pitch) : cell_index(line, gpos, a.pitch);
#pragma unroll
        for (int c = 0; c < 6; c++) q.lam_in[c * a.plane + g] = T(0);
    }
}

// FP32: three 256-thread CTAs per SM (80 registers); FP64: shared memory allows two
// The fold of kernel C for the ghost cells this face tile owns (as
// adj_face_dir assigns them), by the tile itself once its cells hold their
// face terms: every source of these ghosts lies in the tile (AdjArgs::fold_inline).
template <typename T, int TX, int TY>
__device__ __forceinline__ void adj_fold_tile(const AdjArgs<T> &q)
{
    constexpr int NT = TX * TY;
    const StageArgs<T> &a = q.f;
    const int x0 = (q.bx0 + (int)blockIdx.x) * TX, y0 = (q.by0 + (int)blockIdx.y) * TY;
    const long long plane = a.plane;
#pragma unroll
    for (int D = 0; D < 2; D++) {
        const int L = D == 0 ? TX : TY, M = D == 0 ? TY : TX;
        const int o0 = D == 0 ? x0 : y0;
        const int n = D == 0 ? a.nx : a.ny, nt = D == 0 ? a.ny : a.nx;
        for (int e = threadIdx.x; e < 24 * M; e += NT) {
            const int c = e / (4 * M), r = e - c * 4 * M, m = r >> 2, w = r & 3;
            const int line = (D == 0 ? y0 : x0) + m;
            if (line >= nt || (w < 2 ? o0 != 0 : !(o0 <= n - 1 && n - 1 < o0 + L))) continue;
            const int side = 2 * D + (w < 2 ? 0 : 1);
            bool inflow = false;
            for (int f = 0; f < a.n_inflow; f++)
                inflow |= a.inflow[f].side == side && line >= a.inflow[f].i0 && line < a.inflow[f].i1;
            if (inflow) continue;  // the ghost state is a given function of time
            const bool closed = a.ph.bc[side] == 0;
            const bool flip = closed && (D == 0 ? (c == 1 || c == 4) : (c == 2 || c == 5));
            const int kk = w & 1;
            int gpos, src;
            if (w < 2) {
                gpos = -1 - kk;
                src = closed ? (kk < n ? kk : n - 1) : 0;
            } else {
                gpos = n + kk;
                src = closed ? (n - 1 - kk >= 0 ? n - 1 - kk : 0) : n - 1;
            }
            const long long gg = D == 0 ? cell_index(gpos, line, a.pitch) : cell_index(line, gpos, a.pitch);
            const long long gs = D == 0 ? cell_index(src, line, a.pitch) : cell_index(line, src, a.pitch);
            const T v = q.lam_in[c * plane + gg];
            if (v != T(0)) atomicAdd(&q.lam_in[c * plane + gs], flip ? -v : v);
        }
    }
}

template <typename T, int TX, int TY, bool KM = false>
__global__ void __launch_bounds__(TX *TY, (sizeof(T) == 4 ? 768 : 512) / (TX * TY)) adj_face_kernel(const AdjArgs<T> q)
{
    using SM = FaceAdjSmem<T, TX, TY, KM>;
    constexpr int NT = TX * TY, SW3 = SM::SW3, SP3 = SM::SP3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    wait_prior_grid();  // launched after the kernel before it (launch_after)
    T *sU = reinterpret_cast<T *>(smem_raw);
    T *sS = sU + 6 * SP3;
    T *sLum = sS + 6 * SM::NS;
    T *sLup = sLum + 6 * SM::NF;
    T *sLs = sLup + 6 * SM::NF;
    unsigned char *sSel = reinterpret_cast<unsigned char *>(sLs + 6 * SM::NL);
    T *sLam = reinterpret_cast<T *>(smem_raw + SM::base);  // FP32 form: [8][TY+4][TX+4]
    T *sBs = sLam + 8 * SM::LP;                             // FP32 form: [4][TY+4][TX+4] bed slopes
    T *sVs = reinterpret_cast<T *>(smem_raw + SM::staged);  // KM: [2][TY+6][TX+6] solid velocities
    __shared__ double kred[2][NT / 32];
    const StageArgs<T> &a = q.f;
    const int tid = threadIdx.x;
    const int x0 = (q.bx0 + (int)blockIdx.x) * TX, y0 = (q.by0 + (int)blockIdx.y) * TY;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    const long long plane = a.plane;
    if (q.tw && adj_far_from_mass(q, q.bx0 + (int)blockIdx.x, q.by0 + (int)blockIdx.y)) {  // CTA-uniform: no face terms (AdjArgs::tw)
        adj_ghost_zero<T, TX, TY, 0>(q);
        adj_ghost_zero<T, TX, TY, 1>(q);
        return;
    }
    // The stage input's masses with a 3-cell halo come first (cells beyond
    // the 2 ghost layers read 0; no forward face uses them).  Where none of
    // them holds mass, every face state of the tile is dry: the side fluxes'
    // derivatives vanish (velocities, pressures and speeds are 0 and the
    // speed's square root is differentiated as 0 at 0), so the tile has no
    // face terms and skips them; its cells keep their own contributions.
    const auto copy_u = [&](const int tx, const int ty, const bool masses) {
        const int gi = x0 + tx, gj = y0 + ty;
        const bool ok = gi >= -2 && gj >= -2 && gi < nx + 2 && gj < ny + 2;
        const T *src = a.Uin + (ok ? cell_index(gi, gj, pitch) : 0);
        T *dst = sU + (ty + 3) * SW3 + tx + 3;
#pragma unroll
        for (int q4 = 0; q4 < 4; q4++) {
            const int c = masses ? (q4 == 0 ? 0 : 3) : (q4 < 2 ? q4 + 1 : q4 + 2);
            if (!masses || q4 < 2) cp_async_elem(dst + c * SP3, src + (ok ? c * plane : 0), ok);
        }
    };
    copy_u(tid % TX, tid / TX, true);
    for (int h = tid; h < SP3 - NT; h += NT) {
        int tx, ty;
        halo_cell<TX, TY, 3>(h, tx, ty);
        copy_u(tx, ty, true);
    }
    cp_async_wait_all();
    bool has_mass;
    {
        const auto massy = [&](const int tx, const int ty) {
            const int o = (ty + 3) * SW3 + tx + 3;
            return nonzero(sU[o]) | nonzero(sU[3 * SP3 + o]);
        };
        has_mass = massy(tid % TX, tid / TX);
        for (int h = tid; h < SP3 - NT; h += NT) {
            int tx, ty;
            halo_cell<TX, TY, 3>(h, tx, ty);
            has_mass |= massy(tx, ty);
        }
    }
    const bool wet = __syncthreads_or(has_mass) != 0;
    T lres[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    T gKa = T(0), gKp = T(0);
    if (wet) {  // CTA-uniform
        // the momenta; FP32 also the cell adjoints and bed slopes of the box
        if constexpr (SM::STAGE) {
            // lam_pre (6) and lam_dp (2) of the tile and a 2-cell halo; 0 outside the domain
            const auto copy_lam = [&](const int tx, const int ty) {
                const int gi = x0 + tx, gj = y0 + ty;
                const bool ok = gi >= 0 && gj >= 0 && gi < nx && gj < ny;
                const long long g = ok ? cell_index(gi, gj, pitch) : 0;
                T *dst = sLam + (ty + 2) * SM::LW + tx + 2;
#pragma unroll
                for (int c = 0; c < 8; c++)
                    cp_async_elem(dst + c * SM::LP, c < 6 ? q.lam_pre + c * plane + g : q.lam_dp + (c - 6) * plane + g, ok);
            };
            copy_lam(tid % TX, tid / TX);
            for (int h = tid; h < SM::LP - NT; h += NT) {
                int tx, ty;
                halo_cell<TX, TY, 2>(h, tx, ty);
                copy_lam(tx, ty);
            }
            // bed slopes of the same box (computed for cells -2 .. n+1)
            const auto copy_slopes = [&](const int tx, const int ty) {
                const int gi = x0 + tx, gj = y0 + ty;
                const bool ok = gi >= -2 && gj >= -2 && gi <= nx + 1 && gj <= ny + 1;
                const T *src = a.geo + (ok ? GS_SX * plane + cell_index(gi, gj, pitch) : 0);
                T *dst = sBs + (ty + 2) * SM::LW + tx + 2;
#pragma unroll
                for (int c = 0; c < 4; c++) cp_async_elem(dst + c * SM::LP, src + (ok ? c * plane : 0), ok);
            };
            copy_slopes(tid % TX, tid / TX);
            for (int h = tid; h < SM::LP - NT; h += NT) {
                int tx, ty;
                halo_cell<TX, TY, 2>(h, tx, ty);
                copy_slopes(tx, ty);
            }
        }
        copy_u(tid % TX, tid / TX, false);
        for (int h = tid; h < SP3 - NT; h += NT) {
            int tx, ty;
            halo_cell<TX, TY, 3>(h, tx, ty);
            copy_u(tx, ty, false);
        }
        cp_async_wait_all();
        __syncthreads();
        if constexpr (KM) {
            // solid velocity of every cell of the state box, as the forward stage takes it
            for (int e = tid; e < SP3; e += NT) {
                const int gi = x0 + e % SW3 - 3, gj = y0 + e / SW3 - 3;
                T vx = T(NAN), vy = T(NAN);
                if (gi >= -2 && gj >= -2 && gi < nx + 2 && gj < ny + 2) {
                    const T u1 = sU[e];
                    if (gtp(u1, a.geo[GC_JHD * plane + cell_index(gi, gj, pitch)])) {
                        if constexpr (sizeof(T) == 8) {
                            vx = __ddiv_rn(sU[SP3 + e], u1);
                            vy = __ddiv_rn(sU[2 * SP3 + e], u1);
                        } else {
                            vx = __fdiv_rn(sU[SP3 + e], u1);
                            vy = __fdiv_rn(sU[2 * SP3 + e], u1);
                        }
                    }
                }
                sVs[e] = vx;
                sVs[SP3 + e] = vy;
            }
            __syncthreads();
        }
        adj_face_dir<T, TX, TY, 0, KM>(q, sU, sS, sSel, sLum, sLup, sLs, sLam, sBs, sVs, lres, gKa, gKp);
        adj_face_dir<T, TX, TY, 1, KM>(q, sU, sS, sSel, sLum, sLup, sLs, sLam, sBs, sVs, lres, gKa, gKp);
    } else {
        // the ghost cells this tile owns get no face terms either
        adj_ghost_zero<T, TX, TY, 0>(q);
        adj_ghost_zero<T, TX, TY, 1>(q);
    }
    // the face terms of the tile's cells (a dry tile has none)
    const int i = x0 + tid % TX, j = y0 + tid / TX;
    if (wet && i < nx && j < ny) {
        const long long g = cell_index(i, j, pitch);
#pragma unroll
        for (int c = 0; c < 6; c++) q.lam_in[c * plane + g] += lres[c];
    }
    if constexpr (KM) {  // coefficient partials: per warp in T, per CTA and globally in FP64
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            gKa += __shfl_xor_sync(0xffffffffu, gKa, o);
            gKp += __shfl_xor_sync(0xffffffffu, gKp, o);
        }
        if ((tid & 31) == 0) {
            kred[0][tid >> 5] = (double)gKa;
            kred[1][tid >> 5] = (double)gKp;
        }
        __syncthreads();
        if (tid == 0) {
            double s0 = 0.0, s1 = 0.0;
            for (int w = 0; w < NT / 32; w++) {
                s0 += kred[0][w];
                s1 += kred[1][w];
            }
            if (s0 != 0.0) atomicAdd(&q.g_param[2], s0);
            if (s1 != 0.0) atomicAdd(&q.g_param[3], s1);
        }
    }
    if (q.fold_inline && wet) {  // CTA-uniform; a dry tile's ghosts hold 0
        __syncthreads();  // the tile's cells hold their face terms
        adj_fold_tile<T, TX, TY>(q);
    }
}

// ---- kernel C: fold the ghost adjoints into their sources ----------------------
// one thread per (component, side, line along the side)
template <typename T>
__global__ void adj_fold_kernel(const AdjArgs<T> q)
{
    wait_prior_grid();  // launched after the kernel before it (launch_after)
    const StageArgs<T> &a = q.f;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    const long long plane = a.plane;
    const int per_c = 2 * ny + 2 * nx;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 6 * per_c) return;
    const int c = e / per_c;
    int r = e - c * per_c;
    int side, line;
    if (r < 2 * ny) {
        side = r / ny;  // W, E
        line = r - side * ny;
    } else {
        r -= 2 * ny;
        side = 2 + r / nx;  // S, N
        line = r - (side - 2) * nx;
    }
    const bool xs = side < 2;
    for (int f = 0; f < a.n_inflow; f++)
        if (a.inflow[f].side == side && line >= a.inflow[f].i0 && line < a.inflow[f].i1)
            return;  // ghost state is a given function of time
    const bool closed = a.ph.bc[side] == 0;
    const bool flip = closed && (xs ? (c == 1 || c == 4) : (c == 2 || c == 5));
    const int nn = xs ? nx : ny;
    for (int kk = 0; kk < GH; kk++) {
        int gpos, src;
        if (side == 0 || side == 2) {
            gpos = -1 - kk;
            src = closed ? (kk < nn ? kk : nn - 1) : 0;
        } else {
            gpos = nn + kk;
            src = closed ? (nn - 1 - kk >= 0 ? nn - 1 - kk : 0) : nn - 1;
        }
        const long long gg = xs ? cell_index(gpos, line, pitch) : cell_index(line, gpos, pitch);
        const long long gs = xs ? cell_index(src, line, pitch) : cell_index(line, src, pitch);
        const T v = q.lam_in[c * plane + gg];
        if (v != T(0)) atomicAdd(&q.lam_in[c * plane + gs], flip ? -v : v);
    }
}

}  // namespace moses
