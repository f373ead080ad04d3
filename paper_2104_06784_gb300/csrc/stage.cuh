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
// Work decomposition: the stage of one TX x TY tile (stage_tile).  The CTA
// stages the six state planes of the tile plus a 2-cell halo in shared
// memory (cp.async), computes each cell's minmod slopes once, every x- and
// y-face flux once, then updates its cells.  In a combining stage it also
// forms the Heun average (or the Runge-Kutta combination) in place, writes
// the ghost cells of the new state (boundary conditions fused into the
// producer) and reduces the CFL wave speed: warp shuffle max, CTA max, one
// atomicMax on the IEEE bits of a non-negative double (exact, independent of
// order).  The last CTA to finish (ticket counter, no waiting) turns the
// maximum into the next time step.
//
// Wet/dry masking: a tile with no mass within the stencil's reach has the
// zero state as its stage result.  The stepping launches classify every tile
// first (classify_kernel: TMA bulk copies of the mass rows of 32 x 16-cell
// strips, warp votes; a combining stage uses the first stage's per-tile
// flags), write the dry tiles' zero state there (skipping the tiles whose
// output buffer holds it already, per-tile known-zero flags), and run
// stage_tile only on the list of wet tiles (stage_kernel_list, resident
// CTAs); the other launches test each tile inside stage_tile.
//
// GB300 executes two FP64 FMAs per clock per SM, so the FP64 form is bound by
// the FP64 pipe.  Everything that can leave it does: the minmod limiter, the
// dry and zero tests, the stopping decision and every max are integer
// operations on the IEEE bit patterns (exact for the operands they see);
// reciprocals and square roots start from the hardware approximations
// (rcp/rsqrt.approx.ftz.f64) and take one third-order refinement step each
// (frcp, fsqrt, frsqrt below), which lands within an ulp of the correctly
// rounded result; fluxes are kept doubled so the factor 1/2 folds into 1/dx;
// products of parameters and geometry are precomputed per cell and face.
#pragma once
#include <cuda_runtime.h>

#include <utility>

#include "moses_dev.cuh"

namespace moses {

// ---- bit-pattern helpers ----------------------------------------------------
__device__ __forceinline__ long long ibits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ int ibits(float x) { return __float_as_int(x); }

// a > b for b > 0: signed comparison of the bit patterns (negative a, with
// the sign bit set, compare below every positive b)
template <typename T>
__device__ __forceinline__ bool gtp(T a, T b)
{
    return ibits(a) > ibits(b);
}
// max of two non-negative values
template <typename T>
__device__ __forceinline__ T maxnn(T a, T b)
{
    return ibits(a) >= ibits(b) ? a : b;
}
// max(x, 0)
template <typename T>
__device__ __forceinline__ T pos(T x)
{
    return ibits(x) < 0 ? T(0) : x;
}
// x < 0 (and not -0)
__device__ __forceinline__ bool negative(double x) { return ibits(x) < 0 && (ibits(x) << 1) != 0; }
__device__ __forceinline__ bool negative(float x) { return ibits(x) < 0 && (ibits(x) << 1) != 0; }

__device__ __forceinline__ bool nonfinite(double x) { return (__double2hiint(x) & 0x7ff00000) == 0x7ff00000; }
__device__ __forceinline__ bool nonfinite(float x) { return (__float_as_int(x) & 0x7f800000) == 0x7f800000; }

// minmod of two one-sided undivided differences (Sect. 2.2): 0 if the signs
// differ or either is 0, else the one of smaller magnitude
__device__ __forceinline__ double minmod(double a, double b)
{
    const long long ia = ibits(a), ib = ibits(b);
    const long long ma = ia & 0x7fffffffffffffffll, mb = ib & 0x7fffffffffffffffll;
    if ((ia ^ ib) < 0 || ma == 0 || mb == 0) return 0.0;
    return ma < mb ? a : b;
}
// FP32: the sign test as a product (a b > 0: same sign, both nonzero; a
// product that underflows counts as 0), the rest on magnitudes
__device__ __forceinline__ float minmod(float a, float b)
{
    const float m = fabsf(a) < fabsf(b) ? a : b;
    return a * b > 0.0f ? m : 0.0f;
}

// ---- reciprocal and square root ---------------------------------------------
// 1/x for x > 0 normal: hardware approximation y (relative error e ~ 1e-6)
// refined by one third-order step y (1 + e + e^2), e = 1 - x y, whose error
// is O(e^3): within an ulp, as two Newton steps give, in three FMAs instead
// of four (measured max relative error 1.1e-16 over x in [1e-6, 1e6])
__device__ __forceinline__ double frcp(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}
__device__ __forceinline__ float frcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// sqrt(x), 0 for x <= 0 or subnormal: from the approximate reciprocal square
// root y (relative error ~1e-6), t = x y and d = 1 - t y, the third-order
// step sqrt(x) = t (1 - d)^(-1/2) ~ t (1 + d/2 + 3 d^2/8), error O(d^3)
// (measured max 0.75 ulp over x in [1e-12, 1e12])
__device__ __forceinline__ double fsqrt(double x)
{
    if (ibits(x) < 0x0010000000000000ll) return 0.0;
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double t = x * y;
    const double d = fma(-t, y, 1.0);
    return fma(t, d * fma(0.375, d, 0.5), t);
}
__device__ __forceinline__ float fsqrt(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// 1/sqrt(x) for x > 0: approximation, refined in FP64.  The approximation
// flushes subnormal inputs to zero, so those are scaled by 2^512 (2^64 in FP32)
// first and the result by 2^256 (2^32) after.
__device__ __forceinline__ double frsqrt(double x)
{
    // third-order step y (1 + d/2 + 3 d^2/8), d = 1 - x y^2 (measured max
    // 0.98 ulp over x in [1e-12, 1e12])
    const bool sub = ibits(x) < 0x0010000000000000ll;
    const double xs = sub ? x * 0x1p512 : x;
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(xs));
    const double d = fma(-xs * y, y, 1.0);
    y = fma(y, d * fma(0.375, d, 0.5), y);
    return sub ? y * 0x1p256 : y;
}
__device__ __forceinline__ float frsqrt(float x)
{
    const bool sub = ibits(x) < 0x00800000;
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(sub ? x * 0x1p64f : x));
    return sub ? y * 0x1p32f : y;
}
// Asynchronous global -> shared copy of one element (cp.async, no register
// round trip, many in flight per thread); !valid writes 0 and reads nothing.
// The copies of a thread complete at cp_async_wait_all().
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const unsigned n = valid ? (unsigned)sizeof(T) : 0u;
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(sizeof(T)), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Third-order WENO value at the right face of cell b from the cells a, b, c
// (Sect. 2.2 names WENO reconstruction as an option): candidates on {a, b}
// and {b, c}, linear weights 1/3 and 2/3, smoothness indicators the squared
// differences, nonlinear weights d_k / (eps + beta_k)^2 with the
// scale-invariant eps = 1e-6 m^2 + tiny (m = max |a|, |b|, |c|), written as
// one reciprocal: w0 = d0 (eps + beta1)^2 / (d0 (eps + beta1)^2 + d1 (eps + beta0)^2).
// The left-face value of b is the same function of (c, b, a).
// FP32 takes the differences in units of m (a second reciprocal), so that the
// squared indicators cannot underflow; the weights are unchanged by the
// rescaling up to rounding.  Below m = 1e-30 (where a subnormal m would defeat
// the reciprocal) the differences count as 0, which gives the linear weights.
template <typename T>
__device__ __forceinline__ T weno3_face(T a, T b, T c)
{
    const T q0 = fma(T(1.5), b, T(-0.5) * a), q1 = T(0.5) * (b + c);
    T d0 = b - a, d1 = c - b;
    const T m = fmax(fabs(a), fmax(fabs(b), fabs(c)));
    T eps;
    if constexpr (sizeof(T) == 8) {
        eps = fma(1e-6 * m, m, 1e-100);
    } else {
        const float rm = m > 1e-30f ? frcp(m) : 0.0f;
        d0 *= rm;
        d1 *= rm;
        eps = 1e-6f;
    }
    const T e0 = fma(d0, d0, eps), e1 = fma(d1, d1, eps);
    const T n0 = T(1.0 / 3.0) * (e1 * e1), n1 = T(2.0 / 3.0) * (e0 * e0);
    return fma(n0 * frcp(n0 + n1), q0 - q1, q1);
}

// error-free sum (Knuth's TwoSum): s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ double tabs(double x) { return fabs(x); }
__device__ __forceinline__ float tabs(float x) { return fabsf(x); }

// x != 0 (NaN included) on the integer unit: GB300's FP64 pipe is the scarce
// one, and the wet/dry tests read every cell
__device__ __forceinline__ bool nonzero(double x)
{
    return (static_cast<unsigned long long>(__double_as_longlong(x)) << 1) != 0ull;
}
__device__ __forceinline__ bool nonzero(float x) { return (static_cast<unsigned int>(__float_as_int(x)) << 1) != 0u; }

// ---- face flux -----------------------------------------------------------------
template <typename T>
struct FaceGeo {
    T jhd;  // J h_dry
    T sn;   // kap_s A_dd c^2 : solid pressure coefficient of the normal momentum, solid speed
    T st;   // kap_s A_dt c^2 : solid pressure coefficient of the transverse momentum
    T fn, ft, fn2;  // kap_f A_dd c^2, kap_f A_dt c^2, 2 kap_f A_dd c^2
    T hg;   // (g/2) c^2
};

// Physical flux of one reconstructed state through a face of direction d
// (0: xi = X, 1: eta = Y), the per-phase local speeds (R7) and P = J h pbar^f.
// With xi = X, eta = Y the tangential velocity v_xi equals v_X, the mass flux
// J h^p v_xi^p is the momentum component U_{2+d}, and the pressure terms
// eps J h A_dk Nbar^s, eps J h A_dk pbar^f become (kap A_dk c^2) (J h) U.
template <typename T, int D>
__device__ __forceinline__ void side_flux(const T u[6], const FaceGeo<T> &G, T F[6], T &as, T &af, T &P,
                                          T *w = nullptr)
{
    const T Ut = u[0] + u[3];
    const bool ws = gtp(u[0], G.jhd), wf = gtp(u[3], G.jhd);
    const T rs = ws ? frcp(u[0]) : T(0);
    const T rf = wf ? frcp(u[3]) : T(0);
    const T uns = D == 0 ? u[1] : u[2];
    const T unf = D == 0 ? u[4] : u[5];
    const T vns = uns * rs, vnf = unf * rf;
    const T Ps = Ut * u[0], Pf = Ut * Ut;
    // X-momentum uses the normal coefficient on x-faces, the transverse one
    // on y-faces; Y-momentum the other way round
    const T sX = D == 0 ? G.sn : G.st, sY = D == 0 ? G.st : G.sn;
    const T fX = D == 0 ? G.fn : G.ft, fY = D == 0 ? G.ft : G.fn;
    F[0] = ws ? uns : T(0);
    F[1] = fma(sX, Ps, u[1] * vns);
    F[2] = fma(sY, Ps, u[2] * vns);
    F[3] = wf ? unf : T(0);
    F[4] = fma(fX, Pf, u[4] * vnf);
    F[5] = fma(fY, Pf, u[5] * vnf);
    const T cs = fsqrt(G.sn * (Ut + u[0])), cf = fsqrt(G.fn2 * Ut);
    as = tabs(vns) + cs;
    af = tabs(vnf) + cf;
    P = G.hg * Pf;
    if (w) {  // normal velocities and wave-speed terms, for one-sided speeds
        w[0] = vns;
        w[1] = cs;
        w[2] = vnf;
        w[3] = cf;
    }
}

// What the central flux needs of one reconstructed side (as side_flux): the
// mass fluxes (0 where the phase is dry), the normal velocities, the pressure
// products Ut U1 and Ut^2 and the per-phase local speeds (R7).
template <typename T>
struct SideTerms {
    T m0, m3, vs, vf, Ps, Pf, as, af;
};
template <typename T, int D>
__device__ __forceinline__ SideTerms<T> side_terms(const T u[6], const FaceGeo<T> &G)
{
    SideTerms<T> r;
    const T Ut = u[0] + u[3];
    const bool ws = gtp(u[0], G.jhd), wf = gtp(u[3], G.jhd);
    const T rs = ws ? frcp(u[0]) : T(0);
    const T rf = wf ? frcp(u[3]) : T(0);
    const T uns = D == 0 ? u[1] : u[2];
    const T unf = D == 0 ? u[4] : u[5];
    r.vs = uns * rs;
    r.vf = unf * rf;
    r.m0 = ws ? uns : T(0);
    r.m3 = wf ? unf : T(0);
    r.Ps = Ut * u[0];
    r.Pf = Ut * Ut;
    r.as = tabs(r.vs) + fsqrt(G.sn * (Ut + u[0]));
    r.af = tabs(r.vf) + fsqrt(G.fn2 * Ut);
    return r;
}

// Twice the central flux through one face, from the face values um (left /
// lower cell) and up (right / upper cell): H2 = F(um) + F(up) - a (up - um),
// a = max of the two sides' local speeds per phase; H2[6] = P(um) + P(up).
// With F = (U v_n + s P) for a momentum component (s its pressure
// coefficient, P the side's pressure product) the momentum rows are taken as
// um (v_n(um) + a) + up (v_n(up) - a) + (s P(um) + s P(up)), the same sum with
// fewer FP64 operations (the factors v_n +- a and P(um) + P(up) shared by the
// components of a phase).
// Gm, Gp: the face geometry as each side sees it (they differ only in the
// solid pressure coefficients, scaled by each side's earth-pressure
// coefficient with k_mode 1: SAME false; the same otherwise).
template <typename T, int D, bool SAME = true>
__device__ __forceinline__ void face_flux2(const T um[6], const T up[6], const FaceGeo<T> &Gm, const FaceGeo<T> &Gp,
                                           T H[7])
{
    const SideTerms<T> m = side_terms<T, D>(um, Gm), p = side_terms<T, D>(up, Gp);
    const T as = maxnn(m.as, p.as), af = maxnn(m.af, p.af);
    H[0] = fma(-as, up[0] - um[0], m.m0 + p.m0);
    H[3] = fma(-af, up[3] - um[3], m.m3 + p.m3);
    const T As = m.vs + as, Bs = p.vs - as, Af = m.vf + af, Bf = p.vf - af;
    // X-momentum uses the normal coefficient on x-faces, the transverse one
    // on y-faces; Y-momentum the other way round
    const T sXm = D == 0 ? Gm.sn : Gm.st, sYm = D == 0 ? Gm.st : Gm.sn;
    if constexpr (SAME) {
        const T Ss = m.Ps + p.Ps;
        H[1] = fma(um[1], As, fma(up[1], Bs, sXm * Ss));
        H[2] = fma(um[2], As, fma(up[2], Bs, sYm * Ss));
    } else {
        const T sXp = D == 0 ? Gp.sn : Gp.st, sYp = D == 0 ? Gp.st : Gp.sn;
        H[1] = fma(um[1], As, fma(up[1], Bs, fma(sXm, m.Ps, sXp * p.Ps)));
        H[2] = fma(um[2], As, fma(up[2], Bs, fma(sYm, m.Ps, sYp * p.Ps)));
    }
    const T fX = D == 0 ? Gm.fn : Gm.ft, fY = D == 0 ? Gm.ft : Gm.fn;
    const T Sf = m.Pf + p.Pf;
    H[4] = fma(um[4], Af, fma(up[4], Bf, fX * Sf));
    H[5] = fma(um[5], Af, fma(up[5], Bf, fY * Sf));
    H[6] = Gm.hg * Sf;  // hg is the face's (the earth-pressure scaling leaves it)
}

// Twice the central-upwind flux (the second-order scheme Sect. 2.2 cites): per
// phase one-sided speeds ap = max(vn + c, 0) and am = min(vn - c, 0) over the
// two sides, H = (ap F(um) - am F(up)) / (ap - am) + ap am / (ap - am) (up - um);
// the mean of the two fluxes where ap = am = 0.  H2[6] = P(um) + P(up).
template <typename T, int D>
__device__ __forceinline__ void face_flux2_cu(const T um[6], const T up[6], const FaceGeo<T> &G, T H[7])
{
    T Fm[6], Fp[6], wm[4], wp[4], a, Pm, Pp;
    side_flux<T, D>(um, G, Fm, a, a, Pm, wm);
    side_flux<T, D>(up, G, Fp, a, a, Pp, wp);
#pragma unroll
    for (int ph = 0; ph < 2; ph++) {
        const T ap = fmax(fmax(wm[2 * ph] + wm[2 * ph + 1], wp[2 * ph] + wp[2 * ph + 1]), T(0));
        const T am = fmin(fmin(wm[2 * ph] - wm[2 * ph + 1], wp[2 * ph] - wp[2 * ph + 1]), T(0));
        const T w = ap - am;
        const bool moving = w > T(0);
        const T r2 = moving ? T(2) * frcp(w) : T(0);  // doubled flux
#pragma unroll
        for (int c = 3 * ph; c < 3 * ph + 3; c++)
            H[c] = moving ? fma(ap * am * r2, up[c] - um[c], (ap * Fm[c] - am * Fp[c]) * r2) : Fm[c] + Fp[c];
    }
    H[6] = Pm + Pp;
}

// Earth-pressure regime (k_mode 1, reading R10) of the cell at offset o of a
// velocity box (v: the velocity component along the axis, NaN where the
// cell carries no solid; st: the box's offset step along the axis): passive
// where the cell carries solid and its velocity drops along the axis by more
// than the dead band 1e-6 (|v+| + |v-|) + 1e-6 m/s (unfused IEEE operations,
// as the oracle takes them); the stage kernel and its adjoint both use it
template <typename T>
__device__ __forceinline__ bool cell_passive(const T *v, const int o, const int st)
{
    const T vc = v[o], vp = v[o + st], vm = v[o - st];
    T d, band;
    if constexpr (sizeof(T) == 8) {
        d = __dsub_rn(vp, vm);
        band = __dadd_rn(__dmul_rn(1e-6, __dadd_rn(fabs(vp), fabs(vm))), 1e-6);
    } else {
        d = __fsub_rn(vp, vm);
        band = __fadd_rn(__fmul_rn(1e-6f, __fadd_rn(fabsf(vp), fabsf(vm))), 1e-6f);
    }
    return vc == vc && d < -band;
}

// ---- Mode-II inflow and ghost cells ---------------------------------------------
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
    // corners: the S/N rule applied to the W/E mirror or copy ghosts (inflow
    // segments do not reach them); read only by the viscous stencil
    if ((i < 2 || i >= nx - 2) && (j < 2 || j >= ny - 2)) {
#pragma unroll
        for (int sx = 0; sx < 2; sx++) {
            const bool cx = ph.bc[sx] == 0;
            for (int kx = 0; kx < GH; kx++) {
                const int gi = sx == 0 ? -1 - kx : nx + kx;
                int srcx;
                if (sx == 0) srcx = cx ? (kx < nx ? kx : nx - 1) : 0;
                else srcx = cx ? (nx - 1 - kx >= 0 ? nx - 1 - kx : 0) : nx - 1;
                if (srcx != i) continue;
#pragma unroll
                for (int sy = 2; sy < 4; sy++) {
                    const bool cy = ph.bc[sy] == 0;
                    for (int ky = 0; ky < GH; ky++) {
                        const int gj = sy == 2 ? -1 - ky : ny + ky;
                        int srcy;
                        if (sy == 2) srcy = cy ? (ky < ny ? ky : ny - 1) : 0;
                        else srcy = cy ? (ny - 1 - ky >= 0 ? ny - 1 - ky : 0) : ny - 1;
                        if (srcy != j) continue;
                        T u[6] = {v[0], v[1], v[2], v[3], v[4], v[5]};
                        if (cx) {
                            u[1] = -u[1];
                            u[4] = -u[4];
                        }
                        if (cy) {
                            u[2] = -u[2];
                            u[5] = -u[5];
                        }
                        store6(U, plane, cell_index(gi, gj, pitch), u);
                    }
                }
            }
        }
    }
}

// Largest cell-centre wave speed of a state (R7), both phases, both axes,
// from the cell's J h_dry and its four speed coefficients.
template <typename T>
__device__ __forceinline__ T cell_speed(const T u[6], T jhd, T sxs, T sxf, T sys, T syf)
{
    const T Ut = u[0] + u[3];
    const T rs = gtp(u[0], jhd) ? frcp(u[0]) : T(0);
    const T rf = gtp(u[3], jhd) ? frcp(u[3]) : T(0);
    const T cs = Ut + u[0];
    T m = tabs(u[1] * rs) + fsqrt(sxs * cs);
    m = maxnn(m, tabs(u[4] * rf) + fsqrt(sxf * Ut));
    m = maxnn(m, tabs(u[2] * rs) + fsqrt(sys * cs));
    m = maxnn(m, tabs(u[5] * rf) + fsqrt(syf * Ut));
    return m;
}
// the same with the coefficients read from the geometry planes of cell g
template <typename T>
__device__ __forceinline__ T cell_speed(const T u[6], const T *geo, long long plane, long long g)
{
    return cell_speed(u, geo[GC_JHD * plane + g], geo[GC_SXS * plane + g], geo[GC_SXF * plane + g],
                      geo[GC_SYS * plane + g], geo[GC_SYF * plane + g]);
}

// ---- FP32 form: geometry rebuilt from bed slopes in the tile -------------------
// The formulas of the geometry pass (Sect. 2.1): Omega_b = [(1,0,bX),
// (0,1,bY), n], J = sqrt(1 + bX^2 + bY^2), c = 1/J, A = the 2x2 block of the
// inverse metric; curvature terms c bXX, 2 c bXY, c bYY.
struct CellGeo32 {
    float jhd, gc1, gcf, bX, bY, nX, nY, A11, A12, A22, kXX, kXY2, kYY, sxs, sxf, sys, syf;
};
__device__ __forceinline__ CellGeo32 cell_geo32(float sX, float sY, float bXX, float bXY, float bYY, const KT<float> &k)
{
    CellGeo32 G;
    const float s2 = fmaf(sX, sX, fmaf(sY, sY, 1.0f));
    const float c = frsqrt(s2), c2 = c * c;
    G.jhd = s2 * c * k.h_dry;
    G.gc1 = k.g_1ma * c;
    G.gcf = k.g * c;
    G.bX = sX;
    G.bY = sY;
    G.nX = -c * sX;
    G.nY = -c * sY;
    G.A11 = fmaf(sY, sY, 1.0f) * c2;
    G.A12 = -sX * sY * c2;
    G.A22 = fmaf(sX, sX, 1.0f) * c2;
    G.kXX = c * bXX;
    G.kXY2 = 2.0f * c * bXY;
    G.kYY = c * bYY;
    G.sxs = k.kap_s_cfl * G.A11 * c2;
    G.sxf = k.kap_f2 * G.A11 * c2;
    G.sys = k.kap_s_cfl * G.A22 * c2;
    G.syf = k.kap_f2 * G.A22 * c2;
    return G;
}
// face of normal slope bn (the face difference) and transverse slope bt (mean
// of the two cells' central differences)
__device__ __forceinline__ FaceGeo<float> face_geo32(float bn, float bt, const KT<float> &k)
{
    const float s2 = fmaf(bn, bn, fmaf(bt, bt, 1.0f));
    const float c2 = frcp(s2), cc = c2 * c2;
    const float An = fmaf(bt, bt, 1.0f) * cc, At = -bn * bt * cc;
    return FaceGeo<float>{fsqrt(s2) * k.h_dry, k.kap_s * An, k.kap_s * At, k.kap_f * An, k.kap_f * At,
                          k.kap_f2 * An, k.half_g * c2};
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

// Semi-implicit Coulomb friction with stopping (R6): q* = (q1, q2) after all
// other terms, F = dt J p_b^s tan(delta_b); the tangential 3D momentum is
// |q*|_3 = |(q1, q2, bX q1 + bY q2)|; stop if |q*|_3 <= F, else scale by
// 1 - F / |q*|_3.  The decision is taken in FP64 in both forms; the FP32 form
// first decides in FP32 when the two sides differ by more than 2^-10
// relative (far above its rounding), which gives the same outcome.
__device__ __forceinline__ void coulomb(double &q1, double &q2, double bX, double bY, double Fr)
{
    const double qZ = fma(bX, q1, bY * q2);
    const double qn2 = fma(q1, q1, fma(q2, q2, qZ * qZ));
    if (!gtp(qn2, Fr * Fr)) {  // includes qn2 == 0
        q1 = 0.0;
        q2 = 0.0;
        return;
    }
    if (ibits(Fr) <= 0) return;  // no friction (lift-off or dry): r = 1, also for subnormal |q*|
    const double r = fma(-Fr, frsqrt(qn2), 1.0);
    q1 *= r;
    q2 *= r;
}
// FP64 stopping decision of the FP32 form when FP32 cannot tell the two sides
// apart; kept out of line so that the common path carries no FP64 work
static __device__ __noinline__ bool stop_fp64(float q1, float q2, float bX, float bY, double dt, float Jpbs, double tan_d)
{
    const double Frd = dt * (double)Jpbs * tan_d;
    const double dq1 = q1, dq2 = q2, dZ = (double)bX * dq1 + (double)bY * dq2;
    return !(dq1 * dq1 + dq2 * dq2 + dZ * dZ > Frd * Frd);
}

// The FP32 form's stopping decision.  |q*|^2 that underflowed to 0 stops the
// cell: only a cell with a vanishing basal pressure (a dry one) can get there
// with F^2 > 0 in FP64, and the dry rule zeroes its momentum anyway.
__device__ __forceinline__ bool coulomb_stops(float q1, float q2, float bX, float bY, float Fr, float qn2, double dt,
                                              float Jpbs, double tan_d)
{
    const float F2 = Fr * Fr;
    if (qn2 > F2 * (1.0f + 0x1p-10f)) return false;
    if (qn2 < F2 * (1.0f - 0x1p-10f) || ibits(qn2) == 0) return true;
    return stop_fp64(q1, q2, bX, bY, dt, Jpbs, tan_d);
}

__device__ __forceinline__ void coulomb(float &q1, float &q2, float bX, float bY, float Fr, double dt,
                                        float Jpbs, double tan_d)
{
    const float qZ = fmaf(bX, q1, bY * q2);
    const float qn2 = fmaf(q1, q1, fmaf(q2, q2, qZ * qZ));
    const bool stop = coulomb_stops(q1, q2, bX, bY, Fr, qn2, dt, Jpbs, tan_d);
    if (stop) {
        q1 = 0.0f;
        q2 = 0.0f;
        return;
    }
    if (ibits(Fr) <= 0) return;  // no friction: r = 1
    const float r = fmaf(-Fr, frsqrt(qn2), 1.0f);
    q1 *= r;
    q2 *= r;
}
__device__ __forceinline__ void coulomb(double &q1, double &q2, double bX, double bY, double Fr, double,
                                        double, double)
{
    coulomb(q1, q2, bX, bY, Fr);
}

// The first stage of a step publishes its time step to the later stages (and,
// when the step's start time was given, that time too); the adjoint's forward
// run also logs both (StageArgs::fix, t_log).  One thread of one CTA.
template <typename T>
__device__ __forceinline__ void first_stage_clock(const StageArgs<T> &a, double t_now, double dt)
{
    a.ctl->dt = dt;
    if (a.fix) a.ctl->t = t_now;
    if (a.t_log) {
        a.t_log[a.log_idx] = t_now;
        a.dt_log[a.log_idx] = dt;
    }
}

// End of a step, by the last CTA of its last stage: publish a_max (the exact
// maximum of the step's cell speeds, reduced on their IEEE bits) and advance t.
template <typename T>
__device__ __forceinline__ void end_step(const StageArgs<T> &a)
{
    Ctl *ctl = a.ctl;
    const unsigned long long m = atomicExch(&ctl->amax_acc, 0ull);
    if (a.want_amax) ctl->amax = m;
    if (ctl->dt > 0.0) {
        ctl->t = ctl->t + ctl->dt;
        ctl->steps += 1;
    }
}

template <typename T, int TX, int TY, bool VIS = false, bool KM = false>
constexpr size_t stage_smem_bytes()
{
    // state halo tile, slopes, face fluxes; FP32 or viscous: bed-slope tile;
    // viscous: fluid velocities of the slope tile; earth pressure: solid
    // velocities of the state halo tile
    return sizeof(T) * (6 * (TX + 4) * (TY + 4) + 6 * (TX + 2) * TY + 6 * TX * (TY + 2) + 7 * (TX + 1) * TY +
                        7 * TX * (TY + 1) + ((sizeof(T) == 4 || VIS) ? 4 * (TX + 2) * (TY + 2) : 0) +
                        (VIS ? 2 * (TX + 2) * (TY + 2) : 0) + (KM ? 2 * (TX + 4) * (TY + 4) : 0));
}

// Mass bits (MB_*) of a tile of TY rows from the ballots of its rows (bit l
// of rows[r]: column l of row r holds mass; columns and rows outside the
// grid hold none).
template <int TY>
__device__ __forceinline__ unsigned short mass_bits(const unsigned int *rows)
{
    static_assert(TY >= 2, "the side bits take two rows");
    unsigned int all = 0u;
    for (int r = 0; r < TY; r++) all |= rows[r];
    const unsigned int s = rows[0] | rows[1], n = rows[TY - 2] | rows[TY - 1];
    constexpr unsigned int W = 0x3u, E = 0xC0000000u;
    unsigned int b = 0u;
    if (all) b |= MB_ANY;
    if (all & W) b |= MB_W;
    if (all & E) b |= MB_E;
    if (s) b |= MB_S;
    if (n) b |= MB_N;
    if (s & W) b |= MB_SW;
    if (s & E) b |= MB_SE;
    if (n & W) b |= MB_NW;
    if (n & E) b |= MB_NE;
    return (unsigned short)b;
}

// Tile (bx, ty) of a gx x gy grid has mass within two cells of it, from the
// mass bits of its own and its eight neighbours' cells.  The 2-cell halo of a
// tile also takes ghost cells; a closed or transmissive ghost repeats a cell
// of the same row (column) within two cells of the side, so its mass shows
// in those bits too; inflow ghosts are the caller's (on_inflow_side).
__device__ __forceinline__ bool wet_from_bits(const unsigned short *mb, int bx, int ty, int gx, int gy)
{
    unsigned int w = mb[ty * gx + bx] & MB_ANY;
    const bool wx = bx > 0, ex = bx + 1 < gx, sy = ty > 0, ny_ = ty + 1 < gy;
    if (wx) w |= mb[ty * gx + bx - 1] & MB_E;
    if (ex) w |= mb[ty * gx + bx + 1] & MB_W;
    if (sy) {
        w |= mb[(ty - 1) * gx + bx] & MB_N;
        if (wx) w |= mb[(ty - 1) * gx + bx - 1] & MB_NE;
        if (ex) w |= mb[(ty - 1) * gx + bx + 1] & MB_NW;
    }
    if (ny_) {
        w |= mb[(ty + 1) * gx + bx] & MB_S;
        if (wx) w |= mb[(ty + 1) * gx + bx - 1] & MB_SE;
        if (ex) w |= mb[(ty + 1) * gx + bx + 1] & MB_SW;
    }
    return w != 0u;
}

// ---- the stage kernel -------------------------------------------------------------
// One stage on the tile (bx, by) of the simulation described by `a`; nb is the
// number of CTAs working on that simulation in this launch (for the ticket;
// 0: the caller takes it).
// KM: the earth-pressure form (k_mode 1, reading R10): each cell of the staged
// tile and halo gets its solid velocity (NaN where the cell carries no
// solid), from which each side of a face takes its cell's K_act or K_pass.
// P2: two threads per cell (2 TX TY threads): in the face phase the first TX TY
// take the x-faces, the others the y-faces, so that every SM sub-partition
// runs two warps of faces; the staging and the cell update stay on the first
// TX TY.  A step with about one wet tile per SM is bound by the latency of
// that tile's FP64 chain, which the second warp hides.
template <typename T, int TX, int TY, bool REC = false, bool VIS = false, bool CU = false, bool WENO = false,
          bool KM = false, bool P2 = false>
__device__ __forceinline__ void stage_tile(const StageArgs<T> &a, const int bx, const int by, const unsigned int nb)
{
    constexpr int NT = TX * TY;
    constexpr int NTH = P2 ? 2 * NT : NT;  // threads of the CTA
    constexpr int SW = TX + 4, SH = TY + 4, SP = SW * SH;
    constexpr int NSX = (TX + 2) * TY, NSY = TX * (TY + 2);  // cells with x- / y-slopes
    constexpr int NXF = (TX + 1) * TY, NYF = TX * (TY + 1);  // x- / y-faces
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sU = reinterpret_cast<T *>(smem_raw);  // [6][SH][SW]
    T *sSx = sU + 6 * SP;                      // [6][TY][TX+2]   minmod slopes along x
    T *sSy = sSx + 6 * NSX;                    // [6][TY+2][TX]   along y
    T *sHx = sSy + 6 * NSY;                    // [7][TY][TX+1]   2 x flux, 2 x P
    T *sHy = sHx + 7 * NXF;                    // [7][TY+1][TX]
    // FP32 form: bed slopes of the tile + 1-cell halo, [4][TY+2][TX+2]
    // (SX, SY, DBX, DBY); the geometry is rebuilt from them.  With the viscous
    // term (both forms) also the fluid velocities of the same cells, [2][..].
    constexpr bool GL = sizeof(T) == 4;
    constexpr bool SL = GL || VIS;
    constexpr int BW = TX + 2, NB = (TX + 2) * (TY + 2);
    T *sB = sHy + 7 * NYF;                  // allocated in the FP32 and viscous forms only
    T *sVf = sB + (SL ? 4 * NB : 0);        // viscous form only
    // KM: solid velocities (v_X, v_Y) of every staged cell, [2][SH][SW]
    T *sVs = sVf + (VIS ? 2 * NB : 0);
    // the regions above end where the launchers' dynamic allocation ends
    static_assert((6 * SP + 6 * NSX + 6 * NSY + 7 * NXF + 7 * NYF + (SL ? 4 * NB : 0) + (VIS ? 2 * NB : 0) +
                   (KM ? 2 * SP : 0)) * sizeof(T) == stage_smem_bytes<T, TX, TY, VIS, KM>(),
                  "shared-memory layout and allocation differ");
    auto SB = [&](int c, int cx, int cy) -> T { return sB[c * NB + cy * BW + cx]; };
    __shared__ T red[NT / 32];
    __shared__ double acc[4];
    __shared__ unsigned int acc_n;
    __shared__ bool last_block;

    const int tid = threadIdx.x;
    const bool cell_thread = !P2 || tid < NT;  // a thread with a cell of its own
    const int x0 = bx * TX, y0 = by * TY;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    const long long plane = a.plane;
    const KT<T> &k = a.k;
    const T *geo = a.geo;
    Ctl *ctl = a.ctl;
    __shared__ double s_dt, s_tg, s_bwf;
    __shared__ T s_dtT;

    // ---- stage the tile + 2-cell halo of the six state planes -----------
    // (asynchronous copies: every element of the thread in flight at once).
    // Each thread takes its own cell, then one cell of the halo if any, so
    // that only the halo needs index arithmetic.  The two mass planes come
    // first: they decide whether the tile has any work (below).
    constexpr int HMAX = (SP - NT + NT - 1) / NT;  // halo cells per thread, at most
    constexpr int NE = HMAX + 1;
    int eo[NE];        // shared-memory offset of each staged cell (-1: none)
    long long eg[NE];  // its global index
    bool eok[NE];      // inside the ghost-extended grid (else zero-filled)
    if (!cell_thread) {
#pragma unroll
        for (int e = 0; e < NE; e++) eo[e] = -1;
    } else {
        const auto entry = [&](int e, int tx, int ty) {  // tile coordinates, -2 .. TX+1 / TY+1
            const int gi = x0 + tx, gj = y0 + ty;
            eok[e] = gi < nx + 2 && gj < ny + 2;
            eg[e] = eok[e] ? cell_index(gi, gj, pitch) : 0;
            eo[e] = (ty + 2) * SW + tx + 2;
        };
        entry(0, tid % TX, tid / TX);
        constexpr int RW = 2 * SW;  // cells in two full halo rows
#pragma unroll
        for (int r = 0; r < HMAX; r++) {
            const int h = tid + r * NT;
            eo[r + 1] = -1;
            if (h >= SP - NT) continue;
            if (h < RW) entry(r + 1, h % SW - 2, h / SW - 2);                     // rows -2, -1
            else if (h < 2 * RW) entry(r + 1, (h - RW) % SW - 2, TY + (h - RW) / SW);  // rows TY, TY+1
            else {                                                              // columns -2, -1, TX, TX+1
                const int q = h - 2 * RW, kk = q & 3;
                entry(r + 1, kk < 2 ? kk - 2 : TX + kk - 2, q >> 2);
            }
        }
    }
    const auto copy_planes = [&](const int c0, const int c1, const int c2, const int c3, const int n) {
#pragma unroll
        for (int e = 0; e < NE; e++) {
            if (eo[e] < 0) continue;
            const int cs[4] = {c0, c1, c2, c3};
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (q < n) cp_async_elem(sU + cs[q] * SP + eo[e], a.Uin + (eok[e] ? cs[q] * plane + eg[e] : 0), eok[e]);
        }
    };
    // FP32 (and viscous) form: bed slopes of the tile + 1-cell halo
    const auto copy_slope_tile = [&]() {
        if (!cell_thread) return;
        if constexpr (SL) {
            // slope tile: cells x0-1 .. x0+TX, rows y0-1 .. y0+TY
            const auto copy_slopes = [&](int tx, int ty) {  // tile coordinates, -1 .. TX / TY
                const int gi = x0 + tx, gj = y0 + ty;
                const bool ok = gi <= nx && gj <= ny;
                const T *src = geo + (ok ? GS_SX * plane + cell_index(gi, gj, pitch) : 0);
                T *dst = sB + (ty + 1) * BW + tx + 1;
#pragma unroll
                for (int c = 0; c < 4; c++) cp_async_elem(dst + c * NB, src + (ok ? c * plane : 0), ok);
            };
            copy_slopes(tid % TX, tid / TX);
            for (int h = tid; h < NB - NT; h += NT) {
                if (h < BW) copy_slopes(h - 1, -1);                  // row -1
                else if (h < 2 * BW) copy_slopes(h - BW - 1, TY);    // row TY
                else {                                               // columns -1 and TX
                    const int r = h - 2 * BW;
                    copy_slopes((r & 1) ? TX : -1, r >> 1);
                }
            }
        }
    };
    // A tile from the wet-tile list holds mass: it copies everything at once.
    const bool listed = a.wl != nullptr;
    copy_planes(0, 3, 0, 0, 2);
    if (listed) {
        copy_planes(1, 2, 4, 5, 4);
        copy_slope_tile();
    }
    // the step's time and time step, once per CTA (after the copies are
    // issued: thread 0's control-block reads then overlap them)
    if (tid == 0) {
        double t_now, dt;
        if (a.debug_stage) {
            t_now = a.dbg_t;
            dt = a.dbg_dt;
        } else if (a.stage == 1 && a.fix) {
            t_now = a.fix_t;
            dt = a.fix_dt;
        } else if (a.stage == 1) {
            t_now = ctl->t;
            dt = dt_from(ctl, a.ph, __longlong_as_double((long long)ctl->amax));
        } else {
            t_now = ctl->t;
            dt = ctl->dt;
        }
        s_dt = dt;
        s_dtT = (T)dt;
        // ghosts at the time of this stage's output (the second RK3 stage: t + dt/2)
        s_tg = t_now + (a.rk3 == 2 ? 0.5 * dt : dt);
        // budget weight of this stage relative to the two-step Euler's 1/2
        s_bwf = a.rk3 ? 2.0 * a.rk3_bw : 1.0;
        // (thread 0 alone resets the accumulators it alone reads at the end,
        // so a CTA can run the next tile without a barrier in between)
        acc_n = 0;
        acc[0] = acc[1] = acc[2] = acc[3] = 0.0;
    }

    // Wet/dry masking: where no cell of the staged tile and halo holds mass
    // (U1 = U4 = 0; in the FP32 form also the tile's mass remainders, and in
    // a combining stage the tile's masses at U^n), every face flux, source
    // and speed of the tile is exactly 0 and the stage leaves the tile at 0
    // (zero masses, zero momenta by the dry rule; the recording form also
    // zero records).  Such a CTA neither loads the momenta and the geometry
    // nor does the arithmetic; the barrier tells every thread.  NaN counts as
    // mass.  Each thread tests its own cell's remainders and U^n (loaded while
    // the copies are in flight), then the cells it copied itself.
    bool has_mass = listed;
    if (!listed && cell_thread) {
        const int ci = x0 + tid % TX, cj = y0 + tid / TX;
        if (ci < nx && cj < ny) {
            const long long g = cell_index(ci, cj, pitch);
            if constexpr (sizeof(T) == 4) has_mass |= nonzero(a.Rin[g]) | nonzero(a.Rin[plane + g]);
            if (a.stage == 2 && !a.debug_stage) {
                has_mass |= nonzero(a.Un[g]) | nonzero(a.Un[3 * plane + g]);
                if constexpr (sizeof(T) == 4) has_mass |= nonzero(a.Rn[g]) | nonzero(a.Rn[plane + g]);
            }
        }
    }
    cp_async_wait_all();
    if (!listed) {
#pragma unroll
        for (int e = 0; e < NE; e++)
            if (eo[e] >= 0) has_mass |= nonzero(sU[eo[e]]) | nonzero(sU[3 * SP + eo[e]]);
    }
    const bool wet = __syncthreads_or(has_mass) != 0;
    if (wet && !listed) {  // CTA-uniform: the momenta, and the slope tile
        copy_planes(1, 2, 4, 5, 4);
        copy_slope_tile();
        cp_async_wait_all();
        __syncthreads();
    }
    const double dt = s_dt;
    const T dtT = s_dtT;
    const double bwf = s_bwf;
    if (wet) {  // CTA-uniform
        if constexpr (VIS) {
            // fluid velocity of every cell of the slope tile (0 where the fluid is
            // dry), with the same dry threshold as the cell update
            for (int q = tid; q < NB; q += NTH) {
                const int ly = q / BW, lx = q - ly * BW;
                const int gi = x0 - 1 + lx, gj = y0 - 1 + ly;
                const int o = (ly + 1) * SW + lx + 1;
                T jhdn;
                if constexpr (GL) {
                    const float sx = SB(0, lx, ly), sy = SB(1, lx, ly);
                    const float s2 = fmaf(sx, sx, fmaf(sy, sy, 1.0f));
                    jhdn = s2 * frsqrt(s2) * k.h_dry;
                } else {
                    jhdn = (gi <= nx + 1 && gj <= ny + 1) ? geo[GC_JHD * plane + cell_index(gi, gj, pitch)] : T(1);
                }
                const T u3 = sU[3 * SP + o];
                const T rf = gtp(u3, jhdn) ? frcp(u3) : T(0);
                sVf[q] = sU[4 * SP + o] * rf;
                sVf[NB + q] = sU[5 * SP + o] * rf;
            }
        }

        if constexpr (KM) {
            // solid velocity of every staged cell where it carries solid
            // (U1 > J h_dry), by IEEE division as the oracle takes it; NaN
            // elsewhere, so that every comparison with it fails
            for (int q = tid; q < SP; q += NTH) {
                const int gi = x0 + q % SW - 2, gj = y0 + q / SW - 2;
                T vx = T(NAN), vy = T(NAN);
                if (gi < nx + 2 && gj < ny + 2) {
                    const T u1 = sU[q];
                    if (gtp(u1, geo[GC_JHD * plane + cell_index(gi, gj, pitch)])) {
                        if constexpr (sizeof(T) == 8) {
                            vx = __ddiv_rn(sU[SP + q], u1);
                            vy = __ddiv_rn(sU[2 * SP + q], u1);
                        } else {
                            vx = __fdiv_rn(sU[SP + q], u1);
                            vy = __fdiv_rn(sU[2 * SP + q], u1);
                        }
                    }
                }
                sVs[q] = vx;
                sVs[SP + q] = vy;
            }
        }

        // ---- minmod slopes, once per cell and direction -----------------------
        // sSx[c][ly][lx'] holds the x-slope of cell (x0-1+lx', y0+ly), sSy[c][ly'][lx]
        // the y-slope of cell (x0+lx, y0-1+ly').  Each thread takes both slopes of
        // its own cell, then a share of the halo ones (x: columns -1 and TX; y:
        // rows -1 and TY), so that only the halo needs index arithmetic.
        // (The WENO form reconstructs each face value in the face loop instead.)
        if constexpr (!WENO) {
            if (cell_thread) {
                const int lx = tid % TX, ly = tid / TX;
                const T *p = sU + (ly + 2) * SW + lx + 2;
    #pragma unroll
                for (int c = 0; c < 6; c++) {
                    const T *q = p + c * SP;
                    sSx[c * NSX + ly * (TX + 2) + lx + 1] = minmod(q[0] - q[-1], q[1] - q[0]);
                    sSy[c * NSY + (ly + 1) * TX + lx] = minmod(q[0] - q[-SW], q[SW] - q[0]);
                }
            }
            constexpr int NHX = 2 * TY, NHY = 2 * TX, NH1 = NHX + NHY;
            for (int e = tid; e < 6 * NH1; e += NTH) {
                const int c = e / NH1;
                int r = e - c * NH1;
                if (r < NHY) {  // y-slopes of rows -1 (r < TX) and TY
                    const int side = r / TX, col = r - side * TX, row = side ? TY : -1;
                    const T *q = sU + c * SP + (row + 2) * SW + col + 2;
                    sSy[c * NSY + (row + 1) * TX + col] = minmod(q[0] - q[-SW], q[SW] - q[0]);
                } else {  // x-slopes of columns -1 and TX
                    r -= NHY;
                    const int row = r >> 1, col = (r & 1) ? TX : -1;
                    const T *q = sU + c * SP + (row + 2) * SW + col + 2;
                    sSx[c * NSX + row * (TX + 2) + col + 1] = minmod(q[0] - q[-1], q[1] - q[0]);
                }
            }
        }
        __syncthreads();

        // ---- faces: x-faces (i+1/2, j), i = x0-1 .. x0+TX-1, at sHx[c][ly][lx],
        // lx = i - x0 + 1; y-faces (i, j+1/2), j = y0-1 .. y0+TY-1, at
        // sHy[c][ly][lx], ly = j - y0 + 1.  Each thread takes the right and the
        // upper face of its own cell; warp 0 the left faces of column 0, warp 1
        // the lower faces of row 0 (every warp then runs at most three faces).
        // K of the staged cell at offset o for the axis with offset step `st`
        // and velocity component c (KM): K_pass where cell_passive, else K_act
        const auto cellK = [&](const int o, const int st, const int c) -> T {
            return cell_passive(sVs + c * SP, o, st) ? k.Kp : k.Ka;
        };
        const auto x_face = [&](const int lx, const int ly) {
            const int i = x0 + lx - 1, j = y0 + ly;
            if (j >= ny || i >= nx) return;
            const int f = ly * (TX + 1) + lx;
            FaceGeo<T> G;
            if constexpr (GL) {  // lower cell at (lx, ly + 1) of the slope tile
                G = face_geo32(SB(2, lx, ly + 1), 0.5f * (SB(1, lx, ly + 1) + SB(1, lx + 1, ly + 1)), k);
            } else {
                const long long g = cell_index(i, j, pitch);
                G = FaceGeo<T>{geo[GX_JHD * plane + g], geo[GX_SN * plane + g], geo[GX_ST * plane + g],
                               geo[GX_FN * plane + g],  geo[GX_FT * plane + g], geo[GX_FN2 * plane + g],
                               geo[GX_HG * plane + g]};
            }
            const int ou = (ly + 2) * SW + lx + 1;  // left cell in sU
            const int os = ly * (TX + 2) + lx;      // left cell in sSx
            T um[6], up[6];
    #pragma unroll
            for (int c = 0; c < 6; c++) {
                if constexpr (WENO) {
                    const T *p = sU + c * SP + ou;
                    um[c] = weno3_face(p[-1], p[0], p[1]);
                    up[c] = weno3_face(p[2], p[1], p[0]);
                    if (c == 0 || c == 3) {  // masses stay >= 0 at the faces
                        um[c] = fmax(um[c], T(0));
                        up[c] = fmax(up[c], T(0));
                    }
                } else {
                    um[c] = fma(T(0.5), sSx[c * NSX + os], sU[c * SP + ou]);
                    up[c] = fma(T(-0.5), sSx[c * NSX + os + 1], sU[c * SP + ou + 1]);
                }
            }
            T H[7];
            if constexpr (CU) face_flux2_cu<T, 0>(um, up, G, H);
            else if constexpr (KM) {
                FaceGeo<T> Gm = G, Gp = G;
                const T Km = cellK(ou, 1, 0), Kp = cellK(ou + 1, 1, 0);
                Gm.sn *= Km;
                Gm.st *= Km;
                Gp.sn *= Kp;
                Gp.st *= Kp;
                face_flux2<T, 0, false>(um, up, Gm, Gp, H);
            } else face_flux2<T, 0>(um, up, G, G, H);
            if constexpr (sizeof(T) == 4) {
                // FP32: the mass change this face gives each neighbour, rounded once
                H[0] *= dtT * k.hinv_dx;
                H[3] *= dtT * k.hinv_dx;
            }
    #pragma unroll
            for (int c = 0; c < 7; c++) sHx[c * NXF + f] = H[c];
            if (!a.debug_stage && (i == -1 || i == nx - 1) && j >= a.own_j0 && j < a.own_j1) {
                // the stage's budget weight (Heun 1/2; RK3 1/6, 1/6, 2/3) x boundary volume flux
                const double w = (sizeof(T) == 4 ? 0.5 * a.ph.cell_area : 0.25 * dt * a.ph.dy) * (i == -1 ? 1.0 : -1.0) * bwf;
                atomicAdd(&acc[0], w * (double)H[0]);
                atomicAdd(&acc[1], w * (double)H[3]);
            }
        };
        const auto y_face = [&](const int lx, const int ly) {
            const int i = x0 + lx, j = y0 + ly - 1;
            if (i >= nx || j >= ny) return;
            const int f = ly * TX + lx;
            FaceGeo<T> G;
            if constexpr (GL) {  // lower cell at (lx + 1, ly) of the slope tile
                G = face_geo32(SB(3, lx + 1, ly), 0.5f * (SB(0, lx + 1, ly) + SB(0, lx + 1, ly + 1)), k);
            } else {
                const long long g = cell_index(i, j, pitch);
                G = FaceGeo<T>{geo[GY_JHD * plane + g], geo[GY_SN * plane + g], geo[GY_ST * plane + g],
                               geo[GY_FN * plane + g],  geo[GY_FT * plane + g], geo[GY_FN2 * plane + g],
                               geo[GY_HG * plane + g]};
            }
            const int ou = (ly + 1) * SW + lx + 2;  // lower cell in sU
            const int os = ly * TX + lx;            // lower cell in sSy
            T um[6], up[6];
    #pragma unroll
            for (int c = 0; c < 6; c++) {
                if constexpr (WENO) {
                    const T *p = sU + c * SP + ou;
                    um[c] = weno3_face(p[-SW], p[0], p[SW]);
                    up[c] = weno3_face(p[2 * SW], p[SW], p[0]);
                    if (c == 0 || c == 3) {
                        um[c] = fmax(um[c], T(0));
                        up[c] = fmax(up[c], T(0));
                    }
                } else {
                    um[c] = fma(T(0.5), sSy[c * NSY + os], sU[c * SP + ou]);
                    up[c] = fma(T(-0.5), sSy[c * NSY + os + TX], sU[c * SP + ou + SW]);
                }
            }
            T H[7];
            if constexpr (CU) face_flux2_cu<T, 1>(um, up, G, H);
            else if constexpr (KM) {
                FaceGeo<T> Gm = G, Gp = G;
                const T Km = cellK(ou, SW, 1), Kp = cellK(ou + SW, SW, 1);
                Gm.sn *= Km;
                Gm.st *= Km;
                Gp.sn *= Kp;
                Gp.st *= Kp;
                face_flux2<T, 1, false>(um, up, Gm, Gp, H);
            } else face_flux2<T, 1>(um, up, G, G, H);
            if constexpr (sizeof(T) == 4) {
                H[0] *= dtT * k.hinv_dy;
                H[3] *= dtT * k.hinv_dy;
            }
    #pragma unroll
            for (int c = 0; c < 7; c++) sHy[c * NYF + f] = H[c];
            if (!a.debug_stage && ((j == -1 && a.own_j0 == 0) || (j == ny - 1 && a.own_j1 == ny))) {
                const double w = (sizeof(T) == 4 ? 0.5 * a.ph.cell_area : 0.25 * dt * a.ph.dx) * (j == -1 ? 1.0 : -1.0) * bwf;
                atomicAdd(&acc[0], w * (double)H[0]);
                atomicAdd(&acc[1], w * (double)H[3]);
            }
        };
        if constexpr (P2) {
            // the x-faces on the first NT threads, the y-faces on the others;
            // the lower faces of row 0 on warp 2 and the left faces of column 0
            // on the last warp (warps w and w + 4 share a sub-partition: the
            // extra rounds land on two different ones)
            static_assert(TX == 32 && NT >= 96 && TY <= 32, "face assignment of the two-thread form");
            if (tid < NT) x_face(tid % TX + 1, tid / TX);
            else y_face((tid - NT) % TX, (tid - NT) / TX + 1);
            if (tid >= 64 && tid < 64 + TX) y_face(tid - 64, 0);
            else if (tid >= NTH - 32 && tid < NTH - 32 + TY) x_face(0, tid - (NTH - 32));
        } else {
            static_assert(NT >= 32 + TX && TY <= 32, "face assignment needs warps 0 and 1");
            x_face(tid % TX + 1, tid / TX);
            y_face(tid % TX, tid / TX + 1);
            if (tid < TY) x_face(0, tid);
            else if (tid >= 32 && tid < 32 + TX) y_face(tid - 32, 0);
        }
        __syncthreads();
    }

    // ---- cell update ------------------------------------------------------
    const int lx = tid % TX, ly = tid / TX;
    const int i = x0 + lx, j = y0 + ly;
    const bool in_grid = cell_thread && i < nx && j < ny;
    T speed = T(0);
    bool bad = false;
    bool mass = false;  // the cell's output holds mass (mass bits)
    if (!wet && in_grid) {
        const long long g = cell_index(i, j, pitch);
        const T z[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        store6(a.Uout, plane, g, z);
        if constexpr (REC) store6(a.rec, plane, g, z);
        if constexpr (sizeof(T) == 4) {
            a.Rout[g] = 0.0f;
            a.Rout[plane + g] = 0.0f;
        }
        if (!a.debug_stage) write_ghosts(a.Uout, geo, a, i, j, z, s_tg);
    } else if (in_grid) {
        const long long g = cell_index(i, j, pitch);
        const int os = (ly + 2) * SW + lx + 2;
        // the cell's geometry: FP32 rebuilt from the slope tile, FP64 read
        CellGeo32 cgf{};
        if constexpr (GL) {
            const int cx = lx + 1, cy = ly + 1;
            cgf = cell_geo32(SB(0, cx, cy), SB(1, cx, cy), (SB(2, cx, cy) - SB(2, cx - 1, cy)) * k.inv_dx,
                             (SB(1, cx + 1, cy) - SB(1, cx - 1, cy)) * k.inv_2dx,
                             (SB(3, cx, cy) - SB(3, cx, cy - 1)) * k.inv_dy, k);
        }
        const auto CG = [&](const int P) -> T {
            if constexpr (GL) {
                switch (P) {
                case GC_JHD: return cgf.jhd;
                case GC_GC1: return cgf.gc1;
                case GC_GCF: return cgf.gcf;
                case GC_BX: return cgf.bX;
                case GC_BY: return cgf.bY;
                case GC_MNX: return cgf.nX;
                case GC_MNY: return cgf.nY;
                case GC_A11: return cgf.A11;
                case GC_A12: return cgf.A12;
                case GC_A22: return cgf.A22;
                case GC_KXX: return cgf.kXX;
                case GC_KXY2: return cgf.kXY2;
                case GC_KYY: return cgf.kYY;
                case GC_SXS: return cgf.sxs;
                case GC_SXF: return cgf.sxf;
                case GC_SYS: return cgf.sys;
                default: return cgf.syf;
                }
            } else {
                return geo[P * plane + g];
            }
        };
        T u[6];
#pragma unroll
        for (int c = 0; c < 6; c++) u[c] = sU[c * SP + os];
        const T jhd = CG(GC_JHD);
        const T Ut = u[0] + u[3];
        // volume fractions phi^s, phi^f (0 where h <= h_dry)
        const T rUt = gtp(Ut, jhd) ? frcp(Ut) : T(0);
        const T phs = u[0] * rUt, phf = u[3] * rUt;
        const T rs = gtp(u[0], jhd) ? frcp(u[0]) : T(0);
        const T rf = gtp(u[3], jhd) ? frcp(u[3]) : T(0);
        const T vXs = u[1] * rs, vYs = u[2] * rs, vXf = u[4] * rf, vYf = u[5] * rf;
        // -kappa = c (bXX vX^2 + 2 bXY vX vY + bYY vY^2): the centripetal term
        // sum_k v_k (dn_k/dxi v_xi + dn_k/deta v_eta) with v tangent to the bed
        const T kXX = CG(GC_KXX), kXY2 = CG(GC_KXY2), kYY = CG(GC_KYY);
        const T nks = fma(kXX, vXs * vXs, fma(kXY2, vXs * vYs, kYY * (vYs * vYs)));
        const T nkf = fma(kXX, vXf * vXf, fma(kXY2, vXf * vYf, kYY * (vYf * vYf)));
        // J p_b = U (g c (1 - alpha) - eps^chi kappa), clamped at 0 (lift-off)
        const T Jpbs = pos(u[0] * fma(k.eps_chi, nks, CG(GC_GC1)));
        const T Jpbf = pos(u[3] * fma(k.eps_chi, nkf, CG(GC_GCF)));
        const T nX = CG(GC_MNX), nY = CG(GC_MNY);
        // gradient of P = J h pbar^f from its (doubled) face values
        const int fx = ly * (TX + 1) + lx, fy = ly * TX + lx;
        const T dPx = (sHx[6 * NXF + fx + 1] - sHx[6 * NXF + fx]) * k.hinv_dx;
        const T dPy = (sHy[6 * NYF + fy + TX] - sHy[6 * NYF + fy]) * k.hinv_dy;
        const T A11 = CG(GC_A11), A12 = CG(GC_A12), A22 = CG(GC_A22);
        const T gX = fma(A11, dPx, A12 * dPy), gY = fma(A12, dPx, A22 * dPy);
        const T bs = -k.eps_alpha * phs;                         // s_f^s = bs grad
        const T bf = k.eps * (a.ph.pg_mode == 1 ? phf : phs);   // s_f^f = bf grad (R1)
        const T D = k.c_d * phs * phf * Ut;                     // J c_D phi^s phi^f h
        const T aD = k.alpha * D;
        const T dvX = vXf - vXs, dvY = vYf - vYs;
        const T ff = k.k_f * phf * Ut;                          // J phi^f h k_f
        T S[6];
        S[0] = T(0);
        S[3] = T(0);
        S[1] = fma(Jpbs, nX, fma(bs, gX, aD * dvX));
        S[2] = fma(Jpbs, nY, fma(bs, gY, aD * dvY));
        S[4] = fma(Jpbf, nX, fma(bf, gX, -fma(D, dvX, ff * vXf)));
        S[5] = fma(Jpbf, nY, fma(bf, gY, -fma(D, dvY, ff * vYf)));
        if constexpr (VIS) {
            // viscous term s_vis^f = nu_f phi^f (s_vis,X, s_vis,Y) (Eq. SrcF_vis_Topo):
            // brackets J h (A grad v) on the four faces (face-normal differences,
            // transverse derivatives as the mean of the two cells' central
            // differences; face metric from the face slopes), differenced
            if (gtp(Ut, jhd) && gtp(u[3], jhd)) {
                const int cx = lx + 1, cy = ly + 1;
                const auto V = [&](int m, int ddx, int ddy) -> T { return sVf[m * NB + (cy + ddy) * BW + cx + ddx]; };
                const auto JH = [&](int ddx, int ddy) -> T {
                    const int o = (ly + 2 + ddy) * SW + lx + 2 + ddx;
                    return sU[o] + sU[3 * SP + o];
                };
                T brX[2][2], brY[2][2];
#pragma unroll
                for (int sd = 0; sd < 2; sd++) {
                    const int l = sd - 1;  // lower cell of the face, offset along the normal
                    {   // x-face between cells i+l and i+l+1
                        const T bn = SB(2, cx + l, cy), bt = T(0.5) * (SB(1, cx + l, cy) + SB(1, cx + l + 1, cy));
                        const T r2 = frcp(fma(bn, bn, fma(bt, bt, T(1))));
                        const T A11 = fma(bt, bt, T(1)) * r2, A12 = -bn * bt * r2, A22 = fma(bn, bn, T(1)) * r2;
                        const T Jh = T(0.5) * (JH(l, 0) + JH(l + 1, 0));
                        T dX[2], dY[2];
#pragma unroll
                        for (int m = 0; m < 2; m++) {
                            dX[m] = (V(m, l + 1, 0) - V(m, l, 0)) * k.inv_dx;
                            dY[m] = T(0.5) * ((V(m, l, 1) - V(m, l, -1)) + (V(m, l + 1, 1) - V(m, l + 1, -1))) * k.inv_2dy;
                        }
                        brX[sd][0] = Jh * fma(A11, dX[0], A12 * dY[0]);
                        brX[sd][1] = Jh * fma(A12, dX[0], fma(A22, dY[0], fma(A11, dX[1], A12 * dY[1])));
                    }
                    {   // y-face between cells j+l and j+l+1
                        const T bn = SB(3, cx, cy + l), bt = T(0.5) * (SB(0, cx, cy + l) + SB(0, cx, cy + l + 1));
                        const T r2 = frcp(fma(bn, bn, fma(bt, bt, T(1))));
                        const T A11 = fma(bn, bn, T(1)) * r2, A12 = -bn * bt * r2, A22 = fma(bt, bt, T(1)) * r2;
                        const T Jh = T(0.5) * (JH(0, l) + JH(0, l + 1));
                        T dX[2], dY[2];
#pragma unroll
                        for (int m = 0; m < 2; m++) {
                            dY[m] = (V(m, 0, l + 1) - V(m, 0, l)) * k.inv_dy;
                            dX[m] = T(0.5) * ((V(m, 1, l) - V(m, -1, l)) + (V(m, 1, l + 1) - V(m, -1, l + 1))) * k.inv_2dx;
                        }
                        brY[sd][0] = Jh * fma(A12, dX[0], fma(A22, dY[0], fma(A11, dX[1], A12 * dY[1])));
                        brY[sd][1] = Jh * fma(A12, dX[1], A22 * dY[1]);
                    }
                }
                const T svX = fma(T(2) * (brX[1][0] - brX[0][0]), k.inv_dx, (brY[1][0] - brY[0][0]) * k.inv_dy);
                const T svY = fma(T(2) * (brY[1][1] - brY[0][1]), k.inv_dy, (brX[1][1] - brX[0][1]) * k.inv_dx);
                S[4] = fma(k.nu_f * phf, svX, S[4]);
                S[5] = fma(k.nu_f * phf, svY, S[5]);
            }
        }
        T out[6];
        T lo[2] = {T(0), T(0)};  // FP32: rounding remainders of the masses
        const T dthx = dtT * k.hinv_dx, dthy = dtT * k.hinv_dy;
#pragma unroll
        for (int c = 0; c < 6; c++) {
            if constexpr (sizeof(T) == 4) {
                if (c == 0 || c == 3) {
                    // mass: U + R plus the four scaled face terms, summed
                    // without loss (TwoSum), renormalised into (U, R)
                    float s = u[c], e = a.Rin[(c / 3) * plane + g], t;
                    const float terms[4] = {sHx[c * NXF + fx], -sHx[c * NXF + fx + 1], sHy[c * NYF + fy],
                                            -sHy[c * NYF + fy + TX]};
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        two_sum(s, terms[q], s, t);
                        e += t;
                    }
                    out[c] = s + e;
                    lo[c / 3] = e - (out[c] - s);
                    continue;
                }
            }
            // u + dt S - dt (dH_x / 2dx + dH_y / 2dy), the sources first (the
            // mass components have none)
            const T dx2 = sHx[c * NXF + fx + 1] - sHx[c * NXF + fx];
            const T dy2 = sHy[c * NYF + fy + TX] - sHy[c * NYF + fy];
            const T base = (c == 0 || c == 3) ? u[c] : fma(dtT, S[c], u[c]);
            out[c] = fma(-dthy, dy2, fma(-dthx, dx2, base));
        }
        if constexpr (REC) {
#pragma unroll
            for (int c = 0; c < 4; c++) a.rec[c * plane + g] = out[c];
            a.rec[4 * plane + g] = dPx;
            a.rec[5 * plane + g] = dPy;
        }
        if constexpr (sizeof(T) == 8)
            coulomb(out[1], out[2], CG(GC_BX), CG(GC_BY), dt * Jpbs * k.tan_delta);
        else
            coulomb(out[1], out[2], CG(GC_BX), CG(GC_BY), dtT * Jpbs * k.tan_delta, dt,
                    Jpbs, k.tan_delta_d);
        // positivity clamp (counted) and dry momentum
#pragma unroll
        for (int ph = 0; ph < 2; ph++) {
            const int c = 3 * ph;
            if (negative(out[c])) {
                if (!a.debug_stage && j >= a.own_j0 && j < a.own_j1) {
                    atomicAdd(&acc[2 + ph], -0.5 * ((double)out[c] + (double)lo[ph]) * a.ph.cell_area * bwf);
                    atomicAdd(&acc_n, 1u);
                }
                out[c] = T(0);
                lo[ph] = T(0);
            }
            if (!gtp(out[c], jhd)) {
                out[c + 1] = T(0);
                out[c + 2] = T(0);
            }
        }
        if (a.stage == 2 && !a.debug_stage && a.rk3) {
            // three-stage Runge-Kutta: out + w (U^n - out), w = 3/4 (stage 2)
            // or 1/3 (stage 3); the weights sum to 1 exactly in any precision
            const T wn = a.rk3 == 2 ? T(0.75) : T(1.0 / 3.0);
#pragma unroll
            for (int c = 0; c < 6; c++) {
                if constexpr (sizeof(T) == 4) {
                    if (c == 0 || c == 3) {
                        // on (value, remainder) pairs: d = (U^n + R^n) - (out + lo)
                        float dh, dl, sv, e;
                        two_sum(a.Un[c * plane + g], -out[c], dh, dl);
                        dl += a.Rn[(c / 3) * plane + g] - lo[c / 3];
                        const float pr = wn * dh;
                        const float pe = fmaf(wn, dh, -pr) + wn * dl;  // exact product error + low part
                        two_sum(out[c], pr, sv, e);
                        e += lo[c / 3] + pe;
                        out[c] = sv + e;
                        lo[c / 3] = e - (out[c] - sv);
                        continue;
                    }
                }
                out[c] = fma(wn, a.Un[c * plane + g] - out[c], out[c]);
            }
#pragma unroll
            for (int ph = 0; ph < 2; ph++)
                if (!gtp(out[3 * ph], jhd)) {
                    out[3 * ph + 1] = T(0);
                    out[3 * ph + 2] = T(0);
                }
            if (a.rk3 == 3 && a.want_amax)
                speed = cell_speed(out, CG(GC_JHD), CG(GC_SXS), CG(GC_SXF), CG(GC_SYS), CG(GC_SYF));
        } else if (a.stage == 2 && !a.debug_stage) {
            // Heun average with U^n (same cell), dry momentum again
#pragma unroll
            for (int c = 0; c < 6; c++) {
                if constexpr (sizeof(T) == 4) {
                    if (c == 0 || c == 3) {
                        // (U^n + R^n + U** + R**) / 2 on (value, remainder) pairs
                        float s, e;
                        two_sum(a.Un[c * plane + g], out[c], s, e);
                        e += a.Rn[(c / 3) * plane + g] + lo[c / 3];
                        s *= 0.5f;
                        e *= 0.5f;
                        out[c] = s + e;
                        lo[c / 3] = e - (out[c] - s);
                        continue;
                    }
                }
                out[c] = T(0.5) * (a.Un[c * plane + g] + out[c]);
            }
#pragma unroll
            for (int ph = 0; ph < 2; ph++)
                if (!gtp(out[3 * ph], jhd)) {
                    out[3 * ph + 1] = T(0);
                    out[3 * ph + 2] = T(0);
                }
            if (a.want_amax) speed = cell_speed(out, CG(GC_JHD), CG(GC_SXS), CG(GC_SXF), CG(GC_SYS), CG(GC_SYF));
        }
#pragma unroll
        for (int c = 0; c < 6; c++) bad |= nonfinite(out[c]);
        store6(a.Uout, plane, g, out);
        mass = nonzero(out[0]) | nonzero(out[3]);
        if constexpr (sizeof(T) == 4) {
            a.Rout[g] = lo[0];
            a.Rout[plane + g] = lo[1];
            mass |= nonzero(lo[0]) | nonzero(lo[1]);
        }
        if (!a.debug_stage) write_ghosts(a.Uout, geo, a, i, j, out, s_tg);
    }

    if (a.debug_stage) return;
    __shared__ unsigned int s_mrow[TY];  // ballots of the output's mass by row (TX == 32: a warp per row)
    if (TX == 32 && a.mb_out) {
        const unsigned int row = __ballot_sync(0xffffffffu, mass);
        if ((tid & 31) == 0 && cell_thread) s_mrow[tid >> 5] = row;
    }

    // ---- CTA reductions ---------------------------------------------------
    if (bad) atomicOr(&ctl->status, (int)STATUS_NONFINITE);
    const bool finalize = a.stage == 2 && a.rk3 != 2;  // the step's last stage
    if (finalize && a.want_amax) {
        if (j < a.own_j0 || j >= a.own_j1) speed = T(0);  // a row another strip owns
        if (nonfinite(speed)) atomicOr(&ctl->status, (int)STATUS_NONFINITE);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) speed = maxnn(speed, __shfl_xor_sync(0xffffffffu, speed, o));
        if ((tid & 31) == 0 && cell_thread) red[tid >> 5] = speed;
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
        if (a.stage == 1 && bx == 0 && by == 0) first_stage_clock(a, a.fix ? a.fix_t : ctl->t, dt);
        if (TX == 32 && a.mb_out) a.mb_out[by * ((nx + 31) / 32) + bx] = mass_bits<TY>(s_mrow);
        if (finalize) {
            if (a.want_amax) {
                T m = T(0);
                for (int w = 0; w < NT / 32; w++) m = maxnn(m, red[w]);
                atomicMax(&ctl->amax_acc, (unsigned long long)__double_as_longlong((double)m));
            }
            if (nb) {
                __threadfence();
                last_block = (atomicAdd(&ctl->ticket, 1u) == nb - 1);
            }
        }
    }
    if (!finalize || nb == 0) return;  // nb == 0: the caller ends the step
    __syncthreads();
    if (last_block && tid == 0) {
        __threadfence();
        ctl->ticket = 0;
        end_step(a);
    }
}

template <typename T, int TX, int TY, bool REC = false, bool VIS = false, bool CU = false, bool WENO = false,
          bool KM = false>
__global__ void __launch_bounds__(TX *TY, 512 / (TX * TY)) stage_kernel(const StageArgs<T> a)
{
    stage_tile<T, TX, TY, REC, VIS, CU, WENO, KM>(a, blockIdx.x, blockIdx.y, gridDim.x * gridDim.y);
}

// The stepping launches follow one another as programmatic dependent launches
// (stage_launch.cuh): a kernel may start while the one before it finishes, and
// waits here, before its first read of anything that kernel wrote, until it
// has completed and its writes are visible.  Without such a launch the wait
// returns at once.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// A launch that may begin while the stream's previous kernel finishes
// (programmatic dependent launch): its CTAs are scheduled as the previous
// kernel's CTAs retire, and the kernel waits (wait_prior_grid) before its first
// read of that kernel's results.  The stepping launches chain this way, so that
// each one's launch latency overlaps the tail of the one before.
template <typename... KArgs, typename... Args>
cudaError_t launch_after(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                         Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}


// ---- bulk copies (the TMA engine) completed on an mbarrier -------------------------
__device__ __forceinline__ unsigned int smem_u32(const void *p) { return (unsigned int)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// the barrier's memory may be initialised again (no copy or wait pending on it)
__device__ __forceinline__ void mbar_inval(unsigned long long *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned int bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared, `bytes` a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned int bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// wait for phase `parity` of the mbarrier for at most ~`ns` nanoseconds (and
// at most 2^26 tries); false if it gave up
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned int parity, unsigned long long ns)
{
    const unsigned long long t0 = global_ns();
    unsigned int done = 0;
    for (int it = 0; it < (1 << 26) && !done; ++it) {
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(smem_u32(bar)), "r"(parity)
                     : "memory");
        if (!done && (it & 255) == 255 && global_ns() - t0 > ns) break;
    }
    return done != 0;
}

// tile (tx, ty) of a gx x gy grid of tiles lies on a side with an inflow
// segment (its ghost state changes within a step)
template <typename T>
__device__ __forceinline__ bool on_inflow_side(const StageArgs<T> &a, int tx, int ty, int gx, int gy)
{
    bool on = false;
    for (int f = 0; f < a.n_inflow; f++) {
        const int sd = a.inflow[f].side;
        on |= (sd == 0 && tx == 0) || (sd == 1 && tx == gx - 1) || (sd == 2 && ty == 0) || (sd == 3 && ty == gy - 1);
    }
    return on;
}

// Whether the classification leaves tile `idx` unwritten: a tile with work
// (the stage kernel writes it), or a dry tile whose output already holds the
// zero state (known-zero flags; see StageArgs::zk; `known` is the tile's flag,
// loaded early by the caller), which it keeps up to date.
template <typename T>
__device__ __forceinline__ bool keep_tile(const StageArgs<T> &a, bool wet, bool inflow_side, int idx,
                                          unsigned char known)
{
    if (!a.zk) return wet;
    const bool fixed = !wet && !inflow_side;  // the zero state written now stays valid
    if (fixed != (known != 0)) a.zk[idx] = fixed;
    return wet || (fixed && known != 0);
}

// Shared memory of the data classification of one strip (classify_strip):
// the two mass planes of the strip and its 2-cell halo, the strip's own extra
// planes, the copy barrier and the per-row and per-tile votes.  The TMA row
// copies land at 16-byte multiples (rows of 36 elements).
template <typename T>
struct __align__(16) ClassifySmem {
    T m[2][kStripRows + 4][36];                          // U1, U4 of the strip and its halo
    T x[sizeof(T) == 4 ? 6 : 2][kStripRows][36];         // own extras: FP32 R (2); combining: U^n's U1, U4, FP32 R^n
    unsigned long long bar;                              // the copies' mbarrier
    double tg;                                           // time of the ghosts written here
    unsigned int row[kStripRows + 4];                    // row y0 - 2 + r of the strip and halo has work
    unsigned int own[kStripRows];                        // the strip's own cells with mass in Uin, by row
    bool keep[kStripRows];                               // the tile is not zero-written here (keep_tile)
};

// the box b (x min, y min, x max, y max) widened to the tile (x, y)
__device__ __forceinline__ void box_add(int *b, int x, int y)
{
    atomicMin(&b[0], x);
    atomicMin(&b[1], y);
    atomicMax(&b[2], x);
    atomicMax(&b[3], y);
}

// Wet/dry masking over a whole launch, for the stepping of the plain form.
// A tile (32 x TY cells) holds work if a cell of it or of its 2-cell halo has
// mass (U1 or U4 non-zero; NaN counts), or if a cell of it has a non-zero
// FP32 mass remainder or, in a combining stage, mass at U^n.  A dry tile's
// stage result is known -- zero state, zero remainders, the ghost cells it
// owns filled from it -- and is written here, unless the output buffer holds
// it already from an earlier step (known-zero flags); a tile with work is
// appended to the list that stage_kernel_list runs.  One CTA (kStripWarps warps) covers a
// strip of 32 x kStripRows cells: the TMA engine copies the rows of the strip and
// its halo (36 cells from x0 - 2, a 16-byte aligned start) of the planes the
// test reads into shared memory, all in flight together, completed on one
// mbarrier (a bounded wait); each warp then tests whole rows with a warp vote
// and the tiles of the strip OR their rows.  The step's time step is taken
// here as the stage kernel takes it (stage 1 records it).
// The strip (bx, sy) of the simulation `a` (gx tiles across); `append(tx, ty)`
// lists a wet tile.
template <typename T, int TY, typename Append>
__device__ __forceinline__ bool classify_strip(const StageArgs<T> &a, const int bx, const int sy, const int gx,
                                               ClassifySmem<T> &sm, const Append &append)
{
    constexpr int S = kStripRows, H = S + 4, W = 36, NTL = S / TY;
    static_assert(S % TY == 0, "strip of whole tiles");
    constexpr bool F32 = sizeof(T) == 4;
    constexpr int CR = 16 / sizeof(T);  // cells per 16 bytes
    auto &s_m = sm.m;
    auto &s_x = sm.x;
    auto &s_bar = sm.bar;
    auto &s_tg = sm.tg;
    auto &s_row = sm.row;
    auto &s_own = sm.own;
    auto &s_keep = sm.keep;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int x0 = bx * 32, y0 = sy * S;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    const long long plane = a.plane;
    Ctl *ctl = a.ctl;
    const bool combine = a.stage == 2;
    const int nxp = (F32 ? 2 : 0) + (combine ? (F32 ? 4 : 2) : 0);  // extra planes copied
    // cells x0-2 .. x0+33 clipped to the ghost-extended grid (gi < nx + 2),
    // rounded up to 16 bytes (the few cells past nx + 1 lie in the row's
    // padding or the next row, inside the plane, and are never tested)
    const int l0 = min(W, nx + 4 - x0);
    const unsigned int rb = (unsigned int)((l0 + CR - 1) / CR * CR * sizeof(T));
    const int nrow = min(H, ny + 4 - y0);  // rows with gj = y0 - 2 + r < ny + 2
    const int nown = min(S, ny - y0);      // rows of the strip inside the grid
    const int nc = 2 * nrow + nxp * nown;  // row copies
    const bool from_flags = a.tw_prev != nullptr && a.stage == 2;
    // the known-zero flags of the strip's tiles, loaded first: the CTA is
    // latency-bound, and this load then overlaps the row copies (or the flag
    // loads of a combining stage).  Only this CTA reads or writes them.
    unsigned char known = 0;
    if (a.zk && tid < NTL && y0 + tid * TY < ny) known = a.zk[((y0 + tid * TY) / TY) * gx + bx];
    if (from_flags) {
        // a combining stage: its input has mass only in the tiles the stage
        // before found wet (it wrote zeros elsewhere), and U^n only in the
        // first stage's wet tiles, which those include; a tile with a wet
        // neighbour (the 2-cell halo reaches into the neighbours) or on a side
        // with an inflow segment (whose ghost state changes within the step)
        // computes
        if (tid == 0) {
            s_tg = ctl->t + (a.rk3 == 2 ? 0.5 * ctl->dt : ctl->dt);
        }
        if (tid < NTL) {
            const int t = tid, ty0 = y0 + t * TY, ty = ty0 / TY, gy = (ny + TY - 1) / TY;
            bool keep = false;
            if (ty0 < ny) {
                bool w = false;
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        const int xx = bx + dx, yy = ty + dy;
                        if (xx >= 0 && xx < gx && yy >= 0 && yy < gy) w |= a.tw_prev[yy * gx + xx] != 0;
                    }
                const bool inf = on_inflow_side(a, bx, ty, gx, gy);
                w |= inf;
                if (w) append(bx, ty);
                if (w && a.wbox) box_add(a.wbox, bx, ty);
                a.tw_next[ty * gx + bx] = w;
                keep = keep_tile(a, w, inf, ty * gx + bx, known);
            }
            s_keep[t] = keep;
        }
        __syncthreads();
    } else {
        if (tid == 0) mbar_init(&s_bar, 1);
        __syncthreads();
        if (tid == 0) {
            const bool fixed = a.stage == 1 && a.fix;
            const double t_now = fixed ? a.fix_t : ctl->t;
            const double dt = fixed ? a.fix_dt
                            : a.stage == 1 ? dt_from(ctl, a.ph, __longlong_as_double((long long)ctl->amax)) : ctl->dt;
            s_tg = t_now + (a.rk3 == 2 ? 0.5 * dt : dt);
            if (a.stage == 1 && bx == 0 && sy == 0) first_stage_clock(a, t_now, dt);
            // (a.dbg_stall_tx: bytes no copy delivers, so that the wait below runs out; testing only)
            mbar_expect_tx(&s_bar, rb * (unsigned int)nc + a.dbg_stall_tx);
        }
        // the copies, spread over the threads (the barrier's phase cannot end
        // before thread 0's arrival, whichever comes first)
        for (int k = tid; k < nc; k += blockDim.x) {
            if (k < 2 * nrow) {  // masses of the strip and its halo
                const int p = k & 1, r = k >> 1;
                bulk_g2s(&s_m[p][r][0], a.Uin + 3 * p * plane + cell_index(x0 - 2, y0 - 2 + r, pitch), rb, &s_bar);
            } else {  // own extras
                const int kk = k - 2 * nrow, e = kk % nxp, r = kk / nxp;
                const long long g = cell_index(x0 - 2, y0 + r, pitch);
                const T *src;
                if constexpr (F32) {
                    src = e == 0 ? a.Rin + g : e == 1 ? a.Rin + plane + g : e == 2 ? a.Un + g
                        : e == 3 ? a.Un + 3 * plane + g : e == 4 ? a.Rn + g : a.Rn + plane + g;
                } else {
                    src = e == 0 ? a.Un + g : a.Un + 3 * plane + g;
                }
                bulk_g2s(&s_x[e][r][0], src, rb, &s_bar);
            }
        }
        // every thread waits for the copies (bounded); if any gave up, the CTA
        // reports it, lets the copies in flight land, and stops
        const bool got = mbar_wait(&s_bar, 0, 500000000ull);  // 0.5 s
        if (!__syncthreads_and(got)) {
            if (tid == 0) atomicOr(&ctl->status, (int)STATUS_TIMEOUT);
            mbar_wait(&s_bar, 0, 500000000ull);
            return false;
        }
        if (tid == 0) mbar_inval(&s_bar);  // every thread is past its wait: the CTA may classify another strip
        for (int r = warp; r < H; r += nw) {
            const int gj = y0 + r - 2;  // >= -2
            bool m = false;
            if (gj < ny + 2) {
                const int gi = x0 + lane;  // shared column lane + 2
                if (gi < nx + 2) m |= nonzero(s_m[0][r][lane + 2]) | nonzero(s_m[1][r][lane + 2]);
                if (lane < 4) {  // the halo columns x0-2, x0-1, x0+32, x0+33
                    const int col = lane < 2 ? lane : lane + 32;
                    if (x0 - 2 + col < nx + 2) m |= nonzero(s_m[0][r][col]) | nonzero(s_m[1][r][col]);
                }
                if (r >= 2 && r < S + 2 && gj < ny && gi < nx)  // a cell of the strip: its own extras
                    for (int e = 0; e < nxp; e++) m |= nonzero(s_x[e][r - 2][lane + 2]);
            }
            const unsigned int any = __any_sync(0xffffffffu, m);
            if (lane == 0) s_row[r] = any;
            if (r >= 2 && r < S + 2) {  // the input's own mass, for its mass bits
                bool mo = false;
                if (gj < ny && x0 + lane < nx) {
                    mo = nonzero(s_m[0][r][lane + 2]) | nonzero(s_m[1][r][lane + 2]);
                    if constexpr (F32) mo |= nonzero(s_x[0][r - 2][lane + 2]) | nonzero(s_x[1][r - 2][lane + 2]);
                }
                const unsigned int own = __ballot_sync(0xffffffffu, mo);
                if (lane == 0) s_own[r - 2] = own;
            }
        }
        __syncthreads();
        if (threadIdx.x < NTL) {
            const int t = threadIdx.x, ty0 = y0 + t * TY, ty = ty0 / TY;
            bool keep = false;
            if (ty0 < ny) {
                bool w = false;
                for (int r = t * TY; r < t * TY + TY + 4; r++) w |= s_row[r] != 0u;
                if (w) append(bx, ty);
                if (w && a.wbox) box_add(a.wbox, bx, ty);
                if (a.tw_next) a.tw_next[ty * gx + bx] = w;
                if (a.mb_in && a.stage == 1) a.mb_in[ty * gx + bx] = mass_bits<TY>(&s_own[t * TY]);
                if (a.mb_out && !w) a.mb_out[ty * gx + bx] = 0;
                const bool inf = a.zk != nullptr && on_inflow_side(a, bx, ty, gx, (ny + TY - 1) / TY);
                keep = keep_tile(a, w, inf, ty * gx + bx, known);
            }
            s_keep[t] = keep;
        }
        __syncthreads();
    }
    const T z[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    for (int r = warp; r < S; r += nw) {
        const int j = y0 + r, i = x0 + lane;
        if (j >= ny || s_keep[r / TY] || i >= nx) continue;
        const long long g = cell_index(i, j, pitch);
        store6(a.Uout, plane, g, z);
        if (a.rec) store6(a.rec, plane, g, z);  // the recording form: zero records too
        if constexpr (sizeof(T) == 4) {
            a.Rout[g] = 0.0f;
            a.Rout[plane + g] = 0.0f;
        }
        write_ghosts(a.Uout, a.geo, a, i, j, z, s_tg);
    }
    return true;
}

template <typename T, int TY>
__global__ void __launch_bounds__(32 * kStripWarps, 10) classify_kernel(const StageArgs<T> a)
{
    __shared__ ClassifySmem<T> sm;
    wait_prior_grid();
    classify_strip<T, TY>(a, blockIdx.x, blockIdx.y, gridDim.x, sm,
                          [&](int tx, int ty) { a.wl[atomicAdd(&a.wl_n[0], 1u)] = ty * gridDim.x + tx; });
}

// The classification that reads no state: one thread per tile of the gx x gy
// tiles takes the tile as wet
// - from the mass bits of the input (a.mb_ok): where it has mass within two
//   cells (wet_from_bits) or, in a combining stage, U^n has mass in it;
// - else, in a combining stage (a.tw_prev): where it or a neighbouring tile
//   was wet in the stage before (its input has mass only there);
// and where it lies on a side with an inflow segment (as classify_strip
// does), lists it, and keeps its flags; the CTA's warps then write the zero
// state of its dry tiles that do not hold it yet, one row of 32 cells at a
// time.  Few CTAs with short lives: a CTA per strip made this launch
// latency-bound.  A first stage also takes the step's time step here, as
// the data classification does.
constexpr int kFlagThreads = 256;
template <typename T, int TY>
__global__ void __launch_bounds__(kFlagThreads) classify_flags_kernel(const StageArgs<T> a, const int gx, const int gy)
{
    __shared__ int s_list[kFlagThreads];  // the CTA's tiles to zero-write
    __shared__ unsigned int s_n;
    __shared__ double s_tg;
    wait_prior_grid();
    const int tid = threadIdx.x;
    const int idx = blockIdx.x * kFlagThreads + tid;  // tile (idx % gx, idx / gx)
    const bool mine = idx < gx * gy;
    const unsigned char known = (a.zk && mine) ? a.zk[idx] : 0;
    if (tid == 0) s_n = 0u;
    __syncthreads();
    if (mine) {
        const int bx = idx % gx, ty = idx / gx;
        bool w = false;
        if (a.mb_ok) {
            w = wet_from_bits(a.mb_in, bx, ty, gx, gy);
            if (a.mb_n) w |= (a.mb_n[idx] & MB_ANY) != 0;
            // the adjoint's runs: a combining stage also lists the first
            // stage's wet tiles (its reverse relies on that inclusion)
            if (a.tw_prev) w |= a.tw_prev[idx] != 0;
        } else {
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    const int xx = bx + dx, yy = ty + dy;
                    if (xx >= 0 && xx < gx && yy >= 0 && yy < gy) w |= a.tw_prev[yy * gx + xx] != 0;
                }
        }
        const bool inf = on_inflow_side(a, bx, ty, gx, gy);
        w |= inf;
        if (w) a.wl[atomicAdd(&a.wl_n[0], 1u)] = idx;
        if (w && a.wbox) box_add(a.wbox, bx, ty);
        if (a.tw_next) a.tw_next[idx] = w;
        if (a.mb_out && !w) a.mb_out[idx] = 0;
        if (!keep_tile(a, w, inf, idx, known)) s_list[atomicAdd(&s_n, 1u)] = idx;
    }
    // the step's clock (the control block's reads stay off the tiles' path:
    // only a CTA with tiles to zero-write, and the first CTA of a first
    // stage, wait for them)
    const bool clock = a.stage == 1 && blockIdx.x == 0;
    __syncthreads();
    const int nrows = (int)s_n * TY;
    if (tid == 0 && (nrows > 0 || clock)) {
        const Ctl *ctl = a.ctl;
        if (a.stage == 1) {
            const bool fixed = a.fix != 0;
            const double t_now = fixed ? a.fix_t : ctl->t;
            const double dt = fixed ? a.fix_dt : dt_from(ctl, a.ph, __longlong_as_double((long long)ctl->amax));
            s_tg = t_now + dt;
            if (clock) first_stage_clock(a, t_now, dt);
        } else {
            s_tg = ctl->t + (a.rk3 == 2 ? 0.5 * ctl->dt : ctl->dt);
        }
    }
    if (nrows == 0) return;  // CTA-uniform
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    const T z[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    for (int r = warp; r < nrows; r += kFlagThreads / 32) {
        const int t = s_list[r / TY];
        const int i = (t % gx) * 32 + lane, j = (t / gx) * TY + r % TY;
        if (i >= a.nx || j >= a.ny) continue;
        const long long g = cell_index(i, j, a.pitch);
        store6(a.Uout, a.plane, g, z);
        if (a.rec) store6(a.rec, a.plane, g, z);  // the recording form: zero records too
        if constexpr (sizeof(T) == 4) {
            a.Rout[g] = 0.0f;
            a.Rout[a.plane + g] = 0.0f;
        }
        write_ghosts(a.Uout, a.geo, a, i, j, z, s_tg);
    }
}

// The stage on the listed tiles: a grid of resident CTAs takes the list's
// entries in turn; the last CTA to finish empties the list and, after the
// step's last stage, ends the step.
// FP32: three 256-thread CTAs per SM (at most 85 registers); FP64: two
// P2: two threads per cell (stage_tile), 2 TX TY threads
template <typename T, int TX, int TY, bool REC = false, bool KM = false, bool P2 = false>
__global__ void __launch_bounds__(TX *TY * (P2 ? 2 : 1), (sizeof(T) == 4 ? 768 : 512) / (TX * TY * (P2 ? 2 : 1)))
    stage_kernel_list(const StageArgs<T> a, const int gx)
{
    __shared__ bool last;
    wait_prior_grid();
    const unsigned int n = a.wl_n[0];
    // no barrier between tiles: after the last barrier of a tile only thread 0
    // works (its atomics), and the next tile's shared data are written before
    // that tile's first barrier only by thread 0 or by copies into buffers the
    // previous tile no longer reads
    for (unsigned int w = blockIdx.x; w < n; w += gridDim.x) {
        const int t = a.wl[w];
        stage_tile<T, TX, TY, REC, false, false, false, KM, P2>(a, t % gx, t / gx, 0u);
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&a.wl_n[1], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        a.wl_n[0] = 0;
        a.wl_n[1] = 0;
        if (a.stage == 2 && a.rk3 != 2) end_step(a);
    }
}

}  // namespace moses
