/*
 * oracle.c -- plain, slow FP64 CPU oracle of one explicit time step of the
 * depth-integrated two-phase (solid grains + interstitial fluid) model of
 * MoSES_2PDF (arXiv:2104.06784) over a DEM in terrain-following coordinates.
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file; nothing else may.  It
 * shares no code, header, table or helper with the CUDA library and is never
 * a fallback for it.
 *
 * What it follows (arXiv:2104.06784):
 *   Sect. 2.1          terrain-fitted O_xi,eta,zeta whose xi, eta axes project
 *                      on the DEM's X, Y axes; transformation matrix Omega_b
 *   App. A, Eq. MassEq_TopoS0 / MassEq_TopoF0       mass balances
 *   App. A, Eq. MomentumEqS_Topo / MomentumEqF_Topo  momentum balances
 *   App. A, Eqs. FluxEqSxi_Topo .. FluxEqFeta_Topo  fluxes F, G
 *   App. A, Eqs. Src_nd_Topo, Src_f_Topo, Src_v_Topo             solid sources
 *   App. A, Eqs. SrcF_nd_Topo, SrcF_f_Topo, SrcF_v_Topo, SrcF_vis_Topo  fluid
 *   Sect. 2.2          central (Kurganov-Tadmor) scheme, minmod TVD limiter,
 *                      two-step modified Euler, CFL-limited time step
 *   Sect. 3.1.2        Mode-I release, Mode-II boundary inflow,
 *                      non-reflecting boundaries
 *
 * Built plainly (no -fopenmp) for the tests; the OpenMP pragmas on the loops
 * over rows then do nothing.  A second build with -fopenmp, used only to time
 * the multi-core CPU baseline, runs the same rows on every host core (the
 * clamp sums may then add in another order; nothing else changes).
 *
 * Readings where the paper is silent, ambiguous or garbled (same numbering in
 * the library and the tests):
 *   R1  fluid pressure-gradient source uses phi^s (the reaction of the solid
 *       buoyancy); fluid_pg_mode = 1 keeps the printed phi^f.
 *   R2  xi = X, eta = Y as surface parameters, r = (xi, eta, b);
 *       Omega_b = [d_xi r, d_eta r, n]; J_b = det Omega_b; A = Omega_b^{-1};
 *       derivatives of b by central differences (cell centres) and by the
 *       face-normal difference plus the mean transverse central difference
 *       (faces); 3 ghost layers of b by linear extrapolation.
 *   R3  eps^chi is a parameter; dn/dxi, dn/deta by the chain rule from the
 *       second differences of b; the fluid right-hand side includes s_v^f.
 *   R4  closed = mirror with negated normal momentum; transmissive
 *       (the paper's "no reflection") = zero-gradient copy; 2 ghost layers.
 *   R5  minmod on the conserved variables U; face depth h = U / J_face;
 *       velocity q/U only where U > J h_dry; U1, U4 clamped at 0 (counted);
 *       momentum set to 0 where U <= J h_dry.
 *   R6  semi-implicit Coulomb friction with stopping, direction from the
 *       updated momentum, 3D tangential speed; p_b clamped at 0.
 *   R7  per-phase wave speeds with the other phase frozen.
 *   R8  "two-step modified Euler" = Heun (SSP-RK2), dt frozen over both
 *       stages; dt = CFL min(dx,dy)/a_max, a_max over cell centres.
 *   R9  SI units: g multiplies c = n_Z in every pressure; eps = eps^chi = 1
 *       by default; c_D in 1/s, nu_f in m^2/s, k_f in 1/s.
 *   R10 internal friction (k_mode = 1): the Savage-Hutter earth-pressure
 *       coefficient multiplies the solid pressure in the flux of each
 *       direction and the solid wave speed.  Per cell and direction:
 *       K_pass where the cell and its two neighbours along that axis carry
 *       solid (U1 > J h_dry) and the central difference of the solid
 *       velocity along the axis is negative beyond a dead band of 1e-6 of
 *       the two speeds plus 1e-6 m/s (compression), K_act otherwise;
 *       each side of a face takes its own cell's coefficient.  The CFL wave
 *       speed takes K_pass (the larger).  k_mode = 0: K = 1, the paper's.
 *   R11 inflow ghost state at critical depth for the unit discharge Q/W.
 *   R13 (div_xi + div_eta) summed before it is added to U.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2

#define GS 2 /* ghost layers of the state */
#define GB 3 /* ghost layers of the DEM   */
#define MAX_INFLOW 8

typedef struct {
    double g, eps, eps_chi;
    double rho_s, rho_f;
    double delta_b_deg, phi_int_deg;
    int k_mode;
    double c_d, nu_f, k_f;
    double cfl, dt_max, h_dry;
    int bc[4]; /* W, E, S, N : 0 closed, 1 transmissive */
    int fluid_pg_mode;
    int scheme; /* 0: central flux (Sect. 2.2); 1: central-upwind flux with
                   one-sided local speeds (the cited second-order scheme)   */
    int recon;  /* 0: minmod TVD slopes (Sect. 2.2); 1: third-order WENO     */
    int rk;     /* 2: two-step modified Euler (Sect. 2.2); 3: three-stage
                   strong-stability-preserving Runge-Kutta                  */
} orc_params;

/* geometry of one location (cell centre or face) */
typedef struct {
    double bX, bY;          /* surface slopes d b/dX, d b/dY                 */
    double J;               /* J_b = det Omega_b                             */
    double c;               /* c = n_Z                                       */
    double n[3];            /* unit basal normal n = (n_X, n_Y, n_Z)         */
    double Ai[3][3];        /* (A_ij) = Omega_b^{-1}                         */
    double dn[3][2];        /* d n_k / d xi, d n_k / d eta (cell centres)    */
} orc_geom;

typedef struct {
    int side, i0, i1, npts;
    double *t, *Q, *phi;
} orc_inflow;

typedef struct {
    int nx, ny;
    double dx, dy;
    orc_params p;
    double *b;              /* DEM with GB ghost layers                    */
    orc_geom *gc;           /* cell-centre geometry, GS ghost layers       */
    orc_geom *gfx;          /* x-face (i+1/2, j) geometry, indexed by cell i */
    orc_geom *gfy;          /* y-face (i, j+1/2) geometry, indexed by cell j */
    double *U[6];           /* state with GS ghost layers                   */
    double *W1[6], *W2[6];  /* stage outputs                                */
    double *Hx[6], *Hy[6];  /* face fluxes                                  */
    double *Px, *Py;        /* face values of P = J h pbar^f                */
    double *Vx, *Vy;        /* bracketed viscous terms s_vis,X, s_vis,Y     */
    double t;
    long nsteps;
    double last_dt;
    orc_inflow inflow[MAX_INFLOW];
    int n_inflow;
    /* budgets: time-integrated boundary volume inflow per phase, clamp
       counts and clamp-added volume per phase (Heun weights included)      */
    double bnd_in[2];
    double clamp_vol[2];
    long clamp_cells;
    /* per-stage scratch accumulators */
    double st_bnd[2], st_clamp[2];
    long st_clamp_cells;
} orc_sim;

/* ------------------------------------------------------------------------ */
/* indexing                                                                 */

static inline long IS(const orc_sim *s, int i, int j) /* state / geometry */
{
    return (long)(j + GS) * (s->nx + 2 * GS) + (i + GS);
}
static inline long IBd(const orc_sim *s, int i, int j) /* DEM */
{
    return (long)(j + GB) * (s->nx + 2 * GB) + (i + GB);
}

/* ------------------------------------------------------------------------ */
/* small linear algebra                                                     */

static double det3(const double M[3][3])
{
    return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
         - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
         + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

/* inverse through the adjugate (cofactor transpose) divided by det */
static void inv3(const double M[3][3], double d, double R[3][3])
{
    R[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) / d;
    R[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / d;
    R[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / d;
    R[1][0] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) / d;
    R[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / d;
    R[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / d;
    R[2][0] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) / d;
    R[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / d;
    R[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / d;
}

/* Geometry from the two surface slopes (R2): tangent vectors
   d_xi r = (1, 0, bX), d_eta r = (0, 1, bY); n = their normalised cross
   product; Omega_b has columns [d_xi r, d_eta r, n]. */
static void geom_from_slopes(double bX, double bY, orc_geom *G)
{
    double tx[3] = {1.0, 0.0, bX};
    double ty[3] = {0.0, 1.0, bY};
    double m[3] = {tx[1] * ty[2] - tx[2] * ty[1],
                   tx[2] * ty[0] - tx[0] * ty[2],
                   tx[0] * ty[1] - tx[1] * ty[0]};
    double mm = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    double Om[3][3];
    G->bX = bX;
    G->bY = bY;
    for (int k = 0; k < 3; k++) {
        G->n[k] = m[k] / mm;
        Om[k][0] = tx[k];
        Om[k][1] = ty[k];
        Om[k][2] = G->n[k];
    }
    G->J = det3(Om);
    G->c = G->n[2];
    inv3(Om, G->J, G->Ai);
    for (int k = 0; k < 3; k++) G->dn[k][0] = G->dn[k][1] = 0.0;
}

/* d n / d X of n = m/|m|, m = (-bX, -bY, 1), given dm/dX (chain rule, R3) */
static void dnormal(double bX, double bY, const double dm[3], double out[3])
{
    double m[3] = {-bX, -bY, 1.0};
    double mm2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
    double mm = sqrt(mm2);
    double mdm = m[0] * dm[0] + m[1] * dm[1] + m[2] * dm[2];
    for (int k = 0; k < 3; k++) out[k] = dm[k] / mm - m[k] * mdm / (mm2 * mm);
}

/* ------------------------------------------------------------------------ */
/* geometry pass (once per DEM)                                             */

static void build_geometry(orc_sim *s, const double *dem)
{
    int nx = s->nx, ny = s->ny;
    double dx = s->dx, dy = s->dy;
    /* DEM with 3 ghost layers by linear extrapolation, first in X then Y */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) s->b[IBd(s, i, j)] = dem[(long)j * nx + i];
    for (int j = 0; j < ny; j++) {
        for (int k = 1; k <= GB; k++) {
            double b0 = s->b[IBd(s, 0, j)], b1 = (nx > 1) ? s->b[IBd(s, 1, j)] : b0;
            double e0 = s->b[IBd(s, nx - 1, j)], e1 = (nx > 1) ? s->b[IBd(s, nx - 2, j)] : e0;
            s->b[IBd(s, -k, j)] = b0 + k * (b0 - b1);
            s->b[IBd(s, nx - 1 + k, j)] = e0 + k * (e0 - e1);
        }
    }
    for (int i = -GB; i < nx + GB; i++) {
        for (int k = 1; k <= GB; k++) {
            double b0 = s->b[IBd(s, i, 0)], b1 = (ny > 1) ? s->b[IBd(s, i, 1)] : b0;
            double e0 = s->b[IBd(s, i, ny - 1)], e1 = (ny > 1) ? s->b[IBd(s, i, ny - 2)] : e0;
            s->b[IBd(s, i, -k)] = b0 + k * (b0 - b1);
            s->b[IBd(s, i, ny - 1 + k)] = e0 + k * (e0 - e1);
        }
    }
#define B(i, j) s->b[IBd(s, (i), (j))]
    /* cell centres on [-GS, n+GS) */
    for (int j = -GS; j < ny + GS; j++) {
        for (int i = -GS; i < nx + GS; i++) {
            double bX = (B(i + 1, j) - B(i - 1, j)) / (2.0 * dx);
            double bY = (B(i, j + 1) - B(i, j - 1)) / (2.0 * dy);
            double bXX = (B(i + 1, j) - 2.0 * B(i, j) + B(i - 1, j)) / (dx * dx);
            double bYY = (B(i, j + 1) - 2.0 * B(i, j) + B(i, j - 1)) / (dy * dy);
            double bXY = (B(i + 1, j + 1) - B(i + 1, j - 1) - B(i - 1, j + 1) + B(i - 1, j - 1))
                       / (4.0 * dx * dy);
            orc_geom *G = &s->gc[IS(s, i, j)];
            geom_from_slopes(bX, bY, G);
            /* dm/dX = (-bXX, -bXY, 0), dm/dY = (-bXY, -bYY, 0) */
            double dmx[3] = {-bXX, -bXY, 0.0}, dmy[3] = {-bXY, -bYY, 0.0};
            double o1[3], o2[3];
            dnormal(bX, bY, dmx, o1);
            dnormal(bX, bY, dmy, o2);
            for (int k = 0; k < 3; k++) {
                G->dn[k][0] = o1[k];
                G->dn[k][1] = o2[k];
            }
        }
    }
    /* faces: x-face between (i,j) and (i+1,j) for i in [-GS, nx+GS-1) */
    for (int j = -GS; j < ny + GS; j++) {
        for (int i = -GS; i < nx + GS - 1; i++) {
            double bX = (B(i + 1, j) - B(i, j)) / dx;
            double bY = 0.5 * (s->gc[IS(s, i, j)].bY + s->gc[IS(s, i + 1, j)].bY);
            geom_from_slopes(bX, bY, &s->gfx[IS(s, i, j)]);
        }
    }
    for (int j = -GS; j < ny + GS - 1; j++) {
        for (int i = -GS; i < nx + GS; i++) {
            double bY = (B(i, j + 1) - B(i, j)) / dy;
            double bX = 0.5 * (s->gc[IS(s, i, j)].bX + s->gc[IS(s, i, j + 1)].bX);
            geom_from_slopes(bX, bY, &s->gfy[IS(s, i, j)]);
        }
    }
#undef B
}

/* ------------------------------------------------------------------------ */
/* primitive helpers                                                        */

static inline double alpha_rho(const orc_params *p) { return p->rho_f / p->rho_s; }

/* minmod limiter (Sect. 2.2) on two one-sided undivided differences */
static inline double minmod(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    return (a > 0.0) ? fmin(a, b) : fmax(a, b);
}

/* third-order WENO (Sect. 2.2 names WENO reconstruction as an option) of the
   value at the right face of cell b from the cells a, b, c: the two
   second-order candidates on {a, b} and {b, c}, linear weights 1/3 and 2/3,
   smoothness indicators the squared differences, nonlinear weights
   d_k / (eps + beta_k)^2 with eps = 1e-6 m^2 + 1e-100, m the largest of
   |a|, |b|, |c| (so the weights do not change when U is rescaled)         */
static double weno3_right_face(double a, double b, double c)
{
    double q0 = -0.5 * a + 1.5 * b, q1 = 0.5 * b + 0.5 * c;
    double b0 = (b - a) * (b - a), b1 = (c - b) * (c - b);
    double m = fmax(fabs(a), fmax(fabs(b), fabs(c)));
    double eps = 1e-6 * m * m + 1e-100;
    double a0 = (1.0 / 3.0) / ((eps + b0) * (eps + b0));
    double a1 = (2.0 / 3.0) / ((eps + b1) * (eps + b1));
    return (a0 * q0 + a1 * q1) / (a0 + a1);
}
/* the mirror image: the value at the left face of cell b */
static double weno3_left_face(double a, double b, double c)
{
    return weno3_right_face(c, b, a);
}

/* phase velocity (v_X, v_Y) from its depth J h and momenta (R5) */
static inline void phase_velocity(double Jh, double qX, double qY, double J, double hdry,
                                  double *vX, double *vY)
{
    if (Jh > J * hdry) {
        *vX = qX / Jh;
        *vY = qY / Jh;
    } else {
        *vX = 0.0;
        *vY = 0.0;
    }
}

/* tangential components (v_xi, v_eta) = first two rows of Omega_b^{-1} v,
   with v_Z from tangency to the bed (R2) */
static inline void tangential(const orc_geom *G, double vX, double vY, double *vxi, double *veta)
{
    double vZ = G->bX * vX + G->bY * vY;
    *vxi = G->Ai[0][0] * vX + G->Ai[0][1] * vY + G->Ai[0][2] * vZ;
    *veta = G->Ai[1][0] * vX + G->Ai[1][1] * vY + G->Ai[1][2] * vZ;
}

/* centripetal term kappa = sum_k v_k (dn_k/dxi v_xi + dn_k/deta v_eta) of a
   phase velocity (v_X, v_Y) at a cell centre (App. A, below Eq. Src_nd_Topo
   and Eq. SrcF_nd_Topo), v_Z from tangency */
static double kappa_of(const orc_geom *G, double vX, double vY)
{
    double v[3] = {vX, vY, G->bX * vX + G->bY * vY}, xi, eta, k = 0.0;
    tangential(G, vX, vY, &xi, &eta);
    for (int m = 0; m < 3; m++) k += v[m] * (G->dn[m][0] * xi + G->dn[m][1] * eta);
    return k;
}

/* Savage-Hutter earth-pressure coefficients (R10):
   K_act/pass = 2 sec^2(phi_int) (1 -/+ sqrt(1 - cos^2(phi_int) sec^2(delta_b))) - 1,
   defined for delta_b <= phi_int; both 1 when k_mode = 0 (App. A: the solid
   pressure N^s is the basal one)                                           */
static void earth_pressure(const orc_params *p, double *Ka, double *Kp)
{
    if (p->k_mode != 1) {
        *Ka = *Kp = 1.0;
        return;
    }
    double ph = p->phi_int_deg * M_PI / 180.0, de = p->delta_b_deg * M_PI / 180.0;
    double cp2 = cos(ph) * cos(ph), cd2 = cos(de) * cos(de);
    double r = sqrt(1.0 - cp2 / cd2);
    *Ka = 2.0 / cp2 * (1.0 - r) - 1.0;
    *Kp = 2.0 / cp2 * (1.0 + r) - 1.0;
}

/* K of cell k for direction d (0: xi, 1: eta), its neighbours along that
   axis km (behind) and kp (ahead): K_pass where all three carry solid
   (U1 > J h_dry) and the solid velocity along the axis (v_xi = v_X,
   v_eta = v_Y, R2) is definitely smaller ahead than behind, else K_act */
static double cell_earth_pressure(const orc_sim *s, double *const U[6], long km, long k, long kp, int d,
                                  double Ka, double Kp)
{
    if (s->p.k_mode != 1) return 1.0;
    double hd = s->p.h_dry;
    if (!(U[0][km] > s->gc[km].J * hd) || !(U[0][k] > s->gc[k].J * hd) || !(U[0][kp] > s->gc[kp].J * hd))
        return Ka;
    double vm = U[1 + d][km] / U[0][km], vp = U[1 + d][kp] / U[0][kp];
    /* compression needs a definite sign: a drop of more than 1e-6 of the two
       speeds plus 1e-6 m/s (a cell between two neighbours at rest, or on a
       mirror line, is not compressed by rounding noise) */
    return (vp - vm < -(1e-6 * (fabs(vp) + fabs(vm)) + 1e-6)) ? Kp : Ka;
}

/* ------------------------------------------------------------------------ */
/* physical flux through a face of direction d (0 = xi, 1 = eta) of one
   reconstructed state u (Eqs. FluxEqSxi..FluxEqFeta), the per-phase local
   wave speeds (R7) and P = J_b h pbar^f; K multiplies the solid pressure
   (R10; 1 in the paper's form)                                             */

static void face_flux(const orc_params *p, const orc_geom *G, int d, double K, const double u[6], double F[6],
                      double *as, double *af, double *P, double spd[4])
{
    double J = G->J, c = G->c, al = alpha_rho(p);
    double hs = u[0] / J, hf = u[3] / J, h = hs + hf;
    double vXs, vYs, vXf, vYf, xs, es, xf, ef;
    phase_velocity(u[0], u[1], u[2], J, p->h_dry, &vXs, &vYs);
    phase_velocity(u[3], u[4], u[5], J, p->h_dry, &vXf, &vYf);
    tangential(G, vXs, vYs, &xs, &es);
    tangential(G, vXf, vYf, &xf, &ef);
    double vns = d == 0 ? xs : es;     /* v_xi^s or v_eta^s */
    double vnf = d == 0 ? xf : ef;
    double Ad1 = G->Ai[d][0], Ad2 = G->Ai[d][1];  /* A_11, A_12 or A_21, A_22 */
    double Ns = p->g * c * (1.0 - al) * hs / 2.0; /* depth-averaged solid pressure */
    double pf = p->g * c * h / 2.0;               /* mean fluid pressure            */
    F[0] = J * hs * vns;
    F[1] = J * hs * vXs * vns + p->eps * J * h * Ad1 * (K * Ns);
    F[2] = J * hs * vYs * vns + p->eps * J * h * Ad2 * (K * Ns);
    F[3] = J * hf * vnf;
    F[4] = J * hf * vXf * vnf + p->eps * J * h * Ad1 * pf;
    F[5] = J * hf * vYf * vnf + p->eps * J * h * Ad2 * pf;
    double Add = G->Ai[d][d];
    double cs = sqrt(K * (p->eps * p->g * c * Add * (1.0 - al) * (h + hs) / 2.0));
    double cf = sqrt(p->eps * p->g * c * Add * h);
    *as = fabs(vns) + cs;
    *af = fabs(vnf) + cf;
    *P = J * h * pf;
    if (spd) { /* normal velocities and wave-speed terms, for one-sided speeds */
        spd[0] = vns;
        spd[1] = cs;
        spd[2] = vnf;
        spd[3] = cf;
    }
}

/* numerical flux of one component through a face from the two reconstructed
   sides: the central flux (scheme 0) with the larger local speed a, or the
   central-upwind flux (scheme 1) with one-sided speeds ap >= 0 >= am:
   (ap Fm - am Fp) / (ap - am) + ap am / (ap - am) (up - um), which is the
   mean of Fm and Fp when ap = am = 0 (both sides at rest and dry)           */
static double numerical_flux(int scheme, double Fm, double Fp, double um, double up, double a, double ap,
                             double am)
{
    if (scheme == 0) return 0.5 * (Fm + Fp) - 0.5 * a * (up - um);
    double w = ap - am;
    if (!(w > 0.0)) return 0.5 * (Fm + Fp);
    return (ap * Fm - am * Fp) / w + ap * am / w * (up - um);
}

/* largest cell-centre wave speed over both phases and both directions (R7;
   the solid's with the larger earth-pressure coefficient K_pass, R10)     */
static double cell_speed(const orc_sim *s, int i, int j, double *const U[6])
{
    double u[6], F[6], a[4], P, Ka, Kp;
    long k = IS(s, i, j);
    for (int c = 0; c < 6; c++) u[c] = U[c][k];
    const orc_geom *G = &s->gc[k];
    earth_pressure(&s->p, &Ka, &Kp);
    face_flux(&s->p, G, 0, Kp, u, F, &a[0], &a[1], &P, NULL);
    face_flux(&s->p, G, 1, Kp, u, F, &a[2], &a[3], &P, NULL);
    double m = 0.0;
    for (int c = 0; c < 4; c++) m = fmax(m, a[c]);
    return m;
}

static double max_speed(const orc_sim *s, double *const U[6])
{
    double m = 0.0;
#pragma omp parallel for reduction(max : m)
    for (int j = 0; j < s->ny; j++)
        for (int i = 0; i < s->nx; i++) m = fmax(m, cell_speed(s, i, j, U));
    return m;
}

/* ------------------------------------------------------------------------ */
/* boundary ghosts (R4) and Mode-II inflow (R11)                            */

static double interp_series(const double *t, const double *v, int n, double tt)
{
    if (n <= 0 || tt < t[0] || tt > t[n - 1]) return 0.0;
    for (int k = 0; k < n - 1; k++) {
        if (tt <= t[k + 1]) {
            double w = (t[k + 1] > t[k]) ? (tt - t[k]) / (t[k + 1] - t[k]) : 1.0;
            return v[k] + w * (v[k + 1] - v[k]);
        }
    }
    return v[n - 1];
}

/* ghost state of an inflow cell: critical depth for the unit discharge */
static void inflow_state(const orc_sim *s, const orc_inflow *f, const orc_geom *G, double tt,
                         double u[6])
{
    const orc_params *p = &s->p;
    double W = (f->i1 - f->i0) * ((f->side < 2) ? s->dy : s->dx);
    double Q = interp_series(f->t, f->Q, f->npts, tt);
    double phs = interp_series(f->t, f->phi, f->npts, tt);
    for (int c = 0; c < 6; c++) u[c] = 0.0;
    if (!(Q > 0.0) || W <= 0.0) return;
    double q = Q / W;
    int d = (f->side < 2) ? 0 : 1;
    double Ann = G->Ai[d][d];
    double hc = cbrt(q * q / (G->J * G->J * p->eps * p->g * G->c * Ann));
    double vn = q / (G->J * hc);
    double sgn = (f->side == 0 || f->side == 2) ? 1.0 : -1.0; /* inward */
    u[0] = G->J * hc * phs;
    u[3] = G->J * hc * (1.0 - phs);
    if (d == 0) {
        u[1] = u[0] * sgn * vn;
        u[4] = u[3] * sgn * vn;
    } else {
        u[2] = u[0] * sgn * vn;
        u[5] = u[3] * sgn * vn;
    }
}

static void fill_ghosts(orc_sim *s, double *U[6], double tt)
{
    int nx = s->nx, ny = s->ny;
    /* west / east columns, rows 0..ny-1 */
    for (int j = 0; j < ny; j++) {
        for (int k = 0; k < GS; k++) {
            int gw = -1 - k, ge = nx + k;
            int sw = s->p.bc[0] == 0 ? k : 0;            /* mirror source / copy */
            int se = s->p.bc[1] == 0 ? nx - 1 - k : nx - 1;
            if (sw > nx - 1) sw = nx - 1;
            if (se < 0) se = 0;
            for (int c = 0; c < 6; c++) {
                U[c][IS(s, gw, j)] = U[c][IS(s, sw, j)];
                U[c][IS(s, ge, j)] = U[c][IS(s, se, j)];
            }
            if (s->p.bc[0] == 0) {
                U[1][IS(s, gw, j)] = -U[1][IS(s, gw, j)];
                U[4][IS(s, gw, j)] = -U[4][IS(s, gw, j)];
            }
            if (s->p.bc[1] == 0) {
                U[1][IS(s, ge, j)] = -U[1][IS(s, ge, j)];
                U[4][IS(s, ge, j)] = -U[4][IS(s, ge, j)];
            }
        }
    }
    /* south / north rows over all columns, ghost columns included, so that
       the corners follow the S/N rule applied to the W/E ghosts */
    for (int i = -GS; i < nx + GS; i++) {
        for (int k = 0; k < GS; k++) {
            int gs = -1 - k, gn = ny + k;
            int ss = s->p.bc[2] == 0 ? k : 0;
            int sn = s->p.bc[3] == 0 ? ny - 1 - k : ny - 1;
            if (ss > ny - 1) ss = ny - 1;
            if (sn < 0) sn = 0;
            for (int c = 0; c < 6; c++) {
                U[c][IS(s, i, gs)] = U[c][IS(s, i, ss)];
                U[c][IS(s, i, gn)] = U[c][IS(s, i, sn)];
            }
            if (s->p.bc[2] == 0) {
                U[2][IS(s, i, gs)] = -U[2][IS(s, i, gs)];
                U[5][IS(s, i, gs)] = -U[5][IS(s, i, gs)];
            }
            if (s->p.bc[3] == 0) {
                U[2][IS(s, i, gn)] = -U[2][IS(s, i, gn)];
                U[5][IS(s, i, gn)] = -U[5][IS(s, i, gn)];
            }
        }
    }
    /* inflow segments override the side rule on their cells */
    for (int f = 0; f < s->n_inflow; f++) {
        const orc_inflow *fl = &s->inflow[f];
        for (int a = fl->i0; a < fl->i1; a++) {
            for (int k = 0; k < GS; k++) {
                int gi, gj;
                switch (fl->side) {
                case 0: gi = -1 - k; gj = a; break;
                case 1: gi = nx + k; gj = a; break;
                case 2: gi = a; gj = -1 - k; break;
                default: gi = a; gj = ny + k; break;
                }
                double u[6];
                inflow_state(s, fl, &s->gc[IS(s, gi, gj)], tt, u);
                for (int c = 0; c < 6; c++) U[c][IS(s, gi, gj)] = u[c];
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* viscous term s_vis^f = (eps phi^f / N_R) (s_vis,X, s_vis,Y), nu_f = eps/N_R.
   Face-centred differences: an xi-derivative of a bracket at cell i uses the
   bracket on faces i+-1/2; inside it, d/dxi of a velocity is the face
   difference and d/deta the mean of the two cells' central differences.   */

static double vel_comp(const orc_sim *s, double *U[6], int i, int j, int m)
{
    long k = IS(s, i, j);
    double vX, vY;
    phase_velocity(U[3][k], U[4][k], U[5][k], s->gc[k].J, s->p.h_dry, &vX, &vY);
    double vxi, veta;
    tangential(&s->gc[k], vX, vY, &vxi, &veta);
    return m == 0 ? vxi : veta;
}

static void viscous_terms(orc_sim *s, double *Uin[6])
{
    int nx = s->nx, ny = s->ny;
    const orc_params *p = &s->p;
#pragma omp parallel for
    for (int j = 0; j < ny; j++) {
        for (int i = 0; i < nx; i++) {
            long k = IS(s, i, j);
            double J = s->gc[k].J;
            double hs = Uin[0][k] / J, hf = Uin[3][k] / J, h = hs + hf;
            s->Vx[k] = 0.0;
            s->Vy[k] = 0.0;
            if (!(h > p->h_dry) || !(Uin[3][k] > J * p->h_dry)) continue;
            /* brackets on the four faces; index [side][m] */
            double brX[2][2], brY[2][2];
            /* x-faces i-1/2 (side 0) and i+1/2 (side 1) */
            for (int sd = 0; sd < 2; sd++) {
                int il = i - 1 + sd, ir = i + sd;
                const orc_geom *G = &s->gfx[IS(s, il, j)];
                double Jh = 0.5 * (Uin[0][IS(s, il, j)] + Uin[3][IS(s, il, j)] +
                                   Uin[0][IS(s, ir, j)] + Uin[3][IS(s, ir, j)]);
                double dvx[2], dvy[2];
                for (int m = 0; m < 2; m++) {
                    dvx[m] = (vel_comp(s, Uin, ir, j, m) - vel_comp(s, Uin, il, j, m)) / s->dx;
                    dvy[m] = 0.5 * ((vel_comp(s, Uin, il, j + 1, m) - vel_comp(s, Uin, il, j - 1, m)) +
                                    (vel_comp(s, Uin, ir, j + 1, m) - vel_comp(s, Uin, ir, j - 1, m)))
                           / (2.0 * s->dy);
                }
                double A11 = G->Ai[0][0], A12 = G->Ai[0][1], A21 = G->Ai[1][0], A22 = G->Ai[1][1];
                brX[sd][0] = Jh * (A11 * dvx[0] + A21 * dvy[0]);
                brX[sd][1] = Jh * (A12 * dvx[0] + A22 * dvy[0] + A11 * dvx[1] + A21 * dvy[1]);
            }
            for (int sd = 0; sd < 2; sd++) {
                int jl = j - 1 + sd, jr = j + sd;
                const orc_geom *G = &s->gfy[IS(s, i, jl)];
                double Jh = 0.5 * (Uin[0][IS(s, i, jl)] + Uin[3][IS(s, i, jl)] +
                                   Uin[0][IS(s, i, jr)] + Uin[3][IS(s, i, jr)]);
                double dvx[2], dvy[2];
                for (int m = 0; m < 2; m++) {
                    dvy[m] = (vel_comp(s, Uin, i, jr, m) - vel_comp(s, Uin, i, jl, m)) / s->dy;
                    dvx[m] = 0.5 * ((vel_comp(s, Uin, i + 1, jl, m) - vel_comp(s, Uin, i - 1, jl, m)) +
                                    (vel_comp(s, Uin, i + 1, jr, m) - vel_comp(s, Uin, i - 1, jr, m)))
                           / (2.0 * s->dx);
                }
                double A11 = G->Ai[0][0], A12 = G->Ai[0][1], A21 = G->Ai[1][0], A22 = G->Ai[1][1];
                brY[sd][0] = Jh * (A12 * dvx[0] + A22 * dvy[0] + A11 * dvx[1] + A21 * dvy[1]);
                brY[sd][1] = Jh * (A12 * dvx[1] + A22 * dvy[1]);
            }
            double svX = 2.0 * (brX[1][0] - brX[0][0]) / s->dx + (brY[1][0] - brY[0][0]) / s->dy;
            double svY = 2.0 * (brY[1][1] - brY[0][1]) / s->dy + (brX[1][1] - brX[0][1]) / s->dx;
            s->Vx[k] = svX;
            s->Vy[k] = svY;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* one stage of the semi-discrete scheme: Uout = Uin + dt L(Uin)             */

static void stage(orc_sim *s, double *Uin[6], double *Uout[6], double tt, double dt)
{
    int nx = s->nx, ny = s->ny;
    const orc_params *p = &s->p;
    double al = alpha_rho(p);
    double tanb = tan(p->delta_b_deg * M_PI / 180.0);
    double Ka, Kp;
    earth_pressure(p, &Ka, &Kp);
    fill_ghosts(s, Uin, tt);

    /* x-faces i+1/2 for i = -1 .. nx-1: central flux with minmod slopes */
#pragma omp parallel for
    for (int j = 0; j < ny; j++) {
        for (int i = -1; i < nx; i++) {
            double um[6], up[6], Fm[6], Fp[6], asm_, afm, asp, afp, Pm, Pp;
            for (int c = 0; c < 6; c++) {
                double *V = Uin[c];
                double uL = V[IS(s, i, j)], uR = V[IS(s, i + 1, j)];
                if (p->recon == 0) {
                    double sL = minmod(uL - V[IS(s, i - 1, j)], uR - uL);
                    double sR = minmod(uR - uL, V[IS(s, i + 2, j)] - uR);
                    um[c] = uL + 0.5 * sL;   /* u^- : from the left cell  */
                    up[c] = uR - 0.5 * sR;   /* u^+ : from the right cell */
                } else {
                    um[c] = weno3_right_face(V[IS(s, i - 1, j)], uL, uR);
                    up[c] = weno3_left_face(uL, uR, V[IS(s, i + 2, j)]);
                    if (c == 0 || c == 3) { /* masses stay >= 0 at the faces */
                        um[c] = fmax(um[c], 0.0);
                        up[c] = fmax(up[c], 0.0);
                    }
                }
            }
            const orc_geom *G = &s->gfx[IS(s, i, j)];
            double KL = cell_earth_pressure(s, Uin, IS(s, i - 1, j), IS(s, i, j), IS(s, i + 1, j), 0, Ka, Kp);
            double KR = cell_earth_pressure(s, Uin, IS(s, i, j), IS(s, i + 1, j), IS(s, i + 2, j), 0, Ka, Kp);
            double sm[4], sp[4];
            face_flux(p, G, 0, KL, um, Fm, &asm_, &afm, &Pm, sm);
            face_flux(p, G, 0, KR, up, Fp, &asp, &afp, &Pp, sp);
            double as = fmax(asm_, asp), af = fmax(afm, afp);
            long k = IS(s, i, j);
            for (int c = 0; c < 6; c++) {
                int q = c < 3 ? 0 : 2; /* phase: normal velocity and wave term at spd[q], spd[q+1] */
                double ap = fmax(fmax(sm[q] + sm[q + 1], sp[q] + sp[q + 1]), 0.0);
                double am = fmin(fmin(sm[q] - sm[q + 1], sp[q] - sp[q + 1]), 0.0);
                s->Hx[c][k] = numerical_flux(p->scheme, Fm[c], Fp[c], um[c], up[c], c < 3 ? as : af, ap, am);
            }
            s->Px[k] = 0.5 * (Pm + Pp);
        }
    }
    /* y-faces j+1/2 for j = -1 .. ny-1 */
#pragma omp parallel for
    for (int j = -1; j < ny; j++) {
        for (int i = 0; i < nx; i++) {
            double um[6], up[6], Fm[6], Fp[6], asm_, afm, asp, afp, Pm, Pp;
            for (int c = 0; c < 6; c++) {
                double *V = Uin[c];
                double uL = V[IS(s, i, j)], uR = V[IS(s, i, j + 1)];
                if (p->recon == 0) {
                    double sL = minmod(uL - V[IS(s, i, j - 1)], uR - uL);
                    double sR = minmod(uR - uL, V[IS(s, i, j + 2)] - uR);
                    um[c] = uL + 0.5 * sL;
                    up[c] = uR - 0.5 * sR;
                } else {
                    um[c] = weno3_right_face(V[IS(s, i, j - 1)], uL, uR);
                    up[c] = weno3_left_face(uL, uR, V[IS(s, i, j + 2)]);
                    if (c == 0 || c == 3) {
                        um[c] = fmax(um[c], 0.0);
                        up[c] = fmax(up[c], 0.0);
                    }
                }
            }
            const orc_geom *G = &s->gfy[IS(s, i, j)];
            double KL = cell_earth_pressure(s, Uin, IS(s, i, j - 1), IS(s, i, j), IS(s, i, j + 1), 1, Ka, Kp);
            double KR = cell_earth_pressure(s, Uin, IS(s, i, j), IS(s, i, j + 1), IS(s, i, j + 2), 1, Ka, Kp);
            double sm[4], sp[4];
            face_flux(p, G, 1, KL, um, Fm, &asm_, &afm, &Pm, sm);
            face_flux(p, G, 1, KR, up, Fp, &asp, &afp, &Pp, sp);
            double as = fmax(asm_, asp), af = fmax(afm, afp);
            long k = IS(s, i, j);
            for (int c = 0; c < 6; c++) {
                int q = c < 3 ? 0 : 2;
                double ap = fmax(fmax(sm[q] + sm[q + 1], sp[q] + sp[q + 1]), 0.0);
                double am = fmin(fmin(sm[q] - sm[q + 1], sp[q] - sp[q + 1]), 0.0);
                s->Hy[c][k] = numerical_flux(p->scheme, Fm[c], Fp[c], um[c], up[c], c < 3 ? as : af, ap, am);
            }
            s->Py[k] = 0.5 * (Pm + Pp);
        }
    }

    if (p->nu_f > 0.0) viscous_terms(s, Uin);

    /* boundary volume inflow of this stage (per unit time), per phase */
    double bin[2] = {0.0, 0.0};
    for (int j = 0; j < ny; j++) {
        bin[0] += (s->Hx[0][IS(s, -1, j)] - s->Hx[0][IS(s, nx - 1, j)]) * s->dy;
        bin[1] += (s->Hx[3][IS(s, -1, j)] - s->Hx[3][IS(s, nx - 1, j)]) * s->dy;
    }
    for (int i = 0; i < nx; i++) {
        bin[0] += (s->Hy[0][IS(s, i, -1)] - s->Hy[0][IS(s, i, ny - 1)]) * s->dx;
        bin[1] += (s->Hy[3][IS(s, i, -1)] - s->Hy[3][IS(s, i, ny - 1)]) * s->dx;
    }
    s->st_bnd[0] = bin[0];
    s->st_bnd[1] = bin[1];
    /* clamped volume per phase and clamped cells of this stage */
    double cl_s = 0.0, cl_f = 0.0;
    long cl_n = 0;

    /* cell update with the sources of App. A */
#pragma omp parallel for reduction(+ : cl_s, cl_f, cl_n)
    for (int j = 0; j < ny; j++) {
        for (int i = 0; i < nx; i++) {
            long k = IS(s, i, j);
            const orc_geom *G = &s->gc[k];
            double u[6];
            for (int c = 0; c < 6; c++) u[c] = Uin[c][k];
            double J = G->J, c0 = G->c;
            double hs = u[0] / J, hf = u[3] / J, h = hs + hf;
            double phs = 0.0, phf = 0.0;
            if (h > p->h_dry) {
                phs = hs / h;
                phf = hf / h;
            }
            double vs[2], vf[2];
            phase_velocity(u[0], u[1], u[2], J, p->h_dry, &vs[0], &vs[1]);
            phase_velocity(u[3], u[4], u[5], J, p->h_dry, &vf[0], &vf[1]);
            /* centripetal terms kappa^s, kappa^f */
            double ks = kappa_of(G, vs[0], vs[1]);
            double kf = kappa_of(G, vf[0], vf[1]);
            /* basal pressures (R6: clamped at 0) */
            double pbs = hs * (p->g * c0 * (1.0 - al) - p->eps_chi * ks);
            double pbf = hf * (p->g * c0 - p->eps_chi * kf);
            if (pbs < 0.0) pbs = 0.0;
            if (pbf < 0.0) pbf = 0.0;
            /* gradient of P = J h pbar^f from the face values */
            double dPxi = (s->Px[k] - s->Px[IS(s, i - 1, j)]) / s->dx;
            double dPeta = (s->Py[k] - s->Py[IS(s, i, j - 1)]) / s->dy;
            double gX = G->Ai[0][0] * dPxi + G->Ai[1][0] * dPeta;
            double gY = G->Ai[0][1] * dPxi + G->Ai[1][1] * dPeta;
            double fpg = (p->fluid_pg_mode == 1) ? phf : phs; /* R1 */
            double S[6];
            S[0] = 0.0;
            S[3] = 0.0;
            for (int m = 0; m < 2; m++) {
                double grad = m == 0 ? gX : gY;
                double sn_s = J * pbs * G->n[m];                       /* s_n^s */
                double sf_s = -p->eps * al * phs * grad;              /* s_f^s */
                double sv_s = J * al * p->c_d * phs * phf * h * (vf[m] - vs[m]); /* s_v^s */
                double sn_f = J * pbf * G->n[m];                       /* s_n^f */
                double sf_f = p->eps * fpg * grad;                     /* s_f^f */
                double sv_f = -J * p->c_d * phs * phf * h * (vf[m] - vs[m]); /* s_v^f */
                double sd_f = -J * phf * h * p->k_f * vf[m];           /* s_d^f */
                S[1 + m] = sn_s + sf_s + sv_s;
                S[4 + m] = sn_f + sf_f + sv_f + sd_f;
            }
            /* viscous term s_vis^f (App. A, Eq. SrcF_vis_Topo) */
            if (p->nu_f > 0.0) {
                S[4] += p->nu_f * phf * s->Vx[k];
                S[5] += p->nu_f * phf * s->Vy[k];
            }
            double out[6];
            for (int c = 0; c < 6; c++) {
                double divx = (s->Hx[c][k] - s->Hx[c][IS(s, i - 1, j)]) / s->dx;
                double divy = (s->Hy[c][k] - s->Hy[c][IS(s, i, j - 1)]) / s->dy;
                out[c] = u[c] + dt * (S[c] - (divx + divy));
            }
            /* Coulomb basal friction of the solid with stopping (R6) */
            {
                double qX = out[1], qY = out[2];
                double qZ = G->bX * qX + G->bY * qY;
                double qn = sqrt(qX * qX + qY * qY + qZ * qZ);
                double Fr = dt * J * pbs * tanb;
                if (qn <= Fr) {
                    out[1] = 0.0;
                    out[2] = 0.0;
                } else {
                    double r = 1.0 - Fr / qn;
                    out[1] = qX * r;
                    out[2] = qY * r;
                }
            }
            /* positivity clamp and dry momentum (R5) */
            for (int ph = 0; ph < 2; ph++) {
                int c = 3 * ph;
                if (out[c] < 0.0) {
                    if (ph == 0) cl_s += -out[c] * s->dx * s->dy;
                    else cl_f += -out[c] * s->dx * s->dy;
                    cl_n++;
                    out[c] = 0.0;
                }
                if (out[c] <= J * p->h_dry) {
                    out[c + 1] = 0.0;
                    out[c + 2] = 0.0;
                }
            }
            for (int c = 0; c < 6; c++) Uout[c][k] = out[c];
        }
    }
    s->st_clamp[0] = cl_s;
    s->st_clamp[1] = cl_f;
    s->st_clamp_cells = cl_n;
}


/* ------------------------------------------------------------------------ */
/* one time step (Heun / two-step modified Euler)                           */

static void heun_step(orc_sim *s, double dt)
{
    double t0 = s->t;
    stage(s, s->U, s->W1, t0, dt);
    double b1[2] = {s->st_bnd[0], s->st_bnd[1]};
    double c1[2] = {s->st_clamp[0], s->st_clamp[1]};
    long n1 = s->st_clamp_cells;
    stage(s, s->W1, s->W2, t0 + dt, dt);
    for (int ph = 0; ph < 2; ph++) {
        s->bnd_in[ph] += 0.5 * dt * (b1[ph] + s->st_bnd[ph]);
        s->clamp_vol[ph] += 0.5 * (c1[ph] + s->st_clamp[ph]);
    }
    s->clamp_cells += n1 + s->st_clamp_cells;
#pragma omp parallel for
    for (int j = 0; j < s->ny; j++) {
        for (int i = 0; i < s->nx; i++) {
            long k = IS(s, i, j);
            double J = s->gc[k].J;
            for (int c = 0; c < 6; c++) s->U[c][k] = 0.5 * (s->U[c][k] + s->W2[c][k]);
            for (int ph = 0; ph < 2; ph++) {
                int c = 3 * ph;
                if (s->U[c][k] <= J * s->p.h_dry) {
                    s->U[c + 1][k] = 0.0;
                    s->U[c + 2][k] = 0.0;
                }
            }
        }
    }
    s->t = t0 + dt;
    s->last_dt = dt;
    s->nsteps++;
}

/* dry rule on the combined state (R5) */
static void dry_momentum(orc_sim *s, double *U[6])
{
#pragma omp parallel for
    for (int j = 0; j < s->ny; j++)
        for (int i = 0; i < s->nx; i++) {
            long k = IS(s, i, j);
            double J = s->gc[k].J;
            for (int ph = 0; ph < 2; ph++) {
                int c = 3 * ph;
                if (U[c][k] <= J * s->p.h_dry) {
                    U[c + 1][k] = 0.0;
                    U[c + 2][k] = 0.0;
                }
            }
        }
}

/* three-stage SSP Runge-Kutta step: W1 = S(U) at t; W2 = 3/4 U + 1/4 S(W1)
   at t + dt; U' = 1/3 U + 2/3 S(W2) at t + dt/2 (S = one stage: U + dt L(U)
   with friction, clamp and the dry rule); the dry rule after each
   combination.  Boundary fluxes and clamp volumes enter the budgets with the
   weights 1/6, 1/6, 2/3 with which each stage reaches U'. */
static void rk3_step(orc_sim *s, double dt)
{
    double t0 = s->t, b[3][2], c[3][2];
    long n = 0;
    stage(s, s->U, s->W1, t0, dt);
    for (int ph = 0; ph < 2; ph++) b[0][ph] = s->st_bnd[ph], c[0][ph] = s->st_clamp[ph];
    n += s->st_clamp_cells;
    stage(s, s->W1, s->W2, t0 + dt, dt);
    for (int ph = 0; ph < 2; ph++) b[1][ph] = s->st_bnd[ph], c[1][ph] = s->st_clamp[ph];
    n += s->st_clamp_cells;
    for (int j = 0; j < s->ny; j++)
        for (int i = 0; i < s->nx; i++) {
            long k = IS(s, i, j);
            for (int q = 0; q < 6; q++) s->W1[q][k] = 0.75 * s->U[q][k] + 0.25 * s->W2[q][k];
        }
    dry_momentum(s, s->W1);
    stage(s, s->W1, s->W2, t0 + 0.5 * dt, dt);
    for (int ph = 0; ph < 2; ph++) b[2][ph] = s->st_bnd[ph], c[2][ph] = s->st_clamp[ph];
    n += s->st_clamp_cells;
    for (int j = 0; j < s->ny; j++)
        for (int i = 0; i < s->nx; i++) {
            long k = IS(s, i, j);
            for (int q = 0; q < 6; q++) s->U[q][k] = s->U[q][k] / 3.0 + 2.0 * s->W2[q][k] / 3.0;
        }
    dry_momentum(s, s->U);
    for (int ph = 0; ph < 2; ph++) {
        s->bnd_in[ph] += dt * (b[0][ph] / 6.0 + b[1][ph] / 6.0 + 2.0 * b[2][ph] / 3.0);
        s->clamp_vol[ph] += c[0][ph] / 6.0 + c[1][ph] / 6.0 + 2.0 * c[2][ph] / 3.0;
    }
    s->clamp_cells += n;
    s->t = t0 + dt;
    s->last_dt = dt;
    s->nsteps++;
}

static void time_step(orc_sim *s, double dt)
{
    if (s->p.rk == 3) rk3_step(s, dt);
    else heun_step(s, dt);
}

static double cfl_dt(const orc_sim *s, double amax)
{
    double dmin = s->dx < s->dy ? s->dx : s->dy;
    double dt = (amax > 0.0) ? s->p.cfl * dmin / amax : s->p.dt_max;
    if (dt > s->p.dt_max) dt = s->p.dt_max;
    return dt;
}

/* ------------------------------------------------------------------------ */
/* public API (ctypes)                                                      */

static void free_sim(orc_sim *s)
{
    if (!s) return;
    free(s->b);
    free(s->gc);
    free(s->gfx);
    free(s->gfy);
    for (int c = 0; c < 6; c++) {
        free(s->U[c]);
        free(s->W1[c]);
        free(s->W2[c]);
        free(s->Hx[c]);
        free(s->Hy[c]);
    }
    free(s->Px);
    free(s->Py);
    free(s->Vx);
    free(s->Vy);
    for (int f = 0; f < s->n_inflow; f++) {
        free(s->inflow[f].t);
        free(s->inflow[f].Q);
        free(s->inflow[f].phi);
    }
    free(s);
}

int orc_create(const double *dem, int nx, int ny, double dx, double dy, const orc_params *p,
               orc_sim **out)
{
    *out = NULL;
    if (!dem || !p || nx < 1 || ny < 1 || !(dx > 0.0) || !(dy > 0.0)) return ORC_EINVAL;
    if (p->k_mode != 0 && p->k_mode != 1) return ORC_EINVAL;
    /* the Savage-Hutter coefficients need delta_b <= phi_int < 90 deg */
    if (p->k_mode == 1 && !(p->delta_b_deg <= p->phi_int_deg && p->phi_int_deg < 90.0)) return ORC_EINVAL;
    if (p->scheme != 0 && p->scheme != 1) return ORC_EINVAL;
    if ((p->recon != 0 && p->recon != 1) || (p->rk != 2 && p->rk != 3)) return ORC_EINVAL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!s) return ORC_ENOMEM;
    s->nx = nx;
    s->ny = ny;
    s->dx = dx;
    s->dy = dy;
    s->p = *p;
    long ns = (long)(nx + 2 * GS) * (ny + 2 * GS);
    long nb = (long)(nx + 2 * GB) * (ny + 2 * GB);
    s->b = (double *)calloc(nb, sizeof(double));
    s->gc = (orc_geom *)calloc(ns, sizeof(orc_geom));
    s->gfx = (orc_geom *)calloc(ns, sizeof(orc_geom));
    s->gfy = (orc_geom *)calloc(ns, sizeof(orc_geom));
    s->Px = (double *)calloc(ns, sizeof(double));
    s->Py = (double *)calloc(ns, sizeof(double));
    s->Vx = (double *)calloc(ns, sizeof(double));
    s->Vy = (double *)calloc(ns, sizeof(double));
    int ok = s->b && s->gc && s->gfx && s->gfy && s->Px && s->Py && s->Vx && s->Vy;
    for (int c = 0; c < 6; c++) {
        s->U[c] = (double *)calloc(ns, sizeof(double));
        s->W1[c] = (double *)calloc(ns, sizeof(double));
        s->W2[c] = (double *)calloc(ns, sizeof(double));
        s->Hx[c] = (double *)calloc(ns, sizeof(double));
        s->Hy[c] = (double *)calloc(ns, sizeof(double));
        ok = ok && s->U[c] && s->W1[c] && s->W2[c] && s->Hx[c] && s->Hy[c];
    }
    if (!ok) {
        free_sim(s);
        return ORC_ENOMEM;
    }
    build_geometry(s, dem);
    *out = s;
    return ORC_OK;
}

void orc_destroy(orc_sim *s) { free_sim(s); }

/* U: 6 planes of ny*nx, row-major [c][j][i] */
int orc_set_U(orc_sim *s, const double *U)
{
    long n = (long)s->nx * s->ny;
    for (int c = 0; c < 6; c++)
        for (int j = 0; j < s->ny; j++)
            for (int i = 0; i < s->nx; i++) s->U[c][IS(s, i, j)] = U[c * n + (long)j * s->nx + i];
    return ORC_OK;
}

int orc_get_U(const orc_sim *s, double *U)
{
    long n = (long)s->nx * s->ny;
    for (int c = 0; c < 6; c++)
        for (int j = 0; j < s->ny; j++)
            for (int i = 0; i < s->nx; i++) U[c * n + (long)j * s->nx + i] = s->U[c][IS(s, i, j)];
    return ORC_OK;
}

/* Mode-I release: normal thickness h, solid fraction phi_s, phase velocities
   (horizontal-projection components); NULL velocity = 0. */
int orc_set_release(orc_sim *s, const double *h, const double *phi_s, const double *vxs,
                    const double *vys, const double *vxf, const double *vyf)
{
    if (!h || !phi_s) return ORC_EINVAL;
    for (int j = 0; j < s->ny; j++) {
        for (int i = 0; i < s->nx; i++) {
            long q = (long)j * s->nx + i, k = IS(s, i, j);
            double J = s->gc[k].J;
            double U1 = J * h[q] * phi_s[q], U4 = J * h[q] * (1.0 - phi_s[q]);
            s->U[0][k] = U1;
            s->U[1][k] = vxs ? U1 * vxs[q] : 0.0;
            s->U[2][k] = vys ? U1 * vys[q] : 0.0;
            s->U[3][k] = U4;
            s->U[4][k] = vxf ? U4 * vxf[q] : 0.0;
            s->U[5][k] = vyf ? U4 * vyf[q] : 0.0;
        }
    }
    return ORC_OK;
}

int orc_set_inflow(orc_sim *s, int side, int i0, int i1, int npts, const double *t, const double *Q,
                   const double *phi)
{
    if (s->n_inflow >= MAX_INFLOW || side < 0 || side > 3 || npts < 1) return ORC_EINVAL;
    int len = side < 2 ? s->ny : s->nx;
    if (i0 < 0 || i1 > len || i1 <= i0) return ORC_EINVAL;
    orc_inflow *f = &s->inflow[s->n_inflow];
    f->side = side;
    f->i0 = i0;
    f->i1 = i1;
    f->npts = npts;
    f->t = (double *)malloc(npts * sizeof(double));
    f->Q = (double *)malloc(npts * sizeof(double));
    f->phi = (double *)malloc(npts * sizeof(double));
    if (!f->t || !f->Q || !f->phi) return ORC_ENOMEM;
    memcpy(f->t, t, npts * sizeof(double));
    memcpy(f->Q, Q, npts * sizeof(double));
    memcpy(f->phi, phi, npts * sizeof(double));
    s->n_inflow++;
    return ORC_OK;
}

void orc_set_time(orc_sim *s, double t) { s->t = t; }
double orc_get_time(const orc_sim *s) { return s->t; }
double orc_last_dt(const orc_sim *s) { return s->last_dt; }

double orc_max_speed(orc_sim *s) { return max_speed(s, s->U); }

/* the largest cell speed over rows [j0, j1) (a strip's own rows) */
double orc_max_speed_rows(orc_sim *s, int j0, int j1)
{
    double m = 0.0;
    for (int j = j0 < 0 ? 0 : j0; j < j1 && j < s->ny; j++)
        for (int i = 0; i < s->nx; i++) m = fmax(m, cell_speed(s, i, j, s->U));
    return m;
}

double orc_cfl_dt(orc_sim *s) { return cfl_dt(s, max_speed(s, s->U)); }

/* n CFL-limited steps; dts (optional, n entries) receives the time steps */
int orc_step(orc_sim *s, int n, double *dts)
{
    for (int k = 0; k < n; k++) {
        double dt = cfl_dt(s, max_speed(s, s->U));
        time_step(s, dt);
        if (dts) dts[k] = dt;
    }
    return ORC_OK;
}

/* one step whose CFL time step comes from the given largest wave speed
   instead of this simulation's own: a strip of a row-decomposed domain
   steps with the largest speed of all strips (the whole domain's a_max,
   Sect. 2.2), so that every strip takes the undecomposed step.  Returns the
   time step. */
double orc_step_amax(orc_sim *s, double amax)
{
    double dt = cfl_dt(s, amax);
    time_step(s, dt);
    return dt;
}

/* one Heun step with a prescribed time step */
int orc_step_dt(orc_sim *s, double dt)
{
    time_step(s, dt);
    return ORC_OK;
}

/* one stage from the current state: Uout (6 planes ny*nx) = U + dt L(U) at
   time tt, friction, clamp and dry-momentum rule included.  The state is
   left unchanged. */
int orc_stage(orc_sim *s, double tt, double dt, double *Uout)
{
    stage(s, s->U, s->W1, tt, dt);
    long n = (long)s->nx * s->ny;
    for (int c = 0; c < 6; c++)
        for (int j = 0; j < s->ny; j++)
            for (int i = 0; i < s->nx; i++) Uout[c * n + (long)j * s->nx + i] = s->W1[c][IS(s, i, j)];
    return ORC_OK;
}

/* budgets: out[0..1] volume of solid / fluid (sum U ΔxΔy), out[2..5]
   momenta sum(U2,U3,U5,U6) ΔxΔy, out[6..7] time-integrated boundary volume
   inflow per phase, out[8..9] clamp-added volume per phase, out[10] clamp
   cell count, out[11] t, out[12] steps */
int orc_budget(const orc_sim *s, double *out)
{
    double sum[6] = {0, 0, 0, 0, 0, 0};
    for (int j = 0; j < s->ny; j++)
        for (int i = 0; i < s->nx; i++)
            for (int c = 0; c < 6; c++) sum[c] += s->U[c][IS(s, i, j)];
    double a = s->dx * s->dy;
    out[0] = sum[0] * a;
    out[1] = sum[3] * a;
    out[2] = sum[1] * a;
    out[3] = sum[2] * a;
    out[4] = sum[4] * a;
    out[5] = sum[5] * a;
    out[6] = s->bnd_in[0];
    out[7] = s->bnd_in[1];
    out[8] = s->clamp_vol[0];
    out[9] = s->clamp_vol[1];
    out[10] = (double)s->clamp_cells;
    out[11] = s->t;
    out[12] = (double)s->nsteps;
    return ORC_OK;
}

/* geometry export on the interior: 14 planes ny*nx:
   J, c, nX, nY, nZ, A11, A12, A21, A22, dnX/dxi, dnY/dxi, dnZ/dxi,
   dnX/deta, dnY/deta (dnZ/deta as plane 14) -> 15 planes */
int orc_geometry(const orc_sim *s, double *out)
{
    long n = (long)s->nx * s->ny;
    for (int j = 0; j < s->ny; j++) {
        for (int i = 0; i < s->nx; i++) {
            const orc_geom *G = &s->gc[IS(s, i, j)];
            long q = (long)j * s->nx + i;
            double v[15] = {G->J, G->c, G->n[0], G->n[1], G->n[2], G->Ai[0][0], G->Ai[0][1],
                            G->Ai[1][0], G->Ai[1][1], G->dn[0][0], G->dn[1][0], G->dn[2][0],
                            G->dn[0][1], G->dn[1][1], G->dn[2][1]};
            for (int c = 0; c < 15; c++) out[c * n + q] = v[c];
        }
    }
    return ORC_OK;
}

/* curvature term kappa of one phase velocity (v_X, v_Y) at cell (i, j), for
   the pins on curved beds */
double orc_kappa(const orc_sim *s, int i, int j, double vX, double vY)
{
    return kappa_of(&s->gc[IS(s, i, j)], vX, vY);
}

/* tangential components of (vX, vY) at cell (i, j) */
void orc_tangential(const orc_sim *s, int i, int j, double vX, double vY, double *out2)
{
    tangential(&s->gc[IS(s, i, j)], vX, vY, &out2[0], &out2[1]);
}

/* ghost state of inflow segment f at ghost cell (gi, gj) and time tt, for
   the pins of the Mode-II boundary (R11) */
int orc_inflow_state(const orc_sim *s, int f, int gi, int gj, double tt, double *u)
{
    if (f < 0 || f >= s->n_inflow) return ORC_EINVAL;
    inflow_state(s, &s->inflow[f], &s->gc[IS(s, gi, gj)], tt, u);
    return ORC_OK;
}

/* geometry of ghost or interior cell (gi, gj): J, c, A11, A22 */
int orc_cell_geom(const orc_sim *s, int gi, int gj, double *out4)
{
    if (gi < -GS || gj < -GS || gi >= s->nx + GS || gj >= s->ny + GS) return ORC_EINVAL;
    const orc_geom *G = &s->gc[IS(s, gi, gj)];
    out4[0] = G->J;
    out4[1] = G->c;
    out4[2] = G->Ai[0][0];
    out4[3] = G->Ai[1][1];
    return ORC_OK;
}

/* the earth-pressure coefficients K_act, K_pass of a parameter set (R10) */
void orc_earth_pressure(const orc_params *p, double *out2)
{
    earth_pressure(p, &out2[0], &out2[1]);
}
