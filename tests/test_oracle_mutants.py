"""Planted mistakes in the oracle must be caught by its pins.

Each case copies ``oracle/oracle.c`` to a temporary directory, plants one
plausible mistake (a dropped term, a wrong sign, index or factor, a transposed
operand), compiles it on the CPU and runs the pins of ``oracle_pins`` against
it.  At least one pin must fail, which shows the pins constrain that part of
the oracle.  Nothing here touches a GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import tempfile

import pytest

from oracle import oracle as O
from tests import oracle_pins as P

SRC = os.path.join(os.path.dirname(O.__file__), "oracle.c")

# (what the mistake is, text in oracle.c, replacement)
MUTANTS = [
    ("solid buoyancy dropped (Eq. Src_f_Topo)",
     "double sf_s = -p->eps * al * phs * grad;", "double sf_s = 0.0 * grad;"),
    ("fluid pressure-gradient source as printed, phi^f (R1 undone)",
     "double fpg = (p->fluid_pg_mode == 1) ? phf : phs;", "double fpg = phf;"),
    ("A_11 dropped from the solid pressure flux",
     "F[1] = J * hs * vXs * vns + p->eps * J * h * Ad1 * (K * Ns);", "F[1] = J * hs * vXs * vns + p->eps * J * h * (K * Ns);"),
    ("c dropped from the mean fluid pressure",
     "double pf = p->g * c * h / 2.0;", "double pf = p->g * h / 2.0;"),
    ("(1 - alpha) dropped from the solid pressure",
     "double Ns = p->g * c * (1.0 - al) * hs / 2.0;", "double Ns = p->g * c * hs / 2.0;"),
    ("KT numerical diffusion with the wrong sign",
     "return 0.5 * (Fm + Fp) - 0.5 * a * (up - um);", "return 0.5 * (Fm + Fp) + 0.5 * a * (up - um);"),
    ("WENO: the downwind candidate replaced by the cell value",
     "double q0 = -0.5 * a + 1.5 * b, q1 = 0.5 * b + 0.5 * c;", "double q0 = -0.5 * a + 1.5 * b, q1 = b;"),
    ("WENO: equal linear weights instead of 1/3, 2/3",
     "double a0 = (1.0 / 3.0) / ((eps + b0) * (eps + b0));", "double a0 = (2.0 / 3.0) / ((eps + b0) * (eps + b0));"),
    ("WENO: smoothness indicator of the wrong stencil",
     "double b0 = (b - a) * (b - a), b1 = (c - b) * (c - b);", "double b0 = (c - b) * (c - b), b1 = (b - a) * (b - a);"),
    ("RK3: second combination with Heun weights",
     "s->W1[q][k] = 0.75 * s->U[q][k] + 0.25 * s->W2[q][k];", "s->W1[q][k] = 0.5 * s->U[q][k] + 0.5 * s->W2[q][k];"),
    ("RK3: boundary fluxes with equal stage weights",
     "s->bnd_in[ph] += dt * (b[0][ph] / 6.0 + b[1][ph] / 6.0 + 2.0 * b[2][ph] / 3.0);",
     "s->bnd_in[ph] += dt * (b[0][ph] + b[1][ph] + b[2][ph]) / 3.0;"),
    ("central-upwind diffusion term with the wrong sign",
     "return (ap * Fm - am * Fp) / w + ap * am / w * (up - um);",
     "return (ap * Fm - am * Fp) / w - ap * am / w * (up - um);"),
    ("central-upwind with the one-sided speeds swapped between the two sides",
     "return (ap * Fm - am * Fp) / w + ap * am / w * (up - um);",
     "return (ap * Fp - am * Fm) / w + ap * am / w * (up - um);"),
    ("central-upwind left speed without the wave term",
     "double am = fmin(fmin(sm[q] - sm[q + 1], sp[q] - sp[q + 1]), 0.0);",
     "double am = fmin(fmin(sm[q], sp[q]), 0.0);"),
    ("maxmod instead of minmod",
     "return (a > 0.0) ? fmin(a, b) : fmax(a, b);", "return (a > 0.0) ? fmax(a, b) : fmin(a, b);"),
    ("slopes not halved at the faces",
     "um[c] = uL + 0.5 * sL;", "um[c] = uL + sL;"),
    ("Heun average replaced by the second stage",
     "s->U[c][k] = 0.5 * (s->U[c][k] + s->W2[c][k]);", "s->U[c][k] = s->W2[c][k];"),
    ("solid drag with the wrong sign",
     "double sv_s = J * al * p->c_d * phs * phf * h * (vf[m] - vs[m]);",
     "double sv_s = J * al * p->c_d * phs * phf * h * (vs[m] - vf[m]);"),
    ("alpha_rho dropped from the solid drag",
     "double sv_s = J * al * p->c_d * phs * phf * h * (vf[m] - vs[m]);",
     "double sv_s = J * p->c_d * phs * phf * h * (vf[m] - vs[m]);"),
    ("fluid basal friction with the wrong sign",
     "double sd_f = -J * phf * h * p->k_f * vf[m];", "double sd_f = J * phf * h * p->k_f * vf[m];"),
    ("kappa without the v_Z term",
     "for (int m = 0; m < 3; m++) k += v[m] * (G->dn[m][0] * xi + G->dn[m][1] * eta);",
     "for (int m = 0; m < 2; m++) k += v[m] * (G->dn[m][0] * xi + G->dn[m][1] * eta);"),
    ("kappa added to the basal pressure instead of subtracted",
     "double pbs = hs * (p->g * c0 * (1.0 - al) - p->eps_chi * ks);",
     "double pbs = hs * (p->g * c0 * (1.0 - al) + p->eps_chi * ks);"),
    ("lift-off clamp of p_b removed",
     "if (pbs < 0.0) pbs = 0.0;", "if (pbs < -1e300) pbs = 0.0;"),
    ("chain-rule term of dn/dX dropped",
     "out[k] = dm[k] / mm - m[k] * mdm / (mm2 * mm);", "out[k] = dm[k] / mm;"),
    ("Omega_b^-1 entry transposed",
     "R[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / d;",
     "R[0][2] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) / d;"),
    ("central slope over dx instead of 2 dx",
     "double bX = (B(i + 1, j) - B(i - 1, j)) / (2.0 * dx);", "double bX = (B(i + 1, j) - B(i - 1, j)) / dx;"),
    ("face slope over 2 dx",
     "double bX = (B(i + 1, j) - B(i, j)) / dx;", "double bX = (B(i + 1, j) - B(i, j)) / (2.0 * dx);"),
    ("friction without tan(delta_b)",
     "double Fr = dt * J * pbs * tanb;", "double Fr = dt * J * pbs;"),
    ("friction without J_b",
     "double Fr = dt * J * pbs * tanb;", "double Fr = dt * pbs * tanb;"),
    ("friction speed without v_Z",
     "double qn = sqrt(qX * qX + qY * qY + qZ * qZ);", "double qn = sqrt(qX * qX + qY * qY);"),
    ("west wall keeps its normal momentum",
     "U[1][IS(s, gw, j)] = -U[1][IS(s, gw, j)];", "U[1][IS(s, gw, j)] = U[1][IS(s, gw, j)];"),
    ("north wall keeps its normal momentum",
     "U[2][IS(s, i, gn)] = -U[2][IS(s, i, gn)];", "U[2][IS(s, i, gn)] = U[2][IS(s, i, gn)];"),
    ("time step proportional to the wave speed",
     "double dt = (amax > 0.0) ? s->p.cfl * dmin / amax : s->p.dt_max;",
     "double dt = (amax > 0.0) ? s->p.cfl * dmin * amax : s->p.dt_max;"),
    ("solid celerity without the 1/2",
     "(1.0 - al) * (h + hs) / 2.0));", "(1.0 - al) * (h + hs)));"),
    ("inflow depth with a square root instead of a cube root",
     "double hc = cbrt(q * q / (G->J * G->J * p->eps * p->g * G->c * Ann));",
     "double hc = sqrt(q * q / (G->J * G->J * p->eps * p->g * G->c * Ann));"),
    ("boundary budget read on the first interior face",
     "bin[0] += (s->Hx[0][IS(s, -1, j)] - s->Hx[0][IS(s, nx - 1, j)]) * s->dy;",
     "bin[0] += (s->Hx[0][IS(s, 0, j)] - s->Hx[0][IS(s, nx - 1, j)]) * s->dy;"),
    ("viscous stretch term without its factor 2",
     "double svX = 2.0 * (brX[1][0] - brX[0][0]) / s->dx", "double svX = 1.0 * (brX[1][0] - brX[0][0]) / s->dx"),
    ("viscous shear bracket with A_22 dropped",
     "brY[sd][0] = Jh * (A12 * dvx[0] + A22 * dvy[0] + A11 * dvx[1] + A21 * dvy[1]);",
     "brY[sd][0] = Jh * (A12 * dvx[0] + A11 * dvx[1] + A21 * dvy[1]);"),
    ("pressure-gradient difference over the wrong face",
     "double dPxi = (s->Px[k] - s->Px[IS(s, i - 1, j)]) / s->dx;",
     "double dPxi = (s->Px[k] - s->Px[IS(s, i, j)]) / s->dx;"),
    ("mass flux uses v_eta on xi faces",
     "double vns = d == 0 ? xs : es;", "double vns = es;"),
    ("dry momentum rule dropped from the stage output (R5)",
     "                if (out[c] <= J * p->h_dry) {", "                if (0 && out[c] <= J * p->h_dry) {"),
    ("inflow solid fraction given to the fluid",
     "u[0] = G->J * hc * phs;\n    u[3] = G->J * hc * (1.0 - phs);",
     "u[0] = G->J * hc * (1.0 - phs);\n    u[3] = G->J * hc * phs;"),
    ("inflow on the east and north sides pointing out of the domain",
     "double sgn = (f->side == 0 || f->side == 2) ? 1.0 : -1.0;", "double sgn = 1.0;"),
    ("inflow width from the wrong cell side",
     "double W = (f->i1 - f->i0) * ((f->side < 2) ? s->dy : s->dx);",
     "double W = (f->i1 - f->i0) * ((f->side < 2) ? s->dx : s->dy);"),
    ("transmissive west ghost copies the second cell",
     "int sw = s->p.bc[0] == 0 ? k : 0;", "int sw = s->p.bc[0] == 0 ? k : 1;"),
    ("time step not capped at dt_max",
     "if (dt > s->p.dt_max) dt = s->p.dt_max;", ""),
    ("clamp volume counted with the wrong sign",
     "if (ph == 0) cl_s += -out[c] * s->dx * s->dy;\n                    else cl_f += -out[c] * s->dx * s->dy;",
     "if (ph == 0) cl_s += out[c] * s->dx * s->dy;\n                    else cl_f += out[c] * s->dx * s->dy;"),
    ("positivity clamp removed",
     "if (out[c] < 0.0) {", "if (0 && out[c] < 0.0) {"),
    ("Heun second stage's boundary data at the start time",
     "stage(s, s->W1, s->W2, t0 + dt, dt);", "stage(s, s->W1, s->W2, t0, dt);"),
    ("RK3 third stage's boundary data at t + dt instead of t + dt/2",
     "stage(s, s->W1, s->W2, t0 + 0.5 * dt, dt);", "stage(s, s->W1, s->W2, t0 + dt, dt);"),
    ("south / north boundary budget over dy",
     "bin[0] += (s->Hy[0][IS(s, i, -1)] - s->Hy[0][IS(s, i, ny - 1)]) * s->dx;",
     "bin[0] += (s->Hy[0][IS(s, i, -1)] - s->Hy[0][IS(s, i, ny - 1)]) * s->dy;"),
    ("boundary budget misses the east side",
     "bin[0] += (s->Hx[0][IS(s, -1, j)] - s->Hx[0][IS(s, nx - 1, j)]) * s->dy;",
     "bin[0] += s->Hx[0][IS(s, -1, j)] * s->dy;"),
    ("eta divergence over dx",
     "double divy = (s->Hy[c][k] - s->Hy[c][IS(s, i, j - 1)]) / s->dy;",
     "double divy = (s->Hy[c][k] - s->Hy[c][IS(s, i, j - 1)]) / s->dx;"),
    ("dP/deta over dx",
     "double dPeta = (s->Py[k] - s->Py[IS(s, i, j - 1)]) / s->dy;",
     "double dPeta = (s->Py[k] - s->Py[IS(s, i, j - 1)]) / s->dx;"),
    ("cell slope b_Y over 2 dx",
     "double bY = (B(i, j + 1) - B(i, j - 1)) / (2.0 * dy);", "double bY = (B(i, j + 1) - B(i, j - 1)) / (2.0 * dx);"),
    ("y-face slope over dx",
     "double bY = (B(i, j + 1) - B(i, j)) / dy;", "double bY = (B(i, j + 1) - B(i, j)) / dx;"),
    ("viscous X bracket without its A_21 term",
     "brX[sd][0] = Jh * (A11 * dvx[0] + A21 * dvy[0]);", "brX[sd][0] = Jh * (A11 * dvx[0]);"),
    ("viscous cross derivative on y-faces over dy",
     "                           / (2.0 * s->dx);\n                }\n                double A11 = G->Ai[0][0], A12 = G->Ai[0][1], A21 = G->Ai[1][0], A22 = G->Ai[1][1];\n                brY",
     "                           / (2.0 * s->dy);\n                }\n                double A11 = G->Ai[0][0], A12 = G->Ai[0][1], A21 = G->Ai[1][0], A22 = G->Ai[1][1];\n                brY"),
    ("viscous x-face depth from the left cell only",
     "double Jh = 0.5 * (Uin[0][IS(s, il, j)] + Uin[3][IS(s, il, j)] +\n                                   Uin[0][IS(s, ir, j)] + Uin[3][IS(s, ir, j)]);",
     "double Jh = (Uin[0][IS(s, il, j)] + Uin[3][IS(s, il, j)]);"),
    ("fluid pressure-gradient source without eps",
     "double sf_f = p->eps * fpg * grad;", "double sf_f = fpg * grad;"),
    ("RK3 dry rule after the first combination dropped",
     "    dry_momentum(s, s->W1);\n", "\n"),
    ("a_max skips the last column",
     "for (int i = 0; i < s->nx; i++) m = fmax(m, cell_speed(s, i, j, U));",
     "for (int i = 0; i < s->nx - 1; i++) m = fmax(m, cell_speed(s, i, j, U));"),
    ("solid celerity without (1 - alpha)",
     "double cs = sqrt(K * (p->eps * p->g * c * Add * (1.0 - al) * (h + hs) / 2.0));",
     "double cs = sqrt(K * (p->eps * p->g * c * Add * (h + hs) / 2.0));"),
    ("solid basal pressure without (1 - alpha)",
     "double pbs = hs * (p->g * c0 * (1.0 - al) - p->eps_chi * ks);", "double pbs = hs * (p->g * c0 - p->eps_chi * ks);"),
    ("kappa of the fluid from the solid velocity",
     "double kf = kappa_of(G, vf[0], vf[1]);", "double kf = kappa_of(G, vs[0], vs[1]);"),
    ("fluid basal pressure not clamped at 0",
     "if (pbf < 0.0) pbf = 0.0;", ""),
    ("inflow solid fraction held at the hydrograph's first point",
     "double phs = interp_series(f->t, f->phi, f->npts, tt);", "double phs = f->phi[0];"),
    ("west inflow fills its first ghost layer twice and not the second",
     "case 0: gi = -1 - k; gj = a; break;", "case 0: gi = -1; gj = a; break;"),
    ("corner ghosts left unfilled",
     "for (int i = -GS; i < nx + GS; i++) {\n        for (int k = 0; k < GS; k++) {\n            int gs = -1 - k, gn = ny + k;",
     "for (int i = 0; i < nx; i++) {\n        for (int k = 0; k < GS; k++) {\n            int gs = -1 - k, gn = ny + k;"),
    ("dry threshold of the phase velocity on U instead of the normal thickness",
     "if (Jh > J * hdry) {", "if (Jh > hdry) {"),
    ("Heun step drops the first stage's clamp-cell count",
     "s->clamp_cells += n1 + s->st_clamp_cells;", "s->clamp_cells += s->st_clamp_cells;"),
    ("RK3 clamp volume with equal stage weights",
     "s->clamp_vol[ph] += c[0][ph] / 6.0 + c[1][ph] / 6.0 + 2.0 * c[2][ph] / 3.0;",
     "s->clamp_vol[ph] += (c[0][ph] + c[1][ph] + c[2][ph]) / 3.0;"),
    ("hydrograph held at its last value after its end",
     "if (n <= 0 || tt < t[0] || tt > t[n - 1]) return 0.0;", "if (n <= 0 || tt < t[0]) return 0.0;"),
    ("viscous term on cells whose fluid is thinner than h_dry",
     "if (!(h > p->h_dry) || !(Uin[3][k] > J * p->h_dry)) continue;", "if (!(h > p->h_dry)) continue;"),
    ("phase fractions on cells thinner than h_dry",
     "if (h > p->h_dry) {\n                phs = hs / h;", "if (h > 0.0) {\n                phs = hs / h;"),
    ("budget's solid Y momentum from the fluid field",
     "out[3] = sum[2] * a;", "out[3] = sum[5] * a;"),
    ("Heun step not counted",
     "    s->last_dt = dt;\n    s->nsteps++;\n}\n\n/* dry rule", "    s->last_dt = dt;\n}\n\n/* dry rule"),
    ("CFL step from twice the wave speed",
     "double dt = cfl_dt(s, max_speed(s, s->U));", "double dt = cfl_dt(s, 2.0 * max_speed(s, s->U));"),
    ("earth pressure: active and passive regimes swapped",
     "return (vp - vm < -(1e-6 * (fabs(vp) + fabs(vm)) + 1e-6)) ? Kp : Ka;",
     "return (vp - vm < -(1e-6 * (fabs(vp) + fabs(vm)) + 1e-6)) ? Ka : Kp;"),
    ("earth pressure: cos^2(delta_b) in place of sec^2(delta_b)",
     "double r = sqrt(1.0 - cp2 / cd2);", "double r = sqrt(1.0 - cp2 * cd2);"),
    ("earth pressure: solid celerity without K",
     "double cs = sqrt(K * (p->eps * p->g * c * Add * (1.0 - al) * (h + hs) / 2.0));",
     "double cs = sqrt(p->eps * p->g * c * Add * (1.0 - al) * (h + hs) / 2.0);"),
    ("earth pressure: K on the fluid pressure too",
     "F[4] = J * hf * vXf * vnf + p->eps * J * h * Ad1 * pf;", "F[4] = J * hf * vXf * vnf + p->eps * J * h * Ad1 * (K * pf);"),
    ("earth pressure: regime from the transverse velocity component",
     "double vm = U[1 + d][km] / U[0][km], vp = U[1 + d][kp] / U[0][kp];",
     "double vm = U[2 - d][km] / U[0][km], vp = U[2 - d][kp] / U[0][kp];"),
    ("earth pressure: neighbours without solid not set aside",
     "if (!(U[0][km] > s->gc[km].J * hd) || !(U[0][k] > s->gc[k].J * hd) || !(U[0][kp] > s->gc[kp].J * hd))",
     "if (!(U[0][k] > s->gc[k].J * hd))"),
    ("earth pressure: CFL celerity with K_act",
     "face_flux(&s->p, G, 0, Kp, u, F, &a[0], &a[1], &P, NULL);", "face_flux(&s->p, G, 0, Ka, u, F, &a[0], &a[1], &P, NULL);"),
    ("earth pressure: each side with the other cell's coefficient",
     "face_flux(p, G, 0, KL, um, Fm, &asm_, &afm, &Pm, sm);\n            face_flux(p, G, 0, KR, up, Fp, &asp, &afp, &Pp, sp);",
     "face_flux(p, G, 0, KR, um, Fm, &asm_, &afm, &Pm, sm);\n            face_flux(p, G, 0, KL, up, Fp, &asp, &afp, &Pp, sp);"),
    ("row-range speed takes row j1 too",
     "for (int j = j0 < 0 ? 0 : j0; j < j1 && j < s->ny; j++)",
     "for (int j = j0 < 0 ? 0 : j0; j <= j1 && j < s->ny; j++)"),
    ("row-range speed starts one row late",
     "for (int j = j0 < 0 ? 0 : j0; j < j1 && j < s->ny; j++)",
     "for (int j = j0 < 0 ? 1 : j0 + 1; j < j1 && j < s->ny; j++)"),
    ("step with a given speed ignores it",
     "double dt = cfl_dt(s, amax);", "double dt = cfl_dt(s, max_speed(s, s->U));"),
    ("step with a given speed doubles it",
     "double dt = cfl_dt(s, amax);", "double dt = cfl_dt(s, 2.0 * amax);"),
    ("tangency v_Z misses the b_Y term", "double vZ = G->bX * vX + G->bY * vY;", "double vZ = G->bX * vX;"),
    ("v_eta from the first row of Omega^-1", "*veta = G->Ai[1][0] * vX + G->Ai[1][1] * vY + G->Ai[1][2] * vZ;", "*veta = G->Ai[0][0] * vX + G->Ai[1][1] * vY + G->Ai[1][2] * vZ;"),
    ("hydrograph interpolated from the wrong end", "return v[k] + w * (v[k + 1] - v[k]);", "return v[k + 1] + w * (v[k] - v[k + 1]);"),
    ("inflow critical depth with J once", "double hc = cbrt(q * q / (G->J * G->J * p->eps * p->g * G->c * Ann));", "double hc = cbrt(q * q / (G->J * p->eps * p->g * G->c * Ann));"),
    ("inflow velocity without J", "double vn = q / (G->J * hc);", "double vn = q / hc;"),
    ("inflow critical depth without A_nn", "double hc = cbrt(q * q / (G->J * G->J * p->eps * p->g * G->c * Ann));", "double hc = cbrt(q * q / (G->J * G->J * p->eps * p->g * G->c));"),
    ("a_max over the x speeds only", "for (int c = 0; c < 4; c++) m = fmax(m, a[c]);", "for (int c = 0; c < 2; c++) m = fmax(m, a[c]);"),
    ("CFL length from the larger spacing", "double dmin = s->dx < s->dy ? s->dx : s->dy;", "double dmin = s->dx < s->dy ? s->dy : s->dx;"),
    ("normal not normalised", "G->n[k] = m[k] / mm;", "G->n[k] = m[k];"),
    ("c from the first normal component", "G->c = G->n[2];", "G->c = G->n[0];"),
    ("inverse entry R[1][2] sign", "R[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / d;", "R[1][2] = (M[0][0] * M[1][2] - M[0][2] * M[1][0]) / d;"),
    ("dry threshold on the mass without J", "if (Jh > J * hdry) {", "if (Jh > hdry) {"),
    ("y-face right slope from the face's own cells",
     "double sR = minmod(uR - uL, V[IS(s, i, j + 2)] - uR);", "double sR = minmod(uR - uL, V[IS(s, i, j + 1)] - uR);"),
    ("phase speeds swapped between the momentum rows",
     "s->Hx[c][k] = numerical_flux(p->scheme, Fm[c], Fp[c], um[c], up[c], c < 3 ? as : af, ap, am);",
     "s->Hx[c][k] = numerical_flux(p->scheme, Fm[c], Fp[c], um[c], up[c], c < 3 ? af : as, ap, am);"),
    ("x-face P from the left side only", "s->Px[k] = 0.5 * (Pm + Pp);", "s->Px[k] = Pm;"),
    ("phase fraction from the solid depth only", "phf = hf / h;", "phf = hs / h;"),
    ("solid normal source along the wrong normal component",
     "double sn_s = J * pbs * G->n[m];", "double sn_s = J * pbs * G->n[1 - m];"),
    ("fluid drag without J",
     "double sv_f = -J * p->c_d * phs * phf * h * (vf[m] - vs[m]);",
     "double sv_f = -p->c_d * phs * phf * h * (vf[m] - vs[m]);"),
    ("friction speed without q_Z",
     "double qn = sqrt(qX * qX + qY * qY + qZ * qZ);", "double qn = sqrt(qX * qX + qY * qY);"),
    ("solid clamp volume without dy",
     "if (ph == 0) cl_s += -out[c] * s->dx * s->dy;", "if (ph == 0) cl_s += -out[c] * s->dx;"),
    ("dry momentum rule on the other phase's mass",
     "if (out[c] <= J * p->h_dry) {", "if (out[3 - c] <= J * p->h_dry) {"),
    ("west boundary faces not computed",
     "for (int i = -1; i < nx; i++) {\n            double um[6], up[6], Fm[6], Fp[6], asm_, afm, asp, afp, Pm, Pp;",
     "for (int i = 0; i < nx; i++) {\n            double um[6], up[6], Fm[6], Fp[6], asm_, afm, asp, afp, Pm, Pp;"),
    ("east wall mirrors the first cell", "int se = s->p.bc[1] == 0 ? nx - 1 - k : nx - 1;", "int se = s->p.bc[1] == 0 ? nx - 1 : nx - 1;"),
    ("south wall keeps its fluid normal momentum", "U[5][IS(s, i, gs)] = -U[5][IS(s, i, gs)];", "U[5][IS(s, i, gs)] = U[5][IS(s, i, gs)];"),
    ("Heun boundary budget without dt", "s->bnd_in[ph] += 0.5 * dt * (b1[ph] + s->st_bnd[ph]);", "s->bnd_in[ph] += 0.5 * (b1[ph] + s->st_bnd[ph]);"),
    ("Heun clamp volume of the second stage only", "s->clamp_vol[ph] += 0.5 * (c1[ph] + s->st_clamp[ph]);", "s->clamp_vol[ph] += s->st_clamp[ph];"),
    ("Heun dry rule after the average dropped", "if (s->U[c][k] <= J * s->p.h_dry) {\n                    s->U[c + 1][k] = 0.0;", "if (0) {\n                    s->U[c + 1][k] = 0.0;"),
    ("RK3 final combination 1/2, 1/2", "s->U[q][k] = s->U[q][k] / 3.0 + 2.0 * s->W2[q][k] / 3.0;", "s->U[q][k] = 0.5 * s->U[q][k] + 0.5 * s->W2[q][k];"),
    ("RK3 third stage from U instead of W1", "stage(s, s->W1, s->W2, t0 + 0.5 * dt, dt);", "stage(s, s->U, s->W2, t0 + 0.5 * dt, dt);"),
    ("step time not advanced by dt on Heun", "    s->t = t0 + dt;\n    s->last_dt = dt;\n    s->nsteps++;\n}\n\n/* dry rule", "    s->t = t0 + 0.5 * dt;\n    s->last_dt = dt;\n    s->nsteps++;\n}\n\n/* dry rule"),
    ("hydrograph zero only before its start", "if (n <= 0 || tt < t[0] || tt > t[n - 1]) return 0.0;", "if (n <= 0 || tt < t[0]) return 0.0;"),
    ("inflow direction inward on every side", "double sgn = (f->side == 0 || f->side == 2) ? 1.0 : -1.0; /* inward */", "double sgn = 1.0;"),
    ("transmissive east ghost copies the second-last cell", "int se = s->p.bc[1] == 0 ? nx - 1 - k : nx - 1;", "int se = s->p.bc[1] == 0 ? nx - 1 - k : nx - 2;"),
    ("ghost rows over the interior columns only (corner ghosts unset)",
     "the corners follow the S/N rule applied to the W/E ghosts */\n    for (int i = -GS; i < nx + GS; i++) {",
     "the corners follow the S/N rule applied to the W/E ghosts */\n    for (int i = 0; i < nx; i++) {"),
]


def _compile_mutant(src_text: str, old: str, new: str, path: str) -> str:
    assert src_text.count(old) >= 1, f"mutation anchor not found: {old}"
    text = src_text.replace(old, new, 1)
    c = path + ".c"
    with open(c, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", path, c, "-lm"])
    return path


def _build_mutant(src_text: str, old: str, new: str, path: str):
    return O.load(_compile_mutant(src_text, old, new, path))


@pytest.fixture(scope="module")
def mutant_libs():
    """Every planted mistake compiled up front on all host cores (the
    compilations are independent; the pins then run on one mutant at a
    time)."""
    src = open(SRC).read()
    with tempfile.TemporaryDirectory() as d:
        with cf.ThreadPoolExecutor(max(1, os.cpu_count() or 1)) as ex:
            futs = {what: ex.submit(_compile_mutant, src, old, new, os.path.join(d, f"mut{k}.so"))
                    for k, (what, old, new) in enumerate(MUTANTS)}
            paths = {what: f.result() for what, f in futs.items()}
        yield paths


@pytest.mark.parametrize("what,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(what, old, new, mutant_libs):
    L = O.load(mutant_libs[what])
    failed = []
    for pin in P.ALL_PINS:
        try:
            pin(L)
        except Exception as e:  # AssertionError, or NaN/overflow surfacing as errors
            failed.append(f"{pin.__name__}: {type(e).__name__}")
            break
    assert failed, f"planted mistake not caught by any pin: {what}"
