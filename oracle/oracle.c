/*
 * CPU oracle for spin-orbit tracking through a ring lattice.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the package's smoke check and the bench's
 * CPU-baseline / reference leg do.  It shares no code, header or constant with
 * the CUDA library.
 *
 * It is a plain, slow, step-by-step transcription of the method of
 *   Abell, Meiser, Ranjbar, Barber, "Accurate and efficient spin integration
 *   for particle accelerators" (arXiv:1501.03450),
 * in the paper's order and notation, with no blocking, fusion or reordering:
 *
 *   Sec. 2.1  canonical variables z = (X, Px, Y, Py, T, Pt), Eqs. (1)-(3)
 *   Sec. 2.2  Thomas-BMT precession vector in s, Eq. (6b)
 *   Sec. 3.1  exact sector-bend map, Eqs. (7)-(10)       ("bend-kick")
 *   Sec. 3.3  quadrupole matrix-kick split, Eqs. (21)-(27)
 *   Sec. 3.4  multipole drift-kick split, Eqs. (28)-(29)
 *   Sec. 3.3  (closing remark) higher-order versions of the symmetric split of
 *             Eq. (27): Yoshida's fourth-order composition of the
 *             second-order slice map, on elements with split_order 4
 *   Sec. 3.2  rectangular bend: dynamic rotations into and out of the
 *             magnet's Cartesian frame, Eqs. (Hprot), (prot); thin-fringe
 *             orbit map, Eq. (dipolefringe); exact body map, Eqs. (rhob),
 *             (rbend); offsets, Eqs. (Xoffset), (Toffset); fringe spin kick
 *             of a rectangular bend, Eq. (skfringeRB)
 *   Sec. 3.6  TEAPOT split of a sector bend, Eqs. (DKsplit), (teapotD): curved
 *             drift and the kick of the bend's uniform field (Eq. (sbendA))
 *   Sec. 3.5  thin lens: the multipole of Sec. 3.4 in the limit of zero length
 *             at fixed integrated strengths, spin sampled like any element
 *   Sec. 3.7  solenoid: exact body map Eq. (solenoid) of the Hamiltonian
 *             Eq. (Hsolenoid) with the vector potential Eq. (Asol); the
 *             unit velocity from the kinetic momentum, Eq. (mgVSol)
 *   Sec. 4.4  thin-pancake solenoid fringe spin kicks, Eq. (solFringe)
 *   Sec. 4.5  thin-fringe spin kicks of dipole and multipole fringes,
 *             Eq. (skfringe), on elements whose fringe flag is set
 *   Sec. 4.1  piece-wise constant spin rotations composed as quaternions,
 *             later slices on the left, Eq. (37)
 *             or, for the midpoint schemes, with Omega at the middle of each
 *             slice (each slice as two half-slices, or its central kick split;
 *             Sec. 5.3, Fig. oneTurnSpinErrs)
 *   Sec. 4.3  trapezoid-weighted edge rotations, sub-sampled levels Q(h/2^k),
 *             Romberg table and normalisation per element, Eqs. (38)-(39)
 *   Sec. 5    thin Siberian snakes (orbit-transparent spin rotators)
 *
 * Readings where the paper is silent (recorded in the design notes):
 *   - quaternions are Hamilton, scalar first; the spin is rotated actively,
 *     S' = Q S conj(Q); a rotation vector w gives q = (cos|w|/2, sin|w|/2 w^);
 *   - "Romberg order k" is the number of Romberg iterations, result Q_kk;
 *   - the DKD slice is half-drift, kick, half-drift; slice edges are the
 *     states between slices, edge 0 the element entrance;
 *   - the sector-bend vector-potential term of Eq. (7) already contains the
 *     metric factor (1 + hX) of Eq. (3);
 *   - the particle's own gamma = gamma0 (1 + beta0 Pt) enters Eq. (6b);
 *   - elements whose precession vector vanishes identically (drifts) carry no
 *     spin step;
 *   - a particle whose longitudinal momentum becomes imaginary (Ps^2 <= 0) is
 *     lost: it keeps the state it had at the entrance of that element and is
 *     not tracked further.
 *
 * The scalar type `real` is double for the oracle proper.  The same source is
 * also compiled with long double (an extended-precision copy used only to
 * measure the oracle's own rounding noise) and with double complex (complex-
 * step derivatives for exact Jacobians in the symplecticity tests).
 * <tgmath.h> makes sqrt/sin/... dispatch on the argument type.
 */
#ifndef ORACLE_OPCOUNT
#include <tgmath.h>
#include <complex.h>
#endif
#include <stdint.h>
#include <string.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_REAL
#define ORACLE_REAL double
#endif
typedef ORACLE_REAL real;

/* Real part, used for branch decisions only (identity for real builds). */
#define RE(x) ((double)creal(x))

/* Element kinds (own numbering; the CUDA library has its own). */
enum { ORC_DRIFT = 0, ORC_MULT = 1, ORC_QUAD_MK = 2, ORC_SBEND = 3, ORC_SNAKE = 4, ORC_SOLENOID = 5, ORC_RBEND = 6,
       ORC_TEAPOT = 7, ORC_THIN = 8 };

/* Spin integration schemes other than the Romberg orders K >= 0 (Sec. 4.1,
 * Eq. (37) with Omega taken at the middle of each slice):
 *   ORC_MID_HALF  each slice is traversed as two half-slices of its own map,
 *                 the spin rotation by ds Omega between them ("half-DKD,
 *                 spin rotation, half-DKD");
 *   ORC_MID_KICK  the slices of the second-order drift-kick and matrix-kick
 *                 splits keep their map and rotate the spin between the two
 *                 halves of the central kick ("half-drift, half-kick, spin
 *                 rotation, half-kick, half-drift"); exact maps as ORC_MID_HALF. */
enum { ORC_MID_HALF = -1, ORC_MID_KICK = -2 };

typedef struct {
    int32_t type;
    int32_t n_slices;
    double L, k1, k2, angle, eta, snake_phi, snake_mu;
    int32_t fringe;      /* 1: thin fringe spin kicks at both ends (mult, quad_mk, sbend) */
    int32_t split_order; /* mult, quad_mk, teapot: 0 or 2 = Eq. (27), 4 = Yoshida's fourth order */
    double e1;           /* rbend: the beam meets the entrance face at phi_entr = angle/2 + e1
                          * and the exit face at phi_exit = -angle/2 + e1 */
} orc_element;

typedef struct {
    double G, Ggamma0, gamma0, beta0;
} orc_ref;

typedef struct {
    real X, Px, Y, Py, T, Pt;
} orc_orbit;

static orc_ref make_ref(double G, double Ggamma0) {
    orc_ref r;
    r.G = G;
    r.Ggamma0 = Ggamma0;
    r.gamma0 = Ggamma0 / G;
    r.beta0 = sqrt(1.0 - 1.0 / (r.gamma0 * r.gamma0));
    return r;
}

/* Square of the scaled total momentum, 1 + 2 Pt/beta0 + Pt^2 (Eq. (22)). */
static real momentum_sq(const orc_ref* r, real Pt) {
    return 1.0 + 2.0 * Pt / r->beta0 + Pt * Pt;
}

/* ---------------------------------------------------------------------- */
/* orbit maps                                                             */
/* ---------------------------------------------------------------------- */

/* Exact drift: the flow of H_drift = -Ps + Pt/beta0 (Eq. (29b)),
 * dX/ds = Px/Ps, dY/ds = Py/Ps, dT/ds = 1/beta0 - (1/beta0 + Pt)/Ps. */
static int drift(const orc_ref* r, orc_orbit* z, double s) {
    real ps2 = momentum_sq(r, z->Pt) - z->Px * z->Px - z->Py * z->Py;
    if (!(RE(ps2) > 0.0)) return 1;
    real Ps = sqrt(ps2);
    z->X += s * z->Px / Ps;
    z->Y += s * z->Py / Ps;
    z->T += s * (1.0 / r->beta0 - (1.0 / r->beta0 + z->Pt) / Ps);
    return 0;
}

/* Normal multipole coefficients of Eq. (28) for a combined quadrupole and
 * sextupole: H_m = Re[ sum_m (b_m/(m B rho)) (X + iY)^m ] with
 * b_2/(B rho) = k1 and b_3/(B rho) = k2/2 (MAD k2 = B''/(B rho)).
 * The field b = B/(B rho) follows from B_y + i B_x = sum_m c_m (X+iY)^(m-1). */
static void mult_field(double k1, double k2, real X, real Y, real* bx, real* by) {
    /* (X + iY)^1 and (X + iY)^2 written out in real arithmetic so that the
     * complex-step build can use the same code */
    real w1r = X, w1i = Y;
    real w2r = X * X - Y * Y, w2i = 2.0 * X * Y;
    real c2 = k1, c3 = 0.5 * k2;
    *by = c2 * w1r + c3 * w2r;
    *bx = c2 * w1i + c3 * w2i;
}

/* Kick generated by H_m over a length ds: dPx/ds = -dH_m/dX = -b_y,
 * dPy/ds = -dH_m/dY = +b_x (Sec. 3.4). */
static void mult_kick(orc_orbit* z, double k1, double k2, double ds) {
    real bx, by;
    mult_field(k1, k2, z->X, z->Y, &bx, &by);
    z->Px -= ds * by;
    z->Py += ds * bx;
}

/* Exact sector-bend map over a length s, Eq. (10) with P_alpha of Eq. (8) and
 * eta of Eq. (9).  h is the fixed curvature of the magnet. */
static int sbend_map(const orc_ref* r, orc_orbit* z, double h, double eta, double s) {
    real Pa2 = momentum_sq(r, z->Pt) - z->Py * z->Py;           /* Eq. (8) squared */
    real Xi = z->X, Pxi = z->Px;
    real ri2 = Pa2 - Pxi * Pxi;
    if (!(RE(ri2) > 0.0)) return 1;
    real Pa = sqrt(Pa2);
    real root_i = sqrt(ri2);
    double c = cos(h * s), sn = sin(h * s);
    real Pxf = Pxi * c + (root_i - eta * (1.0 + h * Xi)) * sn;               /* Eq. (10b) */
    real dPxf = -h * Pxi * sn + h * (root_i - eta * (1.0 + h * Xi)) * c;     /* d Px / ds */
    real rf2 = Pa2 - Pxf * Pxf;
    if (!(RE(rf2) > 0.0)) return 1;
    real Xf = (1.0 / h) * ((1.0 / eta) * (sqrt(rf2) - dPxf / h) - 1.0);     /* Eq. (10a) */
    real dasin = asin(Pxi / Pa) - asin(Pxf / Pa);
    z->Y = z->Y + (1.0 / eta) * z->Py * s + (1.0 / (eta * h)) * z->Py * dasin;   /* Eq. (10c) */
    z->T = z->T - (1.0 / eta) * z->Pt * s
           - (1.0 / (eta * h)) * (1.0 / r->beta0 + z->Pt) * dasin
           + (1.0 - 1.0 / eta) * s / r->beta0;                                /* Eq. (10e) */
    z->X = Xf;
    z->Px = Pxf;
    return 0;
}

/* TEAPOT split of a sector bend, Sec. 3.6, Eq. (DKsplit): H_T = H_D + H_K.
 * Drift part: the flow of H_D = -(1 + hX) Ps + Pt/beta0 over s, Eq. (teapotD)
 * (a straight line seen from the frame that turns by h s about the centre of
 * curvature).  The arrival time also carries the reference term s/beta0 of
 * the Pt/beta0 part of Eq. (generalH), which the printed Eq. (teapotD) leaves
 * out. */
static int curved_drift(const orc_ref* r, orc_orbit* z, double h, double s) {
    real ps2 = momentum_sq(r, z->Pt) - z->Px * z->Px - z->Py * z->Py;
    if (!(RE(ps2) > 0.0)) return 1;
    real Ps = sqrt(ps2);
    double phi = h * s;
    double t = tan(phi), c = cos(phi), sn = sin(phi);
    real den = 1.0 - (z->Px / Ps) * t;
    if (!(RE(den) > 0.0)) return 1;
    real R = 1.0 / h + z->X;
    real d = R * t / den;                    /* (1/h + X^i) tan(hs) / (1 - (Px^i/Ps^i) tan(hs)) */
    z->X = R / (c * den) - 1.0 / h;          /* Eq. (teapotD), X */
    z->Y = z->Y + (z->Py / Ps) * d;          /* Y */
    z->T = z->T - ((1.0 / r->beta0 + z->Pt) / Ps) * d + s / r->beta0;   /* T, with s/beta0 */
    z->Px = z->Px * c + Ps * sn;             /* Px */
    return 0;
}

/* Kick part: the flow of H_K = -(q/p0)(1 + hX) A_s over s for the sector
 * bend's uniform field, whose vector-potential term is (eta/2)(1 + hX)^2
 * (Eq. (sbendA) with eta of Eq. (9)): dPx/ds = -eta h (1 + hX). */
static void teapot_kick(orc_orbit* z, double h, double eta, double s) {
    z->Px -= s * eta * h * (1.0 + h * z->X);
}

static real sinc_(real x) { return (RE(x) == 0.0 && cimag(x) == 0.0) ? (real)1.0 : sin(x) / x; }
static real sinhc_(real x) { return (RE(x) == 0.0 && cimag(x) == 0.0) ? (real)1.0 : sinh(x) / x; }
static real sin2c_(real x) { return (RE(x) == 0.0 && cimag(x) == 0.0) ? (real)0.0 : sin(x) * sin(x) / x; }
static real sinh2c_(real x) { return (RE(x) == 0.0 && cimag(x) == 0.0) ? (real)0.0 : sinh(x) * sinh(x) / x; }

/* Flow of the linear quadrupole Hamiltonian H_qL (Eq. (21b)) over a length
 * s for a focusing gradient k1 = b2/(B rho) >= 0: Eq. (24) with P of Eq. (22)
 * and kappa of Eq. (23). */
static void quad_linear_focusing(const orc_ref* r, orc_orbit* z, double k1, double s) {
    real P = sqrt(momentum_sq(r, z->Pt));
    real kap = sqrt(k1 / P);
    real ks = kap * s;
    real X = z->X, Px = z->Px, Y = z->Y, Py = z->Py;
    real Xf = X * cos(ks) + s * (Px / P) * sinc_(ks);
    real Pxf = Px * cos(ks) - kap * P * X * sin(ks);
    real Yf = Y * cosh(ks) + s * (Py / P) * sinhc_(ks);
    real Pyf = Py * cosh(ks) + kap * P * Y * sinh(ks);
    real brace =
        (s / 4.0) * ((Px * Px + Py * Py) / (P * P) + kap * kap * (X * X - Y * Y))
        + (s / 4.0) * ((Px / P) * (Px / P) - (kap * X) * (kap * X)) * sinc_(2.0 * ks)
        + (s / 4.0) * ((Py / P) * (Py / P) + (kap * Y) * (kap * Y)) * sinhc_(2.0 * ks)
        - (ks / 2.0) * (X * (Px / P) * sin2c_(ks) - Y * (Py / P) * sinh2c_(ks));
    z->T = z->T - (1.0 / P) * (1.0 / r->beta0 + z->Pt) * brace;
    z->X = Xf;
    z->Px = Pxf;
    z->Y = Yf;
    z->Py = Pyf;
}

/* For a defocusing gradient (k1 < 0) the paper rotates the transverse frame
 * about the longitudinal axis so that the magnet focuses in the first plane
 * (Sec. 3.3): a 90 degree rotation maps (X, Px, Y, Py) -> (Y, Py, -X, -Px)
 * and turns the gradient k1 into -k1. */
static void quad_linear(const orc_ref* r, orc_orbit* z, double k1, double s) {
    if (k1 >= 0.0) {
        quad_linear_focusing(r, z, k1, s);
        return;
    }
    orc_orbit w = *z;
    w.X = z->Y;
    w.Px = z->Py;
    w.Y = -z->X;
    w.Py = -z->Px;
    quad_linear_focusing(r, &w, -k1, s);
    z->X = -w.Y;
    z->Px = -w.Py;
    z->Y = w.X;
    z->Py = w.Px;
    z->T = w.T;
}

/* Flow of the nonlinear quadrupole remainder H_qNL (Eq. (21c)) over s,
 * Eq. (25). */
static int quad_nonlinear(const orc_ref* r, orc_orbit* z, double s) {
    real P2 = momentum_sq(r, z->Pt);
    real P = sqrt(P2);
    real ps2 = P2 - z->Px * z->Px - z->Py * z->Py;
    if (!(RE(ps2) > 0.0)) return 1;
    real Ps = sqrt(ps2);
    real Px = z->Px, Py = z->Py;
    z->X = z->X + s * Px * (1.0 / Ps - 1.0 / P);
    z->Y = z->Y + s * Py * (1.0 / Ps - 1.0 / P);
    z->T = z->T - s * (1.0 / r->beta0 + z->Pt) * (1.0 / Ps - (1.0 / P) * (Px * Px + Py * Py) / (2.0 * P2))
           + s / r->beta0;
    return 0;
}

/* Solenoid body, Sec. 3.7.  The element's k1 holds the normalised body field
 * b0/(B rho) (MAD's ks); eta = b0/(2 B rho) and the scaled vector potential
 * (e/p0)(A_x, A_y) = eta (-Y, X) (Eq. (Asol)), so the kinetic momenta are
 * px = Px + eta Y, py = Py - eta X and Ps = sqrt(P^2 - px^2 - py^2) is
 * conserved.  Over a length s the transverse variables go through the
 * commuting matrices R1(kappa s) R2(kappa s) of Eq. (solenoid) with
 * kappa = eta / Ps, and T shifts by Eq. (solT).  R1's entry sin(kappa s)/eta
 * is written (s/Ps) sinc(kappa s), which stays finite as eta -> 0. */
static void solenoid_kinetic(real eta, const orc_orbit* z, real* px, real* py) {
    *px = z->Px + eta * z->Y;
    *py = z->Py - eta * z->X;
}

static int solenoid_map(const orc_ref* r, orc_orbit* z, double ks, double s) {
    real eta = 0.5 * ks;
    real px, py;
    solenoid_kinetic(eta, z, &px, &py);
    real ps2 = momentum_sq(r, z->Pt) - px * px - py * py;
    if (!(RE(ps2) > 0.0)) return 1;
    real Ps = sqrt(ps2);
    real ks_ = (eta / Ps) * s;                    /* kappa s */
    real c = cos(ks_), sn = sin(ks_);
    real a12 = (s / Ps) * sinc_(ks_);             /* sin(kappa s)/eta */
    real a21 = -eta * sn;                         /* -eta sin(kappa s) */
    /* R1: each plane (U, Pu) -> (c U + a12 Pu, a21 U + c Pu) */
    real X1 = c * z->X + a12 * z->Px, Px1 = a21 * z->X + c * z->Px;
    real Y1 = c * z->Y + a12 * z->Py, Py1 = a21 * z->Y + c * z->Py;
    /* R2: rotation of the transverse plane, (X, Y) -> (c X + sn Y, -sn X + c Y), same for (Px, Py) */
    z->X = c * X1 + sn * Y1;
    z->Y = -sn * X1 + c * Y1;
    z->Px = c * Px1 + sn * Py1;
    z->Py = -sn * Px1 + c * Py1;
    z->T = z->T - (1.0 / r->beta0 + z->Pt) * s / Ps + s / r->beta0;   /* Eq. (solT) */
    return 0;
}

/* One integration slice of length ds of a spin-carrying element. */
/* Rectangular bend, Sec. 3.2.  The magnet's Cartesian frame has both faces
 * normal to its axis; the beam meets the entrance face at phi_entr and the
 * exit face at phi_exit (total bend phi_entr - phi_exit = angle).  The design
 * field makes the reference particle enter with Px = sin(phi_entr) and leave
 * with Px = sin(phi_exit) after the magnet length L, so that
 * b1/(B rho) = 1/rho_b = eta (sin phi_entr - sin phi_exit) / L (Eq. (rhob)). */
static void rbend_geometry(const orc_element* e, double* phi_in, double* phi_out, double* b) {
    *phi_in = 0.5 * e->angle + e->e1;
    *phi_out = -0.5 * e->angle + e->e1;
    *b = e->eta * (sin(*phi_in) - sin(*phi_out)) / e->L;
}

/* Body of the rectangular bend over a length s, Eq. (rbend): Px falls
 * linearly, X follows from the longitudinal momentum, Y and T from the change
 * of the angle asin(Px/P_alpha).  T is the printed form (the reference
 * particle's time across the magnet, -L_arc/beta0, is removed by Eq. (Toffset)
 * at the end of the element). */
static int rbend_body(const orc_ref* r, orc_orbit* z, double b, double s) {
    real Pa2 = momentum_sq(r, z->Pt) - z->Py * z->Py;
    real Pxf = z->Px - s * b;
    real qi = Pa2 - z->Px * z->Px, qf = Pa2 - Pxf * Pxf;
    if (!(RE(qi) > 0.0) || !(RE(qf) > 0.0)) return 1;
    real Pa = sqrt(Pa2);
    real dpsi = asin(z->Px / Pa) - asin(Pxf / Pa);
    z->X += (sqrt(qf) - sqrt(qi)) / b;
    z->Y += z->Py * dpsi / b;
    z->T -= (1.0 / r->beta0 + z->Pt) * dpsi / b;
    z->Px = Pxf;
    return 0;
}

/* Dynamic rotation by phi: the flow of H_prot = -X Ps (Eq. (Hprot)) with phi
 * as the independent variable, Eq. (prot).  The arrival-time update takes the
 * sign of Hamilton's equation dT/dphi = dH/dPt = -X (1/beta0 + Pt)/Ps (the
 * same sign as the drift towards the rotated face implied by the Y update);
 * the printed Eq. (prot) shows the opposite sign for T. */
static int rbend_rotation(const orc_ref* r, orc_orbit* z, double phi) {
    real ps2 = momentum_sq(r, z->Pt) - z->Px * z->Px - z->Py * z->Py;
    if (!(RE(ps2) > 0.0)) return 1;
    real Ps = sqrt(ps2);
    real t = tan(phi);
    real den = 1.0 - z->Px / Ps * t;
    if (!(RE(den) > 0.0)) return 1;
    real d = z->X * t / den;              /* longitudinal distance to the rotated face */
    real Px = z->Px * cos(phi) + Ps * sin(phi);
    z->Y += z->Py / Ps * d;
    z->T -= (1.0 / r->beta0 + z->Pt) / Ps * d;
    z->X = z->X / (cos(phi) * den);
    z->Px = Px;
    return 0;
}

/* Thin dipole fringe of the rectangular bend without a finite-gap correction,
 * Eq. (dipolefringe), sign +1 at the entrance and -1 at the exit; bs =
 * b1/(B rho); x' = Px/Ps, y' = Py/Ps and Ps from the incoming momenta.  The
 * map is the canonical transformation generated by
 *   Phi = -(sign bs / 2) x'/(1 + y'^2) Y_f^2
 * (new coordinates, old momenta): X, Py and T follow Eq. (dipolefringe) as
 * printed; Y_f solves Y_i = Y_f + (sign bs / 2) x'y'/(Ps (1 + y'^2)) Y_f^2,
 * i.e. the printed root with the factor 1/Ps inside the square root, which
 * the printed equation omits (without it the map is not symplectic). */
static int rbend_fringe_orbit(const orc_ref* r, orc_orbit* z, double bs, int sign) {
    real ps2 = momentum_sq(r, z->Pt) - z->Px * z->Px - z->Py * z->Py;
    if (!(RE(ps2) > 0.0)) return 1;
    real Ps = sqrt(ps2);
    real xp = z->Px / Ps, yp = z->Py / Ps;
    real g = 1.0 + yp * yp;
    real sb = sign * bs;
    real arg = 1.0 + sb * (xp * yp / (g * Ps)) * 2.0 * z->Y;
    if (!(RE(arg) > 0.0)) return 1;
    real Yf = 2.0 * z->Y / (1.0 + sqrt(arg));
    z->X += sb / (2.0 * Ps) * ((1.0 + xp * xp) / g - 2.0 * (xp * yp) * (xp * yp) / (g * g)) * Yf * Yf;
    z->Py -= sb * xp / g * Yf;
    z->T -= sb * (1.0 / r->beta0 + z->Pt) * xp / (2.0 * ps2) * (1.0 - yp * yp) / (g * g) * Yf * Yf;
    z->Y = Yf;
    return 0;
}

static int slice_map2(const orc_ref* r, const orc_element* e, orc_orbit* z, double ds) {
    switch (e->type) {
    case ORC_MULT:   /* drift-kick-drift, Sec. 3.4 with the symmetric form of Eq. (27) */
        if (drift(r, z, 0.5 * ds)) return 1;
        mult_kick(z, e->k1, e->k2, ds);
        return drift(r, z, 0.5 * ds);
    case ORC_QUAD_MK: /* matrix-kick, Eq. (27) */
        quad_linear(r, z, e->k1, 0.5 * ds);
        if (quad_nonlinear(r, z, ds)) return 1;
        quad_linear(r, z, e->k1, 0.5 * ds);
        return 0;
    case ORC_SBEND:   /* exact bend, Eq. (10) */
        return sbend_map(r, z, e->angle / e->L, e->eta, ds);
    case ORC_THIN:    /* Sec. 3.5: the drift-kick slice without its drifts; ds is the slice's share of the
                         unit kick parameter and k1, k2 hold integrated strengths */
        mult_kick(z, e->k1, e->k2, ds);
        return 0;
    case ORC_TEAPOT:  /* curved drift - kick - curved drift, Sec. 3.6 in the symmetric form of Eq. (27) */
        if (curved_drift(r, z, e->angle / e->L, 0.5 * ds)) return 1;
        teapot_kick(z, e->angle / e->L, e->eta, ds);
        return curved_drift(r, z, e->angle / e->L, 0.5 * ds);
    case ORC_SOLENOID: /* exact body map, Eq. (solenoid) */
        return solenoid_map(r, z, e->k1, ds);
    case ORC_RBEND: { /* exact body map in the magnet's Cartesian frame, Eq. (rbend) */
        double pi_, po_, b;
        rbend_geometry(e, &pi_, &po_, &b);
        return rbend_body(r, z, b, ds);
    }
    default:
        return 1;
    }
}

/* One slice of an element.  With split_order 4 the symmetric second-order
 * slice map S2 of Eq. (27) is composed as Yoshida's fourth-order product
 * S2(x1 ds) S2(x0 ds) S2(x1 ds), with x1 = 1/(2 - 2^(1/3)) and
 * x0 = 1 - 2 x1, the weights that cancel the third-order error term
 * (2 x1^3 + x0^3 = 0) of a symmetric method (Yoshida 1990). */
static int slice_map(const orc_ref* r, const orc_element* e, orc_orbit* z, double ds) {
    if (e->split_order != 4) return slice_map2(r, e, z, ds);
    double x1 = 1.0 / (2.0 - cbrt(2.0));
    double x0 = 1.0 - 2.0 * x1;
    if (slice_map2(r, e, z, x1 * ds)) return 1;
    if (slice_map2(r, e, z, x0 * ds)) return 1;
    return slice_map2(r, e, z, x1 * ds);
}

/* ---------------------------------------------------------------------- */
/* spin                                                                   */
/* ---------------------------------------------------------------------- */

/* Thomas-BMT precession vector in s, Eq. (6b):
 *   Omega = -(1 + hX)/(B rho Ps) [ (1 + G gamma) B - G (gamma - 1)(u.B) u ] + h y^
 * with u the unit vector along (Px, Py, Ps) and gamma the particle's own
 * Lorentz factor, gamma = gamma0 (1 + beta0 Pt) from Eq. (2). */
static int omega(const orc_ref* r, const orc_element* e, const orc_orbit* z, real out[3]) {
    real P2 = momentum_sq(r, z->Pt);
    real P = sqrt(P2);
    real ps2 = P2 - z->Px * z->Px - z->Py * z->Py;
    if (!(RE(ps2) > 0.0)) return 1;
    real Ps = sqrt(ps2);
    real gamma = r->gamma0 * (1.0 + r->beta0 * z->Pt);
    real b[3] = {0.0, 0.0, 0.0};
    double h = 0.0;
    real u[3] = {z->Px / P, z->Py / P, Ps / P};
    if (e->type == ORC_SBEND || e->type == ORC_TEAPOT) {
        h = e->angle / e->L;
        b[1] = e->eta * h;             /* b1/(B rho) = eta h, Eq. (9) */
    } else if (e->type == ORC_RBEND) {
        double pi_, po_, bs;           /* uniform vertical field, straight frame (h = 0) */
        rbend_geometry(e, &pi_, &po_, &bs);
        b[1] = bs;
    } else if (e->type == ORC_SOLENOID) {
        /* body field along s; u from the kinetic momentum, Eq. (mgVSol) */
        real px, py;
        solenoid_kinetic(0.5 * e->k1, z, &px, &py);
        ps2 = P2 - px * px - py * py;
        if (!(RE(ps2) > 0.0)) return 1;
        Ps = sqrt(ps2);
        b[2] = e->k1;
        u[0] = px / P;
        u[1] = py / P;
        u[2] = Ps / P;
    } else {
        mult_field(e->k1, e->k2, z->X, z->Y, &b[0], &b[1]);
    }
    real ub = u[0] * b[0] + u[1] * b[1] + u[2] * b[2];
    real pre = -(1.0 + h * z->X) / Ps;
    for (int i = 0; i < 3; ++i)
        out[i] = pre * ((1.0 + r->G * gamma) * b[i] - r->G * (gamma - 1.0) * ub * u[i]);
    out[1] += h;
    return 0;
}

/* Hamilton product a (x) b, scalar first. */
static void qmul(const real a[4], const real b[4], real out[4]) {
    real o0 = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    real o1 = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    real o2 = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    real o3 = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    out[0] = o0; out[1] = o1; out[2] = o2; out[3] = o3;
}

/* Unit quaternion of the rotation about w^ by the angle |w|. */
static void quat_from_rotation_vector(const real w[3], real q[4]) {
    real th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    if (RE(th2) == 0.0 && cimag(th2) == 0.0) {
        q[0] = 1.0; q[1] = q[2] = q[3] = 0.0;
        return;
    }
    real th = sqrt(th2);
    real f = sin(0.5 * th) / th;
    q[0] = cos(0.5 * th);
    q[1] = f * w[0];
    q[2] = f * w[1];
    q[3] = f * w[2];
}

/* S <- Q S conj(Q), computed as quaternion products. */
static void rotate_spin(const real Q[4], real S[3]) {
    real s4[4] = {0.0, S[0], S[1], S[2]};
    real qc[4] = {Q[0], -Q[1], -Q[2], -Q[3]};
    real t[4], o[4];
    qmul(Q, s4, t);
    qmul(t, qc, o);
    S[0] = o[1]; S[1] = o[2]; S[2] = o[3];
}

#define ORC_MAX_ORDER 6

/* Net element rotation from the precession vectors recorded at the N+1
 * slice edges (Sec. 4.3): for every level k = 0..K the edges are sub-sampled
 * with stride 2^(K-k), the step is stride*ds, the two end edges get half a
 * step (trapezoid rule), and the edge rotations are multiplied with later
 * edges on the left (Eq. (37b)); this gives Q_0k = Q(h/2^k) of Eqs. (38),
 * (39a).  The Romberg rule Eq. (39b) then builds the table Eq. (39c) and the
 * bottom-right entry Q_KK is normalised.  levels (may be NULL) receives
 * Q_00..Q_0K. */
static void romberg_element_rotation(const real (*Om)[3], int N, double ds, int K,
                                     real Q[4], real* levels) {
    real Tab[ORC_MAX_ORDER + 1][ORC_MAX_ORDER + 1][4];
    for (int k = 0; k <= K; ++k) {
        int stride = 1 << (K - k);
        double step = stride * ds;
        real acc[4] = {1.0, 0.0, 0.0, 0.0};
        for (int i = 0; i <= N; i += stride) {
            double wgt = (i == 0 || i == N) ? 0.5 * step : step;
            real w[3] = {wgt * Om[i][0], wgt * Om[i][1], wgt * Om[i][2]};
            real q[4];
            quat_from_rotation_vector(w, q);
            qmul(q, acc, acc);
        }
        for (int c = 0; c < 4; ++c) {
            Tab[0][k][c] = acc[c];
            if (levels) levels[4 * k + c] = acc[c];
        }
    }
    for (int j = 0; j < K; ++j) {
        double f = 1.0;
        for (int p = 0; p <= j; ++p) f *= 4.0;        /* 4^(j+1) */
        for (int k = j + 1; k <= K; ++k)
            for (int c = 0; c < 4; ++c)
                Tab[j + 1][k][c] = (f * Tab[j][k][c] - Tab[j][k - 1][c]) / (f - 1.0);
    }
    real n = sqrt(Tab[K][K][0] * Tab[K][K][0] + Tab[K][K][1] * Tab[K][K][1] +
                  Tab[K][K][2] * Tab[K][K][2] + Tab[K][K][3] * Tab[K][K][3]);
    for (int c = 0; c < 4; ++c) Q[c] = Tab[K][K][c] / n;
}

/* Half of one slice of length ds for the midpoint schemes: part 0 takes the
 * state from the slice entrance to its middle, part 1 from the middle to the
 * exit.  ORC_MID_KICK splits the central kick of the second-order drift-kick
 * (Sec. 3.4, 3.6) and matrix-kick (Eq. (27)) slices in two (the kicks of a
 * slice commute, so the orbit map is that of the slice); every other map, and
 * every map under ORC_MID_HALF, is run over half the slice. */
static int slice_half(const orc_ref* r, const orc_element* e, orc_orbit* z, double ds, int scheme, int part) {
    if (scheme == ORC_MID_KICK && e->split_order != 4) {
        double hd = 0.5 * ds;
        switch (e->type) {
        case ORC_MULT:
            if (part == 0) {
                if (drift(r, z, hd)) return 1;
                mult_kick(z, e->k1, e->k2, hd);
                return 0;
            }
            mult_kick(z, e->k1, e->k2, hd);
            return drift(r, z, hd);
        case ORC_TEAPOT: {
            double h = e->angle / e->L;
            if (part == 0) {
                if (curved_drift(r, z, h, hd)) return 1;
                teapot_kick(z, h, e->eta, hd);
                return 0;
            }
            teapot_kick(z, h, e->eta, hd);
            return curved_drift(r, z, h, hd);
        }
        case ORC_QUAD_MK:
            if (part == 0) {
                quad_linear(r, z, e->k1, hd);
                return quad_nonlinear(r, z, hd);
            }
            if (quad_nonlinear(r, z, hd)) return 1;
            quad_linear(r, z, e->k1, hd);
            return 0;
        default:
            break;
        }
    }
    return slice_map(r, e, z, 0.5 * ds);
}

/* Piece-wise constant spin integration with Omega at the middle of each slice
 * (Sec. 4.1, Eq. (37)): the rotation of slice i is R(ds Omega(s_i + ds/2)),
 * later slices on the left.  The orbit is advanced through the N slices on
 * the way.  The product is normalised once (it differs from a unit
 * quaternion by rounding only).  Returns 1 if the particle is lost. */
static int midpoint_rotation(const orc_ref* r, const orc_element* e, orc_orbit* z, int N, double ds,
                             int scheme, real Q[4]) {
    Q[0] = 1.0; Q[1] = Q[2] = Q[3] = 0.0;
    for (int i = 0; i < N; ++i) {
        if (slice_half(r, e, z, ds, scheme, 0)) return 1;
        real Om[3], q[4];
        if (omega(r, e, z, Om)) return 1;
        real w[3] = {ds * Om[0], ds * Om[1], ds * Om[2]};
        quat_from_rotation_vector(w, q);
        qmul(q, Q, Q);
        if (slice_half(r, e, z, ds, scheme, 1)) return 1;
    }
    real n = sqrt(Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2] + Q[3] * Q[3]);
    for (int c = 0; c < 4; ++c) Q[c] = Q[c] / n;
    return 0;
}

/* Net spin rotation vector of a thin-pancake solenoid fringe, Eq. (solFringe):
 *   w = sign (b0/2)/(B rho Ps') [ (1 + G gamma)(X, Y, 0)
 *                                 - G (gamma - 1)(X Px + Y Py)/P^2 m gamma V' ],
 * sign +1 at the entrance, -1 at the exit, with the kinetic momentum
 * m gamma V' and Ps' evaluated with half the vector potential (the middle of
 * the fringe). */
static int solenoid_fringe(const orc_ref* r, double ks, int sign, const orc_orbit* z, real w[3]) {
    real P2 = momentum_sq(r, z->Pt);
    real px, py;
    solenoid_kinetic(0.25 * ks, z, &px, &py);
    real ps2 = P2 - px * px - py * py;
    if (!(RE(ps2) > 0.0)) return 1;
    real Ps = sqrt(ps2);
    real gamma = r->gamma0 * (1.0 + r->beta0 * z->Pt);
    real pre = sign * 0.5 * ks / Ps;
    real xp = (z->X * z->Px + z->Y * z->Py) / P2;
    real a = 1.0 + r->G * gamma, cg = r->G * (gamma - 1.0);
    w[0] = pre * (a * z->X - cg * xp * px);
    w[1] = pre * (a * z->Y - cg * xp * py);
    w[2] = pre * (-cg * xp * Ps);
    return 0;
}

static int fringe_rotate(const orc_ref* r, double ks, int sign, const orc_orbit* z, real S[3]) {
    real w[3], q[4];
    if (solenoid_fringe(r, ks, sign, z, w)) return 1;
    quat_from_rotation_vector(w, q);
    rotate_spin(q, S);
    return 0;
}

/* Normal 2m-pole content of an element as (m, b_m/(B rho)) pairs, in the
 * normalisation of Eq. (Amult): a sector bend is a dipole with
 * b_1/(B rho) = eta h (Eq. (9)); a quadrupole has b_2/(B rho) = k1; the
 * sextupole part of a multipole has b_3/(B rho) = k2/2 (MAD's k2 = B''/(B rho)).
 * Returns the number of pairs. */
static int normal_multipoles(const orc_element* e, int m[2], double bm[2]) {
    switch (e->type) {
    case ORC_SBEND:
    case ORC_TEAPOT: m[0] = 1; bm[0] = e->eta * e->angle / e->L; return 1;
    case ORC_QUAD_MK: m[0] = 2; bm[0] = e->k1; return 1;
    case ORC_MULT: m[0] = 2; bm[0] = e->k1; m[1] = 3; bm[1] = 0.5 * e->k2; return 2;
    default: return 0;
    }
}

/* Spin kick of a thin dipole or multipole fringe, Eq. (skfringe), to lowest
 * order in the dynamical variables: a rotation about the longitudinal axis by
 *   omega_s = -sign (1 + G) sum_m (b_m/(B rho)) r^m sin(m phi) / m,
 * with r^m sin(m phi) = Im (X + iY)^m; sign +1 at the entrance, -1 at the
 * exit.  The orbit is unchanged. */
static void multipole_fringe(const orc_ref* r, const orc_element* e, int sign, const orc_orbit* z, real w[3]) {
    int m[2];
    double bm[2];
    int n = normal_multipoles(e, m, bm);
    real sum = 0.0;
    for (int j = 0; j < n; ++j) {
        real re = 1.0, im = 0.0;                 /* (X + iY)^k by repeated multiplication */
        for (int k = 0; k < m[j]; ++k) {
            real re2 = re * z->X - im * z->Y;
            im = re * z->Y + im * z->X;
            re = re2;
        }
        sum += bm[j] * im / m[j];
    }
    w[0] = 0.0;
    w[1] = 0.0;
    w[2] = -sign * (1.0 + r->G) * sum;
}

/* Fringe spin kick of element e at its entrance (sign +1) or exit (-1):
 * solenoids always (thin-pancake model, Sec. 4.4), dipoles and multipoles
 * when the element's fringe flag is set (Sec. 4.5).  Returns 1 if lost. */
static int element_fringe(const orc_ref* r, const orc_element* e, int sign, const orc_orbit* z, real S[3]) {
    if (e->type == ORC_SOLENOID) return fringe_rotate(r, e->k1, sign, z, S);
    if (!e->fringe) return 0;
    real w[3], q[4];
    multipole_fringe(r, e, sign, z, w);
    quat_from_rotation_vector(w, q);
    rotate_spin(q, S);
    return 0;
}

/* Spin kick of a rectangular-bend fringe, Eq. (skfringeRB), sign +1 at the
 * entrance and -1 at the exit, in the magnet's Cartesian frame: the dipole
 * kick of Eq. (skfringe) (m = 1) plus the part of the longitudinal fringe
 * field transverse to a velocity inclined by Px,
 *   w = (+-b1/(B rho)) [ G (gamma - 1) Px Y x^ - (1 + G) Y z^ ].
 * The factor Y of the second term is the fringe's integrated longitudinal
 * field per unit b1/(B rho); the printed equation shows Px alone, which is not
 * an angle. */
static void rbend_fringe_spin(const orc_ref* r, double bs, int sign, const orc_orbit* z, real w[3]) {
    real gamma = r->gamma0 * (1.0 + r->beta0 * z->Pt);
    real sb = sign * bs;
    w[0] = sb * r->G * (gamma - 1.0) * z->Px * z->Y;
    w[1] = 0.0;
    w[2] = -sb * (1.0 + r->G) * z->Y;
}

static void rotate_about_y(double phi, real S[3]) {
    real w[3] = {0.0, phi, 0.0}, q[4];
    quat_from_rotation_vector(w, q);
    rotate_spin(q, S);
}

/* Rectangular bend through its entrance rotation (orbit, Eq. (prot), and the
 * spin components, rotated about y by the same angle), entrance fringe (spin
 * kick if the fringe flag is set, Eq. (skfringeRB); orbit, Eq. (dipolefringe)),
 * the body in n_slices slices with the spin integrated as for every element
 * (Omega of Eq. (6b) with the uniform field and h = 0), exit fringe, the
 * horizontal offset of Eq. (Xoffset) in the magnet frame, the exit rotation by
 * -phi_exit, and the reference time of Eq. (Toffset). */
static int track_rbend(const orc_ref* r, const orc_element* e, orc_orbit* z, real S[3], int K,
                       real* levels_out, real* Q_out) {
    double phi_in, phi_out, b;
    rbend_geometry(e, &phi_in, &phi_out, &b);
    double sd = sin(phi_in) - sin(phi_out);
    double x_offset = -e->L * (cos(phi_in) - cos(phi_out)) / sd;
    double t_offset = -e->L / r->beta0 * (phi_in - phi_out) / sd;
    if (rbend_rotation(r, z, phi_in)) return 1;
    rotate_about_y(phi_in, S);
    if (e->fringe) {
        real w[3], q[4];
        rbend_fringe_spin(r, b, +1, z, w);
        quat_from_rotation_vector(w, q);
        rotate_spin(q, S);
    }
    if (rbend_fringe_orbit(r, z, b, +1)) return 1;
    int N = e->n_slices;
    double ds = e->L / N;
    if (K < 0) {
        real Q[4];
        if (midpoint_rotation(r, e, z, N, ds, K, Q)) return 1;
        rotate_spin(Q, S);
        if (Q_out) memcpy(Q_out, Q, sizeof(Q));
    } else {
        real (*Om)[3] = (real (*)[3])malloc(sizeof(real[3]) * (size_t)(N + 1));
        if (!Om) return 2;
        int lost = omega(r, e, z, Om[0]);
        for (int i = 1; i <= N && !lost; ++i) {
            lost = rbend_body(r, z, b, ds);
            if (!lost) lost = omega(r, e, z, Om[i]);
        }
        if (!lost) {
            real Q[4];
            romberg_element_rotation((const real(*)[3])Om, N, ds, K, Q, levels_out);
            rotate_spin(Q, S);
            if (Q_out) memcpy(Q_out, Q, sizeof(Q));
        }
        free(Om);
        if (lost) return 1;
    }
    if (e->fringe) {
        real w[3], q[4];
        rbend_fringe_spin(r, b, -1, z, w);
        quat_from_rotation_vector(w, q);
        rotate_spin(q, S);
    }
    if (rbend_fringe_orbit(r, z, b, -1)) return 1;
    z->X -= x_offset;
    if (rbend_rotation(r, z, -phi_out)) return 1;
    rotate_about_y(-phi_out, S);
    z->T -= t_offset;
    return 0;
}

/* Track one particle through one element; the spin S is rotated by the
 * element's net rotation.  Returns 0, or 1 if the particle is lost. */
static int track_element(const orc_ref* r, const orc_element* e, orc_orbit* z, real S[3],
                         int K, real* levels_out, real* Q_out) {
    if (e->type == ORC_DRIFT)
        return drift(r, z, e->L);
    if (e->type == ORC_RBEND)
        return track_rbend(r, e, z, S, K, levels_out, Q_out);
    if (e->type == ORC_SNAKE) {
        /* orbit-transparent rotation by snake_mu about (sin phi, 0, cos phi) */
        real Q[4] = {cos(0.5 * e->snake_mu), sin(0.5 * e->snake_mu) * sin(e->snake_phi), 0.0,
                     sin(0.5 * e->snake_mu) * cos(e->snake_phi)};
        rotate_spin(Q, S);
        if (Q_out) memcpy(Q_out, Q, sizeof(Q));
        return 0;
    }
    int N = e->n_slices;
    /* a thin lens (Sec. 3.5) is the L -> 0 limit of the multipole at fixed
     * integrated strengths: in terms of t = s/L in [0, 1] its slices are
     * kicks of 1/N of the integrated field with no drift between them, and
     * Omega (Eq. (6b)) per unit t is that of the integrated field */
    double ds = e->type == ORC_THIN ? 1.0 / N : e->L / N;
    /* entrance fringe kick (orbit unchanged across the fringe) */
    if (element_fringe(r, e, +1, z, S)) return 1;
    if (K < 0) {
        real Q[4];
        if (midpoint_rotation(r, e, z, N, ds, K, Q)) return 1;
        rotate_spin(Q, S);
        if (Q_out) memcpy(Q_out, Q, sizeof(Q));
        return element_fringe(r, e, -1, z, S);
    }
    real (*Om)[3] = (real (*)[3])malloc(sizeof(real[3]) * (size_t)(N + 1));
    if (!Om) return 2;
    int lost = omega(r, e, z, Om[0]);
    for (int i = 1; i <= N && !lost; ++i) {
        lost = slice_map(r, e, z, ds);
        if (!lost) lost = omega(r, e, z, Om[i]);
    }
    if (!lost) {
        real Q[4];
        romberg_element_rotation((const real(*)[3])Om, N, ds, K, Q, levels_out);
        rotate_spin(Q, S);
        if (Q_out) memcpy(Q_out, Q, sizeof(Q));
        /* exit fringe kick */
        lost = element_fringe(r, e, -1, z, S);
    }
    free(Om);
    return lost;
}

/* ---------------------------------------------------------------------- */
/* exported entry points                                                  */
/* ---------------------------------------------------------------------- */

int orc_real_size(void) { return (int)sizeof(real); }

/* Validate a lattice as the tracker reads it: Romberg order k needs every
 * spin-carrying element's slice count divisible by 2^k; the midpoint schemes
 * (K = ORC_MID_HALF, ORC_MID_KICK) take any slice count but not the
 * fourth-order slice maps. */
int orc_check_lattice(const orc_element* els, int n_el, int K) {
    if (K < ORC_MID_KICK || K > ORC_MAX_ORDER) return -1;
    int div = K > 0 ? 1 << K : 1;
    for (int i = 0; i < n_el; ++i) {
        const orc_element* e = &els[i];
        if (e->type < 0 || e->type > ORC_THIN) return -1;
        if (e->type == ORC_MULT || e->type == ORC_QUAD_MK || e->type == ORC_SBEND || e->type == ORC_SOLENOID ||
            e->type == ORC_RBEND || e->type == ORC_TEAPOT || e->type == ORC_THIN) {
            if (e->n_slices < 1 || (e->n_slices % div) != 0) return -1;
            if ((e->L == 0.0) != (e->type == ORC_THIN)) return -1;
        }
        if (e->type == ORC_THIN && (e->fringe || e->split_order == 4)) return -1;
        if (e->type == ORC_SBEND && (e->angle == 0.0 || e->eta == 0.0)) return -1;
        if (e->type == ORC_TEAPOT && (e->angle == 0.0 || !(fabs(e->angle / e->n_slices) < 1.0))) return -1;
        if (K < 0 && e->split_order == 4) return -1;
        if (e->type == ORC_RBEND && (e->angle == 0.0 || e->eta == 0.0 || !(e->L > 0.0) ||
                                     fabs(0.5 * e->angle + e->e1) >= 1.5 || fabs(-0.5 * e->angle + e->e1) >= 1.5))
            return -1;
        if (e->fringe != 0 && e->fringe != 1) return -1;
        if (e->fringe && (e->type == ORC_DRIFT || e->type == ORC_SNAKE)) return -1;
        if (e->split_order != 0 && e->split_order != 2 && e->split_order != 4) return -1;
        if (e->split_order == 4 && e->type != ORC_MULT && e->type != ORC_QUAD_MK && e->type != ORC_TEAPOT) return -1;
    }
    return 0;
}

/* Track n particles for n_turns turns.  z is [6][n] (X, Px, Y, Py, T, Pt),
 * S is [3][n]; lost[n] flags (input and output).  Returns 0, or -1 for an
 * invalid lattice. */
int orc_track(const orc_element* els, int n_el, double G, double Ggamma0, long n,
              real* z, real* S, uint8_t* lost, int n_turns, int K, int n_threads) {
    if (orc_check_lattice(els, n_el, K)) return -1;
    orc_ref r = make_ref(G, Ggamma0);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (long p = 0; p < n; ++p) {
        if (lost[p]) continue;
        orc_orbit o = {z[0 * n + p], z[1 * n + p], z[2 * n + p], z[3 * n + p], z[4 * n + p], z[5 * n + p]};
        real s[3] = {S[0 * n + p], S[1 * n + p], S[2 * n + p]};
        int is_lost = 0;
        for (int t = 0; t < n_turns && !is_lost; ++t) {
            for (int i = 0; i < n_el; ++i) {
                orc_orbit o0 = o;
                real s0[3] = {s[0], s[1], s[2]};
                if (track_element(&r, &els[i], &o, s, K, NULL, NULL)) {
                    o = o0;
                    s[0] = s0[0]; s[1] = s0[1]; s[2] = s0[2];
                    is_lost = 1;
                    break;
                }
            }
        }
        z[0 * n + p] = o.X; z[1 * n + p] = o.Px; z[2 * n + p] = o.Y;
        z[3 * n + p] = o.Py; z[4 * n + p] = o.T; z[5 * n + p] = o.Pt;
        S[0 * n + p] = s[0]; S[1 * n + p] = s[1]; S[2 * n + p] = s[2];
        lost[p] = (uint8_t)is_lost;
    }
    return 0;
}

/* One particle (z6 in/out, S3 in/out) through one element, also returning the
 * trapezoid levels Q_00..Q_0K ([K+1][4], may be NULL) and the normalised
 * element rotation ([4], may be NULL).  Returns 0, 1 (lost) or -1. */
int orc_element_detail(const orc_element* e, double G, double Ggamma0, real* z6, real* S3,
                       int K, real* levels, real* Q) {
    if (orc_check_lattice(e, 1, K)) return -1;
    orc_ref r = make_ref(G, Ggamma0);
    orc_orbit o = {z6[0], z6[1], z6[2], z6[3], z6[4], z6[5]};
    int rc = track_element(&r, e, &o, S3, K, levels, Q);
    z6[0] = o.X; z6[1] = o.Px; z6[2] = o.Y; z6[3] = o.Py; z6[4] = o.T; z6[5] = o.Pt;
    return rc;
}

/* Orbit-only map of one element over its full length with its slicing
 * (n_slices slices; a negative L runs the map backwards).  Returns 0 / 1. */
int orc_orbit_map(const orc_element* e, double G, double Ggamma0, real* z6) {
    orc_ref r = make_ref(G, Ggamma0);
    orc_orbit o = {z6[0], z6[1], z6[2], z6[3], z6[4], z6[5]};
    int rc = 0;
    if (e->type == ORC_DRIFT) {
        rc = drift(&r, &o, e->L);
    } else if (e->type == ORC_SNAKE) {
        rc = 0;
    } else if (e->type == ORC_RBEND) {   /* the whole element: rotations, fringes, body, offsets */
        if (e->n_slices < 1) return -1;
        real S[3] = {0.0, 0.0, 1.0};
        rc = track_rbend(&r, e, &o, S, 0, NULL, NULL);
    } else {
        if (e->n_slices < 1) return -1;
        double ds = e->type == ORC_THIN ? 1.0 / e->n_slices : e->L / e->n_slices;
        for (int i = 0; i < e->n_slices && !rc; ++i) rc = slice_map(&r, e, &o, ds);
    }
    z6[0] = o.X; z6[1] = o.Px; z6[2] = o.Y; z6[3] = o.Py; z6[4] = o.T; z6[5] = o.Pt;
    return rc;
}

/* Individual sub-flows, for the tests that pin them one by one:
 * which = 0 drift, 1 multipole kick, 2 quadrupole linear flow H_qL,
 *         3 quadrupole nonlinear flow H_qNL, 4 sector bend, 5 solenoid body
 *         (k1 = b0/(B rho)), 6 rectangular-bend body (k1 = b1/(B rho)),
 *         7 dynamic rotation by the angle s, 8 rectangular-bend fringe orbit map
 *         (k1 = b1/(B rho), sign of k2 = entrance/exit), 9 TEAPOT curved drift,
 *         10 TEAPOT kick of a sector bend (h, eta). */
int orc_subflow(int which, double G, double Ggamma0, real* z6, double s, double k1, double k2,
                double h, double eta) {
    orc_ref r = make_ref(G, Ggamma0);
    orc_orbit o = {z6[0], z6[1], z6[2], z6[3], z6[4], z6[5]};
    int rc = 0;
    switch (which) {
    case 0: rc = drift(&r, &o, s); break;
    case 1: mult_kick(&o, k1, k2, s); break;
    case 2: quad_linear(&r, &o, k1, s); break;
    case 3: rc = quad_nonlinear(&r, &o, s); break;
    case 4: rc = sbend_map(&r, &o, h, eta, s); break;
    case 5: rc = solenoid_map(&r, &o, k1, s); break;
    case 6: rc = rbend_body(&r, &o, k1, s); break;                 /* k1 = b1/(B rho) */
    case 7: rc = rbend_rotation(&r, &o, s); break;                 /* s = phi */
    case 8: rc = rbend_fringe_orbit(&r, &o, k1, k2 > 0.0 ? 1 : -1); break;   /* k1 = b1/(B rho), k2 = sign */
    case 9: rc = curved_drift(&r, &o, h, s); break;                /* TEAPOT drift, curvature h */
    case 10: teapot_kick(&o, h, eta, s); break;                    /* TEAPOT kick, curvature h, eta */
    default: return -1;
    }
    z6[0] = o.X; z6[1] = o.Px; z6[2] = o.Y; z6[3] = o.Py; z6[4] = o.T; z6[5] = o.Pt;
    return rc;
}

/* Precession vector Omega of Eq. (6b) at state z6 inside element e. */
int orc_omega(const orc_element* e, double G, double Ggamma0, const real* z6, real* out3) {
    orc_ref r = make_ref(G, Ggamma0);
    orc_orbit o = {z6[0], z6[1], z6[2], z6[3], z6[4], z6[5]};
    return omega(&r, e, &o, out3);
}

/* Rotation vector of a solenoid fringe (sign +1 entrance, -1 exit) at z6. */
int orc_solenoid_fringe(double ks, int sign, double G, double Ggamma0, const real* z6, real* out3) {
    orc_ref r = make_ref(G, Ggamma0);
    orc_orbit o = {z6[0], z6[1], z6[2], z6[3], z6[4], z6[5]};
    return solenoid_fringe(&r, ks, sign, &o, out3);
}

/* Rotation vector of the thin fringe spin kick of element e (sign +1
 * entrance, -1 exit) at z6: Eq. (skfringe) for dipoles and multipoles whatever
 * their fringe flag, Eq. (solFringe) for solenoids.  Returns 0, 1 (lost), -1. */
int orc_element_fringe(const orc_element* e, int sign, double G, double Ggamma0, const real* z6, real* out3) {
    orc_ref r = make_ref(G, Ggamma0);
    orc_orbit o = {z6[0], z6[1], z6[2], z6[3], z6[4], z6[5]};
    if (e->type == ORC_SOLENOID) return solenoid_fringe(&r, e->k1, sign, &o, out3);
    if (e->type == ORC_RBEND) {   /* in the magnet's Cartesian frame */
        double pi_, po_, b;
        rbend_geometry(e, &pi_, &po_, &b);
        rbend_fringe_spin(&r, b, sign, &o, out3);
        return 0;
    }
    if (e->type != ORC_MULT && e->type != ORC_QUAD_MK && e->type != ORC_SBEND && e->type != ORC_TEAPOT) return -1;
    multipole_fringe(&r, e, sign, &o, out3);
    return 0;
}
