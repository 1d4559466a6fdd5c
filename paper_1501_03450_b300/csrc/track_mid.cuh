// FP64 tracker with midpoint spin integration: piece-wise constant rotations
// R(ds Omega) with Omega (Eq. (6b)) taken at the middle of each slice (Sec.
// 4.1, Eq. (37)), the spin schemes the paper compares in Sec. 5.3
// (Fig. oneTurnSpinErrs):
//   KICK = false  each slice is traversed as two half-slices of its own map,
//                 the rotation between them ("half-DKD, spin, half-DKD");
//   KICK = true   drift-kick (multipole, TEAPOT bend) and matrix-kick slices
//                 keep their map and rotate the spin between the two halves
//                 of the central kick ("half-drift, half-kick, spin,
//                 half-kick, half-drift"); exact maps (sector and rectangular
//                 bend bodies, solenoid) as for KICK = false.
// Same state layout, staging, loss rule and per-turn spin composition as the
// Romberg tracker of track_fp64.cuh, whose orbit-map helpers it uses; second-
// order slice maps only (the host rejects fourth-order elements).
#pragma once

#include "track_fp64.cuh"

namespace st {

// Exact sector-bend map over len (Eq. (10)) for the midpoint tracker, in the
// rotation form of the Romberg tracker: (Px, A = Ps - eta (1 + hX)) turns by
// h len (cb, sb = its cos, sin); X from Ps_f - A_f = eta (1 + h X_f).
// P_a^2 = P^2 - Py^2 is a constant of the bend (Eq. (8)), so Pa2 and 1/Pa2
// come from the caller, and Ps (in: at the entrance, out: at the exit) is
// carried from step to step.  Returns false if Ps^2 <= 0 at the exit.
__device__ __forceinline__ bool sbend_step(Particle& p, const PConst& pc, const RefConst& ref, double h, double eta,
                                           double ieh, double ieta, double cb, double sb, double len, double Pa2,
                                           double iPa2, double& Ps) {
    const double Psi = Ps;
    const double A = Psi - eta * fma(h, p.X, 1.0);
    const double Pxi = p.Px;
    const double Pxf = Pxi * cb + A * sb;
    const double Af = A * cb - Pxi * sb;
    const double qf = Pa2 - Pxf * Pxf;
    if (!(qf > 0.0)) return false;
    const double Psf = sqrt(qf);
    // asin(Px_i/P_a) - asin(Px_f/P_a) = asin((Px_i Ps_f - Px_f Ps_i)/P_a^2),
    // by its Taylor series when small (truncation < 1e-21 relative)
    const double sd = (Pxi * Psf - Pxf * Psi) * iPa2;
    double dpsi;
    if ((__double2hiint(sd) & 0x7fffffff) < 0x3f847ae1) {   // |sd| < 1e-2, integer test
        const double x2 = sd * sd;
        dpsi = sd * fma(x2, fma(x2, fma(x2, fma(x2, 35.0 / 1152.0, 5.0 / 112.0), 3.0 / 40.0), 1.0 / 6.0), 1.0);
    } else {
        dpsi = asin(sd);
    }
    p.X = (Psf - eta - Af) * ieh;
    p.Px = Pxf;
    p.Y += ieta * p.Py * len + ieh * p.Py * dpsi;
    p.T += -ieta * pc.Pt * len + (1.0 - ieta) * len * ref.inv_beta0 - ieh * pc.b0pt * dpsi;
    Ps = Psf;
    return true;
}

// Precession vector at the current state of element el (Eq. (6b)): transverse
// field of a multipole, quadrupole or thin lens (per unit kick parameter), vertical field eta h with curvature h in
// sector and TEAPOT bends, b1/(B rho) in a rectangular bend's straight frame.
// Returns false if Ps^2 <= 0.
__device__ __forceinline__ bool mid_omega(const DevElem& el, int type, const Particle& p, const PConst& pc,
                                          double& ox, double& oy, double& os) {
    const double pp = p.Px * p.Px + p.Py * p.Py;
    if (!(pc.P2 - pp > 0.0)) return false;
    const double ips = rsqrt(pc.P2 - pp);
    const double Ps = (pc.P2 - pp) * ips;
    double bx = 0.0, by = 0.0, h = 0.0;
    if (type == ST_SBEND || type == ST_TEAPOT) {
        h = el.a[0];
        by = el.a[1] * el.a[0];
    } else if (type == ST_RBEND) {
        by = el.a[0];
    } else {
        const double k1 = el.a[0], k2 = (type == ST_MULT || type == ST_THIN_MULT) ? el.a[1] : 0.0;
        bx = k1 * p.Y + k2 * p.X * p.Y;
        by = k1 * p.X + 0.5 * k2 * (p.X * p.X - p.Y * p.Y);
    }
    precession(p, pc, bx, by, h, ips, Ps, ox, oy, os);
    return true;
}

template <bool KICK>
__device__ __forceinline__ void fp64_track_particle_mid(const DevElem* __restrict__ table,
                                                        const uint16_t* __restrict__ seq, int n_seq,
                                                        const RefConst& ref, double2* __restrict__ xpx,
                                                        double2* __restrict__ ypy, double2* __restrict__ tpt,
                                                        double2* __restrict__ sxy, double* __restrict__ szp,
                                                        uint8_t* __restrict__ lost, int64_t i, int n_turns,
                                                        double* qcache, const TurnOut& tq, int32_t* status) {
    const int n_table = (int)(((const char*)seq - (const char*)table) / sizeof(DevElem));
    Particle p;
    PConst pc;
    double sx, sy, sz;
    load_particle(ref, xpx, ypy, tpt, sxy, szp, i, p, pc, sx, sy, sz);
    const double onepG = 1.0 + ref.G;

    QuadCache qc;
    qc.key_k = -1.0;
    qc.key_s = 0.0;
    qc.col = &qcache[threadIdx.x];
    qc.stride = blockDim.x;
    bool is_lost = false;

    for (int turn = 0; turn < n_turns && !is_lost; ++turn) {
        Quat qt{1.0, 0.0, 0.0, 0.0};
        for (int e = 0; e < n_seq; ++e) {
            const int idx = seq[e];
            if constexpr (kChecked) {
                if (idx >= n_table) {
                    if (status) atomicExch(status, STATUS_BOUNDS);
                    is_lost = true;
                    break;
                }
            }
            const DevElem& el = table[idx];
            const int type = el.type;
            if (type == ST_SNAKE) {
                qt = qmul(Quat{el.a[0], el.a[1], el.a[2], el.a[3]}, qt);
                continue;
            }
            const Particle p0 = p;
            if (type == ST_DRIFT) {
                const double ps2 = pc.P2 - p.Px * p.Px - p.Py * p.Py;
                if (!(ps2 > 0.0)) {
                    is_lost = true;
                    break;
                }
                const double ips = rsqrt(ps2);
                p.X += el.ds * p.Px * ips;
                p.Y += el.ds * p.Py * ips;
                p.T += el.ds * (ref.inv_beta0 - pc.b0pt * ips);
                continue;
            }
            const int N = el.n_slices;
            const double ds = el.ds, hd = 0.5 * ds;
            Quat q_in{1.0, 0.0, 0.0, 0.0}, q_out{1.0, 0.0, 0.0, 0.0}, qe{1.0, 0.0, 0.0, 0.0};
            const bool fringe = (el.flags & ST_ELEM_FRINGE) && type != ST_RBEND;
            if (fringe) q_in = multipole_fringe_quat(el, type, onepG, p, 1.0);
            bool ok = true;
            double ox, oy, os;
            if (type == ST_SOLENOID) {
                // exact body map over half-slices; Ps of the kinetic momentum
                // is conserved, Omega along it as in the Romberg tracker
                const double ks = el.a[0], eta = el.a[1];
                double kx = p.Px + eta * p.Y, ky = p.Py - eta * p.X;
                const double ps2 = pc.P2 - kx * kx - ky * ky;
                if (!(ps2 > 0.0)) {
                    is_lost = true;
                    break;
                }
                const double iPs = rsqrt(ps2), Ps = ps2 * iPs;
                const double f = pc.c * ks * pc.invP2;
                ok = solenoid_fringe_quat(pc, p, ks, el.a[2], 1.0, q_in);
                const double kds = eta * iPs * hd;
                double sn, cs;
                sincos(kds, &sn, &cs);
                const double a12 = fabs(kds) > 1e-4 ? sn / eta
                                                    : hd * iPs * (1.0 - kds * kds * (1.0 / 6.0 - kds * kds / 120.0));
                const double a21 = -eta * sn;
                const double dT = hd * (ref.inv_beta0 - pc.b0pt * iPs);
                for (int s = 0; s < 2 * N; ++s) {
                    const double X1 = cs * p.X + a12 * p.Px, Px1 = a21 * p.X + cs * p.Px;
                    const double Y1 = cs * p.Y + a12 * p.Py, Py1 = a21 * p.Y + cs * p.Py;
                    p.X = cs * X1 + sn * Y1;
                    p.Y = cs * Y1 - sn * X1;
                    p.Px = cs * Px1 + sn * Py1;
                    p.Py = cs * Py1 - sn * Px1;
                    p.T += dT;
                    if ((s & 1) == 0) {   // slice middle
                        kx = p.Px + eta * p.Y;
                        ky = p.Py - eta * p.X;
                        qe = qmul(quat_from_rotvec(ds * f * kx, ds * f * ky, ds * (f * Ps - pc.a * ks * iPs)), qe);
                    }
                }
                ok = solenoid_fringe_quat(pc, p, ks, el.a[2], -1.0, q_out) && ok;
            } else if (type == ST_SBEND) {
                const double h = el.a[0], eta = el.a[1], ieh = el.a[4], ieta = el.a[5];
                double sb, cb;
                sincos(h * hd, &sb, &cb);
                const double Pa2 = pc.P2 - p.Py * p.Py, iPa2 = 1.0 / Pa2;
                const double qi = Pa2 - p.Px * p.Px;
                ok = qi > 0.0;
                double Ps = sqrt(qi);
                for (int s = 0; s < N && ok; ++s) {
                    ok = sbend_step(p, pc, ref, h, eta, ieh, ieta, cb, sb, hd, Pa2, iPa2, Ps);
                    // Omega (Eq. (6b)) with the bend's field and curvature
                    precession(p, pc, 0.0, eta * h, h, 1.0 / Ps, Ps, ox, oy, os);
                    qe = qmul(quat_from_rotvec(ds * ox, ds * oy, ds * os), qe);
                    ok = ok && sbend_step(p, pc, ref, h, eta, ieh, ieta, cb, sb, hd, Pa2, iPa2, Ps);
                }
            } else if (type == ST_TEAPOT) {
                // KICK: D(ds/2) K(ds/2) | K(ds/2) D(ds/2); half-slices:
                // D(ds/4) K(ds/2) D(ds/4) | D(ds/4) K(ds/2) D(ds/4)
                const double h = el.a[0], etah = el.a[1] * el.a[0], ih = 1.0 / h;
                const CurvedDrift d = curved_drift_consts(h, ih, KICK ? hd : 0.5 * hd);
                for (int s = 0; s < N; ++s) {
                    ok = curved_drift(p, pc, ref, d) && ok;
                    teapot_kick(p, h, etah, hd);
                    if constexpr (!KICK) ok = curved_drift(p, pc, ref, d) && ok;
                    ok = mid_omega(el, type, p, pc, ox, oy, os) && ok;
                    qe = qmul(quat_from_rotvec(ds * ox, ds * oy, ds * os), qe);
                    if constexpr (!KICK) ok = curved_drift(p, pc, ref, d) && ok;
                    teapot_kick(p, h, etah, hd);
                    ok = curved_drift(p, pc, ref, d) && ok;
                }
            } else if (type == ST_MULT) {
                const double k1 = el.a[0], k2 = el.a[1];
                const double dl = KICK ? hd : 0.5 * hd;   // drift length of a half step
                for (int s = 0; s < N; ++s) {
                    for (int half = 0; half < 2; ++half) {
                        if (half == 1) {
                            ok = mid_omega(el, type, p, pc, ox, oy, os) && ok;
                            qe = qmul(quat_from_rotvec(ds * ox, ds * oy, ds * os), qe);
                        }
                        double pp = p.Px * p.Px + p.Py * p.Py;
                        ok = (pc.P2 - pp > 0.0) && ok;
                        if (!KICK || half == 0) dkd_drift(p, pc, ref, rsqrt(pc.P2 - pp), dl);
                        mult_kick(p, k1, k2, hd);
                        pp = p.Px * p.Px + p.Py * p.Py;
                        ok = (pc.P2 - pp > 0.0) && ok;
                        if (!KICK || half == 1) dkd_drift(p, pc, ref, rsqrt(pc.P2 - pp), dl);
                    }
                }
            } else if (type == ST_THIN_MULT) {
                // thin lens: half of the slice's partial kick on each side
                for (int s = 0; s < N; ++s) {
                    mult_kick(p, el.a[0], el.a[1], hd);
                    ok = mid_omega(el, type, p, pc, ox, oy, os) && ok;
                    qe = qmul(quat_from_rotvec(ds * ox, ds * oy, ds * os), qe);
                    mult_kick(p, el.a[0], el.a[1], hd);
                }
            } else if (type == ST_QUAD_MK) {
                // KICK: L(ds/2) N(ds/2) | N(ds/2) L(ds/2); half-slices:
                // L(ds/4) N(ds/2) L(ds/4) | L(ds/4) N(ds/2) L(ds/4)
                const double k1 = el.a[0], absk = el.a[1];
                const double ll = KICK ? hd : 0.5 * hd;
                if (qc.key_k != absk || qc.key_s != ll) quad_coeffs(qc, pc, absk, ll);
                for (int s = 0; s < N; ++s) {
                    quad_linear(p, pc, qc, k1);
                    quad_nonlinear(p, pc, ref, hd);
                    if constexpr (!KICK) quad_linear(p, pc, qc, k1);
                    ok = mid_omega(el, type, p, pc, ox, oy, os) && ok;
                    qe = qmul(quat_from_rotvec(ds * ox, ds * oy, ds * os), qe);
                    if constexpr (!KICK) quad_linear(p, pc, qc, k1);
                    quad_nonlinear(p, pc, ref, hd);
                    quad_linear(p, pc, qc, k1);
                }
            } else if (type == ST_RBEND) {
                // as in the Romberg tracker, with the body in half-slices
                const double b = el.a[0];
                ok = rbend_rotation(p, pc, el.a[1]);
                q_in = quat_about_y(el.a[1]);
                if (el.flags & ST_ELEM_FRINGE) q_in = qmul(rbend_fringe_quat(pc, onepG, p, b), q_in);
                ok = ok && rbend_fringe_orbit(p, pc, b);
                for (int s = 0; s < N; ++s) {
                    ok = ok && rbend_body(p, pc, b, hd);
                    ok = ok && mid_omega(el, type, p, pc, ox, oy, os);
                    if (ok) qe = qmul(quat_from_rotvec(ds * ox, ds * oy, ds * os), qe);
                    ok = ok && rbend_body(p, pc, b, hd);
                }
                if (el.flags & ST_ELEM_FRINGE) q_out = rbend_fringe_quat(pc, onepG, p, -b);
                ok = ok && rbend_fringe_orbit(p, pc, -b);
                p.X -= el.a[3];
                ok = ok && rbend_rotation(p, pc, el.a[2]);
                q_out = qmul(quat_about_y(el.a[2]), q_out);
                p.T += el.a[4] * ref.inv_beta0;
            }
            if (fringe) q_out = multipole_fringe_quat(el, type, onepG, p, -1.0);
            if (!ok || !all_finite(p, qe.w, qe.x, qe.y, qe.z)) {
                p = p0;
                is_lost = true;
                break;
            }
            qt = qmul(q_out, qmul(qe, qmul(q_in, qt)));
        }
        end_turn(qt, sx, sy, sz, tq, i);
    }
    store_particle(p, sx, sy, sz, is_lost, xpx, ypy, tpt, sxy, szp, lost, i);
}

}  // namespace st
