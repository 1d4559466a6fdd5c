// Mixed-precision tracker with midpoint spin integration (Sec. 4.1, Eq. (37);
// the schemes the paper compares in Sec. 5.3): piece-wise constant rotations
// R(ds Omega) with Omega (Eq. (6b)) taken at the middle of each slice, in the
// compensated FP32 arithmetic of track_mixed.cuh:
//   KICK = false  each slice as two half-slices of its own map, the rotation
//                 between them;
//   KICK = true   drift-kick (multipole, thin lens, TEAPOT bend) and
//                 matrix-kick slices keep their map and rotate between the two
//                 halves of the central kick; sector bends (exact maps) as for
//                 KICK = false.
// Element by element the same placements as the FP64 midpoint tracker
// (track_mid.cuh) on the element kinds the mixed tracker runs.  The rotation
// of a slice is split into the on-axis reference rotation (about y in bends,
// identity elsewhere) and a near-identity deviation, as the Romberg path splits
// its edge rotations: in a bend every slice's reference rotation is
// q(ds Omega_ref), so the deviation of slice i is conjugated by the reference
// rotation of the i slices before it (angle Omega_ref i ds, the table's edge
// i entry) and the element rotation is R_L (product of the deviations).
// The product is normalised once per element and composed into the
// compensated turn quaternion; FP64 once per turn.  A separate instantiation,
// so that the Romberg kernel keeps its code and register budget.
#pragma once

#include "track_mixed.cuh"

namespace st {

// Constants of one exact bend step (Eq. (10)) of length len, compensated:
// sin(h len), sin(h len)/(eta h), cos(h len) - 1, (cos(h len) - 1)/(eta h),
// len/eta, and the step's T increment without the path term,
// (1 - 1/eta) len/beta0 - Pt len/eta.
struct MixBendStep {
    FF sb, sbieh, cbm1, cbmieh, ietads, dT0;
};

// The exact bend over one step in the increment form of the Romberg path's
// slice (same compensation), carrying the momentum quantities of the step's
// end (px, ps2, ips, Ps, dPsP = Ps - P, PsM1 = Ps - 1) to the next step.
__device__ __forceinline__ void mixed_bend_step(MState& z, const MConst& k, const MixBendStep& c, float etah, bool eta1,
                                                const FF& omeff, const FF& etahff, const FF& iehff, const FF& iPa2ff,
                                                float py, float Pa2, float& px, float& ps2, float& ips, float& Ps,
                                                float& dPsP, FF& PsM1) {
    FF PsE = PsM1;
    if (!eta1) PsE = ff_add(PsM1, omeff);
    const FF Aff = ff_add(PsE, ff_neg(ff_mul(etahff, z.X)));   // A = Ps - eta (1 + h X)
    const FF dPxff = ff_add(ff_mul(Aff, c.sb), ff_mul(z.Px, c.cbm1));
    const FF dPxieh = ff_mul(dPxff, iehff);
    const float pxf = px + dPxff.hi;
    const float ps2f = Pa2 - pxf * pxf;
    const float ipsf = rsqrtf(ps2f);
    const float Psf = ps2f * ipsf;
    const float dPsPf = -__fdividef(pxf * pxf + py * py, Psf + k.P);
    const FF PsfM1 = ff_add_f(k.PM1, dPsPf);
    // Q = (Ps_f - Ps)/(eta h) = -dPx/(eta h) (Px + Px_f) / (Ps + Ps_f)
    const float hu = 0.5f * (PsM1.hi + PsfM1.hi);
    const FF invden = ff_add_f(FF{0.5f, 0.0f}, -0.5f * hu * fmaf(hu, hu - 1.0f, 1.0f));
    const FF pxsum = ff_add(ff_scale2(z.Px, 2.0f), dPxff);
    const FF Q = ff_neg(ff_mul(ff_mul(dPxieh, pxsum), invden));
    // sin(psi_i - psi_f)/(eta h) = (Px Q - dPx/(eta h) Ps) / P_a^2
    const FF Psff = ff_add_f(PsM1, 1.0f);
    const FF sdieh = ff_mul(ff_add_f(ff_neg(ff_mul(dPxieh, Psff)), px * Q.hi), iPa2ff);
    const float sd = sdieh.hi * etah;
    FF dpsieh;   // (psi_i - psi_f)/(eta h)
    if (fabsf(sd) < 1e-2f) {
        const float x2 = sd * sd;
        dpsieh = ff_add_f(sdieh, sdieh.hi * x2 * fmaf(x2, 3.0f / 40.0f, 1.0f / 6.0f));
    } else {
        dpsieh = FF{asinf(sd) / etah, 0.0f};
    }
    const FF dX = ff_add(ff_add(ff_mul(z.Px, c.sbieh), ff_neg(ff_mul(Aff, c.cbmieh))), Q);
    const FF dY = ff_mul(z.Py, ff_add(c.ietads, dpsieh));
    z.X = ff_add(z.X, dX);
    z.Px = ff_add(z.Px, dPxff);
    z.Y = ff_add(z.Y, dY);
    z.T = ff_add(z.T, ff_add(c.dT0, ff_neg(ff_mul(k.b0ptf, dpsieh))));
    px = pxf;
    ps2 = ps2f;
    ips = ipsf;
    Ps = Psf;
    dPsP = dPsPf;
    PsM1 = PsfM1;
}

template <bool KICK, bool FR = false, bool EXT = false, bool RB = false>
__device__ __forceinline__ void mixed_track_particle_mid(const MixElem* __restrict__ table,
                                                         const uint16_t* __restrict__ seq,
                                                         const float2* __restrict__ rho, int n_seq,
                                                         const RefConst& ref, double2* __restrict__ xpx,
                                                         double2* __restrict__ ypy, double2* __restrict__ tpt,
                                                         double2* __restrict__ sxy, double* __restrict__ szp,
                                                         uint8_t* __restrict__ lost, int64_t i, int n_turns,
                                                         int32_t* status, double* __restrict__ spin_sum, int64_t n_all) {
    const int n_table = (int)(((const char*)seq - (const char*)table) / sizeof(MixElem));
    MState z;
    double2 v = xpx[i];
    z.X = ff_make(v.x);
    z.Px = ff_make(v.y);
    v = ypy[i];
    z.Y = ff_make(v.x);
    z.Py = ff_make(v.y);
    v = tpt[i];
    z.T = ff_make(v.x);
    const double Pt = v.y;
    MConst k;
    double invP64;
    mixed_particle_consts(ref, Pt, k, invP64);
    v = sxy[i];
    double sx = v.x, sy = v.y, sz = szp[i];
    MQuad mq;
    mq.key_k = -1.0f;
    mq.key_s = 0.0f;
    bool is_lost = false;
    const CNQ one{0.0f, FF{0.0f, 0.0f}, FF{0.0f, 0.0f}, FF{0.0f, 0.0f}};

    for (int turn = 0; turn < n_turns && !is_lost; ++turn) {
        FQ qt{FF{1.0f, 0.0f}, FF{0.0f, 0.0f}, FF{0.0f, 0.0f}, FF{0.0f, 0.0f}};
        for (int e = 0; e < n_seq; ++e) {
            const int idx = seq[e];
            if constexpr (kChecked) {
                if (idx >= n_table) {
                    if (status) atomicExch(status, STATUS_BOUNDS);
                    is_lost = true;
                    break;
                }
            }
            const MixElem& el = table[idx];
            const int type = FR ? (el.type & 0xff) : el.type;
            if (type == ST_SNAKE) {
                fq_premul_ref(qt, el.rq);
                continue;
            }
            const MState z0 = z;
            if constexpr (RB) {
                if (type == ST_RBEND) {   // in FP64, the body in half-slices (an exact map)
                    const RbendOut o = mixed_rbend_fp64<0, true, true>(z, ref, Pt, &el.d64);
                    if (!o.ok) {
                        is_lost = true;
                        break;
                    }
                    z = o.z;
                    fq_premul_quat64(qt, o.r);
                    continue;
                }
            }
            float d, pp;
            if (type == ST_DRIFT) {
                const FF ips = inv_ps(k, z.Px.hi, z.Py.hi, d, pp);
                drift_inc(z, k, FF{el.ds_ff.x, el.ds_ff.y}, ips, d);
                if (!isfinite(z.X.hi + z.Y.hi + z.T.hi)) {
                    z = z0;
                    is_lost = true;
                    break;
                }
                continue;
            }
            const int N = el.n_slices;
            const float ds = el.ds;
            const FF dsff{el.ds_ff.x, el.ds_ff.y};   // the slice's drift length (0 for a thin lens)
            CNQ D = one;                              // product of the slices' deviations, later on the left
            const bool teapot = EXT && type == ST_TEAPOT;
            if (type == ST_SBEND || teapot) {
                const float h = el.h, eta = el.eta, etah = eta * h;
                const float py = z.Py.hi;
                const float Pa2 = k.P2 - py * py;
                float px = z.Px.hi;
                float ps2 = Pa2 - px * px;
                float ips = rsqrtf(ps2);
                float Ps = ps2 * ips;
                float dPsP = -__fdividef(px * px + py * py, Ps + k.P);
                FF PsM1 = ff_add_f(k.PM1, dPsP);
                const float cu = k.c * py * etah * k.invPf * k.invPf;
                const FF etahff{el.etah_ff.x, el.etah_ff.y};
                const FF omeff{el.ome_ff.x, el.ome_ff.y};
                const bool eta1 = el.ome_ff.x == 0.0f;
                const FF iehff{el.ieh_ff.x, el.ieh_ff.y};
                const FF ietadsh{el.ietadsh_ff.x, el.ietadsh_ff.y};
                MixBendStep half;
                half.sb = FF{el.sbh_ff.x, el.sbh_ff.y};
                half.sbieh = FF{el.sbiehh_ff.x, el.sbiehh_ff.y};
                half.cbm1 = FF{el.cbm1h_ff.x, el.cbm1h_ff.y};
                half.cbmieh = FF{el.cbmiehh_ff.x, el.cbmiehh_ff.y};
                half.ietads = ietadsh;
                half.dT0 = ff_add(FF{el.dTetah_ff.x, el.dTetah_ff.y}, ff_neg(ff_mul(k.Ptf, ietadsh)));
                const float epy = py * py * k.invPf * k.invPf;
                const FF iPa2ff = ff_add_f(k.invP2, k.invP2.hi * epy * (1.0f + epy));
                // deviation of Omega from the on-axis reference, as in the Romberg path
                const FF B0 = ff_mul(etahff, k.c1P);
                const FF B1 = ff_mul(FF{el.eh2_ff.x, el.eh2_ff.y}, k.a0P);
                const float apda = k.a0 + k.da;
                const float2* rh = rho + el.rho_off;
                // TEAPOT: KICK: D(ds/2) K(ds/2) | K(ds/2) D(ds/2); half-slices:
                // D(ds/4) K(ds/2) D(ds/4) | D(ds/4) K(ds/2) D(ds/4)
                const MixCurvedDrift& cd = el.td[KICK ? 0 : 1];
                const FF hehl{0.5f * el.ehl_ff.x, 0.5f * el.ehl_ff.y};
                const FF hehlh{0.5f * el.ehlh_ff.x, 0.5f * el.ehlh_ff.y};
                for (int s = 0; s < N; ++s) {
                    if (teapot) {
                        mixed_curved_drift(z, k, cd, h);
                        mixed_teapot_kick(z, hehl, hehlh);
                        if constexpr (!KICK) mixed_curved_drift(z, k, cd, h);
                        px = z.Px.hi;
                        ps2 = Pa2 - px * px;
                        ips = rsqrtf(ps2);
                        Ps = ps2 * ips;
                        dPsP = -__fdividef(px * px + py * py, Ps + k.P);
                    } else {
                        mixed_bend_step(z, k, half, etah, eta1, omeff, etahff, iehff, iPa2ff, py, Pa2, px, ps2, ips,
                                        Ps, dPsP, PsM1);
                    }
                    // slice middle: ds (Omega - Omega_ref)
                    const float hX = h * z.X.hi;
                    const float g = (1.0f + hX) * ips;
                    const float dd = -dPsP * k.invPf * ips;
                    const float Nf = k.c1 + k.a0 * dPsP - hX * apda;
                    const float rest = etah * ((k.a0 * dPsP - hX * k.da) * k.invPf + Nf * dd) + g * cu * py;
                    const FF doy = ff_addn(ff_add(B0, ff_neg(ff_mul(B1, z.X))), rest);
                    CNQ e = cnq_deviation(el.w[1], ds * (g * cu * px), ff_mul(FF{el.ds_ff.x, el.ds_ff.y}, doy),
                                          ds * (g * cu * Ps));
                    // conjugated by the reference rotation of the s slices before it
                    const float2 r = rh[s];
                    const float ex = e.x.hi * r.x - e.z.hi * r.y;
                    const float ez = e.x.hi * r.y + e.z.hi * r.x;
                    e.x = FF{ex, 0.0f};
                    e.z = FF{ez, 0.0f};
                    D = cnq_mul(e, D);
                    if (teapot) {
                        if constexpr (!KICK) mixed_curved_drift(z, k, cd, h);
                        mixed_teapot_kick(z, hehl, hehlh);
                        mixed_curved_drift(z, k, cd, h);
                    } else {
                        mixed_bend_step(z, k, half, etah, eta1, omeff, etahff, iehff, iPa2ff, py, Pa2, px, ps2, ips,
                                        Ps, dPsP, PsM1);
                    }
                }
            } else if (EXT && type == ST_SOLENOID) {
                // exact body map over half-slices, Omega at the slice middle along the
                // kinetic momentum (its Ps conserved in the body), the deviation in the
                // relabelled frame (y, s, x) as in the Romberg kernel
                const FF eta{el.seta_ff.x, el.seta_ff.y}, ks{el.ks_ff.x, el.ks_ff.y};
                const FF kx = ff_add(z.Px, ff_mul(eta, z.Y)), ky = ff_add(z.Py, ff_neg(ff_mul(eta, z.X)));
                FF dPsPk, dk;
                ps_deviations(k, kx, ky, dPsPk, dk);
                const MSolSlice m =
                    mixed_solenoid_slice(eta, 0.5 * ((double)el.ds_ff.x + (double)el.ds_ff.y), invP64, dk.hi);
                const FF hdff{0.5f * dsff.hi, 0.5f * dsff.lo};
                const FF f = ff_mul(k.cP2, ks);
                const FF ks1G{el.ks1G_ff.x, el.ks1G_ff.y};
                const float2* rh = rho + el.rho_off;
                for (int s = 0; s < N; ++s) {
                    mixed_solenoid_map(z, k, m, hdff, dk.hi);
                    float oxt, ozt;
                    FF oyt;
                    solenoid_dev_omega(k, z, eta, f, ks1G, ks.hi, dPsPk.hi, dk.hi, oxt, oyt, ozt);
                    CNQ e = cnq_deviation(el.w[1], ds * oxt, ff_mul(dsff, oyt), ds * ozt);
                    const float2 r = rh[s];
                    const float ex = e.x.hi * r.x - e.z.hi * r.y;
                    const float ez = e.x.hi * r.y + e.z.hi * r.x;
                    e.x = FF{ex, 0.0f};
                    e.z = FF{ez, 0.0f};
                    D = cnq_mul(e, D);
                    mixed_solenoid_map(z, k, m, hdff, dk.hi);
                }
            } else {   // ST_MULT (drift-kick-drift; thin lenses too) or ST_QUAD_MK (matrix-kick)
                const bool is_mult = type == ST_MULT;
                const float k1 = el.k1;
                const float k2 = is_mult ? el.k2 : 0.0f;
                const FF k1ds{el.k1ds_ff.x, el.k1ds_ff.y};   // quadrupoles: |k1|
                const FF hk1{0.5f * el.k1ds_ff.x, 0.5f * el.k1ds_ff.y};      // half kick (multipole)
                const FF hk2h{0.5f * el.k2h_ff.x, 0.5f * el.k2h_ff.y};
                const FF hk2{0.5f * el.k2ds_ff.x, 0.5f * el.k2ds_ff.y};
                // drift of a half step: ds/2 around the split kick, ds/4 in half-slices
                const float pdl = KICK ? 0.5f : 0.25f;
                const FF dl{pdl * dsff.hi, pdl * dsff.lo};
                const FF zero{0.0f, 0.0f};
                FF Aw;   // (a/P) k1 ds, the first-order rotation per unit Y (x) and X (y) of a slice
                const float hd = 0.5f * ds;
                if (is_mult) {
                    Aw = ff_mul(k.aP, k1ds);
                } else {
                    const float absk = el.k2, ll = KICK ? hd : 0.5f * hd;
                    if (mq.key_k != absk || mq.key_s != ll)
                        mquad_coeffs(mq, invP64, (double)el.k1ds_ff.x + (double)el.k1ds_ff.y,
                                     (KICK ? 0.5 : 0.25) * ((double)el.ds_ff.x + (double)el.ds_ff.y), absk, ll);
                    Aw = ff_mul_f(ff_mul(ff_mul(k.aP, k1ds), dsff), k1 >= 0.0f ? 1.0f : -1.0f);
                }
                const FF hdff{0.5f * dsff.hi, 0.5f * dsff.lo};
                FF ips_ff = inv_ps(k, z.Px.hi, z.Py.hi, d, pp);
                for (int s = 0; s < N; ++s) {
                    // first half
                    if (is_mult) {
                        mixed_mult_half(z, k, dl, KICK ? zero : dl, hk1, hk2h, hk2, ips_ff, d, pp);
                    } else {
                        quad_linear_inc(z, k, mq, k1);
                        inv_ps(k, z.Px.hi, z.Py.hi, d, pp);
                        mixed_quad_nonlinear(z, k, hd, hdff, d, pp);
                        if constexpr (!KICK) quad_linear_inc(z, k, mq, k1);
                        ips_ff = inv_ps(k, z.Px.hi, z.Py.hi, d, pp);
                    }
                    // slice middle: the rotation by ds Omega
                    {
                        const float ips = ips_ff.hi, Ps = (k.P2 - pp) * ips;
                        FF bx, by;
                        float bz;
                        straight_edge(k, z, k1, k2, Aw, ds, d, ips, Ps, bx, by, bz);
                        D = cnq_mul(cnq_from_rotvec(bx, by, bz), D);
                    }
                    // second half
                    if (is_mult) {
                        mixed_mult_half(z, k, KICK ? zero : dl, dl, hk1, hk2h, hk2, ips_ff, d, pp);
                    } else {
                        if constexpr (!KICK) quad_linear_inc(z, k, mq, k1);
                        inv_ps(k, z.Px.hi, z.Py.hi, d, pp);
                        mixed_quad_nonlinear(z, k, hd, hdff, d, pp);
                        quad_linear_inc(z, k, mq, k1);
                        ips_ff = inv_ps(k, z.Px.hi, z.Py.hi, d, pp);
                    }
                }
            }
            CNQ dq = cnq_normalize(D);
            if (EXT && type == ST_SOLENOID) {
                // back from the relabelled frame, between the fringe kicks of Sec. 4.4
                dq = CNQ{dq.w, dq.z, dq.x, dq.y};
                const FF ks{el.ks_ff.x, el.ks_ff.y};
                const CNQ fi = mixed_solenoid_fringe(k, z0, ks, el.setaf_ff.x, 1.0f);
                const CNQ fo = mixed_solenoid_fringe(k, z, ks, el.setaf_ff.x, -1.0f);
                if (!isfinite(z.X.hi + z.Px.hi + z.Y.hi + z.Py.hi + z.T.hi + dq.w + dq.x.hi + dq.y.hi + dq.z.hi +
                              fi.w + fi.x.hi + fi.y.hi + fi.z.hi + fo.w + fo.x.hi + fo.y.hi + fo.z.hi)) {
                    z = z0;
                    is_lost = true;
                    break;
                }
                fq_premul_cnq(qt, fi);
                fq_premul_cnq(qt, dq);
                fq_premul_ref(qt, el.rq);
                fq_premul_cnq(qt, fo);
                continue;
            }
            if (!isfinite(z.X.hi + z.Px.hi + z.Y.hi + z.Py.hi + z.T.hi + dq.w + dq.x.hi + dq.y.hi + dq.z.hi)) {
                z = z0;
                is_lost = true;
                break;
            }
            const bool fr = FR && (el.type & ST_MIX_FRINGE);
            if (fr) fq_premul_cnq(qt, mixed_fringe(el, type, z0, 1.0f, 1.0f + (float)ref.G));
            fq_premul_cnq(qt, dq);
            if (type == ST_SBEND || (EXT && type == ST_TEAPOT)) fq_premul_about_y(qt, el.rq);
            if (fr) fq_premul_cnq(qt, mixed_fringe(el, type, z, -1.0f, 1.0f + (float)ref.G));
        }
        Quat q64{ff_to_double(qt.w), ff_to_double(qt.x), ff_to_double(qt.y), ff_to_double(qt.z)};
        q64 = qnormalize(q64);
        rotate_vec(q64, sx, sy, sz);
        if (spin_sum) {
            spin_sum[i] += sx;
            spin_sum[n_all + i] += sy;
            spin_sum[2 * n_all + i] += sz;
        }
    }
    xpx[i] = make_double2(ff_to_double(z.X), ff_to_double(z.Px));
    ypy[i] = make_double2(ff_to_double(z.Y), ff_to_double(z.Py));
    tpt[i].x = ff_to_double(z.T);
    sxy[i] = make_double2(sx, sy);
    szp[i] = sz;
    if (is_lost) lost[i] = 1;
}

}  // namespace st
