// Mixed-precision spin-orbit tracker: FP32 slice arithmetic, FP64 once per
// turn.  Same method and discretisation as the FP64 tracker (Sec. 3 orbit
// maps, Sec. 4.3 trapezoid levels and Romberg table), rearranged so that
// plain FP32 only carries small quantities:
//
// Orbit: every map is written as an increment (cos(h ds) - 1 instead of
//   cos(h ds), 1/Ps - 1/P instead of 1/Ps, Ps - 1 from (P^2 - 1 - p^2)/(Ps + 1),
//   ...).  Coordinates are compensated (hi, lo) float pairs; first-order
//   (linear) terms multiply compensated coordinates by compensated constants
//   with error-free FMA products and are accumulated with two-sums, so the
//   linear optics carry no FP32 rounding bias (no systematic tune error);
//   second-order terms are plain FP32.
// Spin: an edge rotation q(w Omega) is split exactly into the on-axis,
//   on-momentum reference rotation r = q(w Omega_ref) (about the vertical in
//   bends, identity in multipoles) and the small deviation e = r^-1 q, which
//   is evaluated in FP32 from the deviation of Omega with Taylor coefficients
//   of cos(t/2) and sin(t/2)/t about the reference angle.  Because every
//   Romberg level's trapezoid weights add up to the element length, every
//   level product equals R_L E_k with the same reference rotation R_L, so the
//   Romberg table and the normalisation act on the near-identity deviations
//   E_k (scalar part minus one in FP32, vector part compensated).  The
//   first-order parts of the spin rotations -- the deviation of Omega linear in
//   the coordinates (quadrupole fields, the bend's dispersive and energy
//   terms), the rotation vectors, their sums in the level products, the
//   Romberg combinations and the composition into the turn -- are carried as
//   compensated (hi, lo) pairs like the orbit's linear terms, so that FP32
//   rounding of rotations of order 1e-2 per element (G gamma ~ 500) does not
//   accumulate; second-order parts are plain FP32.  The element rotation
//   R_L D is multiplied into a compensated (hi, lo) turn quaternion; once per
//   turn it is composed and renormalised in FP64 and the spin rotated in FP64.
#pragma once

#include "device_common.cuh"
#include "ff.cuh"
#include "track_mid.cuh"   // the FP64 rectangular-bend maps (tracked in FP64 in the mixed kernels)

namespace st {

// ---- near-identity quaternions (w holds scalar - 1) -------------------------
struct NQ {
    float w, x, y, z;
};

// Rotation q(b) of a small rotation vector b as a near-identity quaternion:
// (cos(t/2) - 1, sin(t/2)/t b), t = |b|, Taylor series in u = t^2.
__device__ __forceinline__ NQ nq_from_small_rotvec(float bx, float by, float bz) {
    const float u = bx * bx + by * by + bz * bz;
    float cm1, S;
    if (u < 0.01f) {
        cm1 = u * fmaf(u, fmaf(u, -1.0f / 46080.0f, 1.0f / 384.0f), -0.125f);
        S = fmaf(u, fmaf(u, fmaf(u, -1.0f / 645120.0f, 1.0f / 3840.0f), -1.0f / 48.0f), 0.5f);
    } else {
        const float t = sqrtf(u);
        float sq, cq;
        sincosf(0.25f * t, &sq, &cq);
        cm1 = -2.0f * sq * sq;                 // cos(t/2) - 1
        S = 2.0f * sq * cq / t;                // sin(t/2) / t
    }
    return NQ{cm1, S * bx, S * by, S * bz};
}

// ---- near-identity quaternions with a compensated vector part ---------------
// w = scalar - 1 (second order) in FP32; x, y, z as (hi, lo).
struct CNQ {
    float w;
    FF x, y, z;
};

__device__ __forceinline__ FF ff_scale2(const FF& a, float p2) { return FF{a.hi * p2, a.lo * p2}; }   // p2 a power of 2

// later rotation a on the left: a b; first-order sums a.v + b.v compensated,
// second-order terms in FP32
__device__ __forceinline__ CNQ cnq_mul(const CNQ& a, const CNQ& b) {
    const float ax = a.x.hi, ay = a.y.hi, az = a.z.hi, bx = b.x.hi, by = b.y.hi, bz = b.z.hi;
    CNQ o;
    o.w = a.w + b.w + (a.w * b.w - (ax * bx + ay * by + az * bz));
    o.x = ff_add3(a.x, b.x, a.w * bx + b.w * ax + (ay * bz - az * by));
    o.y = ff_add3(a.y, b.y, a.w * by + b.w * ay + (az * bx - ax * bz));
    o.z = ff_add3(a.z, b.z, a.w * bz + b.w * az + (ax * by - ay * bx));
    return o;
}

__device__ __forceinline__ CNQ cnq_square(const CNQ& a) {
    const float ax = a.x.hi, ay = a.y.hi, az = a.z.hi;
    CNQ o;
    o.w = 2.0f * a.w + (a.w * a.w - (ax * ax + ay * ay + az * az));
    const float t = 2.0f * a.w;
    o.x = ff_add_f(ff_scale2(a.x, 2.0f), t * ax);
    o.y = ff_add_f(ff_scale2(a.y, 2.0f), t * ay);
    o.z = ff_add_f(ff_scale2(a.z, 2.0f), t * az);
    return o;
}

__device__ __forceinline__ CNQ cnq_normalize(const CNQ& a) {
    const float ax = a.x.hi, ay = a.y.hi, az = a.z.hi;
    const float eps = 2.0f * a.w + (a.w * a.w + ax * ax + ay * ay + az * az);   // |q|^2 - 1
    float g;   // (1 + eps)^(-1/2) - 1
    if (fabsf(eps) < 1e-3f)
        g = eps * fmaf(eps, fmaf(eps, -0.3125f, 0.375f), -0.5f);
    else
        g = rsqrtf(1.0f + eps) - 1.0f;
    return CNQ{a.w + g * (1.0f + a.w), ff_add_f(a.x, g * ax), ff_add_f(a.y, g * ay), ff_add_f(a.z, g * az)};
}

// q(b) for a small rotation vector b: (cos(t/2) - 1, S b), S = sin(t/2)/t =
// 1/2 + O(t^2): the first-order part b/2 exact, the rest in FP32
__device__ __forceinline__ CNQ cnq_from_rotvec(const FF& bx, const FF& by, float bz) {
    const NQ e = nq_from_small_rotvec(bx.hi, by.hi, bz);
    const float u = bx.hi * bx.hi + by.hi * by.hi + bz * bz;
    // S - 1/2 from the same series (u is tiny for these edges)
    const float Sm = u * fmaf(u, fmaf(u, -1.0f / 645120.0f, 1.0f / 3840.0f), -1.0f / 48.0f);
    CNQ o;
    o.w = e.w;
    if (u < 0.01f) {
        o.x = ff_add_f(ff_scale2(bx, 0.5f), Sm * bx.hi);
        o.y = ff_add_f(ff_scale2(by, 0.5f), Sm * by.hi);
    } else {
        o.x = FF{e.x, 0.0f};
        o.y = FF{e.y, 0.0f};
    }
    o.z = FF{e.z, 0.0f};
    return o;
}

// Deviation e = r^-1 q(a + b) of an edge rotation from the reference rotation
// r = q(a), a = alpha y^, for a small deviation vector b:
//   e_w = c C + s S (alpha + b_y),  e_v = c S (a + b) - C s y^ - s S y^ x (a + b)
// with c, s = cos, sin(alpha/2), C = cos(|a+b|/2), S = sin(|a+b|/2)/|a+b|,
// written in the differences C - c and S - S(alpha^2) (Taylor series in
// du = |a+b|^2 - alpha^2, MIX_TAYLOR terms); e_y = Ky b_y compensated + the
// terms of second and higher order in b (FP32).
__device__ __forceinline__ CNQ cnq_deviation(const MixWeight& W, float bx, const FF& byf, float bz) {
    const float by = byf.hi;
    const float bb = bx * bx + by * by + bz * bz;
    const float du = fmaf(2.0f * W.alpha, by, bb);   // |a+b|^2 - alpha^2
    // dC = du (dC0 + du tC), dS = du (dS0 + du tS), tails by Horner
    float tC = W.dC[MIX_TAYLOR - 1], tS = W.dS[MIX_TAYLOR - 1];
#pragma unroll
    for (int n = MIX_TAYLOR - 2; n >= 1; --n) {
        tC = fmaf(du, tC, W.dC[n]);
        tS = fmaf(du, tS, W.dS[n]);
    }
    const float dC = du * fmaf(du, tC, W.dC[0]);
    const float dS = du * fmaf(du, tS, W.dS[0]);
    const float S = W.S0 + dS;
    CNQ e;
    e.w = W.ch * dC + W.sh * (W.alpha * dS + S * by);
    // e_y = Ky b_y + Kq |b|^2 + du^2 (ch alpha tS - sh tC) + ch dS b_y
    const float rest = fmaf(W.Kq, bb, fmaf(du * du, W.ch * W.alpha * tS - W.sh * tC, W.ch * dS * by));
    e.y = ff_addn(ff_mul(FF{W.Ky.x, W.Ky.y}, byf), rest);
    e.x = FF{S * (W.ch * bx - W.sh * bz), 0.0f};
    e.z = FF{S * (W.ch * bz + W.sh * bx), 0.0f};
    return e;
}

// ---- compensated turn quaternion -----------------------------------------------
struct FQ {
    FF w, x, y, z;
};

// Q <- (1 + D) Q for a near-identity D with compensated vector part: the
// first-order products D.v Q compensated, D.w Q (second order) in FP32
// (the four components as two packed FP32x2 pairs, (w, x) and (y, z))
__device__ __forceinline__ FF2 ff2_add_lazy(const FF2& a, const FF2& b) {
    float2 s, e;
    two_sum2(a.hi, b.hi, s, e);
    return FF2{s, __fadd2_rn(e, __fadd2_rn(a.lo, b.lo))};
}
__device__ __forceinline__ FF2 ff2_neg(const FF2& a) { return FF2{f2_neg(a.hi), f2_neg(a.lo)}; }
__device__ __forceinline__ void fq_premul_cnq(FQ& q, const CNQ& d) {
    const FF2 qwx = ff2_pack(q.w, q.x), qyz = ff2_pack(q.y, q.z);
    const FF nx = ff_neg(d.x), ny = ff_neg(d.y), nz = ff_neg(d.z);
    // c_w = -(dx qx + dy qy + dz qz),  c_x = dx qw + dy qz - dz qy
    const FF2 cwx = ff2_add_lazy(ff2_add_lazy(ff2_mul(ff2_pack(nx, d.x), ff2_pack(q.x, q.w)),
                                              ff2_mul(ff2_pack(ny, d.y), ff2_pack(q.y, q.z))),
                                 ff2_mul(ff2_pack(nz, nz), ff2_pack(q.z, q.y)));
    // c_y = dy qw + dz qx - dx qz,  c_z = dz qw + dx qy - dy qx
    const FF2 cyz = ff2_add_lazy(ff2_add_lazy(ff2_mul(ff2_pack(d.y, d.z), ff2_pack(q.w, q.w)),
                                              ff2_mul(ff2_pack(d.z, d.x), ff2_pack(q.x, q.y))),
                                 ff2_mul(ff2_pack(nx, ny), ff2_pack(q.z, q.x)));
    // plus the second-order d_w q in the compensation word
    const FF2 awx{cwx.hi, __ffma2_rn(make_float2(d.w, d.w), qwx.hi, cwx.lo)};
    const FF2 ayz{cyz.hi, __ffma2_rn(make_float2(d.w, d.w), qyz.hi, cyz.lo)};
    const FF2 owx = ff2_add(qwx, awx), oyz = ff2_add(qyz, ayz);
    q.w = ff2_first(owx);
    q.x = ff2_second(owx);
    q.y = ff2_first(oyz);
    q.z = ff2_second(oyz);
}

// Q <- R Q for a compensated reference rotation R = (a0, 0, a2, 0) about y
// (a sector bend's: the other two components vanish)
__device__ __forceinline__ void fq_premul_about_y(FQ& q, const float2* rq) {
    const FF a0{rq[0].x, rq[0].y}, a2{rq[2].x, rq[2].y};
    FQ o;
    o.w = ff_add(ff_mul(a0, q.w), ff_neg(ff_mul(a2, q.y)));
    o.x = ff_add(ff_mul(a0, q.x), ff_mul(a2, q.z));
    o.y = ff_add(ff_mul(a0, q.y), ff_mul(a2, q.w));
    o.z = ff_add(ff_mul(a0, q.z), ff_neg(ff_mul(a2, q.x)));
    q = o;
}

// Q <- R Q for a compensated reference rotation R
__device__ __forceinline__ void fq_premul_ref(FQ& q, const float2* rq) {
    const FF a0{rq[0].x, rq[0].y}, a1{rq[1].x, rq[1].y}, a2{rq[2].x, rq[2].y}, a3{rq[3].x, rq[3].y};
    FQ o;
    o.w = ff_add(ff_add(ff_mul(a0, q.w), ff_neg(ff_mul(a1, q.x))), ff_neg(ff_add(ff_mul(a2, q.y), ff_mul(a3, q.z))));
    o.x = ff_add(ff_add(ff_mul(a0, q.x), ff_mul(a1, q.w)), ff_add(ff_mul(a2, q.z), ff_neg(ff_mul(a3, q.y))));
    o.y = ff_add(ff_add(ff_mul(a0, q.y), ff_neg(ff_mul(a1, q.z))), ff_add(ff_mul(a2, q.w), ff_mul(a3, q.x)));
    o.z = ff_add(ff_add(ff_mul(a0, q.z), ff_mul(a1, q.y)), ff_add(ff_neg(ff_mul(a2, q.x)), ff_mul(a3, q.w)));
    q = o;
}

// ---- per-particle constants ---------------------------------------------------
struct MConst {
    FF invP, tau, PM1;                     // 1/P; 1/beta0 - (1/beta0 + Pt)/P; P - 1
    FF aP, a0P, c1P;                       // a/P, a0/P, c1/P (spin: first-order coefficients)
    FF invP2, Ptf, b0ptf;                  // 1/P^2, Pt, 1/beta0 + Pt
    FF hiP3;                               // 1/(2 P^3) (TEAPOT bends, solenoids)
    FF cP2, PM1P;                          // G (gamma - 1)/P^2, (P - 1)/P (solenoids)
    float Pt, P2, P2m1, invPf, P, b0pt, a, c, da, f3, a0, c1;
};

struct MState {
    FF X, Px, Y, Py, T;
};

// 1/Ps as a compensated value and d = 1/Ps - 1/P in FP32, from the
// transverse momenta: 1/Ps = (1/P)(1 - e)^(-1/2), e = p^2/P^2.
__device__ __forceinline__ FF inv_ps(const MConst& k, float px, float py, float& d, float& pp) {
    pp = px * px + py * py;
    const float e = pp * k.invPf * k.invPf;
    if (e < 1e-4f) {
        d = k.invPf * e * fmaf(e, fmaf(e, 0.3125f, 0.375f), 0.5f);
    } else {
        const float ips = rsqrtf(k.P2 - pp);
        d = pp * k.invPf * ips / (k.P + (k.P2 - pp) * ips);
    }
    return ff_add_f(k.invP, d);
}

__device__ __forceinline__ void drift_inc(MState& z, const MConst& k, const FF& L, const FF& ips, float d) {
    const FF Lips = ff_mul(L, ips);
    // (X, Y) += (L/Ps) (Px, Py), both planes in packed FP32x2 arithmetic
    const FF2 U = ff2_add(ff2_pack(z.X, z.Y), ff2_mul(ff2_pack(z.Px, z.Py), ff2_pack(Lips, Lips)));
    z.X = ff2_first(U);
    z.Y = ff2_second(U);
    z.T = ff_add(z.T, ff_mul(L, ff_add_f(k.tau, -k.b0pt * d)));
}

// Edge rotation vector b = w Omega (Eq. (6b)) in a straight element with field
// b = (k1 Y + k2 X Y, k1 X + k2 (X^2 - Y^2)/2, 0): the quadrupole part of the
// first order, -w (a/P) k1 (Y, X), compensated (Aw = w (a/P) k1); the rest,
// -w [(a/P) b_sext + a (1/Ps - 1/P) b - (c (u.b)/P) p / Ps], in FP32;
// d = 1/Ps - 1/P.
__device__ __forceinline__ void straight_edge(const MConst& k, const MState& z, float k1, float k2, const FF& Aw,
                                              float w, float d, float ips, float Ps, FF& bx, FF& by, float& bz) {
    const float X = z.X.hi, Y = z.Y.hi, px = z.Px.hi, py = z.Py.hi;
    const float sx = k2 * X * Y, sy = 0.5f * k2 * (X * X - Y * Y);
    const float fbx = k1 * Y + sx, fby = k1 * X + sy;
    const float cu = k.c * ((px * fbx + py * fby) * k.invPf) * k.invPf;
    const float aPf = k.aP.hi;
    const float remx = -aPf * sx - d * k.a * fbx + ips * cu * px;
    const float remy = -aPf * sy - d * k.a * fby + ips * cu * py;
    // (bx, by) = -Aw (Y, X) + w (remx, remy), renormalised; both in packed FP32x2
    const FF2 p = ff2_mul(ff2_pack(z.Y, z.X), ff2_pack(Aw, Aw));
    const float2 t = __ffma2_rn(make_float2(w, w), make_float2(remx, remy), f2_neg(p.lo));   // w rem - lo
    const float2 h = f2_neg(p.hi);
    float2 rh = __fadd2_rn(h, t);
    float2 rl = f2_sub(t, f2_sub(rh, h));
    bx = FF{rh.x, rl.x};
    by = FF{rh.y, rl.y};
    bz = w * ips * cu * Ps;
}

// Per-particle constants of the mixed-precision maps (FP64 -> compensated
// FP32) for energy coordinate Pt: Eq. (2)'s P^2 = 1 + 2 Pt/beta0 + Pt^2 and
// the particle's gamma for Eq. (6b); invP64 = 1/P in FP64.
__device__ __forceinline__ void mixed_particle_consts(const RefConst& ref, double Pt, MConst& k, double& invP64) {
    const double P2m1 = 2.0 * Pt * ref.inv_beta0 + Pt * Pt;
    const double P2 = 1.0 + P2m1;
    invP64 = rsqrt(P2);
    const double P = P2 * invP64;
    const double b0pt = ref.inv_beta0 + Pt;
    const double gamma = ref.gamma0 * (1.0 + ref.beta0 * Pt);
    k.invP = ff_make(invP64);
    k.PM1 = ff_make(P2m1 / (P + 1.0));
    // 1/beta0 - (1/beta0 + Pt)/P = ((P - 1) - beta0 Pt) / (beta0 P)
    k.tau = ff_make((P2m1 / (P + 1.0) - ref.beta0 * Pt) * ref.inv_beta0 * invP64);
    k.Pt = (float)Pt;
    k.P2 = (float)P2;
    k.P2m1 = (float)P2m1;
    k.invPf = (float)invP64;
    k.P = (float)P;
    k.b0pt = (float)b0pt;
    k.a = (float)(1.0 + ref.G * gamma);
    k.c = (float)(ref.G * (gamma - 1.0));
    k.da = (float)(ref.G * ref.gamma0 * ref.beta0 * Pt);
    k.f3 = (float)(0.5 * b0pt * invP64 * invP64 * invP64);
    k.a0 = (float)(1.0 + ref.G * ref.gamma0);
    // a0 (P - 1) - da: the energy deviation's first-order terms of the bend's
    // Omega_y, which cancel to O(Pt) for G gamma >> 1, combined in FP64
    const double a0d = 1.0 + ref.G * ref.gamma0;
    const double c1 = a0d * (P2m1 / (P + 1.0)) - ref.G * ref.gamma0 * ref.beta0 * Pt;
    k.c1 = (float)c1;
    k.aP = ff_make((1.0 + ref.G * gamma) * invP64);
    k.a0P = ff_make(a0d * invP64);
    k.c1P = ff_make(c1 * invP64);
    k.invP2 = ff_make(1.0 / P2);
    k.hiP3 = ff_make(0.5 * invP64 * invP64 * invP64);
    k.cP2 = ff_make(ref.G * (gamma - 1.0) / P2);
    k.PM1P = ff_make(P2m1 / (P + 1.0) * invP64);
    k.Ptf = ff_make(Pt);
    k.b0ptf = ff_make(b0pt);
}

// cached matrix-kick coefficients of the half-slice linear flow (computed in
// FP64 when the (|k1|, s) key changes): for the cos plane (1) and the cosh
// plane (2): C - 1, S/P and |k1| S as compensated pairs, and the FP32 time
// coefficients (s + C S)/2, S^2, (s - C S)/2.
struct MQuad {
    float key_k, key_s;
    FF Cm1[2], SP[2], kS[2];
    float al[2], be[2], ga[2];
};

__device__ __forceinline__ void mquad_coeffs(MQuad& q, double invP, double absk, double s, float key_k, float key_s) {
    q.key_k = key_k;
    q.key_s = key_s;
    const double w = sqrt(absk * invP);
    const double ds = s;
    const double ws = w * ds;
    double Cm1[2], S[2];
    if (w > 0.0) {
        double sh, ch;
        sincos(0.5 * ws, &sh, &ch);
        Cm1[0] = -2.0 * sh * sh;
        S[0] = 2.0 * sh * ch / w;
        const double e = exp(0.5 * ws), ei = 1.0 / e;
        const double shh = 0.5 * (e - ei), chh = 0.5 * (e + ei);
        Cm1[1] = 2.0 * shh * shh;
        S[1] = 2.0 * shh * chh / w;
    } else {
        Cm1[0] = Cm1[1] = 0.0;
        S[0] = S[1] = ds;
    }
    for (int p = 0; p < 2; ++p) {
        const double C = 1.0 + Cm1[p];
        q.Cm1[p] = ff_make(Cm1[p]);
        q.SP[p] = ff_make(S[p] * invP);
        q.kS[p] = ff_make(absk * S[p]);
        q.al[p] = (float)(0.5 * (ds + C * S[p]));
        q.be[p] = (float)(S[p] * S[p]);
        q.ga[p] = (float)(0.5 * (ds - C * S[p]));
    }
}

// linear quadrupole flow H_qL over a half slice, Eq. (24), in increment form:
// dU = U (C-1) + Pu (S/P),  dPu = Pu (C-1) -/+ k1 U S.  PX is the coefficient
// set of the x plane (0: the cos plane, k1 >= 0; 1: the cosh plane), a
// compile-time index so that the coefficients stay in registers.
template <int PX>
__device__ __forceinline__ void quad_linear_inc_(MState& z, const MConst& k, const MQuad& q, float k1) {
    constexpr int px_ = PX, py_ = 1 - PX;
    constexpr float sgn = PX == 0 ? 1.0f : -1.0f;
    const float X = z.X.hi, Px = z.Px.hi, Y = z.Y.hi, Py = z.Py.hi;
    const float Pk = k.P * k1;
    const float tsum = Px * Px * q.al[px_] - k1 * X * Px * q.be[px_] + Pk * X * X * q.ga[px_] +
                       Py * Py * q.al[py_] + k1 * Y * Py * q.be[py_] - Pk * Y * Y * q.ga[py_];
    // both planes at once in packed FP32x2 arithmetic: (X, Y) and (Px, Py)
    const FF2 U = ff2_pack(z.X, z.Y), PU = ff2_pack(z.Px, z.Py);
    const FF2 Cm1 = ff2_pack(q.Cm1[px_], q.Cm1[py_]), SP = ff2_pack(q.SP[px_], q.SP[py_]);
    const FF kSx = q.kS[px_], kSy = q.kS[py_];
    const FF2 kS = ff2_pack(FF{-sgn * kSx.hi, -sgn * kSx.lo}, FF{sgn * kSy.hi, sgn * kSy.lo});   // exact sign flips
    const FF2 dU = ff2_add(ff2_mul(U, Cm1), ff2_mul(PU, SP));
    const FF2 dPU = ff2_add(ff2_mul(PU, Cm1), ff2_mul(U, kS));
    const FF2 U1 = ff2_add(U, dU), PU1 = ff2_add(PU, dPU);
    z.X = ff2_first(U1);
    z.Y = ff2_second(U1);
    z.Px = ff2_first(PU1);
    z.Py = ff2_second(PU1);
    z.T = ff_add_f(z.T, -k.f3 * tsum);
}

// the sign of k1 is uniform per element, so the branch does not diverge
__device__ __forceinline__ void quad_linear_inc(MState& z, const MConst& k, const MQuad& q, float k1) {
    if (k1 >= 0.0f)
        quad_linear_inc_<0>(z, k, q, k1);
    else
        quad_linear_inc_<1>(z, k, q, k1);
}

template <int K>
struct MixLevels {
    CNQ q[K + 1];

    // straight elements (no reference rotation): edge rotation vector b of the
    // finest level (x, y compensated); coarser levels by squaring
    __device__ __forceinline__ void add_straight(int i, const FF& bx, const FF& by, float bz) {
        CNQ e = cnq_from_rotvec(bx, by, bz);
        if (i == 0) {
            q[K] = e;
#pragma unroll
            for (int m = 1; m <= K; ++m) {
                e = cnq_square(e);
                q[K - m] = e;
            }
            return;
        }
        q[K] = cnq_mul(e, q[K]);
#pragma unroll
        for (int m = 1; m <= K; ++m) {
            if (i & ((1 << m) - 1)) break;
            e = cnq_square(e);
            q[K - m] = cnq_mul(e, q[K - m]);
        }
    }

    // bends: for every level sampling edge i, the deviation of the level's edge
    // rotation from its reference rotation, conjugated by the reference
    // rotation accumulated over the level's earlier edges (angle
    // omr i ds - alpha_m, the trapezoid end weight alpha_m = omr 2^m ds / 2);
    // the deviation of Omega is (dox, doy, dos) with doy compensated
    // Each coarser level's weight at an edge is twice the finer one's, so its
    // edge rotation is the square of the finer one: with r = q(alpha y^) the
    // finer weight's reference rotation, (r e)^2 = r^2 (r^-1 e r) e, i.e. the
    // coarser deviation is e conjugated by r, times e (no second series).
    __device__ __forceinline__ void add_bend(int i, int N, const MixElem& el, float rc, float rs, float dox,
                                             const FF& doy, float dos) {
        CNQ ep;   // the previous (finer) level's deviation at this edge
#pragma unroll
        for (int m = 0; m <= K; ++m) {
            if (m > 0 && (i & ((1 << m) - 1))) break;
            const int j = (i == 0 || i == N) ? m : m + 1;
            CNQ e;
            if (m == 0) {
                const float p2 = (float)(1 << j) * 0.5f;   // 2^(j-1), exact
                const float w = el.ds * p2;
                const FF wf{el.ds_ff.x * p2, el.ds_ff.y * p2};
                e = cnq_deviation(el.w[j], w * dox, ff_mul(wf, doy), w * dos);
            } else {
                const MixWeight& Wp = el.w[j - 1];
                CNQ c = ep;
                c.x = FF{ep.x.hi * Wp.cf - ep.z.hi * Wp.sf, 0.0f};
                c.z = FF{ep.x.hi * Wp.sf + ep.z.hi * Wp.cf, 0.0f};
                e = cnq_mul(c, ep);
            }
            ep = e;
            if (i == 0) {
                q[K - m] = e;
                continue;
            }
            const MixWeight& Wm = el.w[m];
            const float cphi = rc * Wm.cf + rs * Wm.sf;
            const float sphi = rs * Wm.cf - rc * Wm.sf;
            const float ex = e.x.hi * cphi - e.z.hi * sphi;
            const float ez = e.x.hi * sphi + e.z.hi * cphi;
            e.x = FF{ex, 0.0f};
            e.z = FF{ez, 0.0f};
            q[K - m] = cnq_mul(e, q[K - m]);
        }
    }

    // Romberg table on the deviations (Eq. (39)): q_k <- (4^j q_k - q_{k-1}) / (4^j - 1)
    __device__ __forceinline__ CNQ romberg() {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const float f = (float)(1 << (2 * (j + 1)));
            const float inv = 1.0f / (f - 1.0f);
            const FF invf{inv, fmaf(-inv, f - 1.0f, 1.0f) * inv};   // 1/(f-1) to ~2^-46
#pragma unroll
            for (int k = K; k >= j + 1; --k) {
                q[k].w = (f * q[k].w - q[k - 1].w) * inv;
                q[k].x = ff_mul(ff_add_lazy(ff_scale2(q[k].x, f), ff_neg(q[k - 1].x)), invf);
                q[k].y = ff_mul(ff_add_lazy(ff_scale2(q[k].y, f), ff_neg(q[k - 1].y)), invf);
                q[k].z = ff_mul(ff_add_lazy(ff_scale2(q[k].z, f), ff_neg(q[k - 1].z)), invf);
            }
        }
        return cnq_normalize(q[K]);
    }
};

// ---- TEAPOT bend (Sec. 3.6) in increment form ---------------------------------
// Curved drift over len: the flow of H_D = -(1 + hX) Ps + Pt/beta0 with the
// reference time len/beta0 (Eq. (teapotD)), c = the drift's constants (sn =
// sin(h len), omc = 1 - cos(h len), A1 = omc/h, A2 = sn/h).  With x' = Px/Ps,
// y' = Py/Ps, eps = omc + x' sn (1 - eps is the cos - x' sin denominator) and
// e1 = eps/(1 - eps):
//   dX  = A1 + x' A2 + (X + A1 + x' A2) e1
//   dY  = y' A2 (1 + g),  g = (1 + hX)(1 + e1) - 1
//   dPx = sn + (Ps - 1) sn - Px omc
//   dT  = (len - A2)/beta0 + A2 tau - A2 (1/beta0 + Pt) d - X sn/beta0
//         - A2 [((1/beta0 + Pt) d - tau) hX + (1/beta0 + Pt) e1 (1 + hX)/Ps]
// (tau = 1/beta0 - (1/beta0 + Pt)/P, d = 1/Ps - 1/P).  Unlike the exact bend,
// the drift-kick split swings even the on-axis particle off the axis inside a
// slice (Px by about sin(h ds/2), X by about (1 - cos)/h), so Px^2, Ps - P,
// d, eps and e1 are not small there and are compensated too: with p^2 =
// Px^2 + Py^2 and e = p^2/P^2,
//   Ps - P = -(p^2/(2P)) (1 + e/4 + e^2/8 + 5e^3/64),
//   d      =  (p^2/(2P^3)) (1 + 3e/4 + 5e^2/8 + 35e^3/64),
// the leading terms compensated, the series factors in FP32 (FP32 throughout
// for e >= 4e-3, far from the axis).  If the line does not meet the turned
// frame (1 - eps <= 0) or Ps^2 <= 0, X becomes NaN: the particle is lost.
// Ps - P and d = 1/Ps - 1/P (compensated) for a transverse momentum (px, py)
// with p^2 = px^2 + py^2 not small against the compensation's precision (see
// below); NaN if Ps^2 <= 0.
__device__ __forceinline__ void ps_deviations(const MConst& k, const FF& px, const FF& py, FF& dPsP, FF& d) {
    const FF pp = ff_add(ff_mul(px, px), ff_mul(py, py));
    const float e = pp.hi * k.invPf * k.invPf;
    if (e < 4e-3f) {
        const FF u = ff_mul(pp, FF{0.5f * k.invP.hi, 0.5f * k.invP.lo});   // p^2/(2P)
        dPsP = ff_addn(ff_neg(u), -u.hi * e * fmaf(e, fmaf(e, 5.0f / 64.0f, 0.125f), 0.25f));
        const FF dd = ff_mul(pp, k.hiP3);                                  // p^2/(2P^3)
        d = ff_addn(dd, dd.hi * e * fmaf(e, fmaf(e, 35.0f / 64.0f, 0.625f), 0.75f));
    } else {   // far from the axis (the series would not converge fast): FP32
        const float ipsf = rsqrtf(k.P2 - pp.hi);   // NaN for Ps^2 < 0
        const float Psf = (k.P2 - pp.hi) * ipsf;
        d = FF{pp.hi * k.invPf * ipsf / (k.P + Psf), 0.0f};
        dPsP = FF{-pp.hi / (Psf + k.P), 0.0f};
    }
}

__device__ __forceinline__ void mixed_curved_drift(MState& z, const MConst& k, const MixCurvedDrift& c, float h) {
    const FF sn{c.sn_ff.x, c.sn_ff.y}, A1{c.A1_ff.x, c.A1_ff.y}, A2{c.A2_ff.x, c.A2_ff.y};
    const FF omc{c.omc_ff.x, c.omc_ff.y};
    FF dPsP, d;   // Ps - P, 1/Ps - 1/P
    ps_deviations(k, z.Px, z.Py, dPsP, d);
    const FF ips = ff_add(k.invP, d);
    // (x', y') and (x' A2, y' A2), both planes in packed FP32x2 arithmetic
    const FF2 pr = ff2_mul(ff2_pack(z.Px, z.Py), ff2_pack(ips, ips));
    const FF2 pA = ff2_mul(pr, ff2_pack(A2, A2));
    const FF eps = ff_add(omc, ff_mul(ff2_first(pr), sn));
    const float ome = 1.0f - eps.hi;
    const FF e1 = ff_addn(eps, eps.hi * eps.hi * __frcp_rn(ome));   // eps + eps^2/(1 - eps)
    const float hX = h * z.X.hi;
    const FF xA = ff_add(A1, ff2_first(pA));
    const FF dX = ff_add(xA, ff_mul(ff_add_lazy(z.X, xA), e1));
    const FF yA = ff2_second(pA);
    const FF dY = ff_add_f(yA, yA.hi * fmaf(e1.hi, 1.0f + hX, hX));
    const FF PsM1 = ff_add(k.PM1, dPsP);
    const FF dPx = ff_add(ff_add(sn, ff_mul(PsM1, sn)), ff_neg(ff_mul(z.Px, omc)));
    const FF W = ff_mul(ff_mul(k.b0ptf, ips), ff_mul(A2, e1));        // (1/beta0 + Pt) e1 A2 / Ps
    const float rem = fmaf(A2.hi * (k.b0pt * d.hi - k.tau.hi), hX, W.hi * hX);
    const FF dT0 = ff_add(FF{c.dT0_ff.x, c.dT0_ff.y}, ff_mul(A2, k.tau));
    const FF dT1 = ff_add(ff_mul(ff_mul(A2, d), k.b0ptf), ff_add_lazy(ff_mul(z.X, FF{c.snb0_ff.x, c.snb0_ff.y}), W));
    const FF dT = ff_add_f(ff_add(dT0, ff_neg(dT1)), -rem);
    z.X = ff_add(z.X, dX);
    z.Y = ff_add(z.Y, dY);
    z.Px = ff_add(z.Px, dPx);
    z.T = ff_add(z.T, dT);
    if (!(ome > 0.0f && k.P + dPsP.hi > 0.0f)) z.X.hi = __int_as_float(0x7fc00000);   // quiet NaN
}

// Kick of the bend's uniform field, dPx = -eta h len (1 + hX), from the
// compensated eta h len and eta h^2 len.
__device__ __forceinline__ void mixed_teapot_kick(MState& z, const FF& ehl, const FF& ehlh) {
    z.Px = ff_add(z.Px, ff_neg(ff_add(ehl, ff_mul(z.X, ehlh))));
}

// ---- solenoid (Sec. 3.7, 4.4) ------------------------------------------------
// In the body the kinetic momentum (Px + eta Y, Py - eta X), eta = ks/2, keeps
// its Ps, and a slice of length len is the map of Eq. (solenoid) with
// kappa = eta/Ps, theta = kappa len = theta0 + delta, theta0 = eta len/P (FP64
// once per element and particle) and delta = eta len (1/Ps - 1/P) (of order
// 1e-10 of theta0 near the axis):
//   cos theta - 1 = (cos theta0 - 1) - sin theta0 delta,
//   sin theta = sin theta0 + cos theta0 delta,
//   sin theta / eta = sin theta0 / eta + cos theta0 len (1/Ps - 1/P),
// compensated; d = 1/Ps - 1/P of the kinetic momentum.
struct MSolSlice {
    FF cm1, sn, a12, a21;
};

__device__ __forceinline__ MSolSlice mixed_solenoid_slice(const FF& eta, double len, double invP64, float d) {
    const double eta64 = (double)eta.hi + (double)eta.lo;
    const double th0 = eta64 * len * invP64;
    double s2, c2;
    sincos(0.5 * th0, &s2, &c2);
    const double s0 = 2.0 * s2 * c2, c0m1 = -2.0 * s2 * s2;
    // sin(theta0)/eta = (len/P) sin(theta0)/theta0
    const double s0ieta = fabs(th0) > 1e-4 ? s0 / eta64 : len * invP64 * (1.0 - th0 * th0 * (1.0 / 6.0 - th0 * th0 / 120.0));
    const float c0f = (float)(1.0 + c0m1);
    const float delta = eta.hi * (float)len * d;
    MSolSlice m;
    m.cm1 = ff_add_f(ff_make(c0m1), -(float)s0 * delta);
    m.sn = ff_add_f(ff_make(s0), c0f * delta);
    m.a12 = ff_add_f(ff_make(s0ieta), c0f * (float)len * d);
    m.a21 = ff_neg(ff_mul(eta, m.sn));
    return m;
}

// One body slice, in increment form with both planes in packed FP32x2
// arithmetic: (U, PU) <- (cos U + (sin/eta) PU, -eta sin U + cos PU), then the
// (X, Y) and (Px, Py) planes rotated by -theta; T += len (tau - (1/beta0 + Pt) d).
__device__ __forceinline__ void mixed_solenoid_map(MState& z, const MConst& k, const MSolSlice& m, const FF& lenff,
                                                   float d) {
    const FF2 cm1 = ff2_pack(m.cm1, m.cm1), a12 = ff2_pack(m.a12, m.a12), a21 = ff2_pack(m.a21, m.a21);
    const FF2 rs = ff2_pack(m.sn, ff_neg(m.sn));
    const FF2 U = ff2_pack(z.X, z.Y), PU = ff2_pack(z.Px, z.Py);
    const FF2 U1 = ff2_add(U, ff2_add(ff2_mul(U, cm1), ff2_mul(PU, a12)));
    const FF2 PU1 = ff2_add(PU, ff2_add(ff2_mul(U, a21), ff2_mul(PU, cm1)));
    const FF2 U1s{make_float2(U1.hi.y, U1.hi.x), make_float2(U1.lo.y, U1.lo.x)};
    const FF2 PU1s{make_float2(PU1.hi.y, PU1.hi.x), make_float2(PU1.lo.y, PU1.lo.x)};
    const FF2 U2 = ff2_add(U1, ff2_add(ff2_mul(U1, cm1), ff2_mul(U1s, rs)));
    const FF2 PU2 = ff2_add(PU1, ff2_add(ff2_mul(PU1, cm1), ff2_mul(PU1s, rs)));
    z.X = ff2_first(U2);
    z.Y = ff2_second(U2);
    z.Px = ff2_first(PU2);
    z.Py = ff2_second(PU2);
    z.T = ff_add(z.T, ff_mul(lenff, ff_add_f(k.tau, -k.b0pt * d)));
}

// Deviation of Omega (Eq. (6b), velocity along the kinetic momentum) from the
// on-axis reference -(1 + G) ks s^, in the relabelled frame (x~, y~, z~) =
// (y, s, x) (a cyclic permutation, a proper rotation) where the reference axis
// is y~ as in a sector bend: f = G (gamma - 1) ks/P^2,
//   Omega_x = f kx, Omega_y = f ky (first order, rounded to FP32 once),
//   Omega_s + (1 + G) ks = ks (1 + G)(P - 1)/P + f (Ps - P) - a ks d.
__device__ __forceinline__ void solenoid_dev_omega(const MConst& k, const MState& z, const FF& eta, const FF& f,
                                                   const FF& ks1G, float ks, float dPsP, float d, float& ox_t,
                                                   FF& oy_t, float& oz_t) {
    const FF kx = ff_add(z.Px, ff_mul(eta, z.Y)), ky = ff_add(z.Py, ff_neg(ff_mul(eta, z.X)));
    const FF fx = ff_mul(f, kx), fy = ff_mul(f, ky);
    ox_t = fy.hi + fy.lo;
    oz_t = fx.hi + fx.lo;
    oy_t = ff_addn(ff_mul(ks1G, k.PM1P), f.hi * dPsP - k.a * ks * d);
}

// Thin-pancake fringe spin kick of a solenoid, Eq. (solFringe):
//   w = sign (ks/2)/Ps' [a (X, Y, 0) - G (gamma - 1)(X Px + Y Py)/P^2 (px', py', Ps')]
// with (px', py') = (Px + (ks/4) Y, Py - (ks/4) X); the first-order part
// sign (ks/2)(a/P)(X, Y) compensated, the rest in FP32; NaN if Ps'^2 <= 0.
__device__ __forceinline__ CNQ mixed_solenoid_fringe(const MConst& k, const MState& z, const FF& ks, float etaf,
                                                     float sign) {
    const float pxk = z.Px.hi + etaf * z.Y.hi, pyk = z.Py.hi - etaf * z.X.hi;
    float dk, ppk;
    const FF ipsk = inv_ps(k, pxk, pyk, dk, ppk);
    const float ipsf = ipsk.hi;
    const float hks = 0.5f * sign * ks.hi;
    const float pre = hks * ipsf;
    const float xp = (z.X.hi * z.Px.hi + z.Y.hi * z.Py.hi) * k.invPf * k.invPf * k.c;
    const FF c1 = ff_mul(k.aP, FF{0.5f * sign * ks.hi, 0.5f * sign * ks.lo});
    const FF bx = ff_add_f(ff_mul(z.X, c1), hks * k.a * z.X.hi * dk - pre * xp * pxk);
    const FF by = ff_add_f(ff_mul(z.Y, c1), hks * k.a * z.Y.hi * dk - pre * xp * pyk);
    const float bz = -pre * xp * ((k.P2 - ppk) * ipsf);
    CNQ q = cnq_from_rotvec(bx, by, bz);
    if (!(k.P2 - ppk > 0.0f)) q.w = __int_as_float(0x7fc00000);   // quiet NaN: the particle is lost
    return q;
}

// Thin fringe spin kick of a multipole, quadrupole, sector or TEAPOT bend (Sec. 4.5,
// Eq. (skfringe)) as a near-identity quaternion about the longitudinal axis:
// angle theta = -sign (1 + G) sum_m (b_m/(B rho)) Im (X + iY)^m / m with b_1 =
// eta h, b_2 = k1, b_3 = k2/2 (the kick is below 1e-3 rad, so FP32 and the
// series of cos(theta/2) - 1 and sin(theta/2) to theta^3 suffice).
__device__ __forceinline__ CNQ mixed_fringe(const MixElem& el, int type, const MState& z, float sign, float onepG) {
    const float X = z.X.hi, Y = z.Y.hi;
    float sum;
    if (type == ST_SBEND || type == ST_TEAPOT) {
        sum = el.eta * el.h * Y;
    } else {
        sum = el.k1 * X * Y;
        if (type == ST_MULT) sum += 0.5f * el.k2 * Y * (X * X - Y * Y * (1.0f / 3.0f));
    }
    const float th = -sign * onepG * sum;
    CNQ q;
    q.w = -0.125f * th * th;
    q.x = FF{0.0f, 0.0f};
    q.y = FF{0.0f, 0.0f};
    q.z = FF{0.5f * th * (1.0f - th * th * (1.0f / 24.0f)), 0.0f};
    return q;
}

// One multipole half step of the drift-kick-drift map: drift dl (compensated
// length; 0 skips it), kick of k1, k2 over the compensated lengths k1l = k1 l,
// k2hl = k2 l / 2, k2l = k2 l, drift dl2.  ips_ff, d, pp: 1/Ps and its
// deviation at the current momenta (updated after the kick).
__device__ __forceinline__ void mixed_mult_half(MState& z, const MConst& k, const FF& dl, const FF& dl2, const FF& k1l,
                                                const FF& k2hl, const FF& k2l, FF& ips_ff, float& d, float& pp) {
    if (dl.hi != 0.0f) drift_inc(z, k, dl, ips_ff, d);
    const FF x2my2 = ff_add(ff_mul(z.X, z.X), ff_neg(ff_mul(z.Y, z.Y)));
    const FF kx = ff_add(ff_mul(z.X, k1l), ff_mul(x2my2, k2hl));
    const FF ky = ff_add(ff_mul(z.Y, k1l), ff_mul(ff_mul(z.X, z.Y), k2l));
    z.Px = ff_add(z.Px, ff_neg(kx));
    z.Py = ff_add(z.Py, ky);
    ips_ff = inv_ps(k, z.Px.hi, z.Py.hi, d, pp);
    if (dl2.hi != 0.0f) drift_inc(z, k, dl2, ips_ff, d);
}

// H_qNL over len in increment form (Eq. (25)); d, pp at the current momenta
__device__ __forceinline__ void mixed_quad_nonlinear(MState& z, const MConst& k, float len, const FF& lenff, float d,
                                                     float pp) {
    z.X = ff_add_f(z.X, len * z.Px.hi * d);
    z.Y = ff_add_f(z.Y, len * z.Py.hi * d);
    z.T = ff_add(z.T, ff_mul(lenff, ff_add_f(k.tau, -k.b0pt * (d - 0.5f * pp * k.invPf * k.invPf * k.invPf))));
}

// ---- rectangular bend (Sec. 3.2): an FP64 island ------------------------------
// In the magnet's straight frame the on-axis particle's Px runs from
// sin(phi_in) to sin(phi_out), so its precession rate (1 + G gamma) b/Ps
// changes along the body and the levels of the Romberg table do not share one
// reference rotation: the element is tracked in FP64 with the FP64 tracker's
// maps (entrance rotation, fringe map, body slices, exit fringe, offset, exit
// rotation, time offset; Omega at the slice edges and the Romberg table, or
// Omega at the slice middles for the midpoint schemes), from the compensated
// state converted exactly to FP64, and the element's normalised rotation is
// composed into the compensated turn quaternion.  Returns false if the
// particle is lost (state unchanged then).
__device__ __forceinline__ void fq_premul_quat64(FQ& qt, const Quat& r) {
    float2 rq[4];
    const double c[4] = {r.w, r.x, r.y, r.z};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const FF f = ff_make(c[i]);
        rq[i] = make_float2(f.hi, f.lo);
    }
    fq_premul_ref(qt, rq);
}

__device__ __forceinline__ void pconst_fp64(const RefConst& ref, double Pt, PConst& pc) {
    pc.Pt = Pt;
    pc.P2 = 1.0 + 2.0 * Pt * ref.inv_beta0 + Pt * Pt;
    pc.invP = rsqrt(pc.P2);
    pc.P = pc.P2 * pc.invP;
    pc.invP2 = pc.invP * pc.invP;
    pc.b0pt = ref.inv_beta0 + Pt;
    const double gamma = ref.gamma0 * (1.0 + ref.beta0 * Pt);
    pc.a = 1.0 + ref.G * gamma;
    pc.c = ref.G * (gamma - 1.0);
    pc.cP2 = pc.c * pc.invP2;
    pc.hP3 = 0.5 * pc.invP * pc.invP2;
}

struct RbendOut {
    MState z;
    Quat r;   // the element's normalised rotation (identity without SPIN)
    bool ok;
};

// MID: the midpoint placement (Omega at the slice middles, the body in
// half-slices; both midpoint schemes place it so for exact maps); otherwise
// Romberg order K.  Not inlined: the FP64 state and level products stay out
// of the mixed kernel's register budget.
template <int K, bool SPIN, bool MID>
__device__ __noinline__ RbendOut mixed_rbend_fp64(MState z, RefConst ref, double Pt, const DevElem* elp) {
    const DevElem& el = *elp;
    RbendOut out;
    out.z = z;
    out.r = Quat{1.0, 0.0, 0.0, 0.0};
    out.ok = false;
    Particle p{ff_to_double(z.X), ff_to_double(z.Px), ff_to_double(z.Y), ff_to_double(z.Py), ff_to_double(z.T)};
    PConst pc;
    pconst_fp64(ref, Pt, pc);
    const double onepG = 1.0 + ref.G;
    const int N = el.n_slices;
    const double ds = el.ds, b = el.a[0];
    Quat q_in{1.0, 0.0, 0.0, 0.0}, q_x{1.0, 0.0, 0.0, 0.0}, qe{1.0, 0.0, 0.0, 0.0};
    bool ok = rbend_rotation(p, pc, el.a[1]);
    if constexpr (SPIN) {
        q_in = quat_about_y(el.a[1]);
        if (el.flags & ST_ELEM_FRINGE) q_in = qmul(rbend_fringe_quat(pc, onepG, p, b), q_in);
    }
    ok = ok && rbend_fringe_orbit(p, pc, b);
    double ox, oy, os;
    if constexpr (MID) {
        const double hd = 0.5 * ds;
        for (int s = 0; s < N; ++s) {
            ok = ok && rbend_body(p, pc, b, hd);
            if constexpr (SPIN) {
                ok = ok && mid_omega(el, ST_RBEND, p, pc, ox, oy, os);
                if (ok) qe = qmul(quat_from_rotvec(ds * ox, ds * oy, ds * os), qe);
            }
            ok = ok && rbend_body(p, pc, b, hd);
        }
    } else {
        LevelProducts<K> lv;
        if constexpr (SPIN) {
            const double pp = p.Px * p.Px + p.Py * p.Py;
            const double ips = rsqrt(pc.P2 - pp);
            precession(p, pc, 0.0, b, 0.0, ips, (pc.P2 - pp) * ips, ox, oy, os);
            lv.add_edge(0, N, ds, ox, oy, os);
        }
        for (int s = 1; s <= N; ++s) {
            ok = ok && rbend_body(p, pc, b, ds);
            if constexpr (SPIN) {
                const double pp = p.Px * p.Px + p.Py * p.Py;
                const double ips = rsqrt(pc.P2 - pp);
                precession(p, pc, 0.0, b, 0.0, ips, (pc.P2 - pp) * ips, ox, oy, os);
                lv.add_edge(s, N, ds, ox, oy, os);
            }
        }
        if constexpr (SPIN) qe = lv.romberg();
    }
    if constexpr (SPIN) {
        if (el.flags & ST_ELEM_FRINGE) q_x = rbend_fringe_quat(pc, onepG, p, -b);
    }
    ok = ok && rbend_fringe_orbit(p, pc, -b);
    p.X -= el.a[3];
    ok = ok && rbend_rotation(p, pc, el.a[2]);
    if constexpr (SPIN) q_x = qmul(quat_about_y(el.a[2]), q_x);
    p.T += el.a[4] * ref.inv_beta0;
    if (!ok || !isfinite(p.X + p.Px + p.Y + p.Py + p.T + qe.w + qe.x + qe.y + qe.z)) return out;
    if constexpr (SPIN) out.r = qnormalize(qmul(q_x, qmul(qe, q_in)));
    out.z.X = ff_make(p.X);
    out.z.Px = ff_make(p.Px);
    out.z.Y = ff_make(p.Y);
    out.z.Py = ff_make(p.Py);
    out.z.T = ff_make(p.T);
    out.ok = true;
    return out;
}

// Track particle i for n_turns turns through the mixed-precision tables in
// shared memory (table, seq, rho); state in the FP64 pair-SoA arrays.  If
// spin_sum ([3][n_all]) is given, the spin after every turn is added to it.
// FR: the lattice's table entries may carry ST_MIX_FRINGE (a separate
// instantiation, so that lattices without fringe kicks run the plain loop).
// EXT: the lattice may hold TEAPOT bends and solenoids, O4 (with EXT):
// fourth-order slices, RB (with both): rectangular bends (instantiations of
// their own too, so that each keeps the register budget of what it runs).
template <int K, bool SPIN = true, bool FR = false, bool EXT = false, bool O4 = false, bool RB = false>
__device__ __forceinline__ void mixed_track_particle(const MixElem* __restrict__ table,
                                                     const uint16_t* __restrict__ seq,
                                                     const float2* __restrict__ rho, int n_seq, const RefConst& ref,
                                                     double2* __restrict__ xpx, double2* __restrict__ ypy,
                                                     double2* __restrict__ tpt, double2* __restrict__ sxy,
                                                     double* __restrict__ szp, uint8_t* __restrict__ lost, int64_t i,
                                                     int n_turns, int32_t* status = nullptr,
                                                     double* __restrict__ spin_sum = nullptr, int64_t n_all = 0) {
    // table entries below the sequence (both staged into shared memory back to back)
    const int n_table = (int)(((const char*)seq - (const char*)table) / sizeof(MixElem));
    // state and per-particle constants (FP64 -> compensated FP32)
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

    MQuad mq, mq2;   // mq2: the second coefficient set of fourth-order matrix-kick slices
    mq.key_k = -1.0f;
    mq.key_s = 0.0f;
    mq2.key_k = -1.0f;
    mq2.key_s = 0.0f;
    MixLevels<K> lv;
    bool is_lost = false;

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
                if constexpr (SPIN) fq_premul_ref(qt, el.rq);
                continue;
            }
            const MState z0 = z;
            if constexpr (RB) {
                if (type == ST_RBEND) {
                    const RbendOut o = mixed_rbend_fp64<K, SPIN, false>(z, ref, Pt, &el.d64);
                    if (!o.ok) {
                        is_lost = true;
                        break;
                    }
                    z = o.z;
                    if constexpr (SPIN) fq_premul_quat64(qt, o.r);
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
            float ox, os;
            const bool teapot = EXT && type == ST_TEAPOT;
            if (type == ST_SBEND || teapot) {
                const float h = el.h, eta = el.eta;
                const float py = z.Py.hi;
                const float Pa2 = k.P2 - py * py;
                float px = z.Px.hi;
                float ps2 = Pa2 - px * px;
                float ips = rsqrtf(ps2);
                float Ps = ps2 * ips;
                // Ps - 1 = (P - 1) + (Ps - P), the second term dPsP = -p^2/(Ps + P) second
                // order (about 1e-8), so a reciprocal good to 2 ulp is exact enough for it
                float dPsP = -__fdividef(px * px + py * py, Ps + k.P);
                FF PsM1 = ff_add_f(k.PM1, dPsP);
                const float etah = eta * h;
                const float cu = k.c * py * etah * k.invPf * k.invPf;     // G(gamma-1)(u.b)/P, u.b = Py eta h / P
                const FF ietads{el.ietads_ff.x, el.ietads_ff.y};
                const FF sbieh{el.sbieh_ff.x, el.sbieh_ff.y};
                const FF sbff{el.sb_ff.x, el.sb_ff.y};
                const FF cbmieh{el.cbmieh_ff.x, el.cbmieh_ff.y};
                const FF etahff{el.etah_ff.x, el.etah_ff.y};
                const FF omeff{el.ome_ff.x, el.ome_ff.y};
                const bool eta1 = el.ome_ff.x == 0.0f;   // eta = 1: A needs no 1 - eta term
                const FF iehff{el.ieh_ff.x, el.ieh_ff.y};
                // T increment of the bend without the path term: (1 - 1/eta) ds/beta0 - Pt ds/eta
                const FF dT0 = ff_add(FF{el.dTeta_ff.x, el.dTeta_ff.y}, ff_neg(ff_mul(k.Ptf, ietads)));
                const FF cbm1ff{el.cbm1_ff.x, el.cbm1_ff.y};
                // 1/P_a^2 = (1/P^2) / (1 - Py^2/P^2), compensated (the correction is tiny)
                const float epy = py * py * k.invPf * k.invPf;
                const FF iPa2ff = ff_add_f(k.invP2, k.invP2.hi * epy * (1.0f + epy));
                // deviation of Omega (Eq. (6b)) from the on-axis reference:
                //   dOy = eta h N / Ps + (1 + hX) cu Py / Ps,
                //     N = a0 (Ps - 1 - hX) - (1 + hX) (a - a0) = c1 + a0 (Ps - P) - hX (a0 + da),
                //     c1 = a0 (P - 1) - da (per particle, FP64: its two terms cancel to O(Pt));
                //   its first-order part eta h c1 / P - (eta h^2 a0 / P) X compensated, the rest
                //   eta h [(a0 (Ps - P) - hX da) / P + N (1/Ps - 1/P)] + (1 + hX) cu Py / Ps in FP32;
                //   dOx = (1 + hX) cu Px / Ps,  dOs = (1 + hX) cu
                const FF B0 = ff_mul(etahff, k.c1P);
                const FF B1 = ff_mul(FF{el.eh2_ff.x, el.eh2_ff.y}, k.a0P);
                const float apda = k.a0 + k.da;
                auto dev_omega = [&](const FF& Xf, float Pxv, float Psv, float ipsv, float dPsPv, float& dx, FF& dy,
                                     float& dz) {
                    const float hX = h * Xf.hi;
                    const float g = (1.0f + hX) * ipsv;
                    const float dd = -dPsPv * k.invPf * ipsv;                 // 1/Ps - 1/P
                    const float Nf = k.c1 + k.a0 * dPsPv - hX * apda;
                    const float rest = etah * ((k.a0 * dPsPv - hX * k.da) * k.invPf + Nf * dd) + g * cu * py;
                    dy = ff_addn(ff_add(B0, ff_neg(ff_mul(B1, Xf))), rest);
                    dx = g * cu * Pxv;
                    dz = g * cu * Psv;
                };
                FF oyf;
                const float2* rh = rho + el.rho_off;
                // one loop over the slice edges (edge 0: no orbit step), so that the
                // spin edge code exists once
                for (int s = 0; s <= N; ++s) {
                  if (s > 0 && teapot) {
                    // TEAPOT slice (Sec. 3.6): curved drift, kick, curved drift; the
                    // momentum quantities of the slice edge for Omega (Py is constant)
                    if (O4 && (el.type & ST_MIX_ORDER4)) {
                        // fourth order: CD(x1 ds/2) K(x1 ds) CD((x1 + x0) ds/2) K(x0 ds) ... mirrored
                        const FF ka{el.o4_k1_ff[0].x, el.o4_k1_ff[0].y}, kha{el.o4_k2h_ff[0].x, el.o4_k2h_ff[0].y};
                        const FF kb{el.o4_k1_ff[1].x, el.o4_k1_ff[1].y}, khb{el.o4_k2h_ff[1].x, el.o4_k2h_ff[1].y};
                        mixed_curved_drift(z, k, el.td[0], h);
                        mixed_teapot_kick(z, ka, kha);
                        mixed_curved_drift(z, k, el.td[1], h);
                        mixed_teapot_kick(z, kb, khb);
                        mixed_curved_drift(z, k, el.td[1], h);
                        mixed_teapot_kick(z, ka, kha);
                        mixed_curved_drift(z, k, el.td[0], h);
                    } else {
                        const MixCurvedDrift& cd = el.td[0];
                        mixed_curved_drift(z, k, cd, h);
                        mixed_teapot_kick(z, FF{el.ehl_ff.x, el.ehl_ff.y}, FF{el.ehlh_ff.x, el.ehlh_ff.y});
                        mixed_curved_drift(z, k, cd, h);
                    }
                    px = z.Px.hi;
                    ps2 = Pa2 - px * px;
                    ips = rsqrtf(ps2);
                    Ps = ps2 * ips;
                    dPsP = -__fdividef(px * px + py * py, Ps + k.P);
                  } else if (s > 0) {
                    // exact bend over ds, Eq. (10): (Px, A = Ps - eta(1+hX)) rotates by h ds;
                    // dX = (dPs - dA)/(eta h) with dA = A (cos - 1) - Px sin
                    // A = (Ps - 1) + (1 - eta) - eta h X, compensated (first order in the
                    // momentum deviation and in X)
                    FF PsE = PsM1;
                    if (!eta1) PsE = ff_add(PsM1, omeff);
                    const FF Aff = ff_add(PsE, ff_neg(ff_mul(etahff, z.X)));
                    const FF dPxff = ff_add(ff_mul(Aff, sbff), ff_mul(z.Px, cbm1ff));
                    // dPx / (eta h) = A sin(h ds)/(eta h) + Px (cos(h ds) - 1)/(eta h)
                    const FF dPxieh = ff_mul(dPxff, iehff);
                    const float dPx = dPxff.hi;
                    const float pxf = px + dPx;
                    const float ps2f = Pa2 - pxf * pxf;
                    const float ipsf = rsqrtf(ps2f);
                    const float Psf = ps2f * ipsf;
                    const float dPsPf = -__fdividef(pxf * pxf + py * py, Psf + k.P);
                    const FF PsfM1 = ff_add_f(k.PM1, dPsPf);
                    // The second-order terms below carry the factor 1/(eta h) (hundreds of
                    // metres in a large ring), so they are compensated as well.
                    // Q = (Ps_f - Ps)/(eta h) = -dPx/(eta h) (Px + Px_f) / (Ps + Ps_f), with
                    // 1/(Ps + Ps_f) = (1/2) / (1 + u/2), u = (Ps - 1) + (Ps_f - 1)
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
                    // dX = (dPs - dA)/(eta h), dA = A (cos - 1) - Px sin
                    const FF dX = ff_add(ff_add(ff_mul(z.Px, sbieh), ff_neg(ff_mul(Aff, cbmieh))), Q);
                    const FF dY = ff_mul(z.Py, ff_add(ietads, dpsieh));
                    z.X = ff_add(z.X, dX);
                    z.Px = ff_add(z.Px, dPxff);
                    z.Y = ff_add(z.Y, dY);
                    z.T = ff_add(z.T, ff_add(dT0, ff_neg(ff_mul(k.b0ptf, dpsieh))));
                    // the slice-end momentum quantities carry over (px_f differs from the
                    // compensated Px's high part by at most an ulp: 1e-16 in Ps - P)
                    px = pxf;
                    ps2 = ps2f;
                    ips = ipsf;
                    Ps = Psf;
                    dPsP = dPsPf;
                    PsM1 = PsfM1;
                  }
                    if constexpr (SPIN) {
                        dev_omega(z.X, px, Ps, ips, dPsP, ox, oyf, os);
                        const float2 r = rh[s];
                        lv.add_bend(s, N, el, r.x, r.y, ox, oyf, os);
                    }
                }
            } else if (EXT && type == ST_SOLENOID) {
                // Sec. 3.7: exact body map in N slices, Omega at the slice edges along
                // the kinetic momentum, whose Ps the body conserves; the spin edges in
                // the relabelled frame (y, s, x) with the bend's deviation code
                const FF eta{el.seta_ff.x, el.seta_ff.y}, ks{el.ks_ff.x, el.ks_ff.y};
                const FF kx = ff_add(z.Px, ff_mul(eta, z.Y)), ky = ff_add(z.Py, ff_neg(ff_mul(eta, z.X)));
                FF dPsPk, dk;
                ps_deviations(k, kx, ky, dPsPk, dk);
                const MSolSlice m = mixed_solenoid_slice(eta, (double)el.ds_ff.x + (double)el.ds_ff.y, invP64, dk.hi);
                const FF dsff{el.ds_ff.x, el.ds_ff.y};
                const FF f = ff_mul(k.cP2, ks);
                const FF ks1G{el.ks1G_ff.x, el.ks1G_ff.y};
                const float2* rh = rho + el.rho_off;
                for (int s = 0; s <= N; ++s) {
                    if (s > 0) mixed_solenoid_map(z, k, m, dsff, dk.hi);
                    if constexpr (SPIN) {
                        FF oyt;
                        solenoid_dev_omega(k, z, eta, f, ks1G, ks.hi, dPsPk.hi, dk.hi, ox, oyt, os);
                        const float2 r = rh[s];
                        lv.add_bend(s, N, el, r.x, r.y, ox, oyt, os);
                    }
                }
            } else {   // ST_MULT (drift-kick-drift; thin lenses too) or ST_QUAD_MK (matrix-kick)
                // one loop over the slice edges for both straight element kinds (edge
                // 0: no orbit step), so that the spin edge code exists once
                const bool is_mult = type == ST_MULT;
                const float k1 = el.k1;
                const float k2 = is_mult ? el.k2 : 0.0f;   // quadrupoles keep |k1| in el.k2
                const FF dsff{el.ds_ff.x, el.ds_ff.y};
                const FF half{0.5f * el.ds_ff.x, 0.5f * el.ds_ff.y};   // half drift (0 for a thin lens)
                const FF k1ds{el.k1ds_ff.x, el.k1ds_ff.y};   // quadrupoles: |k1|
                const FF k2h{el.k2h_ff.x, el.k2h_ff.y};
                const FF k2ds{el.k2ds_ff.x, el.k2ds_ff.y};
                FF Aw;   // (a/P) k1 ds, compensated: the first-order rotation per unit Y (x) and X (y)
                if (is_mult) {
                    Aw = ff_mul(k.aP, k1ds);
                } else {
                    const float absk = el.k2, hs = 0.5f * ds;
                    // (fourth-order slices keep their own two coefficient sets)
                    if (!(O4 && (el.type & ST_MIX_ORDER4)) && (mq.key_k != absk || mq.key_s != hs))
                        mquad_coeffs(mq, invP64, (double)el.k1ds_ff.x + (double)el.k1ds_ff.y,
                                     0.5 * ((double)el.ds_ff.x + (double)el.ds_ff.y), absk, hs);
                    Aw = ff_mul_f(ff_mul(ff_mul(k.aP, k1ds), dsff), k1 >= 0.0f ? 1.0f : -1.0f);
                }
                const bool o4 = O4 && (el.type & ST_MIX_ORDER4);
                FF ips_ff = inv_ps(k, z.Px.hi, z.Py.hi, d, pp);
                float ips = ips_ff.hi, Ps = (k.P2 - pp) * ips;
                for (int s = 0; s <= N; ++s) {
                    if (s > 0 && o4) {
                        // fourth order (Sec. 3.3): Yoshida's S2(x1 ds) S2(x0 ds) S2(x1 ds) with
                        // adjacent half steps merged: D K D' K0 D' K D or L N L' N0 L' N L
                        const FF d1{el.o4_d_ff[0].x, el.o4_d_ff[0].y}, d2{el.o4_d_ff[1].x, el.o4_d_ff[1].y};
                        if (is_mult) {
                            const FF zero{0.0f, 0.0f};
                            const FF k1a{el.o4_k1_ff[0].x, el.o4_k1_ff[0].y}, k1b{el.o4_k1_ff[1].x, el.o4_k1_ff[1].y};
                            const FF k2ha{el.o4_k2h_ff[0].x, el.o4_k2h_ff[0].y};
                            const FF k2hb{el.o4_k2h_ff[1].x, el.o4_k2h_ff[1].y};
                            const FF k2a{el.o4_k2_ff[0].x, el.o4_k2_ff[0].y}, k2b{el.o4_k2_ff[1].x, el.o4_k2_ff[1].y};
                            mixed_mult_half(z, k, d1, d2, k1a, k2ha, k2a, ips_ff, d, pp);
                            mixed_mult_half(z, k, zero, d2, k1b, k2hb, k2b, ips_ff, d, pp);
                            mixed_mult_half(z, k, zero, d1, k1a, k2ha, k2a, ips_ff, d, pp);
                        } else {
                            const float absk = el.k2, l1 = d1.hi, l2 = d2.hi;
                            const double absk64 = (double)el.k1ds_ff.x + (double)el.k1ds_ff.y;
                            if (mq.key_k != absk || mq.key_s != l1)
                                mquad_coeffs(mq, invP64, absk64, (double)d1.hi + (double)d1.lo, absk, l1);
                            if (mq2.key_k != absk || mq2.key_s != l2)
                                mquad_coeffs(mq2, invP64, absk64, (double)d2.hi + (double)d2.lo, absk, l2);
                            const FF sa{el.o4_s_ff[0].x, el.o4_s_ff[0].y}, sb{el.o4_s_ff[1].x, el.o4_s_ff[1].y};
                            quad_linear_inc(z, k, mq, k1);
                            inv_ps(k, z.Px.hi, z.Py.hi, d, pp);
                            mixed_quad_nonlinear(z, k, sa.hi, sa, d, pp);
                            quad_linear_inc(z, k, mq2, k1);
                            inv_ps(k, z.Px.hi, z.Py.hi, d, pp);
                            mixed_quad_nonlinear(z, k, sb.hi, sb, d, pp);
                            quad_linear_inc(z, k, mq2, k1);
                            inv_ps(k, z.Px.hi, z.Py.hi, d, pp);
                            mixed_quad_nonlinear(z, k, sa.hi, sa, d, pp);
                            quad_linear_inc(z, k, mq, k1);
                            ips_ff = inv_ps(k, z.Px.hi, z.Py.hi, d, pp);
                        }
                        ips = ips_ff.hi;
                        Ps = (k.P2 - pp) * ips;
                    } else if (s > 0) {
                        if (is_mult) {
                            drift_inc(z, k, half, ips_ff, d);
                            // kick of H_m over ds, compensated (the sextupole kick is first
                            // order in the betatron offset around a dispersive orbit)
                            // (X^2, XY) in one packed product, then X^2 - Y^2
                            const FF2 xx = ff2_mul(ff2_pack(z.X, z.X), ff2_pack(z.X, z.Y));
                            const FF x2my2 = ff_add(ff2_first(xx), ff_neg(ff_mul(z.Y, z.Y)));
                            // (-kx, ky) = -(X, -Y) k1 ds - (x2my2 k2 ds/2, -XY k2 ds), packed
                            const FF2 kk = ff2_add(ff2_mul(ff2_pack(ff_neg(z.X), z.Y), ff2_pack(k1ds, k1ds)),
                                                   ff2_mul(ff2_pack(ff_neg(x2my2), ff2_second(xx)), ff2_pack(k2h, k2ds)));
                            const FF2 PU = ff2_add(ff2_pack(z.Px, z.Py), kk);
                            z.Px = ff2_first(PU);
                            z.Py = ff2_second(PU);
                            ips_ff = inv_ps(k, z.Px.hi, z.Py.hi, d, pp);
                            ips = ips_ff.hi;
                            Ps = (k.P2 - pp) * ips;
                            drift_inc(z, k, half, ips_ff, d);
                        } else {
                            quad_linear_inc(z, k, mq, k1);
                            inv_ps(k, z.Px.hi, z.Py.hi, d, pp);
                            // H_qNL over ds, Eq. (25), in increment form:
                            // dX = ds Px (1/Ps - 1/P); dT = ds [tau - (1/beta0+Pt)(d - p^2/(2P^3))]
                            {   // (X, Y) += ds d (Px, Py): second order, added to the pair
                                const float2 inc = __fmul2_rn(make_float2(z.Px.hi, z.Py.hi), make_float2(ds * d, ds * d));
                                FF2 U = ff2_pack(z.X, z.Y);
                                float2 sh, se;
                                two_sum2(U.hi, inc, sh, se);
                                se = __fadd2_rn(se, U.lo);
                                U.hi = __fadd2_rn(sh, se);
                                U.lo = f2_sub(se, f2_sub(U.hi, sh));
                                z.X = ff2_first(U);
                                z.Y = ff2_second(U);
                            }
                            z.T = ff_add(z.T, ff_mul(dsff, ff_add_f(k.tau, -k.b0pt * (d - 0.5f * pp * k.invPf * k.invPf * k.invPf))));
                            quad_linear_inc(z, k, mq, k1);
                            ips_ff = inv_ps(k, z.Px.hi, z.Py.hi, d, pp);
                            ips = ips_ff.hi;
                            Ps = (k.P2 - pp) * ips;
                        }
                    }
                    if constexpr (SPIN) {
                        const bool end = s == 0 || s == N;   // trapezoid end weights
                        FF bx, by;
                        float bz;
                        straight_edge(k, z, k1, k2, end ? ff_scale2(Aw, 0.5f) : Aw, end ? 0.5f * ds : ds, d, ips, Ps,
                                      bx, by, bz);
                        lv.add_straight(s, bx, by, bz);
                    }
                }
            }
            if constexpr (SPIN) {
                CNQ dq = lv.romberg();
                if (EXT && type == ST_SOLENOID) {
                    // back from the relabelled frame; the fringe kicks of Sec. 4.4 at
                    // the entrance (entry state) and the exit
                    dq = CNQ{dq.w, dq.z, dq.x, dq.y};
                    const FF ks{el.ks_ff.x, el.ks_ff.y};
                    const CNQ fi = mixed_solenoid_fringe(k, z0, ks, el.setaf_ff.x, 1.0f);
                    const CNQ fo = mixed_solenoid_fringe(k, z, ks, el.setaf_ff.x, -1.0f);
                    if (!isfinite(z.X.hi + z.Px.hi + z.Y.hi + z.Py.hi + z.T.hi + dq.w + dq.x.hi + dq.y.hi +
                                  dq.z.hi + fi.w + fi.x.hi + fi.y.hi + fi.z.hi + fo.w + fo.x.hi + fo.y.hi + fo.z.hi)) {
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
                // element rotation R_L (1 + D) into the compensated turn quaternion,
                // between the entrance and exit fringe kicks if the element has them
                const bool fr = FR && (el.type & ST_MIX_FRINGE);
                if (fr) fq_premul_cnq(qt, mixed_fringe(el, type, z0, 1.0f, 1.0f + (float)ref.G));
                fq_premul_cnq(qt, dq);
                if (type == ST_SBEND || (EXT && type == ST_TEAPOT)) fq_premul_about_y(qt, el.rq);
                if (fr) fq_premul_cnq(qt, mixed_fringe(el, type, z, -1.0f, 1.0f + (float)ref.G));
            } else {
                if (!isfinite(z.X.hi + z.Px.hi + z.Y.hi + z.Py.hi + z.T.hi)) {
                    z = z0;
                    is_lost = true;
                    break;
                }
            }
        }
        // FP64 once per turn: compose, renormalise, rotate the spin (a particle lost
        // inside the turn gets the rotation up to the element where it was lost)
        if constexpr (SPIN) {
            Quat q64{ff_to_double(qt.w), ff_to_double(qt.x), ff_to_double(qt.y), ff_to_double(qt.z)};
            q64 = qnormalize(q64);
            rotate_vec(q64, sx, sy, sz);
            if (spin_sum) {   // stroboscopic sum of the spin at the start of the lattice
                spin_sum[i] += sx;
                spin_sum[n_all + i] += sy;
                spin_sum[2 * n_all + i] += sz;
            }
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
