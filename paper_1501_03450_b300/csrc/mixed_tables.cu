// Host-side preparation of the mixed-precision tracker's tables (all in FP64,
// rounded to FP32 once at the end):
//   - per unique element: orbit constants in increment form (cos(h ds) - 1
//     instead of cos(h ds)), the reference precession rate of the on-axis,
//     on-momentum particle, and for every edge weight the constants that give
//     an edge rotation's deviation from the reference rotation;
//   - first-order (linear) map coefficients as compensated (hi, lo) float
//     pairs, the reference rotation of each element as a (hi, lo) quaternion;
//   - the element sequence (uint16) and, for bends, cos/sin of the reference
//     rotation accumulated up to every slice edge.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "st_internal.cuh"

namespace st {

namespace {

float2 split(double x) {
    const float hi = (float)x;
    return make_float2(hi, (float)(x - (double)hi));
}

// Derivatives C^(m)(u0), S^(m)(u0), m = 0..MIX_TAYLOR, of C(u) = cos(sqrt(u)/2)
// and S(u) = sin(sqrt(u)/2)/sqrt(u).
void half_angle_derivatives(double u0, double C[MIX_TAYLOR + 1], double S[MIX_TAYLOR + 1]) {
    if (u0 < 100.0) {
        // power series about 0: C = sum (-1)^n u^n / (4^n (2n)!),
        // S = sum (-1)^n u^n / (2 4^n (2n+1)!); differentiate term by term
        for (int m = 0; m <= MIX_TAYLOR; ++m) {
            double c = 0.0, s = 0.0;
            for (int n = m; n < 80; ++n) {
                double f2n = 1.0, f2n1;
                for (int k = 2; k <= 2 * n; ++k) f2n *= k;
                f2n1 = f2n * (2 * n + 1);
                double p4 = std::pow(4.0, n);
                double fall = 1.0;   // n! / (n-m)!
                for (int k = 0; k < m; ++k) fall *= (n - k);
                double up = std::pow(u0, n - m);
                double sign = (n % 2) ? -1.0 : 1.0;
                c += sign * fall * up / (p4 * f2n);
                s += sign * fall * up / (2.0 * p4 * f2n1);
                if (!std::isfinite(f2n)) break;
            }
            C[m] = c;
            S[m] = s;
        }
    } else {
        // 4u S' = C - 2S and C' = -S/4, differentiated n times:
        // S^(n+1) = (C^(n) - (2 + 4n) S^(n)) / (4u), C^(n+1) = -S^(n)/4
        double th = std::sqrt(u0);
        C[0] = std::cos(0.5 * th);
        S[0] = std::sin(0.5 * th) / th;
        for (int n = 0; n < MIX_TAYLOR; ++n) {
            C[n + 1] = -S[n] / 4.0;
            S[n + 1] = (C[n] - (2.0 + 4.0 * n) * S[n]) / (4.0 * u0);
        }
    }
}

}  // namespace

int build_mixed_tables(LatticeImpl& L) {
    const double G = L.ref.G, gamma0 = L.ref.gamma0, beta0 = L.ref.beta0;
    const double a0 = 1.0 + G * gamma0;
    const int nu = L.n_unique, ne = L.n_elements;
    std::vector<MixElem> me(nu);
    std::vector<float> rho;   // float2 pairs
    for (int u = 0; u < nu; ++u) {
        const DevElem& d = L.h_table[u];
        MixElem m;
        memset(&m, 0, sizeof(m));
        m.type = d.type;
        m.n_slices = d.n_slices;
        m.ds = (float)d.ds;
        m.ds_ff = split(d.ds);
        double rq[4] = {1.0, 0.0, 0.0, 0.0};
        double omr = 0.0;
        switch (d.type) {
        case ST_MULT:
        case ST_THIN_MULT:
            // a thin lens (Sec. 3.5) is the multipole without its drifts, in
            // the unit kick parameter (ds = 1/N, integrated strengths)
            m.type = ST_MULT;
            m.k1 = (float)d.a[0];
            m.k2 = (float)d.a[1];
            m.k1ds_ff = split(d.a[0] * d.ds);
            m.k2h_ff = split(0.5 * d.a[1] * d.ds);
            m.k2ds_ff = split(d.a[1] * d.ds);
            if (d.type == ST_THIN_MULT) m.ds_ff = split(0.0);   // no drift
            break;
        case ST_QUAD_MK:
            m.k1 = (float)d.a[0];
            m.k2 = (float)d.a[1];          // |k1|
            m.k1ds_ff = split(d.a[1]);     // |k1| as (hi, lo): the matrix-kick coefficients need it exactly
            break;
        case ST_SBEND:
        case ST_TEAPOT: {
            const double h = d.a[0], eta = d.a[1];
            // field and curvature: the spin constants are the same for both kinds
            // (Omega at the same slice edges)
            m.h = (float)h;
            m.eta = (float)eta;
            m.etah_ff = split(eta * h);
            m.eh2_ff = split(eta * h * h);
            if (d.type == ST_SBEND) {
                // exact bend over ds (Eq. (10)) and over ds/2 (midpoint schemes)
                const double hs = std::sin(0.5 * h * d.ds);
                m.cbm1 = (float)(-2.0 * hs * hs);
                m.sb = (float)std::sin(h * d.ds);
                m.ieta = (float)(1.0 / eta);
                m.ieh = (float)(1.0 / (eta * h));
                m.ieh_ff = split(1.0 / (eta * h));
                m.dT_eta = (float)((1.0 - 1.0 / eta) * d.ds / beta0);
                m.sbieh_ff = split(std::sin(h * d.ds) / (eta * h));
                m.ietads_ff = split(d.ds / eta);
                m.sb_ff = split(std::sin(h * d.ds));
                m.cbmieh_ff = split(-2.0 * hs * hs / (eta * h));
                m.ome_ff = split(1.0 - eta);
                m.cbm1_ff = split(-2.0 * hs * hs);
                m.dTeta_ff = split((1.0 - 1.0 / eta) * d.ds / beta0);
                const double hq = std::sin(0.25 * h * d.ds);
                m.sbh_ff = split(std::sin(0.5 * h * d.ds));
                m.sbiehh_ff = split(std::sin(0.5 * h * d.ds) / (eta * h));
                m.cbm1h_ff = split(-2.0 * hq * hq);
                m.cbmiehh_ff = split(-2.0 * hq * hq / (eta * h));
                m.ietadsh_ff = split(0.5 * d.ds / eta);
                m.dTetah_ff = split((1.0 - 1.0 / eta) * 0.5 * d.ds / beta0);
            } else {
                // TEAPOT (Sec. 3.6): curved drifts of ds/2 and ds/4 and the kick
                // of the bend's field over ds (eta = 0 is a field-free curved frame)
                L.mix_ext = true;
                for (int jj = 0; jj < 2; ++jj) {
                    const double len = (jj == 0 ? 0.5 : 0.25) * d.ds;
                    const double hs2 = std::sin(0.5 * h * len);
                    const double omc = 2.0 * hs2 * hs2, sn = std::sin(h * len);
                    MixCurvedDrift& c = m.td[jj];
                    c.sn_ff = split(sn);
                    c.A1_ff = split(omc / h);
                    c.A2_ff = split(sn / h);
                    c.omc_ff = split(omc);
                    // len - sin(h len)/h, by its series when h len is small (len (h len)^2 / 6
                    // to leading order)
                    const double x = h * len, x2 = x * x;
                    const double lms = std::fabs(x) < 1e-2
                                           ? len * x2 / 6.0 * (1.0 - x2 / 20.0 * (1.0 - x2 / 42.0))
                                           : len - sn / h;
                    c.dT0_ff = split(lms / beta0);
                    c.snb0_ff = split(sn / beta0);
                }
                m.ehl_ff = split(eta * h * d.ds);
                m.ehlh_ff = split(eta * h * h * d.ds);
            }
            // on-axis, on-momentum particle: Omega = (0, h - (1 + G gamma0) eta h, 0)
            omr = h - a0 * eta * h;
            m.omr = (float)omr;
            const double phi = omr * d.ds * d.n_slices;
            rq[0] = std::cos(0.5 * phi);
            rq[2] = std::sin(0.5 * phi);
            m.rho_off = (int)(rho.size() / 2);
            for (int i = 0; i <= d.n_slices; ++i) {
                rho.push_back((float)std::cos(omr * i * d.ds));
                rho.push_back((float)std::sin(omr * i * d.ds));
            }
            break;
        }
        case ST_SOLENOID: {
            // Sec. 3.7: ks, eta = ks/2 (body), ks/4 (fringes); on-axis, on-momentum
            // particle: Omega = -(1 + G) ks s^ (Eq. (6b) with the velocity along s),
            // a rotation about s; the kernel evaluates the deviations in the
            // relabelled frame (y, s, x), where this axis is the second one as in
            // a bend, so the weights and the rho table below are the bend's
            const double ks = d.a[0];
            L.mix_ext = true;
            m.ks_ff = split(ks);
            m.seta_ff = split(d.a[1]);
            m.setaf_ff = split(d.a[2]);
            m.ks1G_ff = split(ks * (1.0 + G));
            omr = -(1.0 + G) * ks;
            m.omr = (float)omr;
            const double phi = omr * d.ds * d.n_slices;
            rq[0] = std::cos(0.5 * phi);
            rq[3] = std::sin(0.5 * phi);
            m.rho_off = (int)(rho.size() / 2);
            for (int i = 0; i <= d.n_slices; ++i) {
                rho.push_back((float)std::cos(omr * i * d.ds));
                rho.push_back((float)std::sin(omr * i * d.ds));
            }
            break;
        }
        case ST_RBEND:
            // Sec. 3.2: tracked in FP64 inside the mixed kernels (in the magnet's
            // straight frame the on-axis particle's precession rate changes along
            // the body, so the reference-and-deviation split does not apply)
            m.d64 = d;
            L.mix_ext = true;
            L.mix_rb = true;
            break;
        case ST_SNAKE:
            for (int c = 0; c < 4; ++c) rq[c] = d.a[c];
            break;
        default:
            break;
        }
        if (d.flags & ST_ELEM_ORDER4) {
            // fourth-order slice of a multipole, matrix-kick quadrupole or TEAPOT bend
            // (the host packs the sub-step lengths into a[2..5])
            m.type |= ST_MIX_ORDER4;
            L.mix_ext = true;
            L.mix_o4 = true;
            for (int jj = 0; jj < 2; ++jj) {
                const double dl = d.a[2 + jj], sl = d.a[4 + jj];
                m.o4_d_ff[jj] = split(dl);
                m.o4_s_ff[jj] = split(sl);
                if (d.type == ST_MULT) {
                    m.o4_k1_ff[jj] = split(d.a[0] * sl);
                    m.o4_k2h_ff[jj] = split(0.5 * d.a[1] * sl);
                    m.o4_k2_ff[jj] = split(d.a[1] * sl);
                } else if (d.type == ST_TEAPOT) {
                    const double h = d.a[0], eta = d.a[1];
                    m.o4_k1_ff[jj] = split(eta * h * sl);
                    m.o4_k2h_ff[jj] = split(eta * h * h * sl);
                    // the curved drifts of the two lengths take the places of the
                    // second-order ones (no midpoint scheme runs fourth-order maps)
                    const double hs2 = std::sin(0.5 * h * dl);
                    const double omc = 2.0 * hs2 * hs2, sn = std::sin(h * dl);
                    MixCurvedDrift& c = m.td[jj];
                    c.sn_ff = split(sn);
                    c.A1_ff = split(omc / h);
                    c.A2_ff = split(sn / h);
                    c.omc_ff = split(omc);
                    const double x = h * dl, x2 = x * x;
                    const double lms = std::fabs(x) < 1e-2
                                           ? dl * x2 / 6.0 * (1.0 - x2 / 20.0 * (1.0 - x2 / 42.0))
                                           : dl - sn / h;
                    c.dT0_ff = split(lms / beta0);
                    c.snb0_ff = split(sn / beta0);
                }
            }
        }
        if ((d.flags & ST_ELEM_FRINGE) &&
            (d.type == ST_MULT || d.type == ST_QUAD_MK || d.type == ST_SBEND || d.type == ST_TEAPOT)) {
            m.type |= ST_MIX_FRINGE;
            L.mix_fringe = true;
        }
        for (int j = 0; j < 6; ++j) {
            const double w = std::ldexp(d.ds, j) * 0.5;
            const double al = w * omr;
            MixWeight& W = m.w[j];
            W.alpha = (float)al;
            W.ch = (float)std::cos(0.5 * al);
            W.sh = (float)std::sin(0.5 * al);
            W.cf = (float)std::cos(al);
            W.sf = (float)std::sin(al);
            double C[MIX_TAYLOR + 1], S[MIX_TAYLOR + 1];
            half_angle_derivatives(al * al, C, S);
            W.S0 = (float)S[0];
            double fact = 1.0;
            for (int n = 0; n < MIX_TAYLOR; ++n) {
                fact *= (n + 1);
                W.dC[n] = (float)(C[n + 1] / fact);
                W.dS[n] = (float)(S[n + 1] / fact);
            }
            // e_y = ch (alpha dS + S b_y) - sh dC with du = 2 alpha b_y + |b|^2:
            // its first-order coefficient Ky = ch S0 + 2 alpha Kq, where
            // Kq = ch alpha S'(u0) - sh C'(u0) also multiplies |b|^2
            const double ch = std::cos(0.5 * al), sh = std::sin(0.5 * al);
            const double kq = ch * al * S[1] - sh * C[1];
            W.Ky = split(ch * S[0] + 2.0 * al * kq);
            W.Kq = (float)kq;
            // short series: with |du| <= du3 the first neglected term (n = 3) is below
            // 2^-27 of the leading one for both functions, and the later terms fall
            // off faster (|dX[n+1] / dX[n]| du <= 1/4 there)
            double du3 = 1e30;
            for (const double* X : {C, S}) {
                const double c0 = std::fabs(X[1]), c3 = std::fabs(X[4] / 24.0);
                if (c3 > 0.0) du3 = std::min(du3, std::cbrt(std::ldexp(c0, -27) / c3));
                for (int n = 3; n < MIX_TAYLOR - 1; ++n) {   // ratio test of the later terms
                    const double a = std::fabs(X[n + 1]) / std::tgamma(n + 2.0);
                    const double b = std::fabs(X[n + 2]) / std::tgamma(n + 3.0);
                    if (b > 0.0) du3 = std::min(du3, 0.25 * a / b);
                }
            }
            W.du3 = (float)du3;
        }
        for (int c = 0; c < 4; ++c) m.rq[c] = split(rq[c]);
        me[u] = m;
    }
    // blob: [MixElem table] [uint16 sequence, padded to 16 B] [float2 rho table]
    const size_t elem_bytes = (size_t)nu * sizeof(MixElem);
    const size_t seq_bytes = (((size_t)ne * sizeof(uint16_t)) + 15) & ~(size_t)15;
    const size_t rho_bytes = ((rho.size() * sizeof(float)) + 15) & ~(size_t)15;
    L.mix_seq_offset = elem_bytes;
    L.mix_rho_offset = elem_bytes + seq_bytes;
    L.mix_bytes = elem_bytes + seq_bytes + rho_bytes;
    std::vector<unsigned char> blob(L.mix_bytes, 0);
    memcpy(blob.data(), me.data(), elem_bytes);
    memcpy(blob.data() + L.mix_seq_offset, L.h_seq, (size_t)ne * sizeof(uint16_t));
    if (!rho.empty()) memcpy(blob.data() + L.mix_rho_offset, rho.data(), rho.size() * sizeof(float));
    cudaError_t e = cudaMalloc(&L.d_mix, L.mix_bytes);
    if (e != cudaSuccess) return cuda_fail(e, "mixed tables: cudaMalloc");
    e = cudaMemcpy(L.d_mix, blob.data(), L.mix_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(L.d_mix);
        L.d_mix = nullptr;
        return cuda_fail(e, "mixed tables: cudaMemcpy");
    }
    return ST_OK;
}

}  // namespace st
