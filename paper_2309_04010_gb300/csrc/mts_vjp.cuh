// mts_vjp.cuh -- hand-written reverse mode of the per-particle stress laws
// for the adjoint (FP64).  Given the adjoints of the outputs (P, and for J2
// the updated C-bar_p^-1 and alpha), one backward sweep through the law gives
// the adjoints of every input: F, the previous plastic state, the bulk and
// shear moduli and the hardening parameters.  The forward pass is recomputed
// with the same operations as stress_j2 / stress_svk (same branch, same
// Newton iterates); the return-mapping increment is differentiated through
// the converged consistency condition g(dgamma) = 0 (implicit function).
#pragma once

#include "mts_device.cuh"

namespace mts {

// Fb += (d cof(F) / dF)^T [Cb], cof(F)_ij = F[i+1][j+1] F[i+2][j+2] - F[i+1][j+2] F[i+2][j+1]
__device__ __forceinline__ void cof_vjp(const double (&F)[3][3], const double (&Cb)[3][3],
                                        double (&Fb)[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int a = (i + 1) % 3, b = (i + 2) % 3, c = (j + 1) % 3, d = (j + 2) % 3;
            const double w = Cb[i][j];
            Fb[a][c] += w * F[b][d];
            Fb[b][d] += w * F[a][c];
            Fb[a][d] -= w * F[b][c];
            Fb[b][c] -= w * F[a][d];
        }
}

struct LawBar {
    double K, mu, s0, sinf, delta, H;
};

// St Venant-Kirchhoff: P = F S, S = lambda tr(E) I + 2 mu E, E = (F^T F - I)/2
__device__ __forceinline__ void stress_svk_vjp(const double (&F)[3][3], double lambda, double mu,
                                               const double (&Pb)[3][3], double (&Fb)[3][3],
                                               LawBar &pb) {
    double E[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            E[i][j] = 0.5 * (F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j]) -
                      (i == j ? 0.5 : 0.0);
    const double tr = E[0][0] + E[1][1] + E[2][2];
    double S[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S[i][j] = 2.0 * mu * E[i][j] + (i == j ? lambda * tr : 0.0);
    // P = F S
    double Sb[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double a = 0.0, b = 0.0;
            for (int k = 0; k < 3; ++k) {
                a += Pb[i][k] * S[j][k];     // (Pb S^T)_ij
                b += F[k][i] * Pb[k][j];     // (F^T Pb)_ij
            }
            Fb[i][j] += a;
            Sb[i][j] = b;
        }
    const double trSb = Sb[0][0] + Sb[1][1] + Sb[2][2];
    double Eb[3][3], mub = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Eb[i][j] = 2.0 * mu * Sb[i][j] + (i == j ? lambda * trSb : 0.0);
            mub += 2.0 * Sb[i][j] * E[i][j];
        }
    const double lamb = tr * trSb;
    // E = (F^T F - I)/2: Fb += F (Eb + Eb^T)/2
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double a = 0.0;
            for (int k = 0; k < 3; ++k) a += F[i][k] * 0.5 * (Eb[k][j] + Eb[j][k]);
            Fb[i][j] += a;
        }
    // lambda = K - 2 mu / 3
    pb.K += lamb;
    pb.mu += mub - (2.0 / 3.0) * lamb;
}

// Alg. 1 (J2 return mapping with saturation hardening), reverse mode.  cp:
// C-bar_p^-1 as (xx,yy,zz,xy,yz,xz) and alpha before the step; cpb_out: the
// adjoint of the updated state; cpb_in: the adjoint of the previous state.
__device__ __forceinline__ void stress_j2_vjp(const double (&F)[3][3], const double (&cp)[7],
                                              double K, double mu, double s0, double sinf,
                                              double delta, double H, const double (&Pb)[3][3],
                                              const double (&cpb_out)[7], double (&Fbar)[3][3],
                                              double (&cpb_in)[7], LawBar &pb) {
    const double r23 = 0.816496580927726;  // sqrt(2/3)
    // ---- forward, keeping the intermediates
    const double J = m3_det(F);
    const double sc = rcbrt(J);
    double Fb[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Fb[i][j] = sc * F[i][j];
    const double Cp[3][3] = {{cp[0], cp[3], cp[5]}, {cp[3], cp[1], cp[4]}, {cp[5], cp[4], cp[2]}};
    double T[3][3], bpre[3][3];
    m3_mul(Fb, Cp, T);
    m3_mul_bt(T, Fb, bpre);
    const double trb = bpre[0][0] + bpre[1][1] + bpre[2][2];
    double s0m[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) s0m[i][j] = mu * bpre[i][j] - (i == j ? mu * trb / 3.0 : 0.0);
    double sn = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) sn += s0m[i][j] * s0m[i][j];
    sn = sqrt(sn);
    const double al = cp[6];
    const double kal = hard_k(al, s0, sinf, delta, H);
    const bool plastic = sn - r23 * kal > 0.0;
    double s[3][3], fac = 1.0, dg = 0.0, mubr = 0.0, Fi[3][3], be[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) s[i][j] = s0m[i][j];
    if (plastic) {
        mubr = mu * trb / 3.0;
        const double tol = NewtonTol<double>::value;
        for (int it = 0; it < 30; ++it) {
            const double g = sn - r23 * hard_k(al + r23 * dg, s0, sinf, delta, H) - 2.0 * mubr * dg;
            if (fabs(g) <= tol * r23 * kal) break;
            const double dgd = -(2.0 / 3.0) * hard_dk(al + r23 * dg, s0, sinf, delta, H) - 2.0 * mubr;
            dg -= g / dgd;
        }
        fac = 1.0 - 2.0 * mubr * dg / sn;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                s[i][j] = fac * s0m[i][j];
                be[i][j] = s[i][j] / mu + (i == j ? trb / 3.0 : 0.0);
            }
        double Ci[3][3];
        m3_cof(Fb, Ci);
        const double idet = 1.0 / m3_det(Fb);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Fi[i][j] = Ci[j][i] * idet;
    }
    const double pv = 0.5 * K * (J * J - 1.0);
    double tau[3][3], Cf[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) tau[i][j] = s[i][j] + (i == j ? pv : 0.0);
    m3_cof(F, Cf);
    const double iJ = 1.0 / J;

    // ---- reverse
    // P = tau cof(F) / J
    double taub[3][3], Cfb[3][3], iJb = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double a = 0.0, b = 0.0, c = 0.0;
            for (int k = 0; k < 3; ++k) {
                a += Pb[i][k] * Cf[j][k];     // (Pb Cf^T)_ij
                b += tau[k][i] * Pb[k][j];    // (tau^T Pb)_ij
                c += tau[i][k] * Cf[k][j];    // (tau Cf)_ij
            }
            taub[i][j] = a * iJ;
            Cfb[i][j] = b * iJ;
            iJb += Pb[i][j] * c;
        }
    double Jb = -iJb * iJ * iJ;
    cof_vjp(F, Cfb, Fbar);
    // tau = s + pv I, pv = K (J^2 - 1) / 2
    const double pvb = taub[0][0] + taub[1][1] + taub[2][2];
    pb.K += 0.5 * pvb * (J * J - 1.0);
    Jb += pvb * K * J;
    double sb[3][3], s0mb[3][3], Fbb[3][3], trbb = 0.0, snb = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            sb[i][j] = taub[i][j];
            Fbb[i][j] = 0.0;
        }
    if (plastic) {
        // C-bar_p^-1' = sym(Fi be Fi^T), alpha' = alpha + r23 dg
        double Cnb[3][3] = {{cpb_out[0], 0.5 * cpb_out[3], 0.5 * cpb_out[5]},
                            {0.5 * cpb_out[3], cpb_out[1], 0.5 * cpb_out[4]},
                            {0.5 * cpb_out[5], 0.5 * cpb_out[4], cpb_out[2]}};
        // Y = A B A^T: Ab = Yb A B^T + Yb^T A B, Bb = A^T Yb A
        double FiB[3][3], FiBt[3][3], Fib[3][3], beb[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double a = 0.0, b = 0.0;
                for (int k = 0; k < 3; ++k) {
                    a += Fi[i][k] * be[j][k];   // (Fi be^T)_ij
                    b += Fi[i][k] * be[k][j];   // (Fi be)_ij
                }
                FiBt[i][j] = a;
                FiB[i][j] = b;
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double a = 0.0, b = 0.0;
                for (int k = 0; k < 3; ++k) {
                    a += Cnb[i][k] * FiBt[k][j] + Cnb[k][i] * FiB[k][j];
                    double t = 0.0;
                    for (int l = 0; l < 3; ++l) t += Cnb[k][l] * Fi[l][j];
                    b += Fi[k][i] * t;             // (Fi^T Cnb Fi)_ij
                }
                Fib[i][j] = a;
                beb[i][j] = b;
            }
        // Fi = Fb^-1: Fbb -= Fi^T Fib Fi^T
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double a = 0.0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) a += Fi[k][i] * Fib[k][l] * Fi[j][l];
                Fbb[i][j] -= a;
            }
        // be = s / mu + trb/3 I
        double mub_be = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                sb[i][j] += beb[i][j] / mu;
                mub_be -= beb[i][j] * s[i][j] / (mu * mu);
            }
        pb.mu += mub_be;
        trbb += (beb[0][0] + beb[1][1] + beb[2][2]) / 3.0;
        double alb = cpb_out[6];
        double dgb = r23 * cpb_out[6];
        // s = fac s0m, fac = 1 - 2 mubr dg / sn
        double facb = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                facb += sb[i][j] * s0m[i][j];
                s0mb[i][j] = fac * sb[i][j];
            }
        double mubrb = -2.0 * dg / sn * facb;
        dgb += -2.0 * mubr / sn * facb;
        snb += 2.0 * mubr * dg / (sn * sn) * facb;
        // dg from g(dg) = sn - r23 k(alpha + r23 dg) - 2 mubr dg = 0
        const double ap = al + r23 * dg;
        const double kp = hard_dk(ap, s0, sinf, delta, H);
        const double gd = -(2.0 / 3.0) * kp - 2.0 * mubr;
        const double lam = -dgb / gd;
        snb += lam;
        alb += lam * (-r23 * kp);
        mubrb += lam * (-2.0 * dg);
        const double e = exp(-delta * ap);
        pb.s0 += lam * (-r23) * e;
        pb.sinf += lam * (-r23) * (1.0 - e);
        pb.delta += lam * (-r23) * (sinf - s0) * ap * e;
        pb.H += lam * (-r23) * ap;
        // mubr = mu trb / 3
        pb.mu += mubrb * trb / 3.0;
        trbb += mubrb * mu / 3.0;
        for (int k = 0; k < 6; ++k) cpb_in[k] = 0.0;
        cpb_in[6] = alb;
    } else {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) s0mb[i][j] = sb[i][j];
        for (int k = 0; k < 7; ++k) cpb_in[k] = cpb_out[k];
    }
    // sn = |s0m|
    if (sn > 0.0)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) s0mb[i][j] += snb * s0m[i][j] / sn;
    // s0m = mu (bpre - trb/3 I)
    double bpreb[3][3], trs = s0mb[0][0] + s0mb[1][1] + s0mb[2][2], mub0 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            bpreb[i][j] = mu * s0mb[i][j];
            mub0 += s0mb[i][j] * (bpre[i][j] - (i == j ? trb / 3.0 : 0.0));
        }
    pb.mu += mub0;
    trbb -= mu / 3.0 * trs;
    for (int i = 0; i < 3; ++i) bpreb[i][i] += trbb;
    // bpre = Fb Cp Fb^T: Fbb += (bpreb + bpreb^T) Fb Cp, Cpb = Fb^T bpreb Fb
    double Cpb[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double a = 0.0, b = 0.0;
            for (int k = 0; k < 3; ++k) {
                a += (bpreb[i][k] + bpreb[k][i]) * T[k][j];   // T = Fb Cp
                double t = 0.0;
                for (int l = 0; l < 3; ++l) t += bpreb[k][l] * Fb[l][j];
                b += Fb[k][i] * t;
            }
            Fbb[i][j] += a;
            Cpb[i][j] = b;
        }
    cpb_in[0] += Cpb[0][0];
    cpb_in[1] += Cpb[1][1];
    cpb_in[2] += Cpb[2][2];
    cpb_in[3] += Cpb[0][1] + Cpb[1][0];
    cpb_in[4] += Cpb[1][2] + Cpb[2][1];
    cpb_in[5] += Cpb[0][2] + Cpb[2][0];
    // Fb = sc F, sc = J^(-1/3)
    double scb = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Fbar[i][j] += sc * Fbb[i][j];
            scb += Fbb[i][j] * F[i][j];
        }
    Jb += scb * (-1.0 / 3.0) * sc / J;
    // J = det(F)
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Fbar[i][j] += Jb * Cf[i][j];
}

}  // namespace mts
