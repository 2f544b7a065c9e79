// Pointwise reverse-mode pieces shared by the DG and FD adjoint kernels (flat
// metric), each with its branch frozen as the forward pass took it.
#pragma once
#include "ffe_internal.h"
#include "physics.cuh"

namespace ffe {

constexpr int NQ_ADJ = 12;   // U and J~

// Ub += (dJ_drift/dU)^T wd + (dJ_eta/dU)^T wp  (flat metric)
__device__ __forceinline__ void current_vjp(const double* U, double eta, const double* wd, const double* wp, double* Ub) {
    const double* E = U;
    const double* B = U + 3;
    const double B2 = dot3(B, B);
    if (B2 == 0.0) return;
    const double ib2 = 1.0 / B2, q = U[8];
    const double c[3] = {E[1] * B[2] - E[2] * B[1], E[2] * B[0] - E[0] * B[2], E[0] * B[1] - E[1] * B[0]};
    // drift: J_d = q c / B^2
    const double s = dot3(wd, c);
    const double fq = q * ib2;
    Ub[8] += s * ib2;
    Ub[0] += fq * (B[1] * wd[2] - B[2] * wd[1]);
    Ub[1] += fq * (B[2] * wd[0] - B[0] * wd[2]);
    Ub[2] += fq * (B[0] * wd[1] - B[1] * wd[0]);
    Ub[3] += fq * (wd[1] * E[2] - wd[2] * E[1]) - 2.0 * fq * s * ib2 * B[0];
    Ub[4] += fq * (wd[2] * E[0] - wd[0] * E[2]) - 2.0 * fq * s * ib2 * B[1];
    Ub[5] += fq * (wd[0] * E[1] - wd[1] * E[0]) - 2.0 * fq * s * ib2 * B[2];
    if (eta == 0.0) return;
    // eta part: J_p = eta (f B + g E), f = E.B/B^2, g = max(E^2 - B^2, 0)/B^2
    const double EB = dot3(E, B), E2 = dot3(E, E);
    const bool act = E2 - B2 > 0.0;
    const double f = EB * ib2, g = act ? (E2 - B2) * ib2 : 0.0;
    const double wB = dot3(wp, B), wE = dot3(wp, E);
    for (int a = 0; a < 3; ++a) {
        Ub[a] += eta * (wB * B[a] * ib2 + (act ? 2.0 * wE * E[a] * ib2 : 0.0) + g * wp[a]);
        Ub[3 + a] += eta * (wB * (E[a] * ib2 - 2.0 * EB * B[a] * ib2 * ib2) + f * wp[a] +
                            (act ? -2.0 * wE * E2 * B[a] * ib2 * ib2 : 0.0));
    }
}

// Ub += sum_j (dF^j/dU)^T w[j]  with F^j the flat flux of direction j (J~ in the q~ row)
__device__ __forceinline__ void flux_t(const double* U, double eta, const double w[3][NV], double* Ub) {
    double wj[3];
    for (int j = 0; j < 3; ++j) {
        const double* x = w[j];
        // F^j(E^i) = d^ij psi - [ijk] B_k ; F^j(B^i) = d^ij phi + [ijk] E_k
        Ub[6] += x[j];
        Ub[7] += x[3 + j];
        for (int i = 0; i < 3; ++i) {
            if (i == j) continue;
            const int k = 3 - i - j;
            const double sg = ((j - i + 3) % 3 == 1) ? 1.0 : -1.0;
            Ub[3 + k] -= sg * x[i];
            Ub[k] += sg * x[3 + i];
        }
        Ub[j] += x[6];       // F^j(psi) = E^j
        Ub[3 + j] += x[7];   // F^j(phi) = B^j
        wj[j] = x[8];        // F^j(q) = J^j
    }
    current_vjp(U, eta, wj, wj, Ub);
}

// R-bar of the pointwise stiff solve U = S(R) given U-bar (the branch taken by the forward solve).
__device__ __forceinline__ void solve_vjp(const double* R, const Dev& d, double dta, const double* Ub, double* Rb) {
    for (int v = 0; v < NV; ++v) Rb[v] = Ub[v];
    Rb[6] = Ub[6] / fma(d.kpsi, dta, 1.0);
    Rb[7] = Ub[7] / fma(d.kphi, dta, 1.0);
    if (d.eta == 0.0) return;
    const double* E = R;
    const double* B = R + 3;
    const double B2 = dot3(B, B);
    if (B2 == 0.0) return;
    const double c = d.eta * dta, ib2 = 1.0 / B2;
    const double EB = dot3(E, B), f = EB * ib2, RR = dot3(E, E);
    const double* Eb = Ub;
    const double ebB = dot3(Eb, B);
    double pa[3], pe[3], e0[3];
    for (int i = 0; i < 3; ++i) {
        pa[i] = f * B[i];
        pe[i] = E[i] - pa[i];
        e0[i] = fma(pa[i], 1.0 / (1.0 + c), pe[i]);
    }
    double u, v;
    bool nonlin = dot3(e0, e0) > B2;
    double s = 0.0;
    if (nonlin) {
        bool ok;
        s = stiff_root(c, dot3(pe, pe), dot3(pa, pa), B2, ib2, ok);
    }
    u = 1.0 / (1.0 + s);
    v = 1.0 / (1.0 + c + s);
    // E_out = u E + (v - u) f B
    const double k1 = v - u;
    for (int a = 0; a < 3; ++a) {
        Rb[a] = u * Eb[a] + k1 * ebB * B[a] * ib2;
        Rb[3 + a] += k1 * (f * Eb[a] + ebB * (E[a] * ib2 - 2.0 * EB * B[a] * ib2 * ib2));
    }
    if (!nonlin) return;
    // s(R): g(s; E, B) = c (u^2 |E|^2 + (v^2 - u^2) (E.B)^2/B^2 - B^2)/B^2 - s = 0
    const double u2 = u * u, v2 = v * v;
    const double par2 = EB * EB * ib2, perp2 = RR - par2;
    const double gs = -2.0 * c * ib2 * (u2 * u * perp2 + v2 * v * par2) - 1.0;
    double dEds[3];
    for (int a = 0; a < 3; ++a) dEds[a] = -u2 * pe[a] - v2 * pa[a];
    const double es = dot3(Eb, dEds);
    const double coef = -es / gs;
    const double inner = u2 * RR + (v2 - u2) * EB * EB * ib2 - B2;
    for (int a = 0; a < 3; ++a) {
        const double dgE = c * ib2 * (2.0 * u2 * E[a] + 2.0 * (v2 - u2) * EB * ib2 * B[a]);
        const double dgB = c * ((2.0 * (v2 - u2) * EB * ib2 * E[a] - 2.0 * (v2 - u2) * EB * EB * ib2 * ib2 * B[a] -
                                 2.0 * B[a]) * ib2 - 2.0 * ib2 * ib2 * B[a] * inner);
        Rb[a] += coef * dgE;
        Rb[3 + a] += coef * dgB;
    }
}

// Reverse mode of the algebraic clamp Y = hard_clamp(X) (Sec. II.B, HARD
// modes): E1 = E - (E.B/B^2) B, then E1 |B|/|E1| where |E1| > |B|; B, psi,
// phi, q pass through.  Ub holds Y-bar on entry and X-bar on return; the
// branch is the one the forward clamp took at X.
__device__ __forceinline__ void clamp_vjp(const double* X, double* Ub) {
    const double* E = X;
    const double* B = X + 3;
    const double B2 = dot3(B, B);
    if (B2 == 0.0) {   // the forward set E to zero
        Ub[0] = Ub[1] = Ub[2] = 0.0;
        return;
    }
    const double ib2 = 1.0 / B2;
    const double f = dot3(E, B) * ib2;
    double E1[3], e1b[3];
    for (int a = 0; a < 3; ++a) E1[a] = fma(-f, B[a], E[a]);
    const double E12 = dot3(E1, E1);
    const double eb[3] = {Ub[0], Ub[1], Ub[2]};
    if (E12 > B2) {
        // Y = s E1, s = |B|/|E1|: E1-bar = s (eb - (eb.E1) E1/|E1|^2), B-bar += (eb.E1) s B/B^2
        const double s = sqrt(B2 / E12), ebE1 = dot3(eb, E1);
        for (int a = 0; a < 3; ++a) {
            e1b[a] = s * (eb[a] - ebE1 / E12 * E1[a]);
            Ub[3 + a] += ebE1 * s * ib2 * B[a];
        }
    } else {
        for (int a = 0; a < 3; ++a) e1b[a] = eb[a];
    }
    // E1 = E - f B, f = E.B/B^2: E-bar = e1b - (e1b.B) B/B^2,
    // B-bar += -f e1b - (e1b.B)/B^2 (E - 2 f B)
    const double g = dot3(e1b, B) * ib2;
    for (int a = 0; a < 3; ++a) {
        Ub[a] = fma(-g, B[a], e1b[a]);
        Ub[3 + a] += -f * e1b[a] - g * fma(-2.0 * f, B[a], E[a]);
    }
}

// Ub += (dG/dU)^T Gb, G = (-J~_eta, -kpsi psi, -kphi phi)
__device__ __forceinline__ void G_vjp(const double* U, const Dev& d, const double* Gb, double* Ub) {
    const double zero[3] = {0.0, 0.0, 0.0};
    const double wp[3] = {-Gb[0], -Gb[1], -Gb[2]};
    current_vjp(U, d.eta, zero, wp, Ub);
    Ub[6] -= d.kpsi * Gb[3];
    Ub[7] -= d.kphi * Gb[4];
}

// ub[0..11] += (dF^d/dU)^T w for the flat flux of direction d with the current
// taken as three independent quantities (ub[9..11]), as in flux_dir_flat.
__device__ __forceinline__ void flux_dir_t(int d, const double* w, double* ub) {
    if (d == 0) {
        ub[6] += w[0]; ub[5] += w[1]; ub[4] -= w[2];
        ub[7] += w[3]; ub[2] -= w[4]; ub[1] += w[5];
    } else if (d == 1) {
        ub[5] -= w[0]; ub[6] += w[1]; ub[3] += w[2];
        ub[2] += w[3]; ub[7] += w[4]; ub[0] -= w[5];
    } else {
        ub[4] += w[0]; ub[3] -= w[1]; ub[6] += w[2];
        ub[1] -= w[3]; ub[0] += w[4]; ub[7] += w[5];
    }
    ub[d] += w[6];
    ub[3 + d] += w[7];
    ub[9 + d] += w[8];
}

// Exterior adjoint of the lifted Rusanov term C = sc (n.(F(Ue, Je) - F(Ui)) - (Ue - Ui))
// when the exterior current Je is given (not J~(Ue)): z = (dC/dUe)^T lam, zJ = (dC/dJe)^T lam.
__device__ __forceinline__ void lift_ext_tJ(const double* n, double sc, const double* lam, double* z, double* zJ) {
    double ub[NQ_ADJ];
    for (int i = 0; i < NQ_ADJ; ++i) ub[i] = 0.0;
    for (int j = 0; j < 3; ++j) {
        double w[NV];
        for (int v = 0; v < NV; ++v) w[v] = n[j] * lam[v];
        flux_dir_t(j, w, ub);
    }
    for (int v = 0; v < NV; ++v) z[v] = sc * (ub[v] - lam[v]);
    for (int k = 0; k < 3; ++k) zJ[k] = sc * ub[NV + k];
}

// Ui-bar from Uo-bar through the star state Uo = (-v x B, B, 0, 0, 0),
// v = Omega (-y, x, 0) at x; returns the Omega derivative Uo-bar . dUo/dOmega.
__device__ __forceinline__ double bc_star_vjp(const double* Ui, const double* x, double omega, const double* ob,
                                              double* ib) {
    const double vv[3] = {-omega * x[1], omega * x[0], 0.0};
    // Uo_E = B x v, so B-bar += v x Uo_E-bar
    ib[3] += vv[1] * ob[2] - vv[2] * ob[1];
    ib[4] += vv[2] * ob[0] - vv[0] * ob[2];
    ib[5] += vv[0] * ob[1] - vv[1] * ob[0];
    ib[3] += ob[3]; ib[4] += ob[4]; ib[5] += ob[5];
    const double dv[3] = {-x[1], x[0], 0.0};
    const double* B = Ui + 3;
    const double dE[3] = {B[1] * dv[2] - B[2] * dv[1], B[2] * dv[0] - B[0] * dv[2], B[0] * dv[1] - B[1] * dv[0]};
    return dot3(ob, dE);
}

// Ui-bar from Uo-bar through the no-incoming-Poynting state (unit normal n).
__device__ __forceinline__ void bc_no_incoming_vjp(const double* Ui, const double* n, const double* ob, double* ib) {
    const double S[3] = {Ui[1] * Ui[5] - Ui[2] * Ui[4], Ui[2] * Ui[3] - Ui[0] * Ui[5], Ui[0] * Ui[4] - Ui[1] * Ui[3]};
    const bool inward = dot3(S, n) < 0.0;
    if (!inward) { ib[0] += ob[0]; ib[1] += ob[1]; ib[2] += ob[2]; }
    ib[3] += ob[3]; ib[4] += ob[4]; ib[5] += ob[5];
    ib[8] += ob[8];
}

}  // namespace ffe
