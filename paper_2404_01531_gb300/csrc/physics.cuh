// Pointwise GRFFE physics on the device, flat metric (alpha = 1, beta = 0,
// gamma_ij = delta_ij).  Densitised variables U = (E~, B~, psi~, phi~, q~).
//   current:  J~_drift = q~ (E~ x B~)/B~^2,
//             J~_eta   = eta [ (E~.B~)/B~^2 B~ + max(E~^2 - B~^2, 0)/B~^2 E~ ]   (Sec. II.B)
//   fluxes:   F^j(E~^i) = delta^ij psi~ - [ijk] B~_k,  F^j(B~^i) = delta^ij phi~ + [ijk] E~_k,
//             F^j(psi~) = E~^j, F^j(phi~) = B~^j, F^j(q~) = J~^j                       (Sec. II.A)
//   sources:  S(E~) = -J~_drift, S(psi~) = q~ (explicit); the eta part of the
//             current and the cleaning damping are the implicit operator (Sec. III.B).
#pragma once
#include "ffe_internal.h"
#include "fp64util.cuh"

namespace ffe {

__device__ __forceinline__ double dot3(const double* a, const double* b) {
    return fma(a[2], b[2], fma(a[1], b[1], a[0] * b[0]));
}

// J~_drift (jd) and J~ = J~_drift + J~_eta (jf); zero where B~^2 = 0.
__device__ __forceinline__ void current_flat(const double* U, double eta, double* jd, double* jf) {
    const double* E = U;
    const double* B = U + 3;
    double B2 = dot3(B, B);
    if (B2 == 0.0) {
        jd[0] = jd[1] = jd[2] = 0.0;
        jf[0] = jf[1] = jf[2] = 0.0;
        return;
    }
    double ib2 = recip_any(B2);
    double EB = dot3(E, B), E2 = dot3(E, E);
    double cx = E[1] * B[2] - E[2] * B[1];
    double cy = E[2] * B[0] - E[0] * B[2];
    double cz = E[0] * B[1] - E[1] * B[0];
    double fd = U[8] * ib2;
    jd[0] = fd * cx; jd[1] = fd * cy; jd[2] = fd * cz;
    double rr = E2 - B2;
    rr = rr > 0.0 ? rr : 0.0;
    double fb = eta * EB * ib2, fe = eta * rr * ib2;
    jf[0] = jd[0] + fma(fb, B[0], fe * E[0]);
    jf[1] = jd[1] + fma(fb, B[1], fe * E[1]);
    jf[2] = jd[2] + fma(fb, B[2], fe * E[2]);
}

// eta part of the current only (for the implicit operator G).
__device__ __forceinline__ void current_eta_flat(const double* U, double eta, double* jp) {
    const double* E = U;
    const double* B = U + 3;
    double B2 = dot3(B, B);
    if (B2 == 0.0 || eta == 0.0) { jp[0] = jp[1] = jp[2] = 0.0; return; }
    double ib2 = recip_any(B2);
    double EB = dot3(E, B), E2 = dot3(E, E);
    double rr = E2 - B2;
    rr = rr > 0.0 ? rr : 0.0;
    double fb = eta * EB * ib2, fe = eta * rr * ib2;
    jp[0] = fma(fb, B[0], fe * E[0]);
    jp[1] = fma(fb, B[1], fe * E[1]);
    jp[2] = fma(fb, B[2], fe * E[2]);
}

// Flux along axis d (flat): out[v] = F^d(U)_v with J~ (full) for q~.
__device__ __forceinline__ void flux_dir_flat(const double* U, const double* J, int d, double* out) {
    // F^d(E~^i) = delta^{id} psi - [idk] B_k ;  F^d(B~^i) = delta^{id} phi + [idk] E_k
    const double* E = U;
    const double* B = U + 3;
    if (d == 0) {
        out[0] = U[6]; out[1] = B[2]; out[2] = -B[1];
        out[3] = U[7]; out[4] = -E[2]; out[5] = E[1];
    } else if (d == 1) {
        out[0] = -B[2]; out[1] = U[6]; out[2] = B[0];
        out[3] = E[2]; out[4] = U[7]; out[5] = -E[0];
    } else {
        out[0] = B[1]; out[1] = -B[0]; out[2] = U[6];
        out[3] = -E[1]; out[4] = E[0]; out[5] = U[7];
    }
    out[6] = E[d];
    out[7] = B[d];
    out[8] = J[d];
}

// Implicit operator G: (-J~_eta, -kpsi psi~, -kphi phi~).
__device__ __forceinline__ void implicit_G_flat(const double* U, const Dev& d, double* G) {
    double jp[3];
    current_eta_flat(U, d.eta, jp);
    G[0] = -jp[0]; G[1] = -jp[1]; G[2] = -jp[2];
    G[3] = -d.kpsi * U[6];
    G[4] = -d.kphi * U[7];
}

// Algebraic clamp: E <- E - (E.B/B^2) B; if E^2 > B^2, E <- E sqrt(B^2/E^2); E <- 0 if B = 0.
__device__ __forceinline__ void hard_clamp_flat(double* U) {
    double* E = U;
    const double* B = U + 3;
    double B2 = dot3(B, B);
    if (B2 == 0.0) { E[0] = E[1] = E[2] = 0.0; return; }
    double f = dot3(E, B) * recip_any(B2);
    E[0] = fma(-f, B[0], E[0]);
    E[1] = fma(-f, B[1], E[1]);
    E[2] = fma(-f, B[2], E[2]);
    double E2 = dot3(E, E);
    if (E2 > B2) {
        double s = sqrt(B2 * recip_any(E2));
        E[0] *= s; E[1] *= s; E[2] *= s;
    }
}

// Root s >= 0 of g(s) = c (p2/(1+s)^2 + a2/(1+c+s)^2 - B2)/B2 - s when g(0) > 0
// (p2, a2: squared norms of the parts of E* across and along B; ib2 = 1/B2).
// g is decreasing and convex, so Newton from any s0 with g(s0) >= 0 climbs
// monotonically to the root.  Start: with t = 1 + s and K = c p2/B2, every
// t with t^2 (t - 1 + c) <= K has g(t - 1) >= 0, and
// t_a = sqrt(K / (max(c - 1, 0) + K^(1/3))) is such a t (t_a <= K^(1/3)); it is
// within a few per cent of the root unless the along-B part dominates, so a
// handful of steps reach the rounding level of s.  ok = false if the last step
// was not at that level (iteration cap).
__device__ __forceinline__ double stiff_root(double c, double p2, double a2, double B2, double ib2, bool& ok) {
    const double K = c * p2 * ib2;
    double s = 0.0;
    if (K > 0.0) {
        const double ta = sqrt(K / ((c > 1.0 ? c - 1.0 : 0.0) + cbrt(K)));
        s = ta > 1.0 ? ta - 1.0 : 0.0;
    }
    double step = 1.0;
    for (int it = 0; it < 100; ++it) {
        const double a1 = 1.0 + s, b1 = 1.0 + c + s, w = 1.0 / (a1 * b1);
        const double u = b1 * w, v = a1 * w;
        const double pu = p2 * u * u, av = a2 * v * v;
        const double g = c * ((pu + av) - B2) * ib2 - s;
        const double dg = -2.0 * c * (pu * u + av * v) * ib2 - 1.0;
        const double sn = s - g / dg;
        step = sn - s;
        if (!(sn > s)) break;
        s = sn;
        if (step <= 4e-16 * s) break;
    }
    ok = step <= 1e-12 * (s > 1.0 ? s : 1.0);
    return s;
}

// Solve U = R + dta G(U) in place (Sec. III.B).  With c = eta dta and E* split
// along B into E*_par + E*_perp, E(s) = E*_perp/(1+s) + E*_par/(1+c+s); s = 0 when
// |E(0)|^2 <= B^2, otherwise the root of the decreasing convex function
// g(s) = c (|E(s)|^2 - B^2)/B^2 - s (stiff_root).  Returns false if Newton hit
// its iteration cap.
__device__ __forceinline__ bool stiff_solve_flat(double* U, const Dev& d, double dta) {
    U[6] *= recip_any(fma(d.kpsi, dta, 1.0));
    U[7] *= recip_any(fma(d.kphi, dta, 1.0));
    if (d.eta == 0.0) return true;
    double* E = U;
    const double* B = U + 3;
    double B2 = dot3(B, B);
    if (B2 == 0.0) return true;
    double c = d.eta * dta;
    double ib2 = recip_any(B2);
    double f = dot3(E, B) * ib2;
    double pa[3] = {f * B[0], f * B[1], f * B[2]};
    double pe[3] = {E[0] - pa[0], E[1] - pa[1], E[2] - pa[2]};
    double i1c = recip_any(1.0 + c);
    double e0[3] = {fma(pa[0], i1c, pe[0]), fma(pa[1], i1c, pe[1]), fma(pa[2], i1c, pe[2])};
    if (!(dot3(e0, e0) > B2)) {
        E[0] = e0[0]; E[1] = e0[1]; E[2] = e0[2];
        return true;
    }
    bool ok;
    const double s = stiff_root(c, dot3(pe, pe), dot3(pa, pa), B2, ib2, ok);
    double u = recip_any(1.0 + s), v = recip_any(1.0 + c + s);
    E[0] = fma(pe[0], u, pa[0] * v);
    E[1] = fma(pe[1], u, pa[1] * v);
    E[2] = fma(pe[2], u, pa[2] * v);
    return ok;
}

// No-incoming-Poynting outer state (Sec. III.D), outward unit normal n (flat).
__device__ __forceinline__ void bc_no_incoming_flat(const double* Ui, const double* n, double* Uo) {
    for (int v = 0; v < NV; ++v) Uo[v] = Ui[v];
    const double* E = Ui;
    const double* B = Ui + 3;
    double Sx = E[1] * B[2] - E[2] * B[1];
    double Sy = E[2] * B[0] - E[0] * B[2];
    double Sz = E[0] * B[1] - E[1] * B[0];
    double Sn = Sx * n[0] + Sy * n[1] + Sz * n[2];
    if (Sn < 0.0) { Uo[0] = Uo[1] = Uo[2] = 0.0; }
    Uo[6] = 0.0;
    Uo[7] = 0.0;
}

// Rotating perfect-conductor star state (Sec. IV.C): E = -v x B, v = Omega z x x,
// B from the interior, psi = q = 0 (as inside the paper's star) and phi = 0 (as
// in the paper's outer boundary states: the incoming divergence-cleaning wave
// of B then has data; taking phi from the interior lets it grow at the star).
__device__ __forceinline__ void bc_star_flat(const double* Ui, const double* x, double omega, double* Uo) {
    for (int v = 0; v < NV; ++v) Uo[v] = Ui[v];
    double vx = -omega * x[1], vy = omega * x[0];
    const double* B = Ui + 3;
    Uo[0] = -(vy * B[2]);
    Uo[1] = -(-vx * B[2]);
    Uo[2] = -(vx * B[1] - vy * B[0]);
    Uo[6] = 0.0;
    Uo[7] = 0.0;
    Uo[8] = 0.0;
}

}  // namespace ffe
