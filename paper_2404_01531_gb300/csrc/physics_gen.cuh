// Pointwise GRFFE physics for a general static 3+1 metric (Sec. II.A, II.B,
// III.B), densitised variables, with the spatial Levi-Civita tensor
// [ijk]/sqrt(gamma) (convention eps_abcd = sqrt(-g)[abcd], [0123] = +1):
//   F^j(E~^i) = -beta^j E~^i + alpha (gamma^ij psi~ - [ijk] B~_k / sqrt(gamma))
//   F^j(B~^i) = -beta^j B~^i + alpha (gamma^ij phi~ + [ijk] E~_k / sqrt(gamma))
//   F^j(psi~) = -beta^j psi~ + alpha E~^j,  F^j(phi~) = -beta^j phi~ + alpha B~^j,
//   F^j(q~)   = J~^j - beta^j q~,
//   J~_drift  = alpha q~ [ijk] E~_j B~_k / (sqrt(gamma) B~^2),
//   J~_eta    = alpha eta [(E~.B~)/B~^2 B~ + max(E~^2 - B~^2, 0)/B~^2 E~].
#pragma once
#include "ffe_internal.h"
#include "physics.cuh"

namespace ffe {

struct PM {
    double a, b[3], gl[6], gu[6], sg;
};

__device__ __forceinline__ int sym3(int i, int j) {
    return i == j ? (i == 0 ? 0 : (i == 1 ? 3 : 5)) : (i + j == 1 ? 1 : (i + j == 2 ? 2 : 4));
}

__device__ __forceinline__ void load_pm(const double* met, int64_t stride, int64_t p, PM& m) {
    m.a = met[M_ALPHA * stride + p];
    for (int i = 0; i < 3; ++i) m.b[i] = met[(M_BETA + i) * stride + p];
    for (int i = 0; i < 6; ++i) { m.gl[i] = met[(M_GL + i) * stride + p]; m.gu[i] = met[(M_GU + i) * stride + p]; }
    m.sg = met[M_SQRTG * stride + p];
}

__device__ __forceinline__ void lowr(const PM& m, const double* v, double* o) {
    o[0] = fma(m.gl[0], v[0], fma(m.gl[1], v[1], m.gl[2] * v[2]));
    o[1] = fma(m.gl[1], v[0], fma(m.gl[3], v[1], m.gl[4] * v[2]));
    o[2] = fma(m.gl[2], v[0], fma(m.gl[4], v[1], m.gl[5] * v[2]));
}

__device__ __forceinline__ double d3(const double* a, const double* b) { return fma(a[2], b[2], fma(a[1], b[1], a[0] * b[0])); }

__device__ __forceinline__ void current_gen(const double* U, const PM& m, double eta, double* jd, double* jf) {
    const double* E = U;
    const double* B = U + 3;
    double El[3], Bl[3];
    lowr(m, E, El);
    lowr(m, B, Bl);
    const double B2 = d3(Bl, B);
    if (B2 == 0.0) { for (int i = 0; i < 3; ++i) jd[i] = jf[i] = 0.0; return; }
    const double ib2 = 1.0 / B2, EB = d3(El, B), E2 = d3(El, E);
    const double c0 = El[1] * Bl[2] - El[2] * Bl[1], c1 = El[2] * Bl[0] - El[0] * Bl[2], c2 = El[0] * Bl[1] - El[1] * Bl[0];
    const double fd = m.a * U[8] * ib2 / m.sg;
    jd[0] = fd * c0; jd[1] = fd * c1; jd[2] = fd * c2;
    double rr = E2 - B2;
    rr = rr > 0.0 ? rr : 0.0;
    const double fb = m.a * eta * EB * ib2, fe = m.a * eta * rr * ib2;
    for (int i = 0; i < 3; ++i) jf[i] = jd[i] + fma(fb, B[i], fe * E[i]);
}

__device__ __forceinline__ void current_eta_gen(const double* U, const PM& m, double eta, double* jp) {
    const double* E = U;
    const double* B = U + 3;
    double El[3], Bl[3];
    lowr(m, E, El);
    lowr(m, B, Bl);
    const double B2 = d3(Bl, B);
    if (B2 == 0.0 || eta == 0.0) { jp[0] = jp[1] = jp[2] = 0.0; return; }
    const double ib2 = 1.0 / B2, EB = d3(El, B), E2 = d3(El, E);
    double rr = E2 - B2;
    rr = rr > 0.0 ? rr : 0.0;
    const double fb = m.a * eta * EB * ib2, fe = m.a * eta * rr * ib2;
    for (int i = 0; i < 3; ++i) jp[i] = fma(fb, B[i], fe * E[i]);
}

// F[j][v] for j = 0..2
__device__ __forceinline__ void flux_gen(const double* U, const double* J, const PM& m, double F[3][NV]) {
    double El[3], Bl[3];
    lowr(m, U, El);
    lowr(m, U + 3, Bl);
    const double ia = m.a / m.sg;
    for (int j = 0; j < 3; ++j) {
        for (int i = 0; i < 3; ++i) {
            double eB = 0.0, eE = 0.0;
            if (i != j) {
                const int k = 3 - i - j;
                const double sgn = ((j - i + 3) % 3 == 1) ? 1.0 : -1.0;   // [ijk]
                eB = sgn * Bl[k];
                eE = sgn * El[k];
            }
            F[j][i] = fma(-m.b[j], U[i], fma(m.a * m.gu[sym3(i, j)], U[6], -ia * eB));
            F[j][3 + i] = fma(-m.b[j], U[3 + i], fma(m.a * m.gu[sym3(i, j)], U[7], ia * eE));
        }
        F[j][6] = fma(-m.b[j], U[6], m.a * U[j]);
        F[j][7] = fma(-m.b[j], U[7], m.a * U[3 + j]);
        F[j][8] = fma(-m.b[j], U[8], J[j]);
    }
}

// explicit sources; md points to the node's metric derivatives (stride between quantities)
__device__ __forceinline__ void sources_gen(const double* U, const double* jd, const PM& m, const double* met,
                                            int64_t stride, int64_t p, double* S) {
    double da[3], gt[3];
    for (int k = 0; k < 3; ++k) { da[k] = met[(M_DALPHA + k) * stride + p]; gt[k] = met[(M_GTRACE + k) * stride + p]; }
    const double K = met[M_K * stride + p];
    for (int i = 0; i < 3; ++i) {
        double coef = -m.a * gt[i], sE = -jd[i], sB = 0.0;
        for (int j = 0; j < 3; ++j) {
            coef = fma(m.gu[sym3(i, j)], da[j], coef);
            const double dbji = met[(M_DBETA + 3 * j + i) * stride + p];
            sE = fma(-U[j], dbji, sE);
            sB = fma(-U[3 + j], dbji, sB);
        }
        S[i] = fma(U[6], coef, sE);
        S[3 + i] = fma(U[7], coef, sB);
    }
    S[6] = fma(m.a, U[8], -m.a * U[6] * K) + d3(U, da);
    S[7] = -m.a * U[7] * K + d3(U + 3, da);
    S[8] = 0.0;
}

__device__ __forceinline__ void implicit_G_gen(const double* U, const PM& m, const Dev& d, double* G) {
    double jp[3];
    current_eta_gen(U, m, d.eta, jp);
    G[0] = -jp[0]; G[1] = -jp[1]; G[2] = -jp[2];
    G[3] = -m.a * d.kpsi * U[6];
    G[4] = -m.a * d.kphi * U[7];
}

__device__ __forceinline__ void hard_clamp_gen(double* U, const PM& m) {
    double* E = U;
    const double* B = U + 3;
    double Bl[3], El[3];
    lowr(m, B, Bl);
    const double B2 = d3(Bl, B);
    if (B2 == 0.0) { E[0] = E[1] = E[2] = 0.0; return; }
    const double f = d3(Bl, E) / B2;
    for (int i = 0; i < 3; ++i) E[i] = fma(-f, B[i], E[i]);
    lowr(m, E, El);
    const double E2 = d3(El, E);
    if (E2 > B2) {
        const double s = sqrt(B2 / E2);
        for (int i = 0; i < 3; ++i) E[i] *= s;
    }
}

// U = R + dta G(U) with c = alpha eta dta (see stiff_solve_flat; gamma inner products).
__device__ __forceinline__ bool stiff_solve_gen(double* U, const PM& m, const Dev& d, double dta) {
    U[6] = U[6] / fma(m.a * d.kpsi, dta, 1.0);
    U[7] = U[7] / fma(m.a * d.kphi, dta, 1.0);
    if (d.eta == 0.0) return true;
    double* E = U;
    const double* B = U + 3;
    double Bl[3];
    lowr(m, B, Bl);
    const double B2 = d3(Bl, B);
    if (B2 == 0.0) return true;
    const double c = m.a * d.eta * dta, ib2 = 1.0 / B2;
    const double f = d3(Bl, E) * ib2;
    double pa[3] = {f * B[0], f * B[1], f * B[2]};
    double pe[3] = {E[0] - pa[0], E[1] - pa[1], E[2] - pa[2]};
    const double i1c = 1.0 / (1.0 + c);
    double e0[3] = {fma(pa[0], i1c, pe[0]), fma(pa[1], i1c, pe[1]), fma(pa[2], i1c, pe[2])}, l0[3];
    lowr(m, e0, l0);
    if (!(d3(l0, e0) > B2)) { E[0] = e0[0]; E[1] = e0[1]; E[2] = e0[2]; return true; }
    double lp[3], la[3];
    lowr(m, pe, lp);
    lowr(m, pa, la);
    bool ok;
    const double s = stiff_root(c, d3(lp, pe), d3(la, pa), B2, ib2, ok);
    const double u = 1.0 / (1.0 + s), v = 1.0 / (1.0 + c + s);
    for (int i = 0; i < 3; ++i) E[i] = fma(pe[i], u, pa[i] * v);
    return ok;
}

// No-incoming-Poynting outer state (Sec. III.D) with the metric: S.n with
// S_i proportional to [ijk] E_j B_k of the lowered fields and the outward
// unit normal nl (lower index); E~ -> 0 where S.n < 0, psi~ = phi~ = 0.
__device__ __forceinline__ void bc_no_incoming_gen(const double* Ui, const PM& m, const double* nl, double* Uo) {
    for (int v = 0; v < NV; ++v) Uo[v] = Ui[v];
    double El[3], Bl[3];
    lowr(m, Ui, El);
    lowr(m, Ui + 3, Bl);
    const double S[3] = {El[1] * Bl[2] - El[2] * Bl[1], El[2] * Bl[0] - El[0] * Bl[2], El[0] * Bl[1] - El[1] * Bl[0]};
    if (d3(S, nl) < 0.0) { Uo[0] = Uo[1] = Uo[2] = 0.0; }
    Uo[6] = 0.0;
    Uo[7] = 0.0;
}

__device__ __forceinline__ double bnorm_gen(const double* U, const PM& m) {
    double Bl[3];
    lowr(m, U + 3, Bl);
    return sqrt(d3(Bl, U + 3));
}

}  // namespace ffe
