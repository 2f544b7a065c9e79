// Host-side geometry and analytic data for curved meshes: the Kerr-Schild
// metric with its derivatives (complex-step differentiation of the closed
// form, App. B), Wald's field from its vector potential (Sec. IV.B.1, App. C),
// the regularised dipole (Sec. IV.C), and face matching with orientation codes.
#include <cmath>
#include <complex>
#include <map>
#include <tuple>
#include <vector>

#include "ffe_internal.h"
#include "geom_host.h"
#include "shellmap.cuh"

namespace ffe {

typedef std::complex<double> cd;
static const double CSH = 1e-30;

// g_{mu nu} = eta + 2 H l_mu l_nu (App. B), complex-capable.
static void ks4(const cd x[3], double M, double a, cd g[4][4]) {
    const cd R2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    const cd r2 = 0.5 * (R2 - a * a + std::sqrt((R2 - a * a) * (R2 - a * a) + 4.0 * a * a * x[2] * x[2]));
    const cd r = std::sqrt(r2);
    const cd H = M * r * r2 / (r2 * r2 + a * a * x[2] * x[2]);
    const cd l[4] = {cd(1.0), (r * x[0] + a * x[1]) / (r2 + a * a), (r * x[1] - a * x[0]) / (r2 + a * a), x[2] / r};
    for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n) g[m][n] = (m == n ? (m == 0 ? -1.0 : 1.0) : 0.0) + 2.0 * H * l[m] * l[n];
}

template <int N, typename T>
static bool inv(T A[N][N], T I[N][N]) {
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) I[i][j] = i == j ? T(1.0) : T(0.0);
    for (int c = 0; c < N; ++c) {
        int p = c;
        for (int r = c + 1; r < N; ++r)
            if (std::abs(A[r][c]) > std::abs(A[p][c])) p = r;
        for (int k = 0; k < N; ++k) { std::swap(A[c][k], A[p][k]); std::swap(I[c][k], I[p][k]); }
        T piv = A[c][c];
        if (std::abs(piv) == 0.0) return false;
        for (int k = 0; k < N; ++k) { A[c][k] /= piv; I[c][k] /= piv; }
        for (int r = 0; r < N; ++r) {
            if (r == c) continue;
            T f = A[r][c];
            for (int k = 0; k < N; ++k) { A[r][k] -= f * A[c][k]; I[r][k] -= f * I[c][k]; }
        }
    }
    return true;
}

// 3+1 split: gamma_ij = g_ij, beta_i = g_0i, beta^i = gamma^ij beta_j, alpha^2 = beta_i beta^i - g_00.
static void adm(const cd g[4][4], cd& alpha, cd beta[3], cd gl[3][3], cd gu[3][3]) {
    cd A[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { gl[i][j] = g[i + 1][j + 1]; A[i][j] = gl[i][j]; }
    inv<3, cd>(A, gu);
    cd bb = 0.0;
    for (int i = 0; i < 3; ++i) {
        beta[i] = 0.0;
        for (int j = 0; j < 3; ++j) beta[i] += gu[i][j] * g[0][j + 1];
        bb += beta[i] * g[0][i + 1];
    }
    alpha = std::sqrt(bb - g[0][0]);
}

static const int SYM[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};

// The 33 stored metric quantities at x (layout documented in ffe_internal.h).
void ks_point(const double x[3], double M, double a, double out[NMET]) {
    cd xc[3] = {x[0], x[1], x[2]}, g[4][4], al, be[3], gl[3][3], gu[3][3];
    ks4(xc, M, a, g);
    adm(g, al, be, gl, gu);
    double dal[3], dbe[3][3], dgl[3][3][3];   // d_k alpha, d_k beta^i, d_k gamma_ij
    for (int k = 0; k < 3; ++k) {
        cd xp[3] = {x[0], x[1], x[2]}, gp[4][4], ap, bp[3], glp[3][3], gup[3][3];
        xp[k] += cd(0.0, CSH);
        ks4(xp, M, a, gp);
        adm(gp, ap, bp, glp, gup);
        dal[k] = ap.imag() / CSH;
        for (int i = 0; i < 3; ++i) {
            dbe[k][i] = bp[i].imag() / CSH;
            for (int j = 0; j < 3; ++j) dgl[k][i][j] = glp[i][j].imag() / CSH;
        }
    }
    double Gl[3][3][3], Gam[3][3][3];   // Gamma_{l jk}, Gamma^i_jk
    for (int l = 0; l < 3; ++l)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) Gl[l][j][k] = 0.5 * (dgl[j][l][k] + dgl[k][l][j] - dgl[l][j][k]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                double s = 0.0;
                for (int l = 0; l < 3; ++l) s += gu[i][l].real() * Gl[l][j][k];
                Gam[i][j][k] = s;
            }
    double bl[3];
    for (int i = 0; i < 3; ++i) {
        bl[i] = 0.0;
        for (int j = 0; j < 3; ++j) bl[i] += gl[i][j].real() * be[j].real();
    }
    // D_i beta_j = d_i (gamma_jl beta^l) - Gamma^k_ij beta_k ; K = gamma^ij (D_i beta_j + D_j beta_i)/(2 alpha)
    double K = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double dij = 0.0, dji = 0.0;
            for (int l = 0; l < 3; ++l) {
                dij += dgl[i][j][l] * be[l].real() + gl[j][l].real() * dbe[i][l];
                dji += dgl[j][i][l] * be[l].real() + gl[i][l].real() * dbe[j][l];
            }
            for (int k = 0; k < 3; ++k) { dij -= Gam[k][i][j] * bl[k]; dji -= Gam[k][j][i] * bl[k]; }
            K += gu[i][j].real() * (dij + dji) / (2.0 * al.real());
        }
    out[M_ALPHA] = al.real();
    double det = 0.0;
    {
        double m[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) m[i][j] = gl[i][j].real();
        det = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
              m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
    }
    for (int i = 0; i < 3; ++i) out[M_BETA + i] = be[i].real();
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            out[M_GL + SYM[i][j]] = gl[i][j].real();
            out[M_GU + SYM[i][j]] = gu[i][j].real();
        }
    out[M_SQRTG] = std::sqrt(det);
    for (int k = 0; k < 3; ++k) out[M_DALPHA + k] = dal[k];
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) out[M_DBETA + 3 * j + i] = dbe[j][i];
    for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) s += gu[j][k].real() * Gam[i][j][k];
        out[M_GTRACE + i] = s;
    }
    out[M_K] = K;
}

// Wald: A_b = (B0/2)[(d_phi)_b + 2a (d_t)_b], d_t = (1,0,0,0), d_phi = (0,-y,x,0);
// E^i = -alpha F^{i0}, B~^i = [ijk] d_j A_k, E~ = sqrt(gamma) E.
static void wald_A(const cd x[3], double M, double a, double B0, cd A[4]) {
    cd g[4][4];
    ks4(x, M, a, g);
    for (int m = 0; m < 4; ++m) A[m] = 0.5 * B0 * (g[m][1] * (-x[1]) + g[m][2] * x[0] + 2.0 * a * g[m][0]);
}

void wald_point(const double x[3], double M, double a, double B0, double U[NV]) {
    double dA[3][4];
    for (int j = 0; j < 3; ++j) {
        cd xp[3] = {x[0], x[1], x[2]}, A[4];
        xp[j] += cd(0.0, CSH);
        wald_A(xp, M, a, B0, A);
        for (int m = 0; m < 4; ++m) dA[j][m] = A[m].imag() / CSH;
    }
    double F[4][4] = {};
    for (int j = 0; j < 3; ++j) {
        F[0][j + 1] = -dA[j][0];
        F[j + 1][0] = dA[j][0];
        for (int k = 0; k < 3; ++k) F[j + 1][k + 1] = dA[j][k + 1] - dA[k][j + 1];
    }
    cd xc[3] = {x[0], x[1], x[2]}, g[4][4], al, be[3], gl[3][3], gu[3][3];
    ks4(xc, M, a, g);
    adm(g, al, be, gl, gu);
    double G[4][4], Gi[4][4];
    for (int m = 0; m < 4; ++m)
        for (int n = 0; n < 4; ++n) G[m][n] = g[m][n].real();
    inv<4, double>(G, Gi);
    double m3[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) m3[i][j] = gl[i][j].real();
    const double sg = std::sqrt(m3[0][0] * (m3[1][1] * m3[2][2] - m3[1][2] * m3[2][1]) -
                                m3[0][1] * (m3[1][0] * m3[2][2] - m3[1][2] * m3[2][0]) +
                                m3[0][2] * (m3[1][0] * m3[2][1] - m3[1][1] * m3[2][0]));
    for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int m = 0; m < 4; ++m)
            for (int n = 0; n < 4; ++n) s += Gi[i + 1][m] * Gi[0][n] * F[m][n];
        U[i] = -al.real() * sg * s;
    }
    U[3] = dA[1][3] - dA[2][2];
    U[4] = dA[2][1] - dA[0][3];
    U[5] = dA[0][2] - dA[1][1];
    U[6] = U[7] = U[8] = 0.0;
}

// Dipole: A = mu m x x / (r^2 + delta^2)^(3/2), m = (sin chi, 0, cos chi); B~ = curl A.
void dipole_point(const double x[3], double mu, double delta, double chi, double U[NV]) {
    const double m[3] = {std::sin(chi), 0.0, std::cos(chi)};
    double dA[3][3];
    for (int j = 0; j < 3; ++j) {
        cd p[3] = {x[0], x[1], x[2]};
        p[j] += cd(0.0, CSH);
        const cd f = mu / std::pow(p[0] * p[0] + p[1] * p[1] + p[2] * p[2] + delta * delta, 1.5);
        const cd A[3] = {(m[1] * p[2] - m[2] * p[1]) * f, (m[2] * p[0] - m[0] * p[2]) * f, (m[0] * p[1] - m[1] * p[0]) * f};
        for (int i = 0; i < 3; ++i) dA[j][i] = A[i].imag() / CSH;
    }
    for (int v = 0; v < NV; ++v) U[v] = 0.0;
    U[3] = dA[1][2] - dA[2][1];
    U[4] = dA[2][0] - dA[0][2];
    U[5] = dA[0][1] - dA[1][0];
}

// Face matching for a mesh given by its map: neighbours by face-centre
// coordinates, orientation by matching the LGL face nodes.
void match_faces(int E, const MapFn& map, const std::vector<double>& xnodes, int np1, double scale,
                 std::vector<int>& nbr, std::vector<int>& nbf, std::vector<int>& orient) {
    nbr.assign(6 * E, -1);
    nbf.assign(6 * E, -1);
    orient.assign(6 * E, 0);
    std::map<std::tuple<long long, long long, long long>, std::vector<std::pair<int, int>>> keys;
    for (int e = 0; e < E; ++e)
        for (int f = 0; f < 6; ++f) {
            double xi[3] = {0.0, 0.0, 0.0}, x[3], ij[3][3];
            xi[f >> 1] = (f & 1) ? 1.0 : -1.0;
            map(e, xi, x, ij);
            auto k = std::make_tuple(std::llround(x[0] / scale * 1e9), std::llround(x[1] / scale * 1e9),
                                     std::llround(x[2] / scale * 1e9));
            keys[k].push_back({e, f});
        }
    for (auto& kv : keys) {
        if (kv.second.size() != 2) continue;
        for (int s = 0; s < 2; ++s) {
            const int e = kv.second[s].first, f = kv.second[s].second;
            const int e2 = kv.second[1 - s].first, f2 = kv.second[1 - s].second;
            nbr[6 * e + f] = e2;
            nbf[6 * e + f] = f2;
            // orientation: my (a, b) along (t1, t2) vs the neighbour's along its own axes
            const int d = f >> 1, d2 = f2 >> 1;
            const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2, u1 = d2 == 0 ? 1 : 0, u2 = d2 == 2 ? 1 : 2;
            int found = -1;
            for (int o = 0; o < 8 && found < 0; ++o) {
                double worst = 0.0;
                for (int b = 0; b < np1; ++b)
                    for (int a = 0; a < np1; ++a) {
                        int a2, b2;
                        orient_map(o, np1, a, b, a2, b2);
                        double xi[3], xi2[3], x[3], y[3], ij[3][3];
                        xi[d] = (f & 1) ? 1.0 : -1.0;
                        xi[t1] = xnodes[a];
                        xi[t2] = xnodes[b];
                        xi2[d2] = (f2 & 1) ? 1.0 : -1.0;
                        xi2[u1] = xnodes[a2];
                        xi2[u2] = xnodes[b2];
                        map(e, xi, x, ij);
                        map(e2, xi2, y, ij);
                        for (int q = 0; q < 3; ++q) worst = std::fmax(worst, std::fabs(x[q] - y[q]));
                    }
                if (worst < 1e-9 * scale) found = o;
            }
            orient[6 * e + f] = found < 0 ? 0 : found;
            if (found < 0) nbr[6 * e + f] = -2;   // flagged as an error by the caller
        }
    }
}

void shell_ghost_ref(const ShellGeo& ge, int el, const ShellGeo& gn, int eln, int dd, int s, int g, int ta, int tb,
                     int nc, double xn[3]) {
    int ia, ib, ir, w, ja, jb, jr, wn;
    shell_elem(ge, el, ia, ib, ir, w);
    shell_elem(gn, eln, ja, jb, jr, wn);
    const double dxi = 2.0 / nc;
    const int t1 = dd == 0 ? 1 : 0, t2 = dd == 2 ? 1 : 2;
    double xi[3];
    xi[dd] = s ? 1.0 + (g + 0.5) * dxi : -1.0 - (g + 0.5) * dxi;
    xi[t1] = -1.0 + (ta + 0.5) * dxi;
    xi[t2] = -1.0 + (tb + 0.5) * dxi;
    const long double q = 0.785398163397448309615660845819875721L;   // pi/4
    const long double ea = -1.0L + (ia + 0.5L * (xi[0] + 1.0L)) * 2.0L / ge.na;
    const long double eb = -1.0L + (ib + 0.5L * (xi[1] + 1.0L)) * 2.0L / ge.na;
    const long double er = -1.0L + (ir + 0.5L * (xi[2] + 1.0L)) * 2.0L / ge.nr;
    // wedge axes: normal n = (2, 1, 0) for w >> 1 = (0, 1, 2), side s = +-1 by w & 1
    auto axis = [](int ww) { return (ww >> 1) == 0 ? 2 : ((ww >> 1) == 1 ? 1 : 0); };
    auto side = [](int ww) { return (ww & 1) ? -1.0L : 1.0L; };
    long double u[3];
    const int n1 = axis(w);
    u[n1] = side(w);
    u[(n1 + 1) % 3] = std::tan(q * ea);
    u[(n1 + 2) % 3] = std::tan(q * eb);
    const int n2 = axis(wn);
    const long double un = side(wn) * u[n2];
    const long double ean = std::atan(u[(n2 + 1) % 3] / un) / q;
    const long double ebn = std::atan(u[(n2 + 2) % 3] / un) / q;
    xn[0] = (double)(2.0L * ((ean + 1.0L) * 0.5L * gn.na - ja) - 1.0L);
    xn[1] = (double)(2.0L * ((ebn + 1.0L) * 0.5L * gn.na - jb) - 1.0L);
    xn[2] = (double)(2.0L * ((er + 1.0L) * 0.5L * gn.nr - jr) - 1.0L);
}

int fd6_stencil(int nc, double t, double* w) {
    const double dxi = 2.0 / nc;
    int st = (int)std::floor((t + 1.0) / dxi - 0.5) - 2;
    st = st < 0 ? 0 : (st > nc - 6 ? nc - 6 : st);
    double x[6];
    for (int j = 0; j < 6; ++j) x[j] = -1.0 + (st + j + 0.5) * dxi;
    lagrange_at(x, 6, t, w);
    return st;
}

void lagrange_at(const double* x, int n, double t, double* w) {
    for (int m = 0; m < n; ++m) {
        long double v = 1.0L;
        for (int k = 0; k < n; ++k)
            if (k != m) v *= ((long double)t - x[k]) / ((long double)x[m] - x[k]);
        w[m] = (double)v;
    }
}

}  // namespace ffe
