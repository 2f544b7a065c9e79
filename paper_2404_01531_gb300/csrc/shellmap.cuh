// Cubed-sphere wedge map and its Jacobian (host and device).
//
// Wedge w has normal axis n and sign s (w = 0..5: +z, -z, +y, -y, +x, -x) and
// tangential axes t1 = (n+1)%3, t2 = (n+2)%3.  Logical coordinates
// (ea, eb, er) in [-1,1]^3 map to
//   X = tan(pi ea / 4), Y = tan(pi eb / 4), rho = sqrt(1 + X^2 + Y^2),
//   v = (s e_n + X e_t1 + Y e_t2) / rho,  r = r_in exp(c (er + 1)), c = ln(r_out/r_in)/2,
//   x = r v                                           (Sec. IV.B: equiangular + logarithmic).
// Element (ia, ib, ir) of an na x na x nr split covers ea in [-1 + 2 ia/na, -1 + 2 (ia+1)/na]
// etc., so d ea / d xi^1 = 1/na, d eb / d xi^2 = 1/na, d er / d xi^3 = 1/nr.
// Jacobian columns (derived from the closed form):
//   dx/dea = r (pi/4)(1 + X^2) [e_t1/rho - X v/rho^2],
//   dx/deb = r (pi/4)(1 + Y^2) [e_t2/rho - Y v/rho^2],   (d rho/dX = X/rho)
//   dx/der = c r v.
// Spherical Kerr-Schild shell (a != 0, App. B): r is the Kerr-Schild radius and
// the Cartesian Kerr-Schild point is x = r v + a (z^ x v), i.e.
// x = (r cos ph - a sin ph) sin th, y = (r sin ph + a cos ph) sin th, z = r cos th
// for v = (sin th cos ph, sin th sin ph, cos th); the angular columns become
// r dv + a (z^ x dv), the radial column stays c r v.  Only shell_map carries
// this; the closed forms below are for a = 0.
#pragma once
#include <cmath>

namespace ffe {

struct ShellGeo {
    double r_in, c;     // r = r_in exp(c (er + 1))
    int na, nr;         // elements per wedge: angular, radial
    double a;           // spherical Kerr-Schild spin of the map (0: x = r v)
};

__host__ __device__ inline void shell_elem(const ShellGeo& g, int e, int& ia, int& ib, int& ir, int& w) {
    ia = e % g.na;
    ib = (e / g.na) % g.na;
    ir = (e / (g.na * g.na)) % g.nr;
    w = e / (g.na * g.na * g.nr);
}

// Point x and inverse Jacobian ijac[k][i] = d xi^k / d x^i at reference point xi of element e.
__host__ __device__ inline void shell_map(const ShellGeo& g, int e, const double xi[3], double x[3],
                                          double ijac[3][3]) {
    int ia, ib, ir, w;
    shell_elem(g, e, ia, ib, ir, w);
    const int n = (w >> 1) == 0 ? 2 : ((w >> 1) == 1 ? 1 : 0);
    const double s = (w & 1) ? -1.0 : 1.0;
    const int t1 = (n + 1) % 3, t2 = (n + 2) % 3;
    const double ea = -1.0 + (ia + 0.5 * (xi[0] + 1.0)) * 2.0 / g.na;
    const double eb = -1.0 + (ib + 0.5 * (xi[1] + 1.0)) * 2.0 / g.na;
    const double er = -1.0 + (ir + 0.5 * (xi[2] + 1.0)) * 2.0 / g.nr;
    const double q = 0.78539816339744830962;   // pi/4
    const double X = tan(q * ea), Y = tan(q * eb);
    const double rho = sqrt(1.0 + X * X + Y * Y);
    const double r = g.r_in * exp(g.c * (er + 1.0));
    double v[3];
    v[n] = s / rho;
    v[t1] = X / rho;
    v[t2] = Y / rho;
    for (int i = 0; i < 3; ++i) x[i] = r * v[i];
    double J[3][3];   // J[i][k] = d x^i / d xi^k
    const double fa = q * (1.0 + X * X) / g.na, fb = q * (1.0 + Y * Y) / g.na, fr = g.c * r / g.nr;
    double dva[3], dvb[3];   // d v / d xi^1, d v / d xi^2
    for (int i = 0; i < 3; ++i) {
        const double et1 = i == t1 ? 1.0 : 0.0, et2 = i == t2 ? 1.0 : 0.0;
        dva[i] = fa * (et1 / rho - X * v[i] / (rho * rho));
        dvb[i] = fb * (et2 / rho - Y * v[i] / (rho * rho));
        J[i][0] = r * dva[i];
        J[i][1] = r * dvb[i];
        J[i][2] = fr * v[i];
    }
    if (g.a != 0.0) {   // + a (z^ x .): (u_x, u_y) -> (-u_y, u_x)
        x[0] -= g.a * v[1];
        x[1] += g.a * v[0];
        J[0][0] -= g.a * dva[1];
        J[1][0] += g.a * dva[0];
        J[0][1] -= g.a * dvb[1];
        J[1][1] += g.a * dvb[0];
    }
    // inverse by cofactors
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    const double id = 1.0 / det;
    ijac[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * id;
    ijac[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    ijac[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    ijac[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * id;
    ijac[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    ijac[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    ijac[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * id;
    ijac[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    ijac[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
}

// Closed forms of the same map at FD points, from the gnomonic coordinates
// X = x_a/(s x_n), Y = x_b/(s x_n) and r (pn, pa, pb: the wedge's normal and
// tangential physical axes, s its side):
//   grad xi^0 = na rho / (q (1 + X^2) r) (e_a - s X e_n),
//   grad xi^1 = na rho / (q (1 + Y^2) r) (e_b - s Y e_n),
//   grad xi^2 = nr / (c r) x^,   x^ = (s e_n + X e_a + Y e_b) / rho,
// rho = sqrt(1 + X^2 + Y^2), q = pi/4.  wX = 1/(q (1 + X^2)), ir = 1/r.
__host__ __device__ inline void shell_cell_closed(double X, double Y, double wX, double wY, double r, double ir,
                                                  int pn, double s, double na, double nr, double c,
                                                  double ijac[3][3], double x[3]) {
    const int pa = (pn + 1) % 3, pb = (pn + 2) % 3;
    const double rho = sqrt(1.0 + X * X + Y * Y), irho = 1.0 / rho;
    const double fx = na * rho * ir * wX, fy = na * rho * ir * wY, fr = nr * ir / c;
    ijac[0][pa] = fx;
    ijac[0][pb] = 0.0;
    ijac[0][pn] = -s * X * fx;
    ijac[1][pa] = 0.0;
    ijac[1][pb] = fy;
    ijac[1][pn] = -s * Y * fy;
    ijac[2][pn] = fr * s * irho;
    ijac[2][pa] = fr * X * irho;
    ijac[2][pb] = fr * Y * irho;
    if (x) {
        x[pn] = r * s * irho;
        x[pa] = r * X * irho;
        x[pb] = r * Y * irho;
    }
}

// Unit normal grad xi^k / |grad xi^k| (k = 0, 1: T = X or Y on the face; k = 2:
// X, Y at the point).
__host__ __device__ inline void shell_normal_closed(int k, double X, double Y, int pn, double s, double nh[3]) {
    const int pa = (pn + 1) % 3, pb = (pn + 2) % 3;
    if (k == 2) {
        const double irho = 1.0 / sqrt(1.0 + X * X + Y * Y);
        nh[pn] = s * irho;
        nh[pa] = X * irho;
        nh[pb] = Y * irho;
    } else {
        const double T = k == 0 ? X : Y, it = 1.0 / sqrt(1.0 + T * T);
        nh[pn] = -s * T * it;
        nh[k == 0 ? pa : pb] = it;
        nh[k == 0 ? pb : pa] = 0.0;
    }
}

// Neighbour face index (a2, b2) for my face index (a, b) under orientation code
// o: bit 0 swaps a and b, bit 1 reverses the first, bit 2 the second.
__host__ __device__ inline void orient_map(int o, int n, int a, int b, int& a2, int& b2) {
    int x = (o & 1) ? b : a, y = (o & 1) ? a : b;
    a2 = (o & 2) ? n - 1 - x : x;
    b2 = (o & 4) ? n - 1 - y : y;
}

}  // namespace ffe
