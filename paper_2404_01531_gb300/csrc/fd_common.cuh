// Helpers shared by the FD-subcell kernels and their reverse mode: scratch
// layouts (extended blocks, face fluxes), shell geometry of an element, face
// indexing, and the WENO5-Z interpolation (Sec. III.C.2).
#pragma once
#include "ffe_internal.h"
#include "fp64util.cuh"
#include "shellmap.cuh"

namespace ffe {

constexpr int NQ = 12;  // reconstructed quantities: 9 evolved + J~ (3)

__device__ __forceinline__ int64_t ext_size(const Dev& d) {
    const int64_t ne = d.nc + 2 * GH;
    return ne * ne * ne;
}
// ext layout: [NQ][chunk][ext_size] indexed by position in the chunk
__device__ __forceinline__ double* ext_at(const Dev& d, int q, int wl) {
    return d.ext + ((int64_t)q * d.chunk + wl) * ext_size(d);
}
__device__ __forceinline__ int64_t nface(const Dev& d) { return (int64_t)(d.nc + 1) * d.nc * d.nc; }
// flux layout: [3][NV][chunk][nface]; curved meshes keep every physical
// component j: [3 (k)][3 (j)][NV][chunk][nface]
__device__ __forceinline__ double* flux_at(const Dev& d, int k, int v, int wl) {
    return d.flux + (((int64_t)k * NV + v) * d.chunk + wl) * nface(d);
}
__device__ __forceinline__ double* flux_at_c(const Dev& d, int k, int j, int v, int wl) {
    return d.flux + ((((int64_t)k * 3 + j) * NV + v) * d.chunk + wl) * nface(d);
}
// shell map of element e (its instance's geometry and its index inside the instance)
__device__ __forceinline__ ShellGeo shell_for(const Dev& d, int e, int& el) {
    ShellGeo g;
    g.a = 0.0;   // FD subcells run on shells with x = r v only
    if (d.einst) {
        const InstInfo& in = d.inst[d.einst[e]];
        g.r_in = in.r_in;
        g.c = in.c;
        g.na = in.na;
        g.nr = in.nr;
        el = e - in.e0;
    } else {
        g.r_in = d.shell_rin;
        g.c = d.shell_c;
        g.na = d.shell_na;
        g.nr = d.shell_nr;
        el = e;
    }
    return g;
}

// FD-point geometry of a flat-shell element from the tabulated gnomonic
// coordinates and radii of its rows (Dev::stab): base indices of the element's
// angular and radial rows on the half-cell grid, its wedge axes and side.
struct ShellPts {
    const double *tx, *tw, *tr, *tir;
    int gx, gy, gr, pn;
    double s, na, nr, c;
};
__device__ __forceinline__ ShellPts shell_pts(const Dev& d, int e, int nc) {
    int el;
    const ShellGeo g = shell_for(d, e, el);
    int ia, ib, ir, w;
    shell_elem(g, el, ia, ib, ir, w);
    ShellPts p;
    const double* t = d.stab + (d.einst ? d.inst[d.einst[e]].tab : 0);
    const int nx = 2 * nc * g.na + 1, nrr = 2 * nc * g.nr + 1;
    p.tx = t;
    p.tw = t + nx;
    p.tr = t + 2 * nx;
    p.tir = t + 2 * nx + nrr;
    p.gx = 2 * nc * ia;
    p.gy = 2 * nc * ib;
    p.gr = 2 * nc * ir;
    p.pn = (w >> 1) == 0 ? 2 : ((w >> 1) == 1 ? 1 : 0);
    p.s = (w & 1) ? -1.0 : 1.0;
    p.na = g.na;
    p.nr = g.nr;
    p.c = g.c;
    return p;
}
// inverse Jacobian (and the point, if x) at the centre of cell cc
__device__ __forceinline__ void shell_cell(const ShellPts& p, const int* cc, double ij[3][3], double* x) {
    const int hx = p.gx + 2 * cc[0] + 1, hy = p.gy + 2 * cc[1] + 1, hr = p.gr + 2 * cc[2] + 1;
    shell_cell_closed(p.tx[hx], p.tx[hy], p.tw[hx], p.tw[hy], p.tr[hr], p.tir[hr], p.pn, p.s, p.na, p.nr, p.c, ij, x);
}
// unit normal grad xi^k / |grad xi^k| at face m of direction k, tangential cells (ta, tb)
__device__ __forceinline__ void shell_face_normal(const ShellPts& p, int k, int m, int ta, int tb, double* nh) {
    double X, Y;
    if (k == 0) { X = p.tx[p.gx + 2 * m]; Y = 0.0; }
    else if (k == 1) { X = 0.0; Y = p.tx[p.gy + 2 * m]; }
    else { X = p.tx[p.gx + 2 * ta + 1]; Y = p.tx[p.gy + 2 * tb + 1]; }
    shell_normal_closed(k, X, Y, p.pn, p.s, nh);
}

__device__ __forceinline__ void axes_of(int dd, int& t1, int& t2) {
    t1 = dd == 0 ? 1 : 0;
    t2 = dd == 2 ? 1 : 2;
}

// number of listed elements in this chunk
__device__ __forceinline__ int chunk_n(const Dev& d, int ci, int w0) {
    const int n = d.counts[ci] - w0;
    return n < 0 ? 0 : (n > d.chunk ? d.chunk : n);
}

// WENO5-Z at the face right of v2 from v0..v4 (point-value interpolation
// candidates, ideal weights (1, 10, 5)/16, Jiang-Shu indicators, Z weights q = 2).
// The Z weights alpha_k = d_k (1 + tau^2/b_k^2), b_k = beta_k + eps, are scaled
// by b_0^2 b_1^2 b_2^2 so that the normalised combination needs one division:
//   A_k = d_k (b_k^2 + tau^2) prod_{j != k} b_j^2,  value = sum A_k p_k / sum A_k.
// With eps >= 1e-40 every A_k stays above 1e-240, inside the normal range.
// At the other end the products of six indicators overflow once an indicator
// exceeds about 1e51 (stencil differences of about 1e25): the weights then
// become Inf/NaN and the status word reports it.  Field values that large are
// far outside any state of this system (the fields are of order one).
// weno5z_combine: the Z-weighted combination of three candidates from their
// indicators b_k (eps included); the ideal weights are taken as (1, 10, 5)
// (scale-free).
__device__ __forceinline__ double weno5z_combine(double b0, double b1, double b2, double p0, double p1, double p2) {
    // A_k = d_k (b_k^2 + t^2) P_k with P_k the product of the other two b_j^2
    // is d_k (X + t^2 P_k), X = b_0^2 b_1^2 b_2^2 shared by the three
    const double t = b0 - b2;
    const double t2 = t * t;
    const double q0 = b0 * b0, q1 = b1 * b1, q2 = b2 * b2;
    const double P0 = q1 * q2, P1 = q0 * q2, P2 = q0 * q1;
    const double X = q0 * P0;
    const double A0 = fma(t2, P0, X), A1 = 10.0 * fma(t2, P1, X), A2 = 5.0 * fma(t2, P2, X);
    return fma(A0, p0, fma(A1, p1, A2 * p2)) * recip_nr(A0 + A1 + A2);
}

// Both values at the face between v2 and v3 from the six cells v0..v5: uL the
// WENO5-Z value from v0..v4, uR the one from v5..v1 (mirrored).  Everything is
// built from the first differences d_i = v_{i+1} - v_i: the candidates (the
// quadratics through v0..v2, v1..v3, v2..v4 and v3..v5 at the face), the
// second differences a and the one-sided combinations e of the Jiang-Shu
// indicators beta = (13/12) a^2 + (1/4) e^2, of which 4 (beta + eps) enter
// the weights (they are invariant under a common scale of the indicators).
// The two values share two candidates and two second differences.
__device__ __forceinline__ void weno5z_pair(double v0, double v1, double v2, double v3, double v4, double v5,
                                            double eps, double& uL, double& uR) {
    const double d01 = v1 - v0, d12 = v2 - v1, d23 = v3 - v2, d34 = v4 - v3, d45 = v5 - v4;
    const double p123 = fma(0.125, d12, fma(0.375, d23, v2));
    const double p234 = fma(0.625, d23, fma(-0.125, d34, v2));
    const double pL0 = fma(-0.375, d01, fma(0.875, d12, v2));
    const double pR0 = fma(-0.875, d34, fma(0.375, d45, v3));
    const double a012 = d12 - d01, a123 = d23 - d12, a234 = d34 - d23, a345 = d45 - d34;
    const double eL0 = fma(2.0, d12, a012), eL1 = d12 + d23, eL2 = fma(-2.0, d23, a234);
    const double eR0 = fma(-2.0, d34, a345), eR1 = d23 + d34, eR2 = fma(2.0, d23, a123);
    const double c = 13.0 / 3.0, eps4 = 4.0 * eps;
    const double c123 = c * a123, c234 = c * a234;
    const double bL0 = fma(c * a012, a012, fma(eL0, eL0, eps4));
    const double bL1 = fma(c123, a123, fma(eL1, eL1, eps4));
    const double bL2 = fma(c234, a234, fma(eL2, eL2, eps4));
    const double bR0 = fma(c * a345, a345, fma(eR0, eR0, eps4));
    const double bR1 = fma(c234, a234, fma(eR1, eR1, eps4));
    const double bR2 = fma(c123, a123, fma(eR2, eR2, eps4));
    uL = weno5z_combine(bL0, bL1, bL2, pL0, p123, p234);
    uR = weno5z_combine(bR0, bR1, bR2, pR0, p234, p123);
}

// MP5 value at the right face of v2 from v0..v4 (point values): Suresh &
// Huynh's monotonicity-preserving limiter (J. Comput. Phys. 136, 83 (1997))
// on the 5-point interpolant (3 v0 - 20 v1 + 90 v2 + 60 v3 - 5 v4)/128, alpha = 4:
// the interpolant when it lies between v2 and v_MP = v2 + minmod(v3 - v2,
// alpha (v2 - v1)), else its median with the bounds built from v_UL, v_MD,
// v_LC and the minmod4 curvatures of the second differences.
__device__ __forceinline__ double minmod2(double a, double b) {
    return a * b > 0.0 ? (fabs(a) < fabs(b) ? a : b) : 0.0;
}

__device__ __forceinline__ double minmod4(double a, double b, double c, double d) {
    if (a > 0.0 && b > 0.0 && c > 0.0 && d > 0.0) return fmin(fmin(a, b), fmin(c, d));
    if (a < 0.0 && b < 0.0 && c < 0.0 && d < 0.0) return fmax(fmax(a, b), fmax(c, d));
    return 0.0;
}

__device__ __forceinline__ double mp5(double v0, double v1, double v2, double v3, double v4) {
    const double vL = fma(0.0234375, v0, fma(-0.15625, v1, fma(0.703125, v2, fma(0.46875, v3, -0.0390625 * v4))));
    const double vMP = v2 + minmod2(v3 - v2, 4.0 * (v2 - v1));
    if ((vL - v2) * (vL - vMP) <= 0.0) return vL;
    const double d1 = v0 - 2.0 * v1 + v2, d2 = v1 - 2.0 * v2 + v3, d3 = v2 - 2.0 * v3 + v4;
    const double dp = minmod4(4.0 * d2 - d3, 4.0 * d3 - d2, d2, d3);
    const double dm = minmod4(4.0 * d2 - d1, 4.0 * d1 - d2, d2, d1);
    const double vUL = v2 + 4.0 * (v2 - v1);
    const double vMD = 0.5 * (v2 + v3) - 0.5 * dp;
    const double vLC = v2 + 0.5 * (v2 - v1) + (4.0 / 3.0) * dm;
    const double vmin = fmax(fmin(fmin(v2, v3), vMD), fmin(fmin(v2, vUL), vLC));
    const double vmax = fmin(fmax(fmax(v2, v3), vMD), fmax(fmax(v2, vUL), vLC));
    return vL + minmod2(vmin - vL, vmax - vL);
}

// Reverse mode of weno5z_combine for indicators B_k (eps included) and
// candidates p_k: from the value's adjoint yb, the candidates' adjoints pb_k
// and the indicators' adjoints Bb_k.  With A_k = d_k s_k P_k, s_k = b_k^2 +
// t^2, t = b_0 - b_2, P_k the product of the other two b_j^2, d = (1, 10, 5)
// and W_k = d_k dL/dA_k = d_k yb (p_k - value) / sum A:
//   dL/db_0 = 2 (t T + b_0 (W_0 P_0 + W_1 s_1 b_2^2 + W_2 s_2 b_1^2)),
//   dL/db_1 = 2 b_1 (W_0 s_0 b_2^2 + W_1 P_1 + W_2 s_2 b_0^2),
//   dL/db_2 = 2 (-t T + b_2 (W_0 s_0 b_1^2 + W_1 s_1 b_0^2 + W_2 P_2)),
// T = sum_k W_k P_k.  The weights are homogeneous of degree 0 in the b_k, so
// the B_k are first scaled exactly by the power of two of their maximum; the
// A_k are then O(1) and their derivatives stay in range.
__device__ __forceinline__ void weno5z_combine_vjp(double B0, double B1, double B2, double p0, double p1, double p2,
                                                   double yb, double& pb0, double& pb1, double& pb2, double& Bb0,
                                                   double& Bb1, double& Bb2) {
    const double sc = pow2_inv_scale(fmax(B0, fmax(B1, B2)));
    const double b0 = B0 * sc, b1 = B1 * sc, b2 = B2 * sc;
    const double t = b0 - b2, t2 = t * t;
    const double q0 = b0 * b0, q1 = b1 * b1, q2 = b2 * b2;
    const double s0 = q0 + t2, s1 = q1 + t2, s2 = q2 + t2;
    const double P0 = q1 * q2, P1 = q0 * q2, P2 = q0 * q1;
    const double A0 = s0 * P0, A1 = 10.0 * (s1 * P1), A2 = 5.0 * (s2 * P2);
    const double iS = recip_nr(A0 + A1 + A2);
    const double val = fma(A0, p0, fma(A1, p1, A2 * p2)) * iS;
    const double y = yb * iS;
    pb0 = y * A0;
    pb1 = y * A1;
    pb2 = y * A2;
    const double W0 = y * (p0 - val), W1 = (10.0 * y) * (p1 - val), W2 = (5.0 * y) * (p2 - val);
    const double W0P0 = W0 * P0, W0s0 = W0 * s0, W1s1 = W1 * s1, W2s2 = W2 * s2;
    const double T = fma(W1, P1, fma(W2, P2, W0P0));
    const double X0 = fma(W1s1, q2, fma(W2s2, q1, W0P0));
    const double X1 = fma(W0s0, q2, fma(W2s2, q0, W1 * P1));
    const double X2 = fma(W0s0, q1, fma(W1s1, q0, W2 * P2));
    const double sc2 = 2.0 * sc;
    Bb0 = sc2 * fma(t, T, b0 * X0);
    Bb1 = sc2 * (b1 * X1);
    Bb2 = sc2 * fma(-t, T, b2 * X2);
}

// Reverse mode of weno5z_pair: g[i] += ybL d uL/d v_i + ybR d uR/d v_i,
// i = 0..5, through the shared candidates and second differences (same
// first-difference form and 4x-scaled indicators as the forward pair).
__device__ __forceinline__ void weno5z_pair_vjp(double v0, double v1, double v2, double v3, double v4, double v5,
                                                double eps, double ybL, double ybR, double* g) {
    const double d01 = v1 - v0, d12 = v2 - v1, d23 = v3 - v2, d34 = v4 - v3, d45 = v5 - v4;
    const double p123 = fma(0.125, d12, fma(0.375, d23, v2));
    const double p234 = fma(0.625, d23, fma(-0.125, d34, v2));
    const double pL0 = fma(-0.375, d01, fma(0.875, d12, v2));
    const double pR0 = fma(-0.875, d34, fma(0.375, d45, v3));
    const double a012 = d12 - d01, a123 = d23 - d12, a234 = d34 - d23, a345 = d45 - d34;
    const double eL0 = fma(2.0, d12, a012), eL1 = d12 + d23, eL2 = fma(-2.0, d23, a234);
    const double eR0 = fma(-2.0, d34, a345), eR1 = d23 + d34, eR2 = fma(2.0, d23, a123);
    const double c = 13.0 / 3.0, eps4 = 4.0 * eps;
    const double k123 = (c * a123) * a123, k234 = (c * a234) * a234;
    const double BL0 = fma(c * a012, a012, fma(eL0, eL0, eps4));
    const double BL1 = k123 + fma(eL1, eL1, eps4);
    const double BL2 = k234 + fma(eL2, eL2, eps4);
    const double BR0 = fma(c * a345, a345, fma(eR0, eR0, eps4));
    const double BR1 = k234 + fma(eR1, eR1, eps4);
    const double BR2 = k123 + fma(eR2, eR2, eps4);
    double pbL0, pbL1, pbL2, BbL0, BbL1, BbL2, pbR0, pbR1, pbR2, BbR0, BbR1, BbR2;
    weno5z_combine_vjp(BL0, BL1, BL2, pL0, p123, p234, ybL, pbL0, pbL1, pbL2, BbL0, BbL1, BbL2);
    weno5z_combine_vjp(BR0, BR1, BR2, pR0, p234, p123, ybR, pbR0, pbR1, pbR2, BbR0, BbR1, BbR2);
    // adjoints of the shared and one-sided intermediates (B = c a^2 + e^2 + 4 eps)
    const double p123b = pbL1 + pbR2, p234b = pbL2 + pbR1;
    const double c2 = 2.0 * c;
    const double a012b = c2 * a012 * BbL0, a345b = c2 * a345 * BbR0;
    const double a123b = c2 * a123 * (BbL1 + BbR2), a234b = c2 * a234 * (BbL2 + BbR1);
    const double eL0b = 2.0 * eL0 * BbL0, eL1b = 2.0 * eL1 * BbL1, eL2b = 2.0 * eL2 * BbL2;
    const double eR0b = 2.0 * eR0 * BbR0, eR1b = 2.0 * eR1 * BbR1, eR2b = 2.0 * eR2 * BbR2;
    // to the cells: p123 = (-v1 + 6 v2 + 3 v3)/8, p234 = (3 v2 + 6 v3 - v4)/8,
    // pL0 = (3 v0 - 10 v1 + 15 v2)/8, pR0 = (15 v3 - 10 v4 + 3 v5)/8,
    // eL0 = v0 - 4 v1 + 3 v2, eL1 = v3 - v1, eL2 = 3 v2 - 4 v3 + v4,
    // eR0 = 3 v3 - 4 v4 + v5, eR1 = v4 - v2, eR2 = v1 - 4 v2 + 3 v3
    g[0] += fma(0.375, pbL0, a012b + eL0b);
    g[1] += fma(-1.25, pbL0, fma(-0.125, p123b, fma(-2.0, a012b, fma(-4.0, eL0b, a123b - eL1b + eR2b))));
    g[2] += fma(1.875, pbL0, fma(0.75, p123b, fma(0.375, p234b, fma(-2.0, a123b, fma(3.0, eL0b + eL2b,
               fma(-4.0, eR2b, a012b + a234b - eR1b))))));
    g[3] += fma(0.375, p123b, fma(0.75, p234b, fma(1.875, pbR0, fma(-2.0, a234b, fma(3.0, eR0b + eR2b,
               fma(-4.0, eL2b, a123b + a345b + eL1b))))));
    g[4] += fma(-0.125, p234b, fma(-1.25, pbR0, fma(-2.0, a345b, fma(-4.0, eR0b, a234b + eL2b + eR1b))));
    g[5] += fma(0.375, pbR0, a345b + eR0b);
}

// face fi of direction k: position m along k, tangential (ta, tb); false past the element's faces
__device__ __forceinline__ bool face_coords(int64_t fi, int nc, int& m, int& ta, int& tb) {
    const int64_t nf = (int64_t)(nc + 1) * nc * nc;
    if (fi >= nf) return false;
    m = (int)(fi % (nc + 1));
    ta = (int)((fi / (nc + 1)) % nc);
    tb = (int)(fi / ((int64_t)(nc + 1) * nc));
    return true;
}

}  // namespace ffe
