// Helpers shared by the FD-subcell kernels and their reverse mode: scratch
// layouts (extended blocks, face fluxes), shell geometry of an element, face
// indexing, and the WENO5-Z interpolation (Sec. III.C.2).
#pragma once
#include "ffe_internal.h"
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
__device__ __forceinline__ double weno5z(double v0, double v1, double v2, double v3, double v4, double eps) {
    const double p0 = fma(0.375, v0, fma(-1.25, v1, 1.875 * v2));
    const double p1 = fma(-0.125, v1, fma(0.75, v2, 0.375 * v3));
    const double p2 = fma(0.375, v2, fma(0.75, v3, -0.125 * v4));
    const double c13 = 13.0 / 12.0;
    const double s0a = v0 - 2.0 * v1 + v2, s0b = v0 - 4.0 * v1 + 3.0 * v2;
    const double s1a = v1 - 2.0 * v2 + v3, s1b = v1 - v3;
    const double s2a = v2 - 2.0 * v3 + v4, s2b = 3.0 * v2 - 4.0 * v3 + v4;
    const double b0 = fma(c13 * s0a, s0a, 0.25 * s0b * s0b) + eps;
    const double b1 = fma(c13 * s1a, s1a, 0.25 * s1b * s1b) + eps;
    const double b2 = fma(c13 * s2a, s2a, 0.25 * s2b * s2b) + eps;
    const double t = b0 - b2;
    const double t2 = t * t;
    const double q0 = b0 * b0, q1 = b1 * b1, q2 = b2 * b2;
    const double A0 = (0.0625 * (q0 + t2)) * (q1 * q2);
    const double A1 = (0.625 * (q1 + t2)) * (q0 * q2);
    const double A2 = (0.3125 * (q2 + t2)) * (q0 * q1);
    return fma(A0, p0, fma(A1, p1, A2 * p2)) / (A0 + A1 + A2);
}

// Z-weighted combination of three candidates from their indicators b_k (eps
// included); the ideal weights are taken as (1, 10, 5) (scale-free).
__device__ __forceinline__ double weno5z_combine(double b0, double b1, double b2, double p0, double p1, double p2) {
    const double t = b0 - b2;
    const double t2 = t * t;
    const double q0 = b0 * b0, q1 = b1 * b1, q2 = b2 * b2;
    const double A0 = (q0 + t2) * (q1 * q2);
    const double A1 = (10.0 * (q1 + t2)) * (q0 * q2);
    const double A2 = (5.0 * (q2 + t2)) * (q0 * q1);
    return fma(A0, p0, fma(A1, p1, A2 * p2)) / (A0 + A1 + A2);
}

// Both values at the face between v2 and v3 from the six cells v0..v5:
// uL = weno5z(v0..v4), uR = weno5z(v5..v1).  The two share two candidates
// (the quadratics through v1..v3 and v2..v4) and two second differences.
__device__ __forceinline__ void weno5z_pair(double v0, double v1, double v2, double v3, double v4, double v5,
                                            double eps, double& uL, double& uR) {
    const double c13 = 13.0 / 12.0;
    const double p123 = fma(-0.125, v1, fma(0.75, v2, 0.375 * v3));
    const double p234 = fma(0.375, v2, fma(0.75, v3, -0.125 * v4));
    const double pL0 = fma(0.375, v0, fma(-1.25, v1, 1.875 * v2));
    const double pR0 = fma(0.375, v5, fma(-1.25, v4, 1.875 * v3));
    const double a012 = v0 - 2.0 * v1 + v2, a123 = v1 - 2.0 * v2 + v3;
    const double a234 = v2 - 2.0 * v3 + v4, a345 = v3 - 2.0 * v4 + v5;
    const double k123 = c13 * a123 * a123, k234 = c13 * a234 * a234;
    const double eL0 = v0 - 4.0 * v1 + 3.0 * v2, eL1 = v1 - v3, eL2 = 3.0 * v2 - 4.0 * v3 + v4;
    const double eR0 = v5 - 4.0 * v4 + 3.0 * v3, eR1 = v4 - v2, eR2 = 3.0 * v3 - 4.0 * v2 + v1;
    const double bL0 = fma(c13 * a012, a012, fma(0.25 * eL0, eL0, eps));
    const double bL1 = k123 + fma(0.25 * eL1, eL1, eps);
    const double bL2 = k234 + fma(0.25 * eL2, eL2, eps);
    const double bR0 = fma(c13 * a345, a345, fma(0.25 * eR0, eR0, eps));
    const double bR1 = k234 + fma(0.25 * eR1, eR1, eps);
    const double bR2 = k123 + fma(0.25 * eR2, eR2, eps);
    uL = weno5z_combine(bL0, bL1, bL2, pL0, p123, p234);
    uR = weno5z_combine(bR0, bR1, bR2, pR0, p234, p123);
}

// Reverse mode of weno5z: g[i] += yb d weno5z(v0..v4)/d v_i.  The weights are
// homogeneous of degree 0 in (b_0, b_1, b_2), so the b_k are first scaled by
// their maximum; the A_k are then O(1) and their derivatives stay in range.
__device__ __forceinline__ void weno5z_vjp(double v0, double v1, double v2, double v3, double v4, double eps,
                                           double yb, double* g) {
    const double p0 = fma(0.375, v0, fma(-1.25, v1, 1.875 * v2));
    const double p1 = fma(-0.125, v1, fma(0.75, v2, 0.375 * v3));
    const double p2 = fma(0.375, v2, fma(0.75, v3, -0.125 * v4));
    const double c13 = 13.0 / 12.0;
    const double s0a = v0 - 2.0 * v1 + v2, s0b = v0 - 4.0 * v1 + 3.0 * v2;
    const double s1a = v1 - 2.0 * v2 + v3, s1b = v1 - v3;
    const double s2a = v2 - 2.0 * v3 + v4, s2b = 3.0 * v2 - 4.0 * v3 + v4;
    const double B0 = fma(c13 * s0a, s0a, 0.25 * s0b * s0b) + eps;
    const double B1 = fma(c13 * s1a, s1a, 0.25 * s1b * s1b) + eps;
    const double B2 = fma(c13 * s2a, s2a, 0.25 * s2b * s2b) + eps;
    const double bm = fmax(B0, fmax(B1, B2)), ibm = 1.0 / bm;
    const double b0 = B0 * ibm, b1 = B1 * ibm, b2 = B2 * ibm;
    const double t = b0 - b2, t2 = t * t;
    const double q0 = b0 * b0, q1 = b1 * b1, q2 = b2 * b2;
    const double A0 = (0.0625 * (q0 + t2)) * (q1 * q2);
    const double A1 = (0.625 * (q1 + t2)) * (q0 * q2);
    const double A2 = (0.3125 * (q2 + t2)) * (q0 * q1);
    const double iS = 1.0 / (A0 + A1 + A2);
    const double val = fma(A0, p0, fma(A1, p1, A2 * p2)) * iS;
    const double pb0 = yb * A0 * iS, pb1 = yb * A1 * iS, pb2 = yb * A2 * iS;
    const double ab0 = yb * (p0 - val) * iS, ab1 = yb * (p1 - val) * iS, ab2 = yb * (p2 - val) * iS;
    // A0 = d0 (q0 + t^2) q1 q2, A1 = d1 (q1 + t^2) q0 q2, A2 = d2 (q2 + t^2) q0 q1, t = b0 - b2
    const double bb0 = ab0 * 0.0625 * (2.0 * b0 + 2.0 * t) * q1 * q2 +
                       ab1 * 0.625 * (2.0 * t * q0 * q2 + (q1 + t2) * 2.0 * b0 * q2) +
                       ab2 * 0.3125 * (2.0 * t * q0 * q1 + (q2 + t2) * 2.0 * b0 * q1);
    const double bb1 = ab0 * 0.0625 * (q0 + t2) * 2.0 * b1 * q2 + ab1 * 0.625 * 2.0 * b1 * q0 * q2 +
                       ab2 * 0.3125 * (q2 + t2) * q0 * 2.0 * b1;
    const double bb2 = ab0 * 0.0625 * (-2.0 * t * q1 * q2 + (q0 + t2) * q1 * 2.0 * b2) +
                       ab1 * 0.625 * (-2.0 * t * q0 * q2 + (q1 + t2) * q0 * 2.0 * b2) +
                       ab2 * 0.3125 * (2.0 * b2 - 2.0 * t) * q0 * q1;
    // back to the unscaled beta_k (b_k = beta_k / bm; bm is a maximum, whose own
    // derivative cancels because the weights are scale invariant)
    const double be0 = bb0 * ibm, be1 = bb1 * ibm, be2 = bb2 * ibm;
    const double s0ab = be0 * 2.0 * c13 * s0a, s0bb = be0 * 0.5 * s0b;
    const double s1ab = be1 * 2.0 * c13 * s1a, s1bb = be1 * 0.5 * s1b;
    const double s2ab = be2 * 2.0 * c13 * s2a, s2bb = be2 * 0.5 * s2b;
    g[0] += 0.375 * pb0 + s0ab + s0bb;
    g[1] += -1.25 * pb0 - 0.125 * pb1 - 2.0 * s0ab - 4.0 * s0bb + s1ab + s1bb;
    g[2] += 1.875 * pb0 + 0.75 * pb1 + 0.375 * pb2 + s0ab + 3.0 * s0bb - 2.0 * s1ab + s2ab + 3.0 * s2bb;
    g[3] += 0.375 * pb1 + 0.75 * pb2 + s1ab - s1bb - 2.0 * s2ab - 4.0 * s2bb;
    g[4] += -0.125 * pb2 + s2ab + s2bb;
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
