// Hand-written vector-Jacobian products (reverse mode) of the DG path on
// flat-metric shells, with every branch frozen as the forward pass took it:
// the mask (all elements DG), the rectifier max(E^2 - B^2, 0), the branch of
// the stiff solve, the sign of S.n in the no-incoming-Poynting state.  The
// discrete map is smooth between branch changes (piecewise differentiable).
//
//   current_vjp     J~ = J~_drift + J~_eta (Sec. II.B)
//   solve_vjp       U = R + dt a G(U) (Sec. III.B): analytic branch and the
//                   scalar root s of the nonlinear branch by implicit differentiation
//   k_rhs_vjp       lambda^T dF/dU of the DG right-hand side: transposed
//                   derivative contractions of the 11 field weights, sources, the lifted
//                   Rusanov terms of my faces and of my neighbours' faces, the
//                   star / no-incoming boundary states, and d/d Omega at the star
//   k_filter_t      transpose of the exponential filter
#include "ffe_internal.h"
#include "physics.cuh"
#include "shellmap.cuh"
#include "stage.cuh"
#include "adjoint_common.cuh"

namespace ffe {

// ---------------------------------------------------------------------------
template <int P>
struct AVJ {
    static constexpr int np1 = P + 1, nn = np1 * np1 * np1, nf = np1 * np1, NT = ((nn + 31) / 32) * 32;
    // shared doubles: lambda [9][nn] | Y [11][nn] | C [6][9][nf]
    static constexpr int SMEM = (9 * nn + 11 * nn + 54 * nf) * 8;
};

__device__ __forceinline__ void unit_normal(const Dev& d, int64_t p, int dd, int s, double* n, double& norm) {
    double nn2 = 0.0;
    for (int i = 0; i < 3; ++i) {
        n[i] = (s ? 1.0 : -1.0) * d.geo[(int64_t)(3 * dd + i) * d.ndg + p];
        nn2 = fma(n[i], n[i], nn2);
    }
    norm = sqrt(nn2);
    for (int i = 0; i < 3; ++i) n[i] /= norm;
}

// z = (dC/dU_ext)^T lam = sc (sum_j n_j (dF^j/dU|_Ue)^T lam - lam), C the lifted Rusanov term
__device__ __forceinline__ void lift_ext_t(const double* Ue, double eta, const double* n, double sc, const double* lam,
                                           double* z) {
    double w[3][NV];
    for (int j = 0; j < 3; ++j)
        for (int v = 0; v < NV; ++v) w[j][v] = n[j] * lam[v];
    for (int v = 0; v < NV; ++v) z[v] = 0.0;
    flux_t(Ue, eta, w, z);
    for (int v = 0; v < NV; ++v) z[v] = sc * (z[v] - lam[v]);
}

template <int P>
__global__ void __launch_bounds__(AVJ<P>::NT) k_rhs_vjp(Dev d, Field U, Field L, Field out, double* omega_bar) {
    using K = AVJ<P>;
    constexpr int np1 = K::np1, nn = K::nn, nf = K::nf, NT = K::NT;
    extern __shared__ double sm[];
    double* sL = sm;              // [9][nn]
    double* sY = sL + 9 * nn;     // [11][nn]
    double* sC = sY + 11 * nn;    // [6][9][nf]
    __shared__ double s_om[NT];
    const Tables& T = d.tabs[P];
    const int tid = threadIdx.x;
    const bool act = tid < nn;
    const int ci[3] = {tid % np1, (tid / np1) % np1, tid / (np1 * np1)};
    const double w0inv = 1.0 / T.w0;
    for (int w = blockIdx.x; w < d.E; w += gridDim.x) {
        const int e = w;
        const int64_t eb = (int64_t)e * d.nn;
        if (d.mask[e] != 0) {
            // FD element: no DG right-hand side; its DG block of the adjoint is zero
            for (int t = tid; t < NV * nn; t += NT) out.dg(t / nn)[eb + t % nn] = 0.0;
            continue;
        }
        const double om = omega_of(d, e);
        double om_acc = 0.0;
        for (int t = tid; t < NV * nn; t += NT) sL[t] = L.dg(t / nn)[eb + t % nn];
        double lam[NV], u[NV], ij[3][3];
        if (act) {
            for (int v = 0; v < NV; ++v) { lam[v] = L.dg(v)[eb + tid]; u[v] = U.dg(v)[eb + tid]; }
            for (int k = 0; k < 3; ++k)
                for (int i = 0; i < 3; ++i) ij[k][i] = d.geo[(int64_t)(3 * k + i) * d.ndg + eb + tid];
        }
        // volume (flat metric): the forward builds curl, gradient and divergence
        // from the reference derivatives D_k X of the 11 fields X = E~, B~, psi~,
        // phi~, J~; its transpose gathers per axis k the weights Y_k,X(n) that
        // multiply D_k X at node n (lambda and the node's d xi^k/d x^j) and
        // contracts them with D_k^T:  Xbar(m) = sum_k sum_n D_k[n][m] Y_k,X(n)
        double xb[11];
        for (int w = 0; w < 11; ++w) xb[w] = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            __syncthreads();
            if (act) {
                const double ka = ij[k][0], kb = ij[k][1], kc = ij[k][2];
                double* y = sY + tid;
                y[0 * nn] = fma(-kc, lam[4], fma(kb, lam[5], -ka * lam[6]));    // E0
                y[1 * nn] = fma(kc, lam[3], fma(-ka, lam[5], -kb * lam[6]));    // E1
                y[2 * nn] = fma(-kb, lam[3], fma(ka, lam[4], -kc * lam[6]));    // E2
                y[3 * nn] = fma(kc, lam[1], fma(-kb, lam[2], -ka * lam[7]));    // B0
                y[4 * nn] = fma(-kc, lam[0], fma(ka, lam[2], -kb * lam[7]));    // B1
                y[5 * nn] = fma(kb, lam[0], fma(-ka, lam[1], -kc * lam[7]));    // B2
                y[6 * nn] = -fma(ka, lam[0], fma(kb, lam[1], kc * lam[2]));     // psi
                y[7 * nn] = -fma(ka, lam[3], fma(kb, lam[4], kc * lam[5]));     // phi
                y[8 * nn] = -ka * lam[8];                                       // J0
                y[9 * nn] = -kb * lam[8];                                       // J1
                y[10 * nn] = -kc * lam[8];                                      // J2
            }
            __syncthreads();
            if (act) {
                const int stride = k == 0 ? 1 : (k == 1 ? np1 : np1 * np1);
                const int base = tid - ci[k] * stride;
                double Dt[np1];
                for (int m = 0; m < np1; ++m) Dt[m] = T.D[m][ci[k]];
#pragma unroll
                for (int w = 0; w < 11; ++w) {
                    const double* src = sY + w * nn + base;
                    double acc = xb[w];
#pragma unroll
                    for (int m = 0; m < np1; ++m) acc = fma(Dt[m], src[m * stride], acc);
                    xb[w] = acc;
                }
            }
        }
        double ub[NV];
        for (int v = 0; v < NV; ++v) ub[v] = 0.0;
        if (act) {
            // fields directly; J~ (the q~ flux) through the current's Jacobian
            for (int v = 0; v < 8; ++v) ub[v] = xb[v];
            const double jb[3] = {xb[8], xb[9], xb[10]};
            current_vjp(u, d.eta, jb, jb, ub);
            const double wd[3] = {-lam[0], -lam[1], -lam[2]}, zero[3] = {0.0, 0.0, 0.0};
            current_vjp(u, d.eta, wd, zero, ub);
            ub[8] += lam[6];
        }
        // lift terms at face nodes: mine (dU_int) and my neighbours' (their dU_ext)
        for (int t = tid; t < 6 * nf; t += NT) {
            const int f = t / nf, ab = t % nf, ta = ab % np1, tb = ab / np1;
            const int dd = f >> 1, s = f & 1;
            const int t1 = dd == 0 ? 1 : 0, t2 = dd == 2 ? 1 : 2;
            int c[3];
            c[dd] = s ? P : 0;
            c[t1] = ta;
            c[t2] = tb;
            const int me = c[0] + np1 * (c[1] + np1 * c[2]);
            const int64_t p = eb + me;
            double n[3], norm;
            unit_normal(d, p, dd, s, n, norm);
            const double sc = 0.5 * norm * w0inv;
            double lm[NV], Ui[NV], acc[NV];
            for (int v = 0; v < NV; ++v) { lm[v] = sL[v * nn + me]; Ui[v] = U.dg(v)[p]; acc[v] = 0.0; }
            // (a) my term, through U_int: dU -= sc (n.(F(Ue) - F(Ui)) - (Ue - Ui))
            {
                double z[NV];
                lift_ext_t(Ui, d.eta, n, sc, lm, z);
                for (int v = 0; v < NV; ++v) acc[v] += z[v];
            }
            const int nb = d.nbr[e * 6 + f];
            if (nb < 0) {
                const int kind = d.bc[e * 6 + f];
                if (kind == FFE_BC_STAR || kind == FFE_BC_NO_INCOMING) {
                    double Ue[NV], z[NV];
                    double xn[3];
                    for (int q = 0; q < 3; ++q) xn[q] = d.xyz_dg[(int64_t)q * d.ndg + p];
                    if (kind == FFE_BC_STAR) bc_star_flat(Ui, xn, om, Ue);
                    else bc_no_incoming_flat(Ui, n, Ue);
                    lift_ext_t(Ue, d.eta, n, sc, lm, z);   // (dC/dUe)^T lambda
                    if (kind == FFE_BC_STAR) {
                        // Ue: E = B x v, v = Omega (-y, x, 0); B = B_i; psi = phi = q = 0
                        const double vv[3] = {-om * xn[1], om * xn[0], 0.0};
                        acc[3] -= vv[1] * z[2] - vv[2] * z[1];
                        acc[4] -= vv[2] * z[0] - vv[0] * z[2];
                        acc[5] -= vv[0] * z[1] - vv[1] * z[0];
                        acc[3] -= z[3]; acc[4] -= z[4]; acc[5] -= z[5];
                        // d Ue_E / d Omega = B x (z^ x x) = B x (-y, x, 0)
                        const double dv[3] = {-xn[1], xn[0], 0.0};
                        const double* B = Ui + 3;
                        const double dE[3] = {B[1] * dv[2] - B[2] * dv[1], B[2] * dv[0] - B[0] * dv[2], B[0] * dv[1] - B[1] * dv[0]};
                        om_acc -= dot3(z, dE);
                    } else {
                        const double S[3] = {Ui[1] * Ui[5] - Ui[2] * Ui[4], Ui[2] * Ui[3] - Ui[0] * Ui[5], Ui[0] * Ui[4] - Ui[1] * Ui[3]};
                        const bool inward = dot3(S, n) < 0.0;
                        if (!inward) { acc[0] -= z[0]; acc[1] -= z[1]; acc[2] -= z[2]; }
                        acc[3] -= z[3]; acc[4] -= z[4]; acc[5] -= z[5];
                        acc[8] -= z[8];
                    }
                }
            } else if (d.mask[nb] == 1) {
                // (b) my lift used the trace of the FD neighbour's FD -> DG projection
                // (6-point Lagrange per direction) of its cells and of their current as
                // exterior state and current (the flux is linear in both): scatter into its cells
                const int f2 = d.nbr_face[e * 6 + f], d2 = f2 >> 1, s2 = f2 & 1;
                const int u1 = d2 == 0 ? 1 : 0, u2 = d2 == 2 ? 1 : 2;
                int a2, b2, cn[3];
                orient_map(d.orient[e * 6 + f], np1, ta, tb, a2, b2);
                cn[d2] = s2 ? P : 0;
                cn[u1] = a2;
                cn[u2] = b2;
                // the exterior current is the projection of the cells' J~(U): (dC/d(Ue, Je))^T lambda;
                // the adjoint of the trace node goes to the neighbour's trace adjoint (one
                // writer per node), k_fd_traces_vjp takes it back to the cells
                double z[NV], zJ[3];
                lift_ext_tJ(n, sc, lm, z, zJ);   // dU -= C
                const int nfm = d.np1 * d.np1;
                double* tb = d.ftr_b + ((int64_t)fd_slot_of(d, nb) * 6 + f2) * 12 * nfm + cn[u1] + np1 * cn[u2];
                for (int v = 0; v < NV; ++v) tb[v * nfm] = -z[v];
                for (int k = 0; k < 3; ++k) tb[(NV + k) * nfm] = -zJ[k];
            } else {
                // (c) the neighbour's lift term at its node used my U as its exterior state
                const int f2 = d.nbr_face[e * 6 + f], d2 = f2 >> 1, s2 = f2 & 1;
                const int u1 = d2 == 0 ? 1 : 0, u2 = d2 == 2 ? 1 : 2;
                int a2, b2, cn[3];
                orient_map(d.orient[e * 6 + f], np1, ta, tb, a2, b2);
                cn[d2] = s2 ? P : 0;
                cn[u1] = a2;
                cn[u2] = b2;
                const int64_t q = (int64_t)nb * d.nn + cn[0] + np1 * (cn[1] + np1 * cn[2]);
                double n2[3], norm2, lnb[NV], z[NV];
                unit_normal(d, q, d2, s2, n2, norm2);
                for (int v = 0; v < NV; ++v) lnb[v] = L.dg(v)[q];
                lift_ext_t(Ui, d.eta, n2, 0.5 * norm2 * w0inv, lnb, z);
                for (int v = 0; v < NV; ++v) acc[v] -= z[v];
            }
            for (int v = 0; v < NV; ++v) sC[(f * NV + v) * nf + ab] = acc[v];
        }
        __syncthreads();
        if (act) {
            for (int dd = 0; dd < 3; ++dd) {
                const int t1 = dd == 0 ? 1 : 0, t2 = dd == 2 ? 1 : 2;
                const int ab = ci[t1] + np1 * ci[t2];
                if (ci[dd] == 0)
                    for (int v = 0; v < NV; ++v) ub[v] += sC[((2 * dd) * NV + v) * nf + ab];
                if (ci[dd] == P)
                    for (int v = 0; v < NV; ++v) ub[v] += sC[((2 * dd + 1) * NV + v) * nf + ab];
            }
            for (int v = 0; v < NV; ++v) out.dg(v)[eb + tid] = ub[v];
        }
        // Omega-bar: block sum in a fixed order, one atomic per element
        s_om[tid] = om_acc;
        __syncthreads();
        if (tid == 0 && omega_bar) {
            double sacc = 0.0;
            for (int i = 0; i < NT; ++i) sacc += s_om[i];
            if (sacc != 0.0) atomicAdd(omega_bar, sacc);
        }
        __syncthreads();
    }
}

void launch_rhs_vjp(const Dev& d, Field U, Field L, Field out, double* omega_bar, cudaStream_t st) {
    prof_begin("rhs_vjp", st);
    switch (d.P) {
#define FFE_VJP(PP)                                                                                        \
    case PP:                                                                                               \
        cudaFuncSetAttribute(k_rhs_vjp<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, AVJ<PP>::SMEM);  \
        k_rhs_vjp<PP><<<d.nsm * 2, AVJ<PP>::NT, AVJ<PP>::SMEM, st>>>(d, U, L, out, omega_bar);            \
        break;
        FFE_VJP(3)
        FFE_VJP(4)
        FFE_VJP(5)
#undef FFE_VJP
        default: break;
    }
    prof_end(st);
    g_launch_counter += 1;
}

// ---------------------------------------------------------------------------
// Filter (or its transpose) of nv variables of every element, one CTA per element.
__global__ void k_filter(Dev d, Field in, Field outf, int nv, int transpose) {
    extern __shared__ double sm[];
    const int np1 = d.np1, nn = d.nn;
    const Tables& T = d.tabs[d.P];
    double* a = sm;
    double* b = sm + nn;
    for (int e = blockIdx.x; e < d.E; e += gridDim.x) {
        if (d.mask[e] != 0) continue;   // FD elements are not filtered
        const int64_t eb = (int64_t)e * d.nn;
        for (int v = 0; v < nv; ++v) {
            for (int t = threadIdx.x; t < nn; t += blockDim.x) a[t] = in.dg(v)[eb + t];
            __syncthreads();
            for (int k = 0; k < 3; ++k) {
                const double* src = (k == 1) ? b : a;
                double* dst = (k == 1) ? a : b;
                const int stride = k == 0 ? 1 : (k == 1 ? np1 : np1 * np1);
                for (int t = threadIdx.x; t < nn; t += blockDim.x) {
                    const int ck = (t / stride) % np1, base = t - ck * stride;
                    double acc = 0.0;
                    for (int m = 0; m < np1; ++m)
                        acc = fma(transpose ? T.Filt[m][ck] : T.Filt[ck][m], src[base + m * stride], acc);
                    if (k < 2) dst[t] = acc;
                    else outf.dg(v)[eb + t] = acc;
                }
                __syncthreads();
            }
        }
    }
}

void launch_filter(const Dev& d, Field in, Field out, int nv, int transpose, cudaStream_t st) {
    prof_begin("filter", st);
    k_filter<<<d.nsm * 4, 128, 2 * d.nn * sizeof(double), st>>>(d, in, out, nv, transpose);
    prof_end(st);
    g_launch_counter += 1;
}

// ---------------------------------------------------------------------------
// Pointwise kernels of the adjoint step over the active points: DG nodes of
// DG elements and cells of FD elements (fixed mask).

// Point p of [0, ndg + nfd): DG node p, else FD cell p - ndg; q is its index in
// its block.  False unless the point belongs to its element's representation.
__device__ __forceinline__ bool act_point(const Dev& d, int64_t p, bool& isfd, int64_t& q) {
    if (p < d.ndg) {
        isfd = false;
        q = p;
        return d.mask[p / d.nn] == 0;
    }
    isfd = true;
    q = p - d.ndg;
    const int sl = (int)(q / d.ncell);
    const int e = d.slot_elem ? d.slot_elem[sl] : sl;
    return e >= 0 && d.mask[e] == 1;
}

// The same points visited through the FD list: p < ndg is DG node p, else the
// (p - ndg)-th cell of the listed FD elements; act_count is the range.
__device__ __forceinline__ int64_t act_count(const Dev& d) { return d.ndg + (int64_t)d.counts[1] * d.ncell; }
__device__ __forceinline__ bool act_listed(const Dev& d, int64_t p, bool& isfd, int64_t& q) {
    if (p < d.ndg) {
        isfd = false;
        q = p;
        return d.mask[p / d.nn] == 0;
    }
    isfd = true;
    const int64_t r = p - d.ndg;
    const int e = d.fd_list[r / d.ncell];
    const int c = (int)(r % d.ncell);
    q = fdb(d, e) + c;
    return c < esz(d, e).ncell;
}
__device__ __forceinline__ double* fp(const Field& f, int v, bool isfd) { return isfd ? f.fd(v) : f.dg(v); }

// forward recomputation: stage 1-2 (U2, G1, G2)
__global__ void k_adj_s12(Dev d, AdjArgs a) {
    const double dt = d.dt, dta = dt * IM_A;
    const int64_t np_ = act_count(d);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np_; p += (int64_t)gridDim.x * blockDim.x) {
        bool isfd;
        int64_t q;
        if (!act_listed(d, p, isfd, q)) continue;
        double u[NV], U1[NV], g1[NG], g2[NG];
        for (int v = 0; v < NV; ++v) { u[v] = fp(a.un, v, isfd)[q]; U1[v] = u[v]; }
        stiff_solve_flat(U1, d, dta);
        if (d.mode != FFE_RELAX) hard_clamp_flat(U1);
        implicit_G_flat(U1, d, g1);
        u[0] = fma(-dta, g1[0], u[0]);
        u[1] = fma(-dta, g1[1], u[1]);
        u[2] = fma(-dta, g1[2], u[2]);
        u[6] = fma(-dta, g1[3], u[6]);
        u[7] = fma(-dta, g1[4], u[7]);
        stiff_solve_flat(u, d, dta);
        if (d.mode != FFE_RELAX) hard_clamp_flat(u);
        implicit_G_flat(u, d, g2);
        for (int v = 0; v < NV; ++v) fp(a.U2, v, isfd)[q] = u[v];
        for (int c = 0; c < NG; ++c) { fp(a.G1, c, isfd)[q] = g1[c]; fp(a.G2, c, isfd)[q] = g2[c]; }
    }
}

// forward recomputation: R = un + dt (...) of substep sub; T = S(R) (A, B) or W = R (C)
__global__ void k_adj_comb(Dev d, AdjArgs a, int sub) {
    const double dt = d.dt;
    const int gv[NG] = {0, 1, 2, 6, 7};
    const double z = 0.5 - IM_B - IM_H - IM_A;
    const int64_t np_ = act_count(d);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np_; p += (int64_t)gridDim.x * blockDim.x) {
        bool isfd;
        int64_t q;
        if (!act_listed(d, p, isfd, q)) continue;
        double u[NV];
        for (int v = 0; v < NV; ++v) u[v] = fp(a.un, v, isfd)[q];
        if (sub == SUB_A) {
            for (int v = 0; v < NV; ++v) u[v] = fma(dt, fp(a.F2, v, isfd)[q], u[v]);
            for (int c = 0; c < NG; ++c) u[gv[c]] = fma(dt * (1.0 - IM_A), fp(a.G2, c, isfd)[q], u[gv[c]]);
        } else if (sub == SUB_B) {
            for (int v = 0; v < NV; ++v) u[v] = fma(0.25 * dt, fp(a.F2, v, isfd)[q] + fp(a.F3, v, isfd)[q], u[v]);
            for (int c = 0; c < NG; ++c)
                u[gv[c]] = fma(dt, IM_B * fp(a.G1, c, isfd)[q] + IM_H * fp(a.G2, c, isfd)[q] + z * fp(a.G3, c, isfd)[q], u[gv[c]]);
        } else {
            for (int v = 0; v < NV; ++v)
                u[v] = fma(dt, (fp(a.F2, v, isfd)[q] + fp(a.F3, v, isfd)[q]) * (1.0 / 6.0) + fp(a.F4, v, isfd)[q] * (2.0 / 3.0), u[v]);
            for (int c = 0; c < NG; ++c)
                u[gv[c]] = fma(dt, (fp(a.G2, c, isfd)[q] + fp(a.G3, c, isfd)[q]) * (1.0 / 6.0) + fp(a.G4, c, isfd)[q] * (2.0 / 3.0), u[gv[c]]);
        }
        const Field& R = sub == SUB_A ? a.R3 : (sub == SUB_B ? a.R4 : a.W);
        for (int v = 0; v < NV; ++v) fp(R, v, isfd)[q] = u[v];
    }
}

// forward recomputation: U_s = S(T_s) with T_s the filtered explicit part, G_s = G(U_s)
__global__ void k_adj_solve(Dev d, AdjArgs a, int sub) {
    const double dta = d.dt * IM_A;
    const Field& Tt = sub == SUB_A ? a.T3 : a.T4;
    const Field& Us = sub == SUB_A ? a.U3 : a.U4;
    const Field& Gs = sub == SUB_A ? a.G3 : a.G4;
    const int64_t np_ = act_count(d);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np_; p += (int64_t)gridDim.x * blockDim.x) {
        bool isfd;
        int64_t q;
        if (!act_listed(d, p, isfd, q)) continue;
        double u[NV], g[NG];
        for (int v = 0; v < NV; ++v) u[v] = fp(Tt, v, isfd)[q];
        stiff_solve_flat(u, d, dta);
        if (d.mode != FFE_RELAX) hard_clamp_flat(u);
        implicit_G_flat(u, d, g);
        for (int v = 0; v < NV; ++v) fp(Us, v, isfd)[q] = u[v];
        for (int c = 0; c < NG; ++c) fp(Gs, c, isfd)[q] = g[c];
    }
}

// reverse step pieces (see adjoint_step in host.cu for the order)
// (1) from W-bar (in tmp): u-bar = Wb; Fk-bar, Gk-bar seeds
__global__ void k_adj_seed(Dev d, AdjArgs a) {
    const double dt = d.dt;
    const int gv[NG] = {0, 1, 2, 6, 7};
    const int64_t np_ = act_count(d);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np_; p += (int64_t)gridDim.x * blockDim.x) {
        bool isfd;
        int64_t q;
        if (!act_listed(d, p, isfd, q)) continue;
        for (int v = 0; v < NV; ++v) {
            const double w = fp(a.tmp, v, isfd)[q];
            fp(a.ubar, v, isfd)[q] = w;
            fp(a.F2b, v, isfd)[q] = dt / 6.0 * w;
            fp(a.F3b, v, isfd)[q] = dt / 6.0 * w;
            fp(a.F4b, v, isfd)[q] = 2.0 * dt / 3.0 * w;
        }
        for (int c = 0; c < NG; ++c) {
            const double w = fp(a.tmp, gv[c], isfd)[q];
            fp(a.G1b, c, isfd)[q] = 0.0;
            fp(a.G2b, c, isfd)[q] = dt / 6.0 * w;
            fp(a.G3b, c, isfd)[q] = dt / 6.0 * w;
            fp(a.G4b, c, isfd)[q] = 2.0 * dt / 3.0 * w;
        }
    }
}

// (2) tmp = U-bar of stage U_s: RHS-vjp result (in tmp) + G-vjp of Gs-bar at U_s
__global__ void k_adj_addG(Dev d, Field U, Field Gb, Field io) {
    const int64_t np_ = act_count(d);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np_; p += (int64_t)gridDim.x * blockDim.x) {
        bool isfd;
        int64_t q;
        if (!act_listed(d, p, isfd, q)) continue;
        double u[NV], gb[NG], ub[NV];
        for (int v = 0; v < NV; ++v) { u[v] = fp(U, v, isfd)[q]; ub[v] = fp(io, v, isfd)[q]; }
        for (int c = 0; c < NG; ++c) gb[c] = fp(Gb, c, isfd)[q];
        G_vjp(u, d, gb, ub);
        for (int v = 0; v < NV; ++v) fp(io, v, isfd)[q] = ub[v];
    }
}

// (2b) T-bar (in tmp2) = solve_vjp(T_s, U_s-bar in tmp)
__global__ void k_adj_solve_back(Dev d, AdjArgs a, int sub) {
    const double dta = d.dt * IM_A;
    const Field& Tt = sub == SUB_A ? a.T3 : a.T4;
    const int64_t np_ = act_count(d);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np_; p += (int64_t)gridDim.x * blockDim.x) {
        bool isfd;
        int64_t q;
        if (!act_listed(d, p, isfd, q)) continue;
        double t[NV], ub[NV], tb[NV];
        for (int v = 0; v < NV; ++v) { t[v] = fp(Tt, v, isfd)[q]; ub[v] = fp(a.tmp, v, isfd)[q]; }
        if (d.mode != FFE_RELAX) {
            // U_s = clamp(S(T_s)): back through the clamp at S(T_s) first
            double x[NV];
            for (int v = 0; v < NV; ++v) x[v] = t[v];
            stiff_solve_flat(x, d, dta);
            clamp_vjp(x, ub);
        }
        solve_vjp(t, d, dta, ub, tb);
        for (int v = 0; v < NV; ++v) fp(a.tmp2, v, isfd)[q] = tb[v];
    }
}

// (3) given R-bar (in tmp, the filter transpose of T-bar): the contributions of
//     R = un + dt (...) to u-bar, F-bar, G-bar
__global__ void k_adj_back_comb(Dev d, AdjArgs a, int sub) {
    const double dt = d.dt;
    const int gv[NG] = {0, 1, 2, 6, 7};
    const double z = 0.5 - IM_B - IM_H - IM_A;
    const int64_t np_ = act_count(d);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np_; p += (int64_t)gridDim.x * blockDim.x) {
        bool isfd;
        int64_t q;
        if (!act_listed(d, p, isfd, q)) continue;
        double rb[NV];
        for (int v = 0; v < NV; ++v) rb[v] = fp(a.tmp, v, isfd)[q];
        for (int v = 0; v < NV; ++v) fp(a.ubar, v, isfd)[q] += rb[v];
        if (sub == SUB_B) {
            for (int v = 0; v < NV; ++v) {
                fp(a.F2b, v, isfd)[q] += 0.25 * dt * rb[v];
                fp(a.F3b, v, isfd)[q] += 0.25 * dt * rb[v];
            }
            for (int c = 0; c < NG; ++c) {
                fp(a.G1b, c, isfd)[q] += dt * IM_B * rb[gv[c]];
                fp(a.G2b, c, isfd)[q] += dt * IM_H * rb[gv[c]];
                fp(a.G3b, c, isfd)[q] += dt * z * rb[gv[c]];
            }
        } else {
            for (int v = 0; v < NV; ++v) fp(a.F2b, v, isfd)[q] += dt * rb[v];
            for (int c = 0; c < NG; ++c) fp(a.G2b, c, isfd)[q] += dt * (1.0 - IM_A) * rb[gv[c]];
        }
    }
}

// (4) stages 2 and 1: U2-bar in tmp; recompute U1, R2 from un
__global__ void k_adj_back_s12(Dev d, AdjArgs a) {
    const double dta = d.dt * IM_A;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < d.ndg + d.nfd; p += (int64_t)gridDim.x * blockDim.x) {
        bool isfd;
        int64_t q;
        if (!act_point(d, p, isfd, q)) {
            // lambda_n is zero on the representation an element does not use
            for (int v = 0; v < NV; ++v) fp(a.lam, v, isfd)[q] = 0.0;
            continue;
        }
        double un[NV], U1[NV], R2[NV], g1[NG], u2b[NV], r2b[NV], g1b[NG], u1b[NV], r1b[NV];
        const bool clamp = d.mode != FFE_RELAX;
        double V1[NV], V2[NV];   // the solve outputs before the clamp (HARD modes)
        for (int v = 0; v < NV; ++v) { un[v] = fp(a.un, v, isfd)[q]; U1[v] = un[v]; u2b[v] = fp(a.tmp, v, isfd)[q]; }
        stiff_solve_flat(U1, d, dta);
        for (int v = 0; v < NV; ++v) V1[v] = U1[v];
        if (clamp) hard_clamp_flat(U1);
        implicit_G_flat(U1, d, g1);
        for (int v = 0; v < NV; ++v) R2[v] = un[v];
        R2[0] = fma(-dta, g1[0], R2[0]);
        R2[1] = fma(-dta, g1[1], R2[1]);
        R2[2] = fma(-dta, g1[2], R2[2]);
        R2[6] = fma(-dta, g1[3], R2[6]);
        R2[7] = fma(-dta, g1[4], R2[7]);
        if (clamp) {
            for (int v = 0; v < NV; ++v) V2[v] = R2[v];
            stiff_solve_flat(V2, d, dta);
            clamp_vjp(V2, u2b);
        }
        solve_vjp(R2, d, dta, u2b, r2b);
        const int gv[NG] = {0, 1, 2, 6, 7};
        for (int c = 0; c < NG; ++c) g1b[c] = fp(a.G1b, c, isfd)[q] - dta * r2b[gv[c]];
        for (int v = 0; v < NV; ++v) u1b[v] = 0.0;
        G_vjp(U1, d, g1b, u1b);
        if (clamp) clamp_vjp(V1, u1b);
        solve_vjp(un, d, dta, u1b, r1b);
        for (int v = 0; v < NV; ++v) fp(a.lam, v, isfd)[q] = fp(a.ubar, v, isfd)[q] + r2b[v] + r1b[v];
    }
}

// HARD modes, the step's end: u_{n+1} = clamp(X), X = filter(W).
// (7) in place: io = clamp(io)
__global__ void k_adj_clamp(Dev d, Field io) {
    const int64_t np_ = act_count(d);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np_; p += (int64_t)gridDim.x * blockDim.x) {
        bool isfd;
        int64_t q;
        if (!act_listed(d, p, isfd, q)) continue;
        double u[NV];
        for (int v = 0; v < NV; ++v) u[v] = fp(io, v, isfd)[q];
        hard_clamp_flat(u);
        for (int v = 0; v < 3; ++v) fp(io, v, isfd)[q] = u[v];
    }
}

// (8) out = (d clamp/dX at X)^T yb
__global__ void k_adj_clamp_back(Dev d, Field X, Field yb, Field out) {
    const int64_t np_ = act_count(d);
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np_; p += (int64_t)gridDim.x * blockDim.x) {
        bool isfd;
        int64_t q;
        if (!act_listed(d, p, isfd, q)) continue;
        double x[NV], ub[NV];
        for (int v = 0; v < NV; ++v) { x[v] = fp(X, v, isfd)[q]; ub[v] = fp(yb, v, isfd)[q]; }
        clamp_vjp(x, ub);
        for (int v = 0; v < NV; ++v) fp(out, v, isfd)[q] = ub[v];
    }
}

void launch_adj_clamp(const Dev& d, Field io, cudaStream_t st) {
    prof_begin("adj_pointwise", st);
    k_adj_clamp<<<d.nsm * 8, 256, 0, st>>>(d, io);
    prof_end(st);
    g_launch_counter += 1;
}

void launch_adj_clamp_back(const Dev& d, Field X, Field yb, Field out, cudaStream_t st) {
    prof_begin("adj_pointwise", st);
    k_adj_clamp_back<<<d.nsm * 8, 256, 0, st>>>(d, X, yb, out);
    prof_end(st);
    g_launch_counter += 1;
}

void launch_adj(const Dev& d, int which, AdjArgs a, int sub, cudaStream_t st) {
    const int grid = d.nsm * 8;
    prof_begin("adj_pointwise", st);
    switch (which) {
        case 0: k_adj_s12<<<grid, 256, 0, st>>>(d, a); break;
        case 1: k_adj_comb<<<grid, 256, 0, st>>>(d, a, sub); break;
        case 2: k_adj_seed<<<grid, 256, 0, st>>>(d, a); break;
        case 3: k_adj_back_comb<<<grid, 256, 0, st>>>(d, a, sub); break;
        case 4: k_adj_back_s12<<<grid, 256, 0, st>>>(d, a); break;
        case 5: k_adj_solve_back<<<grid, 256, 0, st>>>(d, a, sub); break;
        case 6: k_adj_solve<<<grid, 256, 0, st>>>(d, a, sub); break;
        default: break;
    }
    prof_end(st);
    g_launch_counter += 1;
}

void launch_adj_addG(const Dev& d, Field U, Field Gb, Field io, cudaStream_t st) {
    prof_begin("adj_pointwise", st);
    k_adj_addG<<<d.nsm * 8, 256, 0, st>>>(d, U, Gb, io);
    prof_end(st);
    g_launch_counter += 1;
}

// ---------------------------------------------------------------------------
// Luminosity through r = r_L: L = sum over surface nodes W_n (E x B).rhat at the
// interpolated point; gradient dL/dU at the nodes of the radial element layer.
struct LumArgs {
    const int* elem;        // [ns] element of surface column s
    const double* lk;       // [np1] interpolation weights along xi^3
    const double* wn;       // [ns][np1^2][4]: weight, outward unit normal (3) at (i, j)
    int ns;
    int bflux;              // 1: integrate B~.n (magnetic flux) instead of (E x B).n
};

__global__ void k_luminosity(Dev d, Field U, LumArgs la, double* out, Field grad, double scale) {
    const int np1 = d.np1, nf = np1 * np1;
    __shared__ double red[256];
    double acc = 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < la.ns * nf; t += gridDim.x * blockDim.x) {
        const int s = t / nf, ij = t % nf;
        const int e = la.elem[s];
        const int64_t eb = (int64_t)e * d.nn;
        const bool fde = d.mask[e] == 1;
        const Tables& T = d.tabs[d.P];
        const int nc = T.nc, i0 = ij % np1, j0 = ij / np1;
        const int64_t fb = fde ? fdb(d, e) : 0;
        // node value of variable v at (i0, j0, k): DG node, or the FD -> DG
        // projection (6-point Lagrange per direction) of an FD element's cells
        auto nodal = [&](int v, int k) -> double {
            if (!fde) return U.dg(v)[eb + ij + nf * k];
            const int lo0 = T.f2d_lo[i0], lo1 = T.f2d_lo[j0], lo2 = T.f2d_lo[k];
            double a2 = 0.0;
            for (int n2 = 0; n2 < 6; ++n2) {
                double a1 = 0.0;
                for (int n1 = 0; n1 < 6; ++n1) {
                    const double* row = U.fd(v) + fb + lo0 + nc * ((lo1 + n1) + nc * (lo2 + n2));
                    double a0 = 0.0;
                    for (int n0 = 0; n0 < 6; ++n0) a0 = fma(T.F2D[i0][lo0 + n0], row[n0], a0);
                    a1 = fma(T.F2D[j0][lo1 + n1], a0, a1);
                }
                a2 = fma(T.F2D[k][lo2 + n2], a1, a2);
            }
            return a2;
        };
        double E[3] = {0, 0, 0}, B[3] = {0, 0, 0};
        for (int k = 0; k < np1; ++k) {
            for (int a = 0; a < 3; ++a) {
                E[a] = fma(la.lk[k], nodal(a, k), E[a]);
                B[a] = fma(la.lk[k], nodal(3 + a, k), B[a]);
            }
        }
        const double* w = la.wn + ((int64_t)s * nf + ij) * 4;
        const double r[3] = {w[1], w[2], w[3]};
        const double S[3] = {E[1] * B[2] - E[2] * B[1], E[2] * B[0] - E[0] * B[2], E[0] * B[1] - E[1] * B[0]};
        acc = fma(w[0], la.bflux ? dot3(B, r) : dot3(S, r), acc);
        if (grad.p && !la.bflux) {
            // d/dE = W (B x r), d/dB = W (r x E), spread with l_k
            const double gE[3] = {B[1] * r[2] - B[2] * r[1], B[2] * r[0] - B[0] * r[2], B[0] * r[1] - B[1] * r[0]};
            const double gB[3] = {r[1] * E[2] - r[2] * E[1], r[2] * E[0] - r[0] * E[2], r[0] * E[1] - r[1] * E[0]};
            for (int k = 0; k < np1; ++k) {
                const double f = scale * w[0] * la.lk[k];
                if (!fde) {
                    const int64_t p = eb + ij + nf * k;
                    for (int a = 0; a < 3; ++a) {
                        grad.dg(a)[p] += f * gE[a];
                        grad.dg(3 + a)[p] += f * gB[a];
                    }
                    continue;
                }
                const int lo0 = T.f2d_lo[i0], lo1 = T.f2d_lo[j0], lo2 = T.f2d_lo[k];
                for (int n2 = 0; n2 < 6; ++n2)
                    for (int n1 = 0; n1 < 6; ++n1)
                        for (int n0 = 0; n0 < 6; ++n0) {
                            const double wgt = f * T.F2D[i0][lo0 + n0] * T.F2D[j0][lo1 + n1] * T.F2D[k][lo2 + n2];
                            const int64_t cell = fb + lo0 + n0 + nc * ((lo1 + n1) + nc * (lo2 + n2));
                            for (int a = 0; a < 3; ++a) {
                                atomicAdd(grad.fd(a) + cell, wgt * gE[a]);
                                atomicAdd(grad.fd(3 + a) + cell, wgt * gB[a]);
                            }
                        }
            }
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sacc = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) sacc += red[i];
        out[blockIdx.x] = sacc;
    }
}

void launch_luminosity(const Dev& d, Field U, const int* elem, const double* lk, const double* wn, int ns,
                       double* partial, int nblocks, Field grad, double scale, cudaStream_t st, int bflux) {
    LumArgs la{elem, lk, wn, ns, bflux};
    k_luminosity<<<nblocks, 256, 0, st>>>(d, U, la, partial, grad, scale);
    g_launch_counter += 1;
}

}  // namespace ffe
