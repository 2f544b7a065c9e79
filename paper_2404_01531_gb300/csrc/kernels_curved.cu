// DG substep on curved elements (cubed-sphere shells), flat or Kerr-Schild metric.
//
// Per element (one CTA, one thread per LGL node) the chain-rule strong form
//   dU/dt = - sum_k sum_j (d xi^k/d x^j)_n (D_k F^j)_n + S
//           - sum_faces (|grad xi^d|_gamma / w0) (F*.n^ - F_int.n^)
// with F^j the physical fluxes at the nodes (Sec. II.A), the inverse Jacobian
// of the element map at each node, the Rusanov flux with lambda = alpha +
// |beta.n^|, then the same stage order as the box kernel (explicit part,
// filter, stiff solve, clamp, indicator).  The stiff solve, clamp and indicator
// use the gamma inner product.
#include "dgfilter.cuh"
#include "ffe_internal.h"
#include "physics.cuh"
#include "physics_gen.cuh"
#include "shellmap.cuh"
#include "stage.cuh"

namespace ffe {

template <int P>
struct DGC {
    static constexpr int np1 = P + 1;
    static constexpr int nn = np1 * np1 * np1;
    static constexpr int nf = np1 * np1;
    static constexpr int NT = ((nn + 31) / 32) * 32;
    static constexpr int NW = NT / 32;
    // shared doubles: U[9][nn] | F[27][nn] (the filter buffer [9][nn] aliases it) | C[6][9][nf] | red[2][NW]
    static constexpr int SMEM = (9 * nn + 27 * nn + 54 * nf + 2 * NW + 1) * 8;
};

template <bool KS>
__device__ __forceinline__ void node_metric(const Dev& d, int64_t p, PM& m) {
    if (KS) {
        load_pm(d.met, d.ndg, p, m);
    } else {
        m.a = 1.0;
        m.b[0] = m.b[1] = m.b[2] = 0.0;
        for (int i = 0; i < 6; ++i) m.gl[i] = m.gu[i] = (i == 0 || i == 3 || i == 5) ? 1.0 : 0.0;
        m.sg = 1.0;
    }
}

template <bool KS>
__device__ __forceinline__ void fluxes_at(const double* U, const PM& m, double eta, double F[3][NV], double* jd) {
    double jf[3];
    if (KS) current_gen(U, m, eta, jd, jf);
    else current_flat(U, eta, jd, jf);
    flux_gen(U, jf, m, F);
}

template <int NW>
__device__ __forceinline__ void block_sum2c(double& x, double& y, double* red) {
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_down_sync(0xffffffffu, x, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { red[w] = x; red[NW + w] = y; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sx = 0.0, sy = 0.0;
        for (int i = 0; i < NW; ++i) { sx += red[i]; sy += red[NW + i]; }
        red[0] = sx;
        red[NW] = sy;
    }
    __syncthreads();
    x = red[0];
    y = red[NW];
}

// neighbour's node for my face node (ta, tb) of face f
template <int P>
__device__ __forceinline__ void nbr_node(const Dev& d, int e, int f, int ta, int tb, int c[3]) {
    const int f2 = d.nbr_face[e * 6 + f], d2 = f2 >> 1;
    const int u1 = d2 == 0 ? 1 : 0, u2 = d2 == 2 ? 1 : 2;
    int a2, b2;
    orient_map(d.orient[e * 6 + f], P + 1, ta, tb, a2, b2);
    c[d2] = (f2 & 1) ? P : 0;
    c[u1] = a2;
    c[u2] = b2;
}

// One element of order P processed by a block of NT threads (NT >= (P+1)^3).
template <int P, int NT, int SUB, bool KS>
__device__ __forceinline__ void dg_curved_elem(const Dev& d, const SubArgs& a, int e, double* sm) {
    using K = DGC<P>;
    constexpr int np1 = K::np1, nn = K::nn, nf = K::nf, NW = NT / 32;
    double* sU = sm;                 // [9][nn]
    double* sF = sU + 9 * nn;        // [3][9][nn]
    double* sC = sF + 27 * nn;       // [6][9][nf]
    double* red = sC + 54 * nf;
    const Tables& T = d.tabs[P];
    const int tid = threadIdx.x;
    const bool act = tid < nn;
    const int ci[3] = {tid % np1, (tid / np1) % np1, tid / (np1 * np1)};
    const double w0inv = 1.0 / T.w0;
    {
        const int64_t eb = (int64_t)e * d.nn;
        const double dt = dt_of(d, e);
        for (int t = tid; t < NV * nn; t += NT) sU[t] = a.Uin.dg(t / nn)[eb + t % nn];
        __syncthreads();
        PM m;
        double jd[3] = {0.0, 0.0, 0.0}, ij[3][3];
        if (act) {
            node_metric<KS>(d, eb + tid, m);
            for (int k = 0; k < 3; ++k)
                for (int i = 0; i < 3; ++i) ij[k][i] = d.geo[(int64_t)(3 * k + i) * d.ndg + eb + tid];
            double u[NV];
            for (int v = 0; v < NV; ++v) u[v] = sU[v * nn + tid];
            if (KS) {
                double F[3][NV];
                fluxes_at<KS>(u, m, d.eta, F, jd);
                for (int j = 0; j < 3; ++j)
                    for (int v = 0; v < NV; ++v) sF[(j * NV + v) * nn + tid] = F[j][v];
            } else {
                // flat metric: the fluxes are fixed linear combinations of E~, B~,
                // psi~, phi~ and J~, so only J~ (full) is stored beside U
                double jf[3];
                current_flat(u, d.eta, jd, jf);
                for (int i = 0; i < 3; ++i) sF[i * nn + tid] = jf[i];
            }
        }
        __syncthreads();
        double du[NV];
        if (act && !KS) {
            // flat metric: D_k F^j = +-D_k of one field (D_k is linear), so the
            // volume term is built from the reference derivatives R = D_k X of the
            // 11 fields X = E~, B~, psi~, phi~, J~ and the node's d xi^k/d x^j:
            //   E~: curl B~ - grad psi~,  B~: -curl E~ - grad phi~,
            //   psi~: -div E~,  phi~: -div B~,  q~: -div J~
            for (int v = 0; v < NV; ++v) du[v] = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int stride = k == 0 ? 1 : (k == 1 ? np1 : np1 * np1);
                const int base = tid - ci[k] * stride;
                double Dk[np1];
                for (int mm = 0; mm < np1; ++mm) Dk[mm] = T.D[ci[k]][mm];
                auto R = [&](const double* f) {
                    double acc = 0.0;
#pragma unroll
                    for (int mm = 0; mm < np1; ++mm) acc = fma(Dk[mm], f[base + mm * stride], acc);
                    return acc;
                };
                const double ka = ij[k][0], kb = ij[k][1], kc = ij[k][2];
                double r;
                r = R(sU + 0 * nn);   // E0
                du[4] = fma(-kc, r, du[4]); du[5] = fma(kb, r, du[5]); du[6] = fma(-ka, r, du[6]);
                r = R(sU + 1 * nn);   // E1
                du[3] = fma(kc, r, du[3]); du[5] = fma(-ka, r, du[5]); du[6] = fma(-kb, r, du[6]);
                r = R(sU + 2 * nn);   // E2
                du[3] = fma(-kb, r, du[3]); du[4] = fma(ka, r, du[4]); du[6] = fma(-kc, r, du[6]);
                r = R(sU + 3 * nn);   // B0
                du[1] = fma(kc, r, du[1]); du[2] = fma(-kb, r, du[2]); du[7] = fma(-ka, r, du[7]);
                r = R(sU + 4 * nn);   // B1
                du[0] = fma(-kc, r, du[0]); du[2] = fma(ka, r, du[2]); du[7] = fma(-kb, r, du[7]);
                r = R(sU + 5 * nn);   // B2
                du[0] = fma(kb, r, du[0]); du[1] = fma(-ka, r, du[1]); du[7] = fma(-kc, r, du[7]);
                r = R(sU + 6 * nn);   // psi
                du[0] = fma(-ka, r, du[0]); du[1] = fma(-kb, r, du[1]); du[2] = fma(-kc, r, du[2]);
                r = R(sU + 7 * nn);   // phi
                du[3] = fma(-ka, r, du[3]); du[4] = fma(-kb, r, du[4]); du[5] = fma(-kc, r, du[5]);
                r = R(sF + 0 * nn);   // J0
                du[8] = fma(-ka, r, du[8]);
                r = R(sF + 1 * nn);   // J1
                du[8] = fma(-kb, r, du[8]);
                r = R(sF + 2 * nn);   // J2
                du[8] = fma(-kc, r, du[8]);
            }
        }
        if (act && KS) {
            for (int v = 0; v < NV; ++v) du[v] = 0.0;
            for (int k = 0; k < 3; ++k) {
                const int stride = k == 0 ? 1 : (k == 1 ? np1 : np1 * np1);
                const int base = tid - ci[k] * stride;
                double Dk[np1];
                for (int mm = 0; mm < np1; ++mm) Dk[mm] = T.D[ci[k]][mm];
                for (int j = 0; j < 3; ++j) {
                    const double s = -ij[k][j];
                    for (int v = 0; v < NV; ++v) {
                        const double* src = sF + (j * NV + v) * nn + base;
                        double acc = 0.0;
#pragma unroll
                        for (int mm = 0; mm < np1; ++mm) acc = fma(Dk[mm], src[mm * stride], acc);
                        du[v] = fma(s, acc, du[v]);
                    }
                }
            }
        }
        if (act) {
            double u[NV], S[NV];
            for (int v = 0; v < NV; ++v) u[v] = sU[v * nn + tid];
            if (KS) {
                sources_gen(u, jd, m, d.met, d.ndg, eb + tid, S);
                for (int v = 0; v < NV; ++v) du[v] += S[v];
            } else {
                du[0] -= jd[0]; du[1] -= jd[1]; du[2] -= jd[2];
                du[6] += u[8];
            }
        }
        // lift: one thread per face node
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
            PM mf;
            node_metric<KS>(d, p, mf);
            double nl[3];
            for (int i = 0; i < 3; ++i) nl[i] = (s ? 1.0 : -1.0) * d.geo[(int64_t)(3 * dd + i) * d.ndg + p];
            double nu[3];
            for (int i = 0; i < 3; ++i) nu[i] = fma(mf.gu[sym3(i, 0)], nl[0], fma(mf.gu[sym3(i, 1)], nl[1], mf.gu[sym3(i, 2)] * nl[2]));
            const double norm = sqrt(d3(nu, nl));
            const double inrm = 1.0 / norm;
            for (int i = 0; i < 3; ++i) nl[i] *= inrm;
            double Ui[NV], Ue[NV], Je[3];
            bool jx = false;   // exterior current given (FD neighbour), not J~(Ue)
            for (int v = 0; v < NV; ++v) Ui[v] = sU[v * nn + me];
            const int nb = d.nbr[e * 6 + f];
            if (nb >= 0) {
                int cn[3];
                nbr_node<P>(d, e, f, ta, tb, cn);
                if (d.mask[nb] == 0) {
                    const int64_t q = (int64_t)nb * d.nn + cn[0] + np1 * (cn[1] + np1 * cn[2]);
                    for (int v = 0; v < NV; ++v) Ue[v] = a.Uin.dg(v)[q];
                } else {
                    // FD->DG projection (6-point stencils) of the neighbour's cells and of
                    // their current J~ (the current of a projected state would carry its
                    // projection error in E~.B~ amplified by eta into the q~ flux)
                    // (from the face traces k_fd_traces left for it, indexed along
                    // the neighbour's own face axes)
                    jx = true;
                    const int f2 = d.nbr_face[e * 6 + f], d2 = f2 >> 1;
                    const int u1 = d2 == 0 ? 1 : 0, u2 = d2 == 2 ? 1 : 2;
                    const int nfm = d.np1 * d.np1;
                    const double* tr = d.ftr + ((int64_t)fd_slot_of(d, nb) * 6 + f2) * 12 * nfm + cn[u1] + np1 * cn[u2];
                    for (int v = 0; v < NV; ++v) Ue[v] = tr[v * nfm];
                    for (int q = 0; q < 3; ++q) Je[q] = tr[(NV + q) * nfm];
                }
            } else {
                const int kind = d.bc[e * 6 + f];
                if (kind == FFE_BC_DIRICHLET) {
                    const double* src = d.bdg + (int64_t)d.bface[e * 6 + f] * NV * nf;
                    for (int v = 0; v < NV; ++v) Ue[v] = src[v * nf + ta + np1 * tb];
                } else if (kind == FFE_BC_NO_INCOMING) {
                    if (KS) bc_no_incoming_gen(Ui, mf, nl, Ue);
                    else bc_no_incoming_flat(Ui, nl, Ue);
                } else if (kind == FFE_BC_OUTFLOW) {
                    for (int v = 0; v < NV; ++v) Ue[v] = Ui[v];
                } else {
                    double xn[3];
                    for (int q = 0; q < 3; ++q) xn[q] = d.xyz_dg[(int64_t)q * d.ndg + p];
                    bc_star_flat(Ui, xn, omega_of(d, e), Ue);
                }
            }
            const double lam = mf.a + fabs(d3(mf.b, nl));
            const double sc = 0.5 * norm * w0inv;
            if (KS) {
                double Fe[3][NV], jde[3];
                if (jx) flux_gen(Ue, Je, mf, Fe);
                else fluxes_at<KS>(Ue, mf, d.eta, Fe, jde);
                for (int v = 0; v < NV; ++v) {
                    double dfn = 0.0;
                    for (int j = 0; j < 3; ++j) dfn = fma(nl[j], Fe[j][v] - sF[(j * NV + v) * nn + me], dfn);
                    sC[(f * NV + v) * nf + ab] = sc * fma(-lam, Ue[v] - Ui[v], dfn);
                }
            } else {
                // the flat flux is linear in (U, J~): F(Ue) - F(Ui) = F(Ue - Ui, Je - Ji),
                // Ji the node's stored current, Je the exterior one
                if (!jx) {
                    double jde[3];
                    current_flat(Ue, d.eta, jde, Je);
                }
                double dUv[NV], dJv[3], Fd[3][NV];
                for (int v = 0; v < NV; ++v) dUv[v] = Ue[v] - Ui[v];
                for (int i = 0; i < 3; ++i) dJv[i] = Je[i] - sF[i * nn + me];
                flux_gen(dUv, dJv, mf, Fd);
                for (int v = 0; v < NV; ++v) {
                    const double dfn = fma(nl[2], Fd[2][v], fma(nl[1], Fd[1][v], nl[0] * Fd[0][v]));
                    sC[(f * NV + v) * nf + ab] = sc * fma(-lam, dUv[v], dfn);
                }
            }
        }
        __syncthreads();
        if (act) {
            for (int dd = 0; dd < 3; ++dd) {
                const int t1 = dd == 0 ? 1 : 0, t2 = dd == 2 ? 1 : 2;
                const int ab = ci[t1] + np1 * ci[t2];
                if (ci[dd] == 0)
                    for (int v = 0; v < NV; ++v) du[v] -= sC[((2 * dd) * NV + v) * nf + ab];
                if (ci[dd] == P)
                    for (int v = 0; v < NV; ++v) du[v] -= sC[((2 * dd + 1) * NV + v) * nf + ab];
            }
        }
        if (SUB == SUB_RHS) {
            if (act)
                for (int v = 0; v < NV; ++v) a.Fout.dg(v)[eb + tid] = du[v];
            __syncthreads();
            return;
        }
        double u[NV];
        if (act) {
            if (SUB != SUB_C)
                for (int v = 0; v < NV; ++v) a.Fout.dg(v)[eb + tid] = du[v];
            if (KS) {
                // explicit part of the stage (the metric-aware solve and clamp follow the filter)
                const int gv[NG] = {0, 1, 2, 6, 7};
                for (int v = 0; v < NV; ++v) u[v] = a.un.dg(v)[eb + tid];
                if (SUB == SUB_A) {
                    for (int v = 0; v < NV; ++v) u[v] = fma(dt, du[v], u[v]);
                    for (int c = 0; c < NG; ++c) u[gv[c]] = fma(dt * (1.0 - IM_A), a.G2.dg(c)[eb + tid], u[gv[c]]);
                } else if (SUB == SUB_B) {
                    for (int v = 0; v < NV; ++v) u[v] = fma(0.25 * dt, a.F2.dg(v)[eb + tid] + du[v], u[v]);
                    const double z = 0.5 - IM_B - IM_H - IM_A;
                    for (int c = 0; c < NG; ++c)
                        u[gv[c]] = fma(dt, IM_B * a.G1.dg(c)[eb + tid] + IM_H * a.G2.dg(c)[eb + tid] + z * a.G3.dg(c)[eb + tid], u[gv[c]]);
                } else {
                    for (int v = 0; v < NV; ++v)
                        u[v] = fma(dt, (a.F2.dg(v)[eb + tid] + a.F3.dg(v)[eb + tid]) * (1.0 / 6.0) + du[v] * (2.0 / 3.0), u[v]);
                    for (int c = 0; c < NG; ++c)
                        u[gv[c]] = fma(dt, (a.G2.dg(c)[eb + tid] + a.G3.dg(c)[eb + tid]) * (1.0 / 6.0) + a.G4.dg(c)[eb + tid] * (2.0 / 3.0), u[gv[c]]);
                }
            } else {
                substep_explicit(d, SUB, du, eb + tid, false, a, dt, u);
            }
        }
        __syncthreads();
        if (d.filter_on) {
            if (act)
                for (int v = 0; v < NV; ++v) sU[v * nn + tid] = u[v];
            __syncthreads();
            filter_lowrank<P, NT>(T, sU);
            if (act)
                for (int v = 0; v < NV; ++v) u[v] = sU[v * nn + tid];
        }
        // implicit part after the filter; G at the stage value: G_s = (U_s - R~_s)/(dt a)
        if (act) {
            if (KS) {
                if (SUB != SUB_C && !stiff_solve_gen(u, m, d, dt * IM_A)) atomic_status(d, 2);
                if (d.mode != FFE_RELAX) hard_clamp_gen(u, m);
            } else {
                substep_implicit(d, SUB, dt, u);
            }
            if (SUB != SUB_C) {
                double g[NG];
                if (KS) implicit_G_gen(u, m, d, g);
                else implicit_G_flat(u, d, g);
                for (int c = 0; c < NG; ++c) a.Gout.dg(c)[eb + tid] = g[c];
            }
        }
        bool flagged = false;
        if (d.tci_on) {
            double mag = 0.0;
            if (act) mag = KS ? bnorm_gen(u, m) : sqrt(fma(u[5], u[5], fma(u[4], u[4], u[3] * u[3])));
            if (act) sU[tid] = mag;
            __syncthreads();
            double low = 0.0;
            for (int k = 0; k < 3; ++k) {
                const int stride = k == 0 ? 1 : (k == 1 ? np1 : np1 * np1);
                if (act) {
                    const int base = tid - ci[k] * stride;
                    double acc = 0.0;
                    for (int mm = 0; mm < np1; ++mm) acc = fma(T.Pi[ci[k]][mm], sU[k * nn + base + mm * stride], acc);
                    if (k < 2) sU[(k + 1) * nn + tid] = acc;
                    else low = acc;
                }
                __syncthreads();
            }
            double num = 0.0, den = 0.0;
            if (act) {
                const double uh = mag - low;
                num = uh * uh;
                den = mag * mag;
            }
            block_sum2c<NW>(num, den, red);
            const double ratio = den > 0.0 ? sqrt(num / den) : 0.0;
            const double thr = d.thr_dgP[P];
            if (tid == 0) {
                int fl = ratio > thr;
                if (fabs(ratio - thr) <= 1e-12 * thr) d.near_list[atomicAdd(&d.counts[3], 1) & 4095] = e;
                if (fl && take_fd_slot(d, e)) {
                    d.flag_list[atomicAdd(&d.counts[2], 1)] = e;
                    d.switched[e] = 1;
                } else {
                    fl = 0;
                }
                red[2 * NW] = fl;
            }
            __syncthreads();
            flagged = red[2 * NW] != 0.0;
        }
        if (!flagged && tid == 0) {
            atomicAdd(d.units, (unsigned long long)nn);
            atomicAdd(d.units + 2, 1ull);
        }
        if (!flagged && act) {
            bool bad = false;
            for (int v = 0; v < NV; ++v) {
                a.Uout.dg(v)[eb + tid] = u[v];
                bad |= !isfinite(u[v]);
            }
            if (bad) atomic_status(d, 1);
        }
        __syncthreads();
    }
}


// Persistent kernel over a DG work list of order-P elements (list, count in
// d.counts[ci]); flat metric: two CTAs per SM (four for the 128-thread CTAs of
// orders <= 4; registers bounded accordingly), the metric-aware variant one.
// Batched contexts launch each order's elements separately, in CTAs sized for
// that order (one kernel dispatching on the order would keep every order's
// registers live and spill).
template <int P, int SUB, bool KS>
__global__ void __launch_bounds__(DGC<P>::NT, KS ? 1 : (DGC<P>::NT <= 128 ? 4 : 2))
    k_dg_curved(Dev d, SubArgs a, const int* list, int ci) {
    extern __shared__ double sm[];
    const int nwork = d.counts[ci];
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) dg_curved_elem<P, DGC<P>::NT, SUB, KS>(d, a, list[w], sm);
}

template <int P, bool KS, int SUB>
static void curved_launch(const Dev& d, const SubArgs& a, const int* list, int ci, int grid, cudaStream_t st) {
    using K = DGC<P>;
    cudaFuncSetAttribute(k_dg_curved<P, SUB, KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
    k_dg_curved<P, SUB, KS><<<grid, K::NT, K::SMEM, st>>>(d, a, list, ci);
    g_launch_counter += 1;
}

template <int P, bool KS, int SUB>
static void curved_dispatch_sub(const Dev& d, const SubArgs& a, cudaStream_t st) {
    const int grid = d.dg_grid > 0 ? d.dg_grid : d.nsm * 2;
    curved_launch<P, KS, SUB>(d, a, d.dg_list, 0, grid, st);
    // batches: the elements of orders P-1 and P-2, each in CTAs sized for their order
    if constexpr (P > 3) {
        if (d.dg_list_lo)
            curved_launch<P - 1, KS, SUB>(d, a, d.dg_list_lo, 6, d.dg_grid_lo > 0 ? d.dg_grid_lo : d.nsm * 4, st);
    }
    if constexpr (P > 4) {
        if (d.dg_list_lo2)
            curved_launch<P - 2, KS, SUB>(d, a, d.dg_list_lo2, 7, d.dg_grid_lo2 > 0 ? d.dg_grid_lo2 : d.nsm * 4, st);
    }
}

template <int P, bool KS>
static void curved_dispatch(const Dev& d, int sub, const SubArgs& a, cudaStream_t st) {
    switch (sub) {
        case SUB_A: curved_dispatch_sub<P, KS, SUB_A>(d, a, st); break;
        case SUB_B: curved_dispatch_sub<P, KS, SUB_B>(d, a, st); break;
        case SUB_C: curved_dispatch_sub<P, KS, SUB_C>(d, a, st); break;
        default: curved_dispatch_sub<P, KS, SUB_RHS>(d, a, st); break;
    }
}

void launch_dg_substep_curved(const Dev& d, int sub, Field Uin, Field J, Field un, Field F2, Field F3, Field G1,
                              Field G2, Field G3, Field G4, Field Fout, Field Uout, Field Gout, cudaStream_t st) {
    SubArgs a{Uin, J, un, F2, F3, G1, G2, G3, G4, Fout, Uout, Gout};
    if (!d.ks || d.metfd) launch_fd_traces(d, Uin, J, st);
    prof_begin(sub == SUB_RHS ? "dg_rhs_curved" : "dg_substep_curved", st);
    if (d.ks) {
        switch (d.P) {
            case 3: curved_dispatch<3, true>(d, sub, a, st); break;
            case 4: curved_dispatch<4, true>(d, sub, a, st); break;
            case 5: curved_dispatch<5, true>(d, sub, a, st); break;
            default: break;
        }
    } else {
        switch (d.P) {
            case 3: curved_dispatch<3, false>(d, sub, a, st); break;
            case 4: curved_dispatch<4, false>(d, sub, a, st); break;
            case 5: curved_dispatch<5, false>(d, sub, a, st); break;
            default: break;
        }
    }
    prof_end(st);
}

// Stages 1 and 2 at DG nodes with the Kerr-Schild metric (FD is flat-only).
__global__ void k_stage12_ks(Dev d, Field un, Field Ua, Field G1, Field G2) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const double dta = d.dt * IM_A;
    auto point = [&](const PM& m, double* u, double* g1, double* g2) {
        double U1[NV];
        for (int v = 0; v < NV; ++v) U1[v] = u[v];
        if (!stiff_solve_gen(U1, m, d, dta)) atomic_status(d, 2);
        if (d.mode != FFE_RELAX) hard_clamp_gen(U1, m);
        implicit_G_gen(U1, m, d, g1);
        u[0] = fma(-dta, g1[0], u[0]);
        u[1] = fma(-dta, g1[1], u[1]);
        u[2] = fma(-dta, g1[2], u[2]);
        u[6] = fma(-dta, g1[3], u[6]);
        u[7] = fma(-dta, g1[4], u[7]);
        if (!stiff_solve_gen(u, m, d, dta)) atomic_status(d, 2);
        if (d.mode != FFE_RELAX) hard_clamp_gen(u, m);
        implicit_G_gen(u, m, d, g2);
    };
    for (int64_t p = tid; p < d.ndg; p += stride) {
        if (d.mask[p / d.nn] != 0) continue;
        PM m;
        load_pm(d.met, d.ndg, p, m);
        double u[NV], g1[NG], g2[NG];
        for (int v = 0; v < NV; ++v) u[v] = un.dg(v)[p];
        point(m, u, g1, g2);
        for (int v = 0; v < NV; ++v) Ua.dg(v)[p] = u[v];
        for (int c = 0; c < NG; ++c) { G1.dg(c)[p] = g1[c]; G2.dg(c)[p] = g2[c]; }
    }
    // FD cells of the FD list, with the metric at the subcell centre
    const int64_t nfdq = (int64_t)d.counts[1] * d.ncell;
    for (int64_t q = tid; q < nfdq; q += stride) {
        const int e = d.fd_list[q / d.ncell];
        const int c = (int)(q % d.ncell);
        const int64_t p = fdb(d, e) + c;
        PM m;
        load_pm(d.metfd, (int64_t)d.E * d.ncell, (int64_t)e * d.ncell + c, m);
        double u[NV], g1[NG], g2[NG];
        for (int v = 0; v < NV; ++v) u[v] = un.fd(v)[p];
        point(m, u, g1, g2);
        for (int v = 0; v < NV; ++v) Ua.fd(v)[p] = u[v];
        for (int cg = 0; cg < NG; ++cg) { G1.fd(cg)[p] = g1[cg]; G2.fd(cg)[p] = g2[cg]; }
    }
}

void launch_stage12_ks(const Dev& d, Field un, Field Ua, Field G1, Field G2, cudaStream_t st) {
    prof_begin("stage12", st);
    k_stage12_ks<<<d.nsm * 8, 256, 0, st>>>(d, un, Ua, G1, G2);
    prof_end(st);
    g_launch_counter += 1;
}

}  // namespace ffe
