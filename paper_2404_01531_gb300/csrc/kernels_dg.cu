// DG-side kernels of libffe (flat metric, affine box elements).
//
// k_dg_substep fuses, per DG element (one CTA, one thread per LGL node):
//   volume term  -(d xi^k/d x^j) D_k F^j  (Sec. III.A, nodal DG-SEM),
//   the Rusanov boundary correction lifted with the lumped LGL mass (Sec. III.C.2 flux),
//   the explicit sources, the explicit part of the IMEX-SSP3(4,3,3) stage, the
//   exponential filter (Sec. III.A) of that explicit update, the pointwise stiff
//   solve (Sec. III.B), the optional algebraic clamp (Sec. II.B) and the
//   troubled-cell indicator (Sec. III.C.3).  Filtering before the solve keeps
//   every state the explicit right-hand side sees a solve output: a filter after
//   the solve re-creates a parallel E~ that the eta-current of the q~ flux
//   amplifies by eta (unstable for eta dt >> 1).
#include <cstdio>

#include "dgfilter.cuh"
#include "ffe_internal.h"
#include "physics.cuh"
#include "physics_gen.cuh"
#include "stage.cuh"

namespace ffe {

thread_local int64_t g_launch_counter = 0;

template <int P>
struct DGK {
    static constexpr int np1 = P + 1;
    static constexpr int nn = np1 * np1 * np1;
    static constexpr int nf = np1 * np1;
    static constexpr int NT = ((nn + 31) / 32) * 32;
    static constexpr int NW = NT / 32;
    // shared doubles: U[9][nn] | J[6][nn] + C[6][9][nf] (aliased by the filter buffer [9][nn]) | red[2][NW]
    // | D scaled by the element's d xi/d x, per axis [3][np1][np1]
    static constexpr int AUX = (6 * nn + 54 * nf) > 9 * nn ? (6 * nn + 54 * nf) : 9 * nn;
    static constexpr int SMEM = (9 * nn + AUX + 2 * NW + 3 * nf) * 8;
};

// ---------------------------------------------------------------------------
__global__ void k_build_lists(Dev d) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d.E) return;
    if (d.mask[e] != 0) d.fd_list[atomicAdd(&d.counts[1], 1)] = e;
    else if (!d.dg_list_lo || elem_P(d, e) == d.P) d.dg_list[atomicAdd(&d.counts[0], 1)] = e;
    else if (elem_P(d, e) == d.P - 1) d.dg_list_lo[atomicAdd(&d.counts[6], 1)] = e;
    else d.dg_list_lo2[atomicAdd(&d.counts[7], 1)] = e;
}

void launch_build_lists(const Dev& d, cudaStream_t st) {
    cudaMemsetAsync(d.counts, 0, 2 * sizeof(int), st);
    if (d.dg_list_lo) cudaMemsetAsync(d.counts + 6, 0, 2 * sizeof(int), st);
    prof_begin("build_lists", st);
    k_build_lists<<<(d.E + 255) / 256, 256, 0, st>>>(d);
    prof_end(st);
    g_launch_counter += 1;
}

// ---------------------------------------------------------------------------
// J~ (drift, full) at every DG node of DG elements and at the cells of the FD
// list (counts[1], as built by k_build_lists); with a list, only the FD cells
// of the listed elements.
__global__ void k_current(Dev d, Field U, Field J, const int* list, int count_index) {
    int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (list == nullptr) {
        for (int64_t p = tid; p < d.ndg; p += stride) {
            const int e = (int)(p / d.nn);
            if (d.mask[e] != 0 || (int)(p % d.nn) >= esz(d, e).nn) continue;
            double u[NV], jd[3], jf[3];
            for (int v = 0; v < NV; ++v) u[v] = U.dg(v)[p];
            if (d.ks) {
                PM m;
                load_pm(d.met, d.ndg, p, m);
                current_gen(u, m, d.eta, jd, jf);
            } else {
                current_flat(u, d.eta, jd, jf);
            }
            for (int c = 0; c < 3; ++c) { J.dg(c)[p] = jd[c]; J.dg(3 + c)[p] = jf[c]; }
        }
        list = d.fd_list;
        count_index = 1;
    }
    {
        const int n = d.counts[count_index];
        for (int64_t q = tid; q < (int64_t)n * d.ncell; q += stride) {
            const int e = list[q / d.ncell];
            const int c = (int)(q % d.ncell);
            if (d.mask[e] != 1 || c >= esz(d, e).ncell) continue;
            const int64_t p = fdb(d, e) + c;
            double u[NV], jd[3], jf[3];
            for (int v = 0; v < NV; ++v) u[v] = U.fd(v)[p];
            if (d.ks) {
                PM m;
                load_pm(d.metfd, (int64_t)d.E * d.ncell, (int64_t)e * d.ncell + c, m);
                current_gen(u, m, d.eta, jd, jf);
            } else {
                current_flat(u, d.eta, jd, jf);
            }
            for (int c2 = 0; c2 < 3; ++c2) { J.fd(c2)[p] = jd[c2]; J.fd(3 + c2)[p] = jf[c2]; }
        }
    }
}

void launch_current(const Dev& d, Field U, Field J, const int* list, int count_index, cudaStream_t st) {
    prof_begin("current", st);
    k_current<<<d.nsm * 8, 256, 0, st>>>(d, U, J, list, count_index);
    prof_end(st);
    g_launch_counter += 1;
}

// ---------------------------------------------------------------------------
// Stages 1 and 2 are pointwise: U1 = solve(u_n), G1 = G(U1); U2 = solve(u_n - dt a G1), G2 = G(U2).
// Over the DG nodes of DG elements and the cells of the FD list (built first).
__device__ __forceinline__ void stage12_point(const Dev& d, double dt, double* u, double* g1, double* g2) {
    const double dta = dt * IM_A;
    double U1[NV];
    for (int v = 0; v < NV; ++v) U1[v] = u[v];
    if (!stiff_solve_flat(U1, d, dta)) atomic_status(d, 2);
    if (d.mode != FFE_RELAX) hard_clamp_flat(U1);
    implicit_G_flat(U1, d, g1);
    u[0] = fma(-dta, g1[0], u[0]);
    u[1] = fma(-dta, g1[1], u[1]);
    u[2] = fma(-dta, g1[2], u[2]);
    u[6] = fma(-dta, g1[3], u[6]);
    u[7] = fma(-dta, g1[4], u[7]);
    if (!stiff_solve_flat(u, d, dta)) atomic_status(d, 2);
    if (d.mode != FFE_RELAX) hard_clamp_flat(u);
    implicit_G_flat(u, d, g2);
}

__global__ void k_stage12(Dev d, Field un, Field Ua, Field G1, Field G2) {
    int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = tid; p < d.ndg; p += stride) {
        const int e = (int)(p / d.nn);
        if (d.mask[e] != 0 || (int)(p % d.nn) >= esz(d, e).nn) continue;
        double u[NV], g1[NG], g2[NG];
        for (int v = 0; v < NV; ++v) u[v] = un.dg(v)[p];
        stage12_point(d, dt_of(d, e), u, g1, g2);
        for (int v = 0; v < NV; ++v) Ua.dg(v)[p] = u[v];
        for (int c = 0; c < NG; ++c) { G1.dg(c)[p] = g1[c]; G2.dg(c)[p] = g2[c]; }
    }
    // FD cells: the elements of the FD list only (an FD slot pool may be mostly empty)
    const int64_t nfdq = (int64_t)d.counts[1] * d.ncell;
    for (int64_t q = tid; q < nfdq; q += stride) {
        const int e = d.fd_list[q / d.ncell];
        const int c = (int)(q % d.ncell);
        if (c >= esz(d, e).ncell) continue;
        const int64_t p = fdb(d, e) + c;
        double u[NV], g1[NG], g2[NG];
        for (int v = 0; v < NV; ++v) u[v] = un.fd(v)[p];
        stage12_point(d, dt_of(d, e), u, g1, g2);
        for (int v = 0; v < NV; ++v) Ua.fd(v)[p] = u[v];
        for (int c = 0; c < NG; ++c) { G1.fd(c)[p] = g1[c]; G2.fd(c)[p] = g2[c]; }
    }
}

void launch_stage12(const Dev& d, Field un, Field Ua, Field G1, Field G2, cudaStream_t st) {
    prof_begin("stage12", st);
    k_stage12<<<d.nsm * 8, 256, 0, st>>>(d, un, Ua, G1, G2);
    prof_end(st);
    g_launch_counter += 1;
}

// Deterministic block sum of two values (warp shuffles, then warp 0 in order).
template <int NW>
__device__ __forceinline__ void block_sum2(double& x, double& y, double* red) {
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_down_sync(0xffffffffu, x, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { red[w] = x; red[NW + w] = y; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sx = 0.0, sy = 0.0;
        for (int i = 0; i < NW; ++i) { sx += red[i]; sy += red[NW + i]; }
        red[0] = sx; red[NW] = sy;
    }
    __syncthreads();
    x = red[0];
    y = red[NW];
}

// tangential node coordinates of face direction dd: t1 < t2 are the other two axes
__device__ __forceinline__ void face_axes(int dd, int& t1, int& t2) {
    t1 = dd == 0 ? 1 : 0;
    t2 = dd == 2 ? 1 : 2;
}

template <int P>
__device__ __forceinline__ int node_index(int c0, int c1, int c2) {
    constexpr int np1 = P + 1;
    return c0 + np1 * (c1 + np1 * c2);
}

// External state at face node (face f, tangential a, b) of element e for the DG lift.
template <int P>
__device__ void dg_external_state(const Dev& d, const SubArgs& a, int e, int f, int ta, int tb,
                                  const double* Ui, const double* xnode, double* Ue, double* Je) {
    constexpr int np1 = P + 1;
    constexpr int nn = np1 * np1 * np1;
    const Tables& T = *d.tab;
    int dd = f >> 1, s = f & 1;
    int t1, t2;
    face_axes(dd, t1, t2);
    int nb = d.nbr[e * 6 + f];
    double jd[3];
    if (nb >= 0) {
        int f2 = d.nbr_face[e * 6 + f];
        int c[3];
        c[f2 >> 1] = (f2 & 1) ? P : 0;
        c[t1] = ta;
        c[t2] = tb;
        if (d.mask[nb] == 0) {
            int64_t p = (int64_t)nb * nn + node_index<P>(c[0], c[1], c[2]);
            for (int v = 0; v < NV; ++v) Ue[v] = a.Uin.dg(v)[p];
            for (int q = 0; q < 3; ++q) Je[q] = a.J.dg(3 + q)[p];
            return;
        }
        // FD neighbour: its FD->DG projection evaluated at this node (6-point
        // stencils), for the state and for its current J~ (the current of the
        // projected state would carry the projection error of E~.B~ times eta),
        // from the face traces k_fd_traces left for it (same face axes: boxes)
        (void)T;
        const int nfm = d.np1 * d.np1;
        const double* tr = d.ftr + ((int64_t)fd_slot_of(d, nb) * 6 + f2) * 12 * nfm + ta + np1 * tb;
        for (int v = 0; v < NV; ++v) Ue[v] = tr[v * nfm];
        for (int q = 0; q < 3; ++q) Je[q] = tr[(NV + q) * nfm];
        return;
    }
    int kind = d.bc[e * 6 + f];
    if (kind == FFE_BC_DIRICHLET) {
        int bfs = d.bface[e * 6 + f];
        const double* src = d.bdg + (int64_t)bfs * NV * np1 * np1;
        for (int v = 0; v < NV; ++v) Ue[v] = src[v * np1 * np1 + ta + np1 * tb];
    } else if (kind == FFE_BC_NO_INCOMING) {
        double n[3] = {0.0, 0.0, 0.0};
        n[dd] = s ? 1.0 : -1.0;
        bc_no_incoming_flat(Ui, n, Ue);
    } else if (kind == FFE_BC_OUTFLOW) {
        for (int v = 0; v < NV; ++v) Ue[v] = Ui[v];
    } else {
        bc_star_flat(Ui, xnode, d.omega, Ue);
    }
    current_flat(Ue, d.eta, jd, Je);
}

template <int P, int SUB>
__global__ void __launch_bounds__(DGK<P>::NT, 3) k_dg_substep(Dev d, SubArgs a) {
    using K = DGK<P>;
    constexpr int np1 = K::np1, nn = K::nn, nf = K::nf, NT = K::NT, NW = K::NW;
    extern __shared__ double sm[];
    double* sU = sm;                 // [9][nn]
    double* sJ = sU + 9 * nn;        // [6][nn]
    double* sC = sJ + 6 * nn;        // [6][9][nf]
    double* red = sU + 9 * nn + K::AUX;
    double* sD = red + 2 * NW;       // [3][np1][np1]: (d xi^a/d x^a) D
    __shared__ int s_flag;
    const Tables& T = *d.tab;
    const int tid = threadIdx.x;
    const bool act = tid < nn;
    const int i = tid % np1, j = (tid / np1) % np1, k = tid / (np1 * np1);
    const double w0inv = 1.0 / T.w0;
    const int nwork = d.counts[0];
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        const int e = d.dg_list[w];
        const int64_t eb = (int64_t)e * nn;
        const double sx = d.ijac[3 * e], sy = d.ijac[3 * e + 1], sz = d.ijac[3 * e + 2];
        for (int t = tid; t < NV * nn; t += NT) sU[t] = a.Uin.dg(t / nn)[eb + t % nn];
        for (int t = tid; t < NJ * nn; t += NT) sJ[t] = a.J.dg(t / nn)[eb + t % nn];
        if (tid < 3 * nf) sD[tid] = (tid < nf ? sx : (tid < 2 * nf ? sy : sz)) * T.D[(tid % nf) / np1][tid % np1];
        __syncthreads();

        double du[NV];
        if (act) {
            const double* Dx = sD + np1 * i;
            const double* Dy = sD + nf + np1 * j;
            const double* Dz = sD + 2 * nf + np1 * k;
            const int ox = np1 * (j + np1 * k);   // x-line start
            const int oy = i + np1 * np1 * k;     // y-line start, stride np1
            const int oz = i + np1 * j;           // z-line start, stride np1^2
            auto U = [&](int v, int idx) { return sU[v * nn + idx]; };
            double eX = -sJ[0 * nn + tid], eY = -sJ[1 * nn + tid], eZ = -sJ[2 * nn + tid];
            double bX = 0.0, bY = 0.0, bZ = 0.0;
            double ps = U(8, tid), ph = 0.0, qq = 0.0;
#pragma unroll
            for (int m = 0; m < np1; ++m) {
                const int ix = ox + m, iy = oy + np1 * m, iz = oz + np1 * np1 * m;
                // E: curl B - grad psi
                eX = fma(Dy[m], U(5, iy), eX); eX = fma(-Dz[m], U(4, iz), eX); eX = fma(-Dx[m], U(6, ix), eX);
                eY = fma(Dz[m], U(3, iz), eY); eY = fma(-Dx[m], U(5, ix), eY); eY = fma(-Dy[m], U(6, iy), eY);
                eZ = fma(Dx[m], U(4, ix), eZ); eZ = fma(-Dy[m], U(3, iy), eZ); eZ = fma(-Dz[m], U(6, iz), eZ);
                // B: -curl E - grad phi
                bX = fma(-Dy[m], U(2, iy), bX); bX = fma(Dz[m], U(1, iz), bX); bX = fma(-Dx[m], U(7, ix), bX);
                bY = fma(-Dz[m], U(0, iz), bY); bY = fma(Dx[m], U(2, ix), bY); bY = fma(-Dy[m], U(7, iy), bY);
                bZ = fma(-Dx[m], U(1, ix), bZ); bZ = fma(Dy[m], U(0, iy), bZ); bZ = fma(-Dz[m], U(7, iz), bZ);
                // psi: -div E + q ; phi: -div B ; q: -div J
                ps = fma(-Dx[m], U(0, ix), ps); ps = fma(-Dy[m], U(1, iy), ps); ps = fma(-Dz[m], U(2, iz), ps);
                ph = fma(-Dx[m], U(3, ix), ph); ph = fma(-Dy[m], U(4, iy), ph); ph = fma(-Dz[m], U(5, iz), ph);
                qq = fma(-Dx[m], sJ[3 * nn + ix], qq); qq = fma(-Dy[m], sJ[4 * nn + iy], qq);
                qq = fma(-Dz[m], sJ[5 * nn + iz], qq);
            }
            du[0] = eX; du[1] = eY; du[2] = eZ; du[3] = bX; du[4] = bY; du[5] = bZ;
            du[6] = ps; du[7] = ph; du[8] = qq;
        }
        // lift: one thread per face node
        for (int t = tid; t < 6 * nf; t += NT) {
            const int f = t / nf, ab = t % nf, ta = ab % np1, tb = ab / np1;
            const int dd = f >> 1, s = f & 1;
            int t1, t2;
            face_axes(dd, t1, t2);
            int c[3];
            c[dd] = s ? P : 0;
            c[t1] = ta;
            c[t2] = tb;
            const int me = node_index<P>(c[0], c[1], c[2]);
            double Ui[NV], Ue[NV], Je[3], xn[3];
            for (int v = 0; v < NV; ++v) Ui[v] = sU[v * nn + me];
            if (d.nbr[e * 6 + f] < 0 && d.bc[e * 6 + f] == FFE_BC_STAR)
                for (int q = 0; q < 3; ++q) xn[q] = d.xyz_dg[(int64_t)q * d.ndg + eb + me];
            dg_external_state<P>(d, a, e, f, ta, tb, Ui, xn, Ue, Je);
            double dU[NV], dJ[3], dF[NV];
            for (int v = 0; v < NV; ++v) dU[v] = Ue[v] - Ui[v];
            for (int q = 0; q < 3; ++q) dJ[q] = Je[q] - sJ[(3 + q) * nn + me];
            flux_dir_flat(dU, dJ, dd, dF);
            const double sg = s ? 1.0 : -1.0;
            const double scale = 0.5 * d.ijac[3 * e + dd] * w0inv;   // |grad xi^d| / (2 w0)
            for (int v = 0; v < NV; ++v) sC[(f * NV + v) * nf + ab] = scale * fma(sg, dF[v], -dU[v]);
        }
        __syncthreads();
        if (act) {
            const int cc[3] = {i, j, k};
            for (int dd = 0; dd < 3; ++dd) {
                int t1, t2;
                face_axes(dd, t1, t2);
                const int ab = cc[t1] + np1 * cc[t2];
                if (cc[dd] == 0)
                    for (int v = 0; v < NV; ++v) du[v] -= sC[((2 * dd) * NV + v) * nf + ab];
                if (cc[dd] == P)
                    for (int v = 0; v < NV; ++v) du[v] -= sC[((2 * dd + 1) * NV + v) * nf + ab];
            }
        }
        if (SUB == SUB_RHS) {
            if (act)
                for (int v = 0; v < NV; ++v) a.Fout.dg(v)[eb + tid] = du[v];
            __syncthreads();
            continue;
        }
        double u[NV];
        if (act) {
            if (SUB != SUB_C)
                for (int v = 0; v < NV; ++v) a.Fout.dg(v)[eb + tid] = du[v];
            substep_explicit(d, SUB, du, eb + tid, false, a, d.dt, u);
        }
        __syncthreads();   // sU, sJ, sC are free from here on
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
            substep_implicit(d, SUB, d.dt, u);
            if (SUB != SUB_C) {
                double g[NG];
                implicit_G_flat(u, d, g);
                for (int c = 0; c < NG; ++c) a.Gout.dg(c)[eb + tid] = g[c];
            }
        }
        bool flagged = false;
        if (d.tci_on) {
            // u = |B~| ; u^ = u - (Pi x Pi x Pi) u ; ratio = sqrt(sum u^2 / sum u^)
            double mag = act ? sqrt(fma(u[5], u[5], fma(u[4], u[4], u[3] * u[3]))) : 0.0;
            if (act) sU[tid] = mag;
            __syncthreads();
            if (act) {
                const int ox = np1 * (j + np1 * k);
                double acc = 0.0;
                for (int m = 0; m < np1; ++m) acc = fma(T.Pi[i][m], sU[ox + m], acc);
                sU[nn + tid] = acc;
            }
            __syncthreads();
            if (act) {
                const int oy = i + np1 * np1 * k;
                double acc = 0.0;
                for (int m = 0; m < np1; ++m) acc = fma(T.Pi[j][m], sU[nn + oy + np1 * m], acc);
                sU[2 * nn + tid] = acc;
            }
            __syncthreads();
            double num = 0.0, den = 0.0;
            if (act) {
                const int oz = i + np1 * j;
                double acc = 0.0;
                for (int m = 0; m < np1; ++m) acc = fma(T.Pi[k][m], sU[2 * nn + oz + np1 * np1 * m], acc);
                const double uh = mag - acc;
                num = uh * uh;
                den = mag * mag;
            }
            block_sum2<NW>(num, den, red);
            const double ratio = den > 0.0 ? sqrt(num / den) : 0.0;
            if (tid == 0) {
                int fl = ratio > d.thr_dg;
                if (fabs(ratio - d.thr_dg) <= 1e-12 * d.thr_dg) d.near_list[atomicAdd(&d.counts[3], 1) & 4095] = e;
                if (fl && take_fd_slot(d, e)) {
                    d.flag_list[atomicAdd(&d.counts[2], 1)] = e;
                    d.switched[e] = 1;
                } else {
                    fl = 0;
                }
                s_flag = fl;
            }
            __syncthreads();
            flagged = s_flag != 0;
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

template <int P>
static void dg_sub_dispatch(const Dev& d, int sub, const SubArgs& a, cudaStream_t st) {
    using K = DGK<P>;
    const int grid = d.dg_grid > 0 ? d.dg_grid : d.nsm * 4;
    switch (sub) {
        case SUB_A:
            cudaFuncSetAttribute(k_dg_substep<P, SUB_A>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
            k_dg_substep<P, SUB_A><<<grid, K::NT, K::SMEM, st>>>(d, a);
            break;
        case SUB_B:
            cudaFuncSetAttribute(k_dg_substep<P, SUB_B>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
            k_dg_substep<P, SUB_B><<<grid, K::NT, K::SMEM, st>>>(d, a);
            break;
        case SUB_C:
            cudaFuncSetAttribute(k_dg_substep<P, SUB_C>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
            k_dg_substep<P, SUB_C><<<grid, K::NT, K::SMEM, st>>>(d, a);
            break;
        default:
            cudaFuncSetAttribute(k_dg_substep<P, SUB_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
            k_dg_substep<P, SUB_RHS><<<grid, K::NT, K::SMEM, st>>>(d, a);
    }
    g_launch_counter += 1;
}

void launch_dg_substep(const Dev& d, int sub, Field Uin, Field J, Field un, Field F2, Field F3,
                       Field G1, Field G2, Field G3, Field G4, Field Fout, Field Uout, Field Gout,
                       cudaStream_t st) {
    SubArgs a{Uin, J, un, F2, F3, G1, G2, G3, G4, Fout, Uout, Gout};
    launch_fd_traces(d, Uin, J, st);
    prof_begin(sub == SUB_RHS ? "dg_rhs" : "dg_substep", st);
    switch (d.P) {
        case 2: dg_sub_dispatch<2>(d, sub, a, st); break;
        case 3: dg_sub_dispatch<3>(d, sub, a, st); break;
        case 4: dg_sub_dispatch<4>(d, sub, a, st); break;
        case 5: dg_sub_dispatch<5>(d, sub, a, st); break;
        case 6: dg_sub_dispatch<6>(d, sub, a, st); break;
        default: break;
    }
    prof_end(st);
}

// ---------------------------------------------------------------------------
// Indicator ratio of the DG data of every element (diagnostic entry point).
__global__ void k_tci_ratio(Dev d, const double* Udg, double* ratio) {
    __shared__ double su[MAXNP * MAXNP * MAXNP * 3];
    __shared__ double red[2];
    for (int e = blockIdx.x; e < d.E; e += gridDim.x) {
        const ES es = esz(d, e);
        const Tables& T = d.tabs[es.P];
        const int np1 = es.np1, nn = es.nn;
        for (int t = threadIdx.x; t < nn; t += blockDim.x) {
            const int64_t p = (int64_t)e * d.nn + t;
            const double bx = Udg[3 * d.ndg + p], by = Udg[4 * d.ndg + p], bz = Udg[5 * d.ndg + p];
            su[t] = sqrt(fma(bz, bz, fma(by, by, bx * bx)));
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nn; t += blockDim.x) {
            const int i = t % np1, j = (t / np1) % np1, k = t / (np1 * np1);
            double acc = 0.0;
            for (int m = 0; m < np1; ++m) acc = fma(T.Pi[i][m], su[m + np1 * (j + np1 * k)], acc);
            su[nn + t] = acc;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nn; t += blockDim.x) {
            const int i = t % np1, j = (t / np1) % np1, k = t / (np1 * np1);
            double acc = 0.0;
            for (int m = 0; m < np1; ++m) acc = fma(T.Pi[j][m], su[nn + i + np1 * (m + np1 * k)], acc);
            su[2 * nn + t] = acc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double num = 0.0, den = 0.0;
            for (int t = 0; t < nn; ++t) {
                const int i = t % np1, j = (t / np1) % np1, k = t / (np1 * np1);
                double acc = 0.0;
                for (int m = 0; m < np1; ++m) acc = fma(T.Pi[k][m], su[2 * nn + i + np1 * (j + np1 * m)], acc);
                const double uh = su[t] - acc;
                num += uh * uh;
                den += su[t] * su[t];
            }
            red[0] = den > 0.0 ? sqrt(num / den) : 0.0;
            ratio[e] = red[0];
        }
        __syncthreads();
    }
}

void launch_tci_ratio(const Dev& d, const double* Udg, double* ratio, cudaStream_t st) {
    prof_begin("tci_ratio", st);
    k_tci_ratio<<<d.nsm * 4, 128, 0, st>>>(d, Udg, ratio);
    prof_end(st);
    g_launch_counter += 1;
}

// ---------------------------------------------------------------------------
// Pointwise constraint diagnostics of a state (flat metric, densitised fields):
// per block max |E~.B~|, min (B~^2 - E~^2), max |psi~|, max |phi~| over the DG
// nodes of DG elements and the cells of FD elements.
__device__ __forceinline__ void cons_point(const Field& U, bool fd, int64_t p, double* r) {
    double u[8];
    for (int v = 0; v < 8; ++v) u[v] = fd ? U.fd(v)[p] : U.dg(v)[p];
    const double EB = fma(u[2], u[5], fma(u[1], u[4], u[0] * u[3]));
    const double D = fma(u[5], u[5], fma(u[4], u[4], u[3] * u[3])) - fma(u[2], u[2], fma(u[1], u[1], u[0] * u[0]));
    r[0] = fmax(r[0], fabs(EB));
    r[1] = fmin(r[1], D);
    r[2] = fmax(r[2], fabs(u[6]));
    r[3] = fmax(r[3], fabs(u[7]));
}

__global__ void k_constraints(Dev d, Field U, double* part) {
    __shared__ double sr[4][256];
    double r[4] = {0.0, 1.0e308, 0.0, 0.0};
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = tid; p < d.ndg; p += stride) {
        const int e = (int)(p / d.nn);
        if (d.mask[e] == 0 && (int)(p % d.nn) < esz(d, e).nn) cons_point(U, false, p, r);
    }
    for (int64_t p = tid; p < d.nfd; p += stride) {
        const int sl = (int)(p / d.ncell);
        const int e = d.slot_elem ? d.slot_elem[sl] : sl;
        if (e >= 0 && d.mask[e] == 1 && (int)(p % d.ncell) < esz(d, e).ncell) cons_point(U, true, p, r);
    }
    for (int i = 0; i < 4; ++i) sr[i][threadIdx.x] = r[i];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sr[0][threadIdx.x] = fmax(sr[0][threadIdx.x], sr[0][threadIdx.x + o]);
            sr[1][threadIdx.x] = fmin(sr[1][threadIdx.x], sr[1][threadIdx.x + o]);
            sr[2][threadIdx.x] = fmax(sr[2][threadIdx.x], sr[2][threadIdx.x + o]);
            sr[3][threadIdx.x] = fmax(sr[3][threadIdx.x], sr[3][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int i = 0; i < 4; ++i) part[4 * blockIdx.x + i] = sr[i][0];
}

void launch_constraints(const Dev& d, Field U, double* part, int blocks, cudaStream_t st) {
    k_constraints<<<blocks, 256, 0, st>>>(d, U, part);
    g_launch_counter += 1;
}

// L2 error norm of Sec. IV.B.1 (Table II), sum part: per block the sum over
// the DG nodes of DG elements and the cells of FD elements of
// sum_{v0 <= v < v0 + nv} (U_v - R_v)^2, accumulated per thread in index
// order and reduced by a fixed tree (deterministic for a fixed grid).
__global__ void k_l2_err(Dev d, Field U, Field R, int v0, int nv, double* part) {
    __shared__ double sr[256];
    double acc = 0.0;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = tid; p < d.ndg; p += stride) {
        const int e = (int)(p / d.nn);
        if (d.mask[e] == 0 && (int)(p % d.nn) < esz(d, e).nn)
            for (int v = v0; v < v0 + nv; ++v) {
                const double df = U.dg(v)[p] - R.dg(v)[p];
                acc = fma(df, df, acc);
            }
    }
    for (int64_t p = tid; p < d.nfd; p += stride) {
        const int sl = (int)(p / d.ncell);
        const int e = d.slot_elem ? d.slot_elem[sl] : sl;
        if (e >= 0 && d.mask[e] == 1 && (int)(p % d.ncell) < esz(d, e).ncell)
            for (int v = v0; v < v0 + nv; ++v) {
                const double df = U.fd(v)[p] - R.fd(v)[p];
                acc = fma(df, df, acc);
            }
    }
    sr[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sr[threadIdx.x] += sr[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sr[0];
}

void launch_l2_err(const Dev& d, Field U, Field R, int v0, int nv, double* part, int blocks, cudaStream_t st) {
    k_l2_err<<<blocks, 256, 0, st>>>(d, U, R, v0, nv, part);
    g_launch_counter += 1;
}

}  // namespace ffe
