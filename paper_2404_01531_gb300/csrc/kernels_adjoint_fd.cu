// Reverse mode of the FD-subcell right-hand side on flat-metric shells
// (Sec. III.C.2), for a fixed DG/FD mask:
//   out += (d RHS_FD / d U)^T lambda  over every listed FD element.
// The forward operator of an FD element is: extended block of the 12
// quantities (U and J~ = J~(U)) with 3 ghost layers from FD neighbours
// (copies; interpolated across faces between wedges, k_fdv_ghosts_interp), DG neighbours (their polynomials of U and of the nodal J~ at the
// ghost subcell centres) or the boundary states; WENO5-Z left/right values at every face; Rusanov flux
// of every physical component with the unit face normal; optional 4th-order
// corrector with the cell-centred fluxes; flux difference with the inverse
// Jacobian at the cell centre; sources -J~_drift and q~.
//   k_fdv_faces   face-flux adjoints from the two cells' lambda, back through
//                 corrector, Rusanov and WENO5-Z into the extended-block adjoint
//   k_fdv_cells   interior positions of the extended-block adjoint (U and the
//                 current's chain rule) and the source terms, into out
//   k_fdv_ghosts  ghost positions: into the FD neighbour's cells, through the
//                 transposed DG -> FD evaluation (of U and of the nodal J~) into
//                 the DG neighbour's nodes, or through the boundary state into my
//                 outermost cells
// The faces' contributions to the extended-block adjoint are written per face
// (k_fdv_faces) and summed per cell in a fixed order (k_fdv_gather); where
// several elements meet in out (an element's cells, a neighbour's cells or
// nodes reached through ghosts) they are summed with FP64 atomics (the order
// of those additions, hence the last bits, may differ between runs).
#include "ffe_internal.h"
#include "physics.cuh"
#include "shellmap.cuh"
#include "fd_common.cuh"
#include "adjoint_common.cuh"

namespace ffe {

__device__ __forceinline__ double* extb_at(const Dev& d, double* extb, int q, int wl) {
    return extb + ((int64_t)q * d.chunk + wl) * ext_size(d);
}


// Per-face contributions to the extended-block adjoint: for face fi of
// direction k the adjoints of its 6 stencil cells, gb[k][q][wl][fi][0..5] (the
// stencil starts at extended index m along k); k_fdv_gather sums them per cell.
__device__ __forceinline__ double* gbuf_at(const Dev& d, double* gb, int k, int q, int wl) {
    return gb + (((int64_t)k * NQ + q) * d.chunk + wl) * nface(d) * 6;
}

__global__ void k_fdv_faces(Dev d, const int* list, int ci, int w0, Field L, double* gb) {
    const int n = chunk_n(d, ci, w0);
    const int64_t nfc = nface(d);
    const int64_t total = (int64_t)n * 3 * nfc;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int wl = (int)(q / (3 * nfc));
        const int k = (int)((q / nfc) % 3);
        const int64_t fi = q % nfc;
        const int e = list[w0 + wl];
        const int nc = esz(d, e).nc;
        int m, ta, tb;
        if (!face_coords(fi, nc, m, ta, tb)) continue;
        int t1, t2;
        axes_of(k, t1, t2);
        // unit normal at the face point
        const ShellPts sp = shell_pts(d, e, nc);
        double nh[3];
        shell_face_normal(sp, k, m, ta, tb, nh);
        // flux adjoints: the face is the right face of cell m-1 (du -= sc F) and
        // the left face of cell m (du += sc F)
        double Fb[3][NV];
        for (int j = 0; j < 3; ++j)
            for (int v = 0; v < NV; ++v) Fb[j][v] = 0.0;
        const int64_t fb = fdb(d, e);
        for (int side = 0; side < 2; ++side) {
            const int mc = m - 1 + side;
            if (mc < 0 || mc >= nc) continue;
            int cc[3];
            cc[k] = mc;
            cc[t1] = ta;
            cc[t2] = tb;
            double ij[3][3];
            shell_cell(sp, cc, ij, nullptr);
            const int64_t p = fb + cc[0] + nc * (cc[1] + nc * cc[2]);
            const double sgn = side ? 0.5 * nc : -0.5 * nc;
            for (int v = 0; v < NV; ++v) {
                const double l = L.fd(v)[p];
                for (int j = 0; j < 3; ++j) Fb[j][v] = fma(sgn * ij[k][j], l, Fb[j][v]);
            }
        }
        double ubL[NQ], ubR[NQ], ubm[NQ], ubp[NQ];
        for (int qq = 0; qq < NQ; ++qq) ubL[qq] = ubR[qq] = ubm[qq] = ubp[qq] = 0.0;
        for (int j = 0; j < 3; ++j) {
            // corrector F = (4/3) F_rus - (F(U_m) + F(U_p))/6, then Rusanov
            double fr[NV], w[NV];
            for (int v = 0; v < NV; ++v) fr[v] = d.fd_corr ? (4.0 / 3.0) * Fb[j][v] : Fb[j][v];
            for (int v = 0; v < NV; ++v) w[v] = 0.5 * fr[v];
            flux_dir_t(j, w, ubL);
            flux_dir_t(j, w, ubR);
            for (int v = 0; v < NV; ++v) {
                ubL[v] = fma(0.5 * nh[j], fr[v], ubL[v]);
                ubR[v] = fma(-0.5 * nh[j], fr[v], ubR[v]);
            }
            if (d.fd_corr) {
                for (int v = 0; v < NV; ++v) w[v] = -Fb[j][v] * (1.0 / 6.0);
                flux_dir_t(j, w, ubm);
                flux_dir_t(j, w, ubp);
            }
        }
        // back through WENO5-Z into the extended-block adjoint
        const int ne = nc + 2 * GH;
        int c[3];
        c[k] = m;
        c[t1] = ta + GH;
        c[t2] = tb + GH;
        const int64_t base = c[0] + (int64_t)ne * (c[1] + (int64_t)ne * c[2]);
        const int64_t stride = k == 0 ? 1 : (k == 1 ? ne : (int64_t)ne * ne);
        for (int qq = 0; qq < NQ; ++qq) {
            const double* src = ext_at(d, qq, wl) + base;
            const double v0 = src[0], v1 = src[stride], v2 = src[2 * stride];
            const double v3 = src[3 * stride], v4 = src[4 * stride], v5 = src[5 * stride];
            double g[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            if (ubL[qq] != 0.0 || ubR[qq] != 0.0) weno5z_pair_vjp(v0, v1, v2, v3, v4, v5, d.weno_eps, ubL[qq], ubR[qq], g);
            g[2] += ubm[qq];
            g[3] += ubp[qq];
            double* dst = gbuf_at(d, gb, k, qq, wl) + fi * 6;
            for (int s = 0; s < 6; ++s) dst[s] = g[s];
        }
    }
}

// Extended-block adjoint of cell (x, y, z) and quantity q: the sum, over the
// three directions, of the contributions of the faces whose 6-cell stencil
// along that direction holds it (faces m = c_k - 5 .. c_k of the cell's line,
// the cell being stencil entry c_k - m); every position is written, no
// clearing, no atomics, a fixed order.
__global__ void k_fdv_gather(Dev d, const int* list, int ci, int w0, const double* gb, double* extb) {
    const int n = chunk_n(d, ci, w0);
    const int64_t ext = ext_size(d);
    const int64_t total = (int64_t)n * NQ * ext;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int wl = (int)(t / (NQ * ext));
        const int qq = (int)((t / ext) % NQ);
        const int64_t o = t % ext;
        const int e = list[w0 + wl];
        const int nc = esz(d, e).nc, ne = nc + 2 * GH;
        if (o >= (int64_t)ne * ne * ne) continue;
        const int c3[3] = {(int)(o % ne), (int)((o / ne) % ne), (int)(o / ((int64_t)ne * ne))};
        double acc = 0.0;
        for (int k = 0; k < 3; ++k) {
            int t1, t2;
            axes_of(k, t1, t2);
            const int ta = c3[t1] - GH, tb = c3[t2] - GH;
            if (ta < 0 || ta >= nc || tb < 0 || tb >= nc) continue;
            const double* g = gb + (((int64_t)k * NQ + qq) * d.chunk + wl) * nface(d) * 6;
            for (int sI = 0; sI < 6; ++sI) {
                const int m = c3[k] - sI;
                if (m < 0 || m > nc) continue;
                const int64_t fi = m + (int64_t)(nc + 1) * (ta + (int64_t)nc * tb);
                acc += g[fi * 6 + sI];
            }
        }
        extb_at(d, extb, qq, wl)[o] = acc;
    }
}

__global__ void k_fdv_cells(Dev d, const int* list, int ci, int w0, Field U, Field L, Field out, const double* extb) {
    const int n = chunk_n(d, ci, w0);
    const int64_t total = (int64_t)n * d.ncell;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int wl = (int)(q / d.ncell), c = (int)(q % d.ncell);
        const int e = list[w0 + wl];
        const ES es = esz(d, e);
        if (c >= es.ncell) continue;
        const int nc = es.nc, ne = nc + 2 * GH;
        const int x = c % nc, y = (c / nc) % nc, z = c / (nc * nc);
        const int64_t o = (x + GH) + ne * ((y + GH) + ne * (z + GH));
        const int64_t p = fdb(d, e) + c;
        double u[NV], ub[NV], jb[3];
        for (int v = 0; v < NV; ++v) {
            u[v] = U.fd(v)[p];
            ub[v] = extb_at(d, (double*)extb, v, wl)[o];
        }
        for (int k = 0; k < 3; ++k) jb[k] = extb_at(d, (double*)extb, NV + k, wl)[o];
        current_vjp(u, d.eta, jb, jb, ub);   // the extended block holds J~ = J~(U)
        const double wd[3] = {-L.fd(0)[p], -L.fd(1)[p], -L.fd(2)[p]}, zero[3] = {0.0, 0.0, 0.0};
        current_vjp(u, d.eta, wd, zero, ub);  // source -J~_drift
        ub[8] += L.fd(6)[p];                  // source q~ in the psi~ equation
        for (int v = 0; v < NV; ++v)
            if (ub[v] != 0.0) atomicAdd(out.fd(v) + p, ub[v]);
    }
}

// shared doubles for the DG-neighbour ghosts (U and J~): t1 [12][GH][np1][np1] |
// t2 [12][GH][np1][nc] | ub [12][GH][nc][nc]
size_t fdv_ghost_smem(const Dev& d) {
    return (size_t)(NQ * GH * d.np1 * d.np1 + NQ * GH * d.np1 * d.nc + NQ * GH * d.nc * d.nc) * sizeof(double);
}

__global__ void k_fdv_ghosts(Dev d, const int* list, int ci, int w0, Field U, Field J, Field out,
                             const double* extb, double* omega_bar) {
    const int n = chunk_n(d, ci, w0);
    extern __shared__ double sm[];
    __shared__ double s_om[256];
    double om_acc = 0.0;
    for (int item = blockIdx.x; item < n * 6; item += gridDim.x) {
        const int wl = item / 6, f = item % 6;
        const int e = list[w0 + wl];
        if (d.ginterp && d.ginterp[e * 6 + f]) continue;   // k_fdv_ghosts_interp
        const ES es = esz(d, e);
        const Tables& T = d.tabs[es.P];
        const int nc = es.nc, ne = nc + 2 * GH, np1 = es.np1, nn = es.nn;
        const int dd = f >> 1, s = f & 1;
        int t1, t2;
        axes_of(dd, t1, t2);
        const int nb = d.nbr[e * 6 + f];
        const int nper = GH * nc * nc;
        auto ghost_offset = [&](int g, int ta, int tb) -> int64_t {
            int c[3];
            c[dd] = s ? nc + GH + g : GH - 1 - g;
            c[t1] = ta + GH;
            c[t2] = tb + GH;
            return c[0] + (int64_t)ne * (c[1] + (int64_t)ne * c[2]);
        };
        auto ghost_bar = [&](int64_t og, const double* u, double* ub) {
            double jb[3];
            for (int v = 0; v < NV; ++v) ub[v] = extb_at(d, (double*)extb, v, wl)[og];
            for (int k = 0; k < 3; ++k) jb[k] = extb_at(d, (double*)extb, NV + k, wl)[og];
            current_vjp(u, d.eta, jb, jb, ub);
        };
        if (nb >= 0 && d.mask[nb] == 1) {
            const int f2 = d.nbr_face[e * 6 + f];
            const int d2 = f2 >> 1, s2 = f2 & 1;
            int u1, u2;
            axes_of(d2, u1, u2);
            const int o = d.orient[e * 6 + f];
            const int64_t nbase = fdb(d, nb);
            for (int t = threadIdx.x; t < nper; t += blockDim.x) {
                const int g = t / (nc * nc), ta = t % nc, tb = (t / nc) % nc;
                int a2, b2;
                orient_map(o, nc, ta, tb, a2, b2);
                int c[3];
                c[d2] = s2 ? nc - 1 - g : g;
                c[u1] = a2;
                c[u2] = b2;
                const int64_t p = nbase + c[0] + nc * (c[1] + nc * c[2]);
                double u[NV], ub[NV];
                for (int v = 0; v < NV; ++v) u[v] = U.fd(v)[p];
                ghost_bar(ghost_offset(g, ta, tb), u, ub);
                for (int v = 0; v < NV; ++v)
                    if (ub[v] != 0.0) atomicAdd(out.fd(v) + p, ub[v]);
            }
        } else if (nb >= 0) {
            const int f2 = d.nbr_face[e * 6 + f];
            const int d2 = f2 >> 1, s2 = f2 & 1;
            int u1, u2;
            axes_of(d2, u1, u2);
            const int o = d.orient[e * 6 + f];
            double* t1b = sm;                          // [12][GH][np1][np1]
            double* t2b = t1b + NQ * GH * np1 * np1;   // [12][GH][np1][nc]
            double* ubo = t2b + NQ * GH * np1 * nc;    // [12][GH][nc (u2)][nc (u1)]
            // The ghosts hold the neighbour's polynomial of U and of its nodal J~ at
            // its subcell centres: linear in (U, J~) at its nodes.  Their adjoints go
            // back through the transposed evaluation, then through J~(U) at each node.
            for (int t = threadIdx.x; t < nper; t += blockDim.x) {
                const int g = t / (nc * nc), ta = t % nc, tb = (t / nc) % nc;
                int a2, b2;   // the neighbour's subcell (along u1, u2) under this ghost cell
                orient_map(o, nc, ta, tb, a2, b2);
                const int64_t og = ghost_offset(g, ta, tb);
                for (int v = 0; v < NQ; ++v)
                    ubo[((v * GH + g) * nc + b2) * nc + a2] = extb_at(d, (double*)extb, v, wl)[og];
            }
            __syncthreads();
            // ub -> t2-bar [v][g][m (u2 node)][a2 (u1 cell)]
            for (int t = threadIdx.x; t < NQ * GH * np1 * nc; t += blockDim.x) {
                const int v = t / (GH * np1 * nc), r = t % (GH * np1 * nc);
                const int g = r / (np1 * nc), mm = (r / nc) % np1, a2 = r % nc;
                double acc = 0.0;
                for (int b2 = 0; b2 < nc; ++b2) acc = fma(T.P2F[b2][mm], ubo[((v * GH + g) * nc + b2) * nc + a2], acc);
                t2b[((v * GH + g) * np1 + mm) * nc + a2] = acc;
            }
            __syncthreads();
            // t2-bar -> t1-bar [v][g][a2 (u2 node)][m (u1 node)]
            for (int t = threadIdx.x; t < NQ * GH * np1 * np1; t += blockDim.x) {
                const int v = t / (GH * np1 * np1), r = t % (GH * np1 * np1);
                const int g = r / (np1 * np1), a2 = (r / np1) % np1, mm = r % np1;
                double acc = 0.0;
                for (int ta = 0; ta < nc; ++ta) acc = fma(T.P2F[ta][mm], t2b[((v * GH + g) * np1 + a2) * nc + ta], acc);
                t1b[((v * GH + g) * np1 + a2) * np1 + mm] = acc;
            }
            __syncthreads();
            // t1-bar -> node adjoints of (U, J~), then J~(U) at the node
            for (int node = threadIdx.x; node < nn; node += blockDim.x) {
                const int cc[3] = {node % np1, (node / np1) % np1, node / (np1 * np1)};
                const int mm = cc[d2], a1 = cc[u1], a2 = cc[u2];
                double w[NQ];
                for (int v = 0; v < NQ; ++v) {
                    double acc = 0.0;
                    for (int g = 0; g < GH; ++g) {
                        const int cn = s2 ? nc - 1 - g : g;
                        acc = fma(T.P2F[cn][mm], t1b[((v * GH + g) * np1 + a2) * np1 + a1], acc);
                    }
                    w[v] = acc;
                }
                const int64_t pn = (int64_t)nb * d.nn + node;
                double u[NV], ub[NV];
                for (int v = 0; v < NV; ++v) { u[v] = U.dg(v)[pn]; ub[v] = w[v]; }
                current_vjp(u, d.eta, w + NV, w + NV, ub);
                for (int v = 0; v < NV; ++v)
                    if (ub[v] != 0.0) atomicAdd(out.dg(v) + pn, ub[v]);
            }
            __syncthreads();
        } else {
            const int kind = d.bc[e * 6 + f];
            if (kind != FFE_BC_STAR && kind != FFE_BC_NO_INCOMING) continue;
            for (int t = threadIdx.x; t < nper; t += blockDim.x) {
                const int g = t / (nc * nc), ta = t % nc, tb = (t / nc) % nc;
                int c[3];
                c[dd] = s ? nc - 1 : 0;
                c[t1] = ta;
                c[t2] = tb;
                const int64_t p = fdb(d, e) + c[0] + nc * (c[1] + nc * c[2]);
                double ui[NV], u[NV], ub[NV], ib[NV];
                for (int v = 0; v < NV; ++v) { ui[v] = U.fd(v)[p]; ib[v] = 0.0; }
                const ShellPts sp = shell_pts(d, e, nc);
                if (kind == FFE_BC_NO_INCOMING) {
                    double nrm[3];
                    shell_face_normal(sp, dd, s ? nc : 0, ta, tb, nrm);
                    if (!s)
                        for (int qd = 0; qd < 3; ++qd) nrm[qd] = -nrm[qd];
                    bc_no_incoming_flat(ui, nrm, u);
                    ghost_bar(ghost_offset(g, ta, tb), u, ub);
                    bc_no_incoming_vjp(ui, nrm, ub, ib);
                } else {
                    double x[3], ij[3][3];
                    shell_cell(sp, c, ij, x);
                    const double om = omega_of(d, e);
                    bc_star_flat(ui, x, om, u);
                    ghost_bar(ghost_offset(g, ta, tb), u, ub);
                    om_acc += bc_star_vjp(ui, x, om, ub, ib);
                }
                for (int v = 0; v < NV; ++v)
                    if (ib[v] != 0.0) atomicAdd(out.fd(v) + p, ib[v]);
            }
        }
    }
    // Omega-bar: block sum, one atomic per block
    s_om[threadIdx.x] = om_acc;
    __syncthreads();
    if (threadIdx.x == 0 && omega_bar) {
        double acc = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) acc += s_om[i];
        if (acc != 0.0) atomicAdd(omega_bar, acc);
    }
}

// Reverse of k_fd_traces: the adjoints the DG reverse mode left at the trace
// nodes of FD faces with a DG neighbour (Dev::ftr_b, [slot][6][12][np1^2]) go
// back through the transposed sum-factorised FD->DG projection -- the two
// tangential directions, then the normal one -- to the 6 cell layers next to
// the face, and through J~(U) at each of those cells, into out.  One CTA per
// (element, face); cells shared by two faces of one element or reached by the
// other FD terms meet in out through FP64 atomics.
__global__ void k_fd_traces_vjp(Dev d, Field U, Field out) {
    extern __shared__ double sm[];
    const int n = d.counts[1];
    const int nfm = d.np1 * d.np1;
    for (int item = blockIdx.x; item < n * 6; item += gridDim.x) {
        const int w = item / 6, f = item % 6;
        const int e = d.fd_list[w];
        const int nb = d.nbr[e * 6 + f];
        if (nb < 0 || d.mask[nb] != 0) continue;
        const ES es = esz(d, e);
        const int np1 = es.np1, nc = es.nc, nc2 = nc * nc;
        const Tables& T = d.tabs[es.P];
        const int dd = f >> 1;
        int t1, t2;
        axes_of(dd, t1, t2);
        const int cn = (f & 1) ? es.P : 0;
        const int lo = T.f2d_lo[cn];
        double* Ob = sm;                          // [12][np1 (t2)][np1 (t1)]
        double* Bb = Ob + NQ * np1 * np1;         // [12][nc (t2)][np1 (t1)]
        double* Ab = Bb + NQ * nc * np1;          // [12][nc (t2)][nc (t1)]
        const double* src = d.ftr_b + ((int64_t)fd_slot_of(d, e) * 6 + f) * NQ * nfm;
        for (int t = threadIdx.x; t < NQ * np1 * np1; t += blockDim.x) {
            const int q = t / (np1 * np1), r = t % (np1 * np1);
            Ob[t] = src[q * nfm + r];
        }
        __syncthreads();
        // t2 direction: Bb[q][b][i] = sum_j F2D[j][b] Ob[q][j][i] (F2D is zero off the stencils)
        for (int t = threadIdx.x; t < NQ * nc * np1; t += blockDim.x) {
            const int q = t / (nc * np1), r = t % (nc * np1);
            const int b = r / np1, i = r % np1;
            double acc = 0.0;
            for (int j = 0; j < np1; ++j) acc = fma(T.F2D[j][b], Ob[(q * np1 + j) * np1 + i], acc);
            Bb[t] = acc;
        }
        __syncthreads();
        // t1 direction: Ab[q][b][a] = sum_i F2D[i][a] Bb[q][b][i]
        for (int t = threadIdx.x; t < NQ * nc2; t += blockDim.x) {
            const int q = t / nc2, r = t % nc2;
            const int b = r / nc, a = r % nc;
            double acc = 0.0;
            for (int i = 0; i < np1; ++i) acc = fma(T.F2D[i][a], Bb[(q * nc + b) * np1 + i], acc);
            Ab[t] = acc;
        }
        __syncthreads();
        // normal direction and the current's chain rule, per cell of the 6 layers
        const int64_t base = fdb(d, e);
        for (int t = threadIdx.x; t < 6 * nc2; t += blockDim.x) {
            const int m = t / nc2, r = t % nc2;
            const double wn = T.F2D[cn][lo + m];
            int c[3];
            c[dd] = lo + m;
            c[t1] = r % nc;
            c[t2] = r / nc;
            const int64_t p = base + c[0] + nc * (c[1] + nc * c[2]);
            double u[NV], ub[NV], jb[3];
            for (int v = 0; v < NV; ++v) {
                u[v] = U.fd(v)[p];
                ub[v] = wn * Ab[v * nc2 + r];
            }
            for (int k = 0; k < 3; ++k) jb[k] = wn * Ab[(NV + k) * nc2 + r];
            current_vjp(u, d.eta, jb, jb, ub);
            for (int v = 0; v < NV; ++v)
                if (ub[v] != 0.0) atomicAdd(out.fd(v) + p, ub[v]);
        }
        __syncthreads();
    }
}

void launch_fd_traces_vjp(const Dev& d, Field U, Field out, cudaStream_t st) {
    if (!d.ftr_b) return;
    const size_t smem = (size_t)(NQ * d.np1 * d.np1 + NQ * d.nc * d.np1 + NQ * d.nc * d.nc) * sizeof(double);
    cudaFuncSetAttribute(k_fd_traces_vjp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    prof_begin("fd_traces_vjp", st);
    k_fd_traces_vjp<<<d.nsm * 2, 256, smem, st>>>(d, U, out);
    prof_end(st);
    g_launch_counter += 1;
}

// out (FD block) must be zeroed and the DG right-hand-side adjoint already
// written by the caller; J holds J~(U) at the FD cells (launch_current).
void launch_fd_rhs_vjp(const Dev& dc, Field U, Field J, Field L, Field out, double* extb, double* gb,
                       double* omega_bar, cudaStream_t st) {
    // chunks of at most FDV_CHUNK elements: the per-face contribution buffer gb
    // holds [3][12][FDV_CHUNK][faces][6] doubles
    Dev d = dc;
    d.chunk = d.chunk < FDV_CHUNK ? d.chunk : FDV_CHUNK;
    const size_t smem = fdv_ghost_smem(d);
    cudaFuncSetAttribute(k_fdv_ghosts, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int k = 0, nch = fd_chunks(d); k < nch; ++k) {
        const int w0 = k * d.chunk;
        prof_begin("fdv_fill", st);
        launch_fd_fill(d, d.fd_list, 1, w0, U, J, st);
        prof_end(st);
        prof_begin("fdv_faces", st);
        k_fdv_faces<<<d.nsm * 8, 128, 0, st>>>(d, d.fd_list, 1, w0, L, gb);
        prof_end(st);
        prof_begin("fdv_gather", st);
        k_fdv_gather<<<d.nsm * 8, 256, 0, st>>>(d, d.fd_list, 1, w0, gb, extb);
        prof_end(st);
        prof_begin("fdv_cells", st);
        k_fdv_cells<<<d.nsm * 8, 256, 0, st>>>(d, d.fd_list, 1, w0, U, L, out, extb);
        prof_end(st);
        prof_begin("fdv_ghosts", st);
        k_fdv_ghosts<<<d.nsm * 2, 256, smem, st>>>(d, d.fd_list, 1, w0, U, J, out, extb, omega_bar);
        launch_fdv_ghosts_interp(d, d.fd_list, 1, w0, U, out, extb, st);
        prof_end(st);
        g_launch_counter += 4;
    }
}

}  // namespace ffe
