// FD ghost cells across the faces between cubed-sphere wedges (Sec. III.C.1,
// III.C.2), forward fill and reverse mode.
//
// Inside a wedge (and on boxes) a neighbour's subcells continue this
// element's grid lines, so its ghosts are the neighbour's cells (or, for a DG
// neighbour, its polynomial at its own subcell centres): k_fd_fill_ghosts.
// Across a face between two wedges the grid lines bend, and the neighbour's
// cells are not the points of this element's grid extended past the face.
// There every ghost cell takes the neighbour's data at the ghost centre of the
// extended grid, the sixth-order grid-to-grid transfer of Sec. III.C.1:
//   - ghost centre: this element's reference grid continued past the face
//     (xi_n = +-(1 + (g + 1/2) dxi)), mapped by its wedge map;
//   - the neighbour's reference coordinates of that point from the closed-form
//     inverse of the wedge map (gnomonic coordinates X = x_t1 / (s x_n),
//     Y = x_t2 / (s x_n), eta = (4/pi) atan X; the radius, shared by the two
//     wedges of one shell, keeps its logical coordinate);
//   - an FD neighbour: tensor-product 6-point Lagrange interpolation through
//     the 6 subcell centres nearest the point along each axis (the stencil
//     kept inside the element), of its state and of its cell currents J~ (the
//     current is transferred, as from a DG neighbour: the current of the
//     interpolated state would carry eta (E.B) of the interpolation error,
//     which a stiff eta = 1e5 turns into a charge that grows at wedge faces);
//   - a DG neighbour: its nodal polynomial of U and of its nodal current J~
//     evaluated at the point (as its ghosts are filled everywhere else).
// The geometry is static, so the host tabulates, per ghost, the stencils'
// first cells and weights and the LGL Lagrange weights (Dev::gst, gwf, gwl);
// the kernels only gather and multiply.  The cell currents are those of
// k_current (J.fd(3..5)), on the Kerr-Schild background with the metric at
// the neighbour's cell centres.
#include "ffe_internal.h"
#include "physics.cuh"
#include "physics_gen.cuh"
#include "shellmap.cuh"
#include "fd_common.cuh"
#include "adjoint_common.cuh"

namespace ffe {

namespace {

__device__ __forceinline__ int64_t ghost_off(int dd, int s, int nc, int g, int ta, int tb) {
    const int ne = nc + 2 * GH;
    int t1, t2;
    axes_of(dd, t1, t2);
    int c[3];
    c[dd] = s ? nc + GH + g : GH - 1 - g;
    c[t1] = ta + GH;
    c[t2] = tb + GH;
    return c[0] + (int64_t)ne * (c[1] + (int64_t)ne * c[2]);
}

}  // namespace

// One CTA per (chunk position, face between wedges); other faces are left to
// k_fd_fill_ghosts.  Dynamic shared memory: a DG neighbour's U and J~ [12][nn],
// or the box of an FD neighbour's cells that the face's stencils reach, with
// their U and J~ [12][box].
__global__ void k_fd_fill_ghosts_interp(Dev d, const int* list, int ci, int w0, Field U, Field J) {
    const int n = chunk_n(d, ci, w0);
    extern __shared__ double su[];
    for (int item = blockIdx.x; item < n * 6; item += gridDim.x) {
        const int wl = item / 6, f = item % 6;
        const int e = list[w0 + wl];
        if (!d.ginterp[e * 6 + f]) continue;
        const int nb = d.nbr[e * 6 + f];
        const ES es = esz(d, e);
        const int nc = es.nc, np1 = es.np1, nn = es.nn;
        const int dd = f >> 1, s = f & 1;
        const bool fdnb = d.mask[nb] == 1;
        const int nper = GH * nc * nc, ghn = GH * d.nc * d.nc;
        const int sl = d.gislot[e * 6 + f];
        const int* bx = d.gbox + 6 * sl;   // the neighbour cells the stencils reach
        const int bx0 = bx[3], bxy = bx[3] * bx[4], bvol = bx[3] * bx[4] * bx[5];
        if (!fdnb) {
            for (int t = threadIdx.x; t < NQ * nn; t += blockDim.x) {
                const int qv = t / nn;
                const int64_t pn = (int64_t)nb * d.nn + t % nn;
                su[t] = qv < NV ? U.dg(qv)[pn] : J.dg(3 + qv - NV)[pn];
            }
        } else {
            // the box of the neighbour's cells: state [9] and cell current J~ [3]
            const int64_t base = fdb(d, nb);
            for (int t = threadIdx.x; t < NQ * bvol; t += blockDim.x) {
                const int qv = t / bvol, r = t % bvol;
                const int cx = bx[0] + r % bx0, cy = bx[1] + (r / bx0) % bx[4], cz = bx[2] + r / bxy;
                const int64_t pc = base + cx + (int64_t)nc * (cy + (int64_t)nc * cz);
                su[t] = qv < NV ? U.fd(qv)[pc] : J.fd(3 + qv - NV)[pc];
            }
        }
        __syncthreads();
        if (fdnb) {
            // one thread per (ghost, group of three quantities: E~, B~, (psi~, phi~, q~),
            // J~): 216 FMAs per quantity
            for (int it = threadIdx.x; it < 4 * nper; it += blockDim.x) {
                const int t = it / 4, grp = it % 4;
                const int g = t / (nc * nc), ta = t % nc, tb = (t / nc) % nc;
                const int64_t og = ghost_off(dd, s, nc, g, ta, tb);
                const int64_t gi = (int64_t)sl * ghn + t;
                const int* st3 = d.gst + gi * 3;
                double wf[18];
                for (int m = 0; m < 18; ++m) wf[m] = d.gwf[gi * 18 + m];
                const int sa = st3[0] - bx[0], sb = st3[1] - bx[1], sc = st3[2] - bx[2];
                const double* s0 = su + (3 * grp) * bvol;
                double u0 = 0.0, u1 = 0.0, u2 = 0.0;
                for (int cz = 0; cz < 6; ++cz)
                    for (int cy = 0; cy < 6; ++cy) {
                        const double wzy = wf[12 + cz] * wf[6 + cy];
                        const int row = sa + bx0 * (sb + cy) + bxy * (sc + cz);
#pragma unroll
                        for (int cx = 0; cx < 6; ++cx) {
                            const double w = wzy * wf[cx];
                            u0 = fma(w, s0[row + cx], u0);
                            u1 = fma(w, s0[bvol + row + cx], u1);
                            u2 = fma(w, s0[2 * bvol + row + cx], u2);
                        }
                    }
                ext_at(d, 3 * grp, wl)[og] = u0;
                ext_at(d, 3 * grp + 1, wl)[og] = u1;
                ext_at(d, 3 * grp + 2, wl)[og] = u2;
            }
        } else {
            for (int t = threadIdx.x; t < nper; t += blockDim.x) {
                const int g = t / (nc * nc), ta = t % nc, tb = (t / nc) % nc;
                const int64_t og = ghost_off(dd, s, nc, g, ta, tb);
                const int64_t gi = (int64_t)sl * ghn + t;
                const double* la = d.gwl + gi * 3 * MAXNP;
                const double* lb = la + MAXNP;
                const double* lc = lb + MAXNP;
                for (int qv = 0; qv < NQ; ++qv) {
                    const double* a = su + qv * nn;
                    double acc = 0.0;
                    for (int k = 0; k < np1; ++k) {
                        double ak = 0.0;
                        for (int j = 0; j < np1; ++j) {
                            double aj = 0.0;
                            for (int i = 0; i < np1; ++i) aj = fma(la[i], a[i + np1 * (j + np1 * k)], aj);
                            ak = fma(lb[j], aj, ak);
                        }
                        acc = fma(lc[k], ak, acc);
                    }
                    ext_at(d, qv, wl)[og] = acc;
                }
            }
        }
        __syncthreads();
    }
}

size_t fd_interp_smem(const Dev& d) {
    const size_t a = (size_t)NQ * d.nn, b = (size_t)NQ * d.gbox_max;
    return (a > b ? a : b) * sizeof(double);
}

void launch_fd_fill_interp(const Dev& d, const int* list, int ci, int w0, Field U, Field J, cudaStream_t st) {
    if (!d.ginterp) return;
    const size_t smem = fd_interp_smem(d);
    cudaFuncSetAttribute(k_fd_fill_ghosts_interp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_fd_fill_ghosts_interp<<<d.nsm * 2, 256, smem, st>>>(d, list, ci, w0, U, J);
    g_launch_counter += 1;
}

// ---------------------------------------------------------------------------
// Reverse mode.  The ghosts of a face between wedges are linear in the
// neighbour's data U and J~: an FD neighbour's cells, or a DG neighbour's
// nodes (then J~(U) at each cell or node).  FD neighbour: the ghost adjoints
// go to shared memory, then one warp per ghost scatters its adjoint times its
// stencil weights into a shared-memory copy of the box of cells the face's
// stencils reach (its lanes on distinct entries, so no collisions within a
// warp); each cell of the box takes its J~ adjoint through J~(U) of that cell
// and is added to the neighbour's cells once.  DG neighbour: the ghost
// adjoints and LGL weights go to shared memory and each node gathers its
// share from every ghost, in ghost order.  Faces and elements meeting at one
// cell or node are summed with FP64 atomics.
// Shared layout: FD neighbour acc [12][box max] | ghost adjoints [12][nper]; DG neighbour gb [12][nper] | wts [nper][3][MAXNP].
size_t fdv_interp_smem(const Dev& d) {
    const size_t nper = (size_t)GH * d.nc * d.nc;
    const size_t dg = NQ * nper + nper * 3 * MAXNP, fd = (size_t)NQ * d.gbox_max + NQ * nper;
    return (dg > fd ? dg : fd) * sizeof(double);
}

__device__ __forceinline__ double* extb_ptr(const Dev& d, const double* extb, int q, int wl) {
    return (double*)extb + ((int64_t)q * d.chunk + wl) * ext_size(d);
}

__global__ void k_fdv_ghosts_interp(Dev d, const int* list, int ci, int w0, Field U, Field out, const double* extb) {
    const int n = chunk_n(d, ci, w0);
    extern __shared__ double sm[];
    const int nperm = GH * d.nc * d.nc;
    for (int item = blockIdx.x; item < n * 6; item += gridDim.x) {
        const int wl = item / 6, f = item % 6;
        const int e = list[w0 + wl];
        if (!d.ginterp[e * 6 + f]) continue;
        const int nb = d.nbr[e * 6 + f];
        const ES es = esz(d, e);
        const int nc = es.nc, np1 = es.np1, nn = es.nn;
        const int dd = f >> 1, s = f & 1;
        const bool fdnb = d.mask[nb] == 1;
        const int nper = GH * nc * nc;
        const int sl = d.gislot[e * 6 + f], ghn = GH * d.nc * d.nc;
        if (fdnb) {
            const int* bx = d.gbox + 6 * sl;
            const int bx0 = bx[3], bxy = bx[3] * bx[4], bvol = bx[3] * bx[4] * bx[5];
            double* acc = sm;                      // [12][bvol]
            double* gbv = acc + NQ * d.gbox_max;   // [12][nper]
            for (int t = threadIdx.x; t < NQ * bvol; t += blockDim.x) acc[t] = 0.0;
            for (int t = threadIdx.x; t < nper; t += blockDim.x) {
                const int g = t / (nc * nc), ta = t % nc, tb = (t / nc) % nc;
                const int64_t og = ghost_off(dd, s, nc, g, ta, tb);
                for (int qv = 0; qv < NQ; ++qv) gbv[qv * nperm + t] = extb_ptr(d, extb, qv, wl)[og];
            }
            __syncthreads();
            // one warp per ghost: its lanes take distinct (cell, variable) entries of
            // the stencil, so the shared-memory additions of a warp never collide
            const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
            for (int t = threadIdx.x >> 5; t < nper; t += nwarp) {
                const int64_t gi = (int64_t)sl * ghn + t;
                const int* st3 = d.gst + gi * 3;
                const double* wf = d.gwf + gi * 18;
                const int sa = st3[0] - bx[0], sb = st3[1] - bx[1], sc = st3[2] - bx[2];
                for (int en = lane; en < NQ * 216; en += 32) {
                    const int qv = en / 216, k = en % 216;
                    const int cx = k % 6, cy = (k / 6) % 6, cz = k / 36;
                    const double w = wf[12 + cz] * wf[6 + cy] * wf[cx];
                    atomicAdd(acc + qv * bvol + sa + cx + bx0 * (sb + cy) + bxy * (sc + cz), w * gbv[qv * nperm + t]);
                }
            }
            __syncthreads();
            // per box cell: the J~ adjoint through J~(U) of the cell, then into the neighbour
            const int64_t base = fdb(d, nb);
            for (int r = threadIdx.x; r < bvol; r += blockDim.x) {
                double ub[NV], jb[3];
                bool any = false;
                for (int v = 0; v < NV; ++v) {
                    ub[v] = acc[v * bvol + r];
                    any |= ub[v] != 0.0;
                }
                for (int k = 0; k < 3; ++k) {
                    jb[k] = acc[(NV + k) * bvol + r];
                    any |= jb[k] != 0.0;
                }
                if (!any) continue;
                const int cx = bx[0] + r % bx0, cy = bx[1] + (r / bx0) % bx[4], cz = bx[2] + r / bxy;
                const int64_t pc = base + cx + (int64_t)nc * (cy + (int64_t)nc * cz);
                double u[NV];
                for (int v = 0; v < NV; ++v) u[v] = U.fd(v)[pc];
                current_vjp(u, d.eta, jb, jb, ub);
                for (int v = 0; v < NV; ++v)
                    if (ub[v] != 0.0) atomicAdd(out.fd(v) + pc, ub[v]);
            }
        } else {
            double* gb = sm;                                   // [NQ][nper]
            double* wts = gb + NQ * nperm;                     // [nper][3][MAXNP]
            for (int t = threadIdx.x; t < nper; t += blockDim.x) {
                const int g = t / (nc * nc), ta = t % nc, tb = (t / nc) % nc;
                const int64_t og = ghost_off(dd, s, nc, g, ta, tb);
                const int64_t gi = (int64_t)sl * ghn + t;
                double* w = wts + (size_t)t * 3 * MAXNP;
                for (int a2 = 0; a2 < 3 * MAXNP; ++a2) w[a2] = d.gwl[gi * 3 * MAXNP + a2];
                for (int qv = 0; qv < NQ; ++qv) gb[qv * nperm + t] = extb_ptr(d, extb, qv, wl)[og];
            }
            __syncthreads();
            for (int node = threadIdx.x; node < nn; node += blockDim.x) {
                const int i = node % np1, j = (node / np1) % np1, k = node / (np1 * np1);
                double acc[NQ];
                for (int qv = 0; qv < NQ; ++qv) acc[qv] = 0.0;
                for (int t = 0; t < nper; ++t) {
                    const double* w = wts + (size_t)t * 3 * MAXNP;
                    const double wt = w[2 * MAXNP + k] * w[MAXNP + j] * w[i];
                    for (int qv = 0; qv < NQ; ++qv) acc[qv] = fma(wt, gb[qv * nperm + t], acc[qv]);
                }
                const int64_t pn = (int64_t)nb * d.nn + node;
                double u[NV], ub[NV];
                for (int v = 0; v < NV; ++v) {
                    u[v] = U.dg(v)[pn];
                    ub[v] = acc[v];
                }
                current_vjp(u, d.eta, acc + NV, acc + NV, ub);
                for (int v = 0; v < NV; ++v)
                    if (ub[v] != 0.0) atomicAdd(out.dg(v) + pn, ub[v]);
            }
        }
        __syncthreads();
    }
}

void launch_fdv_ghosts_interp(const Dev& d, const int* list, int ci, int w0, Field U, Field out, const double* extb,
                              cudaStream_t st) {
    if (!d.ginterp) return;
    const size_t smem = fdv_interp_smem(d);
    cudaFuncSetAttribute(k_fdv_ghosts_interp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_fdv_ghosts_interp<<<d.nsm * 2, 256, smem, st>>>(d, list, ci, w0, U, out, extb);
    g_launch_counter += 1;
}

}  // namespace ffe
