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
//     kept inside the element); the ghost current J~ is the current of the
//     interpolated state, as for every FD ghost;
//   - a DG neighbour: its nodal polynomial of U and of its nodal current J~
//     evaluated at the point (as its ghosts are filled everywhere else).
// The geometry is static, so the host tabulates, per ghost, the stencils'
// first cells and weights and the LGL Lagrange weights (Dev::gst, gwf, gwl);
// the kernels only gather and multiply.  On the Kerr-Schild background the
// ghost current takes the metric at the ghost centre (Dev::metgi).
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
// k_fd_fill_ghosts.  Dynamic shared memory: a DG neighbour's U and J~ [12][nn].
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
        if (!fdnb) {
            for (int t = threadIdx.x; t < NQ * nn; t += blockDim.x) {
                const int qv = t / nn;
                const int64_t pn = (int64_t)nb * d.nn + t % nn;
                su[t] = qv < NV ? U.dg(qv)[pn] : J.dg(3 + qv - NV)[pn];
            }
            __syncthreads();
        }
        const int nper = GH * nc * nc, ghn = GH * d.nc * d.nc;
        const int sl = d.gislot[e * 6 + f];
        for (int t = threadIdx.x; t < nper; t += blockDim.x) {
            const int g = t / (nc * nc), ta = t % nc, tb = (t / nc) % nc;
            const int64_t og = ghost_off(dd, s, nc, g, ta, tb);
            const int64_t gi = (int64_t)sl * ghn + t;
            if (fdnb) {
                const int* st3 = d.gst + gi * 3;
                const double* wf = d.gwf + gi * 18;
                const int sa = st3[0], sb = st3[1], sc = st3[2];
                const int64_t base = fdb(d, nb);
                double u[NV];
                for (int v = 0; v < NV; ++v) u[v] = 0.0;
                for (int cz = 0; cz < 6; ++cz)
                    for (int cy = 0; cy < 6; ++cy) {
                        const double wzy = wf[12 + cz] * wf[6 + cy];
                        const int64_t row = base + sa + (int64_t)nc * ((sb + cy) + (int64_t)nc * (sc + cz));
                        for (int cx = 0; cx < 6; ++cx) {
                            const double w = wzy * wf[cx];
                            for (int v = 0; v < NV; ++v) u[v] = fma(w, U.fd(v)[row + cx], u[v]);
                        }
                    }
                double jd[3], jf[3];
                if (d.ks) {
                    PM m;
                    load_pm(d.metgi + (int64_t)sl * NPM * GH * d.nc * d.nc, (int64_t)GH * d.nc * d.nc,
                            (int64_t)g * nc * nc + ta + nc * tb, m);
                    current_gen(u, m, d.eta, jd, jf);
                } else {
                    current_flat(u, d.eta, jd, jf);
                }
                for (int v = 0; v < NV; ++v) ext_at(d, v, wl)[og] = u[v];
                for (int k = 0; k < 3; ++k) ext_at(d, NV + k, wl)[og] = jf[k];
            } else {
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

size_t fd_interp_smem(const Dev& d) { return (size_t)NQ * d.nn * sizeof(double); }

void launch_fd_fill_interp(const Dev& d, const int* list, int ci, int w0, Field U, Field J, cudaStream_t st) {
    if (!d.ginterp) return;
    k_fd_fill_ghosts_interp<<<d.nsm * 2, 256, fd_interp_smem(d), st>>>(d, list, ci, w0, U, J);
    g_launch_counter += 1;
}

// ---------------------------------------------------------------------------
// Reverse mode.  The ghosts of a face between wedges are linear in the
// neighbour's data: an FD neighbour's cells (then J~ = J~(ghost state)), or a
// DG neighbour's nodal U and J~ (then J~(U) at each node).  Per face, the
// ghost adjoints and the interpolation weights go to shared memory, and each
// neighbour cell (or node) gathers its share from every ghost whose stencil
// holds it, in ghost order (deterministic within the face); faces and
// elements meeting at one cell are summed with FP64 atomics.
// Shared layout: gb [12][nper] | wts [nper][3][MAXNP] | st [nper][3] ints | box [6] ints
size_t fdv_interp_smem(const Dev& d) {
    const size_t nper = (size_t)GH * d.nc * d.nc;
    return (NQ * nper + nper * 3 * MAXNP) * sizeof(double) + (nper * 3 + 6) * sizeof(int);
}

__device__ __forceinline__ double* extb_ptr(const Dev& d, const double* extb, int q, int wl) {
    return (double*)extb + ((int64_t)q * d.chunk + wl) * ext_size(d);
}

__global__ void k_fdv_ghosts_interp(Dev d, const int* list, int ci, int w0, Field U, Field out, const double* extb) {
    const int n = chunk_n(d, ci, w0);
    extern __shared__ double sm[];
    const int nperm = GH * d.nc * d.nc;
    double* gb = sm;                                   // [NQ][nper]
    double* wts = gb + NQ * nperm;                     // [nper][3][MAXNP]
    int* sti = (int*)(wts + (size_t)nperm * 3 * MAXNP);  // [nper][3]
    int* box = sti + 3 * nperm;                        // lo[3], hi[3] of the stencil starts
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
        if (threadIdx.x < 3) {
            box[threadIdx.x] = nc;
            box[3 + threadIdx.x] = -1;
        }
        __syncthreads();
        const int sl = d.gislot[e * 6 + f], ghn = GH * d.nc * d.nc;
        for (int t = threadIdx.x; t < nper; t += blockDim.x) {
            const int g = t / (nc * nc), ta = t % nc, tb = (t / nc) % nc;
            const int64_t og = ghost_off(dd, s, nc, g, ta, tb);
            const int64_t gi = (int64_t)sl * ghn + t;
            double gq[NQ];
            for (int qv = 0; qv < NQ; ++qv) gq[qv] = extb_ptr(d, extb, qv, wl)[og];
            double* w = wts + (size_t)t * 3 * MAXNP;
            if (fdnb) {
                for (int a = 0; a < 3; ++a) {
                    const int st = d.gst[gi * 3 + a];
                    for (int m = 0; m < 6; ++m) w[a * MAXNP + m] = d.gwf[gi * 18 + 6 * a + m];
                    sti[3 * t + a] = st;
                    atomicMin(box + a, st);
                    atomicMax(box + 3 + a, st);
                }
                // the ghost current is J~ of the ghost state: chain rule at the ghost
                double u[NV], ub[NV];
                for (int v = 0; v < NV; ++v) {
                    u[v] = ext_at(d, v, wl)[og];
                    ub[v] = gq[v];
                }
                current_vjp(u, d.eta, gq + NV, gq + NV, ub);
                for (int v = 0; v < NV; ++v) gb[v * nperm + t] = ub[v];
            } else {
                for (int a = 0; a < 3 * MAXNP; ++a) w[a] = d.gwl[gi * 3 * MAXNP + a];
                for (int qv = 0; qv < NQ; ++qv) gb[qv * nperm + t] = gq[qv];
            }
        }
        __syncthreads();
        if (fdnb) {
            const int lo0 = box[0], lo1 = box[1], lo2 = box[2];
            const int nx = box[3] + 6 - lo0, ny = box[4] + 6 - lo1, nz = box[5] + 6 - lo2;
            const int64_t base = fdb(d, nb);
            for (int c = threadIdx.x; c < nx * ny * nz; c += blockDim.x) {
                const int cx = lo0 + c % nx, cy = lo1 + (c / nx) % ny, cz = lo2 + c / (nx * ny);
                double acc[NV];
                for (int v = 0; v < NV; ++v) acc[v] = 0.0;
                for (int t = 0; t < nper; ++t) {
                    const int ox = cx - sti[3 * t], oy = cy - sti[3 * t + 1], oz = cz - sti[3 * t + 2];
                    if ((unsigned)ox >= 6u || (unsigned)oy >= 6u || (unsigned)oz >= 6u) continue;
                    const double* w = wts + (size_t)t * 3 * MAXNP;
                    const double wt = w[2 * MAXNP + oz] * w[MAXNP + oy] * w[ox];
                    for (int v = 0; v < NV; ++v) acc[v] = fma(wt, gb[v * nperm + t], acc[v]);
                }
                const int64_t p = base + cx + (int64_t)nc * (cy + (int64_t)nc * cz);
                for (int v = 0; v < NV; ++v)
                    if (acc[v] != 0.0) atomicAdd(out.fd(v) + p, acc[v]);
            }
        } else {
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
