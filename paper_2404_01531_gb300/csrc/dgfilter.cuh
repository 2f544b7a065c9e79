// Exponential filter (Sec. III.A) of the 9 variables of one DG element held in
// shared memory, in its low-rank form.  Along each axis the 1-D filter is
//     V diag(sigma) V^-1 = I - sum_m (1 - sigma_m) P_m(x) (V^-1)_m,
// and only the modes with 1 - sigma_m > 1e-20 are kept (Tables::nfr of them:
// modes P-1 and P at P = 5 with a = 36, b = 50); the others move a nodal value
// by less than 1e-20 of the mode's coefficient.  Per axis: one dot product
// per (kept mode, variable, line) into sc, then every node subtracts its
// modes' contributions.  Equal to the dense tensor-product filter up to
// rounding; 2 nfr 9 instead of 9 (P+1) FMAs per node and axis (a filter that
// damps every mode above 0 costs 2 P 9, more than the dense form's 9 (P+1)).
// nfr = 0 (nothing damped above 1e-20) leaves the fields unchanged.
#pragma once
#include "ffe_internal.h"

namespace ffe {

// sU: [NV][nn] the fields, filtered in place (threads with act own a node);
// sc: scratch of nfr NV (P+1)^2 doubles (less than 9 (P+1)^3).  Every thread
// of the CTA calls it (it holds barriers).
template <int P, int NT>
__device__ __forceinline__ void filter_lowrank(const Tables& T, double* sU, double* sc, bool act) {
    constexpr int np1 = P + 1, nl = np1 * np1, nn = nl * np1;
    const int tid = threadIdx.x;
    const int nfr = T.nfr;
    if (nfr == 0) return;
    const int c0 = tid % np1, c1 = (tid / np1) % np1, c2 = tid / nl;
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
        const int stride = dd == 0 ? 1 : (dd == 1 ? np1 : nl);
        for (int q = tid; q < nfr * NV * nl; q += NT) {
            const int r = q / (NV * nl), rem = q - r * (NV * nl), v = rem / nl, line = rem - v * nl;
            const int base = dd == 0 ? np1 * line : (dd == 1 ? line % np1 + nl * (line / np1) : line);
            const double* src = sU + v * nn + base;
            double acc = 0.0;
#pragma unroll
            for (int m = 0; m < np1; ++m) acc = fma(T.FrW[r][m], src[stride * m], acc);
            sc[q] = acc;
        }
        __syncthreads();
        if (act) {
            const int line = dd == 0 ? c1 + np1 * c2 : (dd == 1 ? c0 + np1 * c2 : c0 + np1 * c1);
            const int i = dd == 0 ? c0 : (dd == 1 ? c1 : c2);
            for (int v = 0; v < NV; ++v) {
                double x = sU[v * nn + tid];
                for (int r = 0; r < nfr; ++r) x = fma(-sc[(r * NV + v) * nl + line], T.FrV[r][i], x);
                sU[v * nn + tid] = x;
            }
        }
        __syncthreads();
    }
}

}  // namespace ffe
