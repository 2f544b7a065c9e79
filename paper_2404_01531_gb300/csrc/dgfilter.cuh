// Exponential filter (Sec. III.A) of the 9 variables of one DG element held in
// shared memory, in its low-rank form.  Along each axis the 1-D filter is
//     V diag(sigma) V^-1 = I - sum_m (1 - sigma_m) P_m(x) (V^-1)_m,
// and only the modes with 1 - sigma_m > 1e-20 are kept (Tables::nfr of them:
// modes P-1 and P at P = 5 with a = 36, b = 50); the others move a nodal value
// by less than 1e-20 of the mode's coefficient.  Per axis one thread owns one
// (variable, line): it loads the line's P+1 values, forms every kept mode's
// projection from those unfiltered values, subtracts the modes' contributions
// and stores the line back, so an axis costs one barrier and no scratch.
// Equal to the dense tensor-product filter up to rounding; 2 nfr 9 instead of
// 9 (P+1) FMAs per node and axis (a filter that damps every mode above 0 costs
// 2 P 9, more than the dense form's 9 (P+1)).  nfr = 0 (nothing damped above
// 1e-20) leaves the fields unchanged.
#pragma once
#include "ffe_internal.h"

namespace ffe {

// sU: [NV][nn] the fields, filtered in place.  Every thread of the CTA calls it
// (it holds barriers); on entry sU must be complete (a barrier after the last
// write), on return it is filtered and visible to the whole CTA.
template <int P, int NT>
__device__ __forceinline__ void filter_lowrank(const Tables& T, double* sU) {
    constexpr int np1 = P + 1, nl = np1 * np1, nn = nl * np1;
    const int nfr = T.nfr;
    if (nfr == 0) return;
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
        const int stride = dd == 0 ? 1 : (dd == 1 ? np1 : nl);
        for (int q = threadIdx.x; q < NV * nl; q += NT) {
            const int v = q / nl, line = q - v * nl;
            const int base = dd == 0 ? np1 * line : (dd == 1 ? line % np1 + nl * (line / np1) : line);
            double* p = sU + v * nn + base;
            // x: the unfiltered line (every projection reads it), y: the filtered
            // line; a runtime loop over the kept modes (an unrolled loop over all
            // P+1 modes under a guard would issue the guarded-off FMAs)
            double x[np1], y[np1];
#pragma unroll
            for (int m = 0; m < np1; ++m) y[m] = x[m] = p[stride * m];
#pragma unroll 1
            for (int r = 0; r < nfr; ++r) {
                double c = 0.0;
#pragma unroll
                for (int m = 0; m < np1; ++m) c = fma(T.FrW[r][m], x[m], c);
#pragma unroll
                for (int m = 0; m < np1; ++m) y[m] = fma(-c, T.FrV[r][m], y[m]);
            }
#pragma unroll
            for (int m = 0; m < np1; ++m) p[stride * m] = y[m];
        }
        __syncthreads();
    }
}

}  // namespace ffe
