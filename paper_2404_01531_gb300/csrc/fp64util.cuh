// FP64 helpers shared by the pointwise physics and the WENO5-Z kernels.
#pragma once

namespace ffe {

// 1/d for a positive normal d whose reciprocal is normal: the hardware
// approximation rcp.approx.ftz.f64 refined by two Newton-Raphson steps for
// f(y) = 1/y - d, y <- y + y (1 - d y) (each squares the relative error; the
// residual 1 - d y is exact in one FMA when y is close to 1/d).  Within about
// one ulp of the rounded quotient (ffe_eval_recip exposes it for tests); used
// for the WENO5-Z weight denominators (positive sums bounded away from zero;
// for sums above 2^1022 the flushed reciprocal is 0, where the quotient it
// replaces would overflow for candidates above 4 in magnitude) and, through
// recip_any, for the pointwise physics.
__device__ __forceinline__ double recip_nr(double d) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
    double r = fma(-d, y, 1.0);
    y = fma(y, r, y);
    r = fma(-d, y, 1.0);
    return fma(y, r, y);
}

// 2^-floor(log2 x) for a positive normal x below 2^1022: x times it lies in
// [1, 2) and the product is exact (integer operations on the exponent field).
__device__ __forceinline__ double pow2_inv_scale(double x) {
    const long long e = __double_as_longlong(x) >> 52;
    return __longlong_as_double((2046LL - e) << 52);
}

// 1/x for any finite nonzero x: recip_nr inside the range where it is
// defined (2^-1000 < |x| < 2^1000), the IEEE quotient outside it.
__device__ __forceinline__ double recip_any(double x) {
    const double ax = fabs(x);
    if (ax > 9.33e-302 && ax < 1.07e301) return x > 0.0 ? recip_nr(x) : -recip_nr(-x);
    return 1.0 / x;
}

}  // namespace ffe
