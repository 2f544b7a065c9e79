// IMEX-SSP3(4,3,3) substep arithmetic shared by the DG and FD kernels (Sec. III.B).
#pragma once
#include "ffe_internal.h"
#include "physics.cuh"

namespace ffe {

struct SubArgs {
    Field Uin, J, un, F2, F3, G1, G2, G3, G4, Fout, Uout, Gout;
};

__device__ __forceinline__ void atomic_status(const Dev& d, int bits) { atomicOr(&d.counts[4], bits); }

// Builds the substep result from the freshly computed explicit RHS f at point p:
//   SUB_A: R = u_n + dt F2 + dt (1-a) G2                       -> solve -> U3
//   SUB_B: R = u_n + dt (F2 + F3)/4 + dt (b G1 + h G2 + z G3)   -> solve -> U4
//   SUB_C: u_{n+1} = u_n + dt ((F2 + F3)/6 + 2 F4/3 + (G2 + G3)/6 + 2 G4/3)
// followed by the algebraic clamp when the constraint mode asks for it.  DG
// kernels filter R between the explicit and the implicit part.
// Explicit part R of the substep (DG elements filter R before the implicit part).
__device__ __forceinline__ void substep_explicit(const Dev& d, int sub, const double* f, int64_t p, bool isfd,
                                                 const SubArgs& a, double dt, double* u) {
    auto ld = [&](const Field& F, int v) { return isfd ? F.fd(v)[p] : F.dg(v)[p]; };
    const int gv[NG] = {0, 1, 2, 6, 7};
    for (int v = 0; v < NV; ++v) u[v] = ld(a.un, v);
    if (sub == SUB_A) {
        for (int v = 0; v < NV; ++v) u[v] = fma(dt, f[v], u[v]);
        for (int c = 0; c < NG; ++c) u[gv[c]] = fma(dt * (1.0 - IM_A), ld(a.G2, c), u[gv[c]]);
    } else if (sub == SUB_B) {
        for (int v = 0; v < NV; ++v) u[v] = fma(0.25 * dt, ld(a.F2, v) + f[v], u[v]);
        const double z = 0.5 - IM_B - IM_H - IM_A;
        for (int c = 0; c < NG; ++c)
            u[gv[c]] = fma(dt, IM_B * ld(a.G1, c) + IM_H * ld(a.G2, c) + z * ld(a.G3, c), u[gv[c]]);
    } else {
        for (int v = 0; v < NV; ++v)
            u[v] = fma(dt, (ld(a.F2, v) + ld(a.F3, v)) * (1.0 / 6.0) + f[v] * (2.0 / 3.0), u[v]);
        for (int c = 0; c < NG; ++c)
            u[gv[c]] = fma(dt, (ld(a.G2, c) + ld(a.G3, c)) * (1.0 / 6.0) + ld(a.G4, c) * (2.0 / 3.0), u[gv[c]]);
    }
}

// Implicit part: stiff solve (stages 3, 4) and the algebraic clamp when asked for.
__device__ __forceinline__ void substep_implicit(const Dev& d, int sub, double dt, double* u) {
    if (sub != SUB_C) {
        if (!stiff_solve_flat(u, d, dt * IM_A)) atomic_status(d, 2);
    }
    if (d.mode != FFE_RELAX) hard_clamp_flat(u);
}

__device__ __forceinline__ void substep_combine(const Dev& d, int sub, const double* f, int64_t p, bool isfd,
                                                const SubArgs& a, double dt, double* u) {
    substep_explicit(d, sub, f, p, isfd, a, dt, u);
    substep_implicit(d, sub, dt, u);
}

// A DG element the indicator flags needs an FD slot.  Contexts with a slot
// pool take one from the free stack; when the pool is empty the element stays
// on DG and status bit 2 (value 4) is raised.  Called by one thread.
__device__ __forceinline__ bool take_fd_slot(const Dev& d, int e) {
    if (!d.fd_slot || d.fd_slot[e] >= 0) return true;
    int old = d.counts[5];
    while (old > 0) {
        const int prev = atomicCAS(&d.counts[5], old, old - 1);
        if (prev == old) break;
        old = prev;
    }
    if (old <= 0) {
        atomic_status(d, 4);
        return false;
    }
    const int sl = d.free_slots[old - 1];
    d.fd_slot[e] = sl;
    d.slot_elem[sl] = e;
    return true;
}

}  // namespace ffe
