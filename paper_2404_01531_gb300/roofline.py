"""Algorithmic FP64 operation counts of the hot kernels (FMA = 2 flops,
add/mul/div/sqrt = 1), counted from the operations the method defines, not
from the instructions the kernels happen to issue.  Used for the roofline
fraction: achieved = count x units per launch / launch time."""
import math


def fp64_peak_tflops(n_sm, sm_mhz):
    """FP64 peak from the unit counts and the clock: 2 FMA lanes per clock per
    SM x 2 flops x SMs x clock (152 SMs at 2070 MHz: the GB300's nominal
    1.25 TFLOP/s FP64)."""
    return 2 * 2 * n_sm * sm_mhz * 1e6 / 1e12


FP64_PEAK_TFLOPS = fp64_peak_tflops(152, 2070.0)   # the GB300's nominal figure


def filter_rank(P, a=36.0, b=50.0):
    """Modes the exponential filter sigma_m = exp(-a (m/P)^(2b)) damps by more
    than 1e-20: the rank of I - F along one axis as the DG kernels apply it."""
    return sum(1 for m in range(P + 1) if -math.expm1(-a * (m / P) ** (2 * b)) > 1e-20)


def dg_flops_per_node(P, sub, filter_on=True, tci_on=True, solve=True, a=36.0, b=50.0):
    """One DG node through k_dg_substep: volume term (27 directional (P+1)-point
    contractions), derivative combination and explicit sources, the lifted
    Rusanov correction (6 (P+1)^2 face nodes per (P+1)^3 nodes), the IMEX stage
    combination, the pointwise stiff solve and implicit operator (substeps A, B),
    the filter of 9 variables in its low-rank form (per axis and kept mode one
    (P+1)-point dot product per line and one FMA per node) and the indicator
    (|B|, 3 low-pass contractions, two sums).  sub: 0 (A), 1 (B), 2 (C)."""
    n = P + 1
    f = 27 * n * 2              # volume contractions
    f += 22                     # combination + sources
    f += 39 * 6 / n             # lift per face node, averaged per node
    f += (28, 57, 84)[sub]      # stage combination
    if sub != 2 and solve:
        f += 38 + 30            # stiff solve + implicit operator
    if filter_on:
        f += 3 * 2 * 2 * 9 * filter_rank(P, a, b)
    if tci_on:
        f += 6 + 3 * n * 2 + 5
    return f


WENO_FLOPS = 73                  # one WENO5-Z face value (3 candidates, 3 indicators, Z weights, 1 div)
FD_FLUX_FLOPS = 24 * WENO_FLOPS + 45 + 36   # 12 quantities x (L, R) + Rusanov + corrector
# MP5 value on its unlimited path: the 5-point interpolant (9), v_MP (4) and the
# bracketing test (3); the limited path adds data-dependent work not counted
MP5_FLOPS = 16
FD_FLUX_FLOPS_MP5 = 24 * MP5_FLOPS + 45 + 36


def fd_flux_flops(recon):
    """Algorithmic flops of one face of the FD flux kernel for the reconstruction (0 WENO5-Z, 1 MP5)."""
    return FD_FLUX_FLOPS_MP5 if recon == 1 else FD_FLUX_FLOPS


def fd_faces_per_element(P):
    nc = 2 * P + 1
    return 3 * (nc + 1) * nc * nc
