"""Pointwise GRFFE physics in densitised variables (Sec. II).

State layout: U[v, ...] with v = 0..8 = (E~x, E~y, E~z, B~x, B~y, B~z, psi~, phi~, q~).
Metric: a `Metric` with alpha, beta^i, gamma_ij, gamma^ij, sqrt(gamma), d_j alpha,
d_j beta^i, gamma^jk Gamma^i_jk and K, each broadcastable against the spatial
shape.  Works for float64 and complex128 (complex-step derivatives): every
branch is taken on the real part.  Test infrastructure only.
"""
import numpy as np

NVAR = 9
LEVI = np.zeros((3, 3, 3))
for (_i, _j, _k), _s in {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1,
                         (0, 2, 1): -1, (2, 1, 0): -1, (1, 0, 2): -1}.items():
    LEVI[_i, _j, _k] = _s


def rpos(x):
    """Rectifier R(x) = max(x, 0) of the current (Sec. II.B), branch on Re(x)."""
    return np.where(np.real(x) > 0, x, 0 * x)


class Metric:
    """3+1 quantities of a static background (Sec. II.A)."""

    def __init__(self, alpha, beta, gl, gu, sqrtg, dalpha, dbeta, gtrace, K):
        self.alpha, self.beta, self.gl, self.gu, self.sqrtg = alpha, beta, gl, gu, sqrtg
        self.dalpha, self.dbeta, self.gtrace, self.K = dalpha, dbeta, gtrace, K

    def take(self, fn):
        """Apply an indexing function to the trailing spatial axes of every field."""
        def sub(a, nlead):
            a = np.asarray(a)
            if a.ndim <= nlead:
                return a
            lead = a.shape[:nlead]
            flat = a.reshape((-1,) + a.shape[nlead:])
            return np.stack([fn(flat[i]) for i in range(flat.shape[0])]).reshape(lead + fn(flat[0]).shape)
        return Metric(sub(self.alpha, 0) if np.ndim(self.alpha) else self.alpha,
                      sub(self.beta, 1), sub(self.gl, 2), sub(self.gu, 2),
                      sub(self.sqrtg, 0) if np.ndim(self.sqrtg) else self.sqrtg,
                      sub(self.dalpha, 1), sub(self.dbeta, 2), sub(self.gtrace, 1),
                      sub(self.K, 0) if np.ndim(self.K) else self.K)


def flat_metric():
    """Minkowski: alpha = 1, beta = 0, gamma_ij = delta_ij; shapes broadcast."""
    z3 = np.zeros((3,))
    I = np.eye(3)
    return Metric(np.float64(1.0), z3, I, I, np.float64(1.0), z3, np.zeros((3, 3)), z3, np.float64(0.0))


def _bc(a, ndim_lead, spatial_ndim):
    """Reshape a metric field so its leading index axes broadcast against
    arrays with `spatial_ndim` trailing spatial axes."""
    a = np.asarray(a)
    extra = spatial_ndim - (a.ndim - ndim_lead)
    return a.reshape(a.shape + (1,) * extra) if extra > 0 else a


def lower(v, m, sp):
    """v_i = gamma_ij v^j."""
    return np.einsum('ij...,j...->i...', _bc(m.gl, 2, sp), v)


def cross_lower(al, bl):
    """c^i = [ijk] a_j b_k (flat antisymmetric symbol on lowered components)."""
    return np.stack([al[1] * bl[2] - al[2] * bl[1],
                     al[2] * bl[0] - al[0] * bl[2],
                     al[0] * bl[1] - al[1] * bl[0]])


def current(U, m, eta):
    """Densitised current J~ = alpha sqrt(gamma) J split into the drift part and
    the eta (parallel + rectifier) part of the driver-term Ohm's law (Sec. II.B):
      J~_drift^i = alpha q~ [ijk] E~_j B~_k / (sqrt(gamma) B~^2)
      J~_eta^i   = alpha eta [ (E~.B~)/B~^2 B~^i + R(E~^2 - B~^2)/B~^2 E~^i ]
    [reading] J~ = 0 where B~^2 = 0."""
    sp = U.ndim - 1
    E, B, q = U[0:3], U[3:6], U[8]
    El, Bl = lower(E, m, sp), lower(B, m, sp)
    B2 = np.sum(Bl * B, axis=0)
    EB = np.sum(El * B, axis=0)
    E2 = np.sum(El * E, axis=0)
    zero = np.real(B2) == 0
    inv = 1.0 / np.where(zero, 1.0, B2)
    alpha, sqrtg = _bc(m.alpha, 0, sp), _bc(m.sqrtg, 0, sp)
    jd = alpha * q * cross_lower(El, Bl) * inv / sqrtg
    jp = alpha * eta * (EB * inv * B + rpos(E2 - B2) * inv * E)
    jd = np.where(zero, 0 * jd, jd)
    jp = np.where(zero, 0 * jp, jp)
    return jd, jp


def fluxes(U, J, m):
    """F^j of the conservative form (Sec. II.A, flux vector); returns F[j, v, ...]:
      F^j(E~^i) = -beta^j E~^i + alpha (gamma^ij psi~ - [ijk] B~_k / sqrt(gamma))
      F^j(B~^i) = -beta^j B~^i + alpha (gamma^ij phi~ + [ijk] E~_k / sqrt(gamma))
      F^j(psi~) = -beta^j psi~ + alpha E~^j
      F^j(phi~) = -beta^j phi~ + alpha B~^j
      F^j(q~)   = J~^j - beta^j q~
    with [ijk]/sqrt(gamma) the spatial Levi-Civita tensor n_d eps^{dijk} for the
    convention eps_{abcd} = sqrt(-g)[abcd], [0123] = +1 (Sec. I)."""
    sp = U.ndim - 1
    E, B, psi, phi, q = U[0:3], U[3:6], U[6], U[7], U[8]
    El, Bl = lower(E, m, sp), lower(B, m, sp)
    alpha, sqrtg = _bc(m.alpha, 0, sp), _bc(m.sqrtg, 0, sp)
    beta, gu = _bc(m.beta, 1, sp), _bc(m.gu, 2, sp)
    F = np.zeros((3, NVAR) + U.shape[1:], dtype=np.result_type(U, alpha, beta))
    for j in range(3):
        for i in range(3):
            epsB = sum(LEVI[i, j, k] * Bl[k] for k in range(3) if LEVI[i, j, k] != 0)
            epsE = sum(LEVI[i, j, k] * El[k] for k in range(3) if LEVI[i, j, k] != 0)
            F[j, i] = -beta[j] * E[i] + alpha * (gu[i, j] * psi - epsB / sqrtg)
            F[j, 3 + i] = -beta[j] * B[i] + alpha * (gu[i, j] * phi + epsE / sqrtg)
        F[j, 6] = -beta[j] * psi + alpha * E[j]
        F[j, 7] = -beta[j] * phi + alpha * B[j]
        F[j, 8] = J[j] - beta[j] * q
    return F


def sources_explicit(U, jdrift, m):
    """Explicit part of the source vector S (Sec. II.A, source vector):
      S(E~^i) = -J~_drift^i - E~^j d_j beta^i + psi~ (gamma^ij d_j alpha - alpha gamma^jk Gamma^i_jk)
      S(B~^i) = -B~^j d_j beta^i + phi~ (gamma^ij d_j alpha - alpha gamma^jk Gamma^i_jk)
      S(psi~) = E~^k d_k alpha + alpha q~ - alpha psi~ K
      S(phi~) = B~^k d_k alpha - alpha phi~ K
      S(q~)   = 0
    The eta part of -J~ and the damping -alpha kappa psi~, -alpha kappa phi~ are
    the implicit operator `implicit_G` (IMEX split, Sec. III.B)."""
    sp = U.ndim - 1
    E, B, psi, phi, q = U[0:3], U[3:6], U[6], U[7], U[8]
    alpha, K = _bc(m.alpha, 0, sp), _bc(m.K, 0, sp)
    da, db = _bc(m.dalpha, 1, sp), _bc(m.dbeta, 2, sp)
    gu, gt = _bc(m.gu, 2, sp), _bc(m.gtrace, 1, sp)
    S = np.zeros(U.shape, dtype=np.result_type(U, alpha, da))
    for i in range(3):
        coef = sum(gu[i, j] * da[j] for j in range(3)) - alpha * gt[i]
        S[i] = -jdrift[i] - sum(E[j] * db[j, i] for j in range(3)) + psi * coef
        S[3 + i] = -sum(B[j] * db[j, i] for j in range(3)) + phi * coef
    S[6] = sum(E[k] * da[k] for k in range(3)) + alpha * q - alpha * psi * K
    S[7] = sum(B[k] * da[k] for k in range(3)) - alpha * phi * K
    return S


def implicit_G(U, m, eta, kpsi, kphi):
    """Stiff operator of the IMEX split (Sec. III.B): G(E~) = -J~_eta,
    G(psi~) = -alpha kappa_psi psi~, G(phi~) = -alpha kappa_phi phi~, zero for B~, q~.
    [reading] the lapse multiplies the damping as in the source vector."""
    sp = U.ndim - 1
    alpha = _bc(m.alpha, 0, sp)
    _, jp = current(U, m, eta)
    G = np.zeros_like(U, dtype=np.result_type(U, jp))
    G[0:3] = -jp
    G[6] = -alpha * kpsi * U[6]
    G[7] = -alpha * kphi * U[7]
    return G


def stiff_solve(R, m, eta, kpsi, kphi, dt_a):
    """Solve U = R + dt_a G(U) pointwise (Sec. III.B implicit equations).

    B~, q~ are explicit: B~ = R_B.  psi~ = R_psi / (1 + alpha kappa_psi dt_a), same for phi~.
    For E~ with c = alpha eta dt_a: E = E* - c [ (E.B/B^2) B + R(E^2-B^2)/B^2 E ].
    Writing E* = E*_par + E*_perp along B (gamma inner product), any solution is
    E(s) = E*_perp/(1+s) + E*_par/(1+c+s) with s = c R(E^2-B^2)/B^2.  If
    |E(0)|^2 <= B^2 the answer is s = 0 (the paper's analytic case); otherwise
    g(s) = c (|E(s)|^2 - B^2)/B^2 - s is strictly decreasing with g(0) > 0 and the
    unique root is found by bisection to adjacent doubles ([reading]: the same root
    the paper's Newton-Raphson solve converges to).  For complex input the real
    root is refined by two complex Newton steps (complex-step derivatives)."""
    sp = R.ndim - 1
    alpha = _bc(m.alpha, 0, sp)
    U = R.copy()
    U[6] = R[6] / (1.0 + alpha * kpsi * dt_a)
    U[7] = R[7] / (1.0 + alpha * kphi * dt_a)
    if eta == 0:
        return U
    E, B = R[0:3], R[3:6]
    Bl = lower(B, m, sp)
    B2 = np.sum(Bl * B, axis=0)
    zero = np.real(B2) == 0
    B2s = np.where(zero, 1.0, B2)
    c = alpha * eta * dt_a * np.ones_like(np.real(B2))
    Epar = np.sum(lower(E, m, sp) * B, axis=0) / B2s * B
    Eperp = E - Epar
    gl = _bc(m.gl, 2, sp)

    def norm2(v):
        return np.einsum('ij...,i...,j...->...', gl, v, v)

    def E_of(s):
        return Eperp / (1 + s) + Epar / (1 + c + s)

    E0 = E_of(0.0 * c)
    need = (np.real(norm2(E0)) > np.real(B2)) & ~zero
    Enew = np.where(zero, E, E0)
    if np.any(need):
        idx = np.nonzero(need)
        ep, ea = Eperp[(slice(None),) + idx], Epar[(slice(None),) + idx]
        cc, b2 = c[idx], B2[idx]
        gli = np.broadcast_to(gl, (3, 3) + B2.shape)[(slice(None), slice(None)) + idx]
        p2 = np.real(np.einsum('ij...,i...,j...->...', gli, ep, ep))
        a2 = np.real(np.einsum('ij...,i...,j...->...', gli, ea, ea))
        cr, b2r = np.real(cc), np.real(b2)

        def g(s):
            return cr * (p2 / (1 + s) ** 2 + a2 / (1 + cr + s) ** 2 - b2r) / b2r - s
        lo = np.zeros_like(cr)
        hi = cr * (p2 + a2) / b2r + cr
        for _ in range(2000):
            mid = 0.5 * (lo + hi)
            done = (mid <= lo) | (mid >= hi)
            if np.all(done):
                break
            gm = g(mid)
            lo = np.where(~done & (gm > 0), mid, lo)
            hi = np.where(~done & (gm <= 0), mid, hi)
        s = np.where(np.abs(g(lo)) <= np.abs(g(hi)), lo, hi)
        if np.iscomplexobj(R):
            s = s.astype(np.complex128)
            p2c = np.einsum('ij...,i...,j...->...', gli, ep, ep)
            a2c = np.einsum('ij...,i...,j...->...', gli, ea, ea)
            for _ in range(2):
                gs = cc * (p2c / (1 + s) ** 2 + a2c / (1 + cc + s) ** 2 - b2) / b2 - s
                dg = cc * (-2 * p2c / (1 + s) ** 3 - 2 * a2c / (1 + cc + s) ** 3) / b2 - 1
                s = s - gs / dg
        Es = ep / (1 + s) + ea / (1 + cc + s)
        Enew[(slice(None),) + idx] = Es
    U[0:3] = Enew
    return U


def hard_clamp(U, m):
    """Algebraic force-free enforcement (Sec. II.B, conventional approach):
    E <- E - (E.B/B^2) B, then if E^2 > B^2, E <- E sqrt(B^2/E^2).
    [reading] E <- 0 where B^2 = 0."""
    sp = U.ndim - 1
    U = U.copy()
    E, B = U[0:3], U[3:6]
    Bl = lower(B, m, sp)
    B2 = np.sum(Bl * B, axis=0)
    zero = np.real(B2) == 0
    B2s = np.where(zero, 1.0, B2)
    E = E - np.sum(Bl * E, axis=0) / B2s * B
    E2 = np.sum(lower(E, m, sp) * E, axis=0)
    big = np.real(E2) > np.real(B2)
    E = np.where(big, E * np.sqrt(np.where(big, B2 / np.where(big, E2, 1.0), 1.0)), E)
    E = np.where(zero, 0 * E, E)
    U[0:3] = E
    return U


def bc_no_incoming_poynting(Uint, m, nlow):
    """Outer boundary state (Sec. III.D): copy E~, B~, q~ from the interior;
    E~_out = 0 where the Poynting flux points inward, S.n < 0 with
    S^i proportional to [ijk] E_j B_k and n the outward unit normal (lower index);
    psi~_out = phi~_out = 0."""
    sp = Uint.ndim - 1
    U = Uint.copy()
    El, Bl = lower(Uint[0:3], m, sp), lower(Uint[3:6], m, sp)
    Sn = np.sum(cross_lower(El, Bl) * nlow, axis=0)
    inward = np.real(Sn) < 0
    U[0:3] = np.where(inward, 0 * U[0:3], U[0:3])
    U[6] = 0 * U[6]
    U[7] = 0 * U[7]
    return U


def bc_star(Uint, xyz, omega):
    """Perfect-conductor rotating star as an inner boundary state (Sec. IV.C,
    ideal-MHD condition), flat space: B~_out = B~_int, E~_out = -v x B~ with
    v = Omega z^ x x, psi~_out = q~_out = 0 (fixed inside the paper's star),
    phi~_out = 0.  [reading] the paper overwrites E inside r <= R and lets B
    and phi evolve there; here r = R is the inner boundary, and its state sets
    the cleaning scalars to zero as the paper's outer boundary state does
    (Sec. III.D): taken from the interior, phi~ leaves the incoming
    divergence-cleaning wave of B without data, and a static dipole then
    grows at the star."""
    U = Uint.copy()
    x, y = xyz[0], xyz[1]
    v = np.stack([-omega * y, omega * x, 0 * x])
    B = Uint[3:6]
    U[0:3] = -cross_lower(v, B)
    U[6] = 0 * U[6]
    U[7] = 0 * U[7]
    U[8] = 0 * U[8]
    return U
