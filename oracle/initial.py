"""Initial data and exact solutions (Sec. IV.A, IV.B, IV.C; App. A, C).
Functions map coordinates xyz (3, ...) to U (9, ...).  Test infrastructure only."""
import numpy as np


def fast_wave(xyz, amp=0.5, t=0.0):
    """Smooth fast wave: B = (1, b, 0), E = (0, 0, -b), b = 1 + amp sin(pi (x - t)).
    E.B = 0, B^2 - E^2 = 1, div E = 0 so q = 0 and J = 0; in flat space the exact
    solution is the translation Q(x, t) = Q(x - t, 0) (Sec. IV.A.1)."""
    x = xyz[0] - t
    b = 1.0 + amp * np.sin(np.pi * x)
    U = np.zeros((9,) + np.shape(x))
    U[3] = 1.0
    U[4] = b
    U[2] = -b
    return U


def breakdown(xyz):
    """Current-sheet data of the breakdown workload: B = (1, By, 0) with
    By = 1 (x < -0.1), -10 x (|x| < 0.1), -1 (x > 0.1); E = (0, 0, 0.5) for
    |x| < 0.1 and (0, 0, 1) outside; q = div E = 0."""
    x = xyz[0]
    U = np.zeros((9,) + np.shape(x))
    U[3] = 1.0
    U[4] = np.where(x < -0.1, 1.0, np.where(x > 0.1, -1.0, -10.0 * x))
    U[2] = np.where(np.abs(x) < 0.1, 0.5, 1.0)
    return U


def cleaning_mode(xyz, eps=1e-3):
    """B = (1 + eps sin(pi x), 0, 0), all else zero."""
    x = xyz[0]
    U = np.zeros((9,) + np.shape(x))
    U[3] = 1.0 + eps * np.sin(np.pi * x)
    return U


def fast_wave_kink(xyz, t=0.0):
    """Fast wave of the paper's 1-D tests (App. A, "Fast wave"): B = (1, b, 0),
    E = (0, 0, -b) with b = 1 (x < -0.1), 0.85 - 1.5 x (|x| < 0.1), 0.7
    (x > 0.1): a ramp between two kinks.  E.B = 0, B^2 - E^2 = 1, div E = 0
    (q = 0) and J = 0: a vacuum fast mode whose exact solution is the
    translation Q(x, t) = Q(x - t, 0) (Sec. IV.A.1)."""
    x = xyz[0] - t
    b = np.where(x < -0.1, 1.0, np.where(x > 0.1, 0.7, 0.85 - 1.5 * x))
    U = np.zeros((9,) + np.shape(x))
    U[3] = 1.0
    U[4] = b
    U[2] = -b
    return U


def alfven_stationary(xyz):
    """Stationary Alfven wave of the paper's 1-D tests (App. A, "Stationary
    Alfven wave"): B = (1, 1, b), E = (-b, 0, 1) with b = 1 (x < -0.1),
    1.15 + 0.15 sin(5 pi x) (|x| < 0.1), 1.3 (x > 0.1).  E.B = 0 and
    B^2 - E^2 = 1.  [reading] The paper lists E and B only; q~ is set by
    Gauss's law, q = div E = -db/dx = -0.75 pi cos(5 pi x) inside the layer
    (0 outside; continuous, since cos(+-pi/2) = 0)."""
    x = xyz[0]
    inside = np.abs(x) < 0.1
    b = np.where(x < -0.1, 1.0, np.where(x > 0.1, 1.3, 1.15 + 0.15 * np.sin(5.0 * np.pi * x)))
    U = np.zeros((9,) + np.shape(x))
    U[0] = -b
    U[2] = 1.0
    U[3] = 1.0
    U[4] = 1.0
    U[5] = b
    U[8] = np.where(inside, -0.75 * np.pi * np.cos(5.0 * np.pi * x), 0.0)
    return U


def breakdown_1d(xyz):
    """FFE breakdown of the paper's 1-D tests (App. A, "FFE breakdown"):
    B = (1, b, b), E = (0, 0.5, -0.5) with b = 1 (x < -0.1), -10 x (|x| < 0.1),
    -1 (x > 0.1).  E.B = 0 and div E = 0 (q = 0); B^2 - E^2 = 0.5 + 2 b^2 falls
    towards zero in the layer as the evolution proceeds."""
    x = xyz[0]
    b = np.where(x < -0.1, 1.0, np.where(x > 0.1, -1.0, -10.0 * x))
    U = np.zeros((9,) + np.shape(x))
    U[1] = 0.5
    U[2] = -0.5
    U[3] = 1.0
    U[4] = b
    U[5] = b
    return U


CS_H = 1e-30


def _cs_grad(fn, xyz):
    """d fn / d x^j by complex step; fn maps (3, ...) -> (n, ...); returns (3, n, ...)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    out = []
    for j in range(3):
        p = xyz.astype(np.complex128)
        p[j] = p[j] + 1j * CS_H
        out.append(np.imag(fn(p)) / CS_H)
    return np.stack(out)


def wald(xyz, M=1.0, a=0.9, B0=1.0, e=1.0):
    """Wald's stationary vacuum field (Sec. IV.B.1): A_b = (B0/2)[(d_phi)_b + 2a (d_t)_b]
    with the Killing vectors d_t = (1,0,0,0) and d_phi = (0,-y,x,0) of the
    Kerr-Schild chart, F_ab = d_a A_b - d_b A_a (stationary: d_t A = 0),
    E^i = F^{ib} n_b = -alpha F^{i0}, B~^i = sqrt(gamma) B^i = [ijk] d_j A_k,
    E~ = sqrt(gamma) E; q~ = 0 (vacuum).  e multiplies E~ (e = 0: the vacuum
    Wald problem's start, Wald's magnetic field with E~ = 0, Sec. IV.B.2)."""
    from .metric import ks_four_metric, adm_from_four

    def A(p):
        g = ks_four_metric(p, M, a)
        x, y = p[0], p[1]
        return 0.5 * B0 * np.stack([g[m, 1] * (-y) + g[m, 2] * x + 2.0 * a * g[m, 0] for m in range(4)])
    xyz = np.asarray(xyz, dtype=np.float64)
    dA = _cs_grad(A, xyz)                         # [j][mu] = d_j A_mu
    shape = xyz.shape[1:]
    F = np.zeros((4, 4) + shape)
    for j in range(3):
        F[0, j + 1] = -dA[j, 0]
        F[j + 1, 0] = dA[j, 0]
        for k in range(3):
            F[j + 1, k + 1] = dA[j, k + 1] - dA[k, j + 1]
    g = np.real(ks_four_metric(xyz, M, a))
    gi = np.moveaxis(np.linalg.inv(np.moveaxis(g, (0, 1), (-2, -1))), (-2, -1), (0, 1))
    alpha, _, gl, _ = adm_from_four(g)
    sqrtg = np.sqrt(np.linalg.det(np.moveaxis(gl, (0, 1), (-2, -1))))
    Fup0 = np.einsum('im...,n...,mn...->i...', gi[1:, :], gi[0, :], F)   # F^{i0}
    U = np.zeros((9,) + shape)
    U[0:3] = -e * alpha * sqrtg * Fup0
    U[3] = dA[1, 3] - dA[2, 2]
    U[4] = dA[2, 1] - dA[0, 3]
    U[5] = dA[0, 2] - dA[1, 1]
    return U


def dipole(xyz, mu=1.0, delta=0.1, chi=0.0):
    """Regularised dipole (Sec. IV.C): A = mu m x x / (r^2 + delta^2)^(3/2) with
    m = (sin chi, 0, cos chi) (the paper's A_phi for chi = 0), B~ = curl A in
    flat space; E = psi = phi = q = 0.  Complex (mu, chi) use the closed form
    of the curl (dipole_closed), pinned against this construction."""
    if np.iscomplexobj(np.asarray(mu)) or np.iscomplexobj(np.asarray(chi)):
        return dipole_closed(xyz, mu, delta, chi)
    m = np.array([np.sin(chi), 0.0, np.cos(chi)])

    def A(p):
        f = mu / (p[0] ** 2 + p[1] ** 2 + p[2] ** 2 + delta * delta) ** 1.5
        return np.stack([(m[1] * p[2] - m[2] * p[1]) * f, (m[2] * p[0] - m[0] * p[2]) * f,
                         (m[0] * p[1] - m[1] * p[0]) * f])
    dA = _cs_grad(A, xyz)
    U = np.zeros((9,) + np.shape(xyz)[1:])
    U[3] = dA[1, 2] - dA[2, 1]
    U[4] = dA[2, 0] - dA[0, 2]
    U[5] = dA[0, 1] - dA[1, 0]
    return U


def dipole_closed(xyz, mu=1.0, delta=0.1, chi=0.0):
    """curl of mu m x x / (r^2+delta^2)^(3/2):
    B~ = mu [3 x (m.x) - m (r^2 - 2 delta^2)] / (r^2 + delta^2)^(5/2)."""
    xyz = np.asarray(xyz)
    m = [np.sin(chi), 0.0 * chi, np.cos(chi)]
    r2 = xyz[0] ** 2 + xyz[1] ** 2 + xyz[2] ** 2
    mx = m[0] * xyz[0] + m[1] * xyz[1] + m[2] * xyz[2]
    f = mu / (r2 + delta * delta) ** 2.5
    U = np.zeros((9,) + np.shape(xyz)[1:], dtype=np.result_type(mu, chi, float))
    for i in range(3):
        U[3 + i] = f * (3 * xyz[i] * mx - m[i] * (r2 - 2 * delta * delta))
    return U


_KINDS = {"fast_wave": fast_wave, "breakdown": breakdown, "cleaning_mode": cleaning_mode,
          "wald": wald, "dipole": dipole, "fast_wave_kink": fast_wave_kink, "alfven": alfven_stationary,
          "breakdown_1d": breakdown_1d}


def evaluate(kind, xyz, **kw):
    return _KINDS[kind](xyz, **kw)
