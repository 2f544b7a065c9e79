"""Background metrics in 3+1 form (Sec. II.A) and their derivatives.
Kerr in Cartesian Kerr-Schild coordinates (App. B).  All derivatives are taken
by complex-step differentiation of the closed forms.  Test infrastructure only."""
import numpy as np

from .physics import Metric

CS_H = 1e-30


def ks_four_metric(xyz, M, a):
    """g_{mu nu} = eta + 2 H l_mu l_nu with H = M r^3/(r^4 + a^2 z^2),
    l = (1, (r x + a y)/(r^2+a^2), (r y - a x)/(r^2+a^2), z/r) and r from
    (x^2+y^2)/(r^2+a^2) + z^2/r^2 = 1 (App. B).  Works for complex xyz."""
    x, y, z = xyz[0], xyz[1], xyz[2]
    R2 = x * x + y * y + z * z
    r2 = 0.5 * (R2 - a * a + np.sqrt((R2 - a * a) ** 2 + 4.0 * a * a * z * z))
    r = np.sqrt(r2)
    H = M * r * r2 / (r2 * r2 + a * a * z * z)
    l = [np.ones_like(x), (r * x + a * y) / (r2 + a * a), (r * y - a * x) / (r2 + a * a), z / r]
    g = np.empty((4, 4) + np.shape(x), dtype=np.result_type(x, float))
    eta = np.diag([-1.0, 1.0, 1.0, 1.0])
    for m in range(4):
        for n in range(4):
            g[m, n] = eta[m, n] + 2.0 * H * l[m] * l[n]
    return g


def adm_from_four(g):
    """lapse, shift^i and gamma_ij from g_{mu nu}: gamma_ij = g_ij,
    beta_i = g_0i, beta^i = gamma^ij beta_j, alpha^2 = beta_i beta^i - g_00."""
    gl = g[1:, 1:]
    gu = np.moveaxis(np.linalg.inv(np.moveaxis(gl, (0, 1), (-2, -1))), (-2, -1), (0, 1))
    bl = g[0, 1:]
    bu = np.einsum('ij...,j...->i...', gu, bl)
    alpha = np.sqrt(np.einsum('i...,i...->...', bl, bu) - g[0, 0])
    return alpha, bu, gl, gu


def ks_metric(xyz, M, a):
    """Metric at points xyz (3, ...) with d_j alpha, d_j beta^i, gamma^jk Gamma^i_jk
    and K = gamma^ij K_ij, K_ij = (D_i beta_j + D_j beta_i)/(2 alpha) for the
    static metric (d_t gamma_ij = 0)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    alpha, bu, gl, gu = [np.real(q) for q in adm_from_four(ks_four_metric(xyz, M, a))]
    sqrtg = np.sqrt(np.linalg.det(np.moveaxis(gl, (0, 1), (-2, -1))))
    da, db, dg = [], [], []
    for k in range(3):
        p = xyz.astype(np.complex128)
        p[k] = p[k] + 1j * CS_H
        ak, bk, glk, _ = adm_from_four(ks_four_metric(p, M, a))
        da.append(np.imag(ak) / CS_H)
        db.append(np.imag(bk) / CS_H)
        dg.append(np.imag(glk) / CS_H)
    da = np.stack(da)                   # [j]
    db = np.stack(db)                   # [j][i] = d_j beta^i
    dg = np.stack(dg)                   # [k][i][j] = d_k gamma_ij
    # Christoffel symbols of gamma: Gamma^i_jk = 1/2 gamma^il (d_j g_lk + d_k g_lj - d_l g_jk)
    Gl = 0.5 * (np.einsum('jlk...->ljk...', dg) + np.einsum('klj...->ljk...', dg) - dg)  # [l][j][k]
    Gam = np.einsum('il...,ljk...->ijk...', gu, Gl)
    gtrace = np.einsum('jk...,ijk...->i...', gu, Gam)
    bl = np.einsum('ij...,j...->i...', gl, bu)
    # D_i beta_j = d_i beta_j - Gamma^k_ij beta_k, with d_i beta_j = d_i (gamma_jl beta^l)
    dbl = np.einsum('ijl...,l...->ij...', dg, bu) + np.einsum('jl...,il...->ij...', gl, db)
    Db = dbl - np.einsum('kij...,k...->ij...', Gam, bl)
    Kij = (Db + np.einsum('ij...->ji...', Db)) / (2.0 * alpha)
    K = np.einsum('ij...,ij...->...', gu, Kij)
    return Metric(alpha, bu, gl, gu, sqrtg, da, db, gtrace, K)
