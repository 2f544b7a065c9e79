"""Fluxes through a shell's coordinate surface r = const: the magnetic flux
through the upper half of the outer horizon of Sec. IV.B.2 (compared there
with King's closed form pi r+^2 B0 (1 - a^4/r+^4)).  Test infrastructure only.

The surface is xi^3 = const on the radial element layer containing r (the
sphere |x| = r, or on a spherical Kerr-Schild shell, App. B, the spheroid of
Kerr-Schild radius r).  [reading] As for the luminosity: the state is
interpolated to r along xi^3 with the element's Lagrange basis, and the flux
integral of a densitised vector V~ is sum over nodes of w_i w_j V~ . (a1 x a2)
with a_k = dx/dxi^k (complex-step derivatives of the mesh map), the coordinate
area element oriented to increasing r.
"""
import numpy as np

from .basis import lagrange_matrix
from .geometry import complex_step_jacobian


def surface_weights(pr, r, upper=False):
    """Elements of the layer containing r, the xi^3 interpolation weights and
    the oriented area vectors A[e][:, j, i] = w_i w_j (a1 x a2) sign(det J).
    upper: only elements whose centre has z > 0."""
    mesh, T = pr.mesh, pr.T
    er = 2.0 * np.log(r / mesh.r_in) / np.log(mesh.r_out / mesh.r_in) - 1.0
    pos = (er + 1.0) / 2.0 * mesh.nr
    ir = min(int(np.floor(pos)), mesh.nr - 1)
    xi_r = 2.0 * (pos - ir) - 1.0
    lk = lagrange_matrix(T.x, np.array([xi_r]))[0]
    Z, Y, X = np.meshgrid(np.array([xi_r]), T.x, T.x, indexing="ij")
    pts = np.stack([X, Y, Z])[:, 0]                           # (3, Np, Np) [j][i]
    elems, A = [], []
    for e in range(mesh.E):
        if mesh.eidx(e)[2] != ir:
            continue
        if upper and not mesh.map(e, np.array([[0.0], [0.0], [xi_r]]))[2, 0] > 0.0:
            continue
        J = complex_step_jacobian(lambda p: mesh.map(e, p), pts)   # [i][k][j][i']
        a, b, c = J[:, 0], J[:, 1], J[:, 2]
        cr = np.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])
        sg = np.sign(np.sum(cr * c, axis=0))
        elems.append(e)
        A.append(cr * sg * np.outer(T.w, T.w))
    return elems, lk, np.array(A)


def flux(udg, sw, var=3):
    """Flux of the densitised vector U[var:var+3] (default B~) of a DG state
    through the surface of surface_weights."""
    elems, lk, A = sw
    U = np.tensordot(lk, udg[var:var + 3][:, elems], axes=(0, 2))   # (3, ne, Np, Np)
    return float(np.sum(U * np.moveaxis(A, 1, 0)))
