"""Spin-down luminosity through a sphere (Sec. IV.C.2) and its gradient with
respect to the initial-data and star parameters by complex-step
differentiation of the whole discrete evolution.  Test infrastructure only.

L(u) = closed integral over r = r_L of S_i dSigma^i with S^i = [ijk] E_j B_k in
flat space, evaluated on the radial element layer containing r_L:
[reading] U is interpolated to r_L along xi^3 with the element's Lagrange
basis (xi^3 of r_L from the logarithmic radial map in closed form) and
integrated with the LGL quadrature in (xi^1, xi^2) and the exact area element
of the equiangular map; Lbar = mean of L(u_n) over steps n = 1..N.
"""
import numpy as np

from . import initial, physics as ph
from .basis import lagrange_matrix
from .ops import apply_3d
from .problem import Problem
from .stepper import Stepper


def luminosity_weights(pr, r_L):
    """Element list, xi^3 interpolation weights and per-node surface weights
    W[e, j, i] (LGL weights x area element x unit radial normal folded in later)."""
    mesh, T = pr.mesh, pr.T
    er = 2.0 * np.log(r_L / mesh.r_in) / np.log(mesh.r_out / mesh.r_in) - 1.0
    pos = (er + 1.0) / 2.0 * mesh.nr
    ir = min(int(np.floor(pos)), mesh.nr - 1)
    xi_r = 2.0 * (pos - ir) - 1.0
    lk = lagrange_matrix(T.x, np.array([xi_r]))[0]           # l_k(xi_r*)
    elems = [e for e in range(mesh.E) if mesh.eidx(e)[2] == ir]
    # area element of the sphere r = r_L in (xi^1, xi^2): |dx/dxi1 x dx/dxi2| by complex step
    from .geometry import complex_step_jacobian, tensor_points
    Z, Y, X = np.meshgrid(np.array([xi_r]), T.x, T.x, indexing="ij")
    pts = np.stack([X, Y, Z])[:, 0]                           # (3, Np, Np) [j][i]
    W, nrm = [], []
    for e in elems:
        J = complex_step_jacobian(lambda p: mesh.map(e, p), pts)   # [i][k][j][i']
        a, b = J[:, 0], J[:, 1]
        cr = np.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])
        x = mesh.map(e, pts)
        rhat = x / np.linalg.norm(x, axis=0)
        area = np.abs(np.sum(cr * rhat, axis=0))
        W.append(area * np.outer(T.w, T.w))
        nrm.append(rhat)
    return elems, lk, np.array(W), np.array(nrm)


def luminosity(pr, udg, lw):
    """L of a DG state (all elements DG)."""
    elems, lk, W, nrm = lw
    U = np.tensordot(lk, udg[:, elems], axes=(0, 2))          # (9, ne, Np, Np): interpolated to r_L
    E, B = U[0:3], U[3:6]
    S = ph.cross_lower(E, B)
    return np.sum(np.sum(S * np.moveaxis(nrm, 1, 0), axis=0) * W)


def lbar(cfg, nsteps, params=None, r_L=20.0, mask=None):
    """Mean luminosity over steps 1..nsteps for dipole (mu, chi) and star Omega;
    params = (mu, chi, Omega) may be complex (complex-step).  mask (optional,
    uint8 per element): a fixed DG/FD mask -- its FD elements start with the
    initial data at their subcell centres, no element switches, and an FD
    element enters the luminosity through its FD -> DG projection."""
    cfg = dict(cfg)
    cfg["params"] = dict(cfg["params"])
    kind, kw = cfg["initial"]
    kw = dict(kw)
    mu, chi, om = params if params is not None else (kw["mu"], kw["chi"], cfg["params"]["omega_star"])
    kw.update(mu=mu, chi=chi)
    cfg["initial"] = (kind, kw)
    if mask is not None:
        cfg["params"]["tci_on"] = 1        # the subcell grid is built; the mask is frozen below
    pr = Problem(cfg)
    pr.prm["omega"] = om
    pr.initial = lambda xyz: initial.evaluate(kind, xyz, **kw)
    pr.prm["dirichlet"] = pr.initial
    d = pr.disc
    udg = initial.evaluate(kind, d.xyz.reshape(3, -1), **kw).reshape((9,) + d.xyz.shape[1:])
    if mask is None:
        st = dict(mask=np.zeros(d.E, np.uint8), udg=udg, ufd=np.zeros((9, d.E, 1, 1, 1), dtype=udg.dtype), t=0.0)
    else:
        pr.prm["tci_on"] = 0
        nc = pr.T.nc
        ufd = np.zeros((9, d.E, nc, nc, nc), dtype=udg.dtype)
        for e in np.nonzero(mask)[0]:
            ufd[:, e] = initial.evaluate(kind, d.xyz_fd[:, e].reshape(3, -1), **kw).reshape((9, nc, nc, nc))
        st = dict(mask=np.asarray(mask, dtype=np.uint8).copy(), udg=udg, ufd=ufd, t=0.0)
    S = Stepper(pr)
    lw = luminosity_weights(pr, r_L)
    acc = 0.0
    for _ in range(nsteps):
        st = S.step(st)
        u = st["udg"]
        if mask is not None and mask.any():
            u = u.copy()
            fd = np.nonzero(st["mask"])[0]
            u[:, fd] = apply_3d(pr.T.R, st["ufd"][:, fd])
        acc = acc + luminosity(pr, u, lw)
    return acc / nsteps


def lbar_gradient_complex_step(cfg, nsteps, h=1e-30, r_L=20.0, mask=None):
    """d Lbar / d (mu, chi, Omega) by complex step (exact to rounding for the
    frozen-branch map: every branch is taken on the real part); mask: a fixed
    DG/FD mask (see lbar)."""
    kw = cfg["initial"][1]
    base = [kw["mu"], kw["chi"], cfg["params"]["omega_star"]]
    g = []
    for k in range(3):
        p = [complex(v) for v in base]
        p[k] += 1j * h
        g.append(np.imag(lbar(cfg, nsteps, p, r_L, mask)) / h)
    return np.array(g)
