"""Pins of the oracle's curved geometry and Kerr-Schild background (Sec. IV.B,
App. B, App. C) against closed forms, identities and convergence."""
import math

import numpy as np
import pytest

import ffe_workloads as W
from oracle import initial
from oracle.dg import rhs_dg
from oracle.geometry import ShellMesh, Discretisation, BC_DIRICHLET
from oracle.metric import ks_metric
from oracle.ops import deriv
from oracle.problem import Problem
from oracle.stepper import Stepper
from oracle.basis import Tables


def test_kerr_schild_identities():
    """alpha sqrt(gamma) = 1 (sqrt(-g) = 1 in Kerr-Schild), K = D_i beta^i / alpha
    for a static metric, and a = 0 gives the Schwarzschild lapse (1 + 2M/r)^(-1/2)."""
    rng = np.random.default_rng(4)
    x = rng.normal(size=(3, 40)) * 4
    x = x[:, np.linalg.norm(x, axis=0) > 2.5]
    m = ks_metric(x, 1.0, 0.9)
    np.testing.assert_allclose(m.alpha * m.sqrtg, 1.0, rtol=1e-14)
    # D_i beta^i = (1/sqrt(gamma)) d_i (sqrt(gamma) beta^i), by complex step of the product
    h = 1e-30
    div = 0.0
    for i in range(3):
        p = x.astype(np.complex128)
        p[i] += 1j * h
        from oracle.metric import ks_four_metric, adm_from_four
        a, bu, gl, _ = adm_from_four(ks_four_metric(p, 1.0, 0.9))
        sg = np.sqrt(np.linalg.det(np.moveaxis(gl, (0, 1), (-2, -1))))
        div = div + np.imag(sg * bu[i]) / h
    np.testing.assert_allclose(m.K, div / m.sqrtg / m.alpha, rtol=1e-10, atol=1e-14)
    m0 = ks_metric(x, 1.0, 0.0)
    r = np.linalg.norm(x, axis=0)
    np.testing.assert_allclose(m0.alpha, (1 + 2 / r) ** -0.5, rtol=1e-14)


def test_wald_a0_closed_form():
    """App. C / Sec. IV.B.1: at a = 0 the construction from A_b gives
    B~ = (0, 0, B0), E~ = (-2 M B0 y / r^2, 2 M B0 x / r^2, 0)."""
    rng = np.random.default_rng(5)
    x = rng.normal(size=(3, 30)) * 5
    U = initial.wald(x, M=1.3, a=0.0, B0=0.7)
    r2 = np.sum(x * x, axis=0)
    np.testing.assert_allclose(U[0], -2 * 1.3 * 0.7 * x[1] / r2, atol=1e-15)
    np.testing.assert_allclose(U[1], 2 * 1.3 * 0.7 * x[0] / r2, atol=1e-15)
    np.testing.assert_allclose(U[2], 0, atol=1e-15)
    np.testing.assert_allclose(U[3:6], np.array([0, 0, 0.7])[:, None] + 0 * x, atol=1e-15)


def test_wald_fields_are_divergence_free_and_force_free_at_a0():
    """div B~ = 0 identically (B~ is a curl); at a = 0 E~.B~ = 0 (Sec. IV.B.1)."""
    rng = np.random.default_rng(6)
    x = rng.normal(size=(3, 20)) * 4 + 0.5
    h = 1e-30
    div = 0
    for i in range(3):
        p = x.astype(np.complex128)
        p[i] += 1j * h
        div = div + np.imag(initial.wald(p.real + 0, 1.0, 0.9)[3 + i]) * 0  # placeholder for shape
    # finite-difference divergence of B~ at a = 0.9 (4th order, small step)
    d = 1e-3
    div = 0
    for i in range(3):
        e = np.zeros((3, 1))
        e[i] = d
        f = lambda s: initial.wald(x + s * e, 1.0, 0.9)[3 + i]
        div = div + (-f(2) + 8 * f(1) - 8 * f(-1) + f(-2)) / (12 * d)
    assert np.abs(div).max() < 1e-9
    U = initial.wald(x, 1.0, 0.0)
    assert np.abs(np.sum(U[0:3] * U[3:6], 0)).max() < 1e-14


def test_dipole_closed_form():
    rng = np.random.default_rng(7)
    x = rng.normal(size=(3, 25)) * 2
    mu, dl, chi = 1.7, 0.1, 0.6
    m = np.array([math.sin(chi), 0, math.cos(chi)])
    r2 = np.sum(x * x, 0)
    B = mu * (3 * x * (m @ x) - m[:, None] * (r2 - 2 * dl * dl)) / (r2 + dl * dl) ** 2.5
    np.testing.assert_allclose(initial.dipole(x, mu, dl, chi)[3:6], B, atol=1e-13)


def test_shell_mesh_geometry():
    """Wedge map pins: nodes on the r_in / r_out spheres, every angular face
    matched (across wedges too), one radial layer on each boundary, and the
    chain-rule gradient of a linear function converging spectrally (the map is
    not polynomial, so it is exact only in the limit)."""
    errs = []
    for P in (4, 7):
        mesh = ShellMesh(1.0, 4.0, 2, 2, BC_DIRICHLET, BC_DIRICHLET)
        T = Tables(P)
        d = Discretisation(mesh, T)
        r = np.linalg.norm(d.xyz, axis=0)
        assert abs(r.min() - 1.0) < 1e-14 and abs(r.max() - 4.0) < 1e-14
        assert np.all(d.nbr[:, :4] >= 0)
        assert (d.nbr[:, 4] < 0).sum() == 6 * 2 * 2 and (d.nbr[:, 5] < 0).sum() == 6 * 2 * 2
        f = 0.3 * d.xyz[0] - 1.1 * d.xyz[1] + 2.0 * d.xyz[2]
        e = 0.0
        for j, c in enumerate((0.3, -1.1, 2.0)):
            g = sum(d.ijac[k, j] * deriv(T.D, f, k) for k in range(3))
            e = max(e, np.abs(g - c).max())
        errs.append(e)
    assert errs[0] < 1e-2 and errs[1] < errs[0] / 20, errs


def test_wald_stationarity_converges():
    """The exact Wald field (a = 0.9) is stationary: the DG right-hand side
    falls with the order on a fixed shell (Sec. IV.B.1, Table II behaviour)."""
    res = []
    for P in (4, 6):
        cfg = W.wald(n_ang=2, n_rad=4, P=P, r_in=2.0, r_out=6.0)
        cfg["params"]["tci_on"] = 0
        pr = Problem(cfg)
        st = pr.initial_state()
        res.append(np.abs(rhs_dg(st, pr.disc, pr.met, pr.prm)[:8]).max())
    assert res[1] < 2e-3 and res[0] / res[1] > 5, res


_WALD_FD = {}


def _wald_fd_residuals(interp):
    """The FD right-hand side of the exact (stationary) Wald field, every
    element on FD subcells, P = 5, on two shells (1 x 1 x 2 and 2 x 2 x 4
    elements per wedge): max |dU/dt| over element interiors (3 cells from every
    face), over the face-centre cells next to radial-boundary faces, faces
    between elements of one wedge and faces between wedges, and over all
    cells.  interp: ghosts across neighbour faces interpolated to the local
    grid's extension (prm["ghost_interp"]) instead of the neighbour's cells."""
    if interp in _WALD_FD:
        return _WALD_FD[interp]
    import warnings
    from oracle.fd import rhs_fd
    out = []
    for na, nr in ((1, 2), (2, 4)):
        cfg = W.wald(n_ang=na, n_rad=nr, P=5, r_in=2.0, r_out=6.0)
        cfg["params"]["fd_corrector"] = 0
        pr = Problem(cfg)
        pr.prm["ghost_interp"] = interp
        st = pr.initial_state(via_fd=True)
        st["mask"][:] = 1
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")   # metric at the never-read corner ghost cells
            r = np.abs(rhs_fd(st, pr.disc, pr.met, pr.prm)[:8]).max(axis=0)
        d, Nc = pr.disc, pr.T.nc
        cen = d.xyz_fd.mean(axis=(2, 3, 4))
        wedge = [(int(np.argmax(np.abs(cen[:, e]))), bool(cen[np.argmax(np.abs(cen[:, e])), e] > 0)) for e in range(d.E)]
        res = {"interior": r[:, 3:Nc - 3, 3:Nc - 3, 3:Nc - 3].max(), "boundary": 0.0, "wedge": 0.0,
               "between_wedges": 0.0, "all": r.max()}
        for e in range(d.E):
            for f in range(6):
                ax = 2 - f // 2
                idx = [slice(3, Nc - 3)] * 3
                idx[ax] = slice(0, 1) if f % 2 == 0 else slice(Nc - 1, Nc)
                nb = d.nbr[e, f]
                k = "boundary" if nb < 0 else ("wedge" if wedge[nb] == wedge[e] else "between_wedges")
                res[k] = max(res[k], r[e][tuple(idx)].max())
        out.append(res)
    _WALD_FD[interp] = out
    return out


def test_fd_wald_residual_converges_within_wedges():
    """The metric-general FD operator (Sec. III.C.2 on the Kerr-Schild
    background, a = 0.9) is consistent inside the wedges: the residual of the
    exact stationary field falls under refinement in element interiors and at
    the radial boundaries (ghosts from the exact field)."""
    c, f = _wald_fd_residuals(False)
    assert f["interior"] < c["interior"] / 4, (c, f)
    assert f["boundary"] < c["boundary"] / 4, (c, f)
    assert f["wedge"] < 2e-3, (c, f)


def test_fd_wald_residual_does_not_converge_between_wedges_with_copied_ghosts():
    """Why the ghosts are interpolated: at faces between wedges the
    neighbour's cells do not continue the local grid lines, and copying them
    as ghosts (prm["ghost_interp"] off) is inconsistent -- the residual there
    does not fall under refinement (1.7e-2 -> 3.0e-2)."""
    c, f = _wald_fd_residuals(False)
    assert f["between_wedges"] > c["between_wedges"] / 3, (c, f)


def test_fd_wald_residual_converges_between_wedges_with_interpolated_ghosts():
    """Ghosts interpolated to the local grid's extension (the neighbour's data
    at those points: sixth-order tensor Lagrange through its cells) make the
    residual fall at faces between wedges too (1.6e-3 -> 4.2e-4), and with it
    the largest residual anywhere (4.6e-3 -> 1.1e-3, against 4.7e-2 -> 5.6e-2
    with copied ghosts)."""
    c, f = _wald_fd_residuals(True)
    assert f["between_wedges"] < c["between_wedges"] / 3, (c, f)
    assert f["all"] < c["all"] / 3, (c, f)
    assert f["all"] < _wald_fd_residuals(False)[1]["all"] / 20


def test_interpolated_ghosts_equal_copied_ghosts_on_aligned_grids():
    """On a box the grids of neighbours continue each other: ghosts
    interpolated to the local grid's extension are the neighbour's cells (FD
    neighbour) or its polynomial at its subcell centres (DG neighbour), so the
    two readings give the same right-hand side up to rounding."""
    from oracle.fd import rhs_fd
    cfg = W.fast_wave(n=2, P=5)
    cfg["n"] = (3, 2, 1)
    pr = Problem(cfg)
    st = pr.initial_state()
    st["mask"][[0, 3]] = 1
    pr.prm["ghost_interp"] = False
    a = rhs_fd(st, pr.disc, pr.met, pr.prm)
    pr.prm["ghost_interp"] = True
    b = rhs_fd(st, pr.disc, pr.met, pr.prm)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def _table2():
    """Rows (P, N_r, N_Omega, dt, error) of tests/golden/table2_wald.txt (the
    paper's Table II, Sec. IV.B.1)."""
    import os
    rows = []
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table2_wald.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        P, res, dt, err = line.split()
        nr, nom = (int(x) for x in res.split("x"))
        rows.append((int(P), nr, nom, float(dt), float(err)))
    return rows


def test_exact_wald_l2_error_in_the_band_of_table2():
    """The paper's exact-Wald convergence test (Sec. IV.B.1, Table II): a = 0,
    r in [1.99 M, 20 M], eta = 0, DG-P5 at the low resolution (1 radial x 6
    angular elements, one per wedge), the table's time step, evolved to
    t = 5 M; L2 = sqrt((1/n) sum_k |B~_k - B~_exact,k|^2) over the n nodes.
    The paper imposes nothing at the inner surface (inside the horizon,
    where every characteristic leaves: the outflow face) and a Dirichlet
    state at the outer one.  With that setup the oracle's error is the
    table's to 0.1% (8.713e-4 against 8.71e-4; a Dirichlet
    inner face gives 7.4e-4), which pins the Wald field, the Kerr-Schild
    sources, the DG scheme, the time stepper, the outflow face and the norm
    at once."""
    P, nr, nom, dt, err = _table2()[0]
    assert (P, nr, nom) == (5, 1, 6)
    na = int(round(np.sqrt(nom / 6)))
    cfg = W.wald(n_ang=na, n_rad=nr, P=P, r_in=1.99, r_out=20.0, spin=0.0)
    cfg["params"].update(tci_on=0, dt=dt)
    cfg["bc_inner"] = "outflow"
    pr = Problem(cfg)
    st = pr.initial_state()
    S = Stepper(pr)
    n = int(round(5.0 / dt))
    for _ in range(n):
        st = S.step(st)
    d = pr.disc
    ex = pr.initial(d.xyz.reshape(3, -1)).reshape((9,) + d.xyz.shape[1:])
    v = st["udg"][3:6] - ex[3:6]
    l2 = np.sqrt((v ** 2).sum() / v[0].size)
    assert abs(l2 / err - 1.0) < 2e-3, (l2, err)


def test_wald_field_horizon_flux_is_kings():
    """The magnetic flux of the exact Wald field through the upper half of
    the outer horizon has the closed form pi r+^2 B0 (1 - a^4/r+^4) (Sec.
    IV.B.2, King et al.), r+ = M (1 + sqrt(1 - a^2)).  In Cartesian Kerr-Schild
    coordinates the horizon r = r+ is a spheroid whose equator is the circle
    x^2 + y^2 = r+^2 + a^2, z = 0, and the densitised B~ has zero coordinate
    divergence, so the flux through the upper half of the coordinate sphere of
    radius sqrt(r+^2 + a^2) (same boundary circle) is the same: the oracle's
    Wald field integrated there (Gauss-Legendre in theta, uniform in phi)
    reproduces the closed form to rounding for a = 0 ... 0.999.  This is the
    reading the flux diagnostic and the vacuum Wald runs use."""
    for a in (0.0, 0.5, 0.9, 0.999):
        M, B0 = 1.0, 1.0
        rp = M * (1 + np.sqrt(1 - a * a))
        R0 = np.sqrt(rp ** 2 + a ** 2)
        xg, wg = np.polynomial.legendre.leggauss(48)
        th, wth = (xg + 1) * np.pi / 4, wg * np.pi / 4
        nph = 64
        ph = np.arange(nph) * 2 * np.pi / nph
        T, Pp = np.meshgrid(th, ph, indexing="ij")
        x = np.stack([R0 * np.sin(T) * np.cos(Pp), R0 * np.sin(T) * np.sin(Pp), R0 * np.cos(T)])
        U = initial.wald(x.reshape(3, -1), M=M, a=a, B0=B0).reshape((9,) + T.shape)
        Br = (U[3:6] * (x / R0)).sum(axis=0)
        flux = (Br * R0 ** 2 * np.sin(T) * wth[:, None] * (2 * np.pi / nph)).sum()
        king = np.pi * rp ** 2 * B0 * (1 - a ** 4 / rp ** 4)
        assert abs(flux - king) <= 1e-12 * king, (a, flux, king)


def test_spherical_kerr_schild_shell_geometry():
    """The shell in the spherical Kerr-Schild radius (App. B): the boundary
    layers' nodes lie on the spheroids (x^2 + y^2)/(r^2 + a^2) + z^2/r^2 = 1 of
    r = r_in and r_out (the relation that defines r), every point agrees with
    App. B's transformation written in (r, theta, phi), the closed-form inverse
    map undoes the map, every angular face is matched, and the chain-rule
    gradient of a linear function converges spectrally."""
    a = 0.9
    errs = []
    for P in (4, 7):
        mesh = ShellMesh(1.0, 4.0, 2, 2, BC_DIRICHLET, BC_DIRICHLET, spin=a)
        T = Tables(P)
        d = Discretisation(mesh, T)
        x = d.xyz
        for k, r, layer in ((0, 1.0, 0), (-1, 4.0, 1)):
            sel = np.array([mesh.eidx(e)[2] == layer for e in range(mesh.E)])
            p = x[:, sel][:, :, k]
            rel = (p[0] ** 2 + p[1] ** 2) / (r * r + a * a) + p[2] ** 2 / (r * r)
            assert np.abs(rel - 1.0).max() < 1e-13
        # App. B in spherical form: theta, phi of the unit vector v of the
        # cubed-sphere map at the same reference point (the a = 0 mesh)
        m0 = ShellMesh(1.0, 4.0, 2, 2, BC_DIRICHLET, BC_DIRICHLET)
        x0 = np.stack([m0.map(e, np.stack(np.meshgrid(T.x, T.x, T.x, indexing="ij")[::-1]))
                       for e in range(mesh.E)], axis=1)
        r = np.linalg.norm(x0, axis=0)
        th, ph = np.arccos(x0[2] / r), np.arctan2(x0[1], x0[0])
        xb = np.stack([(r * np.cos(ph) - a * np.sin(ph)) * np.sin(th),
                       (r * np.sin(ph) + a * np.cos(ph)) * np.sin(th), r * np.cos(th)])
        assert np.abs(xb - x).max() < 1e-13
        rng = np.random.default_rng(P)
        for e in rng.integers(0, mesh.E, 6):
            xi = rng.uniform(-1, 1, size=(3, 5))
            assert np.abs(mesh.inv_map(e, mesh.map(e, xi)) - xi).max() < 1e-12
        assert np.all(d.nbr[:, :4] >= 0)
        assert (d.nbr[:, 4] < 0).sum() == 6 * 2 * 2 and (d.nbr[:, 5] < 0).sum() == 6 * 2 * 2
        f = 0.3 * x[0] - 1.1 * x[1] + 2.0 * x[2]
        e = 0.0
        for j, c in enumerate((0.3, -1.1, 2.0)):
            g = sum(d.ijac[k, j] * deriv(T.D, f, k) for k in range(3))
            e = max(e, np.abs(g - c).max())
        errs.append(e)
    assert errs[0] < 1e-2 and errs[1] < errs[0] / 20, errs


def test_horizon_flux_on_the_spherical_kerr_schild_horizon_converges_to_kings():
    """The coordinate-surface flux of the oracle (oracle.surface) of the exact
    Wald field through the upper half of the outer horizon, which is the
    inner surface r_in = r+ of a spherical Kerr-Schild shell: spectral
    convergence to pi r+^2 B0 (1 - a^4/r+^4) (Sec. IV.B.2) as the angular
    elements are refined (no interpolation in xi^3 there), and on the vacuum
    Wald grid (r+ inside a layer, 16 x 96 elements, P = 5) within 1e-6."""
    from oracle.surface import flux, surface_weights
    for a in (0.9, 0.999):
        rp = 1.0 + math.sqrt(1.0 - a * a)
        king = math.pi * rp * rp * (1.0 - a ** 4 / rp ** 4)
        errs = []
        for na in (2, 4, 6):
            cfg = W.wald_vacuum(spin=a, n_ang=na, n_rad=1, r_in=rp, r_out=2.0 * rp)
            cfg["initial"] = ("wald", dict(M=1.0, a=a, B0=1.0))
            pr = Problem(cfg)
            errs.append(abs(flux(pr.initial_state()["udg"], surface_weights(pr, rp, upper=True)) / king - 1.0))
        assert errs[1] < errs[0] / 50 and errs[2] < errs[1] / 10 and errs[2] < 1e-10, (a, errs)
    cfg = W.wald_vacuum(spin=0.9)
    cfg["initial"] = ("wald", dict(M=1.0, a=0.9, B0=1.0))
    pr = Problem(cfg)
    rp = 1.0 + math.sqrt(1.0 - 0.81)
    king = math.pi * rp * rp * (1.0 - 0.81 ** 2 / rp ** 4)
    assert abs(flux(pr.initial_state()["udg"], surface_weights(pr, rp, upper=True)) / king - 1.0) < 1e-6


def test_vacuum_wald_grid_time_step_is_the_papers():
    """The vacuum Wald grid (spherical Kerr-Schild r in [M, 125 M], 16 x 96
    elements, P = 5, CFL factor 0.25) gives the time step that Sec. IV.B.2
    quotes, 1.97e-3 M, for a = 0.999 -- a check of the mesh reading (radius in
    the spherical Kerr-Schild coordinate, innermost layer at r = M)."""
    pr = Problem(W.wald_vacuum(spin=0.999))
    assert abs(pr.dt - 1.97e-3) < 0.005e-3, pr.dt


def test_wedge_face_ghosts_transfer_the_current_so_a_force_free_state_is_eta_independent():
    """Reading 14 at faces between wedges: an FD neighbour's ghosts carry its
    cells' current interpolated like its state.  Pin: on an all-FD shell
    (6 wedges x 1 x 1 x 2, every element touching wedge faces), a state with
    E~ = -v x B~ (v = 0.1 z^ x x, sub-luminal: E.B = 0 and E^2 < B^2 at every
    point) has no parallel current anywhere, so its right-hand side must not
    depend on eta; it agrees at eta = 1e2 and 1e6 to rounding times eta.  The
    current of the interpolated state instead (planted below in a copy of
    the oracle's FD operator) takes eta (E.B) of the interpolation error at
    those ghosts and moves the q~ right-hand side by O(1) at eta = 1e6."""
    import types
    import oracle.fd as FD
    from oracle import physics as ph
    cfg = W.pulsar(r_lc=3.0, chi=0.3, n_ang=1, n_rad=2, P=5, r_out=4.0)
    cfg["bc_inner"] = cfg["bc_outer"] = "dirichlet"
    pr = Problem(cfg)
    d = pr.disc
    x = d.xyz_fd
    U = pr.initial(x.reshape(3, -1)).reshape((9,) + x.shape[1:])
    v = np.stack([-0.1 * x[1], 0.1 * x[0], 0 * x[0]])
    U[0:3] = -ph.cross_lower(v, U[3:6])
    st = dict(mask=np.ones(d.E, dtype=np.uint8), udg=np.zeros((9,) + d.xyz.shape[1:]), ufd=U, t=0.0)

    def spread(mod):
        out = []
        for eta in (1e2, 1e6):
            pr.prm["eta"] = eta
            out.append(mod.rhs_fd(st, d, pr.met, pr.prm))
        return np.abs(out[1] - out[0]).max()

    assert spread(FD) < 1e-8
    src = open(FD.__file__).read()
    transfer = """                        m = _met_at(met_fn["fd"], np.array([nb]), ())
                        jd, jp = ph.current(st["ufd"][:, nb:nb + 1], m, prm["eta"])
                        jgh[(slice(None),) + tgt[1:]] = _interp_fd((jd + jp)[:, 0], xi_nb, T.xc).reshape(
                            (3,) + ext[tgt].shape[1:])
"""
    assert src.count(transfer) == 1
    mod = types.ModuleType("oracle.fd_state_current")
    mod.__dict__["__package__"] = "oracle"
    exec(compile(src.replace(transfer, ""), "fd_state_current", "exec"), mod.__dict__)
    assert spread(mod) > 1e-2


def test_fd_wald_residual_converges_on_the_spherical_kerr_schild_shell():
    """The oracle's FD operator on the spherical Kerr-Schild shell (App. B,
    a = 0.9, r in [2, 6], every element on FD subcells, P = 5): the residual
    of the exact stationary Wald field falls under refinement (1 x 1 x 2 ->
    2 x 2 x 4 elements per wedge) in element interiors and at faces between
    wedges, where the ghosts are interpolated through the closed-form inverse
    of the map x = r v + a z^ x v (measured 2.2e-3 -> 5.4e-4 and 1.2e-3 ->
    3.6e-4)."""
    import warnings
    from oracle.fd import rhs_fd
    res = []
    for na, nr in ((1, 2), (2, 4)):
        cfg = W.wald(n_ang=na, n_rad=nr, P=5, r_in=2.0, r_out=6.0)
        cfg["shell_ks"] = True
        cfg["params"]["fd_corrector"] = 0
        pr = Problem(cfg)
        st = pr.initial_state(via_fd=True)
        st["mask"][:] = 1
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")   # metric at the never-read corner ghost cells
            r = np.abs(rhs_fd(st, pr.disc, pr.met, pr.prm)[:8]).max(axis=0)
        d, Nc, mesh = pr.disc, pr.T.nc, pr.mesh
        out = {"interior": r[:, 3:Nc - 3, 3:Nc - 3, 3:Nc - 3].max(), "between_wedges": 0.0}
        for e in range(d.E):
            for f in range(6):
                nb = d.nbr[e, f]
                if nb < 0 or mesh.eidx(nb)[3] == mesh.eidx(e)[3]:
                    continue
                idx = [slice(3, Nc - 3)] * 3
                idx[2 - f // 2] = slice(0, 1) if f % 2 == 0 else slice(Nc - 1, Nc)
                out["between_wedges"] = max(out["between_wedges"], r[e][tuple(idx)].max())
        res.append(out)
    c, f = res
    assert f["interior"] < c["interior"] / 3, res
    assert f["between_wedges"] < c["between_wedges"] / 2.5, res
