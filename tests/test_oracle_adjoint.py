"""Pins of the oracle's luminosity functional and complex-step gradient."""
import math

import numpy as np

import ffe_workloads as W
from oracle.adjoint import lbar, lbar_gradient_complex_step, luminosity, luminosity_weights
from oracle.problem import Problem


def _tiny():
    cfg = W.adjoint_pulsar(tiny=True)
    cfg["params"]["tci_on"] = 0
    return cfg


def test_surface_weights_integrate_the_sphere():
    """sum of the quadrature weights = 4 pi r^2 (exact area element, LGL quadrature)."""
    cfg = W.pulsar(r_lc=6.0, n_ang=4, n_rad=2, P=5, r_out=24.0)
    cfg["params"]["tci_on"] = 0
    pr = Problem(cfg)
    for rL in (3.0, 20.0):
        elems, lk, Wt, nrm = luminosity_weights(pr, rL)
        assert len(elems) == 6 * 16
        assert abs(Wt.sum() - 4 * math.pi * rL ** 2) < 1e-7 * 4 * math.pi * rL ** 2
        assert abs(lk.sum() - 1) < 1e-13


def test_luminosity_of_a_radial_poynting_field():
    """With E = r^ x a and B = a (a constant), ((r^ x a) x a).r^ = (a.r^)^2 - |a|^2,
    whose integral over the sphere of radius r is (4 pi/3 - 4 pi) |a|^2 r^2."""
    cfg = W.pulsar(r_lc=6.0, n_ang=3, n_rad=2, P=5, r_out=24.0)
    cfg["params"]["tci_on"] = 0
    pr = Problem(cfg)
    a = np.array([0.3, -0.2, 0.5])
    x = pr.disc.xyz
    r = np.linalg.norm(x, axis=0)
    rhat = x / r
    U = np.zeros((9,) + x.shape[1:])
    U[0:3] = np.cross(rhat, a[:, None, None, None, None], axis=0)
    U[3:6] = a[:, None, None, None, None] + 0 * x
    rL = 7.0
    L = luminosity(pr, U, luminosity_weights(pr, rL))
    assert abs(L + 8 * math.pi / 3 * np.dot(a, a) * rL ** 2) < 1e-6 * abs(L)


def test_complex_step_gradient_matches_central_differences_and_homogeneity():
    cfg = _tiny()
    n, rL = 3, 1.5
    g = lbar_gradient_complex_step(cfg, n, r_L=rL)
    kw = cfg["initial"][1]
    base = [kw["mu"], kw["chi"], cfg["params"]["omega_star"]]
    for k in range(3):
        h = 1e-5 * max(1.0, abs(base[k]))
        p, m = list(base), list(base)
        p[k] += h
        m[k] -= h
        fd = (lbar(cfg, n, p, rL) - lbar(cfg, n, m, rL)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * abs(g[k]), (k, fd, g[k])
    L = lbar(cfg, n, r_L=rL)
    assert abs(base[0] * g[0] - 2 * L) <= 1e-10 * abs(L)


def test_complex_step_gradient_with_a_fixed_hybrid_mask():
    """The same on the tiny shell with its innermost radial layer on FD
    subcells (fixed mask): the complex step runs through WENO5-Z (its |.|
    branches on the real part, eps = 1e-6 so that the flat stencils of the
    dipole data stay differentiable), the interpolated ghosts between wedges,
    the star state in the ghosts and the FD -> DG projection in the
    luminosity; one step, against central differences (eps = 1e-6 makes
    WENO5-Z scale-dependent, so the homogeneity in mu of the other test does
    not hold here)."""
    cfg = _tiny()
    cfg["params"].update(eta=50.0, weno_eps=1e-6)
    na, nr = cfg["n_ang"], cfg["n_rad"]
    e = np.arange(6 * na * na * nr)
    mask = ((e // (na * na)) % nr == 0).astype(np.uint8)
    n, rL = 1, 1.5
    g = lbar_gradient_complex_step(cfg, n, r_L=rL, mask=mask)
    kw = cfg["initial"][1]
    base = [kw["mu"], kw["chi"], cfg["params"]["omega_star"]]
    for k in range(3):
        h = 1e-5 * abs(base[k])
        p, m = list(base), list(base)
        p[k] += h
        m[k] -= h
        fd = (lbar(cfg, n, p, rL, mask) - lbar(cfg, n, m, rL, mask)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-4 * abs(g[k]), (k, fd, g[k])
