"""Pins of the oracle on the paper's one-dimensional tests (Sec. IV.A, Table I,
App. A) at their lowest resolution (32 elements along x, P = 5, eta = 1e6):
the fast wave against its exact translation, the stationary Alfven wave
against its initial state, the FFE breakdown against the invariants it keeps,
and the FD start (every element on subcells) that returns smooth elements to
DG."""
import numpy as np
import pytest

import ffe_workloads as W
from oracle import initial
from oracle.problem import Problem
from oracle.stepper import Stepper


def _run(test, nsteps, via_fd=False):
    cfg = W.oned(test, 0, via_fd=via_fd)
    pr = Problem(cfg)
    st = pr.initial_state(via_fd=via_fd)
    S = Stepper(pr)
    masks = [st["mask"].copy()]
    for _ in range(nsteps):
        st = S.step(st)
        masks.append(st["mask"].copy())
    return pr, st, masks


def test_oned_initial_data_constraints():
    """The three data sets satisfy E.B = 0, B^2 > E^2 and Gauss's law q = div E."""
    x = np.linspace(-0.5, 0.5, 2001)
    xyz = np.stack([x, 0 * x, 0 * x])
    h = 1e-7
    for f in (initial.fast_wave_kink, initial.alfven_stationary, initial.breakdown_1d):
        U = f(xyz)
        E, B = U[0:3], U[3:6]
        assert np.abs((E * B).sum(0)).max() < 1e-15
        assert ((B * B).sum(0) - (E * E).sum(0)).min() > 0.49
        # q = dEx/dx (the data depend on x only), central differences off the kinks
        xs = x[np.abs(np.abs(x) - 0.1) > 1e-3]
        Up = f(np.stack([xs + h, 0 * xs, 0 * xs]))
        Um = f(np.stack([xs - h, 0 * xs, 0 * xs]))
        q = f(np.stack([xs, 0 * xs, 0 * xs]))[8]
        np.testing.assert_allclose(q, (Up[0] - Um[0]) / (2 * h), atol=1e-6)


def test_fast_wave_kink_translates_exactly_away_from_the_kinks():
    """Exact solution Q(x - t, 0): the ramp between the kinks is linear and the
    states outside are constant, so the DG solution is exact there up to what
    the kinks radiate; a wave moving the wrong way or at the wrong speed is off
    by about the ramp slope times the shift."""
    pr, st, _ = _run("fast_wave_kink", 20)
    t = 20 * pr.dt
    d = pr.disc
    ex = initial.fast_wave_kink(d.xyz.reshape(3, -1), t=t).reshape((9,) + d.xyz.shape[1:])
    dg = (st["mask"] == 0)[:, None, None, None]
    xs = d.xyz[0] - t
    far = (np.abs(xs - 0.1) > 0.15) & (np.abs(xs + 0.1) > 0.15) & dg
    err = np.abs(st["udg"] - ex)
    assert err[2][far].max() < 1e-4 and err[4][far].max() < 1e-4
    assert err[2][np.broadcast_to(dg, err[2].shape)].max() < 1e-2
    u = st["udg"]
    assert np.abs(u[3] - 1.0).max() < 1e-12
    assert np.abs((u[0:3] * u[3:6]).sum(0)).max() < 1e-10


def test_alfven_wave_stays_stationary():
    """The stationary Alfven wave keeps its fields up to the initial transient
    of the stiff parallel current (Sec. IV.A.2); Bx and phi~ stay exact (no x-flux
    of Bx in one dimension)."""
    pr, st, _ = _run("alfven", 20)
    d = pr.disc
    U0 = initial.alfven_stationary(d.xyz.reshape(3, -1)).reshape((9,) + d.xyz.shape[1:])
    u = st["udg"]
    for v in range(6):
        assert np.abs(u[v] - U0[v]).max() < 3e-3, v
    assert np.abs(u[3] - 1.0).max() < 1e-12 and np.abs(u[7]).max() < 1e-12
    # IMEX-SSP3(4,3,3) ends on a combination of its stages, not on a stiff
    # solve, so E.B of u_{n+1} sits at the stage-error level, not at 1/eta
    assert np.abs((u[0:3] * u[3:6]).sum(0)).max() < 1e-2


def test_breakdown_1d_keeps_force_free_invariants():
    """FFE breakdown (Sec. IV.A.3): E.B stays zero, Bx stays 1, and B^2 - E^2
    falls from its initial minimum 0.5 in the layer while staying positive."""
    pr, st, _ = _run("breakdown_1d", 20)
    u = st["udg"]
    dg = st["mask"] == 0
    EB = (u[0:3] * u[3:6]).sum(0)[dg]
    B2mE2 = ((u[3:6] ** 2).sum(0) - (u[0:3] ** 2).sum(0))[dg]
    assert np.abs(EB).max() < 1e-10
    assert np.abs(u[3] - 1.0).max() < 1e-12
    assert 0.0 < B2mE2.min() < 0.45


def test_fd_start_returns_smooth_elements_to_dg():
    """FD start (Sec. III.C.1): every element begins on subcells; the FD
    indicator at the end of the first steps moves the smooth ones to DG, and the
    solution still follows the exact translation."""
    pr, st, masks = _run("fast_wave_kink", 3, via_fd=True)
    assert masks[0].all()
    assert masks[-1].sum() <= 4
    d = pr.disc
    ex = initial.fast_wave_kink(d.xyz.reshape(3, -1), t=3 * pr.dt).reshape((9,) + d.xyz.shape[1:])
    dg = (st["mask"] == 0)[:, None, None, None]
    err = np.abs(st["udg"] - ex)[2]
    assert err[np.broadcast_to(dg, err.shape)].max() < 1e-2
