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


def evaluate(kind, xyz, **kw):
    return {"fast_wave": fast_wave, "breakdown": breakdown, "cleaning_mode": cleaning_mode}[kind](xyz, **kw)
