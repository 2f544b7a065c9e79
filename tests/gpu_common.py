"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on
the same workload and compare element by element."""
import numpy as np


def rel_err_split(g_dg, o_dg, g_fd, o_fd, sel_dg, floor_frac=1e-3):
    """Per-variable max|gpu - oracle| over the whole state (DG nodes of DG
    elements and FD cells of FD elements).  A variable whose magnitude is at
    least floor_frac of the largest variable's is measured relative to its own
    max|oracle_v|; a variable below that (an exact zero of the continuum
    problem, e.g. B~x of quasi-1-D data, whose values are rounding noise) is
    measured against the largest variable's magnitude."""
    sel_fd = ~sel_dg
    nv = o_dg.shape[0]
    errs, mags = np.zeros(nv), np.zeros(nv)
    for v in range(nv):
        e = m = 0.0
        if sel_dg.any():
            e = max(e, np.abs(g_dg[v][sel_dg] - o_dg[v][sel_dg]).max())
            m = max(m, np.abs(o_dg[v][sel_dg]).max())
        if sel_fd.any():
            e = max(e, np.abs(g_fd[v][sel_fd] - o_fd[v][sel_fd]).max())
            m = max(m, np.abs(o_fd[v][sel_fd]).max())
        errs[v], mags[v] = e, m
    scale = mags.max()
    den = np.where(mags >= floor_frac * scale, mags, scale)
    den = np.maximum(den, 1e-300)
    return errs / den


def compare_state(ctx, U, st, tol):
    dg, fd = ctx.split(U)
    worst = rel_err_split(dg, st["udg"], fd, st["ufd"], st["mask"] == 0).max()
    assert worst <= tol, worst
    return worst
