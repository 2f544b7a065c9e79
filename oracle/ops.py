"""Tensor-product application of 1-D operators on element blocks.  Test
infrastructure only."""
import numpy as np


def apply_1d(M, u, axis):
    """Contract matrix M (n_out, n_in) with axis `axis` of u."""
    return np.moveaxis(np.tensordot(M, u, axes=(1, axis)), 0, axis)


def apply_3d(M, u):
    """(M x M x M) u on the last three axes of u."""
    for ax in (-1, -2, -3):
        u = apply_1d(M, u, u.ndim + ax)
    return u


def deriv(D, u, d):
    """D applied along reference direction d (0: xi^1 = last axis)."""
    return apply_1d(D, u, u.ndim - 1 - d)
