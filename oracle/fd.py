"""Conservative finite-difference subcell right-hand side (Sec. III.C.2).
Test infrastructure only.

On an FD element with (2N+1)^3 cells of width dxi = 2/(2N+1):
  dU_i/dt = - sum_k sum_j (d xi^k/d x^j)_i (F^j_{i+1/2} - F^j_{i-1/2}) / dxi + S(U_i)
Face values of the nine evolved variables and of the densitised current J~
(Sec. III.C.2: J~ is reconstructed to form the q~ flux) come from WENO5-Z with
exponent q = 2 (Borges et al. 2008, the paper's choice) in point-value
interpolation form (see `weno5z`).  The face flux is
Rusanov; optionally (Cartesian meshes) the 4th-order derivative corrector with
cell-centred fluxes is subtracted:  F = F* - (1/6)(F_i - 2 F* + F_{i+1}).
Three ghost layers per face come from the neighbour (its cells, or its DG
polynomial evaluated at its subcell centres) or from the boundary state.
"""
import numpy as np

from . import physics as ph
from .dg import DG, FD, _met_at
from .geometry import BC_DIRICHLET, BC_NO_INCOMING, BC_OUTFLOW, BC_STAR, layer_slice, axis_of
from .ops import apply_3d

NG = 3


def weno5z(v0, v1, v2, v3, v4, eps, q=2):
    """WENO5-Z value at the face between v2 and v3 from the left-biased stencil
    (v0..v4 = point values v_{i-2}..v_{i+2}).

    [reading] The subcell data are point values (conservative FD in the
    Shu-Osher sense, Sec. III.C.2) and the face states feed a flux that the
    4th-order corrector then turns into the Shu-Osher numerical flux; for the
    corrected scheme to be high order (as the paper reports, and as its
    uncorrected variant is not) the face states must be point-value
    interpolants.  So the three candidates are the quadratic interpolants at
    x_{i+1/2}, combined with the ideal weights (1, 10, 5)/16 of the 5-point
    interpolant; smoothness indicators are Jiang-Shu's, and the Z weights are
    alpha_k = d_k (1 + (tau_5/(beta_k + eps))^q), tau_5 = |beta_0 - beta_2|
    (Borges et al. 2008).  |.| branches on the real part (complex-step safe)."""
    p0 = 0.375 * v0 - 1.25 * v1 + 1.875 * v2
    p1 = -0.125 * v1 + 0.75 * v2 + 0.375 * v3
    p2 = 0.375 * v2 + 0.75 * v3 - 0.125 * v4
    b0 = 13.0 / 12.0 * (v0 - 2 * v1 + v2) ** 2 + 0.25 * (v0 - 4 * v1 + 3 * v2) ** 2
    b1 = 13.0 / 12.0 * (v1 - 2 * v2 + v3) ** 2 + 0.25 * (v1 - v3) ** 2
    b2 = 13.0 / 12.0 * (v2 - 2 * v3 + v4) ** 2 + 0.25 * (3 * v2 - 4 * v3 + v4) ** 2
    t = b0 - b2
    tau = np.where(np.real(t) < 0, -t, t)
    a0 = (1.0 / 16.0) * (1 + (tau / (b0 + eps)) ** q)
    a1 = (10.0 / 16.0) * (1 + (tau / (b1 + eps)) ** q)
    a2 = (5.0 / 16.0) * (1 + (tau / (b2 + eps)) ** q)
    return (a0 * p0 + a1 * p1 + a2 * p2) / (a0 + a1 + a2)


def _minmod(a, b):
    """minmod(a, b) = (sign a + sign b)/2 min(|a|, |b|)."""
    return 0.5 * (np.sign(a) + np.sign(b)) * np.minimum(np.abs(a), np.abs(b))


def _minmod4(a, b, c, d):
    """minmod of four values: the smallest magnitude when all four share a sign, else 0."""
    same = (np.sign(a) == np.sign(b)) & (np.sign(a) == np.sign(c)) & (np.sign(a) == np.sign(d))
    m = np.minimum(np.minimum(np.abs(a), np.abs(b)), np.minimum(np.abs(c), np.abs(d)))
    return np.where(same, np.sign(a) * m, 0.0)


def mp5(v0, v1, v2, v3, v4, alpha=4.0):
    """MP5 value at the face between v2 and v3 from the left-biased stencil:
    the monotonicity-preserving limiter of Suresh & Huynh (J. Comput. Phys.
    136, 83 (1997)) applied to the five-point interpolant.

    [reading] The paper reconstructs with WENO5-Z; MP5 is the alternative the
    task names.  As for WENO5-Z (see `weno5z`) the subcell data are point
    values, so the unlimited value is the point-value interpolant at the face,
    (3 v0 - 20 v1 + 90 v2 + 60 v3 - 5 v4)/128 (the 5-point polynomial through
    v0..v4), and the limiter's bounds are Suresh & Huynh's, written in the same
    second differences:
      v_MP = v2 + minmod(v3 - v2, alpha (v2 - v1));  if (vL - v2)(vL - v_MP) <= 0
      the value is vL; otherwise, with d_j the second differences centred on
      v1, v2, v3, d+ = minmod4(4 d2 - d3, 4 d3 - d2, d2, d3),
      d- = minmod4(4 d2 - d1, 4 d1 - d2, d2, d1), v_UL = v2 + alpha (v2 - v1),
      v_MD = (v2 + v3)/2 - d+/2, v_LC = v2 + (v2 - v1)/2 + (4/3) d-,
      v_min = max(min(v2, v3, v_MD), min(v2, v_UL, v_LC)),
      v_max = min(max(v2, v3, v_MD), max(v2, v_UL, v_LC)),
      value = median(vL, v_min, v_max) = vL + minmod(v_min - vL, v_max - vL).
    The unlimited test uses no tolerance (the median returns vL whenever it
    lies within the bounds, so rounding-level products change nothing)."""
    vL = (3.0 * v0 - 20.0 * v1 + 90.0 * v2 + 60.0 * v3 - 5.0 * v4) / 128.0
    vMP = v2 + _minmod(v3 - v2, alpha * (v2 - v1))
    d1 = v0 - 2.0 * v1 + v2
    d2 = v1 - 2.0 * v2 + v3
    d3 = v2 - 2.0 * v3 + v4
    dp = _minmod4(4.0 * d2 - d3, 4.0 * d3 - d2, d2, d3)
    dm = _minmod4(4.0 * d2 - d1, 4.0 * d1 - d2, d2, d1)
    vUL = v2 + alpha * (v2 - v1)
    vMD = 0.5 * (v2 + v3) - 0.5 * dp
    vLC = v2 + 0.5 * (v2 - v1) + (4.0 / 3.0) * dm
    vmin = np.maximum(np.minimum(np.minimum(v2, v3), vMD), np.minimum(np.minimum(v2, vUL), vLC))
    vmax = np.minimum(np.maximum(np.maximum(v2, v3), vMD), np.maximum(np.maximum(v2, vUL), vLC))
    lim = vL + _minmod(vmin - vL, vmax - vL)
    return np.where((vL - v2) * (vL - vMP) <= 0.0, vL, lim)


def reconstruct(v, prm):
    """Left and right face values from the six cells around each face: WENO5-Z
    (default, the paper's choice) or MP5 (prm["recon"] == 1)."""
    if prm.get("recon", 0) == 1:
        return mp5(v[0], v[1], v[2], v[3], v[4]), mp5(v[5], v[4], v[3], v[2], v[1])
    eps = prm["weno_eps"]
    return weno5z(v[0], v[1], v[2], v[3], v[4], eps), weno5z(v[5], v[4], v[3], v[2], v[1], eps)


def _lagrange_weights(nodes, t):
    """w[..., m]: the Lagrange basis through `nodes` (last axis) evaluated at t
    (the shape of nodes without its last axis, or broadcastable to it)."""
    n = nodes.shape[-1]
    t = np.asarray(t)[..., None]
    w = np.ones(np.broadcast_shapes(t.shape[:-1], nodes.shape[:-1]) + (n,))
    for m in range(n):
        for k in range(n):
            if k != m:
                w[..., m] *= (t[..., 0] - nodes[..., k]) / (nodes[..., m] - nodes[..., k])
    return w


def _interp_dg(u, xi, x_lgl):
    """The nodal polynomial u (q, k, j, i) of an element at reference points
    xi (3, npts): tensor Lagrange interpolation at its LGL nodes."""
    L = [_lagrange_weights(x_lgl, xi[d]) for d in range(3)]    # (npts, P+1) each
    return np.einsum('pa,pb,pc,qcba->qp', L[0], L[1], L[2], u)


def _interp_fd(u, xi, xc, npt=6):
    """Cell values u (q, z, y, x) of an FD element at reference points xi
    (3, npts): tensor Lagrange interpolation through the `npt` cell centres
    nearest each point along every axis (sixth order for npt = 6), the stencil
    kept inside the element."""
    Nc = len(xc)
    dxi = 2.0 / Nc
    starts, ws = [], []
    for d in range(3):
        pos = (xi[d] + 1.0) / dxi - 0.5
        st0 = np.clip(np.floor(pos).astype(np.int64) - (npt // 2 - 1), 0, Nc - npt)
        nodes = xc[st0[:, None] + np.arange(npt)[None, :]]
        starts.append(st0)
        ws.append(_lagrange_weights(nodes, xi[d]))
    a = np.arange(npt)
    iz = (starts[2][:, None] + a)[:, :, None, None]
    iy = (starts[1][:, None] + a)[:, None, :, None]
    ix = (starts[0][:, None] + a)[:, None, None, :]
    g = u[:, iz, iy, ix]                                        # (q, npts, c, b, a)
    return np.einsum('pa,pb,pc,qpcba->qp', ws[0], ws[1], ws[2], g)


def fill_ghosts(st, disc, sel, met_fn, prm):
    """Extended cell arrays (9, n, Nc+6, Nc+6, Nc+6) for FD elements `sel`, the
    coordinates of every filled cell (for the metric), and the current J~ of the
    ghost cells that come from a DG neighbour (NaN elsewhere).  Corner/edge ghost
    regions are never read by the dimension-split scheme and stay NaN.
    [reading] A DG neighbour's ghost cells take its polynomial at its subcell
    centres for U and, for J~, the same evaluation of its nodal current (not the
    current of the evaluated state; see dg.external_fd_current).
    prm["ghost_interp"] (the default reading, Problem sets it): ghosts across
    a neighbour's face are the neighbour's data at the ghost centres of this
    element's grid extended past the face -- a DG neighbour's polynomial
    evaluated there, an FD neighbour's cells interpolated there (6-point
    tensor Lagrange in its reference coordinates, the paper's sixth-order
    transfer, Sec. III.C.1); either way the ghost current is the neighbour's
    current transferred the same way, not the current of the transferred
    state.  Off: the neighbour's own cells (its polynomial
    at its own subcell centres).  Where the grids continue each other (inside
    a cubed-sphere wedge, on boxes) both readings give the same ghosts up to
    rounding; between wedges only the interpolated ghosts are consistent
    (the residual of an exact stationary field converges there with them and
    not with the copies)."""
    T = disc.T
    Nc = T.nc
    n = len(sel)
    ext = np.full((9, n, Nc + 2 * NG, Nc + 2 * NG, Nc + 2 * NG), np.nan, dtype=st["ufd"].dtype)
    jgh = np.full((3,) + ext.shape[1:], np.nan, dtype=st["ufd"].dtype)
    xyz = np.full((3, n) + ext.shape[2:], np.nan)
    inner = (slice(NG, NG + Nc),) * 3
    ext[(slice(None), slice(None)) + inner] = st["ufd"][:, sel]
    xyz[(slice(None), slice(None)) + inner] = disc.xyz_fd[:, sel]
    dxi = 2.0 / Nc
    for a, e in enumerate(sel):
        for f in range(6):
            d, s = f // 2, f % 2
            nb, kind = disc.nbr[e, f], disc.bc[e, f]
            for g in range(NG):
                # ghost layer g (0 = adjacent to the face) in extended indexing
                pos = NG - 1 - g if s == 0 else NG + Nc + g
                idx = [slice(NG, NG + Nc)] * 3
                idx[2 - d] = pos
                tgt = (slice(None), a) + tuple(idx)
                if nb >= 0 and prm.get("ghost_interp", False):
                    gx = _ghost_centres(disc, e, d, s, g, dxi)
                    xi_nb = disc.mesh.inv_map(nb, gx.reshape(3, -1) - disc.mesh.period_shift(e, f)[:, None])
                    if st["mask"][nb] == FD:
                        ext[tgt] = _interp_fd(st["ufd"][:, nb], xi_nb, T.xc).reshape(ext[tgt].shape)
                        # the neighbour's current J~ transferred with the state (as
                        # from a DG neighbour): J~ of the interpolated state carries
                        # eta (E.B) of the interpolation error, which the stiff
                        # eta = 1e5 amplifies into a growing charge at wedge faces
                        m = _met_at(met_fn["fd"], np.array([nb]), ())
                        jd, jp = ph.current(st["ufd"][:, nb:nb + 1], m, prm["eta"])
                        jgh[(slice(None),) + tgt[1:]] = _interp_fd((jd + jp)[:, 0], xi_nb, T.xc).reshape(
                            (3,) + ext[tgt].shape[1:])
                    else:
                        ext[tgt] = _interp_dg(st["udg"][:, nb], xi_nb, T.x).reshape(ext[tgt].shape)
                        m = _met_at(met_fn["dg"], np.array([nb]), ())
                        jd, jp = ph.current(st["udg"][:, nb:nb + 1], m, prm["eta"])
                        jgh[(slice(None),) + tgt[1:]] = _interp_dg((jd + jp)[:, 0], xi_nb, T.x).reshape((3,) + ext[tgt].shape[1:])
                    xyz[tgt] = gx
                elif nb >= 0:
                    src = st["ufd"][:, nb] if st["mask"][nb] == FD else apply_3d(T.P, st["udg"][:, nb])
                    ext[tgt] = src.reshape(9, -1)[:, disc.fd_map[e, f, g]]
                    if st["mask"][nb] == DG:
                        m = _met_at(met_fn["dg"], np.array([nb]), ())
                        jd, jp = ph.current(st["udg"][:, nb:nb + 1], m, prm["eta"])
                        jsrc = apply_3d(T.P, (jd + jp)[:, 0])
                        jgh[(slice(None),) + tgt[1:]] = jsrc.reshape(3, -1)[:, disc.fd_map[e, f, g]]
                    xyz[tgt] = disc.xyz_fd[:, nb].reshape(3, -1)[:, disc.fd_map[e, f, g]]
                else:
                    # ghost centre from the element map continued past the face
                    lay = layer_slice(d, s, Nc, 0)
                    gx = _ghost_centres(disc, e, d, s, g, dxi)
                    xyz[tgt] = gx
                    outer = st["ufd"][:, e][(slice(None),) + lay]
                    if kind == BC_DIRICHLET:
                        ext[tgt] = prm["dirichlet"](gx)
                    elif kind == BC_NO_INCOMING:
                        mf = _met_at(met_fn["fdface"][d], np.array([e]), layer_slice(d, s, Nc + 1, 0))
                        ijf = disc.ijac_ff[d][:, :, e][(slice(None), slice(None)) + layer_slice(d, s, Nc + 1, 0)]
                        nrm = ijf[d] * (1.0 if s == 1 else -1.0)
                        gu = ph._bc(mf.gu, 2, nrm.ndim - 1)
                        nrm = nrm / np.sqrt(np.einsum('ij...,i...,j...->...', gu, nrm, nrm))
                        mo = _met_at(met_fn["fd"], np.array([e]), lay)
                        ext[tgt] = ph.bc_no_incoming_poynting(outer[:, None], mo, nrm[:, None])[:, 0]
                    elif kind == BC_STAR:
                        ext[tgt] = ph.bc_star(outer, disc.xyz_fd[:, e][(slice(None),) + lay], prm["omega"])
                    elif kind == BC_OUTFLOW:
                        ext[tgt] = outer
                    else:
                        raise ValueError("face without neighbour or boundary condition")
    return ext, xyz, jgh


def _ghost_centres(disc, e, d, s, g, dxi):
    """Physical centres (3, Nc, Nc) of ghost layer g past face (d, s) of element
    e: its reference grid continued past the face, mapped by its own map."""
    T = disc.T
    Nc = T.nc
    xi_n = -(1 + (g + 0.5) * dxi) if s == 0 else 1 + (g + 0.5) * dxi
    Z, Y, X = np.meshgrid(T.xc, T.xc, T.xc, indexing="ij")
    pts = np.stack([X, Y, Z])
    pts = pts[(slice(None),) + layer_slice(d, s, Nc, 0)].copy()
    pts[d] = xi_n
    return disc.mesh.map(e, pts)


def rhs_fd(st, disc, met, prm):
    """Explicit FD right-hand side for all elements with mask == FD.

    met: dict with 'fd' (Metric at cell centres), 'fdface' (list over face
    direction of Metric at face points) and 'at' (callable xyz -> Metric) for
    ghost cells.  prm: dict(eta, weno_eps, fd_corrector, dirichlet, omega).
    Returns dudt with the FD-element blocks filled (zeros elsewhere)."""
    T = disc.T
    Nc = T.nc
    sel = np.nonzero(st["mask"] == FD)[0]
    out = np.zeros_like(st["ufd"])
    if len(sel) == 0:
        return out
    ext, xyz, jgh = fill_ghosts(st, disc, sel, met, prm)
    mext = met["at"](np.nan_to_num(xyz))
    jd, jp = ph.current(np.nan_to_num(ext), mext, prm["eta"])
    Jx = np.where(np.isnan(np.real(jgh)), jd + jp, jgh)   # DG-neighbour ghosts: their current
    W = np.concatenate([ext, Jx], axis=0)  # 12 reconstructed quantities
    mc = _met_at(met["fd"], sel, ())
    ijac = disc.ijac_fd[:, :, sel]
    U = st["ufd"][:, sel]
    jdc, _ = ph.current(U, mc, prm["eta"])
    dudt = np.zeros_like(U)
    eps = prm["weno_eps"]
    for k in range(3):
        ax = 1 + axis_of(k)  # axis of W (12, n, z, y, x)

        def sl(lo, hi):
            idx = [slice(None), slice(None), slice(NG, NG + Nc), slice(NG, NG + Nc), slice(NG, NG + Nc)]
            idx[ax] = slice(lo, hi)
            return tuple(idx)
        # face m (0..Nc) between interior cells m-1 and m; extended index of cell c is c + NG
        # v[o+3][m] = cell m+o (o = -3..2) for each face m
        v = [W[sl(NG + o, NG + o + Nc + 1)] for o in range(-3, 3)]
        WL, WR = reconstruct(v, prm)
        UL, UR = WL[:9], WR[:9]
        JL, JR = WL[9:], WR[9:]
        mf = _met_at(met["fdface"][k], sel, ())
        FL = ph.fluxes(UL, JL, mf)
        FR = ph.fluxes(UR, JR, mf)
        ijf = disc.ijac_ff[k][:, :, sel]
        nrm = ijf[k]
        sp = nrm.ndim - 1
        gu = ph._bc(mf.gu, 2, sp)
        nrm = nrm / np.sqrt(np.einsum('ij...,i...,j...->...', gu, nrm, nrm))
        nup = np.einsum('jl...,l...->j...', gu, nrm)
        lam = ph._bc(mf.alpha, 0, sp) + np.abs(np.einsum('j...,j...->...', ph._bc(mf.beta, 1, sp), nrm))
        Fs = 0.5 * (FL + FR) - 0.5 * (lam * nup)[:, None] * (UR - UL)[None]
        if prm["fd_corrector"]:
            # cell-centred fluxes either side of each interior face; the
            # element-boundary faces use the ghost cells' fluxes
            mg = met["at"](np.nan_to_num(xyz))
            Fg = ph.fluxes(np.nan_to_num(ext), Jx, mg)
            def slc(lo, hi):
                idx = [slice(None), slice(None), slice(None), slice(NG, NG + Nc), slice(NG, NG + Nc), slice(NG, NG + Nc)]
                idx[ax + 1] = slice(lo, hi)
                return tuple(idx)
            Fm = Fg[slc(NG - 1, NG + Nc)]
            Fp = Fg[slc(NG, NG + Nc + 1)]
            Fs = Fs - (1.0 / 6.0) * (Fm - 2 * Fs + Fp)
        lo = [slice(None)] * 6
        hi = [slice(None)] * 6
        lo[ax + 1] = slice(0, Nc)
        hi[ax + 1] = slice(1, Nc + 1)
        diff = (Fs[tuple(hi)] - Fs[tuple(lo)]) * (Nc / 2.0)
        for j in range(3):
            dudt -= ijac[k, j][None] * diff[j]
    dudt += ph.sources_explicit(U, jdc, mc)
    out[:, sel] = dudt
    return out
