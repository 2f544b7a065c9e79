"""Nodal DG-SEM right-hand side (Sec. III.A) with Rusanov boundary correction
(Sec. III.C.2) for the GRFFE system.  Test infrastructure only.

For every DG element and node n:
  dU/dt = - sum_k sum_j (d xi^k/d x^j)_n (D_k F^j)_n + S_explicit
          - sum over faces (d, s) containing n of (|grad xi^d|_gamma / w_0)
            (F* . n^ - F_int . n^)
[reading] the volume term is the chain-rule strong form with the analytic
inverse Jacobian at each node, the same form the FD update uses (Sec.
III.C.2); the boundary correction is the lumped-mass LGL lift; the Rusanov
speed is lambda = alpha + |beta^i n^_i|, the light-cone bound of the principal
part.
"""
import numpy as np

from . import physics as ph
from .geometry import BC_DIRICHLET, BC_NO_INCOMING, BC_OUTFLOW, BC_STAR, face_slice
from .ops import apply_3d, deriv

DG, FD = 0, 1


def _met_at(m, e_sel, sl):
    """Metric fields restricted to elements e_sel and node slice sl."""
    def f(a):
        a = np.asarray(a)
        return a[(e_sel,) + sl] if a.ndim == 4 else a
    return m.take(f)


def face_normal(ijac_face, m_face, d, s):
    """Outward unit normal n^_j = +- (d xi^d/d x^j)/|grad xi^d|_gamma and |grad xi^d|_gamma."""
    n = ijac_face[d] * (1.0 if s == 1 else -1.0)
    sp = n.ndim - 1
    gu = ph._bc(m_face.gu, 2, sp)
    norm = np.sqrt(np.einsum('ij...,i...,j...->...', gu, n, n))
    return n / norm, norm


def external_dg_state(st, disc, e, f, Tbl):
    """Neighbour trace at my face nodes of face f: the neighbour's nodal values
    (DG neighbour) or the face trace of its FD->DG projection (FD neighbour)."""
    nb = disc.nbr[e, f]
    if st["mask"][nb] == DG:
        src = st["udg"][:, nb]
    else:
        src = apply_3d(Tbl.R, st["ufd"][:, nb])
    return src.reshape(src.shape[0], -1)[:, disc.dg_map[e, f]]


def external_fd_current(st, disc, met, prm, e, f, Tbl):
    """J~ at my face nodes of face f from an FD neighbour: the FD->DG projection
    of the current of its cells, traced like the state.
    [reading] The current of an exterior state that is a projection is the
    projection of the current, not the current of the projected state: the
    projected E~ is not a stiff-solve output, its E~.B~ is of the size of the
    projection error, and J~_eta = alpha eta (E~.B~) B~/B~^2 would carry it into
    the q~ flux amplified by eta (unstable for eta dt >> 1 at DG-FD interfaces)."""
    nb = disc.nbr[e, f]
    m = _met_at(met["fd"], np.array([nb]), ())
    jd, jp = ph.current(st["ufd"][:, nb:nb + 1], m, prm["eta"])
    src = apply_3d(Tbl.R, (jd + jp)[:, 0])
    return src.reshape(3, -1)[:, disc.dg_map[e, f]]


def rhs_dg(st, disc, met, prm):
    """Explicit DG right-hand side for all elements with mask == DG.

    st: dict(mask (E,), udg (9,E,Np,Np,Np), ufd (9,E,Nc,Nc,Nc)).
    met: dict with 'dg' (Metric at nodes).  prm: dict(eta, dirichlet(xyz)->U,
    omega).  Returns dudt with the DG-element blocks filled (zeros elsewhere)."""
    T = disc.T
    Np = T.np1
    mask = st["mask"]
    sel = np.nonzero(mask == DG)[0]
    U = st["udg"][:, sel]
    m = _met_at(met["dg"], sel, ())
    ijac = disc.ijac[:, :, sel]
    jd, jp = ph.current(U, m, prm["eta"])
    F = ph.fluxes(U, jd + jp, m)
    div = np.zeros_like(U)
    for k in range(3):
        for j in range(3):
            div += ijac[k, j][None] * deriv(T.D, F[j], k)
    dudt = -div + ph.sources_explicit(U, jd, m)
    for f in range(6):
        d, s = f // 2, f % 2
        fs = face_slice(d, s, Np)
        full = (slice(None), slice(None)) + fs
        Ui = U[full]
        mf = _met_at(met["dg"], sel, fs)
        nhat, norm = face_normal(ijac[(slice(None), slice(None), slice(None)) + fs], mf, d, s)
        Ue = np.zeros_like(Ui)
        Jx = {}   # exterior current of faces with an FD neighbour
        for a, e in enumerate(sel):
            nb, kind = disc.nbr[e, f], disc.bc[e, f]
            if nb >= 0:
                Ue[:, a] = external_dg_state(st, disc, e, f, T)
                if mask[nb] == FD:
                    Jx[a] = external_fd_current(st, disc, met, prm, e, f, T)
            elif kind == BC_DIRICHLET:
                Ue[:, a] = prm["dirichlet"](disc.xyz[:, e][(slice(None),) + fs])
            elif kind == BC_NO_INCOMING:
                mfa = _met_at(met["dg"], np.array([e]), fs)
                Ue[:, a] = ph.bc_no_incoming_poynting(Ui[:, a:a + 1], mfa, nhat[:, a:a + 1])[:, 0]
            elif kind == BC_STAR:
                Ue[:, a] = ph.bc_star(Ui[:, a], disc.xyz[:, e][(slice(None),) + fs], prm["omega"])
            elif kind == BC_OUTFLOW:
                # [reading] an excision surface inside a horizon (Sec. IV.B.2: no
                # condition imposed there): the exterior state is the interior one,
                # so the Rusanov flux is the interior flux
                Ue[:, a] = Ui[:, a]
            else:
                raise ValueError("face without neighbour or boundary condition")
        jdi, jpi = ph.current(Ui, mf, prm["eta"])
        jde, jpe = ph.current(Ue, mf, prm["eta"])
        for a, jx in Jx.items():
            jde[:, a] = 0.0
            jpe[:, a] = jx
        Fi = ph.fluxes(Ui, jdi + jpi, mf)
        Fe = ph.fluxes(Ue, jde + jpe, mf)
        Fin = np.einsum('j...,jv...->v...', nhat, Fi)
        Fen = np.einsum('j...,jv...->v...', nhat, Fe)
        sp = nhat.ndim - 1
        lam = ph._bc(mf.alpha, 0, sp) + np.abs(np.einsum('j...,j...->...', ph._bc(mf.beta, 1, sp), nhat))
        Fstar = 0.5 * (Fin + Fen) - 0.5 * lam * (Ue - Ui)
        dudt[full] -= (norm / T.w0)[None] * (Fstar - Fin)
    out = np.zeros_like(st["udg"], dtype=dudt.dtype)
    out[:, sel] = dudt
    return out
