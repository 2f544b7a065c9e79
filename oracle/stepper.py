"""IMEX-SSP3(4,3,3) time step with the DG-FD hybrid control loop
(Sec. III.B, III.C.1, III.C.3).  Test infrastructure only.

Butcher tables (Pareschi & Russo 2005, the scheme the paper cites), with
a = 0.24169426078821, b = 0.06042356519705, h = 0.12915286960590:
  explicit  A = [[0,0,0,0],[0,0,0,0],[0,1,0,0],[0,1/4,1/4,0]]
  implicit  A~ = [[a,0,0,0],[-a,a,0,0],[0,1-a,a,0],[b,h,1/2-b-h-a,a]]
  weights   w = w~ = (0, 1/6, 1/6, 2/3)
Stage s solves U_s = R_s + dt a G(U_s) pointwise (physics.stiff_solve), with
R_s = u_n + dt sum_{j<s} (A_sj F(U_j) + A~_sj G(U_j)).  The explicit column of
stage 1 is zero, so F is evaluated at U_2, U_3, U_4 only: three right-hand
sides ("substeps") per step; u_{n+1} = u_n + dt sum_j w_j (F_j + G_j).

[reading] order inside a substep (U_3, U_4): explicit part R_s -> filter (DG
elements) -> stiff solve -> algebraic clamp (if on) -> TCI (DG elements); for
u_{n+1}, which has no solve: R -> filter -> clamp (if on) -> TCI.  The filter
("after every substep", Sec. III.A) thus acts on each substep's explicit
update, and every state the explicit right-hand side is evaluated at (U_2, U_3,
U_4) is a solve output.  Filtering after the solve re-creates a parallel E~ of
the size of the removed top mode at stage states; with eta dt >> 1 (the regime
Sec. III.B aims for) the q~ flux J~_eta = alpha eta (E~.B~) B~/B~^2 + ... then
carries that field amplified by eta, and the all-DG rotating dipole at
eta = 1e5 diverges.  G_s = G(U_s) = (U_s - R~_s)/(dt a) with R~_s the filtered
explicit part.
A DG element the TCI flags after a substep is rolled back: the substep's
inputs (u_n, the earlier F and G, and the stage state the RHS was taken at) are
projected to its subcells, the RHS is recomputed with the FD operator using the
neighbours' data of the same stage, and the result is rebuilt on FD (Sec.
III.C.1).  At the end of the step every FD element that did not switch during
it is checked with alpha' = alpha + 1 on its FD->DG projection and returns to
DG if admissible (Sec. III.C.3).
"""
import numpy as np

from . import physics as ph
from .dg import DG, FD, rhs_dg, _met_at
from .fd import rhs_fd
from .ops import apply_3d

A_IM = 0.24169426078821
B_IM = 0.06042356519705
H_IM = 0.12915286960590


def tci_threshold(N, M, alpha):
    """(N + 1 - M)^(-alpha) (Sec. III.C.3)."""
    return float(N + 1 - M) ** (-alpha)


def tci_ratio(B, met_dg, T, sel):
    """sqrt(sum u^2 / sum u^) per element, u = |B~|_gamma at the LGL nodes and
    u^ = u - (Pi x Pi x Pi) u the part carried by modes with any index >= N+1-M
    (Sec. III.C.3).  0 when sum u^2 = 0."""
    if len(sel) == 0:
        return np.zeros(0)
    m = _met_at(met_dg, sel, ())
    Bl = ph.lower(B, m, B.ndim - 1)
    u = np.sqrt(np.real(np.sum(Bl * B, axis=0)))
    uh = u - apply_3d(T.Pi, u)
    num = np.sum(uh.reshape(len(sel), -1) ** 2, axis=1)
    den = np.sum(u.reshape(len(sel), -1) ** 2, axis=1)
    return np.where(den > 0, np.sqrt(num / np.where(den > 0, den, 1.0)), 0.0)


class Stepper:
    def __init__(self, prob):
        self.p = prob
        self.last_switched = []
        self.near = []

    # ---- element-wise pointwise helpers on (dg, fd) pairs --------------------
    def _sel(self, mask, rep):
        return np.nonzero(mask == rep)[0]

    def pair_map(self, fn, mask, *pairs):
        """Apply fn(arrays..., metric, rep) to the DG part of DG elements and the
        FD part of FD elements."""
        out_dg = np.zeros_like(pairs[0][0])
        out_fd = np.zeros_like(pairs[0][1])
        for rep, out, key in ((DG, out_dg, "dg"), (FD, out_fd, "fd")):
            sel = self._sel(mask, rep)
            if len(sel) == 0:
                continue
            m = _met_at(self.p.met[key], sel, ())
            arrs = [pr[rep][:, sel] for pr in pairs]
            out[:, sel] = fn(*arrs, m)
        return out_dg, out_fd

    def lin(self, terms):
        """sum of coef * pair."""
        dg = sum(c * p[0] for c, p in terms)
        fd = sum(c * p[1] for c, p in terms)
        return dg, fd

    def solve(self, R, mask):
        p = self.p.prm
        dta = self.p.dt * A_IM
        eta = p["eta"] if p["mode"] != 1 else 0.0

        def f(r, m):
            u = ph.stiff_solve(r, m, eta, p["kappa_psi"], p["kappa_phi"], dta)
            if p["mode"] in (1, 2):
                u = ph.hard_clamp(u, m)
            return u
        return self.pair_map(f, mask, R)

    def G(self, U, mask):
        p = self.p.prm
        eta = p["eta"] if p["mode"] != 1 else 0.0
        return self.pair_map(lambda u, m: ph.implicit_G(u, m, eta, p["kappa_psi"], p["kappa_phi"]), mask, U)

    def rhs(self, U, mask):
        st = dict(mask=mask, udg=U[0], ufd=U[1])
        return rhs_dg(st, self.p.disc, self.p.met, self.p.prm), rhs_fd(st, self.p.disc, self.p.met, self.p.prm)

    def filt(self, U, mask):
        if not self.p.prm["filter_on"]:
            return U
        dg = U[0].copy()
        sel = self._sel(mask, DG)
        dg[:, sel] = apply_3d(self.p.T.F, U[0][:, sel])
        return dg, U[1]

    def to_fd(self, pair, e):
        """Project element e of a pair from DG to FD in place (returns new pair)."""
        fd = pair[1].copy()
        fd[:, e] = apply_3d(self.p.T.P, pair[0][:, e])
        return pair[0], fd

    # ---- the time step --------------------------------------------------------
    def step(self, st):
        P, T, dt = self.p, self.p.T, self.p.dt
        a, b, h = A_IM, B_IM, H_IM
        z = 0.5 - b - h - a
        mask = st["mask"].copy()
        un = (st["udg"].copy(), st["ufd"].copy())
        thr = tci_threshold(T.N, P.prm["tci_M"], P.prm["tci_alpha"])
        switched = set()
        self.near = []

        U1 = self.solve(un, mask)
        G1 = self.G(U1, mask)
        U2 = self.solve(self.lin([(1.0, un), (-dt * a, G1)]), mask)
        G2 = self.G(U2, mask)
        hist = dict(un=un, G1=G1, G2=G2)

        def substep(Uprev, Fprev, build, proj_keys):
            """Compute F at Uprev, build the substep result (filter and solve
            inside build), TCI and roll back."""
            nonlocal mask
            Fs = self.rhs(Uprev, mask)
            Un = build(Fs, mask)
            if not P.prm["tci_on"]:
                return Fs, Un
            sel = self._sel(mask, DG)
            r = tci_ratio(Un[0][3:6, sel], P.met["dg"], T, sel)
            self.near += [int(e) for e, x in zip(sel, r) if abs(x - thr) <= 1e-12 * thr]
            flagged = sel[r > thr]
            if len(flagged) == 0:
                return Fs, Un
            for e in flagged:
                mask[e] = FD
                switched.add(int(e))
                for k in proj_keys:
                    hist[k] = self.to_fd(hist[k], e)
                Uprev = self.to_fd(Uprev, e)
            st2 = dict(mask=mask, udg=Uprev[0], ufd=Uprev[1])
            Ffd = rhs_fd(st2, P.disc, P.met, P.prm)
            Fs = (Fs[0], Fs[1].copy())
            for e in flagged:
                Fs[1][:, e] = Ffd[:, e]
            Un2 = build(Fs, mask)
            Un = (Un[0], Un[1].copy())
            for e in flagged:
                Un[1][:, e] = Un2[1][:, e]
            return Fs, Un

        # substep A: F2 = F(U2), U3
        def build3(F2, mk):
            R = self.lin([(1.0, hist["un"]), (dt, F2), (dt * (1 - a), hist["G2"])])
            return self.solve(self.filt(R, mk), mk)
        F2, U3 = substep(U2, None, build3, ["un", "G1", "G2"])
        hist["F2"] = F2
        G3 = self.G(U3, mask)
        hist["G3"] = G3

        # substep B: F3 = F(U3), U4
        def build4(F3, mk):
            R = self.lin([(1.0, hist["un"]), (0.25 * dt, hist["F2"]), (0.25 * dt, F3),
                          (dt * b, hist["G1"]), (dt * h, hist["G2"]), (dt * z, hist["G3"])])
            return self.solve(self.filt(R, mk), mk)
        F3, U4 = substep(U3, None, build4, ["un", "F2", "G1", "G2", "G3"])
        hist["F3"] = F3
        G4 = self.G(U4, mask)
        hist["G4"] = G4

        # substep C: F4 = F(U4), u_{n+1}
        def buildn(F4, mk):
            R = self.lin([(1.0, hist["un"]), (dt / 6, hist["F2"]), (dt / 6, hist["F3"]), (2 * dt / 3, F4),
                          (dt / 6, hist["G2"]), (dt / 6, hist["G3"]), (2 * dt / 3, hist["G4"])])
            R = self.filt(R, mk)
            if P.prm["mode"] in (1, 2):
                R = self.pair_map(lambda r, m: ph.hard_clamp(r, m), mk, R)
            return R
        _, un1 = substep(U4, None, buildn, ["un", "F2", "F3", "G2", "G3", "G4"])

        udg, ufd = un1[0].copy(), un1[1].copy()
        # end of step: FD -> DG where admissible with alpha' = alpha + 1
        if P.prm["tci_on"]:
            thr2 = tci_threshold(T.N, P.prm["tci_M"], P.prm["tci_alpha"] + 1.0)
            cand = np.array([e for e in self._sel(mask, FD) if int(e) not in switched], dtype=np.int64)
            if len(cand):
                v = apply_3d(T.R, ufd[:, cand])
                r = tci_ratio(v[3:6], P.met["dg"], T, cand)
                self.near += [int(e) for e, x in zip(cand, r) if abs(x - thr2) <= 1e-12 * thr2]
                for e, x, vv in zip(cand, r, np.moveaxis(v, 1, 0)):
                    if not x > thr2:
                        mask[e] = DG
                        udg[:, e] = vv
        self.last_switched = sorted(switched)
        return dict(mask=mask, udg=udg, ufd=ufd, t=st["t"] + dt)
