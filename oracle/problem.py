"""Set up an oracle problem from a workload description.  Test infrastructure only."""
import numpy as np

from . import initial, physics as ph
from .metric import ks_metric
from .basis import Tables
from .geometry import (BoxMesh, ShellMesh, Discretisation, BC_PERIODIC, BC_DIRICHLET, BC_NO_INCOMING, BC_STAR,
                       BC_OUTFLOW)

_BC = {"periodic": BC_PERIODIC, "dirichlet": BC_DIRICHLET, "no_incoming": BC_NO_INCOMING, "star": BC_STAR,
       "outflow": BC_OUTFLOW}


class Problem:
    def __init__(self, cfg):
        self.cfg = cfg
        p = cfg["params"]
        self.T = Tables(cfg["P"], p["filter_a"], p["filter_b"], p["tci_M"])
        if cfg["kind"] == "box":
            self.mesh = BoxMesh(cfg["lo"], cfg["hi"], cfg["n"], [_BC[b] for b in cfg["bc"]])
        else:
            # shell_ks: the shell's radius is the spherical Kerr-Schild r of the
            # metric's spin (App. B)
            spin = cfg["metric"][2] if cfg.get("shell_ks") else 0.0
            self.mesh = ShellMesh(cfg["r_in"], cfg["r_out"], cfg["n_ang"], cfg["n_rad"],
                                  _BC[cfg["bc_inner"]], _BC[cfg["bc_outer"]], spin=spin)
        self.disc = Discretisation(self.mesh, self.T, fd=bool(p["tci_on"]))
        mkind, M, spin = cfg["metric"]
        d = self.disc
        if mkind == "minkowski":
            at = lambda xyz: ph.flat_metric()
        else:
            at = lambda xyz: ks_metric(xyz, M, spin)
        if d.has_fd:
            self.met = {"dg": at(d.xyz), "fd": at(d.xyz_fd), "fdface": [at(x) for x in d.xyz_ff], "at": at}
        else:
            self.met = {"dg": at(d.xyz), "fd": None, "fdface": None, "at": at}
        # lambda_max = max(alpha + |beta|_gamma) over the nodes (Sec. III.B)
        m = self.met["dg"]
        if mkind == "minkowski":
            self.lam_max = 1.0
        else:
            bl = np.einsum('ij...,j...->i...', m.gl, m.beta)
            self.lam_max = float(np.max(m.alpha + np.sqrt(np.einsum('i...,i...->...', bl, m.beta))))
        ikind, ikw = cfg["initial"]
        self.initial = lambda xyz: initial.evaluate(ikind, xyz, **ikw)
        # the algebraic-only mode has no driver current
        self.prm = dict(eta=p["eta"] if p["constraint_mode"] != 1 else 0.0, kappa_psi=p["kappa_psi"], kappa_phi=p["kappa_phi"],
                        weno_eps=p["weno_eps"], fd_corrector=p["fd_corrector"], recon=p.get("recon", 0),
                        dirichlet=self.initial, omega=p["omega_star"],
                        mode=p["constraint_mode"], filter_on=p["filter_on"], tci_on=p["tci_on"],
                        tci_alpha=p["tci_alpha"], tci_M=p["tci_M"],
                        # [reading] FD ghosts across a neighbour's face are the neighbour's
                        # data at the ghost centres of this element's grid continued past
                        # the face (Sec. III.C.1's sixth-order transfer); see fd.fill_ghosts
                        ghost_interp=bool(p.get("ghost_interp", True)))
        self.dxmin = d.min_spacing()
        # an explicit time step (the paper's tables give one) or the CFL step (Sec. III.B)
        self.dt = p["dt"] if p.get("dt", 0.0) > 0.0 else p["cfl"] * self.dxmin / self.lam_max * p["c_over_D"]

    def initial_state(self, via_fd=False):
        """Initial data on the LGL nodes, then the TCI (alpha) on every element;
        flagged elements take the initial data at their subcell centres.
        [reading] the paper initialises on the FD grid (Sec. III.C.1); here the
        nodal start is the default, as the FD start only matters for Gibbs-prone data.
        via_fd: the paper's start, every element on FD with the initial data at
        its subcell centres; the FD indicator at the end of each step returns
        the smooth ones to DG."""
        from .stepper import tci_ratio, tci_threshold
        d, T = self.disc, self.T
        udg = self.initial(d.xyz.reshape(3, -1)).reshape((9,) + d.xyz.shape[1:])
        ufd = np.zeros((9, d.E, T.nc, T.nc, T.nc)) if d.has_fd else np.zeros((9, d.E, 1, 1, 1))
        mask = np.zeros(d.E, dtype=np.uint8)
        if via_fd:
            assert d.has_fd, "an FD start needs the FD grid (indicator on)"
            mask[:] = 1
            ufd[:] = self.initial(d.xyz_fd.reshape(3, -1)).reshape((9,) + d.xyz_fd.shape[1:])
            return dict(mask=mask, udg=udg, ufd=ufd, t=0.0)
        if self.prm["tci_on"]:
            r = tci_ratio(udg[3:6], self.met["dg"], T, np.arange(d.E))
            flag = r > tci_threshold(T.N, self.prm["tci_M"], self.prm["tci_alpha"])
            for e in np.nonzero(flag)[0]:
                mask[e] = 1
                ufd[:, e] = self.initial(d.xyz_fd[:, e].reshape(3, -1)).reshape((9,) + d.xyz_fd.shape[2:])
        return dict(mask=mask, udg=udg, ufd=ufd, t=0.0)
