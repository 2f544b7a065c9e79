"""Element meshes for the oracle (Sec. III.A domain decomposition; Sec. IV.B
cubed-sphere shell).  Test infrastructure only.

A mesh is a set of elements, each a map x(xi) from the reference cube
[-1,1]^3.  Everything the operators need is tabulated here by brute force:
node and subcell-centre coordinates, inverse Jacobians d xi^k / d x^j, and, for
each element face, the neighbour element plus a node-by-node (DG) and
cell-by-cell (FD ghost) correspondence found by matching physical coordinates.

Index conventions: node arrays are [..., e, k, j, i] with i along xi^1 (x
fastest); face f = 2 d + s, d the reference direction (0: xi^1, 1: xi^2,
2: xi^3), s = 0 the face at xi^d = -1, s = 1 at xi^d = +1.
"""
import numpy as np

BC_NONE, BC_PERIODIC, BC_DIRICHLET, BC_NO_INCOMING, BC_STAR = 0, 1, 2, 3, 4


def axis_of(d):
    """Array axis of reference direction d in an [e, k, j, i] block."""
    return 3 - d


def face_slice(d, s, n):
    """Index tuple selecting face (d, s) of an (n, n, n) block [k, j, i]."""
    idx = [slice(None)] * 3
    idx[2 - d] = 0 if s == 0 else n - 1
    return tuple(idx)


def layer_slice(d, s, n, g):
    """Index tuple for the g-th layer (g = 0 outermost) inward from face (d, s)."""
    idx = [slice(None)] * 3
    idx[2 - d] = g if s == 0 else n - 1 - g
    return tuple(idx)


class BoxMesh:
    """Uniform Cartesian box [lo, hi] split into n[0] x n[1] x n[2] affine
    elements; element e = ex + n0 (ey + n1 ez).  `bc[d]` is BC_PERIODIC or a
    physical kind applied at both ends of axis d."""

    def __init__(self, lo, hi, n, bc):
        self.lo, self.hi = np.asarray(lo, float), np.asarray(hi, float)
        self.n = tuple(int(v) for v in n)
        self.bc = tuple(bc)
        self.h = (self.hi - self.lo) / np.asarray(self.n)
        self.E = self.n[0] * self.n[1] * self.n[2]
        self.curved = False

    def eidx(self, e):
        n0, n1, _ = self.n
        return e % n0, (e // n0) % n1, e // (n0 * n1)

    def map(self, e, xi):
        """x(xi) for element e; xi is (3, ...)."""
        c = np.asarray(self.eidx(e))
        out = []
        for d in range(3):
            out.append(self.lo[d] + (c[d] + 0.5 * (xi[d] + 1.0)) * self.h[d])
        return np.stack(out)

    def inv_jac(self, e, xi):
        """d xi^k / d x^j = diag(2/h)."""
        shape = np.shape(xi)[1:]
        J = np.zeros((3, 3) + shape)
        for d in range(3):
            J[d, d] = 2.0 / self.h[d]
        return J

    def neighbour(self, e, f):
        """(neighbour element or -1, boundary kind)."""
        d, s = f // 2, f % 2
        c = list(self.eidx(e))
        c[d] += 1 if s == 1 else -1
        if 0 <= c[d] < self.n[d]:
            return c[0] + self.n[0] * (c[1] + self.n[1] * c[2]), BC_NONE
        if self.bc[d] == BC_PERIODIC:
            c[d] %= self.n[d]
            return c[0] + self.n[0] * (c[1] + self.n[1] * c[2]), BC_PERIODIC
        return -1, self.bc[d]

    def period_shift(self, e, f):
        """Vector to add to the neighbour's coordinates to place it next to e."""
        d, s = f // 2, f % 2
        nb, kind = self.neighbour(e, f)
        sh = np.zeros(3)
        if kind == BC_PERIODIC:
            sh[d] = (self.hi[d] - self.lo[d]) * (-1 if s == 0 else 1)
        return sh


def tensor_points(x1):
    """(3, n, n, n) reference points [k, j, i] from 1-D points x1."""
    Z, Y, X = np.meshgrid(x1, x1, x1, indexing="ij")
    return np.stack([X, Y, Z])


class Discretisation:
    """Tabulated geometry of a mesh for one polynomial degree N."""

    def __init__(self, mesh, T):
        self.mesh, self.T = mesh, T
        E, Np, Nc = mesh.E, T.np1, T.nc
        self.E = E
        xin = tensor_points(T.x)
        xic = tensor_points(T.xc)
        self.xyz = np.stack([mesh.map(e, xin) for e in range(E)], axis=1)      # (3,E,Np,Np,Np)
        self.ijac = np.stack([mesh.inv_jac(e, xin) for e in range(E)], axis=2)  # (3,3,E,...)
        self.xyz_fd = np.stack([mesh.map(e, xic) for e in range(E)], axis=1)
        self.ijac_fd = np.stack([mesh.inv_jac(e, xic) for e in range(E)], axis=2)
        # FD face points: for direction d, faces at xi^d = -1 + m dxi, m = 0..Nc
        xf = -1.0 + np.arange(Nc + 1) * (2.0 / Nc)
        self.xyz_ff, self.ijac_ff = [], []
        for d in range(3):
            axes = [T.xc, T.xc, T.xc]
            axes[d] = xf
            Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
            pts = np.stack([X, Y, Z])
            self.xyz_ff.append(np.stack([mesh.map(e, pts) for e in range(E)], axis=1))
            self.ijac_ff.append(np.stack([mesh.inv_jac(e, pts) for e in range(E)], axis=2))
        self.nbr = np.full((E, 6), -1, dtype=np.int64)
        self.bc = np.zeros((E, 6), dtype=np.int64)
        self.dg_map = np.full((E, 6, Np, Np), -1, dtype=np.int64)      # neighbour flat node index
        self.fd_map = np.full((E, 6, 3, Nc, Nc), -1, dtype=np.int64)   # neighbour flat cell index
        self._build_connectivity()

    def _build_connectivity(self):
        mesh, T = self.mesh, self.T
        Np, Nc = T.np1, T.nc
        for e in range(self.E):
            for f in range(6):
                nb, kind = mesh.neighbour(e, f)
                self.nbr[e, f], self.bc[e, f] = nb, kind
                if nb < 0:
                    continue
                d, s = f // 2, f % 2
                shift = mesh.period_shift(e, f)
                mine = self.xyz[:, e][(slice(None),) + face_slice(d, s, Np)].reshape(3, -1)
                theirs = (self.xyz[:, nb].reshape(3, -1) + shift[:, None])
                dist = np.linalg.norm(mine[:, :, None] - theirs[:, None, :], axis=0)
                j = np.argmin(dist, axis=1)
                assert np.all(dist[np.arange(len(j)), j] < 1e-9 * (1 + np.abs(mine).max()))
                self.dg_map[e, f] = j.reshape(Np, Np)
                # FD ghosts: my face points (tangential cell centres on the face)
                # matched to the neighbour's; layer g of the neighbour counted from its face
                fpts = self.xyz_ff[d][:, e][(slice(None),) + layer_slice(d, s, Nc + 1, 0)].reshape(3, -1)
                best = None
                for f2 in range(6):
                    d2, s2 = f2 // 2, f2 % 2
                    their = self.xyz_ff[d2][:, nb][(slice(None),) + layer_slice(d2, s2, Nc + 1, 0)].reshape(3, -1) + shift[:, None]
                    dd = np.linalg.norm(fpts[:, :, None] - their[:, None, :], axis=0)
                    jj = np.argmin(dd, axis=1)
                    if np.all(dd[np.arange(len(jj)), jj] < 1e-9 * (1 + np.abs(fpts).max())):
                        best = (f2, jj)
                        break
                assert best is not None
                f2, jj = best
                d2, s2 = f2 // 2, f2 % 2
                cell_idx = np.arange(Nc ** 3).reshape(Nc, Nc, Nc)
                for g in range(3):
                    layer = cell_idx[layer_slice(d2, s2, Nc, g)].reshape(-1)
                    # face-point index in the neighbour's face ordering == cell index in its layer ordering
                    self.fd_map[e, f, g] = layer[jj].reshape(Nc, Nc)

    def min_spacing(self):
        """(Delta x)_min: smallest physical distance between adjacent LGL nodes
        along element grid lines (Sec. III.B, DG time step)."""
        x = self.xyz
        best = np.inf
        for ax in (2, 3, 4):
            dx = np.diff(x, axis=ax)
            best = min(best, np.sqrt(np.sum(dx ** 2, axis=0)).min())
        return best
