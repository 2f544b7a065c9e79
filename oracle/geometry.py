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

BC_NONE, BC_PERIODIC, BC_DIRICHLET, BC_NO_INCOMING, BC_STAR, BC_OUTFLOW = 0, 1, 2, 3, 4, 5


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

    def inv_map(self, e, x):
        """xi(x) for element e (the affine map inverted); x is (3, ...)."""
        c = np.asarray(self.eidx(e))
        return np.stack([2.0 * ((x[d] - self.lo[d]) / self.h[d] - c[d]) - 1.0 for d in range(3)])

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

    def __init__(self, mesh, T, fd=True):
        self.mesh, self.T = mesh, T
        E, Np, Nc = mesh.E, T.np1, T.nc
        self.E = E
        xin = tensor_points(T.x)
        xic = tensor_points(T.xc)
        self.xyz = np.stack([mesh.map(e, xin) for e in range(E)], axis=1)      # (3,E,Np,Np,Np)
        self.ijac = np.stack([mesh.inv_jac(e, xin) for e in range(E)], axis=2)  # (3,3,E,...)
        self.has_fd = fd
        if not fd:   # DG-only problem: no subcell geometry
            self.xyz_fd = self.ijac_fd = None
            self.xyz_ff = self.ijac_ff = None
            self.nbr = np.full((E, 6), -1, dtype=np.int64)
            self.bc = np.zeros((E, 6), dtype=np.int64)
            self.dg_map = np.full((E, 6, Np, Np), -1, dtype=np.int64)
            self.fd_map = None
            self._build_connectivity()
            return
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
                if not self.has_fd:
                    continue
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


# wedges of the cubed-sphere shell: (normal axis, sign); tangential axes follow cyclically
WEDGES = ((2, 1), (2, -1), (1, 1), (1, -1), (0, 1), (0, -1))


def complex_step_jacobian(fn, xi, h=1e-30):
    """d fn^i / d xi^k by complex-step differentiation (exact to rounding for
    analytic maps); fn maps (3, ...) -> (3, ...)."""
    xi = np.asarray(xi, dtype=np.complex128)
    cols = []
    for k in range(3):
        p = xi.copy()
        p[k] = p[k] + 1j * h
        cols.append(np.imag(fn(p)) / h)
    return np.stack(cols, axis=1)   # [i][k]


class ShellMesh:
    """Spherical shell r_in <= r <= r_out of six cubed-sphere wedges, each split
    into n_ang x n_ang x n_rad elements (Sec. IV.B).  [reading] Within a wedge the
    logical coordinates (eta_a, eta_b, eta_r) in [-1,1]^3 map to
    X = tan(pi eta_a/4), Y = tan(pi eta_b/4) (equiangular) and
    r = r_in (r_out/r_in)^((eta_r+1)/2) (logarithmic), the point being
    r (sigma e_n + X e_t1 + Y e_t2) / sqrt(1 + X^2 + Y^2); elements split the
    logical cube uniformly.  Element e = ia + na (ib + na (ir + nr w)); the
    reference direction xi^3 is radial; face 4 of ir = 0 lies on r_in, face 5
    of ir = nr-1 on r_out.

    spin = a != 0: the shell of the black-hole tests lives in spherical
    Kerr-Schild coordinates (App. B), so r is the Kerr-Schild radius and the
    unit vector v = (sin th cos ph, sin th sin ph, cos th) of the cubed-sphere
    map gives the Cartesian Kerr-Schild point by App. B's transformation,
    x = (r cos ph - a sin ph) sin th, y = (r sin ph + a cos ph) sin th,
    z = r cos th, i.e. x = r v + a (z^ x v).  Every surface r = const is then an
    oblate spheroid (x^2 + y^2)/(r^2 + a^2) + z^2/r^2 = 1, so a boundary at
    r_in between the two horizons lies wholly in the region that every
    characteristic leaves."""

    def __init__(self, r_in, r_out, n_ang, n_rad, bc_inner, bc_outer, spin=0.0):
        self.spin = float(spin)
        self.r_in, self.r_out = float(r_in), float(r_out)
        self.na, self.nr = int(n_ang), int(n_rad)
        self.bc_inner, self.bc_outer = bc_inner, bc_outer
        self.E = 6 * self.na * self.na * self.nr
        self.curved = True
        self._nbr = None

    def eidx(self, e):
        na, nr = self.na, self.nr
        return e % na, (e // na) % na, (e // (na * na)) % nr, e // (na * na * nr)

    def map(self, e, xi):
        ia, ib, ir, w = self.eidx(e)
        n_ax, sg = WEDGES[w]
        t1, t2 = (n_ax + 1) % 3, (n_ax + 2) % 3
        ea = -1.0 + (ia + 0.5 * (xi[0] + 1.0)) * 2.0 / self.na
        eb = -1.0 + (ib + 0.5 * (xi[1] + 1.0)) * 2.0 / self.na
        er = -1.0 + (ir + 0.5 * (xi[2] + 1.0)) * 2.0 / self.nr
        X, Y = np.tan(np.pi * ea / 4.0), np.tan(np.pi * eb / 4.0)
        r = self.r_in * (self.r_out / self.r_in) ** ((er + 1.0) / 2.0)
        rho = np.sqrt(1.0 + X * X + Y * Y)
        v = [None, None, None]
        v[n_ax] = sg / rho
        v[t1] = X / rho
        v[t2] = Y / rho
        if self.spin == 0.0:
            return np.stack([r * v[0], r * v[1], r * v[2]])
        a = self.spin
        return np.stack([r * v[0] - a * v[1], r * v[1] + a * v[0], r * v[2]])

    def inv_map(self, e, x):
        """xi(x) for element e, the map above inverted in closed form: in the
        element's wedge X = x_t1 / (sigma x_n), Y = x_t2 / (sigma x_n),
        eta_a = (4/pi) atan X, eta_b = (4/pi) atan Y,
        eta_r = 2 log(r / r_in) / log(r_out / r_in) - 1, then the element's
        affine piece of the logical cube.  Valid wherever sigma x_n > 0 (within
        45 degrees of the wedge axis and somewhat beyond)."""
        ia, ib, ir, w = self.eidx(e)
        n_ax, sg = WEDGES[w]
        t1, t2 = (n_ax + 1) % 3, (n_ax + 2) % 3
        if self.spin != 0.0:
            # undo App. B's transformation: r from the spheroid relation
            # (x^2 + y^2)/(r^2 + a^2) + z^2/r^2 = 1 (the root with r^2 > 0), then
            # (v_x, v_y) from [x; y] = [[r, -a], [a, r]] [v_x; v_y], v_z = z / r;
            # r v has the direction of v, which is all the angular part needs
            a = self.spin
            R2 = x[0] ** 2 + x[1] ** 2 + x[2] ** 2
            b = R2 - a * a
            r = np.sqrt(0.5 * (b + np.sqrt(b * b + 4.0 * a * a * x[2] ** 2)))
            q = 1.0 / (r * r + a * a)
            x = np.stack([(r * x[0] + a * x[1]) * q * r, (r * x[1] - a * x[0]) * q * r, x[2]])
        else:
            r = np.sqrt(x[0] ** 2 + x[1] ** 2 + x[2] ** 2)
        xn = sg * x[n_ax]
        ea = 4.0 / np.pi * np.arctan(x[t1] / xn)
        eb = 4.0 / np.pi * np.arctan(x[t2] / xn)
        er = 2.0 * np.log(r / self.r_in) / np.log(self.r_out / self.r_in) - 1.0
        xi0 = 2.0 * ((ea + 1.0) * self.na / 2.0 - ia) - 1.0
        xi1 = 2.0 * ((eb + 1.0) * self.na / 2.0 - ib) - 1.0
        xi2 = 2.0 * ((er + 1.0) * self.nr / 2.0 - ir) - 1.0
        return np.stack([xi0, xi1, xi2])

    def inv_jac(self, e, xi):
        J = complex_step_jacobian(lambda p: self.map(e, p), xi)
        Jm = np.moveaxis(J, (0, 1), (-2, -1))
        return np.moveaxis(np.linalg.inv(Jm), (-2, -1), (0, 1))   # [k][j] = d xi^k / d x^j

    def _face_centre(self, e, f):
        xi = np.zeros((3, 1))
        xi[f // 2, 0] = -1.0 if f % 2 == 0 else 1.0
        return self.map(e, xi)[:, 0]

    def _build(self):
        keys = {}
        nb = np.full((self.E, 6), -1, dtype=np.int64)
        scale = self.r_out
        for e in range(self.E):
            for f in range(6):
                c = self._face_centre(e, f)
                k = tuple(np.round(c / scale * 1e9).astype(np.int64))
                keys.setdefault(k, []).append((e, f))
        for k, lst in keys.items():
            if len(lst) == 2:
                (e1, f1), (e2, f2) = lst
                nb[e1, f1], nb[e2, f2] = e2, e1
            elif len(lst) != 1:
                raise RuntimeError("face matching failed")
        self._nbr = nb

    def neighbour(self, e, f):
        if self._nbr is None:
            self._build()
        nb = self._nbr[e, f]
        if nb >= 0:
            return nb, BC_NONE
        _, _, ir, _ = self.eidx(e)
        if f == 4 and ir == 0:
            return -1, self.bc_inner
        if f == 5 and ir == self.nr - 1:
            return -1, self.bc_outer
        raise RuntimeError("unmatched interior face")

    def period_shift(self, e, f):
        return np.zeros(3)
