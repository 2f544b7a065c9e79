"""1-D operator tables of the nodal DG and FD-subcell discretisations.

Sec. III.A (nodal expansion on Legendre-Gauss-Lobatto points, modal Legendre
expansion, exponential filter) and Sec. III.C.1/III.C.3 (subcell grid of 2N+1
cells, projections, modal troubled-cell indicator).  Test infrastructure only.
"""
import numpy as np


def legendre(n, x):
    """L_n(x) and L_n'(x) by the three-term (Bonnet) recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0, p1 = np.ones_like(x), x.copy()
    if n == 0:
        return p0, np.zeros_like(x)
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    # derivative from (1 - x^2) L_n' = n (L_{n-1} - x L_n), valid off +-1
    with np.errstate(divide="ignore", invalid="ignore"):
        d = n * (p0 - x * p1) / (1.0 - x * x)
    end = np.abs(x) == 1.0
    d = np.where(end, np.sign(x) ** (n + 1) * n * (n + 1) / 2.0, d)
    return p1, d


def lgl_nodes_weights(N):
    """LGL nodes (the end points and the roots of L_N') and weights
    w_j = 2 / (N (N+1) L_N(x_j)^2)  (Sec. III.A: LGL collocation, mass lumping)."""
    c = np.zeros(N + 1)
    c[N] = 1.0
    interior = np.sort(np.polynomial.legendre.legroots(np.polynomial.legendre.legder(c)).real) if N > 1 else np.zeros(0)
    # polish the interior roots by Newton on L_N' (second derivative from the
    # Legendre ODE: (1-x^2) L'' = 2x L' - N(N+1) L)
    for _ in range(4):
        L, dL = legendre(N, interior)
        d2 = (2 * interior * dL - N * (N + 1) * L) / (1 - interior ** 2)
        interior = interior - dL / d2
    x = np.concatenate([[-1.0], interior, [1.0]])
    x = 0.5 * (x - x[::-1])  # exact antisymmetry
    L, _ = legendre(N, x)
    w = 2.0 / (N * (N + 1) * L ** 2)
    return x, w


def diff_matrix(N, x):
    """Nodal differentiation D_ij = l_j'(x_i) on LGL points (closed form)."""
    L, _ = legendre(N, x)
    D = np.zeros((N + 1, N + 1))
    for i in range(N + 1):
        for j in range(N + 1):
            if i != j:
                D[i, j] = L[i] / (L[j] * (x[i] - x[j]))
    D[0, 0] = -N * (N + 1) / 4.0
    D[N, N] = N * (N + 1) / 4.0
    return D


def vandermonde(N, x):
    """V_ij = L_j(x_i): nodal values of the Legendre modes (modal expansion, Sec. III.A)."""
    return np.stack([legendre(j, x)[0] for j in range(N + 1)], axis=1)


def lagrange_matrix(x_nodes, y):
    """M_aj = l_j(y_a), the Lagrange basis on x_nodes evaluated at points y."""
    n = len(x_nodes)
    M = np.ones((len(y), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                M[:, j] *= (y - x_nodes[m]) / (x_nodes[j] - x_nodes[m])
    return M


def filter_sigma(N, a=36.0, b=50.0):
    """sigma_n = exp(-a (n/N)^(2b))  (exponential filter, Sec. III.A)."""
    n = np.arange(N + 1, dtype=np.float64)
    return np.exp(-a * (n / N) ** (2 * b))


def filter_matrix(N, x, a=36.0, b=50.0):
    """1-D nodal filter V diag(sigma) V^-1; the 3-D filter is its tensor cube."""
    V = vandermonde(N, x)
    return V @ np.diag(filter_sigma(N, a, b)) @ np.linalg.inv(V)


def tci_lowpass_matrix(N, x, M):
    """1-D nodal projection onto Legendre modes p <= N - M.

    [reading] Sec. III.C.3 writes the filtered-out part u^ as a sum with all three
    mode indices >= M; read literally a 1-D profile would never be flagged.  The
    oracle keeps every mode with max(p,q,r) >= N+1-M in u^, i.e. u^ = u - (Pi x Pi
    x Pi) u with Pi the projection onto p <= N - M ("lowest modes kept")."""
    V = vandermonde(N, x)
    keep = (np.arange(N + 1) <= N - M).astype(np.float64)
    return V @ np.diag(keep) @ np.linalg.inv(V)


def subcell_centres(N):
    """Centres of the 2N+1 uniform subcells of [-1, 1], dxi = 2/(2N+1) (Sec. III.C.1)."""
    nc = 2 * N + 1
    return -1.0 + (np.arange(nc) + 0.5) * (2.0 / nc)


def dg_to_fd_matrix(N, x):
    """DG -> FD: evaluate the nodal polynomial at the subcell centres (Sec. III.C.1)."""
    return lagrange_matrix(x, subcell_centres(N))


def fd_to_dg_matrix(N, x, width=6):
    """FD -> DG: [reading] the 'general sixth-order accurate interpolation' of
    Sec. III.C.1 is taken as 1-D Lagrange interpolation through the `width`=6
    subcell centres nearest each LGL node, the stencil shifted to stay inside the
    element; its tensor cube maps subcell values to LGL nodes."""
    xc = subcell_centres(N)
    nc = len(xc)
    R = np.zeros((N + 1, nc))
    dxi = 2.0 / nc
    for j, xj in enumerate(x):
        pos = (xj + 1.0) / dxi - 0.5  # fractional subcell index of the node
        start = int(np.floor(pos)) - (width // 2 - 1)
        start = min(max(start, 0), nc - width)
        R[j, start:start + width] = lagrange_matrix(xc[start:start + width], np.array([xj]))[0]
    return R


class Tables:
    """All 1-D tables for one polynomial degree N."""

    def __init__(self, N, filter_a=36.0, filter_b=50.0, tci_M=3):
        self.N = N
        self.np1 = N + 1
        self.nc = 2 * N + 1
        self.x, self.w = lgl_nodes_weights(N)
        self.D = diff_matrix(N, self.x)
        self.V = vandermonde(N, self.x)
        self.F = filter_matrix(N, self.x, filter_a, filter_b)
        self.Pi = tci_lowpass_matrix(N, self.x, tci_M)
        self.P = dg_to_fd_matrix(N, self.x)
        self.R = fd_to_dg_matrix(N, self.x)
        self.xc = subcell_centres(N)
        self.w0 = self.w[0]
