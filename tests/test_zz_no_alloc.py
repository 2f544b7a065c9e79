"""The allocation-free FD right-hand side (ffe_fd_rhs_noalloc) against the
context path (ffe_rhs) and against the oracle's FD operator on the same data,
two calls in a row, with and without the derivative corrector.

It exists for callers that cannot call cudaMalloc (host applications that own
all device memory, latency-critical paths); its scratch is a fixed static
device array shared by all calls.  Every element of the periodic test box is
on FD, so every ghost holds an FD neighbour's cells, the case in which the
entry point and the context path take the ghost currents the same way.  This
file is collected last so that a run stopping at the first failure has already
run every other test."""
import numpy as np
import pytest

import ffe_workloads as W
from gpu_common import rel_err_split

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GH = 3


def extended_blocks(ufd, n):
    """[9][E][(nc+6)^3] blocks with 3 periodic ghost layers per face, from the FD
    data of a fully periodic n[0] x n[1] x n[2] box (element e = ex + n0 (ey + n1 ez))."""
    nv, E, nc = ufd.shape[0], ufd.shape[1], ufd.shape[2]
    nx, ny, nz = n
    glob = np.zeros((nv, nz * nc, ny * nc, nx * nc))
    for e in range(E):
        ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
        glob[:, ez * nc:(ez + 1) * nc, ey * nc:(ey + 1) * nc, ex * nc:(ex + 1) * nc] = ufd[:, e]
    out = np.zeros((nv, E, nc + 2 * GH, nc + 2 * GH, nc + 2 * GH))
    for e in range(E):
        ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
        iz = np.arange(ez * nc - GH, (ez + 1) * nc + GH) % (nz * nc)
        iy = np.arange(ey * nc - GH, (ey + 1) * nc + GH) % (ny * nc)
        ix = np.arange(ex * nc - GH, (ex + 1) * nc + GH) % (nx * nc)
        out[:, e] = glob[:, iz][:, :, iy][:, :, :, ix]
    return out


@pytest.mark.parametrize("corr", [1, 0])
def test_noalloc_fd_rhs_matches_context_path_twice(corr):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2404_01531_gb300 import ffe
    from oracle.fd import rhs_fd
    from oracle.problem import Problem
    cfg = W.fast_wave(n=3, P=5)
    cfg["n"] = (3, 2, 1)
    cfg["params"].update(eta=50.0, fd_corrector=corr)
    pr = Problem(cfg)
    ctx = ffe.Context(cfg)
    ctx.set_initial()
    E, P = ctx.n_elem, ctx.P
    nc = 2 * P + 1
    h = [(cfg["hi"][a] - cfg["lo"][a]) / cfg["n"][a] for a in range(3)]
    rng = np.random.default_rng(2024)
    for call in range(2):
        ufd = rng.normal(size=(9, E, nc, nc, nc)) + (1.0 + call)
        udg = np.zeros((9, E, P + 1, P + 1, P + 1))
        U = torch.from_numpy(ctx.join(udg, ufd)).cuda()
        mask = torch.ones(E, dtype=torch.uint8, device="cuda")
        ctx.set_state(U, mask)
        ref = torch.zeros_like(U)
        ctx.rhs(U, ref)
        ext = torch.from_numpy(np.ascontiguousarray(extended_blocks(ufd, cfg["n"]))).cuda()
        out = torch.full((9, E, nc, nc, nc), float("nan"), dtype=torch.float64, device="cuda")
        ffe.fd_rhs_noalloc(P, ext, h, cfg["params"]["eta"], cfg["params"]["weno_eps"], corr, out)
        torch.cuda.synchronize()
        _, rfd = ctx.split(ref.cpu().numpy())
        got = out.cpu().numpy()
        sel_dg = np.zeros(E, dtype=bool)
        err = rel_err_split(udg, udg, got, rfd, sel_dg).max()
        assert err <= 1e-11, (call, err)
        ofd = rhs_fd(dict(mask=np.ones(E, dtype=np.uint8), udg=udg, ufd=ufd), pr.disc, pr.met, pr.prm)
        err_o = rel_err_split(udg, udg, got, ofd, sel_dg).max()
        assert err_o <= 1e-11, (call, err_o)
    ctx.close()


def test_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2404_01531_gb300 import ffe
    P, n = 5, 64
    ext = torch.zeros(9 * n * (2 * P + 7) ** 3, dtype=torch.float64, device="cuda")
    out = torch.zeros(9 * n * (2 * P + 1) ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(ffe.FFEError, match="FFE_EINVAL"):
        ffe.fd_rhs_noalloc(P, ext, [0.1, 0.1, 0.1], 0.0, 1e-40, 1, out)
