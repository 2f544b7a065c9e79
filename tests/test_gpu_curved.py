"""Curved meshes on the GPU vs the oracle: six-wedge shells with the
Kerr-Schild metric (DG) and flat-space rotating-star shells (DG + FD)."""
import numpy as np
import pytest

import ffe_workloads as W
from gpu_common import compare_state, rel_err_split
from oracle.dg import rhs_dg
from oracle.fd import rhs_fd
from oracle.problem import Problem
from oracle.stepper import Stepper

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ffe():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2404_01531_gb300 import ffe
    ffe.load()
    return ffe


def _full_fd(ctx, ufd):
    nc = ctx.nc
    if ufd.shape[2] == nc:
        return ufd
    return np.zeros((9, ctx.n_elem, nc, nc, nc))


def _rhs_parity(ffe, cfg, st, pr):
    ctx = ffe.Context(cfg)
    ctx.set_initial()
    U = torch.from_numpy(ctx.join(st["udg"], _full_fd(ctx, st["ufd"]))).cuda()
    m = torch.from_numpy(st["mask"].astype(np.uint8)).cuda()
    ctx.set_state(U, m)
    out = torch.zeros_like(U)
    ctx.rhs(U, out)
    torch.cuda.synchronize()
    gdg, gfd = ctx.split(out.cpu().numpy())
    odg = rhs_dg(st, pr.disc, pr.met, pr.prm)
    ofd = rhs_fd(st, pr.disc, pr.met, pr.prm) if pr.disc.has_fd else np.zeros_like(gfd)
    ctx.close()
    return rel_err_split(gdg, odg, gfd, _full_fd(ctx, ofd), st["mask"] == 0).max()


@pytest.mark.parametrize("P", [4, 5])
def test_rhs_kerr_schild_shell(ffe, P):
    """Perturbed Wald data (a = 0.9) with a finite eta: metric fluxes, sources,
    curved lift across wedge faces with orientation, Dirichlet shell faces."""
    cfg = W.wald(n_ang=2, n_rad=2, P=P, r_in=2.0, r_out=6.0)
    cfg["params"].update(eta=10.0, tci_on=0)
    pr = Problem(cfg)
    st = pr.initial_state()
    rng = np.random.default_rng(P)
    st["udg"] = st["udg"] + 0.1 * rng.normal(size=st["udg"].shape)
    assert _rhs_parity(ffe, cfg, st, pr) <= 1e-11


@pytest.mark.parametrize("corr", [0, 1])
def test_rhs_star_shell_mixed_dg_fd(ffe, corr):
    """Flat rotating-star shell, random data, random DG/FD mask: curved FD flux
    and update (with and without the corrector applied per physical flux
    component), ghost fills across wedges, star and no-incoming-Poynting states."""
    cfg = W.pulsar(r_lc=3.0, n_ang=2, n_rad=3, P=5)
    cfg["params"].update(eta=50.0, fd_corrector=corr)
    pr = Problem(cfg)
    rng = np.random.default_rng(11)
    E = pr.disc.E
    mask = (rng.random(E) < 0.4).astype(np.uint8)
    st = dict(mask=mask, udg=rng.normal(size=(9, E, 6, 6, 6)) + 1.0, ufd=rng.normal(size=(9, E, 11, 11, 11)) + 1.0)
    assert _rhs_parity(ffe, cfg, st, pr) <= 1e-11


def _run_both(ffe, cfg, nsteps, tol):
    ctx = ffe.Context(cfg)
    ctx.set_initial()
    pr = Problem(cfg)
    st = pr.initial_state()
    _, m0 = ctx.download()
    assert np.array_equal(m0, st["mask"])
    S = Stepper(pr)
    near = set()
    for _ in range(nsteps):
        st = S.step(st)
        near |= set(S.near)
    ctx.step(nsteps)
    U, mask = ctx.download()
    near |= set(ctx.near_threshold())
    assert ctx.status() == 0
    diff = np.nonzero(mask != st["mask"])[0]
    assert set(diff.tolist()) <= near, (diff, near)
    if st["ufd"].shape[2] != ctx.nc:
        st["ufd"] = _full_fd(ctx, st["ufd"])
    err = compare_state(ctx, U, st, tol)
    ctx.close()
    return err, mask


def test_step_wald_kerr_schild(ffe):
    cfg = W.wald(n_ang=2, n_rad=2, P=5, r_in=2.0, r_out=6.0)
    cfg["params"]["tci_on"] = 0
    _run_both(ffe, cfg, 20, 1e-8)


def test_step_pulsar_tiny(ffe):
    """The tiny adjoint shell (6 wedges x 2 x 2 x 4, P = 5, r in [1, 24]),
    rotating star, eta = 1e5, 5 steps with the indicator on."""
    cfg = W.adjoint_pulsar(tiny=True)
    _run_both(ffe, cfg, 5, 1e-8)
