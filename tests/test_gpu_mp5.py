"""MP5 reconstruction (FFE_RECON_MP5) on the GPU against the oracle: FD
right-hand side on random data (the limiter active at almost every face) on a
box and a curved shell, and 30 hybrid steps of the breakdown sheet."""
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


def _rhs_parity(ffe, cfg, st, pr):
    ctx = ffe.Context(cfg)
    ctx.set_initial()
    U = torch.from_numpy(ctx.join(st["udg"], st["ufd"])).cuda()
    ctx.set_state(U, torch.from_numpy(st["mask"].astype(np.uint8)).cuda())
    out = torch.zeros_like(U)
    ctx.rhs(U, out)
    torch.cuda.synchronize()
    gdg, gfd = ctx.split(out.cpu().numpy())
    ctx.close()
    return rel_err_split(gdg, rhs_dg(st, pr.disc, pr.met, pr.prm), gfd, rhs_fd(st, pr.disc, pr.met, pr.prm),
                         st["mask"] == 0).max()


def test_mp5_rhs_box_mixed(ffe):
    cfg = W.breakdown(nx=6, ny=2, nz=2, x_half=0.1875)
    cfg["params"]["recon"] = 1
    pr = Problem(cfg)
    rng = np.random.default_rng(71)
    E = pr.disc.E
    st = dict(mask=(rng.random(E) < 0.5).astype(np.uint8), udg=rng.normal(size=(9, E, 6, 6, 6)) + 1.0,
              ufd=rng.normal(size=(9, E, 11, 11, 11)) + 1.0)
    assert _rhs_parity(ffe, cfg, st, pr) <= 1e-11


def test_mp5_rhs_star_shell_mixed(ffe):
    cfg = W.pulsar(r_lc=3.0, n_ang=2, n_rad=3, P=5)
    cfg["params"].update(eta=50.0, recon=1)
    pr = Problem(cfg)
    rng = np.random.default_rng(72)
    E = pr.disc.E
    st = dict(mask=(rng.random(E) < 0.4).astype(np.uint8), udg=rng.normal(size=(9, E, 6, 6, 6)) + 1.0,
              ufd=rng.normal(size=(9, E, 11, 11, 11)) + 1.0)
    assert _rhs_parity(ffe, cfg, st, pr) <= 1e-11


def test_mp5_breakdown_30_steps(ffe):
    cfg = W.breakdown(nx=16, ny=2, nz=1, x_half=0.5)
    cfg["params"]["recon"] = 1
    ctx = ffe.Context(cfg)
    ctx.set_initial()
    pr = Problem(cfg)
    st = pr.initial_state()
    S = Stepper(pr)
    near = set()
    for _ in range(30):
        st = S.step(st)
        near |= set(S.near)
    ctx.step(30)
    U, mask = ctx.download()
    near |= set(ctx.near_threshold())
    assert ctx.status() == 0
    assert set(np.nonzero(mask != st["mask"])[0].tolist()) <= near
    assert mask.sum() > 0
    compare_state(ctx, U, st, 1e-8)
    ctx.close()


def test_mp5_has_no_adjoint(ffe):
    cfg = W.adjoint_pulsar(tiny=True, steps=2)
    cfg["params"].update(recon=1, tci_on=0)
    ctx = ffe.Context(cfg)
    ctx.set_initial()
    U, _ = ctx.state()
    lam = torch.zeros_like(U)
    out = torch.zeros_like(U)
    with pytest.raises(ffe.FFEError, match="FFE_ENOTIMPL"):
        ctx.rhs_vjp(U.clone(), lam, out)
    ctx.close()
