"""CUDA path vs the oracle on the same seeded/analytic inputs (through the C ABI).

Bars: 1e-11 relative after one right-hand side, 1e-8 after 100 steps, masks
identical except elements the indicator saw within 1e-12 of its threshold."""
import numpy as np
import pytest

import ffe_workloads as W
from gpu_common import compare_state, rel_err_split
from oracle.dg import rhs_dg
from oracle.fd import rhs_fd
from oracle.problem import Problem
from oracle.stepper import Stepper, tci_ratio

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
    Uh = ctx.join(st["udg"], st["ufd"])
    U = torch.from_numpy(Uh).cuda()
    m = torch.from_numpy(st["mask"].astype(np.uint8)).cuda()
    ctx.set_state(U, m)
    out = torch.zeros_like(U)
    ctx.rhs(U, out)
    torch.cuda.synchronize()
    gdg, gfd = ctx.split(out.cpu().numpy())
    odg = rhs_dg(st, pr.disc, pr.met, pr.prm)
    ofd = rhs_fd(st, pr.disc, pr.met, pr.prm)
    ctx.close()
    return rel_err_split(gdg, odg, gfd, ofd, st["mask"] == 0).max()


def test_rhs_fast_wave_full_size(ffe):
    cfg = W.fast_wave()
    pr = Problem(cfg)
    st = pr.initial_state()
    assert _rhs_parity(ffe, cfg, st, pr) <= 1e-11


@pytest.mark.parametrize("P", [3, 4, 5])
def test_rhs_random_periodic_all_dg(ffe, P):
    """Random data (nonzero q, eta > 0) on a 3x2x2 periodic box, ragged P."""
    cfg = W.fast_wave(n=3, P=P)
    cfg["n"] = (3, 2, 2)
    cfg["params"]["eta"] = 7.0
    pr = Problem(cfg)
    rng = np.random.default_rng(100 + P)
    E = pr.disc.E
    st = dict(mask=np.zeros(E, np.uint8), udg=rng.normal(size=(9, E, P + 1, P + 1, P + 1)) + 0.5,
              ufd=np.zeros((9, E, 2 * P + 1, 2 * P + 1, 2 * P + 1)))
    assert _rhs_parity(ffe, cfg, st, pr) <= 1e-11


def test_rhs_mixed_dg_fd_dirichlet(ffe):
    """Breakdown box (Dirichlet x ends): half the elements FD with random data,
    every kind of face (DG-DG, DG-FD, FD-FD, FD-boundary, DG-boundary)."""
    cfg = W.breakdown(nx=6, ny=2, nz=2, x_half=0.1875)
    pr = Problem(cfg)
    rng = np.random.default_rng(7)
    E = pr.disc.E
    mask = (rng.random(E) < 0.5).astype(np.uint8)
    st = dict(mask=mask, udg=rng.normal(size=(9, E, 6, 6, 6)) + 1.0, ufd=rng.normal(size=(9, E, 11, 11, 11)) + 1.0)
    assert _rhs_parity(ffe, cfg, st, pr) <= 1e-11


def test_rhs_breakdown_full_size(ffe):
    """The 64x8x8 breakdown workload after one oracle step (current sheet on FD)."""
    cfg = W.breakdown()
    pr = Problem(cfg)
    st = pr.initial_state()
    st = Stepper(pr).step(st)
    assert st["mask"].sum() > 0
    assert _rhs_parity(ffe, cfg, st, pr) <= 1e-11


def test_tci_ratio_matches(ffe):
    cfg = W.breakdown(nx=8, ny=2, nz=2, x_half=0.25)
    pr = Problem(cfg)
    ctx = ffe.Context(cfg)
    ctx.set_initial()
    rng = np.random.default_rng(3)
    E = pr.disc.E
    udg = rng.normal(size=(9, E, 6, 6, 6)) * np.linspace(0.1, 3, E)[None, :, None, None, None] + 1.0
    U = torch.from_numpy(ctx.join(udg, np.zeros((9, E, 11, 11, 11)))).cuda()
    r = torch.zeros(E, dtype=torch.float64, device="cuda")
    ctx.tci_ratio(U, r)
    ro = tci_ratio(udg[3:6], pr.met["dg"], pr.T, np.arange(E))
    np.testing.assert_allclose(r.cpu().numpy(), ro, rtol=1e-12)
    ctx.close()


def _run_both(ffe, cfg, nsteps):
    ctx = ffe.Context(cfg)
    ctx.set_initial()
    pr = Problem(cfg)
    st = pr.initial_state()
    U0, m0 = ctx.download()
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
    ctx.close()
    diff = np.nonzero(mask != st["mask"])[0]
    assert set(diff.tolist()) <= near, (diff, near)
    return U, mask, st, ctx


def test_step_fast_wave_100_steps(ffe):
    cfg = W.fast_wave()
    U, mask, st, ctx = _run_both(ffe, cfg, 100)
    assert mask.sum() == 0
    compare_state(ctx, U, st, 1e-8)


@pytest.mark.parametrize("mode", [W.RELAX, W.RELAX_THEN_HARD, W.HARD])
def test_step_breakdown_small(ffe, mode):
    cfg = W.breakdown(nx=16, ny=2, nz=1, x_half=0.5, mode=mode)
    U, mask, st, ctx = _run_both(ffe, cfg, 30)
    assert mask.sum() > 0
    compare_state(ctx, U, st, 1e-8)


def test_step_cleaning_mode_single_element_periodic(ffe):
    """Degenerate mesh: one element, periodic in every direction (its own neighbour)."""
    cfg = W.cleaning_mode(n=1)
    U, mask, st, ctx = _run_both(ffe, cfg, 20)
    compare_state(ctx, U, st, 1e-8)


def test_rhs_mixed_dg_fd_dirichlet_small_chunks(ffe):
    """The mixed box with the FD list walked in chunks of 5 elements (the
    chunk offsets w0 > 0 of the ghost fill, flux and update kernels)."""
    cfg = W.breakdown(nx=6, ny=2, nz=2, x_half=0.1875)
    cfg["params"]["fd_chunk"] = 5
    pr = Problem(cfg)
    rng = np.random.default_rng(8)
    E = pr.disc.E
    mask = (rng.random(E) < 0.6).astype(np.uint8)
    assert mask.sum() > 10
    st = dict(mask=mask, udg=rng.normal(size=(9, E, 6, 6, 6)) + 1.0, ufd=rng.normal(size=(9, E, 11, 11, 11)) + 1.0)
    assert _rhs_parity(ffe, cfg, st, pr) <= 1e-11


def test_step_breakdown_slab_100_steps_chunked(ffe):
    """The breakdown workload's element width and x extent (64 elements along
    x, one across y and z), 100 steps with the indicator switching elements,
    the FD list walked one element per chunk."""
    cfg = W.breakdown(nx=64, ny=1, nz=1, x_half=2.0)
    cfg["params"]["fd_chunk"] = 1
    U, mask, st, ctx = _run_both(ffe, cfg, 100)
    assert mask.sum() >= 2
    compare_state(ctx, U, st, 1e-8)


def test_step_breakdown_with_an_fd_slot_pool(ffe):
    """A single context whose FD block is a pool of 16 slots (half its 32
    elements): elements take a slot when they switch to FD and return it at
    FD -> DG; the steps equal the oracle's as with one slot per element, and
    the state vector is smaller by the unused FD blocks."""
    cfg = W.breakdown(nx=16, ny=2, nz=1, x_half=0.5)
    cfg["params"]["fd_capacity"] = 16
    ctx0 = ffe.Context(W.breakdown(nx=16, ny=2, nz=1, x_half=0.5))
    n_full = ctx0.n_state
    ctx0.close()
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
    assert 0 < mask.sum() <= 16
    assert ctx.n_state == 9 * (ctx.n_dg + 16 * ctx.nc ** 3) < n_full
    compare_state(ctx, U, st, 1e-8)
    ctx.close()
