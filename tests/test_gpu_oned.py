"""GPU against the oracle on the paper's one-dimensional tests (Sec. IV.A,
Table I, App. A) at their lowest resolution, from the nodal start and from
the FD start (every element on subcells, Sec. III.C.1)."""
import numpy as np
import pytest
import torch

import ffe_workloads as W
from oracle.problem import Problem
from oracle.stepper import Stepper
from gpu_common import compare_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ffe():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2404_01531_gb300 import ffe
    ffe.load()
    return ffe


def _run_both(ffe, cfg, nsteps):
    via = bool(cfg.get("init_via_fd", False))
    ctx = ffe.Context(cfg)
    ctx.set_initial()
    pr = Problem(cfg)
    st = pr.initial_state(via_fd=via)
    U0, m0 = ctx.download()
    assert np.array_equal(m0, st["mask"])
    S = Stepper(pr)
    near = set()
    masks = []
    for _ in range(nsteps):
        st = S.step(st)
        near |= set(S.near)
        masks.append(st["mask"].copy())
    gmasks = []
    for _ in range(nsteps):
        ctx.step(1)
        gmasks.append(ctx.download()[1])
    U, mask = ctx.download()
    near |= set(ctx.near_threshold())
    assert ctx.status() == 0
    ctx.close()
    for a, b in zip(gmasks, masks):
        assert set(np.nonzero(a != b)[0].tolist()) <= near, (np.nonzero(a != b)[0], near)
    return U, mask, st, ctx, masks


@pytest.mark.parametrize("test", list(W.ONED))
def test_oned_30_steps(ffe, test):
    cfg = W.oned(test, 0)
    U, mask, st, ctx, _ = _run_both(ffe, cfg, 30)
    compare_state(ctx, U, st, 1e-8)


def test_oned_fd_start(ffe):
    cfg = W.oned("fast_wave_kink", 0, via_fd=True)
    U, mask, st, ctx, masks = _run_both(ffe, cfg, 4)
    assert masks[-1].sum() < cfg["n"][0]
    compare_state(ctx, U, st, 1e-8)


def test_fd_start_needs_the_indicator(ffe):
    cfg = W.oned("breakdown_1d", 0)
    cfg["params"]["tci_on"] = 0
    ctx = ffe.Context(cfg)
    with pytest.raises(ffe.FFEError, match="FFE_EINVAL"):
        ctx.set_initial(via_fd=True)
    ctx.close()


def test_forced_split_alfven_wave(ffe):
    """The paper's DG/FD split experiment (Sec. IV.A.4) on a small version of
    its grid: the stationary Alfven wave on 4 x 8 x 1 cubic elements of width
    3/8 (periodic in y and z), the elements below y = 0 forced onto FD (the
    indicator off, the mask frozen), 10 steps against the oracle."""
    h = 3.0 / 8
    cfg = W.oned("alfven", 0)
    cfg.update(lo=(-0.75, -4 * h, -0.5 * h), hi=(0.75, 4 * h, 0.5 * h), n=(4, 8, 1))
    pr = Problem(cfg)
    E = pr.disc.E
    yc = pr.disc.xyz[1].reshape(E, -1).mean(axis=1)
    mask = (yc < 0).astype(np.uint8)
    assert 0 < mask.sum() < E
    ctx = ffe.Context(cfg)
    ctx.set_initial()
    U0, _ = ctx.state()
    ctx.set_state(U0.clone(), torch.from_numpy(mask).cuda())
    ctx.set_initial(keep_mask=True)
    ctx.freeze_mask(True)
    st = pr.initial_state()
    st["mask"] = mask.copy()
    for e in np.nonzero(mask)[0]:
        st["ufd"][:, e] = pr.initial(pr.disc.xyz_fd[:, e].reshape(3, -1)).reshape((9,) + pr.disc.xyz_fd.shape[2:])
    pr.prm["tci_on"] = 0
    S = Stepper(pr)
    for _ in range(10):
        st = S.step(st)
    ctx.step(10)
    U, m = ctx.download()
    assert np.array_equal(m, mask)
    assert ctx.status() == 0
    compare_state(ctx, U, st, 1e-8)
    ctx.close()
