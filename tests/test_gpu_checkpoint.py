"""Checkpoint / resume (ffe_save, ffe_load) and the pointwise constraint
diagnostics (ffe_constraints) on the GPU."""
import numpy as np
import pytest

import ffe_workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ffe():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2404_01531_gb300 import ffe
    ffe.load()
    return ffe


def test_resume_from_checkpoint_is_exact(ffe):
    """Breakdown sheet with DG<->FD switching: saving after 5 steps and
    resuming in a fresh context gives bit-identical states, masks, time and
    counters after 5 more steps (the forward kernels are deterministic)."""
    cfg = W.breakdown(nx=16, ny=2, nz=1, x_half=0.5)
    a = ffe.Context(cfg)
    a.set_initial()
    a.step(5)
    blob = a.save()
    a.step(5)
    Ua, ma = a.download()
    ia = a.info()
    b = ffe.Context(cfg)
    b.set_initial()
    b.load_checkpoint(blob)
    assert b.info().steps == 5
    b.step(5)
    Ub, mb = b.download()
    ib = b.info()
    assert ma.sum() > 0
    assert np.array_equal(ma, mb)
    assert np.array_equal(Ua, Ub)
    assert (ia.t, ia.steps, ia.node_updates, ia.fd_elem_updates) == (ib.t, ib.steps, ib.node_updates, ib.fd_elem_updates)
    a.close()
    b.close()


def test_resume_batch_with_fd_pool(ffe):
    """A batched context (its FD slots come from a pool, one slot per element
    by default): the slot map and free list are part of the checkpoint."""
    cfgs = [W.pulsar(r_lc=3.0, chi=0.4, n_ang=1, n_rad=4, P=5, r_out=4.0),
            W.pulsar(r_lc=3.5, chi=0.2, n_ang=1, n_rad=6, P=4, r_out=6.0)]
    a = ffe.BatchContext(cfgs)
    a.set_initial()
    a.step(3)
    blob = a.save()
    a.step(3)
    Ua, ma = a.download()
    b = ffe.BatchContext(cfgs)
    b.set_initial()
    b.load_checkpoint(blob)
    b.step(3)
    Ub, mb = b.download()
    assert np.array_equal(ma, mb)
    # FD slots are handed out by atomics, so compare per element, not per slot
    for i in range(len(cfgs)):
        for xa, xb in zip(a.split_instance(Ua, i), b.split_instance(Ub, i)):
            assert np.array_equal(xa, xb)
    a.close()
    b.close()


def test_checkpoint_of_another_mesh_is_rejected(ffe):
    a = ffe.Context(W.breakdown(nx=16, ny=2, nz=1, x_half=0.5))
    a.set_initial()
    blob = a.save()
    b = ffe.Context(W.breakdown(nx=8, ny=2, nz=1, x_half=0.25))
    b.set_initial()
    with pytest.raises(ffe.FFEError, match="FFE_EINVAL"):
        b.load_checkpoint(blob)
    with pytest.raises(ffe.FFEError, match="FFE_EINVAL"):
        a.load_checkpoint(blob[:100])
    a.close()
    b.close()


def test_constraints_match_the_state(ffe):
    cfg = W.breakdown(nx=16, ny=2, nz=1, x_half=0.5)
    ctx = ffe.Context(cfg)
    ctx.set_initial()
    ctx.step(10)
    U, mask = ctx.download()
    dg, fd = ctx.split(U)
    dg = dg.reshape(9, ctx.n_elem, -1)[:, mask == 0].reshape(9, -1)
    fd = fd.reshape(9, ctx.n_elem, -1)[:, mask == 1].reshape(9, -1)
    u = np.concatenate([dg, fd], axis=1)
    EB = np.abs((u[0:3] * u[3:6]).sum(0)).max()
    D = ((u[3:6] ** 2).sum(0) - (u[0:3] ** 2).sum(0)).min()
    got = ctx.constraints()
    assert mask.sum() > 0
    np.testing.assert_allclose(got, (EB, D, np.abs(u[6]).max(), np.abs(u[7]).max()), rtol=1e-12, atol=1e-15)
    ctx.close()
