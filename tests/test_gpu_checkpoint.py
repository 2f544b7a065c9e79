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


def _ckpt_parts(blob, n_elem):
    """Offsets of the checkpoint's sections (the layout ffe_save writes):
    header, initial-data parameters, state, mask, then for FD slot pools the
    element->slot map, the slot->element map and the free list."""
    import struct
    fmt = "<8s5q3qd3Qq"
    hdr = struct.unpack_from(fmt, blob, 0)
    E, ndg, nfd, fd_cap = hdr[1:5]
    nprm = hdr[8]
    off = {"nprm": 64, "free_count": 104}
    off["state"] = struct.calcsize(fmt) + 8 * nprm
    off["mask"] = off["state"] + 8 * 9 * (ndg + nfd)
    off["slot"] = off["mask"] + E
    off["free"] = off["slot"] + 4 * (E + fd_cap)
    assert E == n_elem
    return off, fd_cap


def test_corrupt_checkpoint_is_rejected_and_leaves_the_context_unchanged(ffe):
    """ffe_load checks every count and index of a checkpoint on the host before
    it touches the context: an absurd parameter count, a mask byte other than
    0/1, an FD slot outside the pool and a wrong free-slot count are each
    FFE_EINVAL, and the context keeps its state, mask and counters."""
    import struct
    cfg = W.breakdown(nx=16, ny=2, nz=1, x_half=0.5)
    a = ffe.Context(cfg)
    a.set_initial()
    a.step(3)
    blob = bytearray(a.save())
    off, _ = _ckpt_parts(blob, a.n_elem)
    a.step(2)
    U0, m0 = a.download()
    i0 = a.info()
    bad_count = bytearray(blob)
    struct.pack_into("<q", bad_count, off["nprm"], 1 << 60)
    bad_mask = bytearray(blob)
    bad_mask[off["mask"] + 3] = 7
    for bad in (bad_count, bad_mask):
        with pytest.raises(ffe.FFEError, match="FFE_EINVAL"):
            a.load_checkpoint(bytes(bad))
    U1, m1 = a.download()
    i1 = a.info()
    assert np.array_equal(U0, U1) and np.array_equal(m0, m1)
    assert (i0.t, i0.steps) == (i1.t, i1.steps)
    a.load_checkpoint(bytes(blob))   # the intact checkpoint still loads
    assert a.info().steps == 3
    a.close()

    cfgs = [W.pulsar(r_lc=3.0, chi=0.4, n_ang=1, n_rad=4, P=5, r_out=4.0),
            W.pulsar(r_lc=3.5, chi=0.2, n_ang=1, n_rad=6, P=4, r_out=6.0)]
    b = ffe.BatchContext(cfgs)
    b.set_initial()
    b.step(2)
    blob = bytearray(b.save())
    off, fd_cap = _ckpt_parts(blob, b.n_elem)
    bad_slot = bytearray(blob)
    struct.pack_into("<i", bad_slot, off["slot"], fd_cap)
    bad_free = bytearray(blob)
    (fc,) = struct.unpack_from("<q", blob, off["free_count"])
    struct.pack_into("<q", bad_free, off["free_count"], fc + 1)
    for bad in (bad_slot, bad_free):
        with pytest.raises(ffe.FFEError, match="FFE_EINVAL"):
            b.load_checkpoint(bytes(bad))
    b.load_checkpoint(bytes(blob))
    b.close()


def test_state_replacement_checks_the_mask(ffe):
    """ffe_set_state and ffe_upload refuse a mask byte other than 0/1 and, in a
    batched context, a mask that disagrees with the FD slot pool; nothing is
    replaced.  A consistent mask is accepted."""
    cfg = W.breakdown(nx=16, ny=2, nz=1, x_half=0.5)
    a = ffe.Context(cfg)
    a.set_initial()
    a.step(2)
    U, m = (t.clone() for t in a.state())
    U0, m0 = a.download()
    bad = m.clone()
    bad[5] = 2
    with pytest.raises(ffe.FFEError, match="FFE_EINVAL"):
        a.set_state(U * 2.0, bad)
    U1, m1 = a.download()
    assert np.array_equal(U0, U1) and np.array_equal(m0, m1)
    hm = torch.from_numpy(m0.copy()).pin_memory()
    hm[0] = 9
    hU = torch.from_numpy(U0).pin_memory()
    with pytest.raises(ffe.FFEError, match="FFE_EINVAL"):
        a.upload_from(hU.data_ptr(), hm.data_ptr())
    flipped = m.clone()
    flipped[0] = 1 - flipped[0]   # any 0/1 mask is valid without a slot pool
    a.set_state(U, flipped)
    a.close()

    cfgs = [W.pulsar(r_lc=3.0, chi=0.4, n_ang=1, n_rad=4, P=5, r_out=4.0)]
    b = ffe.BatchContext(cfgs)
    b.set_initial()
    U, m = (t.clone() for t in b.state())
    b.set_state(U, m)                     # the pool's own mask
    flipped = m.clone()
    flipped[0] = 1 - flipped[0]
    with pytest.raises(ffe.FFEError, match="FFE_EINVAL"):
        b.set_state(U, flipped)
    b.close()
