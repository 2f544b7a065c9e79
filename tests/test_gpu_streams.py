"""Contexts on their own CUDA streams, advanced concurrently (the oblique
rotator's inclination sweep runs one context per inclination this way):
every context owns its device memory, step graph and scratch, so interleaved
launches on several streams give bit-for-bit the states of each context
advanced alone."""
import math

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


def test_concurrent_contexts_on_their_own_streams_equal_sequential_runs(ffe):
    cfgs = [W.pulsar(r_lc=5.0, chi=math.radians(c), n_ang=2, n_rad=4, P=5, r_out=20.0) for c in (0.0, 60.0, 90.0)]
    alone = []
    for cfg in cfgs:
        ctx = ffe.Context(cfg)
        ctx.set_initial()
        ctx.step(12)
        alone.append(ctx.download())
        assert ctx.status() == 0
        ctx.close()
    streams = [torch.cuda.Stream() for _ in cfgs]
    ctxs = [ffe.Context(cfg, stream=s) for cfg, s in zip(cfgs, streams)]
    for c in ctxs:
        c.set_initial()
    for _ in range(4):
        for c in ctxs:
            c.step(3)
    torch.cuda.synchronize()
    for c, (U, m) in zip(ctxs, alone):
        Uc, mc = c.download()
        assert c.status() == 0
        assert np.array_equal(mc, m)
        assert np.array_equal(Uc, U)
        c.close()
