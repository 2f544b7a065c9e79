"""The reciprocal inside the WENO5-Z weights (hardware approximation refined by
two Newton-Raphson steps) against the correctly rounded IEEE quotient 1/x that
PyTorch's CUDA division returns, in units in the last place."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ffe():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2404_01531_gb300 import ffe
    ffe.load()
    return ffe


def _ulps(a, b):
    """Distance in ulps of positive finite doubles (their bit patterns are ordered)."""
    return (a.view(torch.int64) - b.view(torch.int64)).abs()


def test_recip_within_one_ulp_over_the_range(ffe):
    g = torch.Generator(device="cuda").manual_seed(1531)
    n = 1 << 22
    # log-uniform over [1e-300, 1e300] with uniform mantissas, plus the
    # denominators of the WENO weights at the default eps (1e-240 .. 1e40)
    e = torch.rand(n, generator=g, device="cuda", dtype=torch.float64) * 600.0 - 300.0
    x = torch.pow(10.0, e)
    x = torch.cat([x, torch.pow(10.0, torch.rand(n, generator=g, device="cuda", dtype=torch.float64) * 280 - 240)])
    # exact powers of two, their neighbours and mantissas next to 1 and 2
    k = torch.arange(-1000, 1001, device="cuda", dtype=torch.float64)
    p2 = torch.pow(2.0, k)
    bits = p2.view(torch.int64)
    x = torch.cat([x, p2, (bits + 1).view(torch.float64), (bits - 1).view(torch.float64),
                   (bits + (1 << 51) - 1).view(torch.float64)])
    y = torch.empty_like(x)
    ffe.eval_recip(x, y)
    ref = 1.0 / x
    u = _ulps(y, ref)
    assert torch.isfinite(y).all()
    assert int(u.max()) <= 1, int(u.max())
    # and most quotients are the correctly rounded ones
    assert float((u == 0).double().mean()) > 0.9


def test_recip_in_place_and_empty(ffe):
    x = torch.tensor([3.0, 7.0, 1e-200, 1e200], device="cuda", dtype=torch.float64)
    ref = 1.0 / x
    ffe.eval_recip(x, x)
    assert int(_ulps(x, ref).max()) <= 1
    z = torch.empty(0, device="cuda", dtype=torch.float64)
    ffe.eval_recip(z, z)
