"""Hand-written adjoint on the GPU: vector-Jacobian products against central
finite differences of the forward kernels, and the luminosity gradient against
the oracle's complex-step gradient (frozen branches, all-DG masks)."""
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


def _tiny(eta=1e5):
    cfg = W.adjoint_pulsar(tiny=True)
    cfg["params"].update(tci_on=0, eta=eta)
    return cfg


def _perturbed_state(ctx, seed, amp=0.05):
    ctx.set_initial()
    U, m = ctx.state()
    g = torch.Generator(device="cpu").manual_seed(seed)
    nd = 9 * ctx.n_dg
    U = U.clone()
    U[:nd] += amp * torch.randn(nd, generator=g, dtype=torch.float64).cuda() * U[:nd].abs().max()
    U[nd:] = 0
    return U, m.clone()


@pytest.mark.parametrize("eta", [0.0, 50.0])
def test_rhs_vjp_matches_finite_differences(ffe, eta):
    ctx = ffe.Context(_tiny(eta))
    U, m = _perturbed_state(ctx, 1)
    ctx.set_state(U, m)
    nd = 9 * ctx.n_dg
    g = torch.Generator(device="cpu").manual_seed(2)
    lam = torch.zeros_like(U)
    lam[:nd] = torch.randn(nd, generator=g, dtype=torch.float64).cuda()
    dlt = torch.zeros_like(U)
    dlt[:nd] = torch.randn(nd, generator=g, dtype=torch.float64).cuda() * U[:nd].abs().max()
    vjp = torch.zeros_like(U)
    ctx.rhs_vjp(U, lam, vjp)
    # central-difference truncation on this state is ~1e-8 relative at h = 1e-6
    # and ~1e-10 at h = 1e-7 (measured against a complex-step derivative on the CPU)
    h = 1e-7
    Fp, Fm = torch.zeros_like(U), torch.zeros_like(U)
    ctx.rhs(U + h * dlt, Fp)
    ctx.rhs(U - h * dlt, Fm)
    fd = float(torch.dot(lam[:nd], (Fp[:nd] - Fm[:nd]) / (2 * h)))
    ad = float(torch.dot(vjp[:nd], dlt[:nd]))
    assert abs(ad - fd) <= 1e-7 * abs(fd), (ad, fd)
    ctx.close()


def test_adjoint_step_matches_finite_differences(ffe):
    """lambda_n . delta = lambda_{n+1} . (d step/d u) delta, one full IMEX step
    with the stiff current (eta = 1e5), filter and star / no-incoming boundaries."""
    ctx = ffe.Context(_tiny())
    U, m = _perturbed_state(ctx, 3, amp=0.02)
    nd = 9 * ctx.n_dg
    g = torch.Generator(device="cpu").manual_seed(4)
    lam = torch.zeros_like(U)
    lam[:nd] = torch.randn(nd, generator=g, dtype=torch.float64).cuda()
    dlt = torch.zeros_like(U)
    dlt[:nd] = torch.randn(nd, generator=g, dtype=torch.float64).cuda() * U[:nd].abs().max()
    out = torch.zeros_like(U)
    ctx.adjoint_step(U, lam, out)

    def step(V):
        ctx.set_state(V, m)
        ctx.step(1)
        return ctx.state()[0].clone()
    # with eta dt ~ 1e3 the central difference of one step is off by ~3e-6 relative
    # at h = 1e-7 and ~3e-9 at h = 1e-8 (complex-step comparison on the CPU)
    h = 1e-8
    fd = float(torch.dot(lam[:nd], (step(U + h * dlt)[:nd] - step(U - h * dlt)[:nd]) / (2 * h)))
    ad = float(torch.dot(out[:nd], dlt[:nd]))
    assert abs(ad - fd) <= 1e-6 * abs(fd), (ad, fd)
    ctx.close()


def test_luminosity_gradient_matches_oracle_complex_step(ffe):
    """d Lbar/d (mu, chi, Omega) over a few steps on the tiny shell, r_L = 1.5:
    GPU adjoint vs the oracle's complex-step derivative of the whole evolution,
    and the exact homogeneity mu dLbar/dmu = 2 Lbar."""
    from oracle.adjoint import lbar, lbar_gradient_complex_step
    from paper_2404_01531_gb300.adjoint import luminosity_gradient
    cfg = _tiny()
    nsteps, rL = 6, 1.5
    ctx = ffe.Context(cfg)
    ctx.set_initial()
    L, g, _ = luminosity_gradient(ctx, nsteps, r_L=rL, every=4)
    Lo = lbar(cfg, nsteps, r_L=rL)
    go = lbar_gradient_complex_step(cfg, nsteps, r_L=rL)
    assert abs(L - Lo) <= 1e-9 * abs(Lo)
    np.testing.assert_allclose(g, go, rtol=1e-6)
    mu = cfg["initial"][1]["mu"]
    assert abs(mu * g[0] - 2 * L) <= 1e-9 * abs(L)
    ctx.close()


def _with(cfg, mu=None, chi=None, omega=None):
    cfg = dict(cfg)
    kind, kw = cfg["initial"]
    kw = dict(kw)
    if mu is not None:
        kw["mu"] = mu
    if chi is not None:
        kw["chi"] = chi
    cfg["initial"] = (kind, kw)
    cfg["params"] = dict(cfg["params"])
    if omega is not None:
        cfg["params"]["omega_star"] = omega
    return cfg


def test_luminosity_gradient_matches_central_differences(ffe):
    """d Lbar/d (mu, chi, Omega) through r = 1.5 over 10 steps against central
    differences of the GPU forward run with a relative step of 1e-6."""
    from paper_2404_01531_gb300.adjoint import lbar_forward, luminosity_gradient
    cfg = _tiny()
    nsteps, rL = 10, 1.5
    ctx = ffe.Context(cfg)
    ctx.set_initial()
    L, g, _ = luminosity_gradient(ctx, nsteps, r_L=rL, every=4)
    ctx.close()
    base = dict(mu=cfg["initial"][1]["mu"], chi=cfg["initial"][1]["chi"], omega=cfg["params"]["omega_star"])
    for k, name in enumerate(("mu", "chi", "omega")):
        h = 1e-6 * base[name]
        vals = []
        for sgn in (1, -1):
            c = ffe.Context(_with(cfg, **{name: base[name] + sgn * h}))
            c.set_initial()
            vals.append(lbar_forward(c, nsteps, rL))
            c.close()
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * abs(fd), (name, g[k], fd)


def test_autograd_function_step(ffe):
    from paper_2404_01531_gb300.adjoint import Step
    ctx = ffe.Context(_tiny())
    ctx.set_initial()
    U0 = ctx.state()[0].clone().requires_grad_(True)
    U1 = Step.apply(U0, ctx)
    U2 = Step.apply(U1, ctx)
    w = torch.zeros_like(U2)
    w[: 9 * ctx.n_dg] = 1.0
    (U2 * w).sum().backward()
    assert torch.isfinite(U0.grad).all() and float(U0.grad.abs().sum()) > 0
    ctx.close()
