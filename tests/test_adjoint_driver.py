"""The checkpointed luminosity-gradient driver (paper_2404_01531_gb300.adjoint)
sequences library calls only: forward steps with a checkpoint every `every`
steps, then per segment (the last one ragged) the recomputation of its states,
the luminosity seeds lambda_{n+1} += dL(u_{n+1})/du / N and the step adjoints
in reverse order, and the Omega derivative summed over the steps.  Here it
drives a fake context on the CPU whose "step" is a small nonlinear map
u -> tanh(A u) + Omega b with a quadratic "luminosity", and its gradient is
compared with the exact forward-mode derivative of the same map."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")


class FakeContext:
    """The calls luminosity_gradient makes, on a toy map (n doubles of state)."""

    def __init__(self, n=6, mu=1.3, chi=0.7, omega=0.4, seed=5):
        rng = np.random.default_rng(seed)
        t = lambda a: torch.tensor(a, dtype=torch.float64)
        self.A = t(rng.normal(size=(n, n)) / math.sqrt(n))
        self.b = t(rng.normal(size=n))
        q = rng.normal(size=(n, n))
        self.Q = t(q @ q.T / n + np.eye(n))
        self.v, self.w = t(rng.normal(size=n)), t(rng.normal(size=n))
        self.mu, self.chi, self.omega = mu, chi, omega
        self.U = self.initial()
        self.mask = torch.zeros(3, dtype=torch.uint8)

    def initial(self):
        return self.mu * self.v + math.sin(self.chi) * self.w

    def f(self, U):
        return torch.tanh(self.A @ U) + self.omega * self.b

    def state(self):
        return self.U, self.mask

    def set_state(self, U, mask):
        self.U, self.mask = U.clone(), mask.clone()

    def step(self, n=1):
        for _ in range(n):
            self.U = self.f(self.U)

    def luminosity(self, U, r_L, grad=None, scale=1.0):
        if grad is not None:
            grad += scale * (self.Q @ U)
        return float(0.5 * U @ (self.Q @ U))

    def adjoint_forward(self, U, stages=None, U_next=None):
        if stages is not None:
            stages.zero_()
            stages[:U.numel()] = self.A @ U      # the "stage" the reverse sweep needs
        if U_next is not None:
            U_next.copy_(self.f(U))

    def _reverse(self, z, lam_in, lam_out):
        lam_out.copy_(self.A.T @ ((1.0 - torch.tanh(z) ** 2) * lam_in))
        return float(self.b @ lam_in)

    def adjoint_reverse(self, U, stages, lam_in, lam_out):
        return self._reverse(stages[:U.numel()], lam_in, lam_out)

    def adjoint_step(self, U, lam_in, lam_out):
        return self._reverse(self.A @ U, lam_in, lam_out)

    def initial_tangent(self, which, out):
        out.copy_(self.v if which == 0 else math.cos(self.chi) * self.w)


def forward_mode(ctx, nsteps):
    """Lbar and its exact derivatives in (mu, chi, Omega) by tangent propagation."""
    u = ctx.initial()
    du = [ctx.v.clone(), math.cos(ctx.chi) * ctx.w, torch.zeros_like(u)]
    L, dL = 0.0, [0.0, 0.0, 0.0]
    for _ in range(nsteps):
        z = ctx.A @ u
        s = 1.0 - torch.tanh(z) ** 2
        du = [s * (ctx.A @ d) + (ctx.b if k == 2 else 0.0) for k, d in enumerate(du)]
        u = torch.tanh(z) + ctx.omega * ctx.b
        L += float(0.5 * u @ (ctx.Q @ u))
        dL = [a + float((ctx.Q @ u) @ d) for a, d in zip(dL, du)]
    return L / nsteps, [a / nsteps for a in dL]


@pytest.mark.parametrize("nsteps,every", [(7, 3), (6, 3), (1, 25), (5, 1)])
@pytest.mark.parametrize("keep_stages", [True, False])
def test_luminosity_gradient_sequencing(monkeypatch, nsteps, every, keep_stages):
    from paper_2404_01531_gb300 import adjoint
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    ctx = FakeContext()
    U0 = ctx.U.clone()
    L, g, _ = adjoint.luminosity_gradient(ctx, nsteps, r_L=20.0, every=every, keep_stages=keep_stages)
    L_ref, g_ref = forward_mode(ctx, nsteps)
    assert L == pytest.approx(L_ref, rel=1e-13)
    np.testing.assert_allclose(g, g_ref, rtol=1e-12, atol=1e-14 * max(abs(x) for x in g_ref))
    assert torch.equal(ctx.U, U0)          # the context is left at its initial state


def test_lbar_forward_matches(monkeypatch):
    from paper_2404_01531_gb300 import adjoint
    ctx = FakeContext()
    L_ref, _ = forward_mode(ctx, 4)
    assert adjoint.lbar_forward(ctx, 4) == pytest.approx(L_ref, rel=1e-13)


def test_autograd_step_wiring():
    """adjoint.Step: forward = one step of the context from U, backward = the
    step adjoint at the saved input U (not at the output)."""
    from paper_2404_01531_gb300 import adjoint
    ctx = FakeContext()
    U = ctx.initial().clone().requires_grad_(True)
    out = adjoint.Step.apply(U, ctx)
    assert torch.allclose(out, ctx.f(U.detach()))
    w = torch.linspace(-1.0, 1.0, U.numel(), dtype=torch.float64)
    (out * w).sum().backward()
    z = ctx.A @ U.detach()
    want = ctx.A.T @ ((1.0 - torch.tanh(z) ** 2) * w)
    assert torch.allclose(U.grad, want, rtol=1e-14, atol=1e-15)
