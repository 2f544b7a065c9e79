"""Reverse-mode differentiation of the hybrid step (DG path, frozen branches)
through the C ABI: a torch.autograd.Function for one step, and a
checkpointed driver for the gradient of the time-averaged spin-down
luminosity with respect to (mu, chi, Omega).  Every vector-Jacobian product
runs in the CUDA library (ffe_adjoint_step, ffe_luminosity, ffe_initial_tangent);
this module only sequences the calls."""
import torch


class Step(torch.autograd.Function):
    """u_{n+1} = step(u_n): forward through ffe_step, backward through
    ffe_adjoint_step (recomputes the step's stages from the saved u_n)."""

    @staticmethod
    def forward(ctx_autograd, U, ffe_ctx):
        ffe_ctx.set_state(U, ffe_ctx.state()[1].clone())
        ffe_ctx.step(1)
        out = ffe_ctx.state()[0].clone()
        ctx_autograd.save_for_backward(U)
        ctx_autograd.ffe_ctx = ffe_ctx
        return out

    @staticmethod
    def backward(ctx_autograd, lam):
        (U,) = ctx_autograd.saved_tensors
        lam_out = torch.empty_like(lam)
        ctx_autograd.ffe_ctx.adjoint_step(U, lam.contiguous(), lam_out)
        return lam_out, None


def freeze_union_mask(ctx, nsteps):
    """The troubled-cell mask frozen from a forward pass: advance the hybrid
    step with the indicator for nsteps from the initial data of ctx, then
    restart from that initial data with every element the indicator flagged at
    any step on FD subcells (initial data at their cell centres) and the mask
    frozen.  Returns the mask."""
    import torch
    U0, m0 = (t.clone() for t in ctx.state())
    union = m0.clone()
    for _ in range(nsteps):
        ctx.step(1)
        torch.bitwise_or(union, ctx.state()[1], out=union)
    ctx.set_state(U0, union)
    ctx.set_initial(keep_mask=True)
    ctx.freeze_mask(True)
    return union


def lbar_forward(ctx, nsteps, r_L=20.0):
    """Lbar = mean of L(u_n), n = 1..nsteps, forward only (no checkpoints);
    the state of ctx is advanced by nsteps."""
    acc = 0.0
    for _ in range(nsteps):
        ctx.step(1)
        acc += ctx.luminosity(ctx.state()[0], r_L)
    return acc / nsteps


def luminosity_gradient(ctx, nsteps, r_L=20.0, every=25, keep_stages=True):
    """Lbar = mean of L(u_n), n = 1..nsteps, and d Lbar/d (mu, chi, Omega).

    ctx: a Context holding the dipole initial data (ffe_set_initial already
    called).  Forward: nsteps steps keeping a checkpoint every `every` steps.
    Reverse: per segment, the states are recomputed from its checkpoint and
    the step adjoints run backward with the luminosity gradient of each state
    added to lambda.  keep_stages: the recomputation keeps every step's stage
    states (5 state vectors per step of the segment, in device memory) and the
    backward sweep uses them (ffe_adjoint_forward / ffe_adjoint_reverse);
    otherwise each step adjoint recomputes its stages (ffe_adjoint_step).
    Returns (Lbar, [dmu, dchi, dOmega], timings)."""
    import time
    U0, mask0 = ctx.state()
    U0 = U0.clone()
    mask0 = mask0.clone()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ckpt = {0: U0.clone()}
    Lsum = 0.0
    for n in range(1, nsteps + 1):
        ctx.step(1)
        U = ctx.state()[0]
        Lsum += ctx.luminosity(U, r_L)
        if n % every == 0 or n == nsteps:
            ckpt[n] = U.clone()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    lam = torch.zeros_like(U0)
    tmp = torch.empty_like(U0)
    om_bar = 0.0
    stages = None
    if keep_stages:
        stages = torch.empty((min(every, nsteps), 5 * U0.numel()), dtype=U0.dtype, device=U0.device)
    starts = list(range(0, nsteps, every))
    for s0 in reversed(starts):
        s1 = min(s0 + every, nsteps)
        # recompute u_{s0} .. u_{s1-1} (and, with keep_stages, every step's stages)
        states = [ckpt[s0]]
        if keep_stages:
            for n in range(s0, s1):
                nxt = torch.empty_like(U0) if n + 1 < s1 else None
                ctx.adjoint_forward(states[n - s0], stages[n - s0], nxt)
                if nxt is not None:
                    states.append(nxt)
        else:
            ctx.set_state(ckpt[s0], mask0)
            for _ in range(s1 - s0 - 1):
                ctx.step(1)
                states.append(ctx.state()[0].clone())
        for n in range(s1 - 1, s0 - 1, -1):
            # lambda_{n+1} += dL(u_{n+1})/du / nsteps, then through step n
            un1 = ckpt[s1] if n + 1 == s1 else states[n + 1 - s0]
            ctx.luminosity(un1, r_L, grad=lam, scale=1.0 / nsteps)
            if keep_stages:
                om_bar += ctx.adjoint_reverse(states[n - s0], stages[n - s0], lam, tmp)
            else:
                om_bar += ctx.adjoint_step(states[n - s0], lam, tmp)
            lam, tmp = tmp, lam
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    grads = []
    for which in (0, 2):
        ctx.initial_tangent(which, tmp)
        grads.append(float(torch.dot(lam, tmp)))
    ctx.set_state(U0, mask0)
    return Lsum / nsteps, [grads[0], grads[1], om_bar], {"forward_s": t1 - t0, "adjoint_s": t2 - t1}
