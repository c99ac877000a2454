"""torch.autograd.Function over the ETD2 trajectory on a frozen domain.

Forward: nsteps ETD2 steps (etd_step_explicit) from u_0 with the node field
beta and the reaction alpha u (1 - u/K); u is kept only at checkpoints every
`checkpoint_every` steps.  Backward: each segment is recomputed from its
checkpoint (the Krylov bases are rebuilt, nothing of them is stored) and the
adjoint steps (etd_adjoint_step) run from the last step to the first,
accumulating the gradients with respect to u_0, beta and alpha.  All
arithmetic runs in the library's kernels; this module only sequences calls.
"""
import torch

from . import etd


class ETD2Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(fctx, u0, beta, alpha, ectx, phi, dt, nsteps, K, checkpoint_every, nquad):
        if not ectx.adjoint_enabled:
            raise ValueError("the context must be created with adjoint=True")
        ectx.set_reaction("logistic_ak", (float(alpha.item()), float(K)))
        ectx.init_domain(0, phi, beta)
        u_prev = u0.detach().contiguous()
        u = u_prev
        ckpt = {0: (u, u)}
        for n in range(nsteps):
            out = torch.empty_like(u)
            ectx.step_explicit(0, dt, u, u_prev, out)
            u_prev, u = u, out
            if (n + 1) % checkpoint_every == 0 and n + 1 < nsteps:
                ckpt[n + 1] = (u, u_prev)
        fctx.ectx, fctx.phi, fctx.dt, fctx.nsteps, fctx.K = ectx, phi, dt, nsteps, K
        fctx.every, fctx.nquad, fctx.ckpt = checkpoint_every, nquad, ckpt
        fctx.save_for_backward(beta, alpha)
        return u

    @staticmethod
    def backward(fctx, grad_u):
        beta, alpha = fctx.saved_tensors
        ectx, dt, nsteps = fctx.ectx, fctx.dt, fctx.nsteps
        ectx.set_reaction("logistic_ak", (float(alpha.item()), float(fctx.K)))
        ectx.init_domain(0, fctx.phi, beta)
        lam = grad_u.detach().clone().contiguous()
        acc = torch.zeros_like(lam)
        gbeta = torch.zeros_like(beta)
        galpha = torch.zeros(1, dtype=torch.float64, device=lam.device)
        starts = sorted(fctx.ckpt.keys())
        for si in range(len(starts) - 1, -1, -1):
            s0 = starts[si]
            s1 = starts[si + 1] if si + 1 < len(starts) else nsteps
            u, u_prev = fctx.ckpt[s0]
            states = [u_prev, u]  # states[j + 1] = u_{s0 + j}
            for _ in range(s0, s1 - 1):
                out = torch.empty_like(u)
                ectx.step_explicit(0, dt, states[-1], states[-2], out)
                states.append(out)
            for n in range(s1 - 1, s0 - 1, -1):
                u_n = states[n - s0 + 1]
                u_nm1 = states[n - s0] if n > 0 else u_n
                ectx.adjoint_step(0, dt, u_n, u_nm1, n == 0, lam, acc, gbeta, galpha, fctx.nquad)
        return lam, gbeta, galpha.reshape(alpha.shape), None, None, None, None, None, None, None


def trajectory(ectx, u0, beta, alpha, phi, dt, nsteps, K=1.0, checkpoint_every=10, nquad=8):
    """u(T) after nsteps ETD2 steps; differentiable in u0, beta and alpha."""
    return ETD2Trajectory.apply(u0, beta, alpha, ectx, phi, dt, nsteps, K, checkpoint_every, nquad)
