"""torch.autograd interface to the likelihood-ratio gradient.

``expectation(lattice, beta, h, ...)`` runs the schedules and returns the
replica mean of an endpoint observable (Sec. 2.3) as a differentiable function
of the inverse temperature and the field.  Its backward pass uses the
likelihood-ratio (score-function) estimator
    d E[A] / d theta = E[(A - E A) * d log P(path) / d theta],
with the path score accumulated by the run kernel (App. A: each uniformised
step has probability a_c/n_d or 1 - R/n_d) and the covariance taken by the
library's estimate kernel, plus the explicit dependence of the observable on
h (e = -J bonds/N - h m).  ``burn_in`` schedules run before the score is
reset, so the gradient is that of E[A] after ``n_schedules`` more schedules
from the state distribution reached by then (a checkpointed segment).
"""
from __future__ import annotations

import torch

from .api import KMC_INIT_RANDOM, KMC_RATE_METROPOLIS, KMC_SCHEDULE_PALINDROME, KMC_TIME_EXPONENTIAL, Lattice

OBSERVABLES = {"e": 0, "m": 1, "em": 2}


class _KmcExpectation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, beta: torch.Tensor, h: torch.Tensor, lattice: Lattice, n_schedules: int,
                observable: int, burn_in: int, law: int, init: int):
        lat = lattice
        nrep = lat.n_replicas
        b = float(beta.item())
        hv = float(h.item())
        lat.reset(init)
        lat.set_rates([b] * nrep, [hv] * nrep, law=law)
        if not lat.grad_enabled:
            lat.enable_grad(True)
        if burn_in > 0:
            lat.run(burn_in)
            lat.score(reset=True)
        obs = lat.run(n_schedules, schedule=KMC_SCHEDULE_PALINDROME, time_mode=KMC_TIME_EXPONENTIAL,
                      obs_every=n_schedules)
        A = obs[-1, :, observable].contiguous()
        grad = lat.lr_estimate(A)
        # e = -J bonds/N - h m and e*m depend on h explicitly as well:
        # d e/dh = -m, d(e m)/dh = -m^2 (m has no explicit dependence)
        m = obs[-1, :, 1]
        if observable == 0:
            grad[1] += -m.mean()
        elif observable == 2:
            grad[1] += -(m * m).mean()
        ctx.save_for_backward(grad)
        return A.mean().to(beta.dtype)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        gb = (g * grad[0]).to(g.dtype)
        gh = (g * grad[1]).to(g.dtype)
        return gb, gh, None, None, None, None, None, None


def expectation(lattice: Lattice, beta: torch.Tensor, h: torch.Tensor, n_schedules: int,
                observable: str = "e", burn_in: int = 0, law: int = KMC_RATE_METROPOLIS,
                init: int = KMC_INIT_RANDOM) -> torch.Tensor:
    """Replica mean of an endpoint observable ('e', 'm' or 'em'); differentiable in beta and h."""
    return _KmcExpectation.apply(beta, h, lattice, n_schedules, OBSERVABLES[observable], burn_in, law, init)
