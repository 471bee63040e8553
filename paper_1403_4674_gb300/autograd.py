"""torch.autograd interface to the likelihood-ratio gradient.

``expectation(lattice, beta, h, ...)`` runs the schedules and returns the
replica mean of an endpoint observable (Sec. 2.3) as a differentiable function
of the inverse temperature and the field.  Its backward pass uses the
likelihood-ratio (score-function) estimator
    d E[A] / d theta = Cov(A, d log P(path) / d theta) + E[dA/dtheta explicit],
with the path score accumulated by the run kernel (App. A: each uniformised
step has probability a_c/n_d or 1 - R/n_d).  The library computes the replica
mean, the covariance and the explicit dependence of the observable on h
(e = -J bonds/N - h m) in one call (``kmc_lr_observable``); this module only
passes arguments and hands the library's numbers to autograd.  ``burn_in``
schedules run before the score is reset, so the gradient is that of E[A]
after ``n_schedules`` more schedules from the state distribution reached by
then (a checkpointed segment).
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
        lat.reset(init)
        lat.set_rates([float(beta.item())] * nrep, [float(h.item())] * nrep, law=law)
        if not lat.grad_enabled:
            lat.enable_grad(True)
        if burn_in > 0:
            lat.run(burn_in)
            lat.score(reset=True)
        obs = lat.run(n_schedules, schedule=KMC_SCHEDULE_PALINDROME, time_mode=KMC_TIME_EXPONENTIAL,
                      obs_every=n_schedules)
        out = lat.lr_observable(obs[-1], observable)  # [mean A, dE[A]/dbeta, dE[A]/dh]
        ctx.save_for_backward(out)
        return out[0].to(beta.dtype)

    @staticmethod
    def backward(ctx, g):
        (out,) = ctx.saved_tensors
        # autograd's chain rule: the incoming gradient times the library's derivatives
        return (g * out[1]).to(g.dtype), (g * out[2]).to(g.dtype), None, None, None, None, None, None


def expectation(lattice: Lattice, beta: torch.Tensor, h: torch.Tensor, n_schedules: int,
                observable: str = "e", burn_in: int = 0, law: int = KMC_RATE_METROPOLIS,
                init: int = KMC_INIT_RANDOM) -> torch.Tensor:
    """Replica mean of an endpoint observable ('e', 'm' or 'em'); differentiable in beta and h."""
    return _KmcExpectation.apply(beta, h, lattice, n_schedules, OBSERVABLES[observable], burn_in, law, init)
