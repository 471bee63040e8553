"""Statistics of the paper's time-scaling protocol (Sec. 2.3 and the appendix).

Host-side analysis of observation records produced on the device by
``Lattice.run(..., obs_every=...)``:

* only domain-process endpoints are valid observation points (Sec. 2.3); the
  records of ``run`` are taken at schedule endpoints, or at every colour pass
  (register-shifted endpoints) when the lattice observes per pass;
* the intrinsic time constant tau_PAR is the decay constant of the
  equilibrium autocorrelation C_A(ds) = C_A(0) exp(-ds / tau_PAR) of
  A = H m, averaged over trajectories (Sec. 2.3);
* the time of a parallel run is rescaled to the reference time scale by
  t = s tau_REF / tau_PAR (Sec. 2.3);
* the ideal efficiency is eta = tau_REF / (tau_PAR N_I) (appendix, Eq. efficiency).

Readings where the paper is terse: the autocorrelation is that of the
fluctuation dA = A - <A> (the mean over all trajectories and times of the
equilibrium window), since <A(s) A(s + ds)> without the mean removed does
not decay to zero; the fit keeps C_A(0) fixed to the measured value (the
form the paper writes) and uses lags while C_A stays above C_A(0) e^-2.
Lags are in integer timesteps s (Eq. 11: one colour pass of N_D domain
processes advances s by N_I N_D).
"""
from __future__ import annotations

import math
from typing import Optional, Sequence

import numpy as np


def autocorrelation(A: np.ndarray, max_lag: Optional[int] = None) -> np.ndarray:
    """Mean over trajectories of the per-trajectory autocorrelation of the
    fluctuation of A.

    A: [n_traj, n_obs] equally spaced equilibrium observations.
    Returns C[0..max_lag], C[d] = mean_i (1/(n-d)) sum_s dA_i(s) dA_i(s+d).
    """
    A = np.asarray(A, dtype=np.float64)
    if A.ndim == 1:
        A = A[None, :]
    n_traj, n = A.shape
    if max_lag is None:
        max_lag = n // 4
    max_lag = int(min(max_lag, n - 1))
    dA = A - A.mean()
    # per-trajectory lag products through the FFT (zero padding: no wrap-around)
    m = 1 << int(math.ceil(math.log2(2 * n)))
    f = np.fft.rfft(dA, n=m, axis=1)
    raw = np.fft.irfft(f * np.conj(f), n=m, axis=1)[:, :max_lag + 1]
    counts = n - np.arange(max_lag + 1)
    return (raw / counts).mean(axis=0)


def fit_tau(C: np.ndarray, dt: float = 1.0, cut: float = math.exp(-2.0)) -> float:
    """Decay constant of C(d) ~ C(0) exp(-d dt / tau), least squares over the
    lags d >= 0 before C first falls below cut * C(0)."""
    C = np.asarray(C, dtype=np.float64)
    if C.size < 2 or not C[0] > 0:
        raise ValueError("autocorrelation must have C(0) > 0 and at least two lags")
    below = np.nonzero(C < cut * C[0])[0]
    last = int(below[0]) if below.size else C.size
    last = max(last, 2)
    d = np.arange(last, dtype=np.float64) * dt
    y = C[:last]

    def sse(log_tau: float) -> float:
        r = y - C[0] * np.exp(-d / math.exp(log_tau))
        return float(r @ r)

    # golden-section search on log tau (the SSE is unimodal in tau for a
    # decaying curve); bounds span far beyond the sampled lags
    lo, hi = math.log(dt * 1e-3), math.log(dt * max(last, 2) * 1e4)
    g = (math.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c1, c2 = b - g * (b - a), a + g * (b - a)
    f1, f2 = sse(c1), sse(c2)
    for _ in range(200):
        if f1 <= f2:
            b, c2, f2 = c2, c1, f1
            c1 = b - g * (b - a)
            f1 = sse(c1)
        else:
            a, c1, f1 = c1, c2, f2
            c2 = a + g * (b - a)
            f2 = sse(c2)
        if b - a < 1e-12:
            break
    return math.exp(0.5 * (a + b))


def tau_par(A: np.ndarray, steps_per_record: float, max_lag: Optional[int] = None) -> float:
    """tau_PAR in timesteps from equilibrium records A[n_traj, n_obs] spaced
    steps_per_record timesteps apart (Sec. 2.3)."""
    return fit_tau(autocorrelation(A, max_lag), dt=steps_per_record)


def steps_per_schedule(N_I: int, N_D: int, passes: int = 2) -> int:
    """Timesteps of one schedule: each colour pass runs N_D / 4 domain
    processes of N_I steps per colour, so a schedule of `passes` visits per
    domain advances s by passes * N_I * N_D (Eq. 11)."""
    return passes * N_I * N_D


def rescale_time(s: np.ndarray, tau_ref: float, tau_par_: float) -> np.ndarray:
    """Parallel timesteps mapped to the reference time scale: t = s tau_REF / tau_PAR."""
    return np.asarray(s, dtype=np.float64) * (tau_ref / tau_par_)


def efficiency(tau_ref: float, tau_par_: float, N_I: int) -> float:
    """Ideal efficiency eta(N_I, N_D) = tau_REF / (tau_PAR N_I) (appendix, Eq. efficiency)."""
    return tau_ref / (tau_par_ * N_I)


def time_dependent_average(A: np.ndarray) -> np.ndarray:
    """<A(s)> = (1/N_TRAJ) sum_i A_i(s) over trajectories (Sec. 3.1)."""
    return np.asarray(A, dtype=np.float64).mean(axis=0)


def ring_ensemble_averages(ens: np.ndarray, n_traj: int, n_sites: int, J: float = 1.0, h: float = 0.0) -> dict:
    """Time-dependent averages over trajectories (Sec. 3.1, Eq. time dependent
    averages) from the ring's device ensemble sums.

    ens: [n_rec, 4 + N_S] int64 rows {sum bonds, sum mag, sum bonds*mag,
    sum mag^2, number of trajectories with spin n up (n = 0..N_S-1)}, as
    kmc_ring_run writes them.  Returns per record: <sigma_n> [n_rec, N_S],
    <H>/N_S, <m>, and <A> = <H m> / N_S^2 (the paper's 1D observable, per
    site), with H = -J bonds - h mag."""
    ens = np.asarray(ens, dtype=np.int64)
    n = float(n_traj)
    N = float(n_sites)
    bonds, mag, bm, m2 = (ens[:, i].astype(np.float64) for i in range(4))
    spins = 2.0 * ens[:, 4:4 + n_sites].astype(np.float64) / n - 1.0
    H = (-J * bonds - h * mag) / n
    A = (-J * bm - h * m2) / n
    return {"spin": spins, "energy": H / N, "magnetisation": mag / (n * N), "A": A / (N * N)}


__all__ = ["autocorrelation", "efficiency", "fit_tau", "rescale_time", "ring_ensemble_averages", "steps_per_schedule",
           "tau_par", "time_dependent_average"]
