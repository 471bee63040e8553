"""Exact equilibrium references for the 2D periodic Ising model (test infrastructure).

Used to pin the oracle's equilibrium statistics.  The paper compares its
simulated energies against the finite-lattice formula of Ferdinand & Fisher
(Sec. 3.2, Table 1), which rests on Kaufman's exact partition function for the
periodic lattice.  This module restates, independently of the simulation code:

  * ``brute_force``: explicit sum over all 2^N states (tiny lattices);
  * ``transfer_matrix``: Z = Tr T^L with the symmetric row-to-row matrix;
  * ``kaufman_lnZ``: Kaufman (Phys. Rev. 76, 1232, 1949) periodic L x L
    partition function, the formula Ferdinand & Fisher evaluate;
  * ``onsager_energy`` / ``yang_magnetisation``: infinite-lattice closed forms
    (Onsager 1944; Yang 1952).

Energies are per site, H = -J sum_<ij> s_i s_j - h sum_i s_i (App. A, with the
field term), k_B = 1.
"""
from __future__ import annotations

import numpy as np
from scipy.special import ellipk


def _all_spins(N: int) -> np.ndarray:
    idx = np.arange(1 << N, dtype=np.int64)
    return (((idx[:, None] >> np.arange(N)) & 1) * 2 - 1).astype(np.int8)


def lattice_energy_all_states(L: int, J: float = 1.0, h: float = 0.0) -> np.ndarray:
    """H(sigma) for every state of an L x L periodic lattice; site i = y*L + x is bit i."""
    N = L * L
    s = _all_spins(N).astype(np.int64)
    bonds = np.zeros(s.shape[0], dtype=np.int64)
    for y in range(L):
        for x in range(L):
            i = y * L + x
            r = y * L + (x + 1) % L
            u = ((y + 1) % L) * L + x
            bonds += s[:, i] * (s[:, r] + s[:, u])
    mag = s.sum(axis=1)
    return -J * bonds - h * mag, mag


def brute_force(L: int, T: float, J: float = 1.0, h: float = 0.0):
    """(e, sd_e, |m|) per site by explicit enumeration of all 2^(L*L) states."""
    H, mag = lattice_energy_all_states(L, J, h)
    beta = 1.0 / T
    w = np.exp(-beta * (H - H.min()))
    Z = w.sum()
    N = L * L
    e = (w * H).sum() / Z / N
    e2 = (w * (H / N) ** 2).sum() / Z
    mabs = (w * np.abs(mag)).sum() / Z / N
    return e, np.sqrt(max(e2 - e * e, 0.0)), mabs


def transfer_matrix_lnZ(L: int, K: float, Hf: float = 0.0) -> float:
    """ln Z of the L x L periodic lattice, K = beta*J, Hf = beta*h, by Tr T^L."""
    idx = np.arange(1 << L, dtype=np.int64)
    s = (((idx[:, None] >> np.arange(L)) & 1) * 2 - 1).astype(np.float64)
    intra = (s * np.roll(s, -1, axis=1)).sum(axis=1)
    field = s.sum(axis=1)
    inter = s @ s.T
    Tm = np.exp(K * inter + 0.5 * K * (intra[:, None] + intra[None, :])
                + 0.5 * Hf * (field[:, None] + field[None, :]))
    lam = np.linalg.eigvalsh(Tm)
    lmax = lam[-1]
    return L * np.log(lmax) + np.log(np.sum((lam / lmax) ** L))


def _log_2cosh(x: np.ndarray):
    ax = np.abs(x)
    return float(np.sum(ax + np.log1p(np.exp(-2 * ax)))), 1


def _log_abs_2sinh(x: np.ndarray):
    ax = np.abs(x)
    if np.any(ax == 0):
        return -np.inf, 0
    return float(np.sum(ax + np.log(-np.expm1(-2 * ax)))), int(np.prod(np.sign(x)))


def kaufman_lnZ(L: int, K: float) -> float:
    """Kaufman's exact ln Z for the L x L periodic lattice at K = beta*J, h = 0.

    Z = 1/2 (2 sinh 2K)^(L^2/2) (Z1 + Z2 + Z3 + Z4) with
      Z1 = prod_r 2 cosh(L g_{2r+1}/2),  Z2 = prod_r 2 sinh(L g_{2r+1}/2),
      Z3 = prod_r 2 cosh(L g_{2r}/2),    Z4 = prod_r 2 sinh(L g_{2r}/2),
    r = 0..L-1, cosh g_l = cosh 2K coth 2K - cos(l pi / L) for l >= 1 and
    g_0 = 2K + ln tanh K (negative above T_c).
    """
    l = np.arange(2 * L)
    c = np.cosh(2 * K) / np.tanh(2 * K) - np.cos(l * np.pi / L)
    g = np.arccosh(np.maximum(c, 1.0))
    g[0] = 2 * K + np.log(np.tanh(K))
    odd = g[1::2]
    even = g[0::2]
    terms = []
    for vals, fn in ((odd, _log_2cosh), (odd, _log_abs_2sinh),
                     (even, _log_2cosh), (even, _log_abs_2sinh)):
        terms.append(fn(L * vals / 2))
    top = max(t[0] for t in terms)
    acc = sum(sg * np.exp(la - top) for la, sg in terms if sg != 0)
    return np.log(0.5) + 0.5 * L * L * np.log(2 * np.sinh(2 * K)) + top + np.log(acc)


def _dlnZ_dK(fn, K: float, step: float = 1e-4) -> float:
    h = step * K
    f = [fn(K + j * h) for j in (-2, -1, 1, 2)]
    return (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * h)


def kaufman_energy(L: int, T: float, J: float = 1.0) -> float:
    """Exact per-site energy e = -(J/N) d lnZ/dK of the L x L periodic lattice."""
    K = J / T
    return -J * _dlnZ_dK(lambda k: kaufman_lnZ(L, k), K) / (L * L)


def transfer_matrix_energy(L: int, T: float, J: float = 1.0) -> float:
    K = J / T
    return -J * _dlnZ_dK(lambda k: transfer_matrix_lnZ(L, k), K) / (L * L)


def onsager_energy(T: float, J: float = 1.0) -> float:
    """Onsager's infinite-lattice energy per site, h = 0."""
    K = J / T
    kap = 2 * np.sinh(2 * K) / np.cosh(2 * K) ** 2
    return -J / np.tanh(2 * K) * (1 + (2 / np.pi) * (2 * np.tanh(2 * K) ** 2 - 1)
                                  * ellipk(kap * kap))


def yang_magnetisation(T: float, J: float = 1.0) -> float:
    """Spontaneous magnetisation per site (0 above T_c)."""
    K = J / T
    x = 1 - np.sinh(2 * K) ** -4
    return float(x ** 0.125) if x > 0 else 0.0


T_CRITICAL = 2.0 / np.log(1 + np.sqrt(2.0))
