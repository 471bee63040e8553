"""Exact transition operators on tiny lattices (test infrastructure).

Builds, over all 2^N states of an L x L periodic lattice, the operators the
paper's proofs are about (arXiv:1403.4674, Sec. 2.2 and App. A):

  * ``step(d)``: one uniformised single-site step of domain d (App. A,
    Eq. Glauber_TM with selection probability 1/n_d): site i of d flips with
    probability a_c(i)/n_d, otherwise the state is kept (T_ii = 1 - sum);
  * ``domain(d)`` = step(d)^k: the domain process T_(lambda_d)^{N_I}
    (Eqs. 4-5);
  * ``colour(c)``: the product over the domains of one colour (they commute,
    Sec. 2.2);
  * ``schedule(colours)``: T_SEQ(Lambda) for a colour sequence (Eq. 8);
  * ``reference_step``: the textbook single-spin kernel over the whole lattice,
    built from H(sigma') - H(sigma) directly (the N_D = 1 special case);
  * ``real_flip_step(d)``: the *other* reading of "k events per visit"
    (always one real flip, chosen proportionally to rate) -- a negative test.

Operators act on column vectors of probabilities, p' = T p.  The acceptance
table is the oracle's own (``oracle.rate_table``); ``quantised=True`` uses the
fixed-point values A_c / 2^P that the sampler actually draws with.
"""
from __future__ import annotations

import numpy as np

from . import oracle as orc
from .exact_ising import lattice_energy_all_states


class Enumerator:
    def __init__(self, L: int, Ld: int, k: int, beta: float, J: float = 1.0,
                 h: float = 0.0, law: int = orc.RATE_METROPOLIS, quantised: bool = True):
        if L * L > 20:
            raise ValueError("state space too large to enumerate")
        self.L, self.Ld, self.k = L, Ld, k
        self.beta, self.J, self.h = beta, J, h
        self.N = L * L
        self.nd = Ld * Ld
        self.Dx = L // Ld
        self.S = 1 << self.N
        idx = np.arange(self.S, dtype=np.int64)
        self.bits = ((idx[:, None] >> np.arange(self.N)) & 1).astype(np.int64)
        self.idx = idx
        H, _ = lattice_energy_all_states(L, J, h)
        self.H = H
        w = np.exp(-beta * (H - H.min()))
        self.pi = w / w.sum()
        log2nd = int(round(np.log2(self.nd)))
        a, A = orc.rate_table(J, beta, h, law, log2nd)
        if quantised:
            P = 63 - log2nd
            self.acc = np.array([float(x) for x in A]) / float(2 ** P)
        else:
            self.acc = a
        # class of every site in every state: c = 5*up + (number of up neighbours)
        self.cls = np.zeros((self.S, self.N), dtype=np.int64)
        for y in range(L):
            for x in range(L):
                i = y * L + x
                nb = [((y - 1) % L) * L + x, ((y + 1) % L) * L + x,
                      y * L + (x - 1) % L, y * L + (x + 1) % L]
                q = sum(self.bits[:, j] for j in nb)
                self.cls[:, i] = 5 * self.bits[:, i] + q

    # -- geometry -----------------------------------------------------------
    def domain_sites(self, d: int):
        bx, by = d % self.Dx, d // self.Dx
        return [(by * self.Ld + yy) * self.L + bx * self.Ld + xx
                for yy in range(self.Ld) for xx in range(self.Ld)]

    def domain_colour(self, d: int) -> int:
        bx, by = d % self.Dx, d // self.Dx
        return (bx & 1) | ((by & 1) << 1)

    def domains_of_colour(self, c: int):
        return [d for d in range(self.Dx * self.Dx) if self.domain_colour(d) == c]

    # -- operators (functions p -> T p) ---------------------------------------
    def _apply_rates(self, p: np.ndarray, sites, rates) -> np.ndarray:
        out = p * (1.0 - sum(rates))
        for i, r in zip(sites, rates):
            out = out + (r * p)[self.idx ^ (1 << i)]
        return out

    def step(self, d: int, p: np.ndarray) -> np.ndarray:
        sites = self.domain_sites(d)
        rates = [self.acc[self.cls[:, i]] / self.nd for i in sites]
        return self._apply_rates(p, sites, rates)

    def domain(self, d: int, p: np.ndarray) -> np.ndarray:
        for _ in range(self.k):
            p = self.step(d, p)
        return p

    def colour(self, c: int, p: np.ndarray) -> np.ndarray:
        for d in self.domains_of_colour(c):
            p = self.domain(d, p)
        return p

    def schedule(self, colours, p: np.ndarray) -> np.ndarray:
        for c in colours:
            p = self.colour(c, p)
        return p

    def reference_step(self, p: np.ndarray, law: int = orc.RATE_METROPOLIS) -> np.ndarray:
        """Textbook random-site kernel on the whole lattice from energy differences."""
        sites = list(range(self.N))
        rates = []
        for i in sites:
            dE = self.H[self.idx ^ (1 << i)] - self.H
            if law == orc.RATE_METROPOLIS:
                acc = np.minimum(1.0, np.exp(-self.beta * dE))
            else:
                acc = 1.0 / (1.0 + np.exp(self.beta * dE))
            rates.append(acc / self.N)
        return self._apply_rates(p, sites, rates)

    def whole_lattice_step(self, p: np.ndarray) -> np.ndarray:
        """One uniformised class-table step with the whole lattice as one domain."""
        sites = list(range(self.N))
        rates = [self.acc[self.cls[:, i]] / self.N for i in sites]
        return self._apply_rates(p, sites, rates)

    def real_flip_step(self, d: int, p: np.ndarray) -> np.ndarray:
        """Negative test: exactly one real flip per step, chosen proportionally to rate."""
        sites = self.domain_sites(d)
        raw = [self.acc[self.cls[:, i]] for i in sites]
        tot = sum(raw)
        rates = [r / tot for r in raw]
        return self._apply_rates(p, sites, rates)

    # -- fixed-time visits (Sec. 2.1 over a horizon) -----------------------------
    def horizon_domain(self, d: int, p: np.ndarray, probs) -> np.ndarray:
        """sum_K probs[K] step(d)^K p: a Poisson number of uniformised steps."""
        acc = probs[0] * p
        q = p
        for K in range(1, len(probs)):
            q = self.step(d, q)
            acc = acc + probs[K] * q
        return acc

    def horizon_schedule(self, colours, p: np.ndarray, probs) -> np.ndarray:
        for c in colours:
            for d in self.domains_of_colour(c):
                p = self.horizon_domain(d, p, probs)
        return p

    # -- exact derivatives (forward mode) ----------------------------------------
    def set_score_table(self, grad30: np.ndarray):
        """Real-valued a_c and dlog a_c/d(beta, h) used for derivatives."""
        self.ga = np.asarray(grad30[0:10], dtype=np.float64)
        self.gb = np.asarray(grad30[10:20], dtype=np.float64)
        self.gh = np.asarray(grad30[20:30], dtype=np.float64)

    def step_deriv(self, d: int, p: np.ndarray, dps):
        """One domain step and its derivative: d(T p) = (dT) p + T (dp), for
        dp in dps = (dp/dbeta, dp/dh).  Rates a_c/n_d, d rate = a_c g_c / n_d."""
        sites = self.domain_sites(d)
        rates = [self.ga[self.cls[:, i]] / self.nd for i in sites]
        out = self._apply_rates(p, sites, rates)
        douts = []
        for dp, g in zip(dps, (self.gb, self.gh)):
            drates = [self.ga[self.cls[:, i]] * g[self.cls[:, i]] / self.nd for i in sites]
            dT_p = -p * sum(drates)
            for i, dr in zip(sites, drates):
                dT_p = dT_p + (dr * p)[self.idx ^ (1 << i)]
            douts.append(dT_p + self._apply_rates(dp, sites, rates))
        return out, douts

    def schedule_deriv(self, colours, p: np.ndarray, dps):
        for c in colours:
            for d in self.domains_of_colour(c):
                for _ in range(self.k):
                    p, dps = self.step_deriv(d, p, dps)
        return p, dps

    # -- checks -----------------------------------------------------------------
    def stationarity_error(self, op) -> float:
        return float(np.max(np.abs(op(self.pi) - self.pi)) / np.max(self.pi))

    def detailed_balance_error(self, op, n_probe: int = 4, seed: int = 0) -> float:
        """max |<x, M D_pi y> - <y, M D_pi x>| / scale over random probes.

        M D_pi is symmetric iff M_ij pi_j = M_ji pi_i (detailed balance).
        """
        rng = np.random.default_rng(seed)
        worst = 0.0
        for _ in range(n_probe):
            x = rng.standard_normal(self.S)
            y = rng.standard_normal(self.S)
            a = float(x @ op(self.pi * y))
            b = float(y @ op(self.pi * x))
            scale = float(np.abs(x) @ op(self.pi * np.abs(y)))
            worst = max(worst, abs(a - b) / scale)
        return worst

    def dense(self, op) -> np.ndarray:
        """Dense matrix of an operator (only for very small state spaces)."""
        if self.S > 4096:
            raise ValueError("too large for a dense matrix")
        M = np.zeros((self.S, self.S))
        for j in range(self.S):
            e = np.zeros(self.S)
            e[j] = 1.0
            M[:, j] = op(e)
        return M


class RingEnumerator:
    """Exact operators of the N_S-spin ring of Sec. 3.1 (all 2^N_S states;
    state index = configuration word, bit n set iff spin n is up).

    ``step(d)``: one uniformised step of domain d (App. A, Eq. Glauber_TM
    with selection probability 1/L_d = N_D/N_S): spin i of d flips with
    probability a_c(i)/L_d.  The halo spins of d (outside it) do not change
    during its process, so the classes read from the current state are the
    classes under the frozen halo.  ``domain(d)`` = step(d)^k (Eqs. 4-5);
    ``phase`` runs a colour (d & 1) or a single domain; ``schedule`` a list
    of phases (Eq. 8); ``random_perm_schedule`` the average over all N_D!
    domain orders (the paper's uniformly random schedule, Sec. 2.2).
    """

    def __init__(self, NS: int, Ld: int, k: int, beta: float, J: float = 1.0, h: float = 0.0,
                 law: int = orc.RATE_BARKER, quantised: bool = True):
        if NS > 14:
            raise ValueError("state space too large to enumerate")
        self.NS, self.Ld, self.k = NS, Ld, k
        self.ND = NS // Ld
        self.beta, self.J, self.h = beta, J, h
        self.S = 1 << NS
        self.idx = np.arange(self.S, dtype=np.int64)
        self.bits = ((self.idx[:, None] >> np.arange(NS)) & 1).astype(np.int64)
        sig = 2 * self.bits - 1
        self.bonds = sum(sig[:, n] * sig[:, (n + 1) % NS] for n in range(NS))
        self.mag = sig.sum(axis=1)
        self.H = -J * self.bonds - h * self.mag
        w = np.exp(-beta * (self.H - self.H.min()))
        self.pi = w / w.sum()
        log2nd = int(round(np.log2(Ld)))
        a, A = orc.ring_rate_table(J, beta, h, law, log2nd)
        self.acc = (np.array([float(x) for x in A]) / float(2 ** (63 - log2nd))) if quantised else a
        self.cls = np.zeros((self.S, NS), dtype=np.int64)
        for n in range(NS):
            self.cls[:, n] = 3 * self.bits[:, n] + self.bits[:, (n - 1) % NS] + self.bits[:, (n + 1) % NS]

    def domain_sites(self, d: int):
        return list(range(d * self.Ld, (d + 1) * self.Ld))

    def _apply_rates(self, p: np.ndarray, sites, rates) -> np.ndarray:
        out = p * (1.0 - sum(rates))
        for i, r in zip(sites, rates):
            out = out + (r * p)[self.idx ^ (1 << i)]
        return out

    def step(self, d: int, p: np.ndarray) -> np.ndarray:
        sites = self.domain_sites(d)
        return self._apply_rates(p, sites, [self.acc[self.cls[:, i]] / self.Ld for i in sites])

    def domain(self, d: int, p: np.ndarray) -> np.ndarray:
        for _ in range(self.k):
            p = self.step(d, p)
        return p

    def phase(self, unit: int, p: np.ndarray, is_domain: bool) -> np.ndarray:
        for d in range(self.ND):
            if (d == unit) if is_domain else ((d & 1) == unit):
                p = self.domain(d, p)
        return p

    def schedule(self, phases, p: np.ndarray, is_domain: bool = False) -> np.ndarray:
        for u in phases:
            p = self.phase(u, p, is_domain)
        return p

    def random_perm_schedule(self, p: np.ndarray) -> np.ndarray:
        import itertools
        perms = list(itertools.permutations(range(self.ND)))
        return sum(self.schedule(list(q), p, True) for q in perms) / len(perms)

    def reference_step(self, p: np.ndarray, law: int = orc.RATE_BARKER) -> np.ndarray:
        """Textbook random-site kernel on the whole ring from energy differences."""
        sites = list(range(self.NS))
        rates = []
        for i in sites:
            dE = self.H[self.idx ^ (1 << i)] - self.H
            acc = np.minimum(1.0, np.exp(-self.beta * dE)) if law == orc.RATE_METROPOLIS \
                else 1.0 / (1.0 + np.exp(self.beta * dE))
            rates.append(acc / self.NS)
        return self._apply_rates(p, sites, rates)

    def spin_means(self, p: np.ndarray) -> np.ndarray:
        """<sigma_n> under p, n = 0..N_S-1."""
        return (2 * self.bits - 1).T @ p

    def stationarity_error(self, op) -> float:
        return float(np.max(np.abs(op(self.pi) - self.pi)) / np.max(self.pi))

    def detailed_balance_error(self, op, n_probe: int = 4, seed: int = 0) -> float:
        rng = np.random.default_rng(seed)
        worst = 0.0
        for _ in range(n_probe):
            x = rng.standard_normal(self.S)
            y = rng.standard_normal(self.S)
            a = float(x @ op(self.pi * y))
            b = float(y @ op(self.pi * x))
            scale = float(np.abs(x) @ op(self.pi * np.abs(y)))
            worst = max(worst, abs(a - b) / scale)
        return worst


class PartEnumerator(Enumerator):
    """Exact operators of an L x L lattice under a block or vertical-stripe
    partition with any domain size n_d (Sec. 3.2).  The sampler's per-step
    flip probability of a class-c site is A_c / M with A_c = round(a_c 2^P),
    M = n_d 2^P, P = 63 - ceil(log2 n_d) (to 2^-64), i.e. (A_c / 2^P) / n_d.
    ``random_perm_schedule`` averages the schedule over all N_D! domain orders."""

    def __init__(self, L: int, kind: int, ND: int, k: int, beta: float, J: float = 1.0, h: float = 0.0,
                 law: int = orc.RATE_BARKER, quantised: bool = True):
        super().__init__(L, L, k, beta, J=J, h=h, law=law, quantised=False)
        self.kind, self.ND = kind, ND
        self.geom = [orc.part_geometry(L, kind, ND, d) for d in range(ND)]
        x0, y0, w, hh, _ = self.geom[0]
        self.nd = w * hh
        self.Dx = None
        P, _ = orc.part_scale(L, kind, ND)
        a, A = orc.rate_table(J, beta, h, law, 63 - P)
        self.acc = (np.array([float(x) for x in A]) / float(2 ** P)) if quantised else a

    def domain_sites(self, d: int):
        x0, y0, w, hh, _ = self.geom[d]
        return [(y0 + yy) * self.L + x0 + xx for yy in range(hh) for xx in range(w)]

    def domain_colour(self, d: int) -> int:
        return self.geom[d][4]

    def domains_of_colour(self, c: int):
        return [d for d in range(self.ND) if self.geom[d][4] == c]

    def phase(self, unit: int, p: np.ndarray, is_domain: bool) -> np.ndarray:
        return self.domain(unit, p) if is_domain else self.colour(unit, p)

    def random_perm_schedule(self, p: np.ndarray) -> np.ndarray:
        import itertools
        perms = list(itertools.permutations(range(self.ND)))
        out = np.zeros_like(p)
        for q in perms:
            pp = p
            for d in q:
                pp = self.domain(d, pp)
            out = out + pp
        return out / len(perms)
