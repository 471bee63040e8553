"""Python side of the CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this module.  The product library never
touches it.  ``build()`` compiles ``kmc_oracle.c`` with gcc into
``oracle/liborc_kmc.so``; the wrappers below only marshal arguments.

Everything here follows the C file's comments: the paper's App. A energy and
single-site kernel, Sec. 2.2 domains/halo/schedule, Sec. 2.1 clock and
Sec. 2.3 endpoint observables (arXiv:1403.4674).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kmc_oracle.c")
LIB = os.path.join(HERE, "liborc_kmc.so")

RATE_METROPOLIS = 0
RATE_BARKER = 1
SCHED_PALINDROME = 0
SCHED_FIXED = 1
SCHED_RANDOM_PERM = 2
TIME_EXPONENTIAL = 0
TIME_EXPECTED = 1
TIME_HORIZON = 2  # each visit runs for domain time dtau: Poisson(n_d nu dtau) steps
INIT_RANDOM = 0
INIT_ALL_UP = 1

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, gcc, no FP contraction)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        i8p = ctypes.POINTER(ctypes.c_int8)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_philox4x32_10.restype = None
        L.orc_rate_table.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, dp, u64p]
        L.orc_rate_table.restype = ctypes.c_int
        L.orc_class_dE.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.orc_class_dE.restype = ctypes.c_double
        L.orc_init_spins.argtypes = [i8p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64]
        L.orc_init_spins.restype = None
        L.orc_schedule_colours.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.POINTER(ctypes.c_int)]
        L.orc_schedule_colours.restype = ctypes.c_int
        L.orc_energy_mag.argtypes = [i8p, ctypes.c_int, i64p, i64p]
        L.orc_energy_mag.restype = None
        L.orc_domain_time.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                      ctypes.c_int, ctypes.c_double]
        L.orc_domain_time.restype = ctypes.c_double
        L.orc_run_replica.argtypes = [i8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p,
                                      ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                      dp, i64p, u64p, i64p, dp]
        L.orc_run_replica.restype = ctypes.c_int
        L.orc_sample_final_states.argtypes = [i8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              u64p, ctypes.c_uint64, ctypes.c_int64,
                                              ctypes.c_int, ctypes.c_int64, i8p]
        L.orc_sample_final_states.restype = ctypes.c_int
        L.orc_score_table.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, dp]
        L.orc_score_table.restype = ctypes.c_int
        L.orc_sum_compensated.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int64]
        L.orc_sum_compensated.restype = ctypes.c_double
        L.orc_run_replica_grad.argtypes = L.orc_run_replica.argtypes + [dp, dp]
        L.orc_run_replica_grad.restype = ctypes.c_int
        ra = L.orc_run_replica.argtypes
        L.orc_run_replica_obs.argtypes = ra[:14] + [ctypes.c_int] + ra[14:] + [dp, dp]
        L.orc_run_replica_obs.restype = ctypes.c_int
        L.orc_run_replica_ex.argtypes = ra[:14] + [ctypes.c_int, ctypes.c_double] + ra[14:] + [dp, dp]
        L.orc_run_replica_ex.restype = ctypes.c_int
        L.orc_horizon_kmax.argtypes = [ctypes.c_double]
        L.orc_horizon_kmax.restype = ctypes.c_int
        L.orc_horizon_table.argtypes = [ctypes.c_double, ctypes.c_int, u64p]
        L.orc_horizon_table.restype = None
        L.orc_sample_final_states_grad.argtypes = L.orc_sample_final_states.argtypes + [dp, dp]
        L.orc_sample_final_states_grad.restype = ctypes.c_int
        L.orc_hash_basis.argtypes = []
        L.orc_hash_basis.restype = ctypes.c_uint64
        L.orc_ring_rate_table.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, ctypes.c_int, dp, u64p]
        L.orc_ring_rate_table.restype = ctypes.c_int
        L.orc_ring_energy_mag.argtypes = [ctypes.c_uint64, ctypes.c_int, i64p, i64p]
        L.orc_ring_energy_mag.restype = None
        L.orc_ring_schedule.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.orc_ring_schedule.restype = ctypes.c_int
        L.orc_ring_run.argtypes = [u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p, ctypes.c_uint64,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                   dp, i64p, u64p, i64p, dp, u64p]
        L.orc_ring_run.restype = ctypes.c_int
        L.orc_part_geometry.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_int)] * 5
        L.orc_part_geometry.restype = ctypes.c_int
        L.orc_part_schedule.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.orc_part_schedule.restype = ctypes.c_int
        L.orc_part_scale.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p]
        L.orc_part_scale.restype = ctypes.c_int
        L.orc_part_run.argtypes = [i8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p, ctypes.c_uint64,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int64, ctypes.c_int64, ctypes.c_int, dp, i64p, u64p, i64p, dp]
        L.orc_part_run.restype = ctypes.c_int
        L.orc_part_run_many.argtypes = [ctypes.c_int64, i8p, u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, u64p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                                        i8p, dp, u64p, i64p]
        L.orc_part_run_many.restype = ctypes.c_int
        L.orc_ring_run_many.argtypes = [ctypes.c_int64, u64p, u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        u64p, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, dp, u64p,
                                        u64p, i64p]
        L.orc_ring_run_many.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                            _ptr(out, ctypes.c_uint32))
    return out


def rate_table(J: float, beta: float, h: float, law: int, log2_nd: int):
    """Returns (a[10] float64, A[10] uint64): App. A acceptance, fixed point."""
    a = np.zeros(10, dtype=np.float64)
    A = np.zeros(10, dtype=np.uint64)
    rc = lib().orc_rate_table(J, beta, h, law, log2_nd, _ptr(a, ctypes.c_double),
                              _ptr(A, ctypes.c_uint64))
    if rc == -2:
        raise ValueError("an acceptance rounds to 0 at 2^-%d (one-way rate)" % (63 - log2_nd))
    if rc != 0:
        raise ValueError("invalid rate-table arguments")
    return a, A


def class_dE(c: int, J: float, h: float) -> float:
    return lib().orc_class_dE(c, J, h)


def init_spins(L: int, init: int, seed: int) -> np.ndarray:
    s = np.zeros(L * L, dtype=np.int8)
    lib().orc_init_spins(_ptr(s, ctypes.c_int8), L, init, seed)
    return s.reshape(L, L)


def schedule_colours(schedule: int, n: int, seed: int):
    out = (ctypes.c_int * 8)()
    nph = lib().orc_schedule_colours(schedule, n, seed, out)
    if nph < 0:
        raise ValueError("bad schedule")
    return [out[i] for i in range(nph)]


def energy_mag(s: np.ndarray):
    s = np.ascontiguousarray(s, dtype=np.int8)
    L = s.shape[0]
    b = ctypes.c_int64()
    m = ctypes.c_int64()
    lib().orc_energy_mag(_ptr(s, ctypes.c_int8), L, ctypes.byref(b), ctypes.byref(m))
    return b.value, m.value


def sum_compensated(x) -> float:
    """The oracle's compensated sum of a float64 sequence."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(lib().orc_sum_compensated(_ptr(x, ctypes.c_double), x.size))


def score_table(J: float, beta: float, h: float, law: int) -> np.ndarray:
    """[a_c (10), dlog a_c/dbeta (10), dlog a_c/dh (10)]."""
    g = np.zeros(30, dtype=np.float64)
    if lib().orc_score_table(J, beta, h, law, _ptr(g, ctypes.c_double)) != 0:
        raise ValueError("bad rate law")
    return g


def sample_final_states_with_score(s0: np.ndarray, Ld: int, k: int, A: np.ndarray, grad: np.ndarray,
                                   seed0: int, n_runs: int, n_sched: int,
                                   schedule: int = SCHED_PALINDROME):
    """Final states and path scores d log P / d(beta, h) of n_runs independent runs."""
    s0 = np.ascontiguousarray(s0, dtype=np.int8)
    L = s0.shape[0]
    A = np.ascontiguousarray(A, dtype=np.uint64)
    grad = np.ascontiguousarray(grad, dtype=np.float64)
    out = np.zeros((n_runs, L, L), dtype=np.int8)
    score = np.zeros((n_runs, 2), dtype=np.float64)
    rc = lib().orc_sample_final_states_grad(_ptr(s0, ctypes.c_int8), L, Ld, k,
                                            _ptr(A, ctypes.c_uint64), seed0, n_runs, schedule,
                                            n_sched, _ptr(out, ctypes.c_int8),
                                            _ptr(grad, ctypes.c_double), _ptr(score, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle rejected the configuration")
    return out, score


def sample_final_states(s0: np.ndarray, Ld: int, k: int, A: np.ndarray, seed0: int,
                        n_runs: int, n_sched: int, schedule: int = SCHED_PALINDROME):
    """Final states of n_runs independent runs (seeds seed0..seed0+n_runs-1) from s0."""
    s0 = np.ascontiguousarray(s0, dtype=np.int8)
    L = s0.shape[0]
    A = np.ascontiguousarray(A, dtype=np.uint64)
    out = np.zeros((n_runs, L, L), dtype=np.int8)
    rc = lib().orc_sample_final_states(_ptr(s0, ctypes.c_int8), L, Ld, k,
                                       _ptr(A, ctypes.c_uint64), seed0, n_runs, schedule,
                                       n_sched, _ptr(out, ctypes.c_int8))
    if rc != 0:
        raise ValueError("oracle rejected the configuration")
    return out


def horizon_kmax(mu: float) -> int:
    return int(lib().orc_horizon_kmax(float(mu)))


def horizon_table(mu: float) -> np.ndarray:
    """Poisson CDF thresholds floor(F(k) 2^64), k < kmax(mu)."""
    kmax = horizon_kmax(mu)
    out = np.zeros(kmax, dtype=np.uint64)
    lib().orc_horizon_table(float(mu), kmax, _ptr(out, ctypes.c_uint64))
    return out


@dataclass
class Replica:
    """One lattice replica and its per-domain counters (oracle side)."""
    L: int
    Ld: int
    k: int
    seed: int
    beta: float
    J: float = 1.0
    h: float = 0.0
    nu: float = 1.0
    law: int = RATE_METROPOLIS
    init: int = INIT_RANDOM
    spins: np.ndarray = field(default=None)
    esum: np.ndarray = field(default=None)
    steps: np.ndarray = field(default=None)
    hash: np.ndarray = field(default=None)
    flips: np.ndarray = field(default=None)
    sched_done: int = 0
    grad: np.ndarray = field(default=None)
    # per domain: running sums of the score d log P / d(beta, h) and their
    # compensations (the oracle's compensated summation)
    score_acc: np.ndarray = field(default=None)
    dtau: float = 0.0  # domain time per visit (time mode TIME_HORIZON)

    def __post_init__(self):
        if self.spins is None:
            self.spins = init_spins(self.L, self.init, self.seed)
        nD = (self.L // self.Ld) ** 2
        self.esum = np.zeros(nD, dtype=np.float64)
        self.steps = np.zeros(nD, dtype=np.int64)
        self.hash = np.full(nD, lib().orc_hash_basis(), dtype=np.uint64)
        self.flips = np.zeros(nD, dtype=np.int64)
        log2nd = int(round(np.log2(self.Ld * self.Ld)))
        self.a, self.A = rate_table(self.J, self.beta, self.h, self.law, log2nd)

    @property
    def n_domains(self) -> int:
        return (self.L // self.Ld) ** 2

    def enable_score(self):
        """Accumulate the likelihood-ratio score per domain from now on."""
        self.grad = score_table(self.J, self.beta, self.h, self.law)
        self.score_acc = np.zeros((self.n_domains, 4), dtype=np.float64)

    @property
    def score(self):
        """Per-domain score [n_domains, 2] (d/dbeta, d/dh), or None before enable_score."""
        if self.score_acc is None:
            return None
        return self.score_acc[:, 0:2] + self.score_acc[:, 2:4]

    def run(self, n_sched: int, schedule: int = SCHED_PALINDROME,
            time_mode: int = TIME_EXPONENTIAL, obs_every: int = 0, obs_per_pass: bool = False) -> np.ndarray:
        """Run schedules; with obs_per_pass the records are taken after every
        obs_every-th colour pass instead of every obs_every-th schedule."""
        passes = 8 if schedule == SCHED_PALINDROME else 4
        units = n_sched * passes if obs_per_pass else n_sched
        n_obs = units // obs_every if obs_every > 0 else 0
        with_score = self.score_acc is not None
        width = 6 if with_score else 4
        obs = np.zeros((max(n_obs, 1), width), dtype=np.float64)
        s = np.ascontiguousarray(self.spins.reshape(-1))
        A = np.ascontiguousarray(self.A)
        gptr = _ptr(self.grad, ctypes.c_double) if with_score else None
        sptr = _ptr(self.score_acc, ctypes.c_double) if with_score else None
        rc = lib().orc_run_replica_ex(
            _ptr(s, ctypes.c_int8), self.L, self.Ld, self.k, _ptr(A, ctypes.c_uint64),
            self.seed, schedule, time_mode, self.nu, self.J, self.h,
            self.sched_done, n_sched, obs_every, 1 if obs_per_pass else 0, float(self.dtau),
            _ptr(self.esum, ctypes.c_double), _ptr(self.steps, ctypes.c_int64),
            _ptr(self.hash, ctypes.c_uint64), _ptr(self.flips, ctypes.c_int64),
            _ptr(obs, ctypes.c_double), gptr, sptr)
        if rc != 0:
            raise ValueError("oracle rejected the configuration")
        self.spins = s.reshape(self.L, self.L)
        self.sched_done += n_sched
        return obs[:n_obs]

    def domain_times(self, time_mode: int = TIME_EXPONENTIAL) -> np.ndarray:
        nd = self.Ld * self.Ld
        return np.array([lib().orc_domain_time(time_mode, float(self.esum[d]),
                                               int(self.steps[d]), nd, self.nu)
                         for d in range(self.n_domains)])

    def score_nu(self) -> float:
        """d log p / d nu of the exponential clock variates drawn so far (Sec.
        2.1): each uniformised step of domain d waits Exp(n_d nu), log density
        ln(n_d nu) - n_d nu tau, derivative 1/nu - n_d tau; summed over the
        steps of every domain this is sum_d (steps_d - esum_d) / nu, esum_d
        being the domain's sum of -ln v = n_d nu tau.  Valid for runs in
        TIME_EXPONENTIAL only."""
        total = 0.0
        for d in range(self.n_domains):
            total += (float(self.steps[d]) - float(self.esum[d])) / self.nu
        return total

    def observables(self, time_mode: int = TIME_EXPONENTIAL):
        """(e, m, e*m, T) at the current state (Sec. 2.3 endpoint)."""
        b, m = energy_mag(self.spins)
        N = float(self.L * self.L)
        e = (-self.J * float(b) - self.h * float(m)) / N
        mm = float(m) / N
        tsum = 0.0
        for t in self.domain_times(time_mode):
            tsum += float(t)
        T = tsum / self.n_domains
        return e, mm, e * mm, T


# ---------------------------------------------------------------------------
# The 1D ring of Sec. 3.1 (configuration = 64-bit word, bit n = spin n up)
# ---------------------------------------------------------------------------
def ring_rate_table(J: float, beta: float, h: float, law: int, log2_nd: int):
    """(a[6], A[6]) for the ring's classes c = 3*up + (number of up neighbours)."""
    a = np.zeros(6, dtype=np.float64)
    A = np.zeros(6, dtype=np.uint64)
    rc = lib().orc_ring_rate_table(J, beta, h, law, log2_nd, _ptr(a, ctypes.c_double), _ptr(A, ctypes.c_uint64))
    if rc == -2:
        raise ValueError("an acceptance rounds to 0 at 2^-%d (one-way rate)" % (63 - log2_nd))
    if rc != 0:
        raise ValueError("invalid ring rate-table arguments")
    return a, A


def ring_energy_mag(S: int, NS: int):
    b = ctypes.c_int64()
    m = ctypes.c_int64()
    lib().orc_ring_energy_mag(int(S), NS, ctypes.byref(b), ctypes.byref(m))
    return b.value, m.value


def ring_schedule(schedule: int, n: int, seed: int, ND: int):
    """(phases, is_domain): colours per phase, or domains for RANDOM_PERM."""
    out = (ctypes.c_int * 64)()
    isd = ctypes.c_int()
    nph = lib().orc_ring_schedule(schedule, n, seed, ND, out, ctypes.byref(isd))
    if nph < 0:
        raise ValueError("bad ring schedule")
    return [out[i] for i in range(nph)], bool(isd.value)


def ring_passes(schedule: int, ND: int) -> int:
    """Phases ("passes") of one ring schedule."""
    if schedule == SCHED_RANDOM_PERM:
        return ND
    ncol = 1 if ND == 1 else 2
    return 2 * ncol if schedule == SCHED_PALINDROME else ncol


@dataclass
class Ring:
    """One trajectory of the N_S-spin ring cut into N_D = N_S/L_d domains."""
    NS: int
    Ld: int
    k: int
    seed: int
    beta: float
    state: int = 0
    J: float = 1.0
    h: float = 0.0
    nu: float = 1.0
    law: int = RATE_BARKER
    esum: np.ndarray = field(default=None)
    steps: np.ndarray = field(default=None)
    hash: int = 0
    flips: int = 0
    sched_done: int = 0

    def __post_init__(self):
        self.state = int(self.state)
        nD = self.NS // self.Ld
        self.esum = np.zeros(nD, dtype=np.float64)
        self.steps = np.zeros(nD, dtype=np.int64)
        self.hash = int(lib().orc_hash_basis())
        log2nd = int(round(np.log2(self.Ld)))
        self.a, self.A = ring_rate_table(self.J, self.beta, self.h, self.law, log2nd)

    @property
    def n_domains(self) -> int:
        return self.NS // self.Ld

    def run(self, n_sched: int, schedule: int = SCHED_PALINDROME, time_mode: int = TIME_EXPONENTIAL,
            obs_every: int = 0):
        """Run schedules; returns (records [n_rec, 4], states [n_rec]) with a
        record after every obs_every-th pass (phase) of this call."""
        n_rec = n_sched * ring_passes(schedule, self.n_domains) // obs_every if obs_every > 0 else 0
        obs = np.zeros((max(n_rec, 1), 4), dtype=np.float64)
        st = np.zeros(max(n_rec, 1), dtype=np.uint64)
        S = np.array([self.state], dtype=np.uint64)
        H = np.array([self.hash], dtype=np.uint64)
        F = np.array([self.flips], dtype=np.int64)
        A = np.ascontiguousarray(self.A)
        rc = lib().orc_ring_run(_ptr(S, ctypes.c_uint64), self.NS, self.Ld, self.k, _ptr(A, ctypes.c_uint64),
                                self.seed, schedule, time_mode, self.nu, self.J, self.h, self.sched_done,
                                n_sched, obs_every, _ptr(self.esum, ctypes.c_double),
                                _ptr(self.steps, ctypes.c_int64), _ptr(H, ctypes.c_uint64),
                                _ptr(F, ctypes.c_int64), _ptr(obs, ctypes.c_double), _ptr(st, ctypes.c_uint64))
        if rc != 0:
            raise ValueError("oracle rejected the ring configuration")
        self.state, self.hash, self.flips = int(S[0]), int(H[0]), int(F[0])
        self.sched_done += n_sched
        return obs[:n_rec], st[:n_rec]

    def spins(self) -> np.ndarray:
        return np.array([1 if (self.state >> n) & 1 else -1 for n in range(self.NS)], dtype=np.int8)

    def clock(self, time_mode: int = TIME_EXPONENTIAL) -> float:
        tsum = 0.0
        for d in range(self.n_domains):
            tsum += lib().orc_domain_time(time_mode, float(self.esum[d]), int(self.steps[d]), self.Ld, self.nu)
        return tsum / self.n_domains


def ring_run_many(states, seeds, NS: int, Ld: int, k: int, beta: float, n_sched: int, *, J: float = 1.0,
                  h: float = 0.0, nu: float = 1.0, law: int = RATE_BARKER, schedule: int = SCHED_PALINDROME,
                  time_mode: int = TIME_EXPONENTIAL, obs_every: int = 0):
    """Independent ring trajectories from schedule 0 (trajectory r: start
    states[r], seed seeds[r]).  Returns (final states, records
    [n_traj, n_rec, 4], record states [n_traj, n_rec], hashes, flips)."""
    S = np.ascontiguousarray(np.asarray(states, dtype=np.uint64)).copy()
    sd = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    n = len(S)
    _, A = ring_rate_table(J, beta, h, law, int(round(np.log2(Ld))))
    n_rec = n_sched * ring_passes(schedule, NS // Ld) // obs_every if obs_every > 0 else 0
    obs = np.zeros((n, max(n_rec, 1), 4), dtype=np.float64)
    st = np.zeros((n, max(n_rec, 1)), dtype=np.uint64)
    H = np.zeros(n, dtype=np.uint64)
    F = np.zeros(n, dtype=np.int64)
    rc = lib().orc_ring_run_many(n, _ptr(S, ctypes.c_uint64), _ptr(sd, ctypes.c_uint64), NS, Ld, k,
                                 _ptr(A, ctypes.c_uint64), schedule, time_mode, nu, J, h, n_sched, obs_every,
                                 max(n_rec, 1), _ptr(obs, ctypes.c_double), _ptr(st, ctypes.c_uint64),
                                 _ptr(H, ctypes.c_uint64), _ptr(F, ctypes.c_int64))
    if rc != 0:
        raise ValueError("oracle rejected the ring configuration")
    return S, obs[:, :n_rec], st[:, :n_rec], H, F


# ---------------------------------------------------------------------------
# Small 2D lattices under block or vertical-stripe partitions (Sec. 3.2)
# ---------------------------------------------------------------------------
PART_BLOCKS = 0
PART_STRIPES = 1


def part_geometry(L: int, kind: int, ND: int, d: int):
    """(x0, y0, width, height, colour) of domain d; colour -1 when the
    partition cannot be coloured (odd number of stripes or blocks per side)."""
    v = [ctypes.c_int() for _ in range(5)]
    if lib().orc_part_geometry(L, kind, ND, d, *[ctypes.byref(x) for x in v]) != 0:
        raise ValueError("bad partition")
    return tuple(x.value for x in v)


def part_schedule(kind: int, schedule: int, n: int, seed: int, ND: int):
    out = (ctypes.c_int * 64)()
    isd = ctypes.c_int()
    nph = lib().orc_part_schedule(kind, schedule, n, seed, ND, out, ctypes.byref(isd))
    if nph < 0:
        raise ValueError("bad partition schedule")
    return [out[i] for i in range(nph)], bool(isd.value)


def part_scale(L: int, kind: int, ND: int):
    """(P, M): fixed-point bits of the acceptance and M = n_d 2^P."""
    M = np.zeros(1, dtype=np.uint64)
    P = lib().orc_part_scale(L, kind, ND, _ptr(M, ctypes.c_uint64))
    if P < 0:
        raise ValueError("bad partition")
    return int(P), int(M[0])


def part_passes(kind: int, schedule: int, ND: int) -> int:
    if schedule == SCHED_RANDOM_PERM:
        return ND
    nc = 1 if ND == 1 else (4 if kind == PART_BLOCKS else 2)
    return 2 * nc if schedule == SCHED_PALINDROME else nc


@dataclass
class Partitioned:
    """One trajectory of an L x L lattice cut into N_D blocks or stripes."""
    L: int
    kind: int
    ND: int
    k: int
    seed: int
    beta: float
    spins: np.ndarray = field(default=None)
    J: float = 1.0
    h: float = 0.0
    nu: float = 1.0
    law: int = RATE_BARKER
    esum: np.ndarray = field(default=None)
    steps: np.ndarray = field(default=None)
    hash: int = 0
    flips: int = 0
    sched_done: int = 0

    def __post_init__(self):
        if self.spins is None:
            self.spins = np.ones((self.L, self.L), dtype=np.int8)
        self.spins = np.ascontiguousarray(self.spins, dtype=np.int8).copy()
        self.esum = np.zeros(self.ND, dtype=np.float64)
        self.steps = np.zeros(self.ND, dtype=np.int64)
        self.hash = int(lib().orc_hash_basis())
        self.P, self.M = part_scale(self.L, self.kind, self.ND)
        self.a, self.A = rate_table(self.J, self.beta, self.h, self.law, 63 - self.P)

    def run(self, n_sched: int, schedule: int = SCHED_PALINDROME, time_mode: int = TIME_EXPONENTIAL,
            obs_every: int = 0) -> np.ndarray:
        n_rec = n_sched * part_passes(self.kind, schedule, self.ND) // obs_every if obs_every > 0 else 0
        obs = np.zeros((max(n_rec, 1), 4), dtype=np.float64)
        s = self.spins.reshape(-1)
        H = np.array([self.hash], dtype=np.uint64)
        F = np.array([self.flips], dtype=np.int64)
        A = np.ascontiguousarray(self.A)
        rc = lib().orc_part_run(_ptr(s, ctypes.c_int8), self.L, self.kind, self.ND, self.k, _ptr(A, ctypes.c_uint64),
                                self.seed, schedule, time_mode, self.nu, self.J, self.h, self.sched_done, n_sched,
                                obs_every, _ptr(self.esum, ctypes.c_double), _ptr(self.steps, ctypes.c_int64),
                                _ptr(H, ctypes.c_uint64), _ptr(F, ctypes.c_int64), _ptr(obs, ctypes.c_double))
        if rc != 0:
            raise ValueError("oracle rejected the partitioned configuration")
        self.hash, self.flips = int(H[0]), int(F[0])
        self.sched_done += n_sched
        return obs[:n_rec]

    def clock(self, time_mode: int = TIME_EXPONENTIAL) -> float:
        x0, y0, w, hh, _ = part_geometry(self.L, self.kind, self.ND, 0)
        tsum = 0.0
        for d in range(self.ND):
            tsum += lib().orc_domain_time(time_mode, float(self.esum[d]), int(self.steps[d]), w * hh, self.nu)
        return tsum / self.ND


def part_run_many(s0, seeds, L: int, kind: int, ND: int, k: int, beta: float, n_sched: int, *, J: float = 1.0,
                  h: float = 0.0, nu: float = 1.0, law: int = RATE_BARKER, schedule: int = SCHED_PALINDROME,
                  time_mode: int = TIME_EXPONENTIAL, obs_every: int = 0):
    """Independent partitioned trajectories from the same start s0 [L, L].
    Returns (final spins [n, L, L], records [n, n_rec, 4], hashes, flips)."""
    s0 = np.ascontiguousarray(s0, dtype=np.int8).reshape(-1)
    sd = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    n = len(sd)
    P, _ = part_scale(L, kind, ND)
    _, A = rate_table(J, beta, h, law, 63 - P)
    n_rec = n_sched * part_passes(kind, schedule, ND) // obs_every if obs_every > 0 else 0
    out = np.zeros((n, L, L), dtype=np.int8)
    obs = np.zeros((n, max(n_rec, 1), 4), dtype=np.float64)
    H = np.zeros(n, dtype=np.uint64)
    F = np.zeros(n, dtype=np.int64)
    rc = lib().orc_part_run_many(n, _ptr(s0, ctypes.c_int8), _ptr(sd, ctypes.c_uint64), L, kind, ND, k,
                                 _ptr(A, ctypes.c_uint64), schedule, time_mode, nu, J, h, n_sched, obs_every,
                                 max(n_rec, 1), _ptr(out, ctypes.c_int8), _ptr(obs, ctypes.c_double),
                                 _ptr(H, ctypes.c_uint64), _ptr(F, ctypes.c_int64))
    if rc != 0:
        raise ValueError("oracle rejected the partitioned configuration")
    return out, obs[:, :n_rec], H, F
