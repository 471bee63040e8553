"""Thin Python binding of the C ABI (include/kmc.h), same names.

Argument marshalling only: every step of the method runs in the CUDA library
(libkmc_gb300.so).  PyTorch provides the device buffers and the stream.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from ._lib import KmcError, load

KMC_INIT_RANDOM, KMC_INIT_ALL_UP, KMC_INIT_KEEP, KMC_INIT_PER_REPLICA = 0, 1, 2, 3
KMC_RATE_METROPOLIS, KMC_RATE_BARKER = 0, 1
KMC_SCHEDULE_PALINDROME, KMC_SCHEDULE_FIXED, KMC_SCHEDULE_RANDOM_PERM = 0, 1, 2
KMC_TIME_EXPONENTIAL, KMC_TIME_EXPECTED, KMC_TIME_HORIZON = 0, 1, 2
KMC_LAUNCH_AUTO, KMC_LAUNCH_CLUSTER, KMC_LAUNCH_GRID, KMC_LAUNCH_THREADS = 0, 1, 2, 3
KMC_OBS_SCHEDULE, KMC_OBS_PASS = 0, 1

_i32, _i64, _u64, _dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double


def _arr(values, ctype):
    vals = list(values)
    return (ctype * len(vals))(*vals)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _check(ctx, status: int):
    if status != 0:
        msg = load().kmc_last_error(ctx)
        raise KmcError(status, msg.decode() if msg else "")


def kmc_version() -> int:
    return load().kmc_version()


def kmc_create_lattice(L: Sequence[int], L_d: int, k_steps: int, init: int, seeds: Sequence[int],
                       spins_dev: torch.Tensor, stream=None) -> ctypes.c_void_p:
    lib = load()
    if not torch.cuda.is_available():
        raise KmcError(-3, "no CUDA device: the library has no CPU path")
    if spins_dev.dtype != torch.int8 or not spins_dev.is_cuda or not spins_dev.is_contiguous():
        raise KmcError(-1, "spins_dev must be a contiguous int8 CUDA tensor")
    need = sum(int(x) * int(x) for x in L)
    if spins_dev.numel() < need:
        raise KmcError(-1, "spins_dev holds %d bytes, %d needed" % (spins_dev.numel(), need))
    ctx = ctypes.c_void_p()
    st = lib.kmc_create_lattice(ctypes.byref(ctx), len(L), _arr(L, _i32), L_d, k_steps, init,
                                _arr(seeds, _u64), ctypes.c_void_p(spins_dev.data_ptr()),
                                ctypes.c_void_p(_stream_handle(stream)))
    if st != 0:
        msg = lib.kmc_last_error(ctx).decode() if ctx.value else ""
        if ctx.value:
            lib.kmc_destroy(ctx)
        raise KmcError(st, msg)
    return ctx


def kmc_set_rates(ctx, J: float, beta: Sequence[float], h: Sequence[float], nu: float, rate_law: int):
    _check(ctx, load().kmc_set_rates(ctx, J, _arr(beta, _dbl), _arr(h, _dbl), nu, rate_law))


def kmc_set_rate_table(ctx, J: float, beta, h, nu: float, a: np.ndarray):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    _check(ctx, load().kmc_set_rate_table(ctx, J, _arr(beta, _dbl), _arr(h, _dbl), nu,
                                          a.ctypes.data_as(ctypes.POINTER(_dbl))))


def kmc_run_schedule(ctx, n_schedules: int, schedule: int, time_mode: int, obs_every: int,
                     obs_dev: Optional[torch.Tensor], stream=None):
    ptr = ctypes.c_void_p(obs_dev.data_ptr()) if obs_dev is not None else ctypes.c_void_p()
    if obs_dev is not None and (obs_dev.dtype != torch.float64 or not obs_dev.is_cuda):
        raise KmcError(-1, "obs_dev must be a float64 CUDA tensor")
    _check(ctx, load().kmc_run_schedule(ctx, n_schedules, schedule, time_mode, obs_every, ptr,
                                        ctypes.c_void_p(_stream_handle(stream))))


def kmc_observables(ctx, n_replicas: int):
    e, m, t = ((_dbl * n_replicas)() for _ in range(3))
    steps, flips = (_i64 * n_replicas)(), (_i64 * n_replicas)()
    _check(ctx, load().kmc_observables(ctx, e, m, t, steps, flips))
    return {"e": np.array(e[:]), "m": np.array(m[:]), "t": np.array(t[:]),
            "steps": np.array(steps[:], dtype=np.int64), "flips": np.array(flips[:], dtype=np.int64)}


def kmc_domain_state(ctx, n_domains: int):
    hs, fl, tt = (_u64 * n_domains)(), (_i64 * n_domains)(), (_dbl * n_domains)()
    _check(ctx, load().kmc_domain_state(ctx, hs, fl, tt))
    return (np.array(hs[:], dtype=np.uint64), np.array(fl[:], dtype=np.int64),
            np.array(tt[:], dtype=np.float64))


def kmc_get_rate_table(ctx, replica: int):
    a, A = (_dbl * 10)(), (_u64 * 10)()
    _check(ctx, load().kmc_get_rate_table(ctx, replica, a, A))
    return np.array(a[:]), np.array(A[:], dtype=np.uint64)


def kmc_rate_table_error(ctx) -> float:
    v = _dbl()
    _check(ctx, load().kmc_rate_table_error(ctx, ctypes.byref(v)))
    return v.value


def kmc_grad(ctx, score_dev: torch.Tensor, reset: int = 0):
    if score_dev.dtype != torch.float64 or not score_dev.is_cuda:
        raise KmcError(-1, "score_dev must be a float64 CUDA tensor")
    _check(ctx, load().kmc_grad(ctx, ctypes.c_void_p(score_dev.data_ptr()), reset))


def kmc_grad_nu(ctx, score_dev: torch.Tensor):
    if score_dev.dtype != torch.float64 or not score_dev.is_cuda:
        raise KmcError(-1, "score_dev must be a float64 CUDA tensor")
    _check(ctx, load().kmc_grad_nu(ctx, ctypes.c_void_p(score_dev.data_ptr())))


def kmc_lr_estimate(ctx, A_dev: torch.Tensor, grad_dev: torch.Tensor, stream=None):
    if A_dev.dtype != torch.float64 or grad_dev.dtype != torch.float64 or not A_dev.is_cuda:
        raise KmcError(-1, "A_dev and grad_dev must be float64 CUDA tensors")
    _check(ctx, load().kmc_lr_estimate(ctx, ctypes.c_void_p(A_dev.data_ptr()),
                                       ctypes.c_void_p(grad_dev.data_ptr())))


def kmc_lr_observable(ctx, rec_dev: torch.Tensor, observable: int, out_dev: torch.Tensor, stream=None):
    if rec_dev.dtype != torch.float64 or not rec_dev.is_cuda or rec_dev.dim() != 2 or rec_dev.stride(1) != 1:
        raise KmcError(-1, "rec_dev must be a float64 CUDA tensor [n_replicas, width] with unit column stride")
    if out_dev.dtype != torch.float64 or not out_dev.is_cuda or out_dev.numel() < 3 or not out_dev.is_contiguous():
        raise KmcError(-1, "out_dev must be a contiguous float64 CUDA tensor of 3 elements")
    _check(ctx, load().kmc_lr_observable(ctx, ctypes.c_void_p(rec_dev.data_ptr()), int(rec_dev.stride(0)),
                                         int(observable), ctypes.c_void_p(out_dev.data_ptr())))


def kmc_enable_grad(ctx, enable: bool):
    _check(ctx, load().kmc_enable_grad(ctx, int(bool(enable))))


def kmc_reset(ctx, init: int, stream=None):
    _check(ctx, load().kmc_reset(ctx, init, ctypes.c_void_p(_stream_handle(stream))))


def kmc_set_replica_params(ctx, k_steps: Optional[Sequence[int]] = None, init: Optional[Sequence[int]] = None):
    kp = ctypes.cast(_arr(k_steps, _i32), ctypes.c_void_p) if k_steps is not None else None
    ip = ctypes.cast(_arr(init, _i32), ctypes.c_void_p) if init is not None else None
    _check(ctx, load().kmc_set_replica_params(ctx, kp, ip))


def kmc_set_horizon(ctx, dtau: float):
    _check(ctx, load().kmc_set_horizon(ctx, float(dtau)))


def kmc_set_observation(ctx, unit: int):
    _check(ctx, load().kmc_set_observation(ctx, unit))


def kmc_sync(ctx):
    _check(ctx, load().kmc_sync(ctx))


def kmc_set_launch(ctx, mode: int, size: int, warps_per_cta: int):
    _check(ctx, load().kmc_set_launch(ctx, mode, size, warps_per_cta))


def kmc_get_launch(ctx):
    """(mode, size, ctas, warps_per_cta, smem_bytes) of the current plan."""
    v = [_i32() for _ in range(5)]
    _check(ctx, load().kmc_get_launch(ctx, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def kmc_debug_barrier(ctx, extra: int, limit_ns: int):
    _check(ctx, load().kmc_debug_barrier(ctx, extra, limit_ns))


def kmc_profile(ctx, enable: bool):
    _check(ctx, load().kmc_profile(ctx, int(bool(enable))))


def kmc_profile_read(ctx):
    ms, n = _dbl(), _i64()
    _check(ctx, load().kmc_profile_read(ctx, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def kmc_profile_polls(ctx) -> int:
    n = _i64()
    _check(ctx, load().kmc_profile_polls(ctx, ctypes.byref(n)))
    return n.value


def kmc_run_schedule_noalloc(L: int, L_d: int, k_steps: int, seed: int, J: float, beta: float, h: float,
                             nu: float, rate_law: int, sched_begin: int, n_schedules: int, schedule: int,
                             time_mode: int, obs_every: int, spins_dev: torch.Tensor,
                             obs_dev: Optional[torch.Tensor] = None, stream=None):
    """One replica, no device allocation (see include/kmc.h); raises KmcError on failure.

    The C function receives bare pointers and cannot check buffer sizes, so
    they are checked here: spins_dev holds at least L*L int8, and with
    obs_every > 0 obs_dev holds at least (records) * 4 float64."""
    if spins_dev.dtype != torch.int8 or not spins_dev.is_cuda or not spins_dev.is_contiguous():
        raise KmcError(-1, "spins_dev must be a contiguous int8 CUDA tensor")
    if spins_dev.numel() < int(L) * int(L):
        raise KmcError(-1, "spins_dev holds %d bytes, %d needed" % (spins_dev.numel(), int(L) * int(L)))
    if obs_every > 0:
        n_rec = int(n_schedules) // int(obs_every)
        if n_rec > 0:
            if obs_dev is None or obs_dev.dtype != torch.float64 or not obs_dev.is_cuda or not obs_dev.is_contiguous():
                raise KmcError(-1, "obs_dev must be a contiguous float64 CUDA tensor when obs_every > 0")
            if obs_dev.numel() < n_rec * 4:
                raise KmcError(-1, "obs_dev holds %d doubles, %d needed" % (obs_dev.numel(), n_rec * 4))
    err = ctypes.create_string_buffer(256)
    obs_ptr = ctypes.c_void_p(obs_dev.data_ptr()) if obs_dev is not None else ctypes.c_void_p()
    st = load().kmc_run_schedule_noalloc(L, L_d, k_steps, seed, J, beta, h, nu, rate_law, sched_begin,
                                         n_schedules, schedule, time_mode, obs_every,
                                         ctypes.c_void_p(spins_dev.data_ptr()), obs_ptr,
                                         ctypes.c_void_p(_stream_handle(stream)), err, len(err))
    if st != 0:
        raise KmcError(st, err.value.decode())


def kmc_kernel_launches(ctx) -> int:
    return load().kmc_kernel_launches(ctx)


def kmc_domain_side(ctx) -> int:
    return load().kmc_domain_side(ctx)


def kmc_destroy(ctx):
    if ctx is not None and ctx.value:
        load().kmc_destroy(ctx)


class Lattice:
    """A batch of replicas bound to one library context (convenience wrapper).

    spins: int8 CUDA tensor, replicas concatenated row-major (allocated here
    unless given).  Methods map one-to-one onto the C entry points.
    """

    def __init__(self, L: Sequence[int], L_d: int, k: int, seeds: Sequence[int],
                 init: int = KMC_INIT_RANDOM, spins: Optional[torch.Tensor] = None, stream=None,
                 device: Optional[torch.device] = None):
        self.L = [int(x) for x in L]
        self.L_d = int(L_d)
        self.k = int(k)
        self.ks = [self.k] * len(self.L)  # per-replica steps per visit
        self.seeds = [int(s) for s in seeds]
        total = sum(x * x for x in self.L)
        if spins is None:
            dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
            spins = torch.empty(total, dtype=torch.int8, device=dev)
        self.spins = spins
        self.offsets = np.concatenate([[0], np.cumsum([x * x for x in self.L])]).astype(np.int64)
        self.ctx = kmc_create_lattice(self.L, self.L_d, self.k, init, self.seeds, self.spins, stream)
        self.L_d = int(load().kmc_domain_side(self.ctx))  # the library's choice when L_d = 0
        self.dom_offsets = np.concatenate([[0], np.cumsum([(x // self.L_d) ** 2 for x in self.L])]).astype(np.int64)
        self.grad_enabled = False
        self.obs_unit = KMC_OBS_SCHEDULE

    @property
    def n_replicas(self) -> int:
        return len(self.L)

    @property
    def n_domains(self) -> int:
        return int(self.dom_offsets[-1])

    def replica_spins(self, r: int) -> torch.Tensor:
        a, b = int(self.offsets[r]), int(self.offsets[r + 1])
        return self.spins[a:b].view(self.L[r], self.L[r])

    def set_rates(self, beta, h=None, J: float = 1.0, nu: float = 1.0, law: int = KMC_RATE_METROPOLIS):
        beta = np.broadcast_to(np.asarray(beta, dtype=np.float64), (self.n_replicas,))
        h = np.zeros(self.n_replicas) if h is None else np.broadcast_to(np.asarray(h, dtype=np.float64), (self.n_replicas,))
        self.J = J
        kmc_set_rates(self.ctx, J, beta.tolist(), h.tolist(), nu, law)

    def run(self, n_schedules: int, schedule: int = KMC_SCHEDULE_PALINDROME,
            time_mode: int = KMC_TIME_EXPONENTIAL, obs_every: int = 0, stream=None,
            out: Optional[torch.Tensor] = None) -> Optional[torch.Tensor]:
        """Run schedules; returns the observation records [n_obs, n_replicas, 4 or 6]
        (written into `out` when given, e.g. a buffer allocated before a graph capture)."""
        obs = None
        units = n_schedules
        if self.obs_unit == KMC_OBS_PASS:
            units *= 8 if schedule == KMC_SCHEDULE_PALINDROME else 4
        if obs_every > 0 and units // obs_every > 0:
            width = 6 if self.grad_enabled else 4
            shape = (units // obs_every, self.n_replicas, width)
            if out is not None:
                if tuple(out.shape) != shape or out.dtype != torch.float64 or not out.is_contiguous():
                    raise KmcError(-1, "out must be a contiguous float64 tensor of shape %s" % (shape,))
                obs = out
            else:
                obs = torch.empty(shape, dtype=torch.float64, device=self.spins.device)
        kmc_run_schedule(self.ctx, n_schedules, schedule, time_mode, obs_every, obs, stream)
        return obs

    def observables(self):
        return kmc_observables(self.ctx, self.n_replicas)

    def domain_state(self):
        return kmc_domain_state(self.ctx, self.n_domains)

    def rate_table(self, r: int = 0):
        return kmc_get_rate_table(self.ctx, r)

    def rate_table_error(self) -> float:
        """Largest relative change |A_c 2^-P - a_c| / a_c of an acceptance by the fixed point."""
        return kmc_rate_table_error(self.ctx)

    def enable_grad(self, enable: bool = True):
        kmc_enable_grad(self.ctx, enable)
        self.grad_enabled = bool(enable)

    def score(self, reset: bool = False) -> torch.Tensor:
        out = torch.empty((self.n_replicas, 2), dtype=torch.float64, device=self.spins.device)
        kmc_grad(self.ctx, out, int(reset))
        return out

    def score_nu(self) -> torch.Tensor:
        """d log P / d nu of the exponential clocks since the last reset, per replica."""
        out = torch.empty(self.n_replicas, dtype=torch.float64, device=self.spins.device)
        kmc_grad_nu(self.ctx, out)
        return out

    def lr_estimate(self, A: torch.Tensor) -> torch.Tensor:
        """d E[A] / d(beta, h) from per-replica A and the accumulated scores."""
        out = torch.empty(2, dtype=torch.float64, device=self.spins.device)
        kmc_lr_estimate(self.ctx, A.contiguous(), out)
        return out

    def lr_observable(self, record: torch.Tensor, observable: int) -> torch.Tensor:
        """[mean A, dE[A]/dbeta, dE[A]/dh] of observable 0 (e), 1 (m) or 2 (e*m)
        from one record row [n_replicas, width] and the accumulated scores."""
        if record.shape[0] != self.n_replicas:
            raise KmcError(-1, "record must have one row per replica")
        out = torch.empty(3, dtype=torch.float64, device=self.spins.device)
        kmc_lr_observable(self.ctx, record, observable, out)
        return out

    def reset(self, init: int = KMC_INIT_RANDOM, stream=None):
        kmc_reset(self.ctx, init, stream)

    def sync(self):
        kmc_sync(self.ctx)

    def set_horizon(self, dtau: float):
        """Domain time per visit for KMC_TIME_HORIZON runs (0 turns it off)."""
        kmc_set_horizon(self.ctx, dtau)

    def set_observation(self, unit: int):
        """KMC_OBS_SCHEDULE: records at schedule endpoints; KMC_OBS_PASS: at
        every colour pass (register-shifted endpoints, Sec. 2.3)."""
        kmc_set_observation(self.ctx, unit)
        self.obs_unit = unit

    def set_replica_params(self, k: Optional[Sequence[int]] = None, init: Optional[Sequence[int]] = None):
        """Per-replica steps per visit and start modes (kmc_reset with
        KMC_INIT_PER_REPLICA uses the modes)."""
        if k is not None:
            k = [int(x) for x in k]
            assert len(k) == self.n_replicas
        if init is not None:
            init = [int(x) for x in init]
            assert len(init) == self.n_replicas
        kmc_set_replica_params(self.ctx, k, init)
        if k is not None:
            self.ks = k

    def events_per_schedule(self, schedule: int = KMC_SCHEDULE_PALINDROME) -> int:
        """Uniformised steps of one schedule over all replicas (Eq. 11)."""
        visits = 2 if schedule == KMC_SCHEDULE_PALINDROME else 1
        return int(sum(visits * (x // self.L_d) ** 2 * k for x, k in zip(self.L, self.ks)))

    def set_launch(self, mode: int = KMC_LAUNCH_AUTO, size: int = 0, warps_per_cta: int = 16):
        """Launch plan (kmc_set_launch): size is the cluster size, the grid's
        CTA count, or for the thread plans of L_d = 16, 32, 64 the domain
        order over the warps (0 or 1 replica after replica, 2 round-robin)."""
        kmc_set_launch(self.ctx, mode, size, warps_per_cta)

    def launch(self):
        return kmc_get_launch(self.ctx)

    def profile(self, enable: bool = True):
        kmc_profile(self.ctx, enable)

    def profile_read(self):
        """(summed run-kernel milliseconds, timed launches) since the last read."""
        return kmc_profile_read(self.ctx)

    def profile_polls(self) -> int:
        """Halo-poll iterations of the profiled launches since the last read."""
        return kmc_profile_polls(self.ctx)

    def kernel_launches(self) -> int:
        return kmc_kernel_launches(self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            kmc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# The 1D ring (Sec. 3.1): C-ABI wrappers and a convenience class
# ---------------------------------------------------------------------------
def _ring_check(ring, status: int):
    if status != 0:
        msg = load().kmc_ring_last_error(ring)
        raise KmcError(status, msg.decode() if msg else "")


def kmc_ring_create(n_sites: int, L_d: int, k_steps: int, seeds: Sequence[int], init: Sequence[int],
                    stream=None) -> ctypes.c_void_p:
    lib = load()
    if not torch.cuda.is_available():
        raise KmcError(-3, "no CUDA device: the library has no CPU path")
    seeds = [int(x) for x in seeds]
    init = [int(x) for x in init]
    if len(seeds) != len(init):
        raise KmcError(-1, "one seed and one starting word per trajectory")
    ring = ctypes.c_void_p()
    st = lib.kmc_ring_create(ctypes.byref(ring), len(seeds), n_sites, L_d, k_steps, _arr(seeds, _u64),
                             _arr(init, _u64), ctypes.c_void_p(_stream_handle(stream)))
    if st != 0:
        raise KmcError(st, "kmc_ring_create rejected n_traj=%d N_S=%d L_d=%d k=%d" % (len(seeds), n_sites, L_d,
                                                                                        k_steps))
    return ring


def kmc_ring_set_rates(ring, J: float, beta: Sequence[float], h: Sequence[float], nu: float, rate_law: int):
    _ring_check(ring, load().kmc_ring_set_rates(ring, J, _arr(beta, _dbl), _arr(h, _dbl), nu, rate_law))


def kmc_ring_run(ring, n_schedules: int, schedule: int, time_mode: int, obs_every: int,
                 obs_dev: Optional[torch.Tensor], state_dev: Optional[torch.Tensor], ens_dev: Optional[torch.Tensor],
                 stream=None):
    def ptr(t, dtype):
        if t is None:
            return None
        if t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
            raise KmcError(-1, "buffers must be contiguous CUDA tensors of dtype %s" % dtype)
        return ctypes.c_void_p(t.data_ptr())
    _ring_check(ring, load().kmc_ring_run(ring, n_schedules, schedule, time_mode, obs_every,
                                          ptr(obs_dev, torch.float64), ptr(state_dev, torch.int64),
                                          ptr(ens_dev, torch.int64), ctypes.c_void_p(_stream_handle(stream))))


def kmc_ring_state(ring, n_traj: int):
    S = (_u64 * n_traj)()
    H = (_u64 * n_traj)()
    F = (_i64 * n_traj)()
    St = (_i64 * n_traj)()
    T = (_dbl * n_traj)()
    _ring_check(ring, load().kmc_ring_state(ring, S, H, F, St, T))
    return (np.frombuffer(S, dtype=np.uint64).copy(), np.frombuffer(H, dtype=np.uint64).copy(),
            np.frombuffer(F, dtype=np.int64).copy(), np.frombuffer(St, dtype=np.int64).copy(),
            np.frombuffer(T, dtype=np.float64).copy())


def kmc_ring_destroy(ring):
    load().kmc_ring_destroy(ring)


def ring_passes(schedule: int, n_domains: int) -> int:
    """Phases of one ring schedule: N_D for random domain orders, else 4 / 2
    colour passes (2 / 1 when N_D = 1)."""
    if schedule == KMC_SCHEDULE_RANDOM_PERM:
        return n_domains
    ncol = 1 if n_domains == 1 else 2
    return 2 * ncol if schedule == KMC_SCHEDULE_PALINDROME else ncol


class Ring:
    """n_traj trajectories of an N_S-spin ring cut into N_S/L_d domains
    (Sec. 3.1), one GPU thread each."""

    def __init__(self, n_sites: int, L_d: int, k: int, seeds: Sequence[int], init: Sequence[int], stream=None):
        self.n_sites, self.L_d, self.k = int(n_sites), int(L_d), int(k)
        self.n_traj = len(seeds)
        self.ctx = kmc_ring_create(n_sites, L_d, k, seeds, init, stream)

    @property
    def n_domains(self) -> int:
        return self.n_sites // self.L_d

    def set_rates(self, beta, h=None, J: float = 1.0, nu: float = 1.0, law: int = KMC_RATE_BARKER):
        beta = list(beta) if hasattr(beta, "__len__") else [float(beta)] * self.n_traj
        h = [0.0] * self.n_traj if h is None else (list(h) if hasattr(h, "__len__") else [float(h)] * self.n_traj)
        kmc_ring_set_rates(self.ctx, J, beta, h, nu, law)

    def n_records(self, n_sched: int, schedule: int, obs_every: int) -> int:
        return n_sched * ring_passes(schedule, self.n_domains) // obs_every if obs_every > 0 else 0

    def run(self, n_sched: int, schedule: int = KMC_SCHEDULE_PALINDROME, time_mode: int = KMC_TIME_EXPONENTIAL,
            obs_every: int = 0, records: bool = True, states: bool = False, ensemble: bool = False, stream=None,
            out=None):
        """Returns (obs [n_rec, n_traj, 4] | None, states [n_rec, n_traj] int64 | None,
        ens [n_rec, 4 + N_S] int64 | None); out = that tuple of buffers to reuse."""
        n_rec = self.n_records(n_sched, schedule, obs_every)
        dev = torch.device("cuda", torch.cuda.current_device())
        if out is not None:
            obs, st, ens = out
        else:
            obs = torch.empty((n_rec, self.n_traj, 4), dtype=torch.float64, device=dev) \
                if (records and n_rec > 0) else None
            st = torch.empty((n_rec, self.n_traj), dtype=torch.int64, device=dev) if (states and n_rec > 0) else None
            ens = torch.empty((n_rec, 4 + self.n_sites), dtype=torch.int64, device=dev) \
                if (ensemble and n_rec > 0) else None
        kmc_ring_run(self.ctx, n_sched, schedule, time_mode, obs_every, obs, st, ens, stream)
        return obs, st, ens

    def state(self):
        """(words, hashes, flips, steps, T) on the host."""
        return kmc_ring_state(self.ctx, self.n_traj)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            kmc_ring_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Small lattices under block or vertical-stripe partitions (Sec. 3.2)
# ---------------------------------------------------------------------------
KMC_PART_BLOCKS, KMC_PART_STRIPES = 0, 1


def _part_check(part, status: int):
    if status != 0:
        msg = load().kmc_part_last_error(part)
        raise KmcError(status, msg.decode() if msg else "")


def kmc_part_create(L: int, partition: int, n_domains: int, k_steps: int, seeds: Sequence[int],
                    spins_dev: torch.Tensor, stream=None) -> ctypes.c_void_p:
    lib = load()
    if not torch.cuda.is_available():
        raise KmcError(-3, "no CUDA device: the library has no CPU path")
    seeds = [int(x) for x in seeds]
    if spins_dev.dtype != torch.int8 or not spins_dev.is_cuda or not spins_dev.is_contiguous() \
            or spins_dev.numel() != len(seeds) * L * L:
        raise KmcError(-1, "spins_dev must be a contiguous int8 CUDA tensor [n_traj, L, L]")
    part = ctypes.c_void_p()
    st = lib.kmc_part_create(ctypes.byref(part), len(seeds), L, partition, n_domains, k_steps, _arr(seeds, _u64),
                             ctypes.c_void_p(spins_dev.data_ptr()), ctypes.c_void_p(_stream_handle(stream)))
    if st != 0:
        raise KmcError(st, "kmc_part_create rejected L=%d partition=%d N_D=%d k=%d" % (L, partition, n_domains,
                                                                                       k_steps))
    return part


def kmc_part_set_rates(part, J: float, beta: Sequence[float], h: Sequence[float], nu: float, rate_law: int):
    _part_check(part, load().kmc_part_set_rates(part, J, _arr(beta, _dbl), _arr(h, _dbl), nu, rate_law))


def kmc_part_run(part, n_schedules: int, schedule: int, time_mode: int, obs_every: int,
                 obs_dev: Optional[torch.Tensor], stream=None):
    if obs_dev is not None and (obs_dev.dtype != torch.float64 or not obs_dev.is_cuda or not obs_dev.is_contiguous()):
        raise KmcError(-1, "obs_dev must be a contiguous float64 CUDA tensor")
    _part_check(part, load().kmc_part_run(part, n_schedules, schedule, time_mode, obs_every,
                                          None if obs_dev is None else ctypes.c_void_p(obs_dev.data_ptr()),
                                          ctypes.c_void_p(_stream_handle(stream))))


def kmc_part_state(part, n_traj: int):
    H = (_u64 * n_traj)()
    F = (_i64 * n_traj)()
    St = (_i64 * n_traj)()
    T = (_dbl * n_traj)()
    _part_check(part, load().kmc_part_state(part, H, F, St, T))
    return (np.frombuffer(H, dtype=np.uint64).copy(), np.frombuffer(F, dtype=np.int64).copy(),
            np.frombuffer(St, dtype=np.int64).copy(), np.frombuffer(T, dtype=np.float64).copy())


def kmc_part_destroy(part):
    load().kmc_part_destroy(part)


def part_passes(partition: int, schedule: int, n_domains: int) -> int:
    if schedule == KMC_SCHEDULE_RANDOM_PERM:
        return n_domains
    nc = 1 if n_domains == 1 else (4 if partition == KMC_PART_BLOCKS else 2)
    return 2 * nc if schedule == KMC_SCHEDULE_PALINDROME else nc


class Partitioned:
    """n_traj trajectories of an L x L lattice (L <= 128) cut into N_D square
    blocks or vertical stripes (Sec. 3.2), one GPU warp each.  `spins` is the
    caller-visible int8 state [n_traj, L, L]."""

    def __init__(self, L: int, partition: int, n_domains: int, k: int, seeds: Sequence[int],
                 spins: Optional[torch.Tensor] = None, stream=None):
        self.L, self.partition, self.n_domains, self.k = int(L), int(partition), int(n_domains), int(k)
        self.n_traj = len(seeds)
        if spins is None:
            spins = torch.ones((self.n_traj, L, L), dtype=torch.int8, device="cuda")
        self.spins = spins
        self.ctx = kmc_part_create(L, partition, n_domains, k, seeds, spins, stream)

    def set_rates(self, beta, h=None, J: float = 1.0, nu: float = 1.0, law: int = KMC_RATE_BARKER):
        beta = list(beta) if hasattr(beta, "__len__") else [float(beta)] * self.n_traj
        h = [0.0] * self.n_traj if h is None else (list(h) if hasattr(h, "__len__") else [float(h)] * self.n_traj)
        kmc_part_set_rates(self.ctx, J, beta, h, nu, law)

    def n_records(self, n_sched: int, schedule: int, obs_every: int) -> int:
        return n_sched * part_passes(self.partition, schedule, self.n_domains) // obs_every if obs_every > 0 else 0

    def run(self, n_sched: int, schedule: int = KMC_SCHEDULE_PALINDROME, time_mode: int = KMC_TIME_EXPONENTIAL,
            obs_every: int = 0, stream=None, out: Optional[torch.Tensor] = None) -> Optional[torch.Tensor]:
        n_rec = self.n_records(n_sched, schedule, obs_every)
        obs = out
        if obs is None and n_rec > 0:
            obs = torch.empty((n_rec, self.n_traj, 4), dtype=torch.float64, device=self.spins.device)
        kmc_part_run(self.ctx, n_sched, schedule, time_mode, obs_every, obs, stream)
        return obs

    def state(self):
        """(hashes, flips, steps, T) on the host."""
        return kmc_part_state(self.ctx, self.n_traj)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            kmc_part_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
