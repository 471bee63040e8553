"""The C-ABI library builds, loads and exports every entry point of include/kmc.h (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1403_4674_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "kmc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kmc_[a-z_]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol():
    build.build()
    lib = ctypes.CDLL(build.LIB)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_null_context():
    lib = _lib.load()
    assert lib.kmc_version() >= 10000
    assert lib.kmc_last_error(None) == b"null context"
    assert lib.kmc_run_schedule(None, 1, 0, 0, 0, None, None) == _lib.KMC_EINVAL
    assert lib.kmc_kernel_launches(None) == 0


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1403_4674_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                for bad in ("import oracle", "from oracle", "liborc", "kmc_oracle"):
                    assert bad not in src, (f, bad)


def test_autotune_host_logic():
    from paper_1403_4674_gb300 import autotune
    assert autotune.max_domain_side(32) == 16
    assert autotune.max_domain_side(48) == 8
    assert autotune.max_domain_side(64) == 32
    assert autotune.max_domain_side(128) == 64
    assert autotune.max_domain_side(96, (8, 16)) == 16
    with pytest.raises(ValueError):
        autotune.max_domain_side(24)
    plans = autotune.plan_candidates(152)
    assert plans[0][0] == 0 and (2, 152, 16) in plans and (1, 16, 16) in plans
    # 16x16 and 32x32 domains: thread plans in both domain orders, no CTA counts
    rows = [p for p in autotune.plan_candidates(152, 32) if p[0] == 3]
    assert (3, 1, 4) in rows and (3, 2, 4) in rows and all(p[1] in (1, 2) for p in rows)
    for name in ("run", "step", "capture", "sync", "close", "events_per_schedule"):
        assert callable(getattr(autotune.Batch, name, None)), name
    assert callable(getattr(autotune.BatchGraph, "replay", None))


def test_missing_library_fails_loudly(monkeypatch):
    """Without the built library the binding raises instead of falling back."""
    monkeypatch.setattr(_lib, "_LIB", None)
    monkeypatch.setattr(_lib, "lib_path", lambda: os.path.join(ROOT, "no_such_dir", "libkmc_gb300.so"))
    with pytest.raises(ImportError):
        _lib.load(build_if_missing=False)


def _has_cuda_device() -> bool:
    import torch
    return torch.cuda.device_count() > 0


@pytest.mark.skipif(_has_cuda_device(), reason="checks the error path of a machine without a CUDA device")
def test_no_cpu_fallback_without_a_device():
    """On a machine without a CUDA device every constructor of the C ABI
    returns KMC_ECUDA (not KMC_ENOMEM, and never a CPU context)."""
    lib = _lib.load()
    seeds = (ctypes.c_uint64 * 4)(1, 2, 3, 4)
    L = (ctypes.c_int32 * 1)(64)
    # a non-null, aligned placeholder: with no device nothing can use it
    placeholder = ctypes.c_void_p(4096)
    for L_d in (0, 16):
        ctx = ctypes.c_void_p()
        assert lib.kmc_create_lattice(ctypes.byref(ctx), 1, L, L_d, 1, 0, seeds, placeholder, None) == _lib.KMC_ECUDA
        assert ctx.value is not None and lib.kmc_last_error(ctx)
        lib.kmc_destroy(ctx)
    ring = ctypes.c_void_p()
    zeros = (ctypes.c_uint64 * 4)(0, 0, 0, 0)
    assert lib.kmc_ring_create(ctypes.byref(ring), 4, 8, 2, 5, seeds, zeros, None) == _lib.KMC_ECUDA
    assert ring.value is None
    part = ctypes.c_void_p()
    assert lib.kmc_part_create(ctypes.byref(part), 4, 12, 1, 2, 5, seeds, placeholder, None) == _lib.KMC_ECUDA
    assert part.value is None
    import paper_1403_4674_gb300 as kmc
    with pytest.raises(kmc.KmcError) as e:
        kmc.Ring(8, 2, 5, [1, 2], [0, 0])
    assert e.value.status == _lib.KMC_ECUDA


# Invalid arguments are refused on the host, before any CUDA call.  A
# placeholder device pointer is passed, so these run only on a machine
# without a CUDA device (the GPU suite checks the same refusals with real
# buffers).
_PLACE = 4096  # non-null, 8-byte aligned; never dereferenced here


@pytest.mark.skipif(_has_cuda_device(), reason="placeholder device pointers: machines without a CUDA device only")
@pytest.mark.parametrize("n_rep,Ls,L_d,k,init,spins,needle", [
    (1, [64], 12, 1, 0, _PLACE, "L_d must be"),
    (1, [64], 16, 0, 0, _PLACE, "k_steps"),
    (1, [64], 16, 65536, 0, _PLACE, "k_steps"),
    (1, [64], 16, 1, 7, _PLACE, "init"),
    (1, [64], 16, 1, 0, _PLACE + 4, "aligned"),
    (1, [64], 16, 1, 0, 0, "non-null"),
    (1, [48], 16, 1, 0, _PLACE, "multiple of 2*L_d"),
    (2, [64, 72], 8, 1, 0, _PLACE, "replica 1"),
    (1, [131072], 64, 1, 0, _PLACE, "multiple of 2*L_d"),
    (1, [65536], 8, 1, 0, _PLACE, "too many domains"),
])
def test_lattice_arguments_refused_on_the_host(n_rep, Ls, L_d, k, init, spins, needle):
    lib = _lib.load()
    ctx = ctypes.c_void_p()
    L = (ctypes.c_int32 * n_rep)(*Ls)
    seeds = (ctypes.c_uint64 * n_rep)(*range(1, n_rep + 1))
    st = lib.kmc_create_lattice(ctypes.byref(ctx), n_rep, L, L_d, k, init, seeds, ctypes.c_void_p(spins), None)
    assert st == _lib.KMC_EINVAL
    assert needle in lib.kmc_last_error(ctx).decode()
    lib.kmc_destroy(ctx)


@pytest.mark.skipif(_has_cuda_device(), reason="placeholder device pointers: machines without a CUDA device only")
def test_ring_and_partition_arguments_refused_on_the_host():
    lib = _lib.load()
    seeds = (ctypes.c_uint64 * 2)(1, 2)
    g = ctypes.c_void_p()
    for NS, Ld, k, init in ((65, 1, 5, 0), (8, 3, 5, 0), (8, 16, 5, 0), (8, 2, 65536, 0), (8, 2, 5, 1 << 8)):
        words = (ctypes.c_uint64 * 2)(init, 0)
        assert lib.kmc_ring_create(ctypes.byref(g), 2, NS, Ld, k, seeds, words, None) == _lib.KMC_EINVAL
        assert g.value is None
    for L, kind, ND, k in ((12, 2, 2, 5), (12, 0, 2, 5), (12, 1, 5, 5), (12, 1, 2, 65536), (12, 1, 65, 5)):
        assert lib.kmc_part_create(ctypes.byref(g), 2, L, kind, ND, k, seeds, ctypes.c_void_p(_PLACE), None) \
            == _lib.KMC_EINVAL
        assert g.value is None


@pytest.mark.skipif(_has_cuda_device(), reason="placeholder device pointers: machines without a CUDA device only")
@pytest.mark.parametrize("L_d", [8, 16, 32, 64])
def test_acceptance_rounding_to_zero_refused_on_the_host(L_d):
    """Eq. 4: an acceptance that rounds to A_c = 0 in the 2^-P fixed point
    would be a one-way rate; the library refuses the table before any CUDA
    call (the no-allocation entry point builds it first).  Just below the
    threshold the call gets past the table and fails later for want of a
    device."""
    import math
    lib = _lib.load()
    P = 63 - int(round(math.log2(L_d * L_d)))
    b0 = (P + 1) * math.log(2.0) / 8.0  # exp(-8 beta) = 2^-(P+1): the largest a that rounds to 0
    err = ctypes.create_string_buffer(256)
    args = lambda beta: (4 * L_d, L_d, 1, 7, 1.0, beta, 0.0, 1.0, 0, 0, 1, 0, 0, 0, ctypes.c_void_p(_PLACE), None,
                         None, err, len(err))
    assert lib.kmc_run_schedule_noalloc(*args(1.01 * b0)) == _lib.KMC_ENOTBALANCED
    assert b"rounds to 0" in err.value
    assert lib.kmc_run_schedule_noalloc(*args(0.99 * b0)) == _lib.KMC_ECUDA
