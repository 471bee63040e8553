"""Exact-enumeration pins of the method's theorems (arXiv:1403.4674, Sec. 2.2).

Eqs. 4-5: each domain step is reversible w.r.t. pi.  Eq. 9: T_SEQ(L) and
T_SEQ(reverse L) are adjoint under pi.  Eq. 10: a schedule mixture with
w(L) = w(reverse L) keeps detailed balance; the palindrome is its own reverse.
Negative pins: a fixed non-palindromic order keeps pi stationary but loses
detailed balance (Sec. 2.2, "as long as the corresponding reverse schedule is
included"); exactly-k-real-flips domain processes lose stationarity.
Special case: with the whole lattice as one domain the class-table step is the
textbook random-site kernel built from H(sigma') - H(sigma) (App. A).
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as orc
from oracle.enumerate import Enumerator

PAL = [0, 1, 2, 3, 3, 2, 1, 0]
FIXED = [0, 1, 2, 3]
CASES = [(2, 1), (4, 1), (4, 2)]


@pytest.fixture(scope="module", params=[(L, Ld, law, q) for (L, Ld) in CASES
                                        for law in (orc.RATE_METROPOLIS, orc.RATE_BARKER)
                                        for q in (False, True)])
def enum(request):
    L, Ld, law, q = request.param
    return Enumerator(L, Ld, 2, beta=0.45, h=0.15, law=law, quantised=q)


def test_palindrome_stationary_and_reversible(enum):
    op = lambda p: enum.schedule(PAL, p)
    assert enum.stationarity_error(op) < 1e-13
    assert enum.detailed_balance_error(op) < 1e-13


def test_each_domain_step_is_reversible(enum):
    for d in range(enum.Dx * enum.Dx):
        assert enum.detailed_balance_error(lambda p: enum.step(d, p), n_probe=2) < 1e-14


def test_fixed_order_stationary_but_not_reversible(enum):
    op = lambda p: enum.schedule(FIXED, p)
    assert enum.stationarity_error(op) < 1e-13
    assert enum.detailed_balance_error(op) > 1e-4


def test_same_colour_domains_commute():
    E = Enumerator(4, 1, 1, beta=0.5, h=0.2)
    rng = np.random.default_rng(3)
    p = rng.random(E.S)
    p /= p.sum()
    for c in range(4):
        ds = E.domains_of_colour(c)
        a = E.step(ds[1], E.step(ds[0], p))
        b = E.step(ds[0], E.step(ds[1], p))
        assert np.max(np.abs(a - b)) < 1e-16


def test_forward_and_reverse_schedule_are_adjoint():
    """Eq. 9 entrywise on a dense 2x2-lattice operator."""
    E = Enumerator(2, 1, 3, beta=0.7, h=0.25, law=orc.RATE_BARKER)
    fwd = E.dense(lambda p: E.schedule([0, 2, 1, 3], p))
    rev = E.dense(lambda p: E.schedule([3, 1, 2, 0], p))
    D = np.diag(E.pi)
    assert np.max(np.abs(fwd @ D - (rev @ D).T)) < 1e-15
    assert np.max(np.abs(fwd @ D - (fwd @ D).T)) > 1e-4


def test_uniform_colour_permutation_mixture_is_reversible():
    """Eq. 10 with w = 1/4! over colour orders (each order's reverse included)."""
    E = Enumerator(4, 2, 1, beta=0.45, h=0.15)
    perms = list(itertools.permutations(range(4)))

    def mix(p):
        return sum(E.schedule(list(pp), p) for pp in perms) / len(perms)

    assert E.stationarity_error(mix) < 1e-13
    assert E.detailed_balance_error(mix, n_probe=2) < 1e-13


def test_k_real_flips_reading_breaks_stationarity():
    E = Enumerator(4, 2, 2, beta=0.45, h=0.15)

    def op(p):
        for c in PAL:
            for d in E.domains_of_colour(c):
                for _ in range(E.k):
                    p = E.real_flip_step(d, p)
        return p

    assert E.stationarity_error(op) > 1e-2


@pytest.mark.parametrize("law", [orc.RATE_METROPOLIS, orc.RATE_BARKER])
@pytest.mark.parametrize("h", [0.0, 0.3, -0.2])
def test_whole_lattice_step_is_textbook_kernel(law, h):
    E = Enumerator(4, 2, 1, beta=0.6, h=h, law=law, quantised=False)
    rng = np.random.default_rng(5)
    p = rng.random(E.S)
    p /= p.sum()
    assert np.max(np.abs(E.whole_lattice_step(p) - E.reference_step(p, law))) < 1e-18


def test_quantised_table_close_to_exact():
    Eq = Enumerator(4, 2, 2, beta=0.45, h=0.15, quantised=True)
    Ee = Enumerator(4, 2, 2, beta=0.45, h=0.15, quantised=False)
    p = np.zeros(Eq.S)
    p[0] = 1.0
    a = Eq.schedule(PAL, p)
    b = Ee.schedule(PAL, p)
    assert np.max(np.abs(a - b)) < 1e-15
