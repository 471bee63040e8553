"""Pin the oracle's rate table (App. A, Eq. Glauber_TM; Metropolis) to closed forms."""
import math

import numpy as np
import pytest

from oracle import oracle as orc

CLASSES = [(sp, q) for sp in (0, 1) for q in range(5)]


def test_class_energy_change_hand_values():
    # sigma=+1 with all four neighbours up: flipping costs 2*(4J + h)
    assert orc.class_dE(9, 1.0, 0.0) == 8.0
    assert orc.class_dE(9, 1.0, 0.25) == 8.5
    # sigma=-1 with all four neighbours up: flipping gains 2*(4J - h)... dE = -2(4J + h)
    assert orc.class_dE(4, 1.0, 0.25) == -8.5
    # sigma=+1, two up neighbours (neighbour sum 0): dE = 2h
    assert orc.class_dE(7, 1.0, 0.1) == pytest.approx(0.2, abs=0)
    assert orc.class_dE(2, 1.0, 0.1) == pytest.approx(-0.2, abs=0)


@pytest.mark.parametrize("law", [orc.RATE_METROPOLIS, orc.RATE_BARKER])
@pytest.mark.parametrize("beta,h", [(0.4, 0.0), (1 / 2.269, 0.01), (1 / 1.5, -0.1), (2.0, 0.3)])
def test_rate_ratio_is_boltzmann(law, beta, h):
    a, A = orc.rate_table(1.0, beta, h, law, 10)
    for c, (sp, q) in enumerate(CLASSES):
        cbar = 5 * (1 - sp) + q  # the same site after its flip
        dE = orc.class_dE(c, 1.0, h)
        assert orc.class_dE(cbar, 1.0, h) == -dE
        assert 0.0 < a[c] <= 1.0
        assert a[c] / a[cbar] == pytest.approx(math.exp(-beta * dE), rel=4e-16)
        if law == orc.RATE_BARKER:
            assert a[c] + a[cbar] == pytest.approx(1.0, rel=1e-15)
        else:
            assert max(a[c], a[cbar]) == 1.0


def test_hand_table_metropolis_beta04():
    a, _ = orc.rate_table(1.0, 0.4, 0.0, orc.RATE_METROPOLIS, 8)
    # down spin (sp=0): q up neighbours, dE = -2(2q-4) = 8 - 4q
    assert a[0] == pytest.approx(math.exp(-0.4 * 8), rel=1e-15)
    assert a[1] == pytest.approx(math.exp(-0.4 * 4), rel=1e-15)
    assert list(a[2:5]) == [1.0, 1.0, 1.0]
    # up spin (sp=1): dE = 2(2q-4) = 4q - 8
    assert list(a[5:8]) == [1.0, 1.0, 1.0]
    assert a[8] == pytest.approx(math.exp(-0.4 * 4), rel=1e-15)
    assert a[9] == pytest.approx(math.exp(-0.4 * 8), rel=1e-15)


@pytest.mark.parametrize("log2nd", [0, 2, 6, 8, 10, 12])
def test_fixed_point_rounding(log2nd):
    a, A = orc.rate_table(1.0, 1 / 2.269, 0.01, orc.RATE_METROPOLIS, log2nd)
    P = 63 - log2nd
    for c in range(10):
        exact = a[c] * 2.0 ** P
        assert abs(int(A[c]) - exact) <= 0.5
    # an all-rate-one domain must not overflow: n_d * 2^P = 2^63
    assert (1 << log2nd) * (1 << P) == 1 << 63


def test_invalid_arguments_rejected():
    with pytest.raises(ValueError):
        orc.rate_table(1.0, -1.0, 0.0, 0, 8)
    with pytest.raises(ValueError):
        orc.rate_table(1.0, 0.4, 0.0, 7, 8)
    with pytest.raises(ValueError):
        orc.rate_table(1.0, 0.4, 0.0, 0, 17)  # n_d <= 2^16 (100^2 stripes need 2^13)


def _beta_at_zero_threshold(P: int, dE: float) -> float:
    """beta at which exp(-beta dE) = 2^-(P+1), the largest acceptance that rounds to A_c = 0."""
    return (P + 1) * math.log(2.0) / dE


@pytest.mark.parametrize("law", [orc.RATE_METROPOLIS, orc.RATE_BARKER])
@pytest.mark.parametrize("log2nd", [6, 8, 10, 12])
def test_acceptance_rounding_to_zero_is_refused(law, log2nd):
    """Eq. 4: a_c > 0 for every class, so a table whose fixed point rounds
    some a_c to 0 would make the flip out of class cbar one-way.  Just below
    the threshold every A_c is at least 1; just above it the table is refused.
    (The largest class energy change at J = 1, h = 0 is 8.)"""
    P = 63 - log2nd
    b0 = _beta_at_zero_threshold(P, 8.0)
    a, A = orc.rate_table(1.0, 0.99 * b0, 0.0, law, log2nd)
    assert int(A.min()) >= 1
    with pytest.raises(ValueError, match="rounds to 0"):
        orc.rate_table(1.0, 1.01 * b0, 0.0, law, log2nd)


@pytest.mark.parametrize("log2ld", [0, 2, 5])
def test_ring_acceptance_rounding_to_zero_is_refused(log2ld):
    """The ring's classes: largest energy change 4 at J = 1, h = 0."""
    P = 63 - log2ld
    b0 = _beta_at_zero_threshold(P, 4.0)
    _, A = orc.ring_rate_table(1.0, 0.99 * b0, 0.0, orc.RATE_METROPOLIS, log2ld)
    assert int(A.min()) >= 1
    with pytest.raises(ValueError):
        orc.ring_rate_table(1.0, 1.01 * b0, 0.0, orc.RATE_METROPOLIS, log2ld)


@pytest.mark.parametrize("log2nd", [6, 10, 12])
def test_rounding_error_bound(log2nd):
    """|A_c 2^-P - a_c| <= 2^-(P+1) for every class, so the relative change
    is at most 2^-(P+1)/a_c; at the benchmark temperatures (T >= 1.5, |h| <=
    0.1) it stays below 1e-12."""
    P = 63 - log2nd
    for T, h in [(1.5, 0.1), (1.5, -0.1), (2.269, 0.01), (3.5, 0.0)]:
        a, A = orc.rate_table(1.0, 1 / T, h, orc.RATE_METROPOLIS, log2nd)
        err = np.abs(A.astype(np.float64) * 2.0 ** -P - a)
        assert np.all(err <= 2.0 ** -(P + 1))
        assert np.max(err / a) < 1e-12
