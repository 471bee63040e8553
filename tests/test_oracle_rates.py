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
