"""Pins of the oracle's diversity of solutions (Fig. 3 (c), (f): solutions
within approximation ratio a_r of the best energy, pairwise more than N / 2
variables apart; readings in oracle/metrics.py): a hand-computed example,
the strict bounds, and the properties that define first fit on brute-force
spectra."""
import numpy as np
import pytest

import instances as I
from oracle import exact, metrics


def test_hand_computed_example():
    # N = 6 spins, E_best = -1000, a_r = 0.01: within the ratio when E < -980.
    # (A state and its global flip are N apart, so once both are counted no
    # third solution can be more than N/2 from both: the example avoids it.)
    X = np.array([[1, 1, 1, 1, 1, 1],        # 0 A: E -1000
                  [1, 1, -1, -1, -1, -1],    # 1 B: 4 from A
                  [-1, -1, 1, 1, -1, -1],    # 2 C: 4 from A and from B
                  [-1, -1, -1, -1, 1, 1],    # 3 D: 4 from A, B and C
                  [-1, -1, -1, -1, -1, 1],   # 4 F: 5 from A, 3 from B, C and 1 from D
                  [-1, 1, -1, 1, -1, 1]])    # 5 G: at the ratio's edge
    E = np.array([-1000, -995, -990, -981, -999, -980])
    # F (E -999) comes second and blocks B, C and D (3 is not more than N/2)
    assert metrics.diversity(X, E, -1000, 0.01) == (2, [0, 4])
    E[4] = -970  # F outside the ratio
    assert metrics.diversity(X, E, -1000, 0.01) == (4, [0, 1, 2, 3])
    E[3] = -980  # the ratio is strict
    assert metrics.diversity(X, E, -1000, 0.01) == (3, [0, 1, 2])
    E[1] = -1000  # equal energies: the lexicographically smaller state first
    assert metrics.diversity(X, E, -1000, 0.01) == (3, [1, 0, 2])


def test_ratio_reading_for_positive_and_negative_best():
    assert metrics.within_ratio(-99, -100, 0.01) and not metrics.within_ratio(-98, -100, 0.01)
    assert metrics.within_ratio(101, 100, 0.01) and not metrics.within_ratio(102, 100, 0.01)
    assert metrics.within_ratio(0, 0, 0.01) is False


@pytest.mark.parametrize("make,a_r", [(lambda: I.chimera(2, 3, cols=1), 0.1),
                                      (lambda: I.square(4, 6), 0.2)])
def test_first_fit_properties_on_the_whole_spectrum(make, a_r):
    inst = make()
    E = exact.all_energies(inst)
    n = inst.n_spins
    X = 2 * ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1) - 1
    e_best = int(E.min())
    keep = np.nonzero(E - e_best < 2 * a_r * abs(e_best))[0]
    count, chosen = metrics.diversity(X[keep], E[keep], e_best, a_r)
    assert count == len(chosen) >= 1
    C = X[keep][chosen]
    for a in range(count):
        for b in range(a + 1, count):
            assert 2 * np.sum(C[a] != C[b]) > n
    # maximal in the counting order: every solution left out is within N/2 of
    # a counted one that comes before it
    order = sorted(range(len(keep)), key=lambda k: (int(E[keep][k]), tuple(X[keep][k])))
    pos = {k: i for i, k in enumerate(order)}
    for k in set(range(len(keep))) - set(chosen):
        assert any(2 * np.sum(X[keep][k] != X[keep][c]) <= n and pos[c] < pos[k] for c in chosen)
    # h = 0: the first counted solution's global flip (N spins away, same
    # energy) is counted, or something counted before it is more than N/2
    # from the first one: at least two either way
    if not np.any(inst.h):
        g = chosen[0]
        assert any(np.array_equal(X[keep][k], -X[keep][g]) for k in range(len(keep)))
        assert count >= 2
