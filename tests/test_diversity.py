"""The library's diversity of solutions (spg_diversity, host only; Fig. 3
(c), (f)) against the oracle's, index for index, on the CPU: random sets of
spin and Potts solutions with tied energies, whole brute-force spectra, and
the refusal of bad arguments."""
import numpy as np
import pytest

import instances as I
from oracle import exact, metrics


@pytest.mark.parametrize("seed", range(6))
def test_random_sets_match_the_oracle(seed):
    import paper_2502_02317_gb300 as spg
    rng = np.random.default_rng(seed)
    n, N = int(rng.integers(1, 60)), int(rng.integers(1, 12))
    X = rng.choice([-1, 1], size=(n, N)) if seed % 2 == 0 else rng.integers(0, 4, size=(n, N))
    E = rng.integers(-60, -40, size=n).astype(np.int64)  # many ties
    e_best = int(E.min()) - int(rng.integers(0, 3))
    for a_r in (0.0, 0.01, 0.05, 0.3):
        assert spg.spg_diversity(X, E, e_best, a_r) == metrics.diversity(X, E, e_best, a_r)


@pytest.mark.parametrize("make", [lambda: I.chimera(2, 3, cols=1), lambda: I.square(4, 6)])
def test_whole_spectra_match_the_oracle(make):
    import paper_2502_02317_gb300 as spg
    inst = make()
    E = exact.all_energies(inst)
    n = inst.n_spins
    X = 2 * ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1) - 1
    keep = np.nonzero(E - E.min() <= 8)[0]
    for a_r in (0.05, 0.2):
        got = spg.spg_diversity(X[keep], E[keep], int(E.min()), a_r)
        assert got == metrics.diversity(X[keep], E[keep], int(E.min()), a_r) and got[0] >= 1


def test_bad_arguments():
    import ctypes

    import paper_2502_02317_gb300 as spg
    cnt = ctypes.c_int32()
    assert spg.lib.spg_diversity(0, 4, None, None, -5, 0.01, ctypes.byref(cnt), None) == 0 and cnt.value == 0
    for args in ((-1, 4, 0.01), (3, 0, 0.01), (0, 4, -0.1)):
        assert spg.lib.spg_diversity(args[0], args[1], None, None, 0, args[2], ctypes.byref(cnt), None) == -1
    assert spg.lib.spg_diversity(2, 4, None, None, 0, 0.01, ctypes.byref(cnt), None) == -1
