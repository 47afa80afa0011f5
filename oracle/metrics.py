"""The diversity of a set of solutions (paper Fig. 3 (c), (f)).

Test infrastructure only (see the package header).

Fig. 3 counts the solutions within approximation ratio a_r = 0.01 of the
best energy, every pair of which differs in more than N / 2 spins.  Readings
taken here:
* the printed ratio test E - E_best < a_r * 2 * E_best never holds for a
  negative E_best; it is read as E - E_best < 2 a_r |E_best| (strict);
* "each pair has a Hamming distance greater than N / 2" (strict, N spins, or
  N Potts variables for a Potts instance) is met by first fit: the solutions
  within the ratio are taken in ascending (energy, state, index) order and a
  solution is counted when it differs in more than N / 2 variables from
  every solution counted before it (the rule the droplets' Hamming cutoff
  follows); a largest such set is a maximum independent set, which the
  paper does not ask for.
"""
from __future__ import annotations

import numpy as np


def within_ratio(E: int, e_best: int, a_r: float) -> bool:
    """E - E_best < 2 a_r |E_best| (reading above)."""
    return float(E - e_best) < 2.0 * a_r * abs(float(e_best))


def diversity(solutions, energies, e_best: int, a_r: float = 0.01):
    """Count and indices of the solutions counted by Fig. 3's diversity.

    solutions: [n, N] arrays of the N variables of each solution (spins, or
    Potts states); energies: int64 [n]; e_best: the best energy considered.
    Returns (count, indices into solutions in counting order)."""
    X = np.asarray(solutions)
    E = np.asarray(energies, dtype=np.int64)
    n, N = X.shape if X.size else (0, 0)
    order = sorted(range(n), key=lambda k: (int(E[k]), tuple(int(v) for v in X[k]), k))
    chosen = []
    for k in order:
        if not within_ratio(int(E[k]), e_best, a_r):
            continue
        if all(2 * int(np.sum(X[k] != X[c])) > N for c in chosen):
            chosen.append(k)
    return len(chosen), chosen
