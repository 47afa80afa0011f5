"""Droplets (low-energy excitations collected in the merges; Sec. 2 and
Sec. 3.1 SingleLayerDroplets, energy and Hamming cutoffs, unpack_droplets)
on the GPU against the oracle's: the best state's droplets, their exact
energies and states, in the same (energy, state) order.  Cases are chosen so
that no list fills up (checked: droplet_overflow == 0); every droplet's
energy is also recomputed from the tables, lies within the cutoff, and the
Hamming separations hold.  Collecting droplets leaves the search unchanged."""
import numpy as np
import pytest

import instances as I
from oracle import search, tables

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spg():
    import paper_2502_02317_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(spg):
    return spg.Context(0)


def fg_of(inst):
    return tables.from_potts(inst) if hasattr(inst, "local_E") else tables.from_ising(inst)


def problem(spg, ctx, inst):
    return spg.spg_problem_potts(ctx, inst) if hasattr(inst, "local_E") else spg.spg_problem_ising(ctx, inst)


CASES = [
    (lambda: I.square(1, 4, cols=7, h_sigma=0.3), 16, 8, 4.0, 0),      # chains: the low-energy spectrum
    (lambda: I.square(1, 4, cols=7, h_sigma=0.3), 16, 8, 4.0, 1),
    (lambda: I.king_potts(1, 3, 9, cols=5), 16, 8, 1.5, 0),
    (lambda: I.chimera(2, 8, couplings="gauss", h_sigma=0.1), 16, 64, 2.0, 0),
    (lambda: I.chimera(2, 8, couplings="gauss", h_sigma=0.1), 16, 64, 2.0, 1),
    (lambda: I.king_potts(3, 3, 5), 16, 32, 1.0, 0),
    (lambda: I.king_potts(3, 3, 5), 16, 32, 2.0, 1),
    (lambda: I.king_ising(3, 3, 2, 6), 16, 32, 1.0, 0),
    (lambda: I.king_ising(3, 3, 2, 6), 16, 32, 2.0, 1),
    (lambda: I.square(4, 3, h_sigma=0.2), 8, 16, 1.0, 0),
    (lambda: I.square(4, 3, h_sigma=0.2), 8, 16, 1.0, 1),
]


@pytest.mark.parametrize("make,chi,beam,cut,ham", CASES)
def test_droplets_match_oracle(spg, ctx, make, chi, beam, cut, ham):
    inst = make()
    fg = fg_of(inst)
    cut_units = int(cut * 2 ** inst.energy_shift)
    ref = search.solve(fg, search.Params(beta=1.0, chi=chi, beam=beam, droplet_energy=cut_units,
                                         droplet_hamming=ham))
    prob = problem(spg, ctx, inst)
    res = spg.spg_solve(ctx, prob, spg.params(beta=1.0, chi=chi, beam=beam, droplet_energy=cut,
                                              droplet_hamming=ham))
    st, E, lp = res.get()
    info = res.info()
    assert info["error_flags"] == 0 and info["droplet_overflow"] == 0
    dE, dst = res.droplets()
    # the droplets' own properties
    for k in range(len(dE)):
        assert tables.energy(fg, dst[k]) == dE[k]
        assert 0 <= dE[k] - E[0] <= cut_units
        others = [st[0]] + [dst[q] for q in range(len(dE)) if q != k]
        assert all(np.sum(dst[k] != a) > ham for a in others)  # pairwise separation
    # the oracle's list, element by element
    if ref.near_ties == 0 and info["near_ties"] == 0:
        assert int(E[0]) == int(ref.energies[0])
        assert len(dE) == len(ref.droplets)
        for k, (eo, so) in enumerate(ref.droplets):
            assert int(dE[k]) == int(eo)
            np.testing.assert_array_equal(dst[k].astype(np.int64), np.asarray(so, np.int64))
    # the search itself is unchanged by the collection
    st0, E0, lp0 = spg.spg_solve(ctx, prob, spg.params(beta=1.0, chi=chi, beam=beam)).get()
    np.testing.assert_array_equal(st0, st)
    np.testing.assert_array_equal(E0, E)
    np.testing.assert_array_equal(lp0, lp)
