"""Pins of the oracle's droplets (Sec. 2 and Sec. 3.1: low-energy excitations
collected in the merge, energy cutoff, Hamming cutoff, ``unpack_droplets``)
against brute-force enumeration of Eq. 1 / Eq. 2 and against properties that
hold whatever the search keeps."""
import numpy as np
import pytest

import instances as I
from oracle import exact, search, tables

BIG = 2 ** 62


def fg_of(inst):
    return tables.from_potts(inst) if hasattr(inst, "local_E") else tables.from_ising(inst)


def spectrum(inst, fg):
    """(E, cluster states) of every configuration, by brute force."""
    if hasattr(inst, "local_E"):
        E, cs = exact.potts_all_energies(inst)
    else:
        E = exact.all_energies(inst)
        cs = exact.cluster_states(inst.n_spins, fg.spins_of_site)
    states = np.stack([np.asarray(c) for c in cs], axis=1)
    return np.asarray(E, np.int64), states


@pytest.mark.parametrize("make,prm", [
    (lambda: I.chimera(2, 8, couplings="gauss", h_sigma=0.1), dict(chi=16, beam=64)),
    (lambda: I.king_potts(3, 3, 5), dict(chi=16, beam=32)),
])
def test_droplets_do_not_change_the_search(make, prm):
    inst = make()
    fg = fg_of(inst)
    a = search.solve(fg, search.Params(beta=1.0, **prm))
    b = search.solve(fg, search.Params(beta=1.0, droplet_energy=BIG, droplet_hamming=1, **prm))
    assert np.array_equal(a.states, b.states) and np.array_equal(a.energies, b.energies)
    assert np.array_equal(a.log_probs, b.log_probs) and a.droplets == []


@pytest.mark.parametrize("make,cut", [
    (lambda: I.square(1, 4, cols=7, h_sigma=0.3), None),
    (lambda: I.square(1, 5, cols=7, h_sigma=0.3), 4.0),
    (lambda: I.king_potts(1, 3, 9, cols=5), None),
    (lambda: I.king_potts(1, 3, 9, cols=5), 1.0),
])
def test_chain_droplets_are_the_low_energy_spectrum(make, cut):
    """On a 1 x L chain the merge key is the newest site alone and the last
    step merges everything, so the best state's droplets are every other
    configuration within the cutoff (Hamming cutoff 0), by brute force."""
    inst = make()
    fg = fg_of(inst)
    E, st = spectrum(inst, fg)
    if cut is not None:
        cut = int(cut * 2 ** inst.energy_shift)  # energy units -> table units
    prm = search.Params(beta=1.0, chi=16, beam=8, droplet_energy=BIG if cut is None else cut)
    res = search.solve(fg, prm)
    E0 = int(res.energies[0])
    assert E0 == int(E.min())
    want = sorted((int(e), tuple(int(v) for v in s)) for e, s in zip(E, st)
                  if tuple(int(v) for v in s) != tuple(int(v) for v in res.states[0])
                  and (cut is None or e - E0 <= cut))
    got = sorted((int(e), tuple(int(v) for v in s)) for e, s in res.droplets)
    assert got == want
    assert len(got) > 0


@pytest.mark.parametrize("make,prm", [
    (lambda: I.chimera(2, 8, couplings="gauss", h_sigma=0.1, cols=3), dict(chi=16, beam=64)),
    (lambda: I.king_potts(3, 3, 5), dict(chi=16, beam=32)),
    (lambda: I.king_ising(3, 3, 2, 4), dict(chi=16, beam=64)),
])
@pytest.mark.parametrize("ham", [0, 2])
def test_droplet_invariants(make, prm, ham):
    """Every droplet is a configuration whose energy (Eq. 1 from the tables;
    Eq. 2 on the spins for Ising instances) is the best energy plus at most
    the cutoff, and the best state and its droplets differ pairwise in more
    than the Hamming cutoff."""
    inst = make()
    fg = fg_of(inst)
    E, _ = spectrum(inst, fg) if fg.n_sites * np.log2(max(fg.d)) <= 20 else (None, None)
    cut = 3 * 2 ** inst.energy_shift
    res = search.solve(fg, search.Params(beta=1.0, droplet_energy=cut, droplet_hamming=ham, **prm))
    E0 = int(res.energies[0])
    assert len(res.droplets) > 0
    seen = [tuple(int(v) for v in res.states[0])]
    for e, s in res.droplets:
        assert tables.energy(fg, s) == e and 0 <= e - E0 <= cut
        if not hasattr(inst, "local_E"):
            assert tables.ising_energy(inst, tables.spins_from_states(fg, s, inst.n_spins)) == e
        if E is not None:
            assert e in set(E.tolist())
        for a in seen:
            assert sum(1 for u, v in zip(a, s) if u != v) > ham
        seen.append(tuple(s))


def test_droplet_energy_cutoff_is_a_filter():
    """Hamming cutoff 0: the droplets at a lower energy cutoff are exactly
    those at a higher one with dE within the lower (the search itself does not
    depend on the droplets)."""
    inst = I.king_potts(3, 3, 5)
    fg = fg_of(inst)
    lo, hi = 2 ** 24, 3 * 2 ** 24
    a = search.solve(fg, search.Params(beta=1.0, chi=16, beam=32, droplet_energy=lo))
    b = search.solve(fg, search.Params(beta=1.0, chi=16, beam=32, droplet_energy=hi))
    E0 = int(b.energies[0])
    assert sorted(a.droplets) == sorted(d for d in b.droplets if d[0] - E0 <= lo)
    assert len(b.droplets) > len(a.droplets) > 0
