"""Pins of the oracle's 8-lattice best-of-8 search (Sec. 3.1, lattice
transformations) against facts that do not depend on it: Eq. 1 / Eq. 2
energies evaluated directly, brute-force ground states, and the search's
exact limit."""
import numpy as np
import pytest

import instances as I
from oracle import exact, lattice, search, tables


@pytest.mark.parametrize("rows,cols", [(3, 3), (3, 4), (2, 5), (1, 4)])
def test_site_maps_are_the_eight_symmetries(rows, cols):
    maps = set()
    for k in range(8):
        m = lattice.site_map(rows, cols, k)
        assert sorted(m.tolist()) == list(range(rows * cols))  # a permutation
        _, _, R, C = lattice.position(0, 0, rows, cols, k)
        maps.add((R, C, tuple(m.tolist())))
        # grid neighbours stay grid neighbours (king's moves included)
        for s in range(rows * cols):
            for t in range(rows * cols):
                a, b = divmod(s, cols)
                c, e = divmod(t, cols)
                near = max(abs(a - c), abs(b - e)) == 1
                a2, b2 = divmod(int(m[s]), C)
                c2, e2 = divmod(int(m[t]), C)
                assert near == (max(abs(a2 - c2), abs(b2 - e2)) == 1)
    assert lattice.site_map(rows, cols, 0).tolist() == list(range(rows * cols))
    assert len(maps) == (8 if min(rows, cols) > 1 else 4)


@pytest.mark.parametrize("make", [
    lambda: I.chimera(2, 5, couplings="gauss", h_sigma=0.1, cols=3),
    lambda: I.square(3, 7, h_sigma=0.3),
    lambda: I.king_potts(3, 3, 12, cols=4),
    lambda: I.king_ising(2, 3, 2, 6),
])
def test_transformed_lattices_keep_every_energy(make):
    """Eq. 1 of a state on the original lattice == Eq. 1 of the same cluster
    states placed on the transformed lattice, for random states."""
    inst = make()
    fg = lattice.factor_graph(inst)
    rng = np.random.default_rng(3)
    xs = [np.array([rng.integers(0, d) for d in fg.d]) for _ in range(20)]
    for k in range(8):
        fgk = lattice.factor_graph(lattice.transform(inst, k))
        m = lattice.site_map(inst.grid_rows, inst.grid_cols, k)
        for x in xs:
            xk = np.empty_like(x)
            xk[m] = x
            assert tables.energy(fgk, xk) == tables.energy(fg, x)


def test_best_of_8_equal_best_energy_in_the_exact_limit():
    """beam >= keys x d makes every lattice's search exact: all 8 best
    energies equal the brute-force ground energy, and the returned states
    have it on the original instance (Eq. 2 on the decoded spins)."""
    for seed in range(2):
        inst = I.square(4, 30 + seed, h_sigma=0.3)
        gs = exact.brute_force(inst, 1.0)["ground"]
        best = lattice.solve_best_of_8(inst, search.Params(beta=1.0, chi=8, beam=32))
        assert best.best_per_lattice.tolist() == [gs] * 8
        assert best.k == 0
        fg = tables.from_ising(inst)
        for e, s in zip(best.energies, best.states):
            assert e == tables.ising_energy(inst, tables.spins_from_states(fg, s, inst.n_spins))


def test_best_of_8_king_potts_exact_limit():
    inst = I.king_potts(3, 2, 14, cols=4)
    gs = int(exact.potts_all_energies(inst)[0].min())
    best = lattice.solve_best_of_8(inst, search.Params(beta=1.0, chi=64, beam=128))
    assert best.best_per_lattice.tolist() == [gs] * 8
    fg = tables.from_potts(inst)
    assert tables.energy(fg, best.states[0]) == gs


@pytest.mark.parametrize("make,k_best", [
    (lambda: I.chimera(3, 1, couplings="gauss", h_sigma=0.1), 5),   # tie with k = 7
    (lambda: I.king_potts(3, 4, 0, cols=4), 2),                      # ties with k = 5, 7
])
def test_best_of_8_is_the_first_minimum_and_maps_back(make, k_best):
    """Heuristic regime (beam 2, chi 2): the lattices reach different best
    energies; the result is the first lattice with the lowest one, and every
    lattice's states, mapped back to the original sites, carry their
    reported energies there (Eq. 1 on the original tables)."""
    inst = make()
    prm = search.Params(beta=1.0, chi=2, beam=2, merge=False)
    best = lattice.solve_best_of_8(inst, prm)
    E = best.best_per_lattice
    assert len(set(E.tolist())) > 1
    assert best.k == int(np.argmin(E)) == k_best and best.energies[0] == E.min()
    fg = lattice.factor_graph(inst)
    for k in range(8):
        res = search.solve(lattice.factor_graph(lattice.transform(inst, k)), prm)
        for e, s in zip(res.energies, best.states_per_lattice[k]):
            assert e == tables.energy(fg, s)
    assert np.array_equal(best.states, best.states_per_lattice[best.k])
