"""The inpainting-shaped Potts instance (Sec. 3 example, Fig. 5 shape: data
on a circular boundary, the inside free) has the stated tables, and the
oracle solves a brute-forceable case exactly."""
import numpy as np
import pytest

import instances as I
from oracle import exact, lattice, search, tables


@pytest.mark.parametrize("L,d,seed", [(8, 3, 1), (12, 4, 2), (6, 2, 3)])
def test_inpainting_tables(L, d, seed):
    t = I.inpainting(L, d, seed)
    unit = 2 ** t.energy_shift
    loc = t.local_E.reshape(L * L, d)
    data = loc.max(axis=1) > 0
    # data pixels: one label at 0, the others at the data cost; inside: no data
    assert np.all(np.sort(loc[data], axis=1)[:, 0] == 0)
    assert np.all(np.sort(loc[data], axis=1)[:, 1:] == int(round(4.0 * unit)))
    assert np.all(loc[~data] == 0) and 0 < (~data).sum() < L * L
    assert len({int(np.argmin(r)) for r in loc[data]}) == d  # every label observed
    # Potts smoothness on all 8-neighbour edges
    pair = t.pair_E.reshape(len(t.em), d, d)
    for m, n, P in zip(t.em, t.en, pair):
        (a, b), (c, e) = divmod(int(m), L), divmod(int(n), L)
        assert max(abs(a - c), abs(b - e)) == 1
        w = unit if (a == c or b == e) else int(round(unit / np.sqrt(2.0)))
        assert np.array_equal(P, w * (1 - np.eye(d, dtype=np.int64)))
    assert len(t.em) == 4 * L * L - 6 * L + 2  # every king's-graph edge once


def test_inpainting_exact_ground_state():
    """4 x 4, 2 labels, ring 0.5 (an interior of 4 free pixels): the oracle's
    search in its exact limit reaches the brute-force ground energy."""
    t = I.inpainting(4, 2, 5, ring=0.5)
    E, _ = exact.potts_all_energies(t)
    loc = t.local_E.reshape(16, 2)
    assert (loc.max(axis=1) == 0).sum() == 4
    res = search.solve(tables.from_potts(t), search.Params(beta=1.0, chi=64, beam=256))
    assert int(res.energies[0]) == int(E.min())


def test_inpainting_lattice_transforms_keep_energies():
    t = I.inpainting(6, 3, 4)
    fg = tables.from_potts(t)
    rng = np.random.default_rng(0)
    xs = [rng.integers(0, 3, size=36) for _ in range(10)]
    for k in range(8):
        fgk = tables.from_potts(lattice.transform(t, k))
        m = lattice.site_map(6, 6, k)
        for x in xs:
            xk = np.empty_like(x)
            xk[m] = x
            assert tables.energy(fgk, xk) == tables.energy(fg, x)
