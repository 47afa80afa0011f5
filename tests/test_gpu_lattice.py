"""The 8 lattice transformations solved as one batch on the GPU (Sec. 3.1)
against the oracle's best of 8 (oracle/lattice.py): the chosen lattice, every
lattice's best energy, and the returned states on the original sites with
their energies, bit-exact (FP64 mode, cases without near ties)."""
import numpy as np
import pytest

import instances as I
from oracle import lattice, search, tables

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spg():
    import paper_2502_02317_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(spg):
    return spg.Context(0)


@pytest.mark.parametrize("make,beta,chi,beam", [
    (lambda: I.chimera(3, 4, cols=2), 1.0, 16, 16),                        # 3 x 2: transposes change the shape
    (lambda: I.square(4, 6, cols=5, h_sigma=0.3), 1.0, 4, 8),
    (lambda: I.king_potts(3, 3, 12, cols=4), 1.0, 8, 16),                  # Potts: sites move with tables
    (lambda: I.king_ising(3, 4, 2, 13), 1.5, 8, 32),
])
def test_best_of_8_matches_oracle(spg, ctx, make, beta, chi, beam):
    inst = make()
    prm_o = search.Params(beta=beta, chi=chi, beam=beam)
    ref = lattice.solve_best_of_8(inst, prm_o)
    prob = (spg.spg_problem_potts(ctx, inst) if hasattr(inst, "local_E") else spg.spg_problem_ising(ctx, inst))
    res, k, per = spg.spg_solve_lattice8(ctx, prob, spg.params(beta=beta, chi=chi, beam=beam))
    st, E, lp = res.get()
    np.testing.assert_array_equal(per, ref.best_per_lattice)
    assert k == ref.k
    fg = lattice.factor_graph(inst)
    for q in range(len(E)):
        assert tables.energy(fg, st[q]) == E[q]  # on the original sites
    near = search.solve(lattice.factor_graph(lattice.transform(inst, k)), prm_o).near_ties
    if near == 0 and res.info()["near_ties"] == 0:
        np.testing.assert_array_equal(E, ref.energies)
        np.testing.assert_array_equal(st.astype(np.int64), ref.states)
        np.testing.assert_allclose(lp, ref.log_probs, rtol=1e-6, atol=1e-6)
