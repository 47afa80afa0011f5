"""New couplings written into an existing Ising problem
(spg_problem_update_ising): solves of the updated problem, captured graphs
replayed, equal solves of a problem built from scratch with the same
couplings, and the oracle's result."""
import numpy as np
import pytest

import instances as I
from oracle import search, tables

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spg():
    import paper_2502_02317_gb300 as m
    return m


def test_update_in_place_replays_the_captured_solve(spg):
    ctx = spg.Context(0)
    prm = spg.params(beta=1.0, chi=16, beam=128, precision=spg.SPG_MIXED, num_sweeps=1)
    a = I.chimera(4, 71, couplings="gauss", h_sigma=0.1)
    prob = spg.spg_problem_ising(ctx, a)
    for _ in range(3):  # uncaptured, captured, replayed
        spg.spg_solve(ctx, prob, prm).get()
    for seed in (72, 73):
        b = I.chimera(4, seed, couplings="gauss", h_sigma=0.1)
        spg.spg_problem_update_ising(prob, b.J, b.h)
        st, E, lp = spg.spg_solve(ctx, prob, prm).get()
        fresh = spg.spg_problem_ising(ctx, b)
        st2, E2, lp2 = spg.spg_solve(ctx, fresh, prm).get()
        np.testing.assert_array_equal(st, st2)
        np.testing.assert_array_equal(E, E2)
        np.testing.assert_array_equal(lp, lp2)
        ref = search.solve(tables.from_ising(b), search.Params(beta=1.0, chi=16, beam=128, num_sweeps=1))
        assert E[0] == ref.energies[0]


def test_update_that_changes_the_structure_is_refused(spg):
    ctx = spg.Context(0)
    a = I.chimera(3, 5)
    prob = spg.spg_problem_ising(ctx, a)
    J = np.array(a.J, copy=True)
    J[:] = 0.0  # every table row equal: the projections collapse
    with pytest.raises(spg.SpgError) as e:
        spg.spg_problem_update_ising(prob, J, a.h)
    assert e.value.code == spg.SPG_EUNSUPPORTED
    # the problem is unchanged
    st, E, _ = spg.spg_solve(ctx, prob, spg.params(beta=1.0, chi=16, beam=64)).get()
    ref = search.solve(tables.from_ising(a), search.Params(beta=1.0, chi=16, beam=64))
    assert E[0] == ref.energies[0]
