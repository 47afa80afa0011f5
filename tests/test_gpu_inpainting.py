"""Generic Potts models on 8-neighbour grids shaped like the paper's
inpainting example (Sec. 3.2; synthetic: labels observed on a circular band
in d arcs, free interior, Potts smoothness on every king's-graph edge),
through the C ABI against the oracle:

* brute-forceable grids (3 x 3 with 3 labels, 4 x 4 with 2): the FP64 search equals the
  oracle's, and with a beam that makes the merged search an exact dynamic
  programme, its best energy is the brute-force ground energy;
* grids wider than the former 32-column limit (2 x 40, 3 x 64): the FP64
  search equals the oracle's state for state;
* a 120 x 120 grid with 4 labels (the size of the paper's example): every
  returned state's energy recomputed on the host, in both modes.
"""
import numpy as np
import pytest

import instances as I
from oracle import exact, search, tables

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spg():
    import paper_2502_02317_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(spg):
    return spg.Context(0)


def compare(spg, ctx, inst, beta, chi, beam):
    fg = tables.from_potts(inst)
    ref = search.solve(fg, search.Params(beta=beta, chi=chi, beam=beam))
    prob = spg.spg_problem_potts(ctx, inst)
    res = spg.spg_solve(ctx, prob, spg.params(beta=beta, chi=chi, beam=beam))
    st, E, lp = res.get()
    assert res.info()["error_flags"] == 0
    assert E[0] == ref.energies[0]
    if ref.near_ties == 0 and res.info()["near_ties"] == 0:
        np.testing.assert_array_equal(E, ref.energies)
        np.testing.assert_array_equal(st.astype(np.int64), ref.states)
        np.testing.assert_allclose(lp, ref.log_probs, rtol=1e-6, atol=1e-6)
    return E


@pytest.mark.parametrize("L,d", [(3, 3), (4, 2)])
def test_small_inpainting_reaches_the_brute_force_ground_state(spg, ctx, L, d):
    """Beam d^(L+1) keeps every class of the merge (the key is at most L + 1
    sites), so the search is an exact dynamic programme."""
    inst = I.inpainting(L, d, 1, ring=1.0)
    Eall, _ = exact.potts_all_energies(inst)
    E = compare(spg, ctx, inst, 1.0, 16, d ** (L + 1))
    assert E[0] == Eall.min()


@pytest.mark.parametrize("rows,cols,d", [(2, 40, 3), (3, 64, 2)])
def test_wide_grids(spg, ctx, rows, cols, d):
    inst = I.king_potts(rows, d, 40 + cols, cols=cols)
    compare(spg, ctx, inst, 1.0, 8, 16)


def test_inpainting_120x120(spg, ctx):
    """The paper's image size: every returned state's energy recomputed on
    the host, energies sorted, log-probabilities finite, in both modes (the
    free interior makes many configurations exactly degenerate, so which of
    them each mode keeps is decided by rounding and the two best energies
    are not compared)."""
    inst = I.inpainting(120, 4, 3)
    fg = tables.from_potts(inst)
    prob = spg.spg_problem_potts(ctx, inst)
    for prec in (spg.SPG_MIXED, spg.SPG_FP64):
        res = spg.spg_solve(ctx, prob, spg.params(beta=1.0, chi=8, beam=64, precision=prec))
        st, E, lp = res.get()
        assert res.info()["error_flags"] == 0
        assert np.all(np.diff(E) >= 0) and np.all(np.isfinite(lp))
        for k in range(min(4, len(E))):
            assert tables.energy(fg, st[k]) == E[k]
