"""Autotuner of tile shapes (spg_autotune_*): the variants of k_gemm (outputs
per thread), k_xgemm (states per block) and the mixed k_marginals (site
staged in shared memory or read through L1) compute every output by the same
operations, so a solve must return the same states, integer energies and
log-probabilities bit for bit whichever variant runs.  Each mode below
solves fresh problems (a problem's first solve is uncaptured, its second is
captured into a graph with the variants of that moment), with the tuner off,
with every variant forced in turn, and tuned; the tuned run must also have
timed the three kernels' shapes."""
import numpy as np
import pytest

import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spg():
    import paper_2502_02317_gb300 as m
    yield m
    m.spg_autotune_set(m.SPG_TUNE_ON)


@pytest.fixture(scope="module")
def ctx(spg):
    return spg.Context(0)


def _run(spg, ctx, case):
    make, insts, prm, group = case
    probs = [make(ctx, x) for x in insts]
    out = []
    for rep in range(2):  # uncaptured (the shapes are timed here), captured
        rs = spg.spg_solve_group(ctx, probs, prm) if group else [spg.spg_solve(ctx, p, prm) for p in probs]
        out.append([r.get() for r in rs])
        assert all(r.info()["error_flags"] == 0 for r in rs)
    return out


def _cases(spg):
    chim = [I.chimera(4, 700 + k, couplings="gauss", h_sigma=0.1) for k in range(2)]
    return {
        "chimera_mixed": (spg.spg_problem_ising, chim[:1],
                          spg.params(beta=1.0, chi=32, beam=256, precision=spg.SPG_MIXED, num_sweeps=1), False),
        "chimera_fp64": (spg.spg_problem_ising, chim[:1],
                         spg.params(beta=1.0, chi=16, beam=128, precision=spg.SPG_FP64, num_sweeps=1), False),
        "chimera_group_mixed": (spg.spg_problem_ising, chim,
                                spg.params(beta=1.0, chi=32, beam=256, precision=spg.SPG_MIXED, num_sweeps=1), True),
        "king_potts_mixed": (spg.spg_problem_potts, [I.king_potts(3, 4, 41)],
                             spg.params(beta=1.0, chi=16, beam=64, precision=spg.SPG_MIXED, num_sweeps=1), False),
    }


@pytest.mark.parametrize("name", ["chimera_mixed", "chimera_fp64", "chimera_group_mixed", "king_potts_mixed"])
def test_every_variant_gives_the_same_solve(spg, ctx, name):
    case = _cases(spg)[name]
    spg.spg_autotune_set(spg.SPG_TUNE_OFF)
    ref = _run(spg, ctx, case)
    for a, b in zip(ref[0], ref[1]):
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
    modes = [spg.SPG_TUNE_FORCE + k for k in range(4)] + [spg.SPG_TUNE_ON]
    for mode in modes:
        spg.spg_autotune_set(mode)
        if mode == spg.SPG_TUNE_ON:
            spg.spg_autotune_clear()
        got = _run(spg, ctx, case)
        for rep in range(2):
            for (sa, Ea, la), (sb, Eb, lb) in zip(got[rep], ref[0]):
                np.testing.assert_array_equal(sa, sb)
                np.testing.assert_array_equal(Ea, Eb)
                np.testing.assert_array_equal(la, lb)
    timed = spg.spg_autotune_report()
    kernels = {t[0] for t in timed}
    assert "k_gemm" in kernels and "k_xgemm" in kernels
    if "mixed" in name:
        assert "k_marginals" in kernels
    group = {t[2] for t in timed}
    assert (2 in group) == name.startswith("chimera_group")
    for kern, dev, grp, shape, choice, us in timed:
        # the chosen variant ran and was the fastest of those that ran
        assert us[choice] >= 0.0
        assert us[choice] == min(t for t in us if t >= 0.0)
