"""The precision pattern through the C ABI: the per-result log-marginal error
against FP64 (check_fp64), and the FP64 truncation of the final boundary
rows in the mixed mode (fp64_rows), against the FP64 oracle.

The reported max_logmarg_err of a mixed result is the largest
|log p_mixed - log p_FP64| / max(1, |log p_FP64|) over the returned states
and their sites, each state's own conditional along its path.  Here it is
recomputed through a separate code path (spg_debug_marginals on the same
prefixes, in both precisions); the two must agree to FP32 rounding, and the
FP64 conditionals must be the oracle's.
"""
import numpy as np
import pytest

import instances as I
from oracle import boundary, peps, search, tables

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spg():
    import paper_2502_02317_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(spg):
    return spg.Context(0)


@pytest.mark.parametrize("make,beta,chi,beam,f64", [
    (lambda: I.chimera(3, 5, couplings="gauss", h_sigma=0.1), 1.0, 8, 16, 0),
    (lambda: I.chimera(3, 6, couplings="gauss", h_sigma=0.1), 2.0, 8, 32, 1),
    (lambda: I.king_ising(3, 3, 2, 4), 2.0, 16, 16, 0),
])
def test_check_fp64_matches_an_independent_computation(spg, ctx, make, beta, chi, beam, f64):
    """The library's figure against the same maximum taken over
    spg_debug_marginals (a separate code path: its own boundary build and
    left-environment kernel) in both precisions, which must agree to FP32
    rounding; and the FP64 side against the oracle wherever no truncation cut
    fell in a degenerate gap (there LAPACK and the GPU may keep different,
    equally valid, singular vectors)."""
    inst = make()
    fg = tables.from_ising(inst)
    prob = spg.spg_problem_ising(ctx, inst)
    prm = spg.params(beta=beta, chi=chi, beam=beam, precision=spg.SPG_MIXED, fp64_rows=f64)
    p64 = spg.params(beta=beta, chi=chi, beam=beam, precision=spg.SPG_FP64)
    res = spg.spg_solve(ctx, prob, spg.params(beta=beta, chi=chi, beam=beam, precision=spg.SPG_MIXED,
                                              fp64_rows=f64, check_fp64=1))
    st, E, lp = res.get()
    err = res.max_logmarg_err()
    info = res.info()
    assert info["max_logmarg_err"] == err and info["fp64_rows"] == min(f64, fg.rows - 1)
    degenerate = spg.spg_solve(ctx, prob, p64).info()["degenerate_cuts"] > 0
    bd = boundary.boundary_mpses(peps.build(fg, beta), chi)
    n = len(E)
    worst = 0.0
    for s in range(fg.n_sites):
        pre = st[:, :s].astype(np.int64)
        g = spg.spg_debug_marginals(ctx, prob, prm, s, pre)[np.arange(n), st[:, s]]
        r = spg.spg_debug_marginals(ctx, prob, p64, s, pre)[np.arange(n), st[:, s]]
        worst = max(worst, float(np.max(np.abs(g - r) / np.maximum(1.0, np.abs(r)))))
        if not degenerate:
            o = search.debug_marginals(fg, search.Params(beta=beta, chi=chi), s, pre, boundary=bd)
            np.testing.assert_allclose(r, o[np.arange(n), st[:, s]], rtol=1e-6, atol=1e-6)
    assert np.isfinite(err)
    assert abs(err - worst) <= 1e-6 + 1e-2 * worst, (err, worst)
    # the same search reached without the check
    st2, E2, lp2 = spg.spg_solve(ctx, prob, prm).get()
    np.testing.assert_array_equal(st2, st)
    np.testing.assert_array_equal(lp2, lp)


def test_check_fp64_reports_zero_in_fp64_and_nan_unchecked(spg, ctx):
    prob = spg.spg_problem_ising(ctx, I.chimera(2, 3))
    r64 = spg.spg_solve(ctx, prob, spg.params(beta=1.0, chi=8, beam=16, check_fp64=1))
    assert r64.max_logmarg_err() == 0.0
    rm = spg.spg_solve(ctx, prob, spg.params(beta=1.0, chi=8, beam=16, precision=spg.SPG_MIXED))
    assert np.isnan(rm.max_logmarg_err())
