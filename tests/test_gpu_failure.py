"""Failure detection through the C ABI, without faulting or hanging the GPU.

* A bounded wait that nothing completes (an mbarrier no thread or copy
  arrives on) gives up after its poll limit; the call returns SPG_ETIMEOUT
  and the context keeps working (a solve afterwards matches the oracle).
* An injected device-allocation failure (host-side hook) makes the solve and
  the problem construction return SPG_ENOMEM; with the hook off the same
  calls succeed on the same context.
"""
import numpy as np
import pytest

import instances as I
from oracle import search, tables

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spg():
    import paper_2502_02317_gb300 as m
    return m


def solve_matches_oracle(spg, ctx, inst):
    prob = spg.spg_problem_ising(ctx, inst)
    st, E, lp = spg.spg_solve(ctx, prob, spg.params(beta=1.0, chi=16, beam=64)).get()
    ref = search.solve(tables.from_ising(inst), search.Params(beta=1.0, chi=16, beam=64))
    np.testing.assert_array_equal(E, ref.energies)


def test_bounded_wait_times_out_and_the_context_stays_usable(spg):
    ctx = spg.Context(0)
    for polls in (0, 1000, 200000):
        assert spg.spg_check_bounded_wait(ctx, polls) == spg.SPG_ETIMEOUT
        assert "gave up" in spg.lib.spg_last_error(ctx.h).decode()
    solve_matches_oracle(spg, ctx, I.chimera(2, 1))


def test_injected_allocation_failure_is_reported_and_recoverable(spg):
    ctx = spg.Context(0)  # no workspace yet: the first solve allocates it
    prob = spg.spg_problem_ising(ctx, I.chimera(2, 2))
    try:
        spg.spg_inject_alloc_failure(0)
        with pytest.raises(spg.SpgError) as e:
            spg.spg_solve(ctx, prob, spg.params(beta=1.0, chi=16, beam=64))
        assert e.value.code == spg.SPG_ENOMEM
        spg.spg_inject_alloc_failure(0)
        with pytest.raises(spg.SpgError) as e:
            spg.spg_problem_ising(ctx, I.chimera(2, 3))
        assert e.value.code == spg.SPG_ENOMEM
    finally:
        spg.spg_inject_alloc_failure(-1)
    solve_matches_oracle(spg, ctx, I.chimera(2, 2))
