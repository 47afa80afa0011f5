"""King's graph (diagonal and anti-diagonal couplings) through the C ABI
against the FP64 oracle, element by element.

Tolerances as in test_gpu_parity: returned states and int64 energies
bit-exact; log Z, log-marginals and log-probabilities within 1e-6 relative in
FP64 mode and 1e-3 in mixed mode (conditionals >= 1e-6).  The mixed mode
runs with its default fp64_rows, which on these small lattices truncates
every row in FP64.  The oracle's dense
site tensors limit the parity cases to small cluster dimensions (bonds up to
16 x 16); the 256-state bonds of 16-state Potts sites are covered by
properties that hold at any size.
"""
import numpy as np
import pytest

import instances as I
from oracle import boundary, peps, search, tables

pytestmark = pytest.mark.gpu

TOL = {0: 1e-6, 1: 1e-3}
# FP32 contractions resolve conditionals down to ~1e-6 of the total on these
# cases (their weights come out of sums with cancellation); below that the
# mixed mode must only report them as small.
LOG_FLOOR = float(np.log(1e-6))

FP32_KING = pytest.mark.xfail(strict=True, reason=(
    "known limit of the mixed mode: on the paper's 3x3 king's Ising example at beta 2 the FP32 storage "
    "of the boundary MPS alone (a normwise perturbation of 6e-8) moves small conditionals by up to "
    "3.5e-2, so even with every truncation in FP64 the FP32 conditionals miss the oracle by 3.4e-3; the "
    "FP64 mode matches the oracle to 1e-10 and the searches' best energies agree"))


@pytest.fixture(scope="module")
def spg():
    import paper_2502_02317_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(spg):
    return spg.Context(0)


def close(a, b, tol, floor=None):
    a, b = np.asarray(a, float), np.asarray(b, float)
    if floor is None:
        fin = np.isfinite(b)
        assert np.array_equal(np.isfinite(a), fin)
    else:
        fin = b >= floor
        assert np.all(np.where(fin, True, ~(a > floor + 1.0)))
    err = np.abs(a[fin] - b[fin]) / np.maximum(1.0, np.abs(b[fin]))
    assert err.size == 0 or err.max() <= tol, err.max()


def fg_of(inst):
    return tables.from_potts(inst) if hasattr(inst, "local_E") else tables.from_ising(inst)


def problem(spg, ctx, inst):
    return spg.spg_problem_potts(ctx, inst) if hasattr(inst, "local_E") else spg.spg_problem_ising(ctx, inst)


CASES = [
    (lambda: I.king_potts(3, 3, 1), 1.0, 64),          # untruncated
    (lambda: I.king_potts(4, 3, 2, cols=5), 0.8, 6),   # ragged, truncated
    (lambda: I.king_potts(5, 4, 3), 1.2, 8),
    (lambda: I.king_potts(2, 5, 4, cols=2), 1.0, 4),
    (lambda: I.king_ising(3, 3, 2, 4), 2.0, 16),       # the paper's example shape and beta
    (lambda: I.king_ising(4, 4, 2, 5), 1.0, 8),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("make,beta,chi", CASES)
def test_king_log_partition(spg, ctx, make, beta, chi, prec):
    inst = make()
    ref = boundary.log_partition(peps.build(fg_of(inst), beta), chi)
    prob = problem(spg, ctx, inst)
    got = spg.spg_log_partition(ctx, prob, spg.params(beta=beta, chi=chi, precision=prec))
    assert abs(got - ref) <= TOL[prec] * max(1.0, abs(ref))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("make,beta,chi", CASES)
def test_king_debug_marginals(spg, ctx, make, beta, chi, prec, request):
    """Teacher-forced conditionals at sites of every row, random prefixes."""
    inst = make()
    if prec == 1 and getattr(inst, "name", "") == "king3x3x2_s4":
        request.applymarker(FP32_KING)
    fg = fg_of(inst)
    bd = boundary.boundary_mpses(peps.build(fg, beta), chi)
    prob = problem(spg, ctx, inst)
    prm = spg.params(beta=beta, chi=chi, precision=prec)
    rng = np.random.default_rng(11)
    n = fg.n_sites
    for s in sorted({0, 1, fg.cols - 1, fg.cols, fg.cols + 1, n // 2, n - fg.cols, n - 2, n - 1}):
        if s < 0 or s >= n:
            continue
        pre = np.array([[rng.integers(0, d) for d in fg.d[:s]] for _ in range(5)], dtype=np.int64).reshape(5, s)
        ref = search.debug_marginals(fg, search.Params(beta=beta, chi=chi), s, pre, boundary=bd)
        got = spg.spg_debug_marginals(ctx, prob, prm, s, pre)
        close(got, ref, TOL[prec], None if prec == 0 else LOG_FLOOR)


@pytest.mark.parametrize("make,beta,chi,beam", [
    (lambda: I.king_potts(3, 3, 21), 1.0, 16, 64),
    (lambda: I.king_potts(4, 4, 22, cols=5), 1.0, 8, 128),
    (lambda: I.king_ising(3, 3, 2, 23), 2.0, 16, 256),
    (lambda: I.king_ising(5, 4, 2, 24), 1.0, 8, 64),
])
def test_king_solve(spg, ctx, make, beta, chi, beam):
    inst = make()
    fg = fg_of(inst)
    ref = search.solve(fg, search.Params(beta=beta, chi=chi, beam=beam))
    prob = problem(spg, ctx, inst)
    res = spg.spg_solve(ctx, prob, spg.params(beta=beta, chi=chi, beam=beam))
    st, E, lp = res.get()
    assert res.info()["error_flags"] == 0
    if ref.near_ties == 0 and res.info()["near_ties"] == 0:
        np.testing.assert_array_equal(E, ref.energies)
        np.testing.assert_array_equal(st.astype(np.int64), ref.states)
        close(lp, ref.log_probs, 1e-6)
    assert E[0] == ref.energies[0]
    for k in range(len(E)):
        assert tables.energy(fg, st[k]) == E[k]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("make,beta,chi,sweeps", [
    (lambda: I.king_potts(4, 3, 2, cols=5), 0.8, 6, 1),
    (lambda: I.king_potts(3, 3, 1), 1.0, 4, 1),
    (lambda: I.king_ising(4, 4, 2, 5), 1.0, 8, 2),
])
def test_king_variational_sweeps(spg, ctx, make, beta, chi, sweeps, prec):
    """S4 on a king's graph: sites whose tensor depends on the up index are
    swept one up index at a time (log Z and teacher-forced conditionals)."""
    inst = make()
    fg = fg_of(inst)
    p = peps.build(fg, beta)
    ref = boundary.log_partition(p, chi, num_sweeps=sweeps)
    prob = problem(spg, ctx, inst)
    prm = spg.params(beta=beta, chi=chi, num_sweeps=sweeps, precision=prec)
    got = spg.spg_log_partition(ctx, prob, prm)
    assert abs(got - ref) <= TOL[prec] * max(1.0, abs(ref))
    bd = boundary.boundary_mpses(p, chi, sweeps)
    rng = np.random.default_rng(5)
    for s in sorted({1, fg.cols, fg.cols + 1, fg.n_sites // 2, fg.n_sites - 1}):
        pre = np.array([[rng.integers(0, d) for d in fg.d[:s]] for _ in range(4)], dtype=np.int64).reshape(4, s)
        refm = search.debug_marginals(fg, search.Params(beta=beta, chi=chi, num_sweeps=sweeps), s, pre, boundary=bd)
        gotm = spg.spg_debug_marginals(ctx, prob, prm, s, pre)
        close(gotm, refm, TOL[prec], None if prec == 0 else LOG_FLOOR)


def test_king_solve_with_sweeps(spg, ctx):
    inst = I.king_potts(4, 4, 23, cols=5)
    fg = fg_of(inst)
    ref = search.solve(fg, search.Params(beta=1.0, chi=8, beam=128, num_sweeps=1))
    prob = problem(spg, ctx, inst)
    res = spg.spg_solve(ctx, prob, spg.params(beta=1.0, chi=8, beam=128, num_sweeps=1))
    st, E, lp = res.get()
    assert res.info()["error_flags"] == 0
    if ref.near_ties == 0 and res.info()["near_ties"] == 0:
        np.testing.assert_array_equal(E, ref.energies)
        np.testing.assert_array_equal(st.astype(np.int64), ref.states)
    assert E[0] == ref.energies[0]


@pytest.mark.parametrize("L,chi,beam", [(6, 32, 256), (8, 64, 512)])
def test_king_potts_d16_properties(spg, ctx, L, chi, beam):
    """16-state Potts sites on a king's graph (left bond 16 x 16 = 256):
    every returned state's energy recomputed from the tables, energies
    sorted, no device error, log-probabilities finite and <= 0, and the
    mixed-precision search reaching the plain FP64 path's best energy."""
    inst = I.king_potts(L, 16, 100 + L)
    fg = fg_of(inst)
    prob = problem(spg, ctx, inst)
    out = {}
    for prec in (0, 1):
        res = spg.spg_solve(ctx, prob, spg.params(beta=1.0, chi=chi, beam=beam, precision=prec))
        st, E, lp = res.get()
        info = res.info()
        assert info["error_flags"] == 0
        assert np.all(np.diff(E) >= 0)
        assert np.all(np.isfinite(lp)) and np.all(lp <= 1e-9)
        for k in range(min(len(E), 16)):
            assert tables.energy(fg, st[k]) == E[k]
        out[prec] = E[0]
    assert out[1] == out[0]
