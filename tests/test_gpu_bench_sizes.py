"""Parity of the CUDA path with the FP64 oracle at the sizes the benchmark
runs, through the C ABI.

* 16 x 16 Chimera, Gaussian J (the benchmark's first instance), chi 32, one
  variational sweep per row: log Z and teacher-forced conditionals.  The
  zipper matrices are 512 x 512 with a 48-column block, so the mixed mode's
  truncations run on the tcgen05 tensor-core products and the guarded
  Cholesky-QR panels; the test checks that those kernels ran.
* King's-graph Potts, d = 8, 4 x 4, chi 64: zipper matrices of 4096 rows, so
  the multi-CTA tall QR and (mixed) the tensor-core products run inside the
  solve.
* Beam 1024 on a 4 x 4 Chimera at chi 32, with and without merging: the
  65,536-bin radix select over up to 262,144 candidates per step; states and
  int64 energies bit-exact, log-probabilities within the FP64 bound.

Tolerances as in test_gpu_parity: 1e-6 * max(1, |oracle|) in FP64, 1e-3 in
mixed mode on conditionals >= 1e-9.  The mixed-mode search returns the
oracle's states exactly when every prune cut of the oracle is wider than
twice the mixed tolerance (no candidate near the cut can swap places).
"""
import numpy as np
import pytest

import instances as I
from oracle import boundary, peps, search, tables

pytestmark = pytest.mark.gpu

TOL = {0: 1e-6, 1: 1e-3}
LOG_FLOOR = float(np.log(1e-9))


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


def log_z_of(p, bd):
    B0 = bd[0]
    return B0.lognorm + float(np.log(boundary.contract_value(B0))) + p.log_offset


def kernels_run(spg, ctx, fn):
    """Names of the library kernels that fn() launched."""
    spg.spg_profile(ctx, True)
    try:
        out = fn()
    finally:
        rep = spg.spg_profile_report(ctx)
        spg.spg_profile(ctx, False)
    return out, set(rep)


@pytest.fixture(scope="module")
def chimera16():
    """The benchmark's first instance: 16 x 16 Chimera (2048 spins, 256-state
    clusters), J ~ N(0, 1), h ~ N(0, 0.1); oracle boundary MPSs at chi 32
    with one variational sweep per row (about half a minute on the host)."""
    inst = I.chimera(16, 0, couplings="gauss", h_sigma=0.1)
    fg = tables.from_ising(inst)
    p = peps.build(fg, 1.0)
    bd = boundary.boundary_mpses(p, 32, 1, down_to=0)
    return inst, fg, p, bd


@pytest.mark.parametrize("prec", [0, 1])
def test_chimera16_log_partition(spg, ctx, chimera16, prec):
    inst, fg, p, bd = chimera16
    ref = log_z_of(p, bd)
    prob = spg.spg_problem_ising(ctx, inst)
    prm = spg.params(beta=1.0, chi=32, num_sweeps=1, precision=prec)
    got, ran = kernels_run(spg, ctx, lambda: spg.spg_log_partition(ctx, prob, prm))
    assert abs(got - ref) <= TOL[prec] * max(1.0, abs(ref)), (got, ref)
    if prec == 1:
        assert "k_umma_tf32x3" in ran and "k_cgs2_rows" in ran


@pytest.mark.parametrize("prec", [0, 1])
def test_chimera16_marginals(spg, ctx, chimera16, prec):
    """Teacher-forced conditionals at sites of the first, a middle and the
    last rows; the prefixes are random states."""
    inst, fg, p, bd = chimera16
    prob = spg.spg_problem_ising(ctx, inst)
    prm = spg.params(beta=1.0, chi=32, num_sweeps=1, precision=prec)
    rng = np.random.default_rng(17)
    n = fg.n_sites
    for s in (0, 5, fg.cols, 7 * fg.cols + 9, n - fg.cols, n - 1):
        pre = np.array([[rng.integers(0, d) for d in fg.d[:s]] for _ in range(4)], dtype=np.int64).reshape(4, s)
        ref = search.debug_marginals(fg, search.Params(beta=1.0, chi=32, num_sweeps=1), s, pre, boundary=bd)
        got, ran = kernels_run(spg, ctx, lambda: spg.spg_debug_marginals(ctx, prob, prm, s, pre))
        close(got, ref, TOL[prec], None if prec == 0 else LOG_FLOOR)
        # the mixed mode's right environments of Chimera rows run on the
        # tensor cores (renv_tc.cu), the FP64 mode's on k_right_envs
        assert ("k_renv_tc" in ran) == (prec == 1) and ("k_right_envs" in ran) == (prec == 0), ran


@pytest.fixture(scope="module")
def king8():
    inst = I.king_potts(4, 8, 31)
    fg = tables.from_potts(inst)
    p = peps.build(fg, 1.0)
    bd = boundary.boundary_mpses(p, 64, 0, down_to=0)
    return inst, fg, p, bd


@pytest.mark.parametrize("prec", [0, 1])
def test_king_d8_chi64_log_partition(spg, ctx, king8, prec):
    inst, fg, p, bd = king8
    ref = log_z_of(p, bd)
    prob = spg.spg_problem_potts(ctx, inst)
    # fp64_rows = 0: FP32 truncations throughout, so that the tensor-core
    # products run (the default truncates every row of a lattice this small
    # in FP64)
    prm = spg.params(beta=1.0, chi=64, precision=prec, fp64_rows=0)
    got, ran = kernels_run(spg, ctx, lambda: spg.spg_log_partition(ctx, prob, prm))
    assert abs(got - ref) <= TOL[prec] * max(1.0, abs(ref)), (got, ref)
    assert "k_tsqr_leaf" in ran
    if prec == 1:
        assert "k_umma_tf32x3" in ran


@pytest.mark.parametrize("prec", [0, 1])
def test_king_d8_chi64_marginals(spg, ctx, king8, prec):
    """The mixed mode as the precision pattern runs it: the final boundary
    row (B_1) truncated in FP64, rows 2 and 3 in FP32 (tall QR and
    tensor-core products).  With every row in FP32 (fp64_rows = 0, the
    log Z test above) the conditionals of this 16-state lattice sit at
    about 1.1e-3 of the oracle: FP32's truncation floor, the limit that the
    FP64 final rows remove."""
    inst, fg, p, bd = king8
    prob = spg.spg_problem_potts(ctx, inst)
    prm = spg.params(beta=1.0, chi=64, precision=prec, fp64_rows=1)
    rng = np.random.default_rng(19)
    for s in (0, 3, 5, 9, 14, 15):
        pre = np.array([[rng.integers(0, d) for d in fg.d[:s]] for _ in range(4)], dtype=np.int64).reshape(4, s)
        ref = search.debug_marginals(fg, search.Params(beta=1.0, chi=64), s, pre, boundary=bd)
        got = spg.spg_debug_marginals(ctx, prob, prm, s, pre)
        close(got, ref, TOL[prec], None if prec == 0 else float(np.log(1e-6)))


_BEAM1024 = {}


def beam1024_ref(merge):
    """Oracle search of the 4 x 4 Chimera at beam 1024 (40-80 s on the host),
    computed once per merge mode."""
    if merge not in _BEAM1024:
        inst = I.chimera(4, 12, couplings="gauss", h_sigma=0.1)
        fg = tables.from_ising(inst)
        _BEAM1024[merge] = (inst, fg, search.solve(fg, search.Params(beta=1.0, chi=32, beam=1024, merge=merge)))
    return _BEAM1024[merge]


@pytest.mark.parametrize("merge", [True, False])
@pytest.mark.parametrize("prec", [0, 1])
def test_beam1024_chimera4x4(spg, ctx, merge, prec):
    """The benchmark's beam width on a 4 x 4 Chimera (Gaussian J, chi 32)."""
    inst, fg, ref = beam1024_ref(merge)
    prob = spg.spg_problem_ising(ctx, inst)
    res = spg.spg_solve(ctx, prob, spg.params(beta=1.0, chi=32, beam=1024, merge=int(merge), precision=prec))
    st, E, lp = res.get()
    info = res.info()
    assert info["error_flags"] == 0
    assert E[0] == ref.energies[0]
    assert len(E) == len(ref.energies)
    exact_set = ref.near_ties == 0 and info["near_ties"] == 0 and (prec == 0 or ref.min_cut_gap > 2 * TOL[prec])
    if prec == 0:
        # FP64: a near tie is the only way the sets may differ
        assert exact_set or ref.near_ties > 0 or info["near_ties"] > 0
    if exact_set:
        np.testing.assert_array_equal(E, ref.energies)
        np.testing.assert_array_equal(st.astype(np.int64), ref.states)
        close(lp, ref.log_probs, TOL[prec])
    for k in range(len(E)):
        assert tables.energy(fg, st[k]) == E[k]
