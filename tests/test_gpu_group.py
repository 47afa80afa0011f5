"""Lockstep groups (spg_solve_group, and spg_solve_batch's grouping): every
instance of a group must come out exactly as its own spg_solve (states,
integer energies and log-probabilities equal bit for bit: the same kernels
run on the same data, only the launch covers several instances), on the
paths a group exercises: the mixed and FP64 modes, the tensor-core products
(tcgen05 tiles read through a tensor map over the instances), the guarded
Cholesky-QR panels, the multi-CTA tall QR (king's Potts), the variational
sweeps, droplets, graph capture and replay, and problems updated in place.
The first instance of a group is also checked against the oracle."""
import numpy as np
import pytest

import instances as I
from oracle import search, tables

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spg():
    import paper_2502_02317_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(spg):
    return spg.Context(0)


def _same(a, b):
    sa, Ea, la = a.get()
    sb, Eb, lb = b.get()
    np.testing.assert_array_equal(sa, sb)
    np.testing.assert_array_equal(Ea, Eb)
    np.testing.assert_array_equal(la, lb)


def _check_group(spg, ctx, insts, prm, oracle_prm=None, make=None):
    make = make or spg.spg_problem_ising
    probs = [make(ctx, x) for x in insts]
    singles = [spg.spg_solve(ctx, p, prm) for p in probs]
    for rep in range(3):  # uncaptured, captured, replayed
        grp = spg.spg_solve_group(ctx, probs, prm)
        for g, s in zip(grp, singles):
            _same(g, s)
            info = g.info()
            assert info["group_size"] == len(probs) and info["error_flags"] == 0
    if oracle_prm is not None:
        fg = tables.from_ising(insts[0]) if make is spg.spg_problem_ising else tables.from_potts(insts[0])
        ref = search.solve(fg, oracle_prm)
        st, E, _ = singles[0].get()
        assert E[0] == ref.energies[0]
    return probs


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_chimera_group_equals_single_solves(spg, ctx, precision):
    p = spg.SPG_MIXED if precision == "mixed" else spg.SPG_FP64
    insts = [I.chimera(4, 500 + k, couplings="gauss", h_sigma=0.1) for k in range(5)]
    prm = spg.params(beta=1.0, chi=16, beam=128, precision=p, num_sweeps=1)
    _check_group(spg, ctx, insts, prm, search.Params(beta=1.0, chi=16, beam=128, num_sweeps=1))


def test_bench_size_group_tensor_cores_and_panels(spg, ctx):
    """16 x 16 Chimera, chi 32, beam 1024: 512 x 512 zipper matrices whose
    products run on tcgen05 (tensor map over the group's instances) and whose
    orthonormalisations take the Cholesky-QR panels."""
    insts = [I.chimera(16, 100 * 1000 + k, couplings="gauss", h_sigma=0.1) for k in range(3)]
    prm = spg.params(beta=1.0, chi=32, beam=1024, precision=spg.SPG_MIXED, num_sweeps=1)
    _check_group(spg, ctx, insts, prm)


def test_king_potts_group_tall_qr(spg, ctx):
    """King's-graph Potts (d = 8, chi 64): zipper columns of >= 2048 entries
    go through the multi-CTA tall QR; anti-diagonal factors in the sweeps."""
    insts = [I.king_potts(4, 8, 30 + k) for k in range(3)]
    prm = spg.params(beta=1.0, chi=64, beam=256, precision=spg.SPG_MIXED, num_sweeps=1, fp64_rows=0)
    _check_group(spg, ctx, insts, prm, make=spg.spg_problem_potts)


def test_droplets_in_a_group(spg, ctx):
    insts = [I.chimera(3, 40 + k, couplings="gauss", h_sigma=0.1) for k in range(4)]
    prm = spg.params(beta=1.0, chi=16, beam=64, precision=spg.SPG_FP64, droplet_energy=2.0,
                     droplet_hamming=2)
    probs = [spg.spg_problem_ising(ctx, x) for x in insts]
    grp = spg.spg_solve_group(ctx, probs, prm)
    for g, p in zip(grp, probs):
        s = spg.spg_solve(ctx, p, prm)
        _same(g, s)
        dg, ds_ = g.droplets(), s.droplets()
        for a, b in zip(dg, ds_):
            np.testing.assert_array_equal(a, b)


def test_group_after_update_in_place(spg, ctx):
    insts = [I.chimera(4, 600 + k, couplings="gauss", h_sigma=0.1) for k in range(4)]
    prm = spg.params(beta=1.0, chi=16, beam=64, precision=spg.SPG_MIXED)
    probs = _check_group(spg, ctx, insts, prm)
    for k, p in enumerate(probs):
        b = I.chimera(4, 700 + k, couplings="gauss", h_sigma=0.1)
        spg.spg_problem_update_ising(p, b.J, b.h)
    grp = spg.spg_solve_group(ctx, probs, prm)  # the captured group, new tables
    for g, p in zip(grp, probs):
        _same(g, spg.spg_solve(ctx, p, prm))


def test_batch_groups_by_structure(spg, ctx):
    """An uneven batch: the items of each size (same parameters) form lockstep
    groups, the others run alone; every result equals its own solve."""
    sizes = [3, 4, 3, 5, 4, 3, 4]
    insts = [I.chimera(L, 800 + k) for k, L in enumerate(sizes)]
    probs = [spg.spg_problem_ising(ctx, x) for x in insts]
    prms = [spg.params(beta=1.0, chi=16, beam=64, precision=spg.SPG_MIXED) for _ in probs]
    prms[6] = spg.params(beta=1.0, chi=8, beam=64, precision=spg.SPG_MIXED)  # other parameters: alone
    res = spg.spg_solve_batch(ctx, probs, prms)
    want = {0: 3, 2: 3, 5: 3, 1: 2, 4: 2, 3: 1, 6: 1}
    for i, r in enumerate(res):
        assert r.info()["group_size"] == want[i], i
        _same(r, spg.spg_solve(ctx, probs[i], prms[i]))
    # group_max 1: every item alone
    one = [spg.params(beta=1.0, chi=16, beam=64, precision=spg.SPG_MIXED, group_max=1) for _ in probs]
    for r in spg.spg_solve_batch(ctx, probs, one):
        assert r.info()["group_size"] == 1
    # group_max 2: groups of at most two, the items of a class spread evenly
    two = [spg.params(beta=1.0, chi=16, beam=64, precision=spg.SPG_MIXED, group_max=2) for _ in probs]
    res2 = spg.spg_solve_batch(ctx, probs, two)
    assert max(r.info()["group_size"] for r in res2) == 2
    for i, r in enumerate(res2):
        _same(r, spg.spg_solve(ctx, probs[i], two[i]))


def test_group_refusals(spg, ctx):
    a = spg.spg_problem_ising(ctx, I.chimera(3, 1))
    b = spg.spg_problem_ising(ctx, I.chimera(4, 1))
    prm = spg.params(beta=1.0, chi=8, beam=32)
    with pytest.raises(spg.SpgError) as e:
        spg.spg_solve_group(ctx, [a, b], prm)
    assert e.value.code == spg.SPG_EINVAL
    with pytest.raises(spg.SpgError) as e:
        spg.spg_solve_group(ctx, [a, a], spg.params(beta=1.0, chi=8, beam=32, precision=spg.SPG_MIXED,
                                                    check_fp64=1))
    assert e.value.code == spg.SPG_EUNSUPPORTED
    # the context is still usable, and the same problem twice is a valid group
    r = spg.spg_solve_group(ctx, [a, a], prm)
    _same(r[0], r[1])
