"""Pins of the oracle's ``Sparsity = Sparse`` construction (paper Sec. 3.1 and
3.1.1: clusters of many spins, Zephyr's 16 and Pegasus' 24, whose explicit
tensors are infeasible), on the CPU.

* Where the dense construction is feasible (clusters of up to 10 spins) the
  sparse one must give the same tables, projectors, classes, Boltzmann
  blocks and site tensors, the same log Z and the same search.
* Beyond it: Eq. 2 on random spin configurations equals the tables' energy
  (exact integers); log Z at an untruncated bond dimension equals brute
  force (24 spins) or ``exact.interface_sum`` (Zephyr-size cells: a sum over
  the interface spins' configurations written from Eq. 2, sharing nothing
  with the tables); teacher-forced conditionals equal the exact ones.
"""
import numpy as np
import pytest

import instances as I
from oracle import boundary, exact, peps, search, tables


def log_z(fg, beta, chi):
    p = peps.build(fg, beta)
    bd = boundary.boundary_mpses(p, chi, 0, down_to=0)
    B0 = bd[0]
    return B0.lognorm + float(np.log(boundary.contract_value(B0))) + p.log_offset


SMALL = [lambda: I.chimera(3, 1), lambda: I.chimera(3, 2, couplings="gauss", h_sigma=0.1),
         lambda: I.king_ising(3, 3, 2, 5), lambda: I.large_cells(2, 2, 8, 3),
         lambda: I.large_cells(2, 3, 6, 7, links=3, node_type=I.SQUARE)]


@pytest.mark.parametrize("make", SMALL)
def test_sparse_tables_and_sites_equal_dense(make):
    inst = make()
    a, b = tables.from_ising(inst, sparse=False), tables.from_ising(inst, sparse=True)
    assert not a.sparse and b.sparse
    assert sorted(a.edges) == sorted(b.edges)
    for s in range(a.n_sites):
        np.testing.assert_array_equal(a.E_loc[s], b.E_loc[s])
    rng = np.random.default_rng(0)
    for k, ea in a.edges.items():
        eb = b.edges[k]
        np.testing.assert_array_equal(ea.R, eb.R)
        np.testing.assert_array_equal(ea.Pm, eb.Pm)
        np.testing.assert_array_equal(ea.Pn, eb.Pn)
        assert ea.min() == eb.min()
        for _ in range(50):
            x, y = int(rng.integers(a.d[k[0]])), int(rng.integers(a.d[k[1]]))
            assert eb.value(x, y) == int(ea.E[x, y]) == int(eb.R[eb.Pm[x], eb.Pn[y]])
    pa, pb = peps.build(a, 1.3), peps.build(b, 1.3)
    assert pa.log_offset == pb.log_offset
    for sa, sb in zip(pa.sites, pb.sites):
        for f in ("PL", "PU", "PR", "PD", "PG", "repR", "repD", "w", "b_left", "b_up", "b_ad", "g_of_u"):
            np.testing.assert_array_equal(getattr(sa, f), getattr(sb, f))
        np.testing.assert_allclose(peps.mpo_site(sb), peps.mpo_site(sa), rtol=1e-13, atol=0)


@pytest.mark.parametrize("make", SMALL[:2] + [lambda: I.large_cells(2, 2, 10, 11, links=2)])
def test_sparse_search_and_log_z_equal_dense(make):
    inst = make()
    a, b = tables.from_ising(inst, sparse=False), tables.from_ising(inst, sparse=True)
    # chi 64 truncates nothing here: the sites differ from the dense ones only
    # by the summation order of their sums over states, which a truncation at
    # a degenerate cut (+-1 couplings) would turn into a different but equally
    # valid subspace
    prm = search.Params(beta=1.0, chi=64, beam=16, num_sweeps=1)
    ra, rb = search.solve(a, prm), search.solve(b, prm)
    np.testing.assert_array_equal(ra.states, rb.states)
    np.testing.assert_array_equal(ra.energies, rb.energies)
    np.testing.assert_allclose(rb.log_probs, ra.log_probs, rtol=1e-10, atol=1e-10)
    assert abs(log_z(a, 1.0, 64) - log_z(b, 1.0, 64)) <= 1e-10 * max(1.0, abs(log_z(a, 1.0, 64)))


def test_eq2_on_sparse_tables_of_zephyr_and_pegasus_size_cells():
    """Exact integers: the sparse tables' energy of random configurations
    equals Eq. 2 on the decoded spins, for cells of 16 (Zephyr) and 24
    (Pegasus) spins; the reduced tables reproduce every sampled entry."""
    rng = np.random.default_rng(3)
    for inst in (I.large_cells(2, 2, 16, 21, links=2), I.large_cells(1, 2, 24, 22, links=3, intra="ring")):
        fg = tables.from_ising(inst)
        assert fg.sparse and max(fg.d) == 2 ** max(len(sp) for sp in fg.spins_of_site)
        for _ in range(40):
            s = rng.choice(np.array([-1, 1]), size=inst.n_spins)
            x = [int(sum(((s[sp[k]] + 1) // 2) << k for k in range(len(sp)))) for sp in fg.spins_of_site]
            assert tables.energy(fg, x) == tables.ising_energy(inst, s) == tables.energy_reduced(fg, x)


def test_24_spins_in_two_cells_against_brute_force():
    """Two 12-spin cells (24 spins): log Z at an untruncated bond dimension,
    and the teacher-forced conditionals of both sites, equal brute force."""
    inst = I.large_cells(1, 2, 12, 31, links=3)
    fg = tables.from_ising(inst)
    assert fg.sparse
    beta = 0.6
    bf = exact.brute_force(inst, beta)
    assert abs(log_z(fg, beta, 64) - bf["logZ"]) <= 1e-9 * abs(bf["logZ"])
    cs = exact.cluster_states(inst.n_spins, fg.spins_of_site)
    prm = search.Params(beta=beta, chi=64, beam=4)
    got0 = search.debug_marginals(fg, prm, 0, [[]])[0]
    ref0 = exact.exact_conditional(bf["E"], beta, 0, cs, 0, [], fg.d[0])
    np.testing.assert_allclose(got0, ref0, rtol=1e-9, atol=1e-9)
    pre = [[int(np.argmax(ref0))], [7], [4095]]
    got1 = search.debug_marginals(fg, prm, 1, pre)
    for k, p in enumerate(pre):
        ref1 = exact.exact_conditional(bf["E"], beta, 0, cs, 1, p, fg.d[1])
        np.testing.assert_allclose(got1[k], ref1, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("rows,cols,links,node", [(1, 3, 2, I.KING), (2, 2, 1, I.KING), (2, 2, 2, I.SQUARE)])
def test_zephyr_size_cells_against_the_interface_sum(rows, cols, links, node):
    """Cells of 16 spins (65,536 states): log Z at an untruncated bond
    dimension, the marginal of the first cell and the teacher-forced
    conditionals of the later cells equal ``exact.interface_sum``; every state the search returns carries its Eq. 2
    energy, none below the exact ground energy."""
    inst = I.large_cells(rows, cols, 16, 40 + rows * 10 + links, links=links, node_type=node)
    fg = tables.from_ising(inst)
    beta = 0.5
    ref = exact.interface_sum(inst, beta)
    assert abs(log_z(fg, beta, 64) - ref["logZ"]) <= 1e-9 * abs(ref["logZ"])
    prm = search.Params(beta=beta, chi=64, beam=2)
    got0 = search.debug_marginals(fg, prm, 0, [[]])[0]
    np.testing.assert_allclose(got0, ref["logp"], rtol=1e-9, atol=1e-9)
    # teacher-forced conditionals of the later sites given random prefixes
    rng = np.random.default_rng(5)
    for site in range(1, fg.n_sites):
        pre = [int(rng.integers(fg.d[t])) for t in range(site)]
        got = search.debug_marginals(fg, prm, site, [pre])[0]
        exact_c = exact.interface_sum(inst, beta, fixed=dict(enumerate(pre)), target=site)["logp"]
        fin = np.isfinite(exact_c)
        assert np.array_equal(np.isfinite(got), fin)
        np.testing.assert_allclose(got[fin], exact_c[fin], rtol=1e-9, atol=1e-8)
    res = search.solve(fg, prm)
    for x, E in zip(res.states, res.energies):
        assert E >= ref["ground"]
        assert E == tables.ising_energy(inst, tables.spins_from_states(fg, x, inst.n_spins))


def test_the_eight_lattice_transformations_keep_log_z_of_large_cells():
    """Sec. 3.1 (all_lattice_transformations): the 8 rotations / reflections of
    a 2 x 3 king's grid of 16-spin cells give the same untruncated log Z."""
    from oracle import lattice
    inst = I.large_cells(2, 3, 16, 77, links=1)
    vals = [log_z(tables.from_ising(lattice.transform(inst, k)), 0.4, 64) for k in range(8)]
    assert max(vals) - min(vals) <= 1e-9 * abs(vals[0])
    assert abs(vals[0] - exact.interface_sum(inst, 0.4)["logZ"]) <= 1e-9 * abs(vals[0])


@pytest.mark.parametrize("make", [lambda: I.large_cells(1, 2, 10, 4), lambda: I.large_cells(2, 2, 4, 9, links=2),
                                  lambda: I.chimera(2, 3, couplings="gauss", h_sigma=0.1, cols=1)])
def test_interface_sum_equals_brute_force(make):
    """exact.interface_sum (used above for cells too large for brute force)
    against exact.brute_force on instances of at most 20 spins: log Z, the
    ground energy and the exact marginal of the first cell's states."""
    inst = make()
    beta = 0.7
    bf = exact.brute_force(inst, beta)
    it = exact.interface_sum(inst, beta)
    assert abs(it["logZ"] - bf["logZ"]) <= 1e-12 * abs(bf["logZ"])
    assert it["ground"] == bf["ground"]
    cos = np.asarray(inst.cluster_of_spin)
    c0 = int(np.nonzero((np.asarray(inst.cluster_row) == 0) & (np.asarray(inst.cluster_col) == 0))[0][0])
    members = np.sort(np.nonzero(cos == c0)[0])
    idx = np.arange(2 ** inst.n_spins, dtype=np.int64)
    x0 = np.zeros_like(idx)
    for k, sp in enumerate(members):
        x0 |= ((idx >> int(sp)) & 1) << k
    u = 2.0 ** -inst.energy_shift
    m = np.full(2 ** len(members), -np.inf)
    np.logaddexp.at(m, x0, -beta * u * bf["E"].astype(np.float64))
    np.testing.assert_allclose(it["logp"], m - bf["logZ"], rtol=0, atol=1e-10)
    # conditionals given the first sites' states, against brute force
    fg = tables.from_ising(inst)
    cs = exact.cluster_states(inst.n_spins, fg.spins_of_site)
    rng = np.random.default_rng(2)
    for site in range(1, fg.n_sites):
        pre = [int(rng.integers(fg.d[t])) for t in range(site)]
        got = exact.interface_sum(inst, beta, fixed=dict(enumerate(pre)), target=site)["logp"]
        ref = exact.exact_conditional(bf["E"], beta, inst.energy_shift, cs, site, pre, fg.d[site])
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10)


def test_28_spins_in_two_cells_against_the_c_brute_force():
    """Two 14-spin cells (28 spins, beyond the NumPy enumeration): log Z at an
    untruncated bond dimension equals the C enumerator's (2^28 configurations
    on the host's cores)."""
    inst = I.large_cells(1, 2, 14, 33, links=3)
    fg = tables.from_ising(inst)
    assert fg.sparse
    ref = exact.brute_force_c(inst, 0.6)
    assert abs(log_z(fg, 0.6, 64) - ref["logZ"]) <= 1e-9 * abs(ref["logZ"])
