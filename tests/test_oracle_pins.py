"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: every expected value comes from
brute-force enumeration of Eq. 2, from spin-level transfer matrices, from a
hand-computed example, from a symmetry of the model, or from a limit in which
the heuristic becomes exact.  The paper prints no worked numbers (its figures
carry no data), so no value is quoted from it.
"""
import itertools

import numpy as np
import pytest

import instances as I
from oracle import boundary, exact, peps, search, tables


def rand_states(fg, rng):
    return [int(rng.integers(0, d)) for d in fg.d]


# ---------------------------------------------------------------- O1 / O2

@pytest.mark.parametrize("make", [
    lambda: I.chimera(2, 3),
    lambda: I.chimera(2, 4, couplings="gauss", h_sigma=0.1, cols=3),
    lambda: I.square(4, 2, h_sigma=0.3),
    lambda: I.king_ising(3, 3, 2, 1),
])
def test_table_energy_equals_eq2(make):
    """Eq. 1 through the cluster tables == Eq. 2 on the decoded spins."""
    inst = make()
    fg = tables.from_ising(inst)
    rng = np.random.default_rng(0)
    for _ in range(40):
        x = rand_states(fg, rng)
        s = tables.spins_from_states(fg, x, inst.n_spins)
        e2 = tables.ising_energy(inst, s)
        assert tables.energy(fg, x) == e2
        assert tables.energy_reduced(fg, x) == e2


def test_projector_hand_example():
    """Two 2-spin clusters joined by one coupler s1*s2 (J = 1)."""
    inst = I.IsingInstance(4, np.array([1], np.int32), np.array([2], np.int32), np.array([1.0]),
                           np.zeros(4), np.array([0, 0, 1, 1], np.int32), 1, 2,
                           np.array([0, 0], np.int32), np.array([0, 1], np.int32), 0, I.SQUARE)
    fg = tables.from_ising(inst)
    e = fg.edges[(0, 1)]
    # rows depend on bit 1 of x_m, columns on bit 0 of x_n (first occurrence order)
    assert e.Pm.tolist() == [0, 0, 1, 1]
    assert e.Pn.tolist() == [0, 1, 0, 1]
    # s = 2b-1: row 0 has s1 = -1, column 0 has s2 = -1 -> +1
    assert e.R.tolist() == [[1, -1], [-1, 1]]
    assert fg.E_loc[0].tolist() == [0, 0, 0, 0]


def test_projectors_reconstruct_and_chimera_dims():
    inst = I.chimera(3, 5, couplings="gauss")
    fg = tables.from_ising(inst)
    for e in fg.edges.values():
        assert np.array_equal(e.R[np.ix_(e.Pm, e.Pn)], e.E)
        assert e.R.shape == (16, 16)  # 4 couplers with J != 0 per edge
    # a zero coupler leaves 8 distinct rows/columns on that edge
    inst.J = inst.J.copy()
    # vertical couplers of cell (0,0)-(1,0) come after the 9*16 intra ones
    inst.J[9 * 16] = 0.0
    fg = tables.from_ising(inst)
    e = fg.edges[(0, 3)]
    assert e.R.shape == (8, 8)
    assert np.array_equal(e.R[np.ix_(e.Pm, e.Pn)], e.E)


def test_inexact_input_rejected():
    inst = I.chimera(2, 0)
    inst.J = inst.J.copy()
    inst.J[0] = 0.3
    with pytest.raises(tables.InexactEnergy):
        tables.from_ising(inst)


# ---------------------------------------------------------------- O3 - O5

@pytest.mark.parametrize("make,beta,chi", [
    (lambda: I.square(4, 1), 0.7, 64),
    (lambda: I.square(3, 7, cols=5, h_sigma=0.5), 1.3, 64),
    (lambda: I.chimera(1, 5, cols=3), 1.0, 256),
    (lambda: I.chimera(3, 2, cols=1), 1.0, 256),
    (lambda: I.chimera(2, 8, couplings="gauss", h_sigma=0.2, cols=1), 2.0, 256),
])
def test_log_partition_vs_brute_force(make, beta, chi):
    """No truncation at this chi: log Z equals the sum over all 2^n states."""
    inst = make()
    bf = exact.brute_force(inst, beta)
    p = peps.build(tables.from_ising(inst), beta)
    assert boundary.log_partition(p, chi) == pytest.approx(bf["logZ"], rel=1e-12, abs=1e-10)


@pytest.mark.parametrize("seed,couplings,h,beta", [(0, "pm1", 0.0, 1.0), (3, "gauss", 0.1, 1.0),
                                                   (4, "gauss", 0.1, 4.0)])
def test_log_partition_vs_transfer_matrix(seed, couplings, h, beta):
    """3x3 Chimera: exact spin-level transfer matrix vs untruncated zipper."""
    inst = I.chimera(3, seed, couplings=couplings, h_sigma=h)
    ref = exact.chimera_strip(inst, beta)
    p = peps.build(tables.from_ising(inst), beta)
    assert boundary.log_partition(p, 256) == pytest.approx(ref["logZ"], rel=1e-12)
    # truncation to chi = 16 is a heuristic, but must stay close on this size
    assert abs(boundary.log_partition(p, 16) - ref["logZ"]) < 0.05


def transform(inst, k):
    """k-th of the 8 symmetries of the square grid applied to the clusters."""
    R, C = inst.grid_rows, inst.grid_cols
    r, c = inst.cluster_row.copy(), inst.cluster_col.copy()
    if k & 4:
        r, c = c, r
        R, C = C, R
    if k & 1:
        r = R - 1 - r
    if k & 2:
        c = C - 1 - c
    out = I.IsingInstance(**{**inst.__dict__})
    out.grid_rows, out.grid_cols, out.cluster_row, out.cluster_col = R, C, r.astype(np.int32), c.astype(np.int32)
    return out


def test_lattice_transformations_same_log_partition():
    """Sec. 3.1: the 8 lattice transformations leave the model unchanged."""
    inst = I.chimera(3, 9)
    ref = exact.chimera_strip(inst, 1.0)["logZ"]
    for k in range(8):
        p = peps.build(tables.from_ising(transform(inst, k)), 1.0)
        assert boundary.log_partition(p, 256) == pytest.approx(ref, rel=1e-12)


def test_mpo_site_definition_hand():
    """W of a single-spin site with left and up neighbours, by hand."""
    inst = I.square(2, 3)
    fg = tables.from_ising(inst)
    p = peps.build(fg, 0.5)
    st = p.site(1, 1)  # bottom-right: left and up edges, no right/down
    W = peps.mpo_site(st)
    assert W.shape == (2, 1, 2, 1)
    J_left = inst.J[[k for k in range(len(inst.J)) if (inst.ei[k], inst.ej[k]) == (2, 3)][0]]
    J_up = inst.J[[k for k in range(len(inst.J)) if (inst.ei[k], inst.ej[k]) == (1, 3)][0]]
    for l, u in itertools.product(range(2), range(2)):
        sl, su = 2 * l - 1, 2 * u - 1
        expect = 0.0
        for x in range(2):
            s = 2 * x - 1
            eL, eU = J_left * sl * s, J_up * su * s
            expect += np.exp(-0.5 * (eL - (-1.0))) * np.exp(-0.5 * (eU - (-1.0)))
        assert W[l, 0, u, 0] == pytest.approx(expect, rel=1e-14)


# ---------------------------------------------------------------- O6

def test_variational_sweeps_monotone_and_exact():
    inst = I.chimera(3, 11, couplings="gauss", h_sigma=0.1)
    p = peps.build(tables.from_ising(inst), 1.0)
    B2 = boundary.zipper(peps.mpo_row(p, 2), boundary.trivial_mps(3), 64)
    Ws = peps.mpo_row(p, 1)
    # truncating: fidelity never decreases and stays <= 1
    z = boundary.zipper(Ws, B2, 8)
    _, fid = boundary.variational(Ws, B2, z, 3)
    assert all(b >= a - 1e-12 for a, b in zip(fid, fid[1:]))
    assert all(f <= 1 + 1e-10 for f in fid)
    # no truncation: fidelity 1 and the state is a fixed point
    z = boundary.zipper(Ws, B2, 256)
    v, fid = boundary.variational(Ws, B2, z, 1)
    assert fid[-1] == pytest.approx(1.0, abs=1e-10)
    assert v.lognorm == pytest.approx(z.lognorm, abs=1e-10)


# ---------------------------------------------------------------- O7

@pytest.mark.parametrize("make,beta,chi,sites", [
    (lambda: I.square(4, 4, h_sigma=0.4), 0.9, 64, [0, 3, 5, 10, 15]),
    (lambda: I.chimera(1, 6, cols=3), 1.0, 256, [0, 1, 2]),
    (lambda: I.chimera(3, 6, cols=1, couplings="gauss", h_sigma=0.1), 1.5, 256, [1, 2]),
])
def test_marginals_vs_brute_force(make, beta, chi, sites):
    """Untruncated contraction: conditionals equal the exact ones."""
    inst = make()
    fg = tables.from_ising(inst)
    E = exact.all_energies(inst)
    cs = exact.cluster_states(inst.n_spins, fg.spins_of_site)
    rng = np.random.default_rng(1)
    prm = search.Params(beta=beta, chi=chi)
    for s in sites:
        prefixes = [rand_states(fg, rng)[:s] for _ in range(3)]
        got = search.debug_marginals(fg, prm, s, prefixes)
        for pre, g in zip(prefixes, got):
            ref = exact.exact_conditional(E, beta, inst.energy_shift, cs, s, pre, fg.d[s])
            np.testing.assert_allclose(g, ref, rtol=1e-10, atol=1e-10)


def test_marginals_uniform_at_beta_zero():
    inst = I.chimera(2, 1, couplings="gauss", h_sigma=0.1)
    fg = tables.from_ising(inst)
    got = search.debug_marginals(fg, search.Params(beta=0.0, chi=16), 3, [[5, 7, 200]])
    np.testing.assert_allclose(got[0], -np.log(256) * np.ones(256), atol=1e-12)


def test_z2_symmetry_first_site():
    """h = 0: flipping every spin is a symmetry, so p(x) = p(~x)."""
    inst = I.chimera(3, 2)
    fg = tables.from_ising(inst)
    got = search.debug_marginals(fg, search.Params(beta=1.0, chi=16), 0, [[]])[0]
    np.testing.assert_allclose(got, got[np.arange(256) ^ 255], rtol=1e-9)


# ---------------------------------------------------------------- O8 / O9 / O11

def test_search_exact_dp_square():
    """beam >= (#boundary keys) x d makes merging exact DP: ground state."""
    for seed in range(4):
        inst = I.square(4, 10 + seed, h_sigma=0.3)
        bf = exact.brute_force(inst, 1.0)
        res = search.solve(tables.from_ising(inst), search.Params(beta=1.0, chi=8, beam=32))
        assert res.energies[0] == bf["ground"]


def test_search_exact_dp_chimera_strip():
    inst = I.chimera(1, 4, cols=3)
    bf = exact.brute_force(inst, 1.0)
    fg = tables.from_ising(inst)
    res = search.solve(fg, search.Params(beta=1.0, chi=16, beam=256))
    assert res.energies.tolist() == [bf["ground"]]  # the empty final key merges all
    # without merging, the beam keeps max_states states to the end
    res = search.solve(fg, search.Params(beta=1.0, chi=16, beam=64, merge=False))
    assert len(res.energies) == 64 and res.energies[0] >= bf["ground"]
    E = exact.all_energies(inst)
    cs = exact.cluster_states(inst.n_spins, fg.spins_of_site)
    code = {tuple(int(c[k]) for c in cs): int(E[k]) for k in np.nonzero(E <= res.energies[-1])[0]}
    for e, st in zip(res.energies, res.states):
        assert code[tuple(int(v) for v in st)] == e


def test_search_output_order_and_energies():
    inst = I.chimera(2, 3, couplings="gauss", h_sigma=0.1)
    fg = tables.from_ising(inst)
    res = search.solve(fg, search.Params(beta=1.0, chi=16, beam=64))
    keys = [(int(e), tuple(s)) for e, s in zip(res.energies, res.states)]
    assert keys == sorted(keys)
    for e, s in zip(res.energies, res.states):
        assert e == tables.ising_energy(inst, tables.spins_from_states(fg, s, inst.n_spins))


def test_search_chimera_3x3_ground_state():
    """cfg: 3x3 Chimera +-1, beta 1, chi 16, beam 256 reaches the exact
    (min-plus transfer) ground energy on these seeds, never below it."""
    for seed in range(2):
        inst = I.chimera(3, seed)
        gs = exact.chimera_strip(inst, 1.0)["ground"]
        res = search.solve(tables.from_ising(inst), search.Params(beta=1.0, chi=16, beam=256))
        assert res.energies[0] >= gs
        assert res.energies[0] == gs


def test_gauge_flip_same_spectrum():
    """s_i -> -s_i on a spin set with the matching sign changes of J and h
    maps states bijectively and keeps every energy."""
    inst = I.chimera(2, 7, couplings="gauss", h_sigma=0.1)
    rng = np.random.default_rng(3)
    flip = rng.random(inst.n_spins) < 0.5
    g = I.IsingInstance(**{**inst.__dict__})
    g.J = np.where(flip[inst.ei] ^ flip[inst.ej], -inst.J, inst.J)
    g.h = np.where(flip, -inst.h, inst.h)
    fa, fb = tables.from_ising(inst), tables.from_ising(g)
    prm = search.Params(beta=1.0, chi=16, beam=64)
    ra, rb = search.solve(fa, prm), search.solve(fb, prm)
    np.testing.assert_array_equal(ra.energies, rb.energies)
    masks = [sum(int(flip[sp]) << k for k, sp in enumerate(spins)) for spins in fa.spins_of_site]
    mapped = sorted(tuple(int(x) ^ m for x, m in zip(st, masks)) for st in ra.states)
    assert mapped == sorted(tuple(int(x) for x in st) for st in rb.states)


def test_cut_off_prob_drops_improbable_children():
    inst = I.chimera(2, 5)
    fg = tables.from_ising(inst)
    a = search.solve(fg, search.Params(beta=1.0, chi=16, beam=256))
    b = search.solve(fg, search.Params(beta=1.0, chi=16, beam=256, cut_off_prob=1e-3))
    assert len(b.states) <= len(a.states)
    assert all(np.max(b.log_probs) - lp <= -np.log(1e-3) * len(fg.d) for lp in b.log_probs)


# ---------------------------------------------------------------- king's graph (diagonal couplings)

def _potts_brute(inst, beta):
    E, cs = exact.potts_all_energies(inst)
    u = 2.0 ** (-inst.energy_shift)
    return E, cs, exact.logsumexp(-beta * u * E.astype(np.float64))


@pytest.mark.parametrize("L,cols,d,seed,beta", [(2, 3, 3, 5, 0.7), (3, 3, 3, 1, 1.3), (3, 4, 2, 2, 0.5),
                                                (4, 3, 2, 3, 1.0)])
def test_king_potts_log_partition_brute_force(L, cols, d, seed, beta):
    """King's-graph Potts (all 8-neighbour edges): untruncated boundary MPSs
    give the exact log Z of Eq. 1."""
    inst = I.king_potts(L, d, seed, cols=cols)
    _, _, ref = _potts_brute(inst, beta)
    p = peps.build(tables.from_potts(inst), beta)
    assert boundary.log_partition(p, 512) == pytest.approx(ref, rel=1e-12)


def test_king_ising_example_shape_log_partition():
    """The paper's example shape and beta: 3x3 king's graph of 2-spin
    clusters (18 spins), beta 2, against Eq. 2 enumerated over all spins.
    No truncation happens (the value is the same at chi 64 and 1024); the
    SVDs carry an absolute error ~eps * s_1, which reaches weights 1e-7
    below the largest at beta 2, hence the looser bound there."""
    inst = I.king_ising(3, 3, 2, 4)
    for beta, rel in ((1.0, 1e-12), (2.0, 1e-9)):
        ref = exact.brute_force(inst, beta)["logZ"]
        p = peps.build(tables.from_ising(inst), beta)
        assert boundary.log_partition(p, 256) == pytest.approx(ref, rel=rel)


def test_king_diagonals_change_log_partition():
    """Dropping the diagonal tables changes Z: the pin above sees them."""
    inst = I.king_potts(3, 3, 7)
    keep = [k for k in range(len(inst.em))
            if abs(int(inst.em[k]) // 3 - int(inst.en[k]) // 3) + abs(int(inst.em[k]) % 3 - int(inst.en[k]) % 3) == 1]
    d = 3
    pair = np.concatenate([inst.pair_E[k * d * d:(k + 1) * d * d] for k in keep])
    sq = I.PottsInstance(inst.grid_rows, inst.grid_cols, inst.d, inst.local_E, inst.em[keep], inst.en[keep], pair,
                         inst.energy_shift, I.SQUARE)
    _, _, ref_sq = _potts_brute(sq, 1.0)
    _, _, ref_k = _potts_brute(inst, 1.0)
    assert abs(ref_sq - ref_k) > 1e-3
    p = peps.build(tables.from_potts(sq), 1.0)
    assert boundary.log_partition(p, 512) == pytest.approx(ref_sq, rel=1e-12)


@pytest.mark.parametrize("k", range(8))
def test_king_lattice_transforms_log_partition(k):
    """The 8 symmetries of the square grid map a king's graph onto itself
    and leave Z unchanged (rotations and reflections move diagonals onto
    anti-diagonals)."""
    inst = I.king_potts(3, 2, 11, cols=4)
    _, _, ref = _potts_brute(inst, 0.8)
    rows, cols = inst.grid_rows, inst.grid_cols
    # k < 4: rotate k times by 90 degrees, (i, j) -> (j, rows - 1 - i) on the
    # current grid; k >= 4: reflect j first
    R2, C2 = (rows, cols) if k % 2 == 0 else (cols, rows)
    new_of = {}
    for i in range(rows):
        for j in range(cols):
            a, b = i, j
            if k >= 4:
                b = cols - 1 - b  # reflect first
            for t in range(k % 4):
                a, b = b, ((rows if t % 2 == 0 else cols) - 1) - a
            new_of[i * cols + j] = a * C2 + b
    n = rows * cols
    d = int(inst.d[0])
    old_of = {v: u for u, v in new_of.items()}
    local = np.concatenate([inst.local_E[old_of[s] * d:(old_of[s] + 1) * d] for s in range(n)])
    em = np.array([new_of[int(v)] for v in inst.em], np.int32)
    en = np.array([new_of[int(v)] for v in inst.en], np.int32)
    t = I.PottsInstance(R2, C2, inst.d, local, em, en, inst.pair_E, inst.energy_shift, I.KING)
    p = peps.build(tables.from_potts(t), 0.8)
    assert boundary.log_partition(p, 512) == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("make,beta,sites", [
    (lambda: I.king_potts(3, 3, 21), 1.0, [0, 2, 3, 4, 5, 7, 8]),
    (lambda: I.king_potts(3, 2, 22, cols=4), 0.6, [1, 4, 5, 6, 9, 11]),
])
def test_king_marginals_vs_brute_force(make, beta, sites):
    """Untruncated contraction on a king's graph: the search's conditionals
    equal the exact conditionals of Eq. 1 for random prefixes."""
    inst = make()
    fg = tables.from_potts(inst)
    E, cs, _ = _potts_brute(inst, beta)
    rng = np.random.default_rng(3)
    prm = search.Params(beta=beta, chi=512)
    for s in sites:
        prefixes = [rand_states(fg, rng)[:s] for _ in range(3)]
        got = search.debug_marginals(fg, prm, s, prefixes)
        for pre, g in zip(prefixes, got):
            ref = exact.exact_conditional(E, beta, inst.energy_shift, cs, s, pre, fg.d[s])
            np.testing.assert_allclose(g, ref, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("seed", range(3))
def test_king_search_finds_brute_force_ground_state(seed):
    """Exact marginals and a beam wide enough to hold every merge class: the
    search returns the brute-force ground state and its energy."""
    inst = I.king_potts(3, 3, 30 + seed)
    fg = tables.from_potts(inst)
    E, cs, _ = _potts_brute(inst, 1.0)
    k = int(np.argmin(E))
    res = search.solve(fg, search.Params(beta=1.0, chi=512, beam=4096))
    assert int(res.energies[0]) == int(E.min())
    assert [int(v) for v in res.states[0]] == [int(c[k]) for c in cs]
    assert tables.energy(fg, res.states[0]) == int(E.min())


# ---------------------------------------------------------------- further pins of the zipper and the search


@pytest.mark.parametrize("L", [3, 4])
def test_truncation_error_falls_with_chi(L):
    """Width-3 Chimera against the exact spin-level transfer matrix: the
    zipper's log Z error decreases at every doubling of chi (1 .. 64) and is
    below 1e-5 at chi 64."""
    inst = I.chimera(L, 7, couplings="gauss", h_sigma=0.1, cols=3)
    ref = exact.chimera_strip(inst, 1.0)["logZ"]
    p = peps.build(tables.from_ising(inst), 1.0)
    errs = [abs(boundary.log_partition(p, chi) - ref) for chi in (1, 2, 4, 8, 16, 32, 64)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-5


def test_untruncated_zipper_reproduces_the_mpo_mps_product():
    """With chi at least the full bond, one zipper row is exactly W B: every
    amplitude of the resulting MPS (times exp(log-norm)) equals the product
    of the row MPO with the MPS below, contracted densely."""
    inst = I.chimera(3, 2, couplings="gauss", h_sigma=0.2, cols=3)
    p = peps.build(tables.from_ising(inst), 0.7)
    Bs = boundary.boundary_mpses(p, 10 ** 6, 0, down_to=1)
    Ws = peps.mpo_row(p, 1)
    B2, B1 = Bs[2], Bs[1]

    def dense(mps):
        T = np.ones((1, 1))  # [configurations, right bond]
        for A in mps.sites:
            a, s, b = A.shape
            T = np.einsum("ca,asb->csb", T, A).reshape(-1, b)
        return T[:, 0] * np.exp(mps.lognorm)

    # W B densely: contract each MPO site with the MPS site (bond pairs)
    T = np.ones((1, 1, 1))  # [configurations u, MPO bond, MPS bond]
    for W, A in zip(Ws, B2.sites):
        t = np.einsum("clb,lrus,bsd->curd", T, W, A)
        T = t.reshape(t.shape[0] * t.shape[1], t.shape[2], t.shape[3])
    exact_amps = T[:, 0, 0] * np.exp(B2.lognorm)
    np.testing.assert_allclose(dense(B1), exact_amps, rtol=1e-10, atol=1e-12 * np.max(np.abs(exact_amps)))


def test_sign_fix_gauge():
    """Every right singular vector comes out with its largest-magnitude entry
    (first on ties) positive, U V^T unchanged; the zipper's sites obey it."""
    rng = np.random.default_rng(5)
    M = rng.standard_normal((7, 9))
    U, S, Vt = np.linalg.svd(M, full_matrices=False)
    U2, Vt2 = boundary.sign_fix(U.copy(), Vt.copy())
    np.testing.assert_allclose((U2 * S) @ Vt2, M, atol=1e-12)
    for row in Vt2:
        assert row[np.argmax(np.abs(row))] > 0
    Vt3 = np.array([[0.5, -0.5, 0.1]])  # a tie: the first maximum decides
    _, Vt3 = boundary.sign_fix(np.ones((1, 1)), Vt3)
    assert Vt3[0, 0] == 0.5
    p = peps.build(tables.from_ising(I.chimera(3, 4, couplings="gauss", h_sigma=0.1)), 1.0)
    B = boundary.boundary_mpses(p, 8, 0, down_to=1)[1]
    for A in B.sites[1:]:
        for row in A.reshape(A.shape[0], -1):
            assert row[np.argmax(np.abs(row))] > 0


def test_degenerate_cut_is_flagged():
    """At beta = 0 every weight is 1, the zipper matrices have rank 1, and a
    cut below their dimensions falls between equal (zero) singular values:
    flagged; a generic instance at beta = 1 is not."""
    fg = tables.from_ising(I.chimera(3, 4, couplings="gauss", h_sigma=0.1))
    assert boundary.boundary_mpses(peps.build(fg, 0.0), 4)[1].degenerate
    assert not boundary.boundary_mpses(peps.build(fg, 1.0), 4)[1].degenerate


def test_near_tie_is_counted():
    """A single-spin lattice with h = 0 is Z2-symmetric: the two states of the
    first site are exactly equally probable, so a beam of 1 cuts between
    them and the prune records a near tie; a field makes the cut clear."""
    sym = I.square(2, 3, cols=2)
    r = search.solve(tables.from_ising(sym), search.Params(beta=1.0, chi=4, beam=1, merge=False))
    assert r.near_ties >= 1
    asym = I.square(2, 3, cols=2, h_sigma=2.0)
    r = search.solve(tables.from_ising(asym), search.Params(beta=1.0, chi=4, beam=1, merge=False))
    assert r.near_ties == 0 and r.min_cut_gap > 1e-6
