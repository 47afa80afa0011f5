"""The library's clustered Hamiltonian (spg_potts_hamiltonian, host only: the
paper's potts_hamiltonian, Sec. 2 Eq. 1-2, Sec. 3.1 Sparsity, Sec. 3.1.1
large clusters) against the oracle's tables, bit for bit, on the CPU: local
tables, the set of edges, reduced tables and projectors, for Chimera cells
(dense oracle tables) and for cells of 16 (Zephyr) and 24 (Pegasus) spins
(sparse oracle tables); and the refusals of inputs outside its limits."""
import numpy as np
import pytest

import instances as I
from oracle import peps, tables

CASES = {
    "chimera_pm1": lambda: I.chimera(3, 1),
    "chimera_gauss": lambda: I.chimera(3, 2, couplings="gauss", h_sigma=0.1),
    "king_ising": lambda: I.king_ising(3, 3, 2, 5),
    "cells8_king": lambda: I.large_cells(2, 2, 8, 3),
    "cells16_king": lambda: I.large_cells(2, 2, 16, 21, links=3),
    "cells16_square": lambda: I.large_cells(2, 3, 16, 23, links=2, node_type=I.SQUARE),
    "cells24_ring": lambda: I.large_cells(1, 2, 24, 22, links=3, intra="ring"),
}


@pytest.mark.parametrize("name", list(CASES))
def test_hamiltonian_equals_the_oracle_tables(name):
    import paper_2502_02317_gb300 as spg
    inst = CASES[name]()
    H = spg.spg_potts_hamiltonian(inst)
    fg = tables.from_ising(inst)
    assert len(H.E_loc) == fg.n_sites
    for s in range(fg.n_sites):
        np.testing.assert_array_equal(H.E_loc[s], fg.E_loc[s])
    assert sorted(H.edges) == sorted(fg.edges)
    for k, e in fg.edges.items():
        R, Pm, Pn = H.edges[k]
        np.testing.assert_array_equal(R, e.R)
        np.testing.assert_array_equal(Pm, e.Pm)
        np.testing.assert_array_equal(Pn, e.Pn)


@pytest.mark.parametrize("name", [n for n in CASES if n != "cells24_ring"])
def test_site_classes_and_class_weights_give_the_oracle_site_tensors(name):
    """The joint projections of every site equal the oracle's PEPS site data
    (classes and representatives), and the site tensor rebuilt from the
    library's class weights, W[l, (a', g'), u, d] = b_ad[a, u] [g' = P_G(u)]
    sum_{h, v} b_left[l, h] b_up[u, v] C[h, v, a', d] with the oracle's
    Boltzmann factors, equals the oracle's W."""
    import paper_2502_02317_gb300 as spg
    inst = CASES[name]()
    beta = 0.8
    H = spg.spg_potts_hamiltonian(inst)
    p = peps.build(tables.from_ising(inst), beta)
    for s, st in enumerate(p.sites):
        for which, field in ((H.L, "PL"), (H.U, "PU"), (H.R, "PR"), (H.D, "PD"), (H.G, "PG")):
            P, reps = H.classes(s, which)
            np.testing.assert_array_equal(P, getattr(st, field))
            assert len(reps) == int(P.max()) + 1 and np.array_equal(P[reps], np.arange(len(reps)))
            if field in ("PR", "PD"):
                np.testing.assert_array_equal(reps, st.repR if field == "PR" else st.repD)
        Cw = H.class_weights(s, beta)
        T = np.einsum("lh,uv,hvrd->lurd", st.b_left, st.b_up, Cw)
        W = np.zeros((st.DL, st.DR, st.DU, st.ND))
        a = np.arange(st.DL) // st.Gin
        for u in range(st.DU):
            cols = np.arange(st.NR) * st.Gout + int(st.g_of_u[u])
            W[:, cols, u, :] = st.b_ad[a, u][:, None, None] * T[:, u, :, :]
        ref = peps.mpo_site(st)
        np.testing.assert_allclose(W, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


def _row_of_cells(k, couplers, J=1.0, cols=2, col_of_cell=None):
    """Cells of k spins on a 1 x cols grid (cell c on column col_of_cell[c]);
    couplers (c, a, c', b) between spin a of cell c and spin b of cell c'."""
    col_of_cell = list(range(cols)) if col_of_cell is None else col_of_cell
    n = len(col_of_cell)
    ei = np.array([c * k + a for c, a, _, _ in couplers], np.int32)
    ej = np.array([c2 * k + b for _, _, c2, b in couplers], np.int32)
    return I.IsingInstance(n * k, ei, ej, np.full(len(couplers), J), np.zeros(n * k),
                           np.repeat(np.arange(n, dtype=np.int32), k), 1, cols, np.zeros(n, np.int32),
                           np.array(col_of_cell, np.int32), 0, I.KING)


def test_hamiltonian_refusals():
    import paper_2502_02317_gb300 as spg

    def code(inst):
        with pytest.raises(spg.SpgError) as e:
            spg.spg_potts_hamiltonian(inst)
        return e.value.code

    # 26 spins in one cluster: beyond SPG_MAX_HAMILTONIAN_SPINS (refused before allocating 2^26 states)
    assert code(_row_of_cells(26, [(0, 0, 1, 0)])) == spg.SPG_EUNSUPPORTED
    # 13 coupled spins on each side of one edge: beyond SPG_MAX_HAMILTONIAN_COUPLED
    assert code(_row_of_cells(14, [(0, q, 1, q) for q in range(13)])) == spg.SPG_EUNSUPPORTED
    # J off the 2^-shift grid
    assert code(_row_of_cells(4, [(0, 0, 1, 0)], J=0.3)) == spg.SPG_EINEXACT
    # cells on columns 0 and 2 are not grid neighbours
    assert code(_row_of_cells(4, [(0, 0, 1, 0)], cols=3, col_of_cell=[0, 2, 1])) == spg.SPG_EINVAL
    # two clusters on one grid cell
    assert code(_row_of_cells(4, [(0, 0, 1, 0)], col_of_cell=[0, 0])) == spg.SPG_EINVAL
    # within the limits the same shapes build
    assert len(spg.spg_potts_hamiltonian(_row_of_cells(12, [(0, q, 1, q) for q in range(12)])).edges) == 1


@pytest.mark.parametrize("name", ["chimera_pm1", "king_ising", "cells8_king", "cells16_king", "cells16_square"])
def test_site_tensors_equal_the_oracle_site_tensors(name):
    import paper_2502_02317_gb300 as spg
    inst = CASES[name]()
    H = spg.spg_potts_hamiltonian(inst)
    p = peps.build(tables.from_ising(inst), 0.8)
    for s, st in enumerate(p.sites):
        ref = peps.mpo_site(st)
        W = H.site_tensor(s, 0.8)
        assert W.shape == ref.shape == (st.DL, st.DR, st.DU, st.ND)
        np.testing.assert_allclose(W, ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


def _contract(Ws, rows, cols):
    """Z of the network of site tensors W[l][r][u][d] (plain einsum over every
    shared bond; the boundary bonds have dimension 1)."""
    letters = iter("abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ")
    hb = {(i, j): next(letters) for i in range(rows) for j in range(cols + 1)}
    vb = {(i, j): next(letters) for i in range(rows + 1) for j in range(cols)}
    terms = [f"{hb[i, j]}{hb[i, j + 1]}{vb[i, j]}{vb[i + 1, j]}" for i in range(rows) for j in range(cols)]
    return float(np.einsum(",".join(terms) + "->", *Ws))


@pytest.mark.parametrize("rows,cols,links,node", [(1, 3, 2, I.KING), (2, 2, 1, I.KING), (2, 2, 2, I.SQUARE)])
def test_site_tensors_of_zephyr_size_cells_give_the_exact_log_z(rows, cols, links, node):
    """16-spin cells: the network of the library's site tensors, contracted
    exactly, with the tables' minima added back, gives the log Z of
    exact.interface_sum (a sum over the interface spins' configurations
    written from Eq. 2; no oracle tables, tensors or MPSs)."""
    import paper_2502_02317_gb300 as spg
    from oracle import exact
    inst = I.large_cells(rows, cols, 16, 60 + rows * 10 + links, links=links, node_type=node)
    beta = 0.5
    H = spg.spg_potts_hamiltonian(inst)
    Ws = [H.site_tensor(s, beta) for s in range(rows * cols)]
    shift = sum(int(E.min()) for E in H.E_loc) + sum(int(R.min()) for R, _, _ in H.edges.values())
    log_z = np.log(_contract(Ws, rows, cols)) - beta * shift
    ref = exact.interface_sum(inst, beta)["logZ"]
    assert abs(log_z - ref) <= 1e-10 * abs(ref)


def test_projection_over_too_many_interface_spins_is_refused():
    """Site (0, 1) of a 2 x 3 king's grid of 22-spin cells couples 7 of its
    spins to each cell below: its P_D spans 21 interface spins (beyond 20)."""
    import paper_2502_02317_gb300 as spg
    k = 22
    ei, ej = [], []
    for t, col in enumerate((0, 1, 2)):
        for q in range(7):
            ei.append(k * 1 + 7 * t + q)        # cell (0, 1)
            ej.append(k * (3 + col))            # spin 0 of cell (1, col)
    n = 6 * k
    inst = I.IsingInstance(n, np.array(ei, np.int32), np.array(ej, np.int32), np.ones(len(ei)), np.zeros(n),
                           np.repeat(np.arange(6, dtype=np.int32), k), 2, 3,
                           np.array([0, 0, 0, 1, 1, 1], np.int32), np.array([0, 1, 2, 0, 1, 2], np.int32), 0,
                           I.KING)
    H = spg.spg_potts_hamiltonian(inst)
    assert len(H.edges) == 3
    with pytest.raises(spg.SpgError) as e:
        H.classes(1, H.D)
    assert e.value.code == spg.SPG_EUNSUPPORTED
    P, reps = H.classes(1, H.L)  # no edge on the left: one class
    assert len(reps) == 1 and not P.any()

