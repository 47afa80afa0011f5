"""The oracle's C brute force (oracle/bruteforce.c, OpenMP) against the NumPy
enumeration of exact.brute_force: the same ground energy and degeneracy
(exact integers) and log Z, on Chimera (Gaussian J and fields), square,
king's and large-cell instances of 16 to 20 spins."""
import numpy as np
import pytest

import instances as I
from oracle import exact


@pytest.mark.parametrize("make,beta", [
    (lambda: I.chimera(2, 3, couplings="gauss", h_sigma=0.1, cols=1), 0.7),
    (lambda: I.square(4, 6, h_sigma=0.3), 1.3),
    (lambda: I.king_ising(2, 2, 4, 1), 0.5),
    (lambda: I.large_cells(1, 2, 10, 5, links=3, intra="ring"), 2.0),
])
def test_c_brute_force_equals_numpy(make, beta):
    inst = make()
    c = exact.brute_force_c(inst, beta)
    ref = exact.brute_force(inst, beta)
    assert c["ground"] == ref["ground"]
    assert c["degeneracy"] == ref["degeneracy"]
    assert abs(c["logZ"] - ref["logZ"]) <= 1e-11 * max(1.0, abs(ref["logZ"]))


def test_c_brute_force_refuses_too_many_spins():
    inst = I.large_cells(1, 2, 16, 1)  # 32 spins
    with pytest.raises(ValueError):
        exact.brute_force_c(inst, 1.0)


def test_king_graph_beyond_the_numpy_enumeration():
    """27 spins (3 x 3 king's graph, 3 spins per cluster, every spin of a
    cluster coupled to every spin of its 8 neighbours): the oracle's log Z
    at an untruncated bond dimension, and the ground energy of its search in
    the exact limit (merging, beam >= boundary keys x states = 8^4 x 8),
    equal the C brute force."""
    from oracle import boundary, peps, search, tables
    inst = I.king_ising(3, 3, 3, 12)
    beta = 0.6
    fg = tables.from_ising(inst)
    p = peps.build(fg, beta)
    B0 = boundary.boundary_mpses(p, 4096, 0, down_to=0)[0]
    log_z = B0.lognorm + float(np.log(boundary.contract_value(B0))) + p.log_offset
    ref = exact.brute_force_c(inst, beta)
    assert abs(log_z - ref["logZ"]) <= 1e-9 * abs(ref["logZ"])
    res = search.solve(fg, search.Params(beta=beta, chi=4096, beam=8 ** 4 * 8))
    assert int(res.energies[0]) == ref["ground"]
