"""Cluster factor graph: integer local and pairwise energy tables + projectors.

Test infrastructure only (see the package header).

Paper: Eq. 1 (generalized Potts energy on a graph of clusters), Eq. 2 (Ising
form, s in {-1,+1}), Sec. 2 (clusters of spins become Potts variables with
2^k states), Sec. 3.1 (``spectrum = full_spectrum``: every cluster state is
enumerated; ``Sparsity``: pairwise interactions act through the internal
structure of a cluster, i.e. through projections of its state).

Readings taken here:
* spin value s = 2b - 1 for the stored bit b; a cluster of spins
  sp[0] < sp[1] < ... (ascending spin index) has state x = sum_k b_k 2^k;
* energies are integers in units of 2**-energy_shift; an input value off that
  grid is rejected;
* intra-cluster couplings and fields go to the cluster's local table, every
  other coupling to the table of the (unordered) cluster pair, stored with
  the row-major-first site as the row variable;
* projector of a pairwise table E_e: P_row[x] = index of row x among the
  distinct rows of E_e numbered in order of first occurrence (x ascending);
  P_col likewise for columns.  The reduced table R_e satisfies
  E_e[x, y] == R_e[P_row[x], P_col[y]] for all x, y.

``Sparsity`` (Sec. 3.1, Sec. 3.1.1: clusters of O(10-20) spins, Pegasus'
24 and Zephyr's 16, for which explicit tensors are infeasible): a sparse
edge never forms the d_m x d_n table.  The couplers of the edge touch only
some spins of each cluster (positions ``pos_m`` in m, ``pos_n`` in n); the
table is a function of those spins' configurations,
E_e[x, y] = Esub[sub_m[x], sub_n[y]], with sub_m[x] = sum_k b_{pos_m[k]}(x) 2^k.
Every configuration of the coupled spins occurs, so two states have equal
rows of E_e exactly when their rows of Esub are equal, and the first state
carrying a given configuration a (only a's spins set) grows with a: the
projectors and the reduced table computed over the configurations a of the
coupled spins are those of the full table (first-occurrence order
included).  ``from_ising`` builds sparse edges for clusters of more than 8
spins, or on request.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SQUARE = 0
KING = 1


class InexactEnergy(ValueError):
    pass


@dataclass
class Edge:
    m: int  # row-major-first site
    n: int
    E: np.ndarray  # int64 [d_m, d_n]  full table (None on a sparse edge)
    R: np.ndarray  # int64 [Dm, Dn]    reduced table
    Pm: np.ndarray  # int64 [d_m]      row projector of site m
    Pn: np.ndarray  # int64 [d_n]      column projector of site n
    # sparse edge (module header): E[x, y] = Esub[sub_m[x], sub_n[y]]
    Esub: np.ndarray = None  # int64 [2^len(pos_m), 2^len(pos_n)]
    pos_m: np.ndarray = None  # positions of the coupled spins in cluster m (ascending)
    pos_n: np.ndarray = None
    sub_m: np.ndarray = None  # int64 [d_m]
    sub_n: np.ndarray = None  # int64 [d_n]

    def value(self, xm, xn) -> int:
        """E[xm, xn]."""
        if self.E is not None:
            return int(self.E[xm, xn])
        return int(self.Esub[self.sub_m[xm], self.sub_n[xn]])

    def min(self) -> int:
        """min over all (xm, xn) of E (every coupled configuration occurs)."""
        return int(self.E.min()) if self.E is not None else int(self.Esub.min())

    def block(self, row_site: int, rs, cs) -> np.ndarray:
        """The table seen from row_site (m: E, n: E^T) at states rs x cs."""
        rs, cs = np.asarray(rs), np.asarray(cs)
        if self.E is not None:
            T = self.E if row_site == self.m else self.E.T
            return T[np.ix_(rs, cs)]
        if row_site == self.m:
            return self.Esub[np.ix_(self.sub_m[rs], self.sub_n[cs])]
        return self.Esub.T[np.ix_(self.sub_n[rs], self.sub_m[cs])]


@dataclass
class FactorGraph:
    rows: int
    cols: int
    d: list  # states per site
    E_loc: list  # int64 [d_s] per site
    edges: dict  # (m, n) -> Edge
    shift: int
    node_type: int
    spins_of_site: list = field(default_factory=list)  # Ising form only
    sparse: bool = False  # Sparsity = Sparse: sparse edges, sites built by projection classes

    @property
    def n_sites(self):
        return self.rows * self.cols

    def edge(self, m, n):
        return self.edges.get((m, n))


def _to_int(values, shift):
    v = np.asarray(values, dtype=np.float64) * (2.0 ** shift)
    r = np.round(v)
    if not np.all(r == v):
        raise InexactEnergy("value not on the 2**-shift grid")
    if np.any(np.abs(r) >= 2.0 ** 52):
        raise InexactEnergy("value too large for exact integer energies")
    return r.astype(np.int64)


def spins_of_state(k):
    """[2^k, k] spin values s = 2b-1 of every state of a k-spin cluster."""
    x = np.arange(2 ** k, dtype=np.int64)[:, None]
    b = (x >> np.arange(k, dtype=np.int64)[None, :]) & 1
    return 2 * b - 1


def _dedupe(rows):
    """First-occurrence class of every row of ``rows`` and the class count."""
    index = {}
    P = np.empty(rows.shape[0], dtype=np.int64)
    for x in range(rows.shape[0]):
        key = np.ascontiguousarray(rows[x]).tobytes()
        if key not in index:
            index[key] = len(index)
        P[x] = index[key]
    return P, len(index)


def project(E):
    """Distinct rows/columns of E in first-occurrence order (reading above)."""
    Pm, Dm = _dedupe(E)
    Pn, Dn = _dedupe(E.T.copy())
    first_m = np.array([int(np.argmax(Pm == a)) for a in range(Dm)])
    first_n = np.array([int(np.argmax(Pn == b)) for b in range(Dn)])
    R = E[np.ix_(first_m, first_n)]
    return R, Pm, Pn


def sub_index(x, pos):
    """Configuration index of the spins at positions ``pos`` in states x:
    sum_k bit pos[k] of x, times 2^k."""
    x = np.asarray(x, dtype=np.int64)
    out = np.zeros_like(x)
    for k, q in enumerate(pos):
        out |= ((x >> int(q)) & 1) << k
    return out


def project_sparse(Esub, sub_m, sub_n):
    """``project`` of the full table Esub[sub_m[x], sub_n[y]] computed on the
    coupled configurations (module header): classes of the rows (columns) of
    Esub in order of a (b) ascending, which is their order of first
    occurrence over x (y) ascending."""
    cm, Dm = _dedupe(Esub)
    cn, Dn = _dedupe(Esub.T.copy())
    first_a = np.array([int(np.argmax(cm == c)) for c in range(Dm)])
    first_b = np.array([int(np.argmax(cn == c)) for c in range(Dn)])
    return Esub[np.ix_(first_a, first_b)], cm[sub_m], cn[sub_n]


def adjacent(node_type, rm, cm, rn, cn):
    dr, dc = abs(rm - rn), abs(cm - cn)
    if node_type == SQUARE:
        return dr + dc == 1
    return max(dr, dc) == 1


def from_ising(inst, sparse=None) -> FactorGraph:
    """Eq. 2 -> Eq. 1: clusters of spins become Potts variables.  sparse:
    True / False, or None for sparse edges when a cluster has more than 8
    spins (module header)."""
    rows, cols = inst.grid_rows, inst.grid_cols
    shift = inst.energy_shift
    n_sites = rows * cols
    if len(inst.cluster_row) != n_sites:
        raise ValueError("one cluster per grid cell is required")
    site_of_cluster = np.asarray(inst.cluster_row) * cols + np.asarray(inst.cluster_col)
    if len(set(site_of_cluster.tolist())) != n_sites:
        raise ValueError("two clusters on one grid cell")
    site_of_spin = site_of_cluster[np.asarray(inst.cluster_of_spin)]
    J = _to_int(inst.J, shift)
    h = _to_int(inst.h, shift)
    spins_of_site = [np.sort(np.nonzero(site_of_spin == s)[0]) for s in range(n_sites)]
    pos_in_site = np.empty(inst.n_spins, dtype=np.int64)
    for s in range(n_sites):
        pos_in_site[spins_of_site[s]] = np.arange(len(spins_of_site[s]))
    d = [2 ** len(sp) for sp in spins_of_site]
    if sparse is None:
        sparse = max(len(sp) for sp in spins_of_site) > 8
    if sparse:
        return _from_ising_sparse(inst, rows, cols, shift, J, h, site_of_spin, spins_of_site, pos_in_site, d)
    S = [spins_of_state(len(sp)) for sp in spins_of_site]

    E_loc = [S[s] @ h[spins_of_site[s]] for s in range(n_sites)]
    pair = {}
    for e in range(len(J)):
        i, j = int(inst.ei[e]), int(inst.ej[e])
        si, sj = int(site_of_spin[i]), int(site_of_spin[j])
        if si == sj:
            E_loc[si] = E_loc[si] + J[e] * S[si][:, pos_in_site[i]] * S[si][:, pos_in_site[j]]
            continue
        if si > sj:
            si, sj, i, j = sj, si, j, i
        rm, cm, rn, cn = si // cols, si % cols, sj // cols, sj % cols
        if not adjacent(inst.node_type, rm, cm, rn, cn):
            raise ValueError(f"coupling between non-neighbouring clusters {si} {sj}")
        T = pair.setdefault((si, sj), np.zeros((d[si], d[sj]), dtype=np.int64))
        T += J[e] * np.outer(S[si][:, pos_in_site[i]], S[sj][:, pos_in_site[j]])
    edges = {}
    for (m, n), E in sorted(pair.items()):
        R, Pm, Pn = project(E)
        edges[(m, n)] = Edge(m, n, E, R, Pm, Pn)
    return FactorGraph(rows, cols, d, [np.asarray(t, dtype=np.int64) for t in E_loc], edges,
                       shift, inst.node_type, spins_of_site)


def _spin_column(n_states, pos):
    """Spin s = 2b - 1 at position pos of every state 0 .. n_states-1."""
    return 2 * ((np.arange(n_states, dtype=np.int64) >> int(pos)) & 1) - 1


def _from_ising_sparse(inst, rows, cols, shift, J, h, site_of_spin, spins_of_site, pos_in_site, d):
    """``from_ising`` with sparse edges: local tables over every state of a
    cluster, pairwise tables over the configurations of the coupled spins."""
    n_sites = rows * cols
    E_loc = []
    xs = [np.arange(d[s], dtype=np.int32) for s in range(n_sites)]  # states (clusters of <= 30 spins)
    for s in range(n_sites):
        E = np.zeros(d[s], dtype=np.int64)
        for q, spin in enumerate(spins_of_site[s]):
            if h[spin] != 0:
                E += h[spin] * (2 * ((xs[s] >> q) & 1) - 1)
        E_loc.append(E)
    couplers = {}
    for e in range(len(J)):
        i, j = int(inst.ei[e]), int(inst.ej[e])
        si, sj = int(site_of_spin[i]), int(site_of_spin[j])
        if si == sj:
            # s_i s_j = +1 when the two bits agree, -1 otherwise
            p, q = int(pos_in_site[i]), int(pos_in_site[j])
            E_loc[si] += J[e] * (1 - 2 * (((xs[si] >> p) ^ (xs[si] >> q)) & 1))
            continue
        if si > sj:
            si, sj, i, j = sj, si, j, i
        if not adjacent(inst.node_type, si // cols, si % cols, sj // cols, sj % cols):
            raise ValueError(f"coupling between non-neighbouring clusters {si} {sj}")
        couplers.setdefault((si, sj), []).append((int(pos_in_site[i]), int(pos_in_site[j]), int(J[e])))
    edges = {}
    for (m, n), cl in sorted(couplers.items()):
        pos_m = np.array(sorted({a for a, _, _ in cl}), dtype=np.int64)
        pos_n = np.array(sorted({b for _, b, _ in cl}), dtype=np.int64)
        A, B = 2 ** len(pos_m), 2 ** len(pos_n)
        Esub = np.zeros((A, B), dtype=np.int64)
        for a, b, Jv in cl:
            ka, kb = int(np.searchsorted(pos_m, a)), int(np.searchsorted(pos_n, b))
            Esub += Jv * np.outer(_spin_column(A, ka), _spin_column(B, kb))
        sub_m = sub_index(np.arange(d[m]), pos_m)
        sub_n = sub_index(np.arange(d[n]), pos_n)
        R, Pm, Pn = project_sparse(Esub, sub_m, sub_n)
        edges[(m, n)] = Edge(m, n, None, R, Pm, Pn, Esub, pos_m, pos_n, sub_m, sub_n)
    return FactorGraph(rows, cols, d, E_loc, edges, shift, inst.node_type, spins_of_site, sparse=True)


def from_potts(inst) -> FactorGraph:
    """Eq. 1 given directly as tables (Potts form)."""
    rows, cols = inst.grid_rows, inst.grid_cols
    n_sites = rows * cols
    d = [int(v) for v in inst.d]
    offs = np.concatenate([[0], np.cumsum(d)])
    E_loc = [np.asarray(inst.local_E[offs[s]:offs[s + 1]], dtype=np.int64).copy() for s in range(n_sites)]
    pair = {}
    off = 0
    for k in range(len(inst.em)):
        m, n = int(inst.em[k]), int(inst.en[k])
        T = np.asarray(inst.pair_E[off:off + d[m] * d[n]], dtype=np.int64).reshape(d[m], d[n])
        off += d[m] * d[n]
        if m > n:
            m, n, T = n, m, T.T
        if not adjacent(inst.node_type, m // cols, m % cols, n // cols, n % cols):
            raise ValueError("pairwise table between non-neighbouring sites")
        acc = pair.setdefault((m, n), np.zeros((d[m], d[n]), dtype=np.int64))
        acc += T
    edges = {}
    for (m, n), E in sorted(pair.items()):
        R, Pm, Pn = project(E)
        edges[(m, n)] = Edge(m, n, E, R, Pm, Pn)
    return FactorGraph(rows, cols, d, E_loc, edges, inst.energy_shift, inst.node_type)


def energy(fg: FactorGraph, x) -> int:
    """Eq. 1 from the tables: sum of local terms and of pairwise terms."""
    x = [int(v) for v in x]
    E = sum(int(fg.E_loc[s][x[s]]) for s in range(fg.n_sites))
    for (m, n), e in fg.edges.items():
        E += e.value(x[m], x[n])
    return E


def energy_reduced(fg: FactorGraph, x) -> int:
    """Eq. 1 through reduced tables and projectors (must equal ``energy``)."""
    x = [int(v) for v in x]
    E = sum(int(fg.E_loc[s][x[s]]) for s in range(fg.n_sites))
    for (m, n), e in fg.edges.items():
        E += int(e.R[e.Pm[x[m]], e.Pn[x[n]]])
    return E


def ising_energy(inst, s) -> int:
    """Eq. 2 directly on spins s in {-1,+1}, integer units of 2**-shift."""
    J = _to_int(inst.J, inst.energy_shift)
    h = _to_int(inst.h, inst.energy_shift)
    s = np.asarray(s, dtype=np.int64)
    return int(np.sum(J * s[inst.ei] * s[inst.ej]) + np.sum(h * s))


def spins_from_states(fg: FactorGraph, x, n_spins):
    """Decode cluster states into spins (s = 2b-1, bit k = spin sp[k])."""
    s = np.zeros(n_spins, dtype=np.int64)
    for site, sp in enumerate(fg.spins_of_site):
        bits = (int(x[site]) >> np.arange(len(sp))) & 1
        s[sp] = 2 * bits - 1
    return s
