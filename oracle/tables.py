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
    E: np.ndarray  # int64 [d_m, d_n]  full table
    R: np.ndarray  # int64 [Dm, Dn]    reduced table
    Pm: np.ndarray  # int64 [d_m]      row projector of site m
    Pn: np.ndarray  # int64 [d_n]      column projector of site n


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


def project(E):
    """Distinct rows/columns of E in first-occurrence order (reading above)."""
    def dedupe(rows):
        index = {}
        P = np.empty(rows.shape[0], dtype=np.int64)
        for x in range(rows.shape[0]):
            key = rows[x].tobytes()
            if key not in index:
                index[key] = len(index)
            P[x] = index[key]
        return P, len(index)

    Pm, Dm = dedupe(E)
    Pn, Dn = dedupe(E.T.copy())
    first_m = np.array([int(np.argmax(Pm == a)) for a in range(Dm)])
    first_n = np.array([int(np.argmax(Pn == b)) for b in range(Dn)])
    R = E[np.ix_(first_m, first_n)]
    return R, Pm, Pn


def adjacent(node_type, rm, cm, rn, cn):
    dr, dc = abs(rm - rn), abs(cm - cn)
    if node_type == SQUARE:
        return dr + dc == 1
    return max(dr, dc) == 1


def from_ising(inst) -> FactorGraph:
    """Eq. 2 -> Eq. 1: clusters of spins become Potts variables."""
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
    S = [spins_of_state(len(sp)) for sp in spins_of_site]
    d = [2 ** len(sp) for sp in spins_of_site]

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
        E += int(e.E[x[m], x[n]])
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
