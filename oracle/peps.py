"""Boltzmann weights and the row MPOs of the PEPS (square and king's lattices).

Test infrastructure only (see the package header).

Paper: Sec. 2 and Fig. 1(b)-(c): the Boltzmann distribution p(x) ~
exp(-beta E(x)) of the clustered Potts model on a king's graph (square
lattice of clusters, with or without the two diagonal couplings of every
plaquette) is a PEPS on the square lattice of clusters; Sec. 3.1
(``PEPSNetwork{KingSingleNode, ...}``, ``Sparsity``): a site tensor is built
from the local weights of the cluster and from the pairwise interactions,
which reach the cluster only through projections of its state.

Readings taken here (the paper gives no formula for the site tensors):
* weights are shifted by the minimum of each table so that every weight is
  <= 1: w_s(x) = exp(-beta u (E_s(x) - min E_s)), b_e = exp(-beta u
  (E_e - min E_e)), u = 2**-energy_shift; the shifts add back into log Z;
* a projection of cluster (i, j) onto a set of its edges numbers the distinct
  combinations of table rows (x as the table's row variable) or columns (x as
  its column variable) of those edges in order of first occurrence, x
  ascending; an empty set gives the single class 0.  The classes used:
      P_L(x): edges to (i, j-1) and (i-1, j-1)        (left, up-left)
      P_U(x): edge to (i-1, j)                         (up)
      P_R(x): edges to (i, j+1) and (i-1, j+1)        (right, up-right)
      P_D(x): edges to (i+1, j-1), (i+1, j), (i+1, j+1) (everything below)
      P_G(x): edge to (i+1, j+1)                       (down-right)
  On the square lattice P_L, P_U, P_R, P_D are the projections of the single
  left, up, right and down edges and P_G has one class;
* the physical index of the boundary MPS below row i-1 at column j is P_D of
  cluster (i-1, j), so every edge between rows i-1 and i is carried in the
  tensors of row i: the up and up-left edges by b_up and b_left below, the
  up-right edge (i-1, j+1)-(i, j) by site (i, j+1), which sees the P_R
  class a of (i, j) on its left bond and the P_D class u of (i-1, j+1)
  above;
* the horizontal bond between columns j-1 and j of row i is the pair
  l = (a, g) = a * G + g: a the P_R class of (i, j-1), g the P_G class of
  (i-1, j-1) (G classes; g carries the up-left edge of (i, j));
* the MPO of row i maps the up index u (P_D class of cluster (i-1, j)) to the
  down index s (P_D class of cluster (i, j)):
      W[(a, g), (a', g'), u, s] = b_ad[a, u] [g' == P_G(u)]
          sum_x w(x) b_left[(a, g), P_L x] b_up[u, P_U x] [a' == P_R x] [s == P_D x]
  with b_left[(a, g), h] the product of the Boltzmann factors of the left and
  up-left edges between class representatives (first states of the
  classes), b_up the up edge's, b_ad the up-right edge's of the left
  neighbour, and P_G(u) the down-right class of the upper cluster's states
  in class u.  Row 0 has u of dimension 1, the last row s of dimension 1.

``Sparsity = Sparse`` (Sec. 3.1; factor graphs with sparse edges, see
``tables``): no pairwise table of the cluster is formed.  A projection of
cluster s onto a set of edges is a function of the configuration of the
union U of the spins those edges couple (its "interface"), so its classes
are found over the 2^|U| interface configurations (first occurrence over
them in ascending order is first occurrence over the states, as for a
single edge) and read off for every state; and the site tensor W is formed
as the sum of the states' terms grouped by their output indices (r, s),
which never builds the one-hot state map of the dense construction.  Both
constructions give the same classes, representatives and W (up to the
summation order of the sums over states).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .tables import FactorGraph


def classes(d: int, vectors: list):
    """First-occurrence classes of x in range(d) by the tuple of vectors[k][x]
    (each an array [d, n_k]); returns (P [d], representatives [n_classes])."""
    index, P, reps = {}, np.empty(d, dtype=np.int64), []
    for x in range(d):
        key = b"".join(np.ascontiguousarray(v[x]).tobytes() for v in vectors)
        if key not in index:
            index[key] = len(index)
            reps.append(x)
        P[x] = index[key]
    return P, np.array(reps, dtype=np.int64)


@dataclass
class SiteData:
    d: int
    E: np.ndarray  # int64 [d] local table
    w: np.ndarray  # float64 [d] shifted local weights
    PL: np.ndarray
    PU: np.ndarray
    PR: np.ndarray
    PD: np.ndarray
    PG: np.ndarray
    repR: np.ndarray  # first state of each P_R class
    repD: np.ndarray  # first state of each P_D class
    NL: int
    NU: int
    NR: int
    ND: int
    NG: int
    DL: int  # left bond = NR(i, j-1) * NG(i-1, j-1)
    DR: int  # right bond = NR(i, j) * NG(i-1, j)
    DU: int  # up index = ND(i-1, j)
    Gin: int  # NG(i-1, j-1): the g range of the left bond
    Gout: int  # NG(i-1, j): the g range of the right bond
    b_left: np.ndarray  # [DL, NL]
    b_up: np.ndarray  # [DU, NU]
    b_ad: np.ndarray  # [NR(i, j-1), DU]
    g_of_u: np.ndarray  # [DU] P_G class of the upper cluster's P_D class u
    sparse: bool = False  # W built by grouping the states' terms (module header)


@dataclass
class PEPS:
    fg: FactorGraph
    beta: float
    sites: list
    log_offset: float  # log Z = log Z(shifted weights) + log_offset

    @property
    def rows(self):
        return self.fg.rows

    @property
    def cols(self):
        return self.fg.cols

    def site(self, i, j) -> SiteData:
        return self.sites[i * self.fg.cols + j]


def _incident(fg: FactorGraph, s: int, t: int):
    """Table rows of cluster s on the edge to cluster t ([d_s, d_t]), or None."""
    e = fg.edge(min(s, t), max(s, t))
    if e is None:
        return None
    return e.E if s < t else e.E.T


def _class_of(fg: FactorGraph, s: int, nbrs: list):
    if fg.sparse:
        return _class_of_sparse(fg, s, nbrs)
    vecs = []
    for t in nbrs:
        if t is None:
            continue
        T = _incident(fg, s, t)
        if T is not None:
            vecs.append(T)
    return classes(fg.d[s], vecs)


def _class_of_sparse(fg: FactorGraph, s: int, nbrs: list):
    """``_class_of`` over the interface configurations of cluster s (module
    header): the key of configuration c is the tuple of the edges' rows
    Esub[sub_e(c)]; P[x] = class of x's interface configuration."""
    from .tables import sub_index
    parts = []  # (positions in s of the edge's coupled spins, Esub with s's index first)
    for t in nbrs:
        if t is None:
            continue
        e = fg.edge(min(s, t), max(s, t))
        if e is None:
            continue
        parts.append((e.pos_m, e.Esub) if s == e.m else (e.pos_n, e.Esub.T))
    U = np.array(sorted({int(q) for pos, _ in parts for q in pos}), dtype=np.int64)
    c = np.arange(2 ** len(U), dtype=np.int64)
    x_of_c = np.zeros_like(c)  # the first state carrying configuration c
    for k, q in enumerate(U):
        x_of_c |= ((c >> k) & 1) << int(q)
    keys = [Es[sub_index(x_of_c, pos)] for pos, Es in parts]
    Pc, reps_c = classes(len(c), keys)
    return Pc[sub_index(np.arange(fg.d[s]), U)], x_of_c[reps_c]


def build(fg: FactorGraph, beta: float) -> PEPS:
    u = 2.0 ** (-fg.shift)
    rows, cols = fg.rows, fg.cols

    def at(i, j):
        return i * cols + j if 0 <= i < rows and 0 <= j < cols else None

    log_offset = 0.0
    cls = []
    for s in range(fg.n_sites):
        i, j = divmod(s, cols)
        PL, repL = _class_of(fg, s, [at(i, j - 1), at(i - 1, j - 1)])
        PU, repU = _class_of(fg, s, [at(i - 1, j)])
        PR, repR = _class_of(fg, s, [at(i, j + 1), at(i - 1, j + 1)])
        PD, repD = _class_of(fg, s, [at(i + 1, j - 1), at(i + 1, j), at(i + 1, j + 1)])
        PG, repG = _class_of(fg, s, [at(i + 1, j + 1)])
        cls.append(dict(PL=PL, repL=repL, PU=PU, repU=repU, PR=PR, repR=repR, PD=PD, repD=repD, PG=PG,
                        repG=repG))

    def boltz(s, t, rs, rt):
        """Boltzmann factors of edge (s, t) between state lists rs of s and
        rt of t, shifted by the table's minimum ([len(rs), len(rt)]), or
        ones when there is no edge."""
        e = fg.edge(min(s, t), max(s, t)) if (s is not None and t is not None) else None
        if e is None:
            return np.ones((len(rs), len(rt)))
        mn = float(e.min())
        return np.exp(-beta * u * (e.block(s, rs, rt) - mn).astype(np.float64))

    sites = []
    for s in range(fg.n_sites):
        i, j = divmod(s, cols)
        d = fg.d[s]
        E = fg.E_loc[s]
        w = np.exp(-beta * u * (E - E.min()).astype(np.float64))
        log_offset += -beta * u * float(E.min())
        c = cls[s]
        left, upleft, up = at(i, j - 1), at(i - 1, j - 1), at(i - 1, j)
        one = np.zeros(1, np.int64)
        # left bond (a, g): P_R class of the left cluster, P_G class of the
        # up-left one
        repRl = cls[left]["repR"] if left is not None else one
        repGul = cls[upleft]["repG"] if upleft is not None else one
        NRl, Gin = len(repRl), len(repGul)
        bh = boltz(left, s, repRl, c["repL"])  # [NRl, NL]
        bd = boltz(upleft, s, repGul, c["repL"])  # [Gin, NL]
        b_left = (bh[:, None, :] * bd[None, :, :]).reshape(NRl * Gin, len(c["repL"]))
        # up index: P_D class of the upper cluster
        repDu = cls[up]["repD"] if up is not None else one
        b_up = boltz(up, s, repDu, c["repU"])  # [DU, NU]
        # up-right edge (i-1, j) - (i, j-1) of the left neighbour
        b_ad = boltz(up, left, repDu, repRl).T  # [NRl, DU]
        if up is not None:
            Gout = len(cls[up]["repG"])
            g_of_u = cls[up]["PG"][repDu]
        else:
            Gout, g_of_u = 1, np.zeros(1, np.int64)
        NR = len(c["repR"])
        sites.append(SiteData(d, E, w, c["PL"], c["PU"], c["PR"], c["PD"], c["PG"], c["repR"], c["repD"],
                              len(c["repL"]), len(c["repU"]), NR, len(c["repD"]), len(c["repG"]),
                              NRl * Gin, NR * Gout, len(repDu), Gin, Gout, b_left, b_up, b_ad, g_of_u,
                              fg.sparse))
    for e in fg.edges.values():
        log_offset += -beta * u * float(e.min())
    return PEPS(fg, beta, sites, log_offset)


def site_terms(st: SiteData, l: int, u: int):
    """The terms of W[l, :, u, :] one state x at a time: for every x the
    weight (everything in W's definition but the sum over x) and the output
    indices r = (P_R x, P_G(u)), s = P_D x.  Returns (coef [d], r [d], s [d])."""
    a = l // st.Gin
    coef = st.b_ad[a, u] * st.w * st.b_left[l, st.PL] * st.b_up[u, st.PU]
    r = st.PR * st.Gout + int(st.g_of_u[u])
    return coef, r, st.PD


def mpo_site(st: SiteData) -> np.ndarray:
    """Dense W[l, r, u, s] of one site (definition in the module header)."""
    W = np.zeros((st.DL, st.DR, st.DU, st.ND))
    if st.sparse:
        # the states' terms summed by output index (r, s)
        for u in range(st.DU):
            for l in range(st.DL):
                coef, r, s = site_terms(st, l, u)
                W[l, :, u, :] = np.bincount(r * st.ND + s, weights=coef,
                                            minlength=st.DR * st.ND).reshape(st.DR, st.ND)
        return W
    for u in range(st.DU):
        terms = [site_terms(st, l, u) for l in range(st.DL)]
        C = np.stack([t[0] for t in terms])  # [DL, d]
        _, r, s = terms[0]  # r and s do not depend on l
        onehot = np.zeros((st.d, st.DR * st.ND))
        onehot[np.arange(st.d), r * st.ND + s] = 1.0
        W[:, :, u, :] = (C @ onehot).reshape(st.DL, st.DR, st.ND)
    return W


def mpo_row(peps: PEPS, i: int) -> list:
    return [mpo_site(peps.site(i, j)) for j in range(peps.cols)]
