"""Boltzmann weights and the row MPOs of the PEPS (square lattice).

Test infrastructure only (see the package header).

Paper: Sec. 2 and Fig. 1(c): the Boltzmann distribution p(x) ~ exp(-beta E(x))
of the clustered Potts model is a PEPS on the square lattice of clusters;
Sec. 3.1 (``PEPSNetwork``, ``Sparsity``): a site tensor is built from the
local weights of the cluster and from the pairwise interactions, which reach
the cluster only through projections of its state.

Readings taken here:
* weights are shifted by the minimum of each table so that every weight is
  <= 1: w_s(x) = exp(-beta u (E_s(x) - min E_s)), b_e = exp(-beta u
  (R_e - min R_e)), u = 2**-energy_shift; the shifts add back into log Z;
* the Boltzmann matrix of an edge is absorbed into its right (horizontal edge)
  or lower (vertical edge) site;
* the MPO of row i maps the up index u (row projection of the cluster above,
  on the vertical edge into site (i,j)) to the down index s (row projection
  of this cluster on the vertical edge below it):
      W[l, r, u, s] = sum_x w(x) b_left[l, P_L(x)] b_up[u, P_U(x)]
                              [r == P_R(x)] [s == P_D(x)]
  where l and r are the horizontal bonds (row projections of the left
  neighbour and of this site on the horizontal edges).  A missing edge is a
  bond of dimension 1 with projector 0 and weight 1.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .tables import SQUARE, FactorGraph


@dataclass
class SiteData:
    d: int
    E: np.ndarray  # int64 [d] local table
    w: np.ndarray  # float64 [d] shifted local weights
    PL: np.ndarray
    PR: np.ndarray
    PU: np.ndarray
    PD: np.ndarray
    DL: int
    DR: int
    DU: int
    DD: int
    b_left: np.ndarray  # [DL, ncols] Boltzmann matrix of the edge from the left
    b_up: np.ndarray  # [DU, ncols] Boltzmann matrix of the edge from above
    E_left: np.ndarray  # int64 full table of the left edge [d_left, d] (or None)
    E_up: np.ndarray  # int64 full table of the up edge [d_up, d] (or None)


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


def build(fg: FactorGraph, beta: float) -> PEPS:
    if fg.node_type != SQUARE:
        raise NotImplementedError("only the square lattice is built here")
    u = 2.0 ** (-fg.shift)
    rows, cols = fg.rows, fg.cols
    log_offset = 0.0
    sites = []
    for s in range(fg.n_sites):
        i, j = divmod(s, cols)
        d = fg.d[s]
        E = fg.E_loc[s]
        w = np.exp(-beta * u * (E - E.min()).astype(np.float64))
        log_offset += -beta * u * float(E.min())
        zeros = np.zeros(d, dtype=np.int64)
        one = np.ones((1, 1))
        eL = fg.edge(s - 1, s) if j > 0 else None
        eR = fg.edge(s, s + 1) if j + 1 < cols else None
        eU = fg.edge(s - cols, s) if i > 0 else None
        eD = fg.edge(s, s + cols) if i + 1 < rows else None
        PL, DL, bL = (eL.Pn, eL.R.shape[0], None) if eL is not None else (zeros, 1, one)
        PU, DU, bU = (eU.Pn, eU.R.shape[0], None) if eU is not None else (zeros, 1, one)
        PR, DR = (eR.Pm, eR.R.shape[0]) if eR is not None else (zeros, 1)
        PD, DD = (eD.Pm, eD.R.shape[0]) if eD is not None else (zeros, 1)
        if eL is not None:
            bL = np.exp(-beta * u * (eL.R - eL.R.min()).astype(np.float64))
        if eU is not None:
            bU = np.exp(-beta * u * (eU.R - eU.R.min()).astype(np.float64))
        sites.append(SiteData(d, E, w, PL, PR, PU, PD, DL, DR, DU, DD, bL, bU,
                              eL.E if eL is not None else None, eU.E if eU is not None else None))
    for e in fg.edges.values():
        log_offset += -beta * u * float(e.R.min())
    return PEPS(fg, beta, sites, log_offset)


def mpo_site(st: SiteData) -> np.ndarray:
    """Dense W[l, r, u, s] of one site (definition in the module header)."""
    W = np.zeros((st.DL, st.DR, st.DU, st.DD))
    for x in range(st.d):
        W[:, st.PR[x], :, st.PD[x]] += st.w[x] * np.outer(st.b_left[:, st.PL[x]], st.b_up[:, st.PU[x]])
    return W


def mpo_row(peps: PEPS, i: int) -> list:
    return [mpo_site(peps.site(i, j)) for j in range(peps.cols)]
