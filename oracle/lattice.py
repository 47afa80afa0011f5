"""The 8 lattice transformations solved together, best of 8.

Test infrastructure only (see the package header).

Paper: Sec. 3.1 (the example solves the instance under every transformation
of the square lattice, ``all_lattice_transformations``, rotations and
reflections, and keeps the best result): the Boltzmann distribution and the
spectrum are the same on every transformed lattice, while the approximate
contraction and the search, which follow the row-major order of the
transformed grid, can reach different low-energy states.

Readings taken here:
* transformation k in 0..7 acts on the grid position (i, j) of every cluster
  of an R x C grid: bit 4 transposes ((i, j) -> (j, i), the grid becomes
  C x R), then bit 1 reverses the rows (i -> R' - 1 - i) and bit 2 the
  columns (j -> C' - 1 - j) of the resulting R' x C' grid; k = 0 is the
  identity;
* Ising form: only the clusters' grid positions change (spins, couplings and
  the cluster of every spin stay), so a cluster's state encoding is the same
  on every lattice;
* Potts form: site (i, j) moves with its local table; every edge keeps its
  table, oriented as before (rows: the first endpoint), with both endpoints
  renumbered; diagonal couplings of a king's graph map onto diagonals;
* best of 8: the lowest best energy; equal best energies go to the lowest k.
  The states of every lattice are mapped back to the sites of the original
  grid before they are compared or returned.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import instances as I

from . import search, tables


def position(i: int, j: int, rows: int, cols: int, k: int):
    """Grid position of (i, j) under transformation k, and the new grid shape."""
    R, C = rows, cols
    if k & 4:
        i, j = j, i
        R, C = C, R
    if k & 1:
        i = R - 1 - i
    if k & 2:
        j = C - 1 - j
    return i, j, R, C


def site_map(rows: int, cols: int, k: int) -> np.ndarray:
    """site_map[s] = site of the transformed grid that holds original site s."""
    out = np.empty(rows * cols, np.int64)
    for i in range(rows):
        for j in range(cols):
            a, b, _, C = position(i, j, rows, cols, k)
            out[i * cols + j] = a * C + b
    return out


def transform(inst, k: int):
    """The instance on the k-th transformed lattice (Ising or Potts form)."""
    rows, cols = inst.grid_rows, inst.grid_cols
    _, _, R, C = position(0, 0, rows, cols, k)
    if isinstance(inst, I.IsingInstance):
        r = np.empty_like(np.asarray(inst.cluster_row))
        c = np.empty_like(np.asarray(inst.cluster_col))
        for q in range(len(r)):
            r[q], c[q], _, _ = position(int(inst.cluster_row[q]), int(inst.cluster_col[q]), rows, cols, k)
        out = I.IsingInstance(**{**inst.__dict__})
        out.grid_rows, out.grid_cols = R, C
        out.cluster_row, out.cluster_col = r.astype(np.int32), c.astype(np.int32)
        return out
    smap = site_map(rows, cols, k)
    n = rows * cols
    d = np.asarray(inst.d)
    off = np.concatenate([[0], np.cumsum(d)])
    old_of = np.empty(n, np.int64)
    old_of[smap] = np.arange(n)
    local = np.concatenate([inst.local_E[off[old_of[s]]:off[old_of[s] + 1]] for s in range(n)])
    em = smap[np.asarray(inst.em)].astype(np.int32)
    en = smap[np.asarray(inst.en)].astype(np.int32)
    return I.PottsInstance(R, C, d[old_of].astype(np.int32), local, em, en, inst.pair_E, inst.energy_shift,
                           inst.node_type, name=getattr(inst, "name", ""))


def factor_graph(inst) -> tables.FactorGraph:
    return tables.from_ising(inst) if isinstance(inst, I.IsingInstance) else tables.from_potts(inst)


@dataclass
class Best:
    k: int  # the lattice that gave the best energy
    states: np.ndarray  # [n, n_sites] on the original grid
    energies: np.ndarray  # int64 [n]
    log_probs: np.ndarray  # float64 [n]
    best_per_lattice: np.ndarray  # int64 [8]
    states_per_lattice: list  # 8 x [n_k, n_sites] on the original grid


def solve_best_of_8(inst, prm: search.Params) -> Best:
    """``low_energy_spectrum`` on each of the 8 lattices; the best of them."""
    rows, cols = inst.grid_rows, inst.grid_cols
    per, best_E = [], []
    for k in range(8):
        res = search.solve(factor_graph(transform(inst, k)), prm)
        back = np.asarray(res.states)[:, site_map(rows, cols, k)]
        per.append((back, np.asarray(res.energies), np.asarray(res.log_probs)))
        best_E.append(int(res.energies[0]))
    kb = int(np.argmin(best_E))  # first minimum: lowest k
    states, E, lp = per[kb]
    return Best(kb, states, E, lp, np.array(best_E, np.int64), [p[0] for p in per])
