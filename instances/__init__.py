"""Seeded synthetic problem instances (no solver arithmetic lives here).

These generators draw the random couplings and fields of the synthetic
workloads and return them as plain NumPy arrays in the problem's input form
(Ising couplings + fields + cluster map, or Potts local and pairwise energy
tables).  Both the oracle and the CUDA path read their inputs from here; the
module holds none of the method's arithmetic (no energy tables, projectors,
Boltzmann weights or contractions).

Energy grid.  Every real value is drawn on the grid ``2**-energy_shift`` so
that energies are exact integers in units of ``2**-energy_shift``:
``energy_shift = 0`` for +-1 instances, ``24`` for Gaussian ones.

Workload shapes (paper Sec. 2 Eq. 1-2; Fig. 4 for the Chimera unit cell):

* ``chimera``: an L x L grid of K_{4,4} unit cells, 8 spins per cell.  Cell
  (i, j) owns spins ``8*(i*L + j) + k``; k = 0..3 form side A, k = 4..7 side B.
  Couplers: all 16 A-B pairs inside a cell, A_k(i,j)-A_k(i+1,j) between
  vertical neighbours and B_k(i,j)-B_k(i,j+1) between horizontal neighbours.
  One cluster per cell.
* ``square``: an L x L grid with one spin per site and nearest-neighbour
  couplings (clusters of a single spin).
* ``king_ising``: an m x n grid of clusters of t spins, all spins of a cluster
  coupled to each other and to every spin of the 8 king's-move neighbour
  clusters (the quasi-2D graph of the paper's Fig. 1(a)).
* ``king_potts``: an L x L grid of Potts variables with d states, local tables
  and d x d pairwise tables on all 8-neighbour edges.
* ``large_cells``: a rows x cols grid (king's-graph or square-lattice
  adjacency) of clusters of k spins -- 16 is the size of a Zephyr unit cell,
  24 of a Pegasus one (paper Sec. 3.1.1, Fig. 4: both map onto king's graphs
  of clusters) -- with K_{k/2,k/2} couplers inside a cell (between its first
  and second halves) and ``links`` couplers between every pair of
  neighbouring cells, each between a spin drawn from each cell (distinct
  pairs), J uniform in {-1,+1}, h = 0.  Only the sizes follow the vendors'
  cells; the wiring is this generator's.
* ``inpainting``: an L x L grid of d labels shaped like an inpainting problem
  (Sec. 3 example, Fig. 5: data on a circular boundary, the inside to be
  filled in): pixels on or outside a ring observe one of d labels in d equal
  arcs (a seeded rotation), local cost 0 for the observed label and
  ``data_cost`` for the others, no data inside; Potts smoothness
  w [x_m != x_n] on the 8-neighbour edges, w = 1 for axis and 1/sqrt(2) for
  diagonal edges.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SQUARE = 0
KING = 1


@dataclass
class IsingInstance:
    """Ising form: E(s) = sum_e J_e s_i s_j + sum_i h_i s_i, s in {-1,+1}."""

    n_spins: int
    ei: np.ndarray  # int32 [n_edges]
    ej: np.ndarray  # int32 [n_edges]
    J: np.ndarray  # float64 [n_edges], on the 2**-energy_shift grid
    h: np.ndarray  # float64 [n_spins], on the grid
    cluster_of_spin: np.ndarray  # int32 [n_spins]
    grid_rows: int
    grid_cols: int
    cluster_row: np.ndarray  # int32 [n_clusters]
    cluster_col: np.ndarray  # int32 [n_clusters]
    energy_shift: int
    node_type: int
    name: str = ""
    meta: dict = field(default_factory=dict)


@dataclass
class PottsInstance:
    """Potts form: E(x) = sum_<m,n> E_mn(x_m, x_n) + sum_n E_n(x_n) (Eq. 1).

    Sites are the grid cells in row-major order.  ``local_E`` concatenates the
    per-site tables; ``pair_E`` concatenates d_m x d_n row-major tables, one per
    edge (em[k], en[k]), in units of 2**-energy_shift (int64)."""

    grid_rows: int
    grid_cols: int
    d: np.ndarray  # int32 [n_sites]
    local_E: np.ndarray  # int64 [sum d]
    em: np.ndarray  # int32 [n_edges]
    en: np.ndarray  # int32 [n_edges]
    pair_E: np.ndarray  # int64 [sum d_m*d_n]
    energy_shift: int
    node_type: int
    name: str = ""


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _on_grid(x: np.ndarray, shift: int) -> np.ndarray:
    """Round real draws onto the 2**-shift grid (exactly representable)."""
    return np.round(np.asarray(x, dtype=np.float64) * (2.0 ** shift)) / (2.0 ** shift)


def chimera(L: int, seed: int, couplings: str = "pm1", h_sigma: float = 0.0,
            cols: int | None = None) -> IsingInstance:
    """Chimera-like grid of K_{4,4} cells.

    couplings: "pm1" -> J uniform in {-1,+1}; "gauss" -> J ~ N(0,1) on the
    2**-24 grid.  h_sigma > 0 draws h ~ N(0, h_sigma) (standard deviation) on
    the same grid; otherwise h = 0."""
    rows, cols = L, (L if cols is None else cols)
    rng = _rng(seed)
    shift = 0 if (couplings == "pm1" and h_sigma == 0.0) else 24
    ei, ej = [], []

    def cell(i, j):
        return 8 * (i * cols + j)

    for i in range(rows):
        for j in range(cols):
            b = cell(i, j)
            for ka in range(4):
                for kb in range(4, 8):
                    ei.append(b + ka)
                    ej.append(b + kb)
    for i in range(rows - 1):
        for j in range(cols):
            for k in range(4):
                ei.append(cell(i, j) + k)
                ej.append(cell(i + 1, j) + k)
    for i in range(rows):
        for j in range(cols - 1):
            for k in range(4, 8):
                ei.append(cell(i, j) + k)
                ej.append(cell(i, j + 1) + k)
    n_edges = len(ei)
    if couplings == "pm1":
        J = rng.choice(np.array([-1.0, 1.0]), size=n_edges)
    elif couplings == "gauss":
        J = _on_grid(rng.standard_normal(n_edges), 24)
    else:
        raise ValueError(couplings)
    n = 8 * rows * cols
    h = _on_grid(rng.normal(0.0, h_sigma, n), 24) if h_sigma > 0 else np.zeros(n)
    if couplings == "pm1" and h_sigma == 0.0:
        J = J.astype(np.float64)
    cos = np.repeat(np.arange(rows * cols, dtype=np.int32), 8)
    crow = (np.arange(rows * cols) // cols).astype(np.int32)
    ccol = (np.arange(rows * cols) % cols).astype(np.int32)
    return IsingInstance(n, np.array(ei, np.int32), np.array(ej, np.int32), J, h, cos,
                         rows, cols, crow, ccol, shift, SQUARE,
                         name=f"chimera{rows}x{cols}_{couplings}_s{seed}")


def square(L: int, seed: int, cols: int | None = None, h_sigma: float = 0.0) -> IsingInstance:
    """L x L square lattice, one spin per cluster, J uniform in {-1,+1}."""
    rows, cols = L, (L if cols is None else cols)
    rng = _rng(seed)
    ei, ej = [], []
    for i in range(rows):
        for j in range(cols):
            s = i * cols + j
            if j + 1 < cols:
                ei.append(s)
                ej.append(s + 1)
            if i + 1 < rows:
                ei.append(s)
                ej.append(s + cols)
    J = rng.choice(np.array([-1.0, 1.0]), size=len(ei))
    n = rows * cols
    shift = 0
    if h_sigma > 0:
        h = _on_grid(rng.normal(0.0, h_sigma, n), 24)
        shift = 24
    else:
        h = np.zeros(n)
    return IsingInstance(n, np.array(ei, np.int32), np.array(ej, np.int32), J, h,
                         np.arange(n, dtype=np.int32), rows, cols,
                         (np.arange(n) // cols).astype(np.int32),
                         (np.arange(n) % cols).astype(np.int32), shift, SQUARE,
                         name=f"square{rows}x{cols}_s{seed}")


def king_ising(m: int, n: int, t: int, seed: int) -> IsingInstance:
    """m x n king's graph of clusters with t spins each, J uniform in {-1,+1}."""
    rng = _rng(seed)
    ei, ej = [], []

    def spins(i, j):
        return [t * (i * n + j) + k for k in range(t)]

    for i in range(m):
        for j in range(n):
            s = spins(i, j)
            for a in range(t):
                for b in range(a + 1, t):
                    ei.append(s[a])
                    ej.append(s[b])
            for di, dj in ((0, 1), (1, -1), (1, 0), (1, 1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < m and 0 <= jj < n:
                    for a in s:
                        for b in spins(ii, jj):
                            ei.append(a)
                            ej.append(b)
    J = rng.choice(np.array([-1.0, 1.0]), size=len(ei))
    N = m * n * t
    return IsingInstance(N, np.array(ei, np.int32), np.array(ej, np.int32), J, np.zeros(N),
                         np.repeat(np.arange(m * n, dtype=np.int32), t), m, n,
                         (np.arange(m * n) // n).astype(np.int32),
                         (np.arange(m * n) % n).astype(np.int32), 0, KING,
                         name=f"king{m}x{n}x{t}_s{seed}")


def king_potts(L: int, d: int, seed: int, cols: int | None = None) -> PottsInstance:
    """L x L king's-graph Potts model: E_n ~ N(0,1), E_mn ~ N(0,1) on all
    8-neighbour edges, every value on the 2**-24 grid (int64 units)."""
    rows, cols = L, (L if cols is None else cols)
    rng = _rng(seed)
    n_sites = rows * cols
    shift = 24
    local = np.round(rng.standard_normal(n_sites * d) * 2.0 ** shift).astype(np.int64)
    em, en, pair = [], [], []
    for i in range(rows):
        for j in range(cols):
            s = i * cols + j
            for di, dj in ((0, 1), (1, -1), (1, 0), (1, 1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < rows and 0 <= jj < cols:
                    em.append(s)
                    en.append(ii * cols + jj)
    for _ in em:
        pair.append(np.round(rng.standard_normal(d * d) * 2.0 ** shift).astype(np.int64))
    return PottsInstance(rows, cols, np.full(n_sites, d, np.int32), local,
                         np.array(em, np.int32), np.array(en, np.int32),
                         np.concatenate(pair) if pair else np.zeros(0, np.int64), shift, KING,
                         name=f"kingpotts{rows}x{cols}_d{d}_s{seed}")


def inpainting(L: int, d: int, seed: int, data_cost: float = 4.0, ring: float = 1.5) -> PottsInstance:
    """Inpainting-shaped Potts model on an L x L king's graph (module header):
    pixel (i, j) at distance r from the grid centre observes a label when
    r >= L / 2 - ring, the label of the angular arc it lies in (d arcs,
    rotated by a seeded angle).  Values on the 2**-24 grid."""
    rng = _rng(seed)
    shift = 24
    unit = 2.0 ** shift
    rot = float(rng.uniform(0.0, 2.0 * np.pi))
    c = (L - 1) / 2.0
    local = np.zeros((L * L, d), np.int64)
    cost = int(round(data_cost * unit))
    for i in range(L):
        for j in range(L):
            y, x = i - c, j - c
            if np.hypot(y, x) >= L / 2.0 - ring:
                lab = int(((np.arctan2(y, x) + rot) % (2.0 * np.pi)) // (2.0 * np.pi / d)) % d
                local[i * L + j, :] = cost
                local[i * L + j, lab] = 0
    w_axis, w_diag = int(round(unit)), int(round(unit / np.sqrt(2.0)))
    em, en, pair = [], [], []
    for i in range(L):
        for j in range(L):
            s = i * L + j
            for di, dj in ((0, 1), (1, -1), (1, 0), (1, 1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < L and 0 <= jj < L:
                    w = w_axis if di == 0 or dj == 0 else w_diag
                    em.append(s)
                    en.append(ii * L + jj)
                    pair.append((w * (1 - np.eye(d, dtype=np.int64))).reshape(-1))
    return PottsInstance(L, L, np.full(L * L, d, np.int32), local.reshape(-1),
                         np.array(em, np.int32), np.array(en, np.int32),
                         np.concatenate(pair) if pair else np.zeros(0, np.int64), shift, KING,
                         name=f"inpainting{L}x{L}_d{d}_s{seed}")


def batch_chimera(n_instances: int, L_lo: int, L_hi: int, base_seed: int,
                  chis=(16, 32)) -> list:
    """Uneven batch: L ~ U{L_lo..L_hi}, +-1 couplings, chi drawn per instance
    from ``chis`` by a seeded coin.  Returns (instance, chi) pairs."""
    rng = _rng(base_seed)
    Ls = rng.integers(L_lo, L_hi + 1, size=n_instances)
    coins = rng.integers(0, len(chis), size=n_instances)
    return [(chimera(int(L), base_seed + 1 + i), int(chis[c])) for i, (L, c) in enumerate(zip(Ls, coins))]


def large_cells(rows: int, cols: int, k: int, seed: int, links: int = 2, node_type: int = KING,
                intra: str = "bipartite") -> IsingInstance:
    """rows x cols grid of clusters of k spins (module header: ``large_cells``).
    intra: "bipartite" (K_{k/2,k/2} inside a cell) or "ring" (spin t coupled
    to spin t+1 mod k: fewer couplers, the same number of states)."""
    if k % 2 or k < 4:
        raise ValueError("k must be even and at least 4")
    rng = _rng(seed)
    ei, ej = [], []

    def spins(i, j):
        return [k * (i * cols + j) + t for t in range(k)]

    nbrs = ((0, 1), (1, -1), (1, 0), (1, 1)) if node_type == KING else ((0, 1), (1, 0))
    for i in range(rows):
        for j in range(cols):
            s = spins(i, j)
            if intra == "ring":
                for a in range(k):
                    ei.append(s[a])
                    ej.append(s[(a + 1) % k])
            else:
                for a in range(k // 2):
                    for b in range(k // 2, k):
                        ei.append(s[a])
                        ej.append(s[b])
            for di, dj in nbrs:
                ii, jj = i + di, j + dj
                if not (0 <= ii < rows and 0 <= jj < cols):
                    continue
                t = spins(ii, jj)
                pairs = set()
                while len(pairs) < links:
                    pairs.add((int(rng.integers(k)), int(rng.integers(k))))
                for a, b in sorted(pairs):
                    ei.append(s[a])
                    ej.append(t[b])
    J = rng.choice(np.array([-1.0, 1.0]), size=len(ei))
    n = rows * cols * k
    return IsingInstance(n, np.array(ei, np.int32), np.array(ej, np.int32), J, np.zeros(n),
                         np.repeat(np.arange(rows * cols, dtype=np.int32), k), rows, cols,
                         (np.arange(rows * cols) // cols).astype(np.int32),
                         (np.arange(rows * cols) % cols).astype(np.int32), 0, node_type,
                         name=f"cells{rows}x{cols}x{k}_l{links}_s{seed}")
