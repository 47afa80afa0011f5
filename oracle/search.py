"""Branch-and-bound (beam) search over cluster states with branch merging.

Test infrastructure only (see the package header).

Paper: Sec. 2 (the search builds the most probable configurations one Potts
variable at a time in a fixed order, keeping a predefined number of them;
marginal and conditional probabilities come from the contracted network;
partial configurations with identical values of the Potts variables on the
boundary next to the unexplored region are merged), Sec. 3.1
(``SearchParameters(max_states, cut_off_prob)``, ``merge_branches(...;
merge_type = :nofit)``, ``low_energy_spectrum``), and the solution's states,
energies and estimated probabilities (Sec. 2.2).

Readings taken here:
* order: row-major over the clusters of the grid;
* conditional of site (i, j) given the fixed prefix (W and its single-state
  terms as in ``peps``): with u_k the up index of site (i, k) (P_D class of
  cluster (i-1, k)), l the left bond fixed by clusters (i, j-1) and
  (i-1, j-1), Lenv = prod_{k<j} B_{i+1}[k][:, P_D(x_{i,k}), :] and the right
  environment
      R_j[a, l] = sum_{r, s, a'} W_j[l, r, u_j, s] B_{i+1}[j][a, s, a'] R_{j+1}[a', r],
  R_L = 1, the weight of state x is
      q(x) = c_x sum_{a,a'} Lenv[a] B_{i+1}[j][a, s_x, a'] R_{j+1}[a', r_x]
  where c_x, r_x, s_x are the coefficient and the output indices of x's term
  of W_j[l, :, u_j, :], and log p(x | prefix) = log q(x) - log sum_x q(x), in
  FP64.  A truncated boundary MPS can make q(x) slightly negative; such a
  weight counts as 0 (log p = -inf);
* a child's log-probability is its parent's plus the log-conditional; its
  partial energy is the parent's plus E_j(x) and the pairwise terms with
  already fixed neighbours (exact integers);
* merge key (``merge`` on, the paper's example): the states of all fixed
  clusters that have an edge to an unfixed cluster; at the last site the key
  is empty, so one state survives.  Among children with equal key the one
  with the lowest partial energy is kept, ties going to the
  lexicographically smaller state; the kept
  child keeps its own log-probability.  Within a key class the exact
  conditional ordering and the energy ordering coincide, so no floating-point
  comparison enters the merge;
* cut_off_prob c > 0 drops children with p < c * max p at that step; then
  the max_states children ranked first by (-log p, partial energy,
  lexicographic state) survive.  A near tie (|delta log p| <= 1e-9 max(1,
  |log p|) between the last survivor and the first dropped child) is
  recorded, since which of the two survives is then decided by rounding;
* the final states are reported sorted by (energy, lexicographic state), the
  energy recomputed from the tables, probability = exp(log p).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import boundary as bnd
from . import peps as peps_mod
from .tables import FactorGraph, energy

NEAR_TIE_RTOL = 1e-9


@dataclass
class Params:
    beta: float = 1.0
    chi: int = 16
    num_sweeps: int = 0
    beam: int = 256
    cut_off_prob: float = 0.0
    merge: bool = True
    droplet_energy: int = -1  # energy cutoff of droplets (units of the tables); < 0: no droplets
    droplet_hamming: int = 0  # an accepted droplet differs in more than this many Potts variables


@dataclass
class Result:
    states: np.ndarray  # [n, n_sites]
    energies: np.ndarray  # int64 [n]
    log_probs: np.ndarray  # float64 [n]
    near_ties: int = 0
    degenerate_cut: bool = False
    steps: list = field(default_factory=list)  # per site: (n candidates, n kept)
    droplets: list = field(default_factory=list)  # (energy, state) excitations of the best state
    # smallest relative log-probability gap between the last survivor and the
    # first dropped child over all prune steps (inf when no step dropped a
    # child); a search in lower precision keeps the same children when its
    # log-probability error stays below half of it
    min_cut_gap: float = float("inf")


def key_sites(fg: FactorGraph, s: int) -> list:
    """Fixed sites (index <= s) with an edge to an unfixed site (index > s)."""
    out = []
    for t in range(s + 1):
        for (m, n) in fg.edges:
            if (m == t and n > s) or (n == t and m > s):
                out.append(t)
                break
    return out


def _u(p: peps_mod.PEPS, i: int, j: int, prefix) -> int:
    """Up index of site (i, j): P_D class of the fixed cluster (i-1, j)."""
    return 0 if i == 0 else int(p.site(i - 1, j).PD[prefix[(i - 1) * p.cols + j]])


def _l(p: peps_mod.PEPS, i: int, j: int, prefix) -> int:
    """Left bond of site (i, j) given the fixed clusters (i, j-1) and
    (i-1, j-1): (P_R class, P_G class)."""
    if j == 0:
        return 0
    st = p.site(i, j)
    a = int(p.site(i, j - 1).PR[prefix[i * p.cols + j - 1]])
    g = int(p.site(i - 1, j - 1).PG[prefix[(i - 1) * p.cols + j - 1]]) if i > 0 else 0
    return a * st.Gin + g


def right_envs(p: peps_mod.PEPS, B: bnd.MPS, i: int, upper_states) -> list:
    """R_{j} for j = 1 .. L (index j -> [chi_j, DL_j]); R_L = [[1]]:
        R_j[a, l] = sum_{r, s, a'} W_j[l, r, u_j, s] B[j][a, s, a'] R_{j+1}[a', r]
    with u_j the up index of site (i, j) (the row above fixed)."""
    L = p.cols
    R = [None] * (L + 1)
    R[L] = np.ones((1, 1))
    for j in range(L - 1, 0, -1):
        st = p.site(i, j)
        uj = 0 if i == 0 else int(p.site(i - 1, j).PD[upper_states[j]])
        A = B.sites[j]
        Rn = np.zeros((A.shape[0], st.DL))
        if st.sparse:
            # the sum over states grouped by their output pair (s, r)
            _, r, s = peps_mod.site_terms(st, 0, uj)
            pairs, inv = np.unique(s * st.DR + r, return_inverse=True)
            Vp = np.einsum("axb,bx->ax", A[:, pairs // st.DR, :], R[j + 1][:, pairs % st.DR])
        for l in range(st.DL):
            coef, r, s = peps_mod.site_terms(st, l, uj)
            if st.sparse:
                Rn[:, l] = Vp @ np.bincount(inv, weights=coef, minlength=len(pairs))
                continue
            V = np.einsum("axb,bx->ax", A[:, s, :], R[j + 1][:, r])  # [chi, d]
            Rn[:, l] = V @ coef
        R[j] = Rn / np.max(np.abs(Rn))
    return R


def log_conditional(p, B, i, j, lenv, R, prefix):
    """log p(x | prefix) for all x of site (i, j) (formula in the header);
    prefix = states of the sites before (i, j) in row-major order."""
    st = p.site(i, j)
    coef, r, s = peps_mod.site_terms(st, _l(p, i, j, prefix), _u(p, i, j, prefix))
    A = B.sites[j]
    # q(x) = coef(x) (lenv A[:, s(x), :] R[:, r(x)]); the contraction depends
    # on x only through (s(x), r(x)), so it is evaluated once per pair (the
    # same expression for every state of the pair)
    pairs, inv = np.unique(s * st.DR + r, return_inverse=True)
    z = np.array([float(lenv @ A[:, int(k) // st.DR, :] @ R[j + 1][:, int(k) % st.DR]) for k in pairs])
    q = coef * z[inv]
    q = np.maximum(q, 0.0)
    with np.errstate(divide="ignore"):
        return np.log(q) - np.log(np.sum(q))


def delta_energies(fg: FactorGraph, s: int, prefix) -> np.ndarray:
    """E_s(x) plus the pairwise terms of x with the fixed clusters, for every
    state x of site s (int64 [d_s])."""
    dE = np.array(fg.E_loc[s], dtype=np.int64)
    for (m, n), e in fg.edges.items():
        if n == s:
            dE = dE + (e.E[prefix[m]] if e.E is not None else e.Esub[e.sub_m[prefix[m]], e.sub_n])
    return dE


@dataclass
class _Partial:
    states: tuple
    E: int
    logp: float
    lenv: np.ndarray
    R: list = None
    drops: list = field(default_factory=list)  # droplets: (dE, ((site, state), ...)) relative to states


def _apply(states, diff):
    st = list(states)
    for t, x in diff:
        st[t] = x
    return tuple(st)


def _hamming(a, b) -> int:
    return sum(1 for u, v in zip(a, b) if u != v)


def _droplets(w_st, w_E, w_parent, losers, prm: "Params") -> list:
    """Droplets of a merge winner (Sec. 2 and Sec. 3.1 ``SingleLayerDroplets``,
    ``energy_cutoff``, ``hamming_cutoff``).  Reading: a partial configuration
    that loses a merge agrees with the winner on every fixed variable next to
    the unexplored region, so where they differ is a region that no later
    variable touches; the loser is an excitation of the winner localised
    there, dE = E_loser - E_winner, valid for every descendant of the winner.
    The winner keeps its parent's droplets; the candidates are each loser and
    each loser with one of its own droplets applied, taken in (dE, state)
    order; a candidate is accepted when dE <= energy cutoff and it differs
    from the winner and from every droplet accepted so far in more than
    hamming cutoff Potts variables."""
    acc = list(w_parent.drops)
    seen = [w_st] + [_apply(w_st, d) for _, d in acc]
    cand = []
    for l_st, l_E, l_parent in losers:
        cand.append((l_E - w_E, l_st))
        for dE, diff in l_parent.drops:
            cand.append((l_E + dE - w_E, _apply(l_st, diff)))
    for dE, st in sorted(cand):
        if dE > prm.droplet_energy:
            continue
        if any(_hamming(st, a) <= prm.droplet_hamming for a in seen):
            continue
        acc.append((dE, tuple((t, st[t]) for t in range(len(st)) if st[t] != w_st[t])))
        seen.append(st)
    return acc


def solve(fg: FactorGraph, prm: Params, boundary=None) -> Result:
    """``low_energy_spectrum`` with ``merge_type = :nofit`` (readings above)."""
    p = peps_mod.build(fg, prm.beta)
    if boundary is None:
        boundary = bnd.boundary_mpses(p, prm.chi, prm.num_sweeps)
    rows, cols = fg.rows, fg.cols
    beam = [_Partial((), 0, 0.0, np.ones(1))]
    near_ties = 0
    min_gap = float("inf")
    steps = []
    for s in range(fg.n_sites):
        i, j = divmod(s, cols)
        B = boundary[i + 1]
        if j == 0:
            for b in beam:
                b.lenv = np.ones(1)
                b.R = right_envs(p, B, i, [b.states[(i - 1) * cols + k] for k in range(cols)] if i > 0 else None)
        ks = key_sites(fg, s)
        children = {}
        drop_on = prm.merge and prm.droplet_energy >= 0
        members = {}
        n_cand = 0
        for b in beam:
            lc = log_conditional(p, B, i, j, b.lenv, b.R, b.states)
            dEs = delta_energies(fg, s, b.states)
            for x in range(fg.d[s]):
                st = b.states + (x,)
                E = b.E + int(dEs[x])
                key = tuple(st[t] for t in ks) if prm.merge else st
                n_cand += 1
                if drop_on:
                    members.setdefault(key, []).append((st, E, b))
                cur = children.get(key)
                if cur is None or (E, st) < (cur[1], cur[0]):
                    children[key] = (st, E, b.logp + float(lc[x]), b)
        cands = list(children.values())
        if prm.cut_off_prob > 0:
            top = max(c[2] for c in cands)
            cands = [c for c in cands if c[2] >= top + np.log(prm.cut_off_prob)]
        cands.sort(key=lambda c: (-c[2], c[1], c[0]))
        if len(cands) > prm.beam:
            a, b2 = cands[prm.beam - 1][2], cands[prm.beam][2]
            if abs(a - b2) <= NEAR_TIE_RTOL * max(1.0, abs(a)):
                near_ties += 1
            min_gap = min(min_gap, abs(a - b2) / max(1.0, abs(a)))
            cands = cands[:prm.beam]
        steps.append((n_cand, len(cands)))
        new = []
        for st, E, lp, parent in sorted(cands, key=lambda c: c[0]):
            x = st[-1]
            A = B.sites[j]
            v = parent.lenv @ A[:, p.site(i, j).PD[x], :]
            m = np.max(np.abs(v))
            drops = []
            if drop_on:
                key = tuple(st[t] for t in ks)
                losers = [mb for mb in members[key] if mb[0] != st]
                drops = _droplets(st, E, parent, losers, prm)
            new.append(_Partial(st, E, lp, v / m if m > 0 else v, parent.R, drops))
        beam = new
    order = sorted(range(len(beam)), key=lambda k: (energy(fg, beam[k].states), beam[k].states))
    states = np.array([beam[k].states for k in order], dtype=np.int64)
    energies = np.array([energy(fg, beam[k].states) for k in order], dtype=np.int64)
    for k in order:
        assert energy(fg, beam[k].states) == beam[k].E
    logps = np.array([beam[k].logp for k in order])
    deg = any(boundary[r].degenerate for r in boundary)
    # unpack_droplets: the best state's excitations as full states
    drops = []
    if order:
        top = beam[order[0]]
        drops = sorted((top.E + dE, _apply(top.states, diff)) for dE, diff in top.drops)
    return Result(states, energies, logps, near_ties, deg, steps, drops, min_gap)


def debug_marginals(fg: FactorGraph, prm: Params, site: int, prefixes, boundary=None):
    """Teacher-forced log-marginals of ``site`` for given prefixes
    (prefix = states of sites 0 .. site-1): [n_prefix, d_site]."""
    p = peps_mod.build(fg, prm.beta)
    if boundary is None:
        boundary = bnd.boundary_mpses(p, prm.chi, prm.num_sweeps)
    cols = fg.cols
    i, j = divmod(site, cols)
    B = boundary[i + 1]
    out = []
    for pre in prefixes:
        pre = [int(v) for v in pre]
        upper = [pre[(i - 1) * cols + k] for k in range(cols)] if i > 0 else None
        R = right_envs(p, B, i, upper)
        lenv = np.ones(1)
        for k in range(j):
            v = lenv @ B.sites[k][:, p.site(i, k).PD[pre[i * cols + k]], :]
            lenv = v / np.max(np.abs(v))
        out.append(log_conditional(p, B, i, j, lenv, R, pre))
    return np.array(out)
