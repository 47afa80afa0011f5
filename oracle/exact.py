"""Exact references that use none of the tables, projectors or MPSs.

Test infrastructure only (see the package header).

Everything here works on spins and Eq. 2, or on Potts configurations and
Eq. 1, directly:
* ``brute_force``: all 2^n spin configurations (n <= 24), giving the exact
  ground energy and degeneracy, log Z = log sum exp(-beta E), and exact
  conditional marginals of cluster states given a prefix of cluster states;
* ``potts_all_energies``: every configuration of a small Potts instance;
* ``interface_sum``: clusters of many spins (up to 24 per cluster) whose
  inter-cluster couplers touch few spins: every cluster's states are
  enumerated for its own energy (fields and couplers inside it), grouped by
  the configuration of its interface spins (those with a coupler to another
  cluster), and every combination of interface configurations is summed
  (log-sum-exp) or minimised with the couplers between clusters, giving the
  exact log Z, ground energy and the exact marginal of one cluster's states,
  also given the states of other clusters (conditionals);
* ``brute_force_c``: the same ground energy, degeneracy and log Z from a C
  enumerator parallel over the host's cores (``bruteforce.c``);
* ``chimera_strip``: row transfer matrices of a Chimera-like strip of width
  <= 3 cells over the 4w side-A spins of a row (the only spins with couplers
  to the next row), giving exact log Z (log-sum-exp) and the exact ground
  energy (min-plus, integer) for any number of rows.
"""
from __future__ import annotations

import numpy as np



def _grid_ints(values, shift):
    """Integers k with value = k * 2^-shift, from each float's exact rational
    value (independent of the tables' conversion, so that a scaling mistake
    there cannot pass the brute-force pins)."""
    out = []
    for v in np.asarray(values, dtype=np.float64).ravel():
        num, den = float(v).as_integer_ratio()  # den is a power of two
        scaled = num * (1 << shift)
        if scaled % den:
            raise ValueError("value not on the 2**-shift grid")
        out.append(scaled // den)
    return np.array(out, dtype=np.int64)


def _spins(n, lo, hi):
    x = np.arange(lo, hi, dtype=np.int64)[:, None]
    return 2 * ((x >> np.arange(n, dtype=np.int64)[None, :]) & 1) - 1


def all_energies(inst) -> np.ndarray:
    """int64 energy of every spin configuration, index = sum_i b_i 2^i.

    Eq. 2 term by term: the coupling sum is taken as s . (J_upper s) with the
    integer couplings held exactly in float64 (all partial sums < 2^53)."""
    n = inst.n_spins
    if n > 24:
        raise ValueError("brute force is limited to 24 spins")
    J = _grid_ints(inst.J, inst.energy_shift)
    h = _grid_ints(inst.h, inst.energy_shift)
    if np.sum(np.abs(J)) + np.sum(np.abs(h)) >= 2 ** 52:
        raise ValueError("energies too large for the float64 path")
    Jm = np.zeros((n, n))
    np.add.at(Jm, (np.asarray(inst.ei), np.asarray(inst.ej)), J.astype(np.float64))
    hf = h.astype(np.float64)
    out = np.empty(2 ** n, dtype=np.int64)
    chunk = 1 << 18
    for lo in range(0, 2 ** n, chunk):
        hi = min(2 ** n, lo + chunk)
        s = _spins(n, lo, hi).astype(np.float64)
        e = np.einsum("ci,ci->c", s @ Jm, s) + s @ hf
        out[lo:hi] = np.rint(e).astype(np.int64)
    return out


def logsumexp(a):
    m = np.max(a)
    return float(m + np.log(np.sum(np.exp(a - m))))


def brute_force(inst, beta: float):
    E = all_energies(inst)
    emin = int(E.min())
    u = 2.0 ** (-inst.energy_shift)
    logZ = logsumexp(-beta * u * E.astype(np.float64))
    return {"E": E, "ground": emin, "degeneracy": int(np.sum(E == emin)), "logZ": logZ}


def cluster_states(n, sites_spins):
    """State of every cluster (bits of its spins, ascending) for all 2^n
    configurations: list over sites of uint16 arrays [2^n]."""
    idx = np.arange(2 ** n, dtype=np.int64)
    out = []
    for sp in sites_spins:
        x = np.zeros(2 ** n, dtype=np.int64)
        for k, spin in enumerate(sp):
            x |= ((idx >> int(spin)) & 1) << k
        out.append(x.astype(np.uint16))
    return out


def exact_conditional(E, beta, shift, cs, site, prefix, d):
    """log p(x_site | x_0..x_{site-1} = prefix) over all d states of ``site``.

    E: all configuration energies; cs: ``cluster_states`` of every site."""
    u = 2.0 ** (-shift)
    mask = np.ones(E.shape[0], dtype=bool)
    for t, xv in enumerate(prefix):
        mask &= cs[t] == int(xv)
    xs = cs[site][mask]
    w = -beta * u * E[mask].astype(np.float64)
    out = np.full(d, -np.inf)
    for x in range(d):
        sel = w[xs == x]
        if sel.size:
            out[x] = logsumexp(sel)
    return out - logsumexp(w)


def potts_all_energies(inst):
    """Eq. 1 directly on a Potts instance: the int64 energy of every
    configuration (mixed radix, site 0 the slowest digit) and the state of
    every site in each ([n_sites] arrays [prod d]).  Limited to 2^24
    configurations."""
    d = [int(v) for v in inst.d]
    n = len(d)
    total = int(np.prod(d))
    if total > 2 ** 24:
        raise ValueError("brute force is limited to 2^24 configurations")
    cs = []
    stride = total
    for s in range(n):
        stride //= d[s]
        cs.append(((np.arange(total, dtype=np.int64) // stride) % d[s]).astype(np.uint16))
    offs = np.concatenate([[0], np.cumsum(d)]).astype(np.int64)
    local = np.asarray(inst.local_E, dtype=np.int64)
    E = np.zeros(total, dtype=np.int64)
    for s in range(n):
        E += local[offs[s] + cs[s].astype(np.int64)]
    off = 0
    pair = np.asarray(inst.pair_E, dtype=np.int64)
    for k in range(len(inst.em)):
        m, q = int(inst.em[k]), int(inst.en[k])
        T = pair[off:off + d[m] * d[q]].reshape(d[m], d[q])
        off += d[m] * d[q]
        E += T[cs[m].astype(np.int64), cs[q].astype(np.int64)]
    return E, cs


def chimera_strip(inst, beta: float):
    """Exact log Z and ground energy of a Chimera-like grid of width <= 3.

    Spin layout: cell (i, j) owns spins 8 (i cols + j) + k, k < 4 side A.
    Couplings may join spins of one row in any way, and side-A spins of
    vertically adjacent cells of rows i and i+1; anything else is rejected."""
    rows, cols = inst.grid_rows, inst.grid_cols
    if cols > 3:
        raise ValueError("width <= 3 only")
    J = _grid_ints(inst.J, inst.energy_shift)
    h = _grid_ints(inst.h, inst.energy_shift)
    u = 2.0 ** (-inst.energy_shift)
    row_of = np.arange(inst.n_spins) // (8 * cols)
    k_of = np.arange(inst.n_spins) % 8
    col_of = (np.arange(inst.n_spins) // 8) % cols
    # position of a spin inside its row's A block (4 cols) or B block
    posA = col_of * 4 + k_of
    posB = col_of * 4 + (k_of - 4)
    nA = 4 * cols
    sA = _spins(nA, 0, 2 ** nA)
    sB = _spins(nA, 0, 2 ** nA)
    intra = [dict(AA=np.zeros((nA, nA), np.int64), BB=np.zeros((nA, nA), np.int64),
                  AB=np.zeros((nA, nA), np.int64), hA=np.zeros(nA, np.int64),
                  hB=np.zeros(nA, np.int64)) for _ in range(rows)]
    vert = [np.zeros((nA, nA), np.int64) for _ in range(max(rows - 1, 0))]
    for e in range(len(J)):
        i, j = int(inst.ei[e]), int(inst.ej[e])
        if row_of[i] > row_of[j]:
            i, j = j, i
        ri, rj = row_of[i], row_of[j]
        Ai, Aj = k_of[i] < 4, k_of[j] < 4
        if ri == rj:
            t = intra[ri]
            if Ai and Aj:
                t["AA"][posA[i], posA[j]] += J[e]
            elif not Ai and not Aj:
                t["BB"][posB[i], posB[j]] += J[e]
            elif Ai:
                t["AB"][posA[i], posB[j]] += J[e]
            else:
                t["AB"][posA[j], posB[i]] += J[e]
        elif rj == ri + 1 and Ai and Aj:
            vert[ri][posA[i], posA[j]] += J[e]
        else:
            raise ValueError("coupling outside the strip's transfer structure")
    for s in range(inst.n_spins):
        t = intra[row_of[s]]
        if k_of[s] < 4:
            t["hA"][posA[s]] += h[s]
        else:
            t["hB"][posB[s]] += h[s]

    def row_tables(t):
        EA = np.einsum("xa,ab,xb->x", sA, t["AA"], sA) + sA @ t["hA"]
        EB = np.einsum("xa,ab,xb->x", sB, t["BB"], sB) + sB @ t["hB"]
        EAB = sA @ t["AB"] @ sB.T  # [A, B]
        Efull = EA[:, None] + EAB + EB[None, :]
        g = Efull.min(axis=1)
        w = -beta * u * Efull.astype(np.float64)
        m = w.max(axis=1)
        lf = m + np.log(np.exp(w - m[:, None]).sum(axis=1))
        return g, lf

    g, lv = row_tables(intra[0])
    G = g
    for r in range(1, rows):
        Ev = sA @ vert[r - 1] @ sA.T  # [A_prev, A_next]
        g, lf = row_tables(intra[r])
        G = g + (G[:, None] + Ev).min(axis=0)
        w = lv[:, None] - beta * u * Ev.astype(np.float64)
        m = w.max(axis=0)
        lv = lf + m + np.log(np.exp(w - m[None, :]).sum(axis=0))
    return {"logZ": logsumexp(lv), "ground": int(G.min())}


def _bits(x, n):
    """Spin values s = 2b - 1 of the n low bits of every x ([len(x), n])."""
    x = np.asarray(x, dtype=np.int64)[:, None]
    return 2 * ((x >> np.arange(n, dtype=np.int64)[None, :]) & 1) - 1


def interface_sum(inst, beta: float, max_bits: int = 22, fixed=None, target: int = 0):
    """Exact log Z, ground energy and the log-marginal of the states of the
    cluster on site `target` (row-major cell index; module header), from
    Eq. 2 on the instance's arrays, with the clusters of the sites in
    `fixed` ({site: state}) held at those states: then log Z and the ground
    energy are those of the configurations that agree with them, and the
    marginal is the conditional given them.  The sum runs over
    2^(total interface spins) <= 2^max_bits combinations."""
    fixed = fixed or {}
    J = _grid_ints(inst.J, inst.energy_shift)
    h = _grid_ints(inst.h, inst.energy_shift)
    u = 2.0 ** (-inst.energy_shift)
    cos = np.asarray(inst.cluster_of_spin)
    n_cl = int(cos.max()) + 1
    members = [np.sort(np.nonzero(cos == c)[0]) for c in range(n_cl)]
    pos = {int(sp): (c, k) for c in range(n_cl) for k, sp in enumerate(members[c])}
    ei, ej = np.asarray(inst.ei), np.asarray(inst.ej)
    inter = [e for e in range(len(J)) if cos[ei[e]] != cos[ej[e]]]
    iface = [sorted({pos[int(v)][1] for e in inter for v in (ei[e], ej[e]) if cos[v] == c}) for c in range(n_cl)]
    off = np.concatenate([[0], np.cumsum([len(f) for f in iface])]).astype(np.int64)
    T = int(off[-1])
    if T > max_bits:
        raise ValueError("too many interface spins")
    F, M, E0, a0 = [], [], None, None
    for c in range(n_cl):
        k = len(members[c])
        S = _bits(np.arange(2 ** k), k)
        E = S @ h[members[c]]
        for e in range(len(J)):
            if cos[ei[e]] == c and cos[ej[e]] == c:
                E = E + J[e] * S[:, pos[int(ei[e])][1]] * S[:, pos[int(ej[e])][1]]
        a = np.zeros(2 ** k, dtype=np.int64)
        for t, q in enumerate(iface[c]):
            a |= ((np.arange(2 ** k, dtype=np.int64) >> q) & 1) << t
        lw = -beta * u * E.astype(np.float64)
        site = int(inst.cluster_row[c]) * inst.grid_cols + int(inst.cluster_col[c])
        keep = np.ones(2 ** k, dtype=bool)
        if site in fixed:  # only the held state contributes
            keep[:] = False
            keep[int(fixed[site])] = True
        Fc = np.full(2 ** len(iface[c]), -np.inf)
        np.logaddexp.at(Fc, a[keep], lw[keep])
        Mc = np.full(2 ** len(iface[c]), np.iinfo(np.int64).max, dtype=np.int64)
        np.minimum.at(Mc, a[keep], E[keep])
        F.append(Fc)
        M.append(Mc)
        if site == target:
            E0, a0, c0 = E, a, c
    # inter-cluster couplers as (bit offset of each end in the combination, J)
    ends = [(off[cos[ei[e]]] + iface[cos[ei[e]]].index(pos[int(ei[e])][1]),
             off[cos[ej[e]]] + iface[cos[ej[e]]].index(pos[int(ej[e])][1]), J[e]) for e in inter]
    G0 = np.full(len(F[c0]), -np.inf)  # log-sum over the rest, per interface configuration of cell (0, 0)
    ground = None
    chunk = 1 << 18
    for lo in range(0, 2 ** T, chunk):
        g = np.arange(lo, min(2 ** T, lo + chunk), dtype=np.int64)
        Ein = np.zeros(len(g), dtype=np.int64)
        for bi, bj, Jv in ends:
            Ein += Jv * (2 * ((g >> bi) & 1) - 1) * (2 * ((g >> bj) & 1) - 1)
        lrest = -beta * u * Ein.astype(np.float64)
        emin = Ein.copy()
        ok = np.ones(len(g), dtype=bool)
        for c in range(n_cl):
            ac = (g >> off[c]) & ((1 << len(iface[c])) - 1)
            ok &= M[c][ac] != np.iinfo(np.int64).max  # combinations a held cluster cannot take
            emin += np.where(M[c][ac] != np.iinfo(np.int64).max, M[c][ac], 0)
            if c != c0:
                lrest += F[c][ac]
        if ok.any():
            g_min = int(emin[ok].min())
            ground = g_min if ground is None else min(ground, g_min)
        np.logaddexp.at(G0, (g >> off[c0]) & ((1 << len(iface[c0])) - 1), lrest)
    logZ = logsumexp(F[c0] + G0)
    logp = -beta * u * E0.astype(np.float64) + G0[a0] - logZ
    if target in fixed:
        logp = np.where(np.arange(len(logp)) == int(fixed[target]), 0.0, -np.inf)
    return {"logZ": logZ, "ground": ground, "logp": logp}


def brute_force_c(inst, beta: float):
    """``brute_force``'s ground energy, degeneracy and log Z from the C
    enumerator (bruteforce.c, OpenMP over the host's cores; up to 30 spins):
    {"ground", "degeneracy", "logZ"}."""
    import ctypes

    from . import native
    J = np.ascontiguousarray(_grid_ints(inst.J, inst.energy_shift), np.int64)
    h = np.ascontiguousarray(_grid_ints(inst.h, inst.energy_shift), np.int64)
    ei = np.ascontiguousarray(inst.ei, np.int32)
    ej = np.ascontiguousarray(inst.ej, np.int32)
    emin, deg, lz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    p32, p64 = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
    rc = native.lib().oracle_brute_force(inst.n_spins, len(J), ei.ctypes.data_as(p32), ej.ctypes.data_as(p32),
                                         J.ctypes.data_as(p64), h.ctypes.data_as(p64),
                                         beta * 2.0 ** (-inst.energy_shift), ctypes.byref(emin), ctypes.byref(deg),
                                         ctypes.byref(lz))
    if rc != 0:
        raise ValueError("the C brute force takes 1..30 spins")
    return {"ground": emin.value, "degeneracy": deg.value, "logZ": lz.value}
