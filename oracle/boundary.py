"""Boundary MPSs: MPO-MPS zipper with SVD truncation, variational sweeps.

Test infrastructure only (see the package header).

Paper: Sec. 2 and Fig. 1(d) (marginals from an approximate contraction of the
PEPS with boundary MPSs), Sec. 3.1 (``MpsParameters(bond_dim, num_sweeps)``,
``MpsContractor(SVDTruncate, ...)``, ``Layout``: the network is divided into
boundary MPSs row by row).

An MPS site has shape [chi_left, p, chi_right]; the physical index p of the
boundary MPS below row i is the down index of row i's MPO (the row projection
of cluster (i, j) on its vertical edge downwards).

Readings taken here:
* bottom-up order: B_L is the trivial MPS (all bonds and the physical index
  of dimension 1, value 1); B_i = trunc(W_i . B_{i+1}) for i = L-1 ... 1 (and
  down to 0 for log Z);
* zipper (SVDTruncate): first bring B_{i+1} to left-canonical form (QR sweep
  left to right, R with non-negative diagonal, norm into the log-norm), so
  that the truncation below sees an orthonormal gauge of the MPS being
  applied; then sweep the row right to left with a carry C[r, a', k]
  (1 x 1 x 1 at the right end).  At site j form
      M[(l, a), (u, k)] = sum_{r, a', s} W[l, r, u, s] B[a, s, a'] C[r, a', k],
  take its full SVD, keep min(chi, rank dims) largest singular values, make
  the rows of V^T the new site and U S the next carry.  Each kept right
  singular vector is flipped so that its entry of largest magnitude (lowest
  index on ties) is positive.  Site 0 absorbs the last carry, then is
  normalised.  The carry is divided by its largest singular value after
  every step; all scales go into the MPS's log-norm;
* a cut is flagged degenerate when s_chi - s_{chi+1} <= 1e-12 s_1;
* one variational sweep (num_sweeps) = left-to-right then right-to-left
  one-site updates of phi that maximise |<phi|W psi>| with the other sites
  orthonormal (QR with positive diagonal moves the centre); the result is
  right-orthonormal on sites 1.. with the norm in site 0, as after the zipper.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import peps as peps_mod

DEGENERATE_RTOL = 1e-12


@dataclass
class MPS:
    sites: list  # [chi_l, p, chi_r]
    lognorm: float  # true MPS = exp(lognorm) * contraction(sites)
    degenerate: bool = False


def trivial_mps(L: int) -> MPS:
    return MPS([np.ones((1, 1, 1)) for _ in range(L)], 0.0)


def sign_fix(U, Vt):
    """Flip each (U column, V^T row) pair so V^T's largest-|.| entry is > 0."""
    for k in range(Vt.shape[0]):
        idx = int(np.argmax(np.abs(Vt[k])))  # first maximum = lowest index
        if Vt[k, idx] < 0:
            Vt[k] = -Vt[k]
            U[:, k] = -U[:, k]
    return U, Vt


def left_canonical(B: MPS) -> MPS:
    """QR sweep left to right; the last site keeps the norm, which is then
    moved into the log-norm."""
    sites = [s.copy() for s in B.sites]
    L = len(sites)
    for j in range(L - 1):
        a, u, b = sites[j].shape
        Q, R = np.linalg.qr(sites[j].reshape(a * u, b))
        sg = np.sign(np.diag(R))
        sg[sg == 0] = 1.0
        Q, R = Q * sg[None, :], R * sg[:, None]
        sites[j] = Q.reshape(a, u, Q.shape[1])
        sites[j + 1] = np.einsum("ab,bsc->asc", R, sites[j + 1])
    nrm = float(np.linalg.norm(sites[L - 1]))
    sites[L - 1] = sites[L - 1] / nrm
    return MPS(sites, B.lognorm + float(np.log(nrm)), B.degenerate)


def zipper(Ws: list, B: MPS, chi: int) -> MPS:
    """One MPO application with SVD truncation, right to left."""
    B = left_canonical(B)
    L = len(Ws)
    C = np.ones((1, 1, 1))
    out = [None] * L
    lognorm = B.lognorm
    degenerate = False
    for j in reversed(range(L)):
        W, A = Ws[j], B.sites[j]
        T1 = np.tensordot(A, C, axes=([2], [1]))  # [a, s, r, k]
        M = np.tensordot(W, T1, axes=([1, 3], [2, 1]))  # [l, u, a, k]
        M = M.transpose(0, 2, 1, 3)  # [l, a, u, k]
        DL, chil, DU, K = M.shape
        Mm = M.reshape(DL * chil, DU * K)
        if j == 0:
            nrm = np.linalg.norm(Mm)
            out[0] = (Mm / nrm).reshape(DL * chil, DU, K)
            lognorm += float(np.log(nrm))
            break
        U, S, Vt = np.linalg.svd(Mm, full_matrices=False)
        keep = min(chi, S.shape[0])
        if keep < S.shape[0] and S[keep - 1] - S[keep] <= DEGENERATE_RTOL * S[0]:
            degenerate = True
        U, S, Vt = U[:, :keep].copy(), S[:keep], Vt[:keep].copy()
        U, Vt = sign_fix(U, Vt)
        out[j] = Vt.reshape(keep, DU, K)
        s1 = S[0]
        C = (U * (S / s1)[None, :]).reshape(DL, chil, keep)
        lognorm += float(np.log(s1))
    return MPS(out, lognorm, degenerate)


def contract_value(mps: MPS) -> float:
    """Value of an MPS whose physical indices all have dimension 1."""
    v = np.ones((1,))
    for A in mps.sites:
        assert A.shape[1] == 1
        v = v @ A[:, 0, :]
    return float(v[0])


def _apply_site(L_env, phi, W, A):
    """L_{j+1}[a', r, b'] = sum L[a,l,b] phi[a,u,a'] W[l,r,u,s] A[b,s,b']."""
    t = np.tensordot(L_env, phi, axes=([0], [0]))  # [l, b, u, a']
    t = np.tensordot(t, W, axes=([0, 2], [0, 2]))  # [b, a', r, s]
    t = np.tensordot(t, A, axes=([0, 3], [0, 1]))  # [a', r, b']
    return t


def _apply_site_right(R_env, phi, W, A):
    """R_{j-1}[a, l, b] = sum phi[a,u,a'] W[l,r,u,s] A[b,s,b'] R[a',r,b']."""
    t = np.tensordot(A, R_env, axes=([2], [2]))  # [b, s, a', r]
    t = np.tensordot(W, t, axes=([1, 3], [3, 1]))  # [l, u, b, a']
    t = np.tensordot(phi, t, axes=([1, 2], [1, 3]))  # [a, l, b]
    return t


def _local(L_env, W, A, R_env):
    """Projection of W psi onto site j: sum L[a,l,b] W[l,r,u,s] A[b,s,b'] R[a',r,b']."""
    t = np.tensordot(A, R_env, axes=([2], [2]))  # [b, s, a', r]
    t = np.tensordot(W, t, axes=([1, 3], [3, 1]))  # [l, u, b, a']
    t = np.tensordot(L_env, t, axes=([1, 2], [0, 2]))  # [a, u, a']
    return t


def _norm_env(E):
    m = float(np.max(np.abs(E)))
    return E / m, float(np.log(m))


def variational(Ws: list, B: MPS, phi: MPS, sweeps: int):
    """num_sweeps one-site sweeps (reading in the module header).

    Returns (new MPS, fidelity history) where fidelity is
    |<phi|W psi>|^2 / (<phi|phi> <W psi|W psi>) after each half sweep.  A QR
    step may shrink a bond to the rank the site allows."""
    L = len(Ws)
    sites = [s.copy() for s in phi.sites]
    if sweeps == 0:
        return MPS(sites, phi.lognorm, phi.degenerate), []
    psi_norm2 = _norm2_exact(Ws, B)
    fid = []
    logc = 0.0
    for _ in range(sweeps):
        # right environments of the current right-orthonormal phi
        R = [None] * L
        R[L - 1] = np.ones((1, 1, 1))
        for j in range(L - 1, 0, -1):
            R[j - 1], _ = _norm_env(_apply_site_right(R[j], sites[j], Ws[j], B.sites[j]))
        # left to right: local optimum, then QR moves the centre right
        Lcache = [None] * L
        Lcache[0] = np.ones((1, 1, 1))
        Ls = 0.0
        for j in range(L - 1):
            c = _local(Lcache[j], Ws[j], B.sites[j], R[j])
            a, u, b = c.shape
            Q, Rm = np.linalg.qr(c.reshape(a * u, b))
            sg = np.sign(np.diag(Rm))
            sg[sg == 0] = 1.0
            Q = Q * sg[None, :]
            sites[j] = Q.reshape(a, u, Q.shape[1])
            Lcache[j + 1], sc = _norm_env(_apply_site(Lcache[j], sites[j], Ws[j], B.sites[j]))
            Ls += sc
        c = _local(Lcache[L - 1], Ws[L - 1], B.sites[L - 1], R[L - 1])
        fid.append(float(np.sum(c * c)) * np.exp(2 * Ls) / psi_norm2)
        sites[L - 1] = c
        # right to left: local optimum, then LQ moves the centre left
        Rj = np.ones((1, 1, 1))
        Rsum = 0.0
        for j in range(L - 1, 0, -1):
            c = _local(Lcache[j], Ws[j], B.sites[j], Rj)
            a, u, b = c.shape
            Q, Rm = np.linalg.qr(c.reshape(a, u * b).T)
            sg = np.sign(np.diag(Rm))
            sg[sg == 0] = 1.0
            Q = Q * sg[None, :]
            sites[j] = Q.T.reshape(Q.shape[1], u, b)
            Rj, sc = _norm_env(_apply_site_right(Rj, sites[j], Ws[j], B.sites[j]))
            Rsum += sc
        c = _local(Lcache[0], Ws[0], B.sites[0], Rj)
        nrm = float(np.linalg.norm(c))
        fid.append(nrm * nrm * np.exp(2 * Rsum) / psi_norm2)
        sites[0] = c / nrm
        logc = float(np.log(nrm)) + Rsum
    return MPS(sites, B.lognorm + logc, phi.degenerate), fid


def _norm2_exact(Ws, B: MPS):
    """<W psi | W psi> with psi = B's sites (scale of B.lognorm excluded)."""
    E = np.ones((1, 1, 1, 1))  # [a (ket psi), l (ket W), r (bra W), b (bra psi)]
    log = 0.0
    for W, A in zip(Ws, B.sites):
        t = np.tensordot(E, A, axes=([0], [0]))  # [l, r, b, s, c]
        t = np.tensordot(t, W, axes=([0, 3], [0, 3]))  # [r, b, c, p, u]
        t = np.tensordot(t, W, axes=([0, 4], [0, 2]))  # [b, c, p, q, v]
        E = np.tensordot(t, A, axes=([0, 4], [0, 1]))  # [c, p, q, d]
        m = float(np.max(np.abs(E)))
        E /= m
        log += np.log(m)
    return float(E.reshape(-1)[0]) * np.exp(log)


def boundary_mpses(p: "peps_mod.PEPS", chi: int, num_sweeps: int = 0, down_to: int = 1):
    """B_i for i = L .. down_to (dict i -> MPS); B_L is the trivial MPS."""
    rows, cols = p.rows, p.cols
    out = {rows: trivial_mps(cols)}
    for i in range(rows - 1, down_to - 1, -1):
        Ws = peps_mod.mpo_row(p, i)
        z = zipper(Ws, out[i + 1], chi)
        if num_sweeps > 0:
            z, _ = variational(Ws, out[i + 1], z, num_sweeps)
        out[i] = z
    return out


def log_partition(p: "peps_mod.PEPS", chi: int, num_sweeps: int = 0) -> float:
    """log Z from the boundary MPS of row 0 (top closed)."""
    Bs = boundary_mpses(p, chi, num_sweeps, down_to=0)
    B0 = Bs[0]
    return B0.lognorm + float(np.log(contract_value(B0))) + p.log_offset
