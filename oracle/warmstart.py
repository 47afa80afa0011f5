"""Learned warm start of the variational compression: coupling features,
the MLP that maps them to boundary-MPS site tensors, its gradients and one
Adam step, in FP64.

Test infrastructure only (see the package header).

The paper compresses each boundary MPS variationally (Sec. 3.1,
``MpsParameters(bond_dim, num_sweeps)``) starting from the SVD zipper.  The
warm start replaces that starting point by a prediction from the couplings
near the row; the paper has no learned part, so every step below is a
reading of the method's own objects:

* features of site (r, j) of the boundary MPS B_r (which contracts rows
  r .. L-1): for every cluster (i, k) with i in {r, r+1, r+2} and
  k in {j-2 .. j+2} (zeros outside the grid), in that order (i outer),
  52 numbers: the couplings between the cluster's spin positions q1 < q2
  (28 slots, pairs in lexicographic order), the fields of the 8 positions,
  and per position q the summed couplings to the cluster below (i+1, k) and
  to the cluster on the right (i, k+1) (8 + 8 slots); position q of a spin
  is its rank among the cluster's spins in ascending index (the order of the
  state encoding).  Then five position features: j == 0, j == cols-1,
  j == 1, j == cols-2, min(L - r, 8) / 8; then zeros up to N_FEATURES.
* network: X -> tanh(X W1^T + b1) -> tanh(. W2^T + b2) -> . W3^T + b3,
  loss 0.5/n * sum of squared errors over the n samples and all outputs;
* outputs: the site tensor A[s][a][a'] of B_r at (r, j) padded to
  [16][chi][chi] (zeros beyond the site's dims), in the gauge the method
  produces, with the sign of every left-bond row fixed so that its entry of
  largest magnitude (first on ties) is positive (the zipper's sign rule);
* Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
  p -= lr * m_hat / (sqrt(v_hat) + eps) with bias-corrected m_hat, v_hat.
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 800
PER_CLUSTER = 52
WINDOW_ROWS = 3
WINDOW_HALF = 2


def _pair_slot(q1: int, q2: int) -> int:
    """Index of the pair q1 < q2 of 8 positions in lexicographic order."""
    return q1 * 8 - q1 * (q1 + 1) // 2 + (q2 - q1 - 1)


def cluster_features(inst) -> np.ndarray:
    """[rows, cols, 52] per-cluster blocks (couplings, fields, down and right
    couplings by spin position)."""
    rows, cols = inst.grid_rows, inst.grid_cols
    out = np.zeros((rows, cols, PER_CLUSTER))
    cos = np.asarray(inst.cluster_of_spin)
    members = {}
    for s in range(inst.n_spins):
        members.setdefault(int(cos[s]), []).append(s)
    pos, cell = {}, {}
    for c, spins in members.items():
        r, k = int(inst.cluster_row[c]), int(inst.cluster_col[c])
        for q, s in enumerate(sorted(spins)):
            pos[s] = q
            cell[s] = (r, k)
    for s in range(inst.n_spins):
        r, k = cell[s]
        out[r, k, 28 + pos[s]] += inst.h[s]
    for a, b, J in zip(inst.ei, inst.ej, inst.J):
        a, b = int(a), int(b)
        (ra, ka), (rb, kb) = cell[a], cell[b]
        if (ra, ka) == (rb, kb):
            q1, q2 = sorted((pos[a], pos[b]))
            out[ra, ka, _pair_slot(q1, q2)] += J
        elif ka == kb and abs(ra - rb) == 1:
            up, qu = (a, pos[a]) if ra < rb else (b, pos[b])
            out[cell[up][0], cell[up][1], 36 + qu] += J
        elif ra == rb and abs(ka - kb) == 1:
            left, ql = (a, pos[a]) if ka < kb else (b, pos[b])
            out[cell[left][0], cell[left][1], 44 + ql] += J
    return out


def features(inst, r: int) -> np.ndarray:
    """[cols, N_FEATURES] inputs of the sites of boundary row r."""
    rows, cols = inst.grid_rows, inst.grid_cols
    cf = cluster_features(inst)
    X = np.zeros((cols, N_FEATURES))
    for j in range(cols):
        v = []
        for i in range(r, r + WINDOW_ROWS):
            for k in range(j - WINDOW_HALF, j + WINDOW_HALF + 1):
                v.append(cf[i, k] if (0 <= i < rows and 0 <= k < cols) else np.zeros(PER_CLUSTER))
        v = np.concatenate(v)
        extra = [j == 0, j == cols - 1, j == 1, j == cols - 2, min(rows - r, 8) / 8.0]
        X[j, :v.size] = v
        X[j, v.size:v.size + 5] = np.asarray(extra, dtype=np.float64)
    return X


def init_params(n_in: int, n_hidden: int, n_out: int, rng) -> dict:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    def u(shape, fan):
        b = 1.0 / np.sqrt(fan)
        return rng.uniform(-b, b, size=shape)
    return {"W1": u((n_hidden, n_in), n_in), "b1": np.zeros(n_hidden),
            "W2": u((n_hidden, n_hidden), n_hidden), "b2": np.zeros(n_hidden),
            "W3": u((n_out, n_hidden), n_hidden), "b3": np.zeros(n_out)}


def forward(p: dict, X: np.ndarray):
    """(Y, cache) for inputs X [n, n_in]."""
    A1 = X @ p["W1"].T + p["b1"]
    H1 = np.tanh(A1)
    A2 = H1 @ p["W2"].T + p["b2"]
    H2 = np.tanh(A2)
    Y = H2 @ p["W3"].T + p["b3"]
    return Y, (X, H1, H2)


def loss_grad(p: dict, X: np.ndarray, T: np.ndarray):
    """(loss, grads) with loss = 0.5/n * sum (Y - T)^2, by the chain rule."""
    n = X.shape[0]
    Y, (X, H1, H2) = forward(p, X)
    D = Y - T
    loss = 0.5 * float(np.sum(D * D)) / n
    dY = D / n
    g = {"W3": dY.T @ H2, "b3": dY.sum(axis=0)}
    dH2 = dY @ p["W3"]
    dA2 = dH2 * (1.0 - H2 * H2)
    g["W2"] = dA2.T @ H1
    g["b2"] = dA2.sum(axis=0)
    dH1 = dA2 @ p["W2"]
    dA1 = dH1 * (1.0 - H1 * H1)
    g["W1"] = dA1.T @ X
    g["b1"] = dA1.sum(axis=0)
    return loss, g


ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def adam_step(p: dict, g: dict, state: dict, lr: float) -> None:
    """One Adam update of p in place; state holds m, v per parameter and t."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = ADAM_B1 * m + (1.0 - ADAM_B1) * g[k]
        v[...] = ADAM_B2 * v + (1.0 - ADAM_B2) * g[k] * g[k]
        mh = m / (1.0 - ADAM_B1 ** t)
        vh = v / (1.0 - ADAM_B2 ** t)
        p[k] -= lr * mh / (np.sqrt(vh) + ADAM_EPS)


def sign_fixed_row(sites: list) -> list:
    """The sign gauge of the targets on a boundary MPS given as sites
    [chi_l, p, chi_r] (the oracle's layout): for j = L-1 .. 1, each left-bond
    row a of site j (entries over (s, a'), s outer) whose largest-magnitude
    entry (first on ties) is negative is negated, together with column a of
    site j-1, so that the MPS is unchanged."""
    out = [s.copy() for s in sites]
    for j in range(len(out) - 1, 0, -1):
        A = out[j]
        for a in range(A.shape[0]):
            row = A[a].reshape(-1)  # entries (s, a') with s outer
            idx = int(np.argmax(np.abs(row)))
            if row[idx] < 0:
                A[a] = -A[a]
                out[j - 1][:, :, a] = -out[j - 1][:, :, a]
    return out
