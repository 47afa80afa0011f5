"""Pins of the warm-start oracle (oracle/warmstart.py) against closed forms,
finite differences and the instance arrays themselves (no GPU)."""
import numpy as np

import instances as I
from oracle import warmstart as ws


def small_params(seed=0, n_in=7, H=5, n_out=4):
    rng = np.random.default_rng(seed)
    p = ws.init_params(n_in, H, n_out, rng)
    for k in p:  # nonzero biases so that every term is exercised
        p[k] = p[k] + 0.1 * rng.standard_normal(p[k].shape)
    return p


def test_gradients_match_central_differences():
    """Every gradient entry against (L(p + h e) - L(p - h e)) / 2h in FP64."""
    rng = np.random.default_rng(1)
    p = small_params()
    X, T = rng.standard_normal((6, 7)), rng.standard_normal((6, 4))
    _, g = ws.loss_grad(p, X, T)
    h = 1e-6
    for k in p:
        num = np.zeros_like(p[k])
        for idx in np.ndindex(p[k].shape):
            old = p[k][idx]
            p[k][idx] = old + h
            lp, _ = ws.loss_grad(p, X, T)
            p[k][idx] = old - h
            lm, _ = ws.loss_grad(p, X, T)
            p[k][idx] = old
            num[idx] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(g[k], num, rtol=1e-6, atol=1e-9)


def test_bias_only_network_reaches_the_mean():
    """With W3 = 0 the output is b3 for every sample: the b3 gradient is
    mean(b3 - T), zero at b3 = mean(T), where the loss is half the summed
    per-output variance."""
    rng = np.random.default_rng(2)
    p = small_params()
    p["W3"][:] = 0.0
    X, T = rng.standard_normal((9, 7)), rng.standard_normal((9, 4))
    _, g = ws.loss_grad(p, X, T)
    np.testing.assert_allclose(g["b3"], p["b3"] - T.mean(axis=0), atol=1e-14)
    assert np.all(g["W1"] == 0) and np.all(g["W2"] == 0)
    p["b3"] = T.mean(axis=0)
    loss, g = ws.loss_grad(p, X, T)
    np.testing.assert_allclose(g["b3"], 0.0, atol=1e-14)
    np.testing.assert_allclose(loss, 0.5 * T.var(axis=0).sum(), rtol=1e-12)


def test_first_adam_step_is_a_signed_step():
    """From zero moments the bias-corrected first step is -lr g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    p = small_params()
    X, T = rng.standard_normal((5, 7)), rng.standard_normal((5, 4))
    _, g = ws.loss_grad(p, X, T)
    q = {k: v.copy() for k, v in p.items()}
    ws.adam_step(q, g, {}, 0.01)
    for k in p:
        np.testing.assert_allclose(q[k], p[k] - 0.01 * g[k] / (np.abs(g[k]) + ws.ADAM_EPS), atol=1e-15)


def test_adam_fits_a_fixed_batch():
    rng = np.random.default_rng(4)
    p = ws.init_params(7, 16, 4, rng)
    X = rng.standard_normal((32, 7))
    T = np.tanh(X[:, :4]) + 0.5
    st = {}
    l0, _ = ws.loss_grad(p, X, T)
    for _ in range(300):
        _, g = ws.loss_grad(p, X, T)
        ws.adam_step(p, g, st, 0.01)
    l1, _ = ws.loss_grad(p, X, T)
    assert l1 < 0.05 * l0


def test_pair_slots_are_a_bijection():
    slots = [ws._pair_slot(a, b) for a in range(8) for b in range(a + 1, 8)]
    assert sorted(slots) == list(range(28))


def test_features_read_the_couplings_of_the_window():
    """Each slot holds the coupling it names, read straight from the
    instance's edge list; clusters outside the grid are zero."""
    inst = I.chimera(3, 5, couplings="gauss", h_sigma=0.1)
    J = {(int(a), int(b)): float(v) for a, b, v in zip(inst.ei, inst.ej, inst.J)}
    X = ws.features(inst, 0)
    assert X.shape == (3, ws.N_FEATURES)
    c = lambda i, k: 8 * (i * 3 + k)  # noqa: E731  first spin of cluster (i, k)
    # site (0, 1): window rows 0..2, columns -1..3; block (i, k) at offset
    blk = lambda i, k: ((i - 0) * 5 + (k - 1 + 2)) * ws.PER_CLUSTER  # noqa: E731
    x = X[1]
    for ka in range(4):
        for kb in range(4, 8):
            assert x[blk(0, 1) + ws._pair_slot(ka, kb)] == J[(c(0, 1) + ka, c(0, 1) + kb)]
        assert x[blk(1, 2) + 36 + ka] == J[(c(1, 2) + ka, c(2, 2) + ka)]          # down
        assert x[blk(2, 0) + 44 + 4 + ka] == J[(c(2, 0) + 4 + ka, c(2, 1) + 4 + ka)]  # right
    for q in range(8):
        assert x[blk(1, 1) + 28 + q] == inst.h[c(1, 1) + q]
    # column 3 of the grid does not exist: its block is zero
    assert np.all(x[blk(0, 3):blk(0, 3) + ws.PER_CLUSTER] == 0)
    # the bottom row has no cluster below
    assert np.all(X[:, ::1][0, blk(2, 1) + 36: blk(2, 1) + 44] == 0)
    tail = 15 * ws.PER_CLUSTER
    # 3 columns: j = 1 is both the second and the second-to-last column
    np.testing.assert_array_equal(X[:, tail:tail + 5], [[1, 0, 0, 0, 3 / 8], [0, 0, 1, 1, 3 / 8],
                                                         [0, 1, 0, 0, 3 / 8]])
    assert np.all(X[:, tail + 5:] == 0)


def test_sign_gauge_keeps_the_mps():
    """The sign fix of the targets changes the sites, not the state: every
    amplitude of the MPS is unchanged, and every fixed row's largest entry
    is positive."""
    rng = np.random.default_rng(6)
    sites = [rng.standard_normal((1, 3, 4)), rng.standard_normal((4, 3, 5)), rng.standard_normal((5, 3, 1))]
    fixed = ws.sign_fixed_row(sites)

    def amp(ss, cfg):
        v = np.ones(1)
        for A, s in zip(ss, cfg):
            v = v @ A[:, s, :]
        return v[0]
    for cfg in np.ndindex(3, 3, 3):
        assert np.isclose(amp(fixed, cfg), amp(sites, cfg), rtol=1e-12)
    for j in (1, 2):
        for a in range(fixed[j].shape[0]):
            row = fixed[j][a].reshape(-1)
            assert row[np.argmax(np.abs(row))] > 0
