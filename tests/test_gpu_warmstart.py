"""Learned warm start through the C ABI against the FP64 oracle
(oracle/warmstart.py, oracle/boundary.py).

* features: bit-exact against the oracle's (FP32 of the same sums);
* the MLP's forward pass, loss and gradients (FP32 kernels) against the
  oracle's chain rule in FP64 on the same FP32 parameters and inputs: 2e-4
  relative to the largest entry of each array (FP32 accumulation over at most
  a few hundred terms); BF16 inference within 2e-2;
* one Adam step against the oracle's update (identical minibatch rows, so
  that the sampling does not enter);
* the exported boundary MPS of a row (FP64, the zipper's SVD sign gauge)
  against the oracle's zipper, site by site, to 1e-8;
* the sweep trace: the overlap <phi_k | W psi> never decreases over sweeps,
  from either start, and both starts reach the same optimum.
"""
import numpy as np
import pytest

import instances as I
from oracle import boundary, peps, tables
from oracle import warmstart as ws

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spg():
    import paper_2502_02317_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(spg):
    return spg.Context(0)


def rel_close(a, b, tol):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    scale = max(1e-30, float(np.max(np.abs(b))))
    err = float(np.max(np.abs(a - b))) / scale
    assert err <= tol, err


@pytest.mark.parametrize("make", [
    lambda: I.chimera(5, 3, couplings="gauss", h_sigma=0.1, cols=4),
    lambda: I.chimera(3, 8),
    lambda: I.square(4, 2, cols=6, h_sigma=0.3),
])
def test_features_match_oracle(spg, ctx, make):
    inst = make()
    prob = spg.spg_problem_ising(ctx, inst)
    for r in range(inst.grid_rows):
        got = spg.spg_warm_features(prob, r)
        ref = ws.features(inst, r).astype(np.float32)
        np.testing.assert_array_equal(got, ref)


def test_features_of_potts_problems_are_unsupported(spg, ctx):
    prob = spg.spg_problem_potts(ctx, I.king_potts(3, 3, 1))
    with pytest.raises(spg.SpgError):
        spg.spg_warm_features(prob, 0)


def oracle_params(net, flat):
    return {k: v.astype(np.float64) for k, v in net.split(flat).items()}


@pytest.mark.parametrize("n_in,H,n_out,n", [(37, 24, 50, 9), (800, 64, 1024, 33), (130, 96, 70, 128)])
def test_mlp_forward_and_gradients_match_oracle(spg, ctx, n_in, H, n_out, n):
    import torch
    net = spg.Mlp(ctx, n_in, H, n_out, seed=5)
    rng = np.random.default_rng(n_in + H)
    flat = net.params()
    flat = flat + (0.05 * rng.standard_normal(flat.size)).astype(np.float32)  # nonzero biases
    net.set_params(flat)
    X = rng.standard_normal((n, n_in)).astype(np.float32)
    T = rng.standard_normal((n, n_out)).astype(np.float32)
    p = oracle_params(net, flat)
    Yref, _ = ws.forward(p, X.astype(np.float64))
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    rel_close(net.forward(Xd).cpu().numpy(), Yref, 2e-5)
    rel_close(net.forward(Xd, bf16=True).cpu().numpy(), Yref, 2e-2)
    loss, g = net.loss_grad(Xd, Td)
    lref, gref = ws.loss_grad(p, X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - lref) <= 1e-5 * abs(lref)
    gs = net.split(g)
    for k in gref:
        rel_close(gs[k], gref[k], 2e-4)


def test_adam_step_matches_oracle(spg, ctx):
    """A one-sample data set makes every minibatch row the same sample, so
    one training step is the oracle's Adam step on that sample."""
    import torch
    net = spg.Mlp(ctx, 40, 16, 30, seed=9)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((1, 40)).astype(np.float32)
    T = rng.standard_normal((1, 30)).astype(np.float32)
    flat0 = net.params()
    p = oracle_params(net, flat0)
    net.train(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"), batch=4, steps=1, lr=1e-3)
    _, g = ws.loss_grad(p, X.astype(np.float64), T.astype(np.float64))
    ws.adam_step(p, g, {}, 1e-3)
    got = net.split(net.params())
    for k in p:
        np.testing.assert_allclose(got[k], p[k], atol=2e-6)


def test_training_fits_a_smooth_target(spg, ctx):
    import torch
    net = spg.Mlp(ctx, 64, 128, 256, seed=1)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((512, 64)).astype(np.float32)
    Wt = rng.standard_normal((256, 64)).astype(np.float32) / 8
    T = np.tanh(X @ Wt.T).astype(np.float32)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    l0, _ = net.loss_grad(Xd, Td)
    net.train(Xd, Td, batch=64, steps=400, lr=3e-3, seed=4)
    l1, _ = net.loss_grad(Xd, Td)
    assert l1 < 0.1 * l0, (l0, l1)


@pytest.mark.parametrize("make,chi,row", [
    (lambda: I.chimera(3, 21, couplings="gauss", h_sigma=0.1), 16, 1),
    (lambda: I.chimera(3, 21, couplings="gauss", h_sigma=0.1), 16, 2),
    (lambda: I.chimera(4, 22, couplings="gauss", h_sigma=0.1, cols=3), 12, 1),
])
def test_export_matches_oracle_zipper(spg, ctx, make, chi, row):
    """The exported row (FP64, no sweeps) is the oracle's zipper output site
    by site: the same truncated SVDs in the same sign gauge."""
    inst = make()
    fg = tables.from_ising(inst)
    bd = boundary.boundary_mpses(peps.build(fg, 1.0), chi, 0, down_to=row)
    prob = spg.spg_problem_ising(ctx, inst)
    out, dims = spg.spg_boundary_export(ctx, prob, spg.params(beta=1.0, chi=chi), row)
    out = out.cpu().numpy()
    for j, A in enumerate(bd[row].sites):
        cl, p, cr = A.shape
        assert tuple(dims[j]) == (p, cl, cr)
        got = out[j, :p, :cl, :cr]
        np.testing.assert_allclose(got, A.transpose(1, 0, 2), atol=1e-8)
        assert np.all(out[j, p:] == 0) and np.all(out[j, :, cl:] == 0) and np.all(out[j, :, :, cr:] == 0)


def test_sweep_trace_is_monotone_from_both_starts(spg, ctx):
    """A briefly trained network on small +-1 Chimera rows: its start and the
    zipper's both climb monotonically to the same best overlap."""
    import torch
    chi = 8
    feats, targs = [], []
    prm = spg.params(beta=1.0, chi=chi, num_sweeps=1, precision=spg.SPG_MIXED)
    for seed in range(6):
        inst = I.chimera(4, 300 + seed)
        prob = spg.spg_problem_ising(ctx, inst)
        for r in range(1, 4):
            out, _ = spg.spg_boundary_export(ctx, prob, prm, r)
            feats.append(spg.spg_warm_features(prob, r))
            targs.append(out.reshape(inst.grid_cols, -1).cpu().numpy())
    X = torch.tensor(np.concatenate(feats), device="cuda")
    T = torch.tensor(np.concatenate(targs), device="cuda")
    net = spg.Mlp(ctx, spg.SPG_WS_FEATURES, 64, 16 * chi * chi, seed=2)
    net.train(X, T, batch=16, steps=200, lr=1e-3, seed=1)
    spg.spg_set_warm_start(ctx, net)
    inst = I.chimera(4, 399)
    prob = spg.spg_problem_ising(ctx, inst)
    for row in (1, 2):
        tz = spg.spg_sweep_trace(ctx, prob, prm, row, 0, 12)
        tn = spg.spg_sweep_trace(ctx, prob, prm, row, 1, 12)
        for t in (tz, tn):
            assert np.all(np.isfinite(t))
            assert np.all(np.diff(t) >= -1e-5 * np.maximum(1.0, np.abs(t[1:])))
        assert abs(tn[-1] - tz[-1]) <= 1e-3 * max(1.0, abs(tz[-1]))
    # a warm-started solve returns exact energies of valid states
    res = spg.spg_solve(ctx, prob, spg.params(beta=1.0, chi=chi, num_sweeps=1, beam=64, warm_start=1,
                                              precision=spg.SPG_MIXED))
    st, E, _ = res.get()
    fg = tables.from_ising(inst)
    for k in range(len(E)):
        assert tables.energy(fg, st[k]) == E[k]
    spg.spg_set_warm_start(ctx, None)


def test_export_of_every_row_equals_the_single_row_exports(spg, ctx):
    inst = I.chimera(4, 31, cols=3)
    prob = spg.spg_problem_ising(ctx, inst)
    prm = spg.params(beta=1.0, chi=8, num_sweeps=1, precision=spg.SPG_MIXED)
    allrows, dall = spg.spg_boundary_export(ctx, prob, prm, 0)
    assert allrows.shape[0] == inst.grid_rows - 1
    for r in range(1, inst.grid_rows):
        one, d1 = spg.spg_boundary_export(ctx, prob, prm, r)
        np.testing.assert_array_equal(allrows[r - 1].cpu().numpy(), one.cpu().numpy())
        np.testing.assert_array_equal(dall[r - 1], d1)


def sweeps_to(trace, best, tol=1e-6):
    """Sweeps until F_k / F_best = exp(2 (trace_k - best)) >= 1 - tol
    (len(trace) + 1 when never)."""
    ok = np.nonzero(2.0 * (trace - best) >= np.log1p(-tol))[0]
    return int(ok[0]) + 1 if ok.size else len(trace) + 1


def test_what_training_gains(spg, ctx):
    """Trained against untrained network (same architecture and start) on
    rows of unseen larger instances (train 6x6, evaluate 8x8, +-1 Chimera,
    chi 16): the trained network predicts their boundary MPSs better (lower
    loss against the MPSs the method builds), and every start -- the
    zipper's, the trained and the untrained network's -- is a valid start of
    the compression, climbing monotonically; the sweeps to fidelity 1 - 1e-6
    of the best compression any start reaches are the measured effect
    (printed; the benchmark reports them at the configuration's sizes)."""
    import torch
    chi = 16
    prm = spg.params(beta=1.0, chi=chi, num_sweeps=1, precision=spg.SPG_MIXED)

    def data(seeds, L):
        X, T = [], []
        for seed in seeds:
            inst = I.chimera(L, seed)
            prob = spg.spg_problem_ising(ctx, inst)
            out, _ = spg.spg_boundary_export(ctx, prob, prm, 0)
            T.append(out.reshape((inst.grid_rows - 1) * inst.grid_cols, -1))
            X.append(np.concatenate([spg.spg_warm_features(prob, r) for r in range(1, inst.grid_rows)]))
        return torch.tensor(np.concatenate(X), device="cuda"), torch.cat(T).contiguous()

    Xd, Td = data(range(500, 512), 6)
    Xe, Te = data(range(900, 902), 8)  # unseen, larger
    untrained = spg.Mlp(ctx, spg.SPG_WS_FEATURES, 128, 16 * chi * chi, seed=3)
    trained = spg.Mlp(ctx, spg.SPG_WS_FEATURES, 128, 16 * chi * chi, seed=3)
    l0, _ = trained.loss_grad(Xd[:128], Td[:128])
    trained.train(Xd, Td, batch=32, steps=600, lr=1e-3, seed=2)
    l1, _ = trained.loss_grad(Xd[:128], Td[:128])
    assert l1 < 0.5 * l0, (l0, l1)
    e_trained, _ = trained.loss_grad(Xe, Te)
    e_untrained, _ = untrained.loss_grad(Xe, Te)
    assert e_trained < 0.7 * e_untrained, (e_trained, e_untrained)
    counts = {"zipper": [], "trained": [], "untrained": []}
    for seed in range(2):
        inst = I.chimera(8, 900 + seed)
        prob = spg.spg_problem_ising(ctx, inst)
        for row in (2, 5):
            spg.spg_set_warm_start(ctx, trained)
            tz, tt = spg.spg_sweep_trace(ctx, prob, prm, row, 2, 30)
            spg.spg_set_warm_start(ctx, untrained)
            tu = spg.spg_sweep_trace(ctx, prob, prm, row, 1, 30)
            for t in (tz, tt, tu):
                assert np.all(np.diff(t) >= -1e-5 * np.maximum(1.0, np.abs(t[1:])))
            best = max(tz.max(), tt.max(), tu.max())
            counts["zipper"].append(sweeps_to(tz, best))
            counts["trained"].append(sweeps_to(tt, best))
            counts["untrained"].append(sweeps_to(tu, best))
    spg.spg_set_warm_start(ctx, None)
    print("unseen-instance loss: trained", e_trained, "untrained", e_untrained)
    print("sweeps to 1-1e-6 of the best compression reached:", counts)
