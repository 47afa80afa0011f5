"""The zipper's truncated SVD (spg_truncate) against LAPACK (numpy.linalg.svd).

Compared quantities are unique: the kept singular values and the rank-keep
projection M V V^T (independent of the sign or rotation freedom of
degenerate singular vectors); V must have orthonormal columns and US = M V.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2502_02317_gb300 as spg
    return spg, torch, spg.Context(0, stream=torch.cuda.current_stream().cuda_stream)


def decaying(m, n, rate, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, min(m, n))))
    V, _ = np.linalg.qr(rng.standard_normal((n, min(m, n))))
    s = np.exp(-rate * np.arange(min(m, n)))
    return (U * s) @ V.T


@pytest.mark.parametrize("m,n,keep,rate,iters", [
    (16, 16, 16, 0.3, 0),       # square, no truncation
    (256, 64, 32, 0.2, 0),      # direct path (n <= 128)
    (64, 256, 16, 0.5, 6),      # subspace iteration, wide
    (512, 512, 32, 0.25, 6),    # the zipper's 512 x 512 at chi = 32
    (100, 300, 7, 0.4, 8),      # ragged sizes
    (5, 400, 5, 0.1, 4),        # fewer rows than the block
    (4096, 512, 64, 0.05, 6),   # long vectors: multi-CTA tall QR
    (3000, 2500, 40, 0.08, 4),  # ragged tall QR on both sides (one level of recursion)
])
def test_truncate_vs_lapack(env, m, n, keep, rate, iters):
    spg, torch, ctx = env
    M = decaying(m, n, rate, m * 7 + n)
    Md = torch.tensor(M, device="cuda")
    V, US, sig = spg.spg_truncate(ctx, Md, keep, iters)
    V, US, sig = V.cpu().numpy(), US.cpu().numpy(), sig.cpu().numpy()
    ref = np.linalg.svd(M, compute_uv=False)[:keep]
    np.testing.assert_allclose(sig, ref, rtol=1e-9, atol=1e-12 * ref[0])
    np.testing.assert_allclose(V.T @ V, np.eye(keep), atol=1e-10)
    np.testing.assert_allclose(US, M @ V, atol=1e-10 * ref[0])
    _, _, Vt = np.linalg.svd(M)
    P_ref = Vt[:keep].T @ Vt[:keep]
    np.testing.assert_allclose(V @ V.T, P_ref, atol=1e-8)


def test_truncate_rejects_bad_sizes(env):
    spg, torch, ctx = env
    Md = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(spg.SpgError):
        spg.spg_truncate(ctx, Md, 9)
