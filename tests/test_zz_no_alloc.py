"""spg_truncate_static (no device allocation inside the library) against
spg_truncate (context workspace) and against LAPACK, through the C ABI, on
two calls in a row.

Callers that cannot allocate device memory (a pool allocator owns it all, a
latency-critical loop, a plug-in after start-up) use the static variant; its
results must be those of the allocating entry point, and both must meet the
LAPACK bounds of test_gpu_truncate.py (kept singular values, the rank-keep
projector, orthonormal V, US = M V).  This file is collected last so that a
failure here stops a -x run only after every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def matrix(m, n, rate, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, min(m, n))))
    V, _ = np.linalg.qr(rng.standard_normal((n, min(m, n))))
    return (U * np.exp(-rate * np.arange(min(m, n)))) @ V.T


def test_static_truncation_matches_allocating_entry_point():
    import torch
    import paper_2502_02317_gb300 as spg
    ctx = spg.Context(0)
    # two calls in a row: a large one (subspace iteration) then a smaller
    # direct one, so stale scratch from the first call must not matter
    for (m, n, keep, rate, iters, seed) in [(256, 256, 32, 0.25, 6, 1), (96, 64, 12, 0.3, 0, 2)]:
        Mh = matrix(m, n, rate, seed)
        M = torch.tensor(Mh, device="cuda")
        V1, US1, s1 = [t.cpu().numpy() for t in spg.spg_truncate(ctx, M, keep, iters)]
        V2, US2, s2 = [t.cpu().numpy() for t in spg.spg_truncate_static(M, keep, iters)]
        np.testing.assert_allclose(s2, s1, rtol=1e-9, atol=1e-12 * s1[0])
        np.testing.assert_allclose(V2 @ V2.T, V1 @ V1.T, atol=1e-8)
        np.testing.assert_allclose(US2 @ V2.T, US1 @ V1.T, atol=1e-8 * s1[0])
        # LAPACK
        _, ref, Vt = np.linalg.svd(Mh)
        np.testing.assert_allclose(s2, ref[:keep], rtol=1e-9, atol=1e-12 * ref[0])
        np.testing.assert_allclose(V2.T @ V2, np.eye(keep), atol=1e-10)
        np.testing.assert_allclose(US2, Mh @ V2, atol=1e-10 * ref[0])
        np.testing.assert_allclose(V2 @ V2.T, Vt[:keep].T @ Vt[:keep], atol=1e-8)
    with pytest.raises(spg.SpgError) as e:
        spg.spg_truncate_static(torch.zeros((300, 8), dtype=torch.float64, device="cuda"), 4)
    assert e.value.code == -7
