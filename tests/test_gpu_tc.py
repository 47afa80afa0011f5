"""Tensor-core product step of the FP32 truncation (spg_tc_product) against
the same product in FP64 (NumPy) on the FP32 inputs.

Bound: |out - ref| <= 1e-5 * (|M| |Bt|^T) elementwise, i.e. FP32-level
accumulation of the split-TF32 products (a single TF32 product would miss
it by ~5e-4).  Two calls in a row must agree bit for bit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2502_02317_gb300 as spg
    return spg, torch, spg.Context(0, stream=torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("m,n,s", [(2048, 512, 80), (3000, 700, 48), (16384, 1024, 80), (1024, 4096, 16),
                                   (1100, 1000, 128), (512, 512, 48), (300, 260, 64)])
@pytest.mark.parametrize("trans", [False, True])
def test_tc_product_vs_fp64(env, m, n, s, trans):
    spg, torch, ctx = env
    rng = np.random.default_rng(m + 3 * n + 7 * s + int(trans))
    M = rng.standard_normal((m, n)).astype(np.float32)
    Bt = rng.standard_normal((s, m if trans else n)).astype(np.float32)
    Md, Bd = torch.tensor(M, device="cuda"), torch.tensor(Bt, device="cuda")
    out = spg.spg_tc_product(ctx, Md, Bd, trans).cpu().numpy()
    M64, B64 = M.astype(np.float64), Bt.astype(np.float64)
    A = M64.T if trans else M64
    ref = (A @ B64.T).T
    scale = (np.abs(A) @ np.abs(B64).T).T
    assert out.shape == ref.shape
    assert np.all(np.abs(out - ref) <= 1e-5 * scale)
    again = spg.spg_tc_product(ctx, Md, Bd, trans).cpu().numpy()
    assert np.array_equal(out, again)


def test_tc_product_rejects_small(env):
    spg, torch, ctx = env
    M = torch.zeros((512, 512), dtype=torch.float32, device="cuda")
    B = torch.zeros((40, 512), dtype=torch.float32, device="cuda")  # s not a multiple of 16
    with pytest.raises(spg.SpgError) as e:
        spg.spg_tc_product(ctx, M, B, False)
    assert e.value.code == -7
