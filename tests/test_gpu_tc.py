"""The split TF32x3 tensor-core contraction engine against an FP64 product of
the same FP32 inputs (through the C ABI).

Bound: each product carries <= ~2^-21 relative error from the split and the
FP32 accumulator adds ~2^-24 per addition; the test requires the error of
every entry to stay below 4e-6 * sum_k |a_k b_k| + 2e-6 * K^(1/2) * 2^-24-scale
slack, i.e. FP32-class accuracy, three orders of magnitude below one-pass
TF32 (2^-11)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch  # noqa: F401
    from paper_2505_00494_b300 import build
    build.build()
    import paper_2505_00494_b300 as q
    return q


@pytest.mark.parametrize("split_k", [False, True])
@pytest.mark.parametrize("M,N,K", [(128, 32, 32), (128, 48, 36), (300, 80, 72), (257, 144, 100),
                                   (1000, 256, 144), (5184, 144, 5184), (4096, 36, 72),
                                   (333, 300, 40), (260, 100, 64), (700, 192, 96),
                                   (200, 150, 40), (300, 400, 600), (130, 520, 1100)])
def test_tf32x3_matches_fp64(q, M, N, K, split_k):
    import torch
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    C = q.gemm_tf32x3(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                      split_k=split_k).cpu().numpy()
    err = np.abs(C - ref)
    print(M, N, K, split_k, "max err/scale", float((err / scale).max()),
          "max err/|C|", float((err / np.maximum(np.abs(ref), 1e-300)).max()))
    assert np.all(err <= 2e-6 * scale + 1e-30), float((err / scale).max())
