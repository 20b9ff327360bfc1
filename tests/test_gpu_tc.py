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


@pytest.mark.parametrize("pre_a", [False, True])
@pytest.mark.parametrize("M,N,K", [(128, 32, 32), (300, 80, 72), (257, 144, 100),
                                   (5184, 144, 5184), (333, 300, 40), (700, 192, 96),
                                   (300, 400, 600), (130, 520, 1100), (144, 5184, 144),
                                   (2600, 3000, 144), (4100, 4200, 100)])
def test_presplit_matches_plain(q, M, N, K, pre_a):
    """Pre-split operands (heads and tails from tf32_split) give the same
    split, hence the same products, as the in-kernel split: bit-identical
    results (one pass over K), and the same FP64 bound."""
    import torch
    rng = np.random.default_rng(M * 5 + N * 11 + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    A[0, 0] = np.float32(1.0 + 2.0 ** -23)          # tail below the TF32 unit
    B[-1, -1] = np.float32(-(1.0 + 2.0 ** -11))      # a tie: head rounds away from zero
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    plain = q.gemm_tf32x3(Ad, Bd, split_k=False).cpu().numpy()
    Ah, Bh = Ad.clone(), Bd.clone()
    Alo = q.tf32_split(Ah) if pre_a else None
    if not pre_a:
        Ah = Ad
    Blo = q.tf32_split(Bh)
    # heads and tails are TF32 (13 low mantissa bits clear); the head is within
    # half a TF32 unit of x and head + tail within 2^-22 |x| (both rounded)
    hb, lb = Bh.cpu().numpy(), Blo.cpu().numpy()
    assert np.all(hb.view(np.uint32) & 0x1FFF == 0) and np.all(lb.view(np.uint32) & 0x1FFF == 0)
    B64 = B.astype(np.float64)
    assert np.all(np.abs(B64 - hb) <= 2.0 ** -11 * np.abs(B64))
    assert np.all(np.abs(B64 - hb - lb.astype(np.float64)) <= 2.0 ** -22 * np.abs(B64))
    assert hb[-1, -1] == np.float32(-(1.0 + 2.0 ** -10))      # tie rounded away from zero
    C = q.gemm_tf32x3_presplit(Ah, Alo, Bh, Blo, split_k=False).cpu().numpy()
    assert np.array_equal(C, plain)
    Cs = q.gemm_tf32x3_presplit(Ah, Alo, Bh, Blo, split_k=True).cpu().numpy()
    err = np.abs(Cs - ref)
    assert np.all(err <= 2e-6 * scale + 1e-30), float((err / scale).max())


def test_presplit_rejects_split_a_with_plain_b(q):
    import ctypes
    import torch
    A = torch.ones((128, 32), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = torch.empty((128, 128), dtype=torch.float64, device="cuda")
    vp = ctypes.c_void_p
    code = q.lib.qrctm_gemm_tf32x3_presplit(128, 128, 32, vp(A.data_ptr()), vp(A.data_ptr()), 32,
                                            vp(A.data_ptr()), None, 32, vp(C.data_ptr()), 128,
                                            None, 0, vp(err.data_ptr()), None)
    assert code == 1
