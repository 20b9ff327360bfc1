"""The allocation-free Householder QR entry point, called through the C ABI.

Some callers cannot obtain device memory of their own (a plug-in given only
input and output pointers, a process whose device memory belongs to another
runtime, code that must stay out of the allocator).  For them the library
offers qrctm_householder_qr_noalloc, whose scratch is a fixed array inside the
library.  This file checks that it returns the same Q and R as the workspace
entry point on two calls in a row (the shared scratch keeps the first call's
contents), and that sizes beyond its stated limit are refused.  It is kept in
a file of its own, collected last.
"""
import ctypes

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


def _cuda(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _noalloc(q, M):
    import torch
    m, n = M.shape
    Mcm = M.t().contiguous()                 # column-major storage
    Qcm = torch.empty((n, m), dtype=torch.float64, device="cuda")
    R = torch.empty((n, n), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = q.lib.qrctm_householder_qr_noalloc(m, n, ctypes.c_void_p(Mcm.data_ptr()),
                                              ctypes.c_void_p(Qcm.data_ptr()),
                                              ctypes.c_void_p(R.data_ptr()), stream)
    return code, Qcm.t(), R


def test_noalloc_matches_workspace_qr_twice(q):
    rng = np.random.default_rng(2024)
    # two calls in a row with different shapes: the second must not see the
    # first call's leftovers in the shared scratch
    # shapes: 5184 x 144 and 1000 x 77 keep each CTA's panel rows in a small
    # shared-memory tile; 40000 x 16 in a tile between 48 and 160 KB (the
    # raised dynamic shared-memory limit); 200000 x 4 too tall for the tile,
    # so the panel runs on the scratch copy in global memory
    for m, n in ((5184, 144), (1000, 77), (40000, 16), (200000, 4)):
        M = _cuda(rng.standard_normal((m, n)))
        code, Qn, Rn = _noalloc(q, M)
        assert code == 0
        Qw, Rw = q.householder_qr(M)
        Qn, Rn, Qw, Rw = (t.cpu().numpy() for t in (Qn, Rn, Qw, Rw))
        assert np.abs(Qn - Qw).max() < 1e-11
        assert np.abs(Rn - Rw).max() < 1e-11 * np.abs(Rw).max()
        assert np.abs(Qn.T @ Qn - np.eye(n)).max() < 1e-13


def test_noalloc_rejects_sizes_beyond_its_scratch(q):
    import torch
    t = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # checked on the host before any device work
    assert q.lib.qrctm_householder_qr_noalloc(100000, 1024, p, p, p, s) == 6
    assert q.lib.qrctm_householder_qr_noalloc(3000, 2000, p, p, p, s) == 6
    assert q.lib.qrctm_householder_qr_noalloc(10, 20, p, p, p, s) == 1
