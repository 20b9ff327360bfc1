"""The standard C4v CTMRG step (the comparison method, full eigendecomposition
of the enlarged corner) on the GPU against the oracle's eigen step: one step
from the same environment (gauge-invariant quantities: sorted |eig C| and the
energies, 1e-10) and the environment converged from the bulk boundary by both
(1e-9; the eigen steps are deterministic up to eigenvector signs)."""
import numpy as np
import pytest

from oracle import qrctm_oracle as o
import qrctm_inputs as qi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch  # noqa: F401
    from paper_2505_00494_b300 import build
    build.build()
    import paper_2505_00494_b300 as q
    return q


def cuda(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("D,chi,seed", [(2, 16, 0), (3, 18, 1), (4, 32, 2)])
def test_single_eigen_step(q, D, chi, seed):
    A = o.normalized_input(qi.raw_tensor(2, D, seed))
    C, T = o.warmup(A, chi)
    ctx = q.QRCTM(2, D, chi, method="eigen", with_nnn=True)
    ctx.init_env(cuda(A), cuda(C), cuda(T))
    ctx.step(1, want_delta=False)
    C1, T1 = o.eigen_step(C, T, o.double_layer(A), chi)
    _, _, s = ctx.get_env(spectrum=True)
    assert np.abs(s - o.corner_spectrum(C1)).max() < 1e-10
    for J2 in (0.0, 0.5):
        assert abs(ctx.energy(1.0, J2) - o.energy(C1, T1, A, 1.0, J2)) < 1e-10


def test_converged_eigen_ctmrg(q):
    A = o.normalized_input(qi.raw_tensor(2, 2, 0))
    C, T, info = o.ctmrg(A, 16, "eigen", tol=1e-13, max_iter=2000)
    ctx = q.QRCTM(2, 2, 16, method="eigen", check_every=1, with_nnn=True)
    ctx.init_env(cuda(A))
    its, dl = ctx.run_to_convergence(tol=1e-13, max_iter=2000)
    _, _, s = ctx.get_env(spectrum=True)
    assert np.abs(s - o.corner_spectrum(C)).max() < 1e-9
    assert abs(ctx.energy(1.0, 0.0) - o.energy(C, T, A, 1.0, 0.0)) < 1e-9
