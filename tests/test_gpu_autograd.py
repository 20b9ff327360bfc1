"""torch.autograd.Function wrapper of the energy (the boundary's Python side):
forward = converged environment + energy, backward = the library's adjoint.
Checked against the context calls it wraps and against central differences."""
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


@pytest.mark.parametrize("mode", ["implicit", "unroll"])
def test_energy_autograd(q, mode):
    import torch
    A0 = o.normalized_input(qi.raw_tensor(2, 2, 0))
    A = torch.tensor(A0, dtype=torch.float64, device="cuda", requires_grad=True)
    ctx = q.QRCTM(2, 2, 8, with_nnn=True, with_grad=True, grad_tol=1e-13, grad_max_iter=400)
    E = q.Energy.apply(A, ctx, 1.0, 0.5, 1e-13, 2000, mode, 12)
    E.backward()
    g = A.grad.detach().cpu().numpy()
    # the same calls by hand
    ctx2 = q.QRCTM(2, 2, 8, with_nnn=True, with_grad=True, grad_tol=1e-13, grad_max_iter=400)
    ctx2.init_env(A.detach())
    ctx2.run_to_convergence(tol=1e-13, max_iter=2000)
    assert abs(float(E) - ctx2.energy(1.0, 0.5)) < 1e-13
    _, g2 = ctx2.energy_grad(1.0, 0.5, mode=mode, k_unroll=12)
    assert np.abs(g - g2.cpu().numpy()).max() < 1e-12 * np.abs(g).max()
    # central differences of the wrapped function along a symmetric direction
    v = torch.tensor(o.normalized_input(qi.raw_direction(2, 2, 1010)), dtype=torch.float64,
                     device="cuda")
    eps = 1e-5
    with torch.no_grad():
        Ep = q.Energy.apply(A.detach() + eps * v, ctx, 1.0, 0.5, 1e-13, 2000, mode, 12)
        Em = q.Energy.apply(A.detach() - eps * v, ctx, 1.0, 0.5, 1e-13, 2000, mode, 12)
    fd = float(Ep - Em) / (2 * eps)
    tol = 1e-5 if mode == "implicit" else 1e-3   # unroll-12 is not the fixed-point derivative
    assert abs(fd - float((A.grad * v).sum())) < tol * max(1.0, abs(fd))
