"""Corner spectrum (convergence test, QR-CTMRG paragraph) on the GPU against
LAPACK: sorted |eig((C + C^T)/2)| of the normalised corner, for every
tridiagonalisation variant (8-CTA cluster for chi <= 360, 16-CTA cluster up
to 512, one CTA beyond).  Tolerance 1e-13 absolute on a unit-norm spectrum
(eigenvalues to the accuracy of a backward-stable FP64 method)."""
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


@pytest.mark.parametrize("chi,seed", [(5, 0), (200, 1), (360, 2), (400, 3), (512, 4), (600, 5), (640, 6), (700, 7)])
def test_corner_spectrum_matches_lapack(q, chi, seed):
    rng = np.random.default_rng(seed)
    A = o.normalized_input(qi.raw_tensor(2, 2, seed))
    C = rng.standard_normal((chi, chi))
    # a decaying spectrum with near-degenerate pairs, like a converged corner
    U, _ = np.linalg.qr(rng.standard_normal((chi, chi)))
    lam = np.exp(-0.05 * np.arange(chi)) * np.where(np.arange(chi) % 2 == 0, 1.0, -1.0)
    lam[1::7] = lam[0::7][: len(lam[1::7])] * (1 + 1e-9)
    C = U @ np.diag(lam) @ U.T + 1e-3 * (C + C.T)
    T = rng.standard_normal((chi, 4, chi))
    ctx = q.QRCTM(2, 2, chi)
    ctx.init_env(cuda(A), cuda(C), cuda(T))
    _, _, s = ctx.get_env(spectrum=True)
    Cs = 0.5 * (C + C.T)
    Cs /= np.linalg.norm(Cs)
    ref = np.sort(np.abs(np.linalg.eigvalsh(Cs)))[::-1]
    assert np.abs(s - ref).max() < 1e-13, np.abs(s - ref).max()
