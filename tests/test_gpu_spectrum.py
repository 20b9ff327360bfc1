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


def _spec(C, n):
    """Sorted |eig| of the symmetrised, unit-norm corner, padded with zeros to n."""
    Cs = 0.5 * (C + C.T)
    Cs = Cs / np.linalg.norm(Cs)
    s = np.sort(np.abs(np.linalg.eigvalsh(Cs)))[::-1]
    return np.concatenate([s, np.zeros(n - len(s))])


@pytest.mark.parametrize("method,warmup,given", [("qr", 0, True), ("qr", 0, False),
                                                 ("qr", 1, False), ("eigen", 1, False)])
def test_first_test_after_init_measures_change_from_initial_corner(q, method, warmup, given):
    """The initial corner's spectrum is taken at the first convergence test,
    beside the current corner's (same size: one set of launches; a corner that
    grew since the initialisation, as the standard method's steps do after a
    short warm-up: one after the other).  The change reported must be the one
    between the two corners' LAPACK spectra (eigenvalues to ~1e-13 each, so
    5e-12 on the norm of 40 differences)."""
    chi, seed = 40, 11
    rng = np.random.default_rng(seed)
    A = o.normalized_input(qi.raw_tensor(2, 2, seed))
    ctx = q.QRCTM(2, 2, chi, warmup_steps=warmup, method=method)
    if given:
        C = rng.standard_normal((chi, chi))
        T = rng.standard_normal((chi, 4, chi))
        ctx.init_env(cuda(A), cuda(C + C.T), cuda(T + T.transpose(2, 1, 0)))
    else:
        ctx.init_env(cuda(A))

    def corner(n):   # the library packs the current n x n corner at the buffer's start
        return ctx.get_env(spectrum=False)[0].cpu().numpy().reshape(-1)[: n * n].reshape(n, n)

    n0 = chi if warmup == 0 else 16                 # D^2 = 4, one warm-up step: 16
    n1 = chi if (warmup == 0 or method == "eigen") else 16   # QR steps keep chi
    Ci = corner(n0)
    d1 = ctx.step(1)
    C1 = corner(n1)
    ref = np.linalg.norm(_spec(C1, chi) - _spec(Ci, chi))
    assert abs(d1 - ref) < 5e-12, (d1, ref)
    # a second test measures the change from the first test's spectrum
    d2 = ctx.step(1)
    C2 = corner(n1)
    ref2 = np.linalg.norm(_spec(C2, chi) - _spec(C1, chi))
    assert abs(d2 - ref2) < 5e-12, (d2, ref2)
