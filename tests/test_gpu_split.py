"""GPU parity of the split-precision path (TF32x3 tensor-core contractions,
FP64 QR, normalisation and traces) against the FP64 CPU oracle.

Tolerances: one step from the same environment, elementwise 2e-5 relative to
the largest entry (TF32x3 products carry ~2^-21 relative error, FP32
partial sums ~2^-24 per addition, and the QR of the reduced corner can
amplify them by its conditioning); energy per site of converged
environments |dE| <= 1e-7 (the split-path target)."""
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


@pytest.mark.parametrize("D,chi,seed", [(2, 16, 3), (3, 27, 4), (4, 32, 5), (6, 36, 6), (6, 53, 7)])
def test_split_single_step(q, D, chi, seed):
    A = o.normalized_input(qi.raw_tensor(2, D, seed))
    C, T = o.warmup(A, chi)
    Cn, Tn = o.qr_step(C, T, A)
    ctx = q.QRCTM(2, D, chi, precision="split")
    ctx.init_env(cuda(A), cuda(C), cuda(T))
    ctx.step(1, want_delta=False)
    Cg, Tg, _ = ctx.get_env(spectrum=False)
    Cg, Tg = Cg.cpu().numpy(), Tg.cpu().numpy()
    assert np.abs(Cg - Cn).max() < 2e-5 * np.abs(Cn).max()
    assert np.abs(Tg - Tn).max() < 2e-5 * np.abs(Tn).max()


def test_split_single_step_wide_qr(q):
    # chi = 520 > 512: the triangular solve forming Q keeps 32 values per
    # lane.  C = I + small symmetric and a random T make the reduced corner a
    # random 4 chi x chi matrix (condition ~3), so Q is well determined and
    # one step compares entry by entry.
    D, chi = 2, 520
    rng = np.random.default_rng(11)
    A = o.normalized_input(qi.raw_tensor(2, D, 7))
    E = rng.standard_normal((chi, chi))
    C, T = o.sym_norm(np.eye(chi) + 0.05 * (E + E.T) / np.sqrt(chi),
                      rng.standard_normal((chi, D * D, chi)))
    Cn, Tn = o.qr_step(C, T, A)
    ctx = q.QRCTM(2, D, chi, precision="split")
    ctx.init_env(cuda(A), cuda(C), cuda(T))
    ctx.step(1, want_delta=False)
    Cg, Tg, _ = ctx.get_env(spectrum=False)
    Cg, Tg = Cg.cpu().numpy(), Tg.cpu().numpy()
    assert np.abs(Cg - Cn).max() < 2e-5 * np.abs(Cn).max()
    assert np.abs(Tg - Tn).max() < 2e-5 * np.abs(Tn).max()


@pytest.mark.parametrize("D,chi,seed,decay", [(2, 16, 0, False), (3, 27, 1, True)])
def test_split_converged_energy(q, D, chi, seed, decay):
    A = o.normalized_input(qi.raw_tensor(2, D, seed, decay))
    C, T = o.warmup(A, chi)
    Co, To, info = o.ctmrg(A, chi, "qr", tol=1e-12, max_iter=400, init=(C, T))
    Eo = o.energy(Co, To, A, 1.0, 0.5)
    ctx = q.QRCTM(2, D, chi, precision="split", with_nnn=True, check_every=5)
    ctx.init_env(cuda(A), cuda(C), cuda(T))
    it, dlt = ctx.run_to_convergence(tol=1e-9, max_iter=400)
    Eg = ctx.energy(1.0, 0.5)
    print("split", D, chi, "iters", it, "delta", dlt, "dE", Eg - Eo)
    assert abs(Eg - Eo) < 1e-7


@pytest.mark.parametrize("D,chi,seed,decay", [(3, 27, 1, True), (6, 144, 0, True)])
def test_split_j2_energy_matches_fp64_from_same_env(q, D, chi, seed, decay):
    """A split-precision context evaluates the one (chi D^2)^3 product of the
    2x2 patch (Ct_open Ct) on the TF32x3 tensor cores; every other
    contraction and the traces are FP64.  From the same environment its J1-J2
    energy must match the FP64 context's (itself the oracle's to 1e-12,
    test_gpu_parity) to 1e-7 per site, the split-path target; the J2 = 0
    energy, which has no such product, to 1e-13."""
    A = o.normalized_input(qi.raw_tensor(2, D, seed, decay))
    s = q.QRCTM(2, D, chi, precision="split", with_nnn=True, check_every=5)
    s.init_env(cuda(A))
    s.run_to_convergence(tol=1e-9, max_iter=300)
    C, T, _ = s.get_env(spectrum=False)
    f = q.QRCTM(2, D, chi, with_nnn=True)
    f.init_env(cuda(A), C, T)
    s.init_env(cuda(A), C, T)
    e_f, e_s = f.energy(1.0, 0.5), s.energy(1.0, 0.5)
    print(f"D{D} chi{chi}: E(J2=0.5) split - fp64 = {e_s - e_f:.3e}")
    assert abs(e_s - e_f) < 1e-7
    assert abs(s.energy(1.0, 0.0) - f.energy(1.0, 0.0)) < 1e-13
    s.close()
    f.close()
