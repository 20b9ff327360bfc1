"""GPU parity of the FP64 path against the CPU oracle, through the C ABI.

Tolerances (FP64 path): elementwise step outputs 1e-11 (the QR with
diag(R) >= 0 is unique for a full-rank reduced corner, so one step from the
same (C, T) is elementwise defined); gauge-invariant quantities of converged
environments (sorted |eig C|, energy) 1e-10 relative."""
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


def host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("d,D,seed", [(2, 2, 0), (2, 3, 1), (3, 4, 2)])
def test_c4v_symmetrize(q, d, D, seed):
    X = qi.raw_tensor(d, D, seed)
    Y = host(q.c4v_symmetrize(cuda(X), normalize=True))
    assert np.abs(Y - o.normalized_input(X)).max() < 1e-15


@pytest.mark.parametrize("m,n,seed", [(64, 16, 0), (100, 33, 1), (1024, 64, 2), (5184, 144, 3),
                                      (77, 77, 4), (300, 1, 5), (2000, 97, 6),
                                      (40000, 16, 7), (200000, 4, 8)])
def test_householder_qr(q, m, n, seed):
    M = np.random.default_rng(seed).standard_normal((m, n))
    Q, R = q.householder_qr(cuda(M))
    Q, R = host(Q), host(R)
    Qo, Ro = o.householder_qr(M)
    assert np.abs(Q - Qo).max() < 1e-11
    assert np.abs(R - Ro).max() < 1e-11 * np.abs(Ro).max()
    assert np.abs(Q.T @ Q - np.eye(n)).max() < 1e-13
    assert np.all(np.diag(R) >= 0) and np.abs(np.tril(R, -1)).max() == 0


def test_householder_qr_rank_deficient(q):
    rng = np.random.default_rng(9)
    M = rng.standard_normal((90, 4)) @ rng.standard_normal((4, 10))
    M[:, 2] = 0.0
    Q, R = q.householder_qr(cuda(M))
    Q, R = host(Q), host(R)
    assert np.abs(Q.T @ Q - np.eye(10)).max() < 1e-12
    assert np.abs(Q @ R - M).max() < 1e-12
    assert np.all(np.diag(R) >= 0)


@pytest.mark.parametrize("layers", ["double", "split"])
@pytest.mark.parametrize("D,chi", [(2, 16), (3, 27)])
def test_single_qr_step_elementwise(q, layers, D, chi):
    A = o.normalized_input(qi.raw_tensor(2, D, 3))
    C, T = o.warmup(A, chi)
    Cn, Tn = o.qr_step(C, T, A)
    ctx = q.QRCTM(2, D, chi, layers=layers)
    ctx.init_env(cuda(A), cuda(C), cuda(T))
    ctx.step(1, want_delta=False)
    Cg, Tg, _ = ctx.get_env(spectrum=False)
    assert np.abs(host(Cg) - Cn).max() < 1e-11
    assert np.abs(host(Tg) - Tn).max() < 1e-11


def test_bulk_initial_boundary(q):
    A = o.normalized_input(qi.raw_tensor(2, 3, 4))
    C0, T0 = o.init_env(A)
    ctx = q.QRCTM(2, 3, 9, warmup_steps=-1)
    ctx.init_env(cuda(A))
    Cg, Tg, _ = ctx.get_env(spectrum=False)
    assert np.abs(host(Cg) - C0).max() < 1e-14
    assert np.abs(host(Tg) - T0).max() < 1e-14


def test_converged_env_and_energy_d2_D2_chi16(q):
    # workload: d2 D2 chi16, 200 iterations or spectrum change < 1e-12
    w = qi.WORKLOADS["d2_D2_chi16"]
    A = o.normalized_input(qi.raw_tensor(2, 2, w["seed"]))
    C, T = o.warmup(A, 16)
    Co, To, info = o.ctmrg(A, 16, "qr", tol=1e-12, max_iter=200, init=(C, T))
    assert info["converged"]
    Eo = o.energy(Co, To, A, 1.0, 0.5)
    ctx = q.QRCTM(2, 2, 16, with_nnn=True)
    ctx.init_env(cuda(A), cuda(C), cuda(T))
    it, dlt = ctx.run_to_convergence(tol=1e-12, max_iter=200)
    assert dlt < 1e-12
    _, _, sg = ctx.get_env()
    assert np.abs(sg - o.corner_spectrum(Co)).max() < 1e-10
    assert abs(ctx.energy(1.0, 0.5) - Eo) < 1e-10 * abs(Eo)


def test_energy_from_identical_env(q):
    A = o.normalized_input(qi.raw_tensor(2, 3, 5))
    C, T = o.warmup(A, 18)
    for _ in range(5):
        C, T = o.qr_step(C, T, A)
    ctx = q.QRCTM(2, 3, 18, with_nnn=True)
    ctx.init_env(cuda(A), cuda(C), cuda(T))
    for J2 in (0.0, 0.5):
        Eo = o.energy(C, T, A, 1.0, J2)
        assert abs(ctx.energy(1.0, J2) - Eo) < 1e-12 * max(1.0, abs(Eo))


def test_gpu_warmup_reaches_same_fixed_point(q):
    A = o.normalized_input(qi.raw_tensor(2, 2, 0))
    Co, To, _ = o.ctmrg(A, 16, "qr", tol=1e-13, max_iter=400)
    Eo = o.energy(Co, To, A, 1.0, 0.0)
    ctx = q.QRCTM(2, 2, 16)
    ctx.init_env(cuda(A))
    ctx.run_to_convergence(tol=1e-13, max_iter=400)
    assert abs(ctx.energy(1.0, 0.0) - Eo) < 1e-10 * abs(Eo)
    _, _, sg = ctx.get_env()
    assert np.abs(sg - o.corner_spectrum(Co)).max() < 1e-9


@pytest.mark.parametrize("env_from", ["oracle", "gpu"])
def test_product_state_energy(q, env_from):
    v = np.array([0.6, -0.8])
    A = np.zeros((2, 2, 2, 2, 2))
    A[:, 0, 0, 0, 0] = v
    ctx = q.QRCTM(2, 2, 8, with_nnn=True)
    if env_from == "oracle":
        C, T = o.warmup(A, 8)
        ctx.init_env(cuda(A), cuda(C), cuda(T))
    else:
        ctx.init_env(cuda(A))
    ctx.step(10, want_delta=False)
    assert abs(ctx.energy(1.0, 0.5) - (-0.25)) < 1e-12


def test_not_symmetric_rejected(q):
    X = qi.raw_tensor(2, 2, 1)
    ctx = q.QRCTM(2, 2, 8)
    with pytest.raises(q.QRCTMError) as ei:
        ctx.init_env(cuda(X / np.linalg.norm(X)))
    assert ei.value.status == "NOT_SYMMETRIC"


def test_host_buffer_entry_points(q):
    """qrctm_init_env_host / qrctm_get_env_host copy inside the library call;
    one step from host inputs equals the oracle's step (1e-11) and the
    device-pointer path to 1e-14 (not bit for bit: the QR panel adds its
    cross-CTA partial sums with atomics in no fixed order)."""
    import torch
    A = o.normalized_input(qi.raw_tensor(2, 3, 3))
    C, T = o.warmup(A, 27)
    Cn, Tn = o.qr_step(C, T, A)
    h = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64).pin_memory()
    ctx = q.QRCTM(2, 3, 27)
    ctx.init_env_host(h(A), h(C), h(T))
    ctx.step(1, want_delta=True)
    oC = torch.empty((27, 27), dtype=torch.float64).pin_memory()
    oT = torch.empty((27, 9, 27), dtype=torch.float64).pin_memory()
    s = ctx.get_env_host(oC, oT, spectrum=True)
    assert np.abs(oC.numpy() - Cn).max() < 1e-11
    assert np.abs(oT.numpy() - Tn).max() < 1e-11
    assert np.abs(s - o.corner_spectrum(Cn)).max() < 1e-12
    ref = q.QRCTM(2, 3, 27)
    ref.init_env(cuda(A), cuda(C), cuda(T))
    ref.step(1, want_delta=True)
    Cg, Tg, _ = ref.get_env(spectrum=False)
    assert np.abs(oC.numpy() - host(Cg)).max() < 1e-14
    assert np.abs(oT.numpy() - host(Tg)).max() < 1e-14
    # the bulk boundary from a host tensor alone (no C0, T0)
    ctx.init_env_host(h(A))
    ctx.step(2, want_delta=False)
    ctx.close()
    ref.close()


def test_energy_without_sublattice_rotation(q):
    """qrctm_model.sublattice_rotation = 0 takes the plain bond on NN pairs:
    the oracle's energy with rotate=False from the same environment (1e-12),
    and the product-state closed form E = J1/2 + J2/2."""
    A = o.normalized_input(qi.raw_tensor(2, 3, 5))
    C, T = o.warmup(A, 18)
    ctx = q.QRCTM(2, 3, 18, with_nnn=True)
    ctx.init_env(cuda(A), cuda(C), cuda(T))
    for J2 in (0.0, 0.5):
        Eo = o.energy(C, T, A, 1.0, J2, rotate=False)
        assert abs(ctx.energy(1.0, J2, rotation=False) - Eo) < 1e-12 * max(1.0, abs(Eo))
    v = np.array([0.6, -0.8])
    P = np.zeros((2, 2, 2, 2, 2))
    P[:, 0, 0, 0, 0] = v
    pc = q.QRCTM(2, 2, 8, with_nnn=True)
    pc.init_env(cuda(P))
    pc.step(4, want_delta=False)
    assert abs(pc.energy(1.0, 0.5, rotation=False) - 0.75) < 1e-12
