"""Failure detection through the C ABI.  Every fault here is made on the host:
a NaN written into an input, an iteration cap that is too small, or a wait
bound that is too short for a barrier that asks for one arrival more than
the CTAs launched.  No test faults, traps or hangs the GPU: the device waits
are bounded and report through the context's error word, and after each
failure the same context (or workspace) must run the next call normally.

Expected statuses: NaN/Inf in C0 or T0 -> QRCTM_ERR_NUMERIC (found by the
FP64 norm of the symmetrise-and-normalise kernel); NaN in A ->
QRCTM_ERR_NUMERIC (host check of the tensor's norm); max_iter reached ->
QRCTM_ERR_NOT_CONVERGED with the context still stepping; a grid wait that
runs out -> QRCTM_ERR_TIMEOUT, with the workspace's arrival counter and
error word left zero so the next QR is exact (1e-11 against the oracle)."""
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


@pytest.fixture(scope="module")
def env():
    A = o.normalized_input(qi.raw_tensor(2, 2, 0))
    C, T = o.warmup(A, 16)
    return A, C, T


@pytest.mark.parametrize("where", ["C0", "T0"])
def test_nan_in_environment_is_numeric(q, env, where):
    A, C, T = env
    Cb, Tb = C.copy(), T.copy()
    if where == "C0":
        Cb[3, 5] = Cb[5, 3] = np.nan
    else:
        Tb[2, 1, 7] = np.inf
    ctx = q.QRCTM(2, 2, 16)
    with pytest.raises(q.QRCTMError) as ei:
        ctx.init_env(cuda(A), cuda(Cb), cuda(Tb))
    assert ei.value.status == "NUMERIC"
    with pytest.raises(q.QRCTMError) as ei:   # no environment was accepted
        ctx.step(1)
    assert ei.value.status == "STATE"
    # the context is usable: a clean environment steps exactly like the oracle
    ctx.init_env(cuda(A), cuda(C), cuda(T))
    ctx.step(1, want_delta=True)
    Cn, Tn = o.qr_step(C, T, A)
    Cg, Tg, _ = ctx.get_env(spectrum=False)
    assert np.abs(Cg.cpu().numpy() - Cn).max() < 1e-11
    assert np.abs(Tg.cpu().numpy() - Tn).max() < 1e-11
    ctx.close()


def test_nan_in_tensor_is_numeric(q, env):
    A, C, T = env
    Ab = A.copy()
    Ab[1, 0, 1, 1, 0] = np.nan
    ctx = q.QRCTM(2, 2, 16)
    with pytest.raises(q.QRCTMError) as ei:
        ctx.init_env(cuda(Ab), cuda(C), cuda(T))
    assert ei.value.status == "NUMERIC"
    ctx.init_env(cuda(A), cuda(C), cuda(T))
    ctx.step(2, want_delta=True)
    ctx.close()


def test_max_iter_reached_is_not_converged(q, env):
    A, C, T = env
    ctx = q.QRCTM(2, 2, 16, check_every=1)
    ctx.init_env(cuda(A), cuda(C), cuda(T))
    with pytest.raises(q.QRCTMError) as ei:
        ctx.run_to_convergence(tol=1e-14, max_iter=1, raise_on_max=True)
    assert ei.value.status == "NOT_CONVERGED"
    assert ctx.iterations == 1
    # the context keeps stepping from where it stopped and converges
    it, dlt = ctx.run_to_convergence(tol=1e-12, max_iter=400, raise_on_max=True)
    assert dlt < 1e-12 and ctx.iterations == 1 + it
    Co, To, _ = o.ctmrg(A, 16, "qr", tol=1e-12, max_iter=400, init=(C, T))
    _, _, sg = ctx.get_env()
    assert np.abs(sg - o.corner_spectrum(Co)).max() < 1e-10
    ctx.close()


@pytest.mark.parametrize("m,n", [(5184, 144), (300, 40)])
def test_grid_wait_timeout_then_recovery(q, m, n):
    """The panel kernel's per-column barrier asks for one arrival more than
    the CTAs launched, so every wait runs out after 4096 polls (about a
    millisecond); the call returns TIMEOUT.  The same workspace then gives
    the exact QR, twice (the control words were left zero)."""
    import torch
    M = np.random.default_rng(5).standard_normal((m, n))
    nb = q.lib.qrctm_qr_workspace_bytes(m, n)
    ws = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    with pytest.raises(q.QRCTMError) as ei:
        q.householder_qr(cuda(M), workspace=ws, wait_spins=4096, extra_arrivals=1)
    assert ei.value.status == "TIMEOUT"
    Qo, Ro = o.householder_qr(M)
    for _ in range(2):
        Q, R = q.householder_qr(cuda(M), workspace=ws)
        assert np.abs(Q.cpu().numpy() - Qo).max() < 1e-11
        assert np.abs(R.cpu().numpy() - Ro).max() < 1e-11 * np.abs(Ro).max()
    # an explicit but sufficient bound behaves like the default
    Q, R = q.householder_qr(cuda(M), workspace=ws, wait_spins=1 << 24)
    assert np.abs(Q.cpu().numpy() - Qo).max() < 1e-11


def test_bounded_qr_rejects_bad_knobs(q):
    import torch
    M = torch.zeros((8, 4), dtype=torch.float64, device="cuda")
    for spins, extra in ((-1, 0), (0, -1)):
        with pytest.raises(q.QRCTMError) as ei:
            q.householder_qr(M, wait_spins=spins, extra_arrivals=extra)
        assert ei.value.status == "INVALID_ARG"
