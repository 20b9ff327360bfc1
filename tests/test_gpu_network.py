"""Classical networks fed directly on the GPU (Discussion: classical partition
functions): the CUDA path against the oracle and against Onsager / Yang /
Potts duality, FP64.  The fixed point of a classical network with a
non-degenerate dominant corner spectrum does not depend on the start, so the
GPU warm-up (subspace iteration) and the oracle's (full eigh) reach the same
ln kappa and <O>."""
import numpy as np
import pytest

from oracle import qrctm_oracle as o

pytestmark = pytest.mark.gpu

BETA_C = 0.5 * np.log1p(np.sqrt(2.0))


def _dev(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def gpu_network(a, chi, method="qr", v=None, a_obs=None, tol=1e-12, max_iter=2000):
    import paper_2505_00494_b300 as q
    b = a.shape[0]
    ctx = q.QRCTM(1, b, chi, layers="network", method=method, check_every=5)
    ctx.init_env_network(_dev(a), None if v is None else _dev(v))
    it, dlt = ctx.run_to_convergence(tol, max_iter)
    assert dlt < tol, (it, dlt)
    lk, M = ctx.network_observables(None if a_obs is None else _dev(a_obs))
    _, _, s = ctx.get_env()
    ctx.close()
    return lk, M, s


def oracle_network(a, chi, method="qr", v=None, a_obs=None):
    env = o.init_env_network(a, v)
    C, T, info = o.ctmrg(a, chi, method, tol=1e-12, max_iter=2000, env=env, layers="network")
    assert info["converged"]
    lk = float(np.log(o.network_kappa(C, T, a)))
    M = float(o.network_kappa(C, T, a, a_obs)) if a_obs is not None else None
    return lk, M, o.corner_spectrum(C)


@pytest.mark.parametrize("method", ["qr", "eigen"])
@pytest.mark.parametrize("beta,chi", [(0.3, 16), (0.6, 16), (0.6, 37)])
def test_ising_network_parity_and_onsager(method, beta, chi):
    a, a_s, W = o.ising_network(beta)
    v = W[0] if beta > BETA_C else None
    lk, M, s = gpu_network(a, chi, method, v, a_s)
    lk_o, M_o, s_o = oracle_network(a, chi, method, v, a_s)
    assert abs(lk - lk_o) < 1e-10
    assert abs(M - M_o) < 1e-9
    assert abs(lk - o.onsager_free_energy(beta)) < 1e-10
    assert abs(M - o.yang_magnetization(beta)) < 1e-9
    # the dominant corner spectrum (gauge invariant); the tail at the
    # truncation edge may depend on the start
    n = 4
    assert np.abs(s[:n] - s_o[:n]).max() < 1e-10


@pytest.mark.parametrize("method", ["qr", "eigen"])
def test_potts3_network_parity_and_duality(method):
    # bond 3: the network layout of the absorption, projection and enlarged
    # corner (no ket/bra halves), chi = 27 = 3^3 and a ragged 40
    q, K = 3, 0.6
    vK = np.exp(K) - 1
    Kd = np.log1p(q / vK)
    a1, _ = o.potts_network(q, K)
    a2, W2 = o.potts_network(q, Kd)
    res = []
    for a, v, chi in ((a1, None, 27), (a2, W2[0], 40)):
        lk, _, _ = gpu_network(a, chi, method, v)
        lk_o, _, _ = oracle_network(a, chi, method, v)
        assert abs(lk - lk_o) < 1e-10
        res.append(lk)
    assert abs((res[0] - res[1]) - (2 * np.log(vK) - np.log(q))) < 1e-9


def test_network_infinite_temperature_rank_one():
    # beta = 0: a is rank one, every reduced corner has rank one
    a, _ = o.potts_network(3, 0.0)
    lk, _, _ = gpu_network(a, 9)
    assert abs(lk - np.log(3.0)) < 1e-13


def test_network_errors():
    import paper_2505_00494_b300 as q
    a, _, _ = o.ising_network(0.3)
    ctx = q.QRCTM(1, 2, 8, layers="network")
    bad = a.copy()
    bad[0, 1, 0, 0] += 1e-3
    with pytest.raises(q.QRCTMError) as ei:
        ctx.init_env_network(_dev(bad))
    assert ei.value.code == 5   # NOT_SYMMETRIC
    with pytest.raises(q.QRCTMError):
        ctx.init_env(_dev(np.zeros((1, 2, 2, 2, 2))))
    with pytest.raises(q.QRCTMError) as ei:
        ctx.network_observables()
    assert ei.value.code == 8   # STATE: no environment yet
    ctx.close()
    # an iPEPS context refuses the network calls
    ctx2 = q.QRCTM(2, 2, 8)
    with pytest.raises(q.QRCTMError):
        ctx2.init_env_network(_dev(a))
    ctx2.close()


def test_network_restart_from_environment():
    # a converged environment handed back in is a fixed point: one more step
    # keeps ln kappa, and a neighbouring coupling starts from it
    import paper_2505_00494_b300 as q
    a, a_s, W = o.ising_network(0.3)
    ctx = q.QRCTM(1, 2, 16, layers="network", check_every=5)
    ctx.init_env_network(_dev(a))
    ctx.run_to_convergence(1e-12, 2000)
    lk0, _ = ctx.network_observables()
    C, T, _ = ctx.get_env(spectrum=False)
    ctx.init_env_network(_dev(a), None, C, T)
    ctx.step(5)
    lk1, _ = ctx.network_observables()
    assert abs(lk1 - lk0) < 1e-12
    a2, _, _ = o.ising_network(0.32)
    ctx.init_env_network(_dev(a2), None, C, T)
    ctx.run_to_convergence(1e-12, 2000)
    lk2, _ = ctx.network_observables()
    assert abs(lk2 - o.onsager_free_energy(0.32)) < 1e-10
    with pytest.raises(q.QRCTMError):
        ctx.init_env_network(_dev(a), None, C, None)
    ctx.close()
