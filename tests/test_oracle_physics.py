"""Physics pins for the oracle: product states, the rotated Heisenberg bond,
the classical Ising model against Onsager/Yang, brute-force patch
contractions, and derivatives (CPU only)."""
import json
import os

import numpy as np
import pytest

from oracle import qrctm_oracle as o
import qrctm_inputs as qi

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def test_rotated_bond_closed_form():
    # exp(i pi sigma^y / 2) on one site flips sigma^x and sigma^z
    X = np.array([[0, 1], [1, 0]])
    Y = np.array([[0, -1j], [1j, 0]])
    Z = np.diag([1, -1])
    ref = (-np.kron(X, X) + np.kron(Y, Y) - np.kron(Z, Z)).real / 4
    assert np.abs(o.rotated_heisenberg_bond() - ref).max() < 1e-15
    # singlet energy -3/4 for the plain bond
    assert abs(np.linalg.eigvalsh(o.heisenberg_bond()).min() + 0.75) < 1e-15


@pytest.mark.parametrize("method", ["qr", "eigen"])
@pytest.mark.parametrize("seed", [0, 1])
def test_product_state_D1_energy_exact(method, seed):
    v = np.random.default_rng(seed).standard_normal(2)
    A = (v / np.linalg.norm(v)).reshape(2, 1, 1, 1, 1)
    C, T, _ = o.ctmrg(A, 4, method, tol=1e-14, max_iter=5)
    g = GOLD["product_state_energy"]
    for J2 in (0.0, 0.5):
        E = o.energy(C, T, A, 1.0, J2)
        assert abs(E - (g["value_J1"] + J2 * g["value_J2"])) < 1e-14


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_product_state_energy_without_rotation(seed):
    # plain NN bond: <h> = (<X>^2 + <Z>^2)/4 = 1/4 for a real unit v
    v = np.random.default_rng(seed).standard_normal(2)
    A = (v / np.linalg.norm(v)).reshape(2, 1, 1, 1, 1)
    C, T, _ = o.ctmrg(A, 4, "qr", tol=1e-14, max_iter=5)
    g = GOLD["product_state_energy_unrotated"]
    for J2 in (0.0, 0.5):
        E = o.energy(C, T, A, 1.0, J2, rotate=False)
        assert abs(E - (g["value_J1"] + J2 * g["value_J2"])) < 1e-14
    # a random D = 2 state: the two NN bonds differ by the rotation alone,
    # <h~> - <h> = -(<XX> + <ZZ>)/2 on the same two-site density matrix
    A2 = o.normalized_input(qi.raw_tensor(2, 2, seed))
    C2, T2 = o.warmup(A2, 8)
    rho = o.rdm_nn(C2, T2, A2)
    d = 2
    R = np.transpose(rho, (0, 2, 1, 3)).reshape(d * d, d * d)
    R = R / np.trace(R)
    X = np.array([[0.0, 1.0], [1.0, 0.0]])
    Z = np.diag([1.0, -1.0])
    diff = -(np.trace(R @ np.kron(X, X)) + np.trace(R @ np.kron(Z, Z))) / 2
    E_r = o.energy(C2, T2, A2, 1.0, 0.0)
    E_p = o.energy(C2, T2, A2, 1.0, 0.0, rotate=False)
    assert abs((E_r - E_p) / 2 - diff) < 1e-13


@pytest.mark.parametrize("method", ["qr", "eigen"])
def test_product_state_embedded_D2(method):
    # rank-deficient reduced corner (R_jj = 0), exact energies survive
    v = np.array([0.6, -0.8])
    A = np.zeros((2, 2, 2, 2, 2))
    A[:, 0, 0, 0, 0] = v
    C, T, _ = o.ctmrg(A, 8, method, tol=1e-14, max_iter=10)
    assert abs(o.energy(C, T, A, 1.0, 0.5) - (-0.5 + 0.25)) < 1e-13
    rho = o.rdm_nn(C, T, A)
    pv = np.einsum("a,b,c,d->abcd", v, v, v, v)
    assert np.abs(rho / np.trace(np.trace(rho, axis1=0, axis2=1)) - pv).max() < 1e-13


def test_onsager_quadrature_at_critical_point():
    g = GOLD["ising_critical_free_energy"]["value"]
    bc = GOLD["ising_beta_c"]["value"]
    assert abs(o.onsager_free_energy(bc, n=4096) - g) < 1e-6


def onsager_nn_correlation(beta, n=512):
    """<s s>_NN = (1/2) d(-beta f)/d beta, differentiated under the integral."""
    t = 2 * np.pi * np.arange(n) / n
    c = np.cos(t)[:, None] + np.cos(t)[None, :]
    ch, sh = np.cosh(2 * beta), np.sinh(2 * beta)
    arg = ch ** 2 - sh * c
    darg = 4 * ch * sh - 2 * ch * c
    return 0.5 * 0.5 * np.mean(darg / arg)


@pytest.mark.parametrize("method", ["qr", "eigen"])
@pytest.mark.parametrize("beta", [0.3, 0.6])
def test_ising_against_onsager_and_yang(method, beta):
    # Discussion: QR-CTMRG applies to classical partition functions
    A = o.ising_A(beta)
    a = o.double_layer(A)
    env = o.init_env(A, fixed_phys=0) if beta > GOLD["ising_beta_c"]["value"] else None
    C, T, _ = o.ctmrg(A, 16, method, tol=1e-12, max_iter=300, env=env)
    assert abs(np.log(o.ising_kappa(C, T, a)) - o.onsager_free_energy(beta)) < 1e-11
    M = o.ising_kappa(C, T, a, o.ising_observable_layer(A))
    assert abs(abs(M) - o.yang_magnetization(beta)) < 1e-9
    # nearest-neighbour correlation from the 2x1 reduced density matrix
    rho = o.rdm_nn(C, T, A)
    p = np.einsum("aabb->ab", rho)
    p = p / p.sum()
    s = np.array([1.0, -1.0])
    assert abs(s @ p @ s - onsager_nn_correlation(beta)) < 1e-9


def network_ln_kappa(a, chi, method="qr", v=None, a_obs=None):
    env = o.init_env_network(a, v)
    C, T, info = o.ctmrg(a, chi, method, tol=1e-12, max_iter=400, env=env, layers="network")
    assert info["converged"]
    lk = float(np.log(o.network_kappa(C, T, a)))
    return (lk, float(o.network_kappa(C, T, a, a_obs))) if a_obs is not None else lk


@pytest.mark.parametrize("method", ["qr", "eigen"])
@pytest.mark.parametrize("beta", [0.3, 0.6])
def test_ising_network_against_onsager_and_yang(method, beta):
    # Discussion: classical partition functions; the network tensor (bond 2)
    # is fed directly instead of a double layer.  Ordered phase: boundary
    # spins fixed to +1 through the vector W[0].
    a, a_s, W = o.ising_network(beta)
    v = W[0] if beta > GOLD["ising_beta_c"]["value"] else None
    lk, M = network_ln_kappa(a, 16, method, v, a_s)
    assert abs(lk - o.onsager_free_energy(beta)) < 1e-11
    assert abs(M - o.yang_magnetization(beta)) < 1e-9


@pytest.mark.parametrize("beta", [0.4, 1.2])
def test_potts2_network_reduces_to_ising(beta):
    # delta(s,s') = (1 + s s')/2: every bond carries e^(beta/2) times the
    # Ising weight at coupling beta/2, two bonds per site
    a, W = o.potts_network(2, beta)
    v = W[0] if beta / 2 > GOLD["ising_beta_c"]["value"] else None
    lk = network_ln_kappa(a, 16, "qr", v)
    assert abs(lk - (beta + o.onsager_free_energy(beta / 2))) < 1e-11


def test_potts3_network_duality():
    # Square-lattice Potts self-duality (Fortuin-Kasteleyn form
    # Z(q, v) = q^(1-N*) v^E Z*(q, q/v), v = e^K - 1, E = 2N bonds, N* ~ N):
    # ln kappa(K) - ln kappa(K*) = 2 ln(e^K - 1) - ln q.  K = 0.6 is
    # disordered, its dual K* = 1.54 ordered (boundary fixed to state 0).
    q, K = 3, 0.6
    vK = np.exp(K) - 1
    Kd = np.log1p(q / vK)
    a1, _ = o.potts_network(q, K)
    a2, W2 = o.potts_network(q, Kd)
    lk1 = network_ln_kappa(a1, 27, "qr")
    lk2 = network_ln_kappa(a2, 27, "qr", W2[0])
    assert abs((lk1 - lk2) - (2 * np.log(vK) - np.log(q))) < 1e-9


def test_network_infinite_temperature():
    # beta = 0: every configuration weighs 1, kappa = q exactly
    a, _ = o.potts_network(3, 0.0)
    assert abs(network_ln_kappa(a, 9, "qr") - np.log(3.0)) < 1e-13


def test_rdm_nnn_by_brute_force_patch():
    # the 2x2 patch written out tensor by tensor (4 C, 8 T, 4 sites), no
    # quadrant symmetry used
    rng = np.random.default_rng(3)
    A = o.normalized_input(qi.raw_tensor(2, 2, 4))
    C, T = o.sym_norm(rng.standard_normal((3, 3)), rng.standard_normal((3, 4, 3)))
    a = o.double_layer(A)
    aO = o.double_layer_open(A)
    ops = [
        C, [0, 1], T, [1, 2, 3], T, [3, 4, 5], C, [5, 6],          # top row
        T, [0, 7, 8], aO, [40, 41, 2, 7, 9, 10], a, [4, 10, 11, 12], T, [6, 12, 13],
        T, [8, 14, 15], a, [9, 14, 16, 17], aO, [42, 43, 11, 17, 18, 19], T, [13, 19, 20],
        C, [15, 21], T, [21, 16, 22], T, [22, 18, 23], C, [23, 20],  # bottom row
    ]
    ref = np.einsum(*ops, [40, 41, 42, 43], optimize="greedy")
    got = o.rdm_nnn(C, T, A)
    assert np.abs(ref - got).max() < 1e-14 * np.abs(ref).max()


def test_rdm_nn_by_brute_force_patch():
    rng = np.random.default_rng(5)
    A = o.normalized_input(qi.raw_tensor(2, 2, 6))
    C, T = o.sym_norm(rng.standard_normal((3, 3)), rng.standard_normal((3, 4, 3)))
    aO = o.double_layer_open(A)
    ops = [
        C, [0, 1], T, [1, 2, 3], T, [3, 4, 5], C, [5, 6],
        T, [0, 7, 8], aO, [40, 41, 2, 7, 9, 10], aO, [42, 43, 4, 10, 11, 12], T, [6, 12, 13],
        C, [8, 14], T, [14, 9, 15], T, [15, 11, 16], C, [16, 13],
    ]
    ref = np.einsum(*ops, [40, 41, 42, 43], optimize="greedy")
    got = o.rdm_nn(C, T, A)
    assert np.abs(ref - got).max() < 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("model,q,beta", [("ising", 2, 0.43), ("potts", 3, 0.95), ("potts", 4, 0.3)])
def test_network_input_is_the_oracle_model(model, q, beta):
    # the bench's input builder and the oracle's model agree exactly
    a, a_obs, v = qi.network_input(model, q, beta)
    if model == "ising":
        a2, a2_obs, W = o.ising_network(beta)
        assert np.abs(a_obs - a2_obs).max() < 1e-15
    else:
        a2, W = o.potts_network(q, beta)
    assert np.abs(a - a2).max() < 1e-15
    assert np.abs(v - W[0]).max() < 1e-15
