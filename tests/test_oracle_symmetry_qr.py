"""Pins for the oracle's C4v projector and Householder QR (CPU only)."""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import qrctm_oracle as o
import qrctm_inputs as qi

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def projector_matrix(d, D):
    n = d * D ** 4
    P = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        P[:, i] = o.c4v_sym(e.reshape(d, D, D, D, D)).ravel()
    return P


@pytest.mark.parametrize("D", [1, 2, 3])
def test_sym_is_projector_with_rank_n(D):
    # footnote of the iPEPS paragraph: n(D) = d/8 (D^4 + 2D^3 + 3D^2 + 2D)
    P = projector_matrix(2, D)
    assert np.allclose(P @ P, P, atol=1e-14)
    assert np.allclose(P, P.T, atol=1e-14)      # orthogonal projector
    assert np.linalg.matrix_rank(P) == o.n_params(2, D)


@pytest.mark.parametrize("D", [2, 4, 6, 8])
def test_orbit_count_matches_n(D):
    # The invariant subspace has one basis vector per C4v orbit of (u,l,d,r);
    # count orbits by brute force, independently of the projector.
    seen, orbits = set(), 0
    for t in itertools.product(range(D), repeat=4):
        if t in seen:
            continue
        orbits += 1
        for p in o.C4V_PERMS:
            seen.add(tuple(t[q] for q in p))
    assert 2 * orbits == o.n_params(2, D)
    if D == 8:
        assert 2 * orbits == GOLD["n_params_d2_D8"]["value"]


def test_sym_output_is_invariant():
    A = o.normalized_input(qi.raw_tensor(2, 3, 5))
    for p in o.C4V_PERMS:
        assert np.allclose(np.transpose(A, (0,) + tuple(1 + q for q in p)), A, atol=1e-15)
    assert abs(o.fro_norm(A) - 1.0) < 1e-14


@pytest.mark.parametrize("m,n,seed", [(40, 7, 1), (64, 16, 2), (144, 36, 3), (9, 9, 4)])
def test_householder_matches_lapack(m, n, seed):
    M = np.random.default_rng(seed).standard_normal((m, n))
    Q, R = o.householder_qr(M)
    assert np.abs(Q.T @ Q - np.eye(n)).max() < 1e-14
    assert np.abs(np.tril(R, -1)).max() == 0.0
    assert np.all(np.diag(R) >= 0)
    assert np.abs(Q @ R - M).max() < 1e-13 * np.abs(M).max() * np.sqrt(m)
    Ql, Rl = np.linalg.qr(M)
    sg = np.sign(np.diag(Rl))
    assert np.abs(Ql * sg - Q).max() < 1e-12
    assert np.abs(Rl * sg[:, None] - R).max() < 1e-12


def test_householder_rank_deficient():
    rng = np.random.default_rng(7)
    M = rng.standard_normal((30, 3)) @ rng.standard_normal((3, 6))
    M[:, 1] = 0.0                                   # an exactly zero column
    Q, R = o.householder_qr(M)
    assert np.abs(Q.T @ Q - np.eye(6)).max() < 1e-13
    assert np.abs(Q @ R - M).max() < 1e-12
    assert R[1, 1] == 0.0


def test_householder_complex_step_matches_fd():
    # analytic continuation: Im qr(M + i h E) / h equals the derivative
    rng = np.random.default_rng(11)
    M = rng.standard_normal((20, 5))
    E = rng.standard_normal((20, 5))
    Qc, Rc = o.householder_qr(M + 1j * 1e-20 * E)
    dQ, dR = np.imag(Qc) / 1e-20, np.imag(Rc) / 1e-20
    eps = 1e-6
    Qp, Rp = o.householder_qr(M + eps * E)
    Qm, Rm = o.householder_qr(M - eps * E)
    assert np.abs(dQ - (Qp - Qm) / (2 * eps)).max() < 1e-7
    assert np.abs(dR - (Rp - Rm) / (2 * eps)).max() < 1e-7
