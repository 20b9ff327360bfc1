"""Pins for the oracle's CTMRG steps (Standard CTMRG and QR-CTMRG paragraphs,
Fig. 1(d)-(f)), CPU only."""
import numpy as np
import pytest

from oracle import qrctm_oracle as o
import qrctm_inputs as qi


def random_env(chi, D, seed):
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((chi, chi))
    T = rng.standard_normal((chi, D * D, chi))
    return o.sym_norm(C, T)


@pytest.mark.parametrize("chi,D,seed", [(5, 2, 0), (8, 3, 1), (12, 2, 2)])
def test_accelerated_corner_equals_projected_enlarged_corner(chi, D, seed):
    # Fig. 1(f): C' from (T', R, Q) equals Q^T Ct Q because ct = Q R.
    A = o.normalized_input(qi.raw_tensor(2, D, seed))
    C, T = random_env(chi, D, seed + 10)
    p = o.qr_step_parts(C, T, A)
    Ct = o.enlarged_corner(C, T, o.double_layer(A))
    ref = p["Q"].T @ Ct @ p["Q"]
    assert np.abs(ref - p["C_raw"]).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("chi,D,seed", [(5, 2, 0), (7, 3, 1)])
def test_split_layers_equal_double_layer(chi, D, seed):
    A = o.normalized_input(qi.raw_tensor(2, D, seed))
    C, T = random_env(chi, D, seed + 20)
    pd = o.qr_step_parts(C, T, A, "double")
    ps = o.qr_step_parts(C, T, A, "split")
    assert np.abs(pd["T_raw"] - ps["T_raw"]).max() < 1e-14
    assert np.abs(pd["C_raw"] - ps["C_raw"]).max() < 1e-14


def test_reduced_corner_rank_and_symmetry_of_outputs():
    A = o.normalized_input(qi.raw_tensor(2, 2, 3))
    C, T = random_env(6, 2, 4)
    ct = o.reduced_corner(C, T)
    assert ct.shape == (6 * 4, 6)
    p = o.qr_step_parts(C, T, A)
    # C' and T' come out reflection-symmetric before sym_norm
    assert np.abs(p["C_raw"] - p["C_raw"].T).max() < 1e-14
    assert np.abs(p["T_raw"] - p["T_raw"].transpose(2, 1, 0)).max() < 1e-14
    # Q is the QR isometry of ct
    assert np.abs(p["Q"] @ p["R"] - ct).max() < 1e-14


def test_enlarged_corner_definition_by_loops():
    # brute-force loops for Ct on a tiny case
    A = o.normalized_input(qi.raw_tensor(2, 2, 1))
    a = o.double_layer(A)
    C, T = random_env(2, 2, 5)
    Ct = o.enlarged_corner(C, T, a)
    chi, D2 = 2, 4
    ref = np.zeros((chi, D2, chi, D2))
    for b in range(chi):
        for l in range(D2):
            for r in range(chi):
                for j in range(D2):
                    s = 0.0
                    for g in range(chi):
                        for h in range(chi):
                            for i in range(D2):
                                for k in range(D2):
                                    s += C[g, h] * T[h, i, r] * T[g, k, b] * a[i, k, l, j]
                    ref[b, l, r, j] = s
    assert np.abs(ref.reshape(chi * D2, chi * D2) - Ct).max() < 1e-15


def test_double_layer_and_init_definitions():
    A = o.normalized_input(qi.raw_tensor(2, 2, 2))
    a = o.double_layer(A)
    # a[(u u'),(l l'),(d d'),(r r')] by loops
    ref = np.zeros((2,) * 8)
    for u, U, l, L, d, Dd, r, R in np.ndindex(*(2,) * 8):
        ref[u, U, l, L, d, Dd, r, R] = sum(A[s, u, l, d, r] * A[s, U, L, Dd, R] for s in range(2))
    assert np.abs(ref.reshape(4, 4, 4, 4) - a).max() < 1e-15
    C0, T0 = o.init_env(A)
    assert C0.shape == (4, 4) and T0.shape == (4, 4, 4)
    assert np.abs(C0 - C0.T).max() < 1e-15
    # corner: trace up and left ket/bra legs
    c = np.zeros((2, 2, 2, 2))
    for d, Dd, r, R in np.ndindex(2, 2, 2, 2):
        c[d, Dd, r, R] = sum(A[s, u, l, d, r] * A[s, u, l, Dd, R]
                             for s in range(2) for u in range(2) for l in range(2))
    c = c.reshape(4, 4)
    assert np.abs(c / np.linalg.norm(c) - C0).max() < 1e-15


def test_eigen_step_diagonalises_corner():
    A = o.normalized_input(qi.raw_tensor(2, 2, 0))
    a = o.double_layer(A)
    C, T = o.init_env(A)
    C1, T1 = o.eigen_step(C, T, a, 16)
    assert C1.shape == (16, 16)
    assert np.abs(C1 - np.diag(np.diag(C1))).max() < 1e-13
    d = np.abs(np.diag(C1))
    assert np.all(np.diff(d) <= 1e-14)             # |lambda| descending


def test_qr_and_eigen_ctmrg_agree_small_chi():
    # Fig. 2(a): QR-CTMRG and standard CTMRG give the same energy at given chi
    A = o.normalized_input(qi.raw_tensor(2, 2, 0))
    Cq, Tq, iq = o.ctmrg(A, 16, "qr", tol=1e-12, max_iter=200)
    Ce, Te, ie = o.ctmrg(A, 16, "eigen", tol=1e-12, max_iter=200)
    assert iq["converged"] and ie["converged"]
    Eq, Ee = o.energy(Cq, Tq, A, 1.0, 0.5), o.energy(Ce, Te, A, 1.0, 0.5)
    assert abs(Eq - Ee) < 1e-10
    sq, se = o.corner_spectrum(Cq), o.corner_spectrum(Ce)
    assert np.abs(sq - se).max() < 1e-8


def test_qr_vs_eigen_difference_shrinks_with_chi():
    # Fig. 2(a): both converge to the same chi -> infinity limit
    A = o.normalized_input(qi.raw_tensor(2, 3, 1))
    diffs = []
    for chi in (9, 27):
        Cq, Tq, _ = o.ctmrg(A, chi, "qr", tol=1e-11, max_iter=400)
        Ce, Te, _ = o.ctmrg(A, chi, "eigen", tol=1e-11, max_iter=400)
        diffs.append(abs(o.energy(Cq, Tq, A) - o.energy(Ce, Te, A)))
    assert diffs[1] <= diffs[0] + 1e-12
