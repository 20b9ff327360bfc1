"""Pins for the oracle's variational optimisation (Automatic differentiation
paragraph: L-BFGS, two untracked then k tracked CTMRG steps, boundary reused
except in the line search), CPU only.

* the C4v orbit basis has n(D) elements (the iPEPS footnote; 1332 at d=2,
  D=8 as the paper prints), is orthonormal and projects like sym();
* the two-loop recursion equals the dense BFGS inverse-Hessian recursion;
* the generic minimiser finds the exact minimiser of a quadratic and the
  Rosenbrock minimum;
* the unrolled gradient matches central finite differences of the same
  k-step energy, is orthogonal to A (scale invariance) and C4v symmetric;
* the iPEPS optimisation lowers the energy at every accepted step and ends
  at the minimum scipy's L-BFGS-B finds from the same start.
"""
import json
import os

import numpy as np
import pytest

import qrctm_inputs as qi
from oracle import qrctm_oracle as o

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


@pytest.mark.parametrize("D", [1, 2, 3, 4])
def test_orbit_basis(D):
    B = o.c4v_orbit_basis(2, D)
    assert len(B) == round(o.n_params(2, D))
    M = np.array([b.ravel() for b in B])
    assert np.abs(M @ M.T - np.eye(len(B))).max() < 1e-14
    X = np.random.default_rng(D).standard_normal((2, D, D, D, D))
    P = sum(np.sum(b * X) * b for b in B)
    assert np.abs(P - o.c4v_sym(X)).max() < 1e-13


def test_orbit_count_d2_D8_is_the_papers():
    assert len(o.c4v_orbit_basis(2, 8)) == GOLD["n_params_d2_D8"]["value"]


def dense_bfgs_direction(g, pairs):
    """-H g with H from the textbook BFGS inverse update applied to each
    pair in turn, H0 = gamma I (gamma from the newest pair)."""
    n = g.size
    s, y = pairs[-1]
    H = np.eye(n) * (s @ y) / (y @ y)
    for s, y in pairs:
        r = 1.0 / (y @ s)
        V = np.eye(n) - r * np.outer(y, s)
        H = V.T @ H @ V + r * np.outer(s, s)
    return -H @ g


def test_two_loop_equals_dense_bfgs():
    rng = np.random.default_rng(0)
    n = 7
    Q = rng.standard_normal((n, n))
    Hs = Q @ Q.T + n * np.eye(n)             # curvature pairs y = Hs s
    pairs = []
    for _ in range(4):
        s = rng.standard_normal(n)
        pairs.append((s, Hs @ s))
    g = rng.standard_normal(n)
    assert np.abs(o.lbfgs_direction(g, []) + g).max() == 0.0
    p = o.lbfgs_direction(g, pairs)
    assert np.abs(p - dense_bfgs_direction(g, pairs)).max() < 1e-12 * np.abs(p).max()
    # secant condition for the newest pair: H y = s
    s, y = pairs[-1]
    assert np.abs(-o.lbfgs_direction(y, pairs) - s).max() < 1e-12 * np.abs(s).max()


def test_lbfgs_quadratic_and_rosenbrock():
    rng = np.random.default_rng(1)
    n = 6
    Q = rng.standard_normal((n, n))
    H = Q @ Q.T + np.eye(n)
    b = rng.standard_normal(n)

    def quad(x, trial):
        return 0.5 * x @ H @ x - b @ x, H @ x - b

    x, fs, _, _ = o.lbfgs_minimize(quad, np.zeros(n), 60, history=10, step0=0.1)
    assert np.abs(x - np.linalg.solve(H, b)).max() < 1e-8
    assert all(f2 <= f1 for f1, f2 in zip(fs, fs[1:]))

    def rosen(x, trial):
        f = (1 - x[0]) ** 2 + 100 * (x[1] - x[0] ** 2) ** 2
        g = np.array([-2 * (1 - x[0]) - 400 * x[0] * (x[1] - x[0] ** 2),
                      200 * (x[1] - x[0] ** 2)])
        return f, g

    x, fs, _, _ = o.lbfgs_minimize(rosen, np.array([-1.2, 1.0]), 200, history=5, step0=0.1,
                                   max_ls=30)
    assert np.abs(x - 1.0).max() < 1e-6


@pytest.fixture(scope="module")
def d2_state():
    A = o.normalized_input(qi.raw_tensor(2, 2, 0, False, 0.1))
    C, T, _ = o.ctmrg(A, 8, "qr", tol=1e-12, max_iter=2000, check_every=5)
    return A, C, T


@pytest.mark.parametrize("J2", [0.0, 0.5])
def test_unrolled_gradient_matches_finite_differences(d2_state, J2):
    A, C, T = d2_state
    k = 4
    E, g, _, _ = o.unrolled_energy_grad(A, C, T, k, 1.0, J2)
    rng = np.random.default_rng(5)

    def Ek(X):
        Ck, Tk = C, T
        for _ in range(k):
            Ck, Tk = o.qr_step(Ck, Tk, X)
        return float(np.real(o.energy(Ck, Tk, X, 1.0, J2)))

    assert abs(Ek(A) - E) < 1e-14
    eps = 1e-5
    for _ in range(3):
        v = o.c4v_sym(rng.standard_normal(A.shape))
        v /= np.linalg.norm(v)
        fd = (Ek(A + eps * v) - Ek(A - eps * v)) / (2 * eps)
        assert abs(fd - np.sum(g * v)) < 1e-8
    assert abs(np.sum(g * A)) < 1e-12 * np.linalg.norm(g)
    assert np.abs(o.c4v_sym(g) - g).max() < 1e-15


def test_optimize_ipeps_descends_to_scipy_minimum():
    from scipy.optimize import minimize
    A0 = o.normalized_input(qi.raw_tensor(2, 2, 0, False, 0.1))
    x, fs, nev, _ = o.optimize_ipeps(A0, 8, n_steps=80, k=6)
    assert all(f2 <= f1 for f1, f2 in zip(fs, fs[1:]))
    assert np.abs(o.c4v_sym(x) - x).max() < 1e-15
    B = o.c4v_orbit_basis(2, 2)

    def fun(c):
        A = sum(ci * b for ci, b in zip(c, B))
        C, T, _ = o.ctmrg(A, 8, "qr", tol=1e-12, max_iter=2000, check_every=5)
        for _ in range(2):
            C, T = o.qr_step(C, T, A)
        E, g, _, _ = o.unrolled_energy_grad(A, C, T, 6)
        return E, np.array([np.sum(b * g) for b in B])

    r = minimize(fun, np.array([np.sum(b * A0) for b in B]), jac=True, method="L-BFGS-B",
                 options=dict(gtol=1e-9, ftol=1e-15, maxiter=300))
    assert abs(fs[-1] - r.fun) < 1e-9
