"""Pins for the oracle's derivatives (Automatic differentiation paragraph;
fixed-point AD named in the Discussion), CPU only."""
import numpy as np
import pytest

from oracle import qrctm_oracle as o
import qrctm_inputs as qi


@pytest.fixture(scope="module")
def converged():
    A = o.normalized_input(qi.raw_tensor(2, 2, 0))
    C, T, info = o.ctmrg(A, 8, "qr", tol=1e-13, max_iter=400)
    assert info["converged"]
    return A, C, T


@pytest.mark.parametrize("J2", [0.0, 0.5])
def test_complex_step_matches_central_difference(converged, J2):
    A, C, T = converged
    v = o.normalized_input(qi.raw_direction(2, 2, 1001))
    g_cs, info = o.directional_derivative_fixed_point(A, v, C, T, 1.0, J2, tol=1e-12)
    eps = 1e-5
    Ep = o.energy_at(A + eps * v, C, T, 1.0, J2, tol=1e-14)
    Em = o.energy_at(A - eps * v, C, T, 1.0, J2, tol=1e-14)
    fd = (Ep - Em) / (2 * eps)
    assert abs(g_cs - fd) < 1e-8
    assert abs(g_cs) > 1e-3


def test_energy_is_scale_invariant(converged):
    # E(lambda A) = E(A)  =>  dE/dA . A = 0
    A, C, T = converged
    g, _ = o.directional_derivative_fixed_point(A, A, C, T, 1.0, 0.5, tol=1e-12)
    assert abs(g) < 1e-11


def test_unrolled_gradient_converges_to_fixed_point(converged):
    # gradient of k tracked steps from a detached converged environment
    A, C, T = converged
    v = o.normalized_input(qi.raw_direction(2, 2, 1002))
    g_fp, _ = o.directional_derivative_fixed_point(A, v, C, T, 1.0, 0.0, tol=1e-12)
    errs = [abs(o.directional_derivative_unrolled(A, v, C, T, k) - g_fp) for k in (2, 10, 40)]
    assert errs[2] < errs[0]
    assert errs[2] < 1e-6
