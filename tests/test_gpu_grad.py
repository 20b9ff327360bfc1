"""Energy gradient dE/dA on the GPU (hand-written adjoint, FP64) against the
oracle's complex-step derivatives and against central differences.

Tolerances: unrolled-k gradient vs the oracle's complex-step derivative of
the same k steps (the same function): 1e-9 relative; implicit fixed-point
gradient vs the complex-step derivative through the fixed point: 1e-8
relative (the FP64 target); central differences of converged GPU energies
(step 1e-6): |fd - g.v| <= 1e-5 |g| |v| (relative to the gradient's norm, so
that a direction along which the derivative happens to be small is not held
to an absolute bound); scale invariance <g, A> = 0: 1e-10 * |g|."""
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
def point():
    A = o.normalized_input(qi.raw_tensor(2, 2, 0))
    C, T, info = o.ctmrg(A, 8, "qr", tol=1e-14, max_iter=600)
    return A, C, T


def make_ctx(q, A, C, T, chi=8):
    ctx = q.QRCTM(2, 2, chi, with_nnn=True, with_grad=True, grad_tol=1e-13, grad_max_iter=400)
    ctx.init_env(cuda(A), cuda(C), cuda(T))
    return ctx


@pytest.mark.parametrize("rotation", [True, False])
@pytest.mark.parametrize("J2", [0.0, 0.5])
def test_unrolled_gradient_matches_complex_step(q, point, J2, rotation):
    A, C, T = point
    ctx = make_ctx(q, A, C, T)
    E, g = ctx.energy_grad(1.0, J2, mode="unroll", k_unroll=6, rotation=rotation)
    g = g.cpu().numpy()
    for seed in (1001, 1002):
        v = o.normalized_input(qi.raw_direction(2, 2, seed))
        ref = o.directional_derivative_unrolled(A, v, C, T, 6, 1.0, J2, rotate=rotation)
        got = float(np.sum(g * v))
        assert abs(got - ref) < 1e-9 * max(1.0, abs(ref)), (got, ref)


@pytest.mark.parametrize("J2", [0.0, 0.5])
def test_implicit_gradient_matches_complex_step(q, point, J2):
    A, C, T = point
    ctx = make_ctx(q, A, C, T)
    E, g = ctx.energy_grad(1.0, J2, mode="implicit")
    g = g.cpu().numpy()
    assert abs(E - o.energy(C, T, A, 1.0, J2)) < 1e-12
    for seed in (1003, 1004):
        v = o.normalized_input(qi.raw_direction(2, 2, seed))
        ref, _ = o.directional_derivative_fixed_point(A, v, C, T, 1.0, J2, tol=1e-13)
        got = float(np.sum(g * v))
        assert abs(got - ref) < 1e-8 * max(abs(ref), np.linalg.norm(g)), (got, ref)
    # E(lambda A) = E(A)  =>  <g, A> = 0 ; the gradient lies in the C4v subspace
    assert abs(float(np.sum(g * A))) < 1e-10 * np.linalg.norm(g)
    assert np.abs(o.c4v_sym(g) - g).max() < 1e-14 * np.abs(g).max()


def test_gradient_central_differences(q, point):
    """Central differences (step 1e-6) of converged GPU energies along 16
    seeded symmetric unit directions (seeds 1001..1016) against g . v, to
    1e-5 |g| |v| (J1-J2 at J2/J1 = 0.5)."""
    A, C, T = point
    ctx = make_ctx(q, A, C, T)
    _, g = ctx.energy_grad(1.0, 0.5, mode="implicit")
    g = g.cpu().numpy()
    gnorm = float(np.linalg.norm(g))
    assert gnorm > 1e-3
    c2 = q.QRCTM(2, 2, 8, with_nnn=True)
    eps = 1e-6
    for seed in range(1001, 1017):
        v = o.normalized_input(qi.raw_direction(2, 2, seed))
        Es = []
        for sgn in (1.0, -1.0):
            c2.init_env(cuda(A + sgn * eps * v), cuda(C), cuda(T))
            c2.run_to_convergence(tol=1e-14, max_iter=800)
            Es.append(c2.energy(1.0, 0.5))
        fd = (Es[0] - Es[1]) / (2 * eps)
        got = float(np.sum(g * v))
        assert abs(fd - got) < 1e-5 * gnorm * np.linalg.norm(v), (seed, fd, got, gnorm)


@pytest.fixture(scope="module")
def point_d3():
    A = o.normalized_input(qi.raw_tensor(2, 3, 7, bias=0.1))
    C, T, info = o.ctmrg(A, 12, "qr", tol=1e-13, max_iter=800)
    return A, C, T


@pytest.mark.parametrize("mode", ["implicit", "unroll"])
def test_split_precision_gradient_matches_fp64(q, point_d3, mode):
    """A split-precision context runs the contractions of the gradient call
    (taped steps, energy, reverse passes) on the TF32x3 tensor-core engine
    with FP32 accumulation: the energy it returns agrees with the FP64 one to
    2e-6 relative (three chained contractions of FP32-class accuracy) and its
    gradient to 1e-4 relative."""
    A, C, T = point_d3
    out = {}
    for prec in ("fp64", "split"):
        ctx = q.QRCTM(2, 3, 12, precision=prec, with_nnn=True, with_grad=True, grad_tol=1e-9,
                      grad_max_iter=300)
        ctx.init_env(cuda(A), cuda(C), cuda(T))
        E, g = ctx.energy_grad(1.0, 0.5, mode=mode, k_unroll=8)
        out[prec] = (E, g.cpu().numpy())
        ctx.close()
    (Ef, gf), (Es, gs) = out["fp64"], out["split"]
    assert abs(Es - Ef) < 2e-6 * abs(Ef), (Es, Ef)
    assert np.linalg.norm(gs - gf) < 1e-4 * np.linalg.norm(gf), np.linalg.norm(gs - gf)
