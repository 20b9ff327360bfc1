"""L-BFGS variational optimisation on the GPU (Automatic differentiation
paragraph) against the oracle's optimiser: same start, same options, FP64.
Both sides take the same decisions (accepted points, line-search halvings),
so the energies of the accepted points and the final tensor agree to
rounding of the gradients."""
import numpy as np
import pytest

import qrctm_inputs as qi
from oracle import qrctm_oracle as o

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("J2", [0.0, 0.5])
def test_optimize_matches_oracle(J2):
    import paper_2505_00494_b300 as q
    A0 = o.normalized_input(qi.raw_tensor(2, 2, 0, False, 0.1))
    x, fs, nev, failed = o.optimize_ipeps(A0, 8, J2=J2, n_steps=6, k=6, nograd=2,
                                          env_tol=1e-12)
    ctx = q.QRCTM(2, 2, 8, check_every=5, with_grad=True, with_nnn=J2 != 0, opt_history=10)
    A = _dev(A0)
    en, evals, gfailed = ctx.optimize(A, 6, J2=J2, k_unroll=6, nograd_steps=2, env_tol=1e-12)
    ctx.close()
    assert not failed and not gfailed
    assert evals == nev
    assert len(en) == len(fs)
    assert np.abs(en - np.array(fs)).max() < 1e-9
    assert all(f2 <= f1 for f1, f2 in zip(en, en[1:]))
    assert np.abs(A.cpu().numpy() - x).max() < 1e-7 * np.abs(x).max()


def test_optimize_split_precision_descends():
    import paper_2505_00494_b300 as q
    A0 = o.normalized_input(qi.raw_tensor(2, 3, 0, True, 0.0))
    ref = q.QRCTM(2, 3, 18, check_every=5, with_grad=True, opt_history=10)
    Ar = _dev(A0)
    e64, _, _ = ref.optimize(Ar, 4, k_unroll=8, env_tol=1e-11)
    ref.close()
    ctx = q.QRCTM(2, 3, 18, precision="split", check_every=5, with_grad=True, opt_history=10)
    As = _dev(A0)
    es, _, _ = ctx.optimize(As, 4, k_unroll=8, env_tol=1e-6)
    ctx.close()
    assert all(f2 <= f1 for f1, f2 in zip(es, es[1:]))
    assert es[-1] < es[0] - 1e-3
    # FP32-class contractions: same path to 1e-5 per site over a few steps
    assert np.abs(np.array(es) - np.array(e64[:len(es)])).max() < 1e-5


def test_optimize_argument_errors():
    import paper_2505_00494_b300 as q
    A0 = _dev(o.normalized_input(qi.raw_tensor(2, 2, 0, False, 0.1)))
    ctx = q.QRCTM(2, 2, 8, with_grad=True)        # no optimiser workspace
    with pytest.raises(q.QRCTMError) as ei:
        ctx.optimize(A0, 2)
    assert ei.value.code == 1
    ctx.close()
    ctx = q.QRCTM(2, 2, 8, with_grad=True, opt_history=4)
    en, evals, _ = ctx.optimize(A0, 0)           # start only
    assert len(en) == 1 and evals == 1
    with pytest.raises(q.QRCTMError):
        ctx.optimize(A0, 1, k_unroll=40)
    ctx.close()
