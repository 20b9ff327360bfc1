"""Seeded synthetic inputs for QR-CTMRG runs.

This module draws the raw random numbers that both the CPU oracle and the
CUDA library consume. It holds none of the method's arithmetic: every array it
returns is a raw draw (or a fixed mask) that each side then symmetrises under
C4v and normalises with its own code.

Recipe (the paper's optimised tensors are not available, so these stand in
for them; see the workload list in the iPEPS and Results paragraphs):

* ``raw_tensor(d, D, seed, decay=False, bias=0.0)`` returns
  ``X = G * w + bias * P`` with ``G ~ N(0,1)`` of shape ``(d, D, D, D, D)``
  drawn from ``numpy.random.default_rng(seed)`` in C order,
  ``w = 0.5 ** (number of nonzero virtual indices)`` when ``decay`` is set
  (else 1), and ``P[s,0,0,0,0] = 1`` for every physical index ``s`` (a
  product-state bias).  The C4v-symmetric input of a run is
  ``A = sym(X) / ||sym(X)||_F``; ``w`` and ``P`` are C4v invariant, so
  ``sym(X) = sym(G) * w + bias * P``.
* ``raw_direction(d, D, seed)`` returns ``N(0,1)`` draws for a
  finite-difference direction ``v = sym(N) / ||sym(N)||``.
* ``network_input(model, q, beta)`` returns the classical spin model itself
  (Discussion: classical partition functions) as the C4v network tensor
  ``a[u,l,d,r] = sum_s W[s,u] W[s,l] W[s,d] W[s,r]`` with ``W = B^(1/2)`` and
  ``B`` the bond Boltzmann weight (``exp(beta s s')`` for Ising, s = +-1;
  ``exp(beta delta_{s s'})`` for q-state Potts), the tensor with the spin
  (Ising) or ``delta_{s,0}`` (Potts) inserted, and the fixed-spin boundary
  vector ``W[0]``.  This is the model's definition, the input both sides
  consume; the CTMRG arithmetic stays in each side's own code.
"""
from __future__ import annotations

import numpy as np

__all__ = ["raw_tensor", "raw_direction", "decay_mask", "network_input", "WORKLOADS",
           "NETWORK_WORKLOADS"]


def decay_mask(d: int, D: int) -> np.ndarray:
    """``w[s,u,l,dn,r] = 0.5 ** #(nonzero virtual indices)``; invariant under C4v."""
    idx = np.indices((d, D, D, D, D))
    nz = (idx[1] > 0).astype(np.int64) + (idx[2] > 0) + (idx[3] > 0) + (idx[4] > 0)
    return np.power(0.5, nz).astype(np.float64)


def raw_tensor(d: int, D: int, seed: int = 0, decay: bool = False,
               bias: float = 0.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((d, D, D, D, D))
    if decay:
        G = G * decay_mask(d, D)
    if bias:
        P = np.zeros((d, D, D, D, D))
        P[:, 0, 0, 0, 0] = 1.0
        G = G + bias * P
    return np.ascontiguousarray(G, dtype=np.float64)


def raw_direction(d: int, D: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((d, D, D, D, D)))


def network_input(model: str, q: int, beta: float):
    """(a, a_obs, v): network tensor (bond q), observable tensor, boundary vector."""
    if model == "ising":
        spins = np.array([1.0, -1.0])
        B = np.exp(beta * np.outer(spins, spins))
        o = spins
    elif model == "potts":
        B = np.exp(beta * np.eye(q))
        o = (np.arange(q) == 0).astype(np.float64)
    else:
        raise ValueError(model)
    lam, V = np.linalg.eigh(B)
    W = (V * np.sqrt(np.clip(lam, 0.0, None))) @ V.T
    a = np.einsum("su,sl,sd,sr->uldr", W, W, W, W)
    a_obs = np.einsum("s,su,sl,sd,sr->uldr", o, W, W, W, W)
    return (np.ascontiguousarray(a), np.ascontiguousarray(a_obs),
            np.ascontiguousarray(W[0]))


# Classical networks fed directly: near (below) the critical coupling, where
# the correlation length is tens of sites (Ising beta_c = 0.4407, 3-state
# Potts beta_c = ln(1 + sqrt 3) = 1.005).
NETWORK_WORKLOADS = {
    "ising_b2_chi256": dict(model="ising", q=2, beta=0.43, chi=256, fixed=False),
    "potts3_b3_chi243": dict(model="potts", q=3, beta=0.95, chi=243, fixed=False),
}


# The workloads, by what they are.  ``chi`` is the environment bond,
# ``decay``/``bias`` select the raw-tensor recipe above.
WORKLOADS = {
    "d2_D2_chi16": dict(d=2, D=2, chi=16, seed=0, decay=False, bias=0.0,
                        tol=1e-12, max_iter=200),
    "d2_D4_chi64": dict(d=2, D=4, chi=64, seed=0, decay=False, bias=0.1,
                        tol=1e-12, max_iter=500),
    "d2_D6_chi144": dict(d=2, D=6, chi=144, seed=0, decay=True, bias=0.0,
                         tol=1e-10, max_iter=500),
    "d2_D6_chi600": dict(d=2, D=6, chi=600, seed=0, decay=True, bias=0.0,
                         tol=1e-10, max_iter=500),
    "d2_D8_chi64": dict(d=2, D=8, chi=64, seed=0, decay=True, bias=0.0,
                        tol=1e-10, max_iter=6000),
    "d2_D8_chi256": dict(d=2, D=8, chi=256, seed=0, decay=True, bias=0.0,
                         tol=1e-10, max_iter=500),
    "d2_D8_chi512": dict(d=2, D=8, chi=512, seed=0, decay=True, bias=0.0,
                         tol=1e-10, max_iter=500),
}
