"""Write complex-step derivatives of the unrolled J1-J2 energy, computed by the
oracle alone, for the d2 D6 chi144 workload.

    python tests/golden/make_grad_golden.py

The unrolled energy is E(A, F^k(A; C0, T0)) with k = 20 tracked QR-CTMRG
steps from a detached environment (C0, T0) (Automatic differentiation
paragraph: the paper backpropagates through the last k steps; k = 20 is its
value for D = 6).  (C0, T0) is reproducible on any host from the oracle
alone: ``warmup(A, 144, layers="split")`` followed by ``N_START`` oracle QR
steps.  The derivative along v is Im E(A + i h v) / h (h = 1e-20), exact to
rounding.  Directions are v = sym(N) / ||sym(N)|| with N drawn by
``qrctm_inputs.raw_direction(2, 6, seed)``.  Nothing here touches the GPU
library.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import qrctm_inputs as qi  # noqa: E402
from oracle import qrctm_oracle as o  # noqa: E402

WORKLOAD = "d2_D6_chi144"
K = 20
N_START = 4
J1, J2 = 1.0, 0.5
SEEDS = (1001, 1002, 1003)
OUT = os.path.join(HERE, "grad_unroll20_d2_D6_chi144.json")


def start_env(A, chi):
    """The detached environment the unrolled derivative starts from."""
    C, T = o.warmup(A, chi, layers="split")
    for _ in range(N_START):
        C, T = o.qr_step(C, T, A, "split")
    return C, T


def main():
    w = qi.WORKLOADS[WORKLOAD]
    d, D, chi = w["d"], w["D"], w["chi"]
    A = o.normalized_input(qi.raw_tensor(d, D, w["seed"], w["decay"], w["bias"]))
    t0 = time.time()
    C, T = start_env(A, chi)
    out = {"workload": WORKLOAD, "k": K, "n_start_steps": N_START, "J1": J1, "J2": J2,
           "h": 1e-20, "layers": "split",
           "start": "oracle warmup(A, chi, layers='split') then n_start_steps oracle qr_step",
           "directions": {},
           "source": "oracle/qrctm_oracle.py directional_derivative_unrolled "
                     "(Automatic differentiation paragraph), energy (Results)"}
    for seed in SEEDS:
        v = o.normalized_input(qi.raw_direction(d, D, seed))
        t1 = time.time()
        val = o.directional_derivative_unrolled(A, v, C, T, K, J1, J2, layers="split")
        out["directions"][str(seed)] = val
        print(seed, repr(val), f"{time.time() - t1:.0f}s", flush=True)
        with open(OUT, "w") as f:
            json.dump(out, f, indent=1)
    out["oracle_seconds"] = time.time() - t0
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
