"""Write converged-environment fixtures computed by the oracle alone.

    python tests/golden/make_golden.py d2_D2_chi16 d2_D4_chi64 d2_D6_chi144 d2_D8_chi64

For each workload (inputs from qrctm_inputs.WORKLOADS) the oracle runs its
warm-up and QR-CTMRG steps until the corner spectrum changes by less than the
tolerance, then records the sorted |eig C| and the energies per site at
J2/J1 = 0 and 0.5.  Nothing here touches the GPU library.
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

TOL = {"d2_D2_chi16": 1e-12, "d2_D4_chi64": 1e-11, "d2_D6_chi144": 1e-10, "d2_D8_chi64": 1e-10}
MAX_ITER = {"d2_D2_chi16": 2000, "d2_D4_chi64": 4000, "d2_D6_chi144": 6000, "d2_D8_chi64": 6000}


def main(names):
    for name in names:
        w = qi.WORKLOADS[name]
        d, D, chi = w["d"], w["D"], w["chi"]
        A = o.normalized_input(qi.raw_tensor(d, D, w["seed"], w["decay"], w["bias"]))
        layers = "split" if 2 * d < D * D else "double"
        t0 = time.time()
        C, T, info = o.ctmrg(A, chi, "qr", tol=TOL[name], max_iter=MAX_ITER[name],
                             layers=layers, check_every=5)
        # the map alternates a sign gauge; an even step count keeps the
        # gauge of the environment used for the energies fixed
        out = {
            "workload": name, "d": d, "D": D, "chi": chi, "layers": layers,
            "tol": TOL[name], "iters": int(info["iters"]), "delta": float(info["delta"]),
            "converged": bool(info["converged"]),
            "spectrum": [float(x) for x in o.corner_spectrum(C)],
            "E_J2_0": float(o.energy(C, T, A, 1.0, 0.0)),
            "E_J2_0.5": float(o.energy(C, T, A, 1.0, 0.5)),
            "oracle_seconds": time.time() - t0,
            "source": "oracle/qrctm_oracle.py ctmrg (QR-CTMRG paragraph), energy (Results)",
        }
        path = os.path.join(HERE, f"converged_{name}.json")
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print(name, out["iters"], out["delta"], out["E_J2_0"], out["E_J2_0.5"],
              f"{out['oracle_seconds']:.0f}s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["d2_D2_chi16", "d2_D4_chi64"])
