"""Writes tests/golden/d5_chi96_8x8.json: the FP64 oracle on an 8x8 lattice at the large
workload's D=5, chi=96 and 4x4 blocks (4 blocks, 8 messages), tensors U[0,1] + 0.1 N(0,1)
rounded to FP32 (seed 4), run for a fixed number of sweeps under the workload's stop rules
(App. A fit rule at 1e-6 with at most 10 fit sweeps, warm-started fits), then <sigma_z> and
<sigma_x> read out on every site.  The benchmark runs the same schedule on the GPU and states
its <O> error against these values.  Calls only the oracle and the seeded input generators.

  python tests/golden/make_d5_chi96_8x8.py      (several minutes on 8 cores)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import blockbp as ob  # noqa: E402
from paper_2301_05844_gb300 import inputs as I  # noqa: E402

PARAMS = dict(L=8, d=2, D=5, block=4, chi=96, seed=4, fit_tol=1e-6, fit_max_sweeps=10, warm_start=True, sweeps=6)


def main():
    p = PARAMS
    T = I.uniform_noise_peps(p["L"], p["L"], p["d"], p["D"], seed=p["seed"], dtype=np.float32)
    o = ob.Lattice(p["L"], p["L"], p["d"], p["D"], p["block"], p["block"], [np.asarray(t, np.float64) for t in T],
                   chi=p["chi"], fit_tol=p["fit_tol"], fit_max_sweeps=p["fit_max_sweeps"], seed=p["seed"],
                   warm_start=p["warm_start"])
    t0 = time.time()
    for k in range(p["sweeps"]):
        r = o.sweep()
        print(f"sweep {k + 1}: residual {r:.3e}, fit sweeps {o.fit_sweeps[-1]}, {time.time() - t0:.0f} s", flush=True)
    t1 = time.time()
    n = p["L"] * p["L"]
    terms = [[(s, I.SIGMA_Z)] for s in range(n)] + [[(s, I.SIGMA_X)] for s in range(n)]
    v = o.expect(terms)
    t2 = time.time()
    out = {"params": p, "residuals": o.residuals, "fit_sweeps": o.fit_sweeps,
           "sz": [float(x) for x in v[:n].real], "sx": [float(x) for x in v[n:].real],
           "max_abs_imag": float(np.max(np.abs(v.imag))), "oracle_seconds": {"sweeps": t1 - t0, "readout": t2 - t1}}
    with open(os.path.join(HERE, "d5_chi96_8x8.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(f"done: sweeps {t1 - t0:.0f} s, read-out {t2 - t1:.0f} s")


if __name__ == "__main__":
    main()
