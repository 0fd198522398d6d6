"""Writes config2_steady.json: the FP64 oracle's steady state of the 1024^2
benchmark case's oracle instance (256 x 256 nodes, Ra = 1e6, Pr = 0.71,
U0 = 0.1, fluid at rest with T = 0.5), run to a velocity residual below 1e-8
(checks every 1000 steps): the mean hot- and cold-wall Nusselt numbers
(Eq. 90) and the temperature on every fourth node of each direction.  Calls
only the oracle.

    python tests/golden/make_config2_steady.py
"""

import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

N, RA, PR, TOL = 256, 1e6, 0.71, 1e-8
MA = 0.1 * math.sqrt(3.0)


def main():
    import oracle

    o = oracle.Oracle.from_groups(N, N, RA, PR, MA)
    t0 = time.time()
    r = float("inf")
    while o.step_count < 20_000_000:
        o.step(1000)
        r = o.residual()
        if r < TOL:
            break
    mean_hot, local_hot, mean_cold, _ = o.nusselt()
    T = o.fields()[3]
    out = {"_source": "FP64 CPU oracle (oracle/lbmfvm_oracle.c) run to a steady residual below 1e-8 "
                      "(checks every 1000 steps) by tests/golden/make_config2_steady.py",
           "nx": N, "ny": N, "Ra": RA, "Pr": PR, "Ma": MA, "tol": TOL, "steps": o.step_count, "residual": r,
           "nu_mean_hot": mean_hot, "nu_mean_cold": mean_cold, "nu_local_hot_max": float(local_hot.max()),
           "T_every_4th": [[float(T[j, i]) for i in range(0, N, 4)] for j in range(0, N, 4)],
           "seconds": time.time() - t0}
    with open(os.path.join(HERE, "config2_steady.json"), "w") as fh:
        json.dump(out, fh)


if __name__ == "__main__":
    main()
