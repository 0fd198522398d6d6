"""Writes steady_nusselt.json (sides 64, 96, 128) or steady_nusselt_<sides>.json
(other sides): the FP64 oracle's steady hot-wall Nusselt numbers (residual
below 1e-8, checked every 1000 steps; Eq. 90, trapezoid mean) of the seeded
uneven-cavity draw that bench.py's time-to-steady measurement runs
(workloads.cavity_batch(count, 20190822, sizes=sides), U0 capped).  Calls
only the oracle; one process per cavity.

    python tests/golden/make_steady_nusselt.py [count] [processes] [sides, e.g. 128,192,256]
"""

import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

SEED = 20190822
SIZES = (64, 96, 128)
TOL = 1e-8


def steady_nusselt(args):
    i, sizes = args
    os.environ["OMP_NUM_THREADS"] = "1"
    import oracle
    from paper_1908_08386_gb300 import workloads as WL

    c = WL.cavity_batch(i + 1, SEED, sizes=sizes)[i]
    o = oracle.Oracle.from_groups(c.nx, c.ny, c.Ra, c.Pr, c.Ma, mask=c.mask, t_init=c.t_init)
    t0 = time.time()
    r = float("inf")
    while o.step_count < 50_000_000:
        o.step(1000)
        r = o.residual()
        if r < TOL:
            break
    nu = o.nusselt()[0]
    return {"index": i, "nx": c.nx, "ny": c.ny, "Ra": c.Ra, "Pr": c.Pr, "Ma": c.Ma, "steps": o.step_count,
            "residual": r, "nu_mean_hot": nu, "seconds": time.time() - t0}


def main():
    count = int(sys.argv[1]) if len(sys.argv) > 1 else 32
    procs = int(sys.argv[2]) if len(sys.argv) > 2 else os.cpu_count()
    sizes = tuple(int(x) for x in sys.argv[3].split(",")) if len(sys.argv) > 3 else SIZES
    name = "steady_nusselt.json" if sizes == SIZES else "steady_nusselt_%s.json" % "_".join(map(str, sizes))
    # rows already stored for this draw are kept (a longer draw extends a
    # shorter one: its first cavities are the same)
    kept = {}
    try:
        old = json.load(open(os.path.join(HERE, name)))
        if old.get("seed") == SEED and tuple(old.get("sizes", ())) == sizes and old.get("tol") == TOL:
            kept = {r["index"]: r for r in old["cavities"] if r["index"] < count}
    except (OSError, ValueError):
        pass
    with mp.get_context("spawn").Pool(procs) as pool:
        # the largest cavities first, so that the pool ends together
        from paper_1908_08386_gb300 import workloads as WL

        cases = WL.cavity_batch(count, SEED, sizes=sizes)
        todo = sorted((i for i in range(count) if i not in kept), key=lambda i: -cases[i].nx * cases[i].ny)
        rows = list(kept.values()) + pool.map(steady_nusselt, [(i, sizes) for i in todo], chunksize=1)
    rows.sort(key=lambda r: r["index"])
    out = {"_source": "FP64 CPU oracle (oracle/lbmfvm_oracle.c) run to a steady residual below 1e-8 "
                      "(checks every 1000 steps) by tests/golden/make_steady_nusselt.py",
           "seed": SEED, "sizes": list(sizes), "velocity": "capped", "tol": TOL, "cavities": rows}
    with open(os.path.join(HERE, name), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
