"""Train the warm-start network on steady fields from the batched solver.

    python -m paper_1908_08386_gb300.train_warmstart --out weights.npz --report report.json

Generates the training cavities (128 x 128, Ra log-uniform in [1e3, 1e6], Pr
0.71 or 7.0, up to three obstacles), solves them to steady state with the
batched FP32 solver, trains the network on the first `--train` of them and
reports on the rest: RMS error of T and of the velocity, and the steps the
LBM-FVM iteration needs from the prediction versus from rest.
"""

from __future__ import annotations

import argparse
import json
import time

import numpy as np


def steps_to_residual(cases, net, tol, warm, check_every=500, max_steps=600000, store="f32"):
    """Steps each cavity needs to reach `tol`, from rest or from the network's prediction."""
    import torch

    from . import Batch
    from . import warmstart as W

    b = Batch(cases, store=store)
    if store == "f32" and tol >= 1e-7:
        b.set_polish("f32", 0)
    if warm:
        W.warm_start(b, net, cases)
    torch.cuda.synchronize()
    t0 = time.time()
    steps, r = b.run(tol=tol, check_every=check_every, max_steps=max_steps)
    torch.cuda.synchronize()
    secs = time.time() - t0
    nus = [b.nusselt(i)[0] for i in range(len(cases))]
    b.close()
    return steps, r, secs, nus


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--count", type=int, default=2000)
    ap.add_argument("--train", type=int, default=1800)
    ap.add_argument("--seed", type=int, default=20190823)
    ap.add_argument("--widths", default="32,64,96,160")
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--gen-tol", type=float, default=1e-6)
    ap.add_argument("--eval-cavities", type=int, default=32)
    ap.add_argument("--out", default="warmstart_weights.npz")
    ap.add_argument("--report", default=None)
    a = ap.parse_args(argv)

    from . import surrogate as S
    from . import warmstart as W
    from . import workloads as WL

    widths = tuple(int(w) for w in a.widths.split(","))
    report = {"widths": widths, "count": a.count, "train": a.train, "seed": a.seed, "epochs": a.epochs,
              "batch": a.batch, "lr": a.lr}
    cases = WL.warm_start_cases(a.count, a.seed)
    t0 = time.time()
    targets, steps, r = W.generate(cases, tol=a.gen_tol)
    report["generate_s"] = time.time() - t0
    report["generate_steps_max"] = int(steps.max())
    train_set = W.Dataset(cases[:a.train], targets[:a.train])
    test_idx = list(range(a.count - a.train))
    test_set = W.Dataset(cases[a.train:], targets[a.train:])
    net = S.Surrogate(widths)
    report["parameters"] = int(sum(np.prod(p.shape) for p in net.get_params()))
    t0 = time.time()
    report["loss"] = W.train(net, train_set, epochs=a.epochs, batch=a.batch, lr=a.lr, seed=a.seed)
    report["train_s"] = time.time() - t0
    pred = W.predict(net, test_set, test_idx)
    tg = targets[a.train:]
    _, _, fluid = W.case_arrays(cases[a.train:])
    report["test_T_rms"], report["test_u_rel_rms"] = W.errors(pred, tg, fluid)
    # the same measures for the rest state (u = 0, T = 1/2) as a yardstick
    rest = np.zeros_like(pred)
    rest[..., 2] = 0.5
    report["rest_T_rms"], report["rest_u_rel_rms"] = W.errors(rest, tg, fluid)
    net.save(a.out)
    ev = cases[a.train:a.train + a.eval_cavities]
    for tol in ((1e-6,) if ev else ()):
        sc, rc, tc, nc = steps_to_residual(ev, net, tol, warm=False)
        sw, rw, tw, nw = steps_to_residual(ev, net, tol, warm=True)
        report[f"steps_cold_{tol:g}"] = [int(x) for x in sc]
        report[f"steps_warm_{tol:g}"] = [int(x) for x in sw]
        report[f"seconds_cold_{tol:g}"] = tc
        report[f"seconds_warm_{tol:g}"] = tw
        report[f"nu_rel_diff_{tol:g}"] = float(max(abs(x - y) / abs(y) for x, y in zip(nw, nc)))
    print(json.dumps({k: v for k, v in report.items() if k != "loss"}, indent=1))
    if a.report:
        with open(a.report, "w") as f:
            json.dump(report, f, indent=1)


if __name__ == "__main__":
    main()
