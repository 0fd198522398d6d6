"""Time to steady state of many cavities: the fast form against the plain loop.

Fast form: every cavity in one batch (one persistent launch per step), 16-bit
storage climbing the precision ladder (FP32, then double-single), initial
states from the learned warm start.  Plain form: one cavity after another,
each its own handle with FP32 storage from rest, switched to double-single
storage by the rule the batch's FP32 level follows (residual below 1e-6, or
within 100x of it and not halved for 32 checks): FP32 storage cannot reach a
1e-8 residual (its rounding floor is about 2e-7), and both forms finish in
the same arithmetic, with the same residual checks and mass
renormalisation.  Both stop each cavity at the same residual tolerance.
"""

from __future__ import annotations

import math
import time

import numpy as np

from . import Batch, Cavity


def plain_loop(cases, tol=1e-8, check_every=1000, max_steps=50_000_000, switch=1e-6, stall_checks=32,
               finish="f32x2", per_cavity=None):
    """(seconds, steps per cavity, final residuals, Nusselt numbers) of the
    per-cavity loop; handles are created before the clock starts.  `finish`
    is the storage the FP32 run switches to; `per_cavity`, if a list, receives
    (seconds, steps) of each cavity."""
    import torch

    pairs = []
    for c in cases:
        kw = dict(Ra=c.Ra, Pr=c.Pr, Ma=c.Ma, mask=c.mask, t_init=c.t_init,
                  fv_substeps=getattr(c, "substeps", 1))
        pairs.append((Cavity(c.nx, c.ny, store="f32", tma_config="auto", **kw),
                      Cavity(c.nx, c.ny, store=finish, tma_config="auto", **kw)))
    torch.cuda.synchronize()
    steps = np.zeros(len(cases), np.int64)
    res = np.zeros(len(cases))
    nus = np.zeros(len(cases))
    t0 = time.time()
    for i, (c32, c64) in enumerate(pairs):
        ti = time.time()
        cav, wide, best, since, r = c32, False, math.inf, 0, math.inf
        while steps[i] < max_steps:
            n, r = cav.run_to_steady(tol, check_every, check_every)
            steps[i] += n
            if r < tol:
                break
            if r < 0.5 * best:
                best, since = r, 0
            else:
                since += 1
            if not wide and (r < switch or (since >= stall_checks and r < 100 * switch)):
                c64.copy_state_from(c32)
                cav, wide, best, since = c64, True, math.inf, 0
        res[i] = r
        nus[i] = cav.nusselt()[0]
        if per_cavity is not None:
            per_cavity.append((time.time() - ti, int(steps[i])))
    torch.cuda.synchronize()
    secs = time.time() - t0
    for a, b in pairs:
        a.close()
        b.close()
    return secs, steps, res, nus


def fast_form(cases, net=None, store="f16", tol=1e-8, check_every=1000, max_steps=50_000_000):
    """(seconds, steps per cavity, final residuals, Nusselt numbers) of one
    batch; the warm start's inference is inside the timed region, creating
    the batch is not."""
    import torch

    from . import warmstart as W

    # cases drawn with energy sub-steps ask for the automatic choice
    auto = any(getattr(c, "substeps", 1) != 1 for c in cases)
    b = Batch(cases, store=store, fv_substeps=0 if auto else 1)
    torch.cuda.synchronize()
    t0 = time.time()
    if net is not None:
        W.warm_start(b, net, cases)
    steps, r = b.run(tol=tol, check_every=check_every, max_steps=max_steps)
    torch.cuda.synchronize()
    secs = time.time() - t0
    nus = np.array([b.nusselt(i)[0] for i in range(len(cases))])
    b.close()
    return secs, steps, r, nus
