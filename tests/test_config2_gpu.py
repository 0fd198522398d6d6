"""The 1024^2 benchmark case's oracle instance: 256^2 nodes, Ra = 1e6,
Pr = 0.71, U0 = 0.1, 100,000 steps (about 39 free-fall times, a transient),
every storage precision against the FP64 oracle after the same step count.

Tolerances, from each storage's rounding: FP64 and double-single agree with
the oracle to rounding (1e-9).  FP32's unit roundoff (6e-8) is incurred every
step; over a transient of n = 1e5 steps it random-walks to about
sqrt(n) * 6e-8 = 2e-5 per node, a few times that at the worst of 65,536 nodes:
|du|/U0 and |dT| <= 1e-4.  (The 1e-5 FP32 bound holds after 1e4 steps, the
64^2 case; here the measured deviations are 1.8e-5 and 3.3e-5.)  FP16 and BF16
store 11 and 8 significant bits; their 0.5 % Nusselt criterion is a
steady-state one (met by the precision-ladder tests); over this transient they
are held to 1 % of the Nusselt number and |dT| <= 1e-2.
"""

import math

import numpy as np
import pytest

import oracle
import paper_1908_08386_gb300 as L

pytestmark = pytest.mark.gpu

N, RA, PR, STEPS = 256, 1e6, 0.71, 100_000
MA = 0.1 * math.sqrt(3.0)


@pytest.fixture(scope="module")
def reference():
    o = oracle.Oracle.from_groups(N, N, RA, PR, MA)
    o.step(STEPS)
    _, u, v, T = o.fields()
    nh, _, nc, _ = o.nusselt()
    return u, v, T, nh, nc


@pytest.mark.parametrize("store,tol_u,tol_T,tol_nu", [("f64", 1e-9, 1e-9, 1e-9), ("f32x2", 1e-9, 1e-9, 1e-9),
                                                      ("f32", 1e-4, 1e-4, 1e-4), ("f16", None, 1e-2, 1e-2),
                                                      ("bf16", None, 1e-2, 1e-2)])
def test_every_storage_against_the_oracle_after_100k_steps(reference, store, tol_u, tol_T, tol_nu):
    uo, vo, To, nho, nco = reference
    g = L.Cavity(N, N, Ra=RA, Pr=PR, Ma=MA, store=store)
    # residual checks every 1000 steps, each followed by the mass
    # renormalisation (which leaves u and T as the oracle's plain run has them)
    steps, _ = g.run_to_steady(tol=0.0, check_every=1000, max_steps=STEPS)
    assert steps == STEPS
    _, u, v, T = g.fields()
    nh, _, nc = g.nusselt()
    du = max(np.abs(u - uo).max(), np.abs(v - vo).max()) / 0.1
    dT = np.abs(T - To).max()
    print(f"{store}: max|du|/U0 = {du:.3e}, max|dT| = {dT:.3e}, Nu {nh:.6f} vs {nho:.6f}")
    assert dT <= tol_T
    if tol_u is not None:
        assert du <= tol_u
    assert abs(nh - nho) <= tol_nu * abs(nho) and abs(nc - nco) <= tol_nu * abs(nco)

