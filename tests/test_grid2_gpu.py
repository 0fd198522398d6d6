"""Grid setting 2 (Section 5.1, Fig. 30: the energy balance on coarse volumes
of 2 x 2 lattice spacings, a coarse explicit step every k lattice steps) on
the GPU against the FP64 oracle: FP64 and double-single storage to rounding
(1e-9), FP32 within max|du|/U0 and max|dT| of 1e-5 after the same step
count; the steady state of every k and of both grid settings."""

import math

import numpy as np
import pytest

import oracle
import paper_1908_08386_gb300 as L

pytestmark = pytest.mark.gpu

U0 = 0.1
MA = U0 * math.sqrt(3.0)
TOL = {"f64": 1e-9, "f32x2": 1e-9, "f32": 1e-5}


def deviation(gpu, orc):
    _, ug, vg, Tg = gpu.fields()
    _, uo, vo, To = orc.fields()
    return max(np.abs(ug - uo).max(), np.abs(vg - vo).max()) / U0, np.abs(Tg - To).max()


@pytest.mark.parametrize("store", ["f64", "f32x2", "f32"])
@pytest.mark.parametrize("k", [1, 4])
@pytest.mark.parametrize("shape", [(65, 65), (129, 65)])
def test_matches_oracle(store, k, shape):
    nx, ny = shape
    gpu = L.Cavity(nx, ny, Ra=1e4, Pr=0.71, Ma=MA, store=store, fv_grid=2, fv_every=k)
    orc = oracle.Oracle.from_groups(nx, ny, 1e4, 0.71, MA, fv_grid=2, fv_every=k)
    # the initial node temperatures already come from the volumes
    du, dT = deviation(gpu, orc)
    assert du == 0 and dT <= 1e-7, (du, dT)
    for n in (1, 2, 3, 5, 600, 2000):  # coarse steps at every k-th step, graph replays aligned
        gpu.step(n)
        orc.step(n)
    du, dT = deviation(gpu, orc)
    assert du <= TOL[store] and dT <= TOL[store], (du, dT)


def test_steady_state_does_not_depend_on_k_and_matches_grid_setting_1():
    n = 41
    nu = {}
    for grid, k in ((1, 1), (2, 1), (2, 4)):
        c = L.Cavity(n, n, Ra=1e4, Pr=0.71, Ma=MA, store="f32x2", fv_grid=grid, fv_every=k)
        _, r = c.run_to_steady(tol=1e-9, check_every=1000, max_steps=400_000)
        assert r < 1e-9
        nu[(grid, k)] = c.nusselt()[0]
    assert abs(nu[(2, 4)] / nu[(2, 1)] - 1) <= 1e-7, nu
    assert abs(nu[(2, 1)] / nu[(1, 1)] - 1) <= 0.01, nu
    orc = oracle.Oracle.from_groups(n, n, 1e4, 0.71, MA, fv_grid=2, fv_every=4)
    for _ in range(400):
        orc.step(1000)
        if orc.residual() < 1e-10:
            break
    assert abs(nu[(2, 4)] / orc.nusselt()[0] - 1) <= 1e-7


def test_checkpoints_are_refused():
    c = L.Cavity(41, 41, Ra=1e4, Pr=0.71, Ma=MA, fv_grid=2)
    with pytest.raises(L.LbmfvmError) as e:
        c.save("/tmp/never_written.ckpt")
    assert e.value.code == L.LBMFVM_ERR_ARG
