"""Finite-difference velocity-gradient box walls (Section 3, hybrid method 2,
Eqs. 61-72) on the GPU against the FP64 oracle, element by element: FP64 and
double-single storage to rounding (1e-9), FP32 within max|du|/U0 and max|dT|
of 1e-5 after the same step count; on the small benchmark cavity, ragged grids
with obstacles (whose surfaces keep the extrapolation), a lid-driven cavity
and a force-driven channel."""

import math

import numpy as np
import pytest

import oracle
import paper_1908_08386_gb300 as L
from paper_1908_08386_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

U0 = 0.1
MA = U0 * math.sqrt(3.0)
TOL = {"f64": 1e-9, "f32x2": 1e-9, "f32": 1e-5}


def obstacle_mask(nx, ny):
    return WL.rasterize([("rect", 0.3 * nx, 0.35 * ny, 0.15 * nx, 0.2 * ny),
                         ("circle", 0.68 * nx, 0.6 * ny, 0.22 * ny)], nx, ny)


def deviation(gpu, orc, u_scale=U0):
    _, ug, vg, Tg = gpu.fields()
    _, uo, vo, To = orc.fields()
    return max(np.abs(ug - uo).max(), np.abs(vg - vo).max()) / u_scale, np.abs(Tg - To).max()


@pytest.mark.parametrize("store", ["f64", "f32x2", "f32"])
def test_small_cavity_matches_oracle(store):
    case = WL.config_small()
    gpu = L.Cavity(case.nx, case.ny, Ra=case.Ra, Pr=case.Pr, Ma=case.Ma, store=store, wall_bc="fd")
    orc = oracle.Oracle.from_groups(case.nx, case.ny, case.Ra, case.Pr, case.Ma, wall_bc="fd")
    assert L.lbmfvm_kernel_info(gpu.h)[0] == L.LBMFVM_KERNEL_GENERIC
    gpu.step(case.steps)
    orc.step(case.steps)
    du, dT = deviation(gpu, orc)
    assert du <= TOL[store] and dT <= TOL[store], (du, dT)


@pytest.mark.parametrize("store", ["f64", "f32"])
@pytest.mark.parametrize("tile_y", [4, 16])
def test_ragged_grid_with_obstacles_matches_oracle(store, tile_y):
    nx, ny = 77, 45
    m = obstacle_mask(nx, ny)
    gpu = L.Cavity(nx, ny, Ra=1e5, Pr=0.71, Ma=MA, store=store, mask=m, wall_bc="fd", tile_y=tile_y)
    orc = oracle.Oracle.from_groups(nx, ny, 1e5, 0.71, MA, mask=m, wall_bc="fd")
    gpu.step(1500)
    orc.step(1500)
    du, dT = deviation(gpu, orc)
    assert du <= TOL[store] and dT <= TOL[store], (du, dT)


@pytest.mark.parametrize("store", ["f64", "f32"])
def test_lid_driven_cavity_and_channel_match_oracle(store):
    tol = TOL[store]
    bc = (L.LBMFVM_BC_DIRICHLET, L.LBMFVM_BC_DIRICHLET, L.LBMFVM_BC_ADIABATIC, L.LBMFVM_BC_MOVING)
    kw = dict(nu=0.05, alpha=0.07, gbeta=2e-4, u_lid=0.05)
    gpu = L.Cavity(50, 41, store=store, bc=bc, wall_bc="fd", **kw)
    orc = oracle.Oracle(50, 41, bc=bc, wall_bc="fd", **kw)
    gpu.step(900)
    orc.step(900)
    du, dT = deviation(gpu, orc, 0.05)
    assert du <= tol and dT <= tol, (du, dT)
    # force-driven channel: periodic along x, the walls' strain from the
    # parabolic profile
    per = (L.LBMFVM_BC_PERIODIC, L.LBMFVM_BC_PERIODIC, L.LBMFVM_BC_ADIABATIC, L.LBMFVM_BC_ADIABATIC)
    H, nu, umax = 32, 0.1, 0.01
    fx = 8 * nu * umax / (H * H)
    gpu = L.Cavity(8, H + 1, store=store, bc=per, nu=nu, alpha=0.1, gbeta=0.0, force=(fx, 0.0), wall_bc="fd")
    orc = oracle.Oracle(8, H + 1, bc=per, nu=nu, alpha=0.1, gbeta=0.0, fx=fx, wall_bc="fd")
    gpu.step(3000)
    orc.step(3000)
    du, _ = deviation(gpu, orc, umax)
    assert du <= 10 * tol, du


def test_options_that_need_other_kernels_are_refused():
    with pytest.raises(L.LbmfvmError) as e:
        L.Cavity(40, 40, Ra=1e4, Pr=0.71, Ma=MA, wall_bc="fd", kernel="tma")
    assert e.value.code == L.LBMFVM_ERR_ARG
    with pytest.raises(L.LbmfvmError) as e:
        L.Cavity(40, 40, Ra=1e4, Pr=0.71, Ma=MA, wall_bc="fd", energy="lbm")
    assert e.value.code == L.LBMFVM_ERR_ARG
