"""The D2Q5 thermal lattice-Boltzmann energy solver (Section 2.4, the paper's
pure-LBM comparison) on the GPU against the FP64 oracle, element by element:
FP64 and double-single storage to rounding (1e-9), FP32 within max|du|/U0 and
max|dT| of 1e-5 after the same step count; on the small benchmark cavity,
ragged grids with obstacles, a lid-driven cavity and a periodic box; the
steady Nusselt number; checkpoints."""

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
    gpu = L.Cavity(case.nx, case.ny, Ra=case.Ra, Pr=case.Pr, Ma=case.Ma, store=store, energy="lbm")
    orc = oracle.Oracle.from_groups(case.nx, case.ny, case.Ra, case.Pr, case.Ma, energy="lbm")
    gpu.step(case.steps)
    orc.step(case.steps)
    du, dT = deviation(gpu, orc)
    assert du <= TOL[store] and dT <= TOL[store], (du, dT)
    nh_g, _, nc_g = gpu.nusselt()
    nh_o, _, nc_o, _ = orc.nusselt()
    assert abs(nh_g - nh_o) <= 10 * TOL[store] * abs(nh_o)


@pytest.mark.parametrize("store", ["f64", "f32x2", "f32"])
@pytest.mark.parametrize("shape", [(77, 45), (130, 67)])
def test_ragged_grid_with_obstacles_matches_oracle(store, shape):
    nx, ny = shape
    m = obstacle_mask(nx, ny)
    gpu = L.Cavity(nx, ny, Ra=1e5, Pr=0.71, Ma=MA, store=store, mask=m, energy="lbm")
    orc = oracle.Oracle.from_groups(nx, ny, 1e5, 0.71, MA, mask=m, energy="lbm")
    gpu.step(1500)
    orc.step(1500)
    du, dT = deviation(gpu, orc)
    assert du <= TOL[store] and dT <= TOL[store], (du, dT)


@pytest.mark.parametrize("store", ["f64", "f32"])
def test_lid_driven_and_periodic_boxes_match_oracle(store):
    tol = TOL[store]
    # moving lid over a heated cavity: wall velocities enter g_eq at the walls
    bc = (L.LBMFVM_BC_DIRICHLET, L.LBMFVM_BC_DIRICHLET, L.LBMFVM_BC_ADIABATIC, L.LBMFVM_BC_MOVING)
    kw = dict(nu=0.05, alpha=0.07, gbeta=2e-4, u_lid=0.05)
    gpu = L.Cavity(50, 41, store=store, bc=bc, energy="lbm", **kw)
    orc = oracle.Oracle(50, 41, bc=bc, energy="lbm", **kw)
    gpu.step(900)
    orc.step(900)
    du, dT = deviation(gpu, orc, 0.05)
    assert du <= tol and dT <= tol, (du, dT)
    # periodic box from a random temperature field (the pulls wrap)
    per = (L.LBMFVM_BC_PERIODIC,) * 4
    # the C-ABI takes FP32 fields: give the oracle the same rounded values
    T0 = WL.random_temperature(33, 40, seed=5).astype(np.float32).astype(np.float64)
    gpu = L.Cavity(40, 33, store=store, bc=per, nu=0.08, alpha=0.1, gbeta=2e-4, t_ref=0.5, energy="lbm")
    orc = oracle.Oracle(40, 33, bc=per, nu=0.08, alpha=0.1, gbeta=2e-4, t_ref=0.5, energy="lbm")
    gpu.set_state(T=T0)
    orc.set_state(T=T0)
    gpu.step(300)
    orc.step(300)
    du, dT = deviation(gpu, orc, 1e-4)
    assert du <= 10 * tol and dT <= tol, (du, dT)


def test_steady_nusselt_matches_oracle():
    """Ra = 1e4 on 41 x 41 nodes run to a 1e-8 residual in double-single
    storage: the steady hot-wall Nusselt number and T field equal the
    oracle's steady state."""
    n = 41
    gpu = L.Cavity(n, n, Ra=1e4, Pr=0.71, Ma=MA, store="f32x2", energy="lbm")
    steps, r = gpu.run_to_steady(tol=1e-8, check_every=1000, max_steps=400_000)
    assert r < 1e-8
    orc = oracle.Oracle.from_groups(n, n, 1e4, 0.71, MA, energy="lbm")
    for _ in range(400):
        orc.step(1000)
        if orc.residual() < 1e-9:
            break
    nh_g, _, _ = gpu.nusselt()
    nh_o, _, _, _ = orc.nusselt()
    assert abs(nh_g - nh_o) <= 1e-6 * abs(nh_o), (nh_g, nh_o)
    assert np.abs(gpu.fields()[3] - orc.fields()[3]).max() <= 1e-6


@pytest.mark.parametrize("store", ["f32", "f32x2"])
def test_checkpoint_round_trip_is_bitwise(tmp_path, store):
    path = tmp_path / "lbm.ckpt"
    mk = lambda: L.Cavity(70, 48, Ra=1e5, Pr=0.71, Ma=MA, store=store, mask=obstacle_mask(70, 48), energy="lbm")
    a = mk()
    a.step(257)
    a.save(path)
    a.step(300)
    want = np.stack(a.fields())
    b = mk()
    b.load(path)
    b.step(300)
    assert np.array_equal(np.stack(b.fields()), want)
    assert L.lbmfvm_checkpoint_info(path)["energy"] == L.LBMFVM_ENERGY_LBM_D2Q5
    c = L.Cavity(70, 48, Ra=1e5, Pr=0.71, Ma=MA, store=store, mask=obstacle_mask(70, 48))
    with pytest.raises(L.LbmfvmError) as e:
        c.load(path)
    assert e.value.code == L.LBMFVM_ERR_ARG
