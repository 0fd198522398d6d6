"""GPU path (through the C-ABI) against the FP64 CPU oracle, element by element.

Tolerances: FP64 storage agrees with the oracle to rounding (1e-9 after
thousands of steps); FP32 storage within max|du|/U0 <= 1e-5 and
max|dT| <= 1e-5 after the same step count; FP16/BF16 storage within 0.5 % of
the steady Nusselt number and max|dT| <= 1e-3.
"""

import math

import numpy as np
import pytest

import oracle
import paper_1908_08386_gb300 as L
from paper_1908_08386_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

U0 = 0.1
MA = U0 * math.sqrt(3.0)


def pair(nx, ny, *, Ra=None, Pr=0.71, Ma=MA, store="f32", tile_y=0, mask=None, kernel="auto", **kw):
    """The same case on the GPU (Cavity) and on the oracle."""
    if Ra is not None:
        gpu = L.Cavity(nx, ny, Ra=Ra, Pr=Pr, Ma=Ma, store=store, tile_y=tile_y, mask=mask, kernel=kernel, **kw)
        orc = oracle.Oracle.from_groups(nx, ny, Ra, Pr, Ma, mask=mask, **kw)
    else:
        lat = {k: kw.pop(k) for k in ("nu", "alpha", "gbeta") if k in kw}
        force = kw.pop("force", None)
        gpu = L.Cavity(nx, ny, store=store, tile_y=tile_y, mask=mask, force=force, kernel=kernel, **lat, **kw)
        fx, fy = force if force is not None else (0.0, 0.0)
        orc = oracle.Oracle(nx, ny, mask=mask, fx=fx, fy=fy, **lat, **kw)
    return gpu, orc


def compare(gpu, orc, u_scale=U0):
    rg, ug, vg, Tg = gpu.fields()
    ro, uo, vo, To = orc.fields()
    return dict(
        du=max(np.abs(ug - uo).max(), np.abs(vg - vo).max()) / u_scale,
        dT=np.abs(Tg - To).max(),
        drho=np.abs(rg - ro).max(),
    )


@pytest.mark.parametrize("store", ["f64", "f32x2"])
def test_config_small_f64_matches_oracle(store):
    # config 1 (64^2, Ra 1e3, 10^4 steps); double-single storage and
    # arithmetic reach FP64's agreement with the oracle
    case = WL.config_small()
    gpu, orc = pair(case.nx, case.ny, Ra=case.Ra, Pr=case.Pr, store=store)
    gpu.step(case.steps)
    orc.step(case.steps)
    d = compare(gpu, orc)
    assert d["du"] <= 1e-9 and d["dT"] <= 1e-9 and d["drho"] <= 1e-9, d


@pytest.mark.parametrize("kernel", ["tma", "generic"])
def test_config_small_f32_matches_oracle(kernel):
    case = WL.config_small()
    gpu, orc = pair(case.nx, case.ny, Ra=case.Ra, Pr=case.Pr, store="f32", kernel=kernel)
    gpu.step(case.steps)
    orc.step(case.steps)
    d = compare(gpu, orc)
    assert d["du"] <= 1e-5 and d["dT"] <= 1e-5, d
    nh_g, loc_g, nc_g = gpu.nusselt()
    nh_o, loc_o, nc_o, _ = orc.nusselt()
    assert abs(nh_g - nh_o) <= 1e-4 * abs(nh_o) and abs(nc_g - nc_o) <= 1e-4 * abs(nc_o)


def obstacle_mask(nx, ny):
    return WL.rasterize([("rect", 0.3 * nx, 0.35 * ny, 0.15 * nx, 0.2 * ny),
                         ("circle", 0.68 * nx, 0.6 * ny, 0.22 * ny)], nx, ny)


@pytest.mark.parametrize("store,tol,kernel", [("f64", 1e-9, "generic"), ("f64", 1e-9, "tma"),
                                              ("f32x2", 1e-9, "generic"), ("f32x2", 1e-9, "tma"),
                                              ("f32", 1e-5, "generic"), ("f32", 1e-5, "tma")])
@pytest.mark.parametrize("tile_y", [4, 8, 16])
def test_ragged_grid_with_obstacles(store, tol, kernel, tile_y):
    nx, ny = 77, 45  # ragged in both directions for every tile shape
    mask = obstacle_mask(nx, ny)
    gpu, orc = pair(nx, ny, Ra=1e5, store=store, tile_y=tile_y, mask=mask, kernel=kernel)
    gpu.step(1500)
    orc.step(1500)
    d = compare(gpu, orc)
    assert d["du"] <= tol and d["dT"] <= tol, d


@pytest.mark.parametrize("kernel", ["tma"])
@pytest.mark.parametrize("cfg", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("store", ["f64", "f32x2", "f32", "f16", "bf16"])
@pytest.mark.parametrize("shape", [(130, 67), (64, 16), (200, 150), (31, 97)])
def test_tma_kernels_agree_with_generic(store, shape, cfg, kernel):
    """The TMA-staged kernels (every shape index) and the global-gather kernel
    compute the same arithmetic; across aligned and ragged grids with
    obstacles crossing tile borders their fields agree to
    the last few rounding steps."""
    nx, ny = shape
    out = {}
    for k in (kernel, "generic"):
        g = L.Cavity(nx, ny, Ra=1e5, Pr=0.71, Ma=MA, store=store, kernel=k, tma_config=cfg,
                     mask=obstacle_mask(nx, ny))
        g.step(500)
        out[k] = np.stack(g.fields())
    d = np.abs(out[kernel] - out["generic"])
    # FP32 storage: a few rounding steps.  16-bit storage re-quantises every
    # step, so one differently contracted FMA grows into storage-level noise;
    # an indexing error would still show up at the scale of U0 and of dT = 1.
    tol_u, tol_T = {"f64": (1e-12 * U0, 1e-12), "f32x2": (1e-11 * U0, 1e-11),
                    "f32": (1e-6 * U0, 1e-6)}.get(store, (2e-3 * U0, 2e-3))
    assert d[1:3].max() <= tol_u and d[3].max() <= tol_T, d.reshape(4, -1).max(axis=1)


def test_bounded_wait_reports_timeout_and_context_survives():
    kernel = "tma"
    case = WL.config_small()
    gpu, orc = pair(case.nx, case.ny, Ra=case.Ra, Pr=case.Pr, store="f32", kernel=kernel)
    L.lbmfvm_inject_stall(gpu.h)
    gpu.step(1)
    with pytest.raises(L.LbmfvmError) as e:
        gpu.residual()
    assert e.value.code == L.LBMFVM_ERR_TIMEOUT
    # the context is still usable: restart and match the oracle again
    gpu.set_state()
    gpu.step(500)
    orc.step(500)
    d = compare(gpu, orc)
    assert d["du"] <= 1e-5 and d["dT"] <= 1e-5, d


def test_inject_stall_needs_the_tma_kernel():
    g = L.Cavity(40, 40, Ra=1e4, Pr=0.71, Ma=MA, store="f64", kernel="generic")
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_inject_stall(g.h)
    assert e.value.code == L.LBMFVM_ERR_ARG


def test_tile_shapes_agree_bitwise():
    nx, ny = 130, 67
    outs = []
    for ty in (4, 8, 16):
        g = L.Cavity(nx, ny, Ra=1e5, Pr=0.71, Ma=MA, store="f32", tile_y=ty, kernel="generic",
                     mask=obstacle_mask(nx, ny))
        g.step(300)
        outs.append(np.stack(g.fields()))
    assert (outs[0] == outs[1]).all() and (outs[0] == outs[2]).all()


@pytest.mark.parametrize("store,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_periodic_channel_with_body_force(store, tol):
    H, nu, umax = 16, 0.1, 0.01
    g = 8 * nu * umax / H**2
    bc = (WL.PERIODIC, WL.PERIODIC, WL.ADIABATIC, WL.ADIABATIC)
    gpu, orc = pair(37, H + 1, store=store, bc=bc, nu=nu, alpha=0.1, gbeta=0.0, force=(g, 0.0))
    gpu.step(3000)
    orc.step(3000)
    d = compare(gpu, orc, u_scale=umax)
    assert d["du"] <= tol, d


@pytest.mark.parametrize("store,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_lid_driven_cavity(store, tol):
    n, u_lid = 50, 0.05
    bc = (WL.ADIABATIC, WL.ADIABATIC, WL.ADIABATIC, WL.MOVING)
    gpu, orc = pair(n, n, store=store, bc=bc, u_lid=u_lid, nu=u_lid * (n - 1) / 100, alpha=0.1, gbeta=0.0)
    gpu.step(2000)
    orc.step(2000)
    d = compare(gpu, orc, u_scale=u_lid)
    assert d["du"] <= tol, d


@pytest.mark.parametrize("store,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_periodic_box_with_buoyancy(store, tol):
    nx, ny = 45, 33
    T0 = WL.random_temperature(ny, nx, seed=11)
    bc = (WL.PERIODIC,) * 4
    gpu, orc = pair(nx, ny, store=store, bc=bc, nu=0.05, alpha=0.15, gbeta=1e-4, t_ref=0.5)
    gpu.set_state(T=T0.astype(np.float32))
    orc.set_state(T=T0.astype(np.float32).astype(np.float64))
    gpu.step(800)
    orc.step(800)
    d = compare(gpu, orc, u_scale=1e-3)
    assert d["du"] <= tol * 10 and d["dT"] <= tol, d


def test_set_state_round_trip_and_step_zero():
    nx, ny = 61, 40
    u, v = WL.random_velocity(ny, nx, seed=5, amp=0.02)
    T = WL.random_temperature(ny, nx, seed=6)
    u, v, T = (a.astype(np.float32) for a in (u, v, T))
    gpu, orc = pair(nx, ny, Ra=1e5, store="f64")
    gpu.set_state(u, v, T)
    orc.set_state(u.astype(np.float64), v.astype(np.float64), T.astype(np.float64))
    assert gpu.steps == 0
    d = compare(gpu, orc)
    assert d["du"] <= 1e-12 and d["dT"] == 0.0 and d["drho"] <= 1e-12, d
    gpu.step(7)
    orc.step(7)
    d = compare(gpu, orc)
    assert d["du"] <= 1e-12 and d["dT"] <= 1e-12, d


def test_nusselt_and_residual_match_oracle():
    case = WL.config_small()
    gpu, orc = pair(case.nx, case.ny, Ra=case.Ra, Pr=case.Pr, store="f64")
    for _ in range(3):
        gpu.step(1000)
        orc.step(1000)
        rg, ro = gpu.residual(), orc.residual()
        assert rg == pytest.approx(ro, rel=1e-8)
    nh_g, loc_g, nc_g = gpu.nusselt()
    nh_o, loc_o, nc_o, _ = orc.nusselt()
    assert nh_g == pytest.approx(nh_o, rel=1e-10) and nc_g == pytest.approx(nc_o, rel=1e-10)
    assert np.abs(loc_g - loc_o).max() <= 1e-9


def test_pure_conduction_is_exact_on_gpu():
    H = 32
    gpu = L.Cavity(H + 1, H + 1, store="f64", nu=0.1, alpha=0.24, gbeta=0.0)
    gpu.step(20000)
    _, u, v, T = gpu.fields()
    x = np.arange(H + 1) / H
    assert np.abs(T - (1 - x)[None, :]).max() <= 1e-12
    assert np.all(u == 0.0) and np.all(v == 0.0)
    nh, _, nc = gpu.nusselt()
    assert abs(nh - 1) <= 1e-11 and abs(nc - 1) <= 1e-11


@pytest.mark.parametrize("store", ["f32", "f64"])
def test_full_size_cavity_sampled_against_oracle(store):
    """1024^2, Ra = 1e6 (the benchmarked workload, default launch shape):
    from the same random state, both sides take 3 steps; every node compared."""
    case = WL.config_large()
    n = case.nx
    u, v = WL.random_velocity(n, n, seed=21, amp=0.01)
    T = WL.random_temperature(n, n, seed=22)
    u, v, T = (a.astype(np.float32) for a in (u, v, T))
    gpu, orc = pair(n, n, Ra=case.Ra, Pr=case.Pr, store=store)
    gpu.set_state(u, v, T)
    orc.set_state(u.astype(np.float64), v.astype(np.float64), T.astype(np.float64))
    gpu.step(3)
    orc.step(3)
    d = compare(gpu, orc)
    tol = 1e-12 if store == "f64" else 1e-6
    assert d["du"] <= tol and d["dT"] <= tol, d


def test_full_size_cavity_over_graph_replays_against_oracle():
    """1024^2 in FP64 over 131 steps (two 64-step graph replays and three
    single launches): enough tiles that the last rounds of each launch are
    drawn from the shared tile counter, through both counter parities."""
    case = WL.config_large()
    n = case.nx
    u, v = WL.random_velocity(n, n, seed=23, amp=0.01)
    T = WL.random_temperature(n, n, seed=24)
    gpu, orc = pair(n, n, Ra=case.Ra, Pr=case.Pr, store="f64")
    gpu.set_state(u.astype(np.float32), v.astype(np.float32), T.astype(np.float32))
    orc.set_state(u.astype(np.float32).astype(np.float64), v.astype(np.float32).astype(np.float64),
                  T.astype(np.float32).astype(np.float64))
    gpu.step(1)
    gpu.step(130)
    orc.step(131)
    d = compare(gpu, orc)
    assert d["du"] <= 1e-12 and d["dT"] <= 1e-12, d


@pytest.mark.parametrize("kernel", ["tma", "generic"])
@pytest.mark.parametrize("store", ["f16", "bf16"])
def test_reduced_precision_steady_nusselt(store, kernel):
    case = WL.config_small()
    gpu, orc = pair(case.nx, case.ny, Ra=case.Ra, Pr=case.Pr, store=store, kernel=kernel)
    steps = 40000
    gpu.step(steps)
    orc.step(steps)
    nh_g, _, _ = gpu.nusselt()
    nh_o, _, _, _ = orc.nusselt()
    assert abs(nh_g - nh_o) <= 0.005 * nh_o, (nh_g, nh_o)
    d = compare(gpu, orc)
    assert d["dT"] <= 1e-3, d


def test_smallest_grid_and_zero_steps():
    gpu, orc = pair(3, 3, store="f64", nu=0.1, alpha=0.2, gbeta=0.01)
    for kernel in ("tma",):
        tiny, orc2 = pair(3, 3, store="f32", kernel=kernel, nu=0.1, alpha=0.2, gbeta=0.01)
        tiny.step(50)
        orc2.step(50)
        d = compare(tiny, orc2)
        assert d["du"] <= 1e-6 and d["dT"] <= 1e-6
    gpu.step(0)
    assert gpu.steps == 0
    gpu.step(50)
    orc.step(50)
    d = compare(gpu, orc)
    assert d["du"] <= 1e-12 and d["dT"] <= 1e-12
    assert gpu.steps == 50


def test_long_runs_use_graph_and_keep_parity():
    # 64-step graph replays plus single launches, starting on odd parity
    case = WL.config_small()
    gpu, orc = pair(case.nx, case.ny, Ra=case.Ra, Pr=case.Pr, store="f64")
    for n in (1, 130, 64, 3, 200):
        gpu.step(n)
        orc.step(n)
    assert gpu.steps == 398
    d = compare(gpu, orc)
    assert d["du"] <= 1e-10 and d["dT"] <= 1e-10


def test_run_to_steady_reaches_tolerance():
    gpu = L.Cavity(33, 33, Ra=1e3, Pr=0.71, Ma=MA, store="f64")
    steps, r = gpu.run_to_steady(tol=1e-9, check_every=500, max_steps=200000)
    assert r < 1e-9 and steps % 500 == 0 and steps < 200000


def test_launch_count_follows_the_steps():
    g = L.Cavity(70, 48, Ra=1e4, Pr=0.71, Ma=MA, store="f32", kernel="tma")
    n0 = L.lbmfvm_launch_count(g.h)
    g.step(1)
    g.step(130)  # single launches and one graph replay of 64
    assert L.lbmfvm_launch_count(g.h) - n0 == 131
