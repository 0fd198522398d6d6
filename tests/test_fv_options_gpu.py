"""The energy update's options on the GPU against the FP64 oracle: QUICK face
values (fused into the step kernel) and m explicit sub-steps per lattice step
(velocity pass, sub-step passes, collision with the final temperature), on
ragged grids with obstacles crossing tile borders, single cavities and
batches.

Tolerances as for the central update: FP64 and double-single storage agree
with the oracle to rounding (1e-9), FP32 within max|du|/U0 and max|dT| of 1e-5
after the same step count.
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
TOL = {"f64": 1e-9, "f32x2": 1e-9, "f32": 1e-5}


def obstacle_mask(nx, ny):
    return WL.rasterize([("rect", 0.3 * nx, 0.35 * ny, 0.15 * nx, 0.2 * ny),
                         ("circle", 0.68 * nx, 0.6 * ny, 0.22 * ny)], nx, ny)


def deviation(gpu_fields, orc):
    _, ug, vg, Tg = gpu_fields
    _, uo, vo, To = orc.fields()
    return max(np.abs(ug - uo).max(), np.abs(vg - vo).max()) / U0, np.abs(Tg - To).max()


def run_pair(nx, ny, Ra, store, scheme, substeps, steps, mask=True):
    m = obstacle_mask(nx, ny) if mask else None
    gpu = L.Cavity(nx, ny, Ra=Ra, Pr=0.71, Ma=MA, store=store, mask=m, fv_scheme=scheme, fv_substeps=substeps)
    k = gpu.substeps
    orc = oracle.Oracle.from_groups(nx, ny, Ra, 0.71, MA, mask=m, fv_scheme=scheme, fv_substeps=k)
    gpu.step(steps)
    orc.step(steps)
    return gpu, orc, k


@pytest.mark.parametrize("store", ["f64", "f32x2", "f32"])
@pytest.mark.parametrize("shape", [(77, 45), (130, 67)])
def test_quick_fused_matches_oracle(store, shape):
    gpu, orc, k = run_pair(*shape, 1e5, store, "quick", 1, 1500)
    assert k == 1
    du, dT = deviation(gpu.fields(), orc)
    assert du <= TOL[store] and dT <= TOL[store], (du, dT)


@pytest.mark.parametrize("store", ["f64", "f32x2", "f32"])
@pytest.mark.parametrize("scheme,substeps,Ra", [("central", 3, 1e4), ("quick", 2, 1e5), ("central", 0, 300.0)])
def test_substeps_match_oracle(store, scheme, substeps, Ra):
    nx, ny = 77, 45
    gpu, orc, k = run_pair(nx, ny, Ra, store, scheme, substeps, 1200)
    if substeps == 0:
        # automatic: alpha = U0 H / sqrt(Ra Pr) = 0.30 needs two sub-steps
        assert k == 2
    du, dT = deviation(gpu.fields(), orc)
    assert du <= TOL[store] and dT <= TOL[store], (du, dT)


def test_substeps_take_the_explicit_limit_beyond_one_step():
    """alpha = 0.6 is beyond one explicit step's diffusion limit (1/4): one
    sub-step is refused, three match the oracle, and the run stays bounded."""
    nx, ny = 70, 41
    with pytest.raises(L.LbmfvmError) as e:
        L.Cavity(nx, ny, nu=0.05, alpha=0.6, gbeta=1e-5, store="f64")
    assert e.value.code == L.LBMFVM_ERR_UNSTABLE
    gpu = L.Cavity(nx, ny, nu=0.05, alpha=0.6, gbeta=1e-5, store="f64", fv_substeps=3,
                   mask=obstacle_mask(nx, ny))
    orc = oracle.Oracle(nx, ny, nu=0.05, alpha=0.6, gbeta=1e-5, mask=obstacle_mask(nx, ny), fv_substeps=3)
    gpu.step(800)
    orc.step(800)
    du, dT = deviation(gpu.fields(), orc)
    assert du <= 1e-9 and dT <= 1e-9, (du, dT)
    assert np.isfinite(gpu.fields()[3]).all()


@pytest.mark.parametrize("store", ["f64", "f32x2", "f32"])
def test_options_resume_bitwise_from_a_checkpoint(tmp_path, store):
    path = tmp_path / "q.ckpt"
    mk = lambda: L.Cavity(77, 45, Ra=1e4, Pr=0.71, Ma=MA, store=store, mask=obstacle_mask(77, 45),
                          fv_scheme="quick", fv_substeps=2)
    a = mk()
    a.step(301)
    a.save(path)
    a.step(200)
    want = np.stack(a.fields())
    b = mk()
    b.load(path)
    b.step(200)
    assert np.array_equal(np.stack(b.fields()), want)
    info = L.lbmfvm_checkpoint_info(path)
    assert (info["fv_scheme"], info["fv_substeps"]) == (L.LBMFVM_FV_QUICK, 2)
    c = L.Cavity(77, 45, Ra=1e4, Pr=0.71, Ma=MA, store=store, mask=obstacle_mask(77, 45), fv_scheme="quick",
                 fv_substeps=3)
    with pytest.raises(L.LbmfvmError) as e:
        c.load(path)
    assert e.value.code == L.LBMFVM_ERR_ARG


def batch_cases():
    """Uneven cavities, some of which need sub-steps at U0 = 0.1."""
    shapes = [(64, 64, 1e3, 0.71), (97, 49, 2e3, 7.0), (48, 48, 1e5, 0.71), (130, 67, 400.0, 0.71)]
    out = []
    for i, (nx, ny, Ra, Pr) in enumerate(shapes):
        m = obstacle_mask(nx, ny) if i % 2 else None
        out.append(WL.CavityCase(nx, ny, Ra, Pr, MA, 0, m, 0.5))
    return out


def test_batch_with_per_cavity_substeps_equals_single_runs():
    """Cavities with one energy update per step and cavities with several run
    in one batch (the fused launch and the sub-step launches side by side);
    each equals its own single-cavity run bit for bit and the oracle to FP32's
    tolerance."""
    cases = batch_cases()
    b = L.Batch(cases, store="f32", fv_substeps=0)
    ms = [b.substeps(i) for i in range(len(cases))]
    assert ms[0] > 1 and ms[2] == 1 and ms[3] > 1
    b.step(700)
    for i, c in enumerate(cases):
        single = L.Cavity(c.nx, c.ny, Ra=c.Ra, Pr=c.Pr, Ma=c.Ma, mask=c.mask, store="f32", fv_substeps=ms[i])
        single.step(700)
        got = np.stack(b.fields(i))
        assert np.array_equal(got, np.stack(single.fields())), i
        orc = oracle.Oracle.from_groups(c.nx, c.ny, c.Ra, c.Pr, c.Ma, mask=c.mask, fv_substeps=ms[i])
        orc.step(700)
        du, dT = deviation(got, orc)
        assert du <= 1e-5 and dT <= 1e-5, (i, du, dT)


def test_batch_substeps_reach_the_oracle_steady_state():
    """A batch whose cavities take different sub-steps climbs the precision
    ladder to a 1e-8 residual; each steady Nusselt number and temperature
    field matches the oracle's steady state."""
    cases = batch_cases()[:3]
    b = L.Batch(cases, store="f16", fv_substeps=0)
    steps, r = b.run(tol=1e-8, check_every=1000, max_steps=2_000_000)
    assert (r < 1e-8).all(), r
    for i, c in enumerate(cases):
        orc = oracle.Oracle.from_groups(c.nx, c.ny, c.Ra, c.Pr, c.Ma, mask=c.mask, fv_substeps=b.substeps(i))
        for _ in range(2000):
            orc.step(1000)
            if orc.residual() < 1e-9:
                break
        nu_o = orc.nusselt()[0]
        nu_g = b.nusselt(i)[0]
        assert abs(nu_g - nu_o) <= 1e-5 * abs(nu_o), (i, nu_g, nu_o)
        assert np.abs(b.fields(i)[3] - orc.fields()[3]).max() <= 1e-5
