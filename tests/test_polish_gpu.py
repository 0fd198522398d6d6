"""Precision ladder and mass renormalisation (GPU, through the C-ABI).

The rounding of the stored populations puts a floor under the steady-state
residual: about 1e-3 for 16-bit storage and 2e-7 for FP32 on these cavities.
A run meets the 1e-8 criterion by finishing in wider storage.  Copying a state
between precisions only converts values (every precision stores f - w_i), so
a copy within one precision leaves a run bit for bit unchanged, and a state
widened and narrowed again is the same state.

Mass renormalisation rescales the populations to a fluid mean rho of 1 after
each residual check.  The step is homogeneous of degree one in f (pinned on
the oracle by the homogeneous_in_f check), so u and T follow the oracle's
plain run while rho differs from it by one constant factor.
"""

import math

import numpy as np
import pytest

import oracle
import paper_1908_08386_gb300 as L
from paper_1908_08386_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

MA = 0.1 * math.sqrt(3.0)


def cavity(store, **kw):
    mask = WL.rasterize([("circle", 40.0, 20.0, 9.0)], 70, 48)
    return L.Cavity(70, 48, Ra=1e4, Pr=0.71, Ma=MA, mask=mask, store=store, kernel="tma", **kw)


@pytest.mark.parametrize("store", ["f32", "f64", "f32x2"])
@pytest.mark.parametrize("first", [1, 130])  # opposite parities; graph replays
def test_copy_state_within_one_precision_is_exact(store, first):
    a = cavity(store)
    a.step(first)
    b = cavity(store)
    b.copy_state_from(a)
    assert b.steps == a.steps == first
    assert np.array_equal(np.stack(b.fields()), np.stack(a.fields()))
    a.step(257)
    b.step(257)
    assert np.array_equal(np.stack(b.fields()), np.stack(a.fields()))
    assert b.residual() == a.residual()  # the residual snapshot came along


@pytest.mark.parametrize("narrow,wide", [("f16", "f32"), ("bf16", "f32"), ("f32", "f64"), ("f16", "f64"),
                                         ("f32", "f32x2"), ("bf16", "f32x2")])
def test_widening_a_state_keeps_it(narrow, wide):
    a = cavity(narrow)
    a.step(501)
    b = cavity(wide)
    b.step(3)  # b's own state is overwritten entirely
    b.copy_state_from(a)
    assert b.steps == 501
    fa, fb = np.stack(a.fields()), np.stack(b.fields())
    if wide == "f32":  # both export in FP32 arithmetic
        assert np.array_equal(fb, fa)
    else:  # the same stored values, moments taken in FP64 or double-single
        assert np.abs(fb - fa).max() <= 1e-6
    # narrowed again, the widened values give back the same stored values
    c = cavity(narrow)
    c.copy_state_from(b)
    assert np.array_equal(np.stack(c.fields()), fa)


def test_copy_state_checks_its_arguments():
    a = cavity("f32")
    other = L.Cavity(64, 48, Ra=1e4, Pr=0.71, Ma=MA, store="f32")
    with pytest.raises(L.LbmfvmError) as e:
        other.copy_state_from(a)
    assert e.value.code == L.LBMFVM_ERR_ARG
    with pytest.raises(L.LbmfvmError) as e:
        a.copy_state_from(a)
    assert e.value.code == L.LBMFVM_ERR_ARG


def small_cases():
    cases = [WL.CavityCase(40, 40, 2e3, 0.71, MA, name="square"),
             WL.CavityCase(64, 33, 5e3, 7.0, MA, name="aspect 2"),
             WL.CavityCase(56, 56, 1e4, 0.71, MA, name="obstacle")]
    cases[2].mask = WL.rasterize([("circle", 30.0, 26.0, 8.0)], 56, 56)
    return cases


def oracle_steady(c, tol=1e-8, check_every=1000, max_steps=400000):
    o = oracle.Oracle.from_groups(c.nx, c.ny, c.Ra, c.Pr, c.Ma, mask=c.mask)
    o.residual()  # snapshot of the initial state
    for _ in range(max_steps // check_every):
        o.step(check_every)
        if o.residual() < tol:
            return o
    raise AssertionError(f"oracle did not reach {tol} for {c.name}")


def test_every_ladder_reaches_the_steady_criterion_and_the_oracle():
    cases = small_cases()
    runs = {}
    for store in ("f16", "bf16", "f32", "f64", "f32x2"):
        b = L.Batch(cases, store=store)
        assert all(b.precision(i) == store for i in range(len(cases)))
        steps, r = b.run(tol=1e-8, check_every=1000, max_steps=600000)
        assert (r < 1e-8).all(), (store, r)
        # the ladder ends in double-single storage (an FP64 batch stays FP64)
        top = "f64" if store == "f64" else "f32x2"
        assert all(b.precision(i) == top for i in range(len(cases))), store
        runs[store] = b
    for i, c in enumerate(cases):
        o = oracle_steady(c)
        nh_o, _, nc_o, _ = o.nusselt()
        _, _, _, To = o.fields()
        for store, b in runs.items():
            nh, _, nc = b.nusselt(i)
            _, _, _, Tg = b.fields(i)
            # the same FP64 steady state, up to the 1e-8 residual criterion
            assert abs(nh - nh_o) <= 1e-5 * abs(nh_o) and abs(nc - nc_o) <= 1e-5 * abs(nc_o), (c.name, store)
            assert np.abs(Tg - To).max() <= 1e-5, (c.name, store)


def test_without_the_ladder_fp16_stalls_above_the_criterion():
    cases = small_cases()[:1]
    b = L.Batch(cases, store="f16")
    b.set_polish("f16", 0)
    steps, r = b.run(tol=1e-8, check_every=1000, max_steps=100000)
    assert r[0] >= 1e-5 and b.precision(0) == "f16"
    # switched on again, the same batch finishes
    b.set_polish("f16", 2e-3, 16)
    steps, r = b.run(tol=1e-8, check_every=1000, max_steps=400000)
    assert r[0] < 1e-8 and b.precision(0) == "f32x2"


def test_a_floor_above_the_switch_value_moves_by_the_stall_rule():
    # FP32 switch value 1e-8 sits below the FP32 floor (about 2e-7); within a
    # factor 100 of it, 8 checks without halving move the cavity up
    cases = small_cases()[:1]
    b = L.Batch(cases, store="f32")
    b.set_polish("f32", 1e-8, 8)
    steps, r = b.run(tol=1e-8, check_every=1000, max_steps=400000)
    assert r[0] < 1e-8 and b.precision(0) == "f32x2"


def test_promoted_cavity_returns_to_its_storage_on_set_state():
    cases = small_cases()[:2]
    b = L.Batch(cases, store="f16")
    b.set_polish("f16", 2.0)  # promote at the first check (the first residual is 1)
    b.set_polish("f32", 0)
    b.run(tol=1e-12, check_every=500, max_steps=1000)
    assert b.precision(0) == "f32" and b.precision(1) == "f32"
    other = np.stack(b.fields(1))
    b.set_state(0)
    assert b.precision(0) == "f16" and b.info(0)[0] == 0
    assert np.array_equal(np.stack(b.fields(1)), other)
    fresh = L.Batch(cases[:1], store="f16")
    b.step(300)
    fresh.step(300)
    assert np.array_equal(np.stack(b.fields(0)), np.stack(fresh.fields(0)))


def test_polish_settings_are_checked():
    cases = small_cases()[:1]
    b64 = L.Batch(cases, store="f64")
    with pytest.raises(L.LbmfvmError) as e:
        b64.set_polish("f64", 1e-9)  # the top of the ladder
    assert e.value.code == L.LBMFVM_ERR_ARG
    b32 = L.Batch(cases, store="f32")
    b32.set_polish("f32", 0)
    with pytest.raises(L.LbmfvmError) as e:
        b32.set_polish("f16", 1e-3)  # not a level of an FP32 batch
    assert e.value.code == L.LBMFVM_ERR_ARG


@pytest.mark.parametrize("store", ["f64", "f32x2", "f32"])
def test_renormalised_run_keeps_the_oracle_velocity_and_temperature(store):
    c = small_cases()[2]
    gpu = L.Cavity(c.nx, c.ny, Ra=c.Ra, Pr=c.Pr, Ma=c.Ma, mask=c.mask, store=store)
    orc = oracle.Oracle.from_groups(c.nx, c.ny, c.Ra, c.Pr, c.Ma, mask=c.mask)
    steps, _ = gpu.run_to_steady(tol=0.0, check_every=1000, max_steps=3000)
    assert steps == 3000
    orc.step(3000)
    rg, ug, vg, Tg = gpu.fields()
    ro, uo, vo, To = orc.fields()
    wide = store in ("f64", "f32x2")
    tol = 1e-10 if wide else 1e-5
    assert max(np.abs(ug - uo).max(), np.abs(vg - vo).max()) / 0.1 <= tol
    assert np.abs(Tg - To).max() <= tol
    fluid = orc.classes()[0] == 0
    assert abs(rg[fluid].mean() - 1.0) <= (1e-12 if wide else 1e-6)
    ratio = rg[fluid] / ro[fluid]
    assert ratio.std() <= (1e-11 if wide else 1e-5) * ratio.mean()
    assert abs(ro[fluid].mean() - 1.0) > 1e-3  # the oracle's mass did drift
