"""Batches: many cavities in one persistent launch per step (GPU).

A cavity in a batch runs the same kernel and tile decomposition as a
single-cavity handle, so its fields equal the single run bit for bit; the
FP64 oracle checks a few cavities directly."""

import math

import numpy as np
import pytest

import oracle
import paper_1908_08386_gb300 as L
from paper_1908_08386_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

MA = 0.1 * math.sqrt(3.0)


def small_cases():
    """Uneven cavities: sizes that are and are not tile multiples, aspect 2,
    obstacles, different Ra and Pr."""
    cases = [
        WL.CavityCase(64, 64, 1e4, 0.71, MA, name="a"),
        WL.CavityCase(97, 49, 3e4, 7.0, MA, name="b"),
        WL.CavityCase(129, 65, 1e5, 0.71, MA, name="c"),
        WL.CavityCase(40, 40, 2e3, 0.71, 0.05 * math.sqrt(3.0), name="d"),
        WL.CavityCase(150, 72, 1e5, 0.71, MA, name="e"),
    ]
    cases[2].mask = WL.rasterize([("circle", 60.0, 30.0, 14.0)], 129, 65)
    cases[4].mask = WL.rasterize([("rect", 40.0, 36.0, 12.0, 20.0), ("circle", 110.0, 30.0, 10.0)], 150, 72)
    return cases


@pytest.mark.parametrize("store", ["f32", "f16"])
def test_batch_equals_single_cavity_runs_bitwise(store):
    cases = small_cases()
    b = L.Batch(cases, store=store)
    b.step(300)
    for i, c in enumerate(cases):
        single = L.Cavity(c.nx, c.ny, Ra=c.Ra, Pr=c.Pr, Ma=c.Ma, mask=c.mask, store=store, kernel="tma")
        single.step(300)
        got = np.stack(b.fields(i))
        want = np.stack(single.fields())
        assert np.array_equal(got, want), (c.name, np.abs(got - want).max())
        assert b.info(i)[0] == 300


def test_batch_cavities_match_the_oracle():
    cases = small_cases()
    b = L.Batch(cases, store="f32")
    b.step(800)
    for i in (1, 2, 4):
        c = cases[i]
        o = oracle.Oracle.from_groups(c.nx, c.ny, c.Ra, c.Pr, c.Ma, mask=c.mask)
        o.step(800)
        _, ug, vg, Tg = b.fields(i)
        _, uo, vo, To = o.fields()
        u_scale = c.Ma / math.sqrt(3.0)
        assert max(np.abs(ug - uo).max(), np.abs(vg - vo).max()) / u_scale <= 1e-5
        assert np.abs(Tg - To).max() <= 1e-5
        nh_g, loc_g, nc_g = b.nusselt(i)
        nh_o, loc_o, nc_o, _ = o.nusselt()
        assert abs(nh_g - nh_o) <= 1e-4 * abs(nh_o) and abs(nc_g - nc_o) <= 1e-4 * abs(nc_o)


def test_batch_residuals_match_single_handles():
    cases = small_cases()[:3]
    b = L.Batch(cases, store="f32")
    singles = [L.Cavity(c.nx, c.ny, Ra=c.Ra, Pr=c.Pr, Ma=c.Ma, mask=c.mask, store="f32", kernel="tma") for c in cases]
    for _ in range(2):
        b.step(500)
        rb = b.residuals()
        for s, r in zip(singles, rb):
            s.step(500)
            assert r == pytest.approx(s.residual(), rel=1e-12)


def test_converged_cavities_leave_the_launch_and_keep_their_state():
    # a tiny conductive cavity converges long before a convective one
    cases = [WL.CavityCase(24, 24, 1e3, 0.71, MA, name="fast"),
             WL.CavityCase(96, 96, 1e5, 0.71, MA, name="slow")]
    b = L.Batch(cases, store="f32")
    steps, r = b.run(tol=1e-6, check_every=500, max_steps=20000)
    assert r[0] < 1e-6 and not b.info(0)[1]
    assert steps[0] < steps[1] or r[1] >= 1e-6
    frozen = np.stack(b.fields(0))
    b.step(1000)  # only the slow cavity, if still active, moves
    assert np.array_equal(np.stack(b.fields(0)), frozen)
    assert b.info(0)[0] == steps[0]


def test_set_state_resets_one_cavity_only():
    cases = small_cases()[:2]
    b = L.Batch(cases, store="f32")
    b.step(200)
    other = np.stack(b.fields(1))
    rng = np.random.default_rng(3)
    T0 = rng.random((cases[0].ny, cases[0].nx)).astype(np.float32)
    b.set_state(0, T=T0)
    assert b.info(0)[0] == 0 and b.info(1)[0] == 200
    assert np.array_equal(np.stack(b.fields(1)), other)
    # the reset cavity now follows a fresh single run from the same state
    single = L.Cavity(cases[0].nx, cases[0].ny, Ra=cases[0].Ra, Pr=cases[0].Pr, Ma=cases[0].Ma, store="f32",
                      kernel="tma")
    single.set_state(T=T0)
    b.step(100)
    single.step(100)
    assert np.array_equal(np.stack(b.fields(0)), np.stack(single.fields()))


def test_fp64_batch_matches_the_oracle_to_rounding():
    cases = small_cases()
    b = L.Batch(cases, store="f64")
    b.step(600)
    for i in (0, 2, 4):
        c = cases[i]
        o = oracle.Oracle.from_groups(c.nx, c.ny, c.Ra, c.Pr, c.Ma, mask=c.mask)
        o.step(600)
        _, ug, vg, Tg = b.fields(i)
        _, uo, vo, To = o.fields()
        assert max(np.abs(ug - uo).max(), np.abs(vg - vo).max()) / (c.Ma / math.sqrt(3.0)) <= 1e-10
        assert np.abs(Tg - To).max() <= 1e-10


def test_batch_rejects_what_it_cannot_run():
    c = WL.CavityCase(64, 64, 1e4, 0.71, MA)
    with pytest.raises(L.LbmfvmError) as e:
        L.Batch([c], store=7)
    assert e.value.code == L.LBMFVM_ERR_ARG
    bad = WL.CavityCase(512, 512, 1e3, 0.71, MA)  # alpha above the explicit limit
    with pytest.raises(L.LbmfvmError) as e:
        L.Batch([c, bad])
    assert e.value.code == L.LBMFVM_ERR_UNSTABLE


def test_autotuned_shapes_change_no_result():
    # the autotuner picks a shape per precision and size class; every shape
    # computes the same arithmetic per node
    case = WL.CavityCase(150, 72, 1e5, 0.71, MA)
    fixed = L.Cavity(case.nx, case.ny, Ra=case.Ra, Pr=case.Pr, Ma=case.Ma, store="f32", kernel="tma", tma_config=1)
    tuned = L.Cavity(case.nx, case.ny, Ra=case.Ra, Pr=case.Pr, Ma=case.Ma, store="f32", kernel="tma",
                     tma_config="auto")
    again = L.Cavity(case.nx, case.ny, Ra=case.Ra, Pr=case.Pr, Ma=case.Ma, store="f32", kernel="tma",
                     tma_config="auto")
    assert 0 <= tuned.tma_config <= 5 and again.tma_config == tuned.tma_config  # remembered per class
    for c in (fixed, tuned):
        c.step(300)
    assert np.array_equal(np.stack(tuned.fields()), np.stack(fixed.fields()))
    b = L.Batch(small_cases(), store="f16")  # autotuned by default
    assert 0 <= b.tma_config("f16") <= 5 and b.tma_config("f32") == -1  # upper levels not created yet


def test_default_shape_spreads_small_grids_over_more_sms():
    """The default tile shape: for a grid with fewer tiles than SMs the
    smaller tiles (64 x 8, two blocks per SM, at 32 and 16 bits; 32 x 8 with
    ring warps at 64 bits), else 64 x 16 with ring warps (two halo rows while
    the state fits in the L2) or 32 x 8, two blocks per SM, at 64 bits."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    for n, store in ((64, "f32"), (128, "f16"), (1024, "f32"), (128, "f32x2"), (1024, "f32x2")):
        # Ra 1e5 at the small sides and 1e7 at 1024 keep alpha below the explicit limit
        cav = L.Cavity(n, n, Ra=1e5 if n < 1024 else 1e7, Pr=0.71, Ma=MA, store=store)
        if store == "f32x2":
            want = 4 if ((n + 31) // 32) * ((n + 7) // 8) < sms else 3
        elif ((n + 63) // 64) * ((n + 15) // 16) < sms:
            want = 2
        else:
            per_node = 2 * (9 * (4 if store == "f32" else 2) + 4)
            want = 4 if per_node * n * n <= l2 else 5
        assert cav.tma_config == want, (n, store, cav.tma_config)
        cav.close()


def test_level_shape_follows_the_active_set_and_changes_no_result():
    """Once the conductive cavities have converged and left, the convective
    one alone fills fewer tiles than the GPU has SMs: its level takes the
    small-grid shape (64 x 8, two blocks per SM) and stays bitwise equal to
    the same batch pinned to one shape."""
    cap = lambda n, Ra, Pr: min(0.1, 0.2 * math.sqrt(Ra * Pr) / (n - 1)) * math.sqrt(3.0)
    cases = [WL.CavityCase(160, 160, 1e3, 0.71, cap(160, 1e3, 0.71), name=f"conduction{k}") for k in range(4)]
    cases.append(WL.CavityCase(256, 256, 1e6, 0.71, MA, name="convection"))
    auto = L.Batch(cases, store="f32", tma_config="default")
    pinned = L.Batch(cases, store="f32", tma_config=1)
    active = None
    for _ in range(40):
        auto.run(tol=1e-5, check_every=500, max_steps=10000)
        pinned.run(tol=1e-5, check_every=500, max_steps=10000)
        active = [auto.info(i)[1] for i in range(len(cases))]
        if not any(active[:4]) or not active[4]:
            break
    assert not any(active[:4]) and active[4], active
    assert auto.tma_config("f32") == 2 and pinned.tma_config("f32") == 1
    for i in range(len(cases)):
        assert np.array_equal(np.stack(auto.fields(i)), np.stack(pinned.fields(i))), cases[i].name
        assert auto.info(i)[0] == pinned.info(i)[0]
