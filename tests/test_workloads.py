"""The seeded input recipes (no GPU): the benchmark configurations, the uneven
cavity draw and the obstacle masks keep the sizes, parameter ranges and
stability conditions they promise, and the same seed gives the same inputs."""

import math

import numpy as np
import pytest

from paper_1908_08386_gb300 import workloads as WL


def test_configurations():
    c = WL.config_small()
    assert (c.nx, c.ny, c.Ra, c.Pr, c.steps, c.t_init) == (64, 64, 1e3, 0.71, 10_000, 0.5)
    assert math.isclose(c.Ma / math.sqrt(3.0), 0.1)  # U0 = 0.1 lattice units
    c = WL.config_large()
    assert (c.nx, c.ny, c.Ra, c.Pr, c.steps) == (1024, 1024, 1e6, 0.71, 100_000)
    assert WL.CAVITY_BC == (WL.DIRICHLET, WL.DIRICHLET, WL.ADIABATIC, WL.ADIABATIC)
    assert WL.CAVITY_T_WALL[:2] == (1.0, 0.0)


def test_same_seed_same_draw_other_seed_other_draw():
    a, b, c = WL.cavity_batch(12, 7), WL.cavity_batch(12, 7), WL.cavity_batch(12, 8)
    key = lambda cs: [(x.nx, x.ny, x.Ra, x.Pr, x.Ma, None if x.mask is None else x.mask.tobytes()) for x in cs]
    assert key(a) == key(b)
    assert key(a) != key(c)


@pytest.fixture(scope="module")
def draw():
    return WL.cavity_batch(256, 20190822)


def test_sides_aspect_and_parameter_ranges(draw):
    sizes = (64, 96, 128, 192, 256, 384, 512)
    for c in draw:
        assert c.ny in sizes
        a = (c.nx - 1) // (c.ny - 1)
        assert a in (1, 2) and c.nx == a * (c.ny - 1) + 1
        assert 1e3 <= c.Ra <= 1e6 and c.Pr in (0.71, 7.0)
        assert c.t_init == 0.5


def test_stability_conditions_of_the_explicit_update(draw):
    for c in draw:
        H = c.ny - 1
        U0 = c.Ma / math.sqrt(3.0)
        alpha = U0 * H / math.sqrt(c.Ra * c.Pr)
        nu = U0 * H * math.sqrt(c.Pr / c.Ra)
        assert U0 <= 0.1 + 1e-15 and alpha <= 0.2 + 1e-12 and U0 ** 2 < 2 * alpha
        tau = 3 * nu + 0.5
        assert tau >= 0.51 or c.ny == 512


def test_log_uniform_rayleigh_and_even_prandtl():
    cs = WL.cavity_batch(4000, 3, obstacles=False)
    lr = np.log10([c.Ra for c in cs])
    assert abs(lr.mean() - 4.5) < 0.05 and abs(lr.std() - 3 / math.sqrt(12)) < 0.05
    frac = np.mean([c.Pr == 0.71 for c in cs])
    assert abs(frac - 0.5) < 0.03


def test_obstacles_keep_clear_of_the_walls_and_stay_small(draw):
    with_mask = [c for c in draw if c.mask is not None]
    assert 0.5 * len(draw) < len(with_mask) < len(draw)  # 0 obstacles is one draw in four
    for c in with_mask:
        m = c.mask
        assert m.shape == (c.ny, c.nx) and m.dtype == np.uint8 and set(np.unique(m)) <= {0, 1}
        assert m.any()
        # two nodes of clearance from every wall
        assert not m[:2, :].any() and not m[-2:, :].any() and not m[:, :2].any() and not m[:, -2:].any()
        N = c.ny
        assert m.sum() <= 3 * (0.2 * N + 1) ** 2


def test_rasterize_rectangles_and_circles():
    m = WL.rasterize([("rect", 10.0, 8.0, 4.0, 2.0)], 21, 17)
    ys, xs = np.nonzero(m)
    assert (xs.min(), xs.max(), ys.min(), ys.max()) == (8, 12, 7, 9)  # |x - 10| <= 2, |y - 8| <= 1
    d = 40.0
    m = WL.rasterize([("circle", 50.0, 50.0, d)], 101, 101)
    assert abs(m.sum() - math.pi * d * d / 4) < 2 * math.pi * d / 2  # within one perimeter of nodes
    both = WL.rasterize([("rect", 10.0, 8.0, 4.0, 2.0), ("circle", 10.0, 8.0, 3.0)], 21, 17)
    assert np.array_equal(both, WL.rasterize([("rect", 10.0, 8.0, 4.0, 2.0)], 21, 17)
                          | WL.rasterize([("circle", 10.0, 8.0, 3.0)], 21, 17))


def test_warm_start_cases_are_square_128():
    cs = WL.warm_start_cases(40)
    assert all(c.nx == c.ny == 128 for c in cs)
    assert all(1e3 <= c.Ra <= 1e6 and c.Pr in (0.71, 7.0) for c in cs)


def test_random_fields_are_seeded_and_bounded():
    T = WL.random_temperature(5, 7, seed=1)
    assert T.shape == (5, 7) and T.min() >= 0 and T.max() <= 1
    assert np.array_equal(T, WL.random_temperature(5, 7, seed=1))
    u, v = WL.random_velocity(5, 7, seed=2, amp=0.01)
    assert np.abs(u).max() <= 0.01 and np.abs(v).max() <= 0.01 and not np.array_equal(u, v)


def test_substep_recipe_keeps_u0_and_the_relaxation_time():
    capped = WL.cavity_batch(64, 20190822)
    sub = WL.cavity_batch(64, 20190822, velocity="substeps")
    # the same groups, drawn from the same stream (a capped U0 lowers tau and
    # may move a cavity to a larger size)
    assert [(c.Ra, c.Pr) for c in capped] == [(c.Ra, c.Pr) for c in sub]
    assert all(c.ny >= d.ny for c, d in zip(capped, sub))
    slowed = 0
    for c, d in zip(capped, sub):
        assert math.isclose(d.Ma / math.sqrt(3.0), 0.1) and d.substeps == 0 and c.substeps == 1
        H = d.ny - 1
        nu = 0.1 * H * math.sqrt(d.Pr / d.Ra)
        assert 3 * nu + 0.5 >= 0.51 or d.ny == 512
        # the cap slows exactly the cavities one explicit step cannot take at
        # U0 = 0.1 (they are the ones that get sub-steps)
        if c.ny == d.ny:
            a01 = 0.1 * H / math.sqrt(d.Ra * d.Pr)
            assert (c.Ma < d.Ma - 1e-15) == (a01 > 0.2 or 0.01 > 1.8 * a01)
        slowed += c.Ma < d.Ma - 1e-15
    assert slowed > 0
    with pytest.raises(ValueError):
        WL.cavity_batch(2, 1, velocity="fast")


def test_stored_oracle_steady_states_belong_to_the_bench_draw():
    """tests/golden/steady_nusselt.json holds the FP64 oracle's steady states of
    the seeded draw the bench's time-to-steady measurement runs: same cavities
    (a draw of fewer cavities is a prefix of it), every residual below 1e-8,
    Nusselt numbers in the range of natural convection in these cavities."""
    import json
    import os

    p = os.path.join(os.path.dirname(__file__), "golden", "steady_nusselt.json")
    d = json.load(open(p))
    rows = d["cavities"]
    cases = WL.cavity_batch(len(rows), d["seed"], sizes=tuple(d["sizes"]), velocity=d["velocity"])
    assert [r["index"] for r in rows] == list(range(len(rows)))
    for r, c in zip(rows, cases):
        assert (r["nx"], r["ny"]) == (c.nx, c.ny)
        assert r["Ra"] == c.Ra and r["Pr"] == c.Pr and r["Ma"] == c.Ma
        assert r["residual"] < d["tol"] and 0.5 < r["nu_mean_hot"] < 20
    short = WL.cavity_batch(16, d["seed"], sizes=tuple(d["sizes"]), velocity=d["velocity"])
    assert [(c.nx, c.ny, c.Ra) for c in short] == [(c.nx, c.ny, c.Ra) for c in cases[:16]]


def test_stored_oracle_steady_state_of_the_256_instance():
    """tests/golden/config2_steady.json: the FP64 oracle's steady state of the
    1024^2 benchmark case's 256^2 instance (Ra 1e6, Pr 0.71, U0 0.1), residual
    below 1e-8, hot- and cold-wall Nusselt numbers equal at steady state (the
    heat entering leaves), the mean within 1 % of 8.8 (the classical
    benchmark value for this cavity at Ra 1e6; the paper prints its maximum,
    Table 1), temperatures inside [0, 1]."""
    import json
    import os

    d = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "config2_steady.json")))
    c = WL.config_large(256, 1e6)
    assert (d["nx"], d["ny"], d["Ra"], d["Pr"]) == (256, 256, 1e6, 0.71)
    assert math.isclose(d["Ma"], c.Ma)
    assert d["residual"] < d["tol"] == 1e-8
    assert abs(d["nu_mean_hot"] - d["nu_mean_cold"]) <= 1e-4 * d["nu_mean_hot"]
    assert abs(d["nu_mean_hot"] - 8.8) <= 0.09
    T = np.array(d["T_every_4th"])
    assert T.shape == (64, 64) and T.min() >= 0.0 and T.max() <= 1.0
