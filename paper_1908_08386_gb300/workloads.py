"""Seeded synthetic inputs for tests, the smoke check and the benchmark.

This module holds workload recipes only (sizes, Rayleigh/Prandtl numbers,
obstacle masks, random initial fields) and none of the method's arithmetic,
so both the CUDA path and the CPU oracle may take their inputs from it.

The differentially heated square cavity (Section 4.1.1: hot west wall, cold
east wall, adiabatic top and bottom, no slip everywhere) is the paper's
workload; it is a textbook benchmark and needs no dataset.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DIRICHLET, ADIABATIC, PERIODIC, MOVING = 0, 1, 2, 3
CAVITY_BC = (DIRICHLET, DIRICHLET, ADIABATIC, ADIABATIC)
CAVITY_T_WALL = (1.0, 0.0, 0.0, 0.0)
U0_DEFAULT = 0.1
MA_DEFAULT = U0_DEFAULT * math.sqrt(3.0)  # Ma = U0 / c_s with c_s = 1/sqrt(3)


@dataclass
class CavityCase:
    """One cavity: nodes nx x ny, groups Ra, Pr, Ma, optional obstacle mask."""

    nx: int
    ny: int
    Ra: float
    Pr: float
    Ma: float = MA_DEFAULT
    steps: int = 0
    mask: np.ndarray | None = field(default=None, repr=False)
    t_init: float = 0.5
    name: str = ""
    # energy-update sub-steps per lattice step: 1, or 0 for the library's
    # automatic choice (cavities drawn at U0 = 0.1 whatever their diffusivity)
    substeps: int = 1


def config_small() -> CavityCase:
    """64 x 64 nodes, Ra = 1e3, Pr = 0.71, U0 = 0.1, 10,000 steps, fluid at rest, T = 0.5."""
    return CavityCase(64, 64, 1e3, 0.71, MA_DEFAULT, 10_000, name="cavity64_Ra1e3")


def config_large(n: int = 1024, Ra: float = 1e6) -> CavityCase:
    """n x n nodes (1024 by default), Ra = 1e6, Pr = 0.71, U0 = 0.1, 100,000 steps.
    Larger cavities need a larger Ra to keep the thermal diffusivity
    U0 H / sqrt(Ra Pr) inside the explicit limit (e.g. Ra = 1e7 at 4096^2)."""
    return CavityCase(n, n, Ra, 0.71, MA_DEFAULT, 100_000, name=f"cavity{n}_Ra{Ra:.0e}")


def random_temperature(ny: int, nx: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=(ny, nx))


def random_velocity(ny: int, nx: int, seed: int, amp: float) -> tuple[np.ndarray, np.ndarray]:
    rng = np.random.default_rng(seed)
    return rng.uniform(-amp, amp, size=(ny, nx)), rng.uniform(-amp, amp, size=(ny, nx))


def rasterize(shapes, nx: int, ny: int) -> np.ndarray:
    """Solid mask (1 = solid) of rectangles and circles; a node is solid when
    its centre lies inside a shape.  shapes: ("rect", cx, cy, w, h) or
    ("circle", cx, cy, d) in node units."""
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    m = np.zeros((ny, nx), dtype=np.uint8)
    for s in shapes:
        if s[0] == "rect":
            _, cx, cy, w, h = s
            m |= ((np.abs(xx - cx) <= w / 2) & (np.abs(yy - cy) <= h / 2)).astype(np.uint8)
        else:
            _, cx, cy, d = s
            m |= (((xx - cx) ** 2 + (yy - cy) ** 2) <= (d / 2) ** 2).astype(np.uint8)
    return m


def random_obstacles(rng: np.random.Generator, nx: int, ny: int, N: int, kmax: int = 3):
    """0..kmax rectangles or circles of size 5-20 % of N, centred so that each
    keeps at least 2 nodes of clearance from every wall."""
    shapes = []
    for _ in range(int(rng.integers(0, kmax + 1))):
        if rng.random() < 0.5:
            w, h = rng.uniform(0.05, 0.2, size=2) * N
            hx, hy = w / 2, h / 2
            cx = rng.uniform(2 + hx, nx - 3 - hx)
            cy = rng.uniform(2 + hy, ny - 3 - hy)
            shapes.append(("rect", cx, cy, w, h))
        else:
            d = rng.uniform(0.05, 0.2) * N
            cx = rng.uniform(2 + d / 2, nx - 3 - d / 2)
            cy = rng.uniform(2 + d / 2, ny - 3 - d / 2)
            shapes.append(("circle", cx, cy, d))
    return shapes


def cavity_batch(count: int, seed: int, sizes=(64, 96, 128, 192, 256, 384, 512), obstacles: bool = True,
                 aspect=(1, 2), velocity: str = "capped") -> list[CavityCase]:
    """Uneven cavities: side N from `sizes`, aspect ratio 1 or 2 (ny = N,
    nx = a (N - 1) + 1), log10 Ra uniform in [3, 6], Pr in {0.71, 7.0}, up to
    three obstacles.  The velocity scale:
      "capped"    U0 = min(0.1, 0.2 sqrt(Ra Pr)/H, 1.8 H/sqrt(Ra Pr)) keeps
                  the thermal diffusivity alpha = U0 H/sqrt(Ra Pr) at or below
                  0.2 and U0^2 below 2 alpha (the stability conditions of one
                  explicit central FV step per lattice step);
      "substeps"  U0 = 0.1 for every cavity, and the energy update takes the
                  sub-steps that keep alpha/m <= 0.2 and U0^2/m <= 1.8 alpha
                  (substeps = 0: the library's automatic choice).
    A size whose relaxation time would fall below 0.51 is redrawn from the
    larger sizes."""
    if velocity not in ("capped", "substeps"):
        raise ValueError(f"velocity must be 'capped' or 'substeps', not {velocity!r}")
    rng = np.random.default_rng(seed)
    out = []
    sizes = sorted(sizes)
    for i in range(count):
        N = int(rng.choice(sizes))
        a = int(rng.choice(aspect))
        log_ra = rng.uniform(3.0, 6.0)
        Ra = 10.0 ** log_ra
        Pr = float(rng.choice([0.71, 7.0]))
        while True:
            H = N - 1
            if velocity == "capped":
                U0 = min(0.1, 0.2 * math.sqrt(Ra * Pr) / H, 1.8 * H / math.sqrt(Ra * Pr))
            else:
                U0 = 0.1
            tau = 3.0 * U0 * H * math.sqrt(Pr / Ra) + 0.5
            bigger = [s for s in sizes if s > N]
            if tau >= 0.51 or not bigger:
                break
            N = bigger[0]
        ny, nx = N, a * (N - 1) + 1
        mask = None
        if obstacles:
            shapes = random_obstacles(rng, nx, ny, N)
            if shapes:
                mask = rasterize(shapes, nx, ny)
        out.append(CavityCase(nx, ny, Ra, Pr, U0 * math.sqrt(3.0), 0, mask, 0.5, name=f"c{i}_N{N}_a{a}",
                              substeps=1 if velocity == "capped" else 0))
    return out


def warm_start_cases(count: int = 2000, seed: int = 20190823) -> list[CavityCase]:
    """Training cavities of the learned warm start: the uneven-batch recipe at
    N = 128 with aspect ratio 1 (Ra log-uniform in [1e3, 1e6], Pr in
    {0.71, 7.0}, up to three obstacles)."""
    return cavity_batch(count, seed, sizes=(128,), aspect=(1,), velocity="capped")


def surrogate_init(widths=(32, 64, 96, 160), seed: int = 0, cin: int = 3, cout: int = 3) -> list[np.ndarray]:
    """Seeded initial parameters of the warm-start network, in the order and
    shapes of its layers: per encoder level two 3x3 convolutions (weights
    [Co, 3, 3, Ci], biases [Co]), per decoder level (coarse to fine) two more,
    then the 1x1 output layer ([Co, Ci], [Co]).  He-normal weights
    (std sqrt(2 / fan_in)), zero biases, a small output layer."""
    rng = np.random.default_rng(seed)
    shapes = []
    c = cin
    for w in widths:
        shapes += [(w, 3, 3, c), (w,), (w, 3, 3, w), (w,)]
        c = w
    for lvl in range(len(widths) - 2, -1, -1):
        w = widths[lvl]
        shapes += [(w, 3, 3, widths[lvl + 1] + w), (w,), (w, 3, 3, w), (w,)]
    shapes += [(cout, widths[0]), (cout,)]
    out = []
    for s in shapes:
        if len(s) == 1:
            out.append(np.zeros(s))
        elif len(s) == 2:
            out.append(rng.standard_normal(s) * 0.01)
        else:
            out.append(rng.standard_normal(s) * math.sqrt(2.0 / (9 * s[3])))
    return out
