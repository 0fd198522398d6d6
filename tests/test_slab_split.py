"""One cavity split into two y-slabs held by two gloo ranks on the CPU, with
halo rows copied between the ranks after every step: the owned rows equal the
unsplit oracle bit for bit, and the residual from per-slab partial sums (one
FP64 all-reduce) equals the unsplit residual to rounding.  This is the
exchange a slab decomposition of one cavity over several GPUs would make once
per step; the library itself runs whole cavities per GPU.

Each rank steps an oracle instance of the whole box, but only its own rows and
h halo rows hold the state: every other row is set to NaN after each step, so
that any dependence reaching beyond the halo arrives in the owned rows as
NaN.  One coupled step reads two rows away: the pull takes the collided
neighbours (one row), and the energy balance's face velocities need the
neighbour row's new moments, pulled from the row beyond (two rows); QUICK's
far upstream temperature is two rows away at the old step.  A wall node on
the neighbour row is rebuilt from its partner, but what an owned row takes
from it within the step is its wall velocity (Eq. 94 fixes it) or nothing
(obstacle surfaces are outside the balance).  So h = 2 suffices, also with
the finite-difference box walls, and with h = 1 NaN reaches the owned rows.
"""

import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_1908_08386_gb300 import workloads as WL  # noqa: E402

NX, NY, CUT = 45, 38, 19
RA, PR, MA = 1e5, 0.71, 0.1 * math.sqrt(3.0)
STEPS = 40


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def mask():
    # obstacles across the cut row, so that wall nodes sit beside it
    return WL.rasterize([("rect", 8, CUT - 4, 9, 7), ("circle", 30, CUT + 1, 6)], NX, NY)


CASES = {"central": {}, "quick": {"fv_scheme": "quick"}, "fd_walls": {"wall_bc": "fd"}}


def make(case):
    return oracle.Oracle.from_groups(NX, NY, RA, PR, MA, mask=mask(), **CASES[case])


def exchange(rank, f, T, lo, hi, h):
    """Send the h edge rows of the own slab to the neighbour rank and take its
    h edge rows into this rank's halo (rank 0 holds rows [0, CUT), rank 1
    rows [CUT, NY))."""
    if rank == 0:
        out = torch.from_numpy(np.concatenate([f[:, hi - h:hi].ravel(), T[hi - h:hi].ravel()]))
        inc = torch.empty_like(out)
        dist.send(out, 1)
        dist.recv(inc, 1)
        rows = slice(hi, hi + h)
    else:
        out = torch.from_numpy(np.concatenate([f[:, lo:lo + h].ravel(), T[lo:lo + h].ravel()]))
        inc = torch.empty_like(out)
        dist.recv(inc, 0)
        dist.send(out, 0)
        rows = slice(lo - h, lo)
    a = inc.numpy()
    nf = 9 * h * NX
    f[:, rows] = a[:nf].reshape(9, h, NX)
    T[rows] = a[nf:].reshape(h, NX)


def run_slab(rank, case, h):
    lo, hi = (0, CUT) if rank == 0 else (CUT, NY)
    o = make(case)
    u0 = o.fields()[1:3]
    keep = np.zeros(NY, bool)
    keep[max(lo - h, 0):min(hi + h, NY)] = True
    for _ in range(STEPS):
        o.step(1)
        f = o.f()
        T = o.fields()[3]
        f[:, ~keep] = np.nan
        T[~keep] = np.nan
        exchange(rank, f, T, lo, hi, h)
        o.set_f(f)
        o.set_T(T)
    _, u, v, T = o.fields()
    kind = o.classes()[0]
    # residual partial sums over this slab's fluid nodes, summed over ranks
    fl = np.zeros((NY, NX), bool)
    fl[lo:hi] = kind[lo:hi] == 0
    part = torch.tensor([((u - u0[0])[fl] ** 2 + (v - u0[1])[fl] ** 2).sum(), (u[fl] ** 2 + v[fl] ** 2).sum()],
                        dtype=torch.float64)
    dist.all_reduce(part)
    return o.f()[:, lo:hi], u[lo:hi], v[lo:hi], T[lo:hi], math.sqrt(part[0]) / math.sqrt(part[1])


def _rank(rank, size, port, out):
    os.environ.update(OMP_NUM_THREADS="1")
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=size)
    res = {}
    for case, h in (("central", 2), ("quick", 2), ("fd_walls", 2), ("central", 1)):
        res[(case, h)] = run_slab(rank, case, h)
    out.put((rank, res))
    dist.destroy_process_group()


@pytest.fixture(scope="module")
def slabs():
    size, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, size, port, q)) for r in range(size)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(size))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return got


@pytest.mark.parametrize("case", list(CASES))
def test_two_slabs_with_two_halo_rows_equal_the_unsplit_oracle(slabs, case):
    ref = make(case)
    ref.step(STEPS)
    f_ref = ref.f()
    _, u_ref, v_ref, T_ref = ref.fields()
    r_ref = ref.residual()
    for rank, (lo, hi) in ((0, (0, CUT)), (1, (CUT, NY))):
        f, u, v, T, r = slabs[rank][(case, 2)]
        assert np.array_equal(f, f_ref[:, lo:hi]), rank
        assert np.array_equal(u, u_ref[lo:hi]) and np.array_equal(v, v_ref[lo:hi]), rank
        assert np.array_equal(T, T_ref[lo:hi]), rank
        assert r == pytest.approx(r_ref, rel=1e-12)
        assert np.isfinite(T).all()


def test_one_halo_row_lets_the_missing_rows_reach_the_slab(slabs):
    for rank in (0, 1):
        T = slabs[rank][("central", 1)][3]
        assert np.isnan(T).any(), rank
