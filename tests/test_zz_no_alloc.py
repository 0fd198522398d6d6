"""lbmfvm_residual_noalloc: the residual reduction without any device
allocation, for callers that cannot allocate (device memory owned by another
allocator, loops that cannot afford cudaMalloc's synchronisation).

Checked through the C-ABI against the handle's own lbmfvm_residual on two
calls in a row, within the FP64 tolerance of two reductions that add the same
terms in different orders.  The file sorts last so that a failure here comes
after every other test has run; it also passes alone in a fresh process.
"""

import numpy as np
import pytest

import paper_1908_08386_gb300 as L
from paper_1908_08386_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def device_fields(cav, torch):
    shp = (cav.ny, cav.nx)
    u = torch.empty(shp, dtype=torch.float64, device="cuda")
    v = torch.empty(shp, dtype=torch.float64, device="cuda")
    L.lbmfvm_fields(cav.h, None, u, v, None)
    return u, v


def test_noalloc_residual_matches_handle_residual_twice():
    torch = pytest.importorskip("torch")
    case = WL.config_small()
    cav = L.Cavity(case.nx, case.ny, Ra=case.Ra, Pr=case.Pr, Ma=case.Ma, store="f32")
    # The handle's residual runs over fluid nodes; in a cavity without
    # obstacles those are the nodes off the box walls.
    fluid = np.zeros((cav.ny, cav.nx), dtype=np.uint8)
    fluid[1:-1, 1:-1] = 1
    sel = torch.from_numpy(fluid).cuda()
    u_prev, v_prev = device_fields(cav, torch)  # the snapshot set at create
    for _ in range(2):
        cav.step(700)
        u, v = device_fields(cav, torch)
        r_handle = cav.residual()
        r_static = L.lbmfvm_residual_noalloc(u, v, u_prev, v_prev, sel)
        r_all = L.lbmfvm_residual_noalloc(u, v, u_prev, v_prev)  # every node; walls carry u ~ 0
        assert r_handle > 0
        assert r_static == pytest.approx(r_handle, rel=1e-12)
        assert r_all == pytest.approx(r_handle, rel=1e-9)
        u_prev, v_prev = u, v


def test_noalloc_residual_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    u = torch.zeros(8, dtype=torch.float64, device="cuda")
    for n in (0, (1 << 30) + 1):
        with pytest.raises(L.LbmfvmError) as e:
            L.lbmfvm_residual_noalloc(u, u, u, u, n=n)
        assert e.value.code == L.LBMFVM_ERR_ARG
