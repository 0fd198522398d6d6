"""The C-ABI library loads without a GPU, exports every entry point its header
declares, and rejects invalid arguments before touching the device."""

import os
import re

import numpy as np
import pytest

import paper_1908_08386_gb300 as L

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "lbmfvm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbmfvm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_what_the_binding_lists():
    assert declared_functions() == sorted(L.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = L.lib()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_opts_defaults():
    o = L.lbmfvm_opts_default()
    assert o.store == L.LBMFVM_F32 and o.tile_y == 0 and o.workspace is None
    assert o.t_ref != o.t_ref  # NaN selects T_l


def test_workspace_size_grows_with_precision():
    g = L.make_grid(100, 70)
    sizes = {}
    for name, p in L.PRECISIONS.items():
        o = L.lbmfvm_opts_default()
        o.store = p
        sizes[name] = L.lbmfvm_workspace_bytes(g, o)
    assert sizes["f16"] == sizes["bf16"] < sizes["f32"] < sizes["f64"]
    # two f planes of 9 populations, pitch rounded to 64 nodes
    assert sizes["f32"] >= 2 * 9 * 70 * 128 * 4


@pytest.mark.parametrize("nx,ny", [(2, 10), (10, 2), (0, 0)])
def test_rejects_tiny_grids(nx, ny):
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_workspace_bytes(L.make_grid(nx, ny))
    assert e.value.code == L.LBMFVM_ERR_ARG


def test_rejects_half_periodic():
    g = L.make_grid(10, 10, bc=(L.LBMFVM_BC_PERIODIC, L.LBMFVM_BC_DIRICHLET, 1, 1))
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_create_lattice(g, None, 0.1, 0.1, 0.0)
    assert e.value.code == L.LBMFVM_ERR_ARG


def test_stability_limits_are_checked_before_any_device_work():
    g = L.make_grid(64, 64)
    with pytest.raises(L.LbmfvmError) as e:  # tau = 3 nu + 1/2 < 0.51
        L.lbmfvm_create_lattice(g, None, 0.001, 0.1, 0.0)
    assert e.value.code == L.LBMFVM_ERR_UNSTABLE
    with pytest.raises(L.LbmfvmError) as e:  # explicit diffusion limit
        L.lbmfvm_create_lattice(g, None, 0.1, 0.3, 0.0)
    assert e.value.code == L.LBMFVM_ERR_UNSTABLE
    with pytest.raises(L.LbmfvmError) as e:  # Ma > 0.3
        L.lbmfvm_create(g, None, 1e4, 0.71, 0.5)
    assert e.value.code == L.LBMFVM_ERR_UNSTABLE
    with pytest.raises(L.LbmfvmError) as e:  # alpha = U0 H / sqrt(Ra Pr) > 0.25
        L.lbmfvm_create(L.make_grid(512, 512), None, 1e3, 0.71, 0.1 * 3**0.5)
    assert e.value.code == L.LBMFVM_ERR_UNSTABLE
    with pytest.raises(L.LbmfvmError) as e:  # no temperature difference
        L.lbmfvm_create(L.make_grid(64, 64, t_wall=(1, 1, 0, 0)), None, 1e4, 0.71, 0.1)
    assert e.value.code == L.LBMFVM_ERR_ARG
    assert "t_wall" in L.lbmfvm_last_error()


def test_workspace_too_small_is_rejected():
    g = L.make_grid(64, 64)
    o = L.lbmfvm_opts_default()
    o.workspace = 256
    o.workspace_bytes = 1024
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_create_lattice(g, None, 0.1, 0.1, 0.0, None, o)
    assert e.value.code == L.LBMFVM_ERR_NOMEM


def test_null_handle_calls_fail_cleanly():
    lib = L.lib()
    assert lib.lbmfvm_step(None, 1) == L.LBMFVM_ERR_ARG
    assert lib.lbmfvm_set_state(None, None, None, None) == L.LBMFVM_ERR_ARG
    lib.lbmfvm_destroy(None)


@pytest.mark.parametrize("cfg", [-3, 6, 99])
def test_rejects_unknown_tile_shapes(cfg):
    o = L.lbmfvm_opts_default()
    o.tma_config = cfg
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_create_lattice(L.make_grid(64, 64), None, 0.1, 0.1, 0.0, None, o)
    assert e.value.code == L.LBMFVM_ERR_ARG
    assert "tma_config" in L.lbmfvm_last_error()


def test_null_handle_queries_fail_cleanly():
    lib = L.lib()
    assert lib.lbmfvm_kernel_info(None, None, None) == L.LBMFVM_ERR_ARG
    assert lib.lbmfvm_copy_state(None, None) == L.LBMFVM_ERR_ARG
    assert lib.lbmfvm_batch_set_polish(None, L.LBMFVM_F32, 1e-6, 0) == L.LBMFVM_ERR_ARG


SG_HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "surrogate.h")


def test_surrogate_header_matches_its_binding_and_the_library():
    from paper_1908_08386_gb300 import surrogate as S

    text = re.sub(r"/\*.*?\*/", "", open(SG_HEADER).read(), flags=re.S)
    declared = sorted(set(re.findall(r"\b(lbmfvm_sg_[a-z0-9_]+)\s*\(", text)))
    assert declared == sorted(S.SG_EXPORTS)
    lib = L.lib()
    assert not [n for n in declared if not hasattr(lib, n)]


def test_surrogate_entry_points_check_shapes_without_a_gpu():
    from paper_1908_08386_gb300 import surrogate as S

    lib = S._lib()
    # H not a multiple of 8: refused before any launch
    assert lib.lbmfvm_sg_conv3x3(16, 16, 16, None, 16, 32, None, 0, 1, 12, 16, 16, 32, 1, None) == -1
    assert "tile rules" in lib.lbmfvm_sg_last_error().decode()
    # the tensor-core convolution's own limits: a padded row of W + 8
    # positions is one TMA box row (W <= 240), Cout <= 256 accumulator columns
    assert lib.lbmfvm_sg_conv3x3(16, 256, 16, None, 16, 32, None, 0, 1, 8, 256, 16, 32, 1, None) == -1
    assert "W <= 240" in lib.lbmfvm_sg_last_error().decode()
    assert lib.lbmfvm_sg_conv3x3(16, 16, 16, None, 16, 288, None, 0, 1, 8, 16, 16, 288, 1, None) == -1
    assert "Cout <= 256" in lib.lbmfvm_sg_last_error().decode()
    assert lib.lbmfvm_sg_adam(None, None, None, None, None, 10, 1e-3, 0.9, 0.999, 1e-8, 1, None) == -1


def test_energy_update_options_are_checked_before_any_device_work():
    g = L.make_grid(64, 64)
    o = L.lbmfvm_opts_default()
    assert (o.fv_scheme, o.fv_substeps) == (L.LBMFVM_FV_CENTRAL, 1)
    o.fv_scheme = 2
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_create_lattice(g, None, 0.1, 0.1, 0.0, None, o)
    assert e.value.code == L.LBMFVM_ERR_ARG
    o = L.lbmfvm_opts_default()
    o.fv_substeps = -1
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_create_lattice(g, None, 0.1, 0.1, 0.0, None, o)
    assert e.value.code == L.LBMFVM_ERR_ARG
    # alpha / m must stay within the explicit diffusion limit 1/4
    o = L.lbmfvm_opts_default()
    o.fv_substeps = 2
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_create_lattice(g, None, 0.1, 0.55, 0.0, None, o)
    assert e.value.code == L.LBMFVM_ERR_UNSTABLE
    # and U0^2 / m within 2 alpha: Ra = 1e6, Pr = 7 on 64^2 at U0 = 0.1 has
    # alpha = 0.0024, so one step is refused
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_create(g, None, 1e6, 7.0, 0.1 * 3**0.5)
    assert e.value.code == L.LBMFVM_ERR_UNSTABLE
    # QUICK and sub-steps run on the TMA kernel only (walls on every side)
    per = L.make_grid(64, 64, bc=(L.LBMFVM_BC_PERIODIC, L.LBMFVM_BC_PERIODIC, 1, 1))
    for scheme, m in ((L.LBMFVM_FV_QUICK, 1), (L.LBMFVM_FV_CENTRAL, 2)):
        o = L.lbmfvm_opts_default()
        o.fv_scheme, o.fv_substeps = scheme, m
        with pytest.raises(L.LbmfvmError) as e:
            L.lbmfvm_create_lattice(per, None, 0.1, 0.1, 0.0, None, o)
        assert e.value.code == L.LBMFVM_ERR_ARG


def test_workspace_holds_the_substep_planes():
    g = L.make_grid(70, 33)
    o = L.lbmfvm_opts_default()
    one = L.lbmfvm_workspace_bytes(g, o)
    o.fv_substeps = 3
    more = L.lbmfvm_workspace_bytes(g, o)
    # velocity planes u, v and two scratch temperature planes, FP32
    assert more - one >= 4 * 33 * 128 * 4


def test_d2q5_energy_solver_options_are_checked():
    g = L.make_grid(40, 40)
    for store in (L.LBMFVM_F16, L.LBMFVM_BF16):
        o = L.lbmfvm_opts_default()
        o.energy, o.store = L.LBMFVM_ENERGY_LBM_D2Q5, store
        with pytest.raises(L.LbmfvmError) as e:
            L.lbmfvm_create_lattice(g, None, 0.1, 0.1, 0.0, None, o)
        assert e.value.code == L.LBMFVM_ERR_ARG
    o = L.lbmfvm_opts_default()
    o.energy, o.fv_substeps = L.LBMFVM_ENERGY_LBM_D2Q5, 2
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_create_lattice(g, None, 0.1, 0.1, 0.0, None, o)
    assert e.value.code == L.LBMFVM_ERR_ARG
    o = L.lbmfvm_opts_default()
    o.energy = 7
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_create_lattice(g, None, 0.1, 0.1, 0.0, None, o)
    assert e.value.code == L.LBMFVM_ERR_ARG
    # the populations add two buffers of five planes
    o = L.lbmfvm_opts_default()
    fv = L.lbmfvm_workspace_bytes(g, o)
    o.energy = L.LBMFVM_ENERGY_LBM_D2Q5
    assert L.lbmfvm_workspace_bytes(g, o) - fv >= 2 * 5 * 40 * 64 * 4


def test_grid_setting_2_options_are_checked():
    def create(nx, ny, k=1, mask=None, alpha=0.1, **kw):
        o = L.lbmfvm_opts_default()
        o.fv_grid, o.fv_every = 2, k
        for a, v in kw.items():
            setattr(o, a, v)
        L.lbmfvm_create_lattice(L.make_grid(nx, ny), mask, 0.1, alpha, 0.0, None, o)

    assert (L.lbmfvm_opts_default().fv_grid, L.lbmfvm_opts_default().fv_every) == (1, 1)
    for args, code in (((40, 41), L.LBMFVM_ERR_ARG),          # odd number of spacings
                       ((41, 41, 0), L.LBMFVM_ERR_ARG),       # k < 1
                       ((41, 41, 9), L.LBMFVM_ERR_UNSTABLE)):  # alpha k > 0.8
        with pytest.raises(L.LbmfvmError) as e:
            create(*args)
        assert e.value.code == code, args
    mask = np.zeros((41, 41), np.uint8)
    mask[20, 20] = 1
    with pytest.raises(L.LbmfvmError) as e:
        create(41, 41, mask=mask)
    assert e.value.code == L.LBMFVM_ERR_ARG
    with pytest.raises(L.LbmfvmError) as e:
        create(41, 41, fv_substeps=2)
    assert e.value.code == L.LBMFVM_ERR_ARG
    o = L.lbmfvm_opts_default()
    o.fv_every = 2  # without grid setting 2
    with pytest.raises(L.LbmfvmError) as e:
        L.lbmfvm_create_lattice(L.make_grid(41, 41), None, 0.1, 0.1, 0.0, None, o)
    assert e.value.code == L.LBMFVM_ERR_ARG
