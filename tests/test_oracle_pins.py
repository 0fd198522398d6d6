"""The FP64 oracle against closed forms, invariants and exact discrete
solutions (CPU only).  See tests/oracle_pins.py for what each pin fixes."""

import numpy as np
import pytest

import oracle
import oracle_pins as P


def make(*a, **k):
    return oracle.Oracle(*a, **k)


PINS = [
    P.rest_state,
    P.mass_periodic,
    P.shear_wave,
    P.advected_wave,
    P.poiseuille,
    P.conduction_linear,
    P.sine_mode_x,
    P.cosine_mode_y,
    P.advected_temperature,
    P.energy_adiabatic,
    P.energy_adiabatic_obstacle,
    P.uniform_buoyancy,
    P.quick_advected_mode,
    P.subcycled_sine_mode,
    P.quick_energy_adiabatic,
    P.quadratic_nusselt,
    P.eq112_conduction,
    P.homogeneous_in_f,
    P.nee_wall_moments,
    P.residual_shear_wave,
    P.residual_cavity_fluid_nodes,
    P.lbm_conduction_linear,
    P.lbm_thermal_decay,
    P.lbm_thermal_advection,
    P.lbm_thermal_conservation,
    P.lbm_thermal_walls,
    P.fd_poiseuille,
    P.fd_couette,
    P.fd_wall_moments,
    P.grid2_conduction_linear,
    P.grid2_periodic_decay,
    P.grid2_conservation,
    P.grid2_same_steady_state,
]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    ok, detail = pin(make)
    assert ok, detail


def test_params_from_groups_config_small():
    # Eqs. 83-89 with H = 63, Ra = 1e3, Pr = 0.71, U0 = 0.1 (Ma = 0.1 sqrt 3):
    # nu = U0 H sqrt(Pr/Ra), alpha = U0 H / sqrt(Ra Pr), g beta dT = U0^2 / H.
    nu, alpha, gbeta, tau = oracle.params_from_groups(1e3, 0.71, 0.1 * 3**0.5, 63)
    assert nu == pytest.approx(6.3 * (0.71e-3) ** 0.5, rel=1e-14)
    assert alpha == pytest.approx(6.3 / (710.0) ** 0.5, rel=1e-14)
    assert gbeta == pytest.approx(0.01 / 63, rel=1e-14)
    assert tau == pytest.approx(3 * nu + 0.5, rel=1e-14)
    # Pr = nu/alpha (Eq. 89's coefficients), Ra = g beta dT H^3 / (nu alpha).
    assert nu / alpha == pytest.approx(0.71, rel=1e-13)
    assert gbeta * 63**3 / (nu * alpha) == pytest.approx(1e3, rel=1e-13)


def test_thread_count_does_not_change_results():
    import os
    import subprocess
    import sys
    code = (
        "import sys; sys.path.insert(0, %r); import oracle, numpy as np\n"
        "o = oracle.Oracle.from_groups(130, 129, 1e5, 0.71, 0.1 * 3**0.5)\n"
        "o.step(300); np.save(sys.argv[1], np.stack(o.fields()))\n" % os.path.dirname(os.path.dirname(__file__))
    )
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        outs = []
        for t in ("1", "4"):
            path = os.path.join(d, f"t{t}.npy")
            env = dict(os.environ, OMP_NUM_THREADS=t)
            subprocess.run([sys.executable, "-c", code, path], check=True, env=env)
            import numpy as np
            outs.append(np.load(path))
        assert (outs[0] == outs[1]).all()


def test_quick_with_subcycling_matches_its_closed_form():
    ok, detail = P.quick_advected_mode(make, n=100, substeps=2)
    assert ok, detail


def test_fv_options_are_checked():
    with pytest.raises(ValueError):
        oracle.Oracle(8, 8, nu=0.1, alpha=0.1, fv_scheme="upwind")
    with pytest.raises(ValueError):
        oracle.Oracle(8, 8, nu=0.1, alpha=0.1, fv_substeps=0)


def test_energy_and_wall_options_are_checked():
    with pytest.raises(ValueError):
        oracle.Oracle(8, 8, nu=0.1, alpha=0.1, energy="mcm")
    with pytest.raises(ValueError):
        oracle.Oracle(8, 8, nu=0.1, alpha=0.1, wall_bc="bounce")
    with pytest.raises(ValueError):  # an odd number of spacings
        oracle.Oracle(8, 9, nu=0.1, alpha=0.1, fv_grid=2)
    mask = np.zeros((9, 9), np.uint8)
    mask[4, 4] = 1
    with pytest.raises(ValueError):  # an obstacle
        oracle.Oracle(9, 9, nu=0.1, alpha=0.1, fv_grid=2, mask=mask)
