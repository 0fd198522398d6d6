"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check that
each one fails at least one pin: the pins constrain every part of the step."""

import os

import pytest

import oracle
import oracle_pins as P

MUTANTS = {
    "collision_sign": ("o->fs[q * n + k] = fv - (fv - fe) / tau + F;", "o->fs[q * n + k] = fv + (fv - fe) / tau + F;"),
    "feq_drop_quadratic": ("eu * eu / (2.0 * CS2 * CS2)", "0.0"),
    "feq_drop_u2": ("- uu / (2.0 * CS2))", ")"),
    "force_drop_minus_u": ("(Gx * (EX[q] - ux) + Gy * (EY[q] - uy))", "(Gx * EX[q] + Gy * EY[q])"),
    "force_missing_cs2": ("* fe / (RHO0 * CS2);", "* fe / RHO0;"),
    "force_without_reference_temperature": ("o->gbeta * (o->T[k] - o->t_ref)", "o->gbeta * o->T[k]"),
    "weight_diagonal": ("1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0}", "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 35.0}"),
    "tau_without_half": ("o->tau = nu / CS2 + 0.5;", "o->tau = nu / CS2 + 0.6;"),
    "stream_push_direction": ("int s = nbr(o, i, j, -EX[q], -EY[q]);\n                o->f[q * n + k]",
                              "int s = nbr(o, i, j, -EX[q], EY[q]);\n                o->f[q * n + k]"),
    # (the finite-difference walls start from the same equilibrium: name the
    # extrapolation's site by the term that follows it)
    "nee_partner_velocity": ("feq(q, rf, o->uw[k], o->vw[k]) + o->f[q * n + p]", "feq(q, rf, uf, vf) + o->f[q * n + p]"),
    "nee_wall_density_unit": ("feq(q, rf, o->uw[k], o->vw[k]) + o->f[q * n + p]",
                              "feq(q, 1.0, o->uw[k], o->vw[k]) + o->f[q * n + p]"),
    "nee_equilibrium_only": ("+ o->f[q * n + p] - feq(q, rf, uf, vf);", ";"),
    "fv_convective_sign": ("acc += -Fl * Tf + alpha", "acc += Fl * Tf + alpha"),
    "quick_downstream_weight": ("0.375 * o->T[down]", "0.25 * o->T[down]"),
    "quick_upstream_side": ("if (un >= 0.0) {", "if (un < 0.0) {"),
    "quick_far_node": ("far = nbr(o, i, j, -dx, -dy);", "far = nbr(o, i, j, dx, dy);"),
    "subcycle_full_step": ("const double dt = 1.0 / m_sub;", "const double dt = 1.0;"),
    "fv_obstacle_faces_open": ("(o->therm[k] == TH_FV || o->therm[k] == TH_DIRICHLET)",
                               "(o->therm[k] == TH_FV || o->therm[k] == TH_DIRICHLET || o->therm[k] == TH_OBSTACLE)"),
    "fv_face_velocity_one_sided": ("(o->ux[k] + o->ux[mm]) * dx", "(o->ux[k] + o->ux[k]) * dx"),
    "fv_half_cv_y": ("return 0.5 * (j > 0) + 0.5 * (j < o->ny - 1);", "return 1.0;"),
    "fv_diffusion_area": ("alpha * A * (o->T[mm] - TP)", "alpha * (o->T[mm] - TP)"),
    "nusselt_first_order": ("(-3.0 * r[0] + 4.0 * r[1] - r[2]) / (2.0 * dT)", "(-r[0] + r[1]) / dT"),
    "nusselt_trapezoid": ("(j == 0 || j == ny - 1) ? 0.5 : 1.0", "1.0"),
    "flux_nusselt_diffusion_area": ("Qs += A * un * Tf - o->alpha * A * (o->T[m] - o->T[k]);",
                                    "Qs += A * un * Tf - o->alpha * (o->T[m] - o->T[k]);"),
    "d2q5_rest_weight": ("static const double W5[Q5] = {1.0 / 3.0,", "static const double W5[Q5] = {0.35,"),
    "d2q5_tau_relation": ("o->tau_T = o->alpha / CS2 + 0.5;", "o->tau_T = o->alpha / 0.5 + 0.5;"),
    "d2q5_equilibrium_velocity_factor": ("return T * W5[q] * (1.0 + (EX[q] * ux + EY[q] * uy) / CS2);",
                                         "return T * W5[q] * (1.0 + (EX[q] * ux + EY[q] * uy));"),
    "d2q5_walls_equilibrium_only": ("+ o->g[q * n + p] - geq(q, Tf, uf, vf);", ";"),
    "d2q5_adiabatic_wall_cold": ("dirichlet_value(o, i, j) : Tf;", "dirichlet_value(o, i, j) : 0.0;"),
    "d2q5_stream_direction": ("int s = nbr(o, i, j, -EX[q], -EY[q]);\n                    o->g[q * n + k]",
                              "int s = nbr(o, i, j, EX[q], -EY[q]);\n                    o->g[q * n + k]"),
    "fd_walls_skipped": ("if (o->wall_bc == WALL_FD) {", "if (0) {"),
    "fd_without_tau": ("- tau * W[q] / CS2 * rf * qs;", "- W[q] / CS2 * rf * qs;"),
    "fd_sign": ("- tau * W[q] / CS2 * rf * qs;", "+ tau * W[q] / CS2 * rf * qs;"),
    "fd_first_order_wall_gradient": ("*du = s * (-3.0 * u0 + 4.0 * u1 - u2) / 2.0;", "*du = s * (u1 - u0);"),
    "fd_wall_density_unit": ("o->f[q * n + k] = feq(q, rf, o->uw[k], o->vw[k]) - tau", "o->f[q * n + k] = feq(q, 1.0, o->uw[k], o->vw[k]) - tau"),
    "fd_shear_half": ("double sxx = dudx, syy = dvdy, sxy = 0.5 * (dudy + dvdx);", "double sxx = dudx, syy = dvdy, sxy = 0.25 * (dudy + dvdx);"),
    "grid2_wall_full_distance": ("acc += alpha * A * (o->t_wall[SIDE[f]] - TP) / 1.0;",
                                 "acc += alpha * A * (o->t_wall[SIDE[f]] - TP) / 2.0;"),
    "grid2_time_step_one": ("const double dt = o->fv_every, V = 4.0, A = 2.0, alpha = o->alpha;",
                            "const double dt = 1.0, V = 4.0, A = 2.0, alpha = o->alpha;"),
    "grid2_interpolation_one_sided": ("else { ia[0] = i / 2 - 1; ia[1] = i / 2; ni = 2; }", "else { ia[0] = i / 2 - 1; ni = 1; }"),
    "grid2_face_node": ("int fi = ci + dx, fj = cj + dy;", "int fi = ci + 2 * dx, fj = cj + dy;"),
    "residual_without_square_roots": ("return sqrt(num) / sqrt(den);", "return num / den;"),
    "residual_normalised_by_snapshot": ("den += o->ux[k] * o->ux[k] + o->uy[k] * o->uy[k];",
                                        "den += o->su[k] * o->su[k] + o->sv[k] * o->sv[k];"),
    "residual_walls_included": ("if (o->kind[k] != K_FLUID) continue;\n        double du", "if (o->kind[k] == K_SOLID) continue;\n        double du"),
}


@pytest.fixture(scope="module")
def source():
    return oracle.source_text()


@pytest.fixture(scope="module")
def builds(source, tmp_path_factory):
    """Every mutant compiled once, the compilers running side by side."""
    from concurrent.futures import ThreadPoolExecutor

    out = tmp_path_factory.mktemp("mutants")

    def build(name):
        old, new = MUTANTS[name]
        if source.count(old) != 1:
            return name, None
        return name, oracle.build_variant(source.replace(old, new), os.path.join(str(out), f"m_{name}.so"))

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as pool:
        return dict(pool.map(build, sorted(MUTANTS)))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, source, builds):
    old, _ = MUTANTS[name]
    assert source.count(old) == 1, f"mutation site for {name} not found exactly once"
    lib = oracle.load_library(builds[name])

    def make(*a, **k):
        return oracle.Oracle(*a, lib=lib, **k)

    # the first pin that fails is enough
    for pin_name, pin in P.QUICK.items():
        try:
            ok, detail = pin(make)
        except Exception as exc:  # a mutant may also blow up outright
            ok, detail = False, f"raised {exc!r}"
        if not ok:
            return
    pytest.fail(f"mutant {name} passed every pin")
