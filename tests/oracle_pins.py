"""Pins of the FP64 oracle: closed forms, invariants and exact discrete
solutions that fix each part of the coupled step independently of the oracle
itself.  Each check takes a factory ``make(nx, ny, **kw) -> Oracle`` so the
same checks run on the real oracle and on copies with planted mistakes.

Every check returns (ok: bool, detail: str).
"""

from __future__ import annotations

import math

import numpy as np

W, E, S, N = 0, 1, 2, 3
DIR, ADI, PER, MOV = 0, 1, 2, 3


def rest_state(make):
    """No force, fluid at rest: f stays at the weights of Eq. 9 and u = 0 exactly."""
    o = make(20, 13, nu=0.1, alpha=0.2, gbeta=0.0)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    o.step(100)
    f = o.f()
    _, u, v, _ = o.fields()
    err = np.abs(f - w).max()
    ok = err <= 4e-16 and np.all(u == 0.0) and np.all(v == 0.0)
    return ok, f"max|f - w| = {err:.3g}, u == 0: {np.all(u == 0.0) and np.all(v == 0.0)}"


def mass_periodic(make, steps=10_000):
    """Periodic box with buoyancy from a random T field: the collision, the
    force (sum_i F_i = 0) and streaming conserve sum f to round-off."""
    rng = np.random.default_rng(7)
    o = make(32, 17, bc=(PER, PER, PER, PER), nu=0.1, alpha=0.2, gbeta=1e-5, t_ref=0.5)
    o.set_state(T=rng.random((17, 32)))
    m0 = o.f().sum()
    o.step(steps)
    rel = abs(o.f().sum() - m0) / m0
    return rel <= 1e-11, f"relative mass change over {steps} steps = {rel:.3g}"


def shear_wave(make):
    """Periodic shear wave u_x = A sin(2 pi y / L): decays as exp(-nu k^2 t)
    with nu = (tau - 1/2)/3 (Eq. 15)."""
    L, nu, A = 64, 0.1, 1e-4
    o = make(3, L, bc=(PER, PER, PER, PER), nu=nu, alpha=0.1, gbeta=0.0)
    y = np.arange(L)
    u0 = np.tile(A * np.sin(2 * np.pi * y / L)[:, None], (1, 3))
    o.set_state(u=u0)
    k = 2 * np.pi / L
    amp = []
    for t in (300, 3000):
        o.step(t - o.step_count)
        u = o.fields()[1][:, 1]
        amp.append(2 / L * np.sum(u * np.sin(k * y)))
    rate = math.log(amp[0] / amp[1]) / 2700
    rel = abs(rate / (nu * k * k) - 1)
    return rel <= 0.01, f"decay rate / (nu k^2) - 1 = {rel:.3g}"


def advected_wave(make):
    """Transverse wave on a uniform stream (Galilean invariance of Eq. 8's
    quadratic terms): v = A sin(k x) on (U, 0) and u = A sin(k y) on (0, U)
    both travel downstream at U."""
    L, nu, A, U, t = 64, 0.05, 1e-4, 0.05, 320
    k = 2 * np.pi / L
    s = np.arange(L)
    speeds = []
    for along_x in (True, False):
        if along_x:
            o = make(L, 3, bc=(PER, PER, PER, PER), nu=nu, alpha=0.1, gbeta=0.0)
            o.set_state(u=np.full((3, L), U), v=np.tile(A * np.sin(k * s), (3, 1)))
        else:
            o = make(3, L, bc=(PER, PER, PER, PER), nu=nu, alpha=0.1, gbeta=0.0)
            o.set_state(u=np.tile(A * np.sin(k * s)[:, None], (1, 3)), v=np.full((L, 3), U))
        o.step(t)
        prof = o.fields()[2][1] if along_x else o.fields()[1][:, 1]
        c = np.sum(prof * np.cos(k * s))
        sn = np.sum(prof * np.sin(k * s))
        shift = math.atan2(-c, sn) / k  # profile ~ sin(k (s - shift))
        speeds.append(shift / t)
    rel = max(abs(sp / U - 1) for sp in speeds)
    return rel <= 0.02, f"phase speeds / U - 1 = {[round(sp / U - 1, 6) for sp in speeds]}"


def poiseuille(make, Hs=(8, 16, 32)):
    """Force-driven channel between non-equilibrium-extrapolation walls:
    steady u(y) = g y (H - y) / (2 nu); L2 error falls at second order."""
    errs = []
    for H in Hs:
        nu, umax = 0.1, 0.01
        g = 8 * nu * umax / H**2
        o = make(3, H + 1, bc=(PER, PER, ADI, ADI), nu=nu, alpha=0.1, gbeta=0.0, fx=g)
        o.step(int(3 * H * H / nu))
        u = o.fields()[1][:, 1]
        y = np.arange(H + 1)
        ex = g * y * (H - y) / (2 * nu)
        errs.append(float(np.sqrt(np.mean((u - ex) ** 2)) / umax))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    ok = min(orders) >= 1.8 and errs[0] < 0.05
    return ok, f"errors {['%.3g' % e for e in errs]}, orders {['%.3f' % p for p in orders]}"


def conduction_linear(make, H=16):
    """Pure conduction between T = 1 (west) and T = 0 (east), adiabatic top
    and bottom: the steady field is T = 1 - x/H to round-off, and the
    one-sided Nusselt number and the heat through every vertical face line
    (normalised by alpha dT) are exactly 1."""
    o = make(H + 1, H + 1, nu=0.1, alpha=0.2, gbeta=0.0)
    o.step(6000)
    T = o.fields()[3]
    x = np.arange(H + 1) / H
    err = np.abs(T - (1 - x)[None, :]).max()
    nh, _, nc, _ = o.nusselt()
    # the heat through every vertical face line is alpha dT (H/H): Nu = 1
    fl = np.abs(o.flux_nusselt() - 1).max()
    ok = err <= 1e-12 and abs(nh - 1) <= 1e-12 and abs(nc - 1) <= 1e-12 and fl <= 1e-12
    return ok, (f"max|T - (1 - x/H)| = {err:.3g}, Nu hot - 1 = {nh - 1:.3g}, Nu cold - 1 = {nc - 1:.3g}, "
                f"max|flux Nu - 1| = {fl:.3g}")


def sine_mode_x(make, H=20, n=500, alpha=0.2):
    """T_W = T_E = 0, adiabatic top/bottom, T0 = sin(pi x / H), no flow: the
    discrete eigenvector decays by (1 - 4 alpha sin^2(pi/(2H))) per step."""
    o = make(H + 1, 9, t_wall=(0, 0, 0, 0), nu=0.1, alpha=alpha, gbeta=0.0)
    x = np.arange(H + 1)
    T0 = np.tile(np.sin(np.pi * x / H), (9, 1))
    o.set_state(T=T0)
    o.step(n)
    g = 1 - 4 * alpha * math.sin(math.pi / (2 * H)) ** 2
    err = np.abs(o.fields()[3] - g**n * T0).max()
    cont = math.exp(-alpha * (math.pi / H) ** 2 * n)
    return err <= 1e-12, f"max error vs exact discrete decay = {err:.3g} (continuum factor {cont:.6f}, discrete {g**n:.6f})"


def cosine_mode_y(make, H=16, n=400, alpha=0.2):
    """Periodic in x, adiabatic bottom/top (half control volumes at the wall
    rows): T0 = cos(pi y / H) decays by (1 - 4 alpha sin^2(pi/(2H))) per step."""
    o = make(5, H + 1, bc=(PER, PER, ADI, ADI), nu=0.1, alpha=alpha, gbeta=0.0)
    y = np.arange(H + 1)
    T0 = np.tile(np.cos(np.pi * y / H)[:, None], (1, 5))
    o.set_state(T=T0)
    o.step(n)
    g = 1 - 4 * alpha * math.sin(math.pi / (2 * H)) ** 2
    err = np.abs(o.fields()[3] - g**n * T0).max()
    return err <= 1e-12, f"max error vs exact discrete decay = {err:.3g}"


def advected_temperature(make, L=32, n=200, alpha=0.05):
    """Uniform stream (U, V) in a periodic box (an exact steady state of the
    lattice Boltzmann part), T0 = cos(k x + l y): the explicit central
    finite-volume update multiplies the Fourier mode by
    g = 1 - 4 alpha (sin^2(k/2) + sin^2(l/2)) - i (U sin k + V sin l) per step."""
    U, V = 0.06, -0.03
    o = make(L, L, bc=(PER, PER, PER, PER), nu=0.1, alpha=alpha, gbeta=0.0)
    k = 2 * np.pi * 2 / L
    l = 2 * np.pi * 1 / L
    yy, xx = np.mgrid[0:L, 0:L]
    o.set_state(u=np.full((L, L), U), v=np.full((L, L), V), T=np.cos(k * xx + l * yy))
    o.step(n)
    g = 1 - 4 * alpha * (math.sin(k / 2) ** 2 + math.sin(l / 2) ** 2) - 1j * (U * math.sin(k) + V * math.sin(l))
    exact = np.real(g**n * np.exp(1j * (k * xx + l * yy)))
    err = np.abs(o.fields()[3] - exact).max()
    return err <= 1e-11, f"max error vs exact discrete mode = {err:.3g}"


def _quick_factor(c, kappa):
    """(T_f+ - T_f-) / T_P for a Fourier mode exp(i kappa j) under QUICK face
    values (6/8 upstream, 3/8 downstream, -1/8 beyond upstream) with a
    uniform velocity c along the axis: for c >= 0 the faces take their values
    from the node behind them, for c < 0 from the node ahead (the mirror)."""
    def qp(k):
        e = np.exp(1j * k)
        return (3 + 3 * e - 7 / e + 1 / (e * e)) / 8
    return qp(kappa) if c >= 0 else -qp(-kappa)


def quick_advected_mode(make, L=32, n=200, alpha=0.05, substeps=1):
    """QUICK face values (Section 3.1's scheme, Leonard's quadratic upstream
    interpolation) on a uniform stream (U, V) in a periodic box: the explicit
    update multiplies the Fourier mode cos(k x + l y) by
    g = (1 + L_h / m)^m per step, L_h = -4 alpha (sin^2(k/2) + sin^2(l/2))
    - U Q(k) - V Q(l) with Q the QUICK flux-difference symbol and m the
    sub-steps."""
    U, V = 0.06, -0.03
    o = make(L, L, bc=(PER, PER, PER, PER), nu=0.1, alpha=alpha, gbeta=0.0, fv_scheme="quick",
             fv_substeps=substeps)
    k = 2 * np.pi * 2 / L
    l = 2 * np.pi * 1 / L
    yy, xx = np.mgrid[0:L, 0:L]
    o.set_state(u=np.full((L, L), U), v=np.full((L, L), V), T=0.5 + 0.1 * np.cos(k * xx + l * yy))
    o.step(n)
    Lh = -4 * alpha * (math.sin(k / 2) ** 2 + math.sin(l / 2) ** 2) - U * _quick_factor(U, k) - V * _quick_factor(V, l)
    g = (1 + Lh / substeps) ** substeps
    exact = 0.5 + 0.1 * np.real(g**n * np.exp(1j * (k * xx + l * yy)))
    err = np.abs(o.fields()[3] - exact).max()
    central = abs(1 - 4 * alpha * (math.sin(k / 2) ** 2 + math.sin(l / 2) ** 2)
                  - 1j * (U * math.sin(k) + V * math.sin(l))) ** n
    return err <= 1e-11, f"max error vs exact discrete mode = {err:.3g} (|g|^n {abs(g)**n:.6f}, central {central:.6f})"


def subcycled_sine_mode(make, H=20, n=300, alpha=0.6, substeps=3):
    """alpha = 0.6 exceeds the explicit limit 1/4 of one step; with m = 3
    sub-steps of dt = 1/3 the Dirichlet sine mode decays by exactly
    (1 - 4 (alpha/m) sin^2(pi/(2H)))^m per step."""
    o = make(H + 1, 9, t_wall=(0, 0, 0, 0), nu=0.1, alpha=alpha, gbeta=0.0, fv_substeps=substeps)
    x = np.arange(H + 1)
    T0 = np.tile(np.sin(np.pi * x / H), (9, 1))
    o.set_state(T=T0)
    o.step(n)
    g = (1 - 4 * (alpha / substeps) * math.sin(math.pi / (2 * H)) ** 2) ** substeps
    err = np.abs(o.fields()[3] - g**n * T0).max()
    return err <= 1e-12, f"max error vs exact discrete decay = {err:.3g} (factor {g**n:.6f})"


def quick_energy_adiabatic(make, n=600):
    """QUICK face values and two sub-steps in an adiabatic box with buoyant
    flow and an insulated obstacle: every face's value is shared by its two
    nodes, so sum V_P T_P stays constant to round-off."""
    rng = np.random.default_rng(9)
    mask = np.zeros((19, 24), np.uint8)
    mask[6:11, 8:14] = 1
    o = make(24, 19, bc=(ADI, ADI, ADI, ADI), mask=mask, nu=0.05, alpha=0.3, gbeta=2e-3, t_ref=0.5,
             fv_scheme="quick", fv_substeps=2)
    o.set_state(T=rng.random((19, 24)))
    V = o.cv_volumes()
    e0 = np.sum(V * o.fields()[3])
    o.step(n)
    _, u, _, T = o.fields()
    rel = abs(np.sum(V * T) - e0) / e0
    moving = np.abs(u).max()
    return rel <= 1e-13 and moving > 1e-5, f"relative energy change = {rel:.3g} (max|u| = {moving:.3g})"


def energy_adiabatic(make, n=1000):
    """All walls adiabatic, buoyant flow from a random T: the conservative
    flux form keeps sum V_P T_P constant to round-off."""
    rng = np.random.default_rng(3)
    o = make(24, 19, bc=(ADI, ADI, ADI, ADI), nu=0.05, alpha=0.15, gbeta=2e-3, t_ref=0.5)
    o.set_state(T=rng.random((19, 24)))
    V = o.cv_volumes()
    e0 = np.sum(V * o.fields()[3])
    o.step(n)
    _, u, _, T = o.fields()
    rel = abs(np.sum(V * T) - e0) / e0
    moving = np.abs(u).max()
    return rel <= 1e-13 and moving > 1e-5, f"relative energy change = {rel:.3g} (max|u| = {moving:.3g})"


def uniform_buoyancy(make, n=100, T=0.7, t_ref=0.5, gbeta=1e-4):
    """A periodic box at a uniform temperature T: the Boussinesq force of
    Eqs. 18 and 81, G = g beta (T - T_ref) upward, is the same at every node,
    the field stays uniform, the energy update leaves T unchanged, and the
    force's momentum source sum_i e_i F_i = rho G makes v grow by exactly G
    per step (rho = 1): v = n G after n steps from rest."""
    o = make(16, 12, bc=(PER, PER, PER, PER), nu=0.05, alpha=0.1, gbeta=gbeta, t_ref=t_ref)
    o.set_state(T=np.full((12, 16), T))
    o.step(n)
    _, u, v, Tn = o.fields()
    G = gbeta * (T - t_ref)
    rel = abs(v.mean() / (n * G) - 1)
    ok = rel <= 1e-11 and np.ptp(v) <= 1e-18 and np.all(u == 0.0) and np.all(Tn == T)
    return ok, f"v / (n G) - 1 = {rel:.3g}, spread of v {np.ptp(v):.3g}, max|u| = {np.abs(u).max():.3g}"


def energy_adiabatic_obstacle(make, n=800):
    """An insulated obstacle in an adiabatic box with buoyant flow: its
    surface faces carry no flux (its nodes copy their partner's temperature
    and take no part in the balance), so sum V_P T_P over the finite-volume
    nodes stays constant to round-off."""
    rng = np.random.default_rng(5)
    mask = np.zeros((19, 24), np.uint8)
    mask[6:11, 8:14] = 1
    o = make(24, 19, bc=(ADI, ADI, ADI, ADI), mask=mask, nu=0.05, alpha=0.15, gbeta=2e-3, t_ref=0.5)
    o.set_state(T=rng.random((19, 24)))
    V = o.cv_volumes()
    e0 = np.sum(V * o.fields()[3])
    o.step(n)
    _, u, _, T = o.fields()
    rel = abs(np.sum(V * T) - e0) / e0
    moving = np.abs(u).max()
    return rel <= 1e-13 and moving > 1e-5, f"relative energy change = {rel:.3g} (max|u| = {moving:.3g})"


def quadratic_nusselt(make, H=20):
    """Eq. 90 from the one-sided second-order stencil is exact for T quadratic
    in x: T = 1 - X + c(Y) X (X - 1) gives Nu(Y) = 1 + c(Y); with c linear in Y
    the trapezoid mean is 1 + c0 + c1/2."""
    ny = H + 1  # X = x/H and Y = y/H share the cavity height H = ny - 1
    o = make(H + 1, ny, nu=0.1, alpha=0.2, gbeta=0.0)
    X = np.arange(H + 1) / H
    Y = np.arange(ny) / (ny - 1)
    c0, c1 = 0.7, -0.4
    c = c0 + c1 * Y
    T = 1 - X[None, :] + c[:, None] * X[None, :] * (X[None, :] - 1)
    o.set_state(T=T)
    mh, loc, _, _ = o.nusselt()
    err = max(np.abs(loc - (1 + c)).max(), abs(mh - (1 + c0 + c1 / 2)))
    return err <= 1e-12, f"max Nusselt error = {err:.3g}"


def eq112_conduction(make, Hs=(8, 16, 32), alpha=0.25):
    """Top-hot square conduction (Section 6.3.1, Eqs. 103-111) against the
    series solution Eq. 112: the error at fixed interior points falls at
    second order with the grid."""
    pts = [(0.25, 0.5), (0.5, 0.5), (0.75, 0.75), (0.5, 0.25)]

    def series(X, Y, terms=400):
        s = 0.0
        for n in range(1, terms + 1):
            s += ((-1) ** (n + 1) + 1) / n * math.sin(n * math.pi * X) * \
                 math.exp(n * math.pi * (Y - 1)) * (1 - math.exp(-2 * n * math.pi * Y)) / (1 - math.exp(-2 * n * math.pi))
        return 2 / math.pi * s

    errs = []
    for H in Hs:
        o = make(H + 1, H + 1, bc=(DIR, DIR, DIR, DIR), t_wall=(0, 0, 0, 1), t_init=0.0, nu=0.1,
                 alpha=alpha, gbeta=0.0)
        o.step(int(4 * H * H / alpha))
        T = o.fields()[3]
        e = max(abs(T[int(round(Y * H)), int(round(X * H))] - series(X, Y)) for X, Y in pts)
        errs.append(e)
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    return min(orders) >= 1.8, f"errors {['%.3g' % e for e in errs]}, orders {['%.3f' % p for p in orders]}"


def homogeneous_in_f(make, c=0.7):
    """With the Eq. 18 force taken with the pressure rho0 cs^2 and the
    non-equilibrium extrapolation walls (Eqs. 94, 96), the step is homogeneous
    of degree one in f: scaling the populations of a buoyant cavity with an
    obstacle by c scales every later population by c and leaves u and T as
    they were (the symmetry that mass renormalisation relies on)."""
    mask = np.zeros((20, 26), np.uint8)
    mask[8:12, 10:15] = 1
    kw = dict(nu=0.05, alpha=0.08, gbeta=5e-4, mask=mask)
    a, b = make(26, 20, **kw), make(26, 20, **kw)
    a.step(200)
    b.step(200)
    b.set_f(c * b.f())
    a.step(150)
    b.step(150)
    _, ua, va, Ta = a.fields()
    _, ub, vb, Tb = b.fields()
    du = max(np.abs(ua - ub).max(), np.abs(va - vb).max())
    dT = np.abs(Ta - Tb).max()
    df = np.abs(b.f() - c * a.f()).max()
    moving = np.abs(ua).max()
    ok = du <= 1e-15 and dT <= 1e-14 and df <= 1e-14 and moving > 1e-5
    return ok, f"max|du| = {du:.3g}, max|dT| = {dT:.3g}, max|f_b - c f_a| = {df:.3g} (max|u| = {moving:.3g})"


def nee_wall_moments(make, u_lid=0.04):
    """Non-equilibrium extrapolation (Eqs. 94, 96) rebuilds a wall node from
    its partner as f_eq(rho_f, u_w) + (f_f - f_eq(rho_f, u_f)): the rebuilt
    populations carry the partner's density and the wall's velocity, since the
    non-equilibrium part has no mass and no momentum.  Checked on every wall
    node of a buoyant cavity with a sliding lid and an obstacle (corners
    belong to the resting vertical walls)."""
    ny, nx = 20, 26
    mask = np.zeros((ny, nx), np.uint8)
    mask[8:12, 10:15] = 1
    o = make(nx, ny, bc=(DIR, DIR, ADI, MOV), u_lid=u_lid, mask=mask, nu=0.05, alpha=0.08, gbeta=5e-4)
    o.step(300)
    rho, u, v, _ = o.fields()
    kind, _, partner = o.classes()
    walls = np.nonzero(kind.ravel() == 1)[0]
    R, U, V = rho.ravel(), u.ravel(), v.ravel()
    drho = np.abs(R[walls] - R[partner.ravel()[walls]]).max()
    lid = walls[(walls // nx == ny - 1) & (walls % nx > 0) & (walls % nx < nx - 1)]
    uw = np.where(np.isin(walls, lid), u_lid, 0.0)
    du = max(np.abs(U[walls] - uw).max(), np.abs(V[walls]).max())
    flow = np.abs(u[kind == 0]).max()
    ok = drho <= 1e-14 and du <= 1e-15 and len(lid) == nx - 2 and flow > 1e-3
    return ok, f"max|rho_b - rho_f| = {drho:.3g}, max|u_b - u_w| = {du:.3g} over {len(walls)} wall nodes"


def residual_shear_wave(make, K=200):
    """Residual ||u^{n+K} - u^n|| / ||u^{n+K}|| of a decaying periodic shear
    wave u_x = A sin(k y): every node's velocity shrinks by the same factor
    g = exp(-nu k^2 K) over K steps (Eq. 15), so the residual is the closed
    form (1 - g)/g.  A residual without the square roots gives its square, one
    normalised by the earlier snapshot gives 1 - g."""
    L, nu, A = 64, 0.1, 1e-4
    o = make(3, L, bc=(PER, PER, PER, PER), nu=nu, alpha=0.1, gbeta=0.0)
    y = np.arange(L)
    o.set_state(u=np.tile(A * np.sin(2 * np.pi * y / L)[:, None], (1, 3)))
    o.step(300)  # the non-equilibrium part settles in a few relaxation times
    o.residual()  # snapshot at step 300
    o.step(K)
    r = o.residual()
    k = 2 * np.pi / L
    g = math.exp(-nu * k * k * K)
    want = (1 - g) / g
    rel = abs(r / want - 1)
    return rel <= 0.005, f"residual {r:.6g} against (1 - g)/g = {want:.6g} (rel. {rel:.3g})"


def residual_cavity_fluid_nodes(make, K=150):
    """Residual of a lid-driven buoyant cavity with an obstacle against the
    definition evaluated from two field snapshots over the fluid nodes only:
    wall nodes (the lid moves at u_lid, obstacle surfaces rest) take no part,
    so including them would change the denominator."""
    ny, nx = 24, 30
    mask = np.zeros((ny, nx), np.uint8)
    mask[9:14, 11:17] = 1
    o = make(nx, ny, bc=(DIR, DIR, ADI, MOV), u_lid=0.05, mask=mask, nu=0.06, alpha=0.08, gbeta=4e-4)
    o.step(100)
    o.residual()
    _, u0, v0, _ = o.fields()
    o.step(K)
    r = o.residual()
    _, u1, v1, _ = o.fields()
    fluid = o.classes()[0] == 0
    num = np.sum((u1 - u0)[fluid] ** 2 + (v1 - v0)[fluid] ** 2)
    den = np.sum(u1[fluid] ** 2 + v1[fluid] ** 2)
    want = math.sqrt(num) / math.sqrt(den)
    lid_share = np.sum(u1[~fluid] ** 2) / den
    rel = abs(r / want - 1)
    ok = rel <= 1e-12 and want > 1e-3 and lid_share > 1e-2
    return ok, f"residual {r:.9g} against {want:.9g} from two snapshots (rel. {rel:.3g}; walls would add {lid_share:.3g} of the denominator)"


# ---- D2Q5 thermal lattice Boltzmann energy solver (Section 2.4) ----

def lbm_conduction_linear(make, H=16):
    """D2Q5 energy populations, pure conduction between T = 1 and T = 0 with
    adiabatic top and bottom: the steady field is T = 1 - x/H to round-off
    (a linear profile has a uniform non-equilibrium part, which the
    extrapolation walls of Eq. 95 carry exactly) and Nu = 1."""
    o = make(H + 1, H + 1, nu=0.1, alpha=0.2, gbeta=0.0, energy="lbm")
    o.step(8000)
    T = o.fields()[3]
    x = np.arange(H + 1) / H
    err = np.abs(T - (1 - x)[None, :]).max()
    nh, _, nc, _ = o.nusselt()
    ok = err <= 1e-12 and abs(nh - 1) <= 1e-12 and abs(nc - 1) <= 1e-12
    return ok, f"max|T - (1 - x/H)| = {err:.3g}, Nu hot - 1 = {nh - 1:.3g}, Nu cold - 1 = {nc - 1:.3g}"


def lbm_thermal_decay(make, L=64, alpha=0.1):
    """A periodic temperature wave T = 1/2 + A sin(k y) at rest decays at the
    rate alpha k^2 with alpha = c_s^2 (tau_T - 1/2) (Eq. 20)."""
    o = make(3, L, bc=(PER, PER, PER, PER), nu=0.1, alpha=alpha, gbeta=0.0, energy="lbm")
    y = np.arange(L)
    k = 2 * np.pi / L
    o.set_state(T=np.tile((0.5 + 1e-3 * np.sin(k * y))[:, None], (1, 3)))
    amp = []
    for t in (300, 3000):
        o.step(t - o.step_count)
        T = o.fields()[3][:, 1]
        amp.append(2 / L * np.sum((T - 0.5) * np.sin(k * y)))
    rate = math.log(amp[0] / amp[1]) / 2700
    rel = abs(rate / (alpha * k * k) - 1)
    return rel <= 0.01, f"decay rate / (alpha k^2) - 1 = {rel:.3g}"


def lbm_thermal_advection(make, L=64, U=0.05, alpha=0.05, t=320):
    """A temperature wave on a uniform stream (U, 0) travels downstream at U
    (the e.u / c_s^2 term of Eq. 21)."""
    k = 2 * np.pi / L
    x = np.arange(L)
    o = make(L, 3, bc=(PER, PER, PER, PER), nu=0.05, alpha=alpha, gbeta=0.0, energy="lbm")
    o.set_state(u=np.full((3, L), U), T=np.tile((0.5 + 1e-3 * np.sin(k * x))[None, :], (3, 1)))
    o.step(t)
    T = o.fields()[3][1] - 0.5
    phase = math.atan2(-np.sum(T * np.cos(k * x)), np.sum(T * np.sin(k * x)))  # T ~ sin(k (x - c t))
    c = phase / (k * t)
    rel = abs(c / U - 1)
    return rel <= 0.02, f"phase speed / U - 1 = {rel:.3g}"


def lbm_thermal_conservation(make, steps=3000):
    """Periodic box with buoyant flow from a random temperature field: the
    D2Q5 collision and streaming conserve sum T = sum g to round-off."""
    rng = np.random.default_rng(11)
    o = make(24, 19, bc=(PER, PER, PER, PER), nu=0.08, alpha=0.1, gbeta=2e-4, t_ref=0.5, energy="lbm")
    o.set_state(T=rng.random((19, 24)))
    e0 = o.fields()[3].sum()
    o.step(100)
    flow = np.abs(o.fields()[1]).max()  # the buoyant flow at its strongest
    o.step(steps - 100)
    T = o.fields()[3]
    rel = abs(T.sum() - e0) / e0
    return rel <= 1e-11 and flow > 1e-5, f"relative change of sum T over {steps} steps = {rel:.3g}"


def lbm_thermal_walls(make):
    """Extrapolation walls of the energy populations (Eq. 95): Dirichlet wall
    nodes hold the wall temperature and adiabatic wall nodes and obstacle
    surfaces their partner's temperature, to round-off (the non-equilibrium
    part carries no energy)."""
    ny, nx = 22, 28
    mask = np.zeros((ny, nx), np.uint8)
    mask[8:13, 10:16] = 1
    o = make(nx, ny, mask=mask, nu=0.05, alpha=0.08, gbeta=5e-4, energy="lbm")
    o.step(400)
    _, _, _, T = o.fields()
    kind, therm, partner = o.classes()
    Tf, K, TH, P = T.ravel(), kind.ravel(), therm.ravel(), partner.ravel()
    walls = np.nonzero(K == 1)[0]
    dirichlet = walls[TH[walls] == 1]
    other = walls[TH[walls] != 1]
    want_d = np.where(dirichlet % nx == 0, 1.0, 0.0)
    d_err = np.abs(Tf[dirichlet] - want_d).max()
    o_err = np.abs(Tf[other] - Tf[P[other]]).max()
    moving = np.ptp(T[kind == 0]) > 0.1
    ok = d_err <= 1e-15 and o_err <= 1e-15 and len(other) > 2 * nx and moving
    return ok, f"Dirichlet walls off by {d_err:.3g}, adiabatic/obstacle walls off their partner by {o_err:.3g}"


# ---- finite-difference velocity-gradient walls (Section 3, Eqs. 61-72) ----

def fd_poiseuille(make, Hs=(8, 16, 32)):
    """Force-driven channel between finite-difference velocity-gradient
    walls: the parabolic profile u = g_x y (H - y) / (2 nu) at second order
    (the one-sided wall gradient is exact on a parabola, so the profile is
    closer than with extrapolation walls)."""
    errs = []
    for H in Hs:
        nu, umax = 0.1, 0.01
        fx = 8 * nu * umax / (H * H)
        o = make(4, H + 1, bc=(PER, PER, ADI, ADI), nu=nu, alpha=0.1, gbeta=0.0, fx=fx, wall_bc="fd")
        o.step(int(30 * H * H / nu) + 2000)
        u = o.fields()[1][:, 1]
        y = np.arange(H + 1)
        errs.append(np.sqrt(np.mean((u - fx * y * (H - y) / (2 * nu)) ** 2)) / umax)
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    ok = min(orders) >= 1.8 and errs[0] < 0.01
    return ok, f"errors {['%.3g' % e for e in errs]}, orders {['%.3f' % p for p in orders]}"


def fd_couette(make, H=16, U=0.02):
    """Plane Couette flow between a resting wall and a sliding lid, both
    finite-difference velocity-gradient walls: the linear profile is exact
    (its strain is uniform, and the wall nodes carry the interior's
    non-equilibrium part tau w_i / c_s^2 rho Q_i : S of Eq. 70)."""
    o = make(4, H + 1, bc=(PER, PER, ADI, MOV), u_lid=U, nu=0.1, alpha=0.1, gbeta=0.0, wall_bc="fd")
    o.step(20000)
    u = o.fields()[1][:, 1]
    err = np.abs(u - U * np.arange(H + 1) / H).max() / U
    return err <= 1e-11, f"max|u - U y/H| / U = {err:.3g}"


def fd_wall_moments(make, u_lid=0.04):
    """Finite-difference walls rebuild box-wall nodes with the partner's
    density (Eq. 96) and the wall velocity: Q_i : S carries no mass and no
    momentum (sum w_i Q_i = 0, sum w_i e_i Q_i = 0)."""
    ny, nx = 20, 26
    mask = np.zeros((ny, nx), np.uint8)
    mask[8:12, 10:15] = 1
    o = make(nx, ny, bc=(DIR, DIR, ADI, MOV), u_lid=u_lid, mask=mask, nu=0.05, alpha=0.08, gbeta=5e-4, wall_bc="fd")
    o.step(300)
    rho, u, v, _ = o.fields()
    kind, _, partner = o.classes()
    walls = np.nonzero(kind.ravel() == 1)[0]
    R, U, V = rho.ravel(), u.ravel(), v.ravel()
    drho = np.abs(R[walls] - R[partner.ravel()[walls]]).max()
    lid = walls[(walls // nx == ny - 1) & (walls % nx > 0) & (walls % nx < nx - 1)]
    uw = np.where(np.isin(walls, lid), u_lid, 0.0)
    du = max(np.abs(U[walls] - uw).max(), np.abs(V[walls]).max())
    ok = drho <= 1e-14 and du <= 1e-15 and np.abs(u[kind == 0]).max() > 1e-3
    return ok, f"max|rho_b - rho_f| = {drho:.3g}, max|u_b - u_w| = {du:.3g}"


# ---- grid setting 2 (Section 5.1, Fig. 30): coarse energy grid ----

def grid2_conduction_linear(make, H=16):
    """Grid setting 2, pure conduction: the coarse volumes and the nodes
    interpolated from them hold T = 1 - x/H to round-off (the half-volume
    wall distance and the two-point means are exact on a linear profile), and
    Nu = 1."""
    o = make(H + 1, H + 1, nu=0.1, alpha=0.2, gbeta=0.0, fv_grid=2, fv_every=2)
    o.step(20000)
    T = o.fields()[3]
    x = np.arange(H + 1) / H
    err = np.abs(T - (1 - x)[None, :]).max()
    nh = o.nusselt()[0]
    return err <= 1e-12 and abs(nh - 1) <= 1e-12, f"max|T - (1 - x/H)| = {err:.3g}, Nu - 1 = {nh - 1:.3g}"


def grid2_periodic_decay(make, L=32, alpha=0.1, k=4, n=40):
    """Grid setting 2 in a periodic box, a temperature wave along x at rest:
    each coarse step (volumes 2 apart, time step k) multiplies it by exactly
    g = 1 - alpha k (1 - cos(4 pi / L)) / 2, the discrete eigenvalue."""
    o = make(L, 4, bc=(PER, PER, PER, PER), nu=0.1, alpha=alpha, gbeta=0.0, fv_grid=2, fv_every=k)
    o.set_state(T=np.tile((0.5 + 1e-3 * np.sin(2 * np.pi * np.arange(L) / L))[None, :], (4, 1)))
    a0 = o.fields()[3][1, 1::2] - 0.5  # the volume centres
    o.step(n * k)
    a1 = o.fields()[3][1, 1::2] - 0.5
    g = 1 - alpha * k * (1 - math.cos(4 * math.pi / L)) / 2
    err = np.abs(a1 - a0 * g ** n).max() / np.abs(a0).max()
    return err <= 1e-11, f"max relative deviation from g^n = {err:.3g}"


def grid2_conservation(make, n=400):
    """Grid setting 2 in a box with adiabatic walls and buoyant flow: the
    conservative flux form keeps the coarse volumes' total energy (4 T per
    volume at the odd-odd centre nodes) to round-off."""
    ny, nx = 25, 33
    o = make(nx, ny, bc=(ADI, ADI, ADI, ADI), nu=0.06, alpha=0.1, gbeta=4e-4, t_ref=0.5, fv_grid=2, fv_every=2)
    o.set_state(T=np.random.default_rng(9).random((ny, nx)))
    e0 = o.fields()[3][1::2, 1::2].sum()
    o.step(60)
    flow = np.abs(o.fields()[1]).max()
    o.step(n - 60)
    rel = abs(o.fields()[3][1::2, 1::2].sum() - e0) / e0
    return rel <= 1e-12 and flow > 1e-4, f"relative change of the volumes' energy = {rel:.3g} (max|u| {flow:.3g})"


def grid2_same_steady_state(make, n=41):
    """Section 5.1: both grid settings reach the same results.  At Ra = 1e4
    the steady mean Nusselt number of setting 2 lies within 1 % of setting
    1's, and a coarse step every 4 lattice steps reaches the steady state of
    a step every lattice step (the steady balance has no time step in it)."""
    out = []
    for grid, k in ((1, 1), (2, 1), (2, 4)):
        U0 = 0.1
        H = n - 1
        o = make(n, n, nu=U0 * H * math.sqrt(0.71 / 1e4), alpha=U0 * H / math.sqrt(1e4 * 0.71), gbeta=U0 * U0 / H,
                 fv_grid=grid, fv_every=k)
        for _ in range(200):
            o.step(1000)
            if o.residual() < 1e-10:
                break
        out.append(o.nusselt()[0])
    d12, dk = abs(out[1] / out[0] - 1), abs(out[2] / out[1] - 1)
    return d12 <= 0.01 and dk <= 1e-7, f"Nu {out}: settings differ by {d12:.3g}, coarse steps by {dk:.3g}"


QUICK = {
    "rest_state": rest_state,
    "mass_periodic": lambda m: mass_periodic(m, 2000),
    "shear_wave": shear_wave,
    "advected_wave": advected_wave,
    "poiseuille": lambda m: poiseuille(m, (8, 16)),
    "conduction_linear": conduction_linear,
    "sine_mode_x": sine_mode_x,
    "cosine_mode_y": cosine_mode_y,
    "advected_temperature": advected_temperature,
    "energy_adiabatic": energy_adiabatic,
    "energy_adiabatic_obstacle": energy_adiabatic_obstacle,
    "uniform_buoyancy": uniform_buoyancy,
    "quick_advected_mode": quick_advected_mode,
    "quick_advected_mode_subcycled": lambda m: quick_advected_mode(m, n=100, substeps=2),
    "subcycled_sine_mode": subcycled_sine_mode,
    "quick_energy_adiabatic": lambda m: quick_energy_adiabatic(m, 300),
    "quadratic_nusselt": quadratic_nusselt,
    "homogeneous_in_f": homogeneous_in_f,
    "nee_wall_moments": nee_wall_moments,
    "residual_shear_wave": residual_shear_wave,
    "residual_cavity_fluid_nodes": residual_cavity_fluid_nodes,
    "lbm_conduction_linear": lbm_conduction_linear,
    "lbm_thermal_decay": lbm_thermal_decay,
    "lbm_thermal_advection": lbm_thermal_advection,
    "lbm_thermal_conservation": lambda m: lbm_thermal_conservation(m, 1000),
    "lbm_thermal_walls": lbm_thermal_walls,
    "fd_poiseuille": lambda m: fd_poiseuille(m, (8, 16)),
    "fd_couette": fd_couette,
    "fd_wall_moments": fd_wall_moments,
    "grid2_conduction_linear": grid2_conduction_linear,
    "grid2_periodic_decay": grid2_periodic_decay,
    "grid2_conservation": grid2_conservation,
}
