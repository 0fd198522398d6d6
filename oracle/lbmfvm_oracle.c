/*
 * FP64 CPU oracle for the hybrid LBM(velocity) + FVM(temperature) step of
 * Li, Yang & Zhang, "Hybrid LBM-FVM and LBM-MCM methods for fluid flow and
 * heat transfer simulation" (arXiv 1908.08386), Section 5.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may build, load or call it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * One time step n -> n+1 follows the paper's coupling order (Section 5: the
 * LBM gives velocity, then the temperature is solved by an energy balance
 * over each control volume with that velocity; the same order is drawn in the
 * LBM-MCM flowchart of Section 6.2):
 *   1. moments rho^n, u^n of f^n                        (Eqs. 16-17)
 *   2. BGK collision with the buoyancy term, using T^n   (Eqs. 5, 8, 18, 81)
 *   3. pull streaming into every fluid node              (Eq. 5)
 *   4. non-equilibrium extrapolation at wall nodes       (Eqs. 60, 94, 96)
 *   5. moments rho^{n+1}, u^{n+1}                        (Eqs. 16-17)
 *   6. explicit finite-volume energy balance over node-centred control
 *      volumes (grid setting 1, Fig. 29) with face velocities interpolated
 *      from u^{n+1} and T^n                             (Eq. 76 / Eq. 24)
 *
 * Readings of points the paper leaves open (listed with reasons in the
 * design notes):
 *   - Eq. 5's collision sign is read as relaxation toward equilibrium,
 *     f* = f - (f - f_eq)/tau + F  (as Eqs. 3 and 19 have it).
 *   - Eq. 18 with dt = 1 and its pressure read as the reference pressure
 *     rho0 cs^2 (rho0 = 1): F_i = G.(e_i - u) f_eq_i/(rho0 cs^2), whose
 *     momentum source rho G is the buoyancy force density of Eq. 75.  Every
 *     part of the step is then homogeneous of degree one in f, so the slow
 *     mass leak of the non-equilibrium extrapolation walls does not feed back
 *     into u or T.  u = sum(e f)/rho (Eq. 17), no half-force velocity shift.
 *   - Wall nodes collide like fluid nodes, with their own T in the force.
 *   - Pr = nu/alpha (Eq. 89's coefficient; Eq. 82 prints it inverted).
 *   - u_c = sqrt(g beta dT H) and Ma = u_c/c_s (Eq. 84), so U0 = Ma/sqrt(3).
 *   - FV: forward Euler with dt_FV = dt_LBM = 1, central face values,
 *     conservative flux form, face velocity = mean of the two node velocities.
 *   - Nodes: N nodes per side, H = ny - 1; vertical walls own the corners.
 *   - Obstacle wall nodes (solid nodes with a fluid 8-neighbour) take
 *     T^{n+1}(b) = T^n(x_f); faces to them carry no heat flux (adiabatic).
 *
 * Options of the energy update (orc_set_fv; off by default):
 *   - QUICK face values, the scheme Section 3.1 names for its finite-volume
 *     solver (Leonard's quadratic upstream interpolation): on a face with
 *     flow from U to D, T_f = 6/8 T_U + 3/8 T_D - 1/8 T_UU, UU the node
 *     beyond U; where UU takes no part in the energy balance (a wall, an
 *     obstacle, outside the box) the face keeps the central value.
 *   - Sub-cycling: m explicit sub-steps of dt/m per lattice step with the
 *     velocity u^{n+1} held, so that alpha up to m/4 stays inside the
 *     explicit diffusion limit; obstacle wall nodes copy their partner's
 *     temperature at every sub-step.
 *
 * Energy solver option (orc_set_energy; the finite-volume update is the
 * default): the D2Q5 thermal lattice-Boltzmann model of Section 2.4, the
 * paper's "LBM" comparison column.  Energy populations g_i (rest, E, N, W, S)
 * relax toward g_eq = T w_i (1 + e_i.u / c_s^2) (Eqs. 19, 21, weights of
 * Eq. 22) with tau_T = alpha / c_s^2 + 1/2 (Eq. 20), stream like f, and give
 * T = sum g (Eq. 23).  Wall nodes are rebuilt by non-equilibrium
 * extrapolation, g_b = g_eq(T_b, u_b) + g(x_f) - g_eq(T_f, u_f) (Eq. 95), with
 * T_b the wall temperature on Dirichlet sides and T_b = T(x_f) on adiabatic
 * sides and obstacle surfaces (zero normal gradient).  One step collides g
 * with T^n and u^n beside f, streams both, extrapolates both at walls, then
 * takes rho, u and T of the new step.
 *
 * Grid setting 2 (orc_set_grid2; grid setting 1 is the default): the
 * energy balance on the coarse grid of Section 5.1's second setting (Fig. 30):
 * for a lattice of 2NX x 2NY spacings, NX x NY control volumes of 2 x 2
 * spacings whose faces pass through lattice nodes, so the face velocities are
 * the lattice velocities at those nodes, with no interpolation.  The volumes'
 * centres are the odd-odd nodes.  The explicit update (central face values,
 * conservative flux form) runs every k lattice steps with the time step k;
 * a Dirichlet wall face lies half a volume from its centre, an adiabatic one
 * carries no flux.  The lattice nodes' temperature is interpolated from the
 * volumes (Section 5.1): the centre's value at a centre, the mean of the two
 * or four nearest centres elsewhere, the nearest volume's value at an
 * adiabatic or periodic-free side (zero gradient), the wall value on a
 * Dirichlet wall.  Between updates the nodes keep their temperature.
 *
 * Wall option (orc_set_wall_bc; extrapolation is the default): the
 * finite-difference velocity-gradient boundary of Section 3 (hybrid method
 * 2, Eqs. 61-72) on the box walls.  A box-wall node takes the first term of
 * the Chapman-Enskog expansion, f_b = f_eq(rho_b, u_b) - (tau w_i / c_s^2)
 * rho_b Q_i : S with Q_i = e_i e_i - c_s^2 I (Eqs. 67, 69-71), rho_b =
 * rho(x_f) (Eq. 96), u_b the wall velocity, and the strain rate S from
 * finite differences of the new velocity field: centred along the wall,
 * second-order one-sided (-3 u_0 + 4 u_1 - u_2)/2 into the fluid, and the
 * normal derivative of the normal velocity from continuity (Eq. 72; corners
 * keep both one-sided derivatives).  Obstacle surfaces keep the
 * extrapolation.
 *
 * D2Q9 numbering used here (results do not depend on it): 0 rest, 1 E, 2 N,
 * 3 W, 4 S, 5 NE, 6 NW, 7 SW, 8 SE.  Weights from Eq. 9, c_s^2 = 1/3.  The
 * D2Q5 set is the first five of these directions.
 *
 * Arrays are row-major [ny][nx] with x fastest and j = 0 the bottom row;
 * distributions are [9][ny][nx].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9
/* Threads pay off only on large grids; results never depend on it. */
#define PARALLEL(o) ((long)(o)->nx * (o)->ny >= 16384)

enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };
enum { BC_DIRICHLET = 0, BC_ADIABATIC = 1, BC_PERIODIC = 2, BC_MOVING = 3 };
enum { K_FLUID = 0, K_WALL = 1, K_SOLID = 2 };
enum { TH_FV = 0, TH_DIRICHLET = 1, TH_OBSTACLE = 2, TH_INERT = 3 };
enum { ENERGY_FV = 0, ENERGY_LBM = 1 };
enum { WALL_NEE = 0, WALL_FD = 1 };
#define Q5 5

static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* Eq. 9: 4/9 for the rest population, 1/9 for the axis ones, 1/36 diagonal. */
static const double W[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;
/* Eq. 22: 1/3 for the rest population of D2Q5, 1/6 for the four axis ones
 * (their second moment gives the same c_s^2 = 1/3). */
static const double W5[Q5] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0};
/* Reference density of the Boussinesq model: the p of Eq. 18 is read as the
 * reference pressure RHO0 cs^2, so the momentum source sum_i e_i F_i equals
 * rho G, the force density rho g beta (T - T_ref) of Eq. 75. */
static const double RHO0 = 1.0;

typedef struct {
    int nx, ny;
    int bc[4];
    double t_wall[4];
    double u_lid;
    double tau, alpha, gbeta, t_ref, fx, fy;
    unsigned char *kind;   /* K_* per node */
    unsigned char *therm;  /* TH_* per node */
    int *partner;          /* NEE partner node index (walls), else -1 */
    double *uw, *vw;       /* wall velocity per node */
    double *f;             /* f^n, post-stream [9][ny][nx] */
    double *fs;            /* post-collision scratch */
    double *T;             /* T^n */
    double *Tn;            /* scratch */
    double *rho, *ux, *uy; /* moments of f^n */
    double *su, *sv;       /* residual snapshot */
    int grid2;             /* energy balance on the coarse grid of setting 2 */
    int fv_every;          /* lattice steps per coarse energy step (k) */
    int ncx, ncy;          /* coarse volumes along x and y */
    double *Tc, *Tcn;      /* volume temperatures and scratch [ncy][ncx] */
    long step;
    int fv_quick;          /* QUICK face values instead of central ones */
    int fv_substeps;       /* explicit FV sub-steps per lattice step (>= 1) */
    int energy;            /* ENERGY_FV or ENERGY_LBM (D2Q5 populations) */
    int wall_bc;           /* WALL_NEE or WALL_FD on the box walls */
    double tau_T;          /* relaxation time of g (Eq. 20) */
    double *g, *gs;        /* D2Q5 populations [5][ny][nx] and post-collision scratch */
} orc_t;

static int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

/* Neighbour of (i, j) in direction (dx, dy), honouring periodic sides.
 * Returns -1 if it lies outside a non-periodic side. */
static int nbr(const orc_t *o, int i, int j, int dx, int dy) {
    int a = i + dx, b = j + dy;
    if (a < 0 || a >= o->nx) {
        if (o->bc[SIDE_W] != BC_PERIODIC) return -1;
        a = wrap(a, o->nx);
    }
    if (b < 0 || b >= o->ny) {
        if (o->bc[SIDE_S] != BC_PERIODIC) return -1;
        b = wrap(b, o->ny);
    }
    return b * o->nx + a;
}

/* Eq. 8 with c_s^2 = 1/3. */
static double feq(int q, double rho, double ux, double uy) {
    double eu = EX[q] * ux + EY[q] * uy;
    double uu = ux * ux + uy * uy;
    return rho * W[q] * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Eq. 21: D2Q5 equilibrium of the energy populations. */
static double geq(int q, double T, double ux, double uy) {
    return T * W5[q] * (1.0 + (EX[q] * ux + EY[q] * uy) / CS2);
}

/* Eqs. 16-17 at node k. */
static void moments(const orc_t *o, const double *f, long k, double *rho, double *ux, double *uy) {
    long n = (long)o->nx * o->ny;
    double r = 0, mx = 0, my = 0;
    for (int q = 0; q < Q; q++) {
        double v = f[q * n + k];
        r += v;
        mx += EX[q] * v;
        my += EY[q] * v;
    }
    *rho = r;
    *ux = mx / r;
    *uy = my / r;
}

void orc_destroy(orc_t *o) {
    if (!o) return;
    free(o->kind); free(o->therm); free(o->partner); free(o->uw); free(o->vw);
    free(o->f); free(o->fs); free(o->T); free(o->Tn);
    free(o->rho); free(o->ux); free(o->uy); free(o->su); free(o->sv);
    free(o->g); free(o->gs);
    free(o->Tc); free(o->Tcn);
    free(o);
}

/* Lattice parameters from the nondimensional groups (Eqs. 83-89, 15).
 * U0 = Ma/sqrt(3) (Eq. 84 with c_s = 1/sqrt(3)); the momentum diffusion
 * coefficient of Eq. 87 is U0 sqrt(Pr/Ra) in units of H and U0, the thermal one
 * of Eq. 89 is U0/sqrt(Ra Pr), and the buoyancy coefficient of Eq. 88 gives
 * g beta dT = U0^2/H. */
void orc_params_from_groups(double Ra, double Pr, double Ma, double H, double dT,
                            double *nu, double *alpha, double *gbeta, double *tau) {
    double U0 = Ma / sqrt(3.0);
    *nu = U0 * H * sqrt(Pr / Ra);
    *alpha = U0 * H / sqrt(Ra * Pr);
    *gbeta = U0 * U0 / (H * dT);
    *tau = *nu / CS2 + 0.5;
}

static int on_side(const orc_t *o, int i, int j, int s) {
    if (s == SIDE_W) return o->bc[SIDE_W] != BC_PERIODIC && i == 0;
    if (s == SIDE_E) return o->bc[SIDE_E] != BC_PERIODIC && i == o->nx - 1;
    if (s == SIDE_S) return o->bc[SIDE_S] != BC_PERIODIC && j == 0;
    return o->bc[SIDE_N] != BC_PERIODIC && j == o->ny - 1;
}

/* Node classes.  mask: 1 = solid (may be NULL).
 * Box-border nodes of non-periodic sides are wall nodes; the partner x_f is
 * the inward normal neighbour (the inward diagonal at corners).  Solid nodes
 * with a fluid 8-neighbour are obstacle wall nodes whose partner is the first
 * fluid neighbour in the order E, N, W, S, NE, NW, SW, SE.  A wall node whose
 * preferred partner is not fluid falls back to the same ordered search; with
 * no fluid neighbour at all it is inert. */
static void classify(orc_t *o, const unsigned char *mask) {
    int nx = o->nx, ny = o->ny;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long k = (long)j * nx + i;
            int border = on_side(o, i, j, SIDE_W) || on_side(o, i, j, SIDE_E) ||
                         on_side(o, i, j, SIDE_S) || on_side(o, i, j, SIDE_N);
            int solid = mask && mask[k];
            o->kind[k] = (solid || border) ? K_WALL : K_FLUID;
            o->partner[k] = -1;
            o->uw[k] = 0.0;
            o->vw[k] = 0.0;
        }
    /* partners */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long k = (long)j * nx + i;
            if (o->kind[k] != K_WALL) continue;
            int solid = mask && mask[k];
            int p = -1;
            if (!solid) {
                int dx = 0, dy = 0;
                if (on_side(o, i, j, SIDE_W)) dx = 1;
                if (on_side(o, i, j, SIDE_E)) dx = -1;
                if (on_side(o, i, j, SIDE_S)) dy = 1;
                if (on_side(o, i, j, SIDE_N)) dy = -1;
                int c = nbr(o, i, j, dx, dy);
                if (c >= 0 && o->kind[c] == K_FLUID) p = c;
            }
            for (int q = 1; q < Q && p < 0; q++) {
                int c = nbr(o, i, j, EX[q], EY[q]);
                if (c >= 0 && o->kind[c] == K_FLUID) p = c;
            }
            o->partner[k] = p;
        }
    for (long k = 0; k < (long)nx * ny; k++)
        if (o->kind[k] == K_WALL && o->partner[k] < 0) o->kind[k] = K_SOLID;

    /* wall velocities (moving sides slide tangentially; vertical walls own corners) */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long k = (long)j * nx + i;
            if (o->kind[k] != K_WALL || (mask && mask[k])) continue;
            int vert = on_side(o, i, j, SIDE_W) ? SIDE_W : on_side(o, i, j, SIDE_E) ? SIDE_E : -1;
            int hor = on_side(o, i, j, SIDE_S) ? SIDE_S : on_side(o, i, j, SIDE_N) ? SIDE_N : -1;
            if (vert >= 0) {
                if (o->bc[vert] == BC_MOVING) o->vw[k] = o->u_lid;
            } else if (hor >= 0) {
                if (o->bc[hor] == BC_MOVING) o->uw[k] = o->u_lid;
            }
        }

    /* thermal roles */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long k = (long)j * nx + i;
            if (o->kind[k] == K_SOLID) { o->therm[k] = TH_INERT; continue; }
            if (mask && mask[k]) { o->therm[k] = TH_OBSTACLE; continue; }
            int vert = on_side(o, i, j, SIDE_W) ? SIDE_W : on_side(o, i, j, SIDE_E) ? SIDE_E : -1;
            int hor = on_side(o, i, j, SIDE_S) ? SIDE_S : on_side(o, i, j, SIDE_N) ? SIDE_N : -1;
            if (vert >= 0 && o->bc[vert] == BC_DIRICHLET) o->therm[k] = TH_DIRICHLET;
            else if (hor >= 0 && o->bc[hor] == BC_DIRICHLET) o->therm[k] = TH_DIRICHLET;
            else o->therm[k] = TH_FV;
        }
}

static double dirichlet_value(const orc_t *o, int i, int j) {
    if (on_side(o, i, j, SIDE_W) && o->bc[SIDE_W] == BC_DIRICHLET) return o->t_wall[SIDE_W];
    if (on_side(o, i, j, SIDE_E) && o->bc[SIDE_E] == BC_DIRICHLET) return o->t_wall[SIDE_E];
    if (on_side(o, i, j, SIDE_S) && o->bc[SIDE_S] == BC_DIRICHLET) return o->t_wall[SIDE_S];
    return o->t_wall[SIDE_N];
}

static void compute_moments(orc_t *o) {
    int nx = o->nx, ny = o->ny;
#pragma omp parallel for schedule(static) if (PARALLEL(o))
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long k = (long)j * nx + i;
            if (o->kind[k] == K_SOLID) {
                o->rho[k] = 0.0; o->ux[k] = 0.0; o->uy[k] = 0.0;
                continue;
            }
            moments(o, o->f, k, &o->rho[k], &o->ux[k], &o->uy[k]);
        }
}

static void grid2_to_nodes(orc_t *o);

/* Energy populations at equilibrium with the current T and u (Eq. 21);
 * inert nodes hold none. */
static void init_g(orc_t *o) {
    long n = (long)o->nx * o->ny;
    for (long k = 0; k < n; k++)
        for (int q = 0; q < Q5; q++)
            o->g[q * n + k] = (o->kind[k] == K_SOLID) ? 0.0 : geq(q, o->T[k], o->ux[k], o->uy[k]);
}

/* Initial state: f = f_eq(1, u0) at every non-inert node (Eq. 8), T = T0 with
 * Dirichlet nodes set to their wall value.  u0, v0, T0 may be NULL (rest, t_init). */
int orc_set_state(orc_t *o, const double *u0, const double *v0, const double *T0, double t_init) {
    int nx = o->nx, ny = o->ny;
    long n = (long)nx * ny;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long k = (long)j * nx + i;
            double u = u0 ? u0[k] : 0.0, v = v0 ? v0[k] : 0.0;
            for (int q = 0; q < Q; q++)
                o->f[q * n + k] = (o->kind[k] == K_SOLID) ? 0.0 : feq(q, 1.0, u, v);
            double t = T0 ? T0[k] : t_init;
            if (o->therm[k] == TH_DIRICHLET) t = dirichlet_value(o, i, j);
            o->T[k] = t;
        }
    o->step = 0;
    compute_moments(o);
    for (long k = 0; k < n; k++) { o->su[k] = o->ux[k]; o->sv[k] = o->uy[k]; }
    if (o->g) init_g(o);
    if (o->grid2) {
        for (int J = 0; J < o->ncy; J++)
            for (int I = 0; I < o->ncx; I++)
                o->Tc[(long)J * o->ncx + I] = o->T[(long)(2 * J + 1) * o->nx + 2 * I + 1];
        grid2_to_nodes(o);
    }
    return 0;
}

orc_t *orc_create(int nx, int ny, const int bc[4], const double t_wall[4], double u_lid,
                  double t_init, const unsigned char *mask, double nu, double alpha, double gbeta,
                  double t_ref, double fx, double fy) {
    if (nx < 3 || ny < 3) return NULL;
    if ((bc[SIDE_W] == BC_PERIODIC) != (bc[SIDE_E] == BC_PERIODIC)) return NULL;
    if ((bc[SIDE_S] == BC_PERIODIC) != (bc[SIDE_N] == BC_PERIODIC)) return NULL;
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    if (!o) return NULL;
    o->nx = nx; o->ny = ny;
    memcpy(o->bc, bc, sizeof(o->bc));
    memcpy(o->t_wall, t_wall, sizeof(o->t_wall));
    o->u_lid = u_lid;
    o->tau = nu / CS2 + 0.5; /* Eq. 15 with dt = 1 */
    o->alpha = alpha;
    o->gbeta = gbeta;
    o->t_ref = t_ref;
    o->fx = fx; o->fy = fy;
    long n = (long)nx * ny;
    o->kind = (unsigned char *)calloc(n, 1);
    o->therm = (unsigned char *)calloc(n, 1);
    o->partner = (int *)calloc(n, sizeof(int));
    o->uw = (double *)calloc(n, sizeof(double));
    o->vw = (double *)calloc(n, sizeof(double));
    o->f = (double *)calloc(Q * n, sizeof(double));
    o->fs = (double *)calloc(Q * n, sizeof(double));
    o->T = (double *)calloc(n, sizeof(double));
    o->Tn = (double *)calloc(n, sizeof(double));
    o->rho = (double *)calloc(n, sizeof(double));
    o->ux = (double *)calloc(n, sizeof(double));
    o->uy = (double *)calloc(n, sizeof(double));
    o->su = (double *)calloc(n, sizeof(double));
    o->sv = (double *)calloc(n, sizeof(double));
    if (!o->kind || !o->therm || !o->partner || !o->uw || !o->vw || !o->f || !o->fs || !o->T ||
        !o->Tn || !o->rho || !o->ux || !o->uy || !o->su || !o->sv) {
        orc_destroy(o);
        return NULL;
    }
    o->fv_quick = 0;
    o->fv_substeps = 1;
    classify(o, mask);
    orc_set_state(o, NULL, NULL, NULL, t_init);
    return o;
}

/* Energy solver: ENERGY_FV (0, the finite-volume update) or ENERGY_LBM (1,
 * the D2Q5 thermal lattice Boltzmann model).  Switching to LBM sets g to the
 * equilibrium of the current T and u.  Returns -1 for another mode or when
 * the populations cannot be allocated. */
int orc_set_energy(orc_t *o, int mode) {
    if (mode != ENERGY_FV && mode != ENERGY_LBM) return -1;
    if (mode == ENERGY_LBM && !o->g) {
        long n = (long)o->nx * o->ny;
        o->g = (double *)calloc(Q5 * n, sizeof(double));
        o->gs = (double *)calloc(Q5 * n, sizeof(double));
        if (!o->g || !o->gs) {
            free(o->g); free(o->gs);
            o->g = o->gs = NULL;
            return -1;
        }
    }
    o->energy = mode;
    o->tau_T = o->alpha / CS2 + 0.5; /* Eq. 20 with dt = 1 */
    if (mode == ENERGY_LBM) init_g(o);
    return 0;
}

/* Box-wall treatment: WALL_NEE (0, extrapolation) or WALL_FD (1, the
 * finite-difference velocity-gradient scheme).  Returns -1 for another mode. */
int orc_set_wall_bc(orc_t *o, int mode) {
    if (mode != WALL_NEE && mode != WALL_FD) return -1;
    o->wall_bc = mode;
    return 0;
}

/* Velocity of node (i, j) in the state being built: wall nodes move with the
 * wall, fluid nodes from their streamed populations, inert nodes rest. */
static void vel_at(const orc_t *o, int i, int j, double *u, double *v) {
    long k = (long)j * o->nx + i;
    if (o->kind[k] == K_WALL) { *u = o->uw[k]; *v = o->vw[k]; return; }
    if (o->kind[k] == K_SOLID) { *u = 0.0; *v = 0.0; return; }
    double r;
    moments(o, o->f, k, &r, u, v);
}

/* d(u, v)/d(axis) at (i, j): second-order one-sided into the domain at a
 * non-periodic box side, centred elsewhere. */
static void grad_at(const orc_t *o, int i, int j, int axis, double *du, double *dv) {
    int lo = axis == 0 ? on_side(o, i, j, SIDE_W) : on_side(o, i, j, SIDE_S);
    int hi = axis == 0 ? on_side(o, i, j, SIDE_E) : on_side(o, i, j, SIDE_N);
    int dx = axis == 0, dy = axis == 1;
    double u0, v0, u1, v1, u2, v2;
    if (lo || hi) {
        int s = lo ? 1 : -1;
        vel_at(o, i, j, &u0, &v0);
        vel_at(o, i + s * dx, j + s * dy, &u1, &v1);
        vel_at(o, i + 2 * s * dx, j + 2 * s * dy, &u2, &v2);
        *du = s * (-3.0 * u0 + 4.0 * u1 - u2) / 2.0;
        *dv = s * (-3.0 * v0 + 4.0 * v1 - v2) / 2.0;
    } else {
        int p = nbr(o, i, j, dx, dy), m = nbr(o, i, j, -dx, -dy);
        vel_at(o, p % o->nx, p / o->nx, &u1, &v1);
        vel_at(o, m % o->nx, m / o->nx, &u2, &v2);
        *du = (u1 - u2) / 2.0;
        *dv = (v1 - v2) / 2.0;
    }
}

/* Node temperatures from the volumes of grid setting 2 (see the header). */
static void grid2_to_nodes(orc_t *o) {
    int nx = o->nx, ny = o->ny, cx = o->ncx, cy = o->ncy;
    int perx = o->bc[SIDE_W] == BC_PERIODIC, pery = o->bc[SIDE_S] == BC_PERIODIC;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long k = (long)j * nx + i;
            if (o->therm[k] == TH_DIRICHLET) { o->T[k] = dirichlet_value(o, i, j); continue; }
            /* volumes (and weights) along each axis: centres at odd nodes */
            int ia[2], ja[2], ni, nj;
            if (i % 2) { ia[0] = (i - 1) / 2; ni = 1; }
            else if (perx) { ia[0] = (i / 2 + cx - 1) % cx; ia[1] = (i / 2) % cx; ni = 2; }
            else if (i == 0) { ia[0] = 0; ni = 1; }
            else if (i == nx - 1) { ia[0] = cx - 1; ni = 1; }
            else { ia[0] = i / 2 - 1; ia[1] = i / 2; ni = 2; }
            if (j % 2) { ja[0] = (j - 1) / 2; nj = 1; }
            else if (pery) { ja[0] = (j / 2 + cy - 1) % cy; ja[1] = (j / 2) % cy; nj = 2; }
            else if (j == 0) { ja[0] = 0; nj = 1; }
            else if (j == ny - 1) { ja[0] = cy - 1; nj = 1; }
            else { ja[0] = j / 2 - 1; ja[1] = j / 2; nj = 2; }
            double t = 0.0;
            for (int b = 0; b < nj; b++)
                for (int a = 0; a < ni; a++) t += o->Tc[(long)ja[b] * cx + ia[a]];
            o->T[k] = t / (ni * nj);
        }
}

/* Grid setting 2 with a coarse energy step every k >= 1 lattice steps.  The
 * lattice must span an even number of spacings along each walled axis (an
 * even number of nodes along a periodic one) and hold no obstacle.  The
 * volumes start from the node temperatures at their centres.  Returns -1
 * (nothing changed) otherwise. */
int orc_set_grid2(orc_t *o, int k) {
    if (k < 1 || o->energy != ENERGY_FV) return -1;
    int perx = o->bc[SIDE_W] == BC_PERIODIC, pery = o->bc[SIDE_S] == BC_PERIODIC;
    if ((perx ? o->nx : o->nx - 1) % 2 || (pery ? o->ny : o->ny - 1) % 2) return -1;
    for (long n = 0; n < (long)o->nx * o->ny; n++)
        if (o->therm[n] == TH_OBSTACLE || o->therm[n] == TH_INERT) return -1;
    o->ncx = perx ? o->nx / 2 : (o->nx - 1) / 2;
    o->ncy = pery ? o->ny / 2 : (o->ny - 1) / 2;
    long m = (long)o->ncx * o->ncy;
    free(o->Tc); free(o->Tcn);
    o->Tc = (double *)calloc(m, sizeof(double));
    o->Tcn = (double *)calloc(m, sizeof(double));
    if (!o->Tc || !o->Tcn) return -1;
    for (int J = 0; J < o->ncy; J++)
        for (int I = 0; I < o->ncx; I++) o->Tc[(long)J * o->ncx + I] = o->T[(long)(2 * J + 1) * o->nx + 2 * I + 1];
    o->grid2 = 1;
    o->fv_every = k;
    grid2_to_nodes(o);
    return 0;
}

/* One explicit energy step of grid setting 2 (time step k) with the current
 * lattice velocities: V (T' - T) = k sum over faces of [-F_f T_f + alpha A_f
 * (T_nb - T_P) / d], V = 4, A = 2, d = 2 between volumes and 1 to a
 * Dirichlet wall face; F_f = A u_face.n with u_face the lattice velocity at
 * the face's middle node; T_f the mean of the two volumes. */
static void grid2_step(orc_t *o) {
    int cx = o->ncx, cy = o->ncy, nx = o->nx;
    int per[2] = {o->bc[SIDE_W] == BC_PERIODIC, o->bc[SIDE_S] == BC_PERIODIC};
    const double dt = o->fv_every, V = 4.0, A = 2.0, alpha = o->alpha;
    static const int FD[4][2] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}};
    static const int SIDE[4] = {SIDE_E, SIDE_N, SIDE_W, SIDE_S};
    for (int J = 0; J < cy; J++)
        for (int I = 0; I < cx; I++) {
            double TP = o->Tc[(long)J * cx + I], acc = 0.0;
            int ci = 2 * I + 1, cj = 2 * J + 1;
            for (int f = 0; f < 4; f++) {
                int dx = FD[f][0], dy = FD[f][1];
                /* the face's middle node, one node from the centre */
                int fi = ci + dx, fj = cj + dy;
                if (per[0]) fi = wrap(fi, nx);
                if (per[1]) fj = wrap(fj, o->ny);
                long kf = (long)fj * nx + fi;
                double un = o->ux[kf] * dx + o->uy[kf] * dy;
                int In = I + dx, Jn = J + dy;
                int inside = 1;
                if (In < 0 || In >= cx) { if (per[0]) In = wrap(In, cx); else inside = 0; }
                if (Jn < 0 || Jn >= cy) { if (per[1]) Jn = wrap(Jn, cy); else inside = 0; }
                if (inside) {
                    double Tn = o->Tc[(long)Jn * cx + In];
                    acc += -A * un * 0.5 * (TP + Tn) + alpha * A * (Tn - TP) / 2.0;
                } else if (o->bc[SIDE[f]] == BC_DIRICHLET) {
                    acc += alpha * A * (o->t_wall[SIDE[f]] - TP) / 1.0;
                }
            }
            o->Tcn[(long)J * cx + I] = TP + dt * acc / V;
        }
    double *t = o->Tc; o->Tc = o->Tcn; o->Tcn = t;
}

/* Energy-update options: quick = 1 for QUICK face values, substeps >= 1.
 * Returns -1 (nothing changed) for substeps < 1. */
int orc_set_fv(orc_t *o, int quick, int substeps) {
    if (substeps < 1) return -1;
    o->fv_quick = quick != 0;
    o->fv_substeps = substeps;
    return 0;
}

/* Control-volume extent of node (i, j) along x or y: the node-centred cell
 * [i - 1/2, i + 1/2] clipped to the box (periodic sides do not clip). */
static double extent_x(const orc_t *o, int i) {
    if (o->bc[SIDE_W] == BC_PERIODIC) return 1.0;
    return 0.5 * (i > 0) + 0.5 * (i < o->nx - 1);
}
static double extent_y(const orc_t *o, int j) {
    if (o->bc[SIDE_S] == BC_PERIODIC) return 1.0;
    return 0.5 * (j > 0) + 0.5 * (j < o->ny - 1);
}

static int fv_member(const orc_t *o, int k) {
    return k >= 0 && (o->therm[k] == TH_FV || o->therm[k] == TH_DIRICHLET);
}

/* One full coupled step n -> n+1. */
static void step_once(orc_t *o) {
    int nx = o->nx, ny = o->ny;
    long n = (long)nx * ny;
    const double tau = o->tau, alpha = o->alpha;

    /* 1. moments of f^n are current in rho/ux/uy (kept up to date by step 5). */

    /* 2. collision with the buoyancy force G = (fx, fy + g beta (T^n - T_ref))
     *    (Eq. 81 with gravity along -y), Eq. 18 forcing, Eq. 5 update. */
#pragma omp parallel for schedule(static) if (PARALLEL(o))
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long k = (long)j * nx + i;
            if (o->kind[k] == K_SOLID) continue;
            double rho = o->rho[k], ux = o->ux[k], uy = o->uy[k];
            double Gx = o->fx;
            double Gy = o->fy + o->gbeta * (o->T[k] - o->t_ref);
            for (int q = 0; q < Q; q++) {
                double fe = feq(q, rho, ux, uy);
                double F = (Gx * (EX[q] - ux) + Gy * (EY[q] - uy)) * fe / (RHO0 * CS2);
                double fv = o->f[q * n + k];
                o->fs[q * n + k] = fv - (fv - fe) / tau + F;
            }
        }

    /* 2b. D2Q5 energy populations (Eq. 19): relaxation toward g_eq(T^n, u^n)
     *     (Eq. 21) with tau_T (Eq. 20). */
    if (o->energy == ENERGY_LBM) {
        const double tau_T = o->tau_T;
#pragma omp parallel for schedule(static) if (PARALLEL(o))
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long k = (long)j * nx + i;
                if (o->kind[k] == K_SOLID) continue;
                for (int q = 0; q < Q5; q++) {
                    double gv = o->g[q * n + k];
                    o->gs[q * n + k] = gv - (gv - geq(q, o->T[k], o->ux[k], o->uy[k])) / tau_T;
                }
            }
    }

    /* 3. pull streaming into fluid nodes: f_q(x) = f*_q(x - e_q). */
#pragma omp parallel for schedule(static) if (PARALLEL(o))
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long k = (long)j * nx + i;
            if (o->kind[k] != K_FLUID) continue;
            for (int q = 0; q < Q; q++) {
                int s = nbr(o, i, j, -EX[q], -EY[q]);
                o->f[q * n + k] = o->fs[q * n + s];
            }
        }

    /* 3b. pull streaming of the energy populations into fluid nodes. */
    if (o->energy == ENERGY_LBM) {
#pragma omp parallel for schedule(static) if (PARALLEL(o))
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long k = (long)j * nx + i;
                if (o->kind[k] != K_FLUID) continue;
                for (int q = 0; q < Q5; q++) {
                    int s = nbr(o, i, j, -EX[q], -EY[q]);
                    o->g[q * n + k] = o->gs[q * n + s];
                }
            }
    }

    /* 4. non-equilibrium extrapolation (Eq. 94 with rho_b = rho(x_f), Eq. 96):
     *    f_b = f_eq(rho_f, u_wall) + f(x_f) - f_eq(rho_f, u_f). */
#pragma omp parallel for schedule(static) if (PARALLEL(o))
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long k = (long)j * nx + i;
            if (o->kind[k] != K_WALL) continue;
            long p = o->partner[k];
            double rf, uf, vf;
            moments(o, o->f, p, &rf, &uf, &vf);
            for (int q = 0; q < Q; q++)
                o->f[q * n + k] = feq(q, rf, o->uw[k], o->vw[k]) + o->f[q * n + p] - feq(q, rf, uf, vf);
        }

    /* 4a. finite-difference velocity-gradient walls (Eqs. 67, 69-72) on the
     *     box walls in place of the extrapolation: f_b = f_eq(rho_f, u_w)
     *     - (tau w_i / c_s^2) rho_f Q_i : S.  The strain rate uses the new
     *     velocities of fluid nodes and the wall velocity of wall nodes. */
    if (o->wall_bc == WALL_FD) {
#pragma omp parallel for schedule(static) if (PARALLEL(o))
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long k = (long)j * nx + i;
                if (o->kind[k] != K_WALL || o->therm[k] == TH_OBSTACLE) continue;
                int vert = on_side(o, i, j, SIDE_W) || on_side(o, i, j, SIDE_E);
                int hor = on_side(o, i, j, SIDE_S) || on_side(o, i, j, SIDE_N);
                if (!vert && !hor) continue;
                double dudx, dvdx, dudy, dvdy;
                grad_at(o, i, j, 0, &dudx, &dvdx);
                grad_at(o, i, j, 1, &dudy, &dvdy);
                if (vert && !hor) dudx = -dvdy; /* Eq. 72 */
                if (hor && !vert) dvdy = -dudx;
                double sxx = dudx, syy = dvdy, sxy = 0.5 * (dudy + dvdx);
                double rf, uf, vf;
                moments(o, o->f, o->partner[k], &rf, &uf, &vf);
                for (int q = 0; q < Q; q++) {
                    double qs = (EX[q] * EX[q] - CS2) * sxx + 2.0 * EX[q] * EY[q] * sxy + (EY[q] * EY[q] - CS2) * syy;
                    o->f[q * n + k] = feq(q, rf, o->uw[k], o->vw[k]) - tau * W[q] / CS2 * rf * qs;
                }
            }
    }

    /* 4b. thermal non-equilibrium extrapolation (Eq. 95):
     *     g_b = g_eq(T_b, u_b) + g(x_f) - g_eq(T_f, u_f), with T_b the wall
     *     temperature on Dirichlet sides and T_f on adiabatic sides and
     *     obstacle surfaces. */
    if (o->energy == ENERGY_LBM) {
#pragma omp parallel for schedule(static) if (PARALLEL(o))
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long k = (long)j * nx + i;
                if (o->kind[k] != K_WALL) continue;
                long p = o->partner[k];
                double rf, uf, vf, Tf = 0.0;
                moments(o, o->f, p, &rf, &uf, &vf);
                for (int q = 0; q < Q5; q++) Tf += o->g[q * n + p];
                double Tb = o->therm[k] == TH_DIRICHLET ? dirichlet_value(o, i, j) : Tf;
                for (int q = 0; q < Q5; q++)
                    o->g[q * n + k] = geq(q, Tb, o->uw[k], o->vw[k]) + o->g[q * n + p] - geq(q, Tf, uf, vf);
            }
    }

    /* 5. moments of f^{n+1}. */
    compute_moments(o);

    /* 6. explicit FV energy balance on node-centred control volumes:
     *    V_P (T^{n+1} - T^n) = sum over open faces of
     *        -F_f T_f + alpha A_f (T_nb - T_P),
     *    F_f = A_f u_face.n_out, u_face = (u_P + u_nb)/2, T_f = (T_P + T_nb)/2
     *    (or the QUICK value, see the header).
     *    A face is open when both sides take part in the FV balance; box walls
     *    and faces to obstacle/inert nodes carry no flux.  With m sub-steps
     *    the balance is applied m times with dt = 1/m. */
    /* 6 (grid setting 2).  Every k-th step the coarse energy step with the
     *     new velocity, then the node temperatures from the volumes. */
    if (o->grid2) {
        if ((o->step + 1) % o->fv_every == 0) {
            grid2_step(o);
            grid2_to_nodes(o);
        }
        o->step++;
        return;
    }

    /* 6 (D2Q5). T^{n+1} = sum g (Eq. 23) at every node that holds
     *     populations; inert nodes keep T. */
    if (o->energy == ENERGY_LBM) {
        for (long k = 0; k < n; k++) {
            if (o->kind[k] == K_SOLID) continue;
            double t = 0.0;
            for (int q = 0; q < Q5; q++) t += o->g[q * n + k];
            o->T[k] = t;
        }
        o->step++;
        return;
    }

    const int m_sub = o->fv_substeps;
    const double dt = 1.0 / m_sub;
    for (int sub = 0; sub < m_sub; sub++) {
        if (sub > 0) { double *t = o->T; o->T = o->Tn; o->Tn = t; }
#pragma omp parallel for schedule(static) if (PARALLEL(o))
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long k = (long)j * nx + i;
                int th = o->therm[k];
                if (th == TH_FV) {
                    double ex = extent_x(o, i), ey = extent_y(o, j);
                    double V = ex * ey, TP = o->T[k], acc = 0.0;
                    /* faces E, N, W, S: outward normal (nx_, ny_), area */
                    static const int FD[4][2] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}};
                    for (int fc = 0; fc < 4; fc++) {
                        int dx = FD[fc][0], dy = FD[fc][1];
                        int mm = nbr(o, i, j, dx, dy);
                        if (!fv_member(o, mm)) continue;
                        double A = (dx != 0) ? ey : ex;
                        double un = 0.5 * ((o->ux[k] + o->ux[mm]) * dx + (o->uy[k] + o->uy[mm]) * dy);
                        double Fl = A * un;
                        double Tf = 0.5 * (TP + o->T[mm]);
                        if (o->fv_quick) {
                            /* upstream node U, downstream D, and UU beyond U */
                            int up, down, far;
                            if (un >= 0.0) {
                                up = (int)k; down = mm; far = nbr(o, i, j, -dx, -dy);
                            } else {
                                up = mm; down = (int)k; far = nbr(o, i + dx, j + dy, dx, dy);
                            }
                            if (fv_member(o, far))
                                Tf = 0.75 * o->T[up] + 0.375 * o->T[down] - 0.125 * o->T[far];
                        }
                        acc += -Fl * Tf + alpha * A * (o->T[mm] - TP);
                    }
                    o->Tn[k] = TP + dt * acc / V;
                } else if (th == TH_OBSTACLE) {
                    o->Tn[k] = o->T[o->partner[k]];
                } else {
                    o->Tn[k] = o->T[k]; /* Dirichlet value held, inert unchanged */
                }
            }
    }
    double *t = o->T; o->T = o->Tn; o->Tn = t;
    o->step++;
}

void orc_step(orc_t *o, long nsteps) {
    for (long s = 0; s < nsteps; s++) step_once(o);
}

long orc_step_count(const orc_t *o) { return o->step; }
double orc_tau(const orc_t *o) { return o->tau; }

/* Macroscopic fields of the current state (any pointer may be NULL).
 * Inert nodes report rho = u = v = 0. */
void orc_fields(const orc_t *o, double *rho, double *u, double *v, double *T) {
    long n = (long)o->nx * o->ny;
    for (long k = 0; k < n; k++) {
        if (rho) rho[k] = o->rho[k];
        if (u) u[k] = o->ux[k];
        if (v) v[k] = o->uy[k];
        if (T) T[k] = o->T[k];
    }
}

void orc_get_f(const orc_t *o, double *f) { memcpy(f, o->f, sizeof(double) * Q * o->nx * o->ny); }

/* Replace the post-stream populations of the current state (Q planes of
 * ny*nx, the layout of orc_get_f); T, the step count and the residual
 * snapshot stay.  For tests of properties of the step as a map of f. */
void orc_set_f(orc_t *o, const double *f) {
    memcpy(o->f, f, sizeof(double) * Q * o->nx * o->ny);
    compute_moments(o);
}

/* Replace the temperature of the current state (ny*nx values, every node,
 * the layout of orc_fields); f and the step count stay.  With orc_set_f it
 * lets a test hand rows of one instance's state to another (a slab split
 * with halo copies). */
void orc_set_T(orc_t *o, const double *T) { memcpy(o->T, T, sizeof(double) * o->nx * o->ny); }

void orc_classes(const orc_t *o, unsigned char *kind, unsigned char *therm, int *partner) {
    long n = (long)o->nx * o->ny;
    for (long k = 0; k < n; k++) {
        if (kind) kind[k] = o->kind[k];
        if (therm) therm[k] = o->therm[k];
        if (partner) partner[k] = o->partner[k];
    }
}

/* Eq. 90, Nu = -d(theta)/dX at the hot (west) wall, discretised with the
 * second-order one-sided difference (-3 T0 + 4 T1 - T2)/2 per node row;
 * the cold (east) wall uses the mirrored stencil.  theta = (T - T_E)/(T_W - T_E),
 * X = x/H with H = ny - 1.  Means are trapezoid integrals over Y in [0, 1]. */
void orc_nusselt(const orc_t *o, double *mean_hot, double *local_hot, double *mean_cold,
                 double *local_cold) {
    int nx = o->nx, ny = o->ny;
    double H = ny - 1, dT = o->t_wall[SIDE_W] - o->t_wall[SIDE_E];
    double sh = 0, sc = 0;
    for (int j = 0; j < ny; j++) {
        const double *r = o->T + (long)j * nx;
        double nh = -H * (-3.0 * r[0] + 4.0 * r[1] - r[2]) / (2.0 * dT);
        double nc = -H * (3.0 * r[nx - 1] - 4.0 * r[nx - 2] + r[nx - 3]) / (2.0 * dT);
        if (local_hot) local_hot[j] = nh;
        if (local_cold) local_cold[j] = nc;
        double wgt = (j == 0 || j == ny - 1) ? 0.5 : 1.0;
        sh += wgt * nh;
        sc += wgt * nc;
    }
    if (mean_hot) *mean_hot = sh / H;
    if (mean_cold) *mean_cold = sc / H;
}

/* Heat crossing each vertical face line between columns i and i+1, from the
 * same face fluxes the FV balance uses, as a Nusselt number
 * Q_i / (alpha (T_W - T_E)).  out has nx - 1 entries. */
void orc_flux_nusselt(const orc_t *o, double *out) {
    int nx = o->nx, ny = o->ny;
    double dT = o->t_wall[SIDE_W] - o->t_wall[SIDE_E];
    for (int i = 0; i + 1 < nx; i++) {
        double Qs = 0;
        for (int j = 0; j < ny; j++) {
            long k = (long)j * nx + i, m = k + 1;
            if (!fv_member(o, (int)k) || !fv_member(o, (int)m)) continue;
            double A = extent_y(o, j);
            double un = 0.5 * (o->ux[k] + o->ux[m]);
            double Tf = 0.5 * (o->T[k] + o->T[m]);
            Qs += A * un * Tf - o->alpha * A * (o->T[m] - o->T[k]);
        }
        out[i] = Qs / (o->alpha * dT);
    }
}

/* Steady-state residual ||u^n - u^s||_2 / ||u^n||_2 over fluid nodes, where
 * u^s is the snapshot taken by the previous call (or by set_state); the
 * current velocity then becomes the new snapshot. */
double orc_residual(orc_t *o) {
    long n = (long)o->nx * o->ny;
    double num = 0, den = 0;
    for (long k = 0; k < n; k++) {
        if (o->kind[k] != K_FLUID) continue;
        double du = o->ux[k] - o->su[k], dv = o->uy[k] - o->sv[k];
        num += du * du + dv * dv;
        den += o->ux[k] * o->ux[k] + o->uy[k] * o->uy[k];
        o->su[k] = o->ux[k];
        o->sv[k] = o->uy[k];
    }
    if (den == 0.0) return num == 0.0 ? 0.0 : INFINITY;
    return sqrt(num) / sqrt(den);
}

/* Control-volume sizes used by the FV balance (0 for nodes outside it). */
void orc_cv_volumes(const orc_t *o, double *V) {
    for (int j = 0; j < o->ny; j++)
        for (int i = 0; i < o->nx; i++) {
            long k = (long)j * o->nx + i;
            V[k] = fv_member(o, (int)k) ? extent_x(o, i) * extent_y(o, j) : 0.0;
        }
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
