// Batches of cavities (included at the end of lbmfvm.cu, same translation unit).
//
// The cavities of a batch are packed into one grid, each in a slot that
// starts on a 128 x 16 corner so that every tile shape of the TMA kernel
// tiles it without touching a neighbour.  One persistent launch of the TMA
// kernel steps every active cavity: its tile list holds the tiles of the
// active cavities and its cavity table their lattice parameters.  Per-cavity
// work (initial state, fields, residual, Nusselt number) runs the existing
// kernels on a view of the cavity: base pointers moved to the cavity's origin,
// the packed grid's row pitch and plane stride, the cavity's own sizes.
// Converged cavities leave the tile list and keep their state where it was.

struct lbmfvm_batch {
    lbmfvm_t *a = nullptr;  // the packed grid (memory, stream, kernels)
    struct Cav {
        lbmfvm_grid_t grid;
        int x0, y0;
        double nu, alpha, gbeta, tau, t_ref;
        int64_t steps;    // steps since this cavity's last set_state
        int parity;       // buffer of the state while frozen
        bool active;
        size_t snap_off;  // first node of the cavity's residual snapshot
        double last_r;
    };
    std::vector<Cav> cav;
    char err[512];
};

namespace {

constexpr int kSlotW = 128, kSlotH = 16;

int bfail(lbmfvm_batch_t *b, int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->err, sizeof(b->err), fmt, ap);
    va_end(ap);
    snprintf(g_err, sizeof(g_err), "%s", b->err);
    return code;
}

// Errors recorded on the packed-grid handle are reported on the batch.
int bcheck(lbmfvm_batch_t *b, int code) {
    if (code != LBMFVM_OK) snprintf(b->err, sizeof(b->err), "%s", b->a->err);
    return code;
}

int cav_parity(const lbmfvm_batch_t *b, int i) { return b->cav[i].active ? b->a->parity : b->cav[i].parity; }

template <class S>
StepArgs<S> cav_view(const lbmfvm_batch_t *b, int i, int cur) {
    using C = typename Compute<S>::type;
    StepArgs<S> v = args_for<S>(b->a, cur);
    const auto &c = b->cav[i];
    const long long off = (long long)c.y0 * v.pitch + c.x0;
    v.fin += off;
    v.fout += off;
    v.Tin += off;
    v.Tout += off;
    v.code += off;
    v.nx = c.grid.nx;
    v.ny = c.grid.ny;
    v.perx = v.pery = 0;
    v.omega = C(1.0 / c.tau);
    v.alpha = C(c.alpha);
    v.gbeta = C(c.gbeta);
    v.t_ref = C(c.t_ref);
    v.fx = v.fy = C(0);
    for (int s = 0; s < 4; s++) {
        const bool moving = c.grid.bc[s] == LBMFVM_BC_MOVING;
        v.wall_u[s] = C(moving && s >= 2 ? c.grid.u_lid : 0.0);
        v.wall_v[s] = C(moving && s < 2 ? c.grid.u_lid : 0.0);
    }
    return v;
}

// View whose inputs are the state of the cavity's current step: the previous
// post-collision buffer (or the unrelaxed initial populations at step 0) and
// the current temperature.
template <class S>
StepArgs<S> cav_read_view(const lbmfvm_batch_t *b, int i, int &direct) {
    const int par = cav_parity(b, i);
    StepArgs<S> v = cav_view<S>(b, i, par);
    const auto &c = b->cav[i];
    const long long off = (long long)c.y0 * v.pitch + c.x0;
    v.fin = reinterpret_cast<const S *>(b->a->base + b->a->L.f[par ^ 1]) + off;
    direct = c.steps == 0;
    return v;
}

template <class S>
void launch_cav_init(lbmfvm_batch_t *b, int i, const float *u0, const float *v0, const float *T0) {
    using C = typename Compute<S>::type;
    lbmfvm_t *h = b->a;
    const auto &c = b->cav[i];
    const int par = h->parity;  // the buffer the next step reads
    StepArgs<S> v = cav_view<S>(b, i, par);
    const long long off = (long long)c.y0 * v.pitch + c.x0;
    S *fstar = reinterpret_cast<S *>(h->base + h->L.f[par]) + off;
    S *f0 = reinterpret_cast<S *>(h->base + h->L.f[par ^ 1]) + off;
    C *Ta = reinterpret_cast<C *>(h->base + h->L.T[par]) + off;
    C *Tb = reinterpret_cast<C *>(h->base + h->L.T[par ^ 1]) + off;
    const double *tw = reinterpret_cast<const double *>(h->base + h->L.twall) + 4 * i;
    dim3 block(32, 8), grid((c.grid.nx + 31) / 32, (c.grid.ny + 7) / 8);
    init_kernel<S><<<grid, block, 0, h->s>>>(v, f0, fstar, u0, v0, T0, c.grid.t_init, tw, c.grid.bc[0], c.grid.bc[1],
                                             c.grid.bc[2], c.grid.bc[3], Ta, Tb);
}

template <class S>
void launch_cav_residual(lbmfvm_batch_t *b, int i, int update_only) {
    lbmfvm_t *h = b->a;
    int direct;
    StepArgs<S> v = cav_read_view<S>(b, i, direct);
    double *su = reinterpret_cast<double *>(h->base + h->L.snap) + b->cav[i].snap_off;
    double *sv = su + (size_t)b->cav[i].grid.nx * b->cav[i].grid.ny;
    double *red = reinterpret_cast<double *>(h->base + h->L.red);
    const int blocks = v.ny < kResidualBlocks ? v.ny : kResidualBlocks;
    residual_kernel<S><<<blocks, 256, 0, h->s>>>(v, direct, su, sv, red, update_only);
    if (!update_only)
        residual_finish_kernel<<<1, 32, 0, h->s>>>(red, blocks, reinterpret_cast<double *>(h->base + h->L.cavres) + 4 * i);
}

template <class S>
void launch_cav_nusselt(lbmfvm_batch_t *b, int i) {
    lbmfvm_t *h = b->a;
    int direct;
    StepArgs<S> v = cav_read_view<S>(b, i, direct);
    const auto &g = b->cav[i].grid;
    double *red = reinterpret_cast<double *>(h->base + h->L.red);
    nusselt_kernel<S><<<1, 256, 0, h->s>>>(v, (double)(g.ny - 1), g.t_wall[LBMFVM_SIDE_W] - g.t_wall[LBMFVM_SIDE_E],
                                           red + 2 * kResidualBlocks + 8,
                                           reinterpret_cast<double *>(h->base + h->L.cavres) + 4 * i + 2);
}

template <class S, class O>
void launch_cav_fields(lbmfvm_batch_t *b, int i, int which, O *o0, O *o1) {
    int direct;
    StepArgs<S> v = cav_read_view<S>(b, i, direct);
    dim3 block(32, 8), grid((v.nx + 31) / 32, (v.ny + 7) / 8);
    fields_kernel<S, O><<<grid, block, 0, b->a->s>>>(v, direct, which, o0, o1);
}

#define BDISPATCH(b, FN, ...)                                         \
    do {                                                              \
        switch ((b)->a->prec) {                                       \
            case LBMFVM_F32: FN<float>(__VA_ARGS__); break;           \
            case LBMFVM_F16: FN<__half>(__VA_ARGS__); break;          \
            case LBMFVM_BF16: FN<__nv_bfloat16>(__VA_ARGS__); break;  \
        }                                                             \
    } while (0)

int check_index(lbmfvm_batch_t *b, int32_t i) {
    if (!b) return fail_thread(LBMFVM_ERR_ARG, "batch is NULL");
    if (i < 0 || i >= (int)b->cav.size())
        return bfail(b, LBMFVM_ERR_ARG, "cavity index %d outside [0, %d)", i, (int)b->cav.size());
    return LBMFVM_OK;
}

int set_active(lbmfvm_batch_t *b, int i, bool active) {
    if (b->cav[i].active == active) return LBMFVM_OK;
    if (!active) b->cav[i].parity = b->a->parity;
    b->cav[i].active = active;
    b->a->atlas_active[i] = active ? 1 : 0;
    return bcheck(b, upload_tiles(b->a, b->a->tile_w, b->a->tile_h));
}

int cav_set_state(lbmfvm_batch_t *b, int i, const float *u, const float *v, const float *T) {
    lbmfvm_t *h = b->a;
    if (int r = set_active(b, i, true)) return r;
    const auto &c = b->cav[i];
    const size_t n = (size_t)c.grid.nx * c.grid.ny;
    float *stage = reinterpret_cast<float *>(h->base + h->L.stage);
    const float *du = nullptr, *dv = nullptr, *dT = nullptr;
    if (int r = bcheck(b, join_in(h))) return r;
    cudaError_t e = cudaSuccess;
    if (u && e == cudaSuccess) {
        e = cudaMemcpyAsync(stage, u, n * sizeof(float), cudaMemcpyDefault, h->s);
        du = stage;
    }
    if (v && e == cudaSuccess) {
        e = cudaMemcpyAsync(stage + n, v, n * sizeof(float), cudaMemcpyDefault, h->s);
        dv = stage + n;
    }
    if (T && e == cudaSuccess) {
        e = cudaMemcpyAsync(stage + 2 * n, T, n * sizeof(float), cudaMemcpyDefault, h->s);
        dT = stage + 2 * n;
    }
    if (e != cudaSuccess) return bfail(b, LBMFVM_ERR_CUDA, "staging the state failed: %s", cudaGetErrorString(e));
    BDISPATCH(b, launch_cav_init, b, i, du, dv, dT);
    b->cav[i].steps = 0;
    BDISPATCH(b, launch_cav_residual, b, i, 1);  // snapshot := u^0
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) return bfail(b, LBMFVM_ERR_CUDA, "initial state failed: %s", cudaGetErrorString(e));
    b->cav[i].last_r = NAN;
    return bcheck(b, join_out(h));
}

}  // namespace

extern "C" {

int lbmfvm_batch_create(int32_t n, const lbmfvm_grid_t *grids, const uint8_t *const *masks, const double *Ra,
                        const double *Pr, const double *Ma, const lbmfvm_opts_t *opts, lbmfvm_batch_t **out) {
    if (!out) return fail_thread(LBMFVM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || !grids || !Ra || !Pr || !Ma) return fail_thread(LBMFVM_ERR_ARG, "need n >= 1 and grids, Ra, Pr, Ma");
    lbmfvm_batch_t *b = new (std::nothrow) lbmfvm_batch_t();
    if (!b) return fail_thread(LBMFVM_ERR_NOMEM, "host allocation failed");
    b->cav.resize(n);
    // lattice parameters (Eqs. 83-89, 15) with the same limits as lbmfvm_create
    for (int i = 0; i < n; i++) {
        const lbmfvm_grid_t &g = grids[i];
        if (int r = check_grid(&g)) {
            delete b;
            return r;
        }
        for (int s = 0; s < 4; s++)
            if (g.bc[s] == LBMFVM_BC_PERIODIC) {
                delete b;
                return fail_thread(LBMFVM_ERR_ARG, "cavity %d: periodic sides are not batched", i);
            }
        const double dT = g.t_wall[LBMFVM_SIDE_W] - g.t_wall[LBMFVM_SIDE_E];
        if (!(Ra[i] > 0) || !(Pr[i] > 0) || !(Ma[i] > 0) || dT == 0.0 || !std::isfinite(dT)) {
            delete b;
            return fail_thread(LBMFVM_ERR_ARG, "cavity %d: Ra, Pr, Ma must be positive and t_wall[W] != t_wall[E]", i);
        }
        const double H = g.ny - 1, U0 = Ma[i] / std::sqrt(3.0);
        auto &c = b->cav[i];
        c.grid = g;
        c.nu = U0 * H * std::sqrt(Pr[i] / Ra[i]);
        c.alpha = U0 * H / std::sqrt(Ra[i] * Pr[i]);
        c.gbeta = U0 * U0 / (H * dT);
        c.tau = 3.0 * c.nu + 0.5;
        c.t_ref = (opts && !std::isnan(opts->t_ref)) ? opts->t_ref : g.t_wall[LBMFVM_SIDE_E];
        const char *why = Ma[i] > 0.3 ? "Ma > 0.3" : c.tau < 0.51 ? "tau < 0.51" : c.alpha > 0.25 ? "alpha > 0.25"
                          : U0 * U0 > 2 * c.alpha ? "U0^2 > 2 alpha" : nullptr;
        if (why) {
            delete b;
            return fail_thread(LBMFVM_ERR_UNSTABLE, "cavity %d: %s", i, why);
        }
        c.active = true;
        c.steps = 0;
        c.parity = 0;
        c.last_r = NAN;
    }
    // shelf packing of 128 x 16 slots, tallest cavities first
    int width = 2048;
    for (int i = 0; i < n; i++) width = std::max(width, (grids[i].nx + kSlotW - 1) / kSlotW * kSlotW);
    std::vector<int> order(n);
    for (int i = 0; i < n; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return grids[p].ny > grids[q].ny; });
    int x = 0, y = 0, shelf = 0;
    size_t snap = 0;
    for (int i : order) {
        const int w = (grids[i].nx + kSlotW - 1) / kSlotW * kSlotW;
        const int hgt = (grids[i].ny + kSlotH - 1) / kSlotH * kSlotH;
        if (x + w > width) {
            y += shelf;
            x = 0;
            shelf = 0;
        }
        b->cav[i].x0 = x;
        b->cav[i].y0 = y;
        x += w;
        shelf = std::max(shelf, hgt);
    }
    for (int i = 0; i < n; i++) {
        b->cav[i].snap_off = snap;
        snap += 2 * (size_t)grids[i].nx * grids[i].ny;
    }
    lbmfvm_grid_t atlas{};
    atlas.nx = width;
    atlas.ny = y + shelf;
    for (int s = 0; s < 4; s++) atlas.bc[s] = LBMFVM_BC_ADIABATIC;
    atlas.t_wall[LBMFVM_SIDE_W] = 1.0;
    if ((long long)atlas.nx * atlas.ny > (1LL << 30)) {
        delete b;
        return fail_thread(LBMFVM_ERR_ARG, "the packed cavities exceed 2^30 nodes");
    }
    AtlasSpec spec;
    const int pitch = (int)align_up((size_t)atlas.nx, 64);
    spec.codes.assign((size_t)atlas.ny * pitch, stored_code(CODE_OUTSIDE));
    for (int i = 0; i < n; i++) {
        const auto &c = b->cav[i];
        const std::vector<uint8_t> codes = classify(c.grid, masks ? masks[i] : nullptr, c.grid.nx);
        for (int j = 0; j < c.grid.ny; j++)
            std::memcpy(&spec.codes[(size_t)(c.y0 + j) * pitch + c.x0], &codes[(size_t)j * c.grid.nx], c.grid.nx);
        CavityDesc cd{};
        cd.x0 = c.x0;
        cd.y0 = c.y0;
        cd.nx = c.grid.nx;
        cd.ny = c.grid.ny;
        cd.omega = (float)(1.0 / c.tau);
        cd.alpha = (float)c.alpha;
        cd.gbeta = (float)c.gbeta;
        cd.t_ref = (float)c.t_ref;
        for (int s = 0; s < 4; s++) {
            const bool moving = c.grid.bc[s] == LBMFVM_BC_MOVING;
            cd.wall_u[s] = (float)(moving && s >= 2 ? c.grid.u_lid : 0.0);
            cd.wall_v[s] = (float)(moving && s < 2 ? c.grid.u_lid : 0.0);
        }
        spec.cavs.push_back(cd);
    }
    lbmfvm_opts_t o;
    lbmfvm_opts_default(&o);
    if (opts) o = *opts;
    if (o.workspace) {
        delete b;
        return fail_thread(LBMFVM_ERR_ARG, "batches allocate their own device memory (workspace must be NULL)");
    }
    if (o.kernel == LBMFVM_KERNEL_GENERIC) {
        delete b;
        return fail_thread(LBMFVM_ERR_ARG, "batches run on the TMA kernel");
    }
    o.kernel = LBMFVM_KERNEL_TMA;
    // the packed grid's own lattice parameters are unused (every tile takes
    // its cavity's); pass valid placeholders
    if (int r = create_impl(&atlas, nullptr, 0.1, 0.1, 0.0, nullptr, &o, &b->a, &spec)) {
        delete b;
        return r;
    }
    // wall temperatures per cavity for the initial-state kernel
    std::vector<double> tw(4 * (size_t)n);
    for (int i = 0; i < n; i++)
        for (int s = 0; s < 4; s++) tw[4 * i + s] = b->cav[i].grid.t_wall[s];
    if (cudaMemcpy(b->a->base + b->a->L.twall, tw.data(), tw.size() * sizeof(double), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
        lbmfvm_batch_destroy(b);
        return fail_thread(LBMFVM_ERR_CUDA, "uploading wall temperatures failed");
    }
    for (int i = 0; i < n; i++)
        if (int r = cav_set_state(b, i, nullptr, nullptr, nullptr)) {
            snprintf(g_err, sizeof(g_err), "%s", b->err);
            lbmfvm_batch_destroy(b);
            return r;
        }
    *out = b;
    return LBMFVM_OK;
}

int lbmfvm_batch_set_state(lbmfvm_batch_t *b, int32_t i, const float *u, const float *v, const float *T) {
    if (int r = check_index(b, i)) return r;
    return cav_set_state(b, i, u, v, T);
}

int lbmfvm_batch_step(lbmfvm_batch_t *b, int64_t n) {
    if (!b) return fail_thread(LBMFVM_ERR_ARG, "batch is NULL");
    if (n < 0) return bfail(b, LBMFVM_ERR_ARG, "n = %lld is negative", (long long)n);
    bool any = false;
    for (auto &c : b->cav) any |= c.active;
    if (!any || n == 0) return LBMFVM_OK;
    if (int r = bcheck(b, lbmfvm_step(b->a, n))) return r;
    for (auto &c : b->cav)
        if (c.active) c.steps += n;
    return LBMFVM_OK;
}

int lbmfvm_batch_residuals(lbmfvm_batch_t *b, double *r) {
    if (!b || !r) return fail_thread(LBMFVM_ERR_ARG, "batch or r is NULL");
    lbmfvm_t *h = b->a;
    if (int e = bcheck(b, join_in(h))) return e;
    const int n = (int)b->cav.size();
    for (int i = 0; i < n; i++)
        if (b->cav[i].active) BDISPATCH(b, launch_cav_residual, b, i, 0);
    std::vector<double> res(4 * (size_t)n);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(res.data(), h->base + h->L.cavres, res.size() * sizeof(double), cudaMemcpyDeviceToHost, h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) return bfail(b, LBMFVM_ERR_CUDA, "batch residual failed: %s", cudaGetErrorString(e));
    if (int e2 = bcheck(b, check_device_status(h))) return e2;
    int status = LBMFVM_OK;
    for (int i = 0; i < n; i++) {
        auto &c = b->cav[i];
        if (c.active) {
            const double num = res[4 * i], den = res[4 * i + 1];
            if (!std::isfinite(num) || !std::isfinite(den)) {
                c.last_r = NAN;
                status = bfail(b, LBMFVM_ERR_DIVERGED, "cavity %d: non-finite velocity", i);
            } else {
                c.last_r = den > 0.0 ? std::sqrt(num) / std::sqrt(den) : (num == 0.0 ? 0.0 : INFINITY);
            }
        }
        r[i] = c.last_r;
    }
    if (int e2 = bcheck(b, join_out(h))) return e2;
    return status;
}

int lbmfvm_batch_run(lbmfvm_batch_t *b, double tol, int64_t check_every, int64_t max_steps, int64_t *steps_out,
                     double *r_out) {
    if (!b) return fail_thread(LBMFVM_ERR_ARG, "batch is NULL");
    if (check_every <= 0 || max_steps < 0) return bfail(b, LBMFVM_ERR_ARG, "check_every must be > 0, max_steps >= 0");
    const int n = (int)b->cav.size();
    std::vector<double> r(n);
    int64_t done = 0;
    int status = LBMFVM_OK;
    while (done < max_steps) {
        bool any = false;
        for (auto &c : b->cav) any |= c.active;
        if (!any) break;
        const int64_t k = check_every < max_steps - done ? check_every : max_steps - done;
        if ((status = lbmfvm_batch_step(b, k))) break;
        done += k;
        if ((status = lbmfvm_batch_residuals(b, r.data()))) break;
        for (int i = 0; i < n; i++)
            if (b->cav[i].active && r[i] < tol)
                if ((status = set_active(b, i, false))) break;
        if (status) break;
    }
    for (int i = 0; i < n; i++) {
        if (steps_out) steps_out[i] = b->cav[i].steps;
        if (r_out) r_out[i] = b->cav[i].last_r;
    }
    return status;
}

int lbmfvm_batch_fields(lbmfvm_batch_t *b, int32_t i, double *rho, double *u, double *v, double *T) {
    if (int r = check_index(b, i)) return r;
    lbmfvm_t *h = b->a;
    const size_t n = (size_t)b->cav[i].grid.nx * b->cav[i].grid.ny;
    double *st = reinterpret_cast<double *>(h->base + h->L.stage);
    if (int r = bcheck(b, join_in(h))) return r;
    double *outs[2][2] = {{rho, u}, {v, T}};
    cudaError_t e = cudaSuccess;
    for (int which = 0; which < 2 && e == cudaSuccess; which++) {
        if (!outs[which][0] && !outs[which][1]) continue;
        switch (h->prec) {
            case LBMFVM_F32: launch_cav_fields<float, double>(b, i, which, st, st + n); break;
            case LBMFVM_F16: launch_cav_fields<__half, double>(b, i, which, st, st + n); break;
            case LBMFVM_BF16: launch_cav_fields<__nv_bfloat16, double>(b, i, which, st, st + n); break;
        }
        e = cudaGetLastError();
        for (int k = 0; k < 2 && e == cudaSuccess; k++)
            if (outs[which][k]) e = cudaMemcpyAsync(outs[which][k], st + k * n, n * sizeof(double), cudaMemcpyDefault, h->s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) return bfail(b, LBMFVM_ERR_CUDA, "batch fields failed: %s", cudaGetErrorString(e));
    if (int r = bcheck(b, check_device_status(h))) return r;
    return bcheck(b, join_out(h));
}

int lbmfvm_batch_nusselt(lbmfvm_batch_t *b, int32_t i, double *mean_hot, double *local_hot, double *mean_cold) {
    if (int r = check_index(b, i)) return r;
    lbmfvm_t *h = b->a;
    if (int r = bcheck(b, join_in(h))) return r;
    BDISPATCH(b, launch_cav_nusselt, b, i);
    double means[2];
    double *red = reinterpret_cast<double *>(h->base + h->L.red);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(means, reinterpret_cast<double *>(h->base + h->L.cavres) + 4 * i + 2, sizeof(means),
                            cudaMemcpyDeviceToHost, h->s);
    if (e == cudaSuccess && local_hot)
        e = cudaMemcpyAsync(local_hot, red + 2 * kResidualBlocks + 8, b->cav[i].grid.ny * sizeof(double),
                            cudaMemcpyDefault, h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) return bfail(b, LBMFVM_ERR_CUDA, "batch Nusselt failed: %s", cudaGetErrorString(e));
    if (mean_hot) *mean_hot = means[0];
    if (mean_cold) *mean_cold = means[1];
    return bcheck(b, join_out(h));
}

int lbmfvm_batch_info(const lbmfvm_batch_t *b, int32_t i, int64_t *steps, int32_t *active, double *params) {
    if (!b) return fail_thread(LBMFVM_ERR_ARG, "batch is NULL");
    if (i < 0 || i >= (int)b->cav.size()) return fail_thread(LBMFVM_ERR_ARG, "cavity index %d out of range", i);
    const auto &c = b->cav[i];
    if (steps) *steps = c.steps;
    if (active) *active = c.active ? 1 : 0;
    if (params) {
        params[0] = c.nu;
        params[1] = c.alpha;
        params[2] = c.gbeta;
        params[3] = c.tau;
    }
    return LBMFVM_OK;
}

void lbmfvm_batch_destroy(lbmfvm_batch_t *b) {
    if (!b) return;
    lbmfvm_destroy(b->a);
    delete b;
}

const char *lbmfvm_batch_last_error(const lbmfvm_batch_t *b) { return b ? b->err : g_err; }

}  // extern "C"
