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
//
// Precision ladder: the rounding of the stored populations puts a floor under
// the residual (about 1e-3 for 16-bit storage, 1e-7 for FP32).  Above the
// storage grid the batch keeps packed grids of the wider precisions with the
// same slots (FP32, then double-single), created when first needed; a cavity whose
// residual reaches its level's switch value, or stops falling, is converted
// into the next grid and stepped there from then on.  The top of the ladder
// is double-single storage and arithmetic (FP64-like precision on the FP32
// units).

struct lbmfvm_batch {
    lbmfvm_t *a = nullptr;          // the storage grid (memory, stream, kernels); lv[0]
    lbmfvm_t *lv[3] = {};           // packed grids of the ladder; upper ones created when first needed
    int prec[3] = {};               // their storage precisions
    int nlv = 1;                    // levels of the ladder
    double switch_r[3] = {};        // residual that moves a cavity from level l to l + 1 (0: never)
    int stall_checks[3] = {};       // checks without halving the residual that also move it (0: never)
    lbmfvm_grid_t atlas_grid;       // what the upper grids are created from
    AtlasSpec spec;
    lbmfvm_opts_t opts;
    bool auto_shape = false;        // tile shapes chosen by the library (not pinned by opts.tma_config)
    int base_cfg[3] = {-1, -1, -1}; // each level's shape for its whole packed grid
    struct Cav {
        lbmfvm_grid_t grid;
        int x0, y0;
        double nu, alpha, gbeta, tau, t_ref;
        int substeps;     // energy-update sub-steps per lattice step
        int64_t steps;    // steps since this cavity's last set_state
        int parity;       // buffer of the state while frozen
        bool active;
        int level;        // ladder level holding the state
        double best_r;    // smallest residual at this level, and the checks since it halved
        int since_best;
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

// The packed grid that holds cavity i's state.
lbmfvm_t *hnd(const lbmfvm_batch_t *b, int i) { return b->lv[b->cav[i].level]; }

int cav_parity(const lbmfvm_batch_t *b, int i) { return b->cav[i].active ? hnd(b, i)->parity : b->cav[i].parity; }

template <class S>
StepArgs<S> cav_view(const lbmfvm_batch_t *b, int i, int cur) {
    using C = typename Compute<S>::type;
    StepArgs<S> v = args_for<S>(hnd(b, i), cur);
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
    v.fin = reinterpret_cast<const S *>(hnd(b, i)->base + hnd(b, i)->L.f[par ^ 1]) + off;
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
    lbmfvm_t *h = hnd(b, i);
    int direct;
    StepArgs<S> v = cav_read_view<S>(b, i, direct);
    double *su = reinterpret_cast<double *>(h->base + h->L.snap) + b->cav[i].snap_off;
    double *sv = su + (size_t)b->cav[i].grid.nx * b->cav[i].grid.ny;
    double *red = reinterpret_cast<double *>(h->base + h->L.red);
    const int blocks = v.ny < kResidualBlocks ? v.ny : kResidualBlocks;
    residual_kernel<S><<<blocks, 256, 0, h->s>>>(v, direct, su, sv, red, update_only);
    if (!update_only)
        residual_finish_kernel<<<1, 32, 0, h->s>>>(red, blocks,
                                                   reinterpret_cast<double *>(h->base + h->L.cavres) + kCavRes * i);
}

template <class S>
void launch_cav_nusselt(lbmfvm_batch_t *b, int i) {
    lbmfvm_t *h = hnd(b, i);
    int direct;
    StepArgs<S> v = cav_read_view<S>(b, i, direct);
    const auto &g = b->cav[i].grid;
    double *red = reinterpret_cast<double *>(h->base + h->L.red);
    nusselt_kernel<S><<<1, 256, 0, h->s>>>(v, (double)(g.ny - 1), g.t_wall[LBMFVM_SIDE_W] - g.t_wall[LBMFVM_SIDE_E],
                                           red + kRedLocal,
                                           reinterpret_cast<double *>(h->base + h->L.cavres) + kCavRes * i + kCavNu);
}

template <class S>
void launch_cav_rescale(lbmfvm_batch_t *b, int i) {
    lbmfvm_t *h = hnd(b, i);
    const auto &c = b->cav[i];
    StepArgs<S> v = cav_view<S>(b, i, cav_parity(b, i));
    const long long off = (long long)c.y0 * v.pitch + c.x0;
    S *f0 = reinterpret_cast<S *>(h->base + h->L.f[0]) + off;
    S *f1 = reinterpret_cast<S *>(h->base + h->L.f[1]) + off;
    const double *tot = reinterpret_cast<const double *>(h->base + h->L.cavres) + kCavRes * i;
    dim3 block(32, 8), grid((c.grid.nx + 31) / 32, (c.grid.ny + 7) / 8, 2);
    rescale_kernel<S><<<grid, block, 0, h->s>>>(v, f0, f1, tot);
}

template <class S, class O>
void launch_cav_fields(lbmfvm_batch_t *b, int i, int which, O *o0, O *o1) {
    int direct;
    StepArgs<S> v = cav_read_view<S>(b, i, direct);
    dim3 block(32, 8), grid((v.nx + 31) / 32, (v.ny + 7) / 8);
    fields_kernel<S, O><<<grid, block, 0, hnd(b, i)->s>>>(v, direct, which, o0, o1);
}

// FN<storage type>(...) for the precision of packed grid h.
#define BDISPATCH(h, FN, ...)                                         \
    do {                                                              \
        switch ((h)->prec) {                                          \
            case LBMFVM_F64: FN<double>(__VA_ARGS__); break;          \
            case LBMFVM_F32: FN<float>(__VA_ARGS__); break;           \
            case LBMFVM_F16: FN<__half>(__VA_ARGS__); break;          \
            case LBMFVM_BF16: FN<__nv_bfloat16>(__VA_ARGS__); break;  \
            case LBMFVM_F32X2: FN<dsf>(__VA_ARGS__); break;           \
        }                                                             \
    } while (0)

int check_index(lbmfvm_batch_t *b, int32_t i) {
    if (!b) return fail_thread(LBMFVM_ERR_ARG, "batch is NULL");
    if (i < 0 || i >= (int)b->cav.size())
        return bfail(b, LBMFVM_ERR_ARG, "cavity index %d outside [0, %d)", i, (int)b->cav.size());
    return LBMFVM_OK;
}

int bcheck_h(lbmfvm_batch_t *b, lbmfvm_t *h, int code) {
    if (code != LBMFVM_OK) snprintf(b->err, sizeof(b->err), "%s", h->err);
    return code;
}

// A level whose active cavities, once some have left it, fill fewer tiles
// than the GPU has SMs is bound by the latency of one tile rather than by
// throughput: it takes the small-grid shape a single cavity of that size
// would (64 x 8 for 32- and 16-bit storage, 32 x 8 with ring warps for
// 64-bit), and its own shape again when the active set grows.  Shapes never
// change results.
int reshape_level(lbmfvm_batch_t *b, int l) {
    lbmfvm_t *h = b->lv[l];
    if (!b->auto_shape || !h || !h->use_tma || h->fv_quick || h->L.split || h->grid2) return LBMFVM_OK;
    if (b->base_cfg[l] < 0) b->base_cfg[l] = h->tma_config;
    long long active = 0, all = 0;
    for (size_t c = 0; c < h->atlas_cavs.size(); c++) {
        const long long nodes = (long long)h->atlas_cavs[c].nx * h->atlas_cavs[c].ny;
        all += nodes;
        if (h->atlas_active[c]) active += nodes;
    }
    if (active == 0) return LBMFVM_OK;  // nothing to step: keep the shape
    const bool wide = store_size(h->prec) == 8;
    const long long tiles = wide ? active / (32 * 8) : active / (64 * 16);
    const int want = (active < all && tiles < h->num_sms) ? (wide ? 4 : 2) : b->base_cfg[l];
    if (want == h->tma_config) return LBMFVM_OK;
    h->tma_config = want;
    return setup_kernels(h);  // new tensor maps and tile lists; the step graph is captured again
}

int set_active(lbmfvm_batch_t *b, int i, bool active) {
    if (b->cav[i].active == active) return LBMFVM_OK;
    lbmfvm_t *h = hnd(b, i);
    if (!active) b->cav[i].parity = h->parity;
    b->cav[i].active = active;
    h->atlas_active[i] = active ? 1 : 0;
    if (int r = bcheck_h(b, h, upload_tiles(h, h->tile_w, h->tile_h))) return r;
    return bcheck_h(b, h, reshape_level(b, b->cav[i].level));
}

// The packed grid of ladder level l, created (every cavity inactive) on first use.
int ladder_grid(lbmfvm_batch_t *b, int l) {
    if (b->lv[l]) return LBMFVM_OK;
    lbmfvm_opts_t o = b->opts;
    o.store = b->prec[l];
    lbmfvm_t *h = nullptr;
    if (int r = create_impl(&b->atlas_grid, nullptr, 0.1, 0.1, 0.0, nullptr, &o, &h, &b->spec))
        return bfail(b, r, "creating a grid of the precision ladder failed: %s", g_err);
    h->atlas_active.assign(b->cav.size(), 0);
    if (int r = upload_tiles(h, h->tile_w, h->tile_h)) {
        bfail(b, r, "%s", h->err);
        lbmfvm_destroy(h);
        return r;
    }
    b->lv[l] = h;
    return LBMFVM_OK;
}

// Moves active cavity i one level up the ladder: both population and
// temperature buffers converted, the residual snapshot carried over, the tile
// lists of both grids rebuilt.  Called between steps, with both grids'
// streams idle.
int promote(lbmfvm_batch_t *b, int i) {
    auto &c = b->cav[i];
    if (c.level + 1 >= b->nlv) return LBMFVM_OK;
    if (int r = ladder_grid(b, c.level + 1)) return r;
    lbmfvm_t *a = b->lv[c.level], *p = b->lv[c.level + 1];
    const long long off = (long long)c.y0 * a->L.pitch + c.x0;
    if (int r = bcheck_h(b, a, join_in(a))) return r;
    if (cudaStreamSynchronize(a->s) != cudaSuccess) return bfail(b, LBMFVM_ERR_CUDA, "stream synchronisation failed");
    if (int r = bcheck_h(b, p, join_in(p))) return r;
    BDISPATCH(a, launch_convert_from, a, p, off, off, c.grid.nx, c.grid.ny, a->parity ^ p->parity);
    cudaError_t e = cudaGetLastError();
    const size_t n = (size_t)c.grid.nx * c.grid.ny;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(reinterpret_cast<double *>(p->base + p->L.snap) + c.snap_off,
                            reinterpret_cast<const double *>(a->base + a->L.snap) + c.snap_off, 2 * n * sizeof(double),
                            cudaMemcpyDeviceToDevice, p->s);
    if (e != cudaSuccess) return bfail(b, LBMFVM_ERR_CUDA, "polish conversion failed: %s", cudaGetErrorString(e));
    if (int r = bcheck_h(b, p, join_out(p))) return r;
    if (int r = set_active(b, i, false)) return r;
    c.level++;
    c.best_r = INFINITY;
    c.since_best = 0;
    return set_active(b, i, true);
}

// Whether cavity i, with residual r, moves up the ladder: below its level's
// switch value, or within a factor 100 of it and without halving its best
// residual for stall_checks checks (a floor above the switch value; the
// factor keeps slow transients at their level).
bool wants_promotion(lbmfvm_batch_t *b, int i, double r) {
    auto &c = b->cav[i];
    if (c.level + 1 >= b->nlv) return false;
    if (r < 0.5 * c.best_r) {
        c.best_r = r;
        c.since_best = 0;
    } else {
        c.since_best++;
    }
    const double sw = b->switch_r[c.level];
    const int stall = b->stall_checks[c.level];
    return sw > 0.0 && (r < sw || (stall > 0 && c.since_best >= stall && r < 100.0 * sw));
}

// Mass renormalisation of every active cavity from the totals of the last
// residual pass (see rescale_kernel).
int rescale_active(lbmfvm_batch_t *b) {
    for (lbmfvm_t *h : b->lv) {
        if (!h) continue;
        if (int r = bcheck_h(b, h, join_in(h))) return r;
        for (int i = 0; i < (int)b->cav.size(); i++)
            if (b->cav[i].active && hnd(b, i) == h) BDISPATCH(h, launch_cav_rescale, b, i);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return bfail(b, LBMFVM_ERR_CUDA, "mass renormalisation failed: %s", cudaGetErrorString(e));
        if (int r = bcheck_h(b, h, join_out(h))) return r;
    }
    return LBMFVM_OK;
}

// Cavity i back to the storage grid (inactive there until set_state).
int unpolish(lbmfvm_batch_t *b, int i) {
    auto &c = b->cav[i];
    if (c.level == 0) return LBMFVM_OK;
    if (int r = set_active(b, i, false)) return r;
    c.level = 0;
    c.active = false;
    return LBMFVM_OK;
}

int cav_set_state(lbmfvm_batch_t *b, int i, const float *u, const float *v, const float *T) {
    lbmfvm_t *h = b->a;
    if (int r = unpolish(b, i)) return r;
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
    BDISPATCH(h, launch_cav_init, b, i, du, dv, dT);
    b->cav[i].steps = 0;
    BDISPATCH(h, launch_cav_residual, b, i, 1);  // snapshot := u^0
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) return bfail(b, LBMFVM_ERR_CUDA, "initial state failed: %s", cudaGetErrorString(e));
    b->cav[i].last_r = NAN;
    b->cav[i].best_r = INFINITY;
    b->cav[i].since_best = 0;
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
        const int req = opts ? opts->fv_substeps : 1;
        if (req < 0 || req > 256) {
            delete b;
            return fail_thread(LBMFVM_ERR_ARG, "fv_substeps = %d is outside [0, 256]", req);
        }
        c.substeps = substeps_for(req, c.alpha, U0);
        const char *why = Ma[i] > 0.3 ? "Ma > 0.3" : c.tau < 0.51 ? "tau < 0.51" : fv_unstable(c.alpha, U0, c.substeps);
        if (why) {
            delete b;
            return fail_thread(LBMFVM_ERR_UNSTABLE, "cavity %d: %s", i, why);
        }
        c.active = true;
        c.level = 0;
        c.best_r = INFINITY;
        c.since_best = 0;
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
        cd.omega = 1.0 / c.tau;
        cd.alpha = c.alpha;
        cd.gbeta = c.gbeta;
        cd.t_ref = c.t_ref;
        cd.substeps = c.substeps;
        for (int s = 0; s < 4; s++) {
            const bool moving = c.grid.bc[s] == LBMFVM_BC_MOVING;
            cd.wall_u[s] = moving && s >= 2 ? c.grid.u_lid : 0.0;
            cd.wall_v[s] = moving && s < 2 ? c.grid.u_lid : 0.0;
            cd.wall_uf[s] = (float)cd.wall_u[s];
            cd.wall_vf[s] = (float)cd.wall_v[s];
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
    // the ladder above the storage precision (see the top of this file)
    b->lv[0] = b->a;
    b->prec[0] = o.store;
    if (o.store == LBMFVM_F16 || o.store == LBMFVM_BF16) {
        b->prec[b->nlv] = LBMFVM_F32;
        b->switch_r[b->nlv - 1] = o.store == LBMFVM_F16 ? 2e-3 : 1e-2;
        b->stall_checks[b->nlv - 1] = 16;
        b->nlv++;
    }
    if (o.store != LBMFVM_F64 && o.store != LBMFVM_F32X2) {
        b->prec[b->nlv] = LBMFVM_F32X2;
        b->switch_r[b->nlv - 1] = 1e-6;
        b->stall_checks[b->nlv - 1] = 32;
        b->nlv++;
    }
    b->atlas_grid = atlas;
    b->spec = std::move(spec);
    b->opts = o;
    b->auto_shape = o.tma_config == LBMFVM_TMA_AUTOTUNE || o.tma_config == LBMFVM_TMA_DEFAULT;
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
    bool any[3] = {false, false, false};
    for (auto &c : b->cav)
        if (c.active) any[c.level] = true;
    if (n == 0) return LBMFVM_OK;
    // The levels' grids are independent (no block of one waits on another),
    // so their launches go on their own streams at once: a level with few
    // tiles left then fills SMs the others leave idle instead of paying its
    // launch fill and drain alone.
    for (int l = 0; l < b->nlv; l++)
        if (any[l])
            if (int r = bcheck_h(b, b->lv[l], join_in(b->lv[l]))) return r;
    for (int l = 0; l < b->nlv; l++)
        if (any[l])
            if (int r = bcheck_h(b, b->lv[l], step_impl(b->lv[l], n))) return r;
    for (int l = 0; l < b->nlv; l++)
        if (any[l])
            if (int r = bcheck_h(b, b->lv[l], join_out(b->lv[l]))) return r;
    for (auto &c : b->cav)
        if (c.active) c.steps += n;
    return LBMFVM_OK;
}

int lbmfvm_batch_residuals(lbmfvm_batch_t *b, double *r) {
    if (!b || !r) return fail_thread(LBMFVM_ERR_ARG, "batch or r is NULL");
    const int n = (int)b->cav.size();
    // per grid: residual kernels of its active cavities, then the table
    std::vector<double> res[3];
    for (int g = 0; g < 3; g++) {
        lbmfvm_t *h = b->lv[g];
        if (!h) continue;
        if (int e = bcheck_h(b, h, join_in(h))) return e;
        for (int i = 0; i < n; i++)
            if (b->cav[i].active && hnd(b, i) == h) BDISPATCH(h, launch_cav_residual, b, i, 0);
        res[g].resize(kCavRes * (size_t)n);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(res[g].data(), h->base + h->L.cavres, res[g].size() * sizeof(double),
                                cudaMemcpyDeviceToHost, h->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
        if (e != cudaSuccess) return bfail(b, LBMFVM_ERR_CUDA, "batch residual failed: %s", cudaGetErrorString(e));
        if (int e2 = bcheck_h(b, h, check_device_status(h))) return e2;
        if (int e2 = bcheck_h(b, h, join_out(h))) return e2;
    }
    int status = LBMFVM_OK;
    for (int i = 0; i < n; i++) {
        auto &c = b->cav[i];
        if (c.active) {
            const std::vector<double> &rs = res[c.level];
            const double num = rs[kCavRes * i], den = rs[kCavRes * i + 1];
            if (!std::isfinite(num) || !std::isfinite(den)) {
                c.last_r = NAN;
                status = bfail(b, LBMFVM_ERR_DIVERGED, "cavity %d: non-finite velocity", i);
            } else {
                c.last_r = den > 0.0 ? std::sqrt(num) / std::sqrt(den) : (num == 0.0 ? 0.0 : INFINITY);
            }
        }
        r[i] = c.last_r;
    }
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
        if ((status = rescale_active(b))) break;
        for (int i = 0; i < n && !status; i++) {
            auto &c = b->cav[i];
            if (!c.active) continue;
            if (r[i] < tol) status = set_active(b, i, false);
            else if (wants_promotion(b, i, r[i])) status = promote(b, i);
        }
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
    lbmfvm_t *h = hnd(b, i);
    const size_t n = (size_t)b->cav[i].grid.nx * b->cav[i].grid.ny;
    double *st = reinterpret_cast<double *>(h->base + h->L.stage);
    if (int r = bcheck_h(b, h, join_in(h))) return r;
    double *outs[2][2] = {{rho, u}, {v, T}};
    cudaError_t e = cudaSuccess;
    for (int which = 0; which < 2 && e == cudaSuccess; which++) {
        if (!outs[which][0] && !outs[which][1]) continue;
        switch (h->prec) {
            case LBMFVM_F64: launch_cav_fields<double, double>(b, i, which, st, st + n); break;
            case LBMFVM_F32: launch_cav_fields<float, double>(b, i, which, st, st + n); break;
            case LBMFVM_F16: launch_cav_fields<__half, double>(b, i, which, st, st + n); break;
            case LBMFVM_BF16: launch_cav_fields<__nv_bfloat16, double>(b, i, which, st, st + n); break;
            case LBMFVM_F32X2: launch_cav_fields<dsf, double>(b, i, which, st, st + n); break;
        }
        e = cudaGetLastError();
        for (int k = 0; k < 2 && e == cudaSuccess; k++)
            if (outs[which][k]) e = cudaMemcpyAsync(outs[which][k], st + k * n, n * sizeof(double), cudaMemcpyDefault, h->s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) return bfail(b, LBMFVM_ERR_CUDA, "batch fields failed: %s", cudaGetErrorString(e));
    if (int r = bcheck_h(b, h, check_device_status(h))) return r;
    return bcheck_h(b, h, join_out(h));
}

int lbmfvm_batch_nusselt(lbmfvm_batch_t *b, int32_t i, double *mean_hot, double *local_hot, double *mean_cold) {
    if (int r = check_index(b, i)) return r;
    lbmfvm_t *h = hnd(b, i);
    if (int r = bcheck_h(b, h, join_in(h))) return r;
    BDISPATCH(h, launch_cav_nusselt, b, i);
    double means[2];
    double *red = reinterpret_cast<double *>(h->base + h->L.red);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(means, reinterpret_cast<double *>(h->base + h->L.cavres) + kCavRes * i + kCavNu, sizeof(means),
                            cudaMemcpyDeviceToHost, h->s);
    if (e == cudaSuccess && local_hot)
        e = cudaMemcpyAsync(local_hot, red + kRedLocal, b->cav[i].grid.ny * sizeof(double),
                            cudaMemcpyDefault, h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) return bfail(b, LBMFVM_ERR_CUDA, "batch Nusselt failed: %s", cudaGetErrorString(e));
    if (mean_hot) *mean_hot = means[0];
    if (mean_cold) *mean_cold = means[1];
    return bcheck_h(b, h, join_out(h));
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

int lbmfvm_batch_substeps(const lbmfvm_batch_t *b, int32_t i, int32_t *substeps) {
    if (!b || !substeps) return fail_thread(LBMFVM_ERR_ARG, "batch or substeps is NULL");
    if (i < 0 || i >= (int)b->cav.size()) return fail_thread(LBMFVM_ERR_ARG, "cavity index %d out of range", i);
    *substeps = b->cav[i].substeps;
    return LBMFVM_OK;
}

int lbmfvm_batch_set_polish(lbmfvm_batch_t *b, int32_t prec, double r_switch, int32_t stall_checks) {
    if (!b) return fail_thread(LBMFVM_ERR_ARG, "batch is NULL");
    if (std::isnan(r_switch)) return bfail(b, LBMFVM_ERR_ARG, "r_switch is NaN");
    for (int l = 0; l + 1 < b->nlv; l++)
        if (b->prec[l] == prec) {
            b->switch_r[l] = r_switch > 0.0 ? r_switch : 0.0;
            b->stall_checks[l] = stall_checks > 0 ? stall_checks : 0;
            return LBMFVM_OK;
        }
    return bfail(b, LBMFVM_ERR_ARG, "precision %d is not a level of this batch's ladder below its top", prec);
}

int lbmfvm_batch_kernel_info(const lbmfvm_batch_t *b, int32_t prec, int32_t *tma_config) {
    if (!b || !tma_config) return fail_thread(LBMFVM_ERR_ARG, "batch or tma_config is NULL");
    *tma_config = -1;
    for (int l = 0; l < b->nlv; l++)
        if (b->prec[l] == prec && b->lv[l]) *tma_config = b->lv[l]->tma_config;
    return LBMFVM_OK;
}

int lbmfvm_batch_precision(const lbmfvm_batch_t *b, int32_t i, int32_t *prec) {
    if (!b || !prec) return fail_thread(LBMFVM_ERR_ARG, "batch or prec is NULL");
    if (i < 0 || i >= (int)b->cav.size()) return fail_thread(LBMFVM_ERR_ARG, "cavity index %d out of range", i);
    *prec = hnd(b, i)->prec;
    return LBMFVM_OK;
}

void lbmfvm_batch_destroy(lbmfvm_batch_t *b) {
    if (!b) return;
    for (int l = 1; l < 3; l++) lbmfvm_destroy(b->lv[l]);
    lbmfvm_destroy(b->a);
    delete b;
}

const char *lbmfvm_batch_last_error(const lbmfvm_batch_t *b) { return b ? b->err : g_err; }

}  // extern "C"
