// Host runtime and C-ABI of the coupled LBM-FVM solver (include/lbmfvm.h).
//
// A handle owns (or borrows, when the caller passes a workspace) one device
// block holding the double-buffered distributions, two temperature planes,
// per-node codes, the residual snapshot and reduction scratch.  Steps run on
// a private non-blocking stream joined to the caller's stream with events,
// so that long runs can replay a captured CUDA graph of many launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include <unistd.h>

#include "kernels.cuh"
#include "lbmfvm.h"

using namespace lbmfvm_dev;

namespace {

constexpr int kGraphSteps = 64;      // launches per captured graph (even)
constexpr int kResidualBlocks = 608; // 4 x 152 SMs
// Reduction scratch (doubles): kResidualSums partials per residual block,
// then the totals, the wall temperatures of the initial state, the two mean
// Nusselt numbers and the local Nusselt numbers of the hot wall.
constexpr int kRedTot = kResidualSums * kResidualBlocks;
constexpr int kRedTwall = kRedTot + 4;
constexpr int kRedNu = kRedTot + 8;
constexpr int kRedLocal = kRedTot + 12;
// Per cavity of a batch: the residual totals, the two mean Nusselt numbers.
constexpr int kCavRes = 8;
constexpr int kCavNu = 4;
constexpr size_t kAlign = 256;

thread_local char g_err[512] = "";

int fail_thread(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Bytes of one temperature value: FP32 next to 32/16-bit storage.
size_t temp_size(int prec) { return prec == LBMFVM_F64 || prec == LBMFVM_F32X2 ? 8 : 4; }

size_t store_size(int prec) {
    switch (prec) {
        case LBMFVM_F64: return 8;
        case LBMFVM_F32: return 4;
        case LBMFVM_F16: return 2;
        case LBMFVM_BF16: return 2;
        case LBMFVM_F32X2: return 8;
    }
    return 0;
}

struct Layout {
    int pitch;
    long long plane;
    size_t f[2], T[2], code, fflags, snap, stage, red, err, cav, tiles, cavres, twall, total;
    size_t tile_cap;  // headers the tile lists hold
    // energy update in sub-steps: velocity planes U, V and the two scratch
    // temperature planes X, Y (0 when the handle takes no sub-steps)
    size_t uv[2], tx[2];
    bool split;
    size_t g[2];  // D2Q5 energy populations [5][ny][pitch] (0 for the FV energy update)
};

Layout make_layout(const lbmfvm_grid_t &g, int prec, int ncav = 1, bool split = false, bool lbm5 = false) {
    Layout L{};
    L.pitch = (int)align_up((size_t)g.nx, 64);
    L.plane = (long long)g.ny * L.pitch;
    const size_t ss = store_size(prec), cs = temp_size(prec);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, kAlign);
        return o;
    };
    L.f[0] = take(9 * (size_t)L.plane * ss);
    L.f[1] = take(9 * (size_t)L.plane * ss);
    L.T[0] = take((size_t)L.plane * cs);
    L.T[1] = take((size_t)L.plane * cs);
    if (lbm5)
        for (int i = 0; i < 2; i++) L.g[i] = take(5 * (size_t)L.plane * ss);
    L.split = split;
    if (split)
        for (int i = 0; i < 2; i++) {
            L.uv[i] = take((size_t)L.plane * cs);
            L.tx[i] = take((size_t)L.plane * cs);
        }
    L.code = take((size_t)L.plane);
    L.fflags = take((size_t)L.plane);  // face flags of the finite-volume update
    L.snap = take(2 * (size_t)g.nx * g.ny * sizeof(double));
    L.stage = take(2 * (size_t)g.nx * g.ny * sizeof(double));
    L.red = take((kRedLocal + (size_t)g.ny) * sizeof(double));
    L.err = take(16);
    // cavity table (one entry) and tile list of the TMA kernel (tiles of at
    // least 64 x 8 nodes), plus the tile count
    L.cav = take(ncav * sizeof(CavityDesc));
    L.cavres = take(ncav * kCavRes * sizeof(double));
    L.twall = take(ncav * 4 * sizeof(double));   // per cavity: wall temperatures W, E, S, N
    // enough for the smallest tile shape (32 x 8) of every configuration
    const size_t max_tiles = ((size_t)g.nx + 31) / 32 * (((size_t)g.ny + 7) / 8);
    L.tile_cap = max_tiles;
    // two lists (fused step; sub-step path), each a count slot and its headers
    L.tiles = take((max_tiles + 2) * sizeof(TileHeader));
    L.total = off;
    return L;
}

int check_grid(const lbmfvm_grid_t *g) {
    if (!g) return fail_thread(LBMFVM_ERR_ARG, "grid is NULL");
    if (g->nx < 3 || g->ny < 3) return fail_thread(LBMFVM_ERR_ARG, "nx and ny must be >= 3 (got %d x %d)", g->nx, g->ny);
    if ((long long)g->nx * g->ny > (1LL << 30))
        return fail_thread(LBMFVM_ERR_ARG, "grid of %d x %d nodes exceeds 2^30 nodes", g->nx, g->ny);
    for (int s = 0; s < 4; s++)
        if (g->bc[s] < LBMFVM_BC_DIRICHLET || g->bc[s] > LBMFVM_BC_MOVING)
            return fail_thread(LBMFVM_ERR_ARG, "bc[%d] = %d is not a LBMFVM_BC_* value", s, g->bc[s]);
    if ((g->bc[0] == LBMFVM_BC_PERIODIC) != (g->bc[1] == LBMFVM_BC_PERIODIC) ||
        (g->bc[2] == LBMFVM_BC_PERIODIC) != (g->bc[3] == LBMFVM_BC_PERIODIC))
        return fail_thread(LBMFVM_ERR_ARG, "periodic sides must come in opposite pairs");
    return LBMFVM_OK;
}

// ---------------------------------------------------------------------------
// Node classification (boundary treatment of the non-equilibrium
// extrapolation scheme, Eqs. 94 and 96; thermal conditions Eqs. 77-80).
//   box-border nodes of non-periodic sides -> wall, partner = inward normal
//   neighbour (inward diagonal at corners);
//   mask-solid nodes with a fluid 8-neighbour -> obstacle wall, partner = first
//   fluid neighbour in the order E, N, W, S, NE, NW, SW, SE (the same search is
//   the fallback of a box wall whose normal neighbour is not fluid);
//   walls without any fluid neighbour -> inert.
// Thermal roles: Dirichlet on DIRICHLET sides (vertical sides own corners,
// a corner is Dirichlet if either side is), obstacle nodes copy their
// partner's temperature, everything else is a finite-volume node.
// ---------------------------------------------------------------------------
std::vector<uint8_t> classify(const lbmfvm_grid_t &g, const uint8_t *mask, int pitch) {
    const int nx = g.nx, ny = g.ny;
    const bool perx = g.bc[LBMFVM_SIDE_W] == LBMFVM_BC_PERIODIC;
    const bool pery = g.bc[LBMFVM_SIDE_S] == LBMFVM_BC_PERIODIC;
    auto at = [&](int i, int j) { return (size_t)j * nx + i; };
    auto onW = [&](int i) { return !perx && i == 0; };
    auto onE = [&](int i) { return !perx && i == nx - 1; };
    auto onS = [&](int j) { return !pery && j == 0; };
    auto onN = [&](int j) { return !pery && j == ny - 1; };
    auto neighbour = [&](int i, int j, int dx, int dy, int &a, int &b) {
        a = i + dx;
        b = j + dy;
        if (a < 0 || a >= nx) {
            if (!perx) return false;
            a = (a + nx) % nx;
        }
        if (b < 0 || b >= ny) {
            if (!pery) return false;
            b = (b + ny) % ny;
        }
        return true;
    };
    std::vector<uint8_t> kind(g.nx * (size_t)g.ny), dir(kind.size(), 0);
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const bool solid = mask && mask[at(i, j)];
            const bool border = onW(i) || onE(i) || onS(j) || onN(j);
            kind[at(i, j)] = (solid || border) ? KIND_WALL : KIND_FLUID;
        }
    auto dir_of = [](int dx, int dy) {
        for (int q = 1; q < 9; q++)
            if (cx(q) == dx && cy(q) == dy) return q;
        return 0;
    };
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const size_t k = at(i, j);
            if (kind[k] != KIND_WALL) continue;
            const bool solid = mask && mask[k];
            int d = 0, a, b;
            if (!solid) {
                const int dx = onW(i) ? 1 : (onE(i) ? -1 : 0);
                const int dy = onS(j) ? 1 : (onN(j) ? -1 : 0);
                if (neighbour(i, j, dx, dy, a, b) && kind[at(a, b)] == KIND_FLUID) d = dir_of(dx, dy);
            }
            for (int q = 1; q < 9 && d == 0; q++)
                if (neighbour(i, j, cx(q), cy(q), a, b) && kind[at(a, b)] == KIND_FLUID) d = q;
            dir[k] = (uint8_t)d;
        }
    std::vector<uint8_t> code((size_t)ny * pitch, CODE_OUTSIDE);
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const size_t k = at(i, j);
            int kd = kind[k];
            if (kd == KIND_WALL && dir[k] == 0) kd = KIND_SOLID;
            int th;
            if (kd == KIND_SOLID) th = TH_INERT;
            else if (mask && mask[k]) th = TH_OBSTACLE;
            else {
                const int vert = onW(i) ? LBMFVM_SIDE_W : (onE(i) ? LBMFVM_SIDE_E : -1);
                const int hor = onS(j) ? LBMFVM_SIDE_S : (onN(j) ? LBMFVM_SIDE_N : -1);
                const bool dv = vert >= 0 && g.bc[vert] == LBMFVM_BC_DIRICHLET;
                const bool dh = hor >= 0 && g.bc[hor] == LBMFVM_BC_DIRICHLET;
                th = (dv || dh) ? TH_DIRICHLET : TH_FV;
            }
            code[(size_t)j * pitch + i] = make_code(kd, kd == KIND_WALL ? dir[k] : 0, th);
        }
    for (auto &c : code) c = stored_code(c);
    return code;
}

// CRC-32 of n bytes continued from crc (0 to start); defined with the
// checkpoint code.
uint32_t crc32_update(uint32_t crc, const void *data, size_t n);

// Face flags (FF_* bits) of every node of the given cavity rectangles of a
// stored-code plane: the finite-volume update's control volume is clipped to
// its cavity, and a face is open when the neighbour across it lies in the
// cavity and is a finite-volume or Dirichlet node.
std::vector<uint8_t> face_flags(const std::vector<uint8_t> &stored, int pitch, const std::vector<CavityDesc> &rects) {
    std::vector<uint8_t> ff(stored.size(), 0);
    for (const CavityDesc &r : rects)
        for (int j = 0; j < r.ny; j++)
            for (int i = 0; i < r.nx; i++) {
                const size_t k = (size_t)(r.y0 + j) * pitch + (r.x0 + i);
                auto open = [&](long long off) { return fv_open(decode(stored[(size_t)((long long)k + off)])); };
                uint8_t f = 0;
                if (i > 0) f |= FF_IN_W | (open(-1) ? FF_OPEN_W : 0);
                if (i < r.nx - 1) f |= FF_IN_E | (open(1) ? FF_OPEN_E : 0);
                if (j > 0) f |= FF_IN_S | (open(-(long long)pitch) ? FF_OPEN_S : 0);
                if (j < r.ny - 1) f |= FF_IN_N | (open(pitch) ? FF_OPEN_N : 0);
                ff[k] = f;
            }
    return ff;
}

}  // namespace

namespace lbmfvm_internal {
// Record a failure message for lbmfvm_last_error(NULL) from another
// translation unit of the library.
int fail_thread_msg(int code, const char *msg) { return fail_thread(code, "%s", msg); }
}  // namespace lbmfvm_internal

struct lbmfvm {
    lbmfvm_grid_t grid;
    int prec;
    int tile_y;
    Layout L;
    double nu, alpha, gbeta, tau, t_ref, force[2];
    unsigned char *base;
    bool owns;
    cudaStream_t user;
    cudaStream_t s;
    cudaEvent_t ev_in, ev_out;
    int parity;       // buffer holding the current post-collision state
    int64_t steps;    // steps since set_state
    cudaGraphExec_t graph;
    int64_t launches; // step-kernel launches issued (a graph replay counts its kernel nodes)
    bool use_tma;     // persistent TMA kernel (walled domains, 32/16-bit storage)
    bool stall_next;  // test hook armed by lbmfvm_inject_stall
    int tma_config;   // tile shape of the TMA kernel
    int num_sms;
    CUtensorMap map_f[2], map_T[2], map_c;
    CUtensorMap map_fo[2], map_To[2];  // output-tile boxes of the TMA tile kernel
    int tma_blocks_per_sm;
    int tma_stages;   // pipeline stages of the tile shape in use
    int ntiles;       // tiles of the fused list (cavities with one energy update per step)
    int ntiles_split; // tiles of the sub-step list
    // tiles of the sub-step list taking part in sub-step s + 1 (the list is
    // sorted by sub-steps, largest first); its size is the largest count
    std::vector<int> split_tiles_at;
    bool fv_quick;    // QUICK face values instead of central ones
    int fv_sub;       // sub-steps of a single cavity (batches: per cavity)
    int blocks_quick, blocks_given;  // blocks per SM of the QUICK and given-temperature kernels
    CUtensorMap map_TX;              // temperature box of the sub-steps' result plane X
    int energy;                      // LBMFVM_ENERGY_*
    int wall_bc;                     // LBMFVM_WALL_*
    bool grid2;                      // energy balance on the coarse volumes of grid setting 2
    int fv_every;                    // lattice steps per coarse energy step
    int ncx, ncy;                    // coarse volumes
    uint64_t tiles_gen, graph_gen;   // tile-list generation, and the one the graph was captured with
    uint32_t code_crc; // CRC-32 of the node codes, identifies the geometry in checkpoints
    int tile_w, tile_h;
    // Several cavities packed in one grid (batch handles); empty for one cavity.
    std::vector<CavityDesc> atlas_cavs;
    std::vector<char> atlas_active;
    char err[512];
};

namespace {

int fail(lbmfvm_t *h, int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof(h->err), fmt, ap);
    va_end(ap);
    snprintf(g_err, sizeof(g_err), "%s", h->err);
    return code;
}

#define CU(h, call)                                                                         \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail((h), LBMFVM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <class S>
StepArgs<S> args_for(const lbmfvm_t *h, int cur) {
    using C = typename Compute<S>::type;
    StepArgs<S> a{};
    a.fin = reinterpret_cast<const S *>(h->base + h->L.f[cur]);
    a.fout = reinterpret_cast<S *>(h->base + h->L.f[cur ^ 1]);
    a.Tin = reinterpret_cast<const C *>(h->base + h->L.T[cur]);
    a.Tout = reinterpret_cast<C *>(h->base + h->L.T[cur ^ 1]);
    a.code = h->base + h->L.code;
    a.err = reinterpret_cast<int *>(h->base + h->L.err);
    a.nx = h->grid.nx;
    a.ny = h->grid.ny;
    a.pitch = h->L.pitch;
    a.plane = h->L.plane;
    a.perx = h->grid.bc[LBMFVM_SIDE_W] == LBMFVM_BC_PERIODIC;
    a.pery = h->grid.bc[LBMFVM_SIDE_S] == LBMFVM_BC_PERIODIC;
    a.omega = C(1.0 / h->tau);
    a.alpha = C(h->alpha);
    a.gbeta = C(h->gbeta);
    a.t_ref = C(h->t_ref);
    a.fx = C(h->force[0]);
    a.fy = C(h->force[1]);
    a.wall_fd = h->wall_bc == LBMFVM_WALL_FD;
    a.fd_coef = C(3.0 * h->tau);
    for (int s = 0; s < 4; s++) {
        const bool moving = h->grid.bc[s] == LBMFVM_BC_MOVING;
        const bool vertical = s < 2;
        a.wall_u[s] = C(moving && !vertical ? h->grid.u_lid : 0.0);
        a.wall_v[s] = C(moving && vertical ? h->grid.u_lid : 0.0);
    }
    return a;
}

template <class S, int TY>
void launch_step_ty(const lbmfvm_t *h, int cur, cudaStream_t s) {
    const StepArgs<S> a = args_for<S>(h, cur);
    dim3 block(32, TY), grid((h->grid.nx + 31) / 32, (h->grid.ny + TY - 1) / TY);
    step_kernel<S, TY><<<grid, block, 0, s>>>(a);
}


// The handle's two tile lists, one after the other in the workspace: the
// cavities stepped by the fused kernel (one energy update per step), then
// those whose energy update takes sub-steps (sorted by their number, largest
// first).  Each list starts with a count slot, whose next two words are the
// step kernel's tile counters (one per step parity).
struct TileList {
    size_t slot;  // workspace offset of the count slot; the headers follow
    int n;        // tiles
};
TileList list_fused(const lbmfvm_t *h) { return {h->L.tiles, h->ntiles}; }
TileList list_split(const lbmfvm_t *h) {
    return {h->L.tiles + (size_t)(h->ntiles + 1) * sizeof(TileHeader), h->ntiles_split};
}

// Persistent grid of the TMA kernel: one block per resident slot, or one per
// tile when there are fewer tiles.
int tma_grid_for(const lbmfvm_t *h, int ntiles, int per_sm) {
    const int resident = h->num_sms * per_sm;
    return ntiles < resident ? ntiles : resident;
}

// Tiles a block of the TMA kernel takes in a fixed order before it draws the
// rest from the shared counter: all but the last kTilesDrawn rounds.
constexpr int kTilesDrawn = 2;
int fixed_tiles(int ntiles, int blocks, int stages) {
    const int per = blocks > 0 ? ntiles / blocks : 0;
    return std::max(stages + 1, per - kTilesDrawn);
}

// Launch arguments of the TMA kernel over one tile list at step parity cur,
// its temperature box loaded through map_T.
template <class S>
lbmfvm_fv::TmaLaunch<S> tma_args(const lbmfvm_t *h, int cur, TileList list, const CUtensorMap *map_T, int per_sm,
                                 int stages, cudaStream_t s, bool stall) {
    lbmfvm_fv::TmaLaunch<S> l{};
    l.a = args_for<S>(h, cur);
    l.a.stall = stall ? 1 : 0;
    l.cavs = reinterpret_cast<const CavityDesc *>(h->base + h->L.cav);
    // the count sits at a fixed address in front of the list, so that a
    // captured graph reads the current count after the list has changed
    int *count = reinterpret_cast<int *>(h->base + list.slot);
    l.count = count;
    l.tiles = reinterpret_cast<const TileHeader *>(h->base + list.slot) + 1;
    l.map_f = &h->map_f[cur];
    l.map_T = map_T;
    l.map_c = &h->map_c;
    l.map_fo = &h->map_fo[cur ^ 1];
    l.map_To = &h->map_To[cur ^ 1];
    l.ctr = count + 1 + cur;
    l.ctr_next = count + 1 + (cur ^ 1);
    l.blocks = tma_grid_for(h, list.n, per_sm);
    l.nfix = fixed_tiles(list.n, l.blocks, stages);
    l.stream = s;
    return l;
}

// The cavities of the sub-step list: velocity pass, the sub-steps, then the
// collision with the temperature the last sub-step left in plane X.
template <class S>
void launch_split(const lbmfvm_t *h, int cur, cudaStream_t s) {
    using C = typename Compute<S>::type;
    using G = typename TmaConfig<S, kTmaConfigFv>::G;
    const TileList list = list_split(h);
    if (list.n < 1) return;
    const TileHeader *tiles = reinterpret_cast<const TileHeader *>(h->base + list.slot) + 1;
    const CavityDesc *cavs = reinterpret_cast<const CavityDesc *>(h->base + h->L.cav);
    C *U = reinterpret_cast<C *>(h->base + h->L.uv[0]);
    C *V = reinterpret_cast<C *>(h->base + h->L.uv[1]);
    C *X = reinterpret_cast<C *>(h->base + h->L.tx[0]);
    C *Y = reinterpret_cast<C *>(h->base + h->L.tx[1]);
    const C *T0 = reinterpret_cast<const C *>(h->base + h->L.T[cur]);
    const S *fin = reinterpret_cast<const S *>(h->base + h->L.f[cur]);
    lbmfvm_fv::launch_uv<S>(fin, h->L.plane, h->L.pitch, h->grid.nx, h->grid.ny, tiles, list.n, cavs,
                            h->base + h->L.code, U, V, h->tile_w, h->tile_h, s);
    for (int sub = 1; sub <= (int)h->split_tiles_at.size(); sub++)
        lbmfvm_fv::launch_substep<C>(h->fv_quick, T0, X, Y, U, V, h->base + h->L.code, h->base + h->L.fflags,
                                     h->L.pitch, h->grid.nx, h->grid.ny, tiles, h->split_tiles_at[sub - 1],
                                     h->tile_w, h->tile_h, sub, s);
    lbmfvm_fv::launch_given<S>(tma_args<S>(h, cur, list, &h->map_TX, h->blocks_given, G::STAGES, s, false));
}

Grid2Args grid2_args(const lbmfvm_t *h) {
    Grid2Args g{};
    g.nx = h->grid.nx;
    g.ny = h->grid.ny;
    g.pitch = h->L.pitch;
    g.ncx = h->ncx;
    g.ncy = h->ncy;
    for (int sd = 0; sd < 4; sd++) {
        g.dirichlet[sd] = h->grid.bc[sd] == LBMFVM_BC_DIRICHLET;
        g.t_wall[sd] = h->grid.t_wall[sd];
    }
    return g;
}

// Grid setting 2: on a coarse step the velocity pass, the coarse energy step
// and the node temperatures from the volumes; every step the collision with
// the node temperatures (plane X).
template <class S>
void launch_grid2(const lbmfvm_t *h, int cur, cudaStream_t s, bool fv_now) {
    using C = typename Compute<S>::type;
    using G = typename TmaConfig<S, kTmaConfigFv>::G;
    const TileList list = list_split(h);
    if (list.n < 1) return;
    const TileHeader *tiles = reinterpret_cast<const TileHeader *>(h->base + list.slot) + 1;
    const CavityDesc *cavs = reinterpret_cast<const CavityDesc *>(h->base + h->L.cav);
    C *U = reinterpret_cast<C *>(h->base + h->L.uv[0]);
    C *V = reinterpret_cast<C *>(h->base + h->L.uv[1]);
    C *X = reinterpret_cast<C *>(h->base + h->L.tx[0]);
    C *Tc = reinterpret_cast<C *>(h->base + h->L.tx[1]);
    C *Tn = Tc + (size_t)h->ncx * h->ncy;
    if (fv_now) {
        const S *fin = reinterpret_cast<const S *>(h->base + h->L.f[cur]);
        lbmfvm_fv::launch_uv<S>(fin, h->L.plane, h->L.pitch, h->grid.nx, h->grid.ny, tiles, list.n, cavs,
                                h->base + h->L.code, U, V, h->tile_w, h->tile_h, s);
        const Grid2Args g = grid2_args(h);
        dim3 b(16, 16), gc((h->ncx + 15) / 16, (h->ncy + 15) / 16), gn((h->grid.nx + 15) / 16, (h->grid.ny + 15) / 16);
        grid2_step_kernel<C><<<gc, b, 0, s>>>(g, Tc, Tn, U, V, C(h->alpha), C((double)h->fv_every));
        const C *Tdir = reinterpret_cast<const C *>(h->base + h->L.T[cur]);
        grid2_nodes_kernel<C><<<gn, b, 0, s>>>(g, h->base + h->L.code, Tdir, Tn, Tc, X, nullptr, nullptr);
    }
    lbmfvm_fv::launch_given<S>(tma_args<S>(h, cur, list, &h->map_TX, h->blocks_given, G::STAGES, s, false));
}

template <class S>
void launch_step_tma(const lbmfvm_t *h, int cur, cudaStream_t s, bool stall, bool fv_now) {
    if (h->fv_quick) {
        using G = typename TmaConfig<S, kTmaConfigFv>::G;
        lbmfvm_fv::launch_quick<S>(
            tma_args<S>(h, cur, list_fused(h), &h->map_T[cur], h->blocks_quick, G::STAGES, s, stall));
    } else {
        lbmfvm_fv::tma_launch<S>(h->tma_config, tma_args<S>(h, cur, list_fused(h), &h->map_T[cur],
                                                            h->tma_blocks_per_sm, h->tma_stages, s, stall));
    }
    if (h->grid2) launch_grid2<S>(h, cur, s, fv_now);
    else if (h->L.split) launch_split<S>(h, cur, s);
}

template <class S>
void launch_step(const lbmfvm_t *h, int cur, cudaStream_t s, bool stall, bool fv_now) {
    if (h->use_tma) {
        launch_step_tma<S>(h, cur, s, stall, fv_now);
        return;
    }
    switch (h->tile_y) {
        case 4: launch_step_ty<S, 4>(h, cur, s); break;
        case 16: launch_step_ty<S, 16>(h, cur, s); break;
        default: launch_step_ty<S, 8>(h, cur, s); break;
    }
}

// Shift T_0 of the stored D2Q5 populations: the mean wall temperature of the
// west and east sides.
double lbm5_shift(const lbmfvm_t *h) { return 0.5 * (h->grid.t_wall[LBMFVM_SIDE_W] + h->grid.t_wall[LBMFVM_SIDE_E]); }

// One step of the D2Q5 thermal lattice-Boltzmann energy solver.
template <class S>
void launch_lbm5(const lbmfvm_t *h, int cur, cudaStream_t s) {
    using C = typename Compute<S>::type;
    Lbm5Args<S> p{};
    p.a = args_for<S>(h, cur);
    p.gin = reinterpret_cast<const S *>(h->base + h->L.g[cur]);
    p.gout = reinterpret_cast<S *>(h->base + h->L.g[cur ^ 1]);
    p.omega_T = C(1.0 / (3.0 * h->alpha + 0.5));  // tau_T = alpha / c_s^2 + 1/2 (Eq. 20)
    p.T0 = C(lbm5_shift(h));
    dim3 block(32, 8), grid((h->grid.nx + 31) / 32, (h->grid.ny + 7) / 8);
    step_lbm5_kernel<S><<<grid, block, 0, s>>>(p);
}

// One coupled step at parity cur; fv_now: grid setting 2 takes its coarse
// energy step in this one.
void launch_one(const lbmfvm_t *h, int cur, cudaStream_t s, bool stall = false, bool fv_now = true) {
    if (h->energy == LBMFVM_ENERGY_LBM_D2Q5) {
        switch (h->prec) {
            case LBMFVM_F64: launch_lbm5<double>(h, cur, s); break;
            case LBMFVM_F32X2: launch_lbm5<dsf>(h, cur, s); break;
            default: launch_lbm5<float>(h, cur, s); break;
        }
        return;
    }
    switch (h->prec) {
        case LBMFVM_F64: launch_step<double>(h, cur, s, stall, fv_now); break;
        case LBMFVM_F32: launch_step<float>(h, cur, s, stall, fv_now); break;
        case LBMFVM_F16: launch_step<__half>(h, cur, s, stall, fv_now); break;
        case LBMFVM_BF16: launch_step<__nv_bfloat16>(h, cur, s, stall, fv_now); break;
        case LBMFVM_F32X2: launch_step<dsf>(h, cur, s, stall, fv_now); break;
    }
}

int join_in(lbmfvm_t *h) {
    CU(h, cudaEventRecord(h->ev_in, h->user));
    CU(h, cudaStreamWaitEvent(h->s, h->ev_in, 0));
    return LBMFVM_OK;
}

int join_out(lbmfvm_t *h) {
    CU(h, cudaEventRecord(h->ev_out, h->s));
    CU(h, cudaStreamWaitEvent(h->user, h->ev_out, 0));
    return LBMFVM_OK;
}

int build_graph(lbmfvm_t *h) {
    cudaGraph_t g = nullptr;
    CU(h, cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
    // a graph starts at a step count that is a multiple of the coarse step
    // interval (which divides kGraphSteps), so its coarse steps sit at fixed places
    for (int i = 0; i < kGraphSteps; i++) launch_one(h, i & 1, h->s, false, (i + 1) % h->fv_every == 0);
    cudaError_t e = cudaStreamEndCapture(h->s, &g);
    if (e != cudaSuccess) return fail(h, LBMFVM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return fail(h, LBMFVM_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    h->graph_gen = h->tiles_gen;
    return LBMFVM_OK;
}

template <class S>
void launch_init(lbmfvm_t *h, const float *u0, const float *v0, const float *T0) {
    using C = typename Compute<S>::type;
    StepArgs<S> a = args_for<S>(h, 0);
    S *fstar = reinterpret_cast<S *>(h->base + h->L.f[0]);
    S *f0 = reinterpret_cast<S *>(h->base + h->L.f[1]);
    C *Ta = reinterpret_cast<C *>(h->base + h->L.T[0]);
    C *Tb = reinterpret_cast<C *>(h->base + h->L.T[1]);
    double *tw = reinterpret_cast<double *>(h->base + h->L.red) + kRedTwall;
    dim3 block(32, 8), grid((h->grid.nx + 31) / 32, (h->grid.ny + 7) / 8);
    init_kernel<S><<<grid, block, 0, h->s>>>(a, f0, fstar, u0, v0, T0, h->grid.t_init, tw, h->grid.bc[0],
                                             h->grid.bc[1], h->grid.bc[2], h->grid.bc[3], Ta, Tb);
    if (h->energy == LBMFVM_ENERGY_LBM_D2Q5)
        init_lbm5_kernel<S><<<grid, block, 0, h->s>>>(a, f0, reinterpret_cast<S *>(h->base + h->L.g[0]),
                                                      reinterpret_cast<S *>(h->base + h->L.g[1]), C(lbm5_shift(h)));
}

// Arguments of the kernels that read the state of the current step: the
// buffer with the previous post-collision populations (or the unrelaxed
// initial populations at step 0) and the current temperature.
template <class S>
StepArgs<S> read_args(const lbmfvm_t *h, int &direct) {
    direct = h->steps == 0;
    StepArgs<S> a = args_for<S>(h, h->parity);
    const int prev = h->parity ^ 1;  // f*^{n-1}, or f^0 at step 0
    a.fin = reinterpret_cast<const S *>(h->base + h->L.f[prev]);
    return a;
}

template <class S>
void launch_residual(lbmfvm_t *h, int update_only) {
    int direct;
    StepArgs<S> a = read_args<S>(h, direct);
    double *su = reinterpret_cast<double *>(h->base + h->L.snap);
    double *sv = su + (size_t)h->grid.nx * h->grid.ny;
    double *red = reinterpret_cast<double *>(h->base + h->L.red);
    residual_kernel<S><<<kResidualBlocks, 256, 0, h->s>>>(a, direct, su, sv, red, update_only);
    if (!update_only) residual_finish_kernel<<<1, 32, 0, h->s>>>(red, kResidualBlocks, red + kRedTot);
}

template <class S, class O>
void launch_fields(lbmfvm_t *h, int which, O *o0, O *o1) {
    int direct;
    StepArgs<S> a = read_args<S>(h, direct);
    dim3 block(32, 8), grid((h->grid.nx + 31) / 32, (h->grid.ny + 7) / 8);
    fields_kernel<S, O><<<grid, block, 0, h->s>>>(a, direct, which, o0, o1);
}

template <class S>
void launch_nusselt(lbmfvm_t *h) {
    StepArgs<S> a = args_for<S>(h, h->parity);
    double *red = reinterpret_cast<double *>(h->base + h->L.red);
    const double dT = h->grid.t_wall[LBMFVM_SIDE_W] - h->grid.t_wall[LBMFVM_SIDE_E];
    nusselt_kernel<S><<<1, 256, 0, h->s>>>(a, (double)(h->grid.ny - 1), dT, red + kRedLocal, red + kRedNu);
}

// Mass renormalisation of the current state (both population buffers) from
// the totals of the last residual pass.
template <class S>
void launch_rescale(lbmfvm_t *h) {
    StepArgs<S> a = args_for<S>(h, h->parity);
    S *f0 = reinterpret_cast<S *>(h->base + h->L.f[0]);
    S *f1 = reinterpret_cast<S *>(h->base + h->L.f[1]);
    const double *tot = reinterpret_cast<const double *>(h->base + h->L.red) + kRedTot;
    dim3 block(32, 8), grid((h->grid.nx + 31) / 32, (h->grid.ny + 7) / 8, 2);
    rescale_kernel<S><<<grid, block, 0, h->s>>>(a, f0, f1, tot);
}

#define DISPATCH(h, FN, ...)                                          \
    do {                                                              \
        switch ((h)->prec) {                                          \
            case LBMFVM_F64: FN<double>(__VA_ARGS__); break;          \
            case LBMFVM_F32: FN<float>(__VA_ARGS__); break;           \
            case LBMFVM_F16: FN<__half>(__VA_ARGS__); break;          \
            case LBMFVM_BF16: FN<__nv_bfloat16>(__VA_ARGS__); break;  \
            case LBMFVM_F32X2: FN<dsf>(__VA_ARGS__); break;           \
        }                                                             \
    } while (0)

int clear_tile_counters(lbmfvm_t *h);

// Grid setting 2 at set_state: the volumes from the node temperatures at
// their centres, then the node temperatures (plane X and both state planes)
// from the volumes, as the oracle starts.
template <class S>
void launch_grid2_init(lbmfvm_t *h) {
    using C = typename Compute<S>::type;
    C *X = reinterpret_cast<C *>(h->base + h->L.tx[0]);
    C *Tc = reinterpret_cast<C *>(h->base + h->L.tx[1]);
    C *Tn = Tc + (size_t)h->ncx * h->ncy;
    C *Ta = reinterpret_cast<C *>(h->base + h->L.T[0]);
    C *Tb = reinterpret_cast<C *>(h->base + h->L.T[1]);
    const Grid2Args g = grid2_args(h);
    dim3 b(16, 16), gc((h->ncx + 15) / 16, (h->ncy + 15) / 16), gn((h->grid.nx + 15) / 16, (h->grid.ny + 15) / 16);
    grid2_gather_kernel<C><<<gc, b, 0, h->s>>>(g, Ta, Tn);
    grid2_nodes_kernel<C><<<gn, b, 0, h->s>>>(g, h->base + h->L.code, Ta, Tn, Tc, X, Ta, Tb);
}

int set_state_impl(lbmfvm_t *h, const float *u, const float *v, const float *T) {
    const size_t n = (size_t)h->grid.nx * h->grid.ny;
    float *stage = reinterpret_cast<float *>(h->base + h->L.stage);
    const float *du = nullptr, *dv = nullptr, *dT = nullptr;
    if (int r = join_in(h)) return r;
    if (u) { CU(h, cudaMemcpyAsync(stage, u, n * sizeof(float), cudaMemcpyDefault, h->s)); du = stage; }
    if (v) { CU(h, cudaMemcpyAsync(stage + n, v, n * sizeof(float), cudaMemcpyDefault, h->s)); dv = stage + n; }
    if (T) { CU(h, cudaMemcpyAsync(stage + 2 * n, T, n * sizeof(float), cudaMemcpyDefault, h->s)); dT = stage + 2 * n; }
    double tw[4];
    for (int s = 0; s < 4; s++) tw[s] = h->grid.t_wall[s];
    double *dtw = reinterpret_cast<double *>(h->base + h->L.red) + kRedTwall;
    CU(h, cudaMemcpyAsync(dtw, tw, sizeof(tw), cudaMemcpyHostToDevice, h->s));
    DISPATCH(h, launch_init, h, du, dv, dT);
    CU(h, cudaGetLastError());
    if (h->grid2) {
        DISPATCH(h, launch_grid2_init, h);
        CU(h, cudaGetLastError());
    }
    h->parity = 0;
    h->steps = 0;
    if (int r = clear_tile_counters(h)) return r;
    DISPATCH(h, launch_residual, h, 1);  // snapshot := u^0
    CU(h, cudaGetLastError());
    // The host copy of the wall temperatures and the staged inputs must stay
    // valid until the kernels above have read them.
    CU(h, cudaStreamSynchronize(h->s));
    return join_out(h);
}

// Converts both population buffers and both temperature buffers of a
// rectangle of `src` (origin off_s) into `dst` (origin off_d); flip swaps the
// buffers' indices when the handles stand at opposite parities.
template <class S, class D>
void launch_convert(const lbmfvm_t *src, lbmfvm_t *dst, long long off_s, long long off_d, int nx, int ny, int flip) {
    using CS = typename Compute<S>::type;
    using CD = typename Compute<D>::type;
    const S *fs0 = reinterpret_cast<const S *>(src->base + src->L.f[0]) + off_s;
    const S *fs1 = reinterpret_cast<const S *>(src->base + src->L.f[1]) + off_s;
    const CS *Ts0 = reinterpret_cast<const CS *>(src->base + src->L.T[0]) + off_s;
    const CS *Ts1 = reinterpret_cast<const CS *>(src->base + src->L.T[1]) + off_s;
    D *fd0 = reinterpret_cast<D *>(dst->base + dst->L.f[0]) + off_d;
    D *fd1 = reinterpret_cast<D *>(dst->base + dst->L.f[1]) + off_d;
    CD *Td0 = reinterpret_cast<CD *>(dst->base + dst->L.T[0]) + off_d;
    CD *Td1 = reinterpret_cast<CD *>(dst->base + dst->L.T[1]) + off_d;
    dim3 block(32, 8), grid((nx + 31) / 32, (ny + 7) / 8, 2);
    convert_kernel<S, D><<<grid, block, 0, dst->s>>>(fs0, fs1, Ts0, Ts1, src->L.pitch, src->L.plane, fd0, fd1, Td0,
                                                      Td1, dst->L.pitch, dst->L.plane, nx, ny, flip);
}

template <class S>
void launch_convert_from(const lbmfvm_t *src, lbmfvm_t *dst, long long off_s, long long off_d, int nx, int ny,
                         int flip) {
    switch (dst->prec) {
        case LBMFVM_F64: launch_convert<S, double>(src, dst, off_s, off_d, nx, ny, flip); break;
        case LBMFVM_F32: launch_convert<S, float>(src, dst, off_s, off_d, nx, ny, flip); break;
        case LBMFVM_F16: launch_convert<S, __half>(src, dst, off_s, off_d, nx, ny, flip); break;
        case LBMFVM_BF16: launch_convert<S, __nv_bfloat16>(src, dst, off_s, off_d, nx, ny, flip); break;
        case LBMFVM_F32X2: launch_convert<S, dsf>(src, dst, off_s, off_d, nx, ny, flip); break;
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no
// link-time dependency on the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

template <class S> constexpr CUtensorMapDataType tmap_type() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> constexpr CUtensorMapDataType tmap_type<double>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT64; }
// double-single pairs travel as opaque 8-byte words (zero fill = 0 + 0)
template <> constexpr CUtensorMapDataType tmap_type<dsf>() { return CU_TENSOR_MAP_DATA_TYPE_UINT64; }
template <> constexpr CUtensorMapDataType tmap_type<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }
template <> constexpr CUtensorMapDataType tmap_type<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }

template <class S>
int encode_maps(lbmfvm_t *h, int fw, int fh, int tw, int th, int cw, int ch, size_t t_plane = 0);
int upload_tiles(lbmfvm_t *h, int tw, int th);
CavityDesc single_cavity_desc(const lbmfvm_t *h);

template <class S>
int setup_tma(lbmfvm_t *h) {
    lbmfvm_fv::TmaShape g{};
    int per_sm = 0;
    CU(h, lbmfvm_fv::tma_prepare<S>(h->tma_config, &g, &per_sm));
    // output boxes first: encode_maps() leaves the load boxes in map_f/map_T
    if (int r = encode_maps<S>(h, g.TW, g.TH, g.TW, g.TH, g.CWD, g.CHT)) return r;
    for (int b = 0; b < 2; b++) {
        h->map_fo[b] = h->map_f[b];
        h->map_To[b] = h->map_T[b];
    }
    if (h->L.split) {
        // the given-temperature kernel loads plane X with the central box
        if (int r = encode_maps<S>(h, g.FW, g.FH, g.TWD, g.THT, g.CWD, g.CHT, h->L.tx[0])) return r;
        h->map_TX = h->map_T[0];
    }
    // QUICK's fused kernel reaches two rows beyond the tile for temperatures
    const int tht = h->fv_quick ? g.THT_QUICK : g.THT;
    if (int r = encode_maps<S>(h, g.FW, g.FH, g.TWD, tht, g.CWD, g.CHT)) return r;
    int dev = 0;
    CU(h, cudaGetDevice(&dev));
    CU(h, cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) return fail(h, LBMFVM_ERR_CUDA, "TMA tile kernel does not fit on an SM");
    h->tma_blocks_per_sm = per_sm;
    h->tma_stages = g.STAGES;
    if (h->fv_quick || h->L.split) {
        CU(h, lbmfvm_fv::prepare_modes<S>(&h->blocks_quick, &h->blocks_given));
        if (h->blocks_quick < 1 || h->blocks_given < 1)
            return fail(h, LBMFVM_ERR_CUDA, "TMA tile kernel of the energy-update options does not fit on an SM");
    }
    h->tile_w = g.TW;
    h->tile_h = g.TH;
    return upload_tiles(h, g.TW, g.TH);
}

// Tile lists of the TMA kernel (row by row over every active cavity) and the
// cavity table, uploaded on the handle's stream: cavities with one energy
// update per step in the fused list, those with sub-steps in the second list,
// ordered by their number of sub-steps (largest first).
int upload_tiles(lbmfvm_t *h, int tw, int th) {
    std::vector<TileHeader> fused, split;
    std::vector<CavityDesc> table;
    if (!h->atlas_cavs.empty()) table = h->atlas_cavs;
    else table.push_back(single_cavity_desc(h));
    std::vector<size_t> order(table.size());
    for (size_t c = 0; c < order.size(); c++) order[c] = c;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t p, size_t q) { return table[p].substeps > table[q].substeps; });
    for (size_t c : order) {
        if (!h->atlas_cavs.empty() && !h->atlas_active[c]) continue;
        const CavityDesc &cd = table[c];
        const int m = cd.substeps < 1 ? 1 : cd.substeps;
        // grid setting 2 collides with the node temperatures of its coarse
        // volumes, like the sub-step path
        std::vector<TileHeader> &tl = m > 1 || h->grid2 ? split : fused;
        for (int y0 = cd.y0; y0 < cd.y0 + cd.ny; y0 += th)
            for (int x0 = cd.x0; x0 < cd.x0 + cd.nx; x0 += tw) {
                TileHeader t{};
                t.x0 = x0;
                t.y0 = y0;
                t.ox = x0 - cd.x0;
                t.oy = y0 - cd.y0;
                t.nx = cd.nx;
                t.ny = cd.ny;
                t.cav = (int)c;
                t.substeps = m;
                t.omega = cd.omega;
                t.alpha = cd.alpha;
                t.gbeta = cd.gbeta;
                t.t_ref = cd.t_ref;
                t.fx = cd.fx;
                t.fy = cd.fy;
                t.omega_f = (float)cd.omega;
                t.alpha_f = (float)cd.alpha;
                t.gbeta_f = (float)cd.gbeta;
                t.t_ref_f = (float)cd.t_ref;
                t.fx_f = (float)cd.fx;
                t.fy_f = (float)cd.fy;
                const double dt = 1.0 / m;
                t.dt_f = (float)dt;
                auto lo = [](double d) { return (float)(d - (double)(float)d); };
                t.omega_lo = lo(cd.omega);
                t.alpha_lo = lo(cd.alpha);
                t.gbeta_lo = lo(cd.gbeta);
                t.t_ref_lo = lo(cd.t_ref);
                t.fx_lo = lo(cd.fx);
                t.fy_lo = lo(cd.fy);
                t.dt_lo = lo(dt);
                tl.push_back(t);
            }
    }
    if (!split.empty() && !h->L.split)
        return fail(h, LBMFVM_ERR_ARG, "a cavity takes energy sub-steps but the workspace has no room for them");
    if (fused.size() + split.size() > h->L.tile_cap)
        return fail(h, LBMFVM_ERR_ARG, "%zu tiles exceed the lists' %zu entries", fused.size() + split.size(),
                    h->L.tile_cap);
    h->ntiles = (int)fused.size();
    h->ntiles_split = (int)split.size();
    h->split_tiles_at.clear();
    for (size_t i = 0; i < split.size(); i++) {
        const int m = split[i].substeps;
        if ((int)h->split_tiles_at.size() < m) h->split_tiles_at.resize(m, 0);
        for (int sub = 0; sub < m; sub++) h->split_tiles_at[sub] = (int)i + 1;
    }
    // count slots (their tile counters cleared), each followed by its headers
    std::vector<TileHeader> all;
    TileHeader slot{};
    slot.x0 = h->ntiles;
    all.push_back(slot);
    all.insert(all.end(), fused.begin(), fused.end());
    slot.x0 = h->ntiles_split;
    all.push_back(slot);
    all.insert(all.end(), split.begin(), split.end());
    h->tiles_gen++;
    // on the handle's stream, after the workspace has been cleared
    CU(h, cudaMemcpyAsync(h->base + h->L.tiles, all.data(), all.size() * sizeof(TileHeader), cudaMemcpyHostToDevice,
                          h->s));
    CU(h, cudaMemcpyAsync(h->base + h->L.cav, table.data(), table.size() * sizeof(CavityDesc),
                          cudaMemcpyHostToDevice, h->s));
    CU(h, cudaStreamSynchronize(h->s));
    return LBMFVM_OK;
}

// Clears the tile counters of both lists (a step of parity p clears the
// counter of parity 1 - p for the next step; restarting at parity 0 clears
// both).
int clear_tile_counters(lbmfvm_t *h) {
    CU(h, cudaMemsetAsync(h->base + list_fused(h).slot + sizeof(int), 0, 2 * sizeof(int), h->s));
    CU(h, cudaMemsetAsync(h->base + list_split(h).slot + sizeof(int), 0, 2 * sizeof(int), h->s));
    return LBMFVM_OK;
}

CavityDesc single_cavity_desc(const lbmfvm_t *h) {
    CavityDesc cd{};
    cd.x0 = 0;
    cd.y0 = 0;
    cd.nx = h->grid.nx;
    cd.ny = h->grid.ny;
    cd.omega = 1.0 / h->tau;
    cd.alpha = h->alpha;
    cd.gbeta = h->gbeta;
    cd.t_ref = h->t_ref;
    cd.fx = h->force[0];
    cd.fy = h->force[1];
    cd.substeps = h->fv_sub;
    for (int sd = 0; sd < 4; sd++) {
        const bool moving = h->grid.bc[sd] == LBMFVM_BC_MOVING;
        cd.wall_u[sd] = moving && sd >= 2 ? h->grid.u_lid : 0.0;
        cd.wall_v[sd] = moving && sd < 2 ? h->grid.u_lid : 0.0;
        cd.wall_uf[sd] = (float)cd.wall_u[sd];
        cd.wall_vf[sd] = (float)cd.wall_v[sd];
    }
    return cd;
}

// Tensor maps of both population buffers (box fw x fh x 9), both
// temperature planes (tw x th) and the node codes (cw x ch); the grid's x
// extent is nx, so boxes reaching past it (or below zero) are zero-filled.
// A non-zero t_plane maps that temperature plane into map_T[0] and map_T[1]
// instead.
template <class S>
int encode_maps(lbmfvm_t *h, int fw, int fh, int tw, int th, int cw, int ch, size_t t_plane) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return fail(h, LBMFVM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    const cuuint64_t nx = (cuuint64_t)h->grid.nx, ny = (cuuint64_t)h->grid.ny, pitch = (cuuint64_t)h->L.pitch;
    const cuuint32_t one[3] = {1, 1, 1};
    for (int b = 0; b < 2; b++) {
        const cuuint64_t dims[3] = {nx, ny, 9};
        const cuuint64_t strides[2] = {pitch * sizeof(S), (cuuint64_t)h->L.plane * sizeof(S)};
        const cuuint32_t box[3] = {(cuuint32_t)fw, (cuuint32_t)fh, 9};
        CUresult r = enc(&h->map_f[b], tmap_type<S>(), 3, h->base + h->L.f[b], dims, strides, box, one,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(h, LBMFVM_ERR_CUDA, "tensor map of the populations failed (%d)", (int)r);
        const cuuint64_t dims2[2] = {nx, ny};
        using C = typename Compute<S>::type;
        const cuuint64_t strides2[1] = {pitch * sizeof(C)};
        const cuuint32_t box2[2] = {(cuuint32_t)tw, (cuuint32_t)th};
        r = enc(&h->map_T[b], tmap_type<C>(), 2, h->base + (t_plane ? t_plane : h->L.T[b]), dims2, strides2, box2, one,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(h, LBMFVM_ERR_CUDA, "tensor map of the temperature failed (%d)", (int)r);
    }
    // codes and face flags: two planes of one box
    const cuuint64_t dims3[3] = {nx, ny, 2};
    const cuuint64_t strides3[2] = {pitch, (cuuint64_t)(h->L.fflags - h->L.code)};
    const cuuint32_t box3[3] = {(cuuint32_t)cw, (cuuint32_t)ch, 2};
    CUresult r = enc(&h->map_c, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, h->base + h->L.code, dims3, strides3, box3, one,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, LBMFVM_ERR_CUDA, "tensor map of the node codes failed (%d)", (int)r);
    return LBMFVM_OK;
}

int setup_kernels(lbmfvm_t *h) {
    if (!h->use_tma) return LBMFVM_OK;
    switch (h->prec) {
        case LBMFVM_F64: return setup_tma<double>(h);
        case LBMFVM_F32: return setup_tma<float>(h);
        case LBMFVM_F16: return setup_tma<__half>(h);
        case LBMFVM_BF16: return setup_tma<__nv_bfloat16>(h);
        case LBMFVM_F32X2: return setup_tma<dsf>(h);
    }
    return LBMFVM_OK;
}

// A bounded device-side wait that ran out leaves a non-zero status word.
int check_device_status(lbmfvm_t *h) {
    int word = 0;
    int *dev = reinterpret_cast<int *>(h->base + h->L.err);
    CU(h, cudaMemcpyAsync(&word, dev, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    CU(h, cudaStreamSynchronize(h->s));
    if (word) {
        CU(h, cudaMemsetAsync(dev, 0, sizeof(int), h->s));
        return fail(h, LBMFVM_ERR_TIMEOUT, "a device-side wait for staged data ran out (status %d)", word);
    }
    return LBMFVM_OK;
}

// Autotuner of the TMA tile shape.  Each shape steps the handle's own grid
// (from the cleared workspace, which is the rest state f = w_i, T = 0) in the
// form the library runs it: a captured graph of kTuneSteps launches chained by
// programmatic dependent launch, replayed once untimed and then timed over
// kTuneReps replays with events on the handle's stream (timing launches one by
// one from the host would measure the host's launch rate, not the kernel).
// The fastest shape is kept and remembered for the storage precision and the
// size class (the power of two of the nodes the tiles cover), so a class is
// measured once per process.  Every shape computes the same arithmetic per
// node, so the choice never changes results.  The population and temperature
// buffers are cleared again afterwards.  Runs at creation, outside any stream
// capture of the caller.
constexpr int kTuneSteps = 32;
constexpr int kTuneReps = 2;
std::mutex g_tune_mu;
std::map<std::pair<int, int>, int> g_tuned;

int size_class(const lbmfvm_t *h) {
    long long n = 0;
    if (h->atlas_cavs.empty()) {
        n = (long long)h->grid.nx * h->grid.ny;
    } else {
        for (size_t c = 0; c < h->atlas_cavs.size(); c++) n += (long long)h->atlas_cavs[c].nx * h->atlas_cavs[c].ny;
    }
    int cls = 0;
    while ((n >>= 1) > 0) cls++;
    return cls;
}

int autotune(lbmfvm_t *h) {
    const std::pair<int, int> key(h->prec, size_class(h));
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            h->tma_config = it->second;
            return setup_kernels(h);
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CU(h, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(h, LBMFVM_ERR_CUDA, "event creation failed");
    }
    int best = -1;
    float best_ms = 0.0f;
    int status = LBMFVM_OK;
    for (int cfg = 0; cfg < kTmaConfigs && status == LBMFVM_OK; cfg++) {
        h->tma_config = cfg;
        if (setup_kernels(h) != LBMFVM_OK) continue;  // a shape that does not fit this device
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        cudaError_t e = cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int i = 0; i < kTuneSteps; i++) launch_one(h, i & 1, h->s);
            e = cudaStreamEndCapture(h->s, &g);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess) e = cudaGraphLaunch(ge, h->s);
        if (e == cudaSuccess) e = cudaEventRecord(e0, h->s);
        for (int r = 0; r < kTuneReps && e == cudaSuccess; r++) e = cudaGraphLaunch(ge, h->s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->s);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (ge) cudaGraphExecDestroy(ge);
        if (e != cudaSuccess) {
            status = fail(h, LBMFVM_ERR_CUDA, "autotuning failed: %s", cudaGetErrorString(e));
            break;
        }
        if (best < 0 || ms < best_ms) {
            best = cfg;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != LBMFVM_OK) return status;
    if (best < 0) return fail(h, LBMFVM_ERR_CUDA, "no TMA tile shape fits this device");
    h->tma_config = best;
    if (int r = setup_kernels(h)) return r;
    if (int r = check_device_status(h)) return r;
    const size_t fbytes = 9 * (size_t)h->L.plane * store_size(h->prec);
    const size_t tbytes = (size_t)h->L.plane * temp_size(h->prec);
    for (int b = 0; b < 2; b++) {
        CU(h, cudaMemsetAsync(h->base + h->L.f[b], 0, fbytes, h->s));
        CU(h, cudaMemsetAsync(h->base + h->L.T[b], 0, tbytes, h->s));
    }
    CU(h, cudaStreamSynchronize(h->s));
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[key] = best;
    return LBMFVM_OK;
}

// Several cavities packed in one grid: their descriptors (rectangles starting
// on 128 x 16 slot corners, lattice parameters) and the packed node codes.
struct AtlasSpec {
    std::vector<CavityDesc> cavs;
    std::vector<uint8_t> codes;  // stored codes, ny * pitch of the packed grid
};

// Sub-steps of the energy update for a cavity: the requested number, or
// (LBMFVM_FV_SUBSTEPS_AUTO) the fewest with alpha/m <= 0.2 and, when the
// velocity scale U0 is known (> 0), U0^2/m <= 1.8 alpha.
int substeps_for(int requested, double alpha, double U0) {
    if (requested != LBMFVM_FV_SUBSTEPS_AUTO) return requested;
    int m = (int)std::ceil(alpha / 0.2 - 1e-12);
    if (U0 > 0.0) m = std::max(m, (int)std::ceil(U0 * U0 / (1.8 * alpha) - 1e-12));
    return std::max(m, 1);
}

// Stability limits of the explicit energy update with m sub-steps: diffusion
// alpha dt (1/dx^2 + 1/dy^2) <= 1/2 and central advection (U dt)^2 <= 2 alpha dt,
// dt = 1/m.  Returns why a cavity fails them, or nullptr.
const char *fv_unstable(double alpha, double U0, int m) {
    if (alpha / m > 0.25) return "alpha / substeps exceeds the explicit diffusion limit 0.25";
    if (U0 > 0.0 && U0 * U0 > 2.0 * alpha * m) return "U0^2 / substeps exceeds 2 alpha (explicit central advection limit)";
    return nullptr;
}

int create_impl(const lbmfvm_grid_t *grid, const uint8_t *mask, double nu, double alpha, double gbeta,
                const double *force, const lbmfvm_opts_t *opts_in, lbmfvm_t **out, const AtlasSpec *atlas = nullptr) {
    if (!out) return fail_thread(LBMFVM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (int r = check_grid(grid)) return r;
    lbmfvm_opts_t opts;
    lbmfvm_opts_default(&opts);
    if (opts_in) opts = *opts_in;
    if (opts.store < LBMFVM_F64 || opts.store > LBMFVM_F32X2)
        return fail_thread(LBMFVM_ERR_ARG, "store = %d is not a LBMFVM_F* value", opts.store);
    if (opts.tile_y != 0 && opts.tile_y != 4 && opts.tile_y != 8 && opts.tile_y != 16)
        return fail_thread(LBMFVM_ERR_ARG, "tile_y must be 0, 4, 8 or 16 (got %d)", opts.tile_y);
    const bool periodic = grid->bc[LBMFVM_SIDE_W] == LBMFVM_BC_PERIODIC || grid->bc[LBMFVM_SIDE_S] == LBMFVM_BC_PERIODIC;
    const bool tma_ok = !periodic;
    if (opts.kernel < LBMFVM_KERNEL_AUTO || opts.kernel > LBMFVM_KERNEL_TMA)
        return fail_thread(LBMFVM_ERR_ARG, "kernel = %d is not a LBMFVM_KERNEL_* value", opts.kernel);
    if (opts.tma_config != LBMFVM_TMA_AUTOTUNE && opts.tma_config != LBMFVM_TMA_DEFAULT &&
        (opts.tma_config < 0 || opts.tma_config >= kTmaConfigs))
        return fail_thread(LBMFVM_ERR_ARG,
                           "tma_config must be LBMFVM_TMA_AUTOTUNE, LBMFVM_TMA_DEFAULT or in [0, %d) (got %d)",
                           kTmaConfigs, opts.tma_config);
    if (opts.kernel == LBMFVM_KERNEL_TMA && !tma_ok)
        return fail_thread(LBMFVM_ERR_ARG, "the TMA kernel needs walls on every side");
    if (!(nu > 0.0) || !std::isfinite(nu) || !(alpha > 0.0) || !std::isfinite(alpha) || !std::isfinite(gbeta))
        return fail_thread(LBMFVM_ERR_ARG, "nu and alpha must be positive and finite, gbeta finite");
    const double tau = 3.0 * nu + 0.5;
    if (tau < 0.51) return fail_thread(LBMFVM_ERR_UNSTABLE, "tau = %.6g < 0.51", tau);
    if (opts.fv_scheme != LBMFVM_FV_CENTRAL && opts.fv_scheme != LBMFVM_FV_QUICK)
        return fail_thread(LBMFVM_ERR_ARG, "fv_scheme = %d is not a LBMFVM_FV_* value", opts.fv_scheme);
    if (opts.fv_substeps < 0 || opts.fv_substeps > 256)
        return fail_thread(LBMFVM_ERR_ARG, "fv_substeps = %d is outside [0, 256]", opts.fv_substeps);
    if (opts.energy != LBMFVM_ENERGY_FV && opts.energy != LBMFVM_ENERGY_LBM_D2Q5)
        return fail_thread(LBMFVM_ERR_ARG, "energy = %d is not a LBMFVM_ENERGY_* value", opts.energy);
    const bool lbm5 = opts.energy == LBMFVM_ENERGY_LBM_D2Q5;
    if (opts.wall_bc != LBMFVM_WALL_NEE && opts.wall_bc != LBMFVM_WALL_FD)
        return fail_thread(LBMFVM_ERR_ARG, "wall_bc = %d is not a LBMFVM_WALL_* value", opts.wall_bc);
    const bool fd = opts.wall_bc == LBMFVM_WALL_FD;
    if (opts.fv_grid != 1 && opts.fv_grid != 2)
        return fail_thread(LBMFVM_ERR_ARG, "fv_grid = %d is not 1 or 2", opts.fv_grid);
    if (opts.fv_every < 1 || opts.fv_every > 4096)
        return fail_thread(LBMFVM_ERR_ARG, "fv_every = %d is outside [1, 4096]", opts.fv_every);
    const bool grid2 = opts.fv_grid == 2;
    if (grid2) {
        if (atlas || lbm5 || fd || !tma_ok || opts.kernel == LBMFVM_KERNEL_GENERIC ||
            opts.fv_scheme != LBMFVM_FV_CENTRAL || opts.fv_substeps != 1)
            return fail_thread(LBMFVM_ERR_ARG, "grid setting 2 runs single walled cavities on the TMA kernel with "
                                               "the central energy update, extrapolation walls and no sub-steps");
        if ((grid->nx - 1) % 2 || (grid->ny - 1) % 2)
            return fail_thread(LBMFVM_ERR_ARG, "grid setting 2 needs an even number of spacings (got %d x %d nodes)",
                               grid->nx, grid->ny);
        if (mask)
            for (size_t k = 0; k < (size_t)grid->nx * grid->ny; k++)
                if (mask[k]) return fail_thread(LBMFVM_ERR_ARG, "grid setting 2 takes no obstacle");
        // positivity of the coarse explicit step next to a Dirichlet wall:
        // (k / 4) (3 alpha + 2 alpha) <= 1
        if (alpha * opts.fv_every > 0.8)
            return fail_thread(LBMFVM_ERR_UNSTABLE, "alpha * fv_every = %.6g exceeds 0.8 (coarse explicit limit)",
                               alpha * opts.fv_every);
    } else if (opts.fv_every != 1) {
        return fail_thread(LBMFVM_ERR_ARG, "fv_every applies to grid setting 2");
    }
    if (fd && (atlas || lbm5 || opts.kernel == LBMFVM_KERNEL_TMA || opts.fv_scheme != LBMFVM_FV_CENTRAL ||
               opts.fv_substeps != 1))
        return fail_thread(LBMFVM_ERR_ARG,
                           "finite-difference walls run single cavities on the generic kernel with the central "
                           "one-step energy update");
    if (lbm5) {
        if (atlas) return fail_thread(LBMFVM_ERR_ARG, "the D2Q5 energy solver runs single cavities only");
        if (opts.store == LBMFVM_F16 || opts.store == LBMFVM_BF16)
            return fail_thread(LBMFVM_ERR_ARG, "the D2Q5 energy solver stores F64, F32 or F32X2");
        if (opts.fv_scheme != LBMFVM_FV_CENTRAL || opts.fv_substeps != 1)
            return fail_thread(LBMFVM_ERR_ARG, "QUICK and sub-steps belong to the finite-volume energy update");
    }
    // a single cavity's sub-steps (a batch's come with its cavity table);
    // the D2Q5 populations have no explicit-step limit (tau_T > 1/2)
    const int m = atlas ? 1 : substeps_for(opts.fv_substeps, alpha, 0.0);
    if (!atlas && !lbm5 && opts.fv_grid != 2)
        if (const char *why = fv_unstable(alpha, 0.0, m))
            return fail_thread(LBMFVM_ERR_UNSTABLE, "alpha = %.6g, %d sub-step(s): %s", alpha, m, why);
    bool split = m > 1 || grid2;
    if (atlas)
        for (const CavityDesc &cd : atlas->cavs) split |= cd.substeps > 1;
    const bool fv_opt = split || opts.fv_scheme == LBMFVM_FV_QUICK;  // (grid setting 2 is split)
    if (fv_opt && (!tma_ok || opts.kernel == LBMFVM_KERNEL_GENERIC))
        return fail_thread(LBMFVM_ERR_ARG, "QUICK face values and energy sub-steps need the TMA kernel (walls on every side)");
    if (atlas && !tma_ok) return fail_thread(LBMFVM_ERR_ARG, "a batch needs walls on every side");
    const Layout L = make_layout(*grid, opts.store, atlas ? (int)atlas->cavs.size() : 1, split, lbm5);
    if (opts.workspace && opts.workspace_bytes < L.total)
        return fail_thread(LBMFVM_ERR_NOMEM, "workspace of %zu bytes is smaller than the %zu needed",
                           opts.workspace_bytes, L.total);
    if (opts.workspace && ((uintptr_t)opts.workspace % kAlign))
        return fail_thread(LBMFVM_ERR_ARG, "workspace must be %zu-byte aligned", kAlign);

    lbmfvm_t *h = new (std::nothrow) lbmfvm_t();
    if (!h) return fail_thread(LBMFVM_ERR_NOMEM, "host allocation failed");
    h->grid = *grid;
    h->prec = opts.store;
    h->tile_y = opts.tile_y ? opts.tile_y : 8;
    h->use_tma = tma_ok && opts.kernel != LBMFVM_KERNEL_GENERIC;
    // the default shapes are the fastest measured ones: 64 x 16 with ring
    // warps for 32- and 16-bit storage (two population halo rows when both
    // population buffers and temperature planes fit in the L2, three
    // otherwise), two blocks of 32 x 8 per SM for 64-bit.  A grid with fewer
    // tiles than SMs is bound by the latency of one tile, not by the SMs'
    // throughput, and takes the smaller tiles that spread it over more SMs:
    // 64 x 8 (two blocks per SM) for 32- and 16-bit storage, 32 x 8 with ring
    // warps for 64-bit.
    int shape_default = 3;
    {
        int dev = 0, l2 = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            l2 = sms = 0;
        const long long tiles = store_size(opts.store) == 8
                                    ? (long long)((grid->nx + 31) / 32) * ((grid->ny + 7) / 8)
                                    : (long long)((grid->nx + 63) / 64) * ((grid->ny + 15) / 16);
        const bool small = tiles < sms;
        if (store_size(opts.store) == 8) {
            shape_default = small ? 4 : 3;
        } else {
            const size_t state = 2 * (9 * store_size(opts.store) + temp_size(opts.store)) * (size_t)L.plane;
            shape_default = small ? 2 : state <= (size_t)l2 ? 4 : 5;
        }
    }
    h->tma_config = opts.tma_config == LBMFVM_TMA_AUTOTUNE || opts.tma_config == LBMFVM_TMA_DEFAULT ? shape_default
                                                                                                  : opts.tma_config;
    h->fv_quick = opts.fv_scheme == LBMFVM_FV_QUICK;
    h->fv_sub = m;
    h->energy = opts.energy;
    h->wall_bc = opts.wall_bc;
    h->grid2 = grid2;
    h->fv_every = opts.fv_every;
    h->ncx = (grid->nx - 1) / 2;
    h->ncy = (grid->ny - 1) / 2;
    if (lbm5 || fd) h->use_tma = false;  // their own or the generic kernel, no staged loads
    if (fv_opt) h->tma_config = kTmaConfigFv;  // the options' kernels come in this shape
    h->L = L;
    h->nu = nu;
    h->alpha = alpha;
    h->gbeta = gbeta;
    h->tau = tau;
    h->t_ref = std::isnan(opts.t_ref) ? grid->t_wall[LBMFVM_SIDE_E] : opts.t_ref;
    h->force[0] = force ? force[0] : 0.0;
    h->force[1] = force ? force[1] : 0.0;
    h->user = (cudaStream_t)opts.cuda_stream;
    auto bail = [&](int code) {
        lbmfvm_destroy(h);
        return code;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        h->s = nullptr;
        fail(h, LBMFVM_ERR_CUDA, "cudaStreamCreateWithFlags failed: %s", cudaGetErrorString(e));
        return bail(LBMFVM_ERR_CUDA);
    }
    if (cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        fail(h, LBMFVM_ERR_CUDA, "cudaEventCreate failed");
        return bail(LBMFVM_ERR_CUDA);
    }
    if (opts.workspace) {
        h->base = static_cast<unsigned char *>(opts.workspace);
        h->owns = false;
    } else {
        e = cudaMalloc(&h->base, L.total);
        if (e != cudaSuccess) {
            h->base = nullptr;
            fail(h, LBMFVM_ERR_NOMEM, "cudaMalloc of %zu bytes failed: %s", L.total, cudaGetErrorString(e));
            return bail(LBMFVM_ERR_NOMEM);
        }
        h->owns = true;
    }
    std::vector<uint8_t> code = atlas ? atlas->codes : classify(*grid, mask, L.pitch);
    if (atlas) {
        h->atlas_cavs = atlas->cavs;
        h->atlas_active.assign(atlas->cavs.size(), 1);
        h->use_tma = true;
    }
    std::vector<CavityDesc> rects = atlas ? atlas->cavs : std::vector<CavityDesc>(1);
    if (!atlas) {
        rects[0].nx = grid->nx;
        rects[0].ny = grid->ny;
    }
    const std::vector<uint8_t> fflags = face_flags(code, L.pitch, rects);
    h->code_crc = crc32_update(0, code.data(), code.size());
    if (join_in(h)) return bail(LBMFVM_ERR_CUDA);
    if (cudaMemsetAsync(h->base, 0, L.total, h->s) != cudaSuccess ||
        cudaMemcpyAsync(h->base + L.code, code.data(), code.size(), cudaMemcpyHostToDevice, h->s) != cudaSuccess ||
        cudaMemcpyAsync(h->base + L.fflags, fflags.data(), fflags.size(), cudaMemcpyHostToDevice, h->s) !=
            cudaSuccess) {
        fail(h, LBMFVM_ERR_CUDA, "device initialisation failed");
        return bail(LBMFVM_ERR_CUDA);
    }
    if (int r = setup_kernels(h)) return bail(r);
    if (h->use_tma && opts.tma_config == LBMFVM_TMA_AUTOTUNE && !fv_opt)
        if (int r = autotune(h)) return bail(r);
    if (!atlas)
        if (int r = set_state_impl(h, nullptr, nullptr, nullptr)) return bail(r);
    *out = h;
    return LBMFVM_OK;
}

template <class O>
int fields_impl(lbmfvm_t *h, O *rho, O *u, O *v, O *T) {
    if (!h) return fail_thread(LBMFVM_ERR_ARG, "handle is NULL");
    const size_t n = (size_t)h->grid.nx * h->grid.ny;
    O *st = reinterpret_cast<O *>(h->base + h->L.stage);
    if (int r = join_in(h)) return r;
    O *outs[2][2] = {{rho, u}, {v, T}};
    for (int which = 0; which < 2; which++) {
        if (!outs[which][0] && !outs[which][1]) continue;
        DISPATCH(h, launch_fields, h, which, st, st + n);
        CU(h, cudaGetLastError());
        for (int i = 0; i < 2; i++)
            if (outs[which][i])
                CU(h, cudaMemcpyAsync(outs[which][i], st + i * n, n * sizeof(O), cudaMemcpyDefault, h->s));
    }
    CU(h, cudaStreamSynchronize(h->s));
    if (int r = check_device_status(h)) return r;
    return join_out(h);
}

}  // namespace

namespace {
// lbmfvm_step without the joins with the caller's stream: the launches of
// n steps on the handle's own stream.
int step_impl(lbmfvm_t *h, int64_t n) {
    // tile lists that changed since the capture need other grids and
    // sub-step launches
    if (h->graph && h->use_tma && h->graph_gen != h->tiles_gen) {
        CU(h, cudaGraphExecDestroy(h->graph));
        h->graph = nullptr;
    }
    if (n >= kGraphSteps && !h->graph && kGraphSteps % h->fv_every == 0)
        if (int r = build_graph(h)) return r;
    while (n > 0) {
        if (h->parity == 0 && n >= kGraphSteps && h->graph && !h->stall_next && h->steps % h->fv_every == 0) {
            CU(h, cudaGraphLaunch(h->graph, h->s));
            n -= kGraphSteps;
            h->steps += kGraphSteps;
            h->launches += kGraphSteps;
        } else {
            launch_one(h, h->parity, h->s, h->stall_next, (h->steps + 1) % h->fv_every == 0);
            h->stall_next = false;
            CU(h, cudaGetLastError());
            h->parity ^= 1;
            n--;
            h->steps++;
            h->launches++;
        }
    }
    return LBMFVM_OK;
}
}  // namespace

extern "C" {

void lbmfvm_opts_default(lbmfvm_opts_t *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->store = LBMFVM_F32;
    o->tile_y = 0;
    o->kernel = LBMFVM_KERNEL_AUTO;
    o->tma_config = LBMFVM_TMA_DEFAULT;
    o->t_ref = NAN;
    o->fv_scheme = LBMFVM_FV_CENTRAL;
    o->fv_substeps = 1;
    o->energy = LBMFVM_ENERGY_FV;
    o->wall_bc = LBMFVM_WALL_NEE;
    o->fv_grid = 1;
    o->fv_every = 1;
}

int lbmfvm_workspace_bytes(const lbmfvm_grid_t *grid, const lbmfvm_opts_t *opts, size_t *bytes) {
    if (!bytes) return fail_thread(LBMFVM_ERR_ARG, "bytes is NULL");
    if (int r = check_grid(grid)) return r;
    const int prec = opts ? opts->store : LBMFVM_F32;
    if (prec < LBMFVM_F64 || prec > LBMFVM_F32X2) return fail_thread(LBMFVM_ERR_ARG, "invalid store precision");
    // sub-steps (or the automatic choice, which may take them) need the planes
    const bool split = opts && (opts->fv_substeps != 1 || opts->fv_grid == 2);
    const bool lbm5 = opts && opts->energy == LBMFVM_ENERGY_LBM_D2Q5;
    *bytes = make_layout(*grid, prec, 1, split, lbm5).total;
    return LBMFVM_OK;
}

int lbmfvm_create(const lbmfvm_grid_t *grid, const uint8_t *mask, double Ra, double Pr, double Ma,
                  const lbmfvm_opts_t *opts, lbmfvm_t **out) {
    if (out) *out = nullptr;
    if (int r = check_grid(grid)) return r;
    if (!(Ra > 0.0) || !(Pr > 0.0) || !(Ma > 0.0) || !std::isfinite(Ra) || !std::isfinite(Pr) || !std::isfinite(Ma))
        return fail_thread(LBMFVM_ERR_ARG, "Ra, Pr and Ma must be positive and finite");
    const double dT = grid->t_wall[LBMFVM_SIDE_W] - grid->t_wall[LBMFVM_SIDE_E];
    if (dT == 0.0 || !std::isfinite(dT))
        return fail_thread(LBMFVM_ERR_ARG, "t_wall[W] - t_wall[E] must be non-zero");
    if (Ma > 0.3) return fail_thread(LBMFVM_ERR_UNSTABLE, "Ma = %.6g exceeds 0.3", Ma);
    const double H = grid->ny - 1;
    const double U0 = Ma / std::sqrt(3.0);
    const double nu = U0 * H * std::sqrt(Pr / Ra);
    const double alpha = U0 * H / std::sqrt(Ra * Pr);
    const double gbeta = U0 * U0 / (H * dT);
    lbmfvm_opts_t o;
    lbmfvm_opts_default(&o);
    if (opts) o = *opts;
    if (o.fv_substeps < 0 || o.fv_substeps > 256)
        return fail_thread(LBMFVM_ERR_ARG, "fv_substeps = %d is outside [0, 256]", o.fv_substeps);
    if (o.energy == LBMFVM_ENERGY_FV && o.fv_grid == 2) {
        // grid setting 2: central advection over k lattice steps, (U0 k)^2 <= 2 alpha k
        if (U0 * U0 * o.fv_every > 2.0 * alpha)
            return fail_thread(LBMFVM_ERR_UNSTABLE, "U0^2 fv_every = %.6g exceeds 2 alpha = %.6g (coarse advection limit)",
                               U0 * U0 * o.fv_every, 2.0 * alpha);
    } else if (o.energy == LBMFVM_ENERGY_FV) {
        o.fv_substeps = substeps_for(o.fv_substeps, alpha, U0);
        if (const char *why = fv_unstable(alpha, U0, o.fv_substeps))
            return fail_thread(LBMFVM_ERR_UNSTABLE, "U0 = %.6g, alpha = %.6g, %d sub-step(s): %s", U0, alpha,
                               o.fv_substeps, why);
    }
    return create_impl(grid, mask, nu, alpha, gbeta, nullptr, &o, out);
}

int lbmfvm_create_lattice(const lbmfvm_grid_t *grid, const uint8_t *mask, double nu, double alpha, double gbeta,
                          const double *force, const lbmfvm_opts_t *opts, lbmfvm_t **out) {
    return create_impl(grid, mask, nu, alpha, gbeta, force, opts, out);
}

int lbmfvm_set_state(lbmfvm_t *h, const float *u, const float *v, const float *T) {
    if (!h) return fail_thread(LBMFVM_ERR_ARG, "handle is NULL");
    return set_state_impl(h, u, v, T);
}

int lbmfvm_step(lbmfvm_t *h, int64_t n) {
    if (!h) return fail_thread(LBMFVM_ERR_ARG, "handle is NULL");
    if (n < 0) return fail(h, LBMFVM_ERR_ARG, "n = %lld is negative", (long long)n);
    if (n == 0) return LBMFVM_OK;
    if (int r = join_in(h)) return r;
    if (int r = step_impl(h, n)) return r;
    return join_out(h);
}

int lbmfvm_fv_info(const lbmfvm_t *h, int32_t *scheme, int32_t *substeps) {
    if (!h) return fail_thread(LBMFVM_ERR_ARG, "handle is NULL");
    if (scheme) *scheme = h->fv_quick ? LBMFVM_FV_QUICK : LBMFVM_FV_CENTRAL;
    if (substeps) *substeps = h->fv_sub;
    return LBMFVM_OK;
}

int lbmfvm_inject_stall(lbmfvm_t *h) {
    if (!h) return fail_thread(LBMFVM_ERR_ARG, "handle is NULL");
    if (!h->use_tma) return fail(h, LBMFVM_ERR_ARG, "the generic step kernel has no staged loads to stall");
    h->stall_next = true;
    return LBMFVM_OK;
}

int lbmfvm_step_count(const lbmfvm_t *h, int64_t *steps) {
    if (!h || !steps) return fail_thread(LBMFVM_ERR_ARG, "handle or steps is NULL");
    *steps = h->steps;
    return LBMFVM_OK;
}

int lbmfvm_fields(lbmfvm_t *h, double *rho, double *u, double *v, double *T) {
    return fields_impl<double>(h, rho, u, v, T);
}

int lbmfvm_fields_f32(lbmfvm_t *h, float *rho, float *u, float *v, float *T) {
    return fields_impl<float>(h, rho, u, v, T);
}

int lbmfvm_nusselt(lbmfvm_t *h, double *mean_hot, double *local_hot, double *mean_cold) {
    if (!h) return fail_thread(LBMFVM_ERR_ARG, "handle is NULL");
    if (h->grid.t_wall[LBMFVM_SIDE_W] == h->grid.t_wall[LBMFVM_SIDE_E])
        return fail(h, LBMFVM_ERR_ARG, "Nusselt number needs t_wall[W] != t_wall[E]");
    if (int r = join_in(h)) return r;
    DISPATCH(h, launch_nusselt, h);
    CU(h, cudaGetLastError());
    double *red = reinterpret_cast<double *>(h->base + h->L.red);
    double means[2];
    CU(h, cudaMemcpyAsync(means, red + kRedNu, sizeof(means), cudaMemcpyDeviceToHost, h->s));
    if (local_hot)
        CU(h, cudaMemcpyAsync(local_hot, red + kRedLocal, h->grid.ny * sizeof(double),
                              cudaMemcpyDefault, h->s));
    CU(h, cudaStreamSynchronize(h->s));
    if (mean_hot) *mean_hot = means[0];
    if (mean_cold) *mean_cold = means[1];
    if (int r = check_device_status(h)) return r;
    if (!std::isfinite(means[0]) || !std::isfinite(means[1]))
        return fail(h, LBMFVM_ERR_DIVERGED, "non-finite Nusselt number");
    return join_out(h);
}

int lbmfvm_residual(lbmfvm_t *h, double *r) {
    if (!h || !r) return fail_thread(LBMFVM_ERR_ARG, "handle or r is NULL");
    if (int e = join_in(h)) return e;
    DISPATCH(h, launch_residual, h, 0);
    CU(h, cudaGetLastError());
    double sums[2];
    double *red = reinterpret_cast<double *>(h->base + h->L.red);
    CU(h, cudaMemcpyAsync(sums, red + kRedTot, sizeof(sums), cudaMemcpyDeviceToHost, h->s));
    CU(h, cudaStreamSynchronize(h->s));
    if (int e = check_device_status(h)) {
        *r = NAN;
        return e;
    }
    if (!std::isfinite(sums[0]) || !std::isfinite(sums[1])) {
        *r = NAN;
        return fail(h, LBMFVM_ERR_DIVERGED, "non-finite velocity in the residual");
    }
    *r = sums[1] > 0.0 ? std::sqrt(sums[0]) / std::sqrt(sums[1]) : (sums[0] == 0.0 ? 0.0 : INFINITY);
    return join_out(h);
}

int lbmfvm_run_to_steady(lbmfvm_t *h, double tol, int64_t check_every, int64_t max_steps, int64_t *steps_done,
                         double *r_final) {
    if (!h) return fail_thread(LBMFVM_ERR_ARG, "handle is NULL");
    if (check_every <= 0 || max_steps < 0) return fail(h, LBMFVM_ERR_ARG, "check_every must be > 0, max_steps >= 0");
    int64_t done = 0;
    double r = INFINITY;
    while (done < max_steps) {
        const int64_t n = check_every < max_steps - done ? check_every : max_steps - done;
        if (int e = lbmfvm_step(h, n)) return e;
        done += n;
        if (int e = lbmfvm_residual(h, &r)) {
            if (steps_done) *steps_done = done;
            if (r_final) *r_final = r;
            return e;
        }
        if (r < tol) break;
        // the residual pass left the mass total of this state in the scratch
        if (int e = join_in(h)) return e;
        DISPATCH(h, launch_rescale, h);
        CU(h, cudaGetLastError());
        if (int e = join_out(h)) return e;
    }
    if (steps_done) *steps_done = done;
    if (r_final) *r_final = r;
    return LBMFVM_OK;
}

int lbmfvm_copy_state(lbmfvm_t *dst, lbmfvm_t *src) {
    if (!dst || !src || dst == src) return fail_thread(LBMFVM_ERR_ARG, "need two distinct handles");
    if (dst->grid.nx != src->grid.nx || dst->grid.ny != src->grid.ny)
        return fail(dst, LBMFVM_ERR_ARG, "grids differ: %dx%d and %dx%d", dst->grid.nx, dst->grid.ny, src->grid.nx,
                    src->grid.ny);
    if (dst->energy != LBMFVM_ENERGY_FV || src->energy != LBMFVM_ENERGY_FV)
        return fail(dst, LBMFVM_ERR_ARG, "state copies hold finite-volume handles");
    // the source's queued steps finish before the copy reads its buffers
    if (int r = join_in(src)) return r;
    CU(src, cudaStreamSynchronize(src->s));
    if (int r = join_in(dst)) return r;
    DISPATCH(src, launch_convert_from, src, dst, 0, 0, dst->grid.nx, dst->grid.ny, src->parity ^ dst->parity);
    CU(dst, cudaGetLastError());
    CU(dst, cudaMemcpyAsync(dst->base + dst->L.snap, src->base + src->L.snap,
                            2 * (size_t)dst->grid.nx * dst->grid.ny * sizeof(double), cudaMemcpyDeviceToDevice, dst->s));
    dst->steps = src->steps;
    return join_out(dst);
}

int lbmfvm_launch_count(const lbmfvm_t *h, int64_t *launches) {
    if (!h || !launches) return fail_thread(LBMFVM_ERR_ARG, "handle or launches is NULL");
    *launches = h->launches;
    return LBMFVM_OK;
}

int lbmfvm_kernel_info(const lbmfvm_t *h, int32_t *kernel, int32_t *tma_config) {
    if (!h) return fail_thread(LBMFVM_ERR_ARG, "handle is NULL");
    if (kernel) *kernel = h->use_tma ? LBMFVM_KERNEL_TMA : LBMFVM_KERNEL_GENERIC;
    if (tma_config) *tma_config = h->use_tma ? h->tma_config : -1;
    return LBMFVM_OK;
}

int lbmfvm_params(const lbmfvm_t *h, double *nu, double *alpha, double *gbeta, double *tau) {
    if (!h) return fail_thread(LBMFVM_ERR_ARG, "handle is NULL");
    if (nu) *nu = h->nu;
    if (alpha) *alpha = h->alpha;
    if (gbeta) *gbeta = h->gbeta;
    if (tau) *tau = h->tau;
    return LBMFVM_OK;
}

void lbmfvm_destroy(lbmfvm_t *h) {
    if (!h) return;
    if (h->s) cudaStreamSynchronize(h->s);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->owns && h->base) cudaFree(h->base);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->s) cudaStreamDestroy(h->s);
    delete h;
}

const char *lbmfvm_last_error(const lbmfvm_t *h) { return h ? h->err : g_err; }

}  // extern "C"

#include "batch.inl"
#include "checkpoint.inl"
