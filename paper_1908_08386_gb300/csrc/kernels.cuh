// Device code of the coupled LBM-FVM step (arXiv 1908.08386, Section 5).
//
// State between launches: the post-collision populations f* of the last step
// (structure of arrays [9][ny][pitch], stored as f* - w_i) and the temperature
// T (plane [ny][pitch]).  One launch of step_kernel takes the state from step
// n to n+1:
//   1. pull f^{n+1}_i(x) = f*_i(x - e_i)                         (Eq. 5)
//   2. wall nodes: f_b = f_eq(rho_f, u_wall) + f(x_f) - f_eq(x_f) (Eqs. 94, 96)
//   3. rho^{n+1}, u^{n+1}                                         (Eqs. 16-17)
//   4. T^{n+1} from an explicit finite-volume balance over the node-centred
//      control volume with face velocities from u^{n+1}           (Eq. 76)
//   5. f* = f - (f - f_eq)/tau + F with the Boussinesq force of T^{n+1}
//                                                        (Eqs. 5, 8, 18, 81)
// Step 4 needs u^{n+1} of the four neighbours, so each block first computes
// rho, u for its tile plus a one-node ring (stored in shared memory), then
// updates T and collides its own nodes.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmfvm_dev {

// Node codes: bits 0-1 kind, bits 2-5 partner direction of wall nodes,
// bits 6-7 thermal role.
enum : uint8_t { KIND_FLUID = 0, KIND_WALL = 1, KIND_SOLID = 2 };
enum : uint8_t { TH_FV = 0, TH_DIRICHLET = 1, TH_OBSTACLE = 2, TH_INERT = 3 };
constexpr uint8_t CODE_OUTSIDE = KIND_SOLID | (TH_INERT << 6);

__host__ __device__ __forceinline__ uint8_t make_code(int kind, int dir, int therm) {
    return (uint8_t)(kind | (dir << 2) | (therm << 6));
}

// D2Q9 velocities (Eq. 4): 0 rest, 1 E, 2 N, 3 W, 4 S, 5 NE, 6 NW, 7 SW, 8 SE.
__host__ __device__ constexpr int cx(int q) {
    return (q == 1 || q == 5 || q == 8) ? 1 : ((q == 3 || q == 6 || q == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int q) {
    return (q == 2 || q == 5 || q == 6) ? 1 : ((q == 4 || q == 7 || q == 8) ? -1 : 0);
}
// Run-time direction lookup (partner directions) without a memory table.
__device__ __forceinline__ int cx_rt(int q) { return (int)((0x20919u >> (2 * q)) & 3u) - 1; }
__device__ __forceinline__ int cy_rt(int q) { return (int)((0x02865u >> (2 * q)) & 3u) - 1; }

// Partner direction of a wall node (1..8); anything else reads as 0 (self),
// so a corrupt code can never index outside the one-node ring.
__device__ __forceinline__ int partner_dir(uint8_t code) {
    const int d = (code >> 2) & 15;
    return d > 8 ? 0 : d;
}

// Weights (Eq. 9).
template <class C>
__host__ __device__ constexpr C wq(int q) {
    return q == 0 ? C(4) / C(9) : (q < 5 ? C(1) / C(9) : C(1) / C(36));
}

template <class S> struct Compute { using type = float; };
template <> struct Compute<double> { using type = double; };

__device__ __forceinline__ float ld(const float *p) { return *p; }
__device__ __forceinline__ double ld(const double *p) { return *p; }
__device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ void st(float *p, float v) { *p = v; }
__device__ __forceinline__ void st(double *p, double v) { *p = v; }
__device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

template <class S>
struct StepArgs {
    using C = typename Compute<S>::type;
    const S *fin;
    S *fout;
    const C *Tin;
    C *Tout;
    const uint8_t *code;
    int nx, ny, pitch, perx, pery;
    long long plane;  // ny * pitch
    C omega, alpha, gbeta, t_ref, fx, fy;
    C wall_u[4], wall_v[4];  // velocity of box walls per side W, E, S, N
};

// Second-order part of Eq. 8 divided by rho w_q:
// 3 e.u + 4.5 (e.u)^2 - 1.5 u.u  (c_s^2 = 1/3).
template <class C>
__device__ __forceinline__ C eq_poly(int q, C ux, C uy, C usq) {
    C eu = C(cx(q)) * ux + C(cy(q)) * uy;
    return C(3) * eu + C(4.5) * eu * eu - C(1.5) * usq;
}

// Shifted populations g_q = f_q - w_q pulled into node (x, y) (Eq. 5).
template <class S, class C>
__device__ __forceinline__ void gather(const S *__restrict__ fin, long long plane, int pitch, int nx,
                                       int ny, int x, int y, C g[9]) {
    const int xm = x > 0 ? x - 1 : nx - 1, xp = x < nx - 1 ? x + 1 : 0;
    const int ym = y > 0 ? y - 1 : ny - 1, yp = y < ny - 1 ? y + 1 : 0;
    const S *r0 = fin + (long long)y * pitch;
    const S *rm = fin + (long long)ym * pitch;
    const S *rp = fin + (long long)yp * pitch;
    g[0] = ld(r0 + x);
    g[1] = ld(r0 + 1 * plane + xm);
    g[2] = ld(rm + 2 * plane + x);
    g[3] = ld(r0 + 3 * plane + xp);
    g[4] = ld(rp + 4 * plane + x);
    g[5] = ld(rm + 5 * plane + xm);
    g[6] = ld(rm + 6 * plane + xp);
    g[7] = ld(rp + 7 * plane + xp);
    g[8] = ld(rp + 8 * plane + xm);
}

// Eqs. 16-17 on shifted populations: rho = 1 + sum g, rho u = sum e g.
template <class C>
__device__ __forceinline__ void moments(const C g[9], C &drho, C &ux, C &uy) {
    C s = C(0), jx = C(0), jy = C(0);
#pragma unroll
    for (int q = 0; q < 9; q++) {
        s += g[q];
        if (cx(q) > 0) jx += g[q];
        if (cx(q) < 0) jx -= g[q];
        if (cy(q) > 0) jy += g[q];
        if (cy(q) < 0) jy -= g[q];
    }
    drho = s;
    const C rho = C(1) + s;
    ux = jx / rho;
    uy = jy / rho;
}

// Pre-collision populations and moments of node (x, y) at the new step:
// streamed populations for fluid nodes, non-equilibrium extrapolation from
// the partner for wall nodes, nothing for inert nodes.
template <class S, class C>
__device__ __forceinline__ void node_state(const StepArgs<S> &a, const S *__restrict__ fin, int x,
                                           int y, uint8_t code, C g[9], C &drho, C &ux, C &uy) {
    const int kind = code & 3;
    if (kind == KIND_SOLID) {
#pragma unroll
        for (int q = 0; q < 9; q++) g[q] = C(0);
        drho = C(-1);
        ux = uy = C(0);
        return;
    }
    int sx = x, sy = y;
    if (kind == KIND_WALL) {
        const int d = partner_dir(code);
        sx = x + cx_rt(d);
        sy = y + cy_rt(d);
        sx = sx < 0 ? sx + a.nx : (sx >= a.nx ? sx - a.nx : sx);
        sy = sy < 0 ? sy + a.ny : (sy >= a.ny ? sy - a.ny : sy);
    }
    gather<S, C>(fin, a.plane, a.pitch, a.nx, a.ny, sx, sy, g);
    moments<C>(g, drho, ux, uy);
    if (kind == KIND_WALL) {
        C uw = C(0), vw = C(0);
        if ((code >> 6) != TH_OBSTACLE) {
            const int side = (!a.perx && x == 0) ? 0 : (!a.perx && x == a.nx - 1) ? 1 : (!a.pery && y == 0) ? 2 : 3;
            uw = a.wall_u[side];
            vw = a.wall_v[side];
        }
        const C rho = C(1) + drho;
        const C usw = uw * uw + vw * vw, usf = ux * ux + uy * uy;
#pragma unroll
        for (int q = 0; q < 9; q++)
            g[q] += rho * wq<C>(q) * (eq_poly<C>(q, uw, vw, usw) - eq_poly<C>(q, ux, uy, usf));
        moments<C>(g, drho, ux, uy);
    }
}

// BGK relaxation with the buoyancy force (Eqs. 5, 8, 18), shifted storage.
// The force's pressure is the reference pressure rho0 c_s^2 with rho0 = 1, so
// its momentum source is rho G (the force density of Eq. 75).
template <class S, class C>
__device__ __forceinline__ void collide_store(S *__restrict__ out, long long plane, const C g[9],
                                              C drho, C ux, C uy, C omega, C Gx, C Gy) {
    const C rho = C(1) + drho;
    const C usq = ux * ux + uy * uy;
#pragma unroll
    for (int q = 0; q < 9; q++) {
        const C P = eq_poly<C>(q, ux, uy, usq);
        const C w = wq<C>(q);
        const C feq = w * rho * (C(1) + P);
        const C dfeq = w * (drho + rho * P);
        const C F = C(3) * (Gx * (C(cx(q)) - ux) + Gy * (C(cy(q)) - uy)) * feq;
        st(out + q * plane, g[q] + omega * (dfeq - g[q]) + F);
    }
}

template <class S, int TY>
struct StepSmem {
    using C = typename Compute<S>::type;
    C u[TY + 2][34], v[TY + 2][34], T[TY + 2][34];
    uint8_t c[TY + 2][34];
};

// Map a (possibly one-off) position to the domain; false if outside.
template <class S>
__device__ __forceinline__ bool map_pos(const StepArgs<S> &a, int &x, int &y) {
    if (x < 0 || x >= a.nx) {
        if (!a.perx || x < -1 || x > a.nx) return false;
        x = x < 0 ? a.nx - 1 : 0;
    }
    if (y < 0 || y >= a.ny) {
        if (!a.pery || y < -1 || y > a.ny) return false;
        y = y < 0 ? a.ny - 1 : 0;
    }
    return true;
}

// Fused coupled step.  Block = 32 x TY threads, one per node of its tile.
template <class S, int TY>
__global__ void __launch_bounds__(32 * TY) step_kernel(const StepArgs<S> a) {
    using C = typename Compute<S>::type;
    __shared__ StepSmem<S, TY> sm;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY;
    const int x = x0 + tx, y = y0 + ty;
    const S *__restrict__ fin = a.fin;

    C g[9], drho = C(-1), ux = C(0), uy = C(0);
    bool own = x < a.nx && y < a.ny;
    {
        int mx = x, my = y;
        const bool in = map_pos(a, mx, my);
        uint8_t c = CODE_OUTSIDE;
        C T = C(0);
        if (in) {
            const long long k = (long long)my * a.pitch + mx;
            c = a.code[k];
            T = a.Tin[k];
            node_state<S, C>(a, fin, mx, my, c, g, drho, ux, uy);
        }
        sm.u[ty + 1][tx + 1] = ux;
        sm.v[ty + 1][tx + 1] = uy;
        sm.T[ty + 1][tx + 1] = T;
        sm.c[ty + 1][tx + 1] = c;
    }
    // One-node ring around the tile: 34 below, 34 above, TY left, TY right.
    const int tid = ty * 32 + tx;
    for (int h = tid; h < 68 + 2 * TY; h += 32 * TY) {
        int hx, hy;
        if (h < 34) { hx = h; hy = 0; }
        else if (h < 68) { hx = h - 34; hy = TY + 1; }
        else { const int r = h - 68; hx = (r & 1) ? 33 : 0; hy = 1 + (r >> 1); }
        int mx = x0 + hx - 1, my = y0 + hy - 1;
        const bool in = map_pos(a, mx, my);
        uint8_t c = CODE_OUTSIDE;
        C T = C(0), hg[9], hd, hu = C(0), hv = C(0);
        if (in) {
            const long long k = (long long)my * a.pitch + mx;
            c = a.code[k];
            T = a.Tin[k];
            node_state<S, C>(a, fin, mx, my, c, hg, hd, hu, hv);
        }
        sm.u[hy][hx] = hu;
        sm.v[hy][hx] = hv;
        sm.T[hy][hx] = T;
        sm.c[hy][hx] = c;
    }
    __syncthreads();
    if (!own) return;
    const uint8_t c = sm.c[ty + 1][tx + 1];
    if ((c & 3) == KIND_SOLID) return;
    const int th = c >> 6;
    const C TP = sm.T[ty + 1][tx + 1];
    C Tn = TP;
    if (th == TH_FV) {
        // Control volume [x-1/2, x+1/2] x [y-1/2, y+1/2] clipped to the box.
        const C ex = a.perx ? C(1) : C(0.5) * C(x > 0) + C(0.5) * C(x < a.nx - 1);
        const C ey = a.pery ? C(1) : C(0.5) * C(y > 0) + C(0.5) * C(y < a.ny - 1);
        const C uP = sm.u[ty + 1][tx + 1], vP = sm.v[ty + 1][tx + 1];
        C acc = C(0);
        // faces E, N, W, S; a face is open when the neighbour takes part in
        // the balance (FV or Dirichlet node).
        {
            const int nx_ = tx + 2, ny_ = ty + 1;
            if ((sm.c[ny_][nx_] >> 6) <= TH_DIRICHLET) {
                const C Tn_ = sm.T[ny_][nx_];
                const C Fl = ey * (C(0.5) * (uP + sm.u[ny_][nx_]));
                acc += -Fl * (C(0.5) * (TP + Tn_)) + a.alpha * ey * (Tn_ - TP);
            }
        }
        {
            const int nx_ = tx + 1, ny_ = ty + 2;
            if ((sm.c[ny_][nx_] >> 6) <= TH_DIRICHLET) {
                const C Tn_ = sm.T[ny_][nx_];
                const C Fl = ex * (C(0.5) * (vP + sm.v[ny_][nx_]));
                acc += -Fl * (C(0.5) * (TP + Tn_)) + a.alpha * ex * (Tn_ - TP);
            }
        }
        {
            const int nx_ = tx, ny_ = ty + 1;
            if ((sm.c[ny_][nx_] >> 6) <= TH_DIRICHLET) {
                const C Tn_ = sm.T[ny_][nx_];
                const C Fl = ey * (C(-0.5) * (uP + sm.u[ny_][nx_]));
                acc += -Fl * (C(0.5) * (TP + Tn_)) + a.alpha * ey * (Tn_ - TP);
            }
        }
        {
            const int nx_ = tx + 1, ny_ = ty;
            if ((sm.c[ny_][nx_] >> 6) <= TH_DIRICHLET) {
                const C Tn_ = sm.T[ny_][nx_];
                const C Fl = ex * (C(-0.5) * (vP + sm.v[ny_][nx_]));
                acc += -Fl * (C(0.5) * (TP + Tn_)) + a.alpha * ex * (Tn_ - TP);
            }
        }
        Tn = TP + acc / (ex * ey);
    } else if (th == TH_OBSTACLE) {
        const int d = partner_dir(c);
        Tn = sm.T[ty + 1 + cy_rt(d)][tx + 1 + cx_rt(d)];
    }
    const long long k = (long long)y * a.pitch + x;
    a.Tout[k] = Tn;
    const C Gy = a.fy + a.gbeta * (Tn - a.t_ref);
    collide_store<S, C>(a.fout + k, a.plane, g, drho, ux, uy, a.omega, a.fx, Gy);
}

// Initial state: f^0 = f_eq(1, u0) (kept unrelaxed in f0_out for the step-0
// field export), T^0, and the post-collision f*^0 in fstar_out.
template <class S>
__global__ void init_kernel(const StepArgs<S> a, S *f0_out, S *fstar_out, const float *u0,
                            const float *v0, const float *T0, double t_init, const double *t_wall_side,
                            int bcW, int bcE, int bcS, int bcN, typename Compute<S>::type *T_a,
                            typename Compute<S>::type *T_b) {
    using C = typename Compute<S>::type;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const long long k = (long long)y * a.pitch + x;
    const long long kin = (long long)y * a.nx + x;
    const uint8_t c = a.code[k];
    C T = T0 ? C(T0[kin]) : C(t_init);
    if ((c >> 6) == TH_DIRICHLET) {
        // Vertical sides own the corners.
        if (!a.perx && x == 0 && bcW == 0) T = C(t_wall_side[0]);
        else if (!a.perx && x == a.nx - 1 && bcE == 0) T = C(t_wall_side[1]);
        else if (!a.pery && y == 0 && bcS == 0) T = C(t_wall_side[2]);
        else T = C(t_wall_side[3]);
    }
    T_a[k] = T;
    T_b[k] = T;
    if ((c & 3) == KIND_SOLID) {
#pragma unroll
        for (int q = 0; q < 9; q++) {
            st(f0_out + k + q * a.plane, C(0));
            st(fstar_out + k + q * a.plane, C(0));
        }
        return;
    }
    const C u = u0 ? C(u0[kin]) : C(0), v = v0 ? C(v0[kin]) : C(0);
    const C usq = u * u + v * v;
    C g[9];
#pragma unroll
    for (int q = 0; q < 9; q++) {
        g[q] = wq<C>(q) * eq_poly<C>(q, u, v, usq);
        st(f0_out + k + q * a.plane, g[q]);
    }
    C drho, ux, uy;
    moments<C>(g, drho, ux, uy);
    const C Gy = a.fy + a.gbeta * (T - a.t_ref);
    collide_store<S, C>(fstar_out + k, a.plane, g, drho, ux, uy, a.omega, a.fx, Gy);
}

// Pre-collision moments of the current step: re-pulled from the previous
// post-collision buffer (direct = 0), or read in place from the unrelaxed
// initial populations (direct = 1, step 0).
template <class S>
__device__ __forceinline__ void current_moments(const StepArgs<S> &a, int direct, int x, int y,
                                                uint8_t c, typename Compute<S>::type &drho,
                                                typename Compute<S>::type &ux,
                                                typename Compute<S>::type &uy) {
    using C = typename Compute<S>::type;
    C g[9];
    if (direct) {
        if ((c & 3) == KIND_SOLID) {
            drho = C(-1);
            ux = uy = C(0);
            return;
        }
        const long long k = (long long)y * a.pitch + x;
#pragma unroll
        for (int q = 0; q < 9; q++) g[q] = ld(a.fin + k + q * a.plane);
        moments<C>(g, drho, ux, uy);
    } else {
        node_state<S, C>(a, a.fin, x, y, c, g, drho, ux, uy);
    }
}

// Field export: two of (rho, u, v, T) selected by `which` (0 = rho,u; 1 = v,T)
// into out0/out1 (row-major ny*nx), in double or float.
template <class S, class O>
__global__ void fields_kernel(const StepArgs<S> a, int direct, int which, O *out0, O *out1) {
    using C = typename Compute<S>::type;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const long long k = (long long)y * a.pitch + x;
    const long long ko = (long long)y * a.nx + x;
    const uint8_t c = a.code[k];
    C drho, ux, uy;
    current_moments<S>(a, direct, x, y, c, drho, ux, uy);
    const bool inert = (c & 3) == KIND_SOLID;
    if (which == 0) {
        out0[ko] = O(inert ? C(0) : C(1) + drho);
        out1[ko] = O(ux);
    } else {
        out0[ko] = O(uy);
        out1[ko] = O(a.Tin[k]);
    }
}

// Residual, pass 1: per-block FP64 sums of |u - u_snap|^2 and |u|^2 over
// fluid nodes, snapshot update; partials[2*b], partials[2*b+1].
// Fixed assignment of nodes to threads and a fixed reduction tree make the
// result independent of scheduling.
template <class S>
__global__ void __launch_bounds__(256) residual_kernel(const StepArgs<S> a, int direct, double *su,
                                                       double *sv, double *partials, int update_only) {
    using C = typename Compute<S>::type;
    __shared__ double red[2][8];
    const long long n = (long long)a.nx * a.ny;
    double num = 0.0, den = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / a.nx), x = (int)(i - (long long)y * a.nx);
        const long long k = (long long)y * a.pitch + x;
        const uint8_t c = a.code[k];
        if ((c & 3) != KIND_FLUID) continue;
        C drho, ux, uy;
        current_moments<S>(a, direct, x, y, c, drho, ux, uy);
        const double du = (double)ux - su[i], dv = (double)uy - sv[i];
        num += du * du + dv * dv;
        den += (double)ux * (double)ux + (double)uy * (double)uy;
        su[i] = (double)ux;
        sv[i] = (double)uy;
    }
    if (update_only) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_down_sync(0xffffffffu, num, o);
        den += __shfl_down_sync(0xffffffffu, den, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = num;
        red[1][wid] = den;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            a0 += red[0][w];
            a1 += red[1][w];
        }
        partials[2 * blockIdx.x] = a0;
        partials[2 * blockIdx.x + 1] = a1;
    }
}

// Residual, pass 2: one warp sums the block partials in a fixed order.
__global__ void residual_finish_kernel(const double *partials, int nblocks, double *out) {
    double a0 = 0.0, a1 = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 32) {
        a0 += partials[2 * b];
        a1 += partials[2 * b + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_down_sync(0xffffffffu, a0, o);
        a1 += __shfl_down_sync(0xffffffffu, a1, o);
    }
    if (threadIdx.x == 0) {
        out[0] = a0;
        out[1] = a1;
    }
}

// Nusselt number (Eq. 90) along the west (hot) and east (cold) walls in FP64:
// local values into loc[0..ny), trapezoid means into out[0], out[1].
template <class S>
__global__ void __launch_bounds__(256) nusselt_kernel(const StepArgs<S> a, double H, double dT,
                                                      double *loc, double *out) {
    __shared__ double red[2][8];
    double sh = 0.0, sc = 0.0;
    const int nx = a.nx;
    for (int j = threadIdx.x; j < a.ny; j += blockDim.x) {
        const auto *r = a.Tin + (long long)j * a.pitch;
        const double t0 = r[0], t1 = r[1], t2 = r[2];
        const double e0 = r[nx - 1], e1 = r[nx - 2], e2 = r[nx - 3];
        const double nh = -H * (-3.0 * t0 + 4.0 * t1 - t2) / (2.0 * dT);
        const double nc = -H * (3.0 * e0 - 4.0 * e1 + e2) / (2.0 * dT);
        loc[j] = nh;
        const double w = (j == 0 || j == a.ny - 1) ? 0.5 : 1.0;
        sh += w * nh;
        sc += w * nc;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sh += __shfl_down_sync(0xffffffffu, sh, o);
        sc += __shfl_down_sync(0xffffffffu, sc, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = sh;
        red[1][wid] = sc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            a0 += red[0][w];
            a1 += red[1][w];
        }
        out[0] = a0 / H;
        out[1] = a1 / H;
    }
}

}  // namespace lbmfvm_dev
