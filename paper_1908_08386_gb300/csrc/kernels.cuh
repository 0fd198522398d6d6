// Device code of the coupled LBM-FVM step (arXiv 1908.08386, Section 5).
//
// State between launches: the post-collision populations f* of the last step
// (structure of arrays [9][ny][pitch], stored as f* - w_i) and the temperature
// T (plane [ny][pitch]).  One launch of a step kernel takes the state from
// step n to n+1:
//   1. pull f^{n+1}_i(x) = f*_i(x - e_i)                         (Eq. 5)
//   2. wall nodes: f_b = f_eq(rho_f, u_wall) + f(x_f) - f_eq(x_f) (Eqs. 94, 96)
//   3. rho^{n+1}, u^{n+1}                                         (Eqs. 16-17)
//   4. T^{n+1} from an explicit finite-volume balance over the node-centred
//      control volume with face velocities from u^{n+1}           (Eq. 76)
//   5. f* = f - (f - f_eq)/tau + F with the Boussinesq force of T^{n+1}
//                                                        (Eqs. 5, 8, 18, 81)
// Step 4 needs u^{n+1} of the four neighbours, so each block first computes
// rho, u for its tile plus a one-node ring (kept in shared memory), then
// updates T and collides its own nodes.
//
// Two kernels share this arithmetic:
//   step_tma_kernel  persistent, one block per SM, each tile's populations,
//                    temperature and node codes staged in shared memory by
//                    TMA through a multi-stage mbarrier pipeline, results
//                    written back by TMA bulk stores (walled domains,
//                    FP32/FP16/BF16 storage);
//   step_kernel      one block per tile, gathers straight from global memory
//                    (periodic sides, FP64 storage).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbmfvm_dev {

// Node codes: bits 0-1 kind, bits 2-5 partner direction of wall nodes,
// bits 6-7 thermal role.  Memory holds code ^ CODE_OUTSIDE, so that the zero
// fill of a TMA box beyond the grid decodes as "outside".
enum : uint8_t { KIND_FLUID = 0, KIND_WALL = 1, KIND_SOLID = 2 };
enum : uint8_t { TH_FV = 0, TH_DIRICHLET = 1, TH_OBSTACLE = 2, TH_INERT = 3 };
constexpr uint8_t CODE_OUTSIDE = KIND_SOLID | (TH_INERT << 6);

__host__ __device__ __forceinline__ uint8_t make_code(int kind, int dir, int therm) {
    return (uint8_t)(kind | (dir << 2) | (therm << 6));
}
__host__ __device__ __forceinline__ uint8_t stored_code(uint8_t code) { return code ^ CODE_OUTSIDE; }
__host__ __device__ __forceinline__ uint8_t decode(uint8_t stored) { return stored ^ CODE_OUTSIDE; }

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

// ---------------------------------------------------------------------------
// Double-single numbers: a value held as the unevaluated sum hi + lo of two
// FP32 numbers (|lo| <= half an ulp of hi), about 48 significant bits,
// computed on the FP32 units.  On this GPU the FP32 units outnumber the
// FP64 ones many times over, so the last stage of a run to a tight residual
// (where FP32 storage and arithmetic leave a rounding floor near 2e-7) runs
// in double-single rather than FP64.  The operations are the error-free
// transformations of floating-point arithmetic: the two-sum of Knuth (exact
// sum and rounding error of two floats), the fast two-sum of Dekker (the same
// when |a| >= |b|) and the two-product from a fused multiply-add (exact
// product and rounding error); additions accumulate the low parts and
// renormalise once (error a few units of 2^-44 of the operands).  The
// intrinsics __fadd_rn/__fmul_rn keep the compiler from contracting these
// sequences into fused operations, which would break their exactness.
// ---------------------------------------------------------------------------
struct __align__(8) dsf {
    float hi, lo;
    dsf() = default;
    __host__ __device__ constexpr dsf(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr dsf(float f) : hi(f), lo(0.0f) {}
    __host__ __device__ constexpr dsf(int i) : hi((float)i), lo(0.0f) {}  // exact for |i| < 2^24
    __host__ __device__ constexpr dsf(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ dsf ds_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return dsf(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ dsf ds_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dsf(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dsf operator+(dsf x, dsf y) {
    const dsf s = ds_two_sum(x.hi, y.hi);
    return ds_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dsf operator-(dsf x) { return dsf(-x.hi, -x.lo); }
__device__ __forceinline__ dsf operator-(dsf x, dsf y) { return x + (-y); }
__device__ __forceinline__ dsf operator*(dsf x, dsf y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);  // exact rounding error of the product
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return ds_fast_two_sum(p, e);
}
__device__ __forceinline__ dsf &operator+=(dsf &x, dsf y) { return x = x + y; }
__device__ __forceinline__ bool operator<(dsf a, dsf b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(dsf a, dsf b) { return b < a; }

template <class S> struct Compute { using type = float; };
template <> struct Compute<dsf> { using type = dsf; };

// The weights in double-single, split from their FP64 values.
template <>
__host__ __device__ constexpr dsf wq<dsf>(int q) {
    return q == 0 ? dsf(4.0 / 9.0) : (q < 5 ? dsf(1.0 / 9.0) : dsf(1.0 / 36.0));
}
template <> struct Compute<double> { using type = double; };

__device__ __forceinline__ float ld(const float *p) { return *p; }
__device__ __forceinline__ double ld(const double *p) { return *p; }
__device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ void st(float *p, float v) { *p = v; }
__device__ __forceinline__ void st(double *p, double v) { *p = v; }
__device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

__device__ __forceinline__ float recip(float r) { return __frcp_rn(r); }
__device__ __forceinline__ dsf ld(const dsf *p) { return *p; }
__device__ __forceinline__ void st(dsf *p, dsf v) { *p = v; }
// 1/r: the FP32 reciprocal of the high part, refined by one Newton step
// q + q (1 - r q) in double-single (the error squares: ~2^-46).
__device__ __forceinline__ dsf recip(dsf r) {
    const dsf q(__frcp_rn(r.hi));
    return q + q * (dsf(1.0f) - r * q);
}
__device__ __forceinline__ double recip(double r) { return 1.0 / r; }

template <class S>
struct StepArgs {
    using C = typename Compute<S>::type;
    const S *fin;
    S *fout;
    const C *Tin;
    C *Tout;
    const uint8_t *code;  // stored codes (code ^ CODE_OUTSIDE)
    int nx, ny, pitch, perx, pery;
    long long plane;  // ny * pitch
    C omega, alpha, gbeta, t_ref, fx, fy;
    C wall_u[4], wall_v[4];  // velocity of box walls per side W, E, S, N
    int *err;                // device status word (bounded waits that ran out)
    int stall;               // test hook: block 0 skips its first staged load
    int wall_fd;             // generic kernel: finite-difference velocity-gradient box walls
    C fd_coef;               // their 3 tau (tau w_i / c_s^2 = 3 tau w_i)
};

// One cavity of the TMA path: its rectangle in the (possibly multi-cavity)
// node arrays, which starts on a tile corner, and its lattice parameters.
// Wall velocities are kept in both arithmetic precisions (FP64 conversions
// are slow on this GPU; no kernel converts).
struct CavityDesc {
    int x0, y0, nx, ny;
    double omega, alpha, gbeta, t_ref, fx, fy;
    double wall_u[4], wall_v[4];    // box-wall velocity per side W, E, S, N
    float wall_uf[4], wall_vf[4];   // the same in FP32
    int substeps;                   // finite-volume sub-steps per lattice step (>= 1)
    int pad;
};

// One tile of the TMA path: what a block needs to know about it.  A tile
// holds nodes of one cavity only (plus unused padding beyond its rectangle).
// The host writes the list; the issuing thread copies a tile's header next
// to its stage with the same bulk-copy barrier as the tile's data.
// The lattice parameters come in every arithmetic precision, rounded by the
// host, so that no kernel converts (FP64 conversions are slow on this GPU):
// FP64, FP32, and the low parts that make (FP32, low) the double-single value.
struct TileHeader {
    int x0, y0, ox, oy, nx, ny, cav;  // origin; origin relative to the cavity; cavity size; cavity
    int substeps;                     // finite-volume sub-steps per lattice step of the cavity (>= 1)
    double omega, alpha, gbeta, t_ref, fx, fy;
    float omega_f, alpha_f, gbeta_f, t_ref_f, fx_f, fy_f, dt_f, pad2;       // dt = 1 / substeps
    float omega_lo, alpha_lo, gbeta_lo, t_ref_lo, fx_lo, fy_lo, dt_lo, pad4;
};
static_assert(sizeof(TileHeader) == 144, "tile headers are 144-byte bulk copies");


// ---------------------------------------------------------------------------
// Arithmetic shared by both step kernels and the export kernels.
// ---------------------------------------------------------------------------

// Second-order part of Eq. 8 divided by rho w_q: 3 e.u + 4.5 (e.u)^2 - 1.5 u.u.
template <class C>
__device__ __forceinline__ C eq_poly(int q, C ux, C uy, C usq) {
    C eu = C(cx(q)) * ux + C(cy(q)) * uy;
    return C(3) * eu + C(4.5) * eu * eu - C(1.5) * usq;
}

// a b + c rounded once and a b rounded on its own, whatever the compiler
// would contract by itself: a product that feeds several sums may be fused
// into some of them, and a choice that differed between kernel
// instantiations would make tile shapes disagree in the last bit.  Double-
// single has no fused form and keeps its compensated product and sum.
__device__ __forceinline__ float fma_c(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_c(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ dsf fma_c(dsf a, dsf b, dsf c) { return a * b + c; }
__device__ __forceinline__ float mul_r(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_r(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ dsf mul_r(dsf a, dsf b) { return a * b; }

// Eqs. 16-17 on shifted populations g = f - w: rho = 1 + sum g, rho u = sum e g.
template <class C>
__device__ __forceinline__ void moments(const C g[9], C &drho, C &ux, C &uy) {
    const C s = (((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7]))) + g[8];
    const C jx = ((g[1] + g[5]) + g[8]) - ((g[3] + g[6]) + g[7]);
    const C jy = ((g[2] + g[5]) + g[6]) - ((g[4] + g[7]) + g[8]);
    const C inv = recip(C(1) + s);
    drho = s;
    ux = mul_r(jx, inv);
    uy = mul_r(jy, inv);
}

// Non-equilibrium extrapolation (Eq. 94): g holds the partner's populations
// and moments on entry; on exit the wall node's, with rho_b = rho_f (Eq. 96)
// and the wall velocity (uw, vw).
template <class C>
__device__ __forceinline__ void nee(C g[9], C &drho, C &ux, C &uy, C uw, C vw) {
    // g_q += rho w_q (P_q(u_w) - P_q(u_f)); opposite directions share the
    // even part 4.5 (e.u)^2 - 1.5 u.u and differ in the sign of 3 e.u.
    const C rho = C(1) + drho;
    const C dP0 = mul_r(C(-1.5), fma_c(uw, uw, mul_r(vw, vw)) - fma_c(ux, ux, mul_r(uy, uy)));
    g[0] = fma_c(mul_r(rho, wq<C>(0)), dP0, g[0]);
    auto pair = [&](int q, int qb, C euw, C euf) {
        const C A = fma_c(C(4.5), fma_c(euw, euw, -mul_r(euf, euf)), dP0), B = mul_r(C(3), euw - euf);
        const C rw = mul_r(rho, wq<C>(q));
        g[q] = fma_c(rw, A + B, g[q]);
        g[qb] = fma_c(rw, A - B, g[qb]);
    };
    pair(1, 3, uw, ux);
    pair(2, 4, vw, uy);
    pair(5, 7, uw + vw, ux + uy);
    pair(6, 8, vw - uw, uy - ux);
    moments<C>(g, drho, ux, uy);
}

// BGK relaxation with the buoyancy force (Eqs. 5, 8, 18) on shifted storage.
// The force's pressure is the reference pressure rho0 c_s^2 with rho0 = 1, so
// its momentum source is rho G (the force density of Eq. 75).  With
// P_q = 3 e.u + 4.5 (e.u)^2 - 1.5 u.u and h_q = G.(e_q - u):
//   f_eq - w = w (drho + rho P),  F = 3 h f_eq = 3 h w rho (1 + P),
//   g* = (1 - omega) g + w [omega drho + 3 rho h + P (omega rho + 3 rho h)].
// Directions are taken in opposite pairs (1, 3), (2, 4), (5, 7), (6, 8): for
// e = e_q, with s = 3 rho e.G - 3 rho G.u, A = 4.5 (e.u)^2 - 1.5 u.u and
// B = 3 e.u, the pair's results are
//   g*_q = (1 - omega) g_q + w [(omega drho + s) + (A + B)(omega rho + s)]
// and the same with -3 rho e.G and -B for the opposite direction; the rest
// direction has e = 0.  s joins omega rho inside one fused multiply-add:
// rounding omega rho first and adding s afterwards would round a value on
// the FP32 grid plus a nearly constant s the same way at every node (a body
// force gives every node the same 3 rho G.e), a mass drift of about 1e-10
// per node and step.
template <class C, class Store>
__device__ __forceinline__ void collide(const C g[9], C drho, C ux, C uy, C omega, C Gx, C Gy, Store store) {
    const C rho = C(1) + drho;
    const C P0 = mul_r(C(-1.5), fma_c(ux, ux, mul_r(uy, uy)));
    const C c = mul_r(C(3), rho);
    const C sx = mul_r(c, Gx), sy = mul_r(c, Gy);
    const C sGu = fma_c(sx, ux, mul_r(sy, uy));
    const C om1 = C(1) - omega;
    auto out = [&](int q, C P, C s) {
        const C w = wq<C>(q);
        store(q, fma_c(om1, g[q], mul_r(w, fma_c(P, fma_c(omega, rho, s), fma_c(omega, drho, s)))));
    };
    out(0, P0, -sGu);
    auto pair = [&](int q, int qb, C eu, C es) {
        const C A = fma_c(C(4.5), mul_r(eu, eu), P0), B = mul_r(C(3), eu);
        out(q, A + B, es - sGu);
        out(qb, A - B, -es - sGu);
    };
    pair(1, 3, ux, sx);
    pair(2, 4, uy, sy);
    pair(5, 7, ux + uy, sx + sy);
    pair(6, 8, uy - ux, sy - sx);
}

// Explicit finite-volume update (forward Euler, dt = 1) of a node-centred
// control volume of extents ex x ey: central face temperatures, face
// velocities the mean of the two node velocities, closed faces carry nothing.
template <class C>
__device__ __forceinline__ C fv_update(C TP, C uP, C vP, C ex, C ey, C alpha, bool oE, C TE, C uE, bool oN, C TN,
                                       C vN, bool oW, C TW, C uW, bool oS, C TS, C vS) {
    const C q = C(0.25);
    const C fe = oE ? alpha * (TE - TP) - q * (uP + uE) * (TP + TE) : C(0);
    const C fw = oW ? alpha * (TW - TP) + q * (uP + uW) * (TP + TW) : C(0);
    const C fn = oN ? alpha * (TN - TP) - q * (vP + vN) * (TP + TN) : C(0);
    const C fs = oS ? alpha * (TS - TP) + q * (vP + vS) * (TP + TS) : C(0);
    // 1/(ex ey) is a power of two (ex, ey in {1/2, 1}): the product is exact.
    const C inv_v = (ex < C(1) ? C(2) : C(1)) * (ey < C(1) ? C(2) : C(1));
    return TP + (ey * (fe + fw) + ex * (fn + fs)) * inv_v;
}

// QUICK face value (Leonard's quadratic upstream interpolation, the scheme
// Section 3.1 names for its finite-volume solver).  un: the face's normal
// velocity, outward from P; Tn: the neighbour across the face.  With U the
// upstream node, D the downstream one and UU the node beyond U,
// T_f = 6/8 T_U + 3/8 T_D - 1/8 T_UU; where UU takes no part in the energy
// balance (farP / farN false) the face keeps the central value.  farP, TfarP:
// the node beyond P (upstream P); farN, TfarN: the node beyond the neighbour.
template <class C>
__device__ __forceinline__ C quick_face(C un, C TP, C Tn, bool farP, C TfarP, bool farN, C TfarN) {
    if (!(un < C(0))) {
        if (farP) return C(0.75) * TP + C(0.375) * Tn - C(0.125) * TfarP;
    } else if (farN) {
        return C(0.75) * Tn + C(0.375) * TP - C(0.125) * TfarN;
    }
    return C(0.5) * (TP + Tn);
}

// Explicit finite-volume update with given face temperatures (QUICK) and a
// time step dt (1/m for m sub-steps): V_P (T' - T_P) = dt sum over open faces
// of [-F_f T_f + alpha A_f (T_nb - T_P)], F_f = A_f u_face.n, u_face the mean
// of the two node velocities.
template <class C>
__device__ __forceinline__ C fv_update_faces(C TP, C uP, C vP, C ex, C ey, C alpha, C dt, bool oE, C TE, C uE, C TfE,
                                             bool oN, C TN, C vN, C TfN, bool oW, C TW, C uW, C TfW, bool oS, C TS,
                                             C vS, C TfS) {
    const C h = C(0.5);
    const C fe = oE ? alpha * (TE - TP) - h * (uP + uE) * TfE : C(0);
    const C fw = oW ? alpha * (TW - TP) + h * (uP + uW) * TfW : C(0);
    const C fn = oN ? alpha * (TN - TP) - h * (vP + vN) * TfN : C(0);
    const C fs = oS ? alpha * (TS - TP) + h * (vP + vS) * TfS : C(0);
    const C inv_v = (ex < C(1) ? C(2) : C(1)) * (ey < C(1) ? C(2) : C(1));
    return TP + dt * ((ey * (fe + fw) + ex * (fn + fs)) * inv_v);
}

__host__ __device__ __forceinline__ bool fv_open(uint8_t code) { return (code >> 6) <= TH_DIRICHLET; }

// Face flags of the finite-volume update, one byte per node in a plane beside
// the codes (written by the host): which faces of the node's control volume
// are open (the neighbour lies in the cavity and is a finite-volume or
// Dirichlet node) and which neighbours lie in the cavity (the control
// volume's extents).  Outside every cavity the byte is 0.
enum : uint8_t {
    FF_OPEN_E = 1, FF_OPEN_N = 2, FF_OPEN_W = 4, FF_OPEN_S = 8,
    FF_IN_W = 16, FF_IN_E = 32, FF_IN_S = 64, FF_IN_N = 128
};

// Velocity of a box wall node from its side (vertical sides own the corners).
template <class S>
__device__ __forceinline__ void wall_velocity(const StepArgs<S> &a, int x, int y, uint8_t code,
                                              typename Compute<S>::type &uw, typename Compute<S>::type &vw) {
    using C = typename Compute<S>::type;
    uw = vw = C(0);
    if ((code >> 6) != TH_OBSTACLE) {
        const int side = (!a.perx && x == 0) ? 0 : (!a.perx && x == a.nx - 1) ? 1 : (!a.pery && y == 0) ? 2 : 3;
        uw = a.wall_u[side];
        vw = a.wall_v[side];
    }
}

// ---------------------------------------------------------------------------
// Generic path: gathers straight from global memory.
// ---------------------------------------------------------------------------

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

// Velocity of node (x, y) at the new step for the finite-difference wall
// gradients: wall nodes move with their wall, fluid nodes from their pulled
// populations, inert nodes rest; positions wrap across periodic sides.
template <class S, class C>
__device__ __forceinline__ void fd_velocity(const StepArgs<S> &a, const S *__restrict__ fin, int x, int y, C &u,
                                            C &v) {
    x = x < 0 ? x + a.nx : (x >= a.nx ? x - a.nx : x);
    y = y < 0 ? y + a.ny : (y >= a.ny ? y - a.ny : y);
    const uint8_t c = decode(a.code[(long long)y * a.pitch + x]);
    u = v = C(0);
    if ((c & 3) == KIND_WALL) {
        wall_velocity<S>(a, x, y, c, u, v);
    } else if ((c & 3) == KIND_FLUID) {
        C g[9], d;
        gather<S, C>(fin, a.plane, a.pitch, a.nx, a.ny, x, y, g);
        moments<C>(g, d, u, v);
    }
}

// d(u, v)/d(axis) at (x, y): second-order one-sided into the domain at a
// walled box side, centred elsewhere.
template <class S, class C>
__device__ __forceinline__ void fd_gradient(const StepArgs<S> &a, const S *__restrict__ fin, int x, int y, int axis,
                                            C &du, C &dv) {
    const int dx = axis == 0, dy = axis == 1;
    const bool lo = axis == 0 ? (!a.perx && x == 0) : (!a.pery && y == 0);
    const bool hi = axis == 0 ? (!a.perx && x == a.nx - 1) : (!a.pery && y == a.ny - 1);
    C u0, v0, u1, v1, u2, v2;
    if (lo || hi) {
        const int sg = lo ? 1 : -1;
        fd_velocity<S, C>(a, fin, x, y, u0, v0);
        fd_velocity<S, C>(a, fin, x + sg * dx, y + sg * dy, u1, v1);
        fd_velocity<S, C>(a, fin, x + 2 * sg * dx, y + 2 * sg * dy, u2, v2);
        const C h = C(0.5) * C(sg);
        du = h * (C(-3) * u0 + C(4) * u1 - u2);
        dv = h * (C(-3) * v0 + C(4) * v1 - v2);
    } else {
        fd_velocity<S, C>(a, fin, x + dx, y + dy, u1, v1);
        fd_velocity<S, C>(a, fin, x - dx, y - dy, u2, v2);
        du = C(0.5) * (u1 - u2);
        dv = C(0.5) * (v1 - v2);
    }
}

// Finite-difference velocity-gradient wall (Section 3, Eqs. 67, 69-72) on
// shifted storage: g_b = w (drho_f + rho_f P(u_w) - 3 tau rho_f Q : S), with
// the partner's density (Eq. 96), the wall velocity, S from the new velocity
// field and the normal strain from continuity off the corners (Eq. 72).
// On entry drho holds the partner's density deviation.
template <class S, class C>
__device__ __forceinline__ void fd_wall(const StepArgs<S> &a, const S *__restrict__ fin, int x, int y,
                                        uint8_t code, C g[9], C &drho, C &ux, C &uy) {
    C uw, vw, dudx, dvdx, dudy, dvdy;
    wall_velocity<S>(a, x, y, code, uw, vw);
    fd_gradient<S, C>(a, fin, x, y, 0, dudx, dvdx);
    fd_gradient<S, C>(a, fin, x, y, 1, dudy, dvdy);
    const bool vert = !a.perx && (x == 0 || x == a.nx - 1), hor = !a.pery && (y == 0 || y == a.ny - 1);
    if (vert && !hor) dudx = -dvdy;
    if (hor && !vert) dvdy = -dudx;
    const C sxx = dudx, syy = dvdy, sxy = C(0.5) * (dudy + dvdx);
    const C rho = C(1) + drho, usq = uw * uw + vw * vw;
    const C third = C(1.0 / 3.0);
#pragma unroll
    for (int q = 0; q < 9; q++) {
        const C ex = C(cx(q)), ey = C(cy(q));
        const C qs = (ex * ex - third) * sxx + C(2) * ex * ey * sxy + (ey * ey - third) * syy;
        g[q] = wq<C>(q) * (drho + rho * eq_poly<C>(q, uw, vw, usq) - a.fd_coef * rho * qs);
    }
    moments<C>(g, drho, ux, uy);
}

// Pre-collision populations and moments of node (x, y) at the new step:
// streamed populations for fluid nodes, non-equilibrium extrapolation from
// the partner for wall nodes (or the finite-difference velocity-gradient
// scheme on box walls), nothing for inert nodes.
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
        if (a.wall_fd && (code >> 6) != TH_OBSTACLE) {
            fd_wall<S, C>(a, fin, x, y, code, g, drho, ux, uy);
        } else {
            C uw, vw;
            wall_velocity<S>(a, x, y, code, uw, vw);
            nee<C>(g, drho, ux, uy, uw, vw);
        }
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

// Fused coupled step, generic path.  Block = 32 x TY threads, one per node.
template <class S, int TY>
__global__ void __launch_bounds__(32 * TY) step_kernel(const StepArgs<S> a) {
    using C = typename Compute<S>::type;
    __shared__ StepSmem<S, TY> sm;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY;
    const int x = x0 + tx, y = y0 + ty;
    const S *__restrict__ fin = a.fin;

    C g[9], drho = C(-1), ux = C(0), uy = C(0);
    const bool own = x < a.nx && y < a.ny;
    {
        int mx = x, my = y;
        const bool in = map_pos(a, mx, my);
        uint8_t c = CODE_OUTSIDE;
        C T = C(0);
        if (in) {
            const long long k = (long long)my * a.pitch + mx;
            c = decode(a.code[k]);
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
            c = decode(a.code[k]);
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
        const C ex = a.perx ? C(1) : C(0.5) * C(x > 0) + C(0.5) * C(x < a.nx - 1);
        const C ey = a.pery ? C(1) : C(0.5) * C(y > 0) + C(0.5) * C(y < a.ny - 1);
        const int i = tx + 1, j = ty + 1;
        Tn = fv_update<C>(TP, sm.u[j][i], sm.v[j][i], ex, ey, a.alpha,
                          fv_open(sm.c[j][i + 1]), sm.T[j][i + 1], sm.u[j][i + 1],
                          fv_open(sm.c[j + 1][i]), sm.T[j + 1][i], sm.v[j + 1][i],
                          fv_open(sm.c[j][i - 1]), sm.T[j][i - 1], sm.u[j][i - 1],
                          fv_open(sm.c[j - 1][i]), sm.T[j - 1][i], sm.v[j - 1][i]);
    } else if (th == TH_OBSTACLE) {
        const int d = partner_dir(c);
        Tn = sm.T[ty + 1 + cy_rt(d)][tx + 1 + cx_rt(d)];
    }
    const long long k = (long long)y * a.pitch + x;
    a.Tout[k] = Tn;
    const C Gy = a.fy + a.gbeta * (Tn - a.t_ref);
    S *out = a.fout + k;
    const long long plane = a.plane;
    collide<C>(g, drho, ux, uy, a.omega, a.fx, Gy, [&](int q, C v) { st(out + q * plane, v); });
}

// ---------------------------------------------------------------------------
// TMA path.
// ---------------------------------------------------------------------------
namespace tma {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Orders this thread's earlier generic-proxy shared-memory accesses (made
// visible to it by a block barrier) before later async-proxy (TMA) writes.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of the barrier; false once `limit_ns` has passed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 0;; it++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && globaltimer() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// Untiled bulk copy (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void load_bytes(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace tma

// Tile geometry of the TMA tile path.  A tile is TW x TH output nodes at
// (x0, y0), NPT of them per thread; the staged input box reaches FHALO (2 or
// 3) nodes beyond it in y and XOFF (>= 4, one 16-byte TMA granule) in x.  Two
// rows are enough for the pull stencil of the one-node ring's fluid nodes and
// of the tile's wall partners (a wall node on the ring needs no pull: its
// velocity after the extrapolation of Eq. 94 is the wall's); a third row
// makes the boxes of vertically adjacent tiles overlap by six rows, which
// measured faster on grids larger than the L2.
// The temperature box reaches THALO rows beyond the tile (1 for central face
// values, 2 for QUICK's far upstream node) and 4 columns.
// Once a tile's moments are taken, its staged populations are dead and the
// same bytes receive the tile's results, which one TMA bulk store writes back.
//
// RING_THREADS > 0 adds that many threads (whole warps) to the block for the
// one-node ring's moments, and the first of them issues the TMA copies, so
// the THREADS compute threads all carry the same load into each tile's block
// barrier; with 0 the first compute threads also take the ring and thread 0
// issues.
template <class S, int TW_, int TH_, int STAGES_, int THREADS_, int MINB_ = 1, int THALO_ = 1, int RT_ = 0,
          int FHALO_ = 2>
struct TmaTile {
    using TC = typename Compute<S>::type;  // temperature and ring element
    static constexpr int TW = TW_, TH = TH_, STAGES = STAGES_, THREADS = THREADS_;
    static constexpr int RING_THREADS = RT_;
    static constexpr int BLOCK = THREADS_ + RT_;       // threads per block
    static constexpr int MINB = MINB_;             // blocks per SM the register budget must allow
    static constexpr int THALO = THALO_;
    static constexpr int NPT = TW * TH / THREADS;  // own nodes per thread
    static constexpr int XOFF = 16 / (int)sizeof(S) < 4 ? 4 : 16 / (int)sizeof(S);
    static constexpr int FHALO = FHALO_;
    static constexpr int FW = TW + 2 * XOFF, FH = TH + 2 * FHALO;  // population box
    static constexpr int TWD = TW + 8, THT = TH + 2 * THALO;  // temperature box (x0-4, y0-THALO)
    static constexpr int CWD = TW + 32, CHT = TH + 2;      // code box (x0-16, y0-1), codes then face flags
    static constexpr int RW = TW + 2, RH = TH + 2;         // tile + ring
    static constexpr int NRING = 2 * RW + 2 * TH;          // ring nodes
    static constexpr uint32_t F_BYTES = 9u * FH * FW * sizeof(S);
    static constexpr uint32_t T_BYTES = (uint32_t)THT * TWD * (uint32_t)sizeof(TC);
    static constexpr uint32_t C_PLANE = (uint32_t)CHT * CWD;
    static constexpr uint32_t C_BYTES = 2u * C_PLANE;
    static constexpr uint32_t align128(uint32_t v) { return (v + 127u) & ~127u; }
    static constexpr uint32_t F_OFF = 0, T_OFF = align128(F_BYTES), C_OFF = T_OFF + align128(T_BYTES);
    static constexpr uint32_t STAGE_BYTES = C_OFF + align128(C_BYTES);
    static constexpr uint32_t TX_BYTES = F_BYTES + T_BYTES + C_BYTES;
    // results, inside the stage's population bytes: [9][TH][TW] then [TH][TW]
    static constexpr uint32_t OF_BYTES = 9u * TH * TW * sizeof(S);
    static constexpr uint32_t OT_OFF = align128(OF_BYTES);
    static constexpr uint32_t OT_BYTES = (uint32_t)TH * TW * (uint32_t)sizeof(TC);
    static constexpr uint32_t RING_OFF = STAGES * STAGE_BYTES;
    static constexpr uint32_t RING_BYTES = align128(2u * RH * RW * (uint32_t)sizeof(TC));  // u, v of tile + ring
    static constexpr uint32_t BAR_OFF = RING_OFF + 2u * RING_BYTES;      // two ring buffers
    static constexpr uint32_t HDR_OFF = BAR_OFF + align128(8u * STAGES + 16u);
    static constexpr uint32_t SMEM_BYTES = HDR_OFF + STAGES * (uint32_t)sizeof(TileHeader);
    static_assert(SMEM_BYTES <= 232448u, "tile configuration exceeds 227 KB of shared memory");
    static_assert(OT_OFF + OT_BYTES <= F_BYTES, "results must fit in the staged population bytes");
    static_assert((FW * sizeof(S)) % 16 == 0 && (TWD * sizeof(TC)) % 16 == 0 && CWD % 16 == 0 &&
                      (TW * sizeof(S)) % 16 == 0 && (TW * sizeof(TC)) % 16 == 0,
                  "TMA boxes need 16-byte inner extents");
    static_assert(TW % 16 == 0, "tile origins must stay 16-byte aligned for every box");
    static_assert(TW >= 32 && TH >= 8, "tile lists are sized for tiles of at least 32 x 8 nodes");
    static_assert(NPT >= 1 && NPT * THREADS == TW * TH && (RT_ > 0 || NRING <= THREADS), "thread mapping");
    static_assert(RT_ % 32 == 0 && THREADS % 32 == 0, "whole warps");
    static_assert(STAGES >= 2, "the pipeline needs two stages");
    static_assert(THALO == 1 || THALO == 2, "temperature halo of one or two rows");
    static_assert(FHALO == 2 || FHALO == 3, "population halo of two or three rows");
    // the same tile with a temperature box of h halo rows
    template <int h>
    using WithTHalo = TmaTile<S, TW_, TH_, STAGES_, THREADS_, MINB_, h, RT_, FHALO_>;
};

// Energy update of a launch of the TMA kernel: the central face values of
// the fused step, QUICK face values in the fused step, or none (the
// temperature of the new step comes from a plane that the finite-volume
// sub-step kernels wrote, and the kernel only collides with it).
enum : int { FV_CENTRAL = 0, FV_QUICK = 1, FV_GIVEN = 2 };

// Tile shapes of the TMA kernel (tile width x height, pipeline stages,
// threads), selected by lbmfvm_opts_t.tma_config.  Stages are as many as the
// 227 KB of shared memory allow for 32-bit storage; 16-bit storage halves the
// population box and takes one more stage where it fits.
template <class S, int CFG> struct TmaConfig;
template <class S> struct TmaConfig<S, 0> { using G = TmaTile<S, 64, 16, 3, 1024, 1, 1, 0, 3>; };
template <class S> struct TmaConfig<S, 1> { using G = TmaTile<S, 64, 16, 3, 512, 1, 1, 0, 3>; };
template <class S> struct TmaConfig<S, 2> { using G = TmaTile<S, 64, 8, sizeof(S) == 4 ? 2 : 3, 512, 2, 1, 0, 3>; };
template <class S> struct TmaConfig<S, 3> { using G = TmaTile<S, 128, 8, sizeof(S) == 4 ? 2 : 3, 1024, 1, 1, 0, 3>; };
// 64 x 16 with four ring warps (which also issue the copies): two halo rows
// (the faster on grids inside the L2), three rows (the faster beyond it)
template <class S> struct TmaConfig<S, 4> { using G = TmaTile<S, 64, 16, 3, 512, 1, 1, 128, 2>; };
template <class S> struct TmaConfig<S, 5> { using G = TmaTile<S, 64, 16, 3, 512, 1, 1, 128, 3>; };
// 64-bit storage: a 32 x 8 tile stages 43 KB, a 64 x 8 tile 78 KB.
template <> struct TmaConfig<double, 0> { using G = TmaTile<double, 64, 8, 2, 256>; };
template <> struct TmaConfig<double, 1> { using G = TmaTile<double, 32, 8, 3, 256>; };
template <> struct TmaConfig<double, 2> { using G = TmaTile<double, 32, 16, 2, 512>; };
template <> struct TmaConfig<double, 3> { using G = TmaTile<double, 32, 8, 2, 256, 2>; };
template <> struct TmaConfig<double, 4> { using G = TmaTile<double, 32, 8, 3, 256, 1, 1, 64>; };
template <> struct TmaConfig<double, 5> { using G = TmaTile<double, 32, 8, 3, 256, 1, 1, 64, 3>; };
// double-single storage: 8-byte elements like FP64, the same shapes
template <> struct TmaConfig<dsf, 0> { using G = TmaTile<dsf, 64, 8, 2, 256>; };
template <> struct TmaConfig<dsf, 1> { using G = TmaTile<dsf, 32, 8, 3, 256>; };
template <> struct TmaConfig<dsf, 2> { using G = TmaTile<dsf, 32, 16, 2, 512>; };
template <> struct TmaConfig<dsf, 3> { using G = TmaTile<dsf, 32, 8, 2, 256, 2>; };
template <> struct TmaConfig<dsf, 4> { using G = TmaTile<dsf, 32, 8, 3, 256, 1, 1, 64>; };
template <> struct TmaConfig<dsf, 5> { using G = TmaTile<dsf, 32, 8, 3, 256, 1, 1, 64, 3>; };
constexpr int kTmaConfigs = 6;
// QUICK face values and the sub-step path use shape 1 (FV_QUICK with a
// temperature box of two halo rows).
constexpr int kTmaConfigFv = 1;

constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s per wait
constexpr int kErrTimeout = 1;

namespace tma {
__device__ __forceinline__ void store_3d(const CUtensorMap *map, const void *src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_addr(src)), "r"(x), "r"(y), "r"(z)
                 : "memory");
}
__device__ __forceinline__ void store_2d(const CUtensorMap *map, const void *src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_addr(src)), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until the committed bulk stores have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Wait until the committed bulk stores are complete.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
}  // namespace tma

// Persistent fused step for walled domains (no periodic sides).  A block's
// first nfix >= STAGES + 1 tiles are fixed (tile blockIdx.x + k gridDim.x);
// the rest come one at a time from a counter in global memory, so that
// blocks on faster SMs take more of them and the grid ends together.  The
// issuing thread runs two tiles ahead of its loads: a ticket taken at one
// refill is turned into a tile index (and its origin read) at the next and
// loaded at the one after, so that neither the atomic nor the list read
// stalls it.  A tile's
// existence is settled, and published in shared memory, before the barrier
// that precedes its iteration.  Each launch uses one of two counters by step
// parity and clears the other one for the next step (which starts after this
// grid has finished).  Tile k of a block runs
//   wait    every thread waits (bounded) for stage k % STAGES to land;
//   phase A moments of the own nodes (kept in registers) and of the ring
//           (u, v to ring buffer k % 2);
//   barrier the only block-wide one per tile;
//   store   thread 0 hands tile k-1's results to a TMA bulk store;
//   phase B energy balance and collision of the own nodes, results into the
//           stage's population bytes;
//   refill  thread 0, once the store of tile k-1 has read its stage, loads
//           tile k-1+STAGES into it.
// A wait that runs out raises a shared abort flag that every thread checks
// after the barrier, so the block leaves together and a device status word
// tells the host.
template <class S, class G, int MODE = FV_CENTRAL>
__global__ void __launch_bounds__(G::BLOCK, G::MINB)
    step_tma_kernel(const StepArgs<S> a, const CavityDesc *__restrict__ cavs, const TileHeader *__restrict__ tiles,
                    const int *__restrict__ ntiles_p, const __grid_constant__ CUtensorMap map_f,
                    const __grid_constant__ CUtensorMap map_T, const __grid_constant__ CUtensorMap map_c,
                    const __grid_constant__ CUtensorMap map_f_out, const __grid_constant__ CUtensorMap map_T_out,
                    int *__restrict__ ctr, int *__restrict__ ctr_next, const int nfix) {
    using C = typename Compute<S>::type;
    constexpr int TW = G::TW, TH = G::TH, FW = G::FW, FH = G::FH, RW = G::RW, NPT = G::NPT;
    constexpr int XOFF = G::XOFF;
    constexpr int OPLANE = TH * TW;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + G::BAR_OFF);
    int *abort_flag = reinterpret_cast<int *>(smem + G::BAR_OFF + 8 * G::STAGES);
    volatile int *known = abort_flag + 1;  // tiles this block is known to have
    TileHeader *hdrs = reinterpret_cast<TileHeader *>(smem + G::HDR_OFF);

    const int tid = threadIdx.x;
    const int ntiles = *ntiles_p;
    // compute threads hold NPT own nodes; with ring threads, the first of
    // them issues the copies (PROD), else thread 0 does
    constexpr int RT = G::RING_THREADS;
    const bool computes = RT == 0 || tid < G::THREADS;
    const int PROD = RT ? G::THREADS : 0;
    auto fixed_tile = [&](int k) {
        const int t = (int)blockIdx.x + k * (int)gridDim.x;
        return t < ntiles ? t : -1;
    };
    auto stage = [&](int k) { return smem + (k % G::STAGES) * G::STAGE_BYTES; };
    auto origin = [&](int t) { return make_int2(tiles[t].x0, tiles[t].y0); };
    // A tile origin off the 16-node grid would give a TMA box an unaligned
    // x coordinate; such a tile is never loaded (its wait then runs out and
    // the block leaves through the abort path with the status word set).
    auto tile_ok = [&](int x0, int y0) { return (x0 & 15) == 0 && x0 >= 0 && y0 >= 0; };
    auto issue = [&](int k, int t, int2 o) {
        const int s = k % G::STAGES;
        const int x0 = o.x, y0 = o.y;
        if (!tile_ok(x0, y0)) {
            atomicOr(a.err, kErrTimeout);
            return;
        }
        unsigned char *stg = stage(k);
        tma::mbar_arrive_expect_tx(&bars[s], G::TX_BYTES + (uint32_t)sizeof(TileHeader));
        tma::load_bytes(&hdrs[s], tiles + t, sizeof(TileHeader), &bars[s]);
        tma::load_3d(stg + G::F_OFF, &map_f, &bars[s], x0 - XOFF, y0 - G::FHALO, 0);
        tma::load_2d(stg + G::T_OFF, &map_T, &bars[s], x0 - 4, y0 - G::THALO);
        tma::load_3d(stg + G::C_OFF, &map_c, &bars[s], x0 - 16, y0 - 1, 0);
    };
    auto store_tile = [&](int k) {
        const int x0 = hdrs[k % G::STAGES].x0, y0 = hdrs[k % G::STAGES].y0;
        if (!tile_ok(x0, y0)) return;
        unsigned char *stg = stage(k);
        tma::fence_proxy_async();
        tma::store_3d(&map_f_out, stg + G::F_OFF, x0, y0, 0);
        tma::store_2d(&map_T_out, stg + G::F_OFF + G::OT_OFF, x0, y0);
        tma::bulk_commit();
    };

    if (tid == 0) {
        for (int s = 0; s < G::STAGES; s++) tma::mbar_init(&bars[s], 1);
        *abort_flag = 0;
        *known = 0;
        tma::fence_mbar_init();
    }
    __syncthreads();
    // Programmatic dependent launch: the next step's blocks may be scheduled
    // as soon as every block of this one has started (they take the SMs this
    // grid frees); a block's global reads and writes of the state wait until
    // the previous step's grid has finished and its stores are visible.
    // Without a programmatic predecessor the wait returns at once.
    if (tid == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // the issuing thread: the next tile to load (index, origin), the ticket
    // in flight, loads issued
    int pre_t = -1, ticket = -1, issued = 0;
    int2 pre_o = make_int2(0, 0);
    if (tid == PROD) {
        if (blockIdx.x == 0) *ctr_next = 0;
        int k = 0;
        for (; k < G::STAGES && fixed_tile(k) >= 0; k++) {
            if (!(a.stall && blockIdx.x == 0 && k == 0)) issue(k, fixed_tile(k), origin(fixed_tile(k)));
            issued = k + 1;
        }
        if (k == G::STAGES) {
            pre_t = fixed_tile(G::STAGES);
            if (pre_t >= 0) {
                k++;
                pre_o = origin(pre_t);
                if (G::STAGES + 1 >= nfix) ticket = atomicAdd(ctr, 1);
            }
        }
        *known = k;
    }
    __syncthreads();

    for (int k = 0; k < *known; k++) {
        unsigned char *stg = stage(k);
        const bool landed = tma::mbar_wait_bounded(&bars[k % G::STAGES], (uint32_t)(k / G::STAGES) & 1u, kWaitLimitNs);
        if (!landed) {
            atomicOr(abort_flag, 1);
            atomicOr(a.err, kErrTimeout);
        }
        // a stage that never landed has no header: use a harmless one (the
        // block leaves at the next barrier)
        const TileHeader hd = landed ? hdrs[k % G::STAGES] : TileHeader{};
        // node (lx, ly) of the tile sits at (ox + lx, oy + ly) of its cavity
        const int ox = hd.ox, oy = hd.oy, cv_nx = hd.nx;
        const CavityDesc *cvp = cavs + hd.cav;
        C alpha, omega, gbeta, t_ref, fx, fy;
        if constexpr (std::is_same<C, double>::value) {
            alpha = hd.alpha, omega = hd.omega, gbeta = hd.gbeta, t_ref = hd.t_ref, fx = hd.fx, fy = hd.fy;
        } else if constexpr (std::is_same<C, dsf>::value) {
            alpha = dsf(hd.alpha_f, hd.alpha_lo), omega = dsf(hd.omega_f, hd.omega_lo);
            gbeta = dsf(hd.gbeta_f, hd.gbeta_lo), t_ref = dsf(hd.t_ref_f, hd.t_ref_lo);
            fx = dsf(hd.fx_f, hd.fx_lo), fy = dsf(hd.fy_f, hd.fy_lo);
        } else {
            alpha = hd.alpha_f, omega = hd.omega_f, gbeta = hd.gbeta_f, t_ref = hd.t_ref_f, fx = hd.fx_f,
            fy = hd.fy_f;
        }
        const S *F = reinterpret_cast<const S *>(stg + G::F_OFF);
        const C *TT = reinterpret_cast<const C *>(stg + G::T_OFF);
        const uint8_t *CC = reinterpret_cast<const uint8_t *>(stg + G::C_OFF);
        const uint8_t *CF = CC + G::C_PLANE;  // face flags
        C *RU = reinterpret_cast<C *>(smem + G::RING_OFF + (k & 1) * G::RING_BYTES), *RV = RU + G::RH * RW;
        // staged-box index of node (lx, ly) relative to the tile origin
        auto fidx = [&](int lx, int ly) { return (ly + G::FHALO) * FW + (lx + XOFF); };
        auto tidx = [&](int lx, int ly) { return (ly + G::THALO) * G::TWD + (lx + 4); };
        auto cidx = [&](int lx, int ly) { return (ly + 1) * G::CWD + (lx + 16); };
        auto pull = [&](int lx, int ly, C g[9]) {
            const S *p = F + fidx(lx, ly);
#pragma unroll
            for (int q = 0; q < 9; q++) g[q] = ld(p + q * (FH * FW) - cy(q) * FW - cx(q));
        };
        // velocity of wall node (lx, ly): 0 on obstacle surfaces, the side's
        // on box walls (vertical sides own the corners)
        auto wall_vel = [&](int lx, int ly, uint8_t c, C &uw, C &vw) {
            uw = vw = C(0);
            if ((c >> 6) != TH_OBSTACLE) {
                const int cx = ox + lx, cy = oy + ly;
                const int side = cx == 0 ? 0 : (cx == cv_nx - 1 ? 1 : (cy == 0 ? 2 : 3));
                if constexpr (std::is_same<C, double>::value || std::is_same<C, dsf>::value) {
                    uw = C(cvp->wall_u[side]);
                    vw = C(cvp->wall_v[side]);
                } else {
                    uw = cvp->wall_uf[side];
                    vw = cvp->wall_vf[side];
                }
            }
        };
        auto state = [&](int lx, int ly, uint8_t c, C g[9], C &drho, C &ux, C &uy) {
            const int kind = c & 3;
            if (kind == KIND_FLUID) {
                pull(lx, ly, g);
                moments<C>(g, drho, ux, uy);
            } else if (kind == KIND_WALL) {
                const int d = partner_dir(c);
                pull(lx + cx_rt(d), ly + cy_rt(d), g);
                moments<C>(g, drho, ux, uy);
                C uw, vw;
                wall_vel(lx, ly, c, uw, vw);
                nee<C>(g, drho, ux, uy, uw, vw);
            } else {
#pragma unroll
                for (int q = 0; q < 9; q++) g[q] = C(0);
                drho = C(-1);
                ux = uy = C(0);
            }
        };

        // Phase A: own nodes into registers (their u, v also to the ring
        // buffer), the ring's u, v.
        C g[NPT][9], dr[NPT], uu[NPT], vv[NPT];
        uint8_t cc[NPT];
        if (computes) {
#pragma unroll
            for (int j = 0; j < NPT; j++) {
                const int i = tid + j * G::THREADS;
                const int ly = i / TW, lx = i - ly * TW;
                cc[j] = decode(CC[cidx(lx, ly)]);
                state(lx, ly, cc[j], g[j], dr[j], uu[j], vv[j]);
                if constexpr (MODE != FV_GIVEN) {
                    const int r = (ly + 1) * RW + (lx + 1);
                    RU[r] = uu[j];
                    RV[r] = vv[j];
                }
            }
        }
        // the ring's velocities feed the energy update's faces only
        if (MODE != FV_GIVEN) {
            const int first = RT ? tid - G::THREADS : tid, stride = RT ? RT : G::NRING;
            for (int hr = first; hr >= 0 && hr < G::NRING; hr += stride) {
                int rx, ry;
                if (hr < RW) { rx = hr; ry = 0; }
                else if (hr < 2 * RW) { rx = hr - RW; ry = TH + 1; }
                else { const int h = hr - 2 * RW; rx = (h & 1) ? RW - 1 : 0; ry = 1 + (h >> 1); }
                const uint8_t c = decode(CC[cidx(rx - 1, ry - 1)]);
                C hu = C(0), hv = C(0);
                if ((c & 3) == KIND_FLUID) {
                    C hg[9], hd;
                    state(rx - 1, ry - 1, c, hg, hd, hu, hv);
                } else if ((c & 3) == KIND_WALL) {
                    // the extrapolated wall node moves with the wall (Eq. 94)
                    wall_vel(rx - 1, ry - 1, c, hu, hv);
                }
                RU[ry * RW + rx] = hu;
                RV[ry * RW + rx] = hv;
            }
        }
        __syncthreads();
        if (*abort_flag) {
            if (tid == PROD) {
                // let the copies already in flight land before the block exits
                for (int j = k + 1; j < issued; j++)
                    tma::mbar_wait_bounded(&bars[j % G::STAGES], (uint32_t)(j / G::STAGES) & 1u, kWaitLimitNs / 2);
                tma::bulk_wait_all();
            }
            return;
        }
        if (tid == PROD && k > 0) store_tile(k - 1);

        // Phase B: energy balance and collision of the own nodes; results go
        // to the stage's (now dead) population bytes.  Inert nodes keep T.
        S *OF = reinterpret_cast<S *>(stg + G::F_OFF);
        C *OT = reinterpret_cast<C *>(stg + G::F_OFF + G::OT_OFF);
#pragma unroll
        for (int j = 0; j < NPT; j++) {
            if (!computes) break;
            const int i = tid + j * G::THREADS;
            const int ly = i / TW, lx = i - ly * TW;
            const uint8_t c = cc[j];
            const int t = tidx(lx, ly);
            const C TP = TT[t];
            S *of = OF + ly * TW + lx;
            if ((c & 3) == KIND_SOLID) {
                OT[ly * TW + lx] = TP;
#pragma unroll
                for (int q = 0; q < 9; q++) st(of + q * OPLANE, C(0));
                continue;
            }
            const int r = (ly + 1) * RW + (lx + 1);
            const int th = c >> 6;
            C Tn = TP;
            if (MODE == FV_GIVEN) {
                // T^{n+1} of every node comes from the sub-step kernels
            } else if (th == TH_FV) {
                // control volume clipped to the cavity; faces beyond it are closed
                const uint8_t ff = CF[cidx(lx, ly)];
                const C ex = ((ff & FF_IN_W) ? C(0.5) : C(0)) + ((ff & FF_IN_E) ? C(0.5) : C(0));
                const C ey = ((ff & FF_IN_S) ? C(0.5) : C(0)) + ((ff & FF_IN_N) ? C(0.5) : C(0));
                if constexpr (MODE == FV_QUICK) {
                    // far upstream nodes: beyond P (P's own flags) or beyond
                    // the neighbour (the neighbour's flag on the same side)
                    const int W2 = G::TWD;
                    const C uP = uu[j], vP = vv[j], TP_ = TP;
                    const C TE = TT[t + 1], TW = TT[t - 1], TN = TT[t + W2], TS = TT[t - W2];
                    const C uE = RU[r + 1], uW = RU[r - 1], vN = RV[r + RW], vS = RV[r - RW];
                    const C TfE = quick_face<C>(uP + uE, TP_, TE, ff & FF_OPEN_W, TW,
                                                CF[cidx(lx + 1, ly)] & FF_OPEN_E, TT[t + 2]);
                    const C TfW = quick_face<C>(-(uP + uW), TP_, TW, ff & FF_OPEN_E, TE,
                                                CF[cidx(lx - 1, ly)] & FF_OPEN_W, TT[t - 2]);
                    const C TfN = quick_face<C>(vP + vN, TP_, TN, ff & FF_OPEN_S, TS,
                                                CF[cidx(lx, ly + 1)] & FF_OPEN_N, TT[t + 2 * W2]);
                    const C TfS = quick_face<C>(-(vP + vS), TP_, TS, ff & FF_OPEN_N, TN,
                                                CF[cidx(lx, ly - 1)] & FF_OPEN_S, TT[t - 2 * W2]);
                    Tn = fv_update_faces<C>(TP_, uP, vP, ex, ey, alpha, C(1), ff & FF_OPEN_E, TE, uE, TfE,
                                            ff & FF_OPEN_N, TN, vN, TfN, ff & FF_OPEN_W, TW, uW, TfW, ff & FF_OPEN_S,
                                            TS, vS, TfS);
                } else {
                    Tn = fv_update<C>(TP, uu[j], vv[j], ex, ey, alpha, ff & FF_OPEN_E, TT[t + 1], RU[r + 1],
                                      ff & FF_OPEN_N, TT[t + G::TWD], RV[r + RW], ff & FF_OPEN_W, TT[t - 1], RU[r - 1],
                                      ff & FF_OPEN_S, TT[t - G::TWD], RV[r - RW]);
                }
            } else if (th == TH_OBSTACLE) {
                const int d = partner_dir(c);
                Tn = TT[tidx(lx + cx_rt(d), ly + cy_rt(d))];
            }
            OT[ly * TW + lx] = Tn;
            const C Gy = fy + gbeta * (Tn - t_ref);
            collide<C>(g[j], dr[j], uu[j], vv[j], omega, fx, Gy, [&](int q, C v) { st(of + q * OPLANE, v); });
        }
        if (tid == PROD && k > 0 && pre_t >= 0) {
            tma::bulk_wait_read();  // the results of tile k-1 have left its stage
            issue(k - 1 + G::STAGES, pre_t, pre_o);
            issued = k + G::STAGES;
            // tile k + STAGES of this block: fixed, or named by the ticket
            // taken at the previous refill
            const int m = k + G::STAGES;
            if (m < nfix) {
                pre_t = fixed_tile(m);
            } else {
                const int t = nfix * (int)gridDim.x + ticket;
                pre_t = ticket >= 0 && t < ntiles ? t : -1;
            }
            if (pre_t >= 0) {
                pre_o = origin(pre_t);
                *known = *known + 1;
                if (m + 1 >= nfix) ticket = atomicAdd(ctr, 1);
            }
        }
    }
    const int count = *known;
    __syncthreads();
    if (tid == PROD && count > 0) {
        store_tile(count - 1);
        tma::bulk_wait_all();
    }
}

// ---------------------------------------------------------------------------
// Energy update in sub-steps (and QUICK face values beside them).  With m
// explicit sub-steps of dt = 1/m per lattice step, each sub-step reads the
// previous one's temperature of the neighbours, so the update leaves the
// fused kernel: per lattice step
//   uv_kernel            u^{n+1}, v^{n+1} of every node of the active tiles
//                        (pull, wall extrapolation, moments) into two planes;
//   fv_substep_kernel    M launches (M = the largest m of the list's
//                        cavities): T_s = T_{s-1} + dt (flux balance) with the
//                        velocity held at u^{n+1}; launch s takes the tiles of
//                        the cavities with m >= s (the list is sorted by m,
//                        largest first), and each cavity's chain of sub-steps
//                        alternates between two scratch planes so that its
//                        last one lands in the plane X;
//   step_tma_kernel      FV_GIVEN: pull, extrapolation, moments, and the
//                        collision with the final sub-step's T^{n+1}.
// Both helper kernels take one tile of the TMA kernel's list per block and
// read global memory directly (their planes are small next to the
// populations and stay in L2).
// ---------------------------------------------------------------------------

// Tile parameters of the helper kernels in the arithmetic precision C.
template <class C> struct TileParams;
template <> struct TileParams<float> {
    __device__ static float alpha(const TileHeader &h) { return h.alpha_f; }
    __device__ static float dt(const TileHeader &h) { return h.dt_f; }
};
template <> struct TileParams<double> {
    __device__ static double alpha(const TileHeader &h) { return h.alpha; }
    __device__ static double dt(const TileHeader &h) { return 1.0 / (double)h.substeps; }
};
template <> struct TileParams<dsf> {
    __device__ static dsf alpha(const TileHeader &h) { return dsf(h.alpha_f, h.alpha_lo); }
    __device__ static dsf dt(const TileHeader &h) { return dsf(h.dt_f, h.dt_lo); }
};

// u^{n+1}, v^{n+1} of every node of the active tiles (tile shape tw x th):
// the same pull, extrapolation and moments as phase A of the step kernel.
// Nodes outside every cavity and inert nodes get 0.
template <class S>
__global__ void __launch_bounds__(256)
    uv_kernel(const S *__restrict__ fin, long long plane, int pitch, int gnx, int gny,
              const TileHeader *__restrict__ tiles, int ntiles, const CavityDesc *__restrict__ cavs,
              const uint8_t *__restrict__ code, typename Compute<S>::type *U, typename Compute<S>::type *V, int tw,
              int th) {
    using C = typename Compute<S>::type;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int x0 = tiles[t].x0, y0 = tiles[t].y0, ox = tiles[t].ox, oy = tiles[t].oy, cnx = tiles[t].nx;
        const CavityDesc *cvp = cavs + tiles[t].cav;
        for (int i = threadIdx.x; i < tw * th; i += blockDim.x) {
            const int ly = i / tw, lx = i - ly * tw;
            const int x = x0 + lx, y = y0 + ly;
            if (x >= gnx || y >= gny) continue;
            const long long k = (long long)y * pitch + x;
            const uint8_t c = decode(code[k]);
            const int kind = c & 3;
            C g[9], drho = C(-1), ux = C(0), uy = C(0);
            if (kind != KIND_SOLID) {
                int sx = x, sy = y;
                if (kind == KIND_WALL) {
                    const int d = partner_dir(c);
                    sx += cx_rt(d);
                    sy += cy_rt(d);
                }
                // a fluid node and a wall partner lie inside their cavity, so
                // the pull stays on the grid; the clamp only guards the reads
                // against a corrupt code
                sx = min(max(sx, 1), gnx - 2);
                sy = min(max(sy, 1), gny - 2);
                const S *p = fin + (long long)sy * pitch + sx;
#pragma unroll
                for (int q = 0; q < 9; q++) g[q] = ld(p + q * plane - cy(q) * pitch - cx(q));
                moments<C>(g, drho, ux, uy);
                if (kind == KIND_WALL) {
                    C uw = C(0), vw = C(0);
                    if ((c >> 6) != TH_OBSTACLE) {
                        const int px = ox + lx, py = oy + ly;
                        const int side = px == 0 ? 0 : (px == cnx - 1 ? 1 : (py == 0 ? 2 : 3));
                        if constexpr (std::is_same<C, float>::value) {
                            uw = cvp->wall_uf[side];
                            vw = cvp->wall_vf[side];
                        } else {
                            uw = C(cvp->wall_u[side]);
                            vw = C(cvp->wall_v[side]);
                        }
                    }
                    nee<C>(g, drho, ux, uy, uw, vw);
                }
            }
            U[k] = ux;
            V[k] = uy;
        }
    }
}

// Sub-step s (1-based) of the energy update on the first ntiles tiles of a
// list (cavities with m >= s sub-steps): the new temperature from the
// previous sub-step's with the velocity planes U, V held (finite-volume
// nodes), the partner's temperature (obstacle surface nodes), unchanged
// otherwise.  A cavity's sub-step s reads T0 (s = 1) or the plane its
// sub-step s - 1 wrote, and writes X when m - s is even, else Y, so its last
// sub-step writes X.
template <class C, bool QUICK>
__global__ void __launch_bounds__(256)
    fv_substep_kernel(const C *__restrict__ T0, C *X, C *Y, const C *__restrict__ U, const C *__restrict__ V,
                      const uint8_t *__restrict__ code, const uint8_t *__restrict__ fflags, int pitch, int gnx, int gny,
                      const TileHeader *__restrict__ tiles, int ntiles, int tw, int th, int s) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileHeader &hd = tiles[t];
        const int x0 = hd.x0, y0 = hd.y0;
        const bool to_x = ((hd.substeps - s) & 1) == 0;
        C *Tout = to_x ? X : Y;
        const C *Tin = s == 1 ? T0 : (to_x ? Y : X);
        if (s > hd.substeps) continue;  // not in this sub-step (the host passes none)
        const C alpha = TileParams<C>::alpha(hd), dt = TileParams<C>::dt(hd);
        for (int i = threadIdx.x; i < tw * th; i += blockDim.x) {
            const int ly = i / tw, lx = i - ly * tw;
            const int x = x0 + lx, y = y0 + ly;
            if (x >= gnx || y >= gny) continue;
            const long long k = (long long)y * pitch + x;
            const C TP = Tin[k];
            const uint8_t c = decode(code[k]);
            const int role = c >> 6;
            C Tn = TP;
            if (role == TH_OBSTACLE && (c & 3) == KIND_WALL) {
                const int d = partner_dir(c);
                Tn = Tin[k + (long long)cy_rt(d) * pitch + cx_rt(d)];
            } else if (role == TH_FV) {
                // open faces name neighbours inside the cavity, and a far
                // node's flag is read only from a node inside it
                const uint8_t ff = fflags[k];
                const bool oE = ff & FF_OPEN_E, oW = ff & FF_OPEN_W, oN = ff & FF_OPEN_N, oS = ff & FF_OPEN_S;
                const C ex = ((ff & FF_IN_W) ? C(0.5) : C(0)) + ((ff & FF_IN_E) ? C(0.5) : C(0));
                const C ey = ((ff & FF_IN_S) ? C(0.5) : C(0)) + ((ff & FF_IN_N) ? C(0.5) : C(0));
                const C uP = U[k], vP = V[k];
                const C TE = oE ? Tin[k + 1] : C(0), TW = oW ? Tin[k - 1] : C(0);
                const C TN = oN ? Tin[k + pitch] : C(0), TS = oS ? Tin[k - pitch] : C(0);
                const C uE = oE ? U[k + 1] : C(0), uW = oW ? U[k - 1] : C(0);
                const C vN = oN ? V[k + pitch] : C(0), vS = oS ? V[k - pitch] : C(0);
                C TfE, TfW, TfN, TfS;
                if constexpr (QUICK) {
                    const bool eE = oE && (fflags[k + 1] & FF_OPEN_E), wW = oW && (fflags[k - 1] & FF_OPEN_W);
                    const bool nN = oN && (fflags[k + pitch] & FF_OPEN_N), sS = oS && (fflags[k - pitch] & FF_OPEN_S);
                    TfE = quick_face<C>(uP + uE, TP, TE, oW, TW, eE, eE ? Tin[k + 2] : C(0));
                    TfW = quick_face<C>(-(uP + uW), TP, TW, oE, TE, wW, wW ? Tin[k - 2] : C(0));
                    TfN = quick_face<C>(vP + vN, TP, TN, oS, TS, nN, nN ? Tin[k + 2 * (long long)pitch] : C(0));
                    TfS = quick_face<C>(-(vP + vS), TP, TS, oN, TN, sS, sS ? Tin[k - 2 * (long long)pitch] : C(0));
                } else {
                    TfE = C(0.5) * (TP + TE);
                    TfW = C(0.5) * (TP + TW);
                    TfN = C(0.5) * (TP + TN);
                    TfS = C(0.5) * (TP + TS);
                }
                Tn = fv_update_faces<C>(TP, uP, vP, ex, ey, alpha, dt, oE, TE, uE, TfE, oN, TN, vN, TfN, oW, TW, uW,
                                        TfW, oS, TS, vS, TfS);
            }
            Tout[k] = Tn;
        }
    }
}

// ---------------------------------------------------------------------------
// D2Q5 thermal lattice Boltzmann energy solver (Section 2.4), the paper's
// pure-LBM comparison: energy populations g_i (rest, E, N, W, S: the first
// five D2Q9 directions) relax toward g_eq = T w_i (1 + 3 e_i.u) (Eqs. 19, 21;
// w = 1/3, 1/6 of Eq. 22) with omega_T = 1/tau_T, tau_T = 3 alpha + 1/2
// (Eq. 20), stream like f and give T = sum g (Eq. 23).  Wall nodes take
// g_b = g_eq(T_b, u_b) + g(x_f) - g_eq(T_f, u_f) (Eq. 95) with T_b the wall
// temperature on Dirichlet sides (held in the temperature plane) and T_f on
// adiabatic sides and obstacle surfaces.  State between launches: the
// post-collision f* and g*; the temperature plane receives T of the new step
// for the field, residual and Nusselt kernels.  One node per thread, pulls
// from global memory (every neighbour lies one node away); no halo exchange
// is needed because the energy update is local.
// ---------------------------------------------------------------------------

// Eq. 22: 1/3 for the rest population, 1/6 for the axis ones.
template <class C>
__device__ __forceinline__ C w5(int q) {
    return q == 0 ? C(1) / C(3) : C(1) / C(6);
}
template <>
__device__ __forceinline__ dsf w5<dsf>(int q) {
    return q == 0 ? dsf(1.0 / 3.0) : dsf(1.0 / 6.0);
}

// The energy populations are stored shifted, s_i = g_i - w_i T_0, with T_0
// the mean of the two wall temperatures (the way f is stored as f - w), and
// the collision works on the shifted values: near T_0 they are small, so their
// rounding is too.  With dT = T - T_0, the shifted equilibrium (Eq. 21 with
// c_s^2 = 1/3) is
//   g_eq,i - w_i T_0 = w_i dT + 3 w_i T e_i.u,
// and for the axis directions 3 w_i T = T/2 exactly.  The rest direction is
// taken as dT minus the four others' dT/6 parts, so that the shifted
// equilibria sum to dT without the bias of a rounded weight.
template <class C>
__device__ __forceinline__ void geq5_shifted(C T, C dT, C ux, C uy, C e[5]) {
    const C a = dT * w5<C>(1), t = C(0.5) * T;
    e[0] = dT - C(4) * a;
    e[1] = a + t * ux;
    e[3] = a - t * ux;
    e[2] = a + t * uy;
    e[4] = a - t * uy;
}

template <class S>
struct Lbm5Args {
    using C = typename Compute<S>::type;
    StepArgs<S> a;     // populations f, temperature plane, codes, lattice parameters
    const S *gin;      // shifted post-collision g of the previous step [5][ny][pitch]
    S *gout;
    C omega_T;         // 1 / tau_T
    C T0;              // the shift of the stored populations
};

template <class S>
__global__ void __launch_bounds__(256) step_lbm5_kernel(const Lbm5Args<S> p) {
    using C = typename Compute<S>::type;
    const StepArgs<S> &a = p.a;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const long long k = (long long)y * a.pitch + x;
    const uint8_t c = decode(a.code[k]);
    const int kind = c & 3;
    S *fo = a.fout + k;
    S *go = p.gout + k;
    if (kind == KIND_SOLID) {
#pragma unroll
        for (int q = 0; q < 9; q++) st(fo + q * a.plane, C(0));
#pragma unroll
        for (int q = 0; q < 5; q++) st(go + q * a.plane, C(0));
        a.Tout[k] = a.Tin[k];
        return;
    }
    // the node itself (fluid) or its partner (wall) receives the pull
    int sx = x, sy = y;
    if (kind == KIND_WALL) {
        const int d = partner_dir(c);
        sx = x + cx_rt(d);
        sy = y + cy_rt(d);
        sx = sx < 0 ? sx + a.nx : (sx >= a.nx ? sx - a.nx : sx);
        sy = sy < 0 ? sy + a.ny : (sy >= a.ny ? sy - a.ny : sy);
    }
    C g[9], h[5], drho, ux, uy;
    gather<S, C>(a.fin, a.plane, a.pitch, a.nx, a.ny, sx, sy, g);
    {
        const int xm = sx > 0 ? sx - 1 : a.nx - 1, xp = sx < a.nx - 1 ? sx + 1 : 0;
        const int ym = sy > 0 ? sy - 1 : a.ny - 1, yp = sy < a.ny - 1 ? sy + 1 : 0;
        const S *gi = p.gin;
        h[0] = ld(gi + (long long)sy * a.pitch + sx);
        h[1] = ld(gi + a.plane + (long long)sy * a.pitch + xm);
        h[2] = ld(gi + 2 * a.plane + (long long)ym * a.pitch + sx);
        h[3] = ld(gi + 3 * a.plane + (long long)sy * a.pitch + xp);
        h[4] = ld(gi + 4 * a.plane + (long long)yp * a.pitch + sx);
    }
    moments<C>(g, drho, ux, uy);
    C dT = (((h[0] + h[1]) + (h[2] + h[3])) + h[4]);  // Eq. 23 on shifted populations
    if (kind == KIND_WALL) {
        C uw, vw;
        wall_velocity<S>(a, x, y, c, uw, vw);
        const C uf = ux, vf = uy, dTf = dT;
        nee<C>(g, drho, ux, uy, uw, vw);
        // Eq. 95 with T_b the wall temperature (Dirichlet) or T_f
        const C dTb = (c >> 6) == TH_DIRICHLET ? a.Tin[k] - p.T0 : dTf;
        C eb[5], ef[5];
        geq5_shifted<C>(p.T0 + dTb, dTb, uw, vw, eb);
        geq5_shifted<C>(p.T0 + dTf, dTf, uf, vf, ef);
#pragma unroll
        for (int q = 0; q < 5; q++) h[q] = eb[q] + h[q] - ef[q];
        dT = (((h[0] + h[1]) + (h[2] + h[3])) + h[4]);
    }
    const C T = p.T0 + dT;
    a.Tout[k] = T;
    const C Gy = a.fy + a.gbeta * (T - a.t_ref);
    const long long plane = a.plane;
    collide<C>(g, drho, ux, uy, a.omega, a.fx, Gy, [&](int q, C v) { st(fo + q * plane, v); });
    // Eq. 19 on shifted populations: s* = s - (s - (g_eq - w T_0)) / tau_T
    C e[5];
    geq5_shifted<C>(T, dT, ux, uy, e);
#pragma unroll
    for (int q = 0; q < 5; q++) st(go + q * plane, h[q] - p.omega_T * (h[q] - e[q]));
}

// Energy populations of the initial state: g^0 = g_eq(T^0, u^0) (Eq. 21),
// stored shifted by w_i T_0, in both buffers (at equilibrium the collision
// leaves g unchanged); u^0 from the initial populations f0 (stored as f - w).
template <class S>
__global__ void init_lbm5_kernel(const StepArgs<S> a, const S *f0, S *g0, S *g1, typename Compute<S>::type T0) {
    using C = typename Compute<S>::type;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const long long k = (long long)y * a.pitch + x;
    const bool inert = (decode(a.code[k]) & 3) == KIND_SOLID;
    C g[9], drho = C(0), ux = C(0), uy = C(0);
    if (!inert) {
#pragma unroll
        for (int q = 0; q < 9; q++) g[q] = ld(f0 + k + q * a.plane);
        moments<C>(g, drho, ux, uy);
    }
    C e[5];
    const C T = a.Tin[k];
    geq5_shifted<C>(T, T - T0, ux, uy, e);
#pragma unroll
    for (int q = 0; q < 5; q++) {
        const C v = inert ? C(0) : e[q];
        st(g0 + k + q * a.plane, v);
        st(g1 + k + q * a.plane, v);
    }
}

// ---------------------------------------------------------------------------
// Grid setting 2 (Section 5.1, Fig. 30): the energy balance on NX x NY
// control volumes of 2 x 2 lattice spacings whose faces pass through lattice
// nodes (face velocities are lattice velocities, no interpolation; centres at
// the odd-odd nodes), an explicit step of k lattice steps every k-th step,
// node temperatures interpolated from the volumes.  Single walled cavities
// without obstacles: the cavity spans 2 NX x 2 NY spacings.
// ---------------------------------------------------------------------------

struct Grid2Args {
    int nx, ny, pitch, ncx, ncy;  // lattice nodes, node pitch, volumes
    int dirichlet[4];             // W, E, S, N: Dirichlet side (else no heat flux)
    double t_wall[4];
};

// One coarse step: Tn = T + (k / V) sum over faces of [-A u_n (T_P + T_nb)/2
// + alpha A (T_nb - T_P) / d], V = 4, A = 2, d = 2 between volumes, d = 1 to a
// Dirichlet wall face, no flux through other walls; u_n the lattice velocity
// at the face's middle node (the velocity planes U, V).
template <class C>
__global__ void grid2_step_kernel(const Grid2Args g, const C *__restrict__ Tc, C *__restrict__ Tn,
                                  const C *__restrict__ U, const C *__restrict__ V, C alpha, C dt) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= g.ncx || J >= g.ncy) return;
    const C TP = Tc[J * g.ncx + I];
    const long long cn = (long long)(2 * J + 1) * g.pitch + (2 * I + 1);  // centre node
    C acc = C(0);
    auto face = [&](int dx, int dy, int side) {
        const int In = I + dx, Jn = J + dy;
        const long long kf = cn + (long long)dy * g.pitch + dx;
        const C un = dx ? C(dx) * U[kf] : C(dy) * V[kf];
        if (In >= 0 && In < g.ncx && Jn >= 0 && Jn < g.ncy) {
            const C TN = Tc[Jn * g.ncx + In];
            acc = acc + (C(-2) * un * C(0.5) * (TP + TN) + alpha * (TN - TP));
        } else if (g.dirichlet[side]) {
            acc = acc + C(2) * alpha * (C(g.t_wall[side]) - TP);
        }
    };
    face(1, 0, 1);
    face(0, 1, 3);
    face(-1, 0, 0);
    face(0, -1, 2);
    Tn[J * g.ncx + I] = TP + dt * acc * C(0.25);
}

// Node temperatures from the volumes (Section 5.1's interpolation): a
// centre takes its volume's value, a node between two (four) centres their
// mean, a node on a wall without heat flux the nearest volume's value, a
// Dirichlet node its wall value (as held in the temperature plane Tdir).
// Writes the node plane X (and, when given, the two temperature planes of
// the state), and copies the new volume values Tn into Tc at the centre
// nodes.
template <class C>
__global__ void grid2_nodes_kernel(const Grid2Args g, const uint8_t *__restrict__ code, const C *Tdir,
                                   const C *__restrict__ Tn, C *__restrict__ Tc, C *X, C *Ta, C *Tb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    int ia0, ia1, ja0, ja1;
    if (i & 1) ia0 = ia1 = (i - 1) / 2;
    else if (i == 0) ia0 = ia1 = 0;
    else if (i == g.nx - 1) ia0 = ia1 = g.ncx - 1;
    else ia0 = i / 2 - 1, ia1 = i / 2;
    if (j & 1) ja0 = ja1 = (j - 1) / 2;
    else if (j == 0) ja0 = ja1 = 0;
    else if (j == g.ny - 1) ja0 = ja1 = g.ncy - 1;
    else ja0 = j / 2 - 1, ja1 = j / 2;
    C t;
    const long long k = (long long)j * g.pitch + i;
    if ((decode(code[k]) >> 6) == TH_DIRICHLET) {
        t = Tdir[k];  // the wall value the temperature planes hold
    } else if (ia0 == ia1 && ja0 == ja1) {
        t = Tn[ja0 * g.ncx + ia0];
    } else if (ja0 == ja1) {
        t = C(0.5) * (Tn[ja0 * g.ncx + ia0] + Tn[ja0 * g.ncx + ia1]);
    } else if (ia0 == ia1) {
        t = C(0.5) * (Tn[ja0 * g.ncx + ia0] + Tn[ja1 * g.ncx + ia0]);
    } else {
        t = C(0.25) * ((Tn[ja0 * g.ncx + ia0] + Tn[ja0 * g.ncx + ia1]) + (Tn[ja1 * g.ncx + ia0] + Tn[ja1 * g.ncx + ia1]));
    }
    X[k] = t;
    if (Ta) Ta[k] = t;
    if (Tb) Tb[k] = t;
    if ((i & 1) && (j & 1)) Tc[((j - 1) / 2) * g.ncx + (i - 1) / 2] = Tn[((j - 1) / 2) * g.ncx + (i - 1) / 2];
}

// Volume values from the node temperatures at the centres (the initial state).
template <class C>
__global__ void grid2_gather_kernel(const Grid2Args g, const C *__restrict__ T, C *__restrict__ Tn) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= g.ncx || J >= g.ncy) return;
    Tn[J * g.ncx + I] = T[(long long)(2 * J + 1) * g.pitch + 2 * I + 1];
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
    const uint8_t c = decode(a.code[k]);
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
    S *out = fstar_out + k;
    const long long plane = a.plane;
    collide<C>(g, drho, ux, uy, a.omega, a.fx, Gy, [&](int q, C v2) { st(out + q * plane, v2); });
}

// State copy between storage precisions.  Every precision stores f - w_i, so
// converting a state is a value conversion of each stored population and
// temperature; buffer b of the source goes to buffer b ^ flip of the
// destination, which keeps the two ping-pong buffers' roles when the two
// handles are at opposite parities.
template <class S, class D>
__global__ void convert_kernel(const S *fs0, const S *fs1, const typename Compute<S>::type *Ts0,
                               const typename Compute<S>::type *Ts1, int pitch_s, long long plane_s, D *fd0, D *fd1,
                               typename Compute<D>::type *Td0, typename Compute<D>::type *Td1, int pitch_d,
                               long long plane_d, int nx, int ny, int flip) {
    using CD = typename Compute<D>::type;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const int b = blockIdx.z;
    const S *fs = b ? fs1 : fs0;
    const typename Compute<S>::type *Ts = b ? Ts1 : Ts0;
    D *fd = (b ^ flip) ? fd1 : fd0;
    CD *Td = (b ^ flip) ? Td1 : Td0;
    const long long ks = (long long)y * pitch_s + x, kd = (long long)y * pitch_d + x;
#pragma unroll
    for (int q = 0; q < 9; q++) st(fd + kd + q * plane_d, CD(ld(fs + ks + q * plane_s)));
    Td[kd] = CD(Ts[ks]);
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
    const uint8_t c = decode(a.code[k]);
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
// A fixed assignment of rows to blocks and a fixed reduction tree make the
// result independent of scheduling.
// Sums of the residual pass, per block and in total: |u - u_s|^2, |u|^2,
// rho - 1 and the node count, all over the fluid nodes.
constexpr int kResidualSums = 4;

template <class S>
__global__ void __launch_bounds__(256) residual_kernel(const StepArgs<S> a, int direct, double *su,
                                                       double *sv, double *partials, int update_only) {
    using C = typename Compute<S>::type;
    __shared__ double red[kResidualSums][8];
    double num = 0.0, den = 0.0, mass = 0.0, cnt = 0.0;
    for (int y = blockIdx.x; y < a.ny; y += gridDim.x) {
        for (int x = threadIdx.x; x < a.nx; x += blockDim.x) {
            const long long k = (long long)y * a.pitch + x;
            const uint8_t c = decode(a.code[k]);
            if ((c & 3) != KIND_FLUID) continue;
            C drho, ux, uy;
            current_moments<S>(a, direct, x, y, c, drho, ux, uy);
            const long long i = (long long)y * a.nx + x;
            const double du = (double)ux - su[i], dv = (double)uy - sv[i];
            num += du * du + dv * dv;
            den += (double)ux * (double)ux + (double)uy * (double)uy;
            mass += (double)drho;
            cnt += 1.0;
            su[i] = (double)ux;
            sv[i] = (double)uy;
        }
    }
    if (update_only) return;
    double v[kResidualSums] = {num, den, mass, cnt};
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kResidualSums; j++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
        if (lane == 0) red[j][wid] = v[j];
    }
    __syncthreads();
    if (threadIdx.x < kResidualSums) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[threadIdx.x][w];
        partials[kResidualSums * blockIdx.x + threadIdx.x] = t;
    }
}

// Residual, pass 2: one warp sums the block partials in a fixed order.
static __global__ void residual_finish_kernel(const double *partials, int nblocks, double *out) {
    double v[kResidualSums] = {};
    for (int b = threadIdx.x; b < nblocks; b += 32)
#pragma unroll
        for (int j = 0; j < kResidualSums; j++) v[j] += partials[kResidualSums * b + j];
#pragma unroll
    for (int j = 0; j < kResidualSums; j++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int j = 0; j < kResidualSums; j++) out[j] = v[j];
}

// Mass renormalisation.  With the Eq. 18 force and the pressure read as
// rho0 cs^2, one step is homogeneous of degree one in f: f -> c f scales the
// whole trajectory by c and leaves u and T unchanged.  The non-equilibrium
// extrapolation walls (Eqs. 94, 96) do not conserve mass, and once the flow
// settles the mass shrinks by a fixed factor per step; rescaling both
// population buffers so that the fluid nodes average rho = 1 keeps the stored
// f - w_i at the size of the flow's own deviations without changing u or T.
// tot: the totals of residual_kernel (tot[2] = sum of rho - 1, tot[3] = node
// count) for this state.
template <class S>
__global__ void rescale_kernel(const StepArgs<S> a, S *f0, S *f1, const double *tot) {
    using C = typename Compute<S>::type;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const double n = tot[3], m = n + tot[2];
    if (!(n > 0.0) || !(m > 0.0) || !isfinite(m)) return;
    const long long k = (long long)y * a.pitch + x;
    if ((decode(a.code[k]) & 3) == KIND_SOLID) return;
    // f' = c f with c = n / m, stored as f' - w = c (f - w) + (c - 1) w
    const C c = C(n / m), cm1 = C(-tot[2] / m);
    S *f = (blockIdx.z ? f1 : f0) + k;
#pragma unroll
    for (int q = 0; q < 9; q++) st(f + q * a.plane, c * ld(f + q * a.plane) + cm1 * wq<C>(q));
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
        const double t0 = (double)r[0], t1 = (double)r[1], t2 = (double)r[2];
        const double e0 = (double)r[nx - 1], e1 = (double)r[nx - 2], e2 = (double)r[nx - 3];
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

// ---------------------------------------------------------------------------
// Host launchers of the energy-update options (QUICK face values, sub-steps),
// compiled in their own translation unit (fv_modes.cu) for every storage
// type; the handle code fills the arguments.
// ---------------------------------------------------------------------------
namespace lbmfvm_fv {

// Arguments of one launch of step_tma_kernel over one tile list.
template <class S>
struct TmaLaunch {
    lbmfvm_dev::StepArgs<S> a;
    const lbmfvm_dev::CavityDesc *cavs;
    const lbmfvm_dev::TileHeader *tiles;  // first header of the list
    const int *count;                     // the list's count slot
    const CUtensorMap *map_f, *map_T, *map_c, *map_fo, *map_To;
    int *ctr, *ctr_next;                  // the list's tile counters of this step and the next
    int nfix, blocks;
    cudaStream_t stream;
};

// Box geometry of a tile shape (the host encodes its tensor maps from it).
struct TmaShape {
    int TW, TH, FW, FH, TWD, THT, THT_QUICK, CWD, CHT, STAGES, BLOCK;
    unsigned SMEM;
};

// Tile shape cfg of the fused step kernel (central energy update): its
// geometry, the shared-memory limit set and its blocks per SM.  Compiled in
// one translation unit per storage type (step_*.cu).
template <class S>
cudaError_t tma_prepare(int cfg, TmaShape *shape, int *blocks_per_sm);
// Launch of the fused step kernel of tile shape cfg.
template <class S>
cudaError_t tma_launch(int cfg, const TmaLaunch<S> &l);

// Shared-memory limits of the QUICK (two temperature halo rows) and the
// given-temperature kernels of shape kTmaConfigFv; blocks per SM of each.
template <class S>
cudaError_t prepare_modes(int *blocks_quick, int *blocks_given);
// Fused step with QUICK face values, and the collision with a given T^{n+1}.
template <class S>
cudaError_t launch_quick(const TmaLaunch<S> &l);
template <class S>
cudaError_t launch_given(const TmaLaunch<S> &l);
// u^{n+1}, v^{n+1} of the tiles of a list into U, V.
template <class S>
cudaError_t launch_uv(const S *fin, long long plane, int pitch, int gnx, int gny,
                      const lbmfvm_dev::TileHeader *tiles, int ntiles, const lbmfvm_dev::CavityDesc *cavs,
                      const uint8_t *code, typename lbmfvm_dev::Compute<S>::type *U,
                      typename lbmfvm_dev::Compute<S>::type *V, int tw, int th, cudaStream_t stream);
// Sub-step s of the first ntiles tiles of a list (fv_substep_kernel).
template <class C>
cudaError_t launch_substep(bool quick, const C *T0, C *X, C *Y, const C *U, const C *V, const uint8_t *code,
                           const uint8_t *fflags, int pitch, int gnx, int gny, const lbmfvm_dev::TileHeader *tiles,
                           int ntiles, int tw, int th, int s, cudaStream_t stream);

}  // namespace lbmfvm_fv
