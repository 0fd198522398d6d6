// Kernels of the learned warm start (include/surrogate.h).
//
// The forward and adjoint 3x3 convolutions run on the fifth-generation tensor
// cores (conv_tc.cu: tcgen05.mma with tensor-memory accumulators, TMA-staged
// operands).  This file holds the rest:
// weight gradient (wgrad_kernel): one block owns 32 output x 16 input
//   channels and a strided share of the pixel tiles (split K); its nine warps
//   take one tap each, so a staged tile serves all taps; products on the
//   tensor cores by warp-level mma (m16n8k16, BF16, FP32 accumulation) from
//   operands staged by cp.async and read transposed with ldmatrix (rows of
//   16 bytes XOR-swizzled so that the eight rows one ldmatrix phase reads fall
//   in distinct bank groups); partial sums end in FP32 atomics.
// Everything else is small and elementwise.

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>

#include "conv_tc.h"
#include "surrogate.h"

namespace {

thread_local char g_sg_err[256] = "";

int sg_fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_sg_err, sizeof(g_sg_err), fmt, ap);
    va_end(ap);
    return code;
}

constexpr int kOk = 0, kErrArg = -1, kErrCuda = -3;

int launched(const char *what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sg_fail(kErrCuda, "%s: %s", what, cudaGetErrorString(e));
    return kOk;
}

using bf16 = __nv_bfloat16;
constexpr float kLeak = 1.0f / 16.0f;

__device__ __forceinline__ float dleaky(float y) { return y > 0.0f ? 1.0f : kLeak; }

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte asynchronous copy global -> shared; src_bytes = 0 fills zeros.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_addr(p)));
}

// d += a (16x16, row) * b (16x8, col), BF16 inputs, FP32 accumulators.
__device__ __forceinline__ void mma16816(float d[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Element offset of 16-byte chunk `c` of a 32-byte row `r` (two chunks per
// row): chunks swap on every other group of four rows.
__device__ __forceinline__ int sw32(int r, int c) { return r * 16 + ((c ^ ((r >> 2) & 1)) << 3); }
// The same for 64-byte rows (four chunks).
__device__ __forceinline__ int sw64(int r, int c) { return r * 32 + ((c ^ ((r >> 1) & 3)) << 3); }

// ---------------------------------------------------------------------------
// weight gradient of the 3x3 convolution
// ---------------------------------------------------------------------------
constexpr int kTH = 8, kTW = 16;             // pixel tile: 8 rows x 16 pixels
constexpr int kPH = kTH + 2, kPW = kTW + 2;  // staged input with halo
constexpr int kWCo = 32, kWCi = 16;  // channels per block

struct WgradArgs {
    const bf16 *x;
    const bf16 *dy;
    float *dw;
    int ldx, lddy, B, H, W, Cin, Cout, ntiles;
};

__global__ void __launch_bounds__(288) wgrad_kernel(const WgradArgs a) {
    __shared__ __align__(128) bf16 dyt[2][kTH * kTW * kWCo];   // [pixel][32 co], 64-byte rows
    __shared__ __align__(128) bf16 xt[2][kPH * kPW * kWCi];    // [halo pixel][16 ci], 32-byte rows
    const int co0 = blockIdx.x * kWCo, ci0 = blockIdx.y * kWCi;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = a.W / kTW, tiles_y = a.H / kTH;
    const int ky = warp / 3, kx = warp % 3;  // this warp's tap

    auto stage_in = [&](int s, int tile) {
        const int b = tile / (tiles_x * tiles_y), r = tile % (tiles_x * tiles_y);
        const int ty0 = (r / tiles_x) * kTH, tx0 = (r % tiles_x) * kTW;
        for (int i = tid; i < kTH * kTW * 4; i += 288) {
            const int pix = i >> 2, ch = i & 3;
            const int gy = ty0 + pix / kTW, gx = tx0 + pix % kTW;
            cp_async16(&dyt[s][sw64(pix, ch)], a.dy + ((long long)(b * a.H + gy) * a.W + gx) * a.lddy + co0 + ch * 8,
                       16);
        }
        for (int i = tid; i < kPH * kPW * 2; i += 288) {
            const int pix = i >> 1, half = i & 1;
            const int gy = ty0 + pix / kPW - 1, gx = tx0 + pix % kPW - 1;
            const bool in = gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
            const bf16 *src = in ? a.x + ((long long)(b * a.H + gy) * a.W + gx) * a.ldx + ci0 + half * 8 : a.x;
            cp_async16(&xt[s][sw32(pix, half)], src, in ? 16 : 0);
        }
        cp_async_commit();
    };

    float acc[2][2][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++)
#pragma unroll
            for (int k = 0; k < 4; k++) acc[i][j][k] = 0.0f;

    const int mi = lane >> 3, lr = lane & 7;
    int s = 0;
    int tile = blockIdx.z;
    if (tile < a.ntiles) stage_in(0, tile);
    for (; tile < a.ntiles; tile += gridDim.z) {
        const int next = tile + gridDim.z;
        if (next < a.ntiles) {
            stage_in(s ^ 1, next);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const bf16 *D = dyt[s];
        const bf16 *X = xt[s];
#pragma unroll 2
        for (int orow = 0; orow < kTH; orow++) {
            // A (co x pixel) from the [pixel][co] tile, transposed on load:
            // (px 0..7, co +0..7), (px 0..7, co +8..15), (px 8..15, co +0..7), (px 8..15, co +8..15)
            uint32_t afr[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; mt++) {
                const int pix = orow * kTW + (mi >> 1) * 8 + lr;
                ldsm_x4_t(afr[mt][0], afr[mt][1], afr[mt][2], afr[mt][3], &D[sw64(pix, mt * 2 + (mi & 1))]);
            }
            // B (pixel x ci) from the halo tile at this warp's tap, transposed:
            // (px 0..7, ci 0..7), (px 8..15, ci 0..7), (px 0..7, ci 8..15), (px 8..15, ci 8..15)
            uint32_t bfr[2][2];
            const int pix = (orow + ky) * kPW + (mi & 1) * 8 + lr + kx;
            ldsm_x4_t(bfr[0][0], bfr[0][1], bfr[1][0], bfr[1][1], &X[sw32(pix, mi >> 1)]);
#pragma unroll
            for (int mt = 0; mt < 2; mt++)
#pragma unroll
                for (int nt = 0; nt < 2; nt++) mma16816(acc[mt][nt], afr[mt], bfr[nt]);
        }
        __syncthreads();
        s ^= 1;
    }
    const int g = lane >> 2, t = lane & 3;
    const int tap = warp;
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int co = co0 + mt * 16 + g + h * 8, ci = ci0 + nt * 8 + 2 * t;
                float *dst = a.dw + ((long long)co * 9 + tap) * a.Cin + ci;
                atomicAdd(dst, acc[mt][nt][2 * h]);
                atomicAdd(dst + 1, acc[mt][nt][2 * h + 1]);
            }
}

// Bias gradient: db[co] += sum over pixels of dy[., co].
__global__ void bias_grad_kernel(const bf16 *dy, int lddy, long long P, int C, float *db) {
    const long long per = (P + gridDim.x - 1) / gridDim.x;
    const long long p0 = blockIdx.x * per, p1 = p0 + per < P ? p0 + per : P;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float s = 0.0f;
        for (long long p = p0; p < p1; p++) s += __bfloat162float(dy[p * lddy + c]);
        atomicAdd(db + c, s);
    }
}

__global__ void flip_kernel(const bf16 *w, bf16 *wt, int Cin, int Cout) {
    const long long n = (long long)Cout * 9 * Cin;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % Cin);
        const int tap = (int)((i / Cin) % 9);
        const int co = (int)(i / (9LL * Cin));
        wt[((long long)ci * 9 + (8 - tap)) * Cout + co] = w[i];
    }
}

// ---------------------------------------------------------------------------
// pooling, up-sampling
// ---------------------------------------------------------------------------
__global__ void pool2_kernel(const bf16 *x, int ldx, bf16 *y, int ldy, int B, int H, int W, int C) {
    const int Ho = H / 2, Wo = W / 2;
    const long long n = (long long)B * Ho * Wo * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long p = i / C;
        const int xo = (int)(p % Wo), yo = (int)((p / Wo) % Ho), b = (int)(p / ((long long)Wo * Ho));
        const long long q = ((long long)(b * H + 2 * yo) * W + 2 * xo) * ldx + c;
        const float s = __bfloat162float(x[q]) + __bfloat162float(x[q + ldx]) + __bfloat162float(x[q + (long long)W * ldx]) +
                        __bfloat162float(x[q + (long long)W * ldx + ldx]);
        y[p * ldy + c] = __float2bfloat16_rn(0.25f * s);
    }
}

__global__ void pool2_backward_kernel(const bf16 *dy, int lddy, const bf16 *add, int ldadd, const bf16 *m, int ldm,
                                      bf16 *dx, int lddx, int B, int H, int W, int C) {
    const long long n = (long long)B * H * W * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long p = i / C;
        const int xx = (int)(p % W), yy = (int)((p / W) % H), b = (int)(p / ((long long)W * H));
        float v = 0.25f * __bfloat162float(dy[((long long)(b * (H / 2) + yy / 2) * (W / 2) + xx / 2) * lddy + c]);
        if (add) v += __bfloat162float(add[p * ldadd + c]);
        if (m) v *= dleaky(__bfloat162float(m[p * ldm + c]));
        dx[p * lddx + c] = __float2bfloat16_rn(v);
    }
}

__global__ void upsample2_kernel(const bf16 *x, int ldx, bf16 *y, int ldy, int B, int H, int W, int C) {
    const int Ho = 2 * H, Wo = 2 * W;
    const long long n = (long long)B * Ho * Wo * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long p = i / C;
        const int xo = (int)(p % Wo), yo = (int)((p / Wo) % Ho), b = (int)(p / ((long long)Wo * Ho));
        y[p * ldy + c] = x[((long long)(b * H + yo / 2) * W + xo / 2) * ldx + c];
    }
}

__global__ void upsample2_backward_kernel(const bf16 *dy, int lddy, const bf16 *m, int ldm, bf16 *dx, int lddx, int B,
                                          int H, int W, int C) {
    const long long n = (long long)B * H * W * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long p = i / C;
        const int xx = (int)(p % W), yy = (int)((p / W) % H), b = (int)(p / ((long long)W * H));
        const long long q = ((long long)(b * 2 * H + 2 * yy) * (2 * W) + 2 * xx) * lddy + c;
        const long long row = 2LL * W * lddy;
        float s = __bfloat162float(dy[q]) + __bfloat162float(dy[q + lddy]) + __bfloat162float(dy[q + row]) +
                  __bfloat162float(dy[q + row + lddy]);
        if (m) s *= dleaky(__bfloat162float(m[p * ldm + c]));
        dx[p * lddx + c] = __float2bfloat16_rn(s);
    }
}

// ---------------------------------------------------------------------------
// output layer (1x1 convolution), loss, optimiser
// ---------------------------------------------------------------------------
constexpr int kMaxCin1 = 64, kMaxCout1 = 8;

__global__ void conv1x1_kernel(const bf16 *x, int ldx, const float *w, const float *bias, float *y, long long P,
                               int Cin, int Cout) {
    __shared__ float ws[kMaxCout1 * kMaxCin1];
    for (int i = threadIdx.x; i < Cin * Cout; i += blockDim.x) ws[i] = w[i];
    __syncthreads();
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        float acc[kMaxCout1];
        for (int o = 0; o < Cout; o++) acc[o] = bias[o];
        for (int c = 0; c < Cin; c++) {
            const float xv = __bfloat162float(x[p * ldx + c]);
            for (int o = 0; o < Cout; o++) acc[o] += ws[o * Cin + c] * xv;
        }
        for (int o = 0; o < Cout; o++) y[p * Cout + o] = acc[o];
    }
}

__global__ void conv1x1_dx_kernel(const bf16 *x, int ldx, const float *w, const float *dy, bf16 *dx, int lddx,
                                  long long P, int Cin, int Cout) {
    __shared__ float ws[kMaxCout1 * kMaxCin1];
    for (int i = threadIdx.x; i < Cin * Cout; i += blockDim.x) ws[i] = w[i];
    __syncthreads();
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        for (int c = 0; c < Cin; c++) {
            float s = 0.0f;
            for (int o = 0; o < Cout; o++) s += dy[p * Cout + o] * ws[o * Cin + c];
            dx[p * lddx + c] = __float2bfloat16_rn(s * dleaky(__bfloat162float(x[p * ldx + c])));
        }
    }
}

// dw[o][c] += sum_p dy[p][o] x[p][c]; db[o] += sum_p dy[p][o]: thread j owns
// (o, c) = (j / Cin, j % Cin) over the block's share of the pixels.
__global__ void conv1x1_dw_kernel(const bf16 *x, int ldx, const float *dy, float *dw, float *db, long long P, int Cin,
                                  int Cout) {
    const long long per = (P + gridDim.x - 1) / gridDim.x;
    const long long p0 = blockIdx.x * per, p1 = p0 + per < P ? p0 + per : P;
    const int j = threadIdx.x;
    if (j >= Cin * Cout) return;
    const int o = j / Cin, c = j % Cin;
    float s = 0.0f, sb = 0.0f;
    for (long long p = p0; p < p1; p++) {
        const float d = dy[p * Cout + o];
        s += d * __bfloat162float(x[p * ldx + c]);
        sb += d;
    }
    atomicAdd(dw + j, s);
    if (c == 0 && db) atomicAdd(db + o, sb);
}

__global__ void mse_kernel(const float *pred, const float *target, const uint8_t *fluid, long long P, int C,
                           double n_inv, float *dpred, double *loss) {
    __shared__ double red[32];
    double s = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const bool f = fluid[p] != 0;
        for (int c = 0; c < C; c++) {
            const long long i = p * C + c;
            const double d = f ? (double)pred[i] - (double)target[i] : 0.0;
            s += d * d;
            dpred[i] = (float)(2.0 * d * n_inv);
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        atomicAdd(loss, t * n_inv);
    }
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, bf16 *pb, long long n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        p[i] = pi;
        if (pb) pb[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void encode_kernel(const uint8_t *mask, const float *scalars, bf16 *x, int B, int H, int W) {
    const long long n = (long long)B * H * W;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(p / ((long long)H * W));
        bf16 *o = x + p * 16;
        o[0] = __float2bfloat16_rn(mask[p] ? 1.0f : 0.0f);
        o[1] = __float2bfloat16_rn(scalars[2 * b]);
        o[2] = __float2bfloat16_rn(scalars[2 * b + 1]);
        for (int c = 3; c < 16; c++) o[c] = __float2bfloat16_rn(0.0f);
    }
}

__global__ void resample_mask_kernel(const uint8_t *mask, int nx, int ny, uint8_t *out, int H, int W) {
    const int n = H * W;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int y = p / W, x = p % W;
        int sy = (int)(((double)y + 0.5) * ny / H), sx = (int)(((double)x + 0.5) * nx / W);
        sy = sy < ny ? sy : ny - 1;
        sx = sx < nx ? sx : nx - 1;
        out[p] = mask[(long long)sy * nx + sx];
    }
}

__global__ void resample_fields_kernel(const float *pred, int H, int W, const uint8_t *mask, int nx, int ny, float U0,
                                       float *u, float *v, float *T) {
    const long long n = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % nx), j = (int)(k / nx);
        float fx = ((float)i + 0.5f) * W / nx - 0.5f, fy = ((float)j + 0.5f) * H / ny - 0.5f;
        fx = fminf(fmaxf(fx, 0.0f), (float)(W - 1));
        fy = fminf(fmaxf(fy, 0.0f), (float)(H - 1));
        const int x0 = (int)fx, y0 = (int)fy;
        const int x1 = x0 + 1 < W ? x0 + 1 : W - 1, y1 = y0 + 1 < H ? y0 + 1 : H - 1;
        const float ax = fx - x0, ay = fy - y0;
        float out[3];
        for (int c = 0; c < 3; c++) {
            const float a00 = pred[((long long)y0 * W + x0) * 3 + c], a01 = pred[((long long)y0 * W + x1) * 3 + c];
            const float a10 = pred[((long long)y1 * W + x0) * 3 + c], a11 = pred[((long long)y1 * W + x1) * 3 + c];
            out[c] = (1 - ay) * ((1 - ax) * a00 + ax * a01) + ay * ((1 - ax) * a10 + ax * a11);
        }
        const bool still = (mask && mask[k]) || i == 0 || j == 0 || i == nx - 1 || j == ny - 1;
        u[k] = still ? 0.0f : out[0] * U0;
        v[k] = still ? 0.0f : out[1] * U0;
        T[k] = fminf(fmaxf(out[2], 0.0f), 1.0f);
    }
}

int grid_for(long long n, int block = 256) {
    long long g = (n + block - 1) / block;
    return (int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" {

const char *lbmfvm_sg_last_error(void) { return g_sg_err; }

int lbmfvm_sg_conv3x3(const uint16_t *x, int32_t ldx, const uint16_t *w, const float *bias, uint16_t *y, int32_t ldy,
                      const uint16_t *m, int32_t ldm, int32_t B, int32_t H, int32_t W, int32_t Cin, int32_t Cout,
                      int32_t mode, void *stream) {
    if (!x || !w || !y || (mode == LBMFVM_SG_DLEAKY && !m)) return sg_fail(kErrArg, "conv3x3: NULL tensor");
    if (mode < LBMFVM_SG_LINEAR || mode > LBMFVM_SG_DLEAKY) return sg_fail(kErrArg, "conv3x3: mode %d", mode);
    if (B < 1 || H < 8 || W < 16 || H % 8 || W % 16 || Cin < 16 || Cin % 16 || Cout < 32 || Cout % 32)
        return sg_fail(kErrArg, "conv3x3: shape B=%d H=%d W=%d Cin=%d Cout=%d breaks the tile rules", B, H, W, Cin,
                       Cout);
    if (ldx < Cin || ldy < Cout || ldx % 8 || ldy % 8 || (m && (ldm < Cout || ldm % 8)) || !aligned16(x) ||
        !aligned16(w) || !aligned16(y) || (m && !aligned16(m)))
        return sg_fail(kErrArg, "conv3x3: strides or alignment");
    return lbmfvm_sg_tc::conv3x3(x, ldx, w, bias, y, ldy, m, ldm, B, H, W, Cin, Cout, mode, (cudaStream_t)stream,
                                 g_sg_err, sizeof(g_sg_err));
}

int lbmfvm_sg_inject_stall(void) {
    lbmfvm_sg_tc::inject_stall();
    return kOk;
}

int lbmfvm_sg_check(void *stream) {
    const int r = lbmfvm_sg_tc::check((cudaStream_t)stream);
    if (r == -4) return sg_fail(-4, "a bounded wait of the tensor-core convolution ran out");
    if (r) return sg_fail(kErrCuda, "status check failed");
    return kOk;
}

int lbmfvm_sg_flip(const uint16_t *w, uint16_t *wt, int32_t Cin, int32_t Cout, void *stream) {
    if (!w || !wt || Cin < 1 || Cout < 1) return sg_fail(kErrArg, "flip: arguments");
    flip_kernel<<<grid_for(9LL * Cin * Cout), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const bf16 *>(w), reinterpret_cast<bf16 *>(wt), Cin, Cout);
    return launched("flip");
}

int lbmfvm_sg_conv3x3_wgrad(const uint16_t *x, int32_t ldx, const uint16_t *dy, int32_t lddy, float *dw, float *db,
                            int32_t B, int32_t H, int32_t W, int32_t Cin, int32_t Cout, void *stream) {
    if (!x || !dy || !dw) return sg_fail(kErrArg, "wgrad: NULL tensor");
    if (B < 1 || H < 8 || W < 16 || H % 8 || W % 16 || Cin < 16 || Cin % 16 || Cout < 32 || Cout % 32)
        return sg_fail(kErrArg, "wgrad: shape B=%d H=%d W=%d Cin=%d Cout=%d breaks the tile rules", B, H, W, Cin, Cout);
    if (ldx < Cin || lddy < Cout || ldx % 8 || lddy % 8 || !aligned16(x) || !aligned16(dy))
        return sg_fail(kErrArg, "wgrad: strides or alignment");
    const int ntiles = B * (H / kTH) * (W / kTW);
    const int gx = Cout / kWCo, gy = Cin / kWCi;
    int split = (4 * 152 + gx * gy - 1) / (gx * gy);
    split = split < ntiles ? split : ntiles;
    WgradArgs a{reinterpret_cast<const bf16 *>(x), reinterpret_cast<const bf16 *>(dy), dw, ldx, lddy, B, H, W, Cin,
                Cout, ntiles};
    wgrad_kernel<<<dim3(gx, gy, split), 288, 0, (cudaStream_t)stream>>>(a);
    if (int r = launched("wgrad")) return r;
    if (db) {
        const long long P = (long long)B * H * W;
        bias_grad_kernel<<<grid_for(P, 1024) < 512 ? grid_for(P, 1024) : 512, 128, 0, (cudaStream_t)stream>>>(
            reinterpret_cast<const bf16 *>(dy), lddy, P, Cout, db);
        return launched("bias gradient");
    }
    return kOk;
}

int lbmfvm_sg_pool2(const uint16_t *x, int32_t ldx, uint16_t *y, int32_t ldy, int32_t B, int32_t H, int32_t W,
                    int32_t C, void *stream) {
    if (!x || !y || B < 1 || H < 2 || W < 2 || H % 2 || W % 2 || C < 1 || ldx < C || ldy < C)
        return sg_fail(kErrArg, "pool2: arguments");
    pool2_kernel<<<grid_for((long long)B * H * W * C / 4), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const bf16 *>(x), ldx, reinterpret_cast<bf16 *>(y), ldy, B, H, W, C);
    return launched("pool2");
}

int lbmfvm_sg_pool2_backward(const uint16_t *dy, int32_t lddy, const uint16_t *add, int32_t ldadd, const uint16_t *m,
                             int32_t ldm, uint16_t *dx, int32_t lddx, int32_t B, int32_t H, int32_t W, int32_t C,
                             void *stream) {
    if (!dy || !dx || B < 1 || H < 2 || W < 2 || H % 2 || W % 2 || C < 1 || lddy < C || lddx < C ||
        (add && ldadd < C) || (m && ldm < C))
        return sg_fail(kErrArg, "pool2_backward: arguments");
    pool2_backward_kernel<<<grid_for((long long)B * H * W * C), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const bf16 *>(dy), lddy, reinterpret_cast<const bf16 *>(add), ldadd,
        reinterpret_cast<const bf16 *>(m), ldm, reinterpret_cast<bf16 *>(dx), lddx, B, H, W, C);
    return launched("pool2_backward");
}

int lbmfvm_sg_upsample2(const uint16_t *x, int32_t ldx, uint16_t *y, int32_t ldy, int32_t B, int32_t H, int32_t W,
                        int32_t C, void *stream) {
    if (!x || !y || B < 1 || H < 1 || W < 1 || C < 1 || ldx < C || ldy < C) return sg_fail(kErrArg, "upsample2: arguments");
    upsample2_kernel<<<grid_for(4LL * B * H * W * C), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const bf16 *>(x), ldx, reinterpret_cast<bf16 *>(y), ldy, B, H, W, C);
    return launched("upsample2");
}

int lbmfvm_sg_upsample2_backward(const uint16_t *dy, int32_t lddy, const uint16_t *m, int32_t ldm, uint16_t *dx,
                                 int32_t lddx, int32_t B, int32_t H, int32_t W, int32_t C, void *stream) {
    if (!dy || !dx || B < 1 || H < 1 || W < 1 || C < 1 || lddy < C || lddx < C || (m && ldm < C))
        return sg_fail(kErrArg, "upsample2_backward: arguments");
    upsample2_backward_kernel<<<grid_for((long long)B * H * W * C), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const bf16 *>(dy), lddy, reinterpret_cast<const bf16 *>(m), ldm, reinterpret_cast<bf16 *>(dx),
        lddx, B, H, W, C);
    return launched("upsample2_backward");
}

int lbmfvm_sg_conv1x1(const uint16_t *x, int32_t ldx, const float *w, const float *b, float *y, int64_t P,
                      int32_t Cin, int32_t Cout, void *stream) {
    if (!x || !w || !b || !y || P < 1 || Cin < 1 || Cin > kMaxCin1 || Cout < 1 || Cout > kMaxCout1 || ldx < Cin)
        return sg_fail(kErrArg, "conv1x1: arguments");
    conv1x1_kernel<<<grid_for(P), 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const bf16 *>(x), ldx, w, b, y, P,
                                                                   Cin, Cout);
    return launched("conv1x1");
}

int lbmfvm_sg_conv1x1_backward(const uint16_t *x, int32_t ldx, const float *w, const float *dy, uint16_t *dx,
                               int32_t lddx, float *dw, float *db, int64_t P, int32_t Cin, int32_t Cout,
                               void *stream) {
    if (!x || !w || !dy || !dw || P < 1 || Cin < 1 || Cin > kMaxCin1 || Cout < 1 || Cout > kMaxCout1 || ldx < Cin ||
        (dx && lddx < Cin) || Cin * Cout > 1024)
        return sg_fail(kErrArg, "conv1x1_backward: arguments");
    cudaStream_t s = (cudaStream_t)stream;
    if (dx) {
        conv1x1_dx_kernel<<<grid_for(P), 256, 0, s>>>(reinterpret_cast<const bf16 *>(x), ldx, w, dy,
                                                      reinterpret_cast<bf16 *>(dx), lddx, P, Cin, Cout);
        if (int r = launched("conv1x1 dx")) return r;
    }
    const int threads = (Cin * Cout + 31) / 32 * 32;
    const int blocks = (int)((P + 1023) / 1024 < 1024 ? (P + 1023) / 1024 : 1024);
    conv1x1_dw_kernel<<<blocks, threads, 0, s>>>(reinterpret_cast<const bf16 *>(x), ldx, dy, dw, db, P, Cin, Cout);
    return launched("conv1x1 dw");
}

int lbmfvm_sg_mse(const float *pred, const float *target, const uint8_t *fluid, int64_t P, int32_t C, double n_inv,
                  float *dpred, double *loss, void *stream) {
    if (!pred || !target || !fluid || !dpred || !loss || P < 1 || C < 1) return sg_fail(kErrArg, "mse: arguments");
    mse_kernel<<<grid_for(P) < 1024 ? grid_for(P) : 1024, 256, 0, (cudaStream_t)stream>>>(pred, target, fluid, P, C,
                                                                                         n_inv, dpred, loss);
    return launched("mse");
}

int lbmfvm_sg_adam(float *p, const float *g, float *m, float *v, uint16_t *p_bf16, int64_t n, float lr, float beta1,
                   float beta2, float eps, int32_t t, void *stream) {
    if (!p || !g || !m || !v || n < 1 || t < 1) return sg_fail(kErrArg, "adam: arguments");
    const float c1 = 1.0f / (1.0f - powf(beta1, (float)t)), c2 = 1.0f / (1.0f - powf(beta2, (float)t));
    adam_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, reinterpret_cast<bf16 *>(p_bf16), n, lr,
                                                                beta1, beta2, eps, c1, c2);
    return launched("adam");
}

int lbmfvm_sg_encode(const uint8_t *mask, const float *scalars, uint16_t *x, int32_t B, int32_t H, int32_t W,
                     void *stream) {
    if (!mask || !scalars || !x || B < 1 || H < 1 || W < 1) return sg_fail(kErrArg, "encode: arguments");
    encode_kernel<<<grid_for((long long)B * H * W), 256, 0, (cudaStream_t)stream>>>(mask, scalars,
                                                                                     reinterpret_cast<bf16 *>(x), B, H, W);
    return launched("encode");
}

int lbmfvm_sg_resample_mask(const uint8_t *mask, int32_t nx, int32_t ny, uint8_t *out, int32_t H, int32_t W,
                            void *stream) {
    if (!mask || !out || nx < 1 || ny < 1 || H < 1 || W < 1) return sg_fail(kErrArg, "resample_mask: arguments");
    resample_mask_kernel<<<grid_for((long long)H * W), 256, 0, (cudaStream_t)stream>>>(mask, nx, ny, out, H, W);
    return launched("resample_mask");
}

int lbmfvm_sg_resample_fields(const float *pred, int32_t H, int32_t W, const uint8_t *mask, int32_t nx, int32_t ny,
                              float U0, float *u, float *v, float *T, void *stream) {
    if (!pred || !u || !v || !T || H < 1 || W < 1 || nx < 1 || ny < 1) return sg_fail(kErrArg, "resample_fields: arguments");
    resample_fields_kernel<<<grid_for((long long)nx * ny), 256, 0, (cudaStream_t)stream>>>(pred, H, W, mask, nx, ny,
                                                                                            U0, u, v, T);
    return launched("resample_fields");
}

}  // extern "C"
