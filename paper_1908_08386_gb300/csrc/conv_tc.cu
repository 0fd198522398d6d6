// 3x3 convolution of the warm-start surrogate on the fifth-generation tensor
// cores: tcgen05.mma (BF16 x BF16, FP32 accumulation in tensor memory),
// operands staged in shared memory by TMA, results read back with tcgen05.ld.
//
// Implicit GEMM.  A tile is M = 128 consecutive output positions of one image
// and all N = Cout output channels; K runs over the nine taps and the input
// channels, 16 per MMA.  Positions are counted in a padded row
// layout of Wp = W + 8 pixels per row: image pixel (y, x) sits at position
// q = (y + 1) Wp + 8 + x, and the eight positions before each row's pixels
// hold zeros, so that the left neighbour of x = 0 (q - 1) and the right
// neighbour of x = W - 1 (the next row's position 0) read zero padding.  Tap
// (ky, kx) of output position q reads input position q + (ky - 1) Wp + kx - 1,
// so for a tile of 128 consecutive positions each tap's A operand is again a
// run of 128 consecutive positions: the shared-memory descriptor of a tap is
// the staged rows' base shifted by one row per position, with no re-staging.
//
// Shared-memory operand layout (K-major, swizzled): a pipeline stage holds KC
// input channels (16, 32 or 64); each staged position (A) and each output
// channel of each tap (B) is one row of 2 KC bytes (32, 64 or 128), rows
// consecutive, in the 32-, 64- or 128-byte swizzle that TMA writes and the
// matrix descriptors name.  The swizzle acts on absolute shared-memory
// address bits, so a descriptor moved by whole rows (a tap's shift) or by 32
// bytes inside a row (a K step of 16 channels) reads the same layout.  One TMA
// box per stage brings the staged rows (one request per position: the
// chunk's channels of a pixel are contiguous in the NHWC tensor), each row
// from x = -8 (the pad positions, which the out-of-bounds fill makes zero) to
// W - 1, rows outside the image zero-filled; a second box brings the chunk's
// weights for all nine taps.
//
// A unit is G tiles of 128 consecutive positions of one image, each with its
// own accumulator in tensor memory: the staged rows and weights of a chunk
// serve all of them (the halo rows and the weights are staged once per G
// tiles).
//
// Persistent pipeline, one block per SM taking units in turn, three roles:
// one thread of warp 0 issues the two TMA loads of every chunk into a ring of
// stages (each refilled once the MMAs that read it have completed); one
// thread of warp 1 issues the 9 (KC / 16) G MMAs of a chunk once it has
// landed, commits the stage back to the loader, and after a unit's last chunk
// commits its accumulator set to the epilogue; warps 2-5 (each one quarter of
// the 128 tensor-memory lanes) read the set, add the bias and apply the
// activation (or multiply by the activation's derivative), store BF16 and
// hand the set back.  Two accumulator sets alternate, so a unit's epilogue
// overlaps the next unit's MMAs.  Every wait is bounded (1 s); a wait that
// runs out sets a device status word, and the block drains its copies and
// MMAs before it leaves.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <atomic>
#include <mutex>

#include "conv_tc.h"
#include "surrogate.h"

namespace lbmfvm_sg_tc {

namespace {

using bf16 = __nv_bfloat16;

constexpr int kM = 128;        // output positions per tile (TMEM lanes)
constexpr int kThreads = 192;  // a loading warp, an issuing warp, four epilogue warps
constexpr int kPad = 8;        // zero positions before each padded row (128 bytes per plane)
constexpr int kMaxStages = 8;
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr float kLeak = 1.0f / 16.0f;

struct Params {
    const float *bias;
    bf16 *y;
    const bf16 *m;
    int *status;
    int ldy, ldm, B, H, W, Cout, mode;
    int Wp;           // padded row length in positions
    int tiles;        // tiles of 128 positions per image
    int supers;       // units per image: ceil(tiles / G)
    uint32_t acc;     // TMEM columns between accumulators
    int nch;          // chunks of KC input channels
    int stages;
    int nrows;        // padded rows staged per block (the largest any block needs)
    uint32_t rowb;    // bytes of one staged row (one position or one output channel): 2 KC
    uint32_t a_bytes; // bytes of the staged rows of activations (nrows Wp rows)
    uint32_t b_off;   // offset of the weights in a stage (a_bytes rounded up to 1 KB)
    uint32_t b_tap;   // bytes of one tap's weights (Cout rows)
    uint32_t stage;   // bytes of one stage: activations, then the nine taps' weights
    uint32_t ncols;   // TMEM columns allocated (two sets of G accumulators)
    uint32_t idesc;   // instruction descriptor
    int stall;        // block 0 skips its first load (a test of the bounded waits)
};

__device__ __forceinline__ uint32_t saddr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for the phase of the given parity to complete, at most kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    for (uint32_t it = 0;; it++) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63u) == 63u && now_ns() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(saddr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(saddr(bar))
        : "memory");
}
// Shared-memory matrix descriptor of a K-major operand in swizzled rows of
// rowb bytes (the layout TMA writes with the matching swizzle): start
// address, the stride between groups of eight rows (8 rowb), the swizzle.
// The swizzle applies to the absolute shared-memory address, so a start
// moved by whole rows (the taps' shifts) or by 32 bytes within a row (the K
// steps) needs no base offset.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t rowb, uint32_t layout) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(((8u * rowb) >> 4) & 0x3FFFu) << 32) |
           (1ull << 46) | ((uint64_t)layout << 61);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float leaky(float v) { return v > 0.0f ? v : kLeak * v; }
__device__ __forceinline__ float dleaky(float y) { return y > 0.0f ? 1.0f : kLeak; }

// First padded row a tile stages (the row of its first input position).
__device__ __forceinline__ int first_row(int q0, int Wp) { return (q0 - Wp - 1) / Wp; }

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

// Persistent: a block takes units (G consecutive tiles of one image) in turn,
// with three roles.  Warp 0 (one thread) loads the stages of every chunk of
// every unit through a ring of p.stages stages; warp 1 (one thread) issues the
// MMAs of a unit into one of two accumulator sets in tensor memory and
// commits each stage back to the loader; warps 2-5 read the finished set
// (each its quarter of the 128 lanes), apply the epilogue and store, and
// hand the set back, so that a unit's epilogue overlaps the next unit's MMAs.
// KC input channels per stage and G tiles per unit are template parameters,
// so that the issuing thread's nine KC / 16 G MMAs per chunk unroll into
// descriptor additions of constants.
template <int KC, int G>
__global__ void __launch_bounds__(kThreads, 1)
    conv3x3_tc_kernel(const Params p, const __grid_constant__ CUtensorMap map_x,
                      const __grid_constant__ CUtensorMap map_w) {
    constexpr uint32_t ROWB = 2 * KC;                                  // bytes per staged row
    constexpr uint32_t LAYOUT = KC == 16 ? 6u : (KC == 32 ? 4u : 2u);  // 32-, 64-, 128-byte swizzle
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], accf[2], acce[2], drain;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int units = p.B * p.supers;
    const uint32_t set_cols = (uint32_t)G * p.acc;  // columns of one accumulator set
    uint8_t *base = smem + ((1024 - (saddr(smem) & 1023u)) & 1023u);
    auto geometry = [&](int u, int &b, int &q0, int &ry0, int &g_n) {
        b = u / p.supers;
        const int t0 = (u % p.supers) * G;
        g_n = p.tiles - t0 < G ? p.tiles - t0 : G;
        q0 = p.Wp + kPad + kM * t0;  // first output position of the unit
        ry0 = first_row(q0, p.Wp);
    };
    auto give_up = [&]() {
        abort_flag = 1;
        atomicExch(p.status, 1);
    };

    if (tid == 0) {
        for (int s = 0; s < p.stages; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int i = 0; i < 2; i++) {
            mbar_init(&accf[i], 1);
            mbar_init(&acce[i], 4);  // one arrival per epilogue warp
        }
        mbar_init(&drain, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                     "r"(p.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // loader: chunk loads n = 0, 1, ... into stage n % stages
            int n = 0;
            for (int u = blockIdx.x; u < units && !abort_flag; u += gridDim.x) {
                int b, q0, ry0, g_n;
                geometry(u, b, q0, ry0, g_n);
                for (int c = 0; c < p.nch; c++, n++) {
                    const int s = n % p.stages;
                    if (n >= p.stages && !mbar_wait(&empty[s], (uint32_t)(n / p.stages - 1) & 1u)) {
                        give_up();
                        break;
                    }
                    if (p.stall && blockIdx.x == 0 && n == 0) continue;  // never issued: its waits run out
                    uint8_t *st = base + (size_t)s * p.stage;
                    mbar_expect_tx(&full[s], p.a_bytes + 9u * p.b_tap);
                    // the chunk's channels of the staged rows, each row from
                    // x = -8 (the pad positions, zero-filled) to W - 1
                    tma_load_4d(st, &map_x, c * KC, -kPad, ry0 - 1, b, &full[s]);
                    // the chunk's channels of every output channel's weights
                    tma_load_3d(st + p.b_off, &map_w, c * KC, 0, 0, &full[s]);
                }
            }
            // every load issued has landed before the block leaves
            for (int m = n - p.stages < 0 ? 0 : n - p.stages; m < n; m++)
                if (!(p.stall && blockIdx.x == 0 && m == 0)) mbar_wait(&full[m % p.stages], (uint32_t)(m / p.stages) & 1u);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            int n = 0, i = 0;
            for (int u = blockIdx.x; u < units && !abort_flag; u += gridDim.x, i++) {
                int b, q0, ry0, g_n;
                geometry(u, b, q0, ry0, g_n);
                const int set = i & 1;
                // the epilogue has emptied this set (its use two units ago)
                if (i >= 2 && !mbar_wait(&acce[set], (uint32_t)((i >> 1) - 1) & 1u)) {
                    give_up();
                    break;
                }
                tc_after_sync();
                const uint32_t acc0 = tmem + (uint32_t)set * set_cols;
                for (int c = 0; c < p.nch; c++, n++) {
                    const int s = n % p.stages;
                    if (!mbar_wait(&full[s], (uint32_t)(n / p.stages) & 1u)) {
                        give_up();
                        break;
                    }
                    tc_after_sync();
                    const uint32_t st = saddr(base + (size_t)s * p.stage);
                    // descriptors of the first tile's centre tap and the first
                    // tap's weights; every other operand is a constant number
                    // of 16-byte units away (start addresses live in the
                    // descriptor's low bits)
                    const uint64_t a0 = sdesc(st + (uint32_t)(q0 - ry0 * p.Wp) * ROWB, ROWB, LAYOUT);
                    const uint64_t b0 = sdesc(st + p.b_off, ROWB, LAYOUT);
                    const int wp16 = p.Wp * (int)(ROWB / 16), tap16 = (int)(p.b_tap / 16);
#pragma unroll
                    for (int tap = 0; tap < 9; tap++) {
                        const int off16 = (tap / 3 - 1) * wp16 + (tap % 3 - 1) * (int)(ROWB / 16);
#pragma unroll
                        for (int kk = 0; kk < KC / 16; kk++) {
                            const uint64_t bd = b0 + (uint64_t)(tap * tap16 + 2 * kk);
#pragma unroll
                            for (int g = 0; g < G; g++)
                                if (g < g_n)
                                    mma(acc0 + (uint32_t)g * p.acc,
                                        a0 + (uint64_t)(off16 + g * kM * (int)(ROWB / 16) + 2 * kk), bd, p.idesc,
                                        (c | tap | kk) != 0);
                        }
                    }
                    mma_commit(&empty[s]);
                }
                if (abort_flag) break;
                mma_commit(&accf[set]);
            }
            // every MMA issued has completed before the block leaves
            mma_commit(&drain);
            mbar_wait(&drain, 0);
        }
        __syncwarp();
    } else {
        // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31
        const int quarter = warp & 3;
        int i = 0;
        for (int u = blockIdx.x; u < units && !abort_flag; u += gridDim.x, i++) {
            int b, q0, ry0, g_n;
            geometry(u, b, q0, ry0, g_n);
            const int set = i & 1;
            if (!mbar_wait(&accf[set], (uint32_t)(i >> 1) & 1u)) {
                give_up();
                break;
            }
            tc_after_sync();
            for (int g = 0; g < g_n; g++) {
                const int q = q0 + kM * g + quarter * 32 + lane;
                const int yy = q / p.Wp - 1, xx = q % p.Wp - kPad;
                const bool valid = yy >= 0 && yy < p.H && xx >= 0 && xx < p.W;
                const long long pix = ((long long)b * p.H + yy) * p.W + xx;
                for (int j = 0; j < p.Cout / 16; j++) {
                    uint32_t r[16];
                    tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)set * set_cols +
                                  (uint32_t)g * p.acc + (uint32_t)(16 * j),
                              r);
                    if (!valid) continue;
                    float v[16];
#pragma unroll
                    for (int k = 0; k < 16; k++) v[k] = __uint_as_float(r[k]);
                    const int co = 16 * j;
                    if (p.mode == LBMFVM_SG_DLEAKY) {
                        const uint4 *mm = reinterpret_cast<const uint4 *>(p.m + pix * p.ldm + co);
                        const uint4 m0 = mm[0], m1 = mm[1];
                        const bf16 *mb0 = reinterpret_cast<const bf16 *>(&m0);
                        const bf16 *mb1 = reinterpret_cast<const bf16 *>(&m1);
#pragma unroll
                        for (int k = 0; k < 8; k++) {
                            v[k] *= dleaky(__bfloat162float(mb0[k]));
                            v[8 + k] *= dleaky(__bfloat162float(mb1[k]));
                        }
                    } else {
                        if (p.bias) {
#pragma unroll
                            for (int k = 0; k < 16; k++) v[k] += p.bias[co + k];
                        }
                        if (p.mode == LBMFVM_SG_LEAKY) {
#pragma unroll
                            for (int k = 0; k < 16; k++) v[k] = leaky(v[k]);
                        }
                    }
                    uint4 o[2];
                    __nv_bfloat162 *ob = reinterpret_cast<__nv_bfloat162 *>(o);
#pragma unroll
                    for (int k = 0; k < 8; k++) ob[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
                    uint4 *dst = reinterpret_cast<uint4 *>(p.y + pix * p.ldy + co);
                    dst[0] = o[0];
                    dst[1] = o[1];
                }
            }
            // the set is free for the unit after next
            tc_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[set]);
        }
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.ncols) : "memory");
    }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// One status word per device, allocated on the device's first use.
std::atomic<bool> g_stall_next{false};

int *status_word() {
    constexpr int kMaxDevices = 64;
    static int *words[kMaxDevices] = {};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!words[dev] && cudaMalloc(&words[dev], sizeof(int)) == cudaSuccess) cudaMemset(words[dev], 0, sizeof(int));
    return words[dev];
}

}  // namespace

int conv3x3(const uint16_t *x, int ldx, const uint16_t *w, const float *bias, uint16_t *y, int ldy,
            const uint16_t *m, int ldm, int B, int H, int W, int Cin, int Cout, int mode, cudaStream_t stream,
            char *msg, size_t msglen, int g_req, int kc_req, int s_req) {
    auto fail = [&](int code, const char *what) {
        snprintf(msg, msglen, "conv3x3: %s", what);
        return code;
    };
    if (W % 16 || W > 240 || Cout > 256 || Cout % 32 || Cin % 16)
        return fail(-1, "the tensor-core kernel needs W % 16 == 0, W <= 240, Cout % 32 == 0, Cout <= 256, Cin % 16 == 0");
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return fail(-3, "cuTensorMapEncodeTiled is not available");
    int *status = status_word();
    if (!status) return fail(-3, "status word allocation failed");

    Params p{};
    p.bias = bias;
    p.y = reinterpret_cast<bf16 *>(y);
    p.m = reinterpret_cast<const bf16 *>(m);
    p.status = status;
    p.stall = g_stall_next.exchange(false) ? 1 : 0;
    p.ldy = ldy;
    p.ldm = ldm;
    p.B = B;
    p.H = H;
    p.W = W;
    p.Cout = Cout;
    p.mode = mode;
    p.Wp = W + kPad;
    const int q_first = p.Wp + kPad, q_end = H * p.Wp + kPad + W;  // output positions [q_first, q_end)
    p.tiles = (q_end - q_first + kM - 1) / kM;
    p.acc = 32;
    while ((int)p.acc < Cout) p.acc <<= 1;
    // instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B,
    // both K-major, N = Cout, M = 128
    p.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Cout >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
    const size_t extra = 1024;  // alignment of the stage area
    const size_t whole = 220 * 1024;
    auto rows_for = [&](int G) {
        int most = 0;
        for (int t0 = 0; t0 < p.tiles; t0 += G) {
            const int g_n = p.tiles - t0 < G ? p.tiles - t0 : G;
            const int q0 = q_first + kM * t0;
            const int rows = (q0 + kM * g_n + p.Wp) / p.Wp - (q0 - p.Wp - 1) / p.Wp + 1;
            if (rows > most) most = rows;
        }
        return most;
    };
    // a stage: the staged rows of KC channels, then the nine taps' weights,
    // each part starting on a 1 KB boundary (every TMA destination on a
    // swizzle-pattern boundary)
    auto up1k = [](size_t v) { return (v + 1023) & ~(size_t)1023; };
    auto stage_for = [&](int G, int KC) {
        const size_t rowb = 2 * (size_t)KC;
        return up1k(up1k((size_t)rows_for(G) * p.Wp * rowb) + 9 * (size_t)Cout * rowb);
    };
    // Channels per stage KC (64, 32 or 16: rows of 128, 64 or 32 bytes, one
    // TMA request per position and chunk) and 128-position tiles per block G
    // (a block stages its rows and the chunk's weights once for all its
    // tiles, each with its own accumulator): the widest rows, then the most
    // tiles (at most four) that let a stage fit twice in shared memory.
    // Measured on the network's layers (16, 32 or 64 channels per stage, 1,
    // 2 or 4 tiles per unit, 2 to 7 stages): 32 channels per stage where the
    // input has a multiple of 32 and two such stages fit, else 16; one tile
    // per unit for accumulators of 128 or 256 columns, else two (32 channels
    // per stage) or four (16); three stages (deeper rings were no faster).
    int KC = kc_req, G = g_req;
    if (KC <= 0) {
        const int g_probe = p.acc >= 128 ? 1 : 2;
        KC = (Cin % 32 == 0 && (whole - extra) / stage_for(g_probe, 32) >= 2) ? 32 : 16;
    }
    if (G <= 0) {
        G = p.acc >= 128 ? 1 : (KC == 16 ? 4 : 2);
        if (2u * (uint32_t)G * p.acc > 512u) G = (int)(256 / p.acc);
        while (G > 1 && G / 2 >= p.tiles) G >>= 1;
    }
    if (KC != 16 && KC != 32 && KC != 64) return fail(-1, "channels per stage must be 16, 32 or 64");
    if (Cin % KC) return fail(-1, "Cin is not a multiple of the channels per stage");
    if (G < 1 || 2u * (uint32_t)G * p.acc > 512u) return fail(-1, "two accumulator sets exceed the tensor memory");
    p.nch = Cin / KC;
    p.rowb = 2u * (uint32_t)KC;
    p.supers = (p.tiles + G - 1) / G;
    p.ncols = 2u * (uint32_t)G * p.acc;  // two accumulator sets
    p.nrows = rows_for(G);
    p.a_bytes = (uint32_t)p.nrows * p.Wp * p.rowb;
    p.b_off = (uint32_t)up1k(p.a_bytes);
    p.b_tap = (uint32_t)Cout * p.rowb;
    p.stage = (uint32_t)stage_for(G, KC);
    // three stages where they fit, else two (one persistent block per SM)
    int stages = s_req > 0 ? s_req : ((whole - extra) / p.stage >= 3 ? 3 : 2);
    if (stages > kMaxStages) stages = kMaxStages;
    if ((size_t)stages * p.stage + extra > whole) return fail(-1, "the stages do not fit in shared memory");
    if (stages < 2) return fail(-1, "a pipeline stage does not fit twice in shared memory");
    p.stages = stages;
    // at least half the shared memory, so that one block holds an SM (its
    // tensor-memory columns are then never contended)
    size_t smem = (size_t)stages * p.stage + extra;
    if (smem < 120 * 1024) smem = 120 * 1024;

    // Activations as (channel, x, y, image): one box of the chunk's KC
    // channels over the staged rows lands as nrows Wp rows of 2 KC bytes in
    // the swizzle of the descriptors; x starts at -8 so that the pad
    // positions come back zero, and rows outside the image are zero-filled.
    const CUtensorMapSwizzle sw = KC == 16 ? CU_TENSOR_MAP_SWIZZLE_32B
                                           : (KC == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
    CUtensorMap mx, mw;
    const cuuint64_t xdim[4] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t xstr[3] = {(cuuint64_t)ldx * 2, (cuuint64_t)W * ldx * 2, (cuuint64_t)H * W * ldx * 2};
    const cuuint32_t xbox[4] = {(cuuint32_t)KC, (cuuint32_t)p.Wp, (cuuint32_t)p.nrows, 1}, one4[4] = {1, 1, 1, 1};
    if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<uint16_t *>(x), xdim, xstr, xbox, one4,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return fail(-3, "activation tensor map");
    // Weights [Cout][9][Cin] as (input channel, output channel, tap): one box
    // of the chunk's channels lands tap after tap, each Cout rows of 2 KC
    // bytes.
    const cuuint64_t wdim[3] = {(cuuint64_t)Cin, (cuuint64_t)Cout, 9};
    const cuuint64_t wstr[2] = {(cuuint64_t)9 * Cin * 2, (cuuint64_t)Cin * 2};
    const cuuint32_t wbox[3] = {(cuuint32_t)KC, (cuuint32_t)Cout, 9};
    if (enc(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t *>(w), wdim, wstr, wbox, one4,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return fail(-3, "weight tensor map");

    using Kernel = void (*)(const Params, const CUtensorMap, const CUtensorMap);
    Kernel kern = nullptr;
    switch (KC * 8 + G) {
        case 16 * 8 + 1: kern = conv3x3_tc_kernel<16, 1>; break;
        case 16 * 8 + 2: kern = conv3x3_tc_kernel<16, 2>; break;
        case 16 * 8 + 4: kern = conv3x3_tc_kernel<16, 4>; break;
        case 32 * 8 + 1: kern = conv3x3_tc_kernel<32, 1>; break;
        case 32 * 8 + 2: kern = conv3x3_tc_kernel<32, 2>; break;
        case 32 * 8 + 4: kern = conv3x3_tc_kernel<32, 4>; break;
        case 64 * 8 + 1: kern = conv3x3_tc_kernel<64, 1>; break;
        case 64 * 8 + 2: kern = conv3x3_tc_kernel<64, 2>; break;
        case 64 * 8 + 4: kern = conv3x3_tc_kernel<64, 4>; break;
        default: return fail(-1, "tiles per block must be 1, 2 or 4");
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return fail(-3, cudaGetErrorString(e));
    // the blocks an SM holds must find their tensor-memory columns free, so
    // that no allocation waits
    if (per_sm < 1 || (uint32_t)per_sm * p.ncols > 512u) return fail(-1, "tensor memory would be oversubscribed");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(-3, "device query failed");
    const int units = B * p.supers;
    const int grid = units < sms * per_sm ? units : sms * per_sm;
    kern<<<grid, kThreads, smem, stream>>>(p, mx, mw);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(-3, cudaGetErrorString(e));
    return 0;
}

void inject_stall() { g_stall_next = true; }

int check(cudaStream_t stream) {
    int *status = status_word();
    if (!status) return -3;
    int word = 0;
    if (cudaMemcpyAsync(&word, status, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return -3;
    if (word) {
        cudaMemsetAsync(status, 0, sizeof(int), stream);
        return -4;
    }
    return 0;
}

}  // namespace lbmfvm_sg_tc
