// 3x3 convolution of the warm-start surrogate on the fifth-generation tensor
// cores: tcgen05.mma (BF16 x BF16, FP32 accumulation in tensor memory),
// operands staged in shared memory by TMA, results read back with tcgen05.ld.
//
// Implicit GEMM.  A tile is M = 128 consecutive output positions of one image
// and all N = Cout output channels; K runs over the nine taps and the input
// channels in chunks of 16.  Positions are counted in a padded row
// layout of Wp = W + 8 pixels per row: image pixel (y, x) sits at position
// q = (y + 1) Wp + 8 + x, and the eight positions before each row's pixels
// hold zeros, so that the left neighbour of x = 0 (q - 1) and the right
// neighbour of x = W - 1 (the next row's position 0) read zero padding.  Tap
// (ky, kx) of output position q reads input position q + (ky - 1) Wp + kx - 1,
// so for a tile of 128 consecutive positions each tap's A operand is again a
// run of 128 consecutive positions: the shared-memory descriptor of a tap is
// the staged rows' base shifted by 16 bytes per position, with no re-staging.
//
// Shared-memory operand layout (no swizzle, K-major): channels in planes of
// eight; within a plane one 16-byte row per position (A) or per output
// channel (B), consecutive, so that eight rows form one 128-byte core matrix
// (stride between eight-row groups 128 bytes) and the second plane of a
// 16-channel chunk lies one plane further (the K-direction stride).  One TMA
// box per stage brings both planes of the staged rows, each row from x = -8
// (the pad positions, which the out-of-bounds fill makes zero) to W - 1, rows
// outside the image zero-filled; a second box brings the chunk's two planes
// of weights for all nine taps.
//
// A block holds G tiles of 128 consecutive positions, each with its own
// accumulator in tensor memory: the staged rows and weights of a chunk serve
// all of them (the halo rows and the weights are staged once per G tiles).
//
// Pipeline: thread 0 issues the two TMA loads of a stage on the stage's full
// barrier, the 9 G MMAs of a chunk once it has landed, and a tcgen05.commit
// on the stage's empty barrier; a stage is refilled once the MMAs of the chunk
// before it have completed, so that the tensor pipe always has the current
// chunk queued.  After the last chunk a commit on the done barrier releases
// the epilogue: each warp reads its 32 TMEM lanes (positions) of every
// accumulator, adds the bias
// and applies the activation (or multiplies by the activation's derivative),
// and stores BF16.  Every wait is bounded (1 s); a wait that runs out sets a
// device status word, and the block drains what it issued before leaving.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>

#include "conv_tc.h"
#include "surrogate.h"

namespace lbmfvm_sg_tc {

namespace {

using bf16 = __nv_bfloat16;

constexpr int kM = 128;        // output positions per block (TMEM lanes)
constexpr int kThreads = 128;  // four warps; warp w reads TMEM lanes 32w..32w+31
constexpr int kPad = 8;        // zero positions before each padded row (128 bytes per plane)
constexpr int kMaxStages = 8;
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr float kLeak = 1.0f / 16.0f;

struct Params {
    const float *bias;
    bf16 *y;
    const bf16 *m;
    int *status;
    int ldy, ldm, H, W, Cout, mode;
    int Wp;           // padded row length in positions
    int tiles;        // tiles of 128 positions per image
    int G;            // tiles per block, each with its own accumulator
    int supers;       // blocks per image: ceil(tiles / G)
    uint32_t acc;     // TMEM columns between accumulators
    int nch;          // 16-channel chunks of the input
    int stages;
    int nrows;        // padded rows staged per tile (the largest any tile needs)
    uint32_t a_plane; // bytes of one 8-channel plane of the staged rows
    uint32_t b_plane; // bytes of one 8-channel plane of one tap's weights (Cout x 16)
    uint32_t stage;   // bytes of one stage: two A planes and 18 B planes
    uint32_t ncols;   // TMEM columns allocated (G * acc)
    uint32_t idesc;   // instruction descriptor
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

__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            int c4, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(saddr(bar))
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
// Shared-memory matrix descriptor, no swizzle: start address, the stride
// between the two 8-channel planes of a K chunk (leading byte offset) and the
// stride between groups of eight rows (stride byte offset, 128 bytes).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((128u >> 4) & 0x3FFFu) << 32) | (1ull << 46);
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

__global__ void __launch_bounds__(kThreads, 1)
    conv3x3_tc_kernel(const Params p, const __grid_constant__ CUtensorMap map_x,
                      const __grid_constant__ CUtensorMap map_w) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], done;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.x / p.supers, t0 = (blockIdx.x % p.supers) * p.G;
    const int g_n = p.tiles - t0 < p.G ? p.tiles - t0 : p.G;  // tiles of this block
    const int q0 = p.Wp + kPad + kM * t0;  // first output position of the block
    const int ry0 = first_row(q0, p.Wp);
    uint8_t *base = smem + ((1024 - (saddr(smem) & 1023u)) & 1023u);

    if (tid == 0) {
        for (int s = 0; s < p.stages; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                     "r"(p.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_base;

    if (tid == 0) {
        auto load = [&](int c) {
            const int s = c % p.stages;
            uint8_t *st = base + (size_t)s * p.stage;
            mbar_expect_tx(&full[s], p.stage);
            // both 8-channel planes of the staged rows, each row from x = -8
            // (the pad positions, zero-filled) to W - 1
            tma_load_5d(st, &map_x, 0, -kPad, ry0 - 1, 2 * c, b, &full[s]);
            // both planes of the chunk's weights for all nine taps
            tma_load_4d(st + 2 * p.a_plane, &map_w, 0, 0, 2 * c, 0, &full[s]);
        };
        const int pre = p.nch < p.stages ? p.nch : p.stages;
        for (int c = 0; c < pre; c++) load(c);
        bool ok = true;
        int issued = 0;  // chunks whose MMAs were issued
        for (int c = 0; c < p.nch && ok; c++) {
            const int s = c % p.stages;
            if (!(ok = mbar_wait(&full[s], (uint32_t)(c / p.stages) & 1u))) break;
            tc_after_sync();
            const uint32_t st = saddr(base + (size_t)s * p.stage);
#pragma unroll
            for (int tap = 0; tap < 9; tap++) {
                const int off = (tap / 3 - 1) * p.Wp + (tap % 3 - 1);
                const uint64_t bd = sdesc(st + 2u * p.a_plane + (uint32_t)tap * 2u * p.b_plane, p.b_plane);
                for (int g = 0; g < g_n; g++) {
                    const uint32_t a = st + (uint32_t)(q0 + kM * g + off - ry0 * p.Wp) * 16u;
                    mma(tmem + (uint32_t)g * p.acc, sdesc(a, p.a_plane), bd, p.idesc, (c | tap) != 0);
                }
            }
            mma_commit(&empty[s]);
            issued = c + 1;
            // refill the stage of the previous chunk once its MMAs are done
            const int cr = c - 1 + p.stages;
            if (c >= 1 && cr < p.nch) {
                const int sp = (c - 1) % p.stages;
                if (!(ok = mbar_wait(&empty[sp], (uint32_t)((c - 1) / p.stages) & 1u))) break;
                load(cr);
            }
        }
        mma_commit(&done);
        if (!ok) {
            failed = 1;
            atomicExch(p.status, 1);
            // drain: the loads issued for chunks past the last waited one
            const int loaded = p.nch < issued - 1 + p.stages ? p.nch : issued - 1 + p.stages;
            for (int c = issued; c < loaded; c++) mbar_wait(&full[c % p.stages], (uint32_t)(c / p.stages) & 1u);
        }
    }
    // every thread waits for the accumulator
    const bool ready = mbar_wait(&done, 0);
    tc_after_sync();
    for (int g = 0; g < g_n && ready && !failed; g++) {
        const int q = q0 + kM * g + warp * 32 + lane;
        const int yy = q / p.Wp - 1, xx = q % p.Wp - kPad;
        const bool valid = yy >= 0 && yy < p.H && xx >= 0 && xx < p.W;
        const long long pix = ((long long)b * p.H + yy) * p.W + xx;
        for (int j = 0; j < p.Cout / 16; j++) {
            uint32_t r[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)g * p.acc + (uint32_t)(16 * j), r);
            if (!valid) continue;
            float v[16];
#pragma unroll
            for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
            const int co = 16 * j;
            if (p.mode == LBMFVM_SG_DLEAKY) {
                const uint4 *mm = reinterpret_cast<const uint4 *>(p.m + pix * p.ldm + co);
                const uint4 m0 = mm[0], m1 = mm[1];
                const bf16 *mb0 = reinterpret_cast<const bf16 *>(&m0);
                const bf16 *mb1 = reinterpret_cast<const bf16 *>(&m1);
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    v[i] *= dleaky(__bfloat162float(mb0[i]));
                    v[8 + i] *= dleaky(__bfloat162float(mb1[i]));
                }
            } else {
                if (p.bias) {
#pragma unroll
                    for (int i = 0; i < 16; i++) v[i] += p.bias[co + i];
                }
                if (p.mode == LBMFVM_SG_LEAKY) {
#pragma unroll
                    for (int i = 0; i < 16; i++) v[i] = leaky(v[i]);
                }
            }
            uint4 o[2];
            __nv_bfloat162 *ob = reinterpret_cast<__nv_bfloat162 *>(o);
#pragma unroll
            for (int i = 0; i < 8; i++) ob[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
            uint4 *dst = reinterpret_cast<uint4 *>(p.y + pix * p.ldy + co);
            dst[0] = o[0];
            dst[1] = o[1];
        }
    }
    if (!ready && tid == 0) atomicExch(p.status, 1);
    tc_before_sync();
    __syncthreads();
    if (warp == 0) {
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

int *status_word() {
    static int *word = nullptr;
    if (!word && cudaMalloc(&word, sizeof(int)) == cudaSuccess) cudaMemset(word, 0, sizeof(int));
    return word;
}

}  // namespace

int conv3x3(const uint16_t *x, int ldx, const uint16_t *w, const float *bias, uint16_t *y, int ldy,
            const uint16_t *m, int ldm, int B, int H, int W, int Cin, int Cout, int mode, cudaStream_t stream,
            char *msg, size_t msglen, int g_req) {
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
    p.ldy = ldy;
    p.ldm = ldm;
    p.H = H;
    p.W = W;
    p.Cout = Cout;
    p.mode = mode;
    p.Wp = W + kPad;
    const int q_first = p.Wp + kPad, q_end = H * p.Wp + kPad + W;  // output positions [q_first, q_end)
    p.tiles = (q_end - q_first + kM - 1) / kM;
    p.nch = Cin / 16;
    p.b_plane = (uint32_t)Cout * 16u;
    p.acc = 32;
    while ((int)p.acc < Cout) p.acc <<= 1;
    // instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B,
    // both K-major, N = Cout, M = 128
    p.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Cout >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
    const size_t extra = 1024;  // alignment of the stage area
    const size_t half = 110 * 1024, whole = 220 * 1024;
    // Tiles per block: a block stages its rows and the chunk's weights once
    // for all its tiles.
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
    auto stage_for = [&](int G) { return 2u * (uint32_t)rows_for(G) * p.Wp * 16u + 18u * p.b_plane; };
    int G = g_req;
    if (G <= 0) {
        // measured on the network's layers: four tiles per block while the
        // tensor memory holds them (two of 160 or 256 channels), fewer when a
        // stage would not fit twice
        G = (int)(512 / p.acc) < 4 ? (int)(512 / p.acc) : 4;
        while (G > 1 && (G / 2 >= p.tiles || (whole - extra) / stage_for(G) < 2)) G >>= 1;
    }
    if (G < 1 || (uint32_t)G * p.acc > 512u) return fail(-1, "tiles per block exceed the tensor memory");
    p.G = G;
    p.supers = (p.tiles + G - 1) / G;
    p.ncols = (uint32_t)G * p.acc;
    p.nrows = rows_for(G);
    p.a_plane = (uint32_t)p.nrows * p.Wp * 16u;
    p.stage = 2u * p.a_plane + 18u * p.b_plane;
    // stages: two blocks per SM when their columns fit the tensor memory and
    // two or more stages fit in half the shared memory, else one block with
    // as many as fit
    int stages = p.ncols <= 256u ? (int)((half - extra) / p.stage) : 0;
    if (stages < 2) stages = (int)((whole - extra) / p.stage);
    if (stages > kMaxStages) stages = kMaxStages;
    if (stages < 2) return fail(-1, "a pipeline stage does not fit twice in shared memory");
    p.stages = stages;
    const size_t smem = (size_t)stages * p.stage + extra;

    // Activations as (8 channels, x, y, plane of 8 channels, image): one box
    // of both planes of a chunk over the staged rows lands plane after plane,
    // each a run of positions; x starts at -8 so that the pad positions come
    // back zero, and rows outside the image are zero-filled.
    CUtensorMap mx, mw;
    const cuuint64_t xdim[5] = {8, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)(Cin / 8), (cuuint64_t)B};
    const cuuint64_t xstr[4] = {(cuuint64_t)ldx * 2, (cuuint64_t)W * ldx * 2, 16, (cuuint64_t)H * W * ldx * 2};
    const cuuint32_t xbox[5] = {8, (cuuint32_t)p.Wp, (cuuint32_t)p.nrows, 2, 1}, one5[5] = {1, 1, 1, 1, 1};
    if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<uint16_t *>(x), xdim, xstr, xbox, one5,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return fail(-3, "activation tensor map");
    // Weights [Cout][9][Cin] as (8 channels, output channel, plane, tap): one
    // box of a chunk's two planes for all taps lands tap-plane after
    // tap-plane, each Cout rows of 16 bytes.
    const cuuint64_t wdim[4] = {8, (cuuint64_t)Cout, (cuuint64_t)(Cin / 8), 9};
    const cuuint64_t wstr[3] = {(cuuint64_t)9 * Cin * 2, 16, (cuuint64_t)Cin * 2};
    const cuuint32_t wbox[4] = {8, (cuuint32_t)Cout, 2, 9};
    if (enc(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<uint16_t *>(w), wdim, wstr, wbox, one5,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return fail(-3, "weight tensor map");

    cudaError_t e = cudaFuncSetAttribute(conv3x3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv3x3_tc_kernel, kThreads, smem);
    if (e != cudaSuccess) return fail(-3, cudaGetErrorString(e));
    // the blocks an SM holds must find their tensor-memory columns free, so
    // that no allocation waits
    if (per_sm < 1 || (uint32_t)per_sm * p.ncols > 512u) return fail(-1, "tensor memory would be oversubscribed");
    conv3x3_tc_kernel<<<B * p.supers, kThreads, smem, stream>>>(p, mx, mw);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(-3, cudaGetErrorString(e));
    return 0;
}

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
