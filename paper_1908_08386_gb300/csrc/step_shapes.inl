// Fused step kernels of every tile shape for the storage types this
// translation unit is compiled for (included by step_*.cu, one per storage
// type, so that the shapes compile in parallel).
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace lbmfvm_fv {

using namespace lbmfvm_dev;

namespace {

template <class S, int CFG>
cudaError_t prepare_cfg(TmaShape *shape, int *blocks_per_sm) {
    using G = typename TmaConfig<S, CFG>::G;
    shape->TW = G::TW;
    shape->TH = G::TH;
    shape->FW = G::FW;
    shape->FH = G::FH;
    shape->TWD = G::TWD;
    shape->THT = G::THT;
    shape->THT_QUICK = G::template WithTHalo<2>::THT;
    shape->CWD = G::CWD;
    shape->CHT = G::CHT;
    shape->STAGES = G::STAGES;
    shape->BLOCK = G::BLOCK;
    shape->SMEM = G::SMEM_BYTES;
    auto kern = step_tma_kernel<S, G>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM_BYTES);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, G::BLOCK, G::SMEM_BYTES);
    return e;
}

template <class S, int CFG>
cudaError_t launch_cfg(const TmaLaunch<S> &l) {
    using G = typename TmaConfig<S, CFG>::G;
    if (l.blocks < 1) return cudaSuccess;  // no active tile
    // launched with programmatic stream serialisation: a step overlaps its
    // launch and prologue with the previous step's last tiles (the kernel
    // waits for the previous grid before touching the state)
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(l.blocks);
    lc.blockDim = dim3(G::BLOCK);
    lc.dynamicSmemBytes = G::SMEM_BYTES;
    lc.stream = l.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, step_tma_kernel<S, G>, l.a, l.cavs, l.tiles, l.count, *l.map_f, *l.map_T,
                              *l.map_c, *l.map_fo, *l.map_To, l.ctr, l.ctr_next, l.nfix);
}

}  // namespace

template <class S>
cudaError_t tma_prepare(int cfg, TmaShape *shape, int *blocks_per_sm) {
    switch (cfg) {
        case 0: return prepare_cfg<S, 0>(shape, blocks_per_sm);
        case 1: return prepare_cfg<S, 1>(shape, blocks_per_sm);
        case 2: return prepare_cfg<S, 2>(shape, blocks_per_sm);
        case 3: return prepare_cfg<S, 3>(shape, blocks_per_sm);
        case 4: return prepare_cfg<S, 4>(shape, blocks_per_sm);
        case 5: return prepare_cfg<S, 5>(shape, blocks_per_sm);
    }
    return cudaErrorInvalidValue;
}

template <class S>
cudaError_t tma_launch(int cfg, const TmaLaunch<S> &l) {
    switch (cfg) {
        case 0: return launch_cfg<S, 0>(l);
        case 1: return launch_cfg<S, 1>(l);
        case 2: return launch_cfg<S, 2>(l);
        case 3: return launch_cfg<S, 3>(l);
        case 4: return launch_cfg<S, 4>(l);
        case 5: return launch_cfg<S, 5>(l);
    }
    return cudaErrorInvalidValue;
}

#define LBMFVM_STEP_INSTANTIATE(S)                                             \
    template cudaError_t tma_prepare<S>(int, TmaShape *, int *);               \
    template cudaError_t tma_launch<S>(int, const TmaLaunch<S> &);

}  // namespace lbmfvm_fv
