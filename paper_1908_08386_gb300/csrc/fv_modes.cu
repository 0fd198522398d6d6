// Launchers of the energy-update options of the coupled step: QUICK face
// values in the fused TMA kernel, and the finite-volume sub-steps (velocity
// pass, sub-step passes, collision with the given temperature).  A
// translation unit of its own so that these instantiations (every storage
// type) compile beside the handle code.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace lbmfvm_fv {

using namespace lbmfvm_dev;

namespace {

template <class S>
using GQuick = typename TmaConfig<S, kTmaConfigFv>::G::template WithTHalo<2>;
template <class S>
using GGiven = typename TmaConfig<S, kTmaConfigFv>::G;

template <class S, class G, int MODE>
cudaError_t launch_mode(const TmaLaunch<S> &l) {
    if (l.blocks < 1) return cudaSuccess;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(l.blocks);
    lc.blockDim = dim3(G::BLOCK);
    lc.dynamicSmemBytes = G::SMEM_BYTES;
    lc.stream = l.stream;
    // programmatic stream serialisation, as for the central kernel: the
    // kernel waits for the previous grid before it touches the state
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, step_tma_kernel<S, G, MODE>, l.a, l.cavs, l.tiles, l.count, *l.map_f, *l.map_T,
                              *l.map_c, *l.map_fo, *l.map_To, l.ctr, l.ctr_next, l.nfix);
}

template <class S, class G, int MODE>
cudaError_t prepare_one(int *blocks) {
    auto kern = step_tma_kernel<S, G, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM_BYTES);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, G::BLOCK, G::SMEM_BYTES);
    return e;
}

// One block per tile (256 threads), at most this many blocks.
int helper_grid(int ntiles) {
    const int cap = 152 * 8;
    return ntiles < cap ? ntiles : cap;
}

}  // namespace

template <class S>
cudaError_t prepare_modes(int *blocks_quick, int *blocks_given) {
    cudaError_t e = prepare_one<S, GQuick<S>, FV_QUICK>(blocks_quick);
    if (e == cudaSuccess) e = prepare_one<S, GGiven<S>, FV_GIVEN>(blocks_given);
    return e;
}

template <class S>
cudaError_t launch_quick(const TmaLaunch<S> &l) {
    return launch_mode<S, GQuick<S>, FV_QUICK>(l);
}

template <class S>
cudaError_t launch_given(const TmaLaunch<S> &l) {
    return launch_mode<S, GGiven<S>, FV_GIVEN>(l);
}

template <class S>
cudaError_t launch_uv(const S *fin, long long plane, int pitch, int gnx, int gny, const TileHeader *tiles, int ntiles,
                      const CavityDesc *cavs, const uint8_t *code, typename Compute<S>::type *U,
                      typename Compute<S>::type *V, int tw, int th, cudaStream_t stream) {
    if (ntiles < 1) return cudaSuccess;
    uv_kernel<S><<<helper_grid(ntiles), 256, 0, stream>>>(fin, plane, pitch, gnx, gny, tiles, ntiles, cavs, code, U,
                                                           V, tw, th);
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_substep(bool quick, const C *T0, C *X, C *Y, const C *U, const C *V, const uint8_t *code,
                           const uint8_t *fflags, int pitch, int gnx, int gny, const TileHeader *tiles, int ntiles,
                           int tw, int th, int s, cudaStream_t stream) {
    if (ntiles < 1) return cudaSuccess;
    if (quick)
        fv_substep_kernel<C, true><<<helper_grid(ntiles), 256, 0, stream>>>(T0, X, Y, U, V, code, fflags, pitch, gnx,
                                                                            gny, tiles, ntiles, tw, th, s);
    else
        fv_substep_kernel<C, false><<<helper_grid(ntiles), 256, 0, stream>>>(T0, X, Y, U, V, code, fflags, pitch, gnx,
                                                                             gny, tiles, ntiles, tw, th, s);
    return cudaGetLastError();
}

#define LBMFVM_FV_INSTANTIATE(S)                                                                                     \
    template cudaError_t prepare_modes<S>(int *, int *);                                                             \
    template cudaError_t launch_quick<S>(const TmaLaunch<S> &);                                                      \
    template cudaError_t launch_given<S>(const TmaLaunch<S> &);                                                      \
    template cudaError_t launch_uv<S>(const S *, long long, int, int, int, const TileHeader *, int,                  \
                                      const CavityDesc *, const uint8_t *, Compute<S>::type *, Compute<S>::type *, \
                                      int, int, cudaStream_t);
LBMFVM_FV_INSTANTIATE(double)
LBMFVM_FV_INSTANTIATE(float)
LBMFVM_FV_INSTANTIATE(__half)
LBMFVM_FV_INSTANTIATE(__nv_bfloat16)
LBMFVM_FV_INSTANTIATE(dsf)
#undef LBMFVM_FV_INSTANTIATE

template cudaError_t launch_substep<float>(bool, const float *, float *, float *, const float *, const float *,
                                           const uint8_t *, const uint8_t *, int, int, int, const TileHeader *, int,
                                           int, int, int, cudaStream_t);
template cudaError_t launch_substep<double>(bool, const double *, double *, double *, const double *, const double *,
                                            const uint8_t *, const uint8_t *, int, int, int, const TileHeader *, int,
                                            int, int, int, cudaStream_t);
template cudaError_t launch_substep<dsf>(bool, const dsf *, dsf *, dsf *, const dsf *, const dsf *, const uint8_t *,
                                         const uint8_t *, int, int, int, const TileHeader *, int, int, int, int,
                                         cudaStream_t);

}  // namespace lbmfvm_fv
