// The tensor-core (tcgen05) 3x3 convolution of the warm-start surrogate,
// called by lbmfvm_sg_conv3x3 (same arguments and conventions as in
// include/surrogate.h).  g_req: 128-position tiles per block (a power of two
// up to the tensor memory's 512 columns), kc_req: input channels per
// pipeline stage (16, 32 or 64), s_req: pipeline stages; 0 = chosen from the
// shape.  Returns 0, -1
// (argument) or -3 (CUDA error), with the message in msg.
#ifndef LBMFVM_CONV_TC_H
#define LBMFVM_CONV_TC_H

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace lbmfvm_sg_tc {

int conv3x3(const uint16_t *x, int ldx, const uint16_t *w, const float *bias, uint16_t *y, int ldy,
            const uint16_t *m, int ldm, int B, int H, int W, int Cin, int Cout, int mode, cudaStream_t stream,
            char *msg, size_t msglen, int g_req = 0, int kc_req = 0, int s_req = 0);

// Synchronises the stream and reads the status word of the bounded waits:
// 0, -4 if a wait ran out since the last check (the word is cleared), -3 on a
// CUDA error.
int check(cudaStream_t stream);

// The next conv3x3 call's block 0 skips its first staged load, so that its
// bounded waits run out (a test of the failure path: nothing faults).
void inject_stall();

}  // namespace lbmfvm_sg_tc

#endif
