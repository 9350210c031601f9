// Host entry points of the tcgen05 convolution (lt_nn_tc.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lt {

// Shapes (and 16-byte aligned pointers) the tcgen05 kernel tiles exactly:
// W a multiple of 64, channel counts multiples of 16, and Ci == 16 with H a
// multiple of 4 (z-walking kernel) or H and D even (chunked kernel).
bool conv3d_tc_supported(const void* in, const void* w, const void* out_bf, int D, int H, int W, int Ci, int Co);

// Which tcgen05 kernel: the faster one for the shape, or one of the two.
enum { kTcBest = 0, kTcChunked = 1, kTcZWalk = 2 };
bool conv3d_tc_variant_supported(int variant, int D, int H, int Ci, int Co);

// Same operation and layouts as lt_nn_conv3d (shape already checked with
// conv3d_tc_supported / conv3d_tc_variant_supported).
cudaError_t launch_conv3d_tc(const uint16_t* in, const uint16_t* w, const float* b, uint16_t* out_bf, float* out_f,
                             int batch, int D, int H, int W, int Ci, int Co, int o_stride, int o_off, int relu,
                             int variant, cudaStream_t st);

// Test hook: with on != 0 the kernels issue no MMA (their waits run out after
// 4096 polls); on == 0 restores normal operation.  Synchronises the stream.
cudaError_t set_tc_stall(int on, cudaStream_t st);

// Reads and clears the device status word of the tcgen05 kernels (0, or
// LT_ETIMEOUT after a bounded wait gave up); synchronises the stream.
cudaError_t take_tc_status(int* status, cudaStream_t st);

}  // namespace lt
