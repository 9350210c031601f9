// Microbenchmarks for the roofline denominators of the on-chip levels:
// shared-memory read bandwidth, L2 read bandwidth and FP32 FMA rate of the
// running GPU.  The projector kernels are bound on chip (their operands come
// from shared memory and L1, their arithmetic is FP32 FMA), so their roofline
// needs these peaks next to the measured HBM bandwidth.  Each kernel does a
// fixed, bounded amount of work and writes one value per thread to a sink so
// that none of it can be removed.
#include "lt_host.h"
#include "lt_peaks.h"

namespace {

constexpr int kThreads = 256;
constexpr int kSmemWords = 2048;   // 16-byte words: 32 KiB per CTA

// Every thread reads 8 16-byte words per round; the 8 lanes of each quarter
// warp read 128 contiguous bytes, so every load is one conflict-free
// wavefront per quarter warp.  The round offset moves the addresses so that
// no load is loop-invariant.
__global__ void __launch_bounds__(kThreads) smem_read_kernel(float* __restrict__ sink, int reps) {
  __shared__ float4 buf[kSmemWords];
  for (int i = threadIdx.x; i < kSmemWords; i += kThreads)
    buf[i] = make_float4((float)i, (float)(i + 1), (float)(i + 2), (float)(i + 3));
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int r = 0; r < reps; ++r) {
    const int base = threadIdx.x + 32 * r;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float4 v = buf[(base + kThreads * j) & (kSmemWords - 1)];
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
  }
  sink[blockIdx.x * kThreads + threadIdx.x] = acc.x + acc.y + acc.z + acc.w;
}

// Grid-stride reads of an L2-resident buffer with L1-bypassing 16-byte
// loads, four independent loads in flight per thread.
__global__ void __launch_bounds__(kThreads) l2_read_kernel(const float4* __restrict__ buf, long long n16,
                                                           float* __restrict__ sink, int reps) {
  const long long stride = (long long)gridDim.x * kThreads;
  const long long t0 = (long long)blockIdx.x * kThreads + threadIdx.x;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int r = 0; r < reps; ++r) {
    long long i = t0;
    for (; i + 3 * stride < n16; i += 4 * stride) {
      const float4 a = __ldcg(buf + i);
      const float4 b = __ldcg(buf + i + stride);
      const float4 c = __ldcg(buf + i + 2 * stride);
      const float4 d = __ldcg(buf + i + 3 * stride);
      acc.x += (a.x + b.x) + (c.x + d.x);
      acc.y += (a.y + b.y) + (c.y + d.y);
      acc.z += (a.z + b.z) + (c.z + d.z);
      acc.w += (a.w + b.w) + (c.w + d.w);
    }
    for (; i < n16; i += stride) {
      const float4 a = __ldcg(buf + i);
      acc.x += a.x;
      acc.y += a.y;
      acc.z += a.z;
      acc.w += a.w;
    }
  }
  sink[t0] = acc.x + acc.y + acc.z + acc.w;
}

// Eight independent FMA chains per thread; m and c come from the host so
// that nothing folds at compile time.
__global__ void __launch_bounds__(kThreads) fma_kernel(float* __restrict__ sink, int reps, float m, float c) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = (float)(threadIdx.x + k);
  for (int r = 0; r < reps; ++r) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

lt_status check(const void* sink, int ctas, int reps) {
  if (!sink) return lt::set_error(LT_EINVAL, "sink is NULL");
  if (ctas <= 0 || reps <= 0) return lt::set_error(LT_EINVAL, "ctas and reps must be positive");
  return LT_OK;
}

lt_status launched(const char* what) {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LT_OK : lt::cuda_error(e, what);
}

}  // namespace

extern "C" lt_status lt_peak_smem_read(float* sink, int32_t ctas, int32_t reps, void* stream, double* bytes) {
  lt::clear_error();
  lt_status s = check(sink, ctas, reps);
  if (s != LT_OK) return s;
  smem_read_kernel<<<ctas, kThreads, 0, (cudaStream_t)stream>>>(sink, reps);
  if (bytes) *bytes = (double)ctas * kThreads * 8.0 * 16.0 * reps;
  return launched("shared-memory read microbenchmark");
}

extern "C" lt_status lt_peak_l2_read(const void* buf, int64_t n16, float* sink, int32_t ctas, int32_t reps,
                                     void* stream, double* bytes) {
  lt::clear_error();
  lt_status s = check(sink, ctas, reps);
  if (s != LT_OK) return s;
  if (!buf || n16 <= 0) return lt::set_error(LT_EINVAL, "buffer is NULL or empty");
  if (reinterpret_cast<uintptr_t>(buf) % 16) return lt::set_error(LT_EINVAL, "buffer is not 16-byte aligned");
  l2_read_kernel<<<ctas, kThreads, 0, (cudaStream_t)stream>>>(static_cast<const float4*>(buf), n16, sink, reps);
  if (bytes) *bytes = (double)n16 * 16.0 * reps;
  return launched("L2 read microbenchmark");
}

extern "C" lt_status lt_peak_fp32_fma(float* sink, int32_t ctas, int32_t reps, void* stream, double* flops) {
  lt::clear_error();
  lt_status s = check(sink, ctas, reps);
  if (s != LT_OK) return s;
  fma_kernel<<<ctas, kThreads, 0, (cudaStream_t)stream>>>(sink, reps, 0.999999f, 1e-7f);
  if (flops) *flops = (double)ctas * kThreads * 8.0 * 2.0 * reps;
  return launched("FP32 FMA microbenchmark");
}
