// 3x3x3 convolution of the warm-start U-Net on the fifth-generation tensor
// cores (tcgen05): bfloat16 operands in shared memory, float32 accumulators
// in tensor memory (TMEM).  Used for volumes whose x extent is a multiple of
// 64 (the full- and half-resolution levels of the network), the warp-level
// MMA kernel of lt_nn.cu for the rest.
//
// Chunked kernel: a CTA owns a TM (x) x 2 (y) x 2 (z) block of output voxels -- four tiles,
// one x run of TM = 128 (or 64) voxels each, one M = 128 MMA row per voxel
// (rows past TM unused) -- and N = 16, 32 or 48 output channels.  Per
// chunk of 16 input channels it stages the input halo (130 x 4 x 4 voxels)
// and the 27 taps' weights in shared memory, in the canonical K-major layout
// without swizzle: 8 (voxels or output channels) x 8 channels of 16 bytes
// form one 128-byte core matrix, consecutive x voxels are 16 bytes apart.  A
// tap (dz, dy, dx) of a tile is then a descriptor whose start moves by whole
// voxels, and one thread issues the 4 x 27 MMAs (M 128, N, K 16) of a chunk
// back to back into the tile's TMEM columns; a commit to an mbarrier tells the
// CTA when the tensor core is done with the staged data.  The epilogue reads
// the accumulators with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31, i.e.
// x voxels 32w..32w+31 of every tile), adds the bias, applies ReLU and stores.
// That is the chunked kernel; layers with 16 input channels and large grids
// take the z-walking kernel below (a CTA walks 8 slices in z over a ring of
// three input planes, so each plane is staged once per CTA and staging
// overlaps the other CTA's MMAs).
//
// Every wait on the mbarrier is bounded; a wait that gives up records
// LT_ETIMEOUT in a device status word (lt_nn_device_status), skips the rest
// of the CTA's work and still frees its TMEM.
#include <cuda_bf16.h>

#include <cstdint>

#include "lt.h"
#include "lt_host.h"
#include "lt_nn.h"
#include "lt_nn_tc.h"
#include "lt_async.cuh"

namespace lt {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int TC_MMA_M = 128;              // rows of every MMA (TMEM lanes)
constexpr int TC_RY = 2, TC_RZ = 2;        // output rows per CTA
constexpr int TC_TILES = TC_RY * TC_RZ;
constexpr int TC_HY = TC_RY + 2, TC_HZ = TC_RZ + 2;
constexpr int TC_THREADS = 128;            // 4 warps = the 128 TMEM lanes
constexpr long long kWaitLimit = 1LL << 24;   // mbarrier polls (with 64 ns back-off) before giving up

// Halo geometry for x runs of TM voxels (128, or 64 for the half-resolution
// level).  An MMA always reads 128 rows of A: with TM = 64 the upper 64 rows
// run on into the next halo row (their accumulator rows are never stored,
// and row m of the product depends on row m of A alone), and past the last
// row into TAIL bytes kept inside the allocation.  The last A start is two
// voxels into the last (hz, hy, channel group 0) row, so the furthest byte
// read is HALO - ROW + 2 * 16 + 128 * 16 - 1 = HALO + TAIL - 1.
template <int TM>
struct TcGeom {
  static constexpr int HX = TM + 2;
  static constexpr int ROW = HX * 16;               // bytes of one (hz, hy, channel group) halo row
  static constexpr int HALO = TC_HZ * TC_HY * 2 * ROW;
  static constexpr int TAIL = (TC_MMA_M - TM) * 16;
  static_assert(TM == 128 || TM == 64, "x run");
};

template <int N>
__host__ __device__ constexpr int tc_weight_bytes() { return 27 * 2 * N * 16; }
template <int TM, int N>
__host__ __device__ constexpr int tc_smem_bytes() {
  return TcGeom<TM>::HALO + TcGeom<TM>::TAIL + tc_weight_bytes<N>() + 16;
}

__device__ int g_tc_status;   // LT_ETIMEOUT after a bounded wait gave up
// Test hook (lt_nn_test_stall_tensor_core, test builds only): no MMA is
// issued, so every wait runs out, after g_tc_wait_limit polls.
#ifdef LT_TEST_HOOKS
__device__ int g_tc_stall = 0;
#define LT_TC_STALL (g_tc_stall != 0)
#else
#define LT_TC_STALL false
#endif
__device__ long long g_tc_wait_limit = kWaitLimit;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K)
// byte offset between core matrices, stride (M/N) byte offset between 8-row
// groups, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(lbo >> 4) << 16) |
         (static_cast<uint64_t>(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: float32 accumulator, bfloat16 A and B,
// both K-major, N >> 3 and M >> 4 in their fields.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait for phase `parity` of the mbarrier.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long limit = g_tc_wait_limit;
  for (long long i = 0; i < limit; ++i) {
    if (mbar_test(bar, parity)) return true;
    __nanosleep(64);
  }
  return false;
}

// D[tmem] (+)= A[smem] x B[smem]^T, one M x N x 16 bfloat16 step.
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// The mbarrier completes a phase once every MMA this thread issued is done.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// 16 consecutive float32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int TM, int N>
__global__ void __launch_bounds__(TC_THREADS, 1)
conv3d_tc_kernel(const bf16* __restrict__ in, const bf16* __restrict__ w, const float* __restrict__ bias,
                 bf16* __restrict__ out_bf, float* __restrict__ out_f, int D, int H, int W, int Ci, int Co,
                 int o_stride, int o_off, int relu, int tiles_x, int tiles_y, int vec_store) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* halo = tc_smem;                                   // [hz][hy][cg][hx][8] bf16
  using G = TcGeom<TM>;
  unsigned char* wts = tc_smem + G::HALO + G::TAIL;               // [tap][cg][co][8] bf16
  uint64_t* mbar = reinterpret_cast<uint64_t*>(wts + tc_weight_bytes<N>());
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  // TMEM columns: TC_TILES x N rounded up to a power of two (64, 128, 256)
  constexpr uint32_t kCols = TC_TILES * N <= 64 ? 64 : TC_TILES * N <= 128 ? 128 : 256;
  static_assert(N % 16 == 0 && N <= 64 && TC_TILES * N <= 256, "tcgen05 tile width");
  constexpr uint32_t kIdesc = mma_idesc(TC_MMA_M, N);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bx = blockIdx.x % tiles_x;
  const int rest = blockIdx.x / tiles_x;
  const int by = rest % tiles_y, bz = rest / tiles_y;
  const int x0 = bx * TM, y0 = by * TC_RY, z0 = bz * TC_RZ;
  const int n0 = blockIdx.y * N;
  const int b = blockIdx.z;
  const long long V = (long long)D * H * W;
  const bf16* inb = in + (long long)b * V * Ci;
  const uint32_t bar = smem_u32(mbar);

  if (warp == 0) tmem_alloc(smem_u32(tslot), kCols);
  if (tid == 0) mbar_init(bar);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;

  const int chunks = Ci / 16;
  const bool stall = LT_TC_STALL;
  bool ok = true;
  for (int c = 0; c < chunks && ok; ++c) {
    if (c > 0) {   // the tensor core has finished reading the previous chunk's tiles
      ok = __syncthreads_and(mbar_wait(bar, (c - 1) & 1));
      if (!ok) break;
    }
    // halo (zero outside the volume) and weights of this chunk, all copies in flight at once
    for (int t = tid; t < TC_HZ * TC_HY * G::HX * 2; t += TC_THREADS) {
      const int cg = t & 1, v = t >> 1;
      const int hx = v % G::HX, r = v / G::HX;
      const int hy = r % TC_HY, hz = r / TC_HY;
      const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
      const bool inside = gx >= 0 && gx < W && gy >= 0 && gy < H && gz >= 0 && gz < D;
      const bf16* src = inside ? inb + (((long long)gz * H + gy) * W + gx) * Ci + c * 16 + cg * 8 : inb;
      cp_async16(smem_u32(halo + ((hz * TC_HY + hy) * 2 + cg) * G::ROW + hx * 16), src, inside);
    }
    for (int t = tid; t < 27 * 2 * N; t += TC_THREADS) {
      const int co = t % N, r = t / N;
      const int cg = r & 1, tap = r >> 1;
      const bool inside = n0 + co < Co;
      const bf16* src = inside ? w + ((long long)(n0 + co) * 27 + tap) * Ci + c * 16 + cg * 8 : w;
      cp_async16(smem_u32(wts + ((tap * 2 + cg) * N + co) * 16), src, inside);
    }
    cp_async_wait_all();
    fence_async_smem();   // make these writes visible to the tensor core (async proxy)
    __syncthreads();
    if (tid == 0 && !stall) {
      tc_fence_after();
      // Descriptors differ only in the start-address field (bits 0-13, in
      // 16-byte units; every address here is below 256 KB), so each MMA's is
      // a base descriptor plus a compile-time offset.
      const uint64_t a0 = smem_desc(smem_u32(halo), G::ROW, 128);
      const uint64_t b0 = smem_desc(smem_u32(wts), N * 16, 128);
      // taps outer, tiles inner: consecutive MMAs go to different
      // accumulators and do not wait for one another's results
#pragma unroll
      for (int tap = 0; tap < 27; ++tap) {
#pragma unroll
        for (int m = 0; m < TC_TILES; ++m) {
          const int ry = m % TC_RY, rz = m / TC_RY;
          const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
          const uint32_t a_off = ((rz + dz + 1) * TC_HY + (ry + dy + 1)) * 2 * G::ROW + (dx + 1) * 16;
          const uint32_t b_off = tap * 2 * N * 16;
          mma_bf16(tbase + m * N, a0 + (a_off >> 4), b0 + (b_off >> 4), kIdesc, (c > 0 || tap > 0) ? 1u : 0u);
        }
      }
      mma_commit(bar);
    }
  }
  if (ok) ok = __syncthreads_and(mbar_wait(bar, (chunks - 1) & 1));
  tc_fence_after();
  if (ok && warp * 32 < TM) {   // warps past TM hold the unused accumulator rows
    for (int m = 0; m < TC_TILES; ++m) {
      const int ry = m % TC_RY, rz = m / TC_RY;
      const int gx = x0 + warp * 32 + lane, gy = y0 + ry, gz = z0 + rz;
      const long long o = ((long long)b * V + ((long long)gz * H + gy) * W + gx) * o_stride + o_off + n0;
#pragma unroll
      for (int j = 0; j < N / 16; ++j) {
        float v[16];
        tmem_ld16(tbase + (static_cast<uint32_t>(warp * 32) << 16) + m * N + j * 16, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          v[i] += bias ? __ldg(bias + n0 + j * 16 + i) : 0.0f;
          if (relu) v[i] = fmaxf(v[i], 0.0f);
        }
        if (out_bf) {
          if (vec_store) {
            uint4 p[2];
            __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(p);
#pragma unroll
            for (int i = 0; i < 8; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
            uint4* dst = reinterpret_cast<uint4*>(out_bf + o + j * 16);
            dst[0] = p[0];
            dst[1] = p[1];
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) out_bf[o + j * 16 + i] = __float2bfloat16_rn(v[i]);
          }
        }
        if (out_f) {
#pragma unroll
          for (int i = 0; i < 16; ++i) out_f[o + j * 16 + i] = v[i];
        }
      }
    }
  }
  if (!ok && tid == 0) {
    atomicExch(&g_tc_status, (int)LT_ETIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, kCols);
}

// z-walking variant for 16 input channels (one channel chunk).  A CTA owns a
// TM (x) x 4 (y) column of output rows and walks ZW_SLICES slices in z.  The
// input halo lives in a ring of three planes of 6 (y) rows in shared memory;
// output slice z needs planes z - 1, z, z + 1.  Per slice: wait for its MMAs,
// load plane z + 2 into the slot of plane z - 1 (now unread) while the
// epilogue drains the accumulators, then issue the next slice's MMAs.  Each
// input plane is staged once per CTA, 6 rows for 4 output rows (1.9x over
// ZW_SLICES = 8 slices, against 4x for the chunked kernel), and two CTAs per
// SM overlap one's staging and epilogue with the other's MMAs.
constexpr int ZW_RY = 4, ZW_HY = ZW_RY + 2;
constexpr int ZW_SLICES = 8;

template <int TM>
struct ZwGeom {
  static constexpr int HX = TM + 2;
  static constexpr int ROW = HX * 16;                   // one (hy, channel group) row of a plane
  static constexpr int PLANE = ZW_HY * 2 * ROW;
  static constexpr int RING = 3 * PLANE;
  // the last A start is two voxels into the last plane's last (hy, cg 0) row:
  // furthest byte RING - ROW + 32 + 2048 - 1 = RING + TAIL - 1
  static constexpr int TAIL = (TC_MMA_M - TM) * 16;
};
template <int TM, int N>
__host__ __device__ constexpr int zw_smem_bytes() {
  return ZwGeom<TM>::RING + ZwGeom<TM>::TAIL + tc_weight_bytes<N>() + 16;
}

template <int TM, int N>
__global__ void __launch_bounds__(TC_THREADS, 1)
conv3d_tc_zwalk_kernel(const bf16* __restrict__ in, const bf16* __restrict__ w, const float* __restrict__ bias,
                       bf16* __restrict__ out_bf, float* __restrict__ out_f, int D, int H, int W, int Co,
                       int o_stride, int o_off, int relu, int tiles_x, int tiles_y, int vec_store) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  using G = ZwGeom<TM>;
  unsigned char* ring = tc_smem;                                     // [slot][hy][cg][hx][8] bf16
  unsigned char* wts = tc_smem + G::RING + G::TAIL;                  // [tap][cg][co][8] bf16
  uint64_t* mbar = reinterpret_cast<uint64_t*>(wts + tc_weight_bytes<N>());
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  constexpr uint32_t kCols = ZW_RY * N <= 64 ? 64 : ZW_RY * N <= 128 ? 128 : 256;
  static_assert(N % 16 == 0 && ZW_RY * N <= 256, "tcgen05 tile width");
  constexpr uint32_t kIdesc = mma_idesc(TC_MMA_M, N);
  constexpr int Ci = 16;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bx = blockIdx.x % tiles_x;
  const int rest = blockIdx.x / tiles_x;
  const int by = rest % tiles_y, bz = rest / tiles_y;
  const int x0 = bx * TM, y0 = by * ZW_RY, z0 = bz * ZW_SLICES;
  const int nsl = min(ZW_SLICES, D - z0);
  const int n0 = blockIdx.y * N;
  const int b = blockIdx.z;
  const long long V = (long long)D * H * W;
  const bf16* inb = in + (long long)b * V * Ci;
  const uint32_t bar = smem_u32(mbar);

  // plane of slice kz (zero outside the volume) into ring slot `slot`
  const auto stage_plane = [&](int kz, int slot) {
    unsigned char* dst = ring + slot * G::PLANE;
    for (int t = tid; t < ZW_HY * G::HX * 2; t += TC_THREADS) {
      const int cg = t & 1, v = t >> 1;
      const int hx = v % G::HX, hy = v / G::HX;
      const int gx = x0 + hx - 1, gy = y0 + hy - 1;
      const bool inside = gx >= 0 && gx < W && gy >= 0 && gy < H && kz >= 0 && kz < D;
      const bf16* src = inside ? inb + (((long long)kz * H + gy) * W + gx) * Ci + cg * 8 : inb;
      cp_async16(smem_u32(dst + (hy * 2 + cg) * G::ROW + hx * 16), src, inside);
    }
  };
  // ring slot of plane kz: planes z0 - 1, z0, z0 + 1, ... take slots 0, 1, 2, 0, ...
  const auto slot_of = [&](int kz) { return (kz - z0 + 1) % 3; };

  if (warp == 0) tmem_alloc(smem_u32(tslot), kCols);
  if (tid == 0) mbar_init(bar);
  for (int t = tid; t < 27 * 2 * N; t += TC_THREADS) {
    const int co = t % N, r = t / N;
    const int cg = r & 1, tap = r >> 1;
    const bool inside = n0 + co < Co;
    const bf16* src = inside ? w + ((long long)(n0 + co) * 27 + tap) * Ci + cg * 8 : w;
    cp_async16(smem_u32(wts + ((tap * 2 + cg) * N + co) * 16), src, inside);
  }
  stage_plane(z0 - 1, 0);
  stage_plane(z0, 1);
  stage_plane(z0 + 1, 2);
  cp_async_wait_all();
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;

  // issue the 27 x ZW_RY MMAs of slice kz (one thread) and commit them
  const auto issue = [&](int kz) {
    const uint64_t a0 = smem_desc(smem_u32(ring), G::ROW, 128);
    const uint64_t b0 = smem_desc(smem_u32(wts), N * 16, 128);
    const uint32_t s0 = slot_of(kz - 1) * G::PLANE, s1 = slot_of(kz) * G::PLANE, s2 = slot_of(kz + 1) * G::PLANE;
#pragma unroll
    for (int tap = 0; tap < 27; ++tap) {
#pragma unroll
      for (int ry = 0; ry < ZW_RY; ++ry) {
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        const uint32_t sb = dz < 0 ? s0 : dz == 0 ? s1 : s2;
        const uint32_t a_off = sb + ((ry + dy + 1) * 2) * G::ROW + (dx + 1) * 16;
        const uint32_t b_off = tap * 2 * N * 16;
        mma_bf16(tbase + ry * N, a0 + (a_off >> 4), b0 + (b_off >> 4), kIdesc, tap > 0 ? 1u : 0u);
      }
    }
    mma_commit(bar);
  };
  const bool stall = LT_TC_STALL;
  if (tid == 0 && !stall) issue(z0);

  bool ok = true;
  for (int s = 0; s < nsl; ++s) {
    const int z = z0 + s;
    ok = __syncthreads_and(mbar_wait(bar, s & 1));   // slice z's MMAs are done
    if (!ok) break;
    tc_fence_after();
    if (s + 1 < nsl) stage_plane(z + 2, slot_of(z + 2));   // the slot of plane z - 1, no longer read
    if (warp * 32 < TM) {   // warps past TM hold the unused accumulator rows
      for (int ry = 0; ry < ZW_RY; ++ry) {
        const int gx = x0 + warp * 32 + lane, gy = y0 + ry;
        const long long o = ((long long)b * V + ((long long)z * H + gy) * W + gx) * o_stride + o_off + n0;
#pragma unroll
        for (int j = 0; j < N / 16; ++j) {
          float v[16];
          tmem_ld16(tbase + (static_cast<uint32_t>(warp * 32) << 16) + ry * N + j * 16, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            v[i] += bias ? __ldg(bias + n0 + j * 16 + i) : 0.0f;
            if (relu) v[i] = fmaxf(v[i], 0.0f);
          }
          if (out_bf) {
            if (vec_store) {
              uint4 p[2];
              __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(p);
#pragma unroll
              for (int i = 0; i < 8; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
              uint4* dst = reinterpret_cast<uint4*>(out_bf + o + j * 16);
              dst[0] = p[0];
              dst[1] = p[1];
            } else {
#pragma unroll
              for (int i = 0; i < 16; ++i) out_bf[o + j * 16 + i] = __float2bfloat16_rn(v[i]);
            }
          }
          if (out_f) {
#pragma unroll
            for (int i = 0; i < 16; ++i) out_f[o + j * 16 + i] = v[i];
          }
        }
      }
    }
    if (s + 1 < nsl) {
      cp_async_wait_all();
      fence_async_smem();   // plane z + 2 visible to the tensor core
      tc_fence_before();    // this slice's tcgen05.ld are complete before the accumulators are rewritten
      __syncthreads();
      if (tid == 0 && !stall) {
        tc_fence_after();
        issue(z + 1);
      }
    }
  }
  if (!ok && tid == 0) atomicExch(&g_tc_status, (int)LT_ETIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, kCols);
}

}  // namespace

// The z-walking kernel takes one channel chunk (Ci == 16) and any D; the
// chunked kernel needs even H and D.
static bool zwalk_applies(int H, int Ci, int Co) { return Ci == 16 && H % ZW_RY == 0 && Co % 48 != 0; }

bool conv3d_tc_supported(const void* in, const void* w, const void* out_bf, int D, int H, int W, int Ci, int Co) {
  const auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (!(W > 0 && W % 64 == 0 && H > 0 && D > 0 && Ci > 0 && Ci % 16 == 0 && Co > 0 && Co % 16 == 0 && al16(in) &&
        al16(w) && al16(out_bf)))
    return false;
  return zwalk_applies(H, Ci, Co) || (H % TC_RY == 0 && D % TC_RZ == 0);
}

bool conv3d_tc_variant_supported(int variant, int D, int H, int Ci, int Co) {
  if (variant == kTcZWalk) return zwalk_applies(H, Ci, Co);
  if (variant == kTcChunked) return H % TC_RY == 0 && D % TC_RZ == 0;
  return true;
}

namespace {
template <int TM, int N>
cudaError_t launch_tc(const bf16* in, const bf16* w, const float* b, bf16* out_bf, float* out_f, dim3 grid, int D,
                      int H, int W, int Ci, int Co, int o_stride, int o_off, int relu, int tx, int ty, int vec,
                      cudaStream_t st) {
  static bool attr_set = false;   // more than 48 KB of dynamic shared memory
  if (!attr_set) {
    const cudaError_t e = cudaFuncSetAttribute(conv3d_tc_kernel<TM, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               tc_smem_bytes<TM, N>());
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  conv3d_tc_kernel<TM, N><<<grid, TC_THREADS, tc_smem_bytes<TM, N>(), st>>>(in, w, b, out_bf, out_f, D, H, W, Ci,
                                                                            Co, o_stride, o_off, relu, tx, ty, vec);
  return cudaGetLastError();
}

template <int TM>
cudaError_t launch_tm(int nb, const bf16* in, const bf16* w, const float* b, bf16* out_bf, float* out_f, dim3 grid,
                      int D, int H, int W, int Ci, int Co, int o_stride, int o_off, int relu, int tx, int ty, int vec,
                      cudaStream_t st) {
  if (nb == 48) return launch_tc<TM, 48>(in, w, b, out_bf, out_f, grid, D, H, W, Ci, Co, o_stride, o_off, relu, tx, ty, vec, st);
  if (nb == 32) return launch_tc<TM, 32>(in, w, b, out_bf, out_f, grid, D, H, W, Ci, Co, o_stride, o_off, relu, tx, ty, vec, st);
  return launch_tc<TM, 16>(in, w, b, out_bf, out_f, grid, D, H, W, Ci, Co, o_stride, o_off, relu, tx, ty, vec, st);
}
}  // namespace

namespace {
template <int TM, int N>
cudaError_t launch_zw(const bf16* in, const bf16* w, const float* b, bf16* out_bf, float* out_f, int batch, int D,
                      int H, int W, int Co, int o_stride, int o_off, int relu, int vec, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    const cudaError_t e = cudaFuncSetAttribute(conv3d_tc_zwalk_kernel<TM, N>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, zw_smem_bytes<TM, N>());
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int tx = W / TM, ty = H / ZW_RY, tz = (D + ZW_SLICES - 1) / ZW_SLICES;
  dim3 grid((unsigned)((long long)tx * ty * tz), Co / N, batch);
  conv3d_tc_zwalk_kernel<TM, N><<<grid, TC_THREADS, zw_smem_bytes<TM, N>(), st>>>(
      in, w, b, out_bf, out_f, D, H, W, Co, o_stride, o_off, relu, tx, ty, vec);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_conv3d_tc(const uint16_t* in, const uint16_t* w, const float* b, uint16_t* out_bf, float* out_f,
                             int batch, int D, int H, int W, int Ci, int Co, int o_stride, int o_off, int relu,
                             int variant, cudaStream_t st) {
  const int tm = W % 128 == 0 ? 128 : 64;
  if ((long long)(W / tm) * H * D > 0x7fffffffLL || batch > 65535) return cudaErrorInvalidValue;
  // 16-byte bfloat16 stores need every voxel's channel run on a 16-byte boundary
  const int vec = (o_stride % 8 == 0 && o_off % 8 == 0) ? 1 : 0;
  // One channel chunk: the z-walking kernel, when its grid (a CTA per
  // 4-row column and 8 slices) still gives every SM two CTAs; the chunked
  // kernel's grid is 4x larger and fills small volumes better.
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 148;
  const long long zw_ctas = (long long)(W / tm) * (H / ZW_RY) * ((D + ZW_SLICES - 1) / ZW_SLICES) * batch;
  const bool zw_ok = zwalk_applies(H, Ci, Co), chunked_ok = H % TC_RY == 0 && D % TC_RZ == 0;
  bool zwalk = zw_ok && (zw_ctas >= 2LL * sms || !chunked_ok);
  if (variant == kTcChunked) zwalk = false;
  if (variant == kTcZWalk) zwalk = true;
  if ((zwalk && !zw_ok) || (!zwalk && !chunked_ok)) return cudaErrorInvalidValue;
  if (zwalk) {
    const bf16* i_ = reinterpret_cast<const bf16*>(in);
    const bf16* w_ = reinterpret_cast<const bf16*>(w);
    bf16* o_ = reinterpret_cast<bf16*>(out_bf);
    if (Co % 32 == 0)
      return tm == 128 ? launch_zw<128, 32>(i_, w_, b, o_, out_f, batch, D, H, W, Co, o_stride, o_off, relu, vec, st)
                       : launch_zw<64, 32>(i_, w_, b, o_, out_f, batch, D, H, W, Co, o_stride, o_off, relu, vec, st);
    return tm == 128 ? launch_zw<128, 16>(i_, w_, b, o_, out_f, batch, D, H, W, Co, o_stride, o_off, relu, vec, st)
                     : launch_zw<64, 16>(i_, w_, b, o_, out_f, batch, D, H, W, Co, o_stride, o_off, relu, vec, st);
  }
  // the widest N that divides Co: the MMA count per output tile does not
  // depend on N (each MMA's time is set by reading its 128 x 16 A tile)
  const int nb = Co % 48 == 0 ? 48 : Co % 32 == 0 ? 32 : 16;
  const int tx = W / tm, ty = H / TC_RY, tz = D / TC_RZ;
  const long long tiles = (long long)tx * ty * tz;
  dim3 grid((unsigned)tiles, Co / nb, batch);
  const bf16* i_ = reinterpret_cast<const bf16*>(in);
  const bf16* w_ = reinterpret_cast<const bf16*>(w);
  bf16* o_ = reinterpret_cast<bf16*>(out_bf);
  if (tm == 128) return launch_tm<128>(nb, i_, w_, b, o_, out_f, grid, D, H, W, Ci, Co, o_stride, o_off, relu, tx, ty, vec, st);
  return launch_tm<64>(nb, i_, w_, b, o_, out_f, grid, D, H, W, Ci, Co, o_stride, o_off, relu, tx, ty, vec, st);
}

#ifdef LT_TEST_HOOKS
cudaError_t set_tc_stall(int on, cudaStream_t st) {
  const int v = on ? 1 : 0;
  const long long limit = on ? (1LL << 12) : kWaitLimit;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc_stall, &v, sizeof(v));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc_wait_limit, &limit, sizeof(limit));
  return e;
}
#endif

cudaError_t take_tc_status(int* status, cudaStream_t st) {
  const int zero = 0;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(status, g_tc_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(int));
  return e;
}

}  // namespace lt
