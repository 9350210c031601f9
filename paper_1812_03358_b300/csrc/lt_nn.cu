// Layers of the learned warm start (3D U-Net): bfloat16 implicit-GEMM 3x3x3
// convolution on the tensor cores (warp-level MMA, float32 accumulation),
// its weight gradient, and the small pooling / upsampling / optimiser
// kernels.  Channels-last activations, every global access bounds-checked.
#include <cuda_bf16.h>
#include <mma.h>

#include <algorithm>
#include <initializer_list>

#include "lt.h"
#include "lt_host.h"
#include "lt_nn.h"
#include "lt_testing.h"
#include "lt_nn_tc.h"
#include "lt_async.cuh"

using namespace nvcuda;

namespace lt {
namespace {

typedef __nv_bfloat16 bf16;


__device__ __forceinline__ void tap_offset(int tap, int& dz, int& dy, int& dx) {
  dz = tap / 9 - 1;
  dy = (tap / 3) % 3 - 1;
  dx = tap % 3 - 1;
}

// Halo-tile implicit GEMM (the convolution used by lt_nn_conv3d).  A CTA owns
// a 16 (x) x 4 (y) x 2 (z) block of output voxels -- eight M tiles of 16
// consecutive x voxels, two per warp -- and NB output channels.  Per chunk of
// 16 input channels it stages, once, the (16+2) x (4+2) x (2+2) input halo
// and the 27 x NB x 16 weights in shared memory; then every tap's A tile is
// a plain 16-row window of the halo (rows 32 bytes apart), so the 27 taps run
// back to back without block barriers.  Out-of-volume halo voxels are zero
// (padding 1); outputs outside the volume are computed and discarded.
constexpr int CT_X = 16, CT_Y = 4, CT_Z = 2;
constexpr int CT_HX = CT_X + 2, CT_HY = CT_Y + 2, CT_HZ = CT_Z + 2;
constexpr int CT_HALO = CT_HX * CT_HY * CT_HZ;   // halo voxels
constexpr int CT_THREADS = 128;                   // 4 warps, 2 M tiles each
constexpr int CT_MT = CT_Y * CT_Z;                // 8 M tiles

template <int NB>
constexpr int ct_smem_bytes() {
  return (CT_HALO * 16 + 27 * NB * 16) * 2 > CT_MT * 16 * NB * 4 ? (CT_HALO * 16 + 27 * NB * 16) * 2
                                                                    : CT_MT * 16 * NB * 4;
}

template <int NB>
__global__ void __launch_bounds__(CT_THREADS)
conv3d_tile_kernel(const bf16* __restrict__ in, const bf16* __restrict__ w, const float* __restrict__ bias,
                   bf16* __restrict__ out_bf, float* __restrict__ out_f, int D, int H, int W, int Ci, int Co,
                   int o_stride, int o_off, int relu, int tiles_x, int tiles_y) {
  extern __shared__ __align__(128) unsigned char ct_smem[];
  bf16* halo = reinterpret_cast<bf16*>(ct_smem);          // [CT_HALO][16]
  bf16* wts = halo + CT_HALO * 16;                        // [27][NB][16]
  float* stage = reinterpret_cast<float*>(ct_smem);       // epilogue [CT_MT * 16][NB], after the last chunk
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bx = blockIdx.x % tiles_x;
  const int rest = blockIdx.x / tiles_x;
  const int by = rest % tiles_y, bz = rest / tiles_y;
  const int x0 = bx * CT_X, y0 = by * CT_Y, z0 = bz * CT_Z;
  const int n0 = blockIdx.y * NB;
  const int b = blockIdx.z;
  const long long V = (long long)D * H * W;
  const bf16* inb = in + (long long)b * V * Ci;

  wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[2][NB / 16];
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int j = 0; j < NB / 16; ++j) wmma::fill_fragment(acc[m][j], 0.0f);

  for (int c0 = 0; c0 < Ci; c0 += 16) {
    __syncthreads();   // the previous chunk's tiles are no longer read
    // halo (zero outside the volume) and weights: all copies in flight at once
    for (int t = tid; t < CT_HALO * 2; t += CT_THREADS) {
      const int v = t >> 1, h = t & 1;
      const int hx = v % CT_HX, hy = (v / CT_HX) % CT_HY, hz = v / (CT_HX * CT_HY);
      const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
      const bool inside = gx >= 0 && gx < W && gy >= 0 && gy < H && gz >= 0 && gz < D;
      const bf16* src = inside ? inb + (((long long)gz * H + gy) * W + gx) * Ci + c0 + h * 8 : inb;
      cp_async16(smem_addr(halo + v * 16 + h * 8), src, inside);
    }
    for (int t = tid; t < 27 * NB * 2; t += CT_THREADS) {
      const int h = t & 1, r = t >> 1;
      const int co = r % NB, tap = r / NB;
      const bool inside = n0 + co < Co;
      const bf16* src = inside ? w + ((long long)(n0 + co) * 27 + tap) * Ci + c0 + h * 8 : w;
      cp_async16(smem_addr(wts + (tap * NB + co) * 16 + h * 8), src, inside);
    }
    cp_async_wait_all();
    __syncthreads();
    for (int tap = 0; tap < 27; ++tap) {
      int dz, dy, dx;
      tap_offset(tap, dz, dy, dx);
      wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::col_major> bfr[NB / 16];
#pragma unroll
      for (int j = 0; j < NB / 16; ++j) wmma::load_matrix_sync(bfr[j], wts + (tap * NB + 16 * j) * 16, 16);
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int mt = warp * 2 + m;
        const int ty = mt % CT_Y, tz = mt / CT_Y;
        const bf16* ap = halo + (((tz + dz + 1) * CT_HY + (ty + dy + 1)) * CT_HX + (dx + 1)) * 16;
        wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> a;
        wmma::load_matrix_sync(a, ap, 16);
#pragma unroll
        for (int j = 0; j < NB / 16; ++j) wmma::mma_sync(acc[m][j], a, bfr[j], acc[m][j]);
      }
    }
  }
  __syncthreads();   // halo and weights are dead; the region becomes the epilogue stage
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int j = 0; j < NB / 16; ++j)
      wmma::store_matrix_sync(stage + ((warp * 2 + m) * 16) * NB + 16 * j, acc[m][j], NB, wmma::mem_row_major);
  __syncwarp();   // each warp reads back only its own 32 rows
  for (int e = lane; e < 32 * NB; e += 32) {
    const int row = e / NB, c = e - row * NB;
    const int mt = warp * 2 + (row >> 4), xr = row & 15;
    const int gx = x0 + xr, gy = y0 + mt % CT_Y, gz = z0 + mt / CT_Y;
    const int co = n0 + c;
    if (gx < W && gy < H && gz < D && co < Co) {
      float val = stage[(warp * 32 + row) * NB + c] + (bias ? bias[co] : 0.0f);
      if (relu) val = fmaxf(val, 0.0f);
      const long long o = ((long long)b * V + ((long long)gz * H + gy) * W + gx) * o_stride + o_off + co;
      if (out_bf) out_bf[o] = __float2bfloat16_rn(val);
      if (out_f) out_f[o] = val;
    }
  }
}

// Weight gradient on halo tiles: dW[co][tap][ci] += sum_v g[v][co] in[v + tap][ci].
// A CTA owns MB output channels, 16 input channels and the 9 taps of one dz,
// and walks a range of 16x4x2 voxel blocks (all frames of the batch laid end
// to end).  Per block it stages the gradient tile g[128 voxels][MB] and the
// input halo once; for each tap and each 16-voxel x run the MMA is
// g_run^T (MB x 16 voxels) times the shifted halo window (16 voxels x 16 ci).
// Warps split the MB/16 channel tiles and, when there are fewer than four,
// the eight runs; the partial sums are combined in shared memory and stored
// once per CTA in row blockIdx.x of the partial-sum array part[gridDim.x][E]
// (E = 27 Co Ci entries, dw's layout), which sum_parts_kernel then adds to dw
// in a fixed order: the result does not depend on CTA scheduling.
template <int MB>
__global__ void __launch_bounds__(CT_THREADS)
conv3d_wgrad_tile_kernel(const bf16* __restrict__ in, const bf16* __restrict__ g, float* __restrict__ part, int D,
                         int H, int W, int Ci, int Co, int tiles_x, int tiles_y, int tiles_z, long long n_tiles,
                         int tiles_per_cta) {
  constexpr int MT = MB / 16;            // channel tiles
  constexpr int RS = 4 / MT;             // warps sharing one channel tile (they split the runs)
  __shared__ __align__(128) bf16 Gs[CT_MT * 16][MB];      // [voxel of the block][co]
  __shared__ __align__(128) bf16 halo[CT_HALO * 16];
  __shared__ __align__(128) float red[4][16][16];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int mt = warp % MT, rsel = warp / MT;
  const int n_ci = Ci / 16, n_co = Co / MB;
  const int tg = blockIdx.y % 3;                 // dz = tg - 1
  const int cc = (blockIdx.y / 3) % n_ci;
  const int nc = blockIdx.y / (3 * n_ci);
  const int c0 = cc * 16, n0 = nc * MB;
  const long long V = (long long)D * H * W;
  const long long t_begin = (long long)blockIdx.x * tiles_per_cta;
  const long long t_end = t_begin + tiles_per_cta < n_tiles ? t_begin + tiles_per_cta : n_tiles;
  (void)n_co;

  wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) wmma::fill_fragment(acc[t], 0.0f);

  for (long long tile = t_begin; tile < t_end; ++tile) {
    long long r = tile;
    const int bx = (int)(r % tiles_x);
    r /= tiles_x;
    const int by = (int)(r % tiles_y);
    r /= tiles_y;
    const int bz = (int)(r % tiles_z);
    const int b = (int)(r / tiles_z);
    const int x0 = bx * CT_X, y0 = by * CT_Y, z0 = bz * CT_Z;
    const bf16* inb = in + (long long)b * V * Ci;
    const bf16* gb = g + (long long)b * V * Co;
    __syncthreads();
    // gradient tile and input halo (zero outside the volume): all copies in flight at once
    for (int t = tid; t < CT_MT * 16 * (MB / 8); t += CT_THREADS) {
      const int v = t / (MB / 8), q = t - v * (MB / 8);
      const int m = v >> 4, xr = v & 15;
      const int gx = x0 + xr, gy = y0 + m % CT_Y, gz = z0 + m / CT_Y;
      const bool inside = gx < W && gy < H && gz < D;
      const bf16* src = inside ? gb + (((long long)gz * H + gy) * W + gx) * Co + n0 + q * 8 : gb;
      cp_async16(smem_addr(&Gs[v][q * 8]), src, inside);
    }
    for (int t = tid; t < CT_HALO * 2; t += CT_THREADS) {
      const int v = t >> 1, h = t & 1;
      const int hx = v % CT_HX, hy = (v / CT_HX) % CT_HY, hz = v / (CT_HX * CT_HY);
      const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
      const bool inside = gx >= 0 && gx < W && gy >= 0 && gy < H && gz >= 0 && gz < D;
      const bf16* src = inside ? inb + (((long long)gz * H + gy) * W + gx) * Ci + c0 + h * 8 : inb;
      cp_async16(smem_addr(halo + v * 16 + h * 8), src, inside);
    }
    cp_async_wait_all();
    __syncthreads();
    for (int run = rsel; run < CT_MT; run += RS) {
      const int ty = run % CT_Y, tz = run / CT_Y;
      wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::col_major> a;
      wmma::load_matrix_sync(a, &Gs[run * 16][mt * 16], MB);
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const int dy = t / 3 - 1, dx = t % 3 - 1, dz = tg - 1;
        const bf16* bp = halo + (((tz + dz + 1) * CT_HY + (ty + dy + 1)) * CT_HX + (dx + 1)) * 16;
        wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> bfr;
        wmma::load_matrix_sync(bfr, bp, 16);
        wmma::mma_sync(acc[t], a, bfr, acc[t]);
      }
    }
  }
  // combine the warps that shared a channel tile, then one store per entry
  float* prow = part + (long long)blockIdx.x * 27 * Co * Ci;
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    __syncthreads();
    wmma::store_matrix_sync(&red[warp][0][0], acc[t], 16, wmma::mem_row_major);
    __syncthreads();
    const int tap = tg * 9 + t;
    for (int e = tid; e < MT * 256; e += CT_THREADS) {
      const int m = e >> 8, i = (e >> 4) & 15, j = e & 15;
      float v = 0.0f;
#pragma unroll
      for (int s2 = 0; s2 < RS; ++s2) v += red[m + s2 * MT][i][j];
      prow[((long long)(n0 + m * 16 + i) * 27 + tap) * Ci + c0 + j] = v;
    }
  }
}

// Weight gradient for 16 output channels (one channel tile) with all 27 taps
// in one CTA: warp w owns taps 7w .. 7w + 6 (the last warp six), each a
// 16 x 16 accumulator, and runs all eight 16-voxel x runs of every staged
// block against them.  Staged once per block for all taps (the kernel above
// stages each block once per dz: three times), and each warp issues 56 MMAs
// per staged block instead of 18.  One partial sum per weight entry per CTA,
// stored in row blockIdx.x of part as above.
__global__ void __launch_bounds__(CT_THREADS)
conv3d_wgrad27_kernel(const bf16* __restrict__ in, const bf16* __restrict__ g, float* __restrict__ part, int D, int H,
                      int W, int Ci, int Co, int tiles_x, int tiles_y, int tiles_z, long long n_tiles,
                      int tiles_per_cta) {
  constexpr int TPW = 7;   // taps per warp: 4 x 7 >= 27
  __shared__ __align__(128) bf16 Gs[CT_MT * 16][16];      // [voxel of the block][co]
  __shared__ __align__(128) bf16 halo[CT_HALO * 16];
  __shared__ __align__(128) float red[4][16][16];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_ci = Ci / 16;
  const int cc = blockIdx.y % n_ci, nc = blockIdx.y / n_ci;
  const int c0 = cc * 16, n0 = nc * 16;
  const long long V = (long long)D * H * W;
  const long long t_begin = (long long)blockIdx.x * tiles_per_cta;
  const long long t_end = t_begin + tiles_per_cta < n_tiles ? t_begin + tiles_per_cta : n_tiles;

  wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[TPW];
#pragma unroll
  for (int j = 0; j < TPW; ++j) wmma::fill_fragment(acc[j], 0.0f);

  for (long long tile = t_begin; tile < t_end; ++tile) {
    long long r = tile;
    const int bx = (int)(r % tiles_x);
    r /= tiles_x;
    const int by = (int)(r % tiles_y);
    r /= tiles_y;
    const int bz = (int)(r % tiles_z);
    const int b = (int)(r / tiles_z);
    const int x0 = bx * CT_X, y0 = by * CT_Y, z0 = bz * CT_Z;
    const bf16* inb = in + (long long)b * V * Ci;
    const bf16* gb = g + (long long)b * V * Co;
    __syncthreads();   // the previous block's tiles are no longer read
    for (int t = tid; t < CT_MT * 16 * 2; t += CT_THREADS) {
      const int v = t >> 1, q = t & 1;
      const int m = v >> 4, xr = v & 15;
      const int gx = x0 + xr, gy = y0 + m % CT_Y, gz = z0 + m / CT_Y;
      const bool inside = gx < W && gy < H && gz < D;
      const bf16* src = inside ? gb + (((long long)gz * H + gy) * W + gx) * Co + n0 + q * 8 : gb;
      cp_async16(smem_addr(&Gs[v][q * 8]), src, inside);
    }
    for (int t = tid; t < CT_HALO * 2; t += CT_THREADS) {
      const int v = t >> 1, h = t & 1;
      const int hx = v % CT_HX, hy = (v / CT_HX) % CT_HY, hz = v / (CT_HX * CT_HY);
      const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
      const bool inside = gx >= 0 && gx < W && gy >= 0 && gy < H && gz >= 0 && gz < D;
      const bf16* src = inside ? inb + (((long long)gz * H + gy) * W + gx) * Ci + c0 + h * 8 : inb;
      cp_async16(smem_addr(halo + v * 16 + h * 8), src, inside);
    }
    cp_async_wait_all();
    __syncthreads();
    for (int run = 0; run < CT_MT; ++run) {
      const int ty = run % CT_Y, tz = run / CT_Y;
      wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::col_major> a;
      wmma::load_matrix_sync(a, &Gs[run * 16][0], 16);
#pragma unroll
      for (int j = 0; j < TPW; ++j) {
        const int tap = warp * TPW + j;
        if (tap < 27) {   // uniform over the warp
          const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
          const bf16* bp = halo + (((tz + dz + 1) * CT_HY + (ty + dy + 1)) * CT_HX + (dx + 1)) * 16;
          wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> bfr;
          wmma::load_matrix_sync(bfr, bp, 16);
          wmma::mma_sync(acc[j], a, bfr, acc[j]);
        }
      }
    }
  }
  float* prow = part + (long long)blockIdx.x * 27 * Co * Ci;
#pragma unroll
  for (int j = 0; j < TPW; ++j) {
    const int tap = warp * TPW + j;
    if (tap < 27) {
      wmma::store_matrix_sync(&red[warp][0][0], acc[j], 16, wmma::mem_row_major);
      __syncwarp();
      for (int e = lane; e < 256; e += 32) {
        const int i = e >> 4, c = e & 15;
        prow[((long long)(n0 + i) * 27 + tap) * Ci + c0 + c] = red[warp][i][c];
      }
      __syncwarp();
    }
  }
}

// out[e] += sum_{p < n_parts} part[p stride + e]: a block owns 32 entries,
// warp w sums the parts p = w (mod 8) with two accumulators, and warp 0 adds
// the eight warp sums in order.  Every entry is summed in the same order on
// every run.
__global__ void __launch_bounds__(256)
sum_parts_kernel(const float* __restrict__ part, int n_parts, long long stride, float* __restrict__ out, long long n) {
  __shared__ float sh[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long e = (long long)blockIdx.x * 32 + lane;
  float a0 = 0.0f, a1 = 0.0f;
  if (e < n) {
    int p = warp;
    for (; p + 8 < n_parts; p += 16) {
      a0 += part[(long long)p * stride + e];
      a1 += part[(long long)(p + 8) * stride + e];
    }
    if (p < n_parts) a0 += part[(long long)p * stride + e];
  }
  sh[warp][lane] = a0 + a1;
  __syncthreads();
  if (warp == 0 && e < n) {
    float s = 0.0f;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += sh[w][lane];
    out[e] += s;
  }
}

// Bias gradient partial sums, part[blockIdx.y][co] (summed into db by
// sum_parts_kernel).
__global__ void bias_grad_kernel(const bf16* __restrict__ g, float* __restrict__ part, long long vtot, int Co) {
  // one block per output channel chunk of 32; threads stride over voxels
  const int co = blockIdx.x * 32 + (threadIdx.x & 31);
  float acc = 0.0f;
  if (co < Co)
    for (long long v = (threadIdx.x >> 5) + (long long)blockIdx.y * 8; v < vtot; v += 8LL * gridDim.y)
      acc += __bfloat162float(g[v * Co + co]);
  __shared__ float sh[8][33];
  sh[threadIdx.x >> 5][threadIdx.x & 31] = acc;
  __syncthreads();
  if (threadIdx.x < 32 && co < Co) {
    float s = 0.0f;
    for (int i = 0; i < 8; ++i) s += sh[i][threadIdx.x];
    part[(long long)blockIdx.y * Co + co] = s;
  }
}

__global__ void flip_kernel(const bf16* __restrict__ w, bf16* __restrict__ wt, int Ci, int Co) {
  const long long n = 27LL * Ci * Co;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    // i indexes wt[ci][tap][co]
    const int co = (int)(i % Co);
    const long long r = i / Co;
    const int tap = (int)(r % 27);
    const int ci = (int)(r / 27);
    wt[i] = w[((long long)co * 27 + (26 - tap)) * Ci + ci];
  }
}

__global__ void f2b_kernel(const float* x, bf16* y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}
__global__ void b2f_kernel(const bf16* x, float* y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __bfloat162float(x[i]);
}
__global__ void relu_bwd_kernel(const bf16* y, bf16* g, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!(__bfloat162float(y[i]) > 0.0f)) g[i] = __float2bfloat16_rn(0.0f);
}

__global__ void avgpool_kernel(const bf16* in, bf16* out, int batch, int D, int H, int W, int C, int is, int io) {
  const int d = D / 2, h = H / 2, w = W / 2;
  const long long n = (long long)batch * d * h * w * C;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    long long r = i / C;
    const int x = (int)(r % w); r /= w;
    const int y = (int)(r % h); r /= h;
    const int z = (int)(r % d);
    const int b = (int)(r / d);
    float s = 0.0f;
    for (int k = 0; k < 8; ++k) {
      const int zz = 2 * z + (k >> 2), yy = 2 * y + ((k >> 1) & 1), xx = 2 * x + (k & 1);
      s += __bfloat162float(in[((((long long)b * D + zz) * H + yy) * W + xx) * is + io + c]);
    }
    out[i] = __float2bfloat16_rn(0.125f * s);
  }
}
__global__ void avgpool_bwd_kernel(const bf16* gout, bf16* gin, int batch, int D, int H, int W, int C, int is, int io) {
  const long long n = (long long)batch * D * H * W * C;
  const int d = D / 2, h = H / 2, w = W / 2;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    long long r = i / C;
    const int x = (int)(r % W); r /= W;
    const int y = (int)(r % H); r /= H;
    const int z = (int)(r % D);
    const int b = (int)(r / D);
    const float v = __bfloat162float(gout[((((long long)b * d + z / 2) * h + y / 2) * w + x / 2) * C + c]);
    gin[((((long long)b * D + z) * H + y) * W + x) * is + io + c] = __float2bfloat16_rn(0.125f * v);
  }
}
__global__ void upsample_kernel(const bf16* in, bf16* out, int batch, int d, int h, int w, int C, int os, int oo) {
  const int D = 2 * d, H = 2 * h, W = 2 * w;
  const long long n = (long long)batch * D * H * W * C;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    long long r = i / C;
    const int x = (int)(r % W); r /= W;
    const int y = (int)(r % H); r /= H;
    const int z = (int)(r % D);
    const int b = (int)(r / D);
    out[((((long long)b * D + z) * H + y) * W + x) * os + oo + c] = in[((((long long)b * d + z / 2) * h + y / 2) * w + x / 2) * C + c];
  }
}
__global__ void upsample_bwd_kernel(const bf16* gout, bf16* gin, int batch, int d, int h, int w, int C, int os, int oo) {
  const long long n = (long long)batch * d * h * w * C;
  const int D = 2 * d, H = 2 * h, W = 2 * w;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    long long r = i / C;
    const int x = (int)(r % w); r /= w;
    const int y = (int)(r % h); r /= h;
    const int z = (int)(r % d);
    const int b = (int)(r / d);
    float s = 0.0f;
    for (int k = 0; k < 8; ++k) {
      const int zz = 2 * z + (k >> 2), yy = 2 * y + ((k >> 1) & 1), xx = 2 * x + (k & 1);
      s += __bfloat162float(gout[((((long long)b * D + zz) * H + yy) * W + xx) * os + oo + c]);
    }
    gin[i] = __float2bfloat16_rn(s);
  }
}
__global__ void copy_channels_kernel(const bf16* src, bf16* dst, long long voxels, int C, int ss, int so, int ds, int dof) {
  const long long n = voxels * C;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long v = i / C;
    const int c = (int)(i - v * C);
    dst[v * ds + dof + c] = src[v * ss + so + c];
  }
}
// Vectorised forms of the pooling, upsampling and channel-copy kernels: one
// thread per (coarse voxel, group of 8 channels), 16-byte loads and stores
// and 32-bit index arithmetic, for channel counts, strides and offsets that
// are multiples of 8 on 16-byte aligned buffers (every use in the network).
// Per element they compute exactly what the scalar kernels above compute,
// summing the eight fine voxels in the same order.
struct V8 {
  float v[8];
};
__device__ __forceinline__ V8 load8(const bf16* p) {
  const uint4 u = *reinterpret_cast<const uint4*>(p);
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
  V8 r;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __bfloat1622float2(h[i]);
    r.v[2 * i] = f.x;
    r.v[2 * i + 1] = f.y;
  }
  return r;
}
__device__ __forceinline__ void store8(bf16* p, const V8& r) {
  uint4 u;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(r.v[2 * i], r.v[2 * i + 1]);
  *reinterpret_cast<uint4*>(p) = u;
}
// thread index i over (batch, z, y, x, channel group) of a d x h x w grid
__device__ __forceinline__ void coarse_index(unsigned i, int C8, int w, int h, int d, int& g, long long& vox, int& x,
                                             int& y, int& z, int& b) {
  g = (int)(i % C8);
  unsigned u = i / C8;
  vox = u;
  x = (int)(u % w);
  u /= w;
  y = (int)(u % h);
  u /= h;
  z = (int)(u % d);
  b = (int)(u / d);
}
// fine voxel k (0..7, z-major as in the scalar kernels) of coarse voxel (x, y, z)
__device__ __forceinline__ long long fine_voxel(int k, int b, int z, int y, int x, int D, int H, int W) {
  const int zz = 2 * z + (k >> 2), yy = 2 * y + ((k >> 1) & 1), xx = 2 * x + (k & 1);
  return (((long long)b * D + zz) * H + yy) * W + xx;
}

__global__ void avgpool_vec_kernel(const bf16* __restrict__ in, bf16* __restrict__ out, int batch, int D, int H,
                                   int W, int C, int is, int io) {
  const int d = D / 2, h = H / 2, w = W / 2, C8 = C / 8;
  const unsigned n = (unsigned)batch * d * h * w * C8;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int g, x, y, z, b;
    long long vox;
    coarse_index(i, C8, w, h, d, g, vox, x, y, z, b);
    V8 s;
#pragma unroll
    for (int c = 0; c < 8; ++c) s.v[c] = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const V8 a = load8(in + fine_voxel(k, b, z, y, x, D, H, W) * is + io + 8 * g);
#pragma unroll
      for (int c = 0; c < 8; ++c) s.v[c] += a.v[c];
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) s.v[c] *= 0.125f;
    store8(out + vox * C + 8 * g, s);
  }
}
__global__ void avgpool_bwd_vec_kernel(const bf16* __restrict__ gout, bf16* __restrict__ gin, int batch, int D, int H,
                                       int W, int C, int is, int io) {
  const int d = D / 2, h = H / 2, w = W / 2, C8 = C / 8;
  const unsigned n = (unsigned)batch * d * h * w * C8;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int g, x, y, z, b;
    long long vox;
    coarse_index(i, C8, w, h, d, g, vox, x, y, z, b);
    V8 v = load8(gout + vox * C + 8 * g);
#pragma unroll
    for (int c = 0; c < 8; ++c) v.v[c] *= 0.125f;
#pragma unroll
    for (int k = 0; k < 8; ++k) store8(gin + fine_voxel(k, b, z, y, x, D, H, W) * is + io + 8 * g, v);
  }
}
__global__ void upsample_vec_kernel(const bf16* __restrict__ in, bf16* __restrict__ out, int batch, int d, int h,
                                    int w, int C, int os, int oo) {
  const int C8 = C / 8;
  const unsigned n = (unsigned)batch * d * h * w * C8;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int g, x, y, z, b;
    long long vox;
    coarse_index(i, C8, w, h, d, g, vox, x, y, z, b);
    const uint4 u = *reinterpret_cast<const uint4*>(in + vox * C + 8 * g);
#pragma unroll
    for (int k = 0; k < 8; ++k)
      *reinterpret_cast<uint4*>(out + fine_voxel(k, b, z, y, x, 2 * d, 2 * h, 2 * w) * os + oo + 8 * g) = u;
  }
}
__global__ void upsample_bwd_vec_kernel(const bf16* __restrict__ gout, bf16* __restrict__ gin, int batch, int d,
                                        int h, int w, int C, int os, int oo) {
  const int C8 = C / 8;
  const unsigned n = (unsigned)batch * d * h * w * C8;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int g, x, y, z, b;
    long long vox;
    coarse_index(i, C8, w, h, d, g, vox, x, y, z, b);
    V8 s;
#pragma unroll
    for (int c = 0; c < 8; ++c) s.v[c] = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const V8 a = load8(gout + fine_voxel(k, b, z, y, x, 2 * d, 2 * h, 2 * w) * os + oo + 8 * g);
#pragma unroll
      for (int c = 0; c < 8; ++c) s.v[c] += a.v[c];
    }
    store8(gin + vox * C + 8 * g, s);
  }
}
__global__ void copy_channels_vec_kernel(const bf16* __restrict__ src, bf16* __restrict__ dst, unsigned n, int C8,
                                         int ss, int so, int ds, int dof) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned v = i / C8;
    const int g = (int)(i - v * C8);
    *reinterpret_cast<uint4*>(dst + (long long)v * ds + dof + 8 * g) =
        *reinterpret_cast<const uint4*>(src + (long long)v * ss + so + 8 * g);
  }
}

// Elementwise kernels on 8 values per thread (16-byte accesses).
__global__ void relu_bwd_vec_kernel(const bf16* __restrict__ y, bf16* __restrict__ g, unsigned n8) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += gridDim.x * blockDim.x) {
    const V8 a = load8(y + 8LL * i);
    V8 b = load8(g + 8LL * i);
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (!(a.v[c] > 0.0f)) b.v[c] = 0.0f;
    store8(g + 8LL * i, b);
  }
}
__global__ void add_vec_kernel(const bf16* __restrict__ a, const bf16* __restrict__ b, bf16* __restrict__ out,
                               unsigned n8) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += gridDim.x * blockDim.x) {
    V8 x = load8(a + 8LL * i);
    const V8 y = load8(b + 8LL * i);
#pragma unroll
    for (int c = 0; c < 8; ++c) x.v[c] += y.v[c];
    store8(out + 8LL * i, x);
  }
}
__global__ void f2b_vec_kernel(const float* __restrict__ x, bf16* __restrict__ y, unsigned n8) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += gridDim.x * blockDim.x) {
    const float4 p = *reinterpret_cast<const float4*>(x + 8LL * i);
    const float4 q = *reinterpret_cast<const float4*>(x + 8LL * i + 4);
    const V8 v{{p.x, p.y, p.z, p.w, q.x, q.y, q.z, q.w}};
    store8(y + 8LL * i, v);
  }
}
// Bias gradient partial sums with 8 channels per lane: Co / 8 = C8 divides
// 32, so lane l always holds channel group l % C8; lanes of one group are
// summed by xor shuffles at multiples of C8, warps in shared memory, and each
// block stores one value per channel in part[blockIdx.x][co].
constexpr int kBiasMaxC = 256;
__global__ void __launch_bounds__(256)
bias_grad_vec_kernel(const bf16* __restrict__ g, float* __restrict__ part, long long vtot, int Co) {
  __shared__ float sh[8][kBiasMaxC];
  const int C8 = Co / 8, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane % C8, vpw = 32 / C8;
  V8 acc;
#pragma unroll
  for (int c = 0; c < 8; ++c) acc.v[c] = 0.0f;
  for (long long v = ((long long)blockIdx.x * 8 + warp) * vpw + lane / C8; v < vtot; v += (long long)gridDim.x * 8 * vpw) {
    const V8 a = load8(g + v * Co + 8 * grp);
#pragma unroll
    for (int c = 0; c < 8; ++c) acc.v[c] += a.v[c];
  }
  for (int off = C8; off < 32; off <<= 1)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc.v[c] += __shfl_xor_sync(0xffffffffu, acc.v[c], off);
  if (lane < C8)
#pragma unroll
    for (int c = 0; c < 8; ++c) sh[warp][8 * grp + c] = acc.v[c];
  __syncthreads();
  for (int ch = threadIdx.x; ch < Co; ch += blockDim.x) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t += sh[w][ch];
    part[(long long)blockIdx.x * Co + ch] = t;
  }
}

// The vectorised kernels apply: channel counts, strides and offsets multiples
// of 8, buffers 16-byte aligned, and fewer than 2^31 thread items.
static bool vec8_ok(const void* a, const void* b, long long items, std::initializer_list<int> mult8) {
  const auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  for (int m : mult8)
    if (m % 8) return false;
  return al(a) && al(b) && items < (1LL << 31);
}

// Squared gradient norm in a fixed order: block b of a fixed grid of
// kNormBlocks sums the elements b*256 + t (mod kNormBlocks*256) per thread,
// then the block's threads in a fixed tree, into part[b]; clip_scale_kernel
// adds the kNormBlocks partial sums in order and writes {scale, norm}, scale =
// min(1, max_norm / norm) (1 if max_norm <= 0; 0 if the norm is not finite,
// so that step's gradient is dropped).
constexpr int kNormBlocks = 148;
static_assert(kNormBlocks <= LT_NN_NORM_WORK, "norm scratch too small");
__global__ void __launch_bounds__(256) sumsq_parts_kernel(const float* __restrict__ g, long long n,
                                                          float* __restrict__ part) {
  __shared__ float sh[8];
  float acc = 0.0f;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)kNormBlocks * 256)
    acc = fmaf(g[i], g[i], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}
__global__ void clip_scale_kernel(const float* __restrict__ part, float max_norm, float* __restrict__ out) {
  double t = 0.0;
  for (int b = 0; b < kNormBlocks; ++b) t += (double)part[b];
  const float norm = (float)sqrt(t);
  float scale = 1.0f;
  if (!isfinite(norm)) scale = 0.0f;
  else if (max_norm > 0.0f && norm > max_norm) scale = max_norm / norm;
  out[0] = scale;
  out[1] = norm;
}

__global__ void adam_kernel(float* p, bf16* pb, const float* g, const float* g_scale, float* m, float* v, long long n,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
  const float gs = g_scale ? *g_scale : 1.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i] * gs;
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void add_kernel(const bf16* a, const bf16* b, bf16* out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}
__global__ void ratio_max_kernel(const float* bp, const float* d, float* r, float* m, long long n) {
  float mx = 0.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float v = d[i] > 0.0f ? fmaxf(bp[i] / d[i], 0.0f) : 0.0f;
    r[i] = v;
    mx = fmaxf(mx, v);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(m), __float_as_int(mx));   // non-negative floats
}
__global__ void pack_input_kernel(const float* r, const float* m, bf16* u, long long n) {
  const float inv = *m > 0.0f ? 1.0f / *m : 0.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n * 16; i += (long long)gridDim.x * blockDim.x)
    u[i] = __float2bfloat16_rn((i & 15) == 0 ? r[i >> 4] * inv : 0.0f);
}
__global__ void unpack_output_kernel(const float* out, const float* m, float* x0, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x0[i] = fmaxf(out[i * 16], 0.0f) * (*m);
}
__global__ void mse_kernel(const float* out, const float* t, const float* m, float* g, float* loss, long long n) {
  const float inv = *m > 0.0f ? 1.0f / *m : 0.0f;
  const float sc = 1.0f / (float)n;
  float acc = 0.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n * 16; i += (long long)gridDim.x * blockDim.x) {
    if ((i & 15) == 0) {
      const float d = out[i] - t[i >> 4] * inv;
      g[i] = 2.0f * d * sc;
      acc += d * d * sc;
    } else {
      g[i] = 0.0f;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

int grid1d(long long n) { return (int)std::min<long long>((n + 255) / 256, 148LL * 32); }

}  // namespace
}  // namespace lt

using namespace lt;

static lt_status launched(const char* what) {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LT_OK : cuda_error(e, what);
}

extern "C" lt_status lt_nn_conv3d(const uint16_t* in, const uint16_t* w, const float* b, uint16_t* out_bf,
                                  float* out_f, int32_t batch, int32_t D, int32_t H, int32_t W, int32_t Ci,
                                  int32_t Co, int32_t o_stride, int32_t o_off, int32_t relu, void* stream) {
  return lt_nn_conv3d_ex(in, w, b, out_bf, out_f, batch, D, H, W, Ci, Co, o_stride, o_off, relu, LT_CONV_AUTO,
                         stream);
}

extern "C" lt_status lt_nn_device_status(void* stream) {
  clear_error();
  int st = 0;
  cudaError_t e = take_tc_status(&st, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "device status");
  if (st != 0) return set_error(LT_ETIMEOUT, "a tcgen05 convolution gave up waiting for the tensor core");
  return LT_OK;
}

#ifdef LT_TEST_HOOKS
extern "C" lt_status lt_nn_test_stall_tensor_core(int32_t on, void* stream) {
  clear_error();
  const cudaError_t e = set_tc_stall(on, (cudaStream_t)stream);
  return e == cudaSuccess ? LT_OK : cuda_error(e, "tensor-core stall hook");
}
#endif

extern "C" lt_status lt_nn_conv3d_ex(const uint16_t* in, const uint16_t* w, const float* b, uint16_t* out_bf,
                                     float* out_f, int32_t batch, int32_t D, int32_t H, int32_t W, int32_t Ci,
                                     int32_t Co, int32_t o_stride, int32_t o_off, int32_t relu, int32_t path,
                                     void* stream) {
  clear_error();
  NvtxRange range("lt_nn_conv3d");
  if (!in || !w || (!out_bf && !out_f) || batch <= 0 || D <= 0 || H <= 0 || W <= 0 || Ci <= 0 || Co <= 0 ||
      Ci % 16 || Co % 16 || o_off < 0 || o_stride < o_off + Co || path < LT_CONV_AUTO || path > LT_CONV_TCGEN05_ZWALK)
    return set_error(LT_EINVAL, "conv3d: bad arguments (channels must be multiples of 16)");
  const bool tc_ok = conv3d_tc_supported(in, w, out_bf, D, H, W, Ci, Co);
  if (path >= LT_CONV_TCGEN05 || (path == LT_CONV_AUTO && tc_ok)) {
    const int variant = path == LT_CONV_TCGEN05_CHUNKED ? kTcChunked : path == LT_CONV_TCGEN05_ZWALK ? kTcZWalk : kTcBest;
    if (!tc_ok || !conv3d_tc_variant_supported(variant, D, H, Ci, Co))
      return set_error(LT_EUNSUPPORTED, "conv3d: this tcgen05 kernel does not tile the shape (W %% 64, aligned pointers; "
                                        "chunked: even H and D; z-walking: Ci == 16, H %% 4 == 0, Co %% 48 != 0)");
    const cudaError_t e = launch_conv3d_tc(in, w, b, out_bf, out_f, batch, D, H, W, Ci, Co, o_stride, o_off, relu,
                                           variant, (cudaStream_t)stream);
    return e == cudaSuccess ? LT_OK : cuda_error(e, "conv3d (tcgen05)");
  }
  const int tx = (W + CT_X - 1) / CT_X, ty = (H + CT_Y - 1) / CT_Y, tz = (D + CT_Z - 1) / CT_Z;
  const long long tiles = (long long)tx * ty * tz;
  if (tiles > 0x7fffffffLL) return set_error(LT_EINVAL, "conv3d: volume too large");
  constexpr long long kNbMinCtasPerSm = 1;
  // the widest channel block that still gives kNbMinCtasPerSm CTAs per SM: a
  // wider block stages its halo once for more output channels, a narrower
  // one keeps small volumes (32^3, 16^3) from leaving SMs idle
  int nb = Co % 64 == 0 ? 64 : Co % 32 == 0 ? 32 : 16;
  while (nb > 16 && tiles * (Co / nb) * batch < 148LL * kNbMinCtasPerSm) nb /= 2;
  dim3 grid((unsigned)tiles, Co / nb, batch);
  cudaStream_t st = (cudaStream_t)stream;
  const bf16* i_ = reinterpret_cast<const bf16*>(in);
  const bf16* w_ = reinterpret_cast<const bf16*>(w);
  bf16* o_ = reinterpret_cast<bf16*>(out_bf);
  static bool attr_set = false;   // the 64-channel variant needs more than 48 KB of shared memory
  if (!attr_set) {
    cudaFuncSetAttribute(conv3d_tile_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, ct_smem_bytes<64>());
    cudaFuncSetAttribute(conv3d_tile_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, ct_smem_bytes<32>());
    cudaFuncSetAttribute(conv3d_tile_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, ct_smem_bytes<16>());
    attr_set = true;
  }
  if (nb == 64)
    conv3d_tile_kernel<64><<<grid, CT_THREADS, ct_smem_bytes<64>(), st>>>(i_, w_, b, o_, out_f, D, H, W, Ci, Co, o_stride,
                                                                         o_off, relu, tx, ty);
  else if (nb == 32)
    conv3d_tile_kernel<32><<<grid, CT_THREADS, ct_smem_bytes<32>(), st>>>(i_, w_, b, o_, out_f, D, H, W, Ci, Co, o_stride,
                                                                         o_off, relu, tx, ty);
  else
    conv3d_tile_kernel<16><<<grid, CT_THREADS, ct_smem_bytes<16>(), st>>>(i_, w_, b, o_, out_f, D, H, W, Ci, Co, o_stride,
                                                                         o_off, relu, tx, ty);
  return launched("conv3d");
}

// Launch shape of the weight gradient and the size of its partial-sum array:
// gx CTAs per channel group, each walking `per` voxel blocks (about four waves
// over the 148 SMs), one row of E = 27 Co Ci partial sums per CTA column, then
// the bias partial sums (one row of Co per block of whichever bias kernel the
// gradient's alignment selects; the array is sized for the larger).
struct WgradShape {
  int mb = 0, tx = 0, ty = 0, tz = 0, per = 0;
  bool all_taps = false;
  long long vtot = 0, n_tiles = 0, groups = 0, E = 0;
  unsigned gx = 0, bias_vec_blocks = 0, bias_rows = 0;
  long long floats = 0;
};

static bool wgrad_shape(int batch, int D, int H, int W, int Ci, int Co, WgradShape& q) {
  if (batch <= 0 || D <= 0 || H <= 0 || W <= 0 || Ci <= 0 || Co <= 0 || Ci % 16 || Co % 16) return false;
  q.vtot = (long long)D * H * W * batch;
  q.mb = Co % 64 == 0 ? 64 : Co % 32 == 0 ? 32 : 16;
  q.tx = (W + CT_X - 1) / CT_X;
  q.ty = (H + CT_Y - 1) / CT_Y;
  q.tz = (D + CT_Z - 1) / CT_Z;
  q.n_tiles = (long long)q.tx * q.ty * q.tz * batch;
  q.all_taps = q.mb == 16;   // one channel tile: every tap in one CTA
  q.groups = (q.all_taps ? 1LL : 3LL) * (Ci / 16) * (Co / q.mb);
  if (q.groups > 65535) return false;
  const long long want = std::max<long long>(1, (148LL * 4 + q.groups - 1) / q.groups);
  q.per = (int)std::max<long long>(1, (q.n_tiles + want - 1) / want);
  q.gx = (unsigned)((q.n_tiles + q.per - 1) / q.per);
  q.E = 27LL * Co * Ci;
  const int c8 = Co / 8;
  const long long per_block = 8LL * (32 / std::max(1, std::min(c8, 32)));   // voxels a vector block reads per sweep
  q.bias_vec_blocks = (unsigned)std::min<long long>(148LL * 8, (q.vtot + per_block - 1) / per_block);
  q.bias_rows = (unsigned)std::min<long long>(1024, (q.vtot + 7) / 8);
  q.floats = (long long)q.gx * q.E + (long long)std::max(q.bias_vec_blocks, q.bias_rows) * Co;
  return true;
}

extern "C" lt_status lt_nn_conv3d_wgrad_workspace(int32_t batch, int32_t D, int32_t H, int32_t W, int32_t Ci,
                                                  int32_t Co, int64_t* floats) {
  clear_error();
  WgradShape q;
  if (!floats || !wgrad_shape(batch, D, H, W, Ci, Co, q))
    return set_error(LT_EINVAL, "conv3d_wgrad_workspace: bad arguments (channels must be multiples of 16)");
  *floats = q.floats;
  return LT_OK;
}

extern "C" lt_status lt_nn_conv3d_wgrad(const uint16_t* in, const uint16_t* g, float* dw, float* db, float* work,
                                        int64_t work_floats, int32_t batch, int32_t D, int32_t H, int32_t W,
                                        int32_t Ci, int32_t Co, void* stream) {
  clear_error();
  WgradShape q;
  if (!in || !g || !dw || !work || !wgrad_shape(batch, D, H, W, Ci, Co, q))
    return set_error(LT_EINVAL, "conv3d_wgrad: bad arguments (channels must be multiples of 16)");
  if (work_floats < q.floats) return set_error(LT_EINVAL, "conv3d_wgrad: workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  dim3 grid(q.gx, (unsigned)q.groups);
  const bf16* i_ = reinterpret_cast<const bf16*>(in);
  const bf16* g_ = reinterpret_cast<const bf16*>(g);
  const int tx = q.tx, ty = q.ty, tz = q.tz, per = q.per;
  const long long n_tiles = q.n_tiles;
  if (q.all_taps)
    conv3d_wgrad27_kernel<<<grid, CT_THREADS, 0, st>>>(i_, g_, work, D, H, W, Ci, Co, tx, ty, tz, n_tiles, per);
  else if (q.mb == 64)
    conv3d_wgrad_tile_kernel<64><<<grid, CT_THREADS, 0, st>>>(i_, g_, work, D, H, W, Ci, Co, tx, ty, tz, n_tiles, per);
  else if (q.mb == 32)
    conv3d_wgrad_tile_kernel<32><<<grid, CT_THREADS, 0, st>>>(i_, g_, work, D, H, W, Ci, Co, tx, ty, tz, n_tiles, per);
  else
    conv3d_wgrad_tile_kernel<16><<<grid, CT_THREADS, 0, st>>>(i_, g_, work, D, H, W, Ci, Co, tx, ty, tz, n_tiles, per);
  sum_parts_kernel<<<(unsigned)((q.E + 31) / 32), 256, 0, st>>>(work, (int)q.gx, q.E, dw, q.E);
  if (db) {
    float* bpart = work + (long long)q.gx * q.E;
    const int c8 = Co / 8;
    unsigned rows;
    if (Co % 8 == 0 && Co <= kBiasMaxC && 32 % c8 == 0 && (reinterpret_cast<uintptr_t>(g) & 15u) == 0) {
      rows = q.bias_vec_blocks;
      bias_grad_vec_kernel<<<rows, 256, 0, st>>>(g_, bpart, q.vtot, Co);
    } else {
      rows = q.bias_rows;
      dim3 gb((Co + 31) / 32, rows);
      bias_grad_kernel<<<gb, 256, 0, st>>>(g_, bpart, q.vtot, Co);
    }
    sum_parts_kernel<<<(unsigned)((Co + 31) / 32), 256, 0, st>>>(bpart, (int)rows, Co, db, Co);
  }
  return launched("conv3d_wgrad");
}

extern "C" lt_status lt_nn_conv3d_flip(const uint16_t* w, uint16_t* wt, int32_t Ci, int32_t Co, void* stream) {
  clear_error();
  if (!w || !wt || Ci <= 0 || Co <= 0) return set_error(LT_EINVAL, "conv3d_flip: bad arguments");
  flip_kernel<<<grid1d(27LL * Ci * Co), 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const bf16*>(w),
                                                                          reinterpret_cast<bf16*>(wt), Ci, Co);
  return launched("conv3d_flip");
}

extern "C" lt_status lt_nn_f32_to_bf16(const float* x, uint16_t* y, int64_t n, void* stream) {
  clear_error();
  if (!x || !y || n < 0) return set_error(LT_EINVAL, "f32_to_bf16: bad arguments");
  if (n && vec8_ok(x, y, n / 8, {(int)(n % 8)}))
    f2b_vec_kernel<<<grid1d(n / 8), 256, 0, (cudaStream_t)stream>>>(x, reinterpret_cast<bf16*>(y), (unsigned)(n / 8));
  else if (n)
    f2b_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(x, reinterpret_cast<bf16*>(y), n);
  return launched("f32_to_bf16");
}

extern "C" lt_status lt_nn_bf16_to_f32(const uint16_t* x, float* y, int64_t n, void* stream) {
  clear_error();
  if (!x || !y || n < 0) return set_error(LT_EINVAL, "bf16_to_f32: bad arguments");
  if (n) b2f_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const bf16*>(x), y, n);
  return launched("bf16_to_f32");
}

extern "C" lt_status lt_nn_relu_backward(const uint16_t* y, uint16_t* g, int64_t n, void* stream) {
  clear_error();
  if (!y || !g || n < 0) return set_error(LT_EINVAL, "relu_backward: bad arguments");
  if (n && vec8_ok(y, g, n / 8, {(int)(n % 8)}))
    relu_bwd_vec_kernel<<<grid1d(n / 8), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const bf16*>(y), reinterpret_cast<bf16*>(g), (unsigned)(n / 8));
  else if (n)
    relu_bwd_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const bf16*>(y),
                                                                  reinterpret_cast<bf16*>(g), n);
  return launched("relu_backward");
}

extern "C" lt_status lt_nn_avgpool2(const uint16_t* in, uint16_t* out, int32_t batch, int32_t D, int32_t H, int32_t W,
                                    int32_t C, int32_t i_stride, int32_t i_off, void* stream) {
  clear_error();
  if (!in || !out || batch <= 0 || D <= 0 || H <= 0 || W <= 0 || D % 2 || H % 2 || W % 2 || C <= 0 ||
      i_stride < i_off + C || i_off < 0)
    return set_error(LT_EINVAL, "avgpool2: bad arguments");
  const long long n = (long long)batch * (D / 2) * (H / 2) * (W / 2) * C;
  if (vec8_ok(in, out, n / 8, {C, i_stride, i_off}))
    avgpool_vec_kernel<<<grid1d(n / 8), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const bf16*>(in), reinterpret_cast<bf16*>(out), batch, D, H, W, C, i_stride, i_off);
  else
    avgpool_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const bf16*>(in),
                                                                 reinterpret_cast<bf16*>(out), batch, D, H, W, C,
                                                                 i_stride, i_off);
  return launched("avgpool2");
}

extern "C" lt_status lt_nn_avgpool2_backward(const uint16_t* gout, uint16_t* gin, int32_t batch, int32_t D, int32_t H,
                                             int32_t W, int32_t C, int32_t i_stride, int32_t i_off, void* stream) {
  clear_error();
  if (!gout || !gin || batch <= 0 || D <= 0 || H <= 0 || W <= 0 || D % 2 || H % 2 || W % 2 || C <= 0 ||
      i_stride < i_off + C || i_off < 0)
    return set_error(LT_EINVAL, "avgpool2_backward: bad arguments");
  const long long n = (long long)batch * D * H * W * C;
  if (vec8_ok(gout, gin, n / 64, {C, i_stride, i_off}))
    avgpool_bwd_vec_kernel<<<grid1d(n / 64), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const bf16*>(gout), reinterpret_cast<bf16*>(gin), batch, D, H, W, C, i_stride, i_off);
  else
    avgpool_bwd_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const bf16*>(gout),
                                                                     reinterpret_cast<bf16*>(gin), batch, D, H, W, C,
                                                                     i_stride, i_off);
  return launched("avgpool2_backward");
}

extern "C" lt_status lt_nn_upsample2(const uint16_t* in, uint16_t* out, int32_t batch, int32_t d, int32_t h, int32_t w,
                                     int32_t C, int32_t o_stride, int32_t o_off, void* stream) {
  clear_error();
  if (!in || !out || batch <= 0 || d <= 0 || h <= 0 || w <= 0 || C <= 0 || o_stride < o_off + C || o_off < 0)
    return set_error(LT_EINVAL, "upsample2: bad arguments");
  const long long n = (long long)batch * 8 * d * h * w * C;
  if (vec8_ok(in, out, n / 64, {C, o_stride, o_off}))
    upsample_vec_kernel<<<grid1d(n / 64), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const bf16*>(in), reinterpret_cast<bf16*>(out), batch, d, h, w, C, o_stride, o_off);
  else
    upsample_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const bf16*>(in),
                                                                  reinterpret_cast<bf16*>(out), batch, d, h, w, C,
                                                                  o_stride, o_off);
  return launched("upsample2");
}

extern "C" lt_status lt_nn_upsample2_backward(const uint16_t* gout, uint16_t* gin, int32_t batch, int32_t d, int32_t h,
                                              int32_t w, int32_t C, int32_t o_stride, int32_t o_off, void* stream) {
  clear_error();
  if (!gout || !gin || batch <= 0 || d <= 0 || h <= 0 || w <= 0 || C <= 0 || o_stride < o_off + C || o_off < 0)
    return set_error(LT_EINVAL, "upsample2_backward: bad arguments");
  const long long n = (long long)batch * d * h * w * C;
  if (vec8_ok(gout, gin, n / 8, {C, o_stride, o_off}))
    upsample_bwd_vec_kernel<<<grid1d(n / 8), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const bf16*>(gout), reinterpret_cast<bf16*>(gin), batch, d, h, w, C, o_stride, o_off);
  else
    upsample_bwd_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const bf16*>(gout),
                                                                      reinterpret_cast<bf16*>(gin), batch, d, h, w, C,
                                                                      o_stride, o_off);
  return launched("upsample2_backward");
}

extern "C" lt_status lt_nn_copy_channels(const uint16_t* src, uint16_t* dst, int64_t voxels, int32_t C, int32_t s_stride,
                                         int32_t s_off, int32_t d_stride, int32_t d_off, void* stream) {
  clear_error();
  if (!src || !dst || voxels < 0 || C <= 0 || s_stride < s_off + C || d_stride < d_off + C || s_off < 0 || d_off < 0)
    return set_error(LT_EINVAL, "copy_channels: bad arguments");
  if (voxels && vec8_ok(src, dst, voxels * C / 8, {C, s_stride, s_off, d_stride, d_off}))
    copy_channels_vec_kernel<<<grid1d(voxels * C / 8), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const bf16*>(src), reinterpret_cast<bf16*>(dst), (unsigned)(voxels * C / 8), C / 8, s_stride,
        s_off, d_stride, d_off);
  else if (voxels)
    copy_channels_kernel<<<grid1d(voxels * C), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const bf16*>(src), reinterpret_cast<bf16*>(dst), voxels, C, s_stride, s_off, d_stride, d_off);
  return launched("copy_channels");
}

extern "C" lt_status lt_nn_grad_norm_clip(const float* g, int64_t n, float max_norm, float* work, float* out,
                                          void* stream) {
  clear_error();
  if (!g || !work || !out || n < 0) return set_error(LT_EINVAL, "grad_norm_clip: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  sumsq_parts_kernel<<<kNormBlocks, 256, 0, st>>>(g, n, work);
  clip_scale_kernel<<<1, 1, 0, st>>>(work, max_norm, out);
  return launched("grad_norm_clip");
}

extern "C" lt_status lt_nn_adam(float* p, uint16_t* pb, const float* g, const float* g_scale, float* m, float* v,
                                int64_t n, float lr, float b1, float b2, float eps, int32_t step, void* stream) {
  clear_error();
  if (!p || !g || !m || !v || n < 0 || step < 1) return set_error(LT_EINVAL, "adam: bad arguments");
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  if (n)
    adam_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(p, reinterpret_cast<bf16*>(pb), g, g_scale, m, v, n, lr,
                                                              b1, b2, eps, c1, c2);
  return launched("adam");
}

extern "C" lt_status lt_nn_add(const uint16_t* a, const uint16_t* b, uint16_t* out, int64_t n, void* stream) {
  clear_error();
  if (!a || !b || !out || n < 0) return set_error(LT_EINVAL, "add: bad arguments");
  if (n && vec8_ok(a, b, n / 8, {(int)(n % 8)}) && (reinterpret_cast<uintptr_t>(out) & 15u) == 0)
    add_vec_kernel<<<grid1d(n / 8), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const bf16*>(a), reinterpret_cast<const bf16*>(b), reinterpret_cast<bf16*>(out),
        (unsigned)(n / 8));
  else if (n)
    add_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const bf16*>(a), reinterpret_cast<const bf16*>(b),
                                                             reinterpret_cast<bf16*>(out), n);
  return launched("add");
}

extern "C" lt_status lt_nn_prepare_input(const float* bp, const float* d, float* r, float* m, uint16_t* u, int64_t voxels,
                                         void* stream) {
  clear_error();
  if (!bp || !d || !r || !m || !u || voxels <= 0) return set_error(LT_EINVAL, "prepare_input: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemsetAsync(m, 0, sizeof(float), st);
  ratio_max_kernel<<<grid1d(voxels), 256, 0, st>>>(bp, d, r, m, voxels);
  pack_input_kernel<<<grid1d(voxels * 16), 256, 0, st>>>(r, m, reinterpret_cast<bf16*>(u), voxels);
  return launched("prepare_input");
}

extern "C" lt_status lt_nn_unpack_output(const float* out, const float* m, float* x0, int64_t voxels, void* stream) {
  clear_error();
  if (!out || !m || !x0 || voxels <= 0) return set_error(LT_EINVAL, "unpack_output: bad arguments");
  unpack_output_kernel<<<grid1d(voxels), 256, 0, (cudaStream_t)stream>>>(out, m, x0, voxels);
  return launched("unpack_output");
}

extern "C" lt_status lt_nn_mse(const float* out, const float* target, const float* m, float* g, float* loss,
                               int64_t voxels, void* stream) {
  clear_error();
  if (!out || !target || !m || !g || !loss || voxels <= 0) return set_error(LT_EINVAL, "mse: bad arguments");
  mse_kernel<<<grid1d(voxels * 16), 256, 0, (cudaStream_t)stream>>>(out, target, m, g, loss, voxels);
  return launched("mse");
}
