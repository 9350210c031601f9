// Beam integration, gather adjoint, with TMA-staged image boxes (Sec. IV-A,
// Sec. IV-B).
//
// x[n][jy][jx] = sum over cameras, cells k, target pixels (it, is) of
// Bt[it][jy] Bs[is][jx] g_k[it][is] x scale_kn: the transpose of the beam
// forward, evaluated as a gather (one writer per voxel, no atomics).  A CTA
// owns a 32 x 8 voxel tile (thread = voxel) and a chunk of ASC consecutive
// slices of one frame, and keeps one accumulator per slice of the chunk in
// registers.  For each (camera, cell) it brings the image box that every
// slice of the chunk reads (the union of the tile's pixel windows over the
// chunk) into shared memory with one cp.async.bulk.tensor load, double
// buffered so that the next cell's box arrives while this one is used; then
// per slice it evaluates the tile's window entries (the same cell_weight of
// the same (pixel, cell) pair as the forward), contracts along t (warp =
// voxel row, lanes over box columns) and then along s from shared memory
// (the separable scheme of Sec. IV-B).  Each image pixel is read from L2
// once per (tile, cell, chunk) instead of once per slice.  Outside the image
// the TMA load fills zeros.  Waits are bounded (status bit 1); a box the
// planner sized too small zeroes that cell's entries and sets status bit 0.
#include <cuda.h>

#include <algorithm>

#include "lt_async.cuh"
#include "lt_beam_math.cuh"
#include "lt_internal.h"

namespace lt {

namespace {

constexpr int AX = 32;          // voxel columns per tile (lanes)
constexpr int AY = 8;           // voxel rows per tile (warps)
constexpr int ASC = 8;          // slices per chunk (register accumulators)
constexpr int AWMAX = 32;       // adjoint window cap (target pixels per voxel per axis)
constexpr long long kAdjWaitPolls = 1LL << 22;

__device__ __forceinline__ void a_mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void a_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool a_try(uint32_t bar, uint32_t parity) {
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
__device__ __forceinline__ bool a_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < kAdjWaitPolls; ++i) {
    if (a_try(bar, parity)) return true;
    if (i > 64) __nanosleep(32);
  }
  return false;
}
__device__ __forceinline__ void a_tma_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ int g_adjoint_status;

// The (camera, cell) pairs a CTA visits, in order: cameras of the batch,
// cells of the subset.
struct UnitCursor {
  int cam, k;
  bool valid;
};
__device__ __forceinline__ void unit_first(const BeamBatch& B, UnitCursor& u) {
  for (; u.cam < B.n_cams; ++u.cam, u.k = 0)
    for (; u.k < B.cam[u.cam].K; ++u.k)
      if (cell_on(B.cam[u.cam].sub_n, B.cam[u.cam].sub_s, u.k)) {
        u.valid = true;
        return;
      }
  u.valid = false;
}
__device__ __forceinline__ void unit_next(const BeamBatch& B, UnitCursor& u) {
  ++u.k;
  unit_first(B, u);
}

// Origin of the image box of (camera, cell) for slices [n0, n0 + ns) of the
// tile (columns [jx0, jx1], rows [jy0, jy1]), by warp 0 (lane = slice), and
// its TMA load by lane 0.  Returns through shared memory: origin and fit.
__device__ __forceinline__ void box_issue(const BeamCam& C, const AdjBatch& A, int cam, int k, int n0, int n_cnt,
                                          int jx0, int jx1, int jy0, int jy1, int frame, int lane, float* box,
                                          uint32_t bar, int* org) {
  int sx_lo = 0x7fffffff, sx_hi = -0x7fffffff, ty_lo = 0x7fffffff, ty_hi = -0x7fffffff;
  if (lane < n_cnt) {
    const SliceParam& p = C.prm[(long long)k * C.nz + n0 + lane];
    const int a0 = window_start(p.s, jx0), a1 = window_start(p.s, jx1);
    const int b0 = window_start(p.t, jy0), b1 = window_start(p.t, jy1);
    sx_lo = min(a0, a1);
    sx_hi = max(a0, a1) + p.wis - 1;
    ty_lo = min(b0, b1);
    ty_hi = max(b0, b1) + p.wit - 1;
  }
  sx_lo = __reduce_min_sync(0xffffffffu, sx_lo);
  sx_hi = __reduce_max_sync(0xffffffffu, sx_hi);
  ty_lo = __reduce_min_sync(0xffffffffu, ty_lo);
  ty_hi = __reduce_max_sync(0xffffffffu, ty_hi);
  const int bx = A.bx[cam], by = A.by[cam];
  const int x0 = sx_lo & ~3;   // a TMA box starts on 16 bytes
  const bool ok = sx_hi - x0 < bx && ty_hi - ty_lo < by;
  if (lane == 0) {
    org[0] = x0;
    org[1] = ty_lo;
    org[2] = ok;
    if (!ok) atomicOr(&g_adjoint_status, 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    a_expect_tx(bar, (uint32_t)(bx * by * sizeof(float)));
    a_tma_3d(smem_addr(box), &A.map[cam], x0, ty_lo, frame * A.zf[cam] + (C.per_cell ? k : 0), bar);
  }
}

__global__ void __launch_bounds__(AX * AY)
beam_adjoint_tma(const __grid_constant__ BeamBatch B, const __grid_constant__ AdjBatch A, float* __restrict__ x,
                 long long x_fs, int accumulate, int tiles_x, int box_floats, int ucols) {
  extern __shared__ __align__(128) unsigned char dsm[];
  float* boxes = reinterpret_cast<float*>(dsm);                   // [2][box_floats]
  float* U = boxes + 2 * (size_t)box_floats;                       // [AY][ucols]
  __shared__ float sw[AWMAX][AX];   // s-window entries of each voxel column
  __shared__ int si[AX];            // first box column of each voxel column's window
  __shared__ float tw[AWMAX][AY];   // t-window entries of each voxel row
  __shared__ int tr[AWMAX][AY];     // their box rows
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int org[2][3];         // box origin (x0, y0) and fit, per buffer
  __shared__ int s_fail;

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nx = B.cam[0].nx, ny = B.cam[0].ny, nz = B.cam[0].nz;
  const int jx0 = (blockIdx.x % tiles_x) * AX;
  const int jy0 = (blockIdx.x / tiles_x) * AY;
  const int jx1 = min(jx0 + AX, nx) - 1;
  const int jy1 = min(jy0 + AY, ny) - 1;
  const int jx = jx0 + lane, jy = jy0 + warp;
  const int n0 = blockIdx.y * ASC;
  const int n_cnt = min(ASC, nz - n0);
  const int frame = blockIdx.z;

  if (threadIdx.x < 2) a_mbar_init(smem_addr(&bars[threadIdx.x]));
  if (threadIdx.x == 0) s_fail = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();

  float acc[ASC];
#pragma unroll
  for (int s = 0; s < ASC; ++s) acc[s] = 0.0f;

  UnitCursor cur{0, 0, false};
  unit_first(B, cur);
  if (cur.valid && warp == 0)
    box_issue(B.cam[cur.cam], A, cur.cam, cur.k, n0, n_cnt, jx0, jx1, jy0, jy1, frame, lane, boxes,
              smem_addr(&bars[0]), org[0]);
  int u = 0;
  bool next_issued = false;
  while (cur.valid) {
    const int buf = u & 1;
    UnitCursor nxt = cur;
    unit_next(B, nxt);
    next_issued = nxt.valid;
    if (nxt.valid && warp == 0)   // the other buffer was released by the last barrier of unit u - 1
      box_issue(B.cam[nxt.cam], A, nxt.cam, nxt.k, n0, n_cnt, jx0, jx1, jy0, jy1, frame, lane,
                boxes + (size_t)(buf ^ 1) * box_floats, smem_addr(&bars[buf ^ 1]), org[buf ^ 1]);
    if (!a_wait(smem_addr(&bars[buf]), (u >> 1) & 1)) {
      if (threadIdx.x == 0) atomicOr(&g_adjoint_status, 2);
      s_fail = 1;
    }
    __syncthreads();
    if (s_fail) {
      // leave no copy in flight behind: wait (bounded) for the box issued next
      if (threadIdx.x == 0 && next_issued) a_wait(smem_addr(&bars[buf ^ 1]), ((u + 1) >> 1) & 1);
      break;
    }
    const BeamCam& C = B.cam[cur.cam];
    const float* box = boxes + (size_t)buf * box_floats;
    const int bx = A.bx[cur.cam];
    const int x0 = org[buf][0], y0 = org[buf][1];
    const bool ok = org[buf][2] != 0;
    for (int s = 0; s < n_cnt; ++s) {
      const SliceParam* p = C.prm + (long long)cur.k * nz + n0 + s;
      const int wis = min(p->wis, AWMAX), wit = min(p->wit, AWMAX);
      // window entries: s (column lane, entry q) and t (row r, entry q)
      for (int task = threadIdx.x; task < AX * wis; task += AX * AY) {
        const int q = task / AX, c = task % AX;
        const int j = jx0 + c;
        const int i0 = window_start(p->s, j);
        float w = 0.0f;
        if (ok && j < nx) {
          int jc;
          float fr;
          footprint_centre(p->s, i0 + q, jc, fr);
          w = cell_weight(j - jc, fr, p->s);
        }
        sw[q][c] = w;
        if (q == 0) si[c] = (ok && j < nx) ? i0 - x0 : 0;
      }
      for (int task = threadIdx.x; task < AY * wit; task += AX * AY) {
        const int q = task / AY, r = task % AY;
        const int j = jy0 + r;
        const int i = window_start(p->t, j) + q;
        float w = 0.0f;
        if (ok && j < ny) {
          int jc;
          float fr;
          footprint_centre(p->t, i, jc, fr);
          w = cell_weight(j - jc, fr, p->t);
        }
        tw[q][r] = w;
        tr[q][r] = (ok && j < ny) ? i - y0 : 0;
      }
      __syncthreads();
      // t-contraction of this warp's voxel row over every box column
      for (int c = lane; c < bx; c += AX) {
        float v = 0.0f;
        for (int q = 0; q < wit; ++q) v = fmaf(tw[q][warp], box[tr[q][warp] * bx + c], v);
        U[warp * ucols + c] = v;
      }
      __syncwarp();
      // s-contraction of this voxel from its row of U
      const float* Ur = U + warp * ucols + si[lane];
      float v = 0.0f;
      for (int q = 0; q < wis; ++q) v = fmaf(sw[q][lane], Ur[q], v);
      acc[s] = fmaf(p->scale, v, acc[s]);
      __syncthreads();
    }
    cur = nxt;
    ++u;
  }
  if (s_fail) return;
  if (jx < nx && jy < ny) {
#pragma unroll
    for (int s = 0; s < ASC; ++s) {
      if (s < n_cnt) {
        float* o = x + (long long)frame * x_fs + ((long long)(n0 + s) * ny + jy) * nx + jx;
        *o = accumulate ? *o + acc[s] : acc[s];
      }
    }
  }
}

size_t adj_smem(int box_floats, int ucols) {
  return (2 * (size_t)box_floats + (size_t)AY * ucols) * sizeof(float);
}

}  // namespace

cudaError_t adjoint_status(int* flags, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(flags, g_adjoint_status, sizeof(int));
  if (e == cudaSuccess && clear) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_adjoint_status, &zero, sizeof(int));
  }
  return e;
}

int adjoint_tile_x() { return AX; }
int adjoint_tile_y() { return AY; }
int adjoint_chunk() { return ASC; }

cudaError_t launch_beam_adjoint_tma(const BeamBatch& b, const AdjBatch& a, float* x, long long x_fs, int accumulate,
                                    cudaStream_t st) {
  const int nx = b.cam[0].nx, ny = b.cam[0].ny, nz = b.cam[0].nz;
  int box = 0, ucols = 32;
  for (int c = 0; c < b.n_cams; ++c) {
    if (b.cam[c].wis > AWMAX || b.cam[c].wit > AWMAX || a.bx[c] <= 0 || a.by[c] <= 0) return cudaErrorInvalidValue;
    box = std::max(box, a.bx[c] * a.by[c]);
    ucols = std::max(ucols, (a.bx[c] + 31) / 32 * 32);
  }
  const int box_floats = (box + 31) / 32 * 32;
  const size_t smem = adj_smem(box_floats, ucols);
  cudaError_t e = cudaFuncSetAttribute(beam_adjoint_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int tiles_x = (nx + AX - 1) / AX, tiles_y = (ny + AY - 1) / AY;
  dim3 grid(tiles_x * tiles_y, (nz + ASC - 1) / ASC, b.frames);
  beam_adjoint_tma<<<grid, AX * AY, smem, st>>>(b, a, x, x_fs, accumulate, tiles_x, box_floats, ucols);
  return cudaGetLastError();
}

}  // namespace lt
