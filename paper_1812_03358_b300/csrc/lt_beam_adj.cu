// Beam integration, gather adjoint, with TMA-staged image boxes and
// plan-built window tables (Sec. IV-A, Sec. IV-B).
//
// x[n][jy][jx] = sum over cameras, cells k, target pixels (it, is) of
// Bt[it][jy] Bs[is][jx] g_k[it][is] x scale_kn: the transpose of the beam
// forward, evaluated as a gather (one writer per voxel, no atomics).  A CTA
// owns a 32 x 8 voxel tile (thread = voxel) and a chunk of SC consecutive
// slices of one frame, and keeps one accumulator per slice of the chunk in
// registers.  For each (camera, cell) one thread brings into shared memory,
// all completing one mbarrier: the image box every slice of the chunk reads
// (the union of the tile's pixel windows over the chunk; one
// cp.async.bulk.tensor load), and the chunk's window entries of the tile's
// columns and rows (two bulk copies of plan-built tables: the same
// cell_weight of the same (pixel, cell) pair as the forward, the t entries
// already multiplied by the slice scale as in the forward).  Buffers are
// double so that the next cell's data arrives while this one is used.  Per
// slice, warp r contracts along t into its own row of U (lanes over pairs of
// box columns, one packed f32x2 FMA per pair) and then every voxel along s
// from that row: no CTA barrier inside a chunk.  The window tables are
// trimmed at plan time to each (tile, slice)'s longest run of nonzero
// entries, so the loops run over the entries the footprints reach rather
// than the camera's largest window.  Each image pixel is read from L2 once
// per (tile, cell, chunk).  Outside the image the TMA load fills zeros.  Waits are bounded
// (status bit 1); a box the planner sized too small is reported when the
// tables are built, and that camera keeps the direct adjoint.
#include <cuda.h>

#include <algorithm>

#include "lt_async.cuh"
#include "lt_beam_math.cuh"
#include "lt_internal.h"

namespace lt {

namespace {

constexpr int AX = 32;          // voxel columns per tile (lanes)
constexpr int AY = 8;           // voxel rows per tile (warps)
constexpr int ASC_MAX = 8;      // slices per chunk (register accumulators): 8, or 4 where 8 slices' box is too big
constexpr int AWMAX = 32;       // adjoint window cap (target pixels per voxel per axis)
constexpr size_t kAdjDoubleMax = 74 * 1024;   // shared bytes up to which the stages are double buffered
constexpr long long kAdjWaitPolls = 1LL << 22;

__device__ int g_adjoint_status;

// Table entry sizes (floats).  S entry (cell, tile column, slice): float
// sw[wqs][AX] (trimmed windows), int i0[AX] (first target pixel of each
// voxel column's window), int {cnt, 0, 0, 0}.  T entry (cell, tile row,
// slice): float weight x slice scale [wqt][AY], int first target row [AY]
// (the entries of a row are consecutive target rows), int {cnt, 0, 0, 0}.
// Both are multiples of 16 bytes (bulk copies).
__host__ __device__ __forceinline__ int s_entry_floats(int wqs) { return wqs * AX + AX + 4; }
__host__ __device__ __forceinline__ int t_entry_floats(int wqt) { return wqt * AY + AY + 4; }

// Column c of a warp's row of U lives at upad(c): one pad word per 32, so
// that the s-contraction's reads (voxel columns about a magnification apart)
// spread over more banks.
__host__ __device__ __forceinline__ int upad(int c) { return c + (c >> 5); }

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
__device__ __forceinline__ void a_bulk(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
               : "memory");
}

// ---------------------------------------------------------------------------
// Plan-time tables (entry layouts at s_entry_floats / t_entry_floats).
// Origin entries (k, chunk, tile): int2 {first box column (a multiple of 4)
// or row, 1 if the chunk's windows fit the planned box}.
// ---------------------------------------------------------------------------
// Window of voxel column jx (or row) trimmed to its nonzero entries: the
// first entry moves to the first nonzero one, and every voxel of the tile
// keeps `cnt` entries, the tile's longest nonzero run; a run starts no later
// than wq - cnt, so that every entry read stays inside the untrimmed window
// (which the planned box covers).  Entries past a voxel's run are zero.
__device__ __forceinline__ void trim_window(int qf, int ql, int wq, int& cnt, int& shift) {
  const int span = ql >= qf ? ql - qf + 1 : 0;
  cnt = __reduce_max_sync(0xffffffffu, span);
  shift = span > 0 ? min(qf, wq - cnt) : 0;
}

__device__ __forceinline__ float s_entry(const SliceParam& p, int jx, int nx, int i0, int q) {
  float w = 0.0f;
  if (q < p.wis && jx < nx) {
    int jc;
    float fr;
    footprint_centre(p.s, i0 + q, jc, fr);
    w = cell_weight(jx - jc, fr, p.s);
  }
  return w;
}

__device__ __forceinline__ float t_entry(const SliceParam& p, int jy, int ny, int i0, int q) {
  float w = 0.0f;
  if (q < p.wit && jy < ny) {
    int jc;
    float fr;
    footprint_centre(p.t, i0 + q, jc, fr);
    w = __fmul_rn(cell_weight(jy - jc, fr, p.t), p.scale);
  }
  return w;
}

// Block (tile column, slice, cell), lane = voxel column.
__global__ void adj_s_table(const SliceParam* __restrict__ prm, int nz, int nx, int wqs, int tiles_x,
                            float* __restrict__ tab) {
  const int tx = blockIdx.x, n = blockIdx.y, k = blockIdx.z, c = threadIdx.x;
  const SliceParam& p = prm[(long long)k * nz + n];
  const int jx = tx * AX + c, je = min(jx, nx - 1);
  float* e = tab + (((long long)k * tiles_x + tx) * nz + n) * s_entry_floats(wqs);
  const int i0 = window_start(p.s, je);
  int qf = wqs, ql = -1;
  for (int q = 0; q < wqs; ++q)
    if (s_entry(p, jx, nx, i0, q) != 0.0f) {
      qf = min(qf, q);
      ql = q;
    }
  int cnt, shift;
  trim_window(qf, ql, wqs, cnt, shift);
  for (int q = 0; q < wqs; ++q) e[q * AX + c] = q < cnt ? s_entry(p, jx, nx, i0, shift + q) : 0.0f;
  int* ei = reinterpret_cast<int*>(e + wqs * AX);
  ei[c] = i0 + shift;
  if (c < 4) ei[AX + c] = c == 0 ? cnt : 0;
}

// Block (tile row, slice, cell), lane r < AY = voxel row.  The window of a
// row is a run of consecutive target rows, so an entry is its weight alone
// (one 4-byte broadcast load per entry in the kernel) and the row's first
// target row is stored once.
__global__ void adj_t_table(const SliceParam* __restrict__ prm, int nz, int ny, int wqt, int tiles_y,
                            float* __restrict__ tab) {
  const int ty = blockIdx.x, n = blockIdx.y, k = blockIdx.z, r = threadIdx.x;
  const SliceParam& p = prm[(long long)k * nz + n];
  int* e = reinterpret_cast<int*>(tab + (((long long)k * tiles_y + ty) * nz + n) * t_entry_floats(wqt));
  const int jy = ty * AY + r, je = min(jy, ny - 1);
  const int i0 = window_start(p.t, je);
  int qf = wqt, ql = -1;
  if (r < AY)
    for (int q = 0; q < wqt; ++q)
      if (t_entry(p, jy, ny, i0, q) != 0.0f) {
        qf = min(qf, q);
        ql = q;
      }
  int cnt, shift;
  trim_window(qf, ql, wqt, cnt, shift);
  if (r < AY) {
    for (int q = 0; q < wqt; ++q) e[q * AY + r] = __float_as_int(q < cnt ? t_entry(p, jy, ny, i0, shift + q) : 0.0f);
    e[wqt * AY + r] = i0 + shift;
  }
  if (r < 4) e[wqt * AY + AY + r] = r == 0 ? cnt : 0;
}

// axis 0: columns (x, s), axis 1: rows (y, t).  Thread = tile; the union of
// the windows of the tile's two end voxels over the chunk's slices.
// Every table row holds wq (the camera's largest window) entries, so the box
// reaches wq pixels past each window start.
__global__ void adj_origins(const SliceParam* __restrict__ prm, int nz, int nvox, int tile, int tiles, int axis,
                            int wq, int box, int sc, int chunks, int2* __restrict__ out, int* __restrict__ bad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int ch = blockIdx.y, k = blockIdx.z;
  if (t >= tiles) return;
  const int j0 = t * tile, j1 = min(j0 + tile, nvox) - 1;
  int lo = 0x7fffffff, hi = -0x7fffffff;
  for (int n = ch * sc; n < min(ch * sc + sc, nz); ++n) {
    const SliceParam& p = prm[(long long)k * nz + n];
    const AxisParam& a = axis == 0 ? p.s : p.t;
    const int s0 = window_start(a, j0), s1 = window_start(a, j1);
    lo = min(lo, min(s0, s1));
    hi = max(hi, max(s0, s1) + wq - 1);
  }
  const int o = axis == 0 ? (lo & ~3) : lo;   // a TMA box starts on 16 bytes
  const int ok = hi - o < box;
  out[((long long)k * chunks + ch) * tiles + t] = make_int2(o, ok);
  if (!ok) atomicOr(bad, 1);
}

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

// Shared-memory stage of one (camera, cell): the image box, then the
// chunk's sc S and T entries (sizes are the launch's largest).
struct AdjStage {
  int box_floats, s_bytes, t_bytes, sc;
  int nbuf;   // 2: double buffered over cells; 1: one stage (large boxes), refilled after each cell
  __host__ __device__ size_t bytes() const {
    return ((size_t)box_floats * 4 + (size_t)sc * s_bytes + (size_t)sc * t_bytes + 127) / 128 * 128;
  }
};

// One thread fills a stage for (camera, cell) and slices [n0, n0 + n_cnt) of
// the tile (tx, ty); the box origin is returned through `org`.
__device__ __forceinline__ void adj_issue(const BeamCam& C, const AdjBatch& A, const AdjStage& L, int cam, int k,
                                          int tx, int ty, int chunk, int n0, int n_cnt, int frame,
                                          unsigned char* stage, uint32_t bar, int* org) {
  const int2 ox = __ldg(&A.ox[cam][((long long)k * A.chunks[cam] + chunk) * A.tiles_x[cam] + tx]);
  const int2 oy = __ldg(&A.oy[cam][((long long)k * A.chunks[cam] + chunk) * A.tiles_y[cam] + ty]);
  org[0] = ox.x;
  org[1] = oy.x;
  const int bx = A.bx[cam], by = A.by[cam];
  const uint32_t sb = (uint32_t)s_entry_floats(A.wqs[cam]) * 4, tb = (uint32_t)t_entry_floats(A.wqt[cam]) * 4;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  a_expect_tx(bar, (uint32_t)(bx * by * 4) + n_cnt * (sb + tb));
  const uint32_t dst = smem_addr(stage);
  a_tma_3d(dst, &A.map[cam], ox.x, oy.x, frame * A.zf[cam] + (C.per_cell ? k : 0), bar);
  const char* s_src = reinterpret_cast<const char*>(A.stab[cam]) +
                      (((long long)k * A.tiles_x[cam] + tx) * C.nz + n0) * (long long)sb;
  const char* t_src = reinterpret_cast<const char*>(A.ttab[cam]) +
                      (((long long)k * A.tiles_y[cam] + ty) * C.nz + n0) * (long long)tb;
  a_bulk(dst + (uint32_t)L.box_floats * 4, s_src, n_cnt * sb, bar);
  a_bulk(dst + (uint32_t)L.box_floats * 4 + (uint32_t)L.sc * (uint32_t)L.s_bytes, t_src, n_cnt * tb, bar);
}

template <int CI, int SC>
__global__ void __launch_bounds__(AX * AY, SC == 4 ? 4 : 3)
beam_adjoint_tma(const __grid_constant__ BeamBatch B, const __grid_constant__ AdjBatch A, float* __restrict__ x,
                 long long x_fs, int accumulate, int tiles_x, AdjStage L, int ucols) {
  extern __shared__ __align__(128) unsigned char dsm[];
  const size_t stage_bytes = L.bytes();
  float* U = reinterpret_cast<float*>(dsm + (size_t)L.nbuf * stage_bytes);    // [AY][ucols], after the stages
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int org[2][2];         // box origin (x0, y0) per buffer
  __shared__ int s_fail;

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nx = B.cam[0].nx, ny = B.cam[0].ny, nz = B.cam[0].nz;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int jx = tx * AX + lane, jy = ty * AY + warp;
  const int chunk = blockIdx.y;
  const int n0 = chunk * SC;
  const int n_cnt = min(SC, nz - n0);
  const int frame = blockIdx.z;

  if (threadIdx.x < 2) a_mbar_init(smem_addr(&bars[threadIdx.x]));
  if (threadIdx.x == 0) s_fail = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();

  float acc[SC];
#pragma unroll
  for (int s = 0; s < SC; ++s) acc[s] = 0.0f;

  UnitCursor cur{0, 0, false};
  unit_first(B, cur);
  if (cur.valid && threadIdx.x == 0)
    adj_issue(B.cam[cur.cam], A, L, cur.cam, cur.k, tx, ty, chunk, n0, n_cnt, frame, dsm, smem_addr(&bars[0]),
              org[0]);
  int u = 0;
  const bool dbl = L.nbuf == 2;
  while (cur.valid) {
    const int buf = dbl ? (u & 1) : 0;
    UnitCursor nxt = cur;
    unit_next(B, nxt);
    if (dbl && nxt.valid && threadIdx.x == 0)   // the other buffer was released by the barrier ending unit u - 1
      adj_issue(B.cam[nxt.cam], A, L, nxt.cam, nxt.k, tx, ty, chunk, n0, n_cnt, frame, dsm + (buf ^ 1) * stage_bytes,
                smem_addr(&bars[buf ^ 1]), org[buf ^ 1]);
    if (!a_wait(smem_addr(&bars[buf]), dbl ? (u >> 1) & 1 : u & 1)) {
      if (threadIdx.x == 0) atomicOr(&g_adjoint_status, 2);
      s_fail = 1;
    }
    __syncthreads();
    if (s_fail) {
      // leave no copy in flight behind: wait (bounded) for the stage issued next
      if (dbl && threadIdx.x == 0 && nxt.valid) a_wait(smem_addr(&bars[buf ^ 1]), ((u + 1) >> 1) & 1);
      break;
    }
    const int cam = cur.cam;
    const unsigned char* stg = dsm + buf * stage_bytes;
    const float* box = reinterpret_cast<const float*>(stg);
    const int bx = A.bx[cam], wqs = A.wqs[cam], wqt = A.wqt[cam];
    const int x0 = org[buf][0], y0 = org[buf][1];
    const float* S0 = reinterpret_cast<const float*>(stg + (size_t)L.box_floats * 4);
    const float* T0 = reinterpret_cast<const float*>(stg + (size_t)L.box_floats * 4 + (size_t)SC * L.s_bytes);
    float* Ur = U + warp * ucols;
#pragma unroll
    for (int s = 0; s < SC; ++s) {
      if (s >= n_cnt) break;
      // t: this warp's voxel row over every box column, two columns per
      // packed FMA; the window's rows are consecutive box rows, each entry
      // one 4-byte broadcast load of its weight
      const float* Tw = T0 + s * t_entry_floats(wqt);
      const int* Ti = reinterpret_cast<const int*>(Tw + wqt * AY);
      const int cnt_t = Ti[AY];
      const float2* row = reinterpret_cast<const float2*>(box + (Ti[warp] - y0) * bx) + lane;   // bx is even
      float2 v[CI];
#pragma unroll
      for (int m = 0; m < CI; ++m) v[m] = make_float2(0.0f, 0.0f);
      for (int q = 0; q < cnt_t; ++q, row += bx >> 1) {
        const float w = Tw[q * AY + warp];
        const float2 w2 = make_float2(w, w);
#pragma unroll
        for (int m = 0; m < CI; ++m)
          if (2 * (lane + AX * m) < bx) v[m] = __ffma2_rn(w2, row[AX * m], v[m]);
      }
#pragma unroll
      for (int m = 0; m < CI; ++m)
        if (2 * (lane + AX * m) < bx) {
          const int c = 2 * (lane + AX * m);
          Ur[upad(c)] = v[m].x;
          Ur[upad(c + 1)] = v[m].y;
        }
      __syncwarp();
      // s: this voxel from its row of U
      const float* S = S0 + s * s_entry_floats(wqs);
      const int* Si = reinterpret_cast<const int*>(S + wqs * AX);
      const int cnt_s = Si[AX], u0 = Si[lane] - x0;
      float a = 0.0f;
      for (int q = 0; q < cnt_s; ++q) a = fmaf(S[q * AX + lane], Ur[upad(u0 + q)], a);
      acc[s] += a;
      __syncwarp();
    }
    __syncthreads();   // this buffer may be refilled
    if (!dbl && nxt.valid && threadIdx.x == 0)
      adj_issue(B.cam[nxt.cam], A, L, nxt.cam, nxt.k, tx, ty, chunk, n0, n_cnt, frame, dsm, smem_addr(&bars[0]),
                org[0]);
    cur = nxt;
    ++u;
  }
  if (s_fail) return;
  if (jx < nx && jy < ny) {
#pragma unroll
    for (int s = 0; s < SC; ++s) {
      if (s < n_cnt) {
        float* o = x + (long long)frame * x_fs + ((long long)(n0 + s) * ny + jy) * nx + jx;
        *o = accumulate ? *o + acc[s] : acc[s];
      }
    }
  }
}

template <int CI, int SC>
const void* adj_kernel() {
  return (const void*)beam_adjoint_tma<CI, SC>;
}
template <int SC>
const void* adj_select_ci(int ci) {
  switch (ci) {
    case 1: return adj_kernel<1, SC>();
    case 2: return adj_kernel<2, SC>();
    case 3: return adj_kernel<3, SC>();
    default: return adj_kernel<4, SC>();
  }
}
const void* adj_select(int ci, int sc) { return sc == 4 ? adj_select_ci<4>(ci) : adj_select_ci<8>(ci); }

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
int adjoint_chunk_max() { return ASC_MAX; }

int adjoint_occupancy(int bx, int by, int wqs, int wqt, int sc) {
  if (sc != 4 && sc != 8) return 0;
  AdjStage L{(bx * by + 31) / 32 * 32, s_entry_floats(wqs) * 4, t_entry_floats(wqt) * 4, sc, 2};
  const int ucols = upad((bx + 31) / 32 * 32);
  if (2 * L.bytes() + (size_t)AY * ucols * sizeof(float) > kAdjDoubleMax) L.nbuf = 1;
  const size_t smem = L.nbuf * L.bytes() + (size_t)AY * ucols * sizeof(float);
  const void* fn = adj_select((bx + 2 * AX - 1) / (2 * AX), sc);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, AX * AY, smem) != cudaSuccess) return 0;
  return n;
}

void adjoint_table_sizes(int K, int nz, int nx, int ny, int wqs, int wqt, int sc, size_t* s_bytes, size_t* t_bytes,
                         size_t* ox_count, size_t* oy_count) {
  const long long tiles_x = (nx + AX - 1) / AX, tiles_y = (ny + AY - 1) / AY, chunks = (nz + sc - 1) / sc;
  *s_bytes = (size_t)K * nz * tiles_x * s_entry_floats(wqs) * 4;
  *t_bytes = (size_t)K * nz * tiles_y * t_entry_floats(wqt) * 4;
  *ox_count = (size_t)K * chunks * tiles_x;
  *oy_count = (size_t)K * chunks * tiles_y;
}

cudaError_t launch_adjoint_tables(const SliceParam* prm, int K, int nz, int nx, int ny, int wqs, int wqt, int bx,
                                  int by, int sc, float* stab, float* ttab, int2* ox, int2* oy, int* bad,
                                  cudaStream_t st) {
  if (sc != 4 && sc != 8) return cudaErrorInvalidValue;
  const int tiles_x = (nx + AX - 1) / AX, tiles_y = (ny + AY - 1) / AY, chunks = (nz + sc - 1) / sc;
  adj_s_table<<<dim3(tiles_x, nz, K), AX, 0, st>>>(prm, nz, nx, wqs, tiles_x, stab);
  adj_t_table<<<dim3(tiles_y, nz, K), 32, 0, st>>>(prm, nz, ny, wqt, tiles_y, ttab);
  adj_origins<<<dim3((tiles_x + 63) / 64, chunks, K), 64, 0, st>>>(prm, nz, nx, AX, tiles_x, 0, wqs, bx, sc, chunks,
                                                                   ox, bad);
  adj_origins<<<dim3((tiles_y + 63) / 64, chunks, K), 64, 0, st>>>(prm, nz, ny, AY, tiles_y, 1, wqt, by, sc, chunks,
                                                                   oy, bad);
  return cudaGetLastError();
}

cudaError_t launch_beam_adjoint_tma(const BeamBatch& b, const AdjBatch& a, int sc, float* x, long long x_fs,
                                    int accumulate, cudaStream_t st) {
  if (sc != 4 && sc != 8) return cudaErrorInvalidValue;
  const int nx = b.cam[0].nx, ny = b.cam[0].ny, nz = b.cam[0].nz;
  int box = 0, bxmax = 4, sb = 16, tb = 16;
  for (int c = 0; c < b.n_cams; ++c) {
    if (a.bx[c] <= 0 || a.by[c] <= 0 || a.wqs[c] > AWMAX || a.wqt[c] > AWMAX) return cudaErrorInvalidValue;
    box = std::max(box, a.bx[c] * a.by[c]);
    bxmax = std::max(bxmax, a.bx[c]);
    sb = std::max(sb, s_entry_floats(a.wqs[c]) * 4);
    tb = std::max(tb, t_entry_floats(a.wqt[c]) * 4);
  }
  if (bxmax > AX * 8) return cudaErrorInvalidValue;
  AdjStage L{(box + 31) / 32 * 32, sb, tb, sc, 2};
  int ucols = upad((bxmax + 31) / 32 * 32);
  // double buffering while it leaves room for three CTAs per SM, else one stage
  if (2 * L.bytes() + (size_t)AY * ucols * sizeof(float) > kAdjDoubleMax) L.nbuf = 1;
  const size_t smem = L.nbuf * L.bytes() + (size_t)AY * ucols * sizeof(float);
  const void* fn = adj_select((bxmax + 2 * AX - 1) / (2 * AX), sc);   // column pairs per lane
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int tiles_x = (nx + AX - 1) / AX;
  const int tiles_y = (ny + AY - 1) / AY;
  const dim3 grid(tiles_x * tiles_y, (nz + sc - 1) / sc, b.frames);
  void* args[] = {(void*)&b, (void*)&a, (void*)&x, (void*)&x_fs, (void*)&accumulate, (void*)&tiles_x, (void*)&L,
                  (void*)&ucols};
  return cudaLaunchKernel(fn, grid, dim3(AX * AY), args, smem, st);
}

}  // namespace lt
