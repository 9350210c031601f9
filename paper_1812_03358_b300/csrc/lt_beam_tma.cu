// Beam integration, forward, with TMA-staged volume bricks (Sec. II-C,
// Sec. III, Sec. IV-B).
//
// For one angular cell k and slice n the slice -> plane transport of a
// 32 x 32 tile of target pixels reads a small rectangle of the slice (a
// "brick": the voxel columns and rows the tile's footprints touch) and
// contracts it twice, along s then along t (eq. xport,sep).  Here every warp
// owns whole slices:
//
//   * a persistent CTA of four warps takes a work item (camera, cell or all
//     cells, tile, frame) from a counter; its warps take every fourth
//     (cell, slice) pair of the item;
//   * three slices ahead of the one it contracts, a warp evaluates the
//     slice's footprint weights (lane = pixel column for s, lane = pixel
//     row for t) into a weight stage in shared memory, derives the brick's
//     origin from them, and lane 0 issues one cp.async.bulk.tensor load of
//     the brick into a ring of four stages guarded by mbarriers, so the
//     volume reaches shared memory through TMA while the warp computes;
//   * the contraction keeps the tile column of every lane in registers: a
//     window of NB s-contracted voxel rows T[k][col] (each computed from the
//     brick once, as the window rolls down the tile) and 32 accumulators,
//     one per pixel row; pixel rows come in groups of four whose taps fall
//     in one band of NB voxel rows, so a group is 4 x NB FMAs against
//     broadcast band weights with no data-dependent register index;
//   * at the end of an item the four warps' partial tiles are summed in a
//     fixed order and written with the mask M (Sec. II-D).
//
// Every matrix entry is the same product of the same footprint integrals as
// in the other beam kernels (lt_beam_math.cuh), so forward and adjoint stay
// exact transposes up to float32 summation order.  Outside the volume the
// TMA load fills zeros, which contribute exact zeros.  Every mbarrier wait is
// bounded: a wait that gives up records bit 1 of the projector status word
// and the CTA stops taking work; a weight stage that would not fit its brick
// or band (the planner sizes both so that this cannot happen) is zeroed and
// records bit 0.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "lt_async.cuh"
#include "lt_beam_math.cuh"
#include "lt_internal.h"

namespace lt {

namespace {

__device__ int g_projector_status;

constexpr int TM_WARPS = 4;
constexpr int TM_STAGES = 4;
constexpr int TM_AHEAD = TM_STAGES - 1;
constexpr unsigned FULL = 0xffffffffu;
constexpr long long kTmaWaitPolls = 1LL << 22;   // polls (with back-off) before a wait gives up

template <int W, int NB>
struct __align__(16) WeightStage {
  float wl[32][NB];   // band weights of each pixel row (t-weight x slice scale at its taps), NB per row
  float ws[W][32];    // s-weights of each pixel column
  int sx[32];         // first tap column of each pixel column, relative to the brick
  int base[8];        // first band row of each group of four pixel rows, relative to the brick
  int up;             // 1: band rows ascend with the row group, 0: they descend
  int pad[3];
};

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_init1(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
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
// Bounded wait for phase `parity`; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < kTmaWaitPolls; ++i) {
    if (mbar_try(bar, parity)) return true;
    if (i > 64) __nanosleep(32);
  }
  return false;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// One target pixel's footprint along one axis: first tap (source index) and
// the W tap integrals, as every beam kernel evaluates them.
template <int W>
__device__ __forceinline__ int taps(const AxisParam& ap, int i, float (&w)[W]) {
  int jc;
  float fr;
  footprint_centre(ap, i, jc, fr);
  const int mlo = (int)floorf(fr - ap.Q + 0.5f);
  float Flo = edge_F(mlo, fr, ap);
#pragma unroll
  for (int a = 0; a < W; ++a) {
    const float Fhi = edge_F(mlo + a + 1, fr, ap);
    w[a] = __fsub_rn(Fhi, Flo);
    Flo = Fhi;
  }
  return jc + mlo;
}

// Weights of slice n, cell k for the tile (is0, it0) into stage S; returns the
// brick origin (x0, y0).  Lane = pixel column for s, pixel row for t.
template <int W, int NB>
__device__ __forceinline__ void stage_weights(const SliceParam* p, int is0, int it0, int lane, int bx, int by,
                                              WeightStage<W, NB>& S, int& x0, int& y0) {
  float ws[W], tw[W];
  const int sx0 = taps<W>(p->s, is0 + lane, ws);
  const int ty0 = taps<W>(p->t, it0 + lane, tw);
  const int smin = __reduce_min_sync(FULL, sx0), smax = __reduce_max_sync(FULL, sx0);
  const int tmin = __reduce_min_sync(FULL, ty0), tmax = __reduce_max_sync(FULL, ty0);
  x0 = smin & ~3;   // floor to a multiple of 4 columns: a TMA box starts on 16 bytes
  y0 = tmin;
  int gb = min(ty0, __shfl_xor_sync(FULL, ty0, 1));
  gb = min(gb, __shfl_xor_sync(FULL, gb, 2));   // band start of this lane's group of four rows
  const bool up = __shfl_sync(FULL, ty0, 31) >= __shfl_sync(FULL, ty0, 0);
  const int g_next = __shfl_down_sync(FULL, gb, 4);
  bool ok = smax + W - 1 - x0 < bx && tmax - tmin + NB <= by && ty0 + W - 1 - gb < NB;
  if (lane < 28) ok = ok && (up ? g_next >= gb : g_next <= gb);
  ok = __all_sync(FULL, ok);
  if (!ok && lane == 0) atomicOr(&g_projector_status, 1);
  const float scale = p->scale;
#pragma unroll
  for (int a = 0; a < W; ++a) S.ws[a][lane] = ok ? ws[a] : 0.0f;
  S.sx[lane] = ok ? sx0 - x0 : 0;
  float wl[NB];
#pragma unroll
  for (int m = 0; m < NB; ++m) wl[m] = 0.0f;
  if (ok) {
#pragma unroll
    for (int b = 0; b < W; ++b) {
      const int m = ty0 + b - gb;
      const float v = __fmul_rn(tw[b], scale);
#pragma unroll
      for (int mm = 0; mm < NB; ++mm)
        if (m == mm) wl[mm] = v;
    }
  }
#pragma unroll
  for (int q = 0; q < NB / 4; ++q)
    reinterpret_cast<float4*>(S.wl[lane])[q] = make_float4(wl[4 * q], wl[4 * q + 1], wl[4 * q + 2], wl[4 * q + 3]);
  if ((lane & 3) == 0) S.base[lane >> 2] = ok ? gb - y0 : 0;
  if (lane == 0) S.up = ok ? (int)up : 1;
}

// s-contraction of brick row `row` for this lane's pixel column.
template <int W>
__device__ __forceinline__ float trow(const float* bc, int off, const float (&ws)[W]) {
  float u = 0.0f;
#pragma unroll
  for (int a = 0; a < W; ++a) u = fmaf(ws[a], bc[off + a], u);
  return u;
}

// t-contraction of one slice into the 32 row accumulators, rolling a window
// of NB s-contracted brick rows down (UP) or up the tile's row groups.
template <int W, int NB, bool UP>
__device__ __forceinline__ void band_rows(const WeightStage<W, NB>& S, const float* bc, int bx, const float (&ws)[W],
                                          float (&acc)[32]) {
  float R[NB];
  int cur = S.base[UP ? 0 : 7];
#pragma unroll
  for (int m = 0; m < NB; ++m) R[m] = trow<W>(bc, (cur + m) * bx, ws);
#pragma unroll
  for (int gg = 0; gg < 8; ++gg) {
    const int g = UP ? gg : 7 - gg;
    for (int d = S.base[g] - cur; d > 0; --d) {   // uniform across the warp
#pragma unroll
      for (int m = 0; m < NB - 1; ++m) R[m] = R[m + 1];
      ++cur;
      R[NB - 1] = trow<W>(bc, (cur + NB - 1) * bx, ws);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int row = 4 * g + i;
      const float4* wr = reinterpret_cast<const float4*>(S.wl[row]);
      float a = acc[row];
#pragma unroll
      for (int q = 0; q < NB / 4; ++q) {
        const float4 w = wr[q];
        a = fmaf(w.x, R[4 * q], a);
        a = fmaf(w.y, R[4 * q + 1], a);
        a = fmaf(w.z, R[4 * q + 2], a);
        a = fmaf(w.w, R[4 * q + 3], a);
      }
      acc[row] = a;
    }
  }
}

// Position in an item's sequence of (cell, slice) pairs: cells k of
// [k, k_end) that belong to the subset, slices [n, n1) of each.
struct PairCursor {
  int k, n, n1, k_end;
  bool valid;
};

__device__ __forceinline__ void cursor_range(const BeamCam& C, int ts, int tt, PairCursor& c) {
  while (c.k < c.k_end) {
    if (cell_on(C.sub_n, C.sub_s, c.k)) {
      const int2 rs = C.srange[c.k * C.tiles_s + ts];
      const int2 rt = C.trange[c.k * C.tiles_t + tt];
      c.n = max(rs.x, rt.x);
      c.n1 = min(rs.y, rt.y);
      if (c.n < c.n1) {
        c.valid = true;
        return;
      }
    }
    ++c.k;
  }
  c.valid = false;
}

__device__ __forceinline__ void cursor_advance(const BeamCam& C, int ts, int tt, PairCursor& c, int steps) {
  while (c.valid && steps > 0) {
    const int left = c.n1 - c.n;
    if (steps < left) {
      c.n += steps;
      return;
    }
    steps -= left;
    ++c.k;
    cursor_range(C, ts, tt, c);
  }
}

// Weights of the cursor's (cell, slice) pair into the warp's next stage, and
// the TMA load of its brick (lane 0); then the cursor moves to the warp's
// next pair.
template <int W, int NB>
__device__ __forceinline__ void issue_pair(const BeamCam& C, const CUtensorMap* map, PairCursor& pf, int is0,
                                           int it0, int lane, int warp, int bx, int by, uint32_t brick_bytes,
                                           int frame, float* bricks, WeightStage<W, NB>* wst, uint64_t* bars,
                                           int bxy, uint32_t& n_issued, int& inflight) {
  const int st = (int)(n_issued % TM_STAGES);
  int x0, y0;
  stage_weights<W, NB>(C.prm + (long long)pf.k * C.nz + pf.n, is0, it0, lane, bx, by, wst[warp * TM_STAGES + st],
                       x0, y0);
  if (lane == 0) {
    const uint32_t bar = smem_addr(bars + warp * TM_STAGES + st);
    fence_proxy_async();   // this stage's earlier generic reads precede the new async-proxy write
    mbar_expect_tx(bar, brick_bytes);
    tma_load_3d(smem_addr(bricks + (size_t)(warp * TM_STAGES + st) * bxy), map, x0, y0, frame * C.nz + pf.n, bar);
  }
  ++n_issued;
  ++inflight;
  cursor_advance(C, is0 / kBeamTileS, it0 / kBeamTileT, pf, TM_WARPS);
}

template <int W, int NB>
__global__ void __launch_bounds__(TM_WARPS * 32)
beam_forward_tma(const __grid_constant__ BeamBatch B, const __grid_constant__ TmaBatch TB,
                 const int4* __restrict__ items, int n_items, int* __restrict__ counter, int bxy) {
  using WS = WeightStage<W, NB>;
  extern __shared__ __align__(128) unsigned char dsm[];
  float* bricks = reinterpret_cast<float*>(dsm);                                   // [warp][stage][bxy]
  WS* wst = reinterpret_cast<WS*>(dsm + (size_t)TM_WARPS * TM_STAGES * bxy * sizeof(float));
  uint64_t* bars = reinterpret_cast<uint64_t*>(wst + TM_WARPS * TM_STAGES);        // [warp][stage]
  float(*red)[32][33] = reinterpret_cast<float(*)[32][33]>(dsm);                    // aliases the bricks
  __shared__ int s_item;
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) s_fail = 0;
  if (threadIdx.x < TM_WARPS * TM_STAGES) mbar_init1(smem_addr(bars + threadIdx.x));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();

  uint32_t n_issued = 0, n_done = 0;   // this warp's brick loads (stage = count % S, phase = count / S)
  bool failed = false;
  const long long total = (long long)n_items * B.frames;

  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const long long it = s_item;
    if (it >= total || s_fail) break;
    const int4 item = items[it / B.frames];
    const int frame = (int)(it % B.frames);
    const BeamCam& C = B.cam[item.x];
    const CUtensorMap* map = &TB.map[item.x];
    const int bx = TB.bx[item.x], by = TB.by[item.x];
    const uint32_t brick_bytes = (uint32_t)(bx * by * sizeof(float));
    const int tile_s = item.z % C.tiles_s;
    const int tile_t = item.z / C.tiles_s;
    const int is0 = tile_s * kBeamTileS;
    const int it0 = tile_t * kBeamTileT;
    const int k_begin = item.y >= 0 ? item.y : 0;
    const int k_end = item.y >= 0 ? item.y + 1 : C.K;
    if (item.y >= 0 && !cell_on(C.sub_n, C.sub_s, item.y)) {   // cell outside the subset: its plane is not written
      __syncthreads();
      continue;
    }

    float acc[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) acc[r] = 0.0f;

    PairCursor pf{k_begin, 0, 0, k_end, false};
    cursor_range(C, tile_s, tile_t, pf);
    cursor_advance(C, tile_s, tile_t, pf, warp);
    int inflight = 0;

    if (!failed) {
      for (int d = 0; d < TM_AHEAD && pf.valid; ++d)
        issue_pair<W, NB>(C, map, pf, is0, it0, lane, warp, bx, by, brick_bytes, frame, bricks, wst, bars, bxy,
                          n_issued, inflight);
      while (inflight > 0) {
        if (pf.valid)
          issue_pair<W, NB>(C, map, pf, is0, it0, lane, warp, bx, by, brick_bytes, frame, bricks, wst, bars, bxy,
                            n_issued, inflight);
        const int st = (int)(n_done % TM_STAGES);
        const bool ready = mbar_wait_bounded(smem_addr(bars + warp * TM_STAGES + st), (n_done / TM_STAGES) & 1);
        if (!ready) {
          failed = true;
          if (lane == 0) {
            atomicOr(&g_projector_status, 2);
            s_fail = 1;
          }
          break;
        }
        const WS& S = wst[warp * TM_STAGES + st];
        float wsr[W];
#pragma unroll
        for (int a = 0; a < W; ++a) wsr[a] = S.ws[a][lane];
        const float* bc = bricks + (size_t)(warp * TM_STAGES + st) * bxy + S.sx[lane];
        if (S.up)
          band_rows<W, NB, true>(S, bc, bx, wsr, acc);
        else
          band_rows<W, NB, false>(S, bc, bx, wsr, acc);
        ++n_done;
        --inflight;
        __syncwarp();
      }
    }

    // the four warps' partial tiles, summed in warp order, masked and written
    __syncthreads();
    if (!s_fail) {
      if (warp > 0) {
#pragma unroll
        for (int r = 0; r < 32; ++r) red[warp - 1][r][lane] = acc[r];
      }
      __syncthreads();
      if (warp == 0) {
        const int is = is0 + lane;
        if (is < C.ns) {
          float* o = C.out + (long long)frame * C.out_fs + (C.per_cell ? (long long)k_begin * C.ns * C.nt : 0);
#pragma unroll
          for (int r = 0; r < 32; ++r) {
            const int itp = it0 + r;
            if (itp < C.nt) {
              float v = acc[r];
#pragma unroll
              for (int g = 0; g < TM_WARPS - 1; ++g) v += red[g][r][lane];
              if (C.mask) v *= C.mask[(long long)itp * C.ns + is];   // M (Sec. II-D)
              o[(long long)itp * C.ns + is] = v;
            }
          }
        }
      }
    }
    __syncthreads();
  }

  // a warp that gave up leaves nothing in flight behind it: wait (bounded)
  // for the loads it issued and did not consume
  if (failed) {
    for (uint32_t q = n_done; q < n_issued; ++q)
      mbar_wait_bounded(smem_addr(bars + warp * TM_STAGES + (q % TM_STAGES)), (q / TM_STAGES) & 1);
  }
}

template <int W, int NB>
const void* tma_kernel() {
  return (const void*)beam_forward_tma<W, NB>;
}

const void* tma_select(int w, int nb) {
  if (nb <= 4) {
    switch (w) {
      case 2: return tma_kernel<2, 4>();
      case 3: return tma_kernel<3, 4>();
      default: return tma_kernel<4, 4>();
    }
  }
  switch (w) {
    case 2: return tma_kernel<2, 8>();
    case 3: return tma_kernel<3, 8>();
    default: return tma_kernel<4, 8>();
  }
}

size_t weight_stage_bytes(int w, int nb) {
  if (nb <= 4) return w == 2 ? sizeof(WeightStage<2, 4>) : w == 3 ? sizeof(WeightStage<3, 4>) : sizeof(WeightStage<4, 4>);
  return w == 2 ? sizeof(WeightStage<2, 8>) : w == 3 ? sizeof(WeightStage<3, 8>) : sizeof(WeightStage<4, 8>);
}

// cuTensorMapEncodeTiled from the driver, found once through the runtime.
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled g_encode = nullptr;
std::once_flag g_encode_once;

EncodeTiled encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<EncodeTiled>(fn);
  });
  return g_encode;
}

}  // namespace

bool tma_forward_available() { return encoder() != nullptr; }

cudaError_t projector_status(int* flags, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(flags, g_projector_status, sizeof(int));
  if (e == cudaSuccess && clear) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_projector_status, &zero, sizeof(int));
  }
  return e;
}

bool tma_encode_volume(CUtensorMap* map, const float* x, int nx, int ny, int nz_total, int bx, int by) {
  EncodeTiled enc = encoder();
  if (!enc || !x || (reinterpret_cast<uintptr_t>(x) & 15) || (nx & 3) || bx <= 0 || by <= 0 || bx > 256 ||
      by > 256 || (bx & 3))
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz_total};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(float), (cuuint64_t)nx * ny * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(x), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t tma_forward_smem(int w, int nb, int bxy) {
  return (size_t)TM_WARPS * TM_STAGES * ((size_t)bxy * sizeof(float) + weight_stage_bytes(w, nb)) +
         (size_t)TM_WARPS * TM_STAGES * sizeof(uint64_t);
}

int tma_forward_bxy(int max_brick) {
  // the reduction buffer of three warps' tiles aliases the bricks
  const int red = (TM_WARPS - 1) * 32 * 33;
  int bxy = (max_brick + 31) / 32 * 32;
  while ((long long)TM_WARPS * TM_STAGES * bxy < red) bxy += 32;
  return bxy;
}

int tma_forward_occupancy(int w, int nb, int bxy) {
  const void* fn = tma_select(w, nb);
  const size_t smem = tma_forward_smem(w, nb, bxy);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int nb_ctas = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_ctas, fn, TM_WARPS * 32, smem) != cudaSuccess) return 0;
  return nb_ctas;
}

cudaError_t launch_beam_forward_tma(const BeamBatch& b, const TmaBatch& tb, const int4* items, int n_items,
                                    int* counter, int w, int nb, int bxy, int ctas, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  if (w < 2 || w > 4) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const void* fn = tma_select(w, nb);
  const size_t smem = tma_forward_smem(w, nb, bxy);
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long total = (long long)n_items * b.frames;
  const int grid = (int)std::min<long long>(ctas, total);
  void* args[] = {(void*)&b, (void*)&tb, (void*)&items, (void*)&n_items, (void*)&counter, (void*)&bxy};
  return cudaLaunchKernel(fn, dim3(grid), dim3(TM_WARPS * 32), args, smem, st);
}

}  // namespace lt
