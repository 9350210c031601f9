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
//   * the footprint weights of every (cell, slice, tile column) and
//     (cell, slice, tile row) are evaluated once per plan into tables
//     (lane = pixel column for s, lane = pixel row for t), together with the
//     brick's origin;
//   * three slices ahead of the one it contracts, lane 0 of a warp fills a
//     stage of a four-stage ring: one cp.async.bulk.tensor load of the
//     brick and two bulk copies of the slice's table entries, all completing
//     one mbarrier, so volume and weights reach shared memory through TMA
//     while the warp computes;
//   * the contraction keeps the tile column of every lane: the s-contracted
//     voxel rows T[k][col] of the brick (each computed once, into the lane's
//     own column of shared memory) and 32 accumulators in registers, one per
//     pixel row; pixel rows come in groups of four whose taps fall in one
//     band of NB voxel rows, so a group is 4 x NB FMAs against broadcast
//     band weights, with every load address known up front;
//   * at the end of an item the four warps' partial tiles are summed in a
//     fixed order and written with the mask M (Sec. II-D).
//
// Every matrix entry is the same product of the same footprint integrals as
// in the other beam kernels (lt_beam_math.cuh), so forward and adjoint stay
// exact transposes up to float32 summation order.  Outside the volume the
// TMA load fills zeros, which contribute exact zeros.  Every mbarrier wait is
// bounded: a wait that gives up records bit 1 of the projector status word
// and the CTA stops taking work.  A table entry whose taps would not fit
// its brick or band is zeroed and reported when the tables are built (the
// planner sizes both so that this cannot happen, and a plan whose tables
// report it keeps the direct kernel).
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
constexpr int TM_STAGES = 3;
constexpr int TM_EMPTY_BATCH = 16;   // empty tiles zeroed per work ticket
constexpr unsigned FULL = 0xffffffffu;
constexpr long long kTmaWaitPolls = 1LL << 22;   // polls (with back-off) before a wait gives up

// Weights of one (cell, slice) for a column of 32-pixel tiles (s) and a row
// of 32-pixel tiles (t), built once per plan (beam_weight_tables) in exactly
// the layout the kernel stages in shared memory, so that a bulk copy brings
// them next to the brick.
template <int W>
struct __align__(16) SPart {
  float ws[W][32];   // s-weights of each pixel column
  int sx[32];        // first tap column of each pixel column, relative to the brick
  int x0;            // brick's first column (a multiple of 4)
  int ok;            // 0: the taps did not fit the planned brick (weights zeroed)
  int pad[2];
};
template <int NB>
struct __align__(16) TPart {
  float wl[32][NB];  // band weights of each pixel row (t-weight x slice scale at its taps)
  int base[8];       // first band row of each group of four pixel rows, relative to the brick
  int y0;            // brick's first row
  int ok;
  int pad[2];
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

// s-part of one (cell, slice, tile column): lane = pixel column.
template <int W>
__device__ __forceinline__ void build_spart(const SliceParam& p, int is0, int lane, int bx, SPart<W>& S, int* bad) {
  float ws[W];
  const int sx0 = taps<W>(p.s, is0 + lane, ws);
  const int smin = __reduce_min_sync(FULL, sx0), smax = __reduce_max_sync(FULL, sx0);
  const int x0 = smin & ~3;   // floor to a multiple of 4 columns: a TMA box starts on 16 bytes
  const bool ok = smax + W - 1 - x0 < bx;
#pragma unroll
  for (int a = 0; a < W; ++a) S.ws[a][lane] = ok ? ws[a] : 0.0f;
  S.sx[lane] = ok ? sx0 - x0 : 0;
  if (lane == 0) {
    S.x0 = x0;
    S.ok = ok;
    S.pad[0] = S.pad[1] = 0;
    if (!ok) atomicOr(bad, 1);
  }
}

// t-part of one (cell, slice, tile row): lane = pixel row.  A group of four
// rows keeps its taps in NB band rows from its smallest first tap.
template <int W, int NB>
__device__ __forceinline__ void build_tpart(const SliceParam& p, int it0, int lane, int by, TPart<NB>& T, int* bad) {
  float tw[W];
  const int ty0 = taps<W>(p.t, it0 + lane, tw);
  const int tmin = __reduce_min_sync(FULL, ty0), tmax = __reduce_max_sync(FULL, ty0);
  int gb = min(ty0, __shfl_xor_sync(FULL, ty0, 1));
  gb = min(gb, __shfl_xor_sync(FULL, gb, 2));
  const bool ok = __all_sync(FULL, tmax - tmin + NB <= by && ty0 + W - 1 - gb < NB);
  float wl[NB];
#pragma unroll
  for (int m = 0; m < NB; ++m) wl[m] = 0.0f;
  if (ok) {
#pragma unroll
    for (int b = 0; b < W; ++b) {
      const int m = ty0 + b - gb;
      const float v = __fmul_rn(tw[b], p.scale);
#pragma unroll
      for (int mm = 0; mm < NB; ++mm)
        if (m == mm) wl[mm] = v;
    }
  }
#pragma unroll
  for (int m = 0; m < NB; ++m) T.wl[lane][m] = wl[m];
  if ((lane & 3) == 0) T.base[lane >> 2] = ok ? gb - tmin : 0;
  if (lane == 0) {
    T.y0 = tmin;
    T.ok = ok;
    T.pad[0] = T.pad[1] = 0;
    if (!ok) atomicOr(bad, 1);
  }
}

// Plan-time tables: block (tile, slice, cell); warp 0 the s-part of tile
// column blockIdx.x, warp 1 the t-part of tile row blockIdx.x.
template <int W, int NB>
__global__ void __launch_bounds__(64) beam_weight_tables(const SliceParam* __restrict__ prm, int nz, int tiles_s,
                                                         int tiles_t, int bx, int by, SPart<W>* __restrict__ stab,
                                                         TPart<NB>* __restrict__ ttab, int* __restrict__ bad) {
  const int tile = blockIdx.x, n = blockIdx.y, k = blockIdx.z;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const SliceParam p = prm[(long long)k * nz + n];
  if (warp == 0 && tile < tiles_s)
    build_spart<W>(p, tile * kBeamTileS, lane, bx, stab[((long long)k * nz + n) * tiles_s + tile], bad);
  if (warp == 1 && tile < tiles_t)
    build_tpart<W, NB>(p, tile * kBeamTileT, lane, by, ttab[((long long)k * nz + n) * tiles_t + tile], bad);
}

// s-contraction of brick row `off` (a row start) for this lane's pixel column.
template <int W>
__device__ __forceinline__ float trow(const float* bc, int off, const float (&ws)[W]) {
  float u = 0.0f;
#pragma unroll
  for (int a = 0; a < W; ++a) u = fmaf(ws[a], bc[off + a], u);
  return u;
}

// One slice of one tile column (this lane's): the s-contraction of every
// brick row into the lane's own column of Tw, then each group of four pixel
// rows against its NB band rows.  Every load's address is known before any
// of them is needed, so the loads of all groups overlap.
template <int W, int NB>
__device__ __forceinline__ void contract_slice(const SPart<W>& S, const TPart<NB>& T, const float* brick, int bx,
                                               int by, float* Tw, int lane, float (&acc)[32]) {
  float ws[W];
#pragma unroll
  for (int a = 0; a < W; ++a) ws[a] = S.ws[a][lane];
  const float* bc = brick + S.sx[lane];
#pragma unroll 2
  for (int k = 0; k < by; ++k) Tw[k * 32] = trow<W>(bc, k * bx, ws);
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    const int b = T.base[g];
    float R[NB];
#pragma unroll
    for (int m = 0; m < NB; ++m) R[m] = Tw[(b + m) * 32];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int row = 4 * g + i;
      const float4* wr = reinterpret_cast<const float4*>(T.wl[row]);
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

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
               : "memory");
}

// Shared-memory layout of the brick-staged forward, per warp: TM_STAGES
// stages of {brick, SPart, TPart}, the lane columns of the s-contracted rows
// (Tw, by_max x 32 floats), and one mbarrier per stage.
template <int W, int NB>
struct StageLayout {
  static constexpr size_t parts = sizeof(SPart<W>) + sizeof(TPart<NB>);
  // 128-byte multiples: every stage's brick starts where a TMA box may land
  __host__ __device__ static size_t stage_bytes(int bxy) {
    return ((size_t)bxy * sizeof(float) + parts + 127) / 128 * 128;
  }
  static size_t bytes(int bxy, int tsz) {
    return (size_t)TM_WARPS * (TM_STAGES * stage_bytes(bxy) + (size_t)tsz * sizeof(float)) +
           (size_t)TM_WARPS * TM_STAGES * sizeof(uint64_t);
  }
};

// Stage fill for the cursor's (cell, slice) pair by lane 0: the pair's table
// parts and its brick, all completing one mbarrier.  (x0, y0), the brick's
// origin, were read from the tables one pair earlier (px, py).
template <int W, int NB>
__device__ __forceinline__ void issue_stage(const CUtensorMap* map, const SPart<W>* S, const TPart<NB>* T,
                                            unsigned char* stage, int bxy, uint32_t brick_bytes, uint32_t bar,
                                            int x0, int y0, int z) {
  fence_proxy_async();   // this stage's earlier generic reads precede the new async-proxy writes
  mbar_expect_tx(bar, brick_bytes + (uint32_t)(sizeof(SPart<W>) + sizeof(TPart<NB>)));
  const uint32_t dst = smem_addr(stage);
  tma_load_3d(dst, map, x0, y0, z, bar);
  bulk_copy(dst + (uint32_t)bxy * 4, S, (uint32_t)sizeof(SPart<W>), bar);
  bulk_copy(dst + (uint32_t)bxy * 4 + (uint32_t)sizeof(SPart<W>), T, (uint32_t)sizeof(TPart<NB>), bar);
}

// Work tickets from *counter: ticket t < n_real * F * chunks is chunk
// t % chunks of unit u = t / chunks, i.e. of (item u / F, frame u % F) among
// the first n_real items (those whose tile meets the volume, listed first);
// the tickets after those each zero TM_EMPTY_BATCH (item, frame) tiles of
// the remaining items, which no slice reaches.
//
// Chunks split an item's (cell, slice) sequence into TB.chunks[camera]
// consecutive parts (at most `chunks`) processed by different CTAs, so that
// a workload with few tiles still spreads evenly over the SMs.  Each chunk's
// partial tile goes to scratch[u][chunk]; the CTA that completes a unit's
// last chunk (a per-unit ticket count, reset by that CTA) sums the partials
// in chunk order and writes the tile, so the result does not depend on which
// CTA ran what.
template <int W, int NB>
__global__ void __launch_bounds__(TM_WARPS * 32, 7)
beam_forward_tma(const __grid_constant__ BeamBatch B, const __grid_constant__ TmaBatch TB,
                 const int4* __restrict__ items, int n_items, int n_real, int* __restrict__ counter, int bxy,
                 int tsz, int chunks, float* __restrict__ scratch, int* __restrict__ unit_count) {
  using L = StageLayout<W, NB>;
  extern __shared__ __align__(128) unsigned char dsm[];
  const size_t stage_bytes = L::stage_bytes(bxy);
  unsigned char* stages = dsm;                                                       // [warp][stage]
  float* tws = reinterpret_cast<float*>(dsm + (size_t)TM_WARPS * TM_STAGES * stage_bytes);   // [warp][tsz]
  uint64_t* bars = reinterpret_cast<uint64_t*>(tws + (size_t)TM_WARPS * tsz);      // [warp][stage]
  float(*red)[32][33] = reinterpret_cast<float(*)[32][33]>(dsm);                    // aliases the stages
  __shared__ int s_item;
  __shared__ int s_fail;
  __shared__ int s_last;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) s_fail = 0;
  if (threadIdx.x < TM_WARPS * TM_STAGES) mbar_init1(smem_addr(bars + threadIdx.x));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();

  unsigned char* my_stages = stages + (size_t)warp * TM_STAGES * stage_bytes;
  float* Tw = tws + (size_t)warp * tsz + lane;
  uint32_t n_issued = 0, n_done = 0;   // this warp's stage fills (stage = count % S, phase = count / S)
  bool failed = false;
  const long long real = (long long)n_real * B.frames * chunks;
  const long long empty = (long long)(n_items - n_real) * B.frames;
  const long long total = real + (empty + TM_EMPTY_BATCH - 1) / TM_EMPTY_BATCH;

  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const long long it = s_item;
    if (it >= total || s_fail) break;
    if (it >= real) {   // a batch of tiles no slice reaches: zeros
      const long long e0 = (it - real) * TM_EMPTY_BATCH;
      for (long long e = e0; e < e0 + TM_EMPTY_BATCH && e < empty; ++e) {
        const int4 item = items[n_real + e / B.frames];
        const int frame = (int)(e % B.frames);
        const BeamCam& C = B.cam[item.x];
        if (item.y >= 0 && !cell_on(C.sub_n, C.sub_s, item.y)) continue;
        const int is0 = (item.z % C.tiles_s) * kBeamTileS, it0 = (item.z / C.tiles_s) * kBeamTileT;
        float* o = C.out + (long long)frame * C.out_fs + (C.per_cell ? (long long)item.y * C.ns * C.nt : 0);
        for (int q = threadIdx.x; q < kBeamTileS * kBeamTileT; q += TM_WARPS * 32) {
          const int r = it0 + q / kBeamTileS, c = is0 + q % kBeamTileS;
          if (r < C.nt && c < C.ns) o[(long long)r * C.ns + c] = 0.0f;
        }
      }
      __syncthreads();   // s_item is rewritten by the next take
      continue;
    }
    const long long unit = it / chunks;
    const int chunk = (int)(it % chunks);
    const int4 item = items[unit / B.frames];
    const int frame = (int)(unit % B.frames);
    const BeamCam& C = B.cam[item.x];
    const int cc = TB.chunks[item.x];
    if (chunk >= cc) {   // this camera splits its items into fewer chunks
      __syncthreads();
      continue;
    }
    const CUtensorMap* map = &TB.map[item.x];
    const SPart<W>* stab = static_cast<const SPart<W>*>(TB.stab[item.x]);
    const TPart<NB>* ttab = static_cast<const TPart<NB>*>(TB.ttab[item.x]);
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

    // this warp's pairs: every TM_WARPS-th (cell, slice) of the item
    // this warp's pairs: every TM_WARPS-th (cell, slice) pair of the chunk,
    // pairs [j_lo, j_hi) of the item's sequence of L pairs
    PairCursor pf{k_begin, 0, 0, k_end, false};
    cursor_range(C, tile_s, tile_t, pf);
    int j_hi = 0x7fffffff, pj = warp;
    if (cc > 1) {
      int L = 0;
      for (PairCursor q = pf; q.valid; ++q.k, cursor_range(C, tile_s, tile_t, q)) L += q.n1 - q.n;
      const int j_lo = (int)((long long)L * chunk / cc);
      j_hi = (int)((long long)L * (chunk + 1) / cc);
      pj = j_lo + warp;
    }
    cursor_advance(C, tile_s, tile_t, pf, pj);
    if (pj >= j_hi) pf.valid = false;
    // the cursor's table parts and brick origin (lane 0 reads the origin one
    // pair before it issues the pair's stage fill)
    const SPart<W>* sp = stab;
    const TPart<NB>* tp = ttab;
    int px = 0, py = 0;
    if (pf.valid) {
      const long long kn = (long long)pf.k * C.nz + pf.n;
      sp = stab + kn * C.tiles_s + tile_s;
      tp = ttab + kn * C.tiles_t + tile_t;
      if (lane == 0) {
        px = __ldg(&sp->x0);
        py = __ldg(&tp->y0);
      }
    }
    int inflight = 0;
    if (!failed) {
      for (;;) {
        while (pf.valid && inflight < TM_STAGES) {
          const int st = (int)(n_issued % TM_STAGES);
          if (lane == 0)
            issue_stage<W, NB>(map, sp, tp, my_stages + st * stage_bytes, bxy, brick_bytes,
                               smem_addr(bars + warp * TM_STAGES + st), px, py, frame * C.nz + pf.n);
          ++n_issued;
          ++inflight;
          cursor_advance(C, tile_s, tile_t, pf, TM_WARPS);
          pj += TM_WARPS;
          if (pj >= j_hi) pf.valid = false;
          if (pf.valid) {
            const long long kn = (long long)pf.k * C.nz + pf.n;
            sp = stab + kn * C.tiles_s + tile_s;
            tp = ttab + kn * C.tiles_t + tile_t;
            if (lane == 0) {
              px = __ldg(&sp->x0);
              py = __ldg(&tp->y0);
            }
          }
        }
        if (inflight == 0) break;
        const int st = (int)(n_done % TM_STAGES);
        if (!mbar_wait_bounded(smem_addr(bars + warp * TM_STAGES + st), (n_done / TM_STAGES) & 1)) {
          failed = true;
          if (lane == 0) {
            atomicOr(&g_projector_status, 2);
            s_fail = 1;
          }
          break;
        }
        const unsigned char* stg = my_stages + st * stage_bytes;
        contract_slice<W, NB>(*reinterpret_cast<const SPart<W>*>(stg + (size_t)bxy * 4),
                              *reinterpret_cast<const TPart<NB>*>(stg + (size_t)bxy * 4 + sizeof(SPart<W>)),
                              reinterpret_cast<const float*>(stg), bx, by, Tw, lane, acc);
        ++n_done;
        --inflight;
        __syncwarp();
      }
    }

    // the four warps' partial tiles, summed in warp order; then either the
    // tile (one chunk) or this chunk's partial, the unit's last chunk summing
    // every partial in chunk order; masked and written
    __syncthreads();
    if (!s_fail) {
      if (warp > 0) {
#pragma unroll
        for (int r = 0; r < 32; ++r) red[warp - 1][r][lane] = acc[r];
      }
      __syncthreads();
      if (warp == 0) {
#pragma unroll
        for (int r = 0; r < 32; ++r) {
#pragma unroll
          for (int g = 0; g < TM_WARPS - 1; ++g) acc[r] += red[g][r][lane];
        }
      }
      bool write = true;
      float* part = scratch + unit * (long long)chunks * 1024;
      if (cc > 1) {
        if (warp == 0) {
#pragma unroll
          for (int r = 0; r < 32; ++r) part[chunk * 1024 + r * 32 + lane] = acc[r];
          __threadfence();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          const int done = atomicAdd(&unit_count[unit], 1);
          s_last = done == cc - 1;
          if (s_last) unit_count[unit] = 0;   // ready for the next launch
        }
        __syncthreads();
        write = s_last;
        if (write && warp == 0) {
          __threadfence();
#pragma unroll
          for (int r = 0; r < 32; ++r) {
            float v = __ldcg(part + r * 32 + lane);
            for (int c = 1; c < cc; ++c) v += __ldcg(part + c * 1024 + r * 32 + lane);
            acc[r] = v;
          }
        }
      }
      if (write && warp == 0) {
        const int is = is0 + lane;
        if (is < C.ns) {
          float* o = C.out + (long long)frame * C.out_fs + (C.per_cell ? (long long)k_begin * C.ns * C.nt : 0);
#pragma unroll
          for (int r = 0; r < 32; ++r) {
            const int itp = it0 + r;
            if (itp < C.nt) {
              float v = acc[r];
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
  // for the fills it issued and did not consume
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

size_t layout_bytes(int w, int nb, int bxy, int tsz) {
  if (nb <= 4)
    return w == 2 ? StageLayout<2, 4>::bytes(bxy, tsz) : w == 3 ? StageLayout<3, 4>::bytes(bxy, tsz)
                                                                : StageLayout<4, 4>::bytes(bxy, tsz);
  return w == 2 ? StageLayout<2, 8>::bytes(bxy, tsz) : w == 3 ? StageLayout<3, 8>::bytes(bxy, tsz)
                                                              : StageLayout<4, 8>::bytes(bxy, tsz);
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
  return tma_encode_planes(map, x, nx, ny, nz_total, (long long)nx * ny, bx, by);
}

bool tma_encode_planes(CUtensorMap* map, const float* x, int nx, int ny, int nz_total, long long z_stride, int bx,
                       int by) {
  EncodeTiled enc = encoder();
  if (!enc || !x || (reinterpret_cast<uintptr_t>(x) & 15) || (nx & 3) || (z_stride & 3) || bx <= 0 || by <= 0 ||
      bx > 256 || by > 256 || (bx & 3))
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz_total};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(float), (cuuint64_t)z_stride * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(x), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t tma_table_bytes(int w, int nb, int K, int nz, int tiles_s, int tiles_t) {
  const size_t sp = w == 2 ? sizeof(SPart<2>) : w == 3 ? sizeof(SPart<3>) : sizeof(SPart<4>);
  const size_t tp = nb <= 4 ? sizeof(TPart<4>) : sizeof(TPart<8>);
  return (size_t)K * nz * ((size_t)tiles_s * sp + (size_t)tiles_t * tp);
}

cudaError_t launch_beam_tables(const SliceParam* prm, int K, int nz, int tiles_s, int tiles_t, int w, int nb, int bx,
                               int by, void* stab, void* ttab, int* bad, cudaStream_t st) {
  const dim3 grid(std::max(tiles_s, tiles_t), nz, K);
#define LT_TABLES(WW, NN)                                                                                    \
  beam_weight_tables<WW, NN><<<grid, 64, 0, st>>>(prm, nz, tiles_s, tiles_t, bx, by,                           \
                                                  static_cast<SPart<WW>*>(stab), static_cast<TPart<NN>*>(ttab), bad)
  if (nb <= 4) {
    if (w == 2) LT_TABLES(2, 4);
    else if (w == 3) LT_TABLES(3, 4);
    else LT_TABLES(4, 4);
  } else {
    if (w == 2) LT_TABLES(2, 8);
    else if (w == 3) LT_TABLES(3, 8);
    else LT_TABLES(4, 8);
  }
#undef LT_TABLES
  return cudaGetLastError();
}

int tma_forward_bxy(int max_brick, int w, int nb) {
  // the reduction buffer of three warps' tiles aliases the stages
  const size_t red = (size_t)(TM_WARPS - 1) * 32 * 33 * sizeof(float);
  int bxy = (max_brick + 31) / 32 * 32;
  const size_t parts = layout_bytes(w, nb, 0, 0) / TM_WARPS / TM_STAGES;   // stage bytes with bxy = 0 (+ bars)
  while ((size_t)TM_WARPS * TM_STAGES * ((size_t)bxy * sizeof(float) + parts) < red) bxy += 32;
  return bxy;
}

int tma_forward_occupancy(int w, int nb, int bxy, int tsz) {
  const void* fn = tma_select(w, nb);
  const size_t smem = layout_bytes(w, nb, bxy, tsz);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int nb_ctas = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_ctas, fn, TM_WARPS * 32, smem) != cudaSuccess) return 0;
  return nb_ctas;
}

cudaError_t launch_beam_forward_tma(const BeamBatch& b, const TmaBatch& tb, const int4* items, int n_items,
                                    int n_real, int* counter, int w, int nb, int bxy, int tsz, int chunks,
                                    float* scratch, int* unit_count, int ctas, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  if (w < 2 || w > 4) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const void* fn = tma_select(w, nb);
  const size_t smem = layout_bytes(w, nb, bxy, tsz);
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (chunks < 1 || (chunks > 1 && (!scratch || !unit_count))) return cudaErrorInvalidValue;
  const long long total = (long long)n_real * b.frames * chunks +
                         ((long long)(n_items - n_real) * b.frames + TM_EMPTY_BATCH - 1) / TM_EMPTY_BATCH;
  const int grid = (int)std::min<long long>(ctas, total);
  void* args[] = {(void*)&b,   (void*)&tb,  (void*)&items,  (void*)&n_items, (void*)&n_real,  (void*)&counter,
                  (void*)&bxy, (void*)&tsz, (void*)&chunks, (void*)&scratch, (void*)&unit_count};
  return cudaLaunchKernel(fn, dim3(grid), dim3(TM_WARPS * 32), args, smem, st);
}

}  // namespace lt
