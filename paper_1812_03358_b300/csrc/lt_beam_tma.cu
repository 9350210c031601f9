// Beam integration, forward, with TMA-staged volume bricks (Sec. II-C,
// Sec. III, Sec. IV-B).
//
// For one angular cell k and slice n the slice -> plane transport of a
// 32 x 32 tile of target pixels reads a small rectangle of the slice (a
// "brick": the voxel columns and rows the tile's footprints touch) and
// contracts it twice, along s then along t (eq. xport,sep).  A persistent
// CTA is one producer warp and four consumer warps:
//
//   * the producer takes work items (camera, cell or all cells, tile, frame;
//     long items split into chunks of about 32 pairs) from a counter, in the
//     order of a list sorted longest first, posts each item's pair count in a
//     small record ring, and for every group of four consecutive slices of a
//     cell fills the next stage of a six-stage ring with one
//     cp.async.bulk.tensor load of the four bricks (a box four slices deep)
//     and two bulk copies of the group's footprint-weight table entries
//     (evaluated once per plan), all completing the stage's mbarrier.  Four
//     lanes fill four stages at a time, so the mbarrier round trips overlap;
//   * consumer warp w takes slices w, w + 4, ... of every group.  Per slice it
//     s-contracts every brick row into its own rows of shared memory (lane =
//     pixel column), then t-contracts them.  Footprints of two taps use the
//     per-row form: each lane owns one pixel row of the tile, keeps its 32
//     accumulators in registers and its tap rows' weights and first row in
//     registers, so every load is a conflict-free 8-byte load of two
//     adjacent pixel columns at an address known before the slice starts.
//     Footprints of three or more taps use the band form: a lane owns four
//     pixel rows of eight columns and reads each of the four brick rows of
//     their common band once for all four.  Every two multiply-adds are one
//     packed f32x2 FMA (the same two round-to-nearest FMAs as fmaf);
//   * at the end of an item the four consumers' partial tiles are summed in
//     warp order and written with the mask M (Sec. II-D).
//
// Every matrix entry is the same product of the same footprint integrals as
// in the other beam kernels (lt_beam_math.cuh), so forward and adjoint stay
// exact transposes up to float32 summation order.  Outside the volume the
// TMA load fills zeros, which contribute exact zeros.  Every mbarrier wait is
// bounded: a wait that gives up records bit 1 of the projector status word
// and the CTA stops taking work.  A table entry whose taps would not fit
// its brick is zeroed and reported when the tables are built (the planner
// sizes bricks so that this cannot happen, and a plan whose tables report
// it keeps the direct kernel).
#include <cuda.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "lt_async.cuh"
#include "lt_beam_math.cuh"
#include "lt_host.h"
#include "lt_internal.h"

namespace lt {

namespace {

__device__ int g_projector_status;

constexpr int FC = 4;                   // consumer warps
constexpr int FTHREADS = (FC + 1) * 32; // + the producer warp
constexpr int FG = 4;                   // slices per stage fill
constexpr int FSLOTS = 6;               // stages
constexpr int FRECS = 4;                // item records
// Row stride (floats) of a consumer's s-contracted rows: 34 for the per-row
// t-contraction (a half-warp's 8-byte loads of rows r then sit 17 r apart in
// bank pairs), 42 for the band form (row groups and column groups of a
// half-warp land 5 r + 4 cg apart); rows are reserved at the larger.
constexpr int FTS_ROW = 34, FTS_BAND = 42, FTS_MAX = 42;
constexpr int FEMPTY = 16;              // empty tiles zeroed per work ticket
constexpr int FMAX_BY = 64;             // brick rows the kernel accepts
constexpr unsigned FULL = 0xffffffffu;
constexpr long long kTmaWaitPolls = 1LL << 22;   // polls (with back-off) before a wait gives up

// Weights of one (cell, slice) for a column of 32-pixel tiles (s, lane =
// pixel column) and a row of 32-pixel tiles (t, lane = pixel row), built
// once per plan (beam_weight_tables) in exactly the layout the kernel
// stages in shared memory, so that a bulk copy brings them next to the
// brick.  The brick origins live in separate arrays, slices innermost.
template <int W>
struct __align__(16) SPart {
  float ws[W][32];   // s-weights of each pixel column
  int sx[32];        // first tap column of each pixel column, relative to the brick
};
template <int W>
struct __align__(16) TPart {
  float tw[W][32];   // t-weights x slice scale of each pixel row
  int ty[32];        // first tap row of each pixel row, relative to the brick
};
// Band form of a t-part, for cameras whose four consecutive pixel rows keep
// their taps within FNB brick rows: group g of rows 4g..4g+3 starts at band
// row base[g]; wl[m][g] holds the weights of the group's four rows at band
// row base[g] + m (zero off a row's taps).  A consumer lane then takes four
// pixel rows of eight columns and reads each band row once for the four.
constexpr int FNB = 4;
template <int W>
struct __align__(16) TPartB {
  float4 wl[FNB][8];
  int base[8];
};
template <int W, bool BAND>
using TPartOf = typename std::conditional<BAND, TPartB<W>, TPart<W>>::type;

// Item record: what the producer tells the consumers about the next item.
struct FwdRec {
  int kind;          // kRecItem, kRecEmpty or kRecEnd
  int ticket;
  int L;             // pairs of the item (this chunk's)
  uint32_t g0;       // stage fill count of its first pair
};
constexpr int kRecItem = 0, kRecEmpty = 1, kRecEnd = 2;

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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
// Bounded wait for the phase of parity `parity`; false if it gave up.
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
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
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

// Table entries are grouped by FG consecutive slices: a stage fill brings
// the bricks of one group (one 3-D TMA box, FG planes) and the group's FG
// s- and t-parts (one bulk copy each), so entries are stored with slices
// innermost, [cell][tile][slice] with the slice count rounded up to a
// multiple of FG (padding entries are zero), and the brick origin is one per
// group: the smallest first tap over the group's slices and the tile's
// pixels (columns rounded down to 4, a TMA box starts on 16 bytes).
__host__ __device__ __forceinline__ int padded_slices(int nz) { return (nz + FG - 1) / FG * FG; }

// First pass, block (tile, slice, cell): the footprint weights of one slice
// for a tile column (warp 0, lane = pixel column) and a tile row (warp 1,
// lane = pixel row), with the absolute first taps; the second pass makes
// them relative to the group's origin.
template <int W>
__global__ void __launch_bounds__(64) beam_weight_tables(const SliceParam* __restrict__ prm, int nz, int tiles_s,
                                                         int tiles_t, SPart<W>* __restrict__ stab,
                                                         TPart<W>* __restrict__ ttab) {
  const int tile = blockIdx.x, n = blockIdx.y, k = blockIdx.z;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const SliceParam p = prm[(long long)k * nz + n];
  const long long nzp = padded_slices(nz);
  if (warp == 0 && tile < tiles_s) {
    float w[W];
    SPart<W>& S = stab[((long long)k * tiles_s + tile) * nzp + n];
    S.sx[lane] = taps<W>(p.s, tile * kBeamTileS + lane, w);
#pragma unroll
    for (int a = 0; a < W; ++a) S.ws[a][lane] = w[a];
  }
  if (warp == 1 && tile < tiles_t) {
    float w[W];
    TPart<W>& T = ttab[((long long)k * tiles_t + tile) * nzp + n];
    T.ty[lane] = taps<W>(p.t, tile * kBeamTileT + lane, w);
#pragma unroll
    for (int a = 0; a < W; ++a) T.tw[a][lane] = __fmul_rn(w[a], p.scale);
  }
}

// Second pass, block (tile, group, cell): the group origin of a tile column
// (warp 0) and a tile row (warp 1), and every first tap of the group made
// relative to it.  An entry whose taps would leave the planned brick is
// zeroed and reported in *bad (the planner sizes bricks so that this does
// not happen).  Origins: ox[(k * tiles_s + tile) * groups + group], oy
// likewise.
template <int W>
__global__ void __launch_bounds__(64) beam_group_origins(int nz, int tiles_s, int tiles_t, int bx, int by,
                                                         SPart<W>* __restrict__ stab, TPart<W>* __restrict__ ttab,
                                                         int* __restrict__ ox, int* __restrict__ oy,
                                                         int* __restrict__ bad) {
  const int tile = blockIdx.x, grp = blockIdx.y, k = blockIdx.z;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long nzp = padded_slices(nz), groups = nzp / FG;
  const int n0 = grp * FG, n1 = min(nz, n0 + FG);
  const int tiles = warp == 0 ? tiles_s : tiles_t;
  if (warp > 1 || tile >= tiles) return;
  const long long base = ((long long)k * tiles + tile) * nzp;
  int lo = 0x7fffffff;
  for (int n = n0; n < n1; ++n) lo = min(lo, warp == 0 ? stab[base + n].sx[lane] : ttab[base + n].ty[lane]);
  lo = __reduce_min_sync(FULL, lo);
  const int org = warp == 0 ? (lo & ~3) : lo;
  const int ext = warp == 0 ? bx : by;
  for (int n = n0; n < n1; ++n) {
    int& f = warp == 0 ? stab[base + n].sx[lane] : ttab[base + n].ty[lane];
    const bool ok = __all_sync(FULL, f - org + W - 1 < ext);
    f = ok ? f - org : 0;
#pragma unroll
    for (int a = 0; a < W; ++a) {
      float& v = warp == 0 ? stab[base + n].ws[a][lane] : ttab[base + n].tw[a][lane];
      if (!ok) v = 0.0f;
    }
    if (!ok && lane == 0) atomicOr(bad, 1);
  }
  if (lane == 0) (warp == 0 ? ox : oy)[((long long)k * tiles + tile) * groups + grp] = org;
}

// Second pass of the band t-parts, block (tile row, group, cell), lane =
// pixel row: the group origin as in beam_group_origins, then per slice each
// four-row group's first band row and band weights, from the per-row
// t-parts of the first pass (tin).  A group whose taps do not fit FNB band
// rows, or a row whose taps leave the brick, zeroes that slice's entry and
// is reported in *bad (the planner checks both in FP64).
template <int W>
__global__ void __launch_bounds__(32) beam_group_band(int nz, int tiles_t, int by, const TPart<W>* __restrict__ tin,
                                                      TPartB<W>* __restrict__ tout, int* __restrict__ oy,
                                                      int* __restrict__ bad) {
  const int tile = blockIdx.x, grp = blockIdx.y, k = blockIdx.z, lane = threadIdx.x;
  const long long nzp = padded_slices(nz), groups = nzp / FG;
  const int n0 = grp * FG, n1 = min(nz, n0 + FG);
  const long long base = ((long long)k * tiles_t + tile) * nzp;
  int lo = 0x7fffffff;
  for (int n = n0; n < n1; ++n) lo = min(lo, tin[base + n].ty[lane]);
  lo = __reduce_min_sync(FULL, lo);
  const int g = lane >> 2, r = lane & 3;
  for (int n = n0; n < n1; ++n) {
    const int ty = tin[base + n].ty[lane] - lo;
    int b = min(ty, __shfl_xor_sync(FULL, ty, 1));
    b = min(b, __shfl_xor_sync(FULL, b, 2));
    const bool ok = __all_sync(FULL, ty - b + W <= FNB && ty + W - 1 < by);
    float* wl = reinterpret_cast<float*>(tout[base + n].wl);
#pragma unroll
    for (int m = 0; m < FNB; ++m) {
      const int a = m - (ty - b);
      float v = 0.0f;
#pragma unroll
      for (int aa = 0; aa < W; ++aa)
        if (aa == a) v = tin[base + n].tw[aa][lane];
      wl[(m * 8 + g) * 4 + r] = ok ? v : 0.0f;
    }
    if (r == 0) tout[base + n].base[g] = ok ? b : 0;
    if (!ok && lane == 0) atomicOr(bad, 1);
  }
  if (lane == 0) oy[((long long)k * tiles_t + tile) * groups + grp] = lo;
}

// Byte offset of the origin array behind a camera's table parts.
template <int W>
__host__ __device__ __forceinline__ size_t s_origin_offset(int K, int nz, int tiles_s) {
  return (size_t)K * tiles_s * padded_slices(nz) * sizeof(SPart<W>);
}
template <int W, bool BAND>
__host__ __device__ __forceinline__ size_t t_origin_offset(int K, int nz, int tiles_t) {
  return (size_t)K * tiles_t * padded_slices(nz) * sizeof(TPartOf<W, BAND>);
}

// Slot header written by the producer: the slices [first, first + count) of
// the group that the consumer contracts.
struct FillHdr {
  int first, count, pad[2];
};

// Shared-memory layout: FSLOTS stages of {FG brick planes (plane = floats
// per brick plane, a multiple of 4), FG SParts, FG TParts, header}, the
// consumers' s-contracted rows (FC x tsz floats), one partial tile (32 x 33
// floats) the consumers sum into in warp order, FRECS item records and the
// mbarriers.
template <int W, bool BAND>
struct FwdLayout {
  static constexpr size_t parts = FG * (sizeof(SPart<W>) + sizeof(TPartOf<W, BAND>));
  __host__ __device__ static size_t brick_bytes(int plane) { return ((size_t)FG * plane * 4 + 127) / 128 * 128; }
  __host__ __device__ static size_t stage_bytes(int plane) {
    return (brick_bytes(plane) + parts + sizeof(FillHdr) + 127) / 128 * 128;
  }
  __host__ __device__ static size_t tw_off(int plane) { return FSLOTS * stage_bytes(plane); }
  __host__ __device__ static size_t red_off(int plane, int tsz) { return tw_off(plane) + (size_t)FC * tsz * 4; }
  __host__ __device__ static size_t rec_off(int plane, int tsz) { return red_off(plane, tsz) + 32 * 33 * 4; }
  __host__ __device__ static size_t bar_off(int plane, int tsz) { return rec_off(plane, tsz) + FRECS * sizeof(FwdRec); }
  // full[FSLOTS], empty[FSLOTS], rec_full[FRECS], rec_empty[FRECS], consumer barrier
  static constexpr int n_bars = 2 * FSLOTS + 2 * FRECS + 1;
  __host__ __device__ static size_t bytes(int plane, int tsz) { return bar_off(plane, tsz) + n_bars * 8; }
};

// Slice interval [nlo, nlo + len) in which the footprints of tile (ts, tt)
// meet the volume for cell k (len = 0 outside [0, ke) or the subset).
__device__ __forceinline__ void cell_interval(const BeamCam& C, int ts, int tt, int k, int ke, int& len, int& nlo) {
  len = 0;
  nlo = 0;
  if (k < ke && cell_on(C.sub_n, C.sub_s, k)) {
    const int2 a = C.srange[k * C.tiles_s + ts], b = C.trange[k * C.tiles_t + tt];
    nlo = max(a.x, b.x);
    len = max(0, min(a.y, b.y) - nlo);
  }
}

// Sum of v over the lanes below this one.
__device__ __forceinline__ int exclusive_sum(int v, int lane) {
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  return x - v;
}

// Barrier of the four consumer warps (an mbarrier of FC arrivals, waited
// with a bound): lane 0 arrives after the warp's earlier shared writes.
__device__ __forceinline__ bool consumer_sync(uint32_t bar, uint32_t& uses, int lane) {
  __syncwarp();
  if (lane == 0) mbar_arrive(bar);
  const bool ok = __all_sync(FULL, mbar_wait_bounded(bar, uses & 1));
  ++uses;
  return ok;
}

// Work tickets from *counter: ticket t < n_real * F * chunks is chunk
// t % chunks of unit u = t / chunks, i.e. of (item u / F, frame u % F) among
// the first n_real items (those whose tile meets the volume, listed first);
// the tickets after those each zero FEMPTY (item, frame) tiles of the
// remaining items, which no slice reaches.
//
// Chunks split an item's (cell, slice) sequence into TB.chunks[camera]
// consecutive parts (at most `chunks`) processed by different CTAs, so that
// a workload with few tiles still spreads evenly over the SMs.  Each chunk's
// partial tile goes to scratch[u][chunk]; the CTA that completes a unit's
// last chunk (a per-unit ticket count, reset by that CTA) sums the partials
// in chunk order and writes the tile, so the result does not depend on which
// CTA ran what.
template <int W, bool BAND>
__global__ void __launch_bounds__(FTHREADS, 4)
beam_forward_tma(const __grid_constant__ BeamBatch B, const __grid_constant__ TmaBatch TB,
                 const int4* __restrict__ items, int n_items, int n_real, int* __restrict__ counter, int plane,
                 int tsz, int chunks, float* __restrict__ scratch, int* __restrict__ unit_count) {
  using L = FwdLayout<W, BAND>;
  using TP = TPartOf<W, BAND>;
  constexpr int FTS = BAND ? FTS_BAND : FTS_ROW;
  extern __shared__ __align__(128) unsigned char dsm[];
  const size_t stage_bytes = L::stage_bytes(plane);
  float* tws = reinterpret_cast<float*>(dsm + L::tw_off(plane));
  float(*red)[33] = reinterpret_cast<float(*)[33]>(dsm + L::red_off(plane, tsz));
  FwdRec* recs = reinterpret_cast<FwdRec*>(dsm + L::rec_off(plane, tsz));
  uint64_t* bars = reinterpret_cast<uint64_t*>(dsm + L::bar_off(plane, tsz));
  const uint32_t full0 = smem_addr(bars), empty0 = smem_addr(bars + FSLOTS);
  const uint32_t rfull0 = smem_addr(bars + 2 * FSLOTS), rempty0 = smem_addr(bars + 2 * FSLOTS + FRECS);
  const uint32_t cbar = smem_addr(bars + 2 * FSLOTS + 2 * FRECS);
  __shared__ int s_fail;
  __shared__ int s_last;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < FSLOTS; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int r = 0; r < FRECS; ++r) {
      mbar_init(rfull0 + 8 * r, 1);
      mbar_init(rempty0 + 8 * r, FC);
    }
    mbar_init(cbar, FC);
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();

  const long long real = (long long)n_real * B.frames * chunks;
  const long long empty = (long long)(n_items - n_real) * B.frames;
  const long long total = real + (empty + FEMPTY - 1) / FEMPTY;

  if (warp == FC) {
    // ------------------------------ producer ------------------------------
    // Tickets come from *counter in list order (items longest first); the
    // next ticket is requested when an item starts, so its atomic is done by
    // the time it is needed.  An item's pairs are issued as fills of slice
    // groups (the group's slices in the item, for one cell), in steps of up
    // to four consecutive fills, lane q < 4 filling the stage of fill g + q.
    uint32_t g = 0;   // stage fills issued
    uint32_t r = 0;   // records written
    bool failed = false;
    int next = 0;
    if (lane == 0) next = atomicAdd(counter, 1);
    for (;;) {
      const long long ticket = __shfl_sync(FULL, next, 0);
      if (lane == 0 && ticket < total) next = atomicAdd(counter, 1);
      const int rs = (int)(r % FRECS);
      if (lane == 0 && r >= FRECS && !failed && !mbar_wait_bounded(rempty0 + 8 * rs, (r / FRECS - 1) & 1))
        failed = true;
      int sf = 0;
      if (lane == 0) sf = *(volatile int*)&s_fail;
      failed = __shfl_sync(FULL, (int)failed, 0) != 0;
      const bool stop = failed || ticket >= total || __shfl_sync(FULL, sf, 0) != 0;
      if (stop || ticket >= real) {
        if (lane == 0 && !failed) {
          recs[rs] = FwdRec{stop ? kRecEnd : kRecEmpty, (int)ticket, 0, g};
          mbar_arrive(rfull0 + 8 * rs);
        }
        ++r;
        if (stop) break;
        continue;
      }
      const long long unit = ticket / chunks;
      const int chunk = (int)(ticket % chunks);
      const int4 item = items[unit / B.frames];
      const int frame = (int)(unit % B.frames);
      const BeamCam& C = B.cam[item.x];
      const int cc = TB.chunks[item.x];
      if (chunk >= cc || (item.y >= 0 && !cell_on(C.sub_n, C.sub_s, item.y))) continue;   // nothing to write
      const int ts = item.z % C.tiles_s, tt = item.z / C.tiles_s;
      const int kb = item.y >= 0 ? item.y : 0, ke = item.y >= 0 ? item.y + 1 : C.K;
      const int nzp = padded_slices(C.nz), groups = nzp / FG;
      // The item's pairs: cells k of [kb, ke) in the subset, the slices of
      // each in the tile's interval [nlo, nlo + len), at positions
      // [jk, jk + len) of the item's sequence; the chunk takes positions
      // [j_lo, j_hi).  Lanes over cells.
      int L_all = 0;
      for (int k0 = kb; k0 < ke; k0 += 32) {
        int len, nlo;
        cell_interval(C, ts, tt, k0 + lane, ke, len, nlo);
        L_all += __reduce_add_sync(FULL, len);
      }
      const int j_lo = (int)((long long)L_all * chunk / cc), j_hi = (int)((long long)L_all * (chunk + 1) / cc);
      int n_fills = 0;
      for (int k0 = kb, jb = 0; k0 < ke; k0 += 32) {
        int len, nlo;
        cell_interval(C, ts, tt, k0 + lane, ke, len, nlo);
        const int jk = jb + exclusive_sum(len, lane);
        const int a = max(jk, j_lo), b = min(jk + len, j_hi);
        const int f = b > a ? (nlo + b - jk - 1) / FG - (nlo + a - jk) / FG + 1 : 0;
        n_fills += __reduce_add_sync(FULL, f);
        jb += __reduce_add_sync(FULL, len);
      }
      if (lane == 0) {
        recs[rs] = FwdRec{kRecItem, (int)ticket, n_fills, g};
        mbar_arrive(rfull0 + 8 * rs);
      }
      ++r;
      const int bx = TB.bx[item.x], by = TB.by[item.x];
      const uint32_t tx_bytes = (uint32_t)(FG * bx * by * 4) + (uint32_t)L::parts;
      const CUtensorMap* map = &TB.map[item.x];
      const char* stab = static_cast<const char*>(TB.stab[item.x]);
      const char* ttab = static_cast<const char*>(TB.ttab[item.x]);
      const int* oxa = reinterpret_cast<const int*>(stab + s_origin_offset<W>(C.K, C.nz, C.tiles_s));
      const int* oya = reinterpret_cast<const int*>(ttab + t_origin_offset<W, BAND>(C.K, C.nz, C.tiles_t));
      for (int k0 = kb, jb = 0; k0 < ke && !failed; k0 += 32) {
        int len, nlo;
        cell_interval(C, ts, tt, k0 + lane, ke, len, nlo);
        const int jkl = jb + exclusive_sum(len, lane);
        jb += __reduce_add_sync(FULL, len);
        for (int q = 0; q < 32 && k0 + q < ke && !failed; ++q) {
          const int lq = __shfl_sync(FULL, len, q), nq = __shfl_sync(FULL, nlo, q), jk = __shfl_sync(FULL, jkl, q);
          const int a = max(jk, j_lo), b = min(jk + lq, j_hi);
          if (b <= a) continue;
          const int k = k0 + q;
          const int n_a = nq + a - jk, n_b = nq + b - jk;   // this cell's slices in the chunk
          const int g_a = n_a / FG, g_b = (n_b - 1) / FG;    // its groups, inclusive
          const long long sbase = (long long)k * C.tiles_s + ts, tbase = (long long)k * C.tiles_t + tt;
          for (int gb0 = g_a; gb0 <= g_b && !failed; gb0 += 32) {
            const int cnt = min(32, g_b - gb0 + 1);
            int ox = 0, oy = 0;
            if (lane < cnt) {
              ox = __ldg(oxa + sbase * groups + gb0 + lane);
              oy = __ldg(oya + tbase * groups + gb0 + lane);
            }
            for (int p = 0; p < cnt && !failed; p += 4) {
              const int nb = min(4, cnt - p);
              const int x0 = __shfl_sync(FULL, ox, (p + lane) & 31), y0 = __shfl_sync(FULL, oy, (p + lane) & 31);
              bool ok = true;
              if (lane < nb) {
                const uint32_t gq = g + lane;
                const int slot = (int)(gq % FSLOTS);
                if (gq >= FSLOTS && !mbar_wait_bounded(empty0 + 8 * slot, (gq / FSLOTS - 1) & 1)) {
                  ok = false;
                } else {
                  const int grp = gb0 + p + lane, n0 = grp * FG;
                  unsigned char* stg = dsm + slot * stage_bytes;
                  const uint32_t dst = smem_addr(stg), bar = full0 + 8 * slot;
                  const uint32_t pb = (uint32_t)L::brick_bytes(plane);
                  const int first = max(n_a, n0) - n0;
                  *reinterpret_cast<FillHdr*>(stg + pb + L::parts) = FillHdr{first, min(n_b, n0 + FG) - n0 - first, {0, 0}};
                  fence_proxy_async();   // the stage's earlier generic reads precede the async-proxy writes
                  mbar_expect_tx(bar, tx_bytes);
                  tma_load_3d(dst, map, x0, y0, frame * C.nz + n0, bar);
                  bulk_copy(dst + pb, stab + (sbase * nzp + n0) * sizeof(SPart<W>), FG * (uint32_t)sizeof(SPart<W>), bar);
                  bulk_copy(dst + pb + FG * (uint32_t)sizeof(SPart<W>), ttab + (tbase * nzp + n0) * sizeof(TP),
                            FG * (uint32_t)sizeof(TP), bar);
                }
              }
              failed = !__all_sync(FULL, ok);
              g += (uint32_t)nb;
            }
          }
        }
      }
      if (failed) {
        if (lane == 0) {
          atomicOr(&g_projector_status, 2);
          s_fail = 1;
        }
        break;   // consumers waiting for fills that were not issued give up on their own bounded waits
      }
    }
    // leave no copy in flight behind: wait (bounded) for the last fill of every stage
    if (lane == 0) {
      const uint32_t q0 = g > FSLOTS ? g - FSLOTS : 0;
      for (uint32_t q = q0; q < g; ++q) mbar_wait_bounded(full0 + 8 * (q % FSLOTS), (q / FSLOTS) & 1);
    }
    return;
  }

  // ------------------------------ consumers -------------------------------
  float* Tw = tws + (size_t)warp * tsz;
  // every value these rows ever hold is a finite product: band rows past a
  // camera's brick rows read zeros or an earlier item's rows, times weight 0
  for (int o = lane; o < tsz; o += 32) Tw[o] = 0.0f;
  __syncwarp();
  uint32_t r = 0, cuses = 0;
  for (;;) {
    const int rs = (int)(r % FRECS);
    if (!__all_sync(FULL, mbar_wait_bounded(rfull0 + 8 * rs, (r / FRECS) & 1))) {
      if (lane == 0) {
        atomicOr(&g_projector_status, 2);
        s_fail = 1;
      }
      break;
    }
    const FwdRec rec = recs[rs];
    __syncwarp();
    if (lane == 0) mbar_arrive(rempty0 + 8 * rs);
    ++r;
    if (rec.kind == kRecEnd) break;
    if (rec.kind == kRecEmpty) {   // a batch of tiles no slice reaches: zeros
      const long long e0 = (rec.ticket - real) * FEMPTY;
      for (long long e = e0 + warp; e < e0 + FEMPTY && e < empty; e += FC) {
        const int4 item = items[n_real + e / B.frames];
        const int frame = (int)(e % B.frames);
        const BeamCam& C = B.cam[item.x];
        if (item.y >= 0 && !cell_on(C.sub_n, C.sub_s, item.y)) continue;
        const int is = (item.z % C.tiles_s) * kBeamTileS + lane, it0 = (item.z / C.tiles_s) * kBeamTileT;
        float* o = C.out + (long long)frame * C.out_fs + (C.per_cell ? (long long)item.y * C.ns * C.nt : 0);
        if (is < C.ns)
          for (int i = 0; i < kBeamTileT && it0 + i < C.nt; ++i) o[(long long)(it0 + i) * C.ns + is] = 0.0f;
      }
      continue;
    }
    const long long unit = rec.ticket / chunks;
    const int chunk = (int)(rec.ticket % chunks);
    const int4 item = items[unit / B.frames];
    const int frame = (int)(unit % B.frames);
    const BeamCam& C = B.cam[item.x];
    const int cc = TB.chunks[item.x];
    const int bx = TB.bx[item.x], by = TB.by[item.x];

    float2 acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = make_float2(0.0f, 0.0f);
    bool ok = true;
    for (int j = warp; j < rec.L; j += FC) {
      const uint32_t gg = rec.g0 + (uint32_t)j;
      const int slot = (int)(gg % FSLOTS);
      if (!__all_sync(FULL, mbar_wait_bounded(full0 + 8 * slot, (gg / FSLOTS) & 1))) {
        ok = false;
        break;
      }
      const unsigned char* stg = dsm + slot * stage_bytes;
      const size_t pb = L::brick_bytes(plane);
      const FillHdr hdr = *reinterpret_cast<const FillHdr*>(stg + pb + L::parts);
      const SPart<W>* Sg = reinterpret_cast<const SPart<W>*>(stg + pb);
      const TP* Tg = reinterpret_cast<const TP*>(stg + pb + FG * sizeof(SPart<W>));
      for (int q = hdr.first; q < hdr.first + hdr.count; ++q) {
        const float* brick = reinterpret_cast<const float*>(stg) + q * bx * by;
        const SPart<W>& S = Sg[q];
        const TP& T = Tg[q];
        // s: every brick row for this lane's pixel column, two rows per packed FMA
        {
          float2 ws2[W];
#pragma unroll
          for (int a = 0; a < W; ++a) ws2[a] = make_float2(S.ws[a][lane], S.ws[a][lane]);
          const float* bc = brick + S.sx[lane];
          int row = 0;
#pragma unroll 2
          for (; row + 1 < by; row += 2) {
            float2 u = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int a = 0; a < W; ++a)
              u = __ffma2_rn(ws2[a], make_float2(bc[row * bx + a], bc[(row + 1) * bx + a]), u);
            Tw[row * FTS + lane] = u.x;
            Tw[(row + 1) * FTS + lane] = u.y;
          }
          if (row < by) {
            float u = 0.0f;
#pragma unroll
            for (int a = 0; a < W; ++a) u = fmaf(ws2[a].x, bc[row * bx + a], u);
            Tw[row * FTS + lane] = u;
          }
        }
        __syncwarp();
        if constexpr (BAND) {
          // t, band form: this lane's four pixel rows 4g..4g+3 over columns
          // 8cg..8cg+7; each of the group's FNB band rows read once
          const int g = lane >> 2, cg = lane & 3;
          const int b = T.base[g];
#pragma unroll
          for (int m = 0; m < FNB; ++m) {
            const float4 w = T.wl[m][g];
            const float2* row = reinterpret_cast<const float2*>(Tw + (b + m) * FTS + 8 * cg);
            float2 R[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) R[j] = row[j];
            const float wr[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
              for (int j = 0; j < 4; ++j) acc[rr * 4 + j] = __ffma2_rn(make_float2(wr[rr], wr[rr]), R[j], acc[rr * 4 + j]);
          }
        } else {
          // t: this lane's pixel row over the tile's 32 columns, two per packed FMA
          const int ty = T.ty[lane];
#pragma unroll
          for (int a = 0; a < W; ++a) {
            const float2 w2 = make_float2(T.tw[a][lane], T.tw[a][lane]);
            const float2* row = reinterpret_cast<const float2*>(Tw + (ty + a) * FTS);
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] = __ffma2_rn(w2, row[c], acc[c]);
          }
        }
        __syncwarp();
      }
      if (lane == 0) mbar_arrive(empty0 + 8 * slot);
    }
    int sf = 0;
    if (lane == 0) sf = *(volatile int*)&s_fail;
    if (!ok || __shfl_sync(FULL, sf, 0) != 0) {
      if (lane == 0) {
        if (!ok) atomicOr(&g_projector_status, 2);
        s_fail = 1;
      }
      break;
    }

    // the four consumers' partial tiles, summed in warp order into one
    // shared tile; then either the tile (one chunk) or this chunk's partial,
    // the unit's last chunk summing every partial in chunk order; masked and
    // written.  Warp w finishes tile rows w, w + 4, ... (lane = pixel column).
    for (int w = 0; w < FC; ++w) {
      if (warp == w) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          // accumulator c: pixel row lane, columns 2c, 2c+1 (per-row form), or
          // row 4g + c / 4, columns 8cg + 2 (c % 4) + {0, 1} (band form)
          const int row = BAND ? 4 * (lane >> 2) + c / 4 : lane;
          const int col = BAND ? 8 * (lane & 3) + 2 * (c % 4) : 2 * c;
          red[row][col] = w == 0 ? acc[c].x : red[row][col] + acc[c].x;
          red[row][col + 1] = w == 0 ? acc[c].y : red[row][col + 1] + acc[c].y;
        }
      }
      if (!consumer_sync(cbar, cuses, lane)) ok = false;
    }
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = red[warp + FC * q][lane];
    if (!consumer_sync(cbar, cuses, lane)) ok = false;   // the shared tile is free again
    if (!ok) {
      if (lane == 0) {
        atomicOr(&g_projector_status, 2);
        s_fail = 1;
      }
      break;
    }
    const int ts = item.z % C.tiles_s, tt = item.z / C.tiles_s;
    const int is = ts * kBeamTileS + lane, it0 = tt * kBeamTileT;
    bool write = true;
    if (cc > 1) {
      float* part = scratch + unit * (long long)chunks * 1024;
#pragma unroll
      for (int q = 0; q < 8; ++q) part[chunk * 1024 + (warp + FC * q) * 32 + lane] = v[q];
      __threadfence();
      if (!consumer_sync(cbar, cuses, lane)) ok = false;
      if (ok && warp == 0 && lane == 0) {
        const int done = atomicAdd(&unit_count[unit], 1);
        s_last = done == cc - 1;
        if (s_last) unit_count[unit] = 0;   // ready for the next launch
      }
      if (!consumer_sync(cbar, cuses, lane)) ok = false;
      if (!ok) {
        if (lane == 0) {
          atomicOr(&g_projector_status, 2);
          s_fail = 1;
        }
        break;
      }
      write = s_last;
      if (write) {
        __threadfence();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int row = warp + FC * q;
          float sum = __ldcg(part + row * 32 + lane);
          for (int c = 1; c < cc; ++c) sum += __ldcg(part + c * 1024 + row * 32 + lane);
          v[q] = sum;
        }
      }
    }
    if (write && is < C.ns) {
      const int kb = item.y >= 0 ? item.y : 0;
      float* o = C.out + (long long)frame * C.out_fs + (C.per_cell ? (long long)kb * C.ns * C.nt : 0);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int itp = it0 + warp + FC * q;
        if (itp < C.nt) {
          float val = v[q];
          if (C.mask) val *= C.mask[(long long)itp * C.ns + is];   // M (Sec. II-D)
          o[(long long)itp * C.ns + is] = val;
        }
      }
    }
  }
}

template <int W, bool BAND>
const void* tma_kernel() {
  return (const void*)beam_forward_tma<W, BAND>;
}

const void* tma_select(int w, bool band) {
  switch (w) {
    case 2: return band ? tma_kernel<2, true>() : tma_kernel<2, false>();
    case 3: return band ? tma_kernel<3, true>() : tma_kernel<3, false>();
    default: return band ? tma_kernel<4, true>() : tma_kernel<4, false>();
  }
}

size_t layout_bytes(int w, bool band, int plane, int tsz) {
  if (band)
    return w == 2 ? FwdLayout<2, true>::bytes(plane, tsz) : w == 3 ? FwdLayout<3, true>::bytes(plane, tsz)
                                                                  : FwdLayout<4, true>::bytes(plane, tsz);
  return w == 2 ? FwdLayout<2, false>::bytes(plane, tsz) : w == 3 ? FwdLayout<3, false>::bytes(plane, tsz)
                                                                   : FwdLayout<4, false>::bytes(plane, tsz);
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
  return tma_encode_planes(map, x, nx, ny, nz_total, (long long)nx * ny, bx, by, FG);
}

bool tma_encode_planes(CUtensorMap* map, const float* x, int nx, int ny, int nz_total, long long z_stride, int bx,
                       int by, int bz) {
  EncodeTiled enc = encoder();
  if (!enc || !x || (reinterpret_cast<uintptr_t>(x) & 15) || (nx & 3) || (z_stride & 3) || bx <= 0 || by <= 0 ||
      bx > 256 || by > 256 || (bx & 3) || bz < 1 || bz > 256)
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz_total};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(float), (cuuint64_t)z_stride * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(x), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int W>
size_t table_bytes_w(bool band, int K, int nz, int tiles_s, int tiles_t) {
  const size_t groups = (size_t)padded_slices(nz) / FG;
  const size_t s = s_origin_offset<W>(K, nz, tiles_s) + ((size_t)K * tiles_s * groups * 4 + 127) / 128 * 128;
  const size_t t = (band ? t_origin_offset<W, true>(K, nz, tiles_t) : t_origin_offset<W, false>(K, nz, tiles_t)) +
                   ((size_t)K * tiles_t * groups * 4 + 127) / 128 * 128;
  return (tiles_s > 0 ? s : 0) + (tiles_t > 0 ? t : 0);
}

size_t tma_table_bytes(int w, bool band, int K, int nz, int tiles_s, int tiles_t) {
  return w == 2 ? table_bytes_w<2>(band, K, nz, tiles_s, tiles_t)
                : w == 3 ? table_bytes_w<3>(band, K, nz, tiles_s, tiles_t) : table_bytes_w<4>(band, K, nz, tiles_s, tiles_t);
}

template <int W>
cudaError_t beam_tables_w(const SliceParam* prm, int K, int nz, int tiles_s, int tiles_t, bool band, int bx, int by,
                          void* stab, void* ttab, int* bad, cudaStream_t st) {
  const int tiles = std::max(tiles_s, tiles_t), groups = padded_slices(nz) / FG;
  int* ox = reinterpret_cast<int*>(static_cast<char*>(stab) + s_origin_offset<W>(K, nz, tiles_s));
  // the first pass writes per-row t-parts: into the table itself, or for the
  // band form into a scratch buffer the second pass reads
  TPart<W>* trow = static_cast<TPart<W>*>(ttab);
  if (band) {
    const size_t rb = t_origin_offset<W, false>(K, nz, tiles_t);
    cudaError_t e = device_alloc((void**)&trow, rb);
    if (e == cudaSuccess) e = cudaMemsetAsync(trow, 0, rb, st);
    if (e != cudaSuccess) {
      cudaFree(trow);
      return e;
    }
  }
  beam_weight_tables<W><<<dim3(tiles, nz, K), 64, 0, st>>>(prm, nz, tiles_s, tiles_t, static_cast<SPart<W>*>(stab),
                                                            trow);
  beam_group_origins<W><<<dim3(tiles, groups, K), 64, 0, st>>>(
      nz, tiles_s, band ? 0 : tiles_t, bx, by, static_cast<SPart<W>*>(stab), trow, ox,
      reinterpret_cast<int*>(static_cast<char*>(ttab) + t_origin_offset<W, false>(K, nz, tiles_t)), bad);
  if (band) {
    beam_group_band<W><<<dim3(tiles_t, groups, K), 32, 0, st>>>(
        nz, tiles_t, by, trow, static_cast<TPartB<W>*>(ttab),
        reinterpret_cast<int*>(static_cast<char*>(ttab) + t_origin_offset<W, true>(K, nz, tiles_t)), bad);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(trow);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_beam_tables(const SliceParam* prm, int K, int nz, int tiles_s, int tiles_t, int w, bool band,
                               int bx, int by, void* stab, void* ttab, int* bad, cudaStream_t st) {
  // padding entries (slices past nz in the last group) stay zero
  cudaError_t e = cudaMemsetAsync(stab, 0, tma_table_bytes(w, band, K, nz, tiles_s, 0), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ttab, 0, tma_table_bytes(w, band, K, nz, 0, tiles_t), st);
  if (e != cudaSuccess) return e;
  if (w == 2) return beam_tables_w<2>(prm, K, nz, tiles_s, tiles_t, band, bx, by, stab, ttab, bad, st);
  if (w == 3) return beam_tables_w<3>(prm, K, nz, tiles_s, tiles_t, band, bx, by, stab, ttab, bad, st);
  return beam_tables_w<4>(prm, K, nz, tiles_s, tiles_t, band, bx, by, stab, ttab, bad, st);
}

int tma_forward_group() { return FG; }

int tma_forward_tsz(int max_by) { return (max_by + FNB) * FTS_MAX; }

int tma_forward_band_rows() { return FNB; }

int tma_forward_max_by() { return FMAX_BY; }

int tma_forward_occupancy(int w, bool band, int plane, int tsz) {
  const void* fn = tma_select(w, band);
  const size_t smem = layout_bytes(w, band, plane, tsz);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int nb_ctas = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_ctas, fn, FTHREADS, smem) != cudaSuccess) return 0;
  return nb_ctas;
}

cudaError_t launch_beam_forward_tma(const BeamBatch& b, const TmaBatch& tb, const int4* items, int n_items,
                                    int n_real, int* counter, int w, bool band, int plane, int tsz, int chunks,
                                    float* scratch, int* unit_count, int ctas, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  if (w < 2 || w > 4) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const void* fn = tma_select(w, band);
  const size_t smem = layout_bytes(w, band, plane, tsz);
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (chunks < 1 || (chunks > 1 && (!scratch || !unit_count))) return cudaErrorInvalidValue;
  const long long real = (long long)n_real * b.frames * chunks;
  const long long total = real + ((long long)(n_items - n_real) * b.frames + FEMPTY - 1) / FEMPTY;
  // with more units than resident CTAs, as many CTAs as give every CTA the
  // same number of rounds (the units are listed longest first), so that the
  // last round does not leave most of the grid idle
  long long grid = std::min<long long>(ctas, total);
  if (real > ctas) {
    const long long rounds = (real + ctas - 1) / ctas;
    grid = (real + rounds - 1) / rounds;
  }
  void* args[] = {(void*)&b,     (void*)&tb,  (void*)&items,  (void*)&n_items, (void*)&n_real,  (void*)&counter,
                  (void*)&plane, (void*)&tsz, (void*)&chunks, (void*)&scratch, (void*)&unit_count};
  return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(FTHREADS), args, smem, st);
}

}  // namespace lt
