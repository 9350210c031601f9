// CUDA kernels of the light-transport camera model (sm_103a).
//
// Two operators carry all the work:
//   * beam integration, slice -> image plane (Sec. II-C, Sec. III): for every
//     target pixel i and angular cell k, sum over slices n of
//     scale_kn * sum_{js,jt} Bs[i_s][js] Bt[i_t][jt] x[n][jt][js]
//     (separable transport, eq. xport,sep), used for the single-lens detector
//     and the plenoptic array plane;
//   * the plenoptic array -> detector stage through each microlens
//     (Sec. II-F2, eq. plenoptic,factor).
// Each has a forward kernel (one thread per output pixel) and a gather
// adjoint (one thread per output voxel / array pixel): one writer per output,
// no atomics (Sec. IV).  Forward and adjoint evaluate every matrix entry with
// the same device functions on the same (target, source) pair, so the two are
// exact transposes up to float32 summation order (Sec. IV-A).
#include <algorithm>

#include "lt_beam_math.cuh"
#include "lt_internal.h"

namespace lt {

namespace {

constexpr int WMAX = 8;      // forward window cap: source cells per target pixel per axis
constexpr int WIMAX = 32;    // adjoint window cap: target pixels per source cell per axis
constexpr int MAXC = 16;     // array pixels per lenslet per axis (stage two)

// ---------------------------------------------------------------------------
// Beam integration, forward: one persistent launch for every camera, cell,
// output tile and frame of a plan.  Work items (host-built, longest first)
// name a camera, a cell (or all cells of a single-lens camera, whose image
// sums them) and a 32 x 32 tile of target pixels; resident CTAs take items
// from a counter.  Per item, only the slices of the tile's interval (host
// table: where the tile's footprints can meet the volume) are visited.  The
// CTA's G warp groups (128 threads each) take alternate batches of SB
// slices; for each batch a group evaluates the s-weights of the 32 columns
// and the t-weights of the 32 rows into shared memory (the separable O(S+T)
// weight work of Sec. IV-B, shared by the tile), then each thread (lane =
// column, warp w of the group = rows w, w+4, ..., w+28) accumulates its 8
// pixels from the L1-resident slices.  W is a compile-time window: a weight
// beyond a slice's own window is exactly zero.
// ---------------------------------------------------------------------------
constexpr int FT_S = kBeamTileS;
constexpr int FT_T = kBeamTileT;
constexpr int FT_GTHREADS = 128;
constexpr int FT_ROWS = FT_T / 4;
constexpr int FT_TR = 16;   // voxel rows of a tile's s-contracted slice kept in shared memory

__device__ __forceinline__ void group_barrier(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(FT_GTHREADS) : "memory");
}

template <int W, int SB, int G>
__global__ void __launch_bounds__(G * FT_GTHREADS, 1024 / (G * FT_GTHREADS))
beam_forward_batched(const __grid_constant__ BeamBatch B, const int4* __restrict__ items, int n_items,
                     int* __restrict__ counter) {
  __shared__ float sw[G][SB][W][FT_S];
  __shared__ int sx[G][SB][W][FT_S];
  __shared__ int ty[G][SB][W][FT_T];
  __shared__ float2 tp[G][SB][W][FT_T];  // (t-weight x slice scale, byte offset of its T row)
  __shared__ float red[G > 1 ? G - 1 : 1][FT_T][FT_S + 1];
  __shared__ float T[G][SB][FT_TR][FT_S];
  __shared__ int s_item;

  const int grp = threadIdx.x / FT_GTHREADS;
  const int gt = threadIdx.x - grp * FT_GTHREADS;
  const int lane = gt & 31;
  const int warp = gt >> 5;
  const long long total = (long long)n_items * B.frames;

  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const long long it = s_item;
    if (it >= total) break;
    const int4 item = items[it / B.frames];
    const int frame = (int)(it % B.frames);
    const BeamCam& C = B.cam[item.x];
    const int nx = C.nx, ny = C.ny, nz = C.nz;
    const int tile_s = item.z % C.tiles_s;
    const int tile_t = item.z / C.tiles_s;
    const int is0 = tile_s * FT_S;
    const int it0 = tile_t * FT_T;
    const int k_begin = item.y >= 0 ? item.y : 0;
    const int k_end = item.y >= 0 ? item.y + 1 : C.K;
    const float* xf = C.x + (long long)frame * C.x_fs;
    if (item.y >= 0 && !cell_on(C.sub_n, C.sub_s, item.y)) {   // cell outside the subset: its plane is not written
      __syncthreads();   // s_item is rewritten by the next take
      continue;
    }

    float acc[FT_ROWS];
#pragma unroll
    for (int r = 0; r < FT_ROWS; ++r) acc[r] = 0.0f;

    for (int k = k_begin; k < k_end; ++k) {
      if (!cell_on(C.sub_n, C.sub_s, k)) continue;   // uniform over the CTA
      const int2 rs = C.srange[k * C.tiles_s + tile_s];
      const int2 rt = C.trange[k * C.tiles_t + tile_t];
      const int n0 = max(rs.x, rt.x);
      const int n1 = min(rs.y, rt.y);
      const SliceParam* pk = C.prm + (long long)k * nz;
      for (int nb = n0 + grp * SB; nb < n1; nb += G * SB) {
        // phase A: weights of SB slices x (32 columns + 32 rows); a thread's
        // tasks are independent and unrolled so that their dependent
        // footprint arithmetic interleaves
        static_assert(SB * (FT_S + FT_T) % FT_GTHREADS == 0, "phase A tasks per thread");
#pragma unroll
        for (int ta = 0; ta < SB * (FT_S + FT_T) / FT_GTHREADS; ++ta) {
          const int task = gt + ta * FT_GTHREADS;
          const int sl = task / (FT_S + FT_T);
          const int q = task - sl * (FT_S + FT_T);
          const int n = nb + sl;
          if (n >= n1) continue;
          const SliceParam* p = pk + n;
          const bool s_axis = q < FT_S;
          const AxisParam& ap = s_axis ? p->s : p->t;
          const int lim = s_axis ? nx : ny;
          const int rr = s_axis ? q : q - FT_S;
          int jc;
          float fr;
          footprint_centre(ap, (s_axis ? is0 : it0) + rr, jc, fr);
          const int mlo = (int)floorf(fr - ap.Q + 0.5f);
          float Flo = edge_F(mlo, fr, ap);
#pragma unroll
          for (int a = 0; a < W; ++a) {
            const int j = jc + mlo + a;
            const float Fhi = edge_F(mlo + a + 1, fr, ap);
            float w = __fsub_rn(Fhi, Flo);
            Flo = Fhi;
            if (j < 0 || j >= lim) w = 0.0f;
            const int jj = min(max(j, 0), lim - 1);
            if (s_axis) {
              sw[grp][sl][a][rr] = w;
              sx[grp][sl][a][rr] = jj;
            } else {
              tp[grp][sl][a][rr].x = __fmul_rn(w, p->scale);
              ty[grp][sl][a][rr] = jj;   // voxel row
            }
          }
        }
        group_barrier(1 + grp);
        // phase B.  Voxel rows the batch's pixel rows reach (monotone in the
        // pixel row, so the tile's first and last rows bound them).
        const int nsl = min(SB, n1 - nb);
        int r_lo[SB], nrows_max = 0;
#pragma unroll
        for (int sl = 0; sl < SB; ++sl) {
          r_lo[sl] = 0;
          if (sl < nsl) {
            const int a0 = ty[grp][sl][0][0], a1 = ty[grp][sl][0][FT_T - 1];
            const int b0 = ty[grp][sl][W - 1][0], b1 = ty[grp][sl][W - 1][FT_T - 1];
            r_lo[sl] = min(a0, a1);
            nrows_max = max(nrows_max, max(b0, b1) - r_lo[sl] + 1);
          }
        }
        if (nrows_max <= FT_TR) {
          // B2's operands: t-weight and the byte offset of its (clamped) T row
          for (int e = gt; e < nsl * W * FT_T; e += FT_GTHREADS) {
            const int sl = e / (W * FT_T);
            const int b = (e / FT_T) % W;
            const int row = e % FT_T;
            const int lo = min(ty[grp][sl][0][0], ty[grp][sl][0][FT_T - 1]);   // r_lo of slice sl
            const int tr = min(max(ty[grp][sl][b][row] - lo, 0), nrows_max - 1);
            tp[grp][sl][b][row].y = __int_as_float((sl * FT_TR + tr) * FT_S * 4);
          }
          // B1: s-contraction T[sl][r][col] = sum_a ws[col][a] x[n][r_lo + r][sx_a(col)]
          for (int sl = 0; sl < nsl; ++sl) {
            const float* xs = xf + (long long)(nb + sl) * ny * nx + (long long)r_lo[sl] * nx;
            float wsr[W];
            int sxr[W];
#pragma unroll
            for (int a = 0; a < W; ++a) {
              wsr[a] = sw[grp][sl][a][lane];
              sxr[a] = sx[grp][sl][a][lane];
            }
            // rows past the volume are never referenced by B2 (clamped
            // indices); the warp's rows are unrolled so that all its gathers
            // are in flight together
            const int r_end = min(nrows_max, ny - r_lo[sl]);
            float u[FT_TR / 4];
#pragma unroll
            for (int i = 0; i < FT_TR / 4; ++i) {
              const int r = warp + 4 * i;
              u[i] = 0.0f;
              if (r < r_end) {
                const float* xr = xs + r * nx;
#pragma unroll
                for (int a = 0; a < W; ++a) u[i] = fmaf(wsr[a], __ldg(xr + sxr[a]), u[i]);
              }
            }
#pragma unroll
            for (int i = 0; i < FT_TR / 4; ++i)
              if (warp + 4 * i < r_end) T[grp][sl][warp + 4 * i][lane] = u[i];
          }
          group_barrier(1 + grp);
          // B2: t-contraction per pixel from shared memory
          const char* Tl = reinterpret_cast<const char*>(&T[grp][0][0][0]) + lane * 4;
          for (int sl = 0; sl < nsl; ++sl) {
#pragma unroll
            for (int r = 0; r < FT_ROWS; ++r) {
              const int row = warp + 4 * r;
#pragma unroll
              for (int b = 0; b < W; ++b) {
                const float2 q = tp[grp][sl][b][row];
                acc[r] = fmaf(q.x, *reinterpret_cast<const float*>(Tl + __float_as_int(q.y)), acc[r]);
              }
            }
          }
        } else {
          // direct gather (footprints spanning many voxel rows)
          for (int sl = 0; sl < nsl; ++sl) {
            const int n = nb + sl;
            const float* xs = xf + (long long)n * ny * nx;
            float wsr[W];
            int sxr[W];
#pragma unroll
            for (int a = 0; a < W; ++a) {
              wsr[a] = sw[grp][sl][a][lane];
              sxr[a] = sx[grp][sl][a][lane];
            }
#pragma unroll
            for (int r = 0; r < FT_ROWS; ++r) {
              const int row = warp + 4 * r;
              float v = 0.0f;
#pragma unroll
              for (int b = 0; b < W; ++b) {
                const float* xr = xs + ty[grp][sl][b][row] * nx;
                float u = 0.0f;
#pragma unroll
                for (int a = 0; a < W; ++a) u = fmaf(wsr[a], __ldg(xr + sxr[a]), u);
                v = fmaf(tp[grp][sl][b][row].x, u, v);
              }
              acc[r] = __fadd_rn(acc[r], v);
            }
          }
        }
        group_barrier(1 + grp);
      }
    }

    // combine the groups' partial sums and write the tile
    if (G > 1 && grp > 0) {
#pragma unroll
      for (int r = 0; r < FT_ROWS; ++r) red[grp - 1][warp + 4 * r][lane] = acc[r];
    }
    __syncthreads();
    if (grp == 0) {
      const int is = is0 + lane;
      if (is < C.ns) {
        float* o = C.out + (long long)frame * C.out_fs + (C.per_cell ? (long long)k_begin * C.ns * C.nt : 0);
#pragma unroll
        for (int r = 0; r < FT_ROWS; ++r) {
          const int row = warp + 4 * r;
          const int itp = it0 + row;
          if (itp < C.nt) {
            float v = acc[r];
#pragma unroll
            for (int g = 1; g < G; ++g) v += red[g - 1][row][lane];
            if (C.mask) v *= C.mask[(long long)itp * C.ns + is];   // M (Sec. II-D)
            o[(long long)itp * C.ns + is] = v;
          }
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Beam integration, gather adjoint.  CTA = 32 x 8 voxels of one slice and
// frame; warp 0 / warp 1 evaluate, for each voxel column / row, the window of
// target pixels whose footprints may cover it and the matching entries (the
// same cell_weight of the same (pixel, cell) pair as the forward), then every
// thread gathers its voxel.
// ---------------------------------------------------------------------------
constexpr int AT_S = 32;
constexpr int AT_T = 8;
constexpr int AT_THREADS = 256;
constexpr int AT_UCOLS = 256;   // pixel columns of the t-contracted rows kept in shared memory
constexpr int AT_SN = 2;        // slices per CTA

// t-contraction of one voxel row (one warp): U[c] = sum_b w_b g[off_b + c_lo + c]
// for c < ncols, lane + 32 j holding column c in a register; the (weight,
// row offset) pair of image row b is one shared-memory broadcast.
template <int NJ>
__device__ __forceinline__ void adjoint_t_rows(const float* __restrict__ g, const float2* twi_row, int wit,
                                               int ncols, float* Urow, int lane) {
  float u[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) u[j] = 0.0f;
  for (int b = 0; b < wit; ++b) {
    const float2 wo = twi_row[b * AT_T];
    const float* gr = g + __float_as_int(wo.y) + lane;
#pragma unroll
    for (int j = 0; j < NJ; ++j)
      if (j < NJ - 1 || lane + 32 * j < ncols) u[j] = fmaf(wo.x, __ldg(gr + 32 * j), u[j]);
  }
#pragma unroll
  for (int j = 0; j < NJ; ++j)
    if (j < NJ - 1 || lane + 32 * j < ncols) Urow[lane + 32 * j] = u[j];
}

// Gather adjoint of the batched beam integration over cameras sharing one
// grid.  CTA = 32 x 8 voxels of one slice and frame (lane = voxel column,
// warp = voxel row).  Per (camera, cell): all threads evaluate the windows of
// target pixels whose footprints may cover each voxel column / row and the
// matching entries (the same cell_weight of the same (pixel, cell) pair as
// the forward); then warp r contracts along t for its voxel row with
// coalesced image-row reads, U[r][c] = sum_b Bt[r][b] g[row_b][c_lo + c], and
// each voxel contracts along s from shared memory (the separable O(S+T)
// scheme of Sec. IV-B).  One writer per voxel, no atomics.
__global__ void __launch_bounds__(AT_THREADS)
beam_adjoint_batched(const __grid_constant__ BeamBatch B, float* __restrict__ x, long long x_fs,
                     int accumulate, int tiles_x) {
  __shared__ float sw[WIMAX][AT_S];
  __shared__ float2 twi[WIMAX][AT_T];   // (t-weight, element offset of its image row)
  __shared__ float U[AT_T][AT_UCOLS];

  const int lane = threadIdx.x & 31;
  const int row = threadIdx.x >> 5;
  const int nx = B.cam[0].nx, ny = B.cam[0].ny, nz = B.cam[0].nz;
  const int jx0 = (blockIdx.x % tiles_x) * AT_S;
  const int jy0 = (blockIdx.x / tiles_x) * AT_T;
  const int jx1 = min(jx0 + AT_S, nx) - 1;
  const int jx = jx0 + lane;
  const int frame = blockIdx.z;
  // AT_SN adjacent slices in turn: their footprints cover nearly the same
  // image pixels, so the later slices find them in L1
  const int n_end = min((int)blockIdx.y * AT_SN + AT_SN, nz);
  for (int n = blockIdx.y * AT_SN; n < n_end; ++n) {
    float acc = 0.0f;
    for (int cam = 0; cam < B.n_cams; ++cam) {
      const BeamCam& C = B.cam[cam];
      const int ns = C.ns, nt = C.nt;
      const float* inf = C.in + (long long)frame * C.out_fs;
      for (int k = 0; k < C.K; ++k) {
        if (!cell_on(C.sub_n, C.sub_s, k)) continue;   // uniform over the CTA
        const SliceParam* p = C.prm + (long long)k * nz + n;
        const int wis = p->wis;
        const int wit = p->wit;
        const float* g = inf + (C.per_cell ? (long long)k * ns * nt : 0);
        // pixel columns covering every voxel column's window (monotone in the voxel index)
        const int a0 = window_start(p->s, jx0), a1 = window_start(p->s, jx1);
        const int c_lo = max(min(a0, a1), 0), c_hi = min(max(a0, a1) + wis - 1, ns - 1);
        const int ncols = c_hi - c_lo + 1;
        const bool sep = ncols > 0 && ncols <= AT_UCOLS;
        const int col_off = sep ? c_lo : 0;   // image column of U / the gather's column 0
        // first pixel column of this voxel column's window; entry q reads column i0 + q
        const int i0 = window_start(p->s, jx);
        int flag_s = 0, flag_t = 0;
        // s windows: lane = voxel column, warp r takes window entries r, r+8, ...
        for (int q = row; q < wis; q += AT_T) {
          const int i = i0 + q;
          float w = 0.0f;
          if (i >= 0 && i < ns && jx < nx) {
            int jc;
            float fr;
            footprint_centre(p->s, i, jc, fr);
            w = cell_weight(jx - jc, fr, p->s);
          }
          sw[q][lane] = w;
          flag_s |= (w != 0.0f);
        }
        // t windows: thread t -> voxel row t & 7, entry t >> 3
        for (int tt = threadIdx.x; tt < AT_T * wit; tt += AT_THREADS) {
          const int r = tt & (AT_T - 1), q = tt >> 3;
          const int jy = jy0 + r;
          const int i = window_start(p->t, jy) + q;
          float w = 0.0f;
          if (i >= 0 && i < nt && jy < ny) {
            int jc;
            float fr;
            footprint_centre(p->t, i, jc, fr);
            w = cell_weight(jy - jc, fr, p->t);
          }
          twi[q][r] = make_float2(w, __int_as_float(min(max(i, 0), nt - 1) * ns + col_off));
          flag_t |= (w != 0.0f);
        }
        const int any_s = __syncthreads_or(flag_s);
        const int any_t = __syncthreads_or(flag_t);
        if (any_s && any_t) {
          // a zero weight may pair with a clamped index; every index stays in range
          if (sep) {
            switch ((ncols + 31) >> 5) {
              case 1: adjoint_t_rows<1>(g, &twi[0][row], wit, ncols, U[row], lane); break;
              case 2: adjoint_t_rows<2>(g, &twi[0][row], wit, ncols, U[row], lane); break;
              case 3: adjoint_t_rows<3>(g, &twi[0][row], wit, ncols, U[row], lane); break;
              case 4: adjoint_t_rows<4>(g, &twi[0][row], wit, ncols, U[row], lane); break;
              case 5: adjoint_t_rows<5>(g, &twi[0][row], wit, ncols, U[row], lane); break;
              case 6: adjoint_t_rows<6>(g, &twi[0][row], wit, ncols, U[row], lane); break;
              case 7: adjoint_t_rows<7>(g, &twi[0][row], wit, ncols, U[row], lane); break;
              default: adjoint_t_rows<8>(g, &twi[0][row], wit, ncols, U[row], lane); break;
            }
            __syncwarp();
            const int u0 = i0 - c_lo;
            float v = 0.0f;
            for (int q = 0; q < wis; ++q) v = fmaf(sw[q][lane], U[row][min(max(u0 + q, 0), ncols - 1)], v);
            acc = fmaf(p->scale, v, acc);
          } else {
            float v = 0.0f;
            for (int b = 0; b < wit; ++b) {
              const float2 wo = twi[b][row];
              const float* gr = g + __float_as_int(wo.y);
              float u = 0.0f;
              for (int q = 0; q < wis; ++q) u = fmaf(sw[q][lane], __ldg(gr + min(max(i0 + q, 0), ns - 1)), u);
              v = fmaf(wo.x, u, v);
            }
            acc = fmaf(p->scale, v, acc);
          }
        }
        __syncthreads();
      }
    }
    const int jy = jy0 + row;
    if (jx < nx && jy < ny) {
      float* o = x + (long long)frame * x_fs + ((long long)n * ny + jy) * nx + jx;
      *o = accumulate ? *o + acc : acc;
    }
  }
}

// ---------------------------------------------------------------------------
// Plenoptic stage two.  For one lenslet mu and cell k the transport from the
// lenslet's array block (nr x nc pixels) to its detector window (ndt x nds)
// is the separable product Bt (x) Bs of two small dense matrices
// (eq. xport,sep); both kernels below give one CTA to a (lenslet, frame),
// evaluate Bs and Bt once per cell into shared memory (one footprint centre
// per detector column/row, consecutive cells sharing their common edge), and
// contract in two steps (the O(S+T) scheme of Sec. IV-B).
// ---------------------------------------------------------------------------
// Exact n / d for small operands (n * d < 2^32, d >= 2) by one multiply-high
// with m = ceil(2^32 / d) = floor((2^32 - 1) / d) + 1: n m / 2^32 exceeds
// n / d by less than n / 2^32 < 1 / d, which never reaches the next integer.
// m = 2^32 does not fit for d = 1, which takes the select.
struct SmallDiv {
  uint32_t m, d;
};
__device__ __forceinline__ SmallDiv small_div(uint32_t d) { return {d > 1u ? 0xFFFFFFFFu / d + 1u : 0u, d}; }
__device__ __forceinline__ uint32_t div_of(SmallDiv f, uint32_t n) { return f.d > 1u ? __umulhi(n, f.m) : n; }

constexpr int L2_W = kStage2Window;
constexpr int S2_THREADS = 256;
constexpr int S2_KB = 4;   // cells per pass of the lenslet adjoint
static_assert(MAXC * MAXC <= S2_THREADS, "one block pixel per thread");
static_assert(S2_KB * 64 <= S2_THREADS && 2 * L2_W <= 64, "one footprint task per thread");

// Entries of one detector column or row of a (lenslet, cell): task < nds is
// column dr.x + task, Bs[c][task] = entry (column, array column cc.x + c);
// otherwise row dr.z + task - nds into Bt likewise.  Consecutive array cells
// share their common edge value.
__device__ __forceinline__ void lenslet_weight_task(const LensletParam* L, int4 dr, int2 cc, int2 rr, int task,
                                                    float (*Bs)[L2_W + 1], float (*Bt)[L2_W + 1]) {
  const int nds = dr.y - dr.x + 1;
  const bool s_axis = task < nds;
  const AxisParam& a = s_axis ? L->s : L->t;
  const int q = s_axis ? task : task - nds;
  const int i = s_axis ? dr.x + q : dr.z + q;
  const int j0 = s_axis ? cc.x : rr.x;
  const int n = s_axis ? cc.y - cc.x : rr.y - rr.x;
  int jc;
  float fr;
  footprint_centre(a, i, jc, fr);
  float Flo = edge_F(j0 - jc, fr, a);
  for (int c = 0; c < n; ++c) {
    const float Fhi = edge_F(j0 + c + 1 - jc, fr, a);
    const float w = __fsub_rn(Fhi, Flo);
    Flo = Fhi;
    if (s_axis) Bs[c][q] = w; else Bt[c][q] = w;
  }
}

// One cell of a pass of the lenslet adjoint (shared memory).
struct S2Cell {
  int4 dr;         // detector window (s0, s1, t0, t1), inclusive
  int nds, ndt;
  int dz, dx;      // offset of the window inside the lenslet's union window
  float scale;
  SmallDiv dd;     // division by nds
  int sub;         // cell in the angular subset
  int on;          // in the subset and with a non-empty window
  int cnt;         // nr * nds contraction outputs, 0 when off
};

// Cell table of the pass starting at cell k0 (threads 0 .. S2_KB - 1).
__device__ __forceinline__ void s2_cell_table(const StageTwo& s2, int mu, int nmu, int k0, int4 du, int nr,
                                              S2Cell* cell) {
  const int kk = threadIdx.x;
  if (kk >= S2_KB) return;
  S2Cell cl{};
  const int k = k0 + kk;
  if (k < s2.K) {
    cl.dr = s2.det_range[(long long)k * nmu + mu];
    cl.nds = cl.dr.y - cl.dr.x + 1;
    cl.ndt = cl.dr.w - cl.dr.z + 1;
    cl.sub = cell_on(s2.sub_n, s2.sub_s, k);
    cl.on = cl.sub && cl.nds > 0 && cl.ndt > 0;
    cl.dz = cl.dr.z - du.z;
    cl.dx = cl.dr.x - du.x;
    cl.scale = s2.lens[(long long)k * nmu + mu].scale;
    cl.dd = small_div(cl.on ? cl.nds : 1);
    cl.cnt = cl.on ? nr * cl.nds : 0;
  }
  cell[kk] = cl;
}

// The cell and local index of flat contraction task e (e < the pass's total).
__device__ __forceinline__ int s2_task_cell(const S2Cell* cell, int& o) {
  int kk = 0;
#pragma unroll
  for (int t = 0; t < S2_KB - 1; ++t)
    if (kk == t && o >= cell[t].cnt) {
      o -= cell[t].cnt;
      kk = t + 1;
    }
  return kk;
}

constexpr int L2_THREADS = 128;

// Bs[c][q] = entry (detector column dr.x + q, array column cc.x + c) and
// Bt[r][b] likewise; one task per detector column / row.
__device__ __forceinline__ void lenslet_weights(const LensletParam* L, int4 dr, int2 cc, int2 rr,
                                                float (*Bs)[L2_W + 1], float (*Bt)[L2_W + 1]) {
  const int nds = dr.y - dr.x + 1, ndt = dr.w - dr.z + 1;
  for (int task = threadIdx.x; task < nds + ndt; task += blockDim.x) lenslet_weight_task(L, dr, cc, rr, task, Bs, Bt);
}

// Forward, pass 1: each lenslet's contribution sum_k Bt (x) Bs fa_k on the
// union over cells of its detector windows, written to zbuf (no overlap).
__global__ void __launch_bounds__(L2_THREADS, 16)
stage2_lenslet_forward(const float* __restrict__ fa, StageTwo s2, long long fa_fs, float* __restrict__ zbuf) {
  __shared__ float Bs[MAXC][L2_W + 1];
  __shared__ float Bt[MAXC][L2_W + 1];
  __shared__ float F[MAXC][MAXC + 1];
  __shared__ float W[MAXC][L2_W + 1];
  __shared__ float Z[L2_W * L2_W];
  const int mu = blockIdx.x;
  const int frame = blockIdx.y;
  const int nmu = s2.mla_ns * s2.mla_nt;
  const int2 cc = s2.cols[mu], rr = s2.rows[mu];
  const int nc = cc.y - cc.x, nr = rr.y - rr.x;
  const int4 du = s2.det_union[mu];
  const int nsu = du.y - du.x + 1, ntu = du.w - du.z + 1;
  float* zout = zbuf + ((long long)frame * nmu + mu) * (L2_W * L2_W);
  const long long Na = (long long)s2.arr_ns * s2.arr_nt;
  for (int o = threadIdx.x; o < L2_W * L2_W; o += blockDim.x) Z[o] = 0.0f;
  if (nc > 0 && nr > 0 && nsu > 0 && ntu > 0) {
    // this thread's block pixels (at most MAXC^2 = 2 x L2_THREADS): array
    // index, -1 where another lenslet (or none) owns the pixel, and the
    // position in F; the same for every cell
    static_assert(MAXC * MAXC <= 2 * L2_THREADS, "two block pixels per thread");
    const SmallDiv dc = small_div(nc);
    int pix[2], fix[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int o = threadIdx.x + e * L2_THREADS;
      pix[e] = -1;
      fix[e] = -1;
      if (o < nr * nc) {
        const int r = div_of(dc, o), c = o - r * nc;
        const int px = (rr.x + r) * s2.arr_ns + cc.x + c;
        pix[e] = __ldg(s2.owner + px) == mu ? px : -1;
        fix[e] = r * (MAXC + 1) + c;
      }
    }
    for (int k = 0; k < s2.K; ++k) {
      if (!cell_on(s2.sub_n, s2.sub_s, k)) continue;   // uniform
      const LensletParam* L = s2.lens + (long long)k * nmu + mu;
      const int4 dr = s2.det_range[(long long)k * nmu + mu];
      const int nds = dr.y - dr.x + 1, ndt = dr.w - dr.z + 1;
      if (nds <= 0 || ndt <= 0) continue;   // uniform
      // this lenslet's own pixels, zero elsewhere: loaded before the
      // footprint entries are evaluated so that the two overlap
      const float* fk = fa + (long long)frame * fa_fs + (long long)k * Na;
      float fv[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) fv[e] = pix[e] >= 0 ? __ldg(fk + pix[e]) : 0.0f;
      lenslet_weights(L, dr, cc, rr, Bs, Bt);
      const SmallDiv dd = small_div(nds);
#pragma unroll
      for (int e = 0; e < 2; ++e)
        if (fix[e] >= 0) (&F[0][0])[fix[e]] = fv[e];
      __syncthreads();
      // W[r][q] = sum_c Bs[c][q] F[r][c]
      for (int o = threadIdx.x; o < nr * nds; o += blockDim.x) {
        const int r = div_of(dd, o), q = o - r * nds;
        float w = 0.0f;
        for (int c = 0; c < nc; ++c) w = fmaf(Bs[c][q], F[r][c], w);
        W[r][q] = w;
      }
      __syncthreads();
      // Z[it][is] += scale * sum_r Bt[r][b] W[r][q] over the cell's own
      // window inside the union (entries owned by one thread)
      const float scale = L->scale;
      const int zoff = (dr.z - du.z) * nsu + (dr.x - du.x);
      for (int o = threadIdx.x; o < ndt * nds; o += blockDim.x) {
        const int b = div_of(dd, o), q = o - b * nds;
        const int zi = zoff + b * nsu + q;
        float z = 0.0f;
        for (int r = 0; r < nr; ++r) z = fmaf(Bt[r][b], W[r][q], z);
        Z[zi] = fmaf(scale, z, Z[zi]);
      }
      __syncthreads();
    }
  }
  for (int o = threadIdx.x; o < ntu * nsu; o += blockDim.x) zout[o] = Z[o];
}

// Forward, pass 2: each detector pixel gathers the sub-images that cover it.
__global__ void __launch_bounds__(256)
stage2_gather(const float* __restrict__ zbuf, float* __restrict__ y, StageTwo s2, long long y_fs) {
  const int is = blockIdx.x * 32 + (threadIdx.x & 31);
  const int it = blockIdx.y * 8 + (threadIdx.x >> 5);
  const int frame = blockIdx.z;
  if (is >= s2.det_ns || it >= s2.det_nt) return;
  const int nmu = s2.mla_ns * s2.mla_nt;
  const int2 cs = s2.cand_all_s[is], ct = s2.cand_all_t[it];
  const float* zf = zbuf + (long long)frame * nmu * (L2_W * L2_W);
  float acc = 0.0f;
  if (cs.y - cs.x < 2 && ct.y - ct.x < 2) {
    // at most 2 x 2 candidates (the usual case): their windows, then their
    // sub-image values, each set of loads in flight together; summed in the
    // same (mt, ms) order as the general loop below
    int4 du[4];
    float v[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int mt = ct.x + (c >> 1), ms = cs.x + (c & 1);
      du[c] = make_int4(1, 0, 1, 0);   // covers nothing
      if (mt <= ct.y && ms <= cs.y) du[c] = __ldg(s2.det_union + mt * s2.mla_ns + ms);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int mu = (ct.x + (c >> 1)) * s2.mla_ns + cs.x + (c & 1);
      const bool in = is >= du[c].x && is <= du[c].y && it >= du[c].z && it <= du[c].w;
      v[c] = in ? __ldg(zf + (long long)mu * (L2_W * L2_W) + (it - du[c].z) * (du[c].y - du[c].x + 1) + (is - du[c].x))
                : 0.0f;
      du[c].x = in;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (du[c].x) acc += v[c];
  } else {
    for (int mt = ct.x; mt <= ct.y; ++mt)
      for (int ms = cs.x; ms <= cs.y; ++ms) {
        const int mu = mt * s2.mla_ns + ms;
        const int4 du = s2.det_union[mu];
        if (is < du.x || is > du.y || it < du.z || it > du.w) continue;
        const int nsu = du.y - du.x + 1;
        acc += __ldg(zf + (long long)mu * (L2_W * L2_W) + (it - du.z) * nsu + (is - du.x));
      }
  }
  y[(long long)frame * y_fs + (long long)it * s2.det_ns + is] = acc;
}

// Adjoint: fa_k[jt][js] = M * scale * sum_b sum_q Bt[r][b] Bs[c][q] y[dr.z+b][dr.x+q]
// for the lenslet's own block (a gather: every array pixel has one lenslet).
// The lenslet's union window of y is staged once; the cells go S2_KB at a
// time through three phases (footprint entries; U = Bt^T Y for every cell;
// each thread's block pixel for every cell), one block barrier per phase.
__global__ void __launch_bounds__(S2_THREADS, 8)
stage2_lenslet_adjoint(const float* __restrict__ y, float* __restrict__ fa, StageTwo s2, long long y_fs,
                       long long fa_fs) {
  __shared__ float Bs[S2_KB][MAXC][L2_W + 1];
  __shared__ float Bt[S2_KB][MAXC][L2_W + 1];
  __shared__ float Y[L2_W][L2_W + 1];
  __shared__ float U[S2_KB][MAXC][L2_W + 1];
  __shared__ S2Cell cell[S2_KB];
  const int mu = blockIdx.x;
  const int frame = blockIdx.y;
  const int nmu = s2.mla_ns * s2.mla_nt;
  const int2 cc = s2.cols[mu], rr = s2.rows[mu];
  const int nc = cc.y - cc.x, nr = rr.y - rr.x;
  if (nc <= 0 || nr <= 0) return;   // uniform
  const int4 du = s2.det_union[mu];
  const int nsu = du.y - du.x + 1, ntu = du.w - du.z + 1;
  const long long Na = (long long)s2.arr_ns * s2.arr_nt;
  const float* yf = y + (long long)frame * y_fs;
  // This thread's block pixel and what is written there, the same for every
  // cell: M g on the lenslet's own pixels (wpx = index, mv = M), zero on
  // unowned pixels of blocks that tile the plane (wpx = -(index + 2)),
  // nothing elsewhere (wpx = -1).
  int wpx = -1, pr = 0, pc = 0;
  float mv = 0.0f;
  if ((int)threadIdx.x < nr * nc) {
    pr = div_of(small_div(nc), threadIdx.x);
    pc = threadIdx.x - pr * nc;
    const int px = (rr.x + pr) * s2.arr_ns + cc.x + pc;
    const int own = __ldg(s2.owner + px);
    if (own == mu) {
      wpx = px;
      mv = __ldg(s2.mask + px);
    } else if (!s2.overlap && own < 0) {
      wpx = -(px + 2);
    }
  }
  if (nsu > 0 && ntu > 0) {   // the union window of y, shared by every cell
    const SmallDiv du_div = small_div(nsu);
    for (int e = threadIdx.x; e < ntu * nsu; e += S2_THREADS) {
      const int bu = div_of(du_div, e), qu = e - bu * nsu;
      Y[bu][qu] = __ldg(yf + (long long)(du.z + bu) * s2.det_ns + du.x + qu);
    }
  }
  float* faf = fa + (long long)frame * fa_fs;
  for (int k0 = 0; k0 < s2.K; k0 += S2_KB) {
    s2_cell_table(s2, mu, nmu, k0, du, nr, cell);
    __syncthreads();
    {
      const int kk = threadIdx.x >> 6, task = threadIdx.x & 63;
      if (cell[kk].on && task < cell[kk].nds + cell[kk].ndt)
        lenslet_weight_task(s2.lens + (long long)(k0 + kk) * nmu + mu, cell[kk].dr, cc, rr, task, Bs[kk], Bt[kk]);
    }
    __syncthreads();
    // U[kk][r][q] = sum_b Bt[kk][r][b] y[dr.z + b][dr.x + q]
    const int tot = cell[0].cnt + cell[1].cnt + cell[2].cnt + cell[3].cnt;
    for (int e = threadIdx.x; e < tot; e += S2_THREADS) {
      int o = e;
      const int kk = s2_task_cell(cell, o);
      const int r = div_of(cell[kk].dd, o), q = o - r * cell[kk].nds;
      const int dz = cell[kk].dz, qx = cell[kk].dx + q;
      float u = 0.0f;
      for (int b = 0; b < cell[kk].ndt; ++b) u = fmaf(Bt[kk][r][b], Y[dz + b][qx], u);
      U[kk][r][q] = u;
    }
    __syncthreads();
    // M (its diagonal) on this lenslet's own pixels; blocks that tile the
    // plane also clear their unowned pixels, overlapping blocks leave them.
    // A cell outside the subset leaves its plane unwritten.
    if (wpx != -1) {
#pragma unroll
      for (int kk = 0; kk < S2_KB; ++kk) {
        if (!cell[kk].sub) continue;
        float* fk = faf + (long long)(k0 + kk) * Na;
        if (wpx >= 0 && cell[kk].on) {
          float g = 0.0f;
          for (int q = 0; q < cell[kk].nds; ++q) g = fmaf(Bs[kk][pc][q], U[kk][pr][q], g);
          fk[wpx] = mv * (cell[kk].scale * g);
        } else {
          fk[wpx >= 0 ? wpx : -(wpx + 2)] = 0.0f;
        }
      }
    }
    if (k0 + S2_KB < s2.K) __syncthreads();
  }
}

}  // namespace

int window_class(int w) { return w <= 2 ? 2 : w <= 3 ? 3 : w <= 4 ? 4 : 8; }

struct FwConfig {
  const void* fn;
  int threads;
};

template <int W, int SB, int G>
static FwConfig fw_kernel() {
  return {(const void*)beam_forward_batched<W, SB, G>, G * FT_GTHREADS};
}

// Variants (slices per batch SB, warp groups G): {4,2} {4,1} {2,2} {2,4} {8,1};
// wider windows use smaller batches so that shared memory stays within 48 KB
// (the kernel and its thread count come from the same instantiation).
template <int W>
static FwConfig fw_select(int variant) {
  if constexpr (W >= 8) {
    return variant == 1 ? fw_kernel<W, 2, 1>() : fw_kernel<W, 2, 2>();
  } else {
    switch (variant) {
      case 1: return fw_kernel<W, 4, 1>();
      case 2: return fw_kernel<W, 2, 2>();
      case 3:
        if constexpr (W >= 4) return fw_kernel<W, 2, 2>();
        else return fw_kernel<W, 2, 4>();
      case 4: return fw_kernel<W, 8, 1>();
      default: return fw_kernel<W, 4, 2>();
    }
  }
}

static FwConfig fw_select_class(int wclass, int variant) {
  switch (wclass) {
    case 2: return fw_select<2>(variant);
    case 3: return fw_select<3>(variant);
    case 4: return fw_select<4>(variant);
    default: return fw_select<8>(variant);
  }
}

int beam_forward_occupancy(int wclass, int variant) {
  int nb = 0;
  const FwConfig cfg = fw_select_class(wclass, variant);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cfg.fn, cfg.threads, 0) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

cudaError_t launch_beam_forward_batched(const BeamBatch& b, const int4* items, int n_items, int* counter,
                                        int wclass, int variant, int ctas, cudaStream_t st) {
  if (wclass > WMAX) return cudaErrorInvalidValue;
  if (n_items <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const long long total = (long long)n_items * b.frames;
  const int grid = (int)std::min<long long>(ctas, total);
  void* args[] = {(void*)&b, (void*)&items, (void*)&n_items, (void*)&counter};
  const FwConfig cfg = fw_select_class(wclass, variant);
  return cudaLaunchKernel(cfg.fn, dim3(grid), dim3(cfg.threads), args, 0, st);
}

cudaError_t launch_beam_adjoint_batched(const BeamBatch& b, float* x, long long x_fs, int accumulate,
                                        cudaStream_t st) {
  for (int c = 0; c < b.n_cams; ++c)
    if (b.cam[c].wis > WIMAX || b.cam[c].wit > WIMAX) return cudaErrorInvalidValue;
  const int nx = b.cam[0].nx, ny = b.cam[0].ny, nz = b.cam[0].nz;
  const int tiles_x = (nx + AT_S - 1) / AT_S;
  const int tiles_y = (ny + AT_T - 1) / AT_T;
  dim3 grid(tiles_x * tiles_y, (nz + AT_SN - 1) / AT_SN, b.frames);
  beam_adjoint_batched<<<grid, AT_THREADS, 0, st>>>(b, x, x_fs, accumulate, tiles_x);
  return cudaGetLastError();
}

cudaError_t launch_stage2_forward(const float* fa, float* y, StageTwo s2, int frames,
                                  long long fa_frame_stride, long long y_frame_stride,
                                  float* zbuf, cudaStream_t st) {
  if (s2.max_cols > MAXC || s2.max_rows > MAXC) return cudaErrorInvalidValue;
  dim3 g1(s2.mla_ns * s2.mla_nt, frames);
  stage2_lenslet_forward<<<g1, L2_THREADS, 0, st>>>(fa, s2, fa_frame_stride, zbuf);
  dim3 g2((s2.det_ns + 31) / 32, (s2.det_nt + 7) / 8, frames);
  stage2_gather<<<g2, 256, 0, st>>>(zbuf, y, s2, y_frame_stride);
  return cudaGetLastError();
}

cudaError_t launch_stage2_adjoint(const float* y, float* fa, StageTwo s2, int frames,
                                  long long y_frame_stride, long long fa_frame_stride,
                                  cudaStream_t st) {
  if (s2.max_cols > MAXC || s2.max_rows > MAXC) return cudaErrorInvalidValue;
  if (!s2.full_cover) {
    // array pixels outside every lenslet block are never written by a lenslet CTA
    for (int f = 0; f < frames; ++f)
      cudaMemsetAsync(fa + (long long)f * fa_frame_stride, 0,
                      (size_t)s2.K * s2.arr_ns * s2.arr_nt * sizeof(float), st);
  }
  dim3 g(s2.mla_ns * s2.mla_nt, frames);
  stage2_lenslet_adjoint<<<g, S2_THREADS, 0, st>>>(y, fa, s2, y_frame_stride, fa_frame_stride);
  return cudaGetLastError();
}

}  // namespace lt
