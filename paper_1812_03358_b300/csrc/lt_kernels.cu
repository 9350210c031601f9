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

#include "lt_async.cuh"
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
// (eq. xport,sep).  Both matrices depend on the geometry alone, so the plan
// evaluates them once (stage2_table_kernel: one footprint centre per detector
// column / row, consecutive array cells sharing their common edge) into a
// table, and describes every (lenslet, cell) by a 32-byte S2Desc.  A table
// entry is Bs[c][q] (nc rows of nds4 = nds rounded up to 4, zero past nds)
// then Bt[r][b] (nr rows of ndt), so that every contraction runs on float4
// rows: a lane computes four adjacent detector columns q at once.
//
// A (lenslet, cell) carries a few hundred multiply-adds on a few hundred
// loaded values, so the kernels are built to keep loads in flight: a
// persistent grid whose warps each walk their own lenslets (warp w of W takes
// lenslet-frames w, w + W, ...) cell after cell.  While a warp contracts one
// cell in two steps (the O(S+T) scheme of Sec. IV-B) in its own shared
// memory, cp.async already brings the next cell's table entry and pixels into
// the other half of a double buffer; the descriptors of the next 64 cells sit
// in a shared-memory ring.  No block barrier anywhere: each warp owns its
// lenslets' outputs.  Every output is accumulated in a fixed order (the
// plain double loop's, c then r, b then q, except the adjoint's last
// contraction, which sums even and odd detector columns apart and adds the
// two), so the result does not depend on the blocking or the schedule.
// ---------------------------------------------------------------------------
constexpr int L2_W = kStage2Window;
static_assert(2 * L2_W <= 64, "one footprint task per thread of the table kernel");

// Entries of one detector column or row of a (lenslet, cell): task < nds is
// column dr.x + task, Bs[c * lds + task] = entry (column, array column
// cc.x + c); otherwise row dr.z + task - nds into Bt[r * ldt + (task - nds)]
// likewise.  Consecutive array cells share their common edge value.
__device__ __forceinline__ void lenslet_weight_task(const LensletParam* L, int4 dr, int2 cc, int2 rr, int task,
                                                    float* Bs, int lds, float* Bt, int ldt) {
  const int nds = dr.y - dr.x + 1;
  const bool s_axis = task < nds;
  const AxisParam& a = s_axis ? L->s : L->t;
  const int q = s_axis ? task : task - nds;
  const int i = s_axis ? dr.x + q : dr.z + q;
  const int j0 = s_axis ? cc.x : rr.x;
  const int n = s_axis ? cc.y - cc.x : rr.y - rr.x;
  float* out = s_axis ? Bs + q : Bt + q;
  const int ld = s_axis ? lds : ldt;
  int jc;
  float fr;
  footprint_centre(a, i, jc, fr);
  float Flo = edge_F(j0 - jc, fr, a);
  for (int c = 0; c < n; ++c) {
    const float Fhi = edge_F(j0 + c + 1 - jc, fr, a);
    out[c * ld] = __fsub_rn(Fhi, Flo);
    Flo = Fhi;
  }
}

__device__ __forceinline__ int d_nc(uint32_t v) { return v & 0xff; }
__device__ __forceinline__ int d_nr(uint32_t v) { return (v >> 8) & 0xff; }
__device__ __forceinline__ int d_nds(uint32_t v) { return (v >> 16) & 0xff; }
__device__ __forceinline__ int d_ndt(uint32_t v) { return v >> 24; }
__device__ __forceinline__ int w_nsu(uint32_t v) { return v & 0xff; }
__device__ __forceinline__ int w_ntu(uint32_t v) { return (v >> 8) & 0xff; }
__device__ __forceinline__ bool w_last(uint32_t v) { return (v >> 16) & 1u; }
__device__ __forceinline__ int up4(int v) { return (v + 3) & ~3; }

// Plan time: the (lenslet, cell) table entries.  Grid (lenslets, cells).
__global__ void __launch_bounds__(64) stage2_table_kernel(StageTwo s2, float* __restrict__ wtab) {
  const int mu = blockIdx.x, k = blockIdx.y;
  const int nmu = s2.mla_ns * s2.mla_nt;
  const S2Desc dsc = s2.desc[(long long)mu * s2.K + k];
  if (dsc.off < 0) return;
  const int4 dr = s2.det_range[(long long)k * nmu + mu];
  const int2 cc = s2.cols[mu], rr = s2.rows[mu];
  const int nds = dr.y - dr.x + 1, ndt = dr.w - dr.z + 1, nds4 = up4(nds), nc = cc.y - cc.x;
  float* bs = wtab + dsc.off;
  float* bt = bs + nc * nds4;
  for (int task = threadIdx.x; task < nds + ndt; task += blockDim.x)
    lenslet_weight_task(s2.lens + (long long)k * nmu + mu, dr, cc, rr, task, bs, nds4, bt, ndt);
  for (int e = threadIdx.x; e < nc * (nds4 - nds); e += blockDim.x) {   // zero padding of the Bs rows
    const int cix = e / (nds4 - nds);
    bs[cix * nds4 + nds + (e - cix * (nds4 - nds))] = 0.0f;
  }
}

__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// floor(o / d) for 0 <= o < 2^12, 1 <= d <= 64 from the reciprocal RN(1/d):
// (o + 1/2) / d lies at least 1 / (2d) >= 1/128 from an integer, and the
// product of o + 1/2 with the rounded reciprocal is off by at most
// 2^12 * 2^-23 < 1/2000, so truncation gives the exact quotient.  The
// reciprocals are constants rounded by the compiler.
#define LT_RCP8(b) 1.0f / (b + 0), 1.0f / (b + 1), 1.0f / (b + 2), 1.0f / (b + 3), 1.0f / (b + 4), 1.0f / (b + 5), \
                   1.0f / (b + 6), 1.0f / (b + 7)
__constant__ float kRcp[72] = {0.0f, 1.0f, 0.5f, 1.0f / 3, 0.25f, 0.2f, 1.0f / 6, 1.0f / 7,
                               LT_RCP8(8), LT_RCP8(16), LT_RCP8(24), LT_RCP8(32), LT_RCP8(40),
                               LT_RCP8(48), LT_RCP8(56), LT_RCP8(64)};
#undef LT_RCP8
__device__ __forceinline__ int div_small(int o, int d) { return __float2int_rz(((float)o + 0.5f) * kRcp[d]); }

// The warp's cells: item j is cell j % K of lenslet-frame unit
// w0 + (j / K) * nw (unit = frame * N_mu + mu, fewer than 2^31).  The walk
// keeps (unit, cell) of the next item to issue and of the item being
// contracted as counters; descriptors come kS2Chunk at a time into a ring of
// kS2Ring in shared memory (slot j % kS2Ring), one per lane of the first
// kS2Chunk: while chunk c is contracted, chunk c + 1 is already in place.
struct S2Walk {
  int w0, nw, n_items, K, nmu;
  __device__ __forceinline__ void load_chunk(const S2Desc* desc, S2Desc* ring, int chunk, int lane) const {
    const int j = chunk * kS2Chunk + lane;
    if (lane < kS2Chunk && j < n_items) {
      const int u = w0 + (j / K) * nw;
      ring[j & (kS2Ring - 1)] = desc[(long long)(u % nmu) * K + j % K];
    }
  }
};
struct S2Pos {
  int unit, k, frame;
  __device__ __forceinline__ void next(const S2Walk& w) {
    if (++k == w.K) {
      k = 0;
      unit += w.nw;
      frame = unit / w.nmu;
    }
  }
};

// Block copies into shared memory: nr rows of n floats starting at src (row
// stride `stride` floats) into dst rows of stride `dstride`.  Aligned mode
// (src - shift 16-byte aligned, stride a multiple of 4, shift = the row start
// mod 4): whole 16-byte chunks covering each row, element c landing at
// dst[r * dstride + shift + c]; otherwise one float per copy at
// dst[r * dstride + c] (shift 0).
__device__ __forceinline__ void s2_copy_rows(float* dst, int dstride, const float* src, int nr, int n,
                                             long long stride, int shift, bool aligned, int lane) {
  if (aligned) {
    const float* s0 = src - shift;
    const int nch = (shift + n + 3) >> 2;
    for (int o = lane; o < nr * nch; o += 32) {
      const int r = div_small(o, nch), ch = o - r * nch;
      cp_async16(smem_addr(dst + r * dstride + 4 * ch), s0 + r * stride + 4 * ch, true);
    }
  } else {
    for (int o = lane; o < nr * n; o += 32) {
      const int r = div_small(o, n), cix = o - r * n;
      cp_async4(smem_addr(dst + r * dstride + cix), src + r * stride + cix);
    }
  }
}

// acc += a * b elementwise as two packed f32x2 FMAs (each lane of a packed
// FMA is the round-to-nearest fmaf of that element).
__device__ __forceinline__ void fma4(float4& acc, float a, const float4& b) {
  const float2 a2 = make_float2(a, a);
  const float2 lo = __ffma2_rn(a2, make_float2(b.x, b.y), make_float2(acc.x, acc.y));
  const float2 hi = __ffma2_rn(a2, make_float2(b.z, b.w), make_float2(acc.z, acc.w));
  acc = make_float4(lo.x, lo.y, hi.x, hi.y);
}

// Forward, pass 1: each lenslet's contribution sum_k scale_k Bt (x) Bs fa_k
// on the union over cells of its detector windows (cells in order), written
// to zbuf (no overlap between lenslets).
__global__ void __launch_bounds__(kStage2Threads)
stage2_lenslet_forward(const float* __restrict__ fa, StageTwo s2, long long fa_fs, int frames, int aligned,
                       float* __restrict__ zbuf) {
  extern __shared__ __align__(16) float s2_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int TB = s2.tab_max, FB = s2.pix_max;
  float* base = s2_smem + (long long)warp * s2.fwd_warp_floats;
  S2Desc* ring = reinterpret_cast<S2Desc*>(base);     // [kS2Ring]
  float* tab = base + kS2Ring * 8;                     // [2][TB]
  float* fv = tab + 2 * TB;                            // [2][FB]: block rows of row_max
  uint32_t* own = reinterpret_cast<uint32_t*>(fv + 2 * FB);   // [2][8]: row intervals (or ownership bits)
  float* wb = reinterpret_cast<float*>(own + 16);      // [w_max]: W[r][q], rows of nds4
  float* zb = wb + s2.w_max;                           // [z_max]
  S2Walk wk;
  wk.K = s2.K;
  wk.nmu = s2.mla_ns * s2.mla_nt;
  const int units = frames * wk.nmu;
  wk.nw = gridDim.x * (kStage2Threads / 32);
  wk.w0 = blockIdx.x * (kStage2Threads / 32) + warp;
  if (wk.w0 >= units) return;
  wk.n_items = ((units - 1 - wk.w0) / wk.nw + 1) * wk.K;
  const long long Na = (long long)s2.arr_ns * s2.arr_nt;
  for (int o = lane; o < s2.z_max; o += 32) zb[o] = 0.0f;
  wk.load_chunk(s2.desc, ring, 0, lane);
  wk.load_chunk(s2.desc, ring, 1, lane);
  __syncwarp();
  S2Pos cur{wk.w0, 0, wk.w0 / wk.nmu}, nxt = cur;

  auto issue = [&](const S2Pos& p, const S2Desc& d, int buf) {
    if (d.off >= 0 && cell_on(s2.sub_n, s2.sub_s, p.k)) {
      const uint32_t dm = d.dims;
      const int n4 = (d_nc(dm) * up4(d_nds(dm)) + d_nr(dm) * d_ndt(dm) + 3) >> 2;
      const float* t = s2.wtab + d.off;
      for (int e = lane; e < n4; e += 32) cp_async16(smem_addr(tab + buf * TB + 4 * e), t + 4 * e, true);
      s2_copy_rows(fv + buf * FB, s2.row_max, fa + p.frame * fa_fs + p.k * Na + d.px0, d_nr(dm), d_nc(dm), s2.arr_ns,
                   aligned ? (d.px0 & 3) : 0, aligned, lane);
      if (lane < 2) {
        const uint32_t* src = s2.iv_ok ? s2.ivals + (long long)d.mu * 8 : s2.bits + (long long)d.mu * 16;
        cp_async16(smem_addr(own + buf * 8 + 4 * lane), src + 4 * lane, true);
      }
    }
    cp_async_commit();
  };

  issue(nxt, ring[0], 0);
  nxt.next(wk);
  for (int j = 0; j < wk.n_items; ++j) {
    if (j % kS2Chunk == 0 && j > 0) {   // chunk c = j / kS2Chunk starts: bring in chunk c + 1
      wk.load_chunk(s2.desc, ring, j / kS2Chunk + 1, lane);
      __syncwarp();
    }
    const S2Desc d = ring[j & (kS2Ring - 1)];
    if (j + 1 < wk.n_items) {
      issue(nxt, ring[(j + 1) & (kS2Ring - 1)], (j + 1) & 1);
      nxt.next(wk);
    } else {
      cp_async_commit();
    }
    cp_async_wait_one();
    __syncwarp();
    const int buf = j & 1;
    const uint32_t dm = d.dims, wn = d.win;
    if (d.off >= 0 && cell_on(s2.sub_n, s2.sub_s, cur.k)) {
      const int nc = d_nc(dm), nr = d_nr(dm), nds = d_nds(dm), ndt = d_ndt(dm), nsu = w_nsu(wn);
      const int nds4 = up4(nds), nq4 = nds4 >> 2;
      const float* F = fv + buf * FB + (aligned ? (d.px0 & 3) : 0);
      const uint32_t* OW = own + buf * 8;
      const float* bs = tab + buf * TB;
      const float* bt = bs + nc * nds4;
      // W[r][q..q+3] = sum_c F[r][c] Bs[c][q..q+3] over the lenslet's own
      // pixels of row r: the interval [c0, c1) of the row (or, when some row's
      // are not one interval, every c with its ownership bit)
      for (int o = lane; o < nr * nq4; o += 32) {
        const int r = div_small(o, nq4), q = (o - r * nq4) << 2;
        const float* fr = F + r * s2.row_max;
        float4 w = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (s2.iv_ok) {
          const uint32_t iv = reinterpret_cast<const uint16_t*>(OW)[r];
          for (int cix = iv & 0xff; cix < (int)(iv >> 8); ++cix)
            fma4(w, fr[cix], *reinterpret_cast<const float4*>(bs + cix * nds4 + q));
        } else {
          for (int cix = 0; cix < nc; ++cix) {
            const uint32_t bit = r * nc + cix;
            const float f = (OW[bit >> 5] >> (bit & 31)) & 1u ? fr[cix] : 0.0f;
            fma4(w, f, *reinterpret_cast<const float4*>(bs + cix * nds4 + q));
          }
        }
        *reinterpret_cast<float4*>(wb + r * nds4 + q) = w;
      }
      __syncwarp();
      // Z[b][q..q+3] += scale sum_r Bt[r][b] W[r][q..q+3] (columns q < nds)
      for (int o = lane; o < ndt * nq4; o += 32) {
        const int bb = div_small(o, nq4), q = (o - bb * nq4) << 2;
        float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int r = 0; r < nr; ++r) fma4(z, bt[r * ndt + bb], *reinterpret_cast<const float4*>(wb + r * nds4 + q));
        float* zr = zb + d.zo + bb * nsu + q;
        zr[0] = fmaf(d.scale, z.x, zr[0]);
        if (q + 1 < nds) zr[1] = fmaf(d.scale, z.y, zr[1]);
        if (q + 2 < nds) zr[2] = fmaf(d.scale, z.z, zr[2]);
        if (q + 3 < nds) zr[3] = fmaf(d.scale, z.w, zr[3]);
      }
    }
    if (w_last(wn)) {
      __syncwarp();
      const int n = w_nsu(wn) * w_ntu(wn);
      float* zout = zbuf + (long long)cur.unit * (L2_W * L2_W);
      for (int o = lane; o < n; o += 32) {
        zout[o] = zb[o];
        zb[o] = 0.0f;
      }
    }
    cur.next(wk);
    __syncwarp();
  }
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
// for the lenslet's own block (a gather: every array pixel has one lenslet),
// one cell after another per warp as in the forward: U = Bt^T Y on the
// cell's window, then every block pixel of the cell, written to that cell's
// plane (one writer per output).  Blocks that tile the plane also clear
// their unowned pixels; a cell outside the subset leaves its plane unwritten.
__global__ void __launch_bounds__(kStage2Threads)
stage2_lenslet_adjoint(const float* __restrict__ y, float* __restrict__ fa, StageTwo s2, long long y_fs,
                       long long fa_fs, int frames) {
  extern __shared__ __align__(16) float s2_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int TB = s2.tab_max, YB = s2.y_max;
  float* base = s2_smem + (long long)warp * s2.adj_warp_floats;
  S2Desc* ring = reinterpret_cast<S2Desc*>(base);     // [kS2Ring]
  float* tab = base + kS2Ring * 8;                     // [2][TB]
  float* yw = tab + 2 * TB;                            // [2][YB]: the cell's window of y, rows of nds4 (zero past nds)
  uint32_t* bits = reinterpret_cast<uint32_t*>(yw + 2 * YB);  // [2][16]: row intervals, or own (0..7), clear (8..15)
  float* ub = reinterpret_cast<float*>(bits + 32);     // [w_max]: U[r][q], rows of nds4
  S2Walk wk;
  wk.K = s2.K;
  wk.nmu = s2.mla_ns * s2.mla_nt;
  const int units = frames * wk.nmu;
  wk.nw = gridDim.x * (kStage2Threads / 32);
  wk.w0 = blockIdx.x * (kStage2Threads / 32) + warp;
  if (wk.w0 >= units) return;
  wk.n_items = ((units - 1 - wk.w0) / wk.nw + 1) * wk.K;
  const long long Na = (long long)s2.arr_ns * s2.arr_nt;
  wk.load_chunk(s2.desc, ring, 0, lane);
  wk.load_chunk(s2.desc, ring, 1, lane);
  __syncwarp();
  S2Pos cur{wk.w0, 0, wk.w0 / wk.nmu}, nxt = cur;

  auto issue = [&](const S2Pos& p, const S2Desc& d, int buf) {
    if (cell_on(s2.sub_n, s2.sub_s, p.k)) {
      const uint32_t dm = d.dims;
      if (d.off >= 0) {
        const int nds = d_nds(dm), ndt = d_ndt(dm), nds4 = up4(nds);
        const int n4 = (d_nc(dm) * nds4 + d_nr(dm) * ndt + 3) >> 2;
        const float* t = s2.wtab + d.off;
        for (int e = lane; e < n4; e += 32) cp_async16(smem_addr(tab + buf * TB + 4 * e), t + 4 * e, true);
        const float* ys = y + p.frame * y_fs + d.y0;
        float* yb = yw + buf * YB;
        // the window one float per copy, so that its rows start 16-byte aligned
        s2_copy_rows(yb, nds4, ys, ndt, nds, s2.det_ns, 0, false, lane);
        if (nds4 > nds)   // the padding columns are zero (plain stores; the copies never touch them)
          for (int o = lane; o < ndt * (nds4 - nds); o += 32) {
            const int bb = div_small(o, nds4 - nds);
            yb[bb * nds4 + nds + (o - bb * (nds4 - nds))] = 0.0f;
          }
      }
      if (s2.iv_ok) {
        if (lane < 2) cp_async16(smem_addr(bits + buf * 16 + 4 * lane), s2.ivals + (long long)d.mu * 8 + 4 * lane, true);
      } else if (lane < 4) {
        cp_async16(smem_addr(bits + buf * 16 + 4 * lane), s2.bits + (long long)d.mu * 16 + 4 * lane, true);
      }
    }
    cp_async_commit();
  };

  issue(nxt, ring[0], 0);
  nxt.next(wk);
  for (int j = 0; j < wk.n_items; ++j) {
    if (j % kS2Chunk == 0 && j > 0) {   // chunk c = j / kS2Chunk starts: bring in chunk c + 1
      wk.load_chunk(s2.desc, ring, j / kS2Chunk + 1, lane);
      __syncwarp();
    }
    const S2Desc d = ring[j & (kS2Ring - 1)];
    if (j + 1 < wk.n_items) {
      issue(nxt, ring[(j + 1) & (kS2Ring - 1)], (j + 1) & 1);
      nxt.next(wk);
    } else {
      cp_async_commit();
    }
    cp_async_wait_one();
    __syncwarp();
    const int buf = j & 1;
    if (cell_on(s2.sub_n, s2.sub_s, cur.k)) {
      const uint32_t dm = d.dims;
      const int nc = d_nc(dm), nr = d_nr(dm), nds = d_nds(dm), ndt = d_ndt(dm);
      const uint32_t* B = bits + buf * 16;
      const uint16_t* IV = reinterpret_cast<const uint16_t*>(B);
      // pixel (r, c) of the block: the lenslet's own (written with its value),
      // or nobody's in blocks that tile the plane (written zero)?
      auto mine_of = [&](int r, int cix, int o) -> bool {
        if (s2.iv_ok) {
          const uint32_t iv = IV[r];
          return cix >= (int)(iv & 0xff) && cix < (int)(iv >> 8);
        }
        return (B[o >> 5] >> (o & 31)) & 1u;
      };
      auto clear_of = [&](int o) -> bool {
        if (s2.iv_ok) return !s2.overlap;
        return (B[8 + (o >> 5)] >> (o & 31)) & 1u;
      };
      float* fk = fa + cur.frame * fa_fs + cur.k * Na + d.px0;
      if (d.off < 0) {   // empty window: zeros
        for (int o = lane; o < nr * nc; o += 32) {
          const int r = div_small(o, nc), cix = o - r * nc;
          if (mine_of(r, cix, o) || clear_of(o)) fk[(long long)r * s2.arr_ns + cix] = 0.0f;
        }
      } else {
        const int nds4 = up4(nds), nq4 = nds4 >> 2;
        const float* bs = tab + buf * TB;
        const float* bt = bs + nc * nds4;
        const float* Y = yw + buf * YB;
        // U[r][q..q+3] = sum_b Bt[r][b] Y[b][q..q+3]
        for (int o = lane; o < nr * nq4; o += 32) {
          const int r = div_small(o, nq4), q = (o - r * nq4) << 2;
          float4 u = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          for (int bb = 0; bb < ndt; ++bb) fma4(u, bt[r * ndt + bb], *reinterpret_cast<const float4*>(Y + bb * nds4 + q));
          *reinterpret_cast<float4*>(ub + r * nds4 + q) = u;
        }
        __syncwarp();
        const float* M = s2.mask + d.px0;   // read once per pixel, from L2: no shared copy
        for (int o = lane; o < nr * nc; o += 32) {
          const int r = div_small(o, nc), cix = o - r * nc;
          const bool mine = mine_of(r, cix, o);
          if (!mine && !clear_of(o)) continue;
          float v = 0.0f;
          if (mine) {
            const float m = __ldg(M + (long long)r * s2.arr_ns + cix);   // in flight during the dot product
            const float* br = bs + cix * nds4;
            const float* ur = ub + r * nds4;
            // two partial sums (even and odd detector columns), one packed
            // FMA per pair of columns, added at the end
            float2 g2 = make_float2(0.0f, 0.0f);
            for (int q = 0; q < nds4; q += 4) {
              const float4 a = *reinterpret_cast<const float4*>(br + q);
              const float4 b = *reinterpret_cast<const float4*>(ur + q);
              g2 = __ffma2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y), g2);
              g2 = __ffma2_rn(make_float2(a.z, a.w), make_float2(b.z, b.w), g2);
            }
            v = m * (d.scale * (g2.x + g2.y));
          }
          fk[(long long)r * s2.arr_ns + cix] = v;
        }
      }
    }
    cur.next(wk);
    __syncwarp();
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

size_t stage2_smem_bytes(const StageTwo& s2, bool adjoint) {
  return (size_t)(kStage2Threads / 32) * (adjoint ? s2.adj_warp_floats : s2.fwd_warp_floats) * sizeof(float);
}

cudaError_t stage2_occupancy(const StageTwo& s2, bool adjoint, int* ctas_per_sm) {
  const void* fn = adjoint ? (const void*)stage2_lenslet_adjoint : (const void*)stage2_lenslet_forward;
  const size_t smem = stage2_smem_bytes(s2, adjoint);
  // the limit is per kernel and other plans may need more: raise it to the
  // device's opt-in maximum, never lower it
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess && smem > (size_t)optin) {
    *ctas_per_sm = 0;
    return cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, fn, kStage2Threads, smem);
  return e;
}

// Persistent grid: every resident CTA, or fewer when there are fewer
// lenslet-frames than warps.
static unsigned stage2_ctas(const StageTwo& s2, int per_sm, int frames) {
  const long long units = (long long)frames * s2.mla_ns * s2.mla_nt;
  const long long need = (units + kStage2Threads / 32 - 1) / (kStage2Threads / 32);
  return (unsigned)std::max<long long>(1, std::min<long long>(need, (long long)s2.sms * std::max(1, per_sm)));
}

cudaError_t launch_stage2_forward(const float* fa, float* y, StageTwo s2, int frames,
                                  long long fa_frame_stride, long long y_frame_stride,
                                  float* zbuf, cudaStream_t st) {
  if (s2.max_cols > MAXC || s2.max_rows > MAXC || !s2.desc || !s2.wtab || !s2.bits) return cudaErrorInvalidValue;
  if (frames <= 0) return cudaSuccess;
  if ((long long)frames * s2.mla_ns * s2.mla_nt >= (1LL << 31)) return cudaErrorInvalidValue;
  // 16-byte block copies when the rows start 4-aligned up to one shift per block
  const int aligned = (reinterpret_cast<uintptr_t>(fa) & 15) == 0 && s2.arr_ns % 4 == 0 && fa_frame_stride % 4 == 0;
  stage2_lenslet_forward<<<stage2_ctas(s2, s2.fwd_per_sm, frames), kStage2Threads, stage2_smem_bytes(s2, false), st>>>(
      fa, s2, fa_frame_stride, frames, aligned, zbuf);
  dim3 g2((s2.det_ns + 31) / 32, (s2.det_nt + 7) / 8, frames);
  stage2_gather<<<g2, 256, 0, st>>>(zbuf, y, s2, y_frame_stride);
  return cudaGetLastError();
}

cudaError_t launch_stage2_adjoint(const float* y, float* fa, StageTwo s2, int frames,
                                  long long y_frame_stride, long long fa_frame_stride,
                                  cudaStream_t st) {
  if (s2.max_cols > MAXC || s2.max_rows > MAXC || !s2.desc || !s2.wtab || !s2.bits) return cudaErrorInvalidValue;
  if (frames <= 0) return cudaSuccess;
  if ((long long)frames * s2.mla_ns * s2.mla_nt >= (1LL << 31)) return cudaErrorInvalidValue;
  if (!s2.full_cover) {
    // array pixels outside every lenslet block are never written by a lenslet warp
    for (int f = 0; f < frames; ++f)
      cudaMemsetAsync(fa + (long long)f * fa_frame_stride, 0,
                      (size_t)s2.K * s2.arr_ns * s2.arr_nt * sizeof(float), st);
  }
  stage2_lenslet_adjoint<<<stage2_ctas(s2, s2.adj_per_sm, frames), kStage2Threads, stage2_smem_bytes(s2, true), st>>>(
      y, fa, s2, y_frame_stride, fa_frame_stride, frames);
  return cudaGetLastError();
}

cudaError_t launch_stage2_tables(StageTwo s2, float* wtab, cudaStream_t st) {
  if (s2.max_cols > MAXC || s2.max_rows > MAXC || !s2.desc) return cudaErrorInvalidValue;
  dim3 g(s2.mla_ns * s2.mla_nt, s2.K);
  stage2_table_kernel<<<g, 64, 0, st>>>(s2, wtab);
  return cudaGetLastError();
}

}  // namespace lt
