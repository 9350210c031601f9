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
#include "lt_internal.h"

namespace lt {

namespace {

constexpr int WMAX = 8;      // forward window cap: source cells per target pixel per axis
constexpr int WIMAX = 16;    // adjoint window cap: target pixels per source cell per axis
constexpr int MAXC = 16;     // array pixels per lenslet per axis (stage two)

// ---------------------------------------------------------------------------
// Matrix entries.  All arithmetic uses explicit round-to-nearest intrinsics so
// that no floating-point contraction can differ between the forward and the
// adjoint instantiations.
// ---------------------------------------------------------------------------

// Footprint centre xi(i) = c0 + c1*i of target pixel i in source-index units,
// returned as an integer cell jc and a fraction fr in [0, 1).  The product and
// sum are compensated (exact product error by fma, TwoSum) so that the
// fraction is accurate to ~1e-7 even where xi is in the hundreds.
__device__ __forceinline__ void footprint_centre(const AxisParam& a, int i, int& jc, float& fr) {
  const float fi = (float)i;
  const float p = __fmul_rn(a.c1_hi, fi);
  const float e = __fmaf_rn(a.c1_hi, fi, -p);
  const float s = __fadd_rn(a.c0_hi, p);
  const float bb = __fsub_rn(s, a.c0_hi);
  const float err = __fadd_rn(__fsub_rn(a.c0_hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  const float lo = __fadd_rn(__fadd_rn(err, e), __fmaf_rn(a.c1_lo, fi, a.c0_lo));
  float fl = floorf(s);
  float f = __fadd_rn(__fsub_rn(s, fl), lo);
  if (f >= 1.0f) {
    fl = __fadd_rn(fl, 1.0f);
    f = __fsub_rn(f, 1.0f);
  } else if (f < 0.0f) {
    fl = __fsub_rn(fl, 1.0f);
    f = __fadd_rn(f, 1.0f);
  }
  jc = (int)fl;
  fr = f;
}

// Antiderivative of the unit-height symmetric trapezoid with plateau
// half-width P and outer half-width Q (odd in x):
//   G(a) = a - max(a - P, 0)^2 / (2 (Q - P))  for a = min(|x|, Q),
// which is a on the plateau, the integrated ramp between P and Q and the
// constant (P + Q)/2 beyond Q (hir = 1/(2(Q-P)), 0 for a box).
__device__ __forceinline__ float trap_F(float x, float P, float Q, float hir) {
  const float a = fminf(fabsf(x), Q);
  const float d = fmaxf(__fsub_rn(a, P), 0.0f);
  const float g = __fsub_rn(a, __fmul_rn(__fmul_rn(d, d), hir));
  return copysignf(g, x);
}

// F at the lower edge of source cell m (relative to jc) for a footprint
// centred at fr: the edge m - 1/2 (equal to the upper edge of cell m - 1;
// both are exact in float for the small integers used here).
__device__ __forceinline__ float edge_F(int m, float fr, const AxisParam& a) {
  return trap_F(__fsub_rn(__fsub_rn((float)m, 0.5f), fr), a.P, a.Q, a.hir);
}

// Integral of the unit trapezoid centred at fr over source cell m (relative
// to jc): [m - 1/2, m + 1/2].  Exactly 0 outside the footprint.
// Equal, bit for bit, to edge_F(m + 1) - edge_F(m).
__device__ __forceinline__ float cell_weight(int m, float fr, const AxisParam& a) {
  const float fm = (float)m;
  const float xh = __fsub_rn(__fadd_rn(fm, 0.5f), fr);
  const float xl = __fsub_rn(__fsub_rn(fm, 0.5f), fr);
  return __fsub_rn(trap_F(xh, a.P, a.Q, a.hir), trap_F(xl, a.P, a.Q, a.hir));
}

// First target pixel whose footprint may overlap source cell j (a superset
// window of the exact range, widened by one pixel for rounding).
__device__ __forceinline__ int window_start(const AxisParam& a, int j) {
  const float c0 = __fadd_rn(a.c0_hi, a.c0_lo);
  const float lo = __fmul_rn(__fsub_rn(__fsub_rn((float)j - 0.5f, a.Q), c0), a.inv_c1);
  const float hi = __fmul_rn(__fsub_rn(__fadd_rn((float)j + 0.5f, a.Q), c0), a.inv_c1);
  return (int)floorf(fminf(lo, hi)) - 1;
}

// ---------------------------------------------------------------------------
// Beam integration, forward.  CTA = 32 x 32 target pixels of one frame (and
// one cell if per_cell); 4 warps, warp w owns rows w, w+4, ..., w+28 and lane
// l column l.  Only the slices in the tile's interval (host table: where the
// tile's footprints can meet the volume) are visited.  For a batch of SB
// slices all threads first evaluate the s-weights of the 32 columns and the
// t-weights of the 32 rows into shared memory (the separable O(S+T) weight
// work of Sec. IV-B, shared by the tile), then every thread accumulates its
// 8 pixels from the L1-resident slices.  WS/WT are compile-time windows; a
// weight beyond a slice's own window is exactly zero.
// ---------------------------------------------------------------------------
constexpr int FT_S = kBeamTileS;
constexpr int FT_T = kBeamTileT;
constexpr int FT_GROUPS = 2;                 // warp groups splitting the slice range
constexpr int FT_GTHREADS = 128;             // threads per group
constexpr int FT_THREADS = FT_GROUPS * FT_GTHREADS;
constexpr int FT_ROWS = FT_T / 4;
constexpr int FT_SB = 4;

__device__ __forceinline__ void group_barrier(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(FT_GTHREADS) : "memory");
}

template <int WS, int WT>
__global__ void __launch_bounds__(FT_THREADS)
beam_forward_kernel(const float* __restrict__ x, float* __restrict__ out,
                    const SliceParam* __restrict__ prm, int nx, int ny, int nz,
                    int ns, int nt, int K, int per_cell, const uint8_t* __restrict__ mask,
                    long long x_fs, long long out_fs, int tiles_s, int tiles_t,
                    const int2* __restrict__ srange, const int2* __restrict__ trange) {
  __shared__ float sw[FT_GROUPS][FT_SB][WS][FT_S];
  __shared__ int sx[FT_GROUPS][FT_SB][WS][FT_S];
  __shared__ float tw[FT_GROUPS][FT_SB][WT][FT_T];
  __shared__ int ty[FT_GROUPS][FT_SB][WT][FT_T];
  __shared__ float red[FT_T][FT_S + 1];

  const int grp = threadIdx.x / FT_GTHREADS;
  const int gt = threadIdx.x - grp * FT_GTHREADS;
  const int lane = gt & 31;
  const int warp = gt >> 5;
  const int tile_s = blockIdx.x % tiles_s;
  const int tile_t = blockIdx.x / tiles_s;
  const int is0 = tile_s * FT_S;
  const int it0 = tile_t * FT_T;
  const int frame = blockIdx.z;
  const int k_begin = per_cell ? (int)blockIdx.y : 0;
  const int k_end = per_cell ? (int)blockIdx.y + 1 : K;
  const float* xf = x + (long long)frame * x_fs;

  float acc[FT_ROWS];
#pragma unroll
  for (int r = 0; r < FT_ROWS; ++r) acc[r] = 0.0f;

  for (int k = k_begin; k < k_end; ++k) {
    const int2 rs = srange[k * tiles_s + tile_s];
    const int2 rt = trange[k * tiles_t + tile_t];
    const int n0 = max(rs.x, rt.x);
    const int n1 = min(rs.y, rt.y);
    const SliceParam* pk = prm + (long long)k * nz;
    // group g takes slice batches g, g + 2, g + 4, ... of the tile's interval
    for (int nb = n0 + grp * FT_SB; nb < n1; nb += FT_GROUPS * FT_SB) {
      // phase A: weights of SB slices x (32 columns + 32 rows)
      for (int task = gt; task < FT_SB * (FT_S + FT_T); task += FT_GTHREADS) {
        const int sl = task / (FT_S + FT_T);
        const int q = task - sl * (FT_S + FT_T);
        const int n = nb + sl;
        if (n >= n1) continue;
        const SliceParam* p = pk + n;
        if (q < FT_S) {
          int jc;
          float fr;
          footprint_centre(p->s, is0 + q, jc, fr);
          const int mlo = (int)floorf(fr - p->s.Q + 0.5f);
          float Flo = edge_F(mlo, fr, p->s);
#pragma unroll
          for (int a = 0; a < WS; ++a) {
            const int j = jc + mlo + a;
            const float Fhi = edge_F(mlo + a + 1, fr, p->s);
            float w = __fsub_rn(Fhi, Flo);
            Flo = Fhi;
            if (j < 0 || j >= nx) w = 0.0f;
            sw[grp][sl][a][q] = w;
            sx[grp][sl][a][q] = min(max(j, 0), nx - 1);
          }
        } else {
          const int r = q - FT_S;
          int jc;
          float fr;
          footprint_centre(p->t, it0 + r, jc, fr);
          const int mlo = (int)floorf(fr - p->t.Q + 0.5f);
          float Flo = edge_F(mlo, fr, p->t);
#pragma unroll
          for (int b = 0; b < WT; ++b) {
            const int j = jc + mlo + b;
            const float Fhi = edge_F(mlo + b + 1, fr, p->t);
            float w = __fsub_rn(Fhi, Flo);
            Flo = Fhi;
            if (j < 0 || j >= ny) w = 0.0f;
            tw[grp][sl][b][r] = w;
            ty[grp][sl][b][r] = min(max(j, 0), ny - 1) * nx;
          }
        }
      }
      group_barrier(1 + grp);
      // phase B: accumulate (loads are always in bounds; zero weights are cheap)
      const int nsl = min(FT_SB, n1 - nb);
      for (int sl = 0; sl < nsl; ++sl) {
        const int n = nb + sl;
        const float scale = pk[n].scale;
        const float* xs = xf + (long long)n * ny * nx;
        float wsr[WS];
        int sxr[WS];
#pragma unroll
        for (int a = 0; a < WS; ++a) {
          wsr[a] = sw[grp][sl][a][lane];
          sxr[a] = sx[grp][sl][a][lane];
        }
#pragma unroll
        for (int r = 0; r < FT_ROWS; ++r) {
          const int row = warp + 4 * r;
          float v = 0.0f;
#pragma unroll
          for (int b = 0; b < WT; ++b) {
            const float* xr = xs + ty[grp][sl][b][row];
            float u = 0.0f;
#pragma unroll
            for (int a = 0; a < WS; ++a) u = fmaf(wsr[a], __ldg(xr + sxr[a]), u);
            v = fmaf(tw[grp][sl][b][row], u, v);
          }
          acc[r] = fmaf(scale, v, acc[r]);
        }
      }
      group_barrier(1 + grp);
    }
  }

  // combine the two groups' partial sums
  if (grp == 1) {
#pragma unroll
    for (int r = 0; r < FT_ROWS; ++r) red[warp + 4 * r][lane] = acc[r];
  }
  __syncthreads();
  if (grp == 0) {
    const int is = is0 + lane;
    if (is < ns) {
      float* o = out + (long long)frame * out_fs + (per_cell ? (long long)blockIdx.y * ns * nt : 0);
#pragma unroll
      for (int r = 0; r < FT_ROWS; ++r) {
        const int row = warp + 4 * r;
        const int it = it0 + row;
        if (it < nt) {
          float v = acc[r] + red[row][lane];
          if (mask && !mask[(long long)it * ns + is]) v = 0.0f;
          o[(long long)it * ns + is] = v;
        }
      }
    }
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

// CTA = 32 x 8 voxels of one slice and frame (lane = voxel column, warp =
// voxel row).  Per cell: all threads evaluate the windows of target pixels
// whose footprints may cover each voxel column / row and the matching entries
// (the same cell_weight of the same (pixel, cell) pair as the forward); then
// warp r contracts along t for its voxel row with coalesced image-row reads,
// U[r][c] = sum_b Bt[r][b] g[row_b][c_lo + c], and each voxel contracts along
// s from shared memory (the separable O(S+T) scheme of Sec. IV-B).
__global__ void __launch_bounds__(AT_THREADS)
beam_adjoint_kernel(const float* __restrict__ in, float* __restrict__ x,
                    const SliceParam* __restrict__ prm, int nx, int ny, int nz,
                    int ns, int nt, int K, int per_cell, int accumulate,
                    long long in_fs, long long x_fs, int tiles_x) {
  __shared__ float sw[WIMAX][AT_S];
  __shared__ int si[WIMAX][AT_S];
  __shared__ float tw[WIMAX][AT_T];
  __shared__ int ti[WIMAX][AT_T];
  __shared__ float U[AT_T][AT_UCOLS];

  const int lane = threadIdx.x & 31;
  const int row = threadIdx.x >> 5;
  const int jx0 = (blockIdx.x % tiles_x) * AT_S;
  const int jy0 = (blockIdx.x / tiles_x) * AT_T;
  const int jx1 = min(jx0 + AT_S, nx) - 1;
  const int n = blockIdx.y;
  const int frame = blockIdx.z;
  const float* inf = in + (long long)frame * in_fs;

  float acc = 0.0f;
  for (int k = 0; k < K; ++k) {
    const SliceParam* p = prm + (long long)k * nz + n;
    const int wis = p->wis;
    const int wit = p->wit;
    const float* g = inf + (per_cell ? (long long)k * ns * nt : 0);
    // pixel columns covering every voxel column's window (monotone in the voxel index)
    const int a0 = window_start(p->s, jx0), a1 = window_start(p->s, jx1);
    const int c_lo = max(min(a0, a1), 0), c_hi = min(max(a0, a1) + wis - 1, ns - 1);
    const int ncols = c_hi - c_lo + 1;
    const bool sep = ncols > 0 && ncols <= AT_UCOLS;
    int flag_s = 0, flag_t = 0;
    for (int task = threadIdx.x; task < AT_S * wis + AT_T * wit; task += AT_THREADS) {
      if (task < AT_S * wis) {
        const int col = task / wis, q = task - col * wis;
        const int jx = jx0 + col;
        const int i = window_start(p->s, jx) + q;
        float w = 0.0f;
        if (i >= 0 && i < ns && jx < nx) {
          int jc;
          float fr;
          footprint_centre(p->s, i, jc, fr);
          w = cell_weight(jx - jc, fr, p->s);
        }
        const int ic = min(max(i, 0), ns - 1);
        sw[q][col] = w;
        si[q][col] = sep ? min(max(ic - c_lo, 0), ncols - 1) : ic;
        flag_s |= (w != 0.0f);
      } else {
        const int u = task - AT_S * wis;
        const int r = u / wit, q = u - r * wit;
        const int jy = jy0 + r;
        const int i = window_start(p->t, jy) + q;
        float w = 0.0f;
        if (i >= 0 && i < nt && jy < ny) {
          int jc;
          float fr;
          footprint_centre(p->t, i, jc, fr);
          w = cell_weight(jy - jc, fr, p->t);
        }
        tw[q][r] = w;
        ti[q][r] = min(max(i, 0), nt - 1) * ns;
        flag_t |= (w != 0.0f);
      }
    }
    const int any_s = __syncthreads_or(flag_s);
    const int any_t = __syncthreads_or(flag_t);
    if (any_s && any_t) {
      if (sep) {
        for (int c = lane; c < ncols; c += 32) {
          float u = 0.0f;
          for (int b = 0; b < wit; ++b) u = fmaf(tw[b][row], __ldg(g + ti[b][row] + c_lo + c), u);
          U[row][c] = u;
        }
        __syncwarp();
        float v = 0.0f;
        for (int q = 0; q < wis; ++q) v = fmaf(sw[q][lane], U[row][si[q][lane]], v);
        acc = fmaf(p->scale, v, acc);
      } else {
        float v = 0.0f;
        for (int b = 0; b < wit; ++b) {
          const float* gr = g + ti[b][row];
          float u = 0.0f;
          for (int q = 0; q < wis; ++q) u = fmaf(sw[q][lane], __ldg(gr + si[q][lane]), u);
          v = fmaf(tw[b][row], u, v);
        }
        acc = fmaf(p->scale, v, acc);
      }
    }
    __syncthreads();
  }
  const int jx = jx0 + lane;
  const int jy = jy0 + row;
  if (jx < nx && jy < ny) {
    float* o = x + (long long)frame * x_fs + ((long long)n * ny + jy) * nx + jx;
    *o = accumulate ? *o + acc : acc;
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
constexpr int L2_THREADS = 128;
constexpr int L2_W = kStage2Window;

// Bs[c][q] = entry (detector column dr.x + q, array column cc.x + c) and
// Bt[r][b] likewise; one task per detector column / row.
__device__ __forceinline__ void lenslet_weights(const LensletParam* L, int4 dr, int2 cc, int2 rr,
                                                float (*Bs)[L2_W + 1], float (*Bt)[L2_W + 1]) {
  const int nds = dr.y - dr.x + 1, ndt = dr.w - dr.z + 1;
  const int nc = cc.y - cc.x, nr = rr.y - rr.x;
  for (int task = threadIdx.x; task < nds + ndt; task += blockDim.x) {
    const bool s_axis = task < nds;
    const AxisParam& a = s_axis ? L->s : L->t;
    const int q = s_axis ? task : task - nds;
    const int i = s_axis ? dr.x + q : dr.z + q;
    const int j0 = s_axis ? cc.x : rr.x;
    const int n = s_axis ? nc : nr;
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
}

// Forward, pass 1: each lenslet's contribution sum_k Bt (x) Bs fa_k on the
// union over cells of its detector windows, written to zbuf (no overlap).
__global__ void __launch_bounds__(L2_THREADS)
stage2_lenslet_forward(const float* __restrict__ fa, StageTwo s2, long long fa_fs, float* __restrict__ zbuf) {
  __shared__ float Bs[MAXC][L2_W + 1];
  __shared__ float Bt[MAXC][L2_W + 1];
  __shared__ float F[MAXC][MAXC + 1];
  __shared__ float W[MAXC][L2_W + 1];
  __shared__ float Z[L2_W * L2_W];
  const int mu = blockIdx.x;
  const int frame = blockIdx.y;
  const int nmu = s2.mla_ns * s2.mla_nt;
  const int ms = mu % s2.mla_ns, mt = mu / s2.mla_ns;
  const int2 cc = s2.cols[ms], rr = s2.rows[mt];
  const int nc = cc.y - cc.x, nr = rr.y - rr.x;
  const int4 du = s2.det_union[mu];
  const int nsu = du.y - du.x + 1, ntu = du.w - du.z + 1;
  float* zout = zbuf + ((long long)frame * nmu + mu) * (L2_W * L2_W);
  const long long Na = (long long)s2.arr_ns * s2.arr_nt;
  for (int o = threadIdx.x; o < L2_W * L2_W; o += blockDim.x) Z[o] = 0.0f;
  if (nc > 0 && nr > 0 && nsu > 0 && ntu > 0) {
    for (int k = 0; k < s2.K; ++k) {
      const LensletParam* L = s2.lens + (long long)k * nmu + mu;
      const int4 dr = s2.det_range[(long long)k * nmu + mu];
      const int nds = dr.y - dr.x + 1, ndt = dr.w - dr.z + 1;
      if (nds <= 0 || ndt <= 0) continue;   // uniform
      lenslet_weights(L, dr, cc, rr, Bs, Bt);
      const float* fk = fa + (long long)frame * fa_fs + (long long)k * Na;
      for (int o = threadIdx.x; o < nr * nc; o += blockDim.x) {
        const int r = o / nc, c = o - r * nc;
        F[r][c] = __ldg(fk + (long long)(rr.x + r) * s2.arr_ns + cc.x + c);
      }
      __syncthreads();
      // W[r][q] = sum_c Bs[c][q] F[r][c]
      for (int o = threadIdx.x; o < nr * nds; o += blockDim.x) {
        const int r = o / nds, q = o - r * nds;
        float w = 0.0f;
        for (int c = 0; c < nc; ++c) w = fmaf(Bs[c][q], F[r][c], w);
        W[r][q] = w;
      }
      __syncthreads();
      // Z[it][is] += scale * sum_r Bt[r][b] W[r][q]  (entries owned by one thread)
      const float scale = L->scale;
      for (int o = threadIdx.x; o < ntu * nsu; o += blockDim.x) {
        const int b = o / nsu + du.z - dr.z, q = o % nsu + du.x - dr.x;
        if (b < 0 || b >= ndt || q < 0 || q >= nds) continue;
        float z = 0.0f;
        for (int r = 0; r < nr; ++r) z = fmaf(Bt[r][b], W[r][q], z);
        Z[o] = fmaf(scale, z, Z[o]);
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
  float acc = 0.0f;
  for (int mt = ct.x; mt <= ct.y; ++mt)
    for (int ms = cs.x; ms <= cs.y; ++ms) {
      const int mu = mt * s2.mla_ns + ms;
      const int4 du = s2.det_union[mu];
      if (is < du.x || is > du.y || it < du.z || it > du.w) continue;
      const int nsu = du.y - du.x + 1;
      acc += __ldg(zbuf + ((long long)frame * nmu + mu) * (L2_W * L2_W) + (it - du.z) * nsu + (is - du.x));
    }
  y[(long long)frame * y_fs + (long long)it * s2.det_ns + is] = acc;
}

// Adjoint: fa_k[jt][js] = M * scale * sum_b sum_q Bt[r][b] Bs[c][q] y[dr.z+b][dr.x+q]
// for the lenslet's own block (a gather: every array pixel has one lenslet).
__global__ void __launch_bounds__(L2_THREADS)
stage2_lenslet_adjoint(const float* __restrict__ y, float* __restrict__ fa, StageTwo s2, long long y_fs,
                       long long fa_fs) {
  __shared__ float Bs[MAXC][L2_W + 1];
  __shared__ float Bt[MAXC][L2_W + 1];
  __shared__ float Y[L2_W][L2_W + 1];
  __shared__ float U[MAXC][L2_W + 1];
  const int mu = blockIdx.x;
  const int frame = blockIdx.y;
  const int nmu = s2.mla_ns * s2.mla_nt;
  const int ms = mu % s2.mla_ns, mt = mu / s2.mla_ns;
  const int2 cc = s2.cols[ms], rr = s2.rows[mt];
  const int nc = cc.y - cc.x, nr = rr.y - rr.x;
  if (nc <= 0 || nr <= 0) return;   // uniform
  const long long Na = (long long)s2.arr_ns * s2.arr_nt;
  const float* yf = y + (long long)frame * y_fs;
  for (int k = 0; k < s2.K; ++k) {
    const LensletParam* L = s2.lens + (long long)k * nmu + mu;
    const int4 dr = s2.det_range[(long long)k * nmu + mu];
    const int nds = dr.y - dr.x + 1, ndt = dr.w - dr.z + 1;
    float* fk = fa + (long long)frame * fa_fs + (long long)k * Na;
    if (nds <= 0 || ndt <= 0) {
      for (int o = threadIdx.x; o < nr * nc; o += blockDim.x)
        fk[(long long)(rr.x + o / nc) * s2.arr_ns + cc.x + o % nc] = 0.0f;
      continue;   // uniform
    }
    lenslet_weights(L, dr, cc, rr, Bs, Bt);
    for (int o = threadIdx.x; o < ndt * nds; o += blockDim.x) {
      const int b = o / nds, q = o - b * nds;
      Y[b][q] = __ldg(yf + (long long)(dr.z + b) * s2.det_ns + dr.x + q);
    }
    __syncthreads();
    // U[r][q] = sum_b Bt[r][b] Y[b][q]
    for (int o = threadIdx.x; o < nr * nds; o += blockDim.x) {
      const int r = o / nds, q = o - r * nds;
      float u = 0.0f;
      for (int b = 0; b < ndt; ++b) u = fmaf(Bt[r][b], Y[b][q], u);
      U[r][q] = u;
    }
    __syncthreads();
    const float scale = L->scale;
    for (int o = threadIdx.x; o < nr * nc; o += blockDim.x) {
      const int r = o / nc, c = o - r * nc;
      const int jt = rr.x + r, js = cc.x + c;
      float g = 0.0f;
      for (int q = 0; q < nds; ++q) g = fmaf(Bs[c][q], U[r][q], g);
      fk[(long long)jt * s2.arr_ns + js] = s2.mask[(long long)jt * s2.arr_ns + js] ? scale * g : 0.0f;
    }
    __syncthreads();
  }
}

}  // namespace

template <int WS, int WT>
static void launch_fw(dim3 grid, cudaStream_t st, const float* x, float* out, const SliceParam* prm, int nx,
                      int ny, int nz, int ns, int nt, int K, int per_cell, const uint8_t* mask, long long xfs,
                      long long ofs, int tiles_s, int tiles_t, const int2* sr, const int2* tr) {
  beam_forward_kernel<WS, WT><<<grid, FT_THREADS, 0, st>>>(x, out, prm, nx, ny, nz, ns, nt, K, per_cell, mask,
                                                           xfs, ofs, tiles_s, tiles_t, sr, tr);
}

static int window_class(int w) { return w <= 2 ? 2 : w <= 3 ? 3 : w <= 4 ? 4 : 8; }

cudaError_t launch_beam_forward(const float* x, float* out, const SliceParam* prm,
                                int nx, int ny, int nz, int ns, int nt, int K,
                                int per_cell, const uint8_t* mask, int frames,
                                long long x_frame_stride, long long out_frame_stride,
                                int wmax_s, int wmax_t, const int2* srange, const int2* trange,
                                cudaStream_t st) {
  if (wmax_s > WMAX || wmax_t > WMAX) return cudaErrorInvalidValue;
  const int tiles_s = (ns + FT_S - 1) / FT_S;
  const int tiles_t = (nt + FT_T - 1) / FT_T;
  dim3 grid(tiles_s * tiles_t, per_cell ? K : 1, frames);
  const int cs = window_class(wmax_s), ct = window_class(wmax_t);
#define LT_FW(A, B)                                                                                     \
  if (cs == A && ct == B) {                                                                           \
    launch_fw<A, B>(grid, st, x, out, prm, nx, ny, nz, ns, nt, K, per_cell, mask, x_frame_stride,     \
                    out_frame_stride, tiles_s, tiles_t, srange, trange);                              \
    return cudaGetLastError();                                                                        \
  }
  LT_FW(2, 2) LT_FW(2, 3) LT_FW(2, 4) LT_FW(2, 8)
  LT_FW(3, 2) LT_FW(3, 3) LT_FW(3, 4) LT_FW(3, 8)
  LT_FW(4, 2) LT_FW(4, 3) LT_FW(4, 4) LT_FW(4, 8)
  LT_FW(8, 2) LT_FW(8, 3) LT_FW(8, 4) LT_FW(8, 8)
#undef LT_FW
  return cudaErrorInvalidValue;
}

cudaError_t launch_beam_adjoint(const float* in, float* x, const SliceParam* prm,
                                int nx, int ny, int nz, int ns, int nt, int K,
                                int per_cell, int accumulate, int frames,
                                long long in_frame_stride, long long x_frame_stride,
                                int wimax_s, int wimax_t, cudaStream_t st) {
  if (wimax_s > WIMAX || wimax_t > WIMAX) return cudaErrorInvalidValue;
  const int tiles_x = (nx + AT_S - 1) / AT_S;
  const int tiles_y = (ny + AT_T - 1) / AT_T;
  dim3 grid(tiles_x * tiles_y, nz, frames);
  beam_adjoint_kernel<<<grid, AT_THREADS, 0, st>>>(in, x, prm, nx, ny, nz, ns, nt, K, per_cell,
                                                   accumulate, in_frame_stride, x_frame_stride,
                                                   tiles_x);
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
  stage2_lenslet_adjoint<<<g, L2_THREADS, 0, st>>>(y, fa, s2, y_frame_stride, fa_frame_stride);
  return cudaGetLastError();
}

}  // namespace lt
