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
// half-width P and outer half-width Q (odd in x).
__device__ __forceinline__ float trap_F(float x, float P, float Q, float hir) {
  const float a = fabsf(x);
  float g;
  if (a <= P) {
    g = a;
  } else if (a < Q) {
    const float d = __fsub_rn(a, P);
    g = __fsub_rn(a, __fmul_rn(__fmul_rn(d, d), hir));
  } else {
    g = __fmul_rn(0.5f, __fadd_rn(P, Q));
  }
  return copysignf(g, x);
}

// Integral of the unit trapezoid centred at fr over source cell m (relative
// to jc): [m - 1/2, m + 1/2].  Exactly 0 outside the footprint.
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
// Beam integration, forward.  CTA = 32 x 16 target pixels of one frame (and
// one cell if per_cell); 4 warps, warp w owns rows w, w+4, w+8, w+12.  For
// each (cell, slice) warp 0 evaluates the s-weights of the 32 columns and warp
// 1 the t-weights of the 16 rows into shared memory (the separable O(S+T)
// weight work of Sec. IV-B, shared by the whole tile); then every thread
// accumulates its pixels from the L1-resident slice.
// ---------------------------------------------------------------------------
constexpr int FT_S = 32;
constexpr int FT_T = 16;
constexpr int FT_THREADS = 128;

__global__ void __launch_bounds__(FT_THREADS)
beam_forward_kernel(const float* __restrict__ x, float* __restrict__ out,
                    const SliceParam* __restrict__ prm, int nx, int ny, int nz,
                    int ns, int nt, int K, int per_cell, const uint8_t* __restrict__ mask,
                    long long x_fs, long long out_fs, int tiles_s) {
  __shared__ float sw[WMAX][FT_S];
  __shared__ int sx[WMAX][FT_S];
  __shared__ float tw[WMAX][FT_T];
  __shared__ int ty[WMAX][FT_T];

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int is0 = (blockIdx.x % tiles_s) * FT_S;
  const int it0 = (blockIdx.x / tiles_s) * FT_T;
  const int frame = blockIdx.z;
  const int k_begin = per_cell ? (int)blockIdx.y : 0;
  const int k_end = per_cell ? (int)blockIdx.y + 1 : K;
  const float* xf = x + (long long)frame * x_fs;

  float acc[FT_T / 4];
#pragma unroll
  for (int r = 0; r < FT_T / 4; ++r) acc[r] = 0.0f;

  for (int k = k_begin; k < k_end; ++k) {
    for (int n = 0; n < nz; ++n) {
      const SliceParam* p = prm + (long long)k * nz + n;
      const int ws = p->ws;
      const int wt = p->wt;
      int flag_s = 0, flag_t = 0;
      if (warp == 0) {
        int jc;
        float fr;
        footprint_centre(p->s, is0 + lane, jc, fr);
        const int mlo = (int)floorf(fr - p->s.Q + 0.5f);
        for (int a = 0; a < ws; ++a) {
          const int j = jc + mlo + a;
          float w = cell_weight(mlo + a, fr, p->s);
          if (j < 0 || j >= nx) w = 0.0f;
          sw[a][lane] = w;
          sx[a][lane] = min(max(j, 0), nx - 1);
          flag_s |= (w != 0.0f);
        }
      } else if (warp == 1 && lane < FT_T) {
        int jc;
        float fr;
        footprint_centre(p->t, it0 + lane, jc, fr);
        const int mlo = (int)floorf(fr - p->t.Q + 0.5f);
        for (int b = 0; b < wt; ++b) {
          const int j = jc + mlo + b;
          float w = cell_weight(mlo + b, fr, p->t);
          if (j < 0 || j >= ny) w = 0.0f;
          tw[b][lane] = w;
          ty[b][lane] = min(max(j, 0), ny - 1);
          flag_t |= (w != 0.0f);
        }
      }
      const int any_s = __syncthreads_or(flag_s);
      const int any_t = __syncthreads_or(flag_t);
      if (any_s && any_t) {
        const float scale = p->scale;
        const float* xs = xf + (long long)n * ny * nx;
#pragma unroll
        for (int r = 0; r < FT_T / 4; ++r) {
          const int row = warp + 4 * r;
          float v = 0.0f;
          for (int b = 0; b < wt; ++b) {
            const float wtb = tw[b][row];
            if (wtb != 0.0f) {
              const float* xr = xs + (long long)ty[b][row] * nx;
              float u = 0.0f;
              for (int a = 0; a < ws; ++a) u = fmaf(sw[a][lane], __ldg(xr + sx[a][lane]), u);
              v = fmaf(wtb, u, v);
            }
          }
          acc[r] = fmaf(scale, v, acc[r]);
        }
      }
      __syncthreads();
    }
  }

  const int is = is0 + lane;
  if (is < ns) {
    float* o = out + (long long)frame * out_fs + (per_cell ? (long long)blockIdx.y * ns * nt : 0);
#pragma unroll
    for (int r = 0; r < FT_T / 4; ++r) {
      const int it = it0 + warp + 4 * r;
      if (it < nt) {
        float v = acc[r];
        if (mask && !mask[(long long)it * ns + is]) v = 0.0f;
        o[(long long)it * ns + is] = v;
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

__global__ void __launch_bounds__(AT_THREADS)
beam_adjoint_kernel(const float* __restrict__ in, float* __restrict__ x,
                    const SliceParam* __restrict__ prm, int nx, int ny, int nz,
                    int ns, int nt, int K, int per_cell, int accumulate,
                    long long in_fs, long long x_fs, int tiles_x) {
  __shared__ float sw[WIMAX][AT_S];
  __shared__ int si[WIMAX][AT_S];
  __shared__ float tw[WIMAX][AT_T];
  __shared__ int ti[WIMAX][AT_T];

  const int lane = threadIdx.x & 31;
  const int row = threadIdx.x >> 5;
  const int jx0 = (blockIdx.x % tiles_x) * AT_S;
  const int jy0 = (blockIdx.x / tiles_x) * AT_T;
  const int n = blockIdx.y;
  const int frame = blockIdx.z;
  const float* inf = in + (long long)frame * in_fs;

  float acc = 0.0f;
  for (int k = 0; k < K; ++k) {
    const SliceParam* p = prm + (long long)k * nz + n;
    const int wis = p->wis;
    const int wit = p->wit;
    int flag_s = 0, flag_t = 0;
    if (row == 0) {
      const int jx = jx0 + lane;
      const int i0 = window_start(p->s, jx);
      for (int q = 0; q < wis; ++q) {
        const int i = i0 + q;
        float w = 0.0f;
        if (i >= 0 && i < ns && jx < nx) {
          int jc;
          float fr;
          footprint_centre(p->s, i, jc, fr);
          w = cell_weight(jx - jc, fr, p->s);
        }
        sw[q][lane] = w;
        si[q][lane] = min(max(i, 0), ns - 1);
        flag_s |= (w != 0.0f);
      }
    } else if (row == 1 && lane < AT_T) {
      const int jy = jy0 + lane;
      const int i0 = window_start(p->t, jy);
      for (int q = 0; q < wit; ++q) {
        const int i = i0 + q;
        float w = 0.0f;
        if (i >= 0 && i < nt && jy < ny) {
          int jc;
          float fr;
          footprint_centre(p->t, i, jc, fr);
          w = cell_weight(jy - jc, fr, p->t);
        }
        tw[q][lane] = w;
        ti[q][lane] = min(max(i, 0), nt - 1);
        flag_t |= (w != 0.0f);
      }
    }
    const int any_s = __syncthreads_or(flag_s);
    const int any_t = __syncthreads_or(flag_t);
    if (any_s && any_t) {
      const float* g = inf + (per_cell ? (long long)k * ns * nt : 0);
      float v = 0.0f;
      for (int b = 0; b < wit; ++b) {
        const float wtb = tw[b][row];
        if (wtb != 0.0f) {
          const float* gr = g + (long long)ti[b][row] * ns;
          float u = 0.0f;
          for (int q = 0; q < wis; ++q) u = fmaf(sw[q][lane], __ldg(gr + si[q][lane]), u);
          v = fmaf(wtb, u, v);
        }
      }
      acc = fmaf(p->scale, v, acc);
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
// Plenoptic stage two, forward: one thread per detector pixel; for each cell,
// the lenslets whose sub-images can reach the pixel (host table), and for each
// lenslet its array block (rows x cols, masked coefficients).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
stage2_forward_kernel(const float* __restrict__ fa, float* __restrict__ y, StageTwo s2,
                      long long fa_fs, long long y_fs) {
  const int is = blockIdx.x * 32 + (threadIdx.x & 31);
  const int it = blockIdx.y * 8 + (threadIdx.x >> 5);
  const int frame = blockIdx.z;
  if (is >= s2.det_ns || it >= s2.det_nt) return;
  const long long Na = (long long)s2.arr_ns * s2.arr_nt;
  const int nmu = s2.mla_ns * s2.mla_nt;
  float acc = 0.0f;
  for (int k = 0; k < s2.K; ++k) {
    const int2 cs = s2.cand_s[(long long)k * s2.det_ns + is];
    const int2 ct = s2.cand_t[(long long)k * s2.det_nt + it];
    const float* fk = fa + (long long)frame * fa_fs + (long long)k * Na;
    for (int mt = ct.x; mt <= ct.y; ++mt) {
      const int2 rr = s2.rows[mt];
      for (int ms = cs.x; ms <= cs.y; ++ms) {
        const int2 cc = s2.cols[ms];
        const int nc = cc.y - cc.x;
        const LensletParam* L = s2.lens + (long long)k * nmu + mt * s2.mla_ns + ms;
        int jcs, jct;
        float frs, frt;
        footprint_centre(L->s, is, jcs, frs);
        footprint_centre(L->t, it, jct, frt);
        float ws[MAXC];
#pragma unroll
        for (int a = 0; a < MAXC; ++a) ws[a] = (a < nc) ? cell_weight(cc.x + a - jcs, frs, L->s) : 0.0f;
        float v = 0.0f;
        for (int r = rr.x; r < rr.y; ++r) {
          const float wt = cell_weight(r - jct, frt, L->t);
          if (wt != 0.0f) {
            const float* fr = fk + (long long)r * s2.arr_ns + cc.x;
            float u = 0.0f;
#pragma unroll
            for (int a = 0; a < MAXC; ++a)
              if (a < nc) u = fmaf(ws[a], __ldg(fr + a), u);
            v = fmaf(wt, u, v);
          }
        }
        acc = fmaf(L->scale, v, acc);
      }
    }
  }
  y[(long long)frame * y_fs + (long long)it * s2.det_ns + is] = acc;
}

// ---------------------------------------------------------------------------
// Plenoptic stage two, gather adjoint: one thread per array pixel and frame;
// for each cell, the window of detector pixels whose footprints (through the
// pixel's own lenslet) may cover it.  Masked pixels get 0 (M^T = M).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
stage2_adjoint_kernel(const float* __restrict__ y, float* __restrict__ fa, StageTwo s2,
                      long long y_fs, long long fa_fs) {
  const int js = blockIdx.x * 32 + (threadIdx.x & 31);
  const int jt = blockIdx.y * 8 + (threadIdx.x >> 5);
  const int frame = blockIdx.z;
  if (js >= s2.arr_ns || jt >= s2.arr_nt) return;
  const long long Na = (long long)s2.arr_ns * s2.arr_nt;
  const int nmu = s2.mla_ns * s2.mla_nt;
  const int ms = s2.col_owner[js];
  const int mt = s2.row_owner[jt];
  const bool on = ms >= 0 && mt >= 0 && s2.mask[(long long)jt * s2.arr_ns + js];
  const float* yf = y + (long long)frame * y_fs;
  for (int k = 0; k < s2.K; ++k) {
    float acc = 0.0f;
    if (on) {
      const LensletParam* L = s2.lens + (long long)k * nmu + mt * s2.mla_ns + ms;
      const int i0s = window_start(L->s, js);
      const int i0t = window_start(L->t, jt);
      float ws[WIMAX];
#pragma unroll
      for (int q = 0; q < WIMAX; ++q) {
        const int i = i0s + q;
        float w = 0.0f;
        if (q < s2.wis && i >= 0 && i < s2.det_ns) {
          int jc;
          float fr;
          footprint_centre(L->s, i, jc, fr);
          w = cell_weight(js - jc, fr, L->s);
        }
        ws[q] = w;
      }
      float v = 0.0f;
      for (int b = 0; b < s2.wit; ++b) {
        const int i = i0t + b;
        if (i < 0 || i >= s2.det_nt) continue;
        int jc;
        float fr;
        footprint_centre(L->t, i, jc, fr);
        const float wt = cell_weight(jt - jc, fr, L->t);
        if (wt != 0.0f) {
          const float* yr = yf + (long long)i * s2.det_ns;
          float u = 0.0f;
#pragma unroll
          for (int q = 0; q < WIMAX; ++q) {
            const int ii = i0s + q;
            if (ws[q] != 0.0f) u = fmaf(ws[q], __ldg(yr + ii), u);
          }
          v = fmaf(wt, u, v);
        }
      }
      acc = L->scale * v;
    }
    fa[(long long)frame * fa_fs + (long long)k * Na + (long long)jt * s2.arr_ns + js] = acc;
  }
}

}  // namespace

cudaError_t launch_beam_forward(const float* x, float* out, const SliceParam* prm,
                                int nx, int ny, int nz, int ns, int nt, int K,
                                int per_cell, const uint8_t* mask, int frames,
                                long long x_frame_stride, long long out_frame_stride,
                                int wmax_s, int wmax_t, cudaStream_t st) {
  if (wmax_s > WMAX || wmax_t > WMAX) return cudaErrorInvalidValue;
  const int tiles_s = (ns + FT_S - 1) / FT_S;
  const int tiles_t = (nt + FT_T - 1) / FT_T;
  dim3 grid(tiles_s * tiles_t, per_cell ? K : 1, frames);
  beam_forward_kernel<<<grid, FT_THREADS, 0, st>>>(x, out, prm, nx, ny, nz, ns, nt, K, per_cell,
                                                   mask, x_frame_stride, out_frame_stride, tiles_s);
  return cudaGetLastError();
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
                                  cudaStream_t st) {
  if (s2.max_cols > MAXC || s2.max_rows > MAXC) return cudaErrorInvalidValue;
  dim3 grid((s2.det_ns + 31) / 32, (s2.det_nt + 7) / 8, frames);
  stage2_forward_kernel<<<grid, 256, 0, st>>>(fa, y, s2, fa_frame_stride, y_frame_stride);
  return cudaGetLastError();
}

cudaError_t launch_stage2_adjoint(const float* y, float* fa, StageTwo s2, int frames,
                                  long long y_frame_stride, long long fa_frame_stride,
                                  cudaStream_t st) {
  if (s2.wis > WIMAX || s2.wit > WIMAX) return cudaErrorInvalidValue;
  dim3 grid((s2.arr_ns + 31) / 32, (s2.arr_nt + 7) / 8, frames);
  stage2_adjoint_kernel<<<grid, 256, 0, st>>>(y, fa, s2, y_frame_stride, fa_frame_stride);
  return cudaGetLastError();
}

}  // namespace lt
