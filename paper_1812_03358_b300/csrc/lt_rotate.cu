// Rotated perspectives (Sec. III-A): quarter turns and the two shear passes
// of the residual yaw, with their exact transposes.  Every pass is a 1-D
// Toeplitz re-projection per column (eq. rot,toeplitz) streamed with one
// thread per output element (HBM bound); forward and adjoint evaluate the
// same entries with the same function, so they are exact transposes up to
// float32 summation order.
#include <climits>

#include "lt_internal.h"

namespace lt {
namespace {

__device__ __forceinline__ float hat(float t) { return fmaxf(0.0f, __fsub_rn(1.0f, fabsf(t))); }

// Average of the hat max(0, 1 - |t|) over [u - beta/2, u + beta/2], summed
// exactly piece by piece between the kinks -1, 0, 1 (no cancellation at small
// beta); hat(u) when beta = 0.
__device__ __forceinline__ float hat_avg(float u, float beta) {
  if (beta == 0.0f) return hat(u);
  const float lo = __fsub_rn(u, __fmul_rn(0.5f, beta));
  const float hi = __fadd_rn(u, __fmul_rn(0.5f, beta));
  float acc = 0.0f, a = lo;
#pragma unroll
  for (int k = -1; k <= 1; ++k) {
    const float kk = (float)k;
    if (a < kk && kk < hi) {
      acc = __fadd_rn(acc, __fmul_rn(__fsub_rn(kk, a), hat(__fmul_rn(0.5f, __fadd_rn(a, kk)))));
      a = kk;
    }
  }
  acc = __fadd_rn(acc, __fmul_rn(__fsub_rn(hi, a), hat(__fmul_rn(0.5f, __fadd_rn(a, hi)))));
  return __fdiv_rn(acc, beta);
}

// u of the entry (output i, source j) in a column whose shift is sh.
__device__ __forceinline__ float shear_u(int i, int j, int pad, float sh) {
  return __fadd_rn((float)(i - j - pad), sh);
}

__device__ __forceinline__ float column_shift(float slope, int c, int n_c) {
  return __fmul_rn(slope, __fsub_rn((float)c, 0.5f * (float)(n_c - 1)));
}

// Index in the original volume of permuted-grid voxel (jz, iy, jx) after NQ
// quarter turns.
template <int NQ>
__device__ __forceinline__ long long perm_index(const RotParam& r, int jz, int iy, int jx) {
  int iz, ix;
  if (NQ == 1) { iz = r.nz - 1 - jx; ix = jz; }
  else if (NQ == 2) { iz = r.nz - 1 - jz; ix = r.nx - 1 - jx; }
  else if (NQ == 3) { iz = jx; ix = r.nx - 1 - jz; }
  else { iz = jz; ix = jx; }
  return ((long long)iz * r.ny + iy) * r.nx + ix;
}

// perm_index is affine in jz: voxel (jz, iy, c) sits at off0 + jz * sj.
template <int NQ>
__device__ __forceinline__ void perm_line(const RotParam& r, int iy, int c, long long& off0, long long& sj) {
  off0 = perm_index<NQ>(r, 0, iy, c);
  sj = perm_index<NQ>(r, 1, iy, c) - off0;
}

// Entries of a shear pass depend on the output/source offset and the
// column's shift only, so each column's band is tabulated once (plan time):
// window offset J = floor(sh - 1 - beta/2) - 1 and, for q = 0..nw-1, the entry
// between output i and source i - pad + J + q, hat_avg(-J - q + sh, beta) --
// the same float operations as shear_u(i, i - pad + J + q, pad, sh), so the
// forward and adjoint passes below read identical entries.
__global__ void shear_tables_kernel(RotParam r) {
  const int n = r.nxp + r.nzr;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const bool zcol = t < r.nxp;
    const int c = zcol ? t : t - r.nxp;
    const float slope = zcol ? r.bz : r.ax, beta = zcol ? r.betaz : r.betax;
    const float sh = column_shift(slope, c, zcol ? r.nxp : r.nzr);
    const int J = (int)floorf(sh - 1.0f - 0.5f * beta) - 1;
    const int w = zcol ? r.wz : r.wx, nw = zcol ? r.nwz : r.wx;
    float* tab = zcol ? r.tz + (long long)c * nw : r.tx + (long long)c * nw;
    for (int q = 0; q < nw; ++q) tab[q] = q < w ? hat_avg(shear_u(0, J + q, 0, sh), beta) : 0.0f;
    (zcol ? r.jz : r.jx)[c] = J;
  }
}

constexpr int kShearZChunk = 16;   // outputs along the sheared axis per thread

// rz[f][izr][iy][c] = sum_q tz[c][q] xp[f][izr - pz + jz[c] + q][iy][c], xp the
// quarter-turned volume.  Thread = (iy, c) column and kShearZChunk outputs
// along izr; the chunk's whole source window (kShearZChunk + NW - 1 values)
// is loaded before any output is formed, so that every load of the chunk is
// in flight at once (one dependent load per output left the pass
// latency-bound at a fifth of the HBM rate).
template <int NW, int NQ>
__global__ void __launch_bounds__(256) shear_z_forward(const float* __restrict__ x, float* __restrict__ rz,
                                                       RotParam r, int frames) {
  const int c = blockIdx.x * 32 + threadIdx.x;
  const int iy = blockIdx.y * 8 + threadIdx.y;
  const int z0 = blockIdx.z * kShearZChunk;
  if (c >= r.nxp || iy >= r.ny) return;
  const long long nvox = (long long)r.nx * r.ny * r.nz;
  const long long per = (long long)r.nzr * r.ny * r.nxp;
  const long long zstride = (long long)r.ny * r.nxp;
  float w[NW];
#pragma unroll
  for (int q = 0; q < NW; ++q) w[q] = __ldg(r.tz + (long long)c * NW + q);
  const int J = __ldg(r.jz + c);
  const int nout = min(kShearZChunk, r.nzr - z0);
  long long off0, sj;
  perm_line<NQ>(r, iy, c, off0, sj);
  for (int f = 0; f < frames; ++f) {
    float* out = rz + (long long)f * per + (long long)iy * r.nxp + c;
    const int jb = z0 - r.pz + J;   // first source of output z0
    // source jb + q at ps + q * sj (formed only where it is in the volume)
    const float* ps = x + (long long)f * nvox + off0 + (long long)jb * sj;
    float v[kShearZChunk + NW - 1];
    if (jb >= 0 && jb + kShearZChunk + NW - 1 <= r.nzp) {   // window inside the volume
#pragma unroll
      for (int q = 0; q < kShearZChunk + NW - 1; ++q) v[q] = __ldg(ps + q * sj);
    } else {
#pragma unroll
      for (int q = 0; q < kShearZChunk + NW - 1; ++q)
        v[q] = (unsigned)(jb + q) < (unsigned)r.nzp ? __ldg(ps + q * sj) : 0.0f;
    }
#pragma unroll
    for (int t = 0; t < kShearZChunk; ++t) {
      if (t < nout) {
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < NW; ++q) acc = fmaf(w[q], v[t + q], acc);
        out[(long long)(z0 + t) * zstride] = acc;
      }
    }
  }
}

constexpr int kShearXWarps = 8;   // rows (one per warp) per CTA of the staged x passes
constexpr int kShearXSmemMax = 48 * 1024;

// xr[f][izr][iy][ixr] = sum_q tx[izr][q] rz[f][izr][iy][ixr - px + jx[izr] + q].
// Warp = one row (izr, iy): the row's nxp inputs are staged in the warp's
// shared-memory slice between WX zeros, so that a window overlapping the row
// reads inputs or zeros with no bounds test per tap; lane = outputs lane +
// 32 k.  The taps run in ascending q with zero weights past wx, which gives
// the generic loop's values bit for bit (a tap outside the row adds w * 0).
template <int WX>
__global__ void __launch_bounds__(32 * kShearXWarps) shear_x_forward_rows(const float* __restrict__ rz,
                                                                          float* __restrict__ xr, RotParam r,
                                                                          int frames) {
  extern __shared__ float smem_rows[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int iy = blockIdx.x * kShearXWarps + wid;
  const int izr = blockIdx.y;
  if (iy >= r.ny) return;   // warp-uniform; no block barrier below
  const int L = r.nxp + 2 * WX;
  float* Rw = smem_rows + wid * L;
  if (lane < WX) {
    Rw[lane] = 0.0f;
    Rw[WX + r.nxp + lane] = 0.0f;
  }
  const long long per_in = (long long)r.nzr * r.ny * r.nxp;
  const long long per = (long long)r.nzr * r.ny * r.nxr;
  const float* tab = r.tx + (long long)izr * r.wx;
  float w[WX];
#pragma unroll
  for (int q = 0; q < WX; ++q) w[q] = q < r.wx ? __ldg(tab + q) : 0.0f;
  const int off = __ldg(r.jx + izr) - r.px;   // output ixr's first source is ixr + off
  for (int f = 0; f < frames; ++f) {
    const float* row = rz + (long long)f * per_in + ((long long)izr * r.ny + iy) * r.nxp;
    __syncwarp();   // the previous frame's reads are done
    for (int j = lane; j < r.nxp; j += 32) Rw[WX + j] = __ldg(row + j);
    __syncwarp();
    float* o = xr + (long long)f * per + ((long long)izr * r.ny + iy) * r.nxr;
    for (int ixr = lane; ixr < r.nxr; ixr += 32) {
      const int jb = ixr + off;
      float acc = 0.0f;
      if (jb > -WX && jb < r.nxp) {   // else every tap lies outside the row
        const float* src = Rw + WX + jb;
#pragma unroll
        for (int q = 0; q < WX; ++q) acc = fmaf(w[q], src[q], acc);
      }
      o[ixr] = acc;
    }
  }
}

// Generic x pass (windows wider than 16): one output per thread.
__global__ void __launch_bounds__(256) shear_x_forward(const float* __restrict__ rz, float* __restrict__ xr,
                                                       RotParam r, int frames) {
  const int ixr = blockIdx.x * 32 + threadIdx.x;
  const int iy = blockIdx.y * 8 + threadIdx.y;
  const int izr = blockIdx.z;
  if (ixr >= r.nxr || iy >= r.ny) return;
  const long long per_in = (long long)r.nzr * r.ny * r.nxp;
  const long long per = (long long)r.nzr * r.ny * r.nxr;
  const float* tab = r.tx + (long long)izr * r.wx;
  const int jb = ixr - r.px + __ldg(r.jx + izr);
  for (int f = 0; f < frames; ++f) {
    const float* row = rz + (long long)f * per_in + ((long long)izr * r.ny + iy) * r.nxp;
    float acc = 0.0f;
    for (int q = 0; q < r.wx; ++q) {
      const int j = jb + q;
      if (j >= 0 && j < r.nxp) acc = fmaf(__ldg(tab + q), __ldg(row + j), acc);
    }
    xr[(long long)f * per + ((long long)izr * r.ny + iy) * r.nxr + ixr] = acc;
  }
}

// grz[f][izr][iy][j] = sum_ixr E^x(ixr, j; izr) g[f][izr][iy][ixr]: outputs
// i = j + px - jx[izr] - q, visited in ascending i.  Warp = one row, its nxr
// values of g staged between WX zeros (as shear_x_forward_rows); lane =
// sources lane + 32 k.
template <int WX>
__global__ void __launch_bounds__(32 * kShearXWarps) shear_x_adjoint_rows(const float* __restrict__ g,
                                                                          float* __restrict__ grz, RotParam r,
                                                                          int frames) {
  extern __shared__ float smem_rows[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int iy = blockIdx.x * kShearXWarps + wid;
  const int izr = blockIdx.y;
  if (iy >= r.ny) return;   // warp-uniform; no block barrier below
  const int L = r.nxr + 2 * WX;
  float* Gw = smem_rows + wid * L;
  if (lane < WX) {
    Gw[lane] = 0.0f;
    Gw[WX + r.nxr + lane] = 0.0f;
  }
  const long long per_in = (long long)r.nzr * r.ny * r.nxr;
  const long long per = (long long)r.nzr * r.ny * r.nxp;
  const float* tab = r.tx + (long long)izr * r.wx;
  float w[WX];
#pragma unroll
  for (int q = 0; q < WX; ++q) w[q] = q < r.wx ? __ldg(tab + q) : 0.0f;
  const int off = r.px - __ldg(r.jx + izr);   // source j's last tap is output j + off
  for (int f = 0; f < frames; ++f) {
    const float* row = g + (long long)f * per_in + ((long long)izr * r.ny + iy) * r.nxr;
    __syncwarp();
    for (int i = lane; i < r.nxr; i += 32) Gw[WX + i] = __ldg(row + i);
    __syncwarp();
    float* o = grz + (long long)f * per + ((long long)izr * r.ny + iy) * r.nxp;
    for (int j = lane; j < r.nxp; j += 32) {
      const int ib = j + off;
      float acc = 0.0f;
      if (ib >= 0 && ib - (WX - 1) < r.nxr) {   // else every tap lies outside the row
        const float* src = Gw + WX + ib;
#pragma unroll
        for (int q = WX - 1; q >= 0; --q) acc = fmaf(w[q], src[-q], acc);
      }
      o[j] = acc;
    }
  }
}

// Generic transposed x pass (windows wider than 16): one source per thread.
__global__ void __launch_bounds__(256) shear_x_adjoint(const float* __restrict__ g, float* __restrict__ grz,
                                                       RotParam r, int frames) {
  const int j = blockIdx.x * 32 + threadIdx.x;
  const int iy = blockIdx.y * 8 + threadIdx.y;
  const int izr = blockIdx.z;
  if (j >= r.nxp || iy >= r.ny) return;
  const long long per_in = (long long)r.nzr * r.ny * r.nxr;
  const long long per = (long long)r.nzr * r.ny * r.nxp;
  const float* tab = r.tx + (long long)izr * r.wx;
  const int ib = j + r.px - __ldg(r.jx + izr);
  for (int f = 0; f < frames; ++f) {
    const float* row = g + (long long)f * per_in + ((long long)izr * r.ny + iy) * r.nxr;
    float acc = 0.0f;
    for (int q = r.wx - 1; q >= 0; --q) {
      const int i = ib - q;
      if (i >= 0 && i < r.nxr) acc = fmaf(__ldg(tab + q), __ldg(row + i), acc);
    }
    grz[(long long)f * per + ((long long)izr * r.ny + iy) * r.nxp + j] = acc;
  }
}

// x[f][perm(jz, iy, c)] (= or +=) sum_i E^z(i, jz; c) grz[f][i][iy][c]:
// outputs i = jz + pz - jz_tab[c] - q in ascending order.  Thread = (iy, c)
// column and kShearZChunk sources along jz, the chunk's whole window of grz
// loaded first (as in shear_z_forward).
template <int NW, int NQ>
__global__ void __launch_bounds__(256) shear_z_adjoint(const float* __restrict__ grz, float* __restrict__ x,
                                                       RotParam r, int frames, int accumulate) {
  const int c = blockIdx.x * 32 + threadIdx.x;
  const int iy = blockIdx.y * 8 + threadIdx.y;
  const int z0 = blockIdx.z * kShearZChunk;
  if (c >= r.nxp || iy >= r.ny) return;
  const long long nvox = (long long)r.nx * r.ny * r.nz;
  const long long per_in = (long long)r.nzr * r.ny * r.nxp;
  const long long zstride = (long long)r.ny * r.nxp;
  float w[NW];   // w[k] weights the k-th value of the window (ascending i)
#pragma unroll
  for (int k = 0; k < NW; ++k) w[k] = __ldg(r.tz + (long long)c * NW + (NW - 1 - k));
  const int J = __ldg(r.jz + c);
  const int nout = min(kShearZChunk, r.nzp - z0);
  long long off0, sj;
  perm_line<NQ>(r, iy, c, off0, sj);
  for (int f = 0; f < frames; ++f) {
    const int ib = z0 + r.pz - J - (NW - 1);   // first output row of source z0
    // row ib + k at gi + k * zstride (formed only where it is in the grid)
    const float* gi = grz + (long long)f * per_in + (long long)iy * r.nxp + c + (long long)ib * zstride;
    float* xo = x + (long long)f * nvox + off0 + (long long)z0 * sj;   // source z0 + t at xo + t * sj
    float v[kShearZChunk + NW - 1];
    if (ib >= 0 && ib + kShearZChunk + NW - 1 <= r.nzr) {   // window inside the grid
#pragma unroll
      for (int k = 0; k < kShearZChunk + NW - 1; ++k) v[k] = __ldg(gi + k * zstride);
    } else {
#pragma unroll
      for (int k = 0; k < kShearZChunk + NW - 1; ++k)
        v[k] = (unsigned)(ib + k) < (unsigned)r.nzr ? __ldg(gi + k * zstride) : 0.0f;
    }
    float res[kShearZChunk];
#pragma unroll
    for (int t = 0; t < kShearZChunk; ++t) {
      float acc = 0.0f;
#pragma unroll
      for (int k = 0; k < NW; ++k) acc = fmaf(w[k], v[t + k], acc);
      res[t] = acc;
    }
    if (accumulate) {   // every old value read before any is written
#pragma unroll
      for (int t = 0; t < kShearZChunk; ++t)
        if (t < nout) res[t] += xo[t * sj];
    }
#pragma unroll
    for (int t = 0; t < kShearZChunk; ++t)
      if (t < nout) xo[t * sj] = res[t];
  }
}

// After one or three quarter turns, column (iy, c) of the permuted grid is a
// row of the original volume (contiguous along the sheared axis, sj = +-1),
// and neighbouring columns c are a whole x-y plane apart.  The per-column
// forward above still streams well there: each thread reads its own
// contiguous run, which the L1 cache serves.  Its transpose does not: each
// thread writes its own run, one float per plane per store.  The transposed
// adjoint below takes 32 columns c0..c0+31 of one iy and kZT sources along
// the sheared axis per CTA and stages the tile in shared memory, so that
// rows of the rotated grid are read by a warp along c and rows of the
// original volume are written by a warp along the row.  Each value is the
// same fmaf chain, in the same order, as in the per-column adjoint.  (A
// transposed forward built the same way measured slower than the per-column
// one, 1.7-2.1 ms against 1.6-1.7 ms per camera at 256^3 x 16 frames.)
constexpr int kZT = 64;   // sources along the sheared axis per tile

// Adjoint: sources jz = z0..z0+kZT-1 of 32 columns need output rows
// ilo .. ilo + rows - 1 of the rotated grid (rows = kZT + NW - 1 plus the
// tile's window spread, at most r.djz).  Warps stage those rows along c
// (row stride 32: lane = column reads its own bank whatever its row), lane =
// column forms sources 8w..8w+7 into a second tile (row stride kZT + 1), and
// warp w then writes columns w, w + 8, ... as contiguous runs of the
// original rows, adding the old values first when accumulating.
template <int NW, int NQ>
__global__ void __launch_bounds__(256, 4) shear_z_adjoint_t(const float* __restrict__ grz, float* __restrict__ x,
                                                         RotParam r, int frames, int accumulate) {
  extern __shared__ float zsm[];
  const int rows_max = kZT + NW - 1 + r.djz;
  float* gt = zsm;                      // [rows_max][32]
  float* ot = zsm + rows_max * 32;      // [32][kZT + 1]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int z0 = blockIdx.x * kZT, c0 = blockIdx.y * 32, iy = blockIdx.z;
  const int c = c0 + lane;
  const bool cin = c < r.nxp;
  const long long nvox = (long long)r.nx * r.ny * r.nz;
  const long long per_in = (long long)r.nzr * r.ny * r.nxp;
  const long long zstride = (long long)r.ny * r.nxp;
  const int J = cin ? __ldg(r.jz + c) : 0;
  int jmax = cin ? J : INT_MIN, jmin = cin ? J : INT_MAX;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    jmax = max(jmax, __shfl_xor_sync(0xffffffffu, jmax, o));
    jmin = min(jmin, __shfl_xor_sync(0xffffffffu, jmin, o));
  }
  // The plan tabulates r.djz from the same offsets, so the spread fits; a
  // tile where it did not would be written as NaN, never read out of range.
  const bool fits = jmax - jmin <= r.djz;
  const int spread = fits ? jmax - jmin : r.djz;
  const int rows = kZT + NW - 1 + spread;
  const int ilo = z0 + r.pz - jmax - (NW - 1);
  const int d = cin ? min(jmax - J, spread) : 0;
  float wk[NW];   // wk[k] weights the k-th value of the window (ascending output row)
#pragma unroll
  for (int k = 0; k < NW; ++k) wk[k] = cin ? __ldg(r.tz + (long long)c * NW + (NW - 1 - k)) : 0.0f;
  const int nout = min(kZT, r.nzp - z0);
  for (int f = 0; f < frames; ++f) {
    const float* g = grz + (long long)f * per_in + (long long)iy * r.nxp + c;
    for (int row = w; row < rows; row += 8) {
      const int i = ilo + row;
      gt[row * 32 + lane] = cin && (unsigned)i < (unsigned)r.nzr ? __ldg(g + (long long)i * zstride) : 0.0f;
    }
    __syncthreads();
    float v[8 + NW - 1];
#pragma unroll
    for (int k = 0; k < 8 + NW - 1; ++k) v[k] = gt[(8 * w + d + k) * 32 + lane];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      float acc = 0.0f;
#pragma unroll
      for (int k = 0; k < NW; ++k) acc = fmaf(wk[k], v[t + k], acc);
      ot[lane * (kZT + 1) + 8 * w + t] = acc;
    }
    __syncthreads();
    float* xf = x + (long long)f * nvox;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int cl = w + 8 * m;
      if (c0 + cl >= r.nxp) continue;
      for (int j = lane; j < nout; j += 32) {
        float* p = xf + perm_index<NQ>(r, z0 + j, iy, c0 + cl);
        float val = ot[cl * (kZT + 1) + j];
        if (accumulate) val += *p;
        *p = fits ? val : __int_as_float(0x7fc00000);
      }
    }
  }
}

int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 148LL * 32); }

__global__ void add_inplace_kernel(float* __restrict__ x, const float* __restrict__ y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] += y[i];
}

template <int NW>
void launch_z_forward_nw(dim3 g, dim3 b, cudaStream_t st, const float* x, float* rz, const RotParam& r, int frames) {
  switch (r.nq) {
    case 1: shear_z_forward<NW, 1><<<g, b, 0, st>>>(x, rz, r, frames); break;
    case 2: shear_z_forward<NW, 2><<<g, b, 0, st>>>(x, rz, r, frames); break;
    case 3: shear_z_forward<NW, 3><<<g, b, 0, st>>>(x, rz, r, frames); break;
    default: shear_z_forward<NW, 0><<<g, b, 0, st>>>(x, rz, r, frames); break;
  }
}
void launch_z_forward(dim3 g, dim3 b, cudaStream_t st, const float* x, float* rz, const RotParam& r, int frames) {
  if (r.nwz == 8) launch_z_forward_nw<8>(g, b, st, x, rz, r, frames);
  else launch_z_forward_nw<16>(g, b, st, x, rz, r, frames);
}
template <int NW>
void launch_z_adjoint_nw(dim3 g, dim3 b, cudaStream_t st, const float* grz, float* x, const RotParam& r, int frames,
                         int acc) {
  switch (r.nq) {
    case 1: shear_z_adjoint<NW, 1><<<g, b, 0, st>>>(grz, x, r, frames, acc); break;
    case 2: shear_z_adjoint<NW, 2><<<g, b, 0, st>>>(grz, x, r, frames, acc); break;
    case 3: shear_z_adjoint<NW, 3><<<g, b, 0, st>>>(grz, x, r, frames, acc); break;
    default: shear_z_adjoint<NW, 0><<<g, b, 0, st>>>(grz, x, r, frames, acc); break;
  }
}
template <int NW>
void launch_z_adjoint_t_nw(cudaStream_t st, const float* grz, float* x, const RotParam& r, int frames, int acc) {
  const dim3 g((r.nzp + kZT - 1) / kZT, (r.nxp + 31) / 32, r.ny);   // tiles along the sheared axis adjacent
  const size_t sm = ((size_t)(kZT + NW - 1 + r.djz) * 32 + 32 * (kZT + 1)) * sizeof(float);
  if (r.nq == 1) shear_z_adjoint_t<NW, 1><<<g, 256, sm, st>>>(grz, x, r, frames, acc);
  else shear_z_adjoint_t<NW, 3><<<g, 256, sm, st>>>(grz, x, r, frames, acc);
}
void launch_z_adjoint(dim3 g, dim3 b, cudaStream_t st, const float* grz, float* x, const RotParam& r, int frames,
                      int acc) {
  if (r.nq % 2 == 1) {
    if (r.nwz == 8) launch_z_adjoint_t_nw<8>(st, grz, x, r, frames, acc);
    else launch_z_adjoint_t_nw<16>(st, grz, x, r, frames, acc);
  } else if (r.nwz == 8) launch_z_adjoint_nw<8>(g, b, st, grz, x, r, frames, acc);
  else launch_z_adjoint_nw<16>(g, b, st, grz, x, r, frames, acc);
}

// ---- general orientations -------------------------------------------------

__device__ double d_hat(double t) { return fmax(0.0, 1.0 - fabs(t)); }

// E[hat(c + U1 + U2)], U1, U2 uniform of widths al, be (>= 0): the density of
// U1 + U2 is a trapezoid on [-h, h] with plateau [-g, g]; the integrand is
// piecewise quadratic between the merged kinks, integrated by two-point
// Gauss-Legendre per piece (exact for cubics).
__device__ double hat_avg2_d(double c, double al, double be) {
  al = fabs(al);
  be = fabs(be);
  if (al < be) {
    const double t = al;
    al = be;
    be = t;
  }
  if (al == 0.0) return d_hat(c);
  const double h = 0.5 * (al + be), g = 0.5 * (al - be);
  double k[7] = {-h, -g, g, h, -c - 1.0, -c, -c + 1.0};
  for (int i = 1; i < 7; ++i)   // insertion sort
    for (int j = i; j > 0 && k[j - 1] > k[j]; --j) {
      const double t = k[j];
      k[j] = k[j - 1];
      k[j - 1] = t;
    }
  const double r3 = 0.5773502691896257645;   // 1 / sqrt(3)
  double total = 0.0;
  for (int i = 0; i < 6; ++i) {
    const double lo = fmax(k[i], -h), hi = fmin(k[i + 1], h);
    if (!(hi > lo)) continue;
    const double m = 0.5 * (lo + hi), rr = 0.5 * (hi - lo) * r3;
    double f = 0.0;
    for (int e = -1; e <= 1; e += 2) {
      const double sv = m + e * rr, a = fabs(sv);
      const double pdf = a >= h ? 0.0 : ((a <= g || be == 0.0) ? 1.0 / al : (h - a) / (al * be));
      f += d_hat(c + sv) * pdf;
    }
    total += 0.5 * (hi - lo) * f;
  }
  return total;
}

// Table of one pass: column (u, v) -> window offset J and nw entries.
__global__ void shear_pass_table_kernel(ShearPass ps, double s1, double s2, double du_dt, double dv_dt,
                                        float* __restrict__ tab, int32_t* __restrict__ jo) {
  const int n = ps.nu * ps.nv;
  const double al = fabs(s1) * du_dt, be = fabs(s2) * dv_dt;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int u = t % ps.nu, v = t / ps.nu;
    const double sh = s1 * du_dt * (u - 0.5 * (ps.nu - 1)) + s2 * dv_dt * (v - 0.5 * (ps.nv - 1));
    const int J = (int)floor(sh - 1.0 - 0.5 * (al + be)) - 1;
    jo[t] = J;
    for (int q = 0; q < ps.nw; ++q) tab[(long long)t * ps.nw + q] = (float)hat_avg2_d(-J - q + sh, al, be);
  }
}

__device__ __forceinline__ void pass_dims(const ShearPass& ps, int out, int& m0, int& m1, int& m2) {
  m0 = ps.n0 + (ps.axis == 0 && out ? 2 * ps.pad : 0);
  m1 = ps.n1 + (ps.axis == 1 && out ? 2 * ps.pad : 0);
  m2 = ps.n2 + (ps.axis == 2 && out ? 2 * ps.pad : 0);
}

// Forward pass (gather per output): out[..i..] = sum_q tab[col][q] in[..i - pad + J + q..].
__global__ void __launch_bounds__(256) shear_pass_forward(const float* __restrict__ in, float* __restrict__ out,
                                                          ShearPass ps, int frames) {
  int o0n, o1n, o2n;
  pass_dims(ps, 1, o0n, o1n, o2n);
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
  if (x >= o0n || y >= o1n || z >= o2n) return;
  const int c[3] = {x, y, z};
  const int i = c[ps.axis];
  const int u = ps.axis == 0 ? y : x;
  const int v = ps.axis == 2 ? y : z;
  const int col = v * ps.nu + u;
  const float* tb = ps.tab + (long long)col * ps.nw;
  const int jb = i - ps.pad + __ldg(ps.jo + col);
  const int n_ax = ps.axis == 0 ? ps.n0 : ps.axis == 1 ? ps.n1 : ps.n2;
  const long long stride = ps.axis == 0 ? 1 : ps.axis == 1 ? (long long)ps.n0 : (long long)ps.n0 * ps.n1;
  const long long base = ((long long)(ps.axis == 2 ? 0 : z) * ps.n1 + (ps.axis == 1 ? 0 : y)) * ps.n0 +
                         (ps.axis == 0 ? 0 : x);
  const long long in_fs = (long long)ps.n0 * ps.n1 * ps.n2, out_fs = (long long)o0n * o1n * o2n;
  const long long o = ((long long)z * o1n + y) * o0n + x;
  for (int f = 0; f < frames; ++f) {
    const float* src = in + f * in_fs + base;
    float acc = 0.0f;
    for (int q = 0; q < ps.nw; ++q) {
      const int j = jb + q;
      if (j >= 0 && j < n_ax) acc = fmaf(__ldg(tb + q), __ldg(src + j * stride), acc);
    }
    out[f * out_fs + o] = acc;
  }
}

// Transposed pass (gather per source): g_in[..j..] = sum_q tab[col][q] g_out[..j + pad - J - q..].
__global__ void __launch_bounds__(256) shear_pass_adjoint(const float* __restrict__ gout, float* __restrict__ gin,
                                                          ShearPass ps, int frames) {
  int o0n, o1n, o2n;
  pass_dims(ps, 1, o0n, o1n, o2n);
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
  if (x >= ps.n0 || y >= ps.n1 || z >= ps.n2) return;
  const int c[3] = {x, y, z};
  const int j = c[ps.axis];
  const int u = ps.axis == 0 ? y : x;
  const int v = ps.axis == 2 ? y : z;
  const int col = v * ps.nu + u;
  const float* tb = ps.tab + (long long)col * ps.nw;
  const int ib = j + ps.pad - __ldg(ps.jo + col);
  const int n_ax = ps.axis == 0 ? o0n : ps.axis == 1 ? o1n : o2n;
  const long long stride = ps.axis == 0 ? 1 : ps.axis == 1 ? (long long)o0n : (long long)o0n * o1n;
  const long long base = ((long long)(ps.axis == 2 ? 0 : z) * o1n + (ps.axis == 1 ? 0 : y)) * o0n +
                         (ps.axis == 0 ? 0 : x);
  const long long in_fs = (long long)ps.n0 * ps.n1 * ps.n2, out_fs = (long long)o0n * o1n * o2n;
  const long long o = ((long long)z * ps.n1 + y) * ps.n0 + x;
  for (int f = 0; f < frames; ++f) {
    const float* src = gout + f * out_fs + base;
    float acc = 0.0f;
    for (int q = ps.nw - 1; q >= 0; --q) {
      const int i = ib - q;
      if (i >= 0 && i < n_ax) acc = fmaf(__ldg(tb + q), __ldg(src + i * stride), acc);
    }
    gin[f * in_fs + o] = acc;
  }
}

// Passes along x, row-staged: warp = one (y, z) row, whose n0 inputs (or, for
// the transpose, n0 + 2 pad outputs) sit in the warp's shared-memory slice
// between WX zeros; the row's WX (>= nw, zero-padded) weights in registers.
// Taps in ascending (forward) or descending (transpose) q, as in
// shear_pass_forward / shear_pass_adjoint, whose values they give bit for bit.
template <int WX>
__global__ void __launch_bounds__(32 * kShearXWarps) shear_pass_row_forward(const float* __restrict__ in,
                                                                            float* __restrict__ out, ShearPass ps,
                                                                            int frames) {
  extern __shared__ float smem_rows[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long row = (long long)blockIdx.x * kShearXWarps + wid;   // z * n1 + y
  if (row >= (long long)ps.n1 * ps.n2) return;   // warp-uniform; no block barrier below
  const int n_out = ps.n0 + 2 * ps.pad;
  const int L = ps.n0 + 2 * WX;
  float* Rw = smem_rows + wid * L;
  if (lane < WX) {
    Rw[lane] = 0.0f;
    Rw[WX + ps.n0 + lane] = 0.0f;
  }
  const int col = (int)row;   // u = y, v = z: col = z * nu + y with nu = n1
  float w[WX];
#pragma unroll
  for (int q = 0; q < WX; ++q) w[q] = q < ps.nw ? __ldg(ps.tab + (long long)col * ps.nw + q) : 0.0f;
  const int off = __ldg(ps.jo + col) - ps.pad;   // output i's first source is i + off
  const long long in_fs = (long long)ps.n0 * ps.n1 * ps.n2, out_fs = (long long)n_out * ps.n1 * ps.n2;
  for (int f = 0; f < frames; ++f) {
    const float* src = in + f * in_fs + row * ps.n0;
    __syncwarp();
    for (int j = lane; j < ps.n0; j += 32) Rw[WX + j] = __ldg(src + j);
    __syncwarp();
    float* o = out + f * out_fs + row * n_out;
    for (int i = lane; i < n_out; i += 32) {
      const int jb = i + off;
      float acc = 0.0f;
      if (jb > -WX && jb < ps.n0) {   // else every tap lies outside the row
        const float* sp = Rw + WX + jb;
#pragma unroll
        for (int q = 0; q < WX; ++q) acc = fmaf(w[q], sp[q], acc);
      }
      o[i] = acc;
    }
  }
}

template <int WX>
__global__ void __launch_bounds__(32 * kShearXWarps) shear_pass_row_adjoint(const float* __restrict__ gout,
                                                                            float* __restrict__ gin, ShearPass ps,
                                                                            int frames) {
  extern __shared__ float smem_rows[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long row = (long long)blockIdx.x * kShearXWarps + wid;
  if (row >= (long long)ps.n1 * ps.n2) return;
  const int n_out = ps.n0 + 2 * ps.pad;
  const int L = n_out + 2 * WX;
  float* Gw = smem_rows + wid * L;
  if (lane < WX) {
    Gw[lane] = 0.0f;
    Gw[WX + n_out + lane] = 0.0f;
  }
  const int col = (int)row;
  float w[WX];
#pragma unroll
  for (int q = 0; q < WX; ++q) w[q] = q < ps.nw ? __ldg(ps.tab + (long long)col * ps.nw + q) : 0.0f;
  const int off = ps.pad - __ldg(ps.jo + col);   // source j's last tap is output j + off
  const long long in_fs = (long long)ps.n0 * ps.n1 * ps.n2, out_fs = (long long)n_out * ps.n1 * ps.n2;
  for (int f = 0; f < frames; ++f) {
    const float* g = gout + f * out_fs + row * n_out;
    __syncwarp();
    for (int i = lane; i < n_out; i += 32) Gw[WX + i] = __ldg(g + i);
    __syncwarp();
    float* o = gin + f * in_fs + row * ps.n0;
    for (int j = lane; j < ps.n0; j += 32) {
      const int ib = j + off;
      float acc = 0.0f;
      if (ib >= 0 && ib - (WX - 1) < n_out) {   // else every tap lies outside the row
        const float* sp = Gw + WX + ib;
#pragma unroll
        for (int q = WX - 1; q >= 0; --q) acc = fmaf(w[q], sp[-q], acc);
      }
      o[j] = acc;
    }
  }
}

// Passes along y (AX = 1) or z (AX = 2), column-walking: thread = column
// (x, other axis) and kShearZChunk outputs along the sheared axis, whose
// whole source window (kShearZChunk + NW - 1 values, NW >= nw with zero
// weights past nw) is loaded before any output is formed; each output's taps
// in ascending q, so every value equals shear_pass_forward's bit for bit.
// Outputs along these axes share most of their window, which the
// one-output-per-thread kernel read again for every output.
template <int NW, int AX>
__global__ void __launch_bounds__(256) shear_pass_col_forward(const float* __restrict__ in, float* __restrict__ out,
                                                              ShearPass ps, int frames) {
  static_assert(AX == 1 || AX == 2, "column passes run along y or z");
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int w2 = blockIdx.y * 8 + threadIdx.y;   // y (AX = 2) or z (AX = 1)
  const int i0 = blockIdx.z * kShearZChunk;      // first output along the axis
  if (x >= ps.n0 || w2 >= (AX == 2 ? ps.n1 : ps.n2)) return;
  const int n_ax = AX == 2 ? ps.n2 : ps.n1;
  const int n_out = n_ax + 2 * ps.pad;
  const int nout = min(kShearZChunk, n_out - i0);
  const int col = w2 * ps.nu + x;               // u = x, v = the other axis
  float w[NW];
#pragma unroll
  for (int q = 0; q < NW; ++q) w[q] = q < ps.nw ? __ldg(ps.tab + (long long)col * ps.nw + q) : 0.0f;
  const int jb = i0 - ps.pad + __ldg(ps.jo + col);   // first source of output i0
  const long long s_in = AX == 2 ? (long long)ps.n0 * ps.n1 : ps.n0;
  const long long b_in = AX == 2 ? (long long)w2 * ps.n0 + x : (long long)w2 * ps.n1 * ps.n0 + x;
  const long long s_out = s_in;
  const long long b_out = AX == 2 ? b_in : (long long)w2 * n_out * ps.n0 + x;
  const long long in_fs = (long long)ps.n0 * ps.n1 * ps.n2, out_fs = in_fs / n_ax * n_out;
  for (int f = 0; f < frames; ++f) {
    const float* src = in + f * in_fs + b_in + (long long)jb * s_in;   // source jb + q at src + q s_in
    float v[kShearZChunk + NW - 1];
    if (jb >= 0 && jb + kShearZChunk + NW - 1 <= n_ax) {
#pragma unroll
      for (int q = 0; q < kShearZChunk + NW - 1; ++q) v[q] = __ldg(src + q * s_in);
    } else {
#pragma unroll
      for (int q = 0; q < kShearZChunk + NW - 1; ++q)
        v[q] = (unsigned)(jb + q) < (unsigned)n_ax ? __ldg(src + q * s_in) : 0.0f;
    }
    float* o = out + f * out_fs + b_out;
#pragma unroll
    for (int t = 0; t < kShearZChunk; ++t) {
      if (t < nout) {
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < NW; ++q) acc = fmaf(w[q], v[t + q], acc);
        o[(long long)(i0 + t) * s_out] = acc;
      }
    }
  }
}

// Transposed column pass: thread = column and kShearZChunk sources along the
// axis, the window of outputs they gather from loaded first; taps in
// descending q as in shear_pass_adjoint, bit for bit.
template <int NW, int AX>
__global__ void __launch_bounds__(256) shear_pass_col_adjoint(const float* __restrict__ gout,
                                                              float* __restrict__ gin, ShearPass ps, int frames) {
  static_assert(AX == 1 || AX == 2, "column passes run along y or z");
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int w2 = blockIdx.y * 8 + threadIdx.y;
  const int j0 = blockIdx.z * kShearZChunk;      // first source along the axis
  if (x >= ps.n0 || w2 >= (AX == 2 ? ps.n1 : ps.n2)) return;
  const int n_ax = AX == 2 ? ps.n2 : ps.n1;
  const int n_out = n_ax + 2 * ps.pad;
  const int nsrc = min(kShearZChunk, n_ax - j0);
  const int col = w2 * ps.nu + x;
  float w[NW];   // w[k] weights the k-th value of the window (ascending output index)
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    const int q = NW - 1 - k;
    w[k] = q < ps.nw ? __ldg(ps.tab + (long long)col * ps.nw + q) : 0.0f;
  }
  const int ib = j0 + ps.pad - __ldg(ps.jo + col) - (NW - 1);   // first output of source j0's window
  const long long s_in = AX == 2 ? (long long)ps.n0 * ps.n1 : ps.n0;
  const long long b_in = AX == 2 ? (long long)w2 * ps.n0 + x : (long long)w2 * ps.n1 * ps.n0 + x;
  const long long b_out = AX == 2 ? b_in : (long long)w2 * n_out * ps.n0 + x;
  const long long in_fs = (long long)ps.n0 * ps.n1 * ps.n2, out_fs = in_fs / n_ax * n_out;
  for (int f = 0; f < frames; ++f) {
    const float* g = gout + f * out_fs + b_out + (long long)ib * s_in;   // output ib + k at g + k s_in
    float v[kShearZChunk + NW - 1];
    if (ib >= 0 && ib + kShearZChunk + NW - 1 <= n_out) {
#pragma unroll
      for (int k = 0; k < kShearZChunk + NW - 1; ++k) v[k] = __ldg(g + k * s_in);
    } else {
#pragma unroll
      for (int k = 0; k < kShearZChunk + NW - 1; ++k)
        v[k] = (unsigned)(ib + k) < (unsigned)n_out ? __ldg(g + k * s_in) : 0.0f;
    }
    float* o = gin + f * in_fs + b_in;
#pragma unroll
    for (int t = 0; t < kShearZChunk; ++t) {
      if (t < nsrc) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < NW; ++k) acc = fmaf(w[k], v[t + k], acc);
        o[(long long)(j0 + t) * s_in] = acc;
      }
    }
  }
}

// Signed permutation: permuted voxel p -> source voxel s, s_m = p[km[m]] or
// n_m - 1 - p[km[m]].  Forward gathers from x; the transpose gathers back.
__global__ void __launch_bounds__(256) grot_permute(const float* __restrict__ x, float* __restrict__ xp, GenRot g,
                                                    int frames) {
  const int p0 = blockIdx.x * 32 + threadIdx.x, p1 = blockIdx.y * 8 + threadIdx.y, p2 = blockIdx.z;
  if (p0 >= g.np[0] || p1 >= g.np[1] || p2 >= g.np[2]) return;
  const int p[3] = {p0, p1, p2};
  const int n[3] = {g.nx, g.ny, g.nz};
  int sidx[3];
  for (int m = 0; m < 3; ++m) sidx[m] = g.sg[m] > 0 ? p[g.km[m]] : n[m] - 1 - p[g.km[m]];
  const long long fs = (long long)g.nx * g.ny * g.nz;
  const long long src = ((long long)sidx[2] * g.ny + sidx[1]) * g.nx + sidx[0];
  const long long dst = ((long long)p2 * g.np[1] + p1) * g.np[0] + p0;
  for (int f = 0; f < frames; ++f) xp[f * fs + dst] = __ldg(x + f * fs + src);
}

__global__ void __launch_bounds__(256) grot_permute_adjoint(const float* __restrict__ xp, float* __restrict__ x,
                                                            GenRot g, int frames, int accumulate) {
  const int s0 = blockIdx.x * 32 + threadIdx.x, s1 = blockIdx.y * 8 + threadIdx.y, s2 = blockIdx.z;
  if (s0 >= g.nx || s1 >= g.ny || s2 >= g.nz) return;
  const int sv[3] = {s0, s1, s2};
  const int n[3] = {g.nx, g.ny, g.nz};
  int p[3];
  for (int m = 0; m < 3; ++m) p[g.km[m]] = g.sg[m] > 0 ? sv[m] : n[m] - 1 - sv[m];
  const long long fs = (long long)g.nx * g.ny * g.nz;
  const long long dst = ((long long)s2 * g.ny + s1) * g.nx + s0;
  const long long src = ((long long)p[2] * g.np[1] + p[1]) * g.np[0] + p[0];
  for (int f = 0; f < frames; ++f) {
    const float v = __ldg(xp + f * fs + src);
    x[f * fs + dst] = accumulate ? x[f * fs + dst] + v : v;
  }
}

inline dim3 grid3(int n0, int n1, int n2) { return dim3((n0 + 31) / 32, (n1 + 7) / 8, n2); }

}  // namespace

cudaError_t launch_add_inplace(float* x, const float* y, long long n, cudaStream_t st) {
  if (n > 0) add_inplace_kernel<<<grid_for(n), 256, 0, st>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t launch_shear_tables(const RotParam& r, cudaStream_t st) {
  const int n = r.nxp + r.nzr;
  shear_tables_kernel<<<(n + 127) / 128, 128, 0, st>>>(r);
  return cudaGetLastError();
}

cudaError_t launch_rotate_forward(const float* x, float* rz, float* xr, const RotParam& r, int frames,
                                  cudaStream_t st) {
  const dim3 blk(32, 8);
  const dim3 gz((r.nxp + 31) / 32, (r.ny + 7) / 8, (r.nzr + kShearZChunk - 1) / kShearZChunk);
  launch_z_forward(gz, blk, st, x, rz, r, frames);
  const int WX = r.wx <= 8 ? 8 : 16;
  const size_t sm = (size_t)kShearXWarps * (r.nxp + 2 * WX) * sizeof(float);
  const dim3 gx((r.ny + kShearXWarps - 1) / kShearXWarps, r.nzr);
  if (r.wx <= 16 && sm <= (size_t)kShearXSmemMax) {
    if (WX == 8) shear_x_forward_rows<8><<<gx, 32 * kShearXWarps, sm, st>>>(rz, xr, r, frames);
    else shear_x_forward_rows<16><<<gx, 32 * kShearXWarps, sm, st>>>(rz, xr, r, frames);
  } else shear_x_forward<<<dim3((r.nxr + 31) / 32, (r.ny + 7) / 8, r.nzr), blk, 0, st>>>(rz, xr, r, frames);
  return cudaGetLastError();
}

cudaError_t launch_rotate_adjoint(const float* g_xr, float* rz, float* x, const RotParam& r, int frames,
                                  int accumulate, cudaStream_t st) {
  const dim3 blk(32, 8);
  const int WX = r.wx <= 8 ? 8 : 16;
  const size_t sm = (size_t)kShearXWarps * (r.nxr + 2 * WX) * sizeof(float);
  const dim3 gx((r.ny + kShearXWarps - 1) / kShearXWarps, r.nzr);
  if (r.wx <= 16 && sm <= (size_t)kShearXSmemMax) {
    if (WX == 8) shear_x_adjoint_rows<8><<<gx, 32 * kShearXWarps, sm, st>>>(g_xr, rz, r, frames);
    else shear_x_adjoint_rows<16><<<gx, 32 * kShearXWarps, sm, st>>>(g_xr, rz, r, frames);
  } else shear_x_adjoint<<<dim3((r.nxp + 31) / 32, (r.ny + 7) / 8, r.nzr), blk, 0, st>>>(g_xr, rz, r, frames);
  const dim3 gz((r.nxp + 31) / 32, (r.ny + 7) / 8, (r.nzp + kShearZChunk - 1) / kShearZChunk);
  launch_z_adjoint(gz, blk, st, rz, x, r, frames, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_shear_pass_table(const ShearPass& ps, double s1, double s2, double du_dt, double dv_dt,
                                    float* tab, int32_t* jo, cudaStream_t st) {
  const int n = ps.nu * ps.nv;
  shear_pass_table_kernel<<<(n + 127) / 128, 128, 0, st>>>(ps, s1, s2, du_dt, dv_dt, tab, jo);
  return cudaGetLastError();
}

static void pass_out_dims(const ShearPass& ps, int& m0, int& m1, int& m2) {
  m0 = ps.n0 + (ps.axis == 0 ? 2 * ps.pad : 0);
  m1 = ps.n1 + (ps.axis == 1 ? 2 * ps.pad : 0);
  m2 = ps.n2 + (ps.axis == 2 ? 2 * ps.pad : 0);
}

cudaError_t launch_grot_forward(const float* x, float* b0, float* b1, float* b2, float* xr, const GenRot& g,
                                int frames, cudaStream_t st) {
  const dim3 blk(32, 8);
  int last = -1;
  for (int k = 0; k < 3; ++k)
    if (g.pass[k].active) last = k;
  float* scratch[3] = {b1, b2, nullptr};
  float* cur = last < 0 ? xr : b0;
  grot_permute<<<grid3(g.np[0], g.np[1], g.np[2]), blk, 0, st>>>(x, cur, g, frames);
  for (int k = 0; k < 3; ++k) {
    const ShearPass& ps = g.pass[k];
    if (!ps.active) continue;
    float* out = k == last ? xr : scratch[k];
    int m0, m1, m2;
    pass_out_dims(ps, m0, m1, m2);
    if (ps.axis != 0 && ps.nw <= 16) {
      const int n_oth = ps.axis == 2 ? ps.n1 : ps.n2;
      const int n_out = (ps.axis == 2 ? ps.n2 : ps.n1) + 2 * ps.pad;
      const dim3 g((ps.n0 + 31) / 32, (n_oth + 7) / 8, (n_out + kShearZChunk - 1) / kShearZChunk);
      if (ps.axis == 2) {
        if (ps.nw <= 8) shear_pass_col_forward<8, 2><<<g, blk, 0, st>>>(cur, out, ps, frames);
        else shear_pass_col_forward<16, 2><<<g, blk, 0, st>>>(cur, out, ps, frames);
      } else {
        if (ps.nw <= 8) shear_pass_col_forward<8, 1><<<g, blk, 0, st>>>(cur, out, ps, frames);
        else shear_pass_col_forward<16, 1><<<g, blk, 0, st>>>(cur, out, ps, frames);
      }
    } else if (ps.axis == 0 && ps.nw <= 16 &&
               (size_t)kShearXWarps * (ps.n0 + 32) * sizeof(float) <= (size_t)kShearXSmemMax) {
      const long long rows = (long long)ps.n1 * ps.n2;
      const dim3 g((unsigned)((rows + kShearXWarps - 1) / kShearXWarps));
      if (ps.nw <= 8)
        shear_pass_row_forward<8><<<g, 32 * kShearXWarps, kShearXWarps * (ps.n0 + 16) * sizeof(float), st>>>(
            cur, out, ps, frames);
      else
        shear_pass_row_forward<16><<<g, 32 * kShearXWarps, kShearXWarps * (ps.n0 + 32) * sizeof(float), st>>>(
            cur, out, ps, frames);
    } else {
      shear_pass_forward<<<grid3(m0, m1, m2), blk, 0, st>>>(cur, out, ps, frames);
    }
    cur = out;
  }
  return cudaGetLastError();
}

cudaError_t launch_grot_adjoint(const float* g_xr, float* b0, float* b1, float* b2, float* x, const GenRot& g,
                                int frames, int accumulate, cudaStream_t st) {
  const dim3 blk(32, 8);
  float* in_buf[3] = {b0, b1, b2};   // input of pass k (its transpose writes there)
  const float* cur = g_xr;
  for (int k = 2; k >= 0; --k) {
    const ShearPass& ps = g.pass[k];
    if (!ps.active) continue;
    if (ps.axis != 0 && ps.nw <= 16) {
      const int n_oth = ps.axis == 2 ? ps.n1 : ps.n2;
      const int n_ax = ps.axis == 2 ? ps.n2 : ps.n1;
      const dim3 g((ps.n0 + 31) / 32, (n_oth + 7) / 8, (n_ax + kShearZChunk - 1) / kShearZChunk);
      if (ps.axis == 2) {
        if (ps.nw <= 8) shear_pass_col_adjoint<8, 2><<<g, blk, 0, st>>>(cur, in_buf[k], ps, frames);
        else shear_pass_col_adjoint<16, 2><<<g, blk, 0, st>>>(cur, in_buf[k], ps, frames);
      } else {
        if (ps.nw <= 8) shear_pass_col_adjoint<8, 1><<<g, blk, 0, st>>>(cur, in_buf[k], ps, frames);
        else shear_pass_col_adjoint<16, 1><<<g, blk, 0, st>>>(cur, in_buf[k], ps, frames);
      }
    } else if (ps.axis == 0 && ps.nw <= 16 &&
               (size_t)kShearXWarps * (ps.n0 + 2 * ps.pad + 32) * sizeof(float) <= (size_t)kShearXSmemMax) {
      const long long rows = (long long)ps.n1 * ps.n2;
      const dim3 g((unsigned)((rows + kShearXWarps - 1) / kShearXWarps));
      const int n_out = ps.n0 + 2 * ps.pad;
      if (ps.nw <= 8)
        shear_pass_row_adjoint<8><<<g, 32 * kShearXWarps, kShearXWarps * (n_out + 16) * sizeof(float), st>>>(
            cur, in_buf[k], ps, frames);
      else
        shear_pass_row_adjoint<16><<<g, 32 * kShearXWarps, kShearXWarps * (n_out + 32) * sizeof(float), st>>>(
            cur, in_buf[k], ps, frames);
    } else {
      shear_pass_adjoint<<<grid3(ps.n0, ps.n1, ps.n2), blk, 0, st>>>(cur, in_buf[k], ps, frames);
    }
    cur = in_buf[k];
  }
  grot_permute_adjoint<<<grid3(g.nx, g.ny, g.nz), blk, 0, st>>>(cur, x, g, frames, accumulate);
  return cudaGetLastError();
}

}  // namespace lt
