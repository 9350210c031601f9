// Reconstruction of Sec. V (Table V): FISTA on the penalised weighted
// non-negative least-squares problem with camera gains (eq. pls), the
// 26-neighbour regulariser (eq. reg) and the diagonal majoriser of Appendix A.
//
// All solver state lives on the device: the gains and the FISTA scalars are
// computed by kernels, so one iteration is a fixed launch sequence that is
// captured once into a CUDA graph and replayed (no host round trip for the
// gain inner products, unlike the paper's implementation).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "lt.h"
#include "lt_host.h"

namespace lt {
namespace {

struct Scalars {
  double t;        // t^{(n)}
  double mom;      // (t^{(n)} - 1) / t^{(n+1)} for the update in flight
  long long iter;  // completed iterations
};

// Reductions use one block per SM (the plan's SM count, nb below) of
// RED_THREADS threads: 32 warps per SM, since they are latency-bound.
constexpr int RED_THREADS = 1024;

__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// part[(f*C + c)*nb + b] = sum over block b's share of camera c's pixels of
// w * a * b (w = 1 if NULL).  grid = (nb, F).
__global__ void __launch_bounds__(RED_THREADS)
dot_partials(const float* __restrict__ a, const float* __restrict__ b, const float* __restrict__ w,
             long long off, long long len, long long m_total, int C, int c, double* __restrict__ part,
             double scale) {
  __shared__ double sh[32];
  const long long base = (long long)blockIdx.y * m_total + off;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    const double wi = w ? (double)w[base + i] : 1.0;
    acc += wi * (double)a[base + i] * (double)b[base + i];
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[((long long)blockIdx.y * C + c) * gridDim.x + blockIdx.x] = scale * acc;
}

// Table V step 1b (gamma_c = y^T W p / y^T W y, c > 0) and the FISTA scalars
// t^{(n+1)} = (1 + sqrt(1 + 4 t^2)) / 2, mom = (t^{(n)} - 1) / t^{(n+1)}.
// FISTA step (Table V): t <- (1 + sqrt(1 + 4 t^2)) / 2 and the momentum
// weight (t_old - 1) / t_new of the coming update; one thread, once per
// iteration.
__device__ __forceinline__ void fista_advance(Scalars* sc) {
  const double t = sc->t;
  const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
  sc->mom = (t - 1.0) / tn;
  sc->t = tn;
  sc->iter += 1;
}

__global__ void finalize_gains(const double* __restrict__ part, const double* __restrict__ ywy,
                               double* __restrict__ gains, int F, int C, int estimate, int nb,
                               Scalars* __restrict__ sc) {
  for (int idx = threadIdx.x; idx < F * C; idx += blockDim.x) {
    const int c = idx % C;
    if (c == 0 || !estimate) {
      gains[idx] = 1.0;
      continue;
    }
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(long long)idx * nb + b];
    gains[idx] = ywy[idx] > 0.0 ? s / ywy[idx] : 0.0;
  }
  if (threadIdx.x == 0) fista_advance(sc);
}

// d = a p - gamma_c y over camera c's pixels, r = a W d (a = K_c / |S_c| of
// the view subset, 1 without subsets); fit partials of 1/2 sum W d^2.
// grid = (nb, F).
__global__ void __launch_bounds__(RED_THREADS)
residual_kernel(const float* __restrict__ y, const float* __restrict__ w, const float* __restrict__ p,
                float* __restrict__ r, const double* __restrict__ gains, long long off, long long len,
                long long m_total, int C, int c, double* __restrict__ fit_part, float alpha,
                Scalars* __restrict__ sc) {
  __shared__ double sh[32];
  if (sc && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) fista_advance(sc);
  const long long base = (long long)blockIdx.y * m_total + off;
  const float g = (float)gains[blockIdx.y * C + c];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    const float d = alpha * p[base + i] - g * y[base + i];
    const float wi = w ? w[base + i] : 1.0f;
    r[base + i] = (alpha * wi) * d;
    acc += (double)(wi * d * d);   // the term in float32 (FP64 units are scarce), the sum in float64
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) fit_part[((long long)blockIdx.y * C + c) * gridDim.x + blockIdx.x] = 0.5 * acc;
}

// Table V step 3: w = [z - (D + s beta)^-1 (g + grad R(z))]_+, x' = [w - nu]_+,
// z' = x' + mom (x' - x).  grad R(z)_j = beta sum_{l in N26(j)} psi'(z_j - z_l).
//
// A CTA owns a 32 x 8 (x, y) column of UPD_ZB slices.  With beta != 0 the z
// values slide through three shared-memory planes of (8 + 2) x (32 + 2)
// (one-voxel halo, zero outside the volume), so each z value is read from
// memory about 1.7 times instead of 27; neighbours outside the volume drop
// out of the sum through per-axis validity masks (no branches).  The walk is
// software-pipelined: while slice k is computed, the plane of slice k + 2
// and the voxel's D, g, x of slice k + 1 are already on their way into
// registers, so memory latency overlaps the 26-neighbour arithmetic.
constexpr int UPD_TX = 32, UPD_TY = 8, UPD_ZB = 8;
constexpr int UPD_PX = UPD_TX + 2, UPD_PY = UPD_TY + 2;
constexpr int UPD_PLANE = UPD_PX * UPD_PY;            // 340 values
constexpr int UPD_THREADS = UPD_TX * UPD_TY;          // 256: at most two plane values per thread
static_assert(UPD_PLANE <= 2 * UPD_THREADS, "plane slots per thread");

// Plane value i (0 <= i < UPD_PLANE) of slice kz: z at the halo position, 0 outside the volume.
__device__ __forceinline__ float plane_value(const float* __restrict__ zf, int i, int kz, int x0, int y0, int nx,
                                             int ny, int nz) {
  const int ly = i / UPD_PX, lx = i - ly * UPD_PX;
  const int gy = y0 + ly - 1, gx = x0 + lx - 1;
  if (i < UPD_PLANE && kz >= 0 && kz < nz && gy >= 0 && gy < ny && gx >= 0 && gx < nx)
    return __ldg(zf + ((long long)kz * ny + gy) * nx + gx);
  return 0.0f;
}

__global__ void __launch_bounds__(UPD_THREADS)
update_kernel(float* __restrict__ x, const float* __restrict__ z, float* __restrict__ zn,
              const float* __restrict__ g, const float* __restrict__ D, int nx, int ny, int nz,
              long long nvox, float beta, float nu, int psi, float inv_delta, float sbeta,
              const Scalars* __restrict__ sc) {
  __shared__ float pl[3][UPD_PLANE];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * UPD_TX + tx;
  const int nzb = (nz + UPD_ZB - 1) / UPD_ZB;
  const int f = blockIdx.z / nzb;
  const int z0 = (blockIdx.z - f * nzb) * UPD_ZB;
  const int x0 = blockIdx.x * UPD_TX, y0 = blockIdx.y * UPD_TY;
  const int ix = x0 + tx, iy = y0 + ty;
  const bool inside = ix < nx && iy < ny;
  const float* zf = z + (long long)f * nvox;
  const bool reg_on = beta != 0.0f;   // uniform
  const bool vy[3] = {iy > 0, true, iy + 1 < ny};
  const bool vx[3] = {ix > 0, true, ix + 1 < nx};
  const float mom = (float)sc->mom;
  const int kend = min(UPD_ZB, nz - z0);   // slices of this CTA (>= 1)
  const int i0 = tid, i1 = tid + UPD_THREADS;
  // voxel (ix, iy, z0 + k): index, and its D, g, x loaded one slice ahead
  const auto vidx = [&](int k) { return (long long)f * nvox + ((long long)(z0 + k) * ny + iy) * nx + ix; };
  float dn = 0.0f, gn = 0.0f, xn_ = 0.0f, zcn = 0.0f;
  if (inside) {
    const long long jf = vidx(0);
    dn = __ldg(D + jf);
    gn = __ldg(g + jf);
    xn_ = x[jf];
    if (!reg_on) zcn = __ldg(z + jf);
  }
  float q0 = 0.0f, q1 = 0.0f;   // plane of slice z0 + k + 1, staged for the next store
  if (reg_on) {
    pl[0][i0] = plane_value(zf, i0, z0 - 1, x0, y0, nx, ny, nz);
    if (i1 < UPD_PLANE) pl[0][i1] = plane_value(zf, i1, z0 - 1, x0, y0, nx, ny, nz);
    pl[1][i0] = plane_value(zf, i0, z0, x0, y0, nx, ny, nz);
    if (i1 < UPD_PLANE) pl[1][i1] = plane_value(zf, i1, z0, x0, y0, nx, ny, nz);
    q0 = plane_value(zf, i0, z0 + 1, x0, y0, nx, ny, nz);
    q1 = plane_value(zf, i1, z0 + 1, x0, y0, nx, ny, nz);
  }
  for (int k = 0; k < kend; ++k) {
    const int iz = z0 + k;
    const float dv = dn, gv = gn, xv = xn_, zv = zcn;
    if (reg_on) {
      pl[(k + 2) % 3][i0] = q0;   // plane iz + 1
      if (i1 < UPD_PLANE) pl[(k + 2) % 3][i1] = q1;
      q0 = plane_value(zf, i0, iz + 2, x0, y0, nx, ny, nz);
      q1 = plane_value(zf, i1, iz + 2, x0, y0, nx, ny, nz);
    }
    if (inside && k + 1 < kend) {   // next slice's operands
      const long long jn = vidx(k + 1);
      dn = __ldg(D + jn);
      gn = __ldg(g + jn);
      xn_ = x[jn];
      if (!reg_on) zcn = __ldg(z + jn);
    }
    if (reg_on) __syncthreads();
    if (inside) {
      const long long jf = vidx(k);
      const float* p3[3] = {pl[k % 3], pl[(k + 1) % 3], pl[(k + 2) % 3]};
      const float zc = reg_on ? p3[1][(ty + 1) * UPD_PX + tx + 1] : zv;
      float reg = 0.0f;
      if (reg_on) {
        const bool vz[3] = {iz > 0, true, iz + 1 < nz};
#pragma unroll
        for (int dz = 0; dz < 3; ++dz)
#pragma unroll
          for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
              if (dz == 1 && dy == 1 && dx == 1) continue;
              const float d = zc - p3[dz][(ty + dy) * UPD_PX + tx + dx];
              const float c = psi ? d * rsqrtf(1.0f + (d * inv_delta) * (d * inv_delta)) : d;
              reg += (vz[dz] && vy[dy] && vx[dx]) ? c : 0.0f;
            }
        reg *= beta;
      }
      const float den = dv + sbeta;
      const float wv = den > 0.0f ? fmaxf(zc - (gv + reg) / den, 0.0f) : 0.0f;
      const float xn = fmaxf(wv - nu, 0.0f);
      zn[jf] = xn + mom * (xn - xv);
      x[jf] = xn;
    }
    if (reg_on) __syncthreads();   // plane k % 3 is overwritten next
  }
}

// The same update for grids whose rows are a multiple of 4 voxels (every
// row 16-byte aligned): a thread owns four consecutive x voxels, so D, g,
// x (and z without the penalty) come and go as 16-byte loads and stores and
// a CTA keeps four times the bytes in flight (the scalar kernel above ran at
// about a third of the HBM rate on 256^3 x 16 frames, latency-bound).  A CTA
// owns a 128 x 8 (x, y) column of zb slices (8, fewer where that leaves
// under four CTAs per SM); the z planes hold 10 rows of
// 128 voxels at offset 4 plus the x halo at 3 and 132, each row one 16-byte
// shared load per thread, the neighbours at x - 1 and x + 4 from the
// adjacent lanes (shuffles) or the halo.  Per voxel the penalty terms are
// formed and summed in the same order as in update_kernel.
constexpr int U4_TX = 32, U4_X = 4 * U4_TX, U4_TY = 8, U4_ZB = 8;   // U4_ZB: the deepest slice chunk
constexpr int U4_PS = U4_X + 8;                       // plane row stride (floats)
constexpr int U4_PR = U4_TY + 2;                      // plane rows
constexpr int U4_PLANE = U4_PR * U4_PS;
constexpr int U4_V4 = U4_PR * U4_TX;                  // 320 interior float4 per plane
constexpr int U4_THREADS = U4_TX * U4_TY;             // 256
static_assert(U4_V4 <= 2 * U4_THREADS && 2 * U4_PR <= U4_THREADS, "plane slots per thread");

struct Plane4 {
  float4 a, b;   // interior float4 slots tid and tid + 256
  float h;       // halo slot tid (tid < 2 * U4_PR)
};

__device__ __forceinline__ void plane4_load(Plane4& q, const float* __restrict__ zf, int tid, int kz, int x0, int y0,
                                            int nx, int ny, int nz) {
  const bool zin = kz >= 0 && kz < nz;
  auto v4 = [&](int i4) {
    const int row = i4 / U4_TX, c4 = i4 - row * U4_TX;
    const int gy = y0 + row - 1, gx = x0 + 4 * c4;
    if (i4 < U4_V4 && zin && gy >= 0 && gy < ny && gx < nx)
      return __ldg(reinterpret_cast<const float4*>(zf + ((long long)kz * ny + gy) * nx + gx));
    return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  };
  q.a = v4(tid);
  q.b = v4(tid + U4_THREADS);
  q.h = 0.0f;
  if (tid < 2 * U4_PR) {
    const int row = tid >> 1, gy = y0 + row - 1, gx = (tid & 1) ? x0 + U4_X : x0 - 1;
    if (zin && gy >= 0 && gy < ny && gx >= 0 && gx < nx) q.h = __ldg(zf + ((long long)kz * ny + gy) * nx + gx);
  }
}

__device__ __forceinline__ void plane4_store(float* __restrict__ pl, const Plane4& q, int tid) {
  auto put = [&](int i4, const float4& v) {
    if (i4 < U4_V4) {
      const int row = i4 / U4_TX, c4 = i4 - row * U4_TX;
      *reinterpret_cast<float4*>(pl + row * U4_PS + 4 + 4 * c4) = v;
    }
  };
  put(tid, q.a);
  put(tid + U4_THREADS, q.b);
  if (tid < 2 * U4_PR) pl[(tid >> 1) * U4_PS + ((tid & 1) ? 4 + U4_X : 3)] = q.h;
}

__global__ void __launch_bounds__(U4_THREADS)
update_kernel4(float* __restrict__ x, const float* __restrict__ z, float* __restrict__ zn,
               const float* __restrict__ g, const float* __restrict__ D, int nx, int ny, int nz, int zb,
               long long nvox, float beta, float nu, int psi, float inv_delta, float sbeta,
               const Scalars* __restrict__ sc) {
  __shared__ __align__(16) float pl[3][U4_PLANE];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * U4_TX + tx;
  const int nzb = (nz + zb - 1) / zb;
  const int f = blockIdx.z / nzb;
  const int z0 = (blockIdx.z - f * nzb) * zb;
  const int x0 = blockIdx.x * U4_X, y0 = blockIdx.y * U4_TY;
  const int ix0 = x0 + 4 * tx, iy = y0 + ty;
  const bool inside = ix0 < nx && iy < ny;   // rows are a multiple of 4: all four voxels or none
  const float* zf = z + (long long)f * nvox;
  const bool reg_on = beta != 0.0f;   // uniform
  const bool vy[3] = {iy > 0, true, iy + 1 < ny};
  const float mom = (float)sc->mom;
  const int kend = min(zb, nz - z0);
  const auto vidx = [&](int k) { return (long long)f * nvox + ((long long)(z0 + k) * ny + iy) * nx + ix0; };
  float4 dn = make_float4(0.f, 0.f, 0.f, 0.f), gn = dn, xn_ = dn, zcn = dn;
  if (inside) {
    const long long jf = vidx(0);
    dn = __ldg(reinterpret_cast<const float4*>(D + jf));
    gn = __ldg(reinterpret_cast<const float4*>(g + jf));
    xn_ = *reinterpret_cast<const float4*>(x + jf);
    if (!reg_on) zcn = __ldg(reinterpret_cast<const float4*>(z + jf));
  }
  Plane4 q;
  if (reg_on) {
    Plane4 p0, p1;
    plane4_load(p0, zf, tid, z0 - 1, x0, y0, nx, ny, nz);
    plane4_load(p1, zf, tid, z0, x0, y0, nx, ny, nz);
    plane4_store(pl[0], p0, tid);
    plane4_store(pl[1], p1, tid);
    plane4_load(q, zf, tid, z0 + 1, x0, y0, nx, ny, nz);
  }
  for (int k = 0; k < kend; ++k) {
    const int iz = z0 + k;
    const float4 dv = dn, gv = gn, xv = xn_, zv = zcn;
    if (reg_on) {
      plane4_store(pl[(k + 2) % 3], q, tid);   // plane iz + 1
      plane4_load(q, zf, tid, iz + 2, x0, y0, nx, ny, nz);
    }
    if (inside && k + 1 < kend) {   // next slice's operands
      const long long jn = vidx(k + 1);
      dn = __ldg(reinterpret_cast<const float4*>(D + jn));
      gn = __ldg(reinterpret_cast<const float4*>(g + jn));
      xn_ = *reinterpret_cast<const float4*>(x + jn);
      if (!reg_on) zcn = __ldg(reinterpret_cast<const float4*>(z + jn));
    }
    if (reg_on) __syncthreads();
    // per (dz, dy) row the six z values x - 1 .. x + 4, one row at a time;
    // each voxel's terms are summed in (dz, dy, dx) order
    float reg[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float zc[4];
    if (reg_on) {
      const float* p3[3] = {pl[k % 3], pl[(k + 1) % 3], pl[(k + 2) % 3]};
      const bool vz[3] = {iz > 0, true, iz + 1 < nz};
      const float4 c11 = *reinterpret_cast<const float4*>(p3[1] + (ty + 1) * U4_PS + 4 + 4 * tx);
      zc[0] = c11.x;
      zc[1] = c11.y;
      zc[2] = c11.z;
      zc[3] = c11.w;
      bool vxl[4], vxr[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        vxl[j] = ix0 + j > 0;
        vxr[j] = ix0 + j + 1 < nx;
      }
#pragma unroll
      for (int dz = 0; dz < 3; ++dz)
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          const float* pr = p3[dz] + (ty + dy) * U4_PS;
          const float4 c = *reinterpret_cast<const float4*>(pr + 4 + 4 * tx);
          float lft = __shfl_up_sync(0xffffffffu, c.w, 1), rgt = __shfl_down_sync(0xffffffffu, c.x, 1);
          if (tx == 0) lft = pr[3];
          if (tx == U4_TX - 1) rgt = pr[4 + U4_X];
          const float r6[6] = {lft, c.x, c.y, c.z, c.w, rgt};
          const bool vzy = vz[dz] && vy[dy];
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
              if (dz == 1 && dy == 1 && dx == 1) continue;
              const float d = zc[j] - r6[j + dx];
              const float cc = psi ? d * rsqrtf(1.0f + (d * inv_delta) * (d * inv_delta)) : d;
              const bool vxx = dx == 0 ? vxl[j] : dx == 2 ? vxr[j] : true;
              reg[j] += (vzy && vxx) ? cc : 0.0f;
            }
        }
#pragma unroll
      for (int j = 0; j < 4; ++j) reg[j] *= beta;
    } else {
      zc[0] = zv.x;
      zc[1] = zv.y;
      zc[2] = zv.z;
      zc[3] = zv.w;
    }
    if (inside) {
      const float dvv[4] = {dv.x, dv.y, dv.z, dv.w}, gvv[4] = {gv.x, gv.y, gv.z, gv.w};
      const float xvv[4] = {xv.x, xv.y, xv.z, xv.w};
      float xo[4], zo[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float den = dvv[j] + sbeta;
        const float wv = den > 0.0f ? fmaxf(zc[j] - (gvv[j] + reg[j]) / den, 0.0f) : 0.0f;
        xo[j] = fmaxf(wv - nu, 0.0f);
        zo[j] = xo[j] + mom * (xo[j] - xvv[j]);
      }
      const long long jf = vidx(k);
      *reinterpret_cast<float4*>(zn + jf) = make_float4(zo[0], zo[1], zo[2], zo[3]);
      *reinterpret_cast<float4*>(x + jf) = make_float4(xo[0], xo[1], xo[2], xo[3]);
    }
    if (reg_on) __syncthreads();   // plane k % 3 is overwritten next
  }
}

// res[f] = sum over cameras and blocks of the fit partials of frame f,
// res[F + f * C + c] = gains[f * C + c].  grid = F, one block per frame.
__global__ void __launch_bounds__(256)
finalize_result(const double* __restrict__ fit_part, const double* __restrict__ gains, double* __restrict__ res,
                int F, int C, int nb) {
  __shared__ double sh[32];
  const int f = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < C * nb; i += blockDim.x) acc += fit_part[(long long)f * C * nb + i];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) res[f] = acc;
  for (int c = threadIdx.x; c < C; c += blockDim.x) res[F + f * C + c] = gains[f * C + c];
}

__global__ void finalize_dots(const double* __restrict__ part, double* __restrict__ out, int n, int nb) {
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) acc += part[(long long)idx * nb + b];
    out[idx] = acc;
  }
}

__global__ void fill_kernel(float* a, long long n, float v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a[i] = v;
}

__global__ void mul_kernel(float* out, const float* a, const float* b, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = b ? a[i] * b[i] : a[i];
}

// Device-to-device copy done by the SMs.  A copy-engine transfer on the
// solver's stream would queue behind host transfers that a streaming caller
// keeps in flight on its own copy streams: in such a loop the engine copies
// of the measurements, the volume and the result cost the solver's stream
// about 0.1 ms per step.
__global__ void copy_kernel(float* __restrict__ dst, const float* __restrict__ src, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long head = 0;
  if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0) {
    head = n & ~3LL;
    for (long long i = i0; i < (head >> 2); i += stride)
      reinterpret_cast<float4*>(dst)[i] = reinterpret_cast<const float4*>(src)[i];
  }
  for (long long i = head + i0; i < n; i += stride) dst[i] = src[i];
}

}  // namespace
}  // namespace lt

using namespace lt;

struct lt_recon {
  lt_plan* plan = nullptr;
  lt_recon_params prm{};
  int F = 0, C = 0;
  int nb = 1;                                      // reduction blocks: one per SM
  int64_t N = 0, M = 0;
  float *y = nullptr, *w = nullptr, *p = nullptr, *r = nullptr, *g = nullptr, *D = nullptr, *x = nullptr;
  float* z[2] = {nullptr, nullptr};
  double *ywy = nullptr, *gains = nullptr, *part = nullptr, *fit_part = nullptr;
  double* res = nullptr;                           // [F] data fit, [F][C] gains (lt_recon_get_async)
  Scalars* sc = nullptr;
  int zsel = 0;
  int64_t iters = 0;
  bool captured = false;
  int kernels_per_iter = 0;
  int n_sub = 1;                                   // view subsets (graphs per subset)
  std::vector<cudaGraphExec_t> exec;               // [2 * n_sub]: (z parity, subset)
  cudaStream_t cap = nullptr;
};

static void recon_free(lt_recon* R) {
  if (!R) return;
  for (cudaGraphExec_t g : R->exec)
    if (g) cudaGraphExecDestroy(g);
  if (R->cap) cudaStreamDestroy(R->cap);
  void* bufs[] = {R->y, R->w, R->p, R->r, R->g, R->D, R->x, R->z[0], R->z[1],
                  R->ywy, R->gains, R->part, R->fit_part, R->res, R->sc};
  for (void* b : bufs) cudaFree(b);
  delete R;
}

template <typename T>
static lt_status dalloc(T** p, size_t n, const char* what) {
  cudaError_t e = device_alloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return set_error(LT_ENOMEM, "cudaMalloc(%s, %zu bytes): %s", what, n * sizeof(T), cudaGetErrorString(e));
  }
  return LT_OK;
}

static int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 148LL * 16); }

// K_c / |S_c| of camera c for view subset `sub` (0 when the subset is empty).
static double subset_scale(const lt_recon* R, int c, int sub) {
  if (R->n_sub <= 1) return 1.0;
  const int K = R->plan->cams[c].K;
  int n = 0;
  for (int k = 0; k < K; ++k) n += k % R->n_sub == sub;
  return n > 0 ? (double)K / n : 0.0;
}

// One iteration of Table V from z[sel] to z[1-sel], using view subset `sub`.
static lt_status recon_step(lt_recon* R, int sel, int sub, cudaStream_t st) {
  lt_plan* P = R->plan;
  const float* z = R->z[sel];
  const SubsetSel ss{R->n_sub, sub};
  lt_status s = plan_forward(P, z, R->p, st, ss);  // step 1a: p_c = A_c z for every camera
  if (s != LT_OK) return s;
  const int est = R->prm.estimate_gains && R->C > 1;
  if (est)  // step 1b inner products (of the scaled subset projection)
    for (int c = 1; c < R->C; ++c)
      dot_partials<<<dim3(R->nb, R->F), RED_THREADS, 0, st>>>(
          R->y, R->p, R->w, P->cams[c].offset, P->cams[c].M, R->M, R->C, c, R->part, subset_scale(R, c, sub));
  // without estimation the gains keep their initial values (1), and the
  // FISTA scalars advance in the first residual block instead
  if (est) finalize_gains<<<1, 256, 0, st>>>(R->part, R->ywy, R->gains, R->F, R->C, est, R->nb, R->sc);
  for (int c = 0; c < R->C; ++c)  // a W (a p - gamma y)
    residual_kernel<<<dim3(R->nb, R->F), RED_THREADS, 0, st>>>(
        R->y, R->w, R->p, R->r, R->gains, P->cams[c].offset, P->cams[c].M, R->M, R->C, c, R->fit_part,
        (float)subset_scale(R, c, sub), !est && c == 0 ? R->sc : nullptr);
  s = plan_adjoint(P, R->r, R->g, st, ss);  // step 1c + 2: g = sum_c A_c^T r_c
  if (s != LT_OK) return s;
  const lt_volume_desc& v = P->vol;
  dim3 grid((v.nx + UPD_TX - 1) / UPD_TX, (v.ny + UPD_TY - 1) / UPD_TY,
            ((v.nz + UPD_ZB - 1) / UPD_ZB) * R->F);
  const float beta = (float)R->prm.beta;
  const float inv_delta = R->prm.psi == 1 ? (float)(1.0 / R->prm.psi_delta) : 1.0f;
  const float sbeta = (float)(R->prm.reg_scale * R->prm.beta);
  if (v.nx % 4 == 0) {   // rows of 16-byte multiples (the state buffers are cudaMalloc'ed, 256-byte aligned)
    const long long cols = (long long)((v.nx + U4_X - 1) / U4_X) * ((v.ny + U4_TY - 1) / U4_TY) * R->F;
    // deep columns (fewer halo planes per slice) unless that leaves SMs
    // without a CTA: at 128^3, 8 slices per CTA (256 CTAs) beat 2 (1024 CTAs)
    int zb = U4_ZB;
    while (zb > 1 && cols * ((v.nz + zb - 1) / zb) < (long long)P->sms) zb /= 2;
    const dim3 g4((v.nx + U4_X - 1) / U4_X, (v.ny + U4_TY - 1) / U4_TY, ((v.nz + zb - 1) / zb) * R->F);
    update_kernel4<<<g4, dim3(U4_TX, U4_TY), 0, st>>>(R->x, z, R->z[1 - sel], R->g, R->D, v.nx, v.ny, v.nz, zb,
                                                      R->N, beta, (float)R->prm.nu, R->prm.psi, inv_delta, sbeta,
                                                      R->sc);
  } else {
    update_kernel<<<grid, dim3(UPD_TX, UPD_TY), 0, st>>>(R->x, z, R->z[1 - sel], R->g, R->D, v.nx, v.ny, v.nz,
                                                         R->N, beta, (float)R->prm.nu, R->prm.psi, inv_delta, sbeta,
                                                         R->sc);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LT_OK : cuda_error(e, "reconstruction iteration");
}

// Copies y (and w), recomputes y^T W y per (frame, camera) on the device and,
// if the weights changed, the majoriser D = diag(sum_c A_c^T W_c A_c 1).
static lt_status load_data(lt_recon* R, const float* y, const float* w, bool new_weights, cudaStream_t st) {
  lt_plan* P = R->plan;
  const size_t FN = (size_t)R->F * R->N, FM = (size_t)R->F * R->M;
  copy_kernel<<<grid_for(FM / 4 + 1), 256, 0, st>>>(R->y, y, (long long)FM);
  if (w && R->w) copy_kernel<<<grid_for(FM / 4 + 1), 256, 0, st>>>(R->w, w, (long long)FM);
  lt_status s = LT_OK;
  if (new_weights) {
    fill_kernel<<<grid_for(FN), 256, 0, st>>>(R->g, (long long)FN, 1.0f);
    s = plan_forward(P, R->g, R->p, st);
    if (s != LT_OK) return s;
    mul_kernel<<<grid_for(FM), 256, 0, st>>>(R->r, R->p, R->w, (long long)FM);
    s = plan_adjoint(P, R->r, R->D, st);
    if (s != LT_OK) return s;
  }
  if (R->prm.estimate_gains && R->C > 1) {   // y^T W y of each camera: the gains' denominators (Table V, step 1b)
    for (int c = 0; c < R->C; ++c)
      dot_partials<<<dim3(R->nb, R->F), RED_THREADS, 0, st>>>(R->y, R->y, R->w, P->cams[c].offset,
                                                                   P->cams[c].M, R->M, R->C, c, R->part, 1.0);
    finalize_dots<<<1, 256, 0, st>>>(R->part, R->ywy, R->F * R->C, R->nb);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LT_OK : cuda_error(e, "loading measurements");
}

extern "C" lt_status lt_recon_create(lt_plan* plan, const float* y, const float* w,
                                     const lt_recon_params* params, const float* x0, void* stream,
                                     lt_recon** out) {
  clear_error();
  if (!out) return set_error(LT_EINVAL, "out is NULL");
  *out = nullptr;
  if (!plan || !y || !params) return set_error(LT_EINVAL, "plan, y and params are required");
  const lt_recon_params& q = *params;
  if (!(q.beta >= 0.0) || !(q.nu >= 0.0) || !std::isfinite(q.beta) || !std::isfinite(q.nu))
    return set_error(LT_EINVAL, "beta and nu must be finite and non-negative");
  if (q.psi != 0 && q.psi != 1) return set_error(LT_EINVAL, "psi must be 0 (quadratic) or 1 (hyperbola)");
  if (q.psi == 1 && !(q.psi_delta > 0.0)) return set_error(LT_EINVAL, "psi_delta must be positive");
  if (!(q.reg_scale >= 0.0)) return set_error(LT_EINVAL, "reg_scale must be non-negative");
  if (q.n_subset < 0 || q.n_subset > 64) return set_error(LT_EINVAL, "n_subset must be in [0, 64]");
  cudaStream_t st = (cudaStream_t)stream;
  lt_recon* R = new (std::nothrow) lt_recon();
  if (!R) return set_error(LT_ENOMEM, "host allocation failed");
  R->plan = plan;
  R->prm = q;
  R->n_sub = q.n_subset > 1 ? q.n_subset : 1;
  R->exec.assign(2 * (size_t)R->n_sub, nullptr);
  R->F = plan->frames;
  R->C = (int)plan->cams.size();
  R->nb = plan->sms > 0 ? plan->sms : 1;
  R->N = plan->nvox;
  R->M = plan->m_total;
  const size_t FN = (size_t)R->F * R->N, FM = (size_t)R->F * R->M;
  lt_status s;
  if ((s = dalloc(&R->y, FM, "y")) || (w && (s = dalloc(&R->w, FM, "w"))) || (s = dalloc(&R->p, FM, "p")) ||
      (s = dalloc(&R->r, FM, "r")) || (s = dalloc(&R->g, FN, "g")) || (s = dalloc(&R->D, FN, "D")) ||
      (s = dalloc(&R->x, FN, "x")) || (s = dalloc(&R->z[0], FN, "z")) || (s = dalloc(&R->z[1], FN, "z")) ||
      (s = dalloc(&R->ywy, (size_t)R->F * R->C, "ywy")) || (s = dalloc(&R->gains, (size_t)R->F * R->C, "gains")) ||
      (s = dalloc(&R->part, (size_t)R->F * R->C * R->nb, "partials")) ||
      (s = dalloc(&R->fit_part, (size_t)R->F * R->C * R->nb, "fit partials")) ||
      (s = dalloc(&R->res, (size_t)R->F * (R->C + 1), "results")) ||
      (s = dalloc(&R->sc, 1, "scalars"))) {
    recon_free(R);
    return s;
  }
  s = load_data(R, y, w, true, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (s != LT_OK || e != cudaSuccess) {
    recon_free(R);
    return s != LT_OK ? s : cuda_error(e, "reconstruction setup");
  }
  std::vector<double> g0((size_t)R->F * R->C, 0.0);
  for (int f = 0; f < R->F; ++f) g0[(size_t)f * R->C] = 1.0;   // gamma_1 = 1, gamma_c = 0
  if (!q.estimate_gains)
    for (auto& v : g0) v = 1.0;
  Scalars sc0{1.0, 0.0, 0};
  cudaMemcpy(R->gains, g0.data(), g0.size() * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(R->sc, &sc0, sizeof(sc0), cudaMemcpyHostToDevice);
  cudaMemset(R->fit_part, 0, (size_t)R->F * R->C * R->nb * sizeof(double));
  if (x0) {
    cudaMemcpy(R->x, x0, FN * sizeof(float), cudaMemcpyDeviceToDevice);
    cudaMemcpy(R->z[0], x0, FN * sizeof(float), cudaMemcpyDeviceToDevice);
  } else {
    cudaMemset(R->x, 0, FN * sizeof(float));
    cudaMemset(R->z[0], 0, FN * sizeof(float));
  }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    recon_free(R);
    return cuda_error(e, "reconstruction setup");
  }
  *out = R;
  return LT_OK;
}

static lt_status capture(lt_recon* R) {
  cudaError_t e = cudaStreamCreateWithFlags(&R->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_error(e, "capture stream");
  for (int gi = 0; gi < 2 * R->n_sub; ++gi) {
    const int sel = gi & 1, sub = gi >> 1;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(R->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_error(e, "begin capture");
    lt_status s = recon_step(R, sel, sub, R->cap);
    e = cudaStreamEndCapture(R->cap, &graph);
    if (s != LT_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (e != cudaSuccess) return cuda_error(e, "end capture");
    size_t n_nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &n_nodes);
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    cudaGraphGetNodes(graph, nodes.data(), &n_nodes);
    int nk = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
    }
    R->kernels_per_iter = nk;
    e = cudaGraphInstantiate(&R->exec[gi], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_error(e, "graph instantiate");
  }
  R->captured = true;
  return LT_OK;
}

extern "C" lt_status lt_recon_iterate(lt_recon* R, int32_t n_iter, void* stream) {
  clear_error();
  if (!R) return set_error(LT_EINVAL, "recon is NULL");
  if (n_iter < 0) return set_error(LT_EINVAL, "n_iter must be non-negative");
  if (!R->captured) {
    lt_status s = capture(R);
    if (s != LT_OK) return s;
  }
  cudaStream_t st = (cudaStream_t)stream;
  NvtxRange range("lt_recon_iterate");
  for (int i = 0; i < n_iter; ++i) {
    cudaError_t e = cudaGraphLaunch(R->exec[2 * (size_t)(R->iters % R->n_sub) + R->zsel], st);
    if (e != cudaSuccess) return cuda_error(e, "graph launch");
    R->zsel = 1 - R->zsel;
    R->iters++;
  }
  return LT_OK;
}

extern "C" lt_status lt_recon_get(lt_recon* R, float* x, double* gains, double* data_fit, void* stream) {
  clear_error();
  if (!R) return set_error(LT_EINVAL, "recon is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t FN = (size_t)R->F * R->N;
  if (x) copy_kernel<<<grid_for(FN / 4 + 1), 256, 0, st>>>(x, R->x, (long long)FN);
  if (gains || data_fit) {
    std::vector<double> g((size_t)R->F * R->C), fp((size_t)R->F * R->C * R->nb);
    cudaMemcpyAsync(g.data(), R->gains, g.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(fp.data(), R->fit_part, fp.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "lt_recon_get");
    if (gains) std::memcpy(gains, g.data(), g.size() * sizeof(double));
    if (data_fit)
      for (int f = 0; f < R->F; ++f) {
        double acc = 0.0;
        for (int c = 0; c < R->C; ++c)
          for (int b = 0; b < R->nb; ++b) acc += fp[((size_t)f * R->C + c) * R->nb + b];
        data_fit[f] = acc;
      }
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LT_OK : cuda_error(e, "lt_recon_get");
}

extern "C" lt_status lt_recon_get_async(lt_recon* R, double* host_out, void* stream) {
  clear_error();
  if (!R || !host_out) return set_error(LT_EINVAL, "recon and host_out are required");
  cudaStream_t st = (cudaStream_t)stream;
  // Page-locked host memory is mapped into the device's address space: the
  // reduction writes the few doubles there itself, and no copy-engine
  // transfer on this stream waits behind the caller's own host transfers.
  // Any other memory gets a copy.
  cudaPointerAttributes pa{};
  double* direct = nullptr;
  if (cudaPointerGetAttributes(&pa, host_out) == cudaSuccess) {
    if (pa.type == cudaMemoryTypeHost && pa.devicePointer) direct = static_cast<double*>(pa.devicePointer);
  } else {
    cudaGetLastError();   // an unregistered pointer is not an error here
  }
  finalize_result<<<R->F, 256, 0, st>>>(R->fit_part, R->gains, direct ? direct : R->res, R->F, R->C, R->nb);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && !direct)
    e = cudaMemcpyAsync(host_out, R->res, (size_t)R->F * (R->C + 1) * sizeof(double), cudaMemcpyDeviceToHost, st);
  return e == cudaSuccess ? LT_OK : cuda_error(e, "lt_recon_get_async");
}

extern "C" lt_status lt_recon_iterations(const lt_recon* R, int64_t* n_iter) {
  clear_error();
  if (!R || !n_iter) return set_error(LT_EINVAL, "NULL argument");
  *n_iter = R->iters;
  return LT_OK;
}

namespace {
struct StateHeader {
  uint64_t magic;
  int64_t F, N, C, iters;
};
constexpr uint64_t kStateMagic = 0x4c54524543535431ull;  // "LTRECST1"
}  // namespace

extern "C" lt_status lt_recon_state_size(const lt_recon* R, int64_t* bytes) {
  clear_error();
  if (!R || !bytes) return set_error(LT_EINVAL, "NULL argument");
  *bytes = (int64_t)(sizeof(StateHeader) + 2 * (size_t)R->F * R->N * sizeof(float) +
                     (size_t)R->F * R->C * sizeof(double) + sizeof(Scalars));
  return LT_OK;
}

extern "C" lt_status lt_recon_get_state(lt_recon* R, void* host_buf) {
  clear_error();
  if (!R || !host_buf) return set_error(LT_EINVAL, "NULL argument");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_error(e, "lt_recon_get_state");
  char* b = (char*)host_buf;
  StateHeader h{kStateMagic, R->F, R->N, R->C, R->iters};
  std::memcpy(b, &h, sizeof(h));
  b += sizeof(h);
  const size_t FN = (size_t)R->F * R->N * sizeof(float);
  cudaMemcpy(b, R->x, FN, cudaMemcpyDeviceToHost);
  b += FN;
  cudaMemcpy(b, R->z[R->zsel], FN, cudaMemcpyDeviceToHost);
  b += FN;
  cudaMemcpy(b, R->gains, (size_t)R->F * R->C * sizeof(double), cudaMemcpyDeviceToHost);
  b += (size_t)R->F * R->C * sizeof(double);
  e = cudaMemcpy(b, R->sc, sizeof(Scalars), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? LT_OK : cuda_error(e, "lt_recon_get_state");
}

extern "C" lt_status lt_recon_set_state(lt_recon* R, const void* host_buf) {
  clear_error();
  if (!R || !host_buf) return set_error(LT_EINVAL, "NULL argument");
  const char* b = (const char*)host_buf;
  StateHeader h;
  std::memcpy(&h, b, sizeof(h));
  if (h.magic != kStateMagic || h.F != R->F || h.N != R->N || h.C != R->C)
    return set_error(LT_EINVAL, "state buffer does not match this reconstruction");
  b += sizeof(h);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_error(e, "lt_recon_set_state");
  const size_t FN = (size_t)R->F * R->N * sizeof(float);
  cudaMemcpy(R->x, b, FN, cudaMemcpyHostToDevice);
  b += FN;
  cudaMemcpy(R->z[R->zsel], b, FN, cudaMemcpyHostToDevice);
  b += FN;
  cudaMemcpy(R->gains, b, (size_t)R->F * R->C * sizeof(double), cudaMemcpyHostToDevice);
  b += (size_t)R->F * R->C * sizeof(double);
  e = cudaMemcpy(R->sc, b, sizeof(Scalars), cudaMemcpyHostToDevice);
  R->iters = h.iters;
  return e == cudaSuccess ? LT_OK : cuda_error(e, "lt_recon_set_state");
}

extern "C" lt_status lt_recon_destroy(lt_recon* R) {
  if (!R) return LT_OK;
  cudaDeviceSynchronize();
  recon_free(R);
  return LT_OK;
}

extern "C" lt_status lt_recon_set_data(lt_recon* R, const float* y, const float* w, void* stream) {
  clear_error();
  if (!R || !y) return set_error(LT_EINVAL, "recon and y are required");
  if (w && !R->w) return set_error(LT_EINVAL, "this reconstruction was created without weights");
  return load_data(R, y, w, w != nullptr, (cudaStream_t)stream);
}

extern "C" lt_status lt_recon_kernels_per_iteration(lt_recon* R, int32_t* n) {
  clear_error();
  if (!R || !n) return set_error(LT_EINVAL, "NULL argument");
  if (!R->captured) {
    lt_status s = capture(R);
    if (s != LT_OK) return s;
  }
  *n = R->kernels_per_iter;
  return LT_OK;
}
