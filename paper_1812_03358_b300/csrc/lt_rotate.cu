// Rotated perspectives (Sec. III-A): quarter turns and the two shear passes
// of the residual yaw, with their exact transposes.  Every pass is a 1-D
// Toeplitz re-projection per column (eq. rot,toeplitz) streamed with one
// thread per output element (HBM bound); forward and adjoint evaluate the
// same entries with the same function, so they are exact transposes up to
// float32 summation order.
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

// Index in the original volume of permuted-grid voxel (jz, iy, jx).
__device__ __forceinline__ long long perm_index(const RotParam& r, int jz, int iy, int jx) {
  int iz, ix;
  switch (r.nq) {
    case 1: iz = r.nz - 1 - jx; ix = jz; break;
    case 2: iz = r.nz - 1 - jz; ix = r.nx - 1 - jx; break;
    case 3: iz = jx; ix = r.nx - 1 - jz; break;
    default: iz = jz; ix = jx; break;
  }
  return ((long long)iz * r.ny + iy) * r.nx + ix;
}

// rz[f][izr][iy][ixp] = sum_j E^z(izr, j; ixp) xp[f][j][iy][ixp]
__global__ void shear_z_forward(const float* __restrict__ x, float* __restrict__ rz, RotParam r, int frames) {
  const long long per = (long long)r.nzr * r.ny * r.nxp;
  const long long nvox = (long long)r.nx * r.ny * r.nz;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < per * frames;
       idx += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(idx / per);
    long long rem = idx - (long long)f * per;
    const int ixp = (int)(rem % r.nxp);
    rem /= r.nxp;
    const int iy = (int)(rem % r.ny);
    const int izr = (int)(rem / r.ny);
    const float sh = column_shift(r.bz, ixp, r.nxp);
    const int j0 = (int)floorf((float)(izr - r.pz) + sh - 1.0f - 0.5f * r.betaz) - 1;
    const float* xf = x + (long long)f * nvox;
    float acc = 0.0f;
    for (int q = 0; q < r.wz; ++q) {
      const int j = j0 + q;
      if (j < 0 || j >= r.nzp) continue;
      const float w = hat_avg(shear_u(izr, j, r.pz, sh), r.betaz);
      if (w != 0.0f) acc = fmaf(w, __ldg(xf + perm_index(r, j, iy, ixp)), acc);
    }
    rz[idx] = acc;
  }
}

// xr[f][izr][iy][ixr] = sum_j E^x(ixr, j; izr) rz[f][izr][iy][j]
__global__ void shear_x_forward(const float* __restrict__ rz, float* __restrict__ xr, RotParam r, int frames) {
  const long long per = (long long)r.nzr * r.ny * r.nxr;
  const long long per_in = (long long)r.nzr * r.ny * r.nxp;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < per * frames;
       idx += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(idx / per);
    long long rem = idx - (long long)f * per;
    const int ixr = (int)(rem % r.nxr);
    rem /= r.nxr;
    const int iy = (int)(rem % r.ny);
    const int izr = (int)(rem / r.ny);
    const float sh = column_shift(r.ax, izr, r.nzr);
    const int j0 = (int)floorf((float)(ixr - r.px) + sh - 1.0f - 0.5f * r.betax) - 1;
    const float* row = rz + (long long)f * per_in + ((long long)izr * r.ny + iy) * r.nxp;
    float acc = 0.0f;
    for (int q = 0; q < r.wx; ++q) {
      const int j = j0 + q;
      if (j < 0 || j >= r.nxp) continue;
      const float w = hat_avg(shear_u(ixr, j, r.px, sh), r.betax);
      if (w != 0.0f) acc = fmaf(w, __ldg(row + j), acc);
    }
    xr[idx] = acc;
  }
}

// grz[f][izr][iy][j] = sum_ixr E^x(ixr, j; izr) g[f][izr][iy][ixr]
__global__ void shear_x_adjoint(const float* __restrict__ g, float* __restrict__ grz, RotParam r, int frames) {
  const long long per = (long long)r.nzr * r.ny * r.nxp;
  const long long per_in = (long long)r.nzr * r.ny * r.nxr;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < per * frames;
       idx += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(idx / per);
    long long rem = idx - (long long)f * per;
    const int j = (int)(rem % r.nxp);
    rem /= r.nxp;
    const int iy = (int)(rem % r.ny);
    const int izr = (int)(rem / r.ny);
    const float sh = column_shift(r.ax, izr, r.nzr);
    // outputs i with |i - j - px + sh| < 1 + beta/2
    const int i0 = (int)floorf((float)(j + r.px) - sh - 1.0f - 0.5f * r.betax) - 1;
    const float* row = g + (long long)f * per_in + ((long long)izr * r.ny + iy) * r.nxr;
    float acc = 0.0f;
    for (int q = 0; q < r.wx; ++q) {
      const int i = i0 + q;
      if (i < 0 || i >= r.nxr) continue;
      const float w = hat_avg(shear_u(i, j, r.px, sh), r.betax);
      if (w != 0.0f) acc = fmaf(w, __ldg(row + i), acc);
    }
    grz[idx] = acc;
  }
}

// x[f][iz][iy][ix] (= or +=) sum_izr E^z(izr, jz; jx) grz[f][izr][iy][jx], (jz, jx) the permuted indices
__global__ void shear_z_adjoint(const float* __restrict__ grz, float* __restrict__ x, RotParam r, int frames,
                                int accumulate) {
  const long long nvox = (long long)r.nx * r.ny * r.nz;
  const long long per_in = (long long)r.nzr * r.ny * r.nxp;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nvox * frames;
       idx += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(idx / nvox);
    long long rem = idx - (long long)f * nvox;
    const int ix = (int)(rem % r.nx);
    rem /= r.nx;
    const int iy = (int)(rem % r.ny);
    const int iz = (int)(rem / r.ny);
    int jz, jx;   // inverse of perm_index
    switch (r.nq) {
      case 1: jx = r.nz - 1 - iz; jz = ix; break;
      case 2: jz = r.nz - 1 - iz; jx = r.nx - 1 - ix; break;
      case 3: jx = iz; jz = r.nx - 1 - ix; break;
      default: jz = iz; jx = ix; break;
    }
    const float sh = column_shift(r.bz, jx, r.nxp);
    const int i0 = (int)floorf((float)(jz + r.pz) - sh - 1.0f - 0.5f * r.betaz) - 1;
    const float* gf = grz + (long long)f * per_in;
    float acc = 0.0f;
    for (int q = 0; q < r.wz; ++q) {
      const int i = i0 + q;
      if (i < 0 || i >= r.nzr) continue;
      const float w = hat_avg(shear_u(i, jz, r.pz, sh), r.betaz);
      if (w != 0.0f) acc = fmaf(w, __ldg(gf + ((long long)i * r.ny + iy) * r.nxp + jx), acc);
    }
    x[idx] = accumulate ? x[idx] + acc : acc;
  }
}

int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 148LL * 32); }

}  // namespace

cudaError_t launch_rotate_forward(const float* x, float* rz, float* xr, const RotParam& r, int frames,
                                  cudaStream_t st) {
  const long long nrz = (long long)r.nzr * r.ny * r.nxp * frames;
  const long long nxr = (long long)r.nzr * r.ny * r.nxr * frames;
  shear_z_forward<<<grid_for(nrz), 256, 0, st>>>(x, rz, r, frames);
  shear_x_forward<<<grid_for(nxr), 256, 0, st>>>(rz, xr, r, frames);
  return cudaGetLastError();
}

cudaError_t launch_rotate_adjoint(const float* g_xr, float* rz, float* x, const RotParam& r, int frames,
                                  int accumulate, cudaStream_t st) {
  const long long nrz = (long long)r.nzr * r.ny * r.nxp * frames;
  const long long nvox = (long long)r.nx * r.ny * r.nz * frames;
  shear_x_adjoint<<<grid_for(nrz), 256, 0, st>>>(g_xr, rz, r, frames);
  shear_z_adjoint<<<grid_for(nvox), 256, 0, st>>>(rz, x, r, frames, accumulate);
  return cudaGetLastError();
}

}  // namespace lt
