// Matrix entries of the separable slice -> plane transport (Sec. II-C,
// Table III), shared by every kernel that evaluates them so that the forward
// and adjoint kernels compute each entry with the same arithmetic.
#pragma once

#include "lt_internal.h"

namespace lt {

// ---------------------------------------------------------------------------
// Matrix entries.  All arithmetic uses explicit round-to-nearest intrinsics so
// that no floating-point contraction can differ between the forward and the
// adjoint instantiations.
// ---------------------------------------------------------------------------

// Footprint centre xi(i) = c0 + c1*i of target pixel i in source-index units,
// returned as an integer cell jc and a fraction fr in [0, 1).  The product and
// sum are compensated (exact product error by fma, TwoSum) so that the
// fraction is accurate to ~1e-7 even where xi is in the hundreds.
static __device__ __forceinline__ void footprint_centre(const AxisParam& a, int i, int& jc, float& fr) {
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
static __device__ __forceinline__ float trap_F(float x, float P, float Q, float hir) {
  const float a = fminf(fabsf(x), Q);
  const float d = fmaxf(__fsub_rn(a, P), 0.0f);
  const float g = __fsub_rn(a, __fmul_rn(__fmul_rn(d, d), hir));
  return copysignf(g, x);
}

// F at the lower edge of source cell m (relative to jc) for a footprint
// centred at fr: the edge m - 1/2 (equal to the upper edge of cell m - 1;
// both are exact in float for the small integers used here).
static __device__ __forceinline__ float edge_F(int m, float fr, const AxisParam& a) {
  return trap_F(__fsub_rn(__fsub_rn((float)m, 0.5f), fr), a.P, a.Q, a.hir);
}

// Integral of the unit trapezoid centred at fr over source cell m (relative
// to jc): [m - 1/2, m + 1/2].  Exactly 0 outside the footprint.
// Equal, bit for bit, to edge_F(m + 1) - edge_F(m).
static __device__ __forceinline__ float cell_weight(int m, float fr, const AxisParam& a) {
  const float fm = (float)m;
  const float xh = __fsub_rn(__fadd_rn(fm, 0.5f), fr);
  const float xl = __fsub_rn(__fsub_rn(fm, 0.5f), fr);
  return __fsub_rn(trap_F(xh, a.P, a.Q, a.hir), trap_F(xl, a.P, a.Q, a.hir));
}

// First target pixel whose footprint may overlap source cell j (a superset
// window of the exact range, widened by one pixel for rounding).
static __device__ __forceinline__ int window_start(const AxisParam& a, int j) {
  const float c0 = __fadd_rn(a.c0_hi, a.c0_lo);
  const float lo = __fmul_rn(__fsub_rn(__fsub_rn((float)j - 0.5f, a.Q), c0), a.inv_c1);
  const float hi = __fmul_rn(__fsub_rn(__fadd_rn((float)j + 0.5f, a.Q), c0), a.inv_c1);
  return (int)floorf(fminf(lo, hi)) - 1;
}

}  // namespace lt
