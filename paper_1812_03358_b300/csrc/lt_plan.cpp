// Host side of the C ABI: descriptor validation, float64 transport planning
// (Sec. II-A/C, Tables II and III), device tables and the operator entry
// points of include/lt.h.
#include "lt.h"
#include "lt_internal.h"
#include "lt_host.h"
#include "lt_testing.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <climits>
#include <atomic>
#define _USE_MATH_DEFINES
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

using lt::AxisParam;
using lt::LensletParam;
using lt::SliceParam;

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace lt {

#ifdef LT_TEST_HOOKS
namespace {
std::atomic<int> g_fail_alloc_in{0};   // > 0: the allocation that brings it to 0 fails
}  // namespace
#endif

cudaError_t device_alloc(void** p, size_t bytes) {
#ifdef LT_TEST_HOOKS
  int n = g_fail_alloc_in.load();
  while (n > 0) {
    if (g_fail_alloc_in.compare_exchange_weak(n, n - 1)) {
      if (n == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
#endif
  return cudaMalloc(p, bytes);
}

NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

lt_status set_error(lt_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

lt_status cuda_error(cudaError_t e, const char* where) {
  return set_error(LT_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

void clear_error() { g_last_error.clear(); }

// Position row (X_ss, X_su, Xbar_s) of an affine ray map (Sec. II-A).
struct Row {
  double ss, su, b;
};

// Slice at object distance d -> image plane d_img behind a lens of focal
// length f: T_{d_img} o R_f o T_d (Table I).  Angular plane: T_d.
static void slice_rows(double d, double d_img, double f, Row* P, Row* L) {
  L->ss = 1.0;
  L->su = d;
  L->b = 0.0;
  P->ss = 1.0 - d_img / f;
  P->su = d + d_img - d * d_img / f;
  P->b = 0.0;
}

// Array plane -> detector through a lenslet (focal f, centre c) and a
// propagation D_mud: T_{D_mud} o R_{f,c}; angular plane: back by D_mum.
static void lenslet_rows(double d_mud, double d_mum, double f, double c, Row* P, Row* L) {
  L->ss = 1.0;
  L->su = -d_mum;
  L->b = 0.0;
  P->ss = 1.0 - d_mud / f;
  P->su = d_mud;
  P->b = d_mud * c / f;
}

static void split(double v, float* hi, float* lo) {
  *hi = (float)v;
  *lo = (float)(v - (double)*hi);
}

// Footprint of target pixel i (centre tgt_first + i*tgt_pitch, width
// tgt_pitch) through angular cell [cell_c +- cell_w/2] on the source grid
// (cell j centred at src_first + j*src_pitch).  The map (s,u) -> (lens
// crossing l, target position p) is affine with Jacobian J = Lss Psu - Lsu Pss;
// inverting it, s = sig_l l + sig_p p + sig_0, so the pixel-and-cell
// rectangle pushes forward to the convolution of boxes of widths
// |sig_l| cell_w and |sig_p| tgt_pitch (Table III's trapezoid) with height
// H = min(cell_w/|Lsu|, tgt_pitch/|Psu|) in the (s,u) measure.  For the Dirac
// basis the cell width collapses and H = cell_w/|Lsu| (Table II).
struct Footprint {
  AxisParam a;
  double H;       // kernel height
  double C0, C1;  // centre in source-index units
  double P, Q;
};

static bool footprint(const Row& L, const Row& P, double cell_c, double cell_w,
                      double tgt_first, double tgt_pitch, double src_first, double src_pitch,
                      int basis, Footprint* out) {
  const double J = L.ss * P.su - L.su * P.ss;
  if (!(std::fabs(J) > 0.0) || !(std::fabs(L.su) > 0.0)) return false;
  const double sig_l = P.su / J;
  const double sig_p = -L.su / J;
  const double sig_0 = (L.su * P.b - P.su * L.b) / J;
  const double C1 = sig_p * tgt_pitch / src_pitch;
  const double C0 = (sig_l * cell_c + sig_p * tgt_first + sig_0 - src_first) / src_pitch;
  const double w2 = std::fabs(sig_p) * tgt_pitch / src_pitch;
  double Pw, Qw, H;
  if (basis == LT_BASIS_DIRAC) {
    Pw = Qw = 0.5 * w2;
    H = cell_w / std::fabs(L.su);
  } else {
    const double w1 = std::fabs(sig_l) * cell_w / src_pitch;
    Pw = 0.5 * std::fabs(w1 - w2);
    Qw = 0.5 * (w1 + w2);
    H = cell_w / std::fabs(L.su);
    if (P.su != 0.0) H = std::min(H, tgt_pitch / std::fabs(P.su));
  }
  if (!std::isfinite(C0) || !std::isfinite(C1) || !std::isfinite(Qw) || C1 == 0.0) return false;
  split(C0, &out->a.c0_hi, &out->a.c0_lo);
  split(C1, &out->a.c1_hi, &out->a.c1_lo);
  out->a.P = (float)Pw;
  out->a.Q = (float)Qw;
  out->a.hir = (out->a.Q > out->a.P) ? (float)(0.5 / ((double)out->a.Q - (double)out->a.P)) : 0.0f;
  out->a.inv_c1 = (float)(1.0 / C1);
  out->H = H;
  out->C0 = C0;
  out->C1 = C1;
  out->P = Pw;
  out->Q = Qw;
  return true;
}

// Forward window: source cells a target pixel's footprint can touch.
static int fwd_window(float Q) { return (int)std::floor(2.0 * (double)Q) + 2; }
// Adjoint window: target pixels whose footprints can touch one source cell
// (with one pixel of margin on each side for rounding).
static int adj_window(float Q, double C1) {
  return (int)std::floor((2.0 * (double)Q + 1.0) / std::fabs(C1)) + 4;
}

static inline double centre(int i, int n, double pitch) { return (i - 0.5 * (n - 1)) * pitch; }

}  // namespace lt

using namespace lt;

// ---------------------------------------------------------------------------
// plan construction
// ---------------------------------------------------------------------------

static lt_status validate_volume(const lt_volume_desc* v) {
  if (!v) return set_error(LT_EINVAL, "volume descriptor is NULL");
  if (v->nx <= 0 || v->ny <= 0 || v->nz <= 0)
    return set_error(LT_EINVAL, "volume sizes must be positive (got %d %d %d)", v->nx, v->ny, v->nz);
  if (!(v->dx > 0) || !(v->dy > 0) || !(v->dz > 0) || !std::isfinite(v->dx) ||
      !std::isfinite(v->dy) || !std::isfinite(v->dz))
    return set_error(LT_EINVAL, "voxel sizes must be positive and finite");
  if ((long long)v->nx * v->ny * v->nz > (1LL << 34))
    return set_error(LT_EINVAL, "volume too large");
  return LT_OK;
}

static bool pos(double v) { return v > 0.0 && std::isfinite(v); }

static lt_status validate_camera(const lt_volume_desc* v, const lt_camera_desc* c, int idx) {
  if (c->kind != LT_CAM_SINGLE && c->kind != LT_CAM_PLENOPTIC)
    return set_error(LT_EINVAL, "camera %d: unknown kind %d", idx, c->kind);
  if (c->basis != LT_BASIS_PILLBOX && c->basis != LT_BASIS_DIRAC)
    return set_error(LT_EINVAL, "camera %d: unknown basis %d", idx, c->basis);
  if (!pos(c->f_main) || !pos(c->r_main) || !pos(c->d_obj))
    return set_error(LT_EINVAL, "camera %d: f_main, r_main, d_obj must be positive", idx);
  if (!std::isfinite(c->yaw) || !std::isfinite(c->pitch) || !std::isfinite(c->roll))
    return set_error(LT_EINVAL, "camera %d: yaw/pitch/roll not finite", idx);
  if (c->det_ns <= 0 || c->det_nt <= 0 || !pos(c->det_ps) || !pos(c->det_pt))
    return set_error(LT_EINVAL, "camera %d: detector sizes/pitches must be positive", idx);
  if (c->ks <= 0 || c->kt <= 0 || c->ks > 256 || c->kt > 256)
    return set_error(LT_EINVAL, "camera %d: angular cells ks, kt must be in [1, 256]", idx);
  // the rotated view's z extent is at most the volume's diagonal in (x, z)
  const double half = 0.5 * std::sqrt((double)v->nz * v->dz * v->nz * v->dz + (double)v->nx * v->dx * v->nx * v->dx +
                                      (c->pitch != 0.0 || c->roll != 0.0 ? (double)v->ny * v->dy * v->ny * v->dy : 0.0));
  const bool turned = c->yaw != 0.0 || c->pitch != 0.0 || c->roll != 0.0;
  const double dmin = c->d_obj - (turned ? 2.0 * half : 0.5 * v->nz * v->dz);
  if (!(dmin > 0.0))
    return set_error(LT_EINVAL, "camera %d: the volume reaches the main lens (nearest slice at %g)", idx, dmin);
  if (c->kind == LT_CAM_SINGLE) {
    if (!pos(c->d_lens_det)) return set_error(LT_EINVAL, "camera %d: d_lens_det must be positive", idx);
  } else {
    if (!pos(c->d_lens_mla) || !pos(c->d_mla_det))
      return set_error(LT_EINVAL, "camera %d: d_lens_mla, d_mla_det must be positive", idx);
    if (c->mla_ns <= 0 || c->mla_nt <= 0 || !pos(c->mla_pitch) || !pos(c->mla_radius))
      return set_error(LT_EINVAL, "camera %d: lenslet grid must be non-empty with positive pitch/radius", idx);
    if (c->mla_layout != LT_MLA_SQUARE && c->mla_layout != LT_MLA_HEX)
      return set_error(LT_EINVAL, "camera %d: unknown mla_layout %d", idx, c->mla_layout);
    if (c->mla_radius > 0.5 * c->mla_pitch * (1.0 + 1e-12))
      return set_error(LT_EINVAL, "camera %d: lenslet radius exceeds half the pitch (discs overlap)", idx);
    if (!c->mla_focal) return set_error(LT_EINVAL, "camera %d: mla_focal is NULL", idx);
    for (long long m = 0; m < (long long)c->mla_ns * c->mla_nt; ++m)
      if (!pos(c->mla_focal[m])) return set_error(LT_EINVAL, "camera %d: lenslet %lld focal length not positive", idx, m);
    if (c->arr_ns <= 0 || c->arr_nt <= 0 || !pos(c->arr_ps) || !pos(c->arr_pt))
      return set_error(LT_EINVAL, "camera %d: array-plane grid must be non-empty with positive pitch", idx);
  }
  return LT_OK;
}

template <typename T>
static lt_status upload(const std::vector<T>& h, T** d, const char* what) {
  if (h.empty()) {
    *d = nullptr;
    return LT_OK;
  }
  cudaError_t e = device_alloc((void**)d, h.size() * sizeof(T));
  if (e != cudaSuccess) {
    *d = nullptr;
    return set_error(LT_ENOMEM, "cudaMalloc(%s, %zu bytes): %s", what, h.size() * sizeof(T),
                     cudaGetErrorString(e));
  }
  e = cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_error(e, what);
  return LT_OK;
}

static void free_camera(CameraPlan& c) {
  cudaFree(c.d_slice);
  cudaFree(c.d_items);
  cudaFree(c.d_rz);
  cudaFree(c.d_xr);
  cudaFree(c.rot.tz);
  cudaFree(c.rot.jz);
  cudaFree(c.rot.tx);
  cudaFree(c.rot.jx);
  for (int k = 0; k < 3; ++k) {
    cudaFree(c.d_gb[k]);
    cudaFree(c.d_gtab[k]);
    cudaFree(c.d_gjo[k]);
  }
  cudaFree(c.d_srange);
  cudaFree(c.d_trange);
  cudaFree(c.d_lens);
  cudaFree(c.d_cols);
  cudaFree(c.d_rows);
  cudaFree(c.d_owner);
  cudaFree(c.d_mask);
  cudaFree(c.d_det_range);
  cudaFree(c.d_det_union);
  cudaFree(c.d_cand_all_s);
  cudaFree(c.d_cand_all_t);
  cudaFree(c.d_zbuf);
  cudaFree(c.d_s2tab);
  cudaFree(c.d_s2desc);
  cudaFree(c.d_s2bits);
  cudaFree(c.d_s2ivals);
  cudaFree(c.d_fa);
  cudaFree(c.d_stab);
  cudaFree(c.d_ttab);
  cudaFree(c.d_adj_s);
  cudaFree(c.d_adj_t);
  cudaFree(c.d_adj_ox);
  cudaFree(c.d_adj_oy);
  c = CameraPlan();
}

// Brick box of the brick-staged forward for camera c.  A stage fill brings
// the bricks of a group of tma_forward_group() consecutive slices (groups
// start at multiples of the group size) with one origin: for a tile of 32
// target pixels along an axis the first taps floor(xi(i) - Q + 1/2) range
// over [lo, hi] over the group's slices (evaluated at the tile's two ends,
// widened by 1e-3 so that float evaluation on the device stays inside); the
// brick starts at the smallest first tap (columns rounded down to a
// multiple of 4) and must hold W taps past the largest.  Cameras whose
// window class exceeds 4, whose bricks exceed 1024 floats or
// tma_forward_max_by() rows, or whose grid rows are not a multiple of 4
// floats keep the direct kernels.  tma_nb marks a camera that runs the
// brick-staged kernel: 4 with its t-parts in band form (footprints of three
// or more taps whose groups of four pixel rows keep their taps within
// tma_forward_band_rows() brick rows), 1 with one row of taps per pixel row.
static void plan_bricks(CameraPlan& c, int grid_nx, int nz, const std::vector<Footprint>& fps,
                        const std::vector<Footprint>& fpt, int tiles_s, int tiles_t) {
  c.tma_bx = c.tma_by = c.tma_nb = 0;
  const int W = window_class(std::max(c.wmax_s, c.wmax_t));
  if (W > 4 || grid_nx % 4 != 0) return;   // a TMA row stride is a multiple of 16 bytes
  auto tap_range = [](const Footprint& f, int i0, int i1, long long& lo, long long& hi) {
    const double a = f.C0 + f.C1 * i0 - (double)f.a.Q + 0.5, b = f.C0 + f.C1 * i1 - (double)f.a.Q + 0.5;
    lo = std::min(lo, (long long)std::floor(std::min(a, b) - 1e-3));
    hi = std::max(hi, (long long)std::floor(std::max(a, b) + 1e-3));
  };
  const int G = tma_forward_group();
  long long need_bx = 0, span_t = 0, need_nb = 0;
  for (int k = 0; k < c.K; ++k)
    for (int n0 = 0; n0 < nz; n0 += G) {
      const int n1 = std::min(nz, n0 + G);
      for (int ts = 0; ts < tiles_s; ++ts) {
        long long lo = LLONG_MAX, hi = LLONG_MIN;
        for (int n = n0; n < n1; ++n)
          tap_range(fps[(size_t)k * nz + n], ts * kBeamTileS, ts * kBeamTileS + kBeamTileS - 1, lo, hi);
        need_bx = std::max(need_bx, hi + W - 1 - (lo & ~3LL) + 1);
      }
      for (int tt = 0; tt < tiles_t; ++tt) {
        long long lo = LLONG_MAX, hi = LLONG_MIN;
        for (int n = n0; n < n1; ++n) {
          tap_range(fpt[(size_t)k * nz + n], tt * kBeamTileT, tt * kBeamTileT + kBeamTileT - 1, lo, hi);
          for (int r0 = tt * kBeamTileT; r0 < tt * kBeamTileT + kBeamTileT; r0 += 4) {   // band rows of a 4-row group
            long long glo = LLONG_MAX, ghi = LLONG_MIN;
            tap_range(fpt[(size_t)k * nz + n], r0, r0 + 3, glo, ghi);
            need_nb = std::max(need_nb, ghi - glo + W);
          }
        }
        span_t = std::max(span_t, hi - lo);
      }
    }
  const long long bx = (need_bx + 3) / 4 * 4, by = span_t + W;
  if (bx > 256 || by > tma_forward_max_by() || bx * by > 1024) return;
  c.tma_bx = (int)bx;
  c.tma_by = (int)by;
  // band t-parts pay where footprints take three or more taps (the W per-row
  // 8-byte loads of a pixel row become four band rows shared by four rows);
  // at two taps the per-row form issues fewer instructions and is faster
  // (measured: 0.079 against 0.085 ms on the 128^3 plenoptic camera; the
  // multi-view step with three-tap cameras 275 -> 247 ms with bands)
  c.tma_nb = W >= 3 && need_nb <= tma_forward_band_rows() ? 4 : 1;
}

// Image box of the box-staged adjoint for camera c: per (cell, chunk of sc
// slices, tile of adjoint_tile_x() x adjoint_tile_y() voxels), the target
// pixels the tile's windows reach, [first window start, last window start +
// largest window - 1] per axis over the chunk's slices (window starts
// floor(min(lo, hi)) - 1 of (j -+ 1/2 -+ Q - c0) / c1 at the tile's two
// ends, widened by 1e-3), the columns rounded to a multiple of 4.  The box
// is the largest span.  Chunks are adjoint_chunk_max() = 8 slices (boxes up
// to 8192 floats) or 4 slices (boxes up to 12288 floats: strongly defocused
// cameras, whose windows span 15 or more pixels per axis, fit only so, and
// the kernel single-buffers such stages to keep three CTAs per SM); of the
// depths that fit, the one whose grid takes fewer whole rounds of resident
// CTAs (a 4-slice chunk counted as 55 % of an 8-slice one) is kept, so that
// small workloads split into more CTAs (the bench camera: 1024 8-slice CTAs
// on 444 resident slots ran 0.085 ms, 2048 4-slice CTAs 0.075 ms).  Cameras
// that fit neither keep the direct adjoint, and so do cameras whose target
// rows are not a multiple of 4 floats.
static void plan_adjoint_box(CameraPlan& c, const lt_volume_desc& v, int tgt_ns, int frames,
                             const std::vector<Footprint>& fps, const std::vector<Footprint>& fpt) {
  c.adj_bx = c.adj_by = 0;
  c.adj_sc = adjoint_chunk_max();
  if (tgt_ns % 4 != 0 || c.wimax_s > 32 || c.wimax_t > 32) return;   // a TMA row stride is a multiple of 16 bytes
  const int TX = adjoint_tile_x(), TY = adjoint_tile_y();
  auto start = [](const Footprint& f, int j, double eps) {
    const double lo = (j - 0.5 - (double)f.a.Q - f.C0) / f.C1, hi = (j + 0.5 + (double)f.a.Q - f.C0) / f.C1;
    return (long long)std::floor(std::min(lo, hi) + eps) - 1;
  };
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long tiles = (long long)((v.nx + TX - 1) / TX) * ((v.ny + TY - 1) / TY) * frames;
  double best = 0.0;
  for (int SC = adjoint_chunk_max(); SC >= 4; SC /= 2) {
    long long need_bx = 0, need_by = 0;
    for (int k = 0; k < c.K; ++k)
      for (int n0 = 0; n0 < v.nz; n0 += SC) {
        for (int j0 = 0; j0 < v.nx; j0 += TX) {
          const int j1 = std::min(j0 + TX, v.nx) - 1;
          long long lo = LLONG_MAX, hi = LLONG_MIN;
          for (int n = n0; n < std::min(n0 + SC, v.nz); ++n) {
            const size_t q = (size_t)k * v.nz + n;
            for (int j : {j0, j1}) {
              lo = std::min(lo, start(fps[q], j, -1e-3));
              hi = std::max(hi, start(fps[q], j, 1e-3) + c.wimax_s - 1);
            }
          }
          need_bx = std::max(need_bx, hi - (lo & ~3LL) + 1);
        }
        for (int j0 = 0; j0 < v.ny; j0 += TY) {
          const int j1 = std::min(j0 + TY, v.ny) - 1;
          long long lo = LLONG_MAX, hi = LLONG_MIN;
          for (int n = n0; n < std::min(n0 + SC, v.nz); ++n) {
            const size_t q = (size_t)k * v.nz + n;
            for (int j : {j0, j1}) {
              lo = std::min(lo, start(fpt[q], j, -1e-3));
              hi = std::max(hi, start(fpt[q], j, 1e-3) + c.wimax_t - 1);
            }
          }
          need_by = std::max(need_by, hi - lo + 1);
        }
      }
    const long long bx = (need_bx + 3) / 4 * 4, by = need_by;
    if (bx < 4 || by < 1 || bx > 256 || by > 256 || bx * by > (SC == 8 ? 8192 : 12288)) continue;
    // whole rounds of resident CTAs, in units of a 4-slice chunk's work (a
    // 4-slice chunk costs about 10 % more per slice: its box is loaded twice
    // as often)
    const int occ = adjoint_occupancy((int)bx, (int)by, c.wimax_s, c.wimax_t, SC);
    if (occ <= 0) continue;
    const long long units = tiles * ((v.nz + SC - 1) / SC), slots = (long long)occ * std::max(1, sms);
    const double cost = (double)((units + slots - 1) / slots) * (SC == 8 ? 2.0 : 1.1);
    if (c.adj_bx == 0 || cost < best) {
      best = cost;
      c.adj_bx = (int)bx;
      c.adj_by = (int)by;
      c.adj_sc = SC;
    }
  }
}

// Window tables and box origins of the box-staged adjoint, built on the
// device from the slice parameters; a camera whose tables exceed
// kMaxTableBytes, or whose boxes do not fit (reported by the build), keeps
// the direct adjoint.
static lt_status plan_adjoint_tables(CameraPlan& c, const lt_volume_desc& v, int idx) {
  constexpr size_t kMaxTableBytes = (size_t)512 << 20;
  if (c.adj_bx == 0 || !tma_forward_available()) {
    c.adj_bx = c.adj_by = 0;
    return LT_OK;
  }
  size_t sb, tb, nox, noy;
  adjoint_table_sizes(c.K, v.nz, v.nx, v.ny, c.wimax_s, c.wimax_t, c.adj_sc, &sb, &tb, &nox, &noy);
  if (sb + tb > kMaxTableBytes) {
    c.adj_bx = c.adj_by = 0;
    return LT_OK;
  }
  int* d_bad = nullptr;
  if (device_alloc((void**)&c.d_adj_s, sb) != cudaSuccess || device_alloc((void**)&c.d_adj_t, tb) != cudaSuccess ||
      device_alloc((void**)&c.d_adj_ox, nox * sizeof(int2)) != cudaSuccess ||
      device_alloc((void**)&c.d_adj_oy, noy * sizeof(int2)) != cudaSuccess ||
      device_alloc((void**)&d_bad, sizeof(int)) != cudaSuccess) {
    cudaFree(d_bad);
    return set_error(LT_ENOMEM, "camera %d: cudaMalloc(adjoint window tables, %zu bytes)", idx, sb + tb);
  }
  int bad = 0;
  cudaError_t e = cudaMemset(d_bad, 0, sizeof(int));
  if (e == cudaSuccess)
    e = launch_adjoint_tables(c.d_slice, c.K, v.nz, v.nx, v.ny, c.wimax_s, c.wimax_t, c.adj_bx, c.adj_by, c.adj_sc,
                              c.d_adj_s, c.d_adj_t, c.d_adj_ox, c.d_adj_oy, d_bad, 0);
  if (e == cudaSuccess) e = cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_bad);
  if (e != cudaSuccess) return cuda_error(e, "adjoint window tables");
  if (bad) {   // a box the planner sized too small: the direct adjoint serves this camera
    cudaFree(c.d_adj_s);
    cudaFree(c.d_adj_t);
    cudaFree(c.d_adj_ox);
    cudaFree(c.d_adj_oy);
    c.d_adj_s = c.d_adj_t = nullptr;
    c.d_adj_ox = c.d_adj_oy = nullptr;
    c.adj_bx = c.adj_by = 0;
  }
  return LT_OK;
}

// Footprint-weight tables of the brick-staged forward (one entry per
// (cell, slice, tile column) and (cell, slice, tile row)), built on the
// device from the slice parameters.  A camera whose tables would exceed
// kMaxTableBytes, or whose build reports a brick or band that does not fit,
// keeps the direct kernel; only a failed allocation is an error.
static lt_status plan_weight_tables(CameraPlan& c, int nz, int idx) {
  constexpr size_t kMaxTableBytes = (size_t)512 << 20;
  if (c.tma_nb == 0 || !tma_forward_available()) {
    c.tma_nb = 0;
    return LT_OK;
  }
  const int W = window_class(std::max(c.wmax_s, c.wmax_t));
  const bool band = c.tma_nb == 4;
  const size_t bytes = tma_table_bytes(W, band, c.K, nz, c.tiles_s, c.tiles_t);
  if (bytes > kMaxTableBytes) {
    c.tma_nb = 0;
    return LT_OK;
  }
  const size_t s_bytes = tma_table_bytes(W, band, c.K, nz, c.tiles_s, 0);
  int* d_bad = nullptr;
  if (device_alloc(&c.d_stab, s_bytes) != cudaSuccess ||
      device_alloc(&c.d_ttab, bytes - s_bytes) != cudaSuccess ||
      device_alloc((void**)&d_bad, sizeof(int)) != cudaSuccess) {
    cudaFree(d_bad);
    return set_error(LT_ENOMEM, "camera %d: cudaMalloc(forward weight tables, %zu bytes)", idx, bytes);
  }
  int bad = 0;
  cudaError_t e = cudaMemset(d_bad, 0, sizeof(int));
  if (e == cudaSuccess)
    e = launch_beam_tables(c.d_slice, c.K, nz, c.tiles_s, c.tiles_t, W, band, c.tma_bx, c.tma_by, c.d_stab,
                           c.d_ttab, d_bad, 0);
  if (e == cudaSuccess) e = cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_bad);
  if (e != cudaSuccess) return cuda_error(e, "forward weight tables");
  if (bad) {   // a brick or band the planner sized too small: the direct kernel serves this camera
    cudaFree(c.d_stab);
    cudaFree(c.d_ttab);
    c.d_stab = c.d_ttab = nullptr;
    c.tma_nb = 0;
  }
  return LT_OK;
}

// Per (cell, slice) parameters of the slice -> image-plane transport.
static lt_status plan_slices(const lt_volume_desc& v, CameraPlan& c, double d_img, int tgt_ns,
                             int tgt_nt, double tgt_ps, double tgt_pt, double extra_scale, int frames, int idx) {
  const lt_camera_desc& d = c.desc;
  std::vector<SliceParam> sp((size_t)c.K * v.nz);
  const int tiles_s = (tgt_ns + kBeamTileS - 1) / kBeamTileS;
  const int tiles_t = (tgt_nt + kBeamTileT - 1) / kBeamTileT;
  std::vector<int2> srange((size_t)c.K * tiles_s, make_int2(INT32_MAX, -1));
  std::vector<int2> trange((size_t)c.K * tiles_t, make_int2(INT32_MAX, -1));
  // Slice n is active for a tile when the union of its pixels' footprints
  // (centres c0 + c1 i, half-width Q, cells [-1/2, n_src - 1/2]) meets the grid.
  auto mark = [](std::vector<int2>& rng, size_t base, int tiles, int tile_w, int n_tgt, int n_src,
                 const Footprint& f, int n) {
    for (int tile = 0; tile < tiles; ++tile) {
      const int i0 = tile * tile_w, i1 = std::min(n_tgt, i0 + tile_w) - 1;
      const double a = f.C0 + f.C1 * i0, b = f.C0 + f.C1 * i1;
      const double lo = std::min(a, b) - f.Q - 1e-3, hi = std::max(a, b) + f.Q + 1e-3;
      if (hi > -0.5 && lo < n_src - 0.5) {
        int2& r = rng[base + tile];
        r.x = std::min(r.x, n);
        r.y = std::max(r.y, n + 1);
      }
    }
  };
  std::vector<Footprint> fps((size_t)c.K * v.nz), fpt((size_t)c.K * v.nz);
  for (int k = 0; k < c.K; ++k) {
    for (int n = 0; n < v.nz; ++n) {
      const double dist = d.d_obj + centre(n, v.nz, v.dz);
      Row P, L;
      slice_rows(dist, d_img, d.f_main, &P, &L);
      Footprint& fs = fps[(size_t)k * v.nz + n];
      Footprint& ft = fpt[(size_t)k * v.nz + n];
      if (!footprint(L, P, c.cells[k].sk, c.cells[k].d0s, centre(0, tgt_ns, tgt_ps), tgt_ps,
                     centre(0, v.nx, v.dx), v.dx, d.basis, &fs) ||
          !footprint(L, P, c.cells[k].tk, c.cells[k].d0t, centre(0, tgt_nt, tgt_pt), tgt_pt,
                     centre(0, v.ny, v.dy), v.dy, d.basis, &ft))
        return set_error(LT_EINVAL, "camera %d: degenerate transport at slice %d", idx, n);
      mark(srange, (size_t)k * tiles_s, tiles_s, kBeamTileS, tgt_ns, v.nx, fs, n);
      mark(trange, (size_t)k * tiles_t, tiles_t, kBeamTileT, tgt_nt, v.ny, ft, n);
      SliceParam& p = sp[(size_t)k * v.nz + n];
      std::memset(&p, 0, sizeof(p));
      p.s = fs.a;
      p.t = ft.a;
      p.scale = (float)(fs.H * v.dx * ft.H * v.dy * v.dz * extra_scale);
      p.ws = fwd_window(p.s.Q);
      p.wt = fwd_window(p.t.Q);
      p.wis = adj_window(p.s.Q, fs.C1);
      p.wit = adj_window(p.t.Q, ft.C1);
      c.wmax_s = std::max(c.wmax_s, p.ws);
      c.wmax_t = std::max(c.wmax_t, p.wt);
      c.wimax_s = std::max(c.wimax_s, p.wis);
      c.wimax_t = std::max(c.wimax_t, p.wit);
    }
  }
  if (c.wmax_s > kMaxForwardWindow || c.wmax_t > kMaxForwardWindow)
    return set_error(LT_EUNSUPPORTED,
                     "camera %d: a pixel footprint spans %d x %d voxels (kernel limit %d); use finer pixels or coarser voxels",
                     idx, c.wmax_s, c.wmax_t, kMaxForwardWindow);
  if (c.wimax_s > kMaxAdjointWindow || c.wimax_t > kMaxAdjointWindow)
    return set_error(LT_EUNSUPPORTED,
                     "camera %d: a voxel is covered by %d x %d pixel footprints (kernel limit %d); use coarser pixels or finer voxels",
                     idx, c.wimax_s, c.wimax_t, kMaxAdjointWindow);
  plan_bricks(c, v.nx, v.nz, fps, fpt, tiles_s, tiles_t);
  plan_adjoint_box(c, v, tgt_ns, frames, fps, fpt);
  for (auto& r : srange)
    if (r.y < 0) r = make_int2(0, 0);
  for (auto& r : trange)
    if (r.y < 0) r = make_int2(0, 0);
  c.h_srange = srange;
  c.h_trange = trange;
  c.tiles_s = tiles_s;
  c.tiles_t = tiles_t;
  // forward work items: one per (cell, tile) when each cell has its own
  // output plane (plenoptic array plane), one per tile over all cells when
  // the cells sum into one image (single lens); cost = slices visited
  const bool per_cell = c.desc.kind == LT_CAM_PLENOPTIC;
  c.h_items.clear();
  for (int tile = 0; tile < tiles_s * tiles_t; ++tile) {
    const int ts = tile % tiles_s, tt = tile / tiles_s;
    int total = 0;
    for (int k = 0; k < c.K; ++k) {
      const int2 a = srange[(size_t)k * tiles_s + ts], b = trange[(size_t)k * tiles_t + tt];
      const int cost = std::max(0, std::min(a.y, b.y) - std::max(a.x, b.x));
      if (per_cell) c.h_items.push_back(make_int4(idx, k, tile, cost));
      total += cost;
    }
    if (!per_cell) c.h_items.push_back(make_int4(idx, -1, tile, total));
  }
  std::stable_sort(c.h_items.begin(), c.h_items.end(), [](const int4& a, const int4& b) { return a.w > b.w; });
  std::vector<int4> local = c.h_items;
  for (auto& it : local) it.x = 0;   // a single-camera batch names this camera 0
  c.n_items = (int)local.size();
  c.n_real_items = (int)std::count_if(local.begin(), local.end(), [](const int4& a) { return a.w > 0; });
  lt_status s = upload(local, &c.d_items, "forward work items");
  if (s != LT_OK) return s;
  s = upload(srange, &c.d_srange, "tile slice ranges");
  if (s == LT_OK) s = upload(trange, &c.d_trange, "tile slice ranges");
  if (s != LT_OK) return s;
  s = upload(sp, &c.d_slice, "slice parameters");
  if (s != LT_OK) return s;
  s = plan_weight_tables(c, v.nz, idx);
  if (s != LT_OK) return s;
  return plan_adjoint_tables(c, v, idx);
}

// Array -> detector stage of a plenoptic camera (Sec. II-D, II-F2).
static lt_status plan_stage_two(CameraPlan& c, int frames, int idx) {
  const lt_camera_desc& d = c.desc;
  const int mns = d.mla_ns, mnt = d.mla_nt;
  const int nmu = mns * mnt;
  if ((long long)d.arr_ns * d.arr_nt >= (1LL << 31))   // the stage-2 kernels index one array plane in 32 bits
    return set_error(LT_EUNSUPPORTED, "camera %d: array plane of %d x %d pixels (limit 2^31 pixels)", idx, d.arr_ns,
                     d.arr_nt);
  const bool hex = d.mla_layout == LT_MLA_HEX;
  // Lenslet centres: the square grid, or the hexagonal lattice (rows
  // pitch sqrt(3)/2 apart, odd rows shifted by half a pitch, centred on the
  // axis with a column offset of -pitch/4).
  const double rowh = hex ? d.mla_pitch * std::sqrt(3.0) / 2.0 : d.mla_pitch;
  std::vector<double> S(nmu), T(nmu);
  for (int mt = 0; mt < mnt; ++mt)
    for (int ms = 0; ms < mns; ++ms) {
      const int mu = mt * mns + ms;
      S[mu] = hex ? (ms - 0.5 * (mns - 1) + 0.5 * (mt & 1) - 0.25) * d.mla_pitch : centre(ms, mns, d.mla_pitch);
      T[mu] = hex ? (mt - 0.5 * (mnt - 1)) * rowh : centre(mt, mnt, d.mla_pitch);
    }
  // Ownership: the lenslet whose disc strictly contains the pixel centre
  // (discs are disjoint, radius <= pitch / 2), searched among the nearest
  // rows / columns.  M = apertures x the coded transmission (Sec. II-D).
  const size_t npix = (size_t)d.arr_ns * d.arr_nt;
  std::vector<int32_t> owner(npix, -1);
  std::vector<float> mask(npix, 0.0f);
  const double r2 = d.mla_radius * d.mla_radius;
  for (int jt = 0; jt < d.arr_nt; ++jt) {
    const double t = centre(jt, d.arr_nt, d.arr_pt);
    const int mt0 = (int)std::nearbyint(t / rowh + 0.5 * (mnt - 1));
    for (int js = 0; js < d.arr_ns; ++js) {
      const double sv = centre(js, d.arr_ns, d.arr_ps);
      int own = -1;
      for (int dm = hex ? -1 : 0; dm <= (hex ? 1 : 0) && own < 0; ++dm) {
        const int mt = mt0 + dm;
        if (mt < 0 || mt >= mnt) continue;
        const int ms = (int)std::nearbyint(sv / d.mla_pitch + 0.5 * (mns - 1) - (hex ? 0.5 * (mt & 1) - 0.25 : 0.0));
        if (ms < 0 || ms >= mns) continue;
        const int mu = mt * mns + ms;
        const double ds = sv - S[mu], dt = t - T[mu];
        if (ds * ds + dt * dt < r2) own = mu;
      }
      owner[(size_t)jt * d.arr_ns + js] = own;
      if (own >= 0) {
        float m = 1.0f;
        if (d.arr_mask) m = std::min(1.0f, std::max(0.0f, d.arr_mask[(size_t)jt * d.arr_ns + js]));
        mask[(size_t)jt * d.arr_ns + js] = m;
      }
    }
  }
  // Lenslet blocks.  Square grid: the lenslet's cell [c - pitch/2, c + pitch/2)
  // (blocks tile the plane; unowned pixels inside a block are written as 0).
  // Hexagonal lattice: the bounding rows / columns of the owned pixels
  // (blocks overlap; each lenslet writes only its own pixels).
  std::vector<int2> cols(nmu, make_int2(INT32_MAX, -1)), rows(nmu, make_int2(INT32_MAX, -1));
  int full_cover = 1;
  if (!hex) {
    const double edge_s = centre(0, mns, d.mla_pitch) - 0.5 * d.mla_pitch;
    const double edge_t = centre(0, mnt, d.mla_pitch) - 0.5 * d.mla_pitch;
    std::vector<int2> cs(mns, make_int2(INT32_MAX, -1)), rs(mnt, make_int2(INT32_MAX, -1));
    for (int j = 0; j < d.arr_ns; ++j) {
      const double m = std::floor((centre(j, d.arr_ns, d.arr_ps) - edge_s) / d.mla_pitch);
      if (m >= 0 && m < mns) {
        cs[(int)m].x = std::min(cs[(int)m].x, j);
        cs[(int)m].y = std::max(cs[(int)m].y, j + 1);
      } else {
        full_cover = 0;
      }
    }
    for (int j = 0; j < d.arr_nt; ++j) {
      const double m = std::floor((centre(j, d.arr_nt, d.arr_pt) - edge_t) / d.mla_pitch);
      if (m >= 0 && m < mnt) {
        rs[(int)m].x = std::min(rs[(int)m].x, j);
        rs[(int)m].y = std::max(rs[(int)m].y, j + 1);
      } else {
        full_cover = 0;
      }
    }
    for (int mt = 0; mt < mnt; ++mt)
      for (int ms = 0; ms < mns; ++ms) {
        cols[(size_t)mt * mns + ms] = cs[ms];
        rows[(size_t)mt * mns + ms] = rs[mt];
      }
  } else {
    full_cover = 0;
    for (int jt = 0; jt < d.arr_nt; ++jt)
      for (int js = 0; js < d.arr_ns; ++js) {
        const int mu = owner[(size_t)jt * d.arr_ns + js];
        if (mu < 0) continue;
        cols[mu].x = std::min(cols[mu].x, js);
        cols[mu].y = std::max(cols[mu].y, js + 1);
        rows[mu].x = std::min(rows[mu].x, jt);
        rows[mu].y = std::max(rows[mu].y, jt + 1);
      }
  }
  int max_cols = 0, max_rows = 0;
  for (int mu = 0; mu < nmu; ++mu) {
    if (cols[mu].y < 0 || rows[mu].y < 0) {
      cols[mu] = make_int2(0, 0);
      rows[mu] = make_int2(0, 0);
    }
    max_cols = std::max(max_cols, cols[mu].y - cols[mu].x);
    max_rows = std::max(max_rows, rows[mu].y - rows[mu].x);
  }
  if (max_cols > kMaxLensletPixels || max_rows > kMaxLensletPixels)
    return set_error(LT_EUNSUPPORTED, "camera %d: %d x %d array pixels per lenslet (kernel limit %d)",
                     idx, max_cols, max_rows, kMaxLensletPixels);
  // Per (cell, lenslet) footprints of detector pixels on the array plane.
  std::vector<LensletParam> lens((size_t)c.K * nmu);
  std::vector<int4> det_range((size_t)c.K * nmu, make_int4(0, -1, 0, -1));
  int wis = 0, wit = 0;
  for (int k = 0; k < c.K; ++k) {
    for (int mt = 0; mt < mnt; ++mt) {
      for (int ms = 0; ms < mns; ++ms) {
        const int mu = mt * mns + ms;
        const double f = c.focal[(size_t)mu];
        Row Ps, Ls, Pt, Lt;
        lenslet_rows(d.d_mla_det, d.d_lens_mla, f, S[mu], &Ps, &Ls);
        lenslet_rows(d.d_mla_det, d.d_lens_mla, f, T[mu], &Pt, &Lt);
        Footprint fs, ft;
        if (!footprint(Ls, Ps, c.cells[k].sk, c.cells[k].d0s, centre(0, d.det_ns, d.det_ps), d.det_ps,
                       centre(0, d.arr_ns, d.arr_ps), d.arr_ps, d.basis, &fs) ||
            !footprint(Lt, Pt, c.cells[k].tk, c.cells[k].d0t, centre(0, d.det_nt, d.det_pt), d.det_pt,
                       centre(0, d.arr_nt, d.arr_pt), d.arr_pt, d.basis, &ft))
          return set_error(LT_EINVAL, "camera %d: degenerate microlens transport (lenslet %d,%d)", idx, mt, ms);
        LensletParam& L = lens[(size_t)k * nmu + (size_t)mt * mns + ms];
        std::memset(&L, 0, sizeof(L));
        L.s = fs.a;
        L.t = ft.a;
        L.scale = (float)(fs.H * d.arr_ps * ft.H * d.arr_pt);
        wis = std::max(wis, adj_window(L.s.Q, fs.C1));
        wit = std::max(wit, adj_window(L.t.Q, ft.C1));
        // detector columns / rows whose footprints can reach this lenslet's block
        if (cols[mu].y > cols[mu].x && rows[mu].y > rows[mu].x) {
          {
            const double lo = cols[mu].x - 0.5 - fs.Q, hi = cols[mu].y - 0.5 + fs.Q;
            double a = (lo - fs.C0) / fs.C1, b = (hi - fs.C0) / fs.C1;
            if (a > b) std::swap(a, b);
            det_range[(size_t)k * nmu + mu].x = (int)std::max<long long>(0, (long long)std::floor(a) - 1);
            det_range[(size_t)k * nmu + mu].y = (int)std::min<long long>(d.det_ns - 1, (long long)std::ceil(b) + 1);
          }
          {
            const double lo = rows[mu].x - 0.5 - ft.Q, hi = rows[mu].y - 0.5 + ft.Q;
            double a = (lo - ft.C0) / ft.C1, b = (hi - ft.C0) / ft.C1;
            if (a > b) std::swap(a, b);
            det_range[(size_t)k * nmu + mu].z = (int)std::max<long long>(0, (long long)std::floor(a) - 1);
            det_range[(size_t)k * nmu + mu].w = (int)std::min<long long>(d.det_nt - 1, (long long)std::ceil(b) + 1);
          }
        }
      }
    }
  }
  // union over cells of each lenslet's detector window, and the lenslets
  // whose union window covers each detector column / row
  std::vector<int4> det_union(nmu, make_int4(INT32_MAX, -1, INT32_MAX, -1));
  for (int k = 0; k < c.K; ++k)
    for (int m = 0; m < nmu; ++m) {
      const int4 r = det_range[(size_t)k * nmu + m];
      int4& u = det_union[m];
      if (r.y >= r.x) { u.x = std::min(u.x, r.x); u.y = std::max(u.y, r.y); }
      if (r.w >= r.z) { u.z = std::min(u.z, r.z); u.w = std::max(u.w, r.w); }
    }
  std::vector<int2> cand_all_s(d.det_ns, make_int2(INT32_MAX, -1)), cand_all_t(d.det_nt, make_int2(INT32_MAX, -1));
  for (int m = 0; m < nmu; ++m) {
    int4& u = det_union[m];
    if (u.y < u.x || u.w < u.z) { u = make_int4(0, -1, 0, -1); continue; }
    if (u.y - u.x + 1 > kStage2Window || u.w - u.z + 1 > kStage2Window)
      return set_error(LT_EUNSUPPORTED, "camera %d: a lenslet's sub-image spans %d x %d detector pixels (kernel limit %d)",
                       idx, u.y - u.x + 1, u.w - u.z + 1, kStage2Window);
    const int ms = m % mns, mt = m / mns;
    for (int i = u.x; i <= u.y; ++i) {
      cand_all_s[i].x = std::min(cand_all_s[i].x, ms);
      cand_all_s[i].y = std::max(cand_all_s[i].y, ms);
    }
    for (int i = u.z; i <= u.w; ++i) {
      cand_all_t[i].x = std::min(cand_all_t[i].x, mt);
      cand_all_t[i].y = std::max(cand_all_t[i].y, mt);
    }
  }
  for (auto& r : cand_all_s)
    if (r.y < 0) r = make_int2(0, -1);
  for (auto& r : cand_all_t)
    if (r.y < 0) r = make_int2(0, -1);
  if (wis > kMaxAdjointWindow || wit > kMaxAdjointWindow)
    return set_error(LT_EUNSUPPORTED, "camera %d: an array pixel is covered by %d x %d detector footprints (kernel limit %d)",
                     idx, wis, wit, kMaxAdjointWindow);
  lt_status s;
  if ((s = upload(lens, &c.d_lens, "lenslet parameters")) != LT_OK) return s;
  if ((s = upload(cols, &c.d_cols, "lenslet columns")) != LT_OK) return s;
  if ((s = upload(rows, &c.d_rows, "lenslet rows")) != LT_OK) return s;
  if ((s = upload(owner, &c.d_owner, "pixel owners")) != LT_OK) return s;
  if ((s = upload(mask, &c.d_mask, "mask")) != LT_OK) return s;
  if ((s = upload(det_range, &c.d_det_range, "lenslet detector ranges")) != LT_OK) return s;
  if ((s = upload(det_union, &c.d_det_union, "lenslet detector windows")) != LT_OK) return s;
  if ((s = upload(cand_all_s, &c.d_cand_all_s, "candidate columns")) != LT_OK) return s;
  if ((s = upload(cand_all_t, &c.d_cand_all_t, "candidate rows")) != LT_OK) return s;
  {
    const size_t zb = (size_t)frames * nmu * kStage2Window * kStage2Window * sizeof(float);
    cudaError_t ez = device_alloc((void**)&c.d_zbuf, zb);
    if (ez != cudaSuccess) {
      c.d_zbuf = nullptr;
      return set_error(LT_ENOMEM, "cudaMalloc(lenslet sub-images, %zu bytes): %s", zb, cudaGetErrorString(ez));
    }
  }
  c.Na = (int64_t)d.arr_ns * d.arr_nt;
  const size_t fa_bytes = (size_t)frames * c.K * c.Na * sizeof(float);
  cudaError_t e = device_alloc((void**)&c.d_fa, fa_bytes);
  if (e != cudaSuccess) {
    c.d_fa = nullptr;
    return set_error(LT_ENOMEM, "cudaMalloc(array plane, %zu bytes): %s", fa_bytes, cudaGetErrorString(e));
  }
  lt::StageTwo& s2 = c.s2;
  s2.lens = c.d_lens;
  s2.cols = c.d_cols;
  s2.rows = c.d_rows;
  s2.owner = c.d_owner;
  s2.mask = c.d_mask;
  s2.overlap = hex ? 1 : 0;
  s2.mla_ns = mns;
  s2.mla_nt = mnt;
  s2.arr_ns = d.arr_ns;
  s2.arr_nt = d.arr_nt;
  s2.det_ns = d.det_ns;
  s2.det_nt = d.det_nt;
  s2.K = c.K;
  s2.wis = wis;
  s2.wit = wit;
  s2.max_cols = max_cols;
  s2.max_rows = max_rows;
  s2.det_range = c.d_det_range;
  s2.det_union = c.d_det_union;
  s2.cand_all_s = c.d_cand_all_s;
  s2.cand_all_t = c.d_cand_all_t;
  s2.zbuf = c.d_zbuf;
  s2.full_cover = full_cover;
  s2.sub_n = 1;
  s2.sub_s = 0;
  // The form the stage-two kernels walk: per (lenslet, cell) a descriptor
  // and, for a non-empty window, a transport table entry Bs (nc x nds) then
  // Bt (nr x ndt), padded to 4 floats and evaluated once here on the device;
  // per lenslet the ownership bits of its block.
  if (c.K >= (1 << 15)) return set_error(LT_EUNSUPPORTED, "camera %d: %d angular cells (limit 32767)", idx, c.K);
  std::vector<lt::S2Desc> desc((size_t)nmu * c.K);
  std::vector<uint32_t> bits((size_t)nmu * 16, 0u);
  std::vector<uint32_t> ivals((size_t)nmu * 8, 0u);   // uint16 per row: c0 | c1 << 8
  int iv_ok = 1;
  long long tab = 0;
  int tab_max = 0, pix_max = 0, w_max = 0, z_max = 0, y_max = 0;
  for (int m = 0; m < nmu; ++m) {
    const int nc = cols[m].y - cols[m].x, nr = rows[m].y - rows[m].x;
    const int4 u = det_union[m];
    const int nsu = u.y - u.x + 1, ntu = u.w - u.z + 1;
    pix_max = std::max(pix_max, nr * nc);
    z_max = std::max(z_max, std::max(nsu, 0) * std::max(ntu, 0));
    for (int r = 0; r < nr; ++r) {
      int c0 = -1, c1 = -1, runs = 0;
      for (int cix = 0; cix < nc; ++cix) {
        const int o = r * nc + cix;
        const int own = owner[(size_t)(rows[m].x + r) * d.arr_ns + cols[m].x + cix];
        if (own == m) {
          bits[(size_t)m * 16 + (o >> 5)] |= 1u << (o & 31);
          if (c1 != cix) {
            ++runs;
            c0 = cix;
          }
          c1 = cix + 1;
        } else if (!hex && own < 0) {
          bits[(size_t)m * 16 + 8 + (o >> 5)] |= 1u << (o & 31);
        } else if (!hex) {
          iv_ok = 0;   // another lenslet's pixel inside a tiling block: keep the bits
        }
      }
      if (runs > 1) iv_ok = 0;
      const uint32_t iv = runs ? (uint32_t)c0 | (uint32_t)c1 << 8 : 0u;
      ivals[(size_t)m * 8 + (r >> 1)] |= iv << (16 * (r & 1));
    }
    for (int k = 0; k < c.K; ++k) {
      const int4 r = det_range[(size_t)k * nmu + m];
      const int nds = r.y - r.x + 1, ndt = r.w - r.z + 1;
      lt::S2Desc& e = desc[(size_t)m * c.K + k];
      e.off = -1;
      e.px0 = rows[m].x * d.arr_ns + cols[m].x;
      e.y0 = 0;
      e.zo = 0;
      e.dims = (uint32_t)nc | (uint32_t)nr << 8;
      e.scale = lens[(size_t)k * nmu + m].scale;
      e.win = (uint32_t)std::max(nsu, 0) | (uint32_t)std::max(ntu, 0) << 8 | (uint32_t)(k == c.K - 1) << 16 |
              (uint32_t)k << 17;
      e.mu = m;
      if (nds <= 0 || ndt <= 0 || nc <= 0 || nr <= 0) continue;
      e.off = (int32_t)tab;
      e.y0 = r.z * d.det_ns + r.x;
      e.zo = (r.z - u.z) * nsu + (r.x - u.x);
      e.dims |= (uint32_t)nds << 16 | (uint32_t)ndt << 24;
      const int nds4 = (nds + 3) / 4 * 4;   // Bs rows and the windows' rows are padded to 4 floats
      const int n = nc * nds4 + nr * ndt, n4 = (n + 3) / 4 * 4;
      tab += n4;
      tab_max = std::max(tab_max, n4);
      w_max = std::max(w_max, nr * nds4);
      y_max = std::max(y_max, nds4 * ndt);
      if (tab >= (1LL << 31))
        return set_error(LT_EUNSUPPORTED, "camera %d: stage-two transport table beyond 2^31 entries", idx);
    }
  }
  auto up4 = [](int v) { return (std::max(v, 1) + 3) / 4 * 4; };
  s2.tab_max = up4(tab_max);
  s2.row_max = up4(max_cols + 3);                  // a block row copied in 16-byte chunks, shifted by up to 3
  s2.pix_max = up4(std::max(max_rows, 1) * s2.row_max);
  s2.w_max = up4(w_max);
  s2.z_max = up4(z_max);
  s2.y_max = up4(y_max);
  // per warp: a ring of kS2Ring descriptors (8 floats each), then the buffers
  s2.fwd_warp_floats = kS2Ring * 8 + 2 * s2.tab_max + 2 * s2.pix_max + 16 + s2.w_max + s2.z_max;
  s2.adj_warp_floats = kS2Ring * 8 + 2 * s2.tab_max + 2 * s2.y_max + 32 + s2.w_max;
  if ((s = upload(desc, &c.d_s2desc, "stage-two descriptors")) != LT_OK) return s;
  if ((s = upload(bits, &c.d_s2bits, "lenslet ownership bits")) != LT_OK) return s;
  if ((s = upload(ivals, &c.d_s2ivals, "lenslet row intervals")) != LT_OK) return s;
  s2.ivals = c.d_s2ivals;
  s2.iv_ok = iv_ok;
  c.s2tab_floats = tab;
  {
    const size_t tb = (size_t)std::max<long long>(tab, 4) * sizeof(float);
    cudaError_t et = device_alloc((void**)&c.d_s2tab, tb);
    if (et != cudaSuccess) {
      c.d_s2tab = nullptr;
      return set_error(LT_ENOMEM, "cudaMalloc(stage-two transport table, %zu bytes): %s", tb, cudaGetErrorString(et));
    }
  }
  s2.desc = c.d_s2desc;
  s2.bits = c.d_s2bits;
  s2.wtab = c.d_s2tab;
  int dev = 0;
  cudaError_t et = cudaGetDevice(&dev);
  if (et == cudaSuccess) et = cudaDeviceGetAttribute(&s2.sms, cudaDevAttrMultiProcessorCount, dev);
  if (et == cudaSuccess) et = lt::stage2_occupancy(s2, false, &s2.fwd_per_sm);
  if (et == cudaSuccess) et = lt::stage2_occupancy(s2, true, &s2.adj_per_sm);
  if (et == cudaSuccess && (s2.fwd_per_sm < 1 || s2.adj_per_sm < 1))
    return set_error(LT_EUNSUPPORTED, "camera %d: stage-two kernels do not fit an SM (%zu / %zu bytes of shared memory)",
                     idx, lt::stage2_smem_bytes(s2, false), lt::stage2_smem_bytes(s2, true));
  if (et == cudaSuccess) et = lt::launch_stage2_tables(s2, c.d_s2tab, 0);
  if (et == cudaSuccess) et = cudaStreamSynchronize(0);
  if (et != cudaSuccess) return cuda_error(et, "stage-two transport table");
  return LT_OK;
}

// Rotated view of the volume for a camera with yaw (Sec. III-A): quarter
// turns, then D = diag(cos, 1, 1/cos) rescales the voxels and the shears
// S_z (z += b x, b = -sin cos) and S_x (x += a z, a = tan) are applied as LS
// re-projections onto grids padded to hold every sheared cell.
static lt_status plan_rotation(const lt_volume_desc& v, CameraPlan& c, int frames, int idx) {
  const double yaw = c.desc.yaw;
  const double q = std::floor(yaw / (M_PI / 2) + 0.5);   // half up at exactly 45 degrees
  const double tr = yaw - q * (M_PI / 2);
  int nq = (int)(((long long)q % 4 + 4) % 4);
  RotParam& r = c.rot;
  r.nq = nq;
  r.nx = v.nx;
  r.ny = v.ny;
  r.nz = v.nz;
  const bool odd = nq % 2 == 1;
  r.nxp = odd ? v.nz : v.nx;
  r.nzp = odd ? v.nx : v.nz;
  const double dxp = odd ? v.dz : v.dx, dzp = odd ? v.dx : v.dz;
  const double cs = std::cos(tr), sn = std::sin(tr);
  const double a = sn / cs, b = -sn * cs;
  const double dxr = dxp / cs, dzr = dzp * cs;    // voxel sizes after D
  r.pz = (int)std::ceil(std::fabs(b) * r.nxp * dxr / 2.0 / dzr) + 1;
  r.nzr = r.nzp + 2 * r.pz;
  r.px = (int)std::ceil(std::fabs(a) * r.nzr * dzr / 2.0 / dxr) + 1;
  r.nxr = r.nxp + 2 * r.px;
  r.bz = (float)(b * dxr / dzr);
  r.betaz = std::fabs(r.bz);
  r.ax = (float)(a * dzr / dxr);
  r.betax = std::fabs(r.ax);
  r.wz = (int)std::floor(2.0 + r.betaz) + 4;
  r.wx = (int)std::floor(2.0 + r.betax) + 4;
  c.vol_c.nx = r.nxr;
  c.vol_c.ny = v.ny;
  c.vol_c.nz = r.nzr;
  c.vol_c.dx = dxr;
  c.vol_c.dy = v.dy;
  c.vol_c.dz = dzr;
  c.nvox_c = (int64_t)r.nxr * v.ny * r.nzr;
  if (c.desc.d_obj - 0.5 * r.nzr * dzr <= 0.0)
    return set_error(LT_EINVAL, "camera %d: the rotated volume reaches the main lens", idx);
  const size_t brz = (size_t)frames * r.nzr * v.ny * r.nxp * sizeof(float);
  const size_t bxr = (size_t)frames * c.nvox_c * sizeof(float);
  if (device_alloc((void**)&c.d_rz, brz) != cudaSuccess || device_alloc((void**)&c.d_xr, bxr) != cudaSuccess)
    return set_error(LT_ENOMEM, "camera %d: rotated-view scratch (%zu + %zu bytes)", idx, brz, bxr);
  if (r.wz > 16 || r.wx > 64)
    return set_error(LT_EUNSUPPORTED, "camera %d: voxel aspect ratio too large for the shear passes "
                     "(windows %d, %d)", idx, r.wz, r.wx);
  r.nwz = r.wz <= 8 ? 8 : 16;
  if (device_alloc((void**)&r.tz, (size_t)r.nxp * r.nwz * sizeof(float)) != cudaSuccess ||
      device_alloc((void**)&r.jz, (size_t)r.nxp * sizeof(int32_t)) != cudaSuccess ||
      device_alloc((void**)&r.tx, (size_t)r.nzr * r.wx * sizeof(float)) != cudaSuccess ||
      device_alloc((void**)&r.jx, (size_t)r.nzr * sizeof(int32_t)) != cudaSuccess)
    return set_error(LT_ENOMEM, "camera %d: shear tables", idx);
  cudaError_t e = launch_shear_tables(r, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) return cuda_error(e, "shear tables");
  // Window spread of each 32-column tile, from the offsets just tabulated:
  // it sizes the staged source rows of the transposed z adjoint.
  std::vector<int32_t> jz(r.nxp);
  e = cudaMemcpy(jz.data(), r.jz, jz.size() * sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(e, "shear table offsets");
  r.djz = 0;
  for (int c0 = 0; c0 < r.nxp; c0 += 32) {
    const auto first = jz.begin() + c0, last = jz.begin() + std::min(c0 + 32, r.nxp);
    r.djz = std::max(r.djz, *std::max_element(first, last) - *std::min_element(first, last));
  }
  return LT_OK;
}

// General orientation (pitch and/or roll, Sec. III-A, eq. rot,decomp):
// Theta = R_y(yaw) R_x(pitch) R_z(roll) = P Theta_r with P the proper signed
// permutation of largest trace(P^T Theta) (first of a fixed enumeration on
// ties; residue below 1e-12 zeroed), Theta_r = D S_z S_x S_y by elimination,
// voxel sizes s / D on the permuted grid, then one shear pass per axis
// (z: a x + b y, x: c y + d z, y: e x + f z), each padding its axis by
// ceil((|s1| n_u du + |s2| n_v dv) / 2 / dt) + 1 (none for a zero pass).
static lt_status plan_rotation_general(const lt_volume_desc& v, CameraPlan& c, int frames, int idx) {
  const lt_camera_desc& d = c.desc;
  auto mul = [](const double A[3][3], const double B[3][3], double C[3][3]) {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double acc = 0.0;
        for (int k = 0; k < 3; ++k) acc += A[i][k] * B[k][j];
        C[i][j] = acc;
      }
  };
  const double cy = std::cos(d.yaw), sy = std::sin(d.yaw), cp = std::cos(d.pitch), sp = std::sin(d.pitch);
  const double cr = std::cos(d.roll), sr = std::sin(d.roll);
  const double Ry[3][3] = {{cy, 0, sy}, {0, 1, 0}, {-sy, 0, cy}};
  const double Rx[3][3] = {{1, 0, 0}, {0, cp, -sp}, {0, sp, cp}};
  const double Rz[3][3] = {{cr, -sr, 0}, {sr, cr, 0}, {0, 0, 1}};
  double T1[3][3], T[3][3];
  mul(Ry, Rx, T1);
  mul(T1, Rz, T);
  static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  double best = -1e300;
  int bp = 0, bs[3] = {1, 1, 1};
  for (int pi = 0; pi < 6; ++pi)
    for (int sx = 1; sx >= -1; sx -= 2)
      for (int syy = 1; syy >= -1; syy -= 2)
        for (int sz = 1; sz >= -1; sz -= 2) {
          const int sg[3] = {sx, syy, sz};
          double P[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
          for (int m = 0; m < 3; ++m) P[m][perms[pi][m]] = sg[m];
          const double det = P[0][0] * (P[1][1] * P[2][2] - P[1][2] * P[2][1]) -
                             P[0][1] * (P[1][0] * P[2][2] - P[1][2] * P[2][0]) +
                             P[0][2] * (P[1][0] * P[2][1] - P[1][1] * P[2][0]);
          if (det < 0.5) continue;
          double tr = 0.0;   // trace(P^T T) = sum_m P[m][k_m] T[m][k_m]
          for (int m = 0; m < 3; ++m) tr += sg[m] * T[m][perms[pi][m]];
          if (tr > best + 1e-12) {
            best = tr;
            bp = pi;
            for (int m = 0; m < 3; ++m) bs[m] = sg[m];
          }
        }
  // Tr = P^T T: row k of Tr = sum_m P[m][k] T[m][.] -> the m with k_m = k
  double Tr[3][3];
  for (int m = 0; m < 3; ++m)
    for (int j = 0; j < 3; ++j) Tr[perms[bp][m]][j] = bs[m] * T[m][j];
  for (auto& row : Tr)
    for (double& e : row)
      if (std::fabs(e) < 1e-12) e = 0.0;
  const double Dy = Tr[1][1], e_ = Tr[1][0] / Dy, f_ = Tr[1][2] / Dy;
  const double Dx = Tr[0][0] - Tr[0][1] * e_, c_ = Tr[0][1] / Dx, d_ = Tr[0][2] / Dx - c_ * f_;
  const double u_ = Tr[2][0] - Tr[2][1] * e_, w_ = Tr[2][1] - u_ * c_;
  const double Dz = Tr[2][2] - u_ * (d_ + c_ * f_) - w_ * f_;
  const double a_ = u_ / Dz, b_ = w_ / Dz;
  if (!(Dx > 0 && Dy > 0 && Dz > 0))
    return set_error(LT_EINVAL, "camera %d: rotation factorisation failed", idx);
  GenRot& g = c.grot;
  g.nx = v.nx;
  g.ny = v.ny;
  g.nz = v.nz;
  const int n_src[3] = {v.nx, v.ny, v.nz};
  const double s_src[3] = {v.dx, v.dy, v.dz};
  double s_new[3];
  for (int m = 0; m < 3; ++m) {
    g.km[m] = perms[bp][m];
    g.sg[m] = bs[m];
    g.np[g.km[m]] = n_src[m];
    s_new[g.km[m]] = s_src[m];
  }
  const double Dg[3] = {Dx, Dy, Dz};
  double srr[3];
  for (int k = 0; k < 3; ++k) srr[k] = s_new[k] / Dg[k];
  const double coef[3][2] = {{a_, b_}, {c_, d_}, {e_, f_}};
  const int axes[3] = {2, 0, 1};   // z, x, y passes
  int dims[3] = {g.np[0], g.np[1], g.np[2]};
  size_t bytes[3];
  for (int k = 0; k < 3; ++k) {
    ShearPass& ps = g.pass[k];
    ps.axis = axes[k];
    ps.n0 = dims[0];
    ps.n1 = dims[1];
    ps.n2 = dims[2];
    bytes[k] = (size_t)frames * dims[0] * dims[1] * dims[2] * sizeof(float);   // this pass's input
    const int ua = ps.axis == 0 ? 1 : 0, va = ps.axis == 2 ? 1 : 2;
    ps.nu = dims[ua];
    ps.nv = dims[va];
    const double s1 = coef[k][0], s2 = coef[k][1];
    ps.active = !(s1 == 0.0 && s2 == 0.0);
    const double dt = srr[ps.axis], du = srr[ua], dv = srr[va];
    if (ps.active) {
      ps.pad = (int)std::ceil((std::fabs(s1) * ps.nu * du + std::fabs(s2) * ps.nv * dv) / 2.0 / dt) + 1;
      ps.nw = (int)std::floor(2.0 + std::fabs(s1) * du / dt + std::fabs(s2) * dv / dt) + 4;
      if (ps.nw > 64) return set_error(LT_EUNSUPPORTED, "camera %d: shear window %d too wide", idx, ps.nw);
      const size_t ncol = (size_t)ps.nu * ps.nv;
      if (device_alloc((void**)&c.d_gtab[k], ncol * ps.nw * sizeof(float)) != cudaSuccess ||
          device_alloc((void**)&c.d_gjo[k], ncol * sizeof(int32_t)) != cudaSuccess)
        return set_error(LT_ENOMEM, "camera %d: shear tables", idx);
      ps.tab = c.d_gtab[k];
      ps.jo = c.d_gjo[k];
      cudaError_t e = launch_shear_pass_table(ps, s1, s2, du / dt, dv / dt, c.d_gtab[k], c.d_gjo[k], 0);
      if (e != cudaSuccess) return cuda_error(e, "shear tables");
      dims[ps.axis] += 2 * ps.pad;
    } else {
      ps.pad = 0;
      ps.nw = 0;
    }
  }
  for (int k = 0; k < 3; ++k)
    if (device_alloc((void**)&c.d_gb[k], bytes[k]) != cudaSuccess)
      return set_error(LT_ENOMEM, "camera %d: rotated-view scratch", idx);
  c.vol_c.nx = dims[0];
  c.vol_c.ny = dims[1];
  c.vol_c.nz = dims[2];
  c.vol_c.dx = srr[0];
  c.vol_c.dy = srr[1];
  c.vol_c.dz = srr[2];
  c.nvox_c = (int64_t)dims[0] * dims[1] * dims[2];
  if (d.d_obj - 0.5 * dims[2] * srr[2] <= 0.0)
    return set_error(LT_EINVAL, "camera %d: the rotated volume reaches the main lens", idx);
  if (device_alloc((void**)&c.d_xr, (size_t)frames * c.nvox_c * sizeof(float)) != cudaSuccess)
    return set_error(LT_ENOMEM, "camera %d: rotated-view scratch", idx);
  cudaError_t e = cudaStreamSynchronize(0);
  return e == cudaSuccess ? LT_OK : cuda_error(e, "shear tables");
}

static lt_status plan_camera(const lt_volume_desc& v0, const lt_camera_desc& src, int frames,
                             CameraPlan& c, int idx) {
  c.desc = src;
  c.vol_c = v0;
  c.nvox_c = (int64_t)v0.nx * v0.ny * v0.nz;
  c.general = src.pitch != 0.0 || src.roll != 0.0;
  c.rotated = src.yaw != 0.0 || c.general;
  if (c.rotated) {
    lt_status s = c.general ? plan_rotation_general(v0, c, frames, idx) : plan_rotation(v0, c, frames, idx);
    if (s != LT_OK) return s;
  }
  const lt_volume_desc& v = c.vol_c;
  if (src.kind == LT_CAM_PLENOPTIC) {
    c.focal.assign(src.mla_focal, src.mla_focal + (size_t)src.mla_ns * src.mla_nt);
    c.desc.mla_focal = nullptr;
  }
  // angular cells tiling [-r, r]^2, kept when the centre is inside the disc
  const double r = src.r_main;
  const double d0s = 2.0 * r / src.ks, d0t = 2.0 * r / src.kt;
  for (int kt = 0; kt < src.kt; ++kt)
    for (int ks = 0; ks < src.ks; ++ks) {
      const double sk = -r + (ks + 0.5) * d0s, tk = -r + (kt + 0.5) * d0t;
      if (sk * sk + tk * tk < r * r) c.cells.push_back({sk, tk, d0s, d0t});
    }
  c.K = (int)c.cells.size();
  if (c.K == 0) return set_error(LT_EINVAL, "camera %d: no angular cell inside the aperture", idx);
  c.M = (int64_t)src.det_ns * src.det_nt;
  if (src.kind == LT_CAM_SINGLE)
    return plan_slices(v, c, src.d_lens_det, src.det_ns, src.det_nt, src.det_ps, src.det_pt, 1.0, frames, idx);
  // plenoptic: V^a = (Da_s D0_s / D_mum)(Da_t D0_t / D_mum)
  const double va = (src.arr_ps * d0s / src.d_lens_mla) * (src.arr_pt * d0t / src.d_lens_mla);
  lt_status s = plan_slices(v, c, src.d_lens_mla, src.arr_ns, src.arr_nt, src.arr_ps, src.arr_pt,
                            1.0 / va, frames, idx);
  if (s != LT_OK) return s;
  s = plan_stage_two(c, frames, idx);
  c.desc.arr_mask = nullptr;   // copied into the plan; the caller's array is not kept
  return s;
}

// Chunks of the brick-staged forward: a camera whose tiles meeting the
// volume (times frames) number at most a quarter of the CTAs the kernel
// keeps resident splits each tile's slices into up to 4 parts, so that more
// SMs share its work (measured: splitting the items of larger workloads
// costs more in combining the partial tiles than it gains in balance);
// the partial tiles and per-tile counts live in plan scratch sized for the
// largest launch (a window-class group of the batched forward, or one
// camera).
static lt_status plan_chunks(lt_plan* p) {
  const long long slots = 4LL * p->sms;   // resident CTAs of the brick-staged kernel
  long long need_part = 0, need_count = 0;
  for (auto& c : p->cams) {
    c.tma_chunks = 1;
    if (c.tma_nb == 0) continue;
    const long long units = (long long)c.n_real_items * p->frames;
    if (units > 0 && 4 * units <= slots) c.tma_chunks = (int)std::min<long long>(4, slots / units);
    if (c.tma_chunks > 1) {
      need_part = std::max(need_part, units * c.tma_chunks);
      need_count = std::max(need_count, units);
    }
  }
  for (int g = 0; g < kForwardGroups; ++g) {
    if (g % 3 == 2 || p->class_count[g] == 0) continue;
    int cmax = 1;
    for (auto& c : p->cams)
      if (c.tma_nb != 0 && forward_group_kind(c.tma_nb) == g % 3 &&
          window_class(std::max(c.wmax_s, c.wmax_t)) == kFwdClasses[g / 3])
        cmax = std::max(cmax, c.tma_chunks);
    if (cmax > 1) {
      const long long units = (long long)p->class_real[g] * p->frames;
      need_part = std::max(need_part, units * cmax);
      need_count = std::max(need_count, units);
    }
  }
  if (need_part == 0) return LT_OK;
  if (device_alloc((void**)&p->d_chunk_part, (size_t)need_part * 1024 * sizeof(float)) != cudaSuccess ||
      device_alloc((void**)&p->d_chunk_count, (size_t)need_count * sizeof(int)) != cudaSuccess)
    return set_error(LT_ENOMEM, "cudaMalloc(forward chunk scratch)");
  cudaError_t e = cudaMemset(p->d_chunk_count, 0, (size_t)need_count * sizeof(int));
  return e == cudaSuccess ? LT_OK : cuda_error(e, "forward chunk scratch");
}

extern "C" lt_status lt_plan_create(const lt_volume_desc* vol, const lt_camera_desc* cams,
                                    int32_t n_cams, int32_t n_frames, lt_plan** out) {
  clear_error();
  if (!out) return set_error(LT_EINVAL, "out is NULL");
  *out = nullptr;
  lt_status s = validate_volume(vol);
  if (s != LT_OK) return s;
  if (n_cams <= 0 || !cams) return set_error(LT_EINVAL, "need at least one camera");
  if (n_frames <= 0) return set_error(LT_EINVAL, "n_frames must be positive");
  for (int c = 0; c < n_cams; ++c)
    if ((s = validate_camera(vol, &cams[c], c)) != LT_OK) return s;
  lt_plan* p = new (std::nothrow) lt_plan();
  if (!p) return set_error(LT_ENOMEM, "host allocation failed");
  p->vol = *vol;
  p->frames = n_frames;
  p->nvox = (int64_t)vol->nx * vol->ny * vol->nz;
  cudaGetDevice(&p->device);
  p->cams.resize(n_cams);
  int64_t off = 0;
  for (int c = 0; c < n_cams; ++c) {
    s = plan_camera(*vol, cams[c], n_frames, p->cams[c], c);
    if (s != LT_OK) {
      lt_plan_destroy(p);
      return s;
    }
    p->cams[c].offset = off;
    off += p->cams[c].M;
  }
  p->m_total = off;
  {
    std::vector<int4> all;
    for (int g = 0; g < kForwardGroups; ++g) {
      const size_t start = all.size();
      for (auto& c : p->cams)
        if (window_class(std::max(c.wmax_s, c.wmax_t)) == kFwdClasses[g / 3] && forward_group_kind(c.tma_nb) == g % 3)
          all.insert(all.end(), c.h_items.begin(), c.h_items.end());
      std::stable_sort(all.begin() + start, all.end(), [](const int4& a, const int4& b) { return a.w > b.w; });
      p->class_begin[g] = (int)start;
      p->class_count[g] = (int)(all.size() - start);
      p->class_real[g] = (int)std::count_if(all.begin() + start, all.end(), [](const int4& a) { return a.w > 0; });
    }
    p->n_items = (int)all.size();
    s = upload(all, &p->d_items, "forward work items");
    if (s == LT_OK && device_alloc((void**)&p->d_counter, sizeof(int)) != cudaSuccess)
      s = set_error(LT_ENOMEM, "cudaMalloc(work counter)");
    cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
    if (s == LT_OK) s = plan_chunks(p);
    if (s != LT_OK) {
      lt_plan_destroy(p);
      return s;
    }
  }
  *out = p;
  return LT_OK;
}

extern "C" lt_status lt_plan_destroy(lt_plan* plan) {
  if (!plan) return LT_OK;
  cudaDeviceSynchronize();
  for (auto& c : plan->cams) free_camera(c);
  cudaFree(plan->d_items);
  cudaFree(plan->d_counter);
  cudaFree(plan->d_chunk_part);
  cudaFree(plan->d_chunk_count);
  delete plan;
  return LT_OK;
}

extern "C" lt_status lt_plan_sizes(const lt_plan* plan, int64_t* n_vox, int64_t* det_offsets) {
  clear_error();
  if (!plan) return set_error(LT_EINVAL, "plan is NULL");
  if (n_vox) *n_vox = plan->nvox;
  if (det_offsets) {
    for (size_t c = 0; c < plan->cams.size(); ++c) det_offsets[c] = plan->cams[c].offset;
    det_offsets[plan->cams.size()] = plan->m_total;
  }
  return LT_OK;
}

extern "C" lt_status lt_camera_cells(const lt_plan* plan, int32_t cam, int32_t* n_cells) {
  clear_error();
  if (!plan || cam < 0 || cam >= (int)plan->cams.size() || !n_cells)
    return set_error(LT_EINVAL, "bad plan/camera/out argument");
  *n_cells = plan->cams[cam].K;
  return LT_OK;
}

extern "C" lt_status lt_camera_grid(const lt_plan* plan, int32_t cam, lt_volume_desc* grid) {
  clear_error();
  if (!plan || cam < 0 || cam >= (int)plan->cams.size() || !grid)
    return set_error(LT_EINVAL, "bad plan/camera/out argument");
  *grid = plan->cams[cam].vol_c;
  return LT_OK;
}

extern "C" lt_status lt_rotate_volume(lt_plan* plan, int32_t cam, const float* x, float* xc, void* stream) {
  clear_error();
  if (!plan || cam < 0 || cam >= (int)plan->cams.size() || !x || !xc)
    return set_error(LT_EINVAL, "bad plan/camera/pointer argument");
  CameraPlan& c = plan->cams[cam];
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = !c.rotated ? cudaMemcpyAsync(xc, x, (size_t)plan->frames * plan->nvox * sizeof(float),
                                               cudaMemcpyDeviceToDevice, st)
                  : c.general ? launch_grot_forward(x, c.d_gb[0], c.d_gb[1], c.d_gb[2], xc, c.grot, plan->frames, st)
                              : launch_rotate_forward(x, c.d_rz, xc, c.rot, plan->frames, st);
  return e == cudaSuccess ? LT_OK : cuda_error(e, "rotate volume");
}

extern "C" lt_status lt_rotate_volume_adjoint(lt_plan* plan, int32_t cam, const float* xc, float* x,
                                              int32_t accumulate, void* stream) {
  clear_error();
  if (!plan || cam < 0 || cam >= (int)plan->cams.size() || !x || !xc)
    return set_error(LT_EINVAL, "bad plan/camera/pointer argument");
  CameraPlan& c = plan->cams[cam];
  cudaStream_t st = (cudaStream_t)stream;
  if (c.rotated) {
    cudaError_t e = c.general ? launch_grot_adjoint(xc, c.d_gb[0], c.d_gb[1], c.d_gb[2], x, c.grot, plan->frames,
                                                    accumulate, st)
                              : launch_rotate_adjoint(xc, c.d_rz, x, c.rot, plan->frames, accumulate, st);
    return e == cudaSuccess ? LT_OK : cuda_error(e, "rotate volume adjoint");
  }
  const long long n = (long long)plan->frames * plan->nvox;
  if (!accumulate) {
    cudaError_t e = cudaMemcpyAsync(x, xc, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? LT_OK : cuda_error(e, "rotate volume adjoint");
  }
  cudaError_t e = launch_add_inplace(x, xc, n, st);
  return e == cudaSuccess ? LT_OK : cuda_error(e, "rotate volume adjoint");
}

// ---------------------------------------------------------------------------
// analytic work counts
// ---------------------------------------------------------------------------

// For target pixels [i0, i1] of a footprint, the number of source cells in
// [0, n_src) each footprint overlaps (open interval (xi - Q, xi + Q)),
// summed (nnz) and the number of pixels with at least one (hits).
// With `tile` > 0, *span also receives the sum over consecutive blocks of
// `tile` target pixels of the number of source cells the block's footprints
// touch together.
static void count_cells(const lt::Footprint& f, long long i0, long long i1, long long c_lo,
                        long long c_hi, long long* nnz, long long* hits, int tile = 0,
                        long long* span = nullptr) {
  *nnz = 0;
  *hits = 0;
  if (span) *span = 0;
  long long blo = LLONG_MAX, bhi = LLONG_MIN;
  for (long long i = i0; i <= i1; ++i) {
    const double xi = f.C0 + f.C1 * (double)i;
    long long jl = (long long)std::floor(xi - f.Q - 0.5) + 1;
    long long jh = (long long)std::ceil(xi + f.Q + 0.5) - 1;
    jl = std::max(jl, c_lo);
    jh = std::min(jh, c_hi);
    if (jh >= jl) {
      *nnz += jh - jl + 1;
      *hits += 1;
      blo = std::min(blo, jl);
      bhi = std::max(bhi, jh);
    }
    if (span && (i == i1 || (i - i0 + 1) % tile == 0)) {
      if (bhi >= blo) *span += bhi - blo + 1;
      blo = LLONG_MAX;
      bhi = LLONG_MIN;
    }
  }
}

extern "C" lt_status lt_camera_stats_get(const lt_plan* plan, int32_t cam, lt_camera_stats* out) {
  clear_error();
  if (!plan || !out || cam < 0 || cam >= (int)plan->cams.size())
    return set_error(LT_EINVAL, "bad plan/camera/out argument");
  const CameraPlan& c = plan->cams[cam];
  const lt_camera_desc& d = c.desc;
  const lt_volume_desc& v = c.vol_c;
  const bool plen = d.kind == LT_CAM_PLENOPTIC;
  const int tns = plen ? d.arr_ns : d.det_ns, tnt = plen ? d.arr_nt : d.det_nt;
  const double tps = plen ? d.arr_ps : d.det_ps, tpt = plen ? d.arr_pt : d.det_pt;
  const double d_img = plen ? d.d_lens_mla : d.d_lens_det;
  lt_camera_stats st{};
  st.n_cells = c.K;
  st.stage1_samples = (int64_t)tns * tnt * c.K * v.nz;
  for (int k = 0; k < c.K; ++k)
    for (int n = 0; n < v.nz; ++n) {
      Row P, L;
      slice_rows(d.d_obj + centre(n, v.nz, v.dz), d_img, d.f_main, &P, &L);
      Footprint fs, ft;
      footprint(L, P, c.cells[k].sk, c.cells[k].d0s, centre(0, tns, tps), tps, centre(0, v.nx, v.dx), v.dx,
                d.basis, &fs);
      footprint(L, P, c.cells[k].tk, c.cells[k].d0t, centre(0, tnt, tpt), tpt, centre(0, v.ny, v.dy), v.dy,
                d.basis, &ft);
      long long ns_, hs, nt_, ht, span_s, span_t;
      count_cells(fs, 0, tns - 1, 0, v.nx - 1, &ns_, &hs, kBeamTileS, &span_s);
      count_cells(ft, 0, tnt - 1, 0, v.ny - 1, &nt_, &ht, kBeamTileT, &span_t);
      st.stage1_nnz += ns_ * nt_;
      st.hit_samples += hs * ht;
      st.stage1_tile_voxels += span_s * span_t;
    }
  if (plen) {
    st.stage2_samples = (int64_t)d.det_ns * d.det_nt * c.K;
    const int mns = d.mla_ns, mnt = d.mla_nt;
    std::vector<int2> cols(mns), rows(mnt);
    cudaMemcpy(cols.data(), c.d_cols, mns * sizeof(int2), cudaMemcpyDeviceToHost);
    cudaMemcpy(rows.data(), c.d_rows, mnt * sizeof(int2), cudaMemcpyDeviceToHost);
    for (int k = 0; k < c.K; ++k)
      for (int mt = 0; mt < mnt; ++mt)
        for (int ms = 0; ms < mns; ++ms) {
          if (cols[ms].y <= cols[ms].x || rows[mt].y <= rows[mt].x) continue;
          const double f = c.focal[(size_t)mt * mns + ms];
          Row Ps, Ls, Pt, Lt;
          lenslet_rows(d.d_mla_det, d.d_lens_mla, f, centre(ms, mns, d.mla_pitch), &Ps, &Ls);
          lenslet_rows(d.d_mla_det, d.d_lens_mla, f, centre(mt, mnt, d.mla_pitch), &Pt, &Lt);
          Footprint fs, ft;
          footprint(Ls, Ps, c.cells[k].sk, c.cells[k].d0s, centre(0, d.det_ns, d.det_ps), d.det_ps,
                    centre(0, d.arr_ns, d.arr_ps), d.arr_ps, d.basis, &fs);
          footprint(Lt, Pt, c.cells[k].tk, c.cells[k].d0t, centre(0, d.det_nt, d.det_pt), d.det_pt,
                    centre(0, d.arr_nt, d.arr_pt), d.arr_pt, d.basis, &ft);
          long long ns_, hs, nt_, ht;
          count_cells(fs, 0, d.det_ns - 1, cols[ms].x, cols[ms].y - 1, &ns_, &hs);
          count_cells(ft, 0, d.det_nt - 1, rows[mt].x, rows[mt].y - 1, &nt_, &ht);
          st.stage2_nnz += ns_ * nt_;
        }
  }
  st.ray_samples = st.stage1_samples + st.stage2_samples;
  st.forward_brick = (int64_t)c.tma_bx * c.tma_by;
  st.adjoint_box = (int64_t)c.adj_bx * c.adj_by;
  st.adjoint_chunk = c.adj_sc;
  st.forward_band = c.tma_nb == 4 ? 1 : 0;
  *out = st;
  return LT_OK;
}

// ---------------------------------------------------------------------------
// operators
// ---------------------------------------------------------------------------

namespace lt {

static cudaError_t rotate_fwd(const CameraPlan& c, const float* x, float* xr, int frames, cudaStream_t st) {
  return c.general ? launch_grot_forward(x, c.d_gb[0], c.d_gb[1], c.d_gb[2], xr, c.grot, frames, st)
                   : launch_rotate_forward(x, c.d_rz, xr, c.rot, frames, st);
}

static cudaError_t rotate_adj(const CameraPlan& c, const float* g_xr, float* x, int frames, int accumulate,
                              cudaStream_t st) {
  return c.general ? launch_grot_adjoint(g_xr, c.d_gb[0], c.d_gb[1], c.d_gb[2], x, c.grot, frames, accumulate, st)
                   : launch_rotate_adjoint(g_xr, c.d_rz, x, c.rot, frames, accumulate, st);
}

// The grid this camera sees: x itself, or its rotated view (into c.d_xr).
static lt_status to_camera_grid(lt_plan* p, CameraPlan& c, const float* x, const float** xc, cudaStream_t st) {
  if (!c.rotated) {
    *xc = x;
    return LT_OK;
  }
  cudaError_t e = rotate_fwd(c, x, c.d_xr, p->frames, st);
  if (e != cudaSuccess) return cuda_error(e, "rotated view");
  *xc = c.d_xr;
  return LT_OK;
}

// Description of camera c's slice -> plane transport for a batched launch:
// camera-grid volume xc, forward output `out` / adjoint input `in`, both with
// frame stride out_fs.
static BeamCam beam_cam(const CameraPlan& c, const float* xc, float* out, const float* in, long long out_fs,
                        SubsetSel sel = SubsetSel{}) {
  const bool plen = c.desc.kind == LT_CAM_PLENOPTIC;
  BeamCam b{};
  b.x = xc;
  b.out = out;
  b.in = in;
  b.prm = c.d_slice;
  b.mask = plen ? c.d_mask : nullptr;
  b.srange = c.d_srange;
  b.trange = c.d_trange;
  b.x_fs = c.nvox_c;
  b.out_fs = out_fs;
  b.nx = c.vol_c.nx;
  b.ny = c.vol_c.ny;
  b.nz = c.vol_c.nz;
  b.ns = plen ? c.desc.arr_ns : c.desc.det_ns;
  b.nt = plen ? c.desc.arr_nt : c.desc.det_nt;
  b.K = c.K;
  b.per_cell = plen ? 1 : 0;
  b.tiles_s = c.tiles_s;
  b.tiles_t = c.tiles_t;
  b.wis = c.wimax_s;
  b.wit = c.wimax_t;
  b.sub_n = sel.n;
  b.sub_s = sel.s;
  return b;
}

// One persistent forward launch over `items` of the cameras in b (cps[i] is
// the plan of b.cam[i]).  The brick-staged TMA kernel runs when the items
// belong to cameras the planner sized bricks for (staged_nb = their tma_nb,
// 0: none), the plan's variant selects it and every source is 16-byte
// aligned; otherwise the direct kernel of the variant (variant kTmaVariant
// falls back to the default direct variant).
static lt_status run_forward(lt_plan* p, const BeamBatch& b, CameraPlan* const* cps, const int4* items,
                             int n_items, int n_real, int wclass, int staged_nb, cudaStream_t st) {
  if (staged_nb > 0 && p->fwd_variant == kTmaVariant && wclass <= 4 && tma_forward_available()) {
    static_assert(sizeof(TmaBatch) % 64 == 0, "tensor maps stay 64-byte aligned");
    TmaBatch tb;
    std::memset(&tb, 0, sizeof(tb));
    bool ok = true;
    int brick = 0, max_by = 1, chunks = 1;
    for (int i = 0; i < b.n_cams && ok; ++i) {
      const CameraPlan& c = *cps[i];
      const BeamCam& bc = b.cam[i];
      if (c.tma_nb != staged_nb || window_class(std::max(c.wmax_s, c.wmax_t)) != wclass)
        continue;   // none of its items are in this launch
      ok = bc.x_fs == (long long)bc.nx * bc.ny * bc.nz &&
           tma_encode_volume(&tb.map[i], bc.x, bc.nx, bc.ny, bc.nz * b.frames, c.tma_bx, c.tma_by);
      if (!ok) break;
      tb.stab[i] = c.d_stab;
      tb.ttab[i] = c.d_ttab;
      tb.chunks[i] = c.tma_chunks;
      chunks = std::max(chunks, c.tma_chunks);
      tb.bx[i] = c.tma_bx;
      tb.by[i] = c.tma_by;
      brick = std::max(brick, c.tma_bx * c.tma_by);
      max_by = std::max(max_by, c.tma_by);
    }
    if (ok) {
      const int tsz = tma_forward_tsz(max_by);
      const bool band = staged_nb == 4;
      const int occ = tma_forward_occupancy(wclass, band, brick, tsz);
      if (occ > 0) {
        cudaError_t e = launch_beam_forward_tma(b, tb, items, n_items, n_real, p->d_counter, wclass, band, brick, tsz,
                                                chunks, p->d_chunk_part, p->d_chunk_count, p->sms * occ, st);
        return e == cudaSuccess ? LT_OK : cuda_error(e, "beam forward (TMA bricks)");
      }
    }
  }
  const int variant = p->fwd_variant == kTmaVariant ? kDefaultDirectVariant : p->fwd_variant;
  const int ctas = p->sms * beam_forward_occupancy(wclass, variant);
  cudaError_t e = launch_beam_forward_batched(b, items, n_items, p->d_counter, wclass, variant, ctas, st);
  return e == cudaSuccess ? LT_OK : cuda_error(e, "beam forward");
}

static int cam_class(const CameraPlan& c) { return window_class(std::max(c.wmax_s, c.wmax_t)); }

// One gather-adjoint launch over the cameras of b (cps[i] is the plan of
// b.cam[i], all on one grid): the box-staged kernel when the plan selects
// it and every camera fits it (planner-sized boxes, 16-byte aligned input
// whose rows and plane strides are multiples of 4 floats), otherwise the
// direct gather kernel.
static lt_status run_adjoint(lt_plan* p, const BeamBatch& b, CameraPlan* const* cps, float* x, long long x_fs,
                             int accumulate, cudaStream_t st) {
  if (p->adj_variant == 1 && tma_forward_available()) {
    AdjBatch a;
    std::memset(&a, 0, sizeof(a));
    bool ok = true;
    for (int i = 0; i < b.n_cams && ok; ++i) {
      const CameraPlan& c = *cps[i];
      const BeamCam& bc = b.cam[i];
      const long long plane = (long long)bc.ns * bc.nt;
      ok = c.adj_bx > 0 && c.adj_sc == cps[0]->adj_sc && (!bc.per_cell || bc.out_fs == plane * bc.K) &&
           tma_encode_planes(&a.map[i], bc.in, bc.ns, bc.nt, b.frames * (bc.per_cell ? bc.K : 1),
                             bc.per_cell ? plane : bc.out_fs, c.adj_bx, c.adj_by);
      a.stab[i] = c.d_adj_s;
      a.ttab[i] = c.d_adj_t;
      a.ox[i] = c.d_adj_ox;
      a.oy[i] = c.d_adj_oy;
      a.bx[i] = c.adj_bx;
      a.by[i] = c.adj_by;
      a.zf[i] = bc.per_cell ? bc.K : 1;
      a.wqs[i] = c.wimax_s;
      a.wqt[i] = c.wimax_t;
      a.tiles_x[i] = (bc.nx + adjoint_tile_x() - 1) / adjoint_tile_x();
      a.tiles_y[i] = (bc.ny + adjoint_tile_y() - 1) / adjoint_tile_y();
      a.chunks[i] = (bc.nz + c.adj_sc - 1) / c.adj_sc;
    }
    if (ok) {
      cudaError_t e = launch_beam_adjoint_tma(b, a, cps[0]->adj_sc, x, x_fs, accumulate, st);
      return e == cudaSuccess ? LT_OK : cuda_error(e, "beam adjoint (TMA boxes)");
    }
  }
  cudaError_t e = launch_beam_adjoint_batched(b, x, x_fs, accumulate, st);
  return e == cudaSuccess ? LT_OK : cuda_error(e, "beam adjoint");
}

// Adjoint of one camera's slice -> plane transport from `in` back to x
// (through the transposed rotation for rotated cameras).
static lt_status beam_adjoint_to_volume(lt_plan* p, CameraPlan& c, const float* in, long long in_fs, float* x,
                                        int accumulate, cudaStream_t st, SubsetSel sel = SubsetSel{}) {
  BeamBatch b{};
  b.n_cams = 1;
  b.frames = p->frames;
  b.cam[0] = beam_cam(c, nullptr, nullptr, in, in_fs, sel);
  float* dst = c.rotated ? c.d_xr : x;
  CameraPlan* cps[1] = {&c};
  lt_status s = run_adjoint(p, b, cps, dst, c.nvox_c, c.rotated ? 0 : accumulate, st);
  if (s != LT_OK) return s;
  if (c.rotated) {
    cudaError_t e = rotate_adj(c, c.d_xr, x, p->frames, accumulate, st);
    if (e != cudaSuccess) return cuda_error(e, "rotated view adjoint");
  }
  return LT_OK;
}

lt_status stage1_forward(lt_plan* p, CameraPlan& c, const float* x, float* fa, long long fa_fs,
                         cudaStream_t st, SubsetSel sel) {
  const float* xc = nullptr;
  lt_status s = to_camera_grid(p, c, x, &xc, st);
  if (s != LT_OK) return s;
  BeamBatch b{};
  b.n_cams = 1;
  b.frames = p->frames;
  b.cam[0] = beam_cam(c, xc, fa, nullptr, fa_fs, sel);
  CameraPlan* cps[1] = {&c};
  return run_forward(p, b, cps, c.d_items, c.n_items, c.n_real_items, cam_class(c), c.tma_nb, st);
}

lt_status stage1_adjoint(lt_plan* p, CameraPlan& c, const float* fa, long long fa_fs, float* x,
                         int accumulate, cudaStream_t st, SubsetSel sel = SubsetSel{}) {
  return beam_adjoint_to_volume(p, c, fa, fa_fs, x, accumulate, st, sel);
}

static StageTwo stage_two(const CameraPlan& c, SubsetSel sel) {
  StageTwo s2 = c.s2;
  s2.sub_n = sel.n;
  s2.sub_s = sel.s;
  return s2;
}

lt_status camera_forward(lt_plan* p, int cam, const float* x, float* y, long long y_fs,
                         cudaStream_t st, SubsetSel sel) {
  CameraPlan& c = p->cams[cam];
  if (c.desc.kind == LT_CAM_SINGLE) return stage1_forward(p, c, x, y, y_fs, st, sel);
  const long long fa_fs = (long long)c.K * c.Na;
  lt_status s = stage1_forward(p, c, x, c.d_fa, fa_fs, st, sel);
  if (s != LT_OK) return s;
  cudaError_t e = launch_stage2_forward(c.d_fa, y, stage_two(c, sel), p->frames, fa_fs, y_fs, c.d_zbuf, st);
  return e == cudaSuccess ? LT_OK : cuda_error(e, "plenoptic stage 2");
}

lt_status camera_adjoint(lt_plan* p, int cam, const float* y, long long y_fs, float* x,
                         int accumulate, cudaStream_t st, SubsetSel sel) {
  CameraPlan& c = p->cams[cam];
  if (c.desc.kind == LT_CAM_SINGLE) return beam_adjoint_to_volume(p, c, y, y_fs, x, accumulate, st, sel);
  const long long fa_fs = (long long)c.K * c.Na;
  cudaError_t e = launch_stage2_adjoint(y, c.d_fa, stage_two(c, sel), p->frames, y_fs, fa_fs, st);
  if (e != cudaSuccess) return cuda_error(e, "plenoptic stage 2 adjoint");
  return stage1_adjoint(p, c, c.d_fa, fa_fs, x, accumulate, st, sel);
}

// Every camera at once: rotated views, ONE persistent beam launch over all
// cameras' work items (longest first), then the plenoptic microlens stages.
lt_status plan_forward(lt_plan* p, const float* x, float* y, cudaStream_t st, SubsetSel sel) {
  const int nc = (int)p->cams.size();
  if (nc > kMaxBatchCams) {
    for (int c = 0; c < nc; ++c) {
      lt_status s = camera_forward(p, c, x, y + p->cams[c].offset, p->m_total, st, sel);
      if (s != LT_OK) return s;
    }
    return LT_OK;
  }
  BeamBatch b{};
  b.n_cams = nc;
  b.frames = p->frames;
  CameraPlan* cps[kMaxBatchCams];
  for (int i = 0; i < nc; ++i) {
    CameraPlan& c = p->cams[i];
    cps[i] = &c;
    const float* xc = nullptr;
    lt_status s = to_camera_grid(p, c, x, &xc, st);
    if (s != LT_OK) return s;
    const bool plen = c.desc.kind == LT_CAM_PLENOPTIC;
    b.cam[i] = beam_cam(c, xc, plen ? c.d_fa : y + c.offset, nullptr, plen ? (long long)c.K * c.Na : p->m_total, sel);
  }
  for (int g = 0; g < kForwardGroups; ++g) {   // one persistent launch per window class and kernel present
    if (p->class_count[g] == 0) continue;
    lt_status s = run_forward(p, b, cps, p->d_items + p->class_begin[g], p->class_count[g], p->class_real[g],
                              kFwdClasses[g / 3], g % 3 == 0 ? 4 : g % 3 == 1 ? 1 : 0, st);
    if (s != LT_OK) return s;
  }
  for (int i = 0; i < nc; ++i) {
    CameraPlan& c = p->cams[i];
    if (c.desc.kind != LT_CAM_PLENOPTIC) continue;
    cudaError_t e = launch_stage2_forward(c.d_fa, y + c.offset, stage_two(c, sel), p->frames, (long long)c.K * c.Na,
                                          p->m_total, c.d_zbuf, st);
    if (e != cudaSuccess) return cuda_error(e, "plenoptic stage 2");
  }
  return LT_OK;
}

// x = sum_c A_c^T y_c: microlens-stage adjoints, ONE gather launch over all
// cameras that see the volume unrotated (one writer per voxel), then each
// rotated camera through its own grid and the transposed rotation.
lt_status plan_adjoint(lt_plan* p, const float* y, float* x, cudaStream_t st, SubsetSel sel) {
  const int nc = (int)p->cams.size();
  for (int i = 0; i < nc; ++i) {
    CameraPlan& c = p->cams[i];
    if (c.desc.kind != LT_CAM_PLENOPTIC) continue;
    cudaError_t e = launch_stage2_adjoint(y + c.offset, c.d_fa, stage_two(c, sel), p->frames, p->m_total,
                                          (long long)c.K * c.Na, st);
    if (e != cudaSuccess) return cuda_error(e, "plenoptic stage 2 adjoint");
  }
  BeamBatch b{};
  b.frames = p->frames;
  CameraPlan* cps[kMaxBatchCams];
  int written = 0;
  for (int i = 0; i <= nc; ++i) {
    // a launch takes cameras of one box-staged chunk depth (or all direct):
    // a camera that differs from the batch's first starts a new launch
    const bool differs = i < nc && b.n_cams > 0 && !p->cams[i].rotated &&
                         (p->cams[i].adj_sc != cps[0]->adj_sc || (p->cams[i].adj_bx > 0) != (cps[0]->adj_bx > 0));
    const bool flush = (i == nc && b.n_cams > 0) || b.n_cams == kMaxBatchCams || differs;
    if (flush) {
      lt_status s = run_adjoint(p, b, cps, x, p->nvox, written ? 1 : 0, st);
      if (s != LT_OK) return s;
      written = 1;
      b.n_cams = 0;
    }
    if (i == nc) break;
    CameraPlan& c = p->cams[i];
    if (c.rotated) continue;
    const bool plen = c.desc.kind == LT_CAM_PLENOPTIC;
    cps[b.n_cams] = &c;
    b.cam[b.n_cams++] = beam_cam(c, nullptr, nullptr, plen ? c.d_fa : y + c.offset,
                                 plen ? (long long)c.K * c.Na : p->m_total, sel);
  }
  for (int i = 0; i < nc; ++i) {
    CameraPlan& c = p->cams[i];
    if (!c.rotated) continue;
    const bool plen = c.desc.kind == LT_CAM_PLENOPTIC;
    lt_status s = beam_adjoint_to_volume(p, c, plen ? c.d_fa : y + c.offset,
                                         plen ? (long long)c.K * c.Na : p->m_total, x, written, st, sel);
    if (s != LT_OK) return s;
    written = 1;
  }
  return LT_OK;
}

}  // namespace lt

static lt_status check_cam(const lt_plan* p, int cam) {
  if (!p) return set_error(LT_EINVAL, "plan is NULL");
  if (cam < 0 || cam >= (int)p->cams.size()) return set_error(LT_EINVAL, "camera index %d out of range", cam);
  return LT_OK;
}

static lt_status check_plenoptic(const lt_plan* p, int cam) {
  lt_status s = check_cam(p, cam);
  if (s != LT_OK) return s;
  if (p->cams[cam].desc.kind != LT_CAM_PLENOPTIC)
    return set_error(LT_EINVAL, "camera %d is not plenoptic", cam);
  return LT_OK;
}

#ifdef LT_TEST_HOOKS
extern "C" void lt_test_fail_allocation_after(int32_t n) { g_fail_alloc_in.store(n > 0 ? n : 0); }
#endif

extern "C" lt_status lt_forward(lt_plan* plan, const float* x, float* y, void* stream) {
  clear_error();
  if (!plan || !x || !y) return set_error(LT_EINVAL, "NULL argument");
  NvtxRange range("lt_forward");
  return plan_forward(plan, x, y, (cudaStream_t)stream);
}

extern "C" lt_status lt_adjoint(lt_plan* plan, const float* y, float* x, void* stream) {
  clear_error();
  if (!plan || !x || !y) return set_error(LT_EINVAL, "NULL argument");
  NvtxRange range("lt_adjoint");
  return plan_adjoint(plan, y, x, (cudaStream_t)stream);
}

extern "C" lt_status lt_forward_subset(lt_plan* plan, const float* x, float* y, int32_t n_subset, int32_t subset,
                                       void* stream) {
  clear_error();
  if (!plan || !x || !y) return set_error(LT_EINVAL, "NULL argument");
  if (n_subset < 1 || subset < 0 || subset >= n_subset)
    return set_error(LT_EINVAL, "subset %d of %d", subset, n_subset);
  return plan_forward(plan, x, y, (cudaStream_t)stream, SubsetSel{n_subset, subset});
}

extern "C" lt_status lt_adjoint_subset(lt_plan* plan, const float* y, float* x, int32_t n_subset, int32_t subset,
                                       void* stream) {
  clear_error();
  if (!plan || !x || !y) return set_error(LT_EINVAL, "NULL argument");
  if (n_subset < 1 || subset < 0 || subset >= n_subset)
    return set_error(LT_EINVAL, "subset %d of %d", subset, n_subset);
  return plan_adjoint(plan, y, x, (cudaStream_t)stream, SubsetSel{n_subset, subset});
}

extern "C" lt_status lt_forward_camera(lt_plan* plan, int32_t cam, const float* x, float* y_cam,
                                       void* stream) {
  clear_error();
  lt_status s = check_cam(plan, cam);
  if (s != LT_OK) return s;
  if (!x || !y_cam) return set_error(LT_EINVAL, "NULL argument");
  return camera_forward(plan, cam, x, y_cam, plan->cams[cam].M, (cudaStream_t)stream);
}

extern "C" lt_status lt_adjoint_camera(lt_plan* plan, int32_t cam, const float* y_cam, float* x,
                                       int32_t accumulate, void* stream) {
  clear_error();
  lt_status s = check_cam(plan, cam);
  if (s != LT_OK) return s;
  if (!x || !y_cam) return set_error(LT_EINVAL, "NULL argument");
  return camera_adjoint(plan, cam, y_cam, plan->cams[cam].M, x, accumulate != 0, (cudaStream_t)stream);
}

extern "C" lt_status lt_plenoptic_stage1(lt_plan* plan, int32_t cam, const float* x, float* fa,
                                         void* stream) {
  clear_error();
  lt_status s = check_plenoptic(plan, cam);
  if (s != LT_OK) return s;
  if (!x || !fa) return set_error(LT_EINVAL, "NULL argument");
  CameraPlan& c = plan->cams[cam];
  return stage1_forward(plan, c, x, fa, (long long)c.K * c.Na, (cudaStream_t)stream);
}

extern "C" lt_status lt_plenoptic_stage1_adjoint(lt_plan* plan, int32_t cam, const float* fa,
                                                 float* x, int32_t accumulate, void* stream) {
  clear_error();
  lt_status s = check_plenoptic(plan, cam);
  if (s != LT_OK) return s;
  if (!x || !fa) return set_error(LT_EINVAL, "NULL argument");
  CameraPlan& c = plan->cams[cam];
  return stage1_adjoint(plan, c, fa, (long long)c.K * c.Na, x, accumulate != 0, (cudaStream_t)stream);
}

extern "C" lt_status lt_plenoptic_stage2(lt_plan* plan, int32_t cam, const float* fa, float* y_cam,
                                         void* stream) {
  clear_error();
  lt_status s = check_plenoptic(plan, cam);
  if (s != LT_OK) return s;
  if (!fa || !y_cam) return set_error(LT_EINVAL, "NULL argument");
  CameraPlan& c = plan->cams[cam];
  cudaError_t e = launch_stage2_forward(fa, y_cam, c.s2, plan->frames, (long long)c.K * c.Na, c.M,
                                        c.d_zbuf, (cudaStream_t)stream);
  return e == cudaSuccess ? LT_OK : cuda_error(e, "plenoptic stage 2");
}

extern "C" lt_status lt_plenoptic_stage2_adjoint(lt_plan* plan, int32_t cam, const float* y_cam,
                                                 float* fa, void* stream) {
  clear_error();
  lt_status s = check_plenoptic(plan, cam);
  if (s != LT_OK) return s;
  if (!fa || !y_cam) return set_error(LT_EINVAL, "NULL argument");
  CameraPlan& c = plan->cams[cam];
  cudaError_t e = launch_stage2_adjoint(y_cam, fa, c.s2, plan->frames, c.M, (long long)c.K * c.Na,
                                        (cudaStream_t)stream);
  return e == cudaSuccess ? LT_OK : cuda_error(e, "plenoptic stage 2 adjoint");
}

extern "C" const char* lt_last_error(void) { return g_last_error.c_str(); }

extern "C" int32_t lt_autotune_variants(void) { return kForwardVariants; }

extern "C" lt_status lt_projector_status(int32_t* flags, int32_t clear) {
  clear_error();
  if (!flags) return set_error(LT_EINVAL, "flags is NULL");
  int f = 0, g = 0;
  cudaError_t e = projector_status(&f, clear != 0);
  if (e == cudaSuccess) e = adjoint_status(&g, clear != 0);
  if (e != cudaSuccess) return cuda_error(e, "projector status");
  *flags = f | g;
  return LT_OK;
}

extern "C" lt_status lt_plan_set_adjoint_variant(lt_plan* plan, int32_t variant) {
  clear_error();
  if (!plan) return set_error(LT_EINVAL, "plan is NULL");
  if (variant != 0 && variant != 1) return set_error(LT_EINVAL, "adjoint variant %d is not 0 or 1", variant);
  plan->adj_variant = variant;
  return LT_OK;
}

extern "C" lt_status lt_plan_autotune(lt_plan* plan, void* stream, double* times_ms, int32_t* chosen) {
  clear_error();
  if (!plan) return set_error(LT_EINVAL, "plan is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nx = (size_t)plan->frames * plan->nvox, ny = (size_t)plan->frames * plan->m_total;
  float *x = nullptr, *y = nullptr;
  if (device_alloc((void**)&x, nx * sizeof(float)) != cudaSuccess ||
      device_alloc((void**)&y, ny * sizeof(float)) != cudaSuccess) {
    cudaFree(x);
    return set_error(LT_ENOMEM, "autotune buffers");
  }
  cudaMemsetAsync(x, 0, nx * sizeof(float), st);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e30;
  int best_v = 0;
  lt_status s = LT_OK;
  const int saved = plan->fwd_variant;
  for (int v = 0; v < kForwardVariants && s == LT_OK; ++v) {
    plan->fwd_variant = v;
    double tv = 1e30;
    for (int rep = 0; rep < 4 && s == LT_OK; ++rep) {
      cudaEventRecord(e0, st);
      s = plan_forward(plan, x, y, st);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tv = std::min(tv, (double)ms);   // first run warms up
    }
    if (times_ms) times_ms[v] = tv;
    if (tv < best) {
      best = tv;
      best_v = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  if (s != LT_OK) {
    plan->fwd_variant = saved;
    return s;
  }
  plan->fwd_variant = best_v;
  if (chosen) *chosen = best_v;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LT_OK : cuda_error(e, "autotune");
}

// Times the plan's adjoint (every camera and frame) with each adjoint kernel
// choice and keeps the faster.
extern "C" lt_status lt_plan_autotune_adjoint(lt_plan* plan, void* stream, double* times_ms, int32_t* chosen) {
  clear_error();
  if (!plan) return set_error(LT_EINVAL, "plan is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nx = (size_t)plan->frames * plan->nvox, ny = (size_t)plan->frames * plan->m_total;
  float *x = nullptr, *y = nullptr;
  if (device_alloc((void**)&x, nx * sizeof(float)) != cudaSuccess ||
      device_alloc((void**)&y, ny * sizeof(float)) != cudaSuccess) {
    cudaFree(x);
    return set_error(LT_ENOMEM, "autotune buffers");
  }
  cudaMemsetAsync(y, 0, ny * sizeof(float), st);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e30;
  int best_v = 1;
  lt_status s = LT_OK;
  const int saved = plan->adj_variant;
  for (int v = 1; v >= 0 && s == LT_OK; --v) {
    plan->adj_variant = v;
    double tv = 1e30;
    for (int rep = 0; rep < 4 && s == LT_OK; ++rep) {
      cudaEventRecord(e0, st);
      s = plan_adjoint(plan, y, x, st);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tv = std::min(tv, (double)ms);   // first run warms up
    }
    if (times_ms) times_ms[v] = tv;
    if (tv < best) {
      best = tv;
      best_v = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  if (s != LT_OK) {
    plan->adj_variant = saved;
    return s;
  }
  plan->adj_variant = best_v;
  if (chosen) *chosen = best_v;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LT_OK : cuda_error(e, "adjoint autotune");
}

extern "C" lt_status lt_plan_set_forward_variant(lt_plan* plan, int32_t variant) {
  clear_error();
  if (!plan) return set_error(LT_EINVAL, "plan is NULL");
  if (variant < 0 || variant >= kForwardVariants)
    return set_error(LT_EINVAL, "forward variant %d outside [0, %d)", variant, kForwardVariants);
  plan->fwd_variant = variant;
  return LT_OK;
}
