// Host-side plan structures shared by the C-ABI translation units.
#pragma once

#include <string>
#include <vector>

#include "lt.h"
#include "lt_internal.h"

namespace lt {

// Every device allocation of the library goes through here, so that a test
// can make the n-th one fail (lt_test_fail_allocation_after).
cudaError_t device_alloc(void** p, size_t bytes);

// NVTX range around a host entry point (visible to profilers; a no-op
// without one attached).
struct NvtxRange {
  explicit NvtxRange(const char* name);
  ~NvtxRange();
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Kernel window limits (must match lt_kernels.cu).
constexpr int kMaxForwardWindow = 8;
constexpr int kFwdClasses[4] = {8, 4, 3, 2};   // the forward kernels' window classes (window_class)
// forward item groups g: window class kFwdClasses[g / 3]; g % 3 = 0: the
// brick-staged kernel with band t-parts (tma_nb = 4), 1: with per-row
// t-parts (tma_nb = 1), 2: the direct kernel
constexpr int kForwardGroups = 12;
inline int forward_group_kind(int tma_nb) { return tma_nb == 4 ? 0 : tma_nb == 1 ? 1 : 2; }
constexpr int kMaxAdjointWindow = 32;
constexpr int kMaxLensletPixels = 16;

struct Cell {
  double sk, tk, d0s, d0t;   // angular cell centre and widths on the main lens
};

struct CameraPlan {
  lt_camera_desc desc{};
  std::vector<double> focal;
  std::vector<Cell> cells;
  int K = 0;
  int64_t M = 0;
  int64_t offset = 0;
  // the grid this camera sees: the object volume, or its rotated view
  bool rotated = false;
  RotParam rot{};
  bool general = false;            // pitch or roll: permutation + three shears (GenRot)
  GenRot grot{};
  float* d_gb[3] = {nullptr, nullptr, nullptr};   // scratch: permuted, after z, after x
  float* d_gtab[3] = {nullptr, nullptr, nullptr};
  int32_t* d_gjo[3] = {nullptr, nullptr, nullptr};
  lt_volume_desc vol_c{};
  int64_t nvox_c = 0;
  float* d_rz = nullptr;           // scratch [F][nzr][ny][nxp] (rotated cameras)
  float* d_xr = nullptr;           // scratch [F][nzr][ny][nxr] (rotated cameras)
  SliceParam* d_slice = nullptr;   // [K][nz]
  std::vector<int2> h_srange, h_trange;   // host copies of the tile slice intervals
  int tiles_s = 0, tiles_t = 0;           // forward tiles of the target plane
  std::vector<int4> h_items;              // forward work items {cam, k or -1, tile, cost}
  int4* d_items = nullptr;                // this camera's items, longest first
  int n_items = 0;
  int n_real_items = 0;                   // leading items of positive cost (the rest meet no slice)
  int2* d_srange = nullptr;        // [K][tiles_s] slice interval per forward tile column
  int2* d_trange = nullptr;        // [K][tiles_t] slice interval per forward tile row
  int wmax_s = 0, wmax_t = 0, wimax_s = 0, wimax_t = 0;
  // brick-staged (TMA) forward: brick box sized at plan time for every
  // (cell, slice, tile); tma_nb = 4 (band t-parts) or 1 (per-row t-parts)
  // when the camera runs that kernel, else 0
  int tma_bx = 0, tma_by = 0, tma_nb = 0;
  int tma_chunks = 1;              // parts each forward item is split into (few tiles: more CTAs per tile)
  int adj_bx = 0, adj_by = 0;      // box-staged adjoint: image box (0: the direct adjoint serves it)
  int adj_sc = 8;                  // its slices per chunk (8 or 4)
  float* d_adj_s = nullptr;        // and its window tables (lt_beam_adj.cu layout)
  float* d_adj_t = nullptr;
  int2* d_adj_ox = nullptr;
  int2* d_adj_oy = nullptr;
  void* d_stab = nullptr;          // its footprint-weight tables (lt_beam_tma.cu layout)
  void* d_ttab = nullptr;
  // plenoptic
  int64_t Na = 0;
  LensletParam* d_lens = nullptr;
  int2* d_cols = nullptr;          // [N_mu] block columns / rows of each lenslet
  int2* d_rows = nullptr;
  int32_t* d_owner = nullptr;      // [arr_nt * arr_ns] owning lenslet or -1
  float* d_mask = nullptr;         // [arr_nt * arr_ns] diagonal of M
  int4* d_det_range = nullptr;
  int4* d_det_union = nullptr;
  int2* d_cand_all_s = nullptr;
  int2* d_cand_all_t = nullptr;
  float* d_zbuf = nullptr;         // scratch [F][N_mu][window^2]
  float* d_s2tab = nullptr;        // stage-two transport table (Bs, Bt per lenslet and cell)
  lt::S2Desc* d_s2desc = nullptr;  // [N_mu][K] stage-two descriptors
  uint32_t* d_s2bits = nullptr;    // [N_mu][16] block ownership bits
  uint32_t* d_s2ivals = nullptr;   // [N_mu][8] per-row intervals of the owned pixels
  int64_t s2tab_floats = 0;
  float* d_fa = nullptr;           // scratch array plane [F][K][Na]
  StageTwo s2{};
};

lt_status set_error(lt_status s, const char* fmt, ...);
lt_status cuda_error(cudaError_t e, const char* where);
void clear_error();

// Angular-plane subset of a projection (Sec. V, eq. subset): the cells k with
// k % n == s take part; n <= 1 selects every cell.
struct SubsetSel {
  int n = 1;
  int s = 0;
};

lt_status camera_forward(lt_plan* p, int cam, const float* x, float* y, long long y_fs,
                         cudaStream_t st, SubsetSel sel = SubsetSel{});
lt_status camera_adjoint(lt_plan* p, int cam, const float* y, long long y_fs, float* x,
                         int accumulate, cudaStream_t st, SubsetSel sel = SubsetSel{});
// Slice -> plane beam integration of camera c (through its rotated view when
// it is rotated, in the plan's scratch) into fa [F][..] with frame stride fa_fs.
lt_status stage1_forward(lt_plan* p, CameraPlan& c, const float* x, float* fa, long long fa_fs,
                         cudaStream_t st, SubsetSel sel = SubsetSel{});


}  // namespace lt

struct lt_plan {
  lt_volume_desc vol{};
  int frames = 1;
  int64_t nvox = 0;
  int64_t m_total = 0;
  int device = 0;
  int sms = 148;
  std::vector<lt::CameraPlan> cams;
  // every camera's forward items, grouped by the camera's forward window
  // class (kFwdClasses order) and by whether the brick-staged kernel serves
  // it, longest first within a group: the batched forward makes one
  // persistent launch per group present, so that a camera runs the same
  // kernel instantiation as in a launch of its own
  int4* d_items = nullptr;
  int n_items = 0;
  int class_begin[lt::kForwardGroups] = {};
  int class_count[lt::kForwardGroups] = {};
  int class_real[lt::kForwardGroups] = {};   // leading items of positive cost in each group
  int* d_counter = nullptr;        // persistent-launch work counter
  float* d_chunk_part = nullptr;   // brick-staged forward: partial tiles of chunked items
  int* d_chunk_count = nullptr;    // and the chunks completed per (item, frame), zero between launches
  int fwd_variant = lt::kTmaVariant;   // forward kernel variant (autotuned; the brick-staged kernel until then)
  int adj_variant = 1;             // 1: box-staged adjoint where it fits, 0: the direct gather adjoint
};

namespace lt {
// Plan-level operators over every camera (one batched launch per stage).
lt_status plan_forward(lt_plan* p, const float* x, float* y, cudaStream_t st, SubsetSel sel = SubsetSel{});
lt_status plan_adjoint(lt_plan* p, const float* y, float* x, cudaStream_t st, SubsetSel sel = SubsetSel{});
}  // namespace lt
