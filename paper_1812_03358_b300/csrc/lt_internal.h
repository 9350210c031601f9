// Internal data structures shared by the host planner and the CUDA kernels.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace lt {

// Footprint of a target pixel i on a source grid, for one axis, one angular
// cell and one source plane (Sec. II-C, eq. xport,int).  The set of source
// rays that cross angular cell k and land in target pixel i, pushed to the
// source plane, has a trapezoidal density: the convolution of two boxes whose
// widths are the cell and the pixel seen from the source plane (Table III; a
// box for the Dirac basis, Table II).  In source-index units (source cell j
// spans [j-1/2, j+1/2]) its centre is xi(i) = c0 + c1 * i, its plateau
// half-width P and its outer half-width Q.  The transport entry is
//     B[i][j] = H * dsrc * integral_{j-1/2}^{j+1/2} T(xi - xi(i)) dxi
// with T the unit-height trapezoid; H * dsrc is folded into a per-plane scale.
struct AxisParam {
  float c0_hi, c0_lo;   // xi(i) = (c0_hi + c0_lo) + (c1_hi + c1_lo) * i
  float c1_hi, c1_lo;
  float P, Q;           // 0 <= P <= Q
  float hir;            // 1 / (2 (Q - P)); 0 when Q == P (box)
  float inv_c1;         // 1 / c1, for the adjoint's target-pixel windows
};

// One (angular cell k, slice n) of a slice -> image-plane transport.
struct SliceParam {
  AxisParam s, t;
  float scale;          // Hs*dx * Ht*dy * dz  (/ V^a for the plenoptic array plane)
  int32_t ws, wt;       // forward windows: source cells per target pixel
  int32_t wis, wit;     // adjoint windows: target pixels per source cell
  int32_t pad[3];
};

// Array plane -> detector through one lenslet, one angular cell (Sec. II-F2).
// Source grid = the array plane, target = detector pixels.
struct LensletParam {
  AxisParam s, t;
  float scale;          // Hs*arr_ps * Ht*arr_pt
  int32_t pad[3];
};

// Device tables of one plenoptic camera's array -> detector stage.
// One (lenslet, cell) of stage two, 32 bytes (plan-built, read by the
// stage-two kernels; lenslet-major, cell k of lenslet mu at mu * K + k).
struct alignas(16) S2Desc {
  int32_t off;     // offset of its transport table entry (floats, a multiple of 4); -1: empty window
  int32_t px0;     // array index of the lenslet block's first pixel
  int32_t y0;      // detector index of the cell window's first pixel
  int32_t zo;      // index of the cell window's first pixel in the lenslet's union window (rows of nsu)
  uint32_t dims;   // nc | nr << 8 | nds << 16 | ndt << 24
  float scale;     // the lenslet's transmission scale for this cell
  uint32_t win;    // nsu | ntu << 8 | (last cell of the lenslet) << 16 | k << 17
  int32_t mu;
};
static_assert(sizeof(S2Desc) == 32, "S2Desc is 32 bytes");

// Threads per CTA of the stage-two kernels (one lenslet walk per warp).
constexpr int kStage2Threads = 256;
// Each warp's item descriptors come kS2Chunk at a time into a ring of
// kS2Ring in its shared memory (S2Desc = 8 floats each).
constexpr int kS2Chunk = 16, kS2Ring = 2 * kS2Chunk;

struct StageTwo {
  const LensletParam* lens;   // [K][mla_nt*mla_ns]
  const int2* cols;           // [mla_nt*mla_ns]: array columns [x, y) of lenslet mu's block
  const int2* rows;           // [mla_nt*mla_ns]: array rows [x, y)
  const int32_t* owner;       // [arr_nt*arr_ns]: lenslet whose disc holds the pixel centre, -1 if none
  const float* mask;          // [arr_nt*arr_ns]: the diagonal of M (aperture x coded transmission)
  int32_t overlap;            // 1 if lenslet blocks overlap (hexagonal lattice): write owned pixels only
  int32_t mla_ns, mla_nt;
  int32_t arr_ns, arr_nt;
  int32_t det_ns, det_nt;
  int32_t K;
  int32_t wis, wit;           // adjoint windows (detector pixels per array pixel)
  int32_t max_cols, max_rows; // forward windows (array pixels per lenslet)
  const int4* det_range;      // [K][mla_nt*mla_ns]: detector pixels a lenslet can reach (s0, s1, t0, t1), inclusive
  const int4* det_union;      // [mla_nt*mla_ns]: union over cells of det_range
  const int2* cand_all_s;     // [det_ns]: lenslet columns whose union window holds the column
  const int2* cand_all_t;     // [det_nt]
  float* zbuf;                // scratch [F][mla_nt*mla_ns][kStage2Window^2]: per-lenslet sub-images
  int32_t full_cover;         // 1 if every array pixel lies in some lenslet block
  int32_t sub_n, sub_s;       // angular-plane subset (cell_on); 1, 0 for all cells
  // The per-(lenslet, cell) form the kernels walk (plan-built):
  const S2Desc* desc;         // [mla_nt*mla_ns][K]
  const float* wtab;          // transport table: per (lenslet, cell) Bs [nc][nds rounded up to 4] (zero padded)
                              // then Bt [nr][ndt], 16-byte aligned
  const uint32_t* bits;       // [mla_nt*mla_ns][16]: bit r*nc+c of words 0..7 = the lenslet owns block pixel (r, c);
                              // of words 8..15 = nobody owns it and blocks tile the plane (the adjoint clears it)
  int32_t tab_max, pix_max, w_max, z_max, y_max;   // largest table entry, block (rows of row_max), nr*nds4, union
                                                   // window, cell window (floats, multiples of 4)
  int32_t row_max;                                 // block row in shared memory: nc + 3 rounded up to 4
  const uint32_t* ivals;      // [mla_nt*mla_ns][8]: per block row r, uint16 c0 | c1 << 8: the lenslet owns
                              // exactly columns [c0, c1) of the row (valid when iv_ok)
  int32_t iv_ok;              // every lenslet's own pixels form one interval per row
  int32_t fwd_warp_floats, adj_warp_floats;        // shared memory per warp of the two kernels
  int32_t fwd_per_sm, adj_per_sm, sms;             // resident CTAs per SM of each kernel, SM count
};

// Largest detector window (per axis) of one lenslet's sub-image.
constexpr int kStage2Window = 24;

// Rotated view of the object volume (Sec. III-A): quarter turns nq about y,
// then the z shear E^z and the x shear E^x of the residual rotation.  The
// permuted grid is [nzp][ny][nxp]; after E^z it is [nzr][ny][nxp] with
// nzr = nzp + 2 pz, after E^x [nzr][ny][nxr] with nxr = nxp + 2 px.  Entry
// between output cell i and source cell j of column c (E^z) / row c (E^x):
// the average of the box-overlap hat over the sheared cell,
//   u = (i - j - pad) + slope * (c - (n_c - 1)/2),  width beta = |slope|.
struct RotParam {
  int32_t nq;
  int32_t nx, ny, nz;      // original volume
  int32_t nxp, nzp;        // after the quarter turns
  int32_t pz, px;
  int32_t nzr, nxr;        // rotated volume
  float bz, betaz;         // E^z slope (b dx'/dz') and |bz|
  float ax, betax;         // E^x slope (a dz'/dx') and |ax|
  int32_t wz, wx;          // source windows
  // Per-column shear entries, filled once at plan time by launch_shear_tables:
  // column c of E^z (c < nxp) has window offset jz[c] and entries
  // tz[c * nwz + q] = E^z(i, i - pz + jz[c] + q) for every output i (zero for
  // q >= wz); row r of E^x (r < nzr) likewise with jx[r], tx[r * wx + q].
  int32_t nwz;             // 8 or 16, >= wz (register window of the z passes)
  int32_t djz;             // largest jz spread over 32 consecutive columns (c = 32k ...)
  float* tz;
  int32_t* jz;
  float* tx;
  int32_t* jx;
};

// General orientation (yaw with pitch and/or roll, Sec. III-A): a signed
// permutation of the grid, then up to three least-squares shear passes
// (z, x, y), each along one axis with a shift linear in the other two.
struct ShearPass {
  int32_t axis;            // 0 = x, 1 = y, 2 = z (the sheared axis)
  int32_t n0, n1, n2;      // input dims (x, y, z); the output pads `axis` by 2 pad
  int32_t pad, nw;         // padding, taps per output
  int32_t nu, nv;          // column dims: the other two axes in increasing order
  const float* tab;        // [nv][nu][nw] entries, tab[(v nu + u) nw + q] = E(i, i - pad + J + q)
  const int32_t* jo;       // [nv][nu] window offsets J
  int32_t active;          // 0: the identity (both coefficients zero), skipped
};
struct GenRot {
  int32_t nx, ny, nz;      // source volume
  int32_t km[3], sg[3];    // source axis m reads permuted axis km[m], flipped when sg[m] < 0
  int32_t np[3];           // permuted dims (x, y, z)
  ShearPass pass[3];       // z, x, y
};

// Forward beam-integration tile: kBeamTileS x kBeamTileT target pixels per CTA.
// The planner computes, per (cell, tile column) and (cell, tile row), the
// slice interval [x, y) outside of which the tile's footprints miss the volume.
constexpr int kBeamTileS = 32;
constexpr int kBeamTileT = 32;

// One camera's slice -> plane transport inside a batched launch.
constexpr int kMaxBatchCams = 24;
struct BeamCam {
  const float* x;          // camera-grid volume [F][nz][ny][nx] (forward input)
  float* out;              // forward output: [F][K][nt][ns] if per_cell, else [F][..][nt][ns]
  const float* in;         // adjoint input, same layout as out
  const SliceParam* prm;   // [K][nz]
  const float* mask;       // per-pixel output mask M (plenoptic array plane, diagonal) or null
  const int2* srange;      // [K][tiles_s]
  const int2* trange;      // [K][tiles_t]
  long long x_fs, out_fs;  // frame strides
  int32_t nx, ny, nz, ns, nt, K, per_cell, tiles_s, tiles_t;
  int32_t wis, wit;        // adjoint windows (max over cells and slices)
  int32_t sub_n, sub_s;    // angular-plane subset: cells k with k % sub_n == sub_s (all if sub_n <= 1)
};

// Cell k takes part in the current angular-plane subset (Sec. V, eq. subset).
__host__ __device__ __forceinline__ bool cell_on(int sub_n, int sub_s, int k) {
  return sub_n <= 1 || k % sub_n == sub_s;
}
struct BeamBatch {
  BeamCam cam[kMaxBatchCams];
  int32_t n_cams;
  int32_t frames;
};

// TMA view of each camera's source volume for the brick-staged forward
// (lt_beam_tma.cu): a 3-D tensor map over [F * nz][ny][nx] float32, the
// brick box (bx columns, a multiple of 4, by rows) the planner sized for the
// camera's 32 x 32 tiles, and the camera's footprint-weight tables.
struct TmaBatch {
  CUtensorMap map[kMaxBatchCams];
  const void* stab[kMaxBatchCams];   // per-(cell, slice, tile column) s-weights, then brick column origins
  const void* ttab[kMaxBatchCams];   // per-(cell, slice, tile row) t-weights, then brick row origins
  int32_t bx[kMaxBatchCams];
  int32_t by[kMaxBatchCams];
  int32_t chunks[kMaxBatchCams];     // parts each of the camera's items is split into (>= 1)
};

// Forward kernel variants chosen by the autotuner: slices per weight batch
// and warp groups (128 threads each) splitting a tile's slices.
// Variants 0-4 are the direct kernel's shapes; variant kTmaVariant is the
// brick-staged TMA kernel (cameras that do not fit it run
// kDefaultDirectVariant).
constexpr int kDirectVariants = 5;
constexpr int kTmaVariant = 5;
constexpr int kForwardVariants = 6;
constexpr int kDefaultDirectVariant = 2;
struct ForwardVariant {
  int32_t sb, groups;
};
constexpr ForwardVariant kForwardVariantTable[kDirectVariants] = {{4, 2}, {4, 1}, {2, 2}, {2, 4}, {8, 1}};

// ---- kernel launchers (lt_kernels.cu) -------------------------------------

// Batched persistent forward: work items (int4 {cam, k or -1 for all cells,
// tile, cost}) for every frame, processed in list order (longest first) by
// a grid of resident CTAs that take the next item from *counter (zeroed by
// the launcher).  Every output tile of every camera appears once in items.
cudaError_t launch_beam_forward_batched(const BeamBatch& b, const int4* items, int n_items, int* counter,
                                        int wclass, int variant, int ctas, cudaStream_t st);
// CTAs per SM of a forward variant (for the persistent grid).
int beam_forward_occupancy(int wclass, int variant);
int window_class(int w);

// Brick-staged forward (lt_beam_tma.cu): W = forward window class (2..4).
// A stage holds the bricks of tma_forward_group() consecutive slices; plane
// = the largest bx * by of the launch, tsz = floats of a consumer warp's
// s-contracted rows (tma_forward_tsz of the largest by; by at most
// tma_forward_max_by()).  Tables: tma_table_bytes for one camera (tiles_t =
// 0: the s-part alone); launch_beam_tables fills them from the camera's
// SliceParam table and sets *bad if a group's brick did not fit.
bool tma_forward_available();
// Tensor map over [nz_total][ny][nx] floats with box {bx, by, tma_forward_group()}.
bool tma_encode_volume(CUtensorMap* map, const float* x, int nx, int ny, int nz_total, int bx, int by);
// The same for a plane stack whose third-axis stride (floats) is z_stride, box depth bz.
bool tma_encode_planes(CUtensorMap* map, const float* x, int nx, int ny, int nz_total, long long z_stride, int bx,
                       int by, int bz = 1);
size_t tma_table_bytes(int w, bool band, int K, int nz, int tiles_s, int tiles_t);
cudaError_t launch_beam_tables(const SliceParam* prm, int K, int nz, int tiles_s, int tiles_t, int w, bool band,
                               int bx, int by, void* stab, void* ttab, int* bad, cudaStream_t st);
int tma_forward_group();
int tma_forward_tsz(int max_by);
int tma_forward_max_by();
// band = the t-parts in band form (four-row groups within
// tma_forward_band_rows() brick rows), else one row of taps per pixel row
int tma_forward_band_rows();
int tma_forward_occupancy(int w, bool band, int plane, int tsz);
// items: the launch's work items, those of positive cost (the first n_real)
// before those whose tile no slice reaches.  chunks: the largest
// tb.chunks[] of the launch; with chunks > 1, scratch holds n_real * F *
// chunks * 1024 floats and unit_count n_real * F ints, zero between launches.
cudaError_t launch_beam_forward_tma(const BeamBatch& b, const TmaBatch& tb, const int4* items, int n_items,
                                    int n_real, int* counter, int w, bool band, int plane, int tsz, int chunks,
                                    float* scratch, int* unit_count, int ctas, cudaStream_t st);
// Device status word of the projector kernels: bit 0 a brick or band that
// did not fit (its weights were zeroed), bit 1 a TMA wait that gave up.
// Read (and optionally cleared) synchronously.
cudaError_t projector_status(int* flags, bool clear);

// TMA view of each camera's adjoint input (the image plane, or the array
// plane of every cell) for the box-staged adjoint (lt_beam_adj.cu): a 3-D
// tensor map over [F * zf][nt][ns] float32 (zf = K per-cell planes or 1),
// the image box (bx columns, a multiple of 4, by rows) the planner sized for
// the camera's voxel tiles and slice chunks, and the camera's plan-built
// window tables (wqs / wqt entries per voxel column / row).
struct AdjBatch {
  CUtensorMap map[kMaxBatchCams];
  const float* stab[kMaxBatchCams];
  const float* ttab[kMaxBatchCams];
  const int2* ox[kMaxBatchCams];
  const int2* oy[kMaxBatchCams];
  int32_t bx[kMaxBatchCams];
  int32_t by[kMaxBatchCams];
  int32_t zf[kMaxBatchCams];
  int32_t wqs[kMaxBatchCams];
  int32_t wqt[kMaxBatchCams];
  int32_t tiles_x[kMaxBatchCams];
  int32_t tiles_y[kMaxBatchCams];
  int32_t chunks[kMaxBatchCams];
};
// Box-staged adjoint: voxel tile adjoint_tile_x() x adjoint_tile_y(), sc
// slices per CTA (8, or 4 for cameras whose 8-slice boxes are too big; at
// most adjoint_chunk_max()); x[F][nz][ny][nx] (= or +=) the sum over the
// batch's cameras and cells (every camera of a launch planned for the same
// sc).  Tables: adjoint_table_sizes gives the bytes of the S and T tables
// and the origin counts of one camera; launch_adjoint_tables fills them and
// sets *bad if a box does not fit.
int adjoint_tile_x();
int adjoint_tile_y();
int adjoint_chunk_max();
// Resident CTAs per SM of the box-staged adjoint for one camera's box and
// windows with sc slices per chunk (0 if it cannot run).
int adjoint_occupancy(int bx, int by, int wqs, int wqt, int sc);
void adjoint_table_sizes(int K, int nz, int nx, int ny, int wqs, int wqt, int sc, size_t* s_bytes, size_t* t_bytes,
                         size_t* ox_count, size_t* oy_count);
cudaError_t launch_adjoint_tables(const SliceParam* prm, int K, int nz, int nx, int ny, int wqs, int wqt, int bx,
                                  int by, int sc, float* stab, float* ttab, int2* ox, int2* oy, int* bad,
                                  cudaStream_t st);
cudaError_t launch_beam_adjoint_tma(const BeamBatch& b, const AdjBatch& a, int sc, float* x, long long x_fs,
                                    int accumulate, cudaStream_t st);
// Status word of the box-staged adjoint (bits as the forward's).
cudaError_t adjoint_status(int* flags, bool clear);

// Batched gather adjoint over cameras that share one grid (cam[0]'s dims):
// x[F][nz][ny][nx] (= or +=) sum over cameras and cells.
cudaError_t launch_beam_adjoint_batched(const BeamBatch& b, float* x, long long x_fs, int accumulate,
                                        cudaStream_t st);

// zbuf: per-lenslet sub-image scratch [F][N_mu][kStage2Window^2] (the plan's,
// or any buffer of that size).
// Plan time: fills s2's transport table wtab (sized by the host from the
// windows, at the offsets of s2.desc) on stream st; the stage-two kernels'
// shared memory and resident CTAs per SM (raises their dynamic shared memory
// limit as needed).
cudaError_t launch_stage2_tables(StageTwo s2, float* wtab, cudaStream_t st);
size_t stage2_smem_bytes(const StageTwo& s2, bool adjoint);
cudaError_t stage2_occupancy(const StageTwo& s2, bool adjoint, int* ctas_per_sm);
cudaError_t launch_stage2_forward(const float* fa, float* y, StageTwo s2, int frames,
                                  long long fa_frame_stride, long long y_frame_stride,
                                  float* zbuf, cudaStream_t st);

cudaError_t launch_stage2_adjoint(const float* y, float* fa, StageTwo s2, int frames,
                                  long long y_frame_stride, long long fa_frame_stride,
                                  cudaStream_t st);

// Rotation passes (lt_rotate.cu).  Frames are consecutive volumes.
cudaError_t launch_rotate_forward(const float* x, float* rz, float* xr, const RotParam& r, int frames,
                                  cudaStream_t st);
// g_xr (rotated grid) -> x (= or +=), using rz as scratch.
cudaError_t launch_rotate_adjoint(const float* g_xr, float* rz, float* x, const RotParam& r, int frames,
                                  int accumulate, cudaStream_t st);

// Fills r.tz/jz/tx/jx (device arrays of nxp*nwz, nxp, nzr*wx, nzr entries).
cudaError_t launch_shear_tables(const RotParam& r, cudaStream_t st);

// General rotations: tables of one pass (built in FP64, stored FP32), and
// the rotation / its transpose through scratch buffers b0 (permuted), b1
// (after z), b2 (after x) of the plan (each large enough for its stage).
cudaError_t launch_shear_pass_table(const ShearPass& ps, double s1, double s2, double du_dt, double dv_dt,
                                    float* tab, int32_t* jo, cudaStream_t st);
cudaError_t launch_grot_forward(const float* x, float* b0, float* b1, float* b2, float* xr, const GenRot& g,
                                int frames, cudaStream_t st);
cudaError_t launch_grot_adjoint(const float* g_xr, float* b0, float* b1, float* b2, float* x, const GenRot& g,
                                int frames, int accumulate, cudaStream_t st);

// x[i] += y[i], i < n.
cudaError_t launch_add_inplace(float* x, const float* y, long long n, cudaStream_t st);

}  // namespace lt
