/*
 * lt.h - C ABI of the B300 light-transport camera library.
 *
 * The library evaluates the matrix-free camera model of McGaffin, Chen,
 * Fessler and Sick ("A practical light transport system model for
 * chemiluminescence distribution reconstruction"): the projector y = A x of
 * single-lens and plenoptic cameras (Sec. II-C..F, Sec. III), its exact
 * adjoint x = A^T y (Sec. IV-A), and the reconstruction of Table V (Sec. V).
 *
 * Conventions (all calls):
 *   - Lengths in millimetres, angles in radians.
 *   - A volume is float32 [nz][ny][nx] (x fastest), voxel (ix, iy, iz)
 *     centred at ((ix-(nx-1)/2) dx, (iy-(ny-1)/2) dy, (iz-(nz-1)/2) dz).
 *   - A camera image is float32 [det_nt][det_ns] (s fastest, Sec. IV).
 *     y of a plan is the concatenation over cameras: camera c occupies
 *     [det_offsets[c], det_offsets[c+1]) of each frame's row.
 *   - With F frames, x is [F][n_vox] and y is [F][det_offsets[n_cams]].
 *   - Data pointers passed to lt_forward / lt_adjoint / lt_recon_* are DEVICE
 *     pointers owned by the caller (borrowed for the call); the library keeps
 *     no reference after the call returns.  Host descriptor arrays are copied.
 *   - Calls are asynchronous on the given cudaStream_t (NULL = legacy default
 *     stream).  Validation errors are returned synchronously; CUDA launch
 *     errors are returned as LT_ECUDA.  Nothing aborts, exits or traps; no C++
 *     exception crosses the ABI.  lt_last_error() describes the last failure
 *     of the calling thread.
 *   - A plan owns device tables and a scratch buffer (the plenoptic array
 *     plane); two calls on the same plan must not overlap in time on
 *     different streams.
 */
#ifndef LT_H
#define LT_H

#include <stdint.h>

#if defined(__GNUC__)
#define LT_API __attribute__((visibility("default")))
#else
#define LT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LT_OK = 0,
  LT_EINVAL = 1,        /* invalid descriptor or argument                    */
  LT_ENOMEM = 2,        /* device or host allocation failed                  */
  LT_ECUDA = 3,         /* CUDA runtime error (launch, copy)                  */
  LT_EUNSUPPORTED = 4,  /* valid but not supported by this build             */
  LT_ETIMEOUT = 5       /* a bounded device wait gave up                      */
} lt_status;

enum { LT_BASIS_PILLBOX = 0, LT_BASIS_DIRAC = 1 };    /* angular basis a(.), Sec. II-B */
enum { LT_MLA_SQUARE = 0, LT_MLA_HEX = 1 };           /* microlens lattice              */
enum { LT_CAM_SINGLE = 0, LT_CAM_PLENOPTIC = 1 };     /* Sec. II-F                     */

/* Pillbox voxel grid (Sec. III, eq. voxel), centred on the object origin. */
typedef struct {
  int32_t nx, ny, nz;
  double dx, dy, dz;
} lt_volume_desc;

/* One camera (Sec. II-F).  The optical axis passes through the volume centre;
 * the main lens is d_obj in front of it.  The angular plane is the main lens,
 * divided into ks x kt cells tiling [-r_main, r_main]^2 (cells whose centre is
 * inside the aperture disc are kept).  The camera is turned by yaw (about
 * the volume's y axis), pitch (about x) and roll (about z, the optical axis):
 * Theta = R_y(yaw) R_x(pitch) R_z(roll), p = Theta p^r (Sec. III-A).  A yaw
 * alone uses quarter turns and two shears; with pitch or roll the rotation
 * is split into a signed permutation and D S_z S_x S_y (three shears). */
typedef struct {
  int32_t kind;            /* LT_CAM_SINGLE or LT_CAM_PLENOPTIC                  */
  int32_t basis;           /* LT_BASIS_PILLBOX or LT_BASIS_DIRAC                 */
  double f_main, r_main;   /* main-lens focal length and aperture radius         */
  double d_obj;            /* main lens -> volume centre                         */
  double yaw;              /* radians                                            */
  double pitch, roll;      /* radians (rotation angles, not pixel pitches)       */
  int32_t det_ns, det_nt;  /* detector pixels                                    */
  double det_ps, det_pt;   /* detector pitch                                     */
  double d_lens_det;       /* single lens: main lens -> detector (D)             */
  int32_t ks, kt;          /* angular cells per axis                             */
  /* plenoptic only (Sec. II-F2) */
  double d_lens_mla;       /* D_mu_m: main lens -> microlens array               */
  double d_mla_det;        /* D_mu_d: microlens array -> detector                */
  int32_t mla_ns, mla_nt;  /* lenslet columns and rows (see mla_layout)          */
  double mla_pitch;        /* lenslet centre spacing                             */
  double mla_radius;       /* lenslet disc radius (<= mla_pitch / 2)             */
  const double* mla_focal; /* host [mla_nt*mla_ns] focal lengths, copied         */
  int32_t arr_ns, arr_nt;  /* array-plane (mask) grid, Sec. II-D                */
  double arr_ps, arr_pt;
  int32_t mla_layout;      /* LT_MLA_SQUARE, or LT_MLA_HEX: rows mla_pitch sqrt(3)/2
                            * apart, odd rows shifted by half a pitch, the
                            * lattice centred on the axis (column offset
                            * -pitch/4); lenslet (mt, ms) = mla_focal[mt][ms]   */
  const float* arr_mask;   /* host [arr_nt*arr_ns] coded-mask transmission in
                            * [0, 1] multiplying the aperture mask M (Sec. II-D,
                            * eq. occlusion), or NULL (= 1); copied            */
} lt_camera_desc;

typedef struct lt_plan lt_plan;

/* Build a plan for n_cams cameras looking at one volume, for batches of
 * n_frames volumes (Sec. III-A "System models": A maps R^N to R^M).  Computes
 * every transport parameter (Tables II/III) in float64 on the host and
 * uploads them.  Uses the current CUDA device.
 * Errors: LT_EINVAL for non-positive sizes/pitches/focal lengths, a slice at
 * or behind the lens, a lenslet radius above half the pitch; LT_EUNSUPPORTED
 * for footprints wider than the kernels' windows (a pixel's footprint over
 * more than 8 voxels per axis, a voxel covered by more than 32 pixels per
 * axis, more than 16 array pixels per lenslet per axis, a lenslet sub-image
 * wider than 24 detector pixels per axis); LT_ENOMEM.
 * The forward makes one persistent launch per forward window class (2, 3,
 * 4, 8 voxels) present among the cameras. */
LT_API lt_status lt_plan_create(const lt_volume_desc* vol, const lt_camera_desc* cams,
                         int32_t n_cams, int32_t n_frames, lt_plan** out);

/* Frees all device memory of the plan (synchronises the device first). */
LT_API lt_status lt_plan_destroy(lt_plan* plan);

/* n_vox = nx*ny*nz; det_offsets[0..n_cams] (host array of n_cams+1). */
LT_API lt_status lt_plan_sizes(const lt_plan* plan, int64_t* n_vox, int64_t* det_offsets);

/* Forward projection y = A x for every camera and frame (Sec. II-F, Sec. III,
 * eq. plenoptic,factor).  x: device [F][n_vox]; y: device [F][M] (overwritten). */
LT_API lt_status lt_forward(lt_plan* plan, const float* x, float* y, void* stream);

/* Exact adjoint x = A^T y = sum_c A_c^T y_c (Sec. IV-A), computed as a gather
 * per voxel (one writer per output, no atomics).  x is overwritten. */
LT_API lt_status lt_adjoint(lt_plan* plan, const float* y, float* x, void* stream);

/* Angular-plane subset operators (Sec. V, eq. subset): sum over the cells k
 * of every camera with k % n_subset == subset (cells in lexicographic order,
 * s index fastest), without the K/|S| factor.  lt_forward_subset writes y;
 * lt_adjoint_subset overwrites x.  The subsets s = 0 .. n_subset - 1 of a
 * partition sum to lt_forward / lt_adjoint.  LT_EINVAL for n_subset < 1 or
 * subset outside [0, n_subset). */
LT_API lt_status lt_forward_subset(lt_plan* plan, const float* x, float* y, int32_t n_subset, int32_t subset,
                                   void* stream);
LT_API lt_status lt_adjoint_subset(lt_plan* plan, const float* y, float* x, int32_t n_subset, int32_t subset,
                                   void* stream);

/* Per-camera forward / adjoint.  y_cam: device [F][M_c] (the camera's own
 * image).  lt_adjoint_camera writes x (accumulate = 0) or adds to it
 * (accumulate = 1). */
LT_API lt_status lt_forward_camera(lt_plan* plan, int32_t cam, const float* x, float* y_cam,
                            void* stream);
LT_API lt_status lt_adjoint_camera(lt_plan* plan, int32_t cam, const float* y_cam, float* x,
                            int32_t accumulate, void* stream);

/* Allocation-free plenoptic forward projection (no counterpart in the paper).
 * Same result as lt_forward_camera for a plenoptic camera, for callers that
 * cannot allocate device memory when they project (frameworks whose memory
 * pools forbid raw cudaMalloc, real-time loops where an allocation and its
 * implicit synchronisation are not allowed): the array-plane intermediate is
 * staged in a static 16 MiB device array inside the library instead of the
 * plan's buffer, and the call allocates and frees nothing.
 *   - frames x cells x array pixels must be <= 4,194,304 floats, else
 *     LT_EINVAL with a message; non-plenoptic cameras give LT_EINVAL.
 *     Rotated cameras are served (their rotated view goes to the scratch
 *     the plan allocated when it was created).
 *   - Every GPU that uses the array holds it until exit.  With CUDA's lazy
 *     module loading (the default since CUDA 12.2) the array is reserved
 *     by the first call on each device, which may also synchronise; later
 *     calls reserve nothing.
 *   - All calls share the array and it keeps the last call's contents; every
 *     element a call reads is first written by that call, but calls that
 *     overlap in time on the GPU (any plan, any stream) race on it.
 *   - The first call on each device looks up the array's device address with
 *     that device current; make that first call before any stream capture. */
LT_API lt_status lt_forward_camera_noalloc(lt_plan* plan, int32_t cam, const float* x, float* y_cam,
                                           void* stream);

/* Rotated perspectives (Sec. III-A, eq. rot): camera `cam`'s yaw is split
 * into quarter turns P and a residual |theta_r| <= 45 deg applied as two 1-D
 * least-squares shear re-projections, x_c = E^x E^z P x, onto the camera's
 * own grid.
 *   lt_camera_grid            the camera grid (sizes and spacings of x_c);
 *                             equal to the plan's volume for yaw = 0.
 *   lt_rotate_volume          x [F][nz][ny][nx] -> xc [F][grid], device
 *                             pointers owned by the caller.
 *   lt_rotate_volume_adjoint  xc -> x (= or += with accumulate), the exact
 *                             transpose (same entries, same rounding).
 * For an unrotated camera both are plain copies.  The passes use the
 * camera's plan-owned scratch, so calls for the same camera must not overlap
 * in time.  LT_EINVAL for a bad plan, camera or pointer. */
LT_API lt_status lt_camera_grid(const lt_plan* plan, int32_t cam, lt_volume_desc* grid);
LT_API lt_status lt_rotate_volume(lt_plan* plan, int32_t cam, const float* x, float* xc, void* stream);
LT_API lt_status lt_rotate_volume_adjoint(lt_plan* plan, int32_t cam, const float* xc, float* x, int32_t accumulate,
                                          void* stream);

/* Plenoptic stages, exposed for testing and composition (eq. plenoptic,factor):
 *   stage 1:  fa[F][K][arr_nt][arr_ns] = M (1/V^a) sum_n B^{an}_k (dz x^n)
 *   stage 2:  y[F][M_c] = sum_k sum_mu B^{d mu}_k fa_k
 * and their adjoints (stage 2^T writes M sum_mu (B^{d mu}_k)^T y).
 * n_cells() gives K of a camera (kept angular cells). */
LT_API lt_status lt_camera_cells(const lt_plan* plan, int32_t cam, int32_t* n_cells);
LT_API lt_status lt_plenoptic_stage1(lt_plan* plan, int32_t cam, const float* x, float* fa, void* stream);
LT_API lt_status lt_plenoptic_stage1_adjoint(lt_plan* plan, int32_t cam, const float* fa, float* x,
                                      int32_t accumulate, void* stream);
LT_API lt_status lt_plenoptic_stage2(lt_plan* plan, int32_t cam, const float* fa, float* y_cam, void* stream);
LT_API lt_status lt_plenoptic_stage2_adjoint(lt_plan* plan, int32_t cam, const float* y_cam, float* fa,
                                      void* stream);

/* Autotuner (no counterpart in the paper): times each forward kernel variant
 * on this plan's own cameras and frames and keeps the fastest for later
 * calls.  Variants 0-4 are the direct beam kernel's shapes (slices per
 * weight batch x warp groups per work item); variant 5, the default of a new
 * plan, is the brick-staged kernel (volume bricks brought to shared memory
 * by TMA, one warp per slice), which cameras whose bricks the planner could
 * not size, or whose source rows are not a multiple of 4 floats, replace by
 * variant 2.  Allocates and
 * frees temporary device buffers and synchronises the stream; call it once
 * after lt_plan_create and before capturing graphs.  times_ms (host array of
 * lt_autotune_variants() entries, may be NULL) receives each variant's best
 * time; *chosen (may be NULL) the index kept. */
LT_API int32_t lt_autotune_variants(void);
LT_API lt_status lt_plan_autotune(lt_plan* plan, void* stream, double* times_ms, int32_t* chosen);
/* Pins the forward variant (0 .. lt_autotune_variants()-1) instead of tuning;
 * every variant computes the same operator (summation order differs).  A new
 * plan uses variant 2 (two slices per weight batch, two warp groups). */
LT_API lt_status lt_plan_set_forward_variant(lt_plan* plan, int32_t variant);

/* Device-side status word of the projector kernels (no counterpart in the
 * paper): bit 0 = a brick or band of the brick-staged forward did not fit
 * its planned size (that slice's weights were zeroed; the planner sizes
 * them so that this does not happen), bit 1 = a bounded wait for a TMA load
 * gave up (the kernel stopped taking work).  0 after correct runs.  Reading
 * synchronises the device; clear != 0 resets the word. */
LT_API lt_status lt_projector_status(int32_t* flags, int32_t clear);

/* Adjoint kernel choice (no counterpart in the paper): 1 (default) = the
 * box-staged gather adjoint (each image box a voxel tile reads over a chunk
 * of slices brought to shared memory once by TMA) where the camera fits it,
 * 0 = the direct gather adjoint.  Both compute the same operator (summation
 * order differs).  LT_EINVAL for another value. */
LT_API lt_status lt_plan_set_adjoint_variant(lt_plan* plan, int32_t variant);

/* Adjoint kernel choice by measurement (no counterpart in the paper): times
 * the plan's whole adjoint (every camera and frame, stage two and the
 * transposed rotations included) with variant 1 (box-staged, where a camera
 * fits it) and variant 0 (direct gather), three timed runs each after a
 * warm-up, and keeps the faster (lt_plan_set_adjoint_variant).  times_ms
 * (host array of 2 entries, indexed by variant, may be NULL) receives the
 * best time of each; *chosen (may be NULL) the variant kept.  Allocates and
 * frees temporary device buffers and synchronises the stream: call it after
 * lt_plan_create and before capturing graphs.  Errors: LT_EINVAL (NULL
 * plan), LT_ENOMEM, LT_ECUDA; on an error the previous choice stays. */
LT_API lt_status lt_plan_autotune_adjoint(lt_plan* plan, void* stream, double* times_ms, int32_t* chosen);

/* Analytic work counts of one camera for one frame, computed on the host in
 * float64 from the plan's footprints (used for throughput and roofline
 * figures).  A ray-sample is one (beam, slice) pair: a beam is a target pixel
 * and an angular cell (Sec. II-B); stage 1 = slices -> detector (single lens)
 * or array plane (plenoptic), stage 2 = array plane -> detector (plenoptic,
 * one sample per detector pixel and cell).  nnz counts the nonzero matrix
 * entries each stage evaluates (the separable s x t footprint products). */
typedef struct {
  int64_t n_cells;          /* K                                              */
  int64_t stage1_samples;   /* target pixels x K x nz                         */
  int64_t stage2_samples;   /* det pixels x K (plenoptic), else 0             */
  int64_t ray_samples;      /* stage1_samples + stage2_samples                */
  int64_t hit_samples;      /* stage-1 samples whose footprint meets the volume */
  int64_t stage1_nnz;       /* nonzero (pixel, cell, voxel) entries of stage 1 */
  int64_t stage2_nnz;       /* nonzero (pixel, cell, array pixel) entries      */
  int64_t stage1_tile_voxels; /* sum over 32 x 32 target-pixel tiles, cells and
                             * slices of the voxels the tile's footprints
                             * touch: what a tiled stage 1 must bring on chip
                             * once per (tile, cell, slice)                   */
  int64_t forward_brick;    /* floats per brick of the brick-staged forward
                             * (box columns x rows), 0 if the camera takes the
                             * direct kernel                                   */
  int64_t adjoint_box;      /* floats per image box of the box-staged adjoint,
                             * 0 if the camera takes the direct adjoint        */
  int64_t adjoint_chunk;    /* slices per box of the box-staged adjoint (8, or
                             * 4 where an 8-slice box would exceed its cap)    */
  int64_t forward_band;     /* 1 if the brick-staged forward takes its
                             * t-contraction in band form (footprints of three
                             * or more taps), 0 if per pixel row or direct     */
} lt_camera_stats;

LT_API lt_status lt_camera_stats_get(const lt_plan* plan, int32_t cam, lt_camera_stats* out);

/* ------------------------------------------------------------------------
 * Reconstruction (Sec. V, Table V): penalised weighted non-negative least
 * squares with unknown camera gains (eq. pls), solved by FISTA with the
 * diagonal majoriser D = diag(sum_c A_c^T W_c A_c 1) (Appendix A).  Every
 * frame of the plan is an independent problem.
 * ------------------------------------------------------------------------ */
typedef struct lt_recon lt_recon;

typedef struct {
  double beta;            /* regulariser weight (eq. reg)                       */
  double nu;              /* l1 weight; x = [w - nu]_+ as in Table V            */
  int32_t psi;            /* 0: psi(t) = t^2/2; 1: delta^2 (sqrt(1+(t/delta)^2)-1) */
  double psi_delta;       /* delta of the hyperbola                             */
  double reg_scale;       /* curvature bound: 26 (as printed) or 36 (exact)     */
  int32_t estimate_gains; /* 1: gamma_c (c > 0) per Table V step 1b; 0: all 1   */
  int32_t n_subset;       /* view subsets (Sec. V, eq. subset); 0 or 1 = none.
                           * Iteration i (0-based) uses the cells k with
                           * k % n_subset == i % n_subset of every camera c and
                           * a_c = K_c / |S_c|: p_c = a_c sum_{k in S} A_ck z,
                           * the gain from p_c, g_c = a_c sum_{k in S} A_ck^T
                           * W (p_c - gamma_c y_c); D stays the full majoriser.
                           * A camera with an empty subset adds no gradient. */
} lt_recon_params;

/* Copies y (device [F][M]) and the optional weights w (device [F][M], NULL =
 * W = I) and computes D (one forward and one adjoint).  x0: optional device
 * [F][N] initial x = z (NULL = 0, as in Table V).  Allocates the solver state
 * on the device.  Errors: LT_EINVAL (NULL plan/y/params, negative beta/nu,
 * psi_delta <= 0 with psi = 1), LT_ENOMEM, LT_ECUDA. */
LT_API lt_status lt_recon_create(lt_plan* plan, const float* y, const float* w,
                                 const lt_recon_params* params, const float* x0,
                                 void* stream, lt_recon** out);

/* Runs n_iter iterations of Table V on the stream.  The first call captures
 * one iteration into a CUDA graph (one per z buffer parity) that later calls
 * replay; no host synchronisation happens inside. */
LT_API lt_status lt_recon_iterate(lt_recon* rec, int32_t n_iter, void* stream);

/* Copies the current x (device [F][N], may be NULL), and, synchronising the
 * stream, the gains (host [F][n_cams] or NULL) and the data-fit term
 * 1/2 sum_c ||A_c z - gamma_c y_c||^2_W of the last iteration (host [F] or
 * NULL; 0 before the first iteration). */
LT_API lt_status lt_recon_get(lt_recon* rec, float* x, double* gains, double* data_fit,
                              void* stream);

/* The same data fit and gains without synchronising: enqueues on the stream
 * a device reduction into host_out = [data_fit[F], gains[F][n_cams]]
 * (F + F * n_cams doubles), valid once the stream has passed this point (an
 * event or a synchronise).  Page-locked host_out (cudaHostAlloc, or a pinned
 * torch tensor) is written by the reduction kernel itself through its
 * device mapping, so nothing on the stream waits for a copy engine; other
 * memory is filled by a copy after the reduction.  host_out must stay
 * alive until then.  For pipelined use: read step i's result while step
 * i + 1 runs. */
LT_API lt_status lt_recon_get_async(lt_recon* rec, double* host_out, void* stream);

/* Replaces the measurements (and weights, if w is not NULL; the majoriser D
 * is then recomputed) of an existing reconstruction without resetting x, z,
 * t or the iteration count: for streams of frames where each new image warm
 * starts from the previous estimate.  Asynchronous on the stream. */
LT_API lt_status lt_recon_set_data(lt_recon* rec, const float* y, const float* w, void* stream);

/* Number of kernel launches one iteration performs (the nodes of its graph). */
LT_API lt_status lt_recon_kernels_per_iteration(lt_recon* rec, int32_t* n);

/* Iterations completed so far. */
LT_API lt_status lt_recon_iterations(const lt_recon* rec, int64_t* n_iter);

/* Checkpoint / resume: the solver state (x, z, t, gains, iteration count) as
 * an opaque host byte buffer of lt_recon_state_size bytes.  Synchronous. */
LT_API lt_status lt_recon_state_size(const lt_recon* rec, int64_t* bytes);
LT_API lt_status lt_recon_get_state(lt_recon* rec, void* host_buf);
LT_API lt_status lt_recon_set_state(lt_recon* rec, const void* host_buf);

/* Frees the solver's device state (D, x, z, scratch, captured graphs) after
 * synchronising the device; the plan it was created on is not freed.
 * NULL is accepted and ignored. */
LT_API lt_status lt_recon_destroy(lt_recon* rec);

/* Description of the last error on the calling thread ("" if none). */
LT_API const char* lt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LT_H */
