/*
 * recon.h -- C-ABI of the GB300 layered unified tomographic reconstruction (UTR).
 *
 * Gureyev, Brown, Quiney, Allen, "Fast unified reconstruction algorithm for
 * conventional, phase-contrast and diffraction tomography" (arXiv 2206.09151).
 *
 * The operator, per plane-wave illumination direction n (any scan geometry, Sec. 2):
 *   g_n      = ln(I_n / I_in)                                  (left side of Eq. 4)
 *   G_n      = 2D DFT of g_n zero-padded to P x P, kernel exp(-i 2 pi r.q)      (Eq. 3)
 *   chi_k(q) = pi lambda (R_n - z_k) q^2 + (pi/2) Cs lambda^3 q^4 - omega,
 *              omega = atan(sigma)                                 (Eq. 5, Eq. 7)
 *   H_k(q)   = lambda / (4 pi sqrt(1+sigma^2)) * sin chi_k / (sin^2 chi_k + eps)
 *              (the real part of the bracket of Eq. 11 at layer k's own defocus;
 *               Eq. 13 when Nz = 1 and eps = 0)
 *   W(q)     = (pi / D) * ramp |q_u| as the band-limited Ram-Lak kernel (Sec. 2:
 *               the sampling-matrix inverse of a single-axis scan)
 *   Y_{n,k}  = crop_N( Re IDFT[ G_n H_k W ] )                     -- the layer stack
 *   vol(r)  += bilinear( Y_{n, k(r)}, u_n(r), v_n(r) )  over all n -- layered backprojection
 * with k(r) the depth layer containing voxel r along direction n.  Nz = 1 with the
 * filter off is conventional filtered backprojection (Eq. 15).
 *
 * Conventions: volume vol[z][y][x] float32, voxel (i,j,k) centred at
 * ((i-(nx-1)/2) delta, (j-(ny-1)/2) delta, (k-(nz-1)/2) delta).  rot[n] is a row-major
 * 3x3 rotation volume frame -> beam frame; its rows are the detector u axis, the
 * detector v axis and the beam direction.  Images img[n][v][u] float32, pixel (u, v) at
 * ((u-(nu-1)/2) delta, (v-(nv-1)/2) delta) in the beam frame.  Defocus R_n is measured
 * from the plane through the rotation centre, positive downstream.  Depth layers are
 * Nz equal slabs over the volume's bounding-box extent along the beam; the layer of a
 * voxel is floor of a 2^-24 fixed-point depth coordinate (exact integer arithmetic).
 *
 * Errors: every entry point returns RECON_OK (0) or a negative code; no exception
 * crosses the ABI.  recon_last_error() gives a message for the calling thread's last
 * failure.  Kernels run asynchronously on the caller's stream: an error inside a
 * kernel surfaces at the next call that synchronises (recon_sync) or in a later
 * launch check.
 *
 * Threading: a plan is immutable after recon_plan and may be used from several host
 * threads, but two runs that share one workspace must not overlap on the GPU.
 */
#ifndef RECON_H_
#define RECON_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define RECON_OK 0
#define RECON_E_INVALID_ARG (-1)      /* null pointer, bad size, bad enum, bad geometry */
#define RECON_E_UNSUPPORTED_SIZE (-2) /* a size beyond the library's limits            */
#define RECON_E_CUDA (-3)             /* a CUDA runtime call or a launch failed        */
#define RECON_E_WORKSPACE (-4)        /* workspace too small or not 256-byte aligned    */
#define RECON_E_NO_MEMORY (-5)        /* host allocation failed                         */
#define RECON_E_NONFINITE (-6)        /* an image holds NaN or Inf (checked only when the
                                         plan's check_finite option is set)             */
#define RECON_E_NO_WEIGHTS (-7)       /* RECON_FILTER_MLP without its network parameters */
#define RECON_E_DEVICE_CHECK (-8)     /* a kernel's own check failed: a bounded wait ran out
                                         (2 s) or a footprint left its staging box; the call
                                         synchronised its stream and the output is incomplete */

/* ---------------------------------------------------------------- option values */
#define RECON_FILTER_OFF 0       /* H = 1: ramp-filtered backprojection of g (Eq. 15)   */
#define RECON_FILTER_TIKHONOV 1  /* H_k above (real part of Eq. 11, per layer)         */
#define RECON_FILTER_MLP 2       /* H_k with eps from the learned network (see below)   */
#define RECON_FILTER_PAIR 3      /* the opposite-pair form of Eq. 10 / Eq. 11: per layer
                                    lambda / (4 pi sqrt(1+sigma^2)) Re{[sin chi / (sin^2 chi
                                    + eps) - i cos chi / (cos^2 chi + eps)] exp(-i pi lambda
                                    z_k q^2)} with chi at the view's image plane (R_n, Cs,
                                    omega); exact (eps -> 0) only when the scan holds each
                                    view's opposite (360-degree or full-sphere scans)       */

/* Parameters of the learned regulariser: a 3 -> 64 -> 64 -> 1 ReLU network, float32,
 * laid out W1[64][3], b1[64], W2[64][64], b2[64], w3[64], b3. */
#define RECON_MLP_PARAMS 4481

#define RECON_INPUT_INTENSITY 0  /* images are I/I_in; g = ln(max(I/I_in, 1e-6))       */
#define RECON_INPUT_CONTRAST 1   /* images already are g (a contrast or a projection)  */

#define RECON_STACK_F32 0        /* layer stack stored in float32                       */
#define RECON_STACK_BF16 1       /* layer stack stored in bfloat16 (FP32 FFT/accumulate) */

#define RECON_RAMP_SINGLE_AXIS 0 /* ramp along u; every rot[n] must share one row 1 (axis) */
#define RECON_RAMP_DENSITY 1     /* any geometry: W = g / (S(q) + eps_S), S the gridded
                                    sampling density of all views' slices (Sec. 2)        */

#define RECON_LAYER_NEAREST 0    /* a voxel takes the layer that contains its depth      */
#define RECON_LAYER_LINEAR 1     /* the linear blend of the two layers whose centres
                                    bracket its depth (layer k centred at k + 1/2 in layer
                                    units; the outer layer alone beyond the outer centres);
                                    four row gathers per sample instead of two, in the
                                    general backprojection kernel for every geometry      */

#define RECON_BP_AUTO 0          /* the variant measured faster on sm_103a: DIRECT for a
                                    single axis along y with the nearest layer, TMA for
                                    every other case where its footprint box fits shared
                                    memory (else the general direct kernel)              */
#define RECON_BP_DIRECT 1        /* bilinear gathers straight from the stack (single-axis
                                    kernel, or the general kernel)                       */
#define RECON_BP_STAGED 2        /* single-axis: footprint staged in shared memory        */
#define RECON_BP_TMA 3           /* any geometry: each (16 x 16 x 16 voxel tile, direction)
                                    footprint box copied into a shared-memory ring by one
                                    TMA load (cp.async.bulk.tensor), gathers from shared
                                    memory; the call then reads a device status word back
                                    (one 4-byte copy and a stream synchronisation)        */

/* Limits (RECON_E_UNSUPPORTED_SIZE beyond them). */
#define RECON_MAX_IMAGE 1024     /* nu, nv <= 1024, so P <= 2048                        */
#define RECON_MAX_LAYERS 96      /* 1 <= nz_layers <= 96                                */
#define RECON_MAX_GRID 4096      /* nx, ny, nz <= 4096                                  */

/* ---------------------------------------------------------------- types */
typedef struct recon_plan_s* recon_plan_t;

typedef struct {
  int nx, ny, nz; /* voxels along x, y, z; pitch = delta */
} recon_grid;

typedef struct {
  int n_dir;         /* D >= 0 directions (D = 0: run writes zeros, or leaves vol)   */
  int nu, nv;        /* image width (u, fastest) and height (v), pixels of pitch delta */
  const double* rot; /* host, [n_dir][3][3] row-major, volume -> beam frame; copied  */
} recon_geometry;

typedef struct {
  double sigma;    /* beta/delta of the monomorphous object (Eq. 7); omega = atan(sigma) */
  double eps;      /* Tikhonov parameter of Eq. 11, > 0 when filter = TIKHONOV or PAIR  */
  double cs;       /* spherical aberration Cs (metres), 0 = none                        */
  int filter;      /* RECON_FILTER_*                                                    */
  int input_mode;  /* RECON_INPUT_*                                                     */
  int stack_dtype; /* RECON_STACK_*                                                     */
  int ramp_mode;   /* RECON_RAMP_* (single-axis ramp, or sampling-density weighting)       */
  int accumulate;  /* 0: run overwrites vol; 1: run adds into vol                       */
  int dir_block;   /* directions per block (stack held in workspace), 0 = automatic    */
  const float* mlp_weights; /* host [RECON_MLP_PARAMS], copied; needed by RECON_FILTER_MLP  */
  double nsr;      /* noise-to-signal ratio of one image pixel (the NSR of Sec. 3); sets
                      the Poisson floor (nsr M)^2 per DFT coefficient of the SNR feature   */
  int stage_block; /* directions per FFT/filter sub-block (their spectra and per-layer
                      intermediates sized for it), 0 = the whole direction block           */
  int bp_kernel;   /* RECON_BP_*: backprojection variant.  DIRECT / STAGED choose between the
                      single-axis kernels (other geometries then use the general direct
                      kernel); TMA runs the TMA-staged kernel for every geometry; AUTO picks
                      the measured-faster kernel for the geometry on sm_103a                 */
  int check_finite; /* 1: recon_run (and recon_run_noalloc) first scans the images for NaN / Inf on the GPU, waits
                       for the scan (the call then synchronises its stream) and returns
                       RECON_E_NONFINITE without touching the volume if it finds any; 0: no
                       scan (a NaN then propagates into the voxels it reaches)             */
  int layer_interp; /* RECON_LAYER_*: nearest layer, or the blend of the two bracketing ones */
  int bp_warp;      /* general backprojection: a warp's patch of voxel columns is bp_warp (x)
                       by 32 / bp_warp (y) of its 32 x 8 tile; 8, 16 or 32, 0 = 8 (measured
                       fastest on the slab; the autotuner can time the others)              */
  double mlp_views; /* RECON_FILTER_MLP: views averaged per voxel (a full scan's D); the
                       network's eps, a per-view noise-to-signal power (Wiener), is divided by
                       it, since the reconstruction averages that many independent views;
                       0 or 1 = a single view's eps                                          */
  int bp_tile_z;    /* TMA-staged backprojection: the voxel tile is 16 x 16 x bp_tile_z, 8 or
                       16; 0 = 16 (measured faster on the slab; the autotuner can time 8)   */
} recon_options;

/* Fills *opts with defaults: sigma 0, eps 0.1 (the value of Sec. 3), cs 0, Tikhonov
 * filter, intensity input, float32 stack, single-axis ramp, overwrite, automatic
 * block, no finiteness scan, nearest layer.  No error (opts NULL is ignored). */
void recon_default_options(recon_options* opts);

/* Builds a plan (host memory only; no CUDA call, no device allocation).
 *   geom      geometry, rot copied                    lambda  wavelength (m), > 0
 *   delta     voxel and pixel pitch (m), > 0           defocus host [n_dir] R_n (m), copied
 *   nz_layers Nz depth layers, or 0 for the smallest Nz whose layers are no thicker
 *             than the depth of field (recon_layers_for_dof; recon_plan_layers reports it)
 *   grid      output volume size
 *   opts      NULL = recon_default_options
 * The per-direction FP64 tables are computed here: layer depths z_k and defocus
 * R_n - z_k (Eq. 5), the CTF phase constants (Eq. 7, Eq. 11), the ramp (Sec. 2).
 * Returns INVALID_ARG / UNSUPPORTED_SIZE / NO_MEMORY on failure (NO_WEIGHTS for
 * RECON_FILTER_MLP with mlp_weights NULL), *out untouched. */
int recon_plan(const recon_geometry* geom, double lambda, double delta, const double* defocus, int nz_layers,
               const recon_grid* grid, const recon_options* opts, recon_plan_t* out);

/* Device workspace bytes that recon_run needs for this plan (tables, spectra, one
 * block of layer stacks).  The caller allocates it (256-byte aligned). */
int recon_workspace_size(recon_plan_t plan, size_t* bytes);

/* Runs the whole operator on `stream` (a cudaStream_t, NULL = legacy default stream).
 *   images    device, float32 [n_dir][nv][nu], caller-owned, read only
 *   volume    device, float32 [nz][ny][nx], caller-owned, written (or added to)
 *   workspace device, >= recon_workspace_size bytes, 256-byte aligned, scratch
 * Asynchronous: returns once every kernel is queued, except where the plan runs the
 * TMA-staged backprojection (RECON_BP_TMA, or AUTO for a general geometry or the layer
 * blend): the call then synchronises `stream` at its end to read that kernel's status
 * word (RECON_E_DEVICE_CHECK if a bounded wait ran out).  Uses the current CUDA device. */
int recon_run(recon_plan_t plan, const float* images, float* volume, void* workspace, size_t ws_bytes,
              void* stream);

/* recon_run with the images in host memory, their upload overlapped with the compute:
 * block b + 1's images are copied (cudaMemcpyAsync on a stream of the plan's own) into one
 * of two device slots while block b is reconstructed on `stream`.
 *   host_images host, float32 [n_dir][nv][nu]; page-locked (cudaHostAlloc / pinned) for
 *             the copies to overlap (pageable memory works, copied without overlap); it must
 *             stay valid until the work queued on `stream` has finished
 *   workspace device, >= recon_run_host_workspace_size bytes (recon_workspace_size plus
 *             two image slots of the plan's direction block), 256-byte aligned
 * Same result as recon_run on the same images.  The plan keeps the copy stream and five
 * events (created on the first call, on the current device), so one plan must not run
 * recon_run_host from two threads at once.  check_finite is not supported here
 * (RECON_E_INVALID_ARG).  Asynchronous like recon_run (including its end-of-call status read
 * for the TMA-staged backprojection). */
int recon_run_host_workspace_size(recon_plan_t plan, size_t* bytes);
int recon_run_host(recon_plan_t plan, const float* host_images, float* volume, void* workspace, size_t ws_bytes,
                   void* stream);

/* Stage A alone (Sec. 2, Eq. 4-11 per layer): the layer stacks of directions
 * [dir_begin, dir_begin + dir_count), dir_count <= the plan's block size, into the
 * workspace.  *stack_out receives a device pointer into the workspace, laid out
 * [dir_count][Nz][nv + 2][su] of horizontal tap pairs (two float32, or two bfloat16, per
 * stack_dtype), su = nu + 1 rounded up to a multiple of 4 (every row starts on a 16-byte
 * boundary): entry [n][k][v + 1][c] = (Y_{n,k}(c - 1, v), Y_{n,k}(c, v)) for c in [0, nu],
 * with Y = 0 outside the image; rows 0 and nv + 1 are zero; entries c > nu are padding
 * (not written, never read). */
int recon_filter_stage(recon_plan_t plan, const float* images, int dir_begin, int dir_count, void* workspace,
                       size_t ws_bytes, void* stream, const void** stack_out);

/* Stage B alone: layered backprojection of the stacks of directions
 * [dir_begin, dir_begin + dir_count) held at `stack` (layout of recon_filter_stage)
 * into `volume` (added when accumulate != 0, else overwritten).  The workspace holds
 * the direction tables, so it must be the one recon_filter_stage used, or any
 * workspace of recon_workspace_size bytes. */
int recon_backproject(recon_plan_t plan, const void* stack, int dir_begin, int dir_count, float* volume,
                      int accumulate, void* workspace, size_t ws_bytes, void* stream);

/* Self-test of the failure detection of the TMA-staged backprojection: launches it on
 * one voxel tile whose producer issues no copy, so every consumer's wait on its
 * stage runs out after the 2 s limit; the kernel then sets its status bit and returns
 * without touching the GPU's state.  Allocates and frees 16 KB of device memory and
 * synchronises `stream`.  RECON_OK when the kernel reported the run-out wait (the
 * expected outcome, after about 2 s), RECON_E_DEVICE_CHECK if it did not, RECON_E_CUDA
 * on a CUDA error. */
int recon_selftest_wait_limit(void* stream);

/* ---------------------------------------------------------------- batches
 * Many tomograms of uneven sizes (each with its own plan: grid, images, directions,
 * layers, filter) reconstructed together.  Directions are taken in rounds of
 * `dir_block` (0 = 32) per tomogram: in each round every tomogram's stage A writes its
 * layer stacks, then ONE persistent backprojection kernel takes (tomogram, voxel tile)
 * items from an atomic counter until all are done.  The workspace holds every plan's
 * tables, one stack slot per tomogram and shared stage-A scratch.
 *   recon_batch_run        uploads tables and descriptors (host copies) and launches.
 *   recon_batch_run_graph  the same launches captured once as a CUDA graph on `stream`
 *                          (a created stream, not the legacy default) and replayed on
 *                          later calls with the same pointers; the tables and descriptors
 *                          stay in the workspace, which must not be reused in between.
 * The plans must outlive the batch.  Images and volumes as in recon_run, one per plan. */
typedef struct recon_batch_s* recon_batch_t;
int recon_batch_create(int n, const recon_plan_t* plans, int dir_block, recon_batch_t* out);
int recon_batch_workspace_size(recon_batch_t batch, size_t* bytes);
int recon_batch_run(recon_batch_t batch, const float* const* images, float* const* volumes, void* workspace,
                    size_t ws_bytes, void* stream);
int recon_batch_run_graph(recon_batch_t batch, const float* const* images, float* const* volumes, void* workspace,
                          size_t ws_bytes, void* stream);
/* The batch with its images in host memory: round r + 1's images (every tomogram's
 * directions of that round) are copied on a stream of the batch's own into one of two
 * device round slots while round r runs on `stream`.  host_images: [n] host arrays laid out
 * as recon_run's images (page-locked for the copies to overlap; valid until the queued
 * work has finished); workspace >= recon_batch_run_host_workspace_size bytes (the batch
 * workspace plus two round slots).  Same volumes as recon_batch_run on the same images; not
 * captured as a graph.  One batch must not run it from two threads at once. */
int recon_batch_run_host_workspace_size(recon_batch_t batch, size_t* bytes);
int recon_batch_run_host(recon_batch_t batch, const float* const* host_images, float* const* volumes, void* workspace,
                         size_t ws_bytes, void* stream);
int recon_batch_destroy(recon_batch_t batch); /* NULL is a no-op */
/* One-call form: create, run, destroy (default rounds of 32 directions). */
int recon_run_batch_workspace_size(int n, const recon_plan_t* plans, size_t* bytes);
int recon_run_batch(int n, const recon_plan_t* plans, const float* const* images, float* const* volumes,
                    void* workspace, size_t ws_bytes, void* stream);

/* The backprojection kernel that recon_run, recon_backproject and recon_swap_ct of this
 * plan launch (the resolution of RECON_BP_AUTO): RECON_BP_DIRECT (the single-axis or the
 * general direct kernel), RECON_BP_STAGED or RECON_BP_TMA.  No CUDA call. */
int recon_plan_bp_kernel(recon_plan_t plan, int* kernel);

/* Depth of field (Sec. 1): DOF = delta^2 / (2 lambda).  Layers thinner than the DOF
 * keep every voxel within its layer's focus; a thicker layer is the plan-time warning of
 * a shallow-DOF scan under too few layers.
 *   recon_plan_dof      *pitch_max = the largest layer pitch h_n = T_n / Nz over the
 *                       directions (T_n the bounding-box extent along beam n, metres),
 *                       *dof = Delta^2 / (2 lambda); either pointer may be NULL.
 *   recon_plan_warning  "" when pitch_max <= dof, else a message with both figures (the
 *                       string lives as long as the plan).
 *   recon_layers_for_dof  the smallest Nz (capped at RECON_MAX_LAYERS) whose layer pitch
 *                       is <= DOF for every direction of `geom` over `grid` (1 when the
 *                       scan has no direction). */
int recon_plan_dof(recon_plan_t plan, double* pitch_max, double* dof);
/* The plan's number of depth layers (the automatic choice when recon_plan had 0). */
int recon_plan_layers(recon_plan_t plan, int* nz_layers);
const char* recon_plan_warning(recon_plan_t plan);
int recon_layers_for_dof(const recon_geometry* geom, const recon_grid* grid, double lambda, double delta, int* nz);

/* ---------------------------------------------------------------- 3D-Fourier forms
 * Eq. 12 (Sec. 2): with one defocus R for every view, the CT reconstruction comes first and
 * the CTF inversion is one 3D filter after it, so another (sigma, eps) reruns only that.
 *   recon_swap_ct     the CT step: the layered reconstruction of the contrasts with the
 *                     Ewald placement and no CTF (per layer cos and sin of pi lambda z_k q^2:
 *                     two real volumes V_c, V_s), packed as V_c + i V_s into a grid zero-
 *                     padded to P3 = the next power of two >= 2 n per axis and transformed;
 *                     the spectrum stays in the workspace.  The plan must use
 *                     RECON_FILTER_PAIR (its depth tables) and one defocus for every view.
 *   recon_swap_phase  the CTF inversion of the kept spectrum: F3 delta = lambda / (4 pi
 *                     sqrt(1+sigma^2)) [s' F3 V_c - c' F3 V_s], s' = sin chi / (sin^2 chi +
 *                     eps), c' = cos chi / (cos^2 chi + eps), chi at the in-plane frequency
 *                     of each 3D frequency's Ewald-paraboloid point (the plan's Cs); inverse
 *                     transform, crop into volume [nz][ny][nx].  Needs a workspace on which
 *                     recon_swap_ct has run; can run any number of times.
 * The Fourier-gridding UTR (Sec. 2 after Eq. 11; Sec. 3 for the noise filter):
 *   recon_grid_run    every 2D DFT coefficient of every view times Eq. 11's bracket at the
 *                     view's own R_n, spread with trilinear weights onto the 8 cells around
 *                     its point Rot_n^T (q_u, q_v, -lambda q^2 / 2) of the padded volume's DFT
 *                     grid; divided by S + eps_S (S the summed weights, eps_S = 1e-3 x its
 *                     mean over the non-empty cells); nsr > 0 zeroes the coefficients whose
 *                     gridded contrast (the same splat without the bracket, over S + eps_S)
 *                     is below nsr M / sqrt(S), M^2 = nu nv; inverse transform, crop.  Any
 *                     geometry; the plan's sigma, eps, cs and input mode; its filter must be
 *                     TIKHONOV or PAIR (eps > 0).
 * The caller owns images, volume and workspace (256-byte aligned, of the *_workspace_size
 * bytes).  Limits: every grid side <= 1024 (UNSUPPORTED_SIZE beyond), images of more than
 * 8 pixels. */
int recon_swap_workspace_size(recon_plan_t plan, size_t* bytes);
int recon_swap_ct(recon_plan_t plan, const float* images, void* workspace, size_t ws_bytes, void* stream);
int recon_swap_phase(recon_plan_t plan, double sigma, double eps, float* volume, void* workspace, size_t ws_bytes,
                     void* stream);
int recon_grid_workspace_size(recon_plan_t plan, size_t* bytes);
int recon_grid_run(recon_plan_t plan, const float* images, float* volume, double nsr, void* workspace,
                   size_t ws_bytes, void* stream);

/* Plan facts: padded FFT size P, directions per block, number of blocks, directions per
 * FFT/filter sub-block (any pointer may be NULL). */
int recon_plan_info(recon_plan_t plan, int* padded, int* dir_block, int* n_blocks, int* stage_block);

/* The learned regulariser (RECON_FILTER_MLP).  eps of Eq. 11 (chosen "ad hoc" in
 * Sec. 3) becomes eps_theta = softplus(network(x)) per (direction, layer, radial bin b),
 * bins b = min(isqrt(m_u^2 + m_v^2) / w, n_b - 1), w = max(1, P/128).  Inputs x:
 * log10(SNR_b)/3 clamped to [-1, 2], with SNR_b the radial power of the image spectrum
 * over the Poisson floor nsr^2 nu nv (the Parseval scaling of Sec. 3's noise filter);
 * the bin-centre radius / (P/2); lambda (R_n - z_k) / delta^2 / 100.
 *
 * recon_mlp_train fits the parameters on training images with known layer contents:
 * it minimises sum over images n, layers k and frequencies q of |H_nk(q) G_n(q) -
 * T_nk(q)|^2 / sum |T_nk(q)|^2 (G: DFT of the contrast, T: DFT of the true projection of
 * layer k's slab, in metres) with Adam (beta 0.9 / 0.999), on the GPU.  steps = 0
 * returns the loss and (if grad != NULL) its gradient at the given weights.  The call
 * waits for `stream` before returning.  The loss is over the call's images (full batch);
 * a training set larger than one workspace is fed as mini-batches in successive calls
 * that pass the same adam_state and advance adam_step by steps each time. */
typedef struct {
  int n_img, nu, nv, nz_layers;  /* training images, image size, layers per image        */
  const double* rot;             /* host [n_img][9] rotations (as in recon_geometry)      */
  const double* defocus;         /* host [n_img] R_n (m)                                  */
  int grid_nx, grid_ny, grid_nz; /* volume whose bounding box defines the layers         */
  double lambda, delta, sigma, cs, nsr;
  int input_mode;                /* RECON_INPUT_*                                         */
  const float* images;           /* device [n_img][nv][nu]                                */
  const float* targets;          /* device [n_img][nz_layers][nv][nu] layer projections   */
  int steps;                     /* Adam steps                                            */
  float lr;                      /* Adam step size                                        */
  float* adam_state;             /* host [2 RECON_MLP_PARAMS]: Adam's first and second
                                    moments, read at the start and written back at the end
                                    (mini-batches in successive calls continue one
                                    optimisation), or NULL: fresh moments, not returned     */
  int adam_step;                 /* Adam steps taken before this call (bias correction)   */
} recon_train_cfg;

int recon_mlp_train_workspace_size(const recon_train_cfg* cfg, size_t* bytes);
/* weights: host [RECON_MLP_PARAMS] in/out; loss_history: host [max(steps, 1)], the loss
 * before each step; grad: host [RECON_MLP_PARAMS] or NULL (filled when steps = 0). */
int recon_mlp_train(const recon_train_cfg* cfg, float* weights, float* loss_history, float* grad, void* workspace,
                    size_t ws_bytes, void* stream);

/* Optional kernel timing.  While enabled, recon_run records CUDA events on its
 * stream around each kernel of each direction block (row FFTs, column filter/iFFTs,
 * row iFFTs, backprojection).  recon_profile_read waits for the last run's events
 * and returns the summed milliseconds of each kernel over that run (ms[4], in the
 * order above) and the number of launches of each (launches[4]).  The events live
 * in the plan (created on enable, destroyed with the plan); a plan being profiled
 * must not run on two streams at once. */
int recon_profile_enable(recon_plan_t plan, int enable);
int recon_profile_read(recon_plan_t plan, double* ms, int* launches);

/* Size of the static device scratch that recon_run_noalloc works in (32 MiB). */
#define RECON_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* recon_run without any device allocation.  The paper has no counterpart: this is a
 * service for callers that may not allocate GPU memory themselves -- a component that
 * lives inside a host application which has already divided the device memory among
 * its parts, a real-time acquisition loop in which cudaMalloc/cudaFree are banned
 * because they can synchronise the device and stall the frame stream, or a plugin in a
 * process whose allocator owns every byte.  The caller still passes the device images
 * and volume (same layout and meaning as recon_run); the plan tables, spectra,
 * intermediates and layer stacks live in one static 32 MiB device array compiled into
 * the library, which every GPU that loads the library keeps until the process exits.
 * Directions are processed in the largest block that fits that array.
 *   Limit: a plan whose table head plus one direction's scratch exceeds
 *   RECON_NOALLOC_SCRATCH_BYTES is refused with RECON_E_UNSUPPORTED_SIZE and a message
 *   giving both sizes.
 *   Set-up: every call looks up the array's device address (cudaGetSymbolAddress) on
 *   the current device, so the address stays right after a cudaDeviceReset.
 *   Streams: the call copies the plan tables from pageable host memory with
 *   cudaMemcpyAsync, which stream capture rejects, so it must not be called while
 *   `stream` is being captured into a CUDA graph.
 *   Sharing: all calls share the one array and it keeps the last call's contents;
 *   nothing in it needs to start at zero (every kernel writes what it later reads), but
 *   two calls that overlap on the GPU (other streams, other threads) race on it.
 *   Kernels: the backprojection is always a direct-gather kernel (the plan's TMA-staged
 *   choice does not apply), so the call never synchronises `stream`.
 * Calls no cudaMalloc, cudaFree or allocating library routine. */
int recon_run_noalloc(recon_plan_t plan, const float* images, float* volume, void* stream);

/* Waits for `stream` and reports a CUDA error raised by earlier kernels. */
int recon_sync(void* stream);

/* Frees the plan.  NULL is a no-op. */
int recon_destroy(recon_plan_t plan);

/* Static text for a status code. */
const char* recon_error_string(int code);

/* Message of the calling thread's last failure ("" if none). */
const char* recon_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RECON_H_ */
