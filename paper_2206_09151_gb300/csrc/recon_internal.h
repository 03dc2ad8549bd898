// Internal types shared by the host plan and the CUDA kernels of the layered UTR path.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

struct recon_plan_s;

namespace recon {

// Streaming multiprocessors of the current device (launch sizing); 1 if the query fails.
inline int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
  return sms;
}

// Voxel tile of the general-geometry backprojection (i, j, k extents).
constexpr int kGenTile[3] = {32, 8, 8};
// Fixed-point scale of the detector coordinates in DirParams: 2^-40 pixel.
constexpr int kPixFracBits = 40;

// Per-direction constants, built by the plan from FP64 (one 128-byte record per direction).
struct DirParams {
  // detector u pixel a(i,j,k) = a[0] i + a[1] j + a[2] k + a[3] and v pixel b(i,j,k), each
  // coefficient rounded to 2^-40 pixel: a tile origin is an exact integer sum (error below
  // 1e-8 pixel at any grid size), formed without FP64 arithmetic on the device
  int64_t a[4];
  int64_t b[4];
  float af[3];      // FP32 copies of the steps a[0..2]
  float bf[3];      // FP32 copies of the steps b[0..2]
  int32_t t[4];     // depth in 2^-24 layer units: T0, Ti, Tj, Tk (exact integer sum)
  // extremes of a and b over a general-kernel tile relative to its origin, in 2^-16 pixel
  // (min a, max a, min b, max b, rounded outwards), and of t (min, max); INT32_MIN in
  // ab_ext[0] or t_ext[0] marks a direction whose extremes do not fit (no fast path)
  int32_t ab_ext[4];
  int32_t t_ext[2];
};
static_assert(sizeof(DirParams) == 128, "DirParams must stay 128 bytes");

// Constants of the sampling-density weighting (density.cuh).
struct DensityConst {
  int enabled;       // ramp_mode == RECON_RAMP_DENSITY
  int s;             // sampling step, DFT bins per cell
  int Gh, G;         // half width, side (2 Gh + 1)
  int n_samples1;    // P / s samples per image axis
  float inv_s;       // 1 / s
  float g_over_p2;   // g / P^2 (the inverse DFT's 1/P^2 folded in)
  float eps_scale;   // 1e-3 / (cells in the band)
};

// Constants of stage A (FFT -> per-layer filter -> inverse FFT -> stack).
struct StageAConst {
  int P, logP;          // padded FFT size and its log2
  int nu, nv;           // image size
  int nz_layers;        // Nz
  int filter;           // RECON_FILTER_* (2: eps from the learned table)
  int input_mode;       // RECON_INPUT_*
  int stack_bf16;       // 0: float32 stack, 1: bfloat16 stack
  uint64_t uC;          // Cs phase per m^2 as a fraction of 2 pi, 2^-64 units
  uint64_t uW;          // omega as a fraction of 2 pi, 2^-64 units
  float eps;            // Tikhonov eps
  float pref;           // lambda / (4 pi sqrt(1 + sigma^2))
  int half;             // P/2 + 1 (columns of the half spectrum)
  int su;               // stack row pitch in tap pairs, nu + 1
  size_t layer_elems;   // pairs per layer, (nv + 2) * (nu + 1)
  DensityConst dens;
  int sub_block;        // directions per stage-A sub-block (S and T sized for it), 0 = whole block
  int pair_mode;        // filter 3 only: 0 the opposite-pair bracket; 1 / 2 the depth factor
                        // cos / sin of pi lambda z_k q^2 alone (the CT step of Eq. 12)
};

// Device pointers into the workspace.
struct Workspace {
  DirParams* dirs;      // [D]
  uint64_t* uA;         // [D][Nz]: pi lambda (R_n - z_k)/(P delta)^2 per unit m, fraction of 2 pi
  float* ramp;          // [P/2+1]: ramp weight, includes pi/D and 1/P^2
  float2* tw;           // [P]: exp(-2 pi i j / P)
  float2* twp;          // [P - 8]: per-pass twiddles of the register FFT (fft_reg.cuh), P >= 16,
                        // then for P >= 256 [P - 16] of the 16-value FFT (fft16.cuh)
  float2* S;            // [DB][nv][P/2+1]: row transforms
  float2* T;            // [DB][Nz][P/2+1][nv]: per-layer column inverse transforms (column-major)
  void* stack;          // [DB][Nz][nv+2][nu+1] tap pairs (Y[v][u-1], Y[v][u]), zero outside
  float* dens;          // [G][G][G] sampling density S (density weighting only)
  double* band_sum;     // sum of S over the band (sets eps_S)
  float* eps;           // [DB][Nz][n_bins] learned regulariser (learned filter only)
  int n_bins, bin_width;
};

// Kernel launchers (stage_a.cu, backproject.cu).  They return cudaGetLastError().
// Optional work between the row FFTs and the column kernel (the learned regulariser's
// power spectrum and eps table).
struct StageAHook {
  cudaError_t (*fn)(void* ctx, int dir_begin, int dir_count, cudaStream_t stream);
  void* ctx;
};

// Optional kernel timing: an event is recorded after every launch and tagged with the
// kernel it ends (0 row FFTs and the learned hook, 1 column kernel, 2 row iFFTs,
// 3 backprojection); the interval between consecutive events is that kernel's time.
struct EventRecorder {
  cudaEvent_t* ev;
  int* kind;
  int n, cap;
  void mark(int k, cudaStream_t s) {
    if (n < cap) {
      cudaEventRecord(ev[n], s);
      kind[n] = k;
      ++n;
    }
  }
};

cudaError_t launch_stage_a(const StageAConst& c, const Workspace& ws, const float* images, int dir_begin,
                           int dir_count, cudaStream_t stream, EventRecorder* rec = nullptr,
                           const StageAHook* hook = nullptr);
// Adds to *count the number of NaN / Inf values among x[0..n).
cudaError_t launch_count_nonfinite(const float* x, size_t n, unsigned int* count, cudaStream_t stream);
// The row FFTs alone (S of `count` images starting at image `first`), P >= 16.
cudaError_t launch_rows_fwd(const StageAConst& c, float2* S, const float2* twp, const float* images, int first,
                            int count, cudaStream_t stream);

struct BackprojConst {
  int nx, ny, nz;
  int nu, nv, nz_layers;
  int su;
  size_t layer_elems;
  int stack_bf16;
  // Every view keeps the detector v axis on the volume y axis (rot row 1 = (0,1,0)
  // exactly): then v = j + b_off for every direction and the layer and u coordinate
  // are constant along a voxel column in y (the single-axis kernel).
  int axis_y;
  int b_int;      // floor(b_off)
  float b_frac;   // b_off - floor(b_off), 0 or 1/2
  int staged;     // single-axis kernel with shared-memory staging of each footprint
  int layer_linear;  // blend the two layers whose centres bracket the depth (general kernel)
  int warp_cols;     // general kernel: a warp's patch of voxel columns is warp_cols x 32/warp_cols
};

cudaError_t launch_backproject(const BackprojConst& c, const DirParams* dirs, const void* stack, int dir_begin,
                               int dir_count, float* volume, int accumulate, cudaStream_t stream);

// Footprint box of the TMA-staged backprojection: every (tile, direction) footprint of the
// plan's directions fits W pairs x H rows x L layers of the stack.
struct TmaBox {
  int W, H, L;        // box extents (W a multiple of 4, so a row of the box is 16-byte aligned)
  int stages;         // shared-memory ring depth
  size_t stage_bytes; // W H L entries rounded up to 128 bytes
  int ok;             // 0: the box is too large for the kernel (it then cannot be used)
  int tile_z;         // voxel tile 16 x 16 x tile_z (8 or 16)
};
TmaBox tma_box_for(const BackprojConst& c, const DirParams* dirs, int n_dirs, int tile_z);
// status: device word; bit 0 = a bounded wait ran out, bit 1 = a footprint outside its box
cudaError_t launch_backproject_tma(const BackprojConst& c, const TmaBox& box, const DirParams* dirs, const void* stack,
                                   int dir_begin, int dir_count, float* volume, int accumulate, unsigned int* status,
                                   cudaStream_t stream);
// Diagnostic launch whose producer issues nothing, so every consumer wait runs out (after
// its 2 s limit) and sets bit 0 of *status; buf: >= 10 KB of device memory, 256-byte aligned.
cudaError_t launch_tma_wait_probe(void* buf, size_t buf_bytes, unsigned int* status, cudaStream_t stream);

// One tomogram's share of a persistent batched backprojection: its constants, pointers,
// kernel kind (general 0/1, single-axis 2..5 (float32 / bfloat16 stack, one or two detector
// rows), general with the layer blend 6/7),
// tile grid and the index of its first work item.
struct BatchBp {
  BackprojConst c;
  const DirParams* dirs;
  const void* stack;
  float* vol;
  int dir_begin, dir_count, accumulate, kind;
  int gx, gy, gz;
  unsigned long long first_item;
  size_t smem;  // shared bytes its tiles need
};
void describe_backproject(const BackprojConst& c, const DirParams* dirs, const void* stack, int dir_begin,
                          int dir_count, float* volume, int accumulate, BatchBp* out);
cudaError_t launch_backproject_persistent(const BatchBp* desc_dev, int n_desc, unsigned long long total,
                                          unsigned long long* counter, size_t smem, cudaStream_t stream);

// The 3D-Fourier forms (fft3.cu, fourier.cu): a zero-padded complex grid [P3z][P3y][P3x]
// holding an n[0] x n[1] x n[2] volume at offset off (centred); scale[a] = P3[a] / P
// converts a 2D frequency in units of 1 / (P delta) to bins of grid axis a.
struct Fourier3Const {
  int P3[3];
  int n[3];
  int off[3];
  float scale[3];
  double lam, delta;
};
// Per view of the gridding: rows of Rot_n (detector u, v, beam), lambda / (2 P delta) (the
// paraboloid's depth per squared frequency bin), and the image-plane CTF phase constant.
struct GridDir {
  float r[9];
  float qz_coef;
  uint64_t uR;
};
cudaError_t launch_fft3(float2* data, const int P3[3], const float2* const tw[3], bool inverse, cudaStream_t s);
cudaError_t launch_swap_pack(const float* vc, const float* vs, float2* grid, const Fourier3Const& f, cudaStream_t s);
cudaError_t launch_swap_phase(const float2* Z, float2* out, const Fourier3Const& f, double R, double sigma, double eps,
                              double cs, cudaStream_t s);
cudaError_t launch_crop_real(const float2* grid, float* vol, const Fourier3Const& f, cudaStream_t s);
cudaError_t launch_grid_splat(const float2* G, const GridDir* dirs, int dir_begin, int n_dirs, const StageAConst& c,
                              const Fourier3Const& f, float2* acc, float2* raw, float* S, bool with_raw,
                              cudaStream_t s);
cudaError_t launch_grid_finish(float2* acc, const float2* raw, const float* S, double* stats, const Fourier3Const& f,
                               float nsr_m, cudaStream_t s);

// Whole-operator run with its workspace carved from `scratch` (tables first, then
// the largest direction block that fits); used by recon_run_noalloc.
int run_in_scratch(struct ::recon_plan_s* plan, const float* images, float* volume, char* scratch,
                   size_t scratch_bytes, cudaStream_t stream);
void set_last_error(const char* msg);

}  // namespace recon
