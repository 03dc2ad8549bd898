// C-ABI of the layered UTR reconstruction: plan building (host, FP64), workspace
// layout, and the run loop over direction blocks.  See include/recon.h.
//
// Compiled with -ffp-contract=off: the layer constants below must be the exact FP64
// results of the written operation order (they define the layer decision).
#include "recon.h"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "density.cuh"
#include "learned.cuh"
#include "recon_internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(RECON_E_CUDA, std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// frac(x / 2) as a 64-bit fixed-point fraction: the phase x*pi taken modulo 2*pi.
uint64_t half_turns_fixed(double x) {
  const double h = 0.5 * x;
  double f = h - std::floor(h);
  if (!(f < 1.0)) f = 0.0;  // h slightly negative may round to exactly 1
  const double scaled = std::ldexp(f, 64);
  if (scaled >= 18446744073709551616.0) return 0;
  return (uint64_t)scaled;
}

// Per-pass twiddles of the register FFTs for length P: the 8-value table of fft_reg.cuh
// (the pass at sub-length Ns, radix R, holds exp(-2 pi i kb r / (Ns R)) at (Ns - 8) +
// kb (R - 1) + (r - 1)), then for P >= 256 that of fft16.cuh at (P - 8) + (Ns - 16) + ...
std::vector<float2> fft_twiddles(int P) {
  std::vector<float2> t(P >= 16 ? (P - 8) + (P >= 256 ? P - 16 : 0) : 1, float2{0.f, 0.f});
  if (P >= 256) {
    for (int Ns = 1; Ns < P;) {
      const int rem = P / Ns;
      const int R = (rem % 16 == 0) ? 16 : rem;
      if (Ns > 1)
        for (int kb = 0; kb < Ns; ++kb)
          for (int r = 1; r < R; ++r) {
            const double ang = -2.0 * M_PI * (double)kb * r / ((double)Ns * R);
            t[(P - 8) + (Ns - 16) + kb * (R - 1) + (r - 1)] = float2{(float)std::cos(ang), (float)std::sin(ang)};
          }
      Ns *= R;
    }
  }
  if (P >= 16) {
    for (int Ns = 1; Ns < P;) {
      const int rem = P / Ns;
      const int R = (rem % 8 == 0) ? 8 : rem;
      if (Ns > 1)
        for (int kb = 0; kb < Ns; ++kb)
          for (int r = 1; r < R; ++r) {
            const double ang = -2.0 * M_PI * (double)kb * r / ((double)Ns * R);
            t[(Ns - 8) + kb * (R - 1) + (r - 1)] = float2{(float)std::cos(ang), (float)std::sin(ang)};
          }
      Ns *= R;
    }
  }
  return t;
}

}  // namespace

struct recon_plan_s {
  int D, nu, nv, nx, ny, nz, nzl, P, logP, half, db, n_blocks;
  double lambda, delta;
  recon_options opt;
  std::vector<recon::DirParams> dirs;
  std::vector<uint64_t> uA;
  std::vector<float> ramp;
  std::vector<float2> tw;
  std::vector<float2> twp;
  std::vector<float> theta, cnt, x2;  // learned regulariser: weights, bin counts, defocus feature
  recon::LearnConst lc;
  bool training = false;
  recon::StageAConst ca;
  recon::BackprojConst cb;
  recon::TmaBox tma{};   // footprint box of the TMA-staged backprojection
  bool use_tma = false;  // stage B runs k_backproject_tma
  // workspace layout (byte offsets)
  size_t off_dirs, off_uA, off_ramp, off_tw, off_twp, off_dens, off_dsum, off_theta, off_cnt, off_x2, off_S, off_T,
      off_stack, off_pow, off_eps, ws_bytes, table_bytes;
  size_t stack_dir_bytes;
  size_t off_flag;                 // device counter of the finiteness scan
  double pitch_max = 0.0, dof = 0.0;  // largest layer pitch and Delta^2 / (2 lambda), metres
  std::string warning;             // plan-time warning ("" if none)
  // the 3D-Fourier forms (Eq. 12, the Fourier-gridding UTR)
  bool uniform_R = false;          // every view has the same defocus (Eq. 12's condition)
  double R0 = 0.0;
  bool f3_ok = false;              // every grid side <= 1024 (padded 3D grid <= 2048 per axis)
  recon::Fourier3Const f3;
  std::vector<float2> tw3[3];      // FFT twiddles of each padded grid axis
  std::vector<recon::GridDir> gdirs;
  // optional profiling: one event after every launch (see recon::EventRecorder)
  bool profile = false;
  std::vector<cudaEvent_t> events;
  std::vector<int> event_kind;
  int profiled_events = 0;
  // recon_run_host: the copy stream and its events (created on first use, per device)
  int copy_dev = -1;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_start = nullptr, ev_ready[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  void release_copy_stream() {
    if (copy_stream) cudaStreamDestroy(copy_stream);
    for (cudaEvent_t e : {ev_start, ev_ready[0], ev_ready[1], ev_free[0], ev_free[1]})
      if (e) cudaEventDestroy(e);
    copy_stream = nullptr;
    ev_start = ev_ready[0] = ev_ready[1] = ev_free[0] = ev_free[1] = nullptr;
    copy_dev = -1;
  }
  ~recon_plan_s() {
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    release_copy_stream();
  }
};

extern "C" {

void recon_default_options(recon_options* o) {
  if (!o) return;
  o->sigma = 0.0;
  o->eps = 0.1;
  o->cs = 0.0;
  o->filter = RECON_FILTER_TIKHONOV;
  o->input_mode = RECON_INPUT_INTENSITY;
  o->stack_dtype = RECON_STACK_F32;
  o->ramp_mode = RECON_RAMP_SINGLE_AXIS;
  o->accumulate = 0;
  o->dir_block = 0;
  o->mlp_weights = nullptr;
  o->nsr = 0.0;
  o->stage_block = 0;
  o->bp_kernel = RECON_BP_AUTO;
  o->check_finite = 0;
  o->layer_interp = RECON_LAYER_NEAREST;
  o->mlp_views = 0.0;
  o->bp_tile_z = 0;
  o->bp_warp = 0;
}

const char* recon_error_string(int code) {
  switch (code) {
    case RECON_OK: return "ok";
    case RECON_E_INVALID_ARG: return "invalid argument";
    case RECON_E_UNSUPPORTED_SIZE: return "unsupported size";
    case RECON_E_CUDA: return "CUDA error";
    case RECON_E_WORKSPACE: return "workspace too small or misaligned";
    case RECON_E_NO_MEMORY: return "host allocation failed";
    case RECON_E_NONFINITE: return "an image holds NaN or Inf";
    case RECON_E_NO_WEIGHTS: return "the learned filter has no network parameters";
    case RECON_E_DEVICE_CHECK: return "a device-side check failed (a bounded wait ran out or a footprint left its box)";
    default: return "unknown status";
  }
}

const char* recon_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// Builds a plan; `training` (recon_mlp_train's internal plan) accepts any geometry and
// skips the ramp, density and learned-filter set-up.
static int plan_create(const recon_geometry* geom, double lambda, double delta, const double* defocus,
                       int nz_layers, const recon_grid* grid, const recon_options* opts, recon_plan_t* out,
                       bool training) {
  if (!geom || !grid || !out) return fail(RECON_E_INVALID_ARG, "recon_plan: null geometry, grid or out");
  const int D = geom->n_dir;
  if (D < 0) return fail(RECON_E_INVALID_ARG, "recon_plan: n_dir < 0");
  if (D > 0 && (!geom->rot || !defocus)) return fail(RECON_E_INVALID_ARG, "recon_plan: null rot or defocus");
  if (geom->nu < 1 || geom->nv < 1) return fail(RECON_E_INVALID_ARG, "recon_plan: image size < 1");
  if (geom->nu > RECON_MAX_IMAGE || geom->nv > RECON_MAX_IMAGE)
    return fail(RECON_E_UNSUPPORTED_SIZE, "recon_plan: image side > RECON_MAX_IMAGE");
  if (grid->nx < 0 || grid->ny < 0 || grid->nz < 0) return fail(RECON_E_INVALID_ARG, "recon_plan: grid < 0");
  if (grid->nx > RECON_MAX_GRID || grid->ny > RECON_MAX_GRID || grid->nz > RECON_MAX_GRID)
    return fail(RECON_E_UNSUPPORTED_SIZE, "recon_plan: grid side > RECON_MAX_GRID");
  if (nz_layers < 0) return fail(RECON_E_INVALID_ARG, "recon_plan: nz_layers < 0");
  if (nz_layers == 0) {  // automatic: layers no thicker than the depth of field
    if (!(lambda > 0.0) || !(delta > 0.0) || !std::isfinite(lambda) || !std::isfinite(delta))
      return fail(RECON_E_INVALID_ARG, "recon_plan: lambda and delta must be > 0");
    const int rc = recon_layers_for_dof(geom, grid, lambda, delta, &nz_layers);
    if (rc) return rc;
  }
  if (nz_layers > RECON_MAX_LAYERS) return fail(RECON_E_UNSUPPORTED_SIZE, "recon_plan: nz_layers > RECON_MAX_LAYERS");
  if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(RECON_E_INVALID_ARG, "recon_plan: lambda must be > 0");
  if (!(delta > 0.0) || !std::isfinite(delta)) return fail(RECON_E_INVALID_ARG, "recon_plan: delta must be > 0");
  recon_options o;
  recon_default_options(&o);
  if (opts) o = *opts;
  if (o.filter != RECON_FILTER_OFF && o.filter != RECON_FILTER_TIKHONOV && o.filter != RECON_FILTER_MLP &&
      o.filter != RECON_FILTER_PAIR)
    return fail(RECON_E_INVALID_ARG, "recon_plan: unknown filter");
  if (o.filter == RECON_FILTER_MLP && !training && !o.mlp_weights)
    return fail(RECON_E_NO_WEIGHTS, "recon_plan: the learned filter needs mlp_weights (RECON_MLP_PARAMS floats)");
  if (o.filter == RECON_FILTER_MLP && !training && (!(o.nsr > 0.0) || !std::isfinite(o.nsr)))
    return fail(RECON_E_INVALID_ARG, "recon_plan: the learned filter needs nsr > 0");
  if (o.check_finite != 0 && o.check_finite != 1) return fail(RECON_E_INVALID_ARG, "recon_plan: check_finite must be 0 or 1");
  if (o.bp_warp != 0 && o.bp_warp != 8 && o.bp_warp != 16 && o.bp_warp != 32)
    return fail(RECON_E_INVALID_ARG, "recon_plan: bp_warp must be 0, 8, 16 or 32");
  if (!(o.mlp_views >= 0.0) || !std::isfinite(o.mlp_views))
    return fail(RECON_E_INVALID_ARG, "recon_plan: mlp_views must be >= 0");
  if (o.bp_tile_z != 0 && o.bp_tile_z != 8 && o.bp_tile_z != 16)
    return fail(RECON_E_INVALID_ARG, "recon_plan: bp_tile_z must be 0, 8 or 16");
  if (o.layer_interp != RECON_LAYER_NEAREST && o.layer_interp != RECON_LAYER_LINEAR)
    return fail(RECON_E_INVALID_ARG, "recon_plan: unknown layer_interp");
  if (o.input_mode != RECON_INPUT_INTENSITY && o.input_mode != RECON_INPUT_CONTRAST)
    return fail(RECON_E_INVALID_ARG, "recon_plan: unknown input_mode");
  if (o.stack_dtype != RECON_STACK_F32 && o.stack_dtype != RECON_STACK_BF16)
    return fail(RECON_E_INVALID_ARG, "recon_plan: unknown stack_dtype");
  if (o.ramp_mode != RECON_RAMP_SINGLE_AXIS && o.ramp_mode != RECON_RAMP_DENSITY)
    return fail(RECON_E_INVALID_ARG, "recon_plan: unknown ramp_mode");
  if (training) {
    o.ramp_mode = RECON_RAMP_SINGLE_AXIS;
    o.filter = RECON_FILTER_MLP;
  }
  if ((o.filter == RECON_FILTER_TIKHONOV || o.filter == RECON_FILTER_PAIR) && !(o.eps > 0.0))
    return fail(RECON_E_INVALID_ARG, "recon_plan: eps must be > 0 with the Tikhonov and pair filters");
  if (!std::isfinite(o.sigma) || !std::isfinite(o.eps) || !std::isfinite(o.cs))
    return fail(RECON_E_INVALID_ARG, "recon_plan: non-finite sigma, eps or cs");
  if (o.dir_block < 0) return fail(RECON_E_INVALID_ARG, "recon_plan: dir_block < 0");
  if (o.stage_block < 0) return fail(RECON_E_INVALID_ARG, "recon_plan: stage_block < 0");
  if (o.bp_kernel < RECON_BP_AUTO || o.bp_kernel > RECON_BP_TMA)
    return fail(RECON_E_INVALID_ARG, "recon_plan: unknown bp_kernel");

  recon_plan_s* p = new (std::nothrow) recon_plan_s();
  if (!p) return fail(RECON_E_NO_MEMORY, "recon_plan: out of host memory");
  p->D = D;
  p->nu = geom->nu;
  p->nv = geom->nv;
  p->nx = grid->nx;
  p->ny = grid->ny;
  p->nz = grid->nz;
  p->nzl = nz_layers;
  p->lambda = lambda;
  p->delta = delta;
  p->opt = o;
  p->training = training;
  int P = 1, logP = 0;
  while (P < 2 * (p->nu > p->nv ? p->nu : p->nv)) {
    P *= 2;
    ++logP;
  }
  p->P = P;
  p->logP = logP;
  p->half = P / 2 + 1;

  try {
    p->dirs.resize(D);
    // per-layer phase constants; the pair filter keeps the image-plane constant after them
    const int uA_row = nz_layers + (o.filter == RECON_FILTER_PAIR ? 1 : 0);
    p->uA.resize((size_t)D * uA_row);
    const double cx = 0.5 * (p->nx - 1), cy = 0.5 * (p->ny - 1), cz = 0.5 * (p->nz - 1);
    const double PD = (double)P * delta;
    for (int n = 0; n < D; ++n) {
      const double* R = geom->rot + 9 * (size_t)n;
      for (int q = 0; q < 9; ++q)
        if (!std::isfinite(R[q])) {
          delete p;
          return fail(RECON_E_INVALID_ARG, "recon_plan: non-finite rotation");
        }
      for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) {
          const double dot = R[3 * r] * R[3 * s] + R[3 * r + 1] * R[3 * s + 1] + R[3 * r + 2] * R[3 * s + 2];
          if (std::fabs(dot - (r == s ? 1.0 : 0.0)) > 1e-6) {
            delete p;
            return fail(RECON_E_INVALID_ARG, "recon_plan: rot[" + std::to_string(n) + "] is not orthonormal");
          }
        }
      if (o.ramp_mode == RECON_RAMP_SINGLE_AXIS && !training &&
          (std::fabs(R[3] - geom->rot[3]) > 1e-9 || std::fabs(R[4] - geom->rot[4]) > 1e-9 ||
           std::fabs(R[5] - geom->rot[5]) > 1e-9)) {
        delete p;
        return fail(RECON_E_INVALID_ARG,
                    "recon_plan: single-axis ramp needs one rotation axis: rot[n] row 1 must equal rot[0] row 1 (n = " +
                        std::to_string(n) + ")");
      }
      if (!std::isfinite(defocus[n])) {
        delete p;
        return fail(RECON_E_INVALID_ARG, "recon_plan: non-finite defocus");
      }
      recon::DirParams& d = p->dirs[n];
      std::memset(&d, 0, sizeof(d));
      const double pix = std::ldexp(1.0, recon::kPixFracBits);
      const double a3 = 0.5 * (p->nu - 1) - ((R[0] * cx + R[1] * cy) + R[2] * cz);
      const double b3 = 0.5 * (p->nv - 1) - ((R[3] * cx + R[4] * cy) + R[5] * cz);
      for (int q = 0; q < 3; ++q) {
        d.a[q] = std::llrint(R[q] * pix);
        d.b[q] = std::llrint(R[3 + q] * pix);
        d.af[q] = (float)R[q];
        d.bf[q] = (float)R[3 + q];
      }
      d.a[3] = std::llrint(a3 * pix);
      d.b[3] = std::llrint(b3 * pix);
      // Depth layers: Nz equal slabs over the bounding-box extent along the beam.
      // Exact operation order (defines the fixed-point layer decision):
      const double ext = (std::fabs(R[6]) * (double)p->nx + std::fabs(R[7]) * (double)p->ny) +
                         std::fabs(R[8]) * (double)p->nz;
      const double scale = (double)nz_layers / ext;
      const double ti = R[6] * scale, tj = R[7] * scale, tk = R[8] * scale;
      const double t0 = 0.5 * (double)nz_layers -
                        ((ti * (0.5 * (p->nx - 1)) + tj * (0.5 * (p->ny - 1))) + tk * (0.5 * (p->nz - 1)));
      const double one = 16777216.0;  // 2^24
      d.t[0] = (int32_t)std::rint(t0 * one);
      d.t[1] = (int32_t)std::rint(ti * one);
      d.t[2] = (int32_t)std::rint(tj * one);
      d.t[3] = (int32_t)std::rint(tk * one);
      {  // extremes over a general-kernel tile, relative to its origin (outward rounding)
        double lo[2] = {0.0, 0.0}, hi[2] = {0.0, 0.0};
        long long tlo = 0, thi = 0;
        for (int q = 0; q < 3; ++q) {
          const int e = recon::kGenTile[q] - 1;
          for (int w = 0; w < 2; ++w) {
            const double v = R[3 * w + q] * e;
            (v < 0 ? lo[w] : hi[w]) += v;
          }
          const long long tv = (long long)d.t[q + 1] * e;
          (tv < 0 ? tlo : thi) += tv;
        }
        const double u16 = 65536.0;
        const double ext16[4] = {std::floor(lo[0] * u16) - 1, std::ceil(hi[0] * u16) + 1,
                                 std::floor(lo[1] * u16) - 1, std::ceil(hi[1] * u16) + 1};
        bool fits = tlo >= INT32_MIN / 2 && thi <= INT32_MAX / 2;
        for (int q = 0; q < 4; ++q) fits = fits && std::fabs(ext16[q]) < 1e9;
        for (int q = 0; q < 4; ++q) d.ab_ext[q] = fits ? (int32_t)ext16[q] : 0;
        d.t_ext[0] = fits ? (int32_t)tlo : 0;
        d.t_ext[1] = fits ? (int32_t)thi : 0;
        if (!fits) d.ab_ext[0] = d.t_ext[0] = INT32_MIN;
      }
      // Per-layer CTF phase constant: chi = pi * [lambda (R_n - z_k) / (P delta)^2] * m^2 + ...
      const double extm = ext * delta;
      if (extm / nz_layers > p->pitch_max) p->pitch_max = extm / nz_layers;
      for (int k = 0; k < nz_layers; ++k) {
        const double zk = -0.5 * extm + (k + 0.5) * (extm / nz_layers);
        if (o.filter == RECON_FILTER_PAIR) {
          // depth phase pi lambda z_k q^2 of the layer; chi's defocus term at the image plane
          p->uA[(size_t)n * uA_row + k] = half_turns_fixed(lambda * zk / (PD * PD));
        } else {
          const double Ak = lambda * (defocus[n] - zk) / (PD * PD);
          p->uA[(size_t)n * uA_row + k] = half_turns_fixed(Ak);
        }
      }
      if (o.filter == RECON_FILTER_PAIR)
        p->uA[(size_t)n * uA_row + nz_layers] = half_turns_fixed(lambda * defocus[n] / (PD * PD));
    }
    // Depth of field (Sec. 1): a layer thicker than Delta^2 / (2 lambda) holds voxels out of
    // its own focus; reported as a warning, not an error.
    p->dof = delta * delta / (2.0 * lambda);
    if (p->pitch_max > p->dof) {
      char msg[256];
      std::snprintf(msg, sizeof msg,
                    "layer pitch %.4g m exceeds the depth of field Delta^2/(2 lambda) = %.4g m: "
                    "recon_layers_for_dof gives the Nz that resolves it",
                    p->pitch_max, p->dof);
      p->warning = msg;
    }
    // Ramp: (pi/D) delta DFT_P[Ram-Lak](m), m = 0..P/2, with the 1/P^2 of the inverse DFT.
    p->ramp.assign(p->half, 0.0f);
    if (D > 0) {
      for (int m = 0; m < p->half; ++m) {
        double s = 1.0 / (4.0 * delta * delta);
        for (int nn = 1; nn < P / 2; nn += 2) {
          const long long ph = ((long long)m * nn) % P;
          s += 2.0 * (-1.0 / ((double)nn * nn * M_PI * M_PI * delta * delta)) * std::cos(2.0 * M_PI * ph / P);
        }
        if ((P / 2) % 2 == 1) {  // the unpaired tap n = -P/2 (odd only when P = 2)
          const double hn = (double)(P / 2);
          s += (-1.0 / (hn * hn * M_PI * M_PI * delta * delta)) * ((m % 2) ? -1.0 : 1.0);
        }
        p->ramp[m] = (float)((M_PI / D) * delta * s / ((double)P * P));
      }
    }
    p->tw.resize(P);
    for (int j = 0; j < P; ++j) {
      p->tw[j].x = (float)std::cos(2.0 * M_PI * j / P);
      p->tw[j].y = (float)-std::sin(2.0 * M_PI * j / P);
    }
    p->twp = fft_twiddles(P);
  } catch (const std::bad_alloc&) {
    delete p;
    return fail(RECON_E_NO_MEMORY, "recon_plan: out of host memory");
  }

  recon::StageAConst& ca = p->ca;
  ca.P = P;
  ca.logP = logP;
  ca.nu = p->nu;
  ca.nv = p->nv;
  ca.nz_layers = nz_layers;
  ca.filter = o.filter;
  ca.input_mode = o.input_mode;
  ca.stack_bf16 = o.stack_dtype == RECON_STACK_BF16;
  const double PD = (double)P * delta;
  ca.uC = half_turns_fixed(o.cs * lambda * lambda * lambda / (2.0 * PD * PD * PD * PD));
  ca.uW = half_turns_fixed(std::atan(o.sigma) / M_PI);
  ca.eps = (float)o.eps;
  ca.pref = (float)(lambda / (4.0 * M_PI * std::sqrt(1.0 + o.sigma * o.sigma)));
  ca.half = p->half;
  // row stride: the nu + 1 tap pairs rounded up to 4 entries, so every row starts on a
  // 16-byte boundary (the TMA-staged backprojection's tensor map needs 16-byte strides)
  ca.su = (p->nu + 1 + 3) & ~3;
  ca.layer_elems = (size_t)(p->nv + 2) * ca.su;
  {  // sampling-density grid (density weighting only), see density.cuh
    recon::DensityConst& dc = ca.dens;
    std::memset(&dc, 0, sizeof(dc));
    dc.enabled = o.ramp_mode == RECON_RAMP_DENSITY;
    dc.s = P / 128 > 1 ? P / 128 : 1;
    dc.Gh = (int)std::ceil(std::sqrt(2.0) * (P / 2.0) / dc.s) + 2;
    dc.G = 2 * dc.Gh + 1;
    dc.n_samples1 = P / dc.s;
    dc.inv_s = 1.0f / (float)dc.s;
    dc.g_over_p2 = (float)((double)dc.s * dc.s * dc.s / ((double)P * delta) / ((double)P * P));
    long long band = 0;
    const long long r2 = (long long)(dc.Gh - 2) * (dc.Gh - 2);
    for (int z = -dc.Gh; z <= dc.Gh; ++z)
      for (int y = -dc.Gh; y <= dc.Gh; ++y) {
        const long long rem = r2 - (long long)z * z - (long long)y * y;
        if (rem < 0) continue;
        const int xm = (int)std::floor(std::sqrt((double)rem));
        band += 2 * (long long)xm + 1;
      }
    dc.eps_scale = (float)(1e-3 / (double)band);
  }
  {  // learned regulariser tables
    recon::LearnConst& lc = p->lc;
    lc.bin_width = P / 128 > 1 ? P / 128 : 1;
    long long half_sq = (long long)P * P / 2, r = (long long)std::sqrt((double)half_sq);
    while (r * r > half_sq) --r;
    while ((r + 1) * (r + 1) <= half_sq) ++r;
    lc.n_bins = (int)(r / lc.bin_width) + 1;
    lc.inv_half_p = 2.0f / (float)P;
    lc.noise_floor = (float)(o.nsr * o.nsr * (double)p->nu * (double)p->nv);
    lc.eps_scale = (training || !(o.mlp_views > 1.0)) ? 1.0f : (float)(1.0 / o.mlp_views);
    if (o.filter == RECON_FILTER_MLP) {
      try {
        p->theta.assign(recon::kMlpParams, 0.f);
        if (o.mlp_weights) std::memcpy(p->theta.data(), o.mlp_weights, sizeof(float) * recon::kMlpParams);
        p->cnt.assign(lc.n_bins, 0.f);
        for (int a = -P / 2; a < P / 2; ++a)
          for (int b = -P / 2; b < P / 2; ++b) {
            const long long msq = (long long)a * a + (long long)b * b;
            long long q = (long long)std::sqrt((double)msq);
            while (q * q > msq) --q;
            while ((q + 1) * (q + 1) <= msq) ++q;
            const int bin = (int)(q / lc.bin_width);
            p->cnt[bin < lc.n_bins - 1 ? bin : lc.n_bins - 1] += 1.f;
          }
        p->x2.assign((size_t)(D > 0 ? D : 1) * nz_layers, 0.f);
        for (int n = 0; n < D; ++n) {
          const double* R = geom->rot + 9 * (size_t)n;
          const double ext = ((std::fabs(R[6]) * p->nx + std::fabs(R[7]) * p->ny) + std::fabs(R[8]) * p->nz) * delta;
          for (int k = 0; k < nz_layers; ++k) {
            const double zk = -0.5 * ext + (k + 0.5) * (ext / nz_layers);
            p->x2[(size_t)n * nz_layers + k] = (float)(lambda * (defocus[n] - zk) / (delta * delta) / 100.0);
          }
        }
      } catch (const std::bad_alloc&) {
        delete p;
        return fail(RECON_E_NO_MEMORY, "recon_plan: out of host memory");
      }
    }
  }

  recon::BackprojConst& cb = p->cb;
  cb.nx = p->nx;
  cb.ny = p->ny;
  cb.nz = p->nz;
  cb.nu = p->nu;
  cb.nv = p->nv;
  cb.nz_layers = nz_layers;
  cb.su = ca.su;
  cb.layer_elems = ca.layer_elems;
  cb.stack_bf16 = ca.stack_bf16;
  cb.axis_y = D > 0;
  for (int n = 0; n < D; ++n) {
    const double* R = geom->rot + 9 * (size_t)n;
    if (!(R[3] == 0.0 && R[4] == 1.0 && R[5] == 0.0 && R[1] == 0.0 && R[7] == 0.0)) cb.axis_y = 0;
  }
  {
    const double boff = 0.5 * (p->nv - 1) - 0.5 * (p->ny - 1);  // v = j + boff when row 1 = (0,1,0)
    const double fl = std::floor(boff);
    cb.b_int = (int)fl;
    cb.b_frac = (float)(boff - fl);
  }
  cb.staged = o.bp_kernel == RECON_BP_STAGED;
  cb.layer_linear = o.layer_interp == RECON_LAYER_LINEAR;
  cb.warp_cols = o.bp_warp ? o.bp_warp : 8;
  // The TMA-staged kernel where the general kernel would run (any geometry but a single
  // axis along y, or the layer blend), measured faster on sm_103a; on request for any geometry.
  const bool general = !cb.axis_y || cb.layer_linear;
  if (o.bp_kernel == RECON_BP_TMA || (o.bp_kernel == RECON_BP_AUTO && general && D > 0)) {
    p->tma = recon::tma_box_for(cb, p->dirs.data(), D, o.bp_tile_z ? o.bp_tile_z : 16);
    if (!p->tma.ok && o.bp_kernel == RECON_BP_TMA) {
      delete p;
      return fail(RECON_E_UNSUPPORTED_SIZE,
                  "recon_plan: a footprint box of the TMA-staged backprojection is too large (more than 256 pairs, "
                  "rows or layers, or 200 KB of shared memory)");
    }
    p->use_tma = p->tma.ok != 0;
  }

  {  // the 3D-Fourier forms: padded grid, per-axis twiddles, per-view gridding constants
    p->uniform_R = true;
    for (int n = 1; n < D; ++n)
      if (defocus[n] != defocus[0]) p->uniform_R = false;
    p->R0 = D > 0 ? defocus[0] : 0.0;
    const int nn[3] = {p->nx, p->ny, p->nz};
    p->f3_ok = true;
    for (int a = 0; a < 3; ++a) {
      int q = 1;
      while (q < 2 * nn[a]) q *= 2;
      if (nn[a] < 1 || q > 2048) p->f3_ok = false;
      p->f3.P3[a] = q;
      p->f3.n[a] = nn[a];
      p->f3.off[a] = (q - nn[a]) / 2;
      p->f3.scale[a] = (float)((double)q / P);
    }
    p->f3.lam = lambda;
    p->f3.delta = delta;
    if (p->f3_ok) {
      try {
        for (int a = 0; a < 3; ++a) p->tw3[a] = fft_twiddles(p->f3.P3[a]);
        p->gdirs.resize(D > 0 ? D : 1);
        for (int n = 0; n < D; ++n) {
          const double* Rr = geom->rot + 9 * (size_t)n;
          recon::GridDir& g = p->gdirs[n];
          for (int q = 0; q < 9; ++q) g.r[q] = (float)Rr[q];
          g.qz_coef = (float)(lambda / (2.0 * P * delta));
          g.uR = half_turns_fixed(lambda * defocus[n] / ((double)P * delta * (double)P * delta));
        }
      } catch (const std::bad_alloc&) {
        delete p;
        return fail(RECON_E_NO_MEMORY, "recon_plan: out of host memory");
      }
    }
  }
  const size_t elem = ca.stack_bf16 ? 4 : 8;  // one tap pair
  p->stack_dir_bytes = (size_t)nz_layers * ca.layer_elems * elem;
  // S and T of one direction (the stage-A intermediates)
  const size_t inter_dir = (size_t)p->nv * p->half * 8 * (1 + (size_t)nz_layers);
  const size_t per_dir = inter_dir + p->stack_dir_bytes;
  // Where one direction's intermediates are large (big images, many layers), stage A runs
  // in sub-blocks whose intermediates fit 2 GiB by default (two directions of 1024^2 images
  // with Nz = 64: the column stage then fills the GPU with fewer layer groups, each of which
  // repeats a column's forward FFT), and the rest of the budget holds stacks: a larger
  // direction block means fewer volume read-modify-writes and tile set-ups in the
  // backprojection.
  const bool big_dir = inter_dir > ((size_t)64 << 20);
  int auto_sub = 0;
  if (big_dir && o.stage_block == 0) auto_sub = (int)std::max<size_t>(1, ((size_t)2 << 30) / inter_dir);
  int db = o.dir_block;
  if (db == 0) {
    // as many directions per block as the stage budget holds (fewer volume
    // read-modify-writes), then balanced so that the blocks are of equal size: 4 GiB, or
    // 16 GiB where one direction's intermediates are large (measured on 1024^2 images: 25,
    // 50 and 100 directions per block took 1359, 1331 and 1320 ms per 1500-view step)
    const size_t budget = (size_t)(big_dir ? 16 : 4) << 30;
    if (auto_sub > 0) {
      const size_t used = (size_t)auto_sub * inter_dir;
      db = used < budget ? (int)std::min<size_t>((budget - used) / p->stack_dir_bytes, 1024) : 1;
    } else
      db = (int)(budget / per_dir);
    if (db < 1) db = 1;
    if (db > 1024) db = 1024;
    if (D > 0) {
      const int nb = (D + db - 1) / db;
      db = (D + nb - 1) / nb;
    }
  }
  if (db > 1024) db = 1024;
  if (D > 0 && db > D) db = D;
  if (db < 1) db = 1;
  p->db = db;
  p->n_blocks = D > 0 ? (D + db - 1) / db : 0;
  {  // stage-A sub-blocks: an option where one direction's intermediates are small (measured
     // slower than whole blocks at 256^2 / Nz = 32, where launch gaps outweigh the L2
     // residency of the intermediates), the default where they are large (above)
    int sub = o.stage_block > 0 ? o.stage_block : (auto_sub > 0 ? auto_sub : db);
    if (sub < 1) sub = 1;
    if (sub > db) sub = db;
    ca.sub_block = P >= 16 ? sub : db;  // the radix-2 path (tiny images) runs whole blocks
  }

  size_t off = 0;
  p->off_dirs = off;
  off = align256(off + sizeof(recon::DirParams) * (size_t)(D > 0 ? D : 1));
  p->off_uA = off;
  off = align256(off + sizeof(uint64_t) * (p->uA.size() > 0 ? p->uA.size() : (size_t)nz_layers + 1));
  p->off_ramp = off;
  off = align256(off + sizeof(float) * p->half);
  p->off_tw = off;
  off = align256(off + sizeof(float2) * P);
  p->off_twp = off;
  off = align256(off + sizeof(float2) * p->twp.size());
  p->off_dens = off;
  if (ca.dens.enabled) off = align256(off + sizeof(float) * (size_t)ca.dens.G * ca.dens.G * ca.dens.G);
  p->off_dsum = off;
  off = align256(off + sizeof(double));
  p->off_theta = off;
  off = align256(off + sizeof(float) * p->theta.size());
  p->off_cnt = off;
  off = align256(off + sizeof(float) * p->cnt.size());
  p->off_x2 = off;
  off = align256(off + sizeof(float) * p->x2.size());
  p->off_flag = off;
  off = align256(off + sizeof(unsigned int));
  p->table_bytes = off;
  p->off_S = off;
  off = align256(off + (size_t)ca.sub_block * p->nv * p->half * 8);
  p->off_T = off;
  off = align256(off + (size_t)ca.sub_block * nz_layers * p->nv * p->half * 8);
  p->off_stack = off;
  off = align256(off + (size_t)db * p->stack_dir_bytes);
  p->off_pow = off;
  p->off_eps = off;
  if (o.filter == RECON_FILTER_MLP && !training) {
    off = align256(off + sizeof(float) * (size_t)ca.sub_block * p->lc.n_bins);
    p->off_eps = off;
    off = align256(off + sizeof(float) * (size_t)ca.sub_block * nz_layers * p->lc.n_bins);
  }
  p->ws_bytes = off;
  if (o.filter == RECON_FILTER_MLP && !training && P < 16) {
    delete p;
    return fail(RECON_E_UNSUPPORTED_SIZE, "recon_plan: the learned filter needs images of more than 4 pixels");
  }
  *out = p;
  return RECON_OK;
}

extern "C" int recon_plan(const recon_geometry* geom, double lambda, double delta, const double* defocus,
                          int nz_layers, const recon_grid* grid, const recon_options* opts, recon_plan_t* out) {
  return plan_create(geom, lambda, delta, defocus, nz_layers, grid, opts, out, false);
}

extern "C" {

int recon_workspace_size(recon_plan_t p, size_t* bytes) {
  if (!p || !bytes) return fail(RECON_E_INVALID_ARG, "recon_workspace_size: null argument");
  *bytes = p->ws_bytes;
  return RECON_OK;
}

int recon_plan_info(recon_plan_t p, int* padded, int* dir_block, int* n_blocks, int* stage_block) {
  if (!p) return fail(RECON_E_INVALID_ARG, "recon_plan_info: null plan");
  if (padded) *padded = p->P;
  if (dir_block) *dir_block = p->db;
  if (n_blocks) *n_blocks = p->n_blocks;
  if (stage_block) *stage_block = p->ca.sub_block;
  return RECON_OK;
}

int recon_destroy(recon_plan_t p) {
  delete p;
  return RECON_OK;
}

int recon_plan_bp_kernel(recon_plan_t p, int* kernel) {
  if (!p || !kernel) return fail(RECON_E_INVALID_ARG, "recon_plan_bp_kernel: null argument");
  *kernel = p->use_tma ? RECON_BP_TMA : ((p->cb.axis_y && !p->cb.layer_linear && p->cb.staged) ? RECON_BP_STAGED
                                                                                                 : RECON_BP_DIRECT);
  return RECON_OK;
}

int recon_plan_dof(recon_plan_t p, double* pitch_max, double* dof) {
  if (!p) return fail(RECON_E_INVALID_ARG, "recon_plan_dof: null plan");
  if (pitch_max) *pitch_max = p->pitch_max;
  if (dof) *dof = p->dof;
  return RECON_OK;
}

const char* recon_plan_warning(recon_plan_t p) { return p ? p->warning.c_str() : ""; }

int recon_plan_layers(recon_plan_t p, int* nz_layers) {
  if (!p || !nz_layers) return fail(RECON_E_INVALID_ARG, "recon_plan_layers: null argument");
  *nz_layers = p->nzl;
  return RECON_OK;
}

int recon_layers_for_dof(const recon_geometry* geom, const recon_grid* grid, double lambda, double delta, int* nz) {
  if (!geom || !grid || !nz) return fail(RECON_E_INVALID_ARG, "recon_layers_for_dof: null argument");
  if (geom->n_dir < 0 || (geom->n_dir > 0 && !geom->rot))
    return fail(RECON_E_INVALID_ARG, "recon_layers_for_dof: bad geometry");
  if (!(lambda > 0.0) || !(delta > 0.0) || !std::isfinite(lambda) || !std::isfinite(delta))
    return fail(RECON_E_INVALID_ARG, "recon_layers_for_dof: lambda and delta must be > 0");
  if (grid->nx < 0 || grid->ny < 0 || grid->nz < 0) return fail(RECON_E_INVALID_ARG, "recon_layers_for_dof: grid < 0");
  // Nz >= T_n / DOF for every direction: T_n in voxels times delta over Delta^2 / (2 lambda)
  const double dof = delta * delta / (2.0 * lambda);
  double need = 1.0;
  for (int n = 0; n < geom->n_dir; ++n) {
    const double* R = geom->rot + 9 * (size_t)n;
    const double ext = ((std::fabs(R[6]) * grid->nx + std::fabs(R[7]) * grid->ny) + std::fabs(R[8]) * grid->nz) * delta;
    if (!std::isfinite(ext)) return fail(RECON_E_INVALID_ARG, "recon_layers_for_dof: non-finite rotation");
    need = std::max(need, std::ceil(ext / dof * (1.0 - 1e-12)));
  }
  *nz = need > RECON_MAX_LAYERS ? RECON_MAX_LAYERS : (int)need;
  return RECON_OK;
}

}  // extern "C"

namespace {

int check_ws(recon_plan_t p, void* ws, size_t ws_bytes, const char* who) {
  if (!ws) return fail(RECON_E_WORKSPACE, std::string(who) + ": null workspace");
  if (((uintptr_t)ws & 255) != 0) return fail(RECON_E_WORKSPACE, std::string(who) + ": workspace not 256-byte aligned");
  if (ws_bytes < p->ws_bytes)
    return fail(RECON_E_WORKSPACE, std::string(who) + ": workspace has " + std::to_string(ws_bytes) + " bytes, needs " +
                                       std::to_string(p->ws_bytes));
  return RECON_OK;
}

recon::Workspace carve(recon_plan_t p, void* ws) {
  char* b = (char*)ws;
  recon::Workspace w;
  w.dirs = (recon::DirParams*)(b + p->off_dirs);
  w.uA = (uint64_t*)(b + p->off_uA);
  w.ramp = (float*)(b + p->off_ramp);
  w.tw = (float2*)(b + p->off_tw);
  w.twp = (float2*)(b + p->off_twp);
  w.dens = (float*)(b + p->off_dens);
  w.band_sum = (double*)(b + p->off_dsum);
  w.eps = (float*)(b + p->off_eps);
  w.n_bins = p->lc.n_bins;
  w.bin_width = p->lc.bin_width;
  w.S = (float2*)(b + p->off_S);
  w.T = (float2*)(b + p->off_T);
  w.stack = (void*)(b + p->off_stack);
  return w;
}

int upload_tables(recon_plan_t p, const recon::Workspace& w, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (p->D > 0) {
    e = cudaMemcpyAsync(w.dirs, p->dirs.data(), sizeof(recon::DirParams) * p->D, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(w.uA, p->uA.data(), sizeof(uint64_t) * p->uA.size(), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w.ramp, p->ramp.data(), sizeof(float) * p->ramp.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w.tw, p->tw.data(), sizeof(float2) * p->tw.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w.twp, p->twp.data(), sizeof(float2) * p->twp.size(), cudaMemcpyHostToDevice, s);
  char* base = (char*)w.dirs - p->off_dirs;
  if (e == cudaSuccess && !p->theta.empty())
    e = cudaMemcpyAsync(base + p->off_theta, p->theta.data(), sizeof(float) * p->theta.size(), cudaMemcpyHostToDevice,
                        s);
  if (e == cudaSuccess && !p->cnt.empty())
    e = cudaMemcpyAsync(base + p->off_cnt, p->cnt.data(), sizeof(float) * p->cnt.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !p->x2.empty())
    e = cudaMemcpyAsync(base + p->off_x2, p->x2.data(), sizeof(float) * p->x2.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "upload of plan tables");
  if (p->ca.dens.enabled) {
    e = recon::launch_density_setup(p->ca.dens, w.dirs, p->D, p->P, w.dens, w.band_sum, s);
    if (e != cudaSuccess) return cuda_fail(e, "sampling-density setup");
  }
  return RECON_OK;
}

// Optional finiteness scan of the images: counts NaN / Inf on the GPU, waits for the
// count and refuses the run if it is not zero.
int scan_finite(recon_plan_t p, const float* images, unsigned int* d_count, cudaStream_t s, const char* who) {
  const size_t n = (size_t)p->D * p->nu * p->nv;
  cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = recon::launch_count_nonfinite(images, n, d_count, s);
  unsigned int h_count = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_count, d_count, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, (std::string(who) + ": finiteness scan").c_str());
  if (h_count != 0)
    return fail(RECON_E_NONFINITE, std::string(who) + ": " + std::to_string(h_count) +
                                       " image values are NaN or Inf; nothing was reconstructed");
  return RECON_OK;
}

// The TMA-staged backprojection's status word: the second word of the flag slot.
unsigned int* tma_status(recon_plan_t p, void* ws) { return (unsigned int*)((char*)ws + p->off_flag) + 1; }

// Stage B of one direction block through the plan's backprojection kernel.
cudaError_t backproject_block(recon_plan_t p, const recon::DirParams* dirs, const void* stack, int d0, int cnt,
                              float* vol, int accumulate, void* ws, cudaStream_t s) {
  if (p->use_tma)
    return recon::launch_backproject_tma(p->cb, p->tma, dirs, stack, d0, cnt, vol, accumulate, tma_status(p, ws), s);
  return recon::launch_backproject(p->cb, dirs, stack, d0, cnt, vol, accumulate, s);
}

// Before a call's first TMA-staged launch: clear the status word.
int tma_begin(recon_plan_t p, void* ws, cudaStream_t s, const char* who) {
  if (!p->use_tma) return RECON_OK;
  const cudaError_t e = cudaMemsetAsync(tma_status(p, ws), 0, sizeof(unsigned int), s);
  return e == cudaSuccess ? RECON_OK : cuda_fail(e, (std::string(who) + ": clearing the status word").c_str());
}

// After its last: read the status word back (a 4-byte copy and a stream synchronisation).
int tma_end(recon_plan_t p, void* ws, cudaStream_t s, const char* who) {
  if (!p->use_tma) return RECON_OK;
  unsigned int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, tma_status(p, ws), sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, (std::string(who) + ": reading the backprojection status").c_str());
  if (h & 1u)
    return fail(RECON_E_DEVICE_CHECK,
                std::string(who) + ": a bounded wait of the TMA-staged backprojection ran out; the volume is incomplete");
  if (h & 2u)
    return fail(RECON_E_DEVICE_CHECK, std::string(who) + ": a footprint left its TMA staging box; the volume is wrong");
  return RECON_OK;
}

// Learned regulariser, between the row FFTs and the column kernel of each block: radial
// power spectrum of every image (column FFTs), then the eps table of the block.
struct MlpHookCtx {
  recon_plan_t p;
  const char* base;  // workspace start (tables)
  float* pow;        // [DB][n_bins]
  float* eps;        // [DB][Nz][n_bins]
  const float2* S;
  const float2* twp;
};

cudaError_t mlp_hook(void* vctx, int dir_begin, int dir_count, cudaStream_t s) {
  MlpHookCtx* x = (MlpHookCtx*)vctx;
  recon_plan_t p = x->p;
  cudaError_t e = cudaMemsetAsync(x->pow, 0, sizeof(float) * (size_t)dir_count * p->lc.n_bins, s);
  if (e != cudaSuccess) return e;
  e = recon::launch_cols_forward(p->ca, p->lc, x->S, nullptr, x->pow, x->twp, dir_count, s);
  if (e != cudaSuccess) return e;
  return recon::launch_eps_table(p->lc, x->pow, (const float*)(x->base + p->off_cnt),
                                 (const float*)(x->base + p->off_x2), (const float*)(x->base + p->off_theta),
                                 x->eps, nullptr, dir_count, p->nzl, dir_begin, s);
}

}  // namespace

extern "C" {

int recon_run(recon_plan_t p, const float* images, float* volume, void* workspace, size_t ws_bytes, void* stream) {
  if (!p) return fail(RECON_E_INVALID_ARG, "recon_run: null plan");
  const size_t nvox = (size_t)p->nx * p->ny * p->nz;
  if (nvox > 0 && !volume) return fail(RECON_E_INVALID_ARG, "recon_run: null volume");
  if (p->D > 0 && !images) return fail(RECON_E_INVALID_ARG, "recon_run: null images");
  cudaStream_t s = (cudaStream_t)stream;
  if (p->D == 0 || nvox == 0) {
    if (nvox > 0 && !p->opt.accumulate) {
      cudaError_t e = cudaMemsetAsync(volume, 0, nvox * sizeof(float), s);
      if (e != cudaSuccess) return cuda_fail(e, "recon_run: clearing the volume");
    }
    return RECON_OK;
  }
  int rc = check_ws(p, workspace, ws_bytes, "recon_run");
  if (rc) return rc;
  if (p->opt.check_finite) {
    rc = scan_finite(p, images, (unsigned int*)((char*)workspace + p->off_flag), s, "recon_run");
    if (rc) return rc;
  }
  const recon::Workspace w = carve(p, workspace);
  rc = upload_tables(p, w, s);
  if (rc) return rc;
  recon::EventRecorder recorder{p->events.data(), p->event_kind.data(), 0, (int)p->events.size()};
  recon::EventRecorder* rec = p->profile ? &recorder : nullptr;
  MlpHookCtx hctx{p, (const char*)workspace, (float*)((char*)workspace + p->off_pow), w.eps, w.S, w.twp};
  const recon::StageAHook hook{mlp_hook, &hctx};
  const recon::StageAHook* hk = p->ca.filter == RECON_FILTER_MLP ? &hook : nullptr;
  rc = tma_begin(p, workspace, s, "recon_run");
  if (rc) return rc;
  if (rec) rec->mark(-1, s);
  for (int b = 0; b < p->n_blocks; ++b) {
    const int d0 = b * p->db;
    const int cnt = (p->D - d0) < p->db ? (p->D - d0) : p->db;
    cudaError_t e = recon::launch_stage_a(p->ca, w, images, d0, cnt, s, rec, hk);
    if (e != cudaSuccess) return cuda_fail(e, "recon_run: stage A launch");
    e = backproject_block(p, w.dirs, w.stack, d0, cnt, volume, p->opt.accumulate || b > 0, workspace, s);
    if (e != cudaSuccess) return cuda_fail(e, "recon_run: backprojection launch");
    if (rec) rec->mark(3, s);
  }
  if (rec) p->profiled_events = recorder.n;
  return tma_end(p, workspace, s, "recon_run");
}

// One device image slot of recon_run_host: a direction block's images.
static size_t host_slot_bytes(recon_plan_t p) {
  return align256(sizeof(float) * (size_t)p->db * p->nv * p->nu);
}

int recon_run_host_workspace_size(recon_plan_t p, size_t* bytes) {
  if (!p || !bytes) return fail(RECON_E_INVALID_ARG, "recon_run_host_workspace_size: null argument");
  *bytes = p->ws_bytes + 2 * host_slot_bytes(p);
  return RECON_OK;
}

int recon_run_host(recon_plan_t p, const float* host_images, float* volume, void* workspace, size_t ws_bytes,
                   void* stream) {
  if (!p) return fail(RECON_E_INVALID_ARG, "recon_run_host: null plan");
  const size_t nvox = (size_t)p->nx * p->ny * p->nz;
  if (nvox > 0 && !volume) return fail(RECON_E_INVALID_ARG, "recon_run_host: null volume");
  if (p->D > 0 && !host_images) return fail(RECON_E_INVALID_ARG, "recon_run_host: null host images");
  if (p->opt.check_finite)
    return fail(RECON_E_INVALID_ARG, "recon_run_host: check_finite is not supported with host images");
  cudaStream_t s = (cudaStream_t)stream;
  if (p->D == 0 || nvox == 0) {
    if (nvox > 0 && !p->opt.accumulate) {
      cudaError_t e = cudaMemsetAsync(volume, 0, nvox * sizeof(float), s);
      if (e != cudaSuccess) return cuda_fail(e, "recon_run_host: clearing the volume");
    }
    return RECON_OK;
  }
  const size_t slot = host_slot_bytes(p), need = p->ws_bytes + 2 * slot;
  if (!workspace || ((uintptr_t)workspace & 255) != 0 || ws_bytes < need)
    return fail(RECON_E_WORKSPACE, "recon_run_host: workspace too small or misaligned (needs " +
                                       std::to_string(need) + " bytes)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "recon_run_host: current device");
  if (p->copy_dev != dev) {  // the copy stream and its events, on this device
    p->release_copy_stream();
    e = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&p->ev_start, &p->ev_ready[0], &p->ev_ready[1], &p->ev_free[0], &p->ev_free[1]})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      p->release_copy_stream();
      return cuda_fail(e, "recon_run_host: creating the copy stream");
    }
    p->copy_dev = dev;
  }
  const recon::Workspace w = carve(p, workspace);
  int rc = upload_tables(p, w, s);
  if (rc) return rc;
  rc = tma_begin(p, workspace, s, "recon_run_host");
  if (rc) return rc;
  float* slots[2] = {(float*)((char*)workspace + p->ws_bytes), (float*)((char*)workspace + p->ws_bytes + slot)};
  const size_t img = (size_t)p->nv * p->nu;
  // the copies overwrite the slots only after everything queued on `stream` before this call
  e = cudaEventRecord(p->ev_start, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->copy_stream, p->ev_start, 0);
  if (e != cudaSuccess) return cuda_fail(e, "recon_run_host: ordering the copy stream");
  auto issue_copy = [&](int b) -> cudaError_t {
    const int d0 = b * p->db, cnt = (p->D - d0) < p->db ? (p->D - d0) : p->db;
    cudaError_t ec = cudaSuccess;
    if (b >= 2) ec = cudaStreamWaitEvent(p->copy_stream, p->ev_free[b % 2], 0);  // block b - 2 read the slot
    if (ec == cudaSuccess)
      ec = cudaMemcpyAsync(slots[b % 2], host_images + (size_t)d0 * img, sizeof(float) * (size_t)cnt * img,
                           cudaMemcpyHostToDevice, p->copy_stream);
    if (ec == cudaSuccess) ec = cudaEventRecord(p->ev_ready[b % 2], p->copy_stream);
    return ec;
  };
  MlpHookCtx hctx{p, (const char*)workspace, (float*)((char*)workspace + p->off_pow), w.eps, w.S, w.twp};
  const recon::StageAHook hook{mlp_hook, &hctx};
  const recon::StageAHook* hk = p->ca.filter == RECON_FILTER_MLP ? &hook : nullptr;
  e = issue_copy(0);
  if (e != cudaSuccess) return cuda_fail(e, "recon_run_host: image copy");
  for (int b = 0; b < p->n_blocks; ++b) {
    const int d0 = b * p->db;
    const int cnt = (p->D - d0) < p->db ? (p->D - d0) : p->db;
    if (b + 1 < p->n_blocks) {
      e = issue_copy(b + 1);
      if (e != cudaSuccess) return cuda_fail(e, "recon_run_host: image copy");
    }
    e = cudaStreamWaitEvent(s, p->ev_ready[b % 2], 0);
    if (e != cudaSuccess) return cuda_fail(e, "recon_run_host: waiting for the images");
    // the kernels index images by absolute direction: the slot's address shifted back by d0
    // images puts direction d0 at the slot's start (only the slot itself is read)
    const float* images = (const float*)((uintptr_t)slots[b % 2] - (uintptr_t)d0 * img * sizeof(float));
    e = recon::launch_stage_a(p->ca, w, images, d0, cnt, s, nullptr, hk);
    if (e != cudaSuccess) return cuda_fail(e, "recon_run_host: stage A launch");
    e = cudaEventRecord(p->ev_free[b % 2], s);  // stage A has read the slot once this point passes
    if (e != cudaSuccess) return cuda_fail(e, "recon_run_host: slot release");
    e = backproject_block(p, w.dirs, w.stack, d0, cnt, volume, p->opt.accumulate || b > 0, workspace, s);
    if (e != cudaSuccess) return cuda_fail(e, "recon_run_host: backprojection launch");
  }
  return tma_end(p, workspace, s, "recon_run_host");
}

int recon_filter_stage(recon_plan_t p, const float* images, int dir_begin, int dir_count, void* workspace,
                       size_t ws_bytes, void* stream, const void** stack_out) {
  if (!p || !stack_out) return fail(RECON_E_INVALID_ARG, "recon_filter_stage: null plan or stack_out");
  if (dir_begin < 0 || dir_count < 0 || dir_begin + dir_count > p->D || dir_count > p->db)
    return fail(RECON_E_INVALID_ARG, "recon_filter_stage: direction range outside the plan or above its block size");
  if (dir_count > 0 && !images) return fail(RECON_E_INVALID_ARG, "recon_filter_stage: null images");
  int rc = check_ws(p, workspace, ws_bytes, "recon_filter_stage");
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const recon::Workspace w = carve(p, workspace);
  rc = upload_tables(p, w, s);
  if (rc) return rc;
  MlpHookCtx hctx{p, (const char*)workspace, (float*)((char*)workspace + p->off_pow), w.eps, w.S, w.twp};
  const recon::StageAHook hook{mlp_hook, &hctx};
  cudaError_t e = recon::launch_stage_a(p->ca, w, images, dir_begin, dir_count, s, nullptr,
                                        p->ca.filter == RECON_FILTER_MLP ? &hook : nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "recon_filter_stage: launch");
  *stack_out = w.stack;
  return RECON_OK;
}

int recon_backproject(recon_plan_t p, const void* stack, int dir_begin, int dir_count, float* volume, int accumulate,
                      void* workspace, size_t ws_bytes, void* stream) {
  if (!p) return fail(RECON_E_INVALID_ARG, "recon_backproject: null plan");
  if (dir_begin < 0 || dir_count < 0 || dir_begin + dir_count > p->D || dir_count > 1024)
    return fail(RECON_E_INVALID_ARG, "recon_backproject: direction range outside the plan (or > 1024 directions)");
  const size_t nvox = (size_t)p->nx * p->ny * p->nz;
  if (nvox > 0 && !volume) return fail(RECON_E_INVALID_ARG, "recon_backproject: null volume");
  if (dir_count > 0 && !stack) return fail(RECON_E_INVALID_ARG, "recon_backproject: null stack");
  cudaStream_t s = (cudaStream_t)stream;
  if (dir_count == 0 || nvox == 0) {
    if (nvox > 0 && !accumulate) {
      cudaError_t e = cudaMemsetAsync(volume, 0, nvox * sizeof(float), s);
      if (e != cudaSuccess) return cuda_fail(e, "recon_backproject: clearing the volume");
    }
    return RECON_OK;
  }
  int rc = check_ws(p, workspace, ws_bytes, "recon_backproject");
  if (rc) return rc;
  const recon::Workspace w = carve(p, workspace);
  rc = upload_tables(p, w, s);
  if (rc) return rc;
  rc = tma_begin(p, workspace, s, "recon_backproject");
  if (rc) return rc;
  cudaError_t e = backproject_block(p, w.dirs, stack, dir_begin, dir_count, volume, accumulate, workspace, s);
  if (e != cudaSuccess) return cuda_fail(e, "recon_backproject: launch");
  return tma_end(p, workspace, s, "recon_backproject");
}

int recon_selftest_wait_limit(void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, 16384);
  if (e != cudaSuccess) return cuda_fail(e, "recon_selftest_wait_limit: allocation");
  unsigned int* d_status = (unsigned int*)((char*)buf + 12288);
  unsigned int h = 0;
  e = cudaMemsetAsync(d_status, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = recon::launch_tma_wait_probe(buf, 12288, d_status, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_status, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  const cudaError_t ef = cudaFree(buf);
  if (e == cudaSuccess) e = ef;
  if (e != cudaSuccess) return cuda_fail(e, "recon_selftest_wait_limit");
  if ((h & 1u) == 0)
    return fail(RECON_E_DEVICE_CHECK, "recon_selftest_wait_limit: the kernel did not report its run-out wait");
  return RECON_OK;
}

int recon_profile_enable(recon_plan_t p, int enable) {
  if (!p) return fail(RECON_E_INVALID_ARG, "recon_profile_enable: null plan");
  if (enable && p->events.empty()) {
    const int sub = p->ca.sub_block > 0 ? p->ca.sub_block : 1;
    const size_t n = 1 + (size_t)p->n_blocks * (3 * (size_t)((p->db + sub - 1) / sub) + 1);
    p->events.resize(n);
    p->event_kind.assign(n, -1);
    for (size_t i = 0; i < n; ++i) {
      cudaError_t e = cudaEventCreate(&p->events[i]);
      if (e != cudaSuccess) {
        p->events.resize(i);
        return cuda_fail(e, "recon_profile_enable: cudaEventCreate");
      }
    }
  }
  p->profile = enable != 0;
  p->profiled_events = 0;
  return RECON_OK;
}

int recon_profile_read(recon_plan_t p, double* ms, int* launches) {
  if (!p || !ms || !launches) return fail(RECON_E_INVALID_ARG, "recon_profile_read: null argument");
  for (int q = 0; q < 4; ++q) {
    ms[q] = 0.0;
    launches[q] = 0;
  }
  if (p->profiled_events < 2) return RECON_OK;
  cudaError_t e = cudaEventSynchronize(p->events[p->profiled_events - 1]);
  if (e != cudaSuccess) return cuda_fail(e, "recon_profile_read: cudaEventSynchronize");
  for (int i = 1; i < p->profiled_events; ++i) {
    const int k = p->event_kind[i];
    if (k < 0 || k > 3) continue;
    float t = 0.f;
    e = cudaEventElapsedTime(&t, p->events[i - 1], p->events[i]);
    if (e != cudaSuccess) return cuda_fail(e, "recon_profile_read: cudaEventElapsedTime");
    ms[k] += t;
    launches[k] += 1;
  }
  return RECON_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ 3D-Fourier forms
namespace {

size_t grid3_cells(recon_plan_t p) { return (size_t)p->f3.P3[0] * p->f3.P3[1] * p->f3.P3[2]; }

struct SwapLayout {
  size_t vc, vs, Z, work, tw[3], total;
};

SwapLayout swap_layout(recon_plan_t p) {
  SwapLayout L;
  const size_t nvox = (size_t)p->nx * p->ny * p->nz;
  size_t off = align256(p->ws_bytes);
  L.vc = off;
  off = align256(off + nvox * sizeof(float));
  L.vs = off;
  off = align256(off + nvox * sizeof(float));
  L.Z = off;
  off = align256(off + grid3_cells(p) * sizeof(float2));
  L.work = off;
  off = align256(off + grid3_cells(p) * sizeof(float2));
  for (int a = 0; a < 3; ++a) {
    L.tw[a] = off;
    off = align256(off + p->tw3[a].size() * sizeof(float2));
  }
  L.total = off;
  return L;
}

struct GridLayout {
  size_t Srows, G, dirs, acc, raw, S, stats, tw[3], total;
  int sub;
};

GridLayout grid_layout(recon_plan_t p) {
  GridLayout L;
  const size_t per_dir = (size_t)p->half * p->P * sizeof(float2) + (size_t)p->nv * p->half * sizeof(float2);
  L.sub = (int)std::max<size_t>(1, std::min<size_t>((size_t)(p->D > 0 ? p->D : 1), ((size_t)1 << 30) / per_dir));
  size_t off = p->table_bytes;
  L.Srows = off;
  off = align256(off + (size_t)L.sub * p->nv * p->half * sizeof(float2));
  L.G = off;
  off = align256(off + (size_t)L.sub * p->half * p->P * sizeof(float2));
  L.dirs = off;
  off = align256(off + p->gdirs.size() * sizeof(recon::GridDir));
  L.acc = off;
  off = align256(off + grid3_cells(p) * sizeof(float2));
  L.raw = off;
  off = align256(off + grid3_cells(p) * sizeof(float2));
  L.S = off;
  off = align256(off + grid3_cells(p) * sizeof(float));
  L.stats = off;
  off = align256(off + 2 * sizeof(double));
  for (int a = 0; a < 3; ++a) {
    L.tw[a] = off;
    off = align256(off + p->tw3[a].size() * sizeof(float2));
  }
  L.total = off;
  return L;
}

int f3_check(recon_plan_t p, const char* who) {
  if (!p) return fail(RECON_E_INVALID_ARG, std::string(who) + ": null plan");
  if (!p->f3_ok)
    return fail(RECON_E_UNSUPPORTED_SIZE,
                std::string(who) + ": the 3D-Fourier forms need every grid side <= 1024 (padded grid <= 2048)");
  if (p->P < 16) return fail(RECON_E_UNSUPPORTED_SIZE, std::string(who) + ": images of more than 8 pixels needed");
  return RECON_OK;
}

int upload_tw3(recon_plan_t p, char* b, const size_t off[3], float2* dev[3], cudaStream_t s) {
  for (int a = 0; a < 3; ++a) {
    dev[a] = (float2*)(b + off[a]);
    const cudaError_t e =
        cudaMemcpyAsync(dev[a], p->tw3[a].data(), sizeof(float2) * p->tw3[a].size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "upload of the 3D FFT twiddles");
  }
  return RECON_OK;
}

// the twiddle table of one axis as the line FFT of that length reads it (fft3.cu)
const float2* axis_tw(recon_plan_t p, float2* dev, int a) {
  return p->f3.P3[a] >= 1024 ? dev + (p->f3.P3[a] - 8) : dev;
}

}  // namespace

extern "C" {

int recon_swap_workspace_size(recon_plan_t p, size_t* bytes) {
  int rc = f3_check(p, "recon_swap_workspace_size");
  if (rc) return rc;
  if (!bytes) return fail(RECON_E_INVALID_ARG, "recon_swap_workspace_size: null bytes");
  *bytes = swap_layout(p).total;
  return RECON_OK;
}

int recon_swap_ct(recon_plan_t p, const float* images, void* workspace, size_t ws_bytes, void* stream) {
  int rc = f3_check(p, "recon_swap_ct");
  if (rc) return rc;
  if (p->opt.filter != RECON_FILTER_PAIR)
    return fail(RECON_E_INVALID_ARG, "recon_swap_ct: the plan must use RECON_FILTER_PAIR (its depth tables)");
  if (!p->uniform_R) return fail(RECON_E_INVALID_ARG, "recon_swap_ct: Eq. 12 needs one defocus for every view");
  if (p->D > 0 && !images) return fail(RECON_E_INVALID_ARG, "recon_swap_ct: null images");
  const SwapLayout L = swap_layout(p);
  if (!workspace || ((uintptr_t)workspace & 255) != 0 || ws_bytes < L.total)
    return fail(RECON_E_WORKSPACE, "recon_swap_ct: workspace too small or misaligned (needs " +
                                       std::to_string(L.total) + " bytes)");
  cudaStream_t s = (cudaStream_t)stream;
  char* b = (char*)workspace;
  const recon::Workspace w = carve(p, workspace);
  rc = upload_tables(p, w, s);
  if (rc) return rc;
  float2* tw[3];
  rc = upload_tw3(p, b, L.tw, tw, s);
  if (rc) return rc;
  float* vc = (float*)(b + L.vc);
  float* vs = (float*)(b + L.vs);
  const size_t nvox = (size_t)p->nx * p->ny * p->nz;
  rc = tma_begin(p, workspace, s, "recon_swap_ct");
  if (rc) return rc;
  for (int mode = 1; mode <= 2; ++mode) {  // cos, then sin of the layer's depth phase, no CTF
    float* vol = mode == 1 ? vc : vs;
    recon::StageAConst ca = p->ca;
    ca.pair_mode = mode;
    ca.pref = 1.0f;
    if (p->D == 0) {
      const cudaError_t e = cudaMemsetAsync(vol, 0, nvox * sizeof(float), s);
      if (e != cudaSuccess) return cuda_fail(e, "recon_swap_ct: clearing");
    }
    for (int bk = 0; bk < p->n_blocks; ++bk) {
      const int d0 = bk * p->db;
      const int cnt = (p->D - d0) < p->db ? (p->D - d0) : p->db;
      cudaError_t e = recon::launch_stage_a(ca, w, images, d0, cnt, s);
      if (e != cudaSuccess) return cuda_fail(e, "recon_swap_ct: stage A launch");
      e = backproject_block(p, w.dirs, w.stack, d0, cnt, vol, bk > 0, workspace, s);
      if (e != cudaSuccess) return cuda_fail(e, "recon_swap_ct: backprojection launch");
    }
  }
  rc = tma_end(p, workspace, s, "recon_swap_ct");
  if (rc) return rc;
  float2* Z = (float2*)(b + L.Z);
  cudaError_t e = recon::launch_swap_pack(vc, vs, Z, p->f3, s);
  const float2* twa[3] = {axis_tw(p, tw[0], 0), axis_tw(p, tw[1], 1), axis_tw(p, tw[2], 2)};
  if (e == cudaSuccess) e = recon::launch_fft3(Z, p->f3.P3, twa, false, s);
  if (e != cudaSuccess) return cuda_fail(e, "recon_swap_ct: 3D transform");
  return RECON_OK;
}

int recon_swap_phase(recon_plan_t p, double sigma, double eps, float* volume, void* workspace, size_t ws_bytes,
                     void* stream) {
  int rc = f3_check(p, "recon_swap_phase");
  if (rc) return rc;
  if (!(eps > 0.0) || !std::isfinite(eps) || !std::isfinite(sigma))
    return fail(RECON_E_INVALID_ARG, "recon_swap_phase: eps > 0 and a finite sigma needed");
  if (!volume) return fail(RECON_E_INVALID_ARG, "recon_swap_phase: null volume");
  const SwapLayout L = swap_layout(p);
  if (!workspace || ((uintptr_t)workspace & 255) != 0 || ws_bytes < L.total)
    return fail(RECON_E_WORKSPACE, "recon_swap_phase: workspace too small or misaligned");
  cudaStream_t s = (cudaStream_t)stream;
  char* b = (char*)workspace;
  float2* tw[3] = {(float2*)(b + L.tw[0]), (float2*)(b + L.tw[1]), (float2*)(b + L.tw[2])};
  const float2* twa[3] = {axis_tw(p, tw[0], 0), axis_tw(p, tw[1], 1), axis_tw(p, tw[2], 2)};
  float2* work = (float2*)(b + L.work);
  cudaError_t e = recon::launch_swap_phase((const float2*)(b + L.Z), work, p->f3, p->R0, sigma, eps, p->opt.cs, s);
  if (e == cudaSuccess) e = recon::launch_fft3(work, p->f3.P3, twa, true, s);
  if (e == cudaSuccess) e = recon::launch_crop_real(work, volume, p->f3, s);
  if (e != cudaSuccess) return cuda_fail(e, "recon_swap_phase");
  return RECON_OK;
}

int recon_grid_workspace_size(recon_plan_t p, size_t* bytes) {
  int rc = f3_check(p, "recon_grid_workspace_size");
  if (rc) return rc;
  if (!bytes) return fail(RECON_E_INVALID_ARG, "recon_grid_workspace_size: null bytes");
  *bytes = grid_layout(p).total;
  return RECON_OK;
}

int recon_grid_run(recon_plan_t p, const float* images, float* volume, double nsr, void* workspace, size_t ws_bytes,
                   void* stream) {
  int rc = f3_check(p, "recon_grid_run");
  if (rc) return rc;
  if (p->opt.filter != RECON_FILTER_TIKHONOV && p->opt.filter != RECON_FILTER_PAIR)
    return fail(RECON_E_INVALID_ARG, "recon_grid_run: the plan's filter must carry eps (Tikhonov or pair)");
  if (!(nsr >= 0.0) || !std::isfinite(nsr)) return fail(RECON_E_INVALID_ARG, "recon_grid_run: nsr must be >= 0");
  if (!volume || (p->D > 0 && !images)) return fail(RECON_E_INVALID_ARG, "recon_grid_run: null images or volume");
  const GridLayout L = grid_layout(p);
  if (!workspace || ((uintptr_t)workspace & 255) != 0 || ws_bytes < L.total)
    return fail(RECON_E_WORKSPACE, "recon_grid_run: workspace too small or misaligned (needs " +
                                       std::to_string(L.total) + " bytes)");
  cudaStream_t s = (cudaStream_t)stream;
  char* b = (char*)workspace;
  const recon::Workspace w = carve(p, workspace);
  rc = upload_tables(p, w, s);
  if (rc) return rc;
  float2* tw[3];
  rc = upload_tw3(p, b, L.tw, tw, s);
  if (rc) return rc;
  recon::GridDir* gd = (recon::GridDir*)(b + L.dirs);
  float2* acc = (float2*)(b + L.acc);
  float2* raw = (float2*)(b + L.raw);
  float* S = (float*)(b + L.S);
  const size_t cells = grid3_cells(p);
  cudaError_t e = cudaMemcpyAsync(gd, p->gdirs.data(), sizeof(recon::GridDir) * p->gdirs.size(),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, cells * sizeof(float2), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(raw, 0, cells * sizeof(float2), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(S, 0, cells * sizeof(float), s);
  float2* Srows = (float2*)(b + L.Srows);
  float2* G = (float2*)(b + L.G);
  for (int d0 = 0; d0 < p->D && e == cudaSuccess; d0 += L.sub) {
    const int cnt = std::min(L.sub, p->D - d0);
    e = recon::launch_rows_fwd(p->ca, Srows, w.twp, images, d0, cnt, s);
    if (e == cudaSuccess) e = recon::launch_cols_forward(p->ca, p->lc, Srows, G, nullptr, w.twp, cnt, s);
    if (e == cudaSuccess) e = recon::launch_grid_splat(G, gd, d0, cnt, p->ca, p->f3, acc, raw, S, nsr > 0.0, s);
  }
  const float nsr_m = (float)(nsr * std::sqrt((double)p->nu * p->nv));
  if (e == cudaSuccess) e = recon::launch_grid_finish(acc, raw, S, (double*)(b + L.stats), p->f3, nsr_m, s);
  const float2* twa[3] = {axis_tw(p, tw[0], 0), axis_tw(p, tw[1], 1), axis_tw(p, tw[2], 2)};
  if (e == cudaSuccess) e = recon::launch_fft3(acc, p->f3.P3, twa, true, s);
  if (e == cudaSuccess) e = recon::launch_crop_real(acc, volume, p->f3, s);
  if (e != cudaSuccess) return cuda_fail(e, "recon_grid_run");
  return RECON_OK;
}

}  // extern "C"

extern "C" {

int recon_sync(void* stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "recon_sync");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "recon_sync");
  return RECON_OK;
}

}  // extern "C"

namespace recon {

void set_last_error(const char* msg) { g_last_error = msg; }

int run_in_scratch(recon_plan_t p, const float* images, float* volume, char* scratch, size_t scratch_bytes,
                   cudaStream_t s) {
  if (!p) return fail(RECON_E_INVALID_ARG, "recon_run_noalloc: null plan");
  const size_t nvox = (size_t)p->nx * p->ny * p->nz;
  if (nvox > 0 && !volume) return fail(RECON_E_INVALID_ARG, "recon_run_noalloc: null volume");
  if (p->D > 0 && !images) return fail(RECON_E_INVALID_ARG, "recon_run_noalloc: null images");
  // Same table head as the caller-owned workspace, then the largest direction block
  // whose spectra, intermediates and stacks still fit the scratch.
  const size_t spec = (size_t)p->nv * p->half * 8;
  const size_t inter = spec * p->nzl;
  const bool mlp = p->ca.filter == RECON_FILTER_MLP;
  const size_t sub = (size_t)(p->ca.sub_block > 0 ? p->ca.sub_block : 1);
  auto need = [&](size_t db) {
    const size_t sb = db < sub ? db : sub;
    size_t b = p->table_bytes + align256(sb * spec) + align256(sb * inter) + align256(db * p->stack_dir_bytes);
    if (mlp) b += align256(sizeof(float) * sb * p->lc.n_bins) + align256(sizeof(float) * sb * p->nzl * p->lc.n_bins);
    return b;
  };
  if (need(1) > scratch_bytes)
    return fail(RECON_E_UNSUPPORTED_SIZE, "recon_run_noalloc: this plan needs " + std::to_string(need(1)) +
                                              " bytes of scratch for one direction; the static scratch holds " +
                                              std::to_string(scratch_bytes));
  if (p->D == 0 || nvox == 0) {
    if (nvox > 0 && !p->opt.accumulate) {
      cudaError_t e = cudaMemsetAsync(volume, 0, nvox * sizeof(float), s);
      if (e != cudaSuccess) return cuda_fail(e, "recon_run_noalloc: clearing the volume");
    }
    return RECON_OK;
  }
  if (p->opt.check_finite) {
    const int rc = scan_finite(p, images, (unsigned int*)(scratch + p->off_flag), s, "recon_run_noalloc");
    if (rc) return rc;
  }
  size_t db = 1;
  while ((int)db < p->db && need(db + 1) <= scratch_bytes) ++db;
  recon::Workspace w;
  w.dirs = (recon::DirParams*)(scratch + p->off_dirs);
  w.uA = (uint64_t*)(scratch + p->off_uA);
  w.ramp = (float*)(scratch + p->off_ramp);
  w.tw = (float2*)(scratch + p->off_tw);
  w.twp = (float2*)(scratch + p->off_twp);
  w.dens = (float*)(scratch + p->off_dens);
  w.band_sum = (double*)(scratch + p->off_dsum);
  const size_t sb = db < sub ? db : sub;
  size_t off = p->table_bytes;
  w.S = (float2*)(scratch + off);
  off += align256(sb * spec);
  w.T = (float2*)(scratch + off);
  off += align256(sb * inter);
  w.stack = (void*)(scratch + off);
  off += align256(db * p->stack_dir_bytes);
  float* pow = (float*)(scratch + off);
  if (mlp) off += align256(sizeof(float) * sb * p->lc.n_bins);
  w.eps = (float*)(scratch + off);
  w.n_bins = p->lc.n_bins;
  w.bin_width = p->lc.bin_width;
  int rc = upload_tables(p, w, s);
  if (rc) return rc;
  MlpHookCtx hctx{p, scratch, pow, w.eps, w.S, w.twp};
  const recon::StageAHook hook{mlp_hook, &hctx};
  recon::StageAConst ca = p->ca;
  if (p->P >= 16) ca.sub_block = (int)sb;
  const int n_blocks = (int)((p->D + db - 1) / db);
  for (int b = 0; b < n_blocks; ++b) {
    const int d0 = b * (int)db;
    const int cnt = (p->D - d0) < (int)db ? (p->D - d0) : (int)db;
    cudaError_t e = recon::launch_stage_a(ca, w, images, d0, cnt, s, nullptr, mlp ? &hook : nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "recon_run_noalloc: stage A launch");
    e = recon::launch_backproject(p->cb, w.dirs, w.stack, d0, cnt, volume, p->opt.accumulate || b > 0, s);
    if (e != cudaSuccess) return cuda_fail(e, "recon_run_noalloc: backprojection launch");
  }
  return RECON_OK;
}

}  // namespace recon

// ------------------------------------------------------------------ training
namespace {

struct TrainLayout {
  size_t S, G, T, pow, eps, acts, deps, theta, grad, m1, m2, sums, loss, total;
};

int train_plan(const recon_train_cfg* c, recon_plan_t* out) {
  recon_geometry g{c->n_img, c->nu, c->nv, c->rot};
  recon_grid gr{c->grid_nx, c->grid_ny, c->grid_nz};
  recon_options o;
  recon_default_options(&o);
  o.sigma = c->sigma;
  o.cs = c->cs;
  o.nsr = c->nsr;
  o.input_mode = c->input_mode;
  o.dir_block = c->n_img;
  return plan_create(&g, c->lambda, c->delta, c->defocus, c->nz_layers, &gr, &o, out, true);
}

int train_check(const recon_train_cfg* c) {
  if (!c) return fail(RECON_E_INVALID_ARG, "recon_mlp_train: null config");
  if (c->n_img < 1 || c->nz_layers < 1 || c->steps < 0)
    return fail(RECON_E_INVALID_ARG, "recon_mlp_train: n_img, nz_layers >= 1 and steps >= 0 needed");
  if (!(c->nsr > 0.0) || !std::isfinite(c->nsr)) return fail(RECON_E_INVALID_ARG, "recon_mlp_train: nsr must be > 0");
  if (c->steps > 0 && !(c->lr > 0.f)) return fail(RECON_E_INVALID_ARG, "recon_mlp_train: lr must be > 0");
  if (c->adam_step < 0) return fail(RECON_E_INVALID_ARG, "recon_mlp_train: adam_step must be >= 0");
  return RECON_OK;
}

TrainLayout train_layout(recon_plan_t p, const recon_train_cfg* c) {
  TrainLayout L;
  const size_t N = c->n_img, K = c->nz_layers, NB = p->lc.n_bins, half = p->half, P = p->P;
  size_t off = p->table_bytes;
  L.S = off;
  off = align256(off + N * K * p->nv * half * 8);
  L.G = off;
  off = align256(off + N * half * P * 8);
  L.T = off;
  off = align256(off + N * K * half * P * 8);
  L.pow = off;
  off = align256(off + N * NB * 4);
  L.eps = off;
  off = align256(off + N * K * NB * 4);
  L.acts = off;
  off = align256(off + N * K * NB * recon::kActStride * 4);
  L.deps = off;
  off = align256(off + N * K * NB * 8);
  L.theta = off;
  off = align256(off + recon::kMlpParams * 4);
  L.grad = off;
  off = align256(off + recon::kMlpParams * 4);
  L.m1 = off;
  off = align256(off + recon::kMlpParams * 4);
  L.m2 = off;
  off = align256(off + recon::kMlpParams * 4);
  L.sums = off;
  off = align256(off + 2 * sizeof(double));
  L.loss = off;
  off = align256(off + sizeof(float) * (size_t)(c->steps > 0 ? c->steps : 1));
  L.total = off;
  return L;
}

}  // namespace

extern "C" int recon_mlp_train_workspace_size(const recon_train_cfg* cfg, size_t* bytes) {
  int rc = train_check(cfg);
  if (rc) return rc;
  if (!bytes) return fail(RECON_E_INVALID_ARG, "recon_mlp_train_workspace_size: null bytes");
  recon_plan_t p = nullptr;
  rc = train_plan(cfg, &p);
  if (rc) return rc;
  *bytes = train_layout(p, cfg).total;
  recon_destroy(p);
  return RECON_OK;
}

extern "C" int recon_mlp_train(const recon_train_cfg* cfg, float* weights, float* loss_history, float* grad,
                               void* workspace, size_t ws_bytes, void* stream) {
  int rc = train_check(cfg);
  if (rc) return rc;
  if (!weights || !loss_history || !cfg->images || !cfg->targets)
    return fail(RECON_E_INVALID_ARG, "recon_mlp_train: null weights, loss_history, images or targets");
  recon_plan_t p = nullptr;
  rc = train_plan(cfg, &p);
  if (rc) return rc;
  struct Guard {
    recon_plan_t p;
    ~Guard() { recon_destroy(p); }
  } guard{p};
  if (p->P < 16) return fail(RECON_E_UNSUPPORTED_SIZE, "recon_mlp_train: images of more than 4 pixels needed");
  const TrainLayout L = train_layout(p, cfg);
  if (!workspace || ((uintptr_t)workspace & 255) != 0 || ws_bytes < L.total)
    return fail(RECON_E_WORKSPACE, "recon_mlp_train: workspace too small or misaligned (needs " +
                                       std::to_string(L.total) + " bytes)");
  cudaStream_t s = (cudaStream_t)stream;
  char* b = (char*)workspace;
  const recon::Workspace w = carve(p, workspace);
  rc = upload_tables(p, w, s);
  if (rc) return rc;
  const int N = cfg->n_img, K = cfg->nz_layers;
  float2* S = (float2*)(b + L.S);
  float2* G = (float2*)(b + L.G);
  float2* T = (float2*)(b + L.T);
  float* pow = (float*)(b + L.pow);
  float* eps = (float*)(b + L.eps);
  float* acts = (float*)(b + L.acts);
  double* deps = (double*)(b + L.deps);
  float* theta = (float*)(b + L.theta);
  float* g = (float*)(b + L.grad);
  float* m1 = (float*)(b + L.m1);
  float* m2 = (float*)(b + L.m2);
  double* sums = (double*)(b + L.sums);
  float* loss = (float*)(b + L.loss);
  const float* cnt = (const float*)(b + p->off_cnt);
  const float* x2 = (const float*)(b + p->off_x2);
  cudaError_t e = cudaMemcpyAsync(theta, weights, sizeof(float) * recon::kMlpParams, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(pow, 0, sizeof(float) * (size_t)N * p->lc.n_bins, s);
  // grad, m1 and m2 (separate 256-byte aligned arrays: the padding between them is not cleared);
  // the moments continue an earlier call's when the caller passes them
  if (e == cudaSuccess) e = cudaMemsetAsync(g, 0, sizeof(float) * recon::kMlpParams, s);
  if (cfg->adam_state) {
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(m1, cfg->adam_state, sizeof(float) * recon::kMlpParams, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(m2, cfg->adam_state + recon::kMlpParams, sizeof(float) * recon::kMlpParams,
                          cudaMemcpyHostToDevice, s);
  } else {
    for (float* a : {m1, m2})
      if (e == cudaSuccess) e = cudaMemsetAsync(a, 0, sizeof(float) * recon::kMlpParams, s);
  }
  // spectra of the images (and their radial power) and of the layer targets
  if (e == cudaSuccess) e = recon::launch_rows_fwd(p->ca, S, w.twp, cfg->images, 0, N, s);
  if (e == cudaSuccess) e = recon::launch_cols_forward(p->ca, p->lc, S, G, pow, w.twp, N, s);
  recon::StageAConst ct = p->ca;
  ct.input_mode = RECON_INPUT_CONTRAST;
  if (e == cudaSuccess) e = recon::launch_rows_fwd(ct, S, w.twp, cfg->targets, 0, N * K, s);
  if (e == cudaSuccess) e = recon::launch_cols_forward(ct, p->lc, S, T, nullptr, w.twp, N * K, s);
  const int iters = cfg->steps > 0 ? cfg->steps : 1;
  for (int it = 0; it < iters && e == cudaSuccess; ++it) {
    e = cudaMemsetAsync(sums, 0, 2 * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(deps, 0, sizeof(double) * (size_t)N * K * p->lc.n_bins, s);
    if (e == cudaSuccess) e = recon::launch_eps_table(p->lc, pow, cnt, x2, theta, eps, acts, N, K, 0, s);
    if (e == cudaSuccess)
      e = recon::launch_train_step(p->ca, p->lc, G, T, eps, w.uA, acts, theta, theta, g, m1, m2, N, sums, deps,
                                   cfg->steps > 0 ? cfg->adam_step + it + 1 : 0, cfg->lr, loss + it, s);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(loss_history, loss, sizeof(float) * iters, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && cfg->steps > 0)
    e = cudaMemcpyAsync(weights, theta, sizeof(float) * recon::kMlpParams, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && cfg->steps > 0 && cfg->adam_state) {
    e = cudaMemcpyAsync(cfg->adam_state, m1, sizeof(float) * recon::kMlpParams, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(cfg->adam_state + recon::kMlpParams, m2, sizeof(float) * recon::kMlpParams,
                          cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess && cfg->steps == 0 && grad)
    e = cudaMemcpyAsync(grad, g, sizeof(float) * recon::kMlpParams, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "recon_mlp_train");
  return RECON_OK;
}

// ------------------------------------------------------------------ batches of tomograms
struct recon_batch_s {
  int n = 0, dbb = 0, n_rounds = 0;
  std::vector<recon_plan_t> plans;
  std::vector<size_t> off_tables, off_stack;
  size_t off_S = 0, off_T = 0, off_pow = 0, off_eps = 0, off_desc = 0, off_ctr = 0, ws_bytes = 0, smem = 0;
  std::vector<recon::BatchBp> desc;        // [n_rounds][n] (first round_count[r] used)
  std::vector<int> round_count;
  std::vector<unsigned long long> round_total;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<const void*> graph_ptrs;     // pointers the captured graph was built for
  // recon_batch_run_host: per tomogram a sub-slot of dbb images in each of two round slots,
  // the copy stream and its events (created on first use, per device)
  std::vector<size_t> off_img;             // sub-slot offsets within a round slot
  size_t slot_bytes = 0;
  int copy_dev = -1;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_start = nullptr, ev_ready[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  void release_copy_stream() {
    if (copy_stream) cudaStreamDestroy(copy_stream);
    for (cudaEvent_t e : {ev_start, ev_ready[0], ev_ready[1], ev_free[0], ev_free[1]})
      if (e) cudaEventDestroy(e);
    copy_stream = nullptr;
    ev_start = ev_ready[0] = ev_ready[1] = ev_free[0] = ev_free[1] = nullptr;
    copy_dev = -1;
  }
  ~recon_batch_s() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    release_copy_stream();
  }
};

namespace {

// Fills the device tables of every plan and the per-round backprojection descriptors.
int batch_prepare(recon_batch_t bt, const float* const* images, float* const* volumes, char* base, cudaStream_t s) {
  for (int q = 0; q < bt->n; ++q) {
    recon_plan_t p = bt->plans[q];
    const recon::Workspace w = carve(p, base + bt->off_tables[q]);
    int rc = upload_tables(p, w, s);
    if (rc) return rc;
  }
  for (int r = 0; r < bt->n_rounds; ++r) {
    unsigned long long first = 0;
    int cntr = 0;
    for (int q = 0; q < bt->n; ++q) {
      recon_plan_t p = bt->plans[q];
      const int d0 = r * bt->dbb;
      if (d0 >= p->D) continue;
      const int cnt = (p->D - d0) < bt->dbb ? (p->D - d0) : bt->dbb;
      recon::BatchBp& d = bt->desc[(size_t)r * bt->n + cntr];
      const recon::Workspace w = carve(p, base + bt->off_tables[q]);
      recon::describe_backproject(p->cb, w.dirs, base + bt->off_stack[q], d0, cnt, volumes[q],
                                  p->opt.accumulate || r > 0, &d);
      d.first_item = first;
      first += (unsigned long long)d.gx * d.gy * d.gz;
      ++cntr;
    }
    bt->round_count[r] = cntr;
    bt->round_total[r] = first;
  }
  cudaError_t e = cudaMemcpyAsync(base + bt->off_desc, bt->desc.data(), sizeof(recon::BatchBp) * bt->desc.size(),
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "recon_batch: descriptor upload");
  (void)images;
  return RECON_OK;
}

// The kernels of one batch run (capturable: no host copies).
// recon_batch_run_host's uploads: host images, round slots in the workspace.
struct HostUpload {
  const float* const* host;  // [n] host images
  char* slots[2];            // round slots
};

// The images of round r, tomogram by tomogram, into round slot r % 2 on the copy stream
// (after the stage A that read that slot two rounds earlier).
cudaError_t batch_upload_round(recon_batch_t bt, const HostUpload* up, int r) {
  cudaError_t e = cudaSuccess;
  if (r >= 2) e = cudaStreamWaitEvent(bt->copy_stream, bt->ev_free[r % 2], 0);
  for (int q = 0; q < bt->n && e == cudaSuccess; ++q) {
    recon_plan_t p = bt->plans[q];
    const int d0 = r * bt->dbb;
    if (d0 >= p->D) continue;
    const int cnt = (p->D - d0) < bt->dbb ? (p->D - d0) : bt->dbb;
    const size_t img = (size_t)p->nv * p->nu;
    e = cudaMemcpyAsync(up->slots[r % 2] + bt->off_img[q], up->host[q] + (size_t)d0 * img,
                        sizeof(float) * (size_t)cnt * img, cudaMemcpyHostToDevice, bt->copy_stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(bt->ev_ready[r % 2], bt->copy_stream);
  return e;
}

int batch_launch(recon_batch_t bt, const float* const* images, float* const* volumes, char* base, cudaStream_t s,
                 const HostUpload* up = nullptr) {
  cudaError_t e = cudaMemsetAsync(base + bt->off_ctr, 0, sizeof(unsigned long long) * bt->n_rounds, s);
  if (e != cudaSuccess) return cuda_fail(e, "recon_batch: counters");
  for (int q = 0; q < bt->n; ++q) {  // tomograms without directions: clear the volume
    recon_plan_t p = bt->plans[q];
    const size_t nvox = (size_t)p->nx * p->ny * p->nz;
    if (p->D == 0 && nvox > 0 && !p->opt.accumulate) {
      e = cudaMemsetAsync(volumes[q], 0, nvox * sizeof(float), s);
      if (e != cudaSuccess) return cuda_fail(e, "recon_batch: clearing a volume");
    }
  }
  if (up && bt->n_rounds > 0) {
    e = batch_upload_round(bt, up, 0);
    if (e != cudaSuccess) return cuda_fail(e, "recon_batch: image copy");
  }
  for (int r = 0; r < bt->n_rounds; ++r) {
    if (up) {  // the next round's images upload while this round runs
      if (r + 1 < bt->n_rounds) e = batch_upload_round(bt, up, r + 1);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, bt->ev_ready[r % 2], 0);
      if (e != cudaSuccess) return cuda_fail(e, "recon_batch: image copy");
    }
    for (int q = 0; q < bt->n; ++q) {
      recon_plan_t p = bt->plans[q];
      const int d0 = r * bt->dbb;
      if (d0 >= p->D) continue;
      const int cnt = (p->D - d0) < bt->dbb ? (p->D - d0) : bt->dbb;
      // host input: the sub-slot shifted back by d0 images (the kernels index images by
      // absolute direction; only the sub-slot is read)
      const float* img_q =
          up ? (const float*)((uintptr_t)(up->slots[r % 2] + bt->off_img[q]) -
                              (uintptr_t)d0 * p->nv * p->nu * sizeof(float))
             : images[q];
      recon::Workspace w = carve(p, base + bt->off_tables[q]);
      w.S = (float2*)(base + bt->off_S);
      w.T = (float2*)(base + bt->off_T);
      w.stack = base + bt->off_stack[q];
      w.eps = (float*)(base + bt->off_eps);
      MlpHookCtx hctx{p, base + bt->off_tables[q], (float*)(base + bt->off_pow), w.eps, w.S, w.twp};
      const recon::StageAHook hook{mlp_hook, &hctx};
      recon::StageAConst ca = p->ca;
      if (p->P >= 16) ca.sub_block = std::min(bt->dbb, p->ca.sub_block > 0 ? p->ca.sub_block : 1);
      e = recon::launch_stage_a(ca, w, img_q, d0, cnt, s, nullptr,
                                p->ca.filter == RECON_FILTER_MLP ? &hook : nullptr);
      if (e != cudaSuccess) return cuda_fail(e, "recon_batch: stage A launch");
    }
    if (up) {  // this round's stage A has read its slot once this point passes
      e = cudaEventRecord(bt->ev_free[r % 2], s);
      if (e != cudaSuccess) return cuda_fail(e, "recon_batch: slot release");
    }
    e = recon::launch_backproject_persistent((const recon::BatchBp*)(base + bt->off_desc) + (size_t)r * bt->n,
                                             bt->round_count[r], bt->round_total[r],
                                             (unsigned long long*)(base + bt->off_ctr) + r, bt->smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "recon_batch: persistent backprojection launch");
  }
  return RECON_OK;
}

int batch_args(recon_batch_t bt, const float* const* images, float* const* volumes, void* ws, size_t ws_bytes,
               const char* who) {
  if (!bt) return fail(RECON_E_INVALID_ARG, std::string(who) + ": null batch");
  if (bt->n > 0 && (!images || !volumes)) return fail(RECON_E_INVALID_ARG, std::string(who) + ": null arrays");
  for (int q = 0; q < bt->n; ++q) {
    recon_plan_t p = bt->plans[q];
    if ((p->D > 0 && !images[q]) || ((size_t)p->nx * p->ny * p->nz > 0 && !volumes[q]))
      return fail(RECON_E_INVALID_ARG, std::string(who) + ": null image or volume of tomogram " + std::to_string(q));
  }
  if (bt->ws_bytes > 0 && (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < bt->ws_bytes))
    return fail(RECON_E_WORKSPACE, std::string(who) + ": workspace too small or misaligned (needs " +
                                       std::to_string(bt->ws_bytes) + " bytes)");
  return RECON_OK;
}

}  // namespace

extern "C" {

int recon_batch_create(int n, const recon_plan_t* plans, int dir_block, recon_batch_t* out) {
  if (n < 0 || (n > 0 && !plans) || !out) return fail(RECON_E_INVALID_ARG, "recon_batch_create: bad arguments");
  if (dir_block < 0 || dir_block > 1024) return fail(RECON_E_INVALID_ARG, "recon_batch_create: dir_block in [0, 1024]");
  for (int q = 0; q < n; ++q)
    if (!plans[q]) return fail(RECON_E_INVALID_ARG, "recon_batch_create: null plan");
  recon_batch_s* bt = new (std::nothrow) recon_batch_s();
  if (!bt) return fail(RECON_E_NO_MEMORY, "recon_batch_create: out of host memory");
  bt->n = n;
  bt->plans.assign(plans, plans + n);
  bt->dbb = dir_block > 0 ? dir_block : 32;
  size_t off = 0, maxS = 0, maxT = 0, maxpow = 0, maxeps = 0, smem = 0;
  bt->off_tables.resize(n);
  bt->off_stack.resize(n);
  int rounds = 0;
  for (int q = 0; q < n; ++q) {
    recon_plan_t p = plans[q];
    bt->off_tables[q] = off;
    off = align256(off + p->table_bytes);
    const size_t db = (size_t)bt->dbb;
    const size_t sb = std::min(db, (size_t)(p->ca.sub_block > 0 ? p->ca.sub_block : 1));
    maxS = std::max(maxS, sb * p->nv * p->half * 8);
    maxT = std::max(maxT, sb * p->nzl * p->nv * p->half * 8);
    maxpow = std::max(maxpow, sb * p->lc.n_bins * 4);
    maxeps = std::max(maxeps, sb * p->nzl * p->lc.n_bins * 4);
    smem = std::max(smem, db * 64);
    rounds = std::max(rounds, (p->D + bt->dbb - 1) / bt->dbb);
  }
  for (int q = 0; q < n; ++q) {
    bt->off_stack[q] = off;
    off = align256(off + (size_t)bt->dbb * plans[q]->stack_dir_bytes);
  }
  bt->off_S = off;
  off = align256(off + maxS);
  bt->off_T = off;
  off = align256(off + maxT);
  bt->off_pow = off;
  off = align256(off + maxpow);
  bt->off_eps = off;
  off = align256(off + maxeps);
  bt->n_rounds = rounds;
  bt->off_desc = off;
  off = align256(off + sizeof(recon::BatchBp) * (size_t)rounds * n);
  bt->off_ctr = off;
  off = align256(off + sizeof(unsigned long long) * (size_t)(rounds > 0 ? rounds : 1));
  bt->ws_bytes = off;
  bt->smem = smem;
  bt->off_img.resize(n);
  size_t soff = 0;
  for (int q = 0; q < n; ++q) {
    bt->off_img[q] = soff;
    if (plans[q]->D > 0) soff = align256(soff + sizeof(float) * (size_t)bt->dbb * plans[q]->nv * plans[q]->nu);
  }
  bt->slot_bytes = soff;
  bt->desc.assign((size_t)rounds * n, recon::BatchBp{});
  bt->round_count.assign(rounds, 0);
  bt->round_total.assign(rounds, 0);
  *out = bt;
  return RECON_OK;
}

int recon_batch_workspace_size(recon_batch_t bt, size_t* bytes) {
  if (!bt || !bytes) return fail(RECON_E_INVALID_ARG, "recon_batch_workspace_size: null argument");
  *bytes = bt->ws_bytes;
  return RECON_OK;
}

int recon_batch_run(recon_batch_t bt, const float* const* images, float* const* volumes, void* ws, size_t ws_bytes,
                    void* stream) {
  int rc = batch_args(bt, images, volumes, ws, ws_bytes, "recon_batch_run");
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  rc = batch_prepare(bt, images, volumes, (char*)ws, s);
  if (rc) return rc;
  return batch_launch(bt, images, volumes, (char*)ws, s);
}

int recon_batch_run_graph(recon_batch_t bt, const float* const* images, float* const* volumes, void* ws,
                          size_t ws_bytes, void* stream) {
  int rc = batch_args(bt, images, volumes, ws, ws_bytes, "recon_batch_run_graph");
  if (rc) return rc;
  if (!stream) return fail(RECON_E_INVALID_ARG, "recon_batch_run_graph: needs a created (non-default) stream");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<const void*> ptrs;
  ptrs.push_back(ws);
  for (int q = 0; q < bt->n; ++q) {
    ptrs.push_back(images[q]);
    ptrs.push_back(volumes[q]);
  }
  if (!bt->gexec || ptrs != bt->graph_ptrs) {
    if (bt->gexec) {
      cudaGraphExecDestroy(bt->gexec);
      bt->gexec = nullptr;
    }
    if (bt->graph) {
      cudaGraphDestroy(bt->graph);
      bt->graph = nullptr;
    }
    rc = batch_prepare(bt, images, volumes, (char*)ws, s);  // host copies stay outside the graph
    if (rc) return rc;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "recon_batch_run_graph: begin capture");
    rc = batch_launch(bt, images, volumes, (char*)ws, s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "recon_batch_run_graph: end capture");
    e = cudaGraphInstantiate(&bt->gexec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(e, "recon_batch_run_graph: instantiate");
    }
    bt->graph = g;
    bt->graph_ptrs = ptrs;
  }
  cudaError_t e = cudaGraphLaunch(bt->gexec, s);
  if (e != cudaSuccess) return cuda_fail(e, "recon_batch_run_graph: launch");
  return RECON_OK;
}

int recon_batch_run_host_workspace_size(recon_batch_t bt, size_t* bytes) {
  if (!bt || !bytes) return fail(RECON_E_INVALID_ARG, "recon_batch_run_host_workspace_size: null argument");
  *bytes = bt->ws_bytes + 2 * bt->slot_bytes;
  return RECON_OK;
}

int recon_batch_run_host(recon_batch_t bt, const float* const* host_images, float* const* volumes, void* ws,
                         size_t ws_bytes, void* stream) {
  if (!bt) return fail(RECON_E_INVALID_ARG, "recon_batch_run_host: null batch");
  const size_t need = bt->ws_bytes + 2 * bt->slot_bytes;
  if (need > 0 && (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < need))
    return fail(RECON_E_WORKSPACE, "recon_batch_run_host: workspace too small or misaligned (needs " +
                                       std::to_string(need) + " bytes)");
  int rc = batch_args(bt, host_images, volumes, ws, ws_bytes, "recon_batch_run_host");
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "recon_batch_run_host: current device");
  if (bt->copy_dev != dev) {
    bt->release_copy_stream();
    e = cudaStreamCreateWithFlags(&bt->copy_stream, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&bt->ev_start, &bt->ev_ready[0], &bt->ev_ready[1], &bt->ev_free[0], &bt->ev_free[1]})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      bt->release_copy_stream();
      return cuda_fail(e, "recon_batch_run_host: creating the copy stream");
    }
    bt->copy_dev = dev;
  }
  rc = batch_prepare(bt, host_images, volumes, (char*)ws, s);
  if (rc) return rc;
  // the copies overwrite the slots only after everything queued on `stream` before this call
  e = cudaEventRecord(bt->ev_start, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(bt->copy_stream, bt->ev_start, 0);
  if (e != cudaSuccess) return cuda_fail(e, "recon_batch_run_host: ordering the copy stream");
  HostUpload up;
  up.host = host_images;
  up.slots[0] = (char*)ws + bt->ws_bytes;
  up.slots[1] = up.slots[0] + bt->slot_bytes;
  return batch_launch(bt, host_images, volumes, (char*)ws, s, &up);
}

int recon_batch_destroy(recon_batch_t bt) {
  delete bt;
  return RECON_OK;
}

int recon_run_batch_workspace_size(int n, const recon_plan_t* plans, size_t* bytes) {
  recon_batch_t bt = nullptr;
  int rc = recon_batch_create(n, plans, 0, &bt);
  if (rc) return rc;
  rc = recon_batch_workspace_size(bt, bytes);
  recon_batch_destroy(bt);
  return rc;
}

int recon_run_batch(int n, const recon_plan_t* plans, const float* const* images, float* const* volumes,
                    void* workspace, size_t ws_bytes, void* stream) {
  recon_batch_t bt = nullptr;
  int rc = recon_batch_create(n, plans, 0, &bt);
  if (rc) return rc;
  rc = recon_batch_run(bt, images, volumes, workspace, ws_bytes, stream);
  recon_batch_destroy(bt);
  return rc;
}

}  // extern "C"
