// Learned regulariser of the CTF inverse (see learned.cu): constants and launchers.
#pragma once

#include <cuda_runtime.h>

#include "recon_internal.h"

namespace recon {

constexpr int kMlpHidden = 64;
constexpr int kMlpParams = 3 * kMlpHidden + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden + kMlpHidden + 1;
constexpr int kActStride = 3 + 2 * kMlpHidden + 1;  // x, a1, a2, o per row
constexpr int kMaxBins = 128;

// Bin of frequency (m_u, m_v): min(isqrt(m_u^2 + m_v^2) / bin_width, n_bins - 1),
// bin_width = max(1, P / 128), n_bins = isqrt(P^2 / 2) / bin_width + 1 (<= 92).
struct LearnConst {
  int n_bins, bin_width;
  float inv_half_p;   // 2 / P
  float noise_floor;  // nsr^2 * nu * nv: Poisson power per DFT coefficient (Parseval)
  float eps_scale;    // 1 / (views averaged per voxel): the network's per-view eps divided (1 in training)
};

cudaError_t launch_cols_forward(const StageAConst& c, const LearnConst& lc, const float2* S, float2* G_out,
                                float* pow, const float2* twp, int n_dirs, cudaStream_t s);
cudaError_t launch_eps_table(const LearnConst& lc, const float* pow, const float* cnt, const float* x2tab,
                             const float* theta, float* eps, float* acts, int n_dirs, int n_layers, int dir_begin,
                             cudaStream_t s);
cudaError_t launch_train_step(const StageAConst& c, const LearnConst& lc, const float2* G, const float2* T,
                              const float* eps, const uint64_t* uA, const float* acts, const float* theta_dev,
                              float* theta_upd, float* grad, float* m1, float* m2, int n_img, double* sums,
                              double* deps, int step, float lr, float* loss_out, cudaStream_t s);

}  // namespace recon
