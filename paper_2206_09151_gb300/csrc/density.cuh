// Sampling-density weighting of an arbitrary scan (Sec. 2: the regularised inverse
// S_eps^-1 of the sampling matrix replaces the 1/n_q of Eq. 11).  S lives on a
// (2 Gh + 1)^3 grid of cells of s DFT bins; every image's DFT samples, taken every s bins
// with weight s^2, are spread trilinearly at +-(m_u u_n + m_v v_n) (half weight each, so
// that S and the weight are even in q; u_n, v_n: rows 0 and 1 of Rot_n).  The weight of frequency (m_u, m_v) of direction n is
//   W = g / (S(m_u u_n + m_v v_n) + eps_S),  g = s^3 / (P delta),
// with S interpolated trilinearly and eps_S = 1e-3 x the mean of S over the band
// (cells within Gh - 2 of the centre).  A 180-degree single-axis scan gives pi |q_u| / D.
#pragma once

#include <cuda_runtime.h>

#include "recon_internal.h"

namespace recon {

#ifdef __CUDACC__
// W(m_u, m_v) / P^2 for the direction with detector axes (u, v) (FP32 rows of Rot_n).
__device__ __forceinline__ float density_weight(const DensityConst& dc, const float* __restrict__ S,
                                                const double* __restrict__ band_sum, const float* u,
                                                const float* v, float mu, float mv) {
  const float qx = (mu * u[0] + mv * v[0]) * dc.inv_s;
  const float qy = (mu * u[1] + mv * v[1]) * dc.inv_s;
  const float qz = (mu * u[2] + mv * v[2]) * dc.inv_s;
  const float bx = floorf(qx), by = floorf(qy), bz = floorf(qz);
  const float fx = qx - bx, fy = qy - by, fz = qz - bz;
  const int ix = (int)bx + dc.Gh, iy = (int)by + dc.Gh, iz = (int)bz + dc.Gh;
  const float* c0 = S + ((size_t)iz * dc.G + iy) * dc.G + ix;
  const float* c1 = c0 + (size_t)dc.G * dc.G;
  const float s00 = fmaf(fx, __ldg(c0 + 1) - __ldg(c0), __ldg(c0));
  const float s01 = fmaf(fx, __ldg(c0 + dc.G + 1) - __ldg(c0 + dc.G), __ldg(c0 + dc.G));
  const float s10 = fmaf(fx, __ldg(c1 + 1) - __ldg(c1), __ldg(c1));
  const float s11 = fmaf(fx, __ldg(c1 + dc.G + 1) - __ldg(c1 + dc.G), __ldg(c1 + dc.G));
  const float s0 = fmaf(fy, s01 - s00, s00), s1 = fmaf(fy, s11 - s10, s10);
  const float Sq = fmaf(fz, s1 - s0, s0);
  const float eps_s = (float)(*band_sum) * dc.eps_scale;
  return dc.g_over_p2 / (Sq + eps_s);
}
#endif

// Builds S and its band sum in the workspace (S: G^3 floats, band_sum: one double).
cudaError_t launch_density_setup(const DensityConst& dc, const DirParams* dirs, int n_dir, int P, float* S,
                                 double* band_sum, cudaStream_t stream);

}  // namespace recon
