// Sampling-matrix construction for the density weighting of arbitrary scans (see
// density.cuh): the trilinear splat of every direction's sub-sampled DFT grid, and the
// band sum that sets the regulariser eps_S.
#include "density.cuh"

namespace recon {
namespace {

__global__ void k_density_splat(const DirParams* __restrict__ dirs, DensityConst dc, int P, float* __restrict__ S) {
  const int n = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n1 = dc.n_samples1;
  if (i >= n1 * n1) return;
  const DirParams& d = dirs[n];
  const float mu = (float)(-P / 2 + (i % n1) * dc.s);
  const float mv = (float)(-P / 2 + (i / n1) * dc.s);
  const float qx = (mu * d.af[0] + mv * d.bf[0]) * dc.inv_s;
  const float qy = (mu * d.af[1] + mv * d.bf[1]) * dc.inv_s;
  const float qz = (mu * d.af[2] + mv * d.bf[2]) * dc.inv_s;
  const float w = 0.5f * (float)(dc.s * dc.s);  // the sample at q and its mirror -q, half weight each
#pragma unroll
  for (int mirror = 0; mirror < 2; ++mirror) {
    const float sx = mirror ? -qx : qx, sy = mirror ? -qy : qy, sz = mirror ? -qz : qz;
    const float bx = floorf(sx), by = floorf(sy), bz = floorf(sz);
    const float fx = sx - bx, fy = sy - by, fz = sz - bz;
    const int ix = (int)bx + dc.Gh, iy = (int)by + dc.Gh, iz = (int)bz + dc.Gh;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const float wt = (dx ? fx : 1.f - fx) * (dy ? fy : 1.f - fy) * (dz ? fz : 1.f - fz);
          atomicAdd(S + ((size_t)(iz + dz) * dc.G + (iy + dy)) * dc.G + (ix + dx), wt * w);
        }
  }
}

__global__ void k_density_band_sum(const float* __restrict__ S, DensityConst dc, double* __restrict__ out) {
  __shared__ double part[32];
  const size_t total = (size_t)dc.G * dc.G * dc.G;
  const int r2max = (dc.Gh - 2) * (dc.Gh - 2);
  double acc = 0.0;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(c % dc.G) - dc.Gh;
    const int y = (int)((c / dc.G) % dc.G) - dc.Gh;
    const int z = (int)(c / ((size_t)dc.G * dc.G)) - dc.Gh;
    if (x * x + y * y + z * z <= r2max) acc += S[c];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) atomicAdd(out, acc);
  }
}

}  // namespace

cudaError_t launch_density_setup(const DensityConst& dc, const DirParams* dirs, int n_dir, int P, float* S,
                                 double* band_sum, cudaStream_t stream) {
  const size_t cells = (size_t)dc.G * dc.G * dc.G;
  cudaError_t e = cudaMemsetAsync(S, 0, cells * sizeof(float), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(band_sum, 0, sizeof(double), stream);
  if (e != cudaSuccess) return e;
  if (n_dir > 0) {
    const int n = dc.n_samples1 * dc.n_samples1;
    k_density_splat<<<dim3((n + 255) / 256, n_dir), 256, 0, stream>>>(dirs, dc, P, S);
  }
  k_density_band_sum<<<device_sm_count() * 4, 256, 0, stream>>>(S, dc, band_sum);
  return cudaGetLastError();
}

}  // namespace recon
