// The method's two 3D-Fourier-space forms, beside the layered real-space path:
//
// Eq. 12 (one defocus R for every view): the CT step -- the layered reconstruction of the
// contrasts with the Ewald placement and no CTF bracket, as two real volumes V_c, V_s
// (per-layer cos and sin of pi lambda z_k q^2, run by the stage-A kernels) -- is packed as
// V_c + i V_s into a zero-padded grid and transformed once; the CTF inversion is then one
// pass over that spectrum:
//   F3 delta(q) = lambda / (4 pi sqrt(1+sigma^2)) [s'(q) V_c^(q) - c'(q) V_s^(q)],
//   V_c^(q) = (Z(q) + conj Z(-q)) / 2,  V_s^(q) = (Z(q) - conj Z(-q)) / (2 i),
//   s' = sin chi / (sin^2 chi + eps), c' = cos chi / (cos^2 chi + eps), chi at the
//   in-plane frequency q_perp of the Ewald-paraboloid point q (q_perp^2 = 2 q^2 /
//   (sqrt(1 + lambda^2 q^2) + 1)), computed in FP64 (chi reaches hundreds of radians).
// The spectrum of the CT step stays in the workspace, so other (sigma, eps) rerun only the
// phase pass and the inverse transform.
//
// The Fourier-gridding UTR (Sec. 2 after Eq. 11): every 2D DFT coefficient of every view,
// taken about the detector centre and multiplied by the bracket of Eq. 11 at its own R_n
// (fixed-point phase, as in stage A), is spread with trilinear weights over the 8 cells
// around its point Rot_n^T (q_u, q_v, -lambda q^2 / 2) of the padded volume's DFT grid
// (float atomics); S sums the weights.  Then F = acc / (S + eps_S), eps_S = 1e-3 x the
// mean of S over its non-zero cells; with the noise filter of Sec. 3, F = 0 where the
// gridded contrast (the same splat without the bracket) over S + eps_S is below
// NSR M / sqrt(S).  The phase back to the grid origin and 1/Delta are applied before the
// inverse transform.
#include <cuda_runtime.h>

#include "recon_internal.h"

namespace recon {
namespace {

__device__ __forceinline__ int signed_bin(int m, int P) { return m < P / 2 ? m : m - P; }

__global__ void k_swap_pack(const float* __restrict__ vc, const float* __restrict__ vs, float2* __restrict__ grid,
                            Fourier3Const f) {
  const long long nvox = (long long)f.n[0] * f.n[1] * f.n[2];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nvox;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % f.n[0]), y = (int)((i / f.n[0]) % f.n[1]), z = (int)(i / ((long long)f.n[0] * f.n[1]));
    const long long g = ((long long)(z + f.off[2]) * f.P3[1] + (y + f.off[1])) * f.P3[0] + (x + f.off[0]);
    grid[g] = make_float2(vc[i], vs[i]);
  }
}

__global__ void k_swap_phase(const float2* __restrict__ Z, float2* __restrict__ out, Fourier3Const f, double R,
                             double sigma, double eps, double cs) {
  const long long nb = (long long)f.P3[0] * f.P3[1] * f.P3[2];
  const double pref = f.lam / (4.0 * 3.14159265358979323846 * sqrt(1.0 + sigma * sigma));
  const double omega = atan(sigma);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % f.P3[0]), iy = (int)((i / f.P3[0]) % f.P3[1]), iz = (int)(i / ((long long)f.P3[0] * f.P3[1]));
    const int jx = (f.P3[0] - ix) & (f.P3[0] - 1), jy = (f.P3[1] - iy) & (f.P3[1] - 1), jz = (f.P3[2] - iz) & (f.P3[2] - 1);
    const float2 a = Z[i];
    const float2 b = Z[((long long)jz * f.P3[1] + jy) * f.P3[0] + jx];  // Z(-q); conj is (b.x, -b.y)
    // V_c = (a + conj b) / 2, V_s = (a - conj b) / (2 i)
    const double vcr = 0.5 * ((double)a.x + b.x), vci = 0.5 * ((double)a.y - b.y);
    const double vsr = 0.5 * ((double)a.y + b.y), vsi = -0.5 * ((double)a.x - b.x);
    const double qx = signed_bin(ix, f.P3[0]) / (f.P3[0] * f.delta);
    const double qy = signed_bin(iy, f.P3[1]) / (f.P3[1] * f.delta);
    const double qz = signed_bin(iz, f.P3[2]) / (f.P3[2] * f.delta);
    const double q2 = qx * qx + qy * qy + qz * qz;
    const double qp2 = 2.0 * q2 / (sqrt(1.0 + f.lam * f.lam * q2) + 1.0);
    const double chi = 3.14159265358979323846 * f.lam * R * qp2 +
                       0.5 * 3.14159265358979323846 * cs * f.lam * f.lam * f.lam * qp2 * qp2 - omega;
    double sn, cn;
    sincos(chi, &sn, &cn);
    const double sp = pref * sn / (sn * sn + eps), cp = pref * cn / (cn * cn + eps);
    out[i] = make_float2((float)(sp * vcr - cp * vsr), (float)(sp * vci - cp * vsi));
  }
}

__global__ void k_crop_real(const float2* __restrict__ grid, float* __restrict__ vol, Fourier3Const f, float scale) {
  const long long nvox = (long long)f.n[0] * f.n[1] * f.n[2];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nvox;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % f.n[0]), y = (int)((i / f.n[0]) % f.n[1]), z = (int)(i / ((long long)f.n[0] * f.n[1]));
    const long long g = ((long long)(z + f.off[2]) * f.P3[1] + (y + f.off[1])) * f.P3[0] + (x + f.off[0]);
    vol[i] = grid[g].x * scale;
  }
}

// ------------------------------------------------------------------ gridding
__device__ __forceinline__ void splat(float2* acc, float2* raw, float* S, const Fourier3Const& f, const float g[3],
                                      float2 z, float2 gc, bool with_raw) {
  int b[3];
  float fr[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float fl = floorf(g[a]);
    b[a] = (int)fl;
    fr[a] = g[a] - fl;
  }
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const float w = (dx ? fr[0] : 1.f - fr[0]) * (dy ? fr[1] : 1.f - fr[1]) * (dz ? fr[2] : 1.f - fr[2]);
        const int ix = (b[0] + dx) & (f.P3[0] - 1), iy = (b[1] + dy) & (f.P3[1] - 1), iz = (b[2] + dz) & (f.P3[2] - 1);
        const long long c = ((long long)iz * f.P3[1] + iy) * f.P3[0] + ix;
        atomicAdd(&S[c], w);
        atomicAdd(&acc[c].x, w * z.x);
        atomicAdd(&acc[c].y, w * z.y);
        if (with_raw) {
          atomicAdd(&raw[c].x, w * gc.x);
          atomicAdd(&raw[c].y, w * gc.y);
        }
      }
}

// One thread per coefficient (n, col, m_v) of the half spectra G [n][col][P]; columns 1 ..
// P/2 - 1 also stand for their mirrors (-col, -m_v) (conjugate contrast, same bracket).
__global__ void k_grid_splat(const float2* __restrict__ G, const GridDir* __restrict__ dirs, int dir_begin,
                             int n_dirs, StageAConst c, Fourier3Const f, float2* __restrict__ acc,
                             float2* __restrict__ raw, float* __restrict__ S, int with_raw) {
  const int P = c.P, half = c.half;
  const long long total = (long long)n_dirs * half * P;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int mvi = (int)(i % P), col = (int)((i / P) % half), n = (int)(i / ((long long)P * half));
    const GridDir& d = dirs[dir_begin + n];
    const int mu = col == P / 2 ? -P / 2 : col;  // the Nyquist column is bin -P/2 of the full grid
    const int mv = signed_bin(mvi, P);
    const float2 G0 = G[((long long)n * half + col) * P + mvi];
    // about the detector centre: times exp(i pi (mu (nu - 1) + mv (nv - 1)) / P), exact phase
    const long long k = ((long long)mu * (c.nu - 1) + (long long)mv * (c.nv - 1)) % (2LL * P);
    float ps, pc;
    sincospif((float)k / (float)P, &ps, &pc);
    const float2 gc = make_float2(G0.x * pc - G0.y * ps, G0.x * ps + G0.y * pc);
    // Eq. 11's bracket at this view's R_n: chi / (2 pi) in 2^-64 turns, exact modulo 1
    const uint32_t m2 = (uint32_t)(mu * mu + mv * mv);
    const uint64_t m64 = m2;
    const uint32_t hi = (uint32_t)((d.uR * m64 + c.uC * (m64 * m64) - c.uW) >> 32);
    float sn, cn;
    sincospif((float)(int32_t)hi * 4.656612873077393e-10f, &sn, &cn);  // hi * 2^-31 = chi / pi
    const float sp = sn / fmaf(sn, sn, c.eps), cp = cn / fmaf(cn, cn, c.eps);
    // Z = pref G_c (s' - i c')
    const float2 z = make_float2(c.pref * (gc.x * sp + gc.y * cp), c.pref * (gc.y * sp - gc.x * cp));
    // the point (q_u, q_v, -lambda q^2 / 2) in DFT bins of each grid axis
    const float qz = -d.qz_coef * (float)m2;  // in units of 1 / (P delta)
    float g[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) g[a] = ((float)mu * d.r[a] + (float)mv * d.r[3 + a] + qz * d.r[6 + a]) * f.scale[a];
    splat(acc, raw, S, f, g, z, gc, with_raw != 0);
    if (col >= 1 && col < P / 2) {  // the mirror (-mu, -mv): conjugate contrast, same bracket
      // its own bin (-P/2 stays -P/2 on the Nyquist row) and its own centring phase
      const int mvm = mv == -P / 2 ? mv : -mv;
      const long long km = ((long long)(-mu) * (c.nu - 1) + (long long)mvm * (c.nv - 1)) % (2LL * P);
      float qs, qc;
      sincospif((float)km / (float)P, &qs, &qc);
      const float2 gm = make_float2(G0.x * qc + G0.y * qs, G0.x * qs - G0.y * qc);  // conj(G0) e^{i pi km / P}
      const float2 zm = make_float2(c.pref * (gm.x * sp + gm.y * cp), c.pref * (gm.y * sp - gm.x * cp));
      float h[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) h[a] = ((float)(-mu) * d.r[a] + (float)mvm * d.r[3 + a] + qz * d.r[6 + a]) * f.scale[a];
      splat(acc, raw, S, f, h, zm, gm, with_raw != 0);
    }
  }
}

__global__ void k_grid_stats(const float* __restrict__ S, long long n, double* __restrict__ stats) {
  double sum = 0.0, cnt = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float s = S[i];
    if (s > 0.f) {
      sum += s;
      cnt += 1.0;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_down_sync(0xffffffffu, sum, o);
    cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  }
  if ((threadIdx.x & 31) == 0 && cnt > 0.0) {
    atomicAdd(&stats[0], sum);
    atomicAdd(&stats[1], cnt);
  }
}

// F = acc / (S + eps_S) (zero where the noise filter drops it), times the phase back to the
// grid origin and 1 / delta, in place.
__global__ void k_grid_finish(float2* __restrict__ acc, const float2* __restrict__ raw, const float* __restrict__ S,
                              const double* __restrict__ stats, Fourier3Const f, float nsr_m) {
  const long long nb = (long long)f.P3[0] * f.P3[1] * f.P3[2];
  const float eps_s = stats[1] > 0.0 ? (float)(1e-3 * stats[0] / stats[1]) : 1.f;
  const float inv_delta = (float)(1.0 / f.delta);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % f.P3[0]), iy = (int)((i / f.P3[0]) % f.P3[1]), iz = (int)(i / ((long long)f.P3[0] * f.P3[1]));
    const float s = S[i];
    const float inv = 1.f / (s + eps_s);
    float2 F = make_float2(acc[i].x * inv, acc[i].y * inv);
    if (nsr_m > 0.f) {
      const float2 r = raw[i];
      const bool keep = s > 0.f && sqrtf(r.x * r.x + r.y * r.y) * inv >= nsr_m * rsqrtf(fmaxf(s, 1e-30f));
      if (!keep) F = make_float2(0.f, 0.f);
    }
    // exp(-2 pi i sum_a m_a c_a / P3_a), c_a = off_a + (n_a - 1) / 2: turns as an exact sum
    // of fractions with power-of-two denominators (2 P3_a), reduced modulo 1 in FP64
    double t = 0.0;
    const int mm[3] = {signed_bin(ix, f.P3[0]), signed_bin(iy, f.P3[1]), signed_bin(iz, f.P3[2])};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const long long num = ((long long)mm[a] * (2LL * f.off[a] + f.n[a] - 1)) % (2LL * f.P3[a]);
      t += (double)num / (2.0 * f.P3[a]);
    }
    t -= floor(t);
    float ps, pc;
    sincospif(-2.f * (float)t, &ps, &pc);
    acc[i] = make_float2((F.x * pc - F.y * ps) * inv_delta, (F.x * ps + F.y * pc) * inv_delta);
  }
}

unsigned grid_blocks(long long n) {
  const long long cap = (long long)device_sm_count() * 16;
  const long long want = (n + 255) / 256;
  return (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t launch_swap_pack(const float* vc, const float* vs, float2* grid, const Fourier3Const& f, cudaStream_t s) {
  const long long nb = (long long)f.P3[0] * f.P3[1] * f.P3[2];
  cudaError_t e = cudaMemsetAsync(grid, 0, sizeof(float2) * (size_t)nb, s);
  if (e != cudaSuccess) return e;
  k_swap_pack<<<grid_blocks((long long)f.n[0] * f.n[1] * f.n[2]), 256, 0, s>>>(vc, vs, grid, f);
  return cudaGetLastError();
}

cudaError_t launch_swap_phase(const float2* Z, float2* out, const Fourier3Const& f, double R, double sigma, double eps,
                              double cs, cudaStream_t s) {
  k_swap_phase<<<grid_blocks((long long)f.P3[0] * f.P3[1] * f.P3[2]), 256, 0, s>>>(Z, out, f, R, sigma, eps, cs);
  return cudaGetLastError();
}

cudaError_t launch_crop_real(const float2* grid, float* vol, const Fourier3Const& f, cudaStream_t s) {
  const float scale = (float)(1.0 / ((double)f.P3[0] * f.P3[1] * f.P3[2]));
  k_crop_real<<<grid_blocks((long long)f.n[0] * f.n[1] * f.n[2]), 256, 0, s>>>(grid, vol, f, scale);
  return cudaGetLastError();
}

cudaError_t launch_grid_splat(const float2* G, const GridDir* dirs, int dir_begin, int n_dirs, const StageAConst& c,
                              const Fourier3Const& f, float2* acc, float2* raw, float* S, bool with_raw,
                              cudaStream_t s) {
  if (n_dirs <= 0) return cudaSuccess;
  k_grid_splat<<<grid_blocks((long long)n_dirs * c.half * c.P), 256, 0, s>>>(G, dirs, dir_begin, n_dirs, c, f, acc, raw,
                                                                          S, with_raw ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_grid_finish(float2* acc, const float2* raw, const float* S, double* stats, const Fourier3Const& f,
                               float nsr_m, cudaStream_t s) {
  const long long nb = (long long)f.P3[0] * f.P3[1] * f.P3[2];
  cudaError_t e = cudaMemsetAsync(stats, 0, 2 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  k_grid_stats<<<grid_blocks(nb), 256, 0, s>>>(S, nb, stats);
  k_grid_finish<<<grid_blocks(nb), 256, 0, s>>>(acc, raw, S, stats, f, nsr_m);
  return cudaGetLastError();
}

}  // namespace recon
