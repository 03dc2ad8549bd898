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
//   (sqrt(1 + lambda^2 q^2) + 1)); chi reaches hundreds of radians, so its exact part is
//   taken modulo one turn in 64-bit fixed point and only a small correction in FP32.
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

#include <algorithm>
#include <cmath>

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

// Constants of the phase pass (host-built in FP64 per call).  With power-of-two grid sides,
// K = sum_a (Pmax / P3_a)^2 m_a^2 is an integer and q^2 = K / (Pmax Delta)^2, so the phase in
// turns, chi / (2 pi) = (lambda R / 2) q_perp^2 + (Cs lambda^3 / 4) q_perp^4 - omega / (2 pi),
// splits into an exact part, uR K + uC K^2 - uW in 64-bit fixed point (2^-64 turns, modulo
// 1; uR, uC, uW the fractional parts of the per-unit constants) with q_perp^2 replaced by
// q^2, and the Ewald correction q_perp^2 = q^2 c(x), c = 2 / (1 + sqrt(1 + x)), x =
// lambda^2 q^2: (lambda R / 2) q^2 (c - 1) + (Cs lambda^3 / 4) q^4 (c^2 - 1), a fraction of a
// turn, in FP32.
struct SwapPhaseConst {
  uint64_t uR, uC, uW;
  float kx;          // x per unit K
  float uRf, uCf;    // lambda R / (2 (Pmax Delta)^2) and Cs lambda^3 / (4 (Pmax Delta)^4), turns
  float pref, eps;   // lambda / (4 pi sqrt(1 + sigma^2)), the Tikhonov eps
  int lx, ly;        // log2 of P3[0], P3[1]
  int sx, sy, sz;    // (Pmax / P3_a)^2
};

__global__ void k_swap_phase(const float2* __restrict__ Z, float2* __restrict__ out, Fourier3Const f,
                             SwapPhaseConst k) {
  const long long nb = (long long)f.P3[0] * f.P3[1] * f.P3[2];
  const int mx = f.P3[0] - 1, my = f.P3[1] - 1, mz = f.P3[2] - 1;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i & mx), iy = (int)((i >> k.lx) & my), iz = (int)(i >> (k.lx + k.ly));
    const int jx = (f.P3[0] - ix) & mx, jy = (f.P3[1] - iy) & my, jz = (f.P3[2] - iz) & mz;
    const float2 a = Z[i];
    const float2 b = Z[(((long long)jz << k.ly) + jy << k.lx) + jx];  // Z(-q); conj is (b.x, -b.y)
    // V_c = (a + conj b) / 2, V_s = (a - conj b) / (2 i)
    const float vcr = 0.5f * (a.x + b.x), vci = 0.5f * (a.y - b.y);
    const float vsr = 0.5f * (a.y + b.y), vsi = -0.5f * (a.x - b.x);
    const int ux = signed_bin(ix, f.P3[0]), uy = signed_bin(iy, f.P3[1]), uz = signed_bin(iz, f.P3[2]);
    const uint64_t K = (uint64_t)k.sx * (uint64_t)(ux * ux) + (uint64_t)k.sy * (uint64_t)(uy * uy) +
                       (uint64_t)k.sz * (uint64_t)(uz * uz);
    const uint64_t ph = k.uR * K + k.uC * (K * K) - k.uW;  // modulo 2^64 = modulo one turn
    const float Kf = (float)K;
    const float x = k.kx * Kf;
    const float r = 1.f + sqrtf(1.f + x);
    const float cm1 = -x / (r * r);  // c - 1
    const float corr = k.uRf * Kf * cm1 + k.uCf * Kf * Kf * (cm1 * (cm1 + 2.f));  // turns
    const int32_t h = (int32_t)(uint32_t)(ph >> 32) + __float2int_rn((corr - rintf(corr)) * 4294967296.0f);
    float sn, cn;
    __sincosf((float)h * 1.4629180792671596e-09f, &sn, &cn);  // h * 2 pi / 2^32
    const float sp = k.pref * __fdividef(sn, fmaf(sn, sn, k.eps));
    const float cp = k.pref * __fdividef(cn, fmaf(cn, cn, k.eps));
    out[i] = make_float2(sp * vcr - cp * vsr, sp * vci - cp * vsi);
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

// Sum and count of the non-zero cells of S: per thread in FP32 over its strided cells, then
// in FP64 across the warp and the grid.
__global__ void k_grid_stats(const float* __restrict__ S, long long n, double* __restrict__ stats) {
  float sum = 0.f;
  unsigned int cnt = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float s = S[i];
    if (s > 0.f) {
      sum += s;
      ++cnt;
    }
  }
  double ds = sum, dc = (double)cnt;
  for (int o = 16; o > 0; o >>= 1) {
    ds += __shfl_down_sync(0xffffffffu, ds, o);
    dc += __shfl_down_sync(0xffffffffu, dc, o);
  }
  if ((threadIdx.x & 31) == 0 && dc > 0.0) {
    atomicAdd(&stats[0], ds);
    atomicAdd(&stats[1], dc);
  }
}

__global__ void k_grid_finish(float2* __restrict__ acc, const float2* __restrict__ raw, const float* __restrict__ S,
                              const double* __restrict__ stats, Fourier3Const f, float nsr_m, int lx, int ly,
                              int Pmax) {
  const long long nb = (long long)f.P3[0] * f.P3[1] * f.P3[2];
  const float eps_s = stats[1] > 0.0 ? (float)(1e-3 * stats[0] / stats[1]) : 1.f;
  const float inv_delta = (float)(1.0 / f.delta);
  const int mx = f.P3[0] - 1, my = f.P3[1] - 1;
  // centre offsets c_a = off_a + (n_a - 1) / 2 as 2 c_a, and Pmax / P3_a
  const int c2[3] = {2 * f.off[0] + f.n[0] - 1, 2 * f.off[1] + f.n[1] - 1, 2 * f.off[2] + f.n[2] - 1};
  const int sc[3] = {Pmax / f.P3[0], Pmax / f.P3[1], Pmax / f.P3[2]};
  const float inv_pmax = 1.f / (float)Pmax;  // a power of two: exact
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i & mx), iy = (int)((i >> lx) & my), iz = (int)(i >> (lx + ly));
    const float s = S[i];
    const float inv = 1.f / (s + eps_s);
    float2 F = make_float2(acc[i].x * inv, acc[i].y * inv);
    if (nsr_m > 0.f) {
      const float2 r = raw[i];
      const bool keep = s > 0.f && sqrtf(r.x * r.x + r.y * r.y) * inv >= nsr_m * rsqrtf(fmaxf(s, 1e-30f));
      if (!keep) F = make_float2(0.f, 0.f);
    }
    // exp(-2 pi i sum_a m_a c_a / P3_a): the turns are T / (2 Pmax), T = sum_a m_a (2 c_a)
    // (Pmax / P3_a) an exact integer, reduced modulo 2 Pmax (a power of two)
    const int T = (signed_bin(ix, f.P3[0]) * c2[0] * sc[0] + signed_bin(iy, f.P3[1]) * c2[1] * sc[1] +
                   signed_bin(iz, f.P3[2]) * c2[2] * sc[2]) & (2 * Pmax - 1);
    float ps, pc;
    sincospif(-(float)T * inv_pmax, &ps, &pc);
    acc[i] = make_float2((F.x * pc - F.y * ps) * inv_delta, (F.x * ps + F.y * pc) * inv_delta);
  }
}

// frac(t) in 2^-64 turns (t >= 0)
uint64_t turns_fixed(double t) {
  double fr = t - std::floor(t);
  if (!(fr < 1.0)) fr = 0.0;
  const double scaled = std::ldexp(fr, 64);
  return scaled >= 18446744073709551616.0 ? 0 : (uint64_t)scaled;
}

int log2_int(int p) {
  int l = 0;
  while ((1 << l) < p) ++l;
  return l;
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
  SwapPhaseConst k;
  const int Pmax = std::max(f.P3[0], std::max(f.P3[1], f.P3[2]));
  const double pd2 = (double)Pmax * f.delta * (double)Pmax * f.delta;  // (Pmax Delta)^2
  const double cR = f.lam * R / (2.0 * pd2);                            // turns per unit K
  const double cC = cs * f.lam * f.lam * f.lam / (4.0 * pd2 * pd2);     // turns per unit K^2
  const double cW = std::atan(sigma) / (2.0 * 3.14159265358979323846);
  k.uR = turns_fixed(cR);
  k.uC = turns_fixed(cC);
  k.uW = turns_fixed(cW);
  k.kx = (float)(f.lam * f.lam / pd2);
  k.uRf = (float)cR;
  k.uCf = (float)cC;
  k.pref = (float)(f.lam / (4.0 * 3.14159265358979323846 * std::sqrt(1.0 + sigma * sigma)));
  k.eps = (float)eps;
  k.lx = log2_int(f.P3[0]);
  k.ly = log2_int(f.P3[1]);
  k.sx = (Pmax / f.P3[0]) * (Pmax / f.P3[0]);
  k.sy = (Pmax / f.P3[1]) * (Pmax / f.P3[1]);
  k.sz = (Pmax / f.P3[2]) * (Pmax / f.P3[2]);
  k_swap_phase<<<grid_blocks((long long)f.P3[0] * f.P3[1] * f.P3[2]), 256, 0, s>>>(Z, out, f, k);
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
  const int Pmax = std::max(f.P3[0], std::max(f.P3[1], f.P3[2]));
  k_grid_finish<<<grid_blocks(nb), 256, 0, s>>>(acc, raw, S, stats, f, nsr_m, log2_int(f.P3[0]), log2_int(f.P3[1]),
                                                Pmax);
  return cudaGetLastError();
}

}  // namespace recon
