// Stage A of the layered UTR path: contrast -> 2D DFT -> per-layer CTF inverse and
// ramp -> inverse 2D DFT -> cropped layer stack (Sec. 2, Eq. 4, 7, 11; ramp of Sec. 2).
//
// Three kernels per block of directions, all shared-memory radix-2 FFTs of length P:
//   k_rows_fwd  two image rows per CTA packed as one complex row (real + i real),
//               forward FFT, split into the two half spectra      -> S[n][v][0..P/2]
//   k_cols      CB adjacent spectrum columns per CTA: forward FFT along v (rows >= nv
//               are the zero padding), kept in shared memory; then for every layer k:
//               multiply by H_k(q) W(q_u), inverse FFT along v, keep v < nv
//                                                                 -> T[n][k][v][0..P/2]
//   k_rows_inv  two rows of one layer per CTA: Hermitian-extend both half spectra,
//               pack as real + i real, inverse FFT, crop u < nu   -> stack (zero border)
// The image sits at offset 0 of the P x P frame; by the shift invariance of the
// circular filters this equals any other placement with the same crop.
#include <cuda_bf16.h>

#include "recon_internal.h"

namespace recon {
namespace {

constexpr int kColsPerCta = 4;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ int bitrev(int i, int logP) { return (int)(__brev((unsigned)i) >> (32 - logP)); }

// In-place radix-2 decimation-in-time FFT of `ntr` transforms of length P held at
// data + t * ld, input in bit-reversed order, output in natural order.  tw[j] =
// exp(-2 pi i j / P); INV uses the conjugate twiddles (no 1/P scaling).
template <bool INV>
__device__ void fft_radix2(float2* data, int ld, int ntr, int P, int logP, const float2* tw) {
  const int halfP = P >> 1;
  const int total = ntr * halfP;
  for (int s = 0; s < logP; ++s) {
    const int half = 1 << s;
    const int tw_shift = logP - 1 - s;
    __syncthreads();
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int t = idx >> (logP - 1);
      const int j = idx & (halfP - 1);
      const int pos = j & (half - 1);
      const int i1 = ((j - pos) << 1) + pos;
      float2* d = data + t * ld;
      float2 w = tw[pos << tw_shift];
      if (INV) w.y = -w.y;
      const float2 a = d[i1];
      const float2 wb = cmul(w, d[i1 + half]);
      d[i1] = make_float2(a.x + wb.x, a.y + wb.y);
      d[i1 + half] = make_float2(a.x - wb.x, a.y - wb.y);
    }
  }
  __syncthreads();
}

__device__ __forceinline__ float contrast_of(float x, int input_mode) {
  // RECON_INPUT_INTENSITY: g = ln(I/I_in), floored at 1e-6 (left side of Eq. 4)
  return input_mode == 0 ? logf(fmaxf(x, 1e-6f)) : x;
}

__global__ void k_rows_fwd(const float* __restrict__ images, float2* __restrict__ S, const float2* __restrict__ twg,
                           StageAConst c, int dir_begin) {
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* z = sm + (c.P >> 1);
  const int n = blockIdx.y;
  const int v0 = blockIdx.x * 2;
  const bool two = v0 + 1 < c.nv;
  const float* im = images + (size_t)(dir_begin + n) * c.nu * c.nv;
  for (int i = threadIdx.x; i < (c.P >> 1); i += blockDim.x) tw[i] = twg[i];
  for (int i = threadIdx.x; i < c.P; i += blockDim.x) {
    float x1 = 0.f, x2 = 0.f;
    if (i < c.nu) {
      x1 = contrast_of(im[(size_t)v0 * c.nu + i], c.input_mode);
      if (two) x2 = contrast_of(im[(size_t)(v0 + 1) * c.nu + i], c.input_mode);
    }
    z[bitrev(i, c.logP)] = make_float2(x1, x2);
  }
  fft_radix2<false>(z, c.P, 1, c.P, c.logP, tw);
  float2* s1 = S + ((size_t)n * c.nv + v0) * c.half;
  for (int m = threadIdx.x; m < c.half; m += blockDim.x) {
    const float2 zm = z[m & (c.P - 1)];
    const float2 zc = z[(c.P - m) & (c.P - 1)];
    // X1 = (Z[m] + conj Z[P-m]) / 2,  X2 = (Z[m] - conj Z[P-m]) / (2i)
    s1[m] = make_float2(0.5f * (zm.x + zc.x), 0.5f * (zm.y - zc.y));
    if (two) s1[c.half + m] = make_float2(0.5f * (zm.y + zc.y), -0.5f * (zm.x - zc.x));
  }
}

// sin(chi_k) for the integer squared frequency msq = m_u^2 + m_v^2.  chi/(2 pi) is
// accumulated modulo 1 in 64-bit fixed point (exact modular products), so the range
// reduction of chi (hundreds of radians at the band edge) loses nothing; the top 32
// bits give chi in (-pi, pi] to 2^-31 turns before the FP32 sine.
__device__ __forceinline__ float sin_chi(uint64_t uA, uint64_t uC, uint64_t uW, uint32_t msq) {
  const uint64_t m = msq;
  const uint64_t x = uA * m + uC * (m * m) - uW;
  const int32_t hi = (int32_t)(x >> 32);
  return sinpif((float)hi * 4.656612873077393e-10f);  // hi * 2^-31 = chi / pi in [-1, 1)
}

__global__ void k_cols(const float2* __restrict__ S, float2* __restrict__ T, const float2* __restrict__ twg,
                       const uint64_t* __restrict__ uA, const float* __restrict__ ramp, StageAConst c,
                       int dir_begin) {
  extern __shared__ float2 sm[];
  const int ld = c.P + 1;  // one-element skew between the columns' transforms
  float2* tw = sm;
  float2* G = tw + (c.P >> 1);
  float2* Wk = G + kColsPerCta * ld;
  const int n = blockIdx.y;
  const int c0 = blockIdx.x * kColsPerCta;
  for (int i = threadIdx.x; i < (c.P >> 1); i += blockDim.x) tw[i] = twg[i];
  const float2* Sn = S + (size_t)n * c.nv * c.half;
  for (int idx = threadIdx.x; idx < kColsPerCta * c.P; idx += blockDim.x) {
    const int t = idx % kColsPerCta;
    const int v = idx / kColsPerCta;
    const int col = c0 + t;
    float2 val = make_float2(0.f, 0.f);
    if (v < c.nv && col < c.half) val = Sn[(size_t)v * c.half + col];
    G[t * ld + bitrev(v, c.logP)] = val;
  }
  fft_radix2<false>(G, ld, kColsPerCta, c.P, c.logP, tw);
  const uint64_t* uAn = uA + (size_t)(dir_begin + n) * c.nz_layers;
  for (int k = 0; k < c.nz_layers; ++k) {
    const uint64_t uAk = uAn[k];
    for (int idx = threadIdx.x; idx < kColsPerCta * c.P; idx += blockDim.x) {
      const int t = idx / c.P;
      const int m = idx - t * c.P;
      const int col = min(c0 + t, c.half - 1);
      const int mv = m < (c.P >> 1) ? m : m - c.P;
      float f = ramp[col];
      if (c.filter) {
        const float s = sin_chi(uAk, c.uC, c.uW, (uint32_t)(col * col + mv * mv));
        f *= c.pref * s / fmaf(s, s, c.eps);  // real part of the Eq. 11 bracket
      }
      const float2 g = G[t * ld + m];
      Wk[t * ld + bitrev(m, c.logP)] = make_float2(g.x * f, g.y * f);
    }
    fft_radix2<true>(Wk, ld, kColsPerCta, c.P, c.logP, tw);
    float2* Tk = T + ((size_t)n * c.nz_layers + k) * c.nv * c.half;
    for (int idx = threadIdx.x; idx < kColsPerCta * c.nv; idx += blockDim.x) {
      const int t = idx % kColsPerCta;
      const int v = idx / kColsPerCta;
      if (c0 + t < c.half) Tk[(size_t)v * c.half + c0 + t] = Wk[t * ld + v];
    }
    __syncthreads();
  }
}

template <typename OutT>
__device__ __forceinline__ OutT to_stack(float x);
template <>
__device__ __forceinline__ float to_stack<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_stack<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

template <typename OutT>
__global__ void k_rows_inv(const float2* __restrict__ T, OutT* __restrict__ stack, const float2* __restrict__ twg,
                           StageAConst c) {
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* z = sm + (c.P >> 1);
  const int n = blockIdx.z;
  const int k = blockIdx.y;
  const int v0 = blockIdx.x * 2;
  const bool two = v0 + 1 < c.nv;
  for (int i = threadIdx.x; i < (c.P >> 1); i += blockDim.x) tw[i] = twg[i];
  const float2* X1 = T + (((size_t)n * c.nz_layers + k) * c.nv + v0) * c.half;
  const float2* X2 = X1 + c.half;
  const int hP = c.P >> 1;
  for (int m = threadIdx.x; m < c.P; m += blockDim.x) {
    float2 a, b;
    if (m <= hP) {
      a = X1[m];
      b = two ? X2[m] : make_float2(0.f, 0.f);
      if (m == 0 || m == hP) {  // C2R: DC and Nyquist bins are real
        a.y = 0.f;
        b.y = 0.f;
      }
    } else {  // Hermitian extension X[m] = conj X[P - m]
      a = X1[c.P - m];
      a.y = -a.y;
      b = two ? X2[c.P - m] : make_float2(0.f, 0.f);
      b.y = -b.y;
    }
    z[bitrev(m, c.logP)] = make_float2(a.x - b.y, a.y + b.x);  // a + i b
  }
  fft_radix2<true>(z, c.P, 1, c.P, c.logP, tw);
  OutT* L = stack + ((size_t)n * c.nz_layers + k) * c.layer_elems;
  const int su = c.su;
  for (int u = (int)threadIdx.x - 1; u <= c.nu; u += blockDim.x) {
    const bool in = u >= 0 && u < c.nu;
    const float2 zu = in ? z[u] : make_float2(0.f, 0.f);
    L[(size_t)(v0 + 1) * su + (u + 1)] = to_stack<OutT>(zu.x);
    if (two) L[(size_t)(v0 + 2) * su + (u + 1)] = to_stack<OutT>(zu.y);
    if (v0 == 0) L[u + 1] = to_stack<OutT>(0.f);                                    // top border row
    if (v0 + 2 >= c.nv) L[(size_t)(c.nv + 1) * su + (u + 1)] = to_stack<OutT>(0.f);  // bottom border row
  }
}

int threads_for(int P) {
  int t = P >> 1;
  if (t < 64) t = 64;
  if (t > 512) t = 512;
  return t;
}

}  // namespace

cudaError_t launch_stage_a(const StageAConst& c, const Workspace& ws, const float* images, int dir_begin,
                           int dir_count, cudaStream_t stream, cudaEvent_t* ev) {
  if (dir_count <= 0) return cudaSuccess;
  const int thr = threads_for(c.P);
  {
    dim3 grid((c.nv + 1) / 2, dir_count);
    size_t smem = (size_t)(c.P / 2 + c.P) * sizeof(float2);
    k_rows_fwd<<<grid, thr, smem, stream>>>(images, ws.S, ws.tw, c, dir_begin);
    if (ev) cudaEventRecord(ev[0], stream);
  }
  {
    dim3 grid((c.half + kColsPerCta - 1) / kColsPerCta, dir_count);
    size_t smem = (size_t)(c.P / 2 + 2 * kColsPerCta * (c.P + 1)) * sizeof(float2);
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    k_cols<<<grid, 256, smem, stream>>>(ws.S, ws.T, ws.tw, ws.uA, ws.ramp, c, dir_begin);
    if (ev) cudaEventRecord(ev[1], stream);
  }
  {
    dim3 grid((c.nv + 1) / 2, c.nz_layers, dir_count);
    size_t smem = (size_t)(c.P / 2 + c.P) * sizeof(float2);
    if (c.stack_bf16)
      k_rows_inv<__nv_bfloat16><<<grid, thr, smem, stream>>>(ws.T, (__nv_bfloat16*)ws.stack, ws.tw, c);
    else
      k_rows_inv<float><<<grid, thr, smem, stream>>>(ws.T, (float*)ws.stack, ws.tw, c);
  }
  return cudaGetLastError();
}

}  // namespace recon
