// In-place 3D FFT of a complex grid [Z][Y][X] (each side a power of two, 1 .. 2048) for the
// two 3D-Fourier forms of the method: Eq. 12's CTF inversion after the CT step, and the
// Fourier-gridding reconstruction (Sec. 2 after Eq. 11).  Three passes of line FFTs, one
// per axis, each line a register-resident Stockham FFT (fft_reg.cuh for lengths 16-512,
// fft16.cuh for 1024-2048; a direct DFT for lengths 2-8).  A CTA takes CB lines: along x
// they are consecutive rows (loaded row by row), along y and z they are neighbours in x
// (loaded CB elements at a time), so the global loads and stores stay coalesced.
#include <cuda_runtime.h>

#include "fft16.cuh"
#include "fft_reg.cuh"
#include "recon_internal.h"

namespace recon {
namespace {

constexpr int kThreads3 = 256;

template <int P>
struct Engine {
  static constexpr bool E16 = P >= 1024;
  static constexpr int T = E16 ? P / 16 : P / 8;  // threads per line
  static constexpr int CB = kThreads3 / T;         // lines per CTA
  static constexpr int L = E16 ? fft16::buffer_len(P) : fft::buffer_len(P, CB);
  static constexpr int NT = E16 ? fft16::table_len(P) : fft::pass_table_len(P);
  __device__ static int idx(int v) { return E16 ? fft16::pad(v) : fft::padded(v); }
};

// Lines: line (o, i) starts at o * outer_stride + i and has element stride es; lines are
// numbered i fastest (2^inner_log2 of them per o: the grid sides are powers of two, so the
// split is a shift and a mask, not a 64-bit division per element).  Along x: one line per o,
// es = 1.
template <int P, bool INV>
__global__ void __launch_bounds__(kThreads3) k_fft3_lines(float2* __restrict__ data, long long n_lines, int inner_log2,
                                                          long long outer_stride, long long es,
                                                          const float2* __restrict__ twg) {
  using E = Engine<P>;
  extern __shared__ float2 smem3[];
  float2* tw = smem3;
  float2* buf_all = smem3 + E::NT;
  const int g = threadIdx.x / E::T, j = threadIdx.x % E::T;
  float2* buf = buf_all + g * E::L;
  for (int i = threadIdx.x; i < E::NT; i += kThreads3) tw[i] = twg[i];
  const long long l0 = (long long)blockIdx.x * E::CB;
  const bool along_x = es == 1;
  // fill: along x row by row (consecutive elements), else CB neighbours in x per element;
  // every load of the thread is issued before the first shared-memory store, so that they
  // are all in flight at once (one at a time left the kernel waiting on DRAM latency)
  constexpr int NQ = E::CB * P / kThreads3;  // elements per thread
  static_assert(NQ * kThreads3 == E::CB * P, "whole lines per CTA");
  float2 val[NQ];
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    const int q = threadIdx.x + k * kThreads3;
    const int t = along_x ? q / P : q % E::CB, v = along_x ? q % P : q / E::CB;
    const long long l = l0 + t;
    val[k] = make_float2(0.f, 0.f);
    if (l < n_lines) {
      const long long o = l >> inner_log2, i = l & ((1LL << inner_log2) - 1);
      val[k] = data[o * outer_stride + i + v * es];
    }
  }
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    const int q = threadIdx.x + k * kThreads3;
    const int t = along_x ? q / P : q % E::CB, v = along_x ? q % P : q / E::CB;
    buf_all[t * E::L + E::idx(v)] = val[k];
  }
  __syncthreads();
  const fft::GroupSync gsync{1 + g, E::T};
  if constexpr (E::E16) {
    float2 x[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) x[s] = buf[E::idx(j + s * E::T)];
    fft16::group_fft_sb<P, INV>(x, buf, tw, j, gsync);
    gsync();
#pragma unroll
    for (int s = 0; s < 16; ++s) buf[E::idx(j + s * E::T)] = x[s];
  } else {
    float2 x[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) x[s] = buf[E::idx(j + s * E::T)];
    fft::block_fft<P, INV>(x, buf, tw, j, gsync);
    gsync();
#pragma unroll
    for (int s = 0; s < 8; ++s) buf[E::idx(j + s * E::T)] = x[s];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    const int q = threadIdx.x + k * kThreads3;
    const int t = along_x ? q / P : q % E::CB, v = along_x ? q % P : q / E::CB;
    val[k] = buf_all[t * E::L + E::idx(v)];
  }
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    const int q = threadIdx.x + k * kThreads3;
    const int t = along_x ? q / P : q % E::CB, v = along_x ? q % P : q / E::CB;
    const long long l = l0 + t;
    if (l < n_lines) {
      const long long o = l >> inner_log2, i = l & ((1LL << inner_log2) - 1);
      data[o * outer_stride + i + v * es] = val[k];
    }
  }
}

// lengths 2, 4, 8: one thread per line, direct DFT
__global__ void k_fft3_small(float2* __restrict__ data, long long n_lines, int n_inner, long long outer_stride,
                             long long es, int P, int inv) {
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_lines) return;
  const long long o = l / n_inner, i = l % n_inner;
  float2* base = data + o * outer_stride + i;
  float2 x[8], y[8];
  for (int v = 0; v < P; ++v) x[v] = base[v * es];
  for (int k = 0; k < P; ++k) {
    float2 acc = make_float2(0.f, 0.f);
    for (int v = 0; v < P; ++v) {
      float sn, cs;
      sincospif((inv ? 2.f : -2.f) * (float)((k * v) % P) / (float)P, &sn, &cs);
      acc.x += x[v].x * cs - x[v].y * sn;
      acc.y += x[v].x * sn + x[v].y * cs;
    }
    y[k] = acc;
  }
  for (int v = 0; v < P; ++v) base[v * es] = y[v];
}

template <int P, bool INV>
cudaError_t lines_p(float2* data, long long n_lines, int n_inner, long long outer_stride, long long es,
                    const float2* tw, cudaStream_t s) {
  using E = Engine<P>;
  const size_t smem = sizeof(float2) * ((size_t)E::NT + (size_t)E::CB * E::L);
  if (smem > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_fft3_lines<P, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const long long ctas = (n_lines + E::CB - 1) / E::CB;
  int inner_log2 = 0;  // n_inner is 1, X or X Y: a power of two
  while ((1LL << inner_log2) < n_inner) ++inner_log2;
  if ((1LL << inner_log2) != n_inner) return cudaErrorInvalidValue;
  k_fft3_lines<P, INV><<<(unsigned)ctas, kThreads3, smem, s>>>(data, n_lines, inner_log2, outer_stride, es, tw);
  return cudaGetLastError();
}

template <bool INV>
cudaError_t lines(int P, float2* data, long long n_lines, int n_inner, long long outer_stride, long long es,
                  const float2* tw, cudaStream_t s) {
  switch (P) {
    case 1: return cudaSuccess;
    case 2: case 4: case 8:
      k_fft3_small<<<(unsigned)((n_lines + 127) / 128), 128, 0, s>>>(data, n_lines, n_inner, outer_stride, es, P,
                                                                     INV ? 1 : 0);
      return cudaGetLastError();
    case 16: return lines_p<16, INV>(data, n_lines, n_inner, outer_stride, es, tw, s);
    case 32: return lines_p<32, INV>(data, n_lines, n_inner, outer_stride, es, tw, s);
    case 64: return lines_p<64, INV>(data, n_lines, n_inner, outer_stride, es, tw, s);
    case 128: return lines_p<128, INV>(data, n_lines, n_inner, outer_stride, es, tw, s);
    case 256: return lines_p<256, INV>(data, n_lines, n_inner, outer_stride, es, tw, s);
    case 512: return lines_p<512, INV>(data, n_lines, n_inner, outer_stride, es, tw, s);
    case 1024: return lines_p<1024, INV>(data, n_lines, n_inner, outer_stride, es, tw, s);
    case 2048: return lines_p<2048, INV>(data, n_lines, n_inner, outer_stride, es, tw, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_fft3(float2* data, const int P3[3], const float2* const tw[3], bool inverse, cudaStream_t s) {
  const long long X = P3[0], Y = P3[1], Z = P3[2];
  cudaError_t e;
  // x lines: Y Z of them, contiguous
  e = inverse ? lines<true>(P3[0], data, Y * Z, 1, X, 1, tw[0], s) : lines<false>(P3[0], data, Y * Z, 1, X, 1, tw[0], s);
  if (e != cudaSuccess) return e;
  // y lines: for every z, X neighbours in x, stride X
  e = inverse ? lines<true>(P3[1], data, X * Z, (int)X, X * Y, X, tw[1], s)
              : lines<false>(P3[1], data, X * Z, (int)X, X * Y, X, tw[1], s);
  if (e != cudaSuccess) return e;
  // z lines: X Y of them, stride X Y
  return inverse ? lines<true>(P3[2], data, X * Y, (int)(X * Y), 0, X * Y, tw[2], s)
                 : lines<false>(P3[2], data, X * Y, (int)(X * Y), 0, X * Y, tw[2], s);
}

}  // namespace recon
