// Stage A of the layered UTR path: contrast -> 2D DFT -> per-layer CTF inverse and
// ramp -> inverse 2D DFT -> cropped layer stack (Sec. 2, Eq. 4, 7, 11; ramp of Sec. 2).
//
// Three kernels per block of directions:
//   k_rows_fwd  two image rows packed as one complex row (real + i real), forward FFT,
//               split into the two half spectra                    -> S[n][v][0..P/2]
//   k_cols      one spectrum column per group of P/8 threads: forward FFT along v (rows
//               >= nv are the zero padding), kept in registers; then for every layer
//               k: multiply by H_k(q) W(q_u), inverse FFT along v, store v < nv
//                                                                   -> T[n][k][col][v]
//   k_rows_inv  two rows of one layer per group: Hermitian-extend both half spectra,
//               pack as real + i real, inverse FFT, crop u < nu    -> stack of tap pairs
// For P >= 16 the FFTs are register-resident mixed-radix Stockham transforms
// (fft_reg.cuh); tiny images (P <= 8) use a shared-memory radix-2 transform.
// The image sits at offset 0 of the P x P frame; by the shift invariance of the
// circular filters this equals any other placement with the same crop.
#include <cuda_bf16.h>

#include <cmath>

#include "density.cuh"
#include "fft16.cuh"
#include "fft_reg.cuh"
#include "recon_internal.h"

namespace recon {
namespace {

using fft::cmul;
using fft::padded;

constexpr int kThreads = 256;

template <int P>
__host__ __device__ constexpr int groups_per_cta() {
  return kThreads / (P / 8) > 0 ? kThreads / (P / 8) : 1;
}

__device__ __forceinline__ float contrast_of(float x, int input_mode) {
  // RECON_INPUT_INTENSITY: g = ln(I/I_in), floored at 1e-6 (left side of Eq. 4)
  return input_mode == 0 ? logf(fmaxf(x, 1e-6f)) : x;
}

// sin(chi_k) from x = chi/(2 pi) modulo 1 in 64-bit fixed point.  The constants are
// fractions of a turn, so the products with the integer squared frequency m are exact
// modulo 2 pi: the range reduction of chi (hundreds of radians at the band edge) loses
// nothing, and the top 32 bits give chi in [-pi, pi) to 2^-31 turns.
__device__ __forceinline__ float sin_from_turns(uint64_t x) {
  const int32_t hi = (int32_t)(x >> 32);
  return sinpif((float)hi * 4.656612873077393e-10f);  // hi * 2^-31 = chi / pi in [-1, 1)
}

// sin(pi t) for t = hi * 2^-31 in [-1, 1) (hi: the top 32 bits of chi / (2 pi) in
// fixed point, so chi = pi t is already reduced to [-pi, pi) exactly by the integer
// phase).  The hardware sine (__sinf, maximum absolute error 2^-21.4 on [-pi, pi])
// measured faster than an odd polynomial after a quadrant fold, at 5.7e-7 instead of
// 5.2e-7 rel-L2 against the FP64 oracle on the 256^3 / 360-view scan.
__device__ __forceinline__ float sin_half_turns(int32_t hi) {
  return __sinf((float)hi * 1.4629180792671596e-09f);  // hi * 2 pi / 2^32
}

// sin and cos of chi = pi t for t = hi * 2^-31 in [-1, 1) (hardware sine and cosine).
__device__ __forceinline__ void sincos_half_turns(int32_t hi, float* sn, float* cs) {
  __sincosf((float)hi * 1.4629180792671596e-09f, sn, cs);  // hi * 2 pi / 2^32
}

// The stack stores horizontal tap pairs: entry (row v + 1, column c) of a layer holds
// (Y[v][c - 1], Y[v][c]) for c in [0, nu], zero outside the image, so a bilinear row is
// one 8-byte (float32) or 4-byte (bfloat16) load.
template <typename PairT>
__device__ __forceinline__ PairT make_pair(float a, float b);
template <>
__device__ __forceinline__ float2 make_pair<float2>(float a, float b) { return make_float2(a, b); }
template <>
__device__ __forceinline__ __nv_bfloat162 make_pair<__nv_bfloat162>(float a, float b) {
  return __floats2bfloat162_rn(a, b);
}

// ------------------------------------------------------------------ register FFT kernels
template <int P>
__global__ void __launch_bounds__(kThreads) k_rows_fwd(const float* __restrict__ images, float2* __restrict__ S,
                                                        const float2* __restrict__ twg, StageAConst c,
                                                        int dir_begin) {
  constexpr int TT = P / 8, G = groups_per_cta<P>(), L = fft::buffer_len(P, G), NT = fft::pass_table_len(P);
  __shared__ float2 tw[NT];
  __shared__ float2 buf_all[G * L];
  const int g = threadIdx.x / TT, j = threadIdx.x % TT;
  float2* buf = buf_all + g * L;
  for (int i = threadIdx.x; i < NT; i += kThreads) tw[i] = twg[i];
  const int n = blockIdx.y;
  const int v0 = 2 * (blockIdx.x * G + g);
  const bool row1 = v0 < c.nv, row2 = v0 + 1 < c.nv;
  const float* im = images + (size_t)(dir_begin + n) * c.nu * c.nv;
  float2 x[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int u = j + s * TT;
    const bool in = u < c.nu;
    const float x1 = (row1 && in) ? contrast_of(im[(size_t)v0 * c.nu + u], c.input_mode) : 0.f;
    const float x2 = (row2 && in) ? contrast_of(im[(size_t)(v0 + 1) * c.nu + u], c.input_mode) : 0.f;
    x[s] = make_float2(x1, x2);
  }
  __syncthreads();
  fft::block_fft<P, false>(x, buf, tw, j);
  __syncthreads();
#pragma unroll
  for (int s = 0; s < 8; ++s) buf[padded(j + s * TT)] = x[s];
  __syncthreads();
  if (!row1) return;
  float2* s1 = S + ((size_t)n * c.nv + v0) * c.half;
  for (int m = j; m < c.half; m += TT) {
    const float2 zm = buf[padded(m & (P - 1))];
    const float2 zc = buf[padded((P - m) & (P - 1))];
    // X1 = (Z[m] + conj Z[P-m]) / 2,  X2 = (Z[m] - conj Z[P-m]) / (2i)
    s1[m] = make_float2(0.5f * (zm.x + zc.x), 0.5f * (zm.y - zc.y));
    if (row2) s1[c.half + m] = make_float2(0.5f * (zm.y + zc.y), -0.5f * (zm.x - zc.x));
  }
}

// FILT: 0 ramp only (filter off), 1 Tikhonov eps, 2 learned eps table, 3 the opposite-pair
// form of Eq. 10 / 11 (real part of the complex bracket at the image plane carried to the
// layer depth); DENS: density
// weighting (any geometry) instead of the ramp.  Compile-time, so that each variant keeps
// only the registers it uses.
// 3 resident CTAs per SM (80 registers) measured faster than 4 (64 registers) at P = 512.
template <int P, int FILT, bool DENS>
__global__ void __launch_bounds__(kThreads, 3) k_cols(const float2* __restrict__ S, float2* __restrict__ T,
                                                    const float2* __restrict__ twg, const uint64_t* __restrict__ uA,
                                                    const float* __restrict__ ramp, const DirParams* __restrict__ dirs,
                                                    const float* __restrict__ dens,
                                                    const double* __restrict__ band_sum,
                                                    const float* __restrict__ eps_tab, int n_bins, int bin_width,
                                                    StageAConst c, int dir_begin) {
  constexpr int TT = P / 8, CB = groups_per_cta<P>(), L = fft::buffer_len(P, CB), NT = fft::pass_table_len(P);
  __shared__ float2 tw[NT];
  __shared__ float2 buf_all[CB * L];
  const int g = threadIdx.x / TT, j = threadIdx.x % TT;
  float2* buf = buf_all + g * L;
  for (int i = threadIdx.x; i < NT; i += kThreads) tw[i] = twg[i];
  const int n = blockIdx.y;
  const int c0 = blockIdx.x * CB;
  const int col = c0 + g;
  const float2* Sn = S + (size_t)n * c.nv * c.half;
  // coalesced fill of rows v < nv of the CTA's CB columns
  for (int idx = threadIdx.x; idx < c.nv * CB; idx += kThreads) {
    const int t = idx % CB, v = idx / CB;
    buf_all[t * L + padded(v)] = (c0 + t < c.half) ? Sn[(size_t)v * c.half + c0 + t] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2 xg[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int v = j + s * TT;
    xg[s] = v < c.nv ? buf[padded(v)] : make_float2(0.f, 0.f);
  }
  // each group owns its exchange buffer from here on: barriers over the group only
  const fft::GroupSync gsync{1 + g, TT};
  fft::block_fft<P, false>(xg, buf, tw, j, gsync);  // G(col, m_v) at m_v = j + s*TT, kept for all layers

  const bool ok = col < c.half;
  const int colc = ok ? col : c.half - 1;
  // ramp (single-axis scans) or sampling-density weight (any geometry), 1/P^2 included
  float wgt[DENS ? 8 : 1];
  if constexpr (DENS) {
    const DirParams& dp = dirs[dir_begin + n];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int m = j + s * TT;
      const int mv = m < P / 2 ? m : m - P;
      float wv = density_weight(c.dens, dens, band_sum, dp.af, dp.bf, (float)colc, (float)mv);
      // the Nyquist bin is its own alias (+-P/2): mean over both, so that W stays even
      const bool nyq_u = colc == P / 2, nyq_v = m == P / 2;
      if (nyq_u || nyq_v) {
        const float w2 = density_weight(c.dens, dens, band_sum, dp.af, dp.bf, nyq_u ? -(float)colc : (float)colc,
                                        (nyq_v && !nyq_u) ? -(float)mv : (float)mv);
        wv = 0.5f * (wv + w2);
      }
      wgt[s] = wv;
    }
  } else {
    wgt[0] = ramp[colc];
  }
  // with a filter, the weight carries the filter's prefactor lambda / (4 pi sqrt(1+sigma^2))
  if constexpr (FILT != 0) {
#pragma unroll
    for (int s = 0; s < (DENS ? 8 : 1); ++s) wgt[s] *= c.pref;
  }
  // chi/(2 pi) in 2^-32 turns needs only the top 32 bits of the 64-bit fixed-point
  // sum: the per-layer product uA_k * m is formed as hi(uA) * m + umulhi(lo(uA), m), and
  // the layer-independent part uC * m^2 - uW once per element (dropped low-word carries
  // cost at most 2^-32 turns).
  uint32_t msq[8], base_hi[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int m = j + s * TT;
    const int mv = m < P / 2 ? m : m - P;
    msq[s] = (uint32_t)(colc * colc + mv * mv);
    const uint64_t m64 = msq[s];
    base_hi[s] = (uint32_t)((c.uC * (m64 * m64) - c.uW) >> 32);
  }
  // learned regulariser: the radial bin of each frequency (isqrt, exact integers)
  int bin[FILT == 2 ? 8 : 1];
  if constexpr (FILT == 2) {
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      int r = (int)sqrtf((float)msq[s]);
      while ((uint32_t)r * (uint32_t)r > msq[s]) --r;
      while ((uint32_t)(r + 1) * (uint32_t)(r + 1) <= msq[s]) ++r;
      const int b = r / bin_width;
      bin[s] = b < n_bins - 1 ? b : n_bins - 1;
    }
  }
  // the opposite-pair filter (FILT 3) keeps one row more per direction: the image-plane
  // phase constant after the Nz per-layer depth constants
  const uint64_t* uAn = uA + (size_t)(dir_begin + n) * (c.nz_layers + (FILT == 3 ? 1 : 0));
  float sp[FILT == 3 ? 8 : 1], cp[FILT == 3 ? 8 : 1];
  if constexpr (FILT == 3) {  // image-plane sin chi / (sin^2 chi + eps), cos chi / (cos^2 chi + eps)
    const uint64_t uR = uAn[c.nz_layers];
    const uint32_t r_hi = (uint32_t)(uR >> 32), r_lo = (uint32_t)uR;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      float sn, cs;
      sincos_half_turns((int32_t)(r_hi * msq[s] + __umulhi(r_lo, msq[s]) + base_hi[s]), &sn, &cs);
      sp[s] = c.pair_mode == 0 ? __fdividef(sn, fmaf(sn, sn, c.eps)) : (c.pair_mode == 1 ? 1.f : 0.f);
      cp[s] = c.pair_mode == 0 ? __fdividef(cs, fmaf(cs, cs, c.eps)) : (c.pair_mode == 1 ? 0.f : -1.f);
    }
  }
  float2* Tn = T + (size_t)n * c.nz_layers * c.half * c.nv;
  // this CTA's layers: group blockIdx.z of gridDim.z equal groups
  const int lg = (c.nz_layers + gridDim.z - 1) / gridDim.z;
  const int k_begin = blockIdx.z * lg;
  const int k_end = min(c.nz_layers, k_begin + lg);
  for (int k = k_begin; k < k_end; ++k) {
    const uint64_t uAk = uAn[k];
    const uint32_t a_hi = (uint32_t)(uAk >> 32), a_lo = (uint32_t)uAk;
    const float* eps_k = eps_tab + ((size_t)n * c.nz_layers + k) * n_bins;
    float2 x[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      float f = wgt[DENS ? s : 0];
      if constexpr (FILT == 3) {  // Re{bracket * exp(-i phi_k)}, phi_k = pi lambda z_k q^2
        float sn, cs;
        sincos_half_turns((int32_t)(a_hi * msq[s] + __umulhi(a_lo, msq[s])), &sn, &cs);
        f *= fmaf(sp[s], cs, -cp[s] * sn);
      } else if constexpr (FILT != 0) {
        const uint32_t hi = a_hi * msq[s] + __umulhi(a_lo, msq[s]) + base_hi[s];
        const float sn = sin_half_turns((int32_t)hi);
        float e;
        if constexpr (FILT == 2) e = __ldg(eps_k + bin[s]);  // learned eps
        else e = c.eps;                                      // Tikhonov eps
        f *= __fdividef(sn, fmaf(sn, sn, e));                // real part of the Eq. 11 bracket
      }
      x[s] = make_float2(xg[s].x * f, xg[s].y * f);
    }
    fft::block_fft<P, true>(x, buf, tw, j, gsync);
    if (ok) {
      float2* out = Tn + ((size_t)k * c.half + col) * c.nv;
      // nv <= P/2: elements s >= 4 (v >= P/2) are never kept (their last butterflies drop)
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int v = j + s * TT;
        if (v < c.nv) out[v] = x[s];
      }
    }
  }
}

template <int P, typename PairT>
__global__ void __launch_bounds__(kThreads) k_rows_inv(const float2* __restrict__ T, PairT* __restrict__ stack,
                                                        const float2* __restrict__ twg, StageAConst c) {
  constexpr int TT = P / 8, G = groups_per_cta<P>(), L = fft::buffer_len(P, G), H = P / 2 + 1;
  // tile row stride HS = 8/G (mod 16) float2: a half-warp of the coalesced fill below
  // (2G rows x 8/G consecutive columns) then writes 16 distinct bank pairs; with G >= 8 a
  // half-warp fills one column and the odd stride H already does
  constexpr int HS = G >= 8 ? H : H + ((8 / G - H % 16) % 16 + 16) % 16;
  constexpr int TILE = 2 * G * HS, BUF = G * L, NT = fft::pass_table_len(P);
  constexpr int USED = 2 * G * H;  // tile entries that hold spectrum values
  constexpr int FILL = (USED + kThreads - 1) / kThreads;
  __shared__ float2 tw[NT];
  // the half-spectrum tile is read once, before the FFT's first exchange: the
  // exchange buffer reuses its memory
  __shared__ float2 shared_mem[TILE > BUF ? TILE : BUF];
  float2* tile = shared_mem;
  const int g = threadIdx.x / TT, j = threadIdx.x % TT;
  float2* buf = shared_mem + g * L;
  for (int i = threadIdx.x; i < NT; i += kThreads) tw[i] = twg[i];
  const int n = blockIdx.z, k = blockIdx.y;
  const int vbase = blockIdx.x * 2 * G;
  const float2* Tk = T + ((size_t)n * c.nz_layers + k) * H * c.nv;
  {  // all loads in flight before the shared stores
    float2 tmp[FILL];
#pragma unroll
    for (int it = 0; it < FILL; ++it) {
      const int idx = threadIdx.x + it * kThreads;
      const int vv = idx % (2 * G), cc = idx / (2 * G);
      const int v = vbase + vv;
      tmp[it] = (idx < USED && v < c.nv) ? Tk[(size_t)cc * c.nv + v] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int it = 0; it < FILL; ++it) {
      const int idx = threadIdx.x + it * kThreads;
      if (idx < USED) tile[(idx % (2 * G)) * HS + idx / (2 * G)] = tmp[it];
    }
  }
  __syncthreads();
  const int v0 = vbase + 2 * g;
  const float2* X1 = tile + (2 * g) * HS;
  const float2* X2 = X1 + HS;
  float2 x[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int m = j + s * TT;
    float2 a, b;
    if (m <= P / 2) {
      a = X1[m];
      b = X2[m];
      if (m == 0 || m == P / 2) {  // C2R: DC and Nyquist bins are real
        a.y = 0.f;
        b.y = 0.f;
      }
    } else {  // Hermitian extension X[m] = conj X[P - m]
      a = X1[P - m];
      b = X2[P - m];
      a.y = -a.y;
      b.y = -b.y;
    }
    x[s] = make_float2(a.x - b.y, a.y + b.x);  // a + i b
  }
  fft::block_fft<P, true>(x, buf, tw, j);
  // rows v0 (real part) and v0 + 1 (imaginary part) at u = j + s*TT; pair them with
  // their right-hand neighbours through the (now free) exchange buffer
  // nu <= P/2 (P is at least twice the image size): the pairs of columns cc <= nu read
  // u < P/2 only, i.e. x[s] for s < 4, so the last pass's butterflies feeding s >= 4 drop;
  // column P/2 (s = 4, thread 0, when nu = P/2) is (Y[nu - 1], 0)
  __syncthreads();
#pragma unroll
  for (int s = 0; s < 4; ++s) buf[padded(j + s * TT)] = x[s];
  __syncthreads();
  PairT* Lk = stack + ((size_t)n * c.nz_layers + k) * c.layer_elems;
  const int sp = c.su;
  if (v0 < c.nv) {
    const bool two = v0 + 1 < c.nv;
    PairT* r1 = Lk + (size_t)(v0 + 1) * sp;
    PairT* r2 = r1 + sp;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      const int cc = j + s * TT;  // pair column: (Y[cc - 1], Y[cc])
      if (cc <= c.nu) {
        const float2 left = cc >= 1 ? buf[padded(cc - 1)] : make_float2(0.f, 0.f);
        const float2 right = cc < c.nu ? buf[padded(cc)] : make_float2(0.f, 0.f);
        r1[cc] = make_pair<PairT>(left.x, right.x);
        if (two) r2[cc] = make_pair<PairT>(left.y, right.y);
      }
    }
  }
  if (blockIdx.x == 0)  // top border row
    for (int i = threadIdx.x; i < sp; i += kThreads) Lk[i] = make_pair<PairT>(0.f, 0.f);
  if (vbase + 2 * G >= c.nv)  // bottom border row
    for (int i = threadIdx.x; i < sp; i += kThreads) Lk[(size_t)(c.nv + 1) * sp + i] = make_pair<PairT>(0.f, 0.f);
}


// ------------------------------------------------------------------ 16-value kernels (P >= 1024)
// The same column and row stages with the 16-value FFT of fft16.cuh: three passes and two
// exchanges per length-2048 transform instead of four and three, exchange addresses that
// are a per-thread base plus constants, and (in the column kernel) double-buffered
// exchanges, so two group barriers per transform instead of six.
constexpr int kThreads16 = 256;

template <int P>
__host__ __device__ constexpr int cols16_per_cta() {
  return kThreads16 / (P / 16);
}

// Column stage: a group of P/16 threads per spectrum column, cols16_per_cta columns per CTA.
// The forward FFT along v stays in registers, multiplied once by the column's weight (ramp
// or density weight, with the filter prefactor and 1/P^2); per layer: the CTF filter,
// inverse FFT, store v < nv.
template <int P, int FILT, bool DENS>
__global__ void __launch_bounds__(kThreads16, FILT == 3 ? 1 : 2) k_cols16(const float2* __restrict__ S, float2* __restrict__ T,
                                                          const float2* __restrict__ twg,
                                                          const uint64_t* __restrict__ uA,
                                                          const float* __restrict__ ramp,
                                                          const DirParams* __restrict__ dirs,
                                                          const float* __restrict__ dens,
                                                          const double* __restrict__ band_sum,
                                                          const float* __restrict__ eps_tab, int n_bins,
                                                          int bin_width, StageAConst c, int dir_begin) {
  constexpr int TT = P / 16, CB = cols16_per_cta<P>(), L = fft16::buffer_len(P), NT = fft16::table_len(P);
  extern __shared__ float2 smem16[];
  float2* tw = smem16;
  const int g = threadIdx.x / TT, j = threadIdx.x % TT;
  float2* buf0 = smem16 + NT + (2 * g) * L;
  float2* buf1 = buf0 + L;
  for (int i = threadIdx.x; i < NT; i += kThreads16) tw[i] = twg[i];
  const int n = blockIdx.y;
  const int col = blockIdx.x * CB + g;
  const bool ok = col < c.half;
  const int colc = ok ? col : c.half - 1;
  const float2* Sn = S + (size_t)n * c.nv * c.half;
  float2 xg[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const int v = j + s * TT;
    xg[s] = v < c.nv ? Sn[(size_t)v * c.half + colc] : make_float2(0.f, 0.f);
  }
  __syncthreads();  // twiddle table
  const fft::GroupSync gsync{1 + g, TT};
  fft16::group_fft_db<P, false>(xg, buf0, buf1, tw, j, gsync);  // G(col, m_v) at m_v = j + s*TT
  // ramp (single-axis scans) or sampling-density weight (any geometry), 1/P^2 included, and
  // with a filter its prefactor lambda / (4 pi sqrt(1+sigma^2)): layer-independent, so
  // folded into the spectrum once
  {
    const float pref = FILT != 0 ? c.pref : 1.f;
    if constexpr (DENS) {
      const DirParams& dp = dirs[dir_begin + n];
#pragma unroll
      for (int s = 0; s < 16; ++s) {
        const int m = j + s * TT;
        const int mv = m < P / 2 ? m : m - P;
        float wv = density_weight(c.dens, dens, band_sum, dp.af, dp.bf, (float)colc, (float)mv);
        const bool nyq_u = colc == P / 2, nyq_v = m == P / 2;  // the Nyquist bin is its own alias
        if (nyq_u || nyq_v) {
          const float w2 = density_weight(c.dens, dens, band_sum, dp.af, dp.bf, nyq_u ? -(float)colc : (float)colc,
                                          (nyq_v && !nyq_u) ? -(float)mv : (float)mv);
          wv = 0.5f * (wv + w2);
        }
        wv *= pref;
        xg[s] = make_float2(xg[s].x * wv, xg[s].y * wv);
      }
    } else {
      const float wv = ramp[colc] * pref;
#pragma unroll
      for (int s = 0; s < 16; ++s) xg[s] = make_float2(xg[s].x * wv, xg[s].y * wv);
    }
  }
  // chi/(2 pi) in 2^-32 turns (top 32 bits of the 64-bit fixed-point phase): per layer
  // hi(uA_k) m + umulhi(lo(uA_k), m), plus the layer-independent uC m^2 - uW
  uint32_t msq[16], base_hi[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const int m = j + s * TT;
    const int mv = m < P / 2 ? m : m - P;
    const uint32_t q2 = (uint32_t)(colc * colc + mv * mv);
    const uint64_t m64 = q2;
    base_hi[s] = (uint32_t)((c.uC * (m64 * m64) - c.uW) >> 32);
    if constexpr (FILT == 2) {  // radial bin (exact isqrt) packed above the 22-bit m
      int r = (int)sqrtf((float)q2);
      while ((uint32_t)r * (uint32_t)r > q2) --r;
      while ((uint32_t)(r + 1) * (uint32_t)(r + 1) <= q2) ++r;
      const int b = min(r / bin_width, n_bins - 1);
      msq[s] = q2 | ((uint32_t)b << 22);
    } else {
      msq[s] = q2;
    }
  }
  const uint64_t* uAn = uA + (size_t)(dir_begin + n) * (c.nz_layers + (FILT == 3 ? 1 : 0));
  float sp[FILT == 3 ? 16 : 1], cp[FILT == 3 ? 16 : 1];
  if constexpr (FILT == 3) {  // image-plane sin chi / (sin^2 chi + eps), cos chi / (cos^2 chi + eps)
    const uint64_t uR = uAn[c.nz_layers];
    const uint32_t r_hi = (uint32_t)(uR >> 32), r_lo = (uint32_t)uR;
#pragma unroll
    for (int s = 0; s < 16; ++s) {
      float sn, cs;
      sincos_half_turns((int32_t)(r_hi * msq[s] + __umulhi(r_lo, msq[s]) + base_hi[s]), &sn, &cs);
      sp[s] = c.pair_mode == 0 ? __fdividef(sn, fmaf(sn, sn, c.eps)) : (c.pair_mode == 1 ? 1.f : 0.f);
      cp[s] = c.pair_mode == 0 ? __fdividef(cs, fmaf(cs, cs, c.eps)) : (c.pair_mode == 1 ? 0.f : -1.f);
    }
  }
  float2* Tn = T + (size_t)n * c.nz_layers * c.half * c.nv;
  const int lg = (c.nz_layers + gridDim.z - 1) / gridDim.z;
  const int k_begin = blockIdx.z * lg;
  const int k_end = min(c.nz_layers, k_begin + lg);
  for (int k = k_begin; k < k_end; ++k) {
    const uint64_t uAk = uAn[k];
    const uint32_t a_hi = (uint32_t)(uAk >> 32), a_lo = (uint32_t)uAk;
    const float* eps_k = eps_tab + ((size_t)n * c.nz_layers + k) * n_bins;
    float2 x[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) {
      if constexpr (FILT == 3) {  // Re{bracket * exp(-i phi_k)}, phi_k = pi lambda z_k q^2
        float sn, cs;
        sincos_half_turns((int32_t)(a_hi * msq[s] + __umulhi(a_lo, msq[s])), &sn, &cs);
        const float f = fmaf(sp[s], cs, -cp[s] * sn);
        x[s] = make_float2(xg[s].x * f, xg[s].y * f);
      } else if constexpr (FILT != 0) {
        const uint32_t q2 = FILT == 2 ? (msq[s] & 0x3FFFFFu) : msq[s];
        const uint32_t hi = a_hi * q2 + __umulhi(a_lo, q2) + base_hi[s];
        const float sn = sin_half_turns((int32_t)hi);
        float e;
        if constexpr (FILT == 2) e = __ldg(eps_k + (msq[s] >> 22));  // learned eps
        else e = c.eps;                                             // Tikhonov eps
        const float f = __fdividef(sn, fmaf(sn, sn, e));           // real part of the Eq. 11 bracket
        x[s] = make_float2(xg[s].x * f, xg[s].y * f);
      } else {
        x[s] = xg[s];
      }
    }
    fft16::group_fft_db<P, true>(x, buf0, buf1, tw, j, gsync);
    if (ok) {
      float2* out = Tn + ((size_t)k * c.half + col) * c.nv;
      // nv <= P/2 (P is at least twice the image size): elements s >= 8 (v >= P/2) are
      // never kept, so the last pass's butterflies that only feed them are dropped
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int v = j + s * TT;
        if (v < c.nv) out[v] = x[s];
      }
    }
  }
}

template <int P, int FILT, bool DENS>
constexpr size_t cols16_smem() {
  return sizeof(float2) * ((size_t)fft16::table_len(P) + 2 * (size_t)cols16_per_cta<P>() * fft16::buffer_len(P));
}

// Row stage: four row pairs (eight detector rows) of one layer per CTA, a group of P/16
// threads per pair.  The CTA reads eight consecutive v of every column of T (64 bytes per
// column), Hermitian-extends both half spectra of a pair, packs them as real + i real,
// inverse FFT, crop u < nu, stores tap pairs.
constexpr int kRowPairs16 = 4;

template <int P>
__host__ __device__ constexpr int rows16_threads() {
  return kRowPairs16 * (P / 16);
}

template <int P>
__host__ __device__ constexpr int rows16_tile_stride() {
  // stride = 2 (mod 16) float2: a half-warp of the fill (8 rows x 2 columns) writes 16
  // distinct bank pairs
  return (P / 2 + 1) + ((2 - (P / 2 + 1) % 16) % 16 + 16) % 16;
}

template <int P>
constexpr size_t rows16_smem() {
  constexpr size_t tile = (size_t)2 * kRowPairs16 * rows16_tile_stride<P>();
  constexpr size_t bufs = (size_t)kRowPairs16 * fft16::buffer_len(P);
  return sizeof(float2) * ((size_t)fft16::table_len(P) + (tile > bufs ? tile : bufs));
}

template <int P, typename PairT>
__global__ void __launch_bounds__(rows16_threads<P>(), 2) k_rows_inv16(const float2* __restrict__ T,
                                                                        PairT* __restrict__ stack,
                                                                        const float2* __restrict__ twg,
                                                                        StageAConst c) {
  constexpr int TT = P / 16, NTH = rows16_threads<P>(), H = P / 2 + 1, HS = rows16_tile_stride<P>();
  constexpr int ROWS = 2 * kRowPairs16, L = fft16::buffer_len(P), NT = fft16::table_len(P);
  constexpr int USED = ROWS * H;
  constexpr int FILL = (USED + NTH - 1) / NTH;
  extern __shared__ float2 smem16[];
  float2* tw = smem16;
  // the half-spectrum tile is read once, before the first exchange: the exchange buffers
  // reuse its memory
  float2* tile = smem16 + NT;
  const int g = threadIdx.x / TT, j = threadIdx.x % TT;
  float2* buf = smem16 + NT + g * L;
  for (int i = threadIdx.x; i < NT; i += NTH) tw[i] = twg[i];
  const int n = blockIdx.z, k = blockIdx.y;
  const int vbase = blockIdx.x * ROWS;
  const float2* Tk = T + ((size_t)n * c.nz_layers + k) * H * c.nv;
  {  // all loads in flight before the shared stores
    float2 tmp[FILL];
#pragma unroll
    for (int it = 0; it < FILL; ++it) {
      const int idx = threadIdx.x + it * NTH;
      const int vv = idx % ROWS, cc = idx / ROWS;
      const int v = vbase + vv;
      tmp[it] = (idx < USED && v < c.nv) ? Tk[(size_t)cc * c.nv + v] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int it = 0; it < FILL; ++it) {
      const int idx = threadIdx.x + it * NTH;
      if (idx < USED) tile[(idx % ROWS) * HS + idx / ROWS] = tmp[it];
    }
  }
  __syncthreads();
  const int v0 = vbase + 2 * g;
  const float2* X1 = tile + (2 * g) * HS;
  const float2* X2 = X1 + HS;
  float2 x[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const int m = j + s * TT;
    float2 a, b;
    if (m <= P / 2) {
      a = X1[m];
      b = X2[m];
      if (m == 0 || m == P / 2) {  // C2R: DC and Nyquist bins are real
        a.y = 0.f;
        b.y = 0.f;
      }
    } else {  // Hermitian extension X[m] = conj X[P - m]
      a = X1[P - m];
      b = X2[P - m];
      a.y = -a.y;
      b.y = -b.y;
    }
    x[s] = make_float2(a.x - b.y, a.y + b.x);  // a + i b
  }
  __syncthreads();  // every group has read its rows: the tile is free for the exchange buffers
  const fft::GroupSync gsync{1 + g, TT};
  fft16::group_fft_sb<P, true, fft::GroupSync, true>(x, buf, tw, j, gsync);
  // rows v0 (real part) and v0 + 1 (imaginary part) at u = j + s*TT.  The tap pair of column
  // cc = j + s*TT is (Y[cc - 1], Y[cc]): the left value comes from lane l - 1 by a warp
  // shuffle; lane 0 takes the last lane of the group's previous warp (same s), and thread 0
  // the group's last thread at s - 1, both published through the exchange buffer.
  gsync();  // the last pass's reads of the buffer are done
  const int lane = threadIdx.x & 31, wg = j >> 5;
  float2* edge = buf;  // [TT / 32][16]
  // nu <= P/2 (P is at least twice the image size): the pair columns cc <= nu need
  // x[s] for s < 8 only (and column P/2, when nu = P/2, the left value x[7] of the last
  // thread and a zero right value), so the last pass's butterflies feeding s >= 8 drop
  if (lane == 31) {
#pragma unroll
    for (int s = 0; s < 8; ++s) edge[wg * 16 + s] = x[s];
  }
  gsync();
  PairT* Lk = stack + ((size_t)n * c.nz_layers + k) * c.layer_elems;
  const int sp = c.su;
  const bool row1 = v0 < c.nv, two = v0 + 1 < c.nv;
  PairT* r1 = Lk + (size_t)(v0 + 1) * sp;
  PairT* r2 = r1 + sp;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    if (s * TT > c.nu) break;  // the same for every thread of the group
    const int cc = j + s * TT;  // pair column: (Y[cc - 1], Y[cc])
    float2 left = make_float2(__shfl_up_sync(0xffffffffu, x[s].x, 1), __shfl_up_sync(0xffffffffu, x[s].y, 1));
    if (lane == 0) {
      if (wg > 0) left = edge[(wg - 1) * 16 + s];
      else left = s > 0 ? edge[(TT / 32 - 1) * 16 + s - 1] : make_float2(0.f, 0.f);
    }
    const float2 right = cc < c.nu ? x[s] : make_float2(0.f, 0.f);
    if (row1 && cc <= c.nu) {
      r1[cc] = make_pair<PairT>(left.x, right.x);
      if (two) r2[cc] = make_pair<PairT>(left.y, right.y);
    }
  }
  if (j == 0 && row1 && c.nu == P / 2) {  // pair column P/2 = nu: (Y[nu - 1], 0)
    const float2 left = edge[(TT / 32 - 1) * 16 + 7];
    r1[P / 2] = make_pair<PairT>(left.x, 0.f);
    if (two) r2[P / 2] = make_pair<PairT>(left.y, 0.f);
  }
  if (blockIdx.x == 0)  // top border row
    for (int i = threadIdx.x; i < sp; i += NTH) Lk[i] = make_pair<PairT>(0.f, 0.f);
  if (vbase + ROWS >= c.nv)  // bottom border row
    for (int i = threadIdx.x; i < sp; i += NTH) Lk[(size_t)(c.nv + 1) * sp + i] = make_pair<PairT>(0.f, 0.f);
}

// ------------------------------------------------------------------ radix-2 fallback (P <= 8)
__device__ __forceinline__ int bitrev(int i, int logP) { return (int)(__brev((unsigned)i) >> (32 - logP)); }

template <bool INV>
__device__ void fft_radix2(float2* data, int P, int logP, const float2* tw) {
  const int halfP = P >> 1;
  for (int s = 0; s < logP; ++s) {
    const int half = 1 << s;
    const int tw_shift = logP - 1 - s;
    __syncthreads();
    for (int jj = threadIdx.x; jj < halfP; jj += blockDim.x) {
      const int pos = jj & (half - 1);
      const int i1 = ((jj - pos) << 1) + pos;
      float2 w = tw[pos << tw_shift];
      if (INV) w.y = -w.y;
      const float2 a = data[i1];
      const float2 wb = cmul(w, data[i1 + half]);
      data[i1] = make_float2(a.x + wb.x, a.y + wb.y);
      data[i1 + half] = make_float2(a.x - wb.x, a.y - wb.y);
    }
  }
  __syncthreads();
}

__global__ void k_small_rows_fwd(const float* __restrict__ images, float2* __restrict__ S,
                                 const float2* __restrict__ twg, StageAConst c, int dir_begin) {
  __shared__ float2 tw[8];
  __shared__ float2 z[8];
  const int n = blockIdx.y;
  const int v0 = blockIdx.x * 2;
  const bool two = v0 + 1 < c.nv;
  const float* im = images + (size_t)(dir_begin + n) * c.nu * c.nv;
  for (int i = threadIdx.x; i < c.P; i += blockDim.x) tw[i] = twg[i];
  for (int i = threadIdx.x; i < c.P; i += blockDim.x) {
    float x1 = 0.f, x2 = 0.f;
    if (i < c.nu) {
      x1 = contrast_of(im[(size_t)v0 * c.nu + i], c.input_mode);
      if (two) x2 = contrast_of(im[(size_t)(v0 + 1) * c.nu + i], c.input_mode);
    }
    z[bitrev(i, c.logP)] = make_float2(x1, x2);
  }
  fft_radix2<false>(z, c.P, c.logP, tw);
  float2* s1 = S + ((size_t)n * c.nv + v0) * c.half;
  for (int m = threadIdx.x; m < c.half; m += blockDim.x) {
    const float2 zm = z[m & (c.P - 1)];
    const float2 zc = z[(c.P - m) & (c.P - 1)];
    s1[m] = make_float2(0.5f * (zm.x + zc.x), 0.5f * (zm.y - zc.y));
    if (two) s1[c.half + m] = make_float2(0.5f * (zm.y + zc.y), -0.5f * (zm.x - zc.x));
  }
}

__global__ void k_small_cols(const float2* __restrict__ S, float2* __restrict__ T, const float2* __restrict__ twg,
                             const uint64_t* __restrict__ uA, const float* __restrict__ ramp,
                             const DirParams* __restrict__ dirs, const float* __restrict__ dens,
                             const double* __restrict__ band_sum, const float* __restrict__ eps_tab, int n_bins,
                             int bin_width, StageAConst c, int dir_begin) {
  __shared__ float2 tw[8];
  __shared__ float2 G[8];
  __shared__ float2 Wk[8];
  const int n = blockIdx.y;
  const int col = blockIdx.x;  // one column per CTA
  for (int i = threadIdx.x; i < c.P; i += blockDim.x) tw[i] = twg[i];
  const float2* Sn = S + (size_t)n * c.nv * c.half;
  for (int v = threadIdx.x; v < c.P; v += blockDim.x)
    G[bitrev(v, c.logP)] = v < c.nv ? Sn[(size_t)v * c.half + col] : make_float2(0.f, 0.f);
  fft_radix2<false>(G, c.P, c.logP, tw);
  const uint64_t* uAn = uA + (size_t)(dir_begin + n) * (c.nz_layers + (c.filter == 3 ? 1 : 0));
  const int hP = c.P >> 1;
  for (int k = 0; k < c.nz_layers; ++k) {
    for (int m = threadIdx.x; m < c.P; m += blockDim.x) {
      const int mv = m < (c.P >> 1) ? m : m - c.P;
      const uint64_t msq = (uint64_t)(col * col + mv * mv);
      float f = ramp[col];
      if (c.dens.enabled) {
        const DirParams& dp = dirs[dir_begin + n];
        f = density_weight(c.dens, dens, band_sum, dp.af, dp.bf, (float)col, (float)mv);
        const bool nyq_u = col == hP, nyq_v = m == hP;  // the Nyquist bin is its own alias
        if (nyq_u || nyq_v)
          f = 0.5f * (f + density_weight(c.dens, dens, band_sum, dp.af, dp.bf, nyq_u ? -(float)col : (float)col,
                                         (nyq_v && !nyq_u) ? -(float)mv : (float)mv));
      }
      if (c.filter == 3) {  // opposite-pair filter: image-plane chi, depth phase of layer k
        float sn, cs, sz, cz;
        sincos_half_turns((int32_t)((uAn[c.nz_layers] * msq + c.uC * (msq * msq) - c.uW) >> 32), &sn, &cs);
        sincos_half_turns((int32_t)((uAn[k] * msq) >> 32), &sz, &cz);
        const float sp = c.pair_mode == 0 ? __fdividef(sn, fmaf(sn, sn, c.eps)) : (c.pair_mode == 1 ? 1.f : 0.f);
        const float cp = c.pair_mode == 0 ? __fdividef(cs, fmaf(cs, cs, c.eps)) : (c.pair_mode == 1 ? 0.f : -1.f);
        f *= c.pref * (sp * cz - cp * sz);
      } else if (c.filter) {
        const float sn = sin_from_turns(uAn[k] * msq + c.uC * (msq * msq) - c.uW);
        float e = c.eps;
        if (c.filter == 2) {
          int r = 0;
          while ((uint64_t)(r + 1) * (uint64_t)(r + 1) <= msq) ++r;
          const int b = r / bin_width;
          e = eps_tab[((size_t)n * c.nz_layers + k) * n_bins + (b < n_bins - 1 ? b : n_bins - 1)];
        }
        f *= c.pref * __fdividef(sn, fmaf(sn, sn, e));
      }
      Wk[bitrev(m, c.logP)] = make_float2(G[m].x * f, G[m].y * f);
    }
    fft_radix2<true>(Wk, c.P, c.logP, tw);
    float2* out = T + (((size_t)n * c.nz_layers + k) * c.half + col) * c.nv;
    for (int v = threadIdx.x; v < c.nv; v += blockDim.x) out[v] = Wk[v];
    __syncthreads();
  }
}

template <typename PairT>
__global__ void k_small_rows_inv(const float2* __restrict__ T, PairT* __restrict__ stack,
                                 const float2* __restrict__ twg, StageAConst c) {
  __shared__ float2 tw[8];
  __shared__ float2 z[8];
  const int n = blockIdx.z, k = blockIdx.y;
  const int v0 = blockIdx.x * 2;
  const bool two = v0 + 1 < c.nv;
  for (int i = threadIdx.x; i < c.P; i += blockDim.x) tw[i] = twg[i];
  const float2* Tk = T + ((size_t)n * c.nz_layers + k) * c.half * c.nv;
  const int hP = c.P >> 1;
  for (int m = threadIdx.x; m < c.P; m += blockDim.x) {
    const int mm = m <= hP ? m : c.P - m;
    float2 a = Tk[(size_t)mm * c.nv + v0];
    float2 b = two ? Tk[(size_t)mm * c.nv + v0 + 1] : make_float2(0.f, 0.f);
    if (m == 0 || m == hP) {
      a.y = 0.f;
      b.y = 0.f;
    } else if (m > hP) {
      a.y = -a.y;
      b.y = -b.y;
    }
    z[bitrev(m, c.logP)] = make_float2(a.x - b.y, a.y + b.x);
  }
  fft_radix2<true>(z, c.P, c.logP, tw);
  PairT* L = stack + ((size_t)n * c.nz_layers + k) * c.layer_elems;
  const int sp = c.su;
  for (int cc = threadIdx.x; cc <= c.nu; cc += blockDim.x) {
    const float2 left = cc >= 1 ? z[cc - 1] : make_float2(0.f, 0.f);
    const float2 right = cc < c.nu ? z[cc] : make_float2(0.f, 0.f);
    L[(size_t)(v0 + 1) * sp + cc] = make_pair<PairT>(left.x, right.x);
    if (two) L[(size_t)(v0 + 2) * sp + cc] = make_pair<PairT>(left.y, right.y);
    if (v0 == 0) L[cc] = make_pair<PairT>(0.f, 0.f);
    if (v0 + 2 >= c.nv) L[(size_t)(c.nv + 1) * sp + cc] = make_pair<PairT>(0.f, 0.f);
  }
}

// ------------------------------------------------------------------ finiteness scan
__global__ void k_count_nonfinite(const float* __restrict__ x, size_t n, unsigned int* __restrict__ count) {
  unsigned int bad = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    bad += isfinite(x[i]) ? 0u : 1u;
  for (int o = 16; o > 0; o >>= 1) bad += __shfl_down_sync(0xffffffffu, bad, o);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(count, bad);
}

// ------------------------------------------------------------------ launch
// Layer groups of the column stage: the split of the Nz layers over CTAs that keeps the
// last wave of `slots` resident CTAs fullest, counting the set-up each group repeats (the
// column's forward FFT and weights, `setup` layers' worth of work) as extra work.
int pick_layer_groups(int ctas_per_group, int nz_layers, int slots, double setup) {
  int best = 1;
  double best_eff = 0.0;
  const int max_lg = nz_layers / 2 > 0 ? (nz_layers / 2 < 16 ? nz_layers / 2 : 16) : 1;
  for (int lg = 1; lg <= max_lg; ++lg) {
    const double waves = (double)ctas_per_group * lg / slots;
    const double fill = waves / std::ceil(waves);
    const double eff = fill * (double)nz_layers / (nz_layers + setup * lg);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = lg;
    }
  }
  return best;
}

template <int P, int FILT, bool DENS>
cudaError_t launch_cols16(const StageAConst& c, const Workspace& ws, const float2* twq, int d0, int cnt, int sms,
                          cudaStream_t stream) {
  constexpr size_t smem = cols16_smem<P, FILT, DENS>();
  static unsigned long long attr_set = 0;  // devices on which the shared-memory limit is raised
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 64 || !(attr_set >> dev & 1ull)) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_cols16<P, FILT, DENS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dev < 64) attr_set |= 1ull << dev;
  }
  constexpr int CB = cols16_per_cta<P>();
  const int col_groups = (c.half + CB - 1) / CB;
  // set-up per group: the forward FFT (about one layer's work), and with the density
  // weighting about one more for the weights' trilinear lookups
  const int lg = pick_layer_groups(col_groups * cnt, c.nz_layers, (FILT == 3 ? 1 : 2) * sms, DENS ? 2.2 : 1.2);
  k_cols16<P, FILT, DENS><<<dim3(col_groups, cnt, lg), kThreads16, smem, stream>>>(
      ws.S, ws.T, twq, ws.uA, ws.ramp, ws.dirs, ws.dens, ws.band_sum, ws.eps, ws.n_bins, ws.bin_width, c, d0);
  return cudaGetLastError();
}

template <int P, typename PairT>
cudaError_t launch_rows_inv16(const StageAConst& c, const float2* T, PairT* stack, const float2* twq, int cnt,
                              cudaStream_t stream) {
  constexpr size_t smem = rows16_smem<P>();
  static unsigned long long attr_set = 0;  // devices on which the shared-memory limit is raised
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 64 || !(attr_set >> dev & 1ull)) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_rows_inv16<P, PairT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dev < 64) attr_set |= 1ull << dev;
  }
  const dim3 gi((c.nv + 2 * kRowPairs16 - 1) / (2 * kRowPairs16), c.nz_layers, cnt);
  k_rows_inv16<P, PairT><<<gi, rows16_threads<P>(), smem, stream>>>(T, stack, twq, c);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_reg(const StageAConst& c, const Workspace& ws, const float* images, int dir_begin, int dir_count,
                       cudaStream_t stream, EventRecorder* rec, const StageAHook* hook) {
  constexpr int G = groups_per_cta<P>();
  // Sub-blocks of c.sub_block directions: S and T of one sub-block stay in L2 between the
  // column and the row kernels; each sub-block writes its part of the block's stack.
  const int sub = c.sub_block > 0 ? c.sub_block : dir_count;
  const int col_groups = (c.half + G - 1) / G;
  const int sms = device_sm_count();
  for (int s0 = 0; s0 < dir_count; s0 += sub) {
    const int cnt = min(sub, dir_count - s0);
    const int d0 = dir_begin + s0;
    k_rows_fwd<P><<<dim3((c.nv + 2 * G - 1) / (2 * G), cnt), kThreads, 0, stream>>>(images, ws.S, ws.twp, c, d0);
    if (hook) {
      const cudaError_t e = hook->fn(hook->ctx, d0, cnt, stream);
      if (e != cudaSuccess) return e;
    }
    if (rec) rec->mark(0, stream);
    const bool dens = c.dens.enabled != 0;
    const size_t stack_off = (size_t)s0 * c.nz_layers * c.layer_elems;
    if constexpr (P >= 1024) {
      // 16-value FFTs (fft16.cuh); their twiddle table follows the 8-value one
      const float2* twq = ws.twp + (P - 8);
      cudaError_t e;
      if (c.filter == 0) e = dens ? launch_cols16<P, 0, true>(c, ws, twq, d0, cnt, sms, stream)
                                  : launch_cols16<P, 0, false>(c, ws, twq, d0, cnt, sms, stream);
      else if (c.filter == 3) e = dens ? launch_cols16<P, 3, true>(c, ws, twq, d0, cnt, sms, stream)
                                       : launch_cols16<P, 3, false>(c, ws, twq, d0, cnt, sms, stream);
      else if (c.filter == 2) e = dens ? launch_cols16<P, 2, true>(c, ws, twq, d0, cnt, sms, stream)
                                       : launch_cols16<P, 2, false>(c, ws, twq, d0, cnt, sms, stream);
      else e = dens ? launch_cols16<P, 1, true>(c, ws, twq, d0, cnt, sms, stream)
                    : launch_cols16<P, 1, false>(c, ws, twq, d0, cnt, sms, stream);
      if (e != cudaSuccess) return e;
      if (rec) rec->mark(1, stream);
      if (c.stack_bf16)
        e = launch_rows_inv16<P, __nv_bfloat162>(c, ws.T, (__nv_bfloat162*)ws.stack + stack_off, twq, cnt, stream);
      else
        e = launch_rows_inv16<P, float2>(c, ws.T, (float2*)ws.stack + stack_off, twq, cnt, stream);
      if (e != cudaSuccess) return e;
      if (rec) rec->mark(2, stream);
      continue;
    }
    // layer groups so that about 2 waves of CTAs run even for a small sub-block
    const int target = 2 * sms * 4;
    int lgroups = (target + col_groups * cnt - 1) / (col_groups * cnt);
    lgroups = max(1, min(lgroups, c.nz_layers / 2 > 0 ? c.nz_layers / 2 : 1));
    const dim3 gc(col_groups, cnt, lgroups);
#define RECON_K_COLS(F, D)                                                                                      \
  k_cols<P, F, D><<<gc, kThreads, 0, stream>>>(ws.S, ws.T, ws.twp, ws.uA, ws.ramp, ws.dirs, ws.dens, ws.band_sum, \
                                               ws.eps, ws.n_bins, ws.bin_width, c, d0)
    if (c.filter == 0) {
      if (dens) RECON_K_COLS(0, true); else RECON_K_COLS(0, false);
    } else if (c.filter == 2) {
      if (dens) RECON_K_COLS(2, true); else RECON_K_COLS(2, false);
    } else if (c.filter == 3) {
      if (dens) RECON_K_COLS(3, true); else RECON_K_COLS(3, false);
    } else {
      if (dens) RECON_K_COLS(1, true); else RECON_K_COLS(1, false);
    }
#undef RECON_K_COLS
    if (rec) rec->mark(1, stream);
    const dim3 gi((c.nv + 2 * G - 1) / (2 * G), c.nz_layers, cnt);
    if (c.stack_bf16)
      k_rows_inv<P, __nv_bfloat162><<<gi, kThreads, 0, stream>>>(ws.T, (__nv_bfloat162*)ws.stack + stack_off, ws.twp,
                                                                 c);
    else
      k_rows_inv<P, float2><<<gi, kThreads, 0, stream>>>(ws.T, (float2*)ws.stack + stack_off, ws.twp, c);
    if (rec) rec->mark(2, stream);
  }
  return cudaGetLastError();
}

template <int P>
cudaError_t rows_fwd_only(const StageAConst& c, float2* S, const float2* twp, const float* images, int first,
                          int count, cudaStream_t stream) {
  constexpr int G = groups_per_cta<P>();
  k_rows_fwd<P><<<dim3((c.nv + 2 * G - 1) / (2 * G), count), kThreads, 0, stream>>>(images, S, twp, c, first);
  return cudaGetLastError();
}

cudaError_t launch_small(const StageAConst& c, const Workspace& ws, const float* images, int dir_begin,
                         int dir_count, cudaStream_t stream, EventRecorder* rec) {
  k_small_rows_fwd<<<dim3((c.nv + 1) / 2, dir_count), 32, 0, stream>>>(images, ws.S, ws.tw, c, dir_begin);
  if (rec) rec->mark(0, stream);
  k_small_cols<<<dim3(c.half, dir_count), 32, 0, stream>>>(ws.S, ws.T, ws.tw, ws.uA, ws.ramp, ws.dirs, ws.dens,
                                                          ws.band_sum, ws.eps, ws.n_bins, ws.bin_width, c,
                                                          dir_begin);
  if (rec) rec->mark(1, stream);
  const dim3 gi((c.nv + 1) / 2, c.nz_layers, dir_count);
  if (c.stack_bf16)
    k_small_rows_inv<__nv_bfloat162><<<gi, 32, 0, stream>>>(ws.T, (__nv_bfloat162*)ws.stack, ws.tw, c);
  else
    k_small_rows_inv<float2><<<gi, 32, 0, stream>>>(ws.T, (float2*)ws.stack, ws.tw, c);
  if (rec) rec->mark(2, stream);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stage_a(const StageAConst& c, const Workspace& ws, const float* images, int dir_begin,
                           int dir_count, cudaStream_t stream, EventRecorder* ev, const StageAHook* hook) {
  if (dir_count <= 0) return cudaSuccess;
  switch (c.P) {
    case 16: return launch_reg<16>(c, ws, images, dir_begin, dir_count, stream, ev, hook);
    case 32: return launch_reg<32>(c, ws, images, dir_begin, dir_count, stream, ev, hook);
    case 64: return launch_reg<64>(c, ws, images, dir_begin, dir_count, stream, ev, hook);
    case 128: return launch_reg<128>(c, ws, images, dir_begin, dir_count, stream, ev, hook);
    case 256: return launch_reg<256>(c, ws, images, dir_begin, dir_count, stream, ev, hook);
    case 512: return launch_reg<512>(c, ws, images, dir_begin, dir_count, stream, ev, hook);
    case 1024: return launch_reg<1024>(c, ws, images, dir_begin, dir_count, stream, ev, hook);
    case 2048: return launch_reg<2048>(c, ws, images, dir_begin, dir_count, stream, ev, hook);
    default: return hook ? cudaErrorInvalidValue : launch_small(c, ws, images, dir_begin, dir_count, stream, ev);
  }
}

cudaError_t launch_count_nonfinite(const float* x, size_t n, unsigned int* count, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const size_t want = (n + 255) / 256;
  const size_t cap = (size_t)device_sm_count() * 8;
  k_count_nonfinite<<<(unsigned)(want < cap ? want : cap), 256, 0, stream>>>(x, n, count);
  return cudaGetLastError();
}

cudaError_t launch_rows_fwd(const StageAConst& c, float2* S, const float2* twp, const float* images, int first,
                            int count, cudaStream_t stream) {
  if (count <= 0) return cudaSuccess;
  switch (c.P) {
    case 16: return rows_fwd_only<16>(c, S, twp, images, first, count, stream);
    case 32: return rows_fwd_only<32>(c, S, twp, images, first, count, stream);
    case 64: return rows_fwd_only<64>(c, S, twp, images, first, count, stream);
    case 128: return rows_fwd_only<128>(c, S, twp, images, first, count, stream);
    case 256: return rows_fwd_only<256>(c, S, twp, images, first, count, stream);
    case 512: return rows_fwd_only<512>(c, S, twp, images, first, count, stream);
    case 1024: return rows_fwd_only<1024>(c, S, twp, images, first, count, stream);
    case 2048: return rows_fwd_only<2048>(c, S, twp, images, first, count, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace recon
