// Learned regulariser of the CTF inverse: eps_theta = softplus(MLP(x)) per (direction n,
// layer k, radial bin b) replaces the Tikhonov eps of Eq. 11 (chosen "ad hoc" in Sec. 3).
// Features x: log10 of the bin's signal-to-noise ratio (radial power spectrum of the
// contrast over the Poisson floor (NSR M)^2 per DFT coefficient, the Parseval scaling of
// Sec. 3's noise filter) / 3, clamped to [-1, 2]; the bin-centre radius / (P/2); the layer's
// effective defocus lambda (R_n - z_k) / delta^2 / 100.  Network 3 -> 64 -> 64 -> 1 (ReLU),
// FP32 weights W1[64][3], b1, W2[64][64], b2, w3, b3.
//
// Kernels:
//   k_cols_forward<P>  column FFTs of the row spectra (as in k_cols), then the radial power
//                      sum_{q in b} mult |G(q)|^2 (mult = 2 for the columns standing for two
//                      of the full grid) and, for training, the column spectra themselves
//   k_eps_table        one thread per (n, k, b): SNR, features, MLP, eps (and activations)
//   k_train_loss       per frequency of every (image, layer): H G - T, the loss sums and
//                      d loss / d eps_b
//   k_mlp_backward     backpropagation of d loss / d eps to the 4481 parameters
//   k_adam             Adam (Kingma and Ba 2015) on the parameters
#include <cuda_runtime.h>

#include "fft_reg.cuh"
#include "learned.cuh"
#include "recon_internal.h"

namespace recon {
namespace {

constexpr int kThreads = 256;
constexpr int H = kMlpHidden;

template <int P>
__host__ __device__ constexpr int groups() {
  return kThreads / (P / 8) > 0 ? kThreads / (P / 8) : 1;
}

__device__ __forceinline__ int isqrt_u32(uint32_t x) {
  int r = (int)sqrtf((float)x);
  while ((uint32_t)r * (uint32_t)r > x) --r;
  while ((uint32_t)(r + 1) * (uint32_t)(r + 1) <= x) ++r;
  return r;
}

__device__ __forceinline__ int radial_bin(const LearnConst& lc, uint32_t msq) {
  const int b = isqrt_u32(msq) / lc.bin_width;
  return b < lc.n_bins - 1 ? b : lc.n_bins - 1;
}

__device__ __forceinline__ float softplus(float o) { return o > 20.f ? o : log1pf(expf(o)); }

// sin(pi t) for t = hi * 2^-31 in [-1, 1) (hi: the top 32 bits of chi / (2 pi) in
// fixed point, so chi = pi t is already reduced to [-pi, pi) exactly by the integer
// phase).  The hardware sine (__sinf, maximum absolute error 2^-21.4 on [-pi, pi])
// measured faster than an odd polynomial after a quadrant fold, at 5.7e-7 instead of
// 5.2e-7 rel-L2 against the FP64 oracle on the 256^3 / 360-view scan.
__device__ __forceinline__ float sin_half_turns(int32_t hi) {
  return __sinf((float)hi * 1.4629180792671596e-09f);  // hi * 2 pi / 2^32
}

// ----------------------------------------------------------------- column forward FFT
template <int P>
__global__ void __launch_bounds__(kThreads) k_cols_forward(const float2* __restrict__ S, float2* __restrict__ G_out,
                                                            float* __restrict__ pow, const float2* __restrict__ twg,
                                                            StageAConst c, LearnConst lc) {
  constexpr int TT = P / 8, CB = groups<P>(), L = fft::buffer_len(P, CB), NT = fft::pass_table_len(P);
  __shared__ float2 tw[NT];
  __shared__ float2 buf_all[CB * L];
  __shared__ float hist[kMaxBins];
  const int g = threadIdx.x / TT, j = threadIdx.x % TT;
  float2* buf = buf_all + g * L;
  for (int i = threadIdx.x; i < NT; i += kThreads) tw[i] = twg[i];
  for (int i = threadIdx.x; i < lc.n_bins; i += kThreads) hist[i] = 0.f;
  const int n = blockIdx.y;
  const int c0 = blockIdx.x * CB;
  const int col = c0 + g;
  const float2* Sn = S + (size_t)n * c.nv * c.half;
  for (int idx = threadIdx.x; idx < c.nv * CB; idx += kThreads) {
    const int t = idx % CB, v = idx / CB;
    buf_all[t * L + fft::padded(v)] = (c0 + t < c.half) ? Sn[(size_t)v * c.half + c0 + t] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2 x[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int v = j + s * TT;
    x[s] = v < c.nv ? buf[fft::padded(v)] : make_float2(0.f, 0.f);
  }
  fft::block_fft<P, false>(x, buf, tw, j);
  const bool ok = col < c.half;
  if (ok && G_out) {
    float2* out = G_out + ((size_t)n * c.half + col) * P;
#pragma unroll
    for (int s = 0; s < 8; ++s) out[j + s * TT] = x[s];
  }
  if (pow) {
    if (ok) {
      const float mult = (col == 0 || col == P / 2) ? 1.f : 2.f;
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int m = j + s * TT;
        const int mv = m < P / 2 ? m : m - P;
        const int b = radial_bin(lc, (uint32_t)(col * col + mv * mv));
        atomicAdd(&hist[b], mult * (x[s].x * x[s].x + x[s].y * x[s].y));
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < lc.n_bins; i += kThreads)
      if (hist[i] != 0.f) atomicAdd(&pow[(size_t)n * lc.n_bins + i], hist[i]);
  }
}

// ----------------------------------------------------------------- MLP forward
__device__ __forceinline__ void features(const LearnConst& lc, const float* __restrict__ pow,
                                         const float* __restrict__ cnt, const float* __restrict__ x2tab, int n,
                                         int k, int b, int n_layers, float x[3]) {
  const float N0 = lc.noise_floor;
  const float pw = pow[(size_t)n * lc.n_bins + b] / fmaxf(cnt[b], 1.f);
  const float snr = fmaxf(pw - N0, 1e-3f * N0) / N0;
  x[0] = fminf(fmaxf(log10f(snr), -3.f), 6.f) * (1.f / 3.f);
  x[1] = ((float)b + 0.5f) * (float)lc.bin_width * lc.inv_half_p;
  x[2] = x2tab[(size_t)n * n_layers + k];
}

__global__ void __launch_bounds__(kThreads) k_eps_table(const float* __restrict__ pow, const float* __restrict__ cnt,
                                                         const float* __restrict__ x2tab,
                                                         const float* __restrict__ theta, float* __restrict__ eps,
                                                         float* __restrict__ acts, LearnConst lc, int n_dirs,
                                                         int n_layers, int dir_begin) {
  __shared__ float w[kMlpParams];
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) w[i] = theta[i];
  __syncthreads();
  const size_t rows = (size_t)n_dirs * n_layers * lc.n_bins;
  const size_t row = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= rows) return;
  const int b = (int)(row % lc.n_bins);
  const int k = (int)((row / lc.n_bins) % n_layers);
  const int n = (int)(row / ((size_t)lc.n_bins * n_layers));
  float x[3];
  features(lc, pow, cnt, x2tab, n, k, b, n_layers, x);
  x[2] = x2tab[(size_t)(dir_begin + n) * n_layers + k];
  const float* W1 = w;
  const float* b1 = W1 + 3 * H;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* w3 = b2 + H;
  const float b3 = w3[H];
  float h1[H];
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const float a = fmaf(W1[3 * i], x[0], fmaf(W1[3 * i + 1], x[1], fmaf(W1[3 * i + 2], x[2], b1[i])));
    if (acts) acts[row * kActStride + 3 + i] = a;
    h1[i] = fmaxf(a, 0.f);
  }
  float o = b3;
  for (int i = 0; i < H; ++i) {
    float a = b2[i];
#pragma unroll
    for (int q = 0; q < H; ++q) a = fmaf(W2[i * H + q], h1[q], a);
    if (acts) acts[row * kActStride + 3 + H + i] = a;
    o = fmaf(w3[i], fmaxf(a, 0.f), o);
  }
  if (acts) {
    acts[row * kActStride + 0] = x[0];
    acts[row * kActStride + 1] = x[1];
    acts[row * kActStride + 2] = x[2];
    acts[row * kActStride + 3 + 2 * H] = o;
  }
  eps[row] = softplus(o) * lc.eps_scale;
}

// ----------------------------------------------------------------- training loss
template <int P>
__global__ void __launch_bounds__(kThreads) k_train_loss(const float2* __restrict__ G, const float2* __restrict__ T,
                                                          const float* __restrict__ eps,
                                                          const uint64_t* __restrict__ uA, StageAConst c,
                                                          LearnConst lc, double* __restrict__ sums,
                                                          double* __restrict__ deps) {
  __shared__ float hist[kMaxBins];
  __shared__ double part[2][kThreads / 32];
  const int n = blockIdx.z, k = blockIdx.y;
  const int nl = c.nz_layers;
  for (int i = threadIdx.x; i < lc.n_bins; i += kThreads) hist[i] = 0.f;
  __syncthreads();
  const size_t idx = (size_t)blockIdx.x * kThreads + threadIdx.x;
  double num = 0.0, den = 0.0;
  if (idx < (size_t)c.half * P) {
    const int col = (int)(idx / P), m = (int)(idx % P);
    const int mv = m < P / 2 ? m : m - P;
    const uint32_t msq = (uint32_t)(col * col + mv * mv);
    const uint64_t m64 = msq;
    const uint64_t x = uA[(size_t)n * nl + k] * m64 + c.uC * (m64 * m64) - c.uW;
    const float sn = sin_half_turns((int32_t)(x >> 32));
    const int b = radial_bin(lc, msq);
    const float e = eps[((size_t)n * nl + k) * lc.n_bins + b];
    const float den_f = fmaf(sn, sn, e);
    const float Hq = c.pref * sn / den_f;
    const float2 gq = G[((size_t)n * c.half + col) * P + m];
    const float2 tq = T[(((size_t)n * nl + k) * c.half + col) * P + m];
    const float rx = Hq * gq.x - tq.x, ry = Hq * gq.y - tq.y;
    const float mult = (col == 0 || col == P / 2) ? 1.f : 2.f;
    num = (double)(mult * (rx * rx + ry * ry));
    den = (double)(mult * (tq.x * tq.x + tq.y * tq.y));
    const float dH = -c.pref * sn / (den_f * den_f);
    atomicAdd(&hist[b], mult * 2.f * (rx * gq.x + ry * gq.y) * dH);
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_down_sync(0xffffffffu, num, o);
    den += __shfl_down_sync(0xffffffffu, den, o);
  }
  if ((threadIdx.x & 31) == 0) {
    part[0][threadIdx.x >> 5] = num;
    part[1][threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, d = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      a += part[0][w];
      d += part[1][w];
    }
    atomicAdd(&sums[0], a);
    atomicAdd(&sums[1], d);
  }
  for (int i = threadIdx.x; i < lc.n_bins; i += kThreads)
    if (hist[i] != 0.f) atomicAdd(&deps[((size_t)n * nl + k) * lc.n_bins + i], (double)hist[i]);
}

// ----------------------------------------------------------------- backward and Adam
__global__ void __launch_bounds__(kThreads) k_mlp_backward(const float* __restrict__ acts,
                                                            const double* __restrict__ deps,
                                                            const double* __restrict__ sums,
                                                            const float* __restrict__ theta, float* __restrict__ grad,
                                                            size_t rows) {
  __shared__ float w[kMlpParams];
  __shared__ float gs[kMlpParams];
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
    w[i] = theta[i];
    gs[i] = 0.f;
  }
  __syncthreads();
  const size_t row = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row < rows) {
    const float* a = acts + row * kActStride;
    const float x0 = a[0], x1 = a[1], x2 = a[2];
    const float* a1 = a + 3;
    const float* a2 = a + 3 + H;
    const float o = a[3 + 2 * H];
    const float d_eps = (float)(deps[row] / sums[1]);
    const float d_o = d_eps / (1.f + expf(-o));  // softplus' = sigmoid
    const float* W2 = w + 3 * H + H;
    const float* w3 = W2 + H * H + H;
    float* gW1 = gs;
    float* gb1 = gW1 + 3 * H;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + H * H;
    float* gw3 = gb2 + H;
    float* gb3 = gw3 + H;
    atomicAdd(gb3, d_o);
    float d_a1[H];
#pragma unroll
    for (int q = 0; q < H; ++q) d_a1[q] = 0.f;
    for (int i = 0; i < H; ++i) {
      const float h2 = fmaxf(a2[i], 0.f);
      atomicAdd(&gw3[i], d_o * h2);
      const float d_a2 = a2[i] > 0.f ? d_o * w3[i] : 0.f;
      if (d_a2 != 0.f) {
        atomicAdd(&gb2[i], d_a2);
#pragma unroll
        for (int q = 0; q < H; ++q) {
          const float h1 = fmaxf(a1[q], 0.f);
          if (h1 != 0.f) atomicAdd(&gW2[i * H + q], d_a2 * h1);
          d_a1[q] = fmaf(W2[i * H + q], d_a2, d_a1[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < H; ++q) {
      const float d = a1[q] > 0.f ? d_a1[q] : 0.f;
      if (d != 0.f) {
        atomicAdd(&gb1[q], d);
        atomicAdd(&gW1[3 * q], d * x0);
        atomicAdd(&gW1[3 * q + 1], d * x1);
        atomicAdd(&gW1[3 * q + 2], d * x2);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x)
    if (gs[i] != 0.f) atomicAdd(&grad[i], gs[i]);
}

__global__ void k_adam(float* __restrict__ theta, float* __restrict__ grad, float* __restrict__ m1,
                       float* __restrict__ m2, int step, float lr, const double* __restrict__ sums,
                       float* __restrict__ loss_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && loss_out) *loss_out = (float)(sums[0] / sums[1]);
  if (i >= kMlpParams) return;
  const float b1 = 0.9f, b2 = 0.999f;
  const float g = grad[i];
  const float m = b1 * m1[i] + (1.f - b1) * g;
  const float v = b2 * m2[i] + (1.f - b2) * g * g;
  m1[i] = m;
  m2[i] = v;
  const float mh = m / (1.f - powf(b1, (float)step));
  const float vh = v / (1.f - powf(b2, (float)step));
  theta[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
  grad[i] = 0.f;
}

__global__ void k_loss_only(const double* __restrict__ sums, float* __restrict__ loss_out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *loss_out = (float)(sums[0] / sums[1]);
}

template <int P>
cudaError_t cols_forward_p(const StageAConst& c, const LearnConst& lc, const float2* S, float2* G_out, float* pow,
                           const float2* twp, int n_dirs, cudaStream_t s) {
  constexpr int G = groups<P>();
  k_cols_forward<P><<<dim3((c.half + G - 1) / G, n_dirs), kThreads, 0, s>>>(S, G_out, pow, twp, c, lc);
  return cudaGetLastError();
}

template <int P>
cudaError_t train_loss_p(const StageAConst& c, const LearnConst& lc, const float2* G, const float2* T,
                         const float* eps, const uint64_t* uA, int n_img, double* sums, double* deps,
                         cudaStream_t s) {
  const size_t elems = (size_t)c.half * P;
  k_train_loss<P><<<dim3((unsigned)((elems + kThreads - 1) / kThreads), c.nz_layers, n_img), kThreads, 0, s>>>(
      G, T, eps, uA, c, lc, sums, deps);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cols_forward(const StageAConst& c, const LearnConst& lc, const float2* S, float2* G_out,
                                float* pow, const float2* twp, int n_dirs, cudaStream_t s) {
  if (n_dirs <= 0) return cudaSuccess;
  switch (c.P) {
    case 16: return cols_forward_p<16>(c, lc, S, G_out, pow, twp, n_dirs, s);
    case 32: return cols_forward_p<32>(c, lc, S, G_out, pow, twp, n_dirs, s);
    case 64: return cols_forward_p<64>(c, lc, S, G_out, pow, twp, n_dirs, s);
    case 128: return cols_forward_p<128>(c, lc, S, G_out, pow, twp, n_dirs, s);
    case 256: return cols_forward_p<256>(c, lc, S, G_out, pow, twp, n_dirs, s);
    case 512: return cols_forward_p<512>(c, lc, S, G_out, pow, twp, n_dirs, s);
    case 1024: return cols_forward_p<1024>(c, lc, S, G_out, pow, twp, n_dirs, s);
    case 2048: return cols_forward_p<2048>(c, lc, S, G_out, pow, twp, n_dirs, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_eps_table(const LearnConst& lc, const float* pow, const float* cnt, const float* x2tab,
                             const float* theta, float* eps, float* acts, int n_dirs, int n_layers, int dir_begin,
                             cudaStream_t s) {
  const size_t rows = (size_t)n_dirs * n_layers * lc.n_bins;
  if (rows == 0) return cudaSuccess;
  k_eps_table<<<(unsigned)((rows + kThreads - 1) / kThreads), kThreads, 0, s>>>(pow, cnt, x2tab, theta, eps, acts,
                                                                                lc, n_dirs, n_layers, dir_begin);
  return cudaGetLastError();
}

cudaError_t launch_train_step(const StageAConst& c, const LearnConst& lc, const float2* G, const float2* T,
                              const float* eps, const uint64_t* uA, const float* acts, const float* theta_dev,
                              float* theta_upd, float* grad, float* m1, float* m2, int n_img, double* sums,
                              double* deps, int step, float lr, float* loss_out, cudaStream_t s) {
  const size_t rows = (size_t)n_img * c.nz_layers * lc.n_bins;
  cudaError_t e;
  switch (c.P) {
    case 16: e = train_loss_p<16>(c, lc, G, T, eps, uA, n_img, sums, deps, s); break;
    case 32: e = train_loss_p<32>(c, lc, G, T, eps, uA, n_img, sums, deps, s); break;
    case 64: e = train_loss_p<64>(c, lc, G, T, eps, uA, n_img, sums, deps, s); break;
    case 128: e = train_loss_p<128>(c, lc, G, T, eps, uA, n_img, sums, deps, s); break;
    case 256: e = train_loss_p<256>(c, lc, G, T, eps, uA, n_img, sums, deps, s); break;
    case 512: e = train_loss_p<512>(c, lc, G, T, eps, uA, n_img, sums, deps, s); break;
    case 1024: e = train_loss_p<1024>(c, lc, G, T, eps, uA, n_img, sums, deps, s); break;
    case 2048: e = train_loss_p<2048>(c, lc, G, T, eps, uA, n_img, sums, deps, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  k_mlp_backward<<<(unsigned)((rows + kThreads - 1) / kThreads), kThreads, 0, s>>>(acts, deps, sums, theta_dev,
                                                                                   grad, rows);
  if (step > 0)
    k_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(theta_upd, grad, m1, m2, step, lr, sums, loss_out);
  else
    k_loss_only<<<1, 32, 0, s>>>(sums, loss_out);
  return cudaGetLastError();
}

}  // namespace recon
