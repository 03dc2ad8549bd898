// Register-resident mixed-radix Stockham FFT with 16 values per thread, for the large
// transforms (P >= 256) of stage A.
//
// Each of the T = P/16 threads of a group holds 16 complex values, element s of thread j
// being position j + s*T of the sequence, on input and on output (natural order).  The
// passes use radix 16 while the remaining length allows, then one radix-8, -4 or -2 pass,
// so a length-2048 transform takes three passes and two shared-memory exchanges (the
// 8-value transform of fft_reg.cuh takes four passes and three exchanges).
//
// Exchange buffers are padded by one entry per 16 (index i -> i + i/16, length P + P/16):
// every pass's 64-bit stores (stride Ns) and loads (consecutive) then keep each half-warp
// on 16 distinct bank pairs, and since all in-pass offsets are multiples of 16 the padded
// address is a per-thread base plus a compile-time constant.
//
// Twiddles: the pass at sub-length Ns (radix R, Ns >= 16) reads exp(-2 pi i kb r / (Ns R))
// at offset (Ns - 16) + kb (R - 1) + (r - 1), kb < Ns, 1 <= r < R; the table has P - 16
// entries (the per-pass entry counts Ns (R - 1) telescope).  Lanes with consecutive kb read
// addresses R - 1 apart, an odd stride, so the loads are free of bank conflicts.
//
// INV selects the inverse (conjugate) transform, unscaled.
#pragma once

#include <cuda_runtime.h>

#include "fft_reg.cuh"

namespace recon {
namespace fft16 {

using fft::cadd;
using fft::cmul;
using fft::csub;

__host__ __device__ constexpr int pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int buffer_len(int P) { return P + P / 16; }
__host__ __device__ constexpr int table_len(int P) { return P - 16; }

// multiply by the constant (c, s): (x c - y s, x s + y c)
__device__ __forceinline__ float2 cmulc(float2 a, float c, float s) {
  return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
}

// Length-16 DFT of v[0..15] in place (4 x 4 decomposition): for a = 0..3 a length-4 DFT of
// v[a], v[a+4], v[a+8], v[a+12]; multiply the result k1 of column a by W16^(a k1); then for
// k1 = 0..3 a length-4 DFT over a, whose output k2 is X[k1 + 4 k2].
template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
  constexpr float c1 = 0.92387953251128676f;  // cos(pi/8)
  constexpr float s1 = 0.38268343236508977f;  // sin(pi/8)
  constexpr float h = 0.70710678118654752f;   // 1/sqrt(2)
  constexpr float sg = INV ? 1.f : -1.f;      // sign of the twiddle angle
#pragma unroll
  for (int a = 0; a < 4; ++a) fft::dft4_packed<INV>(v[a], v[a + 4], v[a + 8], v[a + 12]);
  // column a now holds k1 = 0..3 at v[a], v[a+4], v[a+8], v[a+12]
  v[1 + 4] = cmulc(v[1 + 4], c1, sg * s1);     // W^1
  v[1 + 8] = cmulc(v[1 + 8], h, sg * h);       // W^2
  v[1 + 12] = cmulc(v[1 + 12], s1, sg * c1);   // W^3
  v[2 + 4] = cmulc(v[2 + 4], h, sg * h);       // W^2
  // W^4 = mul_mi on v[2 + 8], applied inside the k1 = 2 length-4 DFT below
  v[2 + 12] = cmulc(v[2 + 12], -h, sg * h);    // W^6
  v[3 + 4] = cmulc(v[3 + 4], s1, sg * c1);     // W^3
  v[3 + 8] = cmulc(v[3 + 8], -h, sg * h);      // W^6
  v[3 + 12] = cmulc(v[3 + 12], -c1, -sg * s1); // W^9
  fft::dft4_packed<INV>(v[0], v[1], v[2], v[3]);
  fft::dft4_packed<INV>(v[4], v[5], v[6], v[7]);
  fft::dft4_packed_cmi<INV>(v[8], v[9], v[10], v[11]);
  fft::dft4_packed<INV>(v[12], v[13], v[14], v[15]);
  // v[4 k1 + k2] holds X[k1 + 4 k2]: transpose the 4 x 4 index
  float2 t[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[4 * k1 + k2];
}

template <int R, bool INV>
__device__ __forceinline__ void dftR(float2* v) {
  if constexpr (R == 16) dft16<INV>(v);
  else if constexpr (R == 8) fft::dft8_packed<INV>(v);
  else if constexpr (R == 4) fft::dft4_packed<INV>(v[0], v[1], v[2], v[3]);
  else fft::dftR<R, INV>(v);
}

// One Stockham pass of radix R at sub-length Ns.  jp = pad(j) for the group's thread j.
// A buffer `out` receives this pass's values (unless it is the last), `in` holds the
// previous pass's (unless it is the first); `sync_in` runs before reading `in`,
// `sync_out` before writing `out` (both no-ops when the caller double-buffers).
// Twiddles of one radix-16 or radix-8 column from a few table entries: w[r] = W^r for
// r = 1..R-1 given W^1, W^4 (and W^8, W^12 for R = 16), each other power one or two complex
// products away (W^2 = (W^1)^2, W^3 = W^2 W^1, W^(4a+b) = W^(4a) W^b), so its rounding error
// stays within a few units in the last place.  Four (R = 16) or two (R = 8) shared-memory loads
// instead of R - 1.
template <int R>
__device__ __forceinline__ void twiddle_powers(const float2* twk, bool inv, float2 (&w)[16]) {
  float2 w1 = twk[1], w4 = twk[4];
  float2 w8, w12;
  if constexpr (R == 16) {
    w8 = twk[8];
    w12 = twk[12];
  }
  if (inv) {  // conj of a product = product of the conjs
    w1.y = -w1.y;
    w4.y = -w4.y;
    if constexpr (R == 16) {
      w8.y = -w8.y;
      w12.y = -w12.y;
    }
  }
  const float2 w2 = make_float2(fmaf(w1.x, w1.x, -w1.y * w1.y), 2.f * w1.x * w1.y);
  const float2 w3 = cmul(w2, w1);
  w[1] = w1;
  w[2] = w2;
  w[3] = w3;
  w[4] = w4;
  w[5] = cmul(w4, w1);
  w[6] = cmul(w4, w2);
  w[7] = cmul(w4, w3);
  if constexpr (R == 16) {
    w[8] = w8;
    w[9] = cmul(w8, w1);
    w[10] = cmul(w8, w2);
    w[11] = cmul(w8, w3);
    w[12] = w12;
    w[13] = cmul(w12, w1);
    w[14] = cmul(w12, w2);
    w[15] = cmul(w12, w3);
  }
}

// TWR: the inter-pass twiddles from twiddle_powers (for kernels whose shared-memory queue,
// not their arithmetic, is the limit) instead of one table load each.
template <int P, int R, int Ns, bool INV, typename Sync, bool TWR = false>
__device__ __forceinline__ void pass(float2 (&x)[16], const float2* in, float2* out, const float2* tw, int j, int jp,
                                     Sync sync_in, bool do_sync_out) {
  constexpr int T = P / 16, NB = 16 / R, STRIDE = P / R;
  constexpr bool FIRST = Ns == 1, LAST = Ns * R == P;
  static_assert(T % 16 == 0, "16-value FFT needs P >= 256");
  float2 v[16];
  if constexpr (FIRST) {
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
      for (int r = 0; r < R; ++r) v[q * R + r] = x[q + r * NB];
  } else {
    sync_in();
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
      for (int r = 0; r < R; ++r) v[q * R + r] = in[jp + pad(q * T + r * STRIDE)];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const float2* twk = tw + (Ns - 16) + ((j + q * T) & (Ns - 1)) * (R - 1) - 1;
      if constexpr (TWR && (R == 16 || R == 8)) {
        float2 w[16];
        twiddle_powers<R>(twk, INV, w);
#pragma unroll
        for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], w[r]);
      } else {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = twk[r];
          if (INV) w.y = -w.y;
          v[q * R + r] = cmul(v[q * R + r], w);
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NB; ++q) dftR<R, INV>(v + q * R);
  if constexpr (LAST) {
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
      for (int r = 0; r < R; ++r) x[q + r * NB] = v[q * R + r];
  } else {
    if (do_sync_out) sync_in();
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int b = j + q * T;
      const int base = (b / Ns) * Ns * R + (b & (Ns - 1));
      const int pb = pad(base);
      // pad(base + r Ns) = pad(base) + r Ns + (r Ns) / 16: base is a multiple of 16 when
      // Ns = 1 (r < 16), and r Ns is one when Ns >= 16
#pragma unroll
      for (int r = 0; r < R; ++r) out[pb + r * Ns + ((r * Ns) >> 4)] = v[q * R + r];
    }
  }
}

template <int P, int Ns, bool INV, typename Sync>
__device__ __forceinline__ void stockham_db(float2 (&x)[16], float2* buf0, float2* buf1, const float2* tw, int j,
                                            int jp, Sync sync) {
  constexpr int rem = P / Ns;
  constexpr int R = (rem % 16 == 0) ? 16 : rem;
  // pass p reads buffer (p - 1) % 2 and writes buffer p % 2
  constexpr int p = Ns == 1 ? 0 : (Ns == 16 ? 1 : (Ns == 256 ? 2 : 3));
  float2* in = (p % 2 == 1) ? buf0 : buf1;
  float2* out = (p % 2 == 0) ? buf0 : buf1;
  // Double buffering: a pass writes the buffer the previous pass did not read from, so
  // only the barrier before each read is needed -- except that the first pass of a
  // transform writes buf0, which the second pass of the previous transform read: the
  // caller's barrier before the previous transform's last pass covers that (every thread
  // has finished its second-pass reads of buf0 before anyone passes it).
  pass<P, R, Ns, INV, Sync>(x, in, out, tw, j, jp, sync, false);
  if constexpr (Ns * R < P) stockham_db<P, Ns * R, INV, Sync>(x, buf0, buf1, tw, j, jp, sync);
}

// Length-P FFT of the 16 values a thread holds, with two exchange buffers of
// buffer_len(P) entries.  Valid when P/16 has at most three radix-16 or final passes
// (P <= 4096) so that no pass reads the buffer it writes.  The first pass writes buf0
// without a barrier: the caller must make sure no thread of the group still reads buf0
// from an earlier use (consecutive calls are safe when the transform has three passes).
template <int P, bool INV, typename Sync>
__device__ __forceinline__ void group_fft_db(float2 (&x)[16], float2* buf0, float2* buf1, const float2* tw, int j,
                                             Sync sync) {
  static_assert(P >= 256 && P <= 4096 && (P & (P - 1)) == 0, "16-value FFT: P in [256, 4096], a power of two");
  stockham_db<P, 1, INV, Sync>(x, buf0, buf1, tw, j, pad(j), sync);
}

// Single-buffer variant: a barrier before every exchange read and write (for kernels whose
// buffer aliases other data).
template <int P, int Ns, bool INV, typename Sync, bool TWR>
__device__ __forceinline__ void stockham_sb(float2 (&x)[16], float2* buf, const float2* tw, int j, int jp,
                                            Sync sync) {
  constexpr int rem = P / Ns;
  constexpr int R = (rem % 16 == 0) ? 16 : rem;
  pass<P, R, Ns, INV, Sync, TWR>(x, buf, buf, tw, j, jp, sync, true);
  if constexpr (Ns * R < P) stockham_sb<P, Ns * R, INV, Sync, TWR>(x, buf, tw, j, jp, sync);
}

template <int P, bool INV, typename Sync, bool TWR = false>
__device__ __forceinline__ void group_fft_sb(float2 (&x)[16], float2* buf, const float2* tw, int j, Sync sync) {
  static_assert(P >= 256 && (P & (P - 1)) == 0, "16-value FFT: P >= 256, a power of two");
  stockham_sb<P, 1, INV, Sync, TWR>(x, buf, tw, j, pad(j), sync);
}

}  // namespace fft16
}  // namespace recon
