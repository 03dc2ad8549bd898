// Register-resident mixed-radix Stockham FFT for one CTA-level group of P/8 threads.
//
// Each of the T = P/8 threads of a group holds 8 complex values, element s of thread j
// being position j + s*T of the sequence, both on input and on output (natural order).
// The passes use radix 8 while the remaining length allows, then one radix-2 or
// radix-4 pass; between passes the values go through a shared-memory buffer with a
// swizzled index (padded(): every pass's 64-bit accesses keep each half-warp on 16
// distinct bank pairs).  Twiddles come from a per-pass table in shared
// memory: the pass at sub-length Ns (radix R) stores exp(-2 pi i kb r / (Ns R)) at
// offset (Ns - 8) + kb (R - 1) + (r - 1) for kb < Ns, 1 <= r < R, so the lanes of a
// warp read addresses R - 1 apart (no bank conflicts); the table has P - 8 entries.
// INV selects the inverse (conjugate) transform, unscaled.  Every thread of the CTA (or,
// with GroupSync, of the group) must call it.
#pragma once

#include <cuda_runtime.h>

namespace recon {
namespace fft {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// The same as one packed FP32x2 instruction each (sm_100 family): each half is rounded as
// its scalar add, so the bits are those of cadd / csub (a - b as the fused b * (-1) + a,
// one rounding of the exact difference).  Used by the 16-value FFT; in the 8-value one,
// held to 80 registers, the register pairs they need measured slower.
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// t + mul_mi(u) and t - mul_mi(u), written out per component (scalar adds: a packed add
// would first have to build the swapped, negated pair)
template <bool INV>
__device__ __forceinline__ float2 add_mi(float2 t, float2 u) {
  return INV ? make_float2(t.x - u.y, t.y + u.x) : make_float2(t.x + u.y, t.y - u.x);
}
template <bool INV>
__device__ __forceinline__ float2 sub_mi(float2 t, float2 u) {
  return INV ? make_float2(t.x + u.y, t.y - u.x) : make_float2(t.x - u.y, t.y + u.x);
}

// Exchange-buffer index of element i: bits 0-3 XORed with bits 3-6, a permutation of
// every aligned block of 128 (so of [0, P) for P >= 16) under which the 64-bit writes and
// reads of every pass keep each half-warp on 16 distinct bank pairs.
__host__ __device__ constexpr int padded(int i) { return i ^ ((i >> 3) & 15); }
// Stride between the buffers of the `groups` FFT groups of a CTA: P + 16/groups (one
// entry for 16 or more groups) staggers the groups over the banks, so a fill that writes
// the groups' columns side by side does not conflict either.
__host__ __device__ constexpr int buffer_len(int P, int groups) { return P + (groups >= 16 ? 1 : 16 / groups); }
// entries of the per-pass twiddle table for length P (P >= 16)
__host__ __device__ constexpr int pass_table_len(int P) { return P - 8; }

template <bool INV>
__device__ __forceinline__ void dft2(float2* v) {
  const float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a, float2& b, float2& c, float2& d) {
  const float2 t0 = cadd(a, c), t1 = csub(a, c), t2 = cadd(b, d), t3 = mul_mi<INV>(csub(b, d));
  a = cadd(t0, t2);
  c = csub(t0, t2);
  b = cadd(t1, t3);
  d = csub(t1, t3);
}

// The length-4 DFT with packed adds (the same bits): the terms multiplied by -+i are
// combined per component, since a packed add would first have to build the swapped pair.
template <bool INV>
__device__ __forceinline__ void dft4_packed(float2& a, float2& b, float2& c, float2& d) {
  const float2 t0 = padd(a, c), t1 = psub(a, c), t2 = padd(b, d), u = psub(b, d);
  a = padd(t0, t2);
  c = psub(t0, t2);
  b = add_mi<INV>(t1, u);  // t1 + mul_mi(u)
  d = sub_mi<INV>(t1, u);
}

// dft4_packed of (a, b, mul_mi(c), d), without forming mul_mi(c)
template <bool INV>
__device__ __forceinline__ void dft4_packed_cmi(float2& a, float2& b, float2& c, float2& d) {
  const float2 t0 = add_mi<INV>(a, c), t1 = sub_mi<INV>(a, c), t2 = padd(b, d), u = psub(b, d);
  a = padd(t0, t2);
  c = psub(t0, t2);
  b = add_mi<INV>(t1, u);
  d = sub_mi<INV>(t1, u);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2* v) {
  dft4<INV>(v[0], v[1], v[2], v[3]);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  constexpr float h = 0.70710678118654752f;  // 1/sqrt(2)
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  // o_k *= W8^k, W8 = exp(-+ i pi / 4)
  o1 = INV ? make_float2(h * (o1.x - o1.y), h * (o1.x + o1.y)) : make_float2(h * (o1.x + o1.y), h * (o1.y - o1.x));
  o2 = mul_mi<INV>(o2);
  o3 = INV ? make_float2(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : make_float2(h * (o3.y - o3.x), -h * (o3.x + o3.y));
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}

// dft8 with packed adds (the same bits)
template <bool INV>
__device__ __forceinline__ void dft8_packed(float2* v) {
  constexpr float h = 0.70710678118654752f;  // 1/sqrt(2)
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4_packed<INV>(e0, e1, e2, e3);
  dft4_packed<INV>(o0, o1, o2, o3);
  o1 = INV ? make_float2(h * (o1.x - o1.y), h * (o1.x + o1.y)) : make_float2(h * (o1.x + o1.y), h * (o1.y - o1.x));
  o3 = INV ? make_float2(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : make_float2(h * (o3.y - o3.x), -h * (o3.x + o3.y));
  v[0] = padd(e0, o0);
  v[4] = psub(e0, o0);
  v[1] = padd(e1, o1);
  v[5] = psub(e1, o1);
  v[2] = add_mi<INV>(e2, o2);  // o2 times W8^2 = mul_mi
  v[6] = sub_mi<INV>(e2, o2);
  v[3] = padd(e3, o3);
  v[7] = psub(e3, o3);
}

template <int R, bool INV>
__device__ __forceinline__ void dftR(float2* v) {
  if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 4) dft4<INV>(v);
  else dft2<INV>(v);
}

// Barrier between the passes.  CtaSync: the whole CTA (needed where the exchange
// buffer aliases memory that other groups read).  GroupSync: only the group's own
// threads, for kernels whose groups each own their exchange buffer: a named barrier per
// group of 64 or more threads, __syncwarp for a group inside one warp.
struct CtaSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct GroupSync {
  int id, n;  // named barrier id (1..15) and thread count (a multiple of 32, or <= 32)
  __device__ __forceinline__ void operator()() const {
    if (n <= 32) __syncwarp();
    else asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory");
  }
};

// One Stockham pass of radix R at sub-length Ns (product of the radices before it).
template <int P, int R, int Ns, bool INV, typename Sync = CtaSync>
__device__ __forceinline__ void pass(float2 (&x)[8], float2* buf, const float2* tw, int j, Sync sync = {}) {
  constexpr int T = P / 8, NB = 8 / R, STRIDE = P / R;
  constexpr bool FIRST = Ns == 1, LAST = Ns * R == P;
  float2 v[8];
  if constexpr (FIRST) {
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
      for (int r = 0; r < R; ++r) v[q * R + r] = x[q + r * NB];
  } else {
    sync();
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
      for (int r = 0; r < R; ++r) v[q * R + r] = buf[padded(j + q * T + r * STRIDE)];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const float2* twk = tw + (Ns - 8) + ((j + q * T) & (Ns - 1)) * (R - 1) - 1;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = twk[r];
        if (INV) w.y = -w.y;
        v[q * R + r] = cmul(v[q * R + r], w);
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
    sync();
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int b = j + q * T;
      const int base = (b / Ns) * Ns * R + (b & (Ns - 1));
#pragma unroll
      for (int r = 0; r < R; ++r) buf[padded(base + r * Ns)] = v[q * R + r];
    }
  }
}

template <int P, int Ns, bool INV, typename Sync>
__device__ __forceinline__ void stockham(float2 (&x)[8], float2* buf, const float2* tw, int j, Sync sync) {
  constexpr int rem = P / Ns;
  constexpr int R = (rem % 8 == 0) ? 8 : rem;
  pass<P, R, Ns, INV, Sync>(x, buf, tw, j, sync);
  if constexpr (Ns * R < P) stockham<P, Ns * R, INV, Sync>(x, buf, tw, j, sync);
}

// Length-P FFT of the 8 values a thread holds (positions j + s*P/8), P >= 16.
template <int P, bool INV, typename Sync = CtaSync>
__device__ __forceinline__ void block_fft(float2 (&x)[8], float2* buf, const float2* tw, int j, Sync sync = {}) {
  static_assert(P >= 16 && (P & (P - 1)) == 0, "P must be a power of two >= 16");
  stockham<P, 1, INV, Sync>(x, buf, tw, j, sync);
}

}  // namespace fft
}  // namespace recon
