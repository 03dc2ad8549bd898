// Stage B for any geometry with the stack staged through the Tensor Memory Accelerator:
// the same sum as k_backproject (every voxel takes, from each direction of a block, the
// bilinear sample of its depth layer; Sec. 2's real-space gridding), but each (voxel
// tile, direction) footprint of the stack is copied into shared memory by one
// cp.async.bulk.tensor load and every gather is a shared-memory load.
//
// Pipeline (persistent CTAs, 3 per SM, each 8 consumer warps + 1 producer warp):
//  * The producer warp walks the CTA's (tile, direction) items in order, 32 at a time (one
//    per lane).  For each it forms the tile's footprint from the exact fixed-point
//    coordinates (2^-40 pixel, 2^-24 layer), i.e. the box of stack pairs x rows x layers
//    that the tile's samples can touch, and the item's box-local origin; then, item by
//    item, the lane that prepared it waits for its ring stage to be released, writes the
//    record and issues one 4D TMA load (pairs, rows, layers, direction) of the plan's
//    fixed W x H x L box, whose "full" mbarrier expects the box's bytes.  Samples outside
//    the detector read the stack's zero border or the TMA's zero fill outside the tensor
//    (pairs 0 .. nu, rows 0 .. nv+1), which is bilinear-with-zero-outside without clamps.
//  * Consumers own a 16 x 16 x 16 voxel tile: a thread keeps 16 voxels along z in
//    registers over all directions, processed two at a time with the packed FP32x2
//    instructions (__ffma2_rn / __fadd2_rn: one instruction for both voxels' adds and
//    fused multiply-adds, each component rounded as its scalar form), then writes them
//    once.  After a stage's samples a warp arrives on the stage's "empty" mbarrier.
//  * Every wait is bounded (2 s of the global timer): a wait that runs out sets bit 0 of
//    a status word in device memory and the thread stops; the producer then waits (again
//    bounded) for its copies in flight before the CTA exits.  A box that the footprint
//    does not fit (cannot happen for boxes sized by tma_box_for) sets bit 1.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "recon_internal.h"

namespace recon {
namespace {

// Compile-time tuning constants: ring depth limit, resident CTAs asked of the register
// allocator, and the odd-chunk row pitch of the staged box (bank spreading).
#ifndef RECON_TMA_MAX_STAGES
#define RECON_TMA_MAX_STAGES 3
#endif
#ifndef RECON_TMA_MIN_CTAS
#define RECON_TMA_MIN_CTAS 3
#endif
#ifndef RECON_TMA_ODD_PITCH
#define RECON_TMA_ODD_PITCH 1
#endif
// The tile is 16 x 16 x TZ voxels, TZ (voxels along z per thread) a run-time choice of
// the plan: 16 (the default, measured faster on the slab) or 8.
constexpr int kMX = 16, kMY = 16;
constexpr int kConsumerWarps = 8;
constexpr int kThreads = (kConsumerWarps + 1) * 32;
constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded waits: 2 s
constexpr long long kMargin = 1LL << 30;               // 2^-10 pixel in 2^-40 pixel units
// a waiting thread may be suspended up to this long (it resumes when the phase completes)
constexpr uint32_t kSuspendNs = 20000;

struct alignas(16) Rec {  // per item, written by the producer (64 bytes)
  float a, b;       // box-local tile-origin coordinates (+1 - box origin, pixels)
  uint32_t t;       // tile-origin depth minus the box's first layer, 2^-24 layer units
  int flags;        // bit 0: every voxel's layer lies inside [0, Nz) (no clamp); [16..]: z0
  float af0, af1, af2, bf0, bf1, bf2;  // the direction's steps per voxel (pixels)
  uint32_t ti, tj, tk;                 // and in depth (2^-24 layer units)
  int pad[3];
};
static_assert(sizeof(Rec) == 64, "Rec layout");

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity to complete; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (now_ns() - t0 > kWaitNs) return false;
  }
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ float2 lds_f2(uint32_t a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
  return v;
}
// The tap pair (Y[u], Y[u + 1]) at a shared-memory address.
template <typename ST>
__device__ __forceinline__ float2 pair_at(uint32_t a);
template <>
__device__ __forceinline__ float2 pair_at<float2>(uint32_t a) {
  return lds_f2(a);
}
template <>
__device__ __forceinline__ float2 pair_at<__nv_bfloat162>(uint32_t a) {
  const uint32_t v = lds_u32(a);
  return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xFFFF0000u));
}

__device__ __forceinline__ void set_status(unsigned int* status, unsigned int bit) {
  atomicOr(status, bit);
}

// Integer part through the FP32 adder (|x| < 2^22): x + 1.5 * 2^23, rounded down, holds
// floor(x) in its low mantissa bits.
constexpr float kMagic = 12582912.0f;
constexpr uint32_t kMagicBits = 0x4B400000u;

struct TmaArgs {
  const DirParams* dirs;
  float* vol;
  unsigned int* status;
  int dir_begin, dir_count, accumulate;
  int nx, ny, nz, gx, gy, n_tiles;
  int nz_layers;
  int W, H, L, stages;
  uint32_t stage_bytes;  // ring stride (the box rounded up to 128 bytes)
  uint32_t box_bytes;    // bytes one TMA load delivers (W H L entries)
  int stall;             // diagnostic: the producer issues nothing, so every consumer wait runs out
};

template <typename ST, bool LIN, int kMZ>
__global__ void __launch_bounds__(kThreads, RECON_TMA_MIN_CTAS) k_backproject_tma(const __grid_constant__ CUtensorMap map,
                                                                 const TmaArgs g) {
  extern __shared__ __align__(128) unsigned char smem[];
  // layout: stages (128-byte aligned) | full[S] | empty[S] | records[S]
  const int S = g.stages;
  const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t bar_full = s_base + (uint32_t)S * g.stage_bytes;
  const uint32_t bar_empty = bar_full + 8u * S;
  Rec* rec = reinterpret_cast<Rec*>(smem + (size_t)S * g.stage_bytes + 16 * S);
  __shared__ int s_abort;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(bar_full + 8u * s, 1);
      mbar_init(bar_empty + 8u * s, kConsumerWarps);
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  const int D = g.dir_count;
  const int my_tiles = blockIdx.x < g.n_tiles ? (g.n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int n_items = my_tiles * D;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == kConsumerWarps) {  // ---------------------------------------------- producer
    if (g.stall) return;
    // The warp prepares 32 items at a time, one per lane (the exact fixed-point footprint
    // of item n0 + lane), then issues them in order: lane j waits for its stage to be
    // released, writes the record and starts the copy.
    const int last = g.nz_layers - 1;
    int issued = 0;
    bool failed = false;
    int ps = 0;            // stage of the next item to issue
    uint32_t pphase = 0;   // and the parity of its use of that stage
    for (int n0 = 0; n0 < n_items && !failed; n0 += 32) {
      const int n = n0 + lane;
      Rec r;
      int x0 = 0, y0 = 0, z0 = 0, d = 0;
      if (n < n_items) {
        const int k = n / D;
        d = n - k * D;
        const int tile = blockIdx.x + k * gridDim.x;
        const int bx = tile % g.gx, by = (tile / g.gx) % g.gy, bz = tile / (g.gx * g.gy);
        const long long i0 = (long long)bx * kMX, j0 = (long long)by * kMY, k0 = (long long)bz * kMZ;
        const DirParams& p = g.dirs[g.dir_begin + d];
        const long long a = p.a[3] + p.a[0] * i0 + p.a[1] * j0 + p.a[2] * k0;
        const long long b = p.b[3] + p.b[0] * i0 + p.b[1] * j0 + p.b[2] * k0;
        const long long T =
            (long long)p.t[0] + (long long)p.t[1] * i0 + (long long)p.t[2] * j0 + (long long)p.t[3] * k0;
        // extremes over the tile's voxels (exact integer sums)
        long long alo = a, ahi = a, blo = b, bhi = b, tlo = T, thi = T;
        const long long ext[3] = {kMX - 1, kMY - 1, kMZ - 1};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const long long va = p.a[q] * ext[q], vb = p.b[q] * ext[q], vt = (long long)p.t[q + 1] * ext[q];
          if (va < 0) alo += va; else ahi += va;
          if (vb < 0) blo += vb; else bhi += vb;
          if (vt < 0) tlo += vt; else thi += vt;
        }
        // stack pairs floor(A) + 1 and rows floor(B) + 1, floor(B) + 2 over the tile (the
        // 2^-10-pixel margin covers the FP32 in-tile coordinates; one pair and one row
        // below are included as well)
        const int x_lo = (int)((alo - kMargin) >> kPixFracBits);
        const int x_hi = (int)((ahi + kMargin) >> kPixFracBits) + 1;
        x0 = x_lo & ~3;  // 16-byte aligned start for 4-byte pairs, and for 8-byte ones
        y0 = (int)((blo - kMargin) >> kPixFracBits);
        const int y_hi = (int)((bhi + kMargin) >> kPixFracBits) + 2;
        long long kl, kh;
        if (LIN) {
          kl = (tlo - (1LL << 23)) >> 24;
          kh = ((thi - (1LL << 23)) >> 24) + 1;
        } else {
          kl = tlo >> 24;
          kh = thi >> 24;
        }
        const int klc = (int)(kl < 0 ? 0 : (kl > last ? last : kl));
        const int khc = (int)(kh < 0 ? 0 : (kh > last ? last : kh));
        z0 = min(klc, g.nz_layers - g.L);
        if (x_hi - x0 >= g.W || y_hi - y0 >= g.H || khc - z0 >= g.L) set_status(g.status, 2u);
        r.a = (float)((a + (1LL << kPixFracBits) - ((long long)x0 << kPixFracBits)) >> 16) * 0x1p-24f;
        r.b = (float)((b + (1LL << kPixFracBits) - ((long long)y0 << kPixFracBits)) >> 16) * 0x1p-24f;
        r.t = (uint32_t)(T - ((long long)z0 << 24));
        r.flags = ((kl >= 0 && kh <= last) ? 1 : 0) | (z0 << 16);
        r.af0 = p.af[0];
        r.af1 = p.af[1];
        r.af2 = p.af[2];
        r.bf0 = p.bf[0];
        r.bf1 = p.bf[1];
        r.bf2 = p.bf[2];
        r.ti = (uint32_t)p.t[1];
        r.tj = (uint32_t)p.t[2];
        r.tk = (uint32_t)p.t[3];
        r.pad[0] = r.pad[1] = r.pad[2] = 0;
      }
      const int cnt = min(32, n_items - n0);
      for (int j = 0; j < cnt; ++j) {
        int bad = 0;
        if (lane == j) {
          if (*(volatile int*)&s_abort || !mbar_wait(bar_empty + 8u * ps, pphase ^ 1u)) {
            bad = 1;
          } else {
            rec[ps] = r;
            mbar_expect_tx(bar_full + 8u * ps, g.box_bytes);
            tma_load_4d(s_base + (uint32_t)ps * g.stage_bytes, &map, x0, y0, z0, d, bar_full + 8u * ps);
          }
        }
        if (__shfl_sync(0xffffffffu, bad, j)) {
          failed = true;
          break;
        }
        ++issued;
        if (++ps == S) {
          ps = 0;
          pphase ^= 1u;
        }
      }
    }
    if (failed && lane == 0) {
      set_status(g.status, 1u);
      *(volatile int*)&s_abort = 1;
    }
    // copies still in flight land before the CTA's shared memory is released
    if (lane == 0)
      for (int n = issued > S ? issued - S : 0; n < issued; ++n)
        mbar_wait(bar_full + 8u * (n % S), (uint32_t)(n / S) & 1u);
    return;
  }

  // ------------------------------------------------------------------------ consumers
  // a warp covers an 8 x 4 patch of the tile's 16 x 16 voxel columns
  const int tx = (warp & 1) * 8 + (lane & 7), ty = (warp >> 1) * 4 + (lane >> 3);
  const float ftx = (float)tx, fty = (float)ty;
  constexpr uint32_t es = sizeof(ST);
  const uint32_t Wb = (uint32_t)g.W * es, HWb = (uint32_t)g.H * Wb;
  // the magic-number bits of the integer column and row, folded into the stage base
  const uint32_t kfold = kMagicBits * es + kMagicBits * Wb;
  const int last = g.nz_layers - 1;
  const float2 kM2 = make_float2(kMagic, kMagic), kMm2 = make_float2(-kMagic, -kMagic);
  const float2 kNeg = make_float2(-1.f, -1.f);
  float2 acc[kMZ / 2];
#pragma unroll
  for (int q = 0; q < kMZ / 2; ++q) acc[q] = make_float2(0.f, 0.f);

  // item n = k D + d sits in stage s = n mod S with phase parity floor(n / S) mod 2; all
  // four are stepped incrementally (no integer division per item)
  int s = 0, d = 0, tile = blockIdx.x;
  uint32_t parity = 0;
  for (int n = 0; n < n_items; ++n) {
    const bool ok = mbar_wait(bar_full + 8u * s, parity) && !*(volatile int*)&s_abort;
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) {
        set_status(g.status, 1u);
        *(volatile int*)&s_abort = 1;
      }
      return;
    }
    const Rec r = rec[s];
    const uint32_t base = s_base + (uint32_t)s * g.stage_bytes - kfold;
    const int z0 = r.flags >> 16, lo = -z0, hi = last - z0;
    const bool inside = (r.flags & 1) != 0;
    const float A = fmaf(r.af0, ftx, fmaf(r.af1, fty, r.a));
    const float B = fmaf(r.bf0, ftx, fmaf(r.bf1, fty, r.b));
    float2 A2 = make_float2(A, A + r.af2), B2 = make_float2(B, B + r.bf2);
    const float2 dA2 = make_float2(2.f * r.af2, 2.f * r.af2), dB2 = make_float2(2.f * r.bf2, 2.f * r.bf2);
    uint32_t t = r.t + r.ti * (uint32_t)tx + r.tj * (uint32_t)ty;
#pragma unroll
    for (int q = 0; q < kMZ / 2; ++q) {
      // voxels 2q and 2q + 1 of the thread's run, packed in the two halves of each float2
      // the magic-number add rounded down holds floor(A) in its low mantissa bits; the
      // box-local coordinate A is the pair index plus the weight on its right tap
      const float2 tA = __fadd2_rd(A2, kM2), tB = __fadd2_rd(B2, kM2);
      const float2 fA = __ffma2_rn(__fadd2_rn(tA, kMm2), kNeg, A2);  // A - floor(A)
      const float2 fB = __ffma2_rn(__fadd2_rn(tB, kMm2), kNeg, B2);
      const uint32_t rc0 = __float_as_uint(tA.x) * es + __float_as_uint(tB.x) * Wb + base;
      const uint32_t rc1 = __float_as_uint(tA.y) * es + __float_as_uint(tB.y) * Wb + base;
      const uint32_t t0 = t, t1 = t + r.tk;
      if constexpr (LIN) {
        float w[2];
        uint32_t a0[2], a1[2];
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const int32_t tp = (int32_t)(v ? t1 : t0) - (1 << 23);
          const int k0r = tp >> 24;
          const bool outer = k0r < lo || k0r >= hi;
          const int kk0 = min(max(k0r, lo), hi);
          const int kk1 = min(kk0 + 1, hi);
          w[v] = outer ? 0.f : (float)(tp & 0xFFFFFF) * 0x1p-24f;
          a0[v] = (v ? rc1 : rc0) + (uint32_t)kk0 * HWb;
          a1[v] = (v ? rc1 : rc0) + (uint32_t)kk1 * HWb;
        }
        const float2 p00 = pair_at<ST>(a0[0]), p01 = pair_at<ST>(a0[0] + Wb);
        const float2 p10 = pair_at<ST>(a0[1]), p11 = pair_at<ST>(a0[1] + Wb);
        const float2 s00 = pair_at<ST>(a1[0]), s01 = pair_at<ST>(a1[0] + Wb);
        const float2 s10 = pair_at<ST>(a1[1]), s11 = pair_at<ST>(a1[1] + Wb);
        const float2 X0 = make_float2(p00.x, p10.x), Y0 = make_float2(p00.y, p10.y);
        const float2 X1 = make_float2(p01.x, p11.x), Y1 = make_float2(p01.y, p11.y);
        const float2 U0 = make_float2(s00.x, s10.x), V0 = make_float2(s00.y, s10.y);
        const float2 U1 = make_float2(s01.x, s11.x), V1 = make_float2(s01.y, s11.y);
        const float2 top0 = __ffma2_rn(fA, __ffma2_rn(X0, kNeg, Y0), X0);
        const float2 bot0 = __ffma2_rn(fA, __ffma2_rn(X1, kNeg, Y1), X1);
        const float2 top1 = __ffma2_rn(fA, __ffma2_rn(U0, kNeg, V0), U0);
        const float2 bot1 = __ffma2_rn(fA, __ffma2_rn(U1, kNeg, V1), U1);
        const float2 v0 = __ffma2_rn(fB, __ffma2_rn(top0, kNeg, bot0), top0);
        const float2 v1 = __ffma2_rn(fB, __ffma2_rn(top1, kNeg, bot1), top1);
        acc[q] = __fadd2_rn(acc[q], __ffma2_rn(make_float2(w[0], w[1]), __ffma2_rn(v0, kNeg, v1), v0));
      } else {
        int l0 = (int32_t)t0 >> 24, l1 = (int32_t)t1 >> 24;
        if (!inside) {
          l0 = min(max(l0, lo), hi);
          l1 = min(max(l1, lo), hi);
        }
        const uint32_t a0 = rc0 + (uint32_t)l0 * HWb, a1 = rc1 + (uint32_t)l1 * HWb;
        const float2 p00 = pair_at<ST>(a0), p01 = pair_at<ST>(a0 + Wb);
        const float2 p10 = pair_at<ST>(a1), p11 = pair_at<ST>(a1 + Wb);
        const float2 X0 = make_float2(p00.x, p10.x), Y0 = make_float2(p00.y, p10.y);
        const float2 X1 = make_float2(p01.x, p11.x), Y1 = make_float2(p01.y, p11.y);
        const float2 top = __ffma2_rn(fA, __ffma2_rn(X0, kNeg, Y0), X0);
        const float2 bot = __ffma2_rn(fA, __ffma2_rn(X1, kNeg, Y1), X1);
        acc[q] = __fadd2_rn(acc[q], __ffma2_rn(fB, __ffma2_rn(top, kNeg, bot), top));
      }
      A2 = __fadd2_rn(A2, dA2);
      B2 = __fadd2_rn(B2, dB2);
      t += 2u * r.tk;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(bar_empty + 8u * s);
    if (++s == S) {
      s = 0;
      parity ^= 1u;
    }
    if (++d == D) {  // the tile's last direction: write its voxels once
      d = 0;
      const int bx = tile % g.gx, by = (tile / g.gx) % g.gy, bz = tile / (g.gx * g.gy);
      tile += gridDim.x;
      const int i = bx * kMX + tx, j = by * kMY + ty;
      if (i < g.nx && j < g.ny) {
#pragma unroll
        for (int q = 0; q < kMZ; ++q) {
          const int kk = bz * kMZ + q;
          if (kk < g.nz) {
            float* v = g.vol + ((size_t)kk * g.ny + j) * g.nx + i;
            const float x = (q & 1) ? acc[q >> 1].y : acc[q >> 1].x;
            *v = g.accumulate ? *v + x : x;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kMZ / 2; ++q) acc[q] = make_float2(0.f, 0.f);
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

template <typename ST, bool LIN, int kMZ>
cudaError_t launch_tma_t(const BackprojConst& c, const TmaBox& box, const DirParams* dirs, const void* stack,
                         int dir_begin, int dir_count, float* volume, int accumulate, unsigned int* status,
                         cudaStream_t stream, int stall = 0) {
  static_assert(kMZ == 8 || kMZ == 16, "tile depth 8 or 16");
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  constexpr size_t es = sizeof(ST);
  // 4D view of the block's stacks: pairs 0 .. nu of a row, rows 0 .. nv+1, layers, directions
  const cuuint64_t dims[4] = {(cuuint64_t)c.nu + 1, (cuuint64_t)c.nv + 2, (cuuint64_t)c.nz_layers,
                              (cuuint64_t)dir_count};
  const cuuint64_t strides[3] = {(cuuint64_t)c.su * es, (cuuint64_t)c.layer_elems * es,
                                 (cuuint64_t)c.layer_elems * c.nz_layers * es};
  const cuuint32_t bdim[4] = {(cuuint32_t)box.W, (cuuint32_t)box.H, (cuuint32_t)box.L, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUtensorMap map;
  const CUresult r = enc(&map, es == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_INT64, 4,
                         const_cast<void*>(stack), dims, strides, bdim, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  TmaArgs g;
  g.dirs = dirs;
  g.vol = volume;
  g.status = status;
  g.dir_begin = dir_begin;
  g.dir_count = dir_count;
  g.accumulate = accumulate;
  g.nx = c.nx;
  g.ny = c.ny;
  g.nz = c.nz;
  g.gx = (c.nx + kMX - 1) / kMX;
  g.gy = (c.ny + kMY - 1) / kMY;
  const long long tiles = (long long)g.gx * g.gy * ((c.nz + kMZ - 1) / kMZ);
  if (tiles > INT32_MAX / 2) return cudaErrorInvalidValue;
  g.n_tiles = (int)tiles;
  g.nz_layers = c.nz_layers;
  g.W = box.W;
  g.H = box.H;
  g.L = box.L;
  g.stages = box.stages;
  g.stage_bytes = (uint32_t)box.stage_bytes;
  g.box_bytes = (uint32_t)((size_t)box.W * box.H * box.L * es);
  g.stall = stall;
  const size_t smem = (size_t)box.stages * (box.stage_bytes + 16 + sizeof(Rec));
  cudaError_t e = cudaFuncSetAttribute(k_backproject_tma<ST, LIN, kMZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backproject_tma<ST, LIN, kMZ>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long ctas = (long long)device_sm_count() * per_sm;
  const unsigned grid = (unsigned)(ctas < tiles ? ctas : tiles);
  k_backproject_tma<ST, LIN, kMZ><<<grid, kThreads, smem, stream>>>(map, g);
  return cudaGetLastError();
}

template <int kMZ>
cudaError_t launch_tz(const BackprojConst& c, const TmaBox& box, const DirParams* dirs, const void* stack, int dir_begin,
                      int dir_count, float* volume, int accumulate, unsigned int* status, cudaStream_t stream) {
  if (c.stack_bf16)
    return c.layer_linear ? launch_tma_t<__nv_bfloat162, true, kMZ>(c, box, dirs, stack, dir_begin, dir_count, volume,
                                                                    accumulate, status, stream)
                          : launch_tma_t<__nv_bfloat162, false, kMZ>(c, box, dirs, stack, dir_begin, dir_count,
                                                                     volume, accumulate, status, stream);
  return c.layer_linear ? launch_tma_t<float2, true, kMZ>(c, box, dirs, stack, dir_begin, dir_count, volume,
                                                          accumulate, status, stream)
                        : launch_tma_t<float2, false, kMZ>(c, box, dirs, stack, dir_begin, dir_count, volume,
                                                           accumulate, status, stream);
}

}  // namespace

TmaBox tma_box_for(const BackprojConst& c, const DirParams* dirs, int n_dirs, int tile_z) {
  TmaBox b{};
  if (tile_z != 8 && tile_z != 16) return b;  // ok = 0
  b.tile_z = tile_z;
  const long long ext[3] = {kMX - 1, kMY - 1, tile_z - 1};
  long long W = 4, H = 2, L = 1;
  for (int n = 0; n < n_dirs; ++n) {
    const DirParams& p = dirs[n];
    long long ea = 0, eb = 0, et = 0;
    for (int q = 0; q < 3; ++q) {
      ea += (p.a[q] < 0 ? -p.a[q] : p.a[q]) * ext[q];
      eb += (p.b[q] < 0 ? -p.b[q] : p.b[q]) * ext[q];
      et += (long long)(p.t[q + 1] < 0 ? -(long long)p.t[q + 1] : (long long)p.t[q + 1]) * ext[q];
    }
    // pairs: floor(A_max + m) + 1 - floor(A_min - m) + 1, plus up to 3 for the aligned start;
    // rows: floor(B_max + m) + 2 - floor(B_min - m) + 1; layers: the span of the depth plus
    // one (nearest) or two (blend)
    W = std::max(W, ((ea + 2 * kMargin) >> kPixFracBits) + 6);
    H = std::max(H, ((eb + 2 * kMargin) >> kPixFracBits) + 4);
    L = std::max(L, (et >> 24) + (c.layer_linear ? 3 : 2));
  }
  W = (W + 3) & ~3LL;
  const size_t es = c.stack_bf16 ? 4 : 8;
#if RECON_TMA_ODD_PITCH
  // a row pitch of an odd number of 16-byte chunks (W * es / 16 odd): consecutive rows of a
  // warp's footprint start 4 banks apart instead of on the same bank
  while (((W * (long long)es / 16) & 1) == 0) W += 16 / (long long)es;
#endif
  L = std::min<long long>(L, c.nz_layers);
  b.W = (int)std::min<long long>(W, 1 << 20);
  b.H = (int)std::min<long long>(H, 1 << 20);
  b.L = (int)L;
  const size_t box_bytes = (size_t)b.W * b.H * b.L * es;
  b.stage_bytes = (box_bytes + 127) & ~(size_t)127;
  // ring depth: up to RECON_TMA_MAX_STAGES stages within 100 KB; 2 (copy and gathers
  // overlap) if two fit in 200 KB, else 1
  const size_t st = b.stage_bytes ? (size_t)(100 * 1024) / b.stage_bytes : 0;
  b.stages = (int)std::min<size_t>(RECON_TMA_MAX_STAGES, st);
  if (b.stages < 2) b.stages = 2 * (b.stage_bytes + 16 + sizeof(Rec)) <= (size_t)200 * 1024 ? 2 : 1;
  const size_t smem = (size_t)b.stages * (b.stage_bytes + 16 + sizeof(Rec));
  b.ok = W <= 256 && H <= 256 && L <= 256 && smem <= 200 * 1024;
  return b;
}

cudaError_t launch_backproject_tma(const BackprojConst& c, const TmaBox& box, const DirParams* dirs, const void* stack,
                                   int dir_begin, int dir_count, float* volume, int accumulate, unsigned int* status,
                                   cudaStream_t stream) {
  if (dir_count <= 0 || c.nx <= 0 || c.ny <= 0 || c.nz <= 0) return cudaSuccess;
  if (!box.ok) return cudaErrorInvalidValue;
  if (box.tile_z == 8) return launch_tz<8>(c, box, dirs, stack, dir_begin, dir_count, volume, accumulate, status, stream);
  return launch_tz<16>(c, box, dirs, stack, dir_begin, dir_count, volume, accumulate, status, stream);
}

cudaError_t launch_tma_wait_probe(void* buf, size_t buf_bytes, unsigned int* status, cudaStream_t stream) {
  // one tile of one direction over a 16 x 16 detector with one layer (stack
  // [1][18][20] bf16 pairs = 1440 bytes, 16-byte strides); the producer issues no copy
  BackprojConst c{};
  c.nx = c.ny = 16;
  c.nz = 8;
  c.nu = c.nv = 16;
  c.nz_layers = 1;
  c.su = 20;
  c.layer_elems = 18 * 20;
  c.stack_bf16 = 1;
  if (!buf || buf_bytes < 2048 + 16 * 16 * 8 * sizeof(float) || ((uintptr_t)buf & 255) != 0)
    return cudaErrorInvalidValue;
  TmaBox b{};
  b.W = 8;
  b.H = 4;
  b.L = 1;
  b.stages = 2;
  b.stage_bytes = 128;
  b.ok = 1;
  float* vol = reinterpret_cast<float*>(static_cast<char*>(buf) + 2048);
  b.tile_z = 16;
  return launch_tma_t<__nv_bfloat162, false, 16>(c, b, nullptr, buf, 0, 1, vol, 0, status, stream, 1);
}

}  // namespace recon
