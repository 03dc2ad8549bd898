// Stage B of the layered UTR path: every voxel takes, from each direction of a block,
// the bilinear sample of the layer that contains its depth and sums over directions
// (the real-space counterpart of gridding each image onto its Ewald patch, Sec. 2).
//
// A CTA owns a 32 x 8 x 8 voxel tile; a thread owns an 8-voxel run along z and keeps
// its sums in registers across the whole direction block, then reads-modifies-writes
// the volume once.  Coordinates: per (tile, direction) the tile-origin pixel
// coordinate is an exact integer sum of 2^-40-pixel fixed-point coefficients, split into
// an integer and an FP32 fraction, so the FP32 arithmetic inside the tile works on small
// numbers (error ~1e-6 pixel at any detector size).  The depth coordinate is an exact 2^-24 fixed-point integer sum, so
// the layer decision does not depend on the traversal order.  Out-of-detector taps
// read the stack's zero border (rows -1 and nv, pairs holding the columns -1 and nu):
// the integer tap is clamped to [-1, n-1] and the weight saturated to [0, 1], which
// gives exactly bilinear-with-zero-outside.  Each stack entry is the tap pair
// (Y[u], Y[u+1]), so a bilinear row is one load.
#include <cuda_bf16.h>

#include "recon_internal.h"

namespace recon {
namespace {

constexpr int kTX = kGenTile[0], kTY = kGenTile[1], kTZ = kGenTile[2];
static_assert(kTX == 32 && kTY == 8, "the warp patches (8 x 4, 16 x 2, 32 x 1) tile 32 x 8 voxel columns");

// Integer pixel (floor) and FP32 fraction of a coordinate in 2^-40 pixel units.
__device__ __forceinline__ int pix_floor(long long x) { return (int)(x >> kPixFracBits); }
__device__ __forceinline__ float pix_frac(long long x) {
  return (float)((x & ((1LL << kPixFracBits) - 1)) >> (kPixFracBits - 24)) * 0x1p-24f;  // exact
}

struct TileDir {  // per (tile, direction), 64 bytes in shared memory
  float fa, fb;   // fractional tile-origin coordinate minus 0.5
  int ia, ib;     // integer tile-origin coordinate
  uint32_t t;     // depth at the tile origin, 2^-24 layer units
  float af0, af1, af2, bf0, bf1, bf2;
  uint32_t ti, tj, tk;
  int pad[2];
};
static_assert(sizeof(TileDir) == 64, "TileDir layout");

// A stack entry is the horizontal tap pair (Y[u], Y[u + 1]) (one 8-byte or 4-byte load).
__device__ __forceinline__ float2 stack_pair(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 stack_pair(const __nv_bfloat162* p) { return __bfloat1622float2(__ldg(p)); }
// Round-to-nearest integer of |x| < 2^22 through the FP32 adder: x + 1.5*2^23 holds
// rint(x) in its low mantissa bits.
constexpr float kMagic = 12582912.0f;
constexpr int kMagicBits = 0x4B400000;

// One direction's samples for a thread's run of kTZ voxels along z.  CLAMP: the taps are
// clamped to the zero border and the weights saturated (any tile); without it the tile
// is known to lie inside the detector and the layer range.  LIN: blend the two layers
// whose centres bracket the depth (layer k centred at k + 1/2 in layer units: t' = t - 1/2,
// k0 = floor t', weight t' - k0 on k0 + 1, the outer layer alone beyond the outer
// centres) instead of taking the layer that contains it.
template <typename ST, bool CLAMP, bool LIN>
__device__ __forceinline__ void generic_run(const TileDir& td, const ST* __restrict__ base, const BackprojConst& c,
                                            float ftx, float fty, int tx, int ty, float (&acc)[kTZ]) {
  float ap = fmaf(td.af0, ftx, fmaf(td.af1, fty, td.fa));
  float bp = fmaf(td.bf0, ftx, fmaf(td.bf1, fty, td.fb));
  uint32_t t = td.t + td.ti * (uint32_t)tx + td.tj * (uint32_t)ty;
  const float loa = (float)(-1 - td.ia), hia = (float)(c.nu - 1 - td.ia);
  const float lob = (float)(-1 - td.ib), hib = (float)(c.nv - 1 - td.ib);
  const int last_layer = c.nz_layers - 1;
  const int LE = (int)c.layer_elems;
#pragma unroll
  for (int z = 0; z < kTZ; ++z) {
    const float ta = (CLAMP ? fminf(fmaxf(ap, loa), hia) : ap) + kMagic;
    const float tb = (CLAMP ? fminf(fmaxf(bp, lob), hib) : bp) + kMagic;
    const int ra = __float_as_int(ta) - kMagicBits;
    const int rb = __float_as_int(tb) - kMagicBits;
    const float fa = CLAMP ? __saturatef(ap - (ta - kMagic) + 0.5f) : ap - (ta - kMagic) + 0.5f;
    const float fb = CLAMP ? __saturatef(bp - (tb - kMagic) + 0.5f) : bp - (tb - kMagic) + 0.5f;
    // one direction's stack holds at most 96 x 1026 x 1025 entries: 32-bit offsets
    if constexpr (LIN) {
      const int32_t tp = (int32_t)t - (1 << 23);
      const int k0r = tp >> 24;
      const bool outer = tp < 0 || k0r >= last_layer;
      const int k0 = tp < 0 ? 0 : min(k0r, last_layer);
      const float w = outer ? 0.f : (float)(tp & 0xFFFFFF) * 0x1p-24f;  // exact 24-bit fraction
      const int k1 = min(k0 + 1, last_layer);
      const ST* p0 = base + (k0 * LE + rb * c.su + ra);
      const ST* p1 = p0 + (k1 - k0) * LE;
      const float2 r0 = stack_pair(p0), r1 = stack_pair(p0 + c.su);
      const float2 s0 = stack_pair(p1), s1 = stack_pair(p1 + c.su);
      const float top0 = fmaf(fa, r0.y - r0.x, r0.x), bot0 = fmaf(fa, r1.y - r1.x, r1.x);
      const float top1 = fmaf(fa, s0.y - s0.x, s0.x), bot1 = fmaf(fa, s1.y - s1.x, s1.x);
      const float v0 = fmaf(fb, bot0 - top0, top0), v1 = fmaf(fb, bot1 - top1, top1);
      acc[z] += fmaf(w, v1 - v0, v0);
    } else {
      const int layer = CLAMP ? min(max((int32_t)t >> 24, 0), last_layer) : (int32_t)t >> 24;
      const ST* p = base + (layer * LE + rb * c.su + ra);
      const float2 r0 = stack_pair(p), r1 = stack_pair(p + c.su);
      const float top = fmaf(fa, r0.y - r0.x, r0.x);
      const float bot = fmaf(fa, r1.y - r1.x, r1.x);
      acc[z] += fmaf(fb, bot - top, top);
    }
    ap += td.af2;
    bp += td.bf2;
    t += td.tk;
  }
}

// One 32 x 8 x 8 tile (tile coordinates bx, by, bz); s_dir: dir_count TileDir records.
template <typename ST, bool LIN>
__device__ __forceinline__ void bp_generic_tile(int bx, int by, int bz, const DirParams* __restrict__ dirs,
                                                const ST* __restrict__ stack, const BackprojConst& c,
                                                int dir_begin, int dir_count, float* __restrict__ vol,
                                                int accumulate, TileDir* s_dir) {
  const int i0 = bx * kTX, j0 = by * kTY, k0 = bz * kTZ;
  // a warp covers a WX (x) x 32/WX (y) patch of voxel columns (8 x 4 by default rather than
  // a line of 32: its samples in one z plane fall on a compact detector patch in any view
  // orientation, so a row gather touches fewer cache lines); the shape only moves voxels
  // between threads, every voxel's arithmetic is the same
  const int kWX = c.warp_cols, kWY = 32 / kWX;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int tx = (w % (kTX / kWX)) * kWX + (l % kWX), ty = (w / (kTX / kWX)) * kWY + l / kWX;
  for (int d = threadIdx.x; d < dir_count; d += blockDim.x) {
    const DirParams& p = dirs[dir_begin + d];
    // tile origin on the detector: exact integer sums in 2^-40 pixel
    const long long a = p.a[3] + p.a[0] * i0 + p.a[1] * j0 + p.a[2] * k0;
    const long long b = p.b[3] + p.b[0] * i0 + p.b[1] * j0 + p.b[2] * k0;
    TileDir td;
    td.ia = pix_floor(a);
    td.ib = pix_floor(b);
    td.fa = pix_frac(a) - 0.5f;
    td.fb = pix_frac(b) - 0.5f;
    td.t = (uint32_t)p.t[0] + (uint32_t)p.t[1] * (uint32_t)i0 + (uint32_t)p.t[2] * (uint32_t)j0 +
           (uint32_t)p.t[3] * (uint32_t)k0;
    td.af0 = p.af[0];
    td.af1 = p.af[1];
    td.af2 = p.af[2];
    td.bf0 = p.bf[0];
    td.bf1 = p.bf[1];
    td.bf2 = p.bf[2];
    td.ti = (uint32_t)p.t[1];
    td.tj = (uint32_t)p.t[2];
    td.tk = (uint32_t)p.t[3];
    // Whole tile (every thread, also those past the volume edge) inside the detector by a
    // margin (1e-3 pixel) far above the FP32 in-tile error, and inside the layer range: then
    // the clamps and the saturation below cannot change anything and are skipped (same
    // bits).  The extremes of the affine maps over the tile (at its corners) come with the
    // direction, in 2^-16 pixel, rounded outwards.
    const long long a16 = a >> (kPixFracBits - 16), b16 = b >> (kPixFracBits - 16);
    const long long t = (long long)p.t[0] + (long long)p.t[1] * i0 + (long long)p.t[2] * j0 + (long long)p.t[3] * k0;
    constexpr long long kMargin16 = 66;  // 1e-3 pixel in 2^-16 pixel
    const long long lo16 = -32768 + kMargin16;
    td.pad[0] = p.ab_ext[0] != INT32_MIN && p.t_ext[0] != INT32_MIN && a16 + p.ab_ext[0] >= lo16 &&
                a16 + p.ab_ext[1] + 1 <= (long long)c.nu * 65536 - 32768 - kMargin16 && b16 + p.ab_ext[2] >= lo16 &&
                b16 + p.ab_ext[3] + 1 <= (long long)c.nv * 65536 - 32768 - kMargin16 && t + p.t_ext[0] >= 0 &&
                t + p.t_ext[1] < ((long long)c.nz_layers << 24);
    td.pad[1] = 0;
    s_dir[d] = td;
  }
  __syncthreads();

  float acc[kTZ];
#pragma unroll
  for (int z = 0; z < kTZ; ++z) acc[z] = 0.f;
  const float ftx = (float)tx, fty = (float)ty;
  for (int d = 0; d < dir_count; ++d) {
    const TileDir& td = s_dir[d];
    const ST* base = stack + (size_t)d * c.nz_layers * c.layer_elems + (ptrdiff_t)(td.ib + 1) * c.su + (td.ia + 1);
    if (td.pad[0]) generic_run<ST, false, LIN>(td, base, c, ftx, fty, tx, ty, acc);
    else generic_run<ST, true, LIN>(td, base, c, ftx, fty, tx, ty, acc);
  }

  const int i = i0 + tx, j = j0 + ty;
  if (i >= c.nx || j >= c.ny) return;
#pragma unroll
  for (int z = 0; z < kTZ; ++z) {
    const int k = k0 + z;
    if (k < c.nz) {
      float* v = vol + ((size_t)k * c.ny + j) * c.nx + i;
      *v = accumulate ? *v + acc[z] : acc[z];
    }
  }
}

// Resident CTAs per SM the general kernel asks for (registers per thread = 65536 / (256 x
// this)); a compile-time tuning constant.
#ifndef RECON_GEN_MIN_CTAS
#define RECON_GEN_MIN_CTAS 4
#endif

template <typename ST, bool LIN>
__global__ void __launch_bounds__(kTX* kTY, RECON_GEN_MIN_CTAS) k_backproject(const DirParams* __restrict__ dirs,
                                                           const ST* __restrict__ stack, BackprojConst c,
                                                           int dir_begin, int dir_count, float* __restrict__ vol,
                                                           int accumulate) {
  extern __shared__ TileDir s_dir[];
  bp_generic_tile<ST, LIN>(blockIdx.x, blockIdx.y, blockIdx.z, dirs, stack, c, dir_begin, dir_count, vol, accumulate,
                      s_dir);
}

// ---------------------------------------------------------------------------------
// Single-axis scans about the volume y axis (rot row 1 = (0,1,0) for every view): the
// detector row is v = j + b_off for every direction, and the u coordinate and the depth
// layer do not depend on j.  A thread owns an (i, k) voxel column segment of kJ voxels
// along y: per direction it forms u and the layer once, then walks kJ detector rows with
// two taps each (four when b_off is a half-integer), accumulating in registers.
constexpr int kAX = 32, kAZ = 8, kJ = 16;
// A warp of the single-axis kernels covers kLaneWX (i) x 32 / kLaneWX (k) voxel columns:
// a compact footprint spans fewer depth layers and detector columns than a line of 32
// along i, so each of its row gathers touches fewer cache lines.
constexpr int kLaneWX = 8;
static_assert(32 % kLaneWX == 0 && kAX % kLaneWX == 0 && kAZ % (32 / kLaneWX) == 0 &&
                  (kAX / kLaneWX) * (kAZ / (32 / kLaneWX)) * 32 == kAX * kAZ,
              "the warps must tile the 32 x 8 voxel columns");
__device__ __forceinline__ void axis_lane(int t, int& tx, int& tz) {
  constexpr int WZ = 32 / kLaneWX, BX = kAX / kLaneWX;  // warp extent in k; warps along i
  const int w = t >> 5, l = t & 31;
  tx = (w % BX) * kLaneWX + (l % kLaneWX);
  tz = (w / BX) * WZ + l / kLaneWX;
}

struct AxisDir {  // per (tile, direction), 32 bytes in shared memory
  float fa;       // fractional tile-origin u coordinate minus 0.5
  int ia;         // integer tile-origin u coordinate
  uint32_t t;     // depth at the tile origin, 2^-24 layer units
  float af0, af2; // du/di, du/dk
  uint32_t ti, tk;
  int pad;
};
static_assert(sizeof(AxisDir) == 32, "AxisDir layout");

template <typename ST>
__device__ __forceinline__ float lerp_row(const ST* p, float fa) {
  const float2 v = stack_pair(p);
  return fmaf(fa, v.y - v.x, v.x);
}

// One 32 (i) x 8 (k) x 16 (j) tile (tile coordinates bx, by = k tile, bz = j tile).
template <typename ST, bool TWO_ROWS>
__device__ __forceinline__ void bp_axis_tile(int bx, int by, int bz, const DirParams* __restrict__ dirs,
                                             const ST* __restrict__ stack, const BackprojConst& c, int dir_begin,
                                             int dir_count, float* __restrict__ vol, int accumulate,
                                             AxisDir* s_ax) {
  const int i0 = bx * kAX, k0 = by * kAZ, j0 = bz * kJ;
  int tx, tz;
  axis_lane(threadIdx.x, tx, tz);
  for (int d = threadIdx.x; d < dir_count; d += blockDim.x) {
    const DirParams& p = dirs[dir_begin + d];
    const long long a = p.a[3] + p.a[0] * i0 + p.a[2] * k0;  // p.a[1] = 0; 2^-40 pixel
    AxisDir ad;
    ad.fa = pix_frac(a) - 0.5f;
    ad.ia = pix_floor(a);
    ad.t = (uint32_t)p.t[0] + (uint32_t)p.t[1] * (uint32_t)i0 + (uint32_t)p.t[3] * (uint32_t)k0;  // Tj = 0
    ad.af0 = p.af[0];
    ad.af2 = p.af[2];
    ad.ti = (uint32_t)p.t[1];
    ad.tk = (uint32_t)p.t[3];
    ad.pad = 0;
    s_ax[d] = ad;
  }
  __syncthreads();

  float acc[kJ];
#pragma unroll
  for (int q = 0; q < kJ; ++q) acc[q] = 0.f;
  // detector row of this thread's first voxel, and whether every row it reads lies in
  // the stack (rows -1 and nv are the zero border)
  const int row0 = j0 + c.b_int;
  const bool rows_inside = row0 >= -1 && row0 + kJ - 1 + (TWO_ROWS ? 1 : 0) <= c.nv;
  const float ftx = (float)tx, ftz = (float)tz;
  const int last_layer = c.nz_layers - 1;
  const float fb = c.b_frac;
  for (int d = 0; d < dir_count; ++d) {
    const AxisDir ad = s_ax[d];
    const float ap = fmaf(ad.af0, ftx, fmaf(ad.af2, ftz, ad.fa));
    const int layer = min(max((int32_t)(ad.t + ad.ti * (uint32_t)tx + ad.tk * (uint32_t)tz) >> 24, 0), last_layer);
    const float ta = fminf(fmaxf(ap, (float)(-1 - ad.ia)), (float)(c.nu - 1 - ad.ia)) + kMagic;
    const int ra = __float_as_int(ta) - kMagicBits;
    const float fa = __saturatef(ap - (ta - kMagic) + 0.5f);
    const ST* p = stack + ((size_t)d * c.nz_layers + layer) * c.layer_elems + (ptrdiff_t)(row0 + 1) * c.su +
                  (ra + ad.ia + 1);
    if (rows_inside) {
      // every tap of this direction is loaded before the first is used; with the kernel's
      // launch bounds the registers hold them all, so the column's gathers are in flight together
      float2 v[kJ + (TWO_ROWS ? 1 : 0)];
#pragma unroll
      for (int q = 0; q < kJ + (TWO_ROWS ? 1 : 0); ++q) v[q] = stack_pair(p + q * c.su);
      if (TWO_ROWS) {
        float prev = fmaf(fa, v[0].y - v[0].x, v[0].x);
#pragma unroll
        for (int q = 0; q < kJ; ++q) {
          const float next = fmaf(fa, v[q + 1].y - v[q + 1].x, v[q + 1].x);
          acc[q] += fmaf(fb, next - prev, prev);
          prev = next;
        }
      } else {
#pragma unroll
        for (int q = 0; q < kJ; ++q) acc[q] += fmaf(fa, v[q].y - v[q].x, v[q].x);
      }
    } else {
#pragma unroll
      for (int q = 0; q < kJ; ++q) {
        const int r = row0 + q;
        const float lo = (r >= -1 && r <= c.nv) ? lerp_row(p + q * c.su, fa) : 0.f;
        if (TWO_ROWS) {
          const float hi = (r + 1 >= -1 && r + 1 <= c.nv) ? lerp_row(p + (q + 1) * c.su, fa) : 0.f;
          acc[q] += fmaf(fb, hi - lo, lo);
        } else {
          acc[q] += lo;
        }
      }
    }
  }

  const int i = i0 + tx, k = k0 + tz;
  if (i >= c.nx || k >= c.nz) return;
#pragma unroll
  for (int q = 0; q < kJ; ++q) {
    const int j = j0 + q;
    if (j < c.ny) {
      float* v = vol + ((size_t)k * c.ny + j) * c.nx + i;
      *v = accumulate ? *v + acc[q] : acc[q];
    }
  }
}

template <typename ST, bool TWO_ROWS>
// At least 4 CTAs per SM (float32 pairs): ptxas then keeps all of a column's gathers in
// registers at once (58 registers); left to itself it chose 40 and issued them in batches
// (256^3 / 120 directions: 1.57 -> 0.75 ms).  The bfloat16 variant, bound by issue (it
// unpacks every pair), runs best at 5 (0.84 -> 0.80 ms).
__global__ void __launch_bounds__(kAX* kAZ, sizeof(ST) == 4 ? 5 : 4) k_backproject_axis(const DirParams* __restrict__ dirs,
                                                                const ST* __restrict__ stack, BackprojConst c,
                                                                int dir_begin, int dir_count,
                                                                float* __restrict__ vol, int accumulate) {
  extern __shared__ AxisDir s_ax[];
  bp_axis_tile<ST, TWO_ROWS>(blockIdx.x, blockIdx.y, blockIdx.z, dirs, stack, c, dir_begin, dir_count, vol,
                             accumulate, s_ax);
}

template <typename ST, bool TWO_ROWS>
cudaError_t launch_axis(const BackprojConst& c, const DirParams* dirs, const void* stack, int dir_begin,
                        int dir_count, float* volume, int accumulate, cudaStream_t stream) {
  dim3 grid((c.nx + kAX - 1) / kAX, (c.nz + kAZ - 1) / kAZ, (c.ny + kJ - 1) / kJ);
  const size_t smem = (size_t)dir_count * sizeof(AxisDir);
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_backproject_axis<ST, TWO_ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_backproject_axis<ST, TWO_ROWS><<<grid, kAX * kAZ, smem, stream>>>(dirs, (const ST*)stack, c, dir_begin,
                                                                      dir_count, volume, accumulate);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Staged single-axis backprojection.  Per (tile, direction) the stack entries the tile
// can touch form a box of layers x (16 or 17) detector rows x a column range (exact: the
// per-thread u coordinate is a chain of FMAs, monotone in the thread indices, so its
// extremes are at the tile corners; the layer is an exact integer sum).  The box of the
// next direction is copied into shared memory with cp.async while the current one is
// consumed (double buffering), so the gathers read shared memory and the copies hide the
// L2/DRAM latency.  A direction whose box exceeds a buffer is read from global memory.
constexpr int kStageBytes = 16 * 1024;

struct AxisBox {  // per (tile, direction), 16 bytes in shared memory
  int L0, nL;     // first layer, layers
  int c0, W;      // first pair column, width (W = 0: read from global memory)
};
static_assert(sizeof(AxisBox) == 16, "AxisBox layout");

__device__ __forceinline__ void cp_async(float2* dst, const float2* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async(__nv_bfloat162* dst, const __nv_bfloat162* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ float2 smem_pair(const float2* p) { return *p; }
__device__ __forceinline__ float2 smem_pair(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
template <typename ST>
__device__ __forceinline__ ST zero_pair();
template <>
__device__ __forceinline__ float2 zero_pair<float2>() { return make_float2(0.f, 0.f); }
template <>
__device__ __forceinline__ __nv_bfloat162 zero_pair<__nv_bfloat162>() { return __floats2bfloat162_rn(0.f, 0.f); }

// pair column a thread reads for u coordinate ap (the clamped tap + 1), see bp_axis_tile
__device__ __forceinline__ int pair_col(float ap, int ia, int nu) {
  const float ta = fminf(fmaxf(ap, (float)(-1 - ia)), (float)(nu - 1 - ia)) + kMagic;
  return __float_as_int(ta) - kMagicBits + ia + 1;
}

template <typename ST, bool TWO_ROWS>
__global__ void __launch_bounds__(kAX* kAZ) k_backproject_axis_staged(const DirParams* __restrict__ dirs,
                                                                       const ST* __restrict__ stack, BackprojConst c,
                                                                       int dir_begin, int dir_count,
                                                                       float* __restrict__ vol, int accumulate) {
  constexpr int NR = kJ + (TWO_ROWS ? 1 : 0);
  constexpr int CAP = kStageBytes / (int)sizeof(ST);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ST* buf0 = (ST*)smem_raw;
  ST* buf1 = buf0 + CAP;
  AxisDir* s_ax = (AxisDir*)(smem_raw + 2 * kStageBytes);
  AxisBox* s_box = (AxisBox*)(s_ax + dir_count);
  const int i0 = blockIdx.x * kAX, k0 = blockIdx.y * kAZ, j0 = blockIdx.z * kJ;
  int tx, tz;
  axis_lane(threadIdx.x, tx, tz);
  const int row0 = j0 + c.b_int;  // detector row of this tile's first voxel row
  const int last_layer = c.nz_layers - 1;
  for (int d = threadIdx.x; d < dir_count; d += blockDim.x) {
    const DirParams& p = dirs[dir_begin + d];
    const long long a = p.a[3] + p.a[0] * i0 + p.a[2] * k0;  // p.a[1] = 0; 2^-40 pixel
    AxisDir ad;
    ad.fa = pix_frac(a) - 0.5f;
    ad.ia = pix_floor(a);
    ad.t = (uint32_t)p.t[0] + (uint32_t)p.t[1] * (uint32_t)i0 + (uint32_t)p.t[3] * (uint32_t)k0;  // Tj = 0
    ad.af0 = p.af[0];
    ad.af2 = p.af[2];
    ad.ti = (uint32_t)p.t[1];
    ad.tk = (uint32_t)p.t[3];
    ad.pad = 0;
    s_ax[d] = ad;
    // the box: extremes of the pair column and of the layer over the corners of the part
    // of the tile inside the volume (threads outside it are clamped into the box)
    const int ex = min(kAX, c.nx - i0) - 1, ez = min(kAZ, c.nz - k0) - 1;
    int cmin = 1 << 30, cmax = -(1 << 30), lmin = 1 << 30, lmax = -(1 << 30);
    for (int cx = 0; cx < 2; ++cx)
      for (int cz = 0; cz < 2; ++cz) {
        const int ux = cx ? ex : 0, uz = cz ? ez : 0;
        const int pc = pair_col(fmaf(ad.af0, (float)ux, fmaf(ad.af2, (float)uz, ad.fa)), ad.ia, c.nu);
        const int layer =
            min(max((int32_t)(ad.t + ad.ti * (uint32_t)ux + ad.tk * (uint32_t)uz) >> 24, 0), last_layer);
        cmin = min(cmin, pc);
        cmax = max(cmax, pc);
        lmin = min(lmin, layer);
        lmax = max(lmax, layer);
      }
    AxisBox bx;
    bx.L0 = lmin;
    bx.nL = lmax - lmin + 1;
    bx.c0 = cmin;
    bx.W = cmax - cmin + 1;
    if (bx.nL * NR * bx.W > CAP) bx.W = 0;  // too large: read from global memory
    s_box[d] = bx;
  }
  __syncthreads();

  // copy the box of direction d into `buf` (rows outside the stack become zero)
  auto issue = [&](int d, ST* buf) {
    const AxisBox bx = s_box[d];
    if (bx.W > 0) {
      // warp w copies box rows w, w + 8, ...; its lanes stride over the columns
      const ST* base = stack + (size_t)d * c.nz_layers * c.layer_elems + bx.c0;
      const int lane = threadIdx.x & 31;
      for (int br = threadIdx.x >> 5; br < bx.nL * NR; br += kAZ) {
        const int l = br / NR, r = br - l * NR;  // NR is a compile-time constant
        const int R = row0 + 1 + r;              // padded row
        ST* dst = buf + br * bx.W;
        if (R >= 0 && R <= c.nv + 1) {
          const ST* src = base + (size_t)(bx.L0 + l) * c.layer_elems + (size_t)R * c.su;
          for (int col = lane; col < bx.W; col += 32) cp_async(dst + col, src + col);
        } else {
          for (int col = lane; col < bx.W; col += 32) dst[col] = zero_pair<ST>();
        }
      }
    }
    cp_commit();
  };

  float acc[kJ];
#pragma unroll
  for (int q = 0; q < kJ; ++q) acc[q] = 0.f;
  const bool rows_inside = row0 >= -1 && row0 + kJ - 1 + (TWO_ROWS ? 1 : 0) <= c.nv;
  const float ftx = (float)tx, ftz = (float)tz;
  const float fb = c.b_frac;
  if (dir_count > 0) issue(0, buf0);
  for (int d = 0; d < dir_count; ++d) {
    ST* cur = (d & 1) ? buf1 : buf0;
    if (d + 1 < dir_count) {
      issue(d + 1, (d & 1) ? buf0 : buf1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();  // the box of d is in `cur` for every thread
    const AxisDir ad = s_ax[d];
    const AxisBox bx = s_box[d];
    const float ap = fmaf(ad.af0, ftx, fmaf(ad.af2, ftz, ad.fa));
    const int layer = min(max((int32_t)(ad.t + ad.ti * (uint32_t)tx + ad.tk * (uint32_t)tz) >> 24, 0), last_layer);
    const float ta = fminf(fmaxf(ap, (float)(-1 - ad.ia)), (float)(c.nu - 1 - ad.ia)) + kMagic;
    const int ra = __float_as_int(ta) - kMagicBits;
    const float fa = __saturatef(ap - (ta - kMagic) + 0.5f);
    if (bx.W > 0) {
      const int bl = min(max(layer - bx.L0, 0), bx.nL - 1);
      const int bc = min(max(ra + ad.ia + 1 - bx.c0, 0), bx.W - 1);
      const ST* sp = cur + (bl * NR) * bx.W + bc;
      if (TWO_ROWS) {
        float2 v = smem_pair(sp);
        float prev = fmaf(fa, v.y - v.x, v.x);
#pragma unroll
        for (int q = 0; q < kJ; ++q) {
          v = smem_pair(sp + (q + 1) * bx.W);
          const float next = fmaf(fa, v.y - v.x, v.x);
          acc[q] += fmaf(fb, next - prev, prev);
          prev = next;
        }
      } else {
#pragma unroll
        for (int q = 0; q < kJ; ++q) {
          const float2 v = smem_pair(sp + q * bx.W);
          acc[q] += fmaf(fa, v.y - v.x, v.x);
        }
      }
    } else {  // box too large for a buffer: gathers from global memory (as bp_axis_tile)
      const ST* p = stack + ((size_t)d * c.nz_layers + layer) * c.layer_elems + (ptrdiff_t)(row0 + 1) * c.su +
                    (ra + ad.ia + 1);
#pragma unroll
      for (int q = 0; q < kJ; ++q) {
        const int r = row0 + q;
        const float lo = (rows_inside || (r >= -1 && r <= c.nv)) ? lerp_row(p + q * c.su, fa) : 0.f;
        if (TWO_ROWS) {
          const float hi = (rows_inside || (r + 1 >= -1 && r + 1 <= c.nv)) ? lerp_row(p + (q + 1) * c.su, fa) : 0.f;
          acc[q] += fmaf(fb, hi - lo, lo);
        } else {
          acc[q] += lo;
        }
      }
    }
    __syncthreads();  // everyone is done with `cur` before it is refilled
  }

  const int i = i0 + tx, k = k0 + tz;
  if (i >= c.nx || k >= c.nz) return;
#pragma unroll
  for (int q = 0; q < kJ; ++q) {
    const int j = j0 + q;
    if (j < c.ny) {
      float* v = vol + ((size_t)k * c.ny + j) * c.nx + i;
      *v = accumulate ? *v + acc[q] : acc[q];
    }
  }
}

template <typename ST, bool TWO_ROWS>
cudaError_t launch_axis_staged(const BackprojConst& c, const DirParams* dirs, const void* stack, int dir_begin,
                               int dir_count, float* volume, int accumulate, cudaStream_t stream) {
  dim3 grid((c.nx + kAX - 1) / kAX, (c.nz + kAZ - 1) / kAZ, (c.ny + kJ - 1) / kJ);
  const size_t smem = 2 * (size_t)kStageBytes + (size_t)dir_count * (sizeof(AxisDir) + sizeof(AxisBox));
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_backproject_axis_staged<ST, TWO_ROWS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_backproject_axis_staged<ST, TWO_ROWS><<<grid, kAX * kAZ, smem, stream>>>(dirs, (const ST*)stack, c, dir_begin,
                                                                             dir_count, volume, accumulate);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Persistent backprojection over many tomograms: CTAs take (tomogram, tile) items from
// one atomic counter until the items run out; each item runs the tile body of its
// tomogram's kind.  No CTA waits on another, so the loop always ends.
__global__ void __launch_bounds__(256) k_backproject_persistent(const BatchBp* __restrict__ desc, int n_desc,
                                                                unsigned long long total,
                                                                unsigned long long* __restrict__ counter) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ unsigned long long s_item;
  __shared__ int s_p;
  for (;;) {
    __syncthreads();  // the previous item is done with the shared records
    if (threadIdx.x == 0) {
      const unsigned long long it = atomicAdd(counter, 1ull);
      int p = 0;
      if (it < total)
        while (p + 1 < n_desc && desc[p + 1].first_item <= it) ++p;
      s_item = it;
      s_p = p;
    }
    __syncthreads();
    const unsigned long long it = s_item;
    if (it >= total) return;
    const BatchBp& d = desc[s_p];
    const unsigned long long t = it - d.first_item;
    const int bx = (int)(t % d.gx), by = (int)((t / d.gx) % d.gy), bz = (int)(t / ((unsigned long long)d.gx * d.gy));
    switch (d.kind) {
      case 0:
        bp_generic_tile<float2, false>(bx, by, bz, d.dirs, (const float2*)d.stack, d.c, d.dir_begin, d.dir_count,
                                       d.vol, d.accumulate, (TileDir*)smem_raw);
        break;
      case 1:
        bp_generic_tile<__nv_bfloat162, false>(bx, by, bz, d.dirs, (const __nv_bfloat162*)d.stack, d.c,
                                               d.dir_begin, d.dir_count, d.vol, d.accumulate, (TileDir*)smem_raw);
        break;
      case 6:
        bp_generic_tile<float2, true>(bx, by, bz, d.dirs, (const float2*)d.stack, d.c, d.dir_begin, d.dir_count,
                                      d.vol, d.accumulate, (TileDir*)smem_raw);
        break;
      case 7:
        bp_generic_tile<__nv_bfloat162, true>(bx, by, bz, d.dirs, (const __nv_bfloat162*)d.stack, d.c,
                                              d.dir_begin, d.dir_count, d.vol, d.accumulate, (TileDir*)smem_raw);
        break;
      case 2:
        bp_axis_tile<float2, false>(bx, by, bz, d.dirs, (const float2*)d.stack, d.c, d.dir_begin, d.dir_count, d.vol,
                                    d.accumulate, (AxisDir*)smem_raw);
        break;
      case 3:
        bp_axis_tile<float2, true>(bx, by, bz, d.dirs, (const float2*)d.stack, d.c, d.dir_begin, d.dir_count, d.vol,
                                   d.accumulate, (AxisDir*)smem_raw);
        break;
      case 4:
        bp_axis_tile<__nv_bfloat162, false>(bx, by, bz, d.dirs, (const __nv_bfloat162*)d.stack, d.c, d.dir_begin,
                                            d.dir_count, d.vol, d.accumulate, (AxisDir*)smem_raw);
        break;
      case 5:
        bp_axis_tile<__nv_bfloat162, true>(bx, by, bz, d.dirs, (const __nv_bfloat162*)d.stack, d.c, d.dir_begin,
                                           d.dir_count, d.vol, d.accumulate, (AxisDir*)smem_raw);
        break;
    }
  }
}

}  // namespace

template <typename ST, bool LIN>
cudaError_t launch_generic(const BackprojConst& c, const DirParams* dirs, const void* stack, int dir_begin,
                           int dir_count, float* volume, int accumulate, cudaStream_t stream) {
  dim3 grid((c.nx + kTX - 1) / kTX, (c.ny + kTY - 1) / kTY, (c.nz + kTZ - 1) / kTZ);
  const size_t smem = (size_t)dir_count * sizeof(TileDir);
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_backproject<ST, LIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_backproject<ST, LIN><<<grid, kTX * kTY, smem, stream>>>(dirs, (const ST*)stack, c, dir_begin, dir_count, volume,
                                                            accumulate);
  return cudaGetLastError();
}

cudaError_t launch_backproject(const BackprojConst& c, const DirParams* dirs, const void* stack, int dir_begin,
                               int dir_count, float* volume, int accumulate, cudaStream_t stream) {
  if (dir_count <= 0 || c.nx <= 0 || c.ny <= 0 || c.nz <= 0) return cudaSuccess;
  // the layer blend runs in the general kernel for every geometry
  if (c.axis_y && !c.staged && !c.layer_linear) {
    const bool two = c.b_frac != 0.f;
    if (c.stack_bf16)
      return two ? launch_axis<__nv_bfloat162, true>(c, dirs, stack, dir_begin, dir_count, volume, accumulate, stream)
                 : launch_axis<__nv_bfloat162, false>(c, dirs, stack, dir_begin, dir_count, volume, accumulate, stream);
    return two ? launch_axis<float2, true>(c, dirs, stack, dir_begin, dir_count, volume, accumulate, stream)
               : launch_axis<float2, false>(c, dirs, stack, dir_begin, dir_count, volume, accumulate, stream);
  }
  if (c.axis_y && !c.layer_linear) {
    const bool two = c.b_frac != 0.f;
    if (c.stack_bf16)
      return two ? launch_axis_staged<__nv_bfloat162, true>(c, dirs, stack, dir_begin, dir_count, volume, accumulate,
                                                            stream)
                 : launch_axis_staged<__nv_bfloat162, false>(c, dirs, stack, dir_begin, dir_count, volume, accumulate,
                                                             stream);
    return two ? launch_axis_staged<float2, true>(c, dirs, stack, dir_begin, dir_count, volume, accumulate, stream)
               : launch_axis_staged<float2, false>(c, dirs, stack, dir_begin, dir_count, volume, accumulate, stream);
  }
  return c.stack_bf16 ? (c.layer_linear ? launch_generic<__nv_bfloat162, true>(c, dirs, stack, dir_begin, dir_count,
                                                                               volume, accumulate, stream)
                                         : launch_generic<__nv_bfloat162, false>(c, dirs, stack, dir_begin, dir_count,
                                                                                 volume, accumulate, stream))
                      : (c.layer_linear ? launch_generic<float2, true>(c, dirs, stack, dir_begin, dir_count, volume,
                                                                       accumulate, stream)
                                        : launch_generic<float2, false>(c, dirs, stack, dir_begin, dir_count, volume,
                                                                        accumulate, stream));
}

void describe_backproject(const BackprojConst& c, const DirParams* dirs, const void* stack, int dir_begin,
                          int dir_count, float* volume, int accumulate, BatchBp* out) {
  out->c = c;
  out->dirs = dirs;
  out->stack = stack;
  out->vol = volume;
  out->dir_begin = dir_begin;
  out->dir_count = dir_count;
  out->accumulate = accumulate;
  const bool axis = c.axis_y && !c.layer_linear;
  if (axis) {
    out->kind = 2 + (c.stack_bf16 ? 2 : 0) + (c.b_frac != 0.f ? 1 : 0);
    out->gx = (c.nx + kAX - 1) / kAX;
    out->gy = (c.nz + kAZ - 1) / kAZ;
    out->gz = (c.ny + kJ - 1) / kJ;
  } else {
    out->kind = (c.stack_bf16 ? 1 : 0) + (c.layer_linear ? 6 : 0);
    out->gx = (c.nx + kTX - 1) / kTX;
    out->gy = (c.ny + kTY - 1) / kTY;
    out->gz = (c.nz + kTZ - 1) / kTZ;
  }
  out->smem = (size_t)dir_count * (axis ? sizeof(AxisDir) : sizeof(TileDir));
}

cudaError_t launch_backproject_persistent(const BatchBp* desc_dev, int n_desc, unsigned long long total,
                                          unsigned long long* counter, size_t smem, cudaStream_t stream) {
  if (total == 0) return cudaSuccess;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_backproject_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int sms = device_sm_count();
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backproject_persistent, 256, smem);
  if (per_sm < 1) per_sm = 1;
  const unsigned long long ctas = (unsigned long long)sms * per_sm;
  const unsigned grid = (unsigned)(ctas < total ? ctas : total);
  k_backproject_persistent<<<grid, 256, smem, stream>>>(desc_dev, n_desc, total, counter);
  return cudaGetLastError();
}

}  // namespace recon
