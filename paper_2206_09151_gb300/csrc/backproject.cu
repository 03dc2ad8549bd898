// Stage B of the layered UTR path: every voxel takes, from each direction of a block,
// the bilinear sample of the layer that contains its depth and sums over directions
// (the real-space counterpart of gridding each image onto its Ewald patch, Sec. 2).
//
// A CTA owns a 32 x 8 x 4 voxel tile; a thread owns a 4-voxel run along z and keeps
// its sums in registers across the whole direction block, then reads-modifies-writes
// the volume once.  Coordinates: per (tile, direction) the tile-origin pixel
// coordinate is formed in FP64 and split into an integer and an FP32 fraction, so the
// FP32 arithmetic inside the tile works on small numbers (error ~1e-6 pixel at any
// detector size).  The depth coordinate is an exact 2^-24 fixed-point integer sum, so
// the layer decision does not depend on the traversal order.  Out-of-detector taps
// read the stack's zero border (rows -1 and nv, pairs holding the columns -1 and nu):
// the integer tap is clamped to [-1, n-1] and the weight saturated to [0, 1], which
// gives exactly bilinear-with-zero-outside.  Each stack entry is the tap pair
// (Y[u], Y[u+1]), so a bilinear row is one load.
#include <cuda_bf16.h>

#include "recon_internal.h"

namespace recon {
namespace {

constexpr int kTX = 32, kTY = 8, kTZ = 4;

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

// One 32 x 8 x 4 tile (tile coordinates bx, by, bz); s_dir: dir_count TileDir records.
template <typename ST>
__device__ __forceinline__ void bp_generic_tile(int bx, int by, int bz, const DirParams* __restrict__ dirs,
                                                const ST* __restrict__ stack, const BackprojConst& c,
                                                int dir_begin, int dir_count, float* __restrict__ vol,
                                                int accumulate, TileDir* s_dir) {
  const int i0 = bx * kTX, j0 = by * kTY, k0 = bz * kTZ;
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
  for (int d = threadIdx.x; d < dir_count; d += blockDim.x) {
    const DirParams& p = dirs[dir_begin + d];
    const double a = fma(p.a[0], (double)i0, fma(p.a[1], (double)j0, fma(p.a[2], (double)k0, p.a[3])));
    const double b = fma(p.b[0], (double)i0, fma(p.b[1], (double)j0, fma(p.b[2], (double)k0, p.b[3])));
    const double fla = floor(a), flb = floor(b);
    TileDir td;
    td.ia = (int)fla;
    td.ib = (int)flb;
    td.fa = (float)(a - fla) - 0.5f;
    td.fb = (float)(b - flb) - 0.5f;
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
    td.pad[0] = td.pad[1] = 0;
    s_dir[d] = td;
  }
  __syncthreads();

  float acc[kTZ];
#pragma unroll
  for (int z = 0; z < kTZ; ++z) acc[z] = 0.f;
  const float ftx = (float)tx, fty = (float)ty;
  const int last_layer = c.nz_layers - 1;
  for (int d = 0; d < dir_count; ++d) {
    const TileDir& td = s_dir[d];
    float ap = fmaf(td.af0, ftx, fmaf(td.af1, fty, td.fa));
    float bp = fmaf(td.bf0, ftx, fmaf(td.bf1, fty, td.fb));
    uint32_t t = td.t + td.ti * (uint32_t)tx + td.tj * (uint32_t)ty;
    const float loa = (float)(-1 - td.ia), hia = (float)(c.nu - 1 - td.ia);
    const float lob = (float)(-1 - td.ib), hib = (float)(c.nv - 1 - td.ib);
    const ST* base = stack + (size_t)d * c.nz_layers * c.layer_elems + (ptrdiff_t)(td.ib + 1) * c.su + (td.ia + 1);
#pragma unroll
    for (int z = 0; z < kTZ; ++z) {
      const int layer = min(max((int32_t)t >> 24, 0), last_layer);
      const float ta = fminf(fmaxf(ap, loa), hia) + kMagic;
      const float tb = fminf(fmaxf(bp, lob), hib) + kMagic;
      const int ra = __float_as_int(ta) - kMagicBits;
      const int rb = __float_as_int(tb) - kMagicBits;
      const float fa = __saturatef(ap - (ta - kMagic) + 0.5f);
      const float fb = __saturatef(bp - (tb - kMagic) + 0.5f);
      const ST* p = base + (size_t)layer * c.layer_elems + (ptrdiff_t)rb * c.su + ra;
      const float2 r0 = stack_pair(p), r1 = stack_pair(p + c.su);
      const float top = fmaf(fa, r0.y - r0.x, r0.x);
      const float bot = fmaf(fa, r1.y - r1.x, r1.x);
      acc[z] += fmaf(fb, bot - top, top);
      ap += td.af2;
      bp += td.bf2;
      t += td.tk;
    }
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

template <typename ST>
__global__ void __launch_bounds__(kTX* kTY) k_backproject(const DirParams* __restrict__ dirs,
                                                           const ST* __restrict__ stack, BackprojConst c,
                                                           int dir_begin, int dir_count, float* __restrict__ vol,
                                                           int accumulate) {
  extern __shared__ TileDir s_dir[];
  bp_generic_tile<ST>(blockIdx.x, blockIdx.y, blockIdx.z, dirs, stack, c, dir_begin, dir_count, vol, accumulate,
                      s_dir);
}

// ---------------------------------------------------------------------------------
// Single-axis scans about the volume y axis (rot row 1 = (0,1,0) for every view): the
// detector row is v = j + b_off for every direction, and the u coordinate and the depth
// layer do not depend on j.  A thread owns an (i, k) voxel column segment of kJ voxels
// along y: per direction it forms u and the layer once, then walks kJ detector rows with
// two taps each (four when b_off is a half-integer), accumulating in registers.
constexpr int kAX = 32, kAZ = 8, kJ = 16;

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
  const int tx = threadIdx.x % kAX, tz = threadIdx.x / kAX;
  for (int d = threadIdx.x; d < dir_count; d += blockDim.x) {
    const DirParams& p = dirs[dir_begin + d];
    const double a = fma(p.a[0], (double)i0, fma(p.a[2], (double)k0, p.a[3]));  // p.a[1] = 0
    const double fla = floor(a);
    AxisDir ad;
    ad.fa = (float)(a - fla) - 0.5f;
    ad.ia = (int)fla;
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
      if (TWO_ROWS) {
        float prev = lerp_row(p, fa);
#pragma unroll
        for (int q = 0; q < kJ; ++q) {
          const float next = lerp_row(p + (q + 1) * c.su, fa);
          acc[q] += fmaf(fb, next - prev, prev);
          prev = next;
        }
      } else {
#pragma unroll
        for (int q = 0; q < kJ; ++q) acc[q] += lerp_row(p + q * c.su, fa);
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
__global__ void __launch_bounds__(kAX* kAZ) k_backproject_axis(const DirParams* __restrict__ dirs,
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
        bp_generic_tile<float2>(bx, by, bz, d.dirs, (const float2*)d.stack, d.c, d.dir_begin, d.dir_count, d.vol,
                                d.accumulate, (TileDir*)smem_raw);
        break;
      case 1:
        bp_generic_tile<__nv_bfloat162>(bx, by, bz, d.dirs, (const __nv_bfloat162*)d.stack, d.c, d.dir_begin,
                                        d.dir_count, d.vol, d.accumulate, (TileDir*)smem_raw);
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
      default:
        bp_axis_tile<__nv_bfloat162, true>(bx, by, bz, d.dirs, (const __nv_bfloat162*)d.stack, d.c, d.dir_begin,
                                           d.dir_count, d.vol, d.accumulate, (AxisDir*)smem_raw);
        break;
    }
  }
}

}  // namespace

cudaError_t launch_backproject(const BackprojConst& c, const DirParams* dirs, const void* stack, int dir_begin,
                               int dir_count, float* volume, int accumulate, cudaStream_t stream) {
  if (dir_count <= 0 || c.nx <= 0 || c.ny <= 0 || c.nz <= 0) return cudaSuccess;
  if (c.axis_y) {
    const bool two = c.b_frac != 0.f;
    if (c.stack_bf16)
      return two ? launch_axis<__nv_bfloat162, true>(c, dirs, stack, dir_begin, dir_count, volume, accumulate, stream)
                 : launch_axis<__nv_bfloat162, false>(c, dirs, stack, dir_begin, dir_count, volume, accumulate, stream);
    return two ? launch_axis<float2, true>(c, dirs, stack, dir_begin, dir_count, volume, accumulate, stream)
               : launch_axis<float2, false>(c, dirs, stack, dir_begin, dir_count, volume, accumulate, stream);
  }
  dim3 grid((c.nx + kTX - 1) / kTX, (c.ny + kTY - 1) / kTY, (c.nz + kTZ - 1) / kTZ);
  const size_t smem = (size_t)dir_count * sizeof(TileDir);
  if (c.stack_bf16) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_backproject<__nv_bfloat162>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    k_backproject<__nv_bfloat162><<<grid, kTX * kTY, smem, stream>>>(
        dirs, (const __nv_bfloat162*)stack, c, dir_begin, dir_count, volume, accumulate);
  } else {
    if (smem > 48 * 1024) {
      cudaError_t e =
          cudaFuncSetAttribute(k_backproject<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    k_backproject<float2><<<grid, kTX * kTY, smem, stream>>>(dirs, (const float2*)stack, c, dir_begin, dir_count,
                                                              volume, accumulate);
  }
  return cudaGetLastError();
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
  if (c.axis_y) {
    out->kind = 2 + (c.stack_bf16 ? 2 : 0) + (c.b_frac != 0.f ? 1 : 0);
    out->gx = (c.nx + kAX - 1) / kAX;
    out->gy = (c.nz + kAZ - 1) / kAZ;
    out->gz = (c.ny + kJ - 1) / kJ;
  } else {
    out->kind = c.stack_bf16 ? 1 : 0;
    out->gx = (c.nx + kTX - 1) / kTX;
    out->gy = (c.ny + kTY - 1) / kTY;
    out->gz = (c.nz + kTZ - 1) / kTZ;
  }
  out->smem = (size_t)dir_count * (c.axis_y ? sizeof(AxisDir) : sizeof(TileDir));
}

cudaError_t launch_backproject_persistent(const BatchBp* desc_dev, int n_desc, unsigned long long total,
                                          unsigned long long* counter, size_t smem, cudaStream_t stream) {
  if (total == 0) return cudaSuccess;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_backproject_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backproject_persistent, 256, smem);
  if (per_sm < 1) per_sm = 1;
  const unsigned long long ctas = (unsigned long long)sms * per_sm;
  const unsigned grid = (unsigned)(ctas < total ? ctas : total);
  k_backproject_persistent<<<grid, 256, smem, stream>>>(desc_dev, n_desc, total, counter);
  return cudaGetLastError();
}

}  // namespace recon
