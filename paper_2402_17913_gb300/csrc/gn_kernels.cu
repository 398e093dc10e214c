// Kernels of the learned initial-guess network: the BF16 implicit-GEMM 3D
// convolution on the fifth-generation tensor cores (forward and data
// gradient), the weight gradient on warp-level tensor-core MMAs, and the
// memory-bound glue (pooling, upsampling, skip sums, ReLU masks, input
// scaling, loss, Adam).
//
// Convolution as a GEMM.  For an output tile of M = 128 voxels (16 along x,
// 8 along y, one z-plane) the 3x3x3 correlation with 16 input and 16 output
// channels is 27 MMAs of shape M x N x K = 128 x 16 x 16, one per tap t:
//     D[v][co] += sum_ci X[v + o_t][ci] * W[t][ci][co].
// A block walks a run of z-planes of one 16 x 8 column.  It keeps, for
// each of three copies of the input (x shifted by dx = -1, 0, +1, with a
// one-voxel halo in y), a ring of four z-planes fetched by TMA as rows of
// one voxel's 16 channels (32 bytes) in the 32-byte-swizzled K-major layout
// that the tensor core reads directly; each step of two output planes
// fetches only the two planes it adds.  The A operand of tap (dz, dy, dx)
// is then a contiguous 4 KB run of copy dx starting at line dy + 1 of the
// ring slot holding plane z + dz: descriptors differ only in their start
// address (a multiple of 256 bytes, so the swizzle phase never shifts) and
// take two values per tap as the ring turns; out-of-range voxels arrive as
// zeros (the zero padding).  Lane 0 of warp zi issues the 27 MMAs of output
// plane zi into its TMEM accumulator (128 lanes x 16 FP32 columns), then,
// once they are done, the next fetch; the four warps read the accumulator back with
// tcgen05.ld, apply the epilogue and store 32 bytes per voxel.

// The data gradient is the same kernel with the mirrored, transposed taps
// (W'[26 - t][co][ci] = W[t][ci][co]).  The weight gradient
//     dW[t][ci][co] = sum_v X[v + o_t][ci] G[v][co]
// reduces over voxels and has M = 27 x 16 rows whose shared-memory views
// are not a single strided pattern, so it uses m16n8k16 MMAs fed by
// ldmatrix.trans, which gathers any eight 16-byte rows from the same
// swizzled [z][y][x][16 channels] tiles (the swizzle puts the 8 rows of one
// channel group in 8 different bank quads).
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>

#include "gn.h"
#include "tma_host.h"
#include "umma.cuh"

namespace npmg {
namespace gn {

namespace {

constexpr int kPlaneZ = (kTY + 2) * kTX * 32;               // one z-plane of one copy: [y][x][16 ch]
constexpr int kRing = kTZ + 2;                               // z-planes kept per copy
constexpr int kCopy = kRing * kPlaneZ;
constexpr int kDescOff = 13824;                              // descriptor table after the 13824-byte weights
constexpr int kDescA = 2 * kTZ * kTaps;                      // A descriptors: [ring phase][zi][tap]
constexpr int kAOff = 14592;                                 // copies start (256-aligned: the swizzle atom)
constexpr int kConvSmem = kAOff + 3 * kCopy + 256;           // + alignment slack; 3 blocks fit an SM
constexpr int kConvThreads = 128;
constexpr uint32_t kConvCols = 32;                           // TMEM columns (kTZ accumulators of 16, min 32)
static_assert(kTZ == 2, "the ring turns by two planes per step");
static_assert(kTZ * 16 <= (int)kConvCols, "TMEM columns");
static_assert(kPlaneZ % 256 == 0 && kAOff % 256 == 0, "swizzled TMA destinations stay 256-aligned");
static_assert(kDescOff + 4 * (kDescA + kTaps) <= kAOff, "descriptor table fits");

constexpr int kXTile = (kWTX + 2) * (kWTY + 2) * (kWTZ + 2) * 32;  // wgrad x tile with halo
constexpr int kGTile = kWTX * kWTY * kWTZ * 32;
constexpr int kWgSmem = kXTile + kGTile + 1024;
constexpr int kWgThreads = 288;  // 9 warps: warp w owns taps 3w .. 3w+2 (dz, dy fixed, dx = -1, 0, 1)
static_assert(kXTile % 256 == 0 && kGTile % 256 == 0, "swizzled TMA destinations stay 256-aligned");

// byte offset of channel group g of voxel v in a 32-byte-swizzled tile
// whose base is 256-byte aligned
__device__ __forceinline__ uint32_t sw32(uint32_t v, uint32_t g) { return v * 32u + ((g ^ ((v >> 2) & 1u)) << 4); }

struct ConvArgs {
  int nx, ny, nz, nn;
  int tx, ty;
  int zc, nzc;  // planes per z-run (a multiple of kTZ) and runs per column
  long long nitems;
  void* out;
  const __nv_bfloat16* mask;
  const float* scale;
  int* err;
};

struct WgArgs {
  int nx, ny, nz, nn;
  int tx, ty, tz;
  long long ntiles;
  float* partials;
  int* err;
};

__device__ __forceinline__ uint32_t pack_bf2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ bool bf_pos(uint32_t h16) { return !(h16 & 0x8000u) && (h16 & 0x7fffu); }

template <int EPI>
__device__ __forceinline__ void store_epi(const ConvArgs& a, size_t vox, int n, const float (&v)[16]) {
  if (EPI == kEpiF32) {
    float4* o = reinterpret_cast<float4*>(static_cast<float*>(a.out) + vox * kC);
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else if (EPI == kEpiOut0) {
    static_cast<float*>(a.out)[vox] = v[0] * (a.scale ? a.scale[n] : 1.f);
  } else {
    float w[16];
    if (EPI == kEpiMask) {
      const uint4* mp = reinterpret_cast<const uint4*>(a.mask + vox * kC);
      const uint4 m0 = mp[0], m1 = mp[1];
      const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        w[2 * k] = bf_pos(mw[k] & 0xffffu) ? v[2 * k] : 0.f;
        w[2 * k + 1] = bf_pos(mw[k] >> 16) ? v[2 * k + 1] : 0.f;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) w[k] = EPI == kEpiRelu ? fmaxf(v[k], 0.f) : v[k];
    }
    uint4* o = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(a.out) + vox * kC);
    o[0] = make_uint4(pack_bf2(w[0], w[1]), pack_bf2(w[2], w[3]), pack_bf2(w[4], w[5]), pack_bf2(w[6], w[7]));
    o[1] = make_uint4(pack_bf2(w[8], w[9]), pack_bf2(w[10], w[11]), pack_bf2(w[12], w[13]), pack_bf2(w[14], w[15]));
  }
}

// Persistent implicit-GEMM convolution (see the file comment).  map4 /
// map2 fetch four / two z-planes of the three copies.
template <int EPI>
__global__ void __launch_bounds__(kConvThreads) k_conv(const __grid_constant__ CUtensorMap map4,
                                                     const __grid_constant__ CUtensorMap map2,
                                                     const uint4* __restrict__ wpack, ConvArgs a) {
  extern __shared__ unsigned char dsm[];
  __shared__ __align__(8) uint64_t bar_ld;
  __shared__ __align__(8) uint64_t bar_mma;
  __shared__ uint32_t tmem_slot;
  const uint32_t pad = (256u - (smem_u32(dsm) & 255u)) & 255u;
  unsigned char* sW = dsm + pad;
  uint32_t* sD = reinterpret_cast<uint32_t*>(sW + kDescOff);  // low words: [ph][zi][t] A, then [t] B
  unsigned char* sA = sW + kAOff;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t sW_u = smem_u32(sW), sA_u = smem_u32(sA);

  for (int i = tid; i < kPackBytes / 16; i += kConvThreads) reinterpret_cast<uint4*>(sW)[i] = wpack[i];
  for (int i = tid; i < kDescA + kTaps; i += kConvThreads) {
    if (i < kDescA) {
      const int t = i % kTaps, zi = (i / kTaps) % kTZ, ph = i / (kTaps * kTZ);
      const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
      const int slot = (2 * ph + zi + dz + 1) & (kRing - 1);
      sD[i] = (uint32_t)smem_desc_sw32(sA_u + (uint32_t)((dx + 1) * kCopy + slot * kPlaneZ + (dy + 1) * kTX * 32),
                                       256);
    } else {
      sD[i] = (uint32_t)smem_desc(sW_u + (uint32_t)((i - kDescA) * 512), 256, 128);
    }
  }
  const uint32_t hiA = (uint32_t)(smem_desc_sw32(0, 256) >> 32), hiB = (uint32_t)(smem_desc(0, 256, 128) >> 32);
  fence_proxy_async_smem();
  if (tid == 0) {
    mbar_init(&bar_ld, 1);
    mbar_init(&bar_mma, kTZ);  // one commit per issuing warp
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_slot, kConvCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  constexpr uint32_t idesc = idesc_bf16(128, 16);

  // item = (x tile, y tile, z run, sample)
  auto origin = [&](long long item, int& x0, int& y0, int& zr0, int& n) {
    long long r = item;
    x0 = (int)(r % a.tx) * kTX;
    r /= a.tx;
    y0 = (int)(r % a.ty) * kTY;
    r /= a.ty;
    zr0 = (int)(r % a.nzc) * a.zc;
    n = (int)(r / a.nzc);
  };
  // four planes z0 - 1 .. z0 + 2 (ring slots 0..3) or the two planes z0 + 1,
  // z0 + 2 of the tile starting at z0 (ring slots `slot`, `slot` + 1)
  auto fetch = [&](bool full, int x0, int y0, int z0, int n, int slot) {
    mbar_arrive_expect_tx(&bar_ld, (full ? kRing : 2) * 3 * kPlaneZ);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (full)
        tma_load_5d(sA + c * kCopy, &map4, &bar_ld, 0, x0 + c - 1, y0 - 1, z0 - 1, n);
      else
        tma_load_5d(sA + c * kCopy + slot * kPlaneZ, &map2, &bar_ld, 0, x0 + c - 1, y0 - 1, z0 + 1, n);
    }
  };

  uint32_t phase = 0;
  long long item = blockIdx.x;
  bool pending = false;
  if (tid == 0 && item < a.nitems) {
    int x0, y0, zr0, n;
    origin(item, x0, y0, zr0, n);
    fetch(true, x0, y0, zr0, n, 0);
  }
  pending = item < a.nitems;
  bool stop = false;
  for (; item < a.nitems && !stop; item += gridDim.x) {
    int x0, y0, zr0, n;
    origin(item, x0, y0, zr0, n);
    const int zend = min(zr0 + a.zc, a.nz);
    for (int z0 = zr0, j = 0; z0 < zend; z0 += kTZ, ++j) {
      const int ph = j & 1;
      const bool ok_ld = mbar_wait_bounded(&bar_ld, phase);
      if (__syncthreads_or(!ok_ld)) {
        // a tile that never lands: report it, give the copy in flight a
        // bounded wait, and stop (no MMA reads it)
        if (tid == 0) atomicExch(a.err, 1);
        mbar_wait_bounded(&bar_ld, phase);
        pending = false;
        stop = true;
        break;
      }
      pending = false;
      // lane 0 of warp zi issues the 27 MMAs of output plane zi (its own
      // accumulator columns) and commits them
      if (warp < kTZ && (tid & 31) == 0) {
        tc_fence_after();
        const int zi = warp;
        const uint32_t* dA = sD + (ph * kTZ + zi) * kTaps;
#pragma unroll
        for (int t = 0; t < kTaps; ++t)
          umma_bf16(tmem + (uint32_t)(zi * 16), ((uint64_t)hiA << 32) | dA[t],
                    ((uint64_t)hiB << 32) | sD[kDescA + t], idesc, t > 0 ? 1u : 0u);
        umma_commit(&bar_mma);
      }
      const bool ok_mma = mbar_wait_bounded(&bar_mma, phase);
      if (__syncthreads_or(!ok_mma)) {
        if (tid == 0) atomicExch(a.err, 2);
        mbar_wait_bounded(&bar_mma, phase);
        stop = true;
        break;
      }
      tc_fence_after();
      // the planes this tile alone needed are free: fetch the next ones
      // (the next tile of this run, else the first tile of the next item)
      if (z0 + kTZ < zend) {
        if (tid == 0) fetch(false, x0, y0, z0 + kTZ, n, (2 * (ph ^ 1) + 2) & (kRing - 1));
        pending = true;
      } else if (item + gridDim.x < a.nitems) {
        int x1, y1, zr1, n1;
        origin(item + gridDim.x, x1, y1, zr1, n1);
        if (tid == 0) fetch(true, x1, y1, zr1, n1, 0);
        pending = true;
      }
      const int row = tid;  // TMEM lane = M row = thread (warp w reads lanes 32w .. 32w + 31)
      const int x = x0 + (row & 15), y = y0 + (row >> 4);
#pragma unroll
      for (int zi = 0; zi < kTZ; ++zi) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(zi * 16), v);
        const int z = z0 + zi;
        if (x < a.nx && y < a.ny && z < a.nz)
          store_epi<EPI>(a, (((size_t)n * a.nz + z) * a.ny + y) * a.nx + x, n, v);
      }
      tc_fence_before();
      __syncthreads();
      phase ^= 1;
    }
  }
  // a fetch still in flight after an early exit: bounded wait before the
  // block's shared memory goes away
  if (pending) mbar_wait_bounded(&bar_ld, phase ^ 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kConvCols);
}

// Weight gradient: per-block partial sums of dW over the block's tiles.
// Staged (32-byte swizzled): x as [z][y][18][16 ch] covering x0 - 1 ..
// x0 + 16, g as [z][y][16][16 ch].
__global__ void __launch_bounds__(kWgThreads) k_wgrad(const __grid_constant__ CUtensorMap xmap,
                                                    const __grid_constant__ CUtensorMap gmap, WgArgs a) {
  extern __shared__ unsigned char dsm[];
  __shared__ __align__(8) uint64_t bar;
  const uint32_t pad = (1024u - (smem_u32(dsm) & 1023u)) & 1023u;
  unsigned char* sX = dsm + pad;
  unsigned char* sG = sX + kXTile;
  const uint32_t sX_u = smem_u32(sX), sG_u = smem_u32(sG);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int dz = warp / 3 - 1, dy = warp % 3 - 1;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  float acc[3][2][4];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[j][q][k] = 0.f;
  // ldmatrix row of this lane: matrix mi = lane / 8, row rr = lane % 8.
  // G (B operand): matrix mi = (channel group mi / 2, voxels 8 (mi % 2) ..).
  // X (A operand): matrix mi = (channel group mi % 2, voxels 8 (mi / 2) ..).
  const int mi = lane >> 3, rr = lane & 7;
  const uint32_t gk = (uint32_t)((mi & 1) * 8 + rr), gg = (uint32_t)(mi >> 1);
  const uint32_t xk = (uint32_t)((mi >> 1) * 8 + rr), xg = (uint32_t)(mi & 1);
  uint32_t phase = 0;
  for (long long tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    long long r = tile;
    const int bx = (int)(r % a.tx);
    r /= a.tx;
    const int by = (int)(r % a.ty);
    r /= a.ty;
    const int bz = (int)(r % a.tz);
    const int n = (int)(r / a.tz);
    const int x0 = bx * kWTX, y0 = by * kWTY, z0 = bz * kWTZ;
    if (tid == 0) {
      mbar_arrive_expect_tx(&bar, kXTile + kGTile);
      tma_load_5d(sX, &xmap, &bar, 0, x0 - 1, y0 - 1, z0 - 1, n);
      tma_load_5d(sG, &gmap, &bar, 0, x0, y0, z0, n);
    }
    const bool ok = mbar_wait_bounded(&bar, phase);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(a.err, 3);
      mbar_wait_bounded(&bar, phase);
      break;
    }
#pragma unroll 2
    for (int line = 0; line < kWTY * kWTZ; ++line) {
      const int yi = line % kWTY, zi = line / kWTY;
      uint32_t b[4];
      ldsm_x4_trans(sG_u + sw32((uint32_t)((zi * kWTY + yi) * kWTX) + gk, gg), b);
      const uint32_t xl = (uint32_t)(((zi + dz + 1) * (kWTY + 2) + (yi + dy + 1)) * (kWTX + 2));
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        uint32_t av[4];
        ldsm_x4_trans(sX_u + sw32(xl + xk + (uint32_t)j, xg), av);
        mma_16816(acc[j][0], av, b[0], b[1]);
        mma_16816(acc[j][1], av, b[2], b[3]);
      }
    }
    __syncthreads();
    phase ^= 1;
  }
  // accumulator fragment: c0, c1 = (row g, cols 2q, 2q+1), c2, c3 = row g + 8
  float* P = a.partials + (size_t)blockIdx.x * kWElems;
  const int g = lane >> 2, c2 = (lane & 3) * 2;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int t = 3 * warp + j;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int co = q * 8 + c2;
      *reinterpret_cast<float2*>(P + (t * kC + g) * kC + co) = make_float2(acc[j][q][0], acc[j][q][1]);
      *reinterpret_cast<float2*>(P + (t * kC + g + 8) * kC + co) = make_float2(acc[j][q][2], acc[j][q][3]);
    }
  }
}

__global__ void k_wgrad_reduce(const float* __restrict__ partials, int nblocks, float* __restrict__ dw, float scale,
                               int accumulate) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kWElems) return;
  float s = 0.f;
  for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * kWElems + e];
  dw[e] = (accumulate ? dw[e] : 0.f) + scale * s;
}

// ---------------------------------------------------------------------------
// glue kernels; one thread per (voxel, channel group of 8) = one uint4
__device__ __forceinline__ void unpack8(uint4 u, float (&f)[8]) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 p = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[k]));
    f[2 * k] = p.x;
    f[2 * k + 1] = p.y;
  }
}
__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
  return make_uint4(pack_bf2(f[0], f[1]), pack_bf2(f[2], f[3]), pack_bf2(f[4], f[5]), pack_bf2(f[6], f[7]));
}
__device__ __forceinline__ void mask8(uint4 act, float (&f)[8]) {
  const uint32_t w[4] = {act.x, act.y, act.z, act.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (!bf_pos(w[k] & 0xffffu)) f[2 * k] = 0.f;
    if (!bf_pos(w[k] >> 16)) f[2 * k + 1] = 0.f;
  }
}

// index helpers: element (n, z, y, x, group) of a level with dims (nx, ny, nz)
struct Lv {
  int nx, ny, nz;
  __device__ size_t u4(size_t n, int z, int y, int x, int g) const {
    return ((((n * nz + z) * ny + y) * nx + x) << 1) + g;
  }
};

__global__ void k_pool(const uint4* __restrict__ fine, uint4* __restrict__ coarse, Lv F, Lv Cc, size_t total) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int g = (int)(i & 1);
    size_t v = i >> 1;
    const int x = (int)(v % Cc.nx);
    v /= Cc.nx;
    const int y = (int)(v % Cc.ny);
    v /= Cc.ny;
    const int z = (int)(v % Cc.nz);
    const size_t n = v / Cc.nz;
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      float f[8];
      unpack8(fine[F.u4(n, 2 * z + (c >> 2), 2 * y + ((c >> 1) & 1), 2 * x + (c & 1), g)], f);
#pragma unroll
      for (int k = 0; k < 8; ++k) s[k] += f[k];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] *= 0.125f;
    coarse[i] = pack8(s);
  }
}

__global__ void k_up_add(const uint4* __restrict__ coarse, const uint4* __restrict__ fine, uint4* __restrict__ out,
                         Lv F, Lv Cc, size_t total) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int g = (int)(i & 1);
    size_t v = i >> 1;
    const int x = (int)(v % F.nx);
    v /= F.nx;
    const int y = (int)(v % F.ny);
    v /= F.ny;
    const int z = (int)(v % F.nz);
    const size_t n = v / F.nz;
    float a[8], b[8];
    unpack8(coarse[Cc.u4(n, z >> 1, y >> 1, x >> 1, g)], a);
    unpack8(fine[i], b);
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] += b[k];
    out[i] = pack8(a);
  }
}

__global__ void k_upbwd_mask(const uint4* __restrict__ gfine, const uint4* __restrict__ act, uint4* __restrict__ out,
                             Lv F, Lv Cc, size_t total) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int g = (int)(i & 1);
    size_t v = i >> 1;
    const int x = (int)(v % Cc.nx);
    v /= Cc.nx;
    const int y = (int)(v % Cc.ny);
    v /= Cc.ny;
    const int z = (int)(v % Cc.nz);
    const size_t n = v / Cc.nz;
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      float f[8];
      unpack8(gfine[F.u4(n, 2 * z + (c >> 2), 2 * y + ((c >> 1) & 1), 2 * x + (c & 1), g)], f);
#pragma unroll
      for (int k = 0; k < 8; ++k) s[k] += f[k];
    }
    mask8(act[i], s);
    out[i] = pack8(s);
  }
}

__global__ void k_poolbwd_add_mask(const uint4* __restrict__ gskip, const uint4* __restrict__ gcoarse,
                                   const uint4* __restrict__ act, uint4* __restrict__ out, Lv F, Lv Cc,
                                   size_t total) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int g = (int)(i & 1);
    size_t v = i >> 1;
    const int x = (int)(v % F.nx);
    v /= F.nx;
    const int y = (int)(v % F.ny);
    v /= F.ny;
    const int z = (int)(v % F.nz);
    const size_t n = v / F.nz;
    float a[8], b[8];
    unpack8(gskip[i], a);
    unpack8(gcoarse[Cc.u4(n, z >> 1, y >> 1, x >> 1, g)], b);
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] += 0.125f * b[k];
    mask8(act[i], a);
    out[i] = pack8(a);
  }
}

__device__ __forceinline__ const float* field(const float* base, const Fields& f, int n) {
  const size_t s = f.idx ? (size_t)f.idx[n] : (size_t)n;
  return base + s * f.stride;
}

// per-sample sums of squares of b (blockIdx.z = 0) and p (= 1): grid
// (blocks, n, 2), partials[(field * n + sample) * blocks + block]
__global__ void k_sumsq(Fields f, size_t vox, float* __restrict__ partials) {
  __shared__ double sh[32];
  const float* a = field(blockIdx.z ? f.p : f.b, f, blockIdx.y);
  float acc = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < vox; i += (size_t)gridDim.x * blockDim.x)
    acc = fmaf(a[i], a[i], acc);
  const double t = block_sum((double)acc, sh);
  if (threadIdx.x == 0) partials[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = (float)t;
}

// rms / inverse rms per (field, sample), pooled over the samples if asked;
// 1 for an all-zero field
__global__ void k_rms_final(const float* __restrict__ partials, int nblk, size_t vox, int n, int pooled,
                            float* __restrict__ rms, float* __restrict__ inv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n) return;
  const int fld = i / n, s = i % n;
  double acc = 0.0;
  const int s0 = pooled ? 0 : s, s1 = pooled ? n : s + 1;
  for (int q = s0; q < s1; ++q)
    for (int b = 0; b < nblk; ++b) acc += (double)partials[(fld * n + q) * nblk + b];
  const double r = sqrt(acc / ((double)vox * (s1 - s0)));
  rms[i] = r > 0.0 ? (float)r : 1.f;
  inv[i] = r > 0.0 ? (float)(1.0 / r) : 1.f;
}

__global__ void k_pack_input(Fields f, const float* __restrict__ inv, uint4* __restrict__ x0, size_t vox, int n) {
  const size_t total = vox * (size_t)n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(i / vox);
    const size_t v = i - (size_t)s * vox;
    const float bv = field(f.b, f, s)[v] * inv[s], pv = field(f.p, f, s)[v] * inv[n + s];
    x0[2 * i] = make_uint4(pack_bf2(bv, pv), 0u, 0u, 0u);
    x0[2 * i + 1] = make_uint4(0u, 0u, 0u, 0u);
  }
}

__global__ void k_loss_grad(const float* __restrict__ y, Fields f, const float* __restrict__ inv,
                            uint4* __restrict__ gy, size_t vox, int n, double* __restrict__ partials) {
  __shared__ double sh[32];
  const size_t total = vox * (size_t)n;
  float acc = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(i / vox);
    const size_t v = i - (size_t)s * vox;
    const float d = y[i] - field(f.t, f, s)[v] * inv[s];
    acc = fmaf(d, d, acc);
    gy[2 * i] = make_uint4(pack_bf2(d, 0.f), 0u, 0u, 0u);
    gy[2 * i + 1] = make_uint4(0u, 0u, 0u, 0u);
  }
  const double t = block_sum((double)acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void k_sum_partials(const double* __restrict__ partials, int nblk, double scale,
                               double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += partials[b];
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = scale * t;
}

// (A_crop v)_c * h^2 on a fluid cell c: sum over fluid face neighbours n in
// the crop of (v_c - v_n).
__device__ __forceinline__ float crop_stencil(const float* v, const float* fl, size_t i, int x, int y, int z, int nx,
                                              int ny, int nz) {
  const size_t sy = (size_t)nx, sz = (size_t)nx * ny;
  const float vc = v[i];
  float acc = 0.f;
  auto nb = [&](bool inside, size_t j) {
    if (inside && (!fl || fl[j] > 0.5f)) acc += vc - v[j];
  };
  nb(x > 0, i - 1);
  nb(x < nx - 1, i + 1);
  nb(y > 0, i - sy);
  nb(y < ny - 1, i + sy);
  nb(z > 0, i - sz);
  nb(z < nz - 1, i + sz);
  return acc;
}

__global__ void k_residual(const float* __restrict__ y, Fields f, const float* __restrict__ inv, int nx, int ny,
                           int nz, int n, float inv_h2, float* __restrict__ r, double* __restrict__ partials) {
  __shared__ double sh[32];
  const size_t vox = (size_t)nx * ny * nz, total = vox * n;
  float acc = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(i / vox);
    const size_t v = i - (size_t)s * vox;
    const int x = (int)(v % nx), yy = (int)((v / nx) % ny), z = (int)(v / ((size_t)nx * ny));
    const float* fl = f.fluid ? field(f.fluid, f, s) : nullptr;
    const bool inner = x > 0 && x < nx - 1 && yy > 0 && yy < ny - 1 && z > 0 && z < nz - 1;
    float rv = 0.f;
    if (inner && (!fl || fl[v] > 0.5f)) {
      rv = crop_stencil(y + (size_t)s * vox, fl, v, x, yy, z, nx, ny, nz) * inv_h2 - field(f.b, f, s)[v] * inv[s];
      acc = fmaf(rv, rv, acc);
    }
    r[i] = rv;
  }
  const double t = block_sum((double)acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void k_apply_crop(const float* __restrict__ r, Fields f, int nx, int ny, int nz, int n, float inv_h2,
                             uint4* __restrict__ gy) {
  const size_t vox = (size_t)nx * ny * nz, total = vox * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(i / vox);
    const size_t v = i - (size_t)s * vox;
    const int x = (int)(v % nx), yy = (int)((v / nx) % ny), z = (int)(v / ((size_t)nx * ny));
    const float* fl = f.fluid ? field(f.fluid, f, s) : nullptr;
    float g = 0.f;
    if (!fl || fl[v] > 0.5f) g = crop_stencil(r + (size_t)s * vox, fl, v, x, yy, z, nx, ny, nz) * inv_h2;
    gy[2 * i] = make_uint4(pack_bf2(g, 0.f), 0u, 0u, 0u);
    gy[2 * i + 1] = make_uint4(0u, 0u, 0u, 0u);
  }
}

// fwd operand: [t][ci / 8][co][ci % 8]; data-gradient operand: tap 26 - t,
// [co / 8][ci][co % 8] (K = output channel, N = input channel).
__global__ void k_adam_pack(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ grad, int update, AdamArgs a, __nv_bfloat16* __restrict__ wf,
                            __nv_bfloat16* __restrict__ wd) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kLayers * kWElems) return;
  float wv = w[e];
  if (update) {
    const float g = grad[e];
    const float mv = a.b1 * m[e] + a.omb1 * g;
    const float vv = a.b2 * v[e] + a.omb2 * g * g;
    m[e] = mv;
    v[e] = vv;
    wv -= a.lr * (mv * a.c1) / (sqrtf(vv * a.c2) + a.eps);
    w[e] = wv;
  }
  const int k = e / kWElems, rem = e % kWElems;
  const int t = rem / (kC * kC), ci = (rem / kC) % kC, co = rem % kC;
  const __nv_bfloat16 h = __float2bfloat16_rn(wv);
  const size_t lb = (size_t)k * kTaps;
  wf[((lb + t) * 2 + (ci >> 3)) * 128 + co * 8 + (ci & 7)] = h;
  wd[((lb + (kTaps - 1 - t)) * 2 + (co >> 3)) * 128 + ci * 8 + (co & 7)] = h;
}

__global__ void k_pack_layer(const float* __restrict__ w, __nv_bfloat16* __restrict__ wf,
                             __nv_bfloat16* __restrict__ wd) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kWElems) return;
  const int t = e / (kC * kC), ci = (e / kC) % kC, co = e % kC;
  const __nv_bfloat16 h = __float2bfloat16_rn(w[e]);
  wf[(t * 2 + (ci >> 3)) * 128 + co * 8 + (ci & 7)] = h;
  wd[((kTaps - 1 - t) * 2 + (co >> 3)) * 128 + ci * 8 + (co & 7)] = h;
}

__global__ void k_crop(const float* __restrict__ b, const float* __restrict__ p_next, const float* __restrict__ dp,
                       const uint8_t* __restrict__ solid, long long fx, long long fy, long long cx, long long cy,
                       long long cz, long long ox, long long oy, long long oz, float* __restrict__ dst) {
  const size_t vox = (size_t)(cx * cy * cz);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < vox; i += (size_t)gridDim.x * blockDim.x) {
    const long long x = (long long)(i % cx), y = (long long)((i / cx) % cy), z = (long long)(i / (cx * cy));
    const size_t src = (size_t)(((z + oz) * fy + (y + oy)) * fx + (x + ox));
    const float d = dp[src];
    dst[i] = b[src];
    dst[vox + i] = p_next[src] - d;
    dst[2 * vox + i] = d;
    dst[3 * vox + i] = (solid && solid[src]) ? 0.f : 1.f;
  }
}

// Resident blocks of `kernel` on all SMs, from its shared memory (dynamic +
// static + the per-block reservation), registers and threads.
template <typename K>
int occupancy_blocks(K kernel, int threads, size_t smem) {
  int dev = 0, nsm = 0, smem_sm = 0, reserved = 0, regs_sm = 0, thr_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return nsm;
  const size_t per_block = smem + fa.sharedSizeBytes + (size_t)reserved;
  int occ = (int)((size_t)smem_sm / per_block);
  const int regs_block = ((fa.numRegs * 32 + 255) / 256) * 256 * ((threads + 31) / 32);
  if (regs_block > 0) occ = std::min(occ, regs_sm / regs_block);
  occ = std::min(occ, thr_sm / threads);
  return nsm * std::max(occ, 1);
}

int grid_1d(size_t work, int threads = 256) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = (work + threads - 1) / threads;
  const size_t cap = (size_t)nsm * 8;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

std::atomic<int64_t> g_launches{0};

bool encode_act(CUtensorMap* m, const void* base, const Dims& d, int bx, int by, int bz) {
  auto fn = (PFN_cuTensorMapEncodeTiled_v12000)tensor_map_encoder();
  if (!fn || ((uintptr_t)base & 15)) return false;
  cuuint64_t gdim[5] = {(cuuint64_t)kC, (cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz, (cuuint64_t)d.n};
  cuuint64_t gstride[4] = {(cuuint64_t)kC * 2, (cuuint64_t)kC * 2 * d.nx, (cuuint64_t)kC * 2 * d.nx * d.ny,
                           (cuuint64_t)kC * 2 * d.nx * d.ny * d.nz};
  cuuint32_t box[5] = {(cuuint32_t)kC, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 1};
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), gdim, gstride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename K>
static int grid_for(K kernel, int threads, int smem) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return -1;
  return occupancy_blocks(kernel, threads, smem);
}

template <int EPI>
static cudaError_t conv_epi(const CUtensorMap& m4, const CUtensorMap& m2, const void* wpack, ConvArgs a,
                            cudaStream_t s) {
  static int grid_cache = 0;
  if (!grid_cache) grid_cache = grid_for(k_conv<EPI>, kConvThreads, kConvSmem);
  if (grid_cache < 0) return cudaErrorInvalidValue;
  // z-runs: long enough to amortise the four-plane start, short enough for
  // about three items per resident block
  const long long columns = (long long)a.tx * a.ty * a.nn;
  long long zc = (a.nz * columns + 3LL * grid_cache - 1) / (3LL * grid_cache);
  zc = std::max(2LL, std::min(32LL, (zc + 1) / 2 * 2));
  a.zc = (int)zc;
  a.nzc = (int)((a.nz + zc - 1) / zc);
  a.nitems = columns * a.nzc;
  const long long g = a.nitems < grid_cache ? a.nitems : grid_cache;
  k_conv<EPI><<<(unsigned)(g > 0 ? g : 1), kConvThreads, kConvSmem, s>>>(m4, m2, (const uint4*)wpack, a);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_conv(const void* x, const void* wpack, void* out, int epi, const void* mask, const float* scale,
                        const Dims& d, int* err, cudaStream_t s) {
  if (d.n <= 0 || d.vox() == 0) return cudaSuccess;
  CUtensorMap m4, m2;
  if (!encode_act(&m4, x, d, kTX, kTY + 2, kRing) || !encode_act(&m2, x, d, kTX, kTY + 2, 2))
    return cudaErrorInvalidValue;
  ConvArgs a;
  a.nx = d.nx;
  a.ny = d.ny;
  a.nz = d.nz;
  a.nn = d.n;
  a.tx = (d.nx + kTX - 1) / kTX;
  a.ty = (d.ny + kTY - 1) / kTY;
  a.zc = a.nzc = 0;
  a.nitems = 0;
  a.out = out;
  a.mask = (const __nv_bfloat16*)mask;
  a.scale = scale;
  a.err = err;
  switch (epi) {
    case kEpiF32: return conv_epi<kEpiF32>(m4, m2, wpack, a, s);
    case kEpiRelu: return conv_epi<kEpiRelu>(m4, m2, wpack, a, s);
    case kEpiLin: return conv_epi<kEpiLin>(m4, m2, wpack, a, s);
    case kEpiMask: return conv_epi<kEpiMask>(m4, m2, wpack, a, s);
    case kEpiOut0: return conv_epi<kEpiOut0>(m4, m2, wpack, a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_wgrad(const void* x, const void* g, float* partials, int max_blocks, int* nblocks, const Dims& d,
                         int* err, cudaStream_t s) {
  static int grid_cache = 0;
  if (!grid_cache) grid_cache = grid_for(k_wgrad, kWgThreads, kWgSmem);
  if (grid_cache < 0) return cudaErrorInvalidValue;
  CUtensorMap xm, gm;
  if (!encode_act(&xm, x, d, kWTX + 2, kWTY + 2, kWTZ + 2) || !encode_act(&gm, g, d, kWTX, kWTY, kWTZ))
    return cudaErrorInvalidValue;
  WgArgs a;
  a.nx = d.nx;
  a.ny = d.ny;
  a.nz = d.nz;
  a.nn = d.n;
  a.tx = (d.nx + kWTX - 1) / kWTX;
  a.ty = (d.ny + kWTY - 1) / kWTY;
  a.tz = (d.nz + kWTZ - 1) / kWTZ;
  a.ntiles = (long long)a.tx * a.ty * a.tz * d.n;
  a.partials = partials;
  a.err = err;
  long long gsz = a.ntiles < grid_cache ? a.ntiles : grid_cache;
  if (gsz > max_blocks) gsz = max_blocks;
  if (gsz < 1) gsz = 1;
  *nblocks = (int)gsz;
  k_wgrad<<<(unsigned)gsz, kWgThreads, kWgSmem, s>>>(xm, gm, a);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_wgrad_reduce(const float* partials, int nblocks, float* dw, float scale, bool accumulate,
                                cudaStream_t s) {
  k_wgrad_reduce<<<(kWElems + 255) / 256, 256, 0, s>>>(partials, nblocks, dw, scale, accumulate ? 1 : 0);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

static Lv lv_of(const Dims& d, int shift) { return Lv{d.nx >> shift, d.ny >> shift, d.nz >> shift}; }

cudaError_t launch_pool(const void* fine, void* coarse, const Dims& d, cudaStream_t s) {
  const size_t total = d.vox() / 8 * d.n * 2;
  k_pool<<<grid_1d(total), 256, 0, s>>>((const uint4*)fine, (uint4*)coarse, lv_of(d, 0), lv_of(d, 1), total);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_up_add(const void* coarse, const void* fine, void* out, const Dims& d, cudaStream_t s) {
  const size_t total = d.vox() * d.n * 2;
  k_up_add<<<grid_1d(total), 256, 0, s>>>((const uint4*)coarse, (const uint4*)fine, (uint4*)out, lv_of(d, 0),
                                          lv_of(d, 1), total);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_upbwd_mask(const void* gfine, const void* act_coarse, void* out_coarse, const Dims& d,
                              cudaStream_t s) {
  const size_t total = d.vox() / 8 * d.n * 2;
  k_upbwd_mask<<<grid_1d(total), 256, 0, s>>>((const uint4*)gfine, (const uint4*)act_coarse, (uint4*)out_coarse,
                                              lv_of(d, 0), lv_of(d, 1), total);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_poolbwd_add_mask(const void* gskip, const void* gcoarse, const void* act, void* out,
                                    const Dims& d, cudaStream_t s) {
  const size_t total = d.vox() * d.n * 2;
  k_poolbwd_add_mask<<<grid_1d(total), 256, 0, s>>>((const uint4*)gskip, (const uint4*)gcoarse, (const uint4*)act,
                                                    (uint4*)out, lv_of(d, 0), lv_of(d, 1), total);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_rms(const Fields& f, const Dims& d, bool pooled, float* partials, float* rms, float* inv_rms,
                       cudaStream_t s) {
  const int nblk = 64;
  k_sumsq<<<dim3(nblk, d.n, 2), 256, 0, s>>>(f, d.vox(), partials);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_rms_final<<<(2 * d.n + 127) / 128, 128, 0, s>>>(partials, nblk, d.vox(), d.n, pooled ? 1 : 0, rms, inv_rms);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_pack_input(const Fields& f, const float* inv_rms, void* x0, const Dims& d, cudaStream_t s) {
  k_pack_input<<<grid_1d(d.vox() * d.n), 256, 0, s>>>(f, inv_rms, (uint4*)x0, d.vox(), d.n);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_loss_grad(const float* y, const Fields& f, const float* inv_rms, void* gy, double* partials,
                             double* loss, const Dims& d, cudaStream_t s) {
  const int g = grid_1d(d.vox() * d.n);
  k_loss_grad<<<g, 256, 0, s>>>(y, f, inv_rms, (uint4*)gy, d.vox(), d.n, partials);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_sum_partials<<<1, 256, 0, s>>>(partials, g, 0.5 / ((double)d.vox() * d.n), loss);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_residual_loss_grad(const float* y, const Fields& f, const float* inv_rms, float inv_h2, float* r,
                                      void* gy, double* partials, double* loss, const Dims& d, cudaStream_t s) {
  const int g = grid_1d(d.vox() * d.n);
  k_residual<<<g, 256, 0, s>>>(y, f, inv_rms, d.nx, d.ny, d.nz, d.n, inv_h2, r, partials);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_sum_partials<<<1, 256, 0, s>>>(partials, g, 0.5 / ((double)d.vox() * d.n), loss);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  k_apply_crop<<<g, 256, 0, s>>>(r, f, d.nx, d.ny, d.nz, d.n, inv_h2, (uint4*)gy);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_adam_pack(float* w, float* m, float* v, const float* grad, bool update, AdamArgs a, void* wf,
                             void* wd, cudaStream_t s) {
  k_adam_pack<<<(kLayers * kWElems + 255) / 256, 256, 0, s>>>(w, m, v, grad, update ? 1 : 0, a,
                                                              (__nv_bfloat16*)wf, (__nv_bfloat16*)wd);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_crop(const float* b, const float* p_next, const float* dp, const uint8_t* solid,
                        const int64_t full[3], const int64_t crop[3], const int64_t origin[3], float* dst,
                        cudaStream_t s) {
  const size_t vox = (size_t)(crop[0] * crop[1] * crop[2]);
  k_crop<<<grid_1d(vox), 256, 0, s>>>(b, p_next, dp, solid, full[0], full[1], crop[0], crop[1], crop[2], origin[0],
                                      origin[1], origin[2], dst);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_pack_layer(const float* w, void* wf, void* wd, cudaStream_t s) {
  k_pack_layer<<<(kWElems + 255) / 256, 256, 0, s>>>(w, (__nv_bfloat16*)wf, (__nv_bfloat16*)wd);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace gn
}  // namespace npmg
