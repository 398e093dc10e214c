// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/npmg.h"

namespace npmg {

constexpr int kMaxLevels = 16;
constexpr int kMaxHalo = 3;            // max Jacobi sweeps fused per tile pass
constexpr int kThreads = 256;          // threads per tile block
constexpr int kHistory = 32;

// Cell byte of a masked level: bit 7 = fluid; bits 0-1, 2-3, 4-5 = number of
// links per axis (x, y, z) that enter the diagonal of A (a fluid neighbour
// inside the domain, or a Dirichlet domain face).  Solid cells hold 0.
constexpr uint8_t kFluidBit = 0x80;

// One grid level as the kernels see it (passed by value).
struct LevelDev {
  int nx, ny, nz;        // cells per axis (nz = 1 in 2D)
  float wx, wy, wz;      // operator weights: c / h_a^2 (c = h_0x^2)
  int bcD;               // bit f set when face f (x-,x+,y-,y+,z-,z+) is Dirichlet
  const uint8_t* cell;   // cell bytes, or nullptr when the level has no solid
};

// Device-resident control block of one solve.  Written by the "last block"
// of the reduction kernels, read by every kernel of the next phase.
struct SolveState {
  // parameters (set at solve start)
  double tol, inner_floor;
  int max_inner, max_outer, krylov, n_fluid;
  // refinement loop
  double bnorm2;         // ||b||^2
  double relres, relres0;
  double sigma;          // d = sigma * d' for the current inner solve
  double eta;            // relative tolerance of the current inner solve
  int outer, outer_done, status, stall;
  double hist[kHistory];
  // inner CG
  int inner_done, it, iters_total, first;
  double r0norm2, rz, rz_old, alpha, beta, rnorm2, pAp;
  // reduction counters (one per reducing kernel family)
  unsigned int counter[8];
  // device-side solve loop: the float-float buffer holding the iterate, and
  // the checks and bodies run by the loop's conditional nodes
  int cur;
  unsigned int loop_checks, loop_bodies, loop_outer;
};

enum Counter { kCntInit = 0, kCntOuter = 1, kCntRZ = 2, kCntPAP = 3, kCntRR = 4, kCntMisc = 5 };

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  The kernels of a solve's launch chain
// (level legs, coarse block, CG updates) are launched with a programmatic
// dependency on the previous one, so that their launch overlaps its drain;
// each first waits until the preceding grid has completed and its writes
// are visible (a no-op when it was launched without the dependency).
// Nothing may be read or written before this call.  No grid releases its
// successor early: measured on GB300, successors parked on the SMs from the
// start of the previous grid made the 2D and 3D solves 5-8% slower (1-7%
// when only grids of at most 32 or 128 blocks release early), while the
// release at exit makes the 2D flow step about 1.5% faster.
__device__ __forceinline__ void chain_enter() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// storage conversions
template <typename T> __device__ __forceinline__ float ld(const T* p, size_t i);
template <> __device__ __forceinline__ float ld<float>(const float* p, size_t i) { return p[i]; }
template <> __device__ __forceinline__ float ld<__half>(const __half* p, size_t i) { return __half2float(p[i]); }
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p, size_t i) { return __bfloat162float(p[i]); }

template <typename T> __device__ __forceinline__ T cvt(float v);
template <> __device__ __forceinline__ float cvt<float>(float v) { return v; }
template <> __device__ __forceinline__ __half cvt<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// ---------------------------------------------------------------------------
// Deterministic reductions: warp shuffles, then a fixed-order block tree;
// grid totals by the last block to finish (fixed-order sum of the partials).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; the result is valid in thread 0.  `sh` holds >= 32
// doubles.  Every thread of the block must call it.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (lane < nw) ? sh[lane] : 0.0;
    v = warp_sum(v);
  }
  return v;
}

__device__ __forceinline__ unsigned linear_block() {
  return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

// Each block contributes `v`; returns true in every thread of the last block
// to arrive, with the grid total in *total (valid in all its threads).
__device__ __forceinline__ bool grid_sum_last(double v, double* partials,
                                              unsigned int* counter,
                                              double* total) {
  __shared__ double sh[32];
  __shared__ bool last;
  __shared__ double tot;
  const double s = block_sum(v, sh);
  const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
  if (threadIdx.x == 0) {
    partials[linear_block()] = s;
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    last = (t == nb - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc = 0.0;
  for (unsigned i = threadIdx.x; i < nb; i += blockDim.x) acc += __ldcg(partials + i);
  const double r = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    tot = r;
    *counter = 0u;
  }
  __syncthreads();
  *total = tot;
  return true;
}

// ---------------------------------------------------------------------------
// Diagonal of the scaled operator at a cell.
__device__ __forceinline__ int axis_count(int g, int n, int bcD, int face_lo) {
  // links along one axis for an unmasked level: 2 inside, minus Neumann faces
  return 2 - ((g == 0) & !((bcD >> face_lo) & 1)) - ((g == n - 1) & !((bcD >> (face_lo + 1)) & 1));
}

template <int DIM, bool MASKED>
__device__ __forceinline__ float diag_at(const LevelDev& L, int gx, int gy, int gz, uint8_t m) {
  if (MASKED) {
    float d = L.wx * (float)(m & 3) + L.wy * (float)((m >> 2) & 3);
    if (DIM == 3) d += L.wz * (float)((m >> 4) & 3);
    return d;
  } else {
    float d = L.wx * (float)axis_count(gx, L.nx, L.bcD, 0) + L.wy * (float)axis_count(gy, L.ny, L.bcD, 2);
    if (DIM == 3) d += L.wz * (float)axis_count(gz, L.nz, L.bcD, 4);
    return d;
  }
}

// Host-side error helper.
void set_error(const char* fmt, ...);

#define NPMG_CUDA(call)                                                        \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      ::npmg::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,             \
                        cudaGetErrorString(e_));                               \
      return MG_ERR_CUDA;                                                      \
    }                                                                          \
  } while (0)

}  // namespace npmg
