// Level kernels of the multigrid cycle (Sec. 2.2): launchers and the
// single-pass building blocks used by the per-kernel entry points.
#include <type_traits>

#include "launch.h"
#include "mg_kernels.cuh"

namespace npmg {

template <int DIM>
static dim3 tile_grid(const LevelDev& L) {
  using TS = TileShape<DIM>;
  return dim3((L.nx + TS::X - 1) / TS::X, (L.ny + TS::Y - 1) / TS::Y, DIM == 3 ? (L.nz + TS::Z - 1) / TS::Z : 1);
}

template <int DIM>
static size_t tile_smem(int halo) {
  using TS = TileShape<DIM>;
  const int h = halo > 0 ? halo : 1;
  const size_t R = (size_t)(TS::X + 2 * h) * (TS::Y + 2 * h) * (DIM == 3 ? TS::Z + 2 * h : 1);
  return 3 * R * sizeof(float) + ((R + 15) & ~size_t(15));
}

// Opt the kernel in to the device's largest dynamic shared memory.  A fixed
// maximum (rather than this handle's size) keeps handles of different sizes
// from lowering each other's limit; the launch still asks only for `bytes`.
template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (bytes + 1024 > (size_t)optin) return cudaErrorInvalidValue;
  // static shared memory of the reductions comes on top of the dynamic part
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024);
}

// Two sweeps (the default) use the compile-time-halo instantiation.
template <int DIM, typename T, bool MASKED, typename TB>
cudaError_t launch_down(const LevelDev& L, const void* b, void* x, void* bcoarse, int pre, float omega,
                        const SolveState* st, cudaStream_t s) {
  const size_t sm = tile_smem<DIM>(pre);
  if (pre == 2)
    return launch_chain(k_down<DIM, 2, T, MASKED, TB>, tile_grid<DIM>(L), kThreads, sm, s, L, (const TB*)b, (T*)x,
                        (T*)bcoarse, pre, omega, st);
  return launch_chain(k_down<DIM, 0, T, MASKED, TB>, tile_grid<DIM>(L), kThreads, sm, s, L, (const TB*)b, (T*)x,
                      (T*)bcoarse, pre, omega, st);
}

template <int DIM, typename T, bool MASKED, bool FINEST, typename TB>
cudaError_t launch_up(const LevelDev& L, const void* b, const void* xin, void* xout, const void* e, int post,
                      float omega, float sc, SolveState* st, double* partials, cudaStream_t s) {
  const size_t sm = tile_smem<DIM>(post);
  if (post == 2)
    return launch_chain(k_up<DIM, 2, T, MASKED, FINEST, TB>, tile_grid<DIM>(L), kThreads, sm, s, L, (const TB*)b,
                        (const T*)xin, (TB*)xout, (const T*)e, post, omega, sc, st, partials);
  return launch_chain(k_up<DIM, 0, T, MASKED, FINEST, TB>, tile_grid<DIM>(L), kThreads, sm, s, L, (const TB*)b,
                      (const T*)xin, (TB*)xout, (const T*)e, post, omega, sc, st, partials);
}

// ---------------------------------------------------------------------------
// Sawtooth down leg (App. B): no sweeps.  Every cell gets x = b / d (one
// Jacobi step from a zero guess, for the up leg) and every coarse cell the
// 2x2(x2) average of b over its fluid children (the residual of x = 0).
// There is no stencil, so the kernel is a plain stream: one thread per
// coarse cell reads its children as pairs along x (coalesced 2-element
// loads; levels with a down leg have even sides), in a grid-stride loop
// over a grid of 8 blocks per SM.
template <typename T> __device__ __forceinline__ float2 ld2(const T* p, size_t i);
template <> __device__ __forceinline__ float2 ld2<float>(const float* p, size_t i) {
  return *reinterpret_cast<const float2*>(p + i);
}
template <> __device__ __forceinline__ float2 ld2<__half>(const __half* p, size_t i) {
  return __half22float2(*reinterpret_cast<const __half2*>(p + i));
}
template <> __device__ __forceinline__ float2 ld2<__nv_bfloat16>(const __nv_bfloat16* p, size_t i) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p + i));
}
template <typename T> __device__ __forceinline__ void st2(T* p, size_t i, float a, float b);
template <> __device__ __forceinline__ void st2<float>(float* p, size_t i, float a, float b) {
  *reinterpret_cast<float2*>(p + i) = make_float2(a, b);
}
template <> __device__ __forceinline__ void st2<__half>(__half* p, size_t i, float a, float b) {
  *reinterpret_cast<__half2*>(p + i) = __floats2half2_rn(a, b);
}
template <> __device__ __forceinline__ void st2<__nv_bfloat16>(__nv_bfloat16* p, size_t i, float a, float b) {
  *reinterpret_cast<__nv_bfloat162*>(p + i) = __floats2bfloat162_rn(a, b);
}

template <int DIM, typename T, bool MASKED, typename TB>
__global__ void __launch_bounds__(256) k_down_saw(LevelDev L, const TB* __restrict__ b, T* __restrict__ x,
                                                  T* __restrict__ bcoarse, const SolveState* __restrict__ st) {
  chain_enter();
  if (st && st->inner_done) return;
  const int cnx = L.nx >> 1, cny = L.ny >> 1, cnz = DIM == 3 ? L.nz >> 1 : 1;
  const size_t nc = (size_t)cnx * cny * cnz;
  const float inv_children = DIM == 3 ? 0.125f : 0.25f;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (size_t)gridDim.x * blockDim.x) {
    const int cx = (int)(c % cnx);
    const size_t t = c / cnx;
    const int cy = (int)(t % cny), cz = (int)(t / cny);
    const int gx = 2 * cx;
    float sum = 0.f;
#pragma unroll
    for (int az = 0; az < (DIM == 3 ? 2 : 1); ++az)
#pragma unroll
      for (int ay = 0; ay < 2; ++ay) {
        const int gy = 2 * cy + ay, gz = DIM == 3 ? 2 * cz + az : 0;
        const size_t i = gidx(L, gx, gy, gz);
        const float2 bv = ld2(b, i);
        uint8_t m0 = kFluidBit, m1 = kFluidBit;
        if (MASKED) {
          m0 = L.cell[i];
          m1 = L.cell[i + 1];
        }
        const float x0 = m0 ? bv.x / diag_at<DIM, MASKED>(L, gx, gy, gz, m0) : 0.f;
        const float x1 = m1 ? bv.y / diag_at<DIM, MASKED>(L, gx + 1, gy, gz, m1) : 0.f;
        st2(x, i, x0, x1);
        if (m0) sum += bv.x;
        if (m1) sum += bv.y;
      }
    bcoarse[c] = cvt<T>(sum * inv_children);
  }
}

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
      n = 1;
  }
  return n;
}

template <int DIM, typename T, bool MASKED, typename TB>
cudaError_t launch_down_saw(const LevelDev& L, const void* b, void* x, void* bcoarse, const SolveState* st,
                            cudaStream_t s) {
  const size_t nc = (size_t)(L.nx / 2) * (L.ny / 2) * (DIM == 3 ? L.nz / 2 : 1);
  const size_t want = (nc + 255) / 256, cap = (size_t)sm_count() * 8;
  const unsigned blocks = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
  return launch_chain(k_down_saw<DIM, T, MASKED, TB>, dim3(blocks), dim3(256), 0, s, L, (const TB*)b, (T*)x,
                      (T*)bcoarse, st);
}

// Raise the dynamic shared-memory limit of the level kernels once (at
// create, outside any stream capture).
template <int DIM, typename T, bool MASKED, typename TB>
static cudaError_t prepare_level_pair(int pre, int post) {
  cudaError_t e = allow_smem(k_down<DIM, 2, T, MASKED, TB>, tile_smem<DIM>(pre));
  if (e == cudaSuccess) e = allow_smem(k_down<DIM, 0, T, MASKED, TB>, tile_smem<DIM>(pre));
  if (e == cudaSuccess) e = allow_smem(k_up<DIM, 2, T, MASKED, false, TB>, tile_smem<DIM>(post));
  if (e == cudaSuccess) e = allow_smem(k_up<DIM, 2, T, MASKED, true, TB>, tile_smem<DIM>(post));
  if (e == cudaSuccess) e = allow_smem(k_up<DIM, 0, T, MASKED, false, TB>, tile_smem<DIM>(post));
  if (e == cudaSuccess) e = allow_smem(k_up<DIM, 0, T, MASKED, true, TB>, tile_smem<DIM>(post));
  return e;
}

// Both storage pairs of a precision: (T, T) and, for 16-bit T, the finest
// level's (T, float).
template <int DIM, typename T, bool MASKED>
cudaError_t prepare_level_kernels(int pre, int post) {
  cudaError_t e = prepare_level_pair<DIM, T, MASKED, T>(pre, post);
  if (e == cudaSuccess && !std::is_same<T, float>::value) e = prepare_level_pair<DIM, T, MASKED, float>(pre, post);
  return e;
}

#define NPMG_INST_LEVEL_TB(DIM, T, M, TB)                                                                    \
  template cudaError_t launch_down<DIM, T, M, TB>(const LevelDev&, const void*, void*, void*, int, float,      \
                                                  const SolveState*, cudaStream_t);                            \
  template cudaError_t launch_down_saw<DIM, T, M, TB>(const LevelDev&, const void*, void*, void*,              \
                                                      const SolveState*, cudaStream_t);                        \
  template cudaError_t launch_up<DIM, T, M, false, TB>(const LevelDev&, const void*, const void*, void*,      \
                                                       const void*, int, float, float, SolveState*, double*,   \
                                                       cudaStream_t);                                          \
  template cudaError_t launch_up<DIM, T, M, true, TB>(const LevelDev&, const void*, const void*, void*,       \
                                                      const void*, int, float, float, SolveState*, double*,    \
                                                      cudaStream_t);
#define NPMG_INST_LEVEL(DIM, T, M)                                 \
  template cudaError_t prepare_level_kernels<DIM, T, M>(int, int); \
  NPMG_INST_LEVEL_TB(DIM, T, M, T)                                 \
  NPMG_INST_LEVEL_TB(DIM, T, M, float)

#define NPMG_INST_LEVEL_F(DIM, M)                                      \
  template cudaError_t prepare_level_kernels<DIM, float, M>(int, int); \
  NPMG_INST_LEVEL_TB(DIM, float, M, float)
NPMG_INST_LEVEL_F(2, false)
NPMG_INST_LEVEL_F(2, true)
NPMG_INST_LEVEL_F(3, false)
NPMG_INST_LEVEL_F(3, true)
NPMG_INST_LEVEL(2, __half, false)
NPMG_INST_LEVEL(2, __half, true)
NPMG_INST_LEVEL(3, __half, false)
NPMG_INST_LEVEL(3, __half, true)
NPMG_INST_LEVEL(2, __nv_bfloat16, false)
NPMG_INST_LEVEL(2, __nv_bfloat16, true)
NPMG_INST_LEVEL(3, __nv_bfloat16, false)
NPMG_INST_LEVEL(3, __nv_bfloat16, true)

// ---------------------------------------------------------------------------
// Single-pass building blocks (float32), one thread per cell.
template <int DIM>
__device__ __forceinline__ bool cell_coords(const LevelDev& L, size_t i, int& x, int& y, int& z) {
  x = (int)(i % L.nx);
  const size_t t = i / L.nx;
  y = (int)(t % L.ny);
  z = (int)(t / L.ny);
  return true;
}

template <int DIM, bool MASKED>
__device__ __forceinline__ float apply_at(const LevelDev& L, const float* __restrict__ x, size_t i, int cx, int cy,
                                          int cz, uint8_t m) {
  const float d = diag_at<DIM, MASKED>(L, cx, cy, cz, m);
  float nb = 0.f;
  if (cx > 0) nb += L.wx * x[i - 1];
  if (cx < L.nx - 1) nb += L.wx * x[i + 1];
  if (cy > 0) nb += L.wy * x[i - L.nx];
  if (cy < L.ny - 1) nb += L.wy * x[i + L.nx];
  if (DIM == 3) {
    const size_t sxy = (size_t)L.nx * L.ny;
    if (cz > 0) nb += L.wz * x[i - sxy];
    if (cz < L.nz - 1) nb += L.wz * x[i + sxy];
  }
  return d * x[i] - nb;
}

template <int DIM, bool MASKED>
__global__ void k_apply(LevelDev L, const float* __restrict__ x, float* __restrict__ y) {
  const size_t n = (size_t)L.nx * L.ny * L.nz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    int cx, cy, cz;
    cell_coords<DIM>(L, i, cx, cy, cz);
    const uint8_t m = MASKED ? L.cell[i] : kFluidBit;
    y[i] = m ? apply_at<DIM, MASKED>(L, x, i, cx, cy, cz, m) : 0.f;
  }
}

template <int DIM, bool MASKED>
__global__ void k_smooth_once(LevelDev L, const float* __restrict__ x, float* __restrict__ y,
                              const float* __restrict__ b, float omega) {
  const size_t n = (size_t)L.nx * L.ny * L.nz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    int cx, cy, cz;
    cell_coords<DIM>(L, i, cx, cy, cz);
    const uint8_t m = MASKED ? L.cell[i] : kFluidBit;
    float v = 0.f;
    if (m) {
      const float d = diag_at<DIM, MASKED>(L, cx, cy, cz, m);
      v = x[i] + omega * (b[i] - apply_at<DIM, MASKED>(L, x, i, cx, cy, cz, m)) / d;
    }
    y[i] = v;
  }
}

template <int DIM, bool MASKED>
__global__ void k_restrict_residual(LevelDev L, const float* __restrict__ x, const float* __restrict__ b,
                                    float* __restrict__ bc) {
  const int cnx = L.nx / 2, cny = L.ny / 2, cnz = DIM == 3 ? L.nz / 2 : 1;
  const size_t n = (size_t)cnx * cny * cnz;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x) {
    const int X = (int)(j % cnx);
    const size_t t = j / cnx;
    const int Y = (int)(t % cny);
    const int Z = (int)(t / cny);
    float sum = 0.f;
    for (int az = 0; az < (DIM == 3 ? 2 : 1); ++az)
      for (int ay = 0; ay < 2; ++ay)
        for (int ax = 0; ax < 2; ++ax) {
          const int cx = 2 * X + ax, cy = 2 * Y + ay, cz = DIM == 3 ? 2 * Z + az : 0;
          const size_t i = gidx(L, cx, cy, cz);
          const uint8_t m = MASKED ? L.cell[i] : kFluidBit;
          if (m) sum += b[i] - apply_at<DIM, MASKED>(L, x, i, cx, cy, cz, m);
        }
    bc[j] = sum * (DIM == 3 ? 0.125f : 0.25f);
  }
}

template <int DIM, bool MASKED>
__global__ void k_prolong_correct(LevelDev L, const float* __restrict__ e, float* __restrict__ x, float sc) {
  const size_t n = (size_t)L.nx * L.ny * L.nz;
  const int cnx = L.nx / 2, cny = L.ny / 2;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    int cx, cy, cz;
    cell_coords<DIM>(L, i, cx, cy, cz);
    const uint8_t m = MASKED ? L.cell[i] : kFluidBit;
    if (!m) {
      x[i] = 0.f;
      continue;
    }
    const size_t ci = ((size_t)(cz >> 1) * cny + (cy >> 1)) * cnx + (cx >> 1);
    x[i] += sc * e[ci];
  }
}

static int blocks_for(size_t n) {
  size_t b = (n + 255) / 256;
  if (b > 4096) b = 4096;
  if (b < 1) b = 1;
  return (int)b;
}

template <int DIM, bool MASKED>
cudaError_t launch_apply(const LevelDev& L, const float* x, float* y, cudaStream_t s) {
  k_apply<DIM, MASKED><<<blocks_for((size_t)L.nx * L.ny * L.nz), 256, 0, s>>>(L, x, y);
  return cudaGetLastError();
}
template <int DIM, bool MASKED>
cudaError_t launch_smooth_once(const LevelDev& L, const float* x, float* y, const float* b, float omega,
                               cudaStream_t s) {
  k_smooth_once<DIM, MASKED><<<blocks_for((size_t)L.nx * L.ny * L.nz), 256, 0, s>>>(L, x, y, b, omega);
  return cudaGetLastError();
}
template <int DIM, bool MASKED>
cudaError_t launch_restrict_residual(const LevelDev& L, const float* x, const float* b, float* bc, cudaStream_t s) {
  k_restrict_residual<DIM, MASKED><<<blocks_for((size_t)L.nx * L.ny * L.nz / (DIM == 3 ? 8 : 4)), 256, 0, s>>>(
      L, x, b, bc);
  return cudaGetLastError();
}
template <int DIM, bool MASKED>
cudaError_t launch_prolong_correct(const LevelDev& L, const float* e, float* x, float sc, cudaStream_t s) {
  k_prolong_correct<DIM, MASKED><<<blocks_for((size_t)L.nx * L.ny * L.nz), 256, 0, s>>>(L, e, x, sc);
  return cudaGetLastError();
}

#define NPMG_INST_BB(DIM, M)                                                                                  \
  template cudaError_t launch_apply<DIM, M>(const LevelDev&, const float*, float*, cudaStream_t);             \
  template cudaError_t launch_smooth_once<DIM, M>(const LevelDev&, const float*, float*, const float*, float, \
                                                  cudaStream_t);                                              \
  template cudaError_t launch_restrict_residual<DIM, M>(const LevelDev&, const float*, const float*, float*,  \
                                                        cudaStream_t);                                        \
  template cudaError_t launch_prolong_correct<DIM, M>(const LevelDev&, const float*, float*, float, cudaStream_t);

NPMG_INST_BB(2, false)
NPMG_INST_BB(2, true)
NPMG_INST_BB(3, false)
NPMG_INST_BB(3, true)

}  // namespace npmg
