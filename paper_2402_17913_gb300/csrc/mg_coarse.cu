// Coarse levels of the cycle in one thread block, and the set-up kernels.
#include <math.h>

#include <stdlib.h>

#include "launch.h"
#include "mg_kernels.cuh"
#include "tma.cuh"
#include "coarse.cuh"

namespace npmg {

static int grid_1d(size_t n, int cap) {
  size_t b = (n + 255) / 256;
  if (b > (size_t)cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// ---------------------------------------------------------------------------
// Below a few thousand cells a level is too small to fill the GPU, so the
// remaining part of the cycle (down legs, the exact coarsest solve, up
// legs) runs inside one block of 1024 threads with every level resident in
// shared memory.  One SM executes it, so it is written for instruction
// count: each level is stored with a zero ghost ring (no bounds checks; the
// ring is the zero padding of Sec. 2.1), the inverse diagonal is computed
// once per launch (0 marks a non-fluid cell), and a sweep is
// x <- (1 - omega) x + omega D^-1 (b + sum_a w_a (x_- + x_+)).  The
// coarsest level is solved exactly up to float32 rounding: its operator is
// inverted once at create (float64 Gauss-Jordan), stored in float32 and
// applied here as a float32 product, a few lanes per row.
// The level table stays in kernel-parameter space (__grid_constant__), so
// indexing it by level needs no local copy.
template <typename T>
__global__ void __launch_bounds__(1024) k_coarse(const __grid_constant__ CoarseArgs a, const T* __restrict__ bin,
                                                 T* __restrict__ xout, SolveState* __restrict__ st,
                                                 int total_floats) {
  chain_enter();
  if (st && st->inner_done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* S = reinterpret_cast<float*>(smem_raw);
  if (a.dim == 3) coarse_cycle<3, T>(a, bin, xout, st, S, total_floats);
  else coarse_cycle<2, T>(a, bin, xout, st, S, total_floats);
}

// Padded shared-memory layout of the single-block kernel for levels
// lv[0 .. nlev-1]: four arrays (x, x', b, 1/diag) per level with a ghost
// ring; returns the bytes needed.
size_t coarse_layout(int* off, const LevelDev* lv, int nlev, int dim) {
  size_t f = 0;
  for (int l = 0; l < nlev; ++l) {
    off[l] = (int)f;
    const size_t P = (size_t)(lv[l].nx + 2) * (lv[l].ny + 2) * (dim == 3 ? lv[l].nz + 2 : 1);
    f += (4 * P + 3) / 4 * 4;
  }
  return f * sizeof(float);
}

// Largest level (cells) the single-block kernel takes: 2048 in 2D and 8192
// in 3D (measured on GB300: the 2048x1024 flow step is 4% faster when the
// 128x64 level runs on the tiled kernels, the 256^3 solve is not), or
// NPMG_COARSE_CELLS (64 .. 8192) to tune it.
static size_t coarse_cells_limit(int dim) {
  const char* e = getenv("NPMG_COARSE_CELLS");
  const long v = e ? atol(e) : 0;
  if (v >= 64 && v <= 8192) return (size_t)v;
  return dim == 3 ? 8192 : 2048;
}

// First level handled by the single-block kernel: levels within the cell
// limit whose padded arrays fit the block's shared memory.
int coarse_start_level(const LevelDev* lv, int L, int dim, size_t smem_limit) {
  int kc = L - 1;
  int off[kMaxLevels];
  const size_t lim = coarse_cells_limit(dim);
  while (kc > 0 && (size_t)lv[kc - 1].nx * lv[kc - 1].ny * lv[kc - 1].nz <= lim &&
         coarse_layout(off, lv + kc - 1, L - kc + 1, dim) <= smem_limit)
    --kc;
  return kc;
}

cudaError_t launch_coarse_image(const CoarseArgs& a, float* image, size_t bytes, cudaStream_t s) {
  // one block: the zeroing must finish before the diagonals are written
  if (a.dim == 3) k_coarse_image<3><<<1, 1024, 0, s>>>(a, image, (int)(bytes / 4));
  else k_coarse_image<2><<<1, 1024, 0, s>>>(a, image, (int)(bytes / 4));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse(const CoarseArgs& a, size_t smem_bytes, const void* b, void* x, SolveState* st,
                          cudaStream_t s) {
  return launch_chain(k_coarse<T>, 1, 1024, smem_bytes, s, a, (const T*)b, (T*)x, st, (int)(smem_bytes / sizeof(float)));
}

template <typename T>
cudaError_t prepare_coarse(size_t smem_bytes) {
  // opt in to the device maximum (see allow_smem in mg_level.cu): handles of
  // different sizes must not lower each other's limit
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (smem_bytes + 1024 > (size_t)optin) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(k_coarse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024);
}
template cudaError_t prepare_coarse<float>(size_t);
template cudaError_t prepare_coarse<__half>(size_t);
template cudaError_t prepare_coarse<__nv_bfloat16>(size_t);
template cudaError_t launch_coarse<float>(const CoarseArgs&, size_t, const void*, void*, SolveState*, cudaStream_t);
template cudaError_t launch_coarse<__half>(const CoarseArgs&, size_t, const void*, void*, SolveState*, cudaStream_t);
template cudaError_t launch_coarse<__nv_bfloat16>(const CoarseArgs&, size_t, const void*, void*, SolveState*,
                                                  cudaStream_t);

// ---------------------------------------------------------------------------
// Set-up kernels (run once in mg_create).
__global__ void k_coarsen_solid(int dim, int nx, int ny, int nz, const uint8_t* __restrict__ sf,
                                uint8_t* __restrict__ sc) {
  const int cnx = nx / 2, cny = ny / 2, cnz = dim == 3 ? nz / 2 : 1;
  const size_t n = (size_t)cnx * cny * cnz;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x) {
    const int X = (int)(j % cnx), Y = (int)((j / cnx) % cny), Z = (int)(j / ((size_t)cnx * cny));
    bool all = true;
    for (int az = 0; az < (dim == 3 ? 2 : 1); ++az)
      for (int ay = 0; ay < 2; ++ay)
        for (int ax = 0; ax < 2; ++ax)
          all = all && sf[((size_t)(2 * Z + az) * ny + (2 * Y + ay)) * nx + (2 * X + ax)];
    sc[j] = all ? 1 : 0;
  }
}

cudaError_t launch_coarsen_solid(int dim, const int64_t f[3], const uint8_t* sf, uint8_t* sc, cudaStream_t s) {
  const size_t n = (size_t)(f[0] / 2) * (f[1] / 2) * (dim == 3 ? f[2] / 2 : 1);
  k_coarsen_solid<<<grid_1d(n, 4096), 256, 0, s>>>(dim, (int)f[0], (int)f[1], (int)f[2], sf, sc);
  return cudaGetLastError();
}

__global__ void k_cell_bytes(int dim, int nx, int ny, int nz, int bcD, const uint8_t* __restrict__ solid,
                             uint8_t* __restrict__ cell) {
  const size_t n = (size_t)nx * ny * nz;
  const size_t sxy = (size_t)nx * ny;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (solid[i]) {
      cell[i] = 0;
      continue;
    }
    const int c[3] = {(int)(i % nx), (int)((i / nx) % ny), (int)(i / sxy)};
    const int N[3] = {nx, ny, nz};
    const size_t stride[3] = {1, (size_t)nx, sxy};
    int byte = kFluidBit;
    for (int a = 0; a < dim; ++a) {
      int k = 0;
      // low side
      if (c[a] > 0) k += solid[i - stride[a]] ? 0 : 1;
      else k += ((bcD >> (2 * a)) & 1);
      // high side
      if (c[a] < N[a] - 1) k += solid[i + stride[a]] ? 0 : 1;
      else k += ((bcD >> (2 * a + 1)) & 1);
      byte |= k << (2 * a);
    }
    cell[i] = (uint8_t)byte;
  }
}

cudaError_t launch_cell_bytes(int dim, const int64_t n[3], int bcD, const uint8_t* solid, uint8_t* cell,
                              cudaStream_t s) {
  const size_t N = (size_t)n[0] * n[1] * (dim == 3 ? n[2] : 1);
  k_cell_bytes<<<grid_1d(N, 4096), 256, 0, s>>>(dim, (int)n[0], (int)n[1], dim == 3 ? (int)n[2] : 1, bcD, solid,
                                                cell);
  return cudaGetLastError();
}

// Dense matrix of the coarsest operator (identity rows on solid cells), then
// in-place Gauss-Jordan inversion in float64 by one block (SPD: no pivoting).
__global__ void k_dense_matrix(int dim, int nx, int ny, int nz, double wx, double wy, double wz, int bcD,
                               const uint8_t* __restrict__ cell, double* __restrict__ A) {
  const int n = nx * ny * nz;
  const double w[3] = {wx, wy, wz};
  const int N[3] = {nx, ny, nz};
  const int stride[3] = {1, nx, nx * ny};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = 0.0;
    const bool fl = cell ? cell[i] != 0 : true;
    if (!fl) {
      A[(size_t)i * n + i] = 1.0;
      continue;
    }
    const int c[3] = {i % nx, (i / nx) % ny, i / (nx * ny)};
    double dg = 0.0;
    for (int a = 0; a < dim; ++a) {
      for (int side = 0; side < 2; ++side) {
        const int cc = c[a] + (side ? 1 : -1);
        if (cc < 0 || cc >= N[a]) {
          if ((bcD >> (2 * a + side)) & 1) dg += w[a];
          continue;
        }
        const int j = i + (side ? stride[a] : -stride[a]);
        const bool nf = cell ? cell[j] != 0 : true;
        if (!nf) continue;
        dg += w[a];
        A[(size_t)i * n + j] = -w[a];
      }
    }
    A[(size_t)i * n + i] = dg;
  }
}

__global__ void k_gauss_jordan(int n, double* __restrict__ A) {
  extern __shared__ double sh[];
  double* rowk = sh;
  double* colk = sh + n;
  for (int k = 0; k < n; ++k) {
    const double piv = 1.0 / A[(size_t)k * n + k];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      rowk[j] = (j == k) ? piv : A[(size_t)k * n + j] * piv;
      colk[j] = A[(size_t)j * n + k];
    }
    __syncthreads();
    for (size_t t = threadIdx.x; t < (size_t)n * n; t += blockDim.x) {
      const int i = (int)(t / n), j = (int)(t % n);
      if (i == k) {
        A[t] = rowk[j];
      } else {
        const double base = (j == k) ? 0.0 : A[t];
        A[t] = base - colk[i] * rowk[j];
      }
    }
    __syncthreads();
  }
}

// The float32 copy the coarse kernels read (column-major; the inverse of the
// symmetric operator is symmetric, so a row is read as a column).
__global__ void k_store_inverse(int n, const double* __restrict__ A, float* __restrict__ At) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)n * n; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    At[(size_t)j * n + i] = (float)A[t];
  }
}

cudaError_t launch_coarse_inverse(int dim, const int64_t nn[3], const double w[3], int bcD, const uint8_t* cell,
                                  double* mat, cudaStream_t s) {
  const int nx = (int)nn[0], ny = (int)nn[1], nz = dim == 3 ? (int)nn[2] : 1;
  const int n = nx * ny * nz;
  double* work = mat + (size_t)n * n;  // caller provides 2 n^2 doubles
  k_dense_matrix<<<1, 256, 0, s>>>(dim, nx, ny, nz, w[0], w[1], w[2], bcD, cell, work);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gauss_jordan<<<1, 1024, 2 * n * sizeof(double), s>>>(n, work);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_store_inverse<<<grid_1d((size_t)n * n, 1024), 256, 0, s>>>(n, work, reinterpret_cast<float*>(mat));
  return cudaGetLastError();
}

}  // namespace npmg
