// Coarse levels of the cycle in one thread block, and the set-up kernels.
#include <math.h>

#include "launch.h"
#include "mg_kernels.cuh"

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
// legs) runs inside one block of 1024 threads with every level, and its
// cell bytes, resident in shared memory.  The coarsest level is solved
// exactly: its operator is inverted once at create (float64 Gauss-Jordan)
// and applied here as a float64 matrix-vector product, one warp per row.
struct CLevel {
  LevelDev L;
  const uint8_t* m;  // cell bytes in shared memory (nullptr: unmasked)
  int n;
};

__device__ __forceinline__ float cl_diag(const CLevel& c, int dim, int x, int y, int z, uint8_t m) {
  if (c.m) return dim == 3 ? diag_at<3, true>(c.L, x, y, z, m) : diag_at<2, true>(c.L, x, y, z, m);
  return dim == 3 ? diag_at<3, false>(c.L, x, y, z, m) : diag_at<2, false>(c.L, x, y, z, m);
}

__device__ __forceinline__ float cl_ax(const CLevel& c, int dim, const float* x, int i, int cx, int cy, int cz,
                                      float d) {
  const LevelDev& L = c.L;
  const int sxy = L.nx * L.ny;
  float nb = 0.f;
  if (cx > 0) nb += L.wx * x[i - 1];
  if (cx < L.nx - 1) nb += L.wx * x[i + 1];
  if (cy > 0) nb += L.wy * x[i - L.nx];
  if (cy < L.ny - 1) nb += L.wy * x[i + L.nx];
  if (dim == 3) {
    if (cz > 0) nb += L.wz * x[i - sxy];
    if (cz < L.nz - 1) nb += L.wz * x[i + sxy];
  }
  return d * x[i] - nb;
}

__device__ void cl_sweep(const CLevel& c, int dim, const float* xin, float* xout, const float* b, float omega,
                         bool from_zero) {
  const LevelDev& L = c.L;
  for (int i = threadIdx.x; i < c.n; i += blockDim.x) {
    const int x = i % L.nx, t = i / L.nx, y = t % L.ny, z = t / L.ny;
    const uint8_t m = c.m ? c.m[i] : kFluidBit;
    float v = 0.f;
    if (m) {
      const float d = cl_diag(c, dim, x, y, z, m);
      v = from_zero ? omega * b[i] / d : xin[i] + omega * (b[i] - cl_ax(c, dim, xin, i, x, y, z, d)) / d;
    }
    xout[i] = v;
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(1024) k_coarse(CoarseArgs a, const T* __restrict__ bin, T* __restrict__ xout,
                                                 SolveState* __restrict__ st) {
  if (st && st->inner_done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* S = reinterpret_cast<float*>(smem_raw);
  const int dim = a.dim;
  CLevel lv[kMaxLevels];
  for (int l = 0; l < a.nlev; ++l) {
    lv[l].L = a.lv[l];
    lv[l].n = a.lv[l].nx * a.lv[l].ny * a.lv[l].nz;
    lv[l].m = a.lv[l].cell ? smem_raw + a.moff[l] : nullptr;
  }
  auto X = [&](int l, int which) { return S + a.off[l] + which * lv[l].n; };
  auto B = [&](int l) { return S + a.off[l] + 2 * lv[l].n; };
  // stage the right-hand side of the first level and all cell bytes
  for (int i = threadIdx.x; i < lv[0].n; i += blockDim.x) B(0)[i] = ld(bin, i);
  for (int l = 0; l < a.nlev; ++l) {
    if (!a.lv[l].cell) continue;
    uint8_t* dst = smem_raw + a.moff[l];
    for (int i = threadIdx.x; i < lv[l].n; i += blockDim.x) dst[i] = a.lv[l].cell[i];
  }
  __syncthreads();
  int cur[kMaxLevels];
  // down legs
  for (int l = 0; l < a.nlev - 1; ++l) {
    const CLevel& c = lv[l];
    int k = 0;
    if (a.pre == 0) {
      for (int i = threadIdx.x; i < c.n; i += blockDim.x) X(l, 0)[i] = 0.f;
      __syncthreads();
    } else {
      cl_sweep(c, dim, nullptr, X(l, 0), B(l), a.omega, true);
      for (int j = 2; j <= a.pre; ++j) {
        cl_sweep(c, dim, X(l, k), X(l, 1 - k), B(l), a.omega, false);
        k = 1 - k;
      }
    }
    cur[l] = k;
    const LevelDev& L = c.L;
    const LevelDev& C = lv[l + 1].L;
    const float* xl = X(l, k);
    const float* bl = B(l);
    float* bc = B(l + 1);
    const float inv_children = dim == 3 ? 0.125f : 0.25f;
    for (int j = threadIdx.x; j < lv[l + 1].n; j += blockDim.x) {
      const int Xc = j % C.nx, t = j / C.nx, Yc = t % C.ny, Zc = t / C.ny;
      float sum = 0.f;
      for (int az = 0; az < (dim == 3 ? 2 : 1); ++az)
        for (int ay = 0; ay < 2; ++ay)
          for (int ax = 0; ax < 2; ++ax) {
            const int cx = 2 * Xc + ax, cy = 2 * Yc + ay, cz = 2 * Zc + az;
            const int i = (cz * L.ny + cy) * L.nx + cx;
            const uint8_t m = c.m ? c.m[i] : kFluidBit;
            if (m) sum += bl[i] - cl_ax(c, dim, xl, i, cx, cy, cz, cl_diag(c, dim, cx, cy, cz, m));
          }
      bc[j] = sum * inv_children;
    }
    __syncthreads();
  }
  // coarsest: x = A^-1 b in float64, one warp per row
  {
    const int l = a.nlev - 1;
    const int n = a.ncoarse;
    float* xc = X(l, 0);
    const float* bc = B(l);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < n; i += nw) {
      double acc = 0.0;
      // the inverse of the symmetric operator is symmetric: read row i
      for (int j = lane; j < n; j += 32) acc += a.inv[(size_t)i * n + j] * (double)bc[j];
      acc = warp_sum(acc);
      if (lane == 0) xc[i] = (float)acc;
    }
    cur[l] = 0;
    __syncthreads();
  }
  // up legs
  for (int l = a.nlev - 2; l >= 0; --l) {
    const CLevel& c = lv[l];
    const LevelDev& L = c.L;
    const LevelDev& C = lv[l + 1].L;
    const float* e = X(l + 1, cur[l + 1]);
    int k = cur[l];
    float* xs = X(l, k);
    for (int i = threadIdx.x; i < c.n; i += blockDim.x) {
      const int x = i % L.nx, t = i / L.nx, y = t % L.ny, z = t / L.ny;
      const uint8_t m = c.m ? c.m[i] : kFluidBit;
      xs[i] = m ? xs[i] + a.s * e[((z >> 1) * C.ny + (y >> 1)) * C.nx + (x >> 1)] : 0.f;
    }
    __syncthreads();
    for (int j = 1; j <= a.post; ++j) {
      cl_sweep(c, dim, X(l, k), X(l, 1 - k), B(l), a.omega, false);
      k = 1 - k;
    }
    cur[l] = k;
  }
  // write the first level handled here
  const float* x0 = X(0, cur[0]);
  const float* b0 = B(0);
  float acc = 0.f;
  for (int i = threadIdx.x; i < lv[0].n; i += blockDim.x) {
    const T zt = cvt<T>(x0[i]);
    xout[i] = zt;
    if (a.finest) acc = fmaf(b0[i], ld(&zt, 0), acc);
  }
  if (a.finest) {
    __shared__ double sh[32];
    const double tot = block_sum((double)acc, sh);
    if (threadIdx.x == 0) {
      st->rz = tot;
      st->beta = (st->first || !st->krylov) ? 0.0 : tot / st->rz_old;
      st->rz_old = tot;
    }
  }
}

template <typename T>
cudaError_t launch_coarse(const CoarseArgs& a, size_t smem_bytes, const void* b, void* x, SolveState* st,
                          cudaStream_t s) {
  k_coarse<T><<<1, 1024, smem_bytes, s>>>(a, (const T*)b, (T*)x, st);
  return cudaGetLastError();
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

// Transpose to column-major for coalesced reads in k_coarse.
__global__ void k_transpose(int n, const double* __restrict__ A, double* __restrict__ At) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)n * n; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    At[(size_t)j * n + i] = A[t];
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
  k_transpose<<<grid_1d((size_t)n * n, 1024), 256, 0, s>>>(n, work, mat);
  return cudaGetLastError();
}

}  // namespace npmg
