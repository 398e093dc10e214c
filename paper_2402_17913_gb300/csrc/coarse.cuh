// The block-local coarse cycle (device code shared by the single-grid and
// the batched solvers).
#pragma once
#include "launch.h"
#include "mg_kernels.cuh"
#include "tma.cuh"

namespace npmg {

struct CGeo {
  int nx, ny, nz, W, WH, n, off;  // interior sizes, padded row / plane, cells, float offset
  int lnx, lny;                   // log2 of nx, ny when powers of two, else -1
  __device__ __forceinline__ int pad(int x, int y, int z) const { return ((z + (nz > 1 ? 1 : 0)) * (ny + 2) + y + 1) * W + x + 1; }
  __device__ __forceinline__ void xyz(int i, int& x, int& y, int& z) const {
    if (lnx >= 0 && lny >= 0) {
      x = i & (nx - 1);
      y = (i >> lnx) & (ny - 1);
      z = i >> (lnx + lny);
    } else {
      x = i % nx;
      const int t = i / nx;
      y = t % ny;
      z = t / ny;
    }
  }
};

__device__ __forceinline__ int ilog2_or_neg(int v) { return (v & (v - 1)) ? -1 : __ffs(v) - 1; }

__device__ __forceinline__ CGeo cgeo(const LevelDev& L, int off) {
  CGeo g;
  g.nx = L.nx;
  g.ny = L.ny;
  g.nz = L.nz;
  g.W = L.nx + 2;
  g.WH = (L.nx + 2) * (L.ny + 2);
  g.n = L.nx * L.ny * L.nz;
  g.off = off;
  g.lnx = ilog2_or_neg(L.nx);
  g.lny = ilog2_or_neg(L.ny);
  return g;
}

template <int DIM>
__device__ __forceinline__ float cl_nb(const LevelDev& L, const CGeo& g, const float* x, int p) {
  float nb = L.wx * (x[p - 1] + x[p + 1]) + L.wy * (x[p - g.W] + x[p + g.W]);
  if (DIM == 3) nb += L.wz * (x[p - g.WH] + x[p + g.WH]);
  return nb;
}

template <int DIM>
__device__ __forceinline__ void cl_sweep(const LevelDev& L, const CGeo& g, const float* xin, float* xout,
                                         const float* b, const float* id, float omega) {
  const float om1 = 1.f - omega;
  for (int i = threadIdx.x; i < g.n; i += blockDim.x) {
    int x, y, z;
    g.xyz(i, x, y, z);
    const int p = g.pad(x, y, z);
    xout[p] = fmaf(om1, xin[p], omega * id[p] * (b[p] + cl_nb<DIM>(L, g, xin, p)));
  }
  __syncthreads();
}

// Zero all arrays (the ghost rings stay zero for good) and write 1/diag
// (0 on non-fluid cells) of every level; into shared memory or into the
// image in global memory that later launches copy in.
// `block_local`: one block fills its own shared memory (else the whole grid
// fills a global image).
template <int DIM>
__device__ void coarse_fill_image(const CoarseArgs& a, float* S, int total_floats, bool block_local) {
  const int t0 = block_local ? threadIdx.x : threadIdx.x + blockIdx.x * blockDim.x;
  const int ts = block_local ? blockDim.x : blockDim.x * gridDim.x;
  for (int i = t0; i < total_floats / 4; i += ts) reinterpret_cast<float4*>(S)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (block_local || gridDim.x == 1) __syncthreads();
  else __threadfence();
  for (int l = 0; l < a.nlev; ++l) {
    const LevelDev& L = a.lv[l];
    const CGeo g = cgeo(L, a.off[l]);
    float* id = S + g.off + 3 * g.WH * (g.nz + (g.nz > 1 ? 2 : 0));
    for (int i = t0; i < g.n; i += ts) {
      int x, y, z;
      g.xyz(i, x, y, z);
      const uint8_t m = L.cell ? L.cell[i] : kFluidBit;
      const float d = L.cell ? diag_at<DIM, true>(L, x, y, z, m) : diag_at<DIM, false>(L, x, y, z, m);
      id[g.pad(x, y, z)] = m ? __frcp_rn(d) : 0.f;
    }
  }
}

template <int DIM>
__global__ void k_coarse_image(const __grid_constant__ CoarseArgs a, float* image, int total_floats) {
  coarse_fill_image<DIM>(a, image, total_floats, false);
}

// PREFETCH: load the first level's right-hand side while the image is in
// flight (callers with few registers to spare turn it off).
template <int DIM, typename T, bool PREFETCH = true>
__device__ void coarse_cycle(const CoarseArgs& a, const T* __restrict__ bin, T* __restrict__ xout,
                             SolveState* __restrict__ st, float* S, int total_floats, bool load_image = true) {
  // level l: X0 | X1 | B | ID, each padded
  auto G = [&](int l) { return cgeo(a.lv[l], a.off[l]); };
  auto PS = [&](const CGeo& g) { return g.WH * (g.nz + (g.nz > 1 ? 2 : 0)); };
  auto X = [&](const CGeo& g, int which) { return S + g.off + which * PS(g); };
  auto B = [&](const CGeo& g) { return S + g.off + 2 * PS(g); };
  auto ID = [&](const CGeo& g) { return S + g.off + 3 * PS(g); };
  // the first two float4 of this thread's share of the right-hand side are
  // loaded before the wait for the image, so that the two global latencies
  // overlap
  const CGeo g0 = G(0);
  const bool vec = (g0.nx & 3) == 0 && std::is_same<T, float>::value;
  const int n4 = vec ? g0.n / 4 : 0;
  const int i40 = (int)threadIdx.x, i41 = i40 + (int)blockDim.x;
  float4 pre0 = make_float4(0.f, 0.f, 0.f, 0.f), pre1 = pre0;
  if (PREFETCH && i40 < n4) pre0 = reinterpret_cast<const float4*>(bin)[i40];
  if (PREFETCH && i41 < n4) pre1 = reinterpret_cast<const float4*>(bin)[i41];
  // a block that keeps the region between calls loads the constant part
  // once: the cycle writes only the arrays' cells, never the rings or 1/diag
  if (load_image && a.image) {
    // the constant part of the image (zero rings, inverse diagonals) comes
    // from global memory in bulk asynchronous copies
    __shared__ __align__(8) uint64_t bar;  // initialised on every call (phase 0)
    if (threadIdx.x == 0) {
      mbar_init(&bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    const uint32_t bytes = (uint32_t)total_floats * 4u;
    if (threadIdx.x == 0) {
      mbar_arrive_expect_tx(&bar, bytes);
      for (uint32_t o = 0; o < bytes; o += 32768u)
        bulk_load(S + o / 4, a.image + o / 4, bytes - o < 32768u ? bytes - o : 32768u, &bar);
    }
    if (!mbar_wait_bounded(&bar, 0)) {
      if (st && threadIdx.x == 0) {
        st->status = MG_TIMEOUT;
        st->inner_done = 1;
        st->outer_done = 1;
      }
      return;
    }
  } else if (load_image) {
    coarse_fill_image<DIM>(a, S, total_floats, true);
  }
  // right-hand side of the first level
  {
    const CGeo g = g0;
    float* b0 = B(g);
    if (vec) {
#pragma unroll 2
      for (int i4 = threadIdx.x; i4 < n4; i4 += blockDim.x) {
        const float4 v = PREFETCH && i4 == i40   ? pre0
                         : PREFETCH && i4 == i41 ? pre1
                                                 : reinterpret_cast<const float4*>(bin)[i4];
        int x, y, z;
        g.xyz(4 * i4, x, y, z);
        float* d = b0 + g.pad(x, y, z);
        d[0] = v.x;
        d[1] = v.y;
        d[2] = v.z;
        d[3] = v.w;
      }
    } else {
      for (int i = threadIdx.x; i < g.n; i += blockDim.x) {
        int x, y, z;
        g.xyz(i, x, y, z);
        b0[g.pad(x, y, z)] = ld(bin, i);
      }
    }
  }
  __syncthreads();
  unsigned cur = 0u;  // bit l: level l's current x is buffer 1
  // a.pre < 0: the sawtooth recursion (App. B): on the way down x = b / d
  // (one Jacobi step from zero) and the restricted residual is that of
  // x = 0, i.e. b; the coarsest level gets the same Jacobi step and the
  // post sweeps instead of the exact solve
  const bool saw = a.pre < 0;
  // down legs
  for (int l = 0; l < a.nlev - 1; ++l) {
    const LevelDev& L = a.lv[l];
    const CGeo g = G(l);
    const float* b = B(g);
    const float* id = ID(g);
    int k = 0;
    {
      float* x0 = X(g, 0);
      for (int i = threadIdx.x; i < g.n; i += blockDim.x) {
        int x, y, z;
        g.xyz(i, x, y, z);
        const int p = g.pad(x, y, z);
        x0[p] = saw ? id[p] * b[p] : (a.pre > 0 ? a.omega * id[p] * b[p] : 0.f);
      }
      __syncthreads();
    }
    for (int j = 2; j <= a.pre; ++j) {
      cl_sweep<DIM>(L, g, X(g, k), X(g, 1 - k), b, id, a.omega);
      k = 1 - k;
    }
    if (k) cur |= 1u << l;
    const float* xl = X(g, k);
    const LevelDev& CL = a.lv[l + 1];
    const CGeo c = G(l + 1);
    float* bc = B(c);
    const float inv_children = DIM == 3 ? 0.125f : 0.25f;
    for (int jc = threadIdx.x; jc < c.n; jc += blockDim.x) {
      int X0, Y0, Z0;
      c.xyz(jc, X0, Y0, Z0);
      float sum = 0.f;
#pragma unroll
      for (int az = 0; az < (DIM == 3 ? 2 : 1); ++az)
#pragma unroll
        for (int ay = 0; ay < 2; ++ay)
#pragma unroll
          for (int ax = 0; ax < 2; ++ax) {
            const int p = g.pad(2 * X0 + ax, 2 * Y0 + ay, 2 * Z0 + az);
            const float idv = id[p];
            if (idv != 0.f) sum += saw ? b[p] : b[p] - (__frcp_rn(idv) * xl[p] - cl_nb<DIM>(L, g, xl, p));
          }
      bc[c.pad(X0, Y0, Z0)] = sum * inv_children;
    }
    (void)CL;
    __syncthreads();
  }
  // coarsest: x = A^-1 b (sawtooth: the Jacobi step from zero and the post
  // sweeps)
  if (saw) {
    const int l = a.nlev - 1;
    const LevelDev& L = a.lv[l];
    const CGeo c = G(l);
    const float* bc = B(c);
    const float* id = ID(c);
    float* x0 = X(c, 0);
    for (int i = threadIdx.x; i < c.n; i += blockDim.x) {
      int x, y, z;
      c.xyz(i, x, y, z);
      const int p = c.pad(x, y, z);
      x0[p] = id[p] * bc[p];
    }
    __syncthreads();
    int k = 0;
    for (int j = 1; j <= a.post; ++j) {
      cl_sweep<DIM>(L, c, X(c, k), X(c, 1 - k), bc, id, a.omega);
      k = 1 - k;
    }
    if (k) cur |= 1u << l;
  } else {
    // Q lanes per row (Q a power of two up to 32 with Q n <= the block's
    // threads): lane q of row i takes columns q, q + Q, q + 2Q, ... (the Q
    // lanes of a row read adjacent floats), float32 products, and the Q
    // partial sums add up by shuffles.  The loop is unrolled so that a lane's
    // loads are in flight together.  (A float64 product with one chunk of
    // columns per lane took 18 us of the 37 us cycle of the 3D flow step on
    // its 128-cell coarsest level: float64 runs at 1/64 of the float32 rate
    // here, and the chunked loads did not coalesce.)
    const CGeo c = G(a.nlev - 1);
    const int n = a.ncoarse;
    float* xc = X(c, 0);
    const float* bc = B(c);
    const int nt = (int)(blockDim.x & ~31u);  // whole warps
    int Q = 1;
    while (Q < 32 && 2 * Q * n <= nt) Q *= 2;
    const int pass = nt / Q;
    if ((int)threadIdx.x < nt) {
      const int q = threadIdx.x & (Q - 1), ri = threadIdx.x / Q;
      for (int i0 = 0; i0 < n; i0 += pass) {
        const int i = i0 + ri;
        float acc = 0.f;
        if (i < n) {
          const float* __restrict__ row = a.inv + (size_t)i * n;
#pragma unroll 8
          for (int j = q; j < n; j += Q) {
            int x, y, z;
            c.xyz(j, x, y, z);
            acc = fmaf(__ldg(row + j), bc[c.pad(x, y, z)], acc);
          }
        }
        for (int o = Q >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i < n && q == 0) {
          int x, y, z;
          c.xyz(i, x, y, z);
          xc[c.pad(x, y, z)] = acc;
        }
      }
    }
    __syncthreads();
  }
  // up legs
  for (int l = a.nlev - 2; l >= 0; --l) {
    const LevelDev& L = a.lv[l];
    const CGeo g = G(l);
    const CGeo c = G(l + 1);
    const float* e = X(c, (cur >> (l + 1)) & 1u);
    const float* b = B(g);
    const float* id = ID(g);
    int k = (cur >> l) & 1u;
    float* xs = X(g, k);
    for (int i = threadIdx.x; i < g.n; i += blockDim.x) {
      int x, y, z;
      g.xyz(i, x, y, z);
      const int p = g.pad(x, y, z);
      if (id[p] != 0.f) xs[p] += a.s * e[c.pad(x >> 1, y >> 1, z >> 1)];
    }
    __syncthreads();
    for (int j = 1; j <= a.post; ++j) {
      cl_sweep<DIM>(L, g, X(g, k), X(g, 1 - k), b, id, a.omega);
      k = 1 - k;
    }
    cur = (cur & ~(1u << l)) | ((unsigned)k << l);
  }
  // write the first level handled here
  const CGeo g = G(0);
  const float* x0 = X(g, cur & 1u);
  const float* b0 = B(g);
  float acc = 0.f;
  for (int i = threadIdx.x; i < g.n; i += blockDim.x) {
    int x, y, z;
    g.xyz(i, x, y, z);
    const int p = g.pad(x, y, z);
    const T zt = cvt<T>(x0[p]);
    xout[i] = zt;
    if (a.finest) acc = fmaf(b0[p], ld(&zt, 0), acc);
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

}  // namespace npmg
