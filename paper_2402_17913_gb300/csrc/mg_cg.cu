// Conjugate-gradient vector kernels and the refinement loop's residual.
//
// Row mapping: a block of 256 threads covers 8 rows x 128 cells; each thread
// owns 4 consecutive cells of one row (one 16-byte load per float32 array),
// and blocks stride over z.  Partial sums are accumulated in float32 per
// thread and in float64 across the block and the grid (fixed order, so
// results are reproducible run to run).
#include <math.h>
#include <stdlib.h>
#include <type_traits>

#include "launch.h"
#include "mg_kernels.cuh"
#include "refine.cuh"

namespace npmg {

// ---------------------------------------------------------------------------
// 4-cell row access (vector loads when the row length is a multiple of 4,
// otherwise guarded scalar loads; cells past the row end read as 0).
template <typename T>
__device__ __forceinline__ void ld4(const T* __restrict__ p, size_t i, int x0, int nx, float v[4]) {
  if ((nx & 3) == 0) {
    if constexpr (std::is_same<T, float>::value) {
      const float4 q = *reinterpret_cast<const float4*>(p + i);
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else if constexpr (std::is_same<T, __half>::value) {
      const uint2 q = *reinterpret_cast<const uint2*>(p + i);
      const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
      const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
      v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
      const uint2 q = *reinterpret_cast<const uint2*>(p + i);
      const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.x));
      const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.y));
      v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (x0 + k < nx) ? ld(p, i + k) : 0.f;
  }
}

template <typename T>
__device__ __forceinline__ void st4(T* __restrict__ p, size_t i, int x0, int nx, const float v[4]) {
  if ((nx & 3) == 0) {
    if constexpr (std::is_same<T, float>::value) {
      *reinterpret_cast<float4*>(p + i) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (std::is_same<T, __half>::value) {
      __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
      uint2 q;
      q.x = *reinterpret_cast<unsigned*>(&a);
      q.y = *reinterpret_cast<unsigned*>(&b);
      *reinterpret_cast<uint2*>(p + i) = q;
    } else {
      __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
      uint2 q;
      q.x = *reinterpret_cast<unsigned*>(&a);
      q.y = *reinterpret_cast<unsigned*>(&b);
      *reinterpret_cast<uint2*>(p + i) = q;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (x0 + k < nx) p[i + k] = cvt<T>(v[k]);
  }
}

template <typename T>
__device__ __forceinline__ float rnd(float v) {
  const T t = cvt<T>(v);
  return ld(&t, 0);
}

__device__ __forceinline__ void ld4_cell(const uint8_t* __restrict__ c, size_t i, int x0, int nx, uint8_t m[4]) {
  if ((nx & 3) == 0) {
    const uchar4 q = *reinterpret_cast<const uchar4*>(c + i);
    m[0] = q.x; m[1] = q.y; m[2] = q.z; m[3] = q.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) m[k] = (x0 + k < nx) ? c[i + k] : 0;
  }
}

template <bool MASKED>
__device__ __forceinline__ void cells4(const LevelDev& L, size_t i, int x0, uint8_t m[4]) {
  if (MASKED) {
    ld4_cell(L.cell, i, x0, L.nx, m);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) m[k] = (x0 + k < L.nx) ? kFluidBit : 0;
  }
}

// Row groups of 8 rows x 128 cells, walked grid-stride by a persistent grid
// (a few blocks per SM), so that each block pays its reduction once.
struct RowIter {
  int g, G, gxn, gyn, x0, y, z;
  bool active;
  __device__ __forceinline__ explicit RowIter(const LevelDev& L) {
    gxn = (L.nx + 127) / 128;
    gyn = (L.ny + 7) / 8;
    G = gxn * gyn * L.nz;
    g = blockIdx.x;
    set(L);
  }
  __device__ __forceinline__ void set(const LevelDev& L) {
    if (g >= G) return;
    const int gx = g % gxn, t = g / gxn, gy = t % gyn;
    z = t / gyn;
    x0 = gx * 128 + (threadIdx.x & 31) * 4;
    y = gy * 8 + (threadIdx.x >> 5);
    active = x0 < L.nx && y < L.ny;
  }
  __device__ __forceinline__ bool more() const { return g < G; }
  __device__ __forceinline__ void next(const LevelDev& L) {
    g += gridDim.x;
    set(L);
  }
};

static int sm_count() {
  static int n[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 148;
  if (!n[dev]) cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev);
  return n[dev] > 0 ? n[dev] : 148;
}

static int row_blocks_per_sm() {
  static int v = 0;
  if (!v) {
    const char* e = getenv("NPMG_ROW_BLOCKS_PER_SM");
    v = (e && atoi(e) > 0) ? atoi(e) : 4;
  }
  return v;
}

static dim3 row_grid(const LevelDev& L) {
  const long groups = (long)((L.nx + 127) / 128) * ((L.ny + 7) / 8) * L.nz;
  const long cap = (long)sm_count() * row_blocks_per_sm();
  return dim3((unsigned)(groups < cap ? groups : cap), 1, 1);
}

// ---------------------------------------------------------------------------
// CG: p = z + beta p ; Ap = A' p ; (p, Ap) -> alpha = (r, z) / (p, Ap).
// p is double-buffered (pold -> pnew) because Ap needs p at neighbours.
// Neighbour addresses of a 4-cell group, clamped into the array so that
// every load can be issued up front; the flags zero the missing neighbours.
struct Nbr {
  size_t i, il, ir, iu, id, ib, iF;
  bool hl, hr, hu, hd, hb, hf;
};

template <int DIM>
__device__ __forceinline__ Nbr neighbours(const LevelDev& L, int x0, int y, int zz) {
  Nbr n;
  const size_t sxy = (size_t)L.nx * L.ny;
  n.i = (size_t)zz * sxy + (size_t)y * L.nx + x0;
  n.hl = x0 > 0;
  n.hr = x0 + 4 < L.nx;
  n.hu = y > 0;
  n.hd = y < L.ny - 1;
  n.hb = DIM == 3 && zz > 0;
  n.hf = DIM == 3 && zz < L.nz - 1;
  n.il = n.hl ? n.i - 1 : n.i;
  n.ir = n.hr ? n.i + 4 : n.i;
  n.iu = n.hu ? n.i - L.nx : n.i;
  n.id = n.hd ? n.i + L.nx : n.i;
  n.ib = n.hb ? n.i - sxy : n.i;
  n.iF = n.hf ? n.i + sxy : n.i;
  return n;
}

template <int DIM, typename T, bool MASKED>
__global__ void __launch_bounds__(256) k_p_update(LevelDev L, const T* __restrict__ z, const T* __restrict__ pold,
                                                  T* __restrict__ pnew, T* __restrict__ Ap,
                                                  SolveState* __restrict__ st, double* __restrict__ partials) {
  chain_enter();
  if (st->inner_done) return;
  const bool first = st->first || !st->krylov;
  const float beta = first ? 0.f : (float)st->beta;

  float acc = 0.f;
  for (RowIter it(L); it.more(); it.next(L)) {
    if (!it.active) continue;
    const int x0 = it.x0, y = it.y, zz = it.z;
    {
      const Nbr n = neighbours<DIM>(L, x0, y, zz);
      // all loads first
      float zc[4], zu[4], zd[4], zb[4], zf[4], qc[4], qu[4], qd[4], qb[4], qf[4];
      ld4(z, n.i, x0, L.nx, zc);
      ld4(z, n.iu, x0, L.nx, zu);
      ld4(z, n.id, x0, L.nx, zd);
      float zl = ld(z, n.il), zr = ld(z, n.ir), ql = 0.f, qr = 0.f;
      if (DIM == 3) {
        ld4(z, n.ib, x0, L.nx, zb);
        ld4(z, n.iF, x0, L.nx, zf);
      }
      if (!first) {
        ld4(pold, n.i, x0, L.nx, qc);
        ld4(pold, n.iu, x0, L.nx, qu);
        ld4(pold, n.id, x0, L.nx, qd);
        ql = ld(pold, n.il);
        qr = ld(pold, n.ir);
        if (DIM == 3) {
          ld4(pold, n.ib, x0, L.nx, qb);
          ld4(pold, n.iF, x0, L.nx, qf);
        }
      }
      uint8_t m[4];
      cells4<MASKED>(L, n.i, x0, m);
      // p = z + beta p_old at the group and its neighbours
      float pc[4], nb[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) pc[k] = first ? zc[k] : fmaf(beta, qc[k], zc[k]);
      const float pl = n.hl ? (first ? zl : fmaf(beta, ql, zl)) : 0.f;
      const float pr = n.hr ? (first ? zr : fmaf(beta, qr, zr)) : 0.f;
      nb[0] = L.wx * (pl + pc[1]);
      nb[1] = L.wx * (pc[0] + pc[2]);
      nb[2] = L.wx * (pc[1] + pc[3]);
      nb[3] = L.wx * (pc[2] + pr);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float pu = n.hu ? (first ? zu[k] : fmaf(beta, qu[k], zu[k])) : 0.f;
        const float pd = n.hd ? (first ? zd[k] : fmaf(beta, qd[k], zd[k])) : 0.f;
        nb[k] = fmaf(L.wy, pu + pd, nb[k]);
        if (DIM == 3) {
          const float pb = n.hb ? (first ? zb[k] : fmaf(beta, qb[k], zb[k])) : 0.f;
          const float pf = n.hf ? (first ? zf[k] : fmaf(beta, qf[k], zf[k])) : 0.f;
          nb[k] = fmaf(L.wz, pb + pf, nb[k]);
        }
      }
      float ap[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (m[k]) {
          ap[k] = diag_at<DIM, MASKED>(L, x0 + k, y, zz, m[k]) * pc[k] - nb[k];
        } else {
          pc[k] = 0.f;
          ap[k] = 0.f;
        }
        acc = fmaf(rnd<T>(pc[k]), rnd<T>(ap[k]), acc);
      }
      st4(pnew, n.i, x0, L.nx, pc);
      st4(Ap, n.i, x0, L.nx, ap);
    }
  }
  double tot;
  if (grid_sum_last((double)acc, partials, &st->counter[kCntPAP], &tot)) {
    if (threadIdx.x == 0) {
      st->pAp = tot;
      st->alpha = st->krylov ? st->rz / tot : 1.0;
    }
  }
}

// CG: d += alpha p ; r -= alpha Ap ; ||r||^2 ; convergence test.
template <typename T>
__global__ void __launch_bounds__(256) k_xr_update(LevelDev L, const T* __restrict__ p, const T* __restrict__ Ap,
                                                   T* __restrict__ d, T* __restrict__ r, SolveState* __restrict__ st,
                                                   double* __restrict__ partials) {
  chain_enter();
  if (st->inner_done) return;
  const float alpha = (float)st->alpha;
  const bool first = st->first;

  float acc = 0.f;
  const size_t sxy = (size_t)L.nx * L.ny;
  for (RowIter it(L); it.more(); it.next(L)) {
    if (!it.active) continue;
    const int x0 = it.x0, y = it.y, zz = it.z;
    {
      const size_t i = (size_t)zz * sxy + (size_t)y * L.nx + x0;
      float pv[4], av[4], dv[4], rv[4];
      ld4(p, i, x0, L.nx, pv);
      ld4(Ap, i, x0, L.nx, av);
      ld4(r, i, x0, L.nx, rv);
      if (first) {
#pragma unroll
        for (int k = 0; k < 4; ++k) dv[k] = alpha * pv[k];
      } else {
        ld4(d, i, x0, L.nx, dv);
#pragma unroll
        for (int k = 0; k < 4; ++k) dv[k] = fmaf(alpha, pv[k], dv[k]);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        rv[k] = fmaf(-alpha, av[k], rv[k]);
        const float rr = rnd<T>(rv[k]);
        acc = fmaf(rr, rr, acc);
      }
      st4(d, i, x0, L.nx, dv);
      st4(r, i, x0, L.nx, rv);
    }
  }
  double tot;
  if (grid_sum_last((double)acc, partials, &st->counter[kCntRR], &tot)) {
    if (threadIdx.x == 0) inner_decide(st, tot);
  }
}

// The same update for float32 3D vectors, marching along z: a block owns
// 8 rows x 128 cells (a warp per row, 4 cells per lane) and a run of planes;
// p = z + beta p_old of the planes below, at and above the current one stay
// in registers, x-neighbours come by shuffles (lanes 0 and 31 load the cell
// beyond the strip) and y-neighbours from the rows of the adjacent warps,
// which those warps have just loaded (L1).  z and p_old are read from DRAM
// about once instead of once per neighbour.
__device__ __forceinline__ void p_row(const float* __restrict__ z, const float* __restrict__ pold, size_t i, bool in,
                                      bool first, float beta, float (&v)[4]) {
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f), q = a;
  if (in) {
    a = *reinterpret_cast<const float4*>(z + i);
    if (!first) q = *reinterpret_cast<const float4*>(pold + i);
  }
  v[0] = fmaf(beta, q.x, a.x);
  v[1] = fmaf(beta, q.y, a.y);
  v[2] = fmaf(beta, q.z, a.z);
  v[3] = fmaf(beta, q.w, a.w);
}

template <bool MASKED>
__global__ void __launch_bounds__(256) k_p_update_z(LevelDev L, const float* __restrict__ z,
                                                    const float* __restrict__ pold, float* __restrict__ pnew,
                                                    float* __restrict__ Ap, int zr, SolveState* __restrict__ st,
                                                    double* __restrict__ partials) {
  chain_enter();
  if (st->inner_done) return;
  const bool first = st->first || !st->krylov;
  const float beta = first ? 0.f : (float)st->beta;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gx = blockIdx.x * 128 + 4 * lane, y = blockIdx.y * 8 + w;
  const int zs = blockIdx.z * zr, ze = min(zs + zr, L.nz);
  const bool ox = gx < L.nx, yin = y < L.ny;
  const bool own = ox && yin, hasu = own && y > 0, hasd = own && y + 1 < L.ny;
  const size_t sxy = (size_t)L.nx * L.ny;
  // the cells beyond the strip: lane 0 the left one, lane 31 the right one
  const int hx = lane == 0 ? gx - 1 : gx + 4;
  const bool hin = (lane == 0 || lane == 31) && yin && hx >= 0 && hx < L.nx;
  float acc = 0.f;
  // planes q - 1, q, q + 1 of p, and the raw z / p_old of plane q + 2
  // loaded one plane ahead (its DRAM latency overlaps plane q's work)
  float pm[4], pc[4], pp[4];
  p_row(z, pold, (size_t)(zs - 1) * sxy + (size_t)y * L.nx + gx, own && zs > 0, first, beta, pm);
  p_row(z, pold, (size_t)zs * sxy + (size_t)y * L.nx + gx, own, first, beta, pc);
  p_row(z, pold, (size_t)(zs + 1) * sxy + (size_t)y * L.nx + gx, own && zs + 1 < L.nz, first, beta, pp);
  for (int q = zs; q < ze; ++q) {
    const size_t i = (size_t)q * sxy + (size_t)y * L.nx + gx;
    float4 za = make_float4(0.f, 0.f, 0.f, 0.f), qa = za;
    if (own && q + 2 < L.nz && q + 1 < ze) {
      za = *reinterpret_cast<const float4*>(z + i + 2 * sxy);
      if (!first) qa = *reinterpret_cast<const float4*>(pold + i + 2 * sxy);
    }
    float pu[4], pd[4];
    p_row(z, pold, i - L.nx, hasu, first, beta, pu);
    p_row(z, pold, i + L.nx, hasd, first, beta, pd);
    float ph = 0.f;
    if (hin) {
      const size_t ih = (size_t)q * sxy + (size_t)y * L.nx + hx;
      ph = first ? z[ih] : fmaf(beta, pold[ih], z[ih]);
    }
    uint8_t m[4] = {0, 0, 0, 0};
    if (own) cells4<MASKED>(L, i, gx, m);
    const float up = __shfl_up_sync(0xffffffffu, pc[3], 1);
    const float dn = __shfl_down_sync(0xffffffffu, pc[0], 1);
    const float left = lane == 0 ? ph : up, right = lane == 31 ? ph : dn;
    float pv[4], av[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float l = k == 0 ? left : pc[k - 1], r = k == 3 ? right : pc[k + 1];
      const float nb = fmaf(L.wx, l + r, fmaf(L.wy, pu[k] + pd[k], L.wz * (pm[k] + pp[k])));
      if (own && m[k]) {
        pv[k] = pc[k];
        av[k] = diag_at<3, MASKED>(L, gx + k, y, q, m[k]) * pc[k] - nb;
      } else {
        pv[k] = 0.f;
        av[k] = 0.f;
      }
      acc = fmaf(pv[k], av[k], acc);
    }
    if (own) {
      *reinterpret_cast<float4*>(pnew + i) = make_float4(pv[0], pv[1], pv[2], pv[3]);
      *reinterpret_cast<float4*>(Ap + i) = make_float4(av[0], av[1], av[2], av[3]);
    }
    const float pn[4] = {fmaf(beta, qa.x, za.x), fmaf(beta, qa.y, za.y), fmaf(beta, qa.z, za.z), fmaf(beta, qa.w, za.w)};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      pm[k] = pc[k];
      pc[k] = pp[k];
      pp[k] = pn[k];
    }
  }
  double tot;
  if (grid_sum_last((double)acc, partials, &st->counter[kCntPAP], &tot)) {
    if (threadIdx.x == 0) {
      st->pAp = tot;
      st->alpha = st->krylov ? st->rz / tot : 1.0;
    }
  }
}

// z-run of the marching update: about four blocks per SM over the level.
static int pz_run(const LevelDev& L) {
  const long cols = (long)((L.nx + 127) / 128) * ((L.ny + 7) / 8);
  const long target = (long)sm_count() * 4;
  long runs = (target + cols - 1) / cols;
  if (runs < 1) runs = 1;
  if (runs > L.nz) runs = L.nz;
  return (int)((L.nz + runs - 1) / runs);
}

template <int DIM, typename T, bool MASKED>
cudaError_t launch_p_update(const LevelDev& L, const void* z, const void* pold, void* pnew, void* Ap,
                            SolveState* st, double* partials, cudaStream_t s) {
  if constexpr (DIM == 3 && std::is_same<T, float>::value) {
    const bool aligned = (((uintptr_t)z | (uintptr_t)pold | (uintptr_t)pnew | (uintptr_t)Ap) & 15) == 0;
    if (aligned && L.nx % 4 == 0 && getenv("NPMG_NO_PZ") == nullptr) {
      const int zr = pz_run(L);
      const dim3 g((L.nx + 127) / 128, (L.ny + 7) / 8, (L.nz + zr - 1) / zr);
      return launch_chain(k_p_update_z<MASKED>, g, 256, 0, s, L, (const float*)z, (const float*)pold, (float*)pnew,
                          (float*)Ap, zr, st, partials);
    }
  }
  return launch_chain(k_p_update<DIM, T, MASKED>, row_grid(L), 256, 0, s, L, (const T*)z, (const T*)pold, (T*)pnew,
                      (T*)Ap, st, partials);
}
template <typename T>
cudaError_t launch_xr_update(const LevelDev& L, const void* p, const void* Ap, void* d, void* r, SolveState* st,
                             double* partials, cudaStream_t s) {
  return launch_chain(k_xr_update<T>, row_grid(L), 256, 0, s, L, (const T*)p, (const T*)Ap, (T*)d, (T*)r, st, partials);
}

// ---------------------------------------------------------------------------
// Refinement residual in float-float.  x is kept as (hi, lo) pairs.  With
// UPDATE it first applies x <- x + sigma d' (sigma a power of two, so
// sigma d' is exact).  Then, in the scaled units of the inner solve
// (A' = c A_h), r = c b - A' x is formed to ~48 bits, ||r|| reduced, and
// r' = r / sigma_new rounded to the inner storage type (sigma_new a power of
// two near rms(r)).  The last block decides: converged, diverged,
// stalled, or the tolerance of the next inner solve.
struct OuterArgs {
  ff w[3];        // c / h_a^2 per axis as float-float
  ff c;           // h_0x^2 as float-float
  double c2;      // c^2 (to turn ||r||^2 back into unscaled units)
};

// With `dyn` the two float-float buffers are xa, xb and the state's `cur`
// says which one holds the iterate (a device-side loop cannot swap the
// pointers); the last block flips it after an update.  Otherwise x is read
// from xa and the update written to xb.
template <int DIM, typename T, bool MASKED, bool UPDATE>
__global__ void __launch_bounds__(256) k_outer(LevelDev L, OuterArgs oa, const float* __restrict__ b,
                                               float2* xa, float2* xb, int dyn,
                                               const T* __restrict__ dprime, T* __restrict__ rprime,
                                               SolveState* __restrict__ st, double* __restrict__ partials) {
  const bool swap = dyn && st->cur;
  const float2* __restrict__ xin = swap ? xb : xa;
  float2* __restrict__ xout = swap ? xa : xb;
  const double sig_old_d = st->sigma;
  double sig_new_d = sig_old_d;
  if (UPDATE) sig_new_d = pow2_floor(sig_old_d * sqrt(fmax(st->rnorm2, 1e-300) / (double)st->n_fluid));
  const float sig_old = (float)sig_old_d;
  const float inv_sig_new = (float)(1.0 / sig_new_d);

  float acc = 0.f;
  auto upd = [&](float2 q, float dv) -> ff {
    if (!UPDATE) return {q.x, q.y};
    const ff s = two_sum(q.x, sig_old * dv);
    return quick_two_sum(s.hi, s.lo + q.y);
  };
  for (RowIter it(L); it.more(); it.next(L)) {
    if (!it.active) continue;
    const int x0 = it.x0, y = it.y, zz = it.z;
    {
      const Nbr n = neighbours<DIM>(L, x0, y, zz);
      const bool vec = (L.nx & 3) == 0;
      // all loads first (x as float2 pairs, d' at the same places)
      float2 qc[4], qu[4], qd[4], qb[4], qf[4];
      float dc[4], du[4], dd[4], db[4], df[4], bv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool ok = vec || x0 + k < L.nx;
        qc[k] = ok ? xin[n.i + k] : make_float2(0.f, 0.f);
        qu[k] = ok ? xin[n.iu + k] : make_float2(0.f, 0.f);
        qd[k] = ok ? xin[n.id + k] : make_float2(0.f, 0.f);
        if (DIM == 3) {
          qb[k] = ok ? xin[n.ib + k] : make_float2(0.f, 0.f);
          qf[k] = ok ? xin[n.iF + k] : make_float2(0.f, 0.f);
        }
      }
      const float2 ql = xin[n.il], qr = xin[n.ir];
      float dl = 0.f, dr = 0.f;
      if (UPDATE) {
        ld4(dprime, n.i, x0, L.nx, dc);
        ld4(dprime, n.iu, x0, L.nx, du);
        ld4(dprime, n.id, x0, L.nx, dd);
        if (DIM == 3) {
          ld4(dprime, n.ib, x0, L.nx, db);
          ld4(dprime, n.iF, x0, L.nx, df);
        }
        dl = ld(dprime, n.il);
        dr = ld(dprime, n.ir);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) dc[k] = du[k] = dd[k] = db[k] = df[k] = 0.f;
      }
      ld4(b, n.i, x0, L.nx, bv);
      uint8_t m[4];
      cells4<MASKED>(L, n.i, x0, m);
      const ff zero = {0.f, 0.f};
      ff xc[6];  // x0-1 .. x0+4
      xc[0] = n.hl ? upd(ql, dl) : zero;
#pragma unroll
      for (int k = 0; k < 4; ++k) xc[k + 1] = upd(qc[k], dc[k]);
      xc[5] = n.hr ? upd(qr, dr) : zero;
      float rv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        rv[k] = 0.f;
        if (!m[k]) {
          if (UPDATE && (vec || x0 + k < L.nx)) xout[n.i + k] = make_float2(0.f, 0.f);
          continue;
        }
        const int cx = x0 + k;
        int kx, ky, kz = 0;
        if (MASKED) {
          kx = m[k] & 3;
          ky = (m[k] >> 2) & 3;
          kz = (m[k] >> 4) & 3;
        } else {
          kx = axis_count(cx, L.nx, L.bcD, 0);
          ky = axis_count(y, L.ny, L.bcD, 2);
          if (DIM == 3) kz = axis_count(zz, L.nz, L.bcD, 4);
        }
        // A' x = sum_a w_a (k_a x_c - x_minus - x_plus)
        ff ax = ff_mul(ff_add(ff_mul(xc[k + 1], ff{(float)kx, 0.f}), ff_neg(ff_add(xc[k], xc[k + 2]))), oa.w[0]);
        {
          ff sy = ff_mul(xc[k + 1], ff{(float)ky, 0.f});
          if (n.hu) sy = ff_add(sy, ff_neg(upd(qu[k], du[k])));
          if (n.hd) sy = ff_add(sy, ff_neg(upd(qd[k], dd[k])));
          ax = ff_add(ax, ff_mul(sy, oa.w[1]));
        }
        if (DIM == 3) {
          ff sz = ff_mul(xc[k + 1], ff{(float)kz, 0.f});
          if (n.hb) sz = ff_add(sz, ff_neg(upd(qb[k], db[k])));
          if (n.hf) sz = ff_add(sz, ff_neg(upd(qf[k], df[k])));
          ax = ff_add(ax, ff_mul(sz, oa.w[2]));
        }
        const ff r = ff_add(ff_mul(ff{bv[k], 0.f}, oa.c), ff_neg(ax));
        const float rs = r.hi + r.lo;
        rv[k] = rs * inv_sig_new;
        acc = fmaf(rs, rs, acc);
        if (UPDATE) xout[n.i + k] = make_float2(xc[k + 1].hi, xc[k + 1].lo);
      }
      st4(rprime, n.i, x0, L.nx, rv);
    }
  }
  double tot;
  if (grid_sum_last((double)acc, partials, &st->counter[kCntOuter], &tot)) {
    if (threadIdx.x == 0) {
      outer_decide(st, tot, oa.c2, sig_new_d, UPDATE);
      if (UPDATE && dyn) st->cur ^= 1;
    }
  }
}

// Refinement step in float64: the iterate x is a float64 array.  With
// UPDATE, k_update64 first writes x + sigma d' (float64) into the other
// buffer; k_outer64 then forms, in the scaled units of the inner solve,
// r = c b - A' x in float64 from the (updated) iterate, reduces ||r|| in
// float64 and writes r' = r / sigma_new rounded to float32.  The last block
// decides as in the float-float form (outer_decide).  The update is its own
// pass so that every cell is updated once (not once per neighbour that
// reads it): GB300's float64 rate is 1/64 of its float32 rate.
__global__ void __launch_bounds__(256) k_update64(size_t n, const uint8_t* __restrict__ cell, double* xa,
                                                  double* xb, int dyn, const float* __restrict__ dprime,
                                                  const SolveState* __restrict__ st) {
  const bool swap = dyn && st->cur;
  const double* __restrict__ xin = swap ? xb : xa;
  double* __restrict__ xout = swap ? xa : xb;
  const double sig = st->sigma;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const bool fl = cell == nullptr || cell[i] != 0;
    xout[i] = fl ? fma(sig, (double)dprime[i], xin[i]) : 0.0;
  }
}

// UNIT: every axis weight is exactly 1 (equal spacings in the scaled units
// c = h_0x^2), so the neighbour sum needs no products.  The diagonal d =
// sum_a w_a k_a comes from a 64-entry float64 table by link counts
// (kx + 4 ky + 16 kz).  A thread whose cells and neighbours all hold 0 (a
// zero guess) has A' x = 0 exactly and forms only r = c b.
template <int DIM, bool MASKED, bool UPDATE, bool UNIT>
__global__ void __launch_bounds__(256) k_outer64(LevelDev L, double w0, double w1, double w2, double c, double c2,
                                                 const float* __restrict__ b, double* xa, double* xb, int dyn,
                                                 float* __restrict__ rprime, SolveState* __restrict__ st,
                                                 double* __restrict__ partials) {
  __shared__ double dtab[64];
  if (threadIdx.x < 64) {
    const int kx = threadIdx.x & 3, ky = (threadIdx.x >> 2) & 3, kz = (threadIdx.x >> 4) & 3;
    dtab[threadIdx.x] = w0 * kx + w1 * ky + w2 * kz;
  }
  __syncthreads();
  // the iterate: the buffer the update wrote (UPDATE), else the current one
  const bool swap = dyn && st->cur;
  const double* __restrict__ x = (swap != UPDATE) ? xb : xa;
  const double sig_old = st->sigma;
  double sig_new = sig_old;
  if (UPDATE) sig_new = pow2_floor(sig_old * sqrt(fmax(st->rnorm2, 1e-300) / (double)st->n_fluid));
  const float inv_sig_new = (float)(1.0 / sig_new);
  double acc = 0.0;
  for (RowIter it(L); it.more(); it.next(L)) {
    if (!it.active) continue;
    const int x0 = it.x0, y = it.y, zz = it.z;
    const Nbr n = neighbours<DIM>(L, x0, y, zz);
    const bool vec = (L.nx & 3) == 0;
    double xc[6], yu[4], yd[4], zb[4], zf[4];  // xc: x0-1 .. x0+4
    xc[0] = n.hl ? x[n.il] : 0.0;
    xc[5] = n.hr ? x[n.ir] : 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool ok = vec || x0 + k < L.nx;
      xc[k + 1] = ok ? x[n.i + k] : 0.0;
      yu[k] = ok && n.hu ? x[n.iu + k] : 0.0;
      yd[k] = ok && n.hd ? x[n.id + k] : 0.0;
      if (DIM == 3) {
        zb[k] = ok && n.hb ? x[n.ib + k] : 0.0;
        zf[k] = ok && n.hf ? x[n.iF + k] : 0.0;
      }
    }
    // any nonzero value among them (integer test of the bits, sign ignored)
    unsigned long long nz = 0ull;
#pragma unroll
    for (int k = 0; k < 6; ++k) nz |= (unsigned long long)__double_as_longlong(xc[k]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      nz |= (unsigned long long)__double_as_longlong(yu[k]) | (unsigned long long)__double_as_longlong(yd[k]);
      if (DIM == 3)
        nz |= (unsigned long long)__double_as_longlong(zb[k]) | (unsigned long long)__double_as_longlong(zf[k]);
    }
    const bool zero = (nz & 0x7fffffffffffffffull) == 0ull;
    float bv[4];
    ld4(b, n.i, x0, L.nx, bv);
    uint8_t m[4];
    cells4<MASKED>(L, n.i, x0, m);
    float rv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      rv[k] = 0.f;
      if (!m[k]) continue;
      double r;
      if (zero) {
        r = c * (double)bv[k];
      } else {
        int q;
        if (MASKED) {
          q = m[k] & 63;
        } else {
          q = axis_count(x0 + k, L.nx, L.bcD, 0) + 4 * axis_count(y, L.ny, L.bcD, 2);
          if (DIM == 3) q += 16 * axis_count(zz, L.nz, L.bcD, 4);
        }
        // A' x = d x_c - sum_a w_a (x_minus + x_plus); a missing link or
        // solid neighbour holds 0
        double sn;
        if (UNIT) {
          sn = (xc[k] + xc[k + 2]) + (yu[k] + yd[k]);
          if (DIM == 3) sn += zb[k] + zf[k];
        } else {
          sn = w0 * (xc[k] + xc[k + 2]);
          sn = fma(w1, yu[k] + yd[k], sn);
          if (DIM == 3) sn = fma(w2, zb[k] + zf[k], sn);
        }
        r = fma(c, (double)bv[k], fma(-dtab[q], xc[k + 1], sn));
      }
      rv[k] = (float)r * inv_sig_new;
      acc = fma(r, r, acc);
    }
    st4(rprime, n.i, x0, L.nx, rv);
  }
  double tot;
  if (grid_sum_last(acc, partials, &st->counter[kCntOuter], &tot)) {
    if (threadIdx.x == 0) {
      outer_decide(st, tot, c2, sig_new, UPDATE);
      if (UPDATE && dyn) st->cur ^= 1;
    }
  }
}

static OuterArgs outer_args(const double w[3], double c) {
  OuterArgs a;
  for (int k = 0; k < 3; ++k) {
    a.w[k].hi = (float)w[k];
    a.w[k].lo = (float)(w[k] - (double)a.w[k].hi);
  }
  a.c.hi = (float)c;
  a.c.lo = (float)(c - (double)a.c.hi);
  a.c2 = c * c;
  return a;
}

template <int DIM, typename T, bool MASKED, bool UPDATE>
cudaError_t launch_outer(const LevelDev& L, const double w[3], double c, const float* b, const void* xin, void* xout,
                         const void* dprime, void* rprime, SolveState* st, double* partials, cudaStream_t s, int dyn,
                         bool f64) {
  if (f64) {
    if (UPDATE) {
      const size_t n = (size_t)L.nx * L.ny * L.nz;
      const size_t want = (n + 255) / 256, cap = (size_t)sm_count() * 8;
      k_update64<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(n, MASKED ? L.cell : nullptr,
                                                                     (double*)xin, (double*)xout, dyn,
                                                                     (const float*)dprime, st);
    }
    if (w[0] == 1.0 && w[1] == 1.0 && (DIM == 2 || w[2] == 1.0))
      k_outer64<DIM, MASKED, UPDATE, true><<<row_grid(L), 256, 0, s>>>(L, w[0], w[1], w[2], c, c * c, b,
                                                                       (double*)xin, (double*)xout, dyn,
                                                                       (float*)rprime, st, partials);
    else
      k_outer64<DIM, MASKED, UPDATE, false><<<row_grid(L), 256, 0, s>>>(L, w[0], w[1], w[2], c, c * c, b,
                                                                        (double*)xin, (double*)xout, dyn,
                                                                        (float*)rprime, st, partials);
    return cudaGetLastError();
  }
  k_outer<DIM, T, MASKED, UPDATE><<<row_grid(L), 256, 0, s>>>(L, outer_args(w, c), b, (float2*)xin, (float2*)xout,
                                                              dyn, (const T*)dprime, (T*)rprime, st, partials);
  return cudaGetLastError();
}

// The conditional values of the device-side solve loop (one thread each):
// the outer loop runs while the refinement is not done, the inner loop of
// CG chunks while the inner solve is not done; `cap` bounds the checks of
// each loop so that it ends whatever the flags say.
__global__ void k_loop_start(cudaGraphConditionalHandle outer, SolveState* st) {
  st->loop_checks = 0;
  st->loop_bodies = 0;
  st->loop_outer = 0;
  cudaGraphSetConditional(outer, st->outer_done ? 0u : 1u);
}

__global__ void k_loop_inner(cudaGraphConditionalHandle inner, SolveState* st, unsigned int cap, int body) {
  const unsigned int n = ++st->loop_checks;
  st->loop_bodies += body;
  cudaGraphSetConditional(inner, (!st->inner_done && !st->outer_done && n <= cap) ? 1u : 0u);
}

__global__ void k_loop_outer(cudaGraphConditionalHandle outer, SolveState* st, unsigned int cap) {
  const unsigned int n = ++st->loop_outer;
  cudaGraphSetConditional(outer, (!st->outer_done && n < cap) ? 1u : 0u);
}

__global__ void k_loop_set_cur(SolveState* st, int cur) { st->cur = cur; }

cudaError_t launch_loop_start(cudaGraphConditionalHandle outer, SolveState* st, cudaStream_t s) {
  k_loop_start<<<1, 1, 0, s>>>(outer, st);
  return cudaGetLastError();
}
cudaError_t launch_loop_inner(cudaGraphConditionalHandle inner, SolveState* st, unsigned int cap, int body,
                              cudaStream_t s) {
  k_loop_inner<<<1, 1, 0, s>>>(inner, st, cap, body);
  return cudaGetLastError();
}
cudaError_t launch_loop_outer(cudaGraphConditionalHandle outer, SolveState* st, unsigned int cap, cudaStream_t s) {
  k_loop_outer<<<1, 1, 0, s>>>(outer, st, cap);
  return cudaGetLastError();
}
cudaError_t launch_loop_set_cur(SolveState* st, int cur, cudaStream_t s) {
  k_loop_set_cur<<<1, 1, 0, s>>>(st, cur);
  return cudaGetLastError();
}

#define NPMG_INST_VEC(DIM, T, M)                                                                                \
  template cudaError_t launch_p_update<DIM, T, M>(const LevelDev&, const void*, const void*, void*, void*,       \
                                                  SolveState*, double*, cudaStream_t);                           \
  template cudaError_t launch_outer<DIM, T, M, false>(const LevelDev&, const double*, double, const float*,     \
                                                      const void*, void*, const void*, void*, SolveState*,       \
                                                      double*, cudaStream_t, int, bool);                         \
  template cudaError_t launch_outer<DIM, T, M, true>(const LevelDev&, const double*, double, const float*,      \
                                                     const void*, void*, const void*, void*, SolveState*,        \
                                                     double*, cudaStream_t, int, bool);

NPMG_INST_VEC(2, float, false)
NPMG_INST_VEC(2, float, true)
NPMG_INST_VEC(3, float, false)
NPMG_INST_VEC(3, float, true)
NPMG_INST_VEC(2, __half, false)
NPMG_INST_VEC(2, __half, true)
NPMG_INST_VEC(3, __half, false)
NPMG_INST_VEC(3, __half, true)
NPMG_INST_VEC(2, __nv_bfloat16, false)
NPMG_INST_VEC(2, __nv_bfloat16, true)
NPMG_INST_VEC(3, __nv_bfloat16, false)
NPMG_INST_VEC(3, __nv_bfloat16, true)

template cudaError_t launch_xr_update<float>(const LevelDev&, const void*, const void*, void*, void*, SolveState*,
                                             double*, cudaStream_t);
template cudaError_t launch_xr_update<__half>(const LevelDev&, const void*, const void*, void*, void*, SolveState*,
                                              double*, cudaStream_t);
template cudaError_t launch_xr_update<__nv_bfloat16>(const LevelDev&, const void*, const void*, void*, void*,
                                                     SolveState*, double*, cudaStream_t);

// ---------------------------------------------------------------------------
// Solve start: x = (guess, 0) on fluid cells; ||b||^2; reset the state.
template <bool F64>
__global__ void __launch_bounds__(256) k_init(LevelDev L, const float* __restrict__ b, const float* __restrict__ xg,
                                              void* __restrict__ xv_, double c, SolveParams prm,
                                              SolveState* __restrict__ st, double* __restrict__ partials) {
  float2* x = (float2*)xv_;
  double* x64 = (double*)xv_;

  float acc = 0.f;
  const size_t sxy = (size_t)L.nx * L.ny;
  for (RowIter it(L); it.more(); it.next(L)) {
    if (!it.active) continue;
    const int x0 = it.x0, y = it.y, zz = it.z;
    {
      const size_t i = (size_t)zz * sxy + (size_t)y * L.nx + x0;
      uint8_t m[4];
      if (L.cell) ld4_cell(L.cell, i, x0, L.nx, m);
      else cells4<false>(L, i, x0, m);
      float bv[4], xv[4];
      ld4(b, i, x0, L.nx, bv);
      if (xg) ld4(xg, i, x0, L.nx, xv);
      else xv[0] = xv[1] = xv[2] = xv[3] = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (x0 + k >= L.nx) continue;
        if (F64) x64[i + k] = m[k] ? (double)xv[k] : 0.0;
        else x[i + k] = make_float2(m[k] ? xv[k] : 0.f, 0.f);
        if (m[k]) acc = fmaf(bv[k], bv[k], acc);
      }
    }
  }
  double tot;
  if (grid_sum_last((double)acc, partials, &st->counter[kCntInit], &tot)) {
    if (threadIdx.x == 0) init_state(st, prm, tot, c);
  }
}

cudaError_t launch_init(const LevelDev& L, const float* b, const float* xguess, void* x, double c, SolveParams prm,
                        SolveState* st, double* partials, cudaStream_t s, bool f64) {
  if (f64) k_init<true><<<row_grid(L), 256, 0, s>>>(L, b, xguess, x, c, prm, st, partials);
  else k_init<false><<<row_grid(L), 256, 0, s>>>(L, b, xguess, x, c, prm, st, partials);
  return cudaGetLastError();
}

// Solve end: the float32 output is the iterate rounded once (float-float:
// hi + lo; float64: the value); a zero right-hand side has the zero
// solution.
template <bool F64>
__global__ void k_finish(size_t n, void* __restrict__ xa_, void* __restrict__ xb_, float* __restrict__ out,
                         const SolveState* __restrict__ st) {
  void* xv_ = (xb_ && st->cur) ? xb_ : xa_;
  float2* x = (float2*)xv_;
  double* x64 = (double*)xv_;
  const bool zero = st->bnorm2 == 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (zero) {
      if (F64) x64[i] = 0.0;
      else x[i] = make_float2(0.f, 0.f);
      out[i] = 0.f;
    } else if (F64) {
      out[i] = (float)x64[i];
    } else {
      const float2 v = x[i];
      out[i] = v.x + v.y;
    }
  }
}

cudaError_t launch_finish(size_t n, void* x, void* xb, float* out, const SolveState* st, int nblocks, cudaStream_t s,
                          bool f64) {
  if (f64) k_finish<true><<<nblocks, 256, 0, s>>>(n, x, xb, out, st);
  else k_finish<false><<<nblocks, 256, 0, s>>>(n, x, xb, out, st);
  return cudaGetLastError();
}

// The float64 value of the iterate: (double)hi + (double)lo, or a copy.
template <bool F64>
__global__ void k_ff_to_f64(size_t n, const void* __restrict__ xv_, double* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (F64) {
      out[i] = ((const double*)xv_)[i];
    } else {
      const float2 v = ((const float2*)xv_)[i];
      out[i] = (double)v.x + (double)v.y;
    }
  }
}

cudaError_t launch_ff_to_f64(size_t n, const void* x, double* out, int nblocks, cudaStream_t s, bool f64) {
  if (f64) k_ff_to_f64<true><<<nblocks, 256, 0, s>>>(n, x, out);
  else k_ff_to_f64<false><<<nblocks, 256, 0, s>>>(n, x, out);
  return cudaGetLastError();
}

}  // namespace npmg
