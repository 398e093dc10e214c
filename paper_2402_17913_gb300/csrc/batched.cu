// Batched solver: many independent 2D pressure-Poisson instances of uneven
// size solved by ONE persistent launch (captured once in a CUDA graph).
//
// Every instance runs the single-grid algorithm (float-float refinement
// around MG-PCG with the V(pre,post) cycle of Sec. 2.2).  The launch walks the
// phases of that algorithm in lockstep over all instances; within a phase the
// blocks share out work items -- (instance, tile) pairs on one level, or
// whole instances for the per-instance steps -- and a grid-wide barrier
// separates phases.  Phases are aligned by level counted from the finest
// grid, so a small instance simply has no items in some phases.  An
// instance that has converged leaves every later work list.  Each
// instance's levels with <= 1024 cells are one block-local item (the same
// cycle code as the single-grid coarse kernel).  Reductions are per
// instance, in a fixed order over per-tile partial slots.
//
// The grid barrier spins a bounded number of times: if a block never
// arrives, the others give up, raise an error flag and return, and the
// solve reports MG_TIMEOUT instead of hanging.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <sys/stat.h>

#include <cmath>
#include <string>
#include <vector>

#include "coarse.cuh"
#include "launch.h"
#include "mg_kernels.cuh"
#include "refine.cuh"

namespace npmg {

constexpr int kBThreads = 256;
constexpr int kBCoarseCells = 1024;

struct BInst {
  int L, kc, nfluid, nx, ny;
  LevelDev lv[kMaxLevels];
  float* b[kMaxLevels];  // right-hand side of level k (k >= 1)
  float* x[kMaxLevels];  // down-leg x of level k (k < kc)
  float* y[kMaxLevels];  // up-leg output of level k (1 <= k <= kc; y[kc] = coarse item output)
  float *r, *z, *p0, *p1, *Ap, *d;
  float2 *xf0, *xf1;
  ff wff[2];             // finest operator weights c / h^2 (float-float)
  ff cff;                // c = h_x^2
  double c, c2;
  int slot0, ntiles0;    // partial-sum slots of the level-0 tiles
  int cfloats;           // shared floats of the coarse item
  CoarseArgs ca;
};

struct BatchArgs {
  BInst* inst;
  SolveState* st;
  int* cur;              // per instance: which xf buffer holds the iterate
  const float* const* rhs;
  const float* const* xin;   // initial guesses (the outputs, except in the tuner)
  float* const* xout;
  int count;
  const int4* items[kMaxLevels];  // (instance, tile x, tile y, slot) per level
  int nitems[kMaxLevels];
  int ntile_levels;      // max kc over instances
  double* partials;      // one per level-0 tile
  unsigned* bar;         // [0] arrivals, [1] generation, [2] error, [4..5] active counts
  int sweeps;
  float omega, s;
  SolveParams prm;
  long long spin_limit;
  int withhold;          // test hook: block 0 never arrives at the first barrier
};

// ---------------------------------------------------------------------------
// bounded grid barrier
__device__ __forceinline__ bool bwait(const BatchArgs& A, unsigned g) {
  volatile unsigned* gen = A.bar + 1;
  volatile unsigned* err = A.bar + 2;
  for (long long i = 0; i < A.spin_limit; ++i) {
    if (*gen != g) return true;
    if (*err) return false;
    __nanosleep(128);
  }
  return false;
}

__device__ __forceinline__ bool grid_barrier(const BatchArgs& A, unsigned& epoch) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    const unsigned g = *(volatile unsigned*)(A.bar + 1);
    __threadfence();
    bool res;
    if (A.withhold && blockIdx.x == 0 && epoch == 0) {
      res = bwait(A, g);  // withheld arrival: nobody can pass this barrier
    } else {
      const unsigned t = atomicAdd(A.bar + 0, 1u);
      if (t == gridDim.x - 1) {
        atomicExch(A.bar + 0, 0u);
        __threadfence();
        atomicAdd(A.bar + 1, 1u);
        res = true;
      } else {
        res = bwait(A, g);
      }
    }
    if (!res) atomicExch(A.bar + 2, 1u);
    __threadfence();
    ok = res && *(volatile unsigned*)(A.bar + 2) == 0;
  }
  __syncthreads();
  ++epoch;
  return ok;
}

// ---------------------------------------------------------------------------
// tile work (2D, tile TX x TY, halo H = sweeps), explicit tile coordinates.
// The sweep depth is a compile-time parameter (1..3, dispatched once per
// call), so every region width is a constant; the tile stores omega / d per
// cell (0 off the fluid) and a sweep is x <- (1 - omega) x + (omega/d)(b + nb).
template <int TX, int TY, int H>
struct BReg {
  static constexpr int RX = TX + 2 * H, RY = TY + 2 * H, R = RX * RY;
  int ox, oy;
  __device__ __forceinline__ BReg(int tx, int ty) : ox(tx * TX - H), oy(ty * TY - H) {}
};

__device__ __forceinline__ float b_diag(const LevelDev& L, int gx, int gy, uint8_t m) {
  return L.cell ? diag_at<2, true>(L, gx, gy, 0, m) : diag_at<2, false>(L, gx, gy, 0, m);
}

// smem of one tile: b, two iterates, omega / d (floats), cell bytes
template <int TX, int TY, int H>
struct BSmem {
  float *sb, *s0, *s1, *sw;
  uint8_t* sm;
  __device__ __forceinline__ explicit BSmem(float* S) {
    constexpr int R = BReg<TX, TY, H>::R;
    sb = S;
    s0 = sb + R;
    s1 = s0 + R;
    sw = s1 + R;
    sm = reinterpret_cast<uint8_t*>(sw + R);
  }
};

// one sweep over the tile grown by M cells; from_zero: x_in = 0.  The block
// is always kBThreads wide, so every loop below has a compile-time trip
// count and is unrolled: a thread's loads are all issued before the first
// of them is used.
template <int TX, int TY, int H, int M>
__device__ __forceinline__ void b_sweep(const LevelDev& L, const float* __restrict__ xin, float* __restrict__ xout,
                                        const float* __restrict__ sb, const float* __restrict__ sw, float omega,
                                        bool from_zero) {
  using G = BReg<TX, TY, H>;
  constexpr int SX = TX + 2 * M, SY = TY + 2 * M, NI = (SX * SY + kBThreads - 1) / kBThreads;
  const float keep = 1.f - omega;
#pragma unroll
  for (int j = 0; j < NI; ++j) {
    const int i = threadIdx.x + j * kBThreads;
    if (i >= SX * SY) break;
    const int li = (i / SX + H - M) * G::RX + i % SX + H - M;
    const float w = sw[li];
    float v;
    if (from_zero) {
      v = w * sb[li];
    } else {
      const float nb = L.wx * (xin[li - 1] + xin[li + 1]) + L.wy * (xin[li - G::RX] + xin[li + G::RX]);
      v = w > 0.f ? keep * xin[li] + w * (sb[li] + nb) : 0.f;
    }
    xout[li] = v;
  }
  __syncthreads();
}

// global index of region element i of a tile, or -1 off the grid (an
// instance has at most 2^31 cells)
template <int TX, int TY, int H>
__device__ __forceinline__ int b_gidx(const LevelDev& L, const BReg<TX, TY, H>& g, int i) {
  using G = BReg<TX, TY, H>;
  const int gx = g.ox + i % G::RX, gy = g.oy + i / G::RX;
  if (i >= G::R || gx < 0 || gx >= L.nx || gy < 0 || gy >= L.ny) return -1;
  return gy * L.nx + gx;
}

// down leg of one tile: H sweeps from zero, x, restricted residual (the
// scalar path, for a level whose width is not a multiple of 4; kept out of
// line so that its registers do not weigh on the float4 path)
template <int TX, int TY, int H>
__device__ __noinline__ void b_down_h(const LevelDev& L, int tx, int ty, const float* __restrict__ b, float* __restrict__ x,
                         float* __restrict__ bc, float omega, float* S) {
  using G = BReg<TX, TY, H>;
  const G g(tx, ty);
  const BSmem<TX, TY, H> M(S);
  constexpr int NR = (G::R + kBThreads - 1) / kBThreads;
  // all of this thread's region loads in flight at once: b is read whatever
  // the cell byte says and discarded off the fluid
  float bv[NR];
  uint8_t mv[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int gi = b_gidx(L, g, threadIdx.x + j * kBThreads);
    mv[j] = gi < 0 ? 0 : (L.cell ? L.cell[gi] : kFluidBit);
    bv[j] = gi < 0 ? 0.f : b[gi];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int i = threadIdx.x + j * kBThreads;
    if (i >= G::R) break;
    const uint8_t m = mv[j];
    M.sb[i] = m ? bv[j] : 0.f;
    M.sw[i] = m ? __fdividef(omega, b_diag(L, g.ox + i % G::RX, g.oy + i / G::RX, m)) : 0.f;
    M.sm[i] = m;
  }
  __syncthreads();
  b_sweep<TX, TY, H, H>(L, nullptr, M.s0, M.sb, M.sw, omega, true);
  float* cur = M.s0;
  if (H >= 2) {
    b_sweep<TX, TY, H, (H >= 2 ? H - 1 : 1)>(L, M.s0, M.s1, M.sb, M.sw, omega, false);
    cur = M.s1;
  }
  if (H >= 3) {
    b_sweep<TX, TY, H, 1>(L, M.s1, M.s0, M.sb, M.sw, omega, false);
    cur = M.s0;
  }
#pragma unroll
  for (int i = threadIdx.x; i < TX * TY; i += kBThreads) {
    const int lx = i % TX + H, ly = i / TX + H;
    const int gx = g.ox + lx, gy = g.oy + ly;
    if (gx < L.nx && gy < L.ny) x[(size_t)gy * L.nx + gx] = cur[ly * G::RX + lx];
  }
  const int cnx = L.nx / 2, cny = L.ny / 2;
#pragma unroll
  for (int i = threadIdx.x; i < (TX / 2) * (TY / 2); i += kBThreads) {
    const int cx = i % (TX / 2), cy = i / (TX / 2);
    const int gcx = tx * (TX / 2) + cx, gcy = ty * (TY / 2) + cy;
    if (gcx >= cnx || gcy >= cny) continue;
    float sum = 0.f;
#pragma unroll
    for (int ay = 0; ay < 2; ++ay)
#pragma unroll
      for (int ax = 0; ax < 2; ++ax) {
        const int lx = H + 2 * cx + ax, ly = H + 2 * cy + ay;
        const int li = ly * G::RX + lx;
        const uint8_t mm = M.sm[li];
        if (!mm) continue;
        const float d = b_diag(L, g.ox + lx, g.oy + ly, mm);
        const float nb = L.wx * (cur[li - 1] + cur[li + 1]) + L.wy * (cur[li - G::RX] + cur[li + G::RX]);
        sum += M.sb[li] - (d * cur[li] - nb);
      }
    bc[(size_t)gcy * cnx + gcx] = 0.25f * sum;
  }
}

// up leg of one tile: x + s P e, H sweeps, output; returns this thread's
// share of (b, out) when `dot`
template <int TX, int TY, int H>
__device__ __noinline__ float b_up_h(const LevelDev& L, int tx, int ty, const float* __restrict__ b,
                        const float* __restrict__ xin, float* __restrict__ xout, const float* __restrict__ e,
                        float omega, float s, bool dot, float* S) {
  using G = BReg<TX, TY, H>;
  const G g(tx, ty);
  const BSmem<TX, TY, H> M(S);
  const int cnx = L.nx / 2;
  constexpr int NR = (G::R + kBThreads - 1) / kBThreads;
  // all of this thread's region loads in flight at once (values off the
  // fluid are read and discarded)
  float xv[NR], ev[NR], bv[NR];
  uint8_t mv[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int i = threadIdx.x + j * kBThreads;
    const int gi = b_gidx(L, g, i);
    const int gx = g.ox + i % G::RX, gy = g.oy + i / G::RX;
    mv[j] = gi < 0 ? 0 : (L.cell ? L.cell[gi] : kFluidBit);
    xv[j] = gi < 0 ? 0.f : xin[gi];
    ev[j] = gi < 0 ? 0.f : e[(size_t)(gy >> 1) * cnx + (gx >> 1)];
    bv[j] = gi < 0 ? 0.f : b[gi];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int i = threadIdx.x + j * kBThreads;
    if (i >= G::R) break;
    const uint8_t m = mv[j];
    M.s0[i] = m ? xv[j] + s * ev[j] : 0.f;
    M.sb[i] = m ? bv[j] : 0.f;
    M.sw[i] = m ? __fdividef(omega, b_diag(L, g.ox + i % G::RX, g.oy + i / G::RX, m)) : 0.f;
    M.sm[i] = m;
  }
  __syncthreads();
  float* cur = M.s0;
  if (H == 1) {
    b_sweep<TX, TY, H, 0>(L, M.s0, M.s1, M.sb, M.sw, omega, false);
    cur = M.s1;
  } else if (H == 2) {
    b_sweep<TX, TY, H, 1>(L, M.s0, M.s1, M.sb, M.sw, omega, false);
    b_sweep<TX, TY, H, 0>(L, M.s1, M.s0, M.sb, M.sw, omega, false);
  } else {
    b_sweep<TX, TY, H, (H >= 3 ? 2 : 0)>(L, M.s0, M.s1, M.sb, M.sw, omega, false);
    b_sweep<TX, TY, H, 1>(L, M.s1, M.s0, M.sb, M.sw, omega, false);
    b_sweep<TX, TY, H, 0>(L, M.s0, M.s1, M.sb, M.sw, omega, false);
    cur = M.s1;
  }
  float acc = 0.f;
#pragma unroll
  for (int i = threadIdx.x; i < TX * TY; i += kBThreads) {
    const int lx = i % TX + H, ly = i / TX + H;
    const int gx = g.ox + lx, gy = g.oy + ly;
    if (gx < L.nx && gy < L.ny) {
      const int li = ly * G::RX + lx;
      xout[(size_t)gy * L.nx + gx] = cur[li];
      if (dot) acc = fmaf(M.sb[li], cur[li], acc);
    }
  }
  return acc;
}

// ---------------------------------------------------------------------------
// float4 tile path, for a level whose width is a multiple of 4 (every level-0
// grid; coarser levels while their width stays a multiple of 4).  The region
// is the tile plus one group of four cells on each side in x and H rows in y,
// so a global access is a whole float4 (uchar4 for the cell bytes) that is
// either all on the grid or all off it, and a sweep updates four cells per
// thread.  A sweep updates every group of its rows: the outermost groups'
// outer neighbours lie outside the region (a pad float), which spoils one
// more cell per sweep from the region's x edges inward -- at most H - 1 <= 2
// cells after the last sweep, so the tile and the one-cell ring around it
// that the restriction reads stay exact.
template <int TX, int TY, int H>
struct VReg {
  static constexpr int RX = TX + 8, RY = TY + 2 * H, R = RX * RY, W4 = RX / 4, PAD = 4;
  static constexpr int A = R + 2 * PAD;  // floats per padded array
  static constexpr int NG = RY * W4;     // groups in the region
  int ox, oy;
  __device__ __forceinline__ VReg(int tx, int ty) : ox(tx * TX - 4), oy(ty * TY - H) {}
  // global index of group q's first cell, or -1 off the grid
  __device__ __forceinline__ int gidx(const LevelDev& L, int q) const {
    const int gx = ox + 4 * (q % W4), gy = oy + q / W4;
    if (q >= NG || gx < 0 || gx >= L.nx || gy < 0 || gy >= L.ny) return -1;
    return gy * L.nx + gx;
  }
};

// smem of one float4 tile: b, two iterates, omega / d (padded float arrays),
// cell bytes
template <int TX, int TY, int H>
struct VSmem {
  float *sb, *s0, *s1, *sw;
  uint8_t* sm;
  __device__ __forceinline__ explicit VSmem(float* S) {
    using G = VReg<TX, TY, H>;
    sb = S + G::PAD;
    s0 = sb + G::A;
    s1 = s0 + G::A;
    sw = s1 + G::A;
    sm = reinterpret_cast<uint8_t*>(S + 4 * G::A);
  }
};

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void sts4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float lane(const float4& v, int k) {
  return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}
__device__ __forceinline__ uint8_t lane(const uchar4& v, int k) {
  return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}
__device__ __forceinline__ void set_lane(float4& v, int k, float a) {
  if (k == 0) v.x = a;
  else if (k == 1) v.y = a;
  else if (k == 2) v.z = a;
  else v.w = a;
}
// cell bytes of a group (all fluid on a level without solid)
__device__ __forceinline__ uchar4 v_cells(const LevelDev& L, int gi) {
  if (gi < 0) return make_uchar4(0, 0, 0, 0);
  if (!L.cell) return make_uchar4(kFluidBit, kFluidBit, kFluidBit, kFluidBit);
  return *reinterpret_cast<const uchar4*>(L.cell + gi);
}
// left / right / down / up neighbours of lane k of the group at li
struct VNb {
  float4 c, d, u;
  float l, r;
  __device__ __forceinline__ VNb(const float* x, int li, int RX)
      : c(lds4(x + li)), d(lds4(x + li - RX)), u(lds4(x + li + RX)), l(x[li - 1]), r(x[li + 4]) {}
  __device__ __forceinline__ float left(int k) const { return k == 0 ? l : lane(c, k - 1); }
  __device__ __forceinline__ float right(int k) const { return k == 3 ? r : lane(c, k + 1); }
};

// one sweep over rows H - M .. H + TY + M - 1 of the region (all groups).
// Thread t owns group column t % W4 of rows t / W4, t / W4 + RPP, ... (RPP
// = rows per pass), so no group index is divided.  Cells off the fluid and
// off the grid hold x = 0 and omega / d = 0, so the update gives them 0
// with no test.
template <int TX, int TY, int H, int M>
__device__ __forceinline__ void v_sweep(const LevelDev& L, const float* __restrict__ xin, float* __restrict__ xout,
                                        const float* __restrict__ sb, const float* __restrict__ sw, float omega,
                                        bool from_zero) {
  using G = VReg<TX, TY, H>;
  constexpr int RPP = kBThreads / G::W4, NROW = TY + 2 * M, NI = (NROW + RPP - 1) / RPP;
  const float keep = 1.f - omega;
  const int c4 = threadIdx.x % G::W4, r0 = threadIdx.x / G::W4;
  if (r0 < RPP) {
#pragma unroll
    for (int j = 0; j < NI; ++j) {
      const int row = r0 + j * RPP;
      if (row >= NROW) break;
      const int li = (row + H - M) * G::RX + 4 * c4;
      const float4 w = lds4(sw + li), bb = lds4(sb + li);
      float4 v;
      if (from_zero) {
        v = make_float4(w.x * bb.x, w.y * bb.y, w.z * bb.z, w.w * bb.w);
      } else {
        const VNb n(xin, li, G::RX);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float nb = L.wx * (n.left(k) + n.right(k)) + L.wy * (lane(n.d, k) + lane(n.u, k));
          set_lane(v, k, keep * lane(n.c, k) + lane(w, k) * (lane(bb, k) + nb));
        }
      }
      sts4(xout + li, v);
    }
  }
  __syncthreads();
}

// b, omega / d and cell bytes of one region group into shared memory
template <int TX, int TY, int H>
__device__ __forceinline__ void v_stage(const LevelDev& L, const VReg<TX, TY, H>& g, const VSmem<TX, TY, H>& M,
                                        int q, uchar4 m4, float4 b4, float omega) {
  using G = VReg<TX, TY, H>;
  const int li = (q / G::W4) * G::RX + 4 * (q % G::W4);
  const int gx = g.ox + 4 * (q % G::W4), gy = g.oy + q / G::W4;
  float4 sb, sw;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint8_t m = lane(m4, k);
    set_lane(sb, k, m ? lane(b4, k) : 0.f);
    set_lane(sw, k, m ? __fdividef(omega, b_diag(L, gx + k, gy, m)) : 0.f);
  }
  sts4(M.sb + li, sb);
  sts4(M.sw + li, sw);
  *reinterpret_cast<uchar4*>(M.sm + li) = m4;
}

// down leg of one tile, float4 path
template <int TX, int TY, int H>
__device__ void v_down(const LevelDev& L, int tx, int ty, const float* __restrict__ b, float* __restrict__ x,
                       float* __restrict__ bc, float omega, float* S) {
  using G = VReg<TX, TY, H>;
  const G g(tx, ty);
  const VSmem<TX, TY, H> M(S);
  constexpr int NR = (G::NG + kBThreads - 1) / kBThreads;
  float4 bv[NR];
  uchar4 mv[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int gi = g.gidx(L, threadIdx.x + j * kBThreads);
    mv[j] = v_cells(L, gi);
    bv[j] = gi < 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(b + gi);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int q = threadIdx.x + j * kBThreads;
    if (q >= G::NG) break;
    v_stage(L, g, M, q, mv[j], bv[j], omega);
  }
  __syncthreads();
  v_sweep<TX, TY, H, H>(L, nullptr, M.s0, M.sb, M.sw, omega, true);
  float* cur = M.s0;
  if (H >= 2) {
    v_sweep<TX, TY, H, (H >= 2 ? H - 1 : 1)>(L, M.s0, M.s1, M.sb, M.sw, omega, false);
    cur = M.s1;
  }
  if (H >= 3) {
    v_sweep<TX, TY, H, 1>(L, M.s1, M.s0, M.sb, M.sw, omega, false);
    cur = M.s0;
  }
  constexpr int T4 = TX / 4;
#pragma unroll
  for (int q = threadIdx.x; q < TY * T4; q += kBThreads) {
    const int row = q / T4, c = q % T4;
    const int gx = tx * TX + 4 * c, gy = ty * TY + row;
    if (gx < L.nx && gy < L.ny)
      *reinterpret_cast<float4*>(x + gy * L.nx + gx) = lds4(cur + (row + H) * G::RX + 4 * (c + 1));
  }
  // residual and restriction, two coarse cells (a 4 x 2 block of fine cells)
  // per thread
  const int cnx = L.nx / 2, cny = L.ny / 2;
#pragma unroll
  for (int q = threadIdx.x; q < (TY / 2) * T4; q += kBThreads) {
    const int cy = q / T4, c = q % T4;
    const int gcx = tx * (TX / 2) + 2 * c, gcy = ty * (TY / 2) + cy;
    if (gcx >= cnx || gcy >= cny) continue;
    float sum[2] = {0.f, 0.f};
#pragma unroll
    for (int ay = 0; ay < 2; ++ay) {
      const int ly = H + 2 * cy + ay, li = ly * G::RX + 4 * (c + 1);
      const VNb n(cur, li, G::RX);
      const float4 b4 = lds4(M.sb + li);
      const uchar4 m4 = *reinterpret_cast<const uchar4*>(M.sm + li);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint8_t mm = lane(m4, k);
        if (!mm) continue;
        const float d = b_diag(L, g.ox + 4 * (c + 1) + k, g.oy + ly, mm);
        const float nb = L.wx * (n.left(k) + n.right(k)) + L.wy * (lane(n.d, k) + lane(n.u, k));
        sum[k >> 1] += lane(b4, k) - (d * lane(n.c, k) - nb);
      }
    }
    *reinterpret_cast<float2*>(bc + gcy * cnx + gcx) = make_float2(0.25f * sum[0], 0.25f * sum[1]);
  }
}

// up leg of one tile, float4 path: x + s P e, H sweeps, output; returns this
// thread's share of (b, out) when `dot`
template <int TX, int TY, int H>
__device__ float v_up(const LevelDev& L, int tx, int ty, const float* __restrict__ b, const float* __restrict__ xin,
                      float* __restrict__ xout, const float* __restrict__ e, float omega, float s, bool dot,
                      float* S) {
  using G = VReg<TX, TY, H>;
  const G g(tx, ty);
  const VSmem<TX, TY, H> M(S);
  const int cnx = L.nx / 2;
  constexpr int NR = (G::NG + kBThreads - 1) / kBThreads;
  float4 xv[NR], bv[NR];
  float2 ev[NR];
  uchar4 mv[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int q = threadIdx.x + j * kBThreads;
    const int gi = g.gidx(L, q);
    const int gx = g.ox + 4 * (q % G::W4), gy = g.oy + q / G::W4;
    mv[j] = v_cells(L, gi);
    xv[j] = gi < 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(xin + gi);
    bv[j] = gi < 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(b + gi);
    ev[j] = gi < 0 ? make_float2(0.f, 0.f) : *reinterpret_cast<const float2*>(e + (gy >> 1) * cnx + (gx >> 1));
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int q = threadIdx.x + j * kBThreads;
    if (q >= G::NG) break;
    const int li = (q / G::W4) * G::RX + 4 * (q % G::W4);
    float4 v;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      set_lane(v, k, lane(mv[j], k) ? lane(xv[j], k) + s * (k < 2 ? ev[j].x : ev[j].y) : 0.f);
    sts4(M.s0 + li, v);
    v_stage(L, g, M, q, mv[j], bv[j], omega);
  }
  __syncthreads();
  float* cur = M.s0;
  if (H == 1) {
    v_sweep<TX, TY, H, 0>(L, M.s0, M.s1, M.sb, M.sw, omega, false);
    cur = M.s1;
  } else if (H == 2) {
    v_sweep<TX, TY, H, 1>(L, M.s0, M.s1, M.sb, M.sw, omega, false);
    v_sweep<TX, TY, H, 0>(L, M.s1, M.s0, M.sb, M.sw, omega, false);
  } else {
    v_sweep<TX, TY, H, (H >= 3 ? 2 : 0)>(L, M.s0, M.s1, M.sb, M.sw, omega, false);
    v_sweep<TX, TY, H, 1>(L, M.s1, M.s0, M.sb, M.sw, omega, false);
    v_sweep<TX, TY, H, 0>(L, M.s0, M.s1, M.sb, M.sw, omega, false);
    cur = M.s1;
  }
  float acc = 0.f;
  constexpr int T4 = TX / 4;
#pragma unroll
  for (int q = threadIdx.x; q < TY * T4; q += kBThreads) {
    const int row = q / T4, c = q % T4;
    const int gx = tx * TX + 4 * c, gy = ty * TY + row;
    if (gx < L.nx && gy < L.ny) {
      const int li = (row + H) * G::RX + 4 * (c + 1);
      const float4 v = lds4(cur + li);
      *reinterpret_cast<float4*>(xout + gy * L.nx + gx) = v;
      if (dot) {
        const float4 bb = lds4(M.sb + li);
        acc = fmaf(bb.x, v.x, acc);
        acc = fmaf(bb.y, v.y, acc);
        acc = fmaf(bb.z, v.z, acc);
        acc = fmaf(bb.w, v.w, acc);
      }
    }
  }
  return acc;
}

// p = z + beta p_old on a level-0 tile and its halo (one group in x, one
// row in y; staged in shared memory, zero off the fluid and off the grid),
// then Ap and the thread's share of (p, Ap) on the tile
template <int TX, int TY>
__device__ float b_pupdate(const LevelDev& L, int tx, int ty, const float* __restrict__ z,
                           const float* __restrict__ pold, float* __restrict__ pnew, float* __restrict__ Ap,
                           float beta, bool first, float* S) {
  using G = VReg<TX, TY, 1>;
  const G g(tx, ty);
  float* sp = S + G::PAD;
  uint8_t* sm = reinterpret_cast<uint8_t*>(S + G::A);
  constexpr int NR = (G::NG + kBThreads - 1) / kBThreads;
  float4 zv[NR], pv[NR];
  uchar4 mv[NR];
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int gi = g.gidx(L, threadIdx.x + j * kBThreads);
    mv[j] = v_cells(L, gi);
    zv[j] = gi < 0 ? zero : *reinterpret_cast<const float4*>(z + gi);
    pv[j] = (gi < 0 || first) ? zero : *reinterpret_cast<const float4*>(pold + gi);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int q = threadIdx.x + j * kBThreads;
    if (q >= G::NG) break;
    const int li = (q / G::W4) * G::RX + 4 * (q % G::W4);
    float4 v;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      set_lane(v, k, lane(mv[j], k) ? (first ? lane(zv[j], k) : fmaf(beta, lane(pv[j], k), lane(zv[j], k))) : 0.f);
    sts4(sp + li, v);
    *reinterpret_cast<uchar4*>(sm + li) = mv[j];
  }
  __syncthreads();
  float acc = 0.f;
  constexpr int T4 = TX / 4;
#pragma unroll
  for (int q = threadIdx.x; q < TY * T4; q += kBThreads) {
    const int row = q / T4, c = q % T4;
    const int gx = tx * TX + 4 * c, gy = ty * TY + row;
    if (gx >= L.nx || gy >= L.ny) continue;
    const int li = (row + 1) * G::RX + 4 * (c + 1);
    const VNb n(sp, li, G::RX);
    const uchar4 m4 = *reinterpret_cast<const uchar4*>(sm + li);
    float4 pc = zero, ap = zero;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint8_t m = lane(m4, k);
      if (!m) continue;
      const float p = lane(n.c, k);
      float nb = 0.f;
      nb += L.wx * n.left(k);
      nb += L.wx * n.right(k);
      nb += L.wy * lane(n.d, k);
      nb += L.wy * lane(n.u, k);
      const float a = b_diag(L, gx + k, gy, m) * p - nb;
      set_lane(pc, k, p);
      set_lane(ap, k, a);
      acc = fmaf(p, a, acc);
    }
    *reinterpret_cast<float4*>(pnew + gy * L.nx + gx) = pc;
    *reinterpret_cast<float4*>(Ap + gy * L.nx + gx) = ap;
  }
  return acc;
}

// d += alpha p (d = alpha p on the first iteration), r -= alpha Ap on a
// level-0 tile, four cells per access; returns the thread's share of ||r||^2
template <int TX, int TY>
__device__ float b_xr(const LevelDev& L, int tx, int ty, float* __restrict__ d, const float* __restrict__ p,
                      const float* __restrict__ Ap, float* __restrict__ r, float alpha, bool first) {
  constexpr int T4 = TX / 4, NG = TY * T4, NI = (NG + kBThreads - 1) / kBThreads;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 dv[NI], pv[NI], av[NI], rv[NI];
  int gi[NI];
#pragma unroll
  for (int j = 0; j < NI; ++j) {
    const int q = threadIdx.x + j * kBThreads;
    const int x = tx * TX + 4 * (q % T4), y = ty * TY + q / T4;
    gi[j] = (q < NG && x < L.nx && y < L.ny) ? y * L.nx + x : -1;
    dv[j] = (gi[j] < 0 || first) ? zero : *reinterpret_cast<const float4*>(d + gi[j]);
    pv[j] = gi[j] < 0 ? zero : *reinterpret_cast<const float4*>(p + gi[j]);
    av[j] = gi[j] < 0 ? zero : *reinterpret_cast<const float4*>(Ap + gi[j]);
    rv[j] = gi[j] < 0 ? zero : *reinterpret_cast<const float4*>(r + gi[j]);
  }
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < NI; ++j) {
    if (gi[j] < 0) continue;
    float4 dn, rn;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float pk = lane(pv[j], k);
      set_lane(dn, k, first ? alpha * pk : fmaf(alpha, pk, lane(dv[j], k)));
      const float rk = fmaf(-alpha, lane(av[j], k), lane(rv[j], k));
      set_lane(rn, k, rk);
      acc = fmaf(rk, rk, acc);
    }
    *reinterpret_cast<float4*>(d + gi[j]) = dn;
    *reinterpret_cast<float4*>(r + gi[j]) = rn;
  }
  return acc;
}

template <int TX, int TY>
__device__ __forceinline__ void b_down(const LevelDev& L, int tx, int ty, const float* __restrict__ b,
                                       float* __restrict__ x, float* __restrict__ bc, int sweeps, float omega,
                                       float* S) {
  if ((L.nx & 3) == 0) {
    if (sweeps <= 1) v_down<TX, TY, 1>(L, tx, ty, b, x, bc, omega, S);
    else if (sweeps == 2) v_down<TX, TY, 2>(L, tx, ty, b, x, bc, omega, S);
    else v_down<TX, TY, 3>(L, tx, ty, b, x, bc, omega, S);
  } else {
    if (sweeps <= 1) b_down_h<TX, TY, 1>(L, tx, ty, b, x, bc, omega, S);
    else if (sweeps == 2) b_down_h<TX, TY, 2>(L, tx, ty, b, x, bc, omega, S);
    else b_down_h<TX, TY, 3>(L, tx, ty, b, x, bc, omega, S);
  }
}

template <int TX, int TY>
__device__ __forceinline__ float b_up(const LevelDev& L, int tx, int ty, const float* __restrict__ b,
                                      const float* __restrict__ xin, float* __restrict__ xout,
                                      const float* __restrict__ e, int sweeps, float omega, float s, bool dot,
                                      float* S) {
  if ((L.nx & 3) == 0) {
    if (sweeps <= 1) return v_up<TX, TY, 1>(L, tx, ty, b, xin, xout, e, omega, s, dot, S);
    if (sweeps == 2) return v_up<TX, TY, 2>(L, tx, ty, b, xin, xout, e, omega, s, dot, S);
    return v_up<TX, TY, 3>(L, tx, ty, b, xin, xout, e, omega, s, dot, S);
  }
  if (sweeps <= 1) return b_up_h<TX, TY, 1>(L, tx, ty, b, xin, xout, e, omega, s, dot, S);
  if (sweeps == 2) return b_up_h<TX, TY, 2>(L, tx, ty, b, xin, xout, e, omega, s, dot, S);
  return b_up_h<TX, TY, 3>(L, tx, ty, b, xin, xout, e, omega, s, dot, S);
}

// ---------------------------------------------------------------------------
// refinement phases on float4 groups of a level-0 tile (the caller's arrays
// 16-byte aligned; else the cell-by-cell loops below)
__device__ __forceinline__ bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// init: x = (guess, 0) on fluid cells (0 elsewhere); returns the thread's
// share of ||b||^2
template <int TX, int TY>
__device__ float v_init(const LevelDev& L, int tx, int ty, const float* __restrict__ b,
                        const float* __restrict__ xg, float2* __restrict__ xf) {
  constexpr int T4 = TX / 4, NG = TY * T4, NI = (NG + kBThreads - 1) / kBThreads;
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < NI; ++j) {
    const int q = threadIdx.x + j * kBThreads;
    const int x = tx * TX + 4 * (q % T4), y = ty * TY + q / T4;
    if (q >= NG || x >= L.nx || y >= L.ny) continue;
    const int gi = y * L.nx + x;
    const uchar4 m = v_cells(L, gi);
    const float4 g = *reinterpret_cast<const float4*>(xg + gi), bb = *reinterpret_cast<const float4*>(b + gi);
    float4* o = reinterpret_cast<float4*>(xf + gi);
    o[0] = make_float4(m.x ? g.x : 0.f, 0.f, m.y ? g.y : 0.f, 0.f);
    o[1] = make_float4(m.z ? g.z : 0.f, 0.f, m.w ? g.w : 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (lane(m, k)) acc = fmaf(lane(bb, k), lane(bb, k), acc);
  }
  return acc;
}

// result: the float32 output hi + lo (0 for a zero right-hand side)
template <int TX, int TY>
__device__ void v_result(const LevelDev& L, int tx, int ty, const float2* __restrict__ xf, float* __restrict__ out,
                         bool zero) {
  constexpr int T4 = TX / 4, NG = TY * T4, NI = (NG + kBThreads - 1) / kBThreads;
#pragma unroll
  for (int j = 0; j < NI; ++j) {
    const int q = threadIdx.x + j * kBThreads;
    const int x = tx * TX + 4 * (q % T4), y = ty * TY + q / T4;
    if (q >= NG || x >= L.nx || y >= L.ny) continue;
    const int gi = y * L.nx + x;
    const float4 a = reinterpret_cast<const float4*>(xf + gi)[0], c = reinterpret_cast<const float4*>(xf + gi)[1];
    *reinterpret_cast<float4*>(out + gi) =
        zero ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4(a.x + a.y, a.z + a.w, c.x + c.y, c.z + c.w);
  }
}

// refinement residual of the float-float iterate after x += sigma_old d
// (when `update`): the iterate of the tile and a one-cell ring is staged in
// shared memory as (hi, lo) planes, then r = c b - A' x per fluid cell in
// float-float, scaled by 1 / sigma_new into the CG right-hand side; returns
// the thread's share of ||r||^2
template <int TX, int TY>
__device__ float v_resid(const BInst& I, const LevelDev& L, int tx, int ty, const float* __restrict__ b,
                         const float2* __restrict__ xin, float2* __restrict__ xo, bool update, float sig_old,
                         float inv_sig_new, float* S) {
  using G = VReg<TX, TY, 1>;
  const G g(tx, ty);
  float* sh = S + G::PAD;
  float* sl = sh + G::A;
  uint8_t* sm = reinterpret_cast<uint8_t*>(S + 2 * G::A);
  auto xv = [&](float hi, float lo, float dd) -> ff {
    if (!update) return {hi, lo};
    const ff s2 = two_sum(hi, sig_old * dd);
    return quick_two_sum(s2.hi, s2.lo + lo);
  };
  __syncthreads();
  for (int q = threadIdx.x; q < G::NG; q += kBThreads) {
    const int gi = g.gidx(L, q);
    const int li = (q / G::W4) * G::RX + 4 * (q % G::W4);
    float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
    uchar4 m = make_uchar4(0, 0, 0, 0);
    if (gi >= 0) {
      m = v_cells(L, gi);
      const float4 a = reinterpret_cast<const float4*>(xin + gi)[0], c = reinterpret_cast<const float4*>(xin + gi)[1];
      const float4 dd = update ? *reinterpret_cast<const float4*>(I.d + gi) : make_float4(0.f, 0.f, 0.f, 0.f);
      const ff v0 = xv(a.x, a.y, dd.x), v1 = xv(a.z, a.w, dd.y), v2 = xv(c.x, c.y, dd.z), v3 = xv(c.z, c.w, dd.w);
      h = make_float4(v0.hi, v1.hi, v2.hi, v3.hi);
      l = make_float4(v0.lo, v1.lo, v2.lo, v3.lo);
    }
    sts4(sh + li, h);
    sts4(sl + li, l);
    *reinterpret_cast<uchar4*>(sm + li) = m;
  }
  __syncthreads();
  float acc = 0.f;
  constexpr int T4 = TX / 4;
  for (int q = threadIdx.x; q < TY * T4; q += kBThreads) {
    const int row = q / T4, c4 = q % T4;
    const int gx = tx * TX + 4 * c4, gy = ty * TY + row;
    if (gx >= L.nx || gy >= L.ny) continue;
    const int gi = gy * L.nx + gx;
    const int li = (row + 1) * G::RX + 4 * (c4 + 1);
    const VNb H(sh, li, G::RX), Lo(sl, li, G::RX);
    const uchar4 m4 = *reinterpret_cast<const uchar4*>(sm + li);
    const float4 bb = *reinterpret_cast<const float4*>(b + gi);
    float4 rv = make_float4(0.f, 0.f, 0.f, 0.f), oh = rv, ol = rv;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint8_t m = lane(m4, k);
      if (!m) continue;
      const int kx = L.cell ? (m & 3) : axis_count(gx + k, L.nx, L.bcD, 0);
      const int ky = L.cell ? ((m >> 2) & 3) : axis_count(gy, L.ny, L.bcD, 2);
      const ff xc = {lane(H.c, k), lane(Lo.c, k)};
      const ff xl = {H.left(k), Lo.left(k)}, xr = {H.right(k), Lo.right(k)};
      const ff xd = {lane(H.d, k), lane(Lo.d, k)}, xu = {lane(H.u, k), lane(Lo.u, k)};
      ff ax = ff_mul(ff_add(ff_mul(xc, ff{(float)kx, 0.f}), ff_neg(ff_add(xl, xr))), I.wff[0]);
      ax = ff_add(ax, ff_mul(ff_add(ff_mul(xc, ff{(float)ky, 0.f}), ff_neg(ff_add(xd, xu))), I.wff[1]));
      const ff r = ff_add(ff_mul(ff{lane(bb, k), 0.f}, I.cff), ff_neg(ax));
      const float rs = r.hi + r.lo;
      set_lane(rv, k, rs * inv_sig_new);
      acc = fmaf(rs, rs, acc);
      set_lane(oh, k, xc.hi);
      set_lane(ol, k, xc.lo);
    }
    *reinterpret_cast<float4*>(I.r + gi) = rv;
    if (update) {
      float4* o = reinterpret_cast<float4*>(xo + gi);
      o[0] = make_float4(oh.x, ol.x, oh.y, ol.y);
      o[1] = make_float4(oh.z, ol.z, oh.w, ol.w);
    }
  }
  return acc;
}

// cells of a level-0 tile, one by one: callback(i, x, y)
template <int TX, int TY, typename F>
__device__ __forceinline__ void b_cells(const BInst& I, int tx, int ty, F&& f) {
  for (int j = threadIdx.x; j < TX * TY; j += blockDim.x) {
    const int x = tx * TX + j % TX, y = ty * TY + j / TX;
    if (x < I.nx && y < I.ny) f((size_t)y * I.nx + x, x, y);
  }
}

__device__ __forceinline__ double block_total(float v) {
  __shared__ double sh[32];
  __shared__ double tot;
  const double t = block_sum((double)v, sh);
  if (threadIdx.x == 0) tot = t;
  __syncthreads();
  return tot;
}

// per-instance fixed-order reduction of the level-0 tile partial slots
__device__ __forceinline__ double reduce_slots(const BatchArgs& A, const BInst& I) {
  double acc = 0.0;
  for (int j = threadIdx.x; j < I.ntiles0; j += blockDim.x) acc += __ldcg(A.partials + I.slot0 + j);
  __shared__ double sh[32];
  __shared__ double tot;
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) tot = t;
  __syncthreads();
  return tot;
}

// active-instance counters alternate between two slots (the reducing phase
// clears the other one for the next count)
__device__ __forceinline__ void count_active(const BatchArgs& A, int slot, bool active) {
  if (threadIdx.x == 0 && active) atomicAdd(A.bar + 4 + slot, 1u);
}

template <int TX, int TY>
__global__ void __launch_bounds__(kBThreads, 4) k_batched(const __grid_constant__ BatchArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* S = reinterpret_cast<float*>(smem_raw);
  unsigned epoch = 0;
  int cslot = 0;
  const int4* it0 = A.items[0];
  const int n0 = A.nitems[0];
  const float omega = A.omega;
  // ---- init: x = (guess, 0) on fluid cells, ||b||^2 per tile
  for (int w = blockIdx.x; w < n0; w += gridDim.x) {
    const int4 item = it0[w];
    const BInst& I = A.inst[item.x];
    const float* b = A.rhs[item.x];
    const float* xg = A.xin[item.x];
    float acc = 0.f;
    if (aligned16(b) && aligned16(xg)) {
      acc = v_init<TX, TY>(I.lv[0], item.y, item.z, b, xg, I.xf0);
    } else {
      b_cells<TX, TY>(I, item.y, item.z, [&](size_t i, int, int) {
        const bool fl = I.lv[0].cell ? I.lv[0].cell[i] != 0 : true;
        I.xf0[i] = make_float2(fl ? xg[i] : 0.f, 0.f);
        if (fl) acc = fmaf(b[i], b[i], acc);
      });
    }
    const double t = block_total(acc);
    if (threadIdx.x == 0) A.partials[item.w] = t;
  }
  if (!grid_barrier(A, epoch)) return;
  for (int w = blockIdx.x; w < A.count; w += gridDim.x) {
    const BInst& I = A.inst[w];
    const double tot = reduce_slots(A, I);
    if (threadIdx.x == 0) {
      SolveParams prm = A.prm;
      prm.n_fluid = I.nfluid > 0 ? I.nfluid : 1;
      init_state(&A.st[w], prm, tot, I.c);
      A.cur[w] = 0;
    }
  }
  if (!grid_barrier(A, epoch)) return;
  // ---- refinement loop
  for (int outer = 0; outer <= A.prm.max_outer; ++outer) {
    const bool update = outer > 0;
    // residual of the float-float iterate (after x += sigma d')
    for (int w = blockIdx.x; w < n0; w += gridDim.x) {
      const int4 item = it0[w];
      SolveState& st = A.st[item.x];
      if (st.outer_done) continue;
      const BInst& I = A.inst[item.x];
      const LevelDev& L = I.lv[0];
      const float* b = A.rhs[item.x];
      const int cur = A.cur[item.x];
      const float2* xin = cur ? I.xf1 : I.xf0;
      float2* xo = cur ? I.xf0 : I.xf1;
      const double sig_old_d = st.sigma;
      const double sig_new_d =
          update ? pow2_floor(sig_old_d * sqrt(fmax(st.rnorm2, 1e-300) / (double)st.n_fluid)) : sig_old_d;
      const float sig_old = (float)sig_old_d, inv_sig_new = (float)(1.0 / sig_new_d);
      auto xv = [&](size_t j) -> ff {
        const float2 q = xin[j];
        if (!update) return {q.x, q.y};
        const ff s2 = two_sum(q.x, sig_old * I.d[j]);
        return quick_two_sum(s2.hi, s2.lo + q.y);
      };
      float acc = 0.f;
      if (aligned16(b)) acc = v_resid<TX, TY>(I, L, item.y, item.z, b, xin, xo, update, sig_old, inv_sig_new, S);
      else b_cells<TX, TY>(I, item.y, item.z, [&](size_t i, int cx, int cy) {
        const uint8_t m = L.cell ? L.cell[i] : kFluidBit;
        if (!m) {
          if (update) xo[i] = make_float2(0.f, 0.f);
          I.r[i] = 0.f;
          return;
        }
        const int kx = L.cell ? (m & 3) : axis_count(cx, L.nx, L.bcD, 0);
        const int ky = L.cell ? ((m >> 2) & 3) : axis_count(cy, L.ny, L.bcD, 2);
        const ff zero = {0.f, 0.f};
        const ff xc = xv(i);
        const ff xl = cx > 0 ? xv(i - 1) : zero, xr = cx < L.nx - 1 ? xv(i + 1) : zero;
        const ff xd = cy > 0 ? xv(i - L.nx) : zero, xu = cy < L.ny - 1 ? xv(i + L.nx) : zero;
        ff ax = ff_mul(ff_add(ff_mul(xc, ff{(float)kx, 0.f}), ff_neg(ff_add(xl, xr))), I.wff[0]);
        ax = ff_add(ax, ff_mul(ff_add(ff_mul(xc, ff{(float)ky, 0.f}), ff_neg(ff_add(xd, xu))), I.wff[1]));
        const ff r = ff_add(ff_mul(ff{b[i], 0.f}, I.cff), ff_neg(ax));
        const float rs = r.hi + r.lo;
        I.r[i] = rs * inv_sig_new;
        acc = fmaf(rs, rs, acc);
        if (update) xo[i] = make_float2(xc.hi, xc.lo);
      });
      const double t = block_total(acc);
      if (threadIdx.x == 0) A.partials[item.w] = t;
    }
    if (!grid_barrier(A, epoch)) return;
    for (int w = blockIdx.x; w < A.count; w += gridDim.x) {
      SolveState& st = A.st[w];
      if (st.outer_done) continue;
      const BInst& I = A.inst[w];
      const double tot = reduce_slots(A, I);
      if (threadIdx.x == 0) {
        const double sig_old_d = st.sigma;
        const double sig_new_d =
            update ? pow2_floor(sig_old_d * sqrt(fmax(st.rnorm2, 1e-300) / (double)st.n_fluid)) : sig_old_d;
        if (update) A.cur[w] ^= 1;
        outer_decide(&st, tot, I.c2, sig_new_d, update);
        st.first = 1;
      }
      __syncthreads();
      count_active(A, cslot, !st.outer_done);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) A.bar[4 + (cslot ^ 1)] = 0u;
    if (!grid_barrier(A, epoch)) return;
    const unsigned active_outer = *(volatile unsigned*)(A.bar + 4 + cslot);
    cslot ^= 1;
    if (active_outer == 0) break;
    // ---- CG iterations
    for (int iter = 0; iter < A.prm.max_inner; ++iter) {
      // down legs, level by level
      for (int k = 0; k < A.ntile_levels; ++k) {
        const int4* its = A.items[k];
        for (int w = blockIdx.x; w < A.nitems[k]; w += gridDim.x) {
          const int4 item = its[w];
          if (A.st[item.x].inner_done) continue;
          const BInst& I = A.inst[item.x];
          b_down<TX, TY>(I.lv[k], item.y, item.z, k == 0 ? I.r : I.b[k], I.x[k], I.b[k + 1], A.sweeps, omega, S);
        }
        if (!grid_barrier(A, epoch)) return;
      }
      // block-local coarse part of each instance
      for (int w = blockIdx.x; w < A.count; w += gridDim.x) {
        if (A.st[w].inner_done) continue;
        const BInst& I = A.inst[w];
        __syncthreads();
        coarse_cycle<2, float, false>(I.ca, I.kc == 0 ? I.r : I.b[I.kc], I.kc == 0 ? I.z : I.y[I.kc], nullptr, S,
                               I.cfloats);
      }
      if (!grid_barrier(A, epoch)) return;
      // up legs; the finest produces z = M r and (r, z)
      for (int k = A.ntile_levels - 1; k >= 0; --k) {
        const int4* its = A.items[k];
        for (int w = blockIdx.x; w < A.nitems[k]; w += gridDim.x) {
          const int4 item = its[w];
          if (A.st[item.x].inner_done) continue;
          const BInst& I = A.inst[item.x];
          const float acc = b_up<TX, TY>(I.lv[k], item.y, item.z, k == 0 ? I.r : I.b[k], I.x[k],
                                         k == 0 ? I.z : I.y[k], I.y[k + 1], A.sweeps, omega, A.s, k == 0, S);
          if (k == 0) {
            const double t = block_total(acc);
            if (threadIdx.x == 0) A.partials[item.w] = t;
          }
        }
        if (!grid_barrier(A, epoch)) return;
      }
      // (r, z) per instance -> beta
      for (int w = blockIdx.x; w < A.count; w += gridDim.x) {
        SolveState& st = A.st[w];
        if (st.inner_done) continue;
        const BInst& I = A.inst[w];
        const double tot = reduce_slots(A, I);
        if (threadIdx.x == 0) {
          st.rz = tot;
          st.beta = (st.first || !st.krylov) ? 0.0 : tot / st.rz_old;
          st.rz_old = tot;
        }
      }
      if (!grid_barrier(A, epoch)) return;
      // p = z + beta p, Ap, (p, Ap)
      for (int w = blockIdx.x; w < n0; w += gridDim.x) {
        const int4 item = it0[w];
        const SolveState& st = A.st[item.x];
        if (st.inner_done) continue;
        const BInst& I = A.inst[item.x];
        const bool first = st.first || !st.krylov;
        const float beta = first ? 0.f : (float)st.beta;
        const float* pold = (st.it & 1) ? I.p1 : I.p0;
        float* pnew = (st.it & 1) ? I.p0 : I.p1;
        const float acc = b_pupdate<TX, TY>(I.lv[0], item.y, item.z, I.z, pold, pnew, I.Ap, beta, first, S);
        const double t = block_total(acc);
        if (threadIdx.x == 0) A.partials[item.w] = t;
      }
      if (!grid_barrier(A, epoch)) return;
      for (int w = blockIdx.x; w < A.count; w += gridDim.x) {
        SolveState& st = A.st[w];
        if (st.inner_done) continue;
        const double tot = reduce_slots(A, A.inst[w]);
        if (threadIdx.x == 0) {
          st.pAp = tot;
          st.alpha = st.krylov ? st.rz / tot : 1.0;
        }
      }
      if (!grid_barrier(A, epoch)) return;
      // d += alpha p, r -= alpha Ap, ||r||^2
      for (int w = blockIdx.x; w < n0; w += gridDim.x) {
        const int4 item = it0[w];
        const SolveState& st = A.st[item.x];
        if (st.inner_done) continue;
        const BInst& I = A.inst[item.x];
        const float alpha = (float)st.alpha;
        const float* p = (st.it & 1) ? I.p0 : I.p1;
        const float acc = b_xr<TX, TY>(I.lv[0], item.y, item.z, I.d, p, I.Ap, I.r, alpha, st.first != 0);
        const double t = block_total(acc);
        if (threadIdx.x == 0) A.partials[item.w] = t;
      }
      if (!grid_barrier(A, epoch)) return;
      for (int w = blockIdx.x; w < A.count; w += gridDim.x) {
        SolveState& st = A.st[w];
        if (st.inner_done) continue;
        const double tot = reduce_slots(A, A.inst[w]);
        if (threadIdx.x == 0) inner_decide(&st, tot);
        __syncthreads();
        count_active(A, cslot, !st.inner_done);
      }
      if (blockIdx.x == 0 && threadIdx.x == 0) A.bar[4 + (cslot ^ 1)] = 0u;
      if (!grid_barrier(A, epoch)) return;
      const unsigned active = *(volatile unsigned*)(A.bar + 4 + cslot);
      cslot ^= 1;
      if (active == 0) break;
    }
  }
  // ---- result: float output = hi + lo; zero right-hand side -> zero solution
  for (int w = blockIdx.x; w < n0; w += gridDim.x) {
    const int4 item = it0[w];
    const BInst& I = A.inst[item.x];
    const SolveState& st = A.st[item.x];
    const float2* xf = A.cur[item.x] ? I.xf1 : I.xf0;
    float* out = A.xout[item.x];
    const bool zero = st.bnorm2 == 0.0;
    if (aligned16(out)) {
      v_result<TX, TY>(I.lv[0], item.y, item.z, xf, out, zero);
    } else {
      b_cells<TX, TY>(I, item.y, item.z, [&](size_t i, int, int) {
        const float2 v = xf[i];
        out[i] = zero ? 0.f : v.x + v.y;
      });
    }
  }
}

// ---------------------------------------------------------------------------
// host side
struct TileChoice {
  int tx, ty;
};
constexpr int kNTiles = 5;
static const TileChoice kTiles[kNTiles] = {{64, 16}, {32, 16}, {128, 8}, {64, 32}, {128, 16}};

template <int TX, int TY>
static void* kernel_ptr() {
  return (void*)k_batched<TX, TY>;
}
static void* batched_kernel(int t) {
  if (t == 0) return kernel_ptr<64, 16>();
  if (t == 1) return kernel_ptr<32, 16>();
  if (t == 2) return kernel_ptr<128, 8>();
  if (t == 3) return kernel_ptr<64, 32>();
  return kernel_ptr<128, 16>();
}

}  // namespace npmg

using namespace npmg;

struct GraphKey {
  double tol, timeout;
  int withhold;
  bool operator==(const GraphKey& o) const { return tol == o.tol && timeout == o.timeout && withhold == o.withhold; }
};

struct mg_batch_s {
  int count, device, nsm;
  mg_options opt;
  double inner_floor;
  std::vector<BInst> inst;       // host copy
  BInst* d_inst;
  SolveState* d_st;
  SolveState* h_st;              // pinned
  int* d_cur;
  const float** d_rhs;
  float** d_xout;
  const float** d_xin;           // guesses read by the init phase
  void** h_ptrs;                 // pinned staging of the pointer tables
  std::vector<int4*> d_items;
  int nitems[kMaxLevels];
  int ntile_levels;
  double* d_partials;
  unsigned* d_bar;
  char* pool;
  size_t pool_bytes;
  int tile, sweeps;              // current choice (autotuned)
  size_t smem[kNTiles][4];             // dynamic shared memory per (tile, sweeps)
  int grid[kNTiles][4];
  cudaGraphExec_t graph[kNTiles][4];
  GraphKey gkey[kNTiles][4];
  int withhold;
  double timeout_s;
  cudaEvent_t ev0, ev1;
  std::string tune_key;
};

static size_t batched_smem(int tx, int ty, int sweeps, size_t coarse_bytes) {
  const int h = sweeps < 1 ? 1 : (sweeps > 3 ? 3 : sweeps);
  // scalar tile: halo h on every side; float4 tile: one group of 4 in x and
  // h rows in y, arrays padded by 4 floats at both ends
  const size_t R = (size_t)(tx + 2 * h) * (ty + 2 * h), Rv = (size_t)(tx + 8) * (ty + 2 * h);
  const size_t t = 4 * R * 4 + ((R + 15) & ~size_t(15));  // b, two iterates, omega/d; cell bytes
  const size_t tv = 4 * (Rv + 8) * 4 + ((Rv + 15) & ~size_t(15));
  size_t m = t > tv ? t : tv;
  return m > coarse_bytes ? m : coarse_bytes;
}

static std::string tune_cache_path() {
  const char* e = getenv("NPMG_TUNE_CACHE");
  if (e && *e) return e;
  const char* home = getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/npmg_batched_tune.txt";
}

// cache lines: "<key> <tile> <sweeps> <ms>"
static bool tune_lookup(const std::string& key, int* tile, int* sweeps) {
  FILE* f = fopen(tune_cache_path().c_str(), "r");
  if (!f) return false;
  char k[512];
  int t, s;
  double ms;
  bool found = false;
  while (fscanf(f, "%511s %d %d %lf", k, &t, &s, &ms) == 4)
    if (key == k && t >= 0 && t < kNTiles && s >= 1 && s <= 3) {
      *tile = t;
      *sweeps = s;
      found = true;
    }
  fclose(f);
  return found;
}

static void tune_store(const std::string& key, int tile, int sweeps, double ms) {
  std::string path = tune_cache_path();
  std::string dir = path.substr(0, path.find_last_of('/'));
  if (!dir.empty()) mkdir(dir.c_str(), 0755);  // may already exist
  FILE* f = fopen(path.c_str(), "a");
  if (!f) return;
  fprintf(f, "%s %d %d %.4f\n", key.c_str(), tile, sweeps, ms);
  fclose(f);
}

static mg_status batched_launch(mg_batch_s* B, int tile, int sweeps, double tol, cudaStream_t s) {
  BatchArgs A;
  memset(&A, 0, sizeof(A));
  A.inst = B->d_inst;
  A.st = B->d_st;
  A.cur = B->d_cur;
  A.rhs = B->d_rhs;
  A.xout = B->d_xout;
  A.xin = B->d_xin;
  A.count = B->count;
  for (int k = 0; k < kMaxLevels; ++k) {
    A.items[k] = k < (int)B->d_items.size() ? B->d_items[k] : nullptr;
    A.nitems[k] = B->nitems[k];
  }
  A.ntile_levels = B->ntile_levels;
  A.partials = B->d_partials;
  A.bar = B->d_bar;
  A.sweeps = sweeps;
  A.omega = (float)B->opt.omega;
  A.s = (float)B->opt.coarse_scale;
  A.prm.tol = tol;
  A.prm.inner_floor = B->inner_floor;
  A.prm.max_inner = B->opt.max_inner;
  A.prm.max_outer = B->opt.max_outer;
  A.prm.krylov = B->opt.krylov;
  A.spin_limit = (long long)(B->timeout_s * 1e9 / 200.0) + 1;
  A.withhold = B->withhold;
  void* args[] = {&A};
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(B->grid[tile][sweeps], 1, 1);
  cfg.blockDim = dim3(kBThreads, 1, 1);
  cfg.dynamicSmemBytes = B->smem[tile][sweeps];
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeCooperative;
  attr.val.cooperative = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  // one persistent launch per solve, captured once in a CUDA graph (per tile
  // shape and sweep depth; recaptured when the tolerance or hooks change)
  GraphKey key{tol, B->timeout_s, B->withhold};
  if (!B->graph[tile][sweeps] || !(B->gkey[tile][sweeps] == key)) {
    if (B->graph[tile][sweeps]) cudaGraphExecDestroy(B->graph[tile][sweeps]);
    B->graph[tile][sweeps] = nullptr;
    cudaStream_t cs;
    NPMG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cfg.stream = cs;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = cudaMemsetAsync(B->d_bar, 0, 8 * sizeof(unsigned), cs);
      cudaError_t e2 = cudaLaunchKernelExC(&cfg, batched_kernel(tile), args);
      e = cudaStreamEndCapture(cs, &g);
      if (e1 != cudaSuccess) e = e1;
      if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&B->graph[tile][sweeps], g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      set_error("batched solve: graph capture failed: %s", cudaGetErrorString(e));
      return MG_ERR_CUDA;
    }
    B->gkey[tile][sweeps] = key;
  }
  NPMG_CUDA(cudaGraphLaunch(B->graph[tile][sweeps], s));
  return MG_OK;
}

static mg_status build_items(mg_batch_s* B, int tile, cudaStream_t s);

extern "C" {

mg_status mg_create_batched(mg_batch* out, int count, const int64_t* shapes, const double* spacing, const int bc[4],
                            const uint8_t* const* d_masks, const mg_options* opt, void* stream) {
  if (!out || count <= 0 || !shapes || !spacing || !bc) {
    set_error("mg_create_batched: invalid arguments");
    return MG_ERR_INVALID;
  }
  *out = nullptr;
  mg_options o;
  if (opt) o = *opt;
  else mg_default_options(&o);
  if (o.prec != MG_FP32) {
    set_error("mg_create_batched: only MG_FP32 inner storage");
    return MG_ERR_INVALID;
  }
  int bcD = 0;
  for (int f = 0; f < 4; ++f) {
    if (bc[f] != MG_BC_DIRICHLET && bc[f] != MG_BC_NEUMANN) {
      set_error("mg_create_batched: bad bc[%d]", f);
      return MG_ERR_INVALID;
    }
    if (bc[f] == MG_BC_DIRICHLET) bcD |= 1 << f;
  }
  cudaStream_t s = (cudaStream_t)stream;
  mg_batch_s* B = new mg_batch_s();
  B->count = count;
  B->opt = o;
  B->inner_floor = o.inner_floor > 0 ? o.inner_floor : 1e-4;
  B->timeout_s = 2.0;
  B->withhold = 0;
  cudaGetDevice(&B->device);
  cudaDeviceGetAttribute(&B->nsm, cudaDevAttrMultiProcessorCount, B->device);
  B->inst.resize(count);
  // --- geometry and memory plan
  size_t bytes = 0;
  auto reserve = [&](size_t n) {
    const size_t o2 = (bytes + 255) / 256 * 256;
    bytes = o2 + n;
    return o2;
  };
  struct Off {
    size_t solid[kMaxLevels], cell[kMaxLevels], b[kMaxLevels], x[kMaxLevels], y[kMaxLevels];
    size_t r, z, p0, p1, Ap, d, xf0, xf1, inv;
  };
  std::vector<Off> off(count);
  int max_kc = 0;
  size_t coarse_bytes = 0;
  long long total_cells = 0;
  int max_side = 0;
  for (int i = 0; i < count; ++i) {
    BInst& I = B->inst[i];
    memset(&I, 0, sizeof(I));
    const int nx = (int)shapes[2 * i], ny = (int)shapes[2 * i + 1];
    if (nx % 4 || ny % 4 || (long long)nx * ny <= kBCoarseCells || !(spacing[2 * i] > 0) ||
        !(spacing[2 * i + 1] > 0)) {
      delete B;
      set_error("mg_create_batched: instance %d: sides must be multiples of 4 with more than %d cells", i,
                kBCoarseCells);
      return MG_ERR_INVALID;
    }
    if (!d_masks || !d_masks[i]) {
      if (!bcD) {
        delete B;
        set_error("mg_create_batched: instance %d is singular (all Neumann, no mask)", i);
        return MG_ERR_INVALID;
      }
    }
    I.nx = nx;
    I.ny = ny;
    total_cells += (long long)nx * ny;
    max_side = nx > max_side ? nx : max_side;
    int L = 1;
    while ((nx >> (L - 1)) % 2 == 0 && (ny >> (L - 1)) % 2 == 0 && (nx >> L) >= 4 && (ny >> L) >= 4 && L < kMaxLevels)
      ++L;
    I.L = L;
    int kc = L - 1;
    while (kc > 0 && (size_t)(nx >> (kc - 1)) * (ny >> (kc - 1)) <= (size_t)kBCoarseCells) --kc;
    I.kc = kc;
    max_kc = kc > max_kc ? kc : max_kc;
    const double c = spacing[2 * i] * spacing[2 * i];
    I.c = c;
    I.c2 = c * c;
    const double w[2] = {1.0, c / (spacing[2 * i + 1] * spacing[2 * i + 1])};
    for (int a = 0; a < 2; ++a) {
      I.wff[a].hi = (float)w[a];
      I.wff[a].lo = (float)(w[a] - (double)I.wff[a].hi);
    }
    I.cff.hi = (float)c;
    I.cff.lo = (float)(c - (double)I.cff.hi);
    const bool masked = d_masks && d_masks[i];
    Off& f = off[i];
    for (int k = 0; k < L; ++k) {
      LevelDev& lv = I.lv[k];
      lv.nx = nx >> k;
      lv.ny = ny >> k;
      lv.nz = 1;
      const double hx = spacing[2 * i] * (1 << k), hy = spacing[2 * i + 1] * (1 << k);
      lv.wx = (float)(c / (hx * hx));
      lv.wy = (float)(c / (hy * hy));
      lv.wz = 0.f;
      lv.bcD = bcD;
      const size_t n = (size_t)lv.nx * lv.ny;
      if (masked) {
        f.solid[k] = reserve(n);
        f.cell[k] = reserve(n);
      }
      if (k >= 1 && k <= kc) f.b[k] = reserve(n * 4);
      if (k < kc) f.x[k] = reserve(n * 4);
      if (k >= 1 && k <= kc) f.y[k] = reserve(n * 4);
    }
    const size_t n0 = (size_t)nx * ny;
    f.r = reserve(n0 * 4);
    f.z = reserve(n0 * 4);
    f.p0 = reserve(n0 * 4);
    f.p1 = reserve(n0 * 4);
    f.Ap = reserve(n0 * 4);
    f.d = reserve(n0 * 4);
    f.xf0 = reserve(n0 * 8);
    f.xf1 = reserve(n0 * 8);
    const int nc = (nx >> (L - 1)) * (ny >> (L - 1));
    if (nc > 1024) {
      delete B;
      set_error("mg_create_batched: instance %d coarsest level too large", i);
      return MG_ERR_INVALID;
    }
    f.inv = reserve((size_t)2 * nc * nc * 8);
    // tiles of every level handled as tiles (k < kc), tile 64 x 16 grid as the
    // slot basis (the item lists are rebuilt per tile shape below)
    I.cfloats = 0;
  }
  B->ntile_levels = max_kc;
  // partial slots: worst case over tile shapes = the smallest tile (32 x 16)
  long long max_slots = 0;
  for (int i = 0; i < count; ++i) max_slots += (long long)((B->inst[i].nx + 31) / 32) * ((B->inst[i].ny + 15) / 16);
  const size_t off_partials = reserve((size_t)max_slots * 8);
  const size_t off_bar = reserve(64);
  cudaError_t ce = cudaMalloc((void**)&B->pool, bytes);
  if (ce != cudaSuccess) {
    delete B;
    set_error("mg_create_batched: cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(ce));
    return MG_ERR_OOM;
  }
  B->pool_bytes = bytes;
  mg_status st = MG_OK;
#define NPMG_BTRY(call)                                                                    \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      set_error("mg_create_batched: %s: %s", #call, cudaGetErrorString(e_));               \
      st = MG_ERR_CUDA;                                                                    \
      goto fail;                                                                           \
    }                                                                                      \
  } while (0)
  NPMG_BTRY(cudaMemsetAsync(B->pool, 0, bytes, s));
  B->d_partials = (double*)(B->pool + off_partials);
  B->d_bar = (unsigned*)(B->pool + off_bar);
  for (int i = 0; i < count; ++i) {
    BInst& I = B->inst[i];
    Off& f = off[i];
    char* P = B->pool;
    const bool masked = d_masks && d_masks[i];
    int nf = I.nx * I.ny;
    for (int k = 0; k < I.L; ++k) {
      if (masked) {
        uint8_t* sd = (uint8_t*)(P + f.solid[k]);
        if (k == 0) NPMG_BTRY(cudaMemcpyAsync(sd, d_masks[i], (size_t)I.nx * I.ny, cudaMemcpyDeviceToDevice, s));
        else {
          const int64_t fine[3] = {I.lv[k - 1].nx, I.lv[k - 1].ny, 1};
          NPMG_BTRY(launch_coarsen_solid(2, fine, (uint8_t*)(P + f.solid[k - 1]), sd, s));
        }
        const int64_t n3[3] = {I.lv[k].nx, I.lv[k].ny, 1};
        NPMG_BTRY(launch_cell_bytes(2, n3, I.lv[k].bcD, sd, (uint8_t*)(P + f.cell[k]), s));
        I.lv[k].cell = (uint8_t*)(P + f.cell[k]);
      } else {
        I.lv[k].cell = nullptr;
      }
      if (k >= 1 && k <= I.kc) {
        I.b[k] = (float*)(P + f.b[k]);
        I.y[k] = (float*)(P + f.y[k]);
      }
      if (k < I.kc) I.x[k] = (float*)(P + f.x[k]);
    }
    if (masked) {
      std::vector<uint8_t> hm((size_t)I.nx * I.ny);
      NPMG_BTRY(cudaMemcpyAsync(hm.data(), d_masks[i], hm.size(), cudaMemcpyDeviceToHost, s));
      NPMG_BTRY(cudaStreamSynchronize(s));
      nf = 0;
      for (uint8_t v : hm) nf += v ? 0 : 1;
    }
    I.nfluid = nf;
    I.r = (float*)(P + f.r);
    I.z = (float*)(P + f.z);
    I.p0 = (float*)(P + f.p0);
    I.p1 = (float*)(P + f.p1);
    I.Ap = (float*)(P + f.Ap);
    I.d = (float*)(P + f.d);
    I.xf0 = (float2*)(P + f.xf0);
    I.xf1 = (float2*)(P + f.xf1);
    // coarsest inverse and the block-local coarse item
    {
      const int Lc = I.L - 1;
      const double hx = std::ldexp(1.0, Lc), c = I.c;
      (void)hx;
      const double wc[3] = {(double)I.lv[Lc].wx, (double)I.lv[Lc].wy, 0.0};
      const double wd[3] = {c / (spacing[2 * i] * spacing[2 * i] * std::ldexp(1.0, 2 * Lc)),
                            c / (spacing[2 * i + 1] * spacing[2 * i + 1] * std::ldexp(1.0, 2 * Lc)), 0.0};
      (void)wc;
      const int64_t n3[3] = {I.lv[Lc].nx, I.lv[Lc].ny, 1};
      NPMG_BTRY(launch_coarse_inverse(2, n3, wd, I.lv[Lc].bcD, I.lv[Lc].cell, (double*)(P + f.inv), s));
      CoarseArgs& ca = I.ca;
      memset(&ca, 0, sizeof(ca));
      ca.nlev = I.L - I.kc;
      ca.dim = 2;
      for (int l = 0; l < ca.nlev; ++l) ca.lv[l] = I.lv[I.kc + l];
      const size_t cb = coarse_layout(ca.off, ca.lv, ca.nlev, 2);
      I.cfloats = (int)(cb / 4);
      coarse_bytes = cb > coarse_bytes ? cb : coarse_bytes;
      ca.ncoarse = I.lv[Lc].nx * I.lv[Lc].ny;
      ca.inv = reinterpret_cast<const float*>(P + f.inv);
      ca.image = nullptr;
      ca.pre = o.pre;
      ca.post = o.post;
      ca.omega = (float)o.omega;
      ca.s = (float)o.coarse_scale;
      ca.finest = 0;
    }
  }
  NPMG_BTRY(cudaMalloc((void**)&B->d_inst, sizeof(BInst) * count));
  NPMG_BTRY(cudaMalloc((void**)&B->d_st, sizeof(SolveState) * count));
  NPMG_BTRY(cudaMalloc((void**)&B->d_cur, sizeof(int) * count));
  NPMG_BTRY(cudaMalloc((void**)&B->d_rhs, sizeof(void*) * count));
  NPMG_BTRY(cudaMalloc((void**)&B->d_xout, sizeof(void*) * count));
  NPMG_BTRY(cudaMalloc((void**)&B->d_xin, sizeof(void*) * count));
  NPMG_BTRY(cudaMallocHost((void**)&B->h_st, sizeof(SolveState) * count));
  NPMG_BTRY(cudaMallocHost((void**)&B->h_ptrs, sizeof(void*) * 2 * count));
  NPMG_BTRY(cudaMemsetAsync(B->d_st, 0, sizeof(SolveState) * count, s));
  NPMG_BTRY(cudaEventCreate(&B->ev0));
  NPMG_BTRY(cudaEventCreate(&B->ev1));
  // shared memory, occupancy and grid per (tile, sweeps)
  for (int t = 0; t < kNTiles; ++t)
    for (int sw = 1; sw <= 3; ++sw) {
      B->smem[t][sw] = batched_smem(kTiles[t].tx, kTiles[t].ty, sw, coarse_bytes);
      NPMG_BTRY(cudaFuncSetAttribute(batched_kernel(t), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)B->smem[t][sw] + 1024));
      int per_sm = 0;
      NPMG_BTRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel(t), kBThreads, B->smem[t][sw]));
      if (per_sm < 1) {
        set_error("mg_create_batched: kernel does not fit on an SM");
        st = MG_ERR_INVALID;
        goto fail;
      }
      B->grid[t][sw] = B->nsm * (per_sm > 4 ? 4 : per_sm);
    }
  {
    char name[256] = {0};
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, B->device) == cudaSuccess) snprintf(name, sizeof name, "%s", prop.name);
    for (char* c = name; *c; ++c)
      if (*c == ' ') *c = '_';
    char key[512];
    snprintf(key, sizeof key, "%s|n%d|cells%lld|max%d|p%d", name, count, total_cells, max_side, o.pre);
    B->tune_key = key;
  }
  B->tile = 0;
  B->sweeps = o.pre >= 1 && o.pre <= 3 ? o.pre : 2;
  tune_lookup(B->tune_key, &B->tile, &B->sweeps);
  NPMG_BTRY(cudaStreamSynchronize(s));
#undef NPMG_BTRY
  // work lists of the initial tile shape (a solve itself allocates nothing)
  st = build_items(B, B->tile, s);
  if (st != MG_OK) goto fail;
  *out = B;
  return MG_OK;
fail:
  mg_destroy_batched(B);
  return st;
}

}  // extern "C"

// Item lists of the current tile shape (rebuilt when the tuner switches).
static mg_status build_items(mg_batch_s* B, int tile, cudaStream_t s) {
  const int TX = kTiles[tile].tx, TY = kTiles[tile].ty;
  std::vector<std::vector<int4>> items(kMaxLevels);
  int slot = 0;
  for (int i = 0; i < B->count; ++i) {
    BInst& I = B->inst[i];
    I.slot0 = slot;
    for (int k = 0; k < I.kc; ++k) {
      const int nx = I.lv[k].nx, ny = I.lv[k].ny;
      for (int ty = 0; ty < (ny + TY - 1) / TY; ++ty)
        for (int tx = 0; tx < (nx + TX - 1) / TX; ++tx) items[k].push_back(make_int4(i, tx, ty, k == 0 ? slot++ : -1));
    }
    I.ntiles0 = slot - I.slot0;
  }
  for (int4* p : B->d_items) cudaFree(p);
  B->d_items.assign(kMaxLevels, nullptr);
  for (int k = 0; k < kMaxLevels; ++k) {
    B->nitems[k] = (int)items[k].size();
    if (items[k].empty()) continue;
    NPMG_CUDA(cudaMalloc((void**)&B->d_items[k], items[k].size() * sizeof(int4)));
    NPMG_CUDA(cudaMemcpyAsync(B->d_items[k], items[k].data(), items[k].size() * sizeof(int4), cudaMemcpyHostToDevice,
                              s));
  }
  for (int i = 0; i < B->count; ++i) {
    B->inst[i].ca.pre = B->sweeps;
    B->inst[i].ca.post = B->sweeps;
  }
  NPMG_CUDA(cudaMemcpyAsync(B->d_inst, B->inst.data(), sizeof(BInst) * B->count, cudaMemcpyHostToDevice, s));
  NPMG_CUDA(cudaStreamSynchronize(s));
  return MG_OK;
}

static mg_status set_pointers(mg_batch_s* B, const float* const* d_rhs, float* const* d_x, cudaStream_t s) {
  for (int i = 0; i < B->count; ++i) {
    if (!d_rhs[i] || !d_x[i]) {
      set_error("batched solve: NULL array for instance %d", i);
      return MG_ERR_INVALID;
    }
    B->h_ptrs[i] = (void*)d_rhs[i];
    B->h_ptrs[B->count + i] = (void*)d_x[i];
  }
  NPMG_CUDA(cudaMemcpyAsync((void*)B->d_rhs, B->h_ptrs, sizeof(void*) * B->count, cudaMemcpyHostToDevice, s));
  NPMG_CUDA(
      cudaMemcpyAsync((void*)B->d_xout, B->h_ptrs + B->count, sizeof(void*) * B->count, cudaMemcpyHostToDevice, s));
  NPMG_CUDA(
      cudaMemcpyAsync((void*)B->d_xin, B->h_ptrs + B->count, sizeof(void*) * B->count, cudaMemcpyHostToDevice, s));
  return MG_OK;
}

static mg_status run_batched(mg_batch_s* B, double tol, cudaStream_t s, mg_stats* out, float* ms_out) {
  if (B->d_items.empty()) {
    mg_status st = build_items(B, B->tile, s);
    if (st != MG_OK) return st;
  }
  NPMG_CUDA(cudaEventRecord(B->ev0, s));
  mg_status st = batched_launch(B, B->tile, B->sweeps, tol, s);
  if (st != MG_OK) return st;
  NPMG_CUDA(cudaEventRecord(B->ev1, s));
  NPMG_CUDA(cudaMemcpyAsync(B->h_st, B->d_st, sizeof(SolveState) * B->count, cudaMemcpyDeviceToHost, s));
  unsigned err = 0;
  NPMG_CUDA(cudaMemcpyAsync(&err, B->d_bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  NPMG_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, B->ev0, B->ev1);
  if (ms_out) *ms_out = ms;
  mg_status worst = MG_OK;
  for (int i = 0; i < B->count; ++i) {
    const SolveState& S = B->h_st[i];
    mg_status si = err ? MG_TIMEOUT : (mg_status)S.status;
    if (!err && !S.outer_done && si == MG_OK) si = MG_NOT_CONVERGED;
    if (si != MG_OK && worst == MG_OK) worst = si;
    if (out) {
      memset(&out[i], 0, sizeof(mg_stats));
      out[i].status = si;
      out[i].iters = S.iters_total;
      out[i].outer = S.outer;
      out[i].levels = B->inst[i].L;
      out[i].relres0 = S.relres0;
      out[i].relres = S.relres;
      out[i].bnorm = sqrt(S.bnorm2);
      out[i].ms = ms;
      for (int k = 0; k < 32; ++k) out[i].history[k] = S.hist[k];
    }
  }
  if (err) set_error("batched solve: a grid barrier timed out");
  return err ? MG_TIMEOUT : worst;
}

extern "C" {

mg_status mg_solve_batched(mg_batch B, const float* const* d_rhs, float* const* d_x, double rel_tol, void* stream,
                           mg_stats* out) {
  if (!B || !d_rhs || !d_x || !(rel_tol > 0)) {
    set_error("mg_solve_batched: invalid arguments");
    return MG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  mg_status st = set_pointers(B, d_rhs, d_x, s);
  if (st != MG_OK) return st;
  return run_batched(B, rel_tol, s, out, nullptr);
}

mg_status mg_tune_batched(mg_batch B, const float* const* d_rhs, float* const* d_x, double rel_tol, void* stream,
                          int* out_tile_x, int* out_tile_y, int* out_sweeps) {
  if (!B || !d_rhs || !d_x || !(rel_tol > 0)) {
    set_error("mg_tune_batched: invalid arguments");
    return MG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  mg_status st = set_pointers(B, d_rhs, d_x, s);
  if (st != MG_OK) return st;
  // every candidate solves from the caller's guesses: the init phase reads a
  // copy of them through the guess table while the results go to d_x (the
  // table points back at d_x when the tuner returns)
  struct GuessCopy {
    mg_batch_s* B;
    cudaStream_t s;
    float* buf = nullptr;
    ~GuessCopy() {
      cudaMemcpyAsync((void*)B->d_xin, B->h_ptrs + B->count, sizeof(void*) * B->count, cudaMemcpyHostToDevice, s);
      cudaStreamSynchronize(s);
      if (buf) cudaFree(buf);
    }
  } gc{B, s};
  {
    size_t total = 0;
    for (int i = 0; i < B->count; ++i) total += (size_t)B->inst[i].nx * B->inst[i].ny;
    NPMG_CUDA(cudaMalloc((void**)&gc.buf, total * sizeof(float)));
    std::vector<const float*> gp(B->count);
    size_t off = 0;
    for (int i = 0; i < B->count; ++i) {
      const size_t n = (size_t)B->inst[i].nx * B->inst[i].ny;
      gp[i] = gc.buf + off;
      NPMG_CUDA(cudaMemcpyAsync(gc.buf + off, d_x[i], n * sizeof(float), cudaMemcpyDeviceToDevice, s));
      off += n;
    }
    NPMG_CUDA(cudaMemcpyAsync((void*)B->d_xin, gp.data(), sizeof(void*) * B->count, cudaMemcpyHostToDevice, s));
    NPMG_CUDA(cudaStreamSynchronize(s));
  }
  int best_t = B->tile, best_s = B->sweeps;
  float best = 1e30f;
  for (int t = 0; t < kNTiles; ++t) {
    for (int sw = 1; sw <= 3; ++sw) {
      B->tile = t;
      B->sweeps = sw;
      st = build_items(B, t, s);
      if (st != MG_OK) return st;
      float ms = 0.f;
      st = run_batched(B, rel_tol, s, nullptr, nullptr);  // warm
      if (st != MG_OK && st != MG_NOT_CONVERGED) continue;
      st = run_batched(B, rel_tol, s, nullptr, &ms);
      if (st == MG_OK && ms < best) {
        best = ms;
        best_t = t;
        best_s = sw;
      }
    }
  }
  B->tile = best_t;
  B->sweeps = best_s;
  st = build_items(B, best_t, s);
  if (st != MG_OK) return st;
  tune_store(B->tune_key, best_t, best_s, best);
  if (out_tile_x) *out_tile_x = kTiles[best_t].tx;
  if (out_tile_y) *out_tile_y = kTiles[best_t].ty;
  if (out_sweeps) *out_sweeps = best_s;
  return MG_OK;
}

mg_status mg_batched_config(mg_batch B, int tile_x, int tile_y, int sweeps, double barrier_timeout_s,
                            int withhold_first_arrival) {
  if (!B || sweeps < 1 || sweeps > 3 || !(barrier_timeout_s > 0)) {
    set_error("mg_batched_config: invalid arguments");
    return MG_ERR_INVALID;
  }
  int t = -1;
  for (int k = 0; k < kNTiles; ++k)
    if (kTiles[k].tx == tile_x && kTiles[k].ty == tile_y) t = k;
  if (t < 0) {
    set_error("mg_batched_config: tile must be 64x16, 32x16, 128x8, 64x32 or 128x16");
    return MG_ERR_INVALID;
  }
  const bool rebuild = t != B->tile || sweeps != B->sweeps || B->d_items.empty();
  B->tile = t;
  B->sweeps = sweeps;
  B->timeout_s = barrier_timeout_s;
  B->withhold = withhold_first_arrival ? 1 : 0;
  if (rebuild) return build_items(B, t, nullptr);
  return MG_OK;
}

mg_status mg_destroy_batched(mg_batch B) {
  if (!B) return MG_OK;
  for (int t = 0; t < kNTiles; ++t)
    for (int k = 0; k < 4; ++k)
      if (B->graph[t][k]) cudaGraphExecDestroy(B->graph[t][k]);
  for (int4* p : B->d_items) cudaFree(p);
  if (B->pool) cudaFree(B->pool);
  if (B->d_inst) cudaFree(B->d_inst);
  if (B->d_st) cudaFree(B->d_st);
  if (B->d_cur) cudaFree(B->d_cur);
  if (B->d_rhs) cudaFree((void*)B->d_rhs);
  if (B->d_xout) cudaFree(B->d_xout);
  if (B->d_xin) cudaFree((void*)B->d_xin);
  if (B->h_st) cudaFreeHost(B->h_st);
  if (B->h_ptrs) cudaFreeHost(B->h_ptrs);
  if (B->ev0) cudaEventDestroy(B->ev0);
  if (B->ev1) cudaEventDestroy(B->ev1);
  delete B;
  return MG_OK;
}

}  // extern "C"
