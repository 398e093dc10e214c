// One implicit backward-Euler step of the 2D advection-diffusion equation,
// A T^{n+1} = T^n (Eq. BE-advection-concise; Eq. A-up for upwind advection),
// solved by multigrid as a stationary iteration (Sec. 2.2 cycle, Sec. 3.2
// solver).  A is a constant nonsymmetric 5-point stencil per level with zero
// padding (Sec. 2.1):
//   (A T)_l = c T_l + xm T_{l-1} + xp T_{l+1} + ym T_{m-1} + yp T_{m+1}.
//
// Layout: node arrays [y][x], x fastest.  The iterate is float-float (a
// pair hi + lo of float32 per node, about 48 significant bits: the
// operator's norm is about 1 + 8 nu dt / h^2, so a float32 iterate alone
// leaves a relative residual near 1e-4); the residual is evaluated in
// float-float with error-free products and sums (FP32 arithmetic: GB300's
// FP64 rate is a small fraction of its FP32 rate) and the cycle runs on it
// in float32.
//
// Per cycle: k_ad_resid (V: r = b - A x of the iterate and ||r||, from
// which its last block takes the convergence decision), on levels 0 .. kc-1
// a tile down leg (V: pre sweeps from zero, residual, 2x2 average;
// sawtooth: x = b / c, average of b, on level 0 after forming r and ||r||
// itself), one single-block kernel
// for levels kc .. L-1 (<= 4096 nodes; coarsest level by a dense inverse
// in the V cycle), tile up legs back to level 0 (x + s P e, post sweeps);
// the level-0 up leg adds the correction to the float-float iterate and sums
// its L1 norm (the paper's stopping gauge).  Every kernel returns at once
// after the state's done flag is set, so a CUDA graph of kChunk cycles is
// replayed until the host sees the flag.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "launch.h"
#include "npmg_internal.cuh"

namespace npmg {
namespace ad {

constexpr int TX = 64, TY = 16;  // tile of the level-leg kernels
constexpr int kT = 256;          // threads per tile block
constexpr int kCB = 1024;        // threads of the coarse block
constexpr int kCoarseCells = 4096;
constexpr int kCoarsestMax = 256;
constexpr int kChunk = 8;        // cycles per graph launch

struct Lev {
  int nx, ny;
  float c, xm, xp, ym, yp, inv_c;
};

struct State {
  double tol, l1_tol;
  int max_cycles;
  double bnorm2, relres, relres0, l1, l1_first;
  int cycles, done, status;
  unsigned int counter[2];
};

// Sum of v over the block, in a fixed shuffle-tree order; the result is
// valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();  // ws may still be read by a previous call
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += ws[w];
  return s;
}

// Grid sum of v: each block writes its sum to partials[bid]; the last block
// to finish adds the nblocks partials with all its threads (a fixed strided
// assignment, then block_sum: deterministic) and gets the total in thread
// 0, which alone returns true.  The counter is reset for the next use.
__device__ bool grid_sum(double v, double* partials, unsigned int* counter, unsigned int nblocks, unsigned int bid,
                         double* total) {
  __shared__ bool is_last;
  const double bs = block_sum(v);
  if (threadIdx.x == 0) {
    partials[bid] = bs;
    __threadfence();
    is_last = atomicAdd(counter, 1u) == nblocks - 1;
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double s = 0.0;
  for (unsigned int k = threadIdx.x; k < nblocks; k += blockDim.x) s += ((volatile double*)partials)[k];
  s = block_sum(s);
  if (threadIdx.x != 0) return false;
  *total = s;
  *counter = 0;
  return true;
}

// Error-free transformations (Knuth's two-sum, the FMA two-product): a + b
// = s + e and a * b = p + e exactly in float32.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

// Nodes are visited row by row: blocks stride over rows, threads over x
// (no 64-bit index division).
#define AD_FOR_NODES(L)                                                 \
  for (int iy = blockIdx.x; iy < (L).ny; iy += gridDim.x)               \
    for (int ix = threadIdx.x; ix < (L).nx; ix += blockDim.x)

// x = x0 (or b) as (hi, lo = 0), ||b||^2, state reset.
__global__ void __launch_bounds__(kT) k_ad_init(Lev L, const float* __restrict__ b, const float* __restrict__ x0,
                                                float2* __restrict__ x, State* st, double tol, double l1_tol,
                                                int max_cycles, double* partials) {
  float acc = 0.f;
  AD_FOR_NODES(L) {
    const size_t i = (size_t)iy * L.nx + ix;
    const float bv = b[i];
    x[i] = make_float2(x0 ? x0[i] : bv, 0.f);
    acc = fmaf(bv, bv, acc);
  }
  double tot;
  if (grid_sum(acc, partials, &st->counter[0], gridDim.x, blockIdx.x, &tot)) {
    st->tol = tol;
    st->l1_tol = l1_tol;
    st->max_cycles = max_cycles;
    st->bnorm2 = tot;
    st->relres = st->relres0 = 1.0;
    st->l1 = st->l1_first = 0.0;
    st->cycles = 0;
    st->done = 0;
    st->status = MG_OK;
    st->counter[1] = 0;
  }
}

// relres from ||b - A x||^2 and, unless `final`, the stopping decision taken
// before each cycle: converged, diverged (1000-fold growth) or out of cycles.
__device__ void decide(State* st, double rr, bool final) {
  const double rel = st->bnorm2 > 0.0 ? sqrt(rr / st->bnorm2) : 0.0;
  st->relres = rel;
  if (final) return;
  if (st->cycles == 0) st->relres0 = rel;
  if (rel <= st->tol) {
    st->status = MG_OK;
    st->done = 1;
  } else if (!isfinite(rel) || rel > 1e3 * fmax(st->relres0, 1.0)) {
    st->status = MG_DIVERGED;
    st->done = 1;
  } else if (st->cycles >= st->max_cycles) {
    st->status = MG_NOT_CONVERGED;
    st->done = 1;
  }
}

// One term -w * (hi + lo) of b - A x into the float-float sum (S, E).
__device__ __forceinline__ void ff_sub_term(float w, float2 x, float& S, float& E) {
  float p, pe, se;
  two_prod(-w, x.x, p, pe);
  two_sum(S, p, S, se);
  E += se + pe;
  E = fmaf(-w, x.y, E);
}

// r = b - A x in float-float (rounded to float32 for the cycle), relres and
// the stopping decision.  `final` computes the relres of the returned
// iterate whatever the flag says and decides nothing.
__global__ void __launch_bounds__(kT) k_ad_resid(Lev L, const float* __restrict__ b, const float2* __restrict__ x,
                                                 float* __restrict__ r, State* st, double* partials, int final) {
  chain_enter();
  if (!final && st->done) return;
  float acc = 0.f;
  AD_FOR_NODES(L) {
    const size_t i = (size_t)iy * L.nx + ix;
    float S = b[i], E = 0.f;
    ff_sub_term(L.c, x[i], S, E);
    if (ix > 0) ff_sub_term(L.xm, x[i - 1], S, E);
    if (ix + 1 < L.nx) ff_sub_term(L.xp, x[i + 1], S, E);
    if (iy > 0) ff_sub_term(L.ym, x[i - L.nx], S, E);
    if (iy + 1 < L.ny) ff_sub_term(L.yp, x[i + L.nx], S, E);
    const float rv = S + E;
    if (!final) r[i] = rv;
    acc = fmaf(rv, rv, acc);
  }
  double tot;
  if (grid_sum(acc, partials, &st->counter[0], gridDim.x, blockIdx.x, &tot)) decide(st, tot, final != 0);
}

// One relaxed Jacobi sweep over window J, [J, RX - J) x [J, RY - J), of a
// shared-memory region RX x RY whose node (0, 0) is node (ox, oy) of the
// level.  The window shrinks by one per sweep, so nothing outside it is
// read again; nodes outside the level are skipped and keep the 0 both
// buffers were loaded with (zero padding).  `interior`: the region lies
// inside the level (block-uniform), no per-node test.
template <int RX, int RY, int J>
__device__ __forceinline__ void region_sweep(const Lev& L, const float* cur, float* nxt, const float* sb, int ox,
                                             int oy, bool interior, float omega) {
  constexpr int WX = RX - 2 * J, WN = WX * (RY - 2 * J);
  for (int k = threadIdx.x; k < WN; k += kT) {
    const int lx = J + k % WX, ly = J + k / WX;
    if (!interior) {
      const int gx = ox + lx, gy = oy + ly;
      if (gx < 0 || gx >= L.nx || gy < 0 || gy >= L.ny) continue;
    }
    const int i = ly * RX + lx;
    const float a = L.c * cur[i] + L.xm * cur[i - 1] + L.xp * cur[i + 1] + L.ym * cur[i - RX] + L.yp * cur[i + RX];
    nxt[i] = cur[i] + omega * (sb[i] - a) * L.inv_c;
  }
}

// Sweeps 1 .. S (S <= 2) over the shrinking windows; returns the buffer
// that holds the last one.
template <int RX, int RY, int S>
__device__ __forceinline__ float* region_sweeps(const Lev& L, float* cur, float* nxt, const float* sb, int ox,
                                                int oy, float omega) {
  static_assert(S >= 0 && S <= 2, "at most two sweeps");
  const bool interior = ox >= 0 && oy >= 0 && ox + RX <= L.nx && oy + RY <= L.ny;
  if constexpr (S >= 1) {
    region_sweep<RX, RY, 1>(L, cur, nxt, sb, ox, oy, interior, omega);
    __syncthreads();
    float* t = cur;
    cur = nxt;
    nxt = t;
  }
  if constexpr (S >= 2) {
    region_sweep<RX, RY, 2>(L, cur, nxt, sb, ox, oy, interior, omega);
    __syncthreads();
    cur = nxt;
  }
  return cur;
}

// V down leg of one level: PRE relaxed Jacobi sweeps from zero on the tile
// grown by PRE + 1 (temporal blocking), x written on the tile, the residual
// of its 2x2 blocks averaged into the coarse right-hand side.
template <int PRE>
__global__ void __launch_bounds__(kT) k_ad_down(Lev L, const float* __restrict__ b, float* __restrict__ x,
                                                float* __restrict__ bc, float omega, const State* st) {
  chain_enter();
  if (st->done) return;
  constexpr int R = PRE + 1, RX = TX + 2 * R, RY = TY + 2 * R, RN = RX * RY;
  __shared__ float sb[RN], sa[RN], sc[RN];
  const int ox = blockIdx.x * TX - R, oy = blockIdx.y * TY - R;
  for (int i = threadIdx.x; i < RN; i += kT) {
    const int gx = ox + i % RX, gy = oy + i / RX;
    const bool in = gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny;
    sb[i] = in ? b[(size_t)gy * L.nx + gx] : 0.f;
    sa[i] = 0.f;
    sc[i] = 0.f;
  }
  __syncthreads();
  const float* cur = region_sweeps<RX, RY, PRE>(L, sa, sc, sb, ox, oy, omega);
  // one coarse node per thread (the tile holds TX/2 x TY/2 = kT of them)
  {
    const int cx = threadIdx.x % (TX / 2), cy = threadIdx.x / (TX / 2);
    const int gcx = blockIdx.x * (TX / 2) + cx, gcy = blockIdx.y * (TY / 2) + cy;
    if (gcx < L.nx / 2 && gcy < L.ny / 2) {
      float sum = 0.f;
#pragma unroll
      for (int ay = 0; ay < 2; ++ay)
#pragma unroll
        for (int ax = 0; ax < 2; ++ax) {
          const int li = (R + 2 * cy + ay) * RX + R + 2 * cx + ax;
          const float a =
              L.c * cur[li] + L.xm * cur[li - 1] + L.xp * cur[li + 1] + L.ym * cur[li - RX] + L.yp * cur[li + RX];
          sum += sb[li] - a;
        }
      bc[(size_t)gcy * (L.nx / 2) + gcx] = 0.25f * sum;
    }
  }
  for (int i = threadIdx.x; i < TX * TY; i += kT) {
    const int tx = i % TX, ty = i / TX;
    const int gx = blockIdx.x * TX + tx, gy = blockIdx.y * TY + ty;
    if (gx < L.nx && gy < L.ny) x[(size_t)gy * L.nx + gx] = cur[(R + ty) * RX + R + tx];
  }
}

// Sawtooth down leg: x = b / c on every node, the 2x2 average of b to the
// coarse right-hand side (no sweeps); one thread per coarse node.  On level
// 0 (FUSED) b is the residual of the float-float iterate, computed here,
// written to r and summed for the stopping decision, which the last block
// takes (the V cycle gets it from k_ad_resid).
template <bool FUSED>
__global__ void __launch_bounds__(kT) k_ad_down_saw(Lev L, const float* __restrict__ b, float* __restrict__ x,
                                                    float* __restrict__ bc, State* st,
                                                    const float2* __restrict__ xff, float* __restrict__ r,
                                                    double* partials) {
  chain_enter();
  if (st->done) return;
  const int cnx = L.nx / 2;
  const size_t nc = (size_t)cnx * (L.ny / 2);
  float acc = 0.f;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (size_t)gridDim.x * blockDim.x) {
    const int cx = (int)(c % cnx), cy = (int)(c / cnx);
    float v[4];
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int ix = 2 * cx + (k & 1), iy = 2 * cy + (k >> 1);
      const size_t i = (size_t)iy * L.nx + ix;
      float bv = b[i];
      if (FUSED) {
        float S = bv, E = 0.f;
        ff_sub_term(L.c, xff[i], S, E);
        if (ix > 0) ff_sub_term(L.xm, xff[i - 1], S, E);
        if (ix + 1 < L.nx) ff_sub_term(L.xp, xff[i + 1], S, E);
        if (iy > 0) ff_sub_term(L.ym, xff[i - L.nx], S, E);
        if (iy + 1 < L.ny) ff_sub_term(L.yp, xff[i + L.nx], S, E);
        bv = S + E;
        r[i] = bv;
        acc = fmaf(bv, bv, acc);
      }
      v[k] = bv;
      x[i] = bv * L.inv_c;
    }
    sum = (v[0] + v[1]) + (v[2] + v[3]);
    bc[c] = 0.25f * sum;
  }
  if (FUSED) {
    double tot;
    if (grid_sum(acc, partials, &st->counter[0], gridDim.x, blockIdx.x, &tot)) decide(st, tot, false);
  }
}

// Up leg of one level: x + s P e (copy of the coarse value to the 2x2
// children), then POST relaxed Jacobi sweeps on A x = b, over the tile
// grown by POST.  Written to y; on level 0 (FINEST) added to the float-float
// iterate instead, with the L1 norm of the correction summed and the
// cycle's bookkeeping done by the last block.
template <int POST, bool FINEST>
__global__ void __launch_bounds__(kT) k_ad_up(Lev L, const float* __restrict__ b, const float* __restrict__ x,
                                              const float* __restrict__ e, float* __restrict__ y,
                                              float2* __restrict__ xff, float s, float omega, State* st,
                                              double* partials) {
  chain_enter();
  if (st->done) return;
  constexpr int R = POST, RX = TX + 2 * R, RY = TY + 2 * R, RN = RX * RY;
  __shared__ float sb[RN], sa[RN], sc[RN];
  const int ox = blockIdx.x * TX - R, oy = blockIdx.y * TY - R;
  const int cnx = L.nx / 2;
  for (int i = threadIdx.x; i < RN; i += kT) {
    const int gx = ox + i % RX, gy = oy + i / RX;
    float bv = 0.f, xv = 0.f;
    if (gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny) {
      const size_t gi = (size_t)gy * L.nx + gx;
      bv = b[gi];
      xv = fmaf(s, e[(size_t)(gy >> 1) * cnx + (gx >> 1)], x[gi]);
    }
    sb[i] = bv;
    sa[i] = xv;
    sc[i] = 0.f;
  }
  __syncthreads();
  const float* cur = region_sweeps<RX, RY, POST>(L, sa, sc, sb, ox, oy, omega);
  float acc = 0.f;
  for (int i = threadIdx.x; i < TX * TY; i += kT) {
    const int tx = i % TX, ty = i / TX;
    const int gx = blockIdx.x * TX + tx, gy = blockIdx.y * TY + ty;
    if (gx < L.nx && gy < L.ny) {
      const size_t gi = (size_t)gy * L.nx + gx;
      const float v = cur[(R + ty) * RX + R + tx];
      if (FINEST) {
        // x += v in float-float, renormalised
        const float2 xo = xff[gi];
        float hs, he;
        two_sum(xo.x, v, hs, he);
        he += xo.y;
        const float hi = hs + he;
        xff[gi] = make_float2(hi, he - (hi - hs));
        acc += fabsf(v);
      } else {
        y[gi] = v;
      }
    }
  }
  if (FINEST) {
    double t;
    if (grid_sum(acc, partials, &st->counter[1], gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x, &t)) {
      st->cycles += 1;
      st->l1 = t;
      if (st->cycles == 1) st->l1_first = t;
      if (t <= st->l1_tol) {
        st->status = MG_OK;
        st->done = 1;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Single-block kernel for levels kc .. L-1 (each <= kCoarseCells nodes, all
// of them held in dynamic shared memory, at most 96 KB: b, and x and a
// sweep buffer with a zero ring per level); the
// right-hand side of level kc comes from global memory and its correction
// goes back there.
constexpr int kCoarseSmemMax = 24576;  // floats (96 KB) of the single block

struct AdCoarseArgs {
  int first, last;  // level range kc .. L-1
  int cycle, pre, post;
  float omega, s;
  Lev lv[kMaxLevels];
  int off[kMaxLevels];  // shared-memory offset of level k: b (nx ny), then
                        // x and t, each (nx + 2)(ny + 2) with a zero ring
  int lnx[kMaxLevels];  // log2(nx) when nx is a power of two, else -1
  int words;            // floats of shared memory in use
  const float* b_first;
  float* y_first;
  const float* inv;  // dense inverse of the coarsest level (V cycle)
};

__device__ __forceinline__ void node_xy(int i, int nx, int lnx, int& ix, int& iy) {
  if (lnx >= 0) {
    ix = i & (nx - 1);
    iy = i >> lnx;
  } else {
    ix = i % nx;
    iy = i / nx;
  }
}

// A x at padded index p (row width W): the zero ring is the zero padding.
__device__ __forceinline__ float apply_pad(const Lev& L, const float* x, int p, int W) {
  return L.c * x[p] + L.xm * x[p - 1] + L.xp * x[p + 1] + L.ym * x[p - W] + L.yp * x[p + W];
}

__device__ void cb_sweeps(const Lev& L, int lnx, const float* b, float*& cur, float*& oth, int sweeps, float omega) {
  const int n = L.nx * L.ny, W = L.nx + 2;
  for (int j = 0; j < sweeps; ++j) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      int ix, iy;
      node_xy(i, L.nx, lnx, ix, iy);
      const int p = (iy + 1) * W + ix + 1;
      oth[p] = cur[p] + omega * (b[i] - apply_pad(L, cur, p, W)) * L.inv_c;
    }
    __syncthreads();
    float* t = cur;
    cur = oth;
    oth = t;
  }
}

__global__ void __launch_bounds__(kCB) k_ad_coarse(AdCoarseArgs a, const State* st) {
  chain_enter();
  if (st->done) return;
  extern __shared__ float sm[];
  float* res[kMaxLevels];
  const bool saw = a.cycle == MG_CYCLE_SAWTOOTH;
  auto B = [&](int k) { return sm + a.off[k]; };
  auto X = [&](int k) { return sm + a.off[k] + a.lv[k].nx * a.lv[k].ny; };
  auto T = [&](int k) { return sm + a.off[k] + a.lv[k].nx * a.lv[k].ny + (a.lv[k].nx + 2) * (a.lv[k].ny + 2); };
  // zero rings, and every iterate starts from zero
  for (int i = threadIdx.x; i < a.words; i += blockDim.x) sm[i] = 0.f;
  __syncthreads();
  {
    const int n = a.lv[a.first].nx * a.lv[a.first].ny;
    for (int i = threadIdx.x; i < n; i += blockDim.x) B(a.first)[i] = a.b_first[i];
    __syncthreads();
  }
  // down: V smooths from zero and restricts the residual; the sawtooth
  // restricts the right-hand side
  for (int k = a.first; k < a.last; ++k) {
    const Lev& L = a.lv[k];
    const Lev& C = a.lv[k + 1];
    const int W = L.nx + 2;
    float* cur = X(k);
    float* oth = T(k);
    const float* b = B(k);
    if (!saw) cb_sweeps(L, a.lnx[k], b, cur, oth, a.pre, a.omega);
    float* bc = B(k + 1);
    for (int c = threadIdx.x; c < C.nx * C.ny; c += blockDim.x) {
      int cx, cy;
      node_xy(c, C.nx, a.lnx[k + 1], cx, cy);
      float sum = 0.f;
      for (int ay = 0; ay < 2; ++ay)
        for (int ax = 0; ax < 2; ++ax) {
          const int ix = 2 * cx + ax, iy = 2 * cy + ay, i = iy * L.nx + ix;
          sum += saw ? b[i] : b[i] - apply_pad(L, cur, (iy + 1) * W + ix + 1, W);
        }
      bc[c] = 0.25f * sum;
    }
    res[k] = cur;
    __syncthreads();
  }
  // coarsest level: dense inverse (V) or r / c and the post sweeps (sawtooth)
  {
    const int k = a.last;
    const Lev& L = a.lv[k];
    const int n = L.nx * L.ny, W = L.nx + 2;
    float* cur = X(k);
    float* oth = T(k);
    const float* b = B(k);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      int ix, iy;
      node_xy(i, L.nx, a.lnx[k], ix, iy);
      float v;
      if (saw) {
        v = b[i] * L.inv_c;
      } else {
        v = 0.f;
        for (int j = 0; j < n; ++j) v = fmaf(a.inv[(size_t)i * n + j], b[j], v);
      }
      cur[(iy + 1) * W + ix + 1] = v;
    }
    __syncthreads();
    if (saw) cb_sweeps(L, a.lnx[k], b, cur, oth, a.post, a.omega);
    res[k] = cur;
  }
  // up: x + s P e (x = the smoothed iterate, or r / c for the sawtooth), post
  // sweeps
  for (int k = a.last - 1; k >= a.first; --k) {
    const Lev& L = a.lv[k];
    const Lev& C = a.lv[k + 1];
    const int W = L.nx + 2, WC = C.nx + 2;
    float* cur = res[k];
    float* oth = cur == X(k) ? T(k) : X(k);
    const float* b = B(k);
    const int n = L.nx * L.ny;
    const float* e = res[k + 1];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      int ix, iy;
      node_xy(i, L.nx, a.lnx[k], ix, iy);
      const int p = (iy + 1) * W + ix + 1;
      const float base = saw ? b[i] * L.inv_c : cur[p];
      cur[p] = fmaf(a.s, e[((iy >> 1) + 1) * WC + (ix >> 1) + 1], base);
    }
    __syncthreads();
    cb_sweeps(L, a.lnx[k], b, cur, oth, a.post, a.omega);
    res[k] = cur;
  }
  {
    const Lev& L = a.lv[a.first];
    const int n = L.nx * L.ny, W = L.nx + 2;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      int ix, iy;
      node_xy(i, L.nx, a.lnx[a.first], ix, iy);
      a.y_first[i] = res[a.first][(iy + 1) * W + ix + 1];
    }
  }
}

// x (float32 output) = the float-float iterate rounded once.
__global__ void __launch_bounds__(kT) k_ad_out(size_t n, const float2* __restrict__ xff, float* __restrict__ x) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float2 v = xff[i];
    x[i] = v.x + v.y;
  }
}

}  // namespace ad
}  // namespace npmg

using namespace npmg;
using namespace npmg::ad;

struct ad_handle_s {
  int nx, ny, L, kc, nsm;
  ad_options opt;
  Lev lv[kMaxLevels];
  char* pool;
  float* b;        // copy of the caller's right-hand side (the graph's input)
  float* r;        // level-0 residual = the cycle's level-0 right-hand side
  float2* xff;     // the iterate (hi, lo)
  float* bk[kMaxLevels];
  float* xk[kMaxLevels];
  float* yk[kMaxLevels];
  float* inv;
  double* partials;
  State* st;
  State* st_host;
  cudaGraphExec_t graph;
  int64_t chunk_kernels;
  int64_t launches;
};

// Stencil of A at spacing h; diff_scale multiplies the diffusion term (1 =
// the re-discretised filter, 2^k = the Galerkin product on level k).
static Lev make_level(int nx, int ny, double h, double dt, double nu, double u, double v, int scheme,
                      double diff_scale) {
  const double kd = diff_scale * nu * dt / (h * h);
  double c = 1.0 + 4.0 * kd, xm = -kd, xp = -kd, ym = -kd, yp = -kd;
  if (scheme == AD_CENTRAL) {
    const double ax = u * dt / (2.0 * h), ay = v * dt / (2.0 * h);
    xm -= ax;
    xp += ax;
    ym -= ay;
    yp += ay;
  } else {
    // first-order upwind: backward difference for a positive velocity
    const double cx = u * dt / h, cy = v * dt / h;
    if (u >= 0) {
      c += cx;
      xm -= cx;
    } else {
      c -= cx;
      xp += cx;
    }
    if (v >= 0) {
      c += cy;
      ym -= cy;
    } else {
      c -= cy;
      yp += cy;
    }
  }
  Lev L;
  L.nx = nx;
  L.ny = ny;
  L.c = (float)c;
  L.xm = (float)xm;
  L.xp = (float)xp;
  L.ym = (float)ym;
  L.yp = (float)yp;
  L.inv_c = (float)(1.0 / c);
  return L;
}

// Dense inverse of a level's matrix by Gauss-Jordan elimination with
// partial pivoting in float64.  Returns false when the matrix is singular.
static bool dense_inverse(const Lev& L, const double* w, std::vector<float>& out) {
  const int n = L.nx * L.ny;
  std::vector<double> M((size_t)n * 2 * n, 0.0);
  auto at = [&](int r, int c) -> double& { return M[(size_t)r * 2 * n + c]; };
  for (int iy = 0; iy < L.ny; ++iy)
    for (int ix = 0; ix < L.nx; ++ix) {
      const int r = iy * L.nx + ix;
      at(r, r) = w[0];
      if (ix > 0) at(r, r - 1) += w[1];
      if (ix + 1 < L.nx) at(r, r + 1) += w[2];
      if (iy > 0) at(r, r - L.nx) += w[3];
      if (iy + 1 < L.ny) at(r, r + L.nx) += w[4];
      at(r, n + r) = 1.0;
    }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(at(r, col)) > fabs(at(piv, col))) piv = r;
    if (!(fabs(at(piv, col)) > 0.0)) return false;
    if (piv != col)
      for (int c = 0; c < 2 * n; ++c) std::swap(at(piv, c), at(col, c));
    const double d = 1.0 / at(col, col);
    for (int c = 0; c < 2 * n; ++c) at(col, c) *= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = at(r, col);
      if (f == 0.0) continue;
      for (int c = 0; c < 2 * n; ++c) at(r, c) -= f * at(col, c);
    }
  }
  out.resize((size_t)n * n);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) out[(size_t)r * n + c] = (float)at(r, n + c);
  return true;
}

static int grid_1d(const ad_handle_s* h, size_t n) {
  size_t b = (n + kT - 1) / kT;
  const size_t cap = (size_t)h->nsm * 8;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// Row-strided kernels: one block per row up to 8 blocks per SM.
static int row_grid(const ad_handle_s* h) { return std::min(h->ny, h->nsm * 8); }

static dim3 tile_grid(const Lev& L) { return dim3((L.nx + TX - 1) / TX, (L.ny + TY - 1) / TY); }

// One cycle: residual, down legs, the coarse block, up legs.
static cudaError_t enqueue_cycle(ad_handle_s* h, cudaStream_t s) {
  const ad_options& o = h->opt;
  const float om = (float)o.omega, sc = (float)o.coarse_scale;
  const bool saw = o.cycle == MG_CYCLE_SAWTOOTH;
  // level 0: the residual of the iterate comes from k_ad_resid for the V
  // cycle (fusing it into the down leg, which recomputes it on the tile's
  // halo, measured slower on GB300: 4096^2 5.55 -> 6.53 ms) and is formed
  // inside the sawtooth's down leg, which has no halo
  cudaError_t e = cudaSuccess;
  if (!saw) {
    e = launch_chain(k_ad_resid, dim3(row_grid(h)), dim3(kT), 0, s, h->lv[0], (const float*)h->b,
                     (const float2*)h->xff, h->r, h->st, h->partials, 0);
    h->launches += 1;
  }
  for (int k = 0; k < h->kc && e == cudaSuccess; ++k) {
    const float* bk = k == 0 ? (saw ? h->b : h->r) : h->bk[k];
    const Lev& L = h->lv[k];
    const float2* xf = h->xff;
    float* rr = h->r;
    double* pt = h->partials;
    if (saw) {
      const size_t nc = (size_t)(L.nx / 2) * (L.ny / 2);
      e = k == 0 ? launch_chain(k_ad_down_saw<true>, dim3(grid_1d(h, nc)), dim3(kT), 0, s, L, bk, h->xk[k],
                                h->bk[k + 1], h->st, xf, rr, pt)
                 : launch_chain(k_ad_down_saw<false>, dim3(grid_1d(h, nc)), dim3(kT), 0, s, L, bk, h->xk[k],
                                h->bk[k + 1], h->st, xf, rr, pt);
    } else {
#define NPMG_AD_DOWN(P) \
  launch_chain(k_ad_down<P>, tile_grid(L), dim3(kT), 0, s, L, bk, h->xk[k], h->bk[k + 1], om, (const State*)h->st)
      e = o.pre == 0 ? NPMG_AD_DOWN(0) : (o.pre == 1 ? NPMG_AD_DOWN(1) : NPMG_AD_DOWN(2));
#undef NPMG_AD_DOWN
    }
    h->launches += 1;
  }
  if (e != cudaSuccess) return e;
  AdCoarseArgs ca;
  memset(&ca, 0, sizeof(ca));
  ca.first = h->kc;
  ca.last = h->L - 1;
  ca.cycle = o.cycle;
  ca.pre = o.pre;
  ca.post = o.post;
  ca.omega = om;
  ca.s = sc;
  int off = 0;
  for (int k = 0; k < h->L; ++k) {
    ca.lv[k] = h->lv[k];
    const int nx = h->lv[k].nx, ny = h->lv[k].ny;
    ca.lnx[k] = (nx & (nx - 1)) ? -1 : __builtin_ctz((unsigned)nx);
    if (k >= h->kc) {
      ca.off[k] = off;
      off += nx * ny + 2 * (nx + 2) * (ny + 2);
    }
  }
  ca.words = off;
  ca.b_first = h->bk[h->kc];
  ca.y_first = h->yk[h->kc];
  const size_t cb_smem = (size_t)off * sizeof(float);
  ca.inv = h->inv;
  e = launch_chain(k_ad_coarse, dim3(1), dim3(kCB), cb_smem, s, ca, (const State*)h->st);
  h->launches += 1;
  for (int k = h->kc - 1; k >= 0 && e == cudaSuccess; --k) {
    const float* bk = k == 0 ? h->r : h->bk[k];
    const Lev& L = h->lv[k];
    const dim3 g = tile_grid(L);
#define NPMG_AD_UP(P, F)                                                                                      \
  launch_chain(k_ad_up<P, F>, g, dim3(kT), 0, s, L, bk, (const float*)h->xk[k], (const float*)h->yk[k + 1], \
               h->yk[k], h->xff, sc, om, h->st, h->partials)
    if (k == 0)
      e = o.post == 0 ? NPMG_AD_UP(0, true) : (o.post == 1 ? NPMG_AD_UP(1, true) : NPMG_AD_UP(2, true));
    else
      e = o.post == 0 ? NPMG_AD_UP(0, false) : (o.post == 1 ? NPMG_AD_UP(1, false) : NPMG_AD_UP(2, false));
#undef NPMG_AD_UP
    h->launches += 1;
  }
  return e;
}

static cudaError_t ensure_graph(ad_handle_s* h) {
  if (h->graph) return cudaSuccess;
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaGraph_t g = nullptr;
  const int64_t before = h->launches;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e2 = cudaSuccess;
    for (int c = 0; c < kChunk && e2 == cudaSuccess; ++c) e2 = enqueue_cycle(h, cs);
    e = cudaStreamEndCapture(cs, &g);
    if (e2 != cudaSuccess) e = e2;
  }
  h->chunk_kernels = h->launches - before;
  h->launches = before;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  return e;
}

extern "C" {

mg_status ad_default_options(ad_options* o) {
  if (!o) {
    set_error("ad_default_options: NULL");
    return MG_ERR_INVALID;
  }
  o->cycle = MG_CYCLE_V;
  o->pre = 2;
  o->post = 2;
  o->omega = 2.0 / 3.0;
  o->coarse_scale = 1.0;
  o->coarse_op = AD_COARSE_REDISCRETISE;
  o->levels = 0;
  o->max_cycles = 1000;
  return MG_OK;
}

mg_status ad_create(ad_handle* out, const int64_t cells[2], double h, double dt, double nu, double u, double v,
                    int scheme, const ad_options* opt, void* stream) {
  if (!out || !cells) {
    set_error("ad_create: NULL argument");
    return MG_ERR_INVALID;
  }
  *out = nullptr;
  ad_options o;
  if (opt) {
    o = *opt;
  } else {
    ad_default_options(&o);
  }
  const int64_t nx = cells[0], ny = cells[1];
  if (!(h > 0) || !(dt > 0) || !(nu >= 0) || !std::isfinite(u) || !std::isfinite(v) ||
      (scheme != AD_UPWIND && scheme != AD_CENTRAL) || nx < 8 || ny < 8 || nx > (1 << 16) || ny > (1 << 16)) {
    set_error("ad_create: invalid grid or coefficients (h, dt > 0, nu >= 0, 8 <= sides <= 65536, scheme)");
    return MG_ERR_INVALID;
  }
  if ((o.cycle != MG_CYCLE_V && o.cycle != MG_CYCLE_SAWTOOTH) || o.pre < 0 || o.pre > 2 || o.post < 0 ||
      o.post > 2 || !(o.omega > 0 && o.omega <= 2) || !(o.coarse_scale > 0) || o.max_cycles < 1 ||
      (o.coarse_op != AD_COARSE_REDISCRETISE && o.coarse_op != AD_COARSE_GALERKIN) || o.levels < 0 ||
      o.levels > kMaxLevels) {
    set_error("ad_create: invalid options (cycle, pre/post in 0..2, omega in (0,2], coarse_scale > 0, "
              "max_cycles >= 1, coarse_op, levels)");
    return MG_ERR_INVALID;
  }
  int L = o.levels;
  if (L == 0) {
    L = 1;
    int64_t sx = nx, sy = ny;
    while (L < kMaxLevels && sx % 2 == 0 && sy % 2 == 0 && sx / 2 >= 4 && sy / 2 >= 4) {
      sx /= 2;
      sy /= 2;
      ++L;
    }
  }
  if (L < 2 || nx % (1LL << (L - 1)) || ny % (1LL << (L - 1))) {
    set_error("ad_create: need >= 2 levels with sides divisible by 2^(levels-1)");
    return MG_ERR_INVALID;
  }
  const int64_t cnx = nx >> (L - 1), cny = ny >> (L - 1);
  if (o.cycle == MG_CYCLE_V && cnx * cny > kCoarsestMax) {
    set_error("ad_create: coarsest level has %lld nodes (> %d); use more levels", (long long)(cnx * cny),
              kCoarsestMax);
    return MG_ERR_INVALID;
  }
  ad_handle_s* hd = new (std::nothrow) ad_handle_s();
  if (!hd) return MG_ERR_OOM;
  hd->nx = (int)nx;
  hd->ny = (int)ny;
  hd->L = L;
  hd->opt = o;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&hd->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (hd->nsm < 1) hd->nsm = 1;
  for (int k = 0; k < L; ++k) {
    const double scale = o.coarse_op == AD_COARSE_GALERKIN ? (double)(1 << k) : 1.0;
    hd->lv[k] = make_level((int)(nx >> k), (int)(ny >> k), h * (1 << k), dt, nu, u, v, scheme, scale);
  }
  // the single block takes every level from the first one of <= 4096 nodes
  // (never the finest, whose up leg updates the iterate)
  hd->kc = L - 1;
  for (int k = 1; k < L; ++k)
    if ((int64_t)hd->lv[k].nx * hd->lv[k].ny <= kCoarseCells) {
      hd->kc = k;
      break;
    }
  if ((int64_t)hd->lv[hd->kc].nx * hd->lv[hd->kc].ny > kCoarseCells) {
    set_error("ad_create: no level of <= %d nodes; use more levels", kCoarseCells);
    delete hd;
    return MG_ERR_INVALID;
  }
  {
    int64_t words = 0;
    for (int k = hd->kc; k < L; ++k) {
      const int64_t nx = hd->lv[k].nx, ny = hd->lv[k].ny;
      words += nx * ny + 2 * (nx + 2) * (ny + 2);
    }
    if (words > kCoarseSmemMax) {
      set_error("ad_create: coarse levels need %lld shared words (> %d)", (long long)words, kCoarseSmemMax);
      delete hd;
      return MG_ERR_INVALID;
    }
  }
  if (cudaFuncSetAttribute(k_ad_coarse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kCoarseSmemMax * sizeof(float))) != cudaSuccess) {
    set_error("ad_create: %s", cudaGetErrorString(cudaGetLastError()));
    delete hd;
    return MG_ERR_CUDA;
  }
  std::vector<float> inv;
  if (o.cycle == MG_CYCLE_V) {
    // the coarsest matrix in float64 from the same rule as the level
    const int k = L - 1;
    const double scale = o.coarse_op == AD_COARSE_GALERKIN ? (double)(1 << k) : 1.0;
    const double hk = h * (1 << k), kd = scale * nu * dt / (hk * hk);
    double wc[5] = {1.0 + 4.0 * kd, -kd, -kd, -kd, -kd};
    if (scheme == AD_CENTRAL) {
      wc[1] -= u * dt / (2 * hk);
      wc[2] += u * dt / (2 * hk);
      wc[3] -= v * dt / (2 * hk);
      wc[4] += v * dt / (2 * hk);
    } else {
      const double cx = u * dt / hk, cy = v * dt / hk;
      if (u >= 0) { wc[0] += cx; wc[1] -= cx; } else { wc[0] -= cx; wc[2] += cx; }
      if (v >= 0) { wc[0] += cy; wc[3] -= cy; } else { wc[0] -= cy; wc[4] += cy; }
    }
    if (!dense_inverse(hd->lv[k], wc, inv)) {
      set_error("ad_create: the coarsest matrix is singular");
      delete hd;
      return MG_ERR_INVALID;
    }
  }
  // one pool: b, r, the iterate, per-level arrays, the inverse, partials, state
  const size_t n0 = (size_t)nx * ny;
  const size_t tiles0 = (size_t)tile_grid(hd->lv[0]).x * tile_grid(hd->lv[0]).y;
  const size_t npart = std::max(tiles0, (size_t)hd->nsm * 8) + 1;
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  size_t bytes = al(n0 * 4) * 2 + al(n0 * 8) + al(npart * 8) + al(sizeof(State)) + al(inv.size() * 4 + 4);
  bytes += al(n0 * 4);  // x on level 0 (the V down leg's smoothed iterate)
  // levels 1 .. kc: right-hand side and correction; below kc also the
  // smoothed iterate; the single block keeps levels kc .. L-1 on chip
  for (int k = 1; k <= hd->kc; ++k) bytes += (k < hd->kc ? 3 : 2) * al((size_t)hd->lv[k].nx * hd->lv[k].ny * 4);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMalloc((void**)&hd->pool, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("ad_create: cudaMalloc of %zu bytes failed", bytes);
    delete hd;
    return MG_ERR_OOM;
  }
  char* p = hd->pool;
  auto take = [&](size_t b) {
    char* q = p;
    p += al(b);
    return q;
  };
  hd->b = (float*)take(n0 * 4);
  hd->r = (float*)take(n0 * 4);
  hd->xff = (float2*)take(n0 * 8);
  hd->partials = (double*)take(npart * 8);
  hd->st = (State*)take(sizeof(State));
  hd->inv = (float*)take(inv.size() * 4 + 4);
  hd->xk[0] = (float*)take(n0 * 4);
  hd->bk[0] = hd->r;
  hd->yk[0] = nullptr;
  for (int k = 1; k < L; ++k) hd->bk[k] = hd->xk[k] = hd->yk[k] = nullptr;
  for (int k = 1; k <= hd->kc; ++k) {
    const size_t nk = (size_t)hd->lv[k].nx * hd->lv[k].ny * 4;
    hd->bk[k] = (float*)take(nk);
    hd->yk[k] = (float*)take(nk);
    if (k < hd->kc) hd->xk[k] = (float*)take(nk);
  }
  mg_status st = MG_OK;
  if (cudaMemsetAsync(hd->pool, 0, bytes, s) != cudaSuccess ||
      (!inv.empty() &&
       cudaMemcpyAsync(hd->inv, inv.data(), inv.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) ||
      cudaMallocHost((void**)&hd->st_host, sizeof(State)) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("ad_create: %s", cudaGetErrorString(cudaGetLastError()));
    st = MG_ERR_CUDA;
  }
  if (st != MG_OK) {
    ad_destroy(hd);
    return st;
  }
  *out = hd;
  return MG_OK;
}

mg_status ad_solve(ad_handle hd, const float* d_b, const float* d_x0, float* d_x, double rel_tol, double l1_tol,
                   void* stream, ad_stats* out) {
  if (!hd || !d_b || !d_x || !(rel_tol >= 0) || !(l1_tol >= 0)) {
    set_error("ad_solve: NULL argument or negative tolerance");
    return MG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n0 = (size_t)hd->nx * hd->ny;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  NPMG_CUDA(cudaEventCreate(&e0));
  NPMG_CUDA(cudaEventCreate(&e1));
  NPMG_CUDA(cudaEventRecord(e0, s));
  NPMG_CUDA(cudaMemcpyAsync(hd->b, d_b, n0 * 4, cudaMemcpyDeviceToDevice, s));
  k_ad_init<<<row_grid(hd), kT, 0, s>>>(hd->lv[0], hd->b, d_x0, hd->xff, hd->st, rel_tol, l1_tol,
                                           hd->opt.max_cycles, hd->partials);
  hd->launches += 1;
  NPMG_CUDA(cudaGetLastError());
  NPMG_CUDA(ensure_graph(hd));
  // each graph launch runs kChunk cycles (kernels return once done); the
  // resid kernel ends the solve at max_cycles, at most one launch later
  const int max_launch = hd->opt.max_cycles / kChunk + 2;
  for (int it = 0; it < max_launch; ++it) {
    NPMG_CUDA(cudaGraphLaunch(hd->graph, s));
    hd->launches += hd->chunk_kernels;
    NPMG_CUDA(cudaMemcpyAsync(hd->st_host, hd->st, sizeof(State), cudaMemcpyDeviceToHost, s));
    NPMG_CUDA(cudaStreamSynchronize(s));
    if (hd->st_host->done) break;
  }
  // relres of the returned iterate, and the float32 output
  k_ad_resid<<<row_grid(hd), kT, 0, s>>>(hd->lv[0], hd->b, hd->xff, hd->r, hd->st, hd->partials, 1);
  k_ad_out<<<grid_1d(hd, n0), kT, 0, s>>>(n0, hd->xff, d_x);
  hd->launches += 2;
  NPMG_CUDA(cudaGetLastError());
  NPMG_CUDA(cudaEventRecord(e1, s));
  NPMG_CUDA(cudaMemcpyAsync(hd->st_host, hd->st, sizeof(State), cudaMemcpyDeviceToHost, s));
  NPMG_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const State& S = *hd->st_host;
  const mg_status status = S.done ? (mg_status)S.status : MG_NOT_CONVERGED;
  if (out) {
    out->status = status;
    out->cycles = S.cycles;
    out->relres0 = S.relres0;
    out->relres = S.relres;
    out->l1_first = S.l1_first;
    out->l1_last = S.l1;
    out->ms = ms;
  }
  return status;
}

int ad_num_levels(ad_handle hd) { return hd ? hd->L : 0; }

int ad_coarse_start(ad_handle hd) { return hd ? hd->kc : 0; }

int64_t ad_kernel_launches(ad_handle hd) { return hd ? hd->launches : 0; }

mg_status ad_destroy(ad_handle hd) {
  if (!hd) return MG_OK;
  if (hd->graph) cudaGraphExecDestroy(hd->graph);
  if (hd->pool) cudaFree(hd->pool);
  if (hd->st_host) cudaFreeHost(hd->st_host);
  delete hd;
  return MG_OK;
}

}  // extern "C"
