// Device code of the 2D thread-block-cluster kernels (the middle levels of
// a V-cycle, mg_cluster2d.cu; the whole preconditioned CG solve of a small
// grid, mg_cluster_pcg2d.cu): the per-block level layout, the sweep,
// restriction and prolongation phases with their ghost-row stores into the
// neighbouring blocks, and the V-cycle between the first and the last sweep
// of its first level.
//
// A distributed level k in block r of a cluster of C blocks holds the rows
// [r R, (r + 1) R) (R = ny_k / C, even) as (R + 2) padded rows of W = nx + 8
// entries (cells at columns 4 .. nx + 3, zero ghost columns 3 and nx + 4,
// ghost rows 0 and R + 1).  A phase that writes a block's first or last row
// also stores it into the neighbour's ghost row (distributed shared memory);
// the ghost rows at the domain's edges stay 0.  Threads work on groups of
// four cells of a row (float4; the cell bytes as one 32-bit word).
#pragma once
#include <cooperative_groups.h>

#include "coarse.cuh"
#include "launch.h"
#include "mg_kernels.cuh"

namespace npmg {
namespace cl2d {

namespace cg = cooperative_groups;


constexpr int kCT = 1024;  // threads per block
constexpr int kG = 4;      // first cell column of a padded row

__device__ __forceinline__ int lpad(const CLev& v) { return (v.R + 2) * v.W; }

// Arrays of level l in this block's shared memory.
struct LPtr {
  float *x0, *x1, *b, *lut;
  uint8_t* m;
};

__device__ __forceinline__ LPtr lptr(const CLev& v, float* S, unsigned char* Sb) {
  LPtr p;
  const int P = lpad(v);
  p.x0 = S + v.off;
  p.x1 = p.x0 + P;
  p.b = p.x1 + P;
  p.lut = S + v.loff;
  p.m = Sb + v.moff;
  return p;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, const float4& v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ uint32_t ld32(const uint8_t* p) { return *reinterpret_cast<const uint32_t*>(p); }
// link-count index (low four bits) and unknown flag of cell j of a word
__device__ __forceinline__ uint32_t nib(uint32_t m, int j) { return (m >> (8 * j)) & 15u; }
__device__ __forceinline__ bool fluid(uint32_t m, int j) { return (m >> (8 * j)) & kFluidBit; }

// Threads over (row, group of cells): thread t takes group t % ng of the
// rows t / ng, t / ng + rp, ... (rp = kCT / ng rows per pass); threads with
// t / ng >= rp stay idle.  sh = log2(ng) when ng is a power of two (shifts
// instead of integer divisions: a phase is issue-bound), else -1.
struct Map {
  int g, r0, rp;
};
__device__ __forceinline__ Map tmap(int ng, int sh) {
  Map t;
  if (sh >= 0) {
    t.g = (int)threadIdx.x & (ng - 1);
    t.r0 = (int)threadIdx.x >> sh;
    t.rp = kCT >> sh;
  } else {
    t.g = (int)threadIdx.x % ng;
    t.r0 = (int)threadIdx.x / ng;
    t.rp = kCT / ng;
  }
  return t;
}
// groups of four cells of level v
__device__ __forceinline__ Map tmap4(const CLev& v) { return tmap(v.L.nx >> 2, v.s4); }

// The same array in the neighbouring blocks (null at the domain's edges).
struct Nb {
  float *up, *dn;
};
__device__ __forceinline__ Nb nbrs(cg::cluster_group& cl, float* a, int rank, int C) {
  Nb n;
  n.up = rank > 0 ? cl.map_shared_rank(a, rank - 1) : nullptr;
  n.dn = rank < C - 1 ? cl.map_shared_rank(a, rank + 1) : nullptr;
  return n;
}

// Store four cells of row r at padded column c, and the first and last rows
// also into the neighbours' ghost rows.
__device__ __forceinline__ void put(float* a, const Nb& n, const CLev& v, int r, int c, const float4& o) {
  st4(a + (r + 1) * v.W + c, o);
  if (r == 0 && n.up) st4(n.up + (v.R + 1) * v.W + c, o);
  if (r == v.R - 1 && n.dn) st4(n.dn + c, o);
}

// The same for two cells at padded column c (8-byte aligned).
__device__ __forceinline__ void put2(float* a, const Nb& n, const CLev& v, int r, int c, const float2& o) {
  *reinterpret_cast<float2*>(a + (r + 1) * v.W + c) = o;
  if (r == 0 && n.up) *reinterpret_cast<float2*>(n.up + (v.R + 1) * v.W + c) = o;
  if (r == v.R - 1 && n.dn) *reinterpret_cast<float2*>(n.dn + c) = o;
}

// One weighted-Jacobi sweep of four cells at padded index q (16-byte
// aligned): (1 - omega) in + (omega / d)(b + nb(in)); 0 where a cell is not
// an unknown (omega / d = 0 and in = 0 there).
__device__ __forceinline__ float4 relax4(const CLev& v, const LPtr& p, const float* in, int q, float keep) {
  const int W = v.W;
  const float4 c = ld4(in + q), u = ld4(in + q - W), d = ld4(in + q + W), b = ld4(p.b + q);
  const float l = in[q - 1], r = in[q + 4];
  const uint32_t m = ld32(p.m + q);
  const float wx = v.L.wx, wy = v.L.wy;
  const float* w = p.lut + 64;
  float4 o;
  o.x = fmaf(keep, c.x, w[nib(m, 0)] * (b.x + (wx * (l + c.y) + wy * (u.x + d.x))));
  o.y = fmaf(keep, c.y, w[nib(m, 1)] * (b.y + (wx * (c.x + c.z) + wy * (u.y + d.y))));
  o.z = fmaf(keep, c.z, w[nib(m, 2)] * (b.z + (wx * (c.y + c.w) + wy * (u.z + d.z))));
  o.w = fmaf(keep, c.w, w[nib(m, 3)] * (b.w + (wx * (c.z + r) + wy * (u.w + d.w))));
  return o;
}

// A sweep of level v from `in` to `out`.
__device__ __forceinline__ void sweep(cg::cluster_group& cl, const CLev& v, const LPtr& p, const float* in,
                                      float* out, float keep, int rank, int C) {
  const Map t = tmap4(v);
  const Nb n = nbrs(cl, out, rank, C);
  if (t.r0 >= t.rp) return;
  const int c = kG + 4 * t.g;
  for (int r = t.r0; r < v.R; r += t.rp) put(out, n, v, r, c, relax4(v, p, in, (r + 1) * v.W + c, keep));
}


// Residual of x1 on level l and its 2x2 average: into the next level's b,
// with that level's first sweep from zero (x0 = (omega / d) b), or for the
// coarse cycle into global memory (bkc, level kd).  A thread takes two
// coarse cells: two rows of four fine cells (a restriction thread's chain
// of loads and sums is the phase's latency, so it is kept short).
__device__ __forceinline__ void restrict_level(cg::cluster_group& cl, const ClusterArgs& a, int l, float* S,
                                               unsigned char* Sb, float* __restrict__ bkc, int rank, int C) {
  const CLev& v = a.lv[l];
  const LPtr p = lptr(v, S, Sb);
  const bool last = l + 1 == a.nlev;
  const CLev& vc = a.lv[last ? l : l + 1];
  const LPtr pc = lptr(vc, S, Sb);
  const Nb n = last ? Nb{nullptr, nullptr} : nbrs(cl, pc.x0, rank, C);
  const int W = v.W, cR = v.R / 2, cnx = v.L.nx / 2;
  const Map t = tmap4(v);
  if (t.r0 >= t.rp) return;
  const float wx = v.L.wx, wy = v.L.wy;
  for (int cr = t.r0; cr < cR; cr += t.rp) {
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int ay = 0; ay < 2; ++ay) {
      const int q = (2 * cr + ay + 1) * W + kG + 4 * t.g;
      const float4 c = ld4(p.x1 + q), u = ld4(p.x1 + q - W), d = ld4(p.x1 + q + W), b = ld4(p.b + q);
      const float xl = p.x1[q - 1], xr = p.x1[q + 4];
      const uint32_t m = ld32(p.m + q);
      if (fluid(m, 0)) s0 += b.x - (p.lut[nib(m, 0)] * c.x - (wx * (xl + c.y) + wy * (u.x + d.x)));
      if (fluid(m, 1)) s0 += b.y - (p.lut[nib(m, 1)] * c.y - (wx * (c.x + c.z) + wy * (u.y + d.y)));
      if (fluid(m, 2)) s1 += b.z - (p.lut[nib(m, 2)] * c.z - (wx * (c.y + c.w) + wy * (u.z + d.z)));
      if (fluid(m, 3)) s1 += b.w - (p.lut[nib(m, 3)] * c.w - (wx * (c.z + xr) + wy * (u.w + d.w)));
    }
    const float2 cb = make_float2(0.25f * s0, 0.25f * s1);
    if (last) {
      *reinterpret_cast<float2*>(bkc + (size_t)(rank * cR + cr) * cnx + 2 * t.g) = cb;
    } else {
      const int c2 = kG + 2 * t.g, qc = (cr + 1) * vc.W + c2;
      *reinterpret_cast<float2*>(pc.b + qc) = cb;
      const uint32_t mc = *reinterpret_cast<const uint16_t*>(pc.m + qc);
      const float* w = pc.lut + 64;
      put2(pc.x0, n, vc, cr, c2, make_float2(w[nib(mc, 0)] * cb.x, w[nib(mc, 1)] * cb.y));
    }
  }
}

// x1 += s e on the last distributed level, e the coarse cycle's correction
// (level kd, global): copy prolongation, unknowns only.
__device__ __forceinline__ void prolong_from_global(cg::cluster_group& cl, const ClusterArgs& a, float* S,
                                                    unsigned char* Sb, const float* ykc, int rank, int C) {
  const CLev& v = a.lv[a.nlev - 1];
  const LPtr p = lptr(v, S, Sb);
  const Nb n = nbrs(cl, p.x1, rank, C);
  const Map t = tmap4(v);
  if (t.r0 >= t.rp) return;
  const int c = kG + 4 * t.g, cnx = v.L.nx / 2;
  const float s = a.s;
  for (int r = t.r0; r < v.R; r += t.rp) {
    const int q = (r + 1) * v.W + c;
    const uint32_t m = ld32(p.m + q);
    float4 x = ld4(p.x1 + q);
    const float2 e = *reinterpret_cast<const float2*>(ykc + (size_t)((rank * v.R + r) >> 1) * cnx + 2 * t.g);
    if (fluid(m, 0)) x.x = fmaf(s, e.x, x.x);
    if (fluid(m, 1)) x.y = fmaf(s, e.x, x.y);
    if (fluid(m, 2)) x.z = fmaf(s, e.y, x.z);
    if (fluid(m, 3)) x.w = fmaf(s, e.y, x.w);
    put(p.x1, n, v, r, c, x);
  }
}

// Last sweep of level l (x0 -> new x1), its scaled value added at once to
// the four children of each cell in level l - 1's x1 (unknowns only).
__device__ __forceinline__ void sweep_prolong(cg::cluster_group& cl, const ClusterArgs& a, int l, float* S,
                                              unsigned char* Sb, float keep, int rank, int C) {
  const CLev& v = a.lv[l];
  const CLev& vf = a.lv[l - 1];
  const LPtr p = lptr(v, S, Sb), pf = lptr(vf, S, Sb);
  const Nb n = nbrs(cl, pf.x1, rank, C);
  const Map t = tmap4(v);
  if (t.r0 >= t.rp) return;
  const int c = kG + 4 * t.g, cf = kG + 8 * t.g;
  const float s = a.s;
  for (int r = t.r0; r < v.R; r += t.rp) {
    const float4 o = relax4(v, p, p.x0, (r + 1) * v.W + c, keep);
#pragma unroll
    for (int ay = 0; ay < 2; ++ay) {
      const int fr = 2 * r + ay, qf = (fr + 1) * vf.W + cf;
      float4 A = ld4(pf.x1 + qf), B = ld4(pf.x1 + qf + 4);
      const uint32_t mA = ld32(pf.m + qf), mB = ld32(pf.m + qf + 4);
      if (fluid(mA, 0)) A.x = fmaf(s, o.x, A.x);
      if (fluid(mA, 1)) A.y = fmaf(s, o.x, A.y);
      if (fluid(mA, 2)) A.z = fmaf(s, o.y, A.z);
      if (fluid(mA, 3)) A.w = fmaf(s, o.y, A.w);
      if (fluid(mB, 0)) B.x = fmaf(s, o.z, B.x);
      if (fluid(mB, 1)) B.y = fmaf(s, o.z, B.y);
      if (fluid(mB, 2)) B.z = fmaf(s, o.w, B.z);
      if (fluid(mB, 3)) B.w = fmaf(s, o.w, B.w);
      put(pf.x1, n, vf, fr, cf, A);
      put(pf.x1, n, vf, fr, cf + 4, B);
    }
  }
}

// Per launch: the zero ghost columns and, at the domain's edges, ghost rows
// of both iterate buffers; the cell bytes of the block's rows (link counts
// of an unmasked level from its coordinates); the diagonal tables.
__device__ __forceinline__ void setup(const ClusterArgs& a, float* S, unsigned char* Sb, int rank, int C) {
  for (int l = 0; l < a.nlev; ++l) {
    const CLev& v = a.lv[l];
    const LPtr p = lptr(v, S, Sb);
    const int nx = v.L.nx, W = v.W, R = v.R;
    for (int i = threadIdx.x; i < 2 * R; i += kCT) {
      const int q = ((i >> 1) + 1) * W + ((i & 1) ? kG + nx : kG - 1);
      p.x0[q] = 0.f;
      p.x1[q] = 0.f;
    }
    for (int i = threadIdx.x; i < nx; i += kCT) {
      if (rank == 0) p.x0[kG + i] = p.x1[kG + i] = 0.f;
      if (rank == C - 1) p.x0[(R + 1) * W + kG + i] = p.x1[(R + 1) * W + kG + i] = 0.f;
    }
    const Map t = tmap4(v);
    if (t.r0 < t.rp) {
      for (int r = t.r0; r < R; r += t.rp) {
        const int gy = rank * R + r, gx = 4 * t.g;
        uint32_t m = 0;
        if (v.L.cell) {
          m = ld32(v.L.cell + (size_t)gy * nx + gx);
        } else {
          const uint32_t my = (uint32_t)axis_count(gy, v.L.ny, v.L.bcD, 2) << 2;
#pragma unroll
          for (int j = 0; j < 4; ++j)
            m |= (uint32_t)(kFluidBit | axis_count(gx + j, nx, v.L.bcD, 0) | my) << (8 * j);
        }
        *reinterpret_cast<uint32_t*>(p.m + (r + 1) * W + kG + gx) = m;
      }
    }
    if (threadIdx.x < 16) {
      const int kx = threadIdx.x & 3, ky = threadIdx.x >> 2;
      const float d = (kx <= 2 && ky <= 2) ? v.L.wx * (float)kx + v.L.wy * (float)ky : 0.f;
      p.lut[threadIdx.x] = d;
      p.lut[64 + threadIdx.x] = d > 0.f ? a.omega / d : 0.f;
    }
  }
}

// The V-cycle from the first sweep of level 0 (x0 with its ghost rows
// stored, after a cluster barrier) to the first of its two up sweeps (x0,
// stored likewise, after a barrier): down legs, the coarse cycle (levels
// kd ..) in block 0 through global memory (bkc, ykc), up legs.  The last
// sweep of level 0 is the caller's.  `st` takes the coarse cycle's timeout
// report; `load_image`: the coarse cycle loads its constant image (a kernel
// that runs several cycles loads it once).
__device__ __forceinline__ void vcycle_body(cg::cluster_group& cl, const ClusterArgs& a, float* S,
                                            unsigned char* Sb, float* bkc, float* ykc, SolveState* st, int rank,
                                            int C, float keep, bool load_image = true) {
  const int n = a.nlev;
  // down legs: second sweep, then residual and restriction (with the next
  // level's first sweep)
  for (int l = 0; l < n; ++l) {
    const CLev& v = a.lv[l];
    const LPtr p = lptr(v, S, Sb);
    sweep(cl, v, p, p.x0, p.x1, keep, rank, C);
    cl.sync();
    restrict_level(cl, a, l, S, Sb, bkc, rank, C);
    cl.sync();
  }
  if (rank == 0) coarse_cycle<2, float>(a.ca, bkc, ykc, st, S + a.ca_off, a.ca_floats, load_image);
  cl.sync();
  prolong_from_global(cl, a, S, Sb, ykc, rank, C);
  cl.sync();
  // up legs: two sweeps; the second adds the level's correction to the
  // finer level
  for (int l = n - 1; l >= 0; --l) {
    const CLev& v = a.lv[l];
    const LPtr p = lptr(v, S, Sb);
    sweep(cl, v, p, p.x1, p.x0, keep, rank, C);
    cl.sync();
    if (l > 0) {
      sweep_prolong(cl, a, l, S, Sb, keep, rank, C);
      cl.sync();
    }
  }
}

}  // namespace cl2d
}  // namespace npmg
