// The whole preconditioned CG solve of a small 2D grid in one launch of a
// thread-block cluster.
//
// A 2D grid whose levels and CG vectors fit the shared memory of a cluster
// of 16 blocks (256^2: about 150 KB per block) spends most of a solve in
// launch latency when every leg, update and reduction is a kernel: about
// 55 us per CG iteration for 65 k cells.  Here one launch runs a whole
// inner CG solve: the levels 0 .. kd-1 distributed over the blocks by rows
// (cluster2d.cuh), the coarse cycle of the levels below in block 0, the CG
// vectors of level 0 in shared memory (r is level 0's b, z its second
// iterate buffer, two p buffers and the inner solution d beside them).  The
// refinement step between inner solves (x += sigma d and the scaled
// residual, in float64) stays with the kernels that use every SM: GB300
// runs float64 at 1/64 of the float32 rate, so on 16 SMs it would cost
// ten times as long.
//
// The iteration is that of the separate kernels (Sec. 2.2 V(2,2) cycle as
// the preconditioner of CG): z = M r and (r, z) -> beta; p = z + beta p,
// A' p and (p, A' p) -> alpha; d += alpha p, r -= alpha A' p (A' p formed
// again from p), ||r||^2 and the inner convergence test, with the next
// cycle's first sweep of level 0 from r.  Each reduction is a block sum
// stored into every block's slot array, one cluster barrier, and the 16
// slots summed in the same order in every block, so every block takes the
// same decisions (the test of the separate kernels' `inner_decide`, on a
// per-block copy of the solve state; the scalars alpha and beta and the
// convergence test in float32).
#include <math.h>

#include "cluster2d.cuh"
#include "refine.cuh"

namespace npmg {

using namespace cl2d;

namespace {

// Float-float sum over a warp (FP32 arithmetic, about 48 bits; GB300 runs
// float64 at 1/64 of the float32 rate, one float64 warp instruction holding
// its sub-partition's pipe for 64 cycles); lane 0 holds the total.
__device__ __forceinline__ ff warp_sum_ff(ff s) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const ff t = {__shfl_down_sync(0xffffffffu, s.hi, o), __shfl_down_sync(0xffffffffu, s.lo, o)};
    s = ff_add(s, t);
  }
  return s;
}

// Block sum (float-float) stored into slot `rank` of every block's `slots`;
// the total is read after the next cluster barrier (slots_total).
__device__ __forceinline__ void push_ff(cg::cluster_group& cl, ff v, float2* slots, float2* wsum, int rank, int C) {
  const ff s = warp_sum_ff(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wsum[w] = make_float2(s.hi, s.lo);
  __syncthreads();
  if (w == 0) {
    const float2 q = wsum[lane];
    ff t = warp_sum_ff({q.x, q.y});
    t.hi = __shfl_sync(0xffffffffu, t.hi, 0);
    t.lo = __shfl_sync(0xffffffffu, t.lo, 0);
    if (lane < C) cl.map_shared_rank(slots, lane)[rank] = make_float2(t.hi, t.lo);
  }
}

// Warp 0: the sum of the slots in a fixed order (the same value in every
// block), in lane 0.
__device__ __forceinline__ ff slots_total(const float2* slots, int C) {
  const int lane = threadIdx.x & 31;
  const float2 q = lane < C ? slots[lane] : make_float2(0.f, 0.f);
  return warp_sum_ff({q.x, q.y});
}

// Level 0's first sweep from zero, x0 = (omega / d) r, ghost rows stored.
__device__ __forceinline__ void first_sweep(cg::cluster_group& cl, const CLev& v, const LPtr& p, int rank, int C) {
  const Nb n = nbrs(cl, p.x0, rank, C);
  const Map t = tmap4(v);
  if (t.r0 >= t.rp) return;
  const int c = kG + 4 * t.g;
  const float* w = p.lut + 64;
  for (int r = t.r0; r < v.R; r += t.rp) {
    const int q = (r + 1) * v.W + c;
    const uint32_t m = ld32(p.m + q);
    const float4 b = ld4(p.b + q);
    put(p.x0, n, v, r, c,
        make_float4(w[nib(m, 0)] * b.x, w[nib(m, 1)] * b.y, w[nib(m, 2)] * b.z, w[nib(m, 3)] * b.w));
  }
}

// z = the last sweep of level 0 (x0 -> x1, ghost rows stored); returns the
// thread's sum of r z.
__device__ __forceinline__ float sweep_z(cg::cluster_group& cl, const CLev& v, const LPtr& p, float keep, int rank,
                                         int C) {
  const Nb n = nbrs(cl, p.x1, rank, C);
  const Map t = tmap4(v);
  float acc = 0.f;
  if (t.r0 >= t.rp) return acc;
  const int c = kG + 4 * t.g;
  for (int r = t.r0; r < v.R; r += t.rp) {
    const int q = (r + 1) * v.W + c;
    const float4 o = relax4(v, p, p.x0, q, keep);
    put(p.x1, n, v, r, c, o);
    const float4 b = ld4(p.b + q);
    acc = fmaf(b.x, o.x, acc);
    acc = fmaf(b.y, o.y, acc);
    acc = fmaf(b.z, o.z, acc);
    acc = fmaf(b.w, o.w, acc);
  }
  return acc;
}

// A' q for four cells at q (a vector with its ghost rows and zero ghost
// columns; 0 off the unknowns).
__device__ __forceinline__ float4 apply4(const CLev& v, const LPtr& p, const float* x, int q, float4& xc) {
  const int W = v.W;
  xc = ld4(x + q);
  const float4 u = ld4(x + q - W), d = ld4(x + q + W);
  const float l = x[q - 1], r = x[q + 4];
  const uint32_t m = ld32(p.m + q);
  const float wx = v.L.wx, wy = v.L.wy;
  float4 a;
  a.x = fluid(m, 0) ? fmaf(p.lut[nib(m, 0)], xc.x, -fmaf(wy, u.x + d.x, wx * (l + xc.y))) : 0.f;
  a.y = fluid(m, 1) ? fmaf(p.lut[nib(m, 1)], xc.y, -fmaf(wy, u.y + d.y, wx * (xc.x + xc.z))) : 0.f;
  a.z = fluid(m, 2) ? fmaf(p.lut[nib(m, 2)], xc.z, -fmaf(wy, u.z + d.z, wx * (xc.y + xc.w))) : 0.f;
  a.w = fluid(m, 3) ? fmaf(p.lut[nib(m, 3)], xc.w, -fmaf(wy, u.w + d.w, wx * (xc.z + r))) : 0.f;
  return a;
}

// p = z + beta p_old (first: p = z) at four cells and their neighbours,
// A' p and the thread's sum of p A' p; p stored (0 off the unknowns) with
// its ghost rows.
__device__ __forceinline__ float p_update(cg::cluster_group& cl, const CLev& v, const LPtr& p, const float* pold,
                                          float* pnew, float beta, bool first, int rank, int C) {
  const Nb n = nbrs(cl, pnew, rank, C);
  const Map t = tmap4(v);
  float acc = 0.f;
  if (t.r0 >= t.rp) return acc;
  const int c = kG + 4 * t.g, W = v.W;
  const float* z = p.x1;
  const float wx = v.L.wx, wy = v.L.wy;
  for (int r = t.r0; r < v.R; r += t.rp) {
    const int q = (r + 1) * W + c;
    float4 pc = ld4(z + q), pu = ld4(z + q - W), pd = ld4(z + q + W);
    float pl = z[q - 1], pr = z[q + 4];
    if (!first) {
      const float4 qc = ld4(pold + q), qu = ld4(pold + q - W), qd = ld4(pold + q + W);
      pc = make_float4(fmaf(beta, qc.x, pc.x), fmaf(beta, qc.y, pc.y), fmaf(beta, qc.z, pc.z), fmaf(beta, qc.w, pc.w));
      pu = make_float4(fmaf(beta, qu.x, pu.x), fmaf(beta, qu.y, pu.y), fmaf(beta, qu.z, pu.z), fmaf(beta, qu.w, pu.w));
      pd = make_float4(fmaf(beta, qd.x, pd.x), fmaf(beta, qd.y, pd.y), fmaf(beta, qd.z, pd.z), fmaf(beta, qd.w, pd.w));
      pl = fmaf(beta, pold[q - 1], pl);
      pr = fmaf(beta, pold[q + 4], pr);
    }
    const uint32_t m = ld32(p.m + q);
    float4 a;
    a.x = fmaf(p.lut[nib(m, 0)], pc.x, -fmaf(wy, pu.x + pd.x, wx * (pl + pc.y)));
    a.y = fmaf(p.lut[nib(m, 1)], pc.y, -fmaf(wy, pu.y + pd.y, wx * (pc.x + pc.z)));
    a.z = fmaf(p.lut[nib(m, 2)], pc.z, -fmaf(wy, pu.z + pd.z, wx * (pc.y + pc.w)));
    a.w = fmaf(p.lut[nib(m, 3)], pc.w, -fmaf(wy, pu.w + pd.w, wx * (pc.z + pr)));
    if (!fluid(m, 0)) pc.x = a.x = 0.f;
    if (!fluid(m, 1)) pc.y = a.y = 0.f;
    if (!fluid(m, 2)) pc.z = a.z = 0.f;
    if (!fluid(m, 3)) pc.w = a.w = 0.f;
    put(pnew, n, v, r, c, pc);
    acc = fmaf(pc.x, a.x, acc);
    acc = fmaf(pc.y, a.y, acc);
    acc = fmaf(pc.z, a.z, acc);
    acc = fmaf(pc.w, a.w, acc);
  }
  return acc;
}

// d += alpha p (first: d = alpha p), r -= alpha A' p, the thread's sum of
// r^2, and the next cycle's first sweep of level 0 from the new r.
__device__ __forceinline__ float xr_update(cg::cluster_group& cl, const CLev& v, const LPtr& p, const float* pn,
                                           float* D, float alpha, bool first, int rank, int C) {
  const Nb n = nbrs(cl, p.x0, rank, C);
  const Map t = tmap4(v);
  float acc = 0.f;
  if (t.r0 >= t.rp) return acc;
  const int c = kG + 4 * t.g;
  const float* w = p.lut + 64;
  for (int r = t.r0; r < v.R; r += t.rp) {
    const int q = (r + 1) * v.W + c;
    float4 pc;
    const float4 a = apply4(v, p, pn, q, pc);
    float4 d;
    if (first) {
      d = make_float4(alpha * pc.x, alpha * pc.y, alpha * pc.z, alpha * pc.w);
    } else {
      d = ld4(D + q);
      d = make_float4(fmaf(alpha, pc.x, d.x), fmaf(alpha, pc.y, d.y), fmaf(alpha, pc.z, d.z), fmaf(alpha, pc.w, d.w));
    }
    st4(D + q, d);
    float4 rv = ld4(p.b + q);
    rv = make_float4(fmaf(-alpha, a.x, rv.x), fmaf(-alpha, a.y, rv.y), fmaf(-alpha, a.z, rv.z),
                     fmaf(-alpha, a.w, rv.w));
    st4(p.b + q, rv);
    acc = fmaf(rv.x, rv.x, acc);
    acc = fmaf(rv.y, rv.y, acc);
    acc = fmaf(rv.z, rv.z, acc);
    acc = fmaf(rv.w, rv.w, acc);
    const uint32_t m = ld32(p.m + q);
    put(p.x0, n, v, r, c,
        make_float4(w[nib(m, 0)] * rv.x, w[nib(m, 1)] * rv.y, w[nib(m, 2)] * rv.z, w[nib(m, 3)] * rv.w));
  }
  return acc;
}

}  // namespace

__global__ void __launch_bounds__(kCT, 1) k_cluster_pcg2d(const __grid_constant__ ClusterPcgArgs pa,
                                                          const float* __restrict__ r0, float* __restrict__ dout,
                                                          float* __restrict__ bkc, float* __restrict__ ykc,
                                                          SolveState* __restrict__ st) {
  chain_enter();
  cg::cluster_group cl = cg::this_cluster();
  const ClusterArgs& a = pa.a;
  const int rank = (int)cl.block_rank(), C = a.C;
  extern __shared__ __align__(16) unsigned char smem_cl[];
  float* S = reinterpret_cast<float*>(smem_cl);
  unsigned char* Sb = smem_cl;
  __shared__ SolveState sst;   // this block's copy of the solve state
  __shared__ SolveState cst;   // block 0: the coarse cycle's timeout report
  __shared__ float2 wsum[32];
  float2* slots = reinterpret_cast<float2*>(S + pa.red_off);
  if (threadIdx.x == 0) {
    sst = *st;
    cst.status = MG_OK;
    cst.inner_done = cst.outer_done = 0;
  }
  __syncthreads();
  if (sst.inner_done || sst.outer_done) return;  // the same state in every block
  const CLev& v0 = a.lv[0];
  const LPtr p0 = lptr(v0, S, Sb);
  const int P = lpad(v0);
  float* const P0 = S + pa.pcg_off;  // p buffers: P0 + k P, k = 0, 1
  float* D = S + pa.pcg_off + 2 * P;
  const float keep = 1.f - a.omega;
  setup(a, S, Sb, rank, C);
  {
    // ghost columns and the domain-edge ghost rows of both p buffers; r
    // from the refinement step (scaled residual)
    const int nx = v0.L.nx, W = v0.W, R = v0.R;
    for (int i = threadIdx.x; i < 2 * R; i += kCT) {
      const int q = ((i >> 1) + 1) * W + ((i & 1) ? kG + nx : kG - 1);
      P0[q] = P0[P + q] = 0.f;
    }
    for (int i = threadIdx.x; i < nx; i += kCT) {
      if (rank == 0) P0[kG + i] = P0[P + kG + i] = 0.f;
      if (rank == C - 1) P0[(R + 1) * W + kG + i] = P0[P + (R + 1) * W + kG + i] = 0.f;
    }
    const Map t = tmap4(v0);
    if (t.r0 < t.rp)
      for (int r = t.r0; r < R; r += t.rp)
        st4(p0.b + (r + 1) * W + kG + 4 * t.g, ld4(r0 + (size_t)(rank * R + r) * nx + 4 * t.g));
  }
  // every block has started and is set up
  cl.sync();
  first_sweep(cl, v0, p0, rank, C);
  cl.sync();
  int par = 0, set = 0;
  bool load = true;
  // block sums into the slots, one cluster barrier; the total in thread 0
  auto reduce = [&](ff v) -> float {
    float2* sl = slots + 16 * set;
    push_ff(cl, v, sl, wsum, rank, C);
    cl.sync();
    set ^= 1;
    const ff t = slots_total(sl, C);
    return __shfl_sync(0xffffffffu, t.hi + t.lo, 0);
  };
  // Every thread runs the inner loop's control itself, in float32, on the
  // totals every warp sums from the slots (the same values in every thread
  // of every block; no block barrier or float64 operation between two
  // cluster barriers): beta, alpha, and the test of inner_decide with its
  // bounds rounded once, ||r||^2 <= eta^2 ||r_0||^2 (converged) and
  // > 1e12 ||r_0||^2 or not finite (diverged).  Thread 0 writes the state
  // at the end.
  __shared__ float bounds[2];
  if (threadIdx.x == 0) {
    bounds[0] = (float)(sst.eta * sst.eta * sst.r0norm2);
    bounds[1] = (float)(1e12 * sst.r0norm2);
  }
  __syncthreads();
  const bool krylov = sst.krylov != 0;
  bool first = sst.first != 0, diverged = false;
  int it = sst.it, done_its = 0;
  float rz = 0.f, rz_old = 0.f, pAp = 0.f, r2 = 0.f, alpha = 0.f, beta = 0.f;
  for (bool more = !sst.inner_done && !sst.outer_done; more;) {
    // z = M r
    vcycle_body(cl, a, S, Sb, bkc, ykc, rank == 0 ? &cst : nullptr, rank, C, keep, load);
    load = false;
    const bool tmo = rank == 0 && cst.status == MG_TIMEOUT;
    const float rzp = sweep_z(cl, v0, p0, keep, rank, C);
    rz = reduce({tmo ? __int_as_float(0x7fc00000) : rzp, 0.f});
    const bool pfirst = first || !krylov;
    beta = pfirst ? 0.f : rz / rz_old;
    rz_old = rz;
    // p = z + beta p, A' p, alpha
    pAp = reduce({p_update(cl, v0, p0, P0 + par * P, P0 + (1 - par) * P, beta, pfirst, rank, C), 0.f});
    alpha = krylov ? rz / pAp : 1.f;
    // d += alpha p, r -= alpha A' p, ||r||^2, the next cycle's first sweep
    r2 = reduce({xr_update(cl, v0, p0, P0 + (1 - par) * P, D, alpha, first, rank, C), 0.f});
    first = false;
    ++it;
    ++done_its;
    par ^= 1;
    if (!(r2 <= bounds[1])) {  // not finite, or blown up
      diverged = true;
      more = false;
    } else if (r2 <= bounds[0] || it >= sst.max_inner || done_its > sst.max_inner + 1) {
      more = false;
    }
  }
  if (threadIdx.x == 0) {
    sst.it = it;
    sst.iters_total += done_its;
    if (done_its > 0) {
      sst.first = 0;
      sst.inner_done = 1;
      sst.rnorm2 = (double)r2;
      sst.rz = sst.rz_old = (double)rz;
      sst.pAp = (double)pAp;
      sst.beta = (double)beta;
      sst.alpha = (double)alpha;
    }
    if (diverged) {
      sst.status = MG_DIVERGED;
      sst.outer_done = 1;
    }
  }
  // the inner solution d' for the refinement step, and the state
  {
    const Map t = tmap4(v0);
    if (t.r0 < t.rp)
      for (int r = t.r0; r < v0.R; r += t.rp)
        st4(dout + (size_t)(rank * v0.R + r) * v0.L.nx + 4 * t.g, ld4(D + (r + 1) * v0.W + kG + 4 * t.g));
  }
  if (rank == 0 && threadIdx.x == 0) {
    if (cst.status == MG_TIMEOUT) {
      sst.status = MG_TIMEOUT;
      sst.inner_done = sst.outer_done = 1;
    }
    *st = sst;
  }
}

int cluster_pcg2d_fit(size_t smem, size_t smem_limit, int C) {
  if (cudaFuncSetAttribute(k_cluster_pcg2d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit) !=
      cudaSuccess)
    return 0;
  if (C > 8 &&
      cudaFuncSetAttribute(k_cluster_pcg2d, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_cluster_pcg2d, &cfg) != cudaSuccess) n = 0;
  cudaGetLastError();
  return n;
}

cudaError_t launch_cluster_pcg2d(const ClusterPcgArgs& pa, size_t smem, const float* r0, float* dout, float* bkc,
                                 float* ykc, SolveState* st, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pa.a.C);
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = pa.a.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = chain_launch_enabled() ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, k_cluster_pcg2d, pa, r0, dout, bkc, ykc, st);
}

}  // namespace npmg
