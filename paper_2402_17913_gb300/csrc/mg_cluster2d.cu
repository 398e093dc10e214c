// The middle levels of the 2D V-cycle in one thread-block cluster.
//
// Below the finest one or two levels a 2D level is too small to fill the
// GPU, and each of its legs used to be a launch of a few microseconds.
// Here the levels k1 .. kd-1 (rows a multiple of 2C, rows a multiple of 8
// cells) run in one launch of a cluster of C blocks (C = 16, or 8): block r
// owns the rows [r R_k, (r + 1) R_k) of level k (R_k = ny_k / C, even, so a
// row pair of the 2x2 restriction and the four children of a coarse cell
// stay in one block: restriction and prolongation are block-local).  Every
// level lives in the blocks' shared memory with a ghost ring: the ghost
// columns stay 0 (the zero padding of Sec. 2.1); a block writes its first
// and last rows also into its neighbours' ghost rows (distributed shared
// memory stores), which stay 0 at the domain's edges.  One cluster barrier
// per phase (a cluster barrier costs about 0.3 us on GB300, a block
// barrier 0.05 us): a phase writes one buffer and reads another, and the
// restriction writes the next level's first sweep, the last sweep of a
// level adds its correction to the finer level directly.  The levels below
// (kd ..), the single-block coarse cycle with the exact coarsest solve, run
// in block 0 between the down and the up legs, handed their right-hand side
// and correction through global memory.
//
// Threads work on groups of four cells of a row (float4 in shared memory,
// the cell bytes as one 32-bit word).
//
// Same arithmetic as the other level kernels: weighted Jacobi
// (Eq. Jacobi-1-relax) x <- (1 - omega) x + (omega / d)(b + nb), two sweeps
// per leg, from zero on the down leg; residual and 2x2 average restriction
// (App. B); copy prolongation plus the scaled correction (Sec. 2.2).  The
// diagonal comes from the cell byte (link counts; 0 = not an unknown)
// through a per-level table.
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "cluster2d.cuh"

namespace npmg {

using namespace cl2d;

__global__ void __launch_bounds__(kCT, 1) k_cluster2d(const __grid_constant__ ClusterArgs a,
                                                      const float* __restrict__ bin, float* __restrict__ yout,
                                                      float* __restrict__ bkc, float* __restrict__ ykc,
                                                      SolveState* __restrict__ st) {
  chain_enter();
  if (st && st->inner_done) return;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), C = a.C;
  extern __shared__ __align__(16) unsigned char smem_cl[];
  float* S = reinterpret_cast<float*>(smem_cl);
  unsigned char* Sb = smem_cl;
  const float keep = 1.f - a.omega;
  setup(a, S, Sb, rank, C);
  // every block has started (its shared memory may be written) and is set up
  cl.sync();
  {
    // level k1: b from global memory, the first sweep from zero
    const CLev& v = a.lv[0];
    const LPtr p = lptr(v, S, Sb);
    const Nb nb = nbrs(cl, p.x0, rank, C);
    const Map t = tmap4(v);
    if (t.r0 < t.rp) {
      const int c = kG + 4 * t.g;
      const float* w = p.lut + 64;
      for (int r = t.r0; r < v.R; r += t.rp) {
        const int q = (r + 1) * v.W + c;
        const uint32_t m = ld32(p.m + q);
        const float4 g = ld4(bin + (size_t)(rank * v.R + r) * v.L.nx + 4 * t.g);
        const float4 b = make_float4(fluid(m, 0) ? g.x : 0.f, fluid(m, 1) ? g.y : 0.f, fluid(m, 2) ? g.z : 0.f,
                                     fluid(m, 3) ? g.w : 0.f);
        st4(p.b + q, b);
        put(p.x0, nb, v, r, c,
            make_float4(w[nib(m, 0)] * b.x, w[nib(m, 1)] * b.y, w[nib(m, 2)] * b.z, w[nib(m, 3)] * b.w));
      }
    }
  }
  cl.sync();
  vcycle_body(cl, a, S, Sb, bkc, ykc, st, rank, C, keep);
  // level k1's last sweep is the result
  {
    const CLev& v = a.lv[0];
    const LPtr p = lptr(v, S, Sb);
    const Map t = tmap4(v);
    if (t.r0 < t.rp) {
      const int c = kG + 4 * t.g;
      for (int r = t.r0; r < v.R; r += t.rp)
        st4(yout + (size_t)(rank * v.R + r) * v.L.nx + 4 * t.g, relax4(v, p, p.x0, (r + 1) * v.W + c, keep));
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// Shared-memory layout of one block: the levels k1 .. kd-1 (three float
// arrays and a diagonal table each), `extra` floats (at *extra_off), the
// coarse cycle's region, the levels' cell bytes.  Returns the bytes.
static size_t cluster_layout(ClusterArgs& a, const LevelDev* lv, int k1, int kd, int C, size_t ca_bytes,
                             size_t extra = 0, int* extra_off = nullptr) {
  size_t f = 0;  // floats
  for (int k = k1; k < kd; ++k) {
    CLev& v = a.lv[k - k1];
    v.L = lv[k];
    v.R = lv[k].ny / C;
    v.W = lv[k].nx + 2 * kG;
    v.off = (int)f;
    f += (size_t)3 * (v.R + 2) * v.W;
    v.loff = (int)f;
    f += 128;
    auto lg = [](int n) { return n > 0 && (n & (n - 1)) == 0 ? __builtin_ctz((unsigned)n) : -1; };
    v.s4 = lg(lv[k].nx / 4);
  }
  if (extra_off) *extra_off = (int)f;
  f += (extra + 3) / 4 * 4;
  a.ca_off = (int)((f + 3) / 4 * 4);
  a.ca_floats = (int)(ca_bytes / 4);
  f = a.ca_off + ca_bytes / 4;
  size_t b = f * 4;
  for (int k = k1; k < kd; ++k) {
    CLev& v = a.lv[k - k1];
    v.moff = (int)b;
    b += ((size_t)(v.R + 2) * v.W + 15) / 16 * 16;
  }
  a.nlev = kd - k1;
  a.C = C;
  return b;
}

// Cells of the first level the cluster's coarse cycle takes at most
// (NPMG_CLUSTER_COARSE_CELLS, 16 .. 8192, to tune it).  2048: a phase of
// the single block costs about a third of a cluster phase, so a 32^2 level
// is cheaper in block 0 (256^2 solves measured 4% faster than with 512).
static size_t cluster_coarse_cells() {
  const char* e = getenv("NPMG_CLUSTER_COARSE_CELLS");
  const long v = e ? atol(e) : 0;
  return v >= 16 && v <= 8192 ? (size_t)v : 2048;
}

// A level the cluster distributes: 2D, an even number of rows per block,
// rows of whole groups of eight cells (the restriction's thread takes
// eight) and at most 4096 cells (a row of groups within one block pass).
static bool distributable(const LevelDev& v, int C) {
  return v.nz == 1 && v.ny % (2 * C) == 0 && v.nx % 8 == 0 && v.nx <= 4096;
}

bool cluster2d_plan(const LevelDev* lv, int L, int kc, ClusterArgs* out, int* k1_out, int* kd_out,
                    size_t* smem_out, size_t* ca_bytes_out) {
  // opt-in (NPMG_CLUSTER2D=1): measured on GB300 a cluster phase costs
  // about 1 us (barrier, ghost-row stores, one group of cells per thread),
  // so a level's four phases cost what its two leg launches do, and the
  // single-block coarse cycle inside the cluster is not faster than alone:
  // the 2048x1024 V-cycle took 64 us against 54 us with the legs launched
  // one by one
  const char* on = getenv("NPMG_CLUSTER2D");
  if (!on || atoi(on) == 0 || kc < 2) return false;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  // the coarse cycle's own static shared memory (its barrier) and slack
  const size_t limit = (size_t)optin - 1024;
  const size_t thr = cluster_coarse_cells();
  for (int C : {16, 8}) {
    // k1 < kc: the legs above k1 are the ones enqueued level by level
    for (int k1 = 1; k1 < kc; ++k1) {
      if (!distributable(lv[k1], C)) continue;
      int kq = k1;  // levels k1 .. kq-1 are distributable
      while (kq < L - 1 && distributable(lv[kq], C)) ++kq;
      // the coarse cycle starts at the first level within the cell limit,
      // not above kc (its buffers are sized for level kc)
      int kd = std::max(k1 + 1, kc);
      while (kd < kq && (size_t)lv[kd].nx * lv[kd].ny > thr) ++kd;
      if (kd > kq) continue;
      ClusterArgs a;
      memset(&a, 0, sizeof(a));
      a.ca.nlev = L - kd;
      a.ca.dim = 2;
      for (int l = 0; l < a.ca.nlev; ++l) a.ca.lv[l] = lv[kd + l];
      const size_t ca_bytes = coarse_layout(a.ca.off, a.ca.lv, a.ca.nlev, 2);
      const size_t bytes = cluster_layout(a, lv, k1, kd, C, ca_bytes);
      if (bytes > limit) continue;
      // opt in to the device maximum: handles of different sizes must not
      // lower each other's limit
      if (cudaFuncSetAttribute(k_cluster2d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit) != cudaSuccess)
        continue;
      if (C > 8 && cudaFuncSetAttribute(k_cluster2d, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        continue;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(C);
      cfg.blockDim = dim3(kCT);
      cfg.dynamicSmemBytes = bytes;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, k_cluster2d, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        break;  // this cluster size cannot run: try the next one
      }
      *out = a;
      *k1_out = k1;
      *kd_out = kd;
      *smem_out = bytes;
      *ca_bytes_out = ca_bytes;
      return true;
    }
  }
  cudaGetLastError();
  return false;
}

// The whole solve in one cluster: level 0 and the levels below it down to
// kd - 1 distributable (kd chosen as for the middle levels), level 0's CG
// vectors (two p buffers, d) and the reduction slots beside them.
bool cluster_pcg2d_plan(const LevelDev* lv, int L, int kc, ClusterPcgArgs* out, int* kd_out, size_t* smem_out,
                        size_t* ca_bytes_out) {
  if (getenv("NPMG_NO_CLUSTER_PCG") || kc < 1 || L < 2) return false;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  // the kernel's static shared memory (two solve states, sums) and slack
  const size_t limit = (size_t)optin - 4096;
  const size_t thr = cluster_coarse_cells();
  for (int C : {16, 8}) {
    if (!distributable(lv[0], C)) continue;
    int kq = 0;
    while (kq < L - 1 && distributable(lv[kq], C)) ++kq;
    int kd = std::max(1, kc);
    while (kd < kq && (size_t)lv[kd].nx * lv[kd].ny > thr) ++kd;
    if (kd > kq) continue;
    ClusterPcgArgs pa;
    memset(&pa, 0, sizeof(pa));
    ClusterArgs& a = pa.a;
    a.ca.nlev = L - kd;
    a.ca.dim = 2;
    for (int l = 0; l < a.ca.nlev; ++l) a.ca.lv[l] = lv[kd + l];
    const size_t ca_bytes = coarse_layout(a.ca.off, a.ca.lv, a.ca.nlev, 2);
    const size_t P = (size_t)(lv[0].ny / C + 2) * (lv[0].nx + 2 * kG);
    int xoff = 0;
    const size_t bytes = cluster_layout(a, lv, 0, kd, C, ca_bytes, 3 * P + 64, &xoff);
    if (bytes > limit) continue;
    if (cluster_pcg2d_fit(bytes, limit, C) < 1) continue;
    pa.pcg_off = xoff;
    pa.red_off = xoff + (int)(3 * P);
    *out = pa;
    *kd_out = kd;
    *smem_out = bytes;
    *ca_bytes_out = ca_bytes;
    return true;
  }
  cudaGetLastError();
  return false;
}

cudaError_t launch_cluster2d(const ClusterArgs& a, size_t smem, const float* bin, float* yout, float* bkc,
                             float* ykc, SolveState* st, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.C);
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = a.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = chain_launch_enabled() ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, k_cluster2d, a, bin, yout, bkc, ykc, st);
}

}  // namespace npmg

