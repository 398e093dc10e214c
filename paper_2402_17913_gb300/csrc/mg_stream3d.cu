// 3D level kernels with two Jacobi sweeps, streamed along z (2.5D temporal
// blocking).
//
// A block owns a 64 x 16 column of cells and walks a run of z-planes.  The
// two sweeps and the residual of one output plane need the input planes one
// and two away in z, so the block keeps three-plane rings in shared memory
// and works with a skew: when plane p arrives it computes the first sweep's
// result there (pointwise on the down leg, which starts from zero), the
// second sweep on plane p - 1 and the residual (down) or output (up) on
// plane p - 2.  Each input plane is read once per run (plus a 2-cell halo in
// x and y, and two planes at each end of the run), instead of the 2.5x
// re-reads of cube tiles with halos on every side.  The next plane's global
// loads are issued into registers before the current plane's arithmetic.
//
// Same arithmetic as k_down / k_up in mg_kernels.cuh: weighted Jacobi
// (Eq. Jacobi-1-relax) from a zero guess on the down leg, residual and
// 2x2x2 average restriction (App. B), copy prolongation plus scaled
// correction and two post sweeps on the up leg (Sec. 2.2), (r, z) and CG's
// beta on the finest level.
#include <algorithm>
#include <type_traits>

#include "launch.h"
#include "mg_kernels.cuh"

namespace npmg {

namespace {

constexpr int SX = 64, SY = 16;             // output cells of a block per plane
constexpr int RX = SX + 4, RY = SY + 4;     // region with a 2-cell halo (68 x 20)
constexpr int RN = RX * RY;
constexpr int TN = SX * SY;
constexpr int BY = 4;                        // thread rows: RX x BY working threads
constexpr int NW = RX * BY;                  // 272 working threads
constexpr int NT = 288;                      // block: 9 full warps (the last 16 threads only sync and reduce)
constexpr int KA = RY / BY;                  // region rows per thread (5)
static_assert(RY % BY == 0 && SY % BY == 0, "rows split evenly");

// Per-thread geometry: the thread owns region column tx (global x = gx) and
// rows ty, ty + 4, ...; per row the in-plane offset of the cell (-1 outside
// the domain), of its coarse parent, and the x + y part of the unmasked
// diagonal, all fixed for the whole run.
struct Col {
  int tx, ty, gx, z0, z1, y0;
  bool on;  // a working thread
  int off[KA], coff[KA];
  float dxy[KA];
};

__device__ __forceinline__ Col col_of(const LevelDev& L, int zr) {
  Col c;
  c.on = threadIdx.x < NW;
  c.tx = c.on ? (int)threadIdx.x % RX : 0;
  c.ty = c.on ? (int)threadIdx.x / RX : 0;
  c.gx = blockIdx.x * SX - 2 + c.tx;
  c.y0 = blockIdx.y * SY;
  c.z0 = blockIdx.z * zr;
  c.z1 = min(c.z0 + zr, L.nz);
  const bool xs = c.on && c.gx >= 0 && c.gx < L.nx;
  const float dxx = L.wx * (float)axis_count(c.gx, L.nx, L.bcD, 0);
#pragma unroll
  for (int k = 0; k < KA; ++k) {
    const int gy = c.y0 - 2 + c.ty + BY * k;
    const bool in = xs && gy >= 0 && gy < L.ny;
    c.off[k] = in ? gy * L.nx + c.gx : -1;
    c.coff[k] = in ? (gy >> 1) * (L.nx >> 1) + (c.gx >> 1) : 0;
    c.dxy[k] = in ? dxx + L.wy * (float)axis_count(gy, L.ny, L.bcD, 2) : 0.f;
  }
  return c;
}

// One plane of this thread's region cells in registers.
struct PlaneRegs {
  float a[KA];   // b (down) or x + s P e (up)
  float bb[KA];  // b (up only)
  uint8_t m[KA];
};

template <typename TB, bool MASKED>
__device__ __forceinline__ void fetch_down(const LevelDev& L, const Col& c, int p, const TB* __restrict__ b,
                                           PlaneRegs& r) {
  const bool zin = p >= 0 && p < L.nz;
  const size_t base = (size_t)(zin ? p : 0) * L.ny * L.nx;
  const TB* bp = b + base;
  const uint8_t* mp = MASKED ? L.cell + base : nullptr;
#pragma unroll
  for (int k = 0; k < KA; ++k) {
    r.a[k] = 0.f;
    r.m[k] = 0;
    if (zin && c.off[k] >= 0) {
      const uint8_t m = MASKED ? mp[c.off[k]] : kFluidBit;
      r.m[k] = m;
      if (m) r.a[k] = ld(bp, c.off[k]);
    }
  }
}

template <typename T, typename TB, bool MASKED>
__device__ __forceinline__ void fetch_up(const LevelDev& L, const Col& c, int p, const TB* __restrict__ b,
                                         const T* __restrict__ xin, const T* __restrict__ e, float s,
                                         PlaneRegs& r) {
  const bool zin = p >= 0 && p < L.nz;
  const size_t base = (size_t)(zin ? p : 0) * L.ny * L.nx;
  const TB* bp = b + base;
  const T* xp = xin + base;
  const T* ep = e + (size_t)(zin ? p >> 1 : 0) * (L.ny >> 1) * (L.nx >> 1);
  const uint8_t* mp = MASKED ? L.cell + base : nullptr;
#pragma unroll
  for (int k = 0; k < KA; ++k) {
    r.a[k] = 0.f;
    r.bb[k] = 0.f;
    r.m[k] = 0;
    if (zin && c.off[k] >= 0) {
      const uint8_t m = MASKED ? mp[c.off[k]] : kFluidBit;
      r.m[k] = m;
      if (m) {
        r.a[k] = ld(xp, c.off[k]) + s * ld(ep, c.coff[k]);
        r.bb[k] = ld(bp, c.off[k]);
      }
    }
  }
}

__device__ __forceinline__ int slot3(int p) { return (p + 3) % 3; }  // p >= -2

// omega / d through the hardware's approximate reciprocal (a couple of ulps
// from a division; the level kernels are compared to the oracle at 1e-5)
__device__ __forceinline__ float omega_over(float omega, float d) { return __fdividef(omega, d); }

// Diagonal of region row k of plane p for this thread (0 off the fluid);
// dz is the plane's z part of the unmasked diagonal.
template <bool MASKED>
__device__ __forceinline__ float diag_k(const LevelDev& L, const Col& c, int k, uint8_t m, float dz) {
  if (!m) return 0.f;
  if (MASKED) return L.wx * (float)(m & 3) + L.wy * (float)((m >> 2) & 3) + L.wz * (float)((m >> 4) & 3);
  return c.dxy[k] + dz;
}

// Weighted neighbour sum at region index i of the middle plane Xc
// (neighbours in x, y from Xc, in z from Xm / Xp).
__device__ __forceinline__ float nbsum(const LevelDev& L, const float* Xm, const float* Xc, const float* Xp, int i) {
  return L.wx * (Xc[i - 1] + Xc[i + 1]) + L.wy * (Xc[i - RX] + Xc[i + RX]) + L.wz * (Xm[i] + Xp[i]);
}

// b - (d x - nb) at region index i of the middle plane Xc.
__device__ __forceinline__ float defect(const LevelDev& L, const float* Xm, const float* Xc, const float* Xp,
                                        float bv, float d, int i) {
  const float nb = L.wx * (Xc[i - 1] + Xc[i + 1]) + L.wy * (Xc[i - RX] + Xc[i + RX]) + L.wz * (Xm[i] + Xp[i]);
  return bv - (d * Xc[i] - nb);
}

}  // namespace

// Down leg: x = two sweeps from zero, bcoarse = R (b - A' x).
template <typename T, bool MASKED, typename TB>
__global__ void __launch_bounds__(NT, 3) k_down_s3(LevelDev L, const TB* __restrict__ b, T* __restrict__ x,
                                               T* __restrict__ bcoarse, float omega, int zr,
                                               const SolveState* __restrict__ st) {
  chain_enter();
  if (st && st->inner_done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sB = reinterpret_cast<float*>(smem_raw);  // [3][RN]
  float* sD = sB + 3 * RN;                           // [3][RN] diagonal, 0 off the fluid
  float* s1 = sD + 3 * RN;                           // [3][RN] first sweep
  float* s2 = s1 + 3 * RN;                           // [3][RN] second sweep
  float* sR = s2 + 3 * RN;                           // [2][TN] residual
  const Col c = col_of(L, zr);
  const int tid = threadIdx.x;
  PlaneRegs nxt;
  fetch_down<TB, MASKED>(L, c, c.z0 - 2, b, nxt);
  for (int p = c.z0 - 2; p <= c.z1 + 1; ++p) {
    // stage A: plane p into the rings; the first sweep from zero is pointwise
    {
      const int sl = slot3(p) * RN;
      const float dz = L.wz * (float)axis_count(p, L.nz, L.bcD, 4);
#pragma unroll
      for (int k = 0; k < KA; ++k) {
        if (!c.on) break;
        const int i = (c.ty + BY * k) * RX + c.tx;
        const float d = diag_k<MASKED>(L, c, k, nxt.m[k], dz);
        sB[sl + i] = nxt.a[k];
        sD[sl + i] = d;
        s1[sl + i] = d > 0.f ? omega_over(omega, d) * nxt.a[k] : 0.f;
      }
    }
    if (p + 1 <= c.z1 + 1) fetch_down<TB, MASKED>(L, c, p + 1, b, nxt);
    __syncthreads();
    // stage B: second sweep on plane q = p - 1, region less one cell
    const int q = p - 1;
    if (q >= c.z0 - 1 && c.on && c.tx >= 1 && c.tx <= RX - 2) {
      const float* Xm = s1 + slot3(q - 1) * RN;
      const float* Xc = s1 + slot3(q) * RN;
      const float* Xp = s1 + slot3(q + 1) * RN;
      const int sq = slot3(q) * RN;
#pragma unroll
      for (int k = 0; k < KA; ++k) {
        const int ly = 1 + c.ty + BY * k;
        if (ly <= RY - 2) {
          const int i = ly * RX + c.tx;
          const float d = sD[sq + i];
          s2[sq + i] = d > 0.f ? Xc[i] + omega_over(omega, d) * defect(L, Xm, Xc, Xp, sB[sq + i], d, i) : 0.f;
        }
      }
    }
    __syncthreads();
    // stage C: x and the residual on plane o = p - 2 (the tile)
    const int o = p - 2;
    if (o >= c.z0 && o < c.z1 && c.on && c.tx >= 2 && c.tx <= RX - 3) {
      const float* Xm = s2 + slot3(o - 1) * RN;
      const float* Xc = s2 + slot3(o) * RN;
      const float* Xp = s2 + slot3(o + 1) * RN;
      const int so = slot3(o) * RN;
      float* R = sR + (o & 1) * TN;
      const size_t base = (size_t)o * L.ny * L.nx + c.gx;
#pragma unroll
      for (int k = 0; k < SY / BY; ++k) {
        const int ly = 2 + c.ty + BY * k, i = ly * RX + c.tx;
        const int gy = c.y0 + ly - 2;
        const float d = sD[so + i];
        R[(ly - 2) * SX + c.tx - 2] = d > 0.f ? defect(L, Xm, Xc, Xp, sB[so + i], d, i) : 0.f;
        if (c.gx < L.nx && gy < L.ny) x[base + (size_t)gy * L.nx] = cvt<T>(Xc[i]);
      }
    }
    __syncthreads();
    // restriction of the plane pair (o - 1, o) when o is odd
    if (o >= c.z0 && o < c.z1 && (o & 1) && tid < (SX / 2) * (SY / 2)) {
      const int cx = tid % (SX / 2), cy = tid / (SX / 2);
      const int gcx = blockIdx.x * (SX / 2) + cx, gcy = c.y0 / 2 + cy;
      if (gcx < L.nx / 2 && gcy < L.ny / 2) {
        float sum = 0.f;
#pragma unroll
        for (int az = 0; az < 2; ++az)
#pragma unroll
          for (int ay = 0; ay < 2; ++ay)
#pragma unroll
            for (int ax = 0; ax < 2; ++ax) sum += sR[az * TN + (2 * cy + ay) * SX + 2 * cx + ax];
        const size_t ci = ((size_t)(o >> 1) * (L.ny / 2) + gcy) * (L.nx / 2) + gcx;
        bcoarse[ci] = cvt<T>(sum * 0.125f);
      }
    }
  }
}

// Up leg: xout = two sweeps from x + s P e; on the finest level (r, z) and
// CG's beta.
template <typename T, bool MASKED, bool FINEST, typename TB>
__global__ void __launch_bounds__(NT, 3) k_up_s3(LevelDev L, const TB* __restrict__ b, const T* __restrict__ xin,
                                             TB* __restrict__ xout, const T* __restrict__ e, float omega, float s,
                                             int zr, SolveState* __restrict__ st, double* __restrict__ partials) {
  chain_enter();
  if (st && st->inner_done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sB = reinterpret_cast<float*>(smem_raw);  // [3][RN]
  float* sW = sB + 3 * RN;                           // [3][RN] omega / d, 0 off the fluid
  float* s0 = sW + 3 * RN;                           // [3][RN] x + s P e
  float* s1 = s0 + 3 * RN;                           // [3][RN] first sweep
  const Col c = col_of(L, zr);
  const float keep = 1.f - omega;  // x + (omega/d)(b - d x + nb) = (1 - omega) x + (omega/d)(b + nb)
  float acc = 0.f;
  PlaneRegs nxt;
  fetch_up<T, TB, MASKED>(L, c, c.z0 - 2, b, xin, e, s, nxt);
  for (int p = c.z0 - 2; p <= c.z1 + 1; ++p) {
    {
      const int sl = slot3(p) * RN;
      const float dz = L.wz * (float)axis_count(p, L.nz, L.bcD, 4);
#pragma unroll
      for (int k = 0; k < KA; ++k) {
        if (!c.on) break;
        const int i = (c.ty + BY * k) * RX + c.tx;
        const float d = diag_k<MASKED>(L, c, k, nxt.m[k], dz);
        sB[sl + i] = nxt.bb[k];
        sW[sl + i] = d > 0.f ? omega_over(omega, d) : 0.f;
        s0[sl + i] = nxt.a[k];
      }
    }
    if (p + 1 <= c.z1 + 1) fetch_up<T, TB, MASKED>(L, c, p + 1, b, xin, e, s, nxt);
    __syncthreads();
    const int q = p - 1;
    if (q >= c.z0 - 1 && c.on && c.tx >= 1 && c.tx <= RX - 2) {
      const float* Xm = s0 + slot3(q - 1) * RN;
      const float* Xc = s0 + slot3(q) * RN;
      const float* Xp = s0 + slot3(q + 1) * RN;
      const int sq = slot3(q) * RN;
#pragma unroll
      for (int k = 0; k < KA; ++k) {
        const int ly = 1 + c.ty + BY * k;
        if (ly <= RY - 2) {
          const int i = ly * RX + c.tx;
          const float w = sW[sq + i];
          s1[sq + i] = w > 0.f ? keep * Xc[i] + w * (sB[sq + i] + nbsum(L, Xm, Xc, Xp, i)) : 0.f;
        }
      }
    }
    __syncthreads();
    const int o = p - 2;
    if (o >= c.z0 && o < c.z1 && c.on && c.tx >= 2 && c.tx <= RX - 3 && c.gx < L.nx) {
      const float* Xm = s1 + slot3(o - 1) * RN;
      const float* Xc = s1 + slot3(o) * RN;
      const float* Xp = s1 + slot3(o + 1) * RN;
      const int so = slot3(o) * RN;
      const size_t base = (size_t)o * L.ny * L.nx + c.gx;
#pragma unroll
      for (int k = 0; k < SY / BY; ++k) {
        const int ly = 2 + c.ty + BY * k, i = ly * RX + c.tx;
        const int gy = c.y0 + ly - 2;
        if (gy < L.ny) {
          const float w = sW[so + i], bv = sB[so + i];
          const float v = w > 0.f ? keep * Xc[i] + w * (bv + nbsum(L, Xm, Xc, Xp, i)) : 0.f;
          const TB zt = cvt<TB>(v);
          xout[base + (size_t)gy * L.nx] = zt;
          if (FINEST) acc = fmaf(bv, ld(&zt, 0), acc);
        }
      }
    }
    // the next plane's stage A overwrites slot3(p + 1) = slot3(o): every
    // read of plane o ends before this barrier
    __syncthreads();
  }
  if (FINEST) {
    double tot;
    if (grid_sum_last((double)acc, partials, &st->counter[kCntRZ], &tot)) {
      if (threadIdx.x == 0) {
        st->rz = tot;
        st->beta = (st->first || !st->krylov) ? 0.0 : tot / st->rz_old;
        st->rz_old = tot;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// host side
static int device_sms();
static size_t s3_smem_down();
static int s3_run(const LevelDev& L, int nsm, int per_sm);

bool stream3d_eligible(int dim, int pre, int post, const LevelDev& L) {
  return dim == 3 && pre == 2 && post == 2 && L.nz >= 8 && (L.nz % 2) == 0 && (L.nx % 2) == 0 &&
         (L.ny % 2) == 0 && s3_run(L, device_sms(), 3) > 0;
}

static size_t s3_smem_down() { return (size_t)(12 * RN + 2 * TN) * sizeof(float); }
static size_t s3_smem_up() { return (size_t)(12 * RN) * sizeof(float); }

// Resident blocks of a streaming kernel per SM (shared memory, registers,
// threads).
template <typename K>
static int s3_per_sm(K kernel, size_t smem) {
  int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0, thr_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  int per = (int)((size_t)smem_sm / (smem + 512 + (size_t)reserved));
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess && fa.numRegs > 0) {
    const int regs_block = ((fa.numRegs * 32 + 255) / 256) * 256 * (NT / 32);
    per = std::min(per, regs_sm / regs_block);
  }
  per = std::min(per, thr_sm / NT);
  return per < 1 ? 1 : per;
}

// z-run length: even, so that the grid is about one wave of resident blocks
// (0 when the level is too small for runs of at least 4 planes to cover
// every SM; the cube-tile kernels take those levels)
static int s3_run(const LevelDev& L, int nsm, int per_sm) {
  const int tiles = ((L.nx + SX - 1) / SX) * ((L.ny + SY - 1) / SY);
  int runs = std::max(1, nsm * per_sm / tiles);
  runs = std::min(runs, std::max(1, L.nz / 4));  // runs of at least 4 planes
  int zr = (L.nz + runs - 1) / runs;
  zr = ((zr + 1) / 2) * 2;
  // more resident blocks only lengthen the grid, so eligibility checked
  // with 2 blocks per SM holds for every launch
  if (tiles * ((L.nz + zr - 1) / zr) < nsm) return 0;
  return zr;
}

static dim3 s3_grid(const LevelDev& L, int zr) {
  return dim3((L.nx + SX - 1) / SX, (L.ny + SY - 1) / SY, (L.nz + zr - 1) / zr);
}

static int device_sms() {
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  return nsm;
}

template <typename T, bool MASKED, typename TB>
cudaError_t launch_down_s3(const LevelDev& L, const void* b, void* x, void* bcoarse, float omega,
                           const SolveState* st, cudaStream_t s) {
  static const int per = s3_per_sm(k_down_s3<T, MASKED, TB>, s3_smem_down());
  const int zr = s3_run(L, device_sms(), per);
  if (zr <= 0) return cudaErrorInvalidValue;
  return launch_chain(k_down_s3<T, MASKED, TB>, s3_grid(L, zr), NT, s3_smem_down(), s, L, (const TB*)b, (T*)x,
                      (T*)bcoarse, omega, zr, st);
}

template <typename T, bool MASKED, bool FINEST, typename TB>
cudaError_t launch_up_s3(const LevelDev& L, const void* b, const void* xin, void* xout, const void* e, float omega,
                         float sc, SolveState* st, double* partials, cudaStream_t s) {
  static const int per = s3_per_sm(k_up_s3<T, MASKED, FINEST, TB>, s3_smem_up());
  const int zr = s3_run(L, device_sms(), per);
  if (zr <= 0) return cudaErrorInvalidValue;
  return launch_chain(k_up_s3<T, MASKED, FINEST, TB>, s3_grid(L, zr), NT, s3_smem_up(), s, L, (const TB*)b,
                      (const T*)xin, (TB*)xout, (const T*)e, omega, sc, zr, st, partials);
}

template <typename T, bool MASKED, typename TB>
static cudaError_t prepare_s3_pair() {
  cudaError_t e = cudaFuncSetAttribute(k_down_s3<T, MASKED, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)s3_smem_down());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_up_s3<T, MASKED, false, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)s3_smem_up());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_up_s3<T, MASKED, true, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)s3_smem_up());
  return e;
}

template <typename T, bool MASKED>
cudaError_t prepare_s3_kernels() {
  cudaError_t e = prepare_s3_pair<T, MASKED, T>();
  if (e == cudaSuccess && !std::is_same<T, float>::value) e = prepare_s3_pair<T, MASKED, float>();
  return e;
}

#define NPMG_INST_S3_TB(T, M, TB)                                                                                \
  template cudaError_t launch_down_s3<T, M, TB>(const LevelDev&, const void*, void*, void*, float,                \
                                                const SolveState*, cudaStream_t);                                \
  template cudaError_t launch_up_s3<T, M, false, TB>(const LevelDev&, const void*, const void*, void*,            \
                                                     const void*, float, float, SolveState*, double*, cudaStream_t); \
  template cudaError_t launch_up_s3<T, M, true, TB>(const LevelDev&, const void*, const void*, void*,             \
                                                    const void*, float, float, SolveState*, double*, cudaStream_t);
#define NPMG_INST_S3(T, M)                      \
  template cudaError_t prepare_s3_kernels<T, M>(); \
  NPMG_INST_S3_TB(T, M, T)                      \
  NPMG_INST_S3_TB(T, M, float)

template cudaError_t prepare_s3_kernels<float, false>();
template cudaError_t prepare_s3_kernels<float, true>();
NPMG_INST_S3_TB(float, false, float)
NPMG_INST_S3_TB(float, true, float)
NPMG_INST_S3(__half, false)
NPMG_INST_S3(__half, true)
NPMG_INST_S3(__nv_bfloat16, false)
NPMG_INST_S3(__nv_bfloat16, true)

}  // namespace npmg
