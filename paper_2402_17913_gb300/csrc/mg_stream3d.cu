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
#include "launch.h"
#include "mg_kernels.cuh"

namespace npmg {

namespace {

constexpr int SX = 64, SY = 16;             // output cells of a block per plane
constexpr int RX = SX + 4, RY = SY + 4;     // region with a 2-cell halo
constexpr int RN = RX * RY;                 // 1360
constexpr int QX = SX + 2, QY = SY + 2;     // second-stage region (1-cell halo)
constexpr int QN = QX * QY;                 // 1188
constexpr int TN = SX * SY;                 // 1024
constexpr int NT = 256;                     // threads
constexpr int LPT = (RN + NT - 1) / NT;     // region cells loaded per thread (6)

struct Geo {
  int x0, y0, z0, z1;  // output column origin and z-run [z0, z1)
};

__device__ __forceinline__ Geo geo_of(const LevelDev& L, int zr) {
  Geo g;
  g.x0 = blockIdx.x * SX;
  g.y0 = blockIdx.y * SY;
  g.z0 = blockIdx.z * zr;
  g.z1 = min(g.z0 + zr, L.nz);
  return g;
}

// Registers holding one plane of the region for this thread.
template <typename T>
struct PlaneRegs {
  float a[LPT];      // b (down) or x + s P e (up)
  float bb[LPT];     // b (up only)
  uint8_t m[LPT];
};

// Global loads of plane p (down leg: b and the cell bytes).
template <typename T, bool MASKED>
__device__ __forceinline__ void fetch_down(const LevelDev& L, const Geo& g, int p, const T* __restrict__ b,
                                           PlaneRegs<T>& r) {
#pragma unroll
  for (int k = 0; k < LPT; ++k) {
    const int i = threadIdx.x + k * NT;
    r.a[k] = 0.f;
    r.m[k] = 0;
    if (i < RN && p >= 0 && p < L.nz) {
      const int gx = g.x0 - 2 + i % RX, gy = g.y0 - 2 + i / RX;
      if (gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny) {
        const size_t gi = gidx(L, gx, gy, p);
        const uint8_t m = MASKED ? L.cell[gi] : kFluidBit;
        r.m[k] = m;
        if (m) r.a[k] = ld(b, gi);
      }
    }
  }
}

// Global loads of plane p (up leg: x + s e_coarse, b, the cell bytes).
template <typename T, bool MASKED>
__device__ __forceinline__ void fetch_up(const LevelDev& L, const Geo& g, int p, const T* __restrict__ b,
                                         const T* __restrict__ xin, const T* __restrict__ e, float s,
                                         PlaneRegs<T>& r) {
  const int cnx = L.nx / 2, cny = L.ny / 2;
#pragma unroll
  for (int k = 0; k < LPT; ++k) {
    const int i = threadIdx.x + k * NT;
    r.a[k] = 0.f;
    r.bb[k] = 0.f;
    r.m[k] = 0;
    if (i < RN && p >= 0 && p < L.nz) {
      const int gx = g.x0 - 2 + i % RX, gy = g.y0 - 2 + i / RX;
      if (gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny) {
        const size_t gi = gidx(L, gx, gy, p);
        const uint8_t m = MASKED ? L.cell[gi] : kFluidBit;
        r.m[k] = m;
        if (m) {
          const size_t ci = ((size_t)(p >> 1) * cny + (gy >> 1)) * cnx + (gx >> 1);
          r.a[k] = ld(xin, gi) + s * ld(e, ci);
          r.bb[k] = ld(b, gi);
        }
      }
    }
  }
}

__device__ __forceinline__ int slot3(int p) { return (p + 3) % 3; }  // p >= -2

// One weighted-Jacobi update at region index i of plane q from the ring of
// iterates X (planes q-1, q, q+1 in slots), b and the diagonal.
__device__ __forceinline__ float jacobi_at(const LevelDev& L, const float* Xm, const float* Xc, const float* Xp,
                                           float bv, float d, float wd, int i) {
  const float xc = Xc[i];
  const float nb = L.wx * (Xc[i - 1] + Xc[i + 1]) + L.wy * (Xc[i - RX] + Xc[i + RX]) + L.wz * (Xm[i] + Xp[i]);
  return xc + wd * (bv - (d * xc - nb));
}

// omega / d as omega times the correctly rounded reciprocal (one rounding
// more than a division; the sweeps' results move by at most an ulp)
__device__ __forceinline__ float omega_over(float omega, float d) { return omega * __frcp_rn(d); }

}  // namespace

// Down leg: x = two sweeps from zero, bcoarse = R (b - A' x).
template <typename T, bool MASKED>
__global__ void __launch_bounds__(NT) k_down_s3(LevelDev L, const T* __restrict__ b, T* __restrict__ x,
                                               T* __restrict__ bcoarse, float omega, int zr,
                                               const SolveState* __restrict__ st) {
  if (st && st->inner_done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sB = reinterpret_cast<float*>(smem_raw);  // [3][RN]
  float* sD = sB + 3 * RN;                           // [3][RN] diagonal, 0 off the fluid
  float* s1 = sD + 3 * RN;                           // [3][RN] first sweep
  float* s2 = s1 + 3 * RN;                           // [3][RN] second sweep
  float* sR = s2 + 3 * RN;                           // [2][TN] residual
  const Geo g = geo_of(L, zr);
  const int tid = threadIdx.x;
  PlaneRegs<T> nxt;
  fetch_down<T, MASKED>(L, g, g.z0 - 2, b, nxt);
  for (int p = g.z0 - 2; p <= g.z1 + 1; ++p) {
    // stage A: plane p into the rings; first sweep from zero is pointwise
    {
      const int sl = slot3(p);
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int i = tid + k * NT;
        if (i < RN) {
          const int gx = g.x0 - 2 + i % RX, gy = g.y0 - 2 + i / RX;
          const float d = nxt.m[k] ? diag_at<3, MASKED>(L, gx, gy, p, nxt.m[k]) : 0.f;
          sB[sl * RN + i] = nxt.a[k];
          sD[sl * RN + i] = d;
          s1[sl * RN + i] = d > 0.f ? omega_over(omega, d) * nxt.a[k] : 0.f;
        }
      }
    }
    if (p + 1 <= g.z1 + 1) fetch_down<T, MASKED>(L, g, p + 1, b, nxt);
    __syncthreads();
    // stage B: second sweep on plane q = p - 1 (region less one cell)
    const int q = p - 1;
    if (q >= g.z0 - 1) {
      const float* Xm = s1 + slot3(q - 1) * RN;
      const float* Xc = s1 + slot3(q) * RN;
      const float* Xp = s1 + slot3(q + 1) * RN;
      const int sq = slot3(q);
      for (int j = tid; j < QN; j += NT) {
        const int i = (1 + j / QX) * RX + 1 + j % QX;
        const float d = sD[sq * RN + i];
        s2[sq * RN + i] = d > 0.f ? jacobi_at(L, Xm, Xc, Xp, sB[sq * RN + i], d, omega_over(omega, d), i) : 0.f;
      }
    }
    __syncthreads();
    // stage C: x and the residual on plane o = p - 2 (the tile)
    const int o = p - 2;
    if (o >= g.z0 && o < g.z1) {
      const float* Xm = s2 + slot3(o - 1) * RN;
      const float* Xc = s2 + slot3(o) * RN;
      const float* Xp = s2 + slot3(o + 1) * RN;
      const int so = slot3(o);
      float* R = sR + (o & 1) * TN;
      for (int c = tid; c < TN; c += NT) {
        const int lx = 2 + c % SX, ly = 2 + c / SX, i = ly * RX + lx;
        const int gx = g.x0 + lx - 2, gy = g.y0 + ly - 2;
        const float d = sD[so * RN + i];
        const float xc = Xc[i];
        float r = 0.f;
        if (d > 0.f) {
          const float nb =
              L.wx * (Xc[i - 1] + Xc[i + 1]) + L.wy * (Xc[i - RX] + Xc[i + RX]) + L.wz * (Xm[i] + Xp[i]);
          r = sB[so * RN + i] - (d * xc - nb);
        }
        R[c] = r;
        if (gx < L.nx && gy < L.ny) x[gidx(L, gx, gy, o)] = cvt<T>(xc);
      }
    }
    __syncthreads();
    // restriction of the plane pair (o - 1, o) when o is odd
    if (o >= g.z0 && o < g.z1 && (o & 1)) {
      const int cx = tid % (SX / 2), cy = tid / (SX / 2);  // 32 x 8 coarse cells, one per thread
      const int gcx = g.x0 / 2 + cx, gcy = g.y0 / 2 + cy;
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
template <typename T, bool MASKED, bool FINEST>
__global__ void __launch_bounds__(NT) k_up_s3(LevelDev L, const T* __restrict__ b, const T* __restrict__ xin,
                                             T* __restrict__ xout, const T* __restrict__ e, float omega, float s,
                                             int zr, SolveState* __restrict__ st, double* __restrict__ partials) {
  if (st && st->inner_done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sB = reinterpret_cast<float*>(smem_raw);  // [3][RN]
  float* sD = sB + 3 * RN;                           // [3][RN]
  float* s0 = sD + 3 * RN;                           // [3][RN] x + s P e
  float* s1 = s0 + 3 * RN;                           // [3][RN] first sweep
  const Geo g = geo_of(L, zr);
  const int tid = threadIdx.x;
  float acc = 0.f;
  PlaneRegs<T> nxt;
  fetch_up<T, MASKED>(L, g, g.z0 - 2, b, xin, e, s, nxt);
  for (int p = g.z0 - 2; p <= g.z1 + 1; ++p) {
    {
      const int sl = slot3(p);
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const int i = tid + k * NT;
        if (i < RN) {
          const int gx = g.x0 - 2 + i % RX, gy = g.y0 - 2 + i / RX;
          sB[sl * RN + i] = nxt.bb[k];
          sD[sl * RN + i] = nxt.m[k] ? diag_at<3, MASKED>(L, gx, gy, p, nxt.m[k]) : 0.f;
          s0[sl * RN + i] = nxt.a[k];
        }
      }
    }
    if (p + 1 <= g.z1 + 1) fetch_up<T, MASKED>(L, g, p + 1, b, xin, e, s, nxt);
    __syncthreads();
    const int q = p - 1;
    if (q >= g.z0 - 1) {
      const float* Xm = s0 + slot3(q - 1) * RN;
      const float* Xc = s0 + slot3(q) * RN;
      const float* Xp = s0 + slot3(q + 1) * RN;
      const int sq = slot3(q);
      for (int j = tid; j < QN; j += NT) {
        const int i = (1 + j / QX) * RX + 1 + j % QX;
        const float d = sD[sq * RN + i];
        s1[sq * RN + i] = d > 0.f ? jacobi_at(L, Xm, Xc, Xp, sB[sq * RN + i], d, omega_over(omega, d), i) : 0.f;
      }
    }
    __syncthreads();
    const int o = p - 2;
    if (o >= g.z0 && o < g.z1) {
      const float* Xm = s1 + slot3(o - 1) * RN;
      const float* Xc = s1 + slot3(o) * RN;
      const float* Xp = s1 + slot3(o + 1) * RN;
      const int so = slot3(o);
      for (int c = tid; c < TN; c += NT) {
        const int lx = 2 + c % SX, ly = 2 + c / SX, i = ly * RX + lx;
        const int gx = g.x0 + lx - 2, gy = g.y0 + ly - 2;
        if (gx < L.nx && gy < L.ny) {
          const float d = sD[so * RN + i];
          const float bv = sB[so * RN + i];
          const float v = d > 0.f ? jacobi_at(L, Xm, Xc, Xp, bv, d, omega_over(omega, d), i) : 0.f;
          const T zt = cvt<T>(v);
          xout[gidx(L, gx, gy, o)] = zt;
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

// Resident blocks of a streaming kernel per SM (shared memory bound).
static int s3_per_sm(size_t smem) {
  int dev = 0, smem_sm = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  const int per = (int)((size_t)smem_sm / (smem + 512 + (size_t)reserved));
  return per < 1 ? 1 : per;
}

// z-run length: even, so that the grid is about one wave of resident blocks
// (0 when the level is too small for runs of at least 8 planes to fill the
// GPU; the cube-tile kernels take those levels)
static int s3_run(const LevelDev& L, int nsm, int per_sm) {
  const int tiles = ((L.nx + SX - 1) / SX) * ((L.ny + SY - 1) / SY);
  const int resident = nsm * per_sm;
  const int runs = resident / tiles;
  if (runs < 1) return ((L.nz + 1) / 2) * 2 >= 8 ? ((L.nz + 1) / 2) * 2 : 0;
  int zr = (L.nz + runs - 1) / runs;
  zr = ((zr + 1) / 2) * 2;
  if (zr < 8 || tiles * ((L.nz + zr - 1) / zr) < nsm) return 0;
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

template <typename T, bool MASKED>
cudaError_t launch_down_s3(const LevelDev& L, const void* b, void* x, void* bcoarse, float omega,
                           const SolveState* st, cudaStream_t s) {
  static const int per = s3_per_sm(s3_smem_down());
  const int zr = s3_run(L, device_sms(), per);
  if (zr <= 0) return cudaErrorInvalidValue;
  k_down_s3<T, MASKED><<<s3_grid(L, zr), NT, s3_smem_down(), s>>>(L, (const T*)b, (T*)x, (T*)bcoarse, omega, zr,
                                                                   st);
  return cudaGetLastError();
}

template <typename T, bool MASKED, bool FINEST>
cudaError_t launch_up_s3(const LevelDev& L, const void* b, const void* xin, void* xout, const void* e, float omega,
                         float sc, SolveState* st, double* partials, cudaStream_t s) {
  static const int per = s3_per_sm(s3_smem_up());
  const int zr = s3_run(L, device_sms(), per);
  if (zr <= 0) return cudaErrorInvalidValue;
  k_up_s3<T, MASKED, FINEST><<<s3_grid(L, zr), NT, s3_smem_up(), s>>>(L, (const T*)b, (const T*)xin, (T*)xout,
                                                                      (const T*)e, omega, sc, zr, st, partials);
  return cudaGetLastError();
}

template <typename T, bool MASKED>
cudaError_t prepare_s3_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_down_s3<T, MASKED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)s3_smem_down());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_up_s3<T, MASKED, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)s3_smem_up());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_up_s3<T, MASKED, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)s3_smem_up());
  return e;
}

#define NPMG_INST_S3(T, M)                                                                                      \
  template cudaError_t launch_down_s3<T, M>(const LevelDev&, const void*, void*, void*, float, const SolveState*, \
                                            cudaStream_t);                                                      \
  template cudaError_t launch_up_s3<T, M, false>(const LevelDev&, const void*, const void*, void*, const void*,  \
                                                 float, float, SolveState*, double*, cudaStream_t);             \
  template cudaError_t launch_up_s3<T, M, true>(const LevelDev&, const void*, const void*, void*, const void*,   \
                                                float, float, SolveState*, double*, cudaStream_t);              \
  template cudaError_t prepare_s3_kernels<T, M>();

NPMG_INST_S3(float, false)
NPMG_INST_S3(float, true)
NPMG_INST_S3(__half, false)
NPMG_INST_S3(__half, true)
NPMG_INST_S3(__nv_bfloat16, false)
NPMG_INST_S3(__nv_bfloat16, true)

}  // namespace npmg
