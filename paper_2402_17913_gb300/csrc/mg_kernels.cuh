// Multigrid level kernels (2D and 3D, templated on storage type).
//
// Notation: A' = c * A_h with c = h_0x^2, so the weights of the paper's
// diffusion filter on level k are w_a = c / h_{k,a}^2 (App. A filters; the
// spacing doubles per level, App. B).  Every vector holds 0 on solid cells
// and outside the domain, which is the zero padding of Sec. 2.1: a
// neighbour outside the domain or solid contributes nothing off the
// diagonal, and the diagonal counts only links that exist (fluid neighbour
// or Dirichlet face).
#pragma once
#include "npmg_internal.cuh"

namespace npmg {

template <int DIM> struct TileShape;
template <> struct TileShape<2> { static constexpr int X = 64, Y = 16, Z = 1; };
template <> struct TileShape<3> { static constexpr int X = 32, Y = 8, Z = 8; };

// Region of a tile plus a halo of H cells on every side (none along z in
// 2D).  HT > 0 fixes the halo at compile time (the default two sweeps), so
// the index arithmetic folds to constants; HT == 0 takes it at run time.
template <int DIM, int HT>
struct Region {
  int H, RX, RY, RZ, R;
  int ox, oy, oz;  // global coordinates of local (0,0,0)
  __device__ __forceinline__ explicit Region(int h_rt) {
    using TS = TileShape<DIM>;
    H = HT > 0 ? HT : h_rt;
    RX = TS::X + 2 * H;
    RY = TS::Y + 2 * H;
    RZ = (DIM == 3) ? TS::Z + 2 * H : 1;
    R = RX * RY * RZ;
    ox = blockIdx.x * TS::X - H;
    oy = blockIdx.y * TS::Y - H;
    oz = (DIM == 3) ? (int)blockIdx.z * TS::Z - H : 0;
  }
  __device__ __forceinline__ int idx(int lx, int ly, int lz) const { return (lz * RY + ly) * RX + lx; }
};

__host__ __device__ inline size_t gidx(const LevelDev& L, int x, int y, int z) {
  return ((size_t)z * L.ny + y) * L.nx + x;
}

template <int DIM>
__device__ __forceinline__ bool inside(const LevelDev& L, int x, int y, int z) {
  return x >= 0 && x < L.nx && y >= 0 && y < L.ny && (DIM == 2 || (z >= 0 && z < L.nz));
}

// Load a field over the region into shared memory (0 outside the domain)
// together with the cell bytes (kFluidBit for an unmasked in-domain cell).
template <int DIM, int HT, typename T, bool MASKED>
__device__ __forceinline__ void load_region(const Region<DIM, HT>& g, const LevelDev& L, const T* __restrict__ f,
                                            float* s, uint8_t* sm) {
  for (int i = threadIdx.x; i < g.R; i += blockDim.x) {
    const int lx = i % g.RX;
    const int t = i / g.RX;
    const int ly = t % g.RY;
    const int lz = t / g.RY;
    const int gx = g.ox + lx, gy = g.oy + ly, gz = g.oz + lz;
    float v = 0.f;
    uint8_t m = 0;
    if (inside<DIM>(L, gx, gy, gz)) {
      const size_t gi = gidx(L, gx, gy, gz);
      m = MASKED ? L.cell[gi] : kFluidBit;
      if (m) v = ld(f, gi);
    }
    s[i] = v;
    sm[i] = m;
  }
}

// One weighted-Jacobi sweep x_out = x_in + omega D^-1 (b - A' x_in) over the
// tile grown by `m` cells (Eq. Jacobi-1-relax); `from_zero` means x_in = 0.
template <int DIM, int HT, bool MASKED>
__device__ __forceinline__ void sweep_region(const Region<DIM, HT>& g, const LevelDev& L, const float* xin,
                                             float* xout, const float* sb, const uint8_t* sm, int m, float omega,
                                             bool from_zero) {
  using TS = TileShape<DIM>;
  const int SX = TS::X + 2 * m, SY = TS::Y + 2 * m, SZ = (DIM == 3) ? TS::Z + 2 * m : 1;
  const int cnt = SX * SY * SZ;
  const int sxy = g.RX * g.RY;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const int sx = i % SX;
    const int t = i / SX;
    const int sy = t % SY;
    const int sz = t / SY;
    const int lx = sx + g.H - m, ly = sy + g.H - m, lz = (DIM == 3) ? sz + g.H - m : 0;
    const int li = g.idx(lx, ly, lz);
    const uint8_t mm = sm[li];
    float v = 0.f;
    if (mm) {
      const float d = diag_at<DIM, MASKED>(L, g.ox + lx, g.oy + ly, g.oz + lz, mm);
      if (from_zero) {
        v = omega * sb[li] / d;
      } else {
        const float xc = xin[li];
        float nb = L.wx * (xin[li - 1] + xin[li + 1]) + L.wy * (xin[li - g.RX] + xin[li + g.RX]);
        if (DIM == 3) nb += L.wz * (xin[li - sxy] + xin[li + sxy]);
        v = xc + omega * (sb[li] - (d * xc - nb)) / d;
      }
    }
    xout[li] = v;
  }
  __syncthreads();
}

// Residual b - A' x at local cell (lx, ly, lz) (fluid assumed).
template <int DIM, int HT, bool MASKED>
__device__ __forceinline__ float residual_at(const Region<DIM, HT>& g, const LevelDev& L, const float* x,
                                             const float* sb, uint8_t mm, int lx, int ly, int lz) {
  const int li = g.idx(lx, ly, lz);
  const int sxy = g.RX * g.RY;
  const float d = diag_at<DIM, MASKED>(L, g.ox + lx, g.oy + ly, g.oz + lz, mm);
  float nb = L.wx * (x[li - 1] + x[li + 1]) + L.wy * (x[li - g.RX] + x[li + g.RX]);
  if (DIM == 3) nb += L.wz * (x[li - sxy] + x[li + sxy]);
  return sb[li] - (d * x[li] - nb);
}

// ---------------------------------------------------------------------------
// Storage types: T for a level's own iterate x, its coarse right-hand side
// and the coarse correction e; TB for the level's right-hand side b and the
// up leg's output (T on every level but the finest, where b and z are the
// float32 CG vectors).
//
// Down leg of one level: `pre` sweeps from x = 0 (the cycle starts every
// level from a zero guess, Sec. 2.2 step list), then r = b - A' x and its
// 2x2(x2) average written to the coarse right-hand side (Sec. 2.2
// restriction filter of 1/4, App. B eight eighths in 3D).  All sweeps of a
// tile run in shared memory (temporal blocking: halo = pre).
template <int DIM, int HT, typename T, bool MASKED, typename TB = T>
__global__ void __launch_bounds__(kThreads)
k_down(LevelDev L, const TB* __restrict__ b, T* __restrict__ x, T* __restrict__ bcoarse, int pre, float omega,
       const SolveState* __restrict__ st) {
  chain_enter();
  if (st && st->inner_done) return;
  using TS = TileShape<DIM>;
  const int pre_c = HT > 0 ? HT : pre;
  const Region<DIM, HT> g(pre_c > 0 ? pre_c : 1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sb = reinterpret_cast<float*>(smem_raw);
  float* s0 = sb + g.R;
  float* s1 = s0 + g.R;
  uint8_t* sm = reinterpret_cast<uint8_t*>(s1 + g.R);
  load_region<DIM, HT, TB, MASKED>(g, L, b, sb, sm);
  __syncthreads();
  float* cur = s0;
  float* nxt = s1;
  // pre_c < 0: the sawtooth down leg (App. B): the residual of x = 0 (that
  // is b) is restricted, and x = b / d (one Jacobi step from zero) is
  // written for the up leg
  if (pre_c <= 0) {
    for (int i = threadIdx.x; i < g.R; i += blockDim.x) s0[i] = 0.f;
    __syncthreads();
  } else {
    sweep_region<DIM, HT, MASKED>(g, L, nullptr, s0, sb, sm, pre_c, omega, true);  // x_1 on T+pre
    for (int j = 2; j <= pre_c; ++j) {
      sweep_region<DIM, HT, MASKED>(g, L, cur, nxt, sb, sm, pre_c - j + 1, omega, false);
      float* t = cur; cur = nxt; nxt = t;
    }
  }
  // write x on the tile
  constexpr int TN = TS::X * TS::Y * TS::Z;
  for (int i = threadIdx.x; i < TN; i += blockDim.x) {
    const int tx = i % TS::X;
    const int t = i / TS::X;
    const int ty = t % TS::Y;
    const int tz = t / TS::Y;
    const int lx = tx + g.H, ly = ty + g.H, lz = (DIM == 3) ? tz + g.H : 0;
    const int gx = g.ox + lx, gy = g.oy + ly, gz = g.oz + lz;
    if (inside<DIM>(L, gx, gy, gz)) {
      const int li = g.idx(lx, ly, lz);
      float v = cur[li];
      if (pre_c < 0) {
        const uint8_t mm = sm[li];
        v = mm ? sb[li] / diag_at<DIM, MASKED>(L, gx, gy, gz, mm) : 0.f;
      }
      x[gidx(L, gx, gy, gz)] = cvt<T>(v);
    }
  }
  // residual and restriction to the coarse right-hand side
  constexpr int CX = TS::X / 2, CY = TS::Y / 2, CZ = (DIM == 3) ? TS::Z / 2 : 1;
  LevelDev C;
  C.nx = L.nx / 2; C.ny = L.ny / 2; C.nz = (DIM == 3) ? L.nz / 2 : 1;
  const float inv_children = (DIM == 3) ? 0.125f : 0.25f;
  for (int i = threadIdx.x; i < CX * CY * CZ; i += blockDim.x) {
    const int cx = i % CX;
    const int t = i / CX;
    const int cy = t % CY;
    const int cz = t / CY;
    const int gcx = blockIdx.x * CX + cx, gcy = blockIdx.y * CY + cy, gcz = (DIM == 3) ? (int)blockIdx.z * CZ + cz : 0;
    if (!inside<DIM>(C, gcx, gcy, gcz)) continue;
    float sum = 0.f;
#pragma unroll
    for (int az = 0; az < ((DIM == 3) ? 2 : 1); ++az)
#pragma unroll
      for (int ay = 0; ay < 2; ++ay)
#pragma unroll
        for (int ax = 0; ax < 2; ++ax) {
          const int lx = g.H + 2 * cx + ax, ly = g.H + 2 * cy + ay, lz = (DIM == 3) ? g.H + 2 * cz + az : 0;
          const uint8_t mm = sm[g.idx(lx, ly, lz)];
          if (mm) sum += residual_at<DIM, HT, MASKED>(g, L, cur, sb, mm, lx, ly, lz);
        }
    bcoarse[gidx(C, gcx, gcy, gcz)] = cvt<T>(sum * inv_children);
  }
}

// ---------------------------------------------------------------------------
// Up leg of one level: x <- x + s * P e (copy of the coarse value to the
// 2^dim children, Sec. 2.2 prolongation filter of ones), then `post` sweeps;
// written to xout (xin is not modified, so tiles never race).  On the finest
// level of the preconditioner it also reduces (r, z) and sets CG's beta.
template <int DIM, int HT, typename T, bool MASKED, bool FINEST, typename TB = T>
__global__ void __launch_bounds__(kThreads)
k_up(LevelDev L, const TB* __restrict__ b, const T* __restrict__ xin, TB* __restrict__ xout,
     const T* __restrict__ e, int post, float omega, float s, SolveState* __restrict__ st,
     double* __restrict__ partials) {
  chain_enter();
  if (st && st->inner_done) return;
  using TS = TileShape<DIM>;
  const int post_c = HT > 0 ? HT : post;
  const Region<DIM, HT> g(post_c > 0 ? post_c : 1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sb = reinterpret_cast<float*>(smem_raw);
  float* s0 = sb + g.R;
  float* s1 = s0 + g.R;
  uint8_t* sm = reinterpret_cast<uint8_t*>(s1 + g.R);
  const int cnx = L.nx / 2, cny = L.ny / 2;
  for (int i = threadIdx.x; i < g.R; i += blockDim.x) {
    const int lx = i % g.RX;
    const int t = i / g.RX;
    const int ly = t % g.RY;
    const int lz = t / g.RY;
    const int gx = g.ox + lx, gy = g.oy + ly, gz = g.oz + lz;
    float v = 0.f, bv = 0.f;
    uint8_t m = 0;
    if (inside<DIM>(L, gx, gy, gz)) {
      const size_t gi = gidx(L, gx, gy, gz);
      m = MASKED ? L.cell[gi] : kFluidBit;
      if (m) {
        const size_t ci = ((size_t)(gz >> 1) * cny + (gy >> 1)) * cnx + (gx >> 1);
        v = ld(xin, gi) + s * ld(e, ci);
        bv = ld(b, gi);
      }
    }
    s0[i] = v;
    sb[i] = bv;
    sm[i] = m;
  }
  __syncthreads();
  float* cur = s0;
  float* nxt = s1;
  for (int j = 1; j <= post_c; ++j) {
    sweep_region<DIM, HT, MASKED>(g, L, cur, nxt, sb, sm, post_c - j, omega, false);
    float* t = cur; cur = nxt; nxt = t;
  }
  constexpr int TN = TS::X * TS::Y * TS::Z;
  float acc = 0.f;
  for (int i = threadIdx.x; i < TN; i += blockDim.x) {
    const int tx = i % TS::X;
    const int t = i / TS::X;
    const int ty = t % TS::Y;
    const int tz = t / TS::Y;
    const int lx = tx + g.H, ly = ty + g.H, lz = (DIM == 3) ? tz + g.H : 0;
    const int gx = g.ox + lx, gy = g.oy + ly, gz = g.oz + lz;
    if (inside<DIM>(L, gx, gy, gz)) {
      const int li = g.idx(lx, ly, lz);
      const TB zt = cvt<TB>(cur[li]);
      xout[gidx(L, gx, gy, gz)] = zt;
      if (FINEST) acc = fmaf(sb[li], ld(&zt, 0), acc);
    }
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

}  // namespace npmg
