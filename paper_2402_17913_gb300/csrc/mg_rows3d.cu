// 3D level kernels with two Jacobi sweeps: a block streams a 128 x 16
// column of cells along z with one warp per row.
//
// The block's region is 20 rows (the 16 output rows and two halo rows on
// each side); warp w owns row y0 - 2 + w, and each lane 4 consecutive
// cells of it (one 16-byte vector per float32 array), lanes 0 and 31 also
// the two cells beyond the strip on their side.  Per z-plane p the block
//   A  takes row (p, y) of its inputs from a per-warp ring of shared-memory
//      slots filled by asynchronous copies two planes ahead, forms the
//      first sweep's input there and writes it to a three-plane buffer;
//   B  runs the first sweep on plane p - 1 (rows 1 .. 18 of the region);
//   C  runs the second sweep (up: the output) or the residual (down) on
//      plane p - 2 (rows 2 .. 17), and on the down leg the 2x2x2 average of
//      the residual pairs of planes p - 3, p - 2.
// x-neighbours come by warp shuffles, y- and z-neighbours as vectors from
// the plane buffers; two block barriers per plane (three on odd planes of
// the down leg).  The diagonal of a cell comes from a 64-entry table of
// d and omega / d by link counts (kx + 4 ky + 16 kz).
//
// Same arithmetic as the other level kernels: weighted Jacobi
// (Eq. Jacobi-1-relax) written x <- (1 - omega) x + (omega / d)(b + nb),
// from a zero guess on the down leg, residual and 2x2x2 average restriction
// (App. B), copy prolongation plus the scaled correction and two post
// sweeps on the up leg (Sec. 2.2); cells outside the domain and solid cells
// hold 0 (the zero padding of Sec. 2.1).  On the finest level the up leg
// also reduces (r, z) and CG's beta.
#include <algorithm>
#include <type_traits>
#include <stdlib.h>

#include "launch.h"
#include "mg_kernels.cuh"

namespace npmg {

namespace {

#ifndef NPMG_R3_TY
#define NPMG_R3_TY 16
#endif
constexpr int V = 4;            // cells per lane
constexpr int TY = NPMG_R3_TY;  // output rows of a block
constexpr int NW = TY + 4;      // warps = region rows
constexpr int NT = 32 * NW;     // threads (640)
constexpr int kD = 2;           // planes in flight ahead of the plane in use
constexpr int kRS = kD + 1;     // ring slots per warp
// the register and ring phases coincide: step i uses ring slot i % 3 = C
// and refills slot (i + kD) % 3 = P (the slot read at step i - 1)
static_assert(kRS == 3, "ring slots follow the three-step phase");
constexpr int ROWF = 136;       // floats per buffered row: local x -4 .. 131
constexpr int PLANE = NW * ROWF;

template <typename T, typename TB, bool MASKED, bool UP>
struct Lay {
  static constexpr int SZ = (int)sizeof(T), SB = (int)sizeof(TB);
  // ring slot of one warp (bytes): x (up), b, e (up), cell bytes (masked),
  // halo pairs of lane 0 (side 0) and lane 31 (side 1)
  static constexpr int BO = UP ? 128 * SZ : 0;
  static constexpr int EO = BO + 128 * SB;
  static constexpr int MO = EO + (UP ? 64 * SZ : 0);
  static constexpr int HO = MO + (MASKED ? 128 : 0);
  static constexpr int SLOT = HO + 64;
  // block (bytes): two three-plane row buffers, the residual pair sums of
  // the down leg, the rings, the diagonal tables
  static constexpr int P0 = 0;
  static constexpr int P1 = P0 + 3 * PLANE * 4;
  static constexpr int RB = P1 + 3 * PLANE * 4;
  static constexpr int RG = RB + (UP ? 0 : 2 * TY * 64 * 4);
  static constexpr int LUT = RG + NW * kRS * SLOT;
  static constexpr int BYTES = LUT + 2 * 64 * 4;
  static_assert(SLOT % 16 == 0 && RG % 16 == 0, "16-byte alignment");
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
template <int N>
__device__ __forceinline__ void cp_async(uint32_t dst, const void* src, bool full) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(dst), "l"(src), "n"(N), "r"(full ? N : 0)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_ring() { asm volatile("cp.async.wait_group %0;\n" ::"n"(kD - 1) : "memory"); }

template <typename T>
__device__ __forceinline__ float2 h2f(unsigned u) {
  if constexpr (std::is_same<T, __half>::value) {
    __half2 h;
    *reinterpret_cast<unsigned*>(&h) = u;
    return __half22float2(h);
  } else {
    __nv_bfloat162 h;
    *reinterpret_cast<unsigned*>(&h) = u;
    return __bfloat1622float2(h);
  }
}
template <typename T>
__device__ __forceinline__ void lds4(const unsigned char* p, float (&v)[4]) {
  if constexpr (std::is_same<T, float>::value) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    const uint2 q = *reinterpret_cast<const uint2*>(p);
    const float2 a = h2f<T>(q.x), c = h2f<T>(q.y);
    v[0] = a.x; v[1] = a.y; v[2] = c.x; v[3] = c.y;
  }
}
template <typename T>
__device__ __forceinline__ float2 lds2(const unsigned char* p) {
  if constexpr (std::is_same<T, float>::value) return *reinterpret_cast<const float2*>(p);
  else return h2f<T>(*reinterpret_cast<const unsigned*>(p));
}
template <typename T>
__device__ __forceinline__ unsigned pack2(float a, float b) {
  T t[2] = {cvt<T>(a), cvt<T>(b)};
  return *reinterpret_cast<unsigned*>(t);
}
template <typename T, int N>
__device__ __forceinline__ void stv(T* p, const float (&v)[N]) {
  if constexpr (std::is_same<T, float>::value) {
    if constexpr (N == 4) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
    if constexpr (N == 4) *reinterpret_cast<uint2*>(p) = make_uint2(pack2<T>(v[0], v[1]), pack2<T>(v[2], v[3]));
    else *reinterpret_cast<unsigned*>(p) = pack2<T>(v[0], v[1]);
  }
}

// Lane geometry: own cells gx .. gx + 3, halo (lane 0: x0 - 1 inner,
// x0 - 2 outer; lane 31: x0 + 128 inner, x0 + 129 outer); link counts in x
// of the own cells and the halo (0 outside the domain).
struct Lane {
  int lane, warp, gx, y, hpair, epair, mword;
  bool ox, hok, yin;
  int hin_off, hout_off;  // float index of the inner / outer halo cell in a buffered row
  int kx[V + 2];
};

__device__ __forceinline__ Lane lane_of(const LevelDev& L, int x0, int y0) {
  Lane c;
  c.lane = threadIdx.x & 31;
  c.warp = threadIdx.x >> 5;
  c.gx = x0 + V * c.lane;
  c.y = y0 - 2 + c.warp;
  c.yin = c.y >= 0 && c.y < L.ny;
  c.ox = c.gx < L.nx;
  const bool left = c.lane == 0;
  const int hin = left ? x0 - 1 : x0 + 32 * V, hout = left ? x0 - 2 : x0 + 32 * V + 1;
  c.hpair = left ? x0 - 2 : x0 + 32 * V;
  c.epair = left ? (x0 >> 1) - 2 : (x0 >> 1) + 16 * V;
  c.mword = left ? x0 - 4 : x0 + 32 * V;
  c.hok = (left || c.lane == 31) && hout >= 0 && hout < L.nx;
  c.hin_off = left ? 3 : 4 + 32 * V;
  c.hout_off = left ? 2 : 5 + 32 * V;
#pragma unroll
  for (int j = 0; j < V + 2; ++j) {
    const int x = j < V ? c.gx + j : (j == V ? hin : hout);
    const bool in = j < V ? c.ox : c.hok;
    c.kx[j] = in ? axis_count(x, L.nx, L.bcD, 0) : 0;
  }
  return c;
}

// Table index of a cell: the cell byte's link counts (masked), or the
// counts of an unmasked level (0 outside the domain: d = 0).
template <bool MASKED>
__device__ __forceinline__ int lut_index(const Lane& c, int j, unsigned m, int kyz) {
  if (MASKED) return (int)(m & 63u);
  return (kyz >= 0 && c.kx[j] > 0) ? c.kx[j] + kyz : 0;
}

// y and z part of the unmasked table index of row c.y in plane p (-1 when
// the row is outside the domain).
__device__ __forceinline__ int kyz_of(const LevelDev& L, const Lane& c, int p) {
  if (!c.yin || p < 0 || p >= L.nz) return -1;
  return 4 * axis_count(c.y, L.ny, L.bcD, 2) + 16 * axis_count(p, L.nz, L.bcD, 4);
}

__device__ __forceinline__ void fill_lut(const LevelDev& L, float omega, float* lut) {
  if (threadIdx.x < 64) {
    const int kx = threadIdx.x & 3, ky = (threadIdx.x >> 2) & 3, kz = (threadIdx.x >> 4) & 3;
    const float d = (kx <= 2 && ky <= 2 && kz <= 2) ? L.wx * (float)kx + L.wy * (float)ky + L.wz * (float)kz : 0.f;
    lut[threadIdx.x] = d;                              // d
    lut[64 + threadIdx.x] = d > 0.f ? omega / d : 0.f;  // omega / d
  }
}

// Sweep value of the own cells and the inner halo of buffered row (pl, w):
// keep * a + wv * (bv + nb), neighbours from the rows w +- 1 and the planes
// pm, pp of the same buffer, x-neighbours by shuffles.
__device__ __forceinline__ void sweep_row(const LevelDev& L, const Lane& c, const float* buf, int pm, int pl, int pp,
                                          bool halo, float keep, const float (&bv)[V + 1], const float (&wv)[V + 1],
                                          float (&out)[V + 1]) {
  const float* row = buf + pl * PLANE + c.warp * ROWF;
  const int own = 4 + V * c.lane;
  float a[V], n0[V], n1[V], n2[V], n3[V];
  *reinterpret_cast<float4*>(a) = *reinterpret_cast<const float4*>(row + own);
  *reinterpret_cast<float4*>(n0) = *reinterpret_cast<const float4*>(row - ROWF + own);
  *reinterpret_cast<float4*>(n1) = *reinterpret_cast<const float4*>(row + ROWF + own);
  *reinterpret_cast<float4*>(n2) = *reinterpret_cast<const float4*>(buf + pm * PLANE + c.warp * ROWF + own);
  *reinterpret_cast<float4*>(n3) = *reinterpret_cast<const float4*>(buf + pp * PLANE + c.warp * ROWF + own);
  const float ah = row[c.hin_off];
  const float up = __shfl_up_sync(0xffffffffu, a[V - 1], 1);
  const float dn = __shfl_down_sync(0xffffffffu, a[0], 1);
  const float left = c.lane == 0 ? ah : up, right = c.lane == 31 ? ah : dn;
#pragma unroll
  for (int j = 0; j < V; ++j) {
    const float l = j == 0 ? left : a[j - 1], r = j == V - 1 ? right : a[j + 1];
    const float nb = fmaf(L.wx, l + r, fmaf(L.wy, n0[j] + n1[j], L.wz * (n2[j] + n3[j])));
    out[j] = fmaf(keep, a[j], wv[j] * (bv[j] + nb));
  }
  if (halo) {
    const float edge = c.lane == 0 ? a[0] : a[V - 1];
    const float nb = fmaf(L.wx, row[c.hout_off] + edge,
                          fmaf(L.wy, row[c.hin_off - ROWF] + row[c.hin_off + ROWF],
                               L.wz * (buf[pm * PLANE + c.warp * ROWF + c.hin_off] +
                                       buf[pp * PLANE + c.warp * ROWF + c.hin_off])));
    out[V] = fmaf(keep, ah, wv[V] * (bv[V] + nb));
  }
}

__device__ __forceinline__ void store_row(const Lane& c, float* buf, int pl, const float (&v)[V + 1]) {
  float* row = buf + pl * PLANE + c.warp * ROWF;
  *reinterpret_cast<float4*>(row + 4 + V * c.lane) = make_float4(v[0], v[1], v[2], v[3]);
  if (c.lane == 0 || c.lane == 31) row[c.hin_off] = v[V];
}

// ---- up leg ------------------------------------------------------------------
template <typename T, typename TB, bool MASKED>
__device__ __forceinline__ void up_issue(const LevelDev& L, const Lane& c, int p, bool want, const TB* __restrict__ b,
                                         const T* __restrict__ xin, const T* __restrict__ e, unsigned char* slot) {
  using S = Lay<T, TB, MASKED, true>;
  if (want) {
    const bool rin = p >= 0 && p < L.nz && c.yin;
    const bool fo = rin && c.ox, fh = rin && c.hok;
    const size_t row = rin ? ((size_t)p * L.ny + c.y) * L.nx : 0;
    const size_t crow = rin ? ((size_t)(p >> 1) * (L.ny >> 1) + (c.y >> 1)) * (L.nx >> 1) : 0;
    const int go = fo ? c.gx : 0;  // zero-fill copies keep an in-bounds source
    const uint32_t sl = smem_addr(slot);
    cp_async<4 * S::SZ>(sl + c.lane * 4 * S::SZ, xin + row + go, fo);
    cp_async<4 * S::SB>(sl + S::BO + c.lane * 4 * S::SB, b + row + go, fo);
    cp_async<2 * S::SZ>(sl + S::EO + c.lane * 2 * S::SZ, e + crow + (go >> 1), fo);
    if (MASKED) cp_async<4>(sl + S::MO + c.lane * 4, L.cell + row + go, fo);
    if (c.lane == 0 || c.lane == 31) {
      const uint32_t hs = sl + S::HO + (c.lane == 31 ? 32 : 0);
      cp_async<2 * S::SZ>(hs, xin + row + (fh ? c.hpair : 0), fh);
      cp_async<2 * S::SB>(hs + 8, b + row + (fh ? c.hpair : 0), fh);
      cp_async<2 * S::SZ>(hs + 16, e + crow + (fh ? c.epair : 0), fh);
      if (MASKED) cp_async<4>(hs + 24, L.cell + row + (fh ? c.mword : 0), fh);
    }
  }
  cp_commit();
}

// Halo pair of a ring slot as (inner, outer) for this lane.
template <typename T>
__device__ __forceinline__ void halo_pair(const Lane& c, const unsigned char* hs, int off, float& inner, float& outer) {
  const float2 v = lds2<T>(hs + off);
  inner = c.lane == 0 ? v.y : v.x;
  outer = c.lane == 0 ? v.x : v.y;
}
__device__ __forceinline__ void halo_bytes(const Lane& c, const unsigned char* hs, unsigned& inner, unsigned& outer) {
  const unsigned w = *reinterpret_cast<const unsigned*>(hs + 24);
  inner = c.lane == 0 ? (w >> 24) : (w & 0xffu);
  outer = c.lane == 0 ? ((w >> 16) & 0xffu) : ((w >> 8) & 0xffu);
}

struct UpRegs {
  float b[3][V + 1];  // b of own cells and inner halo, planes by phase
  float w[3][V + 1];  // omega / d
};

// Step i (plane p = z0 - 2 + i) with phase slots C = i % 3, P = (i - 1) % 3,
// Q = (i - 2) % 3.
template <typename T, typename TB, bool MASKED, bool FINEST, int C, int P, int Q>
__device__ __forceinline__ void up_step(const LevelDev& L, const Lane& c, int i, int z0, int z1, float omega, float s,
                                        const TB* __restrict__ b, const T* __restrict__ xin, const T* __restrict__ e,
                                        TB* __restrict__ xout, unsigned char* sm, UpRegs& R, float& acc) {
  using S = Lay<T, TB, MASKED, true>;
  const int p = z0 - 2 + i;
  float* B0 = reinterpret_cast<float*>(sm + S::P0);
  float* B1 = reinterpret_cast<float*>(sm + S::P1);
  const float* lut = reinterpret_cast<const float*>(sm + S::LUT);
  unsigned char* ring = sm + S::RG + c.warp * (kRS * S::SLOT);
  // A: row (p, y): x + s P e into buffer 0 (own cells and both halo cells)
  cp_wait_ring();
  {
    const unsigned char* sl = ring + C * S::SLOT;
    float xv[V], bv[V];
    lds4<T>(sl + c.lane * 4 * S::SZ, xv);
    lds4<TB>(sl + S::BO + c.lane * 4 * S::SB, bv);
    const float2 ev = lds2<T>(sl + S::EO + c.lane * 2 * S::SZ);
    const unsigned char* hs = sl + S::HO + (c.lane == 31 ? 32 : 0);
    float xh, xo, bh, bo, eh, eo;
    halo_pair<T>(c, hs, 0, xh, xo);
    halo_pair<TB>(c, hs, 8, bh, bo);
    halo_pair<T>(c, hs, 16, eh, eo);
    (void)bo;
    (void)eo;
    unsigned m[V + 2];
    const int kyz = MASKED ? 0 : kyz_of(L, c, p);
    if (MASKED) {
      const unsigned mw = *reinterpret_cast<const unsigned*>(sl + S::MO + c.lane * 4);
#pragma unroll
      for (int j = 0; j < V; ++j) m[j] = (mw >> (8 * j)) & 0xffu;
      halo_bytes(c, hs, m[V], m[V + 1]);
    } else {
#pragma unroll
      for (int j = 0; j < V + 2; ++j) m[j] = 0u;
    }
    float s0[V + 1];
#pragma unroll
    for (int j = 0; j < V + 1; ++j) {
      const int q = lut_index<MASKED>(c, j, m[j], kyz);
      R.w[C][j] = lut[64 + q];
      const float xj = j < V ? xv[j] : xh, ej = j < V ? (j < 2 ? ev.x : ev.y) : eh;
      const bool fl = MASKED ? m[j] != 0u : q != 0;
      s0[j] = fl ? fmaf(s, ej, xj) : 0.f;
      R.b[C][j] = j < V ? bv[j] : bh;
    }
    store_row(c, B0, C, s0);
    if (c.lane == 0 || c.lane == 31) {
      const bool flo = MASKED ? m[V + 1] != 0u : (kyz >= 0 && c.kx[V + 1] > 0);
      B0[C * PLANE + c.warp * ROWF + c.hout_off] = flo ? fmaf(s, eh, xo) : 0.f;
    }
  }
  up_issue<T, TB, MASKED>(L, c, p + kD, p + kD <= z1 + 1, b, xin, e, ring + P * S::SLOT);
  __syncthreads();
  const float keep = 1.f - omega;
  // B: first sweep on plane p - 1, rows 1 .. NW - 2
  if (p >= z0 && c.warp >= 1 && c.warp <= NW - 2) {
    float s1[V + 1];
    sweep_row(L, c, B0, Q, P, C, true, keep, R.b[P], R.w[P], s1);
    store_row(c, B1, P, s1);
  }
  __syncthreads();
  // C: second sweep on plane o = p - 2, rows 2 .. NW - 3, written out
  const int o = p - 2;
  if (o >= z0 && c.warp >= 2 && c.warp <= NW - 3 && c.yin) {
    float z[V + 1];
    sweep_row(L, c, B1, C, Q, P, false, keep, R.b[Q], R.w[Q], z);
    if (c.ox) {
      float zv[V] = {z[0], z[1], z[2], z[3]};
      stv<TB, V>(xout + ((size_t)o * L.ny + c.y) * L.nx + c.gx, zv);
      if (FINEST) {
#pragma unroll
        for (int j = 0; j < V; ++j) {
          const TB zt = cvt<TB>(z[j]);  // (r, z) of the stored z
          acc = fmaf(R.b[Q][j], ld(&zt, 0), acc);
        }
      }
    }
  }
}

// Work of a block: with `units` == 0 one z-run of zr planes of the column
// (blockIdx.x, blockIdx.y); otherwise the range [blockIdx.x * units,
// (blockIdx.x + 1) * units) of column-major (column, plane) units, which may
// end one column's planes and start the next column's (one run each).
struct Sched {
  int zr, units;
};

template <typename F>
__device__ __forceinline__ void for_each_run(const LevelDev& L, Sched sc, F&& run) {
  const int strips = (L.nx + 32 * V - 1) / (32 * V);
  if (sc.units == 0) {
    const int z0 = blockIdx.z * sc.zr;
    run(blockIdx.x * 32 * V, blockIdx.y * TY, z0, min(z0 + sc.zr, L.nz));
    return;
  }
  const long total = (long)strips * ((L.ny + TY - 1) / TY) * L.nz;
  long u = (long)blockIdx.x * sc.units;
  const long uend = min(u + sc.units, total);
  while (u < uend) {
    const int col = (int)(u / L.nz), z0 = (int)(u % L.nz);
    const int z1 = (int)min((long)L.nz, z0 + (uend - u));
    run((col % strips) * 32 * V, (col / strips) * TY, z0, z1);
    u += z1 - z0;
    __syncthreads();  // the next run refills the rings and plane buffers
  }
}

template <typename T, bool MASKED, bool FINEST, typename TB>
__global__ void __launch_bounds__(NT, 1) k_up_r3(LevelDev L, const TB* __restrict__ b, const T* __restrict__ xin,
                                                 TB* __restrict__ xout, const T* __restrict__ e, float omega, float s,
                                                 Sched sc, SolveState* __restrict__ st, double* __restrict__ partials) {
  chain_enter();
  if (st && st->inner_done) return;
  using S = Lay<T, TB, MASKED, true>;
  extern __shared__ __align__(16) unsigned char smem_r3[];
  fill_lut(L, omega, reinterpret_cast<float*>(smem_r3 + S::LUT));
  // zero the plane buffers (the halo cells of rows no lane writes stay 0)
  for (int k = threadIdx.x; k < 6 * PLANE / 4; k += NT)
    reinterpret_cast<float4*>(smem_r3 + S::P0)[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  float acc = 0.f;
  for_each_run(L, sc, [&](int x0, int y0, int z0, int z1) {
    const Lane c = lane_of(L, x0, y0);
    unsigned char* ring = smem_r3 + S::RG + c.warp * (kRS * S::SLOT);
#pragma unroll
    for (int i = 0; i < kD; ++i)
      up_issue<T, TB, MASKED>(L, c, z0 - 2 + i, z0 - 2 + i <= z1 + 1, b, xin, e, ring + i * S::SLOT);
    __syncthreads();
    UpRegs R;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int j = 0; j < V + 1; ++j) R.b[k][j] = R.w[k][j] = 0.f;
    const int n = z1 - z0 + 4;
    for (int i = 0; i < n; i += 3) {
      up_step<T, TB, MASKED, FINEST, 0, 2, 1>(L, c, i, z0, z1, omega, s, b, xin, e, xout, smem_r3, R, acc);
      if (i + 1 >= n) break;
      up_step<T, TB, MASKED, FINEST, 1, 0, 2>(L, c, i + 1, z0, z1, omega, s, b, xin, e, xout, smem_r3, R, acc);
      if (i + 2 >= n) break;
      up_step<T, TB, MASKED, FINEST, 2, 1, 0>(L, c, i + 2, z0, z1, omega, s, b, xin, e, xout, smem_r3, R, acc);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  });
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

// ---- down leg ----------------------------------------------------------------
template <typename T, typename TB, bool MASKED>
__device__ __forceinline__ void down_issue(const LevelDev& L, const Lane& c, int p, bool want, const TB* __restrict__ b,
                                           unsigned char* slot) {
  using S = Lay<T, TB, MASKED, false>;
  if (want) {
    const bool rin = p >= 0 && p < L.nz && c.yin;
    const bool fo = rin && c.ox, fh = rin && c.hok;
    const size_t row = rin ? ((size_t)p * L.ny + c.y) * L.nx : 0;
    const int go = fo ? c.gx : 0;
    const uint32_t sl = smem_addr(slot);
    cp_async<4 * S::SB>(sl + S::BO + c.lane * 4 * S::SB, b + row + go, fo);
    if (MASKED) cp_async<4>(sl + S::MO + c.lane * 4, L.cell + row + go, fo);
    if (c.lane == 0 || c.lane == 31) {
      const uint32_t hs = sl + S::HO + (c.lane == 31 ? 32 : 0);
      cp_async<2 * S::SB>(hs + 8, b + row + (fh ? c.hpair : 0), fh);
      if (MASKED) cp_async<4>(hs + 24, L.cell + row + (fh ? c.mword : 0), fh);
    }
  }
  cp_commit();
}

struct DownRegs {
  float b[3][V + 1];  // own cells and inner halo, planes by phase
  float w[3][V + 1];  // omega / d
  float d[3][V];      // d of the own cells
};

template <typename T, typename TB, bool MASKED, int C, int P, int Q>
__device__ __forceinline__ void down_step(const LevelDev& L, const Lane& c, int i, int z0, int z1, float omega,
                                          const TB* __restrict__ b, T* __restrict__ x, T* __restrict__ bcoarse,
                                          unsigned char* sm, DownRegs& R) {
  using S = Lay<T, TB, MASKED, false>;
  const int p = z0 - 2 + i;
  float* B0 = reinterpret_cast<float*>(sm + S::P0);  // first sweep
  float* B1 = reinterpret_cast<float*>(sm + S::P1);  // second sweep
  float* RB = reinterpret_cast<float*>(sm + S::RB);  // [2][TY][64] residual pair sums
  const float* lut = reinterpret_cast<const float*>(sm + S::LUT);
  unsigned char* ring = sm + S::RG + c.warp * (kRS * S::SLOT);
  // A: row (p, y): b, omega / d, d and the first sweep from zero (omega / d) b
  cp_wait_ring();
  {
    const unsigned char* sl = ring + C * S::SLOT;
    float bv[V];
    lds4<TB>(sl + S::BO + c.lane * 4 * S::SB, bv);
    const unsigned char* hs = sl + S::HO + (c.lane == 31 ? 32 : 0);
    float bh, bo;
    halo_pair<TB>(c, hs, 8, bh, bo);
    unsigned m[V + 2];
    const int kyz = MASKED ? 0 : kyz_of(L, c, p);
    if (MASKED) {
      const unsigned mw = *reinterpret_cast<const unsigned*>(sl + S::MO + c.lane * 4);
#pragma unroll
      for (int j = 0; j < V; ++j) m[j] = (mw >> (8 * j)) & 0xffu;
      halo_bytes(c, hs, m[V], m[V + 1]);
    } else {
#pragma unroll
      for (int j = 0; j < V + 2; ++j) m[j] = 0u;
    }
    float s1[V + 1];
#pragma unroll
    for (int j = 0; j < V + 1; ++j) {
      const int q = lut_index<MASKED>(c, j, m[j], kyz);
      const float bj = j < V ? bv[j] : bh;
      R.w[C][j] = lut[64 + q];
      R.b[C][j] = bj;
      if (j < V) R.d[C][j] = lut[q];
      s1[j] = R.w[C][j] * bj;
    }
    store_row(c, B0, C, s1);
    if (c.lane == 0 || c.lane == 31) {
      const int qo = lut_index<MASKED>(c, V + 1, m[V + 1], kyz);
      B0[C * PLANE + c.warp * ROWF + c.hout_off] = lut[64 + qo] * bo;
    }
  }
  down_issue<T, TB, MASKED>(L, c, p + kD, p + kD <= z1 + 1, b, ring + P * S::SLOT);
  __syncthreads();
  const float keep = 1.f - omega;
  // B: second sweep on plane p - 1, rows 1 .. NW - 2
  if (p >= z0 && c.warp >= 1 && c.warp <= NW - 2) {
    float s2[V + 1];
    sweep_row(L, c, B0, Q, P, C, true, keep, R.b[P], R.w[P], s2);
    store_row(c, B1, P, s2);
  }
  __syncthreads();
  // C: x and the residual on plane o = p - 2, rows 2 .. NW - 3; the x-pair
  // sums of the residual go to the pair buffer of o's parity
  const int o = p - 2;
  if (o >= z0) {
    if (c.warp >= 2 && c.warp <= NW - 3) {
      const float* row = B1 + Q * PLANE + c.warp * ROWF;
      const int own = 4 + V * c.lane;
      float a[V], n0[V], n1[V], n2[V], n3[V];
      *reinterpret_cast<float4*>(a) = *reinterpret_cast<const float4*>(row + own);
      *reinterpret_cast<float4*>(n0) = *reinterpret_cast<const float4*>(row - ROWF + own);
      *reinterpret_cast<float4*>(n1) = *reinterpret_cast<const float4*>(row + ROWF + own);
      *reinterpret_cast<float4*>(n2) = *reinterpret_cast<const float4*>(B1 + C * PLANE + c.warp * ROWF + own);
      *reinterpret_cast<float4*>(n3) = *reinterpret_cast<const float4*>(B1 + P * PLANE + c.warp * ROWF + own);
      const float ah = row[c.hin_off];
      const float up = __shfl_up_sync(0xffffffffu, a[V - 1], 1);
      const float dn = __shfl_down_sync(0xffffffffu, a[0], 1);
      const float left = c.lane == 0 ? ah : up, right = c.lane == 31 ? ah : dn;
      float r[V];
#pragma unroll
      for (int j = 0; j < V; ++j) {
        const float l = j == 0 ? left : a[j - 1], rr = j == V - 1 ? right : a[j + 1];
        const float nb = fmaf(L.wx, l + rr, fmaf(L.wy, n0[j] + n1[j], L.wz * (n2[j] + n3[j])));
        const float dj = R.d[Q][j];
        // cells with d = 0 (solid, outside) are not unknowns: no residual
        r[j] = dj != 0.f ? R.b[Q][j] - (dj * a[j] - nb) : 0.f;
      }
      if (c.yin && c.ox) stv<T, V>(x + ((size_t)o * L.ny + c.y) * L.nx + c.gx, a);
      float* rp = RB + ((o & 1) * TY + (c.warp - 2)) * 64 + 2 * c.lane;
      rp[0] = r[0] + r[1];
      rp[1] = r[2] + r[3];
    }
    if (o & 1) {
      __syncthreads();
      // 2x2x2 average: even rows of the tile, two coarse cells per lane
      const int lr = c.warp - 2, gy = c.y;
      if (lr >= 0 && lr < TY && (lr & 1) == 0 && gy < L.ny && c.ox) {
        const float* r0 = RB + lr * 64 + 2 * c.lane;
        const float* r1 = RB + (TY + lr) * 64 + 2 * c.lane;
        float bc[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) bc[k] = 0.125f * ((r0[k] + r0[64 + k]) + (r1[k] + r1[64 + k]));
        stv<T, 2>(bcoarse + ((size_t)(o >> 1) * (L.ny >> 1) + (gy >> 1)) * (L.nx >> 1) + (c.gx >> 1), bc);
      }
    }
  }
}


template <typename T, bool MASKED, typename TB>
__global__ void __launch_bounds__(NT, 1) k_down_r3(LevelDev L, const TB* __restrict__ b, T* __restrict__ x,
                                                   T* __restrict__ bcoarse, float omega, Sched sc,
                                                   const SolveState* __restrict__ st) {
  chain_enter();
  if (st && st->inner_done) return;
  using S = Lay<T, TB, MASKED, false>;
  extern __shared__ __align__(16) unsigned char smem_r3[];
  fill_lut(L, omega, reinterpret_cast<float*>(smem_r3 + S::LUT));
  for (int k = threadIdx.x; k < 6 * PLANE / 4; k += NT)
    reinterpret_cast<float4*>(smem_r3 + S::P0)[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  for_each_run(L, sc, [&](int x0, int y0, int z0, int z1) {
    const Lane c = lane_of(L, x0, y0);
    unsigned char* ring = smem_r3 + S::RG + c.warp * (kRS * S::SLOT);
#pragma unroll
    for (int i = 0; i < kD; ++i)
      down_issue<T, TB, MASKED>(L, c, z0 - 2 + i, z0 - 2 + i <= z1 + 1, b, ring + i * S::SLOT);
    __syncthreads();
    DownRegs R;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int j = 0; j < V + 1; ++j) {
        R.b[k][j] = R.w[k][j] = 0.f;
        if (j < V) R.d[k][j] = 0.f;
      }
    const int n = z1 - z0 + 4;
    for (int i = 0; i < n; i += 3) {
      down_step<T, TB, MASKED, 0, 2, 1>(L, c, i, z0, z1, omega, b, x, bcoarse, smem_r3, R);
      if (i + 1 >= n) break;
      down_step<T, TB, MASKED, 1, 0, 2>(L, c, i + 1, z0, z1, omega, b, x, bcoarse, smem_r3, R);
      if (i + 2 >= n) break;
      down_step<T, TB, MASKED, 2, 1, 0>(L, c, i + 2, z0, z1, omega, b, x, bcoarse, smem_r3, R);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  });
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
static int r3_sms() {
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 148;
  }
  return nsm;
}

// Schedule of a level (one block per SM): uniform z-runs of zr planes per
// column, the run count minimising waves x (zr + 4 halo planes); or an even
// split of the column-major (column, plane) units over one block per SM,
// each block paying 4 halo planes per column it touches.  The cheaper of the
// two by that count (NPMG_ROWS3D_SPLIT=0 keeps the uniform one, =2 always
// splits).
struct R3Plan {
  Sched sc;
  dim3 grid;
};

static R3Plan r3_plan(const LevelDev& L) {
  const long strips = (L.nx + 32 * V - 1) / (32 * V), tiles = (L.ny + TY - 1) / TY;
  const long cols = strips * tiles;
  const long nsm = r3_sms();
  long best = -1, best_zr = L.nz;
  for (int runs = 1; runs <= L.nz / 2; ++runs) {
    int zr = (L.nz + runs - 1) / runs;
    zr = (zr + 1) / 2 * 2;
    const long nr = (L.nz + zr - 1) / zr;
    const long waves = (cols * nr + nsm - 1) / nsm;
    const long cost = waves * (zr + 4);
    if (best < 0 || cost < best) {
      best = cost;
      best_zr = zr;
    }
  }
  R3Plan p;
  p.sc.zr = (int)best_zr;
  p.sc.units = 0;
  p.grid = dim3((unsigned)strips, (unsigned)tiles, (unsigned)((L.nz + best_zr - 1) / best_zr));
  const char* e = getenv("NPMG_ROWS3D_SPLIT");
  if (e && atoi(e) == 0) return p;
  const bool force = e && atoi(e) == 2;
  const long total = cols * L.nz;
  long units = (total + nsm - 1) / nsm;
  units = (units + 1) / 2 * 2;  // runs start on even planes (restriction pairs)
  const long touched = (units + L.nz - 2) / L.nz + 1;  // columns one range can reach
  const long cost = units + 4 * touched;
  if (force || cost < best) {
    p.sc.units = (int)units;
    p.grid = dim3((unsigned)((total + units - 1) / units), 1, 1);
  }
  return p;
}

// Smallest level (cells) taken by these kernels: 2^15, or NPMG_ROWS3D_MIN
// (measured on GB300: the 256x128x128 flow step is 15% faster with its
// 128x64x64 and 64x32x32 levels here than on the z-streaming and tile
// kernels, the 256^3 solve 3% faster with its 64^3 and 32^3 levels here;
// the single-block coarse kernel stays faster below).
bool rows3d_eligible(int dim, int pre, int post, const LevelDev& L) {
  const char* e = getenv("NPMG_ROWS3D_MIN");
  const size_t lim = e ? (size_t)atol(e) : ((size_t)1 << 15);
  return dim == 3 && pre == 2 && post == 2 && L.nx % 4 == 0 && L.ny % 2 == 0 && L.nz % 2 == 0 && L.nz >= 4 &&
         (size_t)L.nx * L.ny * L.nz >= lim;
}

template <typename T, bool MASKED, typename TB>
cudaError_t launch_down_r3(const LevelDev& L, const void* b, void* x, void* bcoarse, float omega, const SolveState* st,
                           cudaStream_t s) {
  const R3Plan pl = r3_plan(L);
  return launch_chain(k_down_r3<T, MASKED, TB>, pl.grid, NT, (size_t)Lay<T, TB, MASKED, false>::BYTES, s, L,
                      (const TB*)b, (T*)x, (T*)bcoarse, omega, pl.sc, st);
}

template <typename T, bool MASKED, bool FINEST, typename TB>
cudaError_t launch_up_r3(const LevelDev& L, const void* b, const void* xin, void* xout, const void* e, float omega,
                         float sc, SolveState* st, double* partials, cudaStream_t s) {
  const R3Plan pl = r3_plan(L);
  return launch_chain(k_up_r3<T, MASKED, FINEST, TB>, pl.grid, NT, (size_t)Lay<T, TB, MASKED, true>::BYTES, s, L,
                      (const TB*)b, (const T*)xin, (TB*)xout, (const T*)e, omega, sc, pl.sc, st, partials);
}

template <typename T, bool MASKED, typename TB>
static cudaError_t prepare_r3_pair() {
  cudaError_t e = cudaFuncSetAttribute(k_down_r3<T, MASKED, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Lay<T, TB, MASKED, false>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_up_r3<T, MASKED, false, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Lay<T, TB, MASKED, true>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_up_r3<T, MASKED, true, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Lay<T, TB, MASKED, true>::BYTES);
  return e;
}

template <typename T, bool MASKED>
cudaError_t prepare_r3_kernels() {
  cudaError_t e = prepare_r3_pair<T, MASKED, T>();
  if (e == cudaSuccess && !std::is_same<T, float>::value) e = prepare_r3_pair<T, MASKED, float>();
  return e;
}

#define NPMG_INST_R3_TB(T, M, TB)                                                                                 \
  template cudaError_t launch_down_r3<T, M, TB>(const LevelDev&, const void*, void*, void*, float,                 \
                                                const SolveState*, cudaStream_t);                                 \
  template cudaError_t launch_up_r3<T, M, false, TB>(const LevelDev&, const void*, const void*, void*,             \
                                                     const void*, float, float, SolveState*, double*, cudaStream_t); \
  template cudaError_t launch_up_r3<T, M, true, TB>(const LevelDev&, const void*, const void*, void*,              \
                                                    const void*, float, float, SolveState*, double*, cudaStream_t);
#define NPMG_INST_R3(T, M)                       \
  template cudaError_t prepare_r3_kernels<T, M>(); \
  NPMG_INST_R3_TB(T, M, T)                       \
  NPMG_INST_R3_TB(T, M, float)

template cudaError_t prepare_r3_kernels<float, false>();
template cudaError_t prepare_r3_kernels<float, true>();
NPMG_INST_R3_TB(float, false, float)
NPMG_INST_R3_TB(float, true, float)
NPMG_INST_R3(__half, false)
NPMG_INST_R3(__half, true)
NPMG_INST_R3(__nv_bfloat16, false)
NPMG_INST_R3(__nv_bfloat16, true)

}  // namespace npmg
