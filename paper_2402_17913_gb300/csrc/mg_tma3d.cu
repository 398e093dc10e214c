// 3D level kernels with two Jacobi sweeps, fed by TMA plane loads: a block
// streams a 128 x 16 column of cells along z.
//
// Region of a column: x0 - 4 .. x0 + 131 (34 chunks of 4 cells) by
// y0 - 2 .. y0 + 17 (20 rows, 10 row pairs); thread (chunk c, pair q) owns
// the 4 x 2 cells of chunk c in rows 2q and 2q + 1 for the whole z-run, so
// the values of its cells on the planes above and below, and the other row
// of its pair, are in its own registers: only the row above the pair, the
// row below it and the x-neighbours beyond the chunk pass through shared
// memory.  A row pair is also a restriction pair.
//
// One elected thread loads whole planes of the inputs (x, b, the coarse
// correction e, the cell bytes) with cp.async.bulk.tensor into a ring of
// stages (six on the up leg, eight on the down leg), each completed on its
// own mbarrier (zero fill outside the domain is the zero padding of
// Sec. 2.1).  Per z-plane p (step i):
//   A  every thread waits for the stage of plane p and forms the first
//      sweep's input there (up: x + s P e; down: the first sweep from zero,
//      (omega / d) b) into a two-slot plane buffer;
//   B  first sweep (up) / second sweep (down) on plane p - 1;
//   C  second sweep, written out (up) / residual and 2x2x2 average (down) on
//      plane p - 2;
// then one block barrier, after which the elected thread refills the stage
// just consumed with the plane one ring length ahead.  Every wait is bounded: a load that never
// lands ends the kernel with MG_TIMEOUT after the loads in flight drained.
//
// Same arithmetic as the other level kernels: weighted Jacobi
// (Eq. Jacobi-1-relax) written x <- (1 - omega) x + (omega / d)(b + nb),
// from a zero guess on the down leg, residual and 2x2x2 average restriction
// (App. B), copy prolongation plus the scaled correction and two post sweeps
// on the up leg (Sec. 2.2); cells outside the domain and solid cells hold 0.
// On the finest level the up leg also reduces (r, z) and CG's beta.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdlib.h>
#include <type_traits>

#include "launch.h"
#include "mg_kernels.cuh"
#include "refine.cuh"
#include "tma.cuh"
#include "tma_host.h"

namespace npmg {

namespace {

constexpr int TX = 128, TY = 16;   // output cells of a column (x, y)
constexpr int NCH = TX / 4 + 2;    // chunks of 4 cells per region row (34)
constexpr int RY = TY + 4;         // region rows (20)
constexpr int NQ = RY / 2;         // row pairs (10)
constexpr int NT = NCH * NQ;       // threads (340)
constexpr int RS = 4 * NCH + 8;    // floats per plane-buffer row: 4 pad, 136 cells, 4 pad
constexpr int PL = RS * (RY + 2);  // floats per plane buffer: a pad row above and below the region

__host__ __device__ constexpr int al128(int v) { return (v + 127) / 128 * 128; }

template <typename T, typename TB, bool MASKED, bool UP>
struct G3 {
  static constexpr int MT = 16 / (int)sizeof(T), MB = 16 / (int)sizeof(TB);
  // boxes: x and b start 16 bytes left of the region, e (coarse) likewise,
  // the cell bytes 16 cells left
  static constexpr int WX = TX + 2 * MT, WB = TX + 2 * MB, WE = TX / 2 + 2 * MT, EY = RY / 2, WM = TX + 32;
  static constexpr int XB = UP ? WX * RY * (int)sizeof(T) : 0;
  static constexpr int BB = WB * RY * (int)sizeof(TB);
  static constexpr int EB = UP ? WE * EY * (int)sizeof(T) : 0;
  static constexpr int MBY = MASKED ? WM * RY : 0;
  static constexpr uint32_t TXB = (uint32_t)(XB + BB + EB + MBY);  // bytes one stage receives
  static constexpr int OX = 0, OB = al128(OX + XB), OE = al128(OB + BB), OM = al128(OE + EB);
  static constexpr int STAGE = al128(OM + MBY);
  // block: two plane buffers of two slots (float), the stages, the
  // diagonal table (masked), the stage barriers
  static constexpr int NS = UP ? 6 : 8;  // TMA stages (planes in flight + the one in use)
  static constexpr int RING = 4 * PL * 4;
  static constexpr int LUT = RING + NS * STAGE;
  static constexpr int BAR = LUT + 128 * 4;
  static constexpr int BYTES = BAR + NS * 8;
  static_assert(RING % 128 == 0 && STAGE % 128 == 0, "TMA destinations 128-byte aligned");
};

// 4 consecutive elements of storage type T at byte address p (8- or
// 16-byte aligned) as floats; 2 elements (4- or 8-byte aligned).
template <typename T>
__device__ __forceinline__ void lds4(const unsigned char* p, float (&v)[4]) {
  if constexpr (std::is_same<T, float>::value) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    const uint2 q = *reinterpret_cast<const uint2*>(p);
    T t[4];
    *reinterpret_cast<uint2*>(t) = q;
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = ld(t, j);
  }
}
template <typename T>
__device__ __forceinline__ float2 lds2(const unsigned char* p) {
  if constexpr (std::is_same<T, float>::value) {
    return *reinterpret_cast<const float2*>(p);
  } else {
    T t[2];
    *reinterpret_cast<unsigned*>(t) = *reinterpret_cast<const unsigned*>(p);
    return make_float2(ld(t, 0), ld(t, 1));
  }
}
template <typename T>
__device__ __forceinline__ void stg4(T* p, const float (&v)[4]) {
  if constexpr (std::is_same<T, float>::value) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    T t[4] = {cvt<T>(v[0]), cvt<T>(v[1]), cvt<T>(v[2]), cvt<T>(v[3])};
    *reinterpret_cast<uint2*>(p) = *reinterpret_cast<const uint2*>(t);
  }
}
template <typename T>
__device__ __forceinline__ void stg2(T* p, float a, float b) {
  if constexpr (std::is_same<T, float>::value) {
    *reinterpret_cast<float2*>(p) = make_float2(a, b);
  } else {
    T t[2] = {cvt<T>(a), cvt<T>(b)};
    *reinterpret_cast<unsigned*>(p) = *reinterpret_cast<const unsigned*>(t);
  }
}

// Thread geometry.
struct Th {
  int c, q;       // chunk, row pair (rows 2q, 2q + 1 of the region)
  int gx, gy;     // global x of the chunk's first cell, global y of row 2q
  bool xin;       // chunk inside the domain (nx % 16 == 0: a chunk is all in or all out)
  bool yin[2];    // rows inside the domain
  bool own;       // the chunk and both rows belong to the column's output
};

__device__ __forceinline__ Th thread_geom(const LevelDev& L, int x0, int y0) {
  Th t;
  t.c = threadIdx.x % NCH;
  t.q = threadIdx.x / NCH;
  t.gx = x0 - 4 + 4 * t.c;
  t.gy = y0 - 2 + 2 * t.q;
  t.xin = t.gx >= 0 && t.gx < L.nx;
  t.yin[0] = t.gy >= 0 && t.gy < L.ny;
  t.yin[1] = t.gy + 1 >= 0 && t.gy + 1 < L.ny;
  t.own = t.c >= 1 && t.c <= NCH - 2 && t.q >= 1 && t.q <= NQ - 2;
  return t;
}

// omega / d and d of the thread's cells on an unmasked level, for the two
// link counts a plane can have along z (1: a Neumann z face, 2 otherwise);
// 0 for cells outside the domain.
struct Diag {
  float w1[2][4], w2[2][4], d1[2][4], d2[2][4];
};

__device__ __forceinline__ Diag unmasked_diag(const LevelDev& L, const Th& t, float omega) {
  Diag D;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int ky = t.yin[h] ? axis_count(t.gy + h, L.ny, L.bcD, 2) : 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool in = t.xin && t.yin[h];
      const float dxy = in ? L.wx * (float)axis_count(t.gx + j, L.nx, L.bcD, 0) + L.wy * (float)ky : 0.f;
      D.d1[h][j] = in ? dxy + L.wz : 0.f;
      D.d2[h][j] = in ? dxy + 2.f * L.wz : 0.f;
      D.w1[h][j] = in ? omega / D.d1[h][j] : 0.f;
      D.w2[h][j] = in ? omega / D.d2[h][j] : 0.f;
    }
  }
  return D;
}

// z link count of plane p (0 outside the domain).
__device__ __forceinline__ int plane_kz(const LevelDev& L, int p) {
  return (p >= 0 && p < L.nz) ? axis_count(p, L.nz, L.bcD, 4) : 0;
}

// Runs f with a getter of the per-cell value (omega / d or d) of the
// thread's cells on a plane with z link count kz: one uniform branch per
// plane instead of a select per cell.
template <typename F>
__device__ __forceinline__ void with_plane(int kz, const float (&v1)[2][4], const float (&v2)[2][4], F&& f) {
  if (kz == 2) f([&](int h, int j) { return v2[h][j]; });
  else if (kz == 1) f([&](int h, int j) { return v1[h][j]; });
  else f([](int, int) { return 0.f; });
}

__device__ __forceinline__ void fill_lut(const LevelDev& L, float omega, float* lut) {
  if (threadIdx.x < 64) {
    const int kx = threadIdx.x & 3, ky = (threadIdx.x >> 2) & 3, kz = (threadIdx.x >> 4) & 3;
    const float d = (kx <= 2 && ky <= 2 && kz <= 2) ? L.wx * (float)kx + L.wy * (float)ky + L.wz * (float)kz : 0.f;
    lut[threadIdx.x] = d;
    lut[64 + threadIdx.x] = d > 0.f ? omega / d : 0.f;
  }
}

// Row h (0, 1) of a thread's pair in plane buffer `buf` (region row 2q + h;
// the buffer has a pad row above region row 0).
__device__ __forceinline__ float* brow(float* buf, const Th& t, int h) {
  return buf + (2 * t.q + h + 1) * RS + 4 + 4 * t.c;
}
__device__ __forceinline__ const float* brow(const float* buf, const Th& t, int h) {
  return buf + (2 * t.q + h + 1) * RS + 4 + 4 * t.c;
}

// Neighbour sums of a thread's 4 x 2 cells on one plane, a = the cells'
// own values (registers), zm / zp = the same cells one plane below / above
// (registers); the row above the pair, the row below it and the
// x-neighbours beyond the chunk come from plane buffer `buf`:
// nb = wx (left + right) + wy (south + north) + wz (below + above).
__device__ __forceinline__ void neighbours(const LevelDev& L, const Th& t, const float* buf,
                                           const float (&a)[2][4], const float (&zm)[2][4],
                                           const float (&zp)[2][4], float (&nb)[2][4]) {
  const float* r0 = brow(buf, t, 0);
  const float* r1 = r0 + RS;
  const float4 s = *reinterpret_cast<const float4*>(r0 - RS);
  const float4 n = *reinterpret_cast<const float4*>(r1 + RS);
  const float l0 = r0[-1], e0 = r0[4], l1 = r1[-1], e1 = r1[4];
  const float sv[4] = {s.x, s.y, s.z, s.w}, nv[4] = {n.x, n.y, n.z, n.w};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float xl0 = j == 0 ? l0 : a[0][j - 1], xr0 = j == 3 ? e0 : a[0][j + 1];
    const float xl1 = j == 0 ? l1 : a[1][j - 1], xr1 = j == 3 ? e1 : a[1][j + 1];
    nb[0][j] = fmaf(L.wx, xl0 + xr0, fmaf(L.wy, sv[j] + a[1][j], L.wz * (zm[0][j] + zp[0][j])));
    nb[1][j] = fmaf(L.wx, xl1 + xr1, fmaf(L.wy, a[0][j] + nv[j], L.wz * (zm[1][j] + zp[1][j])));
  }
}

__device__ __forceinline__ void sts8(float* buf, const Th& t, const float (&v)[2][4]) {
  float* r0 = brow(buf, t, 0);
  *reinterpret_cast<float4*>(r0) = make_float4(v[0][0], v[0][1], v[0][2], v[0][3]);
  *reinterpret_cast<float4*>(r0 + RS) = make_float4(v[1][0], v[1][1], v[1][2], v[1][3]);
}

// Work of a block: the range [blockIdx.x * units, (blockIdx.x + 1) * units)
// of column-major (column, plane) units (a block may end one column's
// planes and start the next column's), or with units == 0 one z-run of zr
// planes of column (blockIdx.x, blockIdx.y).
struct Sched {
  int zr, units;
};

template <typename F>
__device__ __forceinline__ void for_each_run(const LevelDev& L, Sched sc, F&& run) {
  const int strips = (L.nx + TX - 1) / TX;
  if (sc.units == 0) {
    const int z0 = blockIdx.z * sc.zr;
    run(blockIdx.x * TX, blockIdx.y * TY, z0, min(z0 + sc.zr, L.nz));
    return;
  }
  const long total = (long)strips * ((L.ny + TY - 1) / TY) * L.nz;
  long u = (long)blockIdx.x * sc.units;
  const long uend = min(u + sc.units, total);
  while (u < uend) {
    const int col = (int)(u / L.nz), z0 = (int)(u % L.nz);
    const int z1 = (int)min((long)L.nz, z0 + (uend - u));
    if (!run((col % strips) * TX, (col / strips) * TY, z0, z1)) return;
    u += z1 - z0;
  }
}

// The stage ring of N stages: the elected thread (thread 0) issues global
// step g's loads into stage g % N; every thread waits for it with parity
// (g / N) & 1.
template <int N>
struct Ring {
  uint64_t* bar;
  unsigned char* base;
  unsigned g;        // global step of the next wait
  unsigned issued;   // global steps issued (thread 0)
};

template <typename T, typename TB, bool MASKED, bool UP, int N>
__device__ __forceinline__ void issue_plane(Ring<N>& R, const CUtensorMap* mx, const CUtensorMap* mb,
                                            const CUtensorMap* me, const CUtensorMap* mm, int x0, int y0, int p) {
  using S = G3<T, TB, MASKED, UP>;
  const unsigned st = R.issued % N;
  unsigned char* dst = R.base + st * S::STAGE;
  uint64_t* bar = R.bar + st;
  mbar_arrive_expect_tx(bar, S::TXB);
  if (UP) tma_load_3d(dst + S::OX, mx, bar, x0 - S::MT, y0 - 2, p);
  tma_load_3d(dst + S::OB, mb, bar, x0 - S::MB, y0 - 2, p);
  if (UP) tma_load_3d(dst + S::OE, me, bar, (x0 >> 1) - S::MT, (y0 >> 1) - 1, p >> 1);
  if (MASKED) tma_load_3d(dst + S::OM, mm, bar, x0 - 16, y0 - 2, p);
  ++R.issued;
}

// After a failed wait: the elected thread waits (bounded) for every load
// still in flight, so that none lands in shared memory after the block
// exits.
template <int N>
__device__ __forceinline__ void drain(Ring<N>& R, unsigned from) {
  if (threadIdx.x == 0)
    for (unsigned s = from; s < R.issued; ++s) (void)mbar_wait_bounded(R.bar + s % N, (s / N) & 1);
}

__device__ __forceinline__ void fail(SolveState* st) {
  if (st && threadIdx.x == 0) {
    st->status = MG_TIMEOUT;
    st->inner_done = 1;
    st->outer_done = 1;
  }
}

// ---- up leg ------------------------------------------------------------------
template <typename T, bool MASKED, bool FINEST, typename TB>
__global__ void __launch_bounds__(NT, 1)
    k_up_t3(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mb,
            const __grid_constant__ CUtensorMap me, const __grid_constant__ CUtensorMap mm, LevelDev L,
            TB* __restrict__ xout, float omega, float s, Sched sc, SolveState* __restrict__ st,
            double* __restrict__ partials) {
  chain_enter();
  if (st && st->inner_done) return;
  using S = G3<T, TB, MASKED, true>;
  extern __shared__ __align__(128) unsigned char smem_t3[];
  float* XS = reinterpret_cast<float*>(smem_t3);  // [2][PL]: x + s P e
  float* SS = XS + 2 * PL;                        // [2][PL]: first sweep
  const float* lut = reinterpret_cast<const float*>(smem_t3 + S::LUT);
  Ring<S::NS> R;
  R.bar = reinterpret_cast<uint64_t*>(smem_t3 + S::BAR);
  R.base = smem_t3 + S::RING;
  R.g = R.issued = 0;
  if (MASKED) fill_lut(L, omega, reinterpret_cast<float*>(smem_t3 + S::LUT));
  if (threadIdx.x == 0) {
    for (int k = 0; k < S::NS; ++k) mbar_init(R.bar + k, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const float keep = 1.f - omega;
  float acc = 0.f;
  bool failed = false;
  for_each_run(L, sc, [&](int x0, int y0, int z0, int z1) -> bool {
    const Th t = thread_geom(L, x0, y0);
    Diag D;
    if (!MASKED) D = unmasked_diag(L, t, omega);
    const int n = z1 - z0 + 4;  // steps: A on planes z0 - 2 .. z1 + 1
    if (threadIdx.x == 0)
      for (int k = 0; k < S::NS && k < n; ++k) issue_plane<T, TB, MASKED, true>(R, &mx, &mb, &me, &mm, x0, y0, z0 - 2 + k);
    float XQ[3][2][4], BQ[3][2][4], WQ[3][2][4], SQ[3][2][4];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 4; ++j) XQ[k][h][j] = BQ[k][h][j] = WQ[k][h][j] = SQ[k][h][j] = 0.f;
    auto step = [&](int i, auto phc) -> bool {
      constexpr int C0 = decltype(phc)::value;             // i % 3
      constexpr int C1 = (C0 + 2) % 3, C2 = (C0 + 1) % 3;  // (i - 1) % 3, (i - 2) % 3
      const int p = z0 - 2 + i;
      const bool ok = mbar_wait_bounded(R.bar + R.g % S::NS, (R.g / S::NS) & 1);
      // A: x + s P e of plane p
      {
        const unsigned char* sg = R.base + (R.g % S::NS) * S::STAGE;
        const float2 ev = lds2<T>(sg + S::OE + (t.q * S::WE + S::MT - 2 + 2 * t.c) * (int)sizeof(T));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = 2 * t.q + h;
          float xv[4], bv[4];
          lds4<T>(sg + S::OX + (r * S::WX + S::MT - 4 + 4 * t.c) * (int)sizeof(T), xv);
          lds4<TB>(sg + S::OB + (r * S::WB + S::MB - 4 + 4 * t.c) * (int)sizeof(TB), bv);
          if (MASKED) {
            const unsigned mw = *reinterpret_cast<const unsigned*>(sg + S::OM + r * S::WM + 12 + 4 * t.c);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const unsigned m = (mw >> (8 * j)) & 0xffu;
              WQ[C0][h][j] = lut[64 + (m & 63u)];
              XQ[C0][h][j] = m ? fmaf(s, j < 2 ? ev.x : ev.y, xv[j]) : 0.f;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) XQ[C0][h][j] = fmaf(s, j < 2 ? ev.x : ev.y, xv[j]);  // 0 outside
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) BQ[C0][h][j] = bv[j];
        }
        sts8(XS + (i & 1) * PL, t, XQ[C0]);
      }
      // B: first sweep on plane p - 1 (the pad rows above and below the
      // region make every row's neighbour reads safe; rows 0 and 19 are
      // never read)
      if (i >= 2) {
        float nb[2][4];
        neighbours(L, t, XS + ((i - 1) & 1) * PL, XQ[C1], XQ[C2], XQ[C0], nb);
        auto sweep = [&](auto W) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < 4; ++j) SQ[C1][h][j] = fmaf(keep, XQ[C1][h][j], W(h, j) * (BQ[C1][h][j] + nb[h][j]));
        };
        if constexpr (MASKED) sweep([&](int h, int j) { return WQ[C1][h][j]; });
        else with_plane(plane_kz(L, p - 1), D.w1, D.w2, sweep);
        sts8(SS + ((i - 1) & 1) * PL, t, SQ[C1]);
      }
      // C: second sweep on plane o = p - 2, written out
      const int o = p - 2;
      if (i >= 4 && t.own) {
        float nb[2][4], z[2][4];
        neighbours(L, t, SS + (i & 1) * PL, SQ[C2], SQ[C0], SQ[C1], nb);
        auto sweep = [&](auto W) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < 4; ++j) z[h][j] = fmaf(keep, SQ[C2][h][j], W(h, j) * (BQ[C2][h][j] + nb[h][j]));
        };
        if constexpr (MASKED) sweep([&](int h, int j) { return WQ[C2][h][j]; });
        else with_plane(plane_kz(L, o), D.w1, D.w2, sweep);
        if (t.xin) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (!t.yin[h]) continue;
            stg4<TB>(xout + ((size_t)o * L.ny + t.gy + h) * L.nx + t.gx, z[h]);
            if (FINEST) {
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const TB zt = cvt<TB>(z[h][j]);  // (r, z) of the stored z
                acc = fmaf(BQ[C2][h][j], ld(&zt, 0), acc);
              }
            }
          }
        }
      }
      if (__syncthreads_or(!ok)) {
        drain(R, R.g);
        return false;
      }
      if (threadIdx.x == 0 && i + S::NS < n)
        issue_plane<T, TB, MASKED, true>(R, &mx, &mb, &me, &mm, x0, y0, z0 - 2 + i + S::NS);
      ++R.g;
      return true;
    };
    for (int i = 0; i < n; i += 3) {
      if (!step(i, std::integral_constant<int, 0>())) return !(failed = true);
      if (i + 1 >= n) break;
      if (!step(i + 1, std::integral_constant<int, 1>())) return !(failed = true);
      if (i + 2 >= n) break;
      if (!step(i + 2, std::integral_constant<int, 2>())) return !(failed = true);
    }
    return true;
  });
  if (failed) fail(st);
  if (FINEST) {
    double tot;
    if (grid_sum_last((double)acc, partials, &st->counter[kCntRZ], &tot)) {
      if (threadIdx.x == 0 && !failed) {
        st->rz = tot;
        st->beta = (st->first || !st->krylov) ? 0.0 : tot / st->rz_old;
        st->rz_old = tot;
      }
    }
  }
}

// ---- down leg ----------------------------------------------------------------
template <typename T, bool MASKED, typename TB>
__global__ void __launch_bounds__(NT, 1)
    k_down_t3(const __grid_constant__ CUtensorMap mb, const __grid_constant__ CUtensorMap mm, LevelDev L,
              T* __restrict__ x, T* __restrict__ bcoarse, float omega, Sched sc, SolveState* __restrict__ st) {
  chain_enter();
  if (st && st->inner_done) return;
  using S = G3<T, TB, MASKED, false>;
  extern __shared__ __align__(128) unsigned char smem_t3[];
  float* S1 = reinterpret_cast<float*>(smem_t3);  // [2][PL]: first sweep
  float* XB = S1 + 2 * PL;                        // [2][PL]: second sweep (the leg's x)
  const float* lut = reinterpret_cast<const float*>(smem_t3 + S::LUT);
  Ring<S::NS> R;
  R.bar = reinterpret_cast<uint64_t*>(smem_t3 + S::BAR);
  R.base = smem_t3 + S::RING;
  R.g = R.issued = 0;
  if (MASKED) fill_lut(L, omega, reinterpret_cast<float*>(smem_t3 + S::LUT));
  if (threadIdx.x == 0) {
    for (int k = 0; k < S::NS; ++k) mbar_init(R.bar + k, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const float keep = 1.f - omega;
  bool failed = false;
  for_each_run(L, sc, [&](int x0, int y0, int z0, int z1) -> bool {
    const Th t = thread_geom(L, x0, y0);
    Diag D;
    if (!MASKED) D = unmasked_diag(L, t, omega);
    const int n = z1 - z0 + 4;
    if (threadIdx.x == 0)
      for (int k = 0; k < S::NS && k < n; ++k)
        issue_plane<T, TB, MASKED, false>(R, nullptr, &mb, nullptr, &mm, x0, y0, z0 - 2 + k);
    float S1Q[3][2][4], XQ[3][2][4], BQ[3][2][4], WQ[3][2][4], DQ[3][2][4], zp[2] = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 4; ++j) S1Q[k][h][j] = XQ[k][h][j] = BQ[k][h][j] = WQ[k][h][j] = DQ[k][h][j] = 0.f;
    auto step = [&](int i, auto phc) -> bool {
      constexpr int C0 = decltype(phc)::value;
      constexpr int C1 = (C0 + 2) % 3, C2 = (C0 + 1) % 3;
      const int p = z0 - 2 + i;
      const bool ok = mbar_wait_bounded(R.bar + R.g % S::NS, (R.g / S::NS) & 1);
      // A: b (and omega / d, d) of plane p and the first sweep from zero
      {
        const unsigned char* sg = R.base + (R.g % S::NS) * S::STAGE;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = 2 * t.q + h;
          float bv[4];
          lds4<TB>(sg + S::OB + (r * S::WB + S::MB - 4 + 4 * t.c) * (int)sizeof(TB), bv);
          if (MASKED) {
            const unsigned mw = *reinterpret_cast<const unsigned*>(sg + S::OM + r * S::WM + 12 + 4 * t.c);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const unsigned qq = (mw >> (8 * j)) & 63u;
              WQ[C0][h][j] = lut[64 + qq];
              DQ[C0][h][j] = lut[qq];
            }
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) BQ[C0][h][j] = bv[j];
        }
        auto first = [&](auto W) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < 4; ++j) S1Q[C0][h][j] = W(h, j) * BQ[C0][h][j];
        };
        if constexpr (MASKED) first([&](int h, int j) { return WQ[C0][h][j]; });
        else with_plane(plane_kz(L, p), D.w1, D.w2, first);
        sts8(S1 + (i & 1) * PL, t, S1Q[C0]);
      }
      // B: second sweep on plane p - 1; the output x
      if (i >= 2) {
        float nb[2][4];
        neighbours(L, t, S1 + ((i - 1) & 1) * PL, S1Q[C1], S1Q[C2], S1Q[C0], nb);
        auto sweep = [&](auto W) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < 4; ++j)
              XQ[C1][h][j] = fmaf(keep, S1Q[C1][h][j], W(h, j) * (BQ[C1][h][j] + nb[h][j]));
        };
        if constexpr (MASKED) sweep([&](int h, int j) { return WQ[C1][h][j]; });
        else with_plane(plane_kz(L, p - 1), D.w1, D.w2, sweep);
        sts8(XB + ((i - 1) & 1) * PL, t, XQ[C1]);
        const int o = p - 1;
        if (t.own && t.xin && o >= z0 && o < z1) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
            if (t.yin[h]) stg4<T>(x + ((size_t)o * L.ny + t.gy + h) * L.nx + t.gx, XQ[C1][h]);
        }
      }
      // C: residual on plane o = p - 2 and its 2x2x2 average (x pairs and
      // the row pair in registers, z pairs across consecutive steps)
      const int o = p - 2;
      if (i >= 4 && t.own) {
        float nb[2][4], rx[2] = {0.f, 0.f};
        neighbours(L, t, XB + (i & 1) * PL, XQ[C2], XQ[C0], XQ[C1], nb);
        // solid cells (d = 0) are not unknowns: no residual there; unmasked
        // cells outside the domain belong to threads that store nothing
        auto resid = [&](auto Dg) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const float dj = Dg(h, j);
              const float r = BQ[C2][h][j] - (dj * XQ[C2][h][j] - nb[h][j]);
              rx[j >> 1] += (MASKED && dj == 0.f) ? 0.f : r;
            }
        };
        if constexpr (MASKED) resid([&](int h, int j) { return DQ[C2][h][j]; });
        else with_plane(plane_kz(L, o), D.d1, D.d2, resid);
        if ((o & 1) == 0) {
          zp[0] = rx[0];
          zp[1] = rx[1];
        } else if (t.xin && t.yin[0]) {
          stg2<T>(bcoarse + ((size_t)(o >> 1) * (L.ny >> 1) + (t.gy >> 1)) * (L.nx >> 1) + (t.gx >> 1),
                  0.125f * (zp[0] + rx[0]), 0.125f * (zp[1] + rx[1]));
        }
      }
      if (__syncthreads_or(!ok)) {
        drain(R, R.g);
        return false;
      }
      if (threadIdx.x == 0 && i + S::NS < n)
        issue_plane<T, TB, MASKED, false>(R, nullptr, &mb, nullptr, &mm, x0, y0, z0 - 2 + i + S::NS);
      ++R.g;
      return true;
    };
    for (int i = 0; i < n; i += 3) {
      if (!step(i, std::integral_constant<int, 0>())) return !(failed = true);
      if (i + 1 >= n) break;
      if (!step(i + 1, std::integral_constant<int, 1>())) return !(failed = true);
      if (i + 2 >= n) break;
      if (!step(i + 2, std::integral_constant<int, 2>())) return !(failed = true);
    }
    return true;
  });
  if (failed) fail(st);
}

// ---- CG direction update --------------------------------------------------------
// p = z + beta p_old and Ap = A' p on the finest level (float32), with the
// same column geometry: one elected thread loads the planes of z and p_old
// (and the cell bytes); per plane step i the block forms p of plane
// z0 - 1 + i (A) and A' p of the plane below it (B), writes both and
// reduces (p, Ap); the last block sets CG's alpha.
template <bool MASKED>
struct GP {
  static constexpr int W = TX + 8;                 // z / p_old box width (x0 - 4 .. x0 + 131)
  static constexpr int ZB = W * RY * 4;            // bytes of one field box
  static constexpr int WM = TX + 32;
  static constexpr int MBY = MASKED ? WM * RY : 0;
  static constexpr int OZ = 0, OP = al128(ZB), OM = al128(OP + ZB);
  static constexpr int STAGE = al128(OM + MBY);
  // TMA stages: three, so that two blocks fit an SM (the kernel needs fewer
  // than 96 registers; twice the warps hide the per-plane barrier)
  static constexpr int NS = 3;
  static constexpr int RING = 2 * PL * 4;          // one plane buffer of two slots
  static constexpr int LUT = RING + NS * STAGE;
  static constexpr int BAR = LUT + 128 * 4;
  static constexpr int BYTES = BAR + NS * 8;
  static_assert(RING % 128 == 0 && STAGE % 128 == 0, "TMA destinations 128-byte aligned");
};

template <bool MASKED, int N>
__device__ __forceinline__ void issue_pz(Ring<N>& R, const CUtensorMap* mz, const CUtensorMap* mp,
                                         const CUtensorMap* mm, bool first, int x0, int y0, int p) {
  using S = GP<MASKED>;
  const unsigned st = R.issued % N;
  unsigned char* dst = R.base + st * S::STAGE;
  uint64_t* bar = R.bar + st;
  mbar_arrive_expect_tx(bar, (uint32_t)(S::ZB * (first ? 1 : 2) + S::MBY));
  tma_load_3d(dst + S::OZ, mz, bar, x0 - 4, y0 - 2, p);
  if (!first) tma_load_3d(dst + S::OP, mp, bar, x0 - 4, y0 - 2, p);
  if (MASKED) tma_load_3d(dst + S::OM, mm, bar, x0 - 16, y0 - 2, p);
  ++R.issued;
}

template <bool MASKED, bool STORE_AP>
__global__ void __launch_bounds__(NT, 2)
    k_pup_t3(const __grid_constant__ CUtensorMap mz, const __grid_constant__ CUtensorMap mp,
             const __grid_constant__ CUtensorMap mm, LevelDev L, float* __restrict__ pnew, float* __restrict__ Ap,
             Sched sc, SolveState* __restrict__ st, double* __restrict__ partials) {
  chain_enter();
  if (st->inner_done) return;
  using S = GP<MASKED>;
  extern __shared__ __align__(128) unsigned char smem_t3[];
  float* PS = reinterpret_cast<float*>(smem_t3);  // [2][PL]: p
  const float* lut = reinterpret_cast<const float*>(smem_t3 + S::LUT);
  Ring<S::NS> R;
  R.bar = reinterpret_cast<uint64_t*>(smem_t3 + S::BAR);
  R.base = smem_t3 + S::RING;
  R.g = R.issued = 0;
  const bool first = st->first || !st->krylov;
  const float beta = first ? 0.f : (float)st->beta;
  if (MASKED) fill_lut(L, 1.f, reinterpret_cast<float*>(smem_t3 + S::LUT));
  if (threadIdx.x == 0) {
    for (int k = 0; k < S::NS; ++k) mbar_init(R.bar + k, 1);
    fence_mbar_init();
  }
  __syncthreads();
  float acc = 0.f;
  bool failed = false;
  for_each_run(L, sc, [&](int x0, int y0, int z0, int z1) -> bool {
    const Th t = thread_geom(L, x0, y0);
    Diag D;
    if (!MASKED) D = unmasked_diag(L, t, 1.f);
    const int n = z1 - z0 + 2;  // steps: A on planes z0 - 1 .. z1
    if (threadIdx.x == 0)
      for (int k = 0; k < S::NS && k < n; ++k) issue_pz<MASKED>(R, &mz, &mp, &mm, first, x0, y0, z0 - 1 + k);
    float PQ[3][2][4], DQ[3][2][4];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 4; ++j) PQ[k][h][j] = DQ[k][h][j] = 0.f;
    auto step = [&](int i, auto phc) -> bool {
      constexpr int C0 = decltype(phc)::value;             // i % 3
      constexpr int C1 = (C0 + 2) % 3, C2 = (C0 + 1) % 3;  // (i - 1) % 3, (i - 2) % 3
      const int p = z0 - 1 + i;
      const bool ok = mbar_wait_bounded(R.bar + R.g % S::NS, (R.g / S::NS) & 1);
      // A: p = z + beta p_old of plane p (0 outside the domain: zero fill)
      {
        const unsigned char* sg = R.base + (R.g % S::NS) * S::STAGE;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = 2 * t.q + h;
          float zv[4], qv[4] = {0.f, 0.f, 0.f, 0.f};
          lds4<float>(sg + S::OZ + (r * S::W + 4 * t.c) * 4, zv);
          if (!first) lds4<float>(sg + S::OP + (r * S::W + 4 * t.c) * 4, qv);
          if (MASKED) {
            const unsigned mw = *reinterpret_cast<const unsigned*>(sg + S::OM + r * S::WM + 12 + 4 * t.c);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const unsigned m = (mw >> (8 * j)) & 0xffu;
              DQ[C0][h][j] = lut[m & 63u];
              PQ[C0][h][j] = m ? fmaf(beta, qv[j], zv[j]) : 0.f;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) PQ[C0][h][j] = fmaf(beta, qv[j], zv[j]);
          }
        }
        sts8(PS + (i & 1) * PL, t, PQ[C0]);
      }
      // B: A' p on plane o = p - 1, written with p; (p, Ap) reduced
      const int o = p - 1;
      if (i >= 2 && t.own) {
        float nb[2][4];
        neighbours(L, t, PS + ((i - 1) & 1) * PL, PQ[C1], PQ[C2], PQ[C0], nb);
        auto apply = [&](auto Dg) {
          if (!t.xin) return;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (!t.yin[h]) continue;
            float av[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const float d = Dg(h, j);
              av[j] = d != 0.f ? d * PQ[C1][h][j] - nb[h][j] : 0.f;
              acc = fmaf(PQ[C1][h][j], av[j], acc);
            }
            const size_t gi = ((size_t)o * L.ny + t.gy + h) * L.nx + t.gx;
            stg4<float>(pnew + gi, PQ[C1][h]);
            if (STORE_AP) stg4<float>(Ap + gi, av);
          }
        };
        if constexpr (MASKED) apply([&](int h, int j) { return DQ[C1][h][j]; });
        else with_plane(plane_kz(L, o), D.d1, D.d2, apply);
      }
      if (__syncthreads_or(!ok)) {
        drain(R, R.g);
        return false;
      }
      if (threadIdx.x == 0 && i + S::NS < n) issue_pz<MASKED>(R, &mz, &mp, &mm, first, x0, y0, z0 - 1 + i + S::NS);
      ++R.g;
      return true;
    };
    for (int i = 0; i < n; i += 3) {
      if (!step(i, std::integral_constant<int, 0>())) return !(failed = true);
      if (i + 1 >= n) break;
      if (!step(i + 1, std::integral_constant<int, 1>())) return !(failed = true);
      if (i + 2 >= n) break;
      if (!step(i + 2, std::integral_constant<int, 2>())) return !(failed = true);
    }
    return true;
  });
  if (failed) fail(st);
  double tot;
  if (grid_sum_last((double)acc, partials, &st->counter[kCntPAP], &tot)) {
    if (threadIdx.x == 0 && !failed) {
      st->pAp = tot;
      st->alpha = st->krylov ? st->rz / tot : 1.0;
    }
  }
}

// ---- CG vector update -------------------------------------------------------------
// d += alpha p, r -= alpha A' p and ||r||^2 on the finest level (float32),
// with A' p formed again from p (bit for bit the values the direction update
// reduced (p, A' p) from) instead of being stored by it and read back: the
// elected thread loads the plane of p (with its halo) and, into the same
// stage, the planes of d and r one below it; per step the block forms A' p
// of the plane below the new p and updates d and r there.  The last block
// takes CG's convergence decision (inner_decide).
template <bool MASKED>
struct GX {
  static constexpr int W = TX + 8;                 // p box width (x0 - 4 .. x0 + 131)
  static constexpr int PB = W * RY * 4;            // bytes of the p box
  static constexpr int VB = TX * TY * 4;           // bytes of a d / r box (the column's own cells)
  static constexpr int WM = TX + 32;
  static constexpr int MBY = MASKED ? WM * RY : 0;
  static constexpr int OP = 0, OD = al128(PB), OR = al128(OD + VB), OM = al128(OR + VB);
  static constexpr int STAGE = al128(OM + MBY);
  static constexpr int NS = 5;                     // TMA stages
  static constexpr int RING = 2 * PL * 4;          // one plane buffer of two slots
  static constexpr int LUT = RING + NS * STAGE;
  static constexpr int BAR = LUT + 128 * 4;
  static constexpr int BYTES = BAR + NS * 8;
  static_assert(RING % 128 == 0 && STAGE % 128 == 0, "TMA destinations 128-byte aligned");
};

template <bool MASKED, int N>
__device__ __forceinline__ void issue_xr(Ring<N>& R, const CUtensorMap* mp, const CUtensorMap* md,
                                         const CUtensorMap* mr, const CUtensorMap* mm, bool first, int x0, int y0,
                                         int p) {
  using S = GX<MASKED>;
  const unsigned st = R.issued % N;
  unsigned char* dst = R.base + st * S::STAGE;
  uint64_t* bar = R.bar + st;
  mbar_arrive_expect_tx(bar, (uint32_t)(S::PB + S::VB * (first ? 1 : 2) + S::MBY));
  tma_load_3d(dst + S::OP, mp, bar, x0 - 4, y0 - 2, p);
  if (!first) tma_load_3d(dst + S::OD, md, bar, x0, y0, p - 1);
  tma_load_3d(dst + S::OR, mr, bar, x0, y0, p - 1);
  if (MASKED) tma_load_3d(dst + S::OM, mm, bar, x0 - 16, y0 - 2, p);
  ++R.issued;
}

template <bool MASKED>
__global__ void __launch_bounds__(NT, 1)
    k_xr_t3(const __grid_constant__ CUtensorMap mp, const __grid_constant__ CUtensorMap md,
            const __grid_constant__ CUtensorMap mr, const __grid_constant__ CUtensorMap mm, LevelDev L,
            float* __restrict__ d, float* __restrict__ r, Sched sc, SolveState* __restrict__ st,
            double* __restrict__ partials) {
  chain_enter();
  if (st->inner_done) return;
  using S = GX<MASKED>;
  extern __shared__ __align__(128) unsigned char smem_t3[];
  float* PS = reinterpret_cast<float*>(smem_t3);  // [2][PL]: p
  const float* lut = reinterpret_cast<const float*>(smem_t3 + S::LUT);
  Ring<S::NS> R;
  R.bar = reinterpret_cast<uint64_t*>(smem_t3 + S::BAR);
  R.base = smem_t3 + S::RING;
  R.g = R.issued = 0;
  const bool first = st->first;
  const float alpha = (float)st->alpha;
  if (MASKED) fill_lut(L, 1.f, reinterpret_cast<float*>(smem_t3 + S::LUT));
  if (threadIdx.x == 0) {
    for (int k = 0; k < S::NS; ++k) mbar_init(R.bar + k, 1);
    fence_mbar_init();
  }
  __syncthreads();
  float acc = 0.f;
  bool failed = false;
  for_each_run(L, sc, [&](int x0, int y0, int z0, int z1) -> bool {
    const Th t = thread_geom(L, x0, y0);
    Diag D;
    if (!MASKED) D = unmasked_diag(L, t, 1.f);
    const int n = z1 - z0 + 2;  // steps: p on planes z0 - 1 .. z1
    if (threadIdx.x == 0)
      for (int k = 0; k < S::NS && k < n; ++k) issue_xr<MASKED>(R, &mp, &md, &mr, &mm, first, x0, y0, z0 - 1 + k);
    float PQ[3][2][4], DQ[3][2][4];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 4; ++j) PQ[k][h][j] = DQ[k][h][j] = 0.f;
    auto step = [&](int i, auto phc) -> bool {
      constexpr int C0 = decltype(phc)::value;             // i % 3
      constexpr int C1 = (C0 + 2) % 3, C2 = (C0 + 1) % 3;  // (i - 1) % 3, (i - 2) % 3
      const int p = z0 - 1 + i;
      const bool ok = mbar_wait_bounded(R.bar + R.g % S::NS, (R.g / S::NS) & 1);
      const unsigned char* sg = R.base + (R.g % S::NS) * S::STAGE;
      // A: p of plane p (0 on solid cells and outside the domain)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int rr = 2 * t.q + h;
        lds4<float>(sg + S::OP + (rr * S::W + 4 * t.c) * 4, PQ[C0][h]);
        if (MASKED) {
          const unsigned mw = *reinterpret_cast<const unsigned*>(sg + S::OM + rr * S::WM + 12 + 4 * t.c);
#pragma unroll
          for (int j = 0; j < 4; ++j) DQ[C0][h][j] = lut[(mw >> (8 * j)) & 63u];
        }
      }
      sts8(PS + (i & 1) * PL, t, PQ[C0]);
      // B: A' p on plane o = p - 1; d and r of plane o from this stage
      const int o = p - 1;
      if (i >= 2 && t.own) {
        float nb[2][4];
        neighbours(L, t, PS + ((i - 1) & 1) * PL, PQ[C1], PQ[C2], PQ[C0], nb);
        auto update = [&](auto Dg) {
          if (!t.xin) return;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (!t.yin[h]) continue;
            const int off = ((2 * t.q - 2 + h) * TX + 4 * (t.c - 1)) * 4;  // own row / chunk in a d, r box
            float dv[4], rv[4];
            lds4<float>(sg + S::OR + off, rv);
            if (!first) lds4<float>(sg + S::OD + off, dv);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const float dd = Dg(h, j);
              const float av = dd != 0.f ? dd * PQ[C1][h][j] - nb[h][j] : 0.f;
              dv[j] = first ? alpha * PQ[C1][h][j] : fmaf(alpha, PQ[C1][h][j], dv[j]);
              rv[j] = fmaf(-alpha, av, rv[j]);
              acc = fmaf(rv[j], rv[j], acc);
            }
            const size_t gi = ((size_t)o * L.ny + t.gy + h) * L.nx + t.gx;
            stg4<float>(d + gi, dv);
            stg4<float>(r + gi, rv);
          }
        };
        if constexpr (MASKED) update([&](int h, int j) { return DQ[C1][h][j]; });
        else with_plane(plane_kz(L, o), D.d1, D.d2, update);
      }
      if (__syncthreads_or(!ok)) {
        drain(R, R.g);
        return false;
      }
      if (threadIdx.x == 0 && i + S::NS < n)
        issue_xr<MASKED>(R, &mp, &md, &mr, &mm, first, x0, y0, z0 - 1 + i + S::NS);
      ++R.g;
      return true;
    };
    for (int i = 0; i < n; i += 3) {
      if (!step(i, std::integral_constant<int, 0>())) return !(failed = true);
      if (i + 1 >= n) break;
      if (!step(i + 1, std::integral_constant<int, 1>())) return !(failed = true);
      if (i + 2 >= n) break;
      if (!step(i + 2, std::integral_constant<int, 2>())) return !(failed = true);
    }
    return true;
  });
  if (failed) fail(st);
  double tot;
  if (grid_sum_last((double)acc, partials, &st->counter[kCntRR], &tot)) {
    if (threadIdx.x == 0 && !failed) inner_decide(st, tot);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
static int t3_sms() {
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
// column, the run count minimising waves x (zr + 4 halo planes), or an even
// split of the column-major (column, plane) units over one block per SM,
// each block paying 4 halo planes per column it touches; the cheaper of the
// two.
struct T3Plan {
  Sched sc;
  dim3 grid;
};

// bps: blocks of the kernel an SM holds at once.
static T3Plan t3_plan(const LevelDev& L, int bps = 1) {
  const long strips = (L.nx + TX - 1) / TX, tiles = (L.ny + TY - 1) / TY;
  const long cols = strips * tiles;
  const long nsm = (long)t3_sms() * bps;
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
  T3Plan p;
  p.sc.zr = (int)best_zr;
  p.sc.units = 0;
  p.grid = dim3((unsigned)strips, (unsigned)tiles, (unsigned)((L.nz + best_zr - 1) / best_zr));
  const long total = cols * L.nz;
  long units = (total + nsm - 1) / nsm;
  units = (units + 1) / 2 * 2;  // runs start on even planes (restriction pairs)
  const long touched = (units + L.nz - 2) / L.nz + 1;
  if (units + 4 * touched < best) {
    p.sc.units = (int)units;
    p.grid = dim3((unsigned)((total + units - 1) / units), 1, 1);
  }
  return p;
}

// Smallest level (cells) taken by these kernels: 2^15, or NPMG_TMA3D_MIN.
bool tma3d_eligible(int dim, int pre, int post, const LevelDev& L) {
  if (getenv("NPMG_NO_TMA3D")) return false;
  const char* e = getenv("NPMG_TMA3D_MIN");
  const size_t lim = e ? (size_t)atol(e) : ((size_t)1 << 15);
  return dim == 3 && pre == 2 && post == 2 && L.nx % 16 == 0 && L.ny % 2 == 0 && L.nz % 2 == 0 && L.nz >= 4 &&
         (size_t)L.nx * L.ny * L.nz >= lim && tensor_map_encoder() != nullptr;
}

template <typename T>
static CUtensorMapDataType dtype3() {
  if (std::is_same<T, float>::value) return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  if (std::is_same<T, __half>::value) return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  if (std::is_same<T, __nv_bfloat16>::value) return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  return CU_TENSOR_MAP_DATA_TYPE_UINT8;
}

static bool encode_3d(CUtensorMap* m, const void* base, CUtensorMapDataType dt, int esz, int64_t nx, int64_t ny,
                      int64_t nz, int bw, int bh) {
  auto fn = (PFN_cuTensorMapEncodeTiled_v12000)tensor_map_encoder();
  if (!fn || !base || ((uintptr_t)base & 15) || ((nx * esz) & 15)) return false;
  cuuint64_t gdim[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  cuuint64_t gstride[2] = {(cuuint64_t)(nx * esz), (cuuint64_t)(nx * ny * esz)};
  cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, dt, 3, const_cast<void*>(base), gdim, gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

template <typename T, typename TB>
bool tma3d_encode(Tma3Maps* out, const LevelDev& L, const void* b, const void* x, const void* e) {
  using S = G3<T, TB, true, true>;
  bool ok = encode_3d(&out->b, b, dtype3<TB>(), (int)sizeof(TB), L.nx, L.ny, L.nz, S::WB, RY);
  ok = ok && encode_3d(&out->x, x, dtype3<T>(), (int)sizeof(T), L.nx, L.ny, L.nz, S::WX, RY);
  ok = ok && encode_3d(&out->e, e, dtype3<T>(), (int)sizeof(T), L.nx / 2, L.ny / 2, L.nz / 2, S::WE, S::EY);
  if (L.cell) ok = ok && encode_3d(&out->m, L.cell, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, L.nx, L.ny, L.nz, S::WM, RY);
  else out->m = out->b;  // unused
  return ok;
}

template <typename TB>
bool tma3d_encode_b(CUtensorMap* out, const LevelDev& L, const void* b) {
  using S = G3<TB, TB, false, false>;
  return encode_3d(out, b, dtype3<TB>(), (int)sizeof(TB), L.nx, L.ny, L.nz, S::WB, RY);
}

template <typename T, bool MASKED, typename TB>
cudaError_t launch_down_t3(const Tma3Maps& m, const LevelDev& L, void* x, void* bcoarse, float omega,
                           const SolveState* st, cudaStream_t s) {
  const T3Plan pl = t3_plan(L);
  return launch_chain(k_down_t3<T, MASKED, TB>, pl.grid, NT, (size_t)G3<T, TB, MASKED, false>::BYTES, s, m.b, m.m,
                      L, (T*)x, (T*)bcoarse, omega, pl.sc, const_cast<SolveState*>(st));
}

template <typename T, bool MASKED, bool FINEST, typename TB>
cudaError_t launch_up_t3(const Tma3Maps& m, const LevelDev& L, void* xout, float omega, float sc, SolveState* st,
                         double* partials, cudaStream_t s) {
  const T3Plan pl = t3_plan(L);
  return launch_chain(k_up_t3<T, MASKED, FINEST, TB>, pl.grid, NT, (size_t)G3<T, TB, MASKED, true>::BYTES, s, m.x,
                      m.b, m.e, m.m, L, (TB*)xout, omega, sc, pl.sc, st, partials);
}

bool tma3d_encode_cg(Tma3CgMaps* out, const LevelDev& L, const float* z, const float* p0, const float* p1,
                     const float* d, const float* r) {
  constexpr int W = GP<false>::W;
  bool ok = encode_3d(&out->z, z, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, L.nx, L.ny, L.nz, W, RY);
  ok = ok && encode_3d(&out->d, d, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, L.nx, L.ny, L.nz, TX, TY);
  ok = ok && encode_3d(&out->r, r, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, L.nx, L.ny, L.nz, TX, TY);
  ok = ok && encode_3d(&out->p[0], p0, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, L.nx, L.ny, L.nz, W, RY);
  ok = ok && encode_3d(&out->p[1], p1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, L.nx, L.ny, L.nz, W, RY);
  if (L.cell)
    ok = ok && encode_3d(&out->m, L.cell, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, L.nx, L.ny, L.nz, GP<true>::WM, RY);
  else out->m = out->z;  // unused
  return ok;
}

template <bool MASKED>
cudaError_t launch_p_update_t3(const Tma3CgMaps& m, int parity, const LevelDev& L, float* pnew, float* Ap,
                               bool store_ap, SolveState* st, double* partials, cudaStream_t s) {
  const T3Plan pl = t3_plan(L, 2);
  if (store_ap)
    return launch_chain(k_pup_t3<MASKED, true>, pl.grid, NT, (size_t)GP<MASKED>::BYTES, s, m.z, m.p[parity], m.m, L,
                        pnew, Ap, pl.sc, st, partials);
  return launch_chain(k_pup_t3<MASKED, false>, pl.grid, NT, (size_t)GP<MASKED>::BYTES, s, m.z, m.p[parity], m.m, L,
                      pnew, Ap, pl.sc, st, partials);
}
template cudaError_t launch_p_update_t3<false>(const Tma3CgMaps&, int, const LevelDev&, float*, float*, bool,
                                               SolveState*, double*, cudaStream_t);
template cudaError_t launch_p_update_t3<true>(const Tma3CgMaps&, int, const LevelDev&, float*, float*, bool,
                                              SolveState*, double*, cudaStream_t);

template <bool MASKED>
cudaError_t launch_xr_update_t3(const Tma3CgMaps& m, int pbuf, const LevelDev& L, float* d, float* r,
                                SolveState* st, double* partials, cudaStream_t s) {
  const T3Plan pl = t3_plan(L);
  return launch_chain(k_xr_t3<MASKED>, pl.grid, NT, (size_t)GX<MASKED>::BYTES, s, m.p[pbuf], m.d, m.r, m.m, L, d, r,
                      pl.sc, st, partials);
}
template cudaError_t launch_xr_update_t3<false>(const Tma3CgMaps&, int, const LevelDev&, float*, float*, SolveState*,
                                                double*, cudaStream_t);
template cudaError_t launch_xr_update_t3<true>(const Tma3CgMaps&, int, const LevelDev&, float*, float*, SolveState*,
                                               double*, cudaStream_t);

template <typename T, bool MASKED, typename TB>
static cudaError_t prepare_t3_pair() {
  cudaError_t e = cudaFuncSetAttribute(k_down_t3<T, MASKED, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       G3<T, TB, MASKED, false>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_up_t3<T, MASKED, false, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             G3<T, TB, MASKED, true>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_up_t3<T, MASKED, true, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             G3<T, TB, MASKED, true>::BYTES);
  return e;
}

template <typename T, bool MASKED>
cudaError_t prepare_t3_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_pup_t3<MASKED, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       GP<MASKED>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_pup_t3<MASKED, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, GP<MASKED>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_xr_t3<MASKED>, cudaFuncAttributeMaxDynamicSharedMemorySize, GX<MASKED>::BYTES);
  if (e == cudaSuccess) e = prepare_t3_pair<T, MASKED, T>();
  if (e == cudaSuccess && !std::is_same<T, float>::value) e = prepare_t3_pair<T, MASKED, float>();
  return e;
}

#define NPMG_INST_T3_TB(T, M, TB)                                                                                  \
  template cudaError_t launch_down_t3<T, M, TB>(const Tma3Maps&, const LevelDev&, void*, void*, float,              \
                                                const SolveState*, cudaStream_t);                                  \
  template cudaError_t launch_up_t3<T, M, false, TB>(const Tma3Maps&, const LevelDev&, void*, float, float,         \
                                                     SolveState*, double*, cudaStream_t);                           \
  template cudaError_t launch_up_t3<T, M, true, TB>(const Tma3Maps&, const LevelDev&, void*, float, float,          \
                                                    SolveState*, double*, cudaStream_t);
#define NPMG_INST_T3(T, M)                         \
  template cudaError_t prepare_t3_kernels<T, M>(); \
  NPMG_INST_T3_TB(T, M, T)                         \
  NPMG_INST_T3_TB(T, M, float)

template cudaError_t prepare_t3_kernels<float, false>();
template cudaError_t prepare_t3_kernels<float, true>();
NPMG_INST_T3_TB(float, false, float)
NPMG_INST_T3_TB(float, true, float)
NPMG_INST_T3(__half, false)
NPMG_INST_T3(__half, true)
NPMG_INST_T3(__nv_bfloat16, false)
NPMG_INST_T3(__nv_bfloat16, true)

template bool tma3d_encode<float, float>(Tma3Maps*, const LevelDev&, const void*, const void*, const void*);
template bool tma3d_encode<__half, __half>(Tma3Maps*, const LevelDev&, const void*, const void*, const void*);
template bool tma3d_encode<__half, float>(Tma3Maps*, const LevelDev&, const void*, const void*, const void*);
template bool tma3d_encode<__nv_bfloat16, __nv_bfloat16>(Tma3Maps*, const LevelDev&, const void*, const void*,
                                                         const void*);
template bool tma3d_encode<__nv_bfloat16, float>(Tma3Maps*, const LevelDev&, const void*, const void*, const void*);
template bool tma3d_encode_b<float>(CUtensorMap*, const LevelDev&, const void*);
template bool tma3d_encode_b<__half>(CUtensorMap*, const LevelDev&, const void*);
template bool tma3d_encode_b<__nv_bfloat16>(CUtensorMap*, const LevelDev&, const void*);

}  // namespace npmg
