// 2D level kernels with two Jacobi sweeps, streamed along y by single warps.
//
// A warp owns a strip of 128 consecutive cells of a row (4 per lane, one
// 16-byte vector per float32 array) and walks a run of R rows.  The two
// sweeps and the residual of one output row need the rows one and two away
// in y, so every lane keeps three-row rings of its cells in registers and
// works with a skew: when row p arrives it forms the first sweep's input
// there, the first sweep on row p - 1 and the second sweep (up) or the
// residual (down) on row p - 2.  Neighbours in x come from the adjacent
// lanes by warp shuffles; lanes 0 and 31 also hold the two cells beyond the
// strip on their side (the inner and outer halo), which is what two sweeps
// need.  Rows arrive through a per-warp ring of shared-memory slots filled
// by asynchronous copies four rows ahead of the row in use; each lane reads
// back only what it copied itself, so there is no barrier of any kind.
//
// Same arithmetic as the tiled level kernels: weighted Jacobi
// (Eq. Jacobi-1-relax) written x <- (1 - omega) x + (omega / d)(b + nb),
// from a zero guess on the down leg (the first sweep is then (omega / d) b),
// residual and 2x2 average restriction (App. B), copy prolongation plus the
// scaled correction and two post sweeps on the up leg (Sec. 2.2); cells
// outside the domain and solid cells hold 0 (the zero padding of Sec. 2.1).
// On the finest level the up leg also reduces (r, z) and CG's beta.
#include <algorithm>
#include <stdlib.h>

#include "launch.h"
#include "mg_kernels.cuh"

namespace npmg {

namespace {

constexpr int kWPB = 4;         // warps per block (independent strips / runs)
constexpr int V = 4;            // cells per lane (one 16-byte float32 vector)
constexpr int kD = 4;           // rows in flight ahead of the row in use
constexpr int kSlots = kD + 1;  // ring slots per warp (the slot refilled was read a step earlier)

// ---- asynchronous copies into the warp's ring (cp.async; a copy whose
// source is outside the domain zero-fills its bytes and reads nothing) -----
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
template <int N>
__device__ __forceinline__ void cp_async(uint32_t dst, const void* src, bool full) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(dst), "l"(src), "n"(N), "r"(full ? N : 0)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_ring() { asm volatile("cp.async.wait_group %0;\n" ::"n"(kD - 1) : "memory"); }

// ---- shared-memory reads of consecutive T as float -------------------------
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

// ---- ring slot layout (bytes) ----------------------------------------------
// Own cells of all lanes (lane-major vectors), then the halo of each side:
// side 0 is lane 0's (cells x0 - 2, x0 - 1; coarse parent x0/2 - 1; cell
// bytes x0 - 4 .. x0 - 1), side 1 lane 31's (x0 + 128, x0 + 129; parent
// x0/2 + 64; bytes x0 + 128 .. x0 + 131), each as an aligned pair / word.
template <typename T, typename TB, bool MASKED, bool UP>
struct Slot {
  static constexpr int SZ = (int)sizeof(T), SB = (int)sizeof(TB);
  static constexpr int B = UP ? 128 * SZ : 0;              // TB[128] b (T[128] x at 0, up only)
  static constexpr int E = B + 128 * SB;                   // T[64] e (up)
  static constexpr int M = E + (UP ? 64 * SZ : 0);         // u8[128] cell bytes (masked)
  static constexpr int H = M + (MASKED ? 128 : 0);         // 2 sides x 32 bytes: x pair, b pair, e pair, bytes
  static constexpr int BYTES = H + 64;
  static_assert(BYTES % 16 == 0, "slots keep 16-byte alignment");
};

// ---- lane geometry -----------------------------------------------------------
// Own cells gx .. gx + 3 (all inside the domain or all outside: nx is a
// multiple of 4); halo cells: lane 0 x0 - 1 (inner) and x0 - 2 (outer),
// lane 31 x0 + 128 (inner) and x0 + 129 (outer), both inside or both
// outside.
struct Lane {
  int lane, gx, hin, hout;
  int hpair, epair, mword;  // first element of the halo pair / parent pair / cell-byte word
  bool ox, hok;
  // unmasked levels: omega / d of the own cells and the halo on interior
  // rows (ky = 2) and on rows of a Neumann y face (ky = 1); d of own cells
  // without the y part
  float wI[V + 2], wB[V + 2], dx[V];
  float tabw, tabd;  // masked levels: this lane's entry of the 16-entry LUTs
};

template <bool MASKED>
__device__ __forceinline__ Lane lane_of(const LevelDev& L, int x0, float omega) {
  Lane c;
  c.lane = threadIdx.x & 31;
  c.gx = x0 + V * c.lane;
  c.ox = c.gx < L.nx;
  const bool left = c.lane == 0;
  c.hin = left ? x0 - 1 : x0 + 32 * V;
  c.hout = left ? x0 - 2 : x0 + 32 * V + 1;
  c.hpair = left ? x0 - 2 : x0 + 32 * V;
  c.epair = left ? (x0 >> 1) - 2 : (x0 >> 1) + 16 * V;
  c.mword = left ? x0 - 4 : x0 + 32 * V;
  c.hok = (left || c.lane == 31) && c.hout >= 0 && c.hout < L.nx;
  if (MASKED) {
    // link counts (kx + 4 ky, each 0..2) -> d and omega / d; 0 off the fluid
    const int kx = c.lane & 3, ky = (c.lane >> 2) & 3;
    const float d = (c.lane < 16 && kx <= 2 && ky <= 2) ? L.wx * (float)kx + L.wy * (float)ky : 0.f;
    c.tabd = d;
    c.tabw = d > 0.f ? omega / d : 0.f;
  } else {
#pragma unroll
    for (int j = 0; j < V + 2; ++j) {
      const int x = j < V ? c.gx + j : (j == V ? c.hin : c.hout);
      const bool in = j < V ? c.ox : c.hok;
      const float ddx = in ? L.wx * (float)axis_count(x, L.nx, L.bcD, 0) : 0.f;
      if (j < V) c.dx[j] = ddx;
      const float dI = ddx + 2.f * L.wy, dB = ddx + L.wy;
      c.wI[j] = in ? omega / dI : 0.f;
      c.wB[j] = in ? omega / dB : 0.f;
    }
  }
  return c;
}

// x-neighbours of the first and last own cell of a row of values a (own
// cells, then the inner halo): from the adjacent lanes, or the inner halo on
// lanes 0 and 31.  Every lane executes both shuffles (full-warp masks).
__device__ __forceinline__ void edge_neighbours(const Lane& c, const float* a, float& left, float& right) {
  const float up = __shfl_up_sync(0xffffffffu, a[V - 1], 1);
  const float dn = __shfl_down_sync(0xffffffffu, a[0], 1);
  left = c.lane == 0 ? a[V] : up;
  right = c.lane == 31 ? a[V] : dn;
}

// omega / d of the lane's positions 0 .. N-1 of row p (unmasked), or from
// the cell bytes m[j] (masked; every lane executes the shuffles).
template <bool MASKED, int N>
__device__ __forceinline__ void row_w(const LevelDev& L, const Lane& c, int p, const unsigned (&m)[N], float (&w)[N]) {
  if (MASKED) {
#pragma unroll
    for (int j = 0; j < N; ++j) w[j] = __shfl_sync(0xffffffffu, c.tabw, (int)(m[j] & 15u));
  } else {
    const bool rin = p >= 0 && p < L.ny;
    const bool brow = axis_count(p, L.ny, L.bcD, 2) != 2;
#pragma unroll
    for (int j = 0; j < N; ++j) w[j] = rin ? (brow ? c.wB[j] : c.wI[j]) : 0.f;
  }
}

// Halo values of a slot for this lane: (inner, outer) of a pair and the
// inner / outer cell bytes (lanes other than 0 and 31 read side 0 and never
// use the result).
template <typename T>
__device__ __forceinline__ void halo_of(const Lane& c, const unsigned char* hs, int off, float& inner, float& outer) {
  const float2 v = lds2<T>(hs + off);
  inner = c.lane == 0 ? v.y : v.x;
  outer = c.lane == 0 ? v.x : v.y;
}
__device__ __forceinline__ void halo_bytes(const Lane& c, const unsigned char* hs, unsigned& inner, unsigned& outer) {
  const unsigned w = *reinterpret_cast<const unsigned*>(hs + 24);
  inner = c.lane == 0 ? (w >> 24) : (w & 0xffu);
  outer = c.lane == 0 ? ((w >> 16) & 0xffu) : ((w >> 8) & 0xffu);
}

// Step i of a run uses row y0 - 2 + i from slot i % kSlots; the copies for
// row p + kD go to slot (i + kD) % kSlots, which was read at step i - 1.
__device__ __forceinline__ int slot_of(int i) { return i % kSlots; }

// ---- up leg ------------------------------------------------------------------
template <typename T, typename TB, bool MASKED>
__device__ __forceinline__ void up_issue(const LevelDev& L, const Lane& c, int r, bool want, const TB* __restrict__ b,
                                         const T* __restrict__ xin, const T* __restrict__ e, unsigned char* slot) {
  using S = Slot<T, TB, MASKED, true>;
  if (want) {
    const bool rin = r >= 0 && r < L.ny;
    const bool fo = rin && c.ox, fh = rin && c.hok;
    const size_t row = rin ? (size_t)r * L.nx : 0, crow = rin ? (size_t)(r >> 1) * (L.nx >> 1) : 0;
    const int go = fo ? c.gx : 0;  // zero-fill copies keep an in-bounds source
    const uint32_t sl = smem_addr(slot);
    cp_async<4 * S::SZ>(sl + c.lane * 4 * S::SZ, xin + row + go, fo);
    cp_async<4 * S::SB>(sl + S::B + c.lane * 4 * S::SB, b + row + go, fo);
    cp_async<2 * S::SZ>(sl + S::E + c.lane * 2 * S::SZ, e + crow + (go >> 1), fo);
    if (MASKED) cp_async<4>(sl + S::M + c.lane * 4, L.cell + row + go, fo);
    if (c.lane == 0 || c.lane == 31) {
      const uint32_t hs = sl + S::H + (c.lane == 31 ? 32 : 0);
      cp_async<2 * S::SZ>(hs, xin + row + (fh ? c.hpair : 0), fh);
      cp_async<2 * S::SB>(hs + 8, b + row + (fh ? c.hpair : 0), fh);
      cp_async<2 * S::SZ>(hs + 16, e + crow + (fh ? c.epair : 0), fh);
      if (MASKED) cp_async<4>(hs + 24, L.cell + row + (fh ? c.mword : 0), fh);
    }
  }
  cp_commit();
}

struct UpRegs {
  float s0[3][V + 2];  // x + s P e: own cells, inner halo, outer halo
  float s1[3][V + 1];  // first sweep: own cells, inner halo
  float b[3][V + 1];
  float w[3][V + 1];   // omega / d, 0 off the fluid
};

// One row step with register slots C (row p), P (row p - 1), Q (row p - 2).
template <typename T, typename TB, bool MASKED, bool FINEST, int C, int P, int Q>
__device__ __forceinline__ void up_step(const LevelDev& L, const Lane& c, int i, int y0, int y1, float omega, float s,
                                        const TB* __restrict__ b, const T* __restrict__ xin, const T* __restrict__ e,
                                        TB* __restrict__ xout, unsigned char* ring, UpRegs& R, float& acc) {
  using S = Slot<T, TB, MASKED, true>;
  const int p = y0 - 2 + i;
  // row p from its slot: x + s P e on the own cells and both halo cells, b
  // and omega / d
  cp_wait_ring();
  {
    const unsigned char* sl = ring + slot_of(i) * S::BYTES;
    float xv[V], bv[V];
    lds4<T>(sl + c.lane * 4 * S::SZ, xv);
    lds4<TB>(sl + S::B + c.lane * 4 * S::SB, bv);
    const float2 ev = lds2<T>(sl + S::E + c.lane * 2 * S::SZ);
    const unsigned char* hs = sl + S::H + (c.lane == 31 ? 32 : 0);
    float xh, xo, bh, bo, eh, eo;
    halo_of<T>(c, hs, 0, xh, xo);
    halo_of<TB>(c, hs, 8, bh, bo);
    halo_of<T>(c, hs, 16, eh, eo);
    (void)bo;
    (void)eo;
    unsigned m[V + 1], mo = 0u;
    if (MASKED) {
      const unsigned mw = *reinterpret_cast<const unsigned*>(sl + S::M + c.lane * 4);
#pragma unroll
      for (int j = 0; j < V; ++j) m[j] = (mw >> (8 * j)) & 0xffu;
      halo_bytes(c, hs, m[V], mo);
    } else {
#pragma unroll
      for (int j = 0; j <= V; ++j) m[j] = 0u;
    }
    float w[V + 1];
    row_w<MASKED, V + 1>(L, c, p, m, w);
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const float v = fmaf(s, j < 2 ? ev.x : ev.y, xv[j]);
      R.s0[C][j] = (!MASKED || m[j]) ? v : 0.f;
      R.b[C][j] = bv[j];
      R.w[C][j] = w[j];
    }
    const float vh = fmaf(s, eh, xh), vo = fmaf(s, eh, xo);
    R.s0[C][V] = (!MASKED || m[V]) ? vh : 0.f;
    R.s0[C][V + 1] = (!MASKED || mo) ? vo : 0.f;
    R.b[C][V] = bh;
    R.w[C][V] = w[V];
  }
  up_issue<T, TB, MASKED>(L, c, p + kD, p + kD <= y1 + 1, b, xin, e, ring + slot_of(i + kD) * S::BYTES);
  const float keep = 1.f - omega;
  // first sweep on row p - 1 (own cells and the inner halo)
  if (p >= y0) {
    const float* a = R.s0[P];
    float left, right;
    edge_neighbours(c, a, left, right);
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const float l = j == 0 ? left : a[j - 1], r = j == V - 1 ? right : a[j + 1];
      const float nb = fmaf(L.wx, l + r, L.wy * (R.s0[Q][j] + R.s0[C][j]));
      R.s1[P][j] = fmaf(keep, a[j], R.w[P][j] * (R.b[P][j] + nb));
    }
    const float edge = c.lane == 0 ? a[0] : a[V - 1];
    const float nbh = fmaf(L.wx, a[V + 1] + edge, L.wy * (R.s0[Q][V] + R.s0[C][V]));
    R.s1[P][V] = fmaf(keep, a[V], R.w[P][V] * (R.b[P][V] + nbh));
  }
  // second sweep on row o = p - 2 (own cells), written out; rows o - 1 and
  // o + 1 of the first sweep sit in slots C (row p - 3, not yet
  // overwritten) and P
  const int o = p - 2;
  if (o >= y0) {
    const float* a = R.s1[Q];
    float left, right;
    edge_neighbours(c, a, left, right);
    float z[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const float l = j == 0 ? left : a[j - 1], r = j == V - 1 ? right : a[j + 1];
      const float nb = fmaf(L.wx, l + r, L.wy * (R.s1[C][j] + R.s1[P][j]));
      z[j] = fmaf(keep, a[j], R.w[Q][j] * (R.b[Q][j] + nb));
    }
    if (c.ox) {
      stv<TB, V>(xout + (size_t)o * L.nx + c.gx, z);
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

template <typename T, bool MASKED, bool FINEST, typename TB>
__global__ void __launch_bounds__(32 * kWPB) k_up_w(LevelDev L, const TB* __restrict__ b, const T* __restrict__ xin,
                                                    TB* __restrict__ xout, const T* __restrict__ e, float omega, float s,
                                                    int rows, SolveState* __restrict__ st, double* __restrict__ partials) {
  chain_enter();
  if (st && st->inner_done) return;
  using S = Slot<T, TB, MASKED, true>;
  extern __shared__ __align__(16) unsigned char smem_w[];
  const int nstrips = (L.nx + 32 * V - 1) / (32 * V);
  const int nruns = (L.ny + rows - 1) / rows;
  const int wid = blockIdx.x * kWPB + (int)(threadIdx.x >> 5);
  float acc = 0.f;
  if (wid < nstrips * nruns) {  // whole warps
    unsigned char* ring = smem_w + (threadIdx.x >> 5) * (kSlots * S::BYTES);
    const int x0 = (wid % nstrips) * 32 * V;
    const int y0 = (wid / nstrips) * rows, y1 = min(y0 + rows, L.ny);
    const Lane c = lane_of<MASKED>(L, x0, omega);
    UpRegs R;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
      for (int j = 0; j < V + 2; ++j) R.s0[k][j] = 0.f;
#pragma unroll
      for (int j = 0; j < V + 1; ++j) R.s1[k][j] = R.b[k][j] = R.w[k][j] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < kD; ++i)
      up_issue<T, TB, MASKED>(L, c, y0 - 2 + i, y0 - 2 + i <= y1 + 1, b, xin, e, ring + i * S::BYTES);
    // rows y0 - 2 .. y1 + 1 (step i = row y0 - 2 + i); register slots rotate
    // with period 3
    const int n = y1 - y0 + 4;
    for (int i = 0; i < n; i += 3) {
      up_step<T, TB, MASKED, FINEST, 0, 2, 1>(L, c, i, y0, y1, omega, s, b, xin, e, xout, ring, R, acc);
      if (i + 1 >= n) break;
      up_step<T, TB, MASKED, FINEST, 1, 0, 2>(L, c, i + 1, y0, y1, omega, s, b, xin, e, xout, ring, R, acc);
      if (i + 2 >= n) break;
      up_step<T, TB, MASKED, FINEST, 2, 1, 0>(L, c, i + 2, y0, y1, omega, s, b, xin, e, xout, ring, R, acc);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");  // no copy outlives the warp
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

// ---- down leg ----------------------------------------------------------------
template <typename T, typename TB, bool MASKED>
__device__ __forceinline__ void down_issue(const LevelDev& L, const Lane& c, int r, bool want, const TB* __restrict__ b,
                                           unsigned char* slot) {
  using S = Slot<T, TB, MASKED, false>;
  if (want) {
    const bool rin = r >= 0 && r < L.ny;
    const bool fo = rin && c.ox, fh = rin && c.hok;
    const size_t row = rin ? (size_t)r * L.nx : 0;
    const int go = fo ? c.gx : 0;
    const uint32_t sl = smem_addr(slot);
    cp_async<4 * S::SB>(sl + S::B + c.lane * 4 * S::SB, b + row + go, fo);
    if (MASKED) cp_async<4>(sl + S::M + c.lane * 4, L.cell + row + go, fo);
    if (c.lane == 0 || c.lane == 31) {
      const uint32_t hs = sl + S::H + (c.lane == 31 ? 32 : 0);
      cp_async<2 * S::SB>(hs + 8, b + row + (fh ? c.hpair : 0), fh);
      if (MASKED) cp_async<4>(hs + 24, L.cell + row + (fh ? c.mword : 0), fh);
    }
  }
  cp_commit();
}

struct DownRegs {
  float b[3][V + 2];   // own cells, inner halo, outer halo
  float w[3][V + 1];   // omega / d: own cells, inner halo
  float s1[3][V + 2];  // first sweep (omega / d) b
  float s2[3][V + 1];  // second sweep: own cells, inner halo
  unsigned m[3];       // cell bytes of the own cells (masked)
  float rp[V / 2];     // restriction: residual pair sums of the even row
};

template <typename T, typename TB, bool MASKED, int C, int P, int Q>
__device__ __forceinline__ void down_step(const LevelDev& L, const Lane& c, int i, int y0, int y1, float omega,
                                          const TB* __restrict__ b, T* __restrict__ x, T* __restrict__ bcoarse,
                                          unsigned char* ring, DownRegs& R) {
  using S = Slot<T, TB, MASKED, false>;
  const int p = y0 - 2 + i;
  // row p: b, omega / d and the first sweep from zero, on own cells and halo
  cp_wait_ring();
  {
    const unsigned char* sl = ring + slot_of(i) * S::BYTES;
    float bv[V + 2];
    {
      float bo[V];
      lds4<TB>(sl + S::B + c.lane * 4 * S::SB, bo);
#pragma unroll
      for (int j = 0; j < V; ++j) bv[j] = bo[j];
    }
    const unsigned char* hs = sl + S::H + (c.lane == 31 ? 32 : 0);
    halo_of<TB>(c, hs, 8, bv[V], bv[V + 1]);
    unsigned m[V + 2], mw = 0u;
    if (MASKED) {
      mw = *reinterpret_cast<const unsigned*>(sl + S::M + c.lane * 4);
#pragma unroll
      for (int j = 0; j < V; ++j) m[j] = (mw >> (8 * j)) & 0xffu;
      halo_bytes(c, hs, m[V], m[V + 1]);
    } else {
#pragma unroll
      for (int j = 0; j < V + 2; ++j) m[j] = 0u;
    }
    float w[V + 2];
    row_w<MASKED, V + 2>(L, c, p, m, w);
#pragma unroll
    for (int j = 0; j < V + 2; ++j) {
      R.b[C][j] = bv[j];
      R.s1[C][j] = w[j] * bv[j];
      if (j < V + 1) R.w[C][j] = w[j];
    }
    R.m[C] = mw;
  }
  down_issue<T, TB, MASKED>(L, c, p + kD, p + kD <= y1 + 1, b, ring + slot_of(i + kD) * S::BYTES);
  const float keep = 1.f - omega;
  // second sweep on row p - 1 (own cells and the inner halo)
  if (p >= y0) {
    const float* a = R.s1[P];
    float left, right;
    edge_neighbours(c, a, left, right);
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const float l = j == 0 ? left : a[j - 1], r = j == V - 1 ? right : a[j + 1];
      const float nb = fmaf(L.wx, l + r, L.wy * (R.s1[Q][j] + R.s1[C][j]));
      R.s2[P][j] = fmaf(keep, a[j], R.w[P][j] * (R.b[P][j] + nb));
    }
    const float edge = c.lane == 0 ? a[0] : a[V - 1];
    const float nbh = fmaf(L.wx, a[V + 1] + edge, L.wy * (R.s1[Q][V] + R.s1[C][V]));
    R.s2[P][V] = fmaf(keep, a[V], R.w[P][V] * (R.b[P][V] + nbh));
  }
  // x and the residual on row o = p - 2; rows o - 1 and o + 1 of the second
  // sweep sit in slots C (row p - 3, not yet overwritten) and P
  const int o = p - 2;
  if (o >= y0) {
    const float* a = R.s2[Q];
    float left, right;
    edge_neighbours(c, a, left, right);
    float d[V];
    if (MASKED) {
#pragma unroll
      for (int j = 0; j < V; ++j) d[j] = __shfl_sync(0xffffffffu, c.tabd, (int)((R.m[Q] >> (8 * j)) & 15u));
    } else {
      const float dy = L.wy * (float)axis_count(o, L.ny, L.bcD, 2);  // y0 <= o < y1 <= ny
#pragma unroll
      for (int j = 0; j < V; ++j) d[j] = c.ox ? c.dx[j] + dy : 0.f;
    }
    float r[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const float l = j == 0 ? left : a[j - 1], rr = j == V - 1 ? right : a[j + 1];
      const float nb = fmaf(L.wx, l + rr, L.wy * (R.s2[C][j] + R.s2[P][j]));
      // cells with d = 0 (solid, outside) are not unknowns: no residual
      r[j] = d[j] != 0.f ? R.b[Q][j] - (d[j] * a[j] - nb) : 0.f;
    }
    if (c.ox && o < y1) {
      float xs[V];
#pragma unroll
      for (int j = 0; j < V; ++j) xs[j] = a[j];
      stv<T, V>(x + (size_t)o * L.nx + c.gx, xs);
      if ((o & 1) == 0) {
#pragma unroll
        for (int k = 0; k < V / 2; ++k) R.rp[k] = r[2 * k] + r[2 * k + 1];
      } else {
        float bc[V / 2];
#pragma unroll
        for (int k = 0; k < V / 2; ++k) bc[k] = 0.25f * (R.rp[k] + (r[2 * k] + r[2 * k + 1]));
        stv<T, V / 2>(bcoarse + (size_t)(o >> 1) * (L.nx >> 1) + (c.gx >> 1), bc);
      }
    }
  }
}

template <typename T, bool MASKED, typename TB>
__global__ void __launch_bounds__(32 * kWPB) k_down_w(LevelDev L, const TB* __restrict__ b, T* __restrict__ x,
                                                      T* __restrict__ bcoarse, float omega, int rows,
                                                      const SolveState* __restrict__ st) {
  chain_enter();
  if (st && st->inner_done) return;
  using S = Slot<T, TB, MASKED, false>;
  extern __shared__ __align__(16) unsigned char smem_w[];
  const int nstrips = (L.nx + 32 * V - 1) / (32 * V);
  const int nruns = (L.ny + rows - 1) / rows;
  const int wid = blockIdx.x * kWPB + (int)(threadIdx.x >> 5);
  if (wid >= nstrips * nruns) return;  // whole warps; no block-wide step follows
  unsigned char* ring = smem_w + (threadIdx.x >> 5) * (kSlots * S::BYTES);
  const int x0 = (wid % nstrips) * 32 * V;
  const int y0 = (wid / nstrips) * rows, y1 = min(y0 + rows, L.ny);
  const Lane c = lane_of<MASKED>(L, x0, omega);
  DownRegs R;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int j = 0; j < V + 2; ++j) R.b[k][j] = R.s1[k][j] = 0.f;
#pragma unroll
    for (int j = 0; j < V + 1; ++j) R.w[k][j] = R.s2[k][j] = 0.f;
    R.m[k] = 0u;
  }
#pragma unroll
  for (int k = 0; k < V / 2; ++k) R.rp[k] = 0.f;
#pragma unroll
  for (int i = 0; i < kD; ++i) down_issue<T, TB, MASKED>(L, c, y0 - 2 + i, y0 - 2 + i <= y1 + 1, b, ring + i * S::BYTES);
  const int n = y1 - y0 + 4;
  for (int i = 0; i < n; i += 3) {
    down_step<T, TB, MASKED, 0, 2, 1>(L, c, i, y0, y1, omega, b, x, bcoarse, ring, R);
    if (i + 1 >= n) break;
    down_step<T, TB, MASKED, 1, 0, 2>(L, c, i + 1, y0, y1, omega, b, x, bcoarse, ring, R);
    if (i + 2 >= n) break;
    down_step<T, TB, MASKED, 2, 1, 0>(L, c, i + 2, y0, y1, omega, b, x, bcoarse, ring, R);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
static int s2_sms() {
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 148;
  }
  return nsm;
}

// Rows per warp: even, at least 4 (so the grid has no more blocks than
// 64 x 16 tiles), about NPMG_STREAM2D_WARPS (default 8) warps per SM over
// the level.
static int s2_rows(const LevelDev& L) {
  const char* e = getenv("NPMG_STREAM2D_WARPS");
  const int wps = e && atoi(e) > 0 ? atoi(e) : 8;
  const long strips = (L.nx + 32 * V - 1) / (32 * V);
  const long target = (long)s2_sms() * wps;
  long rows = (strips * L.ny + target - 1) / target;
  rows = (rows + 1) / 2 * 2;
  if (rows < 4) rows = 4;
  if (rows > L.ny) rows = L.ny;
  return (int)rows;
}

static unsigned s2_blocks(const LevelDev& L, int rows) {
  const long strips = (L.nx + 32 * V - 1) / (32 * V);
  const long warps = strips * ((L.ny + rows - 1) / rows);
  return (unsigned)((warps + kWPB - 1) / kWPB);
}

bool stream2d_eligible(int dim, int pre, int post, const LevelDev& L) {
  return dim == 2 && pre == 2 && post == 2 && L.nx % 4 == 0 && L.ny % 2 == 0 && L.nx >= 4 && L.ny >= 2;
}

bool stream2d_aligned(const void* p) { return ((uintptr_t)p & 15) == 0; }

// Smallest level (cells) taken by these kernels: 2^19, or NPMG_STREAM2D_MIN.
// A warp walks its rows one after another, so on small levels, with few
// warps per SM, the tiled kernels finish sooner (measured on GB300: 512 x 256
// is faster tiled, 1024 x 512 streamed).
size_t stream2d_min_cells() {
  const char* e = getenv("NPMG_STREAM2D_MIN");
  return e ? (size_t)atol(e) : ((size_t)1 << 19);
}

template <typename T, bool MASKED, typename TB>
cudaError_t launch_down_w(const LevelDev& L, const void* b, void* x, void* bcoarse, float omega, const SolveState* st,
                          cudaStream_t s) {
  const int rows = s2_rows(L);
  const size_t smem = (size_t)kWPB * kSlots * Slot<T, TB, MASKED, false>::BYTES;
  return launch_chain(k_down_w<T, MASKED, TB>, s2_blocks(L, rows), 32 * kWPB, smem, s, L, (const TB*)b, (T*)x,
                      (T*)bcoarse, omega, rows, st);
}

template <typename T, bool MASKED, bool FINEST, typename TB>
cudaError_t launch_up_w(const LevelDev& L, const void* b, const void* xin, void* xout, const void* e, float omega,
                        float sc, SolveState* st, double* partials, cudaStream_t s) {
  const int rows = s2_rows(L);
  const size_t smem = (size_t)kWPB * kSlots * Slot<T, TB, MASKED, true>::BYTES;
  return launch_chain(k_up_w<T, MASKED, FINEST, TB>, s2_blocks(L, rows), 32 * kWPB, smem, s, L, (const TB*)b,
                      (const T*)xin, (TB*)xout, (const T*)e, omega, sc, rows, st, partials);
}

#define NPMG_INST_S2_TB(T, M, TB)                                                                                \
  template cudaError_t launch_down_w<T, M, TB>(const LevelDev&, const void*, void*, void*, float,                \
                                               const SolveState*, cudaStream_t);                                 \
  template cudaError_t launch_up_w<T, M, false, TB>(const LevelDev&, const void*, const void*, void*, const void*, \
                                                    float, float, SolveState*, double*, cudaStream_t);           \
  template cudaError_t launch_up_w<T, M, true, TB>(const LevelDev&, const void*, const void*, void*, const void*,  \
                                                   float, float, SolveState*, double*, cudaStream_t);

NPMG_INST_S2_TB(float, false, float)
NPMG_INST_S2_TB(float, true, float)
NPMG_INST_S2_TB(__half, false, __half)
NPMG_INST_S2_TB(__half, true, __half)
NPMG_INST_S2_TB(__half, false, float)
NPMG_INST_S2_TB(__half, true, float)
NPMG_INST_S2_TB(__nv_bfloat16, false, __nv_bfloat16)
NPMG_INST_S2_TB(__nv_bfloat16, true, __nv_bfloat16)
NPMG_INST_S2_TB(__nv_bfloat16, false, float)
NPMG_INST_S2_TB(__nv_bfloat16, true, float)

}  // namespace npmg
