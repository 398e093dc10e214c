// Projection time step of Algorithm 1 on a staggered (MAC) grid.
//
// Pressure lives at cell centres; velocity component c on the faces normal
// to axis c (face f along c lies between cells f-1 and f).  Boundaries: x-
// inflow (u fixed, tangential components padded with 0), x+ outflow
// (zero-gradient velocity, pressure 0), the other faces free-slip walls
// (normal component fixed at 0, tangential and pressure zero-gradient).  The
// padding follows Sec. 2.3: a Dirichlet side pads with the given value, a
// zero-derivative side with the adjacent value.
#include <math.h>
#include <string.h>

#include "gn.h"
#include "launch.h"
#include "mg_handle.h"

namespace npmg {

struct NsGeom {
  int dim;
  int n[3];        // cells per axis (n[2] = 1 in 2D)
  float inv_h, inv_h2;
  const uint8_t* solid;  // cells, 1 = solid (nullptr = none)
};

struct FaceArrays {
  const float* q[3];  // velocity components at time n (face arrays)
};

__device__ __forceinline__ void face_dims(const NsGeom& G, int c, int F[3]) {
  F[0] = G.n[0] + (c == 0);
  F[1] = G.n[1] + (c == 1);
  F[2] = G.dim == 3 ? G.n[2] + (c == 2) : 1;
}

__device__ __forceinline__ bool is_fixed(const NsGeom& G, int c, const int f[3]) {
  // the inflow face of u; both wall faces of v and w
  if (c == 0) return f[0] == 0;
  return f[c] == 0 || f[c] == G.n[c];
}

__device__ __forceinline__ float fixed_value(int c, float uin) { return c == 0 ? uin : 0.f; }

// Component c at face index f (may lie one step outside the face array along
// one axis: the padding rule of component c along that axis applies).
// Fixed faces read their prescribed value.
template <int DIM>
__device__ __forceinline__ float q_at(const NsGeom& G, const float* __restrict__ q, int c, int f0, int f1, int f2,
                                      float uin) {
  const int F0 = G.n[0] + (c == 0), F1 = G.n[1] + (c == 1), F2 = DIM == 3 ? G.n[2] + (c == 2) : 1;
  // padding rule along each axis: the inflow pads tangential components with
  // 0; every other side copies the edge value
  if (f0 < 0) {
    if (c != 0) return 0.f;
    f0 = 0;
  } else if (f0 >= F0) {
    f0 = F0 - 1;
  }
  f1 = f1 < 0 ? 0 : (f1 >= F1 ? F1 - 1 : f1);
  if (DIM == 3) f2 = f2 < 0 ? 0 : (f2 >= F2 ? F2 - 1 : f2);
  else f2 = 0;
  // fixed faces read their prescribed value
  const int fc = c == 0 ? f0 : (c == 1 ? f1 : f2);
  if (c == 0 ? fc == 0 : (fc == 0 || fc == G.n[c])) return fixed_value(c, uin);
  return q[((size_t)f2 * F1 + f1) * F0 + f0];
}

__device__ __forceinline__ bool solid_cell(const NsGeom& G, int x, int y, int z) {
  if (!G.solid) return false;
  x = min(max(x, 0), G.n[0] - 1);
  y = min(max(y, 0), G.n[1] - 1);
  z = min(max(z, 0), G.n[2] - 1);
  return G.solid[((size_t)z * G.n[1] + y) * G.n[0] + x] != 0;
}

// Thread mapping of the face/cell kernels: 256 threads = 32 along x times 8
// along y; grid (ceil(nx / 32), ceil(ny / 8), nz).
__device__ __forceinline__ bool face_thread(const int F[3], int f[3]) {
  f[0] = blockIdx.x * 32 + (threadIdx.x & 31);
  f[1] = blockIdx.y * 8 + (threadIdx.x >> 5);
  f[2] = blockIdx.z;
  return f[0] < F[0] && f[1] < F[1] && f[2] < F[2];
}

// Finite-element filters of App. A on the 3^DIM neighbourhood Nb[z][y][x]
// of a face (offsets -1, 0, +1 per axis; Nb[1][..] in 2D):
//   diffusion  2D 1/(4 h^2) [-1 -2 -1; -2 12 -2; -1 -2 -1]; 3D 1/(26 h^2) x
//              (88 centre, -6 face, -3 edge, -2 corner neighbours);
//   advection  along a: the central difference along a smoothed by
//              (1, 4, 1) across every other axis; 2D 1/(12 h), 3D 1/(72 h),
//              + towards +a on every axis.
template <int DIM>
__device__ __forceinline__ void fe_filters(const float (&Nb)[3][3][3], const float U[3], float inv_h, float inv_h2,
                                           float& adv, float& diff) {
  constexpr int Z0 = DIM == 3 ? 0 : 1, Z1 = DIM == 3 ? 2 : 1;
  // diffusion: weight by the number of non-zero offset components
  float faces = 0.f, edges = 0.f, corners = 0.f;
#pragma unroll
  for (int z = Z0; z <= Z1; ++z)
#pragma unroll
    for (int y = 0; y < 3; ++y)
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const int cnt = (x != 1) + (y != 1) + (z != 1);
        if (cnt == 1) faces += Nb[z][y][x];
        else if (cnt == 2) edges += Nb[z][y][x];
        else if (cnt == 3) corners += Nb[z][y][x];
      }
  const float ctr = Nb[1][1][1];
  if (DIM == 2)
    diff = (12.f * ctr - 2.f * faces - edges) * (0.25f * inv_h2);
  else
    diff = (88.f * ctr - 6.f * faces - 3.f * edges - 2.f * corners) * (inv_h2 / 26.f);
  // advection: smoothing weight 4 on the centre line of an axis, 1 off it
  float dx = 0.f, dy = 0.f, dz = 0.f;
#pragma unroll
  for (int z = Z0; z <= Z1; ++z)
#pragma unroll
    for (int y = 0; y < 3; ++y)
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const float v = Nb[z][y][x];
        const float wx = x == 1 ? 4.f : 1.f, wy = y == 1 ? 4.f : 1.f, wz = (DIM == 3 && z == 1) ? 4.f : 1.f;
        if (x != 1) dx = fmaf((x - 1) * (DIM == 3 ? wy * wz : wy), v, dx);
        if (y != 1) dy = fmaf((y - 1) * (DIM == 3 ? wx * wz : wx), v, dy);
        if (DIM == 3 && z != 1) dz = fmaf((z - 1) * wx * wy, v, dz);
      }
  const float s = inv_h / (DIM == 2 ? 12.f : 72.f);
  adv = fmaf(U[0], dx * s, U[1] * (dy * s));
  if (DIM == 3) adv = fmaf(U[2], dz * s, adv);
}

// One pass of the momentum update of component C (Eq. predictor-Burgers
// with implicit absorption, Alg. 1 step 1):
//   (1 + sigma dt) out = q^n - dt [ sum_b U_b^n d_b Q + nu A_nu Q + d_C p^n ]
// with Q = q^n (predictor) or Q = (qt + q^n) / 2 (corrector, CORR); d_b and
// A_nu are the 5/7-point filters, or the finite-element filters (FE).
template <int DIM, int C, bool CORR, bool FE>
__global__ void __launch_bounds__(256) k_momentum(NsGeom G, FaceArrays Qn, const float* __restrict__ qt,
                                                  const float* __restrict__ p, float* __restrict__ out, float dt,
                                                  float nu, float uin, float sigma) {
  int F[3], f[3];
  face_dims(G, C, F);
  if (!face_thread(F, f)) return;
  const size_t i = ((size_t)f[2] * F[1] + f[1]) * F[0] + f[0];
  if (is_fixed(G, C, f)) {
    out[i] = fixed_value(C, uin);
    return;
  }
  const float* qc = Qn.q[C];
  auto Q = [&](int a, int off) {
    int g[3] = {f[0], f[1], f[2]};
    g[a] += off;
    float v = q_at<DIM>(G, qc, C, g[0], g[1], g[2], uin);
    if (CORR) v = 0.5f * (v + q_at<DIM>(G, qt, C, g[0], g[1], g[2], uin));
    return v;
  };
  const float qn_self = qc[i];
  const float q0 = CORR ? 0.5f * (qn_self + qt[i]) : qn_self;
  float adv = 0.f, diff = 0.f;
  // Faces at least two cells from every side read their neighbours
  // directly: none of them is clamped, padded or fixed.
  const bool inner = f[0] >= 2 && f[0] + 2 < F[0] && f[1] >= 2 && f[1] + 2 < F[1] &&
                     (DIM == 2 || (f[2] >= 2 && f[2] + 2 < F[2]));
  if constexpr (FE) {
    float U[3] = {0.f, 0.f, 0.f};
    float Nb[3][3][3];
    constexpr int Z0 = DIM == 3 ? 0 : 1, Z1 = DIM == 3 ? 2 : 1;
    if (inner) {
      const size_t sc[3] = {1, (size_t)F[0], (size_t)F[0] * F[1]};
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        if (a == C) {
          U[a] = qn_self;
        } else {
          const size_t A0 = G.n[0] + (a == 0), A1 = G.n[1] + (a == 1);
          const size_t sa[3] = {1, A0, A0 * A1};
          const size_t ia = ((size_t)f[2] * A1 + f[1]) * A0 + f[0];
          const float* qa = Qn.q[a];
          U[a] = 0.25f * ((qa[ia - sa[C]] + qa[ia - sa[C] + sa[a]]) + (qa[ia] + qa[ia + sa[a]]));
        }
      }
#pragma unroll
      for (int z = Z0; z <= Z1; ++z)
#pragma unroll
        for (int y = 0; y < 3; ++y)
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            const size_t j = i + (z - 1) * sc[2] + (y - 1) * sc[1] + (x - 1);
            float v = qc[j];
            if (CORR) v = 0.5f * (v + qt[j]);
            Nb[z][y][x] = v;
          }
    } else {
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        if (a == C) {
          U[a] = qn_self;
        } else {
          float s = 0.f;
#pragma unroll
          for (int dc = -1; dc <= 0; ++dc)
#pragma unroll
            for (int da = 0; da <= 1; ++da) {
              int g[3] = {f[0], f[1], f[2]};
              g[C] += dc;
              g[a] += da;
              s += q_at<DIM>(G, Qn.q[a], a, g[0], g[1], g[2], uin);
            }
          U[a] = 0.25f * s;
        }
      }
      // corner neighbours take the padding rule of every axis they leave
#pragma unroll
      for (int z = Z0; z <= Z1; ++z)
#pragma unroll
        for (int y = 0; y < 3; ++y)
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            const int g0 = f[0] + x - 1, g1 = f[1] + y - 1, g2 = f[2] + z - 1;
            float v = q_at<DIM>(G, qc, C, g0, g1, g2, uin);
            if (CORR) v = 0.5f * (v + q_at<DIM>(G, qt, C, g0, g1, g2, uin));
            Nb[z][y][x] = v;
          }
    }
    fe_filters<DIM>(Nb, U, G.inv_h, G.inv_h2, adv, diff);
  } else if (inner) {
    const size_t sc[3] = {1, (size_t)F[0], (size_t)F[0] * F[1]};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      float Ua;
      if (a == C) {
        Ua = qn_self;
      } else {
        // component a's face array: cells f-1, f along C, faces j, j+1 along a
        const size_t A0 = G.n[0] + (a == 0), A1 = G.n[1] + (a == 1);
        const size_t sa[3] = {1, A0, A0 * A1};
        const size_t ia = ((size_t)f[2] * A1 + f[1]) * A0 + f[0];
        const float* qa = Qn.q[a];
        Ua = 0.25f * ((qa[ia - sa[C]] + qa[ia - sa[C] + sa[a]]) + (qa[ia] + qa[ia + sa[a]]));
      }
      float qm = qc[i - sc[a]], qp = qc[i + sc[a]];
      if (CORR) {
        qm = 0.5f * (qm + qt[i - sc[a]]);
        qp = 0.5f * (qp + qt[i + sc[a]]);
      }
      adv = fmaf(Ua, (qp - qm) * (0.5f * G.inv_h), adv);
      diff += (2.f * q0 - qm - qp) * G.inv_h2;
    }
  } else {
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    // advecting velocity component a at this C-face (time n)
    float Ua;
    if (a == C) {
      Ua = qn_self;
    } else {
      // cells f-1, f along C; faces j, j+1 along a
      float s = 0.f;
#pragma unroll
      for (int dc = -1; dc <= 0; ++dc)
#pragma unroll
        for (int da = 0; da <= 1; ++da) {
          int g[3] = {f[0], f[1], f[2]};
          g[C] += dc;
          g[a] += da;
          s += q_at<DIM>(G, Qn.q[a], a, g[0], g[1], g[2], uin);
        }
      Ua = 0.25f * s;
    }
    const float qm = Q(a, -1), qp = Q(a, +1);
    adv = fmaf(Ua, (qp - qm) * (0.5f * G.inv_h), adv);
    diff += (2.f * q0 - qm - qp) * G.inv_h2;
  }
  }
  // pressure gradient d_C p^n at the face: cells f-1 and f along C; the
  // outflow ghost is 0 (Dirichlet), faces at walls are fixed (skipped above)
  const int fz = DIM == 3 ? f[2] : 0;
  const int sx = 1, sy = G.n[0], sz = G.n[0] * G.n[1];
  const int stride = C == 0 ? sx : (C == 1 ? sy : sz);
  const size_t ir = ((size_t)fz * G.n[1] + f[1]) * G.n[0] + f[0];  // cell f (valid when f[C] < n[C])
  const bool right_in = f[C] < G.n[C];
  const float pr = right_in ? p[ir] : 0.f;
  const float pl = p[ir - stride];
  const float gp = (pr - pl) * G.inv_h;
  bool sf = false;
  if (G.solid) sf = G.solid[ir - stride] || (right_in && G.solid[ir]) || (!right_in && G.solid[ir - stride]);
  const float denom = 1.f + (sf ? sigma : 0.f) * dt;
  out[i] = (qn_self - dt * (adv + nu * diff + gp)) / denom;
}

// b = -(1/dt) D q* on fluid cells (Alg. 1 step 2 right-hand side).
template <int DIM>
__global__ void __launch_bounds__(256) k_divergence(NsGeom G, FaceArrays Q, float scale, float* __restrict__ b) {
  const int N[3] = {G.n[0], G.n[1], G.n[2]};
  int c[3];
  if (!face_thread(N, c)) return;
  const size_t i = ((size_t)c[2] * N[1] + c[1]) * N[0] + c[0];
  if (G.solid && G.solid[i]) {
    b[i] = 0.f;
    return;
  }
  float d = 0.f;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const int Fx = N[0] + (a == 0), Fy = N[1] + (a == 1);
    const size_t lo = ((size_t)c[2] * Fy + c[1]) * Fx + c[0];
    const size_t stride = a == 0 ? 1 : (a == 1 ? (size_t)Fx : (size_t)Fx * Fy);
    d += Q.q[a][lo + stride] - Q.q[a][lo];
  }
  b[i] = scale * d * G.inv_h;
}

// q = q* - dt G dp on the faces G corrects (interior faces between fluid
// cells; the outflow faces of u beside a fluid cell, with the pressure ghost
// 0) (Alg. 1 step 3).
template <int DIM, int C>
__global__ void __launch_bounds__(256) k_correct(NsGeom G, const float* __restrict__ qs, float* __restrict__ q,
                                                 const float* __restrict__ dp, float dt) {
  int F[3], f[3];
  face_dims(G, C, F);
  if (!face_thread(F, f)) return;
  const size_t i = ((size_t)f[2] * F[1] + f[1]) * F[0] + f[0];
  float v = qs[i];
  const int fc = f[C];
  const bool corr = fc > 0 && (C == 0 ? fc <= G.n[0] : fc < G.n[C]);
  if (corr) {
    const int fz = DIM == 3 ? f[2] : 0;
    const int stride = C == 0 ? 1 : (C == 1 ? G.n[0] : G.n[0] * G.n[1]);
    const size_t ir = ((size_t)fz * G.n[1] + f[1]) * G.n[0] + f[0];
    const size_t il = ir - stride;
    const bool right_in = fc < G.n[C];
    const bool left_fluid = !(G.solid && G.solid[il]);
    const bool right_fluid = !right_in || !(G.solid && G.solid[ir]);
    const float pr = right_in ? dp[ir] : 0.f;
    if (left_fluid && right_fluid) v -= dt * (pr - dp[il]) * G.inv_h;
  }
  q[i] = v;
}

// p += dp (Alg. 1 step 4).
__global__ void k_add(size_t n, float* __restrict__ p, const float* __restrict__ dp) {
  const size_t n4 = n / 4;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    float4 a = reinterpret_cast<float4*>(p)[i];
    const float4 d = reinterpret_cast<const float4*>(dp)[i];
    a.x += d.x; a.y += d.y; a.z += d.z; a.w += d.w;
    reinterpret_cast<float4*>(p)[i] = a;
  }
  for (size_t i = n4 * 4 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    p[i] += dp[i];
}

}  // namespace npmg

using namespace npmg;

struct ns_handle_s {
  int dim;
  int64_t cells[3];
  double h, sigma;
  mg_handle mg;
  char* pool;
  uint8_t* solid;
  float* pred[3];
  float* star[3];
  float* b;
  float* dp;
  size_t nfaces[3], ncells;
  int nsm;
  gn_handle guess;  // learned initial guess of dp (not owned), or nullptr
  int guess_level;  // the network runs on the grid coarsened this many times (0 .. 2)
  // coarse fields of the guess, level 1 then level 2 (b, p, dp each), and a
  // level-1 solid mask, or nullptr until a coarse level is first used
  float* gc;
  uint8_t* gsolid;
  int stencil;  // NS_STENCIL_FD (5/7-point) or NS_STENCIL_FE (9/27-point)
};

static constexpr int kMaxGuessLevel = 2;

// ---------------------------------------------------------------------------
// Grid transfer of the coarse guess.  Restriction is the 2x2x2 average of
// the cycle (App. B); the coarse guess comes back by trilinear interpolation
// between coarse-cell centres (weights 3/4 and 1/4 per axis, the nearest
// coarse cell repeated at the domain faces), so that it carries no
// cell-to-cell jumps into the fine solve; solid fine cells get 0.
__global__ void k_restrict_avg(int nx, int ny, int nz, const float* __restrict__ f, float* __restrict__ c) {
  const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
  const size_t n = (size_t)cx * cy * cz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % cx), y = (int)((i / cx) % cy), z = (int)(i / ((size_t)cx * cy));
    float sum = 0.f;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const size_t r = ((size_t)(2 * z + dz) * ny + (2 * y + dy)) * nx + 2 * x;
        sum += f[r] + f[r + 1];
      }
    c[i] = 0.125f * sum;
  }
}

__global__ void k_prolong_tri(int nx, int ny, int nz, const float* __restrict__ c, const uint8_t* __restrict__ solid,
                              float* __restrict__ f) {
  const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
  const size_t n = (size_t)nx * ny * nz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (solid && solid[i]) {
      f[i] = 0.f;
      continue;
    }
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
    // the parent, and the neighbour on the fine cell's side of it
    const int px = x >> 1, py = y >> 1, pz = z >> 1;
    const int qx = min(max(px + ((x & 1) ? 1 : -1), 0), cx - 1);
    const int qy = min(max(py + ((y & 1) ? 1 : -1), 0), cy - 1);
    const int qz = min(max(pz + ((z & 1) ? 1 : -1), 0), cz - 1);
    const int X[2] = {px, qx}, Y[2] = {py, qy}, Z[2] = {pz, qz};
    const float wgt[2] = {0.75f, 0.25f};
    float v = 0.f;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b2 = 0; b2 < 2; ++b2)
#pragma unroll
        for (int d = 0; d < 2; ++d)
          v = fmaf(wgt[a] * wgt[b2] * wgt[d], c[((size_t)Z[a] * cy + Y[b2]) * cx + X[d]], v);
    f[i] = v;
  }
}

static int ns_blocks(const ns_handle_s* n, size_t count) {
  size_t b = (count + 255) / 256;
  const size_t cap = (size_t)n->nsm * 8;
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

// Grid of the face kernels of component c (c = -1: cells).
static dim3 face_grid(const ns_handle_s* ns, int c) {
  const int64_t fx = ns->cells[0] + (c == 0), fy = ns->cells[1] + (c == 1);
  const int64_t fz = ns->dim == 3 ? ns->cells[2] + (c == 2) : 1;
  return dim3((unsigned)((fx + 31) / 32), (unsigned)((fy + 7) / 8), (unsigned)fz);
}

static void launch_correct(ns_handle_s* ns, const NsGeom& G, float* const* qs, float* const* q, const float* dp,
                           float dt, cudaStream_t s) {
  for (int c = 0; c < ns->dim; ++c) {
    LaunchScope ls(ns->mg, MG_K_CORRECT, s);
    const dim3 g = face_grid(ns, c);
    if (ns->dim == 2) {
      if (c == 0) k_correct<2, 0><<<g, 256, 0, s>>>(G, qs[c], q[c], dp, dt);
      else k_correct<2, 1><<<g, 256, 0, s>>>(G, qs[c], q[c], dp, dt);
    } else {
      if (c == 0) k_correct<3, 0><<<g, 256, 0, s>>>(G, qs[c], q[c], dp, dt);
      else if (c == 1) k_correct<3, 1><<<g, 256, 0, s>>>(G, qs[c], q[c], dp, dt);
      else k_correct<3, 2><<<g, 256, 0, s>>>(G, qs[c], q[c], dp, dt);
    }
  }
}

static NsGeom geom_of(const ns_handle_s* ns) {
  NsGeom G;
  G.dim = ns->dim;
  G.n[0] = (int)ns->cells[0];
  G.n[1] = (int)ns->cells[1];
  G.n[2] = ns->dim == 3 ? (int)ns->cells[2] : 1;
  G.inv_h = (float)(1.0 / ns->h);
  G.inv_h2 = (float)(1.0 / (ns->h * ns->h));
  G.solid = ns->solid;
  return G;
}

extern "C" {

mg_status ns_create(ns_handle* out, int dim, const int64_t cells[3], double h, const uint8_t* d_solid, double sigma,
                    const mg_options* opt, void* stream) {
  if (!out || !cells || (dim != 2 && dim != 3) || !(h > 0.0) || !(sigma >= 0.0)) {
    set_error("ns_create: invalid arguments");
    return MG_ERR_INVALID;
  }
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  ns_handle_s* ns = new ns_handle_s();
  memset(ns, 0, sizeof(*ns));
  ns->dim = dim;
  for (int a = 0; a < 3; ++a) ns->cells[a] = a < dim ? cells[a] : 1;
  ns->h = h;
  ns->sigma = sigma;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&ns->nsm, cudaDevAttrMultiProcessorCount, dev);
  const int bc[6] = {MG_BC_NEUMANN, MG_BC_DIRICHLET, MG_BC_NEUMANN, MG_BC_NEUMANN, MG_BC_NEUMANN, MG_BC_NEUMANN};
  const double sp[3] = {h, h, h};
  mg_status st = mg_create(&ns->mg, dim, ns->cells, sp, bc, d_solid, opt, stream);
  if (st != MG_OK) {
    delete ns;
    return st;
  }
  ns->ncells = (size_t)ns->cells[0] * ns->cells[1] * ns->cells[2];
  size_t total = 0;
  for (int c = 0; c < dim; ++c) {
    ns->nfaces[c] = (size_t)(ns->cells[0] + (c == 0)) * (ns->cells[1] + (c == 1)) * (ns->cells[2] + (c == 2));
    total += 2 * ((ns->nfaces[c] * 4 + 255) / 256 * 256);
  }
  total += 2 * ((ns->ncells * 4 + 255) / 256 * 256) + (ns->ncells + 255) / 256 * 256;
  cudaError_t e = cudaMalloc((void**)&ns->pool, total);
  if (e != cudaSuccess) {
    mg_destroy(ns->mg);
    delete ns;
    set_error("ns_create: cudaMalloc failed: %s", cudaGetErrorString(e));
    return MG_ERR_OOM;
  }
  char* q = ns->pool;
  auto take = [&](size_t bytes) {
    char* r = q;
    q += (bytes + 255) / 256 * 256;
    return r;
  };
  for (int c = 0; c < dim; ++c) {
    ns->pred[c] = (float*)take(ns->nfaces[c] * 4);
    ns->star[c] = (float*)take(ns->nfaces[c] * 4);
  }
  ns->b = (float*)take(ns->ncells * 4);
  ns->dp = (float*)take(ns->ncells * 4);
  if (d_solid) {
    ns->solid = (uint8_t*)take(ns->ncells);
    e = cudaMemcpyAsync(ns->solid, d_solid, ns->ncells, cudaMemcpyDeviceToDevice, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error("ns_create: %s", cudaGetErrorString(e));
    ns_destroy(ns);
    return MG_ERR_CUDA;
  }
  *out = ns;
  return MG_OK;
}

mg_handle ns_pressure_handle(ns_handle ns) { return ns ? ns->mg : nullptr; }

mg_status ns_last_fields(ns_handle ns, const float** d_b, const float** d_dp) {
  if (!ns || !d_b || !d_dp) {
    set_error("ns_last_fields: NULL argument");
    return MG_ERR_INVALID;
  }
  *d_b = ns->b;
  *d_dp = ns->dp;
  return MG_OK;
}

// Level-l coarse buffers of the guess (l = 1, 2): b, p, dp.
static float* gc_level(ns_handle_s* ns, int l, int which) {
  const size_t n1 = ns->ncells / 8, n2 = ns->ncells / 64;
  return l == 1 ? ns->gc + which * n1 : ns->gc + 3 * n1 + which * n2;
}

static mg_status ensure_guess_buffers(ns_handle_s* ns, const char* who) {
  if (ns->gc) return MG_OK;
  const size_t n1 = ns->ncells / 8, n2 = ns->ncells / 64;
  if (cudaMalloc((void**)&ns->gc, 3 * (n1 + n2) * sizeof(float)) != cudaSuccess) {
    ns->gc = nullptr;
    set_error("%s: cudaMalloc of the coarse guess buffers failed", who);
    return MG_ERR_OOM;
  }
  if (cudaMalloc((void**)&ns->gsolid, n1) != cudaSuccess) {
    cudaFree(ns->gc);
    ns->gc = nullptr;
    ns->gsolid = nullptr;
    set_error("%s: cudaMalloc of the coarse guess buffers failed", who);
    return MG_ERR_OOM;
  }
  return MG_OK;
}

// Restrict `level` times (1 or 2): out receives the last field (the
// level-1 one goes to scratch1 when level == 2).
static void restrict_times(ns_handle_s* ns, int level, const float* f, float* scratch1, float* out, cudaStream_t s) {
  const int nx = (int)ns->cells[0], ny = (int)ns->cells[1], nz = (int)ns->cells[2];
  if (level == 1) {
    k_restrict_avg<<<ns_blocks(ns, ns->ncells / 8), 256, 0, s>>>(nx, ny, nz, f, out);
  } else {
    k_restrict_avg<<<ns_blocks(ns, ns->ncells / 8), 256, 0, s>>>(nx, ny, nz, f, scratch1);
    k_restrict_avg<<<ns_blocks(ns, ns->ncells / 64), 256, 0, s>>>(nx / 2, ny / 2, nz / 2, scratch1, out);
  }
}

mg_status ns_coarse_fields(ns_handle ns, int level, const float* d_p, float* d_b_c, float* d_p_c, float* d_dp_c,
                           uint8_t* d_solid_c, void* stream) {
  if (!ns || !d_p || !d_b_c || !d_p_c || !d_dp_c || !d_solid_c || level < 1 || level > kMaxGuessLevel) {
    set_error("ns_coarse_fields: NULL argument or level not 1 / 2");
    return MG_ERR_INVALID;
  }
  const int64_t q = (int64_t)1 << level;
  if (ns->dim != 3 || (ns->cells[0] % q) || (ns->cells[1] % q) || (ns->cells[2] % q)) {
    set_error("ns_coarse_fields: needs a 3D grid with sides divisible by %d", (int)q);
    return MG_ERR_INVALID;
  }
  mg_status st = ensure_guess_buffers(ns, "ns_coarse_fields");
  if (st != MG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  float* tmp = gc_level(ns, 1, 0);  // level-1 scratch
  restrict_times(ns, level, ns->b, tmp, d_b_c, s);
  restrict_times(ns, level, d_p, tmp, d_p_c, s);
  restrict_times(ns, level, ns->dp, tmp, d_dp_c, s);
  if (ns->solid) {
    if (level == 1) {
      NPMG_CUDA(launch_coarsen_solid(3, ns->cells, ns->solid, d_solid_c, s));
    } else {
      const int64_t c1[3] = {ns->cells[0] / 2, ns->cells[1] / 2, ns->cells[2] / 2};
      NPMG_CUDA(launch_coarsen_solid(3, ns->cells, ns->solid, ns->gsolid, s));
      NPMG_CUDA(launch_coarsen_solid(3, c1, ns->gsolid, d_solid_c, s));
    }
  } else {
    NPMG_CUDA(cudaMemsetAsync(d_solid_c, 0, ns->ncells >> (3 * level), s));
  }
  NPMG_CUDA(cudaGetLastError());
  return MG_OK;
}

mg_status ns_set_guess(ns_handle ns, gn_handle g) {
  if (!ns) {
    set_error("ns_set_guess: NULL handle");
    return MG_ERR_INVALID;
  }
  if (g && (ns->dim != 3 || (ns->cells[0] % 4) || (ns->cells[1] % 4) || (ns->cells[2] % 4))) {
    set_error("ns_set_guess: the guess network needs a 3D grid with sides divisible by 4");
    return MG_ERR_INVALID;
  }
  ns->guess = g;
  ns->guess_level = 0;
  return MG_OK;
}

mg_status ns_set_guess_level(ns_handle ns, gn_handle g, int level) {
  if (!ns || level < 0 || level > kMaxGuessLevel) {
    set_error("ns_set_guess_level: NULL handle or level not 0 .. 2");
    return MG_ERR_INVALID;
  }
  const int64_t q = (int64_t)4 << level;
  if (g && (ns->dim != 3 || (ns->cells[0] % q) || (ns->cells[1] % q) || (ns->cells[2] % q))) {
    set_error("ns_set_guess_level: the guess network needs a 3D grid with sides divisible by %d", (int)q);
    return MG_ERR_INVALID;
  }
  if (g && level > 0) {
    mg_status st = ensure_guess_buffers(ns, "ns_set_guess_level");
    if (st != MG_OK) return st;
  }
  ns->guess = g;
  ns->guess_level = g ? level : 0;
  return MG_OK;
}

mg_status ns_set_stencils(ns_handle ns, int stencil) {
  if (!ns || (stencil != NS_STENCIL_FD && stencil != NS_STENCIL_FE)) {
    set_error("ns_set_stencils: NULL handle or stencil not NS_STENCIL_FD / NS_STENCIL_FE");
    return MG_ERR_INVALID;
  }
  ns->stencil = stencil;
  return MG_OK;
}

mg_status ns_momentum(ns_handle ns, const float* d_u, const float* d_v, const float* d_w, const float* d_p,
                      float* d_us, float* d_vs, float* d_ws, double dt, double nu, double u_inflow, void* stream) {
  if (!ns || !d_u || !d_v || !d_p || !d_us || !d_vs || (ns->dim == 3 && (!d_w || !d_ws))) {
    set_error("ns_momentum: NULL argument");
    return MG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const NsGeom G = geom_of(ns);
  FaceArrays Qn;
  Qn.q[0] = d_u;
  Qn.q[1] = d_v;
  Qn.q[2] = ns->dim == 3 ? d_w : nullptr;
  float* outs[3] = {d_us, d_vs, d_ws};
  const float fdt = (float)dt, fnu = (float)nu, fu = (float)u_inflow, fs = (float)ns->sigma;
  const bool fe = ns->stencil == NS_STENCIL_FE;
  for (int pass = 0; pass < 2; ++pass) {
    for (int c = 0; c < ns->dim; ++c) {
      LaunchScope ls(ns->mg, MG_K_MOMENTUM, s);
      const dim3 g = face_grid(ns, c);
      const float* qt = pass ? ns->pred[c] : nullptr;
      float* o = pass ? outs[c] : ns->pred[c];
#define NPMG_MOM2(D, CC, FEF)                                                                       \
  (pass ? k_momentum<D, CC, true, FEF><<<g, 256, 0, s>>>(G, Qn, qt, d_p, o, fdt, fnu, fu, fs)        \
        : k_momentum<D, CC, false, FEF><<<g, 256, 0, s>>>(G, Qn, qt, d_p, o, fdt, fnu, fu, fs))
#define NPMG_MOM(D, CC) (fe ? NPMG_MOM2(D, CC, true) : NPMG_MOM2(D, CC, false))
      if (ns->dim == 2) {
        if (c == 0) NPMG_MOM(2, 0);
        else NPMG_MOM(2, 1);
      } else {
        if (c == 0) NPMG_MOM(3, 0);
        else if (c == 1) NPMG_MOM(3, 1);
        else NPMG_MOM(3, 2);
      }
#undef NPMG_MOM
#undef NPMG_MOM2
    }
  }
  NPMG_CUDA(cudaGetLastError());
  return MG_OK;
}

mg_status ns_divergence_rhs(ns_handle ns, const float* d_us, const float* d_vs, const float* d_ws, double dt,
                            float* d_b, void* stream) {
  if (!ns || !d_us || !d_vs || !d_b || (ns->dim == 3 && !d_ws) || !(dt > 0)) {
    set_error("ns_divergence_rhs: invalid argument");
    return MG_ERR_INVALID;
  }
  FaceArrays Q;
  Q.q[0] = d_us;
  Q.q[1] = d_vs;
  Q.q[2] = d_ws;
  LaunchScope ls(ns->mg, MG_K_DIVERGENCE, (cudaStream_t)stream);
  if (ns->dim == 2)
    k_divergence<2><<<face_grid(ns, -1), 256, 0, (cudaStream_t)stream>>>(geom_of(ns), Q, (float)(-1.0 / dt), d_b);
  else
    k_divergence<3><<<face_grid(ns, -1), 256, 0, (cudaStream_t)stream>>>(geom_of(ns), Q, (float)(-1.0 / dt), d_b);
  NPMG_CUDA(cudaGetLastError());
  return MG_OK;
}

mg_status ns_correct(ns_handle ns, float* d_u, float* d_v, float* d_w, float* d_p, const float* d_dp, double dt,
                     void* stream) {
  if (!ns || !d_u || !d_v || !d_p || !d_dp || (ns->dim == 3 && !d_w)) {
    set_error("ns_correct: NULL argument");
    return MG_ERR_INVALID;
  }
  if (((uintptr_t)d_p | (uintptr_t)d_dp) & 15) {
    set_error("ns_correct: d_p and d_dp must be 16-byte aligned");
    return MG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const NsGeom G = geom_of(ns);
  float* qs[3] = {d_u, d_v, d_w};
  launch_correct(ns, G, qs, qs, d_dp, (float)dt, s);
  {
    LaunchScope ls(ns->mg, MG_K_CORRECT, s);
    k_add<<<ns_blocks(ns, ns->ncells), 256, 0, s>>>(ns->ncells, d_p, d_dp);
  }
  NPMG_CUDA(cudaGetLastError());
  return MG_OK;
}

mg_status ns_step(ns_handle ns, float* d_u, float* d_v, float* d_w, float* d_p, double dt, double nu,
                  double u_inflow, double rel_tol, void* stream, mg_stats* out) {
  if (!ns || !d_u || !d_v || !d_p || (ns->dim == 3 && !d_w) || !(dt > 0) || !(rel_tol > 0)) {
    set_error("ns_step: invalid argument");
    return MG_ERR_INVALID;
  }
  if (((uintptr_t)d_u | (uintptr_t)d_v | (uintptr_t)d_w | (uintptr_t)d_p) & 15) {
    set_error("ns_step: arrays must be 16-byte aligned");
    return MG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  mg_status st = ns_momentum(ns, d_u, d_v, d_w, d_p, ns->star[0], ns->star[1], ns->dim == 3 ? ns->star[2] : nullptr,
                             dt, nu, u_inflow, stream);
  if (st != MG_OK) return st;
  st = ns_divergence_rhs(ns, ns->star[0], ns->star[1], ns->dim == 3 ? ns->star[2] : nullptr, dt, ns->b, stream);
  if (st != MG_OK) return st;
  if (ns->guess) {
    // warm start: dp from the network on (b, p^n); the solve restarts from
    // zero when the guess is worse than zero
    if (ns->guess_level == 0) {
      const int64_t cells[3] = {ns->cells[0], ns->cells[1], ns->cells[2]};
      st = gn_forward(ns->guess, 1, cells, ns->b, d_p, ns->dp, stream);
    } else {
      // on the coarsened grid: restrict b and p^n, run the network,
      // interpolate its dp back level by level (solid fine cells get 0)
      const int lv = ns->guess_level;
      const int nx = (int)ns->cells[0], ny = (int)ns->cells[1], nz = (int)ns->cells[2];
      float *bc = gc_level(ns, lv, 0), *pc = gc_level(ns, lv, 1), *dc = gc_level(ns, lv, 2);
      restrict_times(ns, lv, ns->b, gc_level(ns, 1, 0), bc, s);
      restrict_times(ns, lv, d_p, gc_level(ns, 1, 1), pc, s);
      const int64_t cc[3] = {nx >> lv, ny >> lv, nz >> lv};
      st = gn_forward(ns->guess, 1, cc, bc, pc, dc, stream);
      if (st == MG_OK) {
        if (lv == 2) {
          float* d1 = gc_level(ns, 1, 2);
          k_prolong_tri<<<ns_blocks(ns, ns->ncells / 8), 256, 0, s>>>(nx / 2, ny / 2, nz / 2, dc, nullptr, d1);
          dc = d1;
        }
        k_prolong_tri<<<ns_blocks(ns, ns->ncells), 256, 0, s>>>(nx, ny, nz, dc, ns->solid, ns->dp);
        NPMG_CUDA(cudaGetLastError());
        npmg::gn::g_launches += 1 + 2 * lv;  // counted with the network's kernels
      }
    }
    if (st != MG_OK) return st;
  } else {
    NPMG_CUDA(cudaMemsetAsync(ns->dp, 0, ns->ncells * 4, s));
  }
  ns->mg->guess_check = ns->guess ? 1 : 0;
  mg_status solve = mg_solve(ns->mg, ns->b, ns->dp, rel_tol, stream, out);
  ns->mg->guess_check = 0;
  if (solve != MG_OK && solve != MG_NOT_CONVERGED && solve != MG_DIVERGED) return solve;
  const NsGeom G = geom_of(ns);
  float* qs[3] = {d_u, d_v, d_w};
  {
    float* st3[3] = {ns->star[0], ns->star[1], ns->star[2]};
    launch_correct(ns, G, st3, qs, ns->dp, (float)dt, s);
  }
  {
    LaunchScope ls(ns->mg, MG_K_CORRECT, s);
    k_add<<<ns_blocks(ns, ns->ncells), 256, 0, s>>>(ns->ncells, d_p, ns->dp);
  }
  NPMG_CUDA(cudaGetLastError());
  return solve;
}

mg_status ns_destroy(ns_handle ns) {
  if (!ns) return MG_OK;
  if (ns->mg) mg_destroy(ns->mg);
  if (ns->pool) cudaFree(ns->pool);
  if (ns->gc) cudaFree(ns->gc);
  if (ns->gsolid) cudaFree(ns->gsolid);
  delete ns;
  return MG_OK;
}

}  // extern "C"
