// TMA-staged level kernels (2D, two pre / two post sweeps).
//
// A block owns a 64 x 16 tile.  One thread issues cp.async.bulk.tensor loads
// of the tile plus a 2-cell halo (widened along x so that every box starts
// on a 16-byte boundary) for each input array; the block waits on one
// mbarrier, then runs the sweeps in shared memory.  Out-of-domain box cells
// arrive as 0: the zero padding of Sec. 2.1.  Same arithmetic as k_down /
// k_up in mg_kernels.cuh (weighted Jacobi, Eq. Jacobi-1-relax; 2x2 average
// restriction and copy prolongation, Sec. 2.2).
#include <cudaTypedefs.h>

#include "launch.h"
#include "mg_kernels.cuh"
#include "tma.cuh"
#include "tma_host.h"

namespace npmg {

template <typename T>
struct TmaGeom {
  static constexpr int MX = 16 / (int)sizeof(T);  // x margin keeping box starts 16-byte aligned
  static constexpr int BW = kTmaTX + 2 * MX;      // fine box width (elements)
  static constexpr int BH = kTmaTY + 2 * kTmaH;   // fine box height (rows)
  static constexpr int BWE = kTmaTX / 2 + 2 * MX; // coarse box width
  static constexpr int BHE = kTmaTY / 2 + 2;      // coarse rows y0/2-1 .. y0/2+kTmaTY/2
  static constexpr int BWM = kTmaTX + 32;         // mask box width (bytes), start x0 - 16
  static constexpr int NF = BW * BH;              // fine box elements
  static constexpr int NE = BWE * BHE;
  static constexpr int NM = BWM * BH;
};

__host__ __device__ constexpr int align128(int v) { return (v + 127) / 128 * 128; }

template <typename T>
struct DownLayout {
  using G = TmaGeom<T>;
  static constexpr int B = 0;                                    // T[NF]   b
  static constexpr int M = align128(B + G::NF * (int)sizeof(T)); // u8[NM]  cell bytes
  static constexpr int X1 = align128(M + G::NM);                 // f32[NF] x after sweep 1
  static constexpr int X2 = align128(X1 + G::NF * 4);            // f32[NF] x after sweep 2
  static constexpr int DG = align128(X2 + G::NF * 4);            // f32[NF] diagonal (0: not fluid)
  static constexpr int ID = align128(DG + G::NF * 4);            // f32[NF] 1 / diagonal (0: not fluid)
  static constexpr int BAR = align128(ID + G::NF * 4);
  static constexpr int BYTES = BAR + 128;
};

template <typename T>
struct UpLayout {
  using G = TmaGeom<T>;
  static constexpr int X = 0;                                    // T[NF]   x from the down leg
  static constexpr int B = align128(X + G::NF * (int)sizeof(T)); // T[NF]   b
  static constexpr int E = align128(B + G::NF * (int)sizeof(T)); // T[NE]   coarse correction
  static constexpr int M = align128(E + G::NE * (int)sizeof(T)); // u8[NM]
  static constexpr int S0 = align128(M + G::NM);                 // f32[NF] corrected x
  static constexpr int S1 = align128(S0 + G::NF * 4);            // f32[NF] after sweep 1
  static constexpr int ID = align128(S1 + G::NF * 4);            // f32[NF] 1 / diagonal (0: not fluid)
  static constexpr int BAR = align128(ID + G::NF * 4);
  static constexpr int BYTES = BAR + 128;
};

template <typename T>
__device__ __forceinline__ float lds(const T* s, int i) {
  return ld(s, (size_t)i);
}

// Cell byte of global cell (gx, gy) whose box row is ly.
template <typename T, bool MASKED>
__device__ __forceinline__ uint8_t tma_cell(const LevelDev& L, const uint8_t* sm, int x0, int gx, int gy, int ly) {
  if (MASKED) return sm[ly * TmaGeom<T>::BWM + (gx - x0 + 16)];
  return (gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny) ? kFluidBit : 0;
}

__device__ __forceinline__ void tma_fail(SolveState* st) {
  if (st && threadIdx.x == 0) {
    st->status = MG_TIMEOUT;
    st->inner_done = 1;
    st->outer_done = 1;
  }
}

// Thread layout of the level kernels: 288 threads, the first 272 a 68 x 4
// grid over the 68-wide region (tile + 2 cells each side): thread (tx, ty)
// owns region column tx and rows ty, ty + 4, ...; the last 16 threads fill
// the diagonal tables.
constexpr int kTmaThreads = 288;
constexpr int kRX = kTmaTX + 4, kRY = kTmaTY + 4, kRowStep = 4;
static_assert(kRX * kRowStep + 16 == kTmaThreads, "thread layout");

// d and 1/d of a 2D cell by its link counts (kx + 4 ky, each 0..2): with
// no division per cell, a sweep is x <- (1 - omega) x + omega D^-1 (b + nb).
__device__ __forceinline__ void fill_diag_tables(const LevelDev& L, float* dtab, float* itab) {
  const int j = (int)threadIdx.x - kRX * kRowStep;
  if (j >= 0 && j < 16) {
    const int kx = j & 3, ky = j >> 2;
    const float d = (kx <= 2 && ky <= 2) ? L.wx * (float)kx + L.wy * (float)ky : 0.f;
    dtab[j] = d;
    itab[j] = d > 0.f ? 1.f / d : 0.f;
  }
}

template <bool MASKED>
__device__ __forceinline__ int diag_index(const LevelDev& L, uint8_t m, int kxu, int gy) {
  return MASKED ? (m & 15) : kxu + 4 * axis_count(gy, L.ny, L.bcD, 2);
}

template <typename T, bool MASKED>
__global__ void __launch_bounds__(kTmaThreads)
k_down_tma(const __grid_constant__ CUtensorMap tb, const __grid_constant__ CUtensorMap tm, LevelDev L,
           T* __restrict__ x, T* __restrict__ bcoarse, float omega, SolveState* __restrict__ st) {
  chain_enter();
  if (st && st->inner_done) return;
  using G = TmaGeom<T>;
  using Lo = DownLayout<T>;
  extern __shared__ __align__(128) unsigned char smem[];
  T* sb = reinterpret_cast<T*>(smem + Lo::B);
  uint8_t* sm = smem + Lo::M;
  float* s1 = reinterpret_cast<float*>(smem + Lo::X1);
  float* s2 = reinterpret_cast<float*>(smem + Lo::X2);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Lo::BAR);
  __shared__ float dtab[16], itab[16];
  const int x0 = blockIdx.x * kTmaTX, y0 = blockIdx.y * kTmaTY;
  fill_diag_tables(L, dtab, itab);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, G::NF * sizeof(T) + (MASKED ? G::NM : 0));
    tma_load_2d(sb, &tb, bar, x0 - G::MX, y0 - kTmaH);
    if (MASKED) tma_load_2d(sm, &tm, bar, x0 - 16, y0 - kTmaH);
  }
  if (!mbar_wait_bounded(bar, 0)) {
    tma_fail(st);
    return;
  }
  float* sdg = reinterpret_cast<float*>(smem + Lo::DG);
  float* sid = reinterpret_cast<float*>(smem + Lo::ID);
  const float om1 = 1.f - omega;
  const int tid = threadIdx.x;
  const bool on = tid < kRX * kRowStep;
  const int tx = on ? tid % kRX : 0, ty = on ? tid / kRX : 0;
  const int gx = x0 - 2 + tx;
  const bool xin = gx >= 0 && gx < L.nx;
  const int kxu = MASKED ? 0 : axis_count(gx, L.nx, L.bcD, 0);
  // sweep 1 from zero on the tile + 2: x1 = omega b / d
  if (on) {
#pragma unroll
    for (int k = 0; k < kRY / kRowStep; ++k) {
      const int ly = ty + kRowStep * k, gy = y0 - 2 + ly;
      const int li = ly * G::BW + tx + (G::MX - 2);
      const uint8_t m = MASKED ? sm[ly * G::BWM + tx + 14] : ((xin && gy >= 0 && gy < L.ny) ? kFluidBit : 0);
      const int q = diag_index<MASKED>(L, m, kxu, gy);
      const float d = m ? dtab[q] : 0.f, id = m ? itab[q] : 0.f;
      sdg[li] = d;
      sid[li] = id;
      s1[li] = omega * lds(sb, li) * id;
    }
  }
  __syncthreads();
  // sweep 2 on the tile + 1
  if (on && tx >= 1 && tx <= kRX - 2) {
#pragma unroll
    for (int k = 0; k < kRY / kRowStep; ++k) {
      const int ly = 1 + ty + kRowStep * k;
      if (ly <= kRY - 2) {
        const int li = ly * G::BW + tx + (G::MX - 2);
        const float nb = L.wx * (s1[li - 1] + s1[li + 1]) + L.wy * (s1[li - G::BW] + s1[li + G::BW]);
        s2[li] = fmaf(om1, s1[li], omega * sid[li] * (lds(sb, li) + nb));
      }
    }
  }
  __syncthreads();
  // residual on the tile, its 2x2 average, and x: one coarse cell per thread
  if (tid < 256) {
    const int cx = tid & 31, cy = tid >> 5;  // 32 x 8 coarse cells
    const int gcx = (x0 >> 1) + cx, gcy = (y0 >> 1) + cy;
    float sum = 0.f;
    float xo[2][2];
#pragma unroll
    for (int ay = 0; ay < 2; ++ay)
#pragma unroll
      for (int ax = 0; ax < 2; ++ax) {
        const int li = (2 + 2 * cy + ay) * G::BW + (G::MX + 2 * cx + ax);
        const float xc = s2[li];
        xo[ay][ax] = xc;
        // non-fluid cells (d = 0) are not unknowns: they add nothing
        const float dg = sdg[li];
        if (dg != 0.f)
          sum += lds(sb, li) - (dg * xc - L.wx * (s2[li - 1] + s2[li + 1]) - L.wy * (s2[li - G::BW] + s2[li + G::BW]));
      }
    if (gcx < (L.nx >> 1) && gcy < (L.ny >> 1)) {
#pragma unroll
      for (int ay = 0; ay < 2; ++ay) {
        const size_t gi = (size_t)(y0 + 2 * cy + ay) * L.nx + (x0 + 2 * cx);
        x[gi] = cvt<T>(xo[ay][0]);
        x[gi + 1] = cvt<T>(xo[ay][1]);
      }
      bcoarse[(size_t)gcy * (L.nx >> 1) + gcx] = cvt<T>(0.25f * sum);
    }
  }
}

template <typename T, bool MASKED, bool FINEST>
__global__ void __launch_bounds__(kTmaThreads)
k_up_tma(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tb,
         const __grid_constant__ CUtensorMap te, const __grid_constant__ CUtensorMap tm, LevelDev L,
         T* __restrict__ xout, float omega, float s, SolveState* __restrict__ st, double* __restrict__ partials) {
  chain_enter();
  if (st && st->inner_done) return;
  using G = TmaGeom<T>;
  using Lo = UpLayout<T>;
  extern __shared__ __align__(128) unsigned char smem[];
  T* sx = reinterpret_cast<T*>(smem + Lo::X);
  T* sb = reinterpret_cast<T*>(smem + Lo::B);
  T* se = reinterpret_cast<T*>(smem + Lo::E);
  uint8_t* sm = smem + Lo::M;
  float* s0 = reinterpret_cast<float*>(smem + Lo::S0);
  float* s1 = reinterpret_cast<float*>(smem + Lo::S1);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Lo::BAR);
  __shared__ float dtab[16], itab[16];
  const int x0 = blockIdx.x * kTmaTX, y0 = blockIdx.y * kTmaTY;
  const int ex0 = (x0 >> 1) - G::MX, ey0 = (y0 >> 1) - 1;
  fill_diag_tables(L, dtab, itab);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, (2 * G::NF + G::NE) * sizeof(T) + (MASKED ? G::NM : 0));
    tma_load_2d(sx, &tmx, bar, x0 - G::MX, y0 - kTmaH);
    tma_load_2d(sb, &tb, bar, x0 - G::MX, y0 - kTmaH);
    tma_load_2d(se, &te, bar, ex0, ey0);
    if (MASKED) tma_load_2d(sm, &tm, bar, x0 - 16, y0 - kTmaH);
  }
  if (!mbar_wait_bounded(bar, 0)) {
    tma_fail(st);
    return;
  }
  float* sid = reinterpret_cast<float*>(smem + Lo::ID);
  const float om1 = 1.f - omega;
  const int tid = threadIdx.x;
  const bool on = tid < kRX * kRowStep;
  const int tx = on ? tid % kRX : 0, ty = on ? tid / kRX : 0;
  const int gx = x0 - 2 + tx;
  const bool xin = gx >= 0 && gx < L.nx;
  const int kxu = MASKED ? 0 : axis_count(gx, L.nx, L.bcD, 0);
  const int lex = (gx >> 1) - ex0;
  // x + s P e and D^-1 on the tile + 2
  if (on) {
#pragma unroll
    for (int k = 0; k < kRY / kRowStep; ++k) {
      const int ly = ty + kRowStep * k, gy = y0 - 2 + ly;
      const int li = ly * G::BW + tx + (G::MX - 2);
      const uint8_t m = MASKED ? sm[ly * G::BWM + tx + 14] : ((xin && gy >= 0 && gy < L.ny) ? kFluidBit : 0);
      const int le = ((gy >> 1) - ey0) * G::BWE + lex;
      s0[li] = m ? lds(sx, li) + s * lds(se, le) : 0.f;
      sid[li] = m ? itab[diag_index<MASKED>(L, m, kxu, gy)] : 0.f;
    }
  }
  __syncthreads();
  // sweep 1 on the tile + 1
  if (on && tx >= 1 && tx <= kRX - 2) {
#pragma unroll
    for (int k = 0; k < kRY / kRowStep; ++k) {
      const int ly = 1 + ty + kRowStep * k;
      if (ly <= kRY - 2) {
        const int li = ly * G::BW + tx + (G::MX - 2);
        const float nb = L.wx * (s0[li - 1] + s0[li + 1]) + L.wy * (s0[li - G::BW] + s0[li + G::BW]);
        s1[li] = fmaf(om1, s0[li], omega * sid[li] * (lds(sb, li) + nb));
      }
    }
  }
  __syncthreads();
  // sweep 2 on the tile, straight to global memory
  float acc = 0.f;
  if (on && tx >= 2 && tx <= kRX - 3 && gx < L.nx) {
#pragma unroll
    for (int k = 0; k < kTmaTY / kRowStep; ++k) {
      const int ly = 2 + ty + kRowStep * k, gy = y0 - 2 + ly;
      if (gy < L.ny) {
        const int li = ly * G::BW + tx + (G::MX - 2);
        const float nb = L.wx * (s1[li - 1] + s1[li + 1]) + L.wy * (s1[li - G::BW] + s1[li + G::BW]);
        const float bv = lds(sb, li);
        const float v = fmaf(om1, s1[li], omega * sid[li] * (bv + nb));
        const T zt = cvt<T>(v);
        xout[(size_t)gy * L.nx + gx] = zt;
        if (FINEST) acc = fmaf(bv, ld(&zt, 0), acc);
      }
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

// ---------------------------------------------------------------------------
// host side
void* tensor_map_encoder() {
  static void* fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = p;
  }
  return fn;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  return (PFN_cuTensorMapEncodeTiled_v12000)tensor_map_encoder();
}

static bool encode_2d(CUtensorMap* m, const void* base, CUtensorMapDataType dt, int esz, int64_t nx, int64_t ny,
                      int bw, int bh) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn || ((uintptr_t)base & 15) || ((nx * esz) & 15)) return false;
  cuuint64_t gdim[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
  cuuint64_t gstride[1] = {(cuuint64_t)(nx * esz)};
  cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
  cuuint32_t es[2] = {1, 1};
  return fn(m, dt, 2, const_cast<void*>(base), gdim, gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

template <typename T>
static CUtensorMapDataType tma_dtype() {
  if (std::is_same<T, float>::value) return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  if (std::is_same<T, __half>::value) return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
}

bool tma_level_eligible(int dim, int pre, int post, const LevelDev& L) {
  return dim == 2 && pre == 2 && post == 2 && (L.nx % 16) == 0 && L.nx >= 16 && L.ny >= 2 && encode_fn() != nullptr;
}

template <typename T>
bool tma_encode_level(TmaLevelMaps* out, const LevelDev& L, const void* b, const void* x, const void* e) {
  using G = TmaGeom<T>;
  const int esz = (int)sizeof(T);
  bool ok = encode_2d(&out->b, b, tma_dtype<T>(), esz, L.nx, L.ny, G::BW, G::BH);
  ok = ok && encode_2d(&out->x, x, tma_dtype<T>(), esz, L.nx, L.ny, G::BW, G::BH);
  ok = ok && encode_2d(&out->e, e, tma_dtype<T>(), esz, L.nx / 2, L.ny / 2, G::BWE, G::BHE);
  if (L.cell) ok = ok && encode_2d(&out->m, L.cell, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, L.nx, L.ny, G::BWM, G::BH);
  else out->m = out->b;  // unused
  return ok;
}

template <typename T>
bool tma_encode_b(CUtensorMap* out, const LevelDev& L, const void* b) {
  using G = TmaGeom<T>;
  return encode_2d(out, b, tma_dtype<T>(), (int)sizeof(T), L.nx, L.ny, G::BW, G::BH);
}

static dim3 tma_grid(const LevelDev& L) {
  return dim3((L.nx + kTmaTX - 1) / kTmaTX, (L.ny + kTmaTY - 1) / kTmaTY, 1);
}

template <typename T, bool MASKED>
cudaError_t launch_down_tma(const TmaLevelMaps& m, const LevelDev& L, void* x, void* bcoarse, float omega,
                            SolveState* st, cudaStream_t s) {
  return launch_chain(k_down_tma<T, MASKED>, tma_grid(L), kTmaThreads, DownLayout<T>::BYTES, s, m.b, m.m, L, (T*)x,
                      (T*)bcoarse, omega, st);
}

template <typename T, bool MASKED, bool FINEST>
cudaError_t launch_up_tma(const TmaLevelMaps& m, const LevelDev& L, void* xout, float omega, float sc,
                          SolveState* st, double* partials, cudaStream_t s) {
  return launch_chain(k_up_tma<T, MASKED, FINEST>, tma_grid(L), kTmaThreads, UpLayout<T>::BYTES, s, m.x, m.b, m.e, m.m,
                      L, (T*)xout, omega, sc, st, partials);
}

template <typename K>
static cudaError_t tma_allow(K k, int bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes + 1024);
}

template <typename T, bool MASKED>
cudaError_t prepare_tma_kernels() {
  cudaError_t e = tma_allow(k_down_tma<T, MASKED>, DownLayout<T>::BYTES);
  if (e == cudaSuccess) e = tma_allow(k_up_tma<T, MASKED, false>, UpLayout<T>::BYTES);
  if (e == cudaSuccess) e = tma_allow(k_up_tma<T, MASKED, true>, UpLayout<T>::BYTES);
  return e;
}

#define NPMG_INST_TMA(T, M)                                                                                   \
  template cudaError_t launch_down_tma<T, M>(const TmaLevelMaps&, const LevelDev&, void*, void*, float,      \
                                             SolveState*, cudaStream_t);                                      \
  template cudaError_t launch_up_tma<T, M, false>(const TmaLevelMaps&, const LevelDev&, void*, float, float,  \
                                                  SolveState*, double*, cudaStream_t);                        \
  template cudaError_t launch_up_tma<T, M, true>(const TmaLevelMaps&, const LevelDev&, void*, float, float,   \
                                                 SolveState*, double*, cudaStream_t);                         \
  template cudaError_t prepare_tma_kernels<T, M>();

NPMG_INST_TMA(float, false)
NPMG_INST_TMA(float, true)
NPMG_INST_TMA(__half, false)
NPMG_INST_TMA(__half, true)
NPMG_INST_TMA(__nv_bfloat16, false)
NPMG_INST_TMA(__nv_bfloat16, true)

template bool tma_encode_level<float>(TmaLevelMaps*, const LevelDev&, const void*, const void*, const void*);
template bool tma_encode_level<__half>(TmaLevelMaps*, const LevelDev&, const void*, const void*, const void*);
template bool tma_encode_level<__nv_bfloat16>(TmaLevelMaps*, const LevelDev&, const void*, const void*,
                                              const void*);
template bool tma_encode_b<float>(CUtensorMap*, const LevelDev&, const void*);
template bool tma_encode_b<__half>(CUtensorMap*, const LevelDev&, const void*);
template bool tma_encode_b<__nv_bfloat16>(CUtensorMap*, const LevelDev&, const void*);

}  // namespace npmg
