// Host interface of the TMA-staged level kernels (mg_tma.cu).
#pragma once
#include <cuda.h>

#include "npmg_internal.cuh"

namespace npmg {

constexpr int kTmaTX = 64, kTmaTY = 16, kTmaH = 2;  // tile and halo of the TMA level kernels

// Tensor maps of one level: right-hand side b, the down leg's x, the coarse
// correction e (next level), the cell bytes m.
struct TmaLevelMaps {
  CUtensorMap b, x, e, m;
};

// The driver's cuTensorMapEncodeTiled (version 12000), or nullptr.
void* tensor_map_encoder();

bool tma_level_eligible(int dim, int pre, int post, const LevelDev& L);
template <typename T>
bool tma_encode_level(TmaLevelMaps* out, const LevelDev& L, const void* b, const void* x, const void* e);
template <typename T>
bool tma_encode_b(CUtensorMap* out, const LevelDev& L, const void* b);
template <typename T, bool MASKED>
cudaError_t launch_down_tma(const TmaLevelMaps& m, const LevelDev& L, void* x, void* bcoarse, float omega,
                            SolveState* st, cudaStream_t s);
template <typename T, bool MASKED, bool FINEST>
cudaError_t launch_up_tma(const TmaLevelMaps& m, const LevelDev& L, void* xout, float omega, float sc,
                          SolveState* st, double* partials, cudaStream_t s);
template <typename T, bool MASKED>
cudaError_t prepare_tma_kernels();

// Tensor maps of one 3D level for the TMA-fed z-streaming kernels
// (mg_tma3d.cu): b, the up leg's x, the coarse correction e, the cell bytes.
struct Tma3Maps {
  CUtensorMap x, b, e, m;
};

bool tma3d_eligible(int dim, int pre, int post, const LevelDev& L);
template <typename T, typename TB>
bool tma3d_encode(Tma3Maps* out, const LevelDev& L, const void* b, const void* x, const void* e);
template <typename TB>
bool tma3d_encode_b(CUtensorMap* out, const LevelDev& L, const void* b);
template <typename T, bool MASKED, typename TB>
cudaError_t launch_down_t3(const Tma3Maps& m, const LevelDev& L, void* x, void* bcoarse, float omega,
                           const SolveState* st, cudaStream_t s);
template <typename T, bool MASKED, bool FINEST, typename TB>
cudaError_t launch_up_t3(const Tma3Maps& m, const LevelDev& L, void* xout, float omega, float sc, SolveState* st,
                         double* partials, cudaStream_t s);
template <typename T, bool MASKED>
cudaError_t prepare_t3_kernels();

// Tensor maps of the finest level's CG updates (float32): z, the two p
// buffers, d and r, the cell bytes.
struct Tma3CgMaps {
  CUtensorMap z, p[2], d, r, m;
};
bool tma3d_encode_cg(Tma3CgMaps* out, const LevelDev& L, const float* z, const float* p0, const float* p1,
                     const float* d, const float* r);
// p = z + beta p_old (p_old = p[parity]), (p, A p) and alpha; A p stored
// only with store_ap.
template <bool MASKED>
cudaError_t launch_p_update_t3(const Tma3CgMaps& m, int parity, const LevelDev& L, float* pnew, float* Ap,
                               bool store_ap, SolveState* st, double* partials, cudaStream_t s);
// d += alpha p, r -= alpha A p (A p formed again from p = p[pbuf]), ||r||^2.
template <bool MASKED>
cudaError_t launch_xr_update_t3(const Tma3CgMaps& m, int pbuf, const LevelDev& L, float* d, float* r,
                                SolveState* st, double* partials, cudaStream_t s);

}  // namespace npmg
