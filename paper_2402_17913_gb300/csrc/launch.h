// Kernel launchers exported between the library's translation units.
#pragma once
#include <utility>

#include "npmg_internal.cuh"

namespace npmg {

// Launch a kernel of the solve's launch chain (it starts with chain_enter):
// with the programmatic-serialization attribute unless NPMG_NO_PDL is set.
bool chain_launch_enabled();
template <typename... KArgs, typename... Args>
cudaError_t launch_chain(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = chain_launch_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

struct CoarseArgs {
  int nlev;                    // levels handled by the single-block kernel
  int dim;
  LevelDev lv[kMaxLevels];     // lv[0] = first level handled
  int off[kMaxLevels];         // float offset of level l's padded arrays (x, x', b, 1/diag)
  int ncoarse;                 // cells of the coarsest level
  const float* inv;            // inverse of the coarsest operator (float32, symmetric)
  const float* image;          // constant shared-memory image (zero rings, 1/diag), or nullptr
  int pre, post;
  float omega, s;
  int finest;                  // lv[0] is the finest level: reduce (r, z)
};

size_t coarse_layout(int* off, const LevelDev* lv, int nlev, int dim);
// Write the constant part of the single-block kernel's shared memory (zero
// ghost rings and arrays, inverse diagonals) to `image` (device).
cudaError_t launch_coarse_image(const CoarseArgs& a, float* image, size_t bytes, cudaStream_t s);
int coarse_start_level(const LevelDev* lv, int L, int dim, size_t smem_limit);

// Level legs: T is the storage of a level's iterate and of its coarse-side
// arrays, TB that of its right-hand side b and of the up leg's output (the
// float32 CG vectors on the finest level, else T).
template <int DIM, typename T, bool MASKED, typename TB = T>
cudaError_t launch_down(const LevelDev& L, const void* b, void* x, void* bcoarse, int pre, float omega,
                        const SolveState* st, cudaStream_t s);
// Sawtooth down leg (no sweeps: x = b / d, coarse b = average of b); b and
// x must be 8-byte aligned (levels with a down leg have even sides).
template <int DIM, typename T, bool MASKED, typename TB = T>
cudaError_t launch_down_saw(const LevelDev& L, const void* b, void* x, void* bcoarse, const SolveState* st,
                            cudaStream_t s);
template <int DIM, typename T, bool MASKED, bool FINEST, typename TB = T>
cudaError_t launch_up(const LevelDev& L, const void* b, const void* xin, void* xout, const void* e, int post,
                      float omega, float sc, SolveState* st, double* partials, cudaStream_t s);

template <int DIM, typename T, bool MASKED>
cudaError_t prepare_level_kernels(int pre, int post);

// 3D level kernels streamed along z (two sweeps; mg_stream3d.cu).
bool stream3d_eligible(int dim, int pre, int post, const LevelDev& L);
template <typename T, bool MASKED, typename TB = T>
cudaError_t launch_down_s3(const LevelDev& L, const void* b, void* x, void* bcoarse, float omega,
                           const SolveState* st, cudaStream_t s);
template <typename T, bool MASKED, bool FINEST, typename TB = T>
cudaError_t launch_up_s3(const LevelDev& L, const void* b, const void* xin, void* xout, const void* e, float omega,
                         float sc, SolveState* st, double* partials, cudaStream_t s);
template <typename T, bool MASKED>
cudaError_t prepare_s3_kernels();
// 2D level kernels streamed along y by single warps (two sweeps;
// mg_stream2d.cu); arrays 16-byte aligned.
bool stream2d_eligible(int dim, int pre, int post, const LevelDev& L);
bool stream2d_aligned(const void* p);
size_t stream2d_min_cells();
template <typename T, bool MASKED, typename TB = T>
cudaError_t launch_down_w(const LevelDev& L, const void* b, void* x, void* bcoarse, float omega, const SolveState* st,
                          cudaStream_t s);
template <typename T, bool MASKED, bool FINEST, typename TB = T>
cudaError_t launch_up_w(const LevelDev& L, const void* b, const void* xin, void* xout, const void* e, float omega,
                        float sc, SolveState* st, double* partials, cudaStream_t s);
// 3D level kernels, a block per 128 x 16 column streamed along z with a
// warp per row (two sweeps; mg_rows3d.cu); arrays 16-byte aligned.
bool rows3d_eligible(int dim, int pre, int post, const LevelDev& L);
template <typename T, bool MASKED, typename TB = T>
cudaError_t launch_down_r3(const LevelDev& L, const void* b, void* x, void* bcoarse, float omega, const SolveState* st,
                           cudaStream_t s);
template <typename T, bool MASKED, bool FINEST, typename TB = T>
cudaError_t launch_up_r3(const LevelDev& L, const void* b, const void* xin, void* xout, const void* e, float omega,
                         float sc, SolveState* st, double* partials, cudaStream_t s);
template <typename T, bool MASKED>
cudaError_t prepare_r3_kernels();
template <typename T>
cudaError_t prepare_coarse(size_t smem_bytes);

template <typename T>
cudaError_t launch_coarse(const CoarseArgs& a, size_t smem_bytes, const void* b, void* x, SolveState* st,
                          cudaStream_t s);

// The middle levels of a 2D V-cycle (float32, two sweeps) in one thread-block
// cluster, with the coarse cycle of the levels below in its block 0
// (mg_cluster2d.cu).  A distributed level in every block: three float
// arrays (two iterate buffers, b) and one byte array (cell bytes) of
// (R + 2) rows of W = nx + 8 entries: ghost rows 0 and R + 1, the row's
// cells at columns 4 .. nx + 3 (16-byte aligned), zero ghost columns 3 and
// nx + 4.
struct CLev {
  LevelDev L;      // weights, faces, cell bytes of the whole level (global)
  int R;           // rows per block (even)
  int W;           // padded row (nx + 8)
  int off;         // float offset of the level's arrays
  int moff;        // byte offset of its cell bytes
  int loff;        // float offset of its diagonal table (64 d, 64 omega / d)
  int s4;          // log2 of nx / 4 when a power of two, else -1
};
struct ClusterArgs {
  int nlev, C;              // distributed levels (k1 .. kd-1), blocks in the cluster
  CLev lv[kMaxLevels];
  CoarseArgs ca;            // levels kd .. L-1, on block 0
  int ca_off;               // float offset of the coarse cycle's region
  int ca_floats;
  float omega, s;
};
// Plan the cluster launch: the first distributed level k1, the first level
// of the coarse cycle kd (the first level after k1 within the coarse-cell
// limit, at least kc), the cluster size, the shared-memory bytes, and the
// coarse cycle's level offsets (out->ca.off, out->ca.lv, out->ca.nlev).
// False when no level qualifies.
bool cluster2d_plan(const LevelDev* lv, int L, int kc, ClusterArgs* out, int* k1_out, int* kd_out,
                    size_t* smem_out, size_t* ca_bytes_out);
cudaError_t launch_cluster2d(const ClusterArgs& a, size_t smem, const float* bin, float* yout, float* bkc,
                             float* ykc, SolveState* st, cudaStream_t s);
// A small 2D grid's inner CG solve in one cluster launch
// (mg_cluster_pcg2d.cu): levels 0 .. kd-1 distributed as above (a.lv[0] the
// finest level), level 0's CG vectors beside them (r is level 0's b, z its
// x1; two p buffers and d at pcg_off, each in level 0's padded layout).
struct ClusterPcgArgs {
  ClusterArgs a;
  int pcg_off;             // float offset of p0 | p1 | d
  int red_off;             // float offset of the reduction slots (2 x 16 float pairs)
};
bool cluster_pcg2d_plan(const LevelDev* lv, int L, int kc, ClusterPcgArgs* out, int* kd_out, size_t* smem_out,
                        size_t* ca_bytes_out);
// Set the kernel's shared-memory and cluster attributes; the number of
// clusters of C blocks with `smem` bytes each the GPU can hold (0: none).
int cluster_pcg2d_fit(size_t smem, size_t smem_limit, int C);
// r0: the scaled residual the inner solve starts from; dout: its solution
// d' (for the refinement step); st: the solve state (nothing runs when the
// inner or the outer loop is done).
cudaError_t launch_cluster_pcg2d(const ClusterPcgArgs& pa, size_t smem, const float* r0, float* dout, float* bkc,
                                 float* ykc, SolveState* st, cudaStream_t s);
template <int DIM, typename T, bool MASKED>
cudaError_t launch_p_update(const LevelDev& L, const void* z, const void* pold, void* pnew, void* Ap,
                            SolveState* st, double* partials, cudaStream_t s);
template <typename T>
cudaError_t launch_xr_update(const LevelDev& L, const void* p, const void* Ap, void* d, void* r, SolveState* st,
                             double* partials, cudaStream_t s);
// x: float-float iterate (float2 per cell); w: operator weights c / h_a^2.
// dyn: xin / xout are the two buffers and the state's `cur` picks the one
// holding the iterate (flipped after an update).
// f64: the iterate is a float64 array and the residual is formed in
// float64 (T must then be float); otherwise float-float pairs.
template <int DIM, typename T, bool MASKED, bool UPDATE>
cudaError_t launch_outer(const LevelDev& L, const double w[3], double c, const float* b, const void* xin, void* xout,
                         const void* dprime, void* rprime, SolveState* st, double* partials, cudaStream_t s,
                         int dyn = 0, bool f64 = false);
// Conditional values of the device-side solve loop (see mg_cg.cu).
cudaError_t launch_loop_start(cudaGraphConditionalHandle outer, SolveState* st, cudaStream_t s);
cudaError_t launch_loop_inner(cudaGraphConditionalHandle inner, SolveState* st, unsigned int cap, int body,
                              cudaStream_t s);
cudaError_t launch_loop_outer(cudaGraphConditionalHandle outer, SolveState* st, unsigned int cap, cudaStream_t s);
cudaError_t launch_loop_set_cur(SolveState* st, int cur, cudaStream_t s);

struct SolveParams {
  double tol, inner_floor;
  int max_inner, max_outer, krylov, n_fluid;
};
// f64: the iterate x is a float64 array (else float-float pairs).
cudaError_t launch_init(const LevelDev& L, const float* b, const float* xguess, void* x, double c, SolveParams prm,
                        SolveState* st, double* partials, cudaStream_t s, bool f64);
// xb != nullptr: the iterate is in x when the state's `cur` is 0, else in xb
// (after the device-side loop, which flips `cur`).
cudaError_t launch_finish(size_t n, void* x, void* xb, float* out, const SolveState* st, int nblocks, cudaStream_t s,
                          bool f64);
cudaError_t launch_ff_to_f64(size_t n, const void* x, double* out, int nblocks, cudaStream_t s, bool f64);

// set-up kernels
cudaError_t launch_coarsen_solid(int dim, const int64_t fine[3], const uint8_t* sf, uint8_t* sc, cudaStream_t s);
cudaError_t launch_cell_bytes(int dim, const int64_t n[3], int bcD, const uint8_t* solid, uint8_t* cell,
                              cudaStream_t s);
// `mat`: 2 n^2 doubles of workspace; on return its first n^2 floats hold the
// inverse (computed in float64, stored in float32)
cudaError_t launch_coarse_inverse(int dim, const int64_t n[3], const double w[3], int bcD, const uint8_t* cell,
                                  double* mat, cudaStream_t s);

// per-kernel building blocks (float32 only)
template <int DIM, bool MASKED>
cudaError_t launch_apply(const LevelDev& L, const float* x, float* y, cudaStream_t s);
template <int DIM, bool MASKED>
cudaError_t launch_smooth_once(const LevelDev& L, const float* x, float* y, const float* b, float omega,
                               cudaStream_t s);
template <int DIM, bool MASKED>
cudaError_t launch_restrict_residual(const LevelDev& L, const float* x, const float* b, float* bc, cudaStream_t s);
template <int DIM, bool MASKED>
cudaError_t launch_prolong_correct(const LevelDev& L, const float* e, float* x, float sc, cudaStream_t s);

}  // namespace npmg
