// Definition of the opaque solver handle (host side).
#pragma once
#include <type_traits>

#include "launch.h"
#include "tma_host.h"

namespace npmg {

constexpr int kChunk = 4;              // CG iterations per graph launch
constexpr int kMaxPartials = 1 << 16;  // per-block partial sums
constexpr int kProfEvents = 4096;      // event pairs buffered by the profiler

}  // namespace npmg

struct mg_handle_s {
  int dim, L, kc, device, nsm, esz, use_graph;
  int guess_check;  // restart from zero when the initial guess has relres > 1
  int64_t n[npmg::kMaxLevels][3];
  double h[npmg::kMaxLevels][3];
  size_t ncell[npmg::kMaxLevels];
  int bc[6], bcD;
  bool masked;
  mg_options opt;
  double inner_floor;
  double c;        // h_0x^2: A' = c A_h
  double w0[3];    // finest-level operator weights c / h_0a^2
  int n_fluid;
  npmg::LevelDev lv[npmg::kMaxLevels];
  // device workspace (one allocation)
  char* pool;
  size_t pool_bytes;
  uint8_t* solid[npmg::kMaxLevels];
  uint8_t* cell[npmg::kMaxLevels];
  void* xk[npmg::kMaxLevels];
  void* yk[npmg::kMaxLevels];
  void* bk[npmg::kMaxLevels];
  void *r, *z, *p[2], *Ap, *d;
  void* xff[2];    // refinement iterate per cell (float64, or float-float hi/lo pairs), double-buffered
  int cur64;
  double* inv;
  float* cimage;   // constant shared-memory image of the single-block kernel
  int ncoarse;
  double* partials;
  npmg::SolveState* st;
  npmg::SolveState* st_host;  // pinned
  npmg::CoarseArgs ca;
  size_t ca_smem;
  int nb1d;
  cudaEvent_t ev0, ev1;
  cudaGraphExec_t graph_exec;
  // the whole refinement loop after the first residual as one graph with
  // nested conditional while nodes (built on first use; loop_state 0 = not
  // built, 1 = built, -1 = not available, the host loop runs instead)
  cudaGraphExec_t loop_exec;
  int loop_state;
  float* bsave;            // the right-hand side the loop graph reads (pool)
  int64_t loop_kernels;    // kernels in one inner body of the loop graph
  npmg::TmaLevelMaps tmaps[npmg::kMaxLevels];  // TMA tensor maps per level (levels < kc)
  bool tma_ok[npmg::kMaxLevels];
  bool s3_ok[npmg::kMaxLevels];   // 3D levels on the z-streaming kernels
  bool s2_ok[npmg::kMaxLevels];   // 2D levels on the y-streaming warp kernels
  bool r3_ok[npmg::kMaxLevels];   // 3D levels on the row-warp z-streaming kernels
  npmg::Tma3Maps t3maps[npmg::kMaxLevels];  // tensor maps of the TMA-fed 3D kernels (levels < kc)
  bool t3_ok[npmg::kMaxLevels];   // 3D levels on the TMA-fed z-streaming kernels
  npmg::Tma3CgMaps t3cg;          // the finest level's CG direction update on the TMA-fed kernel
  bool t3cg_ok;
  npmg::ClusterArgs clu;          // 2D: levels clu_k1 .. clu_kd-1 and the coarse cycle in one cluster launch
  bool clu_ok;
  int clu_k1, clu_kd;
  size_t clu_smem;
  float *clu_b, *clu_y;           // right-hand side and correction of level clu_kd (float32)
  float* clu_image;               // constant shared-memory image of the cluster's coarse cycle
  npmg::ClusterPcgArgs cpcg;      // 2D: the whole CG solve of a small grid in one cluster launch
  bool cpcg_ok;
  int cpcg_kd;
  size_t cpcg_smem;
  float* cpcg_image;              // its coarse cycle's constant image
  int64_t chunk_kernels;   // kernels in one graph launch
  // instrumentation
  int64_t launches;
  int prof;
  int capturing;
  cudaEvent_t* pev;        // 2 * kProfEvents events (created on enable)
  int pcls[npmg::kProfEvents];
  int pused;
  cudaStream_t plast;
  double prof_ms[MG_K_COUNT];
  int64_t prof_n[MG_K_COUNT];
};

namespace npmg {
// Brackets one kernel launch: counts it and, with profiling on, records a
// start/end event pair on the launch stream.
struct LaunchScope {
  mg_handle_s* h;
  int idx;
  cudaStream_t s;
  LaunchScope(mg_handle_s* hh, int cls, cudaStream_t ss);
  ~LaunchScope();
};
cudaError_t prof_flush(mg_handle_s* h);
const char* last_error();
mg_status run_solve(mg_handle_s* h, const float* b, float* x, double tol, cudaStream_t s, mg_stats* out);
int default_blocks_1d(const mg_handle_s* h, size_t n);
}  // namespace npmg
