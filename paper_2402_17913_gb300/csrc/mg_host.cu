// C ABI of the multigrid solver: create / solve / destroy and the
// per-kernel building blocks.  Host code only orchestrates: every arithmetic
// step of a solve runs in the library's kernels.
#include <initializer_list>
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "launch.h"
#include "mg_handle.h"

namespace npmg {

static thread_local char g_err[512] = "no error";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

const char* last_error() { return g_err; }

bool chain_launch_enabled() {
  static const bool on = getenv("NPMG_NO_PDL") == nullptr;
  return on;
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

LaunchScope::LaunchScope(mg_handle_s* hh, int cls, cudaStream_t ss) : h(hh), idx(-1), s(ss) {
  h->launches += 1;
  if (!h->prof || h->capturing || !h->pev) return;
  if (h->pused >= kProfEvents) prof_flush(h);
  idx = h->pused++;
  h->pcls[idx] = cls;
  h->plast = s;
  cudaEventRecord(h->pev[2 * idx], s);
}

LaunchScope::~LaunchScope() {
  if (idx >= 0) cudaEventRecord(h->pev[2 * idx + 1], s);
}

cudaError_t prof_flush(mg_handle_s* h) {
  if (!h->pev || h->pused == 0) return cudaSuccess;
  cudaError_t e = cudaEventSynchronize(h->pev[2 * (h->pused - 1) + 1]);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < h->pused; ++i) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, h->pev[2 * i], h->pev[2 * i + 1]);
    if (e != cudaSuccess) return e;
    h->prof_ms[h->pcls[i]] += ms;
    h->prof_n[h->pcls[i]] += 1;
  }
  h->pused = 0;
  return cudaSuccess;
}

// The refinement iterate and residual in float64 (MG_REFINE_FP64, the
// default) or in float-float pairs (MG_REFINE_FF); 8 bytes per cell either way.
static bool f64_iterate(const mg_handle_s* h) { return h->opt.refine != MG_REFINE_FF; }

int default_blocks_1d(const mg_handle_s* h, size_t n) {
  size_t b = (n + 255) / 256;
  const size_t cap = (size_t)h->nsm * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// ---------------------------------------------------------------------------
// Dispatch on (dim, storage type, masked) to a templated functor.
template <typename F>
static cudaError_t dispatch(const mg_handle_s* h, F&& f) {
  const bool m = h->masked;
#define NPMG_D(DIM, T)                                                                          \
  return m ? f(std::integral_constant<int, DIM>(), (T*)nullptr, std::true_type())              \
           : f(std::integral_constant<int, DIM>(), (T*)nullptr, std::false_type())
  if (h->dim == 2) {
    if (h->opt.prec == MG_FP32) NPMG_D(2, float);
    if (h->opt.prec == MG_MIXED_FP16) NPMG_D(2, __half);
    NPMG_D(2, __nv_bfloat16);
  }
  if (h->opt.prec == MG_FP32) NPMG_D(3, float);
  if (h->opt.prec == MG_MIXED_FP16) NPMG_D(3, __half);
  NPMG_D(3, __nv_bfloat16);
#undef NPMG_D
}

// One application of the preconditioner M (one cycle from a zero guess):
// down legs on levels 0 .. kc-1, the single-block kernel for kc .. L-1, up
// legs back to level 0.  With `st` it is the CG preconditioner (kernels skip
// once CG converged; the finest up leg reduces (r, z)).
// Down / up leg of level k with right-hand-side storage TB (float on the
// finest level, whose b and z are CG vectors; T elsewhere).  `tma` selects
// the TMA tile kernels (only for TB == T).
template <int DIM, typename T, bool M, typename TB>
static cudaError_t down_leg(mg_handle_s* h, int k, const void* b, const TmaLevelMaps* tm, const Tma3Maps* t3,
                            SolveState* st, cudaStream_t s) {
  const float om = (float)h->opt.omega;
  // the sawtooth down leg (no sweeps: x = b / d, the restriction of b) is
  // a plain stream; pre = -1 asks the tile kernel for it when b is not
  // aligned for paired loads.  The fused kernels below run V legs.
  if (h->opt.cycle == MG_CYCLE_SAWTOOTH) {
    if (stream2d_aligned(b)) return launch_down_saw<DIM, T, M, TB>(h->lv[k], b, h->xk[k], h->bk[k + 1], st, s);
    return launch_down<DIM, T, M, TB>(h->lv[k], b, h->xk[k], h->bk[k + 1], -1, om, st, s);
  }
  if (DIM == 2 && h->s2_ok[k] && stream2d_aligned(b))
    return launch_down_w<T, M, TB>(h->lv[k], b, h->xk[k], h->bk[k + 1], om, st, s);
  if constexpr (std::is_same<T, TB>::value) {
    if (tm) return launch_down_tma<T, M>(*tm, h->lv[k], h->xk[k], h->bk[k + 1], om, st, s);
  }
  if (DIM == 3 && t3) return launch_down_t3<T, M, TB>(*t3, h->lv[k], h->xk[k], h->bk[k + 1], om, st, s);
  if (DIM == 3 && h->r3_ok[k] && stream2d_aligned(b))
    return launch_down_r3<T, M, TB>(h->lv[k], b, h->xk[k], h->bk[k + 1], om, st, s);
  if (DIM == 3 && h->s3_ok[k]) return launch_down_s3<T, M, TB>(h->lv[k], b, h->xk[k], h->bk[k + 1], om, st, s);
  return launch_down<DIM, T, M, TB>(h->lv[k], b, h->xk[k], h->bk[k + 1], h->opt.pre, om, st, s);
}

template <int DIM, typename T, bool M, bool F, typename TB>
static cudaError_t up_leg(mg_handle_s* h, int k, const void* b, void* xo, const TmaLevelMaps* tm,
                          const Tma3Maps* t3, SolveState* st, cudaStream_t s) {
  const float om = (float)h->opt.omega, sc = (float)h->opt.coarse_scale;
  if (DIM == 2 && h->s2_ok[k] && stream2d_aligned(b))
    return launch_up_w<T, M, F, TB>(h->lv[k], b, h->xk[k], xo, h->yk[k + 1], om, sc, st, h->partials, s);
  if constexpr (std::is_same<T, TB>::value) {
    if (tm) return launch_up_tma<T, M, F>(*tm, h->lv[k], xo, om, sc, st, h->partials, s);
  }
  if (DIM == 3 && t3) return launch_up_t3<T, M, F, TB>(*t3, h->lv[k], xo, om, sc, st, h->partials, s);
  if (DIM == 3 && h->r3_ok[k] && stream2d_aligned(b))
    return launch_up_r3<T, M, F, TB>(h->lv[k], b, h->xk[k], xo, h->yk[k + 1], om, sc, st, h->partials, s);
  if (DIM == 3 && h->s3_ok[k])
    return launch_up_s3<T, M, F, TB>(h->lv[k], b, h->xk[k], xo, h->yk[k + 1], om, sc, st, h->partials, s);
  return launch_up<DIM, T, M, F, TB>(h->lv[k], b, h->xk[k], xo, h->yk[k + 1], h->opt.post, om, sc, st, h->partials,
                                     s);
}

// One application of the preconditioner M (one cycle from a zero guess):
// down legs on levels 0 .. kc-1, the single-block kernel for kc .. L-1, up
// legs back to level 0.  r and z (level 0's right-hand side and output) are
// float32; the level arrays below are T.  With `st` it is the CG
// preconditioner (kernels skip once CG converged; the finest up leg reduces
// (r, z)).
template <int DIM, typename T, bool M>
static cudaError_t enqueue_vcycle(mg_handle_s* h, const void* r, void* z, SolveState* st, cudaStream_t s) {
  cudaError_t e;
  // TMA tensor maps (float32 handles): level 0 reads r, which is the
  // caller's array in the building-block path, so its map is re-encoded
  // when r is not the handle's
  TmaLevelMaps m0;
  bool tma0 = h->tma_ok[0];
  if (tma0) {
    m0 = h->tmaps[0];
    if (r != h->r) tma0 = tma_encode_b<float>(&m0.b, h->lv[0], r);
  }
  Tma3Maps t30;
  bool t3ok0 = h->t3_ok[0];
  if (t3ok0) {
    t30 = h->t3maps[0];
    if (r != h->r) t3ok0 = tma3d_encode_b<float>(&t30.b, h->lv[0], r);
  }
  auto t3of = [&](int k) -> const Tma3Maps* {
    if (k == 0) return t3ok0 ? &t30 : nullptr;
    return h->t3_ok[k] ? &h->t3maps[k] : nullptr;
  };
  // 2D float32 V-cycles: the levels clu_k1 .. clu_kd-1 and the coarse cycle
  // of the levels below in one cluster launch (their legs are not launched
  // one by one)
  const bool clu = DIM == 2 && h->clu_ok;
  const int kdown = clu ? h->clu_k1 : h->kc;
  for (int k = 0; k < kdown; ++k) {
    LaunchScope ls(h, k == 0 ? MG_K_DOWN_FINE : MG_K_DOWN, s);
    if (k == 0)
      e = down_leg<DIM, T, M, float>(h, 0, r, tma0 ? &m0 : nullptr, t3of(0), st, s);
    else
      e = down_leg<DIM, T, M, T>(h, k, h->bk[k], h->tma_ok[k] ? &h->tmaps[k] : nullptr, t3of(k), st, s);
    if (e != cudaSuccess) return e;
  }
  CoarseArgs ca = h->ca;
  ca.finest = (h->kc == 0 && st) ? 1 : 0;
  {
    LaunchScope ls(h, MG_K_COARSE, s);
    if (clu)
      e = launch_cluster2d(h->clu, h->clu_smem, (const float*)h->bk[kdown], (float*)h->yk[kdown], h->clu_b,
                           h->clu_y, st, s);
    else
      e = h->kc == 0 ? launch_coarse<float>(ca, h->ca_smem, r, z, st, s)
                     : launch_coarse<T>(ca, h->ca_smem, h->bk[h->kc], h->yk[h->kc], st, s);
  }
  if (e != cudaSuccess) return e;
  for (int k = kdown - 1; k >= 0; --k) {
    LaunchScope ls(h, k == 0 ? MG_K_UP_FINE : MG_K_UP, s);
    if (k == 0 && st)
      e = up_leg<DIM, T, M, true, float>(h, 0, r, z, tma0 ? &m0 : nullptr, t3of(0), st, s);
    else if (k == 0)
      e = up_leg<DIM, T, M, false, float>(h, 0, r, z, tma0 ? &m0 : nullptr, t3of(0), st, s);
    else
      e = up_leg<DIM, T, M, false, T>(h, k, h->bk[k], h->yk[k], h->tma_ok[k] ? &h->tmaps[k] : nullptr, t3of(k),
                                      st, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One CG iteration: z = M r, p = z + beta p, Ap, alpha, d += alpha p,
// r -= alpha Ap, convergence flag.  `parity` selects the p double buffer.
template <int DIM, typename T, bool M>
static cudaError_t enqueue_iteration(mg_handle_s* h, int parity, cudaStream_t s) {
  cudaError_t e = enqueue_vcycle<DIM, T, M>(h, h->r, h->z, h->st, s);
  if (e != cudaSuccess) return e;
  {
    LaunchScope ls(h, MG_K_P_UPDATE, s);
    // on the TMA-fed kernels A p is not stored: the vector update forms it
    // again from p
    if (DIM == 3 && h->t3cg_ok)
      e = launch_p_update_t3<M>(h->t3cg, parity, h->lv[0], (float*)h->p[1 - parity], (float*)h->Ap, false, h->st,
                                h->partials, s);
    else
      e = launch_p_update<DIM, float, M>(h->lv[0], h->z, h->p[parity], h->p[1 - parity], h->Ap, h->st, h->partials,
                                         s);
  }
  if (e != cudaSuccess) return e;
  LaunchScope ls(h, MG_K_XR_UPDATE, s);
  if (DIM == 3 && h->t3cg_ok)
    return launch_xr_update_t3<M>(h->t3cg, 1 - parity, h->lv[0], (float*)h->d, (float*)h->r, h->st, h->partials, s);
  return launch_xr_update<float>(h->lv[0], h->p[1 - parity], h->Ap, h->d, h->r, h->st, h->partials, s);
}

static cudaError_t enqueue_iterations(mg_handle_s* h, int count, cudaStream_t s) {
  if (h->cpcg_ok) {
    // a small 2D grid: the whole inner solve in one cluster launch (it
    // returns at once when the inner solve is already done)
    LaunchScope ls(h, MG_K_CLUSTER_PCG, s);
    return launch_cluster_pcg2d(h->cpcg, h->cpcg_smem, (const float*)h->r, (float*)h->d, h->clu_b, h->clu_y, h->st,
                                s);
  }
  return dispatch(h, [&](auto dimc, auto* tp, auto mc) -> cudaError_t {
    constexpr int DIM = decltype(dimc)::value;
    using T = std::remove_pointer_t<decltype(tp)>;
    constexpr bool M = decltype(mc)::value;
    for (int j = 0; j < count; ++j) {
      cudaError_t e = enqueue_iteration<DIM, T, M>(h, j & 1, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  });
}

cudaError_t enqueue_chunk(mg_handle_s* h, cudaStream_t s) { return enqueue_iterations(h, kChunk, s); }

// CG iterations per body of the device-side loop (even: the p double
// buffer alternates within a body); 4 measured best on GB300 (2 and 8
// within 1%).
static int loop_chunk() {
  const char* e = getenv("NPMG_LOOP_CHUNK");
  const int v = e ? atoi(e) : 4;
  return v >= 2 && v <= 16 && v % 2 == 0 ? v : 4;
}

static cudaError_t enqueue_outer(mg_handle_s* h, const float* b, bool update, cudaStream_t s) {
  return dispatch(h, [&](auto dimc, auto* tp, auto mc) -> cudaError_t {
    constexpr int DIM = decltype(dimc)::value;
    using T = std::remove_pointer_t<decltype(tp)>;
    constexpr bool M = decltype(mc)::value;
    const void* xin = h->xff[h->cur64];
    void* xout = h->xff[1 - h->cur64];
    LaunchScope ls(h, MG_K_OUTER, s);
    if (update && f64_iterate(h)) h->launches += 1;  // the float64 update pass
    if (update)
      return launch_outer<DIM, float, M, true>(h->lv[0], h->w0, h->c, b, xin, xout, h->d, h->r, h->st, h->partials, s,
                                               0, f64_iterate(h));
    return launch_outer<DIM, float, M, false>(h->lv[0], h->w0, h->c, b, xin, xout, h->d, h->r, h->st, h->partials, s,
                                              0, f64_iterate(h));
  });
}

static cudaError_t read_state(mg_handle_s* h, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(h->st_host, h->st, sizeof(SolveState), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

// Build (once) the CUDA graph of kChunk CG iterations; its kernels touch
// only handle-owned buffers, so one instantiation serves every solve.
static cudaError_t ensure_graph(mg_handle_s* h, cudaStream_t s) {
  if (h->graph_exec) return cudaSuccess;
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaGraph_t g = nullptr;
  const int64_t before = h->launches;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    h->capturing = 1;
    cudaError_t e2 = enqueue_chunk(h, cs);
    h->capturing = 0;
    e = cudaStreamEndCapture(cs, &g);
    if (e2 != cudaSuccess) e = e2;
  }
  h->chunk_kernels = h->launches - before;
  h->launches = before;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph_exec, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  (void)s;
  return e;
}

// Add a conditional while node at the capture point of cs; returns its body.
static cudaError_t capture_while(cudaStream_t cs, cudaGraphConditionalHandle hd, cudaGraph_t* body) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
  p.conditional.handle = hd;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p);
  if (e != cudaSuccess) return e;
  *body = p.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// The refinement loop after the first residual as one graph, so that a solve
// needs no host round trip per CG chunk or refinement step:
//   while (refinement not done) {            // outer conditional
//     while (inner solve not done) { loop_chunk() CG iterations }
//     refinement step (k_outer, buffers picked by the state's `cur`)
//   }
// The loop kernels bound both loops by a count as well as by the flags.
static cudaError_t build_loop_graph(mg_handle_s* h) {
  const mg_options& o = h->opt;
  const int chunk = loop_chunk();
  const unsigned int cap_in = (unsigned int)((o.max_outer + 2) * (o.max_inner / chunk + 3));
  const unsigned int cap_out = (unsigned int)(o.max_outer + 2);
  cudaGraph_t G = nullptr;
  cudaError_t e = cudaGraphCreate(&G, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle ho, hi;
  cudaStream_t cs = nullptr;
  cudaGraph_t body_outer = nullptr, body_inner = nullptr, tmp = nullptr;
  const int64_t before = h->launches;
  h->capturing = 1;
  e = cudaGraphConditionalHandleCreate(&ho, G, 0, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hi, G, 0, 0);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  // top level: reset the loop counters and set the outer condition
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, G, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e2 = launch_loop_start(ho, h->st, cs);
    if (e2 == cudaSuccess) e2 = capture_while(cs, ho, &body_outer);
    e = cudaStreamEndCapture(cs, &tmp);
    if (e2 != cudaSuccess) e = e2;
  }
  // outer body: inner condition, inner loop, refinement step, outer condition
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(cs, body_outer, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e2 = launch_loop_inner(hi, h->st, cap_in, 0, cs);
    if (e2 == cudaSuccess) e2 = capture_while(cs, hi, &body_inner);
    if (e2 == cudaSuccess)
      e2 = dispatch(h, [&](auto dimc, auto*, auto mc) -> cudaError_t {
        constexpr int DIM = decltype(dimc)::value;
        constexpr bool M = decltype(mc)::value;
        return launch_outer<DIM, float, M, true>(h->lv[0], h->w0, h->c, h->bsave, h->xff[0], h->xff[1], h->d, h->r,
                                                 h->st, h->partials, cs, 1, f64_iterate(h));
      });
    if (e2 == cudaSuccess) e2 = launch_loop_outer(ho, h->st, cap_out, cs);
    e = cudaStreamEndCapture(cs, &tmp);
    if (e2 != cudaSuccess) e = e2;
  }
  // inner body: kChunk CG iterations, then the inner condition
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(cs, body_inner, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const int64_t k0 = h->launches;
    cudaError_t e2 = enqueue_iterations(h, chunk, cs);
    h->loop_kernels = h->launches - k0;
    if (e2 == cudaSuccess) e2 = launch_loop_inner(hi, h->st, cap_in, 1, cs);
    e = cudaStreamEndCapture(cs, &tmp);
    if (e2 != cudaSuccess) e = e2;
  }
  h->capturing = 0;
  h->launches = before;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->loop_exec, G, 0);
  cudaGraphDestroy(G);
  if (cs) cudaStreamDestroy(cs);
  return e;
}

mg_status run_solve(mg_handle_s* h, const float* b, float* x, double tol, cudaStream_t s, mg_stats* out) {
  const mg_options& o = h->opt;
  SolveParams prm;
  prm.tol = tol;
  prm.inner_floor = h->inner_floor;
  prm.max_inner = o.max_inner;
  prm.max_outer = o.max_outer;
  prm.krylov = o.krylov;
  prm.n_fluid = h->n_fluid > 0 ? h->n_fluid : 1;
  NPMG_CUDA(cudaEventRecord(h->ev0, s));
  {
    LaunchScope ls(h, MG_K_INIT_FINISH, s);
    NPMG_CUDA(launch_init(h->lv[0], b, x, h->xff[h->cur64], h->c, prm, h->st, h->partials, s, f64_iterate(h)));
  }
  NPMG_CUDA(enqueue_outer(h, b, false, s));
  const bool graph = h->use_graph && !h->prof;
  if (graph) NPMG_CUDA(ensure_graph(h, s));
  if (graph && h->loop_state == 0) {
    // on failure (for instance a driver without conditional nodes) the host
    // loop below runs the same kernels
    h->loop_state = getenv("NPMG_NO_DEVICE_LOOP") == nullptr && build_loop_graph(h) == cudaSuccess ? 1 : -1;
    cudaGetLastError();
  }
  const bool device_loop = graph && h->loop_state == 1;
  // the device-side loop reads the state itself (it skips its body when
  // the first residual already meets the tolerance): without a guess to
  // check, a solve synchronises with the host once, at the end
  const bool one_sync = device_loop && !h->guess_check;
  if (!one_sync) NPMG_CUDA(read_state(h, s));
  const double guess_relres = one_sync ? 0.0 : h->st_host->relres0;
  const bool rejected = !one_sync && h->guess_check && !h->st_host->outer_done && guess_relres > 1.0;
  if (rejected) {
    // the guess is worse than zero: the plain solve from x = 0 takes over
    {
      LaunchScope ls(h, MG_K_INIT_FINISH, s);
      NPMG_CUDA(launch_init(h->lv[0], b, nullptr, h->xff[h->cur64], h->c, prm, h->st, h->partials, s,
                            f64_iterate(h)));
    }
    NPMG_CUDA(enqueue_outer(h, b, false, s));
    NPMG_CUDA(read_state(h, s));
  }
  bool looped = false;
  if (device_loop && (one_sync || !h->st_host->outer_done)) {
    NPMG_CUDA(cudaMemcpyAsync(h->bsave, b, h->ncell[0] * sizeof(float), cudaMemcpyDeviceToDevice, s));
    NPMG_CUDA(launch_loop_set_cur(h->st, h->cur64, s));
    NPMG_CUDA(cudaGraphLaunch(h->loop_exec, s));
    looped = true;
    if (!one_sync) {
      NPMG_CUDA(read_state(h, s));
      h->cur64 = h->st_host->cur;
    }
  }
  int guard = 0;
  while (!looped && !h->st_host->outer_done && guard < 4 * (o.max_outer + 1)) {
    ++guard;
    int launched = 0;
    for (;;) {
      if (graph) {
        NPMG_CUDA(cudaGraphLaunch(h->graph_exec, s));
        h->launches += h->chunk_kernels;
      } else {
        NPMG_CUDA(enqueue_chunk(h, s));
      }
      launched += kChunk;
      NPMG_CUDA(read_state(h, s));
      if (h->st_host->inner_done || launched > o.max_inner + kChunk) break;
    }
    NPMG_CUDA(enqueue_outer(h, b, true, s));
    h->cur64 = 1 - h->cur64;
    NPMG_CUDA(read_state(h, s));
  }
  {
    // after the one-sync device loop the state's `cur` names the buffer
    // (0: xff[0], 1: xff[1])
    LaunchScope ls(h, MG_K_INIT_FINISH, s);
    const bool dyn = one_sync && looped;
    NPMG_CUDA(launch_finish(h->ncell[0], dyn ? h->xff[0] : h->xff[h->cur64], dyn ? h->xff[1] : nullptr, x, h->st,
                            h->nb1d, s, f64_iterate(h)));
  }
  NPMG_CUDA(cudaEventRecord(h->ev1, s));
  NPMG_CUDA(read_state(h, s));
  if (looped) {
    if (one_sync) h->cur64 = h->st_host->cur;
    // per outer body: the inner condition, the refinement step (two kernels
    // with the float64 iterate: update and residual) and the outer condition
    const int64_t per_outer = f64_iterate(h) ? 4 : 3;
    h->launches += 2 + per_outer * (int64_t)h->st_host->loop_outer +
                   (h->loop_kernels + 1) * (int64_t)h->st_host->loop_bodies;
  }
  const SolveState& st = *h->st_host;
  mg_status status = (mg_status)st.status;
  if (!st.outer_done && status == MG_OK) status = MG_NOT_CONVERGED;
  if (out) {
    memset(out, 0, sizeof(*out));
    out->status = status;
    out->iters = st.iters_total;
    out->outer = st.outer;
    out->levels = h->L;
    out->relres0 = st.relres0;
    out->relres = st.relres;
    out->bnorm = sqrt(st.bnorm2);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    out->ms = ms;
    for (int k = 0; k < kHistory && k < 32; ++k) out->history[k] = st.hist[k];
    out->guess_relres = one_sync ? st.relres0 : guess_relres;
    out->guess_rejected = rejected ? 1 : 0;
  }
  return status;
}

}  // namespace npmg

using namespace npmg;

extern "C" {

const char* mg_last_error(void) { return npmg::last_error(); }

void mg_default_options(mg_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->pre = 2;
  o->post = 2;
  o->omega = 2.0 / 3.0;
  o->coarse_scale = 1.0;
  o->levels = 0;
  o->krylov = 1;
  o->max_inner = 200;
  o->max_outer = 12;
  o->prec = MG_FP32;
  o->inner_floor = 0.0;
  o->cycle = MG_CYCLE_V;
  o->refine = MG_REFINE_FP64;
}

mg_status mg_create(mg_handle* out, int dim, const int64_t shape[3], const double spacing[3], const int bc[6],
                    const uint8_t* d_solid, const mg_options* opt, void* stream) {
  if (!out) {
    set_error("mg_create: out is NULL");
    return MG_ERR_INVALID;
  }
  *out = nullptr;
  if (dim != 2 && dim != 3) {
    set_error("mg_create: dim must be 2 or 3 (got %d)", dim);
    return MG_ERR_INVALID;
  }
  if (!shape || !spacing || !bc) {
    set_error("mg_create: shape, spacing and bc must be non-NULL");
    return MG_ERR_INVALID;
  }
  mg_options o;
  if (opt) o = *opt;
  else mg_default_options(&o);
  if (o.pre < 0 || o.pre > kMaxHalo || o.post < 0 || o.post > kMaxHalo) {
    set_error("mg_create: pre/post sweeps must be in [0, %d]", kMaxHalo);
    return MG_ERR_INVALID;
  }
  if (!(o.omega > 0.0 && o.omega <= 2.0) || !(o.coarse_scale > 0.0) || o.max_inner < 1 || o.max_outer < 1 ||
      o.prec < MG_FP32 || o.prec > MG_MIXED_BF16 || o.levels < 0 || o.levels > kMaxLevels ||
      (o.cycle != MG_CYCLE_V && o.cycle != MG_CYCLE_SAWTOOTH) ||
      (o.refine != MG_REFINE_FP64 && o.refine != MG_REFINE_FF)) {
    set_error("mg_create: invalid options (omega in (0,2], coarse_scale > 0, max_inner/max_outer >= 1, "
              "levels in [0,%d], cycle V or sawtooth, refine FP64 or FF)", kMaxLevels);
    return MG_ERR_INVALID;
  }
  int64_t n0[3] = {shape[0], shape[1], dim == 3 ? shape[2] : 1};
  for (int a = 0; a < dim; ++a) {
    if (n0[a] < 2 || n0[a] > (1 << 20) || !(spacing[a] > 0.0)) {
      set_error("mg_create: shape[%d]=%lld / spacing must be >= 2 and > 0", a, (long long)n0[a]);
      return MG_ERR_INVALID;
    }
  }
  for (int f = 0; f < 2 * dim; ++f) {
    if (bc[f] != MG_BC_DIRICHLET && bc[f] != MG_BC_NEUMANN) {
      set_error("mg_create: bc[%d] must be MG_BC_DIRICHLET or MG_BC_NEUMANN", f);
      return MG_ERR_INVALID;
    }
  }
  if (!d_solid) {
    bool anyD = false;
    for (int f = 0; f < 2 * dim; ++f) anyD = anyD || bc[f] == MG_BC_DIRICHLET;
    if (!anyD) {
      set_error("mg_create: all faces Neumann and no mask: the operator is singular");
      return MG_ERR_INVALID;
    }
  }
  // levels
  int L = o.levels;
  if (L == 0) {
    L = 1;
    for (;;) {
      bool ok = L < kMaxLevels;
      for (int a = 0; a < dim; ++a) {
        const int64_t s = n0[a] >> (L - 1);
        ok = ok && (s % 2 == 0) && (s / 2 >= 4 || false);
      }
      // coarsen while every side stays even and the smallest halved side is >= 4
      if (!ok) break;
      ++L;
    }
  }
  for (int a = 0; a < dim; ++a) {
    if (n0[a] % (1LL << (L - 1)) != 0 || (n0[a] >> (L - 1)) < 2) {
      set_error("mg_create: side %lld not divisible by 2^(levels-1)=%lld with >= 2 cells left", (long long)n0[a],
                (long long)(1LL << (L - 1)));
      return MG_ERR_INVALID;
    }
  }
  int dev = 0;
  NPMG_CUDA(cudaGetDevice(&dev));
  mg_handle_s* h = new mg_handle_s();
  memset(h, 0, sizeof(*h));
  h->dim = dim;
  h->L = L;
  h->device = dev;
  h->opt = o;
  h->masked = d_solid != nullptr;
  h->use_graph = getenv("NPMG_NO_GRAPH") ? 0 : 1;
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev);
  h->esz = o.prec == MG_FP32 ? 4 : 2;
  // the CG vectors are float32 at every precision, so one inner solve can
  // reach the same relative tolerance whatever the cycle's storage
  h->inner_floor = o.inner_floor > 0 ? o.inner_floor : 1e-4;
  for (int f = 0; f < 2 * dim; ++f) {
    h->bc[f] = bc[f];
    if (bc[f] == MG_BC_DIRICHLET) h->bcD |= 1 << f;
  }
  h->c = spacing[0] * spacing[0];
  for (int a = 0; a < 3; ++a) h->w0[a] = a < dim ? h->c / (spacing[a] * spacing[a]) : 0.0;
  for (int k = 0; k < L; ++k) {
    for (int a = 0; a < 3; ++a) {
      h->n[k][a] = a < dim ? (n0[a] >> k) : 1;
      h->h[k][a] = a < dim ? spacing[a] * (double)(1 << k) : 1.0;
    }
    h->ncell[k] = (size_t)h->n[k][0] * h->n[k][1] * h->n[k][2];
  }
  // the single-block coarse kernel takes the small levels (<= 8192 cells)
  // whose padded arrays fit its shared memory
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  LevelDev geo[kMaxLevels];
  for (int k = 0; k < L; ++k) {
    geo[k].nx = (int)h->n[k][0];
    geo[k].ny = (int)h->n[k][1];
    geo[k].nz = (int)h->n[k][2];
  }
  const int kc = coarse_start_level(geo, L, dim, (size_t)optin - 2048);
  h->kc = kc;
  {
    int offtmp[kMaxLevels];
    h->ca_smem = coarse_layout(offtmp, geo + kc, L - kc, dim);
  }
  h->ncoarse = (int)h->ncell[L - 1];
  if (h->ncoarse > 1024) {
    const int nc = h->ncoarse;
    delete h;
    set_error("mg_create: coarsest level has %d cells (> 1024); use more levels", nc);
    return MG_ERR_INVALID;
  }
  // ---- workspace layout
  std::vector<std::pair<void**, size_t>> plan;
  const size_t A = 256;
  for (int k = 0; k < L; ++k) {
    if (h->masked) {
      plan.push_back({(void**)&h->solid[k], h->ncell[k]});
      plan.push_back({(void**)&h->cell[k], h->ncell[k]});
    }
  }
  for (int k = 0; k <= kc; ++k) {
    if (k >= 1) plan.push_back({&h->bk[k], h->ncell[k] * h->esz});
    if (k < kc) plan.push_back({&h->xk[k], h->ncell[k] * h->esz});
    if (k >= 1) plan.push_back({&h->yk[k], h->ncell[k] * h->esz});
  }
  const size_t n0c = h->ncell[0];
  // CG vectors: float32 at every precision (the 16-bit storage is the
  // cycle's level arrays)
  plan.push_back({&h->r, n0c * 4});
  plan.push_back({&h->z, n0c * 4});
  plan.push_back({&h->p[0], n0c * 4});
  plan.push_back({&h->p[1], n0c * 4});
  plan.push_back({&h->Ap, n0c * 4});
  plan.push_back({&h->d, n0c * 4});
  plan.push_back({&h->xff[0], n0c * 8});
  plan.push_back({&h->xff[1], n0c * 8});
  plan.push_back({(void**)&h->bsave, n0c * 4});
  plan.push_back({(void**)&h->inv, (size_t)2 * h->ncoarse * h->ncoarse * 8});
  plan.push_back({(void**)&h->cimage, h->ca_smem});
  if (dim == 2 && o.prec == MG_FP32 && kc >= 1) {
    // the cluster path's coarse cycle starts at level kc or below: its
    // right-hand side, correction and shared-memory image fit level kc's
    plan.push_back({(void**)&h->clu_b, h->ncell[kc] * 4});
    plan.push_back({(void**)&h->clu_y, h->ncell[kc] * 4});
    plan.push_back({(void**)&h->clu_image, h->ca_smem});
    plan.push_back({(void**)&h->cpcg_image, h->ca_smem});
  }
  plan.push_back({(void**)&h->partials, (size_t)kMaxPartials * 8});
  plan.push_back({(void**)&h->st, sizeof(SolveState)});
  size_t total = 0;
  for (auto& p : plan) total = align_up(total, A) + align_up(p.second, A);
  cudaError_t ce = cudaMalloc((void**)&h->pool, total);
  if (ce != cudaSuccess) {
    delete h;
    set_error("mg_create: cudaMalloc(%zu bytes) failed: %s", total, cudaGetErrorString(ce));
    return ce == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA;
  }
  h->pool_bytes = total;
  size_t off = 0;
  for (auto& p : plan) {
    off = align_up(off, A);
    *p.first = h->pool + off;
    off += align_up(p.second, A);
  }
  cudaStream_t s = (cudaStream_t)stream;
  mg_status st = MG_OK;
#define NPMG_TRY(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      set_error("mg_create: %s: %s", #call, cudaGetErrorString(e_));                     \
      st = MG_ERR_CUDA;                                                                  \
      goto fail;                                                                         \
    }                                                                                    \
  } while (0)
  NPMG_TRY(cudaMemsetAsync(h->pool, 0, total, s));
  NPMG_TRY(cudaMallocHost((void**)&h->st_host, sizeof(SolveState)));
  NPMG_TRY(cudaEventCreate(&h->ev0));
  NPMG_TRY(cudaEventCreate(&h->ev1));
  if (h->masked) {
    NPMG_TRY(cudaMemcpyAsync(h->solid[0], d_solid, h->ncell[0], cudaMemcpyDeviceToDevice, s));
    for (int k = 1; k < L; ++k) NPMG_TRY(launch_coarsen_solid(dim, h->n[k - 1], h->solid[k - 1], h->solid[k], s));
    for (int k = 0; k < L; ++k) NPMG_TRY(launch_cell_bytes(dim, h->n[k], h->bcD, h->solid[k], h->cell[k], s));
    std::vector<uint8_t> host(h->ncell[0]);
    NPMG_TRY(cudaMemcpyAsync(host.data(), h->solid[0], h->ncell[0], cudaMemcpyDeviceToHost, s));
    NPMG_TRY(cudaStreamSynchronize(s));
    size_t nf = 0;
    for (uint8_t v : host) nf += v ? 0 : 1;
    h->n_fluid = (int)nf;
  } else {
    h->n_fluid = (int)h->ncell[0];
  }
  for (int k = 0; k < L; ++k) {
    LevelDev& lv = h->lv[k];
    lv.nx = (int)h->n[k][0];
    lv.ny = (int)h->n[k][1];
    lv.nz = (int)h->n[k][2];
    lv.wx = (float)(h->c / (h->h[k][0] * h->h[k][0]));
    lv.wy = (float)(h->c / (h->h[k][1] * h->h[k][1]));
    lv.wz = dim == 3 ? (float)(h->c / (h->h[k][2] * h->h[k][2])) : 0.f;
    lv.bcD = h->bcD;
    lv.cell = h->masked ? h->cell[k] : nullptr;
  }
  {
    const double w[3] = {h->c / (h->h[L - 1][0] * h->h[L - 1][0]), h->c / (h->h[L - 1][1] * h->h[L - 1][1]),
                         dim == 3 ? h->c / (h->h[L - 1][2] * h->h[L - 1][2]) : 0.0};
    NPMG_TRY(launch_coarse_inverse(dim, h->n[L - 1], w, h->bcD, h->masked ? h->cell[L - 1] : nullptr, h->inv, s));
  }
  {
    CoarseArgs& ca = h->ca;
    memset(&ca, 0, sizeof(ca));
    ca.nlev = L - kc;
    ca.dim = dim;
    for (int l = 0; l < ca.nlev; ++l) ca.lv[l] = h->lv[kc + l];
    h->ca_smem = coarse_layout(ca.off, ca.lv, ca.nlev, dim);
    ca.ncoarse = h->ncoarse;
    ca.inv = reinterpret_cast<const float*>(h->inv);
    ca.image = nullptr;
    ca.pre = o.cycle == MG_CYCLE_SAWTOOTH ? -1 : o.pre;  // -1: the sawtooth recursion
    ca.post = o.post;
    ca.omega = (float)o.omega;
    ca.s = (float)o.coarse_scale;
    NPMG_TRY(launch_coarse_image(ca, h->cimage, h->ca_smem, s));
    ca.image = h->cimage;
  }
  h->nb1d = default_blocks_1d(h, h->ncell[0]);
  {
    // every grid that reduces must fit the partial-sum buffer
    const size_t rows = (size_t)((h->n[0][0] + 127) / 128) * ((h->n[0][1] + 7) / 8);
    const size_t tiles = dim == 2 ? (size_t)((h->n[0][0] + 63) / 64) * ((h->n[0][1] + 15) / 16)
                                  : (size_t)((h->n[0][0] + 31) / 32) * ((h->n[0][1] + 7) / 8) * ((h->n[0][2] + 7) / 8);
    if (rows > (size_t)kMaxPartials || tiles > (size_t)kMaxPartials) {
      set_error("mg_create: grid too large for the reduction buffer");
      st = MG_ERR_INVALID;
      goto fail;
    }
  }
  NPMG_TRY(dispatch(h, [&](auto dimc, auto* tp, auto mc) -> cudaError_t {
    constexpr int DIM = decltype(dimc)::value;
    using T = std::remove_pointer_t<decltype(tp)>;
    constexpr bool M = decltype(mc)::value;
    cudaError_t e = prepare_level_kernels<DIM, T, M>(o.pre, o.post);
    if (e == cudaSuccess) e = prepare_coarse<T>(h->ca_smem);
    if (e == cudaSuccess && !std::is_same<T, float>::value) e = prepare_coarse<float>(h->ca_smem);
    if (e == cudaSuccess && DIM == 2) e = prepare_tma_kernels<T, M>();
    if (e == cudaSuccess && DIM == 3) e = prepare_s3_kernels<T, M>();
    if (e == cudaSuccess && DIM == 3) e = prepare_r3_kernels<T, M>();
    if (e == cudaSuccess && DIM == 3) e = prepare_t3_kernels<T, M>();
    // the fused kernels serve both legs of the V cycle and the up leg of
    // the sawtooth (whose up leg is the V cycle's: x, here b / d from the
    // down leg, plus the scaled correction, then the post sweeps); their
    // two-sweep form is fixed, so the sawtooth asks them for post = 2 only
    const int pre_e = o.cycle == MG_CYCLE_SAWTOOTH ? 2 : o.pre;
    for (int k = 0; k < h->kc; ++k) {
      h->s3_ok[k] = getenv("NPMG_NO_STREAM3D") == nullptr && stream3d_eligible(dim, pre_e, o.post, h->lv[k]);
      h->s2_ok[k] = getenv("NPMG_NO_STREAM2D") == nullptr && stream2d_eligible(dim, pre_e, o.post, h->lv[k]) &&
                    h->ncell[k] >= stream2d_min_cells();
      h->r3_ok[k] = getenv("NPMG_NO_ROWS3D") == nullptr && rows3d_eligible(dim, pre_e, o.post, h->lv[k]);
    }
    // tensor maps of the TMA level kernels (2D, two sweeps, rows of 16k cells)
    for (int k = 0; k < h->kc && e == cudaSuccess; ++k) {
      // level 0 of a 16-bit handle reads float32 r: no TMA tile kernels there
      h->tma_ok[k] = getenv("NPMG_NO_TMA") == nullptr && tma_level_eligible(dim, pre_e, o.post, h->lv[k]) &&
                     (k > 0 || std::is_same<T, float>::value) &&
                     tma_encode_level<T>(&h->tmaps[k], h->lv[k], k == 0 ? h->r : h->bk[k], h->xk[k],
                                         h->yk[k + 1]);
    }
    // tensor maps of the TMA-fed 3D kernels (two sweeps); level 0 reads the
    // float32 CG residual r
    for (int k = 0; k < h->kc && e == cudaSuccess; ++k) {
      h->t3_ok[k] = DIM == 3 && tma3d_eligible(dim, pre_e, o.post, h->lv[k]) &&
                    (k == 0 ? tma3d_encode<T, float>(&h->t3maps[0], h->lv[0], h->r, h->xk[0], h->yk[1])
                            : tma3d_encode<T, T>(&h->t3maps[k], h->lv[k], h->bk[k], h->xk[k], h->yk[k + 1]));
    }
    // 2D float32 V(2,2) cycles: the middle levels in one cluster launch
    h->clu_ok = false;
    if (DIM == 2 && std::is_same<T, float>::value && o.cycle == MG_CYCLE_V && o.pre == 2 && o.post == 2 &&
        h->kc >= 2 && h->clu_image && e == cudaSuccess) {
      ClusterArgs ca2;
      size_t ca_bytes = 0;
      if (cluster2d_plan(h->lv, h->L, h->kc, &ca2, &h->clu_k1, &h->clu_kd, &h->clu_smem, &ca_bytes) &&
          ca_bytes <= h->ca_smem) {
        // the coarse cycle of levels kd .. with its own constant image
        CoarseArgs cc = h->ca;
        cc.nlev = ca2.ca.nlev;
        for (int l = 0; l < cc.nlev; ++l) {
          cc.lv[l] = ca2.ca.lv[l];
          cc.off[l] = ca2.ca.off[l];
        }
        cc.image = nullptr;
        cc.finest = 0;
        e = launch_coarse_image(cc, h->clu_image, ca_bytes, s);
        cc.image = h->clu_image;
        ca2.ca = cc;
        ca2.omega = (float)o.omega;
        ca2.s = (float)o.coarse_scale;
        h->clu = ca2;
        h->clu_ok = e == cudaSuccess;
      }
    }
    // 2D float32 V(2,2) with the float64 refinement: a grid whose levels and
    // CG vectors fit a cluster's shared memory solves in one launch
    h->cpcg_ok = false;
    if (DIM == 2 && std::is_same<T, float>::value && o.cycle == MG_CYCLE_V && o.pre == 2 && o.post == 2 &&
        f64_iterate(h) && h->kc >= 1 && h->cpcg_image && e == cudaSuccess) {
      ClusterPcgArgs pa;
      size_t ca_bytes = 0;
      if (cluster_pcg2d_plan(h->lv, h->L, h->kc, &pa, &h->cpcg_kd, &h->cpcg_smem, &ca_bytes) &&
          ca_bytes <= h->ca_smem) {
        CoarseArgs cc = h->ca;
        cc.nlev = pa.a.ca.nlev;
        for (int l = 0; l < cc.nlev; ++l) {
          cc.lv[l] = pa.a.ca.lv[l];
          cc.off[l] = pa.a.ca.off[l];
        }
        cc.image = nullptr;
        cc.finest = 0;
        e = launch_coarse_image(cc, h->cpcg_image, ca_bytes, s);
        cc.image = h->cpcg_image;
        pa.a.ca = cc;
        pa.a.omega = (float)o.omega;
        pa.a.s = (float)o.coarse_scale;
        h->cpcg = pa;
        h->cpcg_ok = e == cudaSuccess;
      }
    }
    // the finest level's CG direction update on the TMA-fed kernel where
    // the level's legs are (NPMG_NO_TMA3D_CG keeps the marching kernel)
    h->t3cg_ok = DIM == 3 && h->kc > 0 && h->t3_ok[0] && getenv("NPMG_NO_TMA3D_CG") == nullptr &&
                 tma3d_encode_cg(&h->t3cg, h->lv[0], (const float*)h->z, (const float*)h->p[0],
                                 (const float*)h->p[1], (const float*)h->d, (const float*)h->r);
    return e;
  }));
  NPMG_TRY(cudaStreamSynchronize(s));
  NPMG_TRY(cudaGetLastError());
#undef NPMG_TRY
  *out = h;
  return MG_OK;
fail:
  mg_destroy(h);
  return st;
}

mg_status mg_solve(mg_handle h, const float* d_b, float* d_x, double rel_tol, void* stream, mg_stats* out) {
  if (!h || !d_b || !d_x) {
    set_error("mg_solve: NULL handle or array");
    return MG_ERR_INVALID;
  }
  if (!(rel_tol > 0.0)) {
    set_error("mg_solve: rel_tol must be > 0");
    return MG_ERR_INVALID;
  }
  if (((uintptr_t)d_b | (uintptr_t)d_x) & 15) {
    set_error("mg_solve: d_b and d_x must be 16-byte aligned");
    return MG_ERR_INVALID;
  }
  return run_solve(h, d_b, d_x, rel_tol, (cudaStream_t)stream, out);
}

mg_status mg_get_solution_f64(mg_handle h, double* d_x64, void* stream) {
  if (!h || !d_x64) {
    set_error("mg_get_solution_f64: NULL argument");
    return MG_ERR_INVALID;
  }
  const cudaError_t e =
      launch_ff_to_f64(h->ncell[0], h->xff[h->cur64], d_x64, h->nb1d, (cudaStream_t)stream, f64_iterate(h));
  if (e != cudaSuccess) {
    set_error("mg_get_solution_f64: %s", cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  return MG_OK;
}

int mg_num_levels(mg_handle h) { return h ? h->L : 0; }

mg_status mg_level_shape(mg_handle h, int k, int64_t shape_out[3]) {
  if (!h || !shape_out || k < 0 || k >= h->L) {
    set_error("mg_level_shape: bad handle or level");
    return MG_ERR_INVALID;
  }
  for (int a = 0; a < 3; ++a) shape_out[a] = h->n[k][a];
  return MG_OK;
}

// Caller arrays of the building blocks: non-NULL and 16-byte aligned (the
// level kernels and the coarse block move them as float4 vectors).
static mg_status check_arrays(const char* who, std::initializer_list<const void*> ptrs) {
  for (const void* p : ptrs) {
    if (!p) {
      set_error("%s: NULL array", who);
      return MG_ERR_INVALID;
    }
    if ((uintptr_t)p & 15) {
      set_error("%s: arrays must be 16-byte aligned", who);
      return MG_ERR_INVALID;
    }
  }
  return MG_OK;
}

static mg_status check_bb(mg_handle h, int k, bool need_coarse, const char* who,
                          std::initializer_list<const void*> ptrs) {
  if (!h || k < 0 || k >= h->L || (need_coarse && k >= h->L - 1)) {
    set_error("%s: bad handle or level %d", who, k);
    return MG_ERR_INVALID;
  }
  return check_arrays(who, ptrs);
}

#define NPMG_BB(EXPR)                                                              \
  do {                                                                             \
    cudaError_t e_;                                                                \
    if (h->dim == 2) e_ = h->masked ? EXPR(2, true) : EXPR(2, false);             \
    else e_ = h->masked ? EXPR(3, true) : EXPR(3, false);                         \
    if (e_ != cudaSuccess) {                                                       \
      set_error("building block launch failed: %s", cudaGetErrorString(e_));      \
      return MG_ERR_CUDA;                                                          \
    }                                                                              \
  } while (0)

mg_status mg_apply_operator(mg_handle h, int k, const float* d_x, float* d_y, void* stream) {
  if (check_bb(h, k, false, "mg_apply_operator", {d_x, d_y}) != MG_OK) return MG_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
#define E(D, M) launch_apply<D, M>(h->lv[k], d_x, d_y, s)
  NPMG_BB(E);
#undef E
  return MG_OK;
}

mg_status mg_smooth(mg_handle h, int k, float* d_x, const float* d_b, int sweeps, void* stream) {
  if (check_bb(h, k, false, "mg_smooth", {d_x, d_b}) != MG_OK) return MG_ERR_INVALID;
  if (sweeps < 0) {
    set_error("mg_smooth: sweeps must be >= 0");
    return MG_ERR_INVALID;
  }
  if (sweeps == 0) return MG_OK;
  if (h->opt.prec != MG_FP32) {
    set_error("mg_smooth: building blocks need a float32 handle");
    return MG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // ping-pong through the handle's level-0 scratch vector z (>= any level)
  float* tmp = (float*)h->z;
  for (int j = 0; j < sweeps; ++j) {
    float* src = (j % 2 == 0) ? d_x : tmp;
    float* dst = (j % 2 == 0) ? tmp : d_x;
#define E(D, M) launch_smooth_once<D, M>(h->lv[k], src, dst, d_b, (float)h->opt.omega, s)
    NPMG_BB(E);
#undef E
  }
  if (sweeps % 2 == 1) NPMG_CUDA(cudaMemcpyAsync(d_x, tmp, h->ncell[k] * 4, cudaMemcpyDeviceToDevice, s));
  return MG_OK;
}

mg_status mg_residual_restrict(mg_handle h, int k, const float* d_x, const float* d_b, float* d_bc, void* stream) {
  if (check_bb(h, k, true, "mg_residual_restrict", {d_x, d_b, d_bc}) != MG_OK) return MG_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
#define E(D, M) launch_restrict_residual<D, M>(h->lv[k], d_x, d_b, d_bc, s)
  NPMG_BB(E);
#undef E
  return MG_OK;
}

mg_status mg_prolong_correct(mg_handle h, int k, const float* d_e, float* d_x, void* stream) {
  if (check_bb(h, k, true, "mg_prolong_correct", {d_e, d_x}) != MG_OK) return MG_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
#define E(D, M) launch_prolong_correct<D, M>(h->lv[k], d_e, d_x, (float)h->opt.coarse_scale, s)
  NPMG_BB(E);
#undef E
  return MG_OK;
}

mg_status mg_precondition(mg_handle h, const float* d_r, float* d_z, void* stream) {
  if (!h) {
    set_error("mg_precondition: NULL handle");
    return MG_ERR_INVALID;
  }
  if (check_arrays("mg_precondition", {d_r, d_z}) != MG_OK) return MG_ERR_INVALID;
  if (h->opt.prec != MG_FP32) {
    set_error("mg_precondition: building blocks need a float32 handle");
    return MG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (h->dim == 2)
    e = h->masked ? enqueue_vcycle<2, float, true>(h, d_r, d_z, nullptr, s)
                  : enqueue_vcycle<2, float, false>(h, d_r, d_z, nullptr, s);
  else
    e = h->masked ? enqueue_vcycle<3, float, true>(h, d_r, d_z, nullptr, s)
                  : enqueue_vcycle<3, float, false>(h, d_r, d_z, nullptr, s);
  if (e != cudaSuccess) {
    set_error("mg_precondition: %s", cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  return MG_OK;
}

mg_status mg_profile_enable(mg_handle h, int on) {
  if (!h) {
    set_error("mg_profile_enable: NULL handle");
    return MG_ERR_INVALID;
  }
  if (on && !h->pev) {
    h->pev = (cudaEvent_t*)calloc(2 * kProfEvents, sizeof(cudaEvent_t));
    if (!h->pev) return MG_ERR_OOM;
    for (int i = 0; i < 2 * kProfEvents; ++i) NPMG_CUDA(cudaEventCreate(&h->pev[i]));
  }
  if (!on) NPMG_CUDA(prof_flush(h));
  h->prof = on ? 1 : 0;
  return MG_OK;
}

mg_status mg_profile_read(mg_handle h, double* h_ms, int64_t* h_launches, int reset) {
  if (!h || !h_ms || !h_launches) {
    set_error("mg_profile_read: NULL argument");
    return MG_ERR_INVALID;
  }
  NPMG_CUDA(prof_flush(h));
  for (int k = 0; k < MG_K_COUNT; ++k) {
    h_ms[k] = h->prof_ms[k];
    h_launches[k] = h->prof_n[k];
    if (reset) {
      h->prof_ms[k] = 0.0;
      h->prof_n[k] = 0;
    }
  }
  return MG_OK;
}

int64_t mg_kernel_launches(mg_handle h) { return h ? h->launches : 0; }

mg_status mg_destroy(mg_handle h) {
  if (!h) return MG_OK;
  if (h->pev) {
    for (int i = 0; i < 2 * kProfEvents; ++i)
      if (h->pev[i]) cudaEventDestroy(h->pev[i]);
    free(h->pev);
  }
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->loop_exec) cudaGraphExecDestroy(h->loop_exec);
  if (h->pool) cudaFree(h->pool);
  if (h->st_host) cudaFreeHost(h->st_host);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  delete h;
  return MG_OK;
}

}  // extern "C"
