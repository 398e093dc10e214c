// Host side of the learned initial-guess network: the handle (FP32 master
// weights, Adam moments, packed BF16 operands), activation workspaces per
// shape, the forward and backward passes as kernel sequences, the crop
// dataset and the training loop, and the C ABI (gn_* in npmg.h).
#include <math.h>
#include <string.h>

#include <vector>

#include "gn.h"
#include "mg_handle.h"

using namespace npmg;
using namespace npmg::gn;

namespace {

constexpr int kCin[kLayers] = {2, 16, 16, 16, 16, 16, 16, 16, 16};
constexpr int kCout[kLayers] = {16, 16, 16, 16, 16, 16, 16, 16, 1};
constexpr int kRmsBlocks = 64;
constexpr int kWgMaxBlocks = 1024;
constexpr int kLossSlots = 4096;  // device step losses kept by gn_train

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Activation workspace of one shape: BF16 NDHWC16 tensors per level plus
// the gradients when `train`.
struct Work {
  Dims d[3];  // levels 0, 1, 2 (n samples)
  bool train = false;
  char* pool = nullptr;
  void *x0, *e1a, *e1, *s1, *d1;
  void *p1, *e2a, *e2, *s2, *d2;
  void *p2, *e3a, *e3;
  void *gy, *ga8, *gs1, *ga2, *ga1;
  void *ga7, *gs2, *ga4, *ga3, *gp1;
  void *ga6, *ga5, *gp2;
  float *y, *r;
  float *rms, *inv, *rpart;
  double* lpart;
  bool same(int n, const int64_t c[3], bool tr) const {
    return pool && d[0].n == n && d[0].nx == c[0] && d[0].ny == c[1] && d[0].nz == c[2] && (train || !tr);
  }
  void release() {
    if (pool) cudaFree(pool);
    pool = nullptr;
  }
  cudaError_t alloc(int n, const int64_t c[3], bool tr) {
    release();
    train = tr;
    for (int l = 0; l < 3; ++l) d[l] = Dims{n, (int)(c[0] >> l), (int)(c[1] >> l), (int)(c[2] >> l)};
    const size_t t[3] = {round256(d[0].vox() * n * 32), round256(d[1].vox() * n * 32), round256(d[2].vox() * n * 32)};
    const int n0 = tr ? 10 : 5, n1 = tr ? 10 : 5, n2 = tr ? 6 : 3;
    const size_t total = n0 * t[0] + n1 * t[1] + n2 * t[2] + 2 * round256(d[0].vox() * n * 4) + 3 * round256(2 * n * 4) +
                         round256((size_t)2 * n * kRmsBlocks * 4) + round256(8 * 1024 * 8);
    cudaError_t e = cudaMalloc((void**)&pool, total);
    if (e != cudaSuccess) {
      pool = nullptr;
      return e;
    }
    char* q = pool;
    auto take = [&](size_t b) {
      char* r = q;
      q += round256(b);
      return (void*)r;
    };
    x0 = take(t[0]), e1a = take(t[0]), e1 = take(t[0]), s1 = take(t[0]), d1 = take(t[0]);
    p1 = take(t[1]), e2a = take(t[1]), e2 = take(t[1]), s2 = take(t[1]), d2 = take(t[1]);
    p2 = take(t[2]), e3a = take(t[2]), e3 = take(t[2]);
    if (tr) {
      gy = take(t[0]), ga8 = take(t[0]), gs1 = take(t[0]), ga2 = take(t[0]), ga1 = take(t[0]);
      ga7 = take(t[1]), gs2 = take(t[1]), ga4 = take(t[1]), ga3 = take(t[1]), gp1 = take(t[1]);
      ga6 = take(t[2]), ga5 = take(t[2]), gp2 = take(t[2]);
    }
    y = (float*)take(d[0].vox() * n * 4);
    r = (float*)take(d[0].vox() * n * 4);
    rms = (float*)take(2 * n * 4);  // b then p
    inv = (float*)take(2 * n * 4);
    take(2 * n * 4);
    rpart = (float*)take((size_t)2 * n * kRmsBlocks * 4);
    lpart = (double*)take(8 * 1024 * 8);
    return cudaSuccess;
  }
};

}  // namespace

struct gn_handle_s {
  int device = 0;
  float *w = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;  // [9][6912]
  void *wf = nullptr, *wd = nullptr;                                // packed [9][13824 B]
  int* err = nullptr;
  float* wg_part = nullptr;  // wgrad partials [kWgMaxBlocks][6912]
  double* loss_dev = nullptr;
  int* idx_dev = nullptr;
  size_t idx_cap = 0;
  char* pool = nullptr;
  int adam_t = 0;
  Work infer, train;
  float* ds = nullptr;  // crops: [b, p^n, dp, fluid][z][y][x] each
  int ds_cap = 0, ds_n = 0;
  int64_t crop[3] = {0, 0, 0};
  double ds_h = 1.0;    // grid spacing of the dataset's pressure operator
};

namespace {

const void* pf(gn_handle_s* g, int k) { return (const char*)g->wf + (size_t)k * kPackBytes; }
const void* pd(gn_handle_s* g, int k) { return (const char*)g->wd + (size_t)k * kPackBytes; }

bool cells_ok(const int64_t c[3]) {
  for (int a = 0; a < 3; ++a)
    if (c[a] < 4 || (c[a] % 4) != 0 || c[a] > (1 << 20)) return false;
  return true;
}

// host layout (unpadded layers back to back) <-> padded [9][27][16][16]
void unpadded_to_padded(const float* src, std::vector<float>& dst) {
  dst.assign((size_t)kLayers * kWElems, 0.f);
  size_t o = 0;
  for (int k = 0; k < kLayers; ++k)
    for (int t = 0; t < kTaps; ++t)
      for (int ci = 0; ci < kCin[k]; ++ci)
        for (int co = 0; co < kCout[k]; ++co) dst[(size_t)k * kWElems + (t * kC + ci) * kC + co] = src[o++];
}
void padded_to_unpadded(const std::vector<float>& src, float* dst) {
  size_t o = 0;
  for (int k = 0; k < kLayers; ++k)
    for (int t = 0; t < kTaps; ++t)
      for (int ci = 0; ci < kCin[k]; ++ci)
        for (int co = 0; co < kCout[k]; ++co) dst[o++] = src[(size_t)k * kWElems + (t * kC + ci) * kC + co];
}

#define GN_TRY(x)                                                          \
  do {                                                                     \
    cudaError_t e_ = (x);                                                  \
    if (e_ != cudaSuccess) {                                               \
      set_error("%s: %s (%s)", __func__, cudaGetErrorString(e_), #x); \
      return MG_ERR_CUDA;                                                  \
    }                                                                      \
  } while (0)

mg_status ensure_work(Work& W, int n, const int64_t c[3], bool train) {
  if (W.same(n, c, train)) return MG_OK;
  cudaError_t e = W.alloc(n, c, train);
  if (e != cudaSuccess) {
    set_error("gn: workspace allocation failed: %s", cudaGetErrorString(e));
    return MG_ERR_OOM;
  }
  return MG_OK;
}

// Forward pass; output channel 0 into `out` scaled by `scale` (per sample,
// or nullptr for 1).  Inputs are (b / rms(b), p / rms(p)), the rms taken
// per sample or pooled over the samples.
mg_status forward(gn_handle_s* g, Work& W, const Fields& f, float* out, const float* scale, bool pooled,
                  cudaStream_t s) {
  const Dims* d = W.d;
  GN_TRY(launch_rms(f, d[0], pooled, W.rpart, W.rms, W.inv, s));
  GN_TRY(launch_pack_input(f, W.inv, W.x0, d[0], s));
  GN_TRY(launch_conv(W.x0, pf(g, 0), W.e1a, kEpiRelu, nullptr, nullptr, d[0], g->err, s));
  GN_TRY(launch_conv(W.e1a, pf(g, 1), W.e1, kEpiRelu, nullptr, nullptr, d[0], g->err, s));
  GN_TRY(launch_pool(W.e1, W.p1, d[0], s));
  GN_TRY(launch_conv(W.p1, pf(g, 2), W.e2a, kEpiRelu, nullptr, nullptr, d[1], g->err, s));
  GN_TRY(launch_conv(W.e2a, pf(g, 3), W.e2, kEpiRelu, nullptr, nullptr, d[1], g->err, s));
  GN_TRY(launch_pool(W.e2, W.p2, d[1], s));
  GN_TRY(launch_conv(W.p2, pf(g, 4), W.e3a, kEpiRelu, nullptr, nullptr, d[2], g->err, s));
  GN_TRY(launch_conv(W.e3a, pf(g, 5), W.e3, kEpiRelu, nullptr, nullptr, d[2], g->err, s));
  GN_TRY(launch_up_add(W.e3, W.e2, W.s2, d[1], s));
  GN_TRY(launch_conv(W.s2, pf(g, 6), W.d2, kEpiRelu, nullptr, nullptr, d[1], g->err, s));
  GN_TRY(launch_up_add(W.d2, W.e1, W.s1, d[0], s));
  GN_TRY(launch_conv(W.s1, pf(g, 7), W.d1, kEpiRelu, nullptr, nullptr, d[0], g->err, s));
  GN_TRY(launch_conv(W.d1, pf(g, 8), out, kEpiOut0, nullptr, scale, d[0], g->err, s));
  return MG_OK;
}

mg_status wgrad_into(gn_handle_s* g, const void* x, const void* gr, int layer, const Dims& d, float scale,
                     cudaStream_t s) {
  int nb = 0;
  GN_TRY(launch_wgrad(x, gr, g->wg_part, kWgMaxBlocks, &nb, d, g->err, s));
  GN_TRY(launch_wgrad_reduce(g->wg_part, nb, g->grad + (size_t)layer * kWElems, scale, false, s));
  return MG_OK;
}

#define GN_STEP(x)                \
  do {                            \
    mg_status st_ = (x);          \
    if (st_ != MG_OK) return st_; \
  } while (0)

// Loss of the last forward (W.y, normalised units) into *loss (device) and
// the gradient of every layer into g->grad.  mode GN_LOSS_L2: against the
// target f.t; GN_LOSS_RESIDUAL: the residual of the guess on the crop's
// interior fluid cells (operator spacing h).
mg_status backward(gn_handle_s* g, Work& W, const Fields& f, int mode, double h, double* loss, cudaStream_t s) {
  const Dims* d = W.d;
  const float sc = (float)(1.0 / ((double)d[0].vox() * d[0].n));
  if (mode == GN_LOSS_RESIDUAL)
    GN_TRY(launch_residual_loss_grad(W.y, f, W.inv, (float)(1.0 / (h * h)), W.r, W.gy, W.lpart, loss, d[0], s));
  else
    GN_TRY(launch_loss_grad(W.y, f, W.inv, W.gy, W.lpart, loss, d[0], s));
  GN_STEP(wgrad_into(g, W.d1, W.gy, 8, d[0], sc, s));
  GN_TRY(launch_conv(W.gy, pd(g, 8), W.ga8, kEpiMask, W.d1, nullptr, d[0], g->err, s));
  GN_STEP(wgrad_into(g, W.s1, W.ga8, 7, d[0], sc, s));
  GN_TRY(launch_conv(W.ga8, pd(g, 7), W.gs1, kEpiLin, nullptr, nullptr, d[0], g->err, s));
  GN_TRY(launch_upbwd_mask(W.gs1, W.d2, W.ga7, d[0], s));
  GN_STEP(wgrad_into(g, W.s2, W.ga7, 6, d[1], sc, s));
  GN_TRY(launch_conv(W.ga7, pd(g, 6), W.gs2, kEpiLin, nullptr, nullptr, d[1], g->err, s));
  GN_TRY(launch_upbwd_mask(W.gs2, W.e3, W.ga6, d[1], s));
  GN_STEP(wgrad_into(g, W.e3a, W.ga6, 5, d[2], sc, s));
  GN_TRY(launch_conv(W.ga6, pd(g, 5), W.ga5, kEpiMask, W.e3a, nullptr, d[2], g->err, s));
  GN_STEP(wgrad_into(g, W.p2, W.ga5, 4, d[2], sc, s));
  GN_TRY(launch_conv(W.ga5, pd(g, 4), W.gp2, kEpiLin, nullptr, nullptr, d[2], g->err, s));
  GN_TRY(launch_poolbwd_add_mask(W.gs2, W.gp2, W.e2, W.ga4, d[1], s));
  GN_STEP(wgrad_into(g, W.e2a, W.ga4, 3, d[1], sc, s));
  GN_TRY(launch_conv(W.ga4, pd(g, 3), W.ga3, kEpiMask, W.e2a, nullptr, d[1], g->err, s));
  GN_STEP(wgrad_into(g, W.p1, W.ga3, 2, d[1], sc, s));
  GN_TRY(launch_conv(W.ga3, pd(g, 2), W.gp1, kEpiLin, nullptr, nullptr, d[1], g->err, s));
  GN_TRY(launch_poolbwd_add_mask(W.gs1, W.gp1, W.e1, W.ga2, d[0], s));
  GN_STEP(wgrad_into(g, W.e1a, W.ga2, 1, d[0], sc, s));
  GN_TRY(launch_conv(W.ga2, pd(g, 1), W.ga1, kEpiMask, W.e1a, nullptr, d[0], g->err, s));
  GN_STEP(wgrad_into(g, W.x0, W.ga1, 0, d[0], sc, s));
  return MG_OK;
}

mg_status adam(gn_handle_s* g, double lr, cudaStream_t s) {
  g->adam_t += 1;
  AdamArgs a;
  a.lr = (float)lr;
  a.b1 = 0.9f;
  a.b2 = 0.999f;
  a.omb1 = (float)(1.0 - 0.9);
  a.omb2 = (float)(1.0 - 0.999);
  a.eps = 1e-8f;
  a.c1 = (float)(1.0 / (1.0 - pow(0.9, g->adam_t)));
  a.c2 = (float)(1.0 / (1.0 - pow(0.999, g->adam_t)));
  GN_TRY(launch_adam_pack(g->w, g->m, g->v, g->grad, true, a, g->wf, g->wd, s));
  return MG_OK;
}

// Reads and clears the device error flag (synchronises the stream).
mg_status check_err(gn_handle_s* g, cudaStream_t s, const char* who) {
  int e = 0;
  GN_TRY(cudaMemcpyAsync(&e, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  GN_TRY(cudaStreamSynchronize(s));
  if (e) {
    GN_TRY(cudaMemsetAsync(g->err, 0, sizeof(int), s));
    set_error("%s: a tile load or MMA did not complete in its bounded wait (code %d)", who, e);
    return MG_TIMEOUT;
  }
  return MG_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// splitmix64
uint64_t mix64(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

mg_status gn_create(gn_handle* out, const float* h_weights, void* stream) {
  if (!out || !h_weights) {
    set_error("gn_create: NULL argument");
    return MG_ERR_INVALID;
  }
  *out = nullptr;
  gn_handle_s* g = new gn_handle_s();
  cudaGetDevice(&g->device);
  const size_t wbytes = round256((size_t)kLayers * kWElems * 4);
  const size_t total = 4 * wbytes + 2 * round256((size_t)kLayers * kPackBytes) + 256 +
                       round256((size_t)kWgMaxBlocks * kWElems * 4) + round256(8 * kLossSlots);
  if (cudaMalloc((void**)&g->pool, total) != cudaSuccess) {
    delete g;
    set_error("gn_create: cudaMalloc failed");
    return MG_ERR_OOM;
  }
  char* q = g->pool;
  auto take = [&](size_t b) {
    char* r = q;
    q += round256(b);
    return (void*)r;
  };
  g->w = (float*)take(wbytes);
  g->m = (float*)take(wbytes);
  g->v = (float*)take(wbytes);
  g->grad = (float*)take(wbytes);
  g->wf = take((size_t)kLayers * kPackBytes);
  g->wd = take((size_t)kLayers * kPackBytes);
  g->err = (int*)take(256);
  g->wg_part = (float*)take((size_t)kWgMaxBlocks * kWElems * 4);
  g->loss_dev = (double*)take(8 * kLossSlots);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(g->pool, 0, total, s) != cudaSuccess) {
    gn_destroy(g);
    set_error("gn_create: memset failed");
    return MG_ERR_CUDA;
  }
  *out = g;
  const mg_status st = gn_set_weights(g, h_weights);
  if (st != MG_OK) {
    gn_destroy(g);
    *out = nullptr;
    return st;
  }
  return cudaStreamSynchronize(s) == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

mg_status gn_set_weights(gn_handle g, const float* h_weights) {
  if (!g || !h_weights) {
    set_error("gn_set_weights: NULL argument");
    return MG_ERR_INVALID;
  }
  std::vector<float> pad;
  unpadded_to_padded(h_weights, pad);
  GN_TRY(cudaMemcpy(g->w, pad.data(), pad.size() * 4, cudaMemcpyHostToDevice));
  GN_TRY(cudaMemset(g->m, 0, pad.size() * 4));
  GN_TRY(cudaMemset(g->v, 0, pad.size() * 4));
  g->adam_t = 0;
  AdamArgs a = {};
  GN_TRY(launch_adam_pack(g->w, g->m, g->v, g->grad, false, a, g->wf, g->wd, 0));
  GN_TRY(cudaDeviceSynchronize());
  return MG_OK;
}

mg_status gn_get_weights(gn_handle g, float* h_weights) {
  if (!g || !h_weights) {
    set_error("gn_get_weights: NULL argument");
    return MG_ERR_INVALID;
  }
  std::vector<float> pad((size_t)kLayers * kWElems);
  GN_TRY(cudaDeviceSynchronize());
  GN_TRY(cudaMemcpy(pad.data(), g->w, pad.size() * 4, cudaMemcpyDeviceToHost));
  padded_to_unpadded(pad, h_weights);
  return MG_OK;
}

mg_status gn_forward(gn_handle g, int n, const int64_t cells[3], const float* d_b, const float* d_p, float* d_out,
                     void* stream) {
  if (!g || !cells || !d_b || !d_p || !d_out || n <= 0 || !cells_ok(cells)) {
    set_error("gn_forward: invalid argument (cells must be multiples of 4)");
    return MG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  GN_STEP(ensure_work(g->infer, n, cells, false));
  const size_t vox = (size_t)(cells[0] * cells[1] * cells[2]);
  Fields f = {d_b, d_p, nullptr, nullptr, vox, nullptr};
  return forward(g, g->infer, f, d_out, g->infer.rms, false, s);
}

mg_status gn_gradients(gn_handle g, int n, const int64_t cells[3], const float* d_b, const float* d_p,
                       const float* d_t, const float* d_fluid, int loss_mode, double h, double* h_loss,
                       float* h_grad, void* stream) {
  if (!g || !cells || !d_b || !d_p || n <= 0 || !cells_ok(cells) ||
      (loss_mode != GN_LOSS_L2 && loss_mode != GN_LOSS_RESIDUAL) || (loss_mode == GN_LOSS_L2 && !d_t) ||
      !(h > 0)) {
    set_error("gn_gradients: invalid argument (cells must be multiples of 4)");
    return MG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  GN_STEP(ensure_work(g->train, n, cells, true));
  const size_t vox = (size_t)(cells[0] * cells[1] * cells[2]);
  Fields f = {d_b, d_p, d_t, d_fluid, vox, nullptr};
  GN_STEP(forward(g, g->train, f, g->train.y, nullptr, false, s));
  GN_STEP(backward(g, g->train, f, loss_mode, h, g->loss_dev, s));
  GN_STEP(check_err(g, s, "gn_gradients"));
  if (h_loss) GN_TRY(cudaMemcpy(h_loss, g->loss_dev, sizeof(double), cudaMemcpyDeviceToHost));
  if (h_grad) {
    std::vector<float> pad((size_t)kLayers * kWElems);
    GN_TRY(cudaMemcpy(pad.data(), g->grad, pad.size() * 4, cudaMemcpyDeviceToHost));
    padded_to_unpadded(pad, h_grad);
  }
  return MG_OK;
}

mg_status gn_adam_step(gn_handle g, const float* h_grad, double lr, void* stream) {
  if (!g || !(lr > 0)) {
    set_error("gn_adam_step: invalid argument");
    return MG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (h_grad) {
    std::vector<float> pad;
    unpadded_to_padded(h_grad, pad);
    GN_TRY(cudaStreamSynchronize(s));
    GN_TRY(cudaMemcpy(g->grad, pad.data(), pad.size() * 4, cudaMemcpyHostToDevice));
  }
  GN_STEP(adam(g, lr, s));
  GN_TRY(cudaStreamSynchronize(s));
  return MG_OK;
}

mg_status gn_dataset_reserve(gn_handle g, const int64_t crop[3], int capacity, double h) {
  if (!g || !crop || capacity <= 0 || !cells_ok(crop) || !(h > 0)) {
    set_error("gn_dataset_reserve: invalid argument (crop sides must be multiples of 4)");
    return MG_ERR_INVALID;
  }
  if (g->ds) cudaFree(g->ds);
  g->ds = nullptr;
  g->ds_cap = g->ds_n = 0;
  const size_t vox = (size_t)(crop[0] * crop[1] * crop[2]);
  if (cudaMalloc((void**)&g->ds, (size_t)capacity * 4 * vox * 4) != cudaSuccess) {
    g->ds = nullptr;
    set_error("gn_dataset_reserve: cudaMalloc of %d crops failed", capacity);
    return MG_ERR_OOM;
  }
  g->ds_cap = capacity;
  g->ds_h = h;
  for (int a = 0; a < 3; ++a) g->crop[a] = crop[a];
  return MG_OK;
}

int gn_dataset_size(gn_handle g) { return g ? g->ds_n : 0; }

mg_status gn_dataset_add(gn_handle g, const int64_t cells[3], const float* d_b, const float* d_p_next,
                         const float* d_dp, const uint8_t* d_solid, void* stream) {
  if (!g || !cells || !d_b || !d_p_next || !d_dp || !g->ds) {
    set_error("gn_dataset_add: invalid argument or no dataset reserved");
    return MG_ERR_INVALID;
  }
  for (int a = 0; a < 3; ++a)
    if (cells[a] < g->crop[a]) {
      set_error("gn_dataset_add: field smaller than the crop");
      return MG_ERR_INVALID;
    }
  const size_t vox = (size_t)(g->crop[0] * g->crop[1] * g->crop[2]);
  const int64_t nc[3] = {cells[0] / g->crop[0], cells[1] / g->crop[1], cells[2] / g->crop[2]};
  for (int64_t k = 0; k < nc[2]; ++k)
    for (int64_t j = 0; j < nc[1]; ++j)
      for (int64_t i = 0; i < nc[0]; ++i) {
        if (g->ds_n >= g->ds_cap) return MG_OK;
        const int64_t org[3] = {i * g->crop[0], j * g->crop[1], k * g->crop[2]};
        GN_TRY(launch_crop(d_b, d_p_next, d_dp, d_solid, cells, g->crop, org, g->ds + (size_t)g->ds_n * 4 * vox,
                           (cudaStream_t)stream));
        g->ds_n += 1;
      }
  return MG_OK;
}

mg_status gn_train(gn_handle g, int steps, int batch, uint64_t seed, double lr, int loss_mode, double* h_losses,
                    void* stream) {
  if (!g || steps <= 0 || batch <= 0 || !(lr > 0) || g->ds_n <= 0 ||
      (loss_mode != GN_LOSS_L2 && loss_mode != GN_LOSS_RESIDUAL)) {
    set_error("gn_train: invalid argument or empty dataset");
    return MG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  GN_STEP(ensure_work(g->train, batch, g->crop, true));
  const size_t need = (size_t)steps * batch;
  if (need > g->idx_cap) {
    if (g->idx_dev) cudaFree(g->idx_dev);
    g->idx_dev = nullptr;
    g->idx_cap = 0;
    GN_TRY(cudaMalloc((void**)&g->idx_dev, need * sizeof(int)));
    g->idx_cap = need;
  }
  std::vector<int> idx(need);
  uint64_t st = seed;
  for (size_t i = 0; i < need; ++i) idx[i] = (int)(mix64(st) % (uint64_t)g->ds_n);
  GN_TRY(cudaMemcpyAsync(g->idx_dev, idx.data(), need * sizeof(int), cudaMemcpyHostToDevice, s));
  GN_TRY(cudaStreamSynchronize(s));
  const size_t vox = (size_t)(g->crop[0] * g->crop[1] * g->crop[2]);
  for (int k = 0; k < steps; ++k) {
    Fields f = {g->ds, g->ds + vox, g->ds + 2 * vox, g->ds + 3 * vox, 4 * vox, g->idx_dev + (size_t)k * batch};
    GN_STEP(forward(g, g->train, f, g->train.y, nullptr, true, s));
    GN_STEP(backward(g, g->train, f, loss_mode, g->ds_h, g->loss_dev + (k % kLossSlots), s));
    // cosine decay from lr to lr / 20 over the call
    const double lr_k = lr * (0.05 + 0.95 * 0.5 * (1.0 + cos(M_PI * (double)k / (double)steps)));
    GN_STEP(adam(g, lr_k, s));
    if (h_losses && (k % kLossSlots == kLossSlots - 1 || k == steps - 1)) {
      // the device keeps kLossSlots step losses; drain them to the host
      const int first = k - k % kLossSlots;
      GN_TRY(cudaMemcpyAsync(h_losses + first, g->loss_dev, (size_t)(k - first + 1) * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
      GN_TRY(cudaStreamSynchronize(s));
    }
  }
  GN_STEP(check_err(g, s, "gn_train"));
  return MG_OK;
}

mg_status gn_conv3d(const void* d_x, const float* d_w, void* d_y, int n, const int64_t cells[3], int mode,
                    void* d_scratch, void* stream) {
  if (!d_x || !d_w || !d_y || !d_scratch || !cells || n <= 0 || mode < 0 || mode > 3 ||
      !aligned16(d_x) || !aligned16(d_y) || ((uintptr_t)d_scratch & 255)) {
    set_error("gn_conv3d: invalid argument");
    return MG_ERR_INVALID;
  }
  for (int a = 0; a < 3; ++a)
    if (cells[a] < 1 || cells[a] > (1 << 20)) {
      set_error("gn_conv3d: bad shape");
      return MG_ERR_INVALID;
    }
  cudaStream_t s = (cudaStream_t)stream;
  char* sc = (char*)d_scratch;
  void* wf = sc;
  void* wd = sc + kPackBytes;
  int* err = (int*)(sc + 2 * kPackBytes);
  GN_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  GN_TRY(launch_pack_layer(d_w, wf, wd, s));
  const Dims d{n, (int)cells[0], (int)cells[1], (int)cells[2]};
  const int epi = mode == GN_CONV_RELU ? kEpiRelu : mode == GN_CONV_LIN ? kEpiLin : kEpiF32;
  GN_TRY(launch_conv(d_x, mode == GN_CONV_DGRAD ? wd : wf, d_y, epi, nullptr, nullptr, d, err, s));
  int e = 0;
  GN_TRY(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  GN_TRY(cudaStreamSynchronize(s));
  if (e) {
    set_error("gn_conv3d: bounded wait expired (code %d)", e);
    return MG_TIMEOUT;
  }
  return MG_OK;
}

mg_status gn_conv3d_wgrad(const void* d_x, const void* d_g, float* d_dw, int n, const int64_t cells[3],
                          void* d_scratch, size_t scratch_bytes, void* stream) {
  if (!d_x || !d_g || !d_dw || !d_scratch || !cells || n <= 0 || !aligned16(d_x) || !aligned16(d_g) ||
      ((uintptr_t)d_scratch & 255) || scratch_bytes < (size_t)GN_WGRAD_SCRATCH_MIN) {
    set_error("gn_conv3d_wgrad: invalid argument");
    return MG_ERR_INVALID;
  }
  for (int a = 0; a < 3; ++a)
    if (cells[a] < 1 || cells[a] > (1 << 20)) {
      set_error("gn_conv3d_wgrad: bad shape");
      return MG_ERR_INVALID;
    }
  cudaStream_t s = (cudaStream_t)stream;
  int* err = (int*)d_scratch;
  float* part = (float*)((char*)d_scratch + 256);
  const int maxb = (int)((scratch_bytes - 256) / ((size_t)kWElems * 4));
  GN_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  const Dims d{n, (int)cells[0], (int)cells[1], (int)cells[2]};
  int nb = 0;
  GN_TRY(launch_wgrad(d_x, d_g, part, maxb, &nb, d, err, s));
  GN_TRY(launch_wgrad_reduce(part, nb, d_dw, 1.f, false, s));
  int e = 0;
  GN_TRY(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  GN_TRY(cudaStreamSynchronize(s));
  if (e) {
    set_error("gn_conv3d_wgrad: bounded wait expired (code %d)", e);
    return MG_TIMEOUT;
  }
  return MG_OK;
}

int64_t gn_kernel_launches(void) { return g_launches.load(); }

mg_status gn_destroy(gn_handle g) {
  if (!g) return MG_OK;
  cudaDeviceSynchronize();
  g->infer.release();
  g->train.release();
  if (g->ds) cudaFree(g->ds);
  if (g->idx_dev) cudaFree(g->idx_dev);
  if (g->pool) cudaFree(g->pool);
  delete g;
  return MG_OK;
}

}  // extern "C"
