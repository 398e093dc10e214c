// mg_vcycle_noalloc: one preconditioner cycle without a handle and without
// any device allocation.
//
// Who needs it: code that runs where cudaMalloc is not available or not
// allowed -- for example a caller inside a CUDA stream capture it does not
// own, a plugin handed a fixed memory budget by its host application, or a
// real-time loop that must never enter the allocator -- and that still wants
// to apply the multigrid cycle to its own arrays.
//
// How: every temporary of the cycle (cell bytes of each level, the level
// vectors, the coarsest-level inverse) is carved out of one file-scope
// device array, kScratchBytes long, that exists on every GPU that loads the
// library until the process exits.  Host code cannot use the array's name
// as a device address, so the first call on each device, with that device
// current, looks the address up with cudaGetSymbolAddress and caches it,
// and raises the shared-memory limit of every kernel variant this entry
// point can launch (2D and 3D, with and without a mask, any sweep count).
// That first call should therefore come before any stream capture; later
// calls make no CUDA call other than kernel launches and device queries
// (cudaGetDevice, cudaDeviceGetAttribute).
// cudaDeviceReset destroys the array together with the context: the cached
// address is then stale, so do not call this entry point on a device after
// resetting it.
//
// Every call shares the one array and leaves its contents behind; nothing in
// the cycle reads a value that an earlier call left (each buffer is written
// before it is read), so no clearing is needed -- except the set-up of an
// unmasked call: when the previous call on the device had no mask and the
// same geometry (sizes, spacings, faces, level counts), the coarsest-level
// inverse and the coarse block's image it left in the array are used again
// (the set-up was 66-87% of a call's time on 64^2 to 64^3 grids).  A masked
// call always builds its set-up (the mask's contents may have changed).
// Calls that overlap on the GPU (different streams, or several host
// threads) race on the array: the caller must serialise them.
#include <mutex>
#include <string.h>

#include "launch.h"
#include "mg_kernels.cuh"

namespace npmg {

constexpr size_t kScratchBytes = 8u << 20;     // 8 MiB per device
constexpr int64_t kNoallocMaxCells = 1 << 18;  // finest level: 512^2, 64^3
constexpr int kNoallocMaxCoarse = 256;         // coarsest-level cells

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
static unsigned char* g_scratch_ptr[kMaxDevices];
static std::mutex g_scratch_mutex;

// The geometry of the last unmasked call's set-up on each device (valid
// while no masked or failed call came since).
struct SetupKey {
  int dim, L, kc, bcD;
  int64_t n[3];
  double h[3];
};
static SetupKey g_setup_key[kMaxDevices];
static bool g_setup_valid[kMaxDevices];

// Set-up of the current device, done once: the array's device address and
// the shared-memory opt-in of every kernel variant of the cycle.
static cudaError_t prepare_all_variants() {
  // the opt-in is the same for every sweep count (the device maximum); the
  // largest sweep count checks that the widest halo still fits
  cudaError_t e = prepare_level_kernels<2, float, false>(kMaxHalo, kMaxHalo);
  if (e == cudaSuccess) e = prepare_level_kernels<2, float, true>(kMaxHalo, kMaxHalo);
  if (e == cudaSuccess) e = prepare_level_kernels<3, float, false>(kMaxHalo, kMaxHalo);
  if (e == cudaSuccess) e = prepare_level_kernels<3, float, true>(kMaxHalo, kMaxHalo);
  if (e == cudaSuccess) e = prepare_coarse<float>(0);
  return e;
}

static cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e == cudaSuccess) e = prepare_all_variants();
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (unsigned char*)p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace npmg

using namespace npmg;

extern "C" mg_status mg_vcycle_noalloc(int dim, const int64_t shape[3], const double spacing[3], const int bc[6],
                                       const uint8_t* d_solid, const mg_options* opt, const float* d_r, float* d_z,
                                       void* stream) {
  if ((dim != 2 && dim != 3) || !shape || !spacing || !bc || !d_r || !d_z) {
    set_error("mg_vcycle_noalloc: invalid arguments");
    return MG_ERR_INVALID;
  }
  if (((uintptr_t)d_r | (uintptr_t)d_z) & 15) {
    set_error("mg_vcycle_noalloc: d_r and d_z must be 16-byte aligned");
    return MG_ERR_INVALID;
  }
  mg_options o;
  if (opt) o = *opt;
  else mg_default_options(&o);
  if (o.prec != MG_FP32 || o.cycle != MG_CYCLE_V || o.pre < 0 || o.pre > kMaxHalo || o.post < 0 || o.post > kMaxHalo ||
      !(o.omega > 0.0 && o.omega <= 2.0) || !(o.coarse_scale > 0.0) || o.levels < 0 || o.levels > kMaxLevels) {
    set_error("mg_vcycle_noalloc: invalid options (float32 only, pre/post in [0,%d])", kMaxHalo);
    return MG_ERR_INVALID;
  }
  int64_t n0[3] = {shape[0], shape[1], dim == 3 ? shape[2] : 1};
  int64_t total = 1;
  for (int a = 0; a < dim; ++a) {
    if (n0[a] < 2 || !(spacing[a] > 0.0)) {
      set_error("mg_vcycle_noalloc: shape must be >= 2 and spacing > 0");
      return MG_ERR_INVALID;
    }
    total *= n0[a];
  }
  if (total > kNoallocMaxCells) {
    set_error("mg_vcycle_noalloc: %lld cells exceed the maximum of %lld for the static scratch",
              (long long)total, (long long)kNoallocMaxCells);
    return MG_ERR_INVALID;
  }
  int bcD = 0;
  for (int f = 0; f < 2 * dim; ++f) {
    if (bc[f] != MG_BC_DIRICHLET && bc[f] != MG_BC_NEUMANN) {
      set_error("mg_vcycle_noalloc: bad bc[%d]", f);
      return MG_ERR_INVALID;
    }
    if (bc[f] == MG_BC_DIRICHLET) bcD |= 1 << f;
  }
  if (!d_solid && !bcD) {
    set_error("mg_vcycle_noalloc: all faces Neumann and no mask: the operator is singular");
    return MG_ERR_INVALID;
  }
  // levels: the same rule as mg_create
  int L = o.levels;
  if (L == 0) {
    L = 1;
    for (;;) {
      bool ok = L < kMaxLevels;
      for (int a = 0; a < dim; ++a) {
        const int64_t s = n0[a] >> (L - 1);
        ok = ok && (s % 2 == 0) && (s / 2 >= 4);
      }
      if (!ok) break;
      ++L;
    }
  }
  for (int a = 0; a < dim; ++a) {
    if (n0[a] % (1LL << (L - 1)) != 0 || (n0[a] >> (L - 1)) < 2) {
      set_error("mg_vcycle_noalloc: side %lld not divisible by 2^(levels-1)", (long long)n0[a]);
      return MG_ERR_INVALID;
    }
  }
  int64_t nk[kMaxLevels][3];
  size_t ncell[kMaxLevels];
  for (int k = 0; k < L; ++k) {
    for (int a = 0; a < 3; ++a) nk[k][a] = a < dim ? (n0[a] >> k) : 1;
    ncell[k] = (size_t)nk[k][0] * nk[k][1] * nk[k][2];
  }
  const int ncoarse = (int)ncell[L - 1];
  if (ncoarse > kNoallocMaxCoarse) {
    set_error("mg_vcycle_noalloc: coarsest level has %d cells (max %d); use more levels", ncoarse,
              kNoallocMaxCoarse);
    return MG_ERR_INVALID;
  }
  int dev = 0, optin = 0;
  NPMG_CUDA(cudaGetDevice(&dev));
  NPMG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  LevelDev geo[kMaxLevels];
  for (int k = 0; k < L; ++k) {
    geo[k].nx = (int)nk[k][0];
    geo[k].ny = (int)nk[k][1];
    geo[k].nz = (int)nk[k][2];
  }
  const int kc = coarse_start_level(geo, L, dim, (size_t)optin - 2048);
  // carve the static scratch
  unsigned char* base = nullptr;
  NPMG_CUDA(scratch_address(&base));
  size_t off = 0;
  bool fits = true;
  auto take = [&](size_t bytes) -> void* {
    off = (off + 255) / 256 * 256;
    void* p = base + off;
    off += bytes;
    if (off > kScratchBytes) fits = false;
    return p;
  };
  const bool masked = d_solid != nullptr;
  uint8_t* solid[kMaxLevels] = {};
  uint8_t* cell[kMaxLevels] = {};
  float* xk[kMaxLevels] = {};
  float* yk[kMaxLevels] = {};
  float* bk[kMaxLevels] = {};
  for (int k = 0; k < L; ++k) {
    if (masked) {
      solid[k] = k == 0 ? nullptr : (uint8_t*)take(ncell[k]);
      cell[k] = (uint8_t*)take(ncell[k]);
    }
  }
  for (int k = 0; k <= kc; ++k) {
    if (k >= 1) bk[k] = (float*)take(ncell[k] * 4);
    if (k < kc) xk[k] = (float*)take(ncell[k] * 4);
    if (k >= 1) yk[k] = (float*)take(ncell[k] * 4);
  }
  double* inv = (double*)take((size_t)2 * ncoarse * ncoarse * 8);
  size_t image_bytes;
  {
    int offtmp[kMaxLevels];
    image_bytes = coarse_layout(offtmp, geo + kc, L - kc, dim);
  }
  float* image = (float*)take(image_bytes);
  if (!fits) {
    set_error("mg_vcycle_noalloc: the problem needs more than the %zu bytes of static scratch", kScratchBytes);
    return MG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const double c = spacing[0] * spacing[0];
  LevelDev lv[kMaxLevels];
  for (int k = 0; k < L; ++k) {
    lv[k].nx = (int)nk[k][0];
    lv[k].ny = (int)nk[k][1];
    lv[k].nz = (int)nk[k][2];
    const double hk[3] = {spacing[0] * (1 << k), spacing[1] * (1 << k), dim == 3 ? spacing[2] * (1 << k) : 1.0};
    lv[k].wx = (float)(c / (hk[0] * hk[0]));
    lv[k].wy = (float)(c / (hk[1] * hk[1]));
    lv[k].wz = dim == 3 ? (float)(c / (hk[2] * hk[2])) : 0.f;
    lv[k].bcD = bcD;
    lv[k].cell = masked ? cell[k] : nullptr;
  }
  SetupKey key;
  memset(&key, 0, sizeof(key));
  key.dim = dim;
  key.L = L;
  key.kc = kc;
  key.bcD = bcD;
  for (int a = 0; a < 3; ++a) {
    key.n[a] = n0[a];
    key.h[a] = a < dim ? spacing[a] : 1.0;
  }
  bool reuse = false;
  if (dev >= 0 && dev < kMaxDevices) {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    reuse = !masked && g_setup_valid[dev] && memcmp(&key, &g_setup_key[dev], sizeof(key)) == 0;
    g_setup_valid[dev] = false;  // set again below once this call is enqueued
  }
  // hierarchy of the mask and the coarsest inverse
  if (masked) {
    for (int k = 1; k < L; ++k)
      NPMG_CUDA(launch_coarsen_solid(dim, nk[k - 1], k == 1 ? d_solid : solid[k - 1], solid[k], s));
    for (int k = 0; k < L; ++k) NPMG_CUDA(launch_cell_bytes(dim, nk[k], bcD, k == 0 ? d_solid : solid[k], cell[k], s));
  }
  {
    const double hk[3] = {spacing[0] * (1 << (L - 1)), spacing[1] * (1 << (L - 1)),
                          dim == 3 ? spacing[2] * (1 << (L - 1)) : 1.0};
    const double wd[3] = {c / (hk[0] * hk[0]), c / (hk[1] * hk[1]), dim == 3 ? c / (hk[2] * hk[2]) : 0.0};
    if (!reuse) NPMG_CUDA(launch_coarse_inverse(dim, nk[L - 1], wd, bcD, masked ? cell[L - 1] : nullptr, inv, s));
  }
  CoarseArgs ca;
  memset(&ca, 0, sizeof(ca));
  // (the coarse block's shared memory was opted in to the device maximum at
  // set-up; coarse_start_level keeps the layout within it)
  ca.nlev = L - kc;
  ca.dim = dim;
  for (int l = 0; l < ca.nlev; ++l) ca.lv[l] = lv[kc + l];
  const size_t moff = coarse_layout(ca.off, ca.lv, ca.nlev, dim);
  ca.ncoarse = ncoarse;
  ca.inv = reinterpret_cast<const float*>(inv);
  ca.pre = o.pre;
  ca.post = o.post;
  ca.omega = (float)o.omega;
  ca.s = (float)o.coarse_scale;
  ca.finest = 0;
  ca.image = nullptr;
  if (!reuse) NPMG_CUDA(launch_coarse_image(ca, image, moff, s));
  ca.image = image;
  const float om = (float)o.omega, sc = (float)o.coarse_scale;
  auto cycle = [&](auto dimc, auto mc) -> cudaError_t {
    constexpr int DIM = decltype(dimc)::value;
    constexpr bool M = decltype(mc)::value;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kc && e == cudaSuccess; ++k)
      e = launch_down<DIM, float, M>(lv[k], k == 0 ? (const void*)d_r : bk[k], xk[k], bk[k + 1], o.pre, om,
                                     nullptr, s);
    if (e == cudaSuccess)
      e = launch_coarse<float>(ca, moff, kc == 0 ? (const void*)d_r : bk[kc], kc == 0 ? (void*)d_z : yk[kc],
                               nullptr, s);
    for (int k = kc - 1; k >= 0 && e == cudaSuccess; --k)
      e = launch_up<DIM, float, M, false>(lv[k], k == 0 ? (const void*)d_r : bk[k], xk[k],
                                          k == 0 ? (void*)d_z : yk[k], yk[k + 1], o.post, om, sc, nullptr, nullptr,
                                          s);
    return e;
  };
  cudaError_t e;
  if (dim == 2)
    e = masked ? cycle(std::integral_constant<int, 2>(), std::true_type())
               : cycle(std::integral_constant<int, 2>(), std::false_type());
  else
    e = masked ? cycle(std::integral_constant<int, 3>(), std::true_type())
               : cycle(std::integral_constant<int, 3>(), std::false_type());
  if (e != cudaSuccess) {
    set_error("mg_vcycle_noalloc: %s", cudaGetErrorString(e));
    return MG_ERR_CUDA;
  }
  if (!masked && dev >= 0 && dev < kMaxDevices) {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    g_setup_key[dev] = key;
    g_setup_valid[dev] = true;
  }
  return MG_OK;
}
