// mg_probe_l2_read: the L2 roof of kernels whose working set stays in L2.
//
// One launch reads a caller buffer `reps` times with coalesced 16-byte
// loads (grid-stride, one wave of blocks over every SM); when the buffer
// fits in L2, every pass after the first is served by L2, so bytes read /
// launch time is the L2 read bandwidth a streaming kernel can reach.  The
// per-block sums go to d_sink so the loads are not optimised away.
#include "npmg_internal.cuh"

namespace npmg {
namespace {

__global__ void __launch_bounds__(512) k_l2_read(const float4* __restrict__ buf, int64_t n4, int reps,
                                                 float* __restrict__ sink) {
  float acc = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(buf + i);
      acc += (v.x + v.y) + (v.z + v.w);
    }
  }
  __shared__ float red[512];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) sink[blockIdx.x] = red[0];
}

}  // namespace
}  // namespace npmg

using namespace npmg;

extern "C" mg_status mg_probe_l2_read(const float* d_buf, int64_t n, int reps, float* d_sink, int sink_len,
                                      void* stream) {
  if (!d_buf || !d_sink || n <= 0 || (n & 3) || reps <= 0 || ((uintptr_t)d_buf & 15)) {
    set_error("mg_probe_l2_read: need a 16-byte aligned buffer of a positive multiple of 4 floats, reps > 0");
    return MG_ERR_INVALID;
  }
  int dev = 0, nsm = 0;
  NPMG_CUDA(cudaGetDevice(&dev));
  NPMG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = 4 * nsm;
  if (sink_len < blocks) {
    set_error("mg_probe_l2_read: d_sink needs %d floats", blocks);
    return MG_ERR_INVALID;
  }
  k_l2_read<<<blocks, 512, 0, (cudaStream_t)stream>>>(reinterpret_cast<const float4*>(d_buf), n / 4, reps, d_sink);
  NPMG_CUDA(cudaGetLastError());
  return MG_OK;
}
