// Measured rate of the unit that bounds the NUFFT tier's spreading kernel: non-returning
// 32-bit integer atomic additions to shared memory without bank conflicts.  The
// spreading kernel adds every tap of a record with such atomics (two words per
// component, see k_nufft.cu), so this rate, taken on the device the library runs on,
// is the roofline denominator of that kernel.  The probe has the spreading kernel's
// occupancy (four blocks of 256 threads per SM) and its access pattern: each atomic
// instruction of a warp touches 32 consecutive words, one per bank, of one of four word
// arrays.
#include <cuda_runtime.h>

#include <algorithm>

#include "rsim_ctx.h"

namespace rsim {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeWords = 1024;  // per array
constexpr int kProbeIters = 2048;

__global__ void __launch_bounds__(kProbeThreads) smem_atomic_probe(unsigned* sink) {
  __shared__ unsigned w[4][kProbeWords];
  for (int i = threadIdx.x; i < 4 * kProbeWords; i += blockDim.x) (&w[0][0])[i] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // word (warp 32 + lane + 256 it) mod 1024: a warp's 32 lanes on 32 consecutive words
  int o = warp * 32 + lane;
#pragma unroll 4
  for (int it = 0; it < kProbeIters; ++it) {
    atomicAdd(&w[0][o], 1u);
    atomicAdd(&w[1][o], (unsigned)it);
    atomicAdd(&w[2][o], 3u);
    atomicAdd(&w[3][o], (unsigned)lane);
    o = (o + kProbeThreads) & (kProbeWords - 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(sink, w[0][0] ^ w[1][1] ^ w[2][2] ^ w[3][3]);  // the sums are used
}

}  // namespace
}  // namespace rsim

using namespace rsim;

extern "C" rsim_status rsim_measure_smem_atomics(rsim_ctx* ctx, double* lane_ops_per_s, rsim_stream stream) {
  if (!ctx || !lane_ops_per_s) return fail(RSIM_ERR_INVALID_ARG, "NULL argument");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  // the context's status allocation holds 256 bytes; word 32 onwards is spare
  unsigned* sink = ctx->status_dev + 32;
  const int blocks = 4 * std::max(ctx->num_sms, 1);
  cudaEvent_t a, b;
  e = cudaEventCreate(&a);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
  e = cudaEventCreate(&b);
  if (e != cudaSuccess) {
    cudaEventDestroy(a);
    return cuda_fail(e, "cudaEventCreate");
  }
  float best = 1e30f;
  for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {  // the first run is a warm-up
    cudaEventRecord(a, st);
    smem_atomic_probe<<<blocks, kProbeThreads, 0, st>>>(sink);
    e = cudaGetLastError();
    cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    if (rep > 0 && ms > 0.f) best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(e, "shared-memory atomic probe");
  const double ops = (double)blocks * kProbeThreads * kProbeIters * 4.0;
  *lane_ops_per_s = ops / ((double)best * 1e-3);
  return RSIM_OK;
}
