// Measured peaks of the units that bound two kernels, taken on the device the library
// runs on (the roofline denominators the benchmarks report beside vendor-library figures).
//
// 1. The NUFFT tier's spreading kernel: non-returning
// 32-bit integer atomic additions to shared memory without bank conflicts.  The
// spreading kernel adds every tap of a record with such atomics (two words per
// component, see k_nufft.cu), so this rate, taken on the device the library runs on,
// is the roofline denominator of that kernel.  The probe has the spreading kernel's
// occupancy (four blocks of 256 threads per SM) and its access pattern: each atomic
// instruction of a warp touches 32 consecutive words, one per bank, of one of four word
// arrays.
//
// 2. The contraction's tensor-core instruction: tcgen05.mma kind::f16, M = 128, N = 256,
// K = 16, A from tensor memory and B from shared memory (128-byte-swizzled K-major), FP32
// accumulation, issued in the contraction's 12-MMA stages by one thread per CTA with at
// most three committed stages in flight, one CTA per SM, on zero operands.  Its flop rate
// is the ceiling of the contraction's executed flop rate (a cuBLAS GEMM, the measured
// BF16 peak, also spends time outside its MMAs).
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

constexpr int kMmaProbeThreads = 128;
constexpr int kMmaProbeStages = 2000;
constexpr int kMmaProbeSmem = 128 * 1024 + 1024;  // more than half an SM's: one CTA per SM
constexpr unsigned long long kMmaProbeWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool probe_wait(uint64_t* bar, uint32_t parity) {
  unsigned long long t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255u) == 255u) {
      unsigned long long now;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
      if (t0 == 0)
        t0 = now;
      else if (now - t0 > kMmaProbeWaitNs)
        return false;
    }
  }
}

__device__ __forceinline__ uint64_t probe_sdesc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset: 8-row groups 1024 B apart
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

__global__ void __launch_bounds__(kMmaProbeThreads, 1) mma_rate_probe(int stages, unsigned* err) {
  extern __shared__ unsigned char raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar[3];
  __shared__ uint32_t tbase;
  // B operand: hi and lo images of 256 rows x 128 B
  for (int i = threadIdx.x; i < 65536 / 16; i += blockDim.x) reinterpret_cast<int4*>(sm)[i] = make_int4(0, 0, 0, 0);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    for (int i = 0; i < 3; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_addr(&tbase))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tm = tbase;
  // zero the 512 columns of this warp's lane quarter (accumulator and A)
  const uint32_t lanes = (uint32_t)(32 * (threadIdx.x >> 5)) << 16;
  for (int c = 0; c < 512; c += 16)
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1, %1};" ::"r"(tm + lanes + c),
        "r"(0u)
        : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x == 0) {
    const uint64_t bd = probe_sdesc(smem_addr(sm));
    constexpr uint64_t kLo = 32768 >> 4;
    // kind::f16, FP32 accumulator, FP16 A and B, K-major, N = 256, M = 128
    const uint32_t idesc = (1u << 4) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint32_t a = tm + 256;  // A: hi part in 32 columns, lo part in the next 32
    bool ok = true;
    for (int it = 0; it < stages && ok; ++it) {
      const int s = it % 3;
      if (it >= 3) ok = probe_wait(&bar[s], (uint32_t)((it / 3 - 1) & 1));
      if (!ok) break;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        asm volatile(
            "{\n\t.reg .pred t;\n\tsetp.ne.b32 t, 1, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %5, t;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %3, %5, t;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%4], %2, %5, t;\n\t}" ::"r"(tm),
            "r"(a + 8 * ks), "l"(bd + 2 * ks), "l"(bd + kLo + 2 * ks), "r"(a + 32 + 8 * ks), "r"(idesc)
            : "memory");
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(&bar[s]))
                   : "memory");
    }
    // every committed stage completes before tensor memory is released
    for (int it = stages > 3 ? stages - 3 : 0; it < stages && ok; ++it)
      ok = probe_wait(&bar[it % 3], (uint32_t)((it / 3) & 1));
    if (!ok) atomicAdd(err, 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tm) : "memory");
}

}  // namespace
}  // namespace rsim

using namespace rsim;

extern "C" rsim_status rsim_measure_smem_atomics(rsim_ctx* ctx, double* lane_ops_per_s, rsim_stream stream) {
  if (!ctx || !lane_ops_per_s) return fail(RSIM_ERR_INVALID_ARG, "NULL argument");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  // the probe's word of the context's status allocation
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

extern "C" rsim_status rsim_measure_mma_rate(rsim_ctx* ctx, double* flops_per_s, rsim_stream stream) {
  if (!ctx || !flops_per_s) return fail(RSIM_ERR_INVALID_ARG, "NULL argument");
  if (!(ctx->cc_major == 10 && ctx->cc_minor == 3))
    return fail(RSIM_ERR_UNSUPPORTED, "the tensor-core probe needs an sm_103 device");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* err = ctx->status_dev + 33;  // the probe's word of the status allocation
  e = cudaFuncSetAttribute(mma_rate_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaProbeSmem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  e = cudaMemsetAsync(err, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  const int blocks = std::max(ctx->num_sms, 1);
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
    mma_rate_probe<<<blocks, kMmaProbeThreads, kMmaProbeSmem, st>>>(kMmaProbeStages, err);
    e = cudaGetLastError();
    cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    if (rep > 0 && ms > 0.f) best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core probe");
  unsigned nerr = 0;
  e = cudaMemcpy(&nerr, err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core probe status");
  if (nerr) return fail(RSIM_ERR_TIMEOUT, "tensor-core probe: a wait ran out");
  const double flops = (double)blocks * kMmaProbeStages * 12.0 * 2.0 * 128.0 * 256.0 * 16.0;
  *flops_per_s = flops / ((double)best * 1e-3);
  return RSIM_OK;
}
