// Target estimation on synthesised cubes: range-Doppler maps and the velocity of
// maximum power per CPI (Section III: an FFT of each CPI's cube gives the
// range-Doppler map; the velocity of the strongest response, CPI after CPI, makes
// the Doppler-time plot).
//
//   X_v[k][d]   = sum_n sum_l cube[v][n][l] e^{-j 2 pi (k n / N_s + d l / L)}
//   power[k][d] = sum_v |X_v[k][d]|^2                 (channels added non-coherently)
//   v_est       = velocity of the Doppler bin d of the largest power[k][d]
//
// The slow-time phase of a pixel turns by -f_D T_slow per block, so its Doppler bin
// is (-f_D T_slow L) mod L and bin d (signed d_s in [-L/2, L/2)) maps to
// v = -d_s lambda / (2 T_slow L).  With the static-clutter option the d = 0 column is
// left out of the search (a zero-Doppler notch).
//
// Three kernels, all deterministic:
//   fft_rows   - eight (frame, channel, n) rows per CTA: radix-2 FFT over l in shared memory;
//   fft_cols   - one CTA per (frame, 16 Doppler columns): per channel, radix-2 FFT over
//                n of the 16 columns, |X|^2 added into a shared-memory tile in channel order;
//   rd_argmax  - one CTA per frame: the largest power (first index on ties) -> velocity.
// FFT lengths are powers of two up to 1024 (N_s) and 1024 (L).
#include <vector>

#include "rsim_ctx.h"
#include "rsim_internal.h"

namespace rsim {
namespace {

constexpr int kColBlock = 16;

__device__ __forceinline__ unsigned bitrev(unsigned x, int bits) { return __brev(x) >> (32 - bits); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// exp(-j 2 pi k / len) for 0 <= k < len / 2
__device__ __forceinline__ float2 twiddle(int k, int len) {
  float s, c;
  sincospif(-2.0f * (float)k / (float)len, &s, &c);
  return make_float2(c, s);
}

// In-place radix-2 decimation-in-time butterflies over `count` independent sequences of
// length n held in shared memory, element i of sequence j at x[i * istride + j * jstride],
// already in bit-reversed order.  All threads of the block take part.
__device__ void fft_stages(float2* x, int n, int count, int istride, int jstride) {
  const int half_total = (n / 2) * count;
  for (int len = 2; len <= n; len <<= 1) {
    const int h = len >> 1;
    __syncthreads();
    for (int t = threadIdx.x; t < half_total; t += blockDim.x) {
      const int j = t % count, b = t / count;
      const int grp = b / h, k = b % h;
      const int i0 = grp * len + k, i1 = i0 + h;
      const float2 w = twiddle(k, len);
      float2* p0 = x + i0 * istride + j * jstride;
      float2* p1 = x + i1 * istride + j * jstride;
      const float2 u = *p0, v = cmul(*p1, w);
      *p0 = make_float2(u.x + v.x, u.y + v.y);
      *p1 = make_float2(u.x - v.x, u.y - v.y);
    }
  }
  __syncthreads();
}

// Rows: FFT over l of every (frame, channel, n) row; 8 rows per CTA.
__global__ void fft_rows(const float2* const* __restrict__ cubes, float2* __restrict__ tmp, int F,
                         int V, int Ns, int L, int lbits) {
  extern __shared__ float2 srow[];
  const int rows_per = 8;
  const int64_t rows_total = (int64_t)F * V * Ns;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per;
  for (int e = threadIdx.x; e < rows_per * L; e += blockDim.x) {
    const int rr = e / L, l = e % L;
    const int64_t row = r0 + rr;
    float2 val = make_float2(0.f, 0.f);
    if (row < rows_total) {
      const int64_t f = row / ((int64_t)V * Ns), within = row % ((int64_t)V * Ns);
      val = cubes[f][within * L + l];
    }
    srow[rr * L + bitrev((unsigned)l, lbits)] = val;
  }
  fft_stages(srow, L, rows_per, 1, L);
  for (int e = threadIdx.x; e < rows_per * L; e += blockDim.x) {
    const int rr = e / L, l = e % L;
    const int64_t row = r0 + rr;
    if (row < rows_total) tmp[row * L + l] = srow[rr * L + l];
  }
}

// Columns: per frame and block of 16 Doppler bins, FFT over n for every channel and add
// |X|^2 over the channels in order.
__global__ void fft_cols(const float2* __restrict__ tmp, float* __restrict__ power, int V, int Ns,
                         int L, int nbits) {
  extern __shared__ float2 scol[];  // [Ns][kColBlock] complex, then [Ns][kColBlock] power
  float* pw = reinterpret_cast<float*>(scol + (size_t)Ns * kColBlock);
  const int f = blockIdx.y;
  const int d0 = blockIdx.x * kColBlock;
  for (int e = threadIdx.x; e < Ns * kColBlock; e += blockDim.x) pw[e] = 0.f;
  for (int v = 0; v < V; ++v) {
    const float2* src = tmp + (((int64_t)f * V + v) * Ns) * L;
    __syncthreads();
    for (int e = threadIdx.x; e < Ns * kColBlock; e += blockDim.x) {
      const int n = e / kColBlock, j = e % kColBlock;
      const int d = d0 + j;
      const float2 val = (d < L) ? src[(int64_t)n * L + d] : make_float2(0.f, 0.f);
      scol[bitrev((unsigned)n, nbits) * kColBlock + j] = val;
    }
    fft_stages(scol, Ns, kColBlock, kColBlock, 1);
    for (int e = threadIdx.x; e < Ns * kColBlock; e += blockDim.x) {
      const float2 x = scol[e];
      pw[e] += x.x * x.x + x.y * x.y;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < Ns * kColBlock; e += blockDim.x) {
    const int k = e / kColBlock, j = e % kColBlock;
    const int d = d0 + j;
    if (d < L) power[((int64_t)f * Ns + k) * L + d] = pw[e];
  }
}

// Largest power of one frame (first flat index on ties), optionally without d = 0.
__global__ void rd_argmax(const float* __restrict__ power, int Ns, int L, int skip_static,
                          double v_per_bin, float* __restrict__ v_est, int32_t* __restrict__ peak) {
  const int f = blockIdx.x;
  const float* p = power + (int64_t)f * Ns * L;
  float best = -1.f;
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < Ns * L; i += blockDim.x) {
    const int d = i % L;
    if (skip_static && d == 0) continue;
    const float x = p[i];
    if (x > best || (x == best && i < bi)) {
      best = x;
      bi = i;
    }
  }
  __shared__ float sb[32];
  __shared__ int si[32];
  for (int o = 16; o > 0; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sb[w] = best;
    si[w] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
      if (sb[k] > best || (sb[k] == best && si[k] < bi)) {
        best = sb[k];
        bi = si[k];
      }
    const int d = bi % L;
    const int ds = (d < L / 2) ? d : d - L;
    v_est[f] = (float)(-(double)ds * v_per_bin);
    if (peak) {
      peak[2 * f] = bi / L;
      peak[2 * f + 1] = d;
    }
  }
}

int ilog2(int x) {
  int b = 0;
  while ((1 << b) < x) ++b;
  return b;
}

}  // namespace

cudaError_t launch_range_doppler(const float2* const* cubes_dev, float2* tmp, float* power, int F,
                                 int V, int Ns, int L, int skip_static, double v_per_bin, float* v_est,
                                 int32_t* peak, cudaStream_t st) {
  const int lbits = ilog2(L), nbits = ilog2(Ns);
  const int64_t rows = (int64_t)F * V * Ns;
  const int64_t row_blocks = (rows + 7) / 8;
  if (row_blocks > 0x7fffffffll) return cudaErrorInvalidConfiguration;
  const int rsmem = 8 * L * (int)sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(fft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, rsmem);
  if (e != cudaSuccess) return e;
  fft_rows<<<(unsigned)row_blocks, 256, rsmem, st>>>(cubes_dev, tmp, F, V, Ns, L, lbits);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int smem = Ns * kColBlock * (int)(sizeof(float2) + sizeof(float));
  e = cudaFuncSetAttribute(fft_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  fft_cols<<<dim3((L + kColBlock - 1) / kColBlock, F), 256, smem, st>>>(tmp, power, V, Ns, L, nbits);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  rd_argmax<<<F, 256, 0, st>>>(power, Ns, L, skip_static, v_per_bin, v_est, peak);
  return cudaGetLastError();
}

}  // namespace rsim

using namespace rsim;

extern "C" rsim_status rsim_range_doppler(rsim_ctx* ctx, const rsim_radar_params* params,
                                          void* const* cubes, int32_t F, float* power, float* v_est,
                                          int32_t* peak, int32_t options, rsim_stream stream) {
  if (!ctx || !cubes || !power || !v_est) return fail(RSIM_ERR_INVALID_ARG, "NULL argument");
  if (F < 1) return fail(RSIM_ERR_INVALID_ARG, "F must be >= 1");
  if (options & ~RSIM_RD_SKIP_STATIC) return fail(RSIM_ERR_INVALID_ARG, "unknown option bits");
  Consts k;
  rsim_status s = check_params(params, &k);
  if (s != RSIM_OK) return s;
  auto pow2 = [](int x) { return x >= 2 && x <= 1024 && (x & (x - 1)) == 0; };
  if (!pow2(k.Ns) || !pow2(k.L))
    return fail(RSIM_ERR_UNSUPPORTED, "range-Doppler processing needs N_s and L powers of two in 2..1024");
  for (int f = 0; f < F; ++f)
    if (!cubes[f]) return fail(RSIM_ERR_INVALID_ARG, "a cube pointer is NULL");
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ptr_bytes = ((sizeof(void*) * (size_t)F + 255) / 256) * 256;
  const size_t tmp_bytes = sizeof(float2) * (size_t)F * k.V * k.Ns * k.L;
  s = ensure_workspace(ctx, ptr_bytes + tmp_bytes, st);
  if (s != RSIM_OK) return s;
  char* ws = (char*)ctx->ws;
  cudaError_t e = cudaMemcpyAsync(ws, cubes, sizeof(void*) * (size_t)F, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "upload of the cube table");
  const double t_slow = params->t_slow > 0 ? params->t_slow : params->M * params->t_b;
  const double v_per_bin = params->lambda / (2.0 * t_slow * k.L);
  e = launch_range_doppler((const float2* const*)ws, (float2*)(ws + ptr_bytes), power, F, k.V, k.Ns, k.L,
                           (options & RSIM_RD_SKIP_STATIC) ? 1 : 0, v_per_bin, v_est, peak, st);
  if (e != cudaSuccess) return cuda_fail(e, "range-Doppler kernels");
  return RSIM_OK;
}
