// Ordered split reductions: the cube is the sum over pixel splits s = 0, 1, ... (in this
// order) of the contraction's partial sums, with compensated (Kahan) FP32 additions per
// component, so that the result does not depend on which split finished first and keeps
// about one rounding of error whatever the split count.  Two layouts: the FP32 direct
// sum's partials [split][V N_s][L], and the tensor-core contraction's tiled partials
// [split][row tile][column tile][column pair][128 rows] (see tensor_split_stride).
#include <algorithm>

#include "rsim_internal.h"

namespace rsim {
namespace {

// cube = scale * sum over splits s = 0, 1, ... (in this order) of partial[s], with
// compensated FP32 additions (GB300's FP64 rate is a small fraction of its FP32 rate).
// Loads of kReduceBatch splits are issued together; the additions keep the split order.
__global__ void split_reduce(const FrameIO* __restrict__ frames, int64_t count, int splits,
                             int out_dtype, int scale_mode) {
  wait_prior_grid();
  const FrameIO& fr = frames[blockIdx.y];
  float scale = 1.f;
  if (scale_mode) {
    const float m = __uint_as_float((unsigned)fr.meta[1]);
    scale = (m > 0.f) ? ldexpf(1.f, ilogbf(m) + 1) : 1.f;
  }
  const float2* __restrict__ part = fr.partial;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    float re = 0.f, im = 0.f, cre = 0.f, cim = 0.f;
    for (int s0 = 0; s0 < splits; s0 += kReduceBatch) {
      float2 p[kReduceBatch];
#pragma unroll
      for (int j = 0; j < kReduceBatch; ++j)
        p[j] = (s0 + j < splits) ? __ldcs(part + (int64_t)(s0 + j) * count + i) : make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < kReduceBatch; ++j) {
        if (s0 + j < splits) {
          kahan_add(re, cre, p[j].x);
          kahan_add(im, cim, p[j].y);
        }
      }
    }
    re *= scale;  // power of two: exact
    im *= scale;
    if (out_dtype == RSIM_C128)
      reinterpret_cast<double2*>(fr.cube)[i] = make_double2((double)re, (double)im);
    else
      reinterpret_cast<float2*>(fr.cube)[i] = make_float2(re, im);
  }
}

// cube = scale * sum over splits s = 0, 1, ... (in this order) of the tiled partial
// sums, with compensated FP32 additions per component.  One thread per (accumulator
// row, column pair) of a tile: the loads of consecutive threads are contiguous.  The
// loads of kTileBatch (4) splits are issued together; the additions keep the split
// order.  Four loads at a time fit 40 registers, so six blocks of 256 threads stay
// resident per SM and a 256 x 256-pixel frame's 768 blocks run in one wave: with eight
// (64 registers, four blocks per SM) the last 160 blocks ran as a second, quarter-full
// wave (18.7 against 16.7 us).  Sixteen at a time took 125 registers and was slower still.
constexpr int kTileBatch = 4;
__global__ void __launch_bounds__(256, 6) split_reduce_tiles(const FrameIO* __restrict__ frames, Consts k, int NT, int ntiles,
                                   int64_t sstride, int splits, int out_dtype, int scale_mode) {
  wait_prior_grid();
  const FrameIO& fr = frames[blockIdx.y];
  float scale = 1.f;
  if (scale_mode) {
    const float m = __uint_as_float((unsigned)fr.meta[1]);
    scale = (m > 0.f) ? ldexpf(1.f, ilogbf(m) + 1) : 1.f;
  }
  const int64_t rows = (int64_t)k.V * k.Ns;
  const int64_t n4 = sstride / 2;
  const int pairs = NT / 2;
  const float4* __restrict__ part = reinterpret_cast<const float4*>(fr.partial);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n4; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e & 127);
    const int64_t q = e >> 7;
    const int pr = (int)(q % pairs);
    const int64_t tile = q / pairs;
    const int64_t row = (tile / ntiles) * 128 + r;
    const int l = (int)(tile % ntiles) * NT + 2 * pr;
    if (row >= rows || l >= k.L) continue;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
    for (int b = 0; b < splits; b += kTileBatch) {
      float4 p[kTileBatch];
#pragma unroll
      for (int j = 0; j < kTileBatch; ++j)
        p[j] = (b + j < splits) ? __ldcs(part + (int64_t)(b + j) * n4 + e) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int j = 0; j < kTileBatch; ++j) {
        if (b + j < splits) {
          kahan_add(s0, c0, p[j].x);
          kahan_add(s1, c1, p[j].y);
          kahan_add(s2, c2, p[j].z);
          kahan_add(s3, c3, p[j].w);
        }
      }
    }
    const int64_t o = row * k.L + l;
    const bool two = (l + 1 < k.L);
    if (out_dtype == RSIM_C128) {
      double2* cd = reinterpret_cast<double2*>(fr.cube);
      cd[o] = make_double2((double)(s0 * scale), (double)(s1 * scale));
      if (two) cd[o + 1] = make_double2((double)(s2 * scale), (double)(s3 * scale));
    } else {
      float2* cf = reinterpret_cast<float2*>(fr.cube);
      cf[o] = make_float2(s0 * scale, s1 * scale);
      if (two) cf[o + 1] = make_float2(s2 * scale, s3 * scale);
    }
  }
}

}  // namespace

cudaError_t launch_reduce(const Consts& k, const FrameIO* frames, int F, int splits, int out_dtype,
                          float scale_mode, cudaStream_t st) {
  const int64_t count = (int64_t)k.V * k.Ns * k.L;
  if (count <= 0 || F <= 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  dim3 grid((unsigned)blocks, F);
  return launch_dependent(split_reduce, grid, dim3(256), 0, st, frames, count, splits, out_dtype,
                          scale_mode != 0.f ? 1 : 0);
}

cudaError_t launch_reduce_tiles(const Consts& k, const FrameIO* frames, int F, int splits, int nt,
                                int out_dtype, bool scale_from_meta, int num_sms, cudaStream_t st) {
  const int64_t sstride = tensor_split_stride(k.V, k.Ns, k.L, nt);
  const int64_t n4 = sstride / 2;
  if (n4 <= 0 || F <= 0) return cudaSuccess;
  // at most one wave of resident blocks (6 x 256 threads per SM) over all frames, grid-stride
  int64_t blocks = (n4 + 255) / 256;
  const int64_t wave = std::max<int64_t>(1, 6ll * num_sms / F);
  if (blocks > wave) blocks = wave;
  return launch_dependent(split_reduce_tiles, dim3((unsigned)blocks, F), dim3(256), 0, st, frames, k, nt,
                          (k.L + nt - 1) / nt, sstride, splits, out_dtype, scale_from_meta ? 1 : 0);
}

}  // namespace rsim
