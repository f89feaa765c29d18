// FP32 direct sum of Eq. 2 on CUDA cores.
//
// The phase of Eq. 2 separates into a fast-time/channel part a_{p,v} n + c_{p,v} and a
// slow-time part b_p l, so each cube entry is
//     cube[v][n][l] = sum_q G_v[q][n] * D[q][l],
//     G_v[q][n] = exp(j 2 pi (a_{q,v} n + c_{q,v})),   D[q][l] = sigma_q exp(j 2 pi b_q l),
// over the compacted valid pixels q.  A CTA owns a TN (n) x 64 (l) tile of one channel
// and one contiguous split of the pixels, TN = 128 or 64 (a plan's tile shape); per
// 32-pixel chunk it writes the chunk's phasors to shared memory (phases are exact 32-bit
// fixed-point products, so only a phase in [-1/2, 1/2) cycle is ever converted to float)
// and then every thread accumulates a (TN / 16) x 4 block of complex outputs with 4 FFMA
// per term.
#include <algorithm>

#include "rsim_internal.h"

namespace rsim {
namespace {

constexpr int kTL = kDirectTileL;  // l per tile
constexpr int kThreads = 256;

// exp(j 2 pi x) for a 2^-32-cycle fixed-point phase.  The phase is reinterpreted as
// a signed fraction in [-1/2, 1/2) cycle, so the argument of the hardware sine and
// cosine is within [-pi, pi), where their absolute error is below 2^-21.
__device__ __forceinline__ float2 cis_q32(uint32_t ph) {
  const float ang = (float)(int32_t)ph * 1.46291807926715968e-09f;  // 2 pi / 2^32
  float s, c;
  __sincosf(ang, &s, &c);
  return make_float2(c, s);
}

__device__ __forceinline__ void cmac(float2& acc, float2 g, float2 d) {
  acc.x = fmaf(g.x, d.x, acc.x);
  acc.x = fmaf(-g.y, d.y, acc.x);
  acc.y = fmaf(g.x, d.y, acc.y);
  acc.y = fmaf(g.y, d.x, acc.y);
}

// The raw per-pixel data of one 32-pixel chunk (this channel's phases, the slow-time
// increment and sigma), copied into shared memory asynchronously one chunk ahead of its
// use, so that the phasor fill never waits for global memory.
struct RawChunk {
  uint32_t a[kChunkPx];
  uint32_t c[kChunkPx];
  uint32_t b[kChunkPx];
  float2 sig[kChunkPx];
};
constexpr int kRawCopies = (int)sizeof(RawChunk) / 16;  // 16-byte copies per chunk (40)

// Issue the copies of chunk q0 / 32 into `raw` (threads 0..kRawCopies-1, one 16-byte
// cp.async each) and commit them as one group.  The sources are 16-byte aligned (rows
// of kChunkPx words start at multiples of 128 bytes) and lie within the frame's
// capacity, also for the last chunk.
__device__ __forceinline__ void stage_raw(RawChunk* raw, const FrameIO& fr, const uint32_t* pA,
                                          const uint32_t* pC, int64_t q0) {
  const int t = threadIdx.x;
  if (t < kRawCopies) {
    const char* src;
    if (t < 8)
      src = reinterpret_cast<const char*>(pA + q0) + 16 * t;
    else if (t < 16)
      src = reinterpret_cast<const char*>(pC + q0) + 16 * (t - 8);
    else if (t < 24)
      src = reinterpret_cast<const char*>(fr.phB + q0) + 16 * (t - 16);
    else
      src = reinterpret_cast<const char*>(fr.sig + q0) + 16 * (t - 24);
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(reinterpret_cast<char*>(raw) + 16 * t);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void wait_raw_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void wait_raw_but_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Phasor tiles of one 32-pixel chunk from its staged raw data: G[q][n] = e^{j 2 pi (a n + c)}
// (channel v), D[q][l] = sigma e^{j 2 pi b l}; zero outside the frame / the cube.
template <int TN>
__device__ __forceinline__ void fill_chunk(float2 (*Gs)[TN], float2 (*Ds)[kTL], const RawChunk& raw,
                                           int64_t q0, int64_t pv, int n0, int l0, const Consts& k) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int i = 0; i < (kChunkPx * TN) / kThreads; ++i) {
    const int e = tid + i * kThreads;
    const int qq = e / TN, nn = e % TN;
    const int64_t q = q0 + qq;
    const int n = n0 + nn;
    float2 g = make_float2(0.f, 0.f);
    if (q < pv && n < k.Ns) g = cis_q32(raw.a[qq] * (uint32_t)n + raw.c[qq]);
    Gs[qq][nn] = g;
  }
#pragma unroll
  for (int i = 0; i < (kChunkPx * kTL) / kThreads; ++i) {
    const int e = tid + i * kThreads;
    const int qq = e / kTL, ll = e % kTL;
    const int64_t q = q0 + qq;
    const int l = l0 + ll;
    float2 d = make_float2(0.f, 0.f);
    if (q < pv && l < k.L) {
      const float2 w = cis_q32(raw.b[qq] * (uint32_t)l);
      const float2 sg = raw.sig[qq];
      d = make_float2(sg.x * w.x - sg.y * w.y, sg.x * w.y + sg.y * w.x);
    }
    Ds[qq][ll] = d;
  }
}

// One CTA: a TN (n) x 64 (l) tile of one channel over one pixel split.  Each thread
// owns MI = TN / 16 n x 4 l complex outputs.  The phasor tiles are double-buffered, so
// that the next chunk is filled before the barrier that hands it over, and the raw data
// of the chunk after that is copied into shared memory meanwhile (cp.async).
template <int TN>
__global__ void __launch_bounds__(kThreads, 2)
direct_sum(const FrameIO* __restrict__ frames, Consts k, int splits, int units_per_frame,
           int out_dtype) {
  constexpr int MI = TN / 16;
  wait_prior_grid();
  const int f = blockIdx.x / units_per_frame;
  int r = blockIdx.x % units_per_frame;
  const FrameIO& fr = frames[f];
  const int s = r % splits;
  r /= splits;
  const int ntl = (k.L + kTL - 1) / kTL;
  const int ntn = (k.Ns + TN - 1) / TN;
  const int tl_i = r % ntl;
  r /= ntl;
  const int tn_i = r % ntn;
  const int v = r / ntn;
  const int n0 = tn_i * TN, l0 = tl_i * kTL;

  const int64_t pv = (int64_t)fr.meta[0];
  const int64_t nch = (pv + kChunkPx - 1) / kChunkPx;
  const int64_t c0 = nch * s / splits, c1 = nch * (s + 1) / splits;

  extern __shared__ float2 dsm[];  // 2 x (G [32][TN] + D [32][64]), then 2 raw chunks
  constexpr int kBuf = kChunkPx * (TN + kTL);
  auto gbuf = [&](int b) { return reinterpret_cast<float2 (*)[TN]>(dsm + b * kBuf); };
  auto dbuf = [&](int b) { return reinterpret_cast<float2 (*)[kTL]>(dsm + b * kBuf + kChunkPx * TN); };
  RawChunk* raw = reinterpret_cast<RawChunk*>(dsm + 2 * kBuf);

  const int tid = threadIdx.x;
  const int tn = tid >> 4, tl = tid & 15;  // rows tn*MI .. +MI-1 ; cols tl + 16 j
  float2 acc[MI][4];
#pragma unroll
  for (int i = 0; i < MI; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

  const uint32_t* pA = fr.phA + (int64_t)v * fr.Pcap;
  const uint32_t* pC = fr.phC + (int64_t)v * fr.Pcap;

  // raw chunk c sits in raw[(c - c0) & 1]; it is copied two iterations before its fill
  if (c0 < c1) {
    stage_raw(&raw[0], fr, pA, pC, c0 * kChunkPx);
    if (c0 + 1 < c1) stage_raw(&raw[1], fr, pA, pC, (c0 + 1) * kChunkPx);
    if (c0 + 1 < c1)
      wait_raw_but_one();
    else
      wait_raw_all();
    __syncthreads();
    fill_chunk<TN>(gbuf(0), dbuf(0), raw[0], c0 * kChunkPx, pv, n0, l0, k);
    wait_raw_all();
  }
  __syncthreads();
  for (int64_t c = c0; c < c1; ++c) {
    const int b = (int)((c - c0) & 1);
    // raw[b] held chunk c, whose fill finished before the last barrier: chunk c + 2 goes there
    if (c + 2 < c1) stage_raw(&raw[b], fr, pA, pC, (c + 2) * kChunkPx);
    if (c + 1 < c1) fill_chunk<TN>(gbuf(b ^ 1), dbuf(b ^ 1), raw[b ^ 1], (c + 1) * kChunkPx, pv, n0, l0, k);
    const float2 (*G)[TN] = gbuf(b);
    const float2 (*D)[kTL] = dbuf(b);
#pragma unroll 2
    for (int qq = 0; qq < kChunkPx; ++qq) {
      float2 g[MI], d[4];
#pragma unroll
      for (int i = 0; i < MI; i += 2) {
        const float4 t = *reinterpret_cast<const float4*>(&G[qq][tn * MI + i]);
        g[i] = make_float2(t.x, t.y);
        g[i + 1] = make_float2(t.z, t.w);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) d[j] = D[qq][tl + 16 * j];
#pragma unroll
      for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cmac(acc[i][j], g[i], d[j]);
    }
    wait_raw_all();  // chunk c + 2's copies (issued by this thread) have landed
    __syncthreads();
  }

  // write the tile: final cube when there is one split, else this split's partial
  const int64_t rows = (int64_t)k.V * k.Ns;
#pragma unroll
  for (int i = 0; i < MI; ++i) {
    const int n = n0 + tn * MI + i;
    if (n >= k.Ns) continue;
    const int64_t row = (int64_t)v * k.Ns + n;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int l = l0 + tl + 16 * j;
      if (l >= k.L) continue;
      const int64_t o = row * k.L + l;
      if (splits == 1) {
        if (out_dtype == RSIM_C128)
          reinterpret_cast<double2*>(fr.cube)[o] = make_double2(acc[i][j].x, acc[i][j].y);
        else
          reinterpret_cast<float2*>(fr.cube)[o] = acc[i][j];
      } else {
        fr.partial[(int64_t)s * rows * k.L + o] = acc[i][j];
      }
    }
  }
}

}  // namespace

namespace {
template <int TN>
cudaError_t launch_direct_t(const Consts& k, const FrameIO* frames, int F, int splits, int out_dtype,
                            cudaStream_t st) {
  const int ntn = (k.Ns + TN - 1) / TN, ntl = (k.L + kTL - 1) / kTL;
  const int64_t upf = (int64_t)k.V * ntn * ntl * splits;
  const int64_t blocks = upf * F;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffll) return cudaErrorInvalidConfiguration;
  const int smem = (int)sizeof(float2) * 2 * kChunkPx * (TN + kTL) + 2 * (int)sizeof(RawChunk);
  cudaError_t e = cudaFuncSetAttribute(direct_sum<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return launch_dependent(direct_sum<TN>, dim3((unsigned)blocks), dim3(kThreads), (size_t)smem, st, frames, k,
                          splits, (int)upf, out_dtype);
}
}  // namespace

cudaError_t launch_direct(const Consts& k, const FrameIO* frames, int F, int splits, int tile_n,
                          int out_dtype, cudaStream_t st) {
  if (tile_n == 64) return launch_direct_t<64>(k, frames, F, splits, out_dtype, st);
  if (tile_n == 128) return launch_direct_t<128>(k, frames, F, splits, out_dtype, st);
  return cudaErrorInvalidValue;
}

}  // namespace rsim
