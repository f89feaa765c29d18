// FP32 direct sum of Eq. 2 on CUDA cores, and the ordered split reduction.
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

constexpr int kTL = 64;       // l per tile
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

// Phasor tiles of one 32-pixel chunk: G[q][n] = e^{j 2 pi (a n + c)} (channel v),
// D[q][l] = sigma e^{j 2 pi b l}; zero outside the frame / the cube.
template <int TN>
__device__ __forceinline__ void fill_chunk(float2 (*Gs)[TN], float2 (*Ds)[kTL], const FrameIO& fr,
                                           const uint32_t* pA, const uint32_t* pC, int64_t q0,
                                           int64_t pv, int n0, int l0, const Consts& k) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int i = 0; i < (kChunkPx * TN) / kThreads; ++i) {
    const int e = tid + i * kThreads;
    const int qq = e / TN, nn = e % TN;
    const int64_t q = q0 + qq;
    const int n = n0 + nn;
    float2 g = make_float2(0.f, 0.f);
    if (q < pv && n < k.Ns) g = cis_q32(pA[q] * (uint32_t)n + pC[q]);
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
      const float2 w = cis_q32(fr.phB[q] * (uint32_t)l);
      const float2 sg = fr.sig[q];
      d = make_float2(sg.x * w.x - sg.y * w.y, sg.x * w.y + sg.y * w.x);
    }
    Ds[qq][ll] = d;
  }
}

// One CTA: a TN (n) x 64 (l) tile of one channel over one pixel split.  Each thread
// owns MI = TN / 16 n x 4 l complex outputs; the phasor tiles are double-buffered so that
// the next chunk is filled before the barrier that hands it over.
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

  extern __shared__ float2 dsm[];  // 2 x (G [32][TN] + D [32][64])
  constexpr int kBuf = kChunkPx * (TN + kTL);
  auto gbuf = [&](int b) { return reinterpret_cast<float2 (*)[TN]>(dsm + b * kBuf); };
  auto dbuf = [&](int b) { return reinterpret_cast<float2 (*)[kTL]>(dsm + b * kBuf + kChunkPx * TN); };

  const int tid = threadIdx.x;
  const int tn = tid >> 4, tl = tid & 15;  // rows tn*MI .. +MI-1 ; cols tl + 16 j
  float2 acc[MI][4];
#pragma unroll
  for (int i = 0; i < MI; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

  const uint32_t* pA = fr.phA + (int64_t)v * fr.Pcap;
  const uint32_t* pC = fr.phC + (int64_t)v * fr.Pcap;

  if (c0 < c1) fill_chunk<TN>(gbuf(0), dbuf(0), fr, pA, pC, c0 * kChunkPx, pv, n0, l0, k);
  __syncthreads();
  for (int64_t c = c0; c < c1; ++c) {
    const int b = (int)((c - c0) & 1);
    if (c + 1 < c1) fill_chunk<TN>(gbuf(b ^ 1), dbuf(b ^ 1), fr, pA, pC, (c + 1) * kChunkPx, pv, n0, l0, k);
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
  const int smem = (int)sizeof(float2) * 2 * kChunkPx * (TN + kTL);
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

bool uses_partial(int tier, int64_t P, int splits, int group) {
  if (tier == RSIM_TIER_NUFFT) return false;
  if (splits > 1) return true;
  if (tier == RSIM_TIER_FP32) return false;
  const int64_t chunks = (P + kChunkPx - 1) / kChunkPx;
  return chunks > group;
}

int group_chunks(int tier) {
  return (tier == RSIM_TIER_SPLIT_BF16 || tier == RSIM_TIER_SPLIT_FP16) ? 40 : 96;
}

// The split tiers' 2e-5 bar leaves room for the round-toward-zero bias of at most 40
// chunks (480 accumulating MMAs, a relative shrink of about 1e-5); the plain 16-bit tiers
// (1e-2) allow 384 chunks (1536 MMAs, about 3e-5).
int group_chunks_max(int tier) {
  return (tier == RSIM_TIER_SPLIT_BF16 || tier == RSIM_TIER_SPLIT_FP16) ? 40 : 384;
}

int units_per_split(int tier, int V, int Ns, int L, int tile_n) {
  if (tier == RSIM_TIER_FP32) return V * ((Ns + tile_n - 1) / tile_n) * ((L + kTL - 1) / kTL);
  const int64_t rows = (int64_t)V * Ns;
  const int nt = (L + tile_n - 1) / tile_n;
  return (int)(((rows + 127) / 128) * nt);
}

int default_splits(int tier, int V, int Ns, int L, int tile_n, int64_t P, int num_sms) {
  if (tier == RSIM_TIER_NUFFT) return 1;
  const int tiles = units_per_split(tier, V, Ns, L, tile_n);
  const int64_t chunks = (P + kChunkPx - 1) / kChunkPx;
  // keep at least 8 chunks (256 pixels) per split
  int64_t smax = chunks / 8 > 0 ? chunks / 8 : 1;
  if (smax > kMaxSplits) smax = kMaxSplits;
  if (tier == RSIM_TIER_FP32) {
    // FP32 accumulation: at most 8192 pixels per split, so that the running sum of
    // random-phase terms keeps a relative rounding error of a few 1e-6 (the splits are
    // then added with compensated sums); above that, the split count that fills whole
    // waves of two resident CTAs per SM best
    const int64_t smin = std::min<int64_t>(std::max<int64_t>((P + 8191) / 8192, 1), kMaxSplits);
    const int64_t slots = 2ll * num_sms;
    double best = -1.0;
    int64_t bs = smin;
    for (int64_t s = smin; s <= std::max(smin, smax); ++s) {
      const int64_t units = (int64_t)tiles * s;
      const int64_t waves = (units + slots - 1) / slots;
      const double eff = (double)units / (double)(waves * slots) - 0.001 * s;
      if (eff > best + 1e-9) {
        best = eff;
        bs = s;
      }
    }
    return (int)bs;
  }
  // tensor tiers: one persistent CTA per SM takes equal units from a counter; pick the
  // split count whose unit count fills whole rounds of SMs best, with a small cost per
  // split for the partial buffer it adds
  double best = -1.0;
  int bs = 1;
  for (int s = 1; s <= smax; ++s) {
    const int64_t units = (int64_t)tiles * s;
    const int64_t rounds = (units + num_sms - 1) / num_sms;
    const double eff = (double)units / (double)(rounds * num_sms) - 0.003 * s;
    if (eff > best + 1e-9) {
      best = eff;
      bs = s;
    }
  }
  return bs;
}

void resolve_tile(int tier, const Consts& k, rsim_plan* p) {
  if (tier == RSIM_TIER_FP32) {
    if (p->tile_n == 0) p->tile_n = kDirectTileN;
    p->group_chunks = 0;
  } else if (tensor_tier(tier)) {
    if (p->tile_n == 0) p->tile_n = tile_nt(k.L);
    if (p->group_chunks == 0) p->group_chunks = group_chunks(tier);
  } else {
    p->tile_n = 0;
    p->group_chunks = 0;
  }
  p->chunk_px = kChunkPx;
}

rsim_plan default_plan(int tier, const Consts& k, int64_t P, int num_sms) {
  rsim_plan p{};
  resolve_tile(tier, k, &p);
  p.splits = default_splits(tier, k.V, k.Ns, k.L, p.tile_n, P, num_sms);
  return p;
}

std::string plan_problem(int tier, const Consts& k, const rsim_plan& p) {
  if (p.splits < 1 || p.splits > kMaxSplits) return "plan splits must be in 1..64";
  if (p.grid < 0) return "plan grid must be >= 0";
  if (p.variant != 0) return "plan variant must be 0";
  if (tier == RSIM_TIER_FP32) {
    if (p.tile_n != 0 && p.tile_n != 64 && p.tile_n != 128) return "FP32 tile_n must be 64 or 128";
  } else if (tensor_tier(tier)) {
    const int lmax = std::max(8, (k.L + 7) / 8 * 8);
    if (p.tile_n != 0 && (p.tile_n < 8 || p.tile_n > 128 || p.tile_n % 8 != 0 || p.tile_n > lmax))
      return "tensor-core tile_n must be a multiple of 8 in 8..min(128, L rounded up to 8)";
    if (p.group_chunks < 0 || p.group_chunks > group_chunks_max(tier))
      return "group_chunks must be in 1.." + std::to_string(group_chunks_max(tier)) + " for this tier";
  }
  return std::string();
}

}  // namespace rsim
