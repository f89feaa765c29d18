// NUFFT tier: the sum of Eq. 2 through a two-dimensional type-1 non-uniform FFT per
// virtual channel.  With the fixed-point path phases of the compaction kernel,
//
//   cube[v][n][l] = sum_p q_p exp(j 2 pi (x_p n + y_p l)),
//   x_p = a_{p,v} (2 mu R_{p,v} / (c F_s), cycles per sample),  y_p = b_p (-f_D T_slow),
//   q_p = sigma_p exp(j 2 pi c_{p,v})   (spatial and TDM phases).
//
// Centred modes n = n' + s_x, l = l' + s_y move the shift into the strengths,
// q'_p = q_p exp(j 2 pi (x_p s_x + y_p s_y)).  Each q'_p is spread onto a periodic grid of
// G_x x G_y cells (powers of two >= 2 N_s, 2 L, and >= 16) with the "exponential of
// semicircle" kernel of Barnett, Magland and af Klinteberg (SIAM J. Sci. Comput. 41,
// 2019), psi(t) = exp(beta (sqrt(1 - (2t/w)^2) - 1)), width w = 4..8 cells (7 by default),
// beta = 2.30 w; the grid's inverse-sign DFT at the centred modes, divided by the kernel's
// Fourier transform Psi_x(n') Psi_y(l'), is the cube (relative error ~10^-(w-1): ~1e-6
// at w = 7).
//
// Kernels, per frame:
//   nu_bin_count  each (channel, point) is binned by the 32 x 32 grid tile of its
//                 nearest cell: a shared-memory histogram per block of one channel's
//                 points, one global addition per (block, bin).  An extra row of blocks
//                 builds the geometry's tables: 1 / (Psi_x(n') Psi_y(l')) (one warp per
//                 mode, a 128-node midpoint rule of Psi(k) = (w/2) int phi(z) cos(pi k w z
//                 / G) dz) and the twiddles of both FFTs.  The last counting block scans
//                 the counts and cuts every bin into work items of 512 records;
//   nu_bin_fill   records (x, y, q') stored bin by bin (one global reservation per
//                 (block, bin), ranks within the block from shared memory);
//   nu_spread     persistent CTAs take the work items in turn; a warp takes one record
//                 at a time, lane k adding tap k of its w x w taps into a shared-memory tile
//                 with a w/2 halo, as fixed-point integers (each term split in
//                 16-bit halves summed by non-returning 32-bit atomics), then the tile is
//                 added into the global 64-bit integer grid.  Integer sums are exact and do
//                 not depend on the order of the atomic additions, so the result is
//                 bit-reproducible.  The work items share the crowded tiles among many SMs:
//                 a scene fills only the part of the grid that its ranges and speeds reach;
//   nu_fft_y      rows of the grid: integer -> float, Stockham inverse-sign FFT over the
//                 slow-time axis (radix-16 passes in registers, shared memory between
//                 passes), only the L centred modes kept;
//   nu_fft_x      columns: the same over the fast-time axis, only the N_s centred modes
//                 kept, times the deconvolution factors, written to the cube.
#include <math.h>

#include <algorithm>

#include "rsim_internal.h"

namespace rsim {
namespace {

constexpr int kNWMin = 4, kNWMax = 8;       // kernel widths in cells (the default is 7)
constexpr float kNBetaPerW = 2.30f;         // ES shape beta = 2.30 w for an oversampling of 2
constexpr int kNTile = 32;                  // grid cells per tile side
constexpr int kNQuad = 128;                 // midpoint nodes for Psi
constexpr int kSpreadChunk = 512;           // records per spreading work item
constexpr int kBinThreads = 256;            // binning blocks: one channel, kBinItems points
constexpr int kBinItems = 4 * kBinThreads;
static_assert(kBinThreads % 32 == 0 && kBinThreads <= 1024, "binning blocks are whole warps");

struct NuRec {
  uint32_t x, y;  // positions, 2^-32 cycles
  float2 q;       // shifted strength q'
};

// FFT of length n = 2^k (16 <= n <= 4096) along one grid axis: T = n / 16 threads per
// sequence, S sequences per CTA, each in a shared-memory buffer of `pitch` float2;
// passes of radix 16 then one of 2, 4, 8 or 16; twiddles of pass p (p >= 1) at
// twoff[p], radix[p] x ns[p] entries.
struct FftPlan {
  int n, T, S, pitch, passes;
  int radix[3], ns[3], twoff[3];
  int tw_size;
};

// exp(beta (sqrt(1 - z^2) - 1)) on |z| <= 1, 0 outside
__device__ __forceinline__ float es_kernel(float z, float beta) {
  const float z2 = z * z;
  return z2 < 1.f ? expf(beta * (sqrtf(1.f - z2) - 1.f)) : 0.f;
}

// The same with the hardware exponential and reciprocal square root, for the spreading
// weights: sqrt(x) = x rsqrt(x) for x = 1 - z^2 in (0, 1]; a few ulp per weight, far below
// the kernel's own truncation error (the deconvolution factors keep es_kernel).
__device__ __forceinline__ float es_kernel_fast(float z, float beta) {
  const float x = 1.f - z * z;
  return x > 0.f ? __expf(beta * (x * rsqrtf(x) - 1.f)) : 0.f;
}

// Nearest grid cell of a position (mod G, G a power of two) and the offset of the
// position from it, in [-1/2, 1/2) cells: X = xq G / 2^32.
__device__ __forceinline__ void nearest_cell(uint32_t xq, int G, int& c, float& d) {
  const uint64_t s = (uint64_t)xq * (uint64_t)G + 0x80000000ull;  // (X + 1/2) in 2^-32 cells
  c = (int)(s >> 32) & (G - 1);
  d = (float)(uint32_t)s * 2.3283064365386963e-10f - 0.5f;  // frac(X + 1/2) - 1/2
}

// Channel-local bin (tile) of a point's nearest cell.
__device__ __forceinline__ int bin_of(uint32_t xq, uint32_t yq, const NuGeo& g) {
  int cx, cy;
  float d;
  nearest_cell(xq, g.Gx, cx, d);
  nearest_cell(yq, g.Gy, cy, d);
  return (cx / g.Tx) * g.nty + cy / g.Ty;
}

// int64 -> float from 32-bit conversions of |v| (64-bit conversions run on the slow
// double-precision path): exact rounding below 2^32, within one more rounding above.
__device__ __forceinline__ float ll_to_float(long long v) {
  const unsigned long long u = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const float f = fmaf((float)(unsigned)(u >> 32), 4294967296.f, (float)(unsigned)(u & 0xffffffffull));
  return v < 0 ? -f : f;
}

// Fixed-point scale of the integer grid: every term |q' psi psi| <= sqrt(2) max|sigma|
// becomes an integer below 2^31 in magnitude (2^30 / max|sigma|), and a cell sums at
// most P_valid < 2^31 terms, so the 64-bit sums cannot overflow.
__device__ __forceinline__ float grid_scale(const FrameIO& fr, bool inverse) {
  const float m = __uint_as_float((unsigned)fr.meta[1]);
  if (!(m > 0.f)) return inverse ? 0.f : 1.f;
  return inverse ? ldexpf(m, -30) : ldexpf(1.f, 30) / m;
}

// Add a 32-bit signed term v to a sum kept as two 32-bit words with non-returning
// atomics: `lo` takes v itself (wrapping mod 2^32) and `hi` its signed high part
// v >> 16.  With H = sum of (v >> 16) and LO = sum of v mod 2^32, the sum of the low
// halves v & 0xffff is (LO - H 2^16) mod 2^32, and the exact sum is H 2^16 plus that
// (join_split), while a word receives fewer than 2^16 terms (a work item holds
// kSpreadChunk records, each adding once per cell): then |H| < 2^31 and the low halves
// sum below 2^32.
__device__ __forceinline__ void add_split(unsigned* lo, int* hi, int v) {
  atomicAdd(lo, (unsigned)v);
  atomicAdd(hi, v >> 16);
}
__device__ __forceinline__ long long join_split(unsigned lo, int hi) {
  const unsigned low_halves = lo - ((unsigned)hi << 16);
  return (long long)hi * 65536ll + (long long)low_halves;
}

// Twiddle e of an FFT plan: entry j ns + k of pass p is exp(+j 2 pi j k / (ns R)).
__device__ void plan_twiddle(const FftPlan& pl, int e, float2* __restrict__ tw) {
  for (int p = 1; p < pl.passes; ++p) {
    const int size = pl.radix[p] * pl.ns[p];
    if (e < pl.twoff[p] + size) {
      const int r = e - pl.twoff[p], j = r / pl.ns[p], k = r % pl.ns[p];
      float sn, cs;
      sincospif((float)(2 * j * k) / (float)size, &sn, &cs);  // exact argument: size is a power of two
      tw[e] = make_float2(cs, sn);
      return;
    }
  }
}

// Tables of one frame's geometry, in blocks of kBinThreads threads numbered vb: blocks
// [0, psi_blocks) give the deconvolution factors (one warp per mode), the blocks after
// them the twiddle tables of both FFT plans.
struct NuTables {
  int psi_blocks, blocks;
  FftPlan plx, ply;
  float *inv_x, *inv_y;
  float2 *twx, *twy;
};

__device__ void table_block(const NuGeo& g, const NuTables& tb, int vb) {
  const FftPlan& plx = tb.plx;
  const FftPlan& ply = tb.ply;
  float* __restrict__ inv_x = tb.inv_x;
  float* __restrict__ inv_y = tb.inv_y;
  if (vb >= tb.psi_blocks) {
    const int e = (vb - tb.psi_blocks) * blockDim.x + threadIdx.x;
    float2* __restrict__ twx = tb.twx;
    float2* __restrict__ twy = tb.twy;
    if (e < plx.tw_size)
      plan_twiddle(plx, e, twx);
    else if (e - plx.tw_size < ply.tw_size)
      plan_twiddle(ply, e - plx.tw_size, twy);
    return;
  }
  const int warp = (vb * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= g.Ns + g.L) return;
  const bool xs = warp < g.Ns;
  const int k = xs ? warp - g.sx : (warp - g.Ns) - g.sy;
  const float G = (float)(xs ? g.Gx : g.Gy);
  float s = 0.f;
  for (int j = lane; j < kNQuad; j += 32) {
    const float z = -1.f + ((float)j + 0.5f) * (2.f / kNQuad);
    s += es_kernel(z, g.beta) * cospif((float)k * (float)g.W * z / G);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const float psi = 0.5f * (float)g.W * (2.f / kNQuad) * s;
    if (xs)
      inv_x[warp] = 1.f / psi;
    else
      inv_y[warp - g.Ns] = 1.f / psi;
  }
}

// Spreading work items of a frame: bin offsets and cursors, and the item table
// (item_bin[i] the bin of item i, item_first[i] its first record, items[0] their number).
struct NuItems {
  int *off, *cursor, *items, *item_bin, *item_first;
};

// Exclusive scan of n bin counts by one block into `off` and `cursor`, and of their chunk
// counts into the work-item table.  The counts were added by other blocks' atomics, so
// they are read from L2.
__device__ void scan_bins(const int* __restrict__ count, int n, const NuItems& it) {
  __shared__ int wsum[32], wcsum[32];
  const int nt = blockDim.x, nw = nt >> 5;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int per = (n + nt - 1) / nt;
  const int b0 = min(n, t * per), b1 = min(n, b0 + per);
  int* __restrict__ off = it.off;
  int* __restrict__ cursor = it.cursor;
  int* __restrict__ item_bin = it.item_bin;
  int* __restrict__ item_first = it.item_first;
  // counts in batches of 8 loads issued together (the first batch kept for the second pass)
  constexpr int kBatch = 8;
  int first[kBatch];
  int s = 0, c = 0;
  for (int b = b0; b < b1; b += kBatch) {
    int kk[kBatch];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) kk[j] = b + j < b1 ? __ldcg(count + b + j) : 0;
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      s += kk[j];
      c += (kk[j] + kSpreadChunk - 1) / kSpreadChunk;
      if (b == b0) first[j] = kk[j];
    }
  }
  // inclusive scans of the records and the chunks: within warps, then over the warp sums
  int si = s, ci = c;
  for (int o = 1; o < 32; o <<= 1) {
    const int x = __shfl_up_sync(0xffffffffu, si, o), y = __shfl_up_sync(0xffffffffu, ci, o);
    if (lane >= o) {
      si += x;
      ci += y;
    }
  }
  if (lane == 31) {
    wsum[w] = si;
    wcsum[w] = ci;
  }
  __syncthreads();
  if (w == 0) {
    int a = lane < nw ? wsum[lane] : 0, bb = lane < nw ? wcsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int x = __shfl_up_sync(0xffffffffu, a, o), y = __shfl_up_sync(0xffffffffu, bb, o);
      if (lane >= o) {
        a += x;
        bb += y;
      }
    }
    wsum[lane] = a;
    wcsum[lane] = bb;
  }
  __syncthreads();
  int run = (w ? wsum[w - 1] : 0) + si - s, crun = (w ? wcsum[w - 1] : 0) + ci - c;
  for (int b = b0; b < b1; b += kBatch) {
    int kk[kBatch];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) kk[j] = b == b0 ? first[j] : (b + j < b1 ? __ldcg(count + b + j) : 0);
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      if (b + j >= b1) break;
      off[b + j] = run;
      cursor[b + j] = run;
      for (int q = 0; q < kk[j]; q += kSpreadChunk, ++crun) {
        item_bin[crun] = b + j;
        item_first[crun] = run + q;
      }
      run += kk[j];
    }
  }
  if (t == nt - 1) {
    off[n] = wsum[nw - 1];
    it.items[0] = wcsum[nw - 1];
  }
}

// Binning blocks: blockIdx.y = channel, blockIdx.x = a range of kBinItems points.  The row
// blockIdx.y = V builds the geometry's tables.  The last counting block to finish (a
// ticket taken after its counts are visible: count[nbins]) scans the counts into the work
// items, so no block waits for another.
__global__ void __launch_bounds__(kBinThreads) nu_bin_count(const FrameIO* __restrict__ fp, NuGeo g,
                                                            int* __restrict__ count, NuTables tb, NuItems it) {
  wait_prior_grid();
  if ((int)blockIdx.y == g.V) {
    for (int vb = blockIdx.x; vb < tb.blocks; vb += gridDim.x) table_block(g, tb, vb);
    return;
  }
  extern __shared__ int hist[];  // this channel's bins
  const int nb = g.ntx * g.nty, v = blockIdx.y;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  const FrameIO& fr = *fp;
  const int64_t pv = (int64_t)fr.meta[0];
  const int64_t p0 = (int64_t)blockIdx.x * kBinItems;
  const int64_t p1 = pv < p0 + kBinItems ? pv : p0 + kBinItems;
  for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x)
    atomicAdd(&hist[bin_of(fr.phA[(int64_t)v * fr.Pcap + p], fr.phB[p], g)], 1);
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    if (hist[b]) atomicAdd(&count[v * nb + b], hist[b]);
  __shared__ int ticket;
  __threadfence();
  __syncthreads();
  const int nbins = g.V * nb;
  if (threadIdx.x == 0) ticket = atomicAdd(&count[nbins], 1);
  __syncthreads();
  if (ticket != (int)(gridDim.x * g.V) - 1) return;
  __threadfence();
  scan_bins(count, nbins, it);
}

__global__ void __launch_bounds__(kBinThreads) nu_bin_fill(const FrameIO* __restrict__ fp, NuGeo g,
                                                           int* __restrict__ cursor, NuRec* __restrict__ rec) {
  wait_prior_grid();
  extern __shared__ int hist[];  // [nb] counts in this block, then [nb] reserved bases
  const int nb = g.ntx * g.nty, v = blockIdx.y;
  int* base = hist + nb;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  const FrameIO& fr = *fp;
  const int64_t pv = (int64_t)fr.meta[0];
  const int64_t p0 = (int64_t)blockIdx.x * kBinItems;
  constexpr int kPer = kBinItems / kBinThreads;
  // this thread's points: every load issued before the first use
  uint32_t xq[kPer], yq[kPer], cq[kPer];
  float2 sg[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int64_t p = p0 + threadIdx.x + (int64_t)i * blockDim.x;
    const bool in = p < pv;
    xq[i] = in ? fr.phA[(int64_t)v * fr.Pcap + p] : 0u;
    yq[i] = in ? fr.phB[p] : 0u;
    cq[i] = in ? fr.phC[(int64_t)v * fr.Pcap + p] : 0u;
    sg[i] = in ? fr.sig[p] : make_float2(0.f, 0.f);
  }
  int bins[kPer], rank[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int64_t p = p0 + threadIdx.x + (int64_t)i * blockDim.x;
    bins[i] = -1;
    rank[i] = 0;
    if (p < pv) {
      bins[i] = bin_of(xq[i], yq[i], g);
      rank[i] = atomicAdd(&hist[bins[i]], 1);
    }
  }
  // q' = sigma exp(j 2 pi (c + x s_x + y s_y)), the phase exact mod 1 in 2^-32 cycles
  float2 q[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const uint32_t ph = cq[i] + xq[i] * (uint32_t)g.sx + yq[i] * (uint32_t)g.sy;
    float sn, cs;
    sincospif((float)(int32_t)ph * 4.656612873077393e-10f, &sn, &cs);  // angle pi ph / 2^31
    q[i] = make_float2(sg[i].x * cs - sg[i].y * sn, sg[i].x * sn + sg[i].y * cs);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) base[b] = hist[b] ? atomicAdd(&cursor[v * nb + b], hist[b]) : 0;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    if (bins[i] < 0) continue;
    NuRec r;
    r.x = xq[i];
    r.y = yq[i];
    r.q = q[i];
    rec[base[bins[i]] + rank[i]] = r;
  }
}

// Spreading layout for a kernel of width W.  A warp takes one record at a time and lane k
// owns tap k = W jx + jy (lanes 0..31, then W^2 - 32 more on a second pass for W >= 6).
// A point's taps are the W cells whose centres lie within W/2 of it: for odd W the nearest
// cell and (W - 1)/2 on each side, for even W the start also follows the side of the
// nearest cell's centre the point lies on; the tile halo is H = W/2 cells.  With a tile row
// stride of W + 32 words (W mod 32) a record's taps lie on consecutive banks, so each
// atomic instruction is one shared-memory wavefront.  Lanes past the last tap add zero at
// word base + lane, on banks no active lane of the pass uses.  The weights are computed
// once per record (one lane per record) and staged per warp: (q'_re, q'_im) psi_x by jx,
// psi_y by jy.  All of it sits in dynamic shared memory:
//   [lo re | lo im | hi re | hi im] tile words, then the staging, then a zero row.
constexpr int kSpreadThreads = 512;
constexpr int kSpreadWarps = kSpreadThreads / 32;
constexpr int kSpreadBlocksPerSm = 3;  // persistent CTAs per SM (about 70 KB of shared memory each at w = 7)
constexpr int kStageLd = 33;           // staged values of 32 records per jx (or jy), padded

template <int W>
struct SpreadLayout {
  static constexpr int H = W / 2;                         // halo cells
  static constexpr int PAD = kNTile + 2 * H;              // padded tile side
  static constexpr int STRIDE = W + 32;                   // tile row stride, W (mod 32)
  static constexpr int WORDS = (PAD * STRIDE + 3) / 4 * 4;  // one tile array, 16-byte words
  static constexpr bool TWO = W * W > 32;                 // a second pass of lanes
  static constexpr size_t kTiles = 4 * sizeof(unsigned) * WORDS;
  static constexpr size_t kAx = sizeof(float2) * kSpreadWarps * W * kStageLd;
  static constexpr size_t kWy = sizeof(float) * kSpreadWarps * W * kStageLd;
  static constexpr size_t kBase = sizeof(int) * kSpreadWarps * 32;
  static constexpr size_t kZero = sizeof(float2) * kStageLd;
  static constexpr size_t bytes = kTiles + kAx + kWy + kBase + kZero;
  static_assert(STRIDE >= PAD && STRIDE % 32 == W, "tile row stride");
  static_assert(W * W <= 64, "two passes of 32 lanes cover the taps");
  // a spare lane's word base + lane stays inside the tile array
  static_assert((PAD - W) * STRIDE + (PAD - W) + 31 < WORDS, "spare-lane words in range");
};

// Persistent CTAs take the work items in turn (their number is known on the device only).
template <int W>
__global__ void __launch_bounds__(kSpreadThreads, kSpreadBlocksPerSm) nu_spread(const FrameIO* __restrict__ fp, NuGeo g,
                                                            const int* __restrict__ off,
                                                            const int* __restrict__ items,
                                                            const int* __restrict__ item_bin,
                                                            const int* __restrict__ item_first,
                                                            const NuRec* __restrict__ rec,
                                                            unsigned long long* __restrict__ grid,
                                                            int* __restrict__ row_used) {
  using Lay = SpreadLayout<W>;
  constexpr int H = Lay::H, PAD = Lay::PAD, STRIDE = Lay::STRIDE, WORDS = Lay::WORDS;
  constexpr float beta = kNBetaPerW * W, k2w = 2.f / (float)W;
  wait_prior_grid();
  extern __shared__ __align__(16) unsigned char smem_sp[];
  unsigned* lo_re = reinterpret_cast<unsigned*>(smem_sp);
  unsigned* lo_im = lo_re + WORDS;
  int* hi_re = reinterpret_cast<int*>(lo_im + WORDS);
  int* hi_im = hi_re + WORDS;
  float2(*s_ax)[W][kStageLd] = reinterpret_cast<float2(*)[W][kStageLd]>(smem_sp + Lay::kTiles);
  float(*s_wy)[W][kStageLd] = reinterpret_cast<float(*)[W][kStageLd]>(smem_sp + Lay::kTiles + Lay::kAx);
  int(*s_base)[32] = reinterpret_cast<int(*)[32]>(smem_sp + Lay::kTiles + Lay::kAx + Lay::kWy);
  float2* s_zero = reinterpret_cast<float2*>(smem_sp + Lay::kTiles + Lay::kAx + Lay::kWy + Lay::kBase);
  for (int i = threadIdx.x; i < kStageLd; i += blockDim.x) s_zero[i] = make_float2(0.f, 0.f);
  const int n_items = items[0];
  const int nb = g.ntx * g.nty;
  const float scale = grid_scale(*fp, false);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // This lane's taps on the two passes (a spare lane: the zero row, word base + lane).
  const bool act0 = lane < W * W;
  const int jx0 = act0 ? lane / W : 0, jy0 = act0 ? lane % W : 0;
  const int off0 = act0 ? jx0 * STRIDE + jy0 : lane;
  const bool act1 = lane + 32 < W * W;
  const int jx1 = act1 ? (lane + 32) / W : 0, jy1 = act1 ? (lane + 32) % W : 0;
  const int off1 = act1 ? jx1 * STRIDE + jy1 : off0;
  const float2* ax0 = act0 ? s_ax[warp][jx0] : s_zero;
  const float2* ax1 = act1 ? s_ax[warp][jx1] : s_zero;
  const float* wy0 = s_wy[warp][jy0];
  const float* wy1 = s_wy[warp][jy1];
  const int* sb = s_base[warp];
  auto pass = [&](int base, float2 a, float w, int offs) {
    const int at = base + offs;
    add_split(&lo_re[at], &hi_re[at], __float2int_rn(a.x * w));
    add_split(&lo_im[at], &hi_im[at], __float2int_rn(a.y * w));
  };
  auto taps = [&](int r) {
    const int base = sb[r];
    pass(base, ax0[r], wy0[r], off0);
    if (Lay::TWO) pass(base, ax1[r], wy1[r], off1);
  };
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int bin = item_bin[item];
    const int v = bin / nb, ty = (bin % nb) % g.nty, tx = (bin % nb) / g.nty;
    const int r_begin = item_first[item];
    const int r_end = min(off[bin + 1], r_begin + kSpreadChunk);
    // the grid rows this item adds to (the padded tile's, mod G_x): the row pass skips
    // rows that no item marks, which hold zeros only
    for (int r = threadIdx.x; r < PAD; r += blockDim.x)
      row_used[(int64_t)v * g.Gx + ((tx * g.Tx - H + r) & (g.Gx - 1))] = 1;
    for (int i = threadIdx.x; i < WORDS; i += blockDim.x)  // 4 arrays of WORDS / 4 16-byte words
      reinterpret_cast<uint4*>(smem_sp)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    for (int r0 = r_begin + warp * 32; r0 < r_end; r0 += kSpreadThreads) {
      const int n = min(32, r_end - r0);
      if (lane < n) {
        const NuRec q = rec[r0 + lane];
        int cx, cy;
        float dx, dy;
        nearest_cell(q.x, g.Gx, cx, dx);
        nearest_cell(q.y, g.Gy, cy, dy);
        // first tap relative to the nearest cell
        const int sx = (W & 1) ? -(W - 1) / 2 : -W / 2 + (dx >= 0.f ? 1 : 0);
        const int sy = (W & 1) ? -(W - 1) / 2 : -W / 2 + (dy >= 0.f ? 1 : 0);
        // the nearest cell lies in this tile: local padded coordinates of the first tap
        const int lx = cx - tx * g.Tx + H + sx, ly = cy - ty * g.Ty + H + sy;
        const float qr = q.q.x * scale, qi = q.q.y * scale;
        // tap j sits at z = (s + j - d) 2 / W in kernel units
        const float zx0 = ((float)sx - dx) * k2w, zy0 = ((float)sy - dy) * k2w;
        // the hardware exponential's few-ulp error sets an error floor near 1e-6, below the
        // kernel's own error for w <= 7; the widest kernel (w = 8, chosen for accuracy)
        // keeps the library functions
#pragma unroll
        for (int j = 0; j < W; ++j) {
          const float zx = fmaf((float)j, k2w, zx0), zy = fmaf((float)j, k2w, zy0);
          const float wx = W >= 8 ? es_kernel(zx, beta) : es_kernel_fast(zx, beta);
          s_ax[warp][j][lane] = make_float2(qr * wx, qi * wx);
          s_wy[warp][j][lane] = W >= 8 ? es_kernel(zy, beta) : es_kernel_fast(zy, beta);
        }
        s_base[warp][lane] = lx * STRIDE + ly;
      }
      __syncwarp();
      int r = 0;
      for (; r + 1 < n; r += 2) {
        taps(r);
        taps(r + 1);
      }
      if (r < n) taps(r);
      __syncwarp();
    }
    __syncthreads();
    const int x0 = tx * g.Tx - H, y0 = ty * g.Ty - H;  // padded tile origin (cells)
    const int64_t gbase = (int64_t)v * g.Gx * g.Gy;
    for (int i = threadIdx.x; i < PAD * PAD; i += blockDim.x) {
      const int row = i / PAD, col = i % PAD, at = row * STRIDE + col;
      const long long re = join_split(lo_re[at], hi_re[at]);
      const long long im = join_split(lo_im[at], hi_im[at]);
      if (re == 0 && im == 0) continue;
      const int gx = (x0 + row) & (g.Gx - 1), gy = (y0 + col) & (g.Gy - 1);
      unsigned long long* cell = grid + 2 * (gbase + (int64_t)gx * g.Gy + gy);
      atomicAdd(cell, (unsigned long long)re);
      atomicAdd(cell + 1, (unsigned long long)im);
    }
    __syncthreads();  // the tile is read before the next item clears it
  }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
  return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}

// exp(+j 2 pi m / 16) for 0 <= m < 8: cosines and sines of multiples of pi / 8
__device__ __forceinline__ float2 unit16(int m) {
  constexpr float c1 = 0.92387953251128676f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
  switch (m) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return make_float2(c1, s1);
    case 2: return make_float2(h, h);
    case 3: return make_float2(s1, c1);
    case 4: return make_float2(0.f, 1.f);
    case 5: return make_float2(-s1, c1);
    case 6: return make_float2(-h, h);
    default: return make_float2(-c1, s1);
  }
}

__host__ __device__ constexpr int rev_bits(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}

__host__ __device__ constexpr int log2_c(int r) { return r <= 1 ? 0 : 1 + log2_c(r >> 1); }

// In-register inverse-sign DFT of R <= 16 points, natural order in and out:
// A_m = sum_j a_j exp(+j 2 pi j m / R), by radix-2 decimation in time.
template <int R>
__device__ __forceinline__ void dft_inv(float2 (&a)[R]) {
  constexpr int bits = log2_c(R);
  float2 b[R];
#pragma unroll
  for (int i = 0; i < R; ++i) b[rev_bits(i, bits)] = a[i];
#pragma unroll
  for (int h = 1; h < R; h <<= 1) {
#pragma unroll
    for (int i0 = 0; i0 < R; i0 += 2 * h) {
#pragma unroll
      for (int k = 0; k < h; ++k) {
        const int m = k * (8 / h);  // exp(+j 2 pi k / (2 h)) = unit16(k 16 / (2 h))
        const float2 u = b[i0 + k];
        float2 t = b[i0 + k + h];
        if (m == 4)
          t = make_float2(-t.y, t.x);
        else if (m != 0)
          t = cmul(t, unit16(m));
        b[i0 + k] = make_float2(u.x + t.x, u.y + t.y);
        b[i0 + k + h] = make_float2(u.x - t.x, u.y - t.y);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) a[i] = b[i];
}

// One radix-R pass of a Stockham (self-sorting) inverse-sign FFT of length n; every thread
// holds kFftPer = 16 values, i.e. 16 / R butterflies.  Butterfly b reads inputs
// j < R at b + j n / R, multiplies input j by exp(+j 2 pi j k / (Ns R)) with k = b mod Ns
// (Ns the product of the earlier radices; tw[j Ns + k] holds that factor), takes the R-point
// DFT and writes output m to (b / Ns) Ns R + k + m Ns.  After the last pass the sequence
// is its DFT in natural order.  sync_mid: loads and stores share the buffer.
constexpr int kFftPer = 16;

template <int R, class Load, class Store>
__device__ __forceinline__ void fft_pass(int n, int ns, int t, int T, const float2* __restrict__ tw, bool sync_mid,
                                         Load load, Store store) {
  constexpr int G = kFftPer / R;
  const int nr = n / R;
  float2 a[G][R];
#pragma unroll
  for (int gi = 0; gi < G; ++gi) {
    const int b = t + gi * T;
    const int k = b & (ns - 1);
#pragma unroll
    for (int j = 0; j < R; ++j) {
      float2 x = load(b + j * nr);
      if (j > 0 && ns > 1) x = cmul(x, tw[j * ns + k]);
      a[gi][j] = x;
    }
    dft_inv<R>(a[gi]);
  }
  if (sync_mid) __syncthreads();
#pragma unroll
  for (int gi = 0; gi < G; ++gi) {
    const int b = t + gi * T;
    const int k = b & (ns - 1);
    const int o = (b - k) * R + k;
#pragma unroll
    for (int m = 0; m < R; ++m) store(o + m * ns, a[gi][m]);
  }
}

// All passes of one FFT per sequence, P passes (radix 16, then RL last), from the
// sequence's input `in` (element i at in[i]) to its shared-memory buffer x (element i at
// i + i / 16, so that the stride-16 stores of the first pass fall on distinct banks); the
// transform ends in x, in natural order.  The buffers may overlap the input: the first pass
// holds all its inputs in registers before the block stores anything.  Each (P, RL) is its own kernel, so that a kernel
// holds only the passes it runs.
template <int P, int RL, class In>
__device__ __forceinline__ void fft_all(const FftPlan& pl, const In& in, float2* x, int t,
                                        const float2* __restrict__ tw) {
  static_assert(P > 1 || RL == 16, "a single pass is one radix-16 butterfly");
  auto sload = [=](int i) -> float2 { return x[i + (i >> 4)]; };
  auto sstore = [=](int i, float2 v) { x[i + (i >> 4)] = v; };
  float2 a[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) a[j] = in(t + j * pl.T);
  __syncthreads();  // the buffers overlap the input rows
  dft_inv<16>(a);  // the first pass has Ns = 1: no twiddles, output m at 16 t + m
#pragma unroll
  for (int m = 0; m < 16; ++m) sstore(16 * t + m, a[m]);
  if constexpr (P > 1) {
    __syncthreads();
    if constexpr (P == 3) {
      fft_pass<16>(pl.n, 16, t, pl.T, tw + pl.twoff[1], true, sload, sstore);
      __syncthreads();
    }
    fft_pass<RL>(pl.n, pl.ns[P - 1], t, pl.T, tw + pl.twoff[P - 1], true, sload, sstore);
  }
  __syncthreads();
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

constexpr unsigned long long kNuWaitNs = 2000000000ull;  // 2 s for a copy, then give up

// One CTA's input rows: a single bulk copy (TMA) global -> shared of `bytes` (a multiple of
// 16, both addresses 16-byte aligned), completing the barrier's transaction count.  Every
// thread waits, bounded: on a timeout the status word gets kStatusTimeout and the copy is
// waited for once more (bounded too).  The block agrees on the outcome: false, and every
// thread returns, if any thread timed out.
__device__ bool load_rows(void* dst, const void* src, uint32_t bytes, uint64_t* bar, unsigned* status) {
  if (threadIdx.x == 0) mbar_init_single(bar);
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
  }
  bool ok = wait_phase_bounded(bar, 0, kNuWaitNs);
  if (!ok) {
    atomicOr(status, kStatusTimeout);
    wait_phase_bounded(bar, 0, kNuWaitNs);  // the copy may still be in flight
  }
  return !__syncthreads_or(!ok);
}

// Dynamic shared memory of an FFT kernel: the CTA's raw input rows, overlapped by the S
// transform buffers (whichever is larger), then the copy barrier.
__host__ __device__ inline int fft_smem_in_bytes(const FftPlan& pl, int elem) { return (pl.S * pl.n * elem + 127) / 128 * 128; }
__host__ __device__ inline int fft_smem_bytes(const FftPlan& pl, int elem) {
  const int buf = (pl.S * pl.pitch * 8 + 15) / 16 * 16;
  const int in = fft_smem_in_bytes(pl, elem);
  return (in > buf ? in : buf) + 16;
}

// Rows (v, mx) of the grid, pl.S consecutive rows per CTA, one bulk copy: integer -> float,
// FFT over my, the L centred modes kept and written as midT[v][l][mx] (column-major rows), so
// that the column pass reads its columns as contiguous rows.
template <int P, int RL>
__global__ void nu_fft_y(const FrameIO* __restrict__ fp, NuGeo g, FftPlan pl, const float2* __restrict__ tw,
                         const long long* __restrict__ grid, float2* __restrict__ midT,
                         const int* __restrict__ row_used, unsigned* status) {
  wait_prior_grid();
  extern __shared__ __align__(128) unsigned char smem_y[];
  const longlong2* raw = reinterpret_cast<const longlong2*>(smem_y);
  float2* buf = reinterpret_cast<float2*>(smem_y);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_y + fft_smem_bytes(pl, 16) - 16);
  const int64_t rows = (int64_t)g.V * g.Gx, row0 = (int64_t)blockIdx.x * pl.S;
  const int live_rows = (int)min((int64_t)pl.S, rows - row0);
  // rows no spreading item touched are zero, and so is their transform: no copy, no FFT
  if (!__syncthreads_or((int)threadIdx.x < live_rows && row_used[row0 + threadIdx.x] != 0)) {
    for (int e = threadIdx.x; e < pl.S * g.L; e += blockDim.x) {
      const int rs = e % pl.S, l = e / pl.S;
      if (rs >= live_rows) continue;
      const int64_t row = row0 + rs, v = row / g.Gx, mx = row % g.Gx;
      midT[(v * g.L + l) * g.Gx + mx] = make_float2(0.f, 0.f);
    }
    return;
  }
  if (!load_rows(smem_y, grid + 2 * row0 * g.Gy, (uint32_t)(live_rows * g.Gy * 16), bar, status)) return;
  const int t = threadIdx.x % pl.T, s = threadIdx.x / pl.T;
  const float inv = grid_scale(*fp, true);
  const longlong2* src = raw + (int64_t)s * g.Gy;
  const bool live = s < live_rows;
  auto in = [=](int i) -> float2 {
    if (!live) return make_float2(0.f, 0.f);
    const longlong2 c = src[i];
    return make_float2(ll_to_float(c.x) * inv, ll_to_float(c.y) * inv);
  };
  fft_all<P, RL>(pl, in, buf + s * pl.pitch, t, tw);
  // midT[v][l][mx]: consecutive threads take consecutive rows of one l
  for (int e = threadIdx.x; e < pl.S * g.L; e += blockDim.x) {
    const int rs = e % pl.S, l = e / pl.S;
    if (rs >= live_rows) continue;
    const int i = (l - g.sy) & (g.Gy - 1);
    const int64_t row = row0 + rs, v = row / g.Gx, mx = row % g.Gx;
    midT[(v * g.L + l) * g.Gx + mx] = buf[rs * pl.pitch + i + (i >> 4)];
  }
}

// Columns (v, l) of the row-transformed grid, pl.S columns per CTA (contiguous rows of
// midT, one bulk copy): FFT over mx, the N_s centred modes kept, deconvolved and written
// to the cube.
template <int P, int RL>
__global__ void nu_fft_x(const FrameIO* __restrict__ fp, NuGeo g, FftPlan pl, const float2* __restrict__ tw,
                         const float2* __restrict__ midT, const float* __restrict__ inv_x,
                         const float* __restrict__ inv_y, int out_dtype, unsigned* status) {
  wait_prior_grid();
  extern __shared__ __align__(128) unsigned char smem_x[];
  const float2* raw = reinterpret_cast<const float2*>(smem_x);
  float2* buf = reinterpret_cast<float2*>(smem_x);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_x + fft_smem_bytes(pl, 8) - 16);
  const int cblocks = (g.L + pl.S - 1) / pl.S;
  const int v = blockIdx.x / cblocks, l0 = (blockIdx.x % cblocks) * pl.S;
  const int live_cols = min(pl.S, g.L - l0);
  if (!load_rows(smem_x, midT + ((int64_t)v * g.L + l0) * g.Gx, (uint32_t)(live_cols * g.Gx * 8), bar, status))
    return;
  const int t = threadIdx.x % pl.T, s = threadIdx.x / pl.T;
  const float2* src = raw + (int64_t)s * g.Gx;
  const bool live = s < live_cols;
  auto in = [=](int i) -> float2 { return live ? src[i] : make_float2(0.f, 0.f); };
  fft_all<P, RL>(pl, in, buf + s * pl.pitch, t, tw);
  void* cube = fp->cube;
  // cube[v][n][l]: consecutive threads take consecutive l of one n
  for (int e = threadIdx.x; e < pl.S * g.Ns; e += blockDim.x) {
    const int cs = e % pl.S, n = e / pl.S;
    if (cs >= live_cols) continue;
    const int i = (n - g.sx) & (g.Gx - 1), l = l0 + cs;
    const float2 val = buf[cs * pl.pitch + i + (i >> 4)];
    const float f = inv_x[n] * inv_y[l];
    const int64_t o = ((int64_t)v * g.Ns + n) * g.L + l;
    if (out_dtype == RSIM_C128)
      reinterpret_cast<double2*>(cube)[o] = make_double2((double)(val.x * f), (double)(val.y * f));
    else
      reinterpret_cast<float2*>(cube)[o] = make_float2(val.x * f, val.y * f);
  }
}

int ilog2i(int x) {
  int b = 0;
  while ((1 << b) < x) ++b;
  return b;
}

int pow2_at_least(int x) {
  int g = 1;
  while (g < x) g <<= 1;
  return g;
}

// A sequence's T threads are adjacent, S sequences per CTA.  The pitch puts the 16 threads
// of a half-warp on distinct bank pairs: for T < 16 in the passes (16 / T sequences, the
// same positions), otherwise in the write-out (S sequences read at one position).
FftPlan fft_plan(int n) {
  FftPlan pl{};
  pl.n = n;
  pl.T = n / kFftPer;
  const int logn = ilog2i(n);
  pl.passes = (logn + 3) / 4;
  int ns = 1, off = 0;
  for (int p = 0; p < pl.passes; ++p) {
    pl.radix[p] = p + 1 < pl.passes ? 16 : 1 << (logn - 4 * (pl.passes - 1));
    pl.ns[p] = ns;
    pl.twoff[p] = off;
    if (p > 0) off += pl.radix[p] * ns;
    ns *= pl.radix[p];
  }
  pl.tw_size = off;
  pl.S = std::max(1, 128 / pl.T);
  const int target = pl.T < 16 ? pl.T : 16 / std::min(pl.S, 16);  // wanted pitch mod 16
  const int base = n + n / 16;
  pl.pitch = base + ((target - base % 16) % 16 + 16) % 16;
  return pl;
}

// The kernel instantiation of a plan: passes and the radix of the last pass.
template <template <int, int> class K>
typename K<1, 16>::Fn pick_fft(const FftPlan& pl) {
  const int rl = pl.radix[pl.passes - 1];
  if (pl.passes == 1) return K<1, 16>::fn();
  if (pl.passes == 2)
    return rl == 16 ? K<2, 16>::fn() : rl == 8 ? K<2, 8>::fn() : rl == 4 ? K<2, 4>::fn() : K<2, 2>::fn();
  return rl == 16 ? K<3, 16>::fn() : rl == 8 ? K<3, 8>::fn() : rl == 4 ? K<3, 4>::fn() : K<3, 2>::fn();
}

template <int P, int RL>
struct FftY {
  using Fn = void (*)(const FrameIO*, NuGeo, FftPlan, const float2*, const long long*, float2*, const int*,
                      unsigned*);
  static Fn fn() { return nu_fft_y<P, RL>; }
};

template <int P, int RL>
struct FftX {
  using Fn = void (*)(const FrameIO*, NuGeo, FftPlan, const float2*, const float2*, const float*, const float*, int,
                      unsigned*);
  static Fn fn() { return nu_fft_x<P, RL>; }
};

// Scratch of one frame: bin counts, cursors and offsets; the spreading work items; the
// records; the 64-bit integer grid; the row-transformed grid; the deconvolution factors.
struct NuScratch {
  int *count, *row_used, *cursor, *off, *items, *item_bin, *item_first;
  NuRec* rec;
  unsigned long long* grid;
  float2* mid;
  float *inv_x, *inv_y;
  float2 *tw_x, *tw_y;
  size_t grid_bytes, total;
};

NuScratch nufft_layout(const NuGeo& g, const FftPlan& plx, const FftPlan& ply, char* base) {
  const size_t nbins = (size_t)g.V * g.ntx * g.nty;
  const size_t max_items = nbins + ((size_t)g.V * g.P + kSpreadChunk - 1) / kSpreadChunk;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  NuScratch sc{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + o : nullptr;
    o += up(bytes);
    return p;
  };
  // the bin counts, the finished-block count, the grid rows in use (cleared together)
  sc.count = (int*)take(4 * (nbins + 1 + (size_t)g.V * g.Gx));
  sc.row_used = sc.count ? sc.count + nbins + 1 : nullptr;
  sc.cursor = (int*)take(4 * nbins);
  sc.off = (int*)take(4 * (nbins + 1));
  sc.items = (int*)take(4);
  sc.item_bin = (int*)take(4 * max_items);
  sc.item_first = (int*)take(4 * max_items);
  sc.rec = (NuRec*)take(sizeof(NuRec) * (size_t)g.V * g.P);
  sc.grid_bytes = 16 * (size_t)g.V * g.Gx * g.Gy;
  sc.grid = (unsigned long long*)take(sc.grid_bytes);
  sc.mid = (float2*)take(8 * (size_t)g.V * g.Gx * g.L);
  sc.inv_x = (float*)take(4 * (size_t)(g.Ns + g.L));
  sc.inv_y = sc.inv_x ? sc.inv_x + g.Ns : nullptr;
  sc.tw_x = (float2*)take(8 * (size_t)(plx.tw_size + ply.tw_size + 1));
  sc.tw_y = sc.tw_x ? sc.tw_x + plx.tw_size : nullptr;
  sc.total = o;
  return sc;
}

}  // namespace

NuGeo nufft_geometry(const Consts& k, int64_t P) {
  NuGeo g{};
  g.V = k.V;
  g.Ns = k.Ns;
  g.L = k.L;
  g.Gx = std::max(16, pow2_at_least(2 * k.Ns));  // at least one radix-16 FFT pass
  g.Gy = std::max(16, pow2_at_least(2 * k.L));
  g.Tx = std::min(kNTile, g.Gx);
  g.Ty = std::min(kNTile, g.Gy);
  g.ntx = g.Gx / g.Tx;
  g.nty = g.Gy / g.Ty;
  g.sx = k.Ns / 2;
  g.sy = k.L / 2;
  g.P = std::max<int64_t>(P, 1);
  g.W = k.nu_w;
  g.beta = kNBetaPerW * (float)g.W;
  return g;
}

bool nufft_supported(const Consts& k) {
  // FFT lengths up to 4096 in one CTA's shared memory, at least 8 cells per axis, and a
  // kernel width with a spreading kernel
  return 2 * (int64_t)k.Ns <= 4096 && 2 * (int64_t)k.L <= 4096 && k.Ns >= 4 && k.L >= 4 && k.nu_w >= kNWMin &&
         k.nu_w <= kNWMax;
}

size_t nufft_scratch_bytes(const Consts& k, int64_t P) {
  const NuGeo g = nufft_geometry(k, P);
  return nufft_layout(g, fft_plan(g.Gx), fft_plan(g.Gy), nullptr).total;
}

cudaError_t launch_nufft(const Consts& k, const FrameIO* frame, int64_t P, int out_dtype, char* scratch,
                         unsigned* status, cudaStream_t st, cudaEvent_t spread_begin, cudaEvent_t spread_end) {
  const NuGeo g = nufft_geometry(k, P);
  const int nb = g.ntx * g.nty;
  const int nbins = g.V * nb;
  const int64_t max_items = nbins + ((int64_t)g.V * g.P + kSpreadChunk - 1) / kSpreadChunk;
  const FftPlan plx = fft_plan(g.Gx), ply = fft_plan(g.Gy);
  const NuScratch sc = nufft_layout(g, plx, ply, scratch);
  int dev = 0, num_sms = 0;
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e0 != cudaSuccess) return e0;
  cudaError_t e = cudaMemsetAsync(sc.count, 0, 4 * ((size_t)nbins + 1 + (size_t)g.V * g.Gx), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc.grid, 0, sc.grid_bytes, st);
  if (e != cudaSuccess) return e;
  const dim3 bgrid((unsigned)((g.P + kBinItems - 1) / kBinItems), (unsigned)g.V);
  e = cudaFuncSetAttribute(nu_bin_count, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * nb);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(nu_bin_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * nb);
  if (e != cudaSuccess) return e;
  NuTables tb{};
  tb.psi_blocks = (g.Ns + g.L + kBinThreads / 32 - 1) / (kBinThreads / 32);
  tb.blocks = tb.psi_blocks + (plx.tw_size + ply.tw_size + kBinThreads - 1) / kBinThreads;
  tb.plx = plx;
  tb.ply = ply;
  tb.inv_x = sc.inv_x;
  tb.inv_y = sc.inv_y;
  tb.twx = sc.tw_x;
  tb.twy = sc.tw_y;
  const NuItems it{sc.off, sc.cursor, sc.items, sc.item_bin, sc.item_first};
  e = launch_dependent(nu_bin_count, dim3(bgrid.x, bgrid.y + 1), dim3(kBinThreads), (size_t)(4 * nb), st, frame, g,
                       sc.count, tb, it);
  if (e == cudaSuccess)
    e = launch_dependent(nu_bin_fill, bgrid, dim3(kBinThreads), (size_t)(8 * nb), st, frame, g, sc.cursor, sc.rec);
  // the spreading kernel of the gridding kernel's width, and its shared memory
  using SpreadFn = void (*)(const FrameIO*, NuGeo, const int*, const int*, const int*, const int*, const NuRec*,
                            unsigned long long*, int*);
  SpreadFn spread = nu_spread<7>;
  size_t spread_smem = SpreadLayout<7>::bytes;
  switch (g.W) {
    case 4: spread = nu_spread<4>; spread_smem = SpreadLayout<4>::bytes; break;
    case 5: spread = nu_spread<5>; spread_smem = SpreadLayout<5>::bytes; break;
    case 6: spread = nu_spread<6>; spread_smem = SpreadLayout<6>::bytes; break;
    case 8: spread = nu_spread<8>; spread_smem = SpreadLayout<8>::bytes; break;
    default: break;
  }
  if (e == cudaSuccess) e = cudaFuncSetAttribute(spread, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spread_smem);
  if (e == cudaSuccess && spread_begin) e = cudaEventRecord(spread_begin, st);
  if (e == cudaSuccess)
    e = launch_dependent(spread, dim3((unsigned)std::min<int64_t>(max_items, kSpreadBlocksPerSm * num_sms)),
                         dim3(kSpreadThreads), spread_smem, st, frame, g, (const int*)sc.off,
                         (const int*)sc.items, (const int*)sc.item_bin, (const int*)sc.item_first,
                         (const NuRec*)sc.rec, sc.grid, sc.row_used);
  if (e == cudaSuccess && spread_end) e = cudaEventRecord(spread_end, st);
  if (e != cudaSuccess) return e;
  const int ysmem = fft_smem_bytes(ply, 16);
  const auto fft_y = pick_fft<FftY>(ply);
  e = cudaFuncSetAttribute(fft_y, cudaFuncAttributeMaxDynamicSharedMemorySize, ysmem);
  if (e != cudaSuccess) return e;
  const int64_t yblocks = ((int64_t)g.V * g.Gx + ply.S - 1) / ply.S;
  e = launch_dependent(fft_y, dim3((unsigned)yblocks), dim3((unsigned)(ply.S * ply.T)), (size_t)ysmem, st, frame,
                       g, ply, (const float2*)sc.tw_y, (const long long*)sc.grid, sc.mid, (const int*)sc.row_used,
                       status);
  if (e != cudaSuccess) return e;
  const int xsmem = fft_smem_bytes(plx, 8);
  const auto fft_x = pick_fft<FftX>(plx);
  e = cudaFuncSetAttribute(fft_x, cudaFuncAttributeMaxDynamicSharedMemorySize, xsmem);
  if (e != cudaSuccess) return e;
  const int xblocks = g.V * ((g.L + plx.S - 1) / plx.S);
  return launch_dependent(fft_x, dim3((unsigned)xblocks), dim3((unsigned)(plx.S * plx.T)), (size_t)xsmem, st,
                          frame, g, plx, (const float2*)sc.tw_x, (const float2*)sc.mid, (const float*)sc.inv_x,
                          (const float*)sc.inv_y, out_dtype, status);
}

}  // namespace rsim
