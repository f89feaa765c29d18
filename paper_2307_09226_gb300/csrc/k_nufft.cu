// NUFFT tier: the sum of Eq. 2 through a two-dimensional type-1 non-uniform FFT per
// virtual channel.  With the fixed-point path phases of the compaction kernel,
//
//   cube[v][n][l] = sum_p q_p exp(j 2 pi (x_p n + y_p l)),
//   x_p = a_{p,v} (2 mu R_{p,v} / (c F_s), cycles per sample),  y_p = b_p (-f_D T_slow),
//   q_p = sigma_p exp(j 2 pi c_{p,v})   (spatial and TDM phases).
//
// Centred modes n = n' + s_x, l = l' + s_y move the shift into the strengths,
// q'_p = q_p exp(j 2 pi (x_p s_x + y_p s_y)).  Each q'_p is spread onto a periodic grid of
// G_x x G_y cells (powers of two >= 2 N_s, 2 L) with the "exponential of semicircle"
// kernel of Barnett, Magland and af Klinteberg (SIAM J. Sci. Comput. 41, 2019),
// psi(t) = exp(beta (sqrt(1 - (2t/w)^2) - 1)), width w = 7 cells, beta = 2.30 w; the
// grid's inverse-sign DFT at the centred modes, divided by the kernel's Fourier
// transform Psi_x(n') Psi_y(l'), is the cube (relative error ~1e-6 at w = 7).
//
// Kernels, per frame:
//   nu_psi        1 / (Psi_x(n') Psi_y(l')) factors: one warp per mode, a 128-node
//                 midpoint rule of Psi(k) = (w/2) int phi(z) cos(pi k w z / G) dz;
//   nu_bin_count  each (channel, point) is binned by the 32 x 32 grid tile of its
//                 nearest cell: a shared-memory histogram per block of one channel's
//                 points, one global addition per (block, bin);
//   nu_scan       exclusive scan of the bin counts (one block), and the table of
//                 spreading work items: every bin cut into chunks of 256 records;
//   nu_bin_fill   records (x, y, q') stored bin by bin (one global reservation per
//                 (block, bin), ranks within the block from shared memory);
//   nu_spread     one CTA per work item adds its records' w x w taps into a
//                 shared-memory tile with a (w - 1) / 2 halo, as fixed-point integers
//                 (each term split in 16-bit halves summed by non-returning 32-bit
//                 atomics), then adds the tile into the global 64-bit integer grid.
//                 Integer sums are exact and do not depend on the order of the atomic
//                 additions, so the result is bit-reproducible.  The work items share
//                 the crowded tiles among many SMs: a scene fills only the part of the
//                 grid that its ranges and speeds reach;
//   nu_fft_y      rows of the grid: integer -> float, radix-2 inverse-sign FFT over the
//                 slow-time axis in shared memory (a sequence's butterflies on
//                 consecutive threads, twiddles from a shared table), only the L
//                 centred modes kept;
//   nu_fft_x      columns: FFT over the fast-time axis, only the N_s centred modes kept,
//                 times the deconvolution factors, written to the cube.
#include <math.h>

#include <algorithm>

#include "rsim_internal.h"

namespace rsim {
namespace {

constexpr int kNW = 7;                      // kernel width in cells (odd)
constexpr int kNHalf = (kNW - 1) / 2;       // taps on each side of the nearest cell
constexpr float kNBeta = 2.30f * kNW;       // ES shape for an oversampling of 2
constexpr int kNTile = 32;                  // grid cells per tile side
constexpr int kNPad = kNTile + 2 * kNHalf;  // tile side with the halo
constexpr int kNQuad = 128;                 // midpoint nodes for Psi
constexpr int kSpreadChunk = 256;           // records per spreading work item
constexpr int kBinThreads = 1024;           // binning blocks: one channel, kBinItems points
constexpr int kBinItems = 4 * kBinThreads;

struct NuRec {
  uint32_t x, y;  // positions, 2^-32 cycles
  float2 q;       // shifted strength q'
};

// exp(beta (sqrt(1 - z^2) - 1)) on |z| <= 1, 0 outside
__device__ __forceinline__ float es_kernel(float z) {
  const float z2 = z * z;
  return z2 < 1.f ? expf(kNBeta * (sqrtf(1.f - z2) - 1.f)) : 0.f;
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

// Add a 32-bit signed term to a sum kept as two 32-bit words with non-returning
// atomics: the low 16 bits of each term go to `lo` (unsigned) and the signed high part
// to `hi`, so the sum is hi 2^16 + lo exactly while a word receives fewer than 2^16
// terms (a work item holds kSpreadChunk records, each adding once per cell).
__device__ __forceinline__ void add_split(unsigned* lo, int* hi, int v) {
  if (v == 0) return;
  atomicAdd(lo, (unsigned)(v & 0xffff));
  atomicAdd(hi, v >> 16);
}

__global__ void nu_psi(NuGeo g, float* __restrict__ inv_x, float* __restrict__ inv_y) {
  wait_prior_grid();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= g.Ns + g.L) return;
  const bool xs = warp < g.Ns;
  const int k = xs ? warp - g.sx : (warp - g.Ns) - g.sy;
  const float G = (float)(xs ? g.Gx : g.Gy);
  float s = 0.f;
  for (int j = lane; j < kNQuad; j += 32) {
    const float z = -1.f + ((float)j + 0.5f) * (2.f / kNQuad);
    s += es_kernel(z) * cospif((float)k * (float)kNW * z / G);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const float psi = 0.5f * (float)kNW * (2.f / kNQuad) * s;
    if (xs)
      inv_x[warp] = 1.f / psi;
    else
      inv_y[warp - g.Ns] = 1.f / psi;
  }
}

// Binning blocks: blockIdx.y = channel, blockIdx.x = a range of kBinItems points.
__global__ void __launch_bounds__(kBinThreads) nu_bin_count(const FrameIO* __restrict__ fp, NuGeo g,
                                                            int* __restrict__ count) {
  wait_prior_grid();
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
}

// Exclusive scan of n bin counts (one block of 1024 threads) into `off` and `cursor`, and
// of their chunk counts into the work-item table: item_bin[i] is the bin of item i,
// item_first[i] its first record, items[0] the number of items.
__global__ void __launch_bounds__(1024) nu_scan(const int* __restrict__ count, int n, int* __restrict__ off,
                                                int* __restrict__ cursor, int* __restrict__ items,
                                                int* __restrict__ item_bin, int* __restrict__ item_first) {
  wait_prior_grid();
  __shared__ int part[1024], cpart[1024];
  const int t = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int b0 = min(n, t * per), b1 = min(n, b0 + per);
  int s = 0, c = 0;
  for (int b = b0; b < b1; ++b) {
    s += count[b];
    c += (count[b] + kSpreadChunk - 1) / kSpreadChunk;
  }
  part[t] = s;
  cpart[t] = c;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scans of the chunk sums
    const int x = t >= o ? part[t - o] : 0, y = t >= o ? cpart[t - o] : 0;
    __syncthreads();
    part[t] += x;
    cpart[t] += y;
    __syncthreads();
  }
  int run = part[t] - s, crun = cpart[t] - c;
  for (int b = b0; b < b1; ++b) {
    off[b] = run;
    cursor[b] = run;
    for (int k = 0; k < count[b]; k += kSpreadChunk, ++crun) {
      item_bin[crun] = b;
      item_first[crun] = run + k;
    }
    run += count[b];
  }
  if (t == 1023) {
    off[n] = part[1023];
    items[0] = cpart[1023];
  }
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
  int bins[kPer], rank[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int64_t p = p0 + threadIdx.x + (int64_t)i * blockDim.x;
    bins[i] = -1;
    rank[i] = 0;
    if (p < pv) {
      bins[i] = bin_of(fr.phA[(int64_t)v * fr.Pcap + p], fr.phB[p], g);
      rank[i] = atomicAdd(&hist[bins[i]], 1);
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) base[b] = hist[b] ? atomicAdd(&cursor[v * nb + b], hist[b]) : 0;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    if (bins[i] < 0) continue;
    const int64_t p = p0 + threadIdx.x + (int64_t)i * blockDim.x;
    const uint32_t xq = fr.phA[(int64_t)v * fr.Pcap + p], yq = fr.phB[p];
    // q' = sigma exp(j 2 pi (c + x s_x + y s_y)), the phase exact mod 1 in 2^-32 cycles
    const uint32_t ph = fr.phC[(int64_t)v * fr.Pcap + p] + xq * (uint32_t)g.sx + yq * (uint32_t)g.sy;
    float sn, cs;
    sincospif((float)(int32_t)ph * 4.656612873077393e-10f, &sn, &cs);  // angle pi ph / 2^31
    const float2 sg = fr.sig[p];
    NuRec r;
    r.x = xq;
    r.y = yq;
    r.q = make_float2(sg.x * cs - sg.y * sn, sg.x * sn + sg.y * cs);
    rec[base[bins[i]] + rank[i]] = r;
  }
}

__global__ void __launch_bounds__(256) nu_spread(const FrameIO* __restrict__ fp, NuGeo g,
                                                 const int* __restrict__ off, const int* __restrict__ items,
                                                 const int* __restrict__ item_bin,
                                                 const int* __restrict__ item_first,
                                                 const NuRec* __restrict__ rec,
                                                 unsigned long long* __restrict__ grid) {
  wait_prior_grid();
  if ((int)blockIdx.x >= items[0]) return;
  __shared__ unsigned lo[2][kNPad * kNPad];
  __shared__ int hi[2][kNPad * kNPad];
  const int bin = item_bin[blockIdx.x];
  const int nb = g.ntx * g.nty;
  const int v = bin / nb, ty = (bin % nb) % g.nty, tx = (bin % nb) / g.nty;
  const int r_begin = item_first[blockIdx.x];
  const int r_end = min(off[bin + 1], r_begin + kSpreadChunk);
  for (int i = threadIdx.x; i < kNPad * kNPad; i += blockDim.x) {
    lo[0][i] = lo[1][i] = 0u;
    hi[0][i] = hi[1][i] = 0;
  }
  __syncthreads();
  const float scale = grid_scale(*fp, false);
  const int x0 = tx * g.Tx - kNHalf, y0 = ty * g.Ty - kNHalf;  // padded tile origin (cells)
  for (int r = r_begin + threadIdx.x; r < r_end; r += blockDim.x) {
    const NuRec q = rec[r];
    int cx, cy;
    float dx, dy;
    nearest_cell(q.x, g.Gx, cx, dx);
    nearest_cell(q.y, g.Gy, cy, dy);
    // the nearest cell lies in this tile: local padded coordinates of the first tap
    const int lx = cx - tx * g.Tx, ly = cy - ty * g.Ty;
    float wx[kNW], wy[kNW];
#pragma unroll
    for (int j = 0; j < kNW; ++j) {
      wx[j] = es_kernel(2.f * ((float)(j - kNHalf) - dx) / (float)kNW);
      wy[j] = es_kernel(2.f * ((float)(j - kNHalf) - dy) / (float)kNW);
    }
    const float qr = q.q.x * scale, qi = q.q.y * scale;
#pragma unroll
    for (int jx = 0; jx < kNW; ++jx) {
      const float ar = qr * wx[jx], ai = qi * wx[jx];
      const int row = (lx + jx) * kNPad + ly;
#pragma unroll
      for (int jy = 0; jy < kNW; ++jy) {
        add_split(&lo[0][row + jy], &hi[0][row + jy], __float2int_rn(ar * wy[jy]));
        add_split(&lo[1][row + jy], &hi[1][row + jy], __float2int_rn(ai * wy[jy]));
      }
    }
  }
  __syncthreads();
  const int64_t gbase = (int64_t)v * g.Gx * g.Gy;
  for (int i = threadIdx.x; i < kNPad * kNPad; i += blockDim.x) {
    const long long re = ((long long)hi[0][i] << 16) + (long long)lo[0][i];
    const long long im = ((long long)hi[1][i] << 16) + (long long)lo[1][i];
    if (re == 0 && im == 0) continue;
    const int gx = (x0 + i / kNPad) & (g.Gx - 1), gy = (y0 + i % kNPad) & (g.Gy - 1);
    unsigned long long* cell = grid + 2 * (gbase + (int64_t)gx * g.Gy + gy);
    atomicAdd(cell, (unsigned long long)re);
    atomicAdd(cell + 1, (unsigned long long)im);
  }
}

// twiddles tw[k] = exp(+j 2 pi k / n) for k < n / 2, built once per CTA
__device__ void build_twiddles(float2* tw, int n) {
  for (int k = threadIdx.x; k < n / 2; k += blockDim.x) {
    float sn, cs;
    sincospif(2.f * (float)k / (float)n, &sn, &cs);
    tw[k] = make_float2(cs, sn);
  }
}

// In-place radix-2 inverse-sign butterflies over `count` = 2^logc sequences of length
// n = 2^logn in shared memory, element i of sequence j at x[i * istride + j * jstride],
// already in bit-reversed order.  CONTIG: the elements of a sequence are adjacent
// (istride 1), so a sequence's butterflies go to consecutive threads; otherwise the
// sequences are adjacent (jstride 1) and consecutive threads take consecutive sequences.
// Both keep a warp's shared-memory accesses on distinct banks.
template <bool CONTIG>
__device__ void fft_inv_stages(float2* x, const float2* tw, int logn, int logc, int istride, int jstride) {
  const int half_total = 1 << (logn - 1 + logc);
  const int hmask = (1 << (logn - 1)) - 1, cmask = (1 << logc) - 1;
  for (int s = 1; s <= logn; ++s) {
    const int h = 1 << (s - 1);
    __syncthreads();
    for (int t = threadIdx.x; t < half_total; t += blockDim.x) {
      const int b = CONTIG ? (t & hmask) : (t >> logc);
      const int j = CONTIG ? (t >> (logn - 1)) : (t & cmask);
      const int k = b & (h - 1);
      const int i0 = ((b >> (s - 1)) << s) + k, i1 = i0 + h;
      const float2 w = tw[k << (logn - s)];
      float2* p0 = x + i0 * istride + j * jstride;
      float2* p1 = x + i1 * istride + j * jstride;
      const float2 u = *p0, a = *p1;
      const float2 vv = make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
      *p0 = make_float2(u.x + vv.x, u.y + vv.y);
      *p1 = make_float2(u.x - vv.x, u.y - vv.y);
    }
  }
  __syncthreads();
}

__device__ __forceinline__ unsigned bitrev(unsigned x, int bits) { return __brev(x) >> (32 - bits); }

// Rows (v, mx) of the grid: 2^log_rows rows per CTA, FFT over my, the L centred modes kept.
__global__ void nu_fft_y(const FrameIO* __restrict__ fp, NuGeo g, int log_rows, int ybits,
                         const long long* __restrict__ grid, float2* __restrict__ mid) {
  wait_prior_grid();
  extern __shared__ float2 sy[];  // [rows][Gy], then Gy / 2 twiddles
  const int rows_per = 1 << log_rows;
  float2* tw = sy + rows_per * g.Gy;
  build_twiddles(tw, g.Gy);
  const float inv = grid_scale(*fp, true);
  const int64_t r0 = (int64_t)blockIdx.x * rows_per;  // row = v * Gx + mx
  const int64_t rows = (int64_t)g.V * g.Gx;
  for (int e = threadIdx.x; e < rows_per * g.Gy; e += blockDim.x) {
    const int rr = e >> ybits, m = e & (g.Gy - 1);
    const int64_t row = r0 + rr;
    float2 val = make_float2(0.f, 0.f);
    if (row < rows) {
      const long long* c = grid + 2 * (row * g.Gy + m);
      val = make_float2(ll_to_float(c[0]) * inv, ll_to_float(c[1]) * inv);
    }
    sy[rr * g.Gy + bitrev((unsigned)m, ybits)] = val;
  }
  fft_inv_stages<true>(sy, tw, ybits, log_rows, 1, g.Gy);
  for (int e = threadIdx.x; e < rows_per * g.L; e += blockDim.x) {
    const int rr = e / g.L, l = e % g.L;
    const int64_t row = r0 + rr;
    if (row >= rows) continue;
    mid[row * g.L + l] = sy[rr * g.Gy + ((l - g.sy) & (g.Gy - 1))];
  }
}

// Columns (v, l) of the row-transformed grid: 2^log_cols columns per CTA, FFT over mx,
// the N_s centred modes kept, deconvolved and written to the cube.
__global__ void nu_fft_x(const FrameIO* __restrict__ fp, NuGeo g, int log_cols, int xbits,
                         const float2* __restrict__ mid, const float* __restrict__ inv_x,
                         const float* __restrict__ inv_y, int out_dtype) {
  wait_prior_grid();
  extern __shared__ float2 sx[];  // [Gx][cols], then Gx / 2 twiddles
  const int cols_per = 1 << log_cols;
  float2* tw = sx + g.Gx * cols_per;
  build_twiddles(tw, g.Gx);
  const int cblocks = (g.L + cols_per - 1) / cols_per;
  const int v = blockIdx.x / cblocks, l0 = (blockIdx.x % cblocks) * cols_per;
  const float2* src = mid + (int64_t)v * g.Gx * g.L;
  for (int e = threadIdx.x; e < g.Gx * cols_per; e += blockDim.x) {
    const int m = e >> log_cols, j = e & (cols_per - 1);
    const int l = l0 + j;
    sx[bitrev((unsigned)m, xbits) * cols_per + j] = (l < g.L) ? src[(int64_t)m * g.L + l] : make_float2(0.f, 0.f);
  }
  fft_inv_stages<false>(sx, tw, xbits, log_cols, cols_per, 1);
  const FrameIO& fr = *fp;
  for (int e = threadIdx.x; e < g.Ns * cols_per; e += blockDim.x) {
    const int n = e >> log_cols, j = e & (cols_per - 1);
    const int l = l0 + j;
    if (l >= g.L) continue;
    const float2 s = sx[((n - g.sx) & (g.Gx - 1)) * cols_per + j];
    const float f = inv_x[n] * inv_y[l];
    const int64_t o = ((int64_t)v * g.Ns + n) * g.L + l;
    if (out_dtype == RSIM_C128)
      reinterpret_cast<double2*>(fr.cube)[o] = make_double2((double)(s.x * f), (double)(s.y * f));
    else
      reinterpret_cast<float2*>(fr.cube)[o] = make_float2(s.x * f, s.y * f);
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

// Scratch of one frame: bin counts, cursors and offsets; the spreading work items; the
// records; the 64-bit integer grid; the row-transformed grid; the deconvolution factors.
struct NuScratch {
  int *count, *cursor, *off, *items, *item_bin, *item_first;
  NuRec* rec;
  unsigned long long* grid;
  float2* mid;
  float *inv_x, *inv_y;
  size_t grid_bytes, total;
};

NuScratch nufft_layout(const NuGeo& g, char* base) {
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
  sc.count = (int*)take(4 * nbins);
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
  sc.total = o;
  return sc;
}

}  // namespace

NuGeo nufft_geometry(const Consts& k, int64_t P) {
  NuGeo g{};
  g.V = k.V;
  g.Ns = k.Ns;
  g.L = k.L;
  g.Gx = pow2_at_least(2 * k.Ns);
  g.Gy = pow2_at_least(2 * k.L);
  g.Tx = std::min(kNTile, g.Gx);
  g.Ty = std::min(kNTile, g.Gy);
  g.ntx = g.Gx / g.Tx;
  g.nty = g.Gy / g.Ty;
  g.sx = k.Ns / 2;
  g.sy = k.L / 2;
  g.P = std::max<int64_t>(P, 1);
  return g;
}

bool nufft_supported(const Consts& k) {
  // FFT lengths up to 4096 in one CTA's shared memory, at least 8 cells per axis
  return 2 * (int64_t)k.Ns <= 4096 && 2 * (int64_t)k.L <= 4096 && k.Ns >= 4 && k.L >= 4;
}

size_t nufft_scratch_bytes(const Consts& k, int64_t P) { return nufft_layout(nufft_geometry(k, P), nullptr).total; }

cudaError_t launch_nufft(const Consts& k, const FrameIO* frame, int64_t P, int out_dtype, char* scratch,
                         cudaStream_t st) {
  const NuGeo g = nufft_geometry(k, P);
  const int nb = g.ntx * g.nty;
  const int nbins = g.V * nb;
  const int64_t max_items = nbins + ((int64_t)g.V * g.P + kSpreadChunk - 1) / kSpreadChunk;
  const NuScratch sc = nufft_layout(g, scratch);
  cudaError_t e = cudaMemsetAsync(sc.count, 0, 4 * (size_t)nbins, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc.grid, 0, sc.grid_bytes, st);
  if (e != cudaSuccess) return e;
  const dim3 bgrid((unsigned)((g.P + kBinItems - 1) / kBinItems), (unsigned)g.V);
  e = cudaFuncSetAttribute(nu_bin_count, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * nb);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(nu_bin_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * nb);
  if (e != cudaSuccess) return e;
  e = launch_dependent(nu_psi, dim3((unsigned)((g.Ns + g.L + 7) / 8)), dim3(256), 0, st, g, sc.inv_x, sc.inv_y);
  if (e == cudaSuccess)
    e = launch_dependent(nu_bin_count, bgrid, dim3(kBinThreads), (size_t)(4 * nb), st, frame, g, sc.count);
  if (e == cudaSuccess)
    e = launch_dependent(nu_scan, dim3(1), dim3(1024), 0, st, (const int*)sc.count, nbins, sc.off, sc.cursor,
                         sc.items, sc.item_bin, sc.item_first);
  if (e == cudaSuccess)
    e = launch_dependent(nu_bin_fill, bgrid, dim3(kBinThreads), (size_t)(8 * nb), st, frame, g, sc.cursor, sc.rec);
  if (e == cudaSuccess)
    e = launch_dependent(nu_spread, dim3((unsigned)max_items), dim3(256), 0, st, frame, g, (const int*)sc.off,
                         (const int*)sc.items, (const int*)sc.item_bin, (const int*)sc.item_first,
                         (const NuRec*)sc.rec, sc.grid);
  if (e != cudaSuccess) return e;
  const int log_rows = std::max(0, 10 - ilog2i(g.Gy));  // rows * Gy = 1024 complex per CTA
  const int ysmem = ((1 << log_rows) * g.Gy + g.Gy / 2) * (int)sizeof(float2);
  e = cudaFuncSetAttribute(nu_fft_y, cudaFuncAttributeMaxDynamicSharedMemorySize, ysmem);
  if (e != cudaSuccess) return e;
  const int64_t yblocks = ((int64_t)g.V * g.Gx + (1 << log_rows) - 1) >> log_rows;
  e = launch_dependent(nu_fft_y, dim3((unsigned)yblocks), dim3(256), (size_t)ysmem, st, frame, g, log_rows,
                       ilog2i(g.Gy), (const long long*)sc.grid, sc.mid);
  if (e != cudaSuccess) return e;
  const int log_cols = std::max(0, std::min(2, 11 - ilog2i(g.Gx)));  // cols * Gx <= 2048 complex per CTA
  const int cols_per = 1 << log_cols;
  const int xsmem = (g.Gx * cols_per + g.Gx / 2) * (int)sizeof(float2);
  e = cudaFuncSetAttribute(nu_fft_x, cudaFuncAttributeMaxDynamicSharedMemorySize, xsmem);
  if (e != cudaSuccess) return e;
  const int xblocks = g.V * ((g.L + cols_per - 1) / cols_per);
  return launch_dependent(nu_fft_x, dim3((unsigned)xblocks), dim3(256), (size_t)xsmem, st, frame, g, log_cols,
                          ilog2i(g.Gx), (const float2*)sc.mid, (const float*)sc.inv_x, (const float*)sc.inv_y,
                          out_dtype);
}

}  // namespace rsim
