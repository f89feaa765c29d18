// Valid-pixel compaction (mask step) and FP64 pixel-to-path phases.
//
// A pixel is a point target (Section II, the text before Eq. 2); one with zero
// strength is a background miss and is dropped.  The kept pixels are stored in
// ascending pixel order, together with the quantities Eq. 1 / Eq. 2 need per
// (pixel, virtual channel): the fast-time phase increment 2 mu R_{p,v} / (c F_s),
// the spatial phase v d_rx u_p / lambda and the slow-time increment -f_D T_slow.
// They are computed in FP64 and range-reduced to fractions of a cycle held as
// 32-bit fixed point (2^-32 cycle units), so that a phase at sample n is the exact
// integer product a * n mod 2^32: no phase of tens of cycles is ever formed in FP32.
//
// One cooperative kernel when every block of the grid (one row per frame) can be resident
// at once, else two kernels:
//   prep_count   - valid pixels per 256-pixel tile;
//   prep_scatter - tile offset = sum of earlier tile counts, ordered in-tile rank by
//                  warp ballots, then writes the index and the path phases;
//   prep_coop    - both in one launch with a grid barrier between them: a thread loads its
//                  pixel's fields once and keeps them in registers across the barrier,
//                  which saves a launch and, over a host link, the second read.  For the
//                  tensor-core tiers it writes only the slow-time phase and sigma: their
//                  operand builder computes the fast-time and channel phases (the FP64
//                  trigonometry) while it writes the slow-time operand images, so that
//                  FP64 work runs beside memory-bound work instead of before it.
// All are deterministic (no atomics decide positions), and both forms give the same bits.
#include <math.h>

#include <algorithm>
#include <cooperative_groups.h>

#include "rsim_internal.h"

namespace rsim {
namespace {

template <typename T>
__device__ __forceinline__ bool is_valid(const T* sre, const T* sim, int64_t p) {
  return (sre[p] != T(0)) || (sim[p] != T(0));
}

// `one`: with use_one, the (single) frame's entry, passed by value and stored to
// frames[0] here, so that no host-to-device copy precedes the kernels.  Block 0 of each
// frame clears its meta words and block (0, 0) the work-unit counter of the contraction.
template <typename T>
__global__ void __launch_bounds__(kPrepThreads)
prep_count(FrameIO* __restrict__ frames, FrameIO one, int use_one, int* counter) {
  const FrameIO fr = use_one ? one : frames[blockIdx.y];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (use_one) frames[0] = one;
    fr.meta[0] = 0ull;  // valid-pixel count, written by prep_scatter
    fr.meta[1] = 0ull;  // max |sigma| accumulator, filled by prep_scatter
    if (counter && blockIdx.y == 0)
      for (int i = 0; i < 4; ++i) counter[i] = 0;
  }
  const int64_t base = (int64_t)blockIdx.x * kPrepTile;
  if (base >= fr.P) return;
  const T* sre = (const T*)fr.sre;
  const T* sim = (const T*)fr.sim;
  int cnt = 0;
  for (int i = threadIdx.x; i < kPrepTile; i += kPrepThreads) {
    int64_t p = base + i;
    if (p < fr.P && is_valid(sre, sim, p)) ++cnt;
  }
  // block sum
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  __shared__ int ws[kPrepThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < kPrepThreads / 32; ++w) s += ws[w];
    fr.blk_count[blockIdx.x] = s;
  }
}

template <typename T>
__global__ void __launch_bounds__(kPrepThreads)
prep_scatter(const FrameIO* __restrict__ frames, Consts k, int idx_only, int defer, unsigned* status) {
  wait_prior_grid();
  const FrameIO& fr = frames[blockIdx.y];
  const int64_t base = (int64_t)blockIdx.x * kPrepTile;
  if (base >= fr.P) return;
  const int nblk = (int)((fr.P + kPrepTile - 1) / kPrepTile);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kPrepThreads / 32;
  __shared__ long long s_off;
  __shared__ int s_warp[kWarps];
  __shared__ float s_max[kWarps];

  // this thread's pixel fields, loaded before anything waits on them: over a host link
  // (pixel arrays read in place) their latency then overlaps the offset sum below
  static_assert(kPrepTile == kPrepThreads, "one pixel per thread");
  const T* R = (const T*)fr.range;
  const T* sre = (const T*)fr.sre;
  const T* sim = (const T*)fr.sim;
  const T* az = (const T*)fr.az;
  const T* el = (const T*)fr.el;
  const T* vel = (const T*)fr.vel;
  const int64_t p = base + tid;
  T f_re = T(0), f_im = T(0), f_r = T(0), f_az = T(0), f_el = T(0), f_vel = T(0);
  if (p < fr.P) {
    f_re = sre[p];
    f_im = sim[p];
    if (!idx_only) {
      f_r = R[p];
      f_az = az[p];
      f_el = el[p];
      f_vel = vel[p];
    }
  }

  // offset of this tile = sum of the counts of earlier tiles (fixed order)
  long long part = 0;
  for (int b = tid; b < (int)blockIdx.x; b += kPrepThreads) part += fr.blk_count[b];
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (lane == 0) s_warp[warp] = (int)part;  // each partial < 2^31 (P < 2^31 checked on host)
  __syncthreads();
  if (tid == 0) {
    long long s = 0;
    for (int w = 0; w < kWarps; ++w) s += s_warp[w];
    s_off = s;
  }
  __syncthreads();
  long long off = s_off;
  float mymax = 0.f;

  {
    const bool v = (p < fr.P) && ((f_re != T(0)) || (f_im != T(0)));  // as is_valid
    const unsigned bal = __ballot_sync(0xffffffffu, v);
    __syncthreads();  // s_warp reuse
    if (lane == 0) s_warp[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < kWarps; ++w) {
      int c = s_warp[w];
      before += (w < warp) ? c : 0;
      total += c;
    }
    const long long q = off + before + __popc(bal & ((1u << lane) - 1u));
    if (v) {
      fr.idx[q] = (int32_t)p;
      if (!idx_only) {
        const double r = (double)f_r, a = (double)f_az, e = (double)f_el, w = (double)f_vel;
        double s_re = (double)f_re, s_im = (double)f_im;
        const bool ok = pixel_ok(r, a, e, w, s_re, s_im);
        FastTerms t = {0, 0, 0, 0};
        uint64_t Bq = 0;
        if (ok) {
          Bq = frac_u64(k.k_b * w);  // -2 vel T_slow / lambda
          if (!defer) t = fast_terms(k, r, a, e, w);
        } else {
          atomicOr(status, kStatusNonfinite);
          s_re = 0.0;
          s_im = 0.0;
        }
        if (!defer) {
          for (int ch = 0; ch < k.V; ++ch) {
            fr.phA[(int64_t)ch * fr.Pcap + q] = chan_a(t, ch);
            fr.phC[(int64_t)ch * fr.Pcap + q] = chan_c(t, ch, k.N);
          }
        }
        fr.phB[q] = top32(Bq);
        const float fr_re = (float)s_re, fr_im = (float)s_im;
        fr.sig[q] = make_float2(fr_re, fr_im);
        mymax = fmaxf(mymax, fmaxf(fabsf(fr_re), fabsf(fr_im)));
      }
    }
    off += total;
  }
  if (blockIdx.x == nblk - 1 && tid == 0) fr.meta[0] = (unsigned long long)off;
  if (!idx_only) {
    for (int o = 16; o > 0; o >>= 1) mymax = fmaxf(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
    __syncthreads();
    if (lane == 0) s_max[warp] = mymax;
    __syncthreads();
    if (tid == 0) {
      float m = 0.f;
      for (int w = 0; w < kWarps; ++w) m = fmaxf(m, s_max[w]);
      if (m > 0.f) atomicMax(&fr.meta[1], (unsigned long long)__float_as_uint(m));
    }
  }
}

// One cooperative kernel: the counts, a grid barrier, then the scatter, with each thread's
// pixel fields kept in registers across the barrier (read once).
template <typename T>
__global__ void __launch_bounds__(kPrepThreads)
prep_coop(FrameIO* __restrict__ frames, FrameIO one, int use_one, int* counter, Consts k, int idx_only,
          int defer, unsigned* status) {
  const FrameIO fr = use_one ? one : frames[blockIdx.y];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kPrepThreads / 32;
  __shared__ long long s_off;
  __shared__ int s_warp[kWarps];
  __shared__ float s_max[kWarps];
  if (blockIdx.x == 0 && tid == 0) {
    if (use_one) frames[0] = one;
    fr.meta[0] = 0ull;
    fr.meta[1] = 0ull;
    if (counter && blockIdx.y == 0)
      for (int i = 0; i < 4; ++i) counter[i] = 0;
  }
  const int64_t base = (int64_t)blockIdx.x * kPrepTile;
  const bool live = base < fr.P;
  const T* R = (const T*)fr.range;
  const T* sre = (const T*)fr.sre;
  const T* sim = (const T*)fr.sim;
  const T* az = (const T*)fr.az;
  const T* el = (const T*)fr.el;
  const T* vel = (const T*)fr.vel;
  const int64_t p = base + tid;
  T f_re = T(0), f_im = T(0), f_r = T(0), f_az = T(0), f_el = T(0), f_vel = T(0);
  if (p < fr.P) {
    f_re = sre[p];
    f_im = sim[p];
    if (!idx_only) {
      f_r = R[p];
      f_az = az[p];
      f_el = el[p];
      f_vel = vel[p];
    }
  }
  const bool v = (p < fr.P) && ((f_re != T(0)) || (f_im != T(0)));
  const unsigned bal = __ballot_sync(0xffffffffu, v);
  if (lane == 0) s_warp[warp] = __popc(bal);
  __syncthreads();
  int before = 0, total = 0;
  for (int w = 0; w < kWarps; ++w) {
    const int c = s_warp[w];
    before += (w < warp) ? c : 0;
    total += c;
  }
  if (live && tid == 0) fr.blk_count[blockIdx.x] = total;
  cooperative_groups::this_grid().sync();
  if (!live) return;
  const int nblk = (int)((fr.P + kPrepTile - 1) / kPrepTile);
  long long part = 0;
  for (int b = tid; b < (int)blockIdx.x; b += kPrepThreads) part += fr.blk_count[b];
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  __syncthreads();  // s_warp reuse
  if (lane == 0) s_warp[warp] = (int)part;
  __syncthreads();
  if (tid == 0) {
    long long s2 = 0;
    for (int w = 0; w < kWarps; ++w) s2 += s_warp[w];
    s_off = s2;
  }
  __syncthreads();
  long long off = s_off;
  float mymax = 0.f;
  const long long q = off + before + __popc(bal & ((1u << lane) - 1u));
  if (v) {
    fr.idx[q] = (int32_t)p;
    if (!idx_only) {
      const double r = (double)f_r, a = (double)f_az, e = (double)f_el, w = (double)f_vel;
      double s_re = (double)f_re, s_im = (double)f_im;
      const bool ok = pixel_ok(r, a, e, w, s_re, s_im);
      FastTerms t = {0, 0, 0, 0};
      uint64_t Bq = 0;
      if (ok) {
        Bq = frac_u64(k.k_b * w);
        if (!defer) t = fast_terms(k, r, a, e, w);
      } else {
        atomicOr(status, kStatusNonfinite);
        s_re = 0.0;
        s_im = 0.0;
      }
      if (!defer) {
        for (int ch = 0; ch < k.V; ++ch) {
          fr.phA[(int64_t)ch * fr.Pcap + q] = chan_a(t, ch);
          fr.phC[(int64_t)ch * fr.Pcap + q] = chan_c(t, ch, k.N);
        }
      }
      fr.phB[q] = top32(Bq);
      const float fr_re = (float)s_re, fr_im = (float)s_im;
      fr.sig[q] = make_float2(fr_re, fr_im);
      mymax = fmaxf(mymax, fmaxf(fabsf(fr_re), fabsf(fr_im)));
    }
  }
  off += total;
  if (blockIdx.x == nblk - 1 && tid == 0) fr.meta[0] = (unsigned long long)off;
  if (!idx_only) {
    for (int o = 16; o > 0; o >>= 1) mymax = fmaxf(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
    __syncthreads();
    if (lane == 0) s_max[warp] = mymax;
    __syncthreads();
    if (tid == 0) {
      float m = 0.f;
      for (int w = 0; w < kWarps; ++w) m = fmaxf(m, s_max[w]);
      if (m > 0.f) atomicMax(&fr.meta[1], (unsigned long long)__float_as_uint(m));
    }
  }
}

}  // namespace

cudaError_t launch_prep(const Consts& k, FrameIO* frames, const FrameIO* one, int F, int64_t maxP,
                        int dtype, bool idx_only, bool defer_fast_terms, unsigned* status, int* counter,
                        cudaStream_t st, bool cooperative, int* launched) {
  if (F <= 0) return cudaSuccess;
  const int nblk = (int)std::max<int64_t>(1, (maxP + kPrepTile - 1) / kPrepTile);
  dim3 grid(nblk, F);
  const FrameIO arg = one ? *one : FrameIO{};
  const int use_one = one ? 1 : 0;
  if (cooperative && maxP > 0) {
    // blocks of the cooperative kernel resident per SM (a property of the kernel)
    static const int per_sm_f = [] {
      int n = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, prep_coop<float>, kPrepThreads, 0);
      return n;
    }();
    static const int per_sm_d = [] {
      int n = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, prep_coop<double>, kPrepThreads, 0);
      return n;
    }();
    int dev = 0, sms = 0;
    cudaError_t q = cudaGetDevice(&dev);
    if (q == cudaSuccess) q = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (q != cudaSuccess) return q;
    if ((int64_t)nblk * F <= (int64_t)(dtype == RSIM_F64 ? per_sm_d : per_sm_f) * sms) {
      FrameIO* a_frames = frames;
      FrameIO a_one = arg;
      int a_use_one = use_one, a_idx = idx_only ? 1 : 0, a_defer = defer_fast_terms ? 1 : 0;
      int* a_counter = counter;
      Consts a_k = k;
      unsigned* a_status = status;
      void* args[] = {&a_frames, &a_one, &a_use_one, &a_counter, &a_k, &a_idx, &a_defer, &a_status};
      const void* fn = dtype == RSIM_F64 ? (const void*)prep_coop<double> : (const void*)prep_coop<float>;
      if (launched) *launched = 1;
      return cudaLaunchCooperativeKernel(fn, grid, dim3(kPrepThreads), args, 0, st);
    }
  }
  if (launched) *launched = maxP > 0 ? 2 : 1;
  if (dtype == RSIM_F64) {
    prep_count<double><<<grid, kPrepThreads, 0, st>>>(frames, arg, use_one, counter);
    if (maxP > 0)
      return launch_dependent(prep_scatter<double>, grid, dim3(kPrepThreads), 0, st, (const FrameIO*)frames, k,
                              idx_only ? 1 : 0, defer_fast_terms ? 1 : 0, status);
  } else {
    prep_count<float><<<grid, kPrepThreads, 0, st>>>(frames, arg, use_one, counter);
    if (maxP > 0)
      return launch_dependent(prep_scatter<float>, grid, dim3(kPrepThreads), 0, st, (const FrameIO*)frames, k,
                              idx_only ? 1 : 0, defer_fast_terms ? 1 : 0, status);
  }
  return cudaGetLastError();
}

}  // namespace rsim
