// Internal declarations shared by the CUDA sources of librsim (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>

#include "../../include/rsim.h"

namespace rsim {

constexpr int kChunkPx = 32;        // pixels per pipeline stage / K-chunk (64 real K)
constexpr int kPrepTile = 256;      // pixels per block of the compaction kernels
constexpr int kPrepThreads = 256;
constexpr int kMaxSplits = 64;
constexpr int kReduceBatch = 8;     // split partials a reduction thread loads at once

// Host-resolved constants of one radar configuration.  The per-pixel FP64 phase
// increments are products of these with R, u and vel (Eq. 1 / Eq. 2):
//   a_{p,v} = k_a0 R_p + v k_da u_p    (2 mu R_{p,v} / (c F_s), cycles per sample)
//   c_{p,v} = v k_g u_p                (v d_rx u_p / lambda, cycles)
//   b_p     = k_b vel_p                (-2 vel_p T_slow / lambda, cycles per block)
// and, with RSIM_FLAG_TDM_MOTION, c_{p,v} gains m k_m vel_p (-2 vel_p m T_b / lambda,
// Tx slot m = v / N); k_m = 0 otherwise.
struct Consts {
  int M, N, V, Ns, L;
  double k_a0, k_da, k_g, k_b, k_m;
  int nu_w;  // NUFFT tier: gridding kernel width (cells)
};

// One frame as the kernels see it: caller buffers plus this frame's workspace slices.
struct FrameIO {
  const void* range;
  const void* sre;
  const void* sim;
  const void* az;
  const void* el;
  const void* vel;
  void* cube;                 // [V][Ns][L] complex (out_dtype)
  int64_t P;                  // pixels in the frame
  int64_t Pcap;               // row stride of phA / phC (>= P, multiple of 64)
  int32_t* idx;               // [Pcap] ascending valid indices
  uint32_t* phA;              // [V][Pcap] fast-time increment, 2^-32 cycle/sample
  uint32_t* phC;              // [V][Pcap] spatial phase, 2^-32 cycle
  uint32_t* phB;              // [Pcap]    slow-time increment, 2^-32 cycle/block
  float2* sig;                // [Pcap]    sigma (FP32)
  int32_t* blk_count;         // [ceil(P / kPrepTile)] valid pixels per prep block
  unsigned long long* meta;   // [0] P_valid, [1] max(|re|,|im|) of sigma as float bits
  float2* partial;            // split partial sums (NULL when unused): FP32 tier [splits][V*Ns][L];
                              // tensor tiers in tiles, see tensor_split_stride
  unsigned char* bimg;        // tensor tiers: slow-time operand as shared-memory images
  int64_t bimg_nch;           // chunk capacity of bimg per column tile
  int32_t splits;             // pixel splits of the contraction
  int32_t pad;
};

// NVTX range in the "rsim" domain for the lifetime of a scope (header-only NVTX v3: it
// costs a few nanoseconds unless a profiler is attached).  The ranges mark the host-side
// launches of each stage and of each served request, so a profiler's kernel list can be
// split by stage and by request (ncu's --nvtx range filters select one range's kernels).
inline nvtxDomainHandle_t nvtx_domain() {
  static nvtxDomainHandle_t d = nvtxDomainCreateA("rsim");
  return d;
}
struct NvtxRange {
  explicit NvtxRange(const char* msg) {
    nvtxEventAttributes_t a = {};
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = msg;
    nvtxDomainRangePushEx(nvtx_domain(), &a);
  }
  ~NvtxRange() { nvtxDomainRangePop(nvtx_domain()); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device status word bits (OR-ed by kernels, read by rsim_sync_status).
enum : unsigned { kStatusNonfinite = 1u, kStatusTimeout = 2u };

// Workspace slices of one frame, as byte offsets from a base pointer.
struct FrameLayout {
  size_t idx, phA, phC, phB, sig, blk, meta, partial, bimg, total;
  int64_t Pcap, bimg_nch;
};
// nt: the plan's column tile of the tensor tiers (ignored otherwise).
FrameLayout frame_layout(int V, int Ns, int L, int64_t P, int splits, bool use_partial, bool tensor,
                         int nt, size_t base);
// Default columns of l per tensor-core column tile: min(128, L rounded up to 8).
int tile_nt(int L);
// Complex elements of one split's partial sums on the tensor tiers with column tile nt.
// They are stored by accumulator tile, [row tile][column tile][column pair][128 rows][2
// columns], so that a warp's 32 accumulator rows drain into 512 contiguous bytes.
int64_t tensor_split_stride(int V, int Ns, int L, int nt);

// Tensor-core tiers (the tcgen05 contraction and its operand images).
inline bool tensor_tier(int tier) {
  return tier == RSIM_TIER_BF16 || tier == RSIM_TIER_SPLIT_BF16 || tier == RSIM_TIER_SPLIT_FP16 ||
         tier == RSIM_TIER_FP16;
}

// NUFFT tier: grid and tile geometry of one frame shape.
struct NuGeo {
  int V, Ns, L;   // channels and output modes
  int Gx, Gy;     // oversampled grid (powers of two >= 2 Ns, 2 L)
  int Tx, Ty;     // tile sides (cells)
  int ntx, nty;   // tiles per axis
  int sx, sy;     // centring shifts Ns / 2, L / 2
  int64_t P;      // pixel bound (items per channel)
  int W;          // gridding kernel width (cells)
  float beta;     // its shape parameter, 2.30 W
};
// Kernels launch_nufft starts per frame (binning with the tables and the scan, record
// fill, spreading, two FFT passes).
constexpr int kNufftKernels = 5;
NuGeo nufft_geometry(const Consts& k, int64_t P);
bool nufft_supported(const Consts& k);
size_t nufft_scratch_bytes(const Consts& k, int64_t P);
// One frame (`frame`: device pointer to its table entry, P: its pixel count), using
// nufft_scratch_bytes(k, P) bytes of scratch; a copy that times out sets kStatusTimeout in
// `status`.  Non-null events are recorded just before and after the spreading kernel.
cudaError_t launch_nufft(const Consts& k, const FrameIO* frame, int64_t P, int out_dtype, char* scratch,
                         unsigned* status, cudaStream_t st, cudaEvent_t spread_begin = nullptr,
                         cudaEvent_t spread_end = nullptr);

// Programmatic dependent launch: a kernel launched with launch_dependent may be
// scheduled while the previous kernel in the stream drains its last blocks, hiding the
// launch latency between the stages of one call.  Such a kernel executes
// wait_prior_grid() before it touches anything the previous kernel writes; the wait
// returns once that kernel has completed and its writes are visible (it is a no-op for
// a kernel launched without the attribute).
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Shared-memory mbarrier with one expected arrival, initialised by the calling thread;
// the block synchronises before any other thread uses it.
__device__ __forceinline__ void mbar_init_single(uint64_t* bar) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait for the phase of parity `parity` of the shared-memory mbarrier `bar`: polls
// with try_wait and reads %globaltimer every 256 polls.  True once the phase has
// completed, false when limit_ns passed first (the caller records the timeout).
__device__ __forceinline__ bool wait_phase_bounded(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
  unsigned long long t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255u) == 255u) {
      unsigned long long now;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
      if (t0 == 0)
        t0 = now;
      else if (now - t0 > limit_ns)
        return false;
    }
  }
}

// Failure-detection self test: one CTA waits (wait_phase_bounded) on a barrier phase that
// nothing completes and, after limit_ns, sets kStatusTimeout in `status`.
cudaError_t launch_wait_selftest(unsigned* status, unsigned long long limit_ns, cudaStream_t st);

template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Add x to the compensated sum (s, c) (Kahan): the running error of FP32 additions is
// carried in c, so the sum of a few dozen partials is as accurate as one rounding.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}
// frac(x) = x - floor(x) as an unsigned 64-bit fixed-point number of 2^-64 units, read
// from the binary representation with integer operations (GB300's FP64 rate is a small
// fraction of its integer rate).  x = m 2^(E - 1075) with the 53-bit significand m, so
// frac(x) 2^64 = m 2^(E - 1011) mod 2^64: exact when that shift is >= 0, else rounded to
// the nearest unit (half up).  A negative x gives 2^64 - frac(|x|) 2^64 (mod 2^64).
__device__ __forceinline__ uint64_t frac_u64(double x) {
  const uint64_t bits = (uint64_t)__double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  if (E == 0 || E == 0x7FF) return 0;  // zero, subnormal (< 2^-1022) or not finite
  const uint64_t m = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = E - 1011;
  uint64_t f;
  if (sh >= 64)
    f = 0;  // x is a multiple of 2^64 units: an integer
  else if (sh >= 0)
    f = m << sh;
  else if (sh >= -53)
    f = (m >> -sh) + ((m >> (-sh - 1)) & 1ull);
  else
    f = 0;  // below half a unit
  return (bits >> 63) ? (uint64_t)0 - f : f;
}

// Round a 2^-64 fixed-point fraction to the nearest 2^-32 unit (mod 1).
__device__ __forceinline__ uint32_t top32(uint64_t x) {
  return (uint32_t)((x + 0x80000000ull) >> 32);
}

// A pixel whose fields are all finite and whose range is positive gets its path terms;
// any other gets zero terms and zero strength, and the kernel that reads it reports it.
__device__ __forceinline__ bool pixel_ok(double r, double a, double e, double w, double s_re, double s_im) {
  return isfinite(r) && r > 0.0 && isfinite(a) && isfinite(e) && isfinite(w) && isfinite(s_re) &&
         isfinite(s_im);
}

// The fast-time and channel terms of one pixel (Eq. 1 / Eq. 2, see Consts) in 2^-64-cycle
// units, from FP64 arithmetic: A0 = 2 mu R / (c F_s), dA = mu d_rx u / (c F_s) and
// G = d_rx u / lambda per channel index, Bm = -2 vel T_b / lambda per Tx slot (0 unless
// the TDM motion term is on), with the direction cosine u = cos(el) sin(az).  The
// compaction kernel and the tensor tiers' operand builder both call this, so the two
// write the same bits.
struct FastTerms {
  uint64_t A0, dA, G, Bm;
};
__device__ __forceinline__ FastTerms fast_terms(const Consts& k, double r, double az, double el, double w) {
  const double u = cos(el) * sin(az);
  FastTerms t;
  t.A0 = frac_u64(k.k_a0 * r);
  t.dA = frac_u64(k.k_da * u);
  t.G = frac_u64(k.k_g * u);
  t.Bm = frac_u64(k.k_m * w);
  return t;
}
// Channel ch's fast-time increment a_{p,ch} and spatial phase c_{p,ch}, in 2^-32 cycle.
__device__ __forceinline__ uint32_t chan_a(const FastTerms& t, int ch) {
  return top32(t.A0 + (uint64_t)ch * t.dA);
}
__device__ __forceinline__ uint32_t chan_c(const FastTerms& t, int ch, int N) {
  return top32((uint64_t)ch * t.G + (uint64_t)(ch / N) * t.Bm);
}

// Bytes of one 16-bit part of one chunk's slow-time operand image (2 NT rows of 128 B).
inline size_t bimg_part_bytes(int nt) { return (size_t)2 * nt * 128; }

// Launches (all asynchronous on `st`).  `frames` is a device array of F FrameIO.
// Compaction and phases.  `one` (F == 1 only, else NULL): the frame's entry, which the
// first kernel stores to frames[0] (no upload needed); the kernels also clear each
// frame's meta words and, when `counter` is given, the contraction's work-unit counter.
// defer_fast_terms: write only the index, the slow-time phase and sigma; the fast-time and
// channel phases (phA, phC) are left to the tensor tiers' operand builder.
cudaError_t launch_prep(const Consts& k, FrameIO* frames, const FrameIO* one, int F, int64_t maxP,
                        int dtype, bool write_idx_only, bool defer_fast_terms, unsigned* status, int* counter,
                        cudaStream_t st, bool cooperative = true, int* launched = nullptr);
// tile_n: n values per CTA tile (64 or 128).
cudaError_t launch_direct(const Consts& k, const FrameIO* frames, int F, int splits, int tile_n,
                          int out_dtype, cudaStream_t st);
cudaError_t launch_reduce(const Consts& k, const FrameIO* frames, int F, int splits, int out_dtype,
                          float scale_from_meta, cudaStream_t st);
// The same reduction over the tensor tiers' tiled partial sums.
cudaError_t launch_reduce_tiles(const Consts& k, const FrameIO* frames, int F, int splits, int nt,
                                int out_dtype, bool scale_from_meta, int num_sms, cudaStream_t st);
// nt: column tile (l values, multiple of 8 in 8..128); group: chunks per accumulation
// group.  fast_terms_dtype: RSIM_F32 / RSIM_F64 when the operand builder is to write the
// fast-time and channel phases (launch_prep deferred them; the pixels' dtype), or -1.
// mid: an event recorded between the operand builder and the contraction kernel
// (profiling), or NULL.
cudaError_t launch_umma(const Consts& k, const FrameIO* frames, int F, int splits, int tier,
                        int out_dtype, int grid, int nt, int group, bool use_partial, int num_sms,
                        int64_t max_p, int fast_terms_dtype, unsigned* status, int* unit_counter,
                        cudaStream_t st, cudaEvent_t mid = nullptr);

cudaError_t launch_range_doppler(const float2* const* cubes_dev, float2* tmp, float* power, int F,
                                 int V, int Ns, int L, int skip_static, double v_per_bin, float* v_est,
                                 int32_t* peak, cudaStream_t st);

// Plan rules shared by single-frame and batch paths (they depend on the shape only).
// tile_n: the plan's tile (tensor tiers: column tile NT; FP32: n per CTA tile).
int default_splits(int tier, int V, int Ns, int L, int tile_n, int64_t P, int num_sms);
int units_per_split(int tier, int V, int Ns, int L, int tile_n);
// Default and largest chunks accumulated in one tensor-memory accumulator before it is
// drained into an FP32 running sum (the tensor-core accumulator rounds toward zero, so
// the length bounds the error; see k_umma.cu).
int group_chunks(int tier);
int group_chunks_max(int tier);
// Default n tile of the FP32 direct sum, and its l tile (fixed).
constexpr int kDirectTileN = 128;
constexpr int kDirectTileL = 64;
// Whether a frame of P pixels goes through the split-partial buffer + reduction.
bool uses_partial(int tier, int64_t P, int splits, int group);

// Plans: the default for a shape, defaults filled into zero tile fields, and validity
// (an empty string when the plan can run this shape at this tier's accuracy).
rsim_plan default_plan(int tier, const Consts& k, int64_t P, int num_sms);
void resolve_tile(int tier, const Consts& k, rsim_plan* p);
std::string plan_problem(int tier, const Consts& k, const rsim_plan& p);

}  // namespace rsim
