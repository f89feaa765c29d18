// Factorised contraction of Eq. 2 on the tcgen05 tensor cores (sm_103a).
//
// The phase of Eq. 2 splits into a fast-time/channel phasor F_v[q][n] =
// exp(j 2 pi (a_{q,v} n + c_{q,v})) and a slow-time phasor D[q][l] = sigma_q
// exp(j 2 pi b_q l), so the cube of every channel is a complex matrix product over
// the compacted valid pixels q.  Stacking the channels gives one real GEMM
//     [C_re | C_im] (rows (v, n), V*N_s of them)  =  A_r * B_r,
//     A_r[(v,n)][2q + {0,1}] = (Re F, Im F),
//     B_r[2q + {0,1}][l]     = (Re D, -Im D),   B_r[2q + {0,1}][NT + l] = (Im D, Re D),
// with K = 2 * (valid pixels) and N = 2 * NT columns per column tile (NT <= 128
// values of l).  Split-precision tiers write each operand as hi + lo 16-bit parts and
// accumulate A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32.
//
// B (sigma x slow-time phasors) is shared by every row tile, so an operand-builder
// kernel writes it once per frame as ready-made shared-memory images: for each
// 32-pixel chunk, 2 NT rows of 128 B in the 128-byte-swizzled K-major layout the MMA
// reads.  Blocks of the same kernel compute the frame's FP64 fast-time and channel
// phases (which A is made from) beside the image blocks.  A (fast-time/channel
// phasors) differs for every row tile and is never reused, so it is generated on chip
// and never touches HBM.
//
// The contraction runs one persistent CTA per SM, warp-specialised:
//   warps 0-15  produce A for a 128-row tile straight into tensor memory (one row per
//               thread, tcgen05.st).  Two groups of 8 warps take alternate stages; in a
//               stage, two warps share a lane quarter with 16 pixels each.  The same
//               warps drain the accumulator (tcgen05.ld) after each group of chunks;
//   warp 16     allocates tensor memory and one thread issues tcgen05.mma
//               (M = 128, N = 2 NT, K = 16, A from tensor memory, B from shared memory);
//   warp 17     takes work units from a device counter and bulk-copies each chunk's
//               phases of the tile's channels into a shared-memory ring;
//   warp 18     bulk-copies each chunk's B images into the operand stages.
// A and B have rings of their own: four A stages in tensor memory (the columns the
// accumulator leaves free) and three B stages in shared memory (what its 227 KB hold),
// so a producer group has four MMA stages of time, not three, to make its next A stage.
// Each slot of either ring has a "full" mbarrier (the producer group's arrivals, or the
// B copy's bytes) and an "empty" mbarrier, completed by a tcgen05.commit after the MMAs
// that read it.  Every wait is bounded in time and a timeout sets a status bit instead
// of hanging.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rsim_internal.h"

namespace rsim {
namespace {

constexpr int kStages = 3;                 // B operand stages in shared memory (64 KB each: hi + lo)
constexpr int kAStages = 4;                // A operand stages in tensor memory (64 columns each: hi + lo)
constexpr int kPixStages = 6;              // ring of staged per-chunk pixel phases
constexpr int kUnitSlots = 4;              // ring of work-unit ids
constexpr int kMaxCh = 8;                  // channels a row tile may span for staging
constexpr int kAWarps = 16;                // A producers: two groups that take alternate stages
constexpr int kAGroupWarps = kAWarps / 2;  // 8 warps per group, two per lane quarter
constexpr int kAPx = kChunkPx / (kAGroupWarps / 4);  // pixels per A warp per stage
constexpr int kThreads = 32 * (kAWarps + 3);  // + MMA warp, pixel loader, B loader
constexpr int kBRowsMax = 256;             // N = 2 * NT <= 256
constexpr int kBBytes = kBRowsMax * 128;   // one 16-bit operand part of one stage
constexpr int kStageBytes = 2 * kBBytes;   // hi + lo
constexpr int kAccCols = 256;              // accumulator columns (N <= 256 FP32)
constexpr int kTmemCols = 512;
static_assert(kAccCols + kAStages * 64 <= kTmemCols, "accumulator and A stages fit in tensor memory");
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait, then give up

// Per-chunk fast-time/channel phases staged by the pixel loader (bulk copies).
struct PixStage {
  uint32_t a[kMaxCh][kChunkPx];  // fast-time increments of the tile's channels
  uint32_t c[kMaxCh][kChunkPx];  // spatial phases of the tile's channels
};

struct Shared {
  uint64_t a_full[kAStages];   // the A stage is in tensor memory (producer group arrivals)
  uint64_t a_empty[kAStages];  // the MMAs are done with the A stage (it may be rewritten)
  uint64_t b_full[kStages];    // the B stage is in shared memory (bulk-copy bytes)
  uint64_t b_empty[kStages];   // the MMAs are done with the B stage
  uint64_t pix_full[kPixStages];
  uint64_t pix_empty[kPixStages];
  uint64_t unit_full[kUnitSlots];
  uint64_t unit_empty[kUnitSlots];
  uint64_t acc_full;
  uint64_t acc_empty;
  uint64_t fin;
  long long unit[kUnitSlots];
  uint32_t tmem_base;
  int abort;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b))
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of parity `parity` to complete; false on timeout or abort.
__device__ __noinline__ bool mbar_wait(uint64_t* b, uint32_t parity, Shared* sh, unsigned* status) {
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(b, parity)) return true;
    if ((it & 255u) == 255u) {
      if (*(volatile int*)&sh->abort) return false;
      const uint64_t now = globaltimer();
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > kWaitNs) {
        atomicOr(status, kStatusTimeout);
        *(volatile int*)&sh->abort = 1;
        return false;
      }
    }
  }
}

// Inline fast path of mbar_wait for the MMA thread: one probe of a phase that has
// usually completed already, the bounded polling loop only when it has not.
__device__ __forceinline__ bool mbar_wait_fast(uint64_t* b, uint32_t parity, Shared* sh, unsigned* status) {
  return mbar_try(b, parity) || mbar_wait(b, parity, sh, status);
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   smem_u32(b)),
               "r"(bytes)
               : "memory");
}

// L2 eviction priorities.  A chunk's B images are read by every row tile at about the
// same time and then never again, while the split partial sums wait in L2 for the
// reduction after the contraction: the B copies take evict_first and the partial-sum
// stores and reductions evict_last.  (The partial sums are found in L2 by the reduction
// with evict_normal stores too; what it pays for is that most of its reads are served by
// the other die's L2 partition, over the link between the two partitions.)
// bulk_g2s with a createpolicy policy for the source lines:
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// 16-byte store and FP32 add-reduction with a policy (the reduction is one instruction,
// like atomicAdd on a float4, so each address's additions keep the issuing thread's order).
__device__ __forceinline__ void st_hint_v4(float4* a, float4 v, uint64_t policy) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w), "l"(policy)
               : "memory");
}
__device__ __forceinline__ void red_hint_v4(float4* a, float4 v, uint64_t policy) {
  asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w), "l"(policy)
               : "memory");
}

// 1-D bulk copy global -> shared (16-byte aligned, size a multiple of 16) that
// completes `bytes` of the barrier's transaction count.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 128-byte-swizzled K-major shared-memory matrix descriptor (tcgen05 format): rows of
// 128 B, 8-row groups 1024 B apart (stride byte offset), version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, K-major A and B, M = 128.
__host__ __device__ constexpr uint32_t idesc_f16(int bf16, int n) {
  return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

// All MMAs of one 32-pixel operand stage (K = 64 16-bit elements = four K = 16 steps),
// in one block so that nothing is recomputed between issues.  `a`: tensor-memory column
// of the stage's hi A part (the lo part starts 32 columns on); `bd`: shared-memory
// descriptor of the stage's hi B image (the lo image starts kBBytes on).  K step ks
// reads A columns a + 8 ks and B bytes + 32 ks (2 in the descriptor's 16-byte address
// field).  Split tiers add A_hi B_lo and A_lo B_hi after each A_hi B_hi.  `acc` = 0
// starts a new accumulation with the stage's first MMA.
template <int SPLIT>
__device__ __forceinline__ void mma_stage(uint32_t d, uint32_t a, uint64_t bd, uint32_t idesc, uint32_t acc);

template <>
__device__ __forceinline__ void mma_stage<0>(uint32_t d, uint32_t a, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p, t;\n\t"
      "setp.ne.b32 p, %10, 0;\n\t"
      "setp.ne.b32 t, %9, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %5, %9, p;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%2], %6, %9, t;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%3], %7, %9, t;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%4], %8, %9, t;\n\t}" ::"r"(d),
      "r"(a), "r"(a + 8), "r"(a + 16), "r"(a + 24), "l"(bd), "l"(bd + 2), "l"(bd + 4), "l"(bd + 6),
      "r"(idesc), "r"(acc)
      : "memory");
}

template <>
__device__ __forceinline__ void mma_stage<1>(uint32_t d, uint32_t a, uint64_t bd, uint32_t idesc, uint32_t acc) {
  constexpr uint64_t kLo = kBBytes >> 4;
  asm volatile(
      "{\n\t.reg .pred p, t;\n\t"
      "setp.ne.b32 p, %18, 0;\n\t"
      "setp.ne.b32 t, %17, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %9, %17, p;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %13, %17, t;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%5], %9, %17, t;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%2], %10, %17, t;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%2], %14, %17, t;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%6], %10, %17, t;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%3], %11, %17, t;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%3], %15, %17, t;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%7], %11, %17, t;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%4], %12, %17, t;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%4], %16, %17, t;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%8], %12, %17, t;\n\t}" ::"r"(d),
      "r"(a), "r"(a + 8), "r"(a + 16), "r"(a + 24), "r"(a + 32), "r"(a + 40), "r"(a + 48), "r"(a + 56),
      "l"(bd), "l"(bd + 2), "l"(bd + 4), "l"(bd + 6), "l"(bd + kLo), "l"(bd + kLo + 2), "l"(bd + kLo + 4),
      "l"(bd + kLo + 6), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(b))
               : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                 "=r"(v[7])
               : "r"(taddr)
               : "memory");
}

__device__ __forceinline__ float2 cis_q32(uint32_t ph) {
  const float ang = (float)(int32_t)ph * 1.46291807926715968e-09f;  // 2 pi / 2^32
  float s, c;
  __sincosf(ang, &s, &c);
  return make_float2(c, s);
}

// exp(j 2 pi x) for a 2^-32-cycle phase, the fraction taken from the top 23 bits by
// placing them in the mantissa of a float in [1, 2) (no integer-to-float conversion);
// the quantisation to 2^-23 cycle adds at most 7.5e-7 rad.
__device__ __forceinline__ float2 cis_q32_fast(uint32_t ph) {
  const float x = __int_as_float(0x3F800000u | ((ph ^ 0x80000000u) >> 9)) - 1.5f;  // [-1/2, 1/2)
  float s, c;
  __sincosf(x * 6.28318530717958648f, &s, &c);
  return make_float2(c, s);
}

// Split (x, y) into 16-bit hi and lo pairs, packed low = x, high = y.
template <int BF>
__device__ __forceinline__ void split2(float x, float y, uint32_t& hi, uint32_t& lo) {
  if (BF) {
    __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
    float2 hf = __bfloat1622float2(h);
    __nv_bfloat162 l = __floats2bfloat162_rn(x - hf.x, y - hf.y);
    hi = *reinterpret_cast<uint32_t*>(&h);
    lo = *reinterpret_cast<uint32_t*>(&l);
  } else {
    __half2 h = __floats2half2_rn(x, y);
    float2 hf = __half22float2(h);
    __half2 l = __floats2half2_rn(x - hf.x, y - hf.y);
    hi = *reinterpret_cast<uint32_t*>(&h);
    lo = *reinterpret_cast<uint32_t*>(&l);
  }
}

struct Geo {
  int mtiles, ntiles, NT, splits, upf, group, direct, F;
  int64_t total_units;   // work units (frame, row tile, column tile, split)
  int64_t sstride;       // complex elements of one split's tiled partial sums
  const int32_t* order;  // frames by decreasing valid-pixel count
};

struct Unit {
  int f, mt, nt, s;
  int64_t c0, c1, pv;
  int v_first, span;
};

__device__ __forceinline__ Unit decode(const Geo& g, const FrameIO* frames, const Consts& k, int64_t u) {
  Unit x;
  x.f = g.order ? g.order[u / g.upf] : (int)(u / g.upf);
  // row tile fastest: the CTAs running at the same time share a pixel range and so the
  // same slow-time operand images in L2
  int r = (int)(u % g.upf);
  x.mt = r % g.mtiles;
  r /= g.mtiles;
  x.nt = r % g.ntiles;
  x.s = r / g.ntiles;
  x.pv = (int64_t)frames[x.f].meta[0];
  const int64_t nch = (x.pv + kChunkPx - 1) / kChunkPx;
  x.c0 = nch * x.s / g.splits;
  x.c1 = nch * (x.s + 1) / g.splits;
  const int64_t rows = (int64_t)k.V * k.Ns;
  const int64_t r0 = (int64_t)x.mt * 128;
  const int64_t r1 = (r0 + 127 < rows ? r0 + 127 : rows - 1);
  x.v_first = (int)(r0 / k.Ns);
  x.span = (r0 < rows) ? (int)(r1 / k.Ns) - x.v_first + 1 : 0;
  return x;
}

// Accumulation groups of a unit: its chunks c0 .. c1 - 1 cut into the fewest equal groups
// of at most `gmax` chunks, one drain each (a unit without chunks still has one group,
// whose drain writes zeros).  Equal groups spend no drain on a short tail group.
__device__ __forceinline__ int64_t unit_groups(const Unit& x, int gmax) {
  const int64_t n = x.c1 - x.c0;
  return n > 0 ? (n + gmax - 1) / gmax : 1;
}
__device__ __forceinline__ int64_t group_begin(const Unit& x, int64_t ngr, int64_t k) {
  return x.c0 + (x.c1 - x.c0) * k / ngr;
}

// sigma scale of the FP16 tiers: 2^-e with max(|re|, |im|) * 2^-e in [1/2, 1)
__device__ __forceinline__ float sigma_scale(const FrameIO& fr, int scaled) {
  if (!scaled) return 1.f;
  const float m = __uint_as_float((unsigned)fr.meta[1]);
  return m > 0.f ? ldexpf(1.f, -(ilogbf(m) + 1)) : 1.f;
}

// Warp-collective wait: all lanes poll, the decision is made uniform.
__device__ __forceinline__ bool warp_wait(uint64_t* b, uint32_t parity, Shared* sh, unsigned* status) {
  return __all_sync(0xffffffffu, mbar_wait(b, parity, sh, status));
}

// Next work unit id from the ring filled by the pixel loader (-1: no more work).
__device__ __forceinline__ bool next_unit(Shared* sh, uint32_t ui, unsigned* status, long long* u,
                                          bool warp_collective) {
  const uint32_t slot = ui % kUnitSlots, ph = (ui / kUnitSlots) & 1u;
  const bool ok = warp_collective ? warp_wait(&sh->unit_full[slot], ph, sh, status)
                                  : mbar_wait(&sh->unit_full[slot], ph, sh, status);
  if (!ok) return false;
  *u = *(volatile long long*)&sh->unit[slot];
  if (warp_collective) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&sh->unit_empty[slot]);
  } else {
    mbar_arrive(&sh->unit_empty[slot]);
  }
  return *u >= 0;
}

// ---------------------------------------------------------------------------------
// Operand builder: B images.  For frame f, column tile nt and chunk c, writes
//   hi: 2 NT rows x 128 B, row lt (< NT) = pixels' (Re D, -Im D) at l = nt NT + lt,
//       row NT + lt = (Im D, Re D), with D = sigma e^{j 2 pi b l} (scaled for FP16),
//       16-byte units placed at (unit ^ (row & 7)) as the 128-byte swizzle wants;
//   lo: the same for the low parts of the split tiers.
// With fast_dtype >= 0 (the compaction deferred them) the first F * ph_blocks blocks
// write the fast-time and channel phases phA / phC instead, one valid pixel per thread
// (read through the index list, pixel arrays of that dtype): their FP64 trigonometry
// runs on the SMs beside the image blocks' memory-bound work.
// ---------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ FastTerms gather_fast_terms(const Consts& k, const FrameIO& fr, int64_t p) {
  const double r = (double)((const T*)fr.range)[p], a = (double)((const T*)fr.az)[p];
  const double e = (double)((const T*)fr.el)[p], w = (double)((const T*)fr.vel)[p];
  const double sr = (double)((const T*)fr.sre)[p], si = (double)((const T*)fr.sim)[p];
  FastTerms t = {0, 0, 0, 0};
  if (pixel_ok(r, a, e, w, sr, si)) t = fast_terms(k, r, a, e, w);
  return t;
}

template <int BF, int SPLIT>
__global__ void __launch_bounds__(256, 6)
build_b_images(const FrameIO* __restrict__ frames, Consts k, int NT, int ntiles, int64_t nch, int F,
               int scaled, int fast_dtype, int ph_blocks) {
  wait_prior_grid();
  const int nph = fast_dtype >= 0 ? F * ph_blocks : 0;
  if ((int)blockIdx.x < nph) {
    const FrameIO& fr = frames[blockIdx.x / ph_blocks];
    const int64_t q = (int64_t)(blockIdx.x % ph_blocks) * blockDim.x + threadIdx.x;
    if (q < (int64_t)fr.meta[0]) {
      const int64_t p = fr.idx[q];
      const FastTerms t =
          fast_dtype == RSIM_F64 ? gather_fast_terms<double>(k, fr, p) : gather_fast_terms<float>(k, fr, p);
      for (int ch = 0; ch < k.V; ++ch) {
        fr.phA[(int64_t)ch * fr.Pcap + q] = chan_a(t, ch);
        fr.phC[(int64_t)ch * fr.Pcap + q] = chan_c(t, ch, k.N);
      }
    }
    return;
  }
  const size_t part = (size_t)2 * NT * 128;
  const int64_t items = (int64_t)F * ntiles * nch;
  // one chunk image per block and pass, chunks of a column tile consecutive
  for (int64_t it = blockIdx.x - nph; it < items; it += gridDim.x - nph) {
    const int64_t c = it % nch;
    const int nt = (int)((it / nch) % ntiles);
    const FrameIO& fr = frames[it / (nch * ntiles)];
    const int64_t pv = (int64_t)fr.meta[0];
    if (c * kChunkPx >= pv) continue;
    const float sc = sigma_scale(fr, scaled);
    unsigned char* base = fr.bimg + ((int64_t)nt * fr.bimg_nch + c) * 2 * part;
    const int64_t q0c = c * kChunkPx;
    // element (l, 16-byte column cp): four pixels' D at l, written to the re-row l and
    // the im-row NT + l, which share a swizzle pattern (NT is a multiple of 8).  A thread's
    // elements e, e + 256, ... keep cp = e & 7 and row & 7, so they share the four pixels
    // qg = cp ^ (row & 7): their phases and strengths are loaded once.
    const int cp = threadIdx.x & 7;
    const int qg = cp ^ ((threadIdx.x >> 3) & 7);
    const int64_t q0 = q0c + qg * 4;
    const uint4 b4 = *reinterpret_cast<const uint4*>(fr.phB + q0);
    const float4 s01 = *reinterpret_cast<const float4*>(fr.sig + q0);
    const float4 s23 = *reinterpret_cast<const float4*>(fr.sig + q0 + 2);
    const uint32_t bv[4] = {b4.x, b4.y, b4.z, b4.w};
    const float sa[4] = {s01.x * sc, s01.z * sc, s23.x * sc, s23.z * sc};
    const float sb[4] = {s01.y * sc, s01.w * sc, s23.y * sc, s23.w * sc};
    for (int e = threadIdx.x; e < NT * 8; e += blockDim.x) {
      const int row = e >> 3;
      const int l = nt * NT + row;
      uint32_t rhi[4], rlo[4], ihi[4], ilo[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float dre = 0.f, dim = 0.f;
        if (l < k.L && q0 + i < pv) {
          const float2 w = cis_q32(bv[i] * (uint32_t)l);
          dre = sa[i] * w.x - sb[i] * w.y;
          dim = sa[i] * w.y + sb[i] * w.x;
        }
        split2<BF>(dre, -dim, rhi[i], rlo[i]);
        // the im-row pair (dim, dre): the re-row pair (dre, -dim) with its 16-bit halves
        // swapped and the new low half negated (rounding to nearest is odd, so these are
        // the values a second split would give; only a zero may change sign)
        ihi[i] = __byte_perm(rhi[i], 0, 0x1032) ^ 0x8000u;
        ilo[i] = __byte_perm(rlo[i], 0, 0x1032) ^ 0x8000u;
      }
      const size_t off = (size_t)row * 128 + cp * 16, ioff = off + (size_t)NT * 128;
      *reinterpret_cast<uint4*>(base + off) = make_uint4(rhi[0], rhi[1], rhi[2], rhi[3]);
      *reinterpret_cast<uint4*>(base + ioff) = make_uint4(ihi[0], ihi[1], ihi[2], ihi[3]);
      if (SPLIT) {
        *reinterpret_cast<uint4*>(base + part + off) = make_uint4(rlo[0], rlo[1], rlo[2], rlo[3]);
        *reinterpret_cast<uint4*>(base + part + ioff) = make_uint4(ilo[0], ilo[1], ilo[2], ilo[3]);
      }
    }
  }
}

template <int BF, int SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
umma_contract(const FrameIO* __restrict__ frames, Consts k, Geo g, int scaled, int out_dtype,
              unsigned* status, int* unit_counter) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* bstage = smem;  // kStages x (hi, lo) x 32 KB, 1024-aligned
  PixStage* pix = (PixStage*)(smem + kStages * kStageBytes);
  Shared* sh = (Shared*)(pix + kPixStages);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = 2 * g.NT;
  const uint32_t idesc = idesc_f16(BF, N);
  const uint32_t part = (uint32_t)(2 * g.NT * 128);

  if (threadIdx.x == 0) {
    for (int i = 0; i < kAStages; ++i) {
      mbar_init(&sh->a_full[i], 32 * kAGroupWarps);  // the threads of one producer group
      mbar_init(&sh->a_empty[i], 1);
    }
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&sh->b_full[i], 1);  // the B loader's arrival with the bytes expected
      mbar_init(&sh->b_empty[i], 1);
    }
    for (int i = 0; i < kPixStages; ++i) {
      mbar_init(&sh->pix_full[i], 1);
      mbar_init(&sh->pix_empty[i], kAGroupWarps);
    }
    for (int i = 0; i < kUnitSlots; ++i) {
      mbar_init(&sh->unit_full[i], 1);
      mbar_init(&sh->unit_empty[i], kAWarps + 2);  // A warps, the MMA thread, the B loader
    }
    mbar_init(&sh->acc_full, 1);
    mbar_init(&sh->acc_empty, 32 * kAWarps);
    mbar_init(&sh->fin, 1);
    sh->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kAWarps) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sh->tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  wait_prior_grid();  // the set-up above overlaps the operand builder's last blocks
  const uint32_t tmem = sh->tmem_base;
  const int64_t rows_total = (int64_t)k.V * k.Ns;

  if (warp < kAWarps) {
    // ------- A producers + accumulator drain: thread = accumulator row, kAPx pixels -------
    // A entries of padded pixels and of rows past the cube need no masking: the B image
    // rows of padded pixels are zero, and rows past the cube are never written out.
    // A finished group's drain waits until this warp has made its first stage of the next
    // group (the stage's ring slot belongs to MMAs already issued, so nothing there waits
    // on the drain): the MMAs of the next group then start on a ready stage as soon as the
    // accumulator is read out, instead of waiting for A to be made after the drain.
    const int quarter = warp & 3, part = (warp >> 2) & 1, group = warp >> 3;
    const int r = quarter * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    uint32_t kk = 0, pk = 0, gi = 0, ui = 0;
    long long u;
    bool alive = true;
    // the group whose drain is pending
    struct Pending {
      const FrameIO* fr;
      int64_t gr;
      float oscale;
      int l0, s, mt, nt;
      bool row_ok, none, first, set;
    };
    Pending pend;
    pend.set = false;
    const uint64_t pol_p = policy_evict_last();
    auto drain = [&](const Pending& d) -> bool {
      if (!warp_wait(&sh->acc_full, gi & 1u, sh, status)) return false;
      fence_after();
      const FrameIO& dfr = *d.fr;
      for (int jb = ((warp >> 2) & 3) * 8; jb < g.NT; jb += 8 * (kAWarps / 4)) {
        uint32_t re[8], im[8];
        if (!d.none) {
          tmem_ld8(tmem + lane_base + jb, re);
          tmem_ld8(tmem + lane_base + g.NT + jb, im);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) re[i] = im[i] = 0u;
        }
        if (!d.row_ok) continue;
        if (g.direct) {
#pragma unroll
          for (int i = 0; i < 8; i += 2) {
            const int l = d.l0 + jb + i;
            if (l >= k.L) break;
            const float a0 = __uint_as_float(re[i]), b0 = __uint_as_float(im[i]);
            const float a1 = __uint_as_float(re[i + 1]), b1 = __uint_as_float(im[i + 1]);
            const bool two = (l + 1 < k.L);
            const int64_t o = d.gr * k.L + l;
            if (out_dtype == RSIM_C128) {
              double2* cd = reinterpret_cast<double2*>(dfr.cube);
              cd[o] = make_double2((double)a0 * d.oscale, (double)b0 * d.oscale);
              if (two) cd[o + 1] = make_double2((double)a1 * d.oscale, (double)b1 * d.oscale);
            } else {
              float2* cf = reinterpret_cast<float2*>(dfr.cube);
              cf[o] = make_float2(a0 * d.oscale, b0 * d.oscale);
              if (two) cf[o + 1] = make_float2(a1 * d.oscale, b1 * d.oscale);
            }
          }
        } else {
          // tiled partial sums: column pair p of accumulator row r is float4 p * 128 + r of
          // the tile, so the warp's 32 rows write 512 contiguous bytes.  Later groups are
          // added with reductions: no load round trip, and one thread owns each address, so
          // its additions land in program order (deterministic).  Columns past L (last
          // column tile) land in the tile's padding and are never read.
          float4* t4 = reinterpret_cast<float4*>(dfr.partial + (int64_t)d.s * g.sstride +
                                                 ((int64_t)d.mt * g.ntiles + d.nt) * (128 * g.NT)) +
                       (jb >> 1) * 128 + r;
#pragma unroll
          for (int i = 0; i < 8; i += 2) {
            const float4 v4 = make_float4(__uint_as_float(re[i]), __uint_as_float(im[i]),
                                          __uint_as_float(re[i + 1]), __uint_as_float(im[i + 1]));
            if (d.first)
              st_hint_v4(t4 + (i >> 1) * 128, v4, pol_p);
            else
              red_hint_v4(t4 + (i >> 1) * 128, v4, pol_p);
          }
        }
      }
      fence_before();
      mbar_arrive(&sh->acc_empty);
      ++gi;
      return true;
    };
    while (alive && next_unit(sh, ui++, status, &u, true)) {
      const Unit x = decode(g, frames, k, u);
      const FrameIO& fr = frames[x.f];
      const int64_t gr = (int64_t)x.mt * 128 + r;
      const bool row_ok = gr < rows_total;
      const int v = row_ok ? (int)(gr / k.Ns) : x.v_first;
      const uint32_t n = row_ok ? (uint32_t)(gr % k.Ns) : 0u;
      const bool staged = x.span <= kMaxCh;
      const int vl = row_ok ? v - x.v_first : 0;
      const uint32_t* pA = fr.phA + (int64_t)(row_ok ? v : 0) * fr.Pcap;
      const uint32_t* pC = fr.phC + (int64_t)(row_ok ? v : 0) * fr.Pcap;
      const float oscale = 1.f / sigma_scale(fr, scaled);
      const int l0 = x.nt * g.NT;
      const int64_t ngr = unit_groups(x, g.group);
      for (int64_t gk = 0; gk < ngr; ++gk) {
        const int64_t g0 = group_begin(x, ngr, gk), g1 = group_begin(x, ngr, gk + 1);
        for (int64_t c = g0; c < g1; ++c, ++kk, ++pk) {
          if ((int)(kk & 1u) != group) continue;  // the other group makes this stage
          const uint32_t st = kk % kAStages, ph = (kk / kAStages) & 1u;
          const uint32_t ps = pk % kPixStages, pph = (pk / kPixStages) & 1u;
          if (!warp_wait(&sh->pix_full[ps], pph, sh, status) ||
              !warp_wait(&sh->a_empty[st], ph ^ 1u, sh, status)) {
            alive = false;
            break;
          }
          uint32_t hi[kAPx], lo[kAPx];
          const int j0 = part * kAPx;
          const int64_t q0 = c * kChunkPx + j0;
#pragma unroll
          for (int j4 = 0; j4 < kAPx; j4 += 4) {
            uint4 a4, c4;
            if (staged) {
              a4 = *reinterpret_cast<const uint4*>(&pix[ps].a[vl][j0 + j4]);
              c4 = *reinterpret_cast<const uint4*>(&pix[ps].c[vl][j0 + j4]);
            } else {
              a4 = *reinterpret_cast<const uint4*>(pA + q0 + j4);
              c4 = *reinterpret_cast<const uint4*>(pC + q0 + j4);
            }
            const uint32_t av[4] = {a4.x, a4.y, a4.z, a4.w};
            const uint32_t cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const float2 f = cis_q32_fast(av[t] * n + cv[t]);
              split2<BF>(f.x, f.y, hi[j4 + t], lo[j4 + t]);
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh->pix_empty[ps]);
          static_assert(kAPx == 16, "one x16 tensor-memory store per operand part");
          const uint32_t col = tmem + lane_base + kAccCols + st * 64 + j0;
          tmem_st16(col, hi);
          if (SPLIT) tmem_st16(col + 32, lo);
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          fence_before();
          mbar_arrive(&sh->a_full[st]);
          // the previous group's drain, now that this group's first stage of ours is made
          if (pend.set) {
            if (!drain(pend)) {
              alive = false;
              break;
            }
            pend.set = false;
          }
        }
        if (!alive) break;
        // a group in which this warp made no stage: the previous drain is due now
        if (pend.set) {
          if (!drain(pend)) {
            alive = false;
            break;
          }
        }
        pend = Pending{&fr, gr, oscale, l0, x.s, x.mt, x.nt, row_ok, g1 <= g0, g0 == x.c0, true};
      }
    }
    if (alive && pend.set) drain(pend);  // the last group
  } else if (warp == kAWarps) {
    // ------------- MMA issuer (one thread) -------------
    if (lane == 0) {
      uint32_t kk = 0, gi = 0, ui = 0;
      long long u;
      bool alive = true;
      const uint64_t desc0 = sdesc_sw128(smem_u32(bstage));  // hi image of B stage 0
      while (alive && next_unit(sh, ui++, status, &u, false)) {
        const Unit x = decode(g, frames, k, u);
        const int64_t ngr = unit_groups(x, g.group);
        for (int64_t gk = 0; gk < ngr; ++gk) {
          const int64_t g0 = group_begin(x, ngr, gk), g1 = group_begin(x, ngr, gk + 1);
          if (!mbar_wait(&sh->acc_empty, (gi & 1u) ^ 1u, sh, status)) {
            alive = false;
            break;
          }
          fence_after();
          uint32_t accum = 0;
          for (int64_t c = g0; c < g1; ++c, ++kk) {
            const uint32_t sa = kk % kAStages, pa = (kk / kAStages) & 1u;
            const uint32_t sb = kk % kStages, pb = (kk / kStages) & 1u;
            if (!mbar_wait_fast(&sh->a_full[sa], pa, sh, status) ||
                !mbar_wait_fast(&sh->b_full[sb], pb, sh, status)) {
              alive = false;
              break;
            }
            fence_after();
            mma_stage<SPLIT>(tmem, tmem + kAccCols + sa * 64, desc0 + (uint64_t)(sb * (kStageBytes >> 4)),
                             idesc, accum);
            accum = 1;
            mma_commit(&sh->a_empty[sa]);
            mma_commit(&sh->b_empty[sb]);
          }
          if (!alive) break;
          if (g1 > g0)
            mma_commit(&sh->acc_full);
          else
            mbar_arrive(&sh->acc_full);
          ++gi;
        }
      }
      // every issued MMA completes before tensor memory is released
      mma_commit(&sh->fin);
      mbar_wait(&sh->fin, 0, sh, status);
    }
  } else if (warp == kAWarps + 1) {
    // ------------- pixel loader: work units + bulk copies of the tile's phases -------------
    if (lane == 0) {
      uint32_t pk = 0;
      for (uint32_t ui = 0;; ++ui) {
        const long long uu = (long long)atomicAdd(unit_counter, 1);
        const long long u = uu < g.total_units ? uu : -1;
        const uint32_t slot = ui % kUnitSlots, uph = (ui / kUnitSlots) & 1u;
        if (!mbar_wait(&sh->unit_empty[slot], uph ^ 1u, sh, status)) break;
        *(volatile long long*)&sh->unit[slot] = u;
        mbar_arrive(&sh->unit_full[slot]);
        if (u < 0) break;
        const Unit x = decode(g, frames, k, u);
        const FrameIO& fr = frames[x.f];
        const bool staged = x.span <= kMaxCh;
        bool alive = true;
        for (int64_t c = x.c0; c < x.c1; ++c, ++pk) {
          const uint32_t ps = pk % kPixStages, pph = (pk / kPixStages) & 1u;
          if (!mbar_wait(&sh->pix_empty[ps], pph ^ 1u, sh, status)) {
            alive = false;
            break;
          }
          if (!staged || x.span <= 0) {
            mbar_arrive(&sh->pix_full[ps]);
            continue;
          }
          const int64_t q0 = c * kChunkPx;
          mbar_expect_tx(&sh->pix_full[ps], 8u * kChunkPx * x.span);
          for (int i = 0; i < x.span; ++i) {
            const int64_t ro = (int64_t)(x.v_first + i) * fr.Pcap + q0;
            bulk_g2s(pix[ps].a[i], fr.phA + ro, 4 * kChunkPx, &sh->pix_full[ps]);
            bulk_g2s(pix[ps].c[i], fr.phC + ro, 4 * kChunkPx, &sh->pix_full[ps]);
          }
        }
        if (!alive) break;
      }
    }
  } else {
    // ------------- B loader: bulk copies of the chunk's B images into the operand stage -------------
    if (lane == 0) {
      const uint64_t pol_b = policy_evict_first();
      uint32_t kk = 0, ui = 0;
      long long u;
      bool alive = true;
      while (alive && next_unit(sh, ui++, status, &u, false)) {
        const Unit x = decode(g, frames, k, u);
        const FrameIO& fr = frames[x.f];
        for (int64_t c = x.c0; c < x.c1; ++c, ++kk) {
          const uint32_t st = kk % kStages, ph = (kk / kStages) & 1u;
          if (!mbar_wait(&sh->b_empty[st], ph ^ 1u, sh, status)) {
            alive = false;
            break;
          }
          const unsigned char* src = fr.bimg + ((int64_t)x.nt * fr.bimg_nch + c) * 2 * part;
          unsigned char* dst = bstage + st * kStageBytes;
          mbar_expect_tx(&sh->b_full[st], SPLIT ? 2 * part : part);
          bulk_g2s_hint(dst, src, part, &sh->b_full[st], pol_b);
          if (SPLIT) bulk_g2s_hint(dst + kBBytes, src + part, part, &sh->b_full[st], pol_b);
        }
      }
    }
  }

  fence_before();
  __syncthreads();
  if (warp == kAWarps) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
}

// Frames by decreasing valid-pixel count (ties by index): the persistent kernel takes
// the units of the largest frames first.
__global__ void order_frames(const FrameIO* __restrict__ frames, int F, int32_t* order) {
  for (int f = threadIdx.x; f < F; f += blockDim.x) {
    const unsigned long long pf = frames[f].meta[0];
    int rank = 0;
    for (int h = 0; h < F; ++h) {
      const unsigned long long ph = frames[h].meta[0];
      rank += (ph > pf) || (ph == pf && h < f);
    }
    order[rank] = f;
  }
}

template <int BF, int SPLIT>
cudaError_t launch_t(const Consts& k, const FrameIO* frames, Geo g, int grid, int num_sms, int scaled,
                     int out_dtype, int64_t nch_max, int fast_dtype, unsigned* status, int* counter,
                     cudaStream_t st, cudaEvent_t mid) {
  cudaError_t e;
  if (nch_max > 0) {
    // the phase blocks come first (one valid pixel per thread), then one image block per
    // chunk image (up to 64 per SM, looping beyond): the block scheduler then balances the
    // SMs, where a wave of 8 per SM left some blocks a second image at the end
    const int64_t items = (int64_t)g.F * g.ntiles * nch_max;
    const int ph_blocks = fast_dtype >= 0 ? (int)((nch_max * kChunkPx + 255) / 256) : 0;
    const int64_t blocks = std::min<int64_t>(items, 64ll * num_sms) + (int64_t)g.F * ph_blocks;
    if (blocks > 0x7FFFFFFF) return cudaErrorInvalidValue;
    e = launch_dependent(build_b_images<BF, SPLIT>, dim3((unsigned)blocks), dim3(256), 0, st, frames, k, g.NT,
                         g.ntiles, nch_max, g.F, scaled, fast_dtype, ph_blocks);
    if (e != cudaSuccess) return e;
  }
  if (mid) cudaEventRecord(mid, st);
  const int smem = kStages * kStageBytes + kPixStages * (int)sizeof(PixStage) + (int)sizeof(Shared) + 1024;
  auto fn = umma_contract<BF, SPLIT>;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  // persistent: at most one CTA per SM (shared memory and tensor memory allow no more)
  int ctas = grid > 0 ? std::min(grid, num_sms) : num_sms;
  if (ctas < 1) ctas = 1;
  if (ctas > g.total_units) ctas = (int)g.total_units;
  cfg.gridDim = dim3(ctas);
  return cudaLaunchKernelEx(&cfg, fn, frames, k, g, scaled, out_dtype, status, counter);
}

}  // namespace

cudaError_t launch_umma(const Consts& k, const FrameIO* frames, int F, int splits, int tier,
                        int out_dtype, int grid, int nt, int group, bool use_partial, int num_sms,
                        int64_t max_p, int fast_terms_dtype, unsigned* status, int* unit_counter,
                        cudaStream_t st, cudaEvent_t mid) {
  // N = 2 NT must be a multiple of 16 in 16..256 (kind::f16 with M = 128), and a group
  // holds at least one chunk
  if (nt < 8 || nt > kBRowsMax / 2 || nt % 8 != 0 || group < 1) return cudaErrorInvalidValue;
  Geo g;
  const int64_t rows = (int64_t)k.V * k.Ns;
  g.NT = nt;
  g.ntiles = (k.L + g.NT - 1) / g.NT;
  g.mtiles = (int)((rows + 127) / 128);
  g.splits = splits;
  g.upf = g.mtiles * g.ntiles * splits;
  g.group = group;
  g.direct = use_partial ? 0 : 1;
  g.sstride = tensor_split_stride(k.V, k.Ns, k.L, nt);
  g.F = F;
  g.total_units = (int64_t)g.upf * F;
  if (g.total_units <= 0) {
    if (mid) cudaEventRecord(mid, st);
    return cudaSuccess;
  }
  // the unit counter (int) and the frame order (F ints) share the counter region
  int32_t* order = unit_counter + 4;
  g.order = nullptr;
  cudaError_t e = cudaSuccess;
  if (F > 1) {  // one frame needs no ordering
    g.order = order;
    order_frames<<<1, 256, 0, st>>>(frames, F, order);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int64_t nch_max = (max_p + kChunkPx - 1) / kChunkPx;
  if (fast_terms_dtype >= 0 && fast_terms_dtype != RSIM_F32 && fast_terms_dtype != RSIM_F64)
    return cudaErrorInvalidValue;
  switch (tier) {
    case RSIM_TIER_BF16:
      return launch_t<1, 0>(k, frames, g, grid, num_sms, 0, out_dtype, nch_max, fast_terms_dtype, status, unit_counter, st,
                          mid);
    case RSIM_TIER_SPLIT_BF16:
      return launch_t<1, 1>(k, frames, g, grid, num_sms, 0, out_dtype, nch_max, fast_terms_dtype, status, unit_counter, st,
                          mid);
    case RSIM_TIER_SPLIT_FP16:
      return launch_t<0, 1>(k, frames, g, grid, num_sms, 1, out_dtype, nch_max, fast_terms_dtype, status, unit_counter, st,
                          mid);
    case RSIM_TIER_FP16:
      return launch_t<0, 0>(k, frames, g, grid, num_sms, 1, out_dtype, nch_max, fast_terms_dtype, status, unit_counter, st,
                          mid);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace rsim
