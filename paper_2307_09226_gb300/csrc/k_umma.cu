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
// One persistent CTA per SM, warp-specialised:
//   warps 0-3  produce A for a 128-row tile straight into tensor memory (one row per
//              thread, tcgen05.st), then drain the accumulator (tcgen05.ld) as the
//              epilogue;
//   warps 4-7  produce B (the shared slow-time operand of all row tiles) into shared
//              memory in the 128-byte-swizzled K-major layout the MMA reads;
//   warp 8     allocates tensor memory and one thread issues tcgen05.mma
//              (M = 128, N = 2 NT, K = 16, A from tensor memory, B from shared memory).
// Operands are generated on chip from the FP64-derived fixed-point phases: A has no
// reuse across CTAs and B costs as much to generate as to load, so neither goes
// through HBM.  Stages are handed over with mbarriers; every wait is bounded in time
// and a timeout sets a status bit instead of hanging.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rsim_internal.h"

namespace rsim {
namespace {

constexpr int kStages = 3;                 // operand stages (A in TMEM, B in smem)
constexpr int kPixStages = 6;              // ring of staged per-chunk pixel phases
constexpr int kUnitSlots = 4;              // ring of work-unit ids
constexpr int kMaxCh = 8;                  // channels a row tile may span for staging
constexpr int kThreads = 320;              // 10 warps
constexpr int kBRowsMax = 256;             // N = 2 * NT <= 256
constexpr int kBBytes = kBRowsMax * 128;   // one 16-bit operand part of one stage
constexpr int kStageBytes = 2 * kBBytes;   // hi + lo
constexpr int kAccCols = 256;              // accumulator columns (N <= 256 FP32)
constexpr int kTmemCols = 512;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait, then give up

// Per-chunk pixel data staged by the loader warp (bulk copies from global memory).
struct PixStage {
  uint32_t a[kMaxCh][kChunkPx];  // fast-time increments of the tile's channels
  uint32_t c[kMaxCh][kChunkPx];  // spatial phases of the tile's channels
  uint32_t b[kChunkPx];          // slow-time increments
  float2 s[kChunkPx];            // sigma
};

struct Shared {
  uint64_t a_full[kStages];
  uint64_t b_full[kStages];
  uint64_t empty[kStages];
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

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   smem_u32(b)),
               "r"(bytes)
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

__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(b))
               : "memory");
}

#define RSIM_R32(x)                                                                              \
  "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]), "r"(x[7]),       \
      "r"(x[8]), "r"(x[9]), "r"(x[10]), "r"(x[11]), "r"(x[12]), "r"(x[13]), "r"(x[14]),          \
      "r"(x[15]), "r"(x[16]), "r"(x[17]), "r"(x[18]), "r"(x[19]), "r"(x[20]), "r"(x[21]),        \
      "r"(x[22]), "r"(x[23]), "r"(x[24]), "r"(x[25]), "r"(x[26]), "r"(x[27]), "r"(x[28]),        \
      "r"(x[29]), "r"(x[30]), "r"(x[31])

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, "
      "%29, %30, %31, %32};" ::"r"(taddr),
      RSIM_R32(v)
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
  int64_t total_units;
  const int32_t* order;  // frames by decreasing valid-pixel count
};

struct Unit {
  int f, mt, nt, s;
  int64_t c0, c1, pv;
  int v_first, span;
};

__device__ __forceinline__ Unit decode(const Geo& g, const FrameIO* frames, const Consts& k,
                                       int64_t u) {
  Unit x;
  x.f = g.order[u / g.upf];
  int r = (int)(u % g.upf);
  x.s = r % g.splits;
  r /= g.splits;
  x.nt = r % g.ntiles;
  x.mt = r / g.ntiles;
  x.pv = (int64_t)frames[x.f].meta[0];
  const int64_t nch = (x.pv + kChunkPx - 1) / kChunkPx;
  x.c0 = nch * x.s / g.splits;
  x.c1 = nch * (x.s + 1) / g.splits;
  const int64_t rows = (int64_t)k.V * k.Ns;
  const int64_t r0 = (int64_t)x.mt * 128;
  const int64_t r1 = (r0 + 127 < rows ? r0 + 127 : rows - 1);
  x.v_first = (int)(r0 / k.Ns);
  x.span = (int)(r1 / k.Ns) - x.v_first + 1;
  return x;
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

// Next work unit id from the ring filled by the loader (-1: no more work).
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

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&sh->a_full[i], 128);
      mbar_init(&sh->b_full[i], 128);
      mbar_init(&sh->empty[i], 1);
    }
    for (int i = 0; i < kPixStages; ++i) {
      mbar_init(&sh->pix_full[i], 1);
      mbar_init(&sh->pix_empty[i], 8);  // 4 A warps + 4 B warps
    }
    for (int i = 0; i < kUnitSlots; ++i) {
      mbar_init(&sh->unit_full[i], 1);
      mbar_init(&sh->unit_empty[i], 9);  // 4 A warps + 4 B warps + the MMA thread
    }
    mbar_init(&sh->acc_full, 1);
    mbar_init(&sh->acc_empty, 128);
    mbar_init(&sh->fin, 1);
    sh->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sh->tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sh->tmem_base;
  const int64_t rows_total = (int64_t)k.V * k.Ns;

  if (warp < 4) {
    // ------------- A producers + accumulator drain: thread = accumulator row -------------
    const int r = warp * 32 + lane;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    uint32_t kk = 0, pk = 0, gi = 0, ui = 0;
    long long u;
    bool alive = true;
    while (alive && next_unit(sh, ui++, status, &u, true)) {
      const Unit x = decode(g, frames, k, u);
      const FrameIO& fr = frames[x.f];
      const int64_t gr = (int64_t)x.mt * 128 + r;
      const bool row_ok = gr < rows_total;
      const int v = row_ok ? (int)(gr / k.Ns) : x.v_first;
      const uint32_t n = row_ok ? (uint32_t)(gr % k.Ns) : 0u;
      const bool staged = x.span <= kMaxCh;
      const int vl = v - x.v_first;
      const uint32_t* pA = fr.phA + (int64_t)v * fr.Pcap;
      const uint32_t* pC = fr.phC + (int64_t)v * fr.Pcap;
      const float oscale = 1.f / sigma_scale(fr, scaled);
      const int l0 = x.nt * g.NT;
      int64_t g0 = x.c0;
      do {
        const int64_t g1 = (x.c1 < g0 + g.group) ? x.c1 : g0 + g.group;
        for (int64_t c = g0; c < g1; ++c, ++kk, ++pk) {
          const uint32_t st = kk % kStages, ph = (kk / kStages) & 1u;
          const uint32_t ps = pk % kPixStages, pph = (pk / kPixStages) & 1u;
          if (!warp_wait(&sh->empty[st], ph ^ 1u, sh, status) ||
              !warp_wait(&sh->pix_full[ps], pph, sh, status)) {
            alive = false;
            break;
          }
          uint32_t hi[32], lo[32];
          const int64_t q0 = c * kChunkPx;
#pragma unroll
          for (int j4 = 0; j4 < kChunkPx; j4 += 4) {
            uint4 a4, c4;
            if (staged) {
              a4 = *reinterpret_cast<const uint4*>(&pix[ps].a[vl][j4]);
              c4 = *reinterpret_cast<const uint4*>(&pix[ps].c[vl][j4]);
            } else {
              a4 = *reinterpret_cast<const uint4*>(pA + q0 + j4);
              c4 = *reinterpret_cast<const uint4*>(pC + q0 + j4);
            }
            const uint32_t av[4] = {a4.x, a4.y, a4.z, a4.w};
            const uint32_t cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              float2 f = cis_q32(av[t] * n + cv[t]);
              if (!row_ok || q0 + j4 + t >= x.pv) f = make_float2(0.f, 0.f);
              split2<BF>(f.x, f.y, hi[j4 + t], lo[j4 + t]);
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh->pix_empty[ps]);
          const uint32_t col = tmem + lane_base + kAccCols + st * 64;
          tmem_st32(col, hi);
          if (SPLIT) tmem_st32(col + 32, lo);
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          fence_before();
          mbar_arrive(&sh->a_full[st]);
        }
        if (!alive) break;
        // ---- drain this group's accumulator (round-to-nearest FP32 adds) ----
        if (!warp_wait(&sh->acc_full, gi & 1u, sh, status)) {
          alive = false;
          break;
        }
        fence_after();
        const bool none = (g1 <= g0), first = (g0 == x.c0);
        for (int j0 = 0; j0 < g.NT; j0 += 8) {
          uint32_t re[8], im[8];
          if (!none) {
            tmem_ld8(tmem + lane_base + j0, re);
            tmem_ld8(tmem + lane_base + g.NT + j0, im);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) re[i] = im[i] = 0u;
          }
          if (!row_ok) continue;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int l = l0 + j0 + i;
            if (l >= k.L) break;
            const int64_t o = gr * k.L + l;
            const float a = __uint_as_float(re[i]), b = __uint_as_float(im[i]);
            if (g.direct) {
              if (out_dtype == RSIM_C128)
                reinterpret_cast<double2*>(fr.cube)[o] = make_double2((double)a * oscale, (double)b * oscale);
              else
                reinterpret_cast<float2*>(fr.cube)[o] = make_float2(a * oscale, b * oscale);
            } else {
              float2* dst = fr.partial + (int64_t)x.s * rows_total * k.L + o;
              if (first) {
                *dst = make_float2(a, b);
              } else {
                const float2 p = *dst;
                *dst = make_float2(p.x + a, p.y + b);
              }
            }
          }
        }
        fence_before();
        mbar_arrive(&sh->acc_empty);
        ++gi;
        g0 = g1;
      } while (g0 < x.c1);
    }
  } else if (warp < 8) {
    // ------------- B producers: sigma x slow-time phasors, real-embedded -------------
    const int t = threadIdx.x - 128;
    uint32_t kk = 0, pk = 0, ui = 0;
    long long u;
    bool alive = true;
    while (alive && next_unit(sh, ui++, status, &u, true)) {
      const Unit x = decode(g, frames, k, u);
      const FrameIO& fr = frames[x.f];
      const float sc = sigma_scale(fr, scaled);
      const int l0 = x.nt * g.NT;
      for (int64_t c = x.c0; c < x.c1; ++c, ++kk, ++pk) {
        const uint32_t st = kk % kStages, ph = (kk / kStages) & 1u;
        const uint32_t ps = pk % kPixStages, pph = (pk / kPixStages) & 1u;
        if (!mbar_wait(&sh->empty[st], ph ^ 1u, sh, status) ||
            !mbar_wait(&sh->pix_full[ps], pph, sh, status)) {
          alive = false;
          break;
        }
        unsigned char* bhi = bstage + st * kStageBytes;
        unsigned char* blo = bhi + kBBytes;
        const int64_t q0 = c * kChunkPx;
        for (int e = t; e < g.NT * 8; e += 128) {
          const int lt = e % g.NT, qg = e / g.NT;
          const int l = l0 + lt;
          const uint4 b4 = *reinterpret_cast<const uint4*>(&pix[ps].b[qg * 4]);
          const float4 s01 = *reinterpret_cast<const float4*>(&pix[ps].s[qg * 4]);
          const float4 s23 = *reinterpret_cast<const float4*>(&pix[ps].s[qg * 4 + 2]);
          const uint32_t bv[4] = {b4.x, b4.y, b4.z, b4.w};
          const float sr[4] = {s01.x, s01.z, s23.x, s23.z};
          const float si[4] = {s01.y, s01.w, s23.y, s23.w};
          uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            float dre = 0.f, dim = 0.f;
            if (l < k.L && q0 + qg * 4 + i < x.pv) {
              const float2 w = cis_q32(bv[i] * (uint32_t)l);
              const float a = sr[i] * sc, b = si[i] * sc;
              dre = a * w.x - b * w.y;
              dim = a * w.y + b * w.x;
            }
            split2<BF>(dre, -dim, rh[i], rl[i]);  // row l      : (Re D, -Im D)
            split2<BF>(dim, dre, ih[i], il[i]);   // row NT + l : (Im D,  Re D)
          }
          const int rre = lt, rim = g.NT + lt;
          const uint32_t ore = rre * 128 + (((uint32_t)qg ^ (rre & 7)) << 4);
          const uint32_t oim = rim * 128 + (((uint32_t)qg ^ (rim & 7)) << 4);
          *reinterpret_cast<uint4*>(bhi + ore) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
          *reinterpret_cast<uint4*>(bhi + oim) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
          if (SPLIT) {
            *reinterpret_cast<uint4*>(blo + ore) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
            *reinterpret_cast<uint4*>(blo + oim) = make_uint4(il[0], il[1], il[2], il[3]);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh->pix_empty[ps]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&sh->b_full[st]);
      }
    }
  } else if (warp == 8) {
    // ------------- MMA issuer (one thread) -------------
    if (lane == 0) {
      uint32_t kk = 0, gi = 0, ui = 0;
      long long u;
      bool alive = true;
      while (alive && next_unit(sh, ui++, status, &u, false)) {
        const Unit x = decode(g, frames, k, u);
        int64_t g0 = x.c0;
        do {
          const int64_t g1 = (x.c1 < g0 + g.group) ? x.c1 : g0 + g.group;
          if (!mbar_wait(&sh->acc_empty, (gi & 1u) ^ 1u, sh, status)) {
            alive = false;
            break;
          }
          fence_after();
          uint32_t accum = 0;
          for (int64_t c = g0; c < g1; ++c, ++kk) {
            const uint32_t st = kk % kStages, ph = (kk / kStages) & 1u;
            if (!mbar_wait(&sh->a_full[st], ph, sh, status) || !mbar_wait(&sh->b_full[st], ph, sh, status)) {
              alive = false;
              break;
            }
            fence_after();
            const uint32_t a_hi = tmem + kAccCols + st * 64, a_lo = a_hi + 32;
            const uint32_t b_hi = smem_u32(bstage + st * kStageBytes), b_lo = b_hi + kBBytes;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              mma_ts(tmem, a_hi + ks * 8, sdesc_sw128(b_hi + ks * 32), idesc, accum);
              accum = 1;
              if (SPLIT) {
                mma_ts(tmem, a_hi + ks * 8, sdesc_sw128(b_lo + ks * 32), idesc, 1);
                mma_ts(tmem, a_lo + ks * 8, sdesc_sw128(b_hi + ks * 32), idesc, 1);
              }
            }
            mma_commit(&sh->empty[st]);
          }
          if (!alive) break;
          if (g1 > g0)
            mma_commit(&sh->acc_full);
          else
            mbar_arrive(&sh->acc_full);
          ++gi;
          g0 = g1;
        } while (g0 < x.c1);
      }
      // every issued MMA completes before tensor memory is released
      mma_commit(&sh->fin);
      mbar_wait(&sh->fin, 0, sh, status);
    }
  } else {
    // ------------- loader: work units + bulk copies of per-chunk pixel phases -------------
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
          const int64_t q0 = c * kChunkPx;
          const uint32_t bytes = 4 * kChunkPx + 8 * kChunkPx + (staged ? 8u * kChunkPx * x.span : 0u);
          mbar_expect_tx(&sh->pix_full[ps], bytes);
          bulk_g2s(pix[ps].b, fr.phB + q0, 4 * kChunkPx, &sh->pix_full[ps]);
          bulk_g2s(pix[ps].s, fr.sig + q0, 8 * kChunkPx, &sh->pix_full[ps]);
          if (staged) {
            for (int i = 0; i < x.span; ++i) {
              const int64_t ro = (int64_t)(x.v_first + i) * fr.Pcap + q0;
              bulk_g2s(pix[ps].a[i], fr.phA + ro, 4 * kChunkPx, &sh->pix_full[ps]);
              bulk_g2s(pix[ps].c[i], fr.phC + ro, 4 * kChunkPx, &sh->pix_full[ps]);
            }
          }
        }
        if (!alive) break;
      }
    }
  }

  fence_before();
  __syncthreads();
  if (warp == 8) {
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
cudaError_t launch_t(const Consts& k, const FrameIO* frames, const Geo& g, int grid, int scaled,
                     int out_dtype, unsigned* status, int* counter, cudaStream_t st) {
  const int smem = kStages * kStageBytes + kPixStages * (int)sizeof(PixStage) + (int)sizeof(Shared) + 1024;
  auto fn = umma_contract<BF, SPLIT>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, kThreads, smem, st>>>(frames, k, g, scaled, out_dtype, status, counter);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_umma(const Consts& k, const FrameIO* frames, int F, int splits, int tier,
                        int out_dtype, int grid, bool use_partial, int num_sms, unsigned* status,
                        int* unit_counter, cudaStream_t st) {
  Geo g;
  const int64_t rows = (int64_t)k.V * k.Ns;
  g.NT = k.L >= 128 ? 128 : ((k.L + 7) / 8) * 8;
  g.ntiles = (k.L + g.NT - 1) / g.NT;
  g.mtiles = (int)((rows + 127) / 128);
  g.splits = splits;
  g.upf = g.mtiles * g.ntiles * splits;
  g.group = group_chunks(tier);
  g.direct = use_partial ? 0 : 1;
  g.F = F;
  g.total_units = (int64_t)g.upf * F;
  if (g.total_units <= 0) return cudaSuccess;
  // the unit counter (int) and the frame order (F ints) share the counter region
  int32_t* order = unit_counter + 4;
  g.order = order;
  order_frames<<<1, 256, 0, st>>>(frames, F, order);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int blocks = grid > 0 ? grid : num_sms;
  if (blocks > g.total_units) blocks = (int)g.total_units;
  switch (tier) {
    case RSIM_TIER_BF16:
      return launch_t<1, 0>(k, frames, g, blocks, 0, out_dtype, status, unit_counter, st);
    case RSIM_TIER_SPLIT_BF16:
      return launch_t<1, 1>(k, frames, g, blocks, 0, out_dtype, status, unit_counter, st);
    case RSIM_TIER_SPLIT_FP16:
      return launch_t<0, 1>(k, frames, g, blocks, 1, out_dtype, status, unit_counter, st);
    case RSIM_TIER_FP16:
      return launch_t<0, 0>(k, frames, g, blocks, 1, out_dtype, status, unit_counter, st);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace rsim
