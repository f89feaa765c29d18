// C ABI of librsim: argument checks, context and workspace, plan choice and the
// stage sequence of one synthesis (compaction + FP64 phases -> contraction ->
// ordered split reduction).  Declarations and contracts are in include/rsim.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "rsim_ctx.h"
#include "rsim_internal.h"

namespace rsim {

thread_local std::string g_last_error;

rsim_status fail(rsim_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

rsim_status cuda_fail(cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(RSIM_ERR_CUDA, m);
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// overflow-checked a * b for non-negative 64-bit values
static bool mul_ok(int64_t a, int64_t b, int64_t* out) {
  if (a < 0 || b < 0) return false;
  if (a != 0 && b > INT64_MAX / a) return false;
  *out = a * b;
  return true;
}

FrameLayout frame_layout(int V, int Ns, int L, int64_t P, int splits, bool use_partial, bool tensor,
                         int nt, size_t base) {
  FrameLayout fl{};
  const int64_t Pcap = std::max<int64_t>(64, (P + 63) / 64 * 64);
  fl.Pcap = Pcap;
  size_t o = align_up(base, 256);
  fl.idx = o;      o = align_up(o + 4 * (size_t)Pcap, 256);
  fl.phA = o;      o = align_up(o + 4 * (size_t)Pcap * V, 256);
  fl.phC = o;      o = align_up(o + 4 * (size_t)Pcap * V, 256);
  fl.phB = o;      o = align_up(o + 4 * (size_t)Pcap, 256);
  fl.sig = o;      o = align_up(o + 8 * (size_t)Pcap, 256);
  fl.blk = o;      o = align_up(o + 4 * (size_t)((P + kPrepTile - 1) / kPrepTile + 1), 256);
  fl.meta = 0;     // lives in the batch header
  fl.partial = o;
  if (use_partial) {
    const int64_t per_split = tensor ? tensor_split_stride(V, Ns, L, nt) : (int64_t)V * Ns * L;
    o = align_up(o + 8 * (size_t)splits * per_split, 256);
  }
  // slow-time operand images: [column tile][chunk][hi, lo][2 NT rows x 128 B]
  fl.bimg_nch = Pcap / kChunkPx;
  fl.bimg = align_up(o, 1024);
  o = fl.bimg;
  if (tensor) {
    const int ntiles = (L + nt - 1) / nt;
    o = align_up(o + (size_t)ntiles * fl.bimg_nch * 2 * bimg_part_bytes(nt), 256);
  }
  fl.total = o;
  return fl;
}

rsim_status check_params(const rsim_radar_params* p, Consts* k) {
  if (!p) return fail(RSIM_ERR_INVALID_ARG, "params is NULL");
  if (p->M < 1 || p->N < 1 || p->Ns < 1 || p->L < 1)
    return fail(RSIM_ERR_INVALID_ARG, "M, N, Ns and L must be >= 1");
  if (!(p->lambda > 0) || !isfinite(p->lambda)) return fail(RSIM_ERR_INVALID_ARG, "lambda must be > 0");
  if (!(p->fs > 0) || !isfinite(p->fs)) return fail(RSIM_ERR_INVALID_ARG, "fs must be > 0");
  if (!isfinite(p->mu) || !isfinite(p->t_b) || !isfinite(p->t_slow) || !isfinite(p->d_rx) ||
      !isfinite(p->c))
    return fail(RSIM_ERR_INVALID_ARG, "radar parameters must be finite");
  int64_t V, cells;
  if (!mul_ok(p->M, p->N, &V) || V > (1 << 20)) return fail(RSIM_ERR_OVERFLOW, "M*N too large");
  if (!mul_ok(V, p->Ns, &cells) || !mul_ok(cells, p->L, &cells) || cells > (int64_t(1) << 40))
    return fail(RSIM_ERR_OVERFLOW, "M*N*Ns*L too large");
  const double c = p->c > 0 ? p->c : 299792458.0;
  const double d = p->d_rx > 0 ? p->d_rx : 0.5 * p->lambda;
  const double ts = p->t_slow > 0 ? p->t_slow : p->M * p->t_b;
  k->M = p->M;
  k->N = p->N;
  k->V = (int)V;
  k->Ns = p->Ns;
  k->L = p->L;
  k->k_a0 = 2.0 * p->mu / (c * p->fs);
  k->k_da = p->mu * d / (c * p->fs);
  k->k_g = d / p->lambda;
  k->k_b = -2.0 * ts / p->lambda;
  if (p->flags & ~(RSIM_FLAG_TDM_MOTION | RSIM_NUFFT_WIDTH_MASK))
    return fail(RSIM_ERR_INVALID_ARG, "unknown flag bits");
  k->k_m = (p->flags & RSIM_FLAG_TDM_MOTION) ? -2.0 * p->t_b / p->lambda : 0.0;
  const int w = (p->flags & RSIM_NUFFT_WIDTH_MASK) >> 8;
  if (w != 0 && (w < 4 || w > 8)) return fail(RSIM_ERR_INVALID_ARG, "the NUFFT kernel width must be 4..8");
  k->nu_w = w ? w : 7;
  return RSIM_OK;
}

rsim_status check_pixels(const rsim_pixels* px) {
  if (!px) return fail(RSIM_ERR_INVALID_ARG, "pixels is NULL");
  if (px->P < 0) return fail(RSIM_ERR_INVALID_ARG, "P must be >= 0");
  if (px->P >= (int64_t(1) << 31) - 1024) return fail(RSIM_ERR_OVERFLOW, "P must be < 2^31");
  if (px->dtype != RSIM_F32 && px->dtype != RSIM_F64)
    return fail(RSIM_ERR_INVALID_ARG, "pixel dtype must be RSIM_F32 or RSIM_F64");
  if (px->P > 0 && (!px->range || !px->sigma_re || !px->sigma_im || !px->az || !px->el || !px->vel))
    return fail(RSIM_ERR_INVALID_ARG, "a pixel array pointer is NULL");
  return RSIM_OK;
}

bool tier_ok(int tier) { return tier >= RSIM_TIER_FP32 && tier <= RSIM_TIER_NUFFT; }

// Shape bucket of a plan: the pixel count enters as ceil(log2 P), so frames and requests
// whose counts lie in one power-of-two range share a tuned plan.
std::string plan_key(int tier, const Consts& k, int64_t P) {
  int b = 0;
  while (b < 62 && (int64_t(1) << b) < P) ++b;
  char s[160];
  snprintf(s, sizeof s, "t%d_V%d_Ns%d_L%d_b%d", tier, k.V, k.Ns, k.L, b);
  return s;
}

rsim_plan choose_plan(rsim_ctx* ctx, int tier, const Consts& k, int64_t P) {
  {
    std::lock_guard<std::mutex> g(ctx->plan_mu);
    auto it = ctx->plans.find(plan_key(tier, k, P));
    // a cached plan that cannot run this shape (a cache file written for another build)
    // falls back to the default rule
    if (it != ctx->plans.end() && plan_problem(tier, k, it->second).empty()) {
      rsim_plan p = it->second;
      resolve_tile(tier, k, &p);
      return p;
    }
  }
  return default_plan(tier, k, P, ctx->num_sms);
}

// Workspace bytes of the per-frame regions of F frames of P_f pixels.
size_t frames_bytes(const Consts& k, const int64_t* P, int F, const rsim_plan& plan, int tier) {
  int64_t mp = 0;
  for (int f = 0; f < F; ++f) mp = std::max(mp, P[f]);
  const bool up = uses_partial(tier, mp, plan.splits, plan.group_chunks);
  size_t o = align_up(sizeof(FrameIO) * (size_t)F, 256);  // frame table
  o = align_up(o + 16 * (size_t)F, 256);                  // meta
  o = align_up(o + 16 + 4 * (size_t)F, 256);              // unit counter + frame order
  for (int f = 0; f < F; ++f) {
    FrameLayout fl = frame_layout(k.V, k.Ns, k.L, P[f], plan.splits, up, tensor_tier(tier), plan.tile_n, o);
    o = fl.total;
  }
  return o;
}

// Grid scratch slots of a NUFFT batch: one per stream its frames run on.
int nufft_slots(int F) { return std::max(1, std::min(F, rsim_ctx::kNuStreams)); }

// Workspace bytes for F frames: the per-frame regions, then (NUFFT tier) the grid
// scratch slots that the frames use in turn.
size_t batch_bytes(const Consts& k, const int64_t* P, int F, const rsim_plan& plan, int tier) {
  size_t o = frames_bytes(k, P, F, plan, tier);
  if (tier == RSIM_TIER_NUFFT) {
    int64_t mp = 0;
    for (int f = 0; f < F; ++f) mp = std::max(mp, P[f]);
    o = align_up(o, 256) + (size_t)nufft_slots(F) * align_up(nufft_scratch_bytes(k, mp), 256);
  }
  return o;
}

rsim_status ensure_workspace(rsim_ctx* ctx, size_t bytes, cudaStream_t st) {
  if (ctx->ws_bytes >= bytes) return RSIM_OK;
  if (ctx->budget && bytes > ctx->budget)
    return fail(RSIM_ERR_BUDGET, "workspace of " + std::to_string(bytes) +
                                     " bytes exceeds the context budget of " +
                                     std::to_string(ctx->budget));
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  if (ctx->ws) cudaFree(ctx->ws);
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
  size_t want = align_up(bytes + bytes / 8, 1 << 20);
  if (ctx->budget && want > ctx->budget) want = bytes;
  e = cudaMalloc(&ctx->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(RSIM_ERR_OOM, "cudaMalloc of the workspace (" + std::to_string(want) + " bytes) failed");
  }
  ctx->ws_bytes = want;
  return RSIM_OK;
}

// Fill FrameIO entries for F frames in workspace `ws`.  A batch's table is uploaded
// here; a single frame's entry goes to the first kernel by value (launch_prep), and the
// meta words and the unit counter are cleared by that kernel too.
rsim_status stage_frames(rsim_ctx* ctx, char* ws, const Consts& k, const rsim_pixels* frames,
                         int F, void* const* cubes, int splits, bool use_partial, bool tensor, int nt,
                         cudaStream_t st, std::vector<FrameIO>& host, FrameIO** dev_table,
                         int** counter) {
  host.assign(F, FrameIO{});
  size_t o = align_up(sizeof(FrameIO) * (size_t)F, 256);
  unsigned long long* meta = (unsigned long long*)(ws + o);
  o = align_up(o + 16 * (size_t)F, 256);
  *counter = (int*)(ws + o);
  o = align_up(o + 16 + 4 * (size_t)F, 256);
  for (int f = 0; f < F; ++f) {
    const rsim_pixels& px = frames[f];
    FrameLayout fl = frame_layout(k.V, k.Ns, k.L, px.P, splits, use_partial, tensor, nt, o);
    o = fl.total;
    FrameIO& io = host[f];
    io.range = px.range;
    io.sre = px.sigma_re;
    io.sim = px.sigma_im;
    io.az = px.az;
    io.el = px.el;
    io.vel = px.vel;
    io.cube = cubes ? cubes[f] : nullptr;
    io.P = px.P;
    io.Pcap = fl.Pcap;
    io.idx = (int32_t*)(ws + fl.idx);
    io.phA = (uint32_t*)(ws + fl.phA);
    io.phC = (uint32_t*)(ws + fl.phC);
    io.phB = (uint32_t*)(ws + fl.phB);
    io.sig = (float2*)(ws + fl.sig);
    io.blk_count = (int32_t*)(ws + fl.blk);
    io.meta = meta + 2 * f;
    io.partial = use_partial ? (float2*)(ws + fl.partial) : nullptr;
    io.bimg = tensor ? (unsigned char*)(ws + fl.bimg) : nullptr;
    io.bimg_nch = fl.bimg_nch;
    io.splits = splits;
  }
  *dev_table = (FrameIO*)ws;
  if (F > 1) {
    cudaError_t e = cudaMemcpyAsync(ws, host.data(), sizeof(FrameIO) * (size_t)F,
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "upload of the frame table");
  }
  return RSIM_OK;
}

int64_t max_P(const rsim_pixels* frames, int F) {
  int64_t m = 0;
  for (int f = 0; f < F; ++f) m = std::max(m, frames[f].P);
  return m;
}

// The stage sequence shared by rsim_synth, rsim_synth_batch and the server.
rsim_status run_frames(rsim_ctx* ctx, char* ws, size_t ws_bytes, const Consts& k,
                       const rsim_pixels* frames, int F, void* const* cubes, int tier,
                       int out_dtype, const rsim_plan& plan, unsigned* status, cudaStream_t st) {
  std::vector<int64_t> Ps(F);
  for (int f = 0; f < F; ++f) Ps[f] = frames[f].P;
  static const char* const kTierName[] = {"fp32", "bf16", "split_bf16", "split_fp16", "fp16", "nufft"};
  char what[160];
  snprintf(what, sizeof what, "synth %s F=%d V=%d Ns=%d L=%d P=%lld splits=%d tile=%d", kTierName[tier], F, k.V,
           k.Ns, k.L, (long long)max_P(frames, F), plan.splits, plan.tile_n);
  NvtxRange call_range(what);
  const int splits = plan.splits;
  const std::string bad = plan_problem(tier, k, plan);
  if (!bad.empty()) return fail(RSIM_ERR_INVALID_ARG, bad);
  if (batch_bytes(k, Ps.data(), F, plan, tier) > ws_bytes)
    return fail(RSIM_ERR_INVALID_ARG, "workspace too small for this request");
  const int64_t mp = max_P(frames, F);
  const bool use_partial = uses_partial(tier, mp, splits, plan.group_chunks);
  std::vector<FrameIO> host;
  FrameIO* table = nullptr;
  int* counter = nullptr;
  rsim_status s = stage_frames(ctx, ws, k, frames, F, cubes, splits, use_partial,
                               tensor_tier(tier), plan.tile_n, st, host, &table, &counter);
  if (s != RSIM_OK) return s;
  // stage events when profiling this context's own calls
  // ev: start, after compaction + phases, after the contraction, after the reduction,
  // and (tensor tiers) between the operand builder and the contraction kernel
  cudaEvent_t ev[kProfEvents] = {};
  const bool prof = ctx->prof && status == ctx->status_dev;
  if (prof) {
    const size_t base = kProfEvents * (size_t)ctx->prof_calls;
    while (ctx->ev_pool.size() < base + kProfEvents) {
      cudaEvent_t x;
      if (cudaEventCreate(&x) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaEventCreate");
      ctx->ev_pool.push_back(x);
    }
    for (int i = 0; i < kProfEvents; ++i) ev[i] = ctx->ev_pool[base + i];
    ctx->prof_calls++;
    // compaction + phases (counted when launched: one cooperative kernel or two); FP32:
    // direct sum (1); tensor tiers: operand builder (1 when a frame has valid pixels), frame
    // order (1 for a batch), contraction (1); NUFFT: the NUFFT kernels of each frame; the
    // split reduction (1 when the partial buffer is used)
    const bool tensor = tensor_tier(tier);
    ctx->prof_kernels += (tier == RSIM_TIER_NUFFT ? kNufftKernels * F
                              : tensor ? 1 + (mp > 0 ? 1 : 0) + (F > 1 ? 1 : 0) : 1) + (use_partial ? 1 : 0);
    cudaEventRecord(ev[0], st);
  }
  cudaError_t e;
  // the tensor tiers' operand builder computes the fast-time and channel phases
  const bool defer = tensor_tier(tier);
  {
    NvtxRange r(defer ? "compaction + slow-time phases" : "compaction + FP64 phases");
    int launched = 0;
    e = launch_prep(k, table, F == 1 ? host.data() : nullptr, F, mp, frames[0].dtype, false, defer, status,
                    counter, st, true, &launched);
    if (prof) ctx->prof_kernels += launched;
  }
  if (e != cudaSuccess) return cuda_fail(e, "prep kernels");
  if (prof) cudaEventRecord(ev[1], st);
  if (tier == RSIM_TIER_NUFFT) {
    if (!nufft_supported(k)) return fail(RSIM_ERR_UNSUPPORTED, "the NUFFT tier needs N_s and L in 4..2048");
    char* scratch = ws + align_up(frames_bytes(k, Ps.data(), F, plan, tier), 256);
    const size_t slot = align_up(nufft_scratch_bytes(k, mp), 256);
    const int S = nufft_slots(F);
    if (S > 1 && !ctx->nu_ready) {
      // create what is missing (an earlier call may have failed part way)
      for (cudaStream_t& x : ctx->nu_st) {
        if (x) continue;
        e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
          x = nullptr;
          return cuda_fail(e, "cudaStreamCreate (NUFFT streams)");
        }
      }
      for (cudaEvent_t& x : ctx->nu_ev) {
        if (x) continue;
        e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
        if (e != cudaSuccess) {
          x = nullptr;
          return cuda_fail(e, "cudaEventCreate (NUFFT streams)");
        }
      }
      ctx->nu_ready = true;
    }
    // frame f runs on stream f mod S with scratch slot f mod S; every stream first waits
    // for the compaction and phases on `st`, and `st` then waits for every stream
    if (S > 1) {
      e = cudaEventRecord(ctx->nu_ev[rsim_ctx::kNuStreams], st);
      for (int i = 0; i < S && e == cudaSuccess; ++i)
        e = cudaStreamWaitEvent(ctx->nu_st[i], ctx->nu_ev[rsim_ctx::kNuStreams], 0);
      if (e != cudaSuccess) return cuda_fail(e, "fork of the NUFFT streams");
    }
    cudaError_t le = cudaSuccess;
    NvtxRange r("NUFFT: binning, spreading, FFTs");
    for (int f = 0; f < F && le == cudaSuccess; ++f) {
      // the first frame's spreading kernel is bracketed by ev[4] and ev[5]
      cudaStream_t fs = S > 1 ? ctx->nu_st[f % S] : st;
      le = launch_nufft(k, table + f, frames[f].P, out_dtype, scratch + (size_t)(f % S) * slot, status, fs,
                        prof && f == 0 ? ev[4] : nullptr, prof && f == 0 ? ev[5] : nullptr);
    }
    // the join also follows a failed launch, so that nothing of this call runs on after it
    for (int i = 0; i < S && S > 1; ++i) {
      e = cudaEventRecord(ctx->nu_ev[i], ctx->nu_st[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->nu_ev[i], 0);
      if (e != cudaSuccess) return cuda_fail(e, "join of the NUFFT streams");
    }
    if (le != cudaSuccess) return cuda_fail(le, "NUFFT kernels");
    if (prof) cudaEventRecord(ev[2], st);
  } else if (tier == RSIM_TIER_FP32) {
    if (prof) cudaEventRecord(ev[4], st);
    NvtxRange r("FP32 direct sum + split reduction");
    e = launch_direct(k, table, F, splits, plan.tile_n, out_dtype, st);
    if (e != cudaSuccess) return cuda_fail(e, "direct-sum kernel");
    if (prof) cudaEventRecord(ev[2], st);
    if (prof) cudaEventRecord(ev[5], st);
    if (use_partial) {
      e = launch_reduce(k, table, F, splits, out_dtype, 0.f, st);
      if (e != cudaSuccess) return cuda_fail(e, "split reduction");
    }
  } else {
    NvtxRange r("operand images + tcgen05 contraction + split reduction");
    e = launch_umma(k, table, F, splits, tier, out_dtype, plan.grid, plan.tile_n, plan.group_chunks,
                    use_partial, ctx->num_sms, mp, frames[0].dtype, status, counter, st, prof ? ev[4] : nullptr);
    if (e == cudaErrorNotSupported) return fail(RSIM_ERR_UNSUPPORTED, "tensor-core tier not available");
    if (e != cudaSuccess) return cuda_fail(e, "tcgen05 contraction kernel");
    if (prof) cudaEventRecord(ev[2], st);
    if (prof) cudaEventRecord(ev[5], st);
    if (use_partial) {
      const bool scaled = (tier == RSIM_TIER_SPLIT_FP16 || tier == RSIM_TIER_FP16);
      e = launch_reduce_tiles(k, table, F, splits, plan.tile_n, out_dtype, scaled, ctx->num_sms, st);
      if (e != cudaSuccess) return cuda_fail(e, "split reduction");
    }
  }
  if (prof) cudaEventRecord(ev[3], st);
  return RSIM_OK;
}

// Copy n16 16-byte units from device memory to page-locked host memory through its mapped
// address: coalesced stores that cross the host link as whole lines.  For a cube of a few
// MB this finished sooner on average than a copy-engine transfer (22 vs 27 us for 3.1 MB
// on GB300), with less spread.
__global__ void copy_to_host16(const uint4* __restrict__ src, uint4* __restrict__ dst, size_t n16) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

}  // namespace rsim

using namespace rsim;

extern "C" {

const char* rsim_version(void) { return "rsim 0.1 (sm_103a)"; }

const char* rsim_last_error(void) { return g_last_error.c_str(); }

rsim_status rsim_create(rsim_ctx** out, int device, size_t hbm_budget_bytes) {
  if (!out) return fail(RSIM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= n) return fail(RSIM_ERR_INVALID_ARG, "no such device");
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  rsim_ctx* c = new rsim_ctx();
  c->device = device;
  c->num_sms = prop.multiProcessorCount;
  c->cc_major = prop.major;
  c->cc_minor = prop.minor;
  c->budget = hbm_budget_bytes;
  e = cudaMalloc(&c->status_dev, 256);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaMalloc(status)");
  }
  cudaMemset(c->status_dev, 0, 256);
  load_plan_cache(c);
  *out = c;
  return RSIM_OK;
}

rsim_status rsim_destroy(rsim_ctx* ctx) {
  if (!ctx) return RSIM_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->stage) cudaFree(ctx->stage);
  if (ctx->status_dev) cudaFree(ctx->status_dev);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : ctx->nu_ev)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : ctx->nu_st)
    if (s) cudaStreamDestroy(s);
  delete ctx;
  return RSIM_OK;
}

rsim_status rsim_workspace_size(rsim_ctx* ctx, const rsim_radar_params* params, int64_t P,
                                rsim_tier tier, size_t* bytes) {
  if (!ctx || !bytes) return fail(RSIM_ERR_INVALID_ARG, "ctx or bytes is NULL");
  if (!tier_ok(tier)) return fail(RSIM_ERR_INVALID_ARG, "unknown tier");
  if (P < 0) return fail(RSIM_ERR_INVALID_ARG, "P must be >= 0");
  Consts k;
  rsim_status s = check_params(params, &k);
  if (s != RSIM_OK) return s;
  rsim_plan plan = choose_plan(ctx, tier, k, P);
  *bytes = batch_bytes(k, &P, 1, plan, tier);
  return RSIM_OK;
}

rsim_status rsim_synth(rsim_ctx* ctx, const rsim_radar_params* params, const rsim_pixels* pixels,
                       rsim_tier tier, void* cube, int32_t out_dtype, rsim_stream stream) {
  void* cubes[1] = {cube};
  return rsim_synth_batch(ctx, params, pixels, 1, cubes, tier, out_dtype, stream);
}

// A pointer the device can use for host buffer `p`, or nullptr: page-locked (registered)
// memory through its mapped address, device or managed memory as is, and pageable memory
// only when the device reads it through the host's page tables.
const void* device_view(rsim_ctx* ctx, const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost) return a.devicePointer;
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
  if (ctx->pageable_access < 0) {
    int pma = 0, tables = 0;
    if (cudaDeviceGetAttribute(&pma, cudaDevAttrPageableMemoryAccess, ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, ctx->device) !=
            cudaSuccess) {
      cudaGetLastError();
      pma = tables = 0;
    }
    ctx->pageable_access = (pma && tables) ? 1 : 0;
  }
  return ctx->pageable_access == 1 ? p : nullptr;
}

rsim_status rsim_synth_host(rsim_ctx* ctx, const rsim_radar_params* params, const rsim_pixels* pixels,
                            rsim_tier tier, void* cube, int32_t out_dtype, rsim_stream stream) {
  if (!ctx) return fail(RSIM_ERR_INVALID_ARG, "ctx is NULL");
  if (!cube) return fail(RSIM_ERR_INVALID_ARG, "cube is NULL");
  if (out_dtype != RSIM_C64 && out_dtype != RSIM_C128)
    return fail(RSIM_ERR_INVALID_ARG, "out_dtype must be RSIM_C64 or RSIM_C128");
  Consts k;
  rsim_status s = check_params(params, &k);
  if (s != RSIM_OK) return s;
  s = check_pixels(pixels);
  if (s != RSIM_OK) return s;
  const size_t elem = pixels->dtype == RSIM_F64 ? 8 : 4;
  const size_t arr = align_up((size_t)pixels->P * elem, 256);
  const size_t cube_bytes = (size_t)k.V * (size_t)k.Ns * (size_t)k.L * (out_dtype == RSIM_C128 ? 16 : 8);
  const size_t cube_span = align_up(cube_bytes, 256);
  size_t need = cube_span + 6 * arr;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  // pixel arrays the device can read in place (coalesced loads over the host link) are not
  // staged; the cube always is, and comes back in one copy (the kernels that write it
  // scatter 8- to 16-byte stores, which cross the host link one by one)
  const void* src[6] = {pixels->range, pixels->sigma_re, pixels->sigma_im, pixels->az, pixels->el, pixels->vel};
  const void* view[6] = {};
  bool direct = pixels->P > 0;
  for (int i = 0; i < 6 && direct; ++i) direct = (view[i] = device_view(ctx, src[i])) != nullptr;
  if (direct) need = cube_bytes;
  if (ctx->stage_bytes < need) {
    if (ctx->budget && ctx->ws_bytes + need > ctx->budget)
      return fail(RSIM_ERR_BUDGET, "staging of " + std::to_string(need) + " bytes exceeds the context budget");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (ctx->stage) cudaFree(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
    e = cudaMalloc(&ctx->stage, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(RSIM_ERR_OOM, "cudaMalloc of the staging buffer (" + std::to_string(need) + " bytes) failed");
    }
    ctx->stage_bytes = need;
  }
  char* base = (char*)ctx->stage;
  rsim_pixels dev = *pixels;
  const void** dst[6] = {&dev.range, &dev.sigma_re, &dev.sigma_im, &dev.az, &dev.el, &dev.vel};
  for (int i = 0; i < 6; ++i) {
    if (direct) {
      *dst[i] = view[i];
      continue;
    }
    *dst[i] = base + cube_span + i * arr;
    if (pixels->P > 0) {
      // cudaMemcpyDefault: the direction follows the pointers (unified addressing), so a
      // caller may also pass device or managed memory here
      e = cudaMemcpyAsync(base + cube_span + i * arr, src[i], (size_t)pixels->P * elem, cudaMemcpyDefault, st);
      if (e != cudaSuccess) return cuda_fail(e, "copy of a pixel array to the device");
    }
  }
  void* cube_dev = base;
  s = rsim_synth(ctx, params, &dev, tier, cube_dev, out_dtype, stream);
  if (s != RSIM_OK) return s;
  // the cube back: into page-locked memory by a copy kernel through its mapped address
  // (16-byte aligned, whole 16-byte units), else by a copy-engine transfer
  void* mapped = nullptr;
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, cube) == cudaSuccess) {
    if (pa.type == cudaMemoryTypeHost) mapped = pa.devicePointer;
  } else {
    cudaGetLastError();
  }
  if (mapped && (uintptr_t)mapped % 16 == 0 && cube_bytes % 16 == 0) {
    const size_t n16 = cube_bytes / 16;
    const size_t blocks = std::min<size_t>((n16 + 255) / 256, (size_t)4 * std::max(ctx->num_sms, 1));
    copy_to_host16<<<(unsigned)blocks, 256, 0, st>>>((const uint4*)cube_dev, (uint4*)mapped, n16);
    e = cudaGetLastError();
  } else {
    e = cudaMemcpyAsync(cube, cube_dev, cube_bytes, cudaMemcpyDefault, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "copy of the cube to the host");
  return RSIM_OK;
}

rsim_status rsim_synth_batch(rsim_ctx* ctx, const rsim_radar_params* params,
                             const rsim_pixels* frames, int32_t F, void* const* cubes,
                             rsim_tier tier, int32_t out_dtype, rsim_stream stream) {
  if (!ctx) return fail(RSIM_ERR_INVALID_ARG, "ctx is NULL");
  if (!frames || !cubes) return fail(RSIM_ERR_INVALID_ARG, "frames or cubes is NULL");
  if (F < 1) return fail(RSIM_ERR_INVALID_ARG, "F must be >= 1");
  if (!tier_ok(tier)) return fail(RSIM_ERR_INVALID_ARG, "unknown tier");
  if (out_dtype != RSIM_C64 && out_dtype != RSIM_C128)
    return fail(RSIM_ERR_INVALID_ARG, "out_dtype must be RSIM_C64 or RSIM_C128");
  Consts k;
  rsim_status s = check_params(params, &k);
  if (s != RSIM_OK) return s;
  int64_t maxp = 0;
  for (int f = 0; f < F; ++f) {
    s = check_pixels(&frames[f]);
    if (s != RSIM_OK) return s;
    if (!cubes[f]) return fail(RSIM_ERR_INVALID_ARG, "a cube pointer is NULL");
    if (frames[f].dtype != frames[0].dtype)
      return fail(RSIM_ERR_INVALID_ARG, "all frames of a batch must share the pixel dtype");
    maxp = std::max(maxp, frames[f].P);
  }
  if (tensor_tier(tier) && !(ctx->cc_major == 10 && ctx->cc_minor == 3))
    return fail(RSIM_ERR_UNSUPPORTED, "tensor-core tiers need an sm_103 device");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  // the plan of a batch is the plan of its largest frame: every frame uses the same
  // splits rule, so a frame gives the same bits alone and in a batch of equal-P frames
  rsim_plan plan = choose_plan(ctx, tier, k, maxp);
  std::vector<int64_t> Ps(F);
  for (int f = 0; f < F; ++f) Ps[f] = frames[f].P;
  const size_t need = batch_bytes(k, Ps.data(), F, plan, tier);
  s = ensure_workspace(ctx, need, st);
  if (s != RSIM_OK) return s;
  return run_frames(ctx, (char*)ctx->ws, ctx->ws_bytes, k, frames, F, cubes, tier, out_dtype, plan,
                    ctx->status_dev, st);
}

rsim_status rsim_valid_indices(rsim_ctx* ctx, const rsim_pixels* pixels, int32_t* idx,
                               int64_t* p_valid, rsim_stream stream) {
  if (!ctx || !idx || !p_valid) return fail(RSIM_ERR_INVALID_ARG, "NULL argument");
  rsim_status s = check_pixels(pixels);
  if (s != RSIM_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(ctx->device);
  Consts k{};
  k.V = 1;
  k.Ns = 1;
  k.L = 1;
  int64_t P = pixels->P;
  rsim_plan one{};
  one.splits = 1;
  s = ensure_workspace(ctx, batch_bytes(k, &P, 1, one, RSIM_TIER_FP32), st);
  if (s != RSIM_OK) return s;
  std::vector<FrameIO> host;
  FrameIO* table = nullptr;
  int* counter = nullptr;
  void* cubes[1] = {nullptr};
  s = stage_frames(ctx, (char*)ctx->ws, k, pixels, 1, cubes, 1, false, false, 0, st, host, &table,
                   &counter);
  if (s != RSIM_OK) return s;
  // the index list goes straight to the caller's buffer; the count is copied after
  host[0].idx = idx;
  cudaError_t e = cudaMemcpyAsync(table, host.data(), sizeof(FrameIO), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "upload of the frame table");
  e = launch_prep(k, table, host.data(), 1, P, pixels->dtype, true, false, ctx->status_dev, nullptr, st);
  if (e != cudaSuccess) return cuda_fail(e, "prep kernels");
  e = cudaMemcpyAsync(p_valid, host[0].meta, 8, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "copy of the valid count");
  return RSIM_OK;
}

rsim_status rsim_path_phases(rsim_ctx* ctx, const rsim_radar_params* params,
                             const rsim_pixels* pixels, uint32_t* a, uint32_t* cph, uint32_t* b,
                             float* sigma, int64_t* p_valid, rsim_stream stream) {
  if (!ctx || !a || !cph || !b || !sigma || !p_valid) return fail(RSIM_ERR_INVALID_ARG, "NULL argument");
  Consts k;
  rsim_status s = check_params(params, &k);
  if (s != RSIM_OK) return s;
  s = check_pixels(pixels);
  if (s != RSIM_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(ctx->device);
  int64_t P = pixels->P;
  rsim_plan one{};
  one.splits = 1;
  s = ensure_workspace(ctx, batch_bytes(k, &P, 1, one, RSIM_TIER_FP32), st);
  if (s != RSIM_OK) return s;
  std::vector<FrameIO> host;
  FrameIO* table = nullptr;
  int* counter = nullptr;
  void* cubes[1] = {nullptr};
  s = stage_frames(ctx, (char*)ctx->ws, k, pixels, 1, cubes, 1, false, false, 0, st, host, &table,
                   &counter);
  if (s != RSIM_OK) return s;
  host[0].phA = a;
  host[0].phC = cph;
  host[0].phB = b;
  host[0].sig = (float2*)sigma;
  host[0].Pcap = P;
  cudaError_t e = cudaMemcpyAsync(table, host.data(), sizeof(FrameIO), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "upload of the frame table");
  e = launch_prep(k, table, host.data(), 1, P, pixels->dtype, false, false, ctx->status_dev, nullptr, st);
  if (e != cudaSuccess) return cuda_fail(e, "prep kernels");
  e = cudaMemcpyAsync(p_valid, host[0].meta, 8, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "copy of the valid count");
  return RSIM_OK;
}

rsim_status rsim_sync_status(rsim_ctx* ctx, rsim_stream stream) {
  if (!ctx) return fail(RSIM_ERR_INVALID_ARG, "ctx is NULL");
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  unsigned w = 0;
  e = cudaMemcpy(&w, ctx->status_dev, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read of the status word");
  if (w) cudaMemset(ctx->status_dev, 0, 4);
  if (w & kStatusTimeout) return fail(RSIM_ERR_TIMEOUT, "a device-side wait ran out of time");
  if (w & kStatusNonfinite)
    return fail(RSIM_ERR_NONFINITE, "a valid pixel has a non-finite field or R <= 0");
  return RSIM_OK;
}

rsim_status rsim_selftest_wait_timeout(rsim_ctx* ctx, uint64_t limit_ns, rsim_stream stream) {
  if (!ctx) return fail(RSIM_ERR_INVALID_ARG, "ctx is NULL");
  if (limit_ns < 1000ull || limit_ns > 10000000000ull)
    return fail(RSIM_ERR_INVALID_ARG, "limit_ns must lie in [1 us, 10 s]");
  cudaSetDevice(ctx->device);
  const cudaError_t e = launch_wait_selftest(ctx->status_dev, limit_ns, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "self-test kernel");
  return RSIM_OK;
}

rsim_status rsim_profile_enable(rsim_ctx* ctx, int32_t on) {
  if (!ctx) return fail(RSIM_ERR_INVALID_ARG, "ctx is NULL");
  ctx->prof = on != 0;
  ctx->prof_calls = 0;
  ctx->prof_kernels = 0;
  return RSIM_OK;
}

rsim_status rsim_profile_read(rsim_ctx* ctx, rsim_profile* out) {
  if (!ctx || !out) return fail(RSIM_ERR_INVALID_ARG, "NULL argument");
  cudaSetDevice(ctx->device);
  rsim_profile p{};
  p.calls = ctx->prof_calls;
  p.kernels = ctx->prof_kernels;
  for (int c = 0; c < ctx->prof_calls; ++c) {
    cudaEvent_t* ev = &ctx->ev_pool[kProfEvents * (size_t)c];
    cudaError_t e = cudaEventSynchronize(ev[3]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    float a = 0, b = 0, d = 0, o = 0, m = 0;
    cudaEventElapsedTime(&a, ev[0], ev[1]);
    cudaEventElapsedTime(&b, ev[1], ev[2]);
    cudaEventElapsedTime(&d, ev[2], ev[3]);
    cudaEventElapsedTime(&o, ev[1], ev[4]);
    cudaEventElapsedTime(&m, ev[4], ev[5]);
    p.prep_ms += a;
    p.contract_ms += b;
    p.reduce_ms += d;
    p.operand_ms += o;
    p.main_ms += m;
  }
  ctx->prof_calls = 0;
  ctx->prof_kernels = 0;
  *out = p;
  return RSIM_OK;
}

rsim_status rsim_set_plan(rsim_ctx* ctx, const rsim_radar_params* params, int64_t P,
                          rsim_tier tier, const rsim_plan* plan) {
  // the plan is checked before the context is needed, so a bad plan is reported as such
  if (!plan) return fail(RSIM_ERR_INVALID_ARG, "plan is NULL");
  if (!tier_ok(tier)) return fail(RSIM_ERR_INVALID_ARG, "unknown tier");
  Consts k;
  rsim_status s = check_params(params, &k);
  if (s != RSIM_OK) return s;
  const std::string bad = plan_problem(tier, k, *plan);
  if (!bad.empty()) return fail(RSIM_ERR_INVALID_ARG, bad);
  if (!ctx) return fail(RSIM_ERR_INVALID_ARG, "ctx is NULL");
  rsim_plan p = *plan;
  resolve_tile(tier, k, &p);
  std::lock_guard<std::mutex> g(ctx->plan_mu);
  ctx->plans[plan_key(tier, k, P)] = p;
  return RSIM_OK;
}

rsim_status rsim_get_plan(rsim_ctx* ctx, const rsim_radar_params* params, int64_t P,
                          rsim_tier tier, rsim_plan* plan) {
  if (!ctx || !plan) return fail(RSIM_ERR_INVALID_ARG, "NULL argument");
  if (!tier_ok(tier)) return fail(RSIM_ERR_INVALID_ARG, "unknown tier");
  Consts k;
  rsim_status s = check_params(params, &k);
  if (s != RSIM_OK) return s;
  *plan = choose_plan(ctx, tier, k, P);
  return RSIM_OK;
}

}  // extern "C"
