// Autotuner: times candidate launch plans for a shape bucket and caches the fastest.
//
// A plan holds the tile shapes and the work split of one shape bucket (tier, V, N_s, L,
// ceil(log2 P)): the column tile NT and the accumulation-group length of the
// tensor-core contraction, or the n tile of the FP32 direct sum, plus the pixel split
// count and the persistent grid.  The search is coordinate-wise, so its cost stays a
// dozen or two timed runs: first the tile (each with its own default split count), then
// splits x grid with the best tile, then the group length.  Every candidate keeps the
// accuracy rules (at most 8192 pixels per FP32 split, group lengths within the tier's
// cap), so a tuned plan meets the same error bar as the default.  The key is the shape
// only, never the load or the data, so the same frame always runs the same kernels with
// the same reduction order.  Timings use CUDA events on the caller's stream over
// synthetic full-valid pixels drawn on the device by a counter-based hash.  Results
// live in the context and, when RSIM_TUNE_CACHE names a file, in a small JSON object
// {"key": [splits, grid, tile_n, group_chunks], ...}.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "rsim_ctx.h"

namespace rsim {
namespace {

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  // integer finaliser of MurmurHash3 (Appleby), a published bit mixer
  x ^= x >> 16;
  x *= 0x85ebca6bu;
  x ^= x >> 13;
  x *= 0xc2b2ae35u;
  x ^= x >> 16;
  return x;
}

__device__ __forceinline__ float unit(uint32_t seed, uint32_t i, uint32_t stream) {
  return (hash32(seed ^ hash32(i * 6u + stream)) >> 8) * (1.0f / 16777216.0f);
}

// Full-valid random pixels: R in [0.5, 8) m, unit-magnitude sigma, az in +-60 deg,
// el in +-30 deg, vel in +-2 m/s.
__global__ void fill_synthetic(float* R, float* sre, float* sim, float* az, float* el, float* vel,
                               int64_t P, uint32_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t u = (uint32_t)i;
    R[i] = 0.5f + 7.5f * unit(seed, u, 0);
    float s, c;
    sincospif(2.0f * unit(seed, u, 1), &s, &c);
    sre[i] = c;
    sim[i] = s;
    az[i] = (unit(seed, u, 2) - 0.5f) * 2.0943951f;
    el[i] = (unit(seed, u, 3) - 0.5f) * 1.0471976f;
    vel[i] = (unit(seed, u, 4) - 0.5f) * 4.0f;
  }
}

std::string cache_path() {
  const char* p = getenv("RSIM_TUNE_CACHE");
  return p ? std::string(p) : std::string();
}

// Minimal reader for the flat JSON object written by save_plan_cache.
void parse_cache(const std::string& text, std::map<std::string, rsim_plan>& out) {
  size_t i = 0;
  while (true) {
    size_t a = text.find('"', i);
    if (a == std::string::npos) break;
    size_t b = text.find('"', a + 1);
    if (b == std::string::npos) break;
    std::string key = text.substr(a + 1, b - a - 1);
    size_t lb = text.find('[', b), rb = text.find(']', b);
    if (lb == std::string::npos || rb == std::string::npos) break;
    int s = 0, g = 0, t = 0, gc = 0;
    // entries are checked against the shape again when used (choose_plan)
    if (sscanf(text.c_str() + lb + 1, "%d , %d , %d , %d", &s, &g, &t, &gc) == 4 && s >= 1 && s <= kMaxSplits &&
        g >= 0 && t >= 0 && gc >= 0) {
      rsim_plan p{};
      p.splits = s;
      p.grid = g;
      p.tile_n = t;
      p.group_chunks = gc;
      p.chunk_px = kChunkPx;
      p.tuned = 1;
      out[key] = p;
    }
    i = rb + 1;
  }
}

void save_plan_cache(rsim_ctx* ctx) {
  const std::string path = cache_path();
  if (path.empty()) return;
  std::string tmp = path + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fprintf(f, "{\n");
  bool first = true;
  for (auto& kv : ctx->plans) {
    if (!kv.second.tuned) continue;
    fprintf(f, "%s  \"%s\": [%d, %d, %d, %d]", first ? "" : ",\n", kv.first.c_str(), kv.second.splits,
            kv.second.grid, kv.second.tile_n, kv.second.group_chunks);
    first = false;
  }
  fprintf(f, "\n}\n");
  fclose(f);
  rename(tmp.c_str(), path.c_str());
}

}  // namespace

void load_plan_cache(rsim_ctx* ctx) {
  const std::string path = cache_path();
  if (path.empty()) return;
  FILE* f = fopen(path.c_str(), "r");
  if (!f) return;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
  fclose(f);
  std::lock_guard<std::mutex> g(ctx->plan_mu);
  parse_cache(text, ctx->plans);
}

}  // namespace rsim

using namespace rsim;

extern "C" rsim_status rsim_autotune(rsim_ctx* ctx, const rsim_radar_params* params, int64_t P,
                                     rsim_tier tier, rsim_plan* chosen, rsim_stream stream) {
  if (!ctx || !chosen) return fail(RSIM_ERR_INVALID_ARG, "NULL argument");
  if (!tier_ok(tier)) return fail(RSIM_ERR_INVALID_ARG, "unknown tier");
  if (P < 1) return fail(RSIM_ERR_INVALID_ARG, "P must be >= 1");
  Consts k;
  rsim_status s = check_params(params, &k);
  if (s != RSIM_OK) return s;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;

  // synthetic pixels and an output buffer
  float* px = nullptr;
  void* cube = nullptr;
  const size_t cube_bytes = (size_t)k.V * k.Ns * k.L * 8;
  cudaError_t e = cudaMalloc(&px, 6 * sizeof(float) * (size_t)P);
  if (e != cudaSuccess) return fail(RSIM_ERR_OOM, "autotune: pixel buffer allocation failed");
  e = cudaMalloc(&cube, cube_bytes);
  if (e != cudaSuccess) {
    cudaFree(px);
    return fail(RSIM_ERR_OOM, "autotune: cube allocation failed");
  }
  fill_synthetic<<<256, 256, 0, st>>>(px, px + P, px + 2 * P, px + 3 * P, px + 4 * P, px + 5 * P, P,
                                      0x5eed1234u);
  rsim_pixels pix{P, RSIM_F32, 0, px, px + P, px + 2 * P, px + 3 * P, px + 4 * P, px + 5 * P};

  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  rsim_status err = RSIM_OK;
  // time one plan: a warm-up run, then the best of two (1e30 if it cannot run)
  auto time_plan = [&](const rsim_plan& p) -> float {
    if (err != RSIM_OK || !plan_problem(tier, k, p).empty()) return 1e30f;
    int64_t PP = P;
    rsim_status s2 = ensure_workspace(ctx, batch_bytes(k, &PP, 1, p, tier), st);
    if (s2 != RSIM_OK) {
      err = s2;
      return 1e30f;
    }
    void* cubes[1] = {cube};
    float tbest = 1e30f;
    for (int rep = 0; rep < 3 && s2 == RSIM_OK; ++rep) {
      cudaEventRecord(e0, st);
      s2 = run_frames(ctx, (char*)ctx->ws, ctx->ws_bytes, k, &pix, 1, cubes, tier, RSIM_C64, p, ctx->status_dev,
                      st);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tbest = std::min(tbest, ms);
    }
    if (s2 != RSIM_OK) err = s2;
    return tbest;
  };
  const bool tensor = tensor_tier(tier);
  // FP32: at most 8192 pixels per split (the accuracy rule of the default plan)
  const int smin = tier == RSIM_TIER_FP32 ? (int)std::min<int64_t>(std::max<int64_t>((P + 8191) / 8192, 1), kMaxSplits)
                                          : 1;

  // 1. the tile, each candidate with its own default split count
  rsim_plan best = default_plan(tier, k, P, ctx->num_sms);
  std::vector<int> tiles = {best.tile_n};
  if (tier == RSIM_TIER_FP32) tiles.push_back(64);
  if (tensor && best.tile_n > 64) tiles.push_back(64);
  float tb = 1e30f;
  for (int t : tiles) {
    rsim_plan p = best;
    p.tile_n = t;
    p.splits = default_splits(tier, k.V, k.Ns, k.L, t, P, ctx->num_sms);
    const float ms = time_plan(p);
    if (ms < tb) {
      tb = ms;
      best = p;
    }
  }
  // 2. splits around the tile's default rule, and the persistent grid (tensor tiers)
  {
    const int s0 = best.splits;
    std::vector<int> cand_s;
    for (int m : {2, 3, 4, 6, 8}) {
      int a = std::min(std::max(smin, s0 * m / 4), kMaxSplits);
      if (std::find(cand_s.begin(), cand_s.end(), a) == cand_s.end()) cand_s.push_back(a);
    }
    std::vector<int> cand_g = {0};
    if (tensor) cand_g.push_back(ctx->num_sms / 2);
    const rsim_plan base = best;
    for (int sp : cand_s) {
      for (int g : cand_g) {
        if (sp == base.splits && g == base.grid) continue;
        rsim_plan p = base;
        p.splits = sp;
        p.grid = g;
        const float ms = time_plan(p);
        if (ms < tb) {
          tb = ms;
          best = p;
        }
      }
    }
  }
  // 3. the accumulation-group length (tensor tiers), never above the tier's cap
  if (tensor) {
    const int gmax = group_chunks_max(tier);
    std::vector<int> cand = (tier == RSIM_TIER_SPLIT_BF16 || tier == RSIM_TIER_SPLIT_FP16)
                                ? std::vector<int>{32, gmax}
                                : std::vector<int>{192, gmax};
    const rsim_plan base = best;
    for (int gc : cand) {
      if (gc == base.group_chunks || gc > gmax) continue;
      rsim_plan p = base;
      p.group_chunks = gc;
      const float ms = time_plan(p);
      if (ms < tb) {
        tb = ms;
        best = p;
      }
    }
  }
  best.tuned = 1;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(px);
  cudaFree(cube);
  if (err != RSIM_OK) return err;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  {
    std::lock_guard<std::mutex> g(ctx->plan_mu);
    ctx->plans[plan_key(tier, k, P)] = best;
    save_plan_cache(ctx);
  }
  *chosen = best;
  return RSIM_OK;
}
