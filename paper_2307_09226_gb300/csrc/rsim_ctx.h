// The context object behind the opaque rsim_ctx handle, and host helpers shared by
// the API, the autotuner and the server sources.
#pragma once

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "rsim_internal.h"

// CUDA events a profiled synth call records (stage boundaries).
constexpr int kProfEvents = 6;

struct rsim_ctx {
  int device = 0;
  int num_sms = 0;
  int cc_major = 0, cc_minor = 0;
  size_t budget = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // 256 bytes: word 0 is the status word of the context's own calls (rsim_sync_status);
  // word 32 is the shared-atomic probe's sink and word 33 the tensor-core probe's wait
  // failures (measure.cu); the rest is unused
  unsigned* status_dev = nullptr;
  void* stage = nullptr;  // rsim_synth_host: device copies of the pixel arrays and the cube
  size_t stage_bytes = 0;
  int pageable_access = -1;  // the device reads pageable host memory through the host page tables (-1: not asked yet)
  // NUFFT batches: frames run on kNuStreams streams, each with its own grid scratch, so
  // that the kernels of small frames overlap (created on first use)
  static constexpr int kNuStreams = 8;
  cudaStream_t nu_st[kNuStreams] = {};
  cudaEvent_t nu_ev[kNuStreams + 1] = {};  // one per stream, then the fork
  bool nu_ready = false;                   // all of nu_st and nu_ev exist
  std::mutex plan_mu;
  std::map<std::string, rsim_plan> plans;
  // stage profiling (rsim_profile_enable / rsim_profile_read)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;  // kProfEvents events per recorded call
  int prof_calls = 0;
  int prof_kernels = 0;
};

namespace rsim {
rsim_status fail(rsim_status st, const std::string& msg);
rsim_status cuda_fail(cudaError_t e, const char* where);
rsim_status check_params(const rsim_radar_params* p, Consts* k);
rsim_status check_pixels(const rsim_pixels* px);
bool tier_ok(int tier);
std::string plan_key(int tier, const Consts& k, int64_t P);
rsim_plan choose_plan(rsim_ctx* ctx, int tier, const Consts& k, int64_t P);
size_t batch_bytes(const Consts& k, const int64_t* P, int F, const rsim_plan& plan, int tier);
rsim_status ensure_workspace(rsim_ctx* ctx, size_t bytes, cudaStream_t st);
rsim_status run_frames(rsim_ctx* ctx, char* ws, size_t ws_bytes, const Consts& k,
                       const rsim_pixels* frames, int F, void* const* cubes, int tier,
                       int out_dtype, const rsim_plan& plan, unsigned* status, cudaStream_t st);
void load_plan_cache(rsim_ctx* ctx);
}  // namespace rsim
