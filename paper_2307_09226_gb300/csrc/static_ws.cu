// rsim_synth_static: one-frame synthesis whose scratch memory is a fixed array
// compiled into the library, for callers that must not allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: a real-time radar processing
// loop whose device memory is fixed when it starts, or a host framework that owns
// the device memory budget and forbids libraries from allocating.  rsim_synth needs
// an rsim_ctx, and both the context and its workspace are allocated with cudaMalloc.
// This entry point runs the same stages through a new host path instead.  Its
// workspace (compacted pixels, fixed-point phases, split partial sums, frame table,
// counters and an optional status word) lives in g_static_ws below.  Every GPU that
// loads the library holds that array until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "rsim_ctx.h"
#include "rsim_internal.h"

namespace rsim {
namespace {

constexpr size_t kStaticWsBytes = size_t(64) << 20;  // 64 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_ws[kStaticWsBytes];

// Device address of g_static_ws per device.  In host code the symbol name is only a
// host-side stand-in, so the address is taken once per device, with that device
// current, by cudaGetSymbolAddress.
std::mutex g_ws_mu;
void* g_ws_addr[kMaxDevices] = {};

rsim_status static_ws_address(int dev, char** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(RSIM_ERR_UNSUPPORTED, "device index too large");
  std::lock_guard<std::mutex> g(g_ws_mu);
  if (!g_ws_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(static workspace)");
    g_ws_addr[dev] = p;
  }
  *out = (char*)g_ws_addr[dev];
  return RSIM_OK;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace rsim

using namespace rsim;

extern "C" rsim_status rsim_synth_static(const rsim_radar_params* params, const rsim_pixels* pixels,
                                         rsim_tier tier, void* cube, int32_t out_dtype,
                                         uint32_t* device_status, rsim_stream stream) {
  Consts k;
  rsim_status s = check_params(params, &k);
  if (s != RSIM_OK) return s;
  s = check_pixels(pixels);
  if (s != RSIM_OK) return s;
  if (!tier_ok(tier)) return fail(RSIM_ERR_INVALID_ARG, "unknown tier");
  if (out_dtype != RSIM_C64 && out_dtype != RSIM_C128)
    return fail(RSIM_ERR_INVALID_ARG, "out_dtype must be RSIM_C64 or RSIM_C128");
  if (!cube) return fail(RSIM_ERR_INVALID_ARG, "cube is NULL");
  int dev = 0, sms = 0, major = 0, minor = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device query");
  if (tier == RSIM_TIER_NUFFT) return fail(RSIM_ERR_UNSUPPORTED, "the static workspace serves the direct and tensor-core tiers");
  if (tensor_tier(tier) && !(major == 10 && minor == 3))
    return fail(RSIM_ERR_UNSUPPORTED, "tensor-core tiers need an sm_103 device");

  // the plan is the library's default rule for this shape (what rsim_synth uses
  // without a tuned plan); the scratch layout mirrors the context workspace
  const int64_t P = pixels->P;
  const rsim_plan plan = default_plan(tier, k, P, sms);
  const int splits = plan.splits;
  const bool use_partial = uses_partial(tier, P, splits, plan.group_chunks);
  size_t o = 0;
  const size_t off_table = o;   o = up256(o + sizeof(FrameIO));
  const size_t off_meta = o;    o = up256(o + 16);
  const size_t off_counter = o; o = up256(o + 16 + 4);
  FrameLayout fl = frame_layout(k.V, k.Ns, k.L, P, splits, use_partial, tensor_tier(tier), plan.tile_n, o);
  o = fl.total;
  const size_t off_status = o;  o = up256(o + 4);
  if (o > kStaticWsBytes)
    return fail(RSIM_ERR_BUDGET, "frame needs " + std::to_string(o) +
                                     " bytes of scratch; the static workspace holds " +
                                     std::to_string(kStaticWsBytes));

  char* ws = nullptr;
  s = static_ws_address(dev, &ws);
  if (s != RSIM_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* status = device_status ? (unsigned*)device_status : (unsigned*)(ws + off_status);

  FrameIO io{};
  io.range = pixels->range;
  io.sre = pixels->sigma_re;
  io.sim = pixels->sigma_im;
  io.az = pixels->az;
  io.el = pixels->el;
  io.vel = pixels->vel;
  io.cube = cube;
  io.P = P;
  io.Pcap = fl.Pcap;
  io.idx = (int32_t*)(ws + fl.idx);
  io.phA = (uint32_t*)(ws + fl.phA);
  io.phC = (uint32_t*)(ws + fl.phC);
  io.phB = (uint32_t*)(ws + fl.phB);
  io.sig = (float2*)(ws + fl.sig);
  io.blk_count = (int32_t*)(ws + fl.blk);
  io.meta = (unsigned long long*)(ws + off_meta);
  io.partial = use_partial ? (float2*)(ws + fl.partial) : nullptr;
  io.bimg = tensor_tier(tier) ? (unsigned char*)(ws + fl.bimg) : nullptr;
  io.bimg_nch = fl.bimg_nch;
  io.splits = splits;
  FrameIO* table = (FrameIO*)(ws + off_table);
  int* counter = (int*)(ws + off_counter);

  // the array keeps the previous call's contents: the first kernel stores the frame
  // entry and clears the meta words and the unit counter; the status word is cleared here
  if (!device_status) e = cudaMemsetAsync(status, 0, 4, st);
  if (e != cudaSuccess) return cuda_fail(e, "static workspace set-up");

  const bool defer = tensor_tier(tier);  // the operand builder computes the fast-time phases
  e = launch_prep(k, table, &io, 1, P, pixels->dtype, false, defer, status, counter, st, false);
  if (e != cudaSuccess) return cuda_fail(e, "prep kernels");
  if (tier == RSIM_TIER_FP32) {
    e = launch_direct(k, table, 1, splits, plan.tile_n, out_dtype, st);
    if (e != cudaSuccess) return cuda_fail(e, "direct-sum kernel");
    if (use_partial) e = launch_reduce(k, table, 1, splits, out_dtype, 0.f, st);
  } else {
    e = launch_umma(k, table, 1, splits, tier, out_dtype, 0, plan.tile_n, plan.group_chunks, use_partial, sms,
                    P, pixels->dtype, status, counter, st);
    if (e == cudaErrorNotSupported) return fail(RSIM_ERR_UNSUPPORTED, "tensor-core tier not available");
    if (e != cudaSuccess) return cuda_fail(e, "tcgen05 contraction kernel");
    const bool scaled = (tier == RSIM_TIER_SPLIT_FP16 || tier == RSIM_TIER_FP16);
    if (use_partial) e = launch_reduce_tiles(k, table, 1, splits, plan.tile_n, out_dtype, scaled, sms, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "split reduction");
  return RSIM_OK;
}
