/*
 * rsim.h — C ABI of the GB300 (sm_103a) library for TDM-MIMO FMCW beat-signal
 * data-cube synthesis from per-pixel render buffers.
 *
 * What the library computes (Eq. 1 and Eq. 2 of "A Blender-based channel simulator
 * for FMCW Radar", Section II), with 0-based n < N_s, l < L and virtual channel
 * v = m * N + r (Tx m < M, Rx r < N):
 *
 *   valid_p       = (sigma_p != 0)                         background misses drop out
 *   u_p           = cos(el_p) * sin(az_p)                  direction cosine (Eq. 2 AoA)
 *   R_{p,v}       = R_p + v * d_rx * u_p / 2               path range R_{m,n} (Eq. 1)
 *   f_D,p         = 2 * vel_p / lambda                     Doppler (Eq. 1, Eq. 2)
 *   phi(p,v,n,l)  = 2 mu R_{p,v} / c * n / F_s             fast time (Eq. 1)
 *                 + v * d_rx * u_p / lambda                spatial term (Eq. 2)
 *                 - f_D,p * l * T_slow                     slow time (Eq. 1)
 *   cube[v][n][l] = sum over valid p of sigma_p * exp(j 2 pi phi(p,v,n,l))
 *
 * Readings where the paper is silent or garbled: T_slow is the TDM block period
 * (default M * T_b; Eq. 1 steps the phase once per block of M chirps and Eq. 2's
 * extra "/L" is read as a typo); the sum over m is kept as M*N virtual channels;
 * d_rx defaults to lambda / 2 (Eq. 2 definitions); sigma is a complex amplitude.
 *
 * Conventions for every call:
 *  - All array pointers are DEVICE pointers owned by the caller, unless a comment
 *    says otherwise.  The library never frees caller memory; it owns only the
 *    workspace held by an rsim_ctx.
 *  - Every call returns an rsim_status; no C++ exception crosses the ABI.  On an
 *    error, rsim_last_error() returns a message for the calling thread, and the
 *    contents of output buffers are unspecified.
 *  - Calls that take a stream are asynchronous on it (they enqueue kernels and
 *    return).  Checks that need device data (non-finite fields of valid pixels,
 *    device-side wait limits) set a status word in the context; rsim_sync_status()
 *    waits for the stream and returns and clears it.
 *  - Sizes are checked in 64-bit arithmetic; products that overflow give
 *    RSIM_ERR_OVERFLOW.
 *  - One rsim_ctx must not be used by two host threads at once, and work enqueued
 *    through it on one stream must complete before it is reused on another (its
 *    workspace is shared).  Use one context per stream, or the server below.
 *  - rsim_synth and rsim_synth_host may be captured into a CUDA graph (stream
 *    capture) once an uncaptured call of the same shape and tier has sized the
 *    context's workspace (and, for rsim_synth_host, its staging buffer): the captured
 *    call allocates nothing.  The graph holds those buffers' addresses, so a later call
 *    on the context that grows them frees the memory the graph uses; a graph must not be
 *    replayed after such a call.  A replay runs the whole call (every kernel) again.
 */
#ifndef RSIM_H_
#define RSIM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream handle (cudaStream_t / CUstream); NULL is the legacy default stream. */
typedef struct CUstream_st* rsim_stream;

typedef enum {
  RSIM_OK = 0,
  RSIM_ERR_INVALID_ARG = 1,  /* NULL pointer, non-positive size, unknown enum value */
  RSIM_ERR_NONFINITE = 2,    /* a valid pixel has a non-finite field or R <= 0 */
  RSIM_ERR_OVERFLOW = 3,     /* a size product does not fit in 64 bits / int32 index */
  RSIM_ERR_OOM = 4,          /* device allocation of the workspace failed */
  RSIM_ERR_BUDGET = 5,       /* request larger than the configured HBM budget */
  RSIM_ERR_TIMEOUT = 6,      /* a device-side or host-side wait ran out of time */
  RSIM_ERR_CANCELLED = 7,    /* a server request was cancelled before it ran */
  RSIM_ERR_CUDA = 8,         /* a CUDA runtime call failed (message has the detail) */
  RSIM_ERR_UNSUPPORTED = 9,  /* valid request the library does not handle (shape, tier, device) */
  RSIM_ERR_NOT_FOUND = 10    /* unknown server ticket */
} rsim_status;

/* Arithmetic tier of the contraction over pixels. */
typedef enum {
  RSIM_TIER_FP32 = 0,       /* FP32 direct sum on CUDA cores */
  RSIM_TIER_BF16 = 1,       /* tcgen05 tensor cores, BF16 operands, FP32 accumulate */
  RSIM_TIER_SPLIT_BF16 = 2, /* tcgen05, BF16 hi+lo operands (3 products), FP32 accumulate */
  RSIM_TIER_SPLIT_FP16 = 3, /* tcgen05, FP16 hi+lo operands (3 products), FP32 accumulate */
  RSIM_TIER_FP16 = 4,       /* tcgen05, FP16 operands, FP32 accumulate */
  RSIM_TIER_NUFFT = 5       /* type-1 non-uniform FFT per channel on CUDA cores: ES-kernel
                               gridding (width 4..8, default 7: RSIM_NUFFT_WIDTH; oversampling
                               >= 2) with exact fixed-point
                               sums, FP32 FFTs; relative error ~1e-6.  N_s and L in 4..2048
                               (else UNSUPPORTED) */
} rsim_tier;

/* Element type of the pixel arrays (all six share it). */
enum { RSIM_F32 = 0, RSIM_F64 = 1 };
/* Element type of the cube: interleaved (re, im) pairs. */
enum { RSIM_C64 = 0, RSIM_C128 = 1 };

/* Radar parameters (symbols of Eq. 1; SI units). */
typedef struct {
  int32_t M;       /* Tx antennas, >= 1 */
  int32_t N;       /* Rx antennas, >= 1 */
  int32_t Ns;      /* fast-time samples per chirp, >= 1 */
  int32_t L;       /* TDM blocks (slow-time samples), >= 1 */
  double lambda;   /* carrier wavelength [m], > 0 */
  double d_rx;     /* Rx spacing [m]; <= 0 selects lambda / 2 */
  double mu;       /* chirp slope [Hz/s] */
  double fs;       /* fast-time sampling rate [Hz], > 0 */
  double t_b;      /* chirp duration [s] */
  double t_slow;   /* TDM block period [s]; <= 0 selects M * t_b */
  double c;        /* propagation speed [m/s]; <= 0 selects 299792458 */
  int32_t flags;   /* RSIM_FLAG_* bits; 0 = the model of Eq. 1/Eq. 2 as stated */
  int32_t reserved;
} rsim_radar_params;

/* Add the TDM motion phase: Tx m transmits in slot m of each block, so a moving pixel's
 * Doppler also turns the phase by -f_D m T_b across the Tx slots (a per-(pixel, channel)
 * constant added to phi).  Eq. 1 omits it (every Tx is taken at the block start). */
#define RSIM_FLAG_TDM_MOTION 1

/* NUFFT tier only: the gridding kernel's width w in cells (flags bits 8..11), which sets
 * the accuracy: relative error about 10^-(w-1) (w = 7, the default when the bits are
 * 0, gives ~1e-6) and a spreading cost of w^2 taps per (channel, pixel).  w in 4..8; other
 * tiers ignore the bits. */
#define RSIM_NUFFT_WIDTH(w) ((int32_t)(w) << 8)
#define RSIM_NUFFT_WIDTH_MASK 0xF00

/* One frame's render buffers: six arrays of P elements, flattened [el][az]
 * (structure of arrays), all of element type `dtype`.  sigma = (sigma_re, sigma_im)
 * is the complex amplitude; a pixel with sigma == 0 (either zero sign) is ignored
 * whatever its other fields hold. */
typedef struct {
  int64_t P;
  int32_t dtype;   /* RSIM_F32 or RSIM_F64 */
  int32_t reserved;
  const void* range;    /* R_p [m], > 0 and finite for valid pixels */
  const void* sigma_re;
  const void* sigma_im;
  const void* az;       /* azimuth [rad] */
  const void* el;       /* elevation [rad] */
  const void* vel;      /* radial velocity [m/s] (f_D = 2 vel / lambda) */
} rsim_pixels;

typedef struct rsim_ctx rsim_ctx;

/* Version string of the library (static storage). */
const char* rsim_version(void);

/* Message of the last error on the calling thread ("" if none); static per thread. */
const char* rsim_last_error(void);

/* Create a context on `device`.  hbm_budget_bytes bounds the workspace the context
 * may hold (0 = no bound).  *out receives the context.  Errors: INVALID_ARG, CUDA. */
rsim_status rsim_create(rsim_ctx** out, int device, size_t hbm_budget_bytes);

/* Destroy a context and free its workspace (waits for the device first).  NULL is a no-op. */
rsim_status rsim_destroy(rsim_ctx* ctx);

/* Device workspace (bytes) that rsim_synth needs for P pixels with these parameters
 * and tier.  Host-only computation.  Errors: INVALID_ARG, OVERFLOW. */
rsim_status rsim_workspace_size(rsim_ctx* ctx, const rsim_radar_params* params, int64_t P,
                                rsim_tier tier, size_t* bytes);

/* Synthesise one frame's cube (Eq. 2 summed over all valid pixels).
 * cube: device buffer of M*N*Ns*L complex values, C-contiguous [M*N][Ns][L],
 * complex64 (RSIM_C64) or complex128 (RSIM_C128), fully overwritten.  The pixel
 * buffers are only read.  The context workspace grows if needed (cudaMalloc; the
 * call then synchronises the device once).  Asynchronous on `stream`.
 * Errors: INVALID_ARG, OVERFLOW, OOM, BUDGET, CUDA; NONFINITE via rsim_sync_status. */
rsim_status rsim_synth(rsim_ctx* ctx, const rsim_radar_params* params, const rsim_pixels* pixels,
                       rsim_tier tier, void* cube, int32_t out_dtype, rsim_stream stream);

/* rsim_synth on HOST buffers, for callers whose render buffers live in host memory
 * and who want the cube back there.  The six pixel arrays (`pixels`) and `cube`
 * ([M*N][Ns][L] complex64 or complex128) are HOST pointers.  The call copies the pixel
 * arrays into a device staging buffer owned by the context (one cudaMemcpyAsync per
 * array), synthesises the cube there exactly as rsim_synth does, and copies it back
 * (one cudaMemcpyAsync), all on `stream`.  When the pixel arrays are reachable from the
 * device (page-locked memory, or any host memory on a node whose GPU reads pageable
 * memory through the host page tables, as over NVLink-C2C), the kernels read them in
 * place instead of copies.  The cube is always staged and comes back in one piece: into
 * page-locked memory (16-byte aligned, a whole number of 16-byte units) by a copy kernel
 * through its mapped address, else by one cudaMemcpyAsync.
 * Either way the results are those of rsim_synth, and the host buffers must stay valid
 * and unchanged until the stream has passed the call's work (e.g. rsim_sync_status); with
 * pageable memory and no direct access the copies block the calling thread.  The staging buffer grows when
 * needed (cudaMalloc after one stream synchronisation) and counts against the context's
 * budget with the workspace.
 * Errors: as rsim_synth. */
rsim_status rsim_synth_host(rsim_ctx* ctx, const rsim_radar_params* params, const rsim_pixels* pixels,
                            rsim_tier tier, void* cube, int32_t out_dtype, rsim_stream stream);

/* Synthesise F frames that share one radar configuration in one pass: one launch
 * per stage over all frames, the contraction as one persistent launch whose work
 * units (frame, row tile, column tile, pixel split) are taken from a device
 * counter, longest first.  frames: HOST array of F descriptors; cubes: HOST array
 * of F device pointers, each laid out as in rsim_synth.  Each frame's result is
 * bit-identical to rsim_synth of that frame alone with the same tier.  The NUFFT tier
 * runs the frames on up to eight streams of the context (each with its own grid
 * scratch), which wait for `stream` first; `stream` then waits for all of them, so the
 * call stays ordered on `stream` like every other.
 * Errors: as rsim_synth. */
rsim_status rsim_synth_batch(rsim_ctx* ctx, const rsim_radar_params* params,
                             const rsim_pixels* frames, int32_t F, void* const* cubes,
                             rsim_tier tier, int32_t out_dtype, rsim_stream stream);

/* One-frame synthesis that allocates nothing, for callers that must not allocate
 * device memory (a real-time processing loop whose device memory is fixed at
 * start-up, or a host framework that owns the device memory budget and forbids
 * libraries from calling cudaMalloc).  The paper has no counterpart: this is a
 * deployment variant of rsim_synth.
 *
 * Needs no rsim_ctx.  The scratch memory (compacted pixels, phases, split partial
 * sums, frame table, counters) is one array of 64 MiB compiled into the library;
 * every GPU that loads the library holds it until the process exits.  A frame
 * whose scratch would exceed 64 MiB is rejected with RSIM_ERR_BUDGET before
 * anything is launched.  Calls no cudaMalloc, cudaFree or other allocating routine.
 * Inputs and output are as in rsim_synth (device pointers owned by the caller); the
 * plan is the library's default rule for the shape, so the result equals rsim_synth
 * of a context that has no tuned plan for it.
 *
 * device_status: optional DEVICE pointer to a uint32 that the kernels OR their
 * status bits into (1: a valid pixel had a non-finite field or R <= 0; 2: a
 * device-side wait ran out of time); the caller clears it.  With NULL, the kernels
 * report into a word inside the static array that the next call clears, and nothing
 * reads it: a non-finite pixel or a wait that ran out then leaves a wrong cube while
 * the call still returns RSIM_OK.  Callers that need to know must pass a word.
 *
 * The first call on a device, with that device current, looks up the array's device
 * address (cudaGetSymbolAddress) and caches it per device for the life of the
 * process; make that first call before any stream capture.  With CUDA's lazy module
 * loading (the default) the array is committed in device memory when the library's
 * kernels are first loaded on that device, typically by this first call, so a process
 * with a fixed memory budget should make one warm-up call at start-up.  A device reset
 * (cudaDeviceReset, or a reset of the primary context) may move the array: the cached
 * address is then stale and this entry point must not be used again in that process.
 * All calls on a device share the one array and it keeps the last call's contents (the
 * call clears what must start at zero), so calls whose work overlaps on the GPU (other
 * streams, other host threads) race: serialise them.
 * Asynchronous on `stream`.  Errors: INVALID_ARG, OVERFLOW, BUDGET, UNSUPPORTED, CUDA. */
rsim_status rsim_synth_static(const rsim_radar_params* params, const rsim_pixels* pixels,
                              rsim_tier tier, void* cube, int32_t out_dtype, uint32_t* device_status,
                              rsim_stream stream);

/* Valid-pixel compaction alone (the mask step): idx receives the indices p with
 * sigma_p != 0 in ascending order (int32, capacity P), *p_valid (DEVICE int64) their
 * count.  Asynchronous on `stream`. */
rsim_status rsim_valid_indices(rsim_ctx* ctx, const rsim_pixels* pixels, int32_t* idx,
                               int64_t* p_valid, rsim_stream stream);

/* Pixel-to-path step alone (FP64): for the q-th valid pixel (ascending p) and channel v,
 *   a[v*P + q] = 2 mu R_{p,v} / (c F_s)   mod 1, as uint32 units of 2^-32 cycle/sample
 *   cph[v*P + q] = v d_rx u_p / lambda    mod 1, as uint32 units of 2^-32 cycle
 *   b[q]       = -f_D,p T_slow            mod 1, as uint32 units of 2^-32 cycle/block
 *   sigma[2q], sigma[2q+1] = FP32 (re, im) of sigma_p
 * (rounded to nearest).  a and cph hold V*P uint32, b holds P, sigma 2*P floats;
 * entries past the valid count are left untouched; *p_valid (DEVICE int64) gets the
 * count.  Asynchronous on `stream`.  Errors: as rsim_synth. */
rsim_status rsim_path_phases(rsim_ctx* ctx, const rsim_radar_params* params,
                             const rsim_pixels* pixels, uint32_t* a, uint32_t* cph, uint32_t* b,
                             float* sigma, int64_t* p_valid, rsim_stream stream);

/* Target estimation on complex64 cubes (Section III: an FFT of each CPI's cube gives
 * the range-Doppler map; the velocity of maximum power per CPI gives the Doppler-time
 * plot).  For each of the F cubes (HOST array of device pointers, laid out as in
 * rsim_synth with these params, complex64):
 *   power[f][k][d] = sum over channels v of |sum_n sum_l cube[v][n][l]
 *                    e^{-j 2 pi (k n / N_s + d l / L)}|^2          (DEVICE, float)
 *   v_est[f]       = velocity [m/s] of the Doppler bin of the largest power[f][k][d]
 *                    (first index on ties), v = -d_s lambda / (2 T_slow L) with d_s the
 *                    signed bin in [-L/2, L/2)                       (DEVICE, float)
 *   peak[2f], peak[2f+1] = (k, d) of that maximum (DEVICE int32, may be NULL).
 * options: RSIM_RD_SKIP_STATIC leaves the zero-Doppler column out of the search (a
 * static-clutter notch).  N_s and L must be powers of two up to 1024 (else UNSUPPORTED).
 * Uses the context workspace.  Asynchronous on `stream`. */
#define RSIM_RD_SKIP_STATIC 1
rsim_status rsim_range_doppler(rsim_ctx* ctx, const rsim_radar_params* params, void* const* cubes,
                               int32_t F, float* power, float* v_est, int32_t* peak, int32_t options,
                               rsim_stream stream);

/* ---------------------------------------------------------------------------------
 * Analytic-scene ray-caster: the rendering step that produces the per-pixel buffers
 * the synthesis consumes (Section II: the light source sits at the Tx and the camera at
 * the Rx, and every pixel of the N_az x N_el image gives a range, a strength, an angle
 * of arrival and a velocity, the symbols after Eq. 2).
 *
 * Geometry: radar at the origin, x the horizontal array axis, y boresight, z up.  Pixel
 * (i, j) of the cell-centred grid, p = j n_az + i, with
 *   az_i = az_min + (i + 1/2) (az_max - az_min) / n_az,  el_j likewise,
 * looks along d = (cos el sin az, cos el cos az, sin el), so d_x = cos(el) sin(az) is the
 * direction cosine of the synthesis.  Per pixel:
 *   range    = distance to the first surface with t > 0 along d, +inf when there is none;
 *   sigma_re = rho |n . d| / range^2 (Lambert surface lit from the radar; without the
 *              1/range^2 factor under RSIM_RC_NO_FALLOFF), sigma_im = 0; 0 for a miss;
 *   az, el   = the pixel's angles;
 *   vel      = -(vel + omega x (x - a)) . d, the closing speed of the surface point x the
 *              ray meets (positive when it approaches the radar: the sign under which
 *              Eq. 1's Doppler term f_D = 2 vel / lambda lowers the slow-time phase); 0
 *              for a miss.
 * A pixel whose distance ties between primitives takes the one listed first. */
typedef enum { RSIM_PRIM_PLANE = 0, RSIM_PRIM_CAPSULE = 1, RSIM_PRIM_ELLIPSOID = 2 } rsim_prim_kind;

typedef struct {
  int32_t kind;       /* rsim_prim_kind */
  int32_t reserved;
  double a[3];        /* plane: corner; capsule: end A; ellipsoid: centre (the pivot of omega) */
  double b[3];        /* plane: edge 1; capsule: end B; ellipsoid: semi-axis 1 */
  double c[3];        /* plane: edge 2; capsule: c[0] = radius; ellipsoid: semi-axis 2 */
  double d[3];        /* ellipsoid: semi-axis 3 (the three mutually orthogonal); else unused */
  double vel[3];      /* linear velocity of the pivot a, m/s */
  double omega[3];    /* angular velocity about a, rad/s */
  double rho;         /* reflectivity (scale of the strength) */
} rsim_primitive;     /* 160 bytes.  A plane is the two-sided parallelogram a + s b + t c,
                         0 <= s, t <= 1; a capsule all points within c[0] of the segment
                         a-b; an ellipsoid {a + sum_i s_i e_i : |s| <= 1}, e = (b, c, d) */

typedef struct {
  int32_t n_az, n_el;
  double az_min, az_max;  /* rad */
  double el_min, el_max;  /* rad */
  int32_t flags;          /* RSIM_RC_NO_FALLOFF */
  int32_t reserved;
} rsim_camera;            /* 48 bytes */
#define RSIM_RC_NO_FALLOFF 1

/* Writable pixel buffers (same layout as rsim_pixels): P = n_az n_el elements each, of
 * dtype RSIM_F32 (computed in FP32) or RSIM_F64 (computed in FP64).  DEVICE pointers. */
typedef struct {
  int64_t P;
  int32_t dtype;
  int32_t reserved;
  void *range, *sigma_re, *sigma_im, *az, *el, *vel;
} rsim_pixel_out;

/* Render `n_prims` primitives (HOST array, read before the call returns; may be NULL
 * when n_prims is 0) into `out`, whose arrays the caller owns.  INVALID_ARG for NULL
 * pointers, n_az or n_el < 1, P != n_az n_el, an unknown kind or dtype, a non-finite
 * number, a capsule radius <= 0 or coincident capsule ends, plane edges that are zero
 * or (nearly) parallel (sine of their angle below 1e-6), or ellipsoid semi-axes that
 * are zero or not mutually orthogonal (|e_i . e_j| > 1e-9 |e_i| |e_j|).
 * Uses the context workspace.  Asynchronous on `stream`. */
rsim_status rsim_raycast(rsim_ctx* ctx, const rsim_camera* cam, const rsim_primitive* prims,
                         int32_t n_prims, const rsim_pixel_out* out, rsim_stream stream);

/* Wait for `stream`, then return (and clear) the context's device-side status:
 * RSIM_OK, RSIM_ERR_NONFINITE or RSIM_ERR_TIMEOUT. */
rsim_status rsim_sync_status(rsim_ctx* ctx, rsim_stream stream);

/* Failure-detection self test (no counterpart in the paper: it checks the library's own
 * safeguard).  Every device-side wait in the library gives up after a time limit,
 * records RSIM_ERR_TIMEOUT in the context's status word and returns instead of hanging.
 * This call enqueues one small kernel that runs that bounded wait on a barrier phase
 * that nothing completes, with a limit of limit_ns nanoseconds (1e3 .. 1e10); the
 * kernel returns after about that long, and rsim_sync_status() then reports
 * RSIM_ERR_TIMEOUT once.  The context stays usable.  Asynchronous on `stream`.
 * Errors: INVALID_ARG (NULL ctx, limit out of range), CUDA. */
rsim_status rsim_selftest_wait_timeout(rsim_ctx* ctx, uint64_t limit_ns, rsim_stream stream);

/* Measurement helper for benchmarks (no counterpart in the paper): the rate, in lane
 * operations per second, at which this device performs non-returning 32-bit integer
 * atomic additions to shared memory without bank conflicts, at the NUFFT spreading
 * kernel's occupancy and access pattern.  That unit bounds the spreading kernel, so the
 * rate is its roofline denominator.  Runs a probe kernel six times on `stream` (the first
 * as a warm-up) and returns the best; synchronous.  Allocates nothing.
 * Errors: INVALID_ARG, CUDA. */
rsim_status rsim_measure_smem_atomics(rsim_ctx* ctx, double* lane_ops_per_s, rsim_stream stream);

/* Measurement helper for benchmarks (no counterpart in the paper): the flop rate of this
 * device's tensor cores on the contraction's instruction, tcgen05.mma kind::f16 with
 * M = 128, N = 256, K = 16, A from tensor memory, B from shared memory and FP32
 * accumulation, issued in the contraction's stages of 12 MMAs (one thread per CTA, at
 * most three committed stages in flight, one CTA per SM, zero operands).  It is the
 * ceiling of the contraction's executed flop rate.  Runs the probe six times on `stream`
 * (the first as a warm-up) and returns the best, in flop/s (2 per multiply-add);
 * synchronous.  Allocates nothing; every wait in the probe is bounded.
 * Errors: INVALID_ARG, UNSUPPORTED (not an sm_103 device), TIMEOUT (a probe wait ran
 * out), CUDA. */
rsim_status rsim_measure_mma_rate(rsim_ctx* ctx, double* flops_per_s, rsim_stream stream);

/* Stage timing for benchmarks.  While profiling is on, every rsim_synth /
 * rsim_synth_batch call records CUDA events on its stream around its three stages
 * (compaction + FP64 phases, contraction, split reduction), and around the main kernel
 * of the contraction stage: the tensor-core contraction (after the operand builder),
 * the FP32 direct sum, or the NUFFT tier's spreading kernel (first frame of a batch).  The events
 * stand between the stages' kernels, so profiled calls do not overlap one stage's
 * launch with the previous stage's end.  rsim_profile_read waits for the recorded
 * events, returns the summed stage times and launch counts since profiling was
 * switched on, and starts a new tally. */
typedef struct {
  int32_t calls;            /* synth calls recorded */
  int32_t kernels;          /* kernels those calls launched */
  double prep_ms;           /* summed device time of the compaction + phase kernels */
  double contract_ms;       /* summed device time of the contraction kernel */
  double reduce_ms;         /* summed device time of the split reduction (0 if none) */
  double operand_ms;        /* part of contract_ms before the main kernel: the operand builder
                               (tensor tiers), binning (NUFFT tier) */
  double main_ms;           /* the main kernel: contraction, direct sum, or NUFFT spreading */
} rsim_profile;

rsim_status rsim_profile_enable(rsim_ctx* ctx, int32_t on);
rsim_status rsim_profile_read(rsim_ctx* ctx, rsim_profile* out);

/* Kernel-launch plan of a shape: the tile shapes and the work split that the autotuner
 * decides.  Plans are kept per shape bucket: (tier, V = M N, N_s, L, ceil(log2 P)), so
 * frames and requests whose pixel counts lie in the same power-of-two range share one
 * plan.  Without a tuned or pinned plan for its bucket, a shape gets the default rule
 * (tile_n and group_chunks at their defaults, splits from the exact P).  A plan never
 * depends on the data or on the load, so the same frame always runs the same kernels
 * with the same summation order. */
typedef struct {
  int32_t splits;        /* pixel splits of the contraction (K-split), 1..64 */
  int32_t chunk_px;      /* pixels per pipeline stage (always 32; reported) */
  int32_t grid;          /* CTAs of the persistent tensor-core contraction, 0 = one per SM */
  int32_t variant;       /* reserved: must be 0 */
  int32_t tuned;         /* 1 if chosen by timing, 0 if by the default rule or pinned */
  int32_t tile_n;        /* tile shape.  Tensor-core tiers: l values per column tile, NT,
                            a multiple of 8 in 8..128 and at most L rounded up to 8 (the
                            MMA's N is 2 NT; default min(128, L rounded up to 8)).  FP32
                            tier: n values per CTA tile, 64 or 128 (default 128); the CTA
                            tile is tile_n x 64 (l).  NUFFT tier: ignored.  0 = default */
  int32_t group_chunks;  /* tensor-core tiers: 32-pixel chunks summed in one tensor-memory
                            accumulator before it is drained into round-to-nearest FP32
                            sums.  The accumulator rounds toward zero, so the cap bounds the
                            error: 1..40 for split tiers (default 40), 1..384 for plain
                            16-bit tiers (default 96).  Other tiers: ignored.  0 = default */
  int32_t reserved;
} rsim_plan;

/* Time candidate plans for the bucket of (params, P, tier) on `stream` with synthetic
 * full-valid pixels of count P, and keep the fastest for the bucket in the context's cache
 * (and in the JSON file named by the RSIM_TUNE_CACHE environment variable, if set).
 * Candidates: the split count around the default rule, the contraction's CTA count,
 * the column tile NT (tensor tiers) or the n tile (FP32), and the accumulation-group
 * length (tensor tiers, never above the accuracy caps of rsim_plan).  The choice
 * depends on the shape only.  Synchronous; allocates scratch with cudaMalloc.
 * Errors: as rsim_synth. */
rsim_status rsim_autotune(rsim_ctx* ctx, const rsim_radar_params* params, int64_t P,
                          rsim_tier tier, rsim_plan* chosen, rsim_stream stream);

/* Pin `plan` for the bucket of (params, P, tier) in the context's cache (replaces a tuned
 * or default plan).  splits in 1..64; grid 0 (one CTA per SM) or a positive CTA count
 * (more than the SM count runs as one per SM); variant 0; tile_n and group_chunks 0 or in
 * the ranges stated in rsim_plan.  Host only.  Errors: INVALID_ARG. */
rsim_status rsim_set_plan(rsim_ctx* ctx, const rsim_radar_params* params, int64_t P,
                          rsim_tier tier, const rsim_plan* plan);

/* The plan rsim_synth would use now for (params, P, tier), with tile_n and group_chunks
 * resolved (never 0 for the tiers that use them).  Host only. */
rsim_status rsim_get_plan(rsim_ctx* ctx, const rsim_radar_params* params, int64_t P,
                          rsim_tier tier, rsim_plan* plan);

/* ----------------------------------------------------------------------------------
 * Serving: continuous batching of cube-synthesis requests.
 *
 * A server owns `slots` slots, each with two CUDA streams and its own workspace.
 * submit() queues a request; a host scheduler thread admits queued requests as soon as a
 * slot is free and the request's workspace fits in the HBM budget still unreserved, and
 * launches each on its slot's stream, so requests that arrive while others run start as
 * soon as resources free up and their kernels overlap on the device.
 *
 * Which queued request goes next (rsim_server_opts.policy): RSIM_SERVE_FIRST_FIT takes
 * the oldest request that fits (a request too large for the free budget does not hold
 * back smaller ones behind it); RSIM_SERVE_SHORTEST_FIRST takes, among those that fit,
 * the one with the least estimated device time (path-samples at its tier's nominal rate;
 * oldest first among equals).  Either way a request may be passed over only until it has
 * waited age_limit_ms since its submission: from then on the oldest such request goes
 * next and nothing overtakes it, so no request starves.  A request whose estimated device
 * time is under 2 ms ("short") runs on the slot's high-priority stream, so its blocks
 * start ahead of long requests' pending blocks; the others run at low priority.  Express
 * slots (rsim_server_opts.express_slots), beyond the general ones, take short requests
 * only, so a short request does not wait in the queue while long requests hold every
 * general slot; a short request also goes to a free express slot first.  Results do not
 * depend on the policy or the priority.  Completion is detected by a host function after
 * the request's work; latency is measured from submit() to completion.
 * ---------------------------------------------------------------------------------- */
typedef struct rsim_server rsim_server;

enum { RSIM_SERVE_FIRST_FIT = 0, RSIM_SERVE_SHORTEST_FIRST = 1 };

typedef struct {
  int32_t slots;             /* general slots: concurrent requests of any size (1..64) */
  int32_t max_queue;         /* queued requests accepted before submit() refuses (BUDGET) */
  size_t hbm_budget_bytes;   /* bound on the sum of admitted workspaces (0 = no bound) */
  int32_t policy;            /* RSIM_SERVE_FIRST_FIT (0) or RSIM_SERVE_SHORTEST_FIRST */
  int32_t age_limit_ms;      /* a queued request may be overtaken until it has waited this
                                long (0 selects 100 ms; < 0: never overtaken, strict FIFO) */
  int32_t express_slots;     /* further slots for short requests only (0..64) */
  int32_t reserved;
} rsim_server_opts;

typedef struct {
  rsim_radar_params params;
  rsim_pixels pixels;        /* device buffers; must stay valid until the request completes */
  rsim_tier tier;
  int32_t out_dtype;
  void* cube;                /* device output, as in rsim_synth */
} rsim_request;

typedef struct {
  uint64_t submitted, completed, cancelled, failed;
  double p50_ms, p99_ms, mean_ms, max_ms;   /* submit -> completion latency */
  double busy_s;                            /* wall time from first submit to last completion */
  double path_samples;                      /* sum over completed of P_valid * V * N_s * L */
  size_t peak_reserved_bytes;               /* largest sum of admitted workspaces seen */
  int32_t peak_in_flight;                   /* largest number of concurrently running requests */
  int32_t reserved;
  double p99_queue_ms, max_queue_ms;        /* submit -> admission wait of completed requests */
  uint64_t overtakes;                       /* admissions that passed over an older queued request */
} rsim_server_stats;

rsim_status rsim_server_create(rsim_ctx* ctx, const rsim_server_opts* opts, rsim_server** out);
/* Queue a request; *ticket identifies it.  Errors: INVALID_ARG (bad request),
 * BUDGET (workspace larger than the whole budget, or queue full). */
rsim_status rsim_server_submit(rsim_server* s, const rsim_request* req, uint64_t* ticket);
/* Wait up to timeout_ms (< 0: no limit) for a ticket.  Returns the request's status
 * (OK, NONFINITE, CUDA, CANCELLED), TIMEOUT if it has not finished, NOT_FOUND if
 * the ticket is unknown or already collected.  A finished ticket is collected once. */
rsim_status rsim_server_wait(rsim_server* s, uint64_t ticket, int32_t timeout_ms);
/* Cancel a request that has not been admitted yet (running requests complete). */
rsim_status rsim_server_cancel(rsim_server* s, uint64_t ticket);
rsim_status rsim_server_stats_get(rsim_server* s, rsim_server_stats* out);
/* Start a new tally: clear the counters and latency samples (e.g. after a warm-up), keep
 * the slots and their workspaces.  Requests still in flight are counted in the new tally
 * when they complete. */
rsim_status rsim_server_stats_reset(rsim_server* s);
/* Stop the scheduler, wait for running requests, free slot workspaces. */
rsim_status rsim_server_destroy(rsim_server* s);

#ifdef __cplusplus
}
#endif
#endif /* RSIM_H_ */
