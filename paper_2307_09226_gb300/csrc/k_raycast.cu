// Analytic-scene ray-caster: the rendering step that fills the per-pixel buffers of
// Eq. 2 (range, strength, angles, velocity; Section II renders them with the light at
// the Tx and the camera at the Rx).  See include/rsim.h for the geometry and the
// definition of each output.
//
// One kernel, rc_render, one thread per pixel: the ray direction from the pixel's
// angles, the first positive hit over all primitives, then normal, Lambert strength
// and closing speed at the hit point.  The primitives are staged in shared memory in
// tiles of 64, each thread of a block deriving one primitive's constants (unit normal,
// the dual basis of a plane, the unit-sphere frame of an ellipsoid, the constant terms
// of the quadratics) in the compute precision T = float for FP32 buffers, double for
// FP64 buffers.  A plane's in-plane coordinates use the dual basis b* = (c x n) / |n|^2,
// c* = (n x b) / |n|^2 (n = b x c), which needs no Gram determinant.
// Every curved surface is met as a sphere in some frame (the end caps as they are, the
// cylinder in the plane across its axis, the ellipsoid in its unit-sphere frame).  The
// roots of |f + t u|^2 = rr (u a unit vector) take the discriminant from the distance
// of the centre to the ray's line, rr - |f - (f . u) u|^2, and the near root as c / q,
// which keeps FP32 precision for rays that graze a surface (Haines, Guenther and
// Akenine-Moller, "Precision Improvements for Ray/Sphere Intersection", Ray Tracing
// Gems, 2019).
#include <math.h>

#include <cmath>
#include <string>

#include "rsim_ctx.h"
#include "rsim_internal.h"

namespace rsim {
namespace {

constexpr int kRcTile = 64;  // primitives per shared-memory tile
constexpr int kRcThreads = 256;

template <typename T>
struct RcPrim {
  int kind;
  T a[3], v[3], om[3], rho;
  // plane:     e0 = b*, e1 = c* (dual basis: (x - a) = s b + u c gives s = (x - a) . b*,
  //            u = (x - a) . c*), e2 = unit normal; k0 = a . e2
  // capsule:   e0 = b - a (axis), e1 = ap (the origin's offset from the axis line, across
  //            it), e2 = b; k0 = |ap|^2 - r^2, k1 = |a|^2 - r^2, k2 = |b|^2 - r^2, k3 = 1 / |axis|^2
  // ellipsoid: e0, e1, e2 = e_i / |e_i|^2 (the unit-sphere frame); (k0, k1, k2) = s0 = -a . w_i,
  //            k3 = |s0|^2 - 1
  T e0[3], e1[3], e2[3];
  T k0, k1, k2, k3;
  T rr;  // capsule: r^2
};

template <typename T>
__device__ __forceinline__ T dot3t(const T* x, const T* y) {
  return x[0] * y[0] + x[1] * y[1] + x[2] * y[2];
}

template <typename T>
__device__ __forceinline__ void cross3(const T* x, const T* y, T* z) {
  z[0] = x[1] * y[2] - x[2] * y[1];
  z[1] = x[2] * y[0] - x[0] * y[2];
  z[2] = x[0] * y[1] - x[1] * y[0];
}

// The per-primitive constants of the intersection test, in T.
template <typename T>
__device__ void derive(const rsim_primitive& p, RcPrim<T>& q) {
  T a[3], b[3], c[3], d[3];
  for (int i = 0; i < 3; ++i) {
    a[i] = (T)p.a[i];
    b[i] = (T)p.b[i];
    c[i] = (T)p.c[i];
    d[i] = (T)p.d[i];
    q.a[i] = a[i];
    q.v[i] = (T)p.vel[i];
    q.om[i] = (T)p.omega[i];
  }
  q.kind = p.kind;
  q.rho = (T)p.rho;
  q.k0 = q.k1 = q.k2 = q.k3 = (T)0;
  q.rr = (T)1;
  if (p.kind == RSIM_PRIM_PLANE) {
    T n[3], cn[3], nb[3];
    cross3(b, c, n);
    const T nn = dot3t(n, n), ln = sqrt(nn);
    cross3(c, n, cn);
    cross3(n, b, nb);
    for (int i = 0; i < 3; ++i) {
      q.e0[i] = cn[i] / nn;
      q.e1[i] = nb[i] / nn;
      q.e2[i] = n[i] / ln;
    }
    q.k0 = dot3t(a, q.e2);
  } else if (p.kind == RSIM_PRIM_CAPSULE) {
    const T r = c[0];
    T ax[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const T h2 = dot3t(ax, ax);
    const T f = -dot3t(a, ax) / h2;  // (origin - a) . axis / h2
    for (int i = 0; i < 3; ++i) {
      q.e0[i] = ax[i];
      q.e1[i] = -a[i] - f * ax[i];
      q.e2[i] = b[i];
    }
    q.rr = r * r;
    q.k0 = dot3t(q.e1, q.e1) - q.rr;
    q.k1 = dot3t(a, a) - q.rr;
    q.k2 = dot3t(b, b) - q.rr;
    q.k3 = (T)1 / h2;
  } else {  // ellipsoid
    const T* E[3] = {b, c, d};
    T* W[3] = {q.e0, q.e1, q.e2};
    T s0[3];
    for (int i = 0; i < 3; ++i) {
      const T ee = dot3t(E[i], E[i]);
      for (int j = 0; j < 3; ++j) W[i][j] = E[i][j] / ee;
      s0[i] = -dot3t(a, W[i]);
    }
    q.k0 = s0[0];
    q.k1 = s0[1];
    q.k2 = s0[2];
    q.k3 = dot3t(s0, s0) - (T)1;
  }
}

template <typename T>
__device__ __forceinline__ T t_inf() {
  return (T)INFINITY;
}

// The two roots t1 <= t2 of |f + t u|^2 = rr for a unit vector u, with c = |f|^2 - rr;
// false when the line misses the sphere.
template <typename T>
__device__ __forceinline__ bool sphere_roots(const T* f, const T* u, T rr, T c, T& t1, T& t2) {
  const T b = dot3t(f, u);
  const T g[3] = {f[0] - b * u[0], f[1] - b * u[1], f[2] - b * u[2]};
  const T disc = rr - dot3t(g, g);
  if (!(disc >= (T)0)) return false;
  const T q = -b - copysign(sqrt(disc), b);  // |q| = |b| + sqrt(disc): no cancellation
  t1 = q;
  t2 = (q != (T)0) ? c / q : q;
  if (t1 > t2) {
    const T x = t1;
    t1 = t2;
    t2 = x;
  }
  return true;
}

// Smallest positive root of |f + t u|^2 = rr, +inf if none.
template <typename T>
__device__ __forceinline__ T sphere_first(const T* f, const T* u, T rr, T c) {
  T t1, t2;
  if (!sphere_roots(f, u, rr, c, t1, t2)) return t_inf<T>();
  return t1 > (T)0 ? t1 : (t2 > (T)0 ? t2 : t_inf<T>());
}

// Distance along the unit ray d to the primitive (+inf if it misses).
template <typename T>
__device__ T hit(const RcPrim<T>& p, const T* d) {
  if (p.kind == RSIM_PRIM_PLANE) {
    const T dn = dot3t(d, p.e2);
    if (dn == (T)0) return t_inf<T>();
    const T t = p.k0 / dn;
    if (!(t > (T)0)) return t_inf<T>();
    T x[3] = {t * d[0] - p.a[0], t * d[1] - p.a[1], t * d[2] - p.a[2]};
    const T s = dot3t(x, p.e0), u = dot3t(x, p.e1);
    return (s >= (T)0 && s <= (T)1 && u >= (T)0 && u <= (T)1) ? t : t_inf<T>();
  }
  if (p.kind == RSIM_PRIM_CAPSULE) {
    // lateral surface: in the plane across the axis the ray is t dp (dp = d across the
    // axis) from the offset ap, a circle of radius r about the axis; keep the hits whose
    // foot on the axis lies between a and b
    T best = t_inf<T>();
    const T da = dot3t(d, p.e0);
    const T dp[3] = {d[0] - da * p.k3 * p.e0[0], d[1] - da * p.k3 * p.e0[1], d[2] - da * p.k3 * p.e0[2]};
    const T lp = sqrt(dot3t(dp, dp));
    if (lp > (T)0) {
      const T u[3] = {dp[0] / lp, dp[1] / lp, dp[2] / lp};
      T s1, s2;
      if (sphere_roots(p.e1, u, p.rr, p.k0, s1, s2)) {
        const T aax = dot3t(p.a, p.e0);
        const T ts[2] = {s1 / lp, s2 / lp};
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const T t = ts[i];
          const T foot = (t * da - aax) * p.k3;
          if (t > (T)0 && foot >= (T)0 && foot <= (T)1 && t < best) best = t;
        }
      }
    }
    // the end spheres about a and b, seen from the origin: f = -a, -b
    const T fa[3] = {-p.a[0], -p.a[1], -p.a[2]};
    const T fb[3] = {-p.e2[0], -p.e2[1], -p.e2[2]};
    const T ta = sphere_first(fa, d, p.rr, p.k1);
    const T tb = sphere_first(fb, d, p.rr, p.k2);
    return fmin(best, fmin(ta, tb));
  }
  // ellipsoid: the unit sphere |s0 + t sd|^2 = 1 in its frame, t = tau / |sd|
  const T sd[3] = {dot3t(d, p.e0), dot3t(d, p.e1), dot3t(d, p.e2)};
  const T ls = sqrt(dot3t(sd, sd));
  const T u[3] = {sd[0] / ls, sd[1] / ls, sd[2] / ls};
  const T s0[3] = {p.k0, p.k1, p.k2};
  return sphere_first(s0, u, (T)1, p.k3) / ls;
}

template <typename T>
__device__ void normal_at(const RcPrim<T>& p, const T* x, T* n) {
  if (p.kind == RSIM_PRIM_PLANE) {
    n[0] = p.e2[0];
    n[1] = p.e2[1];
    n[2] = p.e2[2];
  } else if (p.kind == RSIM_PRIM_CAPSULE) {
    const T xa[3] = {x[0] - p.a[0], x[1] - p.a[1], x[2] - p.a[2]};
    T f = dot3t(xa, p.e0) * p.k3;
    f = f < (T)0 ? (T)0 : (f > (T)1 ? (T)1 : f);
    for (int i = 0; i < 3; ++i) n[i] = xa[i] - f * p.e0[i];
  } else {
    const T xa[3] = {x[0] - p.a[0], x[1] - p.a[1], x[2] - p.a[2]};
    const T s[3] = {dot3t(xa, p.e0), dot3t(xa, p.e1), dot3t(xa, p.e2)};
    for (int i = 0; i < 3; ++i) n[i] = s[0] * p.e0[i] + s[1] * p.e1[i] + s[2] * p.e2[i];
  }
}

template <typename T>
__global__ void __launch_bounds__(kRcThreads)
rc_render(const rsim_primitive* __restrict__ prims, int n_prims, int n_az, int n_el, double az0, double az1,
          double el0, double el1, int falloff, T* __restrict__ R, T* __restrict__ sre, T* __restrict__ sim,
          T* __restrict__ az_out, T* __restrict__ el_out, T* __restrict__ vel) {
  wait_prior_grid();
  __shared__ RcPrim<T> tile[kRcTile];
  const int64_t P = (int64_t)n_az * n_el;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = p < P;
  const int i = live ? (int)(p % n_az) : 0, j = live ? (int)(p / n_az) : 0;
  // pixel angles in FP64 in the order of the cell-centred grid formula, unfused
  const double azd = __dadd_rn(az0, __ddiv_rn(__dmul_rn((double)i + 0.5, __dsub_rn(az1, az0)), (double)n_az));
  const double eld = __dadd_rn(el0, __ddiv_rn(__dmul_rn((double)j + 0.5, __dsub_rn(el1, el0)), (double)n_el));
  const T a = (T)azd, e = (T)eld;
  T sa, ca, se, ce;
  if (sizeof(T) == 4) {
    float s1, c1, s2, c2;
    sincosf((float)a, &s1, &c1);
    sincosf((float)e, &s2, &c2);
    sa = (T)s1, ca = (T)c1, se = (T)s2, ce = (T)c2;
  } else {
    double s1, c1, s2, c2;
    sincos((double)a, &s1, &c1);
    sincos((double)e, &s2, &c2);
    sa = (T)s1, ca = (T)c1, se = (T)s2, ce = (T)c2;
  }
  const T d[3] = {ce * sa, ce * ca, se};
  T best = t_inf<T>();
  int which = -1;
  for (int k0 = 0; k0 < n_prims; k0 += kRcTile) {
    const int nt = min(kRcTile, n_prims - k0);
    __syncthreads();
    for (int k = threadIdx.x; k < nt; k += blockDim.x) derive(prims[k0 + k], tile[k]);
    __syncthreads();
    if (live) {
      for (int k = 0; k < nt; ++k) {
        const T t = hit(tile[k], d);
        if (t < best) {  // strict: a tie keeps the primitive listed first
          best = t;
          which = k0 + k;
        }
      }
    }
  }
  if (!live) return;
  T r = t_inf<T>(), s = (T)0, w = (T)0;
  if (which >= 0) {
    RcPrim<T> q;
    if (n_prims <= kRcTile)
      q = tile[which];  // the only tile is still staged
    else
      derive(prims[which], q);
    r = best;
    const T x[3] = {r * d[0], r * d[1], r * d[2]};
    T n[3];
    normal_at(q, x, n);
    const T cosi = fabs(dot3t(n, d)) / sqrt(dot3t(n, n));
    s = q.rho * cosi;
    if (falloff) s = s / (r * r);
    const T xa[3] = {x[0] - q.a[0], x[1] - q.a[1], x[2] - q.a[2]};
    const T u[3] = {q.v[0] + q.om[1] * xa[2] - q.om[2] * xa[1], q.v[1] + q.om[2] * xa[0] - q.om[0] * xa[2],
                    q.v[2] + q.om[0] * xa[1] - q.om[1] * xa[0]};
    w = -dot3t(u, d);
  }
  R[p] = r;
  sre[p] = s;
  sim[p] = (T)0;
  az_out[p] = a;
  el_out[p] = e;
  vel[p] = w;
}

bool finite3(const double* x) { return std::isfinite(x[0]) && std::isfinite(x[1]) && std::isfinite(x[2]); }
double hdot(const double* x, const double* y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; }

// Argument checks of one primitive (the conditions rsim.h lists); "" when valid.
std::string check_prim(const rsim_primitive& p) {
  if (p.kind != RSIM_PRIM_PLANE && p.kind != RSIM_PRIM_CAPSULE && p.kind != RSIM_PRIM_ELLIPSOID)
    return "unknown primitive kind";
  if (!finite3(p.a) || !finite3(p.b) || !finite3(p.c) || !finite3(p.d) || !finite3(p.vel) ||
      !finite3(p.omega) || !std::isfinite(p.rho))
    return "non-finite primitive field";
  if (p.kind == RSIM_PRIM_PLANE) {
    const double bb = hdot(p.b, p.b), cc = hdot(p.c, p.c), bc = hdot(p.b, p.c);
    if (!(bb > 0 && cc > 0 && bb * cc - bc * bc > 1e-12 * bb * cc)) return "plane edges are zero or (nearly) parallel";
  } else if (p.kind == RSIM_PRIM_CAPSULE) {
    if (!(p.c[0] > 0)) return "capsule radius must be > 0";
    const double ax[3] = {p.b[0] - p.a[0], p.b[1] - p.a[1], p.b[2] - p.a[2]};
    if (!(hdot(ax, ax) > 0)) return "capsule ends coincide";
  } else {
    const double* E[3] = {p.b, p.c, p.d};
    for (int i = 0; i < 3; ++i)
      if (!(hdot(E[i], E[i]) > 0)) return "ellipsoid semi-axis is zero";
    for (int i = 0; i < 3; ++i)
      for (int j = i + 1; j < 3; ++j)
        if (std::fabs(hdot(E[i], E[j])) > 1e-9 * std::sqrt(hdot(E[i], E[i]) * hdot(E[j], E[j])))
          return "ellipsoid semi-axes are not orthogonal";
  }
  return "";
}

template <typename T>
cudaError_t launch_raycast(const rsim_primitive* raw, int n, const rsim_camera& cam, const rsim_pixel_out& out,
                           cudaStream_t st) {
  const int64_t blocks = (out.P + kRcThreads - 1) / kRcThreads;
  return launch_dependent(rc_render<T>, dim3((unsigned)blocks), dim3(kRcThreads), 0, st, raw, n, cam.n_az,
                          cam.n_el, cam.az_min, cam.az_max, cam.el_min, cam.el_max,
                          (cam.flags & RSIM_RC_NO_FALLOFF) ? 0 : 1, (T*)out.range, (T*)out.sigma_re,
                          (T*)out.sigma_im, (T*)out.az, (T*)out.el, (T*)out.vel);
}

}  // namespace
}  // namespace rsim

using namespace rsim;

extern "C" rsim_status rsim_raycast(rsim_ctx* ctx, const rsim_camera* cam, const rsim_primitive* prims,
                                    int32_t n_prims, const rsim_pixel_out* out, rsim_stream stream) {
  if (!ctx || !cam || !out) return fail(RSIM_ERR_INVALID_ARG, "NULL argument");
  if (n_prims < 0 || (n_prims > 0 && !prims)) return fail(RSIM_ERR_INVALID_ARG, "bad primitive array");
  if (cam->n_az < 1 || cam->n_el < 1) return fail(RSIM_ERR_INVALID_ARG, "n_az and n_el must be >= 1");
  if (!std::isfinite(cam->az_min) || !std::isfinite(cam->az_max) || !std::isfinite(cam->el_min) ||
      !std::isfinite(cam->el_max))
    return fail(RSIM_ERR_INVALID_ARG, "non-finite camera angle");
  if (cam->flags & ~RSIM_RC_NO_FALLOFF) return fail(RSIM_ERR_INVALID_ARG, "unknown camera flag bits");
  if (out->P != (int64_t)cam->n_az * cam->n_el) return fail(RSIM_ERR_INVALID_ARG, "out->P != n_az * n_el");
  if (out->dtype != RSIM_F32 && out->dtype != RSIM_F64) return fail(RSIM_ERR_INVALID_ARG, "unknown dtype");
  if (!out->range || !out->sigma_re || !out->sigma_im || !out->az || !out->el || !out->vel)
    return fail(RSIM_ERR_INVALID_ARG, "NULL output array");
  if ((out->P + kRcThreads - 1) / kRcThreads > 0x7fffffffll) return fail(RSIM_ERR_OVERFLOW, "too many pixels");
  for (int k = 0; k < n_prims; ++k) {
    const std::string why = check_prim(prims[k]);
    if (!why.empty()) return fail(RSIM_ERR_INVALID_ARG, "primitive " + std::to_string(k) + ": " + why);
  }
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t raw_bytes = ((sizeof(rsim_primitive) * (size_t)n_prims + 255) / 256) * 256;
  rsim_status s = ensure_workspace(ctx, raw_bytes + 256, st);
  if (s != RSIM_OK) return s;
  char* ws = (char*)ctx->ws;
  cudaError_t e = cudaSuccess;
  if (n_prims > 0) {
    e = cudaMemcpyAsync(ws, prims, sizeof(rsim_primitive) * (size_t)n_prims, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "upload of the primitives");
  }
  const rsim_primitive* raw = (const rsim_primitive*)ws;
  if (out->dtype == RSIM_F32)
    e = launch_raycast<float>(raw, n_prims, *cam, *out, st);
  else
    e = launch_raycast<double>(raw, n_prims, *cam, *out, st);
  if (e != cudaSuccess) return cuda_fail(e, "ray-caster kernels");
  return RSIM_OK;
}
