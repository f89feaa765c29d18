"""CPU FP64 oracle of the analytic-scene ray-caster that produces the per-pixel render
buffers (range, strength, angles, velocity) the cube synthesis consumes.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this module.  It shares no code with the CUDA library.

The paper renders each animation frame with Blender's ray tracer (Section II): the
light source sits at the Tx and the camera at the Rx, the camera's angle range stands
for the antenna pattern, and every pixel of the N_az x N_el image gives a range, a
strength, an angle of arrival and a velocity (the symbols after Eq. 2).  This module
is that rendering step for scenes built from analytic primitives, written from the
geometry of ray-surface intersection:

  * radar (camera and light) at the origin; x is the horizontal array axis, y the
    boresight, z up.  Pixel (i, j) of the cell-centred grid looks along
        d = (cos el_j sin az_i, cos el_j cos az_i, sin el_j),
    so d_x = cos(el) sin(az) is the direction cosine u of the cube synthesis;
  * the range of a pixel is the distance t > 0 to the first surface the ray meets,
    +inf when it meets none (a background miss, strength 0);
  * strength (Lambert surface lit by a point light at the radar, as a render with
    the lamp at the Tx gives it): rho |n . d| / R^2, real and non-negative; the
    1/R^2 falloff can be switched off;
  * velocity: the closing speed of the surface point, -(v_lin + omega x (x - a)) . d,
    where a is the primitive's pivot: positive when the point approaches the radar,
    the sign under which Eq. 1's Doppler term f_D = 2 v / lam lowers the slow-time
    phase.

Primitives (all vectors in metres, a scene is a list of dicts with numpy arrays):
  * "plane": parallelogram {a + s b + t c : 0 <= s, t <= 1}, two-sided;
  * "capsule": points within radius r of the segment a-b (a cylinder with
    hemispherical caps);
  * "ellipsoid": centre a, mutually orthogonal semi-axis vectors b, c, d.
Every primitive carries vel (linear velocity of a), omega (angular velocity about a)
and rho (reflectivity).
"""
from __future__ import annotations

import numpy as np

INF = float("inf")


def pixel_directions(n_az, n_el, az_range, el_range):
    """Cell-centred pixel angles and unit ray directions, flattened p = j n_az + i."""
    az0, az1 = az_range
    el0, el1 = el_range
    az1d = az0 + (np.arange(n_az) + 0.5) * (az1 - az0) / n_az
    el1d = el0 + (np.arange(n_el) + 0.5) * (el1 - el0) / n_el
    az = np.tile(az1d, n_el)
    el = np.repeat(el1d, n_az)
    d = np.stack([np.cos(el) * np.sin(az), np.cos(el) * np.cos(az), np.sin(el)], axis=1)
    return az, el, d


def _first_positive(t1, t2):
    """Smallest positive of two candidate distances (inf where neither is)."""
    t1 = np.where(t1 > 0, t1, INF)
    t2 = np.where(t2 > 0, t2, INF)
    return np.minimum(t1, t2)


def _quadratic_roots(qa, qb, qc):
    """Real roots of qa t^2 + qb t + qc = 0 (qa > 0), NaN where there are none."""
    disc = qb * qb - 4.0 * qa * qc
    ok = disc >= 0
    sq = np.sqrt(np.where(ok, disc, 0.0))
    with np.errstate(invalid="ignore", divide="ignore"):
        t1 = np.where(ok, (-qb - sq) / (2.0 * qa), np.nan)
        t2 = np.where(ok, (-qb + sq) / (2.0 * qa), np.nan)
    return t1, t2


def hit_plane(d, prim):
    """Distance along each unit ray d (from the origin) to the parallelogram."""
    a, b, c = (np.asarray(prim[k], float) for k in ("a", "b", "c"))
    n = np.cross(b, c)
    dn = d @ n
    with np.errstate(invalid="ignore", divide="ignore"):
        t = np.where(dn != 0, (a @ n) / dn, INF)
        x = d * t[:, None] - a  # NaN on rays parallel to the plane: dropped below
    # coordinates (s, t) of x in the basis (b, c): solve the 2x2 Gram system
    bb, cc, bc = b @ b, c @ c, b @ c
    det = bb * cc - bc * bc
    xb, xc = x @ b, x @ c
    with np.errstate(invalid="ignore"):
        s = (cc * xb - bc * xc) / det
        u = (bb * xc - bc * xb) / det
        inside = (s >= 0) & (s <= 1) & (u >= 0) & (u <= 1) & np.isfinite(t) & (t > 0)
    return np.where(inside, t, INF)


def hit_ellipsoid(d, prim):
    """Distance to the ellipsoid: in coordinates s_i = (x - a) . e_i / |e_i|^2 it is the
    unit sphere, so |s0 + t s_d|^2 = 1 is a quadratic in t."""
    a = np.asarray(prim["a"], float)
    E = np.stack([np.asarray(prim[k], float) for k in ("b", "c", "d")])  # rows e_i
    w = E / (E * E).sum(axis=1, keepdims=True)  # e_i / |e_i|^2
    s0 = (-a) @ w.T  # (3,)
    sd = d @ w.T  # (P, 3)
    qa = (sd * sd).sum(axis=1)
    qb = 2.0 * (sd @ s0)
    qc = s0 @ s0 - 1.0
    t1, t2 = _quadratic_roots(qa, qb, np.full_like(qa, qc))
    return _first_positive(np.nan_to_num(t1, nan=-1.0), np.nan_to_num(t2, nan=-1.0))


def _hit_sphere(d, centre, r):
    qb = -2.0 * (d @ centre)
    qc = centre @ centre - r * r
    t1, t2 = _quadratic_roots(np.ones(d.shape[0]), qb, np.full(d.shape[0], qc))
    return _first_positive(np.nan_to_num(t1, nan=-1.0), np.nan_to_num(t2, nan=-1.0))


def hit_capsule(d, prim):
    """Distance to the capsule: the infinite cylinder of radius r about the line a-b,
    kept where the foot of the hit point lies between a and b, and the two end
    spheres; the nearest positive of the three."""
    a, b = np.asarray(prim["a"], float), np.asarray(prim["b"], float)
    r = float(prim["c"][0])
    axis = b - a
    h2 = axis @ axis
    # x(t) = t d; the part of x - a across the axis is t d_perp + ap with
    # v_perp = v - (v . axis / h2) axis and ap = (0 - a)_perp: |t d_perp + ap|^2 = r^2
    dp = d - np.outer(d @ axis / h2, axis)
    ap = -a - (((-a) @ axis) / h2) * axis
    qa = (dp * dp).sum(axis=1)
    qb = 2.0 * (dp @ ap)
    qc = ap @ ap - r * r
    with np.errstate(invalid="ignore", divide="ignore"):
        t1, t2 = _quadratic_roots(np.where(qa > 0, qa, 1.0), qb, np.full_like(qa, qc))
    tc = np.full(d.shape[0], INF)
    for tt in (t1, t2):
        tt = np.where(qa > 0, tt, np.nan)
        foot = ((d * tt[:, None] - a) @ axis) / h2
        ok = np.isfinite(tt) & (tt > 0) & (foot >= 0) & (foot <= 1)
        tc = np.where(ok, np.minimum(tc, tt), tc)
    return np.minimum(tc, np.minimum(_hit_sphere(d, a, r), _hit_sphere(d, b, r)))


def surface_normal(x, prim):
    """Outward unit normal of the primitive at surface points x (for a plane, b x c)."""
    kind = prim["kind"]
    a = np.asarray(prim["a"], float)
    if kind == "plane":
        n = np.cross(np.asarray(prim["b"], float), np.asarray(prim["c"], float))
        n = np.broadcast_to(n, x.shape)
    elif kind == "ellipsoid":
        E = np.stack([np.asarray(prim[k], float) for k in ("b", "c", "d")])
        w = E / (E * E).sum(axis=1, keepdims=True)
        s = (x - a) @ w.T  # local coordinates
        n = s @ w  # gradient of |s|^2 / 2: sum_i s_i e_i / |e_i|^2
    elif kind == "capsule":
        b = np.asarray(prim["b"], float)
        axis = b - a
        foot = np.clip(((x - a) @ axis) / (axis @ axis), 0.0, 1.0)
        n = x - (a + foot[:, None] * axis)
    else:
        raise ValueError(kind)
    return n / np.linalg.norm(n, axis=1, keepdims=True)


HITTERS = {"plane": hit_plane, "capsule": hit_capsule, "ellipsoid": hit_ellipsoid}


def raycast(scene, n_az, n_el, az_range, el_range, falloff=True):
    """Render buffers of a scene: dict of P = n_az n_el arrays range, sigma_re,
    sigma_im, az, el, vel (FP64), with p = j n_az + i.  Ties between primitives at
    the same distance go to the one listed first."""
    az, el, _ = pixel_directions(n_az, n_el, az_range, el_range)
    return raycast_angles(scene, az, el, falloff)


def raycast_angles(scene, az, el, falloff=True):
    """The same for rays at arbitrary angles (arrays az, el)."""
    az = np.asarray(az, float)
    el = np.asarray(el, float)
    d = np.stack([np.cos(el) * np.sin(az), np.cos(el) * np.cos(az), np.sin(el)], axis=1)
    P = d.shape[0]
    best = np.full(P, INF)
    which = np.full(P, -1)
    for k, prim in enumerate(scene):
        t = HITTERS[prim["kind"]](d, prim)
        nearer = t < best
        best = np.where(nearer, t, best)
        which = np.where(nearer, k, which)
    R = best.copy()
    sigma = np.zeros(P)
    vel = np.zeros(P)
    for k, prim in enumerate(scene):
        m = which == k
        if not m.any():
            continue
        x = d[m] * R[m, None]
        n = surface_normal(x, prim)
        cosi = np.abs((n * d[m]).sum(axis=1))
        sigma[m] = prim["rho"] * cosi / (R[m] ** 2 if falloff else 1.0)
        a = np.asarray(prim["a"], float)
        v_pt = np.asarray(prim["vel"], float) + np.cross(np.asarray(prim["omega"], float), x - a)
        vel[m] = -(v_pt * d[m]).sum(axis=1)
    return {"range": R, "sigma_re": sigma, "sigma_im": np.zeros(P), "az": az, "el": el, "vel": vel,
            "prim": which}
