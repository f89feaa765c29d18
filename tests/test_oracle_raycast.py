"""Pins of the ray-caster oracle (CPU, no GPU): closed forms of simple geometry,
surface-membership and first-hit checks by brute force, and the velocity checked
against finite differences of ranges rendered at two instants."""
import numpy as np
import pytest

import oracle.raycast as rc
from paper_2307_09226_gb300 import synth

FOV = synth.CAMERA_FOV


def _sphere(centre, r, **kw):
    return synth._prim("ellipsoid", centre, (r, 0, 0), (0, r, 0), (0, 0, r), **kw)


def test_plane_facing_boresight_closed_form():
    # plane y = D spanning the whole field of view: R = D / d_y, cos(incidence) = D / R
    D, rho = 4.0, 0.7
    scene = [synth._prim("plane", (-50.0, D, -50.0), (100.0, 0, 0), (0, 0, 100.0), rho=rho)]
    o = rc.raycast(scene, 24, 12, *FOV)
    _, _, d = rc.pixel_directions(24, 12, *FOV)
    R = D / d[:, 1]
    np.testing.assert_allclose(o["range"], R, rtol=1e-13)
    np.testing.assert_allclose(o["sigma_re"], rho * (D / R) / R ** 2, rtol=1e-12)
    np.testing.assert_allclose(o["range"] * d[:, 1], D, rtol=1e-13)
    assert np.all(o["sigma_im"] == 0) and np.all(o["vel"] == 0)
    # without the 1/R^2 falloff the strength is rho cos(i)
    o2 = rc.raycast(scene, 24, 12, *FOV, falloff=False)
    np.testing.assert_allclose(o2["sigma_re"], rho * D / R, rtol=1e-12)


def test_sphere_silhouette_is_its_angular_radius():
    # a ray hits a sphere of radius r at distance D iff its angle to the centre < asin(r / D)
    D, r = 5.0, 1.2
    c = np.array([1.0, 4.0, 2.0])
    c = D * c / np.linalg.norm(c)
    o = rc.raycast([_sphere(c, r)], 96, 48, *FOV)
    _, _, d = rc.pixel_directions(96, 48, *FOV)
    ang = np.arccos(np.clip(d @ (c / D), -1, 1))
    alpha = np.arcsin(r / D)
    clear = np.abs(ang - alpha) > 1e-6
    assert np.array_equal(np.isfinite(o["range"])[clear], (ang < alpha)[clear])
    assert (ang < alpha).sum() > 50
    # hit points lie on the sphere, and the nearest surface point is D - r away
    hit = np.isfinite(o["range"])
    x = d[hit] * o["range"][hit, None]
    np.testing.assert_allclose(np.linalg.norm(x - c, axis=1), r, rtol=1e-12)
    assert o["range"][hit].min() >= D - r - 1e-12


def _first_crossing_by_marching(d, inside, tmax=20.0, n=20000):
    """Brute force: march each ray in steps of tmax / n and return the first sample
    inside the solid (inf if none)."""
    ts = np.linspace(0.0, tmax, n + 1)[1:]
    out = np.full(d.shape[0], np.inf)
    for i in range(d.shape[0]):
        pts = d[i][None, :] * ts[:, None]
        m = inside(pts)
        if m.any():
            out[i] = ts[np.argmax(m)]
    return out


def _seg_dist(x, a, b):
    ab = b - a
    s = np.clip(((x - a) @ ab) / (ab @ ab), 0, 1)
    return np.linalg.norm(x - (a + s[:, None] * ab), axis=1)


def test_capsule_and_ellipsoid_first_hit_by_marching():
    rng = np.random.default_rng(3)
    caps = synth._prim("capsule", (-0.6, 3.0, -0.2), (0.5, 3.6, 0.4), (0.35, 0, 0))
    ax = synth._orthonormal(rng)
    ell = synth._prim("ellipsoid", (0.3, 5.0, 0.1), ax[0] * 0.9, ax[1] * 0.4, ax[2] * 0.6)
    narrow = ((np.deg2rad(-25.0), np.deg2rad(25.0)), (np.deg2rad(-12.0), np.deg2rad(12.0)))
    _, _, d = rc.pixel_directions(24, 12, *narrow)
    step = 20.0 / 20000
    inside_c = lambda p: _seg_dist(p, caps["a"], caps["b"]) < 0.35
    E = np.stack([ell["b"], ell["c"], ell["d"]])
    w = E / (E * E).sum(axis=1, keepdims=True)
    inside_e = lambda p: (((p - ell["a"]) @ w.T) ** 2).sum(axis=1) < 1.0
    for prim, inside in ((caps, inside_c), (ell, inside_e)):
        t = rc.HITTERS[prim["kind"]](d, prim)
        tb = _first_crossing_by_marching(d, inside)
        both = np.isfinite(t) & np.isfinite(tb)
        assert both.sum() > 5
        # the marched first inside sample is at most one step past the surface
        assert np.all(tb[both] - t[both] >= -1e-9) and np.all(tb[both] - t[both] <= step + 1e-9)
        # rays the oracle says miss never enter the solid (up to grazing within a step)
        miss = ~np.isfinite(t)
        assert not np.any(np.isfinite(tb[miss]))
    # surface membership of the hits
    t = rc.hit_capsule(d, caps)
    hit = np.isfinite(t)
    np.testing.assert_allclose(_seg_dist(d[hit] * t[hit, None], caps["a"], caps["b"]), 0.35, rtol=1e-12)
    t = rc.hit_ellipsoid(d, ell)
    hit = np.isfinite(t)
    np.testing.assert_allclose(((((d[hit] * t[hit, None]) - ell["a"]) @ w.T) ** 2).sum(axis=1), 1.0, rtol=1e-12)


def test_normals_are_perpendicular_to_the_surface():
    rng = np.random.default_rng(5)
    ax = synth._orthonormal(rng)
    ell = synth._prim("ellipsoid", (0.0, 4.0, 0.0), ax[0] * 1.0, ax[1] * 0.5, ax[2] * 0.7)
    _, _, d = rc.pixel_directions(30, 15, *FOV)
    t = rc.hit_ellipsoid(d, ell)
    hit = np.isfinite(t)
    x = d[hit] * t[hit, None]
    n = rc.surface_normal(x, ell)
    # the implicit function f(x) = |s(x)|^2 - 1 changes at first order only along n
    f = lambda p: (((p - ell["a"]) @ (np.stack([ell["b"], ell["c"], ell["d"]]) /
                                      (np.stack([ell["b"], ell["c"], ell["d"]]) ** 2).sum(1, keepdims=True)).T) ** 2).sum(1) - 1
    tang = np.cross(n, rng.normal(size=3))
    tang /= np.linalg.norm(tang, axis=1, keepdims=True)
    h = 1e-6
    assert np.max(np.abs(f(x + h * tang) - f(x - h * tang))) < 1e-9
    assert np.all(f(x + h * n) > 0)  # outward


def _rodrigues(om, dt):
    th = np.linalg.norm(om) * dt
    if th == 0:
        return np.eye(3)
    k = om / np.linalg.norm(om)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K


@pytest.mark.parametrize("kind", ["plane", "capsule", "ellipsoid"])
def test_velocity_is_closing_speed_of_the_surface_point(kind):
    # The Doppler of a scatterer comes from the velocity of the material point it
    # reflects from: carry each hit point rigidly (pivot moved by vel dt, the offset
    # from the pivot rotated by omega dt) and difference its distance from the radar.
    rng = np.random.default_rng({"plane": 1, "capsule": 2, "ellipsoid": 3}[kind])
    ax = synth._orthonormal(rng)
    c = np.array([0.2, 4.0, 0.3])
    if kind == "plane":
        prim = synth._prim(kind, c - 1.5 * (ax[0] + ax[1]), 3 * ax[0], 3 * ax[1])
    elif kind == "capsule":
        prim = synth._prim(kind, c - 0.8 * ax[0], c + 0.8 * ax[0], (0.5, 0, 0))
    else:
        prim = synth._prim(kind, c, ax[0] * 1.0, ax[1] * 0.6, ax[2] * 0.8)
    prim["vel"] = np.array([0.7, -1.3, 0.4])
    prim["omega"] = np.array([0.9, -0.5, 1.7])
    o = rc.raycast([prim], 48, 24, *FOV)
    _, _, d = rc.pixel_directions(48, 24, *FOV)
    hit = np.isfinite(o["range"])
    assert hit.sum() > 20
    x = d[hit] * o["range"][hit, None]
    dt = 1e-5
    moved = lambda h: prim["a"] + prim["vel"] * h + (x - prim["a"]) @ _rodrigues(prim["omega"], h).T
    rate = (np.linalg.norm(moved(dt), axis=1) - np.linalg.norm(moved(-dt), axis=1)) / (2 * dt)
    np.testing.assert_allclose(o["vel"][hit], -rate, atol=1e-7)
    # a surface receding along every ray at speed s: closing speed -s d.v_hat
    prim2 = dict(prim, vel=np.array([0.0, 2.0, 0.0]), omega=np.zeros(3))
    o2 = rc.raycast([prim2], 48, 24, *FOV)
    np.testing.assert_allclose(o2["vel"][hit], -2.0 * d[hit, 1], rtol=1e-13)


def test_occlusion_and_ties():
    d = 3.0
    near = _sphere((0, d, 0), 0.5, rho=0.9)
    far = _sphere((0, 2 * d, 0), 1.5, rho=0.4)
    o = rc.raycast([far, near], 40, 20, *FOV)
    assert (o["prim"] == 1).sum() > 0
    # where both are hit the near sphere wins
    _, _, dd = rc.pixel_directions(40, 20, *FOV)
    tn, tf = rc.hit_ellipsoid(dd, near), rc.hit_ellipsoid(dd, far)
    both = np.isfinite(tn) & np.isfinite(tf)
    assert both.sum() > 0 and np.all(o["prim"][both] == 1)
    # two identical spheres: the first listed wins
    o2 = rc.raycast([near, dict(near, rho=0.1)], 40, 20, *FOV)
    hit = np.isfinite(o2["range"])
    assert np.all(o2["prim"][hit] == 0)


def test_misses_are_background():
    o = rc.raycast([_sphere((0, -5.0, 0), 1.0)], 16, 8, *FOV)  # behind the radar
    assert np.all(np.isinf(o["range"])) and np.all(o["sigma_re"] == 0) and np.all(o["vel"] == 0)
    assert np.all(o["prim"] == -1)


def test_hit_plane_parallelogram_by_hand():
    """Distances to parallelograms worked out by hand: an axis-aligned square in the plane
    y = 3 and a skewed parallelogram (b and c not orthogonal) in y = 4, hit at chosen
    (s, u) coordinates; points outside the edges, parallel rays and rays pointing away
    miss.  The skewed case fails if the 2x2 Gram solve swaps or transposes its terms."""
    sq = synth._prim("plane", (-1.0, 3.0, -1.0), (2.0, 0.0, 0.0), (0.0, 0.0, 2.0))
    sk = synth._prim("plane", (0.0, 4.0, 0.0), (1.0, 0.0, 0.0), (1.0, 0.0, 1.0))

    def unit(v):
        v = np.asarray(v, float)
        return v / np.linalg.norm(v)

    pts_sq = [(0.0, 3.0, 0.0), (0.5, 3.0, -0.7), (0.9, 3.0, 0.9)]
    d = np.stack([unit(p) for p in pts_sq])
    np.testing.assert_allclose(rc.hit_plane(d, sq), [np.linalg.norm(p) for p in pts_sq], rtol=1e-14)
    # skewed: a + s b + u c for (s, u) inside and outside the unit square
    a, b, c = np.array([0.0, 4.0, 0.0]), np.array([1.0, 0.0, 0.0]), np.array([1.0, 0.0, 1.0])
    inside = [a + 0.3 * b + 0.6 * c, a + 0.9 * b + 0.1 * c]
    outside = [a + 1.2 * b + 0.3 * c, a + 0.2 * b - 0.1 * c, a + 0.5 * b + 1.1 * c]
    d_in = np.stack([unit(p) for p in inside])
    np.testing.assert_allclose(rc.hit_plane(d_in, sk), [np.linalg.norm(p) for p in inside], rtol=1e-14)
    d_out = np.stack([unit(p) for p in outside])
    assert np.all(np.isinf(rc.hit_plane(d_out, sk)))
    # parallel to the plane, and pointing away from it
    d_miss = np.stack([unit((1.0, 0.0, 0.0)), unit((0.0, -1.0, 0.0)), unit((0.1, -3.0, 0.2))])
    assert np.all(np.isinf(rc.hit_plane(d_miss, sq)))


def test_raycast_angles_closed_form_and_grid_agreement():
    """A large plane y = 5 seen at arbitrary angles: range 5 / (cos el cos az) and the
    Lambert strength rho cos(incidence) / R^2 (rho cos(incidence) without fall-off), the
    incidence angle's cosine being the ray's y component; the angle form agrees exactly
    with the grid form at the grid's own angles."""
    wall = synth._prim("plane", (-50.0, 5.0, -50.0), (100.0, 0.0, 0.0), (0.0, 0.0, 100.0), rho=0.7)
    az = np.array([0.0, 0.3, -0.7, 1.1])
    el = np.array([0.0, -0.2, 0.4, 0.1])
    out = rc.raycast_angles([wall], az, el)
    cosi = np.cos(el) * np.cos(az)
    R = 5.0 / cosi
    np.testing.assert_allclose(out["range"], R, rtol=1e-13)
    np.testing.assert_allclose(out["sigma_re"], 0.7 * cosi / R ** 2, rtol=1e-12)
    flat = rc.raycast_angles([wall], az, el, falloff=False)
    np.testing.assert_allclose(flat["sigma_re"], 0.7 * cosi, rtol=1e-12)
    scene = synth.random_scene(3)
    grid = rc.raycast(scene, 17, 9, *synth.CAMERA_FOV)
    again = rc.raycast_angles(scene, grid["az"], grid["el"])
    for k in ("range", "sigma_re", "vel"):
        np.testing.assert_array_equal(grid[k], again[k])
