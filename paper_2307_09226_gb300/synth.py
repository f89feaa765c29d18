"""Seeded synthetic per-pixel render buffers for the TDM-MIMO cube synthesis.

The paper's frames come from Blender's Cycles renderer (Section II): every pixel of an
N_az x N_el image carries a range, a strength, an angle of arrival and a velocity
(the symbol list after Eq. 2).  That renderer and the authors' scene are not
available, so this module draws buffers with the same structure from numpy's
``default_rng(seed)``.  It holds none of the method's arithmetic (no phases, no
sums): it only produces radar parameters and pixel arrays, and it is the one module
that both the CUDA path and the CPU oracle are fed from.

Conventions
-----------
* Pixel p = j * N_az + i for elevation row j and azimuth column i (the render
  buffers are indexed [el, az] after Eq. 2).
* Pixel grid is cell-centred: az_i = -60 deg + (i + 1/2) 120 deg / N_az,
  el_j = -30 deg + (j + 1/2) 60 deg / N_el (the camera angle range stands for the
  antenna pattern, Section II).
* sigma is a complex amplitude.  A pixel with sigma == 0 is a background miss and
  its range is +inf.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field, replace
from functools import lru_cache
from typing import Dict, List

import numpy as np

C_LIGHT = 299_792_458.0
CONFIG_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs")


@lru_cache(maxsize=None)
def _config_text(n: int) -> str:
    with open(os.path.join(CONFIG_DIR, f"config{n}.json")) as f:
        return f.read()


def load_config(n: int) -> Dict:
    """The parameters of workload n (1..5) from configs/config<n>.json: radar, pixel grid,
    value distributions, mask fraction, seeds and (config 5) the serving mix."""
    return json.loads(_config_text(n))


@dataclass(frozen=True)
class Radar:
    """FMCW TDM-MIMO radar parameters (symbols of Eq. 1)."""

    M: int  # Tx antennas
    N: int  # Rx antennas
    Ns: int  # fast-time samples per chirp
    L: int  # TDM blocks (slow time)
    lam: float = 3.9e-3  # wavelength [m]
    d_rx: float = 0.0  # Rx spacing [m]; <= 0 means lam / 2
    mu: float = 30e6 / 1e-6  # chirp slope [Hz/s]
    fs: float = 10e6  # ADC sampling rate [Hz]
    t_b: float = 60e-6  # chirp duration [s]
    t_slow: float = 0.0  # TDM block period [s]; <= 0 means M * t_b
    c: float = C_LIGHT
    tdm_motion: bool = False  # add the Doppler phase of the Tx slot within a block
    nufft_width: int = 0  # NUFFT tier: gridding kernel width 4..8 (0: the default, 7)

    @property
    def V(self) -> int:
        return self.M * self.N

    def resolved(self) -> "Radar":
        """Return a copy with the defaulted fields filled in."""
        d = self.d_rx if self.d_rx > 0 else self.lam / 2.0
        t = self.t_slow if self.t_slow > 0 else self.M * self.t_b
        return replace(self, d_rx=d, t_slow=t)


@dataclass
class Pixels:
    """Structure-of-arrays render buffers of one frame (flattened [el, az])."""

    range: np.ndarray
    sigma_re: np.ndarray
    sigma_im: np.ndarray
    az: np.ndarray
    el: np.ndarray
    vel: np.ndarray

    @property
    def P(self) -> int:
        return int(self.range.shape[0])

    @property
    def dtype(self):
        return self.range.dtype

    def astype(self, dt) -> "Pixels":
        return Pixels(*(np.ascontiguousarray(a, dtype=dt) for a in self.arrays()))

    def arrays(self) -> List[np.ndarray]:
        return [self.range, self.sigma_re, self.sigma_im, self.az, self.el, self.vel]

    def subset(self, idx) -> "Pixels":
        return Pixels(*(np.ascontiguousarray(a[idx]) for a in self.arrays()))


@dataclass
class Frame:
    radar: Radar
    pixels: Pixels
    out_dtype: str = "complex64"  # "complex64" | "complex128"
    meta: Dict = field(default_factory=dict)


def grid_angles(n_az: int, n_el: int):
    """Cell-centred az/el grid in radians, flattened with p = j * n_az + i."""
    az1 = np.deg2rad(-60.0 + (np.arange(n_az) + 0.5) * 120.0 / n_az)
    el1 = np.deg2rad(-30.0 + (np.arange(n_el) + 0.5) * 60.0 / n_el)
    az = np.tile(az1, n_el)
    el = np.repeat(el1, n_az)
    return az, el


def _strength(rng, n, mean=0.0, sd=1.0):
    mag = np.exp(rng.normal(mean, sd, n))
    ph = rng.uniform(0.0, 2.0 * np.pi, n)
    return mag * np.cos(ph), mag * np.sin(ph)


def random_frame(radar: Radar, n_az: int, n_el: int, seed: int, mask_frac: float = 0.0,
                 dtype=np.float32, r_lo=0.5, r_hi=8.0, v_max=2.0) -> Pixels:
    """Uniform-range random scene on the az/el grid.

    R ~ U(r_lo, r_hi) m, |sigma| = exp(N(0, 1)) with uniform phase, v ~ U(-v_max, v_max)
    m/s.  A Bernoulli(mask_frac) subset is a background miss: sigma = 0, R = +inf.
    """
    rng = np.random.default_rng(seed)
    P = n_az * n_el
    az, el = grid_angles(n_az, n_el)
    rr = rng.uniform(r_lo, r_hi, P)
    sre, sim = _strength(rng, P)
    vel = rng.uniform(-v_max, v_max, P)
    if mask_frac > 0.0:
        miss = rng.random(P) < mask_frac
        sre[miss] = 0.0
        sim[miss] = 0.0
        rr[miss] = np.inf
    px = Pixels(rr, sre, sim, az, el, vel)
    return px.astype(dtype)


# ----------------------------------------------------------------------------------
# The workloads.  Sizes and distributions follow the five synthetic configurations
# that stand in for the paper's Blender scene (Section III).
# ----------------------------------------------------------------------------------

def _frame_from_config(n: int, seed=None) -> Frame:
    c = load_config(n)
    radar = Radar(**c["radar"])
    p = c["pixels"]
    assert p["log_abs_sigma"] == [0.0, 1.0] and c["grid"]["az_deg"] == [-60, 60] and c["grid"]["el_deg"] == [-30, 30]
    px = random_frame(radar, c["grid"]["n_az"], c["grid"]["n_el"], c["seed"] if seed is None else seed,
                      mask_frac=p["mask_frac"], dtype=np.dtype(c["pixel_dtype"]).type, r_lo=p["range_m"][0],
                      r_hi=p["range_m"][1], v_max=p["vel_max_m_s"])
    return Frame(radar, px, c["out_dtype"], {"workload": c["workload"]})


def config1(seed: int = None) -> Frame:
    """One small frame (configs/config1.json): M=2, N=4, Ns=64, L=32, 32x32 pixels, FP64
    buffers, complex128 out."""
    return _frame_from_config(1, seed)


def config2(seed: int = None) -> Frame:
    """One frame (configs/config2.json): M=3, N=4, Ns=256, L=128, 256x256 pixels, 30%
    background, complex64 out."""
    return _frame_from_config(2, seed)


def parity_frame(seed: int = 11, M=2, N=3, Ns=96, L=48, n_az=71, n_el=70,
                 mask_frac=0.3, dtype=np.float32) -> Frame:
    """A mid-size frame whose dimensions are not multiples of any tile (ragged tails)."""
    radar = Radar(M=M, N=N, Ns=Ns, L=L)
    px = random_frame(radar, n_az, n_el, seed, mask_frac=mask_frac, dtype=dtype)
    return Frame(radar, px, "complex64", {"workload": f"parity-{n_az}x{n_el}-V{M*N}-Ns{Ns}-L{L}"})


def walking_batch(n_frames: int = None, seed: int = None, n_az: int = None, n_el: int = None,
                  dtype=None) -> List[Frame]:
    """Animation of a walking-pedestrian-like scene in front of a static wall
    (configs/config4.json; the arguments override its frame count, seed, grid and dtype).

    Per frame f: a pedestrian cluster of n_f ~ U{2000..20000} pixels in a contiguous
    az/el window whose centre moves as 40 deg * sin(2 pi f / 64); its range is
    R_f + U(-0.3, 0.3) with R_f = 3 + 2 sin(2 pi f / 64 + 0.7) m and its velocity a
    torso term 1.5 sin(2 pi f / 64) plus a limb term U(-1.5, 1.5), clipped to +-3 m/s.
    A wall of w_f ~ U{0..45000} pixels sits at R = min(6 / (cos az cos el), 8) m with
    v = 0 and |sigma| = exp(N(-1, 0.5)).  Everything else is a background miss.
    """
    c = load_config(4)
    n_frames = c["frames"] if n_frames is None else n_frames
    seed = c["seed"] if seed is None else seed
    n_az = c["grid"]["n_az"] if n_az is None else n_az
    n_el = c["grid"]["n_el"] if n_el is None else n_el
    dtype = np.dtype(c["pixel_dtype"]).type if dtype is None else dtype
    ped_c, wall_c = c["pedestrian"], c["wall"]
    rng = np.random.default_rng(seed)
    radar = Radar(**c["radar"])
    P = n_az * n_el
    az, el = grid_angles(n_az, n_el)
    frames = []
    for f in range(n_frames):
        rr = np.full(P, np.inf)
        sre = np.zeros(P)
        sim = np.zeros(P)
        vel = np.zeros(P)
        # wall: a random set of grid cells not covered by the pedestrian
        n_ped = int(rng.integers(ped_c["pixels"][0], ped_c["pixels"][1] + 1))
        n_wall = int(rng.integers(wall_c["pixels"][0], wall_c["pixels"][1] + 1))
        ph = 2.0 * np.pi * f / 64.0
        az_c = np.deg2rad(ped_c["az_swing_deg"] * np.sin(ph))
        i_c = int(np.clip(np.round((np.rad2deg(az_c) + 60.0) / 120.0 * n_az - 0.5), 0, n_az - 1))
        # pedestrian window: tall (el) and narrow (az), height:width about 2.5:1
        w = max(1, int(np.round(np.sqrt(n_ped / ped_c["aspect_el_over_az"]))))
        h = int(np.ceil(n_ped / w))
        h = min(h, n_el)
        w = min(int(np.ceil(n_ped / h)), n_az)
        i0 = int(np.clip(i_c - w // 2, 0, n_az - w))
        j0 = int(np.clip(n_el // 2 - h // 2, 0, n_el - h))
        jj, ii = np.meshgrid(np.arange(j0, j0 + h), np.arange(i0, i0 + w), indexing="ij")
        ped = (jj * n_az + ii).ravel()[:n_ped]
        r_f = ped_c["range_centre_m"] + ped_c["range_swing_m"] * np.sin(ph + ped_c["range_phase"])
        jit, vt, vl, vc = ped_c["range_jitter_m"], ped_c["torso_m_s"], ped_c["limb_m_s"], ped_c["vel_clip_m_s"]
        rr[ped] = r_f + rng.uniform(-jit, jit, ped.size)
        vel[ped] = np.clip(vt * np.sin(ph) + rng.uniform(-vl, vl, ped.size), -vc, vc)
        a, b = _strength(rng, ped.size)
        sre[ped], sim[ped] = a, b
        free = np.setdiff1d(np.arange(P), ped, assume_unique=True)
        wall = np.sort(rng.choice(free, size=min(n_wall, free.size), replace=False))
        rr[wall] = np.minimum(wall_c["range_m"] / (np.cos(az[wall]) * np.cos(el[wall])), wall_c["range_cap_m"])
        a, b = _strength(rng, wall.size, mean=wall_c["log_abs_sigma"][0], sd=wall_c["log_abs_sigma"][1])
        sre[wall], sim[wall] = a, b
        px = Pixels(rr, sre, sim, az.copy(), el.copy(), vel).astype(dtype)
        frames.append(Frame(radar, px, "complex64",
                            {"workload": "walking-256x256-V12-Ns256-L128", "frame": f,
                             "v_torso": vt * np.sin(ph), "n_ped": int(ped.size),
                             "n_wall": int(wall.size)}))
    return frames


SERVE_CHOICES = {k: tuple(v) for k, v in load_config(5)["choices"].items()}


def serving_requests(n: int, seed: int = 5, grids=None, tiers=None) -> List[Dict]:
    """Request mix for the serving loop (configs/config5.json): uniform choices of radar
    and image size.

    Each request is a dict with a Radar, a grid edge and an accuracy tier; the pixel
    buffers are drawn lazily by ``request_frame`` (seed derived from the request id).
    """
    rng = np.random.default_rng(seed)
    grids = grids or SERVE_CHOICES["grid"]
    tiers = tiers or SERVE_CHOICES["tier"]
    out = []
    for k in range(n):
        radar = Radar(M=int(rng.choice(SERVE_CHOICES["M"])), N=int(rng.choice(SERVE_CHOICES["N"])),
                      Ns=int(rng.choice(SERVE_CHOICES["Ns"])), L=int(rng.choice(SERVE_CHOICES["L"])),
                      **load_config(5)["radar"])
        g = int(rng.choice(grids))
        t = str(rng.choice(tiers))
        out.append({"id": k, "radar": radar, "grid": g, "tier": t, "seed": seed * 1_000_003 + k})
    return out


def request_frame(req: Dict, dtype=np.float32) -> Frame:
    p = load_config(5)["pixels"]
    px = random_frame(req["radar"], req["grid"], req["grid"], req["seed"], mask_frac=p["mask_frac"], dtype=dtype,
                      r_lo=p["range_m"][0], r_hi=p["range_m"][1], v_max=p["vel_max_m_s"])
    return Frame(req["radar"], px, "complex64", {"workload": "serve", "id": req["id"]})


def point_scatterer(radar: Radar, R: float, sigma: complex, az: float, el: float, vel: float,
                    dtype=np.float64) -> Pixels:
    """A single-pixel frame holding one point target."""
    a = lambda x: np.array([x], dtype=dtype)
    return Pixels(a(R), a(sigma.real), a(sigma.imag), a(az), a(el), a(vel))


# ----------------------------------------------------------------------------------
# Analytic scenes for the ray-caster (the rendering step of Section II).  A scene is a
# list of primitive dicts: kind ("plane" | "capsule" | "ellipsoid"), vectors a, b, c,
# d (metres), vel (m/s, of the pivot a), omega (rad/s, about a) and rho.  Radar at the
# origin, x the array axis, y boresight, z up.
# ----------------------------------------------------------------------------------

PRIM_KINDS = ("plane", "capsule", "ellipsoid")
CAMERA_FOV = ((np.deg2rad(-60.0), np.deg2rad(60.0)), (np.deg2rad(-30.0), np.deg2rad(30.0)))


def _prim(kind, a, b=(0, 0, 0), c=(0, 0, 0), d=(0, 0, 0), vel=(0, 0, 0), omega=(0, 0, 0), rho=1.0):
    f = lambda x: np.asarray(x, dtype=np.float64)
    return {"kind": kind, "a": f(a), "b": f(b), "c": f(c), "d": f(d), "vel": f(vel), "omega": f(omega),
            "rho": float(rho)}


def _orthonormal(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return q.T  # rows: three orthonormal vectors


def random_scene(seed: int = 7, n_prims: int = 12):
    """Random primitives in front of the radar: ellipsoids with random orientation and
    semi-axes U(0.2, 0.8) m, capsules of radius U(0.05, 0.3) m and length U(0.3, 1.5) m,
    and parallelograms with edges U(0.5, 3) m; centres at range U(1.5, 8) m within
    +-50 deg azimuth and +-25 deg elevation; velocities U(-2, 2) m/s per axis, angular
    velocities U(-3, 3) rad/s per axis, rho U(0.2, 1)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_prims):
        kind = PRIM_KINDS[k % 3]
        rr = rng.uniform(1.5, 8.0)
        az = np.deg2rad(rng.uniform(-50, 50))
        el = np.deg2rad(rng.uniform(-25, 25))
        centre = rr * np.array([np.cos(el) * np.sin(az), np.cos(el) * np.cos(az), np.sin(el)])
        vel = rng.uniform(-2, 2, 3)
        om = rng.uniform(-3, 3, 3)
        rho = rng.uniform(0.2, 1.0)
        ax = _orthonormal(rng)
        if kind == "ellipsoid":
            s = rng.uniform(0.2, 0.8, 3)
            out.append(_prim(kind, centre, ax[0] * s[0], ax[1] * s[1], ax[2] * s[2], vel, om, rho))
        elif kind == "capsule":
            half = 0.5 * rng.uniform(0.3, 1.5)
            out.append(_prim(kind, centre - half * ax[0], centre + half * ax[0], (rng.uniform(0.05, 0.3), 0, 0),
                             (0, 0, 0), vel, om, rho))
        else:
            e1, e2 = ax[0] * rng.uniform(0.5, 3.0), ax[1] * rng.uniform(0.5, 3.0)
            out.append(_prim(kind, centre - 0.5 * (e1 + e2), e1, e2, (0, 0, 0), vel, om, rho))
    return out


def walking_scene(frame: int, n_frames: int = 100, fps: float = 24.0, radius: float = 3.0):
    """A pedestrian walking a circle of `radius` m around a point 4 m in front of the
    radar (one lap in n_frames frames at fps, the walking experiment of Section III),
    in a room with a back wall at y = 8 m and a floor 1 m below the radar.

    Body (capsules and one sphere, heights relative to the floor): torso from the hips
    (0.95 m) to the neck (1.45 m), radius 0.16 m; head sphere of radius 0.11 m at
    1.62 m; legs from the hips to the feet, arms from the shoulders (1.4 m) to the
    hands, radius 0.06 m, swinging +-25 deg (legs) and +-20 deg (arms) at the step
    rate of 2 steps per metre.  Returns (scene, ground truth) where ground truth holds
    the torso position, its velocity vector and its closing speed towards the radar.
    """
    t = frame / fps
    w = 2.0 * np.pi / (n_frames / fps)           # angular rate of the walk
    speed = w * radius
    cx, cy, floor = 0.0, 4.0, -1.0
    ang = w * t
    pos = np.array([cx + radius * np.cos(ang), cy + radius * np.sin(ang), floor])
    fwd = np.array([-np.sin(ang), np.cos(ang), 0.0])
    side = np.array([np.cos(ang), np.sin(ang), 0.0])
    up = np.array([0.0, 0.0, 1.0])
    v = speed * fwd
    om_body = np.array([0.0, 0.0, w])            # the body turns with the path
    step_w = 2.0 * np.pi * speed                 # one stride (two steps) per metre
    scene = [
        _prim("plane", (-6.0, 8.0, floor), (12.0, 0.0, 0.0), (0.0, 0.0, 3.0), rho=0.3),
        _prim("plane", (-6.0, 0.5, floor), (12.0, 0.0, 0.0), (0.0, 7.5, 0.0), rho=0.2),
    ]
    hip = pos + 0.95 * up
    neck = pos + 1.45 * up
    scene.append(_prim("capsule", hip, neck, (0.16, 0, 0), vel=v, omega=om_body, rho=1.0))
    head = pos + 1.62 * up
    scene.append(_prim("ellipsoid", head, (0.11, 0, 0), (0, 0.11, 0), (0, 0, 0.11), vel=v, omega=om_body,
                       rho=0.8))
    for sgn, lim, amp, length, pivot_h, ph in ((1, "leg", 25.0, 0.9, 0.95, 0.0), (-1, "leg", 25.0, 0.9, 0.95, np.pi),
                                               (1, "arm", 20.0, 0.6, 1.40, np.pi), (-1, "arm", 20.0, 0.6, 1.40, 0.0)):
        pivot = pos + pivot_h * up + sgn * (0.1 if lim == "leg" else 0.22) * side
        th = np.deg2rad(amp) * np.sin(step_w * t + ph)
        thd = np.deg2rad(amp) * step_w * np.cos(step_w * t + ph)
        end = pivot + length * (-np.cos(th) * up + np.sin(th) * fwd)
        # the limb swings about the side axis on top of the body's turn; its pivot moves
        # with the body: v_pivot = v + om_body x (pivot - pos)
        v_piv = v + np.cross(om_body, pivot - pos)
        om = om_body - thd * side
        scene.append(_prim("capsule", pivot, end, (0.06, 0, 0), vel=v_piv, omega=om, rho=0.7))
    centre = pos + 1.2 * up
    los = centre / np.linalg.norm(centre)
    truth = {"torso": centre, "vel_vec": v, "closing_speed": float(-(v @ los)), "speed": speed}
    return scene, truth
