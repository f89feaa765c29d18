"""CPU FP64 oracle of the TDM-MIMO beat-signal data cube (Eq. 1 and Eq. 2).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this module.  It shares no code, table or helper with
the CUDA library and imports nothing from it; it takes plain numpy arrays.

What it computes (0-based n, l, m, r; v = m N + r is the virtual channel index):

    valid_p    = sigma_p != 0                                    (background miss)
    u_p        = cos(el_p) sin(az_p)                              direction cosine
    R_{p,v}    = R_p + v * d_rx * u_p / 2                         path range, Eq. 1
    f_D,p      = 2 vel_p / lam                                    Doppler, Eq. 1 / Eq. 2
    phi        = 2 mu R_{p,v} / c * n / F_s                       fast time, Eq. 1
               + v * d_rx * u_p / lam                             spatial, Eq. 2
               - f_D,p * l * T_slow                               slow time, Eq. 1
    cube[v, n, l] = sum over valid p (ascending) of sigma_p exp(j 2 pi phi)

Readings of the paper that this code takes (where it is silent or garbled):
  * the sum over m in Eq. 1/2 is kept apart: v = m N + r indexes M N virtual
    channels, with Tx spacing N d_rx and Rx spacing d_rx = lam / 2 (Eq. 2 defs);
  * the slow-time step is T_slow, one TDM block of M chirps (default M T_b); Eq. 2's
    "(l - 1) / L" factor is read as a typo of Eq. 1's "(l - 1)";
  * f_l in Eq. 2 is the carrier, so 2 f_l V / c = 2 V / lam = f_D;
  * the single AoA of Eq. 2 becomes the direction cosine cos(el) sin(az) along the
    horizontal array;
  * the per-pixel strength is a complex amplitude, constant over m, n, l;
  * the range term uses the per-channel path range R_{p,v} of Eq. 1 and the
    spatial term is the carrier phase of the excess path 2 (R_{p,v} - R_p) / lam;
  * the cube is stored [V][N_s][L];
  * optional TDM motion term (off by default, Eq. 1 has none): Tx m transmits in slot m
    of each block, so phi gains -f_D,p * m * T_b with m = v // N.

Two forms of the same sum:
  * ``cube_literal`` evaluates every term with its own cos/sin (the sum as written);
  * ``cube_separable`` factors the phase into a fast-time phasor per (p, v, n) and a
    slow-time phasor per (p, l) and contracts over p with a library complex matmul.
"""
from __future__ import annotations

import math

import numpy as np


def _params(radar):
    """Resolve defaults: d_rx = lam / 2 (Eq. 2 defs), T_slow = M T_b (Eq. 1 defs)."""
    lam = float(radar.lam)
    d_rx = float(radar.d_rx) if radar.d_rx > 0 else lam / 2.0
    t_slow = float(radar.t_slow) if radar.t_slow > 0 else radar.M * float(radar.t_b)
    return dict(M=int(radar.M), N=int(radar.N), Ns=int(radar.Ns), L=int(radar.L), lam=lam,
                d_rx=d_rx, mu=float(radar.mu), fs=float(radar.fs), t_slow=t_slow,
                c=float(radar.c), t_b=float(radar.t_b),
                tdm=bool(getattr(radar, "tdm_motion", False)))


def valid_mask(sigma_re, sigma_im):
    """Pixels that hit something: non-zero complex strength (+0 and -0 both miss)."""
    sre = np.asarray(sigma_re, dtype=np.float64)
    sim = np.asarray(sigma_im, dtype=np.float64)
    return (sre != 0.0) | (sim != 0.0)


def valid_indices(sigma_re, sigma_im):
    """Ascending indices of the valid pixels (the order the sum runs in)."""
    return np.flatnonzero(valid_mask(sigma_re, sigma_im)).astype(np.int64)


def path_terms(radar, px):
    """Per valid pixel and channel: the FP64 quantities that the phase is made of.

    Returns a dict with the valid indices ``idx``, the complex strengths ``sigma``,
    ``u`` (direction cosine), ``R_pv`` [V, Pv], ``fD`` [Pv] and the resolved params.
    """
    p = _params(radar)
    idx = valid_indices(px.sigma_re, px.sigma_im)
    f64 = lambda a: np.asarray(a, dtype=np.float64)[idx]
    R, az, el, vel = f64(px.range), f64(px.az), f64(px.el), f64(px.vel)
    sigma = f64(px.sigma_re) + 1j * f64(px.sigma_im)
    V = p["M"] * p["N"]
    k = np.arange(V, dtype=np.float64)[:, None]
    u = np.cos(el) * np.sin(az)
    R_pv = R[None, :] + 0.5 * k * p["d_rx"] * u[None, :]
    fD = 2.0 * vel / p["lam"]
    return dict(idx=idx, sigma=sigma, u=u, R_pv=R_pv, fD=fD, k=k, params=p)


def phase_cycles(radar, px, v, n, l):
    """phi(p, v, n, l) in cycles for every valid pixel (a vector over p)."""
    t = path_terms(radar, px)
    p = t["params"]
    fast = 2.0 * p["mu"] * t["R_pv"][v] / p["c"] * n / p["fs"]
    spatial = v * p["d_rx"] * t["u"] / p["lam"] + _tdm(p, t, v)
    slow = -t["fD"] * l * p["t_slow"]
    return fast + spatial + slow


def _tdm(p, t, v):
    """TDM motion phase of channel v (cycles): -f_D * m * T_b for Tx slot m = v // N."""
    if not p["tdm"]:
        return 0.0
    return -t["fD"] * (v // p["N"]) * p["t_b"]


def _pairwise_sum(x):
    """Pairwise (cascade) summation along axis 0, in FP64."""
    x = np.asarray(x)
    while x.shape[0] > 1:
        if x.shape[0] % 2:
            x = np.concatenate([x, np.zeros_like(x[:1])], axis=0)
        x = x[0::2] + x[1::2]
    return x[0] if x.shape[0] else np.zeros(x.shape[1:], dtype=x.dtype)


def cube_literal(radar, px):
    """The sum of Eq. 2 term by term: one cos/sin per (p, v, n, l).

    Each phase is reduced to (-1/2, 1/2] cycles before the trigonometric call and
    the terms are added over p by pairwise summation.  Cost: P V N_s L cos/sin, so
    it is for small frames only.
    """
    t = path_terms(radar, px)
    p = t["params"]
    V, Ns, L = p["M"] * p["N"], p["Ns"], p["L"]
    n = np.arange(Ns, dtype=np.float64)
    l = np.arange(L, dtype=np.float64)
    Pv = t["idx"].size
    out = np.zeros((V, Ns, L), dtype=np.complex128)
    if Pv == 0:
        return out
    chunk = max(1, (1 << 22) // (Ns * L))
    for v in range(V):
        parts = []
        for s in range(0, Pv, chunk):
            sl = slice(s, min(Pv, s + chunk))
            # phi[p, n, l] for this channel and this slice of pixels
            fast = (2.0 * p["mu"] * t["R_pv"][v, sl] / p["c"] / p["fs"])[:, None, None] * n[None, :, None]
            spatial = (v * p["d_rx"] * t["u"][sl] / p["lam"]
                       + (_tdm(p, t, v)[sl] if p["tdm"] else 0.0))[:, None, None]
            slow = -(t["fD"][sl] * p["t_slow"])[:, None, None] * l[None, None, :]
            phi = fast + spatial + slow
            phi = phi - np.round(phi)
            ang = 2.0 * np.pi * phi
            terms = t["sigma"][sl, None, None] * (np.cos(ang) + 1j * np.sin(ang))
            parts.append(_pairwise_sum(terms))
        out[v] = _pairwise_sum(np.stack(parts))
    return out


def cube_separable(radar, px, channels=None):
    """The same sum with the phase split into a fast-time and a slow-time phasor.

    phi = [2 mu R_{p,v} n / (c F_s) + v d_rx u_p / lam] + [-f_D,p l T_slow], so
    cube[v] = F_v^T diag(sigma) D with F_v[p, n] and D[p, l] FP64 phasors; the
    contraction over p is a complex128 matmul.  ``channels`` restricts the output
    to a subset of v (rows of the returned array follow that subset).
    """
    t = path_terms(radar, px)
    p = t["params"]
    V, Ns, L = p["M"] * p["N"], p["Ns"], p["L"]
    chans = list(range(V)) if channels is None else list(channels)
    n = np.arange(Ns, dtype=np.float64)
    l = np.arange(L, dtype=np.float64)
    out = np.zeros((len(chans), Ns, L), dtype=np.complex128)
    if t["idx"].size == 0:
        return out
    slow = -(t["fD"] * p["t_slow"])[:, None] * l[None, :]
    slow = slow - np.round(slow)
    D = t["sigma"][:, None] * np.exp(2j * np.pi * slow)  # [Pv, L]
    for i, v in enumerate(chans):
        fast = (2.0 * p["mu"] * t["R_pv"][v] / p["c"] / p["fs"])[:, None] * n[None, :]
        fast = fast + (v * p["d_rx"] * t["u"] / p["lam"] + _tdm(p, t, v))[:, None]
        fast = fast - np.round(fast)
        F = np.exp(2j * np.pi * fast)  # [Pv, Ns]
        out[i] = F.T @ D
    return out


def cube_entries(radar, px, entries):
    """Selected cube entries, each as its own FP64 sum over p.

    ``entries`` is an int array [K, 3] of (v, n, l).  Used to check a full-size
    result at sampled positions without forming the whole cube.
    """
    t = path_terms(radar, px)
    p = t["params"]
    ent = np.asarray(entries, dtype=np.int64).reshape(-1, 3)
    out = np.zeros(ent.shape[0], dtype=np.complex128)
    if t["idx"].size == 0:
        return out
    for i, (v, n, l) in enumerate(ent):
        phi = (2.0 * p["mu"] * t["R_pv"][v] / p["c"] * n / p["fs"]
               + v * p["d_rx"] * t["u"] / p["lam"] + _tdm(p, t, v)
               - t["fD"] * l * p["t_slow"])
        phi = phi - np.round(phi)
        term = t["sigma"] * (np.cos(2 * np.pi * phi) + 1j * np.sin(2 * np.pi * phi))
        out[i] = math.fsum(term.real) + 1j * math.fsum(term.imag)
    return out


def rel_l2(x, ref):
    """Normwise relative L2 error ||x - ref|| / ||ref|| over all entries (complex as 2 reals)."""
    x = np.asarray(x, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    den = np.linalg.norm(ref.ravel())
    num = np.linalg.norm((x - ref).ravel())
    return float(num / den) if den > 0 else float(num)
