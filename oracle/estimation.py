"""CPU FP64 oracle of target estimation on a cube (Section III).

TEST INFRASTRUCTURE ONLY (see ``oracle/cube.py``).  Section III forms the
range-Doppler map of each CPI's cube by FFT and takes, CPI after CPI, the velocity of
maximum power (the Doppler-time plot); the mean absolute difference to the true
velocity is E_velo.  Readings: channels are added non-coherently (sum of |FFT|^2); a
forward FFT over slow time puts a pixel of Doppler f_D at bin (-f_D T_slow L) mod L, so
signed bin d_s maps to v = -d_s lambda / (2 T_slow L); the optional static-clutter notch
leaves the zero-Doppler column out of the search.
"""
from __future__ import annotations

import numpy as np

from .cube import _params


def range_doppler_power(cube):
    """power[k][d] = sum_v |FFT_n FFT_l cube[v]|^2 (library FFT, FP64)."""
    x = np.fft.fft2(np.asarray(cube, dtype=np.complex128), axes=(1, 2))
    return (x.real ** 2 + x.imag ** 2).sum(axis=0)


def max_power_velocity(radar, power, skip_static=False):
    """(velocity, (k, d)) of the largest power (first flat index on ties)."""
    p = _params(radar)
    pw = np.array(power, dtype=np.float64, copy=True)
    if skip_static:
        pw[:, 0] = -1.0
    i = int(np.argmax(pw))
    k, d = divmod(i, pw.shape[1])
    L = pw.shape[1]
    ds = d if d < L // 2 else d - L
    v = -ds * p["lam"] / (2.0 * p["t_slow"] * L)
    return v, (k, d)


def e_velo(v_est, v_true):
    """Mean absolute velocity error over CPIs."""
    v_est = np.asarray(v_est, dtype=np.float64)
    v_true = np.asarray(v_true, dtype=np.float64)
    return float(np.mean(np.abs(v_est - v_true)))
