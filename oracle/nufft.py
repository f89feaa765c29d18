"""CPU FP64 reference of the NUFFT form of the cube (gridding, FFT, deconvolution).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this module.  It shares no code with the CUDA library.

For one virtual channel v the sum of Eq. 2 is a two-dimensional type-1 non-uniform
discrete Fourier transform: with the path terms of ``oracle.cube``,

    cube[v][n][l] = sum_p q_p exp(j 2 pi (x_p n + y_p l)),
    x_p = 2 mu R_{p,v} / (c F_s)      cycles per fast-time sample (Eq. 1),
    y_p = -f_D,p T_slow               cycles per block (Eq. 1),
    q_p = sigma_p exp(j 2 pi (v d_rx u_p / lam + TDM term))   (Eq. 2).

Centred mode indices n = n' + s_x, l = l' + s_y (s_x = N_s // 2, s_y = L // 2) move the
shift into the strengths, q'_p = q_p exp(j 2 pi (x_p s_x + y_p s_y)).  Gridding onto a
periodic grid of G_x >= 2 N_s by G_y >= 2 L cells (Dutt and Rokhlin 1993; Greengard and
Lee 2004), with the "exponential of semicircle" kernel of Barnett, Magland and
af Klinteberg (SIAM J. Sci. Comput. 41, 2019):

    phi(z) = exp(beta (sqrt(1 - z^2) - 1)) for |z| <= 1, else 0;  psi(t) = phi(2 t / w)
    grid[mx][my] = sum_p q'_p psi(mx - x_p G_x) psi(my - y_p G_y)      (indices mod G)
    S(n', l')    = sum_{mx, my} grid[mx][my] exp(+j 2 pi (mx n' / G_x + my l' / G_y))
    cube[v][n' + s_x][l' + s_y] = S(n', l') / (Psi_x(n') Psi_y(l')),
    Psi(k) = integral of psi(t) exp(j 2 pi k t / G) dt = (w/2) int_{-1}^{1} phi(z) cos(pi k w z / G) dz.

Each point touches the w cells of each axis whose centres lie within w/2 of it.  The
relative error is about 10^-(w-1) for an oversampling of 2 with beta = 2.30 w (Barnett
et al.); w is the kernel width in cells.
"""
from __future__ import annotations

import numpy as np

from .cube import _tdm, path_terms


def es_beta(w):
    """ES kernel shape parameter for kernel width w at an oversampling of 2."""
    return 2.30 * w


def es_kernel(z, beta):
    """phi(z) = exp(beta (sqrt(1 - z^2) - 1)) on |z| <= 1, zero outside."""
    z = np.asarray(z, dtype=np.float64)
    out = np.zeros_like(z)
    m = np.abs(z) <= 1.0
    out[m] = np.exp(beta * (np.sqrt(1.0 - z[m] ** 2) - 1.0))
    return out


def es_transform(k, w, G, n_nodes=128):
    """Psi(k) = (w/2) int_{-1}^{1} phi(z) cos(pi k w z / G) dz by Gauss-Legendre quadrature."""
    z, wt = np.polynomial.legendre.leggauss(n_nodes)
    k = np.asarray(k, dtype=np.float64)
    phi = es_kernel(z, es_beta(w))
    return (w / 2.0) * (np.cos(np.pi * np.outer(k, z) * w / G) * (phi * wt)[None, :]).sum(axis=1)


def grid_size(N):
    """Smallest power of two >= 2 N (oversampling at least 2) and >= 16 cells."""
    g = 16
    while g < 2 * N:
        g *= 2
    return g


def _taps(X, w):
    """The w cells m0 .. m0 + w - 1 whose centres lie within w/2 of positions X (cells),
    and psi(m - X) there."""
    m0 = np.floor(X - w / 2.0).astype(np.int64) + 1
    m = m0[:, None] + np.arange(w)[None, :]
    return m, es_kernel(2.0 * (m - X[:, None]) / w, es_beta(w))


def nufft2_type1(x, y, q, Ns, L, w):
    """sum_p q_p exp(j 2 pi (x_p n + y_p l)) for n < Ns, l < L by gridding + FFT."""
    x = np.mod(np.asarray(x, np.float64), 1.0)
    y = np.mod(np.asarray(y, np.float64), 1.0)
    q = np.asarray(q, np.complex128)
    Gx, Gy = grid_size(Ns), grid_size(L)
    sx, sy = Ns // 2, L // 2
    qs = q * np.exp(2j * np.pi * (x * sx + y * sy))
    mx, wx = _taps(x * Gx, w)
    my, wy = _taps(y * Gy, w)
    grid = np.zeros((Gx, Gy), dtype=np.complex128)
    vals = qs[:, None, None] * wx[:, :, None] * wy[:, None, :]
    np.add.at(grid, (np.mod(mx, Gx)[:, :, None], np.mod(my, Gy)[:, None, :]), vals)
    S = np.fft.ifft2(grid) * (Gx * Gy)  # exp(+j ...) without the 1/N
    n1 = np.arange(Ns) - sx
    l1 = np.arange(L) - sy
    sub = S[np.mod(n1, Gx)][:, np.mod(l1, Gy)]
    return sub / (es_transform(n1, w, Gx)[:, None] * es_transform(l1, w, Gy)[None, :])


def cube_nufft(radar, px, w=7, channels=None):
    """The cube of Eq. 2 through the type-1 NUFFT of each channel."""
    t = path_terms(radar, px)
    p = t["params"]
    V, Ns, L = p["M"] * p["N"], p["Ns"], p["L"]
    chans = list(range(V)) if channels is None else list(channels)
    out = np.zeros((len(chans), Ns, L), dtype=np.complex128)
    y = -t["fD"] * p["t_slow"]
    for i, v in enumerate(chans):
        if t["idx"].size == 0:
            continue
        x = 2.0 * p["mu"] * t["R_pv"][v] / (p["c"] * p["fs"])
        q = t["sigma"] * np.exp(2j * np.pi * (v * p["d_rx"] * t["u"] / p["lam"] + _tdm(p, t, v)))
        out[i] = nufft2_type1(x, y, q, Ns, L, w)
    return out


__all__ = ["es_beta", "es_kernel", "es_transform", "grid_size", "nufft2_type1", "cube_nufft"]
