"""Pins of the NUFFT reference (CPU, no GPU): its kernel transform against adaptive
quadrature, single points against their exact phasors, and the cube against the exact
sum of Eq. 2, with the error falling by about a decade per cell of kernel width."""
import numpy as np
import pytest

import oracle
import oracle.nufft as nu
from paper_2307_09226_gb300 import synth


def test_es_transform_against_adaptive_quadrature():
    integrate = pytest.importorskip("scipy.integrate")
    for w, G in ((7, 512), (6, 256), (8, 64)):
        beta = nu.es_beta(w)
        for k in (0, 3, G // 4 - 1, G // 4):
            f = lambda t: np.exp(beta * (np.sqrt(max(0.0, 1 - (2 * t / w) ** 2)) - 1)) * np.cos(2 * np.pi * k * t / G)
            want = integrate.quad(f, -w / 2, w / 2, limit=200, epsabs=1e-14, epsrel=1e-13)[0]
            got = nu.es_transform([k], w, G)[0]
            assert abs(got - want) <= 1e-11 * abs(want)


@pytest.mark.parametrize("Ns,L", [(32, 16), (33, 17), (64, 8)])
def test_single_point_is_its_phasor(Ns, L):
    rng = np.random.default_rng(Ns * 100 + L)
    n = np.arange(Ns)[:, None]
    l = np.arange(L)[None, :]
    errs = []
    for w in (5, 6, 7, 8):
        e = 0.0
        for _ in range(4):
            x, y = rng.random(), rng.random()
            q = np.exp(2j * np.pi * rng.random())
            f = nu.nufft2_type1([x], [y], [q], Ns, L, w)
            e = max(e, np.abs(f - q * np.exp(2j * np.pi * (x * n + y * l))).max())
        errs.append(e)
        assert e <= 10.0 * 10.0 ** (-(w - 1))  # max error; the relative L2 error is ~10^-(w-1)
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_cube_against_exact_sum():
    f = synth.config1()
    ref = oracle.cube_separable(f.radar, f.pixels)
    errs = [oracle.rel_l2(nu.cube_nufft(f.radar, f.pixels, w=w), ref) for w in (5, 6, 7, 8)]
    assert errs[2] <= 5e-6  # width 7: ~1e-6
    assert all(b < 0.3 * a for a, b in zip(errs, errs[1:]))


def test_ragged_frame_and_tdm_term():
    f = synth.parity_frame(seed=31, M=2, N=3, Ns=24, L=12, n_az=9, n_el=7, dtype=np.float64)
    r = synth.Radar(M=2, N=3, Ns=24, L=12, tdm_motion=True)
    ref = oracle.cube_separable(r, f.pixels)
    assert oracle.rel_l2(nu.cube_nufft(r, f.pixels, w=7), ref) <= 5e-6


def test_empty_frame_is_zero():
    f = synth.config1()
    px = f.pixels.astype(np.float64)
    px.sigma_re[:] = 0.0
    px.sigma_im[:] = 0.0
    assert np.all(nu.cube_nufft(f.radar, px, w=7) == 0)


def test_grid_size_is_the_oversampled_power_of_two():
    """G = the smallest power of two >= 2 N, and at least 16 cells."""
    assert [nu.grid_size(n) for n in (4, 7, 8, 9, 64, 65, 128, 129, 2048)] == \
        [16, 16, 16, 32, 128, 256, 256, 512, 4096]


@pytest.mark.parametrize("beta", [2.3, 9.0, 14.4])
def test_es_kernel_special_values(beta):
    """The exponential-of-semicircle kernel at points where it has a closed form: 1 at the
    centre, e^-beta at the support's edge, e^(-beta/2) where sqrt(1 - z^2) = 1/2, zero
    outside [-1, 1]; it is even and falls monotonically from the centre to the edge."""
    z = np.array([0.0, 1.0, -1.0, np.sqrt(3.0) / 2.0, -np.sqrt(3.0) / 2.0, 0.6])
    want = np.exp(-beta * np.array([0.0, 1.0, 1.0, 0.5, 0.5, 0.2]))
    np.testing.assert_allclose(nu.es_kernel(z, beta), want, rtol=1e-14)
    assert np.all(nu.es_kernel(np.array([1.0 + 1e-12, -1.5, 7.0]), beta) == 0.0)
    t = np.linspace(0.0, 1.0, 101)
    f = nu.es_kernel(t, beta)
    np.testing.assert_array_equal(f, nu.es_kernel(-t, beta))
    assert np.all(np.diff(f) < 0)
