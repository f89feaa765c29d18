"""Pins of the CPU FP64 oracle against facts that do not come from the oracle itself.

Each test states the fact it relies on.  The facts are textbook FMCW/MIMO results
(range, Doppler and angle FFT bins of a point target; Dirichlet-kernel leakage at
off-grid frequencies), aliasing periods, linearity and superposition of a sum, and
brute force on tiny inputs.  Together they fail on a dropped term, a wrong sign, a
wrong factor of two, a swapped channel index or a transposed (n, l) axis.
"""
import cmath
import math

import numpy as np
import pytest

import oracle
from paper_2307_09226_gb300 import synth
from paper_2307_09226_gb300.synth import Radar, Pixels, point_scatterer

RADAR = Radar(M=2, N=4, Ns=64, L=32)  # Ns != L so that a transposed axis shows


def _one(radar, R, sigma, az, el, vel):
    return point_scatterer(radar, R, sigma, az, el, vel)


def _both(radar, px):
    a = oracle.cube_literal(radar, px)
    b = oracle.cube_separable(radar, px)
    assert oracle.rel_l2(b, a) < 1e-12
    return a


def test_range_fft_peak_lands_on_fmcw_bin():
    """Beat frequency 2 mu R / c puts a target at range bin k = 2 mu R N_s / (c F_s)."""
    r = RADAR.resolved()
    k_r = 11
    R = k_r * r.c * r.fs / (2.0 * r.mu * r.Ns)  # textbook FMCW range of bin k_r
    sig = 0.7 - 1.3j
    cube = _both(RADAR, _one(RADAR, R, sig, 0.0, 0.0, 0.0))
    for v in range(r.V):
        spec = np.fft.fft(cube[v, :, 0])
        assert int(np.argmax(np.abs(spec))) == k_r
        assert abs(abs(spec[k_r]) - abs(sig) * r.Ns) < 1e-9
        leak = np.delete(np.abs(spec), k_r)
        assert leak.max() < 1e-9 * abs(sig) * r.Ns
    # range estimate from the bin, the textbook inverse
    assert abs(k_r * r.c * r.fs / (2 * r.mu * r.Ns) - R) < 1e-12


def test_doppler_fft_peak_and_sign():
    """A target closing in (v > 0 read as range rate of the Doppler 2 v / lam) turns
    by -f_D T_slow per TDM block, so a forward FFT over l peaks at (-f_D T_slow L) mod L,
    and |bin| = f_D L M T_b with T_slow = M T_b."""
    r = RADAR.resolved()
    k_d = 5
    vel = k_d * r.lam / (2.0 * r.t_slow * r.L)  # f_D T_slow L = k_d
    cube = _both(RADAR, _one(RADAR, 2.0, 1.0 + 0j, 0.0, 0.0, vel))
    spec = np.fft.fft(cube[0, 0, :])
    assert int(np.argmax(np.abs(spec))) == (-k_d) % r.L
    assert abs(abs(spec[(-k_d) % r.L]) - r.L) < 1e-9
    assert np.delete(np.abs(spec), (-k_d) % r.L).max() < 1e-9 * r.L
    assert abs(2 * vel / r.lam * r.L * r.M * r.t_b - k_d) < 1e-9
    # opposite velocity: the mirrored bin
    cube2 = _both(RADAR, _one(RADAR, 2.0, 1.0 + 0j, 0.0, 0.0, -vel))
    assert int(np.argmax(np.abs(np.fft.fft(cube2[0, 0, :])))) == k_d


@pytest.mark.parametrize("k_a", [1, 2, 3])
def test_angle_fft_peak_is_steering_bin(k_a):
    """With lam/2 spacing the virtual array of M N elements sees e^{j pi v sin(theta)};
    the FFT over v peaks at k with k / V = sin(theta) / 2.  The channel order v = m N + r
    with Tx spacing N d_rx makes the array uniform, so the peak is clean."""
    r = RADAR.resolved()
    V = r.V
    u = 2.0 * k_a / V
    cube = _both(RADAR, _one(RADAR, 3.0, 2.0 + 0.5j, math.asin(u), 0.0, 0.0))
    x = cube[:, 0, 0]
    np.testing.assert_allclose(np.abs(x), abs(2.0 + 0.5j), rtol=1e-12)
    spec = np.fft.fft(x)
    assert int(np.argmax(np.abs(spec))) == k_a
    assert np.delete(np.abs(spec), k_a).max() < 1e-9 * V


def test_elevation_shrinks_the_direction_cosine():
    """Only cos(el) sin(az) matters: (az, el) and (asin(cos(el) sin(az)), 0) agree."""
    az, el = 0.4, 0.3
    px1 = _one(RADAR, 2.5, 1 + 1j, az, el, 0.7)
    px2 = _one(RADAR, 2.5, 1 + 1j, math.asin(math.cos(el) * math.sin(az)), 0.0, 0.7)
    assert oracle.rel_l2(oracle.cube_literal(RADAR, px1), oracle.cube_literal(RADAR, px2)) < 1e-12


def test_channel_dependent_range_term_matches_dirichlet_kernel():
    """Off-grid beat frequency: |sum_n e^{j 2 pi a n} e^{-j 2 pi k n / N}| =
    |sin(pi N d) / sin(pi d)| with d = a - k / N.  The per-channel path range
    R_{p,v} = R + v d_rx u / 2 (Eq. 1's R_{m,n}) sets a for each channel; dropping
    it moves channel 7's frequency by ~0.1 bin, far outside the tolerance."""
    radar = Radar(M=2, N=4, Ns=256, L=8)
    r = radar.resolved()
    u = 0.9
    R = 3.1234
    cube = _both(radar, _one(radar, R, 1.0 + 0j, math.asin(u), 0.0, 0.0))
    for v in (0, 3, 7):
        a = 2 * r.mu * (R + v * r.d_rx * u / 2) / (r.c * r.fs)
        spec = np.abs(np.fft.fft(cube[v, :, 0]))
        k = np.arange(r.Ns)
        d = a - k / r.Ns
        d = d - np.round(d)
        dk = np.abs(np.sin(np.pi * r.Ns * d) / np.sin(np.pi * d))
        np.testing.assert_allclose(spec, dk, rtol=1e-9, atol=1e-9)
    # a run without the channel term would be visibly off for v = 7
    a0 = 2 * r.mu * R / (r.c * r.fs)
    d0 = a0 - np.arange(r.Ns) / r.Ns
    d0 = d0 - np.round(d0)
    wrong = np.abs(np.sin(np.pi * r.Ns * d0) / np.sin(np.pi * d0))
    assert np.max(np.abs(np.abs(np.fft.fft(cube[7, :, 0])) - wrong)) > 1.0


def test_range_and_doppler_aliasing_periods():
    """R -> R + c F_s / (2 mu) adds whole cycles per sample; v -> v + lam / (2 T_slow)
    adds whole cycles per block.  Both leave the cube unchanged."""
    r = RADAR.resolved()
    base = dict(R=1.7, sigma=0.3 + 0.9j, az=0.2, el=-0.1, vel=0.8)
    ref = oracle.cube_literal(RADAR, _one(RADAR, **base))
    b1 = dict(base, R=base["R"] + r.c * r.fs / (2 * r.mu))
    b2 = dict(base, vel=base["vel"] + r.lam / (2 * r.t_slow))
    assert oracle.rel_l2(oracle.cube_literal(RADAR, _one(RADAR, **b1)), ref) < 1e-9
    assert oracle.rel_l2(oracle.cube_literal(RADAR, _one(RADAR, **b2)), ref) < 1e-9


def test_velocity_sign_conjugates_slow_time_factor():
    """The slow-time factor of a point target is e^{-j 2 pi f_D T_slow l}; negating v
    conjugates it and leaves the fast-time/channel factor alone."""
    a = oracle.cube_literal(RADAR, _one(RADAR, 2.2, 1.1 - 0.4j, 0.3, 0.1, 1.3))
    b = oracle.cube_literal(RADAR, _one(RADAR, 2.2, 1.1 - 0.4j, 0.3, 0.1, -1.3))
    ra = a / a[:, :, :1]
    rb = b / b[:, :, :1]
    np.testing.assert_allclose(rb, np.conj(ra), rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(a[:, :, 0], b[:, :, 0], rtol=1e-12)


def test_linearity_and_superposition():
    f = synth.parity_frame(seed=5, n_az=9, n_el=7, Ns=16, L=8, mask_frac=0.2, dtype=np.float64)
    full = oracle.cube_literal(f.radar, f.pixels)
    alpha = 0.37 - 2.1j
    px = f.pixels
    s = (px.sigma_re + 1j * px.sigma_im) * alpha
    scaled = Pixels(px.range, s.real.copy(), s.imag.copy(), px.az, px.el, px.vel)
    assert oracle.rel_l2(oracle.cube_literal(f.radar, scaled), alpha * full) < 1e-12
    acc = np.zeros_like(full)
    for p in oracle.valid_indices(px.sigma_re, px.sigma_im):
        acc += oracle.cube_literal(f.radar, px.subset([p]))
    assert oracle.rel_l2(acc, full) < 1e-12


def test_masked_pixels_leave_the_cube_bit_identical():
    """sigma = 0 (either sign of zero) is a background miss whatever its other fields."""
    f = synth.parity_frame(seed=6, n_az=8, n_el=6, Ns=16, L=8, mask_frac=0.0, dtype=np.float64)
    ref = oracle.cube_literal(f.radar, f.pixels)
    px = f.pixels
    junk = Pixels(np.array([np.inf, np.nan, -1.0]), np.array([0.0, -0.0, 0.0]),
                  np.array([-0.0, 0.0, 0.0]), np.array([np.nan, 1e30, 0.1]),
                  np.array([0.2, np.inf, 0.0]), np.array([np.nan, 3.0, -np.inf]))
    cat = Pixels(*(np.concatenate([a[:5], j, a[5:]]) for a, j in zip(px.arrays(), junk.arrays())))
    got = oracle.cube_literal(f.radar, cat)
    assert np.array_equal(got, ref)
    assert oracle.valid_indices(cat.sigma_re, cat.sigma_im).tolist() == \
        [i for i in range(cat.P) if i not in (5, 6, 7)]


def test_brute_force_tiny_against_cmath():
    """P = 3, V = 2, N_s = 4, L = 2, each term written out with cmath."""
    radar = Radar(M=1, N=2, Ns=4, L=2, mu=2e14, t_b=1e-4)
    r = radar.resolved()
    rng = np.random.default_rng(3)
    R = rng.uniform(0.5, 9, 3)
    sr, si = rng.normal(size=3), rng.normal(size=3)
    az, el, vel = rng.uniform(-1, 1, 3), rng.uniform(-0.5, 0.5, 3), rng.uniform(-3, 3, 3)
    px = Pixels(R, sr, si, az, el, vel)
    got = oracle.cube_literal(radar, px)
    for v in range(2):
        for n in range(4):
            for l in range(2):
                z = 0j
                for p in range(3):
                    u = math.cos(el[p]) * math.sin(az[p])
                    Rv = R[p] + v * r.d_rx * u / 2
                    ph = (2 * r.mu * Rv / r.c * n / r.fs + v * r.d_rx * u / r.lam
                          - 2 * vel[p] / r.lam * l * r.t_slow)
                    z += complex(sr[p], si[p]) * cmath.exp(2j * math.pi * ph)
                assert abs(got[v, n, l] - z) < 1e-12 * max(1.0, abs(z))


def test_phase_cycles_matches_the_phase_written_out_term_by_term():
    """phase_cycles against Eq. 1/Eq. 2's phase written out with `math` per pixel, on a
    frame with a masked pixel (the vector runs over valid pixels, ascending) and with the
    TDM motion term; exp(j 2 pi phase) summed over p reproduces the literal cube."""
    from dataclasses import replace
    rng = np.random.default_rng(11)
    R = rng.uniform(0.5, 9, 5)
    sr, si = rng.normal(size=5), rng.normal(size=5)
    sr[2] = si[2] = 0.0  # background miss
    az, el, vel = rng.uniform(-1, 1, 5), rng.uniform(-0.5, 0.5, 5), rng.uniform(-3, 3, 5)
    px = Pixels(R, sr, si, az, el, vel)
    for tdm in (False, True):
        radar = replace(Radar(M=2, N=2, Ns=4, L=3, mu=2e14, t_b=1e-4), tdm_motion=tdm)
        r = radar.resolved()
        cube = oracle.cube_literal(radar, px)
        for v in range(4):
            for n in range(4):
                for l in range(3):
                    got = oracle.phase_cycles(radar, px, v, n, l)
                    want = []
                    for p in (0, 1, 3, 4):
                        u = math.cos(el[p]) * math.sin(az[p])
                        Rv = R[p] + v * r.d_rx * u / 2
                        ph = (2 * r.mu * Rv / r.c * n / r.fs + v * r.d_rx * u / r.lam
                              - 2 * vel[p] / r.lam * l * r.t_slow)
                        if tdm:
                            ph -= 2 * vel[p] / r.lam * (v // 2) * r.t_b
                        want.append(ph)
                    assert got.shape == (4,)
                    np.testing.assert_allclose(got, want, rtol=0, atol=1e-9)
                    z = sum(complex(sr[p], si[p]) * cmath.exp(2j * math.pi * w)
                            for p, w in zip((0, 1, 3, 4), got))
                    assert abs(cube[v, n, l] - z) < 1e-11 * max(1.0, abs(z))


def test_path_terms_are_the_symbols_of_eq1_and_eq2():
    """path_terms against the definitions written out per pixel with `math`: ascending
    valid indices, complex strengths, the direction cosine, the per-channel path range
    and the Doppler shift."""
    rng = np.random.default_rng(17)
    n = 9
    R = rng.uniform(0.5, 9, n)
    sr, si = rng.normal(size=n), rng.normal(size=n)
    sr[[1, 6]] = 0.0
    si[[1, 6]] = 0.0
    si[4] = -0.0
    sr[4] = 0.0   # -0 and +0: a miss
    az, el, vel = rng.uniform(-1, 1, n), rng.uniform(-0.5, 0.5, n), rng.uniform(-3, 3, n)
    radar = Radar(M=2, N=3, Ns=8, L=4)
    r = radar.resolved()
    t = oracle.path_terms(radar, Pixels(R, sr, si, az, el, vel))
    valid = [p for p in range(n) if p not in (1, 4, 6)]
    assert t["idx"].tolist() == valid
    for q, p in enumerate(valid):
        u = math.cos(el[p]) * math.sin(az[p])
        assert t["sigma"][q] == complex(sr[p], si[p])
        assert abs(t["u"][q] - u) < 1e-15
        assert abs(t["fD"][q] - 2 * vel[p] / r.lam) < 1e-9
        for v in range(6):
            assert abs(t["R_pv"][v, q] - (R[p] + v * r.d_rx * u / 2)) < 1e-12


def test_rel_l2_is_the_normwise_relative_error_over_the_whole_cube():
    """The yardstick of every parity claim, against values worked out by hand."""
    assert oracle.rel_l2(np.array([3 + 4j]), np.array([0j])) == 5.0  # zero reference: absolute
    assert oracle.rel_l2(np.array([1 + 1j, 0]), np.array([1, 0])) == 1.0
    x = np.random.default_rng(0).normal(size=(2, 3, 4)) * (1 + 0.5j)
    assert oracle.rel_l2(x, x) == 0.0
    # normwise, not a per-entry mean or maximum: sqrt(0.1^2) / sqrt(1^2 + 10^2)
    got = oracle.rel_l2(np.array([1.1, 10.0]), np.array([1.0, 10.0]))
    assert abs(got - 0.1 / math.sqrt(101.0)) < 1e-15
    assert abs(got - 0.05) > 1e-2 and abs(got - 0.1) > 1e-2
    # complex entries count as two reals: |(1+2j) - (1+1j)| / |1+1j|
    assert abs(oracle.rel_l2(np.array([1 + 2j]), np.array([1 + 1j])) - 1 / math.sqrt(2)) < 1e-15
    assert abs(oracle.rel_l2(np.array([2 + 1j]), np.array([1 + 1j])) - 1 / math.sqrt(2)) < 1e-15
    # the whole array at once, whatever its shape; not relative to the larger argument
    a = np.array([[1.0, 2.0], [2.0, 4.0]], dtype=complex)
    b = np.array([[1.0, 2.0], [2.0, 0.0]], dtype=complex)
    assert abs(oracle.rel_l2(a, b) - 4.0 / 3.0) < 1e-15
    assert abs(oracle.rel_l2(b, a) - 4.0 / 5.0) < 1e-15


def test_literal_and_separable_agree_on_config1():
    f = synth.config1()
    a = oracle.cube_literal(f.radar, f.pixels)
    b = oracle.cube_separable(f.radar, f.pixels)
    assert oracle.rel_l2(b, a) < 1e-12


def test_separable_and_entries_agree_on_a_config2_subsample():
    f = synth.config2()
    idx = np.arange(0, f.pixels.P, 61)
    px = f.pixels.subset(idx)
    b = oracle.cube_separable(f.radar, px, channels=[0, 11])
    rng = np.random.default_rng(0)
    ent = np.stack([rng.choice([0, 11], 20), rng.integers(0, 256, 20), rng.integers(0, 128, 20)], 1)
    e = oracle.cube_entries(f.radar, px, ent)
    pick = b[(ent[:, 0] == 11).astype(int), ent[:, 1], ent[:, 2]]
    np.testing.assert_allclose(e, pick, rtol=1e-11, atol=1e-11 * np.abs(b).max())


def test_empty_frame_gives_zero_cube():
    px = Pixels(*(np.zeros(4) for _ in range(6)))
    assert not oracle.cube_literal(RADAR, px).any()
    assert not oracle.cube_separable(RADAR, px).any()


def test_generator_is_deterministic_and_has_the_stated_mix():
    a, b = synth.config2(), synth.config2()
    for x, y in zip(a.pixels.arrays(), b.pixels.arrays()):
        assert np.array_equal(x, y, equal_nan=True)
    frac = 1.0 - oracle.valid_mask(a.pixels.sigma_re, a.pixels.sigma_im).mean()
    assert abs(frac - 0.30) < 0.01
    fr = synth.walking_batch(n_frames=6)
    for f in fr:
        pv = int(oracle.valid_mask(f.pixels.sigma_re, f.pixels.sigma_im).sum())
        assert 2000 <= pv <= 65536
        assert pv == f.meta["n_ped"] + f.meta["n_wall"]


def test_config1_golden_entries_are_stable():
    """Regression guard: entries stored by tests/golden/make_golden.py (oracle only)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "config1_entries.txt")
    rows = [l.split() for l in open(path) if not l.startswith("#")]
    f = synth.config1()
    ent = np.array([[int(r[0]), int(r[1]), int(r[2])] for r in rows])
    ref = np.array([float(r[3]) + 1j * float(r[4]) for r in rows])
    got = oracle.cube_entries(f.radar, f.pixels, ent)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-10)


def test_tdm_motion_term_turns_tx_slots_by_the_doppler_of_one_chirp():
    """With Tx m transmitting in slot m of each block, a target of Doppler f_D is seen by
    Tx m a time m T_b later than by Tx 0: at u = 0 channel v = m N + r carries the extra
    phase -f_D m T_b (textbook TDM-MIMO velocity-induced phase); Rx channels of the same
    Tx are unaffected, and without the flag every channel agrees."""
    from dataclasses import replace
    radar = Radar(M=3, N=4, Ns=16, L=8)
    r = radar.resolved()
    vel = 1.7
    px = _one(radar, 2.0, 1.0 + 0j, 0.0, 0.0, vel)
    plain = oracle.cube_literal(radar, px)
    tdm = oracle.cube_literal(replace(radar, tdm_motion=True), px)
    fD = 2 * vel / r.lam
    for v in range(r.V):
        m = v // r.N
        np.testing.assert_allclose(tdm[v] / plain[v], np.exp(-2j * np.pi * fD * m * r.t_b),
                                   rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(plain[4], plain[0], rtol=1e-12)
    assert oracle.rel_l2(oracle.cube_separable(replace(radar, tdm_motion=True), px), tdm) < 1e-12


def test_range_doppler_peak_recovers_range_and_velocity():
    """A point target on integer bins: the range-Doppler peak sits at the FMCW range bin
    and the Doppler bin, and the max-power velocity is the target's velocity."""
    radar = Radar(M=2, N=4, Ns=64, L=32)
    r = radar.resolved()
    k_r, k_d = 9, 5
    R = k_r * r.c * r.fs / (2 * r.mu * r.Ns)
    for sign in (1, -1):
        vel = sign * k_d * r.lam / (2 * r.t_slow * r.L)
        cube = oracle.cube_literal(radar, _one(radar, R, 1 + 0j, 0.0, 0.0, vel))
        pw = oracle.range_doppler_power(cube)
        v, (k, d) = oracle.max_power_velocity(radar, pw)
        assert (k, d) == (k_r, (-sign * k_d) % r.L)
        assert abs(v - vel) < 1e-12
        # all the energy of V unit channels is in that bin: V * (N_s L)^2
        assert abs(pw[k, d] - r.V * (r.Ns * r.L) ** 2) < 1e-6 * pw[k, d]
    # a static reflector dominates unless the zero-Doppler column is notched out
    cube = oracle.cube_literal(radar, _one(radar, R, 3 + 0j, 0.0, 0.0, 0.0)) + \
        oracle.cube_literal(radar, _one(radar, R, 1 + 0j, 0.0, 0.0, vel))
    pw = oracle.range_doppler_power(cube)
    assert oracle.max_power_velocity(radar, pw)[1][1] == 0
    assert abs(oracle.max_power_velocity(radar, pw, skip_static=True)[0] - vel) < 1e-12


def test_e_velo_is_the_mean_absolute_error():
    assert oracle.e_velo([1.0, -2.0, 0.5], [1.5, -1.0, 0.5]) == pytest.approx(0.5)


def test_workload_config_files_drive_the_generator():
    """configs/config<n>.json hold the five workloads; the generator follows them."""
    from paper_2307_09226_gb300 import synth
    for n in range(1, 6):
        c = synth.load_config(n)
        assert c["name"] == f"config{n}"
    for n, make in ((1, synth.config1), (2, synth.config2)):
        c = synth.load_config(n)
        f = make()
        assert f.pixels.P == c["grid"]["n_az"] * c["grid"]["n_el"]
        assert (f.radar.M, f.radar.N, f.radar.Ns, f.radar.L) == tuple(c["radar"][k] for k in ("M", "N", "Ns", "L"))
        assert f.pixels.dtype == np.dtype(c["pixel_dtype"]) and f.out_dtype == c["out_dtype"]
        miss = np.mean((f.pixels.sigma_re == 0) & (f.pixels.sigma_im == 0))
        assert abs(miss - c["pixels"]["mask_frac"]) < 0.02
    c4 = synth.load_config(4)
    frames = synth.walking_batch(n_frames=3)
    for f in frames:
        assert c4["pedestrian"]["pixels"][0] <= f.meta["n_ped"] <= c4["pedestrian"]["pixels"][1]
        assert f.meta["n_wall"] <= c4["wall"]["pixels"][1]
    c5 = synth.load_config(5)
    reqs = synth.serving_requests(50)
    for r in reqs:
        assert r["radar"].M in c5["choices"]["M"] and r["radar"].L in c5["choices"]["L"]
        assert r["grid"] in c5["choices"]["grid"] and r["tier"] in c5["choices"]["tier"]
