"""Pins of the oracle's t -> f transform (Algorithm 1, time-to-frequency step)."""
import math

import numpy as np


def test_sine_on_bin_closed_form(oracle_mod):
    # DFT of sin(2 pi j0 t / nt) with the e^{-i w t} sign: -i nt/2 at j0, 0 at the other bins.
    nt, j0 = 256, 17
    t = np.arange(nt)
    d = np.sin(2 * math.pi * j0 * t / nt)[None, :]
    X = oracle_mod.band_dft(d, 5, 40)[:, 0]
    expect = np.zeros(40, complex)
    expect[j0 - 5] = -0.5j * nt
    assert np.max(np.abs(X - expect)) < 1e-10


def test_cosine_on_bin_closed_form(oracle_mod):
    nt, j0 = 2000, 131
    t = np.arange(nt)
    d = np.cos(2 * math.pi * j0 * t / nt)[None, :]
    X = oracle_mod.band_dft(d, 20, 221)[:, 0]
    expect = np.zeros(221, complex)
    expect[j0 - 20] = nt / 2
    assert np.max(np.abs(X - expect)) < 1e-9


def test_matches_numpy_fft(oracle_mod):
    rng = np.random.default_rng(1)
    for nt in (256, 2000, 4000):
        d = rng.standard_normal((7, nt))
        X = oracle_mod.band_dft(d, 3, nt // 2 - 3)
        ref = np.fft.rfft(d, axis=1)[:, 3:nt // 2].T
        assert np.linalg.norm(X - ref) / np.linalg.norm(ref) < 1e-12


def test_parseval_full_spectrum(oracle_mod):
    rng = np.random.default_rng(2)
    nt = 256
    d = rng.standard_normal((3, nt))
    X = oracle_mod.band_dft(d, 0, nt // 2 + 1)     # bins 0..nt/2
    e = np.abs(X[0]) ** 2 + np.abs(X[-1]) ** 2 + 2 * np.sum(np.abs(X[1:-1]) ** 2, axis=0)
    assert np.allclose(e / nt, np.sum(d * d, axis=1), rtol=1e-12)


def test_band_to_time_inverts_band_dft(oracle_mod):
    rng = np.random.default_rng(3)
    nt, i0, nw = 2000, 20, 221
    P = rng.standard_normal((nw, 5)) + 1j * rng.standard_normal((nw, 5))
    d = oracle_mod.band_to_time(P, i0, nt)
    assert np.linalg.norm(oracle_mod.band_dft(d, i0, nw) - P) / np.linalg.norm(P) < 1e-12


def test_ricker_spectrum_matches_dft_of_samples(oracle_mod):
    # zero-phase Ricker samples: their DFT is dt-spaced samples of the
    # continuous spectrum divided by dt (aliasing is negligible at 1 ms)
    import workloads as W
    dt, nt, fp = 0.001, 4096, 25.0
    t = (np.arange(nt) - nt // 2) * dt
    r = W.ricker(t, fp)
    dft = np.fft.rfft(np.fft.ifftshift(r))
    f = np.fft.rfftfreq(nt, dt)
    S = oracle_mod.ricker_spectrum(f, fp, dt)
    assert np.max(np.abs(dft.imag)) <= 1e-9 * np.max(np.abs(dft))
    assert np.max(np.abs(dft.real - S)) <= 1e-9 * np.max(S)
    # the amplitude spectrum peaks at the peak frequency
    fine = np.linspace(1.0, 100.0, 99001)
    assert abs(fine[np.argmax(oracle_mod.ricker_spectrum(fine, fp))] - fp) < 1e-3
