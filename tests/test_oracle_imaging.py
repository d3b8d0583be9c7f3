"""Pins of the oracle's imaging (Algorithm 1 depth rows summed over frequency)
against exploding-reflector geometry with a known answer."""
import math

import numpy as np
import pytest

import workloads as W


def _migrate_section(oracle_mod, w, d, vm):
    P0 = oracle_mod.band_dft(d, w.i0, w.nw)
    om = oracle_mod.omegas(w.i0, w.nw, w.nt, w.dt)
    kmax = om[-1] / vm
    table = oracle_mod.design_operators(w.nk, kmax, w.dx, w.dz, w.L, w.theta_deg)
    _, dk = oracle_mod.k_grid(w.nk, kmax)
    q = oracle_mod.q_values(om, dk)
    vel = np.full((w.nz, w.nx), vm, np.float32)
    return oracle_mod.migrate(P0, vel, table, q)[1]


def test_point_diffractor_collapses_to_its_position(oracle_mod):
    # Diffractor at x = 640 m, z = 300 m, medium velocity 2000 m/s, migrated
    # with the exploding-reflector velocity 1000 m/s: the focus is trace 64,
    # depth row 60 (z = 60 dz), within one sample.
    w = W.DIFFRACTOR_128
    img = _migrate_section(oracle_mod, w, W.diffractor_section(w), 1000.0)
    iz, ix = np.unravel_index(np.argmax(np.abs(img)), img.shape)
    assert abs(ix - 64) <= 1 and abs(iz - 60) <= 1, (ix, iz)
    assert img[iz, ix] > 0          # zero-phase Ricker: positive peak
    # the collapsed hyperbola is compact: little energy far from the focus
    e = img ** 2
    near = e[max(0, iz - 12):iz + 13, max(0, ix - 12):ix + 13].sum()
    assert near > 0.6 * e.sum()


def test_spike_migrates_to_semicircle(oracle_mod):
    # A spike at (x0, t0) is the impulse response of zero-offset migration:
    # a semicircle of radius v_m t0 centred at (x0, 0).  Along rays within
    # +-60 degrees the envelope peak lies within 2 samples of the circle.
    w = W.DIFFRACTOR_128
    x0, it0, vm = 64, 75, 1000.0          # t0 = 0.3 s -> radius 300 m
    img = _migrate_section(oracle_mod, w, W.spike_section(w, x0, it0), vm)
    r0 = vm * it0 * w.dt
    from scipy.signal import hilbert
    env = np.abs(hilbert(img, axis=0))
    for deg in range(-60, 61, 10):
        th = math.radians(deg)
        radii = np.arange(100.0, 480.0, 1.0)
        xs = x0 + radii * math.sin(th) / w.dx
        zs = radii * math.cos(th) / w.dz
        ok = (xs >= 0) & (xs <= w.nx - 1) & (zs <= w.nz - 1)
        xi = np.rint(xs[ok]).astype(int)
        zi = np.rint(zs[ok]).astype(int)
        vals = env[zi, xi]
        r_peak = radii[ok][np.argmax(vals)]
        assert abs(r_peak - r0) <= 2 * max(w.dx, w.dz), (deg, r_peak)
