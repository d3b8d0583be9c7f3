"""Pins of the 3-D oracle (oracle/fx3d.py): the 2-D operator design, the 2-D
convolution of one depth step and the imaging, against the exact phase shift,
brute force, closed forms and exploding-reflector geometry."""
import math

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def F(oracle_mod):
    import oracle.fx3d as fx3d
    return fx3d


def test_orbits_cover_the_stencil_once(F):
    # every offset of the (2L+1)^2 stencil belongs to exactly one orbit, and
    # the orbit of (a, b) is closed under sign changes and the swap
    for L in (0, 1, 4, 6):
        seen = {}
        orb = F.orbits(L)
        assert len(orb) == (L + 1) * (L + 2) // 2
        for p, ((a, b), pts) in enumerate(orb):
            assert a >= b >= 0
            for i, j in pts:
                assert (i, j) not in seen
                seen[(i, j)] = p
                assert max(abs(i), abs(j)) == a and min(abs(i), abs(j)) == b
        assert len(seen) == (2 * L + 1) ** 2


def test_zero_step_gives_identity(F):
    # dz = 0: the target is 1 everywhere, which the (0, 0) tap alone meets
    h = F.design2d_at([0.0, 0.05, 0.2], 20.0, 0.0, 6)
    for row in h:
        assert abs(row[0] - 1.0) < 1e-12
        assert np.max(np.abs(row[1:])) < 1e-12


def test_normal_equations_hold(F):
    # the unguarded solution satisfies B^T W (B h - D) = 0 for Re and Im
    dx, dz, L, k = 20.0, 10.0, 6, 0.1
    h, info = F.design2d_at([k], dx, dz, L, return_info=True)
    h = h[0] * max(1.0, info["guard"][0])
    M = info["samples"]
    g = np.arange(M) * (math.pi / (dx * (M - 1)))
    ii, jj = np.tril_indices(M)
    kx, ky = g[ii], g[jj]
    kr = np.hypot(kx, ky)
    B = F._basis(kx, ky, dx, L)
    w = np.where(kr <= k * math.sin(math.radians(65.0)), 1.0, 1e-2)
    D = np.where(kr <= k, np.exp(1j * np.sqrt(np.maximum(k * k - kr * kr, 0)) * dz),
                 np.exp(-np.sqrt(np.maximum(kr * kr - k * k, 0)) * dz))
    for part, target in ((h.real, D.real), (h.imag, D.imag)):
        g_res = B.T @ (w * (B @ part - target))
        assert np.max(np.abs(g_res)) < 1e-9 * np.max(np.abs(B.T @ (w * target)))


@pytest.mark.parametrize("f", [10.0, 20.0])
def test_phase_shift_accuracy_in_all_directions(F, f):
    # inside the design dip the response matches exp(i sqrt(k^2 - kr^2) dz)
    # along the axis, the diagonal and in between (a basis missing the swap
    # symmetry, or a sign error in kz, fails the diagonal or the phase)
    dx, dz, L, v = 20.0, 10.0, 6, 1000.0
    k = 2 * math.pi * f / v
    h = F.design2d_at([k], dx, dz, L)[0]
    kr = np.linspace(0.0, 0.9 * k * math.sin(math.radians(65.0)), 40)
    for deg in (0.0, 22.5, 45.0, 67.5, 90.0):
        th = math.radians(deg)
        H = F.response2d(h, kr * math.cos(th), kr * math.sin(th), dx)
        D = np.exp(1j * np.sqrt(k * k - kr * kr) * dz)
        assert np.max(np.abs(np.angle(H / D))) < 2e-2, deg
        assert np.max(np.abs(np.abs(H) - 1.0)) < 4e-2, deg


def test_amplitude_guard(F):
    # |H| <= 1 over the whole square of wavenumbers, so the recursion cannot grow
    dx, dz, L = 20.0, 10.0, 6
    table = F.design2d_operators(64, 0.25, dx, dz, L)
    g = np.linspace(0.0, math.pi / dx, 151)
    KX, KY = np.meshgrid(g, g)
    for row in table[::7]:
        assert np.max(np.abs(F.response2d(row, KX, KY, dx))) <= 1.0 + 1e-3


def test_step_equals_brute_force_convolution(F, oracle_mod):
    # the orbit sums of step3d against a direct double loop over the expanded
    # stencil, with a different operator at every point
    rng = np.random.default_rng(4)
    L, ny, nx, nk = 2, 7, 9, 16
    nu = (L + 1) * (L + 2) // 2
    table = rng.normal(size=(nk, nu)) + 1j * rng.normal(size=(nk, nu))
    P = rng.normal(size=(2, ny, nx)) + 1j * rng.normal(size=(2, ny, nx))
    vplane = rng.uniform(1000.0, 3000.0, (ny, nx)).astype(np.float32)
    q = np.array([4000.0, 9000.0], np.float32)
    out = F.step3d(P, vplane, table, q)
    s = oracle_mod.slowness(vplane)
    for w in range(2):
        for y in range(ny):
            for x in range(nx):
                st = F.expand_stencil(table[int(oracle_mod.lookup_index(q[w], s[y, x], nk))])
                acc = 0j
                for i in range(-L, L + 1):
                    for j in range(-L, L + 1):
                        if 0 <= x + i < nx and 0 <= y + j < ny:
                            acc += st[i + L, j + L] * P[w, y + j, x + i]
                assert abs(out[w, y, x] - acc) < 1e-12


def test_plane_wave_eigenfunction(F, oracle_mod):
    # away from the edges exp(i (kx x + ky y)) is multiplied by H(kx, ky)
    dx, L, n = 20.0, 6, 48
    table = F.design2d_operators(32, 0.2, dx, 10.0, L)
    vplane = np.full((n, n), 1500.0, np.float32)
    _, dk = oracle_mod.k_grid(32, 0.2)
    q = oracle_mod.q_values(np.array([2 * math.pi * 20.0]), dk)
    kx, ky = 0.03, -0.05
    xs = np.arange(n) * dx
    P = np.exp(1j * (kx * xs[None, :] + ky * xs[:, None]))[None]
    out = F.step3d(P, vplane, table, q)
    idx = int(oracle_mod.lookup_index(q[0], oracle_mod.slowness(vplane[:1, :1])[0, 0], 32))
    H = F.response2d(table[idx], np.array([kx]), np.array([ky]), dx)[0]
    inner = (slice(L, n - L), slice(L, n - L))
    assert np.max(np.abs(out[0][inner] - H * P[0][inner])) < 1e-12


def _migrate3d(oracle_mod, F, w, section, vm):
    P0 = oracle_mod.band_dft(section.reshape(w.ny * w.nx, w.nt), w.i0, w.nw).reshape(w.nw, w.ny, w.nx)
    om = oracle_mod.omegas(w.i0, w.nw, w.nt, w.dt)
    kmax = om[-1] / vm
    table = F.design2d_operators(w.nk, kmax, w.dx, w.dz, w.L, w.theta_deg)
    _, dk = oracle_mod.k_grid(w.nk, kmax)
    q = oracle_mod.q_values(om, dk)
    vel = np.full((w.nz, w.ny, w.nx), vm, np.float32)
    return F.migrate3d(P0, vel, table, q)[1]


def test_point_diffractor_collapses_to_its_position(F, oracle_mod):
    # a diffractor at (400 m, 400 m, 200 m) in 2000 m/s, migrated with the
    # exploding-reflector velocity 1000 m/s, focuses at its grid point
    w = W.DIFFRACTOR_3D
    img = _migrate3d(oracle_mod, F, w, W.diffractor_section_3d(w, 400.0, 400.0, 200.0, 2000.0), 1000.0)
    iz, iy, ix = np.unravel_index(np.argmax(np.abs(img)), img.shape)
    assert abs(ix - 20) <= 1 and abs(iy - 20) <= 1 and abs(iz - 20) <= 1, (ix, iy, iz)
    assert img[iz, iy, ix] > 0
    e = img ** 2
    near = e[max(0, iz - 6):iz + 7, max(0, iy - 6):iy + 7, max(0, ix - 6):ix + 7].sum()
    assert near > 0.5 * e.sum()


def test_spike_migrates_to_hemisphere(F, oracle_mod):
    # a spike at (x0, y0, t0) migrates to a hemisphere of radius v_m t0: along
    # rays within 45 degrees of vertical, in several azimuths, the envelope
    # peaks within 2 samples of the sphere
    w = W.DIFFRACTOR_3D
    ix0, iy0, it0, vm = 20, 20, 60, 1000.0       # t0 = 0.24 s -> radius 240 m
    img = _migrate3d(oracle_mod, F, w, W.spike_section_3d(w, ix0, iy0, it0), vm)
    from scipy.signal import hilbert
    env = np.abs(hilbert(img, axis=0))
    r0 = vm * it0 * w.dt
    for az in (0.0, 30.0, 45.0, 90.0, 135.0):
        for dip in (0.0, 20.0, 40.0):
            th, ph = math.radians(dip), math.radians(az)
            radii = np.arange(120.0, 340.0, 2.0)
            xs = ix0 + radii * math.sin(th) * math.cos(ph) / w.dx
            ys = iy0 + radii * math.sin(th) * math.sin(ph) / w.dx
            zs = radii * math.cos(th) / w.dz
            ok = (xs >= 0) & (xs <= w.nx - 1) & (ys >= 0) & (ys <= w.ny - 1) & (zs <= w.nz - 1)
            vals = env[np.rint(zs[ok]).astype(int), np.rint(ys[ok]).astype(int), np.rint(xs[ok]).astype(int)]
            r_peak = radii[ok][np.argmax(vals)]
            assert abs(r_peak - r0) <= 2 * max(w.dx, w.dz), (az, dip, r_peak)
