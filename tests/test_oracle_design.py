"""Pins of the oracle's operator design (Sec. II design trade-off, Sec. III table)."""
import math

import numpy as np
import pytest

DX, DZ = 12.5, 5.0


def _passband(k, kx, theta=65.0):
    return kx <= k * math.sin(math.radians(theta))


def test_zero_step_gives_identity(oracle_mod):
    # dz = 0: the target is 1 at every kx, so the exact fit is the delta filter.
    h = oracle_mod.design_operators(32, 0.4, DX, 0.0, 12)
    assert np.max(np.abs(h[:, 0] - 1.0)) < 1e-12
    assert np.max(np.abs(h[:, 1:])) < 1e-12


def test_weighted_normal_equations_hold(oracle_mod):
    # The unguarded taps minimise ||sqrt(W)(A h - D)||: A^T W (A h - D) = 0.
    _, info = oracle_mod.design_operators(64, 0.5, DX, DZ, 12, return_info=True)
    A, W, D, h = info["A"], info["W"], info["D"], info["h_ls"]
    r = (h @ A.T) - D                                   # [nk][M]
    g = np.einsum("ml,km->kl", A, W * r)
    scale = np.einsum("ml,km->kl", np.abs(A), W * np.abs(D))
    assert np.max(np.abs(g) / scale) < 1e-10


def test_guard_bounds_amplitude(oracle_mod):
    h, info = oracle_mod.design_operators(256, 0.5, DX, DZ, 12, return_info=True)
    H = oracle_mod.response(h, info["kx_guard"], DX)
    assert np.max(np.abs(H)) <= 1.0 + 1e-12
    fine = np.linspace(0, math.pi / DX, 40961)
    assert np.max(np.abs(oracle_mod.response(h, fine, DX))) <= 1.0 + 1e-4
    # the guard only rescales: the shape of the response is unchanged
    assert np.allclose(h, info["h_ls"] * info["scale"][:, None], rtol=0, atol=1e-15)


def test_passband_phase_accuracy(oracle_mod):
    # Inside 45 degrees the 25-tap design tracks exp(+i kz dz) closely; a wrong
    # sign of dz or of the phase, or a wrong basis, fails here.  Above k = pi/dx
    # (spatially aliased wavenumbers, where the whole [0, pi/dx] is passband) the
    # fit is looser.
    nk, kmax = 128, 2 * math.pi * 60 / 750
    h, info = oracle_mod.design_operators(nk, kmax, DX, DZ, 12, return_info=True)
    kx = np.linspace(0, math.pi / DX, 2001)
    worst = {True: 0.0, False: 0.0}
    for j in range(1, nk):
        k = info["k"][j]
        m = kx <= k * math.sin(math.radians(45))
        D = np.exp(1j * np.sqrt(k * k - kx[m] ** 2) * DZ)
        e = np.max(np.abs(oracle_mod.response(h[j], kx[m], DX) - D))
        worst[k <= math.pi / DX] = max(worst[k <= math.pi / DX], e)
    assert worst[True] < 1e-2
    assert worst[False] < 3e-2


@pytest.mark.parametrize("k", [0.1, 0.25, 0.4])
def test_misfit_decreases_with_length(oracle_mod, k):
    # Longer filters span a larger (nested) cosine basis on the same samples, so
    # the weighted least-squares misfit must drop (Sec. II: long filters reach
    # higher angles).  L <= 15 keeps M = 256 samples for every length.
    errs = []
    for L in (4, 8, 12, 15):
        # a 2-entry table whose last entry is exactly k
        _, info = oracle_mod.design_operators(2, k, DX, DZ, L, return_info=True)
        r = info["h_ls"][1] @ info["A"].T - info["D"][1]
        errs.append(float(np.sum(info["W"][1] * np.abs(r) ** 2)))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs


def test_normal_equations_agree_with_qr(oracle_mod):
    # An independent solve of the same weighted problem (Cholesky of A^T W A).
    _, info = oracle_mod.design_operators(48, 0.45, DX, DZ, 17, return_info=True)
    A, W, D = info["A"], info["W"], info["D"]
    for j in range(48):
        G = A.T @ (W[j][:, None] * A)
        c = np.linalg.cholesky(G)
        b = A.T @ (W[j] * D[j])
        y = np.linalg.solve(c, b)
        h = np.linalg.solve(c.T, y)
        assert np.linalg.norm(h - info["h_ls"][j]) <= 1e-10 * np.linalg.norm(h)
