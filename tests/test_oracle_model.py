"""Pins of the oracle's whole depth loop: brute-force dense matrices on tiny
inputs, and the adjoint (modeling) used to synthesise test sections."""
import math

import numpy as np


def _tiny(oracle_mod, rng, nx=14, nz=4, nw=3, L=3, nk=12):
    kmax = 0.6
    table = oracle_mod.design_operators(nk, kmax, 12.5, 5.0, L)
    vel = rng.uniform(700, 2400, (nz, nx)).astype(np.float32)
    q = oracle_mod.q_values(2 * math.pi * np.array([9.0, 27.0, 55.0])[:nw], kmax / (nk - 1))
    P0 = rng.standard_normal((nw, nx)) + 1j * rng.standard_normal((nw, nx))
    return table, vel, q, P0


def _dense_step(oracle_mod, table, vrow, qj, nx):
    """Explicit nx x nx matrix of one step: row i holds the taps of output point i."""
    nk, L1 = table.shape
    s = oracle_mod.slowness(vrow)
    Wm = np.zeros((nx, nx), complex)
    for i in range(nx):
        h = table[int(oracle_mod.lookup_index(qj, s[i], nk))]
        for m in range(nx):
            if abs(i - m) < L1:
                Wm[i, m] = h[abs(i - m)]
    return Wm


def test_depth_loop_equals_dense_matrix_chain(oracle_mod):
    rng = np.random.default_rng(21)
    table, vel, q, P0 = _tiny(oracle_mod, rng)
    nz, nx = vel.shape
    P, img = oracle_mod.migrate(P0, vel, table, q)
    ref_img = np.zeros((nz, nx))
    ref_P = P0.copy()
    for z in range(nz):
        ref_img[z] = np.sum(ref_P.real, axis=0)
        ref_P = np.stack([_dense_step(oracle_mod, table, vel[z], q[j], nx) @ ref_P[j]
                          for j in range(len(q))])
    assert np.max(np.abs(P - ref_P)) <= 1e-14 * np.max(np.abs(ref_P)) * nz * 10
    assert np.max(np.abs(img - ref_img)) <= 1e-14 * np.max(np.abs(ref_img)) * nz * 10


def test_adjoint_step_dot_product(oracle_mod):
    rng = np.random.default_rng(22)
    table, vel, q, P = _tiny(oracle_mod, rng, nx=50, L=6)
    Q = rng.standard_normal(P.shape) + 1j * rng.standard_normal(P.shape)
    lhs = np.vdot(Q, oracle_mod.step(P, vel[0], table, q))
    rhs = np.vdot(oracle_mod.adjoint_step(Q, vel[0], table, q), P)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_model_is_adjoint_of_migrate(oracle_mod):
    # <migrate(P0), r> (real image inner product) = Re <model(r), P0>.
    rng = np.random.default_rng(23)
    table, vel, q, P0 = _tiny(oracle_mod, rng, nx=40, nz=9, L=5)
    r = rng.standard_normal(vel.shape)
    _, img = oracle_mod.migrate(P0, vel, table, q)
    lhs = float(np.sum(img * r))
    rhs = float(np.real(np.vdot(oracle_mod.model(r, vel, table, q), P0)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
