"""Shared helpers of the GPU parity tests: build seeded inputs, run the oracle
and the library on the same values, measure relative L2 errors."""
import math

import numpy as np

import oracle as O
import workloads as W

# Tolerances (FP32 GPU vs FP64 oracle on identical inputs).  Each step of
# Eq. 1 sums 2L+1 fp32 products (relative rounding ~1e-7 per step); over a few
# hundred steps the errors add like a random walk, a few 1e-6 on the
# wavefield.  The bars are the ones the method is held to.
TOL_SLICE = 1e-5      # wavefield P(., z_k, .) over all x and frequencies
TOL_IMAGE = 1e-4      # final image
TOL_T2F = 2e-6        # fp32 FFT against the FP64 DFT
TOL_DESIGN64 = 1e-10  # FP64 taps, Cholesky (GPU) vs QR (oracle)


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def small_layered(nx=700, nz=120, nt=512, dt=0.004, L=12, seed=5, name="layered_700"):
    return W.Workload(name, nx=nx, dx=12.5, nt=nt, dt=dt, nz=nz, dz=5.0, f_lo=5.0, f_hi=60.0, L=L, seed=seed)


def problem(w, v_medium, section):
    """Oracle-side inputs of a workload: migration velocity (v/2), table, q, P0."""
    vm = (0.5 * np.asarray(v_medium)).astype(np.float32)
    om = O.omegas(w.i0, w.nw, w.nt, w.dt)
    k_max = float(om[-1] / float(vm.min()))
    table = O.design_operators(w.nk, k_max, w.dx, w.dz, w.L, w.theta_deg)
    _, dk = O.k_grid(w.nk, k_max)
    q = O.q_values(om, dk)
    P0 = O.band_dft(section, w.i0, w.nw)
    return dict(vm=vm, k_max=k_max, table=table, q=q, P0=P0)


def desc_of(fx, w, k_max):
    return fx.Desc(nx=w.nx, nz=w.nz, nt=w.nt, nw=w.nw, i0=w.i0, L=w.L, nk=w.nk, dx=w.dx, dz=w.dz,
                   dt=w.dt, theta_max_deg=w.theta_deg, k_max=k_max)


def layered_inputs(w):
    v, refl = W.layered_lens_model(w)
    d = W.normal_incidence_section(w, v, refl)
    return v, refl, d
